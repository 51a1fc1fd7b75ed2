"""The comparison models' kernels through the same FMM, against the oracle (marked gpu).

The method is kernel independent (Sec. 3): only kernel evaluations change. The FP64 form
with kernel="helmholtz3" (Sec. 2.2, Eq. (gexp), Table Helcoeff) and kernel="threegroup"
(Sec. 2.3, Eq. (rtetoint), Table threegroupcoeff) is compared point by point with the
oracle KIFMM of the same kernel (same tree, surfaces and cut-off), with the oracle's direct
sum of that kernel, and on rectangular cells; the self term of either self rule is checked
alone on one isolated cell. The mixed form refuses the comparison kernels.
"""
import numpy as np
import pytest

from oracle import direct as D
from oracle import kernel as K
from oracle import kifmm as KF
from paper_2006_03515_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KINDS = ["helmholtz3", "threegroup"]


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _relerr(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mode", ["cell_exact", "paper_gl2"])
def test_kernel_kind_matches_oracle_kifmm(kf, kind, mode):
    pts, h, I = W.config_uniform(24)
    a, b = K.absorption_coefficients(150.0)
    C = K.source_scale(760.0)
    ref = KF.kifmm(pts, h, I, 64, 4, a, b, C, mode=mode, kind=kind)
    p = kf.Plan(_dev(pts), float(h[0]), 64, 4, a, b, precision="fp64", self_mode=mode, kernel=kind)
    got = p.eval(_dev(I), C=C).cpu().numpy()
    p.check()
    p.close()
    assert _relerr(got, ref) <= 1e-10
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= 1e-10


@pytest.mark.parametrize("kind", KINDS)
def test_kernel_kind_against_direct_sum(kf, kind):
    # the FMM of the comparison kernel against that kernel's discrete sum (its own accuracy)
    # a two-level grid (11,971 cells, 4x finer around the head) with the streamer source
    pts, h = W.refined_grid(2.0, 16, 4, (1.0, 1.0, 1.5), 2)
    I = W.streamer_source(pts, seed=5)
    a, b = K.absorption_coefficients(40.0)
    C = K.source_scale(200.0)
    ref = D.direct_sum(pts, h, I, a, b, C, kind=kind)
    p = kf.Plan(_dev(pts), _dev(h), 64, 6, a, b, precision="fp64", kernel=kind)
    got = p.eval(_dev(I), C=C).cpu().numpy()
    p.close()
    err = _relerr(got, ref)
    print("\n%s: FMM (m0 = 6) against the direct sum of the same kernel: %.2e" % (kind, err))
    assert err <= 1e-3   # the oracle KIFMM of the same kernel: 5.8e-4 (helmholtz3), 1.8e-4 (threegroup)


@pytest.mark.parametrize("kind", KINDS)
def test_kernel_kind_rectangular_cells(kf, kind):
    dims = (0.004, 0.004, 0.009)
    g = [(np.arange(n) + 0.5) * d for n, d in zip((16, 16, 12), dims)]
    zz, yy, xx = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    I = W.gaussian(pts, (0.032, 0.032, 0.054), 0.01, 1e22)
    a, b = K.absorption_coefficients(150.0)
    ref = KF.kifmm(pts, None, I, 64, 4, a, b, 1.0, cell_dims=dims, kind=kind)
    p = kf.Plan(_dev(pts), None, 64, 4, a, b, precision="fp64", cell_dims=dims, kernel=kind)
    got = p.eval(_dev(I)).cpu().numpy()
    p.close()
    assert _relerr(got, ref) <= 1e-10


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mode", ["cell_exact", "paper_gl2"])
def test_kernel_kind_self_term(kf, kind, mode):
    # one isolated cell: S = sigma I (C = 1), sigma from the oracle's cell integral
    h = 0.003
    a, b = K.absorption_coefficients(150.0)
    pts = np.array([[0.5 * h, 0.5 * h, 0.5 * h]])
    p = kf.Plan(_dev(pts), h, 64, 4, a, b, precision="fp64", self_mode=mode, kernel=kind)
    got = p.eval(_dev(np.array([1.0]))).cpu().numpy()[0]
    p.close()
    want = K.sigma_cell_any(h, h, h, a, b, kind, mode)
    assert got == pytest.approx(want, rel=1e-10)


@pytest.mark.parametrize("kind", KINDS)
def test_kernel_kind_rejects_mixed(kf, kind):
    pts, h, _ = W.config_uniform(8)
    a, b = K.absorption_coefficients(150.0)
    with pytest.raises(Exception):
        kf.Plan(_dev(pts), float(h[0]), 64, 4, a, b, precision="mixed", kernel=kind)
