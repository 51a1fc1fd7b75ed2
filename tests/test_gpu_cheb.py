"""The Chebyshev-node representation (repr = "cheb") through the C-ABI (marked gpu).

Bars:
* FP64 CUDA path vs the oracle's FP64 Chebyshev FMM (same tree, lists, nodes, weights
  and kernel matrices; no pseudo-inverse, so no amplification of rounding): rel-L2
  <= 1e-12, for p = 4 .. 7 on a uniform grid at two pressures and on two adaptive sets;
* FP64 CUDA path vs the direct sum at p = 8 on the 16^3 cube: within 2x of the oracle's
  own interpolation error there (4.4e-8), i.e. <= 1e-7;
* mixed form vs FP64 Chebyshev: rel-L2 <= 1e-6, the mixed form's target (FP32 node-weight
  sums, FP32 M2M / L2L / X-list / W-list / interpolation, FP16x3 tensor-core M2L with FP32
  accumulation, in 256-row blocks where R > 256); the SIMT FP32 M2L within 2e-6 of it;
* full size (the 128^3 benchmark workload and the 3.2M-point refined grid) at p = 8:
  within 1e-6 of the direct sum (the representation's interpolation error is 4e-8 at
  16^3, so 1e-6 leaves room for the mixed form's rounding);
* the plan rejects orders outside 2..10.
"""
import numpy as np
import pytest

from oracle import cheb as CH
from oracle import direct as D
from oracle import kernel as K
from paper_2006_03515_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _relerr(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def _plan(kf, pts, h, leaf, p, a, b, precision="fp64", uniform=True):
    hh = float(h[0]) if uniform else _dev(h)
    return kf.Plan(_dev(pts), hh, leaf, p, a, b, precision=precision, repr="cheb")


def _streamer(pts):
    return W.streamer_source(pts, axis_xy=(0.5, 0.5), z_range=(0.2, 0.7), radius=0.05, head=(0.5, 0.5, 0.7),
                             head_sigma=0.05, noise_sigma=0.3, seed=7)


@pytest.mark.parametrize("p", [4, 5, 6, 7])
@pytest.mark.parametrize("po2", [150.0, 1.52])
def test_fp64_cheb_matches_oracle_uniform(kf, p, po2):
    pts, h, I = W.config_uniform(16)
    a, b = K.absorption_coefficients(po2)
    C = K.source_scale(760.0)
    ref = CH.fmm(pts, h, I, 8, p, a, b, C)
    pl = _plan(kf, pts, h, 8, p, a, b)
    assert pl.info()["surface_points"] == p ** 3
    got = pl.eval(_dev(I), C=C).cpu().numpy()
    pl.close()
    assert _relerr(got, ref) <= 1e-12


@pytest.mark.parametrize("case", ["random_cloud", "adaptive"])
def test_fp64_cheb_matches_oracle_adaptive(kf, case):
    if case == "adaptive":
        pts, h = W.refined_grid(1.0, 16, 4, (0.5, 0.5, 0.7), 2)
        leaf, uniform = 16, False
    else:
        pts, h = W.random_cloud(3000, 11)[:2]
        leaf, uniform = 10, True
    I = _streamer(pts)
    a, b = 5.32, 304.0
    ref = CH.fmm(pts, h, I, leaf, 5, a, b)
    pl = _plan(kf, pts, h, leaf, 5, a, b, uniform=uniform)
    got = pl.eval(_dev(I)).cpu().numpy()
    pl.close()
    assert _relerr(got, ref) <= 1e-12


def test_fp64_cheb_p8_against_direct_sum(kf):
    pts, h, I = W.config_uniform(16)
    a, b = K.absorption_coefficients(150.0)
    ref = D.direct_sum(pts, h, I, a, b)
    pl = _plan(kf, pts, h, 8, 8, a, b)
    got = pl.eval(_dev(I)).cpu().numpy()
    pl.close()
    assert _relerr(got, ref) <= 1e-7


@pytest.mark.parametrize("p", [4, 6, 7])
@pytest.mark.parametrize("po2", [152.0, 1.52])
def test_mixed_cheb_matches_fp64(kf, p, po2):
    pts, h, I = W.config_uniform(32)
    a, b = K.absorption_coefficients(po2)
    Id = _dev(I)
    p64 = _plan(kf, pts, h, 64, p, a, b)
    p32 = _plan(kf, pts, h, 64, p, a, b, precision="mixed")
    s64 = p64.eval(Id).cpu().numpy()
    s32 = p32.eval(Id).cpu().numpy()
    assert p32.info()["m2l_tensor"]
    assert p32.info()["lattice_far"] and not p64.info()["lattice_far"]   # 64-cell leaves on a lattice
    p64.close()
    p32.close()
    assert _relerr(s32, s64) <= 1e-6


def test_mixed_cheb_row_blocks_against_simt(kf, monkeypatch):
    # p = 8: R = 512 coefficients, two 256-row blocks per tile on the tensor cores; the
    # SIMT FP32 M2L and the FP64 form as references
    pts, h, I = W.config_uniform(32)
    a, b = K.absorption_coefficients(152.0)
    Id = _dev(I)
    s64 = _plan(kf, pts, h, 64, 8, a, b).eval(Id).cpu().numpy()
    ptc = _plan(kf, pts, h, 64, 8, a, b, precision="mixed")
    assert ptc.info()["m2l_tensor"]
    stc = ptc.eval(Id).cpu().numpy()
    monkeypatch.setenv("KIFMM_M2L", "simt")
    psimt = _plan(kf, pts, h, 64, 8, a, b, precision="mixed")
    assert not psimt.info()["m2l_tensor"]
    ssimt = psimt.eval(Id).cpu().numpy()
    ptc.close()
    psimt.close()
    assert _relerr(stc, s64) <= 1e-6
    assert _relerr(stc, ssimt) <= 2e-6


def test_mixed_cheb_adaptive_matches_fp64(kf):
    pts, h = W.refined_grid(1.0, 16, 4, (0.5, 0.5, 0.7), 2)
    I = _streamer(pts)
    a, b = 5.32, 304.0
    s64 = _plan(kf, pts, h, 16, 6, a, b, uniform=False).eval(_dev(I)).cpu().numpy()
    s32 = _plan(kf, pts, h, 16, 6, a, b, uniform=False, precision="mixed").eval(_dev(I)).cpu().numpy()
    assert _relerr(s32, s64) <= 1e-6


def test_cheb_order_range(kf):
    pts, h, _ = W.config_uniform(8)
    for p in (1, 11):
        with pytest.raises(kf.KifmmError):
            _plan(kf, pts, h, 8, p, 5.32, 304.0)
    pl = _plan(kf, pts, h, 8, 2, 5.32, 304.0)
    assert pl.info()["surface_points"] == 8
    pl.close()


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def test_full_size_uniform_128_cheb_against_direct_sum(kf):
    # the benchmark's workload (128^3 cell centres, Gaussian source, 760 Torr, p_O2 = 152,
    # leaf 64) with the Chebyshev representation at p = 8: both forms within 1e-6 of the
    # whole direct-sum field (its FFT form, checked against the plain sum at sampled targets)
    import torch
    pts, h, I = W.config_uniform(128)
    a, b = K.absorption_coefficients(152.0)
    C = K.source_scale(760.0)
    Id = _dev(I)
    full = D.fft_uniform(I.reshape(128, 128, 128), h[0], a, b, C).ravel()
    idx = _sample(len(pts), 256, 4)
    np.testing.assert_allclose(full[idx], D.direct_sum(pts, h, I, a, b, C, targets=idx), rtol=1e-10)
    errs = {}
    for prec in ("mixed", "fp64"):
        pl = _plan(kf, pts, h, 64, 8, a, b, precision=prec)
        errs[prec] = _relerr(pl.eval(Id, C=C).cpu().numpy(), full)
        pl.close()
        torch.cuda.empty_cache()
    assert errs["fp64"] <= 1e-6 and errs["mixed"] <= 1e-6, errs


def test_full_size_adaptive_cheb_against_direct_sum(kf):
    # the two-level refined 2 cm grid (3,219,819 points; W and X lists in use), p = 8,
    # mixed form, against the direct sum at sampled coarse and fine targets
    pts, h, I = W.config_adaptive()
    a, b = K.absorption_coefficients(150.0)
    C = K.source_scale(760.0)
    pl = _plan(kf, pts, h, 64, 8, a, b, uniform=False, precision="mixed")
    got = pl.eval(_dev(I), C=C).cpu().numpy()
    pl.close()
    fine = np.nonzero(h < h.max())[0]
    idx = np.concatenate([_sample(len(pts), 128, 2), fine[_sample(len(fine), 128, 3)]])
    ref = D.direct_sum(pts, h, I, a, b, C, targets=idx)
    assert _relerr(got[idx], ref) <= 1e-6
