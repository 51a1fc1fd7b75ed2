"""Zero-weight padding of box grids to the leaf lattice (kifmm_opts.pad_lattice; marked gpu).

A full grid of n_x x n_y x n_z cubic cells is extended with cells of zero source (I = 0) to
multiples of 2 nc cells per axis (leaf = nc^3), under the root at the grid's corner with side
nc h 2^L. The discrete sum of Eq. (summation) over the caller's cells is unchanged (the added
weights are 0); the FMM follows the padded tree. The reference is therefore the oracle KIFMM
of the padded point set with the same root, read at the caller's points, and every lattice
path of the mixed form engages on grids whose sizes are not multiples of 8.
"""
import numpy as np
import pytest

from oracle import kernel as K
from oracle import kifmm as KF
from paper_2006_03515_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _box(ext, h):
    g = [(np.arange(e) + 0.5) * h for e in ext]
    zz, yy, xx = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


def _padded(ext, h, nc=4):
    """The caller's box grid, then its padding cells (extents rounded up to multiples of
    2 nc), and the root (origin, side)."""
    pad = [-(-e // (2 * nc)) * 2 * nc for e in ext]
    full = _box(pad, h)
    idx = np.rint(full / h - 0.5).astype(np.int64)
    inside = np.all(idx < np.asarray(ext)[None, :], axis=1)
    cells = nc
    while cells < max(pad):
        cells *= 2
    return np.concatenate([_box(ext, h), full[~inside]]), int(np.prod(pad) - np.prod(ext)), cells * h


@pytest.fixture(scope="module")
def case44():
    ext, h = (44, 44, 44), 1.0 / 44
    pts = _box(ext, h)
    I = W.gaussian(pts, (0.5, 0.5, 0.5), 0.1, 1e22)
    a, b = K.absorption_coefficients(152.0)
    C = K.source_scale(760.0)
    pp, nv, side = _padded(ext, h)
    Ip = np.concatenate([I, np.zeros(nv)])
    ref = KF.kifmm(pp, np.full(len(pp), h), Ip, 64, 6, a, b, C, origin=np.zeros(3), side=side)[:len(pts)]
    return pts, h, I, a, b, C, ref, nv


def test_padded_fp64_matches_oracle(kf, case44):
    pts, h, I, a, b, C, ref, nv = case44
    p = kf.Plan(_dev(pts), h, 64, 6, a, b, precision="fp64", pad_lattice=True)
    inf = p.info()
    assert inf["n_padding"] == nv and inf["n_points"] == len(pts) + nv
    got = p.eval(_dev(I), C=C).cpu().numpy()
    p.close()
    assert float(np.linalg.norm(got - ref) / np.linalg.norm(ref)) <= 1e-10
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= 1e-10


def test_padded_mixed_lattice_paths_against_oracle(kf, case44):
    pts, h, I, a, b, C, ref, nv = case44
    plain = kf.Plan(_dev(pts), h, 64, 6, a, b, precision="mixed")
    assert not plain.info()["near_tensor"]   # 44 cells per axis: leaves of mixed levels
    plain.close()
    p = kf.Plan(_dev(pts), h, 64, 6, a, b, precision="mixed", pad_lattice=True)
    inf = p.info()
    assert inf["near_tensor"] and inf["lattice_far"] and inf["m2l_tensor"]
    got = p.eval(_dev(I), C=C).cpu().numpy()
    host = p.eval_host(I, C=C)
    p.check()
    p.close()
    d = np.abs(got - ref)
    m = np.abs(ref).max()
    assert float(np.linalg.norm(got - ref) / np.linalg.norm(ref)) <= 1e-6
    assert float(d.max() / m) <= 1e-6
    sel = np.abs(ref) >= 1e-4 * m
    assert float((d[sel] / np.abs(ref[sel])).max()) <= 1e-4
    assert np.array_equal(host, got)


def test_padded_rectangular_box_and_batch(kf):
    import torch
    ext, h = (36, 44, 28), 1.0 / 48
    pts = _box(ext, h)
    I = W.gaussian(pts, (0.4, 0.45, 0.3), 0.08, 1e22)
    a, b = K.absorption_coefficients(15.2)
    C = K.source_scale(76.0)
    pp, nv, side = _padded(ext, h)
    ref = KF.kifmm(pp, np.full(len(pp), h), np.concatenate([I, np.zeros(nv)]), 64, 6, a, b, C,
                   origin=np.zeros(3), side=side)[:len(pts)]
    st = torch.cuda.Stream()   # (graph capture needs a stream other than the legacy default)
    plans = [kf.Plan(_dev(pts), h, 64, 6, a, b, precision=pr, pad_lattice=True, stream=st)
             for pr in ("fp64", "mixed")]
    assert plans[1].info()["near_tensor"]
    Id = _dev(I)
    outs = [torch.empty_like(Id) for _ in plans]
    torch.cuda.synchronize()
    for _ in range(2):   # recorded, then replayed
        kf.eval_batch(plans, [Id, Id], outs, C=[C, C], capture=True, lanes=2)
    st.synchronize()
    e64 = float(np.linalg.norm(outs[0].cpu().numpy() - ref) / np.linalg.norm(ref))
    e32 = float(np.linalg.norm(outs[1].cpu().numpy() - ref) / np.linalg.norm(ref))
    for pl in plans:
        pl.close()
    assert e64 <= 1e-10 and e32 <= 1e-6


def test_padding_only_for_full_box_grids(kf):
    # a grid with one cell missing, a leaf size that is not a cube, a given root: no padding
    pts = _box((20, 20, 20), 0.05)
    a, b = K.absorption_coefficients(150.0)
    for kw in [dict(points=pts[1:], leaf=64), dict(points=pts, leaf=32),
               dict(points=pts, leaf=64, root=(0.0, 0.0, 0.0, 1.6))]:
        p = kf.Plan(_dev(kw["points"]), 0.05, kw["leaf"], 4, a, b, precision="fp64", pad_lattice=True,
                    root=kw.get("root"))
        assert p.info()["n_padding"] == 0
        p.close()
    # a grid already on the lattice (24 cells a side): no padding, the lattice root all the same
    p = kf.Plan(_dev(_box((24, 24, 24), 0.05)), 0.05, 64, 4, a, b, precision="mixed", pad_lattice=True)
    inf = p.info()
    assert inf["n_padding"] == 0 and inf["side"] == pytest.approx(32 * 0.05) and inf["near_tensor"]
    p.close()
    p = kf.Plan(_dev(pts), 0.05, 64, 4, a, b, precision="fp64", pad_lattice=True)
    inf = p.info()
    assert inf["n_padding"] == 24 ** 3 - 20 ** 3 and inf["side"] == pytest.approx(32 * 0.05)
    assert len(p.sigma()) == 24 ** 3
    perm = p.tree()["perm"]
    assert sorted(perm.tolist()) == list(range(24 ** 3))
    p.close()


def test_tune_with_padding(kf):
    pts = _box((44, 44, 44), 1.0 / 44)
    I = W.gaussian(pts, (0.5, 0.5, 0.5), 0.1, 1e22)
    a, b = K.absorption_coefficients(152.0)
    best, tab = kf.tune(_dev(pts), 1.0 / 44, _dev(I), a, b, leaf=(64,), order=(4, 6), target=1e-2, reps=1,
                        pad_lattice=True)
    assert best["ok"] and all(e["err"] < 5e-2 for e in tab)
