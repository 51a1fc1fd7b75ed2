"""CUDA path against the oracle, through the C-ABI (marked gpu).

Bars:
* tree, Morton keys, permutation and U/V/W/X lists: bit-exact;
* self-cell values: rel 1e-13 (same quadrature, different summation order);
* FP64 KIFMM vs the oracle KIFMM: rel-L2 <= 1e-10. The two share the tree and the
  operator definitions but not the SVD (one-sided Jacobi on the GPU, LAPACK in the
  oracle); the kept spectrum has condition <= 1/eps = 1e5, so the pseudo-inverses
  agree to ~1e5 * 2.2e-16 = 2e-11 relative, and the tolerance leaves a factor 5;
* mixed precision vs FP64 KIFMM: rel-L2 <= 1e-6 (the stated target of the method's
  mixed form: FP32 P2P / check and target evaluations, FP32-accumulated M2L, FP64
  pseudo-inverse applications and L2L chain); on a uniform lattice of full leaves the near
  field runs as per-offset kernel matrices on the tensor cores (FP16 x 3, FP32-accurate),
  held to the same 1e-6 against the FP64 form and against the mixed pair kernel;
* direct-sum parity of the FMM: the paper's own method error (E_V of 0.15-0.7 %
  at m0 = 6), asserted at < 1e-2 where the oracle FMM reaches it.
"""
import numpy as np
import pytest

from oracle import direct as D
from oracle import kernel as K
from oracle import kifmm as KF
from oracle import tree as T
from paper_2006_03515_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _plan(kf, pts, h, leaf, m0, a, b, precision="fp64", uniform=True, **kw):
    hh = float(h[0]) if uniform else _dev(h)
    return kf.Plan(_dev(pts), hh, leaf, m0, a, b, precision=precision, **kw)


def _relerr(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def _adaptive_small():
    # two-level refined grid: base 16^3 on [0, 1]^3, 4x finer in a 5^3 block (4500 fine cells)
    return W.refined_grid(1.0, 16, 4, (0.5, 0.5, 0.7), 2)


CASES = {
    "uniform16_leaf8": lambda: (W.config_uniform(16)[:2] + (8, True)),
    "uniform24_leaf27": lambda: (W.config_uniform(24)[:2] + (27, True)),
    "random_cloud_leaf10": lambda: (W.random_cloud(3000, 11)[:2] + (10, True)),
    "adaptive_leaf16": lambda: (_adaptive_small() + (16, False)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_tree_and_lists_bit_exact(kf, case):
    pts, h, leaf, uni = CASES[case]()
    p = _plan(kf, pts, h, leaf, 4, 5.32, 304.0, uniform=uni)
    t, perm = T.build_tree(pts, h, leaf)
    lists = T.build_lists(t)
    g = p.tree()
    info = p.info()
    assert info["n_boxes"] == len(t.level) and info["n_levels"] == t.nlevels
    assert info["side"] == t.side and info["origin"] == list(t.origin)
    np.testing.assert_array_equal(g["perm"], perm)
    np.testing.assert_array_equal(g["keys"], t.keys)
    np.testing.assert_array_equal(g["level"], t.level)
    np.testing.assert_array_equal(g["parent"], t.parent)
    np.testing.assert_array_equal(g["pstart"], t.pstart)
    np.testing.assert_array_equal(g["pend"], t.pend)
    np.testing.assert_array_equal(g["leaf"].astype(bool), t.leaf)
    np.testing.assert_array_equal(g["anchor"], t.anchor)
    np.testing.assert_array_equal(g["child"], t.child)
    for w in range(4):
        off, items = p.list(w)
        ref = lists[w]
        np.testing.assert_array_equal(np.diff(off), [len(x) for x in ref])
        np.testing.assert_array_equal(items, np.concatenate([np.asarray(x, np.int64) for x in ref] + [np.zeros(0, np.int64)]))
    p.close()


@pytest.mark.parametrize("mode", ["cell_exact", "paper_gl2"])
def test_self_terms(kf, mode):
    pts, h = _adaptive_small()
    a, b = 5.32, 304.0
    p = _plan(kf, pts, h, 16, 4, a, b, uniform=False, self_mode=mode)
    perm = p.tree()["perm"]
    ref = D.self_terms(h[perm], a, b, mode)
    np.testing.assert_allclose(p.sigma(), ref, rtol=1e-13)


@pytest.mark.parametrize("m0", [4, 6, 8])
@pytest.mark.parametrize("po2", [150.0, 1.52])
def test_fp64_kifmm_matches_oracle_uniform(kf, m0, po2):
    pts, h, I = W.config_uniform(16)
    a, b = K.absorption_coefficients(po2)
    C = K.source_scale(760.0)
    ref = KF.kifmm(pts, h, I, 8, m0, a, b, C)
    p = _plan(kf, pts, h, 8, m0, a, b)
    got = p.eval(_dev(I), C=C).cpu().numpy()
    assert _relerr(got, ref) <= 1e-10


@pytest.mark.parametrize("case", ["random_cloud_leaf10", "adaptive_leaf16"])
def test_fp64_kifmm_matches_oracle_adaptive(kf, case):
    pts, h, leaf, uni = CASES[case]()
    I = W.streamer_source(pts, axis_xy=(0.5, 0.5), z_range=(0.2, 0.7), radius=0.05, head=(0.5, 0.5, 0.7),
                          head_sigma=0.05, noise_sigma=0.3, seed=7)
    a, b = 5.32, 304.0
    ref = KF.kifmm(pts, h, I, leaf, 6, a, b)
    p = _plan(kf, pts, h, leaf, 6, a, b, uniform=uni)
    got = p.eval(_dev(I)).cpu().numpy()
    assert _relerr(got, ref) <= 1e-10


@pytest.mark.parametrize("case", ["uniform16_leaf8", "adaptive_leaf16"])
def test_surface_radii_option_matches_oracle(kf, case):
    # surfaces at the radii drawn in Fig. fmulloc, 1.2 r and 2.6 r (plan option; the default
    # is 1.05 / 2.95 r): the FP64 form against the oracle built with the same radii
    pts, h, leaf, uni = CASES[case]()
    I = W.streamer_source(pts, axis_xy=(0.5, 0.5), z_range=(0.2, 0.7), radius=0.05, head=(0.5, 0.5, 0.7),
                          head_sigma=0.05, noise_sigma=0.3, seed=7)
    a, b = 5.32, 304.0
    radii = KF.FIGURE_RADII
    ref = KF.kifmm(pts, h, I, leaf, 6, a, b, radii=radii)
    got = _plan(kf, pts, h, leaf, 6, a, b, uniform=uni, surface_radii=radii).eval(_dev(I)).cpu().numpy()
    assert _relerr(got, ref) <= 1e-10


def test_surface_radii_option_accuracy_and_mixed(kf):
    # 32^3 at 760 Torr (p_O2 150): the default surfaces at 1.05 / 2.95 r keep a lower rank and
    # follow the whole discrete sum (FFT oracle) far closer than the radii drawn in Fig.
    # fmulloc, 1.2 / 2.6 r (oracle: 1.8e-4 against 3.3e-3); the mixed form of both readings
    # (lattice paths, tensor-core M2L) stays within 1e-6 of its FP64 form
    pts, h, I = W.config_uniform(32)
    a, b = K.absorption_coefficients(150.0)
    C = K.source_scale(760.0)
    ref = D.fft_uniform(I.reshape(32, 32, 32), h[0], a, b, C).ravel()
    Id = _dev(I)
    p_def = _plan(kf, pts, h, 64, 6, a, b)
    p_fig = _plan(kf, pts, h, 64, 6, a, b, surface_radii=KF.FIGURE_RADII)
    assert p_def.info()["pinv_rank_min"] < p_fig.info()["pinv_rank_min"]
    s_def = p_def.eval(Id, C=C).cpu().numpy()
    s_fig = p_fig.eval(Id, C=C).cpu().numpy()
    e_def, e_fig = _relerr(s_def, ref), _relerr(s_fig, ref)
    assert e_def < 1e-3 and e_def < e_fig / 5, (e_def, e_fig)
    for radii, s64 in [(None, s_def), (KF.FIGURE_RADII, s_fig)]:
        pm = _plan(kf, pts, h, 64, 6, a, b, precision="mixed", surface_radii=radii)
        inf = pm.info()
        assert inf["m2l_tensor"] and inf["near_tensor"] and inf["lattice_far"]
        assert _relerr(pm.eval(Id, C=C).cpu().numpy(), s64) <= 1e-6
        pm.check()


@pytest.mark.parametrize("m0", [4, 6, 8])
@pytest.mark.parametrize("po2", [152.0, 15.2, 1.52])
def test_mixed_matches_fp64(kf, m0, po2):
    pts, h, I = W.config_uniform(32)
    a, b = K.absorption_coefficients(po2)
    p64 = _plan(kf, pts, h, 64, m0, a, b)
    p32 = _plan(kf, pts, h, 64, m0, a, b, precision="mixed")
    Id = _dev(I)
    s64 = p64.eval(Id).cpu().numpy()
    s32 = p32.eval(Id).cpu().numpy()
    assert _relerr(s32, s64) <= 1e-6


@pytest.mark.parametrize("adaptive", [False, True])
def test_upward_tensor_slices_match_fp64(kf, monkeypatch, adaptive):
    """The mixed form's upward pseudo-inverse on the tensor cores (exact integer slices, FP64
    combination) against the same plan's FP64-pipe GEMM: agreement of the upward coefficients
    c of every box to FP64 accuracy. Each input row is cut to 54-bit fixed point relative to
    its largest element, so both products err by about 2^-53 sum_k |G1_rk chk_k|, which
    exceeds |c_r| by the cancellation in G1 chk (up to ~1e6 here with the default surfaces):
    the bar is 1e-9 of the box's largest coefficient, three orders below the FP32 arithmetic
    of the rest of the mixed form."""
    if adaptive:
        pts, h = _adaptive_small()
        I = W.streamer_source(pts, axis_xy=(0.5, 0.5), z_range=(0.2, 0.7), radius=0.05, head=(0.5, 0.5, 0.7),
                              head_sigma=0.05, noise_sigma=0.3, seed=7)
        a, b, leaf, uniform = 5.32, 304.0, 16, False
    else:
        pts, h, I = W.config_uniform(32)
        a, b = K.absorption_coefficients(152.0)
        leaf, uniform = 64, True

    monkeypatch.setenv("KIFMM_OZ_MIN", "0")   # every level through the slice products
    monkeypatch.setenv("KIFMM_P2P", "generic")   # both runs from the same check potentials

    def run(mode):
        if mode:
            monkeypatch.setenv("KIFMM_UPWARD", mode)
        else:
            monkeypatch.delenv("KIFMM_UPWARD", raising=False)
        p = _plan(kf, pts, h, leaf, 6, a, b, uniform=uniform, precision="mixed")
        s = p.eval(_dev(I)).cpu().numpy()
        c = p.upward()
        p.close()
        return s, c

    s_tc, c_tc = run(None)
    s_64, c_64 = run("fp64")
    scale = np.abs(c_64).max(axis=1, keepdims=True)
    scale[scale == 0] = 1.0
    assert np.max(np.abs(c_tc - c_64) / scale) <= 1e-9
    assert _relerr(s_tc, s_64) <= 1e-9


@pytest.mark.parametrize("n,leaf", [(32, 64), (64, 64)])
def test_near_field_on_tensor_cores(kf, monkeypatch, n, leaf):
    # uniform lattice with full 64-cell leaves: the near field runs as 27 per-offset kernel
    # matrices on the tensor cores, S2M / upward / local L2P as one tabulated matrix per leaf;
    # against the FP64 form and the mixed generic kernels
    pts, h, I = W.config_uniform(n)
    a, b = K.absorption_coefficients(152.0)
    Id = _dev(I)
    s64 = _plan(kf, pts, h, leaf, 6, a, b).eval(Id).cpu().numpy()
    ptc = _plan(kf, pts, h, leaf, 6, a, b, precision="mixed")
    assert ptc.info()["near_tensor"]
    assert ptc.info()["lattice_far"]   # S2M / L2P matrices: leaves at level >= 2, 64 cells
    stc = ptc.eval(Id).cpu().numpy()
    monkeypatch.setenv("KIFMM_P2P", "generic")
    pgen = _plan(kf, pts, h, leaf, 6, a, b, precision="mixed")
    assert not pgen.info()["near_tensor"]
    sgen = pgen.eval(Id).cpu().numpy()
    assert _relerr(stc, s64) <= 1e-6
    assert _relerr(stc, sgen) <= 1e-6


def test_lattice_leaf_coefficients_match_fp64(kf, monkeypatch):
    # on a lattice the leaves' upward coefficients come from their weights through M = G1 P
    # (FP64, sliced exactly on the tensor cores); the FP64 form gets them from check
    # potentials summed in FP64: both are FP64 evaluations of the same operator (reassociated),
    # so they agree to FP64 rounding times the pseudo-inverse's condition (<= 1e5)
    monkeypatch.setenv("KIFMM_OZ_MIN", "0")   # 512 leaves: below the default level size of the slices
    pts, h, I = W.config_uniform(32)
    a, b = K.absorption_coefficients(152.0)
    Id = _dev(I)
    pm = _plan(kf, pts, h, 64, 6, a, b, precision="mixed")
    assert pm.info()["lattice_far"]
    assert pm.info()["upward_flops"] < _plan(kf, pts, h, 64, 6, a, b).info()["upward_flops"]   # leaves: r npl
    pm.eval(Id)
    p64 = _plan(kf, pts, h, 64, 6, a, b)
    p64.eval(Id)
    c_m, c_64 = pm.upward(), p64.upward()
    leaves = np.nonzero(pm.tree()["leaf"])[0]
    scale = np.abs(c_64[leaves]).max(axis=1, keepdims=True)
    assert np.max(np.abs(c_m[leaves] - c_64[leaves]) / scale) <= 1e-8


def _box_grid(nx, ny, nz, h):
    # cell centres of an nx x ny x nz block of cells of edge h, Gaussian source off centre
    g = np.stack(np.meshgrid((np.arange(nx) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nz) + 0.5) * h,
                             indexing="ij"), axis=-1).reshape(-1, 3)
    c = np.array([0.4 * nx, 0.6 * ny, 0.5 * nz]) * h
    I = 1e22 * np.exp(-((g - c) ** 2).sum(1) / 0.08 ** 2) + 1e18
    return g, np.full(len(g), h), I


@pytest.mark.parametrize("shape,leaf,lattice", [((64, 32, 48), 64, True), ((64, 64, 64), 512, False)])
def test_lattice_edge_cases(kf, shape, leaf, lattice):
    # a non-cubic block of cells (the root cube has empty boxes; every present leaf is full):
    # the lattice paths; 512-cell leaves: the generic kernels (a near-field slot of K = 512
    # would bias the tensor core's truncating accumulation); both against the FP64 form
    pts, h, I = _box_grid(*shape, 1.0 / 64)
    a, b = K.absorption_coefficients(152.0)
    Id = _dev(I)
    s64 = _plan(kf, pts, h, leaf, 6, a, b).eval(Id).cpu().numpy()
    pm = _plan(kf, pts, h, leaf, 6, a, b, precision="mixed")
    inf = pm.info()
    assert inf["near_tensor"] == lattice and inf["lattice_far"] == lattice
    assert _relerr(pm.eval(Id).cpu().numpy(), s64) <= 1e-6


@pytest.mark.parametrize("n,lattice", [(40, True), (36, False)])
def test_root_aligned_with_the_cell_lattice(kf, n, lattice):
    # a given root cube aligned with the grid's cells (origin at its corner, side 4 h 2^k):
    # at n = 40 every leaf is a full 4^3 block at one level (the lattice paths); at n = 36
    # the far corner's 4^3 block stays a coarser leaf (generic kernels). FP64 form against
    # the oracle with the same root, mixed form against the FP64 form.
    pts, h, I = W.config_uniform(n)
    a, b = K.absorption_coefficients(152.0)
    side = 64 * h[0]
    root = (0.0, 0.0, 0.0, side)
    pl = KF.plan(pts, h, 64, 6, a, b, origin=np.zeros(3), side=side)
    ref = KF.evaluate(pl, I)
    Id = _dev(I)
    s64 = _plan(kf, pts, h, 64, 6, a, b, root=root).eval(Id).cpu().numpy()
    assert _relerr(s64, ref) <= 1e-10
    pm = _plan(kf, pts, h, 64, 6, a, b, precision="mixed", root=root)
    inf = pm.info()
    assert inf["near_tensor"] == lattice and inf["lattice_far"] == lattice
    assert _relerr(pm.eval(Id).cpu().numpy(), s64) <= 1e-6


def test_near_field_lattice_detection(kf):
    # not a lattice of full leaves: the pair kernel (8-cell leaves, a random cloud, the
    # refined grid, per-point h)
    a, b = 5.32, 304.0
    pts, h, _ = W.config_uniform(16)
    assert not _plan(kf, pts, h, 8, 6, a, b, precision="mixed").info()["near_tensor"]
    pts, h = W.random_cloud(3000, 11)[:2]
    assert not _plan(kf, pts, h, 64, 6, a, b, precision="mixed").info()["near_tensor"]
    pts, h = _adaptive_small()
    assert not _plan(kf, pts, h, 64, 6, a, b, precision="mixed", uniform=False).info()["near_tensor"]
    pts, h, _ = W.config_uniform(32)
    assert not _plan(kf, pts, h, 64, 6, a, b).info()["near_tensor"]   # FP64 form


@pytest.mark.parametrize("adaptive", [False, True])
def test_l2l_tensor_cores_against_simt(kf, monkeypatch, adaptive):
    # L2L and the M2M translations through the tensor-core translation kernel (FP16 x 3 splits;
    # L2L added onto the children's M2L result) against the SIMT FP32 applies and the FP64 form
    if adaptive:
        pts, h = _adaptive_small()
        I = W.streamer_source(pts, axis_xy=(0.5, 0.5), z_range=(0.2, 0.7), radius=0.05, head=(0.5, 0.5, 0.7),
                              head_sigma=0.05, noise_sigma=0.3, seed=7)
        a, b, leaf, uniform = 5.32, 304.0, 16, False
    else:
        pts, h, I = W.config_uniform(64)
        a, b = K.absorption_coefficients(152.0)
        leaf, uniform = 64, True
    Id = _dev(I)
    s64 = _plan(kf, pts, h, leaf, 6, a, b, uniform=uniform).eval(Id).cpu().numpy()
    stc = _plan(kf, pts, h, leaf, 6, a, b, uniform=uniform, precision="mixed").eval(Id).cpu().numpy()
    monkeypatch.setenv("KIFMM_L2L", "simt")
    monkeypatch.setenv("KIFMM_M2M", "simt")
    ssimt = _plan(kf, pts, h, leaf, 6, a, b, uniform=uniform, precision="mixed").eval(Id).cpu().numpy()
    assert _relerr(stc, s64) <= 1e-6
    assert _relerr(stc, ssimt) <= 1e-6


def test_mixed_adaptive_matches_fp64(kf):
    pts, h = _adaptive_small()
    I = W.streamer_source(pts, axis_xy=(0.5, 0.5), z_range=(0.2, 0.7), radius=0.05, head=(0.5, 0.5, 0.7),
                          head_sigma=0.05, noise_sigma=0.3, seed=7)
    a, b = 5.32, 304.0
    s64 = _plan(kf, pts, h, 16, 6, a, b, uniform=False).eval(_dev(I)).cpu().numpy()
    s32 = _plan(kf, pts, h, 16, 6, a, b, uniform=False, precision="mixed").eval(_dev(I)).cpu().numpy()
    assert _relerr(s32, s64) <= 1e-6


def test_config1_against_direct_sum(kf):
    # 32^3 on a 1 cm cube, I = 1e22 exp(-|r-c|^2/0.1^2), p = 760, p_O2 = 150, m0 = 6, leaf 64
    pts, h, I = W.config_uniform(32)
    a, b = K.absorption_coefficients(150.0)
    C = K.source_scale(760.0)
    ref = D.fft_uniform(I.reshape(32, 32, 32), h[0], a, b, C).ravel()
    p = _plan(kf, pts, h, 64, 6, a, b)
    got = p.eval(_dev(I), C=C).cpu().numpy()
    assert _relerr(got, ref) < 1e-2
    # and the oracle FMM at the same settings lands at the same error
    orc = KF.kifmm(pts, h, I, 64, 6, a, b, C)
    assert _relerr(got, orc) <= 1e-10


def test_single_leaf_equals_direct(kf):
    pts, h, I = W.random_cloud(700, 5)
    ref = D.direct_sum(pts, h, I, 5.32, 304.0)
    for prec, tol in [("fp64", 1e-13), ("mixed", 2e-6)]:
        got = _plan(kf, pts, h, 1000, 6, 5.32, 304.0, precision=prec).eval(_dev(I)).cpu().numpy()
        assert _relerr(got, ref) <= tol


def test_one_point(kf):
    pts = np.array([[0.3, 0.2, 0.1]])
    for prec in ("fp64", "mixed"):
        p = _plan(kf, pts, np.array([0.01]), 4, 6, 5.32, 304.0, precision=prec)
        got = p.eval(_dev([2.0]), C=1.5).cpu().numpy()
        assert got[0] == pytest.approx(1.5 * 2.0 * K.sigma_cell_exact(0.01, 5.32, 304.0), rel=1e-13)


def test_float32_io_and_host_path(kf):
    import torch
    pts, h, I = W.config_uniform(16)
    p = _plan(kf, pts, h, 8, 6, 5.32, 304.0, precision="mixed")
    s64 = p.eval(_dev(I)).cpu().numpy()
    s32 = p.eval(_dev(I).to(torch.float32)).cpu().numpy()
    assert _relerr(s32.astype(np.float64), s64) < 1e-6
    sh = p.eval_host(I)
    # small levels add split partial sums atomically, in an order that may vary between evaluations
    np.testing.assert_allclose(sh, s64, rtol=1e-12, atol=0)


def test_batch_and_graph_replay(kf):
    import torch
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plans, Is, refs = [], [], []
        for k, (n, po2) in enumerate([(12, 152.0), (16, 15.2), (20, 152.0)]):
            pts, h, I = W.config_uniform(n)
            a, b = K.absorption_coefficients(po2)
            p = _plan(kf, pts, h, 16, 4, a, b, precision="mixed", stream=st)
            plans.append(p)
            Is.append(_dev(I))
            refs.append(p.eval(Is[-1]).clone())
        # a repeated plan (its entries share the plan's workspace, so they share one lane and
        # run in order); twice the source gives twice the field exactly (power-of-two scaling)
        plans.append(plans[0])
        Is.append(2 * Is[0])
        refs.append(2 * refs[0])
        Ss = [torch.empty_like(x) for x in Is]
        for lanes in (1, 3, 8):
            for capture in (False, True, True):
                for s in Ss:
                    s.zero_()
                kf.eval_batch(plans, Is, Ss, capture=capture, lanes=lanes)
                st.synchronize()
                for s, r in zip(Ss, refs):   # small levels add split partial sums atomically
                    assert torch.allclose(s, r, rtol=1e-12, atol=0)


def test_allocation_failures_are_reported_and_recovered(kf, monkeypatch):
    # host-side fault injection (no device fault): the k-th device allocation of a plan
    # reports out-of-memory; no plan is returned, its partial state is freed, and plans
    # made afterwards are unaffected
    pts, h, I = W.config_uniform(16)
    a, b = 5.32, 304.0
    Id = _dev(I)
    ref = _plan(kf, pts, h, 8, 6, a, b, precision="mixed").eval(Id).cpu().numpy()
    failed = 0
    for k in (1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233):
        monkeypatch.setenv("KIFMM_FAIL_ALLOC", str(k))
        try:
            p = _plan(kf, pts, h, 8, 6, a, b, precision="mixed")
        except kf.KifmmError as e:
            assert e.code == -2, str(e)
            failed += 1
            continue
        monkeypatch.delenv("KIFMM_FAIL_ALLOC")
        np.testing.assert_allclose(p.eval(Id).cpu().numpy(), ref, rtol=1e-12, atol=0)
        p.close()
    assert failed >= 5
    monkeypatch.delenv("KIFMM_FAIL_ALLOC", raising=False)
    again = _plan(kf, pts, h, 8, 6, a, b, precision="mixed").eval(Id).cpu().numpy()
    np.testing.assert_allclose(again, ref, rtol=1e-12, atol=0)


def test_duplicate_and_nonfinite_rejected(kf):
    pts, h, I = W.random_cloud(100, 3)
    bad = pts.copy()
    bad[5] = bad[9]
    with pytest.raises(kf.KifmmError) as e:
        _plan(kf, bad, h, 8, 4, 5.32, 304.0)
    assert e.value.code == -5
    bad = pts.copy()
    bad[3, 1] = np.nan
    with pytest.raises(kf.KifmmError) as e:
        _plan(kf, bad, h, 8, 4, 5.32, 304.0)
    assert e.value.code == -6


def test_given_root_cube(kf):
    pts, h, I = W.config_uniform(12)
    a, b = 5.32, 304.0
    root = (-0.5, -0.5, -0.5, 2.0)
    t, perm = T.build_tree(pts, h, 8, np.array(root[:3]), root[3])
    p = _plan(kf, pts, h, 8, 6, a, b, root=root)
    np.testing.assert_array_equal(p.tree()["keys"], t.keys)
    with pytest.raises(kf.KifmmError):
        _plan(kf, pts, h, 8, 6, a, b, root=(0.2, 0.0, 0.0, 1.0))


def test_tensor_core_m2l_against_simt_and_fp64(kf, monkeypatch):
    # the mixed form's M2L runs on tcgen05 (3xTF32); the SIMT FP32 M2L is the cross-check
    pts, h, I = W.config_uniform(32)
    a, b = K.absorption_coefficients(15.2)
    s64 = _plan(kf, pts, h, 64, 6, a, b).eval(_dev(I)).cpu().numpy()
    p_tc = _plan(kf, pts, h, 64, 6, a, b, precision="mixed")
    assert p_tc.info()["m2l_tensor"]
    s_tc = p_tc.eval(_dev(I)).cpu().numpy()
    assert p_tc.info()["device_error"] == 0
    monkeypatch.setenv("KIFMM_M2L", "simt")
    p_simt = _plan(kf, pts, h, 64, 6, a, b, precision="mixed")
    assert not p_simt.info()["m2l_tensor"]
    s_simt = p_simt.eval(_dev(I)).cpu().numpy()
    assert _relerr(s_tc, s64) <= 1e-6
    assert _relerr(s_simt, s64) <= 1e-6
    assert _relerr(s_tc, s_simt) <= 1e-6


def test_autotune_picks_a_candidate(kf):
    pts, h, I = W.config_uniform(32)
    a, b = K.absorption_coefficients(152.0)
    best, times = kf.autotune(_dev(pts), float(h[0]), candidates=(16, 32, 64, 128), a=a, b=b, reps=2)
    assert best in (16, 32, 64, 128) and all(t > 0 for t in times.values())
    assert times[best] == min(times.values())
    s64 = _plan(kf, pts, h, best, 6, a, b).eval(_dev(I)).cpu().numpy()
    s32 = _plan(kf, pts, h, best, 6, a, b, precision="mixed").eval(_dev(I)).cpu().numpy()
    assert _relerr(s32, s64) <= 1e-6


def test_batched_uneven_fields_graph_captured(kf):
    # the batched workload at reduced size: uneven fields (two tilted channels each, two
    # pressures) in one CUDA graph, back to back and on concurrent lanes, against per-field
    # evaluation
    import torch
    st = torch.cuda.Stream()
    fields = [W.two_channel_field(k, n_min=18, n_max=34) for k in range(6)]
    assert len({len(f[0]) for f in fields}) > 2 and {f[3] for f in fields} == {760.0, 76.0}
    with torch.cuda.stream(st):
        plans, Is, refs, Cs = [], [], [], []
        for pts, h, I, p in fields:
            a, b = K.absorption_coefficients(0.2 * p)
            pl = _plan(kf, pts, h, 32, 6, a, b, precision="mixed", stream=st)
            plans.append(pl)
            Is.append(_dev(I))
            Cs.append(K.source_scale(p))
            refs.append(pl.eval(Is[-1], C=Cs[-1]).clone())
        Ss = [torch.empty_like(x) for x in Is]
        for lanes in (1, 4, 1):
            for _ in range(2):
                for s in Ss:
                    s.fill_(float("nan"))
                kf.eval_batch(plans, Is, Ss, C=Cs, capture=True, lanes=lanes)
                st.synchronize()
                for s, r in zip(Ss, refs):   # small levels add split partial sums atomically
                    assert torch.allclose(s, r, rtol=1e-12, atol=0)
    # one field against the FP64 form
    pts, h, I, p = fields[0]
    a, b = K.absorption_coefficients(0.2 * p)
    s64 = _plan(kf, pts, h, 32, 6, a, b).eval(_dev(I), C=Cs[0]).cpu().numpy()
    assert _relerr(refs[0].cpu().numpy(), s64) <= 1e-6


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def test_full_size_uniform_128(kf):
    # 128^3 cell centres (2,097,152 points), Gaussian source, p = 760 Torr, p_O2 = 152, m0 = 6,
    # leaf 64 (the benchmark's workload and launch configuration)
    pts, h, I = W.config_uniform(128)
    a, b = K.absorption_coefficients(152.0)
    C = K.source_scale(760.0)
    Id = _dev(I)
    s64 = _plan(kf, pts, h, 64, 6, a, b).eval(Id, C=C)
    s32 = _plan(kf, pts, h, 64, 6, a, b, precision="mixed").eval(Id, C=C)
    import torch
    assert float(torch.linalg.norm(s32 - s64) / torch.linalg.norm(s64)) <= 1e-6
    # sampled outputs against the direct sum (the FMM's own approximation error, the paper's
    # E_V magnitude), and the whole field against the FFT form of the same sum
    idx = _sample(len(pts), 512, 1)
    ref = D.direct_sum(pts, h, I, a, b, C, targets=idx)
    got = s64.cpu().numpy()
    e_direct = _relerr(got[idx], ref)
    full = D.fft_uniform(I.reshape(128, 128, 128), h[0], a, b, C).ravel()
    np.testing.assert_allclose(full[idx], ref, rtol=1e-10)
    e_full = _relerr(got, full)
    assert e_direct < 1e-2 and e_full < 1e-2, (e_direct, e_full)


def test_full_size_adaptive(kf):
    # two-level refined grid on a 2 cm cube: base h = 1/64, 8x finer around the head
    # (3,219,819 points), channel + head + log-normal noise, p = 760 Torr, p_O2 = 150
    pts, h, I = W.config_adaptive()
    assert len(pts) == 3219819
    a, b = K.absorption_coefficients(150.0)
    C = K.source_scale(760.0)
    Id = _dev(I)
    p64 = _plan(kf, pts, h, 64, 6, a, b, uniform=False)
    info = p64.info()
    assert info["list_len"][2] > 0 and info["list_len"][3] > 0   # W and X lists in use
    s64 = p64.eval(Id, C=C)
    s32 = _plan(kf, pts, h, 64, 6, a, b, uniform=False, precision="mixed").eval(Id, C=C)
    import torch
    assert float(torch.linalg.norm(s32 - s64) / torch.linalg.norm(s64)) <= 1e-6
    fine = np.nonzero(h < h.max())[0]
    idx = np.concatenate([_sample(len(pts), 128, 2), fine[_sample(len(fine), 128, 3)]])
    ref = D.direct_sum(pts, h, I, a, b, C, targets=idx)
    assert _relerr(s64.cpu().numpy()[idx], ref) < 2e-2


def _rect_grid(nx, ny, nz, hx, hy, hz):
    g = [(np.arange(m) + 0.5) * hh for m, hh in ((nx, hx), (ny, hy), (nz, hz))]
    zz, yy, xx = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


@pytest.mark.parametrize("mode", ["cell_exact", "paper_gl2"])
def test_rectangular_cells_against_oracle(kf, mode):
    # cells of aspect 1 : 1 : 4.5 (the Sec. 4.2 grid's shape), a Gaussian source off centre:
    # the FP64 form against the oracle KIFMM of the same tree (weights hx hy hz, the box's own
    # self term), the mixed form against the FP64 form, and the one-leaf plan against the
    # whole discrete sum of the rectangular grid (FFT oracle)
    nx, ny, nz = 24, 24, 20
    hx, hy, hz = 1.0 / 96, 1.0 / 96, 4.5 / 96
    pts = _rect_grid(nx, ny, nz, hx, hy, hz)
    I = W.gaussian(pts, (0.12, 0.13, 0.45), 0.05, 1e22) + 1e18
    a, b = K.absorption_coefficients(160.0)
    C = K.source_scale(800.0)
    dims = (hx, hy, hz)
    ref = KF.kifmm(pts, None, I, 32, 6, a, b, C, mode=mode, cell_dims=dims)
    p64 = kf.Plan(_dev(pts), None, 32, 6, a, b, precision="fp64", cell_dims=dims, self_mode=mode)
    inf = p64.info()
    assert not inf["near_tensor"]
    s64 = p64.eval(_dev(I), C=C).cpu().numpy()
    assert _relerr(s64, ref) <= 1e-10
    pm = kf.Plan(_dev(pts), None, 32, 6, a, b, precision="mixed", cell_dims=dims, self_mode=mode)
    assert _relerr(pm.eval(_dev(I), C=C).cpu().numpy(), s64) <= 1e-6
    full = D.fft_box_grid(I.reshape(nz, ny, nx), dims, a, b, C, mode=mode).ravel()
    one = kf.Plan(_dev(pts), None, len(pts), 6, a, b, precision="fp64", cell_dims=dims, self_mode=mode)
    assert _relerr(one.eval(_dev(I), C=C).cpu().numpy(), full) <= 1e-12
    with pytest.raises(kf.KifmmError):
        kf.Plan(_dev(pts), None, 32, 6, a, b, cell_dims=(hx, -1.0, hz))


@pytest.mark.parametrize("p,m0", [(760.0, 4), (760.0, 8), (76.0, 6), (7.6, 6)])
def test_full_size_uniform_128_pressures_and_orders(kf, p, m0):
    # the 128^3 Gaussian field at the other pressures (p_O2 = 0.2 p) and surface orders of the
    # target settings: mixed form within 1e-6 of the FP64 form; both forms against the whole
    # discrete sum (oracle FFT convolution) at the surface form's accuracy (below 1e-2)
    import torch
    pts, h, I = W.config_uniform(128)
    a, b = K.absorption_coefficients(0.2 * p)
    C = K.source_scale(p)
    Id = _dev(I)
    s64 = _plan(kf, pts, h, 64, m0, a, b).eval(Id, C=C)
    s32 = _plan(kf, pts, h, 64, m0, a, b, precision="mixed").eval(Id, C=C)
    assert float(torch.linalg.norm(s32 - s64) / torch.linalg.norm(s64)) <= 1e-6
    full = D.fft_uniform(I.reshape(128, 128, 128), h[0], a, b, C).ravel()
    assert _relerr(s64.cpu().numpy(), full) < (5e-2 if m0 == 4 else 2e-2)
