"""The streamer time loop (Sec. 5, Eq. (eM)) on the GPU against its oracle (marked gpu).

The multigrid Poisson solve against the oracle's direct sparse solve; the right-hand side of
the density equations (fields, S_i, drift and diffusion fluxes, and S_ph from an FP64 KIFMM
plan of the grid) against the oracle's with S_ph from the oracle KIFMM of the same tree and
surfaces; Heun steps against the oracle's; the default tolerance of the paper (relative
residual 1e-8) reached; the double-headed streamer initial condition of Sec. 5 advanced on
a grid of the paper's aspect with the mixed-form FMM (finite, positive where it must be).
"""
import numpy as np
import pytest

from oracle import kernel as K
from oracle import kifmm as KF
from oracle import streamer as SD

pytestmark = pytest.mark.gpu

NX, NY, NZ, H = 16, 16, 24, 0.02


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _centres(nx, ny, nz, h):
    g = [(np.arange(m) + 0.5) * h for m in (nx, ny, nz)]
    zz, yy, xx = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


def _state(seed=0, nx=NX, ny=NY, nz=NZ, h=H):
    """Two Gaussian seeds (the double-headed streamer of Sec. 5, scaled to the box) and a
    seeded perturbation, n_e a little above n_p near one seed (a net charge)."""
    rng = np.random.default_rng(seed)
    pts = _centres(nx, ny, nz, h).reshape(nz, ny, nx, 3)
    L = np.array([nx, ny, nz]) * h

    def g(c, s):
        return np.exp(-((pts - np.asarray(c) * L) ** 2).sum(-1) / (s * L[2]) ** 2)
    n0 = 1e14 * (g((0.44, 0.5, 0.41), 0.06) + g((0.56, 0.5, 0.59), 0.06))
    ne = n0 * (1.0 + 0.05 * rng.standard_normal(n0.shape)) + 1e9
    npi = n0 + 1e9
    return ne, npi


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_poisson_matches_direct_solve(kf):
    rng = np.random.default_rng(1)
    rho = rng.standard_normal((NZ, NY, NX)) * 1e8
    s = kf.Streamer(NX, NY, NZ, H, mg_tol=1e-12)
    phi, res, cyc = s.poisson(_dev(rho))
    assert s.info()["mg_levels"] >= 2 and res <= 1e-12 and cyc <= 40
    want = SD.solve_poisson(rho, H, 52e3)
    assert _rel(phi.cpu().numpy(), want) <= 1e-9
    # the paper's stopping rule: relative residual 1e-8 in a few V-cycles
    s2 = kf.Streamer(NX, NY, NZ, H)
    phi2, res2, cyc2 = s2.poisson(_dev(rho))
    assert res2 <= 1e-8 and cyc2 <= 15
    assert _rel(phi2.cpu().numpy(), want) <= 1e-6
    s.close()
    s2.close()


def _oracle_sph(plan_kw):
    pts = _centres(NX, NY, NZ, H)
    a, b = K.absorption_coefficients(150.0)
    C = SD.params()["C"]
    op = KF.plan(pts, np.full(len(pts), H), plan_kw["leaf"], plan_kw["m0"], a, b)

    def sph(Si):
        return KF.evaluate(op, Si.ravel(), C)
    return pts, a, b, sph


def test_rhs_matches_oracle_with_photoionization(kf):
    kw = dict(leaf=64, m0=4)
    pts, a, b, sph = _oracle_sph(kw)
    ne, npi = _state(2)
    pl = kf.Plan(_dev(pts), H, kw["leaf"], kw["m0"], a, b, precision="fp64")
    s = kf.Streamer(NX, NY, NZ, H, plan=pl, mg_tol=1e-12)
    s.set(_dev(ne), _dev(npi))
    dne, dnp = s.rhs()
    _, _, phi, Sph = s.get()
    want_e, want_p, aux = SD.rhs(ne, npi, H, SD.params(), sph)
    assert _rel(phi.cpu().numpy(), aux["phi"]) <= 1e-9
    assert _rel(Sph.cpu().numpy(), aux["Sph"]) <= 1e-8
    assert _rel(dne.cpu().numpy(), want_e) <= 1e-8
    assert _rel(dnp.cpu().numpy(), want_p) <= 1e-8
    s.close()
    pl.close()


def test_heun_steps_match_oracle(kf):
    kw = dict(leaf=64, m0=4)
    pts, a, b, sph = _oracle_sph(kw)
    ne, npi = _state(3)
    pl = kf.Plan(_dev(pts), H, kw["leaf"], kw["m0"], a, b, precision="fp64")
    s = kf.Streamer(NX, NY, NZ, H, plan=pl, mg_tol=1e-12)
    s.set(_dev(ne), _dev(npi))
    dt = 1e-12
    s.step(dt, 2)
    ge, gp, _, _ = s.get()
    we, wp = ne, npi
    for _ in range(2):
        we, wp, _ = SD.heun_step(we, wp, dt, H, SD.params(), sph)
    assert _rel(ge.cpu().numpy(), we) <= 1e-8
    assert _rel(gp.cpu().numpy(), wp) <= 1e-8
    s.close()
    pl.close()


def test_without_photoionization_and_argument_checks(kf):
    ne, npi = _state(4)
    s = kf.Streamer(NX, NY, NZ, H, mg_tol=1e-12)
    s.set(_dev(ne), _dev(npi))
    s.step(1e-12, 1)
    ge, gp, _, Sph = s.get()
    we, wp, _ = SD.heun_step(ne, npi, 1e-12, H, SD.params())
    assert _rel(ge.cpu().numpy(), we) <= 1e-8 and _rel(gp.cpu().numpy(), wp) <= 1e-8
    assert float(Sph.abs().max()) == 0.0
    s.close()
    with pytest.raises(kf.KifmmError):   # a grid that does not coarsen to a small level
        kf.Streamer(67, 67, 67, 0.01)
    pts = _centres(8, 8, 8, 0.1)
    a, b = K.absorption_coefficients(150.0)
    pl = kf.Plan(_dev(pts), 0.1, 64, 4, a, b)
    with pytest.raises(kf.KifmmError):   # a plan of another point count
        kf.Streamer(NX, NY, NZ, H, plan=pl)
    pl.close()


def test_local_and_thresholded_photoionization(kf):
    # S_ph over a sub-box from the sources inside it above 1e-3 of the largest (Sec. 5.1's
    # remark): the plan over the region's cells; zero outside; the oracle KIFMM of the same
    # thresholded region sources
    ne, npi = _state(5)
    reg = (2, 14, 3, 13, 4, 20)
    sub = (slice(reg[4], reg[5]), slice(reg[2], reg[3]), slice(reg[0], reg[1]))
    rp = _centres(NX, NY, NZ, H).reshape(NZ, NY, NX, 3)[sub].reshape(-1, 3)
    a, b = K.absorption_coefficients(150.0)
    C = SD.params()["C"]
    op = KF.plan(rp, np.full(len(rp), H), 64, 4, a, b)
    pl = kf.Plan(_dev(rp), H, 64, 4, a, b, precision="fp64")
    s = kf.Streamer(NX, NY, NZ, H, plan=pl, mg_tol=1e-12, region=reg, threshold=1e-3)

    def sph(Si):
        loc = Si[sub].ravel().copy()
        loc[loc < 1e-3 * Si.max()] = 0.0
        out = np.zeros_like(Si)
        out[sub] = KF.evaluate(op, loc, C).reshape(out[sub].shape)
        return out
    s.set(_dev(ne), _dev(npi))
    dne, _ = s.rhs()
    _, _, _, Sph = s.get()
    want_e, _, aux = SD.rhs(ne, npi, H, SD.params(), sph)
    got = Sph.cpu().numpy()
    assert _rel(got, aux["Sph"]) <= 1e-8 and np.all(got[:reg[4]] == 0.0)
    assert _rel(dne.cpu().numpy(), want_e) <= 1e-8
    s.close()
    pl.close()
    with pytest.raises(kf.KifmmError):   # a region outside the grid
        kf.Streamer(NX, NY, NZ, H, region=(0, NX + 1, 0, NY, 0, NZ))


def test_double_headed_streamers_advance(kf):
    # Sec. 5's two Gaussian seeds in a 0.5 x 0.5 x 1 cm gap at 52 kV, 32 x 32 x 64 cells, the
    # mixed-form FMM for S_ph (a lattice plan, padded), 20 steps of 2.5e-3 ns
    import torch
    nx, ny, nz, h = 32, 32, 64, 1.0 / 64
    pts = _centres(nx, ny, nz, h)
    a, b = K.absorption_coefficients(150.0)
    pl = kf.Plan(_dev(pts), h, 64, 6, a, b, precision="mixed", pad_lattice=True)
    s = kf.Streamer(nx, ny, nz, h, plan=pl)
    c = pts.reshape(nz, ny, nx, 3)

    def g(x0):
        return np.exp(-((c - np.asarray(x0)) ** 2).sum(-1) / 0.03 ** 2)
    n0 = 1e14 * (g((0.22, 0.25, 0.41)) + g((0.28, 0.25, 0.59)))
    s.set(_dev(n0), _dev(n0))
    s.step(2.5e-12, 20)
    ne, npi, phi, Sph = s.get()
    assert torch.isfinite(ne).all() and torch.isfinite(npi).all() and torch.isfinite(phi).all()
    # (far from the heads the FMM's own approximation error leaves values near 0 of either sign)
    assert float(Sph.max()) > 0.0 and float(Sph.min()) >= -1e-4 * float(Sph.max())
    # ionization grew the charge carriers
    assert float(npi.sum()) > float(torch.as_tensor(n0).sum())
    inf = s.info()
    assert inf["last_residual"] <= 1e-8
    s.close()
    pl.close()
