"""Pins of the streamer oracle (Sec. 5, Eq. (eM)) against closed forms and invariants (CPU).

* Poisson: with no charge the discrete potential is the linear profile phi0 z / L_z (the
  cell-centred scheme with the electrodes' face values is exact on it); products of the
  discrete Neumann eigenvectors cos(pi m (i + 1/2) / n) along x and y and the discrete
  Dirichlet eigenvectors sin(pi m (k + 1/2) / n) along z are eigenvectors of the assembled
  matrix with eigenvalue sum_axis (2 - 2 cos(pi m / n)) / h^2 (a wrong boundary row fails).
* Koren's limiter at its break points; MUSCL face values exact on a linear profile in the
  interior (limiter 1 at r = 1) and first order (the upwind cell) at an extremum.
* Fields: a uniform charge-free gap gives |E| = phi0 / L_z everywhere.
* Transport: with phi0 = 0 and no charge the electrons only diffuse, and the total number
  is conserved to rounding (no flux through any face); the ions do not move.
* Heun's method: equal uniform densities in the uniform field of a charge-free gap grow in
  the interior cells as dn/dt = nu n, nu = mu_e alpha(|E|) |E| (the drift fluxes cancel
  there), and the step is the scheme's combination of its two stages; one step multiplies
  the interior density by the Taylor factor 1 + nu dt + (nu dt)^2 / 2 (to 1e-6: the small
  space charge the electrodes' fluxes leave).
"""
import numpy as np
import pytest

from oracle import streamer as SD


def test_poisson_linear_profile_exact():
    nx, ny, nz, h, phi0 = 4, 5, 8, 0.1, 1234.0
    phi = SD.solve_poisson(np.zeros((nz, ny, nx)), h, phi0)
    z = (np.arange(nz) + 0.5) * h
    want = np.broadcast_to((phi0 * z / (nz * h))[:, None, None], phi.shape)
    assert np.allclose(phi, want, rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("mx,my,mz", [(0, 0, 1), (1, 0, 1), (2, 3, 2), (1, 1, 4)])
def test_poisson_matrix_discrete_eigenvectors(mx, my, mz):
    nx, ny, nz, h = 6, 5, 7, 0.05
    A = SD.poisson_matrix(nx, ny, nz, h)
    cx = np.cos(np.pi * mx * (np.arange(nx) + 0.5) / nx)
    cy = np.cos(np.pi * my * (np.arange(ny) + 0.5) / ny)
    sz = np.sin(np.pi * mz * (np.arange(nz) + 0.5) / nz)
    v = (sz[:, None, None] * cy[None, :, None] * cx[None, None, :]).ravel()
    lam = sum(2.0 - 2.0 * np.cos(np.pi * m / n) for m, n in ((mx, nx), (my, ny))) / h ** 2
    # the Dirichlet z direction: the ghost reflection u_{-1} = -u_0 makes sin((k+1/2) theta) exact
    lam += (2.0 - 2.0 * np.cos(np.pi * mz / nz)) / h ** 2
    assert np.allclose(A @ v, lam * v, rtol=1e-10, atol=1e-8 * lam)


def test_koren_break_points():
    r = np.array([-1.0, 0.0, 0.125, 0.25, 1.0, 2.5, 10.0])
    assert np.allclose(SD.koren(r), [0.0, 0.0, 0.25, 0.5, 1.0, 2.0, 2.0])


def test_muscl_linear_profile_and_extremum():
    n = (3.0 + 0.5 * np.arange(8))[None, None, :].repeat(2, 0).repeat(2, 1)
    v = np.ones((2, 2, 9))
    f = SD.muscl_faces(n, v, 2)
    # interior faces 2..6 (two cells on each side inside): the exact midpoint values
    assert np.allclose(f[..., 2:7], 3.0 + 0.5 * (np.arange(2, 7) - 0.5))
    vneg = -v
    g = SD.muscl_faces(n, vneg, 2)
    assert np.allclose(g[..., 2:7], 3.0 + 0.5 * (np.arange(2, 7) - 0.5))
    # a peak: the limiter falls to 0 and the face takes the upwind cell's value
    peak = np.array([1.0, 2.0, 5.0, 2.0, 1.0])[None, None, :]
    fp = SD.muscl_faces(peak, np.ones((1, 1, 6)), 2)
    assert fp[0, 0, 3] == 5.0


def test_uniform_gap_field():
    nx, ny, nz, h, phi0 = 3, 3, 10, 0.02, 5000.0
    phi = SD.solve_poisson(np.zeros((nz, ny, nx)), h, phi0)
    E = SD.centre_field(*SD.face_fields(phi, h, phi0))
    assert np.allclose(E, phi0 / (nz * h), rtol=1e-12)


def test_diffusion_conserves_and_ions_stay():
    rng = np.random.default_rng(3)
    nz, ny, nx, h = 6, 5, 4, 0.01
    ne = rng.uniform(1e10, 1e12, (nz, ny, nx))
    prm = SD.params(phi0=0.0)
    dne, dnp, aux = SD.rhs(ne, ne.copy(), h, prm)   # no charge: n_p = n_e
    assert np.all(aux["Emag"] == 0.0) and np.all(aux["Si"] == 0.0)
    assert abs(dne.sum()) <= 1e-12 * np.abs(dne).sum()
    assert np.all(dnp == 0.0)
    # the diffusion of a profile along z alone: the 1-D second difference with no-flux ends
    prof = np.linspace(1.0, 2.0, nz) ** 2
    ne1 = np.broadcast_to(prof[:, None, None], (nz, ny, nx)).copy()
    d1, _, _ = SD.rhs(ne1, ne1.copy(), h, prm)
    lap = np.zeros(nz)
    lap[1:-1] = prof[2:] - 2 * prof[1:-1] + prof[:-2]
    lap[0] = prof[1] - prof[0]
    lap[-1] = prof[-2] - prof[-1]
    assert np.allclose(d1[:, 1, 1], prm["D_e"] * lap / h ** 2, rtol=1e-12)


def test_heun_growth_in_a_uniform_field():
    nz, ny, nx, h = 12, 3, 3, 0.01
    prm = SD.params(phi0=4e4)
    n0 = 1e8   # (the space charge left by the electrodes' fluxes stays small at this density)
    ne = np.full((nz, ny, nx), n0)
    npi = ne.copy()   # no net charge: phi stays linear, |E| = phi0 / L
    E = prm["phi0"] / (nz * h)
    nu = prm["mu_e"] * SD.alpha(np.array([E]), prm["p"])[0] * E
    dt = 0.05 / nu
    ne1, np1, _ = SD.heun_step(ne, npi, dt, h, prm)
    # away from the electrodes the drift fluxes cancel: the first stage's right-hand side is nu n
    a1, b1, _ = SD.rhs(ne, npi, h, prm)
    mid = slice(3, nz - 3)
    assert np.allclose(a1[mid], nu * n0, rtol=1e-10) and np.allclose(b1[mid], nu * n0, rtol=1e-10)
    u1e, u1p = ne + dt * a1, npi + dt * b1
    a2, b2, _ = SD.rhs(u1e, u1p, h, prm)
    assert np.allclose(ne1, 0.5 * (ne + u1e + dt * a2), rtol=1e-14)
    assert np.allclose(np1, 0.5 * (npi + u1p + dt * b2), rtol=1e-14)
    # with n_e = n_p after stage one in the interior the growth is the Taylor factor to 2nd order
    assert np.allclose(ne1[5:7, 1, 1], n0 * (1 + nu * dt + 0.5 * (nu * dt) ** 2), rtol=1e-6)
