"""Oracle of the streamer time loop (Sec. 5, Eq. (eM)): test infrastructure only.

Plain FP64 numpy / scipy restatement of the discharge model that the photoionization sum
feeds, in the paper's order:
  dn_e/dt - div(mu_e E n_e) - div(D_e grad n_e) = S_i + S_ph,
  dn_p/dt + div(mu_p E n_p) = S_i + S_ph,
  -Laplace(phi) = (e / eps0) (n_p - n_e),  E = -grad(phi),
  S_i = mu_e n_e alpha(|E|) |E|,  alpha = 5.7 p exp(-260 p / |E|) cm^-1,
with phi = 0 on the bottom face (z = 0), phi = phi0 on the top face (z = L_z), homogeneous
Neumann conditions for phi on the four side faces and for the densities on every face
(Sec. 5, below Eq. (eM)). Discretisation as the paper states it: cell-centred finite
volumes on a uniform grid of cubic cells, drift fluxes from MUSCL face values with the
Koren limiter, diffusion by central differences, a second-order explicit time integration
(Heun's method, the two-stage strong-stability-preserving Runge-Kutta scheme, so S_ph is
evaluated twice per step), and the Poisson equation solved to the discrete solution (here
by a direct sparse factorisation; the GPU uses multigrid to a relative residual of 1e-8 or
tighter). Arrays are [z][y][x] (x fastest), cell (i, j, k) centred at ((i+1/2) h, (j+1/2) h,
(k+1/2) h). S_ph is supplied by the caller as a function of the source S_i (the oracle
KIFMM or the direct sum in tests). Units: cm, s, V, Torr.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

E_OVER_EPS0 = 1.602176634e-19 / 8.8541878128e-14   # elementary charge / vacuum permittivity, V cm


def params(p=760.0, phi0=52e3, D_e=1800.0, xi_oa=0.06, p_q=30.0):
    """Sec. 5: mu_e = 2.9e5 / p, mu_p = 2.6e3 / p cm^2 / (V s), D_e = 1800 cm^2 / s,
    phi0 = 52 kV, p = 760 Torr; xi (omega / alpha) = 0.1 x 0.6 and p_q = 30 Torr for S_ph."""
    return dict(p=p, phi0=phi0, mu_e=2.9e5 / p, mu_p=2.6e3 / p, D_e=D_e, C=xi_oa * p_q / (p + p_q))


def alpha(Emag, p):
    """Townsend coefficient of Sec. 5 (Dhali and Williams): 5.7 p exp(-260 p / |E|), 0 at |E| = 0."""
    out = np.zeros_like(Emag)
    nz = Emag > 0
    out[nz] = 5.7 * p * np.exp(-260.0 * p / Emag[nz])
    return out


# ---- Poisson --------------------------------------------------------------------------
def poisson_matrix(nx, ny, nz, h):
    """A phi = b for -Laplace(phi) with the boundary terms: per cell the sum over its faces of
    (phi_c - phi_nb) / h^2; a side face (x or y boundary) contributes nothing (Neumann); a z
    boundary face contributes 2 (phi_c - phi_face) / h^2 (the face value phi_face moves to b)."""
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    diag = np.zeros((nz, ny, nx))
    for axis, m in ((2, nx), (1, ny), (0, nz)):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, m - 1)
        hi[axis] = slice(1, m)
        a, b = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [np.full(a.size, -1.0), np.full(a.size, -1.0)]
        diag[tuple(lo)] += 1.0
        diag[tuple(hi)] += 1.0
    diag[0] += 2.0      # z = 0 face (Dirichlet)
    diag[-1] += 2.0     # z = L face (Dirichlet)
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A / (h * h)


def poisson_rhs(rho, h, phi0):
    """b = rho plus the top face's Dirichlet term 2 phi0 / h^2 (the bottom face is at 0)."""
    b = np.array(rho, dtype=np.float64, copy=True)
    b[-1] += 2.0 * phi0 / (h * h)
    return b


def solve_poisson(rho, h, phi0):
    """The discrete potential for the charge term rho = (e / eps0)(n_p - n_e), [z][y][x]."""
    nz, ny, nx = rho.shape
    A = poisson_matrix(nx, ny, nz, h).tocsc()
    return spla.spsolve(A, poisson_rhs(rho, h, phi0).ravel()).reshape(nz, ny, nx)


# ---- fields ----------------------------------------------------------------------------
def face_fields(phi, h, phi0):
    """E = -grad(phi) on the faces: Ex [nz][ny][nx+1], Ey [nz][ny+1][nx], Ez [nz+1][ny][nx];
    0 on the side boundary faces (Neumann), one-sided over h/2 on the z boundary faces."""
    nz, ny, nx = phi.shape
    Ex = np.zeros((nz, ny, nx + 1))
    Ey = np.zeros((nz, ny + 1, nx))
    Ez = np.zeros((nz + 1, ny, nx))
    Ex[:, :, 1:-1] = -(phi[:, :, 1:] - phi[:, :, :-1]) / h
    Ey[:, 1:-1, :] = -(phi[:, 1:, :] - phi[:, :-1, :]) / h
    Ez[1:-1] = -(phi[1:] - phi[:-1]) / h
    Ez[0] = -(phi[0] - 0.0) / (0.5 * h)
    Ez[-1] = -(phi0 - phi[-1]) / (0.5 * h)
    return Ex, Ey, Ez


def centre_field(Ex, Ey, Ez):
    """|E| at the cell centres from the averages of each component's two faces."""
    ex = 0.5 * (Ex[:, :, 1:] + Ex[:, :, :-1])
    ey = 0.5 * (Ey[:, 1:, :] + Ey[:, :-1, :])
    ez = 0.5 * (Ez[1:] + Ez[:-1])
    return np.sqrt(ex * ex + ey * ey + ez * ez)


# ---- drift and diffusion ---------------------------------------------------------------
def koren(r):
    """Koren's limiter: max(0, min(2r, (1 + 2r) / 3, 2))."""
    return np.maximum(0.0, np.minimum(np.minimum(2.0 * r, (1.0 + 2.0 * r) / 3.0), 2.0))


def _ratio(num, den):
    """r = num / den with r = 0 where den = 0 (a flat upwind pair: first order there)."""
    out = np.zeros_like(num)
    nz = den != 0.0
    out[nz] = num[nz] / den[nz]
    return out


def muscl_faces(n, v, axis):
    """Upwind MUSCL face values with the Koren limiter along `axis` for the face velocities v
    (one more entry than cells along axis), two ghost cells per side copying the boundary cell
    (zero gradient). Positive v: n_L = n_i + phi(r) (n_{i+1} - n_i) / 2 with
    r = (n_i - n_{i-1}) / (n_{i+1} - n_i); negative v: the mirror image from cell i + 1."""
    pad = [(0, 0)] * 3
    pad[axis] = (2, 2)
    g = np.pad(n, pad, mode="edge")
    m = n.shape[axis]

    def sl(a, b):
        s = [slice(None)] * 3
        s[axis] = slice(a, b)
        return g[tuple(s)]
    # faces f = 0..m lie between padded cells f + 1 and f + 2
    um, u0, u1, u2 = sl(0, m + 1), sl(1, m + 2), sl(2, m + 3), sl(3, m + 4)
    left = u0 + 0.5 * koren(_ratio(u0 - um, u1 - u0)) * (u1 - u0)
    right = u1 + 0.5 * koren(_ratio(u1 - u2, u0 - u1)) * (u0 - u1)
    return np.where(v >= 0.0, left, right)


def divergence(Fx, Fy, Fz, h):
    return ((Fx[:, :, 1:] - Fx[:, :, :-1]) + (Fy[:, 1:, :] - Fy[:, :-1, :]) + (Fz[1:] - Fz[:-1])) / h


def diffusion_flux(n, D, h, axis):
    """-D dn/dx on the faces along axis, 0 on the boundary faces (Neumann)."""
    d = -D * np.diff(n, axis=axis) / h
    pad = [(0, 0)] * 3
    pad[axis] = (1, 1)
    return np.pad(d, pad)


def rhs(ne, npi, h, prm, sph=None):
    """Right-hand side of Eq. (eM) for the densities: returns (dne/dt, dnp/dt, aux), aux with
    phi, |E|, S_i and S_ph. sph(S_i) -> S_ph (the photoionization sum of Eq. (integral) with
    C folded in) or None for no photoionization."""
    rho = E_OVER_EPS0 * (npi - ne)
    phi = solve_poisson(rho, h, prm["phi0"])
    Ex, Ey, Ez = face_fields(phi, h, prm["phi0"])
    Emag = centre_field(Ex, Ey, Ez)
    Si = prm["mu_e"] * ne * alpha(Emag, prm["p"]) * Emag
    Sph = np.zeros_like(Si) if sph is None else np.asarray(sph(Si)).reshape(Si.shape)
    Fe, Fp = [], []
    for axis, E in ((2, Ex), (1, Ey), (0, Ez)):
        ve, vp = -prm["mu_e"] * E, prm["mu_p"] * E
        Fe.append(ve * muscl_faces(ne, ve, axis) + diffusion_flux(ne, prm["D_e"], h, axis))
        Fp.append(vp * muscl_faces(npi, vp, axis))
    dne = -divergence(*Fe, h) + Si + Sph
    dnp = -divergence(*Fp, h) + Si + Sph
    return dne, dnp, dict(phi=phi, Emag=Emag, Si=Si, Sph=Sph)


def heun_step(ne, npi, dt, h, prm, sph=None):
    """One step of Heun's method: U1 = U + dt L(U); U' = (U + U1 + dt L(U1)) / 2."""
    a1, b1, _ = rhs(ne, npi, h, prm, sph)
    ne1, np1 = ne + dt * a1, npi + dt * b1
    a2, b2, aux = rhs(ne1, np1, h, prm, sph)
    return 0.5 * (ne + ne1 + dt * a2), 0.5 * (npi + np1 + dt * b2), aux
