"""Oracle: the photoionization kernel, the exponential integral and the self-cell term.

TEST INFRASTRUCTURE ONLY. This module is part of the CPU oracle that the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of ``bench.py`` use to
check the CUDA path. The product path never imports it.

Everything here is plain FP64 numpy written from the paper:

* Zheleznyak model, Sec. 2.1, Eqs. (integral), (Ifun), (gfun): S_ph(x) is the
  convolution of I with g(r) / (4 pi r^2), where
  g(r) / p_O2 = (exp(-chi_min p_O2 r) - exp(-chi_max p_O2 r)) / (p_O2 r ln(chi_max/chi_min)).
  With a = chi_min p_O2 and b = chi_max p_O2 this is the kernel
  K(R) = (exp(-aR) - exp(-bR)) / (4 pi R^3 ln(b/a)).
* Discrete kernel G, Sec. 3, Eq. (summation): midpoint rule for i != j and a
  special value for the cell's own contribution (i == j).

Self-cell modes (Sec. 3, discrete kernel G):
* ``cell_exact``: the exact integral of K over the cell's own cube,
  sigma(h) = int_{[-h/2,h/2]^3} K(|y|) dy. Written as a solid-angle integral over
  the six faces: along each ray from the centre, int_0^rho K(r) r^2 dr =
  F(rho) / (4 pi ln(b/a)) with F(rho) = ln(b/a) + E1(b rho) - E1(a rho); the
  solid angle seen through the face z = h/2 is dOmega = (h/2) / R^3 du dv.
  The face integral has a smooth integrand and is taken with tensor
  Gauss-Legendre quadrature.
* ``paper_gl2``: the paper's value for i == j, 3 g(sqrt(sum h^2 / 12)) / (pi sum h^2),
  times the cell volume. For a cubic cell this is h^3 K(h/2): the 2-point
  Gauss-Legendre rule per axis puts all eight nodes at distance h/2.

E1 follows two published methods: the power series of Abramowitz & Stegun 5.1.11
for x <= 1 and the continued fraction of A&S 5.1.22 (evaluated with the modified
Lentz method) for x > 1.
"""
import math

import numpy as np

CHI_MIN = 0.035  # cm^-1 Torr^-1, Sec. 2.1 after Eq. (gfun)
CHI_MAX = 2.0    # cm^-1 Torr^-1, Sec. 2.1 after Eq. (gfun)
EULER_GAMMA = 0.57721566490153286060651209008240243


def absorption_coefficients(p_o2):
    """(a, b) = (chi_min p_O2, chi_max p_O2) in cm^-1, from Eq. (gfun)."""
    return CHI_MIN * p_o2, CHI_MAX * p_o2


def source_scale(p, p_q=30.0, xi_omega_alpha=0.06):
    """C = xi (omega/alpha) p_q / (p + p_q), Eq. (Ifun). Defaults: p_q = 30 Torr and
    xi omega/alpha = 0.1 * 0.6 (parameters of Sec. 4.1)."""
    return xi_omega_alpha * p_q / (p + p_q)


def kernel(R, a, b):
    """K(R) = (e^{-aR} - e^{-bR}) / (4 pi R^3 ln(b/a)), R > 0, FP64.

    Written as -e^{-aR} expm1(-(b-a)R) so that the difference keeps full precision
    when (b-a)R is small (low pressure)."""
    R = np.asarray(R, dtype=np.float64)
    num = -np.exp(-a * R) * np.expm1(-(b - a) * R)
    return num / (4.0 * math.pi * R ** 3 * math.log(b / a))


# ---- kernels of the comparison models, through the same sum (kernel independence) ----------
# Sec. 2.2, Eq. (gexp), Table Helcoeff: g(r)/p_O2 ~ p_O2 r sum_j C_j exp(-lambda_j p_O2 r), so the
# integrand g/(4 pi r^2) becomes sum_j C_j p_O2^2 exp(-lambda_j p_O2 r) / (4 pi r): the free-space
# Green's functions of the three modified Helmholtz equations, Eq. (Hel).
HELMHOLTZ3 = ((1.986e-4, 0.0553), (0.0051, 0.1460), (0.4886, 0.89))   # (C_j cm^-2 Torr^-2, lambda_j cm^-1 Torr^-1)
# Sec. 2.3, Eq. (rtetoint), Table threegroupcoeff: g(r) ~ sum_j A_j p_O2 exp(-lambda_j p_O2 r), the
# integrand sum_j A_j p_O2 exp(-lambda_j p_O2 r) / (4 pi r^2), Eq. (rteSph).
THREEGROUP = ((0.0067, 0.0447), (0.0346, 0.1121), (0.3059, 0.5994))   # (A_j cm^-1 Torr^-1, lambda_j cm^-1 Torr^-1)
KERNELS = ("zheleznyak", "helmholtz3", "threegroup")


def kernel_terms(kind, p_o2):
    """(alpha, w_j, kappa_j) with K(R) = sum_j w_j exp(-kappa_j R) / R^alpha for the comparison
    kernels at oxygen pressure p_O2 (Torr)."""
    if kind == "helmholtz3":
        return 1, [c * p_o2 ** 2 / (4.0 * math.pi) for c, _ in HELMHOLTZ3], [lam * p_o2 for _, lam in HELMHOLTZ3]
    if kind == "threegroup":
        return 2, [A * p_o2 / (4.0 * math.pi) for A, _ in THREEGROUP], [lam * p_o2 for _, lam in THREEGROUP]
    raise ValueError("unknown kernel %r" % (kind,))


def kernel_any(R, a, b, kind="zheleznyak"):
    """K(R) of the chosen model; (a, b) = (chi_min p_O2, chi_max p_O2) fix p_O2 = a / chi_min."""
    if kind == "zheleznyak":
        return kernel(R, a, b)
    alpha, w, kap = kernel_terms(kind, a / CHI_MIN)
    R = np.asarray(R, dtype=np.float64)
    return sum(wj * np.exp(-kj * R) for wj, kj in zip(w, kap)) / R ** alpha


def mass_within(rho, a, b, kind="zheleznyak"):
    """int_0^rho K(r) r^2 dr (the flux through a sphere of radius rho, divided by 4 pi)."""
    if kind == "zheleznyak":
        return (math.log(b / a) + expint_e1(b * rho) - expint_e1(a * rho)) / (4.0 * math.pi * math.log(b / a))
    alpha, w, kap = kernel_terms(kind, a / CHI_MIN)
    s = 0.0
    for wj, kj in zip(w, kap):
        x = kj * rho
        if alpha == 1:    # int_0^rho r e^{-k r} dr = (1 - (1 + x) e^{-x}) / k^2
            s += wj * (-math.expm1(-x) - x * math.exp(-x)) / kj ** 2
        else:             # int_0^rho e^{-k r} dr = (1 - e^{-x}) / k
            s += wj * (-math.expm1(-x)) / kj
    return s


def sigma_cell_any(hx, hy, hz, a, b, kind="zheleznyak", mode="cell_exact", nodes=64):
    """sigma of a cell hx x hy x hz for any of the kernels: cell_exact by the face-flux form
    sum over the face pairs of 2 int (h_k/2) / R^3 m(R) du dv, m = ``mass_within`` (as
    ``sigma_box_exact``); paper_gl2: hx hy hz K(rho), rho = sqrt(sum h^2 / 12) (the 2-point
    Gauss-Legendre nodes), which for the paper's kernel is ``sigma_box_paper_gl2``."""
    if mode == "paper_gl2":
        rho = math.sqrt((hx * hx + hy * hy + hz * hz) / 12.0)
        return hx * hy * hz * float(kernel_any(rho, a, b, kind))
    t, wgl = np.polynomial.legendre.leggauss(nodes)
    hs = (float(hx), float(hy), float(hz))
    total = 0.0
    for k in range(3):
        hk = hs[k]
        hi, hj = [hs[m] for m in range(3) if m != k]
        u, wu = 0.5 * hi * t, 0.5 * hi * wgl
        v, wv = 0.5 * hj * t, 0.5 * hj * wgl
        for i in range(nodes):
            for j in range(nodes):
                R = math.sqrt(u[i] * u[i] + v[j] * v[j] + 0.25 * hk * hk)
                total += 2.0 * wu[i] * wv[j] * (0.5 * hk) / R ** 3 * mass_within(R, a, b, kind)
    return total


def g_over_po2(r, p_o2):
    """g(r) / p_O2 of Eq. (gfun), as printed (used by the pins, not by the sums)."""
    x = p_o2 * r
    return (np.exp(-CHI_MIN * x) - np.exp(-CHI_MAX * x)) / (x * math.log(CHI_MAX / CHI_MIN))


def expint_e1(x):
    """Exponential integral E1(x), x > 0 (scalar).

    x <= 1: A&S 5.1.11, E1(x) = -gamma - ln x - sum_{n>=1} (-x)^n / (n n!).
    x  > 1: A&S 5.1.22, E1(x) = e^{-x} / (x + 1/(1 + 1/(x + 2/(1 + 2/(x + ...))))),
            evaluated in the equivalent even form
            e^{-x} * 1/(x+1- 1^2/(x+3- 2^2/(x+5- ...))) with the modified Lentz method.
    """
    x = float(x)
    if not x > 0.0:
        raise ValueError("E1 needs x > 0")
    if x <= 1.0:
        s = 0.0
        term = 1.0
        n = 1
        while True:
            term *= -x / n           # (-x)^n / n!
            add = -term / n          # -(-x)^n / (n n!)
            s += add
            if abs(add) < 1e-18 * max(1.0, abs(s)):
                break
            n += 1
        return -EULER_GAMMA - math.log(x) + s
    tiny = 1e-300
    bq = x + 1.0
    c = 1.0 / tiny
    d = 1.0 / bq
    h = d
    i = 1
    while True:
        an = -float(i * i)
        bq += 2.0
        d = 1.0 / (an * d + bq)
        c = bq + an / c
        delta = c * d
        h *= delta
        if abs(delta - 1.0) < 1e-16:
            break
        i += 1
        if i > 10000:
            raise RuntimeError("E1 continued fraction did not converge")
    return h * math.exp(-x)


def radial_mass(rho, a, b):
    """F(rho) / ln(b/a): the fraction of the kernel's mass within distance rho,
    with F(rho) = ln(b/a) + E1(b rho) - E1(a rho) (integral of (e^{-ar}-e^{-br})/r)."""
    return (math.log(b / a) + expint_e1(b * rho) - expint_e1(a * rho)) / math.log(b / a)


def sigma_cell_exact(h, a, b, nodes=64):
    """Exact integral of K over a cube of side h centred on the singularity.

    sigma = 6 * int_{[-h/2,h/2]^2} (h/2) / R^3 * F(R) du dv / (4 pi ln(b/a)),
    R = sqrt(u^2 + v^2 + h^2/4), by tensor Gauss-Legendre with ``nodes`` points
    per axis."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    u = 0.5 * h * t
    wu = 0.5 * h * w
    total = 0.0
    for i in range(nodes):
        for j in range(nodes):
            R = math.sqrt(u[i] * u[i] + u[j] * u[j] + 0.25 * h * h)
            F = math.log(b / a) + expint_e1(b * R) - expint_e1(a * R)
            total += wu[i] * wu[j] * (0.5 * h) / R ** 3 * F
    return 6.0 * total / (4.0 * math.pi * math.log(b / a))


def sigma_paper_gl2(h, a, b):
    """The paper's i == j value times the cell volume: h^3 * 3 g(rho)/(pi * 3 h^2),
    rho = sqrt(3 h^2 / 12) = h/2, i.e. h^3 K(h/2) for a cubic cell."""
    s2 = 3.0 * h * h
    rho = math.sqrt(s2 / 12.0)
    g = (math.exp(-a * rho) - math.exp(-b * rho)) / (rho * math.log(b / a))
    return h ** 3 * 3.0 * g / (math.pi * s2)


def sigma_box_exact(hx, hy, hz, a, b, nodes=64):
    """Exact integral of K over a rectangular cell hx x hy x hz centred on the singularity
    (the cells of the Sec. 4.2 grid are not cubic). The same solid-angle form as
    ``sigma_cell_exact``, face by face: the pair of faces normal to axis k (half-width
    h_k / 2) contributes 2 int (h_k/2) / R^3 F(R) du dv over the other two half-widths,
    R = sqrt(u^2 + v^2 + h_k^2 / 4)."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    hs = (float(hx), float(hy), float(hz))
    lnba = math.log(b / a)
    total = 0.0
    for k in range(3):
        hk = hs[k]
        hi, hj = [hs[m] for m in range(3) if m != k]
        u, wu = 0.5 * hi * t, 0.5 * hi * w
        v, wv = 0.5 * hj * t, 0.5 * hj * w
        U, V = np.meshgrid(u, v, indexing="ij")
        R = np.sqrt(U * U + V * V + 0.25 * hk * hk)
        F = lnba + np.vectorize(expint_e1)(b * R) - np.vectorize(expint_e1)(a * R)
        total += 2.0 * float(np.sum(np.outer(wu, wv) * (0.5 * hk) / R ** 3 * F))
    return total / (4.0 * math.pi * lnba)


def sigma_box_paper_gl2(hx, hy, hz, a, b):
    """The paper's i == j value for a rectangular cell times its volume:
    hx hy hz * 3 g(rho) / (pi sum h^2), rho = sqrt(sum h^2 / 12) (Sec. 3, discrete G)."""
    s2 = hx * hx + hy * hy + hz * hz
    rho = math.sqrt(s2 / 12.0)
    g = (math.exp(-a * rho) - math.exp(-b * rho)) / (rho * math.log(b / a))
    return hx * hy * hz * 3.0 * g / (math.pi * s2)


SELF_MODES = ("cell_exact", "paper_gl2")


def self_sigma(h, a, b, mode):
    """sigma(h) for the chosen self-cell mode."""
    if mode == "cell_exact":
        return sigma_cell_exact(h, a, b)
    if mode == "paper_gl2":
        return sigma_paper_gl2(h, a, b)
    raise ValueError("unknown self mode %r" % (mode,))
