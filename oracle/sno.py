"""Oracle: the spectral neural operator surrogate, forward pass in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (checks the CUDA forward pass and, by finite differences of
this forward pass, the CUDA gradients; never imported by the product path).

The paper has no learned component: this network stands in for the photoionization
solve inside a time loop, with the FMM as fallback and judge. Definition (grid n^3,
width C, m modes per axis, L layers, projection width P):

    v_0(c)   = Wl[c] u + bl[c]                                     (lift, u = log(1 + I))
    s_l      = SpecConv_l(v_l)
    z_l      = s_l + W_l v_l + b_l
    v_{l+1}  = GELU(z_l)  (l < L-1),   v_L = z_{L-1}
    y        = Q2 . GELU(Q1 v_L + q1) + q2                           (target log(1 + S))

    SpecConv(v)(o, x) = (1/n^3) sum_{k in K} w_kz Re[ G(o, k) e^{+2 pi i k.x / n} ],
    G(o, k) = sum_c R(k)[o][c] V(c, k),   V(c, k) = sum_x v(c, x) e^{-2 pi i k.x / n},

with K = Kx x Ky x Kz, Kx = Ky = {0..m-1} U {n-m..n-1}, Kz = {0..m-1}, w_0 = 1 and
w_kz = 2 for kz >= 1 (the conjugate half of the z spectrum). GELU(x) = x (1 + erf(x/sqrt 2))/2.

Period. The transforms may take a period N >= n in place of n (n replaced by N in the
exponentials, the mode sets and the 1/n^3 factor): the grid is then the first n points of
an N-periodic grid whose other points hold zeros, so that the spectral convolution is not
periodic on the n-point grid itself (the photoionization sum is a linear convolution).

Near field. The map I -> S_ph is linear (Sec. 3, Eq. (summation)). With the amplitude
scale s = max I, u = I / s and the target t = S / (C s), the model may add an exact near
part to y: for cubic cells of edge h on the grid,

    near(u)(x) = sigma u(x) + sum_{0 < |d| <= r_out} K(h |d|) w(|d|) h^3 u(x + d),

w = 1 for |d| <= r_in, cos^2(pi/2 (|d| - r_in)/(r_out - r_in)) up to r_out, 0 beyond (|d|
in cells, u = 0 outside the grid), sigma the self-cell value. The rest of the sum is the far
part, the linear convolution with K (1 - w) h^3, whose Fourier multiplier on the N-periodic
grid (``far_multiplier``) is what a spectral layer can carry (``far_init``).
"""
import math

import numpy as np
from scipy import special

from . import kernel as _k


def mode_sets(n, m, period=None):
    N = n if period is None else int(period)
    kxy = np.concatenate([np.arange(m), np.arange(N - m, N)])
    kz = np.arange(m)
    return kxy, kxy.copy(), kz


def param_layout(C, m, L, P):
    """Names and shapes in the flat parameter order shared with the CUDA module's
    sno_set_params / sno_get_params (FP32 flat vector)."""
    K = (2 * m) * (2 * m) * m
    lay = [("Wl", (C,)), ("bl", (C,))]
    for l in range(L):
        lay += [("Rr%d" % l, (K, C, C)), ("Ri%d" % l, (K, C, C)), ("W%d" % l, (C, C)), ("b%d" % l, (C,))]
    lay += [("Q1", (P, C)), ("q1", (P,)), ("Q2", (P,)), ("q2", (1,))]
    return lay


def unflatten(theta, C, m, L, P):
    out, o = {}, 0
    for name, shp in param_layout(C, m, L, P):
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def gelu(x):
    return 0.5 * x * (1.0 + special.erf(x / math.sqrt(2.0)))


def spec_conv(v, Rr, Ri, n, m, period=None):
    """v: (C, n, n, n) real -> (C, n, n, n) real, by explicit truncated DFT sums (period N:
    the exponentials, mode sets and 1/N^3 of the N-periodic grid)."""
    N = n if period is None else int(period)
    kx, ky, kz = mode_sets(n, m, N)
    j = np.arange(n)
    Ex = np.exp(-2j * math.pi * np.outer(kx, j) / N)     # (2m, n)
    Ey = np.exp(-2j * math.pi * np.outer(ky, j) / N)
    Ez = np.exp(-2j * math.pi * np.outer(kz, j) / N)     # (m, n)
    V = np.einsum("cxyz,az->cxya", v, Ez)
    V = np.einsum("cxya,by->cxba", V, Ey)
    V = np.einsum("cxba,ex->ceba", V, Ex)                # (C, 2m, 2m, m)
    R = (Rr + 1j * Ri).reshape(2 * m, 2 * m, m, Rr.shape[1], Rr.shape[2])
    G = np.einsum("ebaoc,ceba->oeba", R, V)
    w = np.where(kz == 0, 1.0, 2.0) / float(N) ** 3
    G = G * w[None, None, None, :]
    S = np.einsum("oeba,ex->oxba", G, np.conj(Ex))
    S = np.einsum("oxba,by->oxya", S, np.conj(Ey))
    S = np.einsum("oxya,az->oxyz", S, np.conj(Ez))
    return S.real


def window(rho, r_in, r_out):
    """w(rho): 1 up to r_in, cos^2 taper to 0 at r_out, 0 beyond (rho in cells)."""
    rho = np.asarray(rho, dtype=np.float64)
    t = np.clip((rho - r_in) / (r_out - r_in), 0.0, 1.0)
    return np.where(rho <= r_in, 1.0, np.where(rho >= r_out, 0.0, np.cos(0.5 * math.pi * t) ** 2))


def near_field(u, a, b, h, sigma, r_in, r_out):
    """sigma u(x) + sum_{0 < |d| <= r_out} K(h |d|) w(|d|) h^3 u(x + d), offset by offset
    (u = 0 outside the grid)."""
    u = np.asarray(u, dtype=np.float64)
    n0, n1, n2 = u.shape
    out = sigma * u
    R = int(math.floor(r_out))
    for dz in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                rho = math.sqrt(dx * dx + dy * dy + dz * dz)
                if rho == 0.0 or rho >= r_out:
                    continue
                wgt = float(_k.kernel(h * rho, a, b)) * float(window(rho, r_in, r_out)) * h ** 3
                src = u[max(0, dx):n0 + min(0, dx), max(0, dy):n1 + min(0, dy), max(0, dz):n2 + min(0, dz)]
                out[max(0, -dx):n0 + min(0, -dx), max(0, -dy):n1 + min(0, -dy), max(0, -dz):n2 + min(0, -dz)] += \
                    wgt * src
    return out


def far_table(N, a, b, h, r_in, r_out):
    """K(h |d|) (1 - w(|d|)) h^3 on the N-periodic grid, d the minimum-image offset (0 at d = 0)."""
    g = np.fft.fftfreq(N, 1.0 / N)
    d0, d1, d2 = np.meshgrid(g, g, g, indexing="ij")
    rho = np.sqrt(d0 ** 2 + d1 ** 2 + d2 ** 2)
    rho[0, 0, 0] = 1.0
    t = _k.kernel(h * rho, a, b) * (1.0 - window(rho, r_in, r_out)) * h ** 3
    t[0, 0, 0] = 0.0
    return t


def far_multiplier(m, N, a, b, h, r_in, r_out):
    """The far table's DFT (real: the table is even in every axis) at the retained modes,
    flattened in the spectral weights' mode order k = (kx_index 2m + ky_index) m + kz."""
    F = np.fft.fftn(far_table(N, a, b, h, r_in, r_out))
    kx, ky, kz = mode_sets(N, m, N)
    return F[np.ix_(kx, ky, kz)].real.reshape(-1)


def far_init(C, m, L, P, mult, sigma_w=0.0, shift=8.0):
    """Parameters whose output is the truncated far convolution of u: channel 0 carries
    mult on layer 0's spectral weights and passes unchanged through the later layers
    (shift keeps GELU in its linear range: GELU(shift + x) = shift + x to 1e-12 for
    |x| <= 2); every other parameter is 0. sigma_w adds sigma_w u through layer 0's
    pointwise weight (the self term, when no near part is added)."""
    p = {name: np.zeros(shp) for name, shp in param_layout(C, m, L, P)}
    p["Wl"][0] = 1.0
    p["Rr0"][:, 0, 0] = mult
    p["W0"][0, 0] = sigma_w
    p["b0"][0] = shift
    for l in range(1, L):
        p["W%d" % l][0, 0] = 1.0
    p["Q1"][0, 0] = 1.0
    p["Q2"][0] = 1.0
    p["q2"][0] = -shift
    return np.concatenate([p[name].ravel() for name, _ in param_layout(C, m, L, P)])


def forward(theta, u, C, m, L, P, period=None, near=None):
    """u: (n, n, n) -> y: (n, n, n). near: None, or a dict with a, b, h, sigma, r_in,
    r_out, whose near part is added to the network's output."""
    n = u.shape[0]
    p = unflatten(theta, C, m, L, P)
    v = p["Wl"][:, None, None, None] * u[None] + p["bl"][:, None, None, None]
    for l in range(L):
        s = spec_conv(v, p["Rr%d" % l], p["Ri%d" % l], n, m, period)
        z = s + np.einsum("oc,cxyz->oxyz", p["W%d" % l], v) + p["b%d" % l][:, None, None, None]
        v = gelu(z) if l < L - 1 else z
    h = gelu(np.einsum("pc,cxyz->pxyz", p["Q1"], v) + p["q1"][:, None, None, None])
    y = np.einsum("p,pxyz->xyz", p["Q2"], h) + p["q2"][0]
    if near is not None:
        y = y + near_field(u, near["a"], near["b"], near["h"], near["sigma"], near["r_in"], near["r_out"])
    return y


def loss(theta, u, t, C, m, L, P, period=None, near=None):
    """Mean squared error over the batch and the grid; u, t: (B, n, n, n)."""
    return float(np.mean([(forward(theta, u[b], C, m, L, P, period, near) - t[b]) ** 2
                          for b in range(u.shape[0])]))
