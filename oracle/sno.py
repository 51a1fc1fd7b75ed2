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
"""
import math

import numpy as np
from scipy import special


def mode_sets(n, m):
    kxy = np.concatenate([np.arange(m), np.arange(n - m, n)])
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


def spec_conv(v, Rr, Ri, n, m):
    """v: (C, n, n, n) real -> (C, n, n, n) real, by explicit truncated DFT sums."""
    kx, ky, kz = mode_sets(n, m)
    j = np.arange(n)
    Ex = np.exp(-2j * math.pi * np.outer(kx, j) / n)     # (2m, n)
    Ey = np.exp(-2j * math.pi * np.outer(ky, j) / n)
    Ez = np.exp(-2j * math.pi * np.outer(kz, j) / n)     # (m, n)
    V = np.einsum("cxyz,az->cxya", v, Ez)
    V = np.einsum("cxya,by->cxba", V, Ey)
    V = np.einsum("cxba,ex->ceba", V, Ex)                # (C, 2m, 2m, m)
    R = (Rr + 1j * Ri).reshape(2 * m, 2 * m, m, Rr.shape[1], Rr.shape[2])
    G = np.einsum("ebaoc,ceba->oeba", R, V)
    w = np.where(kz == 0, 1.0, 2.0) / n ** 3
    G = G * w[None, None, None, :]
    S = np.einsum("oeba,ex->oxba", G, np.conj(Ex))
    S = np.einsum("oxba,by->oxya", S, np.conj(Ey))
    S = np.einsum("oxya,az->oxyz", S, np.conj(Ez))
    return S.real


def forward(theta, u, C, m, L, P):
    """u: (n, n, n) -> y: (n, n, n)."""
    n = u.shape[0]
    p = unflatten(theta, C, m, L, P)
    v = p["Wl"][:, None, None, None] * u[None] + p["bl"][:, None, None, None]
    for l in range(L):
        s = spec_conv(v, p["Rr%d" % l], p["Ri%d" % l], n, m)
        z = s + np.einsum("oc,cxyz->oxyz", p["W%d" % l], v) + p["b%d" % l][:, None, None, None]
        v = gelu(z) if l < L - 1 else z
    h = gelu(np.einsum("pc,cxyz->pxyz", p["Q1"], v) + p["q1"][:, None, None, None])
    return np.einsum("p,pxyz->xyz", p["Q2"], h) + p["q2"][0]


def loss(theta, u, t, C, m, L, P):
    """Mean squared error over the batch and the grid; u, t: (B, n, n, n)."""
    return float(np.mean([(forward(theta, u[b], C, m, L, P) - t[b]) ** 2 for b in range(u.shape[0])]))
