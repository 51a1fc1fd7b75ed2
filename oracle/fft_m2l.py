"""Oracle: the M2L translation of Eq. (m2l) evaluated by FFT, in FP64.

TEST INFRASTRUCTURE ONLY (the CPU oracle; never imported by the product path).

Sec. 3 remarks after Eq. (m2l) that, since the source box A and the target box B have the same
size, the translation can be sped up by the fast Fourier transform (as in the cited KIFMM).
The reason is the surfaces' structure: both the upward equivalent surface of A and the
downward check surface of B are the boundary points of an m0 x m0 x m0 lattice of spacing
delta = 2 r_in r / (m0 - 1) (half-width r, radius r_in in half-widths), so with integer lattice
coordinates g in {0..m0-1}^3,

    x_i - y_j = delta (g_i - g_j) - (c_A - c_B),

and the translation q^{B,d}_i = sum_j K(|x_i - y_j|) phi^{A,u}_j is a linear convolution of
the densities, placed on the full lattice with zeros inside, with the tensor
K_t[u] = K(|delta u - (c_A - c_B)|), u in {-(m0-1)..m0-1}^3. Zero-padded to N = 2 m0 points
per axis, a circular convolution of that length has no wrap-around on the output lattice, so

    q^{B,d} = sample_g IFFT( sum_{A in V(B)} FFT(K_t[c_A - c_B]) * FFT(Phi_A) ),

one forward transform per source box, one kernel transform per offset (and level), the
products summed in frequency space over the V list, one inverse transform per target box.
This module states that computation directly (numpy's real FFT as the library step); the
dense oracle (`kifmm.Operators.m2l`) is the definition it must reproduce.
"""
import numpy as np

from . import kifmm as _kf


def lattice_coords(m0):
    """Integer coordinates of the surface points of `kifmm.surface_lattice(m0)`, same order."""
    s = _kf.surface_lattice(m0)
    return np.rint((s + 1.0) * (m0 - 1) / 2.0).astype(np.int64)


def embed(phi, g, m0):
    """Densities on the surface points placed on the N^3 grid (N = 2 m0), zeros elsewhere."""
    n = 2 * m0
    grid = np.zeros((n, n, n))
    grid[g[:, 2], g[:, 1], g[:, 0]] = phi   # [z][y][x]
    return grid


def kernel_tensor(off, delta, m0, a, b, kind="zheleznyak"):
    """K(|delta u - off|) for u in {-(m0-1)..m0-1}^3, stored at u mod N (N = 2 m0); the
    entry u = m0 (mod N) is never reached by the output lattice and stays 0."""
    n = 2 * m0
    u = np.arange(-(m0 - 1), m0)
    uz, uy, ux = np.meshgrid(u, u, u, indexing="ij")
    d = np.stack([delta * ux - off[0], delta * uy - off[1], delta * uz - off[2]], axis=-1)
    kt = np.zeros((n, n, n))
    kt[uz % n, uy % n, ux % n] = _kf.kmat(d.reshape(-1, 3), np.zeros((1, 3)), a, b, kind).reshape(uz.shape)
    return kt


def m2l_fft(ops, lev, sources, r, a, b):
    """q^{B,d} of one target box at level lev from its V-list sources [(offset d, phi^{A,u})],
    d = anchor(A) - anchor(B): the frequency-space sum of the per-source products, then one
    inverse transform, sampled on the check-surface points."""
    m0 = _m0_of(ops)
    g = lattice_coords(m0)
    delta = 2.0 * ops.r_in * r / (m0 - 1)
    acc = None
    for d, phi in sources:
        off = 2.0 * r * np.asarray(d, dtype=np.float64)
        prod = np.fft.rfftn(kernel_tensor(off, delta, m0, a, b, ops.kind)) * np.fft.rfftn(embed(phi, g, m0))
        acc = prod if acc is None else acc + prod
    conv = np.fft.irfftn(acc, s=(2 * m0,) * 3, axes=(0, 1, 2))
    return conv[g[:, 2], g[:, 1], g[:, 0]]


def m2l_level_fft(ops, lev, r, boxes, vlists, anchors, phi_u, a, b):
    """The V-list sums q^{B,d} of every box B in `boxes` (one level, half-width r), each from
    the boxes A of vlists[B]: one forward transform per source box and one kernel transform
    per offset, the products summed in frequency space, one inverse transform per target."""
    m0 = _m0_of(ops)
    g = lattice_coords(m0)
    delta = 2.0 * ops.r_in * r / (m0 - 1)
    ker, src = {}, {}
    out = np.zeros((len(boxes), ops.S))
    for row, B in enumerate(boxes):
        acc = None
        for A in vlists[B]:
            d = tuple(int(v) for v in anchors[A] - anchors[B])
            if d not in ker:
                ker[d] = np.fft.rfftn(kernel_tensor(2.0 * r * np.asarray(d, dtype=np.float64), delta, m0, a, b,
                                                    ops.kind))
            if A not in src:
                src[A] = np.fft.rfftn(embed(phi_u[A], g, m0))
            prod = ker[d] * src[A]
            acc = prod if acc is None else acc + prod
        if acc is not None:
            out[row] = np.fft.irfftn(acc, s=(2 * m0,) * 3, axes=(0, 1, 2))[g[:, 2], g[:, 1], g[:, 0]]
    return out


def _m0_of(ops):
    """m0 from the surface point count S = m0^3 - (m0 - 2)^3."""
    for m0 in range(2, 64):
        if m0 ** 3 - max(m0 - 2, 0) ** 3 == ops.S:
            return m0
    raise ValueError("not a surface lattice")


def flops_per_pair(m0, rank):
    """Work of one V pair: the frequency-space product of the real FFT (N^2 (N/2 + 1) complex
    multiply-adds, 8 flop each, N = 2 m0) against the dense product in the rank-r basis
    (2 r^2 flop)."""
    n = 2 * m0
    return {"fft": 8.0 * n * n * (n // 2 + 1), "dense_rank": 2.0 * rank * rank}
