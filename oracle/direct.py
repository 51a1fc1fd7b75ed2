"""Oracle: the discrete photoionization sum, by direct summation and, on uniform
grids, by FFT linear convolution.

TEST INFRASTRUCTURE ONLY (the CPU oracle; never imported by the product path).

Sec. 3, Eq. (summation) with the discrete kernel G: with cell centres x_i, cubic
cells of edge h_i and weights q_j = I_j h_j^3 (the source multiplied by the cell
volume),

    S_i = C * ( sum_{j != i} K(|x_i - x_j|) q_j  +  sigma(h_i) I_i ),

C = xi (omega/alpha) p_q/(p + p_q) from Eq. (Ifun) and sigma the self-cell value
(``kernel.self_sigma``). The midpoint rule is used for every i != j, cells of
different sizes included.
"""
import ctypes
import math
import os

import numpy as np

from . import kernel as _k

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def _load_c():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_direct_sum.restype = None
        lib.oracle_direct_sum.argtypes = [
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def c_threads():
    return int(_load_c().oracle_threads())


def self_terms(h, a, b, mode, kind="zheleznyak"):
    """sigma(h_i) for every point (computed once per distinct h); ``kind`` selects one of the
    comparison kernels (``kernel.KERNELS``)."""
    h = np.asarray(h, dtype=np.float64)
    out = np.empty_like(h)
    for hv in np.unique(h):
        out[h == hv] = (_k.self_sigma(float(hv), a, b, mode) if kind == "zheleznyak"
                        else _k.sigma_cell_any(float(hv), float(hv), float(hv), a, b, kind, mode))
    return out


def pair_sum_numpy(targets, t_idx, sources, s_idx, q, a, b, kind="zheleznyak"):
    """sum_{j != i} K(|x_i - y_j|) q_j for the given targets, numpy, chunked."""
    out = np.zeros(targets.shape[0], dtype=np.float64)
    chunk = max(1, 4_000_000 // max(1, sources.shape[0]))
    for s in range(0, targets.shape[0], chunk):
        x = targets[s:s + chunk]
        d = np.sqrt(((x[:, None, :] - sources[None, :, :]) ** 2).sum(-1))
        same = t_idx[s:s + chunk, None] == s_idx[None, :]
        d[same] = 1.0
        kk = _k.kernel_any(d, a, b, kind)
        kk[same] = 0.0
        out[s:s + chunk] = kk @ q
    return out


def pair_sum_c(targets, t_idx, sources, s_idx, q, a, b):
    """The same sum in plain C with OpenMP over targets (liboracle.so)."""
    lib = _load_c()
    targets = np.ascontiguousarray(targets, dtype=np.float64)
    sources = np.ascontiguousarray(sources, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    t_idx = np.ascontiguousarray(t_idx, dtype=np.int64)
    s_idx = np.ascontiguousarray(s_idx, dtype=np.int64)
    out = np.zeros(targets.shape[0], dtype=np.float64)
    lib.oracle_direct_sum(targets.shape[0], targets.ctypes.data, t_idx.ctypes.data,
                          sources.shape[0], sources.ctypes.data, s_idx.ctypes.data, q.ctypes.data,
                          float(a), float(b), out.ctypes.data)
    return out


def direct_sum(points, h, I, a, b, C=1.0, mode="cell_exact", targets=None, impl="c", kind="zheleznyak"):
    """S at ``targets`` (indices into points; all points when None); the comparison kernels
    (``kind``) take the numpy pair sum."""
    points = np.asarray(points, dtype=np.float64)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (points.shape[0],)).copy()
    I = np.asarray(I, dtype=np.float64)
    q = I * h ** 3
    tix = np.arange(points.shape[0]) if targets is None else np.asarray(targets, dtype=np.int64)
    sidx = np.arange(points.shape[0], dtype=np.int64)
    if kind == "zheleznyak" and impl == "c":
        far = pair_sum_c(points[tix], tix, points, sidx, q, a, b)
    else:
        far = pair_sum_numpy(points[tix], tix, points, sidx, q, a, b, kind)
    sig = self_terms(h[tix], a, b, mode, kind)
    return C * (far + sig * I[tix])


def brute_force(points, h, I, a, b, C=1.0, mode="cell_exact"):
    """Pure-Python double loop over (i, j), for tiny inputs only."""
    n = len(points)
    out = []
    for i in range(n):
        s = 0.0
        for j in range(n):
            if j == i:
                continue
            d = math.sqrt(sum((points[i][k] - points[j][k]) ** 2 for k in range(3)))
            kij = (math.exp(-a * d) - math.exp(-b * d)) / (4 * math.pi * d ** 3 * math.log(b / a))
            s += kij * I[j] * h[j] ** 3
        s += _k.self_sigma(h[i], a, b, mode) * I[i]
        out.append(C * s)
    return np.array(out)


def fft_uniform(I3, hgrid, a, b, C=1.0, mode="cell_exact", kind="zheleznyak"):
    """Uniform grid (n0, n1, n2) of cubic cells of edge ``hgrid``: the same sum as a
    linear convolution with the kernel table K(h |d|) (zero at d = 0), zero-padded
    to twice the grid so that nothing wraps around."""
    I3 = np.asarray(I3, dtype=np.float64)
    n = I3.shape
    q = I3 * hgrid ** 3
    grids = [np.arange(-(m - 1), m) for m in n]
    dz, dy, dx = np.meshgrid(*grids, indexing="ij")
    R = hgrid * np.sqrt(dx.astype(np.float64) ** 2 + dy ** 2 + dz ** 2)
    R[n[0] - 1, n[1] - 1, n[2] - 1] = 1.0
    tab = _k.kernel_any(R, a, b, kind)
    tab[n[0] - 1, n[1] - 1, n[2] - 1] = 0.0
    shape = [2 * m for m in n]
    ax = (0, 1, 2)
    F = np.fft.rfftn(q, shape, axes=ax) * np.fft.rfftn(tab, shape, axes=ax)
    conv = np.fft.irfftn(F, shape, axes=ax)
    far = conv[n[0] - 1:2 * n[0] - 1, n[1] - 1:2 * n[1] - 1, n[2] - 1:2 * n[2] - 1]
    sig = (_k.self_sigma(hgrid, a, b, mode) if kind == "zheleznyak"
           else _k.sigma_cell_any(hgrid, hgrid, hgrid, a, b, kind, mode))
    return C * (far + sig * I3)


def fft_box_grid(I3, hxyz, a, b, C=1.0, mode="cell_exact"):
    """Uniform grid of rectangular cells hx x hy x hz (the Sec. 4.2 grid), I3 indexed
    [z][y][x]: weights I hx hy hz, the kernel table K(|(hx dx, hy dy, hz dz)|) (zero at
    d = 0) in a linear convolution zero-padded to twice the grid, and the rectangular
    cell's own term."""
    I3 = np.asarray(I3, dtype=np.float64)
    hx, hy, hz = (float(v) for v in hxyz)
    n = I3.shape
    q = I3 * (hx * hy * hz)
    grids = [np.arange(-(m - 1), m) for m in n]
    dz, dy, dx = np.meshgrid(*grids, indexing="ij")
    R = np.sqrt((hx * dx) ** 2 + (hy * dy) ** 2 + (hz * dz.astype(np.float64)) ** 2)
    R[n[0] - 1, n[1] - 1, n[2] - 1] = 1.0
    tab = _k.kernel(R, a, b)
    tab[n[0] - 1, n[1] - 1, n[2] - 1] = 0.0
    shape = [2 * m for m in n]
    ax = (0, 1, 2)
    F = np.fft.rfftn(q, shape, axes=ax) * np.fft.rfftn(tab, shape, axes=ax)
    conv = np.fft.irfftn(F, shape, axes=ax)
    far = conv[n[0] - 1:2 * n[0] - 1, n[1] - 1:2 * n[1] - 1, n[2] - 1:2 * n[2] - 1]
    if mode == "cell_exact":
        sig = _k.sigma_box_exact(hx, hy, hz, a, b)
    elif mode == "paper_gl2":
        sig = _k.sigma_box_paper_gl2(hx, hy, hz, a, b)
    else:
        raise ValueError("unknown self mode %r" % (mode,))
    return C * (far + sig * I3)
