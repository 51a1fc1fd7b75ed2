"""Oracle: the FMM with a volumetric Chebyshev representation, plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (the CPU oracle of the `repr = CHEB` option; never imported by
the product path).

The paper's surface representation (Sec. 3) cannot approach the direct sum closer than the
pseudo-inverse allows for this non-harmonic kernel. This option keeps the paper's tree,
interaction lists (U/V/W/X), near field, self term and pass order (outline of Sec. 3) and
replaces each box's equivalent density by values at the p^3 tensor Chebyshev nodes of the
box (the black-box FMM of Fong and Darve, 2009):

* nodes: xbar_k = cos((2k - 1) pi / (2p)), k = 1..p, on [-1, 1]; a box with centre c and
  half-width r has the nodes c + r xbar (x fastest);
* interpolation weight S(x, xbar_m) = 1/p + (2/p) sum_{k=1}^{p-1} T_k(x) T_k(xbar_m) per
  axis (T_k the Chebyshev polynomials), the 3-D weight the product over the axes;
* P2M: W_m = sum_j S(xbar_m, (y_j - c)/r) q_j over the leaf's sources;
* M2M: W^P_n = sum_children sum_m S(xbar_n, (c_C + r_C xbar_m - c_P)/r_P) W^C_m;
* M2L (V list): g^B_m += sum_n K(|c_B + r xbar_m - c_A - r xbar_n|) W^A_n;
* X list: g^B_m += sum_{j in A} K(|c_B + r xbar_m - y_j|) q_j;
* L2L: g^C_m += sum_n S(xbar_n, (c_C + r_C xbar_m - c_P)/r_P) g^P_n;
* L2P: f(x_i) = sum_m S(xbar_m, (x_i - c_B)/r_B) g^B_m; W list: f(x_i) += sum_n
  K(|x_i - c_A - r_A xbar_n|) W^A_n.
"""
import numpy as np

from . import tree as _t
from .direct import pair_sum_c, self_terms
from .kifmm import kmat, _offset_index, _octant


def nodes1(p):
    """The p Chebyshev nodes of the first kind on [-1, 1]."""
    k = np.arange(1, p + 1)
    return np.cos((2 * k - 1) * np.pi / (2 * p))


def cheb_T(x, p):
    """T_0..T_{p-1} at the points x (shape (..., p)) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty(x.shape + (p,))
    out[..., 0] = 1.0
    if p > 1:
        out[..., 1] = x
    for k in range(2, p):
        out[..., k] = 2.0 * x * out[..., k - 1] - out[..., k - 2]
    return out


def s1(x, p):
    """Matrix S(x_i, xbar_m) (points x, the p nodes)."""
    Tx = cheb_T(x, p)
    Tn = cheb_T(nodes1(p), p)
    w = np.full(p, 2.0 / p)
    w[0] = 1.0 / p
    return (Tx * w) @ Tn.T


def nodes3(p):
    """The p^3 tensor nodes in [-1, 1]^3, x fastest."""
    g = nodes1(p)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def s3(xn, p):
    """Matrix S3(x_i, node_m) for normalised points xn (n, 3) and the p^3 nodes (x fastest)."""
    Sx, Sy, Sz = s1(xn[:, 0], p), s1(xn[:, 1], p), s1(xn[:, 2], p)
    return np.einsum("ik,ij,il->iljk", Sx, Sy, Sz).reshape(xn.shape[0], p ** 3)


class ChebOperators:
    """Level-independent M2M / L2L interpolation matrices and per-level M2L kernel
    matrices between the nodes of two boxes."""

    def __init__(self, side, nlevels, p, a, b):
        self.p = p
        nd = nodes3(p)
        self.nodes = nd
        self.S = nd.shape[0]
        # M2M for child octant o: M[o][n][m] = S3(parent node n, child node m in parent units)
        self.m2m = {}
        for o in range(8):
            cn = 0.5 * (2.0 * _octant(o) - 1.0) + 0.5 * nd
            self.m2m[o] = s3(cn, p).T
        self.m2l = {}
        for lev in range(2, nlevels):
            r = side / 2.0 ** (lev + 1)
            for dz in range(-3, 4):
                for dy in range(-3, 4):
                    for dx in range(-3, 4):
                        if max(abs(dx), abs(dy), abs(dz)) < 2:
                            continue
                        off = 2.0 * r * np.array([dx, dy, dz], dtype=np.float64)
                        self.m2l[(lev, _offset_index((dx, dy, dz)))] = kmat(r * nd, off + r * nd, a, b)


def plan(points, h, leaf_size, p, a, b, origin=None, side=None):
    points = np.asarray(points, dtype=np.float64)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (points.shape[0],)).copy()
    t, perm = _t.build_tree(points, h, leaf_size, origin, side)
    U, V, W, X = _t.build_lists(t)
    ops = ChebOperators(t.side, t.nlevels, p, a, b)
    return dict(tree=t, perm=perm, U=U, V=V, W=W, X=X, ops=ops, points=points[perm],
                h=h[perm], a=a, b=b, p=p)


def evaluate(pl, I, C=1.0, mode="cell_exact"):
    """S in input order for source values I (input order)."""
    t, ops, a, b, p = pl["tree"], pl["ops"], pl["a"], pl["b"], pl["p"]
    perm = pl["perm"]
    pts, h = pl["points"], pl["h"]
    Is = np.asarray(I, dtype=np.float64)[perm]
    q = Is * h ** 3
    nd = ops.nodes
    nb = len(t.level)
    S = ops.S
    centre = np.array([_t.box_center(t, b_) for b_ in range(nb)])
    rad = t.side / 2.0 ** (t.level + 1)

    # ---- upward pass (deepest level first): P2M at the leaves, M2M above
    Wu = np.zeros((nb, S))
    for lev in range(t.nlevels - 1, 1, -1):
        for B in range(t.level_start[lev], t.level_start[lev + 1]):
            if t.leaf[B]:
                sl = slice(t.pstart[B], t.pend[B])
                Wu[B] = s3((pts[sl] - centre[B]) / rad[B], p).T @ q[sl]
            else:
                for o in range(8):
                    c = t.child[B][o]
                    if c >= 0:
                        Wu[B] += ops.m2m[o] @ Wu[c]

    # ---- downward pass (shallowest level first): M2L by offset, X list, L2L
    g = np.zeros((nb, S))
    for lev in range(2, t.nlevels):
        lo, hi = t.level_start[lev], t.level_start[lev + 1]
        acc = np.zeros((hi - lo, S))
        groups = {}
        for B in range(lo, hi):
            for A in pl["V"][B]:
                d = t.anchor[A] - t.anchor[B]
                groups.setdefault(_offset_index(d), []).append((B - lo, A))
        for key, pairs in groups.items():
            tb = np.array([x[0] for x in pairs])
            sa = np.array([x[1] for x in pairs])
            np.add.at(acc, tb, Wu[sa] @ ops.m2l[(lev, key)].T)
        for B in range(lo, hi):
            xn = centre[B] + rad[B] * nd
            for A in pl["X"][B]:
                sl = slice(t.pstart[A], t.pend[A])
                acc[B - lo] += kmat(xn, pts[sl], a, b) @ q[sl]
            P = int(t.parent[B])
            if t.level[P] >= 2:
                o = int((t.anchor[B][0] & 1) | ((t.anchor[B][1] & 1) << 1) | ((t.anchor[B][2] & 1) << 2))
                acc[B - lo] += ops.m2m[o].T @ g[P]
        g[lo:hi] = acc

    # ---- targets: interpolation of the local values, W list, near field
    out = np.zeros(pts.shape[0])
    for B in range(nb):
        if not t.leaf[B]:
            continue
        sl = slice(t.pstart[B], t.pend[B])
        x = pts[sl]
        acc = np.zeros(x.shape[0])
        if t.level[B] >= 2:
            acc += s3((x - centre[B]) / rad[B], p) @ g[B]
        for A in pl["W"][B]:
            acc += kmat(x, centre[A] + rad[A] * nd, a, b) @ Wu[A]
        src = np.concatenate([np.arange(t.pstart[A], t.pend[A]) for A in pl["U"][B]])
        acc += pair_sum_c(x, np.arange(t.pstart[B], t.pend[B]), pts[src], src, q[src], a, b)
        out[sl] = acc
    out += self_terms(h, a, b, mode) * Is
    res = np.empty_like(out)
    res[perm] = C * out
    return res


def fmm(points, h, I, leaf_size, p, a, b, C=1.0, mode="cell_exact"):
    return evaluate(plan(points, h, leaf_size, p, a, b), I, C, mode)
