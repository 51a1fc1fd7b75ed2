"""Oracle: adaptive octree and the U/V/W/X interaction lists, plain Python.

TEST INFRASTRUCTURE ONLY (the CPU oracle; never imported by the product path).

Sec. 3: a hierarchical octree is built from a root cube large enough to hold
every point, and a cube is split into eight equal sub-cubes while it holds
more than m points (outline step 1). The near range N(B) of a box B of side 2r is
the concentric box of side 6r and the far range F(B) the rest (Eq. (nearfar),
Fig. fNF). For non-uniform point sets the method follows the adaptive
kernel-independent FMM cited in Sec. 3, whose lists are:

* U(B), B a leaf: B and every leaf adjacent to B;
* V(B): children of the colleagues of B's parent that are not adjacent to B
  (colleagues = boxes of the same level adjacent to it, itself included);
* W(B), B a leaf: descendants of B's colleagues that are not adjacent to B but
  whose parent is adjacent to B;
* X(B): every box A with B in W(A).

Readings taken where the paper is silent:
* root cube: origin = min_i (x_i - h_i/2) per axis, side = the largest extent
  max_i (x_i + h_i/2) - origin over the three axes (recovers [0, L]^3 for a
  cell-centred grid of a cube);
* keys: 21 bits per axis, k = clamp(floor((x - o) * (2^21 / side)), 0, 2^21 - 1)
  with one FP64 subtraction and one FP64 multiplication (no fused multiply-add),
  interleaved z-y-x (x in the lowest bit of each triple); points are sorted
  stably by (key, input index);
* boxes split while count > m and level < 20; empty children are not created;
  boxes are numbered level by level, in Morton order within a level;
* adjacency: two boxes are adjacent when their closed cubes intersect.
"""
import numpy as np

MAX_LEVEL = 20
KEY_BITS = 21


class Tree:
    """Levelled octree over Morton-sorted points.

    Arrays (length = number of boxes, boxes numbered level by level):
    level, anchor[:, 3] (integer coordinates at the box's own level), parent
    (-1 for the root), child[:, 8] (-1 where the octant is empty), pstart, pend
    (range in sorted point order), leaf (bool). ``level_start[l]`` is the first
    box of level l (with a final sentinel)."""


def root_cube(points, h):
    """Origin min(x - h/2) per axis and side the largest extent; h per point (cubic cells)
    or (n, 3) per point and axis (rectangular cells)."""
    ext = h if h.ndim == 2 else h[:, None]
    lo = (points - 0.5 * ext).min(axis=0)
    hi = (points + 0.5 * ext).max(axis=0)
    side = float((hi - lo).max())
    return lo.astype(np.float64), side


def quantize(points, origin, side):
    """Integer cell coordinates at level 21 (one division for the scale, then a
    separate subtraction and multiplication per coordinate)."""
    scale = float(2 ** KEY_BITS) / side
    t = (points - origin[None, :])          # FP64 subtraction
    t = t * scale                           # FP64 multiplication (not fused)
    k = np.floor(t)
    k = np.clip(k, 0, 2 ** KEY_BITS - 1).astype(np.int64)
    return k


def interleave(k):
    """63-bit Morton key from three 21-bit integers (x lowest bit of each triple)."""
    key = np.zeros(k.shape[0], dtype=np.uint64)
    for bit in range(KEY_BITS):
        for axis in range(3):
            b = ((k[:, axis] >> bit) & 1).astype(np.uint64)
            key |= b << np.uint64(3 * bit + axis)
    return key


def build_tree(points, h, leaf_size, origin=None, side=None):
    """Returns (tree, perm): perm[k] is the input index of the k-th sorted point."""
    points = np.asarray(points, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    n = points.shape[0]
    if origin is None:
        origin, side = root_cube(points, h)
    kq = quantize(points, origin, side)
    key = interleave(kq)
    perm = np.lexsort((np.arange(n), key))       # stable by (key, index)
    skey = key[perm]
    # duplicate points (identical coordinates) make the sum undefined
    same = np.nonzero(skey[1:] == skey[:-1])[0]
    if same.size:
        # compare every pair inside each run of equal keys
        runs = {}
        for i in same:
            runs.setdefault(int(skey[i]), set()).update((int(i), int(i) + 1))
        for members in runs.values():
            m = sorted(members)
            p = points[perm[m]]
            for u in range(len(m)):
                for v in range(u + 1, len(m)):
                    if np.all(p[u] == p[v]):
                        raise ValueError("duplicate point")

    level, anchor, parent, pstart, pend = [0], [(0, 0, 0)], [-1], [0], [n]
    child = [[-1] * 8]
    leaf = [False]
    frontier = [0]
    lev = 0
    while frontier:
        nxt = []
        for b in frontier:
            cnt = pend[b] - pstart[b]
            if cnt <= leaf_size or lev >= MAX_LEVEL:
                leaf[b] = True
                continue
            shift = np.uint64(3 * (KEY_BITS - lev - 1))
            digits = (skey[pstart[b]:pend[b]] >> shift) & np.uint64(7)
            ax, ay, az = anchor[b]
            for o in range(8):
                lo = pstart[b] + int(np.searchsorted(digits, o, side="left"))
                hi = pstart[b] + int(np.searchsorted(digits, o, side="right"))
                if hi == lo:
                    continue
                cid = len(level)
                level.append(lev + 1)
                anchor.append((2 * ax + (o & 1), 2 * ay + ((o >> 1) & 1), 2 * az + ((o >> 2) & 1)))
                parent.append(b)
                pstart.append(lo)
                pend.append(hi)
                child.append([-1] * 8)
                leaf.append(False)
                child[b][o] = cid
                nxt.append(cid)
        frontier = nxt
        lev += 1

    t = Tree()
    t.level = np.array(level, dtype=np.int64)
    t.anchor = np.array(anchor, dtype=np.int64)
    t.parent = np.array(parent, dtype=np.int64)
    t.child = np.array(child, dtype=np.int64)
    t.pstart = np.array(pstart, dtype=np.int64)
    t.pend = np.array(pend, dtype=np.int64)
    t.leaf = np.array(leaf, dtype=bool)
    t.nlevels = int(t.level.max()) + 1
    t.level_start = np.searchsorted(t.level, np.arange(t.nlevels + 1))
    t.origin = np.asarray(origin, dtype=np.float64)
    t.side = float(side)
    t.keys = skey
    return t, perm


def box_center(t, b):
    r = t.side / 2.0 ** (t.level[b] + 1)
    return t.origin + (2.0 * t.anchor[b] + 1.0) * r


def half_width(t, lev):
    return t.side / 2.0 ** (lev + 1)


def adjacent(t, a, b):
    """Closed cubes of boxes a and b intersect (integer test at the finer level)."""
    la, lb = t.level[a], t.level[b]
    L = max(la, lb)
    sa, sb = 1 << (L - la), 1 << (L - lb)
    lo_a, lo_b = t.anchor[a] * sa, t.anchor[b] * sb
    hi_a, hi_b = lo_a + sa, lo_b + sb
    return bool(np.all(lo_a <= hi_b) and np.all(lo_b <= hi_a))


def _index(t):
    return {(int(t.level[b]), tuple(int(v) for v in t.anchor[b])): b for b in range(len(t.level))}


def colleagues(t, b, idx=None):
    """Same-level boxes adjacent to b, b itself included."""
    if idx is None:
        idx = _index(t)
    lev = int(t.level[b])
    ax, ay, az = (int(v) for v in t.anchor[b])
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                c = idx.get((lev, (ax + dx, ay + dy, az + dz)))
                if c is not None:
                    out.append(c)
    return sorted(out)


def _descendants(t, b):
    out = []
    stack = [b]
    while stack:
        c = stack.pop()
        for k in t.child[c]:
            if k >= 0:
                out.append(int(k))
                stack.append(int(k))
    return out


def build_lists(t):
    """U, V, W, X as lists of sorted box-id lists (empty where undefined)."""
    nb = len(t.level)
    idx = _index(t)
    U = [[] for _ in range(nb)]
    V = [[] for _ in range(nb)]
    W = [[] for _ in range(nb)]
    X = [[] for _ in range(nb)]
    leaves = [b for b in range(nb) if t.leaf[b]]
    # U: all leaves adjacent to a leaf B (B included). A leaf adjacent to B lies in
    # one of B's 27 same-level neighbour cells: either as that cell's box or a
    # descendant of it, or as a coarser leaf covering the cell.
    for b in leaves:
        lev = int(t.level[b])
        ax, ay, az = (int(v) for v in t.anchor[b])
        found = set()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    cell = (ax + dx, ay + dy, az + dz)
                    if min(cell) < 0 or max(cell) >= (1 << lev):
                        continue
                    c = idx.get((lev, cell))
                    if c is not None:
                        for d in [c] + _descendants(t, c):
                            if t.leaf[d] and adjacent(t, d, b):
                                found.add(d)
                    else:
                        for up in range(1, lev + 1):
                            c2 = idx.get((lev - up, tuple(v >> up for v in cell)))
                            if c2 is not None:
                                if t.leaf[c2]:
                                    found.add(c2)
                                break
        U[b] = sorted(found)
    # V: children of the parent's colleagues, not adjacent to B
    for b in range(nb):
        p = int(t.parent[b])
        if p < 0:
            continue
        out = []
        for c in colleagues(t, p, idx):
            for k in t.child[c]:
                if k >= 0 and not adjacent(t, int(k), b):
                    out.append(int(k))
        V[b] = sorted(out)
    # W: descendants of a leaf's colleagues, not adjacent, parent adjacent
    for b in leaves:
        out = []
        for c in colleagues(t, b, idx):
            if c == b or t.leaf[c]:
                continue
            stack = [c]
            while stack:
                d = stack.pop()
                for k in t.child[d]:
                    if k < 0:
                        continue
                    k = int(k)
                    if not adjacent(t, k, b):
                        out.append(k)          # its parent d is adjacent to b
                    elif not t.leaf[k]:
                        stack.append(k)
        W[b] = sorted(out)
    for b in leaves:
        for a in W[b]:
            X[a].append(b)
    X = [sorted(x) for x in X]
    return U, V, W, X


def build_lists_bruteforce(t):
    """The same four lists straight from their set definitions, O(B^2); a check
    for small trees."""
    nb = len(t.level)
    boxes = range(nb)
    leaves = [b for b in boxes if t.leaf[b]]

    def is_desc(d, c):
        while d >= 0:
            if d == c:
                return True
            d = int(t.parent[d])
        return False

    coll = {b: [c for c in boxes if t.level[c] == t.level[b] and adjacent(t, c, b)] for b in boxes}
    U = [[] for _ in boxes]
    V = [[] for _ in boxes]
    W = [[] for _ in boxes]
    X = [[] for _ in boxes]
    for b in leaves:
        U[b] = sorted(a for a in leaves if adjacent(t, a, b))
    for b in boxes:
        p = int(t.parent[b])
        if p >= 0:
            V[b] = sorted(a for a in boxes if t.parent[a] >= 0 and int(t.parent[a]) in coll[p]
                          and not adjacent(t, a, b))
    for b in leaves:
        W[b] = sorted(a for a in boxes
                      if any(c != b and a != c and is_desc(a, c) for c in coll[b])
                      and not adjacent(t, a, b) and t.parent[a] >= 0 and adjacent(t, int(t.parent[a]), b))
    for b in boxes:
        X[b] = sorted(a for a in leaves if b in W[a])
    return U, V, W, X


def coverage(t, U, V, W, X):
    """For every leaf B, how many times each source point is counted by
    U(B) (directly), W(B) (through upward expansions), and V/X of B and its
    ancestors (through downward expansions). Returns the (leaf, count-array)
    pairs; the lists are complete and disjoint when every count is 1."""
    n = int(t.pend[0])
    out = []
    for b in range(len(t.level)):
        if not t.leaf[b]:
            continue
        cnt = np.zeros(n, dtype=np.int64)
        for a in U[b]:
            cnt[t.pstart[a]:t.pend[a]] += 1
        for a in W[b]:
            cnt[t.pstart[a]:t.pend[a]] += 1
        d = b
        while d >= 0:
            for a in V[d]:
                cnt[t.pstart[a]:t.pend[a]] += 1
            for a in X[d]:
                cnt[t.pstart[a]:t.pend[a]] += 1
            d = int(t.parent[d])
        out.append((b, cnt))
    return out
