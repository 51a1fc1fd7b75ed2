"""Python binding of libkifmm (include/kifmm.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module passes
device pointers of torch tensors (or host buffers for ``eval_host``) and maps
status codes to exceptions. It fails loudly when the library is missing: there
is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libkifmm.so")

KIFMM_FP64, KIFMM_MIXED = 0, 1
KIFMM_SELF_CELL_EXACT, KIFMM_SELF_PAPER_GL2 = 0, 1
KIFMM_F32, KIFMM_F64 = 0, 1
KIFMM_MAX_LANES = 8   # concurrent streams of one batch (kifmm_eval_batch)
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_TIMEOUT",
          -5: "ERR_DUPLICATE_POINT", -6: "ERR_NONFINITE", -7: "ERR_NUMERIC"}
PRECISION = {"fp64": KIFMM_FP64, "mixed": KIFMM_MIXED}
SELF_MODE = {"cell_exact": KIFMM_SELF_CELL_EXACT, "paper_gl2": KIFMM_SELF_PAPER_GL2}
REPR = {"surface": 0, "cheb": 1}
KERNEL = {"zheleznyak": 0, "helmholtz3": 1, "threegroup": 2}


def model_constants(p, p_o2, p_q=30.0, xi_omega_alpha=0.06):
    """(a, b, C) of the Zheleznyak model for pressure p and oxygen pressure p_O2 (Torr),
    computed by kifmm_model_constants (Sec. 2.1, Eqs. (gfun), (Ifun))."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().kifmm_model_constants(float(p), float(p_o2), float(p_q), float(xi_omega_alpha), ctypes.byref(a),
                                        ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def absorption(p_o2):
    """(a, b) = (chi_min p_O2, chi_max p_O2) from kifmm_model_constants."""
    a, b, _ = model_constants(760.0, p_o2)
    return a, b


def scale_c(p, p_q=30.0, xi_omega_alpha=0.06):
    """C = xi (omega/alpha) p_q / (p + p_q) of Eq. (Ifun), from kifmm_model_constants."""
    return model_constants(p, 1.0, p_q, xi_omega_alpha)[2]


class KifmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("self_mode", ctypes.c_int), ("pinv_eps", ctypes.c_double),
                ("has_root", ctypes.c_int), ("root", ctypes.c_double * 4), ("stream", ctypes.c_void_p),
                ("repr", ctypes.c_int), ("radii", ctypes.c_double * 2), ("cell_dims", ctypes.c_double * 3),
                ("kernel", ctypes.c_int), ("pad_lattice", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_boxes", ctypes.c_int64), ("n_levels", ctypes.c_int32),
                ("surface_points", ctypes.c_int32), ("n_leaves", ctypes.c_int64),
                ("list_len", ctypes.c_int64 * 4), ("origin", ctypes.c_double * 3), ("side", ctypes.c_double),
                ("pinv_rank_min", ctypes.c_double), ("eval_launches", ctypes.c_int64),
                ("p2p_pairs", ctypes.c_int64), ("m2l_tensor", ctypes.c_int64), ("device_error", ctypes.c_int64),
                ("m2l_flops", ctypes.c_double), ("upward_flops", ctypes.c_double),
                ("upward_mma_flops", ctypes.c_double), ("near_tensor", ctypes.c_int64),
                ("lattice_far", ctypes.c_int64), ("m2m_tensor_levels", ctypes.c_int64),
                ("l2l_tensor_levels", ctypes.c_int64), ("upward_tensor_levels", ctypes.c_int64),
                ("n_padding", ctypes.c_int64)]


class _StreamerParams(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double), ("phi0", ctypes.c_double), ("mu_e", ctypes.c_double),
                ("mu_p", ctypes.c_double), ("D_e", ctypes.c_double), ("C", ctypes.c_double),
                ("mg_tol", ctypes.c_double), ("mg_max_cycles", ctypes.c_int), ("region", ctypes.c_int * 6),
                ("threshold", ctypes.c_double)]


class _TuneEntry(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int), ("order", ctypes.c_int), ("radii", ctypes.c_double * 2),
                ("ms", ctypes.c_float), ("err", ctypes.c_double), ("ok", ctypes.c_int)]


EXPORTS = ["kifmm_default_opts", "kifmm_plan", "kifmm_eval", "kifmm_eval_host", "kifmm_eval_batch",
           "kifmm_destroy", "kifmm_last_error", "kifmm_check", "kifmm_model_constants", "kifmm_get_info",
           "kifmm_get_tree", "kifmm_get_list",
           "kifmm_get_sigma", "kifmm_get_upward", "kifmm_get_phase_times", "kifmm_direct_noalloc", "kifmm_autotune", "kifmm_tune",
           "sno_create", "sno_destroy", "sno_num_params", "sno_set_params", "sno_get_params", "sno_get_grads",
           "sno_save", "sno_load", "sno_save_checkpoint", "sno_load_checkpoint",
           "sno_set_bf16", "sno_set_period", "sno_set_near_field", "sno_init_far_field", "sno_forward",
           "sno_loss_grad", "sno_adam_step", "photo_solve", "photo_solve_batch",
           "streamer_default_params", "streamer_create", "streamer_set", "streamer_get", "streamer_rhs",
           "streamer_step", "streamer_poisson", "streamer_info", "streamer_destroy"]

_lib = None


def lib_path():
    return _LIB_PATH


def load():
    """Loads libkifmm.so (built by ``paper_2006_03515_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("libkifmm.so is not built (%s); run paper_2006_03515_gb300.build.build()" % _LIB_PATH)
    L = ctypes.CDLL(_LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.kifmm_default_opts.argtypes = [ctypes.POINTER(_Opts)]
    L.kifmm_default_opts.restype = None
    L.kifmm_plan.argtypes = [ctypes.POINTER(vp), vp, i64, vp, dbl, i32, i32, dbl, dbl, ctypes.POINTER(_Opts)]
    L.kifmm_eval.argtypes = [vp, vp, vp, i32, dbl]
    L.kifmm_eval_host.argtypes = [vp, vp, vp, i32, dbl]
    L.kifmm_eval_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i32, i32,
                                   ctypes.POINTER(dbl), i32, i32]
    L.kifmm_check.argtypes = [vp]
    L.kifmm_model_constants.argtypes = [dbl, dbl, dbl, dbl, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                        ctypes.POINTER(dbl)]
    L.kifmm_destroy.argtypes = [vp]
    L.kifmm_destroy.restype = None
    L.kifmm_last_error.restype = ctypes.c_char_p
    L.kifmm_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
    L.kifmm_get_tree.argtypes = [vp] + [vp] * 9
    L.kifmm_get_list.argtypes = [vp, i32, vp, vp]
    L.kifmm_get_sigma.argtypes = [vp, vp]
    L.kifmm_get_upward.argtypes = [vp, vp, ctypes.POINTER(i32)]
    L.kifmm_get_phase_times.argtypes = [vp, vp, i32]
    L.kifmm_direct_noalloc.argtypes = [vp, i64, dbl, vp, vp, dbl, dbl, dbl, i32, vp]
    L.kifmm_autotune.argtypes = [vp, i64, vp, dbl, vp, i32, i32, dbl, dbl, ctypes.POINTER(_Opts), i32, vp, vp]
    L.kifmm_tune.argtypes = [vp, i64, vp, dbl, vp, dbl, dbl, ctypes.POINTER(_Opts), vp, i32, vp, i32, vp, i32, dbl,
                             i32, i32, ctypes.POINTER(_TuneEntry), ctypes.POINTER(_TuneEntry)]
    for name in ("kifmm_plan", "kifmm_eval", "kifmm_eval_host", "kifmm_eval_batch", "kifmm_check",
                 "kifmm_model_constants", "kifmm_get_info",
                 "kifmm_get_tree", "kifmm_get_list", "kifmm_get_sigma", "kifmm_get_upward", "kifmm_get_phase_times",
                 "kifmm_direct_noalloc", "kifmm_autotune", "kifmm_tune"):
        getattr(L, name).restype = ctypes.c_int
    _load_sno(L)
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise KifmmError(rc, load().kifmm_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


class Plan:
    """A KIFMM plan over fixed points (outline step 1 and the operators)."""

    def __init__(self, points, h, leaf_size=64, surface_order=6, a=None, b=None, precision="fp64",
                 self_mode="cell_exact", pinv_eps=1e-5, root=None, stream=None, repr="surface",
                 surface_radii=None, cell_dims=None, kernel="zheleznyak", pad_lattice=False):
        import torch
        L = load()
        if not (isinstance(points, torch.Tensor) and points.is_cuda):
            raise TypeError("points must be a CUDA tensor")
        self._points = points.detach().to(torch.float64).contiguous()
        if self._points.dim() != 2 or self._points.shape[1] != 3:
            raise ValueError("points must be N x 3")
        self.n = int(self._points.shape[0])
        hp, uh = None, 0.0
        if isinstance(h, torch.Tensor):
            self._h = h.detach().to(device=self._points.device, dtype=torch.float64).contiguous()
            if self._h.numel() != self.n:
                raise ValueError("h must have N entries")
            hp = ctypes.c_void_p(self._h.data_ptr())
        else:
            self._h = None
            uh = 0.0 if h is None else float(h)
        o = _Opts()
        L.kifmm_default_opts(ctypes.byref(o))
        o.precision = PRECISION[precision]
        o.self_mode = SELF_MODE[self_mode]
        o.pinv_eps = float(pinv_eps)
        o.repr = REPR[repr]
        o.kernel = KERNEL[kernel]
        o.pad_lattice = 1 if pad_lattice else 0   # zero-weight cells up to the leaf lattice (full box grids)
        if root is not None:
            o.has_root = 1
            for k in range(4):
                o.root[k] = float(root[k])
        if surface_radii is not None:   # (inner, outer) in box half-widths; default (1.05, 2.95)
            o.radii[0], o.radii[1] = float(surface_radii[0]), float(surface_radii[1])
        if cell_dims is not None:       # rectangular cells (hx, hy, hz); h is then ignored
            for k in range(3):
                o.cell_dims[k] = float(cell_dims[k])
            if isinstance(h, torch.Tensor):
                raise ValueError("cell_dims and per-point h exclude each other")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o.stream = _stream_ptr(self.stream)
        self.precision = precision
        self._h_ptr = ctypes.c_void_p()
        _check(L.kifmm_plan(ctypes.byref(self._h_ptr), ctypes.c_void_p(self._points.data_ptr()), self.n, hp, uh,
                            int(leaf_size), int(surface_order), float(a), float(b), ctypes.byref(o)))

    @property
    def handle(self):
        return self._h_ptr

    def eval(self, I, S=None, C=1.0):
        """S = C * (sum over the FMM + near field + self term); I: CUDA tensor (N,) f32/f64."""
        import torch
        if not (isinstance(I, torch.Tensor) and I.is_cuda and I.is_contiguous() and I.numel() == self.n):
            raise TypeError("I must be a contiguous CUDA tensor with N entries")
        dt = {torch.float64: KIFMM_F64, torch.float32: KIFMM_F32}[I.dtype]
        if S is None:
            S = torch.empty_like(I)
        _check(load().kifmm_eval(self._h_ptr, ctypes.c_void_p(I.data_ptr()), ctypes.c_void_p(S.data_ptr()), dt,
                                 float(C)))
        return S

    def eval_host(self, I, S=None, C=1.0):
        """The same evaluation from host numpy buffers (copies inside the call)."""
        I = np.ascontiguousarray(I)
        dt = {np.dtype(np.float64): KIFMM_F64, np.dtype(np.float32): KIFMM_F32}[I.dtype]
        if S is None:
            S = np.empty_like(I)
        _check(load().kifmm_eval_host(self._h_ptr, ctypes.c_void_p(I.ctypes.data), ctypes.c_void_p(S.ctypes.data),
                                      dt, float(C)))
        return S

    def check(self):
        """Synchronises the plan's stream and raises KifmmError (ERR_TIMEOUT) if a bounded
        device wait of its work gave up since the last check (kifmm_check)."""
        _check(load().kifmm_check(self._h_ptr))

    def info(self):
        inf = _Info()
        _check(load().kifmm_get_info(self._h_ptr, ctypes.byref(inf)))
        return dict(n_points=inf.n_points, n_boxes=inf.n_boxes, n_levels=inf.n_levels,
                    surface_points=inf.surface_points, n_leaves=inf.n_leaves, list_len=list(inf.list_len),
                    origin=list(inf.origin), side=inf.side, pinv_rank_min=int(inf.pinv_rank_min),
                    eval_launches=int(inf.eval_launches), p2p_pairs=int(inf.p2p_pairs),
                    m2l_tensor=bool(inf.m2l_tensor), device_error=int(inf.device_error),
                    m2l_flops=float(inf.m2l_flops), upward_flops=float(inf.upward_flops),
                    upward_mma_flops=float(inf.upward_mma_flops), near_tensor=bool(inf.near_tensor),
                    lattice_far=bool(inf.lattice_far), m2m_tensor_levels=int(inf.m2m_tensor_levels),
                    l2l_tensor_levels=int(inf.l2l_tensor_levels), upward_tensor_levels=int(inf.upward_tensor_levels),
                    n_padding=int(inf.n_padding))

    def tree(self):
        inf = self.info()
        n, nb = inf["n_points"], inf["n_boxes"]
        out = dict(perm=np.empty(n, np.int64), keys=np.empty(n, np.uint64), level=np.empty(nb, np.int32),
                   parent=np.empty(nb, np.int32), pstart=np.empty(nb, np.int64), pend=np.empty(nb, np.int64),
                   leaf=np.empty(nb, np.int32), anchor=np.empty((nb, 3), np.int32),
                   child=np.empty((nb, 8), np.int32))
        order = ["perm", "keys", "level", "parent", "pstart", "pend", "leaf", "anchor", "child"]
        _check(load().kifmm_get_tree(self._h_ptr, *[ctypes.c_void_p(out[k].ctypes.data) for k in order]))
        return out

    def list(self, which):
        inf = self.info()
        off = np.empty(inf["n_boxes"] + 1, np.int64)
        items = np.empty(max(1, inf["list_len"][which]), np.int32)
        _check(load().kifmm_get_list(self._h_ptr, int(which), ctypes.c_void_p(off.ctypes.data),
                                     ctypes.c_void_p(items.ctypes.data)))
        return off, items[:inf["list_len"][which]]

    def sigma(self):
        s = np.empty(self.info()["n_points"], np.float64)
        _check(load().kifmm_get_sigma(self._h_ptr, ctypes.c_void_p(s.ctypes.data)))
        return s

    def upward(self):
        """Upward coefficients c of the last evaluation, (n_boxes, stride) FP64."""
        inf = self.info()
        st = ctypes.c_int()
        _check(load().kifmm_get_upward(self._h_ptr, None, ctypes.byref(st)))
        buf = np.empty(inf["n_boxes"] * st.value, np.float64)
        _check(load().kifmm_get_upward(self._h_ptr, ctypes.c_void_p(buf.ctypes.data), ctypes.byref(st)))
        return buf.reshape(inf["n_boxes"], st.value)

    def phase_times(self):
        ms = (ctypes.c_float * 8)()
        k = load().kifmm_get_phase_times(self._h_ptr, ms, 8)
        return list(ms)[:k]

    def close(self):
        if self._h_ptr:
            load().kifmm_destroy(self._h_ptr)
            self._h_ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(points, h, candidates=(32, 48, 64, 96, 128), surface_order=6, a=None, b=None, precision="mixed",
             self_mode="cell_exact", pinv_eps=1e-5, reps=3, stream=None):
    """Leaf size chosen by timing kifmm_eval for each candidate (kifmm_autotune).
    Returns (best_leaf, {leaf: ms})."""
    import torch
    L = load()
    pts = points.detach().to(torch.float64).contiguous()
    hp, uh = None, 0.0
    if isinstance(h, torch.Tensor):
        hh = h.detach().to(device=pts.device, dtype=torch.float64).contiguous()
        hp = ctypes.c_void_p(hh.data_ptr())
    else:
        uh = float(h)
    o = _Opts()
    L.kifmm_default_opts(ctypes.byref(o))
    o.precision = PRECISION[precision]
    o.self_mode = SELF_MODE[self_mode]
    o.pinv_eps = float(pinv_eps)
    o.stream = _stream_ptr(stream)
    cand = (ctypes.c_int * len(candidates))(*[int(c) for c in candidates])
    ms = (ctypes.c_float * len(candidates))()
    best = ctypes.c_int(-1)
    _check(L.kifmm_autotune(ctypes.c_void_p(pts.data_ptr()), int(pts.shape[0]), hp, uh, cand, len(candidates),
                            int(surface_order), float(a), float(b), ctypes.byref(o), int(reps), ctypes.byref(best), ms))
    return best.value, {int(c): float(t) for c, t in zip(candidates, ms)}


def tune(points, h, I, a, b, leaf=(32, 64, 128), order=(4, 6, 8), radii=None, target=1e-3, precision="mixed",
         k_samples=256, reps=3, root=None, stream=None, pad_lattice=False):
    """The fastest (leaf, order, radii) whose estimated error against the direct sum is at most
    target / 2 (kifmm_tune). I: representative source, CUDA float64 (N,). radii: a list of
    (inner, outer) pairs, or None for the default surfaces. Returns (best, table), dicts
    with leaf, order, radii, ms, err, ok."""
    import torch
    L = load()
    pts = points.detach().to(torch.float64).contiguous()
    if not (isinstance(I, torch.Tensor) and I.is_cuda and I.dtype == torch.float64 and I.is_contiguous()
            and I.numel() == pts.shape[0]):
        raise TypeError("I must be a contiguous CUDA float64 tensor with N entries")
    hp, uh = None, 0.0
    if isinstance(h, torch.Tensor):
        hh = h.detach().to(device=pts.device, dtype=torch.float64).contiguous()
        hp = ctypes.c_void_p(hh.data_ptr())
    else:
        uh = float(h)
    o = _Opts()
    L.kifmm_default_opts(ctypes.byref(o))
    o.precision = PRECISION[precision]
    o.stream = _stream_ptr(stream)
    o.pad_lattice = 1 if pad_lattice else 0
    if root is not None:
        o.has_root = 1
        for k in range(4):
            o.root[k] = float(root[k])
    lf = (ctypes.c_int * len(leaf))(*[int(x) for x in leaf])
    od = (ctypes.c_int * len(order))(*[int(x) for x in order])
    rl = [] if radii is None else [float(v) for pair in radii for v in pair]
    rd = (ctypes.c_double * max(1, len(rl)))(*rl) if rl else None
    nr = len(rl) // 2
    ncand = len(leaf) * len(order) * max(1, nr)
    tab = (_TuneEntry * ncand)()
    best = _TuneEntry()
    _check(L.kifmm_tune(ctypes.c_void_p(pts.data_ptr()), int(pts.shape[0]), hp, uh, ctypes.c_void_p(I.data_ptr()),
                        float(a), float(b), ctypes.byref(o), lf, len(leaf), od, len(order), rd, nr, float(target),
                        int(k_samples), int(reps), tab, ctypes.byref(best)))

    def d(e):
        return dict(leaf=e.leaf, order=e.order, radii=(e.radii[0], e.radii[1]), ms=float(e.ms), err=float(e.err),
                    ok=bool(e.ok))
    return d(best), [d(e) for e in tab]


NOALLOC_MAX_POINTS = 65536


def direct_noalloc(points, h, I, a, b, C=1.0, S=None, self_mode="cell_exact", stream=None):
    """Direct FP64 sum for cells of one edge h through kifmm_direct_noalloc, which uses a
    fixed device work space instead of allocating (for callers that cannot allocate, e.g.
    code whose device memory belongs to another allocator). points (n, 3), I and S (n,) are
    contiguous CUDA float64 tensors on one device; n <= 65536. Nothing is copied: a tensor
    of the wrong dtype, shape, device or layout raises before the call."""
    import torch

    def ok(x, shape):
        return (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
                and tuple(x.shape) == shape)

    if not (isinstance(points, torch.Tensor) and points.dim() == 2):
        raise TypeError("points must be an (n, 3) CUDA float64 tensor")
    n = int(points.shape[0])
    if not ok(points, (n, 3)):
        raise TypeError("points must be a contiguous (n, 3) CUDA float64 tensor")
    if not ok(I, (n,)):
        raise TypeError("I must be a contiguous CUDA float64 tensor of n = %d entries" % n)
    if S is None:
        S = torch.empty_like(I)
    if not ok(S, (n,)):
        raise TypeError("S must be a contiguous CUDA float64 tensor of n = %d entries" % n)
    if not (points.device == I.device == S.device):
        raise ValueError("points, I and S must be on one device")
    _check(load().kifmm_direct_noalloc(ctypes.c_void_p(points.data_ptr()), n, float(h),
                                       ctypes.c_void_p(I.data_ptr()), ctypes.c_void_p(S.data_ptr()), float(a),
                                       float(b), float(C), SELF_MODE[self_mode], _stream_ptr(stream)))
    return S


def eval_batch(plans, Is, Ss, C=None, capture=False, lanes=4):
    """Evaluates several fields (plans) as one unit of work ordered on plans[0]'s stream.

    With lanes > 1 the fields run concurrently on up to `lanes` streams forked from and
    joined back to plans[0]'s stream (entries repeating a plan stay in order on one lane);
    capture=True records the whole batch once as a CUDA graph and replays it afterwards.
    """
    import torch
    n = len(plans)
    dt = {torch.float64: KIFMM_F64, torch.float32: KIFMM_F32}[Is[0].dtype]
    ph = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    ip = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Is])
    sp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Ss])
    cc = (ctypes.c_double * n)(*([1.0] * n if C is None else [float(c) for c in C]))
    _check(load().kifmm_eval_batch(ph, ip, sp, n, dt, cc, 1 if capture else 0, int(lanes)))
    return Ss


def _load_sno(L):
    vp, i64, i32, dbl, flt = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_float
    L.sno_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32, i32, i32, vp]
    L.sno_destroy.argtypes = [vp]
    L.sno_destroy.restype = None
    L.sno_num_params.argtypes = [vp]
    L.sno_num_params.restype = i64
    L.sno_set_params.argtypes = [vp, vp]
    L.sno_get_params.argtypes = [vp, vp]
    L.sno_get_grads.argtypes = [vp, vp]
    L.sno_save.argtypes = [vp, ctypes.c_char_p]
    L.sno_load.argtypes = [vp, ctypes.c_char_p]
    L.sno_save_checkpoint.argtypes = [vp, ctypes.c_char_p]
    L.sno_load_checkpoint.argtypes = [vp, ctypes.c_char_p]
    L.sno_set_bf16.argtypes = [vp, i32]
    L.sno_set_period.argtypes = [vp, i32]
    L.sno_set_near_field.argtypes = [vp, dbl, dbl, dbl, i32, dbl, dbl]
    L.sno_init_far_field.argtypes = [vp, dbl]
    L.sno_forward.argtypes = [vp, vp, vp, i32]
    L.sno_loss_grad.argtypes = [vp, vp, vp, i32, ctypes.POINTER(dbl)]
    L.sno_adam_step.argtypes = [vp, flt, flt, flt, flt]
    L.photo_solve.argtypes = [vp, vp, vp, vp, dbl, dbl, i32, ctypes.c_uint64, ctypes.POINTER(i32),
                              ctypes.POINTER(dbl)]
    L.photo_solve_batch.argtypes = [vp, i32, vp, vp, vp, vp, dbl, i32, ctypes.c_uint64, vp, vp]
    L.streamer_default_params.argtypes = [ctypes.POINTER(_StreamerParams), dbl]
    L.streamer_default_params.restype = None
    L.streamer_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, dbl, ctypes.POINTER(_StreamerParams), vp, vp]
    L.streamer_set.argtypes = [vp, vp, vp]
    L.streamer_get.argtypes = [vp, vp, vp, vp, vp]
    L.streamer_rhs.argtypes = [vp, vp, vp]
    L.streamer_step.argtypes = [vp, dbl, i32]
    L.streamer_poisson.argtypes = [vp, vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(i32)]
    L.streamer_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(dbl)]
    L.streamer_destroy.argtypes = [vp]
    L.streamer_destroy.restype = None
    for name in ("streamer_create", "streamer_set", "streamer_get", "streamer_rhs", "streamer_step",
                 "streamer_poisson", "streamer_info"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("photo_solve_batch", "sno_create", "sno_save", "sno_load", "sno_save_checkpoint", "sno_load_checkpoint", "sno_set_params",
                 "sno_get_params", "sno_get_grads", "sno_set_bf16", "sno_set_period", "sno_set_near_field",
                 "sno_init_far_field", "sno_forward", "sno_loss_grad", "sno_adam_step", "photo_solve"):
        getattr(L, name).restype = ctypes.c_int


class SNO:
    """The spectral neural operator surrogate (sno_* in kifmm.h): grid n^3, ``width``
    channels, ``modes`` frequencies per axis, ``layers`` spectral layers, projection width
    ``proj``. Fields are CUDA float32 tensors of shape (batch, n^3) or (n^3,): inputs
    u = I / max I, outputs S / (C max I)."""

    def __init__(self, n, width=32, modes=8, layers=4, proj=64, max_batch=8, stream=None):
        L = load()
        self.n, self.width, self.modes, self.layers, self.proj, self.max_batch = n, width, modes, layers, proj, max_batch
        self._h = ctypes.c_void_p()
        self._stream = stream
        self.period, self.near = n, None
        _check(L.sno_create(ctypes.byref(self._h), int(n), int(width), int(modes), int(layers), int(proj),
                            int(max_batch), _stream_ptr(stream)))

    @property
    def handle(self):
        return self._h

    def num_params(self):
        return int(load().sno_num_params(self._h))

    def layout(self):
        """(name, shape) of each parameter block in the flat vector's order."""
        C, m, P = self.width, self.modes, self.proj
        K = (2 * m) * (2 * m) * m
        lay = [("Wl", (C,)), ("bl", (C,))]
        for l in range(self.layers):
            lay += [("Rr%d" % l, (K, C, C)), ("Ri%d" % l, (K, C, C)), ("W%d" % l, (C, C)), ("b%d" % l, (C,))]
        return lay + [("Q1", (P, C)), ("q1", (P,)), ("Q2", (P,)), ("q2", (1,))]

    def init_params(self, seed=0):
        """Seeded initial parameters (scaled normal weights, zero biases)."""
        import numpy as np
        rng = np.random.Generator(np.random.PCG64(seed))
        parts = []
        C = self.width
        for name, shp in self.layout():
            k = int(np.prod(shp))
            if name.startswith("b") or name in ("q1", "q2"):
                parts.append(np.zeros(k))
            elif name == "Wl":
                parts.append(rng.standard_normal(k))
            elif name.startswith("R"):
                parts.append(rng.standard_normal(k) * (1.0 / C))
            elif name == "Q1":
                parts.append(rng.standard_normal(k) / np.sqrt(C))
            elif name == "Q2":
                parts.append(rng.standard_normal(k) / np.sqrt(self.proj))
            else:
                parts.append(rng.standard_normal(k) / np.sqrt(C))
        theta = np.concatenate(parts).astype(np.float32)
        self.set_params(theta)
        return theta

    def set_params(self, theta):
        import numpy as np
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != self.num_params():
            raise ValueError("expected %d parameters" % self.num_params())
        _check(load().sno_set_params(self._h, t.ctypes.data_as(ctypes.c_void_p)))

    def params(self):
        import numpy as np
        t = np.empty(self.num_params(), dtype=np.float32)
        _check(load().sno_get_params(self._h, t.ctypes.data_as(ctypes.c_void_p)))
        return t

    def grads(self):
        import numpy as np
        g = np.empty(self.num_params(), dtype=np.float32)
        _check(load().sno_get_grads(self._h, g.ctypes.data_as(ctypes.c_void_p)))
        return g

    def set_bf16(self, on):
        _check(load().sno_set_bf16(self._h, 1 if on else 0))

    def set_period(self, period):
        """Period N >= n of the truncated transforms (sno_set_period)."""
        _check(load().sno_set_period(self._h, int(period)))
        self.period = int(period)

    def set_near_field(self, a, b, h, r_in, r_out, self_mode="cell_exact"):
        """Exact near part added to the output (sno_set_near_field); a = b = 0 switches it off."""
        _check(load().sno_set_near_field(self._h, float(a), float(b), float(h), SELF_MODE[self_mode], float(r_in),
                                         float(r_out)))
        self.near = None if a == 0 and b == 0 else dict(a=a, b=b, h=h, r_in=r_in, r_out=r_out, self_mode=self_mode)

    def init_far_field(self, shift=8.0):
        """Channel 0 carries the far part's Fourier multiplier (sno_init_far_field)."""
        _check(load().sno_init_far_field(self._h, float(shift)))

    def save(self, path):
        _check(load().sno_save(self._h, os.fsencode(path)))

    def load(self, path):
        _check(load().sno_load(self._h, os.fsencode(path)))

    def save_checkpoint(self, path):
        """Parameters, Adam moments and step count (training resumes exactly)."""
        _check(load().sno_save_checkpoint(self._h, os.fsencode(path)))

    def load_checkpoint(self, path):
        _check(load().sno_load_checkpoint(self._h, os.fsencode(path)))

    def _batch(self, u):
        import torch
        if not (isinstance(u, torch.Tensor) and u.is_cuda and u.dtype == torch.float32 and u.is_contiguous()):
            raise TypeError("fields must be contiguous CUDA float32 tensors")
        if u.numel() % (self.n ** 3):
            raise ValueError("field size is not a multiple of n^3")
        return u.numel() // (self.n ** 3)

    def forward(self, u, y=None):
        import torch
        B = self._batch(u)
        if y is None:
            y = torch.empty_like(u)
        _check(load().sno_forward(self._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(y.data_ptr()), B))
        return y

    def loss_grad(self, u, t):
        B = self._batch(u)
        if t.shape != u.shape:
            raise ValueError("target shape differs from input shape")
        loss = ctypes.c_double()
        _check(load().sno_loss_grad(self._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(t.data_ptr()), B,
                                    ctypes.byref(loss)))
        return loss.value

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(load().sno_adam_step(self._h, float(lr), float(beta1), float(beta2), float(eps)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().sno_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def photo_solve(plan, model, I, S=None, C=1.0, tol=0.05, k_samples=256, seed=0):
    """Surrogate-first solve (photo_solve in kifmm.h): S = C max|I| network(I / max|I|), judged
    at k_samples sampled targets against the direct sum, kifmm_eval above tol. I, S: CUDA
    float64 tensors (N,). Returns (S, used_fallback, judged_error)."""
    import torch
    if S is None:
        S = torch.empty_like(I)
    fb = ctypes.c_int()
    err = ctypes.c_double()
    _check(load().photo_solve(plan.handle, model.handle, ctypes.c_void_p(I.data_ptr()), ctypes.c_void_p(S.data_ptr()),
                              float(C), float(tol), int(k_samples), int(seed), ctypes.byref(fb), ctypes.byref(err)))
    return S, bool(fb.value), err.value


def photo_solve_batch(plans, model, Is, Ss=None, C=None, tol=0.05, k_samples=256, seed=0):
    """photo_solve for several fields at once (photo_solve_batch in kifmm.h): one plan, source
    and result per field (CUDA float64 tensors of the model's grid). Returns (Ss,
    used_fallback list, judged_error list); returns when every result is complete."""
    import torch
    k = len(plans)
    if not (len(Is) == k and k >= 1):
        raise ValueError("one source per plan")
    for I in Is:
        if not (isinstance(I, torch.Tensor) and I.is_cuda and I.dtype == torch.float64 and I.is_contiguous()):
            raise TypeError("sources must be contiguous CUDA float64 tensors")
    if Ss is None:
        Ss = [torch.empty_like(I) for I in Is]
    for S, I in zip(Ss, Is):
        if not (isinstance(S, torch.Tensor) and S.is_cuda and S.dtype == torch.float64 and S.is_contiguous()
                and S.numel() == I.numel()):
            raise TypeError("results must be contiguous CUDA float64 tensors of the sources' size")
    hp = (ctypes.c_void_p * k)(*[pl.handle.value for pl in plans])
    ip = (ctypes.c_void_p * k)(*[I.data_ptr() for I in Is])
    sp = (ctypes.c_void_p * k)(*[S.data_ptr() for S in Ss])
    cs = (ctypes.c_double * k)(*([1.0] * k if C is None else [float(c) for c in C]))
    fb = (ctypes.c_int * k)()
    err = (ctypes.c_double * k)()
    _check(load().photo_solve_batch(hp, k, model.handle, ip, sp, cs, float(tol), int(k_samples), int(seed), fb, err))
    return Ss, [bool(x) for x in fb], [float(x) for x in err]


class Streamer:
    """The streamer time loop of Sec. 5, Eq. (eM) (streamer_* in kifmm.h): fields [z][y][x] on
    nx x ny x nz cubic cells of edge h (cm), CUDA float64 tensors of nx ny nz entries. plan: a
    Plan over the cell centres in that order (the FMM of S_ph; over the region's cells when
    region = (x0, x1, y0, y1, z0, z1) is given) or None; params: overrides of the paper's
    values (p, phi0, mu_e, mu_p, D_e, C, mg_tol, mg_max_cycles, threshold)."""

    def __init__(self, nx, ny, nz, h, p=760.0, plan=None, stream=None, **params):
        import torch
        L = load()
        prm = _StreamerParams()
        L.streamer_default_params(ctypes.byref(prm), float(p))
        for k, v in params.items():
            if k == "region":
                for q in range(6):
                    prm.region[q] = int(v[q])
                continue
            if not hasattr(prm, k):
                raise KeyError(k)
            setattr(prm, k, v)
        self.shape = (int(nz), int(ny), int(nx))
        self.n = int(nx) * int(ny) * int(nz)
        self.plan = plan   # (kept alive with the streamer)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        _check(L.streamer_create(ctypes.byref(self._h), int(nx), int(ny), int(nz), float(h), ctypes.byref(prm),
                                 plan.handle if plan is not None else None, _stream_ptr(self.stream)))

    def _t(self, x):
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
                and x.numel() == self.n):
            raise TypeError("fields must be contiguous CUDA float64 tensors of nx ny nz entries")
        return ctypes.c_void_p(x.data_ptr())

    def _new(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    def set(self, ne, np_):
        _check(load().streamer_set(self._h, self._t(ne), self._t(np_)))

    def get(self):
        """(n_e, n_p, phi, S_ph) of the current state / last right-hand side."""
        out = [self._new() for _ in range(4)]
        _check(load().streamer_get(self._h, *[self._t(x) for x in out]))
        self.stream.synchronize()
        return tuple(out)

    def rhs(self):
        dne, dnp = self._new(), self._new()
        _check(load().streamer_rhs(self._h, self._t(dne), self._t(dnp)))
        self.stream.synchronize()
        return dne, dnp

    def step(self, dt, nsteps=1):
        _check(load().streamer_step(self._h, float(dt), int(nsteps)))

    def poisson(self, rho):
        phi = self._new()
        res, cyc = ctypes.c_double(), ctypes.c_int()
        _check(load().streamer_poisson(self._h, self._t(rho), self._t(phi), ctypes.byref(res), ctypes.byref(cyc)))
        return phi, res.value, cyc.value

    def info(self):
        lv, cyc, res = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(load().streamer_info(self._h, ctypes.byref(lv), ctypes.byref(cyc), ctypes.byref(res)))
        return dict(mg_levels=lv.value, last_cycles=cyc.value, last_residual=res.value)

    def close(self):
        if self._h:
            self.stream.synchronize()
            load().streamer_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
