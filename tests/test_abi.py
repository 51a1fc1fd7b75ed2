"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/*.h declares, and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2006_03515_gb300 import build, kifmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ERR_ARG = -1


def _declared():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(hdr).read()
        names += re.findall(r"^\s*(?:int|int64_t|void|const char\s*\*)\s+(\w+)\s*\(", txt, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return kifmm.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(kifmm.EXPORTS) == names


def test_argtypes_match_the_header(lib):
    # every declared entry point: the binding passes as many arguments as the header takes
    hdr = open(os.path.join(ROOT, "include", "kifmm.h")).read()
    decls = re.findall(r"^\s*(?:int|int64_t|void|const char\s*\*)\s+(\w+)\s*\(([^;]*?)\)\s*;", hdr, re.M | re.S)
    assert len(decls) == len(_declared())
    for name, params in decls:
        params = re.sub(r"/\*.*?\*/", "", params, flags=re.S).strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(getattr(lib, name).argtypes or []) == n, name


def test_struct_layouts_match_the_header(tmp_path):
    # kifmm_opts and kifmm_info as the C compiler lays them out against the ctypes mirrors
    opts = [f[0] for f in kifmm._Opts._fields_]
    info = [f[0] for f in kifmm._Info._fields_]
    tune = [f[0] for f in kifmm._TuneEntry._fields_]
    strm = [f[0] for f in kifmm._StreamerParams._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "kifmm.h"', "int main(void) {"]
    src.append('printf("%zu\\n", sizeof(kifmm_opts));')
    src += ['printf("%%zu\\n", offsetof(kifmm_opts, %s));' % f for f in opts]
    src.append('printf("%zu\\n", sizeof(kifmm_info));')
    src += ['printf("%%zu\\n", offsetof(kifmm_info, %s));' % f for f in info]
    src.append('printf("%zu\\n", sizeof(kifmm_tune_entry));')
    src += ['printf("%%zu\\n", offsetof(kifmm_tune_entry, %s));' % f for f in tune]
    src.append('printf("%zu\\n", sizeof(streamer_params));')
    src += ['printf("%%zu\\n", offsetof(streamer_params, %s));' % f for f in strm]
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(kifmm._Opts)] + [getattr(kifmm._Opts, f).offset for f in opts]
    want += [ctypes.sizeof(kifmm._Info)] + [getattr(kifmm._Info, f).offset for f in info]
    want += [ctypes.sizeof(kifmm._TuneEntry)] + [getattr(kifmm._TuneEntry, f).offset for f in tune]
    want += [ctypes.sizeof(kifmm._StreamerParams)] + [getattr(kifmm._StreamerParams, f).offset for f in strm]
    assert got == want


def test_default_opts(lib):
    o = kifmm._Opts()
    lib.kifmm_default_opts(ctypes.byref(o))
    assert o.precision == kifmm.KIFMM_FP64
    assert o.self_mode == kifmm.KIFMM_SELF_CELL_EXACT
    assert o.pinv_eps == 1e-5 and o.has_root == 0 and not o.stream
    assert tuple(o.radii) == (1.05, 2.95)


def _plan(lib, **kw):
    args = dict(out=ctypes.byref(ctypes.c_void_p()), pts=ctypes.c_void_p(16), n=10, h=None, uh=0.1, leaf=8, m0=6,
                a=5.0, b=300.0, opts=None)
    args.update(kw)
    return lib.kifmm_plan(args["out"], args["pts"], args["n"], args["h"], args["uh"], args["leaf"], args["m0"],
                          args["a"], args["b"], args["opts"])


@pytest.mark.parametrize("kw", [dict(out=None), dict(pts=None), dict(n=0), dict(n=-3), dict(uh=0.0),
                                dict(uh=float("nan")), dict(leaf=0), dict(m0=2), dict(m0=13), dict(a=0.0),
                                dict(b=4.0), dict(a=float("inf"))])
def test_plan_rejects_bad_arguments(lib, kw):
    assert _plan(lib, **kw) == -1
    assert lib.kifmm_last_error().decode().startswith("kifmm_plan")


def test_plan_rejects_bad_options(lib):
    for field, value in [("precision", 7), ("self_mode", 3), ("pinv_eps", 0.0), ("pinv_eps", 1.5)]:
        o = kifmm._Opts()
        lib.kifmm_default_opts(ctypes.byref(o))
        setattr(o, field, value)
        assert _plan(lib, opts=ctypes.byref(o)) == -1
    o = kifmm._Opts()
    lib.kifmm_default_opts(ctypes.byref(o))
    o.has_root = 1
    o.root[3] = -1.0
    assert _plan(lib, opts=ctypes.byref(o)) == -1
    # surface radii: 1 < inner < outer < 3
    for radii in [(1.0, 2.6), (1.2, 1.1), (1.2, 3.0), (0.0, 2.6), (float("nan"), 2.6), (1.2, float("inf"))]:
        o = kifmm._Opts()
        lib.kifmm_default_opts(ctypes.byref(o))
        o.radii[0], o.radii[1] = radii
        assert _plan(lib, opts=ctypes.byref(o)) == -1
        assert "radii" in lib.kifmm_last_error().decode()


def test_eval_rejects_null(lib):
    assert lib.kifmm_eval(None, None, None, 1, 1.0) == -1
    assert lib.kifmm_eval_host(None, None, None, 1, 1.0) == -1
    assert lib.kifmm_get_info(None, None) == -1
    lib.kifmm_destroy(None)


def test_batch_rejects_bad_arguments(lib):
    vp = ctypes.c_void_p
    null = (vp * 2)(None, None)
    c = (ctypes.c_double * 2)(1.0, 1.0)
    for count, lanes in [(0, 1), (2, 0), (2, kifmm.KIFMM_MAX_LANES + 1), (-1, 2)]:
        assert lib.kifmm_eval_batch(null, null, null, count, 1, c, 0, lanes) == ERR_ARG
        assert "invalid argument" in lib.kifmm_last_error().decode()
    assert lib.kifmm_eval_batch(null, null, null, 2, 1, c, 1, 2) == ERR_ARG
    assert "NULL plan" in lib.kifmm_last_error().decode()
    hdr = open(os.path.join(ROOT, "include", "kifmm.h")).read()
    assert re.search(r"#define KIFMM_MAX_LANES (\d+)", hdr).group(1) == str(kifmm.KIFMM_MAX_LANES)


def test_physics_constants(lib):
    # Eq. (gfun) and Eq. (Ifun) with the parameters the paper prints (Sec. 2.1, Sec. 4.1),
    # computed by kifmm_model_constants behind the C-ABI
    from golden import read as G
    c = G.paper_constants()
    a, b = kifmm.absorption(c["p_O2"])
    assert a == pytest.approx(c["chi_min"] * c["p_O2"], rel=1e-15) and b == c["chi_max"] * c["p_O2"]
    assert a == pytest.approx(5.25, rel=1e-15) and b == 300.0
    C = c["xi"] * c["omega_over_alpha"] * c["p_q"] / (c["p"] + c["p_q"])
    assert kifmm.scale_c(c["p"]) == pytest.approx(C, rel=1e-15)
    a2, b2, C2 = kifmm.model_constants(c["p"], c["p_O2"], c["p_q"], c["xi"] * c["omega_over_alpha"])
    assert (a2, b2) == (a, b) and C2 == pytest.approx(C, rel=1e-15)
    d = ctypes.c_double()
    for bad in [(0.0, 150.0, 30.0, 0.06), (760.0, -1.0, 30.0, 0.06), (760.0, 150.0, float("nan"), 0.06),
                (760.0, 150.0, 30.0, float("inf"))]:
        assert lib.kifmm_model_constants(*bad, ctypes.byref(d), None, None) == ERR_ARG
        assert "kifmm_model_constants" in lib.kifmm_last_error().decode()


def test_tune_rejects_bad_arguments(lib):
    best = kifmm._TuneEntry()
    leaf = (ctypes.c_int * 1)(64)
    order = (ctypes.c_int * 1)(6)
    vp = ctypes.c_void_p
    for args in [(None, 10, None, 0.1, vp(8), 5.0, 300.0, None, leaf, 1, order, 1, None, 0, 1e-3, 64, 1),
                 (vp(8), 10, None, 0.1, None, 5.0, 300.0, None, leaf, 1, order, 1, None, 0, 1e-3, 64, 1),
                 (vp(8), 10, None, 0.1, vp(8), 5.0, 300.0, None, leaf, 0, order, 1, None, 0, 1e-3, 64, 1),
                 (vp(8), 10, None, 0.1, vp(8), 5.0, 300.0, None, leaf, 1, order, 1, None, 0, 0.0, 64, 1),
                 (vp(8), 10, None, 0.1, vp(8), 5.0, 300.0, None, leaf, 1, order, 1, None, 0, 1e-3, 5000, 1)]:
        assert lib.kifmm_tune(*args, None, ctypes.byref(best)) == ERR_ARG
        assert lib.kifmm_last_error().decode().startswith("kifmm_tune")


def test_check_rejects_null(lib):
    assert lib.kifmm_check(None) == ERR_ARG
    assert lib.kifmm_last_error().decode().startswith("kifmm_check")


def test_sno_rejects_bad_sizes_on_the_host(lib):
    h = ctypes.c_void_p()
    for n, width, modes, layers, proj, mb in [(3, 4, 1, 1, 4, 1), (8, 65, 2, 1, 4, 1), (8, 4, 5, 1, 4, 1),
                                              (8, 4, 0, 1, 4, 1), (8, 4, 2, 0, 4, 1), (8, 4, 2, 1, 129, 1),
                                              (8, 4, 2, 1, 4, 0)]:
        assert lib.sno_create(ctypes.byref(h), n, width, modes, layers, proj, mb, None) == ERR_ARG
        assert not h.value
    assert lib.sno_num_params(None) == -1
    assert lib.sno_forward(None, None, None, 1) == ERR_ARG
    assert lib.sno_loss_grad(None, None, None, 1, None) == ERR_ARG
    assert lib.sno_save(None, b"x") == ERR_ARG
    assert lib.sno_save_checkpoint(None, b"x") == ERR_ARG and lib.sno_load_checkpoint(None, b"x") == ERR_ARG
    assert lib.photo_solve(None, None, None, None, 1.0, 1e-2, 256, 0, None, None) == ERR_ARG
