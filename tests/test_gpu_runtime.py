"""Runtime behaviour of the C-ABI on the GPU (marked gpu): device-side error reporting,
the batch graph's replay rule, and the argument checks of the no-allocation sum.

The device error word is set on the host (KIFMM_INJECT_DEVICE_ERROR at plan time), as if
a bounded tensor-core wait had given up; no device wait is made to run out.
"""
import numpy as np
import pytest

from oracle import kernel as K
from paper_2006_03515_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_device_error_word_reported_as_timeout(kf, monkeypatch):
    pts, h, I = W.config_uniform(16)
    a, b = K.absorption_coefficients(152.0)
    ref = kf.Plan(_dev(pts), float(h[0]), 8, 6, a, b, precision="mixed").eval(_dev(I)).cpu().numpy()
    monkeypatch.setenv("KIFMM_INJECT_DEVICE_ERROR", "1")
    p = kf.Plan(_dev(pts), float(h[0]), 8, 6, a, b, precision="mixed")
    q = kf.Plan(_dev(pts), float(h[0]), 8, 6, a, b, precision="mixed")
    monkeypatch.delenv("KIFMM_INJECT_DEVICE_ERROR")
    # the host-buffer evaluation reads the word after its synchronisation
    with pytest.raises(kf.KifmmError) as e:
        p.eval_host(I)
    assert e.value.code == -4 and "bounded device wait" in str(e.value)
    # reported once: the word is cleared, the next evaluation is valid
    np.testing.assert_allclose(p.eval_host(I), ref, rtol=1e-12, atol=0)
    p.check()
    # the asynchronous evaluation leaves the report to kifmm_check
    q.eval(_dev(I))
    with pytest.raises(kf.KifmmError) as e:
        q.check()
    assert e.value.code == -4
    q.check()
    assert q.info()["device_error"] == 0


def test_batch_replay_follows_new_scale_factors(kf):
    # C is an argument of the captured kernels: a call with new C values records a new graph
    import torch
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plans, Is = [], []
        for n, po2 in [(12, 152.0), (16, 15.2)]:
            pts, h, I = W.config_uniform(n)
            a, b = K.absorption_coefficients(po2)
            plans.append(kf.Plan(_dev(pts), float(h[0]), 16, 4, a, b, precision="mixed", stream=st))
            Is.append(_dev(I))
        Ss = [torch.empty_like(x) for x in Is]
        for C in ([1.0, 2.0], [1.0, 2.0], [3.0, 0.5], [3.0, 0.5]):
            kf.eval_batch(plans, Is, Ss, C=C, capture=True, lanes=2)
            st.synchronize()
            for pl, x, s, c in zip(plans, Is, Ss, C):
                ref = pl.eval(x, C=c)
                st.synchronize()
                assert torch.allclose(s, ref, rtol=1e-12, atol=0)


def test_batch_replay_after_destroy_and_recreate(kf):
    # a plan destroyed and recreated (possibly at the same address) is a new plan: the
    # cached graph of the old one is not replayed on it
    import torch
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        pts0, h0, I0 = W.config_uniform(12)
        a, b = K.absorption_coefficients(152.0)
        p0 = kf.Plan(_dev(pts0), float(h0[0]), 16, 4, a, b, precision="mixed", stream=st)
        I0d = _dev(I0)
        S0 = torch.empty_like(I0d)
        pts1, h1, I1 = W.config_uniform(14)
        I1d = _dev(I1)
        S1 = torch.empty_like(I1d)
        for po2 in (152.0, 15.2, 1.52):
            a1, b1 = K.absorption_coefficients(po2)
            p1 = kf.Plan(_dev(pts1), float(h1[0]), 16, 4, a1, b1, precision="mixed", stream=st)
            for _ in range(2):
                kf.eval_batch([p0, p1], [I0d, I1d], [S0, S1], capture=True, lanes=2)
                st.synchronize()
                assert torch.allclose(S1, p1.eval(I1d), rtol=1e-12, atol=0)
                assert torch.allclose(S0, p0.eval(I0d), rtol=1e-12, atol=0)
            p1.close()


def test_direct_noalloc_checks_its_tensors(kf):
    import torch
    pts, h = W.uniform_grid(6, 0.2)
    dp = _dev(pts)
    I = torch.ones(len(pts), dtype=torch.float64, device="cuda")
    a, b = K.absorption_coefficients(150.0)
    with pytest.raises(TypeError):
        kf.direct_noalloc(dp, h, I.float(), a, b)                       # FP32 source
    with pytest.raises(TypeError):
        kf.direct_noalloc(dp, h, I[:-1], a, b)                          # too short
    with pytest.raises(TypeError):
        kf.direct_noalloc(dp.t().contiguous().t(), h, I, a, b)          # not contiguous
    with pytest.raises(TypeError):
        kf.direct_noalloc(dp.cpu(), h, I, a, b)                         # host tensor
    with pytest.raises(TypeError):
        kf.direct_noalloc(dp, h, I, a, b, S=torch.empty(len(pts), dtype=torch.float32, device="cuda"))
    S = kf.direct_noalloc(dp, h, I, a, b)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(S).all())


def test_near_sums_stream_changes_no_bit(kf, monkeypatch):
    # the lattice near sums run on the plan's second stream (forked at the M2L by default,
    # after the scatter with KIFMM_NEAR_STREAM=early) or on its own stream (=same): the same
    # kernels on the same data, so every result is bit-identical, alone, from host buffers
    # and in a captured batch on two lanes; the forked plans report the near sums' span as an
    # eighth phase time
    import torch
    pts, h, I = W.config_uniform(32)
    a, b = K.absorption_coefficients(152.0)
    st = torch.cuda.Stream()
    monkeypatch.setenv("KIFMM_TIMING", "1")
    with torch.cuda.stream(st):
        dp, dI = _dev(pts), _dev(I)
        plans = {}
        for mode in ("default", "early", "same"):
            if mode == "default":
                monkeypatch.delenv("KIFMM_NEAR_STREAM", raising=False)
            else:
                monkeypatch.setenv("KIFMM_NEAR_STREAM", mode)
            plans[mode] = kf.Plan(dp, float(h[0]), 64, 6, a, b, precision="mixed", stream=st)
        monkeypatch.delenv("KIFMM_NEAR_STREAM", raising=False)
        assert all(p.info()["near_tensor"] for p in plans.values())
        out = {m: p.eval(dI) for m, p in plans.items()}
        st.synchronize()
        ref = out["same"].cpu().numpy()
        for m in ("default", "early"):
            assert np.array_equal(out[m].cpu().numpy(), ref), m
            assert len(plans[m].phase_times()) == 8
        assert len(plans["same"].phase_times()) == 7
        assert np.array_equal(plans["default"].eval_host(I), ref)
        Ss = [torch.empty_like(dI) for _ in range(3)]
        for _ in range(2):   # recorded, then replayed
            kf.eval_batch([plans["default"], plans["early"], plans["same"]], [dI] * 3, Ss, capture=True, lanes=2)
            st.synchronize()
            for s in Ss:
                assert np.array_equal(s.cpu().numpy(), ref)
        for p in plans.values():
            p.close()
