"""kifmm_direct_noalloc: the direct sum without device allocation, for callers that cannot
allocate when they need S (inside a stream capture, in allocation-free real-time loops, or
with device memory owned by another allocator). Its output is checked against
kifmm_eval, whose plan with one leaf holding every point sums every pair directly. Two
calls in a row, with different sources, check that nothing stale from the first call's
use of the shared work space reaches the second. This file is collected last."""
import numpy as np
import pytest

from paper_2006_03515_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_direct_noalloc_matches_kifmm_eval(kf):
    import torch
    pts, h = W.uniform_grid(12, 0.4)                          # 1728 cells of edge 1/30 cm
    rng = np.random.default_rng(2006)
    a, b = kf.absorption(150.0)
    C = kf.scale_c(760.0)
    dp = torch.as_tensor(pts, device="cuda")
    ref_plan = kf.Plan(dp, h, leaf_size=len(pts), surface_order=6, a=a, b=b, precision="fp64")
    for call in range(2):
        I = torch.as_tensor(rng.random(len(pts)) * 1e22 * (call + 1), device="cuda")
        ref = ref_plan.eval(I, C=C)
        got = kf.direct_noalloc(dp, h, I, a, b, C=C)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
        assert err <= 1e-12, (call, err)


def test_direct_noalloc_rejects_oversize(kf):
    import torch
    n = kf.NOALLOC_MAX_POINTS + 1
    pts = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    I = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(kf.KifmmError) as e:
        kf.direct_noalloc(pts, 0.1, I, 5.0, 300.0)
    assert e.value.code == -1 and "exceeds" in str(e.value)
