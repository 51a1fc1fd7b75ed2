"""The accuracy-targeted autotuner kifmm_tune on the GPU (marked gpu): the setting it returns
meets the caller's target against the whole discrete sum (the oracle's FFT convolution), and it
is the fastest of the candidates the tuner accepted; its error estimates (FP64 direct sum at
importance-sampled targets) follow the candidates' true errors."""
import numpy as np
import pytest

from oracle import direct as D
from oracle import kernel as K
from paper_2006_03515_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("target", [2e-3, 3e-2])
def test_tune_meets_the_target(kf, target):
    n = 48
    pts, h, I = W.config_uniform(n)
    a, b = K.absorption_coefficients(152.0)
    ref = D.fft_uniform(I.reshape(n, n, n), h[0], a, b).ravel()
    dp, dI = _dev(pts), _dev(I)
    radii = [(1.05, 2.95), (1.2, 2.6)]
    best, tab = kf.tune(dp, float(h[0]), dI, a, b, leaf=(32, 64), order=(4, 6, 8), radii=radii, target=target,
                        reps=2)
    assert len(tab) == 2 * 3 * 2 and best["ok"]
    assert best["ms"] == min(e["ms"] for e in tab if e["ok"])
    p = kf.Plan(dp, float(h[0]), best["leaf"], best["order"], a, b, precision="mixed", surface_radii=best["radii"])
    got = p.eval(dI).cpu().numpy()
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert err <= target, (err, best)
    # the estimates follow the true errors of the candidates (sampling error well inside 2x)
    for e in tab[:4]:
        q = kf.Plan(dp, float(h[0]), e["leaf"], e["order"], a, b, precision="mixed", surface_radii=e["radii"])
        true = float(np.linalg.norm(q.eval(dI).cpu().numpy() - ref) / np.linalg.norm(ref))
        assert 0.5 * true <= e["err"] <= 2.0 * true, (e, true)
