"""The FMM against the whole discrete sum at the sizes of the paper's own accuracy study
(marked gpu).

Sec. 4.1 (one Gaussian source; a 0.4 x 0.4 x 0.2 cm box with sigma = 0.01 cm and a box
ten times smaller with sigma = 0.001 cm) and Sec. 4.3 (the multi-peak source in the
larger box): 320 x 320 x 160 cubic cells (16,384,000 points), p = 760 Torr,
p_O2 = 150 Torr, m0 = 6, leaves of at most 128 points (125-cell leaves). The reference
is the discrete sum of Eq. (integral) over every cell, from the oracle's FFT convolution with the kernel table; the errors are E_V and
E_delta(x0) of Eq. (relativefun), delta = 5 sigma (Sec. 4.1) or 0.05 cm (Sec. 4.3). The
paper's FMM reaches E_V = 0.21 %, 0.22 %, 0.69 % and E_delta = 1.30 %, 0.53 %, 0.82 %
on these cases (Tables tonegaussiansrc001, tonegaussiansrc0001, tmultipeak). The surface
form with the pseudo-inverse cut-off eps = 1e-5 measures E_V = 1.2-2.2 % and E_delta =
2.7-7.1 % here (a few times the paper's figures; the paper does not state its leaf size
or regulariser) and is held to E_V <= 3 %, E_delta <= 10 %; its mixed form to 1e-6 of its
FP64 form; the Chebyshev option (p = 8, mixed) measures E_V about 1e-6 and is held to
E_V, E_delta <= 1e-5.
"""
import numpy as np
import pytest

from oracle import direct as D
from oracle import kernel as K
from paper_2006_03515_gb300 import workloads as W
from golden import read as G

pytestmark = pytest.mark.gpu

SHAPE = (320, 320, 160)      # cells along x, y, z
CASES = {
    "gaussian_0.4cm": ((0.4, 0.4, 0.2), 0.01, 0.05),
    "gaussian_0.04cm": ((0.04, 0.04, 0.02), 0.001, 0.005),
    "multipeak_0.4cm": ((0.4, 0.4, 0.2), None, 0.05),
}


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _errors(s, ref, pts, x0, delta):
    e_v = float(np.linalg.norm(s - ref) / np.linalg.norm(ref))
    ball = ((pts - np.asarray(x0)[None, :]) ** 2).sum(1) <= delta * delta
    e_d = float(np.mean(np.abs(s[ball] - ref[ball]) / ref[ball]))
    return e_v, e_d


@pytest.mark.parametrize("case", sorted(CASES))
def test_paper_accuracy_full_size(kf, case):
    dims, sigma, delta = CASES[case]
    pts, h = W.uniform_grid(None, n_xyz=SHAPE, Lxyz=dims)
    x0 = tuple(0.5 * d for d in dims)
    I = W.gaussian(pts, x0, sigma, 1.53e25) if sigma else W.multipeak(pts, dims)
    a, b = K.absorption_coefficients(150.0)
    C = K.source_scale(760.0)
    ref = D.fft_uniform(I.reshape(SHAPE[2], SHAPE[1], SHAPE[0]), h, a, b, C).ravel()
    dp, Id = _dev(pts), _dev(I)
    out = {}
    for name, kw in [("fp64", dict(precision="fp64")), ("mixed", dict(precision="mixed")),
                     ("cheb8", dict(precision="mixed", repr="cheb"))]:
        m0 = 8 if name == "cheb8" else 6
        p = kf.Plan(dp, h, 128, m0, a, b, **kw)
        out[name] = p.eval(Id, C=C).cpu().numpy()
        p.close()
    e_v, e_d = _errors(out["fp64"], ref, pts, x0, delta)
    e_vc, e_dc = _errors(out["cheb8"], ref, pts, x0, delta)
    mixed = float(np.linalg.norm(out["mixed"] - out["fp64"]) / np.linalg.norm(out["fp64"]))
    paper_ev, paper_ed = G.paper_fmm_errors()[case]
    print("\n%s: surface m0=6 E_V %.3f %% E_delta %.3f %% (paper %.2f %%, %.2f %%); mixed vs fp64 %.2e; "
          "Chebyshev p=8 E_V %.2e %% E_delta %.2e %%" % (case, 100 * e_v, 100 * e_d, 100 * paper_ev, 100 * paper_ed,
                                                        mixed, 100 * e_vc, 100 * e_dc))
    assert e_v <= 3e-2 and e_d <= 1e-1
    assert mixed <= 1e-6
    assert e_vc <= 1e-5 and e_dc <= 1e-5
    # the Chebyshev option beats the paper's own FMM by two orders of magnitude or more
    assert e_vc <= paper_ev / 100 and e_dc <= paper_ed / 100
