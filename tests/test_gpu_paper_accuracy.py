"""The FMM against the whole discrete sum at the sizes of the paper's own accuracy study
(marked gpu).

Sec. 4.1 (one Gaussian source; a 0.4 x 0.4 x 0.2 cm box with sigma = 0.01 cm and a box ten
times smaller with sigma = 0.001 cm) and Sec. 4.3 (the multi-peak source in the larger box):
320 x 320 x 160 cubic cells (16,384,000 points), p = 760 Torr, p_O2 = 150 Torr. Sec. 4.2 (the
Gaussian source 4 pi xi c exp(-r^2 / sigma^2), sigma = 0.01 cm, in the 0.25 x 0.25 x 1.4 cm
box): 256 x 256 x 320 rectangular cells (20,971,520 points, cells 1 : 1 : 4.48), p_O2 = 160
and 10 Torr with p_O2 / p = 0.2. m0 = 6, leaves of at most 128 points. The reference is the
discrete sum of Eq. (integral) over every cell, from the oracle's FFT convolution with the
kernel table (cubic or rectangular cells); the errors are E_V and E_delta(x0) of Eq.
(relativefun), delta = 5 sigma (Sec. 4.1) or 0.05 cm (Sec. 4.2, 4.3).

The paper's FMM reaches E_V = 0.21, 0.22, 0.69, 0.15, 0.19 % and E_delta = 1.30, 0.53, 0.82,
1.24, 0.44 % on these cases (Tables tonegaussiansrc001, tonegaussiansrc0001, tmultipeak,
tdiffpi, tdiffpiii; tests/golden/paper_fmm_errors.txt). The surface form with its default
surfaces (1.05 / 2.95 r) measures E_V = 0.103, 0.122, 0.399, 0.097, 0.110 % and E_delta =
1.01, 0.145, 0.466, 1.11, 0.138 %: at or below the paper's figures on every case. The test
holds it to the paper's own figures and to 1.25 times its measured values; the mixed form to
1e-6 of the FP64 form; the Chebyshev option (p = 8, mixed) to E_V, E_delta <= 1e-5 (measured
4e-7 to 3e-6), two orders of magnitude below the paper's FMM.
"""
import numpy as np
import pytest

from oracle import direct as D
from oracle import kernel as K
from paper_2006_03515_gb300 import workloads as W
from golden import read as G

pytestmark = pytest.mark.gpu

# dims (cm), cells (x, y, z), sigma (cm; None: multi-peak), delta (cm), p_O2, p (Torr), source amplitude
CASES = {
    "gaussian_0.4cm": ((0.4, 0.4, 0.2), (320, 320, 160), 0.01, 0.05, 150.0, 760.0, 1.53e25),
    "gaussian_0.04cm": ((0.04, 0.04, 0.02), (320, 320, 160), 0.001, 0.005, 150.0, 760.0, 1.53e25),
    "multipeak_0.4cm": ((0.4, 0.4, 0.2), (320, 320, 160), None, 0.05, 150.0, 760.0, 1.53e25),
    "pressure_pO2_160": ((0.25, 0.25, 1.4), (256, 256, 320), 0.01, 0.05, 160.0, 800.0,
                         4 * np.pi * 0.1 * 2.99792458e10),
    "pressure_pO2_10": ((0.25, 0.25, 1.4), (256, 256, 320), 0.01, 0.05, 10.0, 50.0,
                        4 * np.pi * 0.1 * 2.99792458e10),
}
# the surface form's measured (E_V, E_delta) with the default surfaces
MEASURED = {
    "gaussian_0.4cm": (1.034e-3, 1.011e-2),
    "gaussian_0.04cm": (1.216e-3, 1.446e-3),
    "multipeak_0.4cm": (3.989e-3, 4.665e-3),
    "pressure_pO2_160": (9.65e-4, 1.108e-2),
    "pressure_pO2_10": (1.101e-3, 1.383e-3),
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
    dims, shape, sigma, delta, po2, p, amp = CASES[case]
    hs = [dims[k] / shape[k] for k in range(3)]
    rect = max(hs) - min(hs) > 1e-12 * max(hs)
    g = [(np.arange(shape[k]) + 0.5) * hs[k] for k in range(3)]
    zz, yy, xx = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    x0 = tuple(0.5 * d for d in dims)
    I = W.gaussian(pts, x0, sigma, amp) if sigma else W.multipeak(pts, dims)
    a, b = K.absorption_coefficients(po2)
    C = K.source_scale(p)
    I3 = I.reshape(shape[2], shape[1], shape[0])
    ref = (D.fft_box_grid(I3, hs, a, b, C) if rect else D.fft_uniform(I3, hs[0], a, b, C)).ravel()
    dp, Id = _dev(pts), _dev(I)
    cells = dict(cell_dims=tuple(hs)) if rect else {}
    hval = None if rect else hs[0]
    out = {}
    for name, kw in [("fp64", dict(precision="fp64")), ("mixed", dict(precision="mixed")),
                     ("cheb8", dict(precision="mixed", repr="cheb"))]:
        m0 = 8 if name == "cheb8" else 6
        pl = kf.Plan(dp, hval, 128, m0, a, b, **kw, **cells)
        out[name] = pl.eval(Id, C=C).cpu().numpy()
        pl.check()
        pl.close()
    e_v, e_d = _errors(out["fp64"], ref, pts, x0, delta)
    e_vc, e_dc = _errors(out["cheb8"], ref, pts, x0, delta)
    mixed = float(np.linalg.norm(out["mixed"] - out["fp64"]) / np.linalg.norm(out["fp64"]))
    paper_ev, paper_ed = G.paper_fmm_errors()[case]
    print("\n%s: surface m0=6 E_V %.3f %% E_delta %.3f %% (paper %.2f %%, %.2f %%); mixed vs fp64 %.2e; "
          "Chebyshev p=8 E_V %.2e %% E_delta %.2e %%" % (case, 100 * e_v, 100 * e_d, 100 * paper_ev, 100 * paper_ed,
                                                        mixed, 100 * e_vc, 100 * e_dc))
    mv, md = MEASURED[case]
    assert e_v <= min(paper_ev, 1.25 * mv) and e_d <= min(paper_ed, 1.25 * md), (e_v, e_d)
    assert mixed <= 1e-6
    assert e_vc <= 1e-5 and e_dc <= 1e-5
    # the Chebyshev option beats the paper's own FMM by two orders of magnitude or more
    assert e_vc <= paper_ev / 100 and e_dc <= paper_ed / 100
