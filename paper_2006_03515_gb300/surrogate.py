"""Training data and training loop of the spectral neural operator surrogate.

The map I -> S_ph is linear (Sec. 3, Eq. (summation)), so the surrogate works in the
amplitude-normalised form: u = I / max I, t = S / (C max I). Fields are seeded Gaussian
mixtures on a uniform n^3 grid (``workloads.surrogate_field``); their labels S come from the
GPU KIFMM of a plan over the grid. The model adds the exact near part of the sum
(``SNO.set_near_field``) and its network learns the smooth far part; ``init_far`` starts
the network at the far part's Fourier multiplier. The rescalings of inputs and labels run
as plain tensor arithmetic on the device; every network pass runs in the sno_* kernels.
"""
import numpy as np

from . import kifmm, workloads


def grid_plan(n, L=1.0, leaf=64, m0=6, p_torr=760.0, p_o2=150.0, precision="mixed", stream=None,
              surface_radii=None):
    """A KIFMM plan over the cell centres of the n^3 grid on [0, L]^3 (point index
    z*n^2 + y*n + x, the order the surrogate sees), the points, and the source scale C."""
    import torch
    pts, h = workloads.uniform_grid(n, L)
    a, b = kifmm.absorption(p_o2)
    plan = kifmm.Plan(torch.as_tensor(pts, device="cuda"), h, leaf, m0, a, b, precision=precision, stream=stream,
                      surface_radii=surface_radii)
    plan.grid = dict(n=n, h=h, a=a, b=b)
    return plan, pts, kifmm.scale_c(p_torr)


def make_dataset(plan, pts, C, count, seed=0, field=workloads.surrogate_field):
    """count (u, t) pairs as CUDA float32 tensors (count, n^3): u = I / max I for seeded
    fields I, t = S / (C max I) with S from the plan's KIFMM evaluation (factor C included)."""
    import torch
    n3 = pts.shape[0]
    U = torch.empty((count, n3), dtype=torch.float32, device="cuda")
    T = torch.empty_like(U)
    S = torch.empty(n3, dtype=torch.float64, device="cuda")
    for k in range(count):
        I = torch.as_tensor(field(pts, seed * 1000003 + k), device="cuda")
        plan.eval(I, S, C=C)
        s = float(I.abs().max())
        U[k] = (I / s).float()
        T[k] = (S / (C * s)).float()
    return U, T


def configure(model, plan, period=None, r_in=3.0, r_out=7.0):
    """Sets the model's period (default 1.5 times the grid: a zero band of half the grid
    beyond every face, so that the spectral convolution does not wrap around onto the
    kernel's range, with the kept modes still reaching a sixth of the grid's frequencies at
    12 modes on 64 cells) and its exact near part for the plan's kernel and cells."""
    g = plan.grid
    model.set_period(period if period is not None else (3 * g["n"]) // 2)
    model.set_near_field(g["a"], g["b"], g["h"], r_in, r_out)


def init_far(model, seed=0, rest_scale=1e-3, shift=8.0):
    """Seeded small random parameters, then channel 0 set to carry the far part's Fourier
    multiplier (sno_init_far_field); the other channels start small so that training can use
    them."""
    theta = model.init_params(seed) * np.float32(rest_scale)
    model.set_params(theta)
    model.init_far_field(shift)


def init_from_data(model, U, T, seed=0):
    """Seeded initial parameters matched to the data's scale: the lift maps u to zero mean
    and unit variance, the output bias starts at the mean target and the last projection
    is small, so the first steps learn the field's shape rather than its offset."""
    theta = model.init_params(seed)
    lay = model.layout()
    off, o = {}, 0
    for name, shp in lay:
        k = int(np.prod(shp))
        off[name] = (o, k)
        o += k
    mu, sd = float(U.mean()), float(U.std()) + 1e-6
    o, k = off["Wl"]
    theta[o:o + k] /= sd
    wl = theta[o:o + k].copy()
    o, k = off["bl"]
    theta[o:o + k] = -wl * mu
    o, k = off["Q2"]
    theta[o:o + k] *= 0.1
    o, k = off["q2"]
    theta[o:o + k] = float(T.mean())
    model.set_params(theta)
    return theta


def train(model, U, T, steps, batch=4, lr=1e-3, seed=0, log_every=0):
    """Adam on the mean squared error over random mini-batches; returns the loss history."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    hist = []
    ub = torch.empty((batch, U.shape[1]), dtype=torch.float32, device="cuda")
    tb = torch.empty_like(ub)
    for s in range(steps):
        idx = torch.as_tensor(rng.choice(U.shape[0], size=batch, replace=U.shape[0] < batch), device="cuda")
        torch.index_select(U, 0, idx, out=ub)
        torch.index_select(T, 0, idx, out=tb)
        hist.append(model.loss_grad(ub, tb))
        model.adam_step(lr)
        if log_every and s % log_every == 0:
            print("step %d loss %.4e" % (s, hist[-1]))
    return hist


def rel_errors(model, U, T, batch=8):
    """Relative L2 error of the model's output against T, field by field."""
    import torch
    out = []
    for k in range(0, U.shape[0], batch):
        ub = U[k:k + batch].contiguous()
        y = model.forward(ub)
        t = T[k:k + batch]
        out += (torch.linalg.norm(y - t, dim=1) / torch.linalg.norm(t, dim=1)).tolist()
    return out
