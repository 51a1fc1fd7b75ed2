"""Training data and training loop of the spectral neural operator surrogate.

Fields I are seeded Gaussian mixtures on a uniform n^3 grid; their labels S are the
photoionization source computed by the GPU KIFMM (mixed form) at the given pressure.
The network learns u = log(1 + I) -> log(1 + S). The transforms of the labels run as
plain tensor arithmetic on the device; every network pass runs in the sno_* kernels.
"""
import numpy as np

from . import kifmm, workloads


def grid_plan(n, L=1.0, leaf=64, m0=6, p_torr=760.0, p_o2=150.0, precision="mixed", stream=None):
    """A KIFMM plan over the cell centres of the n^3 grid on [0, L]^3 (point index
    z*n^2 + y*n + x, the order the surrogate sees) and the source scale C."""
    import torch
    pts, h = workloads.uniform_grid(n, L)
    a, b = kifmm.absorption(p_o2)
    plan = kifmm.Plan(torch.as_tensor(pts, device="cuda"), h, leaf, m0, a, b, precision=precision, stream=stream)
    return plan, pts, kifmm.scale_c(p_torr)


def make_dataset(plan, pts, C, count, seed=0):
    """count (u, t) pairs as CUDA float32 tensors (count, n^3): u = log(1 + I) for seeded
    Gaussian-mixture fields, t = log(1 + S) with S from the plan's KIFMM evaluation."""
    import torch
    n3 = pts.shape[0]
    U = torch.empty((count, n3), dtype=torch.float32, device="cuda")
    T = torch.empty_like(U)
    S = torch.empty(n3, dtype=torch.float64, device="cuda")
    for k in range(count):
        I = torch.as_tensor(workloads.gaussian_mixture(pts, seed * 1000003 + k), device="cuda")
        plan.eval(I, S, C=C)
        U[k] = torch.log1p(I.clamp_min(0)).float()
        T[k] = torch.log1p(S.clamp_min(0)).float()
    return U, T


def init_from_data(model, U, T, seed=0):
    """Seeded initial parameters matched to the data's scale: the lift maps u to zero mean
    and unit variance, the output bias starts at the mean target and the last projection
    is small, so the first steps learn the field's shape rather than its offset."""
    import numpy as np
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
