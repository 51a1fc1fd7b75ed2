"""Seeded synthetic inputs: cell-centred point sets, cell sizes and source fields.

This module holds no arithmetic of the photoionization method: it only builds
coordinates, cell edges and source values, and it is shared by the oracle and
the CUDA path so that both see the same inputs. Every random draw comes from a
numpy PCG64 generator seeded by the caller.

Shapes follow the paper's workloads (Sec. 4): cell centres of uniform grids on a
box, and a Gaussian emission source; the adaptive case is a two-level refined
grid with a streamer-shaped source (a thin channel with a Gaussian head).
"""
import numpy as np


def uniform_grid(n, L=1.0, n_xyz=None, Lxyz=None):
    """Cell centres of an n x n x n grid on [0, L]^3 (x fastest), and the cell edge.
    ``n_xyz``/``Lxyz`` give a box grid instead; its cells must be cubic."""
    if n_xyz is None:
        n_xyz = (n, n, n)
    if Lxyz is None:
        Lxyz = (L, L, L)
    hs = [Lxyz[k] / n_xyz[k] for k in range(3)]
    if max(hs) - min(hs) > 1e-12 * max(hs):
        raise ValueError("cells must be cubic")
    h = hs[0]
    g = [(np.arange(n_xyz[k], dtype=np.float64) + 0.5) * hs[k] for k in range(3)]
    z, y, x = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    return pts, h


def gaussian(points, centre, sigma, amp):
    d2 = ((points - np.asarray(centre, dtype=np.float64)[None, :]) ** 2).sum(1)
    return amp * np.exp(-d2 / sigma ** 2)


def multipeak(points, dims, amp=1.53e25, k=50.0):
    """Multi-peak source of Sec. 4.3 (Eq. (multipeaksource)): amp sin^2(k pi x) sin^2(k pi y)
    sin^2(k pi z) inside the middle half [d/4, 3d/4] of the domain along every axis (d =
    ``dims``), zero outside."""
    d = np.asarray(dims, dtype=np.float64)[None, :]
    inside = np.all((points >= 0.25 * d) & (points <= 0.75 * d), axis=1)
    v = amp * np.prod(np.sin(k * np.pi * points) ** 2, axis=1)
    return np.where(inside, v, 0.0)


def refined_grid(L=2.0, base_n=128, fine_factor=8, centre=(1.0, 1.0, 1.5), half_cells=6):
    """Two-level grid: base cells of edge L/base_n, and in the block of
    (2*half_cells+1)^3 base cells around ``centre`` each base cell replaced by
    fine_factor^3 fine cells. Returns points, per-point cell edge."""
    hb = L / base_n
    kc = np.floor(np.asarray(centre) / hb).astype(np.int64)
    lo = kc - half_cells
    hi = kc + half_cells + 1
    g = np.arange(base_n)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    idx = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    inside = np.all((idx >= lo[None, :]) & (idx < hi[None, :]), axis=1)
    base = (idx[~inside] + 0.5) * hb
    hf = hb / fine_factor
    nf = (hi - lo) * fine_factor
    gf = [(np.arange(nf[k]) + 0.5) * hf + lo[k] * hb for k in range(3)]
    zf, yf, xf = np.meshgrid(gf[2], gf[1], gf[0], indexing="ij")
    fine = np.stack([xf.ravel(), yf.ravel(), zf.ravel()], axis=1)
    pts = np.concatenate([base, fine], axis=0)
    h = np.concatenate([np.full(base.shape[0], hb), np.full(fine.shape[0], hf)])
    return pts, h


def streamer_source(points, axis_xy=(1.0, 1.0), z_range=(0.5, 1.5), radius=0.05, i_channel=1e21,
                    head=(1.0, 1.0, 1.5), head_sigma=0.02, i_head=1e23, noise_sigma=0.3, seed=2006,
                    tilt_deg=0.0):
    """Thin cylindrical channel (Gaussian profile across the axis, on z in
    z_range) plus a Gaussian head, times seeded log-normal noise of unit median."""
    p = np.asarray(points, dtype=np.float64)
    th = np.deg2rad(tilt_deg)
    # coordinates in the channel frame (tilted about y through the channel's base)
    base = np.array([axis_xy[0], axis_xy[1], z_range[0]])
    rel = p - base[None, :]
    ax = np.array([np.sin(th), 0.0, np.cos(th)])
    along = rel @ ax
    perp2 = (rel ** 2).sum(1) - along ** 2
    length = z_range[1] - z_range[0]
    on = (along >= 0.0) & (along <= length)
    I = np.where(on, i_channel * np.exp(-perp2 / radius ** 2), 0.0)
    I = I + gaussian(p, head, head_sigma, i_head)
    if noise_sigma > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        I = I * np.exp(noise_sigma * rng.standard_normal(p.shape[0]))
    return I


def config_uniform(n, sigma=0.1, amp=1e22, L=1.0):
    """Uniform n^3 grid on [0, L]^3 with the centred Gaussian source
    amp * exp(-|r - c|^2 / sigma^2)."""
    pts, h = uniform_grid(n, L)
    I = gaussian(pts, (0.5 * L, 0.5 * L, 0.5 * L), sigma, amp)
    return pts, np.full(pts.shape[0], h), I


def config_adaptive(base_n=128, half_cells=6, seed=2006):
    """2 cm cube, base h = 1/64 cm, 8x finer cells in the block of 13^3 base cells
    around the streamer head at (1, 1, 1.5) cm; channel + head + log-normal noise."""
    pts, h = refined_grid(2.0, base_n, 8, (1.0, 1.0, 1.5), half_cells)
    I = streamer_source(pts, seed=seed)
    return pts, h, I


def random_cloud(n, seed, L=1.0, h=None):
    """Distinct random points in [0, L]^3 (tests of the tree on irregular sets)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((n, 3)) * L
    if h is None:
        h = L / max(2.0, round(n ** (1 / 3)))
    return pts, np.full(n, h), rng.random(n) + 0.1


def two_channel_field(k, n_min=80, n_max=158, base_seed=3515):
    """Field k of the batched workload: a uniform n^3 grid on [0, 1]^3 with n drawn from
    N = n^3 log-uniform in [n_min^3, n_max^3]; two streamer channels of length 0.5 cm
    centred at z = 0.5, at x = 0.5 -/+ d/2 (d ~ U[0.2, 0.8] cm), the second tilted by
    theta ~ U[0, 30] degrees about y, each with a Gaussian head at its upper tip; pressure
    drawn from {760, 76} Torr. Returns (points, h, I, p_torr)."""
    rng = np.random.Generator(np.random.PCG64(base_seed + k))
    logN = rng.uniform(3 * np.log(n_min), 3 * np.log(n_max))
    n = int(round(np.exp(logN / 3.0)))
    d = rng.uniform(0.2, 0.8)
    theta = rng.uniform(0.0, 30.0)
    p = float(rng.choice([760.0, 76.0]))
    pts, h = uniform_grid(n, 1.0)
    x1, x2 = 0.5 - d / 2, 0.5 + d / 2
    I = streamer_source(pts, axis_xy=(x1, 0.5), z_range=(0.25, 0.75), radius=0.05, i_channel=1e21,
                        head=(x1, 0.5, 0.75), head_sigma=0.02, i_head=1e23, noise_sigma=0.0)
    th = np.deg2rad(theta)
    head2 = (x2 + 0.5 * np.sin(th), 0.5, 0.25 + 0.5 * np.cos(th))
    I = I + streamer_source(pts, axis_xy=(x2, 0.5), z_range=(0.25, 0.75), radius=0.05, i_channel=1e21,
                            head=head2, head_sigma=0.02, i_head=1e23, noise_sigma=0.0, tilt_deg=theta)
    return pts, np.full(len(pts), h), I, p


PRESSURES = {  # p (Torr) -> p_O2 (Torr); p_O2 = 0.2 p except the paper's 150 Torr at 760
    "760/150": (760.0, 150.0),
    "760": (760.0, 152.0),
    "76": (76.0, 15.2),
    "7.6": (7.6, 1.52),
}


def surrogate_field(points, seed, L=1.0):
    """Training and test field of the learned surrogate: 1-5 Gaussian blobs (count uniform),
    widths log-uniform in [0.02, 0.2] cm, amplitudes log-uniform in [1e20, 1e23] cm^-3 s^-1,
    centres uniform in [0.1, 0.9]^3 cm (scaled by L)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = int(rng.integers(1, 6))
    I = np.zeros(points.shape[0])
    for _ in range(k):
        c = L * rng.uniform(0.1, 0.9, 3)
        s = L * float(np.exp(rng.uniform(np.log(0.02), np.log(0.2))))
        amp = 10.0 ** rng.uniform(20.0, 23.0)
        I += gaussian(points, c, s, amp)
    return I


def gaussian_mixture(points, seed, n_blobs=(1, 4), sigma=(0.03, 0.12), log10_amp=(20.0, 23.0), L=1.0):
    """Sum of 1-4 Gaussian blobs with centres uniform in the inner 80 % of [0, L]^3, widths
    uniform in ``sigma`` (cm) and amplitudes log-uniform in 10^log10_amp (training fields of
    the surrogate)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = int(rng.integers(n_blobs[0], n_blobs[1] + 1))
    I = np.zeros(points.shape[0])
    for _ in range(k):
        c = L * (0.1 + 0.8 * rng.random(3))
        s = rng.uniform(*sigma)
        amp = 10.0 ** rng.uniform(*log10_amp)
        I += gaussian(points, c, s, amp)
    return I
