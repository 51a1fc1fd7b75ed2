// Self-cell value sigma(h) of the discrete kernel G (i == j term, Sec. 3), device side.
#pragma once
#include "kernel.cuh"
#include <cuda_runtime.h>

#include "../../include/kifmm.h"

namespace kifmm {

// E1(x), x > 0: Abramowitz & Stegun 5.1.11 (power series) for x <= 1, and the
// continued fraction 5.1.22 in its even-contracted form, evaluated with the
// modified Lentz method, for x > 1.
__device__ __forceinline__ double e1_dev(double x) {
    if (x <= 1.0) {
        double s = 0.0, term = 1.0;
        for (int n = 1; n < 60; ++n) {
            term *= -x / n;
            double add = -term / n;
            s += add;
            if (fabs(add) < 1e-18 * fmax(1.0, fabs(s))) break;
        }
        return -0.57721566490153286061 - log(x) + s;
    }
    const double tiny = 1e-300;
    double bq = x + 1.0, c = 1.0 / tiny, d = 1.0 / bq, h = d;
    for (int i = 1; i < 10000; ++i) {
        double an = -(double)i * i;
        bq += 2.0;
        d = 1.0 / (an * d + bq);
        c = bq + an / c;
        double del = c * d;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    return h * exp(-x);
}

// Node i of the n-point Gauss-Legendre rule on [-1, 1], by Newton's method on the
// three-term recurrence of the Legendre polynomials.
__device__ __forceinline__ void gl_node(int n, int i, double* x, double* w) {
    double z = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
    double pp = 0;
    for (int it = 0; it < 100; ++it) {
        double p1 = 1.0, p2 = 0.0;
        for (int k = 1; k <= n; ++k) {
            double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
        }
        pp = n * (z * p1 - p2) / (z * z - 1.0);
        double z1 = z;
        z = z1 - p1 / pp;
        if (fabs(z - z1) < 1e-16) break;
    }
    *x = -z;
    *w = 2.0 / ((1.0 - z * z) * pp * pp);
}

// sigma(h) for one cell edge, computed by a block of 256 threads (red: 256 doubles of
// shared memory); the value is returned to thread 0.
//  cell_exact: 6 * sum_{ij} w_i w_j (h/2)/R^3 F(R) / (4 pi ln(b/a)), R = sqrt(u_i^2 + u_j^2 + h^2/4),
//              u = (h/2) t, F(R) = ln(b/a) + E1(bR) - E1(aR), tensor Gauss-Legendre (gx, gw; nq nodes);
//  paper_gl2:  the paper's 2-point Gauss-Legendre value h^3 * 3 g(rho) / (pi * 3h^2), rho = h/2.
__device__ __forceinline__ double self_sigma_block(double h, double a, double b, int mode, int nq,
                                                   const double* gx, const double* gw, double* red) {
    const double lba = log(b / a);
    if (mode == KIFMM_SELF_PAPER_GL2) {
        double s2 = 3.0 * h * h;
        double rho = sqrt(s2 / 12.0);
        double g = (exp(-a * rho) - exp(-b * rho)) / (rho * lba);
        return h * h * h * 3.0 * g / (3.14159265358979323846 * s2);
    }
    double acc = 0;
    for (int e = threadIdx.x; e < nq * nq; e += blockDim.x) {
        int i = e / nq, j = e % nq;
        double ui = 0.5 * h * gx[i], uj = 0.5 * h * gx[j];
        double wi = 0.5 * h * gw[i], wj = 0.5 * h * gw[j];
        double R = sqrt(ui * ui + uj * uj + 0.25 * h * h);
        double F = lba + e1_dev(b * R) - e1_dev(a * R);
        acc += wi * wj * (0.5 * h) / (R * R * R) * F;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    return 6.0 * red[0] / (4.0 * 3.14159265358979323846 * lba);
}

// sigma for a rectangular cell hx x hy x hz (the same block reduction): cell_exact: the
// solid-angle form face pair by face pair, sum_k 2 int (h_k/2)/R^3 F(R) du dv over the other
// two half-widths, R = sqrt(u^2 + v^2 + h_k^2/4), divided by 4 pi ln(b/a); paper_gl2: the
// paper's discrete self value hx hy hz 3 g(rho) / (pi sum h^2), rho = sqrt(sum h^2 / 12).
__device__ __forceinline__ double self_sigma_box_block(double hx, double hy, double hz, double a, double b, int mode,
                                                       int nq, const double* gx, const double* gw, double* red) {
    const double lba = log(b / a);
    if (mode == KIFMM_SELF_PAPER_GL2) {
        const double s2 = hx * hx + hy * hy + hz * hz;
        const double rho = sqrt(s2 / 12.0);
        const double g = (exp(-a * rho) - exp(-b * rho)) / (rho * lba);
        return hx * hy * hz * 3.0 * g / (3.14159265358979323846 * s2);
    }
    const double hs[3] = {hx, hy, hz};
    double acc = 0;
    for (int e = threadIdx.x; e < 3 * nq * nq; e += blockDim.x) {
        const int k = e / (nq * nq), i = (e / nq) % nq, j = e % nq;
        const double hk = hs[k], hi = hs[(k + 1) % 3], hj = hs[(k + 2) % 3];
        const double ui = 0.5 * hi * gx[i], uj = 0.5 * hj * gx[j];
        const double wi = 0.5 * hi * gw[i], wj = 0.5 * hj * gw[j];
        const double R = sqrt(ui * ui + uj * uj + 0.25 * hk * hk);
        const double F = lba + e1_dev(b * R) - e1_dev(a * R);
        acc += 2.0 * wi * wj * (0.5 * hk) / (R * R * R) * F;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    return red[0] / (4.0 * 3.14159265358979323846 * lba);
}

// sigma of an hx x hy x hz cell for any kernel kind (the same block reduction): cell_exact by
// the face-flux form, sum over the face pairs of 2 int (h_k/2) / R^3 m(R) du dv with
// m(R) = int_0^R K r^2 dr (kern_mass); paper_gl2: hx hy hz K(rho), rho = sqrt(sum h^2 / 12).
__device__ __forceinline__ double self_sigma_kind_block(double hx, double hy, double hz, const KParams& kp, int mode,
                                                        int nq, const double* gx, const double* gw, double* red) {
    if (mode == KIFMM_SELF_PAPER_GL2) return hx * hy * hz * kern_f64(sqrt((hx * hx + hy * hy + hz * hz) / 12.0), kp);
    const double hs[3] = {hx, hy, hz};
    double acc = 0;
    for (int e = threadIdx.x; e < 3 * nq * nq; e += blockDim.x) {
        const int k = e / (nq * nq), i = (e / nq) % nq, j = e % nq;
        const double hk = hs[k], hi = hs[(k + 1) % 3], hj = hs[(k + 2) % 3];
        const double ui = 0.5 * hi * gx[i], uj = 0.5 * hj * gx[j];
        const double wi = 0.5 * hi * gw[i], wj = 0.5 * hj * gw[j];
        const double R = sqrt(ui * ui + uj * uj + 0.25 * hk * hk);
        acc += 2.0 * wi * wj * (0.5 * hk) / (R * R * R) * kern_mass(R, kp, [](double x) { return e1_dev(x); });
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    return red[0];
}

}  // namespace kifmm
