// Streamer time loop (Sec. 5, Eq. (eM)): the drift-diffusion equations of electrons and
// positive ions, the Poisson equation of the potential, the impact ionization source S_i and
// the photoionization source S_ph, which the FMM evaluates twice per time step on a plan
// built once for the grid.
//
//   dn_e/dt - div(mu_e E n_e) - div(D_e grad n_e) = S_i + S_ph,
//   dn_p/dt + div(mu_p E n_p) = S_i + S_ph,
//   -Laplace(phi) = (e / eps0)(n_p - n_e),  E = -grad(phi),
//   S_i = mu_e n_e alpha(|E|) |E|,  alpha = 5.7 p exp(-260 p / |E|),
//   S_ph = C (sum_{j != i} K(|x_i - x_j|) S_i,j h^3 + sigma S_i,i)   (Eqs. (integral), (Ifun)).
//
// Cell-centred finite volumes on nx x ny x nz cubic cells of edge h, arrays [z][y][x]. phi = 0
// on the bottom face, phi0 on the top face, homogeneous Neumann conditions for phi on the side
// faces and for the densities on every face (boundary cells copied into the ghost layers).
// Drift fluxes from MUSCL face values with the Koren limiter, diffusion by central
// differences, Heun's two-stage explicit scheme in time. The Poisson equation is solved by
// geometric multigrid V-cycles (red-black Gauss-Seidel, full-weighting restriction of the
// residual, trilinear prolongation of the correction) until the relative residual is below
// the tolerance (1e-8 in Sec. 5), as iterative refinement: the potential and its residual in
// FP64, each V-cycle on the error equation in FP32 (this GPU's FP64 pipe is scarce; the FP64
// residual keeps the result at FP64 accuracy). The densities, fields and fluxes are FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

namespace kifmm {

namespace {

constexpr double kEoverEps0 = 1.602176634e-19 / 8.8541878128e-14;   // V cm

inline unsigned nbs(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct Grid {
    int nx, ny, nz;
    double h, ih, ih2;   // edge, 1 / h, 1 / h^2
    __host__ __device__ int64_t n() const { return (int64_t)nx * ny * nz; }
};
inline Grid make_grid(int nx, int ny, int nz, double h) { return Grid{nx, ny, nz, h, 1.0 / h, 1.0 / (h * h)}; }
// cell (i, j, k) of index c < 2^31 (32-bit arithmetic)
__device__ __forceinline__ void cell_ijk(const Grid& g, int c, int& i, int& j, int& k) {
    const int xy = g.nx * g.ny;
    k = c / xy;
    const int r = c - k * xy;
    j = r / g.nx;
    i = r - j * g.nx;
}

// ---- multigrid -------------------------------------------------------------------------
// diagonal of the discrete -Laplace(u) h^2 at cell (i, j, k): one per interior neighbour,
// two per z boundary face (Dirichlet at the face), none for a side boundary face (Neumann)
__device__ __forceinline__ double mg_diag(const Grid& g, int i, int j, int k) {
    double d = 0.0;
    d += (i > 0) + (i < g.nx - 1) + (j > 0) + (j < g.ny - 1);
    d += k > 0 ? 1.0 : 2.0;
    d += k < g.nz - 1 ? 1.0 : 2.0;
    return d;
}
// 1 / diagonal: the diagonal is an integer from 2 to 8 (a table instead of a division)
__device__ __forceinline__ double mg_rdiag(const Grid& g, int i, int j, int k) {
    const int d = (i > 0) + (i < g.nx - 1) + (j > 0) + (j < g.ny - 1) + (k > 0 ? 1 : 2) + (k < g.nz - 1 ? 1 : 2);
    constexpr double inv[9] = {0.0, 1.0, 0.5, 1.0 / 3.0, 0.25, 0.2, 1.0 / 6.0, 1.0 / 7.0, 0.125};
    return inv[d];
}
template <class T>
__device__ __forceinline__ T mg_nbsum(const Grid& g, const T* u, int i, int j, int k) {
    const int64_t sx = 1, sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const int64_t c = (int64_t)k * sz + (int64_t)j * sy + i;
    T s = 0;
    if (i > 0) s += u[c - sx];
    if (i < g.nx - 1) s += u[c + sx];
    if (j > 0) s += u[c - sy];
    if (j < g.ny - 1) s += u[c + sy];
    if (k > 0) s += u[c - sz];
    if (k < g.nz - 1) s += u[c + sz];
    return s;
}

// red-black Gauss-Seidel sweep of one colour: u = (b h^2 + sum of neighbours) / diag
template <class T>
__global__ void k_mg_smooth(Grid g, T* u, const T* b, int color) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    // the cells of one colour: two per pair along x
    const int hx = (g.nx + 1) / 2;
    if (e >= hx * g.ny * g.nz) return;
    const int k = e / (hx * g.ny), r = e - k * (hx * g.ny), j = r / hx;
    const int i = 2 * (r - j * hx) + ((j + k + color) & 1);
    if (i >= g.nx) return;
    const int64_t c = ((int64_t)k * g.ny + j) * g.nx + i;
    u[c] = (b[c] * (T)(g.h * g.h) + mg_nbsum(g, u, i, j, k)) * (T)mg_rdiag(g, i, j, k);
}

// r = b - A u, with A = -Laplace (including the z boundary faces' Dirichlet terms); r32 (when
// given) receives r rounded to FP32, the right-hand side of the FP32 error equation
template <class T>
__global__ void k_mg_residual(Grid g, const T* u, const T* b, T* r, float* r32) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.n()) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const T v = b[c] - ((T)mg_diag(g, i, j, k) * u[c] - mg_nbsum(g, u, i, j, k)) * (T)g.ih2;
    r[c] = v;
    if (r32) r32[c] = (float)v;
}

// u += e (the FP32 correction into the FP64 potential)
__global__ void k_mg_correct(int64_t n, const float* e, double* u) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) u[c] += (double)e[c];
}

// coarse right-hand side: the average of the 8 fine residuals of each coarse cell
template <class T>
__global__ void k_mg_restrict(Grid f, Grid cg, const T* r, T* bc) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cg.n()) return;
    int I, J, K;
    cell_ijk(cg, c, I, J, K);
    T s = 0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di)
                s += r[((int64_t)(2 * K + dk) * f.ny + (2 * J + dj)) * f.nx + (2 * I + di)];
    bc[c] = (T)0.125 * s;
}

// coarse value at integer coarse index (I, J, K) with the ghost rules of the correction:
// mirrored across the side faces (Neumann), negated across the z faces (zero at the face)
template <class T>
__device__ __forceinline__ T mg_coarse_at(const Grid& cg, const T* e, int I, int J, int K) {
    T sgn = 1;
    if (I < 0) I = 0;
    if (I >= cg.nx) I = cg.nx - 1;
    if (J < 0) J = 0;
    if (J >= cg.ny) J = cg.ny - 1;
    if (K < 0) {
        K = 0;
        sgn = -1;
    }
    if (K >= cg.nz) {
        K = cg.nz - 1;
        sgn = -1;
    }
    return sgn * e[((int64_t)K * cg.ny + J) * cg.nx + I];
}

// u_fine += trilinear interpolation of the coarse correction (cell-centred: weights 3/4 and
// 1/4 per axis towards the nearer coarse neighbour)
template <class T>
__global__ void k_mg_prolong(Grid f, Grid cg, const T* e, T* u) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= f.n()) return;
    const int i = (int)(c % f.nx), j = (int)((c / f.nx) % f.ny), k = (int)(c / ((int64_t)f.nx * f.ny));
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int oi = (i & 1) ? 1 : -1, oj = (j & 1) ? 1 : -1, ok = (k & 1) ? 1 : -1;
    T s = 0;
    for (int a = 0; a < 2; ++a)
        for (int b2 = 0; b2 < 2; ++b2)
            for (int d = 0; d < 2; ++d) {
                const T w = (T)((a ? 0.25 : 0.75) * (b2 ? 0.25 : 0.75) * (d ? 0.25 : 0.75));
                s += w * mg_coarse_at(cg, e, I + a * oi, J + b2 * oj, K + d * ok);
            }
    u[c] += s;
}

// the coarsest level: many red-black sweeps in one block
template <class T>
__global__ void k_mg_coarse_solve(Grid g, T* u, const T* b, int sweeps) {
    const int64_t n = g.n();
    for (int s = 0; s < sweeps; ++s)
        for (int color = 0; color < 2; ++color) {
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                int i, j, k;
                cell_ijk(g, c, i, j, k);
                if (((i + j + k) & 1) != color) continue;
                u[c] = (b[c] * (T)(g.h * g.h) + mg_nbsum(g, u, i, j, k)) * (T)mg_rdiag(g, i, j, k);
            }
            __syncthreads();
        }
}

// partial sums of squares (block-level), for the residual norm
__global__ void k_sumsq(const double* x, int64_t n, double* out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        s += x[e] * x[e];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// ---- fields and transport -------------------------------------------------------------
// b = (e / eps0)(n_p - n_e), plus the top face's Dirichlet term 2 phi0 / h^2
__global__ void k_sd_charge(Grid g, const double* ne, const double* np, double phi0, double* b) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.n()) return;
    const int k = c / (g.nx * g.ny);
    b[c] = kEoverEps0 * (np[c] - ne[c]) + (k == g.nz - 1 ? 2.0 * phi0 * g.ih2 : 0.0);
}

// E on the face between cells c - s and c along an axis of m cells (f = 0..m: face index)
__device__ __forceinline__ double face_E(const double* phi, int64_t c_lo, int64_t stride, int f, int m, double ih,
                                         bool zaxis, double phi0) {
    if (f > 0 && f < m) return -(phi[c_lo + stride] - phi[c_lo]) * ih;
    if (!zaxis) return 0.0;                                         // side faces: Neumann
    if (f == 0) return -(phi[c_lo + stride] - 0.0) * (2.0 * ih);   // bottom electrode, phi = 0
    return -(phi0 - phi[c_lo]) * (2.0 * ih);                        // top electrode, phi = phi0
}

// |E| at the cell centres (averages of each component's two faces) and S_i = mu_e n_e alpha |E|
__global__ void k_sd_source(Grid g, const double* phi, double phi0, const double* ne, double mu_e, double p,
                            double* Emag, double* Si) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.n()) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const double ex = 0.5 * (face_E(phi, c - 1, 1, i, g.nx, g.ih, false, phi0) +
                             face_E(phi, c, 1, i + 1, g.nx, g.ih, false, phi0));
    const double ey = 0.5 * (face_E(phi, c - sy, sy, j, g.ny, g.ih, false, phi0) +
                             face_E(phi, c, sy, j + 1, g.ny, g.ih, false, phi0));
    const double ez = 0.5 * (face_E(phi, c - sz, sz, k, g.nz, g.ih, true, phi0) +
                             face_E(phi, c, sz, k + 1, g.nz, g.ih, true, phi0));
    const double E = sqrt(ex * ex + ey * ey + ez * ez);
    const double a = E > 0.0 ? 5.7 * p * exp(-260.0 * p / E) : 0.0;
    Emag[c] = E;
    Si[c] = mu_e * ne[c] * a * E;
}

// Koren's limiter times the slope, phi(num / den) den with phi(r) = max(0, min(2r, (1 + 2r) / 3, 2)),
// without the division: for den > 0 it is max(0, min(2 num, (den + 2 num) / 3, 2 den)), for
// den < 0 the mirror image with min and max exchanged, and 0 for den = 0 (r taken as 0)
__device__ __forceinline__ double koren_slope(double num, double den) {
    const double a = 2.0 * num, b = (den + 2.0 * num) * (1.0 / 3.0), c = 2.0 * den;
    if (den > 0.0) return fmax(0.0, fmin(fmin(a, b), c));
    if (den < 0.0) return fmin(0.0, fmax(fmax(a, b), c));
    return 0.0;
}

// upwind MUSCL face value (Koren limiter) at face f of a line of m cells starting at c0 with
// the given stride; cells beyond the ends repeat the boundary cell (zero gradient)
__device__ __forceinline__ double muscl(const double* n, int64_t c0, int64_t stride, int f, int m, double v) {
    auto at = [&](int q) { return n[c0 + (int64_t)min(max(q, 0), m - 1) * stride]; };
    const double um = at(f - 2), u0 = at(f - 1), u1 = at(f), u2 = at(f + 1);
    if (v >= 0.0) return u0 + 0.5 * koren_slope(u0 - um, u1 - u0);
    return u1 + 0.5 * koren_slope(u1 - u2, u0 - u1);
}

// fluxes through the faces of one axis: electrons F_e = -mu_e E n_e^face - D_e dn_e/dx (zero
// diffusion through boundary faces), ions F_p = mu_p E n_p^face; faces [lines][m + 1]
__global__ void k_sd_flux(Grid g, int axis, const double* phi, double phi0, const double* ne, const double* np,
                          double mu_e, double mu_p, double D_e, double* Fe, double* Fp) {
    const int m = axis == 0 ? g.nx : axis == 1 ? g.ny : g.nz;
    const int64_t stride = axis == 0 ? 1 : axis == 1 ? (int64_t)g.nx : (int64_t)g.nx * g.ny;
    const int lines = (int)(g.n() / m);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= lines * (m + 1)) return;
    const int line = e / (m + 1);
    const int f = e - line * (m + 1);
    // first cell of the line: the other two indices
    int c0;
    if (axis == 0) c0 = line * g.nx;
    else if (axis == 1) {
        const int k = line / g.nx;
        c0 = k * (g.nx * g.ny) + (line - k * g.nx);
    } else c0 = line;
    const double E = face_E(phi, c0 + (int64_t)(f - 1) * stride, stride, f, m, g.ih, axis == 2, phi0);
    const double ve = -mu_e * E, vp = mu_p * E;
    double fe = ve * muscl(ne, c0, stride, f, m, ve);
    if (f > 0 && f < m) fe += -D_e * (ne[c0 + (int64_t)f * stride] - ne[c0 + (int64_t)(f - 1) * stride]) * g.ih;
    Fe[e] = fe;
    Fp[e] = vp * muscl(np, c0, stride, f, m, vp);
}

// dn/dt = -div F + S_i + S_ph for both species (faces of the three axes as k_sd_flux lays them)
__global__ void k_sd_div(Grid g, const double* Fex, const double* Fey, const double* Fez, const double* Fpx,
                         const double* Fpy, const double* Fpz, const double* Si, const double* Sph, double* dne,
                         double* dnp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.n()) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const int64_t lx = (int64_t)k * g.ny + j, ly = (int64_t)k * g.nx + i, lz = (int64_t)j * g.nx + i;
    const int64_t fx = lx * (g.nx + 1) + i, fy = ly * (g.ny + 1) + j, fz = lz * (g.nz + 1) + k;
    const double src = Si[c] + (Sph ? Sph[c] : 0.0), rh = g.ih;
    dne[c] = -((Fex[fx + 1] - Fex[fx]) + (Fey[fy + 1] - Fey[fy]) + (Fez[fz + 1] - Fez[fz])) * rh + src;
    dnp[c] = -((Fpx[fx + 1] - Fpx[fx]) + (Fpy[fy + 1] - Fpy[fy]) + (Fpz[fz + 1] - Fpz[fz])) * rh + src;
}

// the region's sources in its own order (x fastest), those below thr * max S_i dropped (the
// maximum read from the device: the bits of a non-negative double order like integers)
__global__ void k_sd_gather(Grid g, const int* reg, const double* Si, const unsigned long long* maxbits, double thr,
                            double* out) {
    const int rx = reg[1] - reg[0], ry = reg[3] - reg[2], rz = reg[5] - reg[4];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rx * ry * rz) return;
    const int i = reg[0] + (int)(e % rx), j = reg[2] + (int)((e / rx) % ry), k = reg[4] + (int)(e / ((int64_t)rx * ry));
    const double v = Si[((int64_t)k * g.ny + j) * g.nx + i];
    const double cut = maxbits ? thr * __longlong_as_double((long long)*maxbits) : 0.0;
    out[e] = v >= cut ? v : 0.0;
}
// S_ph of the region back into the grid (the rest was zeroed)
__global__ void k_sd_scatter(Grid g, const int* reg, const double* in, double* Sph) {
    const int rx = reg[1] - reg[0], ry = reg[3] - reg[2], rz = reg[5] - reg[4];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rx * ry * rz) return;
    const int i = reg[0] + (int)(e % rx), j = reg[2] + (int)((e / rx) % ry), k = reg[4] + (int)(e / ((int64_t)rx * ry));
    Sph[((int64_t)k * g.ny + j) * g.nx + i] = in[e];
}
__global__ void k_sd_absmax(const double* x, int64_t n, unsigned long long* out) {
    double m = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(x[e]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// b[e] += v for the n cells of the top layer (its Dirichlet term)
__global__ void k_sd_addtop(double* b, int64_t n, double v) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] += v;
}

// y = a x + b y + c z (Heun's combinations), elementwise over two fields
__global__ void k_sd_comb(int64_t n, double a, const double* x1, const double* x2, double b, double* y1, double* y2,
                          double cz, const double* z1, const double* z2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    y1[e] = a * x1[e] + b * y1[e] + cz * z1[e];
    y2[e] = a * x2[e] + b * y2[e] + cz * z2[e];
}

}  // namespace

struct Streamer {
    Grid g{};
    streamer_params prm{};
    kifmm_plan_t plan = nullptr;
    cudaStream_t st = nullptr;
    int num_sms = 1;
    DevBuf ne, np, ne0, np0, dne, dnp, phi, Emag, Si, Sph, F[6], red;
    DevBuf reg, rsrc, rout, rmax;   // local evaluation: region bounds, its sources and S_ph, max S_i
    int64_t nreg = 0;               // cells of the region (0: the whole grid, no gather)
    std::vector<Grid> lv;           // multigrid levels, lv[0] = the grid
    std::vector<DevBuf> u, b, r;    // level 0: phi, right-hand side, residual (FP64); then the
                                    // FP32 error equation per level: unknown, right-hand side, residual
    DevBuf e0, rhs0, t0;            // level 0 of the FP32 error equation
    int last_cycles = 0;
    double last_res = 0.0;
};

namespace {

int mg_norm(Streamer& S, const double* x, int64_t n, double* out) {
    const int nb = (int)std::min<int64_t>(nbs(n, 256), 2LL * S.num_sms);
    k_sumsq<<<nb, 256, 0, S.st>>>(x, n, ptr<double>(S.red));
    KF_LAUNCH();
    std::vector<double> part(nb);
    KF_CUDA(cudaMemcpyAsync(part.data(), S.red.p, nb * 8, cudaMemcpyDeviceToHost, S.st));
    KF_CUDA(cudaStreamSynchronize(S.st));
    double s = 0.0;
    for (double v : part) s += v;
    *out = std::sqrt(s);
    return KIFMM_OK;
}

// one FP32 V-cycle on the error equation A e = rhs of level l (l = 0: e0 / rhs0 / t0, else
// u[l] / b[l] / r[l]), from e = 0 below level 0 (the caller zeroes e0)
int vcycle(Streamer& S, int l) {
    const Grid& g = S.lv[l];
    const int64_t n = g.n();
    float* e = l == 0 ? ptr<float>(S.e0) : ptr<float>(S.u[l]);
    const float* rhs = l == 0 ? ptr<float>(S.rhs0) : ptr<float>(S.b[l]);
    float* res = l == 0 ? ptr<float>(S.t0) : ptr<float>(S.r[l]);
    const unsigned half = nbs((int64_t)((g.nx + 1) / 2) * g.ny * g.nz, 256);
    if (l + 1 == (int)S.lv.size()) {   // coarsest: sweeps in one block
        // (the V-cycle needs the coarse error reduced by about its own factor, not solved exactly)
        k_mg_coarse_solve<float><<<1, 1024, 0, S.st>>>(g, e, rhs, 8 * (g.nx + g.ny + g.nz));
        KF_LAUNCH();
        return KIFMM_OK;
    }
    for (int s = 0; s < 2; ++s)
        for (int color = 0; color < 2; ++color) k_mg_smooth<float><<<half, 256, 0, S.st>>>(g, e, rhs, color);
    k_mg_residual<float><<<nbs(n, 256), 256, 0, S.st>>>(g, e, rhs, res, nullptr);
    const Grid& cg = S.lv[l + 1];
    k_mg_restrict<float><<<nbs(cg.n(), 256), 256, 0, S.st>>>(g, cg, res, ptr<float>(S.b[l + 1]));
    KF_CUDA(cudaMemsetAsync(S.u[l + 1].p, 0, cg.n() * 4, S.st));
    KF_LAUNCH();
    KF_TRY(vcycle(S, l + 1));
    k_mg_prolong<float><<<nbs(n, 256), 256, 0, S.st>>>(g, cg, ptr<float>(S.u[l + 1]), e);
    for (int s = 0; s < 2; ++s)
        for (int color = 0; color < 2; ++color) k_mg_smooth<float><<<half, 256, 0, S.st>>>(g, e, rhs, color);
    KF_LAUNCH();
    return KIFMM_OK;
}

// phi (in S.u[0], warm start kept) for the right-hand side in S.b[0]
int poisson(Streamer& S) {
    const Grid& g = S.lv[0];
    double bn = 0.0, rn = 0.0;
    KF_TRY(mg_norm(S, ptr<double>(S.b[0]), g.n(), &bn));
    int c = 0;
    for (;;) {   // iterative refinement: the residual in FP64, the correction by an FP32 V-cycle
        k_mg_residual<double><<<nbs(g.n(), 256), 256, 0, S.st>>>(g, ptr<double>(S.u[0]), ptr<double>(S.b[0]),
                                                                   ptr<double>(S.r[0]), ptr<float>(S.rhs0));
        KF_LAUNCH();
        KF_TRY(mg_norm(S, ptr<double>(S.r[0]), g.n(), &rn));
        if (!(bn > 0.0) || rn <= S.prm.mg_tol * bn || c >= S.prm.mg_max_cycles) break;
        KF_CUDA(cudaMemsetAsync(S.e0.p, 0, g.n() * 4, S.st));
        KF_TRY(vcycle(S, 0));
        k_mg_correct<<<nbs(g.n(), 256), 256, 0, S.st>>>(g.n(), ptr<float>(S.e0), ptr<double>(S.u[0]));
        KF_LAUNCH();
        ++c;
    }
    S.last_cycles = c;
    S.last_res = bn > 0.0 ? rn / bn : 0.0;
    if (bn > 0.0 && !(rn <= S.prm.mg_tol * bn)) {
        set_error("streamer: the multigrid solve did not reach the tolerance within mg_max_cycles");
        return KIFMM_ERR_TIMEOUT;
    }
    return KIFMM_OK;
}

// L(U) of the densities in (ne, np): Poisson, |E|, S_i, S_ph, fluxes, divergence -> (dne, dnp)
int rhs(Streamer& S, const double* ne, const double* np, double* dne, double* dnp) {
    const Grid& g = S.g;
    const int64_t n = g.n();
    cudaStream_t st = S.st;
    k_sd_charge<<<nbs(n, 256), 256, 0, st>>>(g, ne, np, S.prm.phi0, ptr<double>(S.b[0]));
    KF_LAUNCH();
    KF_TRY(poisson(S));
    KF_CUDA(cudaMemcpyAsync(S.phi.p, S.u[0].p, n * 8, cudaMemcpyDeviceToDevice, st));
    k_sd_source<<<nbs(n, 256), 256, 0, st>>>(g, ptr<double>(S.phi), S.prm.phi0, ne, S.prm.mu_e, S.prm.p,
                                              ptr<double>(S.Emag), ptr<double>(S.Si));
    KF_LAUNCH();
    const double* sph = nullptr;
    if (S.plan) {   // the photoionization sum of S_i (Eq. (integral) with C = prm.C)
        const bool thr = S.prm.threshold > 0.0;
        if (thr) {
            KF_CUDA(cudaMemsetAsync(S.rmax.p, 0, 8, st));
            k_sd_absmax<<<(unsigned)std::min<int64_t>(nbs(n, 256), 4LL * S.num_sms), 256, 0, st>>>(
                ptr<double>(S.Si), n, ptr<unsigned long long>(S.rmax));
            KF_LAUNCH();
        }
        if (S.nreg > 0 || thr) {   // local and / or thresholded: gather, evaluate, scatter
            const int64_t nr = S.nreg > 0 ? S.nreg : n;
            k_sd_gather<<<nbs(nr, 256), 256, 0, st>>>(g, ptr<int>(S.reg), ptr<double>(S.Si),
                                                       thr ? ptr<unsigned long long>(S.rmax) : nullptr,
                                                       S.prm.threshold, ptr<double>(S.rsrc));
            KF_LAUNCH();
            KF_TRY(kifmm_eval(S.plan, S.rsrc.p, S.rout.p, KIFMM_F64, S.prm.C));
            KF_CUDA(cudaMemsetAsync(S.Sph.p, 0, n * 8, st));
            k_sd_scatter<<<nbs(nr, 256), 256, 0, st>>>(g, ptr<int>(S.reg), ptr<double>(S.rout), ptr<double>(S.Sph));
            KF_LAUNCH();
        } else {
            KF_TRY(kifmm_eval(S.plan, S.Si.p, S.Sph.p, KIFMM_F64, S.prm.C));
        }
        sph = ptr<double>(S.Sph);
    }
    const int m[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        const int64_t faces = n / m[a] * (m[a] + 1);
        k_sd_flux<<<nbs(faces, 256), 256, 0, st>>>(g, a, ptr<double>(S.phi), S.prm.phi0, ne, np, S.prm.mu_e,
                                                    S.prm.mu_p, S.prm.D_e, ptr<double>(S.F[a]), ptr<double>(S.F[3 + a]));
    }
    k_sd_div<<<nbs(n, 256), 256, 0, st>>>(g, ptr<double>(S.F[0]), ptr<double>(S.F[1]), ptr<double>(S.F[2]),
                                           ptr<double>(S.F[3]), ptr<double>(S.F[4]), ptr<double>(S.F[5]),
                                           ptr<double>(S.Si), sph, dne, dnp);
    KF_LAUNCH();
    return KIFMM_OK;
}

void release(Streamer& S) {
    for (DevBuf* d : {&S.ne, &S.np, &S.ne0, &S.np0, &S.dne, &S.dnp, &S.phi, &S.Emag, &S.Si, &S.Sph, &S.red, &S.reg,
                      &S.rsrc, &S.rout, &S.rmax})
        dev_free(*d);
    for (DevBuf& d : S.F) dev_free(d);
    for (auto* v : {&S.u, &S.b, &S.r})
        for (DevBuf& d : *v) dev_free(d);
    for (DevBuf* d : {&S.e0, &S.rhs0, &S.t0}) dev_free(*d);
}

}  // namespace
}  // namespace kifmm

using namespace kifmm;

struct streamer_s {
    Streamer s;
};

extern "C" {

void streamer_default_params(streamer_params* prm, double p_torr) {
    if (!prm) return;
    std::memset(prm, 0, sizeof(*prm));
    prm->p = p_torr;
    prm->phi0 = 52e3;
    prm->mu_e = 2.9e5 / p_torr;
    prm->mu_p = 2.6e3 / p_torr;
    prm->D_e = 1800.0;
    prm->C = 0.06 * 30.0 / (p_torr + 30.0);
    prm->mg_tol = 1e-8;
    prm->mg_max_cycles = 100;
}

int streamer_create(streamer_t* out, int nx, int ny, int nz, double h, const streamer_params* prm,
                    kifmm_plan_t plan, void* stream) {
    set_error("");
    if (!out || !prm || nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !(prm->p > 0.0) || !(prm->mg_tol > 0.0) ||
        prm->mg_max_cycles < 1 || (int64_t)nx * ny * nz >= (int64_t)1 << 31) {
        set_error("streamer_create: invalid argument");
        return KIFMM_ERR_ARG;
    }
    *out = nullptr;
    const int* rg = prm->region;
    const bool has_reg = rg[0] || rg[1] || rg[2] || rg[3] || rg[4] || rg[5];
    if (has_reg && !(rg[0] >= 0 && rg[0] < rg[1] && rg[1] <= nx && rg[2] >= 0 && rg[2] < rg[3] && rg[3] <= ny &&
                     rg[4] >= 0 && rg[4] < rg[5] && rg[5] <= nz)) {
        set_error("streamer_create: region must be cell ranges inside the grid");
        return KIFMM_ERR_ARG;
    }
    if (!(prm->threshold >= 0.0 && prm->threshold < 1.0)) {
        set_error("streamer_create: threshold must lie in [0, 1)");
        return KIFMM_ERR_ARG;
    }
    const int64_t ncell = has_reg ? (int64_t)(rg[1] - rg[0]) * (rg[3] - rg[2]) * (rg[5] - rg[4]) : (int64_t)nx * ny * nz;
    if (plan && kifmm_plan_internal(plan)->n_real != ncell) {
        set_error("streamer_create: the plan's point count differs from the grid's (or the region's) cells");
        return KIFMM_ERR_ARG;
    }
    auto* h_ = new (std::nothrow) streamer_s();
    if (!h_) return KIFMM_ERR_OOM;
    Streamer& S = h_->s;
    S.g = make_grid(nx, ny, nz, h);
    S.prm = *prm;
    S.plan = plan;
    S.st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&S.num_sms, cudaDevAttrMultiProcessorCount, dev);
    S.num_sms = std::max(S.num_sms, 1);
    // multigrid levels: halve while every extent is even and at least 4, then the coarsest
    S.lv.push_back(S.g);
    while (S.lv.back().nx % 2 == 0 && S.lv.back().ny % 2 == 0 && S.lv.back().nz % 2 == 0 && S.lv.back().nx >= 4 &&
           S.lv.back().ny >= 4 && S.lv.back().nz >= 4) {
        const Grid& f = S.lv.back();
        S.lv.push_back(make_grid(f.nx / 2, f.ny / 2, f.nz / 2, 2.0 * f.h));
    }
    auto fail = [&](int rc) {
        release(S);
        delete h_;
        return rc;
    };
    {   // the coarsest level is solved by sweeps in one block: keep it small
        const Grid& c = S.lv.back();
        if (c.n() > 8192 || std::max(c.nx, std::max(c.ny, c.nz)) > 32) {
            set_error("streamer_create: the grid must coarsen (extents m 2^L, all even down to 8) to at most 32 "
                      "cells per axis and 8192 cells");
            return fail(KIFMM_ERR_ARG);
        }
    }
    const int64_t n = S.g.n();
    int rc = KIFMM_OK;
    for (DevBuf* d : {&S.ne, &S.np, &S.ne0, &S.np0, &S.dne, &S.dnp, &S.phi, &S.Emag, &S.Si, &S.Sph})
        if (!rc) rc = dev_alloc(*d, n * 8);
    const int64_t faces[3] = {n / nx * (nx + 1), n / ny * (ny + 1), n / nz * (nz + 1)};
    for (int a = 0; a < 6 && !rc; ++a) rc = dev_alloc(S.F[a], faces[a % 3] * 8);
    if (!rc) rc = dev_alloc(S.red, (size_t)2 * S.num_sms * 8 + 64);
    {   // local / thresholded evaluation: the region's bounds (the whole grid without one)
        const int whole[6] = {0, nx, 0, ny, 0, nz};
        const int* r6 = has_reg ? rg : whole;
        S.nreg = has_reg ? ncell : 0;
        if (!rc) rc = dev_alloc(S.reg, 6 * sizeof(int));
        if (!rc && cudaMemcpy(S.reg.p, r6, 6 * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) rc = KIFMM_ERR_CUDA;
        if (!rc) rc = dev_alloc(S.rsrc, ncell * 8);
        if (!rc) rc = dev_alloc(S.rout, ncell * 8);
        if (!rc) rc = dev_alloc(S.rmax, 8);
    }
    S.u.resize(S.lv.size());
    S.b.resize(S.lv.size());
    S.r.resize(S.lv.size());
    for (size_t l = 0; l < S.lv.size() && !rc; ++l) {   // level 0 FP64, the error equation's levels FP32
        const size_t w = l == 0 ? 8 : 4;
        rc = dev_alloc(S.u[l], S.lv[l].n() * w);
        if (!rc) rc = dev_alloc(S.b[l], S.lv[l].n() * w);
        if (!rc) rc = dev_alloc(S.r[l], S.lv[l].n() * w);
    }
    for (DevBuf* d : {&S.e0, &S.rhs0, &S.t0})
        if (!rc) rc = dev_alloc(*d, n * 4);
    if (rc) return fail(rc);
    for (DevBuf* d : {&S.ne, &S.np, &S.phi, &S.Sph, &S.u[0]})
        if (cudaMemsetAsync(d->p, 0, n * 8, S.st) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    *out = h_;
    return KIFMM_OK;
}

int streamer_set(streamer_t s, const double* ne_dev, const double* np_dev) {
    set_error("");
    if (!s || !ne_dev || !np_dev) {
        set_error("streamer_set: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Streamer& S = s->s;
    const int64_t n = S.g.n();
    KF_CUDA(cudaMemcpyAsync(S.ne.p, ne_dev, n * 8, cudaMemcpyDeviceToDevice, S.st));
    KF_CUDA(cudaMemcpyAsync(S.np.p, np_dev, n * 8, cudaMemcpyDeviceToDevice, S.st));
    return KIFMM_OK;
}

int streamer_get(streamer_t s, double* ne_dev, double* np_dev, double* phi_dev, double* sph_dev) {
    set_error("");
    if (!s) {
        set_error("streamer_get: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Streamer& S = s->s;
    const int64_t n = S.g.n();
    const std::pair<void*, const DevBuf*> cp[4] = {{ne_dev, &S.ne}, {np_dev, &S.np}, {phi_dev, &S.phi}, {sph_dev, &S.Sph}};
    for (const auto& c : cp)
        if (c.first) KF_CUDA(cudaMemcpyAsync(c.first, c.second->p, n * 8, cudaMemcpyDeviceToDevice, S.st));
    return KIFMM_OK;
}

int streamer_rhs(streamer_t s, double* dne_dev, double* dnp_dev) {
    set_error("");
    if (!s || !dne_dev || !dnp_dev) {
        set_error("streamer_rhs: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Streamer& S = s->s;
    return rhs(S, ptr<double>(S.ne), ptr<double>(S.np), dne_dev, dnp_dev);
}

int streamer_step(streamer_t s, double dt, int nsteps) {
    set_error("");
    if (!s || !(dt > 0.0) || nsteps < 0) {
        set_error("streamer_step: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Streamer& S = s->s;
    const int64_t n = S.g.n();
    double* ne = ptr<double>(S.ne);
    double* np = ptr<double>(S.np);
    for (int it = 0; it < nsteps; ++it) {
        // Heun: U1 = U + dt L(U) (in ne0/np0 after keeping U), U' = (U + U1 + dt L(U1)) / 2
        KF_TRY(rhs(S, ne, np, ptr<double>(S.dne), ptr<double>(S.dnp)));
        KF_CUDA(cudaMemcpyAsync(S.ne0.p, ne, n * 8, cudaMemcpyDeviceToDevice, S.st));
        KF_CUDA(cudaMemcpyAsync(S.np0.p, np, n * 8, cudaMemcpyDeviceToDevice, S.st));
        k_sd_comb<<<nbs(n, 256), 256, 0, S.st>>>(n, 0.0, ne, np, 1.0, ne, np, dt, ptr<double>(S.dne), ptr<double>(S.dnp));
        KF_LAUNCH();
        KF_TRY(rhs(S, ne, np, ptr<double>(S.dne), ptr<double>(S.dnp)));
        // U' = 0.5 U0 + 0.5 U1 + 0.5 dt L(U1)
        k_sd_comb<<<nbs(n, 256), 256, 0, S.st>>>(n, 0.5, ptr<double>(S.ne0), ptr<double>(S.np0), 0.5, ne, np, 0.5 * dt,
                                                  ptr<double>(S.dne), ptr<double>(S.dnp));
        KF_LAUNCH();
    }
    return KIFMM_OK;
}

int streamer_poisson(streamer_t s, const double* rho_dev, double* phi_dev, double* rel_residual, int* cycles) {
    set_error("");
    if (!s || !rho_dev || !phi_dev) {
        set_error("streamer_poisson: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Streamer& S = s->s;
    const Grid& g = S.g;
    const int64_t n = g.n();
    // b = rho (the caller's charge term) plus the top face's Dirichlet term
    KF_CUDA(cudaMemcpyAsync(S.b[0].p, rho_dev, n * 8, cudaMemcpyDeviceToDevice, S.st));
    const int64_t nt = (int64_t)g.nx * g.ny;
    k_sd_addtop<<<nbs(nt, 256), 256, 0, S.st>>>(ptr<double>(S.b[0]) + (n - nt), nt, 2.0 * S.prm.phi0 / (g.h * g.h));
    KF_LAUNCH();
    const int rc = poisson(S);
    KF_CUDA(cudaMemcpyAsync(phi_dev, S.u[0].p, n * 8, cudaMemcpyDeviceToDevice, S.st));
    KF_CUDA(cudaStreamSynchronize(S.st));
    if (rel_residual) *rel_residual = S.last_res;
    if (cycles) *cycles = S.last_cycles;
    return rc;
}

int streamer_info(streamer_t s, int* mg_levels, int* last_cycles, double* last_residual) {
    if (!s) return KIFMM_ERR_ARG;
    if (mg_levels) *mg_levels = (int)s->s.lv.size();
    if (last_cycles) *last_cycles = s->s.last_cycles;
    if (last_residual) *last_residual = s->s.last_res;
    return KIFMM_OK;
}

void streamer_destroy(streamer_t s) {
    if (!s) return;
    cudaStreamSynchronize(s->s.st);
    release(s->s);
    delete s;
}

}  // extern "C"
