// Plan, part 2: equivalent/check surfaces, the per-level translation matrices
// (Eqs. (s2m), (m2m), (m2l), (l2l), (s2l) of the paper), their truncated-SVD
// pseudo-inverses, and the self-cell values of the discrete kernel G (Sec. 3).
// For the Chebyshev-node representation: the nodes, interpolation and node-to-node M2L
// matrices instead of surfaces and pseudo-inverses.
#include <algorithm>
#include <cstdlib>
#include <string>
#include <cmath>

#include "internal.cuh"
#include "kernel.cuh"
#include "selfcell.cuh"
#include "cheb.cuh"

namespace kifmm {

// Lattice {-1 + 2j/(m0-1)}^3 restricted to the cube's boundary, x fastest.
__global__ void surface_lattice(int m0, double* s) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int n = 0;
    for (int k = 0; k < m0; ++k)
        for (int j = 0; j < m0; ++j)
            for (int i = 0; i < m0; ++i)
                if (i == 0 || i == m0 - 1 || j == 0 || j == m0 - 1 || k == 0 || k == m0 - 1) {
                    s[3 * n + 0] = -1.0 + 2.0 * i / (m0 - 1);
                    s[3 * n + 1] = -1.0 + 2.0 * j / (m0 - 1);
                    s[3 * n + 2] = -1.0 + 2.0 * k / (m0 - 1);
                    ++n;
                }
}

// out[i*S + j] = K(|(d + rx s_i) - (ry s_j)|): target point i on a surface of radius rx
// about the origin shifted by d, source point j on a surface of radius ry about the origin.
// blockIdx.y selects one of `nmat` matrices with shifts d[3*blockIdx.y ...].
__global__ void surface_kmat(const double* s, int S, double rx, double ry, const double* d,
                             KParams kp, double* out, int64_t stride) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)S * S) return;
    int i = (int)(e / S), j = (int)(e % S);
    const double* dd = d + 3 * blockIdx.y;
    double r2 = 0;
    for (int k = 0; k < 3; ++k) {
        double x = dd[k] + rx * s[3 * i + k] - ry * s[3 * j + k];
        r2 += x * x;
    }
    out[blockIdx.y * stride + e] = (dd[0] == 0.0 && dd[1] == 0.0 && dd[2] == 0.0 && r2 == 0.0)
                                       ? 0.0 : kern_f64(sqrt(r2), kp);
}

// One-sided (Hestenes) Jacobi SVD, one CTA per matrix, column-major A (S x S) and V.
// Column pairs follow the round-robin (circle) ordering: in round r player n-1 meets r
// and (r+i) meets (r-i) mod (n-1), so every round rotates n/2 disjoint pairs.
// On return A holds U*Sigma (columns), V the right singular vectors; conv[0] = sweeps
// used, or -1 if the off-diagonal criterion was not met within max_sweeps.
__global__ void jacobi_svd(double* Aall, double* Vall, int S, int max_sweeps, int* conv) {
    double* A = Aall + (int64_t)blockIdx.x * S * S;
    double* V = Vall + (int64_t)blockIdx.x * S * S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t e = threadIdx.x; e < (int64_t)S * S; e += blockDim.x) V[e] = (e / S == e % S) ? 1.0 : 0.0;
    __shared__ int rotated;
    __syncthreads();
    const int n = S;          // S is even for every m0
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < n - 1; ++r) {
            for (int pi = warp; pi < n / 2; pi += nw) {
                int p, q;
                if (pi == 0) {
                    p = r;
                    q = n - 1;
                } else {
                    p = (r + pi) % (n - 1);
                    q = (r - pi + (n - 1)) % (n - 1);
                }
                double* ap = A + (int64_t)p * S;
                double* aq = A + (int64_t)q * S;
                double al = 0, be = 0, ga = 0;
                for (int i = lane; i < S; i += 32) {
                    double x = ap[i], y = aq[i];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                if (al == 0.0 || be == 0.0) continue;
                if (fabs(ga) <= 1e-14 * sqrt(al * be)) continue;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = c * t;
                for (int i = lane; i < S; i += 32) {
                    double x = ap[i], y = aq[i];
                    ap[i] = c * x - sn * y;
                    aq[i] = sn * x + c * y;
                }
                double* vp = V + (int64_t)p * S;
                double* vq = V + (int64_t)q * S;
                for (int i = lane; i < S; i += 32) {
                    double x = vp[i], y = vq[i];
                    vp[i] = c * x - sn * y;
                    vq[i] = sn * x + c * y;
                }
                if (lane == 0) rotated = 1;
            }
            __syncthreads();
        }
        __syncthreads();
        if (!rotated) break;
        __syncthreads();
    }
    if (threadIdx.x == 0) conv[blockIdx.x] = (sweep < max_sweeps) ? sweep + 1 : -1;
}

// sigma_k = |a_k| and the kept rank for the relative cut-off eps.
__global__ void svd_sigma(const double* Aall, int S, double eps, double* sig_all, int* rank) {
    const double* A = Aall + (int64_t)blockIdx.x * S * S;
    double* sig = sig_all + (int64_t)blockIdx.x * S;
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        double s = 0;
        for (int i = 0; i < S; ++i) s += A[(int64_t)k * S + i] * A[(int64_t)k * S + i];
        sig[k] = sqrt(s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0;
        for (int k = 0; k < S; ++k) mx = fmax(mx, sig[k]);
        int r = 0;
        for (int k = 0; k < S; ++k) {
            if (sig[k] >= eps * mx) ++r;
            else sig[k] = 0.0;   // dropped
        }
        rank[blockIdx.x] = r;
    }
}

// Basis matrices of the truncated SVD A_l = K(x^{B,u}, y^{B,u}) = U Sigma V^T (kept columns
// listed in idx, r of them), padded with zeros to R coefficients:
//   G1 = Sigma^+ U^T (R x S)  upward check potential -> coefficients c   (phi^u = V c)
//   Vb = V           (S x R)  coefficients -> upward equivalent density
//   Ub = U Sigma^+   (S x R)  coefficients d -> downward equivalent density (phi^d = Ub d)
//   Vt = V^T         (R x S)  downward check potential -> coefficients d
// The downward system K(x^{B,d}, y^{B,d}) is A_l^T (the surfaces swap roles and K is
// symmetric), so its truncated pseudo-inverse is U Sigma^+ V^T = Ub Vt.
__global__ void svd_basis(const double* Acol, const double* Vcol, const double* sig, const int* idx, int r,
                          int S, int R, double* G1, double* Vb, double* Ub, double* Vt) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)S * R) return;
    int i = (int)(e / R), j = (int)(e % R);   // i < S, j < R
    double vb = 0, ub = 0;
    if (j < r) {
        int k = idx[j];
        double s = sig[k];
        vb = Vcol[(int64_t)k * S + i];
        ub = Acol[(int64_t)k * S + i] / (s * s);
    }
    Vb[(int64_t)i * R + j] = vb;
    Ub[(int64_t)i * R + j] = ub;
    G1[(int64_t)j * S + i] = ub;
    Vt[(int64_t)j * S + i] = vb;
}

__global__ void transpose_to_colmajor(const double* in, double* out, int S, int nmat) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)S * S * nmat) return;
    int64_t m = e / ((int64_t)S * S);
    int64_t r = e % ((int64_t)S * S);
    int i = (int)(r / S), j = (int)(r % S);
    out[m * S * S + (int64_t)j * S + i] = in[e];
}

// Batched FP64 GEMM for the plan: C[b] = A[b] (M x K) * B[b] (K x N), row-major,
// batch strides sA/sB/sC (sA = 0 or sB = 0 shares a factor). 16 x 16 tiles.
__global__ void gemm64_batched(int M, int N, int K, const double* A, int lda, int64_t sA, const double* B,
                               int ldb, int64_t sB, double* C, int ldc, int64_t sC) {
    __shared__ double As[16][17], Bs[16][17];
    const double* a = A + blockIdx.z * sA;
    const double* b = B + blockIdx.z * sB;
    double* c = C + blockIdx.z * sC;
    int row = blockIdx.y * 16 + threadIdx.y, col = blockIdx.x * 16 + threadIdx.x;
    double acc = 0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        As[threadIdx.y][threadIdx.x] = (row < M && ka < K) ? a[(int64_t)row * lda + ka] : 0.0;
        Bs[threadIdx.y][threadIdx.x] = (kb < K && col < N) ? b[(int64_t)kb * ldb + col] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc += As[threadIdx.y][k] * Bs[k][threadIdx.x];
        __syncthreads();
    }
    if (row < M && col < N) c[(int64_t)row * ldc + col] = acc;
}

__global__ void to_f32(const double* in, float* out, int64_t n) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = (float)in[e];
}

static inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static int gemm64(cudaStream_t st, int M, int N, int K, const double* A, int lda, int64_t sA, const double* B,
                  int ldb, int64_t sB, double* C, int ldc, int64_t sC, int batch) {
    dim3 g(nb(N, 16), nb(M, 16), batch);
    gemm64_batched<<<g, dim3(16, 16), 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
    KF_LAUNCH();
    return KIFMM_OK;
}

static int f32_copy(cudaStream_t st, const DevBuf& src, DevBuf& dst, int64_t n) {
    KF_TRY(dev_alloc(dst, n * 4));
    to_f32<<<nb(n, 256), 256, 0, st>>>(ptr<double>(src), ptr<float>(dst), n);
    KF_LAUNCH();
    return KIFMM_OK;
}

// ------------------------------------------------------------------------------------
// Chebyshev-node representation: nodes, weight table, interpolation and M2L matrices
// ------------------------------------------------------------------------------------
// The p^3 tensor nodes (x fastest) and tab[n][k] = c_k T_k(xbar_n); one thread per node.
__global__ void cheb_nodes(int p, double* s, double* tab, float* tab32) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int S = p * p * p;
    if (m < p * kChebTab) {
        const int n = m / kChebTab, k = m % kChebTab;
        double v = 0.0;
        if (k < p) v = (k == 0 ? 1.0 : 2.0) / p * cos(k * (2 * n + 1) * 3.14159265358979323846 / (2.0 * p));
        tab[m] = v;
        tab32[m] = (float)v;
    }
    if (m < S) {
        const int idx[3] = {m % p, (m / p) % p, m / (p * p)};
        for (int a = 0; a < 3; ++a) s[3 * m + a] = cos((2 * idx[a] + 1) * 3.14159265358979323846 / (2.0 * p));
    }
}

// M2M for child octant o (parent level -> itself, level independent):
//   M_o[n][m] = S3(xbar_n, 0.5 (2 o - 1) + 0.5 xbar_m)  (child node m in parent units)
// stored as Mc [8][S][R] (rows parent nodes) and, for L2L, its transpose Lo [8][R][R]
// (rows child nodes); the padding is zeroed by the caller.
__global__ void cheb_m2m(int p, int S, int R, const double* s, const double* tab, double* Mc, double* Lo) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 8LL * S * S) return;
    const int o = (int)(e / ((int64_t)S * S));
    const int n = (int)((e / S) % S), m = (int)(e % S);
    const int nidx[3] = {n % p, (n / p) % p, n / (p * p)};
    double v = 1.0;
    for (int a = 0; a < 3; ++a) {
        const double x = 0.5 * (2.0 * ((o >> a) & 1) - 1.0) + 0.5 * s[3 * m + a];
        double t[kChebMaxP];
        cheb_T(x, p, t);
        v *= cheb_S(t, p, tab + nidx[a] * kChebTab);
    }
    Mc[((int64_t)o * S + n) * R + m] = v;
    Lo[((int64_t)o * R + m) * R + n] = v;
}

// The 1-D factors of M_o: A[b][n][m] = S(0.5 (2b - 1) + 0.5 xbar_m, xbar_n), b = 0, 1 (the
// child in the lower / upper half of the parent along an axis); M_o = A[oz] (x) A[oy] (x) A[ox].
__global__ void cheb_factors(int p, const double* tab, double* A) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * p * p) return;
    const int b = e / (p * p), n = (e / p) % p, m = e % p;
    const double xm = cos((2 * m + 1) * 3.14159265358979323846 / (2.0 * p));
    double t[kChebMaxP];
    cheb_T(0.5 * (2.0 * b - 1.0) + 0.5 * xm, p, t);
    A[e] = cheb_S(t, p, tab + n * kChebTab);
}

// out[mat][i][j] = in[mat][i][j] for i, j < S (row stride S -> R); the padding stays zero.
__global__ void pad_square(const double* in, int S, int R, int nmat, double* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nmat * S * S) return;
    const int64_t mat = e / ((int64_t)S * S);
    const int i = (int)((e / S) % S), j = (int)(e % S);
    out[(mat * R + i) * R + j] = in[e];
}

// Operators of the Chebyshev representation. No pseudo-inverse: a box's values are its
// node weights (the coefficients c, d of the surface form with rank S), so the G1, Vb, Ub,
// Vt steps of the evaluation become the identity and are skipped there.
//   M2L: T_{l,delta}[m][n] = K(|r xbar_m - (2 r delta + r xbar_n)|)  (B's nodes, A's nodes)
//   M2M: Mc_{l,o} = M_o, L2L: Lo_{l,o} = M_o^T (the same at every level)
static int build_operators_cheb(Plan& p) {
    cudaStream_t st = p.stream;
    const int S = p.S, pc = p.m0;
    const int L = p.tree.nlevels;
    const KParams kp = make_kparams_kind(p.kind, p.a, p.b);
    KF_TRY(dev_alloc(p.surf, 3 * S * sizeof(double)));
    KF_TRY(dev_alloc(p.ctab, kChebMaxP * kChebTab * sizeof(double)));
    KF_TRY(dev_alloc(p.ctab32, kChebMaxP * kChebTab * sizeof(float)));
    cheb_nodes<<<nb(std::max(S, pc * kChebTab), 128), 128, 0, st>>>(pc, ptr<double>(p.surf), ptr<double>(p.ctab),
                                                                     ptr<float>(p.ctab32));
    KF_LAUNCH();
    p.ops.clear();
    p.ops.resize(std::max(L, 1));
    // R: S rounded up so that the tensor-core M2L's row blocks (at most 256 rows) are whole
    // multiples of 32
    const int nblk = (S + 255) / 256;
    const int R = (S + 32 * nblk - 1) / (32 * nblk) * (32 * nblk);
    p.R = R;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev);
        p.num_sms = std::max(p.num_sms, 1);
        const char* m2l = std::getenv("KIFMM_M2L");
        p.m2l_tensor = p.precision == KIFMM_MIXED && m2l_tc_supported(R) && !(m2l && std::string(m2l) == "simt");
    }
    if (L <= 2) return KIFMM_OK;   // no box has a far field
    const int64_t SS = (int64_t)S * S, RR = (int64_t)R * R;
    DevBuf m2l, shifts, mc, lo;
    KF_TRY(dev_alloc(m2l, kOffsetSlots * SS * 8));
    KF_TRY(dev_alloc(shifts, kOffsetSlots * 3 * 8));
    KF_TRY(dev_alloc(mc, 8 * (int64_t)S * R * 8));
    KF_TRY(dev_alloc(lo, 8 * RR * 8));
    KF_CUDA(cudaMemsetAsync(mc.p, 0, 8 * (int64_t)S * R * 8, st));
    KF_CUDA(cudaMemsetAsync(lo.p, 0, 8 * RR * 8, st));
    KF_TRY(dev_alloc(p.cheb_A, 2 * kChebMaxP * kChebMaxP * sizeof(double)));
    cheb_factors<<<nb(2 * pc * pc, 128), 128, 0, st>>>(pc, ptr<double>(p.ctab), ptr<double>(p.cheb_A));
    KF_LAUNCH();
    cheb_m2m<<<nb(8 * SS, 256), 256, 0, st>>>(pc, S, R, ptr<double>(p.surf), ptr<double>(p.ctab), ptr<double>(mc),
                                              ptr<double>(lo));
    KF_LAUNCH();
    std::vector<double> sh(kOffsetSlots * 3);
    for (int l = 2; l < L; ++l) {
        LevelOps& op = p.ops[l];
        const double r = p.tree.side / (double)(2ll << l);
        op.level = l;
        op.r = r;
        op.rank = S;
        for (int dz = -3; dz <= 3; ++dz)
            for (int dy = -3; dy <= 3; ++dy)
                for (int dx = -3; dx <= 3; ++dx) {
                    const int sl = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
                    sh[3 * sl + 0] = -2.0 * r * dx;
                    sh[3 * sl + 1] = -2.0 * r * dy;
                    sh[3 * sl + 2] = -2.0 * r * dz;
                }
        KF_CUDA(cudaMemcpyAsync(shifts.p, sh.data(), sh.size() * 8, cudaMemcpyHostToDevice, st));
        surface_kmat<<<dim3(nb(SS, 256), kOffsetSlots), 256, 0, st>>>(ptr<double>(p.surf), S, r, r, ptr<double>(shifts),
                                                                     kp, ptr<double>(m2l), SS);
        KF_LAUNCH();
        for (int dz = -1; dz <= 1; ++dz)   // near slots are never used: zero them
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sl = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
                    KF_CUDA(cudaMemsetAsync(ptr<double>(m2l) + sl * SS, 0, SS * 8, st));
                }
        KF_TRY(dev_alloc(op.T, kOffsetSlots * RR * 8));
        KF_CUDA(cudaMemsetAsync(op.T.p, 0, kOffsetSlots * RR * 8, st));
        pad_square<<<nb(kOffsetSlots * SS, 256), 256, 0, st>>>(ptr<double>(m2l), S, R, kOffsetSlots, ptr<double>(op.T));
        KF_LAUNCH();
        if (l + 1 < L) {
            KF_TRY(dev_alloc(op.Mc, 8 * (int64_t)S * R * 8));
            KF_TRY(dev_alloc(op.Lo, 8 * RR * 8));
            KF_CUDA(cudaMemcpyAsync(op.Mc.p, mc.p, 8 * (int64_t)S * R * 8, cudaMemcpyDeviceToDevice, st));
            KF_CUDA(cudaMemcpyAsync(op.Lo.p, lo.p, 8 * RR * 8, cudaMemcpyDeviceToDevice, st));
        }
        if (p.precision == KIFMM_MIXED) {
            if (p.m2l_tensor) {
                KF_TRY(dev_alloc(op.Thi, (size_t)m2l_tc_table_elems(R) * 2));
                KF_TRY(dev_alloc(op.Tlo, (size_t)m2l_tc_table_elems(R) * 2));
                KF_TRY(m2l_tc_prepare(st, ptr<double>(op.T), R, op.Thi.p, op.Tlo.p, &op.tc_sT));
            } else {
                KF_TRY(f32_copy(st, op.T, op.T32, kOffsetSlots * RR));
            }
            if (l + 1 < L) {
                KF_TRY(f32_copy(st, op.Lo, op.Lo32, 8 * RR));
                KF_TRY(f32_copy(st, op.Mc, op.Mc32, 8 * (int64_t)S * R));
            }
        }
        KF_CUDA(cudaStreamSynchronize(st));   // shifts and m2l are reused by the next level
    }
    for (DevBuf* d : {&m2l, &shifts, &mc, &lo}) dev_free(*d);
    return KIFMM_OK;
}

int build_operators(Plan& p) {
    if (p.cheb) return build_operators_cheb(p);
    cudaStream_t st = p.stream;
    const int S = p.S;
    const int L = p.tree.nlevels;
    const KParams kp = make_kparams_kind(p.kind, p.a, p.b);
    KF_TRY(dev_alloc(p.surf, 3 * S * sizeof(double)));
    surface_lattice<<<1, 1, 0, st>>>(p.m0, ptr<double>(p.surf));
    KF_LAUNCH();
    p.ops.clear();
    p.ops.resize(std::max(L, 1));
    p.R = 32;
    if (L <= 2) return KIFMM_OK;   // no box has a far field

    const int nlev = L - 2;        // levels 2 .. L-1
    const int64_t SS = (int64_t)S * S;
    DevBuf A, V, sig, rank, conv, shifts, tmp, z, idxb;
    KF_TRY(dev_alloc(A, nlev * SS * 8));
    KF_TRY(dev_alloc(V, nlev * SS * 8));
    KF_TRY(dev_alloc(sig, nlev * S * 8));
    KF_TRY(dev_alloc(rank, nlev * 4));
    KF_TRY(dev_alloc(conv, nlev * 4));
    KF_TRY(dev_alloc(shifts, kOffsetSlots * 3 * 8));
    KF_TRY(dev_alloc(tmp, SS * 8));
    KF_TRY(dev_alloc(z, 3 * 8));
    KF_TRY(dev_alloc(idxb, S * 4));
    double zero3[3] = {0, 0, 0};
    KF_CUDA(cudaMemcpyAsync(z.p, zero3, 24, cudaMemcpyHostToDevice, st));
    // ---- upward check-to-equivalent systems K(x^{B,u}, y^{B,u}) and their SVDs
    for (int l = 2; l < L; ++l) {
        double r = p.tree.side / (double)(2ll << l);
        p.ops[l].level = l;
        p.ops[l].r = r;
        surface_kmat<<<dim3(nb(SS, 256), 1), 256, 0, st>>>(ptr<double>(p.surf), S, p.r_out * r, p.r_in * r,
                                                           ptr<double>(z), kp, ptr<double>(tmp), SS);
        KF_LAUNCH();
        transpose_to_colmajor<<<nb(SS, 256), 256, 0, st>>>(ptr<double>(tmp), ptr<double>(A) + (l - 2) * SS, S, 1);
        KF_LAUNCH();
    }
    jacobi_svd<<<nlev, 1024, 0, st>>>(ptr<double>(A), ptr<double>(V), S, 60, ptr<int>(conv));
    KF_LAUNCH();
    svd_sigma<<<nlev, 256, 0, st>>>(ptr<double>(A), S, p.pinv_eps, ptr<double>(sig), ptr<int>(rank));
    KF_LAUNCH();
    std::vector<double> hsig((size_t)nlev * S);
    std::vector<int> hconv(nlev);
    KF_CUDA(cudaMemcpyAsync(hsig.data(), sig.p, hsig.size() * 8, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaMemcpyAsync(hconv.data(), conv.p, nlev * 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    // kept singular values per level, in decreasing order (ties by index)
    std::vector<std::vector<int>> keep(L);
    int rmax = 1;
    for (int l = 2; l < L; ++l) {
        if (hconv[l - 2] < 0) {
            set_error("kifmm_plan: Jacobi SVD did not converge at level " + std::to_string(l));
            return KIFMM_ERR_NUMERIC;
        }
        const double* s = hsig.data() + (size_t)(l - 2) * S;
        for (int k = 0; k < S; ++k)
            if (s[k] > 0.0) keep[l].push_back(k);
        std::stable_sort(keep[l].begin(), keep[l].end(), [&](int x, int y) { return s[x] > s[y]; });
        p.ops[l].rank = (int)keep[l].size();
        rmax = std::max(rmax, p.ops[l].rank);
    }
    const int R = (rmax + 31) / 32 * 32;
    p.R = R;
    {
        const char* m2l = std::getenv("KIFMM_M2L");
        {
            int dev = 0;
            if (cudaGetDevice(&dev) == cudaSuccess)
                cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev);
            p.num_sms = std::max(p.num_sms, 1);
        }
        p.m2l_tensor = p.precision == KIFMM_MIXED && m2l_tc_supported(R) && !(m2l && std::string(m2l) == "simt");
    }
    const int64_t SR = (int64_t)S * R, RR = (int64_t)R * R;
    for (int l = 2; l < L; ++l) {
        LevelOps& op = p.ops[l];
        KF_CUDA(cudaMemcpyAsync(idxb.p, keep[l].data(), keep[l].size() * 4, cudaMemcpyHostToDevice, st));
        KF_TRY(dev_alloc(op.G1, SR * 8));
        KF_TRY(dev_alloc(op.Vb, SR * 8));
        KF_TRY(dev_alloc(op.Ub, SR * 8));
        KF_TRY(dev_alloc(op.Vt, SR * 8));
        svd_basis<<<nb(SR, 256), 256, 0, st>>>(ptr<double>(A) + (l - 2) * SS, ptr<double>(V) + (l - 2) * SS,
                                               ptr<double>(sig) + (l - 2) * S, ptr<int>(idxb), op.rank, S, R,
                                               ptr<double>(op.G1), ptr<double>(op.Vb), ptr<double>(op.Ub),
                                               ptr<double>(op.Vt));
        KF_LAUNCH();
        KF_CUDA(cudaStreamSynchronize(st));   // idxb is reused by the next level
    }
    // ---- M2L in coefficients: T_{l,delta} = V^T K(x^{B,d}, y^{A,u}) V, c_A - c_B = 2 r delta
    DevBuf m2l, w;
    KF_TRY(dev_alloc(m2l, kOffsetSlots * SS * 8));
    KF_TRY(dev_alloc(w, kOffsetSlots * SR * 8));
    std::vector<double> sh(kOffsetSlots * 3);
    for (int l = 2; l < L; ++l) {
        LevelOps& op = p.ops[l];
        double r = op.r;
        for (int dz = -3; dz <= 3; ++dz)
            for (int dy = -3; dy <= 3; ++dy)
                for (int dx = -3; dx <= 3; ++dx) {
                    int sl = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
                    sh[3 * sl + 0] = -2.0 * r * dx;
                    sh[3 * sl + 1] = -2.0 * r * dy;
                    sh[3 * sl + 2] = -2.0 * r * dz;
                }
        KF_CUDA(cudaMemcpyAsync(shifts.p, sh.data(), sh.size() * 8, cudaMemcpyHostToDevice, st));
        surface_kmat<<<dim3(nb(SS, 256), kOffsetSlots), 256, 0, st>>>(ptr<double>(p.surf), S, p.r_in * r, p.r_in * r,
                                                                     ptr<double>(shifts), kp, ptr<double>(m2l), SS);
        KF_LAUNCH();
        for (int dz = -1; dz <= 1; ++dz)   // near slots are never used: zero them
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int sl = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
                    KF_CUDA(cudaMemsetAsync(ptr<double>(m2l) + sl * SS, 0, SS * 8, st));
                }
        KF_TRY(gemm64(st, S, R, S, ptr<double>(m2l), S, SS, ptr<double>(op.Vb), R, 0, ptr<double>(w), R, SR,
                      kOffsetSlots));
        KF_TRY(dev_alloc(op.T, kOffsetSlots * RR * 8));
        KF_TRY(gemm64(st, R, R, S, ptr<double>(op.Vt), S, 0, ptr<double>(w), R, SR, ptr<double>(op.T), R, RR,
                      kOffsetSlots));
        KF_CUDA(cudaStreamSynchronize(st));
    }
    // ---- M2M and L2L, parent level l -> child level l + 1
    //   Mc_{l,o} = K(x^{P,u}, y^{C_o,u}) Vb_{l+1}   (child coefficients -> parent check potential;
    //              the parent's coefficients then follow from its pseudo-inverse, as at the leaves)
    //   Lo_{l,o} = Vt_{l+1} K(x^{C_o,d}, y^{P,d}) Ub_l
    for (int l = 2; l + 1 < L; ++l) {
        LevelOps& op = p.ops[l];
        LevelOps& ch = p.ops[l + 1];
        double r = op.r, rc = r / 2.0;
        for (int o = 0; o < 8; ++o) {
            double cc[3] = {rc * (2.0 * (o & 1) - 1.0), rc * (2.0 * ((o >> 1) & 1) - 1.0),
                            rc * (2.0 * ((o >> 2) & 1) - 1.0)};
            for (int k = 0; k < 3; ++k) {
                sh[3 * o + k] = -cc[k];        // M2M: parent check (centre 0) - child equivalent at cc
                sh[24 + 3 * o + k] = cc[k];    // L2L: child check at cc - parent equivalent at 0
            }
        }
        KF_CUDA(cudaMemcpyAsync(shifts.p, sh.data(), 48 * 8, cudaMemcpyHostToDevice, st));
        KF_TRY(dev_alloc(op.Mc, 8 * SR * 8));
        KF_TRY(dev_alloc(op.Lo, 8 * RR * 8));
        surface_kmat<<<dim3(nb(SS, 256), 8), 256, 0, st>>>(ptr<double>(p.surf), S, p.r_out * r, p.r_in * rc,
                                                          ptr<double>(shifts), kp, ptr<double>(m2l), SS);
        KF_LAUNCH();
        KF_TRY(gemm64(st, S, R, S, ptr<double>(m2l), S, SS, ptr<double>(ch.Vb), R, 0, ptr<double>(op.Mc), R, SR, 8));
        surface_kmat<<<dim3(nb(SS, 256), 8), 256, 0, st>>>(ptr<double>(p.surf), S, p.r_in * rc, p.r_out * r,
                                                          ptr<double>(shifts) + 24, kp, ptr<double>(m2l), SS);
        KF_LAUNCH();
        KF_TRY(gemm64(st, S, R, S, ptr<double>(m2l), S, SS, ptr<double>(op.Ub), R, 0, ptr<double>(w), R, SR, 8));
        KF_TRY(gemm64(st, R, R, S, ptr<double>(ch.Vt), S, 0, ptr<double>(w), R, SR, ptr<double>(op.Lo), R, RR, 8));
        KF_CUDA(cudaStreamSynchronize(st));
    }
    // ---- FP32 copies for the mixed form's FP32 phases (M2L, L2L, S2L, local/W evaluation)
    if (p.precision == KIFMM_MIXED) {
        for (int l = 2; l < L; ++l) {
            LevelOps& op = p.ops[l];
            if (p.m2l_tensor) {
                KF_TRY(dev_alloc(op.Thi, (size_t)m2l_tc_table_elems(R) * 2));
                KF_TRY(dev_alloc(op.Tlo, (size_t)m2l_tc_table_elems(R) * 2));
                KF_TRY(m2l_tc_prepare(st, ptr<double>(op.T), R, op.Thi.p, op.Tlo.p, &op.tc_sT));
            } else {
                KF_TRY(f32_copy(st, op.T, op.T32, kOffsetSlots * RR));
            }
            KF_TRY(f32_copy(st, op.Ub, op.Ub32, SR));
            KF_TRY(f32_copy(st, op.Vb, op.Vb32, SR));
            KF_TRY(f32_copy(st, op.Vt, op.Vt32, SR));
            if (l + 1 < L) {
                KF_TRY(f32_copy(st, op.Lo, op.Lo32, 8 * RR));
                KF_TRY(f32_copy(st, op.Mc, op.Mc32, 8 * SR));
            }
        }
    }
    KF_CUDA(cudaStreamSynchronize(st));
    for (DevBuf* d : {&A, &V, &sig, &rank, &conv, &shifts, &tmp, &z, &idxb, &m2l, &w}) dev_free(*d);
    return KIFMM_OK;
}

// ------------------------------------------------------------------------------------
// self-cell values sigma(h) (discrete kernel G, i == j)
// ------------------------------------------------------------------------------------
__global__ void gauss_legendre(int n, double* x, double* w) {
    int i = threadIdx.x;
    if (i < n) gl_node(n, i, &x[i], &w[i]);
}

// One block (256 threads) per distinct cell edge.
__global__ void self_sigma(const double* hs, int nh, double a, double b, int mode, int nq,
                           const double* gx, const double* gw, double* out) {
    int k = blockIdx.x;
    if (k >= nh) return;
    __shared__ double red[256];
    double s = self_sigma_block(hs[k], a, b, mode, nq, gx, gw, red);
    if (threadIdx.x == 0) out[k] = s;
}

__global__ void h_bits(const double* h, const int32_t* perm, int64_t n, uint64_t* key, int32_t* val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = __double_as_longlong(h[perm[i]]);
    val[i] = (int32_t)i;
}
__global__ void uniq_flags(const uint64_t* key, int64_t n, int32_t* flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}
__global__ void uniq_gather(const uint64_t* key, const int32_t* flag, const int32_t* pos, int64_t n,
                            double* hs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    hs[pos[i]] = __longlong_as_double(key[i]);
}
// sorted-order point k: sigma[k] = sig_u[unique index of h(perm[k])]; w[k] = h^3
__global__ void scatter_sigma(const uint64_t* key, const int32_t* val, const int32_t* flag,
                              const int32_t* pos, int64_t n, const double* sig_u, double* sigma,
                              double* w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int u = pos[i] + flag[i] - 1;
    int k = val[i];
    sigma[k] = sig_u[u];
    double h = __longlong_as_double(key[i]);
    w[k] = h * h * h;
}
__global__ void fill_uniform(int64_t n, double s, double vol, double* sigma, double* w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sigma[i] = s;
    w[i] = vol;
}
__global__ void self_sigma_box(double hx, double hy, double hz, double a, double b, int mode, int nq,
                               const double* gx, const double* gw, double* out) {
    __shared__ double red[256];
    const double s = self_sigma_box_block(hx, hy, hz, a, b, mode, nq, gx, gw, red);
    if (threadIdx.x == 0) out[0] = s;
}
// the comparison kernels: sigma of cubes of edge hs[k] (or of the rectangular cell dims when hs is
// NULL), one block each
__global__ void self_sigma_kind(const double* hs, int nh, double hx, double hy, double hz, KParams kp, int mode,
                                int nq, const double* gx, const double* gw, double* out) {
    const int k = blockIdx.x;
    if (k >= nh) return;
    __shared__ double red[256];
    const double s = hs ? self_sigma_kind_block(hs[k], hs[k], hs[k], kp, mode, nq, gx, gw, red)
                        : self_sigma_kind_block(hx, hy, hz, kp, mode, nq, gx, gw, red);
    if (threadIdx.x == 0) out[k] = s;
}

int build_self_terms(Plan& p, const double* h_dev, double uh) {
    cudaStream_t st = p.stream;
    const int64_t n = p.tree.n;
    const int NQ = 64;
    DevBuf gx, gw;
    KF_TRY(dev_alloc(gx, NQ * 8));
    KF_TRY(dev_alloc(gw, NQ * 8));
    gauss_legendre<<<1, NQ, 0, st>>>(NQ, ptr<double>(gx), ptr<double>(gw));
    KF_LAUNCH();
    KF_TRY(dev_alloc(p.sigma, n * 8));
    KF_TRY(dev_alloc(p.w, n * 8));
    if (!h_dev) {   // one cell shape for every point: a cube of edge uh, or the plan's rectangular cell
        DevBuf hb, sb;
        KF_TRY(dev_alloc(hb, 8));
        KF_TRY(dev_alloc(sb, 8));
        KF_CUDA(cudaMemcpyAsync(hb.p, &uh, 8, cudaMemcpyHostToDevice, st));
        double vol = uh * uh * uh;
        if (p.kind) {
            const double hx = p.rect ? p.cell_dims[0] : uh, hy = p.rect ? p.cell_dims[1] : uh,
                         hz = p.rect ? p.cell_dims[2] : uh;
            self_sigma_kind<<<1, 256, 0, st>>>(nullptr, 1, hx, hy, hz, make_kparams_kind(p.kind, p.a, p.b),
                                               p.self_mode, NQ, ptr<double>(gx), ptr<double>(gw), ptr<double>(sb));
            vol = hx * hy * hz;
        } else if (p.rect) {
            self_sigma_box<<<1, 256, 0, st>>>(p.cell_dims[0], p.cell_dims[1], p.cell_dims[2], p.a, p.b, p.self_mode,
                                              NQ, ptr<double>(gx), ptr<double>(gw), ptr<double>(sb));
            vol = p.cell_dims[0] * p.cell_dims[1] * p.cell_dims[2];
        } else {
            self_sigma<<<1, 256, 0, st>>>(ptr<double>(hb), 1, p.a, p.b, p.self_mode, NQ, ptr<double>(gx),
                                          ptr<double>(gw), ptr<double>(sb));
        }
        KF_LAUNCH();
        double s = 0;
        KF_CUDA(cudaMemcpyAsync(&s, sb.p, 8, cudaMemcpyDeviceToHost, st));
        KF_CUDA(cudaStreamSynchronize(st));
        fill_uniform<<<nb(n, 256), 256, 0, st>>>(n, s, vol, ptr<double>(p.sigma), ptr<double>(p.w));
        KF_LAUNCH();
        KF_CUDA(cudaStreamSynchronize(st));
        dev_free(hb); dev_free(sb); dev_free(gx); dev_free(gw);
        return KIFMM_OK;
    }
    DevBuf key, val, tk, tv, hist, flag, pos, scan_tmp, hs, su;
    KF_TRY(dev_alloc(key, n * 8));
    KF_TRY(dev_alloc(val, n * 4));
    KF_TRY(dev_alloc(flag, n * 4));
    KF_TRY(dev_alloc(pos, n * 4));
    h_bits<<<nb(n, 256), 256, 0, st>>>(h_dev, ptr<int32_t>(p.tree.perm), n, ptr<uint64_t>(key), ptr<int32_t>(val));
    KF_LAUNCH();
    KF_TRY(radix_sort_pairs(ptr<uint64_t>(key), ptr<int32_t>(val), n, 64, st, tk, tv, hist));
    uniq_flags<<<nb(n, 256), 256, 0, st>>>(ptr<uint64_t>(key), n, ptr<int32_t>(flag));
    KF_LAUNCH();
    int32_t nu = 0;
    KF_TRY(device_scan_i32(ptr<int32_t>(flag), ptr<int32_t>(pos), n, &nu, st, scan_tmp));
    KF_TRY(dev_alloc(hs, (size_t)nu * 8));
    KF_TRY(dev_alloc(su, (size_t)nu * 8));
    uniq_gather<<<nb(n, 256), 256, 0, st>>>(ptr<uint64_t>(key), ptr<int32_t>(flag), ptr<int32_t>(pos), n,
                                            ptr<double>(hs));
    KF_LAUNCH();
    if (p.kind)
        self_sigma_kind<<<nu, 256, 0, st>>>(ptr<double>(hs), nu, 0.0, 0.0, 0.0, make_kparams_kind(p.kind, p.a, p.b),
                                            p.self_mode, NQ, ptr<double>(gx), ptr<double>(gw), ptr<double>(su));
    else
        self_sigma<<<nu, 256, 0, st>>>(ptr<double>(hs), nu, p.a, p.b, p.self_mode, NQ, ptr<double>(gx),
                                       ptr<double>(gw), ptr<double>(su));
    KF_LAUNCH();
    scatter_sigma<<<nb(n, 256), 256, 0, st>>>(ptr<uint64_t>(key), ptr<int32_t>(val), ptr<int32_t>(flag),
                                              ptr<int32_t>(pos), n, ptr<double>(su), ptr<double>(p.sigma),
                                              ptr<double>(p.w));
    KF_LAUNCH();
    KF_CUDA(cudaStreamSynchronize(st));
    for (DevBuf* d : {&key, &val, &tk, &tv, &hist, &flag, &pos, &scan_tmp, &hs, &su, &gx, &gw}) dev_free(*d);
    return KIFMM_OK;
}

}  // namespace kifmm
