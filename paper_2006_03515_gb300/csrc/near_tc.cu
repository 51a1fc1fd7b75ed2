// Near field (Eq. (nearfar), first sum) on a uniform lattice, on the tensor cores.
//
// When every leaf is a full block of nc x nc x nc cells of one uniform grid (the same
// level for all leaves, cell centres on the lattice, the points of each leaf in the same
// local order), the contribution of a neighbour leaf A at offset delta (in {-1, 0, 1}^3)
// to the targets of B is one fixed matrix applied to A's weights:
//   near[B][i] += sum_j K_delta[i][j] q[A][j],  K_delta[i][j] = K(h |nc delta + c_j - c_i|),
// c_i the integer cell of local point i, and K_0[i][i] = 0 (the self term is added apart).
// Every pair of the U lists is still summed; only the kernel values, which depend on the
// geometry alone, are tabulated at plan time, like the far-field translation operators.
// The 27 matrices (R = nc^3 rows) go through the tensor-core translation kernel of M2L
// (FP16 x 3 split, per-offset FP32 accumulators), with the leaves' weight rows as its
// coefficient rows. Plans whose points are not such a lattice use the pair kernel.
//
// On the same lattice (leaves at level >= 2, no W or X lists) every leaf also shares the
// operators between its cells and its own surfaces or nodes, tabulated here in FP64:
//  * S2M: the check matrix P[j][i] = K(|r_out r s_j - y_i|) (surface form), or the P2M
//    interpolation weights S3(xbar_m, u_i) (Chebyshev form), applied per leaf in FP32;
//  * the leaves' upward coefficients c = (G1 P) q, sliced exactly on the tensor cores like
//    the other upward solves (surface form, FP64 accuracy, no check potentials);
//  * the local part of L2P from the leaves' d through Q = P^T U Sigma^+ (surface form), on
//    the tensor cores or in FP32.
// In exact arithmetic each is the generic path's operator, reassociated.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>

#include "internal.cuh"
#include "kernel.cuh"
#include "cheb.cuh"

namespace kifmm {

static inline unsigned nbn(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// local cell index ix + nc (iy + nc iz) of every sorted point inside its leaf; *bad is set
// where a point is off the lattice (more than 1e-6 cells) or outside its leaf
__global__ void k_nf_local(const double* pts, const int32_t* leaf_of, const double* centre, int64_t n, double h,
                           double r, int nc, int32_t* lidx, int* bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int B = leaf_of[i];
    int idx[3];
    for (int k = 0; k < 3; ++k) {
        const double u = (pts[3 * i + k] - (centre[3 * (int64_t)B + k] - r)) / h - 0.5;
        const double ur = rint(u);
        idx[k] = (int)ur;
        if (fabs(u - ur) > 1e-6 || idx[k] < 0 || idx[k] >= nc) atomicOr(bad, 1);
    }
    lidx[i] = idx[0] + nc * (idx[1] + nc * idx[2]);
}

// every leaf: npl points, the k-th of them at local cell ref[k], at level lf, and leaf
// ordinal o holding the points o npl .. (o + 1) npl - 1
__global__ void k_nf_check(const int32_t* leaves, int64_t nleaves, const int32_t* pstart, const int32_t* pend,
                           const int32_t* level, int lf, int npl, const int32_t* lidx, const int32_t* ref, int* bad) {
    const int64_t o = blockIdx.x;
    if (o >= nleaves) return;
    const int B = leaves[o];
    if (threadIdx.x == 0 && (pend[B] - pstart[B] != npl || pstart[B] != o * npl || level[B] != lf)) atomicOr(bad, 1);
    if (pend[B] - pstart[B] != npl) return;
    for (int k = threadIdx.x; k < npl; k += blockDim.x)
        if (lidx[pstart[B] + k] != ref[k]) atomicOr(bad, 1);
}

// utab[o][slot]: ordinal of the neighbour leaf of leaf o at the offset slot (-1 if none);
// every member of U(B) must be a same-level box within one box of B
__global__ void k_nf_utab(const int32_t* leaves, int64_t nleaves, const int32_t* uoff, const int32_t* uitems,
                          const int32_t* anchor, const int32_t* level, const int32_t* pstart, int npl, int32_t* utab,
                          int* bad) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nleaves) return;
    const int B = leaves[o];
    utab[o * kOffsetSlots + 3 + 7 * 3 + 49 * 3] = (int32_t)o;   // the leaf itself (offset 0)
    for (int u = uoff[B]; u < uoff[B + 1]; ++u) {
        const int A = uitems[u];
        const int dx = anchor[3 * A] - anchor[3 * B], dy = anchor[3 * A + 1] - anchor[3 * B + 1],
                  dz = anchor[3 * A + 2] - anchor[3 * B + 2];
        if (level[A] != level[B] || abs(dx) > 1 || abs(dy) > 1 || abs(dz) > 1) {
            atomicOr(bad, 1);
            continue;
        }
        utab[o * kOffsetSlots + (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3)] = pstart[A] / npl;
    }
}

// T[slot][i][j] = K(h |nc delta + c_j - c_i|) for the 27 near slots (zero on the diagonal of
// delta = 0); the other slots are left as they are (zero)
__global__ void k_nf_table(const int32_t* ref, int nc, int R, double h, KParams kp, double* T) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 27LL * R * R) return;
    const int d = (int)(e / ((int64_t)R * R)), i = (int)((e / R) % R), j = (int)(e % R);
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    const int ci = ref[i], cj = ref[j];
    const int ix = ci % nc, iy = (ci / nc) % nc, iz = ci / (nc * nc);
    const int jx = cj % nc, jy = (cj / nc) % nc, jz = cj / (nc * nc);
    const double ux = nc * dx + jx - ix, uy = nc * dy + jy - iy, uz = nc * dz + jz - iz;
    const int slot = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
    const double rr = h * sqrt(ux * ux + uy * uy + uz * uz);
    T[((int64_t)slot * R + i) * R + j] = rr > 0.0 ? kern_f64(rr, kp) : 0.0;
}

// S in the caller's order: C (near + far + sigma I); the far part from far[i], or, when fst is
// given, from the FP32 rows of the tensor-core L2P (row of the leaf's box, npl cells, stride R)
template <class TO>
__global__ void k_nf_finish(const float* near, const double* far, const float* fst, const int32_t* leaves, int npl,
                            int R, const double* sigma, const double* Is, const int32_t* perm, int64_t n,
                            int64_t n_real, double C, TO* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || perm[i] >= n_real) return;   // (padding cells have no output)
    const double fa = fst ? (double)fst[(int64_t)leaves[i / npl] * R + i % npl] : far[i];
    out[perm[i]] = (TO)(C * ((double)near[i] + fa + sigma[i] * Is[i]));
}

// T[i][k] = sum_j P[j][i] Ub[j][k] in FP64 for i < npl, k < R: the leaf's local expansion from
// its d as the square table [1][R][R] of the tensor-core kernel (rows >= npl zero)
__global__ void k_lat_QT(const double* Ub, int S, int R, const double* surf, const int32_t* ref, int nc, double r,
                         double ro, double h, KParams kp, double* T) {
    const int npl = nc * nc * nc;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)npl * R) return;
    const int i = (int)(e / R), k = (int)(e % R);
    const int ci = ref[i];
    const double y[3] = {(ci % nc + 0.5) * h - r, ((ci / nc) % nc + 0.5) * h - r, (ci / (nc * nc) + 0.5) * h - r};
    double sum = 0.0;
    for (int j = 0; j < S; ++j) {
        double d2 = 0;
        for (int a = 0; a < 3; ++a) {
            const double d = ro * r * surf[3 * j + a] - y[a];
            d2 += d * d;
        }
        sum += kern_f64(sqrt(d2), kp) * Ub[(int64_t)j * R + k];
    }
    T[(int64_t)i * R + k] = sum;
}

__global__ void k_iota(int32_t* v, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) v[e] = (int32_t)e;
}

// ------------------------------------------------------------------------------------
// S2M and the local part of L2P on the same lattice: every leaf sees the same matrix
//   P[j][i] = K(|ro r s_j - y_i|),  y_i = (c_i + 1/2) h - r  (leaf-centred coordinates),
// between its check / downward equivalent surface (radius ro r) and its own cells, so
//   chk[B][j] = sum_i P[j][i] q[B][i]   and   far[B][i] = sum_j P[j][i] phi_d[B][j].
// FP64 kernel values rounded once to FP32; sums in FP32 blocks of 8 terms, compensated
// across blocks (as the kernels that evaluate the kernel do).
// ------------------------------------------------------------------------------------
__global__ void k_lat_table(const double* surf, int S, const int32_t* ref, int nc, double r, double ro, double h,
                            KParams kp, float* P) {
    const int npl = nc * nc * nc;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)S * npl) return;
    const int j = (int)(e / npl), i = (int)(e % npl);
    const int ci = ref[i];
    const int c3[3] = {ci % nc, (ci / nc) % nc, ci / (nc * nc)};
    double d2 = 0;
    for (int k = 0; k < 3; ++k) {
        const double d = ro * r * surf[3 * j + k] - ((c3[k] + 0.5) * h - r);
        d2 += d * d;
    }
    P[(int64_t)j * (npl + 1) + i] = (float)kern_f64(sqrt(d2), kp);
}

constexpr int LT_T = 128, LT_LV = 8;   // threads; leaves per pass of the S2M kernel
constexpr int LT_LT = 4;               // leaves per thread and pass of the L2P kernel

// the matrix (n floats) into shared memory: 16-byte loads, several in flight per thread, and
// the last n % 4 floats one by one
__device__ __forceinline__ void lat_load(const float* __restrict__ P, float* Ps, int n) {
    const int n4 = n / 4;
    const float4* src = reinterpret_cast<const float4*>(P);
    float4* dst = reinterpret_cast<float4*>(Ps);
    int e = threadIdx.x;
    for (; e + 3 * LT_T < n4; e += 4 * LT_T) {
        const float4 a = src[e], b = src[e + LT_T], c = src[e + 2 * LT_T], d = src[e + 3 * LT_T];
        dst[e] = a;
        dst[e + LT_T] = b;
        dst[e + 2 * LT_T] = c;
        dst[e + 3 * LT_T] = d;
    }
    for (; e < n4; e += LT_T) dst[e] = src[e];
    for (int k = 4 * n4 + threadIdx.x; k < n; k += LT_T) Ps[k] = P[k];
}

// chk[leaf B][j] = sum_i P[j][i] q[B][i]; rows j over the threads (P rows padded to npl + 1
// floats: conflict-free), LT_LV leaves per pass sharing each P load
__global__ void __launch_bounds__(LT_T) k_lat_s2m(const float* __restrict__ P, int S, int npl,
                                                  const int32_t* __restrict__ leaves, int64_t nl,
                                                  const double* __restrict__ q, double* __restrict__ chk, int ldo) {
    extern __shared__ float lsm[];
    float* Ps = lsm;                          // [S][npl + 1]
    float* qs = Ps + (int64_t)S * (npl + 1);   // [LT_LV][npl]
    lat_load(P, Ps, S * (npl + 1));
    for (int64_t o0 = (int64_t)blockIdx.x * LT_LV; o0 < nl; o0 += (int64_t)gridDim.x * LT_LV) {
        __syncthreads();
        for (int e = threadIdx.x; e < LT_LV * npl; e += LT_T) {
            const int64_t o = o0 + e / npl;
            qs[e] = o < nl ? (float)q[o * npl + e % npl] : 0.f;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < S; j += LT_T) {
            const float* row = Ps + (int64_t)j * (npl + 1);
            Kahan k[LT_LV];
            for (int i0 = 0; i0 < npl; i0 += 8) {
                float part[LT_LV] = {};
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float w = row[i0 + u];
#pragma unroll
                    for (int l = 0; l < LT_LV; ++l) part[l] = fmaf(w, qs[l * npl + i0 + u], part[l]);
                }
#pragma unroll
                for (int l = 0; l < LT_LV; ++l) k[l].add(part[l]);
            }
#pragma unroll
            for (int l = 0; l < LT_LV; ++l)
                if (o0 + l < nl) chk[(int64_t)leaves[o0 + l] * ldo + j] = k[l].value();
        }
    }
}

// Chebyshev form on the lattice: P[m][i] = S3(xbar_m, u_i) and Q[m][i] = P[m][i] (the same
// weights read the other way in L2P), u_i = ((c_i + 1/2) h - r) / r the cell centre in box units
__global__ void k_lat_cheb_table(int p, const double* tab, const int32_t* ref, int nc, double r, double h, float* P,
                                 float* Q) {
    const int npl = nc * nc * nc, S = p * p * p;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)S * npl) return;
    const int m = (int)(e / npl), i = (int)(e % npl);
    const int ci = ref[i];
    const int c3[3] = {ci % nc, (ci / nc) % nc, ci / (nc * nc)};
    const int m3[3] = {m % p, (m / p) % p, m / (p * p)};
    double w = 1.0;
    for (int a = 0; a < 3; ++a) {
        double t[kChebMaxP];
        cheb_T(((c3[a] + 0.5) * h - r) / r, p, t);
        w *= cheb_S(t, p, tab + m3[a] * kChebTab);
    }
    P[(int64_t)m * (npl + 1) + i] = (float)w;
    Q[(int64_t)m * (npl + 1) + i] = (float)w;
}

// Q[k][i] = sum_j P[j][i] Ub[j][k] in FP64, rounded once: the local expansion of a leaf
// straight from its downward coefficients d (phi_d = Ub d), rows padded to npl + 1
__global__ void k_lat_Q(const double* Ub, int S, int R, const double* surf, const int32_t* ref, int nc, double r,
                        double ro, double h, KParams kp, float* Q) {
    const int npl = nc * nc * nc;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)R * npl) return;
    const int k = (int)(e / npl), i = (int)(e % npl);
    const int ci = ref[i];
    const double y[3] = {(ci % nc + 0.5) * h - r, ((ci / nc) % nc + 0.5) * h - r, (ci / (nc * nc) + 0.5) * h - r};
    double sum = 0.0;
    for (int j = 0; j < S; ++j) {
        double d2 = 0;
        for (int a = 0; a < 3; ++a) {
            const double d = ro * r * surf[3 * j + a] - y[a];
            d2 += d * d;
        }
        sum += kern_f64(sqrt(d2), kp) * Ub[(int64_t)j * R + k];
    }
    Q[(int64_t)k * (npl + 1) + i] = (float)sum;
}

// far[o npl + i] = sum_k Q[k][i] d[leaf B][k] for the leaves (ordinal o, box B), k < K (d rows
// of stride K); per pass LT_T / npl thread groups of npl targets, each group LT_LT leaves
__global__ void __launch_bounds__(LT_T) k_lat_l2p(const float* __restrict__ P, int S, int npl,
                                                  const int32_t* __restrict__ leaves, int64_t nl,
                                                  const float* __restrict__ phid, double* __restrict__ far) {
    extern __shared__ float lsm[];
    float* Ps = lsm;                          // [S][npl + 1]
    float* ps = Ps + (int64_t)S * (npl + 1);   // [LT_T / npl * LT_LT][S]
    const int lpp = LT_T / npl * LT_LT;
    lat_load(P, Ps, S * (npl + 1));
    const int grp = threadIdx.x / npl, i = threadIdx.x % npl;
    for (int64_t o0 = (int64_t)blockIdx.x * lpp; o0 < nl; o0 += (int64_t)gridDim.x * lpp) {
        __syncthreads();
        for (int e = threadIdx.x; e < lpp * S; e += LT_T) {
            const int64_t o = o0 + e / S;
            ps[e] = o < nl ? phid[(int64_t)leaves[o] * S + e % S] : 0.f;
        }
        __syncthreads();
        const float* pr = ps + grp * LT_LT * S;
        Kahan k[LT_LT];
        int j = 0;
        for (; j + 7 < S; j += 8) {
            float part[LT_LT] = {};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float w = Ps[(int64_t)(j + u) * (npl + 1) + i];
#pragma unroll
                for (int l = 0; l < LT_LT; ++l) part[l] = fmaf(w, pr[l * S + j + u], part[l]);
            }
#pragma unroll
            for (int l = 0; l < LT_LT; ++l) k[l].add(part[l]);
        }
        for (; j < S; ++j) {
            const float w = Ps[(int64_t)j * (npl + 1) + i];
#pragma unroll
            for (int l = 0; l < LT_LT; ++l) k[l].add(w * pr[l * S + j]);
        }
#pragma unroll
        for (int l = 0; l < LT_LT; ++l) {
            const int64_t o = o0 + grp * LT_LT + l;
            if (o < nl) far[o * npl + i] = k[l].value();
        }
    }
}

static size_t lat_s2m_smem(int S, int npl) { return ((size_t)S * (npl + 1) + (size_t)LT_LV * npl) * 4; }
static size_t lat_l2p_smem(int S, int npl) { return ((size_t)S * (npl + 1) + (size_t)(LT_T / npl) * LT_LT * S) * 4; }

int lat_s2m(Plan& p) {   // surface form: check potentials; Chebyshev: node weights straight into c
    const unsigned g = (unsigned)std::min<int64_t>((p.nleaves + LT_LV - 1) / LT_LV, 8LL * p.num_sms);
    k_lat_s2m<<<g, LT_T, lat_s2m_smem(p.S, p.nf_R), p.stream>>>(ptr<float>(p.lat_P), p.S, p.nf_R,
                                                                ptr<int32_t>(p.leaves), p.nleaves, ptr<double>(p.q),
                                                                p.cheb ? ptr<double>(p.cu) : ptr<double>(p.chk),
                                                                p.cheb ? p.R : p.S);
    KF_LAUNCH();
    return KIFMM_OK;
}

int lat_l2p(Plan& p) {
    if (p.lat_l2p_tc) {   // tensor cores: the leaves' d split FP16 x 3, one slot (the leaf itself)
        cudaStream_t st = p.stream;
        const int R = p.R, lf = p.nf_level;
        const int64_t lo = p.tree.level_start[lf], cnt = p.tree.level_start[lf + 1] - lo;
        KF_TRY(m2l_tc_split_f32(st, ptr<float>(p.dd) + lo * R, cnt, R, static_cast<char*>(p.chi.p) + lo * R * 2,
                                static_cast<char*>(p.clo.p) + lo * R * 2, ptr<int>(p.cexp) + lo));
        M2LTables tabs{};
        tabs.hi[lf] = p.lat_Thi.p;
        tabs.lo[lf] = p.lat_Tlo.p;
        tabs.sT[lf] = p.lat_sT;
        return launch_tc_translate(st, tabs, R, ptr<int4>(p.nf_tiles), p.nf_ntiles, ptr<int32_t>(p.leaves),
                                   ptr<int32_t>(p.lat_iota), 1, ptr<int32_t>(p.lat_slots), p.chi.p, p.clo.p,
                                   ptr<int>(p.cexp), ptr<float>(p.lat_fst), 0, ptr<int>(p.err));
    }
    const int lpp = LT_T / p.nf_R * LT_LT;
    const unsigned g = (unsigned)std::min<int64_t>((p.nleaves + lpp - 1) / lpp, 8LL * p.num_sms);
    k_lat_l2p<<<g, LT_T, lat_l2p_smem(p.R, p.nf_R), p.stream>>>(ptr<float>(p.lat_Q), p.R, p.nf_R,
                                                                ptr<int32_t>(p.leaves), p.nleaves, ptr<float>(p.dd),
                                                                ptr<double>(p.far));
    KF_LAUNCH();
    return KIFMM_OK;
}

int near_tc_plan(Plan& p) {
    p.near_tc = false;
    const char* env = std::getenv("KIFMM_P2P");
    if (env && std::string(env) == "generic") return KIFMM_OK;
    Tree& t = p.tree;
    if (p.precision != KIFMM_MIXED || !(p.uniform_h > 0.0) || p.nleaves < 1) return KIFMM_OK;
    // the level of the first leaf; k_nf_check below requires every leaf on it
    int32_t first = 0, lf = 0;
    cudaStream_t st = p.stream;
    KF_CUDA(cudaMemcpyAsync(&first, p.leaves.p, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    KF_CUDA(cudaMemcpyAsync(&lf, ptr<int32_t>(t.level) + first, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    if (lf < 0 || lf > kMaxLevel) return KIFMM_OK;
    const double h = p.uniform_h, r = t.side / (double)(2ll << lf);
    const int nc = (int)std::lround(2.0 * r / h);
    if (nc < 1 || std::fabs(nc * h - 2.0 * r) > 1e-9 * 2.0 * r) return KIFMM_OK;
    const int npl = nc * nc * nc, R = npl;
    // 64-cell leaves: with K = 512 (8^3 cells) a slot's truncating tensor-core accumulation
    // biased the near field by about 2e-6, beyond the mixed form's target
    if (npl != 64 || !m2l_tc_supported(R) || (int64_t)npl * p.nleaves != t.n) return KIFMM_OK;
    const int64_t n = t.n, nl = p.nleaves;
    DevBuf lidx, bad;
    DevBuf& ref = p.nf_ref;   // kept for the leaves' upward operator
    KF_TRY(dev_alloc(lidx, n * 4));
    KF_TRY(dev_alloc(ref, npl * 4));
    KF_TRY(dev_alloc(bad, 4));
    KF_CUDA(cudaMemsetAsync(bad.p, 0, 4, st));
    k_nf_local<<<nbn(n, 256), 256, 0, st>>>(ptr<double>(p.pts), ptr<int32_t>(p.leaf_of), ptr<double>(t.centre), n, h,
                                             r, nc, ptr<int32_t>(lidx), ptr<int>(bad));
    KF_LAUNCH();
    // the local order of the first leaf is the reference; it must be a permutation of the cells
    int32_t p0 = 0;
    KF_CUDA(cudaMemcpyAsync(&p0, ptr<int32_t>(t.pstart) + first, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    auto release = [&]() {
        for (DevBuf* d : {&lidx, &bad}) dev_free(*d);
    };
    auto give_up = [&]() {
        release();
        dev_free(ref);
        return KIFMM_OK;
    };
    if (p0 != 0) return give_up();   // else the first leaf holds points 0 .. npl - 1 (npl nleaves = n)
    std::vector<int32_t> href(npl);
    KF_CUDA(cudaMemcpyAsync(href.data(), lidx.p, npl * 4, cudaMemcpyDeviceToHost, st));
    int hbad = 0;
    KF_CUDA(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    if (hbad) return give_up();
    {
        std::vector<char> seen(npl, 0);
        for (int k = 0; k < npl; ++k) {
            if (href[k] < 0 || href[k] >= npl || seen[href[k]]) return give_up();
            seen[href[k]] = 1;
        }
    }
    KF_CUDA(cudaMemcpyAsync(ref.p, href.data(), npl * 4, cudaMemcpyHostToDevice, st));
    k_nf_check<<<(unsigned)nl, 128, 0, st>>>(ptr<int32_t>(p.leaves), nl, ptr<int32_t>(t.pstart), ptr<int32_t>(t.pend),
                                              ptr<int32_t>(t.level), lf, npl, ptr<int32_t>(lidx), ptr<int32_t>(ref),
                                              ptr<int>(bad));
    KF_LAUNCH();
    KF_TRY(dev_alloc(p.nf_utab, (size_t)nl * kOffsetSlots * 4));
    KF_CUDA(cudaMemsetAsync(p.nf_utab.p, 0xFF, (size_t)nl * kOffsetSlots * 4, st));
    k_nf_utab<<<nbn(nl, 128), 128, 0, st>>>(ptr<int32_t>(p.leaves), nl, ptr<int32_t>(p.lists[0].off),
                                             ptr<int32_t>(p.lists[0].items), ptr<int32_t>(t.anchor),
                                             ptr<int32_t>(t.level), ptr<int32_t>(t.pstart), npl,
                                             ptr<int32_t>(p.nf_utab), ptr<int>(bad));
    KF_LAUNCH();
    KF_CUDA(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    if (hbad) {
        dev_free(p.nf_utab);
        return give_up();
    }
    // the 27 near-offset matrices, FP64, then their FP16 hi / lo images for the tensor cores
    DevBuf T;
    const int64_t RR = (int64_t)R * R;
    KF_TRY(dev_alloc(T, kOffsetSlots * RR * 8));
    KF_CUDA(cudaMemsetAsync(T.p, 0, kOffsetSlots * RR * 8, st));
    k_nf_table<<<nbn(27 * RR, 256), 256, 0, st>>>(ptr<int32_t>(ref), nc, R, h, make_kparams_kind(p.kind, p.a, p.b), ptr<double>(T));
    KF_LAUNCH();
    KF_TRY(dev_alloc(p.nf_Thi, (size_t)m2l_tc_table_elems(R) * 2));
    KF_TRY(dev_alloc(p.nf_Tlo, (size_t)m2l_tc_table_elems(R) * 2));
    KF_TRY(m2l_tc_prepare(st, ptr<double>(T), R, p.nf_Thi.p, p.nf_Tlo.p, &p.nf_sT));
    // S2M (P2M) and local L2P on the lattice: leaves at level >= 2, no W / X lists. Surface
    // form: the check matrix P and Q = P^T U Sigma^+; Chebyshev form: the interpolation
    // weights S3(xbar_m, u_i) of the leaf's cells for P2M (its L2P keeps the interpolation
    // kernel: with 512 rows the matrix kernel fits one block per SM and ran slower).
    p.lat_far = false;
    const size_t lat_smem_max = 200 * 1024;
    if (p.cheb && lf >= 2 && p.lists[2].len == 0 && p.lists[3].len == 0 && LT_T % npl == 0 &&
        lat_s2m_smem(p.S, npl) <= lat_smem_max && lat_l2p_smem(p.R, npl) <= lat_smem_max) {
        KF_TRY(dev_alloc(p.lat_P, (size_t)p.S * (npl + 1) * 4));
        KF_TRY(dev_alloc(p.lat_Q, (size_t)p.R * (npl + 1) * 4));
        KF_CUDA(cudaMemsetAsync(p.lat_P.p, 0, (size_t)p.S * (npl + 1) * 4, st));
        KF_CUDA(cudaMemsetAsync(p.lat_Q.p, 0, (size_t)p.R * (npl + 1) * 4, st));
        k_lat_cheb_table<<<nbn((int64_t)p.S * npl, 128), 128, 0, st>>>(p.m0, ptr<double>(p.ctab), ptr<int32_t>(ref), nc,
                                                                       r, h, ptr<float>(p.lat_P), ptr<float>(p.lat_Q));
        KF_LAUNCH();
        for (const void* fn : {(const void*)k_lat_s2m, (const void*)k_lat_l2p})
            KF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lat_smem_max));
        p.lat_far = true;
    }
    if (!p.cheb && lf >= 2 && p.lists[2].len == 0 && p.lists[3].len == 0 && LT_T % npl == 0 &&
        lat_s2m_smem(p.S, npl) <= 96 * 1024 && lat_l2p_smem(p.R, npl) <= 96 * 1024) {
        KF_TRY(dev_alloc(p.lat_P, (size_t)p.S * (npl + 1) * 4));
        KF_CUDA(cudaMemsetAsync(p.lat_P.p, 0, (size_t)p.S * (npl + 1) * 4, st));
        k_lat_table<<<nbn((int64_t)p.S * npl, 256), 256, 0, st>>>(ptr<double>(p.surf), p.S, ptr<int32_t>(ref), nc, r,
                                                                   p.r_out, h, make_kparams_kind(p.kind, p.a, p.b),
                                                                   ptr<float>(p.lat_P));
        KF_LAUNCH();
        KF_TRY(dev_alloc(p.lat_Q, (size_t)p.R * (npl + 1) * 4));
        KF_CUDA(cudaMemsetAsync(p.lat_Q.p, 0, (size_t)p.R * (npl + 1) * 4, st));
        k_lat_Q<<<nbn((int64_t)p.R * npl, 128), 128, 0, st>>>(ptr<double>(p.ops[lf].Ub), p.S, p.R, ptr<double>(p.surf),
                                                               ptr<int32_t>(ref), nc, r, p.r_out, h,
                                                               make_kparams_kind(p.kind, p.a, p.b),
                                                               ptr<float>(p.lat_Q));
        KF_LAUNCH();
        for (const void* fn : {(const void*)k_lat_s2m, (const void*)k_lat_l2p})
            KF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        p.lat_far = true;
        // the same local expansion through the tensor-core kernel (mixed form with the tensor M2L)
        if (p.m2l_tensor) {
            DevBuf QT;
            const int64_t RR = (int64_t)p.R * p.R;
            KF_TRY(dev_alloc(QT, RR * 8));
            KF_CUDA(cudaMemsetAsync(QT.p, 0, RR * 8, st));
            k_lat_QT<<<nbn((int64_t)npl * p.R, 128), 128, 0, st>>>(ptr<double>(p.ops[lf].Ub), p.S, p.R,
                                                                    ptr<double>(p.surf), ptr<int32_t>(ref), nc, r,
                                                                    p.r_out, h,
                                                                    make_kparams_kind(p.kind, p.a, p.b), ptr<double>(QT));
            KF_LAUNCH();
            KF_TRY(dev_alloc(p.lat_Thi, (size_t)m2l_tc_table_elems(p.R, 1) * 2));
            KF_TRY(dev_alloc(p.lat_Tlo, (size_t)m2l_tc_table_elems(p.R, 1) * 2));
            KF_TRY(m2l_tc_prepare(st, ptr<double>(QT), p.R, p.lat_Thi.p, p.lat_Tlo.p, &p.lat_sT, 1));
            KF_TRY(dev_alloc(p.lat_iota, (size_t)t.nboxes * 4));
            k_iota<<<nbn(t.nboxes, 256), 256, 0, st>>>(ptr<int32_t>(p.lat_iota), t.nboxes);
            KF_LAUNCH();
            KF_TRY(dev_alloc(p.lat_fst, (size_t)t.nboxes * p.R * 4));
            KF_CUDA(cudaStreamSynchronize(st));
            dev_free(QT);
            p.lat_l2p_tc = true;
        }
    }
    // tiles of 128 leaves (ordinals), every tile over the 27 near slots
    const int ntiles = (int)((nl + 127) / 128);
    std::vector<int4> tiles(ntiles);
    for (int k = 0; k < ntiles; ++k) tiles[k] = make_int4(lf, 128 * k, (int)std::min<int64_t>(128, nl - 128LL * k), 0);
    std::vector<int32_t> slots((size_t)ntiles * kSlotStride, 0), ids(nl);
    for (int k = 0; k < ntiles; ++k) {
        int32_t* s = slots.data() + (size_t)k * kSlotStride;
        s[0] = 27;
        int c = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) s[1 + c++] = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
    }
    for (int64_t o = 0; o < nl; ++o) ids[o] = (int32_t)o;
    if (p.lat_l2p_tc) {   // one slot (0) per leaf tile
        std::vector<int32_t> ls((size_t)ntiles * kSlotStride, 0);
        for (int k = 0; k < ntiles; ++k) ls[(size_t)k * kSlotStride] = 1;
        KF_TRY(dev_alloc(p.lat_slots, ls.size() * 4));
        KF_CUDA(cudaMemcpyAsync(p.lat_slots.p, ls.data(), ls.size() * 4, cudaMemcpyHostToDevice, st));
    }
    KF_TRY(dev_alloc(p.nf_tiles, tiles.size() * sizeof(int4)));
    KF_TRY(dev_alloc(p.nf_slots, slots.size() * 4));
    KF_TRY(dev_alloc(p.nf_boxes, ids.size() * 4));
    KF_CUDA(cudaMemcpyAsync(p.nf_tiles.p, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    KF_CUDA(cudaMemcpyAsync(p.nf_slots.p, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice, st));
    KF_CUDA(cudaMemcpyAsync(p.nf_boxes.p, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice, st));
    KF_TRY(dev_alloc(p.nf_qhi, (size_t)n * 2));
    KF_TRY(dev_alloc(p.nf_qlo, (size_t)n * 2));
    KF_TRY(dev_alloc(p.nf_qexp, (size_t)nl * 4));
    KF_TRY(dev_alloc(p.nf_near, (size_t)n * 4));
    KF_CUDA(cudaStreamSynchronize(st));
    dev_free(T);
    release();
    p.nf_R = R;
    p.nf_level = lf;
    p.nf_ntiles = ntiles;
    p.near_tc = true;
    // the near sums need only the sorted weights: their own stream lets them fill the SMs that
    // the M2L's last wave and the downward pass leave idle (KIFMM_NEAR_STREAM=same keeps them
    // on the plan's stream, =early forks them right after the scatter of the weights)
    const char* ns = std::getenv("KIFMM_NEAR_STREAM");
    p.near_fork_early = ns && std::string(ns) == "early";
    if (!(ns && std::string(ns) == "same") && !p.near_st) {
        KF_CUDA(cudaStreamCreateWithFlags(&p.near_st, cudaStreamNonBlocking));
        for (auto& e : p.near_ev) KF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    return KIFMM_OK;
}

// M[r][i] = sum_j G1[r][j] P[j][i] in FP64: the leaves' upward coefficients c = M q straight
// from their weights (G1 the level's pseudo-inverse, P the check matrix of k_lat_table)
__global__ void k_lat_M(const double* G1, int S, int rank, const double* surf, const int32_t* ref, int nc, double r,
                        double ro, double h, KParams kp, double* M) {
    const int npl = nc * nc * nc;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rank * npl) return;
    const int rr = (int)(e / npl), i = (int)(e % npl);
    const int ci = ref[i];
    const double y[3] = {(ci % nc + 0.5) * h - r, ((ci / nc) % nc + 0.5) * h - r, (ci / (nc * nc) + 0.5) * h - r};
    double sum = 0.0;
    for (int j = 0; j < S; ++j) {
        double d2 = 0;
        for (int k = 0; k < 3; ++k) {
            const double d = ro * r * surf[3 * j + k] - y[k];
            d2 += d * d;
        }
        sum += G1[(int64_t)rr * S + j] * kern_f64(sqrt(d2), kp);
    }
    M[e] = sum;
}

int lat_up_plan(Plan& p) {
    p.lat_up = false;
    const int lf = p.nf_level, npl = p.nf_R;
    if (!p.lat_far || !p.oz || lf < 2 || lf >= p.tree.nlevels || p.nleaves <= p.oz_min) return KIFMM_OK;
    if (p.lv[lf].n_par != 0 || p.lv[lf].n_up != p.nleaves || !pinv_oz_supported(npl)) return KIFMM_OK;
    cudaStream_t st = p.stream;
    const LevelOps& op = p.ops[lf];
    const double h = p.uniform_h, r = p.tree.side / (double)(2ll << lf);
    const int nc = (int)std::lround(std::cbrt((double)npl));
    DevBuf M;
    KF_TRY(dev_alloc(M, (size_t)op.rank * npl * 8));
    k_lat_M<<<nbn((int64_t)op.rank * npl, 128), 128, 0, st>>>(ptr<double>(op.G1), p.S, op.rank, ptr<double>(p.surf),
                                                               ptr<int32_t>(p.nf_ref), nc, r, p.r_out, h,
                                                               make_kparams_kind(p.kind, p.a, p.b),
                                                               ptr<double>(M));
    KF_LAUNCH();
    KF_TRY(dev_alloc(p.lat_Mimg, pinv_oz_op_bytes(npl, op.rank)));
    KF_TRY(dev_alloc(p.lat_Mer, (size_t)((op.rank + 47) / 48 * 48) * 4));
    KF_TRY(pinv_oz_prepare(st, ptr<double>(M), npl, op.rank, p.lat_Mimg.p, ptr<int>(p.lat_Mer)));
    KF_CUDA(cudaStreamSynchronize(st));
    dev_free(M);
    p.lat_up = true;
    return KIFMM_OK;
}

int lat_up_apply(Plan& p, double* cu, int64_t& nl) {
    int64_t extra = 0;
    KF_TRY(pinv_oz_apply(p.stream, ptr<double>(p.q), p.nf_R, ptr<int32_t>(p.leaves), ptr<int32_t>(p.nf_boxes),
                         (int)p.nleaves, p.lat_Mimg.p, ptr<int>(p.lat_Mer), p.ops[p.nf_level].rank, p.ozBox.p,
                         ptr<int>(p.ozEb), cu, p.R, ptr<int>(p.err), &extra));
    nl += extra;
    return KIFMM_OK;
}

// the per-offset contractions of the near field into nf_near, on stream st (they read only the
// sorted weights q)
int near_tc_contract(Plan& p, cudaStream_t st, int64_t& nl) {
    KF_TRY(m2l_tc_split(st, ptr<double>(p.q), p.nleaves, p.nf_R, p.nf_qhi.p, p.nf_qlo.p, ptr<int>(p.nf_qexp)));
    ++nl;
    M2LTables tabs{};
    tabs.hi[p.nf_level] = p.nf_Thi.p;
    tabs.lo[p.nf_level] = p.nf_Tlo.p;
    tabs.sT[p.nf_level] = p.nf_sT;
    KF_TRY(launch_m2l_tc(st, tabs, p.nf_R, ptr<int4>(p.nf_tiles), p.nf_ntiles, ptr<int32_t>(p.nf_boxes),
                         ptr<int32_t>(p.nf_utab), ptr<int32_t>(p.nf_slots), p.nf_qhi.p, p.nf_qlo.p, ptr<int>(p.nf_qexp),
                         ptr<float>(p.nf_near), ptr<int>(p.err)));
    ++nl;
    return KIFMM_OK;
}

// out = far + near + self term, on the plan's stream once nf_near is complete there
int near_tc_finish(Plan& p, const double* far, double C, void* out, int dtype, int64_t& nl) {
    cudaStream_t st = p.stream;
    const int64_t n = p.tree.n;
    const float* fst = p.lat_l2p_tc && p.tree.nlevels > 2 ? ptr<float>(p.lat_fst) : nullptr;
    if (dtype == KIFMM_F64)
        k_nf_finish<double><<<nbn(n, 256), 256, 0, st>>>(ptr<float>(p.nf_near), far, fst, ptr<int32_t>(p.leaves),
                                                          p.nf_R, p.R, ptr<double>(p.sigma), ptr<double>(p.Isort),
                                                          ptr<int32_t>(p.tree.perm), n, p.n_real, C, (double*)out);
    else
        k_nf_finish<float><<<nbn(n, 256), 256, 0, st>>>(ptr<float>(p.nf_near), far, fst, ptr<int32_t>(p.leaves),
                                                         p.nf_R, p.R, ptr<double>(p.sigma), ptr<double>(p.Isort),
                                                         ptr<int32_t>(p.tree.perm), n, p.n_real, C, (float*)out);
    KF_LAUNCH();
    ++nl;
    return KIFMM_OK;
}

}  // namespace kifmm
