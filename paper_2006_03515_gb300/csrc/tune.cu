// Importance-sampled error estimates and the accuracy-targeted autotuner.
//
// An estimate of the relative L2 error of a field S against the discrete sum (Sec. 3,
// Eq. (summation)) needs the sum only at k targets if they are drawn in proportion to the
// field: probability m_i = 0.5 |S_i| / sum |S| + 0.5 / n (a defensive mixture, every point
// keeps probability >= 0.5 / n), systematic sampling u_t = (t + U) / k, weight 1 / (k m_i).
// Then sum_t w_t e_t^2 and sum_t w_t S_t^2 estimate the whole field's sums, and a
// concentrated source is not missed the way uniform targets miss it.
//
// kifmm_tune builds a plan for every candidate (leaf size, surface order, surface radii),
// evaluates a representative source, estimates its error against the FP64 direct sum at
// such targets, times the evaluation, and keeps the fastest candidate whose estimate is at
// most half the caller's target (the factor covers the sampling error of the estimate).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "kernel.cuh"

namespace kifmm {

constexpr int IS_SC = 1024;   // prefix-sum block
constexpr int TR_T = 256, TR_CH = 1024;

__global__ void k_is_abs_sum(const double* S, int64_t n, double* out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += fabs(S[i]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, red[0]);
}
// m_i, inclusive prefix sums within blocks of 1024 (Hillis-Steele), block totals in blk
__global__ void k_is_scan(const double* S, int64_t n, const double* tot, double* cdf, double* blk) {
    __shared__ double sh[IS_SC];
    const int64_t i = (int64_t)blockIdx.x * IS_SC + threadIdx.x;
    const double t = tot[0];
    double v = 0.0;
    if (i < n) v = (t > 0.0 ? 0.5 * fabs(S[i]) / t : 0.0) + (t > 0.0 ? 0.5 : 1.0) / (double)n;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < IS_SC; o <<= 1) {
        const double x = threadIdx.x >= o ? sh[threadIdx.x - o] : 0.0;
        __syncthreads();
        sh[threadIdx.x] += x;
        __syncthreads();
    }
    if (i < n) cdf[i] = sh[threadIdx.x];
    if (threadIdx.x == IS_SC - 1) blk[blockIdx.x] = sh[IS_SC - 1];
}
// exclusive prefix sums of the nb block totals, one warp (each lane a contiguous run)
__global__ void k_is_scan_blocks(double* blk, int nb) {
    const int lane = threadIdx.x;
    const int per = (nb + 31) / 32, b0 = lane * per, b1 = min(nb, b0 + per);
    double s = 0.0;
    for (int b = b0; b < b1; ++b) s += blk[b];
    double x = s;   // inclusive scan of the lanes' run totals
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    double acc = x - s;
    for (int b = b0; b < b1; ++b) {
        const double v = blk[b];
        blk[b] = acc;
        acc += v;
    }
}
__global__ void k_is_add(double* cdf, int64_t n, const double* blk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cdf[i] += blk[i / IS_SC];
}
__global__ void k_is_inv(const int32_t* perm, int64_t nperm, int64_t n, int32_t* inv) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nperm && perm[k] < n) inv[perm[k]] = (int32_t)k;   // (perm >= n: padding cells)
}
// target t: the first i (caller order) with cdf[i] > u_t, its sorted index and weight
__global__ void k_is_draw(const double* cdf, int64_t n, int k, double U, const int32_t* inv, int32_t* tcaller,
                          int32_t* tsorted, double* wt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= k) return;
    const double total = cdf[n - 1];
    const double u = ((double)t + U) / (double)k * total;
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (cdf[mid] > u) hi = mid;
        else lo = mid + 1;
    }
    const double mi = (cdf[lo] - (lo > 0 ? cdf[lo - 1] : 0.0)) / total;
    if (tcaller) tcaller[t] = (int32_t)lo;
    if (tsorted) tsorted[t] = inv ? inv[lo] : (int32_t)lo;
    wt[t] = 1.0 / ((double)k * mi);
}

size_t importance_ws_bytes(int64_t n, int k) {
    return 8 * (size_t)n + 8 * (size_t)(n / IS_SC + 2) + 16 + 4 * (size_t)((n + 1) & ~(int64_t)1) + 8 * (size_t)k +
           64;
}

int importance_targets(cudaStream_t st, const double* S, int64_t n, int k, uint64_t seed, const int32_t* perm,
                       int64_t nperm, void* ws, int32_t* tcaller, int32_t* tsorted, double* wt, int num_sms) {
    uint64_t sst = seed * 6364136223846793005ull + 1442695040888963407ull;
    sst = sst * 6364136223846793005ull + 1442695040888963407ull;
    const double U = (double)(sst >> 11) * (1.0 / 9007199254740992.0);
    double* cdf = static_cast<double*>(ws);
    const int64_t nbk = (n + IS_SC - 1) / IS_SC;
    double* blk = cdf + n;
    double* tot = blk + nbk + 1;
    int32_t* inv = reinterpret_cast<int32_t*>(tot + 2);
    KF_CUDA(cudaMemsetAsync(tot, 0, 8, st));
    k_is_abs_sum<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4LL * num_sms), 256, 0, st>>>(S, n, tot);
    k_is_scan<<<(unsigned)nbk, IS_SC, 0, st>>>(S, n, tot, cdf, blk);
    k_is_scan_blocks<<<1, 32, 0, st>>>(blk, (int)nbk);
    k_is_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cdf, n, blk);
    if (perm) k_is_inv<<<(unsigned)((nperm + 255) / 256), 256, 0, st>>>(perm, nperm, n, inv);
    k_is_draw<<<(unsigned)((k + 127) / 128), 128, 0, st>>>(cdf, n, k, U, perm ? inv : nullptr, tcaller, tsorted, wt);
    KF_LAUNCH();
    return KIFMM_OK;
}

// FP64 direct sum at k targets (sorted indices), sources streamed once in chunks:
// acc[t] += sum_{j != i_t} K(|x_i - x_j|) q_j
__global__ void __launch_bounds__(TR_T) k_tune_ref(const double* pts, const double* q, const int32_t* targets, int k,
                                                   int64_t n, KParams kp, double* acc) {
    __shared__ double sx[TR_CH], sy[TR_CH], sz[TR_CH], sq[TR_CH];
    const int64_t j0 = (int64_t)blockIdx.x * TR_CH;
    const int m = (int)min((int64_t)TR_CH, n - j0);
    for (int e = threadIdx.x; e < m; e += TR_T) {
        const int64_t j = j0 + e;
        sx[e] = pts[3 * j];
        sy[e] = pts[3 * j + 1];
        sz[e] = pts[3 * j + 2];
        sq[e] = q[j];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += TR_T) {
        const int64_t i = targets[t];
        const double xi = pts[3 * i], yi = pts[3 * i + 1], zi = pts[3 * i + 2];
        const int self = (i >= j0 && i < j0 + m) ? (int)(i - j0) : -1;
        double a = 0.0;
        for (int e = 0; e < m; ++e) {
            if (e == self) continue;
            const double dx = xi - sx[e], dy = yi - sy[e], dz = zi - sz[e];
            a += kern_f64(sqrt(dx * dx + dy * dy + dz * dz), kp) * sq[e];
        }
        atomicAdd(acc + t, a);
    }
}
// ref[t] = acc[t] + sigma_i I_i (C = 1), in the sorted order's arrays
__global__ void k_tune_ref_fin(const double* acc, const int32_t* targets, int k, const double* sigma,
                               const double* Isort, double* ref) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < k) ref[t] = acc[t] + sigma[targets[t]] * Isort[targets[t]];
}
// importance-weighted relative error of S (caller order) at the targets
__global__ void k_tune_err(const double* S, const int32_t* tcaller, const double* ref, const double* wt, int k,
                           double* out) {
    __shared__ double a[256], b[256];
    double num = 0, den = 0;
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        const double d = S[tcaller[t]] - ref[t];
        num += wt[t] * d * d;
        den += wt[t] * ref[t] * ref[t];
    }
    a[threadIdx.x] = num;
    b[threadIdx.x] = den;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            a[threadIdx.x] += a[threadIdx.x + o];
            b[threadIdx.x] += b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(a[0] / fmax(b[0], 1e-300));
}

}  // namespace kifmm

using namespace kifmm;

extern "C" int kifmm_tune(const double* points, int64_t n, const double* cell_h, double uniform_h, const double* I,
                          double a, double b, const kifmm_opts* opts_in, const int* leaf, int nleaf, const int* order,
                          int norder, const double* radii, int nradii, double target, int k_samples, int reps,
                          kifmm_tune_entry* entries, kifmm_tune_entry* best) {
    set_error("");
    if (!points || n < 1 || !I || !leaf || nleaf < 1 || !order || norder < 1 || (nradii > 0 && !radii) ||
        nradii < 0 || !(target > 0.0) || k_samples < 1 || k_samples > 4096 || reps < 1 || !best) {
        set_error("kifmm_tune: need points, a source, candidate lists, target > 0, 1 <= k_samples <= 4096, reps >= 1");
        return KIFMM_ERR_ARG;
    }
    kifmm_opts o;
    if (opts_in) o = *opts_in;
    else kifmm_default_opts(&o);
    cudaStream_t st = (cudaStream_t)o.stream;
    const int nr = nradii > 0 ? nradii : 1;
    const int64_t ncand = (int64_t)nleaf * norder * nr;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // work space: S of a candidate (8 n), the draw's work space, targets (caller, sorted),
    // weights, per-target sums and references, the error
    const size_t wsb = importance_ws_bytes(n, k_samples);
    DevBuf Sb, wsd, tc, ts, wt, acc, ref, err;
    int rc = dev_alloc(Sb, (size_t)n * 8);
    if (!rc) rc = dev_alloc(wsd, wsb);
    if (!rc) rc = dev_alloc(tc, (size_t)k_samples * 4);
    if (!rc) rc = dev_alloc(ts, (size_t)k_samples * 4);
    if (!rc) rc = dev_alloc(wt, (size_t)k_samples * 8);
    if (!rc) rc = dev_alloc(acc, (size_t)k_samples * 8);
    if (!rc) rc = dev_alloc(ref, (size_t)k_samples * 8);
    if (!rc) rc = dev_alloc(err, 8);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = KIFMM_ERR_CUDA;
    bool have_ref = false;
    int ibest = -1, imin = -1;
    std::vector<kifmm_tune_entry> tab(ncand);
    for (int64_t c = 0; c < ncand && !rc; ++c) {
        kifmm_tune_entry& E = tab[c];
        E.leaf = leaf[c / ((int64_t)norder * nr)];
        E.order = order[(c / nr) % norder];
        kifmm_opts oc = o;
        if (nradii > 0) {
            oc.radii[0] = radii[2 * (c % nr)];
            oc.radii[1] = radii[2 * (c % nr) + 1];
        }
        E.radii[0] = oc.radii[0];
        E.radii[1] = oc.radii[1];
        kifmm_plan_t p = nullptr;
        rc = kifmm_plan(&p, points, n, cell_h, uniform_h, E.leaf, E.order, a, b, &oc);
        if (rc) break;
        rc = kifmm_eval(p, I, Sb.p, KIFMM_F64, 1.0);
        Plan& P = *kifmm_plan_internal(p);
        if (!rc && !have_ref) {
            // targets drawn from this first evaluation, the FP64 direct sum there (the plan's
            // sorted points, weights and self terms; C = 1)
            rc = importance_targets(st, ptr<double>(Sb), n, k_samples, 0x5eedULL, ptr<int32_t>(P.tree.perm), P.tree.n, wsd.p,
                                    ptr<int32_t>(tc), ptr<int32_t>(ts), ptr<double>(wt), nsm);
            if (!rc && cudaMemsetAsync(acc.p, 0, (size_t)k_samples * 8, st) != cudaSuccess) rc = KIFMM_ERR_CUDA;
            if (!rc) {
                k_tune_ref<<<(unsigned)((P.tree.n + TR_CH - 1) / TR_CH), TR_T, 0, st>>>(   // (padding cells: q = 0)
                    ptr<double>(P.pts), ptr<double>(P.q), ptr<int32_t>(ts), k_samples, P.tree.n, make_kparams_kind(P.kind, a, b),
                    ptr<double>(acc));
                k_tune_ref_fin<<<(unsigned)((k_samples + 127) / 128), 128, 0, st>>>(
                    ptr<double>(acc), ptr<int32_t>(ts), k_samples, ptr<double>(P.sigma), ptr<double>(P.Isort),
                    ptr<double>(ref));
                if (cudaGetLastError() != cudaSuccess) rc = KIFMM_ERR_CUDA;
            }
            have_ref = !rc;
        }
        if (!rc) {
            k_tune_err<<<1, 256, 0, st>>>(ptr<double>(Sb), ptr<int32_t>(tc), ptr<double>(ref), ptr<double>(wt),
                                          k_samples, ptr<double>(err));
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(&E.err, err.p, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                rc = KIFMM_ERR_CUDA;
        }
        if (!rc) {   // timing: reps evaluations between two events
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && !rc; ++r) rc = kifmm_eval(p, I, Sb.p, KIFMM_F64, 1.0);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = KIFMM_ERR_CUDA;
            E.ms = ms / reps;
        }
        if (!rc) rc = kifmm_check(p);
        kifmm_destroy(p);
        if (rc) break;
        E.ok = E.err <= 0.5 * target ? 1 : 0;
        if (imin < 0 || E.err < tab[imin].err) imin = (int)c;
        if (E.ok && (ibest < 0 || E.ms < tab[ibest].ms)) ibest = (int)c;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (DevBuf* d : {&Sb, &wsd, &tc, &ts, &wt, &acc, &ref, &err}) dev_free(*d);
    if (rc) return rc;
    if (entries)
        for (int64_t c = 0; c < ncand; ++c) entries[c] = tab[c];
    *best = tab[ibest >= 0 ? ibest : imin];   // no candidate met the target: the most accurate (ok = 0)
    return KIFMM_OK;
}
