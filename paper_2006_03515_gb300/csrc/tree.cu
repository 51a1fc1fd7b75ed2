// Plan, part 1: root cube, Morton keys, stable radix sort, levelled octree and the
// U/V/W/X interaction lists (outline step 1 of Sec. 3; near/far split of Eq. (nearfar);
// adaptive lists of the kernel-independent FMM the paper builds on).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace kifmm {

// ------------------------------------------------------------------------------------
// generic helpers
// ------------------------------------------------------------------------------------
// Allocation-failure injection for the tests of the error paths: inside one kifmm_plan call,
// KIFMM_FAIL_ALLOC=k makes the k-th device allocation report an out-of-memory error.
static thread_local long g_alloc_count = 0, g_alloc_fail_at = 0;

AllocFaultScope::AllocFaultScope() {
    const char* f = std::getenv("KIFMM_FAIL_ALLOC");
    g_alloc_count = 0;
    g_alloc_fail_at = f ? std::max(0L, std::atol(f)) : 0;
}

AllocFaultScope::~AllocFaultScope() { g_alloc_fail_at = 0; }

int dev_alloc(DevBuf& b, size_t bytes) {
    dev_free(b);
    if (bytes == 0) bytes = 16;
    if (g_alloc_fail_at > 0 && ++g_alloc_count == g_alloc_fail_at) {
        set_error("device allocation " + std::to_string(g_alloc_fail_at) + " failed (injected)");
        return KIFMM_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? KIFMM_ERR_OOM : KIFMM_ERR_CUDA;
    }
    b.bytes = bytes;
    return KIFMM_OK;
}

void dev_free(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

static int grow(DevBuf& b, size_t bytes, cudaStream_t st) {
    if (b.bytes >= bytes) return KIFMM_OK;
    DevBuf nb;
    KF_TRY(dev_alloc(nb, bytes));
    if (b.p) {
        KF_CUDA(cudaMemcpyAsync(nb.p, b.p, b.bytes, cudaMemcpyDeviceToDevice, st));
        KF_CUDA(cudaStreamSynchronize(st));
    }
    dev_free(b);
    b = nb;
    return KIFMM_OK;
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
__device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}
__device__ __forceinline__ uint64_t morton3(int x, int y, int z) {
    return spread3((uint32_t)x) | (spread3((uint32_t)y) << 1) | (spread3((uint32_t)z) << 2);
}

// ------------------------------------------------------------------------------------
// exclusive scan of int32 (three kernels: block sums, scan of sums, block scans)
// ------------------------------------------------------------------------------------
constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_TILE = SCAN_T * SCAN_I;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* warp_tot, int32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;   // inclusive
    }
    __syncthreads();
    int32_t before = (warp > 0 ? warp_tot[warp - 1] : 0) + x - v;
    if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
    return before;
}

__global__ void scan_block_sums(const int32_t* in, int64_t n, int32_t* sums) {
    __shared__ int32_t wt[32];
    __shared__ int32_t tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k)
        if (base + k < n) s += in[base + k];
    block_excl_scan(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums_single(int32_t* sums, int64_t nb, int32_t* grand) {
    __shared__ int32_t wt[32];
    __shared__ int32_t tot;
    int32_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        int64_t i = b0 + threadIdx.x;
        int32_t v = i < nb ? sums[i] : 0;
        int32_t e = block_excl_scan(v, wt, &tot);
        __syncthreads();
        if (i < nb) sums[i] = e + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void scan_apply(const int32_t* in, int32_t* out, int64_t n, const int32_t* sums) {
    __shared__ int32_t wt[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int32_t v[SCAN_I];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int32_t e = block_excl_scan(s, wt, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        if (base + k < n) out[base + k] = e;
        e += v[k];
    }
}

int device_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_host,
                    cudaStream_t st, DevBuf& scratch) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb < 1) nb = 1;
    KF_TRY(grow(scratch, (size_t)(nb + 1) * sizeof(int32_t), st));
    int32_t* sums = ptr<int32_t>(scratch);
    scan_block_sums<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, sums);
    KF_LAUNCH();
    scan_sums_single<<<1, SCAN_T, 0, st>>>(sums, nb, sums + nb);
    KF_LAUNCH();
    scan_apply<<<(unsigned)nb, SCAN_T, 0, st>>>(in, out, n, sums);
    KF_LAUNCH();
    if (total_host) {
        KF_CUDA(cudaMemcpyAsync(total_host, sums + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        KF_CUDA(cudaStreamSynchronize(st));
    }
    return KIFMM_OK;
}

// ------------------------------------------------------------------------------------
// stable LSD radix sort of (u64 key, i32 value), 8 bits per pass
// ------------------------------------------------------------------------------------
constexpr int RS_T = 256, RS_R = 8, RS_TILE = RS_T * RS_R;

__global__ void rs_hist(const uint64_t* keys, int64_t n, int shift, int32_t* hist, int nblk) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int r = 0; r < RS_R; ++r) {
        int64_t i = base + r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

__global__ void rs_scatter(const uint64_t* kin, const int32_t* vin, uint64_t* kout, int32_t* vout,
                           int64_t n, int shift, const int32_t* offs, int nblk) {
    __shared__ int32_t base_off[256];
    __shared__ int32_t wcount[RS_T / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base_off[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_R; ++r) {
        int64_t i = base + r * RS_T + tid;
        bool valid = i < n;
        uint64_t k = valid ? kin[i] : 0ull;
        int32_t v = valid ? vin[i] : 0;
        int d = valid ? (int)((k >> shift) & 255u) : 256;
#pragma unroll
        for (int w = 0; w < RS_T / 32; ++w) wcount[w][tid] = 0;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        int64_t dst = 0;
        if (valid) {
            int pre = 0;
            for (int w = 0; w < warp; ++w) pre += wcount[w][d];
            dst = (int64_t)base_off[d] + pre + rank;
        }
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < RS_T / 32; ++w) tot += wcount[w][tid];
        base_off[tid] += tot;
        if (valid) {
            kout[dst] = k;
            vout[dst] = v;
        }
        __syncthreads();
    }
}

int radix_sort_pairs(uint64_t* keys, int32_t* vals, int64_t n, int key_bits, cudaStream_t st,
                     DevBuf& tk, DevBuf& tv, DevBuf& hist) {
    if (n <= 1) return KIFMM_OK;
    int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    KF_TRY(grow(tk, n * sizeof(uint64_t), st));
    KF_TRY(grow(tv, n * sizeof(int32_t), st));
    KF_TRY(grow(hist, (size_t)256 * nblk * 2 * sizeof(int32_t), st));
    DevBuf scan_tmp;
    uint64_t *ka = keys, *kb = ptr<uint64_t>(tk);
    int32_t *va = vals, *vb = ptr<int32_t>(tv);
    int32_t* h = ptr<int32_t>(hist);
    int32_t* ho = h + (size_t)256 * nblk;
    int passes = (key_bits + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
        int shift = 8 * ps;
        rs_hist<<<nblk, RS_T, 0, st>>>(ka, n, shift, h, nblk);
        KF_LAUNCH();
        int rc = device_scan_i32(h, ho, (int64_t)256 * nblk, nullptr, st, scan_tmp);
        if (rc != KIFMM_OK) { dev_free(scan_tmp); return rc; }
        rs_scatter<<<nblk, RS_T, 0, st>>>(ka, va, kb, vb, n, shift, ho, nblk);
        KF_LAUNCH();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        KF_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        KF_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    }
    KF_CUDA(cudaStreamSynchronize(st));
    dev_free(scan_tmp);
    return KIFMM_OK;
}

// ------------------------------------------------------------------------------------
// root cube and keys
// ------------------------------------------------------------------------------------
constexpr int RED_BLOCKS = 304, RED_T = 256;

// cell extents: h[i] per point (cubic cells), else ux, uy, uz for every point (one cube, or
// the rectangular cell of the plan)
__global__ void root_partial(const double* pts, const double* h, double ux, double uy, double uz, int64_t n,
                             double* part, int* bad) {
    __shared__ double s[6][RED_T];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int nonfinite = 0;
    const double ue[3] = {ux, uy, uz};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            const double hh = h ? h[i] : ue[k];
            if (!isfinite(hh) || !(hh > 0.0)) nonfinite = 1;
            double x = pts[3 * i + k];
            if (!isfinite(x)) nonfinite = 1;
            double half = __dmul_rn(0.5, hh);
            lo[k] = fmin(lo[k], __dsub_rn(x, half));
            hi[k] = fmax(hi[k], __dadd_rn(x, half));
        }
    }
    if (nonfinite) atomicExch(bad, 1);
    for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = lo[k];
        s[3 + k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int o = RED_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) {
                s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + o]);
                s[3 + k][threadIdx.x] = fmax(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void root_final(const double* part, int nb, double* root) {
    if (threadIdx.x != 0) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], part[6 * b + k]);
            hi[k] = fmax(hi[k], part[6 * b + 3 + k]);
        }
    double side = 0;
    for (int k = 0; k < 3; ++k) side = fmax(side, __dsub_rn(hi[k], lo[k]));
    root[0] = lo[0];
    root[1] = lo[1];
    root[2] = lo[2];
    root[3] = side;
    // extents, for the check that a given root contains every cell
    root[4] = hi[0];
    root[5] = hi[1];
    root[6] = hi[2];
}

__global__ void make_keys(const double* pts, int64_t n, const double* root, uint64_t* keys,
                          int32_t* idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double scale = __ddiv_rn((double)(1 << kKeyBits), root[3]);
    int c[3];
    for (int k = 0; k < 3; ++k) {
        double t = __dmul_rn(__dsub_rn(pts[3 * i + k], root[k]), scale);
        double f = floor(t);
        f = fmin(fmax(f, 0.0), (double)((1 << kKeyBits) - 1));
        c[k] = (int)f;
    }
    keys[i] = morton3(c[0], c[1], c[2]);
    idx[i] = (int32_t)i;
}

__global__ void check_duplicates(const uint64_t* keys, const int32_t* perm, const double* pts,
                                 int64_t n, int* dup) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i + 1 >= n) return;
    if (keys[i] != keys[i + 1]) return;
    const double* p = pts + 3 * (int64_t)perm[i];
    for (int64_t j = i + 1; j < n && keys[j] == keys[i]; ++j) {
        const double* q = pts + 3 * (int64_t)perm[j];
        if (p[0] == q[0] && p[1] == q[1] && p[2] == q[2]) atomicExch(dup, 1);
    }
}

// ------------------------------------------------------------------------------------
// levelled tree
// ------------------------------------------------------------------------------------
__global__ void tb_flags(const uint64_t* keys, const int32_t* active, int64_t n, int lev,
                         int32_t* flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = active[i];
    int f = 0;
    if (a >= 0) {
        int sh = 3 * (kKeyBits - lev - 1);
        if (i == 0 || active[i - 1] != a || (keys[i] >> sh) != (keys[i - 1] >> sh)) f = 1;
    }
    flag[i] = f;
}

__global__ void tb_children(const uint64_t* keys, const int32_t* active, const int32_t* flag,
                            const int32_t* cidx, int64_t n, int lev, int base, int32_t* level,
                            int32_t* anchor, uint64_t* mcode, int32_t* parent, int32_t* child,
                            int32_t* pstart, int32_t* leaf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    int c = base + cidx[i];
    int P = active[i];
    int cl = lev + 1;
    uint64_t code = keys[i] >> (3 * (kKeyBits - cl));
    level[c] = cl;
    mcode[c] = code;
    anchor[3 * c + 0] = (int)compact3(code);
    anchor[3 * c + 1] = (int)compact3(code >> 1);
    anchor[3 * c + 2] = (int)compact3(code >> 2);
    parent[c] = P;
    pstart[c] = (int32_t)i;
    leaf[c] = 1;
    for (int o = 0; o < 8; ++o) child[8 * (int64_t)c + o] = -1;
    leaf[P] = 0;
    child[8 * (int64_t)P + (int)(code & 7u)] = c;
}

__global__ void tb_pend(int base, int cnt, const int32_t* parent, const int32_t* pstart, int32_t* pend) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    int c = base + k;
    int P = parent[c];
    pend[c] = (k + 1 < cnt && parent[c + 1] == P) ? pstart[c + 1] : pend[P];
}

__global__ void tb_active(const int32_t* flag, const int32_t* cidx, int64_t n, int base, int lev,
                          int leaf_size, const int32_t* pstart, const int32_t* pend, int32_t* active) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || active[i] < 0) return;
    int c = base + cidx[i] + flag[i] - 1;
    int cnt = pend[c] - pstart[c];
    active[i] = (cnt > leaf_size && lev + 1 < kMaxLevel) ? c : -1;
}

__global__ void tb_root(int32_t* level, int32_t* anchor, uint64_t* mcode, int32_t* parent,
                        int32_t* child, int32_t* pstart, int32_t* pend, int32_t* leaf, int n) {
    level[0] = 0;
    anchor[0] = anchor[1] = anchor[2] = 0;
    mcode[0] = 0;
    parent[0] = -1;
    for (int o = 0; o < 8; ++o) child[o] = -1;
    pstart[0] = 0;
    pend[0] = n;
    leaf[0] = 1;
}

__global__ void tb_fill_i32(int32_t* a, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void tb_centres(const int32_t* level, const int32_t* anchor, int64_t nb, double ox,
                           double oy, double oz, double side, double* centre) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double r = side / (double)(2ll << level[b]);   // exact: division by a power of two
    double o[3] = {ox, oy, oz};
    for (int k = 0; k < 3; ++k)
        centre[3 * b + k] = __dadd_rn(o[k], __dmul_rn(2.0 * anchor[3 * b + k] + 1.0, r));
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- zero-weight padding of a box grid to the leaf lattice ------------------------------------
// every point must be a cell centre lo + (i + 1/2) h with 0 <= i_k < n_k (within 1e-6 cells)
__global__ void k_lattice_member(const double* pts, int64_t n, double lx, double ly, double lz, double h, int64_t nx,
                                 int64_t ny, int64_t nz, int* bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double lo[3] = {lx, ly, lz};
    const int64_t ext[3] = {nx, ny, nz};
    for (int k = 0; k < 3; ++k) {
        const double u = (pts[3 * i + k] - lo[k]) / h - 0.5;
        const double ur = rint(u);
        if (!(fabs(u - ur) <= 1e-6) || ur < 0.0 || ur >= (double)ext[k]) atomicExch(bad, 1);
    }
}

int pad_to_lattice(cudaStream_t st, const double* pts, int64_t n, double h, int nc, DevBuf& out, int64_t* n_total,
                   double root[4]) {
    *n_total = n;
    root[3] = 0.0;   // (no lattice root unless the points are a full box grid)
    DevBuf part, rootb, flags;
    auto release = [&]() {
        for (DevBuf* d : {&part, &rootb, &flags}) dev_free(*d);
    };
    // the body returns through the error macros; the work buffers are released on every path
    auto body = [&]() -> int {
        KF_TRY(dev_alloc(part, RED_BLOCKS * 6 * sizeof(double)));
        KF_TRY(dev_alloc(rootb, 8 * sizeof(double)));
        KF_TRY(dev_alloc(flags, 4 * sizeof(int)));
        KF_CUDA(cudaMemsetAsync(flags.p, 0, 4 * sizeof(int), st));
        root_partial<<<RED_BLOCKS, RED_T, 0, st>>>(pts, nullptr, h, h, h, n, ptr<double>(part), ptr<int>(flags));
        KF_LAUNCH();
        root_final<<<1, 32, 0, st>>>(ptr<double>(part), RED_BLOCKS, ptr<double>(rootb));
        KF_LAUNCH();
        double r8[8];
        int hflags[4];
        KF_CUDA(cudaMemcpyAsync(r8, rootb.p, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
        KF_CUDA(cudaMemcpyAsync(hflags, flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        KF_CUDA(cudaStreamSynchronize(st));
        if (hflags[0]) {   // non-finite input: the tree build reports it
            return KIFMM_OK;
        }
        int64_t ext[3], pad[3];
        double prod = 1.0;
        for (int k = 0; k < 3; ++k) {
            const double e = (r8[4 + k] - r8[k]) / h;
            ext[k] = (int64_t)std::llround(e);
            if (!(std::fabs(e - (double)ext[k]) <= 1e-6 * std::max(1.0, e)) || ext[k] < 1) {
                return KIFMM_OK;
            }
            prod *= (double)ext[k];
            pad[k] = (ext[k] + 2 * nc - 1) / (2 * nc) * (2 * nc);
        }
        if (prod != (double)n) {   // not every cell of the box: no padding
            return KIFMM_OK;
        }
        k_lattice_member<<<nblk(n, 256), 256, 0, st>>>(pts, n, r8[0], r8[1], r8[2], h, ext[0], ext[1], ext[2],
                                                        ptr<int>(flags) + 1);
        KF_LAUNCH();
        KF_CUDA(cudaMemcpyAsync(hflags, flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        KF_CUDA(cudaStreamSynchronize(st));
        if (hflags[1]) return KIFMM_OK;
        // the root: origin at the grid's corner, side nc h 2^L >= every padded extent
        int64_t cells = nc;
        while (cells < std::max(pad[0], std::max(pad[1], pad[2]))) cells *= 2;
        root[0] = r8[0];
        root[1] = r8[1];
        root[2] = r8[2];
        root[3] = (double)cells * h;
        const int64_t nt = pad[0] * pad[1] * pad[2];
        if (nt >= (int64_t)1 << 31) {
            root[3] = 0.0;
            return KIFMM_OK;
        }
        const int64_t nv = nt - n;
        if (nv == 0) return KIFMM_OK;   // already on the lattice: the root alone
        KF_TRY(dev_alloc(out, (size_t)nt * 3 * sizeof(double)));
        KF_CUDA(cudaMemcpyAsync(out.p, pts, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (nv > 0) {   // the padding cells in z, y, x order, after the caller's points
            std::vector<double> v;
            v.reserve((size_t)nv * 3);
            for (int64_t z = 0; z < pad[2]; ++z)
                for (int64_t y = 0; y < pad[1]; ++y)
                    for (int64_t x = 0; x < pad[0]; ++x) {
                        if (x < ext[0] && y < ext[1] && z < ext[2]) continue;
                        v.push_back(r8[0] + ((double)x + 0.5) * h);
                        v.push_back(r8[1] + ((double)y + 0.5) * h);
                        v.push_back(r8[2] + ((double)z + 0.5) * h);
                    }
            KF_CUDA(cudaMemcpyAsync(static_cast<double*>(out.p) + 3 * n, v.data(), v.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, st));
            KF_CUDA(cudaStreamSynchronize(st));   // v is released on return
        }
        *n_total = nt;
        return KIFMM_OK;
    };
    const int rc = body();
    release();
    return rc;
}

int build_tree(Plan& p, const double* pts, const double* h, double uh, const kifmm_opts& o) {
    Tree& t = p.tree;
    cudaStream_t st = p.stream;
    const int64_t n = t.n;
    // ---- root cube
    DevBuf part, rootb, flags;
    KF_TRY(dev_alloc(part, RED_BLOCKS * 6 * sizeof(double)));
    KF_TRY(dev_alloc(rootb, 8 * sizeof(double)));
    KF_TRY(dev_alloc(flags, 4 * sizeof(int)));
    KF_CUDA(cudaMemsetAsync(flags.p, 0, 4 * sizeof(int), st));
    const double ux = p.rect ? p.cell_dims[0] : uh, uy = p.rect ? p.cell_dims[1] : uh, uz = p.rect ? p.cell_dims[2] : uh;
    root_partial<<<RED_BLOCKS, RED_T, 0, st>>>(pts, h, ux, uy, uz, n, ptr<double>(part), ptr<int>(flags));
    KF_LAUNCH();
    root_final<<<1, 32, 0, st>>>(ptr<double>(part), RED_BLOCKS, ptr<double>(rootb));
    KF_LAUNCH();
    double root[8];
    int hflags[4];
    KF_CUDA(cudaMemcpyAsync(root, rootb.p, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaMemcpyAsync(hflags, flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    if (hflags[0]) {
        set_error("kifmm_plan: non-finite coordinate or cell size <= 0");
        return KIFMM_ERR_NONFINITE;
    }
    if (o.has_root) {
        for (int k = 0; k < 3; ++k)
            if (!(root[k] >= o.root[k]) || !(root[4 + k] <= o.root[k] + o.root[3])) {
                set_error("kifmm_plan: a cell lies outside the given root cube");
                return KIFMM_ERR_ARG;
            }
        for (int k = 0; k < 4; ++k) root[k] = o.root[k];
        KF_CUDA(cudaMemcpyAsync(rootb.p, root, 4 * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    if (!(root[3] > 0.0)) {
        set_error("kifmm_plan: degenerate root cube (side 0)");
        return KIFMM_ERR_ARG;
    }
    for (int k = 0; k < 3; ++k) t.origin[k] = root[k];
    t.side = root[3];

    // ---- keys and sort
    KF_TRY(dev_alloc(t.keys, n * sizeof(uint64_t)));
    KF_TRY(dev_alloc(t.perm, n * sizeof(int32_t)));
    make_keys<<<nblk(n, 256), 256, 0, st>>>(pts, n, ptr<double>(rootb), ptr<uint64_t>(t.keys),
                                            ptr<int32_t>(t.perm));
    KF_LAUNCH();
    {
        DevBuf tk, tv, hist;
        int rc = radix_sort_pairs(ptr<uint64_t>(t.keys), ptr<int32_t>(t.perm), n, 3 * kKeyBits, st,
                                  tk, tv, hist);
        dev_free(tk); dev_free(tv); dev_free(hist);
        KF_TRY(rc);
    }
    check_duplicates<<<nblk(n, 256), 256, 0, st>>>(ptr<uint64_t>(t.keys), ptr<int32_t>(t.perm), pts,
                                                    n, ptr<int>(flags) + 1);
    KF_LAUNCH();
    KF_CUDA(cudaMemcpyAsync(hflags, flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    if (hflags[1]) {
        set_error("kifmm_plan: two points have identical coordinates");
        return KIFMM_ERR_DUPLICATE_POINT;
    }

    // ---- levelled tree
    int64_t cap = std::max<int64_t>(1024, 4 * (n / std::max(1, p.leaf_size)) + 64);
    auto alloc_boxes = [&](int64_t c) -> int {
        KF_TRY(grow(t.level, c * 4, st));
        KF_TRY(grow(t.anchor, c * 12, st));
        KF_TRY(grow(t.mcode, c * 8, st));
        KF_TRY(grow(t.parent, c * 4, st));
        KF_TRY(grow(t.child, c * 32, st));
        KF_TRY(grow(t.pstart, c * 4, st));
        KF_TRY(grow(t.pend, c * 4, st));
        KF_TRY(grow(t.leaf, c * 4, st));
        return KIFMM_OK;
    };
    KF_TRY(alloc_boxes(cap));
    tb_root<<<1, 1, 0, st>>>(ptr<int32_t>(t.level), ptr<int32_t>(t.anchor), ptr<uint64_t>(t.mcode),
                             ptr<int32_t>(t.parent), ptr<int32_t>(t.child), ptr<int32_t>(t.pstart),
                             ptr<int32_t>(t.pend), ptr<int32_t>(t.leaf), (int)n);
    KF_LAUNCH();
    DevBuf active, flag, cidx, scan_tmp;
    KF_TRY(dev_alloc(active, n * 4));
    KF_TRY(dev_alloc(flag, n * 4));
    KF_TRY(dev_alloc(cidx, n * 4));
    tb_fill_i32<<<nblk(n, 256), 256, 0, st>>>(ptr<int32_t>(active), n, n > p.leaf_size ? 0 : -1);
    KF_LAUNCH();
    t.level_start.assign(1, 0);
    int64_t base = 1;
    int lev = 0;
    while (true) {
        t.level_start.push_back(base);   // start of level lev + 1
        if (lev >= kMaxLevel) break;
        tb_flags<<<nblk(n, 256), 256, 0, st>>>(ptr<uint64_t>(t.keys), ptr<int32_t>(active), n, lev,
                                               ptr<int32_t>(flag));
        KF_LAUNCH();
        int32_t cnt = 0;
        KF_TRY(device_scan_i32(ptr<int32_t>(flag), ptr<int32_t>(cidx), n, &cnt, st, scan_tmp));
        if (cnt == 0) break;
        if (base + cnt > cap) {
            cap = std::max<int64_t>(2 * cap, base + cnt + 1024);
            KF_TRY(alloc_boxes(cap));
        }
        tb_children<<<nblk(n, 256), 256, 0, st>>>(
            ptr<uint64_t>(t.keys), ptr<int32_t>(active), ptr<int32_t>(flag), ptr<int32_t>(cidx), n,
            lev, (int)base, ptr<int32_t>(t.level), ptr<int32_t>(t.anchor), ptr<uint64_t>(t.mcode),
            ptr<int32_t>(t.parent), ptr<int32_t>(t.child), ptr<int32_t>(t.pstart), ptr<int32_t>(t.leaf));
        KF_LAUNCH();
        tb_pend<<<nblk(cnt, 256), 256, 0, st>>>((int)base, cnt, ptr<int32_t>(t.parent),
                                                ptr<int32_t>(t.pstart), ptr<int32_t>(t.pend));
        KF_LAUNCH();
        tb_active<<<nblk(n, 256), 256, 0, st>>>(ptr<int32_t>(flag), ptr<int32_t>(cidx), n, (int)base,
                                                lev, p.leaf_size, ptr<int32_t>(t.pstart),
                                                ptr<int32_t>(t.pend), ptr<int32_t>(active));
        KF_LAUNCH();
        base += cnt;
        ++lev;
    }
    // level_start has one entry per level plus the sentinel; drop a trailing empty level
    while (t.level_start.size() >= 2 &&
           t.level_start[t.level_start.size() - 1] == t.level_start[t.level_start.size() - 2])
        t.level_start.pop_back();
    t.nboxes = base;
    t.nlevels = (int)t.level_start.size() - 1;
    KF_TRY(dev_alloc(t.centre, t.nboxes * 3 * sizeof(double)));
    tb_centres<<<nblk(t.nboxes, 256), 256, 0, st>>>(ptr<int32_t>(t.level), ptr<int32_t>(t.anchor),
                                                    t.nboxes, t.origin[0], t.origin[1], t.origin[2],
                                                    t.side, ptr<double>(t.centre));
    KF_LAUNCH();
    KF_CUDA(cudaStreamSynchronize(st));
    dev_free(active); dev_free(flag); dev_free(cidx); dev_free(scan_tmp);
    dev_free(part); dev_free(rootb); dev_free(flags);
    return KIFMM_OK;
}

// ------------------------------------------------------------------------------------
// interaction lists
// ------------------------------------------------------------------------------------
struct TreeView {
    const int32_t* level;
    const int32_t* anchor;
    const uint64_t* mcode;
    const int32_t* parent;
    const int32_t* child;
    const int32_t* leaf;
    int64_t ls[kMaxLevel + 3];
    int nlevels;
};

__device__ int lookup(const TreeView& T, int lev, int x, int y, int z) {
    if (lev < 0 || lev >= T.nlevels) return -1;
    int lim = 1 << lev;
    if (x < 0 || y < 0 || z < 0 || x >= lim || y >= lim || z >= lim) return -1;
    uint64_t code = morton3(x, y, z);
    int64_t lo = T.ls[lev], hi = T.ls[lev + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (T.mcode[mid] < code) lo = mid + 1;
        else hi = mid;
    }
    if (lo < T.ls[lev + 1] && T.mcode[lo] == code) return (int)lo;
    return -1;
}

__device__ bool adjacent(const TreeView& T, int a, int b) {
    int la = T.level[a], lb = T.level[b];
    int L = la > lb ? la : lb;
    int sa = 1 << (L - la), sb = 1 << (L - lb);
    for (int k = 0; k < 3; ++k) {
        int loa = T.anchor[3 * a + k] * sa, lob = T.anchor[3 * b + k] * sb;
        if (loa > lob + sb || lob > loa + sa) return false;
    }
    return true;
}

__device__ void sort_range(int32_t* a, int n) {
    for (int i = 1; i < n; ++i) {
        int32_t v = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > v) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = v;
    }
}

constexpr int STACK = 200;

// U(B) for leaves: B and all leaves adjacent to it.
__global__ void list_u(TreeView T, int64_t nb, const int32_t* off, int32_t* cnt, int32_t* items,
                       int* overflow) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || !T.leaf[b]) {
        if (b < nb && cnt) cnt[b] = 0;
        return;
    }
    int lev = T.level[b];
    int ax = T.anchor[3 * b], ay = T.anchor[3 * b + 1], az = T.anchor[3 * b + 2];
    int n = 0;
    int coarse[27];
    int nc = 0;
    int stack[STACK];
    int32_t* out = items ? items + off[b] : nullptr;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int cx = ax + dx, cy = ay + dy, cz = az + dz;
                int lim = 1 << lev;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= lim || cy >= lim || cz >= lim) continue;
                int c = lookup(T, lev, cx, cy, cz);
                if (c >= 0) {
                    int sp = 0;
                    stack[sp++] = c;
                    while (sp > 0) {
                        int d = stack[--sp];
                        if (T.leaf[d]) {
                            if (adjacent(T, d, (int)b)) {
                                if (out) out[n] = d;
                                ++n;
                            }
                        } else {
                            for (int o = 0; o < 8; ++o) {
                                int k = T.child[8 * (int64_t)d + o];
                                if (k >= 0 && adjacent(T, k, (int)b)) {
                                    if (sp < STACK) stack[sp++] = k;
                                    else atomicExch(overflow, 1);
                                }
                            }
                        }
                    }
                } else {
                    for (int up = 1; up <= lev; ++up) {
                        int c2 = lookup(T, lev - up, cx >> up, cy >> up, cz >> up);
                        if (c2 >= 0) {
                            if (T.leaf[c2]) {
                                bool seen = false;
                                for (int s = 0; s < nc; ++s) seen |= (coarse[s] == c2);
                                if (!seen) {
                                    coarse[nc++] = c2;
                                    if (out) out[n] = c2;
                                    ++n;
                                }
                            }
                            break;
                        }
                    }
                }
            }
    if (cnt) cnt[b] = n;
    if (out) sort_range(out, n);
}

__device__ __forceinline__ int offset_slot(int dx, int dy, int dz) {
    return (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
}

// V(B): children of the parent's colleagues that are not adjacent to B.
__global__ void list_v(TreeView T, int64_t nb, const int32_t* off, int32_t* cnt, int32_t* items,
                       int32_t* vtab) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int P = T.parent[b];
    if (P < 0) {
        if (cnt) cnt[b] = 0;
        return;
    }
    int lp = T.level[P];
    int px = T.anchor[3 * P], py = T.anchor[3 * P + 1], pz = T.anchor[3 * P + 2];
    int bx = T.anchor[3 * b], by = T.anchor[3 * b + 1], bz = T.anchor[3 * b + 2];
    int n = 0;
    int32_t* out = items ? items + off[b] : nullptr;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int c = lookup(T, lp, px + dx, py + dy, pz + dz);
                if (c < 0) continue;
                for (int o = 0; o < 8; ++o) {
                    int k = T.child[8 * (int64_t)c + o];
                    if (k < 0 || adjacent(T, k, (int)b)) continue;
                    if (out) {
                        out[n] = k;
                        if (vtab)
                            vtab[b * kOffsetSlots + offset_slot(T.anchor[3 * k] - bx, T.anchor[3 * k + 1] - by,
                                                                T.anchor[3 * k + 2] - bz)] = k;
                    }
                    ++n;
                }
            }
    if (cnt) cnt[b] = n;
    if (out) sort_range(out, n);
}

// W(B) for leaves: descendants of B's colleagues, not adjacent to B, with a parent adjacent to B.
__global__ void list_w(TreeView T, int64_t nb, const int32_t* off, int32_t* cnt, int32_t* items,
                       int* overflow) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || !T.leaf[b]) {
        if (b < nb && cnt) cnt[b] = 0;
        return;
    }
    int lev = T.level[b];
    int ax = T.anchor[3 * b], ay = T.anchor[3 * b + 1], az = T.anchor[3 * b + 2];
    int n = 0;
    int stack[STACK];
    int32_t* out = items ? items + off[b] : nullptr;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                int c = lookup(T, lev, ax + dx, ay + dy, az + dz);
                if (c < 0 || T.leaf[c]) continue;
                int sp = 0;
                stack[sp++] = c;
                while (sp > 0) {
                    int d = stack[--sp];
                    for (int o = 0; o < 8; ++o) {
                        int k = T.child[8 * (int64_t)d + o];
                        if (k < 0) continue;
                        if (!adjacent(T, k, (int)b)) {
                            if (out) out[n] = k;
                            ++n;
                        } else if (!T.leaf[k]) {
                            if (sp < STACK) stack[sp++] = k;
                            else atomicExch(overflow, 1);
                        }
                    }
                }
            }
    if (cnt) cnt[b] = n;
    if (out) sort_range(out, n);
}

// X(A) = {B : A in W(B)}: counted and filled from the W lists.
__global__ void list_x_count(const int32_t* woff, const int32_t* witems, int64_t nb, int32_t* xcnt) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    for (int k = woff[b]; k < woff[b + 1]; ++k) atomicAdd(&xcnt[witems[k]], 1);
}
__global__ void list_x_fill(const int32_t* woff, const int32_t* witems, int64_t nb, const int32_t* xoff,
                            int32_t* xpos, int32_t* xitems) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    for (int k = woff[b]; k < woff[b + 1]; ++k) {
        int a = witems[k];
        int s = atomicAdd(&xpos[a], 1);
        xitems[xoff[a] + s] = (int32_t)b;
    }
}
__global__ void list_sort_each(const int32_t* off, int32_t* items, int64_t nb) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    sort_range(items + off[b], off[b + 1] - off[b]);
}

int build_lists(Plan& p) {
    Tree& t = p.tree;
    cudaStream_t st = p.stream;
    const int64_t nb = t.nboxes;
    TreeView T;
    T.level = ptr<int32_t>(t.level);
    T.anchor = ptr<int32_t>(t.anchor);
    T.mcode = ptr<uint64_t>(t.mcode);
    T.parent = ptr<int32_t>(t.parent);
    T.child = ptr<int32_t>(t.child);
    T.leaf = ptr<int32_t>(t.leaf);
    T.nlevels = t.nlevels;
    for (int l = 0; l <= kMaxLevel + 2; ++l)
        T.ls[l] = l <= t.nlevels ? t.level_start[l] : t.level_start[t.nlevels];
    DevBuf cnt, scan_tmp, ovf;
    KF_TRY(dev_alloc(cnt, (nb + 1) * 4));
    KF_TRY(dev_alloc(ovf, 4));
    KF_CUDA(cudaMemsetAsync(ovf.p, 0, 4, st));
    KF_TRY(dev_alloc(p.vtab, (size_t)nb * kOffsetSlots * 4));
    KF_CUDA(cudaMemsetAsync(p.vtab.p, 0xff, (size_t)nb * kOffsetSlots * 4, st));
    const unsigned g = nblk(nb, 128);
    for (int which = 0; which < 3; ++which) {
        Csr& L = p.lists[which == 0 ? 0 : (which == 1 ? 1 : 2)];
        KF_TRY(dev_alloc(L.off, (nb + 1) * 4));
        // count
        if (which == 0) list_u<<<g, 128, 0, st>>>(T, nb, nullptr, ptr<int32_t>(cnt), nullptr, ptr<int>(ovf));
        if (which == 1) list_v<<<g, 128, 0, st>>>(T, nb, nullptr, ptr<int32_t>(cnt), nullptr, nullptr);
        if (which == 2) list_w<<<g, 128, 0, st>>>(T, nb, nullptr, ptr<int32_t>(cnt), nullptr, ptr<int>(ovf));
        KF_LAUNCH();
        KF_CUDA(cudaMemsetAsync(ptr<int32_t>(cnt) + nb, 0, 4, st));
        int32_t total = 0;
        KF_TRY(device_scan_i32(ptr<int32_t>(cnt), ptr<int32_t>(L.off), nb + 1, &total, st, scan_tmp));
        L.len = total;
        KF_TRY(dev_alloc(L.items, (size_t)std::max<int64_t>(total, 1) * 4));
        if (which == 0) list_u<<<g, 128, 0, st>>>(T, nb, ptr<int32_t>(L.off), nullptr, ptr<int32_t>(L.items), ptr<int>(ovf));
        if (which == 1) list_v<<<g, 128, 0, st>>>(T, nb, ptr<int32_t>(L.off), nullptr, ptr<int32_t>(L.items), ptr<int32_t>(p.vtab));
        if (which == 2) list_w<<<g, 128, 0, st>>>(T, nb, ptr<int32_t>(L.off), nullptr, ptr<int32_t>(L.items), ptr<int>(ovf));
        KF_LAUNCH();
    }
    // X from W
    {
        Csr& W = p.lists[2];
        Csr& X = p.lists[3];
        KF_CUDA(cudaMemsetAsync(cnt.p, 0, (nb + 1) * 4, st));
        list_x_count<<<g, 128, 0, st>>>(ptr<int32_t>(W.off), ptr<int32_t>(W.items), nb, ptr<int32_t>(cnt));
        KF_LAUNCH();
        KF_TRY(dev_alloc(X.off, (nb + 1) * 4));
        int32_t total = 0;
        KF_TRY(device_scan_i32(ptr<int32_t>(cnt), ptr<int32_t>(X.off), nb + 1, &total, st, scan_tmp));
        X.len = total;
        KF_TRY(dev_alloc(X.items, (size_t)std::max<int64_t>(total, 1) * 4));
        KF_CUDA(cudaMemsetAsync(cnt.p, 0, (nb + 1) * 4, st));
        list_x_fill<<<g, 128, 0, st>>>(ptr<int32_t>(W.off), ptr<int32_t>(W.items), nb, ptr<int32_t>(X.off),
                                       ptr<int32_t>(cnt), ptr<int32_t>(X.items));
        KF_LAUNCH();
        list_sort_each<<<g, 128, 0, st>>>(ptr<int32_t>(X.off), ptr<int32_t>(X.items), nb);
        KF_LAUNCH();
    }
    int hovf = 0;
    KF_CUDA(cudaMemcpyAsync(&hovf, ovf.p, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    dev_free(cnt); dev_free(scan_tmp); dev_free(ovf);
    if (hovf) {
        set_error("kifmm_plan: list traversal stack overflow");
        return KIFMM_ERR_ARG;
    }
    return KIFMM_OK;
}

}  // namespace kifmm
