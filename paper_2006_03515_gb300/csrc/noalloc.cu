// kifmm_direct_noalloc: the photoionization sum by direct summation, without any
// device allocation.
//
// Some callers cannot call cudaMalloc at the moment they need S: code running while a
// CUDA graph is being captured on its stream (allocation would break or be illegal in the
// capture), real-time loops that forbid allocation after start-up, and processes whose
// device memory is fully reserved by another allocator. For them this entry point keeps
// its only work space, the cell weights q_j = I_j h^3 and the self-cell value, in one
// fixed array in device global memory that exists for as long as the library is loaded
// (on every GPU that loads it). The caller passes inputs and outputs as device pointers.
#include <cmath>
#include <mutex>

#include "internal.cuh"
#include "kernel.cuh"
#include "selfcell.cuh"

namespace kifmm {

// Work space: n weights followed by the self-cell value; every call writes it before
// reading it, so nothing needs clearing, but two calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_noalloc_scratch[KIFMM_NOALLOC_MAX_POINTS + 32];

// q_j = I_j h^3 into the work space, and sigma(h) (one block, 64-node Gauss-Legendre)
__global__ void k_na_prepare(const double* I, int64_t n, double h, double a, double b, int mode, double* ws) {
    __shared__ double gx[64], gw[64], red[256];
    const double w = h * h * h;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        ws[j] = I[j] * w;
    if (blockIdx.x == 0) {
        if (threadIdx.x < 64) gl_node(64, threadIdx.x, &gx[threadIdx.x], &gw[threadIdx.x]);
        __syncthreads();
        const double s = self_sigma_block(h, a, b, mode, 64, gx, gw, red);
        if (threadIdx.x == 0) ws[n] = s;
    }
}

// S_i = C * (sum_{j != i} K(|x_i - x_j|) q_j + sigma I_i), FP64, sources staged in shared memory.
constexpr int NA_T = 256;
__global__ void __launch_bounds__(NA_T) k_na_direct(const double* pts, const double* I, int64_t n, KParams kp,
                                                    double C, const double* ws, double* S) {
    __shared__ double sx[NA_T], sy[NA_T], sz[NA_T], sq[NA_T];
    const int64_t i = (int64_t)blockIdx.x * NA_T + threadIdx.x;
    const bool act = i < n;
    const double x = act ? pts[3 * i] : 0.0, y = act ? pts[3 * i + 1] : 0.0, z = act ? pts[3 * i + 2] : 0.0;
    double acc = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += NA_T) {
        const int64_t j = j0 + threadIdx.x;
        __syncthreads();
        if (j < n) {
            sx[threadIdx.x] = pts[3 * j];
            sy[threadIdx.x] = pts[3 * j + 1];
            sz[threadIdx.x] = pts[3 * j + 2];
            sq[threadIdx.x] = ws[j];
        }
        __syncthreads();
        const int m = (int)((n - j0) < NA_T ? (n - j0) : NA_T);
        if (act)
            for (int k = 0; k < m; ++k) {
                if (j0 + k == i) continue;
                const double dx = x - sx[k], dy = y - sy[k], dz = z - sz[k];
                acc += kern_f64(sqrt(dx * dx + dy * dy + dz * dz), kp) * sq[k];
            }
    }
    if (act) S[i] = C * (acc + ws[n] * I[i]);
}

// Device address of the work space, looked up once per device (with that device current).
static std::mutex g_na_mutex;
static double* g_na_addr[64] = {};

static int scratch_address(double** out) {
    int dev = 0;
    KF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("kifmm_direct_noalloc: device index out of range");
        return KIFMM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_error(std::string("kifmm_direct_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return KIFMM_ERR_CUDA;
        }
        g_na_addr[dev] = static_cast<double*>(p);
    }
    *out = g_na_addr[dev];
    return KIFMM_OK;
}

}  // namespace kifmm

using namespace kifmm;

extern "C" int kifmm_direct_noalloc(const double* points_dev, int64_t n, double h, const double* I_dev,
                                    double* S_dev, double a, double b, double C, int self_mode, void* stream) {
    set_error("");
    if (!points_dev || !I_dev || !S_dev || n < 1) {
        set_error("kifmm_direct_noalloc: need non-NULL pointers and n >= 1");
        return KIFMM_ERR_ARG;
    }
    if (n > KIFMM_NOALLOC_MAX_POINTS) {
        set_error("kifmm_direct_noalloc: n = " + std::to_string(n) + " exceeds the fixed work space of " +
                  std::to_string(KIFMM_NOALLOC_MAX_POINTS) + " points");
        return KIFMM_ERR_ARG;
    }
    if (!(h > 0.0) || !std::isfinite(h) || !(a > 0.0) || !(b > a) || !std::isfinite(b) || !std::isfinite(C)) {
        set_error("kifmm_direct_noalloc: need h > 0, 0 < a < b and finite C");
        return KIFMM_ERR_ARG;
    }
    if (self_mode != KIFMM_SELF_CELL_EXACT && self_mode != KIFMM_SELF_PAPER_GL2) {
        set_error("kifmm_direct_noalloc: unknown self_mode");
        return KIFMM_ERR_ARG;
    }
    double* ws = nullptr;
    KF_TRY(scratch_address(&ws));
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = (unsigned)((n + NA_T - 1) / NA_T);
    k_na_prepare<<<nb, 256, 0, st>>>(I_dev, n, h, a, b, self_mode, ws);
    KF_LAUNCH();
    k_na_direct<<<nb, NA_T, 0, st>>>(points_dev, I_dev, n, make_kparams(a, b), C, ws, S_dev);
    KF_LAUNCH();
    return KIFMM_OK;
}
