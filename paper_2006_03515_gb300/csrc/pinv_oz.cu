// Upward pseudo-inverse application c = Sigma^+ U^T chk (UC2UE, Eqs. (s2m), (m2m)) to FP64
// accuracy on the tensor cores, by exact integer slicing (the scheme of Ozaki et al. for
// error-free matrix products):
//
//   chk_b = 2^{e_b} sum_{i=1..9} a_i 2^{-6i},   G1_r = 2^{e_r} sum_{j=1..9} g_j 2^{-6j},
//
// per box b and per operator row r, with integer slices |a_i|, |g_j| <= 64 held exactly in
// FP16. Each slice product a_i . g_j (K <= 192 terms of magnitude <= 2^12) is an integer
// below 2^20; the products of one level L = i + j (at most 9 of them) sum below 2^23, so the
// tensor core's FP32 accumulation of a level is exact. Levels L <= 10 are kept (the dropped
// terms are below 2^-54 of the largest products), and the epilogue combines the 9 level sums
// in FP64:  c[b][r] = 2^{e_b + e_r} sum_L 2^{-6L} P_L[b][r].
// The result equals the FP64 product to the rounding of an FP64 GEMM.
//
// One CTA takes 48 operator rows (MMA N) and, persistently, the box tiles of 128 boxes (MMA M)
// bt, bt + gridDim.x, ... (one wave of CTAs): it keeps all 9 operator slices of its rows in
// shared memory (loaded once), streams the 9 box slices of each tile chunk by chunk (K-chunks
// of 64 FP16, 128-byte swizzled images written by the slicing kernel) through a ring of
// stages, and for box slice i issues the MMAs against operator slices j = 1..10-i into the
// accumulator of level i + j (9 accumulators of 48 columns in tensor memory). Roles: warp 8
// lane 0 moves the images with bulk copies, warp 9 lane 0 issues the MMAs, warps 0-7 drain
// the accumulators and hand them back (a "drained" barrier) before the next tile's MMAs.
// Every wait is bounded; a timeout raises the abort flag and an error code.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace kifmm {

constexpr int OZ_S = 9;          // slices per operand
constexpr int OZ_W = 6;          // bits per slice
constexpr int OZ_N = 48;         // operator rows per CTA (MMA N)
constexpr int OZ_M = 128;        // boxes per CTA (MMA M)
constexpr int OZ_KC = 64;        // FP16 per K-chunk (one 128-byte swizzle row)
constexpr int OZ_NS = 3;         // box-slice stages (eight for K of one chunk measured no faster)
__host__ __device__ constexpr int oz_stages(int nk) { return OZ_NS + 0 * nk; }
constexpr int OZ_THREADS = 320;  // warps 0-7 epilogue, 8 producer, 9 MMA

__host__ __device__ inline int oz_kp(int S) { return (S + 31) / 32 * 32; }   // K padded to a multiple of 32
__host__ __device__ inline int oz_nk(int S) { return (oz_kp(S) + OZ_KC - 1) / OZ_KC; }
static inline size_t oz_b_bytes(int S) { return (size_t)OZ_S * oz_nk(S) * OZ_N * 128; }   // per row tile
static inline size_t oz_smem(int S) { return 1024 + oz_b_bytes(S) + (size_t)oz_stages(oz_nk(S)) * OZ_M * 128; }

int pinv_oz_supported(int S) { return oz_smem(S) <= 227 * 1024 ? 1 : 0; }

// Slices of one row v[0..S) written as FP16 integers into the swizzled image
// img + slice * slice_stride + (k / 64) * chunk_stride + sw128(row, k % 64), in integer
// arithmetic only (FP64 throughput is scarce): each value becomes the 54-bit fixed-point
// integer X = round(v 2^{54 - e}) (|X| < 2^54), split into balanced base-64 digits
// X = sum_i a_i 64^{9-i}, rounding each digit to nearest (|a_1| <= 64, |a_i| <= 32 after).
__device__ __forceinline__ void oz_slice_row(const double* v, int S, int KP, int e, __half* img,
                                             int64_t slice_stride, int64_t chunk_stride, int row, int lane) {
    for (int k = lane; k < KP; k += 32) {
        long long X = 0;
        if (k < S) {
            const long long bits = __double_as_longlong(v[k]);
            const int ex = (int)((bits >> 52) & 0x7FF);
            if (ex != 0) {   // zero and subnormal values (below 2^-1022) count as zero
                const long long m = (bits & ((1LL << 52) - 1)) | (1LL << 52);
                const int sh = ex - 1021 - e;   // X = m 2^sh
                if (sh >= 0) X = m << sh;
                else if (sh > -64) X = (m + (1LL << (-sh - 1))) >> (-sh);
                if (bits < 0) X = -X;
            }
        }
        const int64_t base = (int64_t)(k / OZ_KC) * chunk_stride;
        const uint32_t off = sw128_off_h(row, k % OZ_KC) / 2;
#pragma unroll
        for (int i = 0; i < OZ_S; ++i) {
            const int s = OZ_W * (OZ_S - 1 - i);   // 48, 42, ..., 0
            const long long a = s > 0 ? (X + (1LL << (s - 1))) >> s : X;
            X -= a << s;
            img[(int64_t)i * slice_stride + base + off] = __int2half_rn((int)a);
        }
    }
}

// power-of-two exponent of a row's largest magnitude: |v| 2^-e < 1 (0 for a zero row),
// from the exponent fields alone
__device__ __forceinline__ int oz_row_exp(const double* v, int S, int lane) {
    int mx = 0;
    for (int k = lane; k < S; k += 32) mx = max(mx, (int)((__double_as_longlong(v[k]) >> 52) & 0x7FF));
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    return mx ? mx - 1022 : 0;   // |v| < 2^(mx - 1022)
}

// operator image: [row tile][slice][K-chunk][48 rows][128-byte row]; one warp per row
__global__ void k_oz_slice_op(const double* G1, int S, int rank, int ntile, __half* img, int* er) {
    const int r = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= ntile * OZ_N) return;
    const int KP = oz_kp(S), NK = oz_nk(S);
    const int tile = r / OZ_N, row = r % OZ_N;
    const int64_t chunk_stride = (int64_t)OZ_N * 64, slice_stride = (int64_t)NK * chunk_stride;
    __half* base = img + (int64_t)tile * OZ_S * slice_stride;
    if (r < rank) {
        const double* v = G1 + (int64_t)r * S;
        const int e = oz_row_exp(v, S, lane);
        oz_slice_row(v, S, KP, e, base, slice_stride, chunk_stride, row, lane);
        if (lane == 0) er[r] = e;
    } else {
        oz_slice_row(G1, 0, KP, 0, base, slice_stride, chunk_stride, row, lane);   // zero row
        if (lane == 0) er[r] = 0;
    }
}

// box image: [slice][box tile][K-chunk][128 rows][128-byte row] for the boxes boxes[0..n)
// (input row in_rows[p] when given, else boxes[p]); rows beyond n are zero. One warp per row.
__global__ void k_oz_slice_boxes(const double* chk, int S, const int32_t* boxes, const int32_t* in_rows, int n,
                                 int nbt, __half* img, int* eb) {
    const int p = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= nbt * OZ_M) return;
    const int KP = oz_kp(S), NK = oz_nk(S);
    const int tile = p / OZ_M, row = p % OZ_M;
    const int64_t chunk_stride = (int64_t)OZ_M * 64, slice_stride = (int64_t)nbt * NK * chunk_stride;
    __half* base = img + (int64_t)tile * NK * chunk_stride;
    if (p < n) {
        const double* v = chk + (int64_t)(in_rows ? in_rows[p] : boxes[p]) * S;
        const int e = oz_row_exp(v, S, lane);
        oz_slice_row(v, S, KP, e, base, slice_stride, chunk_stride, row, lane);
        if (lane == 0) eb[p] = e;
    } else {
        oz_slice_row(chk, 0, KP, 0, base, slice_stride, chunk_stride, row, lane);
        if (lane == 0) eb[p] = 0;
    }
}

// 2^k as a double (exponent bits in the normal range, ldexp outside it)
__device__ __forceinline__ double pow2d(int k) {
    if (k >= -1022 && k <= 1023) return __longlong_as_double((long long)(k + 1023) << 52);
    return ldexp(1.0, k);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

template <int NK>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_pinv_oz(const __half* __restrict__ bimg, const __half* __restrict__ opimg, const int* __restrict__ eb,
              const int* __restrict__ er, const int32_t* __restrict__ boxes, int n, int nbt, int rank, int S,
              double* __restrict__ cu, int R, int* err) {
    constexpr uint32_t CHUNK = OZ_M * 128;              // one box-slice K-chunk image
    constexpr uint32_t OPCH = OZ_N * 128;               // one operator-slice K-chunk image
    constexpr uint32_t OPB = OZ_S * NK * OPCH;          // all operator slices of the row tile
    constexpr uint32_t NCOLS = 512;                     // 9 accumulators x 48 columns
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int NS = oz_stages(NK);
    __shared__ uint64_t full[NS], empty[NS], opfull, done, drained;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ int ers[OZ_N];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* ops = base;                // operator slices
    unsigned char* stg = base + OPB;          // box-slice stages
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bt = blockIdx.x, rt = blockIdx.y;
    const int r0 = rt * OZ_N;
    const int KP = oz_kp(S);
    const int total = OZ_S * NK;
    if (tid < OZ_N) ers[tid] = (r0 + tid < rank) ? er[r0 + tid] : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&opfull), 1);
        mbar_init(smem_u32(&done), 1);
        mbar_init(smem_u32(&drained), 8);   // one arrival per epilogue warp and box tile
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 8) {
        // ---------------- producer ----------------
        // persistent: the operator slices once, then the box slices of the CTA's box tiles
        // bt, bt + gridDim.x, ... through the stage ring (g counts stages over the tiles)
        if (lane == 0) {
            const uint32_t ob = smem_u32(&opfull);
            mbar_expect(ob, OPB);
            const unsigned char* src = reinterpret_cast<const unsigned char*>(opimg) + (int64_t)rt * OPB;
            for (int c = 0; c < OZ_S * NK; ++c) bulk_g2s(smem_u32(ops + c * OPCH), src + (int64_t)c * OPCH, OPCH, ob);
            const int64_t slice_stride = (int64_t)nbt * NK * CHUNK;
            int g = 0;
            bool ok = true;
            for (int btile = bt; ok && btile < nbt; btile += gridDim.x) {
                for (int it = 0; it < total; ++it, ++g) {
                    const int s = g % NS;
                    if (g >= NS && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((g / NS - 1) & 1), &abort_flag)) {
                        ok = false;
                        break;
                    }
                    const int i = it / NK, kc = it % NK;
                    const uint32_t fb = smem_u32(&full[s]);
                    mbar_expect(fb, CHUNK);
                    const unsigned char* a = reinterpret_cast<const unsigned char*>(bimg) + i * slice_stride +
                                             ((int64_t)btile * NK + kc) * CHUNK;
                    bulk_g2s(smem_u32(stg + s * CHUNK), a, CHUNK, fb);
                }
            }
        }
        __syncwarp();
    } else if (warp == 9) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = f16_idesc(OZ_M, OZ_N);
            bool ok = mbar_wait(smem_u32(&opfull), 0, &abort_flag);
            uint32_t fphase[NS] = {};
            int g = 0, tl = 0;
            for (int btile = bt; ok && btile < nbt; btile += gridDim.x, ++tl) {
                // the accumulators are reused: wait until the epilogue has read the last tile's
                if (tl > 0) {
                    if (!mbar_wait(smem_u32(&drained), (uint32_t)((tl - 1) & 1), &abort_flag)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                for (int it = 0; it < total; ++it, ++g) {
                    const int s = g % NS;
                    if (!mbar_wait(smem_u32(&full[s]), fphase[s], &abort_flag)) {
                        ok = false;
                        break;
                    }
                    fphase[s] ^= 1u;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int i = it / NK, kc = it % NK;
                    const int ksteps = min(OZ_KC, KP - kc * OZ_KC) / 16;
                    const uint32_t a0 = smem_u32(stg + s * CHUNK);
                    for (int j = 0; i + j < OZ_S; ++j) {   // levels i + j = 0 .. 8 (slices 1-based: 2 .. 10)
                        const uint32_t dacc = tmem + (uint32_t)((i + j) * OZ_N);
                        const uint32_t b0 = smem_u32(ops + (j * NK + kc) * OPCH);
                        for (int k = 0; k < ksteps; ++k) {
                            const uint32_t acc = (i > 0 || kc > 0 || k > 0) ? 1u : 0u;
                            mma_f16(dacc, sw128_desc(a0 + 32u * k), sw128_desc(b0 + 32u * k), idesc, acc);
                        }
                    }
                    mma_commit(smem_u32(&empty[s]));
                }
                if (ok) mma_commit(smem_u32(&done));
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 0-7 ----------------
        const int q = warp & 3, half = warp >> 2;   // rows 32q..32q+31, columns 24 half .. +23
        const uint32_t t_row = (uint32_t)(32 * q) << 16;
        int tl = 0;
        for (int btile = bt; btile < nbt; btile += gridDim.x, ++tl) {
            const bool ok = mbar_wait(smem_u32(&done), (uint32_t)(tl & 1), &abort_flag);
            if (__any_sync(0xffffffffu, !ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // level sums are exact integers below 2^22 in FP32: read them as integers (magic-number
            // add) and combine exactly in 64-bit integers, levels 2..6 (hi) and 7..10 (lo)
            long long hi[24], lo[24];
#pragma unroll
            for (int c = 0; c < 24; ++c) hi[c] = lo[c] = 0;
            for (int L = 0; L < OZ_S; ++L) {
                uint32_t v[24];
                const uint32_t ta = tmem + t_row + (uint32_t)(L * OZ_N + 24 * half);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(ta));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
                      "=r"(v[23])
                    : "r"(ta + 16u));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int c = 0; c < 24; ++c) {
                    const long long P = (long long)(__float_as_int(__uint_as_float(v[c]) + 12582912.0f) - 0x4B400000);
                    if (L <= 4) hi[c] += P << (OZ_W * (4 - L));
                    else lo[c] += P << (OZ_W * (8 - L));
                }
            }
            // every level is in registers: hand the accumulators back to the MMA warp
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&drained));
            const int p = btile * OZ_M + 32 * q + lane;
            if (p < n) {
                const int e_b = eb[p];
                double* o = cu + (int64_t)boxes[p] * R + r0 + 24 * half;
#pragma unroll
                for (int c = 0; c < 24; ++c) {
                    if (r0 + 24 * half + c >= rank) break;
                    // c = 2^{e_b + e_r} (hi 2^-36 + lo 2^-60)
                    const int E = e_b + ers[24 * half + c];
                    o[c] = fma((double)hi[c], pow2d(E - 36), (double)lo[c] * pow2d(E - 60));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(err, 2);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------
size_t pinv_oz_op_bytes(int S, int rank) { return (size_t)((rank + OZ_N - 1) / OZ_N) * oz_b_bytes(S); }
double pinv_oz_mma_flops(int S, int rank, int n) {
    if (n <= 0) return 0.0;
    const double pairs = OZ_S * (OZ_S + 1) / 2;   // slice pairs with i + j <= 10
    return pairs * 2.0 * OZ_M * OZ_N * oz_kp(S) * ((n + OZ_M - 1) / OZ_M) * ((rank + OZ_N - 1) / OZ_N);
}
size_t pinv_oz_box_bytes(int S, int n) { return (size_t)OZ_S * ((n + OZ_M - 1) / OZ_M) * oz_nk(S) * OZ_M * 128; }

int pinv_oz_prepare(cudaStream_t st, const double* G1, int S, int rank, void* img, int* er) {
    const int ntile = (rank + OZ_N - 1) / OZ_N;
    const int64_t th = (int64_t)ntile * OZ_N * 32;
    k_oz_slice_op<<<(unsigned)((th + 255) / 256), 256, 0, st>>>(G1, S, rank, ntile, reinterpret_cast<__half*>(img),
                                                                 er);
    KF_LAUNCH();
    return KIFMM_OK;
}

template <int NK>
static int launch_oz(cudaStream_t st, const void* bimg, const void* opimg, const int* eb, const int* er,
                     const int32_t* boxes, int n, int nbt, int rank, int S, double* cu, int R, int* err) {
    const size_t smem = oz_smem(S);
    static bool configured = false;
    if (!configured) {
        KF_CUDA(cudaFuncSetAttribute(k_pinv_oz<NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    static int num_sms = 0;
    if (!num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        num_sms = std::max(num_sms, 1);
    }
    const int nrt = (rank + OZ_N - 1) / OZ_N;   // one wave: about one CTA per SM over the row tiles
    dim3 g(std::min(nbt, std::max(1, num_sms / nrt)), nrt);
    k_pinv_oz<NK><<<g, OZ_THREADS, smem, st>>>(reinterpret_cast<const __half*>(bimg),
                                                 reinterpret_cast<const __half*>(opimg), eb, er, boxes, n, nbt, rank, S,
                                                 cu, R, err);
    KF_LAUNCH();
    return KIFMM_OK;
}

int pinv_oz_apply(cudaStream_t st, const double* chk, int S, const int32_t* boxes, const int32_t* in_rows, int n,
                  const void* opimg, const int* er, int rank, void* bimg, int* eb, double* cu, int R, int* err,
                  int64_t* launches) {
    if (n <= 0) return KIFMM_OK;
    const int nbt = (n + OZ_M - 1) / OZ_M;
    const int64_t th = (int64_t)nbt * OZ_M * 32;
    k_oz_slice_boxes<<<(unsigned)((th + 255) / 256), 256, 0, st>>>(chk, S, boxes, in_rows, n, nbt,
                                                                    reinterpret_cast<__half*>(bimg), eb);
    KF_LAUNCH();
    switch (oz_nk(S)) {
        case 1: KF_TRY(launch_oz<1>(st, bimg, opimg, eb, er, boxes, n, nbt, rank, S, cu, R, err)); break;
        case 2: KF_TRY(launch_oz<2>(st, bimg, opimg, eb, er, boxes, n, nbt, rank, S, cu, R, err)); break;
        case 3: KF_TRY(launch_oz<3>(st, bimg, opimg, eb, er, boxes, n, nbt, rank, S, cu, R, err)); break;
        default: set_error("FP64-exact upward solve: surface too large"); return KIFMM_ERR_ARG;
    }
    if (launches) *launches += 2;
    return KIFMM_OK;
}

}  // namespace kifmm
