// M2L (Eq. (m2l)) on the 5th-generation tensor cores, split 3xTF32 with FP32 accumulation.
//
// In the coefficient basis the translation of one level is, for every target box B,
//   d[B] = sum over the offset slots of V(B):  T[slot] c[A(B, slot)],
// T[slot] (R x R) shared by every pair with that relative offset. One CTA takes a tile of
// 128 consecutive boxes of a level and keeps D[128 x R] (boxes x output coefficients) in
// tensor memory across all slots of the tile. Per slot and 32-wide k-chunk the CTA
// gathers the 128 source rows c[A] (A operand, K-major) and the chunk of T[slot]
// (B operand, K-major), splits each FP32 value x into x_hi = tf32(x) and
// x_lo = tf32(x - x_hi) while writing them to shared memory in the 128-byte swizzled
// layout, and one thread issues 4 k-steps x 3 MMAs (hi*hi + hi*lo + lo*hi).
// Two shared-memory stages alternate; an mbarrier per stage (tcgen05.commit) tells the
// producers when the tensor core has finished reading a stage. Every wait is bounded: on
// timeout the kernel records an error code, frees its tensor memory and returns.
#include "internal.cuh"

namespace kifmm {

constexpr int TC_M = 128;          // boxes per tile = MMA M
constexpr int TC_T = 256;          // threads per CTA
constexpr int TC_KC = 32;          // k-chunk: 32 FP32 = one 128-byte swizzle atom per row
constexpr uint32_t TC_SPIN = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return u;
}

// Shared-memory matrix descriptor (tcgen05): K-major operand, 128-byte swizzle, rows of
// 128 bytes grouped by 8 (1024-byte atoms). start >> 4 in bits [0,14), leading byte
// offset >> 4 in [16,30) (unused for this layout), stride byte offset >> 4 in [32,46)
// (= 1024 between 8-row groups), fixed 0b01 in [46,48), swizzle mode 2 (128B) in [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < TC_SPIN; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Split 4 FP32 values into TF32 hi/lo and store them at the swizzled position of
// (row, 16-byte chunk j) of two 128-byte-row tiles.
__device__ __forceinline__ void store_split(unsigned char* hi, unsigned char* lo, int row, int j, float4 v) {
    const uint32_t off = (uint32_t)row * 128u + (uint32_t)((j ^ (row & 7)) * 16);
    uint32_t h0 = tf32_rna(v.x), h1 = tf32_rna(v.y), h2 = tf32_rna(v.z), h3 = tf32_rna(v.w);
    uint32_t l0 = tf32_rna(v.x - __uint_as_float(h0)), l1 = tf32_rna(v.y - __uint_as_float(h1));
    uint32_t l2 = tf32_rna(v.z - __uint_as_float(h2)), l3 = tf32_rna(v.w - __uint_as_float(h3));
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h0, h1, h2, h3);
    *reinterpret_cast<uint4*>(lo + off) = make_uint4(l0, l1, l2, l3);
}

// d[b] = sum_slots T[slot] c[src(b, slot)] for the boxes [lo + 128*blockIdx.x, +128) of one level.
// Dynamic shared memory: 2 stages x (A_hi, A_lo: 128 x 128 B; B_hi, B_lo: R x 128 B), 1024-aligned.
// Tensor memory: two accumulators of R columns, ACC apart (ACC = R rounded up to a power
// of two). The MMAs of one
// slot go to one accumulator (restarted at its first k-step); while the next slot's MMAs
// run, every thread adds its row-half of the finished accumulator into FP32 registers
// with round-to-nearest additions. The tensor core's internal accumulation therefore
// spans one slot (R/8 x 3 MMAs) instead of the whole V list. NC = R / 32.
template <int NC>
__global__ void __launch_bounds__(TC_T, 1) k_m2l_tc(const float* __restrict__ Tm, const int32_t* __restrict__ vtab,
                                                    const int32_t* __restrict__ slots, int64_t lo, int64_t hi,
                                                    const float* __restrict__ c, float* __restrict__ d, int* err) {
    constexpr int R = 32 * NC;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t mbar[2];     // shared-memory stage s free again
    __shared__ uint64_t accbar[2];   // accumulator j holds a finished slot
    __shared__ uint32_t tmem_base;
    __shared__ int bad;
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int a_bytes = TC_M * 128, b_bytes = R * 128;
    constexpr int stage_bytes = 2 * a_bytes + 2 * b_bytes;
    const int64_t b0 = lo + (int64_t)blockIdx.x * TC_M;
    const int32_t* sl = slots + (int64_t)blockIdx.x * 344;
    const int ns = sl[0];
    constexpr int nk = R / TC_KC;
    const int total = ns * nk;
    constexpr int ACC = R <= 32 ? 32 : (R <= 64 ? 64 : (R <= 128 ? 128 : 256));
    constexpr uint32_t ncols = 2 * ACC;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        bad = 0;
        for (int k = 0; k < 2; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[k])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accbar[k])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tf32_idesc(TC_M, R);
    uint32_t phase[2] = {0u, 0u}, aphase[2] = {0u, 0u};
    // this thread's share of the result: row 32*(warp%4)+lane, columns [half*R/2, +R/2)
    const int q = warp & 3, half = warp >> 2;
    const uint32_t t_row = (uint32_t)(32 * q) << 16;
    const int col0 = half * (R / 2);
    float acc[R / 2];
#pragma unroll
    for (int k = 0; k < R / 2; ++k) acc[k] = 0.f;

    // adds accumulator j (finished slot) into acc[]
    auto drain = [&](int j) -> bool {
        const bool ok = mbar_wait(smem_u32(&accbar[j]), aphase[j]);
        aphase[j] ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int cc = 0; cc < R / 2; cc += 16) {
            uint32_t v[16];
            const uint32_t ta = tmem + t_row + (uint32_t)(j * ACC + col0 + cc);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[cc + k] += __uint_as_float(v[k]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        return ok;
    };

    for (int it = 0; it < total; ++it) {
        const int s = it & 1;
        const int si = it / nk, kc = it % nk;
        unsigned char* A_hi = base + s * stage_bytes;
        unsigned char* A_lo = A_hi + a_bytes;
        unsigned char* B_hi = A_lo + a_bytes;
        unsigned char* B_lo = B_hi + b_bytes;
        if (it >= 2) {   // the MMAs of iteration it-2 read this stage: wait until they are done
            const int timed_out = mbar_wait(smem_u32(&mbar[s]), phase[s]) ? 0 : 1;
            phase[s] ^= 1u;
            if (__syncthreads_or(timed_out)) {   // uniform decision for the whole CTA
                if (tid == 0) bad = 1;
                break;
            }
        }
        const int slot = sl[1 + si];
        const int k0 = kc * TC_KC;
        // A: 128 gathered rows x 8 chunks of 16 bytes
        for (int e = tid; e < TC_M * 8; e += TC_T) {
            const int row = e >> 3, j = e & 7;
            const int64_t b = b0 + row;
            const int a = (b < hi) ? vtab[b * kOffsetSlots + slot] : -1;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a >= 0) v = *reinterpret_cast<const float4*>(c + (int64_t)a * R + k0 + 4 * j);
            store_split(A_hi, A_lo, row, j, v);
        }
        // B: R rows of T[slot] x 8 chunks
        const float* Ts = Tm + (int64_t)slot * R * R;
        for (int e = tid; e < R * 8; e += TC_T) {
            const int row = e >> 3, j = e & 7;
            float4 v = *reinterpret_cast<const float4*>(Ts + (int64_t)row * R + k0 + 4 * j);
            store_split(B_hi, B_lo, row, j, v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(A_hi), al = smem_u32(A_lo), bh = smem_u32(B_hi), bl = smem_u32(B_lo);
            const uint32_t dacc = tmem + (uint32_t)((si & 1) * ACC);
#pragma unroll
            for (int k = 0; k < TC_KC / 8; ++k) {
                const uint32_t ko = 32u * k;   // 8 TF32 = 32 bytes along K inside the swizzle atom
                const uint32_t first = (kc > 0 || k > 0) ? 1u : 0u;
                mma_tf32(dacc, sw128_desc(ah + ko), sw128_desc(bh + ko), idesc, first);
                mma_tf32(dacc, sw128_desc(ah + ko), sw128_desc(bl + ko), idesc, 1u);
                mma_tf32(dacc, sw128_desc(al + ko), sw128_desc(bh + ko), idesc, 1u);
            }
            mma_commit(smem_u32(&mbar[s]));
            if (kc == nk - 1) mma_commit(smem_u32(&accbar[si & 1]));
        }
        if (kc == 0 && si >= 1) {   // the previous slot's accumulator, while this slot's MMAs run
            const int timed_out = drain((si - 1) & 1) ? 0 : 1;
            if (__syncthreads_or(timed_out)) {
                if (tid == 0) bad = 1;
                break;
            }
        }
    }
    // drain: the last slot's accumulator, then the last commit of each used stage (also
    // after a timeout, so that the MMAs in flight finish before the tensor memory is freed)
    __syncthreads();
    int timed_out = 0;
    if (!bad && ns > 0 && !drain((ns - 1) & 1)) timed_out = 1;
    for (int s = 0; s < 2; ++s)
        if (s < total && !mbar_wait(smem_u32(&mbar[s]), phase[s])) timed_out = 1;
    if (__syncthreads_or(timed_out) && tid == 0) bad = 1;
    __syncthreads();
    if (!bad) {
        const int64_t b = b0 + 32 * q + lane;
        if (b < hi) {
            float4* o = reinterpret_cast<float4*>(d + b * R + col0);
#pragma unroll
            for (int k = 0; k < R / 8; ++k) o[k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

size_t m2l_tc_smem(int R) { return 1024 + 2 * (size_t)(2 * TC_M * 128 + 2 * R * 128); }

int m2l_tc_supported(int R) { return (R % 32 == 0 && R >= 32 && R <= 256 && m2l_tc_smem(R) <= 227 * 1024) ? 1 : 0; }

template <int NC>
static int launch_nc(cudaStream_t st, const float* Tm, const int32_t* vtab, const int32_t* slots, int64_t lo,
                     int64_t hi, const float* c, float* d, int* err, int64_t ntiles) {
    const size_t smem = m2l_tc_smem(32 * NC);
    static bool configured = false;   // one attribute per instantiation (its size never changes)
    if (!configured) {
        KF_CUDA(cudaFuncSetAttribute(k_m2l_tc<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    k_m2l_tc<NC><<<(unsigned)ntiles, TC_T, smem, st>>>(Tm, vtab, slots, lo, hi, c, d, err);
    KF_LAUNCH();
    return KIFMM_OK;
}

int launch_m2l_tc(cudaStream_t st, const float* Tm, int R, const int32_t* vtab, const int32_t* slots, int64_t lo,
                  int64_t hi, const float* c, float* d, int* err) {
    const int64_t ntiles = (hi - lo + TC_M - 1) / TC_M;
    if (ntiles <= 0) return KIFMM_OK;
    switch (R / 32) {
        case 1: return launch_nc<1>(st, Tm, vtab, slots, lo, hi, c, d, err, ntiles);
        case 2: return launch_nc<2>(st, Tm, vtab, slots, lo, hi, c, d, err, ntiles);
        case 3: return launch_nc<3>(st, Tm, vtab, slots, lo, hi, c, d, err, ntiles);
        case 4: return launch_nc<4>(st, Tm, vtab, slots, lo, hi, c, d, err, ntiles);
        case 5: return launch_nc<5>(st, Tm, vtab, slots, lo, hi, c, d, err, ntiles);
        case 6: return launch_nc<6>(st, Tm, vtab, slots, lo, hi, c, d, err, ntiles);
        case 7: return launch_nc<7>(st, Tm, vtab, slots, lo, hi, c, d, err, ntiles);
        case 8: return launch_nc<8>(st, Tm, vtab, slots, lo, hi, c, d, err, ntiles);
        default: set_error("M2L tensor path: unsupported coefficient count"); return KIFMM_ERR_ARG;
    }
}

}  // namespace kifmm
