// M2L (Eq. (m2l)) on the 5th-generation tensor cores: a 3-term FP16 split with FP32
// accumulation (x = x_hi + x_lo, both FP16 with the 11-bit significand of TF32, products
// hi*hi + hi*lo + lo*hi), so the result carries the accuracy of a 3xTF32 product at half
// the operand bytes and twice the MMA rate of kind::tf32. FP16's exponent range is handled by
// exact power-of-two scaling: each box's coefficient row c[A] by 2^{e_A} and each level's T
// table by 2^{e_T} (largest magnitude near 2^14); the epilogue undoes 2^{e_A + e_T} per slot.
//
// In the coefficient basis the translation of one level is, for every target box B,
//   d[B] = sum over the offset slots of V(B):  T[slot] c[A(B, slot)],
// with T[slot] (R x R) shared by every pair with that relative offset. One CTA takes a
// tile of 128 target boxes of a level (boxes grouped by their octant inside the parent,
// so that the tile's boxes share one set of about 189 offsets) and a block of NT <= 256
// output rows (one block when R <= 256), and, per offset slot and 64-wide k-chunk,
// multiplies the gathered source rows c[A] (A operand, 128 x 64) by the chunk's rows of
// T[slot] (B operand, NT x 64), both K-major in the 128-byte swizzled layout.
//
// Roles (warp specialization, 11 warps):
//  * warps 8-9, producers: per iteration each thread gathers two source rows with
//    16-byte cp.async copies (hi and lo, zero-filled where the box has no source at this
//    offset); thread 0 of warp 8 also moves the pre-swizzled B chunk with two 1-D bulk
//    copies. Completion arrives on the stage's "full" mbarrier.
//  * warp 10, lane 0: waits for a full stage, issues its k-steps x 3 MMAs into the slot's
//    tensor-memory accumulator and commits the stage's "empty" mbarrier; after the last
//    chunk of a slot it commits the accumulator's "ready" mbarrier.
//  * warps 0-7, epilogue: a ring of up to four accumulators takes the slots in turn; the
//    epilogue scales a finished one by the slot's 2^{-(e_A + e_T)} into FP32 registers
//    (round-to-nearest) and releases it. The tensor core's own (truncating) accumulation
//    thus spans one slot, not the V list, and (R <= 256) within a k-chunk the small cross
//    terms are accumulated before the hi x hi terms.
// Every wait is bounded; a timeout sets an abort flag that ends the other roles' waits,
// records an error code, and the tensor memory is freed before the CTA exits.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace kifmm {

constexpr int TC_M = 128;                 // target boxes per tile = MMA M
constexpr int TC_KH = 64;                 // k-chunk: 64 FP16 = one 128-byte swizzle row
constexpr int TC_HI_EXP = 14;             // scaled operands keep their largest magnitude near 2^14
constexpr int TC_EPI = 256;               // epilogue threads (warps 0-7)
constexpr int TC_PROD = 64;               // producer threads (warps 8-9), two source rows each
constexpr int TC_THREADS = TC_EPI + TC_PROD + 32;

// ------------------------------------------------------------------------------------
// plan and per-evaluation operand preparation
// ------------------------------------------------------------------------------------
// largest |T| of a level's table, as the bits of a non-negative double (ordered like integers)
__global__ void k_absmax(const double* x, int64_t n, unsigned long long* out) {
    double m = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(x[e]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// T (FP64 [343][R][R]) * 2^sT -> Thi/Tlo (FP16) in the order [slot][k-chunk][row][128-byte
// swizzled row of 64 FP16], k >= R zero, so that one chunk of one slot is a contiguous
// R*128-byte image of the shared-memory B tile.
__global__ void k_swizzle_T(const double* T, int R, int NK, int nslots, int sT, __half* Thi, __half* Tlo) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)R * NK * TC_KH;
    if (e >= (int64_t)nslots * per) return;
    const int64_t slot = e / per;
    const int row = (int)((e % per) / (NK * TC_KH)), k = (int)(e % (NK * TC_KH));
    const float x = k < R ? (float)ldexp(T[(slot * R + row) * R + k], sT) : 0.f;
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(x - __half2float(h));
    const int64_t byte = (slot * NK + k / TC_KH) * (int64_t)R * 128 + sw128_off_h(row, k % TC_KH);
    Thi[byte / 2] = h;
    Tlo[byte / 2] = l;
}

// upward coefficients (FP64, rows of R) -> their FP32 values scaled by 2^{e_b} per box (largest
// magnitude near 2^14), split into FP16 hi/lo; one warp per box
template <class TIN>
__global__ void k_split_c(const TIN* c, int64_t nb, int R, __half* chi, __half* clo, int* cexp, int ldo) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    const TIN* row = c + b * R;
    float m = 0.f;
    for (int k = lane; k < R; k += 32) m = fmaxf(m, fabsf((float)row[k]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = 0;
    if (m > 0.f) {
        int ex;
        frexpf(m, &ex);             // m = f 2^ex, f in [0.5, 1)
        e = TC_HI_EXP + 1 - ex;     // m 2^e in [2^13, 2^14)
    }
    for (int k = lane; k < ldo; k += 32) {   // (output rows of ldo, zero beyond R)
        const float x = k < R ? ldexpf((float)row[k], e) : 0.f;
        const __half h = __float2half_rn(x);
        chi[b * ldo + k] = h;
        clo[b * ldo + k] = __float2half_rn(x - __half2float(h));
    }
    if (lane == 0) cexp[b] = e;
}

// ------------------------------------------------------------------------------------
// the kernel
// ------------------------------------------------------------------------------------
// R = NB NT coefficients per box; each CTA computes the NT = 32 NC output rows
// n0 = blockIdx.y NT .. of its tile (NB > 1 where R exceeds the MMA's N of 256).
template <int NC, int NS, int NB>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc(M2LTables tabs, const int4* __restrict__ tiles, const int32_t* __restrict__ all_boxes,
             const int32_t* __restrict__ vtab, int vstride, const int32_t* __restrict__ slots,
             const __half* __restrict__ chi, const __half* __restrict__ clo, const int* __restrict__ cexp,
             float* __restrict__ d, int accum, int* err) {
    constexpr int NT = 32 * NC;
    constexpr int R = NB * NT;
    constexpr int NK = (R + TC_KH - 1) / TC_KH;
    const int n0 = blockIdx.y * NT;
    constexpr int A_BYTES = TC_M * 128, B_BYTES = NT * 128;
    constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    // a ring of NACC slot accumulators of ACC columns each in the 512 TMEM columns, so that the
    // MMAs of a slot wait for the drain of the slot NACC back, not the one before last
    constexpr int ACC = (NT + 31) / 32 * 32;
    constexpr int NACC = 512 / ACC >= 4 ? 4 : 512 / ACC;
    constexpr uint32_t NCOLS = NACC * ACC <= 32 ? 32 : (NACC * ACC <= 64 ? 64 : (NACC * ACC <= 128 ? 128 : (NACC * ACC <= 256 ? 256 : 512)));
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t full[NS], empty[NS], ready[NACC], freed[NACC];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ int sl[344];   // [count, slot_0, ...] of this tile
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 tile = tiles[blockIdx.x];   // level, first box (index into all_boxes), box count
    const __half* __restrict__ Thi = reinterpret_cast<const __half*>(tabs.hi[tile.x]);
    const __half* __restrict__ Tlo = reinterpret_cast<const __half*>(tabs.lo[tile.x]);
    const int sT = tabs.sT[tile.x];
    const int32_t* __restrict__ boxes = all_boxes + tile.y;
    const int nbox = tile.z;
    const int t0 = 0;
    for (int e = tid; e < 344; e += TC_THREADS) sl[e] = slots[(int64_t)blockIdx.x * 344 + e];
    __syncthreads();
    const int ns = sl[0];
    const int total = ns * NK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), TC_PROD + 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int j = 0; j < NACC; ++j) {
            mbar_init(smem_u32(&ready[j]), 1);
            mbar_init(smem_u32(&freed[j]), TC_EPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp >= 8 && warp < 10) {
        // ---------------- producers ----------------
        const int p = tid - TC_EPI;          // 0..63: rows p and p + 64 of the tile
        int box2[2];
        for (int h = 0; h < 2; ++h) box2[h] = (t0 + p + 64 * h < nbox) ? boxes[t0 + p + 64 * h] : -1;
        // source box of each row for the current slot; the next slot's are fetched one slot
        // ahead so that the index load is off the critical path
        auto lookup = [&](int si, int h) -> int {
            return (si < ns && box2[h] >= 0) ? vtab[(int64_t)box2[h] * vstride + sl[1 + si]] : -1;
        };
        int acur[2] = {lookup(0, 0), lookup(0, 1)};
        int anext[2] = {lookup(1, 0), lookup(1, 1)};
        for (int it = 0; it < total; ++it) {
            const int s = it % NS;
            if (it % NK == 0 && it > 0) {
                const int si = it / NK;
                acur[0] = anext[0];
                acur[1] = anext[1];
                anext[0] = lookup(si + 1, 0);
                anext[1] = lookup(si + 1, 1);
            }
            if (it >= NS && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((it / NS - 1) & 1), &abort_flag)) break;
            const int slot = sl[1 + it / NK];
            const int kc = it % NK;
            const int k0 = kc * TC_KH;
            const int kvalid = min(TC_KH, R - k0);
            unsigned char* st = base + s * STAGE;
            if (p == 0) {   // B: two pre-swizzled bulk copies (hi, lo) of rows n0 .. n0 + NT - 1, 128 bytes each
                const uint32_t fb = smem_u32(&full[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(2 * B_BYTES)
                             : "memory");
                const int64_t off = (((int64_t)slot * NK + kc) * R + n0) * TC_KH;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(st + 2 * A_BYTES)),
                    "l"(Thi + off), "r"(B_BYTES), "r"(fb)
                    : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(st + 2 * A_BYTES + B_BYTES)),
                    "l"(Tlo + off), "r"(B_BYTES), "r"(fb)
                    : "memory");
            }
            // A: rows p, p + 64 = c[source of the row's box at this slot], chunk k0..k0+kvalid-1,
            // hi and lo (8 FP16 per 16-byte copy)
            const uint32_t ah = smem_u32(st), al = smem_u32(st + A_BYTES);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = p + 64 * h;
                const int a = acur[h];
                const uint32_t nbytes = a >= 0 ? 16u : 0u;   // 0: zero fill
                const int64_t src = (int64_t)(a >= 0 ? a : 0) * R + k0;
#pragma unroll
                for (int j = 0; j < TC_KH / 8; ++j) {
                    if (8 * j < kvalid) {
                        const uint32_t o = sw128_off_h(row, 8 * j);
                        cp_async16(ah + o, chi + src + 8 * j, nbytes);
                        cp_async16(al + o, clo + src + 8 * j, nbytes);
                    }
                }
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[s])) : "memory");
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 10) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = f16_idesc(TC_M, NT);
            uint32_t fphase[NS] = {};
            for (int si = 0; si < ns && !abort_flag; ++si) {
                const int j = si % NACC;
                if (si >= NACC && !mbar_wait(smem_u32(&freed[j]), (uint32_t)(((si - NACC) / NACC) & 1), &abort_flag))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dacc = tmem + (uint32_t)(j * ACC);
                bool ok = true;
                for (int kc = 0; kc < NK; ++kc) {
                    const int it = si * NK + kc, s = it % NS;
                    if (!mbar_wait(smem_u32(&full[s]), fphase[s], &abort_flag)) {
                        ok = false;
                        break;
                    }
                    fphase[s] ^= 1u;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const unsigned char* st = base + s * STAGE;
                    const uint32_t ah = smem_u32(st), al = ah + A_BYTES, bh = ah + 2 * A_BYTES, bl = bh + B_BYTES;
                    const int ksteps = min(TC_KH, R - kc * TC_KH) / 16;
                    if (NB == 1) {
                        // the small cross terms of the chunk first, then its hi x hi terms: the
                        // accumulator truncates each addition, so most additions then land on a
                        // small partial sum (16 FP16 = 32 bytes along K inside the swizzle row)
                        for (int k = 0; k < ksteps; ++k) {
                            const uint32_t ko = 32u * k;
                            const uint32_t acc = (kc > 0 || k > 0) ? 1u : 0u;
                            mma_f16(dacc, sw128_desc(ah + ko), sw128_desc(bl + ko), idesc, acc);
                            mma_f16(dacc, sw128_desc(al + ko), sw128_desc(bh + ko), idesc, 1u);
                        }
                        for (int k = 0; k < ksteps; ++k) {
                            const uint32_t ko = 32u * k;
                            mma_f16(dacc, sw128_desc(ah + ko), sw128_desc(bh + ko), idesc, 1u);
                        }
                    } else {
                        // row blocks of 256 (R > 256): the interleaved order, which measured 8 %
                        // faster there (consecutive MMAs on the same A tile)
                        for (int k = 0; k < ksteps; ++k) {
                            const uint32_t ko = 32u * k;
                            const uint32_t acc = (kc > 0 || k > 0) ? 1u : 0u;
                            mma_f16(dacc, sw128_desc(ah + ko), sw128_desc(bh + ko), idesc, acc);
                            mma_f16(dacc, sw128_desc(ah + ko), sw128_desc(bl + ko), idesc, 1u);
                            mma_f16(dacc, sw128_desc(al + ko), sw128_desc(bh + ko), idesc, 1u);
                        }
                    }
                    mma_commit(smem_u32(&empty[s]));
                }
                if (!ok) break;
                mma_commit(smem_u32(&ready[j]));
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 0-7 ----------------
        const int q = warp & 3, half = warp >> 2;
        const uint32_t t_row = (uint32_t)(32 * q) << 16;
        const int col0 = half * (NT / 2);
        float acc[NT / 2];
#pragma unroll
        for (int k = 0; k < NT / 2; ++k) acc[k] = 0.f;
        // this row's box and the scale 2^{-(e_A + e_T)} of its source at each slot (one slot ahead)
        const int brow = t0 + 32 * q + lane;
        const int bbox = brow < nbox ? boxes[brow] : -1;
        auto slot_scale = [&](int si) -> float {
            if (si >= ns || bbox < 0) return 0.f;
            const int a = vtab[(int64_t)bbox * vstride + sl[1 + si]];
            return a >= 0 ? pow2i(-(cexp[a] + sT)) : 0.f;
        };
        float fnext = slot_scale(0);
        for (int si = 0; si < ns; ++si) {
            const int j = si % NACC;
            const float f = fnext;
            fnext = slot_scale(si + 1);
            const bool ok = mbar_wait(smem_u32(&ready[j]), (uint32_t)((si / NACC) & 1), &abort_flag);
            if (__any_sync(0xffffffffu, !ok)) break;   // warp-uniform exit (tcgen05.ld is .sync.aligned)
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int cc = 0; cc < NT / 2; cc += 16) {
                uint32_t v[16];
                const uint32_t ta = tmem + t_row + (uint32_t)(j * ACC + col0 + cc);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int k = 0; k < 16; ++k) acc[cc + k] = fmaf(__uint_as_float(v[k]), f, acc[cc + k]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&freed[j]));
        }
        const int bi = t0 + 32 * q + lane;
        if (!abort_flag && bi < nbox) {
            float4* o = reinterpret_cast<float4*>(d + (int64_t)boxes[bi] * R + n0 + col0);
#pragma unroll
            for (int k = 0; k < NT / 8; ++k) {
                float4 v = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
                if (accum) {   // add to the row already there (L2L onto the M2L result)
                    const float4 u = o[k];
                    v = make_float4(u.x + v.x, u.y + v.y, u.z + v.z, u.w + v.w);
                }
                o[k] = v;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(err, 1);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------
static int stages_for(int R) {
    const size_t stage = 2 * (size_t)TC_M * 128 + 2 * (size_t)R * 128;
    const size_t avail = 227 * 1024 - 1024 - 1024;
    int ns = (int)(avail / stage);
    return ns > 4 ? 4 : ns;
}

size_t m2l_tc_smem(int R) {
    const size_t stage = 2 * (size_t)TC_M * 128 + 2 * (size_t)R * 128;
    return 1024 + (size_t)stages_for(R) * stage;
}

// row blocks per tile: the MMA's N is at most 256
static int row_blocks(int R) { return (R + 255) / 256; }

// coefficient counts with a compiled kernel: R <= 256 in one row block, and the Chebyshev
// counts 384, 512, 768, 1024 in blocks of 192 or 256 rows
int m2l_tc_supported(int R) {
    if (R % 32 != 0 || R < 32) return 0;
    if (R > 256 && R != 384 && R != 512 && R != 768 && R != 1024) return 0;
    const int nb = row_blocks(R);
    return (R % (32 * nb) == 0 && stages_for(R / nb) >= 2) ? 1 : 0;
}

int64_t m2l_tc_table_elems(int R, int nslots) { return (int64_t)nslots * ((R + TC_KH - 1) / TC_KH) * R * TC_KH; }

int m2l_tc_prepare(cudaStream_t st, const double* T, int R, void* Thi, void* Tlo, int* sT_out, int nslots) {
    const int64_t n = (int64_t)nslots * R * R;
    DevBuf mx;
    KF_TRY(dev_alloc(mx, 8));
    KF_CUDA(cudaMemsetAsync(mx.p, 0, 8, st));
    k_absmax<<<1024, 256, 0, st>>>(T, n, ptr<unsigned long long>(mx));
    KF_LAUNCH();
    unsigned long long bits = 0;
    KF_CUDA(cudaMemcpyAsync(&bits, mx.p, 8, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    dev_free(mx);
    double m;
    std::memcpy(&m, &bits, 8);
    int ex = 0;
    if (m > 0.0) std::frexp(m, &ex);
    const int sT = m > 0.0 ? TC_HI_EXP + 1 - ex : 0;   // max |T| 2^sT in [2^13, 2^14)
    *sT_out = sT;
    const int NK = (R + TC_KH - 1) / TC_KH;
    const int64_t ne = m2l_tc_table_elems(R, nslots);
    k_swizzle_T<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(T, R, NK, nslots, sT, reinterpret_cast<__half*>(Thi),
                                                              reinterpret_cast<__half*>(Tlo));
    KF_LAUNCH();
    return KIFMM_OK;
}

int m2l_tc_split(cudaStream_t st, const double* c, int64_t nb, int R, void* chi, void* clo, int* cexp) {
    if (nb <= 0) return KIFMM_OK;
    k_split_c<double><<<(unsigned)((nb * 32 + 255) / 256), 256, 0, st>>>(c, nb, R, reinterpret_cast<__half*>(chi),
                                                                         reinterpret_cast<__half*>(clo), cexp, R);
    KF_LAUNCH();
    return KIFMM_OK;
}

int m2l_tc_split_pad(cudaStream_t st, const double* c, int64_t nb, int R, int ldo, void* chi, void* clo, int* cexp) {
    if (nb <= 0) return KIFMM_OK;
    k_split_c<double><<<(unsigned)((nb * 32 + 255) / 256), 256, 0, st>>>(c, nb, R, reinterpret_cast<__half*>(chi),
                                                                         reinterpret_cast<__half*>(clo), cexp, ldo);
    KF_LAUNCH();
    return KIFMM_OK;
}

int m2l_tc_split_f32(cudaStream_t st, const float* c, int64_t nb, int R, void* chi, void* clo, int* cexp) {
    if (nb <= 0) return KIFMM_OK;
    k_split_c<float><<<(unsigned)((nb * 32 + 255) / 256), 256, 0, st>>>(c, nb, R, reinterpret_cast<__half*>(chi),
                                                                        reinterpret_cast<__half*>(clo), cexp, R);
    KF_LAUNCH();
    return KIFMM_OK;
}

// Launch arguments other than the tile set: the source table (vtab, row stride vstride), the
// per-tile slot lists, the split coefficients, the output and whether it is added to.
struct TcArgs {
    const int32_t* vtab;
    int vstride;
    const int32_t* slots;
    const void* chi;
    const void* clo;
    const int* cexp;
    float* d;
    int accum;
    int* err;
};

template <int NC, int NS, int NB>
static int launch_cfg(cudaStream_t st, const M2LTables& tabs, const int4* tiles, int ntiles, const int32_t* boxes,
                      const TcArgs& a) {
    const size_t smem = m2l_tc_smem(32 * NC);
    static bool configured = false;   // one attribute per instantiation (its size never changes)
    if (!configured) {
        KF_CUDA(cudaFuncSetAttribute(k_m2l_tc<NC, NS, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    k_m2l_tc<NC, NS, NB><<<dim3(ntiles, NB), TC_THREADS, smem, st>>>(
        tabs, tiles, boxes, a.vtab, a.vstride, a.slots, reinterpret_cast<const __half*>(a.chi),
        reinterpret_cast<const __half*>(a.clo), a.cexp, a.d, a.accum, a.err);
    KF_LAUNCH();
    return KIFMM_OK;
}

template <int NC, int NB>
static int launch_nc(cudaStream_t st, const M2LTables& tabs, const int4* tiles, int ntiles, const int32_t* boxes,
                     const TcArgs& a) {
    switch (stages_for(32 * NC)) {
        case 2: return launch_cfg<NC, 2, NB>(st, tabs, tiles, ntiles, boxes, a);
        case 3: return launch_cfg<NC, 3, NB>(st, tabs, tiles, ntiles, boxes, a);
        default: return launch_cfg<NC, 4, NB>(st, tabs, tiles, ntiles, boxes, a);
    }
}

int launch_tc_translate(cudaStream_t st, const M2LTables& tabs, int R, const int4* tiles, int ntiles,
                        const int32_t* boxes, const int32_t* vtab, int vstride, const int32_t* slots, const void* chi,
                        const void* clo, const int* cexp, float* d, int accum, int* err) {
    if (ntiles <= 0) return KIFMM_OK;
    const TcArgs a{vtab, vstride, slots, chi, clo, cexp, d, accum, err};
#define KF_M2L_TC(NC, NB) return launch_nc<NC, NB>(st, tabs, tiles, ntiles, boxes, a)
    switch (m2l_tc_supported(R) ? R : 0) {
        case 32: KF_M2L_TC(1, 1);
        case 64: KF_M2L_TC(2, 1);
        case 96: KF_M2L_TC(3, 1);
        case 128: KF_M2L_TC(4, 1);
        case 160: KF_M2L_TC(5, 1);
        case 192: KF_M2L_TC(6, 1);
        case 224: KF_M2L_TC(7, 1);
        case 256: KF_M2L_TC(8, 1);
        case 384: KF_M2L_TC(6, 2);    // Chebyshev p = 7
        case 512: KF_M2L_TC(8, 2);    // p = 8
        case 768: KF_M2L_TC(8, 3);    // p = 9
        case 1024: KF_M2L_TC(8, 4);   // p = 10
        default: set_error("M2L tensor path: unsupported coefficient count"); return KIFMM_ERR_ARG;
    }
#undef KF_M2L_TC
}

int launch_m2l_tc(cudaStream_t st, const M2LTables& tabs, int R, const int4* tiles, int ntiles, const int32_t* boxes,
                  const int32_t* vtab, const int32_t* slots, const void* chi, const void* clo, const int* cexp, float* d,
                  int* err) {
    return launch_tc_translate(st, tabs, R, tiles, ntiles, boxes, vtab, kOffsetSlots, slots, chi, clo, cexp, d, 0, err);
}

}  // namespace kifmm
