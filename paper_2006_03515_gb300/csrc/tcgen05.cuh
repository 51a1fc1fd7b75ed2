// tcgen05 / TMA / mbarrier building blocks (inline PTX) shared by the tensor-core kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kifmm {

constexpr uint32_t TC_SPIN = 1u << 20;   // polls before a wait gives up (a normal wait needs a few hundred)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of (row, k) inside a [rows x 64 FP16] tile in the 128-byte swizzled layout:
// rows of 128 bytes, 16-byte chunk j of row r stored at chunk j ^ (r mod 8).
__host__ __device__ __forceinline__ uint32_t sw128_off_h(int row, int k) {
    return (uint32_t)row * 128u + (uint32_t)((((k >> 3) ^ (row & 7)) << 4) | ((k & 7) << 1));
}

// 2^e as a float for integer e (0 below the normal range, infinity above it)
__device__ __forceinline__ float pow2i(int e) {
    if (e < -126) return 0.f;
    if (e > 127) return __int_as_float(0x7f800000);
    return __int_as_float((127 + e) << 23);
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 in bits [0,14), leading byte
// offset >> 4 in [16,30) (not used by this layout), stride byte offset >> 4 in [32,46)
// (1024 bytes between 8-row groups), fixed 0b001 in [46,49), swizzle mode 2 = 128-byte
// swizzle in [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B FP16 (bits 7-9 and
// 10-12 = 0), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Bounded wait for the phase of the given parity; gives up on timeout or when another
// role has raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile int* abort_flag) {
    for (uint32_t it = 0; it < TC_SPIN; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 255u && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}


}  // namespace kifmm
