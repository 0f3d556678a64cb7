// sk_device.cuh -- device helpers shared by the sampler's kernels: the
// Philox4x32-10 generator, mbarrier / bulk-copy (TMA) primitives, 2^x on the
// special-function unit, and the coupling-type traits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sk {
namespace dev {

constexpr uint32_t kFull = 0xffffffffu;
constexpr long long kWaitBudgetCycles = 4000000000ll;  // ~2 s at 2 GHz

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA) helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Stage `bytes` (multiple of 16, both addresses 16-byte aligned) of global
// memory into shared memory; completion is signalled on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false after ~2 s without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > kWaitBudgetCycles) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// small warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_min(int v) { return __reduce_min_sync(kFull, v); }
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ int warp_sum(int v) { return __reduce_add_sync(kFull, v); }
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    return v;
}
__device__ __forceinline__ float warp_incl_scan(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    return v;
}
__device__ __forceinline__ int sbyte(uint32_t w, int e) {
    return static_cast<int>(static_cast<int32_t>(w << (24 - 8 * e)) >> 24);
}

template <typename JT>
struct Types;
template <>
struct Types<int8_t> {
    using H = int;        // fields and energy differences: exact integers
    using W = unsigned long long;
};
template <>
struct Types<float> {
    using H = float;
    using W = float;
};




// Spins +-1 (padding 0) as tensor-core operands: four spins of a 32-bit word
// as four e4m3 bytes (+-1.0 = 0x38 / 0xB8), or spins e, e+1 of it as two bf16
// words (+-1.0 = 0x3F80 / 0xBF80).
__device__ __forceinline__ uint32_t e4m3_of4(uint32_t w) {
    uint32_t o = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int v = static_cast<int>(static_cast<int32_t>(w << (24 - 8 * e)) >> 24);
        o |= static_cast<uint32_t>(v == 0 ? 0u : (v > 0 ? 0x38u : 0xB8u)) << (8 * e);
    }
    return o;
}
__device__ __forceinline__ uint32_t bf16_of2(uint32_t w, int e) {
    uint32_t o = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int v = static_cast<int>(static_cast<int32_t>(w << (24 - 8 * (e + k))) >> 24);
        o |= static_cast<uint32_t>(v == 0 ? 0u : (v > 0 ? 0x3F80u : 0xBF80u)) << (16 * k);
    }
    return o;
}
// Sixteen spins (one 16-byte word) written as operands at spin index i16*16
// of the operand array (bf: bf16, else e4m3).
__device__ __forceinline__ void spins_to_op16(void* op, size_t i16, uint4 w, bool bf) {
    if (bf) {
        uint4* o = static_cast<uint4*>(op) + 2 * i16;
        o[0] = make_uint4(bf16_of2(w.x, 0), bf16_of2(w.x, 2), bf16_of2(w.y, 0), bf16_of2(w.y, 2));
        o[1] = make_uint4(bf16_of2(w.z, 0), bf16_of2(w.z, 2), bf16_of2(w.w, 0), bf16_of2(w.w, 2));
    } else {
        static_cast<uint4*>(op)[i16] = make_uint4(e4m3_of4(w.x), e4m3_of4(w.y), e4m3_of4(w.z), e4m3_of4(w.w));
    }
}

// A field of the CTA's shared job descriptor read where it is used (a
// volatile shared-memory load) instead of being held in a register across
// the whole step loop.
template <typename T>
__device__ __forceinline__ T at_use(const T& x) {
    return *const_cast<const volatile T*>(&x);
}

// 2^x on the special-function unit (ex2.approx.ftz: relative error < 2^-22
// over the range used here, x <= 0).  exp(-beta dE) = 2^(-beta log2(e) dE).
__device__ __forceinline__ float pow2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace dev
}  // namespace sk
