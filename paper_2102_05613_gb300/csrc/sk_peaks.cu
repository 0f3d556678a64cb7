// sk_peaks.cu -- measured ceilings of L2 and shared memory, and the tensor
// pipe under the recompute kernel's MMA loop (sk_peaks.h).
//
// Small probe kernels whose only work is loads, timed with CUDA events; the
// step kernel's roofline divides its algorithmic bytes by these.  Every
// access stays inside the buffers the probes allocate: the L2 sweep is
// bounded by the element count, the shared-memory probes mask their word
// index to the 64 KiB array.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>

#include "sk_internal.h"
#include "sk_peaks.h"

namespace {

sk_status pfail(sk_status s, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    sk::set_error_message(msg);
    return s;
}

#define PK_CU(call)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            st_ = pfail(SK_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
            goto out;                                                                 \
        }                                                                             \
    } while (0)

// L2 sweep: every thread reads 16-byte words i, i + stride, ... of the working
// set with ld.global.cg (cached in L2 only), four loads in flight per thread.
__global__ void __launch_bounds__(512) l2_read_kernel(const uint4* __restrict__ p, uint64_t n16, uint32_t passes,
                                                      unsigned int* __restrict__ sink) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t first = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (uint32_t r = 0; r < passes; ++r) {
        uint64_t i = first;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = __ldcg(p + i);
            const uint4 b = __ldcg(p + i + stride);
            const uint4 c = __ldcg(p + i + 2 * stride);
            const uint4 d = __ldcg(p + i + 3 * stride);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(p + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);  // keeps the loads; the buffer is zero
}

constexpr uint32_t kSmemWords = 16384;  // 64 KiB
constexpr int kSmemLoads = 16;          // independent loads per thread per iteration

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

// Shared-memory loads at addresses fixed per thread; ld.volatile keeps every
// load in the loop (a plain ld.shared of a loop-invariant address with no
// store in the loop may be hoisted out of it by the assembler).  VEC16: load j of thread t reads 16-byte word
// (t + 1024 j) mod 4096 -- a warp reads 512 contiguous bytes; GATHER4: load j
// reads a random word of the array.
template <int MODE>
__global__ void __launch_bounds__(1024) smem_kernel(uint32_t iters, unsigned int* __restrict__ sink) {
    extern __shared__ __align__(16) uint32_t sm[];
    for (uint32_t i = threadIdx.x; i < kSmemWords; i += blockDim.x) sm[i] = i * 2654435761u;
    __syncthreads();
    uint32_t addr[kSmemLoads];
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(sm));
#pragma unroll
    for (int j = 0; j < kSmemLoads; ++j) {
        uint32_t w;
        if (MODE == 0)
            w = ((threadIdx.x + 1024u * j) & (kSmemWords / 4 - 1)) * 4u;
        else
            w = mix32(blockIdx.x * 1048576u + threadIdx.x * kSmemLoads + j) & (kSmemWords - 1);
        addr[j] = base + 4u * w;
    }
    uint32_t acc = 0;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kSmemLoads; ++j) {
            if (MODE == 0) {
                uint32_t a, b, c, d;
                asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
                             : "r"(addr[j]));
                acc ^= a ^ b ^ c ^ d;
            } else {
                uint32_t a;
                asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(a) : "r"(addr[j]));
                acc ^= a;
            }
        }
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);
}

}  // namespace

extern "C" sk_status sk_peak_l2_read(uint64_t working_set_bytes, uint32_t passes, uint32_t reps, void* stream,
                                     double* gbps) {
    if (!gbps) return pfail(SK_ERR_INVALID_ARG, "NULL output");
    if (working_set_bytes < (16ull << 20) || working_set_bytes > (96ull << 20) || working_set_bytes % 16)
        return pfail(SK_ERR_INVALID_ARG, "working set must be 16..96 MiB, a multiple of 16 bytes");
    if (passes == 0 || reps == 0) return pfail(SK_ERR_INVALID_ARG, "passes and reps must be >= 1");
    sk_status st_ = SK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* buf = nullptr;
    unsigned int* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = 0, sms = 0;
    float ms = 0.0f;
    const uint64_t n16 = working_set_bytes / 16;
    PK_CU(cudaGetDevice(&dev));
    PK_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PK_CU(cudaMalloc(&buf, working_set_bytes));
    PK_CU(cudaMalloc(&sink, sizeof(unsigned int)));
    PK_CU(cudaMemsetAsync(buf, 0, working_set_bytes, st));
    PK_CU(cudaEventCreate(&e0));
    PK_CU(cudaEventCreate(&e1));
    l2_read_kernel<<<4 * sms, 512, 0, st>>>(static_cast<const uint4*>(buf), n16, passes, sink);  // warm-up
    PK_CU(cudaGetLastError());
    PK_CU(cudaEventRecord(e0, st));
    for (uint32_t r = 0; r < reps; ++r)
        l2_read_kernel<<<4 * sms, 512, 0, st>>>(static_cast<const uint4*>(buf), n16, passes, sink);
    PK_CU(cudaGetLastError());
    PK_CU(cudaEventRecord(e1, st));
    PK_CU(cudaEventSynchronize(e1));
    PK_CU(cudaEventElapsedTime(&ms, e0, e1));
    *gbps = static_cast<double>(working_set_bytes) * passes * reps / (ms * 1e-3) / 1e9;
out:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    return st_;
}

extern "C" sk_status sk_peak_smem(uint32_t mode, uint32_t iters, uint32_t reps, void* stream, double* gbps) {
    if (!gbps) return pfail(SK_ERR_INVALID_ARG, "NULL output");
    if (mode != SK_PEAK_SMEM_VEC16 && mode != SK_PEAK_SMEM_GATHER4) return pfail(SK_ERR_INVALID_ARG, "unknown mode");
    if (iters == 0 || reps == 0) return pfail(SK_ERR_INVALID_ARG, "iters and reps must be >= 1");
    sk_status st_ = SK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = 0, sms = 0;
    float ms = 0.0f;
    const size_t smem = kSmemWords * 4;
    const int grid_per_sm = 2;  // 64 warps per SM
    auto launch = [&](cudaStream_t s) {
        if (mode == SK_PEAK_SMEM_VEC16)
            smem_kernel<0><<<grid_per_sm * sms, 1024, smem, s>>>(iters, sink);
        else
            smem_kernel<1><<<grid_per_sm * sms, 1024, smem, s>>>(iters, sink);
    };
    PK_CU(cudaGetDevice(&dev));
    PK_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PK_CU(cudaFuncSetAttribute(smem_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    PK_CU(cudaFuncSetAttribute(smem_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    PK_CU(cudaMalloc(&sink, sizeof(unsigned int)));
    PK_CU(cudaEventCreate(&e0));
    PK_CU(cudaEventCreate(&e1));
    launch(st);  // warm-up
    PK_CU(cudaGetLastError());
    PK_CU(cudaEventRecord(e0, st));
    for (uint32_t r = 0; r < reps; ++r) launch(st);
    PK_CU(cudaGetLastError());
    PK_CU(cudaEventRecord(e1, st));
    PK_CU(cudaEventSynchronize(e1));
    PK_CU(cudaEventElapsedTime(&ms, e0, e1));
    {
        const double bytes_per_load = mode == SK_PEAK_SMEM_VEC16 ? 16.0 : 4.0;
        const double loads = static_cast<double>(grid_per_sm) * sms * 1024.0 * kSmemLoads * iters * reps;
        *gbps = loads * bytes_per_load / (ms * 1e-3) / 1e9;
    }
out:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return st_;
}

extern "C" sk_status sk_peak_tensor(uint32_t kind, uint32_t tiles, uint32_t reps, void* stream, double* tflops) {
    if (!tflops) return pfail(SK_ERR_INVALID_ARG, "NULL output");
    if (kind > 1) return pfail(SK_ERR_INVALID_ARG, "kind must be 0 (FP8) or 1 (bf16)");
    if (tiles == 0 || tiles > 4096 || reps == 0) return pfail(SK_ERR_INVALID_ARG, "tiles must be 1..4096, reps >= 1");
    const cudaError_t e = sk::tensor_peak_probe(kind, tiles, reps, static_cast<cudaStream_t>(stream), tflops);
    if (e == cudaErrorLaunchTimeout) return pfail(SK_ERR_TIMEOUT, "a wait of the tensor probe expired");
    if (e != cudaSuccess) return pfail(SK_ERR_CUDA, "tensor probe: %s", cudaGetErrorString(e));
    return SK_OK;
}
