// sk_fused.cu -- every star work item of a batch in one persistent launch.
//
// The per-class launches (one step-kernel variant per launch class) let each
// class have its own CTA shape; this kernel instead fixes one shape for the
// whole batch -- whole-warp chains (32 lanes), rows of J read through L1, W
// warps per CTA, the 128-register budget -- and dispatches each work item to
// the variant its run needs: coupling type (+-J int8 / Gaussian fp32), rule
// (MCMCMC with 1 or 2 Philox blocks per lane, i.e. K <= 128 or K <= 256;
// Metropolis with the unrolled or the chunked field update).  A CTA takes
// items from one device queue, ordered largest first; an item holds at most W
// chains of one run (an even number for runs of several chains, so that
// overlap pairs share the CTA) and fills its chains' slices of the launch's
// shared memory with its own run's slice size.  Each item runs exactly the
// code of the per-class variant with the same lanes, rows and register
// budget (run_item in sk_step.cuh), so trajectories and records are the same
// as those of whole-warp per-class launches bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sk_step.cuh"

namespace sk {
namespace {

using step::kWCache;

constexpr int kFusedMaxThreads = 512;  // W <= 16 warps; 65536 / 512 = 128 registers

__global__ void __launch_bounds__(kFusedMaxThreads, 1)
    fused_kernel(const JobDev* __restrict__ jobs, const WorkItem* __restrict__ items, uint32_t n_items,
                 uint32_t* __restrict__ queue, uint32_t nsteps) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) JobDev s_job;
    __shared__ __align__(8) uint64_t bars[2 * (kFusedMaxThreads / 32)];  // (rows are not staged: unused)
    __shared__ unsigned long long s_wt[kWCache];
    __shared__ uint32_t s_item;
    uint32_t phase = 0;
    bool dead = false;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= n_items) break;
        const WorkItem wi = items[it];
        if (threadIdx.x < sizeof(JobDev) / 16)
            reinterpret_cast<uint4*>(&s_job)[threadIdx.x] = reinterpret_cast<const uint4*>(&jobs[wi.job])[threadIdx.x];
        __syncthreads();
        const JobDev& jb = s_job;
        if (jb.kind == 0) {  // the start of the +-J weight table (0 past its end)
            for (uint32_t i = threadIdx.x; i < kWCache; i += blockDim.x)
                s_wt[i] = i < jb.wlen ? reinterpret_cast<const unsigned long long*>(jb.W)[i] : 0ull;
            __syncthreads();
        }
        const uint32_t pc = wi.pad & 0xFFFFFFu;  // the run's shared bytes per chain
        switch (wi.pad >> 24) {                  // fused_variant
            case 0: step::run_item<int8_t, 0, 1, 32, 0, 8, false>(wi, jb, smem, bars, s_wt, nsteps, pc, phase, dead); break;
            case 1: step::run_item<int8_t, 0, 2, 32, 0, 8, false>(wi, jb, smem, bars, s_wt, nsteps, pc, phase, dead); break;
            case 2: step::run_item<int8_t, 1, 1, 32, 0, 8, false>(wi, jb, smem, bars, s_wt, nsteps, pc, phase, dead); break;
            case 3: step::run_item<int8_t, 1, 1, 32, 0, 8, true>(wi, jb, smem, bars, s_wt, nsteps, pc, phase, dead); break;
            case 4: step::run_item<float, 0, 1, 32, 0, 8, false>(wi, jb, smem, bars, s_wt, nsteps, pc, phase, dead); break;
            case 5: step::run_item<float, 0, 2, 32, 0, 8, false>(wi, jb, smem, bars, s_wt, nsteps, pc, phase, dead); break;
            case 6: step::run_item<float, 1, 1, 32, 0, 8, false>(wi, jb, smem, bars, s_wt, nsteps, pc, phase, dead); break;
            default: step::run_item<float, 1, 1, 32, 0, 8, true>(wi, jb, smem, bars, s_wt, nsteps, pc, phase, dead); break;
        }
        __syncthreads();  // s_job, s_wt and the slices are reused by the next item
    }
}

}  // namespace

uint32_t fused_variant(uint32_t kind, uint32_t rule, uint32_t K, uint32_t npad) {
    uint32_t v;
    if (rule == 0)
        v = blocks_per_lane(0, K, 32) == 2 ? 1u : 0u;
    else
        v = (npad / 128u) % 8u != 0u ? 3u : 2u;  // Metropolis: chunked update unless whole 8-word passes
    return (kind == 0 ? 0u : 4u) + v;
}

cudaError_t launch_fused(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                         uint64_t nsteps, uint32_t W, uint32_t smem, uint32_t grid, uint32_t n_jobs, bool bump,
                         cudaStream_t st) {
    if (W < 1 || 32 * W > static_cast<uint32_t>(kFusedMaxThreads) || grid == 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    fused_kernel<<<grid, 32 * W, smem, st>>>(jobs, items, n_items, queue, static_cast<uint32_t>(nsteps));
    if ((e = cudaGetLastError()) != cudaSuccess || !bump) return e;
    return launch_bump_steps(jobs, n_jobs, nsteps, st);
}

int fused_occupancy(uint32_t W, uint32_t smem) {
    if (W < 1 || 32 * W > static_cast<uint32_t>(kFusedMaxThreads)) return 0;
    int n = 0;
    if (cudaFuncSetAttribute(fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_kernel, 32 * W, smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace sk
