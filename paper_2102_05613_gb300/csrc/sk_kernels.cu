// sk_kernels.cu -- start-state, energy and step-counter kernels, and the
// dispatch of the step kernel (sk_step.cuh, instantiated per coupling type
// and rule in sk_step_*.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sk_device.cuh"
#include "sk_internal.h"

namespace sk {

cudaError_t launch_step_pm1_mcmcmc_staged(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_pm1_mcmcmc_staged(int, int, uint32_t, uint32_t);
cudaError_t launch_step_pm1_mcmcmc_direct(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_pm1_mcmcmc_direct(int, int, uint32_t, uint32_t);
cudaError_t launch_step_pm1_metropolis_staged(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_pm1_metropolis_staged(int, int, uint32_t, uint32_t);
cudaError_t launch_step_pm1_metropolis_direct(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_pm1_metropolis_direct(int, int, uint32_t, uint32_t);
cudaError_t launch_step_gauss_mcmcmc_staged(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_gauss_mcmcmc_staged(int, int, uint32_t, uint32_t);
cudaError_t launch_step_gauss_mcmcmc_direct(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_gauss_mcmcmc_direct(int, int, uint32_t, uint32_t);
cudaError_t launch_step_gauss_metropolis_staged(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_gauss_metropolis_staged(int, int, uint32_t, uint32_t);
cudaError_t launch_step_gauss_metropolis_direct(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_gauss_metropolis_direct(int, int, uint32_t, uint32_t);

namespace {

using dev::kFull;
using dev::philox4x32_10;
using dev::warp_sum;

__global__ void bump_steps(const JobDev* __restrict__ jobs, uint32_t n_jobs, uint64_t nsteps) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_jobs) {
        const uint64_t lim = jobs[j].step_limit;
        const uint64_t s = *jobs[j].step + nsteps;
        *jobs[j].step = s < lim ? s : lim;
    }
}

// Start state: spins from `init` (chains x N, +-1) or Philox domain 1
// (128 spins per block, bit set -> -1); fields h_i = sum_j J_ji s_j for
// kInitChains chains per CTA (each J element read once for all of them),
// exact integers for +-J, compensated (Kahan) float sums for Gaussian J.
constexpr uint32_t kInitChains = 8;

template <typename JT>
__global__ void __launch_bounds__(256) init_kernel(JobDev jb, const int8_t* __restrict__ init) {
    extern __shared__ __align__(16) unsigned char sm[];
    int8_t* s = reinterpret_cast<int8_t*>(sm);  // [kInitChains][npad]
    const uint32_t N = jb.N, npad = jb.Npad;
    const uint32_t c0 = blockIdx.x * kInitChains;
    const uint32_t nc = min(kInitChains, jb.chains - c0);
    for (uint32_t c = 0; c < nc; ++c) {
        const uint32_t chain = c0 + c;
        int8_t* sc = s + static_cast<size_t>(c) * npad;
        if (init) {
            for (uint32_t i = threadIdx.x; i < npad; i += blockDim.x)
                sc[i] = i < N ? init[static_cast<size_t>(chain) * N + i] : 0;
        } else {
            const uint32_t k0 = static_cast<uint32_t>(jb.seed), k1 = static_cast<uint32_t>(jb.seed >> 32);
            const uint32_t c3 = (1u << 24) | (jb.stream & 0xFFFFFFu);
            for (uint32_t b = threadIdx.x; b * 128u < npad; b += blockDim.x) {
                const uint4 r = philox4x32_10(make_uint4(b, 0u, chain, c3), k0, k1);
                const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
                for (uint32_t k = 0; k < 128u && b * 128u + k < npad; ++k) {
                    const uint32_t i = b * 128u + k;
                    sc[i] = i < N ? (((wv[k >> 5] >> (k & 31)) & 1u) ? -1 : 1) : 0;
                }
            }
        }
    }
    __syncthreads();
    for (uint32_t c = 0; c < nc; ++c)
        for (uint32_t i = threadIdx.x; i < npad; i += blockDim.x)
            jb.s[static_cast<size_t>(c0 + c) * npad + i] = s[static_cast<size_t>(c) * npad + i];
    const JT* J = static_cast<const JT*>(jb.J);
    for (uint32_t i = threadIdx.x; i < npad; i += blockDim.x) {
        if constexpr (sizeof(JT) == 1) {
            int acc[kInitChains] = {};
            for (uint32_t j = 0; j < N; ++j) {
                const int v = J[static_cast<size_t>(j) * npad + i];
#pragma unroll
                for (uint32_t c = 0; c < kInitChains; ++c) acc[c] += v * s[c * npad + j];
            }
            for (uint32_t c = 0; c < nc; ++c)
                static_cast<int*>(jb.h)[static_cast<size_t>(c0 + c) * npad + i] = acc[c];
        } else {
            float sum[kInitChains] = {}, comp[kInitChains] = {};
            for (uint32_t j = 0; j < N; ++j) {
                const float v = J[static_cast<size_t>(j) * npad + i];
#pragma unroll
                for (uint32_t c = 0; c < kInitChains; ++c) {
                    const float y = (s[c * npad + j] > 0 ? v : -v) - comp[c];
                    const float tsum = sum[c] + y;
                    comp[c] = (tsum - sum[c]) - y;
                    sum[c] = tsum;
                }
            }
            for (uint32_t c = 0; c < nc; ++c)
                static_cast<float*>(jb.h)[static_cast<size_t>(c0 + c) * npad + i] = sum[c];
        }
    }
    if (threadIdx.x < nc) {
        const uint32_t chain = c0 + threadIdx.x;
        jb.acc_run[chain] = 0;
        jb.work[2 * static_cast<size_t>(chain)] = 0;
        jb.work[2 * static_cast<size_t>(chain) + 1] = 0;
    }
}

// E(s) = -scale sum_{i<j} J_ij s_i s_j = -scale/2 sum_i s_i sum_j J_ij s_j.
template <typename JT>
__global__ void energy_kernel(const JT* __restrict__ J, uint32_t N, uint32_t npad, double scale,
                              const int8_t* __restrict__ spins, double* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    int8_t* s = reinterpret_cast<int8_t*>(sm);
    __shared__ double red[32];
    const uint32_t c = blockIdx.x;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) s[i] = spins[static_cast<size_t>(c) * N + i];
    __syncthreads();
    double part = 0.0;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
        double hi = 0.0;
        for (uint32_t j = 0; j < N; ++j) hi += static_cast<double>(J[static_cast<size_t>(j) * npad + i]) * s[j];
        part += hi * s[i];
    }
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) out[c] = -0.5 * scale * v;
    }
}

}  // namespace

// Philox blocks of sites a step draws, rounded up to a power of two
// (MCMCMC: ceil(K/4); Metropolis draws block 0 only).
uint32_t site_blocks_pow2(uint32_t rule, uint32_t K) {
    uint32_t kb = 1;
    if (rule == 0)
        while (4 * kb < K) kb <<= 1;
    return kb;
}
// Blocks per lane for G lanes per chain, or 0 when no kernel has that shape:
// NB = 1 for every G, 2 for G = 8, 16, 32, 4 for G = 8, 16.
uint32_t blocks_per_lane(uint32_t rule, uint32_t K, uint32_t G) {
    const uint32_t kb = site_blocks_pow2(rule, K);
    const uint32_t nb = kb > G ? kb / G : 1u;
    if (nb == 1) return (G == 4 || G == 8 || G == 16 || G == 32) ? 1u : 0u;
    if (nb == 2) return (G == 8 || G == 16 || G == 32) ? 2u : 0u;
    if (nb == 4) return (G == 8 || G == 16) ? 4u : 0u;
    return 0u;
}

// class = kind * 128 + rule * 64 + stage * 32 + log2(NB) * 8 + log2(G), or -1
int step_class(uint32_t kind, uint32_t rule, uint32_t K, uint32_t G, uint32_t stage) {
    const uint32_t nb = blocks_per_lane(rule, K, G);
    if (!nb) return -1;
    int lg = 0;
    while ((1u << lg) < G) ++lg;
    const int lnb = nb == 1 ? 0 : (nb == 2 ? 1 : 2);
    return static_cast<int>(kind) * 128 + static_cast<int>(rule) * 64 + static_cast<int>(stage != 0) * 32 +
           lnb * 8 + lg;
}
uint32_t class_lanes(int cls) { return 1u << (cls & 7); }
bool class_staged(int cls) { return ((cls >> 5) & 1) != 0; }

#define SK_DISPATCH(F, ...)                                                          \
    do {                                                                             \
        const int kind_ = cls >> 7, rule_ = (cls >> 6) & 1, stage_ = (cls >> 5) & 1; \
        if (kind_ == 0 && rule_ == 0) return stage_ ? F##_pm1_mcmcmc_staged(__VA_ARGS__) : F##_pm1_mcmcmc_direct(__VA_ARGS__); \
        if (kind_ == 0) return stage_ ? F##_pm1_metropolis_staged(__VA_ARGS__) : F##_pm1_metropolis_direct(__VA_ARGS__); \
        if (rule_ == 0) return stage_ ? F##_gauss_mcmcmc_staged(__VA_ARGS__) : F##_gauss_mcmcmc_direct(__VA_ARGS__); \
        return stage_ ? F##_gauss_metropolis_staged(__VA_ARGS__) : F##_gauss_metropolis_direct(__VA_ARGS__); \
    } while (0)

namespace {
cudaError_t launch_class(int cls, int nb, int G, const JobDev* jobs, const WorkItem* items, uint32_t n_items,
                         uint32_t* queue, uint32_t ns, uint32_t W, uint32_t per_chain, uint32_t grid, cudaStream_t st) {
    SK_DISPATCH(launch_step, nb, G, jobs, items, n_items, queue, ns, W, per_chain, grid, st);
}
int occupancy_class(int cls, int nb, int G, uint32_t W, uint32_t pc) {
    SK_DISPATCH(occupancy, nb, G, W, pc);
}
}  // namespace

cudaError_t launch_step(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                        uint64_t nsteps, uint32_t W, uint32_t per_chain, uint32_t grid, int cls, uint32_t n_jobs,
                        bool bump, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const uint32_t ns = static_cast<uint32_t>(nsteps);
    const int nb = 1 << ((cls >> 3) & 3), G = 1 << (cls & 7);
    e = launch_class(cls, nb, G, jobs, items, n_items, queue, ns, W, per_chain, grid, st);
    if (e != cudaSuccess || !bump) return e;
    bump_steps<<<(n_jobs + 127) / 128, 128, 0, st>>>(jobs, n_jobs, nsteps);
    return cudaGetLastError();
}

int step_kernel_occupancy(int cls, uint32_t W, size_t per_chain) {
    const int nb = 1 << ((cls >> 3) & 3), G = 1 << (cls & 7);
    return occupancy_class(cls, nb, G, W, static_cast<uint32_t>(per_chain));
}

cudaError_t launch_init(const JobDev* job, const int8_t* init, uint32_t chains, uint32_t N,
                        uint32_t Npad, uint32_t kind, cudaStream_t st) {
    (void)N;
    const uint32_t blocks = (chains + kInitChains - 1) / kInitChains;
    const size_t sm = static_cast<size_t>(kInitChains) * Npad;
    cudaError_t e;
    if (kind == 0) {
        e = cudaFuncSetAttribute(init_kernel<int8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
        if (e != cudaSuccess) return e;
        init_kernel<int8_t><<<blocks, 256, sm, st>>>(*job, init);
    } else {
        e = cudaFuncSetAttribute(init_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
        if (e != cudaSuccess) return e;
        init_kernel<float><<<blocks, 256, sm, st>>>(*job, init);
    }
    return cudaGetLastError();
}

cudaError_t launch_energy(const void* J, uint32_t kind, uint32_t N, uint32_t Npad, double scale,
                          const int8_t* spins, uint32_t count, double* out, cudaStream_t st) {
    const size_t sm = (N + 15) / 16 * 16;
    if (kind == 0)
        energy_kernel<int8_t><<<count, 256, sm, st>>>(static_cast<const int8_t*>(J), N, Npad, scale, spins, out);
    else
        energy_kernel<float><<<count, 256, sm, st>>>(static_cast<const float*>(J), N, Npad, scale, spins, out);
    return cudaGetLastError();
}

}  // namespace sk
