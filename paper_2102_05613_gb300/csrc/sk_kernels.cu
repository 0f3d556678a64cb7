// sk_kernels.cu -- start-state, energy and step-counter kernels, and the
// dispatch of the step kernel (sk_step.cuh, instantiated per coupling type
// and rule in sk_step_*.cu).
#include <cuda_runtime.h>
#include <algorithm>
#include <type_traits>
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
cudaError_t launch_step_pm1_mcmcmc_direct_nw(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_pm1_mcmcmc_direct_nw(int, int, uint32_t, uint32_t);
cudaError_t launch_step_pm1_metropolis_direct_nw(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_pm1_metropolis_direct_nw(int, int, uint32_t, uint32_t);
cudaError_t launch_step_gauss_mcmcmc_direct_nw(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_gauss_mcmcmc_direct_nw(int, int, uint32_t, uint32_t);
cudaError_t launch_step_gauss_metropolis_direct_nw(int, int, const JobDev*, const WorkItem*, uint32_t, uint32_t*,
                                      uint32_t, uint32_t, uint32_t, uint32_t, cudaStream_t);
int occupancy_gauss_metropolis_direct_nw(int, int, uint32_t, uint32_t);

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

// Start spins: from `init` (chains x N, +-1) or Philox domain 1 (128 spins
// per block, bit set -> -1), written padded to the chain's row (padding 0);
// each thread writes 4 spins.  Also clears the per-chain counters.
__global__ void spins_kernel(JobDev jb, const int8_t* __restrict__ init) {
    const uint32_t npad = jb.Npad, N = jb.N;
    const uint32_t words = npad / 4;  // 4 spins per thread
    const uint64_t total = static_cast<uint64_t>(jb.chains) * words;
    const uint32_t k0 = static_cast<uint32_t>(jb.seed), k1 = static_cast<uint32_t>(jb.seed >> 32);
    const uint32_t c3 = (1u << 24) | (jb.stream & 0xFFFFFFu);
    for (uint64_t x = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t chain = static_cast<uint32_t>(x / words);
        const uint32_t i0 = static_cast<uint32_t>(x % words) * 4u;
        uint32_t packed = 0;
        if (init) {
            for (uint32_t k = 0; k < 4u; ++k) {
                const uint32_t i = i0 + k;
                const int v = i < N ? init[static_cast<size_t>(chain) * N + i] : 0;
                packed |= (static_cast<uint32_t>(v) & 0xFFu) << (8u * k);
            }
        } else {
            const uint4 r = philox4x32_10(make_uint4(i0 / 128u, 0u, chain, c3), k0, k1);
            const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
            const uint32_t w = wv[(i0 % 128u) / 32u];
            for (uint32_t k = 0; k < 4u; ++k) {
                const uint32_t i = i0 + k, b = (i % 128u) & 31u;
                const int v = i < N ? (((w >> b) & 1u) ? -1 : 1) : 0;
                packed |= (static_cast<uint32_t>(v) & 0xFFu) << (8u * k);
            }
        }
        reinterpret_cast<uint32_t*>(jb.s)[static_cast<size_t>(chain) * words + i0 / 4u] = packed;
        if (i0 == 0) {
            jb.acc_run[chain] = 0;
            jb.work[2 * static_cast<size_t>(chain)] = 0;
            jb.work[2 * static_cast<size_t>(chain) + 1] = 0;
        }
    }
}

// Start states of several runs in one launch (blockIdx.y = run): the spins
// as spins_kernel writes them, and the run's step counter, error word,
// records, trace and recompute statistics cleared.
__global__ void start_batch_kernel(const StartJob* __restrict__ jobs) {
    const StartJob& sj = jobs[blockIdx.y];
    const JobDev& jb = sj.job;
    const uint32_t npad = jb.Npad, N = jb.N;
    const uint32_t words = npad / 4;
    const uint32_t k0 = static_cast<uint32_t>(jb.seed), k1 = static_cast<uint32_t>(jb.seed >> 32);
    const uint32_t c3 = (1u << 24) | (jb.stream & 0xFFFFFFu);
    const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const bool init4 = sj.init && (N % 4u) == 0u && (reinterpret_cast<uintptr_t>(sj.init) & 3u) == 0u;
    // chain c by CTA, its words of 4 spins by thread (no 64-bit divisions)
    for (uint32_t chain = blockIdx.x; chain < jb.chains; chain += gridDim.x)
        for (uint32_t wd = threadIdx.x; wd < words; wd += blockDim.x) {
            const uint32_t i0 = 4u * wd;
            uint32_t packed = 0;
            if (init4) {
                packed = i0 < N ? reinterpret_cast<const uint32_t*>(sj.init + static_cast<size_t>(chain) * N)[wd] : 0u;
            } else if (sj.init) {
                for (uint32_t k = 0; k < 4u; ++k) {
                    const uint32_t i = i0 + k;
                    const int v = i < N ? sj.init[static_cast<size_t>(chain) * N + i] : 0;
                    packed |= (static_cast<uint32_t>(v) & 0xFFu) << (8u * k);
                }
            } else {
                const uint4 r = philox4x32_10(make_uint4(i0 / 128u, 0u, chain, c3), k0, k1);
                const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
                const uint32_t w = wv[(i0 % 128u) / 32u];
                for (uint32_t k = 0; k < 4u; ++k) {
                    const uint32_t i = i0 + k, b = (i % 128u) & 31u;
                    const int v = i < N ? (((w >> b) & 1u) ? -1 : 1) : 0;
                    packed |= (static_cast<uint32_t>(v) & 0xFFu) << (8u * k);
                }
            }
            const size_t at = static_cast<size_t>(chain) * words + wd;
            reinterpret_cast<uint32_t*>(jb.s)[at] = packed;
            if (sj.s_op) {  // +-1 / padding 0 as e4m3 (0x38 / 0xB8) or bf16 (0x3F80 / 0xBF80)
                uint32_t e8 = 0;
                uint16_t b16[4];
                for (uint32_t k = 0; k < 4u; ++k) {
                    const int v = static_cast<int8_t>((packed >> (8u * k)) & 0xFFu);
                    e8 |= static_cast<uint32_t>(v == 0 ? 0 : (v > 0 ? 0x38 : 0xB8)) << (8u * k);
                    b16[k] = static_cast<uint16_t>(v == 0 ? 0 : (v > 0 ? 0x3F80 : 0xBF80));
                }
                if (jb.kind == 0)
                    reinterpret_cast<uint32_t*>(sj.s_op)[at] = e8;
                else
                    reinterpret_cast<uint2*>(sj.s_op)[at] =
                        make_uint2(b16[0] | (static_cast<uint32_t>(b16[1]) << 16), b16[2] | (static_cast<uint32_t>(b16[3]) << 16));
            }
        }
    for (uint64_t c = tid; c < jb.chains; c += stride) {
        jb.acc_run[c] = 0;
        jb.work[2 * c] = 0;
        jb.work[2 * c + 1] = 0;
        if (sj.ddE) sj.ddE[c] = 0.0;
    }
    const uint64_t nrec = jb.rec_capacity * jb.chains;
    for (uint64_t q = tid; q < nrec; q += stride) {
        jb.rec_E[q] = 0.0;
        jb.rec_acc[q] = 0;
        if (jb.rec_Enw) jb.rec_Enw[q] = 0.0;
        if ((q % jb.chains) < jb.chains / 2) jb.rec_q[(q / jb.chains) * (jb.chains / 2) + q % jb.chains] = 0.0;
    }
    const uint64_t ntr = static_cast<uint64_t>(jb.trace_chains) * jb.trace_steps;
    for (uint64_t q = tid; q < ntr; q += stride) jb.trace[q] = -1;
    if (tid == 0) {
        *jb.step = 0;
        *jb.err = 0;
        if (sj.dstats)
            for (int k = 0; k < 6; ++k) sj.dstats[k] = 0;
    }
}

// Local fields h[c][i] = sum_j J_ij s[c][j] of every chain, a register-tiled
// product: a CTA computes 128 sites x 64 chains, a thread 8 sites x 4
// chains, with j in chunks of 32 staged through shared memory (J is
// symmetric, so rows j of J give the columns needed).  +-J: exact int32.
// Gaussian: fp32 sums per chunk of 32 terms, added into the running total
// (blocked summation; rounding error ~ (32 + N/32) 2^-24 sum |J|).
constexpr uint32_t kFI = 128, kFC = 64, kFJ = 32;

template <typename JT>
__global__ void __launch_bounds__(256) fields_kernel(const JT* __restrict__ J, const int8_t* __restrict__ S,
                                                     void* __restrict__ Hout, uint32_t npad, uint32_t chains) {
    using A = typename dev::Types<JT>::H;  // int for +-J, float for Gaussian
    __shared__ __align__(16) A Js[kFJ][kFI];
    __shared__ __align__(16) A Ss[kFJ][kFC];
    const uint32_t tid = threadIdx.x;
    const uint32_t tx = tid & 15u, ty = tid >> 4;  // sites 4tx..4tx+3 and 64+4tx..; chains 4ty..4ty+3
    const uint32_t i0 = blockIdx.x * kFI, c0 = blockIdx.y * kFC;
    A acc[4][8], tot[4][8];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[c][k] = tot[c][k] = A(0);
    for (uint32_t j0 = 0; j0 < npad; j0 += kFJ) {
        // J rows j0..j0+31, sites i0..i0+127
        for (uint32_t e = tid; e < kFJ * kFI / 4u; e += 256u) {
            const uint32_t jj = e / (kFI / 4u), ii = (e % (kFI / 4u)) * 4u;
            const uint32_t i = i0 + ii;
            A v[4] = {A(0), A(0), A(0), A(0)};
            if (i < npad) {  // npad is a multiple of 32: all four are inside
                const JT* src = J + static_cast<size_t>(j0 + jj) * npad + i;
                if constexpr (sizeof(JT) == 1) {
                    const uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(src));
                    v[0] = dev::sbyte(w, 0); v[1] = dev::sbyte(w, 1); v[2] = dev::sbyte(w, 2); v[3] = dev::sbyte(w, 3);
                } else {
                    const float4 f = __ldg(reinterpret_cast<const float4*>(src));
                    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
                }
            }
            Js[jj][ii] = v[0]; Js[jj][ii + 1] = v[1]; Js[jj][ii + 2] = v[2]; Js[jj][ii + 3] = v[3];
        }
        // spins of chains c0..c0+63 at j0..j0+31, transposed
        for (uint32_t e = tid; e < kFC * kFJ / 4u; e += 256u) {
            const uint32_t cc = e / (kFJ / 4u), jj = (e % (kFJ / 4u)) * 4u;
            const uint32_t c = c0 + cc;
            uint32_t w = 0;
            if (c < chains) w = __ldg(reinterpret_cast<const unsigned int*>(S + static_cast<size_t>(c) * npad + j0 + jj));
#pragma unroll
            for (uint32_t k = 0; k < 4u; ++k) Ss[jj + k][cc] = static_cast<A>(dev::sbyte(w, k));
        }
        __syncthreads();
#pragma unroll 8
        for (uint32_t jj = 0; jj < kFJ; ++jj) {
            A a[8], b[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                a[k] = Js[jj][4 * tx + k];
                a[4 + k] = Js[jj][64 + 4 * tx + k];
                b[k] = Ss[jj][4 * ty + k];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[c][k] += b[c] * a[k];
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                tot[c][k] += acc[c][k];
                acc[c][k] = A(0);
            }
    }
    A* H = static_cast<A*>(Hout);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const uint32_t chain = c0 + 4u * ty + c;
        if (chain >= chains) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const uint32_t i = i0 + 64u * half + 4u * tx;
            if (i < npad)
                *reinterpret_cast<typename std::conditional<sizeof(JT) == 1, int4, float4>::type*>(
                    H + static_cast<size_t>(chain) * npad + i) = {tot[c][4 * half], tot[c][4 * half + 1],
                                                                  tot[c][4 * half + 2], tot[c][4 * half + 3]};
        }
    }
}

constexpr uint32_t kCheckThreads = 256;
// Validation of host-supplied inputs on the device.  *flag (initialised to
// all ones) receives the smallest (position << 2 | code) of a violation.
//   couplings: code 1 diagonal entry != 0, 2 entry outside {-1,0,1} (+-J) or
//   not finite (Gaussian), 3 J_ij != J_ji; position i * 2^16 + j.
// The checks run on an input stream of their own while the step kernel may
// hold most of every SM (768 threads x 80 registers leave 4096 of 65536
// registers): at 16 registers per thread a 256-thread CTA of them fits in
// what is left.  (ptxas reports raising the bound to 24, yet the kernels
// launch with 16: at 24 they wait for the step kernel's CTAs and the
// end-to-end bench step took 21.7 ms instead of 15.6 ms.)
template <typename JT>
__global__ void __maxnreg__(16) check_couplings_kernel(const JT* __restrict__ J, uint32_t N, uint32_t npad,
                                       unsigned long long* __restrict__ flag) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    // rows i = blockIdx.y, blockIdx.y + gridDim.y, ...
    for (uint32_t i = blockIdx.y; i < N; i += gridDim.y) {
        const JT a = J[static_cast<size_t>(i) * npad + j];
        const JT b = J[static_cast<size_t>(j) * npad + i];
        unsigned code = 0;
        if (i == j && a != JT(0)) code = 1;
        else if constexpr (sizeof(JT) == 1) {
            if (a < JT(-1) || a > JT(1)) code = 2;
            else if (a != b) code = 3;
        } else {
            if (!isfinite(a)) code = 2;
            else if (a != b) code = 3;
        }
        if (code) atomicMin(flag, ((static_cast<unsigned long long>(i) << 16 | j) << 2) | code);
    }
}
// Couplings drawn on the device for an instance created without couplings
// (sk_create_instance with couplings NULL): Philox4x32-10 with key = seed,
// domain 2, one draw per pair i < j, shared by J_ij and J_ji:
//   +-J:      block (j >> 7, i, 0, 2 << 24), bit j & 127 (word (j & 127) >> 5,
//             bit j & 31): set -> -1, clear -> +1;
//   Gaussian: block (j, i, 1, 2 << 24) = (w0, w1, w2, w3); two 53-bit
//             uniforms u1 = (2^26 (w0 >> 5) + (w1 >> 6)) 2^-53 and u2 from
//             (w2, w3) alike; the Box-Muller normal z = sqrt(-2 ln(1 - u1))
//             cos(2 pi u2) in double precision, J_ij = (float)(z / sqrt(N)),
//             a sample of N(0, 1/N).
// The diagonal and the padding are 0.  One thread per element of the padded
// matrix (each pair is drawn twice, once for each of its two elements).
template <typename JT>
__global__ void gen_couplings_kernel(JT* __restrict__ J, uint32_t N, uint32_t npad, uint32_t k0, uint32_t k1) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= npad) return;
    for (uint32_t r = blockIdx.y; r < npad; r += gridDim.y) {
        JT v = JT(0);
        if (r < N && c < N && r != c) {
            const uint32_t i = min(r, c), j = max(r, c);
            if constexpr (sizeof(JT) == 1) {
                const uint4 w = dev::philox4x32_10(make_uint4(j >> 7, i, 0u, 2u << 24), k0, k1);
                const uint32_t b = j & 127u;
                const uint32_t word = b < 32u ? w.x : b < 64u ? w.y : b < 96u ? w.z : w.w;
                v = ((word >> (b & 31u)) & 1u) ? JT(-1) : JT(1);
            } else {
                const uint4 w = dev::philox4x32_10(make_uint4(j, i, 1u, 2u << 24), k0, k1);
                const double u1 = (static_cast<double>(w.x >> 5) * 67108864.0 + static_cast<double>(w.y >> 6)) *
                                  0x1p-53;
                const double u2 = (static_cast<double>(w.z >> 5) * 67108864.0 + static_cast<double>(w.w >> 6)) *
                                  0x1p-53;
                const double z = sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586476925286766559 * u2);
                v = static_cast<float>(z / sqrt(static_cast<double>(N)));
            }
        }
        J[static_cast<size_t>(r) * npad + c] = v;
    }
}

//   spins: code 1 for a value other than +-1; position = index.  A few CTAs
//   per array (grid-stride loop), so that the check can run beside a
//   resident step kernel without thousands of CTA launches.
__global__ void __maxnreg__(16) check_spins_kernel(const int8_t* __restrict__ s, uint64_t n,
                                                   unsigned long long* __restrict__ flag) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t x = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; x < n; x += stride) {
        const int v = __ldg(s + x);
        if (v != 1 && v != -1) atomicMin(flag, (x << 2) | 1ull);
    }
}

// E(s) = -scale sum_i s_i g_i with g_i = sum_{j>i} J_ij s_j (the couplings
// below the diagonal, read down column i), for kEnergyChains configurations
// per CTA, so that each coupling is read once per block of configurations
// rather than once per configuration.  A thread takes the column pair
// (p, N-1-p), N-1 terms in all, so that threads and CTAs get equal work.
// Bit c of sb[j] is set when configuration c has s_j = -1.  +-J: g_i summed
// in int32 (|g_i| < N), exact; Gaussian: in double, the terms in the order
// j = i+1, i+2, ...; the per-thread parts are reduced in a fixed order, so
// results repeat bit for bit.  With gridDim.y > 1 the CTA (x, y) takes the
// pairs p = y B + t (mod gridDim.y B) and writes its part to partial[c][y]
// (summed by energy_finish); configuration blocks vary fastest in launch
// order, so the CTAs resident at a time share a few column tiles of J in L2.
constexpr uint32_t kEnergyChains = 8;
template <typename JT>
__global__ void __launch_bounds__(256) energy_kernel(const JT* __restrict__ J, uint32_t N, uint32_t npad,
                                                      double scale, const int8_t* __restrict__ spins,
                                                      uint32_t count, double* __restrict__ out,
                                                      double* __restrict__ partial) {
    using A = typename std::conditional<sizeof(JT) == 1, int, double>::type;
    constexpr uint32_t CB = kEnergyChains;
    extern __shared__ __align__(16) unsigned char sb[];
    __shared__ double red[CB][8];
    const uint32_t c0 = blockIdx.x * CB;
    const uint32_t nc = min(CB, count - c0);
    for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) {
        uint32_t m = 0;
        for (uint32_t c = 0; c < nc; ++c)
            if (spins[static_cast<size_t>(c0 + c) * N + j] < 0) m |= 1u << c;
        sb[j] = static_cast<unsigned char>(m);
    }
    __syncthreads();
    double part[CB];
#pragma unroll
    for (uint32_t c = 0; c < CB; ++c) part[c] = 0.0;
    const uint32_t P = (N + 1) / 2;  // column pairs; the middle column of an odd N stands alone
    for (uint32_t p = blockIdx.y * blockDim.x + threadIdx.x; p < P; p += gridDim.y * blockDim.x) {
        for (uint32_t half = 0; half < 2; ++half) {
            const uint32_t i = half ? N - 1 - p : p;
            if (half && i == p) break;
            A hi[CB];
#pragma unroll
            for (uint32_t c = 0; c < CB; ++c) hi[c] = A(0);
#pragma unroll 4
            for (uint32_t j = i + 1; j < N; ++j) {
                const A v = static_cast<A>(J[static_cast<size_t>(j) * npad + i]);
                const uint32_t m = sb[j];
#pragma unroll
                for (uint32_t c = 0; c < CB; ++c) hi[c] += ((m >> c) & 1u) ? -v : v;
            }
            const uint32_t mi = sb[i];
#pragma unroll
            for (uint32_t c = 0; c < CB; ++c) part[c] += static_cast<double>(((mi >> c) & 1u) ? -hi[c] : hi[c]);
        }
    }
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (uint32_t c = 0; c < CB; ++c) {
        const double v = warp_sum(part[c]);
        if (lane == 0) red[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        double v = 0.0;
        for (uint32_t w = 0; w < blockDim.x / 32; ++w) v += red[threadIdx.x][w];
        if (gridDim.y == 1)
            out[c0 + threadIdx.x] = -scale * v;
        else
            partial[static_cast<size_t>(c0 + threadIdx.x) * gridDim.y + blockIdx.y] = v;
    }
}

__global__ void energy_finish(const double* __restrict__ partial, uint32_t tiles, uint32_t count, double scale,
                              double* __restrict__ out) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count) return;
    double v = 0.0;
    for (uint32_t y = 0; y < tiles; ++y) v += partial[static_cast<size_t>(c) * tiles + y];
    out[c] = -scale * v;
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

// class = kind * 256 + rule * 128 + stage * 32 + log2(NB) * 8 + log2(G), or -1;
// stage 0 rows through L1, 1 rows staged by TMA, 2 rows through L1 with
// node-weighted energy records.  Metropolis draws one block; its NB field
// names the field update of the 128-register variant instead: 2 (chunks)
// when a lane's share of a row of npad couplings, npad / (4 G) float4 or
// int32 words, is not a whole number of 8-word passes, else 1.
int step_class(uint32_t kind, uint32_t rule, uint32_t K, uint32_t G, uint32_t stage, uint32_t npad) {
    uint32_t nb = blocks_per_lane(rule, K, G);
    if (!nb) return -1;
    if (rule == 1 && npad && (npad / (4u * G)) % 8u != 0u) nb = 2;
    int lg = 0;
    while ((1u << lg) < G) ++lg;
    const int lnb = nb == 1 ? 0 : (nb == 2 ? 1 : 2);
    return static_cast<int>(kind) * 256 + static_cast<int>(rule) * 128 + static_cast<int>(stage > 2 ? 0 : stage) * 32 +
           lnb * 8 + lg;
}
uint32_t class_lanes(int cls) { return 1u << (cls & 7); }
bool class_staged(int cls) { return ((cls >> 5) & 3) == 1; }

#define SK_DISPATCH(F, ...)                                                          \
    do {                                                                             \
        const int kind_ = cls >> 8, rule_ = (cls >> 7) & 1, stage_ = (cls >> 5) & 3; \
        if (kind_ == 0 && rule_ == 0)                                                \
            return stage_ == 1 ? F##_pm1_mcmcmc_staged(__VA_ARGS__)                  \
                 : stage_ == 2 ? F##_pm1_mcmcmc_direct_nw(__VA_ARGS__) : F##_pm1_mcmcmc_direct(__VA_ARGS__); \
        if (kind_ == 0)                                                              \
            return stage_ == 1 ? F##_pm1_metropolis_staged(__VA_ARGS__)              \
                 : stage_ == 2 ? F##_pm1_metropolis_direct_nw(__VA_ARGS__) : F##_pm1_metropolis_direct(__VA_ARGS__); \
        if (rule_ == 0)                                                              \
            return stage_ == 1 ? F##_gauss_mcmcmc_staged(__VA_ARGS__)                \
                 : stage_ == 2 ? F##_gauss_mcmcmc_direct_nw(__VA_ARGS__) : F##_gauss_mcmcmc_direct(__VA_ARGS__); \
        return stage_ == 1 ? F##_gauss_metropolis_staged(__VA_ARGS__)                \
             : stage_ == 2 ? F##_gauss_metropolis_direct_nw(__VA_ARGS__) : F##_gauss_metropolis_direct(__VA_ARGS__); \
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
    return launch_bump_steps(jobs, n_jobs, nsteps, st);
}

cudaError_t launch_bump_steps(const JobDev* jobs, uint32_t n_jobs, uint64_t nsteps, cudaStream_t st) {
    bump_steps<<<(n_jobs + 127) / 128, 128, 0, st>>>(jobs, n_jobs, nsteps);
    return cudaGetLastError();
}

int step_kernel_occupancy(int cls, uint32_t W, size_t per_chain) {
    const int nb = 1 << ((cls >> 3) & 3), G = 1 << (cls & 7);
    return occupancy_class(cls, nb, G, W, static_cast<uint32_t>(per_chain));
}

cudaError_t launch_init(const JobDev* job, const int8_t* init, uint32_t chains, uint32_t N,
                        uint32_t Npad, uint32_t kind, cudaStream_t st, bool with_fields) {
    (void)N;
    const uint64_t words = static_cast<uint64_t>(chains) * (Npad / 4);
    const uint32_t blocks = static_cast<uint32_t>(std::min<uint64_t>((words + 255) / 256, 152ull * 64));
    spins_kernel<<<blocks, 256, 0, st>>>(*job, init);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !with_fields) return e;
    const dim3 grid((Npad + kFI - 1) / kFI, (chains + kFC - 1) / kFC);
    if (kind == 0)
        fields_kernel<int8_t><<<grid, 256, 0, st>>>(static_cast<const int8_t*>(job->J), job->s, job->h, Npad, chains);
    else
        fields_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(job->J), job->s, job->h, Npad, chains);
    return cudaGetLastError();
}

cudaError_t launch_start_batch(const StartJob* jobs_dev, uint32_t n, uint64_t max_words, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    (void)max_words;
    start_batch_kernel<<<dim3(512, n), 128, 0, st>>>(jobs_dev);
    return cudaGetLastError();
}

cudaError_t launch_check_couplings(const void* J, uint32_t kind, uint32_t N, uint32_t Npad,
                                   unsigned long long* flag, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(flag, 0xFF, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const dim3 grid((N + kCheckThreads - 1) / kCheckThreads, std::min<uint32_t>(N, 64));
    if (kind == 0)
        check_couplings_kernel<int8_t><<<grid, kCheckThreads, 0, st>>>(static_cast<const int8_t*>(J), N, Npad, flag);
    else
        check_couplings_kernel<float><<<grid, kCheckThreads, 0, st>>>(static_cast<const float*>(J), N, Npad, flag);
    return cudaGetLastError();
}

cudaError_t launch_gen_couplings(void* J, uint32_t kind, uint32_t N, uint32_t Npad, uint64_t seed, cudaStream_t st) {
    const dim3 grid((Npad + 255) / 256, std::min<uint32_t>(Npad, 1024));
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    if (kind == 0)
        gen_couplings_kernel<int8_t><<<grid, 256, 0, st>>>(static_cast<int8_t*>(J), N, Npad, k0, k1);
    else
        gen_couplings_kernel<float><<<grid, 256, 0, st>>>(static_cast<float*>(J), N, Npad, k0, k1);
    return cudaGetLastError();
}

cudaError_t launch_check_spins(const int8_t* s, uint64_t n, unsigned long long* flag, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(flag, 0xFF, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const uint32_t blocks = static_cast<uint32_t>(std::min<uint64_t>((n + 4095) / 4096, 64));
    if (blocks) check_spins_kernel<<<blocks, kCheckThreads, 0, st>>>(s, n, flag);
    return cudaGetLastError();
}

uint32_t energy_tiles(uint32_t N, uint32_t count) {
    // enough CTAs for two waves of 152 SMs, at most one column pair per thread
    const uint32_t blocks = (count + kEnergyChains - 1) / kEnergyChains;
    const uint32_t most = ((N + 1) / 2 + 255) / 256;
    return std::max(1u, std::min(most, (304u + blocks - 1) / blocks));
}

cudaError_t launch_energy(const void* J, uint32_t kind, uint32_t N, uint32_t Npad, double scale,
                          const int8_t* spins, uint32_t count, double* out, cudaStream_t st, double* partial) {
    const size_t sm = (N + 15) / 16 * 16;
    const uint32_t tiles = partial ? energy_tiles(N, count) : 1u;
    const dim3 grid((count + kEnergyChains - 1) / kEnergyChains, tiles);
    if (kind == 0)
        energy_kernel<int8_t><<<grid, 256, sm, st>>>(static_cast<const int8_t*>(J), N, Npad, scale, spins, count,
                                                     out, partial);
    else
        energy_kernel<float><<<grid, 256, sm, st>>>(static_cast<const float*>(J), N, Npad, scale, spins, count,
                                                    out, partial);
    if (tiles > 1) energy_finish<<<(count + 255) / 256, 256, 0, st>>>(partial, tiles, count, scale, out);
    return cudaGetLastError();
}

}  // namespace sk
