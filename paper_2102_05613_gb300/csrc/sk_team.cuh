// sk_team.cuh -- the team layout of the star sampler (a3-a5 of the step):
// one chain per team of T warps (T = 2 or 4), one proposal slot per thread
// (MCMCMC with K <= 32 T, or Metropolis), for runs of few chains, where a
// step is a chain of latencies rather than a share of the GPU's throughput.
//
// The warp layout (sk_step.cuh) runs a chain's step on one warp, i.e. on one
// of an SM's four schedulers, each lane holding up to four slots and a
// 32nd of the field update.  A team spreads the slots and the update over T
// warps and joins them with team barriers (named barriers of 32 T threads):
//   1. the minimum of the candidates' dE, the reference of the weights;
//   2. the warps' weight totals, which give each warp its prefix offset and
//      every thread the total (summed in warp order);
//   3. the chosen slot, published by the warp whose range of prefixes holds
//      the draw u (left out when the root is kept, u < w0);
//   4. the updated fields and spins (left out when nothing flips).
// Metropolis takes two when it accepts (every warp at the step before the
// update, then the fourth) and none when it rejects.
// Writes to a chain's spins and fields happen only between a barrier that
// every warp of the team has reached at the same step and the fourth, so
// that no warp reads a state another has moved on from; the exchange words
// of one step are read before the barrier that follows their use, so the
// next step's writes cannot overtake them.
//
// The draws are the warp layout's: block 0 of each step (every warp keeps
// its own copy of 32 steps, so that no barrier orders its refills), and the
// sites of slots 4 (b - 1) + 1 .. 4 b from block b of the step, drawn for
// 32 T / SL steps at once (SL = the blocks a step needs, rounded up to a
// power of two) into one half of a double-buffered ring in shared memory
// while the other half is read.  The choice is the same categorical draw in
// slot order, so +-J trajectories are the warp layout's and the oracle's bit
// for bit; Gaussian weight sums are taken in another order (fp32 rounding,
// within the decision-replay tolerance).  Records use the warp layout's
// record() in the team's first warp; the CTA holds two teams for runs of
// several chains, so that overlap pairs share it.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sk_step.cuh"

namespace sk {
namespace team {

using dev::kFull;
using dev::Types;
using step::Grp;
using step::kWCache;

// Offsets in one chain's shared memory: spins (npad bytes), fields (4 npad),
// the site ring (2 x 32 T words of 8 bytes), block 0 of 32 steps per warp
// (512 bytes each), the team's exchange words (64 bytes).  team_chain_bytes
// in sk_internal.h is the total, rounded up to 128.
__device__ __forceinline__ size_t ring_off(uint32_t npad) { return static_cast<size_t>(5) * npad; }
template <int T>
__device__ __forceinline__ size_t b0_off(uint32_t npad) {
    return ring_off(npad) + 512u * T;
}
template <int T>
__device__ __forceinline__ size_t xch_off(uint32_t npad) {
    return ring_off(npad) + 1024u * T;
}

__device__ __forceinline__ void team_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// h_k -= c1 J[x1][k] (+ c2 J[x2][k] when c2 != 0) for this thread's share of
// the fields, k = 4 tid + 4 NT v: row loads of up to four passes issued
// before any field of them is read or written; per element the terms are
// added in the warp layout's order (the first flip's, then the second's).
template <typename JT, int NT>
__device__ __forceinline__ void team_update(typename Types<JT>::H* hf, const JT* r1, const JT* r2, int c1, int c2,
                                            uint32_t npad, int tid) {
    constexpr uint32_t kStride = 4u * NT;
    constexpr int U = 4;
    for (uint32_t k0 = 4u * tid; k0 < npad; k0 += kStride * U) {
        if constexpr (sizeof(JT) == 1) {
            uint32_t j1[U], j2[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t k = k0 + kStride * u;
                j1[u] = j2[u] = 0u;
                if (k < npad) {
                    j1[u] = __ldg(reinterpret_cast<const unsigned int*>(r1 + k));
                    if (c2) j2[u] = __ldg(reinterpret_cast<const unsigned int*>(r2 + k));
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t k = k0 + kStride * u;
                if (k < npad) {
                    int4 hv = *reinterpret_cast<int4*>(hf + k);
                    hv.x -= c1 * dev::sbyte(j1[u], 0);
                    hv.y -= c1 * dev::sbyte(j1[u], 1);
                    hv.z -= c1 * dev::sbyte(j1[u], 2);
                    hv.w -= c1 * dev::sbyte(j1[u], 3);
                    if (c2) {
                        hv.x -= c2 * dev::sbyte(j2[u], 0);
                        hv.y -= c2 * dev::sbyte(j2[u], 1);
                        hv.z -= c2 * dev::sbyte(j2[u], 2);
                        hv.w -= c2 * dev::sbyte(j2[u], 3);
                    }
                    *reinterpret_cast<int4*>(hf + k) = hv;
                }
            }
        } else {
            float4 j1[U], j2[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t k = k0 + kStride * u;
                j1[u] = j2[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k < npad) {
                    j1[u] = __ldg(reinterpret_cast<const float4*>(r1 + k));
                    if (c2) j2[u] = __ldg(reinterpret_cast<const float4*>(r2 + k));
                }
            }
            const float f1 = static_cast<float>(c1);
            const float f2 = static_cast<float>(c2);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t k = k0 + kStride * u;
                if (k < npad) {
                    float4 hv = *reinterpret_cast<float4*>(hf + k);
                    hv.x = fmaf(-f1, j1[u].x, hv.x);
                    hv.y = fmaf(-f1, j1[u].y, hv.y);
                    hv.z = fmaf(-f1, j1[u].z, hv.z);
                    hv.w = fmaf(-f1, j1[u].w, hv.w);
                    if (c2) {
                        hv.x = fmaf(-f2, j2[u].x, hv.x);
                        hv.y = fmaf(-f2, j2[u].y, hv.y);
                        hv.z = fmaf(-f2, j2[u].z, hv.z);
                        hv.w = fmaf(-f2, j2[u].w, hv.w);
                    }
                    *reinterpret_cast<float4*>(hf + k) = hv;
                }
            }
        }
    }
}

// Steps t0..t1-1 of one chain on its team (team index `team` of the CTA,
// named barrier 1 + team).  `write`: the chain is real (stores records and
// its trace).  The caller has loaded the chain's spins and fields into
// `base` and synchronised the CTA.
template <typename JT, int RULE, int T>
__device__ __forceinline__ void team_loop(const JobDev& jb, bool write, uint32_t chain, unsigned char* base,
                                          int partner_off, const unsigned long long* wsm, uint32_t t0, uint32_t t1,
                                          uint32_t& acc, uint32_t& n_flips, uint32_t& n_rows, int team) {
    using H = typename Types<JT>::H;
    using W = typename Types<JT>::W;
    constexpr int NT = 32 * T;
    const Grp<32> g;
    const int tid = static_cast<int>(threadIdx.x) - team * NT;
    const int warp = tid >> 5, lane = tid & 31;
    const int bar = 1 + team;
    const uint32_t N = jb.N, npad = jb.Npad, K = jb.K;
    const uint32_t nblk = (K + 3u) >> 2;
    const uint32_t k0 = static_cast<uint32_t>(jb.seed), k1 = static_cast<uint32_t>(jb.seed >> 32);
    const uint32_t c3 = jb.stream & 0xFFFFFFu;  // domain 0: step draws
    auto Jrow = [&](uint32_t r) -> const JT* {
        return static_cast<const JT*>(dev::at_use(jb.J)) + static_cast<size_t>(r) * npad;
    };
    const unsigned long long* Wt = reinterpret_cast<const unsigned long long*>(jb.W);
    const uint32_t wlen = jb.wlen;
    const float nbl2 = -jb.beta_eff * 1.4426950408889634f;  // -beta log2(e)
    const bool root_weighted = jb.fcen + jb.fleaf != (2u << 20);
    const uint32_t trace_end = (write && chain < jb.trace_chains)
                                   ? static_cast<uint32_t>(min(jb.trace_steps, static_cast<uint64_t>(0xFFFFFFFFu)))
                                   : 0u;
    int8_t* S = reinterpret_cast<int8_t*>(base);
    H* hf = reinterpret_cast<H*>(base + npad);
    uint2* ring = reinterpret_cast<uint2*>(base + ring_off(npad));
    uint4* b0w = reinterpret_cast<uint4*>(base + b0_off<T>(npad)) + 32 * warp;
    unsigned char* xch = base + xch_off<T>(npad);
    H* red = reinterpret_cast<H*>(xch);            // per warp: minimum dE of its slots
    W* tots = reinterpret_cast<W*>(xch + 16);      // per warp: total weight of its slots
    uint4* selw = reinterpret_cast<uint4*>(xch + 48);  // the choice: slot, site, spin at the site
    uint32_t next_rec = jb.record_every ? (t0 / jb.record_every + 1u) * jb.record_every : 0u;

    step::fill_block0<32>(b0w, t0 & ~31u, chain, c3, k0, k1, g);
    // sites: SL blocks per step (a power of two), SPB = NT / SL steps per batch
    uint32_t SL = 1, lg = 0;
    while (SL < nblk) {
        SL <<= 1;
        ++lg;
    }
    const uint32_t SPB = static_cast<uint32_t>(NT) >> lg;
    auto fill_ring = [&](uint32_t half, uint32_t tb) {
        const uint32_t b = 1u + (static_cast<uint32_t>(tid) & (SL - 1u));
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        if (b <= nblk) r = dev::philox4x32_10(make_uint4(b, tb + (static_cast<uint32_t>(tid) >> lg), chain, c3), k0, k1);
        ring[half * NT + tid] = make_uint2(__umulhi(r.x, N) | (__umulhi(r.y, N) << 16),
                                           __umulhi(r.z, N) | (__umulhi(r.w, N) << 16));
    };
    uint32_t tb = t0, half = 0;
    if constexpr (RULE == 0) fill_ring(0u, t0);
    (void)SPB;
    team_sync(bar, NT);

    for (uint32_t t = t0; t < t1; ++t) {
        const uint4 b0 = b0w[t & 31u];
        if (((t + 1u) & 31u) == 0u && t + 1u < t1) {  // the next 32 steps' block 0 (this warp's copy)
            __syncwarp();
            step::fill_block0<32>(b0w, t + 1u, chain, c3, k0, k1, g);
        }
        const unsigned long long U1 = (static_cast<unsigned long long>(b0.w) << 32) | b0.z;
        int sel = 0;    // slot chosen (Metropolis: accepted)
        int nflip = 0;  // spins flipped: x1 (c1 = 2 s_x1), x2 (c2 = 2 s_x2)
        int rows = 0;   // J rows the step needs: row a of a leaf root, flipped spins' rows
        uint32_t x1 = 0, x2 = 0;
        int c1 = 0, c2 = 0;
        if constexpr (RULE == 1) {
            // ---- Metropolis: one single-flip proposal ----
            const uint32_t i = __umulhi(b0.x, N);
            const int si = S[i];
            const H dE = static_cast<H>(2 * si) * hf[i];
            bool accept;
            if constexpr (sizeof(JT) == 1) {
                const uint32_t k = static_cast<uint32_t>(dE) >> 1;
                accept = dE <= 0 || (U1 >> 11) < step::wt_lookup(wsm, Wt, wlen, k);
            } else {
                accept = dE <= 0.0f || static_cast<float>(U1 >> 40) * 0x1p-24f < dev::pow2(nbl2 * dE);
            }
            if (accept) {
                sel = 1;
                nflip = 1;
                x1 = i;
                c1 = 2 * si;
            }
            rows = nflip;
        } else {
            // ---- MCMCMC: K proposals on the uniform-root star, slot d = tid + 1 ----
            uint32_t j = t - tb;
            if (j == SPB) {
                tb += SPB;
                half ^= 1u;
                j = 0;
            }
            if (j == 0) fill_ring(half ^ 1u, tb + SPB);  // the next batch, into the other half
            const uint2* rb = ring + half * NT + (j << lg);
            const uint2 e = rb[(static_cast<uint32_t>(tid) >> 2) & (SL - 1u)];
            const uint32_t wv = (tid & 2) ? e.y : e.x;
            const uint32_t i = (wv >> (16 * (tid & 1))) & 0xFFFFu;
            const uint32_t a = rb[0].x & 0xFFFFu;  // slot 1's site
            const unsigned long long U0 = (static_cast<unsigned long long>(b0.y) << 32) | b0.x;
            const bool leaf = U0 >= dev::at_use(jb.root_thr);
            const int sa = S[a];
            const H dEa = static_cast<H>(2 * sa) * hf[a];
            const uint32_t d = static_cast<uint32_t>(tid) + 1u;
            const int si = S[i];
            const H single = static_cast<H>(2 * si) * hf[i];
            // leaf root: the centre flipped at b = site_d (0 if b = a)
            const JT jab = __ldg(Jrow(a) + i);
            const H dbl = (i == a) ? H(0) : dEa + single - static_cast<H>(4 * sa * si) * static_cast<H>(jab);
            const H v = !leaf ? single : (d == 1u ? dEa : dbl);
            H mloc = 0;
            if (d <= K) mloc = mloc < v ? mloc : v;
            const H mw = step::gmin<true>(g, mloc);
            if (lane == 0) red[warp] = mw;
            team_sync(bar, NT);  // 1: the warps' minima
            H m = red[0];
#pragma unroll
            for (int w = 1; w < T; ++w) m = red[w] < m ? red[w] : m;
            // weights in slot order, exp(-beta (dE - m)) times the root factor
            W x = 0;
            if (d <= K) {
                const bool centre = leaf && d == 1u;
                if constexpr (sizeof(JT) == 1) {
                    x = step::wt_lookup(wsm, Wt, wlen, static_cast<uint32_t>(v - m) >> 1);
                    if (root_weighted)  // floor(x F / 2^20)
                        x = __umul64hi(x << 11, static_cast<unsigned long long>(centre ? jb.fcen : jb.fleaf) << 33);
                } else {
                    x = dev::pow2(fmaf(nbl2, v - m, centre ? jb.lcen : jb.lleaf));
                }
            }
            W w0;  // slot 0, the root: the centre of a centre root, else a leaf
            if constexpr (sizeof(JT) == 1) {
                w0 = step::wt_lookup(wsm, Wt, wlen, static_cast<uint32_t>(-m) >> 1);
                if (root_weighted)
                    w0 = __umul64hi(w0 << 11, static_cast<unsigned long long>(leaf ? jb.fleaf : jb.fcen) << 33);
            } else {
                w0 = dev::pow2(fmaf(-nbl2, m, leaf ? jb.lleaf : jb.lcen));
            }
            const W incl = step::gscan(g, x);
            if (lane == 31) tots[warp] = incl;
            team_sync(bar, NT);  // 2: the warps' totals
            W total = w0;
#pragma unroll
            for (int w = 0; w < T; ++w) total += tots[w];
            W u;
            if constexpr (sizeof(JT) == 1) {
                u = __umul64hi(U1, total);
            } else {
                u = static_cast<float>(U1 >> 40) * 0x1p-24f * total;
                if (u >= total) u = nextafterf(total, 0.0f);
            }
            if (!(u < w0)) {  // a slot d >= 1 (the same decision in every thread)
                // the warp whose range of prefixes holds u, its prefix offset
                W run = w0, pre = 0;
                int ws = T - 1;
                bool got = false;
#pragma unroll
                for (int w = 0; w < T; ++w) {
                    const W nx = run + tots[w];
                    if (!got && nx > u) {
                        ws = w;
                        pre = run;
                        got = true;
                    }
                    run = nx;
                }
                if (!got) pre = run - tots[T - 1];
                if (warp == ws) {
                    // the first lane whose prefix exceeds u; a rounding guard
                    // takes the last lane up to it with a positive weight
                    const unsigned over = __ballot_sync(kFull, pre + incl > u);
                    const int L0 = over ? __ffs(over) - 1 : 31;
                    const unsigned pos = __ballot_sync(kFull, x > W(0)) & ((2u << L0) - 1u);
                    const int L = pos ? 31 - __clz(pos) : 0;
                    const uint32_t sb = __shfl_sync(kFull, i, L);
                    const int ssb = __shfl_sync(kFull, si, L);
                    if (lane == 0)
                        *selw = make_uint4(pos ? static_cast<uint32_t>(32 * ws + L + 1) : 0u, sb,
                                           static_cast<uint32_t>(ssb), 0u);
                }
                team_sync(bar, NT);  // 3: the choice
                const uint4 sv = *selw;
                sel = static_cast<int>(sv.x);
                const uint32_t sel_site = sv.y;
                const int s_b = static_cast<int>(sv.z);
                if (sel != 0) {
                    if (!leaf) {
                        nflip = 1;
                        x1 = sel_site;
                        c1 = 2 * s_b;
                    } else if (sel == 1) {
                        nflip = 1;
                        x1 = a;
                        c1 = 2 * sa;
                    } else if (sel_site != a) {
                        nflip = 2;
                        x1 = a;
                        c1 = 2 * sa;
                        x2 = sel_site;
                        c2 = 2 * s_b;
                    }
                }
            }
            rows = leaf ? 1 + (nflip == 2 ? 1 : 0) : nflip;
        }
        // ---- field update and flips (the same decision in every thread) ----
        if (nflip) {
            // Metropolis steps that reject pass no barrier, so the team's
            // warps may be at different steps here: none writes before every
            // warp has reached this one (each has then read the state it
            // decides on).  MCMCMC is there already (barrier 3).
            if constexpr (RULE == 1) team_sync(bar, NT);
            team_update<JT, NT>(hf, Jrow(x1), Jrow(x2), c1, c2, npad, tid);
            if (tid == 0) {
                S[x1] = static_cast<int8_t>(-S[x1]);
                if (nflip == 2) S[x2] = static_cast<int8_t>(-S[x2]);
            }
            team_sync(bar, NT);  // 4: fields and spins of the next step
            acc += 1u;
        }
        n_flips += static_cast<uint32_t>(nflip);
        n_rows += static_cast<uint32_t>(rows);
        if (t < trace_end && tid == 0) jb.trace[static_cast<size_t>(chain) * jb.trace_steps + t] = sel;
        if (t + 1u == next_rec) {
            step::record<JT, RULE, 1, 32, false>(jb, write && warp == 0, chain, next_rec / jb.record_every - 1u, S,
                                                 hf, partner_off, acc, next_rec);
            acc = 0;
            next_rec += jb.record_every;
        }
    }
}

// The team kernel: persistent CTAs of `teams` (1 or 2) teams of T warps take
// work items (at most `teams` chains of one run) from the class's queue.  A
// team without a chain in the item meets the CTA's record barriers only.
template <typename JT, int RULE, int T>
__global__ void __launch_bounds__(64 * T, 1)
    team_kernel(const JobDev* __restrict__ jobs, const WorkItem* __restrict__ items, uint32_t n_items,
                uint32_t* __restrict__ queue, uint32_t nsteps, uint32_t per_chain) {
    constexpr int NT = 32 * T;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) JobDev s_job;
    __shared__ unsigned long long s_wt[sizeof(JT) == 1 ? kWCache : 1];
    __shared__ uint32_t s_item;
    const int team = static_cast<int>(threadIdx.x) / NT;
    const int tid = static_cast<int>(threadIdx.x) - team * NT;
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
        if constexpr (sizeof(JT) == 1) {  // the start of the +-J weight table (0 past its end)
            for (uint32_t i = threadIdx.x; i < kWCache; i += blockDim.x)
                s_wt[i] = i < jb.wlen ? reinterpret_cast<const unsigned long long*>(jb.W)[i] : 0ull;
        }
        const bool own = static_cast<uint32_t>(team) < wi.nchains;
        const uint32_t chain = wi.chain0 + (own ? static_cast<uint32_t>(team) : 0u);
        const uint32_t npad = jb.Npad;
        unsigned char* base = smem + static_cast<size_t>(team) * per_chain;
        const uint32_t t0 = static_cast<uint32_t>(*jb.step);
        const uint32_t t1 =
            static_cast<uint32_t>(min(static_cast<uint64_t>(t0) + nsteps, static_cast<uint64_t>(jb.step_limit)));
        uint32_t acc = 0, n_flips = 0, n_rows = 0;
        if (own) {  // the chain's spins (npad bytes) and fields (4 npad bytes)
            const uint4* gs = reinterpret_cast<const uint4*>(jb.s + static_cast<size_t>(chain) * npad);
            uint4* ss = reinterpret_cast<uint4*>(base);
            for (uint32_t k = tid; k < npad / 16; k += NT) ss[k] = gs[k];
            const uint4* gh =
                reinterpret_cast<const uint4*>(static_cast<const int*>(jb.h) + static_cast<size_t>(chain) * npad);
            uint4* sh = reinterpret_cast<uint4*>(base + npad);
            for (uint32_t k = tid; k < npad / 4; k += NT) sh[k] = gh[k];
            acc = jb.acc_run[chain];
        }
        __syncthreads();
        if (t1 > t0) {
            const int partner_off = (team & 1) ? -static_cast<int>(per_chain) : static_cast<int>(per_chain);
            if (own) {
                team_loop<JT, RULE, T>(jb, true, chain, base, partner_off, s_wt, t0, t1, acc, n_flips, n_rows, team);
            } else {
                const uint32_t R = jb.record_every;
                if (R)
                    for (uint32_t p = (t0 / R + 1u) * R, r = t0 / R; p <= t1; p += R, ++r)
                        step::record<JT, RULE, 1, 32, false>(jb, false, chain, r,
                                                             reinterpret_cast<const int8_t*>(base), base + npad,
                                                             partner_off, 0u, p);
            }
        }
        __syncthreads();
        if (own) {
            uint4* gs = reinterpret_cast<uint4*>(jb.s + static_cast<size_t>(chain) * npad);
            const uint4* ss = reinterpret_cast<const uint4*>(base);
            for (uint32_t k = tid; k < npad / 16; k += NT) gs[k] = ss[k];
            if (jb.s_op) {  // the spins as tensor-core operands for the next recompute
                const size_t base16 = static_cast<size_t>(chain) * (npad / 16);
                for (uint32_t k = tid; k < npad / 16; k += NT) dev::spins_to_op16(jb.s_op, base16 + k, ss[k], sizeof(JT) != 1);
            }
            uint4* gh = reinterpret_cast<uint4*>(static_cast<int*>(jb.h) + static_cast<size_t>(chain) * npad);
            const uint4* sh = reinterpret_cast<const uint4*>(base + npad);
            for (uint32_t k = tid; k < npad / 4; k += NT) gh[k] = sh[k];
            if (tid == 0) {
                jb.acc_run[chain] = acc;
                jb.work[2 * static_cast<size_t>(chain)] += n_flips;
                jb.work[2 * static_cast<size_t>(chain) + 1] += n_rows;
            }
        }
        __syncthreads();  // s_job and the slices are reused by the next item
    }
}

template <typename JT, int RULE, int T>
cudaError_t launch_variant(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                           uint32_t nsteps, uint32_t teams, uint32_t per_chain, uint32_t grid, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(per_chain) * teams;
    cudaError_t e = cudaFuncSetAttribute(team_kernel<JT, RULE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    team_kernel<JT, RULE, T><<<grid, 32 * T * teams, smem, st>>>(jobs, items, n_items, queue, nsteps, per_chain);
    return cudaGetLastError();
}

template <typename JT, int RULE, int T>
int occupancy_variant(uint32_t teams, uint32_t per_chain) {
    const size_t smem = static_cast<size_t>(per_chain) * teams;
    int n = 0;
    if (cudaFuncSetAttribute(team_kernel<JT, RULE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, team_kernel<JT, RULE, T>, 32 * T * teams, smem) !=
            cudaSuccess)
        return 0;
    return n;
}

// The variants of one coupling type: rule x T.
template <typename JT>
cudaError_t launch_kind(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                        uint32_t nsteps, uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain, uint32_t grid,
                        cudaStream_t st) {
    if (rule == 0)
        return T == 2 ? launch_variant<JT, 0, 2>(jobs, items, n_items, queue, nsteps, teams, per_chain, grid, st)
                      : launch_variant<JT, 0, 4>(jobs, items, n_items, queue, nsteps, teams, per_chain, grid, st);
    return T == 2 ? launch_variant<JT, 1, 2>(jobs, items, n_items, queue, nsteps, teams, per_chain, grid, st)
                  : launch_variant<JT, 1, 4>(jobs, items, n_items, queue, nsteps, teams, per_chain, grid, st);
}
template <typename JT>
int occupancy_kind(uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain) {
    if (rule == 0) return T == 2 ? occupancy_variant<JT, 0, 2>(teams, per_chain) : occupancy_variant<JT, 0, 4>(teams, per_chain);
    return T == 2 ? occupancy_variant<JT, 1, 2>(teams, per_chain) : occupancy_variant<JT, 1, 4>(teams, per_chain);
}

}  // namespace team
}  // namespace sk
