// sk_step.cuh -- the persistent MCMCMC / Metropolis step kernel.
//
// A chain is owned by a group of G lanes (G = 4, 8, 16 or 32; 32/G chains per
// warp).  Its spins s[Npad] (int8) and maintained local fields h[Npad] (int32
// for +-J, float for Gaussian couplings) stay in the chain's slice of shared
// memory for the whole launch, and the row of J that the next step needs
// first is bulk-copied (TMA, cp.async.bulk) into a double-buffered
// shared-memory slot one step ahead: the sites a step proposes do not depend
// on the chain's state.  Groups only talk to their own lanes (width-G
// shuffles under the group's lane mask), so the groups of a warp are
// independent chains.
//
// One Monte Carlo step (Sec. A.2, Eq. eq_det_balance_graph_solution, on the
// star of App. B.2 with a uniform root, p_r = 1/(K+1)):
//   a1  Philox4x32-10 draws, counter (block, step, chain, stream): block 0
//       gives U0 (root: a leaf iff U0 >= root_thr; for the uniform root
//       root_thr = ceil(2^64/(K+1)), i.e. floor(U0 (K+1) / 2^64) != 0) and
//       U1 (node);
//       blocks 1..ceil(K/4) give site_d = floor(w N / 2^32), d = 1..K.
//       Group lane l computes blocks 1 + l + G q for q < NB (NB blocks per
//       lane), so its slots are d = 4Gq + 4l + 1..4 (slot order is lane order
//       within a q, then q); block 0 is computed G steps at a time.  With
//       K <= 32 and one block per lane (16- and 32-lane groups), the blocks
//       of G/SL steps are drawn in one pass (draw_site_batch) and handed out
//       by shuffles, and whole-warp groups then hold one slot per lane,
//       d = l + 1 (take_site1): the same draws, hence the same choices.
//   a2  the row of J at a = site_1 of the NEXT step is staged by TMA.
//   a3  candidate energies: centre root dE_d = 2 s_i h_i (i = site_d);
//       leaf root dE_1 = 2 s_a h_a, dE_d = 2 s_a h_a + 2 s_b h_b - 4 J_ab s_a s_b
//       (b = site_d != a), 0 when b = a; slot 0 (the current state) is 0.
//   a4  node choice with probability ~ exp(-beta dE) p_r(slot): group min,
//       weights (+-J: integer table W[(dE-min)/2] ~ 2^52 exp(-2 beta d), times
//       F / 2^20 of the slot's root class when the root is not uniform;
//       Gaussian: 2^(-beta log2(e) (dE-min) + log2 f)), group inclusive scan
//       in slot order, u = U1 * total, first slot whose prefix exceeds u.
//   a5  field update for the 0, 1 or 2 flipped spins x: h_k -= 2 s_x J_kx.
//   a6  records every R steps: E = -scale/2 sum s h, accepted count, and the
//       overlap q of chain pairs (2m, 2m+1), which share a CTA.
// The Metropolis comparator (Sec. II / IV.B) shares the layout: one site per
// step from block 0, accept iff dE <= 0 or U < exp(-beta dE).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "sk_device.cuh"
#include "sk_internal.h"

namespace sk {
namespace step {

using dev::kFull;
using dev::sbyte;
using dev::Types;

// The G lanes of one chain inside a warp.
template <int G>
struct Grp {
    int gl;         // lane within the group
    int base;       // first warp lane of the group
    unsigned mask;  // the group's lanes
    __device__ __forceinline__ Grp() {
        const int lane = threadIdx.x & 31;
        gl = lane & (G - 1);
        base = lane & ~(G - 1);
        mask = G == 32 ? kFull : (((1u << G) - 1u) << base);
    }
};

template <int G, typename T>
__device__ __forceinline__ T gshfl(const Grp<G>& g, T v, int src) {
    return __shfl_sync(g.mask, v, src, G);
}
// Group minimum: log2(G) butterfly shuffles, or (REDUX) one warp reduction
// over the group's lanes (redux.sync; the groups of a warp reduce
// independently, each under its own mask).  The reduction is shorter on a
// lone chain's critical path but costs issue slots where many chains share an
// SM, so only the few-chain variant takes it.
template <bool REDUX, int G, typename T>
__device__ __forceinline__ T gmin(const Grp<G>& g, T v) {
    if constexpr (REDUX) {
        if constexpr (std::is_integral<T>::value) {
            return __reduce_min_sync(g.mask, v);
        } else {
            float r;
            asm volatile("redux.sync.min.f32 %0, %1, %2;" : "=f"(r) : "f"(v), "r"(g.mask));
            return r;
        }
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const T y = __shfl_xor_sync(g.mask, v, o, G);
            v = y < v ? y : v;
        }
        return v;
    }
}
template <int G, typename T>
__device__ __forceinline__ T gsum(const Grp<G>& g, T v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(g.mask, v, o, G);
    return v;
}
template <int G, typename T>
__device__ __forceinline__ T gscan(const Grp<G>& g, T v) {  // inclusive, in lane order
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        const T y = __shfl_up_sync(g.mask, v, o, G);
        if (g.gl >= o) v += y;
    }
    return v;
}
// The same scan over the group's first L lanes (L a power of two <= G): the
// levels whose offset reaches past them are left out.  Those lanes get the
// prefixes of the full scan bit for bit (a lane below L adds nothing at a
// left-out level); the lanes past them hold partial sums and must be ignored.
// Where the other lanes hold 0 and the values are integers, lane L-1 holds the
// group total exactly.
template <int L, int G, typename T>
__device__ __forceinline__ T gscan_first(const Grp<G>& g, T v) {
    static_assert(L <= G && (L & (L - 1)) == 0, "L: a power of two <= G");
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
        const T y = __shfl_up_sync(g.mask, v, o, G);
        if (g.gl >= o) v += y;
    }
    return v;
}
template <int G>
__device__ __forceinline__ unsigned gballot(const Grp<G>& g, bool p) {
    const unsigned b = __ballot_sync(g.mask, p);
    return G == 32 ? b : ((b >> g.base) & ((1u << G) - 1u));
}

// Shared memory of one chain: spins, fields, two staged J rows, two mbarriers.
struct ChainMem {
    int8_t* s;
    void* h;
    void* row[2];
    uint64_t* bar;
    uint4* b0;  // block 0 of G consecutive steps (kB0Bytes reserved)
    const unsigned long long* wsm;  // +-J: the first kWCache weight-table entries
};

// +-J weight-table entries held in shared memory per work item: at moderate
// beta the table is this short (W[d] ~ 2^52 e^{-2 beta d} rounds to 0 past
// d ~ 18/beta), and the lookups then cost a shared-memory load instead of a
// trip to L2; longer tables read the rest from global memory.
constexpr uint32_t kWCache = 64;
// SMALL: the whole table is in wsm (wlen <= kWCache, zeros past its end), and
// the lookup is compiled without the global-memory fallback.
template <bool SMALL = false>
__device__ __forceinline__ unsigned long long wt_lookup(const unsigned long long* wsm,
                                                        const unsigned long long* Wt, uint32_t wlen,
                                                        uint32_t idx) {
    if constexpr (SMALL) {
        (void)Wt;
        (void)wlen;
        return idx < kWCache ? wsm[idx] : 0ull;
    } else {
        return idx < kWCache ? wsm[idx] : (idx < wlen ? __ldg(&Wt[idx]) : 0ull);
    }
}

// Block 0 (U0, U1) of the G steps base .. base+G-1, computed one step per
// group lane into the chain's shared memory, where every lane of the group
// reads the block of its current step.  Steps are 32-bit.
template <int G>
__device__ __forceinline__ void fill_block0(uint4* b0s, uint32_t base, uint32_t chain, uint32_t c3, uint32_t k0,
                                            uint32_t k1, const Grp<G>& g) {
    b0s[g.gl] = dev::philox4x32_10(make_uint4(0u, base + g.gl, chain, c3), k0, k1);
    __syncwarp(g.mask);
}

// Sites of step t held by this lane: slots d = 4 G q + 4 gl + e + 1, two
// 16-bit sites per register (N <= 8192): site k is half k & 1 of sp[k >> 1].
template <int NB, int G>
__device__ __forceinline__ void draw_sites(uint32_t (&sp)[2 * NB], uint32_t t, uint32_t chain, uint32_t c3,
                                           uint32_t k0, uint32_t k1, uint32_t nblk, uint32_t N, const Grp<G>& g) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        const uint32_t b = 1u + static_cast<uint32_t>(G) * q + g.gl;
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        if (b <= nblk) r = dev::philox4x32_10(make_uint4(b, t, chain, c3), k0, k1);
        sp[2 * q + 0] = __umulhi(r.x, N) | (__umulhi(r.y, N) << 16);
        sp[2 * q + 1] = __umulhi(r.z, N) | (__umulhi(r.w, N) << 16);
    }
}
// Small-K chains (every slot in group lanes 0 .. SL-1, i.e. K <= 4 SL) draw
// the sites of G / SL steps at once, one Philox block per lane: lane l
// computes what lane l % SL of draw_sites computes for step tb + l / SL, and
// at each step a shuffle hands each lane the words of lane SL j + gl % SL
// (j = t - tb).  Lanes past SL-1 so get copies of real sites where
// draw_sites gives them zeros; their slots are past K, where the sites only
// serve as (in-range) indices of loads whose values are not used.
template <int SL, int G>
__device__ __forceinline__ void draw_site_batch(uint32_t (&bat)[2], uint32_t tb, uint32_t chain, uint32_t c3,
                                                uint32_t k0, uint32_t k1, uint32_t nblk, uint32_t N,
                                                const Grp<G>& g) {
    const uint32_t b = 1u + static_cast<uint32_t>(g.gl % SL);
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (b <= nblk) r = dev::philox4x32_10(make_uint4(b, tb + static_cast<uint32_t>(g.gl / SL), chain, c3), k0, k1);
    bat[0] = __umulhi(r.x, N) | (__umulhi(r.y, N) << 16);
    bat[1] = __umulhi(r.z, N) | (__umulhi(r.w, N) << 16);
}
template <int SL, int G>
__device__ __forceinline__ void take_sites(uint32_t (&sp)[2], const uint32_t (&bat)[2], uint32_t j, const Grp<G>& g) {
    const int src = static_cast<int>(j) * SL + (g.gl & (SL - 1));
    sp[0] = __shfl_sync(g.mask, bat[0], src, G);
    sp[1] = __shfl_sync(g.mask, bat[1], src, G);
}
// One slot per lane (slot d = gl + 1): lane gl takes site gl % 4 of what
// draw_sites gives lane gl / 4, i.e. of batch lane SL j + gl / 4 (lanes past
// 4 SL - 1, whose slots are past K, take in-range sites of the same step).
template <int SL, int G>
__device__ __forceinline__ void take_site1(uint32_t (&sp)[2], const uint32_t (&bat)[2], uint32_t j, const Grp<G>& g) {
    const int src = static_cast<int>(j) * SL + ((g.gl >> 2) & (SL - 1));
    const uint32_t w0 = __shfl_sync(g.mask, bat[0], src, G);
    const uint32_t w1 = __shfl_sync(g.mask, bat[1], src, G);
    const uint32_t w = (g.gl & 2) ? w1 : w0;
    sp[0] = (w >> (16 * (g.gl & 1))) & 0xFFFFu;
    sp[1] = 0u;
}
template <int NB>
__device__ __forceinline__ uint32_t site_of(const uint32_t (&sp)[2 * NB], int k) {
    return (sp[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
}

// h_k -= c1 J[x1][k] + c2 J[x2][k] for k < Npad (c2 = 0: one flip); lane gl
// owns elements 4 gl + 4 G v.  r1 is the staged row (shared memory) when
// STAGED, else a row of J in global memory; r2 is global and read only when
// c2 != 0.  Two forms:
//  - CHUNKED (the 128-register variant: few warps per SM, where a lone
//    chain waits for each round trip and an MCMCMC double flip reads two
//    rows): chunks of UNROLL iterations whose row loads are all issued
//    before any field of the chunk is read or written, so that a chunk costs
//    one round trip to L2 even when the first row is staged in shared memory
//    beside the fields (loads could not otherwise move past the stores);
//    without TWO (Metropolis) there is no second row;
//  - otherwise one loop unrolled UNROLL times: 2 where many chains per SM
//    hide each other's L2 latency within tight registers, 8 for Metropolis
//    in the 128-register variant when each lane's share of the row is a
//    multiple of 8 passes (otherwise the loop's remainder would take one
//    round trip per element, and the planner takes the chunked form).
// The terms are added in the same order either way (the first flip's, then
// the second's), so both give the same fields bit for bit.
template <typename JT, bool STAGED, int G, int UNROLL, bool CHUNKED, bool TWO = true>
__device__ __forceinline__ void update_fields(typename Types<JT>::H* hf, const JT* r1, const JT* r2, int c1,
                                              int c2, uint32_t npad, int gl) {
    if constexpr (CHUNKED) {
        constexpr uint32_t kStride = 4u * G;
        for (uint32_t k0 = 4u * gl; k0 < npad; k0 += kStride * UNROLL) {
            if constexpr (sizeof(JT) == 1) {
                uint32_t j1[UNROLL], j2[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const uint32_t k = k0 + kStride * u;
                    j1[u] = j2[u] = 0u;
                    if (k < npad) {
                        j1[u] = STAGED ? *reinterpret_cast<const uint32_t*>(r1 + k)
                                       : __ldg(reinterpret_cast<const unsigned int*>(r1 + k));
                        if (TWO && c2) j2[u] = __ldg(reinterpret_cast<const unsigned int*>(r2 + k));
                    }
                }
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const uint32_t k = k0 + kStride * u;
                    if (k < npad) {
                        int4 hv = *reinterpret_cast<int4*>(hf + k);
                        hv.x -= c1 * sbyte(j1[u], 0);
                        hv.y -= c1 * sbyte(j1[u], 1);
                        hv.z -= c1 * sbyte(j1[u], 2);
                        hv.w -= c1 * sbyte(j1[u], 3);
                        if (TWO && c2) {
                            hv.x -= c2 * sbyte(j2[u], 0);
                            hv.y -= c2 * sbyte(j2[u], 1);
                            hv.z -= c2 * sbyte(j2[u], 2);
                            hv.w -= c2 * sbyte(j2[u], 3);
                        }
                        *reinterpret_cast<int4*>(hf + k) = hv;
                    }
                }
            } else {
                float4 j1[UNROLL], j2[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const uint32_t k = k0 + kStride * u;
                    j1[u] = j2[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (k < npad) {
                        j1[u] = STAGED ? *reinterpret_cast<const float4*>(r1 + k)
                                       : __ldg(reinterpret_cast<const float4*>(r1 + k));
                        if (TWO && c2) j2[u] = __ldg(reinterpret_cast<const float4*>(r2 + k));
                    }
                }
                const float f1 = static_cast<float>(c1);
                const float f2 = static_cast<float>(c2);
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const uint32_t k = k0 + kStride * u;
                    if (k < npad) {
                        float4 hv = *reinterpret_cast<float4*>(hf + k);
                        hv.x = fmaf(-f1, j1[u].x, hv.x);
                        hv.y = fmaf(-f1, j1[u].y, hv.y);
                        hv.z = fmaf(-f1, j1[u].z, hv.z);
                        hv.w = fmaf(-f1, j1[u].w, hv.w);
                        if (TWO && c2) {
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
    } else {
#pragma unroll UNROLL
        for (uint32_t k = 4u * gl; k < npad; k += 4u * G) {
            if constexpr (sizeof(JT) == 1) {
                int4 hv = *reinterpret_cast<int4*>(hf + k);
                const uint32_t j1 = STAGED ? *reinterpret_cast<const uint32_t*>(r1 + k)
                                           : __ldg(reinterpret_cast<const unsigned int*>(r1 + k));
                hv.x -= c1 * sbyte(j1, 0);
                hv.y -= c1 * sbyte(j1, 1);
                hv.z -= c1 * sbyte(j1, 2);
                hv.w -= c1 * sbyte(j1, 3);
                if (c2) {
                    const uint32_t j2 = __ldg(reinterpret_cast<const unsigned int*>(r2 + k));
                    hv.x -= c2 * sbyte(j2, 0);
                    hv.y -= c2 * sbyte(j2, 1);
                    hv.z -= c2 * sbyte(j2, 2);
                    hv.w -= c2 * sbyte(j2, 3);
                }
                *reinterpret_cast<int4*>(hf + k) = hv;
            } else {
                float4 hv = *reinterpret_cast<float4*>(hf + k);
                const float4 j1 = STAGED ? *reinterpret_cast<const float4*>(r1 + k)
                                         : __ldg(reinterpret_cast<const float4*>(r1 + k));
                const float f1 = static_cast<float>(c1);
                hv.x = fmaf(-f1, j1.x, hv.x);
                hv.y = fmaf(-f1, j1.y, hv.y);
                hv.z = fmaf(-f1, j1.z, hv.z);
                hv.w = fmaf(-f1, j1.w, hv.w);
                if (c2) {
                    const float4 j2 = __ldg(reinterpret_cast<const float4*>(r2 + k));
                    const float f2 = static_cast<float>(c2);
                    hv.x = fmaf(-f2, j2.x, hv.x);
                    hv.y = fmaf(-f2, j2.y, hv.y);
                    hv.z = fmaf(-f2, j2.z, hv.z);
                    hv.w = fmaf(-f2, j2.w, hv.w);
                }
                *reinterpret_cast<float4*>(hf + k) = hv;
            }
        }
    }
}

// E = -scale/2 sum_k s_k h_k of the group's chain.
template <typename JT, int G>
__device__ __forceinline__ double chain_energy(const int8_t* S, const void* h, uint32_t npad, double scale,
                                               const Grp<G>& g) {
    if constexpr (sizeof(JT) == 1) {
        const int* hf = static_cast<const int*>(h);
        int acc = 0;
        for (uint32_t k = 4u * g.gl; k < npad; k += 4u * G) {
            const uint32_t sw = *reinterpret_cast<const uint32_t*>(S + k);
            const int4 hv = *reinterpret_cast<const int4*>(hf + k);
            acc += sbyte(sw, 0) * hv.x + sbyte(sw, 1) * hv.y + sbyte(sw, 2) * hv.z + sbyte(sw, 3) * hv.w;
        }
        const int tot = gsum(g, acc);  // = 2 sum_{i<j} J s s, even
        return scale * static_cast<double>(-(tot / 2));
    } else {
        // each lane sums its npad/G terms s_k h_k in fp32 (the products are
        // exact; relative rounding ~ (npad/G) 2^-24), the lanes' partial sums
        // are combined in double precision (FP64 is slow on this part)
        const float* hf = static_cast<const float*>(h);
        float acc = 0.0f;
        for (uint32_t k = 4u * g.gl; k < npad; k += 4u * G) {
            const uint32_t sw = *reinterpret_cast<const uint32_t*>(S + k);
            const float4 hv = *reinterpret_cast<const float4*>(hf + k);
            acc = fmaf(static_cast<float>(sbyte(sw, 0)), hv.x, acc);
            acc = fmaf(static_cast<float>(sbyte(sw, 1)), hv.y, acc);
            acc = fmaf(static_cast<float>(sbyte(sw, 2)), hv.z, acc);
            acc = fmaf(static_cast<float>(sbyte(sw, 3)), hv.w, acc);
        }
        return -0.5 * scale * gsum(g, static_cast<double>(acc));
    }
}

// Candidate energies of the star (a3): dE[q] of this lane's slots d =
// 4 G (q/4) + 4 gl + (q%4) + 1 (slots past K excluded from the minimum), a =
// site_1 (the centre's flip of a leaf root); returns the group minimum of dE
// over the K+1 slots (slot 0 has dE = 0).
template <typename JT, int NB, int G, bool STAGED>
__device__ __forceinline__ typename Types<JT>::H star_energies(const int8_t* S, const typename Types<JT>::H* hf,
                                                               const JT* rowA, const uint32_t (&site)[2 * NB],
                                                               bool leaf, uint32_t K, const Grp<G>& g,
                                                               typename Types<JT>::H (&dE)[4 * NB], uint32_t& a) {
    using H = typename Types<JT>::H;
    a = gshfl(g, site[0], 0) & 0xFFFFu;
    const int sa = S[a];
    const H dEa = static_cast<H>(2 * sa) * hf[a];
    H mloc = 0;
#pragma unroll
    for (int q = 0; q < 4 * NB; ++q) {
        const uint32_t d = 4u * G * (q >> 2) + 4u * g.gl + (q & 3) + 1u;
        const uint32_t i = site_of<NB>(site, q);
        const int si = S[i];
        const H hi = hf[i];
        const H single = static_cast<H>(2 * si) * hi;
        // leaf root: the centre flipped at b = site_d (0 if b = a)
        const JT jab = STAGED ? rowA[i] : __ldg(rowA + i);
        const H dbl = (i == a) ? H(0) : dEa + single - static_cast<H>(4 * sa * si) * static_cast<H>(jab);
        const H v = !leaf ? single : (d == 1u ? dEa : dbl);
        dE[q] = v;
        if (d <= K) mloc = mloc < v ? mloc : v;
    }
    return gmin<false>(g, mloc);
}

// Weight of a slot with candidate energy dEq (a4): exp(-beta (dEq - m)) times
// its root factor (`centre`: the centre slot, else a leaf).  +-J: the integer
// table (0 past its end), times F / 2^20 when the root is not uniform;
// Gaussian: 2^(-beta log2(e) (dEq - m) + log2 f).
template <typename JT>
__device__ __forceinline__ typename Types<JT>::W slot_weight(const JobDev& jb, const uint64_t* Wt, uint32_t wlen,
                                                             typename Types<JT>::H dEq, typename Types<JT>::H m,
                                                             bool centre, float nbl2, bool root_weighted) {
    typename Types<JT>::W x;
    if constexpr (sizeof(JT) == 1) {
        const uint32_t idx = static_cast<uint32_t>(dEq - m) >> 1;
        x = idx < wlen ? __ldg(&Wt[idx]) : 0ull;
        if (root_weighted)  // floor(x F / 2^20)
            x = __umul64hi(x << 11, static_cast<unsigned long long>(centre ? jb.fcen : jb.fleaf) << 33);
    } else {
        (void)Wt;
        (void)wlen;
        x = dev::pow2(fmaf(nbl2, dEq - m, centre ? jb.lcen : jb.lleaf));
    }
    return x;
}

// Node-weighted energy change of the graph that step t generates from the
// chain's current state (Eq. eq_monte_carlo_graph), without taking the step:
// sum_j P_node(j) dE_j over its K+1 slots with the weights the step chooses
// with (Metropolis: p_acc dE of its proposal).  The draws are those of step
// t (Philox again), so the step loop carries nothing for it.
template <typename JT, int RULE, int NB, int G>
__device__ __forceinline__ double graph_mean_dE(const JobDev& jb, uint32_t chain, uint32_t t, const int8_t* S,
                                                const typename Types<JT>::H* hf, const Grp<G>& g) {
    using H = typename Types<JT>::H;
    using W = typename Types<JT>::W;
    const uint32_t N = jb.N, K = jb.K;
    const uint32_t k0 = static_cast<uint32_t>(jb.seed), k1 = static_cast<uint32_t>(jb.seed >> 32);
    const uint32_t c3 = jb.stream & 0xFFFFFFu;
    const float nbl2 = -jb.beta_eff * 1.4426950408889634f;
    const uint64_t* Wt = static_cast<const uint64_t*>(jb.W);
    const uint4 b0 = dev::philox4x32_10(make_uint4(0u, t, chain, c3), k0, k1);
    if constexpr (RULE == 1) {
        const uint32_t i = __umulhi(b0.x, N);
        const H dE = static_cast<H>(2 * S[i]) * hf[i];
        double pacc = 1.0;
        if (dE > H(0)) {
            if constexpr (sizeof(JT) == 1) {
                const uint32_t k = static_cast<uint32_t>(dE) >> 1;
                pacc = k < jb.wlen ? static_cast<double>(__ldg(&Wt[k])) * 0x1p-53 : 0.0;
            } else {
                pacc = static_cast<double>(dev::pow2(nbl2 * dE));
            }
        }
        return pacc * static_cast<double>(dE);
    } else {
        const unsigned long long U0 = (static_cast<unsigned long long>(b0.y) << 32) | b0.x;
        const bool leaf = U0 >= jb.root_thr;
        const bool root_weighted = jb.fcen + jb.fleaf != (2u << 20);
        uint32_t site[2 * NB];
        draw_sites<NB, G>(site, t, chain, c3, k0, k1, (K + 3u) >> 2, N, g);
        const uint32_t a0 = gshfl(g, site[0], 0) & 0xFFFFu;
        const JT* rowA = static_cast<const JT*>(jb.J) + static_cast<size_t>(a0) * jb.Npad;
        H dE[4 * NB];
        uint32_t a;
        const H m = star_energies<JT, NB, G, false>(S, hf, rowA, site, leaf, K, g, dE, a);
        double num = 0.0, den = 0.0;
#pragma unroll
        for (int q = 0; q < 4 * NB; ++q) {
            const uint32_t d = 4u * G * (q >> 2) + 4u * g.gl + (q & 3) + 1u;
            if (d <= K) {
                const W x = slot_weight<JT>(jb, Wt, jb.wlen, dE[q], m, leaf && d == 1u, nbl2, root_weighted);
                num += static_cast<double>(x) * static_cast<double>(dE[q]);
                den += static_cast<double>(x);
            }
        }
        const W w0 = slot_weight<JT>(jb, Wt, jb.wlen, H(0), m, !leaf, nbl2, root_weighted);  // slot 0
        return gsum(g, num) / (gsum(g, den) + static_cast<double>(w0));
    }
}

// Record point shared by every thread of the CTA (two CTA barriers).  Only
// `write` groups (real chains, not shadows) read their slices and store:
// groups without a chain may have no slice of their own (the fused launch
// sizes its shared memory for the item's chains only).
template <typename JT, int RULE, int NB, int G, bool NWR>
__device__ __noinline__ void record(const JobDev& jb, bool write, uint32_t chain, uint32_t rec, const int8_t* S,
                                    const void* h, int partner_off, uint32_t acc, uint32_t t_next) {
    const Grp<G> g;
    const int8_t* partner_s = S + partner_off;
    const bool store = write && rec < jb.rec_capacity;
    const double E = write ? chain_energy<JT, G>(S, h, jb.Npad, jb.scale, g) : 0.0;
    // node-weighted energy of this state with the graph of the next step
    // (kernels built for runs that record it; groups without a chain skip it)
    double dm = 0.0;
    if constexpr (NWR) {
        if (store)
            dm = graph_mean_dE<JT, RULE, NB, G>(jb, chain, t_next, S, static_cast<const typename Types<JT>::H*>(h), g);
    }
    (void)t_next;
    if (store && g.gl == 0) {
        jb.rec_E[static_cast<size_t>(rec) * jb.chains + chain] = E;
        jb.rec_acc[static_cast<size_t>(rec) * jb.chains + chain] = acc;
        if (NWR) jb.rec_Enw[static_cast<size_t>(rec) * jb.chains + chain] = E + jb.scale * dm;
    }
    __syncthreads();
    if (write && (chain & 1u) == 0u && chain + 1u < jb.chains) {
        int dot = 0;
        for (uint32_t k = 4u * g.gl; k < jb.Npad; k += 4u * G) {
            const uint32_t a = *reinterpret_cast<const uint32_t*>(S + k);
            const uint32_t b = *reinterpret_cast<const uint32_t*>(partner_s + k);
            dot += sbyte(a, 0) * sbyte(b, 0) + sbyte(a, 1) * sbyte(b, 1) + sbyte(a, 2) * sbyte(b, 2) +
                   sbyte(a, 3) * sbyte(b, 3);
        }
        dot = gsum(g, dot);
        if (store && g.gl == 0)
            jb.rec_q[static_cast<size_t>(rec) * (jb.chains / 2) + chain / 2] =
                static_cast<double>(dot) / static_cast<double>(jb.N);
    }
    __syncthreads();
}

// Steps t0..t1-1 of one chain (or of a shadow: a group without a chain of
// its own in a partly filled warp runs a copy of a real chain and stores
// nothing, so that every lane reaches the same barriers).  `dead` is set
// after a timed-out wait: the group then stops working but still meets the
// CTA's record barriers.
// FAST (+-J work items only): every chain of the item has the uniform root,
// no traced steps and a weight table held whole in shared memory, and the loop
// is compiled without the code for the other cases (about 10 % of a lone
// chain's step).  SL > 0 (MCMCMC with K <= 4 SL and one block per lane in
// the few-chain variant, or in 16-lane and whole-warp chains of the others;
// rows through L1): the sites come in batches of G / SL steps (draw_site_batch; whole-warp
// chains hold one slot per lane), and for +-J the slot-weight scan covers
// only the lanes that hold slots (the integer total is the same in any order).
template <typename JT, int RULE, int NB, int G, int STAGE, int UNROLL, bool RCH, bool FAST = false, int SL = 0>
__device__ __forceinline__ void chain_loop(const JobDev& jb, bool write, uint32_t chain, const ChainMem& cm,
                                           int partner_off, uint32_t t0, uint32_t t1, uint32_t& acc,
                                           uint32_t& phase, bool& dead, uint32_t& n_flips, uint32_t& n_rows) {
    using H = typename Types<JT>::H;
    using W = typename Types<JT>::W;
    constexpr bool STAGED = STAGE == 1;  // 0: rows through L1, 2: the same with node-weighted records
    constexpr bool NWR = STAGE == 2;
    // the 128-register variant (few warps per SM, where one chain's step is a
    // chain of latencies) keeps the slot weights in registers for the node
    // search and draws the next step's sites during the current step
    constexpr bool KEEPW = UNROLL >= 8;
    constexpr bool AHEAD = STAGED || KEEPW;
    // staged rows in the few-chain variant: sites drawn two steps ahead, so
    // that the copy of the next step's row goes out at the start of a step
    // with no Philox rounds in front of it
    constexpr bool AHEAD2 = STAGED && KEEPW && RULE == 0;
    constexpr bool BATCH = SL > 0;                     // sites in batches of SPB steps
    constexpr bool SCANSL = BATCH && sizeof(JT) == 1;  // +-J: the scan over SL lanes
    static_assert(!BATCH || (RULE == 0 && NB == 1 && !STAGED && (SL & (SL - 1)) == 0 && G >= 2 * SL),
                  "site batches: MCMCMC with one block per lane, rows through L1");
    constexpr uint32_t SPB = BATCH ? G / SL : 1;
    // whole-warp groups with site batches hold one slot per lane (slot
    // d = lane + 1, K <= 32), so that a step's candidate work is one slot
    // deep instead of four; their +-J scan covers the first 4 SL lanes
    constexpr bool SPL1 = BATCH && G == 32;
    // the slot weights are kept for the node search also in the throughput
    // variants with two Philox blocks per lane (their register budget holds
    // the 8 weights without spills there; a recomputation costs 4 exponentials
    // and their lookups in the owning lanes of every group) and with one slot
    // per lane (one weight)
    constexpr bool KEEPXS = KEEPW || NB == 2 || SPL1;
    constexpr int NQ = SPL1 ? 1 : 4 * NB;  // slots per lane
    constexpr int SCANL = SPL1 ? (4 * SL < G ? 4 * SL : G) : (SL > 0 ? SL : 1);
    const Grp<G> g;
    // next record point (0: none; a record follows step t when t + 1 == next_rec)
    uint32_t next_rec = jb.record_every ? (t0 / jb.record_every + 1u) * jb.record_every : 0u;
    // job parameters held in registers for the whole loop
    const uint32_t N = jb.N, npad = jb.Npad, K = jb.K;
    const uint32_t nblk = (K + 3u) >> 2;
    const uint32_t k0 = static_cast<uint32_t>(jb.seed), k1 = static_cast<uint32_t>(jb.seed >> 32);
    const uint32_t c3 = jb.stream & 0xFFFFFFu;  // domain 0: step draws
    // row r of J (the base pointer is re-read from the job descriptor at each use)
    auto Jrow = [&](uint32_t r) -> const JT* {
        return static_cast<const JT*>(dev::at_use(jb.J)) + static_cast<size_t>(r) * npad;
    };
    const uint32_t rowbytes = npad * static_cast<uint32_t>(sizeof(JT));
    const W* __restrict__ Wt = reinterpret_cast<const W*>(jb.W);
    const uint32_t wlen = jb.wlen;
    const float nbl2 = -jb.beta_eff * 1.4426950408889634f;  // -beta log2(e)
    const bool root_weighted = !FAST && jb.fcen + jb.fleaf != (2u << 20);  // not both factors 1
    // steps this chain logs its choice for (0: not traced)
    const uint32_t trace_end = (!FAST && write && chain < jb.trace_chains)
                                   ? static_cast<uint32_t>(min(jb.trace_steps, static_cast<uint64_t>(0xFFFFFFFFu)))
                                   : 0u;
    int8_t* S = cm.s;
    H* hf = static_cast<H*>(cm.h);

    fill_block0<G>(cm.b0, t0 & ~static_cast<uint32_t>(G - 1), chain, c3, k0, k1, g);
    uint32_t site[2 * NB];  // packed sites of this step (site_of)
    uint32_t site1[AHEAD2 ? 2 * NB : 1];  // AHEAD2: the sites of the next step

    uint32_t bat[2];      // BATCH: this lane's words of the site batch of steps tb .. tb+SPB-1
    uint32_t tb = t0;
    if constexpr (BATCH) {
        draw_site_batch<SL, G>(bat, tb, chain, c3, k0, k1, nblk, N, g);
        if constexpr (SPL1)
            take_site1<SL, G>(site, bat, 0u, g);
        else
            take_sites<SL, G>(site, bat, 0u, g);
    } else if constexpr (!STAGED && AHEAD && RULE == 0) {
        draw_sites<NB, G>(site, t0, chain, c3, k0, k1, nblk, N, g);
    }
    (void)SPB;
    (void)tb;
    // prologue (staged rows): draw the first step and stage its row
    if constexpr (STAGED) {
        uint32_t first;
        if constexpr (RULE == 0) {
            draw_sites<NB, G>(site, t0, chain, c3, k0, k1, nblk, N, g);
            first = gshfl(g, site[0], 0) & 0xFFFFu;
            if constexpr (AHEAD2) draw_sites<NB, G>(site1, t0 + 1u, chain, c3, k0, k1, nblk, N, g);
        } else {
            first = __umulhi(cm.b0[t0 & (G - 1)].x, N);
        }
        // (a test of the bounded wait may withhold chain 0's first copy)
        const bool withhold = (jb.fault & kFaultWithholdRow) && chain == 0u && t0 == 0u;
        if (g.gl == 0 && !dead && !withhold) {
            dev::fence_proxy_async();
            dev::bulk_load(cm.row[t0 & 1u], Jrow(first), rowbytes, &cm.bar[t0 & 1u]);
        }
    }
    (void)rowbytes;

    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t buf = t & 1u;
        const uint4 b0 = cm.b0[t & (G - 1)];
        if (((t + 1u) & (G - 1)) == 0u && t + 1u < t1) {  // the next G steps' block 0
            __syncwarp(g.mask);  // every lane has read this step's entry
            fill_block0<G>(cm.b0, t + 1u, chain, c3, k0, k1, g);
        }
        const unsigned long long U1 = (static_cast<unsigned long long>(b0.w) << 32) | b0.z;
        int sel = 0;  // slot chosen (Metropolis: accepted)
        int nflip = 0;
        int rows = 0;  // J rows this step needs: row a of a leaf root, flipped spins' rows
        uint32_t x1 = 0, x2 = 0;
        bool x1_staged = false;

        // direct rows: this step's sites now; staged rows: the next step's
        // sites and the TMA of its first row, one step ahead
        if constexpr (BATCH && !AHEAD) {  // this step's sites out of the batch
            uint32_t j = t - tb;
            if (j == SPB) {
                tb += SPB;
                j = 0;
                draw_site_batch<SL, G>(bat, tb, chain, c3, k0, k1, nblk, N, g);
            }
            if constexpr (SPL1)
                take_site1<SL, G>(site, bat, j, g);
            else
                take_sites<SL, G>(site, bat, j, g);
        } else if constexpr (!AHEAD && RULE == 0) {
            draw_sites<NB, G>(site, t, chain, c3, k0, k1, nblk, N, g);
        }
        uint32_t nsite[2 * NB];
        if (STAGED && t + 1u < t1) {
            uint32_t nx;
            if constexpr (AHEAD2) {
                nx = gshfl(g, site1[0], 0) & 0xFFFFu;
            } else if constexpr (RULE == 0) {
                draw_sites<NB, G>(nsite, t + 1u, chain, c3, k0, k1, nblk, N, g);
                nx = gshfl(g, nsite[0], 0) & 0xFFFFu;
            } else {
                nx = __umulhi(cm.b0[(t + 1u) & (G - 1)].x, N);
            }
            if constexpr (STAGED) {
                __syncwarp(g.mask);  // every lane of the group is done with buffer buf^1 (step t-1)
                if (g.gl == 0 && !dead) {
                    dev::fence_proxy_async();
                    dev::bulk_load(cm.row[buf ^ 1u], Jrow(nx), rowbytes, &cm.bar[buf ^ 1u]);
                }
            }
            (void)nx;
        }
        if (STAGED && !dead) {
            // every lane waits; the outcome is made group-uniform
            const uint32_t par = (phase >> buf) & 1u;
            const bool okl = dev::mbar_wait_bounded(&cm.bar[buf], par);
            const bool ok = gballot(g, okl) == (G == 32 ? kFull : ((1u << G) - 1u));
            phase ^= 1u << buf;
            if (!ok) {
                dead = true;
                if (g.gl == 0) atomicExch(jb.err, kDevTimeout);
                // let this group's copies in flight land before it can leave
                // the kernel (each wait again bounded): the row just waited
                // for and the next step's row, issued before the wait
                dev::mbar_wait_bounded(&cm.bar[buf], par);
                if (t + 1u < t1) dev::mbar_wait_bounded(&cm.bar[buf ^ 1u], (phase >> (buf ^ 1u)) & 1u);
                __syncwarp(g.mask);
            }
        }
        // row a of this step: staged in shared memory, or read through L1 from J
        const JT* rowA;
        if constexpr (STAGED) {
            rowA = static_cast<const JT*>(cm.row[buf]);
        } else {
            const uint32_t a0 = RULE == 0 ? (gshfl(g, site[0], 0) & 0xFFFFu) : __umulhi(b0.x, N);
            rowA = Jrow(a0);
        }

        if (!dead) {
            if constexpr (RULE == 1) {
                // ---- Metropolis: one single-flip proposal ----
                const uint32_t i = __umulhi(b0.x, N);
                const int si = S[i];
                const H dE = static_cast<H>(2 * si) * hf[i];
                bool accept;
                if constexpr (sizeof(JT) == 1) {
                    const uint32_t k = static_cast<uint32_t>(dE) >> 1;
                    accept = dE <= 0 || (U1 >> 11) < wt_lookup<FAST>(cm.wsm, Wt, wlen, k);
                } else {
                    accept = dE <= 0.0f || static_cast<float>(U1 >> 40) * 0x1p-24f < dev::pow2(nbl2 * dE);
                }
                sel = accept ? 1 : 0;
                if (accept) {
                    nflip = 1;
                    x1 = i;
                    x1_staged = true;
                }
                rows = nflip;
            } else {
                // ---- MCMCMC: K proposals on the uniform-root star ----
                // (few-chain variant: the next step's sites, interleaved with this step's work)
                if constexpr (BATCH && AHEAD) {
                    uint32_t j = t + 1u - tb;
                    if (j == SPB) {
                        tb += SPB;
                        j = 0;
                        draw_site_batch<SL, G>(bat, tb, chain, c3, k0, k1, nblk, N, g);
                    }
                    if constexpr (SPL1)
                        take_site1<SL, G>(nsite, bat, j, g);
                    else
                        take_sites<SL, G>(nsite, bat, j, g);
                } else if constexpr (!STAGED && AHEAD) {
                    draw_sites<NB, G>(nsite, t + 1u, chain, c3, k0, k1, nblk, N, g);
                }
                if constexpr (AHEAD2) draw_sites<NB, G>(nsite, t + 2u, chain, c3, k0, k1, nblk, N, g);
                const unsigned long long U0 = (static_cast<unsigned long long>(b0.y) << 32) | b0.x;
                const bool leaf = U0 >= dev::at_use(jb.root_thr);
                const uint32_t a = gshfl(g, site[0], 0) & 0xFFFFu;
                const int sa = S[a];
                const H dEa = static_cast<H>(2 * sa) * hf[a];
                // slot of this lane's entry q
                auto slot_d = [&](int q) -> uint32_t {
                    return SPL1 ? static_cast<uint32_t>(g.gl) + 1u
                                : 4u * G * (q >> 2) + 4u * g.gl + static_cast<uint32_t>(q & 3) + 1u;
                };
                H dE[4 * NB];
                H mloc = 0;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const uint32_t d = slot_d(q);
                    const uint32_t i = SPL1 ? site[0] : site_of<NB>(site, q);
                    const int si = S[i];
                    const H hi = hf[i];
                    const H single = static_cast<H>(2 * si) * hi;
                    // leaf root: the centre flipped at b = site_d (0 if b = a)
                    const JT jab = STAGED ? rowA[i] : __ldg(rowA + i);
                    const H dbl = (i == a) ? H(0) : dEa + single - static_cast<H>(4 * sa * si) * static_cast<H>(jab);
                    const H v = !leaf ? single : (d == 1u ? dEa : dbl);
                    dE[q] = v;
                    if (d <= K) mloc = mloc < v ? mloc : v;
                }
                const H m = gmin<KEEPW>(g, mloc);
                // weights in slot order: exp(-beta (dE - m)) times the slot's
                // root factor (the centre: slot 1 of a leaf root, slot 0 of a
                // centre root); recomputed, not stored, where the choice needs them
                auto slot_w = [&](int q) -> W {
                    const uint32_t d = slot_d(q);
                    W x = 0;
                    const bool centre = leaf && d == 1u;
                    if (d <= K) {
                        if constexpr (sizeof(JT) == 1) {
                            const uint32_t idx = static_cast<uint32_t>(dE[q] - m) >> 1;
                            x = wt_lookup<FAST>(cm.wsm, Wt, wlen, idx);
                            if (root_weighted)  // floor(x F / 2^20)
                                x = __umul64hi(x << 11, static_cast<unsigned long long>(centre ? jb.fcen : jb.fleaf) << 33);
                        } else {
                            x = dev::pow2(fmaf(nbl2, dE[q] - m, centre ? jb.lcen : jb.lleaf));
                        }
                    }
                    return x;
                };
                W gsum_[NB];
                W xs[KEEPXS ? 4 * NB : 1];
#pragma unroll
                for (int q = 0; q < NB; ++q) gsum_[q] = 0;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const W xq = slot_w(q);
                    if constexpr (KEEPXS) xs[q] = xq;
                    gsum_[q >> 2] += xq;
                }
                W w0;  // slot 0, the root: the centre of a centre root, else a leaf
                if constexpr (sizeof(JT) == 1) {
                    const uint32_t idx0 = static_cast<uint32_t>(-m) >> 1;
                    w0 = wt_lookup<FAST>(cm.wsm, Wt, wlen, idx0);
                    if (root_weighted)
                        w0 = __umul64hi(w0 << 11, static_cast<unsigned long long>(leaf ? jb.fleaf : jb.fcen) << 33);
                } else {
                    w0 = dev::pow2(fmaf(-nbl2, m, leaf ? jb.lleaf : jb.lcen));
                }
                W incl[NB], tot[NB];
                W total = w0;
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    if constexpr (SCANSL) {  // slots in lanes 0 .. SCANL-1 only
                        incl[q] = gscan_first<SCANL>(g, gsum_[q]);
                        tot[q] = gshfl(g, incl[q], SCANL - 1);
                    } else {
                        incl[q] = gscan(g, gsum_[q]);
                        tot[q] = gshfl(g, incl[q], G - 1);
                    }
                    total += tot[q];
                }
                W u;
                if constexpr (sizeof(JT) == 1) {
                    u = __umul64hi(U1, total);
                } else {
                    u = static_cast<float>(U1 >> 40) * 0x1p-24f * total;
                    if (u >= total) u = nextafterf(total, 0.0f);
                }
                // first slot whose inclusive prefix exceeds u; the owning
                // lane finds its entry (else, a rounding guard, its last
                // positive weight), one packed shuffle broadcasts it
                int sel_d = 0;
                uint32_t sel_site = 0;
                bool found = u < w0;
                W base = w0;
                if constexpr (SPL1) {
                    // the first lane whose prefix exceeds u; a rounding guard
                    // takes the last lane up to it with a positive weight
                    if (!found) {
                        const unsigned over = gballot(g, base + incl[0] > u && (!SCANSL || g.gl < SCANL));
                        const int L0 = over ? __ffs(over) - 1 : G - 1;
                        const unsigned pos = gballot(g, xs[0] > W(0)) & ((2u << L0) - 1u);
                        if (pos) {
                            const int L = 31 - __clz(pos);
                            sel_site = gshfl(g, site[0], L) & 0xFFFFu;
                            sel_d = L + 1;
                            found = true;
                        }
                    }
                }
                // Gaussian weights with several blocks per lane: all blocks'
                // ballots first (a block's only where no earlier one holds u),
                // then one search in the block that does, so that the groups of
                // a warp search together even when their draws fall in
                // different blocks (for the 64-bit +-J weights the selects cost
                // more than the second pass they save)
                constexpr bool ONESEARCH = KEEPXS && !SPL1 && NB > 1 && sizeof(JT) == 4;
                if constexpr (ONESEARCH) {
                    unsigned ballq[NB];
                    W baseq[NB];
                    bool prior = false;
#pragma unroll
                    for (int q = 0; q < NB; ++q) {
                        ballq[q] = gballot(g, !found && !prior && base + incl[q] > u);
                        baseq[q] = base;
                        prior = prior || ballq[q] != 0u;
                        base += tot[q];
                    }
                    if (!found && prior) {
                        int qf = 0;
                        unsigned ball = 0;
                        W bse = 0, inc = 0;
                        W x[4];
#pragma unroll
                        for (int q = NB - 1; q >= 0; --q)
                            if (ballq[q]) {
                                qf = q;
                                ball = ballq[q];
                                bse = baseq[q];
                                inc = incl[q];
                            }
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            x[e] = xs[e];
#pragma unroll
                            for (int q = 1; q < NB; ++q)
                                if (q == qf) x[e] = xs[4 * q + e];
                        }
                        const int L = __ffs(ball) - 1;
                        W mine = 0;
#pragma unroll
                        for (int e = 0; e < 4; ++e) mine += x[e];
                        W run = bse + (inc - mine);
                        int my_e = -1, last_pos = -1;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (x[e] > W(0)) {
                                last_pos = e;
                                if (my_e < 0) {
                                    run += x[e];
                                    if (run > u) my_e = e;
                                }
                            }
                        }
                        if (my_e < 0) my_e = last_pos;
                        uint32_t my_site = 0;
#pragma unroll
                        for (int q = 0; q < NB; ++q)
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (q == qf && e == my_e) my_site = site_of<NB>(site, 4 * q + e);
                        const uint32_t packed = gshfl(g, (my_site << 2) | static_cast<uint32_t>(my_e & 3), L);
                        sel_site = packed >> 2;
                        sel_d = 4 * G * qf + 4 * L + static_cast<int>(packed & 3u) + 1;
                        found = true;
                    }
                }
#pragma unroll
                for (int q = 0; q < ((SPL1 || ONESEARCH) ? 0 : NB); ++q) {
                    const unsigned ball =
                        gballot(g, !found && base + incl[q] > u && (!SCANSL || g.gl < SCANL));
                    if (!found && ball) {
                        const int L = __ffs(ball) - 1;
                        // this lane's 4 weights (kept, or recomputed bit-identically),
                        // their sum in the order of the first pass
                        W x[4];
                        W mine = 0;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if constexpr (KEEPXS)
                                x[e] = xs[4 * q + e];
                            else
                                x[e] = slot_w(4 * q + e);
                            mine += x[e];
                        }
                        W run = base + (incl[q] - mine);
                        int my_e = -1, last_pos = -1;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (x[e] > W(0)) {
                                last_pos = e;
                                if (my_e < 0) {
                                    run += x[e];
                                    if (run > u) my_e = e;
                                }
                            }
                        }
                        if (my_e < 0) my_e = last_pos;
                        uint32_t my_site = 0;
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (e == my_e) my_site = site_of<NB>(site, 4 * q + e);
                        const uint32_t packed = gshfl(g, (my_site << 2) | static_cast<uint32_t>(my_e & 3), L);
                        sel_site = packed >> 2;
                        sel_d = 4 * G * q + 4 * L + static_cast<int>(packed & 3u) + 1;
                        found = true;
                    }
                    base += tot[q];
                }
                sel = sel_d;
                if (sel_d != 0) {
                    if (!leaf) {
                        nflip = 1;
                        x1 = sel_site;
                        x1_staged = (sel_site == a);
                    } else if (sel_d == 1) {
                        nflip = 1;
                        x1 = a;
                        x1_staged = true;
                    } else if (sel_site != a) {
                        nflip = 2;
                        x1 = a;
                        x1_staged = true;
                        x2 = sel_site;
                    }
                }
                rows = leaf ? 1 + (nflip == 2 ? 1 : 0) : nflip;
            }
            // ---- field update and flips ----
            if (nflip) {
                const int c1 = 2 * S[x1];
                const int c2 = nflip == 2 ? 2 * S[x2] : 0;
                // MCMCMC in the 128-register variant: chunks; Metropolis there:
                // chunks in the RCH instantiation (rows whose per-lane share is
                // not a whole number of unrolled passes), else the unrolled loop
                constexpr bool CHUNKED = UNROLL >= 8 && (RULE == 0 || RCH);
                if (x1_staged)
                    update_fields<JT, STAGED, G, UNROLL, CHUNKED, RULE == 0>(hf, rowA, Jrow(x2), c1, c2, npad, g.gl);
                else
                    update_fields<JT, false, G, UNROLL, CHUNKED, false>(hf, Jrow(x1), nullptr, c1, 0, npad, g.gl);
                __syncwarp(g.mask);
                if (g.gl == 0) {
                    S[x1] = static_cast<int8_t>(-S[x1]);
                    if (nflip == 2) S[x2] = static_cast<int8_t>(-S[x2]);
                }
                acc += 1u;
            }
            n_flips += static_cast<uint32_t>(nflip);
            n_rows += static_cast<uint32_t>(rows);
            if (t < trace_end && g.gl == 0) jb.trace[static_cast<size_t>(chain) * jb.trace_steps + t] = sel;
            __syncwarp(g.mask);
        }
        if constexpr (AHEAD2) {
#pragma unroll
            for (int q = 0; q < 2 * NB; ++q) {
                site[q] = site1[q];
                site1[q] = nsite[q];
            }
        } else if constexpr (RULE == 0 && AHEAD) {
#pragma unroll
            for (int q = 0; q < 2 * NB; ++q) site[q] = nsite[q];
        }
        if (t + 1u == next_rec) {
            record<JT, RULE, NB, G, NWR>(jb, write && !dead, chain, next_rec / jb.record_every - 1u, S, hf, partner_off, acc,
                                    next_rec);
            acc = 0;
            next_rec += jb.record_every;
        }
    }
}

// One work item (a block of chains of one run) on the CTA: every warp loads
// its chains' spins and fields into their shared-memory slices (per_chain
// bytes each, chain slot = warp * 32/G + lane / G), runs the steps of the
// launch, and writes the state back (spins, fields, the spins' tensor-core
// operands of a recomputing run, counters).  Warps without a chain meet the
// CTA's record barriers only.  The job descriptor `jb` (and, +-J, the start of
// the weight table in `s_wt`) is in shared memory, filled by the caller.
template <typename JT, int RULE, int NB, int G, int STAGE, int UNROLL, bool RCH>
__device__ __forceinline__ void run_item(const WorkItem& wi, const JobDev& jb, unsigned char* smem, uint64_t* bars,
                                         const unsigned long long* s_wt, uint32_t nsteps, uint32_t per_chain,
                                         uint32_t& phase, bool& dead) {
    constexpr int SPW = 32 / G;  // chains per warp
    constexpr size_t bj = sizeof(JT);
    const Grp<G> g;
    const int warp = threadIdx.x >> 5;
    const int slot = warp * SPW + (threadIdx.x & 31) / G;  // chain slot of this group in the CTA
    const bool warp_busy = static_cast<uint32_t>(warp * SPW) < wi.nchains;  // some group has a chain
    const bool own = static_cast<uint32_t>(slot) < wi.nchains;              // this group has a chain
    const uint32_t chain = own ? wi.chain0 + slot : wi.chain0;              // shadows copy the first
    const uint32_t npad = jb.Npad;
    ChainMem cm;
    unsigned char* base = smem + static_cast<size_t>(slot) * per_chain;
    cm.s = reinterpret_cast<int8_t*>(base);
    cm.h = base + npad;
    cm.row[0] = base + 5 * static_cast<size_t>(npad);
    cm.row[1] = base + (5 + bj) * static_cast<size_t>(npad);
    cm.bar = &bars[2 * slot];
    cm.b0 = reinterpret_cast<uint4*>(base + (STAGE == 1 ? 5 + 2 * bj : 5) * static_cast<size_t>(npad));
    cm.wsm = s_wt;
    // the overlap partner (chain slot ^ 1) lives one slice up or down
    const int partner_off = (slot & 1) ? -static_cast<int>(per_chain) : static_cast<int>(per_chain);
    const uint32_t t0 = static_cast<uint32_t>(*jb.step);
    const uint32_t t1 =
        static_cast<uint32_t>(min(static_cast<uint64_t>(t0) + nsteps, static_cast<uint64_t>(jb.step_limit)));
    uint32_t acc = 0, n_flips = 0, n_rows = 0;
    if (warp_busy) {
        // load the chain's state: spins (npad bytes), fields (4 npad bytes)
        const uint4* gs = reinterpret_cast<const uint4*>(jb.s + static_cast<size_t>(chain) * npad);
        uint4* ss = reinterpret_cast<uint4*>(cm.s);
        for (uint32_t k = g.gl; k < npad / 16; k += G) ss[k] = gs[k];
        const uint4* gh =
            reinterpret_cast<const uint4*>(static_cast<const int*>(jb.h) + static_cast<size_t>(chain) * npad);
        uint4* sh = reinterpret_cast<uint4*>(cm.h);
        for (uint32_t k = g.gl; k < npad / 4; k += G) sh[k] = gh[k];
        acc = jb.acc_run[chain];
    }
    __syncwarp();
    if (t1 > t0) {
        if (warp_busy) {
            // +-J items whose chains all have the uniform root, no traced
            // steps and a weight table that fits the shared copy take the loop
            // compiled for that case; MCMCMC items with K <= 8 or K <= 32 in
            // the few-chain variant, or in 16-lane and whole-warp chains of the
            // others (rows through L1), take their sites in batches of G/2 or
            // G/8 steps (a choice for the whole CTA: its groups meet the same
            // record barriers)
            const bool fast = sizeof(JT) == 1 && jb.wlen <= kWCache && jb.fcen + jb.fleaf == (2u << 20) &&
                              jb.trace_chains <= wi.chain0;
            // (throughput variants: 16-lane and whole-warp chains)
            constexpr bool kBatch = RULE == 0 && NB == 1 && STAGE != 1 && (UNROLL >= 8 || G >= 16);
            constexpr int kSL2 = kBatch && G >= 4 ? 2 : 0;
            constexpr int kSL8 = kBatch && G >= 16 ? 8 : 0;
            auto loop = [&](auto fast_c, auto sl_c) {
                chain_loop<JT, RULE, NB, G, STAGE, UNROLL, RCH, decltype(fast_c)::value, decltype(sl_c)::value>(
                    jb, own, chain, cm, partner_off, t0, t1, acc, phase, dead, n_flips, n_rows);
            };
            using Fast = std::integral_constant<bool, sizeof(JT) == 1>;
            using Slow = std::integral_constant<bool, false>;
            const uint32_t K = jb.K;
            if (kSL2 && K <= 4u * kSL2) {
                if (fast) loop(Fast{}, std::integral_constant<int, kSL2>{});
                else loop(Slow{}, std::integral_constant<int, kSL2>{});
            } else if (kSL8 && K <= 4u * kSL8) {
                if (fast) loop(Fast{}, std::integral_constant<int, kSL8>{});
                else loop(Slow{}, std::integral_constant<int, kSL8>{});
            } else if (fast) {
                loop(Fast{}, std::integral_constant<int, 0>{});
            } else {
                loop(Slow{}, std::integral_constant<int, 0>{});
            }
        } else {
            // no chain in this warp: meet the CTA's record barriers only
            const uint32_t R = jb.record_every;
            if (R)
                for (uint32_t p = (t0 / R + 1u) * R, r = t0 / R; p <= t1; p += R, ++r)
                    record<JT, RULE, NB, G, STAGE == 2>(jb, false, chain, r, cm.s, cm.h, partner_off, 0u, p);
        }
    }
    __syncwarp();
    if (own) {
        uint4* gs = reinterpret_cast<uint4*>(jb.s + static_cast<size_t>(chain) * npad);
        const uint4* ss = reinterpret_cast<const uint4*>(cm.s);
        for (uint32_t k = g.gl; k < npad / 16; k += G) gs[k] = ss[k];
        if (jb.s_op) {  // the spins as tensor-core operands for the next recompute
            const size_t base16 = static_cast<size_t>(chain) * (npad / 16);
            for (uint32_t k = g.gl; k < npad / 16; k += G) dev::spins_to_op16(jb.s_op, base16 + k, ss[k], bj != 1);
        }
        uint4* gh = reinterpret_cast<uint4*>(static_cast<int*>(jb.h) + static_cast<size_t>(chain) * npad);
        const uint4* sh = reinterpret_cast<const uint4*>(cm.h);
        for (uint32_t k = g.gl; k < npad / 4; k += G) gh[k] = sh[k];
        if (g.gl == 0) {
            jb.acc_run[chain] = acc;
            jb.work[2 * static_cast<size_t>(chain)] += n_flips;
            jb.work[2 * static_cast<size_t>(chain) + 1] += n_rows;
        }
    }
}

// MAXT bounds the CTA size and so the register budget per thread
// (65536 / MAXT): 1024 -> 64, 768 -> 80, 640 -> 96, 512 -> 128 registers.
// STAGE: 1 stages row a by TMA (two row buffers per chain in shared memory),
// 0 reads it through L1 (no buffers: more chains fit in shared memory), 2 is
// 0 with node-weighted energy records (for runs that ask for them).
template <typename JT, int RULE, int NB, int G, int STAGE, int MAXT, bool RCH = false>
__global__ void __launch_bounds__(MAXT, 1)
    step_kernel(const JobDev* __restrict__ jobs, const WorkItem* __restrict__ items, uint32_t n_items,
                uint32_t* __restrict__ queue, uint32_t nsteps, uint32_t per_chain) {
    constexpr int SPW = 32 / G;  // chains per warp
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) JobDev s_job;
    __shared__ __align__(8) uint64_t bars[2 * 256];
    __shared__ unsigned long long s_wt[sizeof(JT) == 1 ? kWCache : 1];
    __shared__ uint32_t s_item;
    const Grp<G> g;
    const int warp = threadIdx.x >> 5;
    const int slot = warp * SPW + (threadIdx.x & 31) / G;  // chain slot of this group in the CTA
    if (g.gl == 0) {
        dev::mbar_init(&bars[2 * slot], 1);
        dev::mbar_init(&bars[2 * slot + 1], 1);
    }
    dev::fence_mbar_init();
    __syncthreads();
    uint32_t phase = 0;
    bool dead = false;  // a bounded wait of this group expired: skip all further work
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
            __syncthreads();
        }
        run_item<JT, RULE, NB, G, STAGE, (MAXT <= 512 ? 8 : 2), RCH>(wi, jb, smem, bars, s_wt, nsteps, per_chain,
                                                                     phase, dead);
        __syncthreads();  // s_job and the smem slices are reused by the next item
    }
}

template <typename JT, int RULE, int NB, int G, int STAGE, int MAXT, bool RCH = false>
cudaError_t launch_variant(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                           uint32_t nsteps, uint32_t W, uint32_t per_chain, uint32_t grid, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(per_chain) * W * (32 / G);
    cudaError_t e = cudaFuncSetAttribute(step_kernel<JT, RULE, NB, G, STAGE, MAXT, RCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    step_kernel<JT, RULE, NB, G, STAGE, MAXT, RCH><<<grid, 32 * W, smem, st>>>(jobs, items, n_items, queue, nsteps,
                                                                               per_chain);
    return cudaGetLastError();
}

template <typename JT, int RULE, int NB, int G, int STAGE, int MAXT, bool RCH = false>
int occupancy_variant(uint32_t W, uint32_t per_chain) {
    const size_t smem = static_cast<size_t>(per_chain) * W * (32 / G);
    int n = 0;
    if (cudaFuncSetAttribute(step_kernel<JT, RULE, NB, G, STAGE, MAXT, RCH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<JT, RULE, NB, G, STAGE, MAXT, RCH>, 32 * W,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

// The register budget follows the CTA size: the largest variant that fits W
// warps.  RCH (Metropolis) selects the chunked field update of the
// 128-register variant; the larger CTAs have one form.
template <typename JT, int RULE, int NB, int G, int STAGE, bool RCH = false>
cudaError_t launch_g(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                     uint32_t nsteps, uint32_t W, uint32_t per_chain, uint32_t grid, cudaStream_t st) {
    if (W <= 16)
        return launch_variant<JT, RULE, NB, G, STAGE, 512, RCH>(jobs, items, n_items, queue, nsteps, W, per_chain,
                                                                grid, st);
    if (W <= 20) return launch_variant<JT, RULE, NB, G, STAGE, 640>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
    if (W <= 24) return launch_variant<JT, RULE, NB, G, STAGE, 768>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
    return launch_variant<JT, RULE, NB, G, STAGE, 1024>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
}
template <typename JT, int RULE, int NB, int G, int STAGE, bool RCH = false>
int occupancy_g(uint32_t W, uint32_t per_chain) {
    if (W <= 16) return occupancy_variant<JT, RULE, NB, G, STAGE, 512, RCH>(W, per_chain);
    if (W <= 20) return occupancy_variant<JT, RULE, NB, G, STAGE, 640>(W, per_chain);
    if (W <= 24) return occupancy_variant<JT, RULE, NB, G, STAGE, 768>(W, per_chain);
    return occupancy_variant<JT, RULE, NB, G, STAGE, 1024>(W, per_chain);
}

// Dispatch over (Philox blocks per lane NB, lanes per chain G) for one
// coupling type, rule and staging choice.  NB = 1 for every G; NB = 2 for
// G = 8, 16, 32 and NB = 4 for G = 8, 16 (MCMCMC only: K up to 4 G NB).
template <typename JT, int RULE, int STAGE>
cudaError_t launch_rule(int nb, int G, const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                        uint32_t nsteps, uint32_t W, uint32_t per_chain, uint32_t grid, cudaStream_t st) {
    if constexpr (RULE == 0) {
        if (nb == 2) {
            switch (G) {
                case 8: return launch_g<JT, RULE, 2, 8, STAGE>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
                case 16: return launch_g<JT, RULE, 2, 16, STAGE>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
                case 32: return launch_g<JT, RULE, 2, 32, STAGE>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
                default: return cudaErrorInvalidValue;
            }
        }
        if (nb == 4) {
            switch (G) {
                case 8: return launch_g<JT, RULE, 4, 8, STAGE>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
                case 16: return launch_g<JT, RULE, 4, 16, STAGE>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    if constexpr (RULE == 1) {  // Metropolis: nb = 2 names the chunked field update (one Philox block)
        if (nb == 2) {
            switch (G) {
                case 4: return launch_g<JT, RULE, 1, 4, STAGE, true>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
                case 8: return launch_g<JT, RULE, 1, 8, STAGE, true>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
                case 16: return launch_g<JT, RULE, 1, 16, STAGE, true>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
                case 32: return launch_g<JT, RULE, 1, 32, STAGE, true>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    if (nb != 1) return cudaErrorInvalidValue;
    switch (G) {
        case 4: return launch_g<JT, RULE, 1, 4, STAGE>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
        case 8: return launch_g<JT, RULE, 1, 8, STAGE>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
        case 16: return launch_g<JT, RULE, 1, 16, STAGE>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
        case 32: return launch_g<JT, RULE, 1, 32, STAGE>(jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
        default: return cudaErrorInvalidValue;
    }
}
template <typename JT, int RULE, int STAGE>
int occupancy_rule(int nb, int G, uint32_t W, uint32_t per_chain) {
    if constexpr (RULE == 0) {
        if (nb == 2) {
            switch (G) {
                case 8: return occupancy_g<JT, RULE, 2, 8, STAGE>(W, per_chain);
                case 16: return occupancy_g<JT, RULE, 2, 16, STAGE>(W, per_chain);
                case 32: return occupancy_g<JT, RULE, 2, 32, STAGE>(W, per_chain);
                default: return 0;
            }
        }
        if (nb == 4) {
            switch (G) {
                case 8: return occupancy_g<JT, RULE, 4, 8, STAGE>(W, per_chain);
                case 16: return occupancy_g<JT, RULE, 4, 16, STAGE>(W, per_chain);
                default: return 0;
            }
        }
    }
    if constexpr (RULE == 1) {
        if (nb == 2) {
            switch (G) {
                case 4: return occupancy_g<JT, RULE, 1, 4, STAGE, true>(W, per_chain);
                case 8: return occupancy_g<JT, RULE, 1, 8, STAGE, true>(W, per_chain);
                case 16: return occupancy_g<JT, RULE, 1, 16, STAGE, true>(W, per_chain);
                case 32: return occupancy_g<JT, RULE, 1, 32, STAGE, true>(W, per_chain);
                default: return 0;
            }
        }
    }
    if (nb != 1) return 0;
    switch (G) {
        case 4: return occupancy_g<JT, RULE, 1, 4, STAGE>(W, per_chain);
        case 8: return occupancy_g<JT, RULE, 1, 8, STAGE>(W, per_chain);
        case 16: return occupancy_g<JT, RULE, 1, 16, STAGE>(W, per_chain);
        case 32: return occupancy_g<JT, RULE, 1, 32, STAGE>(W, per_chain);
        default: return 0;
    }
}

}  // namespace step
}  // namespace sk
