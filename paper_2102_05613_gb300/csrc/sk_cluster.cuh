// sk_cluster.cuh -- the cluster-per-chain layout of the star step (and of the
// Metropolis comparator): one chain's spins, fields and couplings spread over
// the C CTAs of a thread-block cluster.
//
// A cluster of C CTAs (C = 1, 2, 4, 8 or 16) runs the W chains of one work
// item, one warp per chain in every CTA.  CTA r owns the slice k in
// [r Ws, (r+1) Ws), Ws = Npad / C, of every chain's spins and fields and the
// same columns of every row of J, Jr[x][c] = J[x][r Ws + c] (x < N), which it
// bulk-copies (cp.async.bulk, one copy per row, from this GPU's memory, no
// multicast) into its own shared memory when a work item of a new run
// starts.  All a step needs about a site i then lives in the CTA that owns
// i: s_i, h_i and, for the double flip of a leaf root, J_ai.  One step:
//   1  draws: every CTA draws all of the step's sites and its block 0 with
//      the counters of the warp layouts (Philox4x32-10, (block, step, chain,
//      stream)), so each CTA knows the proposals without communication;
//   2  publish: the owner of each proposed site i = site_d writes the entry
//      (h_i, J_ai, s_i) of slot d, a = site_1, into its own exchange array and
//      lists the slot; the warp's lanes then copy the listed entries into the
//      same slot of every CTA's exchange array (lane l to CTA l mod C) as
//      st.async stores whose bytes complete on the receiving CTA's own
//      mbarrier, and every CTA sends every CTA a 4-byte header for the step;
//      Metropolis publishes its one site;
//   3  each CTA waits (bounded) on its own mbarrier for the step's 16 K + 4 C
//      bytes, the only synchronisation of the step; the next step's sites are
//      drawn while the stores travel.  The exchange arrays alternate with the
//      step's parity: a CTA that has all headers of step t knows that every
//      CTA has finished reading step t-1's array, which step t+1 reuses, and
//      a receiver arms the barrier of step t+2 right after its wait of step t,
//      before its own header of step t+1 can let any sender into step t+2;
//   4  choose: every CTA computes the candidate energies, their minimum, the
//      slot weights, the scan in slot order and the chosen slot from the
//      exchange array with the arithmetic of the warp layout's 32-lane chains
//      (Sec. A.2 on the star of App. B.2), so the CTAs of a cluster make the
//      same choice bit for bit, and trajectories equal the warp layout's at 32
//      lanes per chain for both coupling types;
//   5  update: each CTA applies h_k -= 2 s_x J_xk (k in its slice) from its own
//      columns of J -- the field update of the warp layout, element by element
//      in the same order -- and the owner of a flipped site flips it.
// Records (E = -scale/2 sum s h, the accepted count, the overlap q of chains
// 2m, 2m+1, which share the cluster) are formed in rank 0, equal to the
// whole-warp layout's bit for bit.
// C = 1 is a plain CTA with the whole of J in shared memory: the exchange is
// local and the barrier a warp synchronisation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "sk_step.cuh"

namespace sk {
namespace cl {

using dev::kFull;
using dev::Types;
using step::Grp;

constexpr uint32_t kMaxW = kClusterMaxChains;  // chains (warps) per cluster
constexpr uint32_t kMaxC = kClusterMaxCtas;    // CTAs per cluster

__device__ __forceinline__ uint32_t cta_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_ctas() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Shared-memory address `local` of this CTA mapped to the same offset in CTA r.
__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t r) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(local), "r"(r));
    return a;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, uint4 v) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}
// Stores into CTA r's shared memory that count their bytes on an mbarrier of
// that CTA (complete_tx): the receiver learns of their arrival by waiting on
// its own barrier, without a cluster-wide barrier.
__device__ __forceinline__ void st_async(uint32_t addr, uint4 v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(rbar));
}
__device__ __forceinline__ void st_async(uint32_t addr, uint32_t v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr), "r"(v),
                 "r"(rbar));
}
// One local arrival that also expects `bytes` of complete_tx in this phase.
__device__ __forceinline__ void expect_bytes(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(dev::smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double a, double b) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(a), "d"(b) : "memory");
}
// Cluster barrier: every thread of every CTA of the cluster arrives (release:
// its earlier shared-memory stores, local and remote, are visible to the
// threads that pass the wait) and waits (acquire).
__device__ __forceinline__ void arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
template <bool ONE>
__device__ __forceinline__ void sync_all() {
    if constexpr (ONE) {
        __syncthreads();
    } else {
        arrive();
        wait();
    }
}

template <typename T>
__device__ __forceinline__ uint32_t to_bits(T v) {
    if constexpr (std::is_same<T, float>::value)
        return __float_as_uint(v);
    else
        return static_cast<uint32_t>(static_cast<int>(v));
}
template <typename T>
__device__ __forceinline__ T from_bits(uint32_t b) {
    if constexpr (std::is_same<T, float>::value)
        return __uint_as_float(b);
    else
        return static_cast<T>(static_cast<int>(b));
}

// One chain's view of its cluster: this CTA's columns of J, its slices of
// the chain's spins and fields, the chain's block-0 draws and exchange arrays.
struct ClMem {
    const void* jr;            // Jr[x][c], x < N, c < ws (row stride ws elements)
    int8_t* s;                 // s[lo + c], c < ws
    void* h;                   // h[lo + c], c < ws
    uint4* b0;                 // block 0 of 32 consecutive steps
    unsigned char* xg;         // exchange arrays (two, by step parity): generic pointer
    uint32_t xs;               // the same as a shared-memory address
    uint16_t* list;            // slots whose entries this CTA owns in the current step
    uint64_t* xbar;            // two mbarriers (by step parity): the step's entries and headers arrived
    uint32_t xr;               // the exchange region of CTA (lane mod C), where this lane's fan-out goes
    uint32_t xbr;              // that CTA's two mbarriers
    uint32_t xbytes;           // bytes each CTA receives per step (entries and headers)
    uint32_t lc;               // log2 C
    uint32_t ws, lo, C, rank;
    const unsigned long long* wsm;  // +-J: the first kWCache weight-table entries
};

// Record point (one CTA barrier, two cluster barriers): the CTA's partial sum
// of the overlap with the partner chain (and, +-J, of s.h) goes to rank 0,
// which adds them in rank order; for Gaussian couplings rank 0 reads the
// spins and fields of every CTA's slice and sums s_k h_k in the order of the
// whole-warp layout (lane l: fp32 over k = 4l + 128v .. 4l + 128v + 3 for
// v = 0, 1, ..., the lanes' sums added in double precision by a butterfly),
// so the records equal that layout's bit for bit.  The other CTAs keep their
// slices unchanged until rank 0 has read them (the second barrier).  Shadow
// warps meet the same barriers in shadow_steps.
// (The chain's slices come as values, not as its ClMem: a struct whose
// address escapes to a call stays in local memory, and accesses through its
// pointers would become generic instead of shared-memory ones.)
template <typename JT, bool ONE>
__device__ __noinline__ void record(const JobDev& jb, bool write, uint32_t chain, uint32_t rec, const int8_t* cs,
                                    const void* ch, uint32_t ws, uint32_t C, uint32_t rank, const int8_t* partner_s,
                                    uint32_t acc, uint32_t rec_xs, const double* rec_g, uint32_t slot) {
    const uint32_t lane = threadIdx.x & 31;
    __syncthreads();  // the partner chain's flips of this step are done
    double e_part = 0.0;
    int dot = 0;
    if constexpr (sizeof(JT) == 1) {
        const int* hf = static_cast<const int*>(ch);
        int e = 0;
        for (uint32_t k = lane; k < ws; k += 32) e += cs[k] * hf[k];
        e_part = static_cast<double>(__reduce_add_sync(kFull, e));
    }
    const bool pair = (chain & 1u) == 0u && chain + 1u < jb.chains && partner_s != nullptr;
    if (pair)
        for (uint32_t k = lane; k < ws; k += 32) dot += cs[k] * partner_s[k];
    const double q_part = static_cast<double>(__reduce_add_sync(kFull, dot));
    const uint32_t at = rec_xs + (slot * kMaxC + rank) * 16u;
    if (lane == 0) {
        if constexpr (ONE)
            asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(at), "d"(e_part), "d"(q_part) : "memory");
        else
            st_cluster(map_rank(at, 0), e_part, q_part);
    }
    sync_all<ONE>();  // partial sums in rank 0; every slice holds this step's state
    if (rank == 0) {
        double E;
        if constexpr (sizeof(JT) == 1) {
            double es = 0.0;
            for (uint32_t r = 0; r < C; ++r) es += rec_g[2 * (slot * kMaxC + r)];
            const long long tot = static_cast<long long>(es);  // 2 sum_{i<j} J s s, even
            E = jb.scale * static_cast<double>(-(tot / 2));
        } else {
            const uint32_t s_xs = dev::smem_addr(cs), h_xs = dev::smem_addr(ch);
            float e = 0.0f;
            for (uint32_t k0 = 4u * lane; k0 < jb.Npad; k0 += 128u) {
#pragma unroll
                for (uint32_t u = 0; u < 4; ++u) {
                    const uint32_t k = k0 + u, r = k / ws, c = k - r * ws;
                    float hv;
                    int sv;
                    if constexpr (ONE) {
                        hv = static_cast<const float*>(ch)[c];
                        sv = cs[c];
                    } else {
                        asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(hv) : "r"(map_rank(h_xs + 4u * c, r)));
                        asm volatile("ld.shared::cluster.s8 %0, [%1];" : "=r"(sv) : "r"(map_rank(s_xs + c, r)));
                    }
                    e = fmaf(static_cast<float>(sv), hv, e);
                }
            }
            E = -0.5 * jb.scale * dev::warp_sum(static_cast<double>(e));
        }
        if (lane == 0 && write && rec < jb.rec_capacity) {
            double qs = 0.0;
            for (uint32_t r = 0; r < C; ++r) qs += rec_g[2 * (slot * kMaxC + r) + 1];
            jb.rec_E[static_cast<size_t>(rec) * jb.chains + chain] = E;
            jb.rec_acc[static_cast<size_t>(rec) * jb.chains + chain] = acc;
            if (pair) jb.rec_q[static_cast<size_t>(rec) * (jb.chains / 2) + chain / 2] = qs / static_cast<double>(jb.N);
        }
    }
    sync_all<ONE>();  // rank 0 has read the slices
}

// A warp without a chain of its own meets the barriers of the chains'
// records, in the same order.
template <bool ONE>
__device__ __forceinline__ void shadow_steps(const JobDev& jb, uint32_t t0, uint32_t t1) {
    const uint32_t R = jb.record_every;
    uint32_t next_rec = R ? (t0 / R + 1u) * R : 0u;
    for (uint32_t t = t0; t < t1; ++t) {
        if (t + 1u == next_rec) {
            __syncthreads();
            sync_all<ONE>();
            sync_all<ONE>();
            next_rec += R;
        }
    }
}

// Steps t0..t1-1 of one chain (one warp of each CTA of the cluster).
template <typename JT, int RULE, int NB, bool ONE>
__device__ __forceinline__ void chain_steps(const JobDev& jb, bool write, uint32_t chain, const ClMem& cm,
                                            const int8_t* partner_s, uint32_t rec_xs, const double* rec_g,
                                            uint32_t slot, uint32_t t0, uint32_t t1, uint32_t& acc,
                                            uint32_t& n_flips, uint32_t& n_rows, uint32_t& xph, bool& xdead) {
    using H = typename Types<JT>::H;
    using W = typename Types<JT>::W;
    constexpr int G = 32;
    constexpr uint32_t kXBuf = cluster_xbuf_bytes(RULE, NB);  // one exchange array
    constexpr uint32_t kHdr = 2u * kXBuf + cluster_list_bytes(RULE, NB);  // the step headers
    const Grp<G> g;
    const uint32_t lane = static_cast<uint32_t>(g.gl);
    uint32_t next_rec = jb.record_every ? (t0 / jb.record_every + 1u) * jb.record_every : 0u;
    const uint32_t N = jb.N, K = jb.K;
    const uint32_t nblk = (K + 3u) >> 2;
    const uint32_t k0 = static_cast<uint32_t>(jb.seed), k1 = static_cast<uint32_t>(jb.seed >> 32);
    const uint32_t c3 = jb.stream & 0xFFFFFFu;  // domain 0: step draws
    const W* __restrict__ Wt = reinterpret_cast<const W*>(jb.W);
    const uint32_t wlen = jb.wlen;
    const float nbl2 = -jb.beta_eff * 1.4426950408889634f;  // -beta log2(e)
    const bool root_weighted = jb.fcen + jb.fleaf != (2u << 20);
    const uint32_t trace_end = (write && cm.rank == 0 && chain < jb.trace_chains)
                                   ? static_cast<uint32_t>(min(jb.trace_steps, static_cast<uint64_t>(0xFFFFFFFFu)))
                                   : 0u;
    const JT* Jr = static_cast<const JT*>(cm.jr);
    const uint32_t ws = cm.ws, lo = cm.lo;
    int8_t* S = cm.s;
    H* hf = static_cast<H*>(cm.h);

    step::fill_block0<G>(cm.b0, t0 & ~31u, chain, c3, k0, k1, g);
    uint32_t site[2 * NB], nsite[2 * NB];
    if constexpr (RULE == 0) step::draw_sites<NB, G>(site, t0, chain, c3, k0, k1, nblk, N, g);

    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t xo = (t & 1u) * kXBuf;  // this step's exchange array
        const uint4 b0 = cm.b0[t & 31u];
        if (((t + 1u) & 31u) == 0u && t + 1u < t1) {  // the next 32 steps' block 0
            __syncwarp();
            step::fill_block0<G>(cm.b0, t + 1u, chain, c3, k0, k1, g);
        }
        const unsigned long long U1 = (static_cast<unsigned long long>(b0.w) << 32) | b0.z;

        // ---- publish the entries of the proposed sites this CTA owns ----
        // (a) each owner writes its slot's entry into this CTA's exchange
        // array and lists the slot; (b) the lanes copy the listed entries to
        // the other CTAs, lane l to CTA l mod C, 32/C entries at a time
        uint4* X = reinterpret_cast<uint4*>(cm.xg + xo);
        uint32_t a = 0, n_own = 0;
        if constexpr (RULE == 0) {
            a = step::gshfl(g, site[0], 0) & 0xFFFFu;
            const JT* rowa = Jr + static_cast<size_t>(a) * ws;
            const unsigned lt = (1u << lane) - 1u;
            // all of the lane's entries are loaded before any is stored (the
            // stores could otherwise alias the next slot's loads)
            uint4 ent[4 * NB];
            uint32_t owned = 0;
#pragma unroll
            for (int q = 0; q < 4 * NB; ++q) {
                const uint32_t d = 128u * (q >> 2) + 4u * lane + (q & 3) + 1u;
                const uint32_t c = step::site_of<NB>(site, q) - lo;  // wraps when not owned
                ent[q] = make_uint4(0u, 0u, 0u, 0u);
                if (d <= K && c < ws) {
                    owned |= 1u << q;
                    ent[q] = make_uint4(to_bits(hf[c]), to_bits(rowa[c]), static_cast<uint32_t>(static_cast<int>(S[c])), 0u);
                }
            }
#pragma unroll
            for (int q = 0; q < 4 * NB; ++q) {
                const bool own_q = (owned >> q) & 1u;
                const uint32_t slot = static_cast<uint32_t>(q) * 32u + lane;
                if (own_q) X[slot] = ent[q];
                if constexpr (!ONE) {
                    const unsigned ball = __ballot_sync(kFull, own_q);
                    if (own_q) cm.list[n_own + __popc(ball & lt)] = static_cast<uint16_t>(slot);
                    n_own += __popc(ball);
                }
            }
        } else {
            const uint32_t c = __umulhi(b0.x, N) - lo;
            const bool owned = c < ws;  // the same in every lane
            if (lane == 0 && owned)
                X[0] = make_uint4(to_bits(hf[c]), 0u, static_cast<uint32_t>(static_cast<int>(S[c])), 0u);
            if constexpr (!ONE) {
                if (lane == 0 && owned) cm.list[0] = 0;
                n_own = owned ? 1u : 0u;
            }
        }
        __syncwarp();
        const uint32_t p = t & 1u;
        if constexpr (!ONE) {
            // every CTA also sends every CTA a header for the step: a CTA that
            // has received all headers of step t knows that every CTA is done
            // reading the exchange array of step t - 1, which step t + 1 reuses
            // (those reads returned their values, which decided step t - 1,
            // before the header of step t was issued)
#pragma unroll 4
            for (uint32_t e = lane >> cm.lc; e < n_own; e += 32u >> cm.lc) {
                const uint32_t off = xo + 16u * cm.list[e];
                st_async(cm.xr + off, *reinterpret_cast<const uint4*>(cm.xg + off), cm.xbr + 8u * p);
            }
            if (lane < cm.C) st_async(cm.xr + kHdr + 64u * p + 4u * cm.rank, t, cm.xbr + 8u * p);
        }
        // the next step's sites, while the stores travel
        if constexpr (RULE == 0) step::draw_sites<NB, G>(nsite, t + 1u, chain, c3, k0, k1, nblk, N, g);
        if constexpr (!ONE) {
            if (!xdead) {
                // every lane waits (bounded); the outcome is made warp-uniform
                const bool ok = __all_sync(kFull, dev::mbar_wait_bounded(&cm.xbar[p], (xph >> p) & 1u));
                xph ^= 1u << p;
                if (!ok) {
                    xdead = true;
                    if (lane == 0) atomicExch(jb.err, kDevTimeout);
                } else if (lane == 0 && t + 2u < t1) {
                    expect_bytes(&cm.xbar[p], cm.xbytes);  // the phase of step t + 2
                }
            }
            __syncwarp();
        }

        // ---- choose (the same in every CTA) ----
        int sel = 0, nflip = 0, rows = 0;
        uint32_t x1 = 0, x2 = 0;
        int c1 = 0, c2 = 0;
        if constexpr (RULE == 1) {
            const uint4 e = X[0];
            const int si = static_cast<int>(e.z);
            const H dE = static_cast<H>(2 * si) * from_bits<H>(e.x);
            bool accept;
            if constexpr (sizeof(JT) == 1) {
                const uint32_t k = static_cast<uint32_t>(dE) >> 1;
                accept = dE <= 0 || (U1 >> 11) < step::wt_lookup(cm.wsm, Wt, wlen, k);
            } else {
                accept = dE <= 0.0f || static_cast<float>(U1 >> 40) * 0x1p-24f < dev::pow2(nbl2 * dE);
            }
            if (accept) {
                sel = 1;
                nflip = 1;
                x1 = __umulhi(b0.x, N);
                c1 = 2 * si;
            }
            rows = nflip;
        } else {
            const unsigned long long U0 = (static_cast<unsigned long long>(b0.y) << 32) | b0.x;
            const bool leaf = U0 >= jb.root_thr;
            const uint4 ea = X[0];  // slot 1: site a
            const int sa = static_cast<int>(ea.z);
            const H dEa = static_cast<H>(2 * sa) * from_bits<H>(ea.x);
            H dE[4 * NB];
            uint32_t sneg = 0;  // bit q: the spin at this lane's slot q is -1
            H mloc = 0;
#pragma unroll
            for (int q = 0; q < 4 * NB; ++q) {
                const uint32_t d = 128u * (q >> 2) + 4u * lane + (q & 3) + 1u;
                const uint32_t i = step::site_of<NB>(site, q);
                const uint4 e = X[static_cast<uint32_t>(q) * 32u + lane];
                const int si = d <= K ? static_cast<int>(e.z) : 1;  // no entry past K
                const H hi = from_bits<H>(e.x);
                const JT jab = from_bits<JT>(e.y);
                const H single = static_cast<H>(2 * si) * hi;
                // leaf root: the centre flipped at b = site_d (0 if b = a)
                const H dbl = (i == a) ? H(0) : dEa + single - static_cast<H>(4 * sa * si) * static_cast<H>(jab);
                const H v = !leaf ? single : (d == 1u ? dEa : dbl);
                dE[q] = v;
                if (si < 0) sneg |= 1u << q;
                if (d <= K) mloc = mloc < v ? mloc : v;
            }
            const H m = step::gmin<true>(g, mloc);
            // weights exp(-beta (dE - m)) times the slot's root factor, kept
            // in registers for the node search
            W xs[4 * NB], gsum_[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) gsum_[q] = 0;
#pragma unroll
            for (int q = 0; q < 4 * NB; ++q) {
                const uint32_t d = 128u * (q >> 2) + 4u * lane + (q & 3) + 1u;
                W x = 0;
                const bool centre = leaf && d == 1u;
                if (d <= K) {
                    if constexpr (sizeof(JT) == 1) {
                        const uint32_t idx = static_cast<uint32_t>(dE[q] - m) >> 1;
                        x = step::wt_lookup(cm.wsm, Wt, wlen, idx);
                        if (root_weighted)  // floor(x F / 2^20)
                            x = __umul64hi(x << 11, static_cast<unsigned long long>(centre ? jb.fcen : jb.fleaf) << 33);
                    } else {
                        x = dev::pow2(fmaf(nbl2, dE[q] - m, centre ? jb.lcen : jb.lleaf));
                    }
                }
                xs[q] = x;
                gsum_[q >> 2] += x;
            }
            W w0;  // slot 0, the root: the centre of a centre root, else a leaf
            if constexpr (sizeof(JT) == 1) {
                const uint32_t idx0 = static_cast<uint32_t>(-m) >> 1;
                w0 = step::wt_lookup(cm.wsm, Wt, wlen, idx0);
                if (root_weighted)
                    w0 = __umul64hi(w0 << 11, static_cast<unsigned long long>(leaf ? jb.fleaf : jb.fcen) << 33);
            } else {
                w0 = dev::pow2(fmaf(-nbl2, m, leaf ? jb.lleaf : jb.lcen));
            }
            W incl[NB], tot[NB];
            W total = w0;
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                incl[q] = step::gscan(g, gsum_[q]);
                tot[q] = step::gshfl(g, incl[q], G - 1);
                total += tot[q];
            }
            W u;
            if constexpr (sizeof(JT) == 1) {
                u = __umul64hi(U1, total);
            } else {
                u = static_cast<float>(U1 >> 40) * 0x1p-24f * total;
                if (u >= total) u = nextafterf(total, 0.0f);
            }
            // first slot whose inclusive prefix exceeds u (else, a rounding
            // guard, the owning lane's last positive weight); one packed
            // shuffle gives every lane the site, its spin and the slot
            int sel_d = 0;
            uint32_t sel_site = 0, sel_neg = 0;
            bool found = u < w0;
            W base = w0;
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const unsigned ball = __ballot_sync(kFull, !found && base + incl[q] > u);
                if (!found && ball) {
                    const int L = __ffs(ball) - 1;
                    W mine = 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e) mine += xs[4 * q + e];
                    W run = base + (incl[q] - mine);
                    int my_e = -1, last_pos = -1;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (xs[4 * q + e] > W(0)) {
                            last_pos = e;
                            if (my_e < 0) {
                                run += xs[4 * q + e];
                                if (run > u) my_e = e;
                            }
                        }
                    }
                    if (my_e < 0) my_e = last_pos;
                    uint32_t my = 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (e == my_e)
                            my = (step::site_of<NB>(site, 4 * q + e) << 3) | (((sneg >> (4 * q + e)) & 1u) << 2) |
                                 static_cast<uint32_t>(e);
                    const uint32_t packed = __shfl_sync(kFull, my, L);
                    sel_site = packed >> 3;
                    sel_neg = (packed >> 2) & 1u;
                    sel_d = 128 * q + 4 * L + static_cast<int>(packed & 3u) + 1;
                    found = true;
                }
                base += tot[q];
            }
            sel = sel_d;
            const int csel = sel_neg ? -2 : 2;
            if (sel_d != 0) {
                if (!leaf) {
                    nflip = 1;
                    x1 = sel_site;
                    c1 = csel;
                } else if (sel_d == 1) {
                    nflip = 1;
                    x1 = a;
                    c1 = 2 * sa;
                } else if (sel_site != a) {
                    nflip = 2;
                    x1 = a;
                    c1 = 2 * sa;
                    x2 = sel_site;
                    c2 = csel;
                }
            }
            rows = leaf ? 1 + (nflip == 2 ? 1 : 0) : nflip;
        }

        // ---- field update of this CTA's slice, flips by the owner ----
        if (nflip) {
            const JT* r1 = Jr + static_cast<size_t>(x1) * ws;
            const JT* r2 = Jr + static_cast<size_t>(x2) * ws;
            for (uint32_t k = lane; k < ws; k += 32) {
                if constexpr (sizeof(JT) == 1) {
                    int hv = hf[k];
                    hv -= c1 * static_cast<int>(r1[k]);
                    if (c2) hv -= c2 * static_cast<int>(r2[k]);
                    hf[k] = hv;
                } else {
                    float hv = hf[k];
                    hv = fmaf(-static_cast<float>(c1), r1[k], hv);
                    if (c2) hv = fmaf(-static_cast<float>(c2), r2[k], hv);
                    hf[k] = hv;
                }
            }
            if (lane == 0) {
                if (x1 - lo < ws) S[x1 - lo] = static_cast<int8_t>(-S[x1 - lo]);
                if (nflip == 2 && x2 - lo < ws) S[x2 - lo] = static_cast<int8_t>(-S[x2 - lo]);
            }
            acc += 1u;
        }
        n_flips += static_cast<uint32_t>(nflip);
        n_rows += static_cast<uint32_t>(rows);
        if (t < trace_end && lane == 0) jb.trace[static_cast<size_t>(chain) * jb.trace_steps + t] = sel;
        __syncwarp();
        if constexpr (RULE == 0) {
#pragma unroll
            for (int q = 0; q < 2 * NB; ++q) site[q] = nsite[q];
        }
        if (t + 1u == next_rec) {
            record<JT, ONE>(jb, write, chain, next_rec / jb.record_every - 1u, cm.s, cm.h, cm.ws, cm.C, cm.rank,
                            partner_s, acc, rec_xs, rec_g, slot);
            acc = 0;
            next_rec += jb.record_every;
        }
    }
}

// Persistent kernel: each cluster takes work items (W chains of one run) from
// the class's queue; rank 0 draws the item and hands it to the other CTAs.
// Dynamic shared memory: this CTA's columns of J (jbytes), then per chain
// slot (pc bytes each) the exchange arrays, block 0, the spin and the field
// slice (cluster_chain_bytes).
template <typename JT, int RULE, int NB, bool ONE>
__global__ void __launch_bounds__(32 * kClusterMaxChains, 1)
    cluster_kernel(const JobDev* __restrict__ jobs, const WorkItem* __restrict__ items, uint32_t n_items,
                   uint32_t* __restrict__ queue, uint32_t nsteps, uint32_t jbytes, uint32_t pc) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) JobDev s_job;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ unsigned long long s_wt[sizeof(JT) == 1 ? step::kWCache : 1];
    __shared__ __align__(16) double s_rec[kMaxW * kMaxC * 2];
    __shared__ uint32_t s_item, s_fail;
    constexpr uint32_t kX = cluster_x_bytes(RULE, NB);
    const uint32_t C = ONE ? 1u : cluster_ctas();
    const uint32_t rank = ONE ? 0u : cta_rank();
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        dev::mbar_init(&s_bar, 1);
        s_fail = 0;
    }
    // the exchange mbarriers of this warp's chain slot
    uint64_t* xbar = reinterpret_cast<uint64_t*>(smem + jbytes + static_cast<size_t>(warp) * pc + kX - 16u);
    if (!ONE && lane == 0) {
        dev::mbar_init(&xbar[0], 1);
        dev::mbar_init(&xbar[1], 1);
    }
    uint32_t xph = 0;    // parity each exchange mbarrier's current phase completes with
    bool xdead = false;  // an exchange wait expired: no further waits in this launch
    dev::fence_mbar_init();
    __syncthreads();
    if constexpr (!ONE) sync_all<false>();  // every CTA of the cluster runs before any remote store
    uint32_t phase = 0;
    uint32_t loaded = 0xFFFFFFFFu;  // run whose columns of J this CTA holds
    bool broken = false;            // a slice copy timed out: no further copies
    const uint32_t item_xs = dev::smem_addr(&s_item), fail_xs = dev::smem_addr(&s_fail);
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const uint32_t it = atomicAdd(queue, 1u);
            if constexpr (ONE)
                s_item = it;
            else
                for (uint32_t r = 0; r < C; ++r) st_cluster(map_rank(item_xs, r), it);
        }
        sync_all<ONE>();
        const uint32_t it = s_item;
        if (it >= n_items) break;
        const WorkItem wi = items[it];
        if (threadIdx.x < sizeof(JobDev) / 16)
            reinterpret_cast<uint4*>(&s_job)[threadIdx.x] = reinterpret_cast<const uint4*>(&jobs[wi.job])[threadIdx.x];
        __syncthreads();
        const JobDev& jb = s_job;
        if constexpr (sizeof(JT) == 1) {  // the start of the +-J weight table (0 past its end)
            for (uint32_t i = threadIdx.x; i < step::kWCache; i += blockDim.x)
                s_wt[i] = i < jb.wlen ? reinterpret_cast<const unsigned long long*>(jb.W)[i] : 0ull;
        }
        const uint32_t npad = jb.Npad, N = jb.N;
        const uint32_t ws = npad / C, lo = rank * ws;
        const uint32_t t0 = static_cast<uint32_t>(*jb.step);
        const uint32_t t1 = static_cast<uint32_t>(
            min(static_cast<uint64_t>(t0) + nsteps, static_cast<uint64_t>(jb.step_limit)));
        // this CTA's columns of J: one bulk copy of ws elements per row
        if (wi.job != loaded || broken) {
            if (warp == 0) {
                bool ok = false;
                if (!broken) {
                    const uint32_t rb = ws * static_cast<uint32_t>(sizeof(JT));
                    // (a test of the bounded wait may withhold one row of the first item)
                    const bool withhold = (jb.fault & kFaultWithholdRow) && rank == 0 && wi.chain0 == 0u && t0 == 0u;
                    if (lane == 0) {
                        dev::fence_proxy_async();
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                         dev::smem_addr(&s_bar)),
                                     "r"(N * rb)
                                     : "memory");
                    }
                    __syncwarp();
                    const unsigned char* src = static_cast<const unsigned char*>(jb.J) +
                                               static_cast<size_t>(lo) * sizeof(JT);
                    for (uint32_t x = lane; x < N; x += 32) {
                        if (withhold && x == N - 1u) continue;
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                            "[%3];" ::"r"(dev::smem_addr(smem + static_cast<size_t>(x) * rb)),
                            "l"(src + static_cast<size_t>(x) * npad * sizeof(JT)), "r"(rb),
                            "r"(dev::smem_addr(&s_bar))
                            : "memory");
                    }
                    ok = __all_sync(kFull, dev::mbar_wait_bounded(&s_bar, phase));
                    phase ^= 1u;
                    if (!ok) {
                        // let the copies in flight land before the CTA can leave (bounded)
                        dev::mbar_wait_bounded(&s_bar, phase ^ 1u);
                        broken = true;
                    }
                }
                if (!ok && lane == 0) {
                    atomicExch(jb.err, kDevTimeout);
                    if constexpr (ONE)
                        s_fail = it + 1u;
                    else
                        for (uint32_t r = 0; r < C; ++r) st_cluster(map_rank(fail_xs, r), it + 1u);
                }
            }
            loaded = wi.job;
        }
        sync_all<ONE>();  // the slices of every CTA are in place (or a copy failed)
        const bool dead = s_fail == it + 1u;
        const bool own = warp < wi.nchains;
        const uint32_t chain = wi.chain0 + (own ? warp : 0u);
        unsigned char* base = smem + jbytes + static_cast<size_t>(warp) * pc;
        ClMem cm;
        cm.jr = smem;
        cm.xg = base;
        cm.xs = dev::smem_addr(base);
        cm.list = reinterpret_cast<uint16_t*>(base + 2u * cluster_xbuf_bytes(RULE, NB));
        cm.lc = static_cast<uint32_t>(__ffs(static_cast<int>(C)) - 1);
        cm.xr = ONE ? cm.xs : map_rank(cm.xs, lane & (C - 1u));
        cm.xbar = xbar;
        cm.xbr = ONE ? 0u : map_rank(dev::smem_addr(xbar), lane & (C - 1u));
        cm.xbytes = 16u * (RULE == 1 ? 1u : jb.K) + 4u * C;
        cm.b0 = reinterpret_cast<uint4*>(base + kX);
        cm.s = reinterpret_cast<int8_t*>(base + kX + kB0Bytes);
        cm.h = base + kX + kB0Bytes + ((ws + 15u) & ~15u);
        cm.ws = ws;
        cm.lo = lo;
        cm.C = C;
        cm.rank = rank;
        cm.wsm = s_wt;
        // the overlap partner (chain slot warp ^ 1), if the CTA has that slot
        const int8_t* partner_s =
            (warp ^ 1u) < (blockDim.x >> 5)
                ? reinterpret_cast<const int8_t*>(smem + jbytes + static_cast<size_t>(warp ^ 1u) * pc + kX + kB0Bytes)
                : nullptr;
        uint32_t acc = 0, n_flips = 0, n_rows = 0;
        constexpr size_t bh = sizeof(typename Types<JT>::H);
        if (own) {
            const int8_t* gs = jb.s + static_cast<size_t>(chain) * npad + lo;
            const unsigned char* gh = static_cast<const unsigned char*>(jb.h) + (static_cast<size_t>(chain) * npad + lo) * bh;
            for (uint32_t k = lane; k < ws; k += 32) {
                cm.s[k] = gs[k];
                reinterpret_cast<uint32_t*>(cm.h)[k] = reinterpret_cast<const uint32_t*>(gh)[k];
            }
            acc = jb.acc_run[chain];
        }
        __syncwarp();
        if constexpr (!ONE) {
            // arm the exchange barriers for the first two steps before any CTA
            // of the cluster can send them
            if (!dead && own && !xdead && lane == 0) {
                if (t0 < t1) expect_bytes(&xbar[t0 & 1u], cm.xbytes);
                if (t0 + 1u < t1) expect_bytes(&xbar[(t0 + 1u) & 1u], cm.xbytes);
            }
            sync_all<false>();
        }
        if (!dead && t1 > t0) {
            if (own)
                chain_steps<JT, RULE, NB, ONE>(jb, true, chain, cm, partner_s, dev::smem_addr(s_rec), s_rec, warp, t0,
                                               t1, acc, n_flips, n_rows, xph, xdead);
            else
                shadow_steps<ONE>(jb, t0, t1);
        }
        if (own && !dead) {
            int8_t* gs = jb.s + static_cast<size_t>(chain) * npad + lo;
            unsigned char* gh = static_cast<unsigned char*>(jb.h) + (static_cast<size_t>(chain) * npad + lo) * bh;
            for (uint32_t k = lane; k < ws; k += 32) {
                gs[k] = cm.s[k];
                reinterpret_cast<uint32_t*>(gh)[k] = reinterpret_cast<const uint32_t*>(cm.h)[k];
            }
            if (jb.s_op) {  // the spins as tensor-core operands for the next recompute
                const size_t o = static_cast<size_t>(chain) * npad + lo;
                for (uint32_t k = lane; k < ws; k += 32) {
                    const int v = cm.s[k];
                    if constexpr (sizeof(JT) == 1)
                        static_cast<uint8_t*>(jb.s_op)[o + k] = v == 0 ? 0 : (v > 0 ? 0x38 : 0xB8);
                    else
                        static_cast<uint16_t*>(jb.s_op)[o + k] = v == 0 ? 0 : (v > 0 ? 0x3F80 : 0xBF80);
                }
            }
            if (rank == 0 && lane == 0) {
                jb.acc_run[chain] = acc;
                jb.work[2 * static_cast<size_t>(chain)] += n_flips;
                jb.work[2 * static_cast<size_t>(chain) + 1] += n_rows;
            }
        }
        __syncthreads();  // s_job, s_wt and the chain slots are reused by the next item
    }
    if (xdead) {
        // an exchange wait expired: give stores still in flight to this CTA
        // (about a millisecond) time to land before it leaves
        const long long start = clock64();
        while (clock64() - start < 2000000ll) {
        }
    }
}

template <typename JT, int RULE, int NB, bool ONE>
cudaError_t launch_variant(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                           uint32_t nsteps, uint32_t C, uint32_t W, uint32_t jbytes, uint32_t pc, uint32_t clusters,
                           cudaStream_t st) {
    auto k = cluster_kernel<JT, RULE, NB, ONE>;
    const size_t smem = static_cast<size_t>(jbytes) + static_cast<size_t>(W) * pc;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if constexpr (ONE) {
        k<<<clusters, 32 * W, smem, st>>>(jobs, items, n_items, queue, nsteps, jbytes, pc);
        return cudaGetLastError();
    } else {
        if (C > 8 && (e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
            return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(clusters * C, 1, 1);
        cfg.blockDim = dim3(32 * W, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k, jobs, items, n_items, queue, nsteps, jbytes, pc);
    }
}

// Clusters of C CTAs of W warps that can be resident at once (0: none).
template <typename JT, int RULE, int NB, bool ONE>
int occupancy_variant(uint32_t C, uint32_t W, uint32_t jbytes, uint32_t pc) {
    auto k = cluster_kernel<JT, RULE, NB, ONE>;
    const size_t smem = static_cast<size_t>(jbytes) + static_cast<size_t>(W) * pc;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return 0;
    int n = 0;
    if constexpr (ONE) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * W, smem) != cudaSuccess) return 0;
        return n * sms;
    } else {
        if (C > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(32 * W, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) return 0;
        return n;
    }
}

// Dispatch over rule, Philox blocks per lane and C = 1 for one coupling type.
template <typename JT>
cudaError_t launch_kind(uint32_t rule, uint32_t nb, const JobDev* jobs, const WorkItem* items, uint32_t n_items,
                        uint32_t* queue, uint32_t nsteps, uint32_t C, uint32_t W, uint32_t jbytes, uint32_t pc,
                        uint32_t clusters, cudaStream_t st) {
#define SK_CL_LAUNCH(R, B)                                                                                        \
    return C == 1 ? launch_variant<JT, R, B, true>(jobs, items, n_items, queue, nsteps, C, W, jbytes, pc, clusters, \
                                                   st)                                                            \
                  : launch_variant<JT, R, B, false>(jobs, items, n_items, queue, nsteps, C, W, jbytes, pc, clusters, st)
    if (rule == 1) {
        if (nb != 1) return cudaErrorInvalidValue;
        SK_CL_LAUNCH(1, 1);
    }
    if (nb == 1) SK_CL_LAUNCH(0, 1);
    if (nb == 2) SK_CL_LAUNCH(0, 2);
#undef SK_CL_LAUNCH
    return cudaErrorInvalidValue;
}
template <typename JT>
int occupancy_kind(uint32_t rule, uint32_t nb, uint32_t C, uint32_t W, uint32_t jbytes, uint32_t pc) {
#define SK_CL_OCC(R, B) \
    return C == 1 ? occupancy_variant<JT, R, B, true>(C, W, jbytes, pc) : occupancy_variant<JT, R, B, false>(C, W, jbytes, pc)
    if (rule == 1) {
        if (nb != 1) return 0;
        SK_CL_OCC(1, 1);
    }
    if (nb == 1) SK_CL_OCC(0, 1);
    if (nb == 2) SK_CL_OCC(0, 2);
#undef SK_CL_OCC
    return 0;
}

}  // namespace cl
}  // namespace sk
