// sk_graph.cu -- MCMCMC on deeper graphs: full k-ary trees populated from a
// uniformly drawn root position and the line of L nodes with the addition
// process's binomial root position (App. B.1, B.2).
//
// A chain is owned by a team of NW warps (NW = 1, 2, 4, 8 or 16; teams of
// several warps meet at a named barrier of their own).  Its spins s and fields
// h stay in the team's shared-memory slice for the whole launch.  One step:
//   draws   Philox block 0 of the step (U0, U1) and blocks 1..ceil((V-1)/4)
//           for the edge sites: template edge v (between node v and its
//           template parent; the line's edge v joins nodes v-1 and v) flips
//           site_v = floor(w N / 2^32), word (v-1) % 4 of block 1 + (v-1)/4
//           (the star's slot draws, slot d = v);
//   root    r = the first node whose inclusive prefix of the node factors F
//           exceeds floor(U0 sum F / 2^64) (tree: floor(U0 V / 2^64));
//   nodes   node v is the current state with the sites of the path r -> v
//           flipped.  With p(v) the neighbour of v toward r and x_v the site
//           of the edge between them,
//             dE_v = dE_p(v) + delta_v,
//             delta_v = 2 sigma_v (h_x - 2 sum_w sigma_w J[x_v][x_w]),
//           the single-flip change of x_v in configuration p(v): sigma_w is
//           the spin of x_w just before its flip on the path (s times -1 for
//           every earlier flip of the same site, so repeated sites cancel as
//           they do when flipped in turn), the sum runs over the nodes w
//           strictly between r and v.  Three passes over the nodes, a node
//           per thread: x and sigma (integer work on the sites), delta (the J
//           lookups of its path, issued four at a time), dE (the deltas along
//           its path);
//   choice  weight ~ exp(-beta (dE_v - min)) F_v over the nodes in order
//           (+-J: the integer table times F / 2^20; Gaussian: 2^x), each
//           thread a contiguous chunk of nodes, a team scan of the chunk
//           sums, the first node whose inclusive prefix exceeds u = U1 total;
//   move    the chosen path's flips: h_k -= 2 sum_w sigma_w J[x_w][k] over its
//           nodes, then each flip negates its spin in path order.
// The oracle (sko_run_graph) defines the same chain in double precision, a
// node's energy change being the sum of the sequential single-flip changes
// along its path, which the delta recursion restates term by term.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sk_device.cuh"
#include "sk_internal.h"
#include "sk_step.cuh"

namespace sk {
namespace graphk {

using dev::kFull;
using dev::Types;

constexpr uint32_t kMaxTeamsMulti = 14;  // chains per CTA when a chain has several warps (barriers 1..15)
constexpr uint32_t kMiscBytes = 512;     // block 0, per-warp partials, chosen node, path length

struct GTab {
    const uint32_t* F;
    const uint64_t* P;    // inclusive prefix sums of F
    const float* lg;      // log2(F / 2^20)
    const uint8_t* dep;   // depth of each node in the tree template
};
__device__ __forceinline__ GTab gtab(const JobDev& jb) {
    const size_t V16 = (static_cast<size_t>(jb.V) + 3u) & ~static_cast<size_t>(3u);
    const unsigned char* b = static_cast<const unsigned char*>(jb.gtab);
    GTab t;
    t.F = reinterpret_cast<const uint32_t*>(b);
    t.P = reinterpret_cast<const uint64_t*>(b + 4 * V16);
    t.lg = reinterpret_cast<const float*>(b + 12 * V16);
    t.dep = b + 16 * V16;
    return t;
}

// Full k-ary tree in level order: parent (v - 1) / k by a 32-bit reciprocal,
// exact for v, k < 2^16 (the error term (v - 1) (kinv k - 2^32) stays below
// 2^32); node depths come from the run's graph table.
struct Tree {
    uint32_t k, kinv;
    __device__ __forceinline__ uint32_t par(uint32_t v) const { return __umulhi(v - 1u, kinv); }
};

// Team barrier: the NW warps of one chain (a warp barrier when NW = 1); the
// non-aligned form, so that lanes of a warp may arrive from divergent code.
__device__ __forceinline__ void team_sync(uint32_t nw, uint32_t team) {
    if (nw == 1u) {
        __syncwarp();
    } else {
        asm volatile("barrier.sync %0, %1;" ::"r"(team + 1u), "r"(nw * 32u) : "memory");
    }
}
// Team barrier that also returns whether any thread of the team passed true.
__device__ __forceinline__ bool team_any(uint32_t nw, uint32_t team, bool v) {
    if (nw == 1u) return __any_sync(kFull, v);
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n barrier.red.or.pred p, %2, %3, q;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"(v ? 1u : 0u), "r"(team + 1u), "r"(nw * 32u)
        : "memory");
    return r != 0u;
}

// Shared memory of one chain (offsets in chain_bytes order).
struct GMem {
    int8_t* s;
    void* h;
    uint16_t* site;  // [V] template edge sites (site[0] unused)
    uint16_t* xs;    // [V] x_v, the site of the edge from v toward the root
    void* dl;        // [V] delta_v (H)
    void* dE;        // [V] node energy changes (H)
    uint16_t* fx;    // [V] the move: sites flipped; during the node passes (trees) the
                     // node's depth and its meeting depth with the root (8 bits each)
    int8_t* sg;      // [V] sigma_v
    int8_t* fs;      // [V] the move: the spin of each flipped site before its flip
    uint4* b0;       // block 0 of the step
    void* red;       // [2][16] per-warp partial results (8 bytes each)
    uint32_t* misc;  // [0] chosen node, [1] path length of the move, [2] the root
    uint16_t* anc;   // [17] trees: the root's ancestor at each depth 0..depth(root)
};

size_t chain_bytes(uint32_t npad, uint32_t V) {
    const size_t v16 = (static_cast<size_t>(V) + 15u) & ~static_cast<size_t>(15u);
    return 5u * static_cast<size_t>(npad) + 16u * v16 + kMiscBytes;
}

__device__ __forceinline__ GMem chain_mem(unsigned char* base, uint32_t npad, uint32_t V) {
    const size_t v16 = (static_cast<size_t>(V) + 15u) & ~static_cast<size_t>(15u);
    const size_t o = 5u * static_cast<size_t>(npad);
    GMem g;
    g.s = reinterpret_cast<int8_t*>(base);
    g.h = base + npad;
    g.site = reinterpret_cast<uint16_t*>(base + o);
    g.xs = reinterpret_cast<uint16_t*>(base + o + 2u * v16);
    g.dl = base + o + 4u * v16;
    g.dE = base + o + 8u * v16;
    g.fx = reinterpret_cast<uint16_t*>(base + o + 12u * v16);
    g.sg = reinterpret_cast<int8_t*>(base + o + 14u * v16);
    g.fs = reinterpret_cast<int8_t*>(base + o + 15u * v16);
    unsigned char* m = base + o + 16u * v16;
    g.b0 = reinterpret_cast<uint4*>(m);
    g.red = m + 16;
    g.misc = reinterpret_cast<uint32_t*>(m + 16 + 256);
    g.anc = reinterpret_cast<uint16_t*>(m + 16 + 256 + 16);
    return g;
}

// sum over n path nodes w (next() yields them) of sigma_w row[x_w], the J
// loads issued eight at a time (the remainder together too)
template <typename JT, typename H, typename Next>
__device__ __forceinline__ H path_dot(const JT* __restrict__ row, uint32_t n, const uint16_t* xs, const int8_t* sg,
                                      Next&& next) {
    H acc = H(0);
    uint32_t i = 0;
    for (; i + 8u <= n; i += 8u) {
        uint32_t w[8];
        JT j[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = next();
#pragma unroll
        for (int q = 0; q < 8; ++q) j[q] = __ldg(row + xs[w[q]]);
#pragma unroll
        for (int q = 0; q < 8; ++q) acc += static_cast<H>(sg[w[q]]) * static_cast<H>(j[q]);
    }
    if (i < n) {  // the last n - i < 8 terms, their loads issued together
        const uint32_t r = n - i;
        uint32_t w[8];
        JT j[8];
#pragma unroll
        for (uint32_t q = 0; q < 8u; ++q) w[q] = q < r ? next() : 0u;
#pragma unroll
        for (uint32_t q = 0; q < 8u; ++q) j[q] = q < r ? __ldg(row + xs[w[q]]) : JT(0);
#pragma unroll
        for (uint32_t q = 0; q < 8u; ++q)
            if (q < r) acc += static_cast<H>(sg[w[q]]) * static_cast<H>(j[q]);
    }
    return acc;
}

// One chain's steps t0..t1-1 by its team (T = 32 nw threads, tid in [0, T)).
template <typename JT, int GRAPH>
__device__ __forceinline__ void graph_loop(const JobDev& jb, bool write, uint32_t chain, const GMem& gm,
                                           int partner_off, uint32_t t0, uint32_t t1, uint32_t nw, uint32_t team,
                                           uint32_t& acc, uint32_t& n_flips) {
    using H = typename Types<JT>::H;
    using W = typename Types<JT>::W;
    const uint32_t T = 32u * nw;
    const uint32_t tid = threadIdx.x - team * T;
    const uint32_t lane = threadIdx.x & 31u, wt = tid >> 5;
    const step::Grp<32> g;
    const uint32_t N = jb.N, npad = jb.Npad, V = jb.V;
    Tree tr;
    tr.k = jb.arity < 2u ? 2u : jb.arity;
    tr.kinv = 0xFFFFFFFFu / tr.k + 1u;
    const uint32_t k0 = static_cast<uint32_t>(jb.seed), k1 = static_cast<uint32_t>(jb.seed >> 32);
    const uint32_t c3 = jb.stream & 0xFFFFFFu;
    const JT* __restrict__ Jg = static_cast<const JT*>(jb.J);
    const uint64_t* __restrict__ Wt = static_cast<const uint64_t*>(jb.W);
    const float nbl2 = -jb.beta_eff * 1.4426950408889634f;
    const GTab tab = gtab(jb);
    const uint32_t trace_end = (write && chain < jb.trace_chains)
                                   ? static_cast<uint32_t>(min(jb.trace_steps, static_cast<uint64_t>(0xFFFFFFFFu)))
                                   : 0u;
    int8_t* S = gm.s;
    H* hf = static_cast<H*>(gm.h);
    H* dl = static_cast<H*>(gm.dl);
    H* dE = static_cast<H*>(gm.dE);
    H* rmin = static_cast<H*>(gm.red);                                    // [16] warp minima
    W* rsum = reinterpret_cast<W*>(static_cast<unsigned char*>(gm.red) + 128);  // [16] warp sums
    const uint32_t nblk = (V + 2u) / 4u;  // blocks 1..nblk hold the V-1 edge sites
    const uint32_t chunk = (V + T - 1u) / T;
    uint32_t next_rec = jb.record_every ? (t0 / jb.record_every + 1u) * jb.record_every : 0u;

    for (uint32_t t = t0; t < t1; ++t) {
        // ---- draws: block 0 and the edge sites ----
        for (uint32_t b = tid; b <= nblk; b += T) {
            const uint4 r = dev::philox4x32_10(make_uint4(b, t, chain, c3), k0, k1);
            if (b == 0u) {
                *gm.b0 = r;
                // root: tree floor(U0 V / 2^64); line the first v with
                // P[v] > floor(U0 sum F / 2^64)
                const unsigned long long U0 = (static_cast<unsigned long long>(r.y) << 32) | r.x;
                uint32_t root;
                if constexpr (GRAPH == 1) {
                    root = static_cast<uint32_t>(__umul64hi(U0, static_cast<unsigned long long>(V)));
                    // the root's ancestors by depth
                    uint32_t a = root;
                    for (uint32_t d = __ldg(&tab.dep[root]) + 1u; d-- > 0u;) {
                        gm.anc[d] = static_cast<uint16_t>(a);
                        a = d ? tr.par(a) : 0u;
                    }
                } else {
                    const unsigned long long x = __umul64hi(U0, __ldg(&tab.P[V - 1u]));
                    uint32_t lo = 0, hi = V - 1u;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (__ldg(&tab.P[mid]) > x) hi = mid;
                        else lo = mid + 1u;
                    }
                    root = lo;
                }
                gm.misc[2] = root;
            } else {
                const uint32_t v0 = 4u * (b - 1u) + 1u;
                const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (v0 + e < V) gm.site[v0 + e] = static_cast<uint16_t>(__umulhi(w[e], N));
            }
        }
        if (tid == 0u) gm.misc[0] = V;  // no node chosen yet
        team_sync(nw, team);
        const uint4 b0 = *gm.b0;
        const unsigned long long U0 = (static_cast<unsigned long long>(b0.y) << 32) | b0.x;
        const unsigned long long U1 = (static_cast<unsigned long long>(b0.w) << 32) | b0.z;

        const uint32_t root = gm.misc[2];
        const uint32_t dr = GRAPH == 1 ? __ldg(&tab.dep[root]) : 0u;
        const uint16_t* anc = gm.anc;

        // ---- pass 1: x_v and sigma_v ----
        for (uint32_t v = tid; v < V; v += T) {
            if (v == root) {
                gm.xs[v] = 0;
                gm.sg[v] = 0;
                if constexpr (GRAPH == 1) gm.fx[v] = static_cast<uint16_t>(dr | (dr << 8));
                continue;
            }
            uint32_t x, cnt = 0;
            if constexpr (GRAPH == 1) {
                const uint32_t dv = __ldg(&tab.dep[v]);
                // the edge at v: v's own unless v is an ancestor of r, then
                // the edge from the child of v toward r
                const bool v_anc = dv <= dr && anc[dv] == v;
                const uint32_t own = v_anc ? anc[dv + 1u] : v;
                x = gm.site[own];
                // climb from v to the meeting node m with r's ancestors,
                // counting x among v's side of the path (edges below m) ...
                uint32_t a = v, d = dv;
                while (d > dr || a != anc[d]) {
                    cnt += (a != own && gm.site[a] == x) ? 1u : 0u;
                    a = tr.par(a);
                    --d;
                }
                const uint32_t dm = d;
                gm.fx[v] = static_cast<uint16_t>(dv | (dm << 8));
                // ... and on r's side (the edges of r's ancestors below m)
#pragma unroll 4
                for (uint32_t e = dm + 1u; e <= dr; ++e) {
                    const uint32_t c = anc[e];
                    cnt += (c != own && gm.site[c] == x) ? 1u : 0u;
                }
            } else {
                // line: edge e joins nodes e-1 and e; the path's edges are
                // lo+1..hi and the edge at v is v (v > r) or v+1 (v < r)
                const uint32_t own = v > root ? v : v + 1u;
                const uint32_t lo = min(root, v), hi = max(root, v);
                x = gm.site[own];
#pragma unroll 4
                for (uint32_t e = lo + 1u; e <= hi; ++e) cnt += (e != own && gm.site[e] == x) ? 1u : 0u;
            }
            gm.xs[v] = static_cast<uint16_t>(x);
            gm.sg[v] = static_cast<int8_t>((cnt & 1u) ? -S[x] : S[x]);
        }
        team_sync(nw, team);

        // ---- pass 2: delta_v ----
        for (uint32_t v = tid; v < V; v += T) {
            if (v == root) {
                dl[v] = H(0);
                continue;
            }
            const uint32_t x = gm.xs[v];
            const JT* row = Jg + static_cast<size_t>(x) * npad;
            H corr;
            if constexpr (GRAPH == 1) {
                // nodes strictly between r and v: the ancestors of r up to
                // the meeting node m (m excluded when m = v), then the
                // ancestors of v below m
                const uint32_t dd = gm.fx[v], dv = dd & 0xFFu, dm = dd >> 8;
                const uint32_t nb = dv - dm;
                uint32_t ra = dr - dm - (nb == 0u ? 1u : 0u), rb = nb ? nb - 1u : 0u;
                uint32_t ia = dr, b = nb ? tr.par(v) : 0u;
                auto next = [&]() -> uint32_t {
                    if (ra) {  // r's ancestors from its parent up
                        --ra;
                        return anc[--ia];
                    }
                    const uint32_t w = b;
                    b = tr.par(b);
                    return w;
                };
                corr = path_dot<JT, H>(row, ra + rb, gm.xs, gm.sg, next);
            } else {
                const uint32_t lo = min(root, v), hi = max(root, v);
                uint32_t w = lo;  // nodes lo+1 .. hi-1 strictly between
                corr = path_dot<JT, H>(row, hi - lo - 1u, gm.xs, gm.sg, [&]() -> uint32_t { return ++w; });
            }
            dl[v] = static_cast<H>(2 * gm.sg[v]) * (hf[x] - static_cast<H>(2) * corr);
        }
        team_sync(nw, team);

        // ---- pass 3: dE_v = sum of delta over the path's nodes after r ----
        for (uint32_t v = tid; v < V; v += T) {
            H d = H(0);
            if constexpr (GRAPH == 1) {
                const uint32_t dd = gm.fx[v], dv = dd & 0xFFu, dm = dd >> 8;
#pragma unroll 4
                for (uint32_t e = dm; e < dr; ++e) d += dl[anc[e]];  // r's ancestors up to m
                uint32_t a = v;
#pragma unroll 4
                for (uint32_t d_ = dv; d_ > dm; --d_) {
                    d += dl[a];
                    a = tr.par(a);
                }
            } else {
                if (v > root) {
#pragma unroll 4
                    for (uint32_t w = root + 1u; w <= v; ++w) d += dl[w];
                } else {
#pragma unroll 4
                    for (uint32_t w = v; w < root; ++w) d += dl[w];
                }
            }
            dE[v] = d;
        }
        team_sync(nw, team);

        // ---- choice: weights over contiguous node chunks, team scan ----
        const uint32_t v0 = tid * chunk, v1 = min(V, v0 + chunk);
        H mloc = H(0);
        for (uint32_t v = v0; v < v1; ++v)
            if (__ldg(&tab.F[v]) && dE[v] < mloc) mloc = dE[v];
        mloc = step::gmin<false>(g, mloc);
        if (nw > 1u) {
            if (lane == 0u) rmin[wt] = mloc;
            team_sync(nw, team);
            for (uint32_t w = 0; w < nw; ++w) {
                const H x = rmin[w];
                mloc = x < mloc ? x : mloc;
            }
        }
        const H m = mloc;
        auto node_w = [&](uint32_t v) -> W {
            const uint32_t F = __ldg(&tab.F[v]);
            if (!F) return W(0);
            if constexpr (sizeof(JT) == 1) {
                const uint32_t idx = static_cast<uint32_t>(dE[v] - m) >> 1;
                unsigned long long x = idx < jb.wlen ? __ldg(&Wt[idx]) : 0ull;
                if (F != (1u << 20)) x = __umul64hi(x << 11, static_cast<unsigned long long>(F) << 33);
                return x;
            } else {
                return dev::pow2(fmaf(nbl2, dE[v] - m, __ldg(&tab.lg[v])));
            }
        };
        W lsum = W(0);
        for (uint32_t v = v0; v < v1; ++v) lsum += node_w(v);
        const W incl = step::gscan(g, lsum);
        const W wtot = __shfl_sync(kFull, incl, 31);
        W excl = W(0), total = wtot;
        if (nw > 1u) {
            if (lane == 31u) rsum[wt] = wtot;
            team_sync(nw, team);
            W run = W(0);
            for (uint32_t w = 0; w < nw; ++w) {
                if (w == wt) excl = run;
                run += rsum[w];
            }
            total = run;
        }
        W u;
        if constexpr (sizeof(JT) == 1) {
            u = __umul64hi(U1, total);
        } else {
            u = static_cast<float>(U1 >> 40) * 0x1p-24f * total;
            if (u >= total) u = nextafterf(total, 0.0f);
        }
        // the warp whose range [excl, excl + wtot) holds u: its first lane
        // whose prefix exceeds u searches its chunk (else, a rounding guard,
        // its last positive weight)
        if (wtot > W(0) && u >= excl && u < excl + wtot) {
            const unsigned ball = __ballot_sync(kFull, excl + incl > u);
            const int L = ball ? __ffs(ball) - 1 : 31;
            if (static_cast<int>(lane) == L) {
                W run = excl + (incl - lsum);
                int found = -1, last = -1;
                for (uint32_t v = v0; v < v1; ++v) {
                    const W x = node_w(v);
                    if (x > W(0)) {
                        last = static_cast<int>(v);
                        if (found < 0) {
                            run += x;
                            if (run > u) found = static_cast<int>(v);
                        }
                    }
                }
                const uint32_t js = static_cast<uint32_t>(found >= 0 ? found : last);
                gm.misc[0] = js;
                if constexpr (GRAPH == 1) gm.misc[3] = js < V ? gm.fx[js] : 0u;
            }
        }
        team_sync(nw, team);
        uint32_t jsel = gm.misc[0];
        if (jsel >= V) jsel = root;  // no positive weight found (cannot happen for finite fields): stay

        // ---- move: the chosen path's flips ----
        // the path's nodes after r, one per thread: the ancestors of r up to
        // the meeting node, then jsel and its ancestors below it (the order
        // of the flips does not matter: the signs are those of the path)
        uint32_t n;
        if constexpr (GRAPH == 1) {
            const uint32_t dd = jsel == root ? (dr | (dr << 8)) : gm.misc[3];
            const uint32_t dj = dd & 0xFFu, dm = dd >> 8;
            const uint32_t na = dr - dm;
            n = na + dj - dm;
            for (uint32_t i = tid; i < n; i += T) {
                uint32_t w;
                if (i < na) {
                    w = anc[dr - 1u - i];
                } else {
                    w = jsel;
                    for (uint32_t q = na; q < i; ++q) w = tr.par(w);
                }
                gm.fx[i] = gm.xs[w];
                gm.fs[i] = gm.sg[w];
            }
        } else {
            const uint32_t lo = min(root, jsel), hi = max(root, jsel);
            n = hi - lo;
            for (uint32_t i = tid; i < n; i += T) {
                const uint32_t w = lo + 1u + i;  // the nodes lo+1..hi: one of them is r, the other end jsel
                const uint32_t ww = jsel > root ? w : w - 1u;
                gm.fx[i] = gm.xs[ww];
                gm.fs[i] = gm.sg[ww];
            }
        }
        team_sync(nw, team);
        // fields: h_k -= 2 sum_i fs_i J[fx_i][k], four elements per thread,
        // the rows' loads issued four flips at a time
        for (uint32_t k = 4u * tid; k < npad; k += 4u * T) {
            const JT* col = Jg + k;
            if constexpr (sizeof(JT) == 1) {
                int4 hv = *reinterpret_cast<int4*>(hf + k);
                auto upd = [&](uint32_t j, int c) {
                    hv.x -= c * dev::sbyte(j, 0);
                    hv.y -= c * dev::sbyte(j, 1);
                    hv.z -= c * dev::sbyte(j, 2);
                    hv.w -= c * dev::sbyte(j, 3);
                };
                uint32_t i = 0;
                for (; i + 4u <= n; i += 4u) {
                    uint32_t j[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        j[q] = __ldg(reinterpret_cast<const unsigned int*>(col + static_cast<size_t>(gm.fx[i + q]) * npad));
#pragma unroll
                    for (int q = 0; q < 4; ++q) upd(j[q], 2 * gm.fs[i + q]);
                }
                if (i < n) {  // the last n - i < 4 rows together
                    const uint32_t r = n - i;
                    uint32_t j[3];
#pragma unroll
                    for (uint32_t q = 0; q < 3u; ++q)
                        j[q] = q < r ? __ldg(reinterpret_cast<const unsigned int*>(
                                           col + static_cast<size_t>(gm.fx[i + q]) * npad))
                                     : 0u;
#pragma unroll
                    for (uint32_t q = 0; q < 3u; ++q)
                        if (q < r) upd(j[q], 2 * gm.fs[i + q]);
                }
                *reinterpret_cast<int4*>(hf + k) = hv;
            } else {
                float4 hv = *reinterpret_cast<float4*>(hf + k);
                auto upd = [&](const float4& j, float c) {
                    hv.x = fmaf(-c, j.x, hv.x);
                    hv.y = fmaf(-c, j.y, hv.y);
                    hv.z = fmaf(-c, j.z, hv.z);
                    hv.w = fmaf(-c, j.w, hv.w);
                };
                uint32_t i = 0;
                for (; i + 4u <= n; i += 4u) {
                    float4 j[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        j[q] = __ldg(reinterpret_cast<const float4*>(col + static_cast<size_t>(gm.fx[i + q]) * npad));
#pragma unroll
                    for (int q = 0; q < 4; ++q) upd(j[q], static_cast<float>(2 * gm.fs[i + q]));
                }
                if (i < n) {  // the last n - i < 4 rows together
                    const uint32_t r = n - i;
                    float4 j[3];
#pragma unroll
                    for (uint32_t q = 0; q < 3u; ++q)
                        j[q] = q < r ? __ldg(reinterpret_cast<const float4*>(col + static_cast<size_t>(gm.fx[i + q]) * npad))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (uint32_t q = 0; q < 3u; ++q)
                        if (q < r) upd(j[q], static_cast<float>(2 * gm.fs[i + q]));
                }
                *reinterpret_cast<float4*>(hf + k) = hv;
            }
        }
        // spins: the first occurrence of each site flips it if the site
        // occurs an odd number of times; the state changed iff one does
        bool odd = false;
        for (uint32_t i = tid; i < n; i += T) {
            const uint32_t x = gm.fx[i];
            bool first = true;
            uint32_t c = 0;
            for (uint32_t j = 0; j < n; ++j) {
                const bool eq = gm.fx[j] == x;
                c += eq ? 1u : 0u;
                first = first && !(eq && j < i);
            }
            if (first && (c & 1u)) {
                odd = true;
                S[x] = static_cast<int8_t>(-S[x]);
            }
        }
        const bool changed = team_any(nw, team, odd);
        acc += changed ? 1u : 0u;
        n_flips += n;
        if (t < trace_end && tid == 0u) jb.trace[static_cast<size_t>(chain) * jb.trace_steps + t] = static_cast<int32_t>(jsel);
        team_sync(nw, team);
        if (t + 1u == next_rec) {
            step::record<JT, 0, 1, 32, false>(jb, write && wt == 0u, chain, next_rec / jb.record_every - 1u, S, hf,
                                              partner_off, acc, next_rec);
            acc = 0;
            next_rec += jb.record_every;
        }
    }
}

template <typename JT, int GRAPH, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
    graph_kernel(const JobDev* __restrict__ jobs, const WorkItem* __restrict__ items, uint32_t n_items,
                 uint32_t* __restrict__ queue, uint32_t nsteps, uint32_t per_chain, uint32_t nw) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) JobDev s_job;
    __shared__ uint32_t s_item;
    const uint32_t T = 32u * nw;
    const uint32_t team = threadIdx.x / T, tid = threadIdx.x - team * T, wt = tid >> 5;
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
        const bool own = team < wi.nchains;
        const uint32_t chain = own ? wi.chain0 + team : wi.chain0;
        const uint32_t npad = jb.Npad;
        unsigned char* base = smem + static_cast<size_t>(team) * per_chain;
        const GMem gm = chain_mem(base, npad, jb.V);
        const int partner_off = (team & 1u) ? -static_cast<int>(per_chain) : static_cast<int>(per_chain);
        const uint32_t t0 = static_cast<uint32_t>(*jb.step);
        const uint32_t t1 = static_cast<uint32_t>(
            min(static_cast<uint64_t>(t0) + nsteps, static_cast<uint64_t>(jb.step_limit)));
        uint32_t acc = 0, n_flips = 0;
        if (own) {
            const uint4* gs = reinterpret_cast<const uint4*>(jb.s + static_cast<size_t>(chain) * npad);
            uint4* ss = reinterpret_cast<uint4*>(gm.s);
            for (uint32_t q = tid; q < npad / 16; q += T) ss[q] = gs[q];
            const uint4* gh = reinterpret_cast<const uint4*>(static_cast<const int*>(jb.h) + static_cast<size_t>(chain) * npad);
            uint4* sh = reinterpret_cast<uint4*>(gm.h);
            for (uint32_t q = tid; q < npad / 4; q += T) sh[q] = gh[q];
            acc = jb.acc_run[chain];
        }
        __syncthreads();
        if (t1 > t0) {
            if (own) {
                graph_loop<JT, GRAPH>(jb, true, chain, gm, partner_off, t0, t1, nw, team, acc, n_flips);
            } else {  // no chain in this team: meet the CTA's record barriers only
                const uint32_t R = jb.record_every;
                if (R)
                    for (uint32_t p = (t0 / R + 1u) * R, r = t0 / R; p <= t1; p += R, ++r)
                        step::record<JT, 0, 1, 32, false>(jb, false, chain, r, gm.s, gm.h, partner_off, 0u, p);
            }
        }
        __syncthreads();
        if (own) {
            uint4* gs = reinterpret_cast<uint4*>(jb.s + static_cast<size_t>(chain) * npad);
            const uint4* ss = reinterpret_cast<const uint4*>(gm.s);
            for (uint32_t q = tid; q < npad / 16; q += T) gs[q] = ss[q];
            uint4* gh = reinterpret_cast<uint4*>(static_cast<int*>(jb.h) + static_cast<size_t>(chain) * npad);
            const uint4* sh = reinterpret_cast<const uint4*>(gm.h);
            for (uint32_t q = tid; q < npad / 4; q += T) gh[q] = sh[q];
            if (tid == 0u) {
                jb.acc_run[chain] = acc;
                jb.work[2 * static_cast<size_t>(chain)] += n_flips;
                jb.work[2 * static_cast<size_t>(chain) + 1] += n_flips;
            }
        }
        (void)wt;
        __syncthreads();
    }
}

template <typename JT, int GRAPH, int MAXT>
cudaError_t launch_t(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue, uint32_t ns,
                     uint32_t W, uint32_t nw, uint32_t per_chain, uint32_t grid, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(per_chain) * (W / nw);
    cudaError_t e = cudaFuncSetAttribute(graph_kernel<JT, GRAPH, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    graph_kernel<JT, GRAPH, MAXT><<<grid, 32 * W, smem, st>>>(jobs, items, n_items, queue, ns, per_chain, nw);
    return cudaGetLastError();
}
template <typename JT, int GRAPH, int MAXT>
int occupancy_t(uint32_t W, uint32_t nw, uint32_t per_chain) {
    const size_t smem = static_cast<size_t>(per_chain) * (W / nw);
    int n = 0;
    if (cudaFuncSetAttribute(graph_kernel<JT, GRAPH, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, graph_kernel<JT, GRAPH, MAXT>, 32 * W, smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace graphk

size_t graph_smem_bytes(uint32_t npad, uint32_t V, uint32_t graph) {
    (void)graph;
    return (graphk::chain_bytes(npad, V) + 127u) / 128u * 128u;
}
size_t graph_table_bytes(uint32_t V) {
    const size_t V16 = (static_cast<size_t>(V) + 3u) & ~static_cast<size_t>(3u);
    return 17u * V16;
}
bool graph_team_ok(uint32_t W, uint32_t nw) {
    if (nw != 1u && nw != 2u && nw != 4u && nw != 8u && nw != 16u) return false;
    if (W == 0u || W > 32u || W % nw) return false;
    const uint32_t chains = W / nw;
    return chains % 2u == 0u && (nw == 1u || chains <= graphk::kMaxTeamsMulti);
}

namespace {
__global__ void bump_graph_steps(const JobDev* __restrict__ jobs, uint32_t n_jobs, uint64_t nsteps) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_jobs) {
        const uint64_t lim = jobs[j].step_limit;
        const uint64_t s = *jobs[j].step + nsteps;
        *jobs[j].step = s < lim ? s : lim;
    }
}
}  // namespace

namespace {
template <typename JT, int GRAPH>
cudaError_t launch_g(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue, uint32_t ns,
                     uint32_t W, uint32_t nw, uint32_t per_chain, uint32_t grid, cudaStream_t st) {
    return W <= 16 ? graphk::launch_t<JT, GRAPH, 512>(jobs, items, n_items, queue, ns, W, nw, per_chain, grid, st)
                   : graphk::launch_t<JT, GRAPH, 1024>(jobs, items, n_items, queue, ns, W, nw, per_chain, grid, st);
}
template <typename JT, int GRAPH>
int occupancy_g(uint32_t W, uint32_t nw, uint32_t pc) {
    return W <= 16 ? graphk::occupancy_t<JT, GRAPH, 512>(W, nw, pc) : graphk::occupancy_t<JT, GRAPH, 1024>(W, nw, pc);
}
}  // namespace

cudaError_t launch_graph(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                         uint64_t nsteps, uint32_t W, uint32_t nw, uint32_t per_chain, uint32_t grid, uint32_t kind,
                         uint32_t graph, uint32_t n_jobs, bool bump, cudaStream_t st) {
    if (!graph_team_ok(W, nw) || (graph != 1u && graph != 2u)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const uint32_t ns = static_cast<uint32_t>(nsteps);
    if (kind == 0)
        e = graph == 1u ? launch_g<int8_t, 1>(jobs, items, n_items, queue, ns, W, nw, per_chain, grid, st)
                        : launch_g<int8_t, 2>(jobs, items, n_items, queue, ns, W, nw, per_chain, grid, st);
    else
        e = graph == 1u ? launch_g<float, 1>(jobs, items, n_items, queue, ns, W, nw, per_chain, grid, st)
                        : launch_g<float, 2>(jobs, items, n_items, queue, ns, W, nw, per_chain, grid, st);
    if (e != cudaSuccess || !bump) return e;
    bump_graph_steps<<<(n_jobs + 127) / 128, 128, 0, st>>>(jobs, n_jobs, nsteps);
    return cudaGetLastError();
}

int graph_kernel_occupancy(uint32_t kind, uint32_t graph, uint32_t W, uint32_t nw, size_t per_chain) {
    if (!graph_team_ok(W, nw) || (graph != 1u && graph != 2u)) return 0;
    const uint32_t pc = static_cast<uint32_t>(per_chain);
    if (kind == 0) return graph == 1u ? occupancy_g<int8_t, 1>(W, nw, pc) : occupancy_g<int8_t, 2>(W, nw, pc);
    return graph == 1u ? occupancy_g<float, 1>(W, nw, pc) : occupancy_g<float, 2>(W, nw, pc);
}

}  // namespace sk
