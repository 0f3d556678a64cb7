// sk_graph.cu -- MCMCMC on deeper graphs: full k-ary trees populated from a
// uniformly drawn root position and the line of L nodes with the addition
// process's binomial root position (App. B.1, B.2).
//
// One step of one chain (one warp per chain, the chain's spins s and fields h
// in its shared-memory slice for the whole launch):
//   draws   Philox block 0 of the step (U0, U1) and blocks 1..ceil((V-1)/4)
//           for the edge sites: the edge between template node v and its
//           parent flips site_v = floor(w N / 2^32), word (v-1) % 4 of block
//           1 + (v-1)/4 (the star's slot draws, edge v for slot d = v);
//   root    r = the first node whose inclusive prefix of the node factors F
//           exceeds floor(U0 sum F / 2^64) (uniform for the tree:
//           floor(U0 V / 2^64));
//   nodes   node v is the current state with the sites of the template path
//           between r and v flipped; its energy change dE_v is the sum of the
//           single-flip changes along the path.  Trees: one lane per node,
//           from the path's sites (<= 2 depth flips) with the pairwise
//           coupling corrections; lines: the whole warp walks from r toward
//           each end, one node per step, the coupling corrections of the
//           flips behind it summed across lanes;
//   choice  weight ~ exp(-beta (dE_v - min)) F_v in node order (+-J: the
//           integer table times F / 2^20; Gaussian: 2^x), warp inclusive scan
//           over contiguous node chunks, first prefix above u;
//   move    the chosen path's flips, each a field update h_k -= 2 s_x J_kx.
// The oracle (sko_run_graph) defines the same chain in double precision.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sk_device.cuh"
#include "sk_internal.h"
#include "sk_step.cuh"

namespace sk {
namespace graphk {

using dev::kFull;
using dev::Types;

constexpr uint32_t kMaxTreePath = 32;  // 2 x depth

struct GTab {
    const uint32_t* F;
    const uint64_t* P;  // inclusive prefix sums of F
    const float* lg;    // log2(F / 2^20)
};
__device__ __forceinline__ GTab gtab(const JobDev& jb) {
    const size_t V16 = (static_cast<size_t>(jb.V) + 3u) & ~static_cast<size_t>(3u);
    const unsigned char* b = static_cast<const unsigned char*>(jb.gtab);
    GTab t;
    t.F = reinterpret_cast<const uint32_t*>(b);
    t.P = reinterpret_cast<const uint64_t*>(b + 4 * V16);
    t.lg = reinterpret_cast<const float*>(b + 12 * V16);
    return t;
}

__device__ __forceinline__ uint32_t tparent(uint32_t graph, uint32_t k, uint32_t v) {
    return graph == 1u ? (v - 1u) / k : v - 1u;
}
__device__ __forceinline__ uint32_t tdepth(uint32_t graph, uint32_t k, uint32_t v) {
    uint32_t d = 0;
    while (v) {
        v = tparent(graph, k, v);
        ++d;
    }
    return d;
}

// The template path's edges (child node ids) between a and b, into e[]
// (order: a upward, then b upward; the flips commute).  Returns their number.
__device__ __forceinline__ uint32_t tree_path(uint32_t k, uint32_t a, uint32_t b, uint32_t (&e)[kMaxTreePath]) {
    uint32_t da = tdepth(1u, k, a), db = tdepth(1u, k, b), n = 0;
    while (da > db) {
        e[n++] = a;
        a = (a - 1u) / k;
        --da;
    }
    while (db > da) {
        e[n++] = b;
        b = (b - 1u) / k;
        --db;
    }
    while (a != b) {
        e[n++] = a;
        e[n++] = b;
        a = (a - 1u) / k;
        b = (b - 1u) / k;
    }
    return n;
}

// Shared memory of one chain.
struct GMem {
    int8_t* s;
    void* h;
    uint16_t* site;  // [V] edge sites (site[0] unused)
    void* dE;        // [V] node energy changes (H)
    uint16_t* fx;    // [V] lines: the walk's flips in order
    int8_t* fsig;    // [V] lines: the sign of each flip's spin before it
};

size_t chain_bytes(uint32_t npad, uint32_t V, uint32_t graph) {
    const size_t v16 = (static_cast<size_t>(V) + 15u) & ~static_cast<size_t>(15u);
    return 5u * static_cast<size_t>(npad) + 6u * v16 + (graph == 2u ? 3u * v16 : 0u);
}

// One chain's steps t0..t1-1.
template <typename JT>
__device__ __forceinline__ void graph_loop(const JobDev& jb, bool write, uint32_t chain, const GMem& gm,
                                           int partner_off, uint32_t t0, uint32_t t1, uint32_t& acc,
                                           uint32_t& n_flips) {
    using H = typename Types<JT>::H;
    using W = typename Types<JT>::W;
    const int lane = threadIdx.x & 31;
    const step::Grp<32> g;
    const uint32_t N = jb.N, npad = jb.Npad, V = jb.V, graph = jb.graph, k = jb.arity;
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
    H* dEs = static_cast<H*>(gm.dE);
    const uint32_t nblk = (V + 2u) / 4u;  // blocks 1..nblk hold the V-1 edge sites
    const uint32_t chunk = (V + 31u) / 32u;
    uint32_t next_rec = jb.record_every ? (t0 / jb.record_every + 1u) * jb.record_every : 0u;

    for (uint32_t t = t0; t < t1; ++t) {
        // ---- draws ----
        const uint4 b0 = dev::philox4x32_10(make_uint4(0u, t, chain, c3), k0, k1);
        const unsigned long long U0 = (static_cast<unsigned long long>(b0.y) << 32) | b0.x;
        const unsigned long long U1 = (static_cast<unsigned long long>(b0.w) << 32) | b0.z;
        for (uint32_t b = 1u + lane; b <= nblk; b += 32u) {
            const uint4 r = dev::philox4x32_10(make_uint4(b, t, chain, c3), k0, k1);
            const uint32_t v0 = 4u * (b - 1u) + 1u;
            const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (v0 + e < V) gm.site[v0 + e] = static_cast<uint16_t>(__umulhi(w[e], N));
        }
        // ---- root ----
        uint32_t root;
        if (graph == 1u) {
            root = static_cast<uint32_t>(__umul64hi(U0, static_cast<unsigned long long>(V)));
        } else {  // first v with P[v] > floor(U0 sum F / 2^64)
            const unsigned long long x = __umul64hi(U0, tab.P[V - 1u]);
            uint32_t lo = 0, hi = V - 1u;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (__ldg(&tab.P[mid]) > x) hi = mid;
                else lo = mid + 1u;
            }
            root = lo;
        }
        __syncwarp();

        // ---- node energy changes ----
        if (graph == 1u) {
            for (uint32_t v = lane; v < V; v += 32u) {
                uint32_t e[kMaxTreePath];
                const uint32_t n = tree_path(k, root, v, e);
                // flips in path order: dE += 2 sigma_i h'_i, sigma_i the spin's
                // sign before its flip, h'_i its field after the earlier flips
                H d = H(0);
                int sig[kMaxTreePath];
                for (uint32_t i = 0; i < n; ++i) {
                    const uint32_t x = gm.site[e[i]];
                    int sg = S[x];
                    H hx = hf[x];
                    for (uint32_t j = 0; j < i; ++j) {
                        const uint32_t y = gm.site[e[j]];
                        if (y == x) sg = -sg;
                        else hx -= static_cast<H>(2 * sig[j]) * static_cast<H>(__ldg(Jg + static_cast<size_t>(x) * npad + y));
                    }
                    sig[i] = sg;
                    d += static_cast<H>(2 * sg) * hx;
                }
                dEs[v] = d;
            }
        } else {
            // the walk from the root toward node 0 and toward node V-1
            if (lane == 0) dEs[root] = H(0);
            for (int dir = -1; dir <= 1; dir += 2) {
                H accd = H(0);
                uint32_t n = 0;
                for (int v = static_cast<int>(root) + dir; v >= 0 && v < static_cast<int>(V); v += dir, ++n) {
                    const uint32_t x = gm.site[dir > 0 ? v : v + 1];  // edge between v and its neighbour toward r
                    H part = H(0);
                    uint32_t dup = 0;
                    for (uint32_t j = lane; j < n; j += 32u) {
                        const uint32_t y = gm.fx[j];
                        if (y == x) dup ^= 1u;
                        else part += static_cast<H>(gm.fsig[j]) * static_cast<H>(__ldg(Jg + static_cast<size_t>(x) * npad + y));
                    }
                    part = step::gsum(g, part);
                    const uint32_t odd = __popc(__ballot_sync(kFull, dup != 0u)) & 1u;
                    const int sg = odd ? -S[x] : S[x];
                    accd += static_cast<H>(2 * sg) * (hf[x] - static_cast<H>(2) * part);
                    __syncwarp();
                    if (lane == 0) {
                        dEs[v] = accd;
                        gm.fx[n] = static_cast<uint16_t>(x);
                        gm.fsig[n] = static_cast<int8_t>(sg);
                    }
                    __syncwarp();
                }
            }
        }
        __syncwarp();

        // ---- choice: weights over contiguous node chunks, warp scan ----
        const uint32_t v0 = lane * chunk, v1 = min(V, v0 + chunk);
        H mloc = H(0);
        for (uint32_t v = v0; v < v1; ++v)
            if (__ldg(&tab.F[v]) && dEs[v] < mloc) mloc = dEs[v];
        const H m = step::gmin(g, mloc);
        auto node_w = [&](uint32_t v) -> W {
            const uint32_t F = __ldg(&tab.F[v]);
            if (!F) return W(0);
            if constexpr (sizeof(JT) == 1) {
                const uint32_t idx = static_cast<uint32_t>(dEs[v] - m) >> 1;
                unsigned long long x = idx < jb.wlen ? __ldg(&Wt[idx]) : 0ull;
                if (F != (1u << 20)) x = __umul64hi(x << 11, static_cast<unsigned long long>(F) << 33);
                return x;
            } else {
                return dev::pow2(fmaf(nbl2, dEs[v] - m, __ldg(&tab.lg[v])));
            }
        };
        W lsum = W(0);
        for (uint32_t v = v0; v < v1; ++v) lsum += node_w(v);
        const W incl = step::gscan(g, lsum);
        const W total = __shfl_sync(kFull, incl, 31);
        W u;
        if constexpr (sizeof(JT) == 1) {
            u = __umul64hi(U1, total);
        } else {
            u = static_cast<float>(U1 >> 40) * 0x1p-24f * total;
            if (u >= total) u = nextafterf(total, 0.0f);
        }
        const unsigned ball = __ballot_sync(kFull, incl > u);
        const int L = ball ? __ffs(ball) - 1 : 31;
        uint32_t mine = 0;
        if (lane == L) {
            W run = incl - lsum;
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
            mine = static_cast<uint32_t>(found >= 0 ? found : last);
        }
        uint32_t jsel = __shfl_sync(kFull, mine, L);
        if (jsel >= V) jsel = root;  // no positive weight found (cannot happen for finite fields): stay

        // ---- move: the chosen path's flips ----
        uint32_t changed = 0, nfl = 0;
        auto flip = [&](uint32_t x) {
            const int c = 2 * S[x];
            const JT* row = Jg + static_cast<size_t>(x) * npad;
            for (uint32_t kk = lane; kk < npad; kk += 32u)
                hf[kk] -= static_cast<H>(c) * static_cast<H>(__ldg(row + kk));
            __syncwarp();
            if (lane == 0) S[x] = static_cast<int8_t>(-S[x]);
            __syncwarp();
            ++nfl;
        };
        if (graph == 1u) {
            uint32_t e[kMaxTreePath];
            const uint32_t n = tree_path(k, root, jsel, e);
            for (uint32_t i = 0; i < n; ++i) flip(gm.site[e[i]]);
            for (uint32_t i = 0; i < n; ++i) {
                uint32_t c = 0;
                for (uint32_t j = 0; j < n; ++j) c += gm.site[e[j]] == gm.site[e[i]];
                changed |= c & 1u;
            }
        } else {
            const uint32_t lo = min(root, jsel), hi = max(root, jsel);
            for (uint32_t v = lo + 1u; v <= hi; ++v) flip(gm.site[v]);
            for (uint32_t v = lo + 1u + lane; v <= hi; v += 32u) {
                uint32_t c = 0;
                for (uint32_t q = lo + 1u; q <= hi; ++q) c += gm.site[q] == gm.site[v];
                changed |= c & 1u;
            }
            changed = __any_sync(kFull, changed != 0u) ? 1u : 0u;
        }
        acc += changed;
        n_flips += nfl;
        if (t < trace_end && lane == 0) jb.trace[static_cast<size_t>(chain) * jb.trace_steps + t] = static_cast<int32_t>(jsel);
        __syncwarp();
        if (t + 1u == next_rec) {
            step::record<JT, 0, 1, 32, false>(jb, write, chain, next_rec / jb.record_every - 1u, S, hf, partner_off, acc,
                                              next_rec);
            acc = 0;
            next_rec += jb.record_every;
        }
    }
}

template <typename JT, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
    graph_kernel(const JobDev* __restrict__ jobs, const WorkItem* __restrict__ items, uint32_t n_items,
                 uint32_t* __restrict__ queue, uint32_t nsteps, uint32_t per_chain) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) JobDev s_job;
    __shared__ uint32_t s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
        const bool own = static_cast<uint32_t>(warp) < wi.nchains;
        const uint32_t chain = own ? wi.chain0 + warp : wi.chain0;
        const uint32_t npad = jb.Npad;
        const size_t v16 = (static_cast<size_t>(jb.V) + 15u) & ~static_cast<size_t>(15u);
        unsigned char* base = smem + static_cast<size_t>(warp) * per_chain;
        GMem gm;
        gm.s = reinterpret_cast<int8_t*>(base);
        gm.h = base + npad;
        gm.site = reinterpret_cast<uint16_t*>(base + 5u * static_cast<size_t>(npad));
        gm.dE = base + 5u * static_cast<size_t>(npad) + 2u * v16;
        gm.fx = reinterpret_cast<uint16_t*>(base + 5u * static_cast<size_t>(npad) + 6u * v16);
        gm.fsig = reinterpret_cast<int8_t*>(base + 5u * static_cast<size_t>(npad) + 8u * v16);
        const int partner_off = (warp & 1) ? -static_cast<int>(per_chain) : static_cast<int>(per_chain);
        const uint32_t t0 = static_cast<uint32_t>(*jb.step);
        const uint32_t t1 = static_cast<uint32_t>(
            min(static_cast<uint64_t>(t0) + nsteps, static_cast<uint64_t>(jb.step_limit)));
        uint32_t acc = 0, n_flips = 0;
        if (own) {
            const uint4* gs = reinterpret_cast<const uint4*>(jb.s + static_cast<size_t>(chain) * npad);
            uint4* ss = reinterpret_cast<uint4*>(gm.s);
            for (uint32_t q = lane; q < npad / 16; q += 32) ss[q] = gs[q];
            const uint4* gh = reinterpret_cast<const uint4*>(static_cast<const int*>(jb.h) + static_cast<size_t>(chain) * npad);
            uint4* sh = reinterpret_cast<uint4*>(gm.h);
            for (uint32_t q = lane; q < npad / 4; q += 32) sh[q] = gh[q];
            acc = jb.acc_run[chain];
        }
        __syncwarp();
        if (t1 > t0) {
            if (own) {
                graph_loop<JT>(jb, true, chain, gm, partner_off, t0, t1, acc, n_flips);
            } else {  // no chain in this warp: meet the CTA's record barriers only
                const uint32_t R = jb.record_every;
                if (R)
                    for (uint32_t p = (t0 / R + 1u) * R, r = t0 / R; p <= t1; p += R, ++r)
                        step::record<JT, 0, 1, 32, false>(jb, false, chain, r, gm.s, gm.h, partner_off, 0u, p);
            }
        }
        __syncwarp();
        if (own) {
            uint4* gs = reinterpret_cast<uint4*>(jb.s + static_cast<size_t>(chain) * npad);
            const uint4* ss = reinterpret_cast<const uint4*>(gm.s);
            for (uint32_t q = lane; q < npad / 16; q += 32) gs[q] = ss[q];
            uint4* gh = reinterpret_cast<uint4*>(static_cast<int*>(jb.h) + static_cast<size_t>(chain) * npad);
            const uint4* sh = reinterpret_cast<const uint4*>(gm.h);
            for (uint32_t q = lane; q < npad / 4; q += 32) gh[q] = sh[q];
            if (lane == 0) {
                jb.acc_run[chain] = acc;
                jb.work[2 * static_cast<size_t>(chain)] += n_flips;
                jb.work[2 * static_cast<size_t>(chain) + 1] += n_flips;
            }
        }
        __syncthreads();
    }
}

template <typename JT, int MAXT>
cudaError_t launch_t(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue, uint32_t ns,
                     uint32_t W, uint32_t per_chain, uint32_t grid, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(per_chain) * W;
    cudaError_t e = cudaFuncSetAttribute(graph_kernel<JT, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    graph_kernel<JT, MAXT><<<grid, 32 * W, smem, st>>>(jobs, items, n_items, queue, ns, per_chain);
    return cudaGetLastError();
}
template <typename JT, int MAXT>
int occupancy_t(uint32_t W, uint32_t per_chain) {
    const size_t smem = static_cast<size_t>(per_chain) * W;
    int n = 0;
    if (cudaFuncSetAttribute(graph_kernel<JT, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, graph_kernel<JT, MAXT>, 32 * W, smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace graphk

size_t graph_smem_bytes(uint32_t npad, uint32_t V, uint32_t graph) {
    return (graphk::chain_bytes(npad, V, graph) + 127u) / 128u * 128u;
}
size_t graph_table_bytes(uint32_t V) {
    const size_t V16 = (static_cast<size_t>(V) + 3u) & ~static_cast<size_t>(3u);
    return 16u * V16;
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

cudaError_t launch_graph(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                         uint64_t nsteps, uint32_t W, uint32_t per_chain, uint32_t grid, uint32_t kind,
                         uint32_t n_jobs, bool bump, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const uint32_t ns = static_cast<uint32_t>(nsteps);
    if (kind == 0)
        e = W <= 16 ? graphk::launch_t<int8_t, 512>(jobs, items, n_items, queue, ns, W, per_chain, grid, st)
                    : graphk::launch_t<int8_t, 1024>(jobs, items, n_items, queue, ns, W, per_chain, grid, st);
    else
        e = W <= 16 ? graphk::launch_t<float, 512>(jobs, items, n_items, queue, ns, W, per_chain, grid, st)
                    : graphk::launch_t<float, 1024>(jobs, items, n_items, queue, ns, W, per_chain, grid, st);
    if (e != cudaSuccess || !bump) return e;
    bump_graph_steps<<<(n_jobs + 127) / 128, 128, 0, st>>>(jobs, n_jobs, nsteps);
    return cudaGetLastError();
}

int graph_kernel_occupancy(uint32_t kind, uint32_t W, size_t per_chain) {
    const uint32_t pc = static_cast<uint32_t>(per_chain);
    if (kind == 0) return W <= 16 ? graphk::occupancy_t<int8_t, 512>(W, pc) : graphk::occupancy_t<int8_t, 1024>(W, pc);
    return W <= 16 ? graphk::occupancy_t<float, 512>(W, pc) : graphk::occupancy_t<float, 1024>(W, pc);
}

}  // namespace sk
