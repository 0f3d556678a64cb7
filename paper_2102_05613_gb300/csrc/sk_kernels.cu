// sk_kernels.cu -- sm_103a kernels of the MCMCMC sampler for the SK spin glass.
//
// One warp owns one chain.  Its spins s[Npad] (int8) and maintained local
// fields h[Npad] (int32 for +-J, float for Gaussian couplings) live in the
// warp's slice of shared memory for the whole launch; the row of J that the
// next step will need first is bulk-copied (TMA, cp.async.bulk) from global
// memory / L2 into a double-buffered shared-memory slot one step ahead,
// because the sites a step proposes do not depend on the chain's state.
//
// A Monte Carlo step of the many-configuration rule (Sec. A.2, Eq.
// eq_det_balance_graph_solution) on the star graph of App. B.2 with a uniform
// root (p_r = 1/(K+1)):
//   a1  Philox4x32-10 draws, counter (block, step, chain, stream): block 0
//       gives U0 (root: leaf iff floor(U0 (K+1) / 2^64) != 0) and U1 (node);
//       blocks 1..ceil(K/4) give site_d = floor(w N / 2^32), d = 1..K.
//       Lane l computes block 1+l (+32), so its slots are d = 4l+1..4l+4
//       (+128); block 0 is computed 32 steps at a time, one step per lane.
//   a2  the row of J at a = site_1 of the NEXT step is staged by TMA.
//   a3  candidate energies: centre root dE_d = 2 s_i h_i (i = site_d);
//       leaf root dE_1 = 2 s_a h_a, dE_d = 2 s_a h_a + 2 s_b h_b - 4 J_ab s_a s_b
//       (b = site_d != a), 0 when b = a; slot 0 (the current state) is 0.
//   a4  node choice with probability ~ exp(-beta dE): warp min, weights
//       (+-J: integer table W[(dE-min)/2] ~ 2^52 exp(-2 beta d); Gaussian:
//       expf), warp inclusive scan in slot order, u = U1 * total, first slot
//       whose prefix exceeds u.
//   a5  field update for the 0, 1 or 2 flipped spins x: h_k -= 2 s_x J_kx.
//   a6  records every R steps: E = -scale/2 sum s h, accepted count, and the
//       overlap q of chain pairs (2m, 2m+1), which share a CTA.
// The Metropolis comparator (Sec. II / IV.B) shares the layout: one site per
// step from block 0, accept iff dE <= 0 or U < exp(-beta dE).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sk_internal.h"

namespace sk {
namespace {

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

struct WarpMem {
    int8_t* s;
    void* h;
    void* row[2];
    uint64_t* bar;  // two mbarriers, one per row buffer
};

// Block 0 of each step, computed for 32 consecutive steps at once (lane l
// holds the step base + l) and broadcast by shuffle.  Steps are 32-bit.
struct Block0 {
    uint4 v;
    uint32_t base;
    bool valid;
};
__device__ __forceinline__ uint4 block0(Block0& c, uint32_t t, uint32_t chain, uint32_t c3,
                                        uint32_t k0, uint32_t k1, int lane) {
    if (!c.valid || t - c.base >= 32u) {
        c.base = t & ~31u;
        c.valid = true;
        c.v = philox4x32_10(make_uint4(0u, c.base + lane, chain, c3), k0, k1);
    }
    const int src = static_cast<int>(t - c.base);
    return make_uint4(__shfl_sync(kFull, c.v.x, src), __shfl_sync(kFull, c.v.y, src),
                      __shfl_sync(kFull, c.v.z, src), __shfl_sync(kFull, c.v.w, src));
}

// Sites of step t held by this lane: slots d = 128 g + 4 lane + e + 1.
template <int NB>
__device__ __forceinline__ void draw_sites(uint32_t (&site)[4 * NB], uint32_t t, uint32_t chain,
                                           uint32_t c3, uint32_t k0, uint32_t k1, uint32_t nblk,
                                           uint32_t N, int lane) {
#pragma unroll
    for (int g = 0; g < NB; ++g) {
        const uint32_t b = 1u + 32u * g + lane;
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        if (b <= nblk) r = philox4x32_10(make_uint4(b, t, chain, c3), k0, k1);
        site[4 * g + 0] = __umulhi(r.x, N);
        site[4 * g + 1] = __umulhi(r.y, N);
        site[4 * g + 2] = __umulhi(r.z, N);
        site[4 * g + 3] = __umulhi(r.w, N);
    }
}

// 2^x on the special-function unit (ex2.approx.ftz: relative error < 2^-22
// over the range used here, x <= 0).  exp(-beta dE) = 2^(-beta log2(e) dE).
__device__ __forceinline__ float pow2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// h_k -= c1 J[x1][k] (+ c2 J[x2][k]) for k < Npad; lane l owns elements
// 4l + 128v.  r1 is the staged row (shared memory) when STAGED, else a row of
// J in global memory; r2 (the second flip of a double move) is global.
template <typename JT, bool STAGED, bool TWO>
__device__ __forceinline__ void update_fields(typename Types<JT>::H* hf, const JT* r1, const JT* r2,
                                              int c1, int c2, uint32_t npad, int lane) {
    for (uint32_t k = 4u * lane; k < npad; k += 128u) {
        if constexpr (sizeof(JT) == 1) {
            int4 hv = *reinterpret_cast<int4*>(hf + k);
            const uint32_t j1 = STAGED ? *reinterpret_cast<const uint32_t*>(r1 + k)
                                       : __ldg(reinterpret_cast<const unsigned int*>(r1 + k));
            hv.x -= c1 * sbyte(j1, 0);
            hv.y -= c1 * sbyte(j1, 1);
            hv.z -= c1 * sbyte(j1, 2);
            hv.w -= c1 * sbyte(j1, 3);
            if constexpr (TWO) {
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
            if constexpr (TWO) {
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

// E = -scale/2 sum_k s_k h_k of the warp's chain.
template <typename JT>
__device__ __forceinline__ double chain_energy(const int8_t* S, const void* h, uint32_t npad,
                                               double scale, int lane) {
    if constexpr (sizeof(JT) == 1) {
        const int* hf = static_cast<const int*>(h);
        int acc = 0;
        for (uint32_t k = 4u * lane; k < npad; k += 128u) {
            const uint32_t sw = *reinterpret_cast<const uint32_t*>(S + k);
            const int4 hv = *reinterpret_cast<const int4*>(hf + k);
            acc += sbyte(sw, 0) * hv.x + sbyte(sw, 1) * hv.y + sbyte(sw, 2) * hv.z +
                   sbyte(sw, 3) * hv.w;
        }
        const int tot = warp_sum(acc);  // = 2 sum_{i<j} J s s, even
        return scale * static_cast<double>(-(tot / 2));
    } else {
        const float* hf = static_cast<const float*>(h);
        double acc = 0.0;
        for (uint32_t k = 4u * lane; k < npad; k += 128u) {
            const uint32_t sw = *reinterpret_cast<const uint32_t*>(S + k);
            const float4 hv = *reinterpret_cast<const float4*>(hf + k);
            acc += static_cast<double>(sbyte(sw, 0)) * hv.x + static_cast<double>(sbyte(sw, 1)) * hv.y +
                   static_cast<double>(sbyte(sw, 2)) * hv.z + static_cast<double>(sbyte(sw, 3)) * hv.w;
        }
        return -0.5 * scale * warp_sum(acc);
    }
}

// Record point shared by every warp of the CTA (two CTA barriers).
template <typename JT>
__device__ __noinline__ void record(const JobDev& jb, bool active, uint32_t chain, uint32_t rec,
                                    const int8_t* S, const void* h, const int8_t* partner_s,
                                    uint32_t acc) {
    const int lane = threadIdx.x & 31;
    const bool store = rec < jb.rec_capacity;
    if (active) {
        const double E = chain_energy<JT>(S, h, jb.Npad, jb.scale, lane);
        if (store && lane == 0) {
            jb.rec_E[static_cast<size_t>(rec) * jb.chains + chain] = E;
            jb.rec_acc[static_cast<size_t>(rec) * jb.chains + chain] = acc;
        }
    }
    __syncthreads();
    if (active && store && (chain & 1u) == 0u && chain + 1u < jb.chains) {
        int dot = 0;
        for (uint32_t k = 4u * lane; k < jb.Npad; k += 128u) {
            const uint32_t a = *reinterpret_cast<const uint32_t*>(S + k);
            const uint32_t b = *reinterpret_cast<const uint32_t*>(partner_s + k);
            dot += sbyte(a, 0) * sbyte(b, 0) + sbyte(a, 1) * sbyte(b, 1) + sbyte(a, 2) * sbyte(b, 2) +
                   sbyte(a, 3) * sbyte(b, 3);
        }
        dot = warp_sum(dot);
        if (lane == 0)
            jb.rec_q[static_cast<size_t>(rec) * (jb.chains / 2) + chain / 2] =
                static_cast<double>(dot) / static_cast<double>(jb.N);
    }
    __syncthreads();
}

// Steps t0..t1-1 of one chain.  `dead` is set after a timed-out wait: the
// warp then stops working but still meets the CTA's record barriers.
template <typename JT, int RULE, int NB>
__device__ __forceinline__ void chain_loop(const JobDev& jb, bool active, uint32_t chain,
                                           const WarpMem& wm, const int8_t* partner_s, uint32_t t0,
                                           uint32_t t1, uint32_t& acc, uint32_t& phase, bool& dead,
                                           uint32_t& n_flips, uint32_t& n_rows) {
    using H = typename Types<JT>::H;
    using W = typename Types<JT>::W;
    const int lane = threadIdx.x & 31;
    const uint32_t R = jb.record_every;
    // next record point (step count after which a record falls) and its index
    uint32_t next_rec = R ? (t0 / R + 1u) * R : 0xFFFFFFFFu;
    uint32_t rec_idx = R ? t0 / R : 0u;
    if (!active) {
        for (; R && next_rec <= t1; next_rec += R, ++rec_idx)
            record<JT>(jb, false, chain, rec_idx, wm.s, wm.h, partner_s, 0u);
        return;
    }
    // job parameters held in registers for the whole loop
    const uint32_t N = jb.N, npad = jb.Npad, K = jb.K;
    const uint32_t nblk = (K + 3u) >> 2;
    const uint32_t k0 = static_cast<uint32_t>(jb.seed), k1 = static_cast<uint32_t>(jb.seed >> 32);
    const uint32_t c3 = jb.stream & 0xFFFFFFu;  // domain 0: step draws
    const JT* __restrict__ Jg = static_cast<const JT*>(jb.J);
    const uint32_t rowbytes = npad * static_cast<uint32_t>(sizeof(JT));
    const W* __restrict__ Wt = reinterpret_cast<const W*>(jb.W);
    const uint32_t wlen = jb.wlen;
    const float nbl2 = -jb.beta_eff * 1.4426950408889634f;  // -beta log2(e)
    int32_t* trace = (chain < jb.trace_chains) ? jb.trace + static_cast<size_t>(chain) * jb.trace_steps
                                               : nullptr;
    const uint32_t trace_end = trace ? static_cast<uint32_t>(jb.trace_steps) : 0u;
    int8_t* S = wm.s;
    H* hf = static_cast<H*>(wm.h);

    Block0 bc;
    bc.valid = false;
    uint32_t site[4 * NB];

    // prologue: the first step's row
    uint32_t first;
    if constexpr (RULE == 0) {
        draw_sites<NB>(site, t0, chain, c3, k0, k1, nblk, N, lane);
        first = __shfl_sync(kFull, site[0], 0);
    } else {
        first = __umulhi(block0(bc, t0, chain, c3, k0, k1, lane).x, N);
    }
    if (lane == 0 && !dead) {
        fence_proxy_async();
        bulk_load(wm.row[t0 & 1u], Jg + static_cast<size_t>(first) * npad, rowbytes,
                  &wm.bar[t0 & 1u]);
    }

    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t buf = t & 1u;
        const uint4 b0 = block0(bc, t, chain, c3, k0, k1, lane);
        const unsigned long long U1 = (static_cast<unsigned long long>(b0.w) << 32) | b0.z;
        int sel = 0;  // slot chosen (Metropolis: accepted)
        int nflip = 0;
        int rows = 0;  // J rows this step needs: row a of a leaf root, flipped spins' rows
        uint32_t x1 = 0, x2 = 0;
        bool x1_staged = false;

        // stage the row the next step needs first
        uint32_t nsite[4 * NB];
        if (t + 1u < t1) {
            uint32_t nx;
            if constexpr (RULE == 0) {
                draw_sites<NB>(nsite, t + 1u, chain, c3, k0, k1, nblk, N, lane);
                nx = __shfl_sync(kFull, nsite[0], 0);
            } else {
                nx = __umulhi(block0(bc, t + 1u, chain, c3, k0, k1, lane).x, N);
            }
            __syncwarp();  // every lane is done with buffer buf^1 (step t-1)
            if (lane == 0 && !dead) {
                fence_proxy_async();
                bulk_load(wm.row[buf ^ 1u], Jg + static_cast<size_t>(nx) * npad, rowbytes,
                          &wm.bar[buf ^ 1u]);
            }
        }
        if (!dead) {
            // every lane waits; the outcome is made warp-uniform
            const bool ok = __all_sync(kFull, mbar_wait_bounded(&wm.bar[buf], (phase >> buf) & 1u));
            phase ^= 1u << buf;
            if (!ok) {
                dead = true;
                if (lane == 0) atomicExch(jb.err, kDevTimeout);
            }
        }
        const JT* rowA = static_cast<const JT*>(wm.row[buf]);

        if (!dead) {
            if constexpr (RULE == 1) {
                // ---- Metropolis: one single-flip proposal ----
                const uint32_t i = __umulhi(b0.x, N);
                const int si = S[i];
                const H dE = static_cast<H>(2 * si) * hf[i];
                bool accept;
                if constexpr (sizeof(JT) == 1) {
                    const uint32_t k = static_cast<uint32_t>(dE) >> 1;
                    accept = dE <= 0 || (k < wlen && (U1 >> 11) < __ldg(&Wt[k]));
                } else {
                    accept = dE <= 0.0f || static_cast<float>(U1 >> 40) * 0x1p-24f < pow2(nbl2 * dE);
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
                const unsigned long long U0 = (static_cast<unsigned long long>(b0.y) << 32) | b0.x;
                const bool leaf = __umul64hi(U0, static_cast<unsigned long long>(K) + 1ull) != 0ull;
                const uint32_t a = __shfl_sync(kFull, site[0], 0);
                const int sa = S[a];
                const H dEa = static_cast<H>(2 * sa) * hf[a];
                H dE[4 * NB];
                H mloc = 0;
#pragma unroll
                for (int q = 0; q < 4 * NB; ++q) {
                    const uint32_t d = 128u * (q >> 2) + 4u * lane + (q & 3) + 1u;
                    const uint32_t i = site[q];
                    const int si = S[i];
                    const H hi = hf[i];
                    H v;
                    if (!leaf) {
                        v = static_cast<H>(2 * si) * hi;
                    } else if (d == 1u) {
                        v = dEa;
                    } else if (i == a) {
                        v = 0;
                    } else {
                        v = dEa + static_cast<H>(2 * si) * hi -
                            static_cast<H>(4 * sa * si) * static_cast<H>(rowA[i]);
                    }
                    dE[q] = v;
                    if (d <= K) mloc = mloc < v ? mloc : v;
                }
                const H m = warp_min(mloc);
                // weights in slot order
                W w[4 * NB];
                W gsum[NB];
#pragma unroll
                for (int g = 0; g < NB; ++g) gsum[g] = 0;
#pragma unroll
                for (int q = 0; q < 4 * NB; ++q) {
                    const uint32_t d = 128u * (q >> 2) + 4u * lane + (q & 3) + 1u;
                    W x = 0;
                    if (d <= K) {
                        if constexpr (sizeof(JT) == 1) {
                            const uint32_t idx = static_cast<uint32_t>(dE[q] - m) >> 1;
                            x = idx < wlen ? __ldg(&Wt[idx]) : 0ull;
                        } else {
                            x = pow2(nbl2 * (dE[q] - m));
                        }
                    }
                    w[q] = x;
                    gsum[q >> 2] += x;
                }
                W w0;
                if constexpr (sizeof(JT) == 1) {
                    const uint32_t idx0 = static_cast<uint32_t>(-m) >> 1;
                    w0 = idx0 < wlen ? __ldg(&Wt[idx0]) : 0ull;
                } else {
                    w0 = pow2(-nbl2 * m);
                }
                W incl[NB], tot[NB];
                W total = w0;
#pragma unroll
                for (int g = 0; g < NB; ++g) {
                    incl[g] = warp_incl_scan(gsum[g], lane);
                    tot[g] = __shfl_sync(kFull, incl[g], 31);
                    total += tot[g];
                }
                W u;
                if constexpr (sizeof(JT) == 1) {
                    u = __umul64hi(U1, total);
                } else {
                    u = static_cast<float>(U1 >> 40) * 0x1p-24f * total;
                    if (u >= total) u = nextafterf(total, 0.0f);
                }
                // first slot whose inclusive prefix exceeds u
                int sel_d = 0;
                uint32_t sel_site = 0;
                if (!(u < w0)) {
                    W base = w0;
#pragma unroll
                    for (int g = 0; g < NB; ++g) {
                        const unsigned ball = __ballot_sync(kFull, base + incl[g] > u);
                        if (ball) {
                            const int L = __ffs(ball) - 1;
                            W run = base + (incl[g] - gsum[g]);
                            int my_e = -1;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                if (my_e < 0 && w[4 * g + e] > W(0)) {
                                    run += w[4 * g + e];
                                    if (run > u) my_e = e;
                                }
                            }
                            if (my_e < 0) {  // rounding guard: last positive weight
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (w[4 * g + e] > W(0)) my_e = e;
                            }
                            uint32_t my_site = 0;
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (e == my_e) my_site = site[4 * g + e];
                            const int e_sel = __shfl_sync(kFull, my_e, L);
                            sel_site = __shfl_sync(kFull, my_site, L);
                            sel_d = 128 * g + 4 * L + e_sel + 1;
                            break;
                        }
                        base += tot[g];
                    }
                }
                sel = sel_d;
                if (sel_d == 0) {
                    nflip = 0;
                } else if (!leaf) {
                    nflip = 1;
                    x1 = sel_site;
                    x1_staged = (sel_site == a);
                } else if (sel_d == 1) {
                    nflip = 1;
                    x1 = a;
                    x1_staged = true;
                } else if (sel_site == a) {
                    nflip = 0;
                } else {
                    nflip = 2;
                    x1 = a;
                    x1_staged = true;
                    x2 = sel_site;
                }
                rows = leaf ? 1 + (nflip == 2 ? 1 : 0) : nflip;
            }
            // ---- field update and flips ----
            if (nflip) {
                const int c1 = 2 * S[x1];
                const int c2 = nflip == 2 ? 2 * S[x2] : 0;
                const JT* g1 = Jg + static_cast<size_t>(x1) * npad;
                const JT* g2 = Jg + static_cast<size_t>(x2) * npad;
                if (nflip == 2)
                    update_fields<JT, true, true>(hf, rowA, g2, c1, c2, npad, lane);
                else if (x1_staged)
                    update_fields<JT, true, false>(hf, rowA, nullptr, c1, 0, npad, lane);
                else
                    update_fields<JT, false, false>(hf, g1, nullptr, c1, 0, npad, lane);
                __syncwarp();
                if (lane == 0) {
                    S[x1] = static_cast<int8_t>(-S[x1]);
                    if (nflip == 2) S[x2] = static_cast<int8_t>(-S[x2]);
                }
                acc += 1u;
            }
            n_flips += static_cast<uint32_t>(nflip);
            n_rows += static_cast<uint32_t>(rows);
            if (t < trace_end && lane == 0) trace[t] = sel;
            __syncwarp();
        }
        if constexpr (RULE == 0) {
#pragma unroll
            for (int q = 0; q < 4 * NB; ++q) site[q] = nsite[q];
        }
        if (t + 1u == next_rec) {
            record<JT>(jb, !dead, chain, rec_idx, S, hf, partner_s, acc);
            acc = 0;
            next_rec += R;
            ++rec_idx;
        }
    }
}

// MAXT bounds the CTA size and so sets the register budget per thread
// (65536 / MAXT): 1024 -> 64, 640 -> 96, 512 -> 128 registers.
template <typename JT, int RULE, int NB, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
    step_kernel(const JobDev* __restrict__ jobs, const WorkItem* __restrict__ items,
                uint32_t n_items, uint32_t* __restrict__ queue, uint32_t nsteps,
                uint32_t per_warp) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) JobDev s_job;
    __shared__ __align__(8) uint64_t bars[64];
    __shared__ uint32_t s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        mbar_init(&bars[2 * warp], 1);
        mbar_init(&bars[2 * warp + 1], 1);
    }
    fence_mbar_init();
    __syncthreads();
    uint32_t phase = 0;
    bool dead = false;  // a bounded wait of this warp expired: skip all further work
    constexpr size_t bj = sizeof(JT);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= n_items) break;
        const WorkItem wi = items[it];
        if (threadIdx.x < sizeof(JobDev) / 16)
            reinterpret_cast<uint4*>(&s_job)[threadIdx.x] =
                reinterpret_cast<const uint4*>(&jobs[wi.job])[threadIdx.x];
        __syncthreads();
        const JobDev& jb = s_job;
        const bool active = static_cast<uint32_t>(warp) < wi.nchains;
        const uint32_t chain = wi.chain0 + warp;
        const uint32_t npad = jb.Npad;
        WarpMem wm;
        unsigned char* base = smem + static_cast<size_t>(warp) * per_warp;
        wm.s = reinterpret_cast<int8_t*>(base);
        wm.h = base + npad;
        wm.row[0] = base + 5 * static_cast<size_t>(npad);
        wm.row[1] = base + (5 + bj) * static_cast<size_t>(npad);
        wm.bar = &bars[2 * warp];
        const int8_t* partner_s =
            reinterpret_cast<const int8_t*>(smem + static_cast<size_t>(warp ^ 1) * per_warp);
        const uint32_t t0 = static_cast<uint32_t>(*jb.step);
        const uint32_t t1 = static_cast<uint32_t>(min(static_cast<uint64_t>(t0) + nsteps,
                                                      static_cast<uint64_t>(jb.step_limit)));
        uint32_t acc = 0, n_flips = 0, n_rows = 0;
        if (active) {
            // load the chain's state: spins (npad bytes), fields (4 npad bytes)
            const uint4* gs = reinterpret_cast<const uint4*>(jb.s + static_cast<size_t>(chain) * npad);
            uint4* ss = reinterpret_cast<uint4*>(wm.s);
            for (uint32_t k = lane; k < npad / 16; k += 32) ss[k] = gs[k];
            const uint4* gh = reinterpret_cast<const uint4*>(static_cast<const int*>(jb.h) +
                                                             static_cast<size_t>(chain) * npad);
            uint4* sh = reinterpret_cast<uint4*>(wm.h);
            for (uint32_t k = lane; k < npad / 4; k += 32) sh[k] = gh[k];
            acc = jb.acc_run[chain];
        }
        __syncwarp();
        if (t1 > t0)
            chain_loop<JT, RULE, NB>(jb, active, chain, wm, partner_s, t0, t1, acc, phase, dead,
                                     n_flips, n_rows);
        __syncwarp();
        if (active) {
            uint4* gs = reinterpret_cast<uint4*>(jb.s + static_cast<size_t>(chain) * npad);
            const uint4* ss = reinterpret_cast<const uint4*>(wm.s);
            for (uint32_t k = lane; k < npad / 16; k += 32) gs[k] = ss[k];
            uint4* gh = reinterpret_cast<uint4*>(static_cast<int*>(jb.h) + static_cast<size_t>(chain) * npad);
            const uint4* sh = reinterpret_cast<const uint4*>(wm.h);
            for (uint32_t k = lane; k < npad / 4; k += 32) gh[k] = sh[k];
            if (lane == 0) {
                jb.acc_run[chain] = acc;
                jb.work[2 * static_cast<size_t>(chain)] += n_flips;
                jb.work[2 * static_cast<size_t>(chain) + 1] += n_rows;
            }
        }
        __syncthreads();  // s_job and the smem slices are reused by the next item
    }
}

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

template <typename JT, int RULE, int NB, int MAXT>
cudaError_t launch_variant(const JobDev* jobs, const WorkItem* items, uint32_t n_items,
                           uint32_t* queue, uint32_t nsteps, uint32_t W, uint32_t per_warp,
                           uint32_t grid, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(per_warp) * W;
    cudaError_t e = cudaFuncSetAttribute(step_kernel<JT, RULE, NB, MAXT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    step_kernel<JT, RULE, NB, MAXT><<<grid, 32 * W, smem, st>>>(jobs, items, n_items, queue, nsteps, per_warp);
    return cudaGetLastError();
}

template <typename JT, int RULE, int NB, int MAXT>
int occupancy_variant(uint32_t W, size_t smem) {
    int n = 0;
    if (cudaFuncSetAttribute(step_kernel<JT, RULE, NB, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<JT, RULE, NB, MAXT>, 32 * W, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

// The register budget follows the CTA size: the largest variant that fits W warps.
template <typename JT, int RULE, int NB>
cudaError_t launch_class(const JobDev* jobs, const WorkItem* items, uint32_t n_items,
                         uint32_t* queue, uint32_t nsteps, uint32_t W, uint32_t per_warp,
                         uint32_t grid, cudaStream_t st) {
    if (W <= 16) return launch_variant<JT, RULE, NB, 512>(jobs, items, n_items, queue, nsteps, W, per_warp, grid, st);
    if (W <= 20) return launch_variant<JT, RULE, NB, 640>(jobs, items, n_items, queue, nsteps, W, per_warp, grid, st);
    return launch_variant<JT, RULE, NB, 1024>(jobs, items, n_items, queue, nsteps, W, per_warp, grid, st);
}

template <typename JT, int RULE, int NB>
int occupancy_class(uint32_t W, size_t smem) {
    if (W <= 16) return occupancy_variant<JT, RULE, NB, 512>(W, smem);
    if (W <= 20) return occupancy_variant<JT, RULE, NB, 640>(W, smem);
    return occupancy_variant<JT, RULE, NB, 1024>(W, smem);
}

}  // namespace

cudaError_t launch_step(const JobDev* jobs, const WorkItem* items, uint32_t n_items,
                        uint32_t* queue, uint64_t nsteps, uint32_t W, uint32_t per_warp,
                        uint32_t grid, int cls, uint32_t n_jobs, bool bump, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const uint32_t ns = static_cast<uint32_t>(nsteps);
    switch (cls) {
        case 0: e = launch_class<int8_t, 0, 1>(jobs, items, n_items, queue, ns, W, per_warp, grid, st); break;
        case 1: e = launch_class<int8_t, 0, 2>(jobs, items, n_items, queue, ns, W, per_warp, grid, st); break;
        case 2: e = launch_class<int8_t, 1, 1>(jobs, items, n_items, queue, ns, W, per_warp, grid, st); break;
        case 4: e = launch_class<float, 0, 1>(jobs, items, n_items, queue, ns, W, per_warp, grid, st); break;
        case 5: e = launch_class<float, 0, 2>(jobs, items, n_items, queue, ns, W, per_warp, grid, st); break;
        case 6: e = launch_class<float, 1, 1>(jobs, items, n_items, queue, ns, W, per_warp, grid, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || !bump) return e;
    bump_steps<<<(n_jobs + 127) / 128, 128, 0, st>>>(jobs, n_jobs, nsteps);
    return cudaGetLastError();
}

int step_kernel_occupancy(int cls, uint32_t W, size_t smem) {
    switch (cls) {
        case 0: return occupancy_class<int8_t, 0, 1>(W, smem);
        case 1: return occupancy_class<int8_t, 0, 2>(W, smem);
        case 2: return occupancy_class<int8_t, 1, 1>(W, smem);
        case 4: return occupancy_class<float, 0, 1>(W, smem);
        case 5: return occupancy_class<float, 0, 2>(W, smem);
        case 6: return occupancy_class<float, 1, 1>(W, smem);
        default: return 0;
    }
}

int step_class(uint32_t kind, uint32_t rule, uint32_t K) {
    return static_cast<int>(kind) * 4 + (rule == 1 ? 2 : (K > 128 ? 1 : 0));
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
