// sk_recompute.cu -- the periodic local-field recompute H = S J^T of all
// chains of a run on the fifth-generation tensor cores (tcgen05), and the
// drift check / resynchronisation of the maintained fields against it.
//
// H[c][n] = sum_k S[c][k] J[n][k] (J symmetric), M = chains, N = K = Npad.
//   +-J couplings:     S and J as FP8 e4m3 (+-1 and 0 are exact), kind::f8f6f4,
//                      FP32 accumulation: every partial sum is an integer below
//                      2^24, so H is exact and must equal the maintained int32
//                      fields bit for bit.
//   Gaussian couplings: S as bf16 (+-1 exact), J split into `terms` bf16
//                      matrices J = J1 + J2 + J3 (three round-to-nearest terms
//                      reproduce every fp32 value exactly), kind::f16 with FP32
//                      accumulation of all terms into one accumulator.
//
// A persistent CTA per SM works through 128 x 256 output tiles with three
// roles: one thread of warp 0 streams A and B tiles with TMA (128-byte
// swizzle) through a 4-stage mbarrier ring, one thread of warp 1 issues the
// MMAs (K = 32 bytes each) into one of two 128-lane x 256-column FP32
// accumulators in tensor memory (all 512 columns) and commits each stage back
// to its "empty" barrier and each finished tile to its accumulator's "full"
// barrier, and warps 2-9 (two per 32-lane quadrant of tensor memory, one per
// half of the columns) read the finished accumulator with tcgen05.ld and
// compare it with (or replace) the maintained fields, then hand the
// accumulator back -- so one tile's epilogue overlaps the next tile's main
// loop, with eight warps' loads of the fields in flight.  Every wait is bounded; an expired wait
// sets the run's error word and stops the CTA's roles.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <set>
#include <vector>

#include "sk_device.cuh"
#include "sk_internal.h"

namespace sk {
namespace {

constexpr uint32_t BM = 128, BN = 256, NS = 4;  // 4 pipeline stages, one CTA per SM
constexpr uint32_t TILE_A = BM * 128, TILE_B = BN * 128;  // bytes, 128 B of K per row
constexpr uint32_t STAGE_BYTES = TILE_A + TILE_B;
constexpr uint32_t EW = 8;                                 // epilogue warps: 2 per tensor-memory quadrant
constexpr uint32_t SMEM_BYTES = NS * STAGE_BYTES + 1024;  // + 1 KB alignment slack
constexpr uint32_t TMEM_COLS = 512;                        // two 256-column accumulators
constexpr uint32_t WS_THREADS = 64 + 32 * EW;              // producer, MMA, epilogue warps
constexpr long long kBudget = 4000000000ll;  // ~2 s of clock cycles per wait

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity) {
    if (try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!try_wait(bar, parity))
        if (clock64() - t0 > kBudget) return false;
    return true;
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// Shared-memory matrix descriptor: K-major tile, 128-byte rows with the
// 128-byte swizzle, 8-row groups 1024 bytes apart (tile base 1024-aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);  // start address
    d |= static_cast<uint64_t>(1) << 16;                 // leading byte offset (unused here)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;         // stride byte offset
    d |= static_cast<uint64_t>(1) << 46;                 // descriptor version
    d |= static_cast<uint64_t>(2) << 61;                 // 128-byte swizzle
    return d;
}
// Instruction descriptor: FP32 accumulator, A/B format code `fmt` (kind::f16:
// 1 = bf16; kind::f8f6f4: 0 = e4m3), both K-major, N = 256, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((BN >> 3) << 17) | ((BM >> 4) << 24);
}

template <bool F8>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (F8) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct Args {
    void* h;                        // maintained fields [chains][npad]: int32 (+-J) or float
    const int8_t* s;                // spins [chains][npad]
    float* out;                     // OUTPUT mode: H [chains][npad]
    double* dE;                     // per chain: sum_n s_n (h_n - H_n)
    unsigned long long* stats;      // [0] max |h - H| (double bits), [1] mismatches, [2] max |dE|
    unsigned int* cnt;              // per 32 chains: epilogue warps done with their rows (or null)
    double scale;                   // energy scale of the drift
    int* err;
    uint32_t chains, npad, kblocks, terms, mode;  // mode: 0 check, 1 resync, 2 output, 3 set fields
    uint32_t pm1;
    uint32_t fault;                 // kFaultWithholdTile: tests of the bounded waits
    uint32_t compute_only;          // tensor-pipe probe: operands loaded once, MMAs only
};

// Several operand sets in one launch: the tensor maps and arguments of each
// set in global memory (maps 64-byte aligned, written before the launch).
struct alignas(64) BatchJob {
    CUtensorMap A, B[3];
    Args args;
};
struct BatchTask {
    uint32_t job, m0, n0, pad;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Byte e (0..3) of a 32-bit word as a signed value.
__device__ __forceinline__ int sbyte32(uint32_t w, int e) {
    return static_cast<int>(static_cast<int32_t>(w << (24 - 8 * e)) >> 24);
}
__device__ __forceinline__ uint32_t word_of(const uint4& q, int e) {
    return e == 0 ? q.x : e == 1 ? q.y : e == 2 ? q.z : q.w;
}

// The epilogue of one finished accumulator for one warp: accumulator rows
// row0 .. row0 + 31 (tcgen05.ld 32x32b gives lane l the accumulator row
// row0 + l), the NCB blocks of 32 columns starting at column c0.  Each lane
// reads and writes its own row's segment of the fields and spins -- 128
// bytes of int32 / float fields as eight 16-byte loads and 32 bytes of spins
// as two -- so no transpose is needed, and the row's sum s (h - H) stays in
// the lane (an int32 for +-J, exact; a float otherwise) until one
// double-precision atomic per row.  A block's loads are issued before its
// accumulator columns are read from tensor memory (the first block's before
// the wait for the accumulator), so that their round trip covers that read.
constexpr uint32_t NCB = BN / 2 / 32;  // column blocks per epilogue warp and tile
// One column block's fields and spins of this lane's row (check and resync).
struct RowBlock {
    uint4 h[8], s[2];
};
__device__ __forceinline__ void load_row_block(RowBlock& rb, const Args& args, uint32_t row, uint32_t n, bool ok) {
    if (args.mode < 2 && ok && n < args.npad) {  // npad is a multiple of 32
        const size_t idx = static_cast<size_t>(row) * args.npad + n;  // 32-element aligned
        const uint4* hp = reinterpret_cast<const uint4*>(static_cast<const unsigned int*>(args.h) + idx);
#pragma unroll
        for (int q = 0; q < 8; ++q) rb.h[q] = __ldg(hp + q);
        const uint4* sp = reinterpret_cast<const uint4*>(args.s + idx);
        rb.s[0] = __ldg(sp);
        rb.s[1] = __ldg(sp + 1);
    }
}
// first: the first column block, loaded by the caller (before it waited for
// the accumulator) with load_row_block(first, args, row0 + lane, n0 + c0, ..).
__device__ __forceinline__ void epilogue_rows(uint32_t taddr, const Args& args, uint32_t row0, uint32_t n0,
                                              uint32_t c0, bool tile_ok, const RowBlock& first) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t row = row0 + lane;
    const bool row_ok = tile_ok && row < args.chains;
    const bool reads = args.mode < 2;
    int isum = 0, imax = 0;
    float fsum = 0.0f, pmax = 0.0f;
    unsigned mism = 0;
    RowBlock rb = first;
#pragma unroll
    for (uint32_t cb = 0; cb < NCB; ++cb) {
        if (cb > 0) load_row_block(rb, args, row, n0 + c0 + 32u * cb, row_ok);
        const uint32_t n = n0 + c0 + 32u * cb;
        const bool ok = row_ok && n < args.npad;
        const size_t idx = static_cast<size_t>(row) * args.npad + n;
        uint32_t v[32];
        tmem_ld32(taddr + c0 + 32u * cb, v);  // every lane: the load is warp-collective
        if (!ok) continue;
        if (args.mode >= 2) {  // output H, or the fields of a start state (h = H)
            uint4* dst = args.mode == 2 ? reinterpret_cast<uint4*>(args.out + idx)
                                        : reinterpret_cast<uint4*>(static_cast<unsigned int*>(args.h) + idx);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                uint4 w = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                if (args.mode == 3 && args.pm1) {
                    w.x = static_cast<uint32_t>(__float2int_rn(__uint_as_float(w.x)));
                    w.y = static_cast<uint32_t>(__float2int_rn(__uint_as_float(w.y)));
                    w.z = static_cast<uint32_t>(__float2int_rn(__uint_as_float(w.z)));
                    w.w = static_cast<uint32_t>(__float2int_rn(__uint_as_float(w.w)));
                }
                dst[q] = w;
            }
            continue;
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float H = __uint_as_float(v[k]);
            const uint32_t hw = word_of(rb.h[k >> 2], k & 3);
            const int sv = sbyte32(word_of(rb.s[k >> 4], (k >> 2) & 3), k & 3);
            if (args.pm1) {
                const int d = static_cast<int>(hw) - __float2int_rn(H);
                mism += d != 0;
                imax = max(imax, abs(d));
                isum += sv * d;
            } else {
                const float d = __uint_as_float(hw) - H;
                pmax = fmaxf(pmax, fabsf(d));
                fsum = fmaf(static_cast<float>(sv), d, fsum);
            }
        }
        if (args.mode == 1) {  // resync: the maintained fields become H
            uint4* dst = reinterpret_cast<uint4*>(static_cast<unsigned int*>(args.h) + idx);
#pragma unroll
            for (int q = 0; q < 8; ++q) dst[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
    }
    if (tile_ok && reads) {
        if (row_ok) atomicAdd(&args.dE[row], args.pm1 ? static_cast<double>(isum) : static_cast<double>(fsum));
        // the warp's maximum and mismatch count, then one atomic each (every
        // warp of every tile updates the same two words)
        if (args.pm1) {
            imax = __reduce_max_sync(0xffffffffu, imax);
        } else {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
        }
        const unsigned mw = __reduce_add_sync(0xffffffffu, mism);
        if (lane == 0) {
            const double dmax = args.pm1 ? static_cast<double>(imax) : static_cast<double>(pmax);
            atomicMax(&args.stats[0], static_cast<unsigned long long>(__double_as_longlong(dmax)));
            if (mw) atomicAdd(&args.stats[1], static_cast<unsigned long long>(mw));
        }
        if (args.cnt) {
            // the energy drift of these 32 chains is complete once the epilogue
            // warps of all their tiles (two column halves each) have added to
            // it: the last of them takes |scale/2 dE| of each chain into the
            // maximum and clears dE and the count for the next recompute
            const uint32_t arrivals = 2u * ((args.npad + BN - 1) / BN);
            unsigned last = 0;
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                last = atomicAdd(&args.cnt[row0 / 32u], 1u) == arrivals - 1u;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                double e = 0.0;
                if (row < args.chains)
                    e = fabs(0.5 * args.scale * __longlong_as_double(static_cast<long long>(
                                                    atomicExch(reinterpret_cast<unsigned long long*>(&args.dE[row]), 0ull))));
                unsigned long long bmax = static_cast<unsigned long long>(__double_as_longlong(e));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, bmax, o);
                    bmax = y > bmax ? y : bmax;
                }
                if (lane == 0) {
                    atomicMax(&args.stats[2], bmax);  // non-negative doubles order as their bits
                    args.cnt[row0 / 32u] = 0u;
                }
            }
        }
    }
    __syncwarp();
}

// The persistent kernel.  BATCH: task t is tasks[t] of operand set
// jobs[tasks[t].job] (maps in global memory, acquired before use); else the
// maps and arguments are the kernel's parameters and task t is output tile
// (t / tiles_n, t % tiles_n).
template <bool F8, bool BATCH>
__global__ void __launch_bounds__(WS_THREADS, 1)
    recompute_ws_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB0,
                        const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2,
                        const Args args0, const BatchJob* __restrict__ jobs, const BatchTask* __restrict__ tasks,
                        uint32_t ntasks, uint32_t tiles_n) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull[2], tempty[2], drain;
    __shared__ uint32_t tmem_holder;
    __shared__ int dead;
    // 128-byte-swizzled tiles must start on a 1024-byte boundary of shared memory
    unsigned char* smem = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t kElems = F8 ? 128u : 64u;  // K elements per 128-byte row
    constexpr uint32_t idesc = instr_desc(F8 ? 0u : 1u);
    volatile int* vdead = &dead;

    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < NS; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[i])) : "memory");
        }
        for (uint32_t i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&tfull[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&tempty[i])), "r"(EW) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&drain)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        dead = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;

    // the task's maps, arguments and tile origin
    auto task = [&](uint32_t t, const CUtensorMap*& A, const CUtensorMap* (&B)[3], const Args*& a, uint32_t& m0,
                    uint32_t& n0) {
        if constexpr (BATCH) {
            const BatchTask tk = tasks[t];
            const BatchJob& j = jobs[tk.job];
            A = &j.A;
            B[0] = &j.B[0];
            B[1] = &j.B[1];
            B[2] = &j.B[2];
            a = &j.args;
            m0 = tk.m0;
            n0 = tk.n0;
        } else {
            A = &tA;
            B[0] = &tB0;
            B[1] = &tB1;
            B[2] = &tB2;
            a = &args0;
            m0 = (t / tiles_n) * BM;
            n0 = (t % tiles_n) * BN;
        }
    };

    if (warp == 0) {
        if (lane == 0) {  // producer: A (spins) and B (couplings, term by term) tiles by TMA
            uint32_t g = 0;
            uint32_t withheld = 0xFFFFFFFFu;  // a stage a test of the bounded waits leaves unfilled
            for (uint32_t t = blockIdx.x; t < ntasks && !*vdead; t += gridDim.x) {
                const CUtensorMap* A;
                const CUtensorMap* B[3];
                const Args* a;
                uint32_t m0, n0;
                task(t, A, B, a, m0, n0);
                if constexpr (BATCH) {  // maps written to global memory by a copy: acquire them for TMA
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(A) : "memory");
                    for (int q = 0; q < 3; ++q)
                        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(B[q]) : "memory");
                }
                const uint32_t total = a->terms * a->kblocks;
                for (uint32_t i = 0; i < total; ++i, ++g) {
                    const uint32_t st = g % NS;
                    if (a->compute_only && g >= NS) break;  // the probe fills the ring once
                    if (g >= NS && !wait_bounded(saddr(&empty[st]), ((g / NS) - 1u) & 1u)) {
                        atomicExch(a->err, kDevTimeout);
                        *vdead = 1;
                    }
                    if (*vdead) break;
                    if ((a->fault & kFaultWithholdTile) && blockIdx.x == 0 && g == 0) {
                        withheld = g;
                        continue;
                    }
                    const uint32_t term = i / a->kblocks, kb = i % a->kblocks;
                    unsigned char* sa = smem + st * STAGE_BYTES;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&full[st])),
                                 "r"(STAGE_BYTES)
                                 : "memory");
                    tma_2d(saddr(sa), A, static_cast<int>(kb * kElems), static_cast<int>(m0), saddr(&full[st]));
                    tma_2d(saddr(sa + TILE_A), B[term], static_cast<int>(kb * kElems), static_cast<int>(n0),
                           saddr(&full[st]));
                }
            }
            // the copies of the last NS stages issued have landed before the
            // CTA may leave (at once after a normal run, where the MMA warp
            // consumed them; bounded after an expired wait)
            for (uint32_t q = g > NS ? g - NS : 0u; q < g; ++q)
                if (q != withheld) wait_bounded(saddr(&full[q % NS]), (q / NS) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer: 4 MMAs of K = 32 bytes per stage into accumulator j % 2
            uint32_t g = 0, j = 0;
            for (uint32_t t = blockIdx.x; t < ntasks && !*vdead; t += gridDim.x, ++j) {
                const CUtensorMap* A;
                const CUtensorMap* B[3];
                const Args* a;
                uint32_t m0, n0;
                task(t, A, B, a, m0, n0);
                const uint32_t b = j & 1u;
                if (j >= 2 && !wait_bounded(saddr(&tempty[b]), ((j >> 1) - 1u) & 1u)) {  // epilogue done with it
                    atomicExch(a->err, kDevTimeout);
                    *vdead = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + 256u * b;
                const uint32_t total = a->terms * a->kblocks;
                for (uint32_t i = 0; i < total; ++i, ++g) {
                    const uint32_t st = g % NS;
                    // (the probe waits for each stage once, then reuses it)
                    if ((!a->compute_only || g < NS) && !wait_bounded(saddr(&full[st]), (g / NS) & 1u)) {
                        atomicExch(a->err, kDevTimeout);
                        *vdead = 1;
                    }
                    if (*vdead) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = saddr(smem + st * STAGE_BYTES);
                    const uint32_t sb = sa + TILE_A;
#pragma unroll
                    for (uint32_t kk = 0; kk < 4; ++kk)
                        mma<F8>(acc, sw128_desc(sa + 32 * kk), sw128_desc(sb + 32 * kk), idesc, (i | kk) != 0u);
                    if (!a->compute_only) mma_commit(saddr(&empty[st]));
                }
                mma_commit(saddr(&tfull[b]));  // completes when the tile's MMAs have
            }
            // every MMA issued has finished before the accumulators' tensor
            // memory is released (at once after a normal run; bounded after an
            // expired wait)
            mma_commit(saddr(&drain));
            wait_bounded(saddr(&drain), 0u);
        }
    } else {
        // epilogue warps 2..9: tensor-memory lane quadrant warp % 4, column
        // half (warp - 2) / 4
        const uint32_t qd = warp & 3u, half = (warp - 2u) >> 2;
        uint32_t j = 0;
        for (uint32_t t = blockIdx.x; t < ntasks; t += gridDim.x, ++j) {
            const CUtensorMap* A;
            const CUtensorMap* B[3];
            const Args* a;
            uint32_t m0, n0;
            task(t, A, B, a, m0, n0);
            const uint32_t b = j & 1u;
            // the first column block's fields and spins do not depend on the
            // accumulator: their loads go out before the wait for it
            RowBlock first;
            if (!a->compute_only)
                load_row_block(first, *a, m0 + qd * 32u + lane, n0 + half * (BN / 2), m0 + qd * 32u + lane < a->chains);
            // every lane waits; the outcome is made warp-uniform
            const bool ok = __all_sync(0xffffffffu, !*vdead && wait_bounded(saddr(&tfull[b]), (j >> 1) & 1u));
            if (!ok && lane == 0) {
                atomicExch(a->err, kDevTimeout);
                *vdead = 1;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const bool live = __all_sync(0xffffffffu, !*vdead);
            if (!a->compute_only)
                epilogue_rows(tmem + ((qd * 32u) << 16) + 256u * b, *a, m0 + qd * 32u, n0, half * (BN / 2),
                              ok && live, first);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(saddr(&tempty[b]));
            if (!ok) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 1;
    }
    return n;
}

// Spin operands of several runs (blockIdx.y = run): +-1 -> e4m3 / bf16.
struct SegSpins {
    const int8_t* s;
    void* o;
    size_t n;
};
__global__ void spins_to_op_batch(const SegSpins* __restrict__ seg, uint32_t bf16) {
    const SegSpins g = seg[blockIdx.y];
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < g.n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int v = g.s[i];
        if (bf16)
            static_cast<uint16_t*>(g.o)[i] = v == 0 ? 0 : (v > 0 ? 0x3F80 : 0xBF80);
        else
            static_cast<uint8_t*>(g.o)[i] = v == 0 ? 0 : (v > 0 ? 0x38 : 0xB8);
    }
}

// max over chains of |dE| = |-scale/2 sum s (h - H)| into stats[2]; clears dE.
__global__ void finish_energy(double* dE, uint32_t chains, double scale, unsigned long long* stats) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (c < chains) {
        e = fabs(0.5 * scale * dE[c]);
        dE[c] = 0.0;
    }
    // the warp's largest drift, then one atomic per warp (non-negative doubles
    // order as their bit patterns)
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(e));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
        b = y > b ? y : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&stats[2], b);
}

// Operand conversion: spins +-1 (padding 0) -> e4m3 bytes or bf16 words,
// 16 spins per thread and iteration (n is a multiple of 32: rows of npad).
using dev::bf16_of2;
using dev::e4m3_of4;
__global__ void spins_to_e4m3(const int8_t* __restrict__ s, uint8_t* __restrict__ o, size_t n) {
    const uint4* in = reinterpret_cast<const uint4*>(s);
    uint4* out = reinterpret_cast<uint4*>(o);
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n / 16;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const uint4 w = in[i];
        out[i] = make_uint4(e4m3_of4(w.x), e4m3_of4(w.y), e4m3_of4(w.z), e4m3_of4(w.w));
    }
}
__global__ void spins_to_bf16(const int8_t* __restrict__ s, uint16_t* __restrict__ o, size_t n) {
    const uint4* in = reinterpret_cast<const uint4*>(s);
    uint4* out = reinterpret_cast<uint4*>(o);
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n / 16;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const uint4 w = in[i];
        out[2 * i] = make_uint4(bf16_of2(w.x, 0), bf16_of2(w.x, 2), bf16_of2(w.y, 0), bf16_of2(w.y, 2));
        out[2 * i + 1] = make_uint4(bf16_of2(w.z, 0), bf16_of2(w.z, 2), bf16_of2(w.w, 0), bf16_of2(w.w, 2));
    }
}
// J in {-1, 0, +1} -> e4m3 bytes.
__global__ void pm1_to_e4m3(const int8_t* __restrict__ j, uint8_t* __restrict__ o, size_t n) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int v = j[i];
        o[i] = v == 0 ? 0 : (v > 0 ? 0x38 : 0xB8);
    }
}
// fp32 J -> J1 + J2 + J3, each rounded to nearest bf16 from the remainder of
// the previous terms; the remainders are exact in fp32.
__global__ void gauss_to_bf16x3(const float* __restrict__ j, uint16_t* __restrict__ o, size_t n) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        float r = j[i];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const __nv_bfloat16 b = __float2bfloat16_rn(r);
            o[t * n + i] = __bfloat16_as_ushort(b);
            r -= __bfloat162float(b);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

cudaError_t encoder(PFN_cuTensorMapEncodeTiled_v12000* fn) {
    std::call_once(g_encode_once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    *fn = g_encode;
    return g_encode ? cudaSuccess : cudaErrorNotSupported;
}

// 2-D K-major map: rows x cols elements (cols innermost), box = 128 bytes of
// K x box_rows rows, 128-byte swizzle, out-of-range elements read as zero.
cudaError_t make_map(CUtensorMap* m, const void* base, bool bf16, uint64_t rows, uint64_t cols,
                     uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc;
    cudaError_t e = encoder(&enc);
    if (e != cudaSuccess) return e;
    const uint32_t esz = bf16 ? 2 : 1;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * esz};
    const cuuint32_t box[2] = {128u / esz, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                           const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

uint32_t grid1d(size_t n) {
    const size_t b = (n + 255) / 256;
    return static_cast<uint32_t>(b < 4096 ? (b ? b : 1) : 4096);
}

}  // namespace

size_t recompute_j_bytes(uint32_t kind, uint32_t npad) {
    const size_t n = static_cast<size_t>(npad) * npad;
    return kind == 0 ? n : 3 * n * 2;
}
size_t recompute_s_bytes(uint32_t kind, uint32_t chains, uint32_t npad) {
    return static_cast<size_t>(chains) * npad * (kind == 0 ? 1 : 2);
}

cudaError_t recompute_prepare_j(const void* J, uint32_t kind, uint32_t npad, void* j_op, cudaStream_t st) {
    const size_t n = static_cast<size_t>(npad) * npad;
    if (kind == 0)
        pm1_to_e4m3<<<grid1d(n), 256, 0, st>>>(static_cast<const int8_t*>(J), static_cast<uint8_t*>(j_op), n);
    else
        gauss_to_bf16x3<<<grid1d(n), 256, 0, st>>>(static_cast<const float*>(J), static_cast<uint16_t*>(j_op), n);
    return cudaGetLastError();
}

namespace {
// The coupling operands of several instances of one kind in one launch
// (blockIdx.y = instance): the conversions of pm1_to_e4m3 / gauss_to_bf16x3.
__global__ void prepare_j_batch(const PrepareJ* __restrict__ jobs, uint32_t pm1) {
    const PrepareJ p = jobs[blockIdx.y];
    const size_t n = static_cast<size_t>(p.npad) * p.npad;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        if (pm1) {
            const int v = static_cast<const int8_t*>(p.J)[i];
            static_cast<uint8_t*>(p.j_op)[i] = v == 0 ? 0 : (v > 0 ? 0x38 : 0xB8);
        } else {
            float r = static_cast<const float*>(p.J)[i];
            uint16_t* o = static_cast<uint16_t*>(p.j_op);
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const __nv_bfloat16 b = __float2bfloat16_rn(r);
                o[t * n + i] = __bfloat16_as_ushort(b);
                r -= __bfloat162float(b);
            }
        }
    }
}
}  // namespace

cudaError_t recompute_prepare_j_batch(uint32_t kind, const PrepareJ* jobs, uint32_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    size_t maxn = 0;
    for (uint32_t i = 0; i < n; ++i) maxn = std::max(maxn, static_cast<size_t>(jobs[i].npad) * jobs[i].npad);
    PrepareJ* d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, n * sizeof(PrepareJ), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, jobs, n * sizeof(PrepareJ), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        prepare_j_batch<<<dim3(std::min<uint32_t>(grid1d(maxn), 512u), n), 256, 0, st>>>(d, kind == 0 ? 1u : 0u);
        e = cudaGetLastError();
    }
    if (d) cudaFreeAsync(d, st);
    return e;
}

cudaError_t launch_set_fields_batch(uint32_t kind, const RecomputeSet* sets, uint32_t n, cudaStream_t st,
                                   bool spins_converted) {
    if (n == 0) return cudaSuccess;
    const bool bf = kind != 0;
    std::vector<SegSpins> seg(n);
    std::vector<BatchJob> jobs(n);
    std::vector<BatchTask> tasks;
    size_t maxn = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const RecomputeSet& q = sets[i];
        seg[i] = SegSpins{q.s, q.s_op, static_cast<size_t>(q.chains) * q.npad};
        maxn = std::max(maxn, seg[i].n);
        BatchJob& b = jobs[i];
        std::memset(&b, 0, sizeof b);
        cudaError_t e = make_map(&b.A, q.s_op, bf, q.chains, q.npad, BM);
        const size_t term_bytes = static_cast<size_t>(q.npad) * q.npad * (bf ? 2 : 1);
        for (uint32_t t = 0; t < 3 && e == cudaSuccess; ++t)
            e = make_map(&b.B[t], static_cast<const unsigned char*>(q.j_op) + (bf ? t : 0) * term_bytes, bf, q.npad,
                         q.npad, BN);
        if (e != cudaSuccess) return e;
        b.args.h = q.h;
        b.args.s = q.s;
        b.args.err = q.err;
        b.args.chains = q.chains;
        b.args.npad = q.npad;
        b.args.kblocks = (q.npad + (bf ? 63u : 127u)) / (bf ? 64u : 128u);
        b.args.terms = bf ? 3u : 1u;
        b.args.mode = 3;
        b.args.pm1 = bf ? 0u : 1u;
        b.args.fault = 0u;
        for (uint32_t m0 = 0; m0 < q.chains; m0 += BM)
            for (uint32_t n0 = 0; n0 < q.npad; n0 += BN) tasks.push_back(BatchTask{i, m0, n0, 0});
    }
    SegSpins* dseg = nullptr;
    BatchJob* djobs = nullptr;
    BatchTask* dtasks = nullptr;
    cudaError_t e = cudaMallocAsync(&dseg, n * sizeof(SegSpins), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&djobs, n * sizeof(BatchJob), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dtasks, tasks.size() * sizeof(BatchTask), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dseg, seg.data(), n * sizeof(SegSpins), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(djobs, jobs.data(), n * sizeof(BatchJob), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtasks, tasks.data(), tasks.size() * sizeof(BatchTask), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !spins_converted) {
        const dim3 g(std::min<uint32_t>(grid1d(maxn), 1024u), n);
        spins_to_op_batch<<<g, 256, 0, st>>>(dseg, bf ? 1u : 0u);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        CUtensorMap none;
        std::memset(&none, 0, sizeof none);
        Args a0;
        std::memset(&a0, 0, sizeof a0);
        const uint32_t nt = static_cast<uint32_t>(tasks.size());
        const uint32_t grid = std::max<uint32_t>(1u, std::min<uint32_t>(nt, static_cast<uint32_t>(sm_count())));
        if (bf) {
            e = cudaFuncSetAttribute(recompute_ws_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_BYTES);
            if (e == cudaSuccess)
                recompute_ws_kernel<false, true><<<grid, WS_THREADS, SMEM_BYTES, st>>>(none, none, none, none, a0,
                                                                                      djobs, dtasks, nt, 0u);
        } else {
            e = cudaFuncSetAttribute(recompute_ws_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_BYTES);
            if (e == cudaSuccess)
                recompute_ws_kernel<true, true><<<grid, WS_THREADS, SMEM_BYTES, st>>>(none, none, none, none, a0,
                                                                                     djobs, dtasks, nt, 0u);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    cudaFreeAsync(dseg, st);
    cudaFreeAsync(djobs, st);
    cudaFreeAsync(dtasks, st);
    return e;
}

namespace {
// The dynamic shared-memory attribute of a recompute kernel variant, set once
// per device and variant.
template <typename F>
cudaError_t smem_attribute(F kernel, int variant) {
    static std::mutex mu;
    static std::set<std::pair<int, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, variant})) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess) done.insert({dev, variant});
    return e;
}

// Operand tensor maps by (spin operand, coupling operand, type, shape): a map
// holds only addresses and shapes, so one encoded for the same buffers and
// shape is valid again; a few recent entries are kept.
cudaError_t cached_maps(const void* s_op, const void* j_op, bool bf, uint32_t chains, uint32_t npad, CUtensorMap* tA,
                        CUtensorMap* tB) {
    struct Entry {
        const void *s_op, *j_op;
        bool bf;
        uint32_t chains, npad;
        CUtensorMap A, B[3];
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& c : cache)
        if (c.s_op == s_op && c.j_op == j_op && c.bf == bf && c.chains == chains && c.npad == npad) {
            *tA = c.A;
            for (int t = 0; t < 3; ++t) tB[t] = c.B[t];
            return cudaSuccess;
        }
    Entry c{s_op, j_op, bf, chains, npad, {}, {}};
    cudaError_t e = make_map(&c.A, s_op, bf, chains, npad, BM);
    const size_t term_bytes = static_cast<size_t>(npad) * npad * (bf ? 2 : 1);
    for (uint32_t t = 0; t < 3 && e == cudaSuccess; ++t)
        e = make_map(&c.B[t], static_cast<const unsigned char*>(j_op) + (bf ? t : 0) * term_bytes, bf, npad, npad, BN);
    if (e != cudaSuccess) return e;
    if (cache.size() >= 32) cache.erase(cache.begin());
    cache.push_back(c);
    *tA = c.A;
    for (int t = 0; t < 3; ++t) tB[t] = c.B[t];
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_recompute(uint32_t kind, const int8_t* s, void* h, float* out, void* s_op,
                             const void* j_op, double* dE, unsigned long long* stats, int* err,
                             uint32_t chains, uint32_t npad, uint32_t terms, uint32_t mode, double scale,
                             cudaStream_t st, uint32_t fault, bool spins_converted, unsigned int* cnt) {
    const bool bf = kind != 0;
    if (!bf) terms = 1;
    if (terms < 1 || terms > 3) return cudaErrorInvalidValue;
    const size_t ns = static_cast<size_t>(chains) * npad;  // a multiple of 32
    cudaError_t e = cudaSuccess;
    if (!spins_converted) {
        if (bf)
            spins_to_bf16<<<grid1d(ns / 16), 256, 0, st>>>(s, static_cast<uint16_t*>(s_op), ns);
        else
            spins_to_e4m3<<<grid1d(ns / 16), 256, 0, st>>>(s, static_cast<uint8_t*>(s_op), ns);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // the operand maps of this (spins, couplings, shape): encoded once and
    // reused by later recomputes of the same buffers, so that the host work
    // between the conversion and the main kernel stays short
    CUtensorMap tA, tB[3];
    if ((e = cached_maps(s_op, j_op, bf, chains, npad, &tA, tB)) != cudaSuccess) return e;
    Args a;
    a.h = h;
    a.s = s;
    a.out = out;
    a.dE = dE;
    a.stats = stats;
    a.cnt = mode < 2 ? cnt : nullptr;
    a.scale = scale;
    a.err = err;
    a.chains = chains;
    a.npad = npad;
    a.kblocks = (npad + (bf ? 63u : 127u)) / (bf ? 64u : 128u);
    a.terms = terms;
    a.mode = mode;
    a.pm1 = bf ? 0u : 1u;
    a.fault = fault;
    a.compute_only = 0;
    const uint32_t tiles_n = (npad + BN - 1) / BN;
    const uint32_t nt = ((chains + BM - 1) / BM) * tiles_n;
    if (nt == 0) return cudaSuccess;
    const uint32_t grid = std::min<uint32_t>(nt, static_cast<uint32_t>(sm_count()));
    if (bf) {
        if ((e = smem_attribute(recompute_ws_kernel<false, false>, 0)) != cudaSuccess) return e;
        recompute_ws_kernel<false, false><<<grid, WS_THREADS, SMEM_BYTES, st>>>(tA, tB[0], tB[1], tB[2], a, nullptr,
                                                                               nullptr, nt, tiles_n);
    } else {
        if ((e = smem_attribute(recompute_ws_kernel<true, false>, 1)) != cudaSuccess) return e;
        recompute_ws_kernel<true, false><<<grid, WS_THREADS, SMEM_BYTES, st>>>(tA, tB[0], tB[0], tB[0], a, nullptr,
                                                                              nullptr, nt, tiles_n);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || mode >= 2 || a.cnt) return e;
    finish_energy<<<(chains + 255) / 256, 256, 0, st>>>(dE, chains, scale, stats);
    return cudaGetLastError();
}

cudaError_t tensor_peak_probe(uint32_t kind, uint32_t tiles, uint32_t reps, cudaStream_t st, double* tflops) {
    const bool bf = kind != 0;
    const uint32_t kblocks = 16;  // K = 2048 (FP8) or 1024 (bf16): 16 stages of 128 bytes per row
    const uint32_t K = kblocks * (bf ? 64u : 128u);
    const uint32_t grid = static_cast<uint32_t>(sm_count());
    const uint32_t nt = grid * tiles;
    const size_t esz = bf ? 2 : 1;
    void* A = nullptr;
    void* B = nullptr;
    int* err = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    // operands of each CTA's first tile (all zero: the values do not matter)
    cudaError_t e = cudaMalloc(&A, static_cast<size_t>(grid) * BM * K * esz);
    if (e == cudaSuccess) e = cudaMalloc(&B, static_cast<size_t>(BN) * K * esz);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(A, 0, static_cast<size_t>(grid) * BM * K * esz, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(B, 0, static_cast<size_t>(BN) * K * esz, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    CUtensorMap tA, tB;
    if (e == cudaSuccess) e = make_map(&tA, A, bf, static_cast<uint64_t>(grid) * BM, K, BM);
    if (e == cudaSuccess) e = make_map(&tB, B, bf, BN, K, BN);
    Args a{};
    a.err = err;
    a.chains = grid * BM;
    a.npad = K;
    a.kblocks = kblocks;
    a.terms = 1;
    a.mode = 2;
    a.pm1 = bf ? 0u : 1u;
    a.compute_only = 1;
    auto launch = [&]() {
        // task t: rows (t / 1) * BM, columns 0; each CTA's first task is its own block of A
        if (bf)
            recompute_ws_kernel<false, false><<<grid, WS_THREADS, SMEM_BYTES, st>>>(tA, tB, tB, tB, a, nullptr,
                                                                                   nullptr, nt, 1u);
        else
            recompute_ws_kernel<true, false><<<grid, WS_THREADS, SMEM_BYTES, st>>>(tA, tB, tB, tB, a, nullptr,
                                                                                  nullptr, nt, 1u);
        return cudaGetLastError();
    };
    if (e == cudaSuccess)
        e = bf ? smem_attribute(recompute_ws_kernel<false, false>, 0) : smem_attribute(recompute_ws_kernel<true, false>, 1);
    if (e == cudaSuccess) e = launch();  // warm-up
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (uint32_t r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && herr) e = cudaErrorLaunchTimeout;  // a bounded wait expired
    if (e == cudaSuccess)
        *tflops = 2.0 * BM * BN * static_cast<double>(K) * nt * reps / (ms * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(A);
    cudaFree(B);
    cudaFree(err);
    return e;
}

}  // namespace sk
