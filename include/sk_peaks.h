/*
 * sk_peaks.h -- measured ceilings of the memory levels that bound the
 * sampler's step kernel, and of the tensor pipe as the field recompute's own
 * MMA loop drives it, for their rooflines.
 *
 * The batched MCMCMC step is bound by the memory level that holds the
 * couplings and the chains' state: the couplings' rows come from L2 (through
 * L1), the spins, fields and proposal gathers live in shared memory.  Its
 * roofline divides the algorithmic bytes of a step (J rows r N b_J from L2;
 * K (b_s + b_h) of proposal gathers and 2 f N b_h of field read-modify-write
 * in shared memory) by the kernel's time and by these measured peaks.  The
 * paper has no counterpart: it reports no hardware figures.
 *
 * Each call allocates its own buffers (cudaMalloc), warms up, times `reps`
 * launches with CUDA events on `stream` (cudaStream_t as void*, NULL = the
 * legacy default stream), frees what it allocated and returns the result;
 * it synchronises `stream`.  Status codes as in sk_mcmcmc.h.
 */
#ifndef SK_PEAKS_H
#define SK_PEAKS_H

#include <stdint.h>

#include "sk_mcmcmc.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * sk_peak_l2_read: read bandwidth of L2 on a working set that stays resident
 * in it: `working_set_bytes` (16 MiB .. 96 MiB, a multiple of 16) read with
 * 16-byte loads that bypass L1 (ld.global.cg), one persistent grid of 4 CTAs
 * of 512 threads per SM, `passes` sweeps per launch.  *gbps = bytes read /
 * time (1e9 bytes per second).
 */
sk_status sk_peak_l2_read(uint64_t working_set_bytes, uint32_t passes, uint32_t reps, void* stream,
                          double* gbps);

/*
 * sk_peak_smem: shared-memory load bandwidth of the whole GPU, one CTA of
 * 1024 threads per SM over a 64 KiB array.
 *   mode SK_PEAK_SMEM_VEC16:  16-byte loads, the 32 lanes of a warp reading 512
 *                             contiguous bytes (no bank conflicts);
 *   mode SK_PEAK_SMEM_GATHER4: 4-byte loads at independent random word
 *                             addresses per lane (the bank conflicts of random
 *                             gathers, as at the proposal sites); the useful
 *                             4 bytes per lane are counted.
 * *gbps = bytes loaded / time.
 */
typedef enum { SK_PEAK_SMEM_VEC16 = 0, SK_PEAK_SMEM_GATHER4 = 1 } sk_peak_smem_mode;
sk_status sk_peak_smem(uint32_t mode, uint32_t iters, uint32_t reps, void* stream, double* gbps);

/*
 * sk_peak_tensor: the tensor-pipe rate of the library's own field-recompute
 * kernel (the tcgen05 MMA loop that the periodic J.S recompute runs) with
 * nothing else to do: each CTA (one per SM) fills its 4-stage operand ring
 * once by TMA and then issues the MMAs of `tiles` 128 x 256 output tiles over
 * it (K = 2048 for kind 0, FP8 e4m3 with kind::f8f6f4; K = 1024 for kind 1,
 * bf16 with kind::f16), accumulators in tensor memory, no epilogue work.
 * *tflops = 2 x 128 x 256 x K x tiles x SMs / time (1e12 per second).
 * kind 0 or 1; tiles 1..4096; reps >= 1.
 */
sk_status sk_peak_tensor(uint32_t kind, uint32_t tiles, uint32_t reps, void* stream, double* tflops);

#ifdef __cplusplus
}
#endif
#endif
