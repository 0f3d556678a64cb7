// sk_internal.h -- structures shared by the host runtime and the kernels of
// the sampler library (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sk {

constexpr uint32_t kMaxK = 256;      // proposals per step
constexpr uint32_t kPadTo = 32;      // Npad = round_up(N, 32)

// Error codes written by kernels into the launch's error word.
enum : int { kDevOk = 0, kDevTimeout = 1, kDevBounds = 2 };
// JobDev::fault bits (sk_run_params.fault_inject; tests of the bounded waits)
constexpr uint32_t kFaultWithholdRow = 1u;
constexpr uint32_t kFaultWithholdTile = 2u;

// One run as seen by the kernels.  Row-major layouts, leading dimension Npad:
//   J[Npad][Npad] (int8 or float), s[chains][Npad] int8 (+-1, padding 0),
//   h[chains][Npad] (int32 for +-J, float for Gaussian, padding 0).
struct alignas(16) JobDev {
    const void* J;
    int8_t* s;
    void* h;
    const uint64_t* W;      // +-J tables: MCMCMC W[d] or Metropolis M[k], wlen entries (0 past the end)
    uint64_t* step;         // device step counter of the run
    uint32_t* acc_run;      // per chain: accepted steps since the last record
    double* rec_E;          // [rec][chains]
    uint32_t* rec_acc;      // [rec][chains]
    double* rec_q;          // [rec][chains/2]
    double* rec_Enw;        // [rec][chains] node-weighted energy of the record step (or null)
    int32_t* trace;         // [trace_chains][trace_steps]
    int* err;               // error word of the run (kDev* codes)
    unsigned long long* work;  // per chain: [spins flipped, J rows the steps needed]
    uint64_t seed;
    uint64_t rec_capacity;
    uint64_t trace_steps;
    double scale;           // energy scale of the records
    float beta_eff;         // beta * scale (Gaussian weights)
    uint32_t stream;        // Philox stream id (24 bits)
    uint32_t N, Npad, chains, K;
    uint32_t kind, rule, wlen, record_every;
    uint32_t trace_chains;
    uint32_t step_limit;    // the run stops at this step (0xFFFFFFFF: no limit)
    // root of the star: a leaf iff U0 >= root_thr; slot weight factors of the
    // centre and the leaves as 20-bit integers (+-J, 2^20 = 1) and as log2
    // (Gaussian, 0 = 1); see root_setup
    uint32_t fcen, fleaf;
    uint64_t root_thr;
    float lcen, lleaf;
    // graph runs (graph = 1 k-ary tree, 2 line; 0 the star of the step kernel):
    // gtab = node factors F[V] (u32, 2^20 = 1), their inclusive prefix sums
    // (u64) and log2(F / 2^20) (float), each array 16-byte aligned
    const void* gtab;
    uint32_t graph, arity, V;
    uint32_t fault;         // sk_run_params.fault_inject (tests of the bounded waits)
    // the chains' spins as tensor-core operands [chains][Npad] (e4m3 bytes for
    // +-J, bf16 words for Gaussian couplings), written by the step kernels when
    // they write the spins back, so that the periodic recompute needs no
    // conversion; null when the run does not recompute periodically
    void* s_op;
    uint64_t pad_;
};
static_assert(sizeof(JobDev) % 16 == 0, "JobDev is copied as 16-byte words");

// A block of consecutive chains of one run, processed by one CTA (G lanes
// per chain).  chain0 is even so that overlap pairs stay inside a CTA.
struct WorkItem {
    uint32_t job, chain0, nchains, pad;
};

// Shared memory of the block-0 draws one chain keeps (16 bytes for each of
// up to 32 steps).
constexpr size_t kB0Bytes = 512;

// Bytes of shared memory one chain needs for spins, fields, (staged) the two
// J-row buffers and its block-0 draws.
inline size_t warp_smem_bytes(uint32_t npad, uint32_t kind, bool staged = true) {
    size_t bj = kind == 0 ? 1 : 4;
    return (size_t)npad * (1 + 4 + (staged ? 2 * bj : 0)) + kB0Bytes;
}

// Kernel launchers (sk_kernels.cu).  All return cudaGetLastError().
//
// The step kernel is instantiated per class = step_class(kind, rule, K, G,
// stage): the coupling type, the rule, whether row a is staged in shared
// memory by TMA (stage) or read through L1, the lanes per chain G (4, 8, 16,
// 32; 32/G chains per warp) and the Philox blocks of sites each lane draws,
// NB = blocks_per_lane(rule, K, G) (1, 2 or 4: K up to 4 G NB; Metropolis,
// which draws one block, takes NB = 2 for the chunked field update of the
// 128-register variant when npad / (4 G) is not a multiple of 8, see
// update_fields in sk_step.cuh); stage 2 is stage 0 with node-weighted
// energy records.  step_class
// returns -1 for a (K, G) no kernel covers.  A CTA holds W warps, i.e.
// W * 32/G chains, each with `per_chain` bytes of shared memory.  launch_step
// runs the items of one class; `bump` advances every job's step counter
// afterwards (set it on the last class).
uint32_t site_blocks_pow2(uint32_t rule, uint32_t K);
uint32_t blocks_per_lane(uint32_t rule, uint32_t K, uint32_t G);
int step_class(uint32_t kind, uint32_t rule, uint32_t K, uint32_t G, uint32_t stage, uint32_t npad = 0);
uint32_t class_lanes(int cls);
bool class_staged(int cls);
cudaError_t launch_step(const JobDev* jobs, const WorkItem* items, uint32_t n_items,
                        uint32_t* queue, uint64_t nsteps, uint32_t warps_per_cta,
                        uint32_t per_chain_bytes, uint32_t grid, int cls, uint32_t n_jobs,
                        bool bump, cudaStream_t st);
int step_kernel_occupancy(int cls, uint32_t warps_per_cta, size_t per_chain_bytes);
// Advances every job's step counter by nsteps (capped at its step limit):
// what `bump` does, for launches whose classes ran on several streams.
cudaError_t launch_bump_steps(const JobDev* jobs, uint32_t n_jobs, uint64_t nsteps, cudaStream_t st);
// Start state: spins from `init` (device, chains x N) or the Philox start,
// then (with_fields) h = J s on the CUDA cores (register-tiled fp32 / int32).
cudaError_t launch_init(const JobDev* job, const int8_t* init, uint32_t chains, uint32_t N,
                        uint32_t Npad, uint32_t kind, cudaStream_t st, bool with_fields = true);
// Start states of several runs in one launch: spins (from `init`, chains x N
// on the device, or the Philox start) and the run's counters, records,
// trace and recompute statistics cleared.  jobs_dev: a device array.
struct StartJob {
    JobDev job;
    const int8_t* init;
    unsigned long long* dstats;  // 6 words, or null
    double* ddE;                 // per chain, or null
    void* s_op;                  // or null: the spins also written as tensor-core operands
                                 // (e4m3 for +-J, bf16 for Gaussian couplings)
};
cudaError_t launch_start_batch(const StartJob* jobs_dev, uint32_t n, uint64_t max_words, cudaStream_t st);
// Device checks of host-supplied inputs: *flag receives the smallest
// (position << 2 | code) of a violation, all ones when there is none
// (couplings: position i * 2^16 + j, code 1 diagonal, 2 range or not finite,
// 3 asymmetric; spins: position = index, code 1 not +-1).
// Couplings of N spins drawn on the device from `seed` (Philox domain 2)
// into the padded Npad x Npad matrix J (see gen_couplings_kernel).
cudaError_t launch_gen_couplings(void* J, uint32_t kind, uint32_t N, uint32_t Npad, uint64_t seed, cudaStream_t st);
cudaError_t launch_check_couplings(const void* J, uint32_t kind, uint32_t N, uint32_t Npad,
                                   unsigned long long* flag, cudaStream_t st);
cudaError_t launch_check_spins(const int8_t* s, uint64_t n, unsigned long long* flag, cudaStream_t st);
// E of `count` configurations (spins count x N, device) into out[count].
// With `partial` (energy_tiles(N, count) * count doubles of scratch) the
// columns of J are split over several CTAs per block of configurations;
// without it one CTA covers all columns.
uint32_t energy_tiles(uint32_t N, uint32_t count);
cudaError_t launch_energy(const void* J, uint32_t kind, uint32_t N, uint32_t Npad, double scale,
                          const int8_t* spins, uint32_t count, double* out, cudaStream_t st,
                          double* partial = nullptr);

// Cluster-per-chain layout (sk_cluster*.cu): a cluster of C CTAs (1, 2, 4,
// 8 or 16) holds W chains of one run (one warp per chain in each CTA; W = 1,
// 2, 4 or 8); CTA r keeps the slice [r Npad/C, (r+1) Npad/C) of each chain's
// spins and fields and the same columns of every row of J.  Shared memory of
// a CTA: cluster_slice_bytes for J, then cluster_chain_bytes per chain.
// cluster_shape_ok: Npad splits into C slices whose rows of J are whole
// 16-byte units (bulk copies).  launch_cluster runs the items of one class
// (W chains each) on `clusters` clusters; nb = Philox blocks per lane at 32
// lanes (blocks_per_lane(rule, K, 32)).
constexpr uint32_t kClusterMaxChains = 8;
constexpr uint32_t kClusterMaxCtas = 16;
// Exchange region of one chain in each CTA: two exchange arrays (by step
// parity) of 4 nb x 32 slot entries of 16 bytes (Metropolis: one entry),
// the list of the slots this CTA owns in a step (16-bit slot numbers), two
// arrays of kClusterMaxCtas 4-byte step headers and two mbarriers.
__host__ __device__ constexpr uint32_t cluster_xbuf_bytes(uint32_t rule, uint32_t nb) {
    return rule == 1 ? 16u : 4u * nb * 32u * 16u;
}
__host__ __device__ constexpr uint32_t cluster_list_bytes(uint32_t rule, uint32_t nb) {
    return rule == 1 ? 16u : 4u * nb * 32u * 2u;
}
constexpr uint32_t kClusterHdrBytes = 2u * 16u * 4u;
__host__ __device__ constexpr uint32_t cluster_x_bytes(uint32_t rule, uint32_t nb) {
    return 2u * cluster_xbuf_bytes(rule, nb) + cluster_list_bytes(rule, nb) + kClusterHdrBytes + 16u;
}
bool cluster_shape_ok(uint32_t kind, uint32_t npad, uint32_t C);
size_t cluster_slice_bytes(uint32_t kind, uint32_t N, uint32_t npad, uint32_t C);
size_t cluster_chain_bytes(uint32_t rule, uint32_t nb, uint32_t npad, uint32_t C);
cudaError_t launch_cluster(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                           uint64_t nsteps, uint32_t kind, uint32_t rule, uint32_t nb, uint32_t C, uint32_t W,
                           uint32_t jbytes, uint32_t pc, uint32_t clusters, uint32_t n_jobs, bool bump,
                           cudaStream_t st);
// Clusters that can be resident at once with this shape (0: none).
int cluster_occupancy(uint32_t kind, uint32_t rule, uint32_t nb, uint32_t C, uint32_t W, uint32_t jbytes,
                      uint32_t pc);
// Per coupling type (sk_cluster_pm1.cu, sk_cluster_gauss.cu).
cudaError_t launch_cluster_pm1(uint32_t rule, uint32_t nb, const JobDev* jobs, const WorkItem* items,
                               uint32_t n_items, uint32_t* queue, uint32_t nsteps, uint32_t C, uint32_t W,
                               uint32_t jbytes, uint32_t pc, uint32_t clusters, cudaStream_t st);
cudaError_t launch_cluster_gauss(uint32_t rule, uint32_t nb, const JobDev* jobs, const WorkItem* items,
                                 uint32_t n_items, uint32_t* queue, uint32_t nsteps, uint32_t C, uint32_t W,
                                 uint32_t jbytes, uint32_t pc, uint32_t clusters, cudaStream_t st);
int occupancy_cluster_pm1(uint32_t rule, uint32_t nb, uint32_t C, uint32_t W, uint32_t jbytes, uint32_t pc);
int occupancy_cluster_gauss(uint32_t rule, uint32_t nb, uint32_t C, uint32_t W, uint32_t jbytes, uint32_t pc);

// Team layout (sk_team*.cu): one chain per team of T = 2 or 4 warps, one
// proposal slot per thread (MCMCMC takes K <= 32 T; Metropolis any run),
// `teams` (1 or 2) chains of one run per CTA, team_chain_bytes of shared
// memory per chain: spins, fields, the site ring, T block-0 buffers and the
// team's exchange words.  launch_team runs the items of one class.
inline size_t team_chain_bytes(uint32_t npad, uint32_t T) {
    return ((size_t)5 * npad + 1024u * T + 64u + 127u) & ~(size_t)127;
}
inline bool team_ok(uint32_t rule, uint32_t K, uint32_t T) {
    return (T == 2 || T == 4) && (rule == 1 || (K >= 1 && K <= 32u * T));
}
cudaError_t launch_team(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                        uint64_t nsteps, uint32_t kind, uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain,
                        uint32_t grid, uint32_t n_jobs, bool bump, cudaStream_t st);
int team_occupancy(uint32_t kind, uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain);  // CTAs per SM
// Per coupling type (sk_team_pm1.cu, sk_team_gauss.cu).
cudaError_t launch_team_pm1(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                            uint32_t nsteps, uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain,
                            uint32_t grid, cudaStream_t st);
cudaError_t launch_team_gauss(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                              uint32_t nsteps, uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain,
                              uint32_t grid, cudaStream_t st);
int occupancy_team_pm1(uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain);
int occupancy_team_gauss(uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain);

// Fused launch (sk_fused.cu): every star work item of a batch in one
// persistent kernel of W warps per CTA (W <= 16), whole-warp chains, rows
// through L1.  WorkItem::pad = (fused_variant << 24) | shared bytes per chain
// of the item's run; `smem` the launch's dynamic shared memory (at least the
// largest item's chains times its slice).
uint32_t fused_variant(uint32_t kind, uint32_t rule, uint32_t K, uint32_t npad);
cudaError_t launch_fused(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                         uint64_t nsteps, uint32_t W, uint32_t smem, uint32_t grid, uint32_t n_jobs, bool bump,
                         cudaStream_t st);
int fused_occupancy(uint32_t W, uint32_t smem);  // CTAs per SM (0: none)

// MCMCMC on deeper graphs (sk_graph.cu): a team of nw warps per chain (1, 2,
// 4, 8 or 16), W warps per CTA, i.e. W / nw chains (even; at most 14 when
// nw > 1, the teams' named barriers), `per_chain` bytes of shared memory per
// chain (graph_smem_bytes).  Work items hold W / nw chains.
size_t graph_smem_bytes(uint32_t npad, uint32_t V, uint32_t graph);
size_t graph_table_bytes(uint32_t V);
bool graph_team_ok(uint32_t W, uint32_t nw);
cudaError_t launch_graph(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                         uint64_t nsteps, uint32_t W, uint32_t nw, uint32_t per_chain, uint32_t grid, uint32_t kind,
                         uint32_t graph, uint32_t n_jobs, bool bump, cudaStream_t st);
int graph_kernel_occupancy(uint32_t kind, uint32_t graph, uint32_t W, uint32_t nw, size_t per_chain);

// Tensor-core field recompute (sk_recompute.cu).  Operand buffers: J as
// e4m3 (+-J, npad^2 bytes) or three bf16 terms (Gaussian, 3 npad^2 x 2
// bytes); spins as e4m3 / bf16 (chains x npad).  mode 0 checks the maintained
// fields, 1 also replaces them (resync), 2 writes H to `out` only, 3 sets
// the fields h = H (start state; +-J exact, no statistics).
// stats[0] = max |h - H| (double bits), [1] = mismatches, [2] = max |dE|.
size_t recompute_j_bytes(uint32_t kind, uint32_t npad);
size_t recompute_s_bytes(uint32_t kind, uint32_t chains, uint32_t npad);
cudaError_t recompute_prepare_j(const void* J, uint32_t kind, uint32_t npad, void* j_op, cudaStream_t st);
// recompute_prepare_j for several instances of one kind in one launch.
struct PrepareJ {
    const void* J;
    void* j_op;
    uint32_t npad, pad_;
};
cudaError_t recompute_prepare_j_batch(uint32_t kind, const PrepareJ* jobs, uint32_t n, cudaStream_t st);
// The fields h = J s of several runs of one coupling kind in one launch
// (mode 3 of launch_recompute for each set, spin operands converted too).
struct RecomputeSet {
    const int8_t* s;
    void* h;
    void* s_op;
    const void* j_op;
    int* err;
    uint32_t chains, npad;
};
cudaError_t launch_set_fields_batch(uint32_t kind, const RecomputeSet* sets, uint32_t n, cudaStream_t st,
                                   bool spins_converted = false);
// spins_converted: s_op already holds the spins (written by the step
// kernels); cnt: ceil(chains / 32) zeroed words that the check and resync
// modes use to find the last tile of each group of 32 chains, which then
// takes the group's energy-drift maximum (and leaves the words zero).
// Tensor-pipe probe: the recompute kernel with its operand ring filled once
// and the MMAs re-issued over it (no epilogue), `tiles` 128 x 256 tiles of
// K = 2048 (FP8, kind 0) or 1024 (bf16, kind 1) per CTA, one CTA per SM;
// *tflops = 2 M N K per tile x tiles / time of `reps` launches.
cudaError_t tensor_peak_probe(uint32_t kind, uint32_t tiles, uint32_t reps, cudaStream_t st, double* tflops);
cudaError_t launch_recompute(uint32_t kind, const int8_t* s, void* h, float* out, void* s_op,
                             const void* j_op, double* dE, unsigned long long* stats, int* err,
                             uint32_t chains, uint32_t npad, uint32_t terms, uint32_t mode, double scale,
                             cudaStream_t st, uint32_t fault = 0, bool spins_converted = false,
                             unsigned int* cnt = nullptr);

}  // namespace sk
struct sk_run;
namespace sk {
// Host-side helpers for the request server (sk_capi.cu).
void set_step_limit(sk_run* r, uint32_t limit);
uint64_t host_step(const sk_run* r);
size_t run_footprint(uint32_t N, uint32_t kind, uint32_t chains, uint64_t records);
size_t instance_footprint(uint32_t N, uint32_t kind);

// Root distribution of the MCMCMC star (sk_capi.cu): p_center = 0 is the
// uniform root (root_thr = ceil(2^64/(K+1)), i.e. a leaf iff
// floor(U0 (K+1) / 2^64) != 0, factors 1); 0 < p_center < 1 puts the centre at
// the root with probability p~_c = F_c / (F_c + K F_l), where F = round(2^20
// p_r / max(p_c, p_l)) and p_l = (1 - p_center)/K, and weights the centre
// slot by F_c and the leaf slots by F_l.  Returns false for a p_center
// outside (0, 1) or one whose smaller factor rounds to 0.
bool root_setup(JobDev& j, uint32_t K, double p_center);

// Sets the message sk_last_error() returns on this thread (sk_capi.cu).
void set_error_message(const char* msg);

}  // namespace sk
