/*
 * sk_mcmcmc.h -- C ABI of the GB300 (sm_103a) Many-Configuration Markov-Chain
 * Monte Carlo sampler for the Sherrington-Kirkpatrick spin glass
 * (Simkovic & Rossi, arXiv:2102.05613).
 *
 * The problem (Sec. II): draw samples of P_eq(c) = exp(-beta E(c)) / Z over
 * spin configurations c = (s_1..s_N), s_i = +-1, visiting K+1 configurations
 * per Monte Carlo step.  The energy is the SK energy of Sec. IV.A written as
 *     E(s) = -scale * sum_{i<j} J_ij s_i s_j
 * with J symmetric, zero diagonal, J_ij ~ N(0, 1/N) (Gaussian) or +-1 (+-J).
 *
 * Each step of the many-configuration rule (Sec. A.2, Eq.
 * eq_det_balance_graph_solution, on the star graph of App. B.2 with a uniform
 * root) proposes K configurations from the current one by single spin flips,
 * picks the next state among the K+1 nodes with probability proportional to
 * exp(-beta E), and updates the maintained local fields h_i = sum_j J_ij s_j.
 * SK_RULE_METROPOLIS is the single-flip Metropolis comparator of Sec. IV.B.
 *
 * Conventions for every call:
 *  - the return value is an sk_status; on error nothing is written to the
 *    caller's outputs and sk_last_error() describes the failure (per thread);
 *  - buffers marked "mem" are host pointers when mem == SK_MEM_HOST and
 *    device pointers (of the current device) when mem == SK_MEM_DEVICE; input
 *    buffers are copied before the call returns (device inputs: enqueued on
 *    the object's stream), so the caller keeps ownership and may reuse them
 *    once the call (host) or the stream (device) has moved on;
 *  - objects (sk_instance, sk_run, sk_batch) are owned by the library and
 *    released by their *_destroy / *_free call;
 *  - work is enqueued on the CUDA stream given at creation (NULL = the legacy
 *    default stream); calls that return data to the host synchronise it.
 *  - there is no CPU fallback: without a usable sm_103a device every call
 *    that needs one returns SK_ERR_CUDA.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), counter
 * (block, step, chain, domain<<24 | stream_id), key = seed.  A chain's
 * trajectory depends only on (seed, stream_id, chain index, couplings, K,
 * beta, rule, start), never on how chains are batched or launched.
 */
#ifndef SK_MCMCMC_H
#define SK_MCMCMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SK_OK = 0,
    SK_ERR_INVALID_ARG = 1, /* an argument is out of range or inconsistent     */
    SK_ERR_OOM = 2,         /* a device or host allocation failed              */
    SK_ERR_CUDA = 3,        /* a CUDA runtime call failed (no device, ...)     */
    SK_ERR_TIMEOUT = 4,     /* a bounded device wait expired; state is invalid */
    SK_ERR_NOT_READY = 5,   /* work still in flight (non-blocking query)       */
    SK_ERR_DEVICE = 6,      /* a kernel reported an inconsistency (bounds)     */
    SK_ERR_BUSY = 7,        /* the object is still in use by another object    */
    SK_ERR_CANCELLED = 8    /* the request was cancelled before it finished    */
} sk_status;

typedef enum { SK_J_PM1 = 0, SK_J_GAUSS = 1 } sk_jkind;      /* int8 +-1 / float32 */
typedef enum { SK_RULE_MCMCMC = 0, SK_RULE_METROPOLIS = 1 } sk_rule;

/* Graph of an MCMCMC step (App. B): the star (K proposals, the default), the
 * full k-ary tree of depth D populated from a uniformly drawn root position
 * (App. B.2), or the line of L nodes grown by the addition process, whose
 * starting configuration ends at position v with probability
 * binom(L-1, v)/2^(L-1) (App. B.1, Eq. eq_create_line_graph). */
typedef enum { SK_GRAPH_STAR = 0, SK_GRAPH_TREE = 1, SK_GRAPH_LINE = 2 } sk_graph;
typedef enum { SK_MEM_HOST = 0, SK_MEM_DEVICE = 1 } sk_mem;

#define SK_MAX_K 256u        /* proposals per step                         */
#define SK_MAX_N 8192u       /* spins per configuration                    */

typedef struct sk_instance sk_instance;  /* couplings resident on the device */
typedef struct sk_run sk_run;            /* chains of one instance            */
typedef struct sk_batch sk_batch;        /* runs advanced by one launch       */

/* ---------------------------------------------------------------------- */
/* Instances (Sec. IV.A: one disorder realisation {J_ij})                  */
/* ---------------------------------------------------------------------- */

/*
 * sk_create_instance: one disorder realisation of N spins on the device,
 * uploaded from the caller or drawn from a seed.
 *   N          2 .. SK_MAX_N spins.
 *   kind       SK_J_PM1: couplings are int8 with values in {-1, 0, +1};
 *              SK_J_GAUSS: couplings are float32.
 *   couplings  N*N row-major, symmetric, zero diagonal, in the memory `mem`
 *              says (copied; checked on the device: SK_ERR_INVALID_ARG
 *              names the first offending entry); or NULL: the couplings are
 *              drawn on the device from `seed` (mem is ignored) --
 *              Philox4x32-10 (Salmon et al., SC'11) with key = seed, domain 2,
 *              one draw per pair i < j shared by J_ij and J_ji:
 *                SK_J_PM1:   counter (j >> 7, i, 0, 2 << 24), bit j & 127 of
 *                            the block (word (j & 127) >> 5, bit j & 31):
 *                            set -> -1, clear -> +1 (equiprobable +-1);
 *                SK_J_GAUSS: counter (j, i, 1, 2 << 24) = (w0, w1, w2, w3),
 *                            uniforms u1 = (2^26 (w0 >> 5) + (w1 >> 6)) 2^-53
 *                            and u2 alike from (w2, w3), the Box-Muller normal
 *                            z = sqrt(-2 ln(1 - u1)) cos(2 pi u2) in double
 *                            precision, J_ij = (float)(z / sqrt(N)): the
 *                            N(0, 1/N) couplings of Sec. IV.A's model after
 *                            J -> -J/sqrt(N); the device's double-precision
 *                            log and cos may round the last bit differently
 *                            from another library's, so another
 *                            implementation of this recipe agrees to within
 *                            one float32 unit in the last place;
 *   seed       the Philox key when couplings is NULL, else unused.
 *   scale      energy multiplier (> 0): E = -scale sum_{i<j} J s s.  1.0 for
 *              the +-J model with integer energies; 1/sqrt(N) gives the +-J
 *              model on the paper's Gaussian temperature scale.
 *   stream     cudaStream_t (as void*) for this instance's copies, or NULL.
 * The device copy is padded to Npad = ceil(N/32)*32 rows and columns.
 */
sk_status sk_create_instance(uint32_t N, uint32_t kind, const void* couplings, uint32_t mem, uint64_t seed,
                             double scale, void* stream, sk_instance** out);

/* sk_get_couplings: copies the instance's N x N couplings (row-major, int8
 * for SK_J_PM1, float32 for SK_J_GAUSS) into `out` (mem: host or device) and
 * synchronises the instance's stream -- to save a drawn realisation or check
 * it against another implementation. */
sk_status sk_get_couplings(const sk_instance* inst, void* out, uint32_t mem);

/* Replaces the couplings of an existing instance (same N and kind); used to
 * re-upload a disorder realisation without reallocating. */
sk_status sk_set_couplings(sk_instance* inst, const void* couplings, uint32_t mem);

/* sk_set_couplings for n distinct instances at once: every copy and check is
 * enqueued first (host couplings on the library's input stream, apart from
 * the compute, so they overlap it), the checks are read with one wait, and
 * only if all pass do the
 * new couplings become current -- all or nothing: on SK_ERR_INVALID_ARG no
 * instance changes and the message names the first failing instance. */
sk_status sk_set_couplings_many(sk_instance* const* insts, uint32_t n, const void* const* couplings, uint32_t mem);

/* Releases an instance (waits for its streams).  Runs keep a pointer to
 * their instance: while a run created on it has not been freed
 * (mcmcmc_free), the call returns SK_ERR_BUSY and releases nothing. */
sk_status sk_destroy_instance(sk_instance* inst);

/*
 * sk_energy: E(s) = -scale sum_{i<j} J_ij s_i s_j for `count` configurations
 * (Sec. IV.A), computed on the device in double precision (exact for +-J).
 *   spins  count*N int8 values +-1, row-major (mem: SK_MEM_HOST/DEVICE);
 *   out_E  count doubles, always a host pointer.
 */
sk_status sk_energy(const sk_instance* inst, const int8_t* spins, uint32_t count, uint32_t mem,
                    double* out_E);

/* ---------------------------------------------------------------------- */
/* Runs: `chains` independent Markov chains on one instance                */
/* ---------------------------------------------------------------------- */
typedef struct {
    uint32_t chains;        /* >= 1; pairs (2m, 2m+1) give the overlap q        */
    uint32_t K;             /* proposals per step, 1..SK_MAX_K (MCMCMC only)    */
    uint32_t rule;          /* sk_rule                                          */
    uint32_t record_every;  /* record observables after every R-th step; 0=off  */
    uint64_t max_records;   /* record capacity (records past it are dropped)    */
    double beta;            /* inverse temperature, >= 0                        */
    uint64_t seed;          /* Philox key                                       */
    uint32_t stream_id;     /* Philox stream (24 bits), e.g. the instance index */
    uint32_t trace_chains;  /* chains 0..trace_chains-1 log the slot chosen at  */
    uint64_t trace_steps;   /*   each of their first trace_steps steps (debug)  */
    const int8_t* init_spins; /* chains*N start (+-1), or NULL: Philox start   */
    uint32_t init_mem;      /* sk_mem of init_spins                             */
    uint32_t recompute_every; /* recompute the fields on the tensor cores after */
                            /*   every M-th step (0 = never): +-J check, Gaussian */
                            /*   resync (see mcmcmc_recompute)                  */
    uint32_t recompute_terms; /* bf16 terms of the Gaussian J split, 1..3 (0=3) */
    double p_center;        /* root distribution of the star (App. B.2, p_r     */
                            /*   free; MCMCMC only): 0 = uniform, 1/(K+1) each  */
                            /*   slot; 0 < p_center < 1: the centre is the root */
                            /*   with ~p_center, each leaf with (1-p_center)/K, */
                            /*   and slot weights carry the root probability.  */
                            /*   The ratio p_center / p_leaf is rounded to a    */
                            /*   ratio of 20-bit integers F_c : F_l (the larger */
                            /*   2^20) and the root drawn with F_c/(F_c+K F_l); */
                            /*   both factors must round to >= 1 (else          */
                            /*   SK_ERR_INVALID_ARG)                            */
    uint32_t node_weighted; /* 1: records also hold the node-weighted energy    */
                            /*   (mcmcmc_observables_nw); such runs read row a  */
                            /*   through L1 (no staging)                        */
    uint32_t graph;         /* sk_graph (MCMCMC only; 0 = the star of K)        */
    uint32_t arity, depth;  /* SK_GRAPH_TREE: k >= 2, 1 <= D <= 16              */
    uint32_t line_nodes;    /* SK_GRAPH_LINE: L >= 2                            */
                            /*   Graphs hold at most 8192 nodes; K is then the  */
                            /*   number of other nodes (V - 1), traces log the  */
                            /*   node index; p_center and node_weighted apply   */
                            /*   to the star only.  One chain per warp; node v  */
                            /*   is the current state with the sites of the     */
                            /*   template path from the root to v flipped, and  */
                            /*   is chosen with probability ~ P_eq F_v (F_v the */
                            /*   line's binomial factor in 20-bit fixed point,  */
                            /*   1 for trees).                                  */
    uint32_t fault_inject;  /* tests of the failure path only, 0 otherwise:     */
                            /*   SK_FAULT_WITHHOLD_ROW withholds the first row  */
                            /*   copy of chain 0 in a layout with staged rows   */
                            /*   (mcmcmc_batch_set_layout staging 1), or the    */
                            /*   last row of the first CTA's slice of J in the  */
                            /*   cluster layout (mcmcmc_batch_set_cluster);     */
                            /*   SK_FAULT_WITHHOLD_TILE withholds the first     */
                            /*   operand tile of the first CTA of each field    */
                            /*   recompute (mcmcmc_recompute): the waits for    */
                            /*   them expire (~2 s each), the kernel lets its   */
                            /*   other copies and MMAs finish, returns, and the */
                            /*   call reports SK_ERR_TIMEOUT; nothing faults    */
} sk_run_params;

#define SK_FAULT_WITHHOLD_ROW 1u
#define SK_FAULT_WITHHOLD_TILE 2u

/*
 * mcmcmc_create: allocates the chains' state (spins, local fields, records)
 * and initialises it: spins from init_spins or from Philox domain 1, fields
 * h = J s computed on the tensor cores (exact for +-J; for Gaussian
 * couplings J is split into three bf16 terms, which represent it exactly,
 * and the products are summed in FP32).  Host start spins are copied to a
 * per-run staging buffer and checked on the device (each must be +-1;
 * SK_ERR_INVALID_ARG names the first offending index) before anything of the
 * run is written.  The run is at step 0.  Device memory: 5 bytes per spin
 * per chain for spins and fields, plus the tensor-core spin operand (1 byte
 * per spin for +-J, 2 for Gaussian), 1 byte per spin for a host start, the
 * records, and once per instance the couplings' operand (Npad^2 bytes for
 * +-J, 6 Npad^2 for Gaussian).  Synchronises the stream when init_spins is
 * given (for the check); otherwise asynchronous on the instance's stream.
 */
sk_status mcmcmc_create(sk_instance* inst, const sk_run_params* p, sk_run** out);

/*
 * mcmcmc_advance: enqueues `steps` Monte Carlo steps of every chain of the
 * run (one persistent kernel launch).  Records fall at global steps t with
 * (t+1) % record_every == 0, record index (t+1)/record_every - 1.
 * Step counts are limited to 2^32 in total per run.
 */
sk_status mcmcmc_advance(sk_run* run, uint64_t steps);

/* mcmcmc_run: mcmcmc_create followed by mcmcmc_advance(steps). */
sk_status mcmcmc_run(sk_instance* inst, const sk_run_params* p, uint64_t steps, sk_run** out);

/*
 * mcmcmc_reset: restarts the run at step 0 from new spins (chains*N, mem) or
 * from the Philox start when spins == NULL; fields are recomputed, records
 * and acceptance counters cleared.  Reuses the run's device memory.
 */
sk_status mcmcmc_reset(sk_run* run, const int8_t* spins, uint32_t mem);

/* mcmcmc_reset for n distinct runs at once (spins[i] for run i, or spins ==
 * NULL / spins[i] == NULL for the Philox start): the copies and checks of
 * all start spins are enqueued, read with one wait, and only if all pass are
 * the runs restarted -- all or nothing, as sk_set_couplings_many. */
sk_status mcmcmc_reset_many(sk_run* const* runs, uint32_t n, const int8_t* const* spins, uint32_t mem);

/*
 * mcmcmc_wait: blocks until the run's stream is idle, at most timeout_ns
 * nanoseconds (0 = no limit): SK_ERR_TIMEOUT if work is still in flight then.
 * Reports SK_ERR_TIMEOUT / SK_ERR_DEVICE raised by a kernel of the run.
 */
sk_status mcmcmc_wait(sk_run* run, uint64_t timeout_ns);

/*
 * mcmcmc_observables: copies records [first, first+count) (synchronises):
 *   energy[r*chains + c]       E of chain c (scale included), double;
 *   overlap[r*(chains/2) + m]  q = (1/N) sum_i s_i s'_i of chains 2m, 2m+1;
 *   accepted[r*chains + c]     steps of the interval whose configuration
 *                              changed (uint32).
 * Any output may be NULL.  mem says where the outputs live.
 */
sk_status mcmcmc_observables(sk_run* run, uint64_t first, uint64_t count, double* energy,
                             double* overlap, uint32_t* accepted, uint32_t mem);

/* mcmcmc_observables for n runs with two waits in all: energy[i], overlap[i],
 * accepted[i] receive run i's records (each array of n pointers, and each
 * pointer, may be NULL).  Device errors of any run are reported (with the
 * run's index) before anything is copied. */
sk_status mcmcmc_observables_many(sk_run* const* runs, uint32_t n, uint64_t first, uint64_t count,
                                  double* const* energy, double* const* overlap, uint32_t* const* accepted,
                                  uint32_t mem);

/*
 * mcmcmc_observables_nw: copies the node-weighted energies of records
 * [first, first+count) of a run created with node_weighted = 1
 * (synchronises; SK_ERR_INVALID_ARG otherwise): energy_nw[r*chains + c]
 * (double, scale included) is, for the recorded state c and the graph T that
 * the next step generates from it (Sec. A.2, Eq. eq_monte_carlo_graph),
 * sum_j P_node(j|T) E(c_j) = E(c) + sum_j P_node(j|T) dE_j over the K+1
 * slots with the probabilities that step chooses with: the expectation of the
 * next state's energy given T, an estimator of <E> with less variance than
 * the energy one step later.  For the Metropolis comparator it is
 * E(c) + p_acc dE of the next step's proposal.  Summed in double precision
 * from the step's weights.
 */
sk_status mcmcmc_observables_nw(sk_run* run, uint64_t first, uint64_t count, double* energy_nw, uint32_t mem);

/*
 * mcmcmc_state: copies the current spins (chains*N int8) and, if non-NULL,
 * the maintained fields (chains*N, int32 for +-J, float32 for Gaussian) and
 * the step counter (synchronises; spins/fields per mem, step a host pointer).
 */
sk_status mcmcmc_state(sk_run* run, int8_t* spins, void* fields, uint64_t* step, uint32_t mem);

/* ---------------------------------------------------------------------- */
/* Field recompute on the tensor cores                                     */
/* ---------------------------------------------------------------------- */
typedef enum { SK_RECOMPUTE_CHECK = 0, SK_RECOMPUTE_RESYNC = 1, SK_RECOMPUTE_OUTPUT = 2 } sk_recompute_mode;

typedef struct {
    double max_field_drift;   /* max over chains and spins of |h_maintained - H|   */
    double max_energy_drift;  /* max over chains of |E(h_maintained) - E(H)|,     */
                              /*   E = -scale/2 sum_i s_i h_i                     */
    uint64_t mismatches;      /* fields with h_maintained != H (+-J: must be 0)   */
    uint64_t recomputes;      /* recomputes these figures cover                   */
} sk_recompute_stats;

/*
 * mcmcmc_recompute: recomputes every chain's local fields H = J s (the
 * definition h_i = sum_j J_ij s_j behind the energy of Sec. IV.A) as one
 * matrix product on the tensor cores (tcgen05, TMA, tensor memory):
 *   +-J:      spins and couplings as FP8 e4m3 (+-1, 0 exact), FP32
 *             accumulation; exact, since every partial sum is an integer
 *             below 2^24;
 *   Gaussian: spins as bf16 (exact), J split into `terms` bf16 matrices
 *             (1..3; three round-to-nearest terms reproduce fp32 J exactly),
 *             all accumulated in FP32.
 * mode SK_RECOMPUTE_CHECK compares H with the maintained fields;
 * SK_RECOMPUTE_RESYNC also replaces the maintained fields by H;
 * SK_RECOMPUTE_OUTPUT only writes H to fields_out (chains*N float32, mem).
 * Per-element differences are exact integers (+-J) or float32 (Gaussian);
 * per-chain energy differences are summed in double precision.  With
 * `stats` non-NULL (host) the call synchronises and returns this call's
 * figures; with stats NULL (modes CHECK/RESYNC) it only enqueues the work on
 * the run's stream.
 */
sk_status mcmcmc_recompute(sk_run* run, uint32_t mode, uint32_t terms, sk_recompute_stats* stats,
                           float* fields_out, uint32_t mem);

/* Figures accumulated by the periodic recomputes (recompute_every) since
 * the run's creation or last reset.  Synchronises. */
sk_status mcmcmc_recompute_stats(sk_run* run, sk_recompute_stats* stats);

/* mcmcmc_trace: copies the slot log (trace_chains*trace_steps int32; slot
 * 0..K for MCMCMC, 1/0 accepted/rejected for Metropolis). */
sk_status mcmcmc_trace(sk_run* run, int32_t* slots, uint32_t mem);

/*
 * mcmcmc_counters: work done since the run's last reset, summed over its
 * chains (synchronises): spins flipped, and rows of J the steps needed (row a
 * of every leaf-rooted step, for the J_ab terms, plus the row of every other
 * flipped spin).  Both host pointers, either may be NULL.
 */
sk_status mcmcmc_counters(sk_run* run, uint64_t* flips, uint64_t* rows);

/* Releases a run (waits for its stream).  While the run belongs to a batch
 * that has not been freed (mcmcmc_batch_free), the call returns SK_ERR_BUSY
 * and releases nothing. */
sk_status mcmcmc_free(sk_run* run);

/* ---------------------------------------------------------------------- */
/* Batches: many runs (instances, N, K, beta, rule may differ) advanced by */
/* one persistent launch; the runs must share one CUDA stream.            */
/* ---------------------------------------------------------------------- */

/*
 * mcmcmc_batch_create: plans work items (blocks of chains of one run) for
 * the runs.  warps_per_cta 0 lets the library choose (as many as fit);
 * otherwise at most that many warps per CTA (1..32).  Whole-warp chains
 * (32 lanes) of a pair share a CTA, so an odd count is raised by one for
 * launch classes with runs of several chains; one warp is allowed where
 * every run of the class has one chain.
 */
sk_status mcmcmc_batch_create(sk_run* const* runs, uint32_t n_runs, uint32_t warps_per_cta,
                              sk_batch** out);

/* Advances every run of the batch by `steps` steps in one kernel launch. */
sk_status mcmcmc_batch_advance(sk_batch* b, uint64_t steps);

/*
 * mcmcmc_batch_capture: records the launches that advance every run of the
 * batch by `steps` steps -- the step kernels of each class, the step-counter
 * update and, for runs with recompute_every, the tensor-core recomputes --
 * into a CUDA graph (stream capture on the runs' stream, which must not be
 * the legacy default stream).  Nothing runs at capture.  With recomputing
 * runs, `steps` and the runs' current step must be multiples of
 * recompute_every.  A later mcmcmc_batch_autotune drops the graph.
 */
sk_status mcmcmc_batch_capture(sk_batch* b, uint64_t steps);

/* Launches the captured graph `times` times (each advances `steps` steps). */
sk_status mcmcmc_batch_replay(sk_batch* b, uint32_t times);

/*
 * mcmcmc_batch_autotune: for each launch class of the batch, times a
 * `trial_steps`-step launch (the better of two, after a warm-up launch) for
 * each staging choice, each lanes-per-chain
 * value K allows and each warps-per-CTA value that fits in shared memory
 * (the CTA size also selects the kernel's register budget) and keeps the
 * fastest; graph classes try 1, 2, 4, 8 and 16 warps per chain with every
 * even number of chains per CTA that fits; star classes of at most 64 chains
 * also try the cluster-per-chain layout (mcmcmc_batch_set_cluster) at every
 * cluster size and chains-per-cluster value the class can take, and star
 * classes of at most 1024 chains the team layout (64 and 128 lanes, see
 * mcmcmc_batch_set_layout) where the class can take it.  Then the
 * whole batch is timed with those per-class launches and with its star runs
 * in one fused launch (mcmcmc_batch_set_fused) of 4, 8 and 16 warps per CTA,
 * and the fastest of the four is kept.
 * Trials start from a copy of the runs' state, which is restored afterwards,
 * and run with records and traces off: the runs' trajectories, records and
 * step counters are unchanged.  *warps_per_cta (may be NULL) receives the
 * first class's choice.  Synchronises.
 */
sk_status mcmcmc_batch_autotune(sk_batch* b, uint32_t trial_steps, uint32_t* warps_per_cta);

/*
 * mcmcmc_batch_set_layout: forces the layout of every launch class.
 *   lanes    lanes per chain, 4, 8, 16 or 32 (32/lanes chains share a warp),
 *            raised to the fewest a class's K allows (each lane draws up to
 *            4 Philox blocks of 4 proposals: see below);
 *            0 = default (whole-warp chains, 32 lanes); a value that
 *            leaves no room for one warp's chains in a CTA's shared memory
 *            is raised until they fit.  Kernels exist
 *            for 1 block per lane at every width, 2 blocks at 8, 16 and 32
 *            lanes and 4 blocks at 8 and 16 lanes, so K <= 16 allows 4
 *            lanes, K <= 128 8 lanes and K <= 256 16 lanes;
 *            Graph runs (trees and lines) take 64, 128, 256 or 512 lanes
 *            = 2, 4, 8 or 16 warps per chain (any smaller value: one warp);
 *            star classes take 64 lanes as the team layout of 2 warps per
 *            chain and 128 or more as that of 4 warps: one proposal slot per
 *            thread, one chain per team, one team per CTA where every run of
 *            the class has one chain, else two (overlap pairs share a CTA);
 *            MCMCMC with K <= 32 x warps per chain, or Metropolis, and no
 *            node-weighted records (other classes fall back to 32 lanes).
 *            +-J trajectories are those of the warp layouts bit for bit;
 *   staging  0 = default (rows through L1), 1 = the next step's row of J is
 *            staged in shared memory by TMA (two row buffers per chain),
 *            2 = rows are read through L1 (no buffers, so more chains fit in
 *            shared memory).
 * Drops autotuned choices and a captured graph.  Results do not depend on it.
 */
sk_status mcmcmc_batch_set_layout(sk_batch* b, uint32_t lanes, uint32_t staging);

/*
 * mcmcmc_batch_set_cluster: forces the cluster-per-chain layout (ctas > 0) or
 * returns to the warp layouts (ctas = 0) for every star launch class that can
 * take it; the other classes keep their layout.
 *   ctas     CTAs per thread-block cluster: 1, 2, 4, 8 or 16 (16 needs the
 *            device's non-portable cluster size).  CTA r of a cluster holds
 *            the slice [r Npad/ctas, (r+1) Npad/ctas) of each of its chains'
 *            spins and fields and the same columns of every row of J, copied
 *            once per work item into its shared memory; the owner of each
 *            proposed site publishes what the step needs about it to every
 *            CTA of the cluster, one cluster barrier per step, and every CTA
 *            makes the same choice (sk_cluster.cuh in the sources).  A class
 *            can take it when each run's Npad/ctas spins make whole 16-byte
 *            rows of J (int8: 16 spins, fp32: 4), K <= 256, the run records
 *            no node-weighted energies, and N (Npad/ctas) bytes of J (x4 for
 *            Gaussian couplings) plus the chains' slices fit in one CTA's
 *            shared memory (about 220 KB): e.g. N <= 1536 for +-J and
 *            N <= 896 for Gaussian couplings at 16 CTAs;
 *   chains   chains per cluster (one warp each in every CTA): 1, 2, 4 or 8;
 *            0 = 2, or 1 when every run of the class has one chain; 1 is
 *            raised to 2 for runs of several chains (overlap pairs share a
 *            cluster).
 * Results do not depend on it: trajectories and records equal those of
 * whole-warp chains (mcmcmc_batch_set_layout lanes 32) bit for bit.  Drops autotuned
 * choices and a captured graph.  SK_ERR_CUDA when no cluster of that size can
 * be resident; the previous plan is kept on any error.
 */
sk_status mcmcmc_batch_set_cluster(sk_batch* b, uint32_t ctas, uint32_t chains);

/*
 * mcmcmc_batch_set_fused: runs every star run of the batch (MCMCMC and
 * Metropolis, any coupling kind, N, K; not graph runs nor runs that record
 * node-weighted energies, which keep their own launches) in one persistent
 * launch (warps_per_cta = 2, 4, 8 or 16), or returns to one launch per
 * launch class (0).  The fused launch fixes one CTA shape for all its runs:
 * whole-warp chains (32 lanes), rows of J through L1, the 128-register
 * budget; each work item holds up to warps_per_cta chains of one run (an
 * even number for runs of several chains) and is dispatched to its run's
 * kernel variant (coupling kind, rule, Philox blocks per lane); items run
 * largest first.  Results do not depend on it: trajectories and records equal
 * those of whole-warp per-class launches (mcmcmc_batch_set_layout lanes 32,
 * staging 2) bit for bit.  mcmcmc_batch_set_layout and a nonzero
 * mcmcmc_batch_set_cluster turn it off; mcmcmc_batch_autotune may turn it on
 * or off (it keeps whichever runs the whole batch faster).  Drops autotuned
 * choices and a captured graph; the previous plan is kept on any error.
 */
sk_status mcmcmc_batch_set_fused(sk_batch* b, uint32_t warps_per_cta);

/* Launch geometry of the batch (for reports): the largest grid, warps per
 * CTA and dynamic shared memory of the first launch class, total work items. */
sk_status mcmcmc_batch_info(const sk_batch* b, uint32_t* grid, uint32_t* warps_per_cta,
                            uint32_t* smem_bytes, uint32_t* items);

/*
 * mcmcmc_batch_classes: the batch's launch classes.  Work items are grouped
 * by coupling kind and rule, by the Philox blocks of proposals a step draws
 * (ceil(K/4) rounded up to a power of two, so that one kernel shape serves
 * every run of the class) and by shared-memory size bucket (chains of
 * similar N), one persistent launch per
 * class, so small-N runs keep many chains per CTA next to large-N runs.
 * *count receives the number of classes; desc (6 x max uint32, may be NULL)
 * receives per class: kernel class, lanes per chain, shared bytes per chain,
 * warps per CTA, work items, CTAs.  Cluster-per-chain classes report kernel
 * class 1024 + 2 kind + rule, 32 x (CTAs per cluster) lanes per chain, the
 * bytes of one chain's slices per CTA and chains per cluster as warps per CTA;
 * the fused launch (mcmcmc_batch_set_fused) reports kernel class 2048, 32
 * lanes, the largest run's bytes per chain and its warps per CTA; team
 * classes report kernel class 4096 + 2 kind + rule, 32 x (warps per chain)
 * lanes, the bytes per chain and the chains per CTA as warps per CTA.
 */
sk_status mcmcmc_batch_classes(const sk_batch* b, uint32_t max, uint32_t* count, uint32_t* desc);

sk_status mcmcmc_batch_free(sk_batch* b);

/* ---------------------------------------------------------------------- */
/* Allocation-free run.  The paper has no counterpart: this entry point   */
/* exists for callers of this library that cannot allocate device memory. */
/* ---------------------------------------------------------------------- */

/* Size of the fixed device array that mcmcmc_run_noalloc works in. */
#define SK_NOALLOC_SCRATCH_BYTES (16u << 20)

/*
 * mcmcmc_run_noalloc: runs `steps` Monte Carlo steps of `chains` chains, the
 * same step kernel as mcmcmc_run with these arguments, without allocating
 * anything: no cudaMalloc, no cudaFree, no allocating library routine.  Its
 * start fields h = J s come from the CUDA cores (no tensor-core operand
 * buffers), so results equal mcmcmc_run's bit for bit for +-J couplings and
 * within the Gaussian parity tolerance otherwise.  It is for callers that cannot allocate device memory or let a
 * library do so: applications whose device memory is owned entirely by their
 * own pool allocator (an extra cudaMalloc would fail or fragment the pool),
 * latency-critical loops that cannot afford cudaMalloc's implicit device
 * synchronisation, and plug-in hosts that forbid libraries from allocating.
 *
 *   N, kind, scale       as for sk_create_instance;
 *   couplings            device pointer, N*N row-major (int8 for SK_J_PM1,
 *                        float32 for SK_J_GAUSS), symmetric, zero diagonal
 *                        (not checked: the caller vouches for it);
 *   chains, K, rule, beta, seed, stream_id   as in sk_run_params;
 *   spins                device pointer, chains*N int8 +-1: the start state
 *                        on input, the state after `steps` steps on output;
 *                        checked on the device first: a value other than +-1
 *                        returns SK_ERR_INVALID_ARG naming its chain and site
 *                        and leaves every buffer unchanged;
 *   energy               device pointer, chains doubles: E of the final states;
 *   stream               cudaStream_t (as void*) or NULL.
 * No records, traces or counters are kept.
 *
 * Working memory: a file-scope device array of SK_NOALLOC_SCRATCH_BYTES
 * (16 MiB), which every GPU that loads the library holds until the process
 * exits.  It must hold the padded couplings (Npad^2 bytes for +-J, 4 Npad^2
 * for Gaussian; Npad = N rounded up to a multiple of 32), 5 bytes per spin of
 * every chain (chains*Npad*5), 20 bytes per chain, the launch descriptors and
 * the +-J weight table; a larger problem returns SK_ERR_INVALID_ARG with the
 * size it would need (e.g. N = 512 Gaussian fits about 6,000 chains).
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins.  Every call reuses the same array, which
 * keeps the previous call's contents; the call clears what must start at
 * zero.  Calls that overlap on the GPU (from several host threads or
 * streams) race on the array: serialise them.  The call is synchronous: it
 * waits on `stream` for the spin check, for its descriptor copies and for the
 * final error word, and returns when all its work on `stream` has finished; a
 * timed-out device wait gives SK_ERR_TIMEOUT.
 */
sk_status mcmcmc_run_noalloc(uint32_t N, uint32_t kind, const void* couplings, double scale,
                             uint32_t chains, uint32_t K, uint32_t rule, double beta,
                             uint64_t seed, uint32_t stream_id, uint64_t steps, int8_t* spins,
                             double* energy, void* stream);

/* ---------------------------------------------------------------------- */
/* Generation probabilities of sets of configurations (App. D)             */
/* ---------------------------------------------------------------------- */
/*
 * sk_set_generation: for a set S of n elements and a generation
 * probability P_gen(e | p) between them, the probability that the growth
 * process of App. D.1 -- add one element at a time, generated from a parent
 * chosen uniformly in the current set -- produces S from S \ M, for every
 * subset M of S (Eq. eq_def_rec_P), by the recursion on the first addition
 * (App. D.2; the printed recursion's normalisation differs from the process
 * by a factor that depends only on |M|, which cancels between sets of one
 * cardinality).  Computed on the device in double precision, one launch per
 * cardinality, in one of two forms:
 *   SK_SETGEN_DIRECT      every sum_{p in S \ M} P_gen(e | p) afresh,
 *                         O(n^2 2^n) work;
 *   SK_SETGEN_CUMULATIVE  the paper's cumulative table (Eq. eq_rec_set_short),
 *                         O(n 2^n) work and n 2^n doubles of device memory
 *                         (SK_ERR_OOM if they cannot be allocated);
 *   SK_SETGEN_AUTO        the cumulative form when its table can be
 *                         allocated, else the direct one.
 * The two agree to rounding (the cumulative table subtracts terms).
 *   n      1..28 elements;
 *   P      n*n doubles, host, P[e*n + p] = P_gen(e | p) (finite, >= 0; the
 *          diagonal is not used);
 *   out    2^n doubles (mem): out[M] for the bit mask M of the missing
 *          elements, out[0] = 1, out[2^n - 1] = 0 (no starting element);
 *   stream cudaStream_t (as void*) or NULL.  Synchronises.
 */
typedef enum { SK_SETGEN_AUTO = 0, SK_SETGEN_DIRECT = 1, SK_SETGEN_CUMULATIVE = 2 } sk_setgen_method;
sk_status sk_set_generation(uint32_t n, const double* P, double* out, uint32_t mem, uint32_t method,
                            void* stream);

/* ---------------------------------------------------------------------- */
/* Request server: continuous batching of sampling jobs                    */
/* ---------------------------------------------------------------------- */
typedef struct sk_server sk_server;

typedef enum {
    SK_JOB_QUEUED = 0,
    SK_JOB_RUNNING = 1,
    SK_JOB_DONE = 2,
    SK_JOB_FAILED = 3,
    SK_JOB_CANCELLED = 4
} sk_job_state;

typedef struct {
    uint32_t N, kind;         /* couplings: N spins, sk_jkind                       */
    const void* couplings;    /* host N*N, copied at submit (couplings_id == 0)      */
    uint64_t couplings_id;    /* nonzero: couplings registered with                 */
                              /*   sk_server_add_couplings (couplings may be NULL)  */
    double scale;             /* energy scale, > 0                                  */
    uint32_t chains, K, rule; /* as in sk_run_params                                */
    double beta;
    uint64_t seed;
    uint32_t stream_id;
    uint64_t steps;           /* Monte Carlo steps of every chain, 1 .. 2^32-1      */
    const int8_t* init_spins; /* host chains*N (+-1) copied at submit, or NULL      */
    double p_center;          /* root distribution, as in sk_run_params (0=uniform) */
} sk_job;

typedef struct {
    uint32_t state;           /* sk_job_state                                       */
    sk_status error;          /* SK_ERR_OOM: larger than the server's budget        */
    double t_submit, t_admit, t_done;  /* seconds since the server's creation       */
    uint64_t footprint_bytes; /* device bytes charged against the budget            */
} sk_job_status;

typedef struct {
    uint64_t chain_steps, candidates, quanta, completed;
    double busy_seconds, elapsed_seconds;  /* device-busy and wall time              */
    uint64_t device_bytes_in_use, queued, running;
    /* the worker's host time between quanta: admitting jobs (their device
     * state and start fields), retiring them (read-back and release), and
     * rebuilding the batch plan when the mix of jobs changed              */
    double admit_seconds, retire_seconds, plan_seconds;
} sk_server_stats_t;

/*
 * sk_server_create: starts a request server with a worker thread and its own
 * CUDA stream on the current device.  It runs the admitted jobs in quanta of
 * `quantum_steps` steps: between quanta it retires finished jobs (final spins
 * and energies copied back, device memory released) and admits queued jobs,
 * first in first out, while their device footprint (couplings and their
 * tensor-core operand unless already resident, the run's memory as listed
 * under mcmcmc_create) fits
 * `budget_bytes`; each quantum advances every admitted job in one launch per
 * kernel class.  A job's result does not depend on the other jobs it shared
 * launches with (counter-based draws).  The paper's problem statement
 * (Sec. II) applied to many independent requests.
 */
sk_status sk_server_create(uint64_t budget_bytes, uint32_t quantum_steps, sk_server** out);

/* Registers couplings (host copy kept by the server) under a nonzero id for
 * jobs to share; the device copy is made when a job first needs it and kept
 * while the budget allows. */
sk_status sk_server_add_couplings(sk_server* s, uint64_t couplings_id, uint32_t N, uint32_t kind,
                                  const void* couplings, double scale);

/* Queues a job; *ticket identifies it.  Jobs larger than the budget are
 * marked failed with SK_ERR_OOM at once. */
sk_status sk_server_submit(sk_server* s, const sk_job* job, uint64_t* ticket);

/* Current status of a job (host struct). */
sk_status sk_server_poll(sk_server* s, uint64_t ticket, sk_job_status* status);

/* Result of a finished job: energies (chains doubles), spins (chains*N int8,
 * may be NULL), spins flipped in total (may be NULL); host pointers.  Returns
 * SK_ERR_NOT_READY while the job is queued or running, the job's error if it
 * failed, SK_ERR_CANCELLED if it was cancelled.  The job is forgotten
 * afterwards. */
sk_status sk_server_result(sk_server* s, uint64_t ticket, double* energies, int8_t* spins,
                           uint64_t* flips);

/*
 * sk_server_cancel: withdraws a job.  A queued job leaves the queue at once;
 * a running job stops at the end of the quantum in flight and its device
 * memory is released (its partial state is not kept).  Either way its state
 * becomes SK_JOB_CANCELLED and sk_server_result returns SK_ERR_CANCELLED; the
 * other jobs are not affected (their draws do not depend on the mix).
 * Cancelling a cancelled job is a no-op; a finished or failed job, or an
 * unknown ticket, gives SK_ERR_INVALID_ARG.
 */
sk_status sk_server_cancel(sk_server* s, uint64_t ticket);

/* Blocks until no job is queued or running (timeout_ns 0 = no limit). */
sk_status sk_server_wait_all(sk_server* s, uint64_t timeout_ns);

sk_status sk_server_stats(sk_server* s, sk_server_stats_t* out);

/* Stops the worker (queued jobs are dropped) and frees everything. */
sk_status sk_server_destroy(sk_server* s);

/* Message of the last failed call on this thread ("" if none). */
const char* sk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SK_MCMCMC_H */
