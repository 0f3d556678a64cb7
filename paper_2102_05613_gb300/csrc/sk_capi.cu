// sk_capi.cu -- host runtime behind the C ABI of include/sk_mcmcmc.h:
// coupling store, run state and records, +-J weight tables, work-item
// planning for batched persistent launches, bounded waits and errors.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <set>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sk_internal.h"
#include "sk_mcmcmc.h"

using sk::JobDev;
using sk::WorkItem;

namespace {

thread_local std::string g_err;

sk_status fail(sk_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define SK_CU(call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(SK_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

uint32_t pad_n(uint32_t n) { return (n + sk::kPadTo - 1) / sk::kPadTo * sk::kPadTo; }
size_t jbytes(uint32_t kind) { return kind == SK_J_PM1 ? 1 : 4; }

// The device the library runs on must be an sm_103 part (the only target
// the kernels are built for).
sk_status check_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0)
        return fail(SK_ERR_CUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
    int dev = 0, major = 0, minor = 0;
    SK_CU(cudaGetDevice(&dev));
    SK_CU(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    SK_CU(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    if (major != 10 || minor != 3)
        return fail(SK_ERR_CUDA, "device compute capability %d.%d: this library is built for sm_103a only",
                    major, minor);
    return SK_OK;
}

template <typename T>
sk_status dalloc(T** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return SK_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SK_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    return SK_OK;
}

// +-J weight tables (exact integer arithmetic on both the chain and its
// checks): MCMCMC W[d] = round(2^52 exp(-2 beta_eff d)) for d = (dE - min)/2
// until the first entry that rounds to zero; Metropolis M[k] =
// round(2^53 exp(-2 beta_eff k)) for dE = 2k, k = 0..N.
std::vector<uint64_t> mcmcmc_table(double beta_eff, uint32_t N) {
    std::vector<uint64_t> w;
    const uint32_t dmax = 4 * N + 4;
    for (uint32_t d = 0; d <= dmax; ++d) {
        const double v = std::nearbyint(std::ldexp(std::exp(-2.0 * beta_eff * d), 52));
        if (!(v > 0.0)) break;
        w.push_back(static_cast<uint64_t>(v));
    }
    return w;
}
std::vector<uint64_t> metropolis_table(double beta_eff, uint32_t N) {
    std::vector<uint64_t> m(N + 1);
    for (uint32_t k = 0; k <= N; ++k)
        m[k] = static_cast<uint64_t>(std::nearbyint(std::ldexp(std::exp(-2.0 * beta_eff * k), 53)));
    // entries that round to 0 are dropped from the end: lookups past the
    // table's end read 0, and a short table fits the kernels' shared copy
    while (m.size() > 1 && m.back() == 0) m.pop_back();
    return m;
}

// Node count of a graph template (0 if the parameters are outside the
// supported range): the full k-ary tree of depth D (k >= 2, 1 <= D <= 16)
// or the line of L nodes (2 <= L <= 8192); at most 8192 nodes.
uint32_t graph_nodes(uint32_t graph, uint32_t k, uint32_t D, uint32_t L) {
    if (graph == SK_GRAPH_TREE) {
        if (k < 2 || D < 1 || D > 16) return 0;
        uint64_t V = 1, lvl = 1;
        for (uint32_t d = 1; d <= D; ++d) {
            lvl *= k;
            V += lvl;
            if (V > 8192) return 0;
        }
        return static_cast<uint32_t>(V);
    }
    if (graph == SK_GRAPH_LINE) return (L >= 2 && L <= 8192) ? L : 0;
    return 0;
}

// Node factors of a graph (App. B): F_v = 2^20 for the tree (uniform root);
// for the line, F_v = round(2^20 c_v / max c) with c_0 = 1, c_(v+1) =
// c_v (L-1-v)/(v+1) in double precision (c_v = binom(L-1, v), the addition
// process's root distribution).  Table layout: F (u32), inclusive prefix
// sums (u64), log2(F / 2^20) (float), the node's depth in the tree template
// (u8; 0 for the line), each of V rounded up to 4 entries.
std::vector<unsigned char> graph_table(uint32_t graph, uint32_t V, uint32_t arity) {
    const size_t V16 = (static_cast<size_t>(V) + 3u) & ~static_cast<size_t>(3u);
    std::vector<unsigned char> t(sk::graph_table_bytes(V), 0);
    uint32_t* F = reinterpret_cast<uint32_t*>(t.data());
    uint64_t* P = reinterpret_cast<uint64_t*>(t.data() + 4 * V16);
    float* lg = reinterpret_cast<float*>(t.data() + 12 * V16);
    uint8_t* dep = t.data() + 16 * V16;
    if (graph == SK_GRAPH_TREE)
        for (uint32_t v = 1; v < V; ++v) dep[v] = static_cast<uint8_t>(dep[(v - 1) / arity] + 1);
    if (graph == SK_GRAPH_LINE) {
        std::vector<double> c(V);
        const uint32_t n = V - 1;
        double cmax = 1.0;
        c[0] = 1.0;
        for (uint32_t v = 0; v < n; ++v) {
            c[v + 1] = c[v] * static_cast<double>(n - v) / static_cast<double>(v + 1);
            if (c[v + 1] > cmax) cmax = c[v + 1];
        }
        for (uint32_t v = 0; v < V; ++v) F[v] = static_cast<uint32_t>(c[v] / cmax * 1048576.0 + 0.5);
    } else {
        for (uint32_t v = 0; v < V; ++v) F[v] = 1u << 20;
    }
    uint64_t acc = 0;
    for (uint32_t v = 0; v < V; ++v) {
        acc += F[v];
        P[v] = acc;
        lg[v] = F[v] ? static_cast<float>(std::log2(static_cast<double>(F[v])) - 20.0) : -INFINITY;
    }
    return t;
}

}  // namespace

namespace sk {
void set_error_message(const char* msg) { g_err = msg; }
}  // namespace sk

struct sk_instance {
    std::atomic<int> runs{0};  // runs created on the instance and not yet freed
    uint32_t N = 0, Npad = 0, kind = 0;
    double scale = 1.0;
    void* dJ = nullptr;
    void* dJop = nullptr;   // couplings as tensor-core operands (built on first recompute)
    bool jop_valid = false;
    void* dJstage = nullptr;              // new couplings, checked before they replace dJ
    unsigned long long* dflag = nullptr;  // result word of the device input checks
    // host inputs are copied and checked on the shared input stream (or, when
    // the staging buffer is still being read, on this side stream), so that
    // the check does not wait for the compute queued on st; events order the
    // staging buffers between the streams
    cudaStream_t side = nullptr;
    cudaStream_t stage_st = nullptr;  // where the last couplings stage was made (input_stream() or side)
    cudaEvent_t ev_side = nullptr;   // side: copy and check done
    cudaEvent_t ev_jfree = nullptr;  // st: dJstage copied into dJ
    cudaEvent_t ev_main = nullptr;   // st: work queued before a start state written on side
    unsigned long long* hflag = nullptr;  // pinned host copy of dflag
    cudaStream_t st = nullptr;
};

struct sk_batch {
    // Work items are grouped by launch class: the kernel class (coupling
    // kind, rule, Philox blocks per lane), the fewest lanes per chain the
    // runs' K allows, and a shared-memory size bucket, so that runs with small
    // N get many chains per CTA even when the batch also holds large-N runs.
    // Each class is one persistent launch with its own lanes per chain G and
    // warps per CTA W (W * 32/G chains per CTA).
    struct Class {
        uint64_t key;
        int cls;                 // kernel class incl. G and staging (step_class)
        uint32_t G, gmin;        // lanes per chain: chosen, fewest allowed
        uint32_t graph;          // 1 k-ary tree, 2 line: the graph kernel (one chain per warp); 0 the star
        uint32_t stage;          // row a staged by TMA (1) or read through L1 (0)
        uint32_t per_chain_staged, per_chain_direct;
        uint32_t per_chain;      // shared memory per chain
        uint32_t W;              // warps per CTA (cluster classes: chains per cluster)
        uint32_t nw = 1;         // graph classes: warps per chain
        uint32_t first_item, n_items, grid;
        // cluster-per-chain layout: CTAs per cluster (0: a warp layout), the
        // J columns each CTA holds, the coupling kind, rule and Philox blocks
        // per lane of the kernel
        uint32_t cluster = 0, jbytes = 0, kind = 0, rule = 0, nb = 0;
        // fused launch: every star item of the batch in one kernel (fsmem:
        // its dynamic shared memory)
        bool fused = false;
        uint32_t fsmem = 0;
        // team layout: warps per chain (2 or 4; 0: another layout); W is then
        // the chains (teams) per CTA
        uint32_t team = 0;
    };
    std::vector<sk_run*> runs;
    std::vector<Class> classes;
    std::map<uint64_t, uint32_t> tuned;  // key -> (stage << 16) | (G << 8) | W chosen by the autotuner
                                         // (graph classes: (warps per chain << 16) | (32 << 8) | W;
                                         // cluster layout: (CTAs per cluster << 24) | (32 << 8) | chains;
                                         // team layout: G = 64 or 128 lanes, W = chains per CTA)
    uint32_t W_override = 0;             // warps_per_cta given at creation (0: as many as fit)
    uint32_t G_override = 0;             // mcmcmc_batch_set_layout lanes (0: default; graph classes
                                         // take lanes / 32 warps per chain when lanes >= 64)
    uint32_t S_override = 0;             // mcmcmc_batch_set_layout staging (0: default = staged)
    uint32_t C_override = 0;             // mcmcmc_batch_set_cluster CTAs per cluster (0: warp layouts)
    uint32_t CW_override = 0;            // mcmcmc_batch_set_cluster chains per cluster (0: default)
    uint32_t fused_W = 0;                // mcmcmc_batch_set_fused warps per CTA (0: per-class launches)
    JobDev* djobs = nullptr;
    WorkItem* ditems = nullptr;
    uint32_t* dqueue = nullptr;  // one work counter per class (up to kMaxClasses)
    uint32_t n_items = 0, grid = 0;
    cudaStream_t st = nullptr;
    cudaGraphExec_t graph = nullptr;  // mcmcmc_batch_capture
    uint64_t graph_steps = 0;
    // several classes: their launches fork from `st` onto side streams and
    // join back, so that one class's last CTAs share the SMs with the next
    // class's first ones instead of leaving them idle
    static constexpr uint32_t kSide = 4;
    cudaStream_t side[kSide] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kSide] = {};
};

struct sk_run {
    std::atomic<int> batches{0};  // live batches holding the run (its own included)
    sk_instance* inst = nullptr;
    sk_run_params p{};
    uint32_t chains = 0;
    int8_t* ds = nullptr;
    void* dh = nullptr;
    int8_t* dstage = nullptr;  // start spins from the host, checked before use
    cudaStream_t stage_st = nullptr;  // where the last spins stage was made (input_stream() or side)
    cudaEvent_t ev_sfree = nullptr;  // st: the start kernel has read dstage
    unsigned long long* dflag = nullptr;  // result word of the start-spin check
    unsigned long long* hflag = nullptr;  // its pinned host copy
    uint32_t* dacc = nullptr;
    unsigned long long* dwork = nullptr;
    double* drecE = nullptr;
    uint32_t* drecAcc = nullptr;
    double* drecQ = nullptr;
    double* drecEnw = nullptr;
    unsigned char* dgtab = nullptr;  // graph runs: node factors and their prefix sums
    int32_t* dtrace = nullptr;
    uint64_t* dW = nullptr;
    uint32_t wlen = 0;
    uint64_t* dstep = nullptr;
    int* derr = nullptr;
    void* dSop = nullptr;                 // spins as tensor-core operands
    bool sop_valid = false;               // dSop holds the current spins (queued work included)
    unsigned int* dCnt = nullptr;         // per 32 chains: the recompute's tile arrivals (zero between)
    double* ddE = nullptr;                // per chain energy drift accumulator
    unsigned long long* dstats = nullptr; // [0..2] periodic recomputes, [3..5] last explicit one
    uint64_t n_recomputes = 0;
    uint64_t step = 0;  // host mirror of the device step counter
    JobDev job{};
    sk_batch* self = nullptr;
};

namespace {


// Couplings (host or device, N x N) into the padded device layout, checked
// on the device: zero diagonal, entries in {-1,0,1} (+-J) or finite
// (Gaussian), symmetry.  A new instance takes them directly; an existing one
// receives them in a staging copy first, so that couplings that fail the
// check leave the instance unchanged.  Host couplings go through the side
// stream (the check then does not wait for work queued on st); device
// couplings, which work on st may still be producing, through st.
// Three phases, so that many instances can be checked with one wait:
// couplings_stage enqueues copy, check and the read-back of the result;
// couplings_verify (after the stream it returns has been synchronised)
// reports a violation; couplings_commit makes the staged copy current.
// One stream per device for the copies and checks of host inputs, shared by
// all instances (created on first use, kept until the process exits).
// Per-instance streams would be many more streams than the device has
// hardware work queues, and a stream that shares a queue with a stream
// running a step kernel waits for it: the input copies would no longer
// overlap the compute.  A stage that has to wait for its buffer (still read
// by queued work) goes on the instance's own side stream instead, so that the
// shared stream never waits for compute.
cudaStream_t input_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

// The stream for a stage that must follow `busy` (an event on the main stream):
// the shared input stream when the event has completed, else `own` after it.
cudaStream_t stage_stream(cudaEvent_t busy, cudaStream_t own) {
    const cudaError_t q = cudaEventQuery(busy);
    if (q == cudaSuccess) {
        cudaStream_t in = input_stream();
        if (in) return in;
    } else if (q != cudaErrorNotReady) {
        cudaGetLastError();
    }
    return own;
}

sk_status couplings_stage(sk_instance* in, const void* J, uint32_t mem, bool fresh, cudaStream_t* used) {
    const size_t b = jbytes(in->kind);
    const size_t bytes = static_cast<size_t>(in->Npad) * in->Npad * b;
    if (!J) return fail(SK_ERR_INVALID_ARG, "couplings are NULL");
    if (mem != SK_MEM_HOST && mem != SK_MEM_DEVICE)
        return fail(SK_ERR_INVALID_ARG, "mem must be SK_MEM_HOST or SK_MEM_DEVICE");
    void* dst = in->dJ;
    if (!fresh) {
        if (!in->dJstage) {
            sk_status s = dalloc(&in->dJstage, bytes);
            if (s != SK_OK) return s;
        }
        dst = in->dJstage;
    }
    const bool via_side = !fresh && mem == SK_MEM_HOST;
    cudaStream_t cs = via_side ? stage_stream(in->ev_jfree, in->side) : in->st;
    if (via_side) SK_CU(cudaStreamWaitEvent(cs, in->ev_jfree, 0));  // the last copy out of the stage is done
    in->stage_st = cs;
    if (in->N != in->Npad) SK_CU(cudaMemsetAsync(dst, 0, bytes, cs));
    SK_CU(cudaMemcpy2DAsync(dst, in->Npad * b, J, in->N * b, in->N * b, in->N, cudaMemcpyDefault, cs));
    SK_CU(sk::launch_check_couplings(dst, in->kind, in->N, in->Npad, in->dflag, cs));
    SK_CU(cudaMemcpyAsync(in->hflag, in->dflag, sizeof(unsigned long long), cudaMemcpyDeviceToHost, cs));
    *used = cs;
    return SK_OK;
}
sk_status couplings_verify(const sk_instance* in) {
    const unsigned long long f = *in->hflag;
    if (f == ~0ull) return SK_OK;
    const unsigned code = static_cast<unsigned>(f & 3u);
    const unsigned i = static_cast<unsigned>((f >> 18) & 0xFFFFu), j = static_cast<unsigned>((f >> 2) & 0xFFFFu);
    if (code == 1) return fail(SK_ERR_INVALID_ARG, "J[%u][%u] != 0 (diagonal must be zero)", i, j);
    if (code == 2)
        return fail(SK_ERR_INVALID_ARG, in->kind == SK_J_PM1 ? "J[%u][%u] is not in {-1,0,1}"
                                                             : "J[%u][%u] is not finite", i, j);
    return fail(SK_ERR_INVALID_ARG, "J is not symmetric at (%u,%u)", i, j);
}
sk_status couplings_commit(sk_instance* in, bool fresh) {
    if (!fresh) {
        const size_t bytes = static_cast<size_t>(in->Npad) * in->Npad * jbytes(in->kind);
        SK_CU(cudaEventRecord(in->ev_side, in->stage_st ? in->stage_st : in->side));  // the stage before the copy
        SK_CU(cudaStreamWaitEvent(in->st, in->ev_side, 0));
        SK_CU(cudaMemcpyAsync(in->dJ, in->dJstage, bytes, cudaMemcpyDeviceToDevice, in->st));
        SK_CU(cudaEventRecord(in->ev_jfree, in->st));
    }
    in->jop_valid = false;
    return SK_OK;
}
sk_status upload_couplings(sk_instance* in, const void* J, uint32_t mem, bool fresh) {
    cudaStream_t cs = nullptr;
    sk_status s = couplings_stage(in, J, mem, fresh, &cs);
    if (s != SK_OK) return s;
    SK_CU(cudaStreamSynchronize(cs));
    if ((s = couplings_verify(in)) != SK_OK) return s;
    return couplings_commit(in, fresh);
}

sk_status check_run_error(sk_run* r) {
    int h = 0;
    SK_CU(cudaMemcpyAsync(&h, r->derr, sizeof(int), cudaMemcpyDeviceToHost, r->inst->st));
    SK_CU(cudaStreamSynchronize(r->inst->st));
    if (h == sk::kDevTimeout) return fail(SK_ERR_TIMEOUT, "a bounded device wait expired in the step kernel");
    if (h == sk::kDevBounds) return fail(SK_ERR_DEVICE, "a kernel reported an out-of-range index");
    return SK_OK;
}

sk_status ensure_recompute(sk_run* r, cudaStream_t cs, bool prepare_j = true);

// Start spins of a run in three phases, as for the couplings: spins_stage
// enqueues the copy of host spins into the run's staging buffer (side
// stream) and their check (+-1) with the read-back of its result;
// spins_verify reports a bad spin; init_commit writes the start state.
sk_status spins_stage(sk_run* r, const int8_t* spins, uint32_t mem, cudaStream_t* used, const int8_t** dinit) {
    sk_instance* in = r->inst;
    *dinit = nullptr;
    *used = nullptr;
    if (!spins) return SK_OK;
    const size_t n = static_cast<size_t>(r->chains) * in->N;
    if (mem == SK_MEM_DEVICE) {
        *dinit = spins;
    } else if (mem == SK_MEM_HOST) {
        if (!r->dstage) {
            sk_status s = dalloc(&r->dstage, n);
            if (s != SK_OK) return s;
        }
        r->stage_st = stage_stream(r->ev_sfree, in->side);
        SK_CU(cudaStreamWaitEvent(r->stage_st, r->ev_sfree, 0));  // the last start has read the stage
        SK_CU(cudaMemcpyAsync(r->dstage, spins, n, cudaMemcpyHostToDevice, r->stage_st));
        *dinit = r->dstage;
    } else {
        return fail(SK_ERR_INVALID_ARG, "init_mem must be SK_MEM_HOST or SK_MEM_DEVICE");
    }
    cudaStream_t cs = mem == SK_MEM_HOST ? r->stage_st : in->st;
    SK_CU(sk::launch_check_spins(*dinit, n, r->dflag, cs));
    SK_CU(cudaMemcpyAsync(r->hflag, r->dflag, sizeof(unsigned long long), cudaMemcpyDeviceToHost, cs));
    *used = cs;
    return SK_OK;
}
sk_status spins_verify(const sk_run* r) {
    const unsigned long long f = *r->hflag;
    if (f != ~0ull) return fail(SK_ERR_INVALID_ARG, "initial spin %llu is not +-1", f >> 2);
    return SK_OK;
}
sk_status init_commit(sk_run* r, const int8_t* dinit, bool on_side = false);

sk_status init_state(sk_run* r, const int8_t* spins, uint32_t mem) {
    cudaStream_t cs = nullptr;
    const int8_t* dinit = nullptr;
    sk_status s = spins_stage(r, spins, mem, &cs, &dinit);
    if (s != SK_OK) return s;
    if (dinit) {  // spins given and checked on cs (which may be the legacy stream, 0)
        SK_CU(cudaStreamSynchronize(cs));
        if ((s = spins_verify(r)) != SK_OK) return s;
    }
    return init_commit(r, dinit);
}

// Writes the start state of a run (records and counters cleared, spins from
// dinit or the Philox start, fields on the tensor cores).  on_side: the work
// goes on the instance's side stream after everything queued on st, and st
// then waits for it -- the starts of runs on different instances overlap.
sk_status init_commit(sk_run* r, const int8_t* dinit, bool on_side) {
    sk_instance* in = r->inst;
    cudaStream_t cs = in->st;
    if (on_side) {
        if (dinit && dinit == r->dstage && r->stage_st && r->stage_st != in->side) {  // staged elsewhere
            SK_CU(cudaEventRecord(in->ev_side, r->stage_st));
            SK_CU(cudaStreamWaitEvent(in->side, in->ev_side, 0));
        }
        SK_CU(cudaEventRecord(in->ev_main, in->st));
        SK_CU(cudaStreamWaitEvent(in->side, in->ev_main, 0));
        cs = in->side;
    } else if (dinit && dinit == r->dstage) {  // the staged copy was made on its stage stream
        SK_CU(cudaEventRecord(in->ev_side, r->stage_st ? r->stage_st : in->side));
        SK_CU(cudaStreamWaitEvent(in->st, in->ev_side, 0));
    }
    SK_CU(cudaMemsetAsync(r->dstep, 0, sizeof(uint64_t), cs));
    SK_CU(cudaMemsetAsync(r->derr, 0, sizeof(int), cs));
    const uint64_t R = r->p.max_records;
    if (R && r->p.record_every) {
        SK_CU(cudaMemsetAsync(r->drecE, 0, R * r->chains * sizeof(double), cs));
        SK_CU(cudaMemsetAsync(r->drecAcc, 0, R * r->chains * sizeof(uint32_t), cs));
        if (r->chains >= 2) SK_CU(cudaMemsetAsync(r->drecQ, 0, R * (r->chains / 2) * sizeof(double), cs));
        if (r->drecEnw) SK_CU(cudaMemsetAsync(r->drecEnw, 0, R * r->chains * sizeof(double), cs));
    }
    if (r->dtrace)
        SK_CU(cudaMemsetAsync(r->dtrace, 0xff, static_cast<size_t>(r->p.trace_chains) * r->p.trace_steps * 4, cs));
    // spins, then the fields h = J s on the tensor cores (e4m3 for +-J:
    // exact; three bf16 terms of J for Gaussian couplings: fp32 accumulation)
    SK_CU(sk::launch_init(&r->job, dinit, r->chains, in->N, in->Npad, in->kind, cs, false));
    if (dinit == r->dstage && dinit) SK_CU(cudaEventRecord(r->ev_sfree, cs));
    {
        sk_status s = ensure_recompute(r, cs);
        if (s != SK_OK) return s;
        SK_CU(sk::launch_recompute(in->kind, r->ds, r->dh, nullptr, r->dSop, in->dJop, r->ddE, r->dstats,
                                   r->derr, r->chains, in->Npad, 3, 3, in->scale, cs));
        r->sop_valid = true;  // the conversion of the start spins
    }
    SK_CU(cudaMemsetAsync(r->dstats, 0, 6 * sizeof(unsigned long long), cs));
    SK_CU(cudaMemsetAsync(r->ddE, 0, static_cast<size_t>(r->chains) * sizeof(double), cs));
    if (on_side) {
        SK_CU(cudaEventRecord(in->ev_side, in->side));
        SK_CU(cudaStreamWaitEvent(in->st, in->ev_side, 0));
    }
    r->n_recomputes = 0;
    r->step = 0;
    return SK_OK;
}

void free_run_buffers(sk_run* r) {
    cudaFree(r->ds);
    cudaFree(r->dh);
    cudaFree(r->dacc);
    cudaFree(r->dwork);
    cudaFree(r->drecE);
    cudaFree(r->drecAcc);
    cudaFree(r->drecQ);
    cudaFree(r->drecEnw);
    cudaFree(r->dgtab);
    cudaFree(r->dtrace);
    cudaFree(r->dW);
    cudaFree(r->dstep);
    cudaFree(r->derr);
    cudaFree(r->dSop);
    cudaFree(r->dCnt);
    cudaFree(r->ddE);
    cudaFree(r->dstats);
    cudaFree(r->dstage);
    if (r->ev_sfree) cudaEventDestroy(r->ev_sfree);
    cudaFree(r->dflag);
    if (r->hflag) cudaFreeHost(r->hflag);
}

// Operand buffers of the tensor-core recompute, allocated on first use.
sk_status ensure_recompute(sk_run* r, cudaStream_t cs, bool prepare_j) {
    sk_instance* in = r->inst;
    sk_status s = SK_OK;
    if (!in->dJop) s = dalloc(&in->dJop, sk::recompute_j_bytes(in->kind, in->Npad));
    if (s == SK_OK && !r->dSop) s = dalloc(&r->dSop, sk::recompute_s_bytes(in->kind, r->chains, in->Npad));
    if (s == SK_OK && !r->dCnt) {  // groups of 32 chains of the 128-chain tiles
        const size_t words = 4 * ((static_cast<size_t>(r->chains) + 127) / 128);
        s = dalloc(&r->dCnt, words * sizeof(unsigned int));
        if (s == SK_OK) SK_CU(cudaMemsetAsync(r->dCnt, 0, words * sizeof(unsigned int), cs));
    }
    if (s == SK_OK && !r->ddE) {
        s = dalloc(&r->ddE, static_cast<size_t>(r->chains) * sizeof(double));
        if (s == SK_OK) SK_CU(cudaMemsetAsync(r->ddE, 0, static_cast<size_t>(r->chains) * sizeof(double), cs));
    }
    if (s == SK_OK && !r->dstats) {
        s = dalloc(&r->dstats, 6 * sizeof(unsigned long long));
        if (s == SK_OK) SK_CU(cudaMemsetAsync(r->dstats, 0, 6 * sizeof(unsigned long long), cs));
    }
    if (s != SK_OK) return s;
    if (prepare_j && !in->jop_valid) {
        SK_CU(sk::recompute_prepare_j(in->dJ, in->kind, in->Npad, in->dJop, cs));
        in->jop_valid = true;
    }
    return SK_OK;
}

uint32_t terms_of(const sk_run* r) { return r->p.recompute_terms ? r->p.recompute_terms : 3u; }

// Periodic recompute after a step segment: +-J check, Gaussian resync.
sk_status periodic_recompute(sk_run* r) {
    sk_status s = ensure_recompute(r, r->inst->st);
    if (s != SK_OK) return s;
    sk_instance* in = r->inst;
    const uint32_t mode = in->kind == SK_J_PM1 ? 0u : 1u;
    SK_CU(sk::launch_recompute(in->kind, r->ds, r->dh, nullptr, r->dSop, in->dJop, r->ddE, r->dstats, r->derr,
                               r->chains, in->Npad, terms_of(r), mode, in->scale, in->st, 0, r->sop_valid, r->dCnt));
    r->sop_valid = true;
    ++r->n_recomputes;
    return SK_OK;
}

constexpr size_t kSmemBudget = 232448 - 5120;  // dynamic smem per CTA; the step kernel's static
                                                // part (mbarriers of 256 chains, job) reserved

}  // namespace

extern "C" {

const char* sk_last_error(void) { return g_err.c_str(); }

sk_status sk_create_instance(uint32_t N, uint32_t kind, const void* couplings, uint32_t mem, uint64_t seed,
                             double scale, void* stream, sk_instance** out) {
    if (!out) return fail(SK_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (N < 2 || N > SK_MAX_N) return fail(SK_ERR_INVALID_ARG, "N = %u outside 2..%u", N, SK_MAX_N);
    if (kind != SK_J_PM1 && kind != SK_J_GAUSS) return fail(SK_ERR_INVALID_ARG, "unknown coupling kind %u", kind);
    if (couplings && mem != SK_MEM_HOST && mem != SK_MEM_DEVICE)
        return fail(SK_ERR_INVALID_ARG, "mem must be SK_MEM_HOST or SK_MEM_DEVICE");
    if (!(scale > 0.0) || !std::isfinite(scale)) return fail(SK_ERR_INVALID_ARG, "scale must be > 0");
    sk_status s = check_device();
    if (s != SK_OK) return s;
    sk_instance* in = new sk_instance();
    in->N = N;
    in->Npad = pad_n(N);
    in->kind = kind;
    in->scale = scale;
    in->st = static_cast<cudaStream_t>(stream);
    s = dalloc(&in->dJ, static_cast<size_t>(in->Npad) * in->Npad * jbytes(kind));
    if (s == SK_OK) s = dalloc(&in->dflag, sizeof(unsigned long long));
    if (s == SK_OK) {
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&in->hflag), sizeof(unsigned long long), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&in->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&in->ev_side, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&in->ev_jfree, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&in->ev_main, cudaEventDisableTiming);
        if (e != cudaSuccess) s = fail(SK_ERR_CUDA, "stream/event creation: %s", cudaGetErrorString(e));
    }
    if (s == SK_OK) {
        if (couplings) {
            s = upload_couplings(in, couplings, mem, true);
        } else {  // drawn on the device from the seed, then checked like any input
            cudaError_t e = sk::launch_gen_couplings(in->dJ, kind, N, in->Npad, seed, in->st);
            if (e == cudaSuccess) e = sk::launch_check_couplings(in->dJ, kind, N, in->Npad, in->dflag, in->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(in->hflag, in->dflag, sizeof(unsigned long long), cudaMemcpyDeviceToHost, in->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(in->st);
            if (e != cudaSuccess) s = fail(SK_ERR_CUDA, "coupling generation: %s", cudaGetErrorString(e));
            if (s == SK_OK) s = couplings_verify(in);
            if (s == SK_OK) s = couplings_commit(in, true);
        }
    }
    if (s != SK_OK) {
        cudaFree(in->dJ);
        cudaFree(in->dflag);
        if (in->hflag) cudaFreeHost(in->hflag);
        if (in->ev_side) cudaEventDestroy(in->ev_side);
        if (in->ev_jfree) cudaEventDestroy(in->ev_jfree);
        if (in->ev_main) cudaEventDestroy(in->ev_main);
        if (in->side) cudaStreamDestroy(in->side);
        delete in;
        return s;
    }
    *out = in;
    return SK_OK;
}

sk_status sk_get_couplings(const sk_instance* in, void* out, uint32_t mem) {
    if (!in || !out) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (mem != SK_MEM_HOST && mem != SK_MEM_DEVICE)
        return fail(SK_ERR_INVALID_ARG, "mem must be SK_MEM_HOST or SK_MEM_DEVICE");
    const size_t b = jbytes(in->kind);
    SK_CU(cudaMemcpy2DAsync(out, in->N * b, in->dJ, in->Npad * b, in->N * b, in->N, cudaMemcpyDefault, in->st));
    SK_CU(cudaStreamSynchronize(in->st));
    return SK_OK;
}

sk_status sk_set_couplings(sk_instance* in, const void* couplings, uint32_t mem) {
    if (!in || !couplings) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    return upload_couplings(in, couplings, mem, false);
}

sk_status sk_set_couplings_many(sk_instance* const* insts, uint32_t n, const void* const* couplings, uint32_t mem) {
    if (!insts || !couplings) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    std::set<const sk_instance*> seen;
    for (uint32_t i = 0; i < n; ++i) {
        if (!insts[i] || !couplings[i]) return fail(SK_ERR_INVALID_ARG, "instance or couplings %u is NULL", i);
        if (!seen.insert(insts[i]).second) return fail(SK_ERR_INVALID_ARG, "instance %u appears twice", i);
    }
    std::vector<cudaStream_t> used(n, nullptr);
    for (uint32_t i = 0; i < n; ++i) {
        sk_status s = couplings_stage(insts[i], couplings[i], mem, false, &used[i]);
        if (s != SK_OK) return s;
    }
    std::set<cudaStream_t> streams(used.begin(), used.end());
    for (cudaStream_t cs : streams) SK_CU(cudaStreamSynchronize(cs));
    for (uint32_t i = 0; i < n; ++i) {
        sk_status s = couplings_verify(insts[i]);
        if (s != SK_OK) return fail(s, "instance %u: %s", i, g_err.c_str());
    }
    for (uint32_t i = 0; i < n; ++i) {
        sk_status s = couplings_commit(insts[i], false);
        if (s != SK_OK) return s;
    }
    return SK_OK;
}

sk_status sk_destroy_instance(sk_instance* in) {
    if (!in) return fail(SK_ERR_INVALID_ARG, "instance is NULL");
    if (const int n = in->runs.load(); n > 0)
        return fail(SK_ERR_BUSY, "%d run(s) created on this instance are not freed", n);
    cudaStreamSynchronize(in->st);
    cudaStreamSynchronize(in->side);
    cudaFree(in->dJ);
    cudaFree(in->dJop);
    cudaFree(in->dJstage);
    cudaFree(in->dflag);
    cudaFreeHost(in->hflag);
    cudaEventDestroy(in->ev_side);
    cudaEventDestroy(in->ev_jfree);
    cudaEventDestroy(in->ev_main);
    cudaStreamDestroy(in->side);
    delete in;
    return SK_OK;
}

sk_status sk_energy(const sk_instance* in, const int8_t* spins, uint32_t count, uint32_t mem,
                    double* out_E) {
    if (!in || !spins || !out_E) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (count == 0) return SK_OK;
    const size_t n = static_cast<size_t>(count) * in->N;
    int8_t* tmp = nullptr;
    double* dE = nullptr;
    const int8_t* dsp = spins;
    sk_status s = SK_OK;
    if (mem == SK_MEM_HOST) {
        for (size_t i = 0; i < n; ++i)
            if (spins[i] != 1 && spins[i] != -1) return fail(SK_ERR_INVALID_ARG, "spin %zu is not +-1", i);
        if ((s = dalloc(&tmp, n)) != SK_OK) return s;
        const cudaError_t e = cudaMemcpyAsync(tmp, spins, n, cudaMemcpyHostToDevice, in->st);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return fail(SK_ERR_CUDA, "sk_energy: %s", cudaGetErrorString(e));
        }
        dsp = tmp;
    } else if (mem != SK_MEM_DEVICE) {
        return fail(SK_ERR_INVALID_ARG, "mem must be SK_MEM_HOST or SK_MEM_DEVICE");
    }
    const size_t tiles = sk::energy_tiles(in->N, count);
    if ((s = dalloc(&dE, count * (1 + tiles) * sizeof(double))) != SK_OK) {
        cudaFree(tmp);
        return s;
    }
    cudaError_t e = sk::launch_energy(in->dJ, in->kind, in->N, in->Npad, in->scale, dsp, count, dE, in->st,
                                      tiles > 1 ? dE + count : nullptr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_E, dE, count * sizeof(double), cudaMemcpyDeviceToHost, in->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(in->st);
    cudaFree(tmp);
    cudaFree(dE);
    if (e != cudaSuccess) return fail(SK_ERR_CUDA, "sk_energy: %s", cudaGetErrorString(e));
    return SK_OK;
}

sk_status mcmcmc_create(sk_instance* in, const sk_run_params* p, sk_run** out) {
    if (!in || !p || !out) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (p->chains == 0 || p->chains > (1u << 30)) return fail(SK_ERR_INVALID_ARG, "chains = %u", p->chains);
    if (p->rule != SK_RULE_MCMCMC && p->rule != SK_RULE_METROPOLIS)
        return fail(SK_ERR_INVALID_ARG, "unknown rule %u", p->rule);
    if (p->rule == SK_RULE_MCMCMC && (p->K < 1 || p->K > SK_MAX_K))
        return fail(SK_ERR_INVALID_ARG, "K = %u outside 1..%u", p->K, SK_MAX_K);
    if (!(p->beta >= 0.0) || !std::isfinite(p->beta)) return fail(SK_ERR_INVALID_ARG, "beta must be >= 0");
    if (p->stream_id > 0xFFFFFFu) return fail(SK_ERR_INVALID_ARG, "stream_id must fit 24 bits");
    if (p->trace_chains > p->chains) return fail(SK_ERR_INVALID_ARG, "trace_chains > chains");
    if (p->recompute_terms > 3) return fail(SK_ERR_INVALID_ARG, "recompute_terms must be 0..3");
    if (p->fault_inject & ~(SK_FAULT_WITHHOLD_ROW | SK_FAULT_WITHHOLD_TILE))
        return fail(SK_ERR_INVALID_ARG, "unknown fault_inject bits");
    if (p->graph) {
        if (p->graph != SK_GRAPH_TREE && p->graph != SK_GRAPH_LINE)
            return fail(SK_ERR_INVALID_ARG, "unknown graph %u", p->graph);
        if (p->rule != SK_RULE_MCMCMC) return fail(SK_ERR_INVALID_ARG, "graphs need the MCMCMC rule");
        if (!graph_nodes(p->graph, p->arity, p->depth, p->line_nodes))
            return fail(SK_ERR_INVALID_ARG, "graph outside the supported range (k >= 2, 1 <= depth <= 16, "
                        "2 <= line_nodes, at most 8192 nodes)");
        if (p->p_center != 0.0 || p->node_weighted)
            return fail(SK_ERR_INVALID_ARG, "p_center and node_weighted apply to the star only");
    } else if (p->rule == SK_RULE_MCMCMC) {
        JobDev probe{};
        if (!root_setup(probe, p->K, p->p_center))
            return fail(SK_ERR_INVALID_ARG, "p_center = %g: need 0 (uniform) or 0 < p_center < 1 with both root "
                        "factors >= 2^-21", p->p_center);
    }
    sk_run* r = new sk_run();
    r->inst = in;
    r->p = *p;
    r->chains = p->chains;
    if (r->p.rule == SK_RULE_METROPOLIS) r->p.K = 1;
    const uint32_t V = r->p.graph ? graph_nodes(r->p.graph, r->p.arity, r->p.depth, r->p.line_nodes) : 0;
    if (V) r->p.K = V - 1;  // proposals per step: the graph's other nodes
    if (!r->p.record_every) r->p.max_records = 0;
    if (!r->p.trace_chains || !r->p.trace_steps) r->p.trace_chains = 0, r->p.trace_steps = 0;
    const size_t C = r->chains, np = in->Npad, R = r->p.max_records;
    sk_status s = SK_OK;
    if (s == SK_OK) s = dalloc(&r->ds, C * np);
    if (s == SK_OK) s = dalloc(&r->dh, C * np * 4);
    if (s == SK_OK) s = dalloc(&r->dacc, C * 4);
    if (s == SK_OK) s = dalloc(&r->dwork, C * 16);
    if (s == SK_OK) s = dalloc(&r->drecE, R * C * 8);
    if (s == SK_OK) s = dalloc(&r->drecAcc, R * C * 4);
    if (s == SK_OK) s = dalloc(&r->drecQ, R * (C / 2) * 8);
    if (s == SK_OK && r->p.node_weighted) s = dalloc(&r->drecEnw, R * C * 8);
    if (s == SK_OK && V) {
        const std::vector<unsigned char> t = graph_table(r->p.graph, V, r->p.arity);
        s = dalloc(&r->dgtab, t.size());
        if (s == SK_OK) {
            cudaError_t e = cudaMemcpy(r->dgtab, t.data(), t.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) s = fail(SK_ERR_CUDA, "graph table upload: %s", cudaGetErrorString(e));
        }
    }
    if (s == SK_OK) s = dalloc(&r->dtrace, static_cast<size_t>(r->p.trace_chains) * r->p.trace_steps * 4);
    if (s == SK_OK) s = dalloc(&r->dstep, 8);
    if (s == SK_OK) s = dalloc(&r->derr, 4);
    if (s == SK_OK && cudaEventCreateWithFlags(&r->ev_sfree, cudaEventDisableTiming) != cudaSuccess)
        s = fail(SK_ERR_CUDA, "event creation failed");
    if (s == SK_OK) s = dalloc(&r->dflag, sizeof(unsigned long long));
    if (s == SK_OK && cudaHostAlloc(reinterpret_cast<void**>(&r->hflag), sizeof(unsigned long long),
                                    cudaHostAllocDefault) != cudaSuccess)
        s = fail(SK_ERR_OOM, "pinned host allocation failed");
    if (s == SK_OK && in->kind == SK_J_PM1) {
        const double be = r->p.beta * in->scale;
        std::vector<uint64_t> t = r->p.rule == SK_RULE_MCMCMC ? mcmcmc_table(be, in->N) : metropolis_table(be, in->N);
        r->wlen = static_cast<uint32_t>(t.size());
        s = dalloc(&r->dW, std::max<size_t>(t.size(), 1) * 8);
        if (s == SK_OK && !t.empty()) {
            cudaError_t e = cudaMemcpy(r->dW, t.data(), t.size() * 8, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) s = fail(SK_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
        }
    }
    if (s != SK_OK) {
        free_run_buffers(r);
        delete r;
        return s;
    }
    JobDev& j = r->job;
    j.J = in->dJ;
    j.s = r->ds;
    j.h = r->dh;
    j.W = r->dW;
    j.step = r->dstep;
    j.acc_run = r->dacc;
    j.rec_E = r->drecE;
    j.rec_acc = r->drecAcc;
    j.rec_q = r->drecQ;
    j.rec_Enw = r->drecEnw;
    j.trace = r->dtrace;
    j.err = r->derr;
    j.work = r->dwork;
    j.seed = r->p.seed;
    j.rec_capacity = R;
    j.trace_steps = r->p.trace_steps;
    j.scale = in->scale;
    j.beta_eff = static_cast<float>(r->p.beta * in->scale);
    j.stream = r->p.stream_id;
    j.N = in->N;
    j.Npad = in->Npad;
    j.chains = r->chains;
    j.K = r->p.K;
    j.kind = in->kind;
    j.rule = r->p.rule;
    j.wlen = r->wlen;
    j.record_every = r->p.record_every;
    j.trace_chains = r->p.trace_chains;
    j.step_limit = 0xFFFFFFFFu;
    j.gtab = r->dgtab;
    j.graph = r->p.graph;
    j.arity = r->p.arity;
    j.V = V;
    static_assert(sk::kFaultWithholdRow == SK_FAULT_WITHHOLD_ROW && sk::kFaultWithholdTile == SK_FAULT_WITHHOLD_TILE,
                  "fault bits of the ABI and the kernels");
    j.fault = r->p.fault_inject;
    root_setup(j, r->p.K, r->p.rule == SK_RULE_MCMCMC ? r->p.p_center : 0.0);
    s = init_state(r, p->init_spins, p->init_mem);
    // runs that recompute periodically have the step kernels write their
    // spins' tensor-core operands too
    j.s_op = r->p.recompute_every ? r->dSop : nullptr;
    if (s == SK_OK) {
        sk_run* one[1] = {r};
        s = mcmcmc_batch_create(one, 1, 0, &r->self);
    }
    if (s != SK_OK) {
        std::string keep = g_err;
        cudaStreamSynchronize(in->st);
        free_run_buffers(r);
        delete r;
        g_err = keep;
        return s;
    }
    in->runs++;
    *out = r;
    return SK_OK;
}

sk_status mcmcmc_advance(sk_run* r, uint64_t steps) {
    if (!r) return fail(SK_ERR_INVALID_ARG, "run is NULL");
    return mcmcmc_batch_advance(r->self, steps);
}

sk_status mcmcmc_run(sk_instance* in, const sk_run_params* p, uint64_t steps, sk_run** out) {
    sk_status s = mcmcmc_create(in, p, out);
    if (s != SK_OK) return s;
    s = mcmcmc_advance(*out, steps);
    if (s != SK_OK) {
        mcmcmc_free(*out);
        *out = nullptr;
    }
    return s;
}

sk_status mcmcmc_reset(sk_run* r, const int8_t* spins, uint32_t mem) {
    if (!r) return fail(SK_ERR_INVALID_ARG, "run is NULL");
    return init_state(r, spins, mem);
}

sk_status mcmcmc_reset_many(sk_run* const* runs, uint32_t n, const int8_t* const* spins, uint32_t mem) {
    if (!runs) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    std::set<const sk_run*> seen;
    for (uint32_t i = 0; i < n; ++i) {
        if (!runs[i]) return fail(SK_ERR_INVALID_ARG, "run %u is NULL", i);
        if (!seen.insert(runs[i]).second) return fail(SK_ERR_INVALID_ARG, "run %u appears twice", i);
    }
    std::vector<cudaStream_t> used(n, nullptr);
    std::vector<const int8_t*> dinit(n, nullptr);
    for (uint32_t i = 0; i < n; ++i) {
        sk_status s = spins_stage(runs[i], spins ? spins[i] : nullptr, mem, &used[i], &dinit[i]);
        if (s != SK_OK) return s;
    }
    std::set<cudaStream_t> streams;  // where the checks ran (the legacy stream is 0)
    for (uint32_t i = 0; i < n; ++i)
        if (dinit[i]) streams.insert(used[i]);
    for (cudaStream_t cs : streams) SK_CU(cudaStreamSynchronize(cs));
    for (uint32_t i = 0; i < n; ++i) {
        if (!dinit[i]) continue;
        sk_status s = spins_verify(runs[i]);
        if (s != SK_OK) return fail(s, "run %u: %s", i, g_err.c_str());
    }
    // runs on one stream with one coupling kind: one launch for all start
    // states and one for all their fields; otherwise each run on its own
    bool together = n > 1;
    for (uint32_t i = 0; i < n && together; ++i)
        together = runs[i]->inst->st == runs[0]->inst->st && runs[i]->inst->kind == runs[0]->inst->kind;
    if (!together) {
        for (uint32_t i = 0; i < n; ++i) {
            sk_status s = init_commit(runs[i], dinit[i], true);
            if (s != SK_OK) return s;
        }
        return SK_OK;
    }
    cudaStream_t bs = runs[0]->inst->st;
    for (uint32_t i = 0; i < n; ++i) {  // the staged copies were made on their stage streams
        if (!dinit[i] || dinit[i] != runs[i]->dstage) continue;
        sk_instance* in = runs[i]->inst;
        SK_CU(cudaEventRecord(in->ev_side, runs[i]->stage_st ? runs[i]->stage_st : in->side));
        SK_CU(cudaStreamWaitEvent(bs, in->ev_side, 0));
    }
    std::vector<sk::StartJob> sj(n);
    std::vector<sk::RecomputeSet> rs(n);
    uint64_t max_words = 0;
    // operand buffers, then the coupling operands of every instance whose
    // couplings changed in one launch
    std::vector<sk::PrepareJ> prep;
    for (uint32_t i = 0; i < n; ++i) {
        sk_run* r = runs[i];
        sk_status s = ensure_recompute(r, bs, false);
        if (s != SK_OK) return s;
        sk_instance* in = r->inst;
        if (!in->jop_valid) {
            prep.push_back(sk::PrepareJ{in->dJ, in->dJop, in->Npad, 0});
            in->jop_valid = true;
        }
    }
    SK_CU(sk::recompute_prepare_j_batch(runs[0]->inst->kind, prep.data(), static_cast<uint32_t>(prep.size()), bs));
    for (uint32_t i = 0; i < n; ++i) {
        sk_run* r = runs[i];
        std::memset(&sj[i], 0, sizeof(sk::StartJob));
        sj[i].job = r->job;
        sj[i].init = dinit[i];
        sj[i].dstats = r->dstats;
        sj[i].ddE = r->ddE;
        sj[i].s_op = r->dSop;  // the start kernel writes the spin operands too
        max_words = std::max<uint64_t>(max_words, static_cast<uint64_t>(r->chains) * (r->inst->Npad / 4));
        rs[i] = sk::RecomputeSet{r->ds, r->dh, r->dSop, r->inst->dJop, r->derr, r->chains, r->inst->Npad};
    }
    sk::StartJob* dsj = nullptr;
    SK_CU(cudaMallocAsync(&dsj, n * sizeof(sk::StartJob), bs));
    SK_CU(cudaMemcpyAsync(dsj, sj.data(), n * sizeof(sk::StartJob), cudaMemcpyHostToDevice, bs));
    SK_CU(sk::launch_start_batch(dsj, n, max_words, bs));
    SK_CU(cudaFreeAsync(dsj, bs));
    for (uint32_t i = 0; i < n; ++i)
        if (dinit[i] && dinit[i] == runs[i]->dstage) SK_CU(cudaEventRecord(runs[i]->ev_sfree, bs));
    SK_CU(sk::launch_set_fields_batch(runs[0]->inst->kind, rs.data(), n, bs, true));
    for (uint32_t i = 0; i < n; ++i) runs[i]->sop_valid = true;  // written by the start kernel
    for (uint32_t i = 0; i < n; ++i) {
        runs[i]->n_recomputes = 0;
        runs[i]->step = 0;
    }
    return SK_OK;
}

sk_status mcmcmc_observables_many(sk_run* const* runs, uint32_t n, uint64_t first, uint64_t count,
                                  double* const* energy, double* const* overlap, uint32_t* const* accepted,
                                  uint32_t mem) {
    if (!runs) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (mem != SK_MEM_HOST && mem != SK_MEM_DEVICE) return fail(SK_ERR_INVALID_ARG, "bad mem");
    std::set<cudaStream_t> streams;
    for (uint32_t i = 0; i < n; ++i) {
        sk_run* r = runs[i];
        if (!r) return fail(SK_ERR_INVALID_ARG, "run %u is NULL", i);
        if (first + count > r->p.max_records)
            return fail(SK_ERR_INVALID_ARG, "run %u: records [%llu, %llu) beyond capacity %llu", i,
                        (unsigned long long)first, (unsigned long long)(first + count),
                        (unsigned long long)r->p.max_records);
        streams.insert(r->inst->st);
        SK_CU(cudaMemcpyAsync(r->hflag, r->derr, sizeof(int), cudaMemcpyDeviceToHost, r->inst->st));
    }
    for (cudaStream_t cs : streams) SK_CU(cudaStreamSynchronize(cs));
    for (uint32_t i = 0; i < n; ++i) {
        const int h = *reinterpret_cast<const int*>(runs[i]->hflag);
        if (h == sk::kDevTimeout) return fail(SK_ERR_TIMEOUT, "run %u: a bounded device wait expired", i);
        if (h == sk::kDevBounds) return fail(SK_ERR_DEVICE, "run %u: a kernel reported an out-of-range index", i);
    }
    if (count == 0) return SK_OK;
    for (uint32_t i = 0; i < n; ++i) {
        sk_run* r = runs[i];
        const size_t C = r->chains;
        cudaStream_t st = r->inst->st;
        if (energy && energy[i])
            SK_CU(cudaMemcpyAsync(energy[i], r->drecE + first * C, count * C * 8, cudaMemcpyDefault, st));
        if (accepted && accepted[i])
            SK_CU(cudaMemcpyAsync(accepted[i], r->drecAcc + first * C, count * C * 4, cudaMemcpyDefault, st));
        if (overlap && overlap[i] && C >= 2)
            SK_CU(cudaMemcpyAsync(overlap[i], r->drecQ + first * (C / 2), count * (C / 2) * 8, cudaMemcpyDefault, st));
    }
    for (cudaStream_t cs : streams) SK_CU(cudaStreamSynchronize(cs));
    return SK_OK;
}

sk_status mcmcmc_wait(sk_run* r, uint64_t timeout_ns) {
    if (!r) return fail(SK_ERR_INVALID_ARG, "run is NULL");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(r->inst->st);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return fail(SK_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
        if (timeout_ns) {
            const auto ns = std::chrono::duration_cast<std::chrono::nanoseconds>(
                                std::chrono::steady_clock::now() - t0).count();
            if (static_cast<uint64_t>(ns) >= timeout_ns)
                return fail(SK_ERR_TIMEOUT, "run still in flight after %llu ns", (unsigned long long)timeout_ns);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return check_run_error(r);
}

sk_status mcmcmc_observables(sk_run* r, uint64_t first, uint64_t count, double* energy,
                             double* overlap, uint32_t* accepted, uint32_t mem) {
    if (!r) return fail(SK_ERR_INVALID_ARG, "run is NULL");
    if (mem != SK_MEM_HOST && mem != SK_MEM_DEVICE) return fail(SK_ERR_INVALID_ARG, "bad mem");
    if (first + count > r->p.max_records)
        return fail(SK_ERR_INVALID_ARG, "records [%llu, %llu) beyond capacity %llu", (unsigned long long)first,
                    (unsigned long long)(first + count), (unsigned long long)r->p.max_records);
    sk_status s = mcmcmc_wait(r, 0);
    if (s != SK_OK) return s;
    const size_t C = r->chains;
    cudaStream_t st = r->inst->st;
    if (count == 0) return SK_OK;
    if (energy) SK_CU(cudaMemcpyAsync(energy, r->drecE + first * C, count * C * 8, cudaMemcpyDefault, st));
    if (accepted) SK_CU(cudaMemcpyAsync(accepted, r->drecAcc + first * C, count * C * 4, cudaMemcpyDefault, st));
    if (overlap && C >= 2)
        SK_CU(cudaMemcpyAsync(overlap, r->drecQ + first * (C / 2), count * (C / 2) * 8, cudaMemcpyDefault, st));
    SK_CU(cudaStreamSynchronize(st));
    return SK_OK;
}

sk_status mcmcmc_observables_nw(sk_run* r, uint64_t first, uint64_t count, double* energy_nw, uint32_t mem) {
    if (!r || !energy_nw) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (!r->drecEnw) return fail(SK_ERR_INVALID_ARG, "the run was created without node_weighted records");
    if (mem != SK_MEM_HOST && mem != SK_MEM_DEVICE) return fail(SK_ERR_INVALID_ARG, "bad mem");
    if (first + count > r->p.max_records)
        return fail(SK_ERR_INVALID_ARG, "records [%llu, %llu) beyond capacity %llu", (unsigned long long)first,
                    (unsigned long long)(first + count), (unsigned long long)r->p.max_records);
    sk_status s = mcmcmc_wait(r, 0);
    if (s != SK_OK) return s;
    if (count == 0) return SK_OK;
    const size_t C = r->chains;
    SK_CU(cudaMemcpyAsync(energy_nw, r->drecEnw + first * C, count * C * 8, cudaMemcpyDefault, r->inst->st));
    SK_CU(cudaStreamSynchronize(r->inst->st));
    return SK_OK;
}

sk_status mcmcmc_state(sk_run* r, int8_t* spins, void* fields, uint64_t* step, uint32_t mem) {
    if (!r) return fail(SK_ERR_INVALID_ARG, "run is NULL");
    if (mem != SK_MEM_HOST && mem != SK_MEM_DEVICE) return fail(SK_ERR_INVALID_ARG, "bad mem");
    sk_status s = mcmcmc_wait(r, 0);
    if (s != SK_OK) return s;
    sk_instance* in = r->inst;
    cudaStream_t st = in->st;
    if (spins)
        SK_CU(cudaMemcpy2DAsync(spins, in->N, r->ds, in->Npad, in->N, r->chains, cudaMemcpyDefault, st));
    if (fields)
        SK_CU(cudaMemcpy2DAsync(fields, in->N * 4, r->dh, in->Npad * 4, in->N * 4, r->chains, cudaMemcpyDefault, st));
    uint64_t ds = 0;
    SK_CU(cudaMemcpyAsync(&ds, r->dstep, 8, cudaMemcpyDeviceToHost, st));
    SK_CU(cudaStreamSynchronize(st));
    if (step) *step = ds;
    return SK_OK;
}

sk_status mcmcmc_trace(sk_run* r, int32_t* slots, uint32_t mem) {
    if (!r || !slots) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    if (mem != SK_MEM_HOST && mem != SK_MEM_DEVICE) return fail(SK_ERR_INVALID_ARG, "bad mem");
    sk_status s = mcmcmc_wait(r, 0);
    if (s != SK_OK) return s;
    const size_t n = static_cast<size_t>(r->p.trace_chains) * r->p.trace_steps;
    if (n) {
        SK_CU(cudaMemcpyAsync(slots, r->dtrace, n * 4, cudaMemcpyDefault, r->inst->st));
        SK_CU(cudaStreamSynchronize(r->inst->st));
    }
    return SK_OK;
}

sk_status mcmcmc_counters(sk_run* r, uint64_t* flips, uint64_t* rows) {
    if (!r) return fail(SK_ERR_INVALID_ARG, "run is NULL");
    sk_status s = mcmcmc_wait(r, 0);
    if (s != SK_OK) return s;
    std::vector<unsigned long long> w(2 * static_cast<size_t>(r->chains));
    SK_CU(cudaMemcpyAsync(w.data(), r->dwork, w.size() * 8, cudaMemcpyDeviceToHost, r->inst->st));
    SK_CU(cudaStreamSynchronize(r->inst->st));
    uint64_t f = 0, q = 0;
    for (size_t c = 0; c < r->chains; ++c) {
        f += w[2 * c];
        q += w[2 * c + 1];
    }
    if (flips) *flips = f;
    if (rows) *rows = q;
    return SK_OK;
}

sk_status mcmcmc_recompute(sk_run* r, uint32_t mode, uint32_t terms, sk_recompute_stats* stats,
                           float* fields_out, uint32_t mem) {
    if (!r) return fail(SK_ERR_INVALID_ARG, "run is NULL");
    if (mode > 2) return fail(SK_ERR_INVALID_ARG, "unknown recompute mode %u", mode);
    if (terms > 3) return fail(SK_ERR_INVALID_ARG, "terms must be 0..3");
    if (mode == 2 && !fields_out) return fail(SK_ERR_INVALID_ARG, "fields_out is NULL");
    if (mem != SK_MEM_HOST && mem != SK_MEM_DEVICE) return fail(SK_ERR_INVALID_ARG, "bad mem");
    sk_status s = ensure_recompute(r, r->inst->st);
    if (s != SK_OK) return s;
    sk_instance* in = r->inst;
    cudaStream_t st = in->st;
    float* dout = nullptr;
    if (mode == 2 && (s = dalloc(&dout, static_cast<size_t>(r->chains) * in->Npad * 4)) != SK_OK) return s;
    SK_CU(cudaMemsetAsync(r->dstats + 3, 0, 3 * sizeof(unsigned long long), st));
    cudaError_t e = sk::launch_recompute(in->kind, r->ds, r->dh, dout, r->dSop, in->dJop, r->ddE, r->dstats + 3,
                                         r->derr, r->chains, in->Npad, terms ? terms : 3u, mode, in->scale, st,
                                         r->job.fault & sk::kFaultWithholdTile, r->sop_valid, r->dCnt);
    r->sop_valid = true;
    if (!stats && mode != 2) {  // enqueue only
        if (e != cudaSuccess) return fail(SK_ERR_CUDA, "recompute: %s", cudaGetErrorString(e));
        return SK_OK;
    }
    if (e == cudaSuccess && mode == 2)
        e = cudaMemcpy2DAsync(fields_out, in->N * 4, dout, in->Npad * 4, in->N * 4, r->chains, cudaMemcpyDefault,
                              st);
    unsigned long long h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, r->dstats + 3, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(SK_ERR_CUDA, "recompute: %s", cudaGetErrorString(e));
    if ((s = check_run_error(r)) != SK_OK) return s;
    if (stats) {
        double d0, d2;
        std::memcpy(&d0, &h[0], 8);
        std::memcpy(&d2, &h[2], 8);
        stats->max_field_drift = d0;
        stats->max_energy_drift = d2;
        stats->mismatches = h[1];
        stats->recomputes = 1;
    }
    return SK_OK;
}

sk_status mcmcmc_recompute_stats(sk_run* r, sk_recompute_stats* stats) {
    if (!r || !stats) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    sk_status s = mcmcmc_wait(r, 0);
    if (s != SK_OK) return s;
    unsigned long long h[3] = {0, 0, 0};
    if (r->dstats) {
        SK_CU(cudaMemcpyAsync(h, r->dstats, sizeof h, cudaMemcpyDeviceToHost, r->inst->st));
        SK_CU(cudaStreamSynchronize(r->inst->st));
    }
    double d0, d2;
    std::memcpy(&d0, &h[0], 8);
    std::memcpy(&d2, &h[2], 8);
    stats->max_field_drift = d0;
    stats->max_energy_drift = d2;
    stats->mismatches = h[1];
    stats->recomputes = r->n_recomputes;
    return SK_OK;
}

sk_status mcmcmc_free(sk_run* r) {
    if (!r) return fail(SK_ERR_INVALID_ARG, "run is NULL");
    if (const int n = r->batches.load() - (r->self ? 1 : 0); n > 0)
        return fail(SK_ERR_BUSY, "the run belongs to %d batch(es) that are not freed", n);
    cudaStreamSynchronize(r->inst->st);
    if (r->self) mcmcmc_batch_free(r->self);
    sk_instance* in = r->inst;
    free_run_buffers(r);
    delete r;
    in->runs--;
    return SK_OK;
}

namespace {

constexpr uint32_t kMaxClasses = 64;
// The autotuner tries the cluster-per-chain layout for classes of at most
// this many chains (where one chain's latency, not throughput, is at stake).
constexpr uint64_t kClusterTuneChains = 64;
// ... and the team layout for classes of at most this many chains (a few
// teams per SM at most).
constexpr uint64_t kTeamTuneChains = 1024;

uint32_t run_per_chain(const sk_run* r, bool staged = true) {
    return static_cast<uint32_t>((sk::warp_smem_bytes(r->inst->Npad, r->inst->kind, staged) + 127) / 128 * 128);
}
// Fewest lanes per chain a kernel covers for the run's K (NB up to 4 Philox
// blocks per lane).
uint32_t run_gmin(const sk_run* r) {
    for (uint32_t g = 4; g < 32; g <<= 1)
        if (sk::blocks_per_lane(r->p.rule, r->p.K, g)) return g;
    return 32;
}
// Runs share a launch class when their kernels agree for every G: same
// coupling type, rule, node-weighted records or not, Philox blocks of sites
// (as a power of two) and shared-memory bucket.
bool run_nw(const sk_run* r) { return r->p.node_weighted && r->p.record_every && r->p.max_records; }
uint64_t class_key(const sk_run* r) {
    uint32_t b = 128;
    if (r->p.graph) {  // graph runs: by coupling kind, graph type and node count
        const uint32_t pc = static_cast<uint32_t>(sk::graph_smem_bytes(r->inst->Npad, r->job.V, r->p.graph));
        while (b < pc) b <<= 1;
        return (static_cast<uint64_t>(r->inst->kind) << 62) | (1ull << 59) |
               (static_cast<uint64_t>(r->p.graph) << 56) | (static_cast<uint64_t>(r->job.V) << 32) | b;
    }
    const uint32_t pc = run_per_chain(r);
    while (b < pc) b <<= 1;
    const uint64_t kb = sk::site_blocks_pow2(r->p.rule, r->p.K);
    return (static_cast<uint64_t>(r->inst->kind) << 62) | (static_cast<uint64_t>(r->p.rule) << 61) |
           (static_cast<uint64_t>(run_nw(r)) << 60) | (kb << 32) | b;
}
// Most warps per CTA for G lanes per chain: chains of a pair share a CTA,
// so with whole-warp chains W is even.
uint32_t fit_warps(uint32_t per_chain, uint32_t G) {
    const uint32_t spw = 32 / G;
    uint32_t w = static_cast<uint32_t>(std::min<size_t>(32, kSmemBudget / (static_cast<size_t>(per_chain) * spw)));
    if (G == 32) w &= ~1u;
    return w;
}

// The cluster-per-chain layout for the star class of runs `idx` with C CTAs
// per cluster and W chains per cluster (0: 2, or 1 when every run has one
// chain; W = 1 only then, so that overlap pairs share a cluster).  Returns
// false, with c untouched, when the class cannot take it: node-weighted
// records, K beyond 2 Philox blocks per lane, a slice that is not whole
// 16-byte units or shared memory that does not fit.
bool plan_cluster_class(const sk_batch* b, const std::vector<uint32_t>& idx, uint32_t C, uint32_t W,
                        sk_batch::Class& c) {
    const sk_run* r0 = b->runs[idx[0]];
    if (run_nw(r0) || r0->p.graph) return false;
    bool single = true;
    uint32_t nb = 0;
    size_t jbytes = 0, pc = 0;
    for (uint32_t i : idx) {
        const sk_run* r = b->runs[i];
        if (r->chains > 1) single = false;
        const uint32_t n = sk::blocks_per_lane(r->p.rule, r->p.K, 32);
        if (n == 0 || n > 2) return false;
        nb = std::max(nb, n);
        if (!sk::cluster_shape_ok(r->inst->kind, r->inst->Npad, C)) return false;
        jbytes = std::max(jbytes, sk::cluster_slice_bytes(r->inst->kind, r->inst->N, r->inst->Npad, C));
    }
    for (uint32_t i : idx) pc = std::max(pc, sk::cluster_chain_bytes(r0->p.rule, nb, b->runs[i]->inst->Npad, C));
    if (W == 0) W = single ? 1u : 2u;
    if (W == 1 && !single) W = 2;
    if (W != 1 && W != 2 && W != 4 && W != sk::kClusterMaxChains) return false;
    if (jbytes + W * pc > kSmemBudget) return false;
    c.cluster = C;
    c.W = W;
    c.G = 32 * C;
    c.gmin = 32;
    c.stage = 0;
    c.per_chain = static_cast<uint32_t>(pc);
    c.jbytes = static_cast<uint32_t>(jbytes);
    c.kind = r0->inst->kind;
    c.rule = r0->p.rule;
    c.nb = nb;
    c.cls = 1024 + static_cast<int>(c.kind) * 2 + static_cast<int>(c.rule);
    return true;
}

// The team layout for the star class of runs `idx`: T warps per chain, W
// chains per CTA (0: 2, or 1 when every run has one chain; W = 1 only then, so
// that overlap pairs share a CTA).  Returns false for classes it cannot take:
// graph runs, node-weighted records, MCMCMC with K > 32 T, or more shared
// memory than a CTA has.
bool plan_team_class(const sk_batch* b, const std::vector<uint32_t>& idx, uint32_t T, uint32_t W,
                     sk_batch::Class& c) {
    const sk_run* r0 = b->runs[idx[0]];
    if (run_nw(r0) || r0->p.graph) return false;
    bool single = true;
    size_t pc = 0;
    for (uint32_t i : idx) {
        const sk_run* r = b->runs[i];
        if (!sk::team_ok(r->p.rule, r->p.K, T)) return false;
        single = single && r->chains == 1;
        pc = std::max(pc, sk::team_chain_bytes(r->inst->Npad, T));
    }
    if (W == 0) W = single ? 1u : 2u;
    if ((W != 1 && W != 2) || (W == 1 && !single)) return false;
    if (W * pc > kSmemBudget) return false;
    c.team = T;
    c.W = W;
    c.G = 32 * T;
    c.gmin = 32;
    c.stage = 0;
    c.per_chain = static_cast<uint32_t>(pc);
    c.kind = r0->inst->kind;
    c.rule = r0->p.rule;
    c.nb = 0;
    c.cls = 4096 + static_cast<int>(c.kind) * 2 + static_cast<int>(c.rule);
    return true;
}

// Work items of the batch, grouped by launch class, each class with its own
// lanes per chain and warps per CTA: the autotuned or forced values, else
// the fewest lanes K allows (whole-warp chains for runs of few chains, where
// latency matters) and as many warps as fit.  Uploads them.
sk_status ensure_side_streams(sk_batch* b);
void free_side_streams(sk_batch* b);

// Runs the fused launch takes: star runs without node-weighted records.
bool fused_eligible(const sk_run* r) { return !r->p.graph && !run_nw(r); }

sk_status plan_batch(sk_batch* b) {
    std::map<uint64_t, std::vector<uint32_t>> groups;  // key -> run indices (in order)
    std::vector<uint32_t> fidx;                        // runs of the fused launch
    const uint32_t n = static_cast<uint32_t>(b->runs.size());
    for (uint32_t i = 0; i < n; ++i) {
        if (b->fused_W && fused_eligible(b->runs[i]))
            fidx.push_back(i);
        else
            groups[class_key(b->runs[i])].push_back(i);
    }
    if (groups.size() + (fidx.empty() ? 0 : 1) > kMaxClasses)
        return fail(SK_ERR_INVALID_ARG, "too many launch classes in one batch");
    std::vector<WorkItem> items;
    std::vector<sk_batch::Class> classes;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint32_t grid = 0;
    for (auto& g : groups) {
        sk_batch::Class c{};
        c.key = g.first;
        const sk_run* r0 = b->runs[g.second[0]];
        c.gmin = run_gmin(r0);
        for (uint32_t i : g.second) {
            c.per_chain_staged = std::max(c.per_chain_staged, run_per_chain(b->runs[i], true));
            c.per_chain_direct = std::max(c.per_chain_direct, run_per_chain(b->runs[i], false));
        }
        if ((c.key >> 59) & 1u) {  // graph runs: a team of nw warps per chain, an even number of chains per CTA
            c.graph = r0->p.graph;
            c.gmin = 32;
            c.stage = 0;
            c.per_chain = 0;
            for (uint32_t i : g.second)
                c.per_chain = std::max(c.per_chain, static_cast<uint32_t>(sk::graph_smem_bytes(
                                                        b->runs[i]->inst->Npad, b->runs[i]->job.V, c.graph)));
            const uint32_t fitc = static_cast<uint32_t>(std::min<size_t>(32, kSmemBudget / c.per_chain)) & ~1u;
            if (fitc < 2) return fail(SK_ERR_INVALID_ARG, "graph too large: %u bytes of shared memory per chain", c.per_chain);
            auto tg = b->tuned.find(c.key);
            if (tg != b->tuned.end()) {
                c.nw = tg->second >> 16;
                c.W = tg->second & 0xFFu;
            } else {
                c.nw = b->G_override >= 64 ? std::min<uint32_t>(16, b->G_override / 32) : 1u;
                uint32_t chains = c.nw == 1 ? fitc : std::min<uint32_t>(fitc, 32 / c.nw) & ~1u;
                if (c.nw > 1) chains = std::min<uint32_t>(chains, 14);
                if (b->W_override) chains = std::max<uint32_t>(2, std::min(chains, (b->W_override / c.nw) & ~1u));
                if (chains < 2) return fail(SK_ERR_INVALID_ARG, "graph: %u warps per chain leave no room for two chains", c.nw);
                c.W = chains * c.nw;
            }
            if (!sk::graph_team_ok(c.W, c.nw)) return fail(SK_ERR_INVALID_ARG, "graph layout %u warps, %u per chain", c.W, c.nw);
            c.G = 32 * c.nw;
            c.cls = 512 + static_cast<int>(r0->inst->kind) * 4 + static_cast<int>(c.graph);
            int occg = sk::graph_kernel_occupancy(r0->inst->kind, c.graph, c.W, c.nw, c.per_chain);
            while (occg <= 0 && tg == b->tuned.end() && c.W > 2 * c.nw) {
                c.W -= 2 * c.nw;
                occg = sk::graph_kernel_occupancy(r0->inst->kind, c.graph, c.W, c.nw, c.per_chain);
            }
            if (occg <= 0) return fail(SK_ERR_CUDA, "graph kernel cannot be resident with %u warps", c.W);
            c.first_item = static_cast<uint32_t>(items.size());
            const uint32_t cpi = c.W / c.nw;  // chains per item
            for (uint32_t i : g.second) {
                const sk_run* r = b->runs[i];
                for (uint32_t ch = 0; ch < r->chains; ch += cpi)
                    items.push_back(WorkItem{i, ch, std::min(cpi, r->chains - ch), 0});
            }
            c.n_items = static_cast<uint32_t>(items.size()) - c.first_item;
            c.grid = std::min<uint32_t>(c.n_items, static_cast<uint32_t>(occg * sms));
            grid = std::max(grid, c.grid);
            classes.push_back(c);
            continue;
        }
        {  // the cluster-per-chain layout: autotuned, or forced by mcmcmc_batch_set_cluster
            auto tc = b->tuned.find(c.key);
            const bool tuned_cl = tc != b->tuned.end() && (tc->second >> 24) != 0;
            const uint32_t C = tuned_cl ? (tc->second >> 24) : (tc == b->tuned.end() ? b->C_override : 0u);
            const uint32_t Wc = tuned_cl ? (tc->second & 0xFFu) : b->CW_override;
            if (C && plan_cluster_class(b, g.second, C, Wc, c)) {
                const int occ = sk::cluster_occupancy(c.kind, c.rule, c.nb, C, c.W, c.jbytes, c.per_chain);
                if (occ <= 0)
                    return fail(SK_ERR_CUDA, "no cluster of %u CTAs with %u bytes of shared memory can be resident", C,
                                c.jbytes + c.W * c.per_chain);
                c.first_item = static_cast<uint32_t>(items.size());
                for (uint32_t i : g.second) {
                    const sk_run* r = b->runs[i];
                    for (uint32_t ch = 0; ch < r->chains; ch += c.W)
                        items.push_back(WorkItem{i, ch, std::min(c.W, r->chains - ch), 0});
                }
                c.n_items = static_cast<uint32_t>(items.size()) - c.first_item;
                c.grid = std::min<uint32_t>(c.n_items, static_cast<uint32_t>(occ)) * C;  // CTAs
                grid = std::max(grid, c.grid);
                classes.push_back(c);
                continue;
            }
            if (tuned_cl) return fail(SK_ERR_INVALID_ARG, "launch class cannot take %u-CTA clusters", C);
        }
        {  // the team layout: autotuned (64 or 128 lanes in the tuned code), or
           // forced by mcmcmc_batch_set_layout with 64 or more lanes
            auto tt = b->tuned.find(c.key);
            const bool tuned_t = tt != b->tuned.end() && (tt->second >> 24) == 0 && ((tt->second >> 8) & 0xFFu) >= 64;
            const uint32_t lanes = tuned_t ? ((tt->second >> 8) & 0xFFu) : (tt == b->tuned.end() ? b->G_override : 0u);
            if (lanes >= 64 &&
                plan_team_class(b, g.second, lanes >= 128 ? 4u : 2u, tuned_t ? (tt->second & 0xFFu) : 0u, c)) {
                const int occ = sk::team_occupancy(c.kind, c.rule, c.team, c.W, c.per_chain);
                if (occ <= 0)
                    return fail(SK_ERR_CUDA, "no team CTA of %u warps with %u bytes of shared memory can be resident",
                                c.team * c.W, c.W * c.per_chain);
                c.first_item = static_cast<uint32_t>(items.size());
                for (uint32_t i : g.second) {
                    const sk_run* r = b->runs[i];
                    for (uint32_t ch = 0; ch < r->chains; ch += c.W)
                        items.push_back(WorkItem{i, ch, std::min(c.W, r->chains - ch), 0});
                }
                c.n_items = static_cast<uint32_t>(items.size()) - c.first_item;
                c.grid = std::min<uint32_t>(c.n_items, static_cast<uint32_t>(occ * sms));
                grid = std::max(grid, c.grid);
                classes.push_back(c);
                continue;
            }
            if (tuned_t) return fail(SK_ERR_INVALID_ARG, "launch class cannot take the %u-lane team layout", lanes);
        }
        const bool nw = ((c.key >> 60) & 1u) != 0;  // node-weighted records: rows through L1 only
        bool single = true;  // every run of the class has one chain: no overlap pairs
        for (uint32_t i : g.second) single = single && b->runs[i]->chains == 1;
        auto t = b->tuned.find(c.key);
        if (t != b->tuned.end()) {
            c.stage = (t->second >> 16) & 0xFFu;
            c.G = (t->second >> 8) & 0xFFu;
            c.W = t->second & 0xFFu;
            c.per_chain = c.stage ? c.per_chain_staged : c.per_chain_direct;
        } else {
            // untuned default: rows through L1 and whole-warp chains, the
            // layout the autotuner picks for most classes; forced lanes that
            // leave no room for one warp's chains are raised until they fit
            c.stage = (b->S_override == 1 && !nw) ? 1u : 0u;
            c.per_chain = c.stage ? c.per_chain_staged : c.per_chain_direct;
            c.G = b->G_override ? std::min(32u, std::max(b->G_override, c.gmin)) : 32u;
            uint32_t fit = fit_warps(c.per_chain, c.G);
            while (c.G < 32 && fit < 1) fit = fit_warps(c.per_chain, c.G <<= 1);
            if (c.G == 32 && single && fit < 1 && kSmemBudget >= c.per_chain) fit = 1;
            if (b->W_override) {
                c.W = std::min(b->W_override, fit);
                // whole-warp chains come in pairs (overlap q) unless every run has one chain
                if (c.G == 32 && (c.W & 1u) && !single) c.W = std::min(c.W + 1u, fit);
            } else {
                // as many warps as the class's chains need when spread over the
                // SMs, at most as many as fit: a class of few chains gets small
                // CTAs and with them the 128-register step kernel (8 row loads of
                // the field update in flight), which is what a lone chain's
                // latency wants; whole-warp chains keep an even count so that
                // overlap pairs share a CTA (one warp where every run has one chain)
                uint64_t total = 0;
                for (uint32_t i : g.second) total += b->runs[i]->chains;
                const uint32_t spw = 32u / c.G;
                const uint64_t per_sm = (total + static_cast<uint64_t>(sms) - 1) / static_cast<uint64_t>(sms);
                uint32_t need = static_cast<uint32_t>(std::min<uint64_t>(32, (per_sm + spw - 1) / spw));
                if (c.G == 32) need = single ? std::max(1u, need) : std::max(2u, (need + 1u) & ~1u);
                c.W = std::max(1u, std::min(fit, need));
            }
        }
        if (c.W < 1 || (c.G == 32 && c.W < 2 && !single))
            return fail(SK_ERR_INVALID_ARG, "N too large: %u bytes of shared memory per chain", c.per_chain);
        c.cls = sk::step_class(r0->inst->kind, r0->p.rule, r0->p.K, c.G, nw ? 2u : c.stage, r0->inst->Npad);
        if (c.cls < 0) return fail(SK_ERR_INVALID_ARG, "no step kernel for K = %u with %u lanes per chain", r0->p.K, c.G);
        int occ = sk::step_kernel_occupancy(c.cls, c.W, c.per_chain);
        while (occ <= 0 && t == b->tuned.end() && c.W > (c.G == 32 ? 2u : 1u)) {  // default choice: step down
            c.W -= c.G == 32 ? 2u : 1u;
            occ = sk::step_kernel_occupancy(c.cls, c.W, c.per_chain);
        }
        if (occ <= 0)
            return fail(SK_ERR_CUDA, "step kernel cannot be resident with %u warps of %u-lane chains", c.W, c.G);
        const uint32_t cpc = c.W * (32 / c.G);  // chains per CTA
        c.first_item = static_cast<uint32_t>(items.size());
        for (uint32_t i : g.second) {
            const sk_run* r = b->runs[i];
            for (uint32_t ch = 0; ch < r->chains; ch += cpc)
                items.push_back(WorkItem{i, ch, std::min(cpc, r->chains - ch), 0});
        }
        c.n_items = static_cast<uint32_t>(items.size()) - c.first_item;
        c.grid = std::min<uint32_t>(c.n_items, static_cast<uint32_t>(occ * sms));
        grid = std::max(grid, c.grid);
        classes.push_back(c);
    }
    if (!fidx.empty()) {
        // one launch of W-warp CTAs for all of them: whole-warp chains, rows
        // through L1.  Each CTA gets the share of an SM's shared memory that
        // its register budget (W warps x 32 lanes x 128 registers) leaves it,
        // at least room for two chains of the largest run; an item holds as
        // many chains of one run as fit, up to W, an even number for runs of
        // several chains (overlap pairs share a CTA).
        sk_batch::Class c{};
        c.fused = true;
        c.key = ~0ull;
        c.W = b->fused_W;
        c.G = 32;
        c.gmin = 32;
        c.cls = 2048;
        uint32_t pcmax = 0;
        bool multi = false;
        for (uint32_t i : fidx) {
            pcmax = std::max(pcmax, run_per_chain(b->runs[i], false));
            multi = multi || b->runs[i]->chains > 1;
        }
        const uint32_t ctas = std::max<uint32_t>(1, 65536u / (32u * c.W * 128u));
        // an SM's 228 KB less, per CTA, the kilobyte the hardware reserves and
        // the kernel's static arrays (under a kilobyte)
        size_t S = std::min<size_t>(kSmemBudget, (228u * 1024u) / ctas - 2048u);
        S = std::max<size_t>(S, std::min<size_t>(kSmemBudget, (multi ? 2u : 1u) * pcmax));
        if (pcmax > S || (multi && 2u * pcmax > S))
            return fail(SK_ERR_INVALID_ARG, "N too large for the fused launch: %u bytes of shared memory per chain",
                        pcmax);
        c.fsmem = static_cast<uint32_t>(S);
        c.per_chain = pcmax;
        c.first_item = static_cast<uint32_t>(items.size());
        for (uint32_t i : fidx) {
            const sk_run* r = b->runs[i];
            const uint32_t pc = run_per_chain(r, false);
            uint32_t cpi = std::min<uint32_t>(c.W, static_cast<uint32_t>(S / pc));
            if (r->chains > 1) cpi &= ~1u;
            const uint32_t v = sk::fused_variant(r->inst->kind, r->p.rule, r->p.K, r->inst->Npad);
            for (uint32_t ch = 0; ch < r->chains; ch += cpi)
                items.push_back(WorkItem{i, ch, std::min(cpi, r->chains - ch), (v << 24) | pc});
        }
        // largest items first (work per step ~ chains x (Npad + 4 K)), so the
        // launch does not end on a few long items
        auto cost = [&](const WorkItem& w) {
            const sk_run* r = b->runs[w.job];
            return static_cast<uint64_t>(w.nchains) * (r->inst->Npad + 4u * r->p.K);
        };
        std::stable_sort(items.begin() + c.first_item, items.end(),
                         [&](const WorkItem& x, const WorkItem& y) { return cost(x) > cost(y); });
        c.n_items = static_cast<uint32_t>(items.size()) - c.first_item;
        const int occ = sk::fused_occupancy(c.W, c.fsmem);
        if (occ <= 0) return fail(SK_ERR_CUDA, "fused kernel cannot be resident with %u warps", c.W);
        c.grid = std::min<uint32_t>(c.n_items, static_cast<uint32_t>(occ * sms));
        grid = std::max(grid, c.grid);
        classes.push_back(c);
    }
    WorkItem* d = nullptr;
    sk_status s = dalloc(&d, items.size() * sizeof(WorkItem));
    if (s != SK_OK) return s;
    cudaError_t e = cudaMemcpy(d, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return fail(SK_ERR_CUDA, "batch upload: %s", cudaGetErrorString(e));
    }
    cudaStreamSynchronize(b->st);  // no launch of the batch may still read the old items
    cudaFree(b->ditems);
    b->ditems = d;
    b->classes = classes;
    if (sk_status s2 = ensure_side_streams(b); s2 != SK_OK) return s2;
    b->n_items = static_cast<uint32_t>(items.size());
    b->grid = grid;
    if (b->graph) {  // the captured launches used the old plan
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_steps = 0;
    }
    return SK_OK;
}

}  // namespace

sk_status mcmcmc_batch_create(sk_run* const* runs, uint32_t n, uint32_t W, sk_batch** out) {
    if (!runs || !out || n == 0) return fail(SK_ERR_INVALID_ARG, "empty batch");
    *out = nullptr;
    if (W > 32) return fail(SK_ERR_INVALID_ARG, "warps_per_cta = %u must be at most 32", W);
    cudaStream_t st = runs[0]->inst->st;
    for (uint32_t i = 0; i < n; ++i) {
        if (!runs[i]) return fail(SK_ERR_INVALID_ARG, "run %u is NULL", i);
        if (runs[i]->inst->st != st) return fail(SK_ERR_INVALID_ARG, "runs of a batch must share a stream");
    }
    sk_batch* b = new sk_batch();
    b->runs.assign(runs, runs + n);
    b->W_override = W;
    b->st = st;
    std::vector<JobDev> jobs(n);
    for (uint32_t i = 0; i < n; ++i) jobs[i] = runs[i]->job;
    sk_status s = dalloc(&b->djobs, n * sizeof(JobDev));
    if (s == SK_OK) s = dalloc(&b->dqueue, kMaxClasses * sizeof(uint32_t));
    if (s == SK_OK) {
        cudaError_t e = cudaMemcpy(b->djobs, jobs.data(), n * sizeof(JobDev), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) s = fail(SK_ERR_CUDA, "batch upload: %s", cudaGetErrorString(e));
    }
    if (s == SK_OK) s = plan_batch(b);
    if (s != SK_OK) {
        free_side_streams(b);
        cudaFree(b->djobs);
        cudaFree(b->ditems);
        cudaFree(b->dqueue);
        delete b;
        return s;
    }
    for (sk_run* r : b->runs) r->batches++;
    *out = b;
    return SK_OK;
}

sk_status mcmcmc_batch_set_layout(sk_batch* b, uint32_t lanes, uint32_t staging) {
    if (!b) return fail(SK_ERR_INVALID_ARG, "batch is NULL");
    if (lanes && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32 && lanes != 64 && lanes != 128 &&
        lanes != 256 && lanes != 512)
        return fail(SK_ERR_INVALID_ARG, "lanes per chain must be 0, 4, 8, 16, 32, 64, 128, 256 or 512");
    if (staging > 2) return fail(SK_ERR_INVALID_ARG, "staging must be 0, 1 or 2");
    b->G_override = lanes;
    b->S_override = staging;
    b->C_override = 0;
    b->CW_override = 0;
    b->fused_W = 0;
    b->tuned.clear();
    return plan_batch(b);
}

sk_status mcmcmc_batch_set_fused(sk_batch* b, uint32_t warps_per_cta) {
    if (!b) return fail(SK_ERR_INVALID_ARG, "batch is NULL");
    const uint32_t W = warps_per_cta;
    if (W != 0 && W != 2 && W != 4 && W != 8 && W != 16)
        return fail(SK_ERR_INVALID_ARG, "warps per CTA of the fused launch must be 0, 2, 4, 8 or 16");
    const uint32_t w0 = b->fused_W, c0 = b->C_override, cw0 = b->CW_override;
    const std::map<uint64_t, uint32_t> t0 = b->tuned;
    b->fused_W = W;
    if (W) {
        b->C_override = 0;
        b->CW_override = 0;
    }
    b->tuned.clear();
    const sk_status s = plan_batch(b);
    if (s != SK_OK) {  // keep the previous plan
        b->fused_W = w0;
        b->C_override = c0;
        b->CW_override = cw0;
        b->tuned = t0;
        plan_batch(b);
    }
    return s;
}

sk_status mcmcmc_batch_set_cluster(sk_batch* b, uint32_t ctas, uint32_t chains) {
    if (!b) return fail(SK_ERR_INVALID_ARG, "batch is NULL");
    if (ctas != 0 && ctas != 1 && ctas != 2 && ctas != 4 && ctas != 8 && ctas != 16)
        return fail(SK_ERR_INVALID_ARG, "CTAs per cluster must be 0, 1, 2, 4, 8 or 16");
    if (chains != 0 && chains != 1 && chains != 2 && chains != 4 && chains != sk::kClusterMaxChains)
        return fail(SK_ERR_INVALID_ARG, "chains per cluster must be 0, 1, 2, 4 or 8");
    const uint32_t c0 = b->C_override, w0 = b->CW_override, f0 = b->fused_W;
    const std::map<uint64_t, uint32_t> t0 = b->tuned;
    b->C_override = ctas;
    b->CW_override = chains;
    if (ctas) b->fused_W = 0;
    b->tuned.clear();
    const sk_status s = plan_batch(b);
    if (s != SK_OK) {  // keep the previous plan
        b->C_override = c0;
        b->CW_override = w0;
        b->fused_W = f0;
        b->tuned = t0;
        plan_batch(b);
    }
    return s;
}

namespace {
// Launches `steps` steps of the batch's classes (only class `only` if >= 0);
// the step counters are bumped after the last launched class.
// Creates the side streams and events of a batch with several classes
// (before any capture: creation is not a stream operation to record).
sk_status ensure_side_streams(sk_batch* b) {
    if (b->classes.size() < 2 || b->ev_fork) return SK_OK;
    cudaError_t e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    for (uint32_t i = 0; i < sk_batch::kSide && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return fail(SK_ERR_CUDA, "side streams: %s", cudaGetErrorString(e));
    return SK_OK;
}

void free_side_streams(sk_batch* b) {
    for (uint32_t i = 0; i < sk_batch::kSide; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
        b->side[i] = nullptr;
        b->ev_join[i] = nullptr;
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    b->ev_fork = nullptr;
}

// Launches `steps` steps of every class (or of class `only`, on the batch's
// stream).  Several classes: class k runs on side stream k mod kSide after
// the work queued so far on the batch's stream, the batch's stream waits for
// all of them, then the runs' step counters advance.  The classes touch
// disjoint runs and have their own work counters, and no kernel waits for
// another, so any overlap of their CTAs is safe.
sk_status launch_segment(sk_batch* b, uint64_t steps, int only = -1) {
    const size_t nc = b->classes.size();
    const bool fork = only < 0 && nc > 1 && b->ev_fork;
    const uint32_t nside = fork ? static_cast<uint32_t>(std::min<size_t>(nc, sk_batch::kSide)) : 0u;
    if (fork) {
        SK_CU(cudaEventRecord(b->ev_fork, b->st));
        for (uint32_t i = 0; i < nside; ++i) SK_CU(cudaStreamWaitEvent(b->side[i], b->ev_fork, 0));
    }
    for (size_t k = 0; k < nc; ++k) {
        if (only >= 0 && static_cast<size_t>(only) != k) continue;
        const sk_batch::Class& c = b->classes[k];
        const bool last = !fork && (only >= 0 || k + 1 == nc);
        cudaStream_t cs = fork ? b->side[k % nside] : b->st;
        cudaError_t e =
            c.fused ? sk::launch_fused(b->djobs, b->ditems + c.first_item, c.n_items, b->dqueue + k, steps, c.W,
                                       c.fsmem, c.grid, static_cast<uint32_t>(b->runs.size()), last, cs)
            : c.cluster ? sk::launch_cluster(b->djobs, b->ditems + c.first_item, c.n_items, b->dqueue + k, steps, c.kind,
                                           c.rule, c.nb, c.cluster, c.W, c.jbytes, c.per_chain, c.grid / c.cluster,
                                           static_cast<uint32_t>(b->runs.size()), last, cs)
            : c.team  ? sk::launch_team(b->djobs, b->ditems + c.first_item, c.n_items, b->dqueue + k, steps, c.kind,
                                        c.rule, c.team, c.W, c.per_chain, c.grid,
                                        static_cast<uint32_t>(b->runs.size()), last, cs)
            : c.graph ? sk::launch_graph(b->djobs, b->ditems + c.first_item, c.n_items, b->dqueue + k, steps, c.W,
                                       c.nw, c.per_chain, c.grid, static_cast<uint32_t>((c.cls - 512) / 4), c.graph,
                                       static_cast<uint32_t>(b->runs.size()), last, cs)
                    : sk::launch_step(b->djobs, b->ditems + c.first_item, c.n_items, b->dqueue + k, steps, c.W,
                                      c.per_chain, c.grid, c.cls, static_cast<uint32_t>(b->runs.size()), last, cs);
        if (e != cudaSuccess) return fail(SK_ERR_CUDA, "step launch: %s", cudaGetErrorString(e));
    }
    if (fork) {
        for (uint32_t i = 0; i < nside; ++i) {
            SK_CU(cudaEventRecord(b->ev_join[i], b->side[i]));
            SK_CU(cudaStreamWaitEvent(b->st, b->ev_join[i], 0));
        }
        const cudaError_t e = sk::launch_bump_steps(b->djobs, static_cast<uint32_t>(b->runs.size()), steps, b->st);
        if (e != cudaSuccess) return fail(SK_ERR_CUDA, "step counters: %s", cudaGetErrorString(e));
    }
    for (sk_run* r : b->runs) {
        r->step = std::min<uint64_t>(r->step + steps, r->job.step_limit);
        // the step and cluster kernels rewrite the operands of runs that keep
        // them; the graph kernel does not
        r->sop_valid = r->job.s_op != nullptr && !r->p.graph;
    }
    return SK_OK;
}
}  // namespace

namespace {

// Recompute period shared by the batch's recomputing runs (0 if none) and
// the run whose phase defines the segments; errors if they disagree.
sk_status recompute_period(const sk_batch* b, uint32_t* M, const sk_run** lead) {
    *M = 0;
    *lead = nullptr;
    for (const sk_run* r : b->runs) {
        if (!r->p.recompute_every) continue;
        if (!*lead) {
            *lead = r;
            *M = r->p.recompute_every;
        } else if (r->p.recompute_every != *M || r->step % *M != (*lead)->step % *M) {
            return fail(SK_ERR_INVALID_ARG, "runs of a batch that recompute must share recompute_every and phase");
        }
    }
    return SK_OK;
}

// Enqueues `steps` steps of every run (segments ending on recompute points).
sk_status enqueue_advance(sk_batch* b, uint64_t steps) {
    uint32_t M;
    const sk_run* lead;
    sk_status s = recompute_period(b, &M, &lead);
    if (s != SK_OK) return s;
    if (!M) return launch_segment(b, steps);
    while (steps) {
        const uint64_t seg = std::min<uint64_t>(steps, M - lead->step % M);
        if ((s = launch_segment(b, seg)) != SK_OK) return s;
        steps -= seg;
        if (lead->step % M == 0)
            for (sk_run* r : b->runs)
                if (r->p.recompute_every && (s = periodic_recompute(r)) != SK_OK) return s;
    }
    return SK_OK;
}

}  // namespace

sk_status mcmcmc_batch_advance(sk_batch* b, uint64_t steps) {
    if (!b) return fail(SK_ERR_INVALID_ARG, "batch is NULL");
    if (steps == 0) return SK_OK;
    for (sk_run* r : b->runs)
        if (r->step + steps > 0xFFFFFFFFull) return fail(SK_ERR_INVALID_ARG, "a run would pass 2^32 steps");
    return enqueue_advance(b, steps);
}

sk_status mcmcmc_batch_capture(sk_batch* b, uint64_t steps) {
    if (!b || steps == 0) return fail(SK_ERR_INVALID_ARG, "NULL batch or zero steps");
    if (!b->st) return fail(SK_ERR_INVALID_ARG, "graph capture needs a stream other than the legacy default stream");
    uint32_t M;
    const sk_run* lead;
    sk_status s = recompute_period(b, &M, &lead);
    if (s != SK_OK) return s;
    if (M && (steps % M || lead->step % M))
        return fail(SK_ERR_INVALID_ARG, "with recompute_every = %u, capture %u-aligned multiples of it", M, M);
    for (sk_run* r : b->runs)  // allocations happen before the capture
        if (r->p.recompute_every && (s = ensure_recompute(r, r->inst->st)) != SK_OK) return s;
    SK_CU(cudaStreamSynchronize(b->st));
    std::vector<uint64_t> mirror;
    std::vector<uint64_t> nrec;
    for (sk_run* r : b->runs) {
        mirror.push_back(r->step);
        nrec.push_back(r->n_recomputes);
    }
    SK_CU(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    s = enqueue_advance(b, steps);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->st, &g);
    for (size_t i = 0; i < b->runs.size(); ++i) {  // nothing ran yet
        b->runs[i]->step = mirror[i];
        b->runs[i]->n_recomputes = nrec[i];
    }
    if (s != SK_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return fail(SK_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
    cudaGraphExec_t x = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return fail(SK_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e2));
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = x;
    b->graph_steps = steps;
    return SK_OK;
}

sk_status mcmcmc_batch_replay(sk_batch* b, uint32_t times) {
    if (!b || !b->graph) return fail(SK_ERR_INVALID_ARG, "no captured graph");
    for (sk_run* r : b->runs)
        if (r->step + b->graph_steps * times > 0xFFFFFFFFull)
            return fail(SK_ERR_INVALID_ARG, "a run would pass 2^32 steps");
    for (uint32_t k = 0; k < times; ++k) {
        SK_CU(cudaGraphLaunch(b->graph, b->st));
        for (sk_run* r : b->runs) {
            if (r->p.recompute_every) r->n_recomputes += b->graph_steps / r->p.recompute_every;
            r->step = std::min<uint64_t>(r->step + b->graph_steps, r->job.step_limit);
        }
    }
    return SK_OK;
}

sk_status mcmcmc_batch_autotune(sk_batch* b, uint32_t trial_steps, uint32_t* out_W) {
    if (!b || trial_steps == 0) return fail(SK_ERR_INVALID_ARG, "NULL batch or zero trial steps");
    // back up every run's mutable state; trials run with records and traces off
    struct Backup {
        void* s;
        void* h;
        void* acc;
        void* work;
        void* step;
    };
    std::vector<Backup> bk;
    sk_status s = SK_OK;
    SK_CU(cudaStreamSynchronize(b->st));
    for (sk_run* r : b->runs) {
        Backup x{};
        const size_t C = r->chains, np = r->inst->Npad;
        if (s == SK_OK) s = dalloc(&x.s, C * np);
        if (s == SK_OK) s = dalloc(&x.h, C * np * 4);
        if (s == SK_OK) s = dalloc(&x.acc, C * 4);
        if (s == SK_OK) s = dalloc(&x.work, C * 16);
        if (s == SK_OK) s = dalloc(&x.step, 8);
        bk.push_back(x);
        if (s != SK_OK) break;
        cudaMemcpyAsync(x.s, r->ds, C * np, cudaMemcpyDeviceToDevice, b->st);
        cudaMemcpyAsync(x.h, r->dh, C * np * 4, cudaMemcpyDeviceToDevice, b->st);
        cudaMemcpyAsync(x.acc, r->dacc, C * 4, cudaMemcpyDeviceToDevice, b->st);
        cudaMemcpyAsync(x.work, r->dwork, C * 16, cudaMemcpyDeviceToDevice, b->st);
        cudaMemcpyAsync(x.step, r->dstep, 8, cudaMemcpyDeviceToDevice, b->st);
    }
    auto restore = [&]() {
        for (size_t i = 0; i < b->runs.size() && i < bk.size(); ++i) {
            sk_run* r = b->runs[i];
            const size_t C = r->chains, np = r->inst->Npad;
            cudaMemcpyAsync(r->ds, bk[i].s, C * np, cudaMemcpyDeviceToDevice, b->st);
            cudaMemcpyAsync(r->dh, bk[i].h, C * np * 4, cudaMemcpyDeviceToDevice, b->st);
            cudaMemcpyAsync(r->dacc, bk[i].acc, C * 4, cudaMemcpyDeviceToDevice, b->st);
            cudaMemcpyAsync(r->dwork, bk[i].work, C * 16, cudaMemcpyDeviceToDevice, b->st);
            cudaMemcpyAsync(r->dstep, bk[i].step, 8, cudaMemcpyDeviceToDevice, b->st);
        }
    };
    std::vector<JobDev> quiet;
    for (sk_run* r : b->runs) {
        JobDev j = r->job;
        j.rec_capacity = 0;
        j.trace_chains = 0;
        quiet.push_back(j);
    }
    const std::map<uint64_t, uint32_t> tuned0 = b->tuned;
    const uint32_t fused_before = b->fused_W;
    std::vector<uint64_t> mirror;
    for (sk_run* r : b->runs) mirror.push_back(r->step);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s == SK_OK) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaMemcpy(b->djobs, quiet.data(), quiet.size() * sizeof(JobDev), cudaMemcpyHostToDevice);
        // each launch class is tuned on its own (its launches do not interact),
        // with the star runs in their per-class launches
        const uint32_t fused0 = b->fused_W;
        if (fused0) {
            b->fused_W = 0;
            if ((s = plan_batch(b)) != SK_OK) b->fused_W = fused0;
        }
        const std::vector<sk_batch::Class> cls0 = b->classes;
        for (size_t k = 0; k < cls0.size() && s == SK_OK; ++k) {
            if (cls0[k].fused) continue;  // one shape for all its runs, set by mcmcmc_batch_set_fused
            const uint64_t key = cls0[k].key;
            uint32_t best = cls0[k].graph     ? ((cls0[k].nw << 16) | (32u << 8) | cls0[k].W)
                            : cls0[k].cluster ? ((cls0[k].cluster << 24) | (32u << 8) | cls0[k].W)
                                              : ((cls0[k].stage << 16) | (cls0[k].G << 8) | cls0[k].W);
            float best_ms = 1e30f;
            std::vector<uint32_t> cand;  // (stage << 16) | (G << 8) | W
            const uint32_t max_stage = ((key >> 60) & 1u) ? 0u : 1u;  // node-weighted classes: no staging
            bool single_k = true;  // one-chain runs only: whole-warp chains need no partner warp
            for (const sk_run* r : b->runs)
                if (class_key(r) == key) single_k = single_k && r->chains == 1;
            if ((key >> 59) & 1u) {  // graph classes: warps per chain and chains per CTA (even)
                const uint32_t fitc = static_cast<uint32_t>(std::min<size_t>(32, kSmemBudget / cls0[k].per_chain)) & ~1u;
                for (uint32_t nw : {1u, 2u, 4u, 8u, 16u})
                    for (uint32_t ch : {32u, 24u, 16u, 14u, 12u, 8u, 6u, 4u, 2u})
                        if (ch <= fitc && sk::graph_team_ok(nw * ch, nw)) cand.push_back((nw << 16) | (32u << 8) | (nw * ch));
            }
            for (uint32_t stage = 0; stage <= max_stage && !((key >> 59) & 1u); ++stage)
                for (uint32_t G = cls0[k].gmin; G <= 32; G <<= 1) {
                    const uint32_t fit =
                        fit_warps(stage ? cls0[k].per_chain_staged : cls0[k].per_chain_direct, G);
                    for (uint32_t w : {32u, 24u, 20u, 16u, 12u, 8u, 6u, 4u, 2u, 1u})
                        if (w <= std::max(fit, single_k ? 1u : 0u) && (G < 32 || (w & 1u) == 0 || single_k))
                            cand.push_back((stage << 16) | (G << 8) | w);
                }
            // star classes of few chains: the cluster-per-chain layout as well
            // (shapes the class cannot take fail to plan and are skipped)
            if (!((key >> 59) & 1u) && !((key >> 60) & 1u)) {
                uint64_t total = 0;
                bool single = true;
                for (const sk_run* r : b->runs)
                    if (class_key(r) == key) {
                        total += r->chains;
                        single = single && r->chains == 1;
                    }
                if (total <= kClusterTuneChains)
                    for (uint32_t C : {1u, 2u, 4u, 8u, 16u})
                        for (uint32_t w : {1u, 2u, 4u, 8u})
                            if ((w > 1 || single) && w <= std::max<uint64_t>(2, total))
                                cand.push_back((C << 24) | (32u << 8) | w);
                // and the team layout (2 or 4 warps per chain) for classes of at
                // most a few chains per SM (shapes it cannot take are skipped)
                if (total <= kTeamTuneChains)
                    for (uint32_t T : {2u, 4u}) cand.push_back(((32u * T) << 8) | (single ? 1u : 2u));
            }
            for (uint32_t gw : cand) {
                b->tuned[key] = gw;
                if (plan_batch(b) != SK_OK) continue;  // not resident: skip the candidate
                size_t idx = 0;
                while (idx < b->classes.size() && b->classes[idx].key != key) ++idx;
                if ((s = launch_segment(b, trial_steps, static_cast<int>(idx))) != SK_OK) break;  // warm-up
                restore();
                float ms = 1e30f;
                for (int rep = 0; rep < 2 && s == SK_OK; ++rep) {  // the better of two timed trials
                    cudaEventRecord(e0, b->st);
                    s = launch_segment(b, trial_steps, static_cast<int>(idx));
                    cudaEventRecord(e1, b->st);
                    cudaEventSynchronize(e1);
                    float m = 0;
                    cudaEventElapsedTime(&m, e0, e1);
                    ms = std::min(ms, m);
                    restore();
                }
                if (s != SK_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = gw;
                }
            }
            b->tuned[key] = best;
        }
        // then the whole batch with those per-class launches against the
        // fused launch of its star runs at 4, 8 and 16 warps per CTA; the
        // fastest is kept
        bool star_runs = false;
        for (const sk_run* r : b->runs) star_runs = star_runs || fused_eligible(r);
        if (s == SK_OK && star_runs) {
            auto time_batch = [&](float* out) -> sk_status {
                sk_status s2 = launch_segment(b, trial_steps);  // warm-up
                restore();
                float t = 1e30f;
                for (int rep = 0; rep < 2 && s2 == SK_OK; ++rep) {
                    cudaEventRecord(e0, b->st);
                    s2 = launch_segment(b, trial_steps);
                    cudaEventRecord(e1, b->st);
                    cudaEventSynchronize(e1);
                    float m = 0;
                    cudaEventElapsedTime(&m, e0, e1);
                    t = std::min(t, m);
                    restore();
                }
                *out = t;
                return s2;
            };
            uint32_t best_w = 0;
            float best_ms = 1e30f;
            for (uint32_t w : {0u, 4u, 8u, 16u}) {
                b->fused_W = w;
                if (plan_batch(b) != SK_OK) continue;  // not resident: skip
                float ms = 0;
                if ((s = time_batch(&ms)) != SK_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_w = w;
                }
            }
            b->fused_W = best_w;
        } else if (s == SK_OK) {
            b->fused_W = fused0;
        }
        for (size_t i = 0; i < b->runs.size(); ++i) {
            b->runs[i]->step = mirror[i];
            b->runs[i]->sop_valid = false;  // the trials' spins, not the restored ones
        }
        std::vector<JobDev> jobs;
        for (sk_run* r : b->runs) jobs.push_back(r->job);
        cudaMemcpy(b->djobs, jobs.data(), jobs.size() * sizeof(JobDev), cudaMemcpyHostToDevice);
        cudaStreamSynchronize(b->st);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    for (Backup& x : bk) {
        cudaFree(x.s);
        cudaFree(x.h);
        cudaFree(x.acc);
        cudaFree(x.work);
        cudaFree(x.step);
    }
    if (s != SK_OK) {
        b->tuned = tuned0;
        b->fused_W = fused_before;
        plan_batch(b);
        return s;
    }
    if ((s = plan_batch(b)) != SK_OK) return s;
    if (out_W) *out_W = b->classes.empty() ? 0 : b->classes[0].W;
    return SK_OK;
}

sk_status mcmcmc_batch_info(const sk_batch* b, uint32_t* grid, uint32_t* W, uint32_t* smem,
                            uint32_t* items) {
    if (!b) return fail(SK_ERR_INVALID_ARG, "batch is NULL");
    if (grid) *grid = b->grid;
    if (W) *W = b->classes.empty() ? 0 : b->classes[0].W;
    if (smem) {
        const sk_batch::Class* c = b->classes.empty() ? nullptr : &b->classes[0];
        *smem = !c ? 0
                : c->fused ? c->fsmem
                : c->cluster ? c->jbytes + c->W * c->per_chain
                : c->team    ? c->W * c->per_chain
                             : c->per_chain * c->W * (32 / c->G);
    }
    if (items) *items = b->n_items;
    return SK_OK;
}

sk_status mcmcmc_batch_classes(const sk_batch* b, uint32_t max, uint32_t* count, uint32_t* desc) {
    if (!b || !count) return fail(SK_ERR_INVALID_ARG, "NULL argument");
    *count = static_cast<uint32_t>(b->classes.size());
    for (uint32_t k = 0; k < *count && k < max && desc; ++k) {
        const sk_batch::Class& c = b->classes[k];
        desc[6 * k + 0] = static_cast<uint32_t>(c.cls);
        desc[6 * k + 1] = c.G;
        desc[6 * k + 2] = c.per_chain;
        desc[6 * k + 3] = c.W;
        desc[6 * k + 4] = c.n_items;
        desc[6 * k + 5] = c.grid;
    }
    return SK_OK;
}

sk_status mcmcmc_batch_free(sk_batch* b) {
    if (!b) return fail(SK_ERR_INVALID_ARG, "batch is NULL");
    cudaStreamSynchronize(b->st);
    for (sk_run* r : b->runs) r->batches--;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    free_side_streams(b);
    cudaFree(b->djobs);
    cudaFree(b->ditems);
    cudaFree(b->dqueue);
    delete b;
    return SK_OK;
}

}  // extern "C"

namespace sk {
// The run stops at `limit` steps in every later advance (used by the server).
void set_step_limit(sk_run* r, uint32_t limit) { r->job.step_limit = limit; }

bool root_setup(JobDev& j, uint32_t K, double p_center) {
    j.fcen = j.fleaf = 1u << 20;
    j.lcen = j.lleaf = 0.0f;
    if (K < 1) K = 1;
    if (p_center == 0.0) {  // uniform: centre iff U0 < ceil(2^64 / (K+1))
        j.root_thr = UINT64_MAX / (static_cast<uint64_t>(K) + 1u) + 1u;
        return true;
    }
    if (!(p_center > 0.0 && p_center < 1.0)) return false;
    const double pl = (1.0 - p_center) / static_cast<double>(K);
    const double pm = p_center > pl ? p_center : pl;
    const uint64_t Fc = static_cast<uint64_t>(p_center / pm * 1048576.0 + 0.5);
    const uint64_t Fl = static_cast<uint64_t>(pl / pm * 1048576.0 + 0.5);
    if (Fc < 1u || Fl < 1u) return false;
    const double pc = static_cast<double>(Fc) / (static_cast<double>(Fc) + static_cast<double>(K) * static_cast<double>(Fl));
    j.root_thr = static_cast<uint64_t>(std::ldexp(pc, 64));
    j.fcen = static_cast<uint32_t>(Fc);
    j.fleaf = static_cast<uint32_t>(Fl);
    j.lcen = static_cast<float>(std::log2(static_cast<double>(Fc)) - 20.0);
    j.lleaf = static_cast<float>(std::log2(static_cast<double>(Fl)) - 20.0);
    return true;
}
uint64_t host_step(const sk_run* r) { return r->step; }
// Device bytes of a run: spins and fields, per-chain counters, records, the
// +-J table, the tensor-core spin operand and drift accumulator (the start
// fields are computed on the tensor cores) and the host-start staging copy.
size_t run_footprint(uint32_t N, uint32_t kind, uint32_t chains, uint64_t records) {
    const size_t np = pad_n(N);
    return static_cast<size_t>(chains) * np * 5 + static_cast<size_t>(chains) * 20 +
           records * (static_cast<size_t>(chains) * 12 + static_cast<size_t>(chains / 2) * 8) +
           (kind == SK_J_PM1 ? (4 * static_cast<size_t>(N) + 5) * 8 : 0) +
           sk::recompute_s_bytes(kind, chains, static_cast<uint32_t>(np)) + static_cast<size_t>(chains) * 8 +
           static_cast<size_t>(chains) * N + 4096;
}
// Device bytes of an instance: the couplings and their tensor-core operand.
size_t instance_footprint(uint32_t N, uint32_t kind) {
    const size_t np = pad_n(N);
    return np * np * jbytes(kind) + sk::recompute_j_bytes(kind, static_cast<uint32_t>(np));
}
}  // namespace sk
