// sk_noalloc.cu -- mcmcmc_run_noalloc: a run of the MCMCMC step kernel whose
// working memory lives in a fixed array of device globals instead of memory
// obtained from cudaMalloc.
//
// Who needs it: callers that cannot allocate device memory themselves or let
// a library do so -- an application whose device memory is entirely owned by
// its own pool allocator (a framework that reserved the GPU's memory for its
// caching allocator, where an extra cudaMalloc fails or fragments the pool),
// a latency-critical loop that cannot afford cudaMalloc's implicit device
// synchronisation, or a plug-in host that forbids libraries from allocating.
// They pass their couplings and spins in device memory and get the final
// spins and energies back in their own buffers.
//
// The array costs every GPU that loads this library SK_NOALLOC_SCRATCH_BYTES
// (16 MiB) of device memory until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "sk_internal.h"
#include "sk_mcmcmc.h"

namespace {

// The scratch array.  In host code its name is only a host-side stand-in for
// the symbol: kernels must be given the address returned by
// cudaGetSymbolAddress for the current device, never &g_noalloc_scratch.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SK_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Failures are reported through sk_last_error(), like every other entry point.
sk_status nfail(sk_status s, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    sk::set_error_message(msg);
    return s;
}

#define NA_CU(call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return nfail(SK_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

// Device address of the scratch array on the current device; looked up once
// per device (with that device current) on the first call made on it.
sk_status scratch_address(void** out) {
    int dev = 0;
    NA_CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return nfail(SK_ERR_CUDA, "device index %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return nfail(SK_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SK_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

constexpr size_t kSmemBudget = 232448 - 5120;  // the step kernel's static shared memory reserved

}  // namespace

extern "C" sk_status mcmcmc_run_noalloc(uint32_t N, uint32_t kind, const void* couplings,
                                        double scale, uint32_t chains, uint32_t K, uint32_t rule,
                                        double beta, uint64_t seed, uint32_t stream_id,
                                        uint64_t steps, int8_t* spins, double* energy,
                                        void* stream) {
    if (!couplings || !spins || !energy) return nfail(SK_ERR_INVALID_ARG, "NULL device buffer");
    if (N < 2 || N > SK_MAX_N) return nfail(SK_ERR_INVALID_ARG, "N = %u outside 2..%u", N, SK_MAX_N);
    if (kind != SK_J_PM1 && kind != SK_J_GAUSS) return nfail(SK_ERR_INVALID_ARG, "unknown coupling kind");
    if (rule != SK_RULE_MCMCMC && rule != SK_RULE_METROPOLIS) return nfail(SK_ERR_INVALID_ARG, "unknown rule");
    if (rule == SK_RULE_METROPOLIS) K = 1;
    if (K < 1 || K > SK_MAX_K) return nfail(SK_ERR_INVALID_ARG, "K = %u outside 1..%u", K, SK_MAX_K);
    if (chains == 0) return nfail(SK_ERR_INVALID_ARG, "chains = 0");
    if (!(beta >= 0.0) || !std::isfinite(beta) || !(scale > 0.0) || !std::isfinite(scale))
        return nfail(SK_ERR_INVALID_ARG, "beta must be >= 0 and scale > 0");
    if (stream_id > 0xFFFFFFu) return nfail(SK_ERR_INVALID_ARG, "stream_id must fit 24 bits");
    if (steps > 0xFFFFFFFFull) return nfail(SK_ERR_INVALID_ARG, "steps must be < 2^32");

    const uint32_t Npad = (N + sk::kPadTo - 1) / sk::kPadTo * sk::kPadTo;
    const size_t bj = kind == SK_J_PM1 ? 1 : 4;
    size_t per_warp = (sk::warp_smem_bytes(Npad, kind) + 127) / 128 * 128;
    const uint32_t W = static_cast<uint32_t>(std::min<size_t>(32, kSmemBudget / per_warp)) & ~1u;
    if (W < 2) return nfail(SK_ERR_INVALID_ARG, "N too large for one CTA");
    const uint32_t n_items = (chains + W - 1) / W;

    // table of the +-J weights: W[d] (MCMCMC) or M[k] (Metropolis)
    const uint32_t tab_max = rule == SK_RULE_MCMCMC ? 4 * N + 5 : N + 1;
    const size_t tab_bytes = kind == SK_J_PM1 ? static_cast<size_t>(tab_max) * 8 : 0;

    // layout of the scratch array
    size_t off = 0;
    const size_t o_job = off;    off += up256(sizeof(sk::JobDev));
    const size_t o_ctl = off;    off += 256;  // queue (4 B), error word (4 B), step (8 B)
    const size_t o_items = off;  off += up256(static_cast<size_t>(n_items) * sizeof(sk::WorkItem));
    const size_t o_tab = off;    off += up256(tab_bytes);
    const size_t o_J = off;      off += up256(static_cast<size_t>(Npad) * Npad * bj);
    const size_t o_s = off;      off += up256(static_cast<size_t>(chains) * Npad);
    const size_t o_h = off;      off += up256(static_cast<size_t>(chains) * Npad * 4);
    const size_t o_acc = off;    off += up256(static_cast<size_t>(chains) * 4);
    const size_t o_work = off;   off += up256(static_cast<size_t>(chains) * 16);
    if (off > SK_NOALLOC_SCRATCH_BYTES)
        return nfail(SK_ERR_INVALID_ARG,
                     "problem needs %zu bytes of scratch, more than the %u-byte allocation-free limit "
                     "(N = %u, chains = %u); use mcmcmc_run",
                     off, SK_NOALLOC_SCRATCH_BYTES, N, chains);

    void* base_v = nullptr;
    sk_status st_ = scratch_address(&base_v);
    if (st_ != SK_OK) return st_;
    unsigned char* base = static_cast<unsigned char*>(base_v);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t* queue = reinterpret_cast<uint32_t*>(base + o_ctl);
    int* err = reinterpret_cast<int*>(base + o_ctl + 4);
    uint64_t* step = reinterpret_cast<uint64_t*>(base + o_ctl + 8);
    unsigned long long* bad_spin = reinterpret_cast<unsigned long long*>(base + o_ctl + 16);

    // the array keeps the previous call's contents: clear what starts at zero
    NA_CU(cudaMemsetAsync(base + o_ctl, 0, 256, st));

    // the start spins must be +-1: the first offending index is recorded in
    // the control block (the check sets its word to all ones first)
    {
        NA_CU(sk::launch_check_spins(spins, static_cast<uint64_t>(chains) * N, bad_spin, st));
        unsigned long long hbad = 0;
        NA_CU(cudaMemcpyAsync(&hbad, bad_spin, sizeof hbad, cudaMemcpyDeviceToHost, st));
        NA_CU(cudaStreamSynchronize(st));
        if (hbad != ~0ull)
            return nfail(SK_ERR_INVALID_ARG, "start spin %llu (chain %llu, site %llu) is not +-1", hbad >> 2,
                         (hbad >> 2) / N, (hbad >> 2) % N);
    }
    NA_CU(cudaMemsetAsync(base + o_J, 0, static_cast<size_t>(Npad) * Npad * bj, st));
    NA_CU(cudaMemcpy2DAsync(base + o_J, Npad * bj, couplings, N * bj, N * bj, N,
                            cudaMemcpyDeviceToDevice, st));

    // +-J table, built on the host in a fixed stack buffer and copied in chunks
    uint32_t wlen = 0;
    if (kind == SK_J_PM1) {
        const double be = beta * scale;
        uint64_t chunk[512];
        uint32_t n_in_chunk = 0, first = 0;
        bool done = false;
        for (uint32_t d = 0; d < tab_max && !done; ++d) {
            const double x = rule == SK_RULE_MCMCMC ? std::ldexp(std::exp(-2.0 * be * d), 52)
                                                    : std::ldexp(std::exp(-2.0 * be * d), 53);
            const double v = std::nearbyint(x);
            if (!(v > 0.0)) {  // the table ends where its entries round to 0
                done = true;
                break;
            }
            chunk[n_in_chunk++] = static_cast<uint64_t>(v);
            ++wlen;
            if (n_in_chunk == 512) {
                NA_CU(cudaMemcpyAsync(base + o_tab + 8ull * first, chunk, 8ull * n_in_chunk,
                                      cudaMemcpyHostToDevice, st));
                NA_CU(cudaStreamSynchronize(st));
                first += n_in_chunk;
                n_in_chunk = 0;
            }
        }
        if (n_in_chunk) {
            NA_CU(cudaMemcpyAsync(base + o_tab + 8ull * first, chunk, 8ull * n_in_chunk,
                                  cudaMemcpyHostToDevice, st));
            NA_CU(cudaStreamSynchronize(st));
        }
    }

    sk::JobDev job;
    std::memset(&job, 0, sizeof job);
    job.J = base + o_J;
    job.s = reinterpret_cast<int8_t*>(base + o_s);
    job.h = base + o_h;
    job.W = kind == SK_J_PM1 ? reinterpret_cast<const uint64_t*>(base + o_tab) : nullptr;
    job.step = step;
    job.acc_run = reinterpret_cast<uint32_t*>(base + o_acc);
    job.err = err;
    job.work = reinterpret_cast<unsigned long long*>(base + o_work);
    job.seed = seed;
    job.scale = scale;
    job.beta_eff = static_cast<float>(beta * scale);
    job.stream = stream_id;
    job.N = N;
    job.Npad = Npad;
    job.chains = chains;
    job.K = K;
    job.kind = kind;
    job.rule = rule;
    job.wlen = wlen;
    job.step_limit = 0xFFFFFFFFu;  // no per-run step limit
    sk::root_setup(job, K, 0.0);   // uniform root
    NA_CU(cudaMemcpyAsync(base + o_job, &job, sizeof job, cudaMemcpyHostToDevice, st));

    // work items: blocks of W chains, copied from a fixed stack buffer
    {
        sk::WorkItem buf[256];
        uint32_t n = 0, first = 0;
        for (uint32_t c = 0; c < chains; c += W) {
            buf[n++] = sk::WorkItem{0u, c, std::min(W, chains - c), 0u};
            if (n == 256 || c + W >= chains) {
                NA_CU(cudaMemcpyAsync(base + o_items + sizeof(sk::WorkItem) * first, buf,
                                      sizeof(sk::WorkItem) * n, cudaMemcpyHostToDevice, st));
                NA_CU(cudaStreamSynchronize(st));
                first += n;
                n = 0;
            }
        }
    }

    NA_CU(sk::launch_init(&job, spins, chains, N, Npad, kind, st));
    const int cls = sk::step_class(kind, rule, K, 32, 1);  // whole-warp chains, staged rows
    int dev = 0, sms = 0;
    NA_CU(cudaGetDevice(&dev));
    NA_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int occ = sk::step_kernel_occupancy(cls, W, per_warp);  // bytes per chain (one chain per warp)
    if (occ <= 0) return nfail(SK_ERR_CUDA, "step kernel cannot be resident");
    const uint32_t grid = std::min<uint32_t>(n_items, static_cast<uint32_t>(occ * sms));
    if (steps)
        NA_CU(sk::launch_step(reinterpret_cast<const sk::JobDev*>(base + o_job),
                              reinterpret_cast<const sk::WorkItem*>(base + o_items), n_items, queue,
                              steps, W, static_cast<uint32_t>(per_warp), grid, cls, 1, true, st));
    NA_CU(cudaMemcpy2DAsync(spins, N, base + o_s, Npad, N, chains, cudaMemcpyDeviceToDevice, st));
    NA_CU(sk::launch_energy(base + o_J, kind, N, Npad, scale, spins, chains, energy, st));
    int herr = 0;
    NA_CU(cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, st));
    NA_CU(cudaStreamSynchronize(st));
    if (herr == sk::kDevTimeout) return nfail(SK_ERR_TIMEOUT, "a bounded device wait expired");
    if (herr != 0) return nfail(SK_ERR_DEVICE, "kernel error %d", herr);
    return SK_OK;
}
