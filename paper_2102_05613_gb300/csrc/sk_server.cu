// sk_server.cu -- continuous-batching request server for sampling jobs.
//
// A worker thread owns one CUDA stream and runs the scheduling loop in
// quanta of `quantum_steps` Monte Carlo steps:
//   1. retire: jobs whose chains reached their step count are read back
//      (final spins and energies) and their device memory is released;
//   2. admit: queued jobs are admitted first-in first-out while the sum of
//      the admitted jobs' device footprints (couplings, unless already
//      resident under the same couplings_id, + 5 bytes per spin per chain +
//      per-chain counters) fits the budget;
//   3. advance: every admitted job moves by up to one quantum in ONE
//      persistent launch per kernel class (the batch plan is rebuilt when
//      the mix changed); a job stops at its own step count.
// Jobs that arrive while others are on the GPU join at the next quantum, and
// their chains run in the same launches as the others'.  A chain's draws are
// addressed by (seed, stream_id, chain, step), so a job's result does not
// depend on which other jobs shared its launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "sk_internal.h"
#include "sk_mcmcmc.h"

namespace {

using Clock = std::chrono::steady_clock;

// Couplings registered under an id: the host copy lives as long as the
// server; the device copy is made on first use and dropped when idle jobs
// need the room.
struct Resident {
    std::vector<unsigned char> host;
    sk_instance* inst = nullptr;
    size_t bytes = 0;
    int users = 0;
    uint32_t N = 0, kind = 0;
    double scale = 1.0;
};

struct Job {
    uint64_t ticket = 0;
    sk_job spec{};
    std::vector<unsigned char> couplings;  // copied at submit
    std::vector<int8_t> init;
    sk_job_status status{};
    size_t run_bytes = 0, inst_bytes = 0;
    sk_instance* own_inst = nullptr;  // couplings_id == 0: private instance
    Resident* shared = nullptr;
    sk_run* run = nullptr;
    std::vector<double> energies;
    std::vector<int8_t> spins;
    uint64_t flips = 0;
    std::atomic<bool> cancel{false};  // set by sk_server_cancel while the job runs
};

}  // namespace

// Threads: the worker alone creates and frees device objects; `mu` guards
// the queue, the job table, the active list's changes, job statuses and the
// counters, which the caller's threads read; `used` is atomic because the
// worker changes it while admitting without holding `mu`.
struct sk_server {
    uint64_t budget = 0;
    std::atomic<uint64_t> used{0};
    uint32_t quantum = 256;
    cudaStream_t st = nullptr;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<std::shared_ptr<Job>> queue;             // submitted, not admitted
    std::vector<std::shared_ptr<Job>> active;           // admitted, on the device
    std::map<uint64_t, std::shared_ptr<Job>> jobs;      // every job until its result is taken
    std::map<uint64_t, std::unique_ptr<Resident>> resident;  // couplings_id -> instance
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    Clock::time_point t0;
    // counters
    uint64_t chain_steps = 0, candidates = 0, quanta = 0, completed = 0;
    double busy_s = 0, admit_s = 0, retire_s = 0, plan_s = 0;
    sk_status fatal = SK_OK;
};

namespace {

double since(const sk_server* s) {
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

// Device footprint of a job: its chains plus its couplings unless they are
// already resident (shared couplings_id).
void footprint(sk_server* s, Job& j) {
    j.run_bytes = sk::run_footprint(j.spec.N, j.spec.kind, j.spec.chains, 0);
    j.inst_bytes = sk::instance_footprint(j.spec.N, j.spec.kind);
}

bool fits(sk_server* s, const Job& j) {
    size_t need = j.run_bytes;
    if (!j.spec.couplings_id) {
        need += j.inst_bytes;
    } else {
        auto it = s->resident.find(j.spec.couplings_id);
        if (it == s->resident.end() || !it->second->inst) need += j.inst_bytes;
    }
    return s->used + need <= s->budget;
}

sk_status admit(sk_server* s, Job& j) {
    sk_status r = SK_OK;
    sk_instance* inst = nullptr;
    if (j.spec.couplings_id) {
        Resident* res;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            auto it = s->resident.find(j.spec.couplings_id);
            if (it == s->resident.end()) return SK_ERR_INVALID_ARG;
            res = it->second.get();
        }
        if (res->N != j.spec.N || res->kind != j.spec.kind || res->scale != j.spec.scale)
            return SK_ERR_INVALID_ARG;
        if (!res->inst) {
            r = sk_create_instance(res->N, res->kind, res->host.data(), SK_MEM_HOST, 0, res->scale, s->st,
                                   &res->inst);
            if (r != SK_OK) {
                res->inst = nullptr;
                return r;
            }
            s->used += res->bytes;
        }
        inst = res->inst;
        j.shared = res;
        res->users++;
    } else {
        r = sk_create_instance(j.spec.N, j.spec.kind, j.couplings.data(), SK_MEM_HOST, 0, j.spec.scale, s->st,
                               &inst);
        if (r != SK_OK) return r;
        j.own_inst = inst;
        s->used += j.inst_bytes;
    }
    j.couplings.clear();
    j.couplings.shrink_to_fit();
    sk_run_params p{};
    p.chains = j.spec.chains;
    p.K = j.spec.K;
    p.rule = j.spec.rule;
    p.beta = j.spec.beta;
    p.seed = j.spec.seed;
    p.stream_id = j.spec.stream_id;
    p.p_center = j.spec.p_center;
    p.init_spins = j.init.empty() ? nullptr : j.init.data();
    p.init_mem = SK_MEM_HOST;
    r = mcmcmc_create(inst, &p, &j.run);
    if (r != SK_OK) return r;
    sk::set_step_limit(j.run, static_cast<uint32_t>(j.spec.steps));
    s->used += j.run_bytes;
    j.init.clear();
    j.init.shrink_to_fit();
    return SK_OK;
}

void release(sk_server* s, Job& j) {
    if (j.run) {
        mcmcmc_free(j.run);
        j.run = nullptr;
        s->used -= j.run_bytes;
    }
    if (j.own_inst) {
        sk_destroy_instance(j.own_inst);
        j.own_inst = nullptr;
        s->used -= j.inst_bytes;
    }
    if (j.shared) {
        j.shared->users--;
        j.shared = nullptr;  // resident couplings stay until evicted for room
    }
}

// Drops the device copies of idle registered couplings until `need` more
// bytes fit (their host copies stay for later jobs).
void evict_for(sk_server* s, size_t need) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->resident) {
        if (s->used + need <= s->budget) break;
        Resident* r = kv.second.get();
        if (r->users == 0 && r->inst) {
            sk_destroy_instance(r->inst);
            r->inst = nullptr;
            s->used -= r->bytes;
        }
    }
}

void retire(sk_server* s, Job& j) {
    const size_t C = j.spec.chains, N = j.spec.N;
    j.spins.resize(C * N);
    j.energies.resize(C);
    sk_status r = mcmcmc_state(j.run, j.spins.data(), nullptr, nullptr, SK_MEM_HOST);
    sk_instance* inst = j.own_inst ? j.own_inst : j.shared->inst;
    if (r == SK_OK) r = sk_energy(inst, j.spins.data(), static_cast<uint32_t>(C), SK_MEM_HOST, j.energies.data());
    if (r == SK_OK) r = mcmcmc_counters(j.run, &j.flips, nullptr);
    release(s, j);
    std::lock_guard<std::mutex> lk(s->mu);
    j.status.state = r == SK_OK ? SK_JOB_DONE : SK_JOB_FAILED;
    j.status.error = r;
    j.status.t_done = since(s);
    s->completed++;
    s->done_cv.notify_all();
}

void loop(sk_server* s) {
    sk_batch* batch = nullptr;
    bool dirty = true;
    for (;;) {
        // 1. retire finished jobs
        const auto tr0 = Clock::now();
        std::vector<std::shared_ptr<Job>> still;
        for (auto& j : s->active) {
            if (j->cancel.load()) {  // withdrawn while running: release, keep nothing
                if (batch) {
                    mcmcmc_batch_free(batch);
                    batch = nullptr;
                }
                release(s, *j);
                std::lock_guard<std::mutex> lk(s->mu);
                j->status.state = SK_JOB_CANCELLED;
                j->status.error = SK_ERR_CANCELLED;
                j->status.t_done = since(s);
                s->completed++;
                s->done_cv.notify_all();
                dirty = true;
            } else if (sk::host_step(j->run) >= j->spec.steps) {
                if (batch) {
                    mcmcmc_batch_free(batch);
                    batch = nullptr;
                }
                retire(s, *j);
                dirty = true;
            } else {
                still.push_back(j);
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->active.swap(still);
            s->retire_s += std::chrono::duration<double>(Clock::now() - tr0).count();
        }
        // 2. admit queued jobs that fit, first in first out
        {
            std::unique_lock<std::mutex> lk(s->mu);
            while (!s->stop && s->queue.empty() && s->active.empty()) s->cv.wait(lk);
            if (s->stop && s->queue.empty() && s->active.empty()) break;
            while (!s->queue.empty()) {
                auto j = s->queue.front();
                if (!fits(s, *j)) {
                    lk.unlock();
                    evict_for(s, j->run_bytes + j->inst_bytes);
                    lk.lock();
                    if (!fits(s, *j)) break;
                }
                s->queue.pop_front();
                lk.unlock();
                if (batch) {
                    mcmcmc_batch_free(batch);
                    batch = nullptr;
                }
                const auto ta0 = Clock::now();
                const sk_status r = admit(s, *j);
                lk.lock();
                s->admit_s += std::chrono::duration<double>(Clock::now() - ta0).count();
                if (r != SK_OK) {
                    release(s, *j);
                    j->status.state = SK_JOB_FAILED;
                    j->status.error = r;
                    j->status.t_done = since(s);
                    s->completed++;
                    s->done_cv.notify_all();
                    continue;
                }
                j->status.state = SK_JOB_RUNNING;
                j->status.t_admit = since(s);
                s->active.push_back(j);
                dirty = true;
            }
        }
        if (s->active.empty()) continue;
        // 3. one quantum of every admitted job in one launch per kernel class
        if (dirty || !batch) {
            const auto tp0 = Clock::now();
            if (batch) mcmcmc_batch_free(batch);
            batch = nullptr;
            std::vector<sk_run*> runs;
            for (auto& j : s->active) runs.push_back(j->run);
            if (mcmcmc_batch_create(runs.data(), static_cast<uint32_t>(runs.size()), 0, &batch) != SK_OK) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->fatal = SK_ERR_CUDA;
                for (auto& j : s->active) {
                    j->status.state = SK_JOB_FAILED;
                    j->status.error = SK_ERR_CUDA;
                    j->status.t_done = since(s);
                    s->completed++;
                }
                s->done_cv.notify_all();
                break;
            }
            dirty = false;
            std::lock_guard<std::mutex> lk(s->mu);
            s->plan_s += std::chrono::duration<double>(Clock::now() - tp0).count();
        }
        uint64_t cs = 0, cand = 0;
        for (auto& j : s->active) {
            const uint64_t left = j->spec.steps - sk::host_step(j->run);
            const uint64_t n = std::min<uint64_t>(left, s->quantum);
            cs += n * j->spec.chains;
            cand += n * j->spec.chains * (j->spec.rule == SK_RULE_MCMCMC ? j->spec.K : 1u);
        }
        const auto a = Clock::now();
        sk_status r = mcmcmc_batch_advance(batch, s->quantum);
        if (r == SK_OK && cudaStreamSynchronize(s->st) != cudaSuccess) r = SK_ERR_CUDA;
        std::lock_guard<std::mutex> lk(s->mu);
        s->busy_s += std::chrono::duration<double>(Clock::now() - a).count();
        s->chain_steps += cs;
        s->candidates += cand;
        s->quanta++;
        if (r != SK_OK) {
            s->fatal = r;
            s->done_cv.notify_all();
            break;
        }
    }
    if (batch) mcmcmc_batch_free(batch);
    for (auto& j : s->active) release(s, *j);
    std::lock_guard<std::mutex> lk(s->mu);
    s->active.clear();
}

}  // namespace

extern "C" {

sk_status sk_server_create(uint64_t budget_bytes, uint32_t quantum_steps, sk_server** out) {
    if (!out || budget_bytes == 0 || quantum_steps == 0) return SK_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return SK_ERR_CUDA;
    sk_server* s = new sk_server();
    s->budget = budget_bytes;
    s->quantum = quantum_steps;
    s->t0 = Clock::now();
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return SK_ERR_CUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    s->worker = std::thread([s, dev] {
        cudaSetDevice(dev);
        loop(s);
    });
    *out = s;
    return SK_OK;
}

sk_status sk_server_add_couplings(sk_server* s, uint64_t id, uint32_t N, uint32_t kind, const void* couplings,
                                  double scale) {
    if (!s || !id || !couplings || N < 2 || N > SK_MAX_N || (kind != SK_J_PM1 && kind != SK_J_GAUSS) ||
        !(scale > 0.0))
        return SK_ERR_INVALID_ARG;
    auto r = std::make_unique<Resident>();
    const size_t jb = static_cast<size_t>(N) * N * (kind == SK_J_PM1 ? 1 : 4);
    const unsigned char* c = static_cast<const unsigned char*>(couplings);
    r->host.assign(c, c + jb);
    r->N = N;
    r->kind = kind;
    r->scale = scale;
    r->bytes = sk::instance_footprint(N, kind);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->resident.count(id)) return SK_ERR_INVALID_ARG;
    s->resident[id] = std::move(r);
    return SK_OK;
}

sk_status sk_server_submit(sk_server* s, const sk_job* job, uint64_t* ticket) {
    if (!s || !job || !ticket || (!job->couplings && !job->couplings_id)) return SK_ERR_INVALID_ARG;
    if (job->N < 2 || job->N > SK_MAX_N || (job->kind != SK_J_PM1 && job->kind != SK_J_GAUSS) ||
        job->chains == 0 || job->steps == 0 || job->steps > 0xFFFFFFFFull ||
        (job->rule == SK_RULE_MCMCMC && (job->K < 1 || job->K > SK_MAX_K)) ||
        (job->rule != SK_RULE_MCMCMC && job->rule != SK_RULE_METROPOLIS) || !(job->beta >= 0.0) ||
        !(job->scale > 0.0) || job->stream_id > 0xFFFFFFu)
        return SK_ERR_INVALID_ARG;
    if (job->rule == SK_RULE_MCMCMC) {
        sk::JobDev probe{};
        if (!sk::root_setup(probe, job->K, job->p_center)) return SK_ERR_INVALID_ARG;
    }
    auto j = std::make_shared<Job>();
    j->spec = *job;
    if (j->spec.rule == SK_RULE_METROPOLIS) j->spec.K = 1;
    if (!job->couplings_id) {  // private couplings: copied now
        const size_t jb = static_cast<size_t>(job->N) * job->N * (job->kind == SK_J_PM1 ? 1 : 4);
        const unsigned char* c = static_cast<const unsigned char*>(job->couplings);
        j->couplings.assign(c, c + jb);
    }
    if (job->init_spins)
        j->init.assign(job->init_spins, job->init_spins + static_cast<size_t>(job->chains) * job->N);
    j->spec.couplings = nullptr;
    j->spec.init_spins = nullptr;
    footprint(s, *j);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != SK_OK) return s->fatal;
    if (job->couplings_id && !s->resident.count(job->couplings_id)) return SK_ERR_INVALID_ARG;
    j->ticket = s->next_ticket++;
    j->status.state = SK_JOB_QUEUED;
    j->status.t_submit = since(s);
    j->status.footprint_bytes = j->run_bytes + j->inst_bytes;
    if (j->run_bytes + j->inst_bytes > s->budget) {
        j->status.state = SK_JOB_FAILED;
        j->status.error = SK_ERR_OOM;
        j->status.t_done = j->status.t_submit;
        s->completed++;
    } else {
        s->queue.push_back(j);
    }
    s->jobs[j->ticket] = j;
    *ticket = j->ticket;
    s->cv.notify_all();
    return SK_OK;
}

sk_status sk_server_poll(sk_server* s, uint64_t ticket, sk_job_status* st) {
    if (!s || !st) return SK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return SK_ERR_INVALID_ARG;
    *st = it->second->status;
    return SK_OK;
}

sk_status sk_server_result(sk_server* s, uint64_t ticket, double* energies, int8_t* spins, uint64_t* flips) {
    if (!s) return SK_ERR_INVALID_ARG;
    std::shared_ptr<Job> j;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return SK_ERR_INVALID_ARG;
        j = it->second;
        if (j->status.state == SK_JOB_QUEUED || j->status.state == SK_JOB_RUNNING) return SK_ERR_NOT_READY;
        s->jobs.erase(it);
    }
    if (j->status.state == SK_JOB_CANCELLED) return SK_ERR_CANCELLED;
    if (j->status.state == SK_JOB_FAILED) return j->status.error ? j->status.error : SK_ERR_CUDA;
    if (energies) std::memcpy(energies, j->energies.data(), j->energies.size() * sizeof(double));
    if (spins) std::memcpy(spins, j->spins.data(), j->spins.size());
    if (flips) *flips = j->flips;
    return SK_OK;
}

sk_status sk_server_cancel(sk_server* s, uint64_t ticket) {
    if (!s) return SK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return SK_ERR_INVALID_ARG;
    Job& j = *it->second;
    switch (j.status.state) {
        case SK_JOB_CANCELLED:
            return SK_OK;
        case SK_JOB_QUEUED: {
            for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
                if (q->get() == &j) {
                    s->queue.erase(q);
                    break;
                }
            j.status.state = SK_JOB_CANCELLED;
            j.status.error = SK_ERR_CANCELLED;
            j.status.t_done = since(s);
            s->completed++;
            s->done_cv.notify_all();
            return SK_OK;
        }
        case SK_JOB_RUNNING:  // the worker releases it at the next quantum boundary
            j.cancel = true;
            return SK_OK;
        default:
            return SK_ERR_INVALID_ARG;
    }
}

sk_status sk_server_wait_all(sk_server* s, uint64_t timeout_ns) {
    if (!s) return SK_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [s] { return s->fatal != SK_OK || (s->queue.empty() && s->active.empty() && [s] {
                                 for (auto& kv : s->jobs)
                                     if (kv.second->status.state == SK_JOB_QUEUED ||
                                         kv.second->status.state == SK_JOB_RUNNING)
                                         return false;
                                 return true;
                             }()); };
    if (timeout_ns) {
        if (!s->done_cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), idle)) return SK_ERR_TIMEOUT;
    } else {
        s->done_cv.wait(lk, idle);
    }
    return s->fatal;
}

sk_status sk_server_stats(sk_server* s, sk_server_stats_t* out) {
    if (!s || !out) return SK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->chain_steps = s->chain_steps;
    out->candidates = s->candidates;
    out->quanta = s->quanta;
    out->completed = s->completed;
    out->busy_seconds = s->busy_s;
    out->elapsed_seconds = since(s);
    out->device_bytes_in_use = s->used;
    out->queued = s->queue.size();
    out->running = s->active.size();
    out->admit_seconds = s->admit_s;
    out->retire_seconds = s->retire_s;
    out->plan_seconds = s->plan_s;
    return SK_OK;
}

sk_status sk_server_destroy(sk_server* s) {
    if (!s) return SK_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& kv : s->resident)
        if (kv.second->inst) sk_destroy_instance(kv.second->inst);
    s->resident.clear();
    cudaStreamDestroy(s->st);
    delete s;
    return SK_OK;
}

}  // extern "C"
