// sk_cluster.cu -- host side of the cluster-per-chain layout: shared-memory
// sizes, shape rules and the launch (see sk_cluster.cuh for the kernel).
#include <cuda_runtime.h>

#include "sk_internal.h"

namespace sk {

namespace {
constexpr size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }
}  // namespace

bool cluster_shape_ok(uint32_t kind, uint32_t npad, uint32_t C) {
    if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16) return false;
    if (npad == 0 || npad % C) return false;
    const size_t ws = npad / C;
    return (ws * (kind == 0 ? 1 : 4)) % 16 == 0;
}

size_t cluster_slice_bytes(uint32_t kind, uint32_t N, uint32_t npad, uint32_t C) {
    return round_up(static_cast<size_t>(N) * (npad / C) * (kind == 0 ? 1 : 4), 128);
}

size_t cluster_chain_bytes(uint32_t rule, uint32_t nb, uint32_t npad, uint32_t C) {
    const size_t ws = npad / C;
    return round_up(cluster_x_bytes(rule, nb) + kB0Bytes + round_up(ws, 16) + 4 * ws, 128);
}

cudaError_t launch_cluster(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                           uint64_t nsteps, uint32_t kind, uint32_t rule, uint32_t nb, uint32_t C, uint32_t W,
                           uint32_t jbytes, uint32_t pc, uint32_t clusters, uint32_t n_jobs, bool bump,
                           cudaStream_t st) {
    if (W < 1 || W > kClusterMaxChains || clusters == 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const uint32_t ns = static_cast<uint32_t>(nsteps);
    e = kind == 0 ? launch_cluster_pm1(rule, nb, jobs, items, n_items, queue, ns, C, W, jbytes, pc, clusters, st)
                  : launch_cluster_gauss(rule, nb, jobs, items, n_items, queue, ns, C, W, jbytes, pc, clusters, st);
    if (e != cudaSuccess || !bump) return e;
    return launch_bump_steps(jobs, n_jobs, nsteps, st);
}

int cluster_occupancy(uint32_t kind, uint32_t rule, uint32_t nb, uint32_t C, uint32_t W, uint32_t jbytes,
                      uint32_t pc) {
    if (W < 1 || W > kClusterMaxChains) return 0;
    return kind == 0 ? occupancy_cluster_pm1(rule, nb, C, W, jbytes, pc)
                     : occupancy_cluster_gauss(rule, nb, C, W, jbytes, pc);
}

}  // namespace sk
