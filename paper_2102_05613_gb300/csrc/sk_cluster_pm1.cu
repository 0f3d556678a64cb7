// sk_cluster_pm1.cu -- the cluster-per-chain step kernels for +-J couplings
// (int8 J, int32 fields); see sk_cluster.cuh.
#include "sk_cluster.cuh"

namespace sk {
cudaError_t launch_cluster_pm1(uint32_t rule, uint32_t nb, const JobDev* jobs, const WorkItem* items,
                               uint32_t n_items, uint32_t* queue, uint32_t nsteps, uint32_t C, uint32_t W,
                               uint32_t jbytes, uint32_t pc, uint32_t clusters, cudaStream_t st) {
    return cl::launch_kind<int8_t>(rule, nb, jobs, items, n_items, queue, nsteps, C, W, jbytes, pc, clusters, st);
}
int occupancy_cluster_pm1(uint32_t rule, uint32_t nb, uint32_t C, uint32_t W, uint32_t jbytes, uint32_t pc) {
    return cl::occupancy_kind<int8_t>(rule, nb, C, W, jbytes, pc);
}
}  // namespace sk
