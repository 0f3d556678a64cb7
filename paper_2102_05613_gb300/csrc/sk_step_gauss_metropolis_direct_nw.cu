// sk_step_gauss_metropolis_direct_nw.cu -- step-kernel instantiations for Gaussian (float) couplings, the Metropolis rule, row a read through L1, node-weighted energy records (compiled as its own
// translation unit so that the variants build in parallel).
#include "sk_step.cuh"

namespace sk {

cudaError_t launch_step_gauss_metropolis_direct_nw(int nb, int G, const JobDev* jobs, const WorkItem* items, uint32_t n_items,
                           uint32_t* queue, uint32_t nsteps, uint32_t W, uint32_t per_chain, uint32_t grid,
                           cudaStream_t st) {
    return step::launch_rule<float, 1, 2>(nb, G, jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
}

int occupancy_gauss_metropolis_direct_nw(int nb, int G, uint32_t W, uint32_t per_chain) {
    return step::occupancy_rule<float, 1, 2>(nb, G, W, per_chain);
}

}  // namespace sk
