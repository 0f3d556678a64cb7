// sk_step_pm1_metropolis_staged.cu -- step-kernel instantiations for +-J (int8) couplings, the Metropolis rule, row a staged by TMA (compiled as its own
// translation unit so that the variants build in parallel).
#include "sk_step.cuh"

namespace sk {

cudaError_t launch_step_pm1_metropolis_staged(int nb, int G, const JobDev* jobs, const WorkItem* items, uint32_t n_items,
                           uint32_t* queue, uint32_t nsteps, uint32_t W, uint32_t per_chain, uint32_t grid,
                           cudaStream_t st) {
    return step::launch_rule<int8_t, 1, 1>(nb, G, jobs, items, n_items, queue, nsteps, W, per_chain, grid, st);
}

int occupancy_pm1_metropolis_staged(int nb, int G, uint32_t W, uint32_t per_chain) {
    return step::occupancy_rule<int8_t, 1, 1>(nb, G, W, per_chain);
}

}  // namespace sk
