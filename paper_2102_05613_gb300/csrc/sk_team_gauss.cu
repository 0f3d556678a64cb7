// sk_team_gauss.cu -- the team-layout step kernels for Gaussian couplings
// (fp32 J and fields); see sk_team.cuh.
#include "sk_team.cuh"

namespace sk {
cudaError_t launch_team_gauss(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                              uint32_t nsteps, uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain,
                              uint32_t grid, cudaStream_t st) {
    return team::launch_kind<float>(jobs, items, n_items, queue, nsteps, rule, T, teams, per_chain, grid, st);
}
int occupancy_team_gauss(uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain) {
    return team::occupancy_kind<float>(rule, T, teams, per_chain);
}
}  // namespace sk
