// sk_team_pm1.cu -- the team-layout step kernels for +-J couplings (int8 J,
// int32 fields); see sk_team.cuh.
#include "sk_team.cuh"

namespace sk {
cudaError_t launch_team_pm1(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                            uint32_t nsteps, uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain,
                            uint32_t grid, cudaStream_t st) {
    return team::launch_kind<int8_t>(jobs, items, n_items, queue, nsteps, rule, T, teams, per_chain, grid, st);
}
int occupancy_team_pm1(uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain) {
    return team::occupancy_kind<int8_t>(rule, T, teams, per_chain);
}
}  // namespace sk
