// sk_team.cu -- host side of the team layout: the launch of one class's
// items (see sk_team.cuh for the kernel).
#include <cuda_runtime.h>

#include "sk_internal.h"

namespace sk {

cudaError_t launch_team(const JobDev* jobs, const WorkItem* items, uint32_t n_items, uint32_t* queue,
                        uint64_t nsteps, uint32_t kind, uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain,
                        uint32_t grid, uint32_t n_jobs, bool bump, cudaStream_t st) {
    if ((T != 2 && T != 4) || (teams != 1 && teams != 2) || grid == 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const uint32_t ns = static_cast<uint32_t>(nsteps);
    e = kind == 0 ? launch_team_pm1(jobs, items, n_items, queue, ns, rule, T, teams, per_chain, grid, st)
                  : launch_team_gauss(jobs, items, n_items, queue, ns, rule, T, teams, per_chain, grid, st);
    if (e != cudaSuccess || !bump) return e;
    return launch_bump_steps(jobs, n_jobs, nsteps, st);
}

int team_occupancy(uint32_t kind, uint32_t rule, uint32_t T, uint32_t teams, uint32_t per_chain) {
    if ((T != 2 && T != 4) || (teams != 1 && teams != 2)) return 0;
    return kind == 0 ? occupancy_team_pm1(rule, T, teams, per_chain) : occupancy_team_gauss(rule, T, teams, per_chain);
}

}  // namespace sk
