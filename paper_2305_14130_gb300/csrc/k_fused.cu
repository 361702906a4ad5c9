// Batched execution: every shot (any window width) advances in the same
// launches.  Interim version: the per-half-step kernels over all shots
// (grid.z = shot), in place on buffer scur.
#include "plan.hpp"

namespace efwi {

void launch_step_fused(efwi_plan *p, int n, float *vseg_x, float *vseg_z, cudaStream_t st) {
    launch_vel_plain(p, -1, vseg_x, vseg_z, st);
    launch_stress_plain(p, -1, st);
    launch_inject(p, state_fields(p, p->scur), n, -1, st);
}

void launch_adj_fused(efwi_plan *p, int n, const float *vfx, const float *vfz, cudaStream_t st) {
    (void)n;
    launch_adj_vel_plain(p, -1, vfx, vfz, st);
    launch_adj_stress_plain(p, -1, vfx, vfz, st);
    p->apsi_v ^= 1;
}

}  // namespace efwi

int efwi_autotune(efwi_plan *p) {
    if (p->tile_x == 0) p->tile_x = 32;
    if (p->tile_z == 0) p->tile_z = 8;
    return EFWI_OK;
}
