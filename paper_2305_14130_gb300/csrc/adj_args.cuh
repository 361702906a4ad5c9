// Arguments of the batched adjoint steps with per-thread loads (the stress form of
// k_fused.cu and the scaled-stress form of k_adjs.cu) and the load helpers they share.
#pragma once

#include "plan.hpp"

namespace efwi {

struct AdjArgsF {
    const ShotDev *shots;
    const int4 *tiles;
    int ntiles;
    Fields in, out;             // adjoint fields
    Mat M;
    Pml pml;                    // current adjoint PML memory (V and S blocks, read)
    float *n1, *n3, *n2, *n4;   // next V block
    float *n5, *n8, *n6, *n7;   // next S block
    const float *vfx, *vfz;     // forward v^{n+1/2} (FP32), or
    SnapR sr;                   // its reduced-precision snapshot (sr.h non-null)
    float *Glam, *Gmu, *Gmuxz, *Gbx, *Gbz;
    float dt, rdx, rdz;
    // L2 prefetch of the CTA's next tile (persistent grid): tensor maps, on/off, the
    // read adjoint buffer's first field, the forward velocities' first field (-1: none)
    const AdjMaps *maps;
    int pf, acur5, sgf;
};

// Read-only load that asks L2 to fetch the 256-byte block around the address: the
// adjacent 128 bytes of a row belong to the neighbouring tile, read soon after.
// Coherent load (the imaging sums are read, then written by the same thread) with the
// same 256-byte L2 fetch.
__device__ __forceinline__ float ld256(const float *p) {
    float v;
    asm("ld.global.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ float ldg256(const float *p) {
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// The arguments of an adjoint step of plan p reading the forward velocities si.
AdjArgsF adj_args_f(efwi_plan *p, const SnapIn &si);

}  // namespace efwi
