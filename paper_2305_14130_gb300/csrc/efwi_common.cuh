// Internal definitions shared by the sm_103a translation units of libefwi_gb300.
//
// Grid layout in HBM (every shot, every field kind):
//   A shot s is modelled on its window of w_s physical columns, padded by
//   P = npml + 1 cells on every side: NX = w_s + 2P, NZ = nz + 2P.
//   Each field of shot s is a block of (NZ + 2*GZ) rows x pitch floats; cell
//   (i, j) of the padded grid sits at  off_s + (j + GZ) * pitch + (i + GX).
//   GX = 4 left ghost columns keep every row's first interior cell 16-byte
//   aligned (float4); pitch = roundup(NX, 4) + 8 leaves >= 4 zero columns on
//   the right; GZ = 2 zero rows above and below.  Ghost cells are zero and
//   never written, so the radius-2 staggered stencils need no bounds checks
//   and the discrete derivative operators are exact transposes up to sign.
//   Field kinds (vx, vz, sxx, szz, sxz, materials, adjoint fields, imaging
//   accumulators) are separate arrays sharing the per-shot offsets off_s.
//
//   Staggering (Virieux): sxx, szz, lambda, mu at (i, j); vx, b_x at
//   (i+1/2, j); vz, b_z at (i, j+1/2); sxz, mu_xz at (i+1/2, j+1/2); all four
//   positions of index (i, j) share one array offset.
//
//   CPML memory variables live only in strips of width P: x-strips are
//   NZ x 2P per shot (columns [0,P) and [NX-P,NX)), z-strips 2P x NX per shot.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "efwi.h"

// bits of a plan's device error flag (read and cleared by efwi_sync_status)
#define EFWI_FLAG_TIMEOUT 1      // a kernel gave up a bounded wait
#define EFWI_FLAG_BAD_MODEL 2    // a model value was not finite, or a density not positive

#define EFWI_GX 4
#define EFWI_GZ 2

namespace efwi {

constexpr float C1 = 9.0f / 8.0f;
constexpr float C2 = -1.0f / 24.0f;

// Per-shot geometry and source, resident in device memory.
struct ShotDev {
    int NX, NZ, pitch, x0, w;
    int P;
    long long off;      // offset (floats) of this shot's block in every field array
    long long psx;      // offset into x-strip CPML arrays (NZ * 2P per shot)
    long long psz;      // offset into z-strip CPML arrays (2P * NX per shot)
    int profx;          // offset into the x-profile arrays (NX per shot)
    int tr0, ntr;       // traces of this shot
    int inj_n[4];       // node-grid injection cells (offsets within the shot block)
    float inj_nw[4];    // bilinear weight / (dx dz)
    int inj_x[4];       // sxz-grid injection cells
    float inj_xw[4];
    float mxx, mzz, mxz;  // zero for a force source
    int inj_vx[4];      // vx-grid cells of a vector-force source (bilinear)
    float inj_vxw[4];   // bilinear weight (the 1/(dx dz) sits in the wavelet copy wv)
    int inj_vz[4];      // vz-grid cells
    float inj_vzw[4];
    float fx, fz;       // force components; zero for a moment-tensor source
};

// The five wavefield (or adjoint-wavefield) arrays.
struct Fields {
    float *vx, *vz, *sxx, *szz, *sxz;
};

// Materials per shot on the staggered positions.
struct Mat {
    const float *lam, *mu, *muxz, *bx, *bz;
};

// CPML memory variables and profiles.
//   x-strip arrays: 0 = psi1 (vx, d/dx at half), 1 = psi3 (vz, d/dx at int),
//                   2 = psi5 (nodes, d/dx vx at int), 3 = psi8 (sxz, d/dx vz at half)
//   z-strip arrays: 0 = psi2 (vx, d/dz at int), 1 = psi4 (vz, d/dz at half),
//                   2 = psi6 (nodes, d/dz vz at int), 3 = psi7 (sxz, d/dz vx at half)
struct Pml {
    float *x[4];
    float *z[4];
    const float *ax_i, *bx_i, *ax_h, *bx_h;   // per shot, length NX, offset profx
    const float *az_i, *bz_i, *az_h, *bz_h;   // length NZ (shared by all shots)
};

__device__ __forceinline__ long long cell_of(const ShotDev &s, int i, int j) {
    return s.off + (long long)(j + EFWI_GZ) * s.pitch + (i + EFWI_GX);
}

// Index in the x-strip of column i, or -1 outside the strips (also for ghosts).
__device__ __forceinline__ int xstrip(const ShotDev &s, int i) {
    if (i >= 0 && i < s.P) return i;
    if (i >= s.NX - s.P && i < s.NX) return i - s.NX + 2 * s.P;
    return -1;
}

__device__ __forceinline__ int zstrip(const ShotDev &s, int j) {
    if (j >= 0 && j < s.P) return j;
    if (j >= s.NZ - s.P && j < s.NZ) return j - s.NZ + 2 * s.P;
    return -1;
}

// 4th-order staggered differences (unscaled).
//   dfwd: value at c + 1/2 from integer-position samples  (D^+)
//   dbwd: value at c from half-position samples c - 1/2, c + 1/2  (D^-)
__device__ __forceinline__ float dfwd(const float *f, long long c, long long st) {
    return C1 * (f[c + st] - f[c]) + C2 * (f[c + 2 * st] - f[c - st]);
}
__device__ __forceinline__ float dbwd(const float *f, long long c, long long st) {
    return C1 * (f[c] - f[c - st]) + C2 * (f[c + st] - f[c - 2 * st]);
}

}  // namespace efwi
