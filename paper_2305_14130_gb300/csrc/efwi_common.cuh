// Internal definitions shared by the sm_103a translation units of libefwi_gb300.
//
// Grid layout in HBM (every shot, every field kind):
//   A shot s is modelled on its window of w_s physical columns, padded by
//   P = npml + 1 cells on every side: NX = w_s + 2P, NZ = nz + 2P.
//   Each field of shot s is a block of (NZ + 2*GZ) rows x pitch floats; cell
//   (i, j) of the padded grid sits at  off_s + (j + GZ) * pitch + (i + GX).
//   GX = 4 left ghost columns keep every row's first interior cell 16-byte
//   aligned (float4); pitch = roundup(NX, 8) + 8 leaves >= 4 zero columns on
//   the right and keeps rows of 2-byte snapshot elements 16-byte aligned too
//   (tensor copies); GZ = 2 zero rows above and below.  Ghost cells are zero and
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
#define EFWI_FLAG_SELFTEST 4     // the timeout self-test's wait expired (as intended)
#define EFWI_FLAG_SHEAR 8        // a gradient call met mu <= 0 (or lambda + mu <= 0, scaled-stress adjoint)

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

// Reduced-precision storage of a wavefield snapshot (checkpoints and stored
// forward velocities): with s = max |x| over the snapshot, every element is
// stored as RNE(x * 2^k), k chosen from the exponent of s so that s * 2^k lies in
// [2^14, 2^15) (clamped to |k| <= 126 for extreme s), and read back as y * 2^-k.
// Both multiplications by a power of two are exact, so the only error is the
// rounding to the storage type, and magnitudes down to s * 2^-28 stay normal FP16
// numbers (relative error <= 2^-11; BF16: 2^-8).
__device__ __forceinline__ int store_exp(float s) {
    const int E = (__float_as_int(fabsf(s)) >> 23) & 0xff;   // biased exponent of s (0 for s = 0)
    const int k = 141 - E;                                    // 15 - e with s = m 2^e, m in [0.5, 1)
    return k < -126 ? -126 : (k > 126 ? 126 : k);
}
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }   // |k| <= 126

template <class T>
__device__ __forceinline__ T to_store(float v);
template <>
__device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from_store(__half v) { return __half2float(v); }
__device__ __forceinline__ float from_store(__nv_bfloat16 v) { return __bfloat162float(v); }

// Forward velocities v^{n+1/2} kept for the adjoint in FP16 / BF16 ("snapshots").
// The step that computes v^{n+1/2} accumulates max |vx| and max |vz| of every shot
// (atomicMax on the float bits after a per-tile reduction); the maxima are complete
// when that launch ends, so the NEXT step, which stages v^{n+1/2} in shared memory
// anyway, writes the scaled 2-byte copy of its own tile cells (a separate small
// kernel packs the last step of a pass).  Maxima of one snapshot: [2][ns] floats,
// each in its own 128-byte line (kMaxPad floats apart) so the atomics of different
// shots and fields do not serialise on one line.
constexpr int kMaxPad = 32;

struct SnapW {                 // reduced-precision snapshot work of one forward step
    void *h;                   // copy of the previous step's v: vx at [F], vz at [F + F]; null = none
    const float *hmax;         // maxima of that previous step's snapshot
    float *amax;               // maxima accumulator of this step's snapshot, or null
    long long F;               // elements per field (fsz_total)
    int ns, kind;              // shots; EFWI_STORE_FP16 or EFWI_STORE_BF16
};

struct SnapR {                 // reduced-precision forward velocities read by an adjoint step
    const void *h;             // vx at [0, F), vz at [F, 2F); null = FP32 velocities
    const float *hmax;
    long long F;
    int ns, kind;
};

__device__ __forceinline__ float snap_scale_up(const float *mx, int f, int shot, int ns) {
    return pow2f(store_exp(__ldg(mx + (long long)(f * ns + shot) * kMaxPad)));
}
__device__ __forceinline__ float snap_scale_down(const float *mx, int f, int shot, int ns) {
    return pow2f(-store_exp(__ldg(mx + (long long)(f * ns + shot) * kMaxPad)));
}

// two adjacent elements (idx even, 4-byte aligned) / one element of a 2-byte snapshot;
// SK = EFWI_STORE_FP16 or EFWI_STORE_BF16 (compile time in the stencil kernels)
template <int SK>
__device__ __forceinline__ void snap_put2(void *h, long long idx, float a, float b) {
    if constexpr (SK == EFWI_STORE_FP16)
        *reinterpret_cast<__half2 *>(static_cast<__half *>(h) + idx) = __floats2half2_rn(a, b);
    else
        *reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(h) + idx) = __floats2bfloat162_rn(a, b);
}
template <int SK>
__device__ __forceinline__ void snap_put1(void *h, long long idx, float a) {
    if constexpr (SK == EFWI_STORE_FP16) static_cast<__half *>(h)[idx] = __float2half_rn(a);
    else static_cast<__nv_bfloat16 *>(h)[idx] = __float2bfloat16_rn(a);
}
// read-only 2-byte load asking L2 for the 256-byte block around it (the neighbouring
// tile reads the rest of the block soon after), widened exactly to FP32
template <int SK>
__device__ __forceinline__ float snap_get(const void *h, long long idx) {
    unsigned short u;
    asm("ld.global.nc.L2::256B.b16 %0, [%1];"
        : "=h"(u)
        : "l"(static_cast<const unsigned short *>(h) + idx));
    if constexpr (SK == EFWI_STORE_FP16) return __half2float(__ushort_as_half(u));
    else return __bfloat162float(__ushort_as_bfloat16(u));
}
__device__ __forceinline__ float snap_get_rt(const void *h, long long idx, int kind) {
    return kind == EFWI_STORE_FP16 ? snap_get<EFWI_STORE_FP16>(h, idx) : snap_get<EFWI_STORE_BF16>(h, idx);
}

// Per-tile maximum of |v| for the snapshot scale: every thread passes its running
// maxima (non-negative), each warp reduces them, and lane 0 leaves them in wsm
// ([2][warps]); after the next __syncthreads snap_max_commit folds the warps and
// issues one atomicMax per field.  Must be called by every thread of the block.
__device__ __forceinline__ void snap_max_warp(float mx, float mz, unsigned *wsm) {
    const unsigned ux = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
    const unsigned uz = __reduce_max_sync(0xffffffffu, __float_as_uint(mz));
    if ((threadIdx.x & 31) == 0) {
        wsm[threadIdx.x >> 5] = ux;
        wsm[(blockDim.x >> 5) + (threadIdx.x >> 5)] = uz;
    }
}
__device__ __forceinline__ void snap_max_commit(const unsigned *wsm, float *amax, int shot, int ns) {
    const int nw = blockDim.x >> 5;
    unsigned ux = 0, uz = 0;
    for (int w = 0; w < nw; ++w) {
        ux = max(ux, wsm[w]);
        uz = max(uz, wsm[nw + w]);
    }
    atomicMax(reinterpret_cast<unsigned *>(amax + (long long)shot * kMaxPad), ux);
    atomicMax(reinterpret_cast<unsigned *>(amax + (long long)(ns + shot) * kMaxPad), uz);
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
