// Plain FP32 path: one shot per launch, one kernel per half-step, one thread
// per padded cell, in-place updates (each kernel reads only fields it does
// not write).  This is the reference GPU path the batched engine is measured
// against, and it shares the exact arithmetic definitions of the batched one.
//
// Forward step n (eq. 1 as a velocity-stress system):
//   velocity  v^{n+1/2} = v^{n-1/2} + dt b (D sigma^n + psi)           (vel)
//   stress    sigma^{n+1} = sigma^n + dt C (D' v^{n+1/2} + psi)        (stress)
//             then the moment-tensor source (eq. 2) in k_misc.cu
// Adjoint step n (exact transpose, run after the DAS adjoint source):
//   adj_vel   v^ += D^T f^(sigma^, psi5..8);  b-imaging;  psi1..4 adjoint
//   adj_stress sigma^ += D^T e^(v^, psi1..4); C-imaging;  psi5..8 adjoint
#include "plan.hpp"

namespace efwi {
namespace {

struct StepArgs {
    const ShotDev *shots;
    int s0;            // shot of blockIdx.z == 0
    float *segx, *segz;   // optional copy of v^{n+1/2} (segment buffer), or null
    Fields F;
    Mat M;
    Pml pml;
    float dt, rdx, rdz;
};

__global__ void k_vel(StepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const ShotDev s = a.shots[a.s0 + blockIdx.z];
    if (i >= s.NX || j >= s.NZ) return;
    const long long c = cell_of(s, i, j);
    const long long P = s.pitch;
    float e1 = dfwd(a.F.sxx, c, 1) * a.rdx;     // d sxx / dx at (i+1/2, j)
    float e2 = dbwd(a.F.sxz, c, P) * a.rdz;     // d sxz / dz at (i+1/2, j)
    float e3 = dbwd(a.F.sxz, c, 1) * a.rdx;     // d sxz / dx at (i, j+1/2)
    float e4 = dfwd(a.F.szz, c, P) * a.rdz;     // d szz / dz at (i, j+1/2)
    const int xs = xstrip(s, i), zs = zstrip(s, j);
    if (xs >= 0) {
        const long long k = s.psx + (long long)j * 2 * s.P + xs;
        const int q = s.profx + i;
        const float p1 = a.pml.bx_h[q] * a.pml.x[0][k] + a.pml.ax_h[q] * e1;
        const float p3 = a.pml.bx_i[q] * a.pml.x[1][k] + a.pml.ax_i[q] * e3;
        a.pml.x[0][k] = p1; a.pml.x[1][k] = p3;
        e1 += p1; e3 += p3;
    }
    if (zs >= 0) {
        const long long k = s.psz + (long long)zs * s.NX + i;
        const float p2 = a.pml.bz_i[j] * a.pml.z[0][k] + a.pml.az_i[j] * e2;
        const float p4 = a.pml.bz_h[j] * a.pml.z[1][k] + a.pml.az_h[j] * e4;
        a.pml.z[0][k] = p2; a.pml.z[1][k] = p4;
        e2 += p2; e4 += p4;
    }
    const float vx = a.F.vx[c] + a.dt * a.M.bx[c] * (e1 + e2);
    const float vz = a.F.vz[c] + a.dt * a.M.bz[c] * (e3 + e4);
    a.F.vx[c] = vx;
    a.F.vz[c] = vz;
    if (a.segx) {
        a.segx[c] = vx;
        a.segz[c] = vz;
    }
}

__global__ void k_stress(StepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const ShotDev s = a.shots[a.s0 + blockIdx.z];
    if (i >= s.NX || j >= s.NZ) return;
    const long long c = cell_of(s, i, j);
    const long long P = s.pitch;
    float f1 = dbwd(a.F.vx, c, 1) * a.rdx;      // d vx / dx at (i, j)
    float f2 = dbwd(a.F.vz, c, P) * a.rdz;      // d vz / dz at (i, j)
    float f3 = dfwd(a.F.vx, c, P) * a.rdz;      // d vx / dz at (i+1/2, j+1/2)
    float f4 = dfwd(a.F.vz, c, 1) * a.rdx;      // d vz / dx at (i+1/2, j+1/2)
    const int xs = xstrip(s, i), zs = zstrip(s, j);
    if (xs >= 0) {
        const long long k = s.psx + (long long)j * 2 * s.P + xs;
        const int q = s.profx + i;
        const float p5 = a.pml.bx_i[q] * a.pml.x[2][k] + a.pml.ax_i[q] * f1;
        const float p8 = a.pml.bx_h[q] * a.pml.x[3][k] + a.pml.ax_h[q] * f4;
        a.pml.x[2][k] = p5; a.pml.x[3][k] = p8;
        f1 += p5; f4 += p8;
    }
    if (zs >= 0) {
        const long long k = s.psz + (long long)zs * s.NX + i;
        const float p6 = a.pml.bz_i[j] * a.pml.z[2][k] + a.pml.az_i[j] * f2;
        const float p7 = a.pml.bz_h[j] * a.pml.z[3][k] + a.pml.az_h[j] * f3;
        a.pml.z[2][k] = p6; a.pml.z[3][k] = p7;
        f2 += p6; f3 += p7;
    }
    const float lam = a.M.lam[c], mu2 = 2.f * a.M.mu[c];
    const float tr = lam * (f1 + f2);
    a.F.sxx[c] += a.dt * (tr + mu2 * f1);
    a.F.szz[c] += a.dt * (tr + mu2 * f2);
    a.F.sxz[c] += a.dt * a.M.muxz[c] * (f3 + f4);
}

// ---------------------------------------------------------------------------
// Adjoint kernels.  Each output cell gathers the transposed stencils; the
// quantities it gathers are recomputed from fields this kernel does not write.
// ---------------------------------------------------------------------------

struct AdjArgs {
    const ShotDev *shots;
    int s0;
    Fields A;          // adjoint fields
    Mat M;
    Pml pml;           // adjoint psi (P1..P8, same strip layout as forward)
    float *p1n, *p3n;  // next buffers of P1, P3 (x-strips)
    float *p2n, *p4n;  // next buffers of P2, P4 (z-strips)
    const float *vfx, *vfz;      // forward v^{n+1/2} (segment buffer)
    float *Glam, *Gmu, *Gmuxz, *Gbx, *Gbz;
    float dt, rdx, rdz;
};

// f^1 (conjugate of d vx/dx, P5) and f^2 (conjugate of d vz/dz, P6) at node (i, j).
__device__ __forceinline__ void fhat_node(const AdjArgs &a, const ShotDev &s, int i, int j, float &f1, float &f2) {
    const long long c = cell_of(s, i, j);
    const float sxx = a.A.sxx[c], szz = a.A.szz[c];
    const float lam = a.M.lam[c], l2m = lam + 2.f * a.M.mu[c];
    const float Ex = a.dt * (l2m * sxx + lam * szz);
    const float Ez = a.dt * (lam * sxx + l2m * szz);
    f1 = Ex; f2 = Ez;
    const int xs = xstrip(s, i), zs = zstrip(s, j);
    if (xs >= 0) {
        const long long k = s.psx + (long long)j * 2 * s.P + xs;
        f1 += a.pml.ax_i[s.profx + i] * (a.pml.x[2][k] + Ex);
    }
    if (zs >= 0) {
        const long long k = s.psz + (long long)zs * s.NX + i;
        f2 += a.pml.az_i[j] * (a.pml.z[2][k] + Ez);
    }
}

// f^3 (conjugate of d vx/dz, P7) and f^4 (conjugate of d vz/dx, P8) at sxz point (i, j).
__device__ __forceinline__ void fhat_xz(const AdjArgs &a, const ShotDev &s, int i, int j, float &f3, float &f4) {
    const long long c = cell_of(s, i, j);
    const float E = a.dt * a.M.muxz[c] * a.A.sxz[c];
    f3 = E; f4 = E;
    const int xs = xstrip(s, i), zs = zstrip(s, j);
    if (zs >= 0) {
        const long long k = s.psz + (long long)zs * s.NX + i;
        f3 += a.pml.az_h[j] * (a.pml.z[3][k] + E);
    }
    if (xs >= 0) {
        const long long k = s.psx + (long long)j * 2 * s.P + xs;
        f4 += a.pml.ax_h[s.profx + i] * (a.pml.x[3][k] + E);
    }
}

__global__ void k_adj_vel(AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const ShotDev s = a.shots[a.s0 + blockIdx.z];
    if (i >= s.NX || j >= s.NZ) return;
    const long long c = cell_of(s, i, j);
    // f^ on the stencil of vx at (i+1/2, j): nodes i-1..i+2 (row j); sxz points j-2..j+1 (column i)
    float n1[4], n2[4], x3[4], x4[4], d;
    for (int k = 0; k < 4; ++k) fhat_node(a, s, i - 1 + k, j, n1[k], d);
    for (int k = 0; k < 4; ++k) fhat_xz(a, s, i, j - 2 + k, x3[k], d);
    const float inc_x = -(C1 * (n1[2] - n1[1]) + C2 * (n1[3] - n1[0])) * a.rdx
                        - (C1 * (x3[2] - x3[1]) + C2 * (x3[3] - x3[0])) * a.rdz;
    // f^ on the stencil of vz at (i, j+1/2): nodes j-1..j+2 (column i); sxz points i-2..i+1 (row j)
    for (int k = 0; k < 4; ++k) fhat_node(a, s, i, j - 1 + k, d, n2[k]);
    for (int k = 0; k < 4; ++k) fhat_xz(a, s, i - 2 + k, j, d, x4[k]);
    const float inc_z = -(C1 * (n2[2] - n2[1]) + C2 * (n2[3] - n2[0])) * a.rdz
                        - (C1 * (x4[2] - x4[1]) + C2 * (x4[3] - x4[0])) * a.rdx;
    const float vx = a.A.vx[c] + inc_x;
    const float vz = a.A.vz[c] + inc_z;
    a.A.vx[c] = vx;
    a.A.vz[c] = vz;
    // b-imaging: sum_n v^{n+1/2} * (increment of the adjoint of v^{n+1/2}) over the
    // positions whose buoyancy depends on a physical node
    if (i >= s.P - 1 && i <= s.P + s.w && j >= s.P - 1 && j <= s.NZ - s.P) {
        a.Gbx[c] += a.vfx[c] * inc_x;
        a.Gbz[c] += a.vfz[c] * inc_z;
    }
    // CPML memory of the velocity sub-step, transposed (written to the next buffer)
    const float qx = a.dt * a.M.bx[c] * vx, qz = a.dt * a.M.bz[c] * vz;
    const int xs = xstrip(s, i), zs = zstrip(s, j);
    if (xs >= 0) {
        const long long k = s.psx + (long long)j * 2 * s.P + xs;
        const int q = s.profx + i;
        a.p1n[k] = a.pml.bx_h[q] * (a.pml.x[0][k] + qx);
        a.p3n[k] = a.pml.bx_i[q] * (a.pml.x[1][k] + qz);
    }
    if (zs >= 0) {
        const long long k = s.psz + (long long)zs * s.NX + i;
        a.p2n[k] = a.pml.bz_i[j] * (a.pml.z[0][k] + qx);
        a.p4n[k] = a.pml.bz_h[j] * (a.pml.z[1][k] + qz);
    }
}

// e^ at a vx point: e^1 (conjugate of d sxx/dx, P1), e^2 (conjugate of d sxz/dz, P2)
__device__ __forceinline__ void ehat_vx(const AdjArgs &a, const ShotDev &s, int i, int j, float &e1, float &e2) {
    const long long c = cell_of(s, i, j);
    const float q = a.dt * a.M.bx[c] * a.A.vx[c];
    e1 = q; e2 = q;
    const int xs = xstrip(s, i), zs = zstrip(s, j);
    if (xs >= 0) {
        const long long k = s.psx + (long long)j * 2 * s.P + xs;
        e1 += a.pml.ax_h[s.profx + i] * (a.pml.x[0][k] + q);
    }
    if (zs >= 0) {
        const long long k = s.psz + (long long)zs * s.NX + i;
        e2 += a.pml.az_i[j] * (a.pml.z[0][k] + q);
    }
}

// e^ at a vz point: e^3 (conjugate of d sxz/dx, P3), e^4 (conjugate of d szz/dz, P4)
__device__ __forceinline__ void ehat_vz(const AdjArgs &a, const ShotDev &s, int i, int j, float &e3, float &e4) {
    const long long c = cell_of(s, i, j);
    const float q = a.dt * a.M.bz[c] * a.A.vz[c];
    e3 = q; e4 = q;
    const int xs = xstrip(s, i), zs = zstrip(s, j);
    if (xs >= 0) {
        const long long k = s.psx + (long long)j * 2 * s.P + xs;
        e3 += a.pml.ax_i[s.profx + i] * (a.pml.x[1][k] + q);
    }
    if (zs >= 0) {
        const long long k = s.psz + (long long)zs * s.NX + i;
        e4 += a.pml.az_h[j] * (a.pml.z[1][k] + q);
    }
}

__global__ void k_adj_stress(AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const ShotDev s = a.shots[a.s0 + blockIdx.z];
    if (i >= s.NX || j >= s.NZ) return;
    const long long c = cell_of(s, i, j);
    const long long P = s.pitch;
    const float sxx = a.A.sxx[c], szz = a.A.szz[c], sxz = a.A.sxz[c];
    const float lam = a.M.lam[c], mu = a.M.mu[c], l2m = lam + 2.f * mu;
    // CPML memory of the stress sub-step, transposed (in place: read by k_adj_vel only)
    const int xs = xstrip(s, i), zs = zstrip(s, j);
    const float Ex = a.dt * (l2m * sxx + lam * szz);
    const float Ez = a.dt * (lam * sxx + l2m * szz);
    const float Exz = a.dt * a.M.muxz[c] * sxz;
    if (xs >= 0) {
        const long long k = s.psx + (long long)j * 2 * s.P + xs;
        const int q = s.profx + i;
        a.pml.x[2][k] = a.pml.bx_i[q] * (a.pml.x[2][k] + Ex);
        a.pml.x[3][k] = a.pml.bx_h[q] * (a.pml.x[3][k] + Exz);
    }
    if (zs >= 0) {
        const long long k = s.psz + (long long)zs * s.NX + i;
        a.pml.z[2][k] = a.pml.bz_i[j] * (a.pml.z[2][k] + Ez);
        a.pml.z[3][k] = a.pml.bz_h[j] * (a.pml.z[3][k] + Exz);
    }
    // C-imaging: zero-lag products of sigma^ (adjoint of sigma^{n+1}) with the forward
    // strain rates of step n; the PML memory is zero on these positions
    if (i >= s.P && i < s.P + s.w && j >= s.P && j < s.NZ - s.P) {
        const float fx = dbwd(a.vfx, c, 1) * a.rdx;
        const float fz = dbwd(a.vfz, c, P) * a.rdz;
        a.Glam[c] += a.dt * (sxx + szz) * (fx + fz);
        a.Gmu[c] += 2.f * a.dt * (sxx * fx + szz * fz);
    }
    if (i >= s.P - 1 && i < s.P + s.w && j >= s.P - 1 && j < s.NZ - s.P) {
        const float fxz = dfwd(a.vfx, c, P) * a.rdz + dfwd(a.vfz, c, 1) * a.rdx;
        a.Gmuxz[c] += a.dt * sxz * fxz;
    }
    // sigma^ += D^T e^ :  sxx from e^1 at vx points i-2..i+1 (row j);
    // szz from e^4 at vz points j-2..j+1 (column i);
    // sxz from e^2 at vx points j-1..j+2 (column i) and e^3 at vz points i-1..i+2 (row j)
    float e1[4], e2[4], e3[4], e4[4], d;
    for (int k = 0; k < 4; ++k) ehat_vx(a, s, i - 2 + k, j, e1[k], d);
    for (int k = 0; k < 4; ++k) ehat_vz(a, s, i, j - 2 + k, d, e4[k]);
    for (int k = 0; k < 4; ++k) ehat_vx(a, s, i, j - 1 + k, d, e2[k]);
    for (int k = 0; k < 4; ++k) ehat_vz(a, s, i - 1 + k, j, e3[k], d);
    a.A.sxx[c] = sxx - (C1 * (e1[2] - e1[1]) + C2 * (e1[3] - e1[0])) * a.rdx;
    a.A.szz[c] = szz - (C1 * (e4[2] - e4[1]) + C2 * (e4[3] - e4[0])) * a.rdz;
    a.A.sxz[c] = sxz - (C1 * (e2[2] - e2[1]) + C2 * (e2[3] - e2[0])) * a.rdz
                     - (C1 * (e3[2] - e3[1]) + C2 * (e3[3] - e3[0])) * a.rdx;
}

StepArgs step_args(efwi_plan *p, int shot, float *segx, float *segz) {
    StepArgs a;
    a.shots = p->shots_d;
    a.s0 = shot < 0 ? 0 : shot;
    a.segx = segx;
    a.segz = segz;
    a.F = state_fields(p, p->scur);
    a.M = materials(p);
    a.pml = fwd_pml(p, p->psi_v, p->psi_s);
    a.dt = (float)p->d.dt;
    a.rdx = (float)(1.0 / p->d.dx);
    a.rdz = (float)(1.0 / p->d.dz);
    return a;
}

AdjArgs adj_args(efwi_plan *p, int shot, const float *vfx, const float *vfz) {
    AdjArgs a;
    a.shots = p->shots_d;
    a.s0 = shot < 0 ? 0 : shot;
    a.A = adj_fields(p, p->acur);
    a.M = materials(p);
    a.pml = adj_pml(p, p->apsi_v, p->apsi_s);
    // next buffer of the velocity-sub-step adjoint memory P1..P4
    float *vn = psi_block(p->apsi, p, 1 - p->apsi_v);
    a.p1n = vn;
    a.p3n = vn + p->psx_total;
    a.p2n = vn + 2 * p->psx_total;
    a.p4n = vn + 2 * p->psx_total + p->psz_total;
    a.vfx = vfx; a.vfz = vfz;
    a.Glam = G_field(p, 0); a.Gmu = G_field(p, 1); a.Gmuxz = G_field(p, 2);
    a.Gbx = G_field(p, 3); a.Gbz = G_field(p, 4);
    a.dt = (float)p->d.dt;
    a.rdx = (float)(1.0 / p->d.dx);
    a.rdz = (float)(1.0 / p->d.dz);
    return a;
}

// One shot (shot >= 0) or every shot along grid.z (shot < 0, sized to the widest window).
dim3 grid_of(efwi_plan *p, int shot, dim3 b) {
    const int nx = shot >= 0 ? p->shots[shot].NX : p->max_nx;
    return dim3((nx + b.x - 1) / b.x, (p->nzp + b.y - 1) / b.y, shot >= 0 ? 1 : p->d.ns);
}

}  // namespace

void launch_vel_plain(efwi_plan *p, int shot, float *segx, float *segz, cudaStream_t st) {
    StepArgs a = step_args(p, shot, segx, segz);
    dim3 b(32, 8);
    k_vel<<<grid_of(p, shot, b), b, 0, st>>>(a);
    p->launches++;
}

void launch_stress_plain(efwi_plan *p, int shot, cudaStream_t st) {
    StepArgs a = step_args(p, shot, nullptr, nullptr);
    dim3 b(32, 8);
    int slot;
    prof_begin(p, st, &slot, EFWI_KERNEL_STEP);
    k_stress<<<grid_of(p, shot, b), b, 0, st>>>(a);
    prof_end(p, st, slot);
    p->launches++;
}

void launch_adj_vel_plain(efwi_plan *p, int shot, const float *vfx, const float *vfz, cudaStream_t st) {
    AdjArgs a = adj_args(p, shot, vfx, vfz);
    dim3 b(32, 8);
    k_adj_vel<<<grid_of(p, shot, b), b, 0, st>>>(a);
    p->launches++;
}

void launch_adj_stress_plain(efwi_plan *p, int shot, const float *vfx, const float *vfz, cudaStream_t st) {
    AdjArgs a = adj_args(p, shot, vfx, vfz);
    dim3 b(32, 8);
    int slot;
    prof_begin(p, st, &slot, EFWI_KERNEL_ADJ);
    k_adj_stress<<<grid_of(p, shot, b), b, 0, st>>>(a);
    prof_end(p, st, slot);
    p->launches++;
}

}  // namespace efwi
