// Batched execution: one fused launch per time step for every shot (any
// window width), over a flat list of (shot, tile) work items.
//
// Forward step (k_step_fused), per TX x TZ tile of one shot:
//   1. stage sigma^n of the tile + 4-cell halo in shared memory (float4 loads);
//   2. v^{n+1/2} = v^{n-1/2} + dt b (D sigma^n + psi) on the tile + 2-cell halo
//      (the halo is recomputed by each neighbour, so no grid-wide barrier is
//      needed between the two half-steps), kept in shared memory;
//   3. sigma^{n+1} = sigma^n + dt C (D' v^{n+1/2} + psi) - M dw delta_h on the tile.
// The state is read from buffer scur and written to the other buffer; the
// CPML memory of the velocity sub-step (read in halos) is double-buffered too.
//
// Adjoint step (k_adj_fused), the exact transpose with the same staging:
//   1. f^ = (C sigma^ + PML) of the tile + 4-cell halo in shared memory; the
//      stress-sub-step adjoint PML memory of the tile advances;
//   2. v^ += D^T f^ on the tile + 2-cell halo, then e^ = (dt b v^ + PML) kept in
//      shared memory; b-imaging and velocity adjoint PML memory on the tile;
//   3. sigma^ += D^T e^ on the tile with the C-imaging (zero-lag products with
//      the forward strain rates of step n).
// Every per-cell expression matches the plain kernels term by term.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <type_traits>
#include <vector>

#include "plan.hpp"
#include "tma.cuh"
#include "adj_args.cuh"

namespace efwi {
namespace {

constexpr int kThreads = 256;

struct FwdArgs {
    const ShotDev *shots;
    const int4 *tiles;
    int ntiles;
    Fields in, out;
    Mat M;
    Pml pml;                    // V block = current (read), S block = in place
    float *n1, *n3, *n2, *n4;   // next V block: psi1, psi3 (x-strips), psi2, psi4 (z-strips)
    float *segx, *segz;         // optional copy of v^{n+1/2}
    const float *dw;
    const float *wv;            // w_n / (dx dz) of force sources (null without)
    int nt, n;
    float dt, rdx, rdz;
    SnapW sw;                   // reduced-precision snapshot work (sw.h / sw.amax null: none)
};

template <int TX, int TZ, int SK = 0>
__global__ void __launch_bounds__(kThreads) k_step_fused(FwdArgs a) {
    constexpr bool SNAP = SK != 0;   // FP16 / BF16 snapshot work compiled in
    constexpr int SX = TX + 8, SZ = TZ + 8;     // sigma staging: tile + 4 halo
    constexpr int VX = TX + 4, VZ = TZ + 4;     // velocity: tile + 2 halo
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *sxx = sm, *szz = sm + SX * SZ, *sxz = sm + 2 * SX * SZ;
    float *svx = sm + 3 * SX * SZ, *svz = svx + VX * VZ;
    __shared__ unsigned wmax_s[2 * (kThreads / 32)];   // per-warp snapshot maxima of a tile
    const int tid = threadIdx.x;

    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 tl = a.tiles[t];
        const ShotDev *sp = a.shots + tl.x;
        const int NX = sp->NX, NZ = sp->NZ, PP = sp->P, profx = sp->profx, pitch = sp->pitch;
        const long long off = sp->off, psx = sp->psx, psz = sp->psz;
        const bool edge = (tl.w & 2) != 0;
        const int i0 = tl.y, j0 = tl.z;
        const int rowlim = pitch - EFWI_GX;
        const float dt = a.dt, rdx = a.rdx, rdz = a.rdz;
        // scales of the previous step's snapshot (written for the tile's own cells) and
        // this thread's max |v^{n+1/2}| for the scale of this step's
        const float upx = SNAP && a.sw.h ? snap_scale_up(a.sw.hmax, 0, tl.x, a.sw.ns) : 1.f;
        const float upz = SNAP && a.sw.h ? snap_scale_up(a.sw.hmax, 1, tl.x, a.sw.ns) : 1.f;
        float mxv = 0.f, mzv = 0.f;

        // 1. sigma^n with a 4-cell halo (zero outside the padded grid)
        constexpr int Q4 = SX / 4;
#pragma unroll 4
        for (int q = tid; q < 3 * SZ * Q4; q += kThreads) {
            const int f = q / (SZ * Q4), r = q - f * SZ * Q4;
            const int y = r / Q4, x4 = r - y * Q4;
            const int i = i0 - 4 + 4 * x4, j = j0 - 4 + y;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j >= 0 && j < NZ && i + 4 <= rowlim) {
                const float *src = f == 0 ? a.in.sxx : (f == 1 ? a.in.szz : a.in.sxz);
                v = __ldg(reinterpret_cast<const float4 *>(src + off + (j + EFWI_GZ) * pitch + (i + EFWI_GX)));
            }
            reinterpret_cast<float4 *>(sm + f * SX * SZ + y * SX)[x4] = v;
        }
        __syncthreads();

        // 2. v^{n+1/2} on the tile + 2-cell halo
        for (int q = tid; q < VX * VZ; q += kThreads) {
            const int y = q / VX, x = q - y * VX;
            const int i = i0 - 2 + x, j = j0 - 2 + y;
            float vx = 0.f, vz = 0.f;
            if (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ)) {
                const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                const int o = (y + 2) * SX + (x + 2);       // (i, j) in sigma staging
                float e1 = (C1 * (sxx[o + 1] - sxx[o]) + C2 * (sxx[o + 2] - sxx[o - 1])) * rdx;
                float e2 = (C1 * (sxz[o] - sxz[o - SX]) + C2 * (sxz[o + SX] - sxz[o - 2 * SX])) * rdz;
                float e3 = (C1 * (sxz[o] - sxz[o - 1]) + C2 * (sxz[o + 1] - sxz[o - 2])) * rdx;
                float e4 = (C1 * (szz[o + SX] - szz[o]) + C2 * (szz[o + 2 * SX] - szz[o - SX])) * rdz;
                const bool own = x >= 2 && x < TX + 2 && y >= 2 && y < TZ + 2;
                if (edge) {
                    const int xs = i < PP ? i : (i >= NX - PP ? i - NX + 2 * PP : -1);
                    const int zs = j < PP ? j : (j >= NZ - PP ? j - NZ + 2 * PP : -1);
                    if (xs >= 0) {
                        const long long k = psx + (long long)j * 2 * PP + xs;
                        const int pq = profx + i;
                        const float p1 = a.pml.bx_h[pq] * a.pml.x[0][k] + a.pml.ax_h[pq] * e1;
                        const float p3 = a.pml.bx_i[pq] * a.pml.x[1][k] + a.pml.ax_i[pq] * e3;
                        if (own) { a.n1[k] = p1; a.n3[k] = p3; }
                        e1 += p1; e3 += p3;
                    }
                    if (zs >= 0) {
                        const long long k = psz + (long long)zs * NX + i;
                        const float p2 = a.pml.bz_i[j] * a.pml.z[0][k] + a.pml.az_i[j] * e2;
                        const float p4 = a.pml.bz_h[j] * a.pml.z[1][k] + a.pml.az_h[j] * e4;
                        if (own) { a.n2[k] = p2; a.n4[k] = p4; }
                        e2 += p2; e4 += p4;
                    }
                }
                const float vxo = __ldg(a.in.vx + c), vzo = __ldg(a.in.vz + c);
                vx = vxo + dt * __ldg(a.M.bx + c) * (e1 + e2);
                vz = vzo + dt * __ldg(a.M.bz + c) * (e3 + e4);
                if (tl.w & 8) {                      // vector force of this shot (k_force's expression)
                    const int lc = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    const float wvn = a.wv[(long long)tl.x * a.nt + a.n];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (lc == sp->inj_vx[k]) vx = vx + dt * __ldg(a.M.bx + c) * (sp->fx * wvn * sp->inj_vxw[k]);
                        if (lc == sp->inj_vz[k]) vz = vz + dt * __ldg(a.M.bz + c) * (sp->fz * wvn * sp->inj_vzw[k]);
                    }
                }
                if (own && (!edge || (i < NX && j < NZ))) {
                    a.out.vx[c] = vx;
                    a.out.vz[c] = vz;
                    if (a.segx) { a.segx[c] = vx; a.segz[c] = vz; }
                    if (SNAP && a.sw.h) {            // snapshot of v^{n-1/2}
                        snap_put1<SK>(a.sw.h, c, vxo * upx);
                        snap_put1<SK>(a.sw.h, a.sw.F + c, vzo * upz);
                    }
                    mxv = fmaxf(mxv, fabsf(vx));
                    mzv = fmaxf(mzv, fabsf(vz));
                }
            }
            svx[q] = vx;
            svz[q] = vz;
        }
        if (SNAP && a.sw.amax) snap_max_warp(mxv, mzv, wmax_s);
        __syncthreads();
        if (SNAP && a.sw.amax && tid == 32) snap_max_commit(wmax_s, a.sw.amax, tl.x, a.sw.ns);

        // 3. sigma^{n+1} on the tile, then the moment-tensor source
        const bool inj = (tl.w & 1) != 0;
        const float dwn = inj ? a.dw[(long long)tl.x * a.nt + a.n] : 0.f;
        for (int q = tid; q < TX * TZ; q += kThreads) {
            const int y = q / TX, x = q - y * TX;
            const int i = i0 + x, j = j0 + y;
            if (edge && (i >= NX || j >= NZ)) continue;
            const int lc = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
            const long long c = off + lc;
            const int o = (y + 2) * VX + (x + 2);           // (i, j) in velocity staging
            float f1 = (C1 * (svx[o] - svx[o - 1]) + C2 * (svx[o + 1] - svx[o - 2])) * rdx;
            float f2 = (C1 * (svz[o] - svz[o - VX]) + C2 * (svz[o + VX] - svz[o - 2 * VX])) * rdz;
            float f3 = (C1 * (svx[o + VX] - svx[o]) + C2 * (svx[o + 2 * VX] - svx[o - VX])) * rdz;
            float f4 = (C1 * (svz[o + 1] - svz[o]) + C2 * (svz[o + 2] - svz[o - 1])) * rdx;
            if (edge) {
                const int xs = i < PP ? i : (i >= NX - PP ? i - NX + 2 * PP : -1);
                const int zs = j < PP ? j : (j >= NZ - PP ? j - NZ + 2 * PP : -1);
                if (xs >= 0) {
                    const long long k = psx + (long long)j * 2 * PP + xs;
                    const int pq = profx + i;
                    const float p5 = a.pml.bx_i[pq] * a.pml.x[2][k] + a.pml.ax_i[pq] * f1;
                    const float p8 = a.pml.bx_h[pq] * a.pml.x[3][k] + a.pml.ax_h[pq] * f4;
                    a.pml.x[2][k] = p5; a.pml.x[3][k] = p8;
                    f1 += p5; f4 += p8;
                }
                if (zs >= 0) {
                    const long long k = psz + (long long)zs * NX + i;
                    const float p6 = a.pml.bz_i[j] * a.pml.z[2][k] + a.pml.az_i[j] * f2;
                    const float p7 = a.pml.bz_h[j] * a.pml.z[3][k] + a.pml.az_h[j] * f3;
                    a.pml.z[2][k] = p6; a.pml.z[3][k] = p7;
                    f2 += p6; f3 += p7;
                }
            }
            const int os = (y + 4) * SX + (x + 4);          // (i, j) in sigma staging
            const float lam = __ldg(a.M.lam + c), mu2 = 2.f * __ldg(a.M.mu + c);
            const float tr = lam * (f1 + f2);
            float nxx = sxx[os] + dt * (tr + mu2 * f1);
            float nzz = szz[os] + dt * (tr + mu2 * f2);
            float nxz = sxz[os] + dt * __ldg(a.M.muxz + c) * (f3 + f4);
            if (inj) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (lc == sp->inj_n[k]) {
                        nxx -= sp->mxx * dwn * sp->inj_nw[k];
                        nzz -= sp->mzz * dwn * sp->inj_nw[k];
                    }
                    if (lc == sp->inj_x[k]) nxz -= sp->mxz * dwn * sp->inj_xw[k];
                }
            }
            a.out.sxx[c] = nxx;
            a.out.szz[c] = nzz;
            a.out.sxz[c] = nxz;
        }
        __syncthreads();
    }
}

template <int TX, int TZ, int SK = 0>
__global__ void __launch_bounds__(kThreads, TX * TZ <= 512 ? 4 : 2) k_adj_fused(AdjArgsF a) {
    // SK: the forward velocities are FP32 (0) or FP16 / BF16 snapshots
    constexpr int SX = TX + 8, SZ = TZ + 8;
    constexpr int VX = TX + 4, VZ = TZ + 4;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *f1s = sm, *f2s = sm + SX * SZ, *f3s = sm + 2 * SX * SZ, *f4s = sm + 3 * SX * SZ;
    float *e1s = sm + 4 * SX * SZ, *e2s = e1s + VX * VZ, *e3s = e2s + VX * VZ, *e4s = e3s + VX * VZ;
    float *vfxs = e4s + VX * VZ, *vfzs = vfxs + VX * VZ;   // forward v^{n+1/2} on the tile + 2-cell halo
    const int tid = threadIdx.x;

    // With a persistent grid (fewer CTAs than tiles) the next tile's work item, and
    // the block offset and row pitch of its shot, are loaded one tile ahead, so an
    // interior tile issues its first global loads without a dependent load in front.
    int4 tl_next = blockIdx.x < a.ntiles ? __ldg(a.tiles + blockIdx.x) : make_int4(0, 0, 0, 0);
    long long off_next = __ldg(&a.shots[tl_next.x].off);
    int pitch_next = __ldg(&a.shots[tl_next.x].pitch);
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 tl = tl_next;
        const long long off = off_next;
        const int pitch = pitch_next;
        if (t + gridDim.x < a.ntiles) {
            tl_next = __ldg(a.tiles + t + gridDim.x);
            off_next = __ldg(&a.shots[tl_next.x].off);
            pitch_next = __ldg(&a.shots[tl_next.x].pitch);
        }
        // interior tiles (no CPML strip or grid edge within the 4-cell halo) run a
        // copy of the body without any of the edge tests
        auto tile = [&](auto edge_c) {
            const ShotDev *sp = a.shots + tl.x;
            const int NX = sp->NX, NZ = sp->NZ, PP = sp->P, profx = sp->profx, w = sp->w;
            const long long psx = sp->psx, psz = sp->psz;
            constexpr bool edge = decltype(edge_c)::value;   // 4-cell halo touches a strip or the grid edge
            const int i0 = tl.y, j0 = tl.z;
            const float dt = a.dt, rdx = a.rdx, rdz = a.rdz;
            const float dnx = SK ? snap_scale_down(a.sr.hmax, 0, tl.x, a.sr.ns) : 1.f;
            const float dnz = SK ? snap_scale_down(a.sr.hmax, 1, tl.x, a.sr.ns) : 1.f;

            // Each phase first issues every global load of the thread's cells into
            // registers (no store in between, so all are in flight together), then
            // computes; each cell's arithmetic is unchanged.
            // 1. f^ on the tile + 4-cell halo; the tile's stress-sub-step PML memory advances
            constexpr int N1 = (SX * SZ + kThreads - 1) / kThreads;
            float lxx[N1], lzz[N1], lxz[N1], llam[N1], lmu[N1], lmxz[N1];
#pragma unroll
            for (int r = 0; r < N1; ++r) {
                const int q = tid + r * kThreads;
                lxx[r] = lzz[r] = lxz[r] = llam[r] = lmu[r] = lmxz[r] = 0.f;
                const int y = q / SX, x = q - y * SX;
                const int i = i0 - 4 + x, j = j0 - 4 + y;
                if (q < SX * SZ && (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ))) {
                    const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    lxx[r] = ldg256(a.in.sxx + c); lzz[r] = ldg256(a.in.szz + c); lxz[r] = ldg256(a.in.sxz + c);
                    llam[r] = ldg256(a.M.lam + c); lmu[r] = ldg256(a.M.mu + c); lmxz[r] = ldg256(a.M.muxz + c);
                }
            }
#pragma unroll
            for (int r = 0; r < N1; ++r) {
                const int q = tid + r * kThreads;
                if (q >= SX * SZ) break;
                const int y = q / SX, x = q - y * SX;
                const int i = i0 - 4 + x, j = j0 - 4 + y;
                float g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f;
                if (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ)) {
                    const float hxx = lxx[r], hzz = lzz[r], hxz = lxz[r];
                    const float lam = llam[r], l2m = lam + 2.f * lmu[r];
                    const float Ex = dt * (l2m * hxx + lam * hzz);
                    const float Ez = dt * (lam * hxx + l2m * hzz);
                    const float Exz = dt * lmxz[r] * hxz;
                    g1 = Ex; g2 = Ez; g3 = Exz; g4 = Exz;
                    if (edge) {
                        const bool own = x >= 4 && x < TX + 4 && y >= 4 && y < TZ + 4;
                        const int xs = i < PP ? i : (i >= NX - PP ? i - NX + 2 * PP : -1);
                        const int zs = j < PP ? j : (j >= NZ - PP ? j - NZ + 2 * PP : -1);
                        if (xs >= 0) {
                            const long long k = psx + (long long)j * 2 * PP + xs;
                            const int pq = profx + i;
                            const float P5 = a.pml.x[2][k], P8 = a.pml.x[3][k];
                            g1 += a.pml.ax_i[pq] * (P5 + Ex);
                            g4 += a.pml.ax_h[pq] * (P8 + Exz);
                            if (own) {
                                a.n5[k] = a.pml.bx_i[pq] * (P5 + Ex);
                                a.n8[k] = a.pml.bx_h[pq] * (P8 + Exz);
                            }
                        }
                        if (zs >= 0) {
                            const long long k = psz + (long long)zs * NX + i;
                            const float P6 = a.pml.z[2][k], P7 = a.pml.z[3][k];
                            g2 += a.pml.az_i[j] * (P6 + Ez);
                            g3 += a.pml.az_h[j] * (P7 + Exz);
                            if (own) {
                                a.n6[k] = a.pml.bz_i[j] * (P6 + Ez);
                                a.n7[k] = a.pml.bz_h[j] * (P7 + Exz);
                            }
                        }
                    }
                }
                f1s[q] = g1; f2s[q] = g2; f3s[q] = g3;
                if (edge) f4s[q] = g4;                     // f^4 == f^3 away from the CPML
            }
            if (a.pf && tid == 0 && t + (int)gridDim.x < a.ntiles) {
                // the next tile's inputs into L2 while this one computes
                const AdjMaps *mp = a.maps + tl_next.x;
                tma_prefetch_3d(&mp->ad, tl_next.y, tl_next.z - 2, a.acur5);
                tma_prefetch_3d(&mp->m5, tl_next.y, tl_next.z - 2, 0);
                if (a.sgf >= 0) tma_prefetch_3d(&mp->sg, tl_next.y, tl_next.z - 2, a.sgf);
                tma_prefetch_3d(&mp->gi, tl_next.y + 4, tl_next.z + 2, 0);
            }
            __syncthreads();

            // 2. v^ += D^T f^ on the tile + 2-cell halo; e^ in shared memory
            constexpr int N2 = (VX * VZ + kThreads - 1) / kThreads;
            float *f4r = edge ? f4s : f3s;
            float lvx[N2], lvz[N2], lbx[N2], lbz[N2], lfx[N2], lfz[N2], lgx[N2], lgz[N2];
#pragma unroll
            for (int r = 0; r < N2; ++r) {
                const int q = tid + r * kThreads;
                lvx[r] = lvz[r] = lbx[r] = lbz[r] = lfx[r] = lfz[r] = lgx[r] = lgz[r] = 0.f;
                const int y = q / VX, x = q - y * VX;
                const int i = i0 - 2 + x, j = j0 - 2 + y;
                if (q < VX * VZ && (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ))) {
                    const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    lvx[r] = ldg256(a.in.vx + c); lvz[r] = ldg256(a.in.vz + c);
                    lbx[r] = ldg256(a.M.bx + c); lbz[r] = ldg256(a.M.bz + c);
                    if constexpr (SK != 0) {
                        lfx[r] = snap_get<SK>(a.sr.h, c) * dnx;
                        lfz[r] = snap_get<SK>(a.sr.h, a.sr.F + c) * dnz;
                    } else {
                        lfx[r] = ldg256(a.vfx + c); lfz[r] = ldg256(a.vfz + c);
                    }
                    const bool own = x >= 2 && x < TX + 2 && y >= 2 && y < TZ + 2 && (!edge || (i < NX && j < NZ));
                    if (own && (!edge || (i >= PP - 1 && i <= PP + w && j >= PP - 1 && j <= NZ - PP))) {
                        lgx[r] = ld256(a.Gbx + c); lgz[r] = ld256(a.Gbz + c);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < N2; ++r) {
                const int q = tid + r * kThreads;
                if (q >= VX * VZ) break;
                const int y = q / VX, x = q - y * VX;
                const int i = i0 - 2 + x, j = j0 - 2 + y;
                float h1 = 0.f, h2 = 0.f, h3 = 0.f, h4 = 0.f;
                if (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ)) {
                    const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    const int o = (y + 2) * SX + (x + 2);
                    const float inc_x = -(C1 * (f1s[o + 1] - f1s[o]) + C2 * (f1s[o + 2] - f1s[o - 1])) * rdx
                                        - (C1 * (f3s[o] - f3s[o - SX]) + C2 * (f3s[o + SX] - f3s[o - 2 * SX])) * rdz;
                    const float inc_z = -(C1 * (f2s[o + SX] - f2s[o]) + C2 * (f2s[o + 2 * SX] - f2s[o - SX])) * rdz
                                        - (C1 * (f4r[o] - f4r[o - 1]) + C2 * (f4r[o + 1] - f4r[o - 2])) * rdx;
                    const float vx = lvx[r] + inc_x;
                    const float vz = lvz[r] + inc_z;
                    const float qx = dt * lbx[r] * vx, qz = dt * lbz[r] * vz;
                    h1 = qx; h2 = qx; h3 = qz; h4 = qz;
                    const bool own = x >= 2 && x < TX + 2 && y >= 2 && y < TZ + 2 && (!edge || (i < NX && j < NZ));
                    if (edge) {
                        const int xs = i < PP ? i : (i >= NX - PP ? i - NX + 2 * PP : -1);
                        const int zs = j < PP ? j : (j >= NZ - PP ? j - NZ + 2 * PP : -1);
                        if (xs >= 0) {
                            const long long k = psx + (long long)j * 2 * PP + xs;
                            const int pq = profx + i;
                            const float P1 = a.pml.x[0][k], P3 = a.pml.x[1][k];
                            h1 += a.pml.ax_h[pq] * (P1 + qx);
                            h3 += a.pml.ax_i[pq] * (P3 + qz);
                            if (own) {
                                a.n1[k] = a.pml.bx_h[pq] * (P1 + qx);
                                a.n3[k] = a.pml.bx_i[pq] * (P3 + qz);
                            }
                        }
                        if (zs >= 0) {
                            const long long k = psz + (long long)zs * NX + i;
                            const float P2 = a.pml.z[0][k], P4 = a.pml.z[1][k];
                            h2 += a.pml.az_i[j] * (P2 + qx);
                            h4 += a.pml.az_h[j] * (P4 + qz);
                            if (own) {
                                a.n2[k] = a.pml.bz_i[j] * (P2 + qx);
                                a.n4[k] = a.pml.bz_h[j] * (P4 + qz);
                            }
                        }
                    }
                    if (own) {
                        a.out.vx[c] = vx;
                        a.out.vz[c] = vz;
                        if (!edge || (i >= PP - 1 && i <= PP + w && j >= PP - 1 && j <= NZ - PP)) {
                            a.Gbx[c] = lgx[r] + lfx[r] * inc_x;
                            a.Gbz[c] = lgz[r] + lfz[r] * inc_z;
                        }
                    }
                }
                e1s[q] = h1; e3s[q] = h3;
                if (edge) { e2s[q] = h2; e4s[q] = h4; }    // e^2 == e^1, e^4 == e^3 away from the CPML
                vfxs[q] = lfx[r]; vfzs[q] = lfz[r];
            }
            __syncthreads();
            const float *e2r = edge ? e2s : e1s, *e4r = edge ? e4s : e3s;

            // 3. sigma^ += D^T e^ on the tile, with the C-imaging
            constexpr int N3 = (TX * TZ + kThreads - 1) / kThreads;
            float sxx_r[N3], szz_r[N3], sxz_r[N3], g0[N3], g1v[N3], g2v[N3];
#pragma unroll
            for (int r = 0; r < N3; ++r) {
                const int q = tid + r * kThreads;
                const int y = q / TX, x = q - y * TX;
                const int i = i0 + x, j = j0 + y;
                sxx_r[r] = szz_r[r] = sxz_r[r] = g0[r] = g1v[r] = g2v[r] = 0.f;
                if (q < TX * TZ && !(edge && (i >= NX || j >= NZ))) {
                    const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    sxx_r[r] = ldg256(a.in.sxx + c); szz_r[r] = ldg256(a.in.szz + c); sxz_r[r] = ldg256(a.in.sxz + c);
                    const bool node = !edge || (i >= PP && i < PP + w && j >= PP && j < NZ - PP);
                    const bool half = !edge || (i >= PP - 1 && i < PP + w && j >= PP - 1 && j < NZ - PP);
                    if (node) { g0[r] = ld256(a.Glam + c); g1v[r] = ld256(a.Gmu + c); }
                    if (half) g2v[r] = ld256(a.Gmuxz + c);
                }
            }
#pragma unroll
            for (int r = 0; r < N3; ++r) {
                const int q = tid + r * kThreads;
                if (q >= TX * TZ) break;
                const int y = q / TX, x = q - y * TX;
                const int i = i0 + x, j = j0 + y;
                if (edge && (i >= NX || j >= NZ)) continue;
                const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                const float hxx = sxx_r[r], hzz = szz_r[r], hxz = sxz_r[r];
                const int o = (y + 2) * VX + (x + 2);      // (i, j) in the halo-2 staging
                const float *fvx = vfxs + o, *fvz = vfzs + o;
                if (!edge || (i >= PP && i < PP + w && j >= PP && j < NZ - PP)) {
                    const float fx = (C1 * (fvx[0] - fvx[-1]) + C2 * (fvx[1] - fvx[-2])) * rdx;
                    const float fz = (C1 * (fvz[0] - fvz[-VX]) + C2 * (fvz[VX] - fvz[-2 * VX])) * rdz;
                    a.Glam[c] = g0[r] + dt * (hxx + hzz) * (fx + fz);
                    a.Gmu[c] = g1v[r] + 2.f * dt * (hxx * fx + hzz * fz);
                }
                if (!edge || (i >= PP - 1 && i < PP + w && j >= PP - 1 && j < NZ - PP)) {
                    const float fxz = (C1 * (fvx[VX] - fvx[0]) + C2 * (fvx[2 * VX] - fvx[-VX])) * rdz +
                                      (C1 * (fvz[1] - fvz[0]) + C2 * (fvz[2] - fvz[-1])) * rdx;
                    a.Gmuxz[c] = g2v[r] + dt * hxz * fxz;
                }
                a.out.sxx[c] = hxx - (C1 * (e1s[o] - e1s[o - 1]) + C2 * (e1s[o + 1] - e1s[o - 2])) * rdx;
                a.out.szz[c] = hzz - (C1 * (e4r[o] - e4r[o - VX]) + C2 * (e4r[o + VX] - e4r[o - 2 * VX])) * rdz;
                a.out.sxz[c] = hxz - (C1 * (e2r[o + VX] - e2r[o]) + C2 * (e2r[o + 2 * VX] - e2r[o - VX])) * rdz
                                   - (C1 * (e3s[o + 1] - e3s[o]) + C2 * (e3s[o + 2] - e3s[o - 1])) * rdx;
            }
            __syncthreads();
        };
        if (tl.w & 4) tile(std::true_type{});
        else tile(std::false_type{});
    }
}

// ---------------------------------------------------------------------------
// Tile shapes: compile-time instantiations the autotuner chooses from.
// ---------------------------------------------------------------------------
struct Shape {
    int tx, tz;
};
constexpr Shape kShapes[] = {{32, 8}, {32, 16}, {64, 8}, {64, 16}, {32, 32}, {128, 8}, {64, 32}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

size_t fwd_smem(int tx, int tz) { return sizeof(float) * (3 * (tx + 8) * (tz + 8) + 2 * (tx + 4) * (tz + 4)); }
size_t adj_smem(int tx, int tz) { return sizeof(float) * (4 * (tx + 8) * (tz + 8) + 6 * (tx + 4) * (tz + 4)); }

// sk: the plan's snapshot store (EFWI_STORE_*), a compile-time parameter of the kernels
template <int TX, int TZ>
void fwd_launch(const FwdArgs &a, int grid, cudaStream_t st, int sk) {
    if (sk == EFWI_STORE_FP16) k_step_fused<TX, TZ, EFWI_STORE_FP16><<<grid, kThreads, fwd_smem(TX, TZ), st>>>(a);
    else if (sk == EFWI_STORE_BF16) k_step_fused<TX, TZ, EFWI_STORE_BF16><<<grid, kThreads, fwd_smem(TX, TZ), st>>>(a);
    else k_step_fused<TX, TZ><<<grid, kThreads, fwd_smem(TX, TZ), st>>>(a);
}
template <int TX, int TZ>
void adj_launch(const AdjArgsF &a, int grid, cudaStream_t st, int sk) {
    if (sk == EFWI_STORE_FP16) k_adj_fused<TX, TZ, EFWI_STORE_FP16><<<grid, kThreads, adj_smem(TX, TZ), st>>>(a);
    else if (sk == EFWI_STORE_BF16) k_adj_fused<TX, TZ, EFWI_STORE_BF16><<<grid, kThreads, adj_smem(TX, TZ), st>>>(a);
    else k_adj_fused<TX, TZ><<<grid, kThreads, adj_smem(TX, TZ), st>>>(a);
}

template <int TX, int TZ, int SK>
void set_attrs_sk() {
    cudaFuncSetAttribute(k_step_fused<TX, TZ, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(TX, TZ));
    cudaFuncSetAttribute(k_adj_fused<TX, TZ, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_smem(TX, TZ));
}
template <int TX, int TZ>
void set_attrs() {
    set_attrs_sk<TX, TZ, 0>();
    set_attrs_sk<TX, TZ, EFWI_STORE_FP16>();
    set_attrs_sk<TX, TZ, EFWI_STORE_BF16>();
}

void set_all_attrs() {
    static bool done = false;
    if (done) return;
    done = true;
    set_attrs<32, 8>(); set_attrs<32, 16>(); set_attrs<64, 8>(); set_attrs<64, 16>();
    set_attrs<32, 32>(); set_attrs<128, 8>(); set_attrs<64, 32>();
}

#define EFWI_DISPATCH(tx, tz, FN, ...)                                   \
    do {                                                                 \
        if (tx == 32 && tz == 8) FN<32, 8>(__VA_ARGS__);                 \
        else if (tx == 32 && tz == 16) FN<32, 16>(__VA_ARGS__);          \
        else if (tx == 64 && tz == 8) FN<64, 8>(__VA_ARGS__);            \
        else if (tx == 64 && tz == 16) FN<64, 16>(__VA_ARGS__);          \
        else if (tx == 32 && tz == 32) FN<32, 32>(__VA_ARGS__);          \
        else if (tx == 128 && tz == 8) FN<128, 8>(__VA_ARGS__);          \
        else FN<64, 32>(__VA_ARGS__);                                    \
    } while (0)

bool shape_ok(int tx, int tz) {
    for (auto &s : kShapes)
        if (s.tx == tx && s.tz == tz) return true;
    return false;
}

// Work items (shot, i0, j0, flags).  flags bit 0: the tile holds a source
// injection cell; bit 1 (bit 2): the tile or its 2-cell (4-cell) halo touches
// a CPML strip or leaves the padded grid, so kernels take the checked path.
std::vector<int4> make_tiles_of(const std::vector<ShotDev> &shots, int tx, int tz) {
    std::vector<int4> t;
    for (int s = 0; s < (int)shots.size(); ++s) {
        const ShotDev &sh = shots[s];
        for (int j0 = 0; j0 < sh.NZ; j0 += tz)
            for (int i0 = 0; i0 < sh.NX; i0 += tx) {
                int flags = 0;
                for (int q = 0; q < 4; ++q)
                    for (int o : {sh.inj_n[q], sh.inj_x[q]}) {
                        const int j = o / sh.pitch - EFWI_GZ, i = o % sh.pitch - EFWI_GX;
                        if (i >= i0 && i < i0 + tx && j >= j0 && j < j0 + tz) flags |= 1;
                    }
                for (int h : {2, 4}) {
                    const int xa = i0 - h, xb = i0 + tx + h, za = j0 - h, zb = j0 + tz + h;
                    if (xa < sh.P || xb > sh.NX - sh.P || za < sh.P || zb > sh.NZ - sh.P) flags |= h;
                }
                // bit 3: a vector-force cell lies in the tile or its 2-cell velocity halo
                if (sh.fx != 0.f || sh.fz != 0.f)
                    for (int q = 0; q < 4; ++q)
                        for (int o : {sh.inj_vx[q], sh.inj_vz[q]}) {
                            const int j = o / sh.pitch - EFWI_GZ, i = o % sh.pitch - EFWI_GX;
                            if (i >= i0 - 2 && i < i0 + tx + 2 && j >= j0 - 2 && j < j0 + tz + 2) flags |= 8;
                        }
                t.push_back(make_int4(s, i0, j0, flags));
            }
    }
    return t;
}

std::vector<int4> make_tiles(efwi_plan *p, int tx, int tz) { return make_tiles_of(p->shots, tx, tz); }

}  // namespace

std::vector<int4> tiles_of(const std::vector<ShotDev> &shots, const TileList &tl) {
    return tl.tiles ? make_tiles_of(shots, tl.tx, tl.tz) : std::vector<int4>();
}

int upload_tiles(efwi_plan *p, TileList &tl, int tx, int tz) {
    std::vector<int4> t = make_tiles(p, tx, tz);
    if (tl.tiles) cudaFree(tl.tiles);
    tl.tiles = nullptr;
    if (cudaMalloc((void **)&tl.tiles, sizeof(int4) * t.size()) != cudaSuccess) return EFWI_ERR_OOM;
    cudaMemcpy(tl.tiles, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice);
    tl.n = (int)t.size();
    tl.tx = tx;
    tl.tz = tz;
    return EFWI_OK;
}

// Recompute the flags of a tile list (source and force cells) for the plan's
// current acquisition and copy them over the list in place (same geometry, so
// the same tiles; the pointer, which captured graphs hold, stays).
int refresh_tiles(efwi_plan *p, TileList &tl, cudaStream_t st) {
    if (!tl.tiles) return EFWI_OK;
    std::vector<int4> t = make_tiles(p, tl.tx, tl.tz);
    if ((int)t.size() != tl.n) return EFWI_ERR_ARG;
    cudaMemcpyAsync(tl.tiles, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice, st);
    return EFWI_OK;
}

namespace {

FwdArgs fwd_args(efwi_plan *p, int n, const SnapOut &so) {
    float *segx = so.fx, *segz = so.fz;
    FwdArgs a;
    a.shots = p->shots_d;
    a.tiles = p->tiles.tiles;
    a.ntiles = p->tiles.n;
    a.in = state_fields(p, p->scur);
    a.out = state_fields(p, 1 - p->scur);
    a.M = materials(p);
    a.pml = fwd_pml(p, p->psi_v, p->psi_s);
    float *vn = psi_block(p->psi, p, 1 - p->psi_v);
    a.n1 = vn; a.n3 = vn + p->psx_total; a.n2 = vn + 2 * p->psx_total; a.n4 = vn + 2 * p->psx_total + p->psz_total;
    a.segx = segx; a.segz = segz;
    a.dw = p->dw;
    a.wv = p->wv;
    a.nt = p->d.nt;
    a.n = n;
    a.dt = (float)p->d.dt;
    a.rdx = (float)(1.0 / p->d.dx);
    a.rdz = (float)(1.0 / p->d.dz);
    a.sw = so.sw;
    return a;
}


}  // namespace

AdjArgsF adj_args_f(efwi_plan *p, const SnapIn &si) {
    const float *vfx = si.fx, *vfz = si.fz;
    AdjArgsF a;
    a.shots = p->shots_d;
    a.tiles = p->adj_tiles.tiles;
    a.ntiles = p->adj_tiles.n;
    a.in = adj_fields(p, p->acur);
    a.out = adj_fields(p, 1 - p->acur);
    a.M = materials(p);
    a.pml = adj_pml(p, p->apsi_v, p->apsi_s);
    const long long X = p->psx_total, Z = p->psz_total;
    float *vn = psi_block(p->apsi, p, 1 - p->apsi_v), *sn = psi_block(p->apsi, p, 2 + (1 - p->apsi_s));
    a.n1 = vn; a.n3 = vn + X; a.n2 = vn + 2 * X; a.n4 = vn + 2 * X + Z;
    a.n5 = sn; a.n8 = sn + X; a.n6 = sn + 2 * X; a.n7 = sn + 2 * X + Z;
    a.vfx = vfx; a.vfz = vfz;
    a.sr = si.sr;
    a.maps = p->adj_maps;
    a.pf = p->adj_pf && p->adj_maps && p->adj_grid > 0;
    a.acur5 = 5 * p->acur;
    a.sgf = (vfx && p->seg) ? (int)(2 * ((vfx - p->seg) / (2 * p->fsz_total))) : -1;
    a.Glam = G_field(p, 0); a.Gmu = G_field(p, 1); a.Gmuxz = G_field(p, 2);
    a.Gbx = G_field(p, 3); a.Gbz = G_field(p, 4);
    a.dt = (float)p->d.dt;
    a.rdx = (float)(1.0 / p->d.dx);
    a.rdz = (float)(1.0 / p->d.dz);
    return a;
}

void launch_step_fused(efwi_plan *p, int n, const SnapOut &so, cudaStream_t st) {
    int slot;
    prof_begin(p, st, &slot, EFWI_KERNEL_STEP);
    if (p->stencil >= EFWI_STENCIL_TMA) {
        launch_step_tma(p, n, so, st);
    } else {
        FwdArgs a = fwd_args(p, n, so);
        const int grid = p->grid_fwd_override > 0 ? std::min(p->grid_fwd_override, a.ntiles) : a.ntiles;
        EFWI_DISPATCH(p->tiles.tx, p->tiles.tz, fwd_launch, a, grid, st, p->snap_store);
    }
    prof_end(p, st, slot);
    p->launches++;
    p->scur ^= 1;
    p->psi_v ^= 1;
}

void launch_adj_fused(efwi_plan *p, int n, const SnapIn &si, cudaStream_t st) {
    (void)n;
    int slot;
    prof_begin(p, st, &slot, EFWI_KERNEL_ADJ);
    if (p->adj_form == EFWI_ADJ_FORM_SCALED) {
        if (p->adj_stencil == EFWI_STENCIL_TMA) launch_adj_scaled_tma(p, si, st);   // FP32 snapshots only
        else launch_adj_scaled(p, si, st);
    } else if (p->adj_stencil == EFWI_STENCIL_TMA) {
        launch_adj_tma(p, si.fx, st);         // FP32 snapshots only (the autotuner's candidates)
    } else {
        AdjArgsF a = adj_args_f(p, si);
        const int grid = p->grid_adj_override > 0 ? std::min(p->grid_adj_override, a.ntiles)
                         : p->adj_grid > 0        ? std::min(p->adj_grid, a.ntiles)
                                                  : a.ntiles;
        EFWI_DISPATCH(p->adj_tiles.tx, p->adj_tiles.tz, adj_launch, a, grid, st, p->snap_store);
    }
    prof_end(p, st, slot);
    p->launches++;
    p->acur ^= 1;
    p->apsi_v ^= 1;
    p->apsi_s ^= 1;
}

}  // namespace efwi

using namespace efwi;

// Tile autotuner: times a few fused forward and adjoint steps of the plan's
// own shots for every compiled variant (staging kind x tile shape) and keeps
// the fastest.  Variants change only the work decomposition and staging, never
// the arithmetic, so the choice does not change results.
namespace {

struct Variant {
    int kind, tx, tz, nst, vec = 1, st = 0;
};

float time_steps(efwi_plan *p, bool adj, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps = 3) {
    // the snapshot traffic of a real step: FP32 copy of v into slot 0, or the
    // reduced-precision pack of slot 0 and the maxima of slot 1
    const SnapOut so = snap_out(p, p->K > 1 ? 1 : 0, 0);
    const SnapIn si = snap_in(p, 0);
    float t = 0;
    for (int w = 0; w < 2; ++w) {              // warm-up, then timed
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) {
            if (adj) launch_adj_fused(p, 0, si, st);
            else launch_step_fused(p, 0, so, st);
        }
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t, e0, e1);
    }
    return cudaGetLastError() == cudaSuccess ? t : 1e30f;
}

int select_adj(efwi_plan *p, const Variant &v) {
    p->adj_stencil = v.kind;
    p->adj_grid = 0;
    if (v.kind == EFWI_STENCIL_LOADS && v.vec == 2 && p->adj_form == EFWI_ADJ_FORM_SCALED) {
        p->adj_grid = std::max(1, adj_scaled_blocks_per_sm(v.tx, v.tz, p->snap_store)) * p->n_sms;
    } else if (v.kind == EFWI_STENCIL_LOADS && v.vec == 2 && v.tx == 32 && v.tz == 16) {   // loads: vec 2 = persistent
        int nb = 0;
        if (p->snap_store == EFWI_STORE_FP16)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_fused<32, 16, EFWI_STORE_FP16>, kThreads,
                                                          adj_smem(32, 16));
        else if (p->snap_store == EFWI_STORE_BF16)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_fused<32, 16, EFWI_STORE_BF16>, kThreads,
                                                          adj_smem(32, 16));
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_fused<32, 16>, kThreads, adj_smem(32, 16));
        p->adj_grid = std::max(1, nb) * p->n_sms;
    }
    int rc = upload_tiles(p, p->adj_tiles, v.tx, v.tz);
    if (!rc && v.kind == EFWI_STENCIL_TMA)
        rc = p->adj_form == EFWI_ADJ_FORM_SCALED ? adj_scaled_tma_prepare(p, v.tx, v.tz, v.vec)
                                                 : tma_prepare_adj(p, v.tx, v.tz, v.nst);
    p->adj_tile_x = v.tx;
    p->adj_tile_z = v.tz;
    return rc;
}

int select_fwd(efwi_plan *p, const Variant &v) {
    p->stencil = v.kind;
    int rc = upload_tiles(p, p->tiles, v.tx, v.tz);
    if (!rc && v.kind >= EFWI_STENCIL_TMA) rc = tma_prepare_fwd(p, v.tx, v.tz, v.nst, v.vec, v.st);
    p->tile_x = v.tx;
    p->tile_z = v.tz;
    return rc;
}

}  // namespace

int efwi_autotune(efwi_plan *p) {
    set_all_attrs();
    const int want = p->d.stencil;
    const int want_a = p->d.adj_stencil;
    const bool fixed = p->tile_x > 0 && p->tile_z > 0;
    const bool fixed_a = p->adj_tile_x > 0 && p->adj_tile_z > 0;
    std::vector<Variant> fwd, adj;
    // EFWI_TMA_STAGES=n / EFWI_TMA_VEC=v keep only n-stage / v-layout TMA forward variants
    // (reproducible profiles, tests of one layout)
    const char *fs = getenv("EFWI_TMA_STAGES"), *fv = getenv("EFWI_TMA_VEC");
    const int only_nst = fs ? atoi(fs) : 0, only_vec = fv ? atoi(fv) : 0;
    for (auto &s : kShapes) {
        if (fixed && (s.tx != p->tile_x || s.tz != p->tile_z)) continue;
        if (want == EFWI_STENCIL_AUTO || want == EFWI_STENCIL_LOADS) fwd.push_back({EFWI_STENCIL_LOADS, s.tx, s.tz, 0});
        for (int vec = 1; vec <= 3; ++vec)
            for (int stg = 0; stg <= 1; ++stg) {
                const int kind = vec == 1 ? EFWI_STENCIL_TMA : stg ? EFWI_STENCIL_TMA_STAGED : EFWI_STENCIL_TMA_PAIRS;
                if (want != EFWI_STENCIL_AUTO && want != kind) continue;
                for (int nst = 2; nst <= 4; ++nst)
                    if ((!only_nst || nst == only_nst) && (!only_vec || vec == only_vec || vec == 1) &&
                        tma_shape_ok(s.tx, s.tz, nst, vec, stg, p->snap_store))
                        fwd.push_back({kind, s.tx, s.tz, nst, vec, stg});
            }
    }
    // the adjoint's stress variable: the scaled form (per-thread loads) unless the stress
    // form is asked for, or a TMA adjoint (which exists in the stress form only)
    p->adj_form = p->d.adj_form == EFWI_ADJ_FORM_STRESS ? EFWI_ADJ_FORM_STRESS
                  : p->d.adj_form == EFWI_ADJ_FORM_SCALED ? EFWI_ADJ_FORM_SCALED
                  : (want_a == EFWI_STENCIL_AUTO || want_a == EFWI_STENCIL_LOADS || want_a == EFWI_STENCIL_TMA)
                      ? EFWI_ADJ_FORM_SCALED
                      : EFWI_ADJ_FORM_STRESS;
    const bool scaled = p->adj_form == EFWI_ADJ_FORM_SCALED;
    if (scaled) adj_scaled_set_attrs();
    // the adjoint follows its own request, or the forward one when it has none
    const int wa = want_a != EFWI_STENCIL_AUTO ? want_a : want;
    for (auto &s : kShapes) {
        if (!scaled) break;
        if (fixed_a && (s.tx != p->adj_tile_x || s.tz != p->adj_tile_z)) continue;
        // per-thread loads: every compiled tile, 32x16 also on a persistent grid
        // (EFWI_ADJ_PERSIST=0|1 keeps only one of the two); TMA staging: 32x16
        const char *fp = getenv("EFWI_ADJ_PERSIST");
        const int only_p = fp ? atoi(fp) : -1;
        if (want_a != EFWI_STENCIL_TMA && adj_scaled_shape_ok(s.tx, s.tz)) {
            if (only_p <= 0 || !(s.tx == 32 && s.tz == 16)) adj.push_back({EFWI_STENCIL_LOADS, s.tx, s.tz, 0});
            if (s.tx == 32 && s.tz == 16 && only_p != 0) adj.push_back({EFWI_STENCIL_LOADS, 32, 16, 0, 2});
        }
        // TMA staging, one cell or a cell pair per thread (EFWI_ADJ_VEC=1|2 keeps only one)
        const char *fa = getenv("EFWI_ADJ_VEC");
        const int only_av = fa ? atoi(fa) : 0;
        if (want_a != EFWI_STENCIL_LOADS && adj_scaled_tma_shape_ok(s.tx, s.tz))
            for (int av = 1; av <= 3; ++av)   // 3: cell pairs, 512-thread CTAs
                if (!only_av || av == only_av) adj.push_back({EFWI_STENCIL_TMA, s.tx, s.tz, 2, av});
    }
    if (scaled && adj.empty()) {
        p->err = "no scaled-stress adjoint variant matches the request (per-thread loads: tiles 32x8 32x16 64x8 "
                 "64x16; TMA: 32x16)";
        return EFWI_ERR_ARG;
    }
    for (auto &s : kShapes) {
        if (scaled) break;
        if (fixed_a ? (s.tx != p->adj_tile_x || s.tz != p->adj_tile_z)
                    : (fixed && (s.tx != p->tile_x || s.tz != p->tile_z)))
            continue;
        if (wa == EFWI_STENCIL_AUTO || wa == EFWI_STENCIL_LOADS) {
            // 32x16 also on a persistent grid (the next tile's descriptor loaded ahead);
            // EFWI_ADJ_PERSIST=0|1 keeps only one of the two (tests of one variant)
            const char *fp = getenv("EFWI_ADJ_PERSIST");
            const int only_p = fp ? atoi(fp) : -1;
            if (only_p <= 0) adj.push_back({EFWI_STENCIL_LOADS, s.tx, s.tz, 0});
            if (s.tx == 32 && s.tz == 16 && only_p != 0) adj.push_back({EFWI_STENCIL_LOADS, 32, 16, 0, 2});
        }
        for (int nst = 1; nst <= 2; ++nst)   // (the TMA adjoint reads FP32 snapshots only)
            if (wa != EFWI_STENCIL_LOADS && p->snap_store == EFWI_STORE_FP32 && tma_adj_shape_ok(s.tx, s.tz, nst))
                adj.push_back({EFWI_STENCIL_TMA, s.tx, s.tz, nst});
    }
    // a requested staging without an instantiation for this tile falls back to per-thread loads
    for (auto &s : kShapes) {
        if (fwd.empty() && (!fixed || (s.tx == p->tile_x && s.tz == p->tile_z)))
            fwd.push_back({EFWI_STENCIL_LOADS, s.tx, s.tz, 0});
        if (adj.empty() && !scaled && (!fixed_a || (s.tx == p->adj_tile_x && s.tz == p->adj_tile_z)))
            adj.push_back({EFWI_STENCIL_LOADS, s.tx, s.tz, 0});
    }
    if (fwd.empty() || adj.empty()) {
        p->err = "no compiled stencil variant matches the requested tile/stencil "
                 "(loads: 32x8 32x16 64x8 64x16 32x32 128x8 64x32; tma: 32x8 32x16 64x8 64x16; tma_staged: 32x16)";
        return EFWI_ERR_ARG;
    }
    int rc = EFWI_OK;
    Variant bf = fwd[0], ba = adj[0];
    if (fwd.size() > 1 || adj.size() > 1) {
        cudaStream_t st;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        // EFWI_AUTOTUNE_LOG=1 reports every timed variant on stderr
        const char *lg = getenv("EFWI_AUTOTUNE_LOG");
        const bool log = lg && lg[0] == '1';
        float best = 1e30f;
        for (auto &v : fwd) {
            if (select_fwd(p, v)) continue;
            const float t = time_steps(p, false, st, e0, e1);
            if (log) fprintf(stderr, "efwi autotune fwd kind %d tile %dx%d param %d vec %d staged %d: %.1f us\n",
                             v.kind, v.tx, v.tz, v.nst, v.vec, v.st, t * 1e3f / 3);
            if (t < best) { best = t; bf = v; }
        }
        best = 1e30f;
        for (auto &v : adj) {
            if (select_adj(p, v)) continue;
            const float t = time_steps(p, true, st, e0, e1);
            if (log) fprintf(stderr, "efwi autotune adj kind %d tile %dx%d param %d vec/persistent %d: %.1f us\n",
                             v.kind, v.tx, v.tz, v.nst, v.vec, t * 1e3f / 3);
            if (t < best) { best = t; ba = v; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(st);
    }
    // overlap of recompute and adjoint: time both chains on two streams for a few
    // splits of the SMs' blocks, against running them one after the other
    rc = select_fwd(p, bf);
    if (!rc) rc = select_adj(p, ba);
    // L2 prefetch one tile beyond what the chosen forward (TMA) and adjoint (persistent
    // per-thread loads) steps load: kept when it saves more than 1 %.  EFWI_PREFETCH=0|1
    // forces it off or on (reproducible profiles and tests of one variant).
    {
        const char *fe = getenv("EFWI_PREFETCH");
        const int force_pf = fe ? atoi(fe) : -1;
        p->tma_pf = p->adj_pf = 0;
        const bool fwd_ok = !rc && p->stencil >= EFWI_STENCIL_TMA;
        const bool adj_ok = !rc && p->adj_stencil == EFWI_STENCIL_LOADS && p->adj_grid > 0 &&
                            p->adj_form == EFWI_ADJ_FORM_STRESS &&
                            tma_encode_adj_maps(p, p->adj_tile_x, p->adj_tile_z) == EFWI_OK;
        if (force_pf >= 0) {
            p->tma_pf = fwd_ok && force_pf;
            p->adj_pf = adj_ok && force_pf;
        } else if (fwd_ok || adj_ok) {
            cudaStream_t st;
            cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            const char *lg = getenv("EFWI_AUTOTUNE_LOG");
            const bool log = lg && lg[0] == '1';
            for (int adj = 0; adj < 2; ++adj) {
                if (!(adj ? adj_ok : fwd_ok)) continue;
                int &flag = adj ? p->adj_pf : p->tma_pf;
                flag = 0;
                const float t0 = time_steps(p, adj, st, e0, e1, 12);
                flag = 1;
                const float t1 = time_steps(p, adj, st, e0, e1, 12);
                if (log) fprintf(stderr, "efwi autotune %s L2 prefetch: off %.1f us, on %.1f us\n", adj ? "adj" : "fwd",
                                 t0 * 1e3f / 12, t1 * 1e3f / 12);
                flag = t1 < 0.99f * t0;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaStreamDestroy(st);
        }
    }
    p->ov_fwd = p->ov_adj = 0;
    const long long segbytes = sizeof(float) * (long long)p->K * 2 * p->fsz_total;
    float *seg2 = nullptr;
    if (!rc && p->K < p->d.nt && p->n_split >= p->d.nt && p->d.overlap != EFWI_OVERLAP_OFF &&
        p->snap_store == EFWI_STORE_FP32 &&
        cudaMalloc((void **)&seg2, segbytes) != cudaSuccess) {
        cudaGetLastError();
        seg2 = nullptr;
        if (p->d.overlap == EFWI_OVERLAP_ON) {
            p->err = "autotune: no memory for the second segment buffer of the overlapped schedule";
            return EFWI_ERR_OOM;
        }
    }
    if (seg2) {
        cudaStream_t sa, sr;
        cudaStreamCreateWithFlags(&sa, cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&sr, cudaStreamNonBlocking);
        cudaEvent_t e0, e1, ej;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventCreateWithFlags(&ej, cudaEventDisableTiming);
        float *sx0 = p->seg, *sz0 = p->seg + p->fsz_total;
        float *sx1 = seg2, *sz1 = seg2 + p->fsz_total;
        const int reps = 4;
        const bool tma_adj = p->adj_stencil == EFWI_STENCIL_TMA;
        auto run = [&](int of, int oa) {
            float t = 0;
            for (int w = 0; w < 2; ++w) {
                cudaEventRecord(e0, sa);
                cudaStreamWaitEvent(sr, e0);
                p->grid_fwd_override = of * p->n_sms;
                SnapOut so1;
                so1.fx = sx1; so1.fz = sz1;
                for (int r = 0; r < reps; ++r) launch_step_fused(p, 0, so1, of ? sr : sa);
                p->grid_fwd_override = 0;
                p->grid_adj_override = oa * p->n_sms;
                SnapIn si0;
                si0.fx = sx0; si0.fz = sz0;
                for (int r = 0; r < reps; ++r) launch_adj_fused(p, 0, si0, sa);
                p->grid_adj_override = 0;
                cudaEventRecord(ej, sr);
                cudaStreamWaitEvent(sa, ej);
                cudaEventRecord(e1, sa);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&t, e0, e1);
            }
            return cudaGetLastError() == cudaSuccess ? t : 1e30f;
        };
        (void)tma_adj;
        const bool force = p->d.overlap == EFWI_OVERLAP_ON;
        float best = force ? 1e30f : run(0, 0);
        const int splits[][2] = {{1, 1}, {1, 2}, {2, 1}, {2, 2}, {1, 3}, {3, 1}};
        for (auto &sp : splits) {
            const float t = run(sp[0], sp[1]);
            if (t < (force ? 1.f : 0.97f) * best) { best = t; p->ov_fwd = sp[0]; p->ov_adj = sp[1]; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(ej);
        cudaStreamDestroy(sa);
        cudaStreamDestroy(sr);
        cudaDeviceSynchronize();
        cudaFree(seg2);
        if (p->ov_fwd > 0) {
            // keep the schedule: one contiguous two-half segment buffer (the TMA adjoint
            // map covers both halves), maps re-encoded for it
            float *both = nullptr;
            if (cudaMalloc((void **)&both, 2 * segbytes) != cudaSuccess) {
                cudaGetLastError();
                p->ov_fwd = p->ov_adj = 0;
            } else {
                cudaFree(p->seg);
                p->seg = both;
                p->bytes += segbytes;
                p->seg_double = true;
                p->nslots = 2 * p->K;
                rc = select_adj(p, ba);
                if (!rc) rc = select_fwd(p, bf);   // the forward segment map covers both halves
            }
        }
    }
    // the timing runs touched workspace only; clear what the next call expects zeroed
    cudaDeviceSynchronize();
    for (int k = 0; k < 2; ++k)
        if (p->state[k]) cudaMemset(p->state[k], 0, sizeof(float) * 5 * p->fsz_total);
    for (int k = 0; k < 2; ++k)
        if (p->adj[k]) cudaMemset(p->adj[k], 0, sizeof(float) * 5 * p->fsz_total);
    cudaMemset(p->psi, 0, sizeof(float) * 4 * p->H);
    cudaMemset(p->apsi, 0, sizeof(float) * 4 * p->H);
    cudaMemset(p->G, 0, sizeof(float) * 5 * p->fsz_total);
    if (p->seg) cudaMemset(p->seg, 0, sizeof(float) * (size_t)p->nslots * 2 * p->fsz_total);
    cudaMemset(p->dev_err, 0, sizeof(int));
    p->scur = p->acur = p->psi_v = p->psi_s = p->apsi_v = p->apsi_s = 0;
    p->launches = 0;
    p->prof_counter[0] = p->prof_counter[1] = 0;
    p->ev_used = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        p->err = std::string("autotune: ") + cudaGetErrorString(e);
        return EFWI_ERR_CUDA;
    }
    if (rc && p->err.empty()) p->err = "autotune: could not prepare the selected variant";
    return rc;
}
