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
#include <vector>

#include "plan.hpp"

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
    int nt, n;
    float dt, rdx, rdz;
};

template <int TX, int TZ>
__global__ void __launch_bounds__(kThreads) k_step_fused(FwdArgs a) {
    constexpr int SX = TX + 8, SZ = TZ + 8;     // sigma staging: tile + 4 halo
    constexpr int VX = TX + 4, VZ = TZ + 4;     // velocity: tile + 2 halo
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *sxx = sm, *szz = sm + SX * SZ, *sxz = sm + 2 * SX * SZ;
    float *svx = sm + 3 * SX * SZ, *svz = svx + VX * VZ;
    const int tid = threadIdx.x;

    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 tl = a.tiles[t];
        const ShotDev s = a.shots[tl.x];
        const int i0 = tl.y, j0 = tl.z;
        const long long P = s.pitch;
        const int rowlim = s.pitch - EFWI_GX;

        // 1. sigma^n with a 4-cell halo (zero outside the padded grid)
        constexpr int Q4 = SX / 4;
        for (int q = tid; q < 3 * SZ * Q4; q += kThreads) {
            const int f = q / (SZ * Q4), r = q - f * SZ * Q4;
            const int y = r / Q4, x4 = r - y * Q4;
            const int i = i0 - 4 + 4 * x4, j = j0 - 4 + y;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j >= 0 && j < s.NZ && i + 4 <= rowlim) {
                const float *src = f == 0 ? a.in.sxx : (f == 1 ? a.in.szz : a.in.sxz);
                v = __ldg(reinterpret_cast<const float4 *>(src + cell_of(s, i, j)));
            }
            reinterpret_cast<float4 *>(sm + f * SX * SZ + y * SX)[x4] = v;
        }
        __syncthreads();

        // 2. v^{n+1/2} on the tile + 2-cell halo
        for (int q = tid; q < VX * VZ; q += kThreads) {
            const int y = q / VX, x = q - y * VX;
            const int i = i0 - 2 + x, j = j0 - 2 + y;
            float vx = 0.f, vz = 0.f;
            if (i >= 0 && i < s.NX && j >= 0 && j < s.NZ) {
                const long long c = cell_of(s, i, j);
                const int o = (y + 2) * SX + (x + 2);       // (i, j) in sigma staging
                float e1 = (C1 * (sxx[o + 1] - sxx[o]) + C2 * (sxx[o + 2] - sxx[o - 1])) * a.rdx;
                float e2 = (C1 * (sxz[o] - sxz[o - SX]) + C2 * (sxz[o + SX] - sxz[o - 2 * SX])) * a.rdz;
                float e3 = (C1 * (sxz[o] - sxz[o - 1]) + C2 * (sxz[o + 1] - sxz[o - 2])) * a.rdx;
                float e4 = (C1 * (szz[o + SX] - szz[o]) + C2 * (szz[o + 2 * SX] - szz[o - SX])) * a.rdz;
                const bool own = i >= i0 && i < i0 + TX && j >= j0 && j < j0 + TZ;
                const int xs = xstrip(s, i), zs = zstrip(s, j);
                if (xs >= 0) {
                    const long long k = s.psx + (long long)j * 2 * s.P + xs;
                    const int pq = s.profx + i;
                    const float p1 = a.pml.bx_h[pq] * a.pml.x[0][k] + a.pml.ax_h[pq] * e1;
                    const float p3 = a.pml.bx_i[pq] * a.pml.x[1][k] + a.pml.ax_i[pq] * e3;
                    if (own) { a.n1[k] = p1; a.n3[k] = p3; }
                    e1 += p1; e3 += p3;
                }
                if (zs >= 0) {
                    const long long k = s.psz + (long long)zs * s.NX + i;
                    const float p2 = a.pml.bz_i[j] * a.pml.z[0][k] + a.pml.az_i[j] * e2;
                    const float p4 = a.pml.bz_h[j] * a.pml.z[1][k] + a.pml.az_h[j] * e4;
                    if (own) { a.n2[k] = p2; a.n4[k] = p4; }
                    e2 += p2; e4 += p4;
                }
                vx = __ldg(a.in.vx + c) + a.dt * __ldg(a.M.bx + c) * (e1 + e2);
                vz = __ldg(a.in.vz + c) + a.dt * __ldg(a.M.bz + c) * (e3 + e4);
                if (own) {
                    a.out.vx[c] = vx;
                    a.out.vz[c] = vz;
                    if (a.segx) { a.segx[c] = vx; a.segz[c] = vz; }
                }
            }
            svx[q] = vx;
            svz[q] = vz;
        }
        __syncthreads();

        // 3. sigma^{n+1} on the tile, then the moment-tensor source
        const float dwn = a.dw[(long long)tl.x * a.nt + a.n];
        for (int q = tid; q < TX * TZ; q += kThreads) {
            const int y = q / TX, x = q - y * TX;
            const int i = i0 + x, j = j0 + y;
            if (i >= s.NX || j >= s.NZ) continue;
            const long long c = cell_of(s, i, j);
            const int o = (y + 2) * VX + (x + 2);           // (i, j) in velocity staging
            float f1 = (C1 * (svx[o] - svx[o - 1]) + C2 * (svx[o + 1] - svx[o - 2])) * a.rdx;
            float f2 = (C1 * (svz[o] - svz[o - VX]) + C2 * (svz[o + VX] - svz[o - 2 * VX])) * a.rdz;
            float f3 = (C1 * (svx[o + VX] - svx[o]) + C2 * (svx[o + 2 * VX] - svx[o - VX])) * a.rdz;
            float f4 = (C1 * (svz[o + 1] - svz[o]) + C2 * (svz[o + 2] - svz[o - 1])) * a.rdx;
            const int xs = xstrip(s, i), zs = zstrip(s, j);
            if (xs >= 0) {
                const long long k = s.psx + (long long)j * 2 * s.P + xs;
                const int pq = s.profx + i;
                const float p5 = a.pml.bx_i[pq] * a.pml.x[2][k] + a.pml.ax_i[pq] * f1;
                const float p8 = a.pml.bx_h[pq] * a.pml.x[3][k] + a.pml.ax_h[pq] * f4;
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
            const int os = (y + 4) * SX + (x + 4);          // (i, j) in sigma staging
            const float lam = __ldg(a.M.lam + c), mu2 = 2.f * __ldg(a.M.mu + c);
            const float tr = lam * (f1 + f2);
            float nxx = sxx[os] + a.dt * (tr + mu2 * f1);
            float nzz = szz[os] + a.dt * (tr + mu2 * f2);
            float nxz = sxz[os] + a.dt * __ldg(a.M.muxz + c) * (f3 + f4);
            const int lc = (int)(c - s.off);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (lc == s.inj_n[k]) {
                    nxx -= s.mxx * dwn * s.inj_nw[k];
                    nzz -= s.mzz * dwn * s.inj_nw[k];
                }
                if (lc == s.inj_x[k]) nxz -= s.mxz * dwn * s.inj_xw[k];
            }
            a.out.sxx[c] = nxx;
            a.out.szz[c] = nzz;
            a.out.sxz[c] = nxz;
        }
        __syncthreads();
    }
}

struct AdjArgsF {
    const ShotDev *shots;
    const int4 *tiles;
    int ntiles;
    Fields in, out;             // adjoint fields
    Mat M;
    Pml pml;                    // current adjoint PML memory (V and S blocks, read)
    float *n1, *n3, *n2, *n4;   // next V block
    float *n5, *n8, *n6, *n7;   // next S block
    const float *vfx, *vfz;     // forward v^{n+1/2}
    float *Glam, *Gmu, *Gmuxz, *Gbx, *Gbz;
    float dt, rdx, rdz;
};

template <int TX, int TZ>
__global__ void __launch_bounds__(kThreads) k_adj_fused(AdjArgsF a) {
    constexpr int SX = TX + 8, SZ = TZ + 8;
    constexpr int VX = TX + 4, VZ = TZ + 4;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *f1s = sm, *f2s = sm + SX * SZ, *f3s = sm + 2 * SX * SZ, *f4s = sm + 3 * SX * SZ;
    float *e1s = sm + 4 * SX * SZ, *e2s = e1s + VX * VZ, *e3s = e2s + VX * VZ, *e4s = e3s + VX * VZ;
    const int tid = threadIdx.x;

    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 tl = a.tiles[t];
        const ShotDev s = a.shots[tl.x];
        const int i0 = tl.y, j0 = tl.z;
        const long long P = s.pitch;

        // 1. f^ on the tile + 4-cell halo; the tile's stress-sub-step PML memory advances
        for (int q = tid; q < SX * SZ; q += kThreads) {
            const int y = q / SX, x = q - y * SX;
            const int i = i0 - 4 + x, j = j0 - 4 + y;
            float g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f;
            if (i >= 0 && i < s.NX && j >= 0 && j < s.NZ) {
                const long long c = cell_of(s, i, j);
                const float hxx = __ldg(a.in.sxx + c), hzz = __ldg(a.in.szz + c), hxz = __ldg(a.in.sxz + c);
                const float lam = __ldg(a.M.lam + c), l2m = lam + 2.f * __ldg(a.M.mu + c);
                const float Ex = a.dt * (l2m * hxx + lam * hzz);
                const float Ez = a.dt * (lam * hxx + l2m * hzz);
                const float Exz = a.dt * __ldg(a.M.muxz + c) * hxz;
                g1 = Ex; g2 = Ez; g3 = Exz; g4 = Exz;
                const bool own = i >= i0 && i < i0 + TX && j >= j0 && j < j0 + TZ;
                const int xs = xstrip(s, i), zs = zstrip(s, j);
                if (xs >= 0) {
                    const long long k = s.psx + (long long)j * 2 * s.P + xs;
                    const int pq = s.profx + i;
                    const float P5 = a.pml.x[2][k], P8 = a.pml.x[3][k];
                    g1 += a.pml.ax_i[pq] * (P5 + Ex);
                    g4 += a.pml.ax_h[pq] * (P8 + Exz);
                    if (own) {
                        a.n5[k] = a.pml.bx_i[pq] * (P5 + Ex);
                        a.n8[k] = a.pml.bx_h[pq] * (P8 + Exz);
                    }
                }
                if (zs >= 0) {
                    const long long k = s.psz + (long long)zs * s.NX + i;
                    const float P6 = a.pml.z[2][k], P7 = a.pml.z[3][k];
                    g2 += a.pml.az_i[j] * (P6 + Ez);
                    g3 += a.pml.az_h[j] * (P7 + Exz);
                    if (own) {
                        a.n6[k] = a.pml.bz_i[j] * (P6 + Ez);
                        a.n7[k] = a.pml.bz_h[j] * (P7 + Exz);
                    }
                }
            }
            f1s[q] = g1; f2s[q] = g2; f3s[q] = g3; f4s[q] = g4;
        }
        __syncthreads();

        // 2. v^ += D^T f^ on the tile + 2-cell halo; e^ in shared memory
        for (int q = tid; q < VX * VZ; q += kThreads) {
            const int y = q / VX, x = q - y * VX;
            const int i = i0 - 2 + x, j = j0 - 2 + y;
            float h1 = 0.f, h2 = 0.f, h3 = 0.f, h4 = 0.f;
            if (i >= 0 && i < s.NX && j >= 0 && j < s.NZ) {
                const long long c = cell_of(s, i, j);
                const int o = (y + 2) * SX + (x + 2);
                const float inc_x = -(C1 * (f1s[o + 1] - f1s[o]) + C2 * (f1s[o + 2] - f1s[o - 1])) * a.rdx
                                    - (C1 * (f3s[o] - f3s[o - SX]) + C2 * (f3s[o + SX] - f3s[o - 2 * SX])) * a.rdz;
                const float inc_z = -(C1 * (f2s[o + SX] - f2s[o]) + C2 * (f2s[o + 2 * SX] - f2s[o - SX])) * a.rdz
                                    - (C1 * (f4s[o] - f4s[o - 1]) + C2 * (f4s[o + 1] - f4s[o - 2])) * a.rdx;
                const float vx = __ldg(a.in.vx + c) + inc_x;
                const float vz = __ldg(a.in.vz + c) + inc_z;
                const float qx = a.dt * __ldg(a.M.bx + c) * vx, qz = a.dt * __ldg(a.M.bz + c) * vz;
                h1 = qx; h2 = qx; h3 = qz; h4 = qz;
                const bool own = i >= i0 && i < i0 + TX && j >= j0 && j < j0 + TZ;
                const int xs = xstrip(s, i), zs = zstrip(s, j);
                if (xs >= 0) {
                    const long long k = s.psx + (long long)j * 2 * s.P + xs;
                    const int pq = s.profx + i;
                    const float P1 = a.pml.x[0][k], P3 = a.pml.x[1][k];
                    h1 += a.pml.ax_h[pq] * (P1 + qx);
                    h3 += a.pml.ax_i[pq] * (P3 + qz);
                    if (own) {
                        a.n1[k] = a.pml.bx_h[pq] * (P1 + qx);
                        a.n3[k] = a.pml.bx_i[pq] * (P3 + qz);
                    }
                }
                if (zs >= 0) {
                    const long long k = s.psz + (long long)zs * s.NX + i;
                    const float P2 = a.pml.z[0][k], P4 = a.pml.z[1][k];
                    h2 += a.pml.az_i[j] * (P2 + qx);
                    h4 += a.pml.az_h[j] * (P4 + qz);
                    if (own) {
                        a.n2[k] = a.pml.bz_i[j] * (P2 + qx);
                        a.n4[k] = a.pml.bz_h[j] * (P4 + qz);
                    }
                }
                if (own) {
                    a.out.vx[c] = vx;
                    a.out.vz[c] = vz;
                    if (i >= s.P - 1 && i <= s.P + s.w && j >= s.P - 1 && j <= s.NZ - s.P) {
                        a.Gbx[c] += __ldg(a.vfx + c) * inc_x;
                        a.Gbz[c] += __ldg(a.vfz + c) * inc_z;
                    }
                }
            }
            e1s[q] = h1; e2s[q] = h2; e3s[q] = h3; e4s[q] = h4;
        }
        __syncthreads();

        // 3. sigma^ += D^T e^ on the tile, with the C-imaging
        for (int q = tid; q < TX * TZ; q += kThreads) {
            const int y = q / TX, x = q - y * TX;
            const int i = i0 + x, j = j0 + y;
            if (i >= s.NX || j >= s.NZ) continue;
            const long long c = cell_of(s, i, j);
            const float hxx = __ldg(a.in.sxx + c), hzz = __ldg(a.in.szz + c), hxz = __ldg(a.in.sxz + c);
            if (i >= s.P && i < s.P + s.w && j >= s.P && j < s.NZ - s.P) {
                const float fx = dbwd(a.vfx, c, 1) * a.rdx;
                const float fz = dbwd(a.vfz, c, P) * a.rdz;
                a.Glam[c] += a.dt * (hxx + hzz) * (fx + fz);
                a.Gmu[c] += 2.f * a.dt * (hxx * fx + hzz * fz);
            }
            if (i >= s.P - 1 && i < s.P + s.w && j >= s.P - 1 && j < s.NZ - s.P) {
                const float fxz = dfwd(a.vfx, c, P) * a.rdz + dfwd(a.vfz, c, 1) * a.rdx;
                a.Gmuxz[c] += a.dt * hxz * fxz;
            }
            const int o = (y + 2) * VX + (x + 2);
            a.out.sxx[c] = hxx - (C1 * (e1s[o] - e1s[o - 1]) + C2 * (e1s[o + 1] - e1s[o - 2])) * a.rdx;
            a.out.szz[c] = hzz - (C1 * (e4s[o] - e4s[o - VX]) + C2 * (e4s[o + VX] - e4s[o - 2 * VX])) * a.rdz;
            a.out.sxz[c] = hxz - (C1 * (e2s[o + VX] - e2s[o]) + C2 * (e2s[o + 2 * VX] - e2s[o - VX])) * a.rdz
                               - (C1 * (e3s[o + 1] - e3s[o]) + C2 * (e3s[o + 2] - e3s[o - 1])) * a.rdx;
        }
        __syncthreads();
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
size_t adj_smem(int tx, int tz) { return sizeof(float) * (4 * (tx + 8) * (tz + 8) + 4 * (tx + 4) * (tz + 4)); }

template <int TX, int TZ>
void fwd_launch(const FwdArgs &a, int grid, cudaStream_t st) {
    k_step_fused<TX, TZ><<<grid, kThreads, fwd_smem(TX, TZ), st>>>(a);
}
template <int TX, int TZ>
void adj_launch(const AdjArgsF &a, int grid, cudaStream_t st) {
    k_adj_fused<TX, TZ><<<grid, kThreads, adj_smem(TX, TZ), st>>>(a);
}

template <int TX, int TZ>
void set_attrs() {
    cudaFuncSetAttribute(k_step_fused<TX, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(TX, TZ));
    cudaFuncSetAttribute(k_adj_fused<TX, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_smem(TX, TZ));
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

std::vector<int4> make_tiles(efwi_plan *p, int tx, int tz) {
    std::vector<int4> t;
    for (int s = 0; s < p->d.ns; ++s) {
        const ShotDev &sh = p->shots[s];
        for (int j0 = 0; j0 < sh.NZ; j0 += tz)
            for (int i0 = 0; i0 < sh.NX; i0 += tx) t.push_back(make_int4(s, i0, j0, 0));
    }
    return t;
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

FwdArgs fwd_args(efwi_plan *p, int n, float *segx, float *segz) {
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
    a.nt = p->d.nt;
    a.n = n;
    a.dt = (float)p->d.dt;
    a.rdx = (float)(1.0 / p->d.dx);
    a.rdz = (float)(1.0 / p->d.dz);
    return a;
}

AdjArgsF adj_args_f(efwi_plan *p, const float *vfx, const float *vfz) {
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
    a.Glam = G_field(p, 0); a.Gmu = G_field(p, 1); a.Gmuxz = G_field(p, 2);
    a.Gbx = G_field(p, 3); a.Gbz = G_field(p, 4);
    a.dt = (float)p->d.dt;
    a.rdx = (float)(1.0 / p->d.dx);
    a.rdz = (float)(1.0 / p->d.dz);
    return a;
}

}  // namespace

void launch_step_fused(efwi_plan *p, int n, float *vseg_x, float *vseg_z, cudaStream_t st) {
    FwdArgs a = fwd_args(p, n, vseg_x, vseg_z);
    int slot;
    prof_begin(p, st, &slot, EFWI_KERNEL_STEP);
    EFWI_DISPATCH(p->tiles.tx, p->tiles.tz, fwd_launch, a, a.ntiles, st);
    prof_end(p, st, slot);
    p->launches++;
    p->scur ^= 1;
    p->psi_v ^= 1;
}

void launch_adj_fused(efwi_plan *p, int n, const float *vfx, const float *vfz, cudaStream_t st) {
    (void)n;
    AdjArgsF a = adj_args_f(p, vfx, vfz);
    int slot;
    prof_begin(p, st, &slot, EFWI_KERNEL_ADJ);
    EFWI_DISPATCH(p->adj_tiles.tx, p->adj_tiles.tz, adj_launch, a, a.ntiles, st);
    prof_end(p, st, slot);
    p->launches++;
    p->acur ^= 1;
    p->apsi_v ^= 1;
    p->apsi_s ^= 1;
}

}  // namespace efwi

using namespace efwi;

// Tile autotuner: times a few fused forward steps and adjoint steps of the
// plan's own shots for every compiled tile shape and keeps the fastest (the
// shapes change no arithmetic, only the work decomposition).
int efwi_autotune(efwi_plan *p) {
    set_all_attrs();
    const bool fixed = p->tile_x > 0 && p->tile_z > 0;
    if (fixed && !shape_ok(p->tile_x, p->tile_z)) {
        p->err = "tile shape not among the compiled shapes (32x8, 32x16, 64x8, 64x16, 32x32, 128x8, 64x32)";
        return EFWI_ERR_ARG;
    }
    if (fixed) {
        int rc = upload_tiles(p, p->tiles, p->tile_x, p->tile_z);
        if (!rc) rc = upload_tiles(p, p->adj_tiles, p->tile_x, p->tile_z);
        p->adj_tile_x = p->tile_x; p->adj_tile_z = p->tile_z;
        return rc;
    }
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_f = 1e30f, best_a = 1e30f;
    int bf = 0, ba = 0;
    const int reps = 3;
    for (int k = 0; k < kNumShapes; ++k) {
        const int tx = kShapes[k].tx, tz = kShapes[k].tz;
        if (upload_tiles(p, p->tiles, tx, tz) || upload_tiles(p, p->adj_tiles, tx, tz)) continue;
        float *vs_x = p->seg, *vs_z = p->seg + p->fsz_total;
        for (int w = 0; w < 2; ++w) {          // warm-up, then timed
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps; ++r) launch_step_fused(p, 0, vs_x, vs_z, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
        }
        float tf = 0;
        cudaEventElapsedTime(&tf, e0, e1);
        for (int w = 0; w < 2; ++w) {
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps; ++r) launch_adj_fused(p, 0, vs_x, vs_z, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
        }
        float ta = 0;
        cudaEventElapsedTime(&ta, e0, e1);
        if (tf < best_f) { best_f = tf; bf = k; }
        if (ta < best_a) { best_a = ta; ba = k; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    // the tuning runs touched workspace only; clear what the next call expects zeroed
    for (int k = 0; k < 2; ++k)
        if (p->state[k]) cudaMemset(p->state[k], 0, sizeof(float) * 5 * p->fsz_total);
    for (int k = 0; k < 2; ++k)
        if (p->adj[k]) cudaMemset(p->adj[k], 0, sizeof(float) * 5 * p->fsz_total);
    cudaMemset(p->psi, 0, sizeof(float) * 4 * p->H);
    cudaMemset(p->apsi, 0, sizeof(float) * 4 * p->H);
    cudaMemset(p->G, 0, sizeof(float) * 5 * p->fsz_total);
    cudaMemset(p->seg, 0, sizeof(float) * 2 * p->fsz_total);
    p->scur = p->acur = p->psi_v = p->psi_s = p->apsi_v = p->apsi_s = 0;
    p->launches = 0;
    p->tile_x = kShapes[bf].tx; p->tile_z = kShapes[bf].tz;
    p->adj_tile_x = kShapes[ba].tx; p->adj_tile_z = kShapes[ba].tz;
    int rc = upload_tiles(p, p->tiles, p->tile_x, p->tile_z);
    if (!rc) rc = upload_tiles(p, p->adj_tiles, p->adj_tile_x, p->adj_tile_z);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        p->err = std::string("autotune: ") + cudaGetErrorString(e);
        return EFWI_ERR_CUDA;
    }
    return rc;
}
