// Adjoint step in scaled-stress form (k_adj_scaled): the transposed time step of
// k_adj_fused with the adjoint stress carried as F = dt C sigma^ (C the stiffness
// of the cell: lambda + 2 mu / lambda on the normal stresses, mu_xz on the shear)
// instead of sigma^ itself.
//
// Why: in the transposed step the adjoint stresses enter the velocity sub-step
// only through dt C sigma^ (plus the CPML memory), so the stress form first
// multiplies sigma^ by C on the tile + 4-cell halo (six loads per halo cell,
// lambda, mu and mu_xz included) and later reads sigma^ of the tile again for
// its update.  Carrying F makes the step the forward step's shape: per TX x TZ
// tile of one shot,
//   1. F of the tile + 4-cell halo into shared memory (three loads per cell; on
//      tiles whose halo touches a CPML strip, the stress-sub-step adjoint CPML
//      terms are added and that memory advances, with the expressions of the
//      stress form with dt C sigma^ replaced by F);
//   2. v^ += D^T F on the tile + 2-cell halo, e^ = dt b v^ (+ CPML) in shared
//      memory, b-imaging -- unchanged;
//   3. F += dt C (-D^T e^) on the tile, with lambda, mu, mu_xz read on the tile
//      only, and the zero-lag imaging in F:
//        A  += (F_xx + F_zz)(d_x v_x + d_z v_z)
//        B  += (F_xx - F_zz)(d_x v_x - d_z v_z)
//        Cs += F_xz (d_z v_x + d_x v_z)
//      with v the forward velocities of the step.
// Since F = dt C sigma^ and C is constant in time, the stress form's sums follow
// once per gradient (k_imag_unscale):
//   G_lambda = A / (2 (lambda + mu)),  G_mu = G_lambda + B / (2 mu),  G_mu_xz = Cs / mu_xz,
// which needs mu > 0 and lambda + mu > 0 (Vs > 0 and Vp > Vs) wherever the imaging
// sums live; the materials kernel flags a model without that.  Results equal the
// stress form's up to FP32 rounding (the tests bound the difference); all tile
// shapes of this form give bitwise-identical results.
#include <algorithm>
#include <type_traits>

#include "plan.hpp"
#include "tma.cuh"
#include "adj_args.cuh"

namespace efwi {
namespace {

constexpr int kThreads = 256;

template <int TX, int TZ>
struct ScaledLayout {
    static constexpr int SX = TX + 8, SZ = TZ + 8, VX = TX + 4, VZ = TZ + 4, NT = TX * TZ;
    static constexpr int H4 = SX * SZ, H2 = VX * VZ;
    // f1..f4 (halo 4), e1..e4, forward vx, vz (halo 2), F of the tile (3 x NT, edge tiles)
    static constexpr int FLOATS = 4 * H4 + 6 * H2 + 3 * NT;
    static constexpr size_t smem() { return sizeof(float) * FLOATS; }
};

template <int TX, int TZ, int SK = 0>
__global__ void __launch_bounds__(kThreads, TX * TZ <= 512 ? 4 : 2) k_adj_scaled(AdjArgsF a) {
    // SK: the forward velocities are FP32 (0) or FP16 / BF16 snapshots
    using L = ScaledLayout<TX, TZ>;
    constexpr int SX = L::SX, SZ = L::SZ, VX = L::VX, VZ = L::VZ;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *f1s = sm, *f2s = sm + L::H4, *f3s = sm + 2 * L::H4, *f4s = sm + 3 * L::H4;
    float *e1s = sm + 4 * L::H4, *e2s = e1s + L::H2, *e3s = e2s + L::H2, *e4s = e3s + L::H2;
    float *vfxs = e4s + L::H2, *vfzs = vfxs + L::H2;   // forward v^{n+1/2} on the tile + 2-cell halo
    float *txx = vfzs + L::H2, *tzz = txx + L::NT, *txz = tzz + L::NT;   // F of the tile (edge tiles)
    const int tid = threadIdx.x;

    // persistent grid: the next tile's work item and its shot's block offset and row
    // pitch are loaded one tile ahead
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
        auto tile = [&](auto edge_c) {
            const ShotDev *sp = a.shots + tl.x;
            const int NX = sp->NX, NZ = sp->NZ, PP = sp->P, profx = sp->profx, w = sp->w;
            const long long psx = sp->psx, psz = sp->psz;
            constexpr bool edge = decltype(edge_c)::value;   // 4-cell halo touches a strip or the grid edge
            const int i0 = tl.y, j0 = tl.z;
            const float dt = a.dt, rdx = a.rdx, rdz = a.rdz;
            const float dnx = SK ? snap_scale_down(a.sr.hmax, 0, tl.x, a.sr.ns) : 1.f;
            const float dnz = SK ? snap_scale_down(a.sr.hmax, 1, tl.x, a.sr.ns) : 1.f;

            // 1. F on the tile + 4-cell halo; on edge tiles the CPML terms and the
            //    tile's stress-sub-step adjoint CPML memory
            constexpr int N1 = (SX * SZ + kThreads - 1) / kThreads;
            float lxx[N1], lzz[N1], lxz[N1];
#pragma unroll
            for (int r = 0; r < N1; ++r) {
                const int q = tid + r * kThreads;
                lxx[r] = lzz[r] = lxz[r] = 0.f;
                const int y = q / SX, x = q - y * SX;
                const int i = i0 - 4 + x, j = j0 - 4 + y;
                if (q < SX * SZ && (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ))) {
                    const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    lxx[r] = ldg256(a.in.sxx + c); lzz[r] = ldg256(a.in.szz + c); lxz[r] = ldg256(a.in.sxz + c);
                }
            }
#pragma unroll
            for (int r = 0; r < N1; ++r) {
                const int q = tid + r * kThreads;
                if (q >= SX * SZ) break;
                if constexpr (!edge) {
                    f1s[q] = lxx[r]; f2s[q] = lzz[r]; f3s[q] = lxz[r];   // f^4 == f^3 away from the CPML
                } else {
                    const int y = q / SX, x = q - y * SX;
                    const int i = i0 - 4 + x, j = j0 - 4 + y;
                    float g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f;
                    if (i >= 0 && i < NX && j >= 0 && j < NZ) {
                        const float Ex = lxx[r], Ez = lzz[r], Exz = lxz[r];
                        g1 = Ex; g2 = Ez; g3 = Exz; g4 = Exz;
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
                        if (own) {
                            const int u = (y - 4) * TX + (x - 4);
                            txx[u] = Ex; tzz[u] = Ez; txz[u] = Exz;
                        }
                    }
                    f1s[q] = g1; f2s[q] = g2; f3s[q] = g3; f4s[q] = g4;
                }
            }
            __syncthreads();

            // 2. v^ += D^T f^ on the tile + 2-cell halo; e^ in shared memory (as the stress form)
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

            // 3. F += dt C (-D^T e^) on the tile, with the imaging in F
            constexpr int N3 = (TX * TZ + kThreads - 1) / kThreads;
            float lam_r[N3], mu_r[N3], mxz_r[N3], g0[N3], g1v[N3], g2v[N3];
#pragma unroll
            for (int r = 0; r < N3; ++r) {
                const int q = tid + r * kThreads;
                const int y = q / TX, x = q - y * TX;
                const int i = i0 + x, j = j0 + y;
                lam_r[r] = mu_r[r] = mxz_r[r] = g0[r] = g1v[r] = g2v[r] = 0.f;
                if (q < TX * TZ && !(edge && (i >= NX || j >= NZ))) {
                    const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    lam_r[r] = ldg256(a.M.lam + c); mu_r[r] = ldg256(a.M.mu + c); mxz_r[r] = ldg256(a.M.muxz + c);
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
                const int oh = (y + 4) * SX + (x + 4);     // (i, j) in the halo-4 staging
                const float Fxx = edge ? txx[q] : f1s[oh];
                const float Fzz = edge ? tzz[q] : f2s[oh];
                const float Fxz = edge ? txz[q] : f3s[oh];
                const int o = (y + 2) * VX + (x + 2);      // (i, j) in the halo-2 staging
                const float *fvx = vfxs + o, *fvz = vfzs + o;
                if (!edge || (i >= PP && i < PP + w && j >= PP && j < NZ - PP)) {
                    const float fx = (C1 * (fvx[0] - fvx[-1]) + C2 * (fvx[1] - fvx[-2])) * rdx;
                    const float fz = (C1 * (fvz[0] - fvz[-VX]) + C2 * (fvz[VX] - fvz[-2 * VX])) * rdz;
                    a.Glam[c] = g0[r] + (Fxx + Fzz) * (fx + fz);
                    a.Gmu[c] = g1v[r] + (Fxx - Fzz) * (fx - fz);
                }
                if (!edge || (i >= PP - 1 && i < PP + w && j >= PP - 1 && j < NZ - PP)) {
                    const float fxz = (C1 * (fvx[VX] - fvx[0]) + C2 * (fvx[2 * VX] - fvx[-VX])) * rdz +
                                      (C1 * (fvz[1] - fvz[0]) + C2 * (fvz[2] - fvz[-1])) * rdx;
                    a.Gmuxz[c] = g2v[r] + Fxz * fxz;
                }
                const float dxx = -(C1 * (e1s[o] - e1s[o - 1]) + C2 * (e1s[o + 1] - e1s[o - 2])) * rdx;
                const float dzz = -(C1 * (e4r[o] - e4r[o - VX]) + C2 * (e4r[o + VX] - e4r[o - 2 * VX])) * rdz;
                const float dxz = -(C1 * (e2r[o + VX] - e2r[o]) + C2 * (e2r[o + 2 * VX] - e2r[o - VX])) * rdz
                                  - (C1 * (e3s[o + 1] - e3s[o]) + C2 * (e3s[o + 2] - e3s[o - 1])) * rdx;
                const float lam = lam_r[r], l2m = lam + 2.f * mu_r[r];
                a.out.sxx[c] = Fxx + dt * (l2m * dxx + lam * dzz);
                a.out.szz[c] = Fzz + dt * (lam * dxx + l2m * dzz);
                a.out.sxz[c] = Fxz + dt * (mxz_r[r] * dxz);
            }
            __syncthreads();
        };
        if (tl.w & 4) tile(std::true_type{});
        else tile(std::false_type{});
    }
}

// The stress form's imaging sums from the scaled form's (in place, every cell of
// every shot block; cells without an imaging sum hold zeros and stay zero).
__global__ void k_imag_unscale(float *Glam, float *Gmu, float *Gmuxz, Mat M, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const float A = Glam[c], B = Gmu[c], Cs = Gmuxz[c];
        const float lam = M.lam[c], mu = M.mu[c];
        const float gl = A == 0.f ? 0.f : A / (2.f * (lam + mu));
        Glam[c] = gl;
        Gmu[c] = gl + (B == 0.f ? 0.f : B / (2.f * mu));
        Gmuxz[c] = Cs == 0.f ? 0.f : Cs / M.muxz[c];
    }
}

template <int TX, int TZ>
void launch_sk(const AdjArgsF &a, int grid, cudaStream_t st, int sk) {
    constexpr size_t sm = ScaledLayout<TX, TZ>::smem();
    if (sk == EFWI_STORE_FP16) k_adj_scaled<TX, TZ, EFWI_STORE_FP16><<<grid, kThreads, sm, st>>>(a);
    else if (sk == EFWI_STORE_BF16) k_adj_scaled<TX, TZ, EFWI_STORE_BF16><<<grid, kThreads, sm, st>>>(a);
    else k_adj_scaled<TX, TZ><<<grid, kThreads, sm, st>>>(a);
}

template <int TX, int TZ>
void attrs() {
    constexpr int sm = (int)ScaledLayout<TX, TZ>::smem();
    cudaFuncSetAttribute(k_adj_scaled<TX, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_adj_scaled<TX, TZ, EFWI_STORE_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_adj_scaled<TX, TZ, EFWI_STORE_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <int TX, int TZ>
int blocks(int sk) {
    constexpr size_t sm = ScaledLayout<TX, TZ>::smem();
    int nb = 0;
    if (sk == EFWI_STORE_FP16)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_scaled<TX, TZ, EFWI_STORE_FP16>, kThreads, sm);
    else if (sk == EFWI_STORE_BF16)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_scaled<TX, TZ, EFWI_STORE_BF16>, kThreads, sm);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_scaled<TX, TZ>, kThreads, sm);
    return nb;
}

#define EFWI_SCALED_DISPATCH(tx, tz, FN, ...)                           \
    (tx == 32 && tz == 8    ? FN<32, 8>(__VA_ARGS__)                    \
     : tx == 64 && tz == 8  ? FN<64, 8>(__VA_ARGS__)                    \
     : tx == 64 && tz == 16 ? FN<64, 16>(__VA_ARGS__)                   \
                            : FN<32, 16>(__VA_ARGS__))

}  // namespace

bool adj_scaled_shape_ok(int tx, int tz) {
    return (tx == 32 && (tz == 8 || tz == 16)) || (tx == 64 && (tz == 8 || tz == 16));
}

void adj_scaled_set_attrs() {
    static bool done = false;
    if (done) return;
    done = true;
    attrs<32, 8>(); attrs<32, 16>(); attrs<64, 8>(); attrs<64, 16>();
}

int adj_scaled_blocks_per_sm(int tx, int tz, int snap_store) {
    adj_scaled_set_attrs();
    return EFWI_SCALED_DISPATCH(tx, tz, blocks, snap_store);
}

void launch_adj_scaled(efwi_plan *p, const SnapIn &si, cudaStream_t st) {
    AdjArgsF a = adj_args_f(p, si);
    a.pf = 0;
    const int grid = p->grid_adj_override > 0 ? std::min(p->grid_adj_override, a.ntiles)
                     : p->adj_grid > 0        ? std::min(p->adj_grid, a.ntiles)
                                              : a.ntiles;
    const int tx = p->adj_tiles.tx, tz = p->adj_tiles.tz;
    if (tx == 32 && tz == 8) launch_sk<32, 8>(a, grid, st, p->snap_store);
    else if (tx == 64 && tz == 8) launch_sk<64, 8>(a, grid, st, p->snap_store);
    else if (tx == 64 && tz == 16) launch_sk<64, 16>(a, grid, st, p->snap_store);
    else launch_sk<32, 16>(a, grid, st, p->snap_store);
}

void launch_imag_unscale(efwi_plan *p, float *G, cudaStream_t st) {
    const long long n = p->fsz_total;
    const int grid = (int)std::min<long long>((n + 255) / 256, 16LL * std::max(p->n_sms, 1));
    k_imag_unscale<<<grid, 256, 0, st>>>(G, G + n, G + 2 * n, materials(p), n);
    p->launches++;
}

}  // namespace efwi
