// Adjoint step in scaled-stress form with TMA staging (k_adj_scaled_tma): the step of
// k_adjs.cu (adjoint stresses carried as F = dt C sigma^) on a persistent grid whose
// CTAs copy every input of a tile into shared memory with cp.async.bulk.tensor, one
// tile ahead (two stages completing on mbarriers):
//   * v^x, v^z, b_x, b_z and the forward v_x, v_z of the step (FP32, or the 2-byte
//     FP16/BF16 snapshot elements, scaled when read) on the tile + 4-cell halo
//     in x and the tile + 2 rows in z, F_xx on the same rows, F_zz and F_xz on the rows
//     the velocity sub-step reads (tile + 3 rows on one side, 4 on the other);
//   * lambda, mu, mu_xz and the five imaging sums on the tile.
// A tile then computes from shared memory only: on tiles whose halo touches a CPML
// strip, the stress-sub-step CPML terms are added to the staged F in place (the tile's
// F kept for its update); v^ += D^T F on the tile + 2-cell halo with e^ = dt b v^ (+
// CPML) written over the staged v^; F += dt C (-D^T e^) on the tile with the imaging.
// Every expression is k_adj_scaled's, so both give bitwise-identical results; so does the
// cell-pair layout (VEC = 2), whose adjacent x-stencils share 64-bit shared-memory loads.
// Out-of-range box elements are zero-filled by the copy engine, as the zero ghosts of
// the layout.  Every mbarrier wait is bounded; on expiry the CTA records the error,
// waits (bounded) for the copy it still has in flight and returns.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "plan.hpp"
#include "tma.cuh"
#include "adj_args.cuh"

namespace efwi {
namespace {

constexpr int kThreads = 256;

struct TmaAdjsArgs {
    const ShotDev *shots;
    const int4 *tiles;
    const AdjsMaps *maps;
    int ntiles;
    int af;                     // first field of the read adjoint buffer in the adjoint-state maps
    int vf;                     // first field of this step's forward velocities in the segment map
    Fields out;                 // adjoint buffer written
    Pml pml;                    // current adjoint PML memory (V and S blocks, read)
    float *n1, *n3, *n2, *n4;   // next V block
    float *n5, *n8, *n6, *n7;   // next S block
    float *Glam, *Gmu, *Gmuxz, *Gbx, *Gbz;
    float dt, rdx, rdz;
    int *err;
    const float *hmax;          // snapshot maxima of the step (SK != 0): the power-of-two scales
    int ns;
};

// One stage (halo-4 coordinates: column x = cell i - i0 + 4, row y = cell j - j0 + 4):
// R2 arrays hold rows 2 .. TZ+5, F_zz rows 1 .. TZ+7, F_xz rows 0 .. TZ+6 (R3 rows each,
// padded to 128 bytes); tile arrays TX x TZ.  Every array starts 128-byte aligned.
template <int TX, int TZ, int SK>
struct AdjsLayout {
    static constexpr int SX = TX + 8;
    static constexpr int R2 = TZ + 4, R3 = TZ + 7;
    static constexpr int A2 = SX * R2;
    static constexpr int A3 = SX * R3, A3P = (A3 + 31) & ~31;
    static constexpr int NC = TX * TZ;
    // forward velocities: FP32, or 2-byte FP16/BF16 snapshot elements (SK != 0)
    static constexpr int WB = SK ? 2 : 4, AW = A2 * WB / 4;                    // floats of one of them
    static constexpr int OVX = 0, OVZ = A2, OFXX = 2 * A2, OFZZ = 3 * A2, OFXZ = OFZZ + A3P, OBX = OFXZ + A3P,
                         OBZ = OBX + A2, OWX = OBZ + A2, OWZ = OWX + AW, OLAM = (OWZ + AW + 31) & ~31,
                         OG = OLAM + 3 * NC;
    static constexpr int BUF = (OG + 5 * NC + 31) & ~31;                      // floats per stage
    static constexpr unsigned LOADED = (5u * A2 + 2u * A3 + 8u * NC) * 4u + 2u * A2 * WB;   // bytes the copies bring
    // per CTA, edge tiles only: F_xz with its x-strip CPML term (g4), e^2, e^4 (R2 rows)
    // and F of the tile before its update
    static constexpr int EXTRA = 3 * A2 + 3 * NC;
    static constexpr size_t smem() { return (2 * (size_t)BUF + EXTRA) * 4 + 128; }
    static_assert(A2 % 32 == 0 && NC % 32 == 0, "arrays must keep 128-byte alignment");
};

// tl: the tile's work item, already in a register (no global load on the issuing thread's
// path between the tile's barriers)
template <int TX, int TZ, int SK>
__device__ __forceinline__ void issue_adjs(const TmaAdjsArgs &a, const int4 tl, float *buf, uint64_t *bar) {
    using L = AdjsLayout<TX, TZ, SK>;
    const AdjsMaps *m = a.maps + tl.x;
    mbar_expect_tx(bar, L::LOADED);
    // element x = cell i + GX (halo-4 column 0 = cell i0 - 4), row y = cell j + GZ: halo-4 row r
    // of the tile is map row j0 - 4 + r + GZ = tl.z - 2 + r
    tma_load_3d(buf + L::OVX, &m->a2, bar, tl.y, tl.z, a.af);            // v^x, v^z: rows 2..
    tma_load_3d(buf + L::OFXX, &m->a1, bar, tl.y, tl.z, a.af + 2);       // F_xx: rows 2..
    tma_load_3d(buf + L::OFZZ, &m->a3, bar, tl.y, tl.z - 1, a.af + 3);   // F_zz: rows 1..
    tma_load_3d(buf + L::OFXZ, &m->a3, bar, tl.y, tl.z - 2, a.af + 4);   // F_xz: rows 0..
    tma_load_3d(buf + L::OBX, &m->mb, bar, tl.y, tl.z, 3);               // b_x, b_z: rows 2..
    tma_load_3d(buf + L::OWX, &m->sv, bar, tl.y, tl.z, a.vf);            // forward v_x, v_z: rows 2..
    tma_load_3d(buf + L::OLAM, &m->mc, bar, tl.y + 4, tl.z + 2, 0);      // lambda, mu, mu_xz: tile
    tma_load_3d(buf + L::OG, &m->gi, bar, tl.y + 4, tl.z + 2, 0);        // imaging sums: tile
}

// A 2-byte snapshot element as a float (the conversion of the per-thread-load kernels).
template <int SK>
__device__ __forceinline__ float h2f(unsigned short u) {
    if constexpr (SK == EFWI_STORE_FP16) return __half2float(__ushort_as_half(u));
    else return __bfloat162float(__ushort_as_bfloat16(u));
}

// Read access to a tile's staged forward velocity: FP32 (SK = 0), or 2-byte FP16/BF16
// snapshot elements times the snapshot's power-of-two scale s, the value the per-thread
// kernels compute from the same element.  at(base, o0, s): element o0 of the array that
// starts at base (shared memory).
template <int SK>
struct FvView {
    using T = typename std::conditional<SK == 0, float, unsigned short>::type;
    const T *p;
    float s;
    __device__ __forceinline__ static FvView at(const float *base, int o0, float s) {
        return {reinterpret_cast<const T *>(base) + o0, s};
    }
    __device__ __forceinline__ FvView operator+(int o) const { return {p + o, s}; }
    __device__ __forceinline__ float operator[](int o) const {
        if constexpr (SK == 0) return p[o];
        else return h2f<SK>(p[o]) * s;
    }
    __device__ __forceinline__ float2 pair(int o) const {   // elements o, o + 1; o even
        if constexpr (SK == 0) {
            return ld2(p + o);
        } else {
            const unsigned int w = *reinterpret_cast<const unsigned int *>(p + o);
            return make_float2(h2f<SK>((unsigned short)(w & 0xffffu)) * s, h2f<SK>((unsigned short)(w >> 16)) * s);
        }
    }
};

// C1 (a - b) + C2 (c - d): the 4th-order staggered difference, one rounding per operation
__device__ __forceinline__ float st4(float a, float b, float c, float d) { return C1 * (a - b) + C2 * (c - d); }

// VEC = 1: one cell per thread and iteration; VEC = 2: cell pairs with 64-bit shared-memory
// accesses (one pair of the tile per thread, the velocity halo ring as single cells)
// NT: threads per CTA: 256, or 512 with cell pairs (the tile's pairs and the halo ring on separate
// threads: 32 warps per SM at the same shared memory)
template <int TX, int TZ, int VEC, int SK, int NT = kThreads>
__global__ void __launch_bounds__(NT, 2) k_adj_scaled_tma(TmaAdjsArgs a) {
    static_assert(NT == kThreads || (VEC == 2 && (TX / 2) * TZ + 4 * (TX + 4) + 4 * TZ <= NT),
                  "512-thread CTAs: one tile pair or one ring cell per thread");
    using L = AdjsLayout<TX, TZ, SK>;
    constexpr int SX = L::SX, NC = L::NC;
    extern __shared__ float4 smem_raw[];
    float *smb = align128(smem_raw);
    float *xg4 = smb + 2 * L::BUF, *xe2 = xg4 + L::A2, *xe4 = xe2 + L::A2;
    float *txx = xe4 + L::A2, *tzz = txx + NC, *txz = tzz + NC;
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int ok_s;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    int t = blockIdx.x;
    int4 tl_next = t < a.ntiles ? __ldg(a.tiles + t) : make_int4(0, 0, 0, 0);
    if (tid == 0 && t < a.ntiles) issue_adjs<TX, TZ, SK>(a, tl_next, smb, &bar[0]);
    // the work item of the tile the next refill copies (thread 0), loaded one tile ahead
    int4 tl_fill = make_int4(0, 0, 0, 0);
    if (tid == 0 && t + (int)gridDim.x < a.ntiles) tl_fill = __ldg(a.tiles + t + gridDim.x);
    for (int k = 0; t < a.ntiles; t += gridDim.x, ++k) {
        const int b = k & 1;
        float *buf = smb + b * L::BUF;
        const int4 tl = tl_next;
        const ShotDev *sp = a.shots + tl.x;
        const int NX = __ldg(&sp->NX), NZ = __ldg(&sp->NZ), PP = __ldg(&sp->P), profx = __ldg(&sp->profx),
                  pitch = __ldg(&sp->pitch), w = __ldg(&sp->w);
        const long long off = __ldg(&sp->off), psx = __ldg(&sp->psx), psz = __ldg(&sp->psz);
        // power-of-two scales of the shot's reduced-precision snapshot (loaded before the wait)
        const float dnx = SK ? snap_scale_down(a.hmax, 0, tl.x, a.ns) : 1.f;
        const float dnz = SK ? snap_scale_down(a.hmax, 1, tl.x, a.ns) : 1.f;
        if (t + (int)gridDim.x < a.ntiles) tl_next = __ldg(a.tiles + t + gridDim.x);
        if (tid == 0) ok_s = mbar_wait_bounded(&bar[b], (phase >> b) & 1u);
        __syncthreads();
        if (!ok_s) {
            if (tid == 0) {
                atomicOr(a.err, EFWI_FLAG_TIMEOUT);
                // the copy in flight is this tile's (the next tile's is issued after the wait);
                // no copy is issued after this point
                mbar_drain_bounded(bar, phase, k, 2, 1);
            }
            return;
        }
        mbar_wait_bounded(&bar[b], (phase >> b) & 1u);   // completed: acquire for every thread
        phase ^= 1u << b;
        // refill the other stage with the CTA's next tile: every thread has passed the barrier
        // above, so none still reads that stage (it held the previous tile)
        if (tid == 0 && t + (int)gridDim.x < a.ntiles) {
            issue_adjs<TX, TZ, SK>(a, tl_fill, smb + (b ^ 1) * L::BUF, &bar[b ^ 1]);   // tile t + gridDim.x
            if (t + 2 * (int)gridDim.x < a.ntiles) tl_fill = __ldg(a.tiles + t + 2 * gridDim.x);
        }

        auto tile = [&](auto edge_c) {
            constexpr bool edge = decltype(edge_c)::value;   // 4-cell halo touches a strip or the grid edge
            const int i0 = tl.y, j0 = tl.z;
            const float dt = a.dt, rdx = a.rdx, rdz = a.rdz;
            // base pointers in halo-4 coordinates (element y * SX + x), offset by each array's first row
            float *svx = buf + L::OVX - 2 * SX, *svz = buf + L::OVZ - 2 * SX;
            float *fxx = buf + L::OFXX - 2 * SX, *fzz = buf + L::OFZZ - SX, *fxz = buf + L::OFXZ;
            const float *sbx = buf + L::OBX - 2 * SX, *sbz = buf + L::OBZ - 2 * SX;
            const FvView<SK> wvx = FvView<SK>::at(buf + L::OWX, -2 * SX, dnx),
                             wvz = FvView<SK>::at(buf + L::OWZ, -2 * SX, dnz);
            const float *slam = buf + L::OLAM, *smu = slam + NC, *smxz = smu + NC;
            const float *sg = buf + L::OG;                    // [5][NC]: lambda, mu, mu_xz, b_x, b_z sums
            float *g4 = edge ? xg4 - 2 * SX : fxz;            // f^4 == f^3 away from the CPML
            float *e2w = edge ? xe2 - 2 * SX : svx;           // e^2 == e^1, e^4 == e^3 away from the CPML
            float *e4w = edge ? xe4 - 2 * SX : svz;

            // 1. edge tiles: the stress-sub-step CPML terms over the staged F, in place, and the
            //    tile's stress-sub-step adjoint CPML memory; F of the tile kept for its update
            if constexpr (edge) {
                for (int q = tid; q < SX * (TZ + 8); q += NT) {
                    const int y = q / SX, x = q - y * SX;
                    const int i = i0 - 4 + x, j = j0 - 4 + y;
                    const int o = y * SX + x;
                    const bool rxx = y >= 2 && y < TZ + 6, rzz = y >= 1, rxz = y < TZ + 7;
                    if (!(i >= 0 && i < NX && j >= 0 && j < NZ)) {
                        if (rxx) g4[o] = 0.f;       // the staged F is zero there (ghosts, fill)
                        continue;
                    }
                    const float Ex = rxx ? fxx[o] : 0.f, Ez = rzz ? fzz[o] : 0.f, Exz = rxz ? fxz[o] : 0.f;
                    float g1 = Ex, g2 = Ez, g3 = Exz, gg4 = Exz;
                    const bool own = x >= 4 && x < TX + 4 && y >= 4 && y < TZ + 4;
                    const int xs = i < PP ? i : (i >= NX - PP ? i - NX + 2 * PP : -1);
                    const int zs = j < PP ? j : (j >= NZ - PP ? j - NZ + 2 * PP : -1);
                    if (xs >= 0) {
                        const long long kk = psx + (long long)j * 2 * PP + xs;
                        const int pq = profx + i;
                        const float P5 = a.pml.x[2][kk], P8 = a.pml.x[3][kk];
                        g1 += a.pml.ax_i[pq] * (P5 + Ex);
                        gg4 += a.pml.ax_h[pq] * (P8 + Exz);
                        if (own) {
                            a.n5[kk] = a.pml.bx_i[pq] * (P5 + Ex);
                            a.n8[kk] = a.pml.bx_h[pq] * (P8 + Exz);
                        }
                    }
                    if (zs >= 0) {
                        const long long kk = psz + (long long)zs * NX + i;
                        const float P6 = a.pml.z[2][kk], P7 = a.pml.z[3][kk];
                        g2 += a.pml.az_i[j] * (P6 + Ez);
                        g3 += a.pml.az_h[j] * (P7 + Exz);
                        if (own) {
                            a.n6[kk] = a.pml.bz_i[j] * (P6 + Ez);
                            a.n7[kk] = a.pml.bz_h[j] * (P7 + Exz);
                        }
                    }
                    if (own) {
                        const int u = (y - 4) * TX + (x - 4);
                        txx[u] = Ex; tzz[u] = Ez; txz[u] = Exz;
                    }
                    if (rxx) { fxx[o] = g1; g4[o] = gg4; }
                    if (rzz) fzz[o] = g2;
                    if (rxz) fxz[o] = g3;
                }
                __syncthreads();
            }

            // the velocity-sub-step adjoint CPML terms of cell (i, j) and, for an own cell, its memory
            auto vel_pml = [&](const int i, const int j, const bool own, const float qx, const float qz, float &h1,
                               float &h2, float &h3, float &h4) {
                const int xs = i < PP ? i : (i >= NX - PP ? i - NX + 2 * PP : -1);
                const int zs = j < PP ? j : (j >= NZ - PP ? j - NZ + 2 * PP : -1);
                if (xs >= 0) {
                    const long long kk = psx + (long long)j * 2 * PP + xs;
                    const int pq = profx + i;
                    const float P1 = a.pml.x[0][kk], P3 = a.pml.x[1][kk];
                    h1 += a.pml.ax_h[pq] * (P1 + qx);
                    h3 += a.pml.ax_i[pq] * (P3 + qz);
                    if (own) {
                        a.n1[kk] = a.pml.bx_h[pq] * (P1 + qx);
                        a.n3[kk] = a.pml.bx_i[pq] * (P3 + qz);
                    }
                }
                if (zs >= 0) {
                    const long long kk = psz + (long long)zs * NX + i;
                    const float P2 = a.pml.z[0][kk], P4 = a.pml.z[1][kk];
                    h2 += a.pml.az_i[j] * (P2 + qx);
                    h4 += a.pml.az_h[j] * (P4 + qz);
                    if (own) {
                        a.n2[kk] = a.pml.bz_i[j] * (P2 + qx);
                        a.n4[kk] = a.pml.bz_h[j] * (P4 + qz);
                    }
                }
            };
            // the cell pair (x, x+1) of the tile at halo-4 row y, x even: every cell's expression
            // is vcell's, term by term
            auto vpair = [&](const int x, const int y) {
                const int i = i0 - 4 + x, j = j0 - 4 + y;
                const int o = y * SX + x;
                const float2 a0 = ld2(fxx + o - 2), a1 = ld2(fxx + o), a2 = ld2(fxx + o + 2);
                const float2 zm2 = ld2(fxz + o - 2 * SX), zm1 = ld2(fxz + o - SX), z0 = ld2(fxz + o),
                             zp1 = ld2(fxz + o + SX);
                const float2 cm1 = ld2(fzz + o - SX), c0 = ld2(fzz + o), cp1 = ld2(fzz + o + SX),
                             cp2 = ld2(fzz + o + 2 * SX);
                const float2 b0 = ld2(g4 + o - 2), b1 = ld2(g4 + o), b2 = ld2(g4 + o + 2);
                float inc_x[2], inc_z[2];
                inc_x[0] = -st4(a1.y, a1.x, a2.x, a0.y) * rdx - st4(z0.x, zm1.x, zp1.x, zm2.x) * rdz;
                inc_x[1] = -st4(a2.x, a1.y, a2.y, a1.x) * rdx - st4(z0.y, zm1.y, zp1.y, zm2.y) * rdz;
                inc_z[0] = -st4(cp1.x, c0.x, cp2.x, cm1.x) * rdz - st4(b1.x, b0.y, b1.y, b0.x) * rdx;
                inc_z[1] = -st4(cp1.y, c0.y, cp2.y, cm1.y) * rdz - st4(b1.y, b1.x, b2.x, b0.y) * rdx;
                const float2 vxo = ld2(svx + o), vzo = ld2(svz + o), bxo = ld2(sbx + o), bzo = ld2(sbz + o);
                const float vx[2] = {vxo.x + inc_x[0], vxo.y + inc_x[1]};
                const float vz[2] = {vzo.x + inc_z[0], vzo.y + inc_z[1]};
                const float bxv[2] = {bxo.x, bxo.y}, bzv[2] = {bzo.x, bzo.y};
                float h1[2], h2[2], h3[2], h4[2];
                bool in[2] = {true, true};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float qx = dt * bxv[h] * vx[h], qz = dt * bzv[h] * vz[h];
                    h1[h] = qx; h2[h] = qx; h3[h] = qz; h4[h] = qz;
                    if (edge) {
                        in[h] = i + h < NX && j < NZ;
                        if (in[h]) vel_pml(i + h, j, true, qx, qz, h1[h], h2[h], h3[h], h4[h]);
                        else h1[h] = h2[h] = h3[h] = h4[h] = 0.f;
                    }
                }
                const long long c = off + (long long)(j + EFWI_GZ) * pitch + (i + EFWI_GX);
                const int u = (y - 4) * TX + (x - 4);
                const float2 gbx = ld2(sg + 3 * NC + u), gbz = ld2(sg + 4 * NC + u);
                const float2 fvx = wvx.pair(o), fvz = wvz.pair(o);
                if (!edge) {
                    st2g(a.out.vx + c, make_float2(vx[0], vx[1]));
                    st2g(a.out.vz + c, make_float2(vz[0], vz[1]));
                    st2g(a.Gbx + c, make_float2(gbx.x + fvx.x * inc_x[0], gbx.y + fvx.y * inc_x[1]));
                    st2g(a.Gbz + c, make_float2(gbz.x + fvz.x * inc_z[0], gbz.y + fvz.y * inc_z[1]));
                } else {
                    const float gbxv[2] = {gbx.x, gbx.y}, gbzv[2] = {gbz.x, gbz.y};
                    const float fvxv[2] = {fvx.x, fvx.y}, fvzv[2] = {fvz.x, fvz.y};
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (!in[h]) continue;
                        const int ih = i + h;
                        a.out.vx[c + h] = vx[h];
                        a.out.vz[c + h] = vz[h];
                        if (ih >= PP - 1 && ih <= PP + w && j >= PP - 1 && j <= NZ - PP) {
                            a.Gbx[c + h] = gbxv[h] + fvxv[h] * inc_x[h];
                            a.Gbz[c + h] = gbzv[h] + fvzv[h] * inc_z[h];
                        }
                    }
                }
                st2(svx + o, make_float2(h1[0], h1[1]));
                st2(svz + o, make_float2(h3[0], h3[1]));
                if (edge) {
                    st2(e2w + o, make_float2(h2[0], h2[1]));
                    st2(e4w + o, make_float2(h4[0], h4[1]));
                }
            };

            // 2. v^ += D^T f^ on the tile + 2-cell halo; e^ over the staged v^.  One cell at
            //    halo-4 (x, y): the tile's cells are own (outputs, imaging, CPML memory), the
            //    ring around them is only staged for the update below.
            auto vcell = [&](const int x, const int y) {
                const int i = i0 - 4 + x, j = j0 - 4 + y;
                const int o = y * SX + x;
                float h1 = 0.f, h2 = 0.f, h3 = 0.f, h4 = 0.f;
                if (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ)) {
                    const float inc_x = -st4(fxx[o + 1], fxx[o], fxx[o + 2], fxx[o - 1]) * rdx
                                        - st4(fxz[o], fxz[o - SX], fxz[o + SX], fxz[o - 2 * SX]) * rdz;
                    const float inc_z = -st4(fzz[o + SX], fzz[o], fzz[o + 2 * SX], fzz[o - SX]) * rdz
                                        - st4(g4[o], g4[o - 1], g4[o + 1], g4[o - 2]) * rdx;
                    const float vx = svx[o] + inc_x;
                    const float vz = svz[o] + inc_z;
                    const float qx = dt * sbx[o] * vx, qz = dt * sbz[o] * vz;
                    h1 = qx; h2 = qx; h3 = qz; h4 = qz;
                    const bool own = x >= 4 && x < TX + 4 && y >= 4 && y < TZ + 4 && (!edge || (i < NX && j < NZ));
                    if (edge) vel_pml(i, j, own, qx, qz, h1, h2, h3, h4);
                    if (own) {
                        const long long c = off + (long long)(j + EFWI_GZ) * pitch + (i + EFWI_GX);
                        a.out.vx[c] = vx;
                        a.out.vz[c] = vz;
                        if (!edge || (i >= PP - 1 && i <= PP + w && j >= PP - 1 && j <= NZ - PP)) {
                            const int u = (y - 4) * TX + (x - 4);
                            a.Gbx[c] = sg[3 * NC + u] + wvx[o] * inc_x;
                            a.Gbz[c] = sg[4 * NC + u] + wvz[o] * inc_z;
                        }
                    }
                }
                // each thread reads only its own staged v^ before writing e^ over it
                svx[o] = h1; svz[o] = h3;
                if (edge) { e2w[o] = h2; e4w[o] = h4; }
            };
            if constexpr (VEC == 1) {
                constexpr int VX = TX + 4, VZ = TZ + 4;
                for (int q = tid; q < VX * VZ; q += NT) {
                    const int yv = q / VX, xv = q - yv * VX;
                    vcell(xv + 2, yv + 2);
                }
            } else {
                // every thread: at most one cell of the ring (rows 2, 3, TZ+4, TZ+5 over the
                // velocity width, columns 2, 3, TX+4, TX+5 between them), then one cell pair of
                // the tile, whose x-stencils share their inputs (64-bit shared-memory accesses)
                constexpr int RW = TX + 4, NRING = 4 * RW + 4 * TZ, NPAIR = (TX / 2) * TZ;
                // 512 threads: pairs on threads 0 .. NPAIR-1, the ring on the next NRING threads
                const int rq0 = NT == kThreads ? tid : tid - NPAIR;
                for (int q = rq0; q >= 0 && q < NRING; q += NT) {
                    int x, y;
                    if (q < 4 * RW) {
                        const int r = q / RW;
                        x = 2 + (q - r * RW);
                        y = r < 2 ? 2 + r : TZ + 2 + r;
                    } else {
                        const int r = q - 4 * RW, cc = r & 3;
                        y = 4 + (r >> 2);
                        x = cc < 2 ? 2 + cc : TX + 2 + cc;
                    }
                    vcell(x, y);
                }
                for (int q = tid; q < (TX / 2) * TZ; q += NT) {
                    const int yy = q / (TX / 2);
                    vpair(4 + 2 * (q - yy * (TX / 2)), 4 + yy);
                }
            }
            __syncthreads();
            const float *e1r = svx, *e3r = svz, *e2r = e2w, *e4r = e4w;

            // 3. F += dt C (-D^T e^) on the tile, with the imaging in F; one cell (x, y) of the tile
            auto scell = [&](const int x, const int y) {
                const int q = y * TX + x;
                const int i = i0 + x, j = j0 + y;
                if (edge && (i >= NX || j >= NZ)) return;
                const long long c = off + (long long)(j + EFWI_GZ) * pitch + (i + EFWI_GX);
                const int o = (y + 4) * SX + (x + 4);
                const float Fxx = edge ? txx[q] : fxx[o];
                const float Fzz = edge ? tzz[q] : fzz[o];
                const float Fxz = edge ? txz[q] : fxz[o];
                const FvView<SK> fvx = wvx + o, fvz = wvz + o;
                if (!edge || (i >= PP && i < PP + w && j >= PP && j < NZ - PP)) {
                    const float fx = st4(fvx[0], fvx[-1], fvx[1], fvx[-2]) * rdx;
                    const float fz = st4(fvz[0], fvz[-SX], fvz[SX], fvz[-2 * SX]) * rdz;
                    a.Glam[c] = sg[q] + (Fxx + Fzz) * (fx + fz);
                    a.Gmu[c] = sg[NC + q] + (Fxx - Fzz) * (fx - fz);
                }
                if (!edge || (i >= PP - 1 && i < PP + w && j >= PP - 1 && j < NZ - PP)) {
                    const float fxzv = st4(fvx[SX], fvx[0], fvx[2 * SX], fvx[-SX]) * rdz +
                                       st4(fvz[1], fvz[0], fvz[2], fvz[-1]) * rdx;
                    a.Gmuxz[c] = sg[2 * NC + q] + Fxz * fxzv;
                }
                const float dxx = -st4(e1r[o], e1r[o - 1], e1r[o + 1], e1r[o - 2]) * rdx;
                const float dzz = -st4(e4r[o], e4r[o - SX], e4r[o + SX], e4r[o - 2 * SX]) * rdz;
                const float dxz = -st4(e2r[o + SX], e2r[o], e2r[o + 2 * SX], e2r[o - SX]) * rdz
                                  - st4(e3r[o + 1], e3r[o], e3r[o + 2], e3r[o - 1]) * rdx;
                const float lam = slam[q], l2m = lam + 2.f * smu[q];
                a.out.sxx[c] = Fxx + dt * (l2m * dxx + lam * dzz);
                a.out.szz[c] = Fzz + dt * (lam * dxx + l2m * dzz);
                a.out.sxz[c] = Fxz + dt * (smxz[q] * dxz);
            };
            if constexpr (VEC == 1) {
                for (int q = tid; q < NC; q += NT) {
                    const int y = q / TX;
                    scell(q - y * TX, y);
                }
            } else {
                // cell pairs (x, x+1), x even: every cell's expression is scell's, term by term
                for (int q2 = tid; q2 < NC / 2; q2 += NT) {
                    const int y = q2 / (TX / 2), x = 2 * (q2 - y * (TX / 2));
                    const int i = i0 + x, j = j0 + y;
                    if (edge && (i >= NX || j >= NZ)) continue;
                    const int q = y * TX + x;
                    const long long c = off + (long long)(j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    const int o = (y + 4) * SX + (x + 4);
                    const float2 Fx2 = edge ? ld2(txx + q) : ld2(fxx + o);
                    const float2 Fz2 = edge ? ld2(tzz + q) : ld2(fzz + o);
                    const float2 Fs2 = edge ? ld2(txz + q) : ld2(fxz + o);
                    const float2 pm2 = wvx.pair(o - 2), p0 = wvx.pair(o), p2 = wvx.pair(o + 2),
                                 pS = wvx.pair(o + SX), p2S = wvx.pair(o + 2 * SX), pmS = wvx.pair(o - SX);
                    const float2 qm2 = wvz.pair(o - 2), q0 = wvz.pair(o), q2v = wvz.pair(o + 2),
                                 qS = wvz.pair(o + SX), qmS = wvz.pair(o - SX), qm2S = wvz.pair(o - 2 * SX);
                    const float fx[2] = {st4(p0.x, pm2.y, p0.y, pm2.x) * rdx, st4(p0.y, p0.x, p2.x, pm2.y) * rdx};
                    const float fz[2] = {st4(q0.x, qmS.x, qS.x, qm2S.x) * rdz, st4(q0.y, qmS.y, qS.y, qm2S.y) * rdz};
                    const float fxzv[2] = {
                        st4(pS.x, p0.x, p2S.x, pmS.x) * rdz + st4(q0.y, q0.x, q2v.x, qm2.y) * rdx,
                        st4(pS.y, p0.y, p2S.y, pmS.y) * rdz + st4(q2v.x, q0.y, q2v.y, q0.x) * rdx};
                    const float2 Em2 = ld2(e1r + o - 2), E0 = ld2(e1r + o), E2 = ld2(e1r + o + 2);
                    const float2 R0 = ld2(e4r + o), RmS = ld2(e4r + o - SX), RS = ld2(e4r + o + SX),
                                 Rm2S = ld2(e4r + o - 2 * SX);
                    const float2 W0 = ld2(e2r + o), WS = ld2(e2r + o + SX), W2S = ld2(e2r + o + 2 * SX),
                                 WmS = ld2(e2r + o - SX);
                    const float2 Tm2 = ld2(e3r + o - 2), T0 = ld2(e3r + o), T2 = ld2(e3r + o + 2);
                    const float dxx[2] = {-st4(E0.x, Em2.y, E0.y, Em2.x) * rdx, -st4(E0.y, E0.x, E2.x, Em2.y) * rdx};
                    const float dzz[2] = {-st4(R0.x, RmS.x, RS.x, Rm2S.x) * rdz, -st4(R0.y, RmS.y, RS.y, Rm2S.y) * rdz};
                    const float dxz[2] = {
                        -st4(WS.x, W0.x, W2S.x, WmS.x) * rdz - st4(T0.y, T0.x, T2.x, Tm2.y) * rdx,
                        -st4(WS.y, W0.y, W2S.y, WmS.y) * rdz - st4(T2.x, T0.y, T2.y, T0.x) * rdx};
                    const float2 la = ld2(slam + q), mu2 = ld2(smu + q), mx2 = ld2(smxz + q);
                    const float2 gl = ld2(sg + q), gm = ld2(sg + NC + q), gs = ld2(sg + 2 * NC + q);
                    const float Fxx[2] = {Fx2.x, Fx2.y}, Fzz[2] = {Fz2.x, Fz2.y}, Fxz[2] = {Fs2.x, Fs2.y};
                    const float lam[2] = {la.x, la.y}, muv[2] = {mu2.x, mu2.y}, mxz[2] = {mx2.x, mx2.y};
                    const float glv[2] = {gl.x, gl.y}, gmv[2] = {gm.x, gm.y}, gsv[2] = {gs.x, gs.y};
                    float nl[2], nm[2], ns[2], oxx[2], ozz[2], oxz[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        nl[h] = glv[h] + (Fxx[h] + Fzz[h]) * (fx[h] + fz[h]);
                        nm[h] = gmv[h] + (Fxx[h] - Fzz[h]) * (fx[h] - fz[h]);
                        ns[h] = gsv[h] + Fxz[h] * fxzv[h];
                        const float l2m = lam[h] + 2.f * muv[h];
                        oxx[h] = Fxx[h] + dt * (l2m * dxx[h] + lam[h] * dzz[h]);
                        ozz[h] = Fzz[h] + dt * (lam[h] * dxx[h] + l2m * dzz[h]);
                        oxz[h] = Fxz[h] + dt * (mxz[h] * dxz[h]);
                    }
                    if (!edge) {
                        st2g(a.Glam + c, make_float2(nl[0], nl[1]));
                        st2g(a.Gmu + c, make_float2(nm[0], nm[1]));
                        st2g(a.Gmuxz + c, make_float2(ns[0], ns[1]));
                        st2g(a.out.sxx + c, make_float2(oxx[0], oxx[1]));
                        st2g(a.out.szz + c, make_float2(ozz[0], ozz[1]));
                        st2g(a.out.sxz + c, make_float2(oxz[0], oxz[1]));
                    } else {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int ih = i + h;
                            if (ih >= NX) continue;
                            if (ih >= PP && ih < PP + w && j >= PP && j < NZ - PP) {
                                a.Glam[c + h] = nl[h];
                                a.Gmu[c + h] = nm[h];
                            }
                            if (ih >= PP - 1 && ih < PP + w && j >= PP - 1 && j < NZ - PP) a.Gmuxz[c + h] = ns[h];
                            a.out.sxx[c + h] = oxx[h];
                            a.out.szz[c + h] = ozz[h];
                            a.out.sxz[c + h] = oxz[h];
                        }
                    }
                }
            }
        };
        if (tl.w & 4) tile(std::true_type{});
        else tile(std::false_type{});
    }
}

template <int TX, int TZ, int VEC, int SK, int NT>
int attrs_and_blocks() {
    constexpr int sm = (int)AdjsLayout<TX, TZ, SK>::smem();
    cudaFuncSetAttribute(k_adj_scaled_tma<TX, TZ, VEC, SK, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_adj_scaled_tma<TX, TZ, VEC, SK, NT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_scaled_tma<TX, TZ, VEC, SK, NT>, NT, sm);
    return nb;
}

template <int VEC, int NT>
int blocks_sk(int sk) {
    return sk == EFWI_STORE_FP16   ? attrs_and_blocks<32, 16, VEC, EFWI_STORE_FP16, NT>()
           : sk == EFWI_STORE_BF16 ? attrs_and_blocks<32, 16, VEC, EFWI_STORE_BF16, NT>()
                                   : attrs_and_blocks<32, 16, VEC, 0, NT>();
}

template <int VEC, int SK, int NT>
void launch_v(const TmaAdjsArgs &a, int grid, cudaStream_t st) {
    k_adj_scaled_tma<32, 16, VEC, SK, NT><<<grid, NT, AdjsLayout<32, 16, SK>::smem(), st>>>(a);
}

template <int VEC, int NT>
void launch_sk(const TmaAdjsArgs &a, int grid, cudaStream_t st, int sk) {
    if (sk == EFWI_STORE_FP16) launch_v<VEC, EFWI_STORE_FP16, NT>(a, grid, st);
    else if (sk == EFWI_STORE_BF16) launch_v<VEC, EFWI_STORE_BF16, NT>(a, grid, st);
    else launch_v<VEC, 0, NT>(a, grid, st);
}

}  // namespace

bool adj_scaled_tma_shape_ok(int tx, int tz) { return tx == 32 && tz == 16; }

int adj_scaled_tma_prepare(efwi_plan *p, int tx, int tz, int vec) {
    const bool half = p->snap_store != EFWI_STORE_FP32;
    if (!adj_scaled_tma_shape_ok(tx, tz) || (half ? !p->segh : !p->seg) || vec < 1 || vec > 3) return EFWI_ERR_ARG;
    std::vector<AdjsMaps> h(p->d.ns);
    const long long F = p->fsz_total;
    for (int s = 0; s < p->d.ns; ++s) {
        const ShotDev &sh = p->shots[s];
        int rc = encode_map(&h[s].a2, p->adj[0], sh, F, 10, tx + 8, tz + 4, 2);
        if (!rc) rc = encode_map(&h[s].a1, p->adj[0], sh, F, 10, tx + 8, tz + 4, 1);
        if (!rc) rc = encode_map(&h[s].a3, p->adj[0], sh, F, 10, tx + 8, tz + 7, 1);
        if (!rc) rc = encode_map(&h[s].mb, p->mat, sh, F, 5, tx + 8, tz + 4, 2);
        if (!rc) rc = encode_map(&h[s].mc, p->mat, sh, F, 5, tx, tz, 3);
        if (!rc) rc = half ? encode_map(&h[s].sv, p->segh, sh, F, 2 * p->nslots, tx + 8, tz + 4, 2, 2)
                           : encode_map(&h[s].sv, p->seg, sh, F, 2 * p->nslots, tx + 8, tz + 4, 2);
        if (!rc) rc = encode_map(&h[s].gi, p->G, sh, F, 5, tx, tz, 5);
        if (rc) {
            p->err = "cuTensorMapEncodeTiled failed for the scaled-stress adjoint maps";
            return rc;
        }
    }
    if (!p->adjs_maps && cudaMalloc((void **)&p->adjs_maps, sizeof(AdjsMaps) * p->d.ns) != cudaSuccess)
        return EFWI_ERR_OOM;
    cudaMemcpy(p->adjs_maps, h.data(), sizeof(AdjsMaps) * p->d.ns, cudaMemcpyHostToDevice);
    const int nb = vec == 3   ? blocks_sk<2, 512>(p->snap_store)
                   : vec == 2 ? blocks_sk<2, kThreads>(p->snap_store) : blocks_sk<1, kThreads>(p->snap_store);
    p->tma_adj_grid = std::max(1, nb) * std::max(1, p->n_sms);
    p->tma_adj_stages = 2;
    p->adjs_vec = vec;
    return EFWI_OK;
}

void launch_adj_scaled_tma(efwi_plan *p, const SnapIn &si, cudaStream_t st) {
    const AdjArgsF f = adj_args_f(p, si);
    TmaAdjsArgs a;
    a.shots = p->shots_d;
    a.tiles = p->adj_tiles.tiles;
    a.maps = p->adjs_maps;
    a.ntiles = p->adj_tiles.n;
    a.af = 5 * p->acur;
    // field of the step's vx in the snapshot map: 2 x its slot
    a.vf = si.sr.h ? (int)(2 * ((static_cast<const char *>(si.sr.h) - static_cast<const char *>(p->segh)) /
                                 (2 * 2 * p->fsz_total)))
                   : (int)(2 * ((si.fx - p->seg) / (2 * p->fsz_total)));
    a.hmax = si.sr.hmax;
    a.ns = p->d.ns;
    a.out = f.out;
    a.pml = f.pml;
    a.n1 = f.n1; a.n3 = f.n3; a.n2 = f.n2; a.n4 = f.n4;
    a.n5 = f.n5; a.n8 = f.n8; a.n6 = f.n6; a.n7 = f.n7;
    a.Glam = f.Glam; a.Gmu = f.Gmu; a.Gmuxz = f.Gmuxz; a.Gbx = f.Gbx; a.Gbz = f.Gbz;
    a.dt = f.dt; a.rdx = f.rdx; a.rdz = f.rdz;
    a.err = p->dev_err;
    const int grid = std::min(p->grid_adj_override > 0 ? p->grid_adj_override : p->tma_adj_grid, a.ntiles);
    if (p->adjs_vec == 3) launch_sk<2, 512>(a, grid, st, p->snap_store);
    else if (p->adjs_vec == 2) launch_sk<2, kThreads>(a, grid, st, p->snap_store);
    else launch_sk<1, kThreads>(a, grid, st, p->snap_store);
}

}  // namespace efwi
