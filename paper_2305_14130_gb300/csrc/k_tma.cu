// Forward time step with TMA staging (sm_103a): a persistent kernel in which
// every CTA walks the flat (shot, tile) list, and for each tile
//   * one thread issues three cp.async.bulk.tensor copies into shared memory:
//     the 5 wavefields of the tile + 4-cell halo (one 3D box over the field
//     dimension), b_x, b_z on the same halo box, and lambda, mu, mu_xz on the
//     tile, all completing on one mbarrier;
//   * the copies of the CTA's next tile are issued before the current tile is
//     computed (two shared-memory buffers), so loads overlap arithmetic;
//   * the arithmetic is the fused step of k_fused.cu, term by term: v^{n+1/2}
//     on the tile + 2-cell halo, then sigma^{n+1} and the moment-tensor source
//     on the tile, stored to the other state buffer.
// Out-of-range box elements (negative rows, past the row pitch) are zero-filled
// by the copy engine, matching the zero ghosts of the layout.  Every mbarrier
// wait is bounded (about 1 s of clock cycles); on expiry the CTA records the
// error in the plan's device flag and returns.
#include <type_traits>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <string>
#include <vector>

#include "plan.hpp"
#include "tma.cuh"

namespace efwi {
namespace {

constexpr int kThreads = 256;

struct TmaFwdArgs {
    const ShotDev *shots;
    const int4 *tiles;
    const FwdMaps *maps;
    int ntiles;
    int scur;                   // state buffer read (z offset 5 * scur in the state map)
    Fields out;                 // state buffer written
    Pml pml;                    // V block = current (read), S block = in place
    float *n1, *n3, *n2, *n4;   // next V block
    float *segx, *segz;
    const float *dw;
    const float *wv;            // w_n / (dx dz) of force sources (null without)
    int nt, n;
    float dt, rdx, rdz;
    int *err;
    int ofield;                 // state-map field of the written buffer's vx (output staging)
    int segf;                   // segment-map field of this step's vx, or -1 (output staging)
    SnapW sw;                   // reduced-precision snapshot work (sw.h / sw.amax null: none)
    int pf;                     // 1: L2 prefetch of the tile one beyond the shared-memory pipeline
};

// Shared-memory stage of one tile.  Fields are staged on the tile + 4-cell halo in x
// (SX columns) and, in z, only on the rows their readers use (halo-4 row coordinates,
// rows 0 .. TZ+7): vx, vz, sigma_xx, b_x, b_z on rows 2 .. TZ+5 (R2 rows), sigma_zz on
// rows 1 .. TZ+7 and sigma_xz on rows 0 .. TZ+6 (R3 rows each); lambda, mu, mu_xz on the
// tile.  Every array starts 128-byte aligned; vx|vz and b_x|b_z are 2-field boxes.
template <int TX, int TZ, int NST, int VEC = 1>
struct FwdLayout {
    static constexpr int SX = TX + 8, SZ = TZ + 8;
    static constexpr int R2 = TZ + 4, R3 = TZ + 7;
    static constexpr int A2 = SX * R2;                              // floats of an R2 field
    static constexpr int A3 = SX * R3, A3P = (A3 + 31) & ~31;       // R3 field, padded to 128 B
    static constexpr int NC = TX * TZ;                              // one tile field
    static constexpr int OVX = 0, OVZ = A2, OSXX = 2 * A2, OSZZ = 3 * A2, OSXZ = OSZZ + A3P,
                         OBX = OSXZ + A3P, OBZ = OBX + A2, OLAM = OBZ + A2;
    static constexpr int BUF = (OLAM + 3 * NC + 31) & ~31;          // floats per stage
    static constexpr unsigned LOADED = (5u * A2 + 2u * A3 + 3u * NC) * 4u;   // bytes the copies bring
    static constexpr size_t smem() { return NST * (size_t)BUF * 4 + 128; }
    static_assert(A2 % 32 == 0, "R2 fields must keep 128-byte alignment");
    static_assert(2 * NC <= 2 * A2, "staged velocities must fit over b_x, b_z");
};

// tl: the tile's work item, already in a register (the issuing thread's refill then has no
// dependent global load between the tile's barriers)
template <int TX, int TZ, int NST, int VEC>
__device__ __forceinline__ void issue_fwd(const TmaFwdArgs &a, const int4 tl, float *buf, uint64_t *bar) {
    using L = FwdLayout<TX, TZ, NST, VEC>;
    const FwdMaps *m = a.maps + tl.x;
    mbar_expect_tx(bar, L::LOADED);
    // element x = cell i + GX (halo-4 column 0 = cell i0 - 4), row y = cell j + GZ: halo-4 row r
    // of the tile is map row j0 - 4 + r + GZ = tl.z - 2 + r
    const int f = 5 * a.scur;
    tma_load_3d(buf + L::OVX, &m->s2, bar, tl.y, tl.z, f);          // vx, vz: rows 2..
    tma_load_3d(buf + L::OSXX, &m->s1, bar, tl.y, tl.z, f + 2);     // sigma_xx: rows 2..
    tma_load_3d(buf + L::OSZZ, &m->s3, bar, tl.y, tl.z - 1, f + 3); // sigma_zz: rows 1..
    tma_load_3d(buf + L::OSXZ, &m->s3, bar, tl.y, tl.z - 2, f + 4); // sigma_xz: rows 0..
    tma_load_3d(buf + L::OBX, &m->mb, bar, tl.y, tl.z, 3);          // b_x, b_z: rows 2..
    tma_load_3d(buf + L::OLAM, &m->mc, bar, tl.y + 4, tl.z + 2, 0); // lambda, mu, mu_xz: tile
}

// The boxes issue_fwd copies, brought into L2 only (a tile beyond the pipeline).
__device__ __forceinline__ void prefetch_fwd(const TmaFwdArgs &a, int4 tl) {
    const FwdMaps *m = a.maps + tl.x;
    const int f = 5 * a.scur;
    tma_prefetch_3d(&m->s2, tl.y, tl.z, f);
    tma_prefetch_3d(&m->s1, tl.y, tl.z, f + 2);
    tma_prefetch_3d(&m->s3, tl.y, tl.z - 1, f + 3);
    tma_prefetch_3d(&m->s3, tl.y, tl.z - 2, f + 4);
    tma_prefetch_3d(&m->mb, tl.y, tl.z, 3);
    tma_prefetch_3d(&m->mc, tl.y + 4, tl.z + 2, 0);
}

// Shared-memory output staging (ST = 1, cell pairs only): the new stresses of the
// tile overwrite lambda, mu, mu_xz of the stage (each cell reads its own three
// materials before writing), the new velocities go densely over b_x/b_z (read
// only by the velocity sub-step), and after the tile one thread stores them with
// bulk tensor copies.  The stores of tile k are issued once every thread has
// passed the first barrier of tile k + 1; their shared-memory reads finish before
// that stage is refilled.
template <int TX, int TZ, int NST>
__device__ __forceinline__ void store_fwd(const TmaFwdArgs &a, int4 tl, const float *buf) {
    using L = FwdLayout<TX, TZ, NST, 2>;
    const FwdMaps *m = a.maps + tl.x;
    const int x = tl.y + EFWI_GX, y = tl.z + EFWI_GZ;
    tma_store_3d(&m->o2, buf + L::OBX, x, y, a.ofield);
    tma_store_3d(&m->o3, buf + L::OLAM, x, y, a.ofield + 2);
    if (a.segf >= 0) tma_store_3d(&m->sg, buf + L::OBX, x, y, a.segf);
    bulk_commit();
}

template <int TX, int TZ, int NST, int VEC, int ST = 0, int SK = 0>
__global__ void __launch_bounds__(kThreads, 3) k_step_tma(TmaFwdArgs a) {
    static_assert(ST == 0 || VEC >= 2, "output staging is implemented for cell pairs");
    // SK: EFWI_STORE_FP16 / BF16 compiles the reduced-precision snapshot work in (0: none)
    constexpr bool SNAP = SK != 0;
    using L = FwdLayout<TX, TZ, NST, VEC>;
    constexpr int SX = L::SX;
    extern __shared__ float4 smem_raw[];
    float *smb = align128(smem_raw);
    __shared__ __align__(8) uint64_t bar[NST];
    __shared__ int ok_s;
    __shared__ unsigned wmax_s[2 * (kThreads / 32)];   // per-warp snapshot maxima of a tile
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int b = 0; b < NST; ++b) mbar_init(&bar[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // prologue: the first NST-1 tiles of this CTA are in flight before any compute
    if (tid == 0)
        for (int b = 0; b < NST - 1; ++b) {
            const int tb = blockIdx.x + b * gridDim.x;
            if (tb < a.ntiles) issue_fwd<TX, TZ, NST, VEC>(a, __ldg(a.tiles + tb), smb + b * L::BUF, &bar[b]);
        }
    // the work item of the tile the next refill copies (thread 0), loaded one tile ahead
    int4 tl_fill = make_int4(0, 0, 0, 0);
    if (tid == 0 && blockIdx.x + (NST - 1) * gridDim.x < a.ntiles)
        tl_fill = __ldg(a.tiles + blockIdx.x + (NST - 1) * gridDim.x);
    uint32_t phase = 0;
    int t = blockIdx.x;
    // the work item of the next tile is loaded one tile ahead, and its shot scalars
    // before the tile's barrier, so neither load's latency follows the barrier
    int4 tl_next = t < a.ntiles ? __ldg(a.tiles + t) : make_int4(0, 0, 0, 0);
    int4 tl_prev = tl_next;
    int k = 0;
    for (; t < a.ntiles; t += gridDim.x, ++k) {
        const int b = k % NST;
        float *buf = smb + b * L::BUF;
        const int4 tl = tl_next;
        const ShotDev *sp = a.shots + tl.x;
        const int NX = __ldg(&sp->NX), NZ = __ldg(&sp->NZ), P = __ldg(&sp->P), profx = __ldg(&sp->profx),
                  pitch = __ldg(&sp->pitch);
        const long long off = __ldg(&sp->off), psx = __ldg(&sp->psx), psz = __ldg(&sp->psz);
        // scales of the previous step's snapshot, written below for this tile's own cells
        const float upx = SNAP && a.sw.h ? snap_scale_up(a.sw.hmax, 0, tl.x, a.sw.ns) : 1.f;
        const float upz = SNAP && a.sw.h ? snap_scale_up(a.sw.hmax, 1, tl.x, a.sw.ns) : 1.f;
        if (t + gridDim.x < a.ntiles) tl_next = __ldg(a.tiles + t + gridDim.x);
        const int tp = t + NST * gridDim.x;                      // L2 prefetch target (pf)
        const int4 tl_pf = a.pf && tid == 0 && tp < a.ntiles ? __ldg(a.tiles + tp) : make_int4(0, 0, 0, 0);
        if (tid == 0) ok_s = mbar_wait_bounded(&bar[b], (phase >> b) & 1u);
        __syncthreads();
        if (!ok_s) {
            if (tid == 0) {
                atomicOr(a.err, EFWI_FLAG_TIMEOUT);
                // copies in flight: this tile's and the next NST-2 tiles' (the refill of the
                // NST-1-th follows the wait); no copy is issued after this point
                int inflight = 0;
                for (int j = 0; j < NST - 1; ++j)
                    if (t + j * (int)gridDim.x < a.ntiles) ++inflight;
                mbar_drain_bounded(bar, phase, k, NST, inflight);
                if (ST) bulk_wait0();       // stores already issued finish before the CTA exits
            }
            return;
        }
        mbar_wait_bounded(&bar[b], (phase >> b) & 1u);   // completed: acquire for every thread
        phase ^= 1u << b;
        // refill the stage consumed in the previous iteration with tile k + NST - 1: every
        // thread has passed the barrier above, so none still reads that stage
        const int tn = t + (NST - 1) * gridDim.x;
        const int bn = (k + NST - 1) % NST;
        if (tid == 0) {
            if (ST && k > 0) {
                store_fwd<TX, TZ, NST>(a, tl_prev, smb + bn * L::BUF);   // stage bn held tile k - 1
                bulk_wait_read0();
            }
            if (tn < a.ntiles) issue_fwd<TX, TZ, NST, VEC>(a, tl_fill, smb + bn * L::BUF, &bar[bn]);
            if (a.pf && tp < a.ntiles) prefetch_fwd(a, tl_pf);
            if (tn + (int)gridDim.x < a.ntiles) tl_fill = __ldg(a.tiles + tn + gridDim.x);   // next refill
        }
        tl_prev = tl;

        // interior tiles (no CPML strip or grid edge within the halo) run a copy of
        // the body without any of the edge tests
        auto tile = [&](auto edge_c) {
            constexpr bool edge = decltype(edge_c)::value;
            const int i0 = tl.y, j0 = tl.z;
            // base pointers in halo-4 coordinates (element y * SX + x), offset by each array's first row
            float *svx = buf + L::OVX - 2 * SX, *svz = buf + L::OVZ - 2 * SX, *sxx = buf + L::OSXX - 2 * SX,
                  *szz = buf + L::OSZZ - SX, *sxz = buf + L::OSXZ;
            const float *sbx = buf + L::OBX - 2 * SX, *sbz = buf + L::OBZ - 2 * SX;
            const float *slam = buf + L::OLAM, *smu = slam + L::NC, *smxz = smu + L::NC;
            // output staging: dense [2][TZ][TX] velocities over b_x/b_z, [3][TZ][TX] stresses over
            // lambda, mu, mu_xz
            float *dv = buf + L::OBX, *ds = buf + L::OLAM;
            float *__restrict__ ovx = a.out.vx + off;
            float *__restrict__ ovz = a.out.vz + off;
            const float dt = a.dt, rdx = a.rdx, rdz = a.rdz;
            float mxv = 0.f, mzv = 0.f;                     // this thread's max |v^{n+1/2}| (snapshot scale)

            if constexpr (VEC >= 2) {
                // Cell pairs (x, x+1) in halo-4 coordinates, x even: adjacent x-stencils share
                // their inputs and every shared-memory access moves two cells.  Each cell's
                // arithmetic is the scalar expression, term by term.
                constexpr int NPX = (TX + 4) / 2;           // pairs per row of the velocity region
                auto vpair = [&](const int x, const int y) {
                    const int i = i0 - 4 + x, j = j0 - 4 + y;
                    const int o = y * SX + x;
                    const float2 xa = ld2(sxx + o - 2), xb = ld2(sxx + o), xc = ld2(sxx + o + 2);
                    const float2 za = ld2(sxz + o - 2), zb = ld2(sxz + o), zc = ld2(sxz + o + 2);
                    const float2 zm2 = ld2(sxz + o - 2 * SX), zm1 = ld2(sxz + o - SX), zp1 = ld2(sxz + o + SX);
                    const float2 cm1 = ld2(szz + o - SX), c0 = ld2(szz + o), cp1 = ld2(szz + o + SX),
                                 cp2 = ld2(szz + o + 2 * SX);
                    float e1[2], e2[2], e3[2], e4[2];
                    e1[0] = (C1 * (xb.y - xb.x) + C2 * (xc.x - xa.y)) * rdx;
                    e1[1] = (C1 * (xc.x - xb.y) + C2 * (xc.y - xb.x)) * rdx;
                    e2[0] = (C1 * (zb.x - zm1.x) + C2 * (zp1.x - zm2.x)) * rdz;
                    e2[1] = (C1 * (zb.y - zm1.y) + C2 * (zp1.y - zm2.y)) * rdz;
                    e3[0] = (C1 * (zb.x - za.y) + C2 * (zb.y - za.x)) * rdx;
                    e3[1] = (C1 * (zb.y - zb.x) + C2 * (zc.x - za.y)) * rdx;
                    e4[0] = (C1 * (cp1.x - c0.x) + C2 * (cp2.x - cm1.x)) * rdz;
                    e4[1] = (C1 * (cp1.y - c0.y) + C2 * (cp2.y - cm1.y)) * rdz;
                    const bool own = x >= 4 && x < TX + 4 && y >= 4 && y < TZ + 4;
                    bool in[2] = {true, true};
                    if (edge) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int ih = i + h;
                            in[h] = ih >= 0 && ih < NX && j >= 0 && j < NZ;
                            if (!in[h]) continue;
                            const int xs = ih < P ? ih : (ih >= NX - P ? ih - NX + 2 * P : -1);
                            const int zs = j < P ? j : (j >= NZ - P ? j - NZ + 2 * P : -1);
                            if (xs >= 0) {
                                const long long kk = psx + (long long)j * 2 * P + xs;
                                const int pq = profx + ih;
                                const float p1 = a.pml.bx_h[pq] * a.pml.x[0][kk] + a.pml.ax_h[pq] * e1[h];
                                const float p3 = a.pml.bx_i[pq] * a.pml.x[1][kk] + a.pml.ax_i[pq] * e3[h];
                                if (own) { a.n1[kk] = p1; a.n3[kk] = p3; }
                                e1[h] += p1; e3[h] += p3;
                            }
                            if (zs >= 0) {
                                const long long kk = psz + (long long)zs * NX + ih;
                                const float p2 = a.pml.bz_i[j] * a.pml.z[0][kk] + a.pml.az_i[j] * e2[h];
                                const float p4 = a.pml.bz_h[j] * a.pml.z[1][kk] + a.pml.az_h[j] * e4[h];
                                if (own) { a.n2[kk] = p2; a.n4[kk] = p4; }
                                e2[h] += p2; e4[h] += p4;
                            }
                        }
                    }
                    const float2 vxo = ld2(svx + o), vzo = ld2(svz + o), bxo = ld2(sbx + o), bzo = ld2(sbz + o);
                    float2 vx, vz;
                    vx.x = in[0] ? vxo.x + dt * bxo.x * (e1[0] + e2[0]) : 0.f;
                    vx.y = in[1] ? vxo.y + dt * bxo.y * (e1[1] + e2[1]) : 0.f;
                    vz.x = in[0] ? vzo.x + dt * bzo.x * (e3[0] + e4[0]) : 0.f;
                    vz.y = in[1] ? vzo.y + dt * bzo.y * (e3[1] + e4[1]) : 0.f;
                    if (tl.w & 8) {                  // vector force of this shot (k_force's expression)
                        const int lc = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                        const float wvn = a.wv[(long long)tl.x * a.nt + a.n];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (lc == sp->inj_vx[k]) vx.x = vx.x + dt * bxo.x * (sp->fx * wvn * sp->inj_vxw[k]);
                            if (lc + 1 == sp->inj_vx[k]) vx.y = vx.y + dt * bxo.y * (sp->fx * wvn * sp->inj_vxw[k]);
                            if (lc == sp->inj_vz[k]) vz.x = vz.x + dt * bzo.x * (sp->fz * wvn * sp->inj_vzw[k]);
                            if (lc + 1 == sp->inj_vz[k]) vz.y = vz.y + dt * bzo.y * (sp->fz * wvn * sp->inj_vzw[k]);
                        }
                    }
                    st2(svx + o, vx);
                    st2(svz + o, vz);
                    if (SNAP && own && (a.sw.h || a.sw.amax)) {
                        // snapshot of v^{n-1/2} (staged input of this step) and the scale of v^{n+1/2}
                        const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                        if (a.sw.h) {
                            if (!edge || (i + 1 < NX && j < NZ)) {
                                snap_put2<SK>(a.sw.h, c, vxo.x * upx, vxo.y * upx);
                                snap_put2<SK>(a.sw.h, a.sw.F + c, vzo.x * upz, vzo.y * upz);
                            } else if (i < NX && j < NZ) {
                                snap_put1<SK>(a.sw.h, c, vxo.x * upx);
                                snap_put1<SK>(a.sw.h, a.sw.F + c, vzo.x * upz);
                            }
                        }
                        mxv = fmaxf(mxv, fmaxf(fabsf(vx.x), fabsf(vx.y)));
                        mzv = fmaxf(mzv, fmaxf(fabsf(vz.x), fabsf(vz.y)));
                    }
                    if (!ST && own) {
                        const int c = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                        if (!edge || (i + 1 < NX && j < NZ)) {
                            st2g(ovx + c, vx);
                            st2g(ovz + c, vz);
                            if (a.segx) { st2g(a.segx + off + c, vx); st2g(a.segz + off + c, vz); }
                        } else if (i < NX && j < NZ) {
                            ovx[c] = vx.x; ovz[c] = vz.x;
                            if (a.segx) { a.segx[off + c] = vx.x; a.segz[off + c] = vz.x; }
                        }
                    }
                };
                if constexpr (VEC == 3) {
                    // Split velocity region: every thread takes one cell pair of the tile and
                    // at most one single cell of the 2-cell halo ring (rows 2, 3, TZ+4, TZ+5
                    // over the full width, columns 2, 3, TX+4, TX+5 in between), so no thread
                    // waits at the barrier below for a second round of pairs.  A ring cell is
                    // never owned: its velocity is only staged for the stress sub-step.
                    auto vcell = [&](const int x, const int y) {
                        const int i = i0 - 4 + x, j = j0 - 4 + y;
                        const int o = y * SX + x;
                        float vx = 0.f, vz = 0.f;
                        if (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ)) {
                            float e1 = (C1 * (sxx[o + 1] - sxx[o]) + C2 * (sxx[o + 2] - sxx[o - 1])) * rdx;
                            float e2 = (C1 * (sxz[o] - sxz[o - SX]) + C2 * (sxz[o + SX] - sxz[o - 2 * SX])) * rdz;
                            float e3 = (C1 * (sxz[o] - sxz[o - 1]) + C2 * (sxz[o + 1] - sxz[o - 2])) * rdx;
                            float e4 = (C1 * (szz[o + SX] - szz[o]) + C2 * (szz[o + 2 * SX] - szz[o - SX])) * rdz;
                            if (edge) {
                                const int xs = i < P ? i : (i >= NX - P ? i - NX + 2 * P : -1);
                                const int zs = j < P ? j : (j >= NZ - P ? j - NZ + 2 * P : -1);
                                if (xs >= 0) {
                                    const long long kk = psx + (long long)j * 2 * P + xs;
                                    const int pq = profx + i;
                                    e1 += a.pml.bx_h[pq] * a.pml.x[0][kk] + a.pml.ax_h[pq] * e1;
                                    e3 += a.pml.bx_i[pq] * a.pml.x[1][kk] + a.pml.ax_i[pq] * e3;
                                }
                                if (zs >= 0) {
                                    const long long kk = psz + (long long)zs * NX + i;
                                    e2 += a.pml.bz_i[j] * a.pml.z[0][kk] + a.pml.az_i[j] * e2;
                                    e4 += a.pml.bz_h[j] * a.pml.z[1][kk] + a.pml.az_h[j] * e4;
                                }
                            }
                            vx = svx[o] + dt * sbx[o] * (e1 + e2);
                            vz = svz[o] + dt * sbz[o] * (e3 + e4);
                            if (tl.w & 8) {          // vector force of this shot (k_force's expression)
                                const int lc = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                                const float wvn = a.wv[(long long)tl.x * a.nt + a.n];
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    if (lc == sp->inj_vx[k]) vx = vx + dt * sbx[o] * (sp->fx * wvn * sp->inj_vxw[k]);
                                    if (lc == sp->inj_vz[k]) vz = vz + dt * sbz[o] * (sp->fz * wvn * sp->inj_vzw[k]);
                                }
                            }
                        }
                        svx[o] = vx;
                        svz[o] = vz;
                    };
                    constexpr int RW = TX + 4, NRING = 4 * RW + 4 * TZ;
                    for (int q = tid; q < NRING; q += kThreads) {
                        int x, y;
                        if (q < 4 * RW) {
                            const int r = q / RW;                   // ring rows 2, 3, TZ+4, TZ+5
                            x = 2 + (q - r * RW);
                            y = r < 2 ? 2 + r : TZ + 2 + r;
                        } else {
                            const int r = q - 4 * RW, c = r & 3;   // columns 2, 3, TX+4, TX+5
                            y = 4 + (r >> 2);
                            x = c < 2 ? 2 + c : TX + 2 + c;
                        }
                        vcell(x, y);
                    }
                    for (int q = tid; q < (TX / 2) * TZ; q += kThreads) {
                        const int yy = q / (TX / 2);
                        vpair(4 + 2 * (q - yy * (TX / 2)), 4 + yy);
                    }
                } else {
                    for (int q = tid; q < NPX * (TZ + 4); q += kThreads) {
                        const int yy = q / NPX;
                        vpair(2 + 2 * (q - yy * NPX), 2 + yy);
                    }
                }
                if (SNAP && a.sw.amax) snap_max_warp(mxv, mzv, wmax_s);
                __syncthreads();
                if (SNAP && a.sw.amax && tid == 32) snap_max_commit(wmax_s, a.sw.amax, tl.x, a.sw.ns);

                float *__restrict__ oxx = a.out.sxx + off;
                float *__restrict__ ozz = a.out.szz + off;
                float *__restrict__ oxz = a.out.sxz + off;
                const bool inj = (tl.w & 1) != 0;
                const float dwn = inj ? a.dw[(long long)tl.x * a.nt + a.n] : 0.f;
                constexpr int NPT = TX / 2;
                for (int q = tid; q < NPT * TZ; q += kThreads) {
                    const int yy = q / NPT;
                    const int xx = 2 * (q - yy * NPT);
                    const int x = 4 + xx, y = 4 + yy;
                    const int i = i0 + xx, j = j0 + yy;
                    if (edge && (i >= NX || j >= NZ)) {
                        if (ST) {                   // cells past the grid: the ghosts stay zero
                            const int oc = yy * TX + xx;
                            const float2 z2 = make_float2(0.f, 0.f);
                            st2(dv + oc, z2); st2(dv + L::NC + oc, z2);
                            st2(ds + oc, z2); st2(ds + L::NC + oc, z2); st2(ds + 2 * L::NC + oc, z2);
                        }
                        continue;
                    }
                    const int o = y * SX + x;
                    const float2 va = ld2(svx + o - 2), vb = ld2(svx + o), vc = ld2(svx + o + 2);
                    const float2 wa = ld2(svz + o - 2), wb = ld2(svz + o), wc = ld2(svz + o + 2);
                    const float2 wm2 = ld2(svz + o - 2 * SX), wm1 = ld2(svz + o - SX), wp1 = ld2(svz + o + SX);
                    const float2 um1 = ld2(svx + o - SX), up1 = ld2(svx + o + SX), up2 = ld2(svx + o + 2 * SX);
                    float f1[2], f2[2], f3[2], f4[2];
                    f1[0] = (C1 * (vb.x - va.y) + C2 * (vb.y - va.x)) * rdx;
                    f1[1] = (C1 * (vb.y - vb.x) + C2 * (vc.x - va.y)) * rdx;
                    f2[0] = (C1 * (wb.x - wm1.x) + C2 * (wp1.x - wm2.x)) * rdz;
                    f2[1] = (C1 * (wb.y - wm1.y) + C2 * (wp1.y - wm2.y)) * rdz;
                    f3[0] = (C1 * (up1.x - vb.x) + C2 * (up2.x - um1.x)) * rdz;
                    f3[1] = (C1 * (up1.y - vb.y) + C2 * (up2.y - um1.y)) * rdz;
                    f4[0] = (C1 * (wb.y - wb.x) + C2 * (wc.x - wa.y)) * rdx;
                    f4[1] = (C1 * (wc.x - wb.y) + C2 * (wc.y - wb.x)) * rdx;
                    if (edge) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int ih = i + h;
                            if (ih >= NX) continue;
                            const int xs = ih < P ? ih : (ih >= NX - P ? ih - NX + 2 * P : -1);
                            const int zs = j < P ? j : (j >= NZ - P ? j - NZ + 2 * P : -1);
                            if (xs >= 0) {
                                const long long kk = psx + (long long)j * 2 * P + xs;
                                const int pq = profx + ih;
                                const float p5 = a.pml.bx_i[pq] * a.pml.x[2][kk] + a.pml.ax_i[pq] * f1[h];
                                const float p8 = a.pml.bx_h[pq] * a.pml.x[3][kk] + a.pml.ax_h[pq] * f4[h];
                                a.pml.x[2][kk] = p5; a.pml.x[3][kk] = p8;
                                f1[h] += p5; f4[h] += p8;
                            }
                            if (zs >= 0) {
                                const long long kk = psz + (long long)zs * NX + ih;
                                const float p6 = a.pml.bz_i[j] * a.pml.z[2][kk] + a.pml.az_i[j] * f2[h];
                                const float p7 = a.pml.bz_h[j] * a.pml.z[3][kk] + a.pml.az_h[j] * f3[h];
                                a.pml.z[2][kk] = p6; a.pml.z[3][kk] = p7;
                                f2[h] += p6; f3[h] += p7;
                            }
                        }
                    }
                    const int oc = yy * TX + xx;
                    const float2 lam = ld2(slam + oc), mu = ld2(smu + oc), mxz = ld2(smxz + oc);
                    const float2 oxxv = ld2(sxx + o), ozzv = ld2(szz + o), oxzv = ld2(sxz + o);
                    float nxx[2], nzz[2], nxz[2];
                    const float lm[2] = {lam.x, lam.y}, m2[2] = {2.f * mu.x, 2.f * mu.y}, mx[2] = {mxz.x, mxz.y};
                    const float sx0[2] = {oxxv.x, oxxv.y}, sz0[2] = {ozzv.x, ozzv.y}, sc0[2] = {oxzv.x, oxzv.y};
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float tr = lm[h] * (f1[h] + f2[h]);
                        nxx[h] = sx0[h] + dt * (tr + m2[h] * f1[h]);
                        nzz[h] = sz0[h] + dt * (tr + m2[h] * f2[h]);
                        nxz[h] = sc0[h] + dt * mx[h] * (f3[h] + f4[h]);
                    }
                    const int c = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    if (inj) {
#pragma unroll
                        for (int h = 0; h < 2; ++h)
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                if (c + h == sp->inj_n[kk]) {
                                    nxx[h] -= sp->mxx * dwn * sp->inj_nw[kk];
                                    nzz[h] -= sp->mzz * dwn * sp->inj_nw[kk];
                                }
                                if (c + h == sp->inj_x[kk]) nxz[h] -= sp->mxz * dwn * sp->inj_xw[kk];
                            }
                    }
                    if (ST) {
                        // lambda, mu, mu_xz of these cells were read above by this thread only
                        const bool two = !edge || i + 1 < NX;
                        st2(ds + oc, make_float2(nxx[0], two ? nxx[1] : 0.f));
                        st2(ds + L::NC + oc, make_float2(nzz[0], two ? nzz[1] : 0.f));
                        st2(ds + 2 * L::NC + oc, make_float2(nxz[0], two ? nxz[1] : 0.f));
                        st2(dv + oc, vb);          // v^{n+1/2} of the pair (zero past the grid)
                        st2(dv + L::NC + oc, wb);
                    } else if (!edge || i + 1 < NX) {
                        st2g(oxx + c, make_float2(nxx[0], nxx[1]));
                        st2g(ozz + c, make_float2(nzz[0], nzz[1]));
                        st2g(oxz + c, make_float2(nxz[0], nxz[1]));
                    } else {
                        oxx[c] = nxx[0]; ozz[c] = nzz[0]; oxz[c] = nxz[0];
                    }
                }
                if (ST) fence_proxy_async_smem();   // the staged outputs are read by bulk copies
            } else {
            // v^{n+1/2} on the tile + 2-cell halo, in place over v^{n-1/2}
                constexpr int VX = TX + 4, VZ = TZ + 4;
                for (int q = tid; q < VX * VZ; q += kThreads) {
                    const int y = q / VX, x = q - y * VX;
                    const int i = i0 - 2 + x, j = j0 - 2 + y;
                    const int o = (y + 2) * SX + (x + 2);
                    float vx = 0.f, vz = 0.f;
                    if (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ)) {
                        float e1 = (C1 * (sxx[o + 1] - sxx[o]) + C2 * (sxx[o + 2] - sxx[o - 1])) * rdx;
                        float e2 = (C1 * (sxz[o] - sxz[o - SX]) + C2 * (sxz[o + SX] - sxz[o - 2 * SX])) * rdz;
                        float e3 = (C1 * (sxz[o] - sxz[o - 1]) + C2 * (sxz[o + 1] - sxz[o - 2])) * rdx;
                        float e4 = (C1 * (szz[o + SX] - szz[o]) + C2 * (szz[o + 2 * SX] - szz[o - SX])) * rdz;
                        const bool own = x >= 2 && x < TX + 2 && y >= 2 && y < TZ + 2;
                        if (edge) {
                            const int xs = i < P ? i : (i >= NX - P ? i - NX + 2 * P : -1);
                            const int zs = j < P ? j : (j >= NZ - P ? j - NZ + 2 * P : -1);
                            if (xs >= 0) {
                                const long long kk = psx + (long long)j * 2 * P + xs;
                                const int pq = profx + i;
                                const float p1 = a.pml.bx_h[pq] * a.pml.x[0][kk] + a.pml.ax_h[pq] * e1;
                                const float p3 = a.pml.bx_i[pq] * a.pml.x[1][kk] + a.pml.ax_i[pq] * e3;
                                if (own) { a.n1[kk] = p1; a.n3[kk] = p3; }
                                e1 += p1; e3 += p3;
                            }
                            if (zs >= 0) {
                                const long long kk = psz + (long long)zs * NX + i;
                                const float p2 = a.pml.bz_i[j] * a.pml.z[0][kk] + a.pml.az_i[j] * e2;
                                const float p4 = a.pml.bz_h[j] * a.pml.z[1][kk] + a.pml.az_h[j] * e4;
                                if (own) { a.n2[kk] = p2; a.n4[kk] = p4; }
                                e2 += p2; e4 += p4;
                            }
                        }
                        const float vxo = svx[o], vzo = svz[o];
                        vx = vxo + dt * sbx[o] * (e1 + e2);
                        vz = vzo + dt * sbz[o] * (e3 + e4);
                        if (tl.w & 8) {              // vector force of this shot (k_force's expression)
                            const int lc = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                            const float wvn = a.wv[(long long)tl.x * a.nt + a.n];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                if (lc == sp->inj_vx[k]) vx = vx + dt * sbx[o] * (sp->fx * wvn * sp->inj_vxw[k]);
                                if (lc == sp->inj_vz[k]) vz = vz + dt * sbz[o] * (sp->fz * wvn * sp->inj_vzw[k]);
                            }
                        }
                        if (own && (!edge || (i < NX && j < NZ))) {
                            const int c = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                            ovx[c] = vx;
                            ovz[c] = vz;
                            if (a.segx) { a.segx[off + c] = vx; a.segz[off + c] = vz; }
                            if (SNAP && a.sw.h) {    // snapshot of v^{n-1/2}
                                snap_put1<SK>(a.sw.h, off + c, vxo * upx);
                                snap_put1<SK>(a.sw.h, a.sw.F + off + c, vzo * upz);
                            }
                            mxv = fmaxf(mxv, fabsf(vx));
                            mzv = fmaxf(mzv, fabsf(vz));
                        }
                    }
                    svx[o] = vx;
                    svz[o] = vz;
                }
                if (SNAP && a.sw.amax) snap_max_warp(mxv, mzv, wmax_s);
                __syncthreads();
                if (SNAP && a.sw.amax && tid == 32) snap_max_commit(wmax_s, a.sw.amax, tl.x, a.sw.ns);
    
                // sigma^{n+1} on the tile, then the moment-tensor source
                float *__restrict__ oxx = a.out.sxx + off;
                float *__restrict__ ozz = a.out.szz + off;
                float *__restrict__ oxz = a.out.sxz + off;
                const bool inj = (tl.w & 1) != 0;
                const float dwn = inj ? a.dw[(long long)tl.x * a.nt + a.n] : 0.f;
                for (int q = tid; q < TX * TZ; q += kThreads) {
                    const int y = q / TX, x = q - y * TX;
                    const int i = i0 + x, j = j0 + y;
                    if (edge && (i >= NX || j >= NZ)) continue;
                    const int o = (y + 4) * SX + (x + 4);
                    float f1 = (C1 * (svx[o] - svx[o - 1]) + C2 * (svx[o + 1] - svx[o - 2])) * rdx;
                    float f2 = (C1 * (svz[o] - svz[o - SX]) + C2 * (svz[o + SX] - svz[o - 2 * SX])) * rdz;
                    float f3 = (C1 * (svx[o + SX] - svx[o]) + C2 * (svx[o + 2 * SX] - svx[o - SX])) * rdz;
                    float f4 = (C1 * (svz[o + 1] - svz[o]) + C2 * (svz[o + 2] - svz[o - 1])) * rdx;
                    if (edge) {
                        const int xs = i < P ? i : (i >= NX - P ? i - NX + 2 * P : -1);
                        const int zs = j < P ? j : (j >= NZ - P ? j - NZ + 2 * P : -1);
                        if (xs >= 0) {
                            const long long kk = psx + (long long)j * 2 * P + xs;
                            const int pq = profx + i;
                            const float p5 = a.pml.bx_i[pq] * a.pml.x[2][kk] + a.pml.ax_i[pq] * f1;
                            const float p8 = a.pml.bx_h[pq] * a.pml.x[3][kk] + a.pml.ax_h[pq] * f4;
                            a.pml.x[2][kk] = p5; a.pml.x[3][kk] = p8;
                            f1 += p5; f4 += p8;
                        }
                        if (zs >= 0) {
                            const long long kk = psz + (long long)zs * NX + i;
                            const float p6 = a.pml.bz_i[j] * a.pml.z[2][kk] + a.pml.az_i[j] * f2;
                            const float p7 = a.pml.bz_h[j] * a.pml.z[3][kk] + a.pml.az_h[j] * f3;
                            a.pml.z[2][kk] = p6; a.pml.z[3][kk] = p7;
                            f2 += p6; f3 += p7;
                        }
                    }
                    const int oc = y * TX + x;
                    const float lam = slam[oc], mu2 = 2.f * smu[oc];
                    const float tr = lam * (f1 + f2);
                    float nxx = sxx[o] + dt * (tr + mu2 * f1);
                    float nzz = szz[o] + dt * (tr + mu2 * f2);
                    float nxz = sxz[o] + dt * smxz[oc] * (f3 + f4);
                    const int c = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    if (inj) {
        #pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            if (c == sp->inj_n[kk]) {
                                nxx -= sp->mxx * dwn * sp->inj_nw[kk];
                                nzz -= sp->mzz * dwn * sp->inj_nw[kk];
                            }
                            if (c == sp->inj_x[kk]) nxz -= sp->mxz * dwn * sp->inj_xw[kk];
                        }
                    }
                    oxx[c] = nxx;
                    ozz[c] = nzz;
                    oxz[c] = nxz;
                }
            }
        };
        if (tl.w & 2) tile(std::true_type{});
        else tile(std::false_type{});
    }
    if (ST) {
        __syncthreads();                    // every thread has staged the last tile's outputs
        if (tid == 0) {
            if (k > 0) store_fwd<TX, TZ, NST>(a, tl_prev, smb + ((k - 1) % NST) * L::BUF);
            bulk_wait0();
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

template <int TX, int TZ, int NST, int VEC, int ST, int SK = 0>
void launch_tma(const TmaFwdArgs &a, int grid, cudaStream_t st) {
    k_step_tma<TX, TZ, NST, VEC, ST, SK><<<grid, kThreads, FwdLayout<TX, TZ, NST, VEC>::smem(), st>>>(a);
}

template <int TX, int TZ, int NST, int VEC, int ST, int SK = 0>
int occupancy() {
    cudaFuncSetAttribute(k_step_tma<TX, TZ, NST, VEC, ST, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)FwdLayout<TX, TZ, NST, VEC>::smem());
    cudaFuncSetAttribute(k_step_tma<TX, TZ, NST, VEC, ST, SK>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_tma<TX, TZ, NST, VEC, ST, SK>, kThreads,
                                                  FwdLayout<TX, TZ, NST, VEC>::smem());
    return nb;
}

// compiled TMA variants: tile shape x pipeline stages x cells per thread (1, 2, or 3 = cell
// pairs with the velocity halo ring split into single cells) x
// output staging (0: per-thread global stores, 1: shared memory + bulk tensor stores)
#define EFWI_TMA_VARIANTS(X)                                                                             \
    X(32, 8, 2, 1, 0) X(32, 8, 3, 1, 0) X(32, 16, 2, 1, 0) X(64, 8, 2, 1, 0) X(64, 16, 2, 1, 0)          \
    X(32, 8, 2, 2, 0) X(32, 8, 3, 2, 0) X(32, 16, 2, 2, 0) X(32, 16, 3, 2, 0) X(64, 8, 2, 2, 0)          \
    X(64, 16, 2, 2, 0) X(32, 16, 2, 2, 1) X(32, 16, 2, 3, 0) X(32, 16, 2, 3, 1)
// the variants also compiled with FP16 / BF16 snapshot work (plans with a reduced-precision snapshot store)
#define EFWI_TMA_SNAP_VARIANTS(X) \
    X(32, 16, 2, 1, 0) X(32, 16, 2, 2, 0) X(32, 16, 2, 2, 1) X(32, 16, 2, 3, 0) X(32, 16, 2, 3, 1) X(32, 8, 2, 2, 0)

}  // namespace

// 3D tensor map over a stack of nfield arrays (stride F floats) of one shot:
// dims {pitch, rows, nfield}, box {bx, by, bz}.
int encode_map(CUtensorMap *m, void *base, const ShotDev &s, long long F, int nfield, int bx, int by, int bz,
               int elem_bytes) {
    auto enc = encode_fn();
    if (!enc || (elem_bytes != 4 && elem_bytes != 2)) return EFWI_ERR_CUDA;
    const cuuint64_t eb = (cuuint64_t)elem_bytes;
    cuuint64_t dims[3] = {(cuuint64_t)s.pitch, (cuuint64_t)(s.NZ + 2 * EFWI_GZ), (cuuint64_t)nfield};
    cuuint64_t strides[2] = {(cuuint64_t)s.pitch * eb, (cuuint64_t)F * eb};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                     static_cast<char *>(base) + s.off * elem_bytes, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? EFWI_OK : EFWI_ERR_CUDA;
}

bool tma_shape_ok(int tx, int tz, int nst, int vec, int st, int snap) {
#define EFWI_OK_X(a, b, c, d, e) if (tx == a && tz == b && nst == c && vec == d && st == e) return true;
    if (snap != EFWI_STORE_FP32) {
        EFWI_TMA_SNAP_VARIANTS(EFWI_OK_X)
        return false;
    }
    EFWI_TMA_VARIANTS(EFWI_OK_X)
#undef EFWI_OK_X
    return false;
}

// Encode the forward maps of every shot for tile shape (tx, tz) into p->fwd_maps.
int tma_prepare_fwd(efwi_plan *p, int tx, int tz, int nst, int vec, int stg) {
    std::vector<FwdMaps> h(p->d.ns);
    const long long F = p->fsz_total;
    for (int s = 0; s < p->d.ns; ++s) {
        const ShotDev &sh = p->shots[s];
        int rc = encode_map(&h[s].s2, p->state[0], sh, F, 10, tx + 8, tz + 4, 2);
        if (!rc) rc = encode_map(&h[s].s1, p->state[0], sh, F, 10, tx + 8, tz + 4, 1);
        if (!rc) rc = encode_map(&h[s].s3, p->state[0], sh, F, 10, tx + 8, tz + 7, 1);
        if (!rc) rc = encode_map(&h[s].mb, p->mat, sh, F, 5, tx + 8, tz + 4, 2);
        if (!rc) rc = encode_map(&h[s].mc, p->mat, sh, F, 5, tx, tz, 3);
        if (!rc) rc = encode_map(&h[s].o2, p->state[0], sh, F, 10, tx, tz, 2);
        if (!rc) rc = encode_map(&h[s].o3, p->state[0], sh, F, 10, tx, tz, 3);
        if (!rc && p->seg) rc = encode_map(&h[s].sg, p->seg, sh, F, 2 * p->nslots, tx, tz, 2);
        if (rc) {
            p->err = "cuTensorMapEncodeTiled failed for the forward maps";
            return rc;
        }
    }
    if (!p->fwd_maps && cudaMalloc((void **)&p->fwd_maps, sizeof(FwdMaps) * p->d.ns) != cudaSuccess)
        return EFWI_ERR_OOM;
    cudaMemcpy(p->fwd_maps, h.data(), sizeof(FwdMaps) * p->d.ns, cudaMemcpyHostToDevice);
    int nb = 0;
    const int sk = p->snap_store;
#define EFWI_OCC_X(a, b, c, d, e) \
    if (tx == a && tz == b && nst == c && vec == d && stg == e) nb = occupancy<a, b, c, d, e>();
#define EFWI_OCC_SNAP_X(a, b, c, d, e)                                                                 \
    if (tx == a && tz == b && nst == c && vec == d && stg == e)                                        \
        nb = sk == EFWI_STORE_FP16 ? occupancy<a, b, c, d, e, EFWI_STORE_FP16>()                       \
                                   : occupancy<a, b, c, d, e, EFWI_STORE_BF16>();
    if (sk == EFWI_STORE_FP32) { EFWI_TMA_VARIANTS(EFWI_OCC_X) }
    else { EFWI_TMA_SNAP_VARIANTS(EFWI_OCC_SNAP_X) }
#undef EFWI_OCC_X
#undef EFWI_OCC_SNAP_X
    p->tma_stages = nst;
    p->tma_vec = vec;
    p->tma_store = stg;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->tma_grid = std::max(1, nb) * sms;
    return EFWI_OK;
}

void launch_step_tma(efwi_plan *p, int n, const SnapOut &so, cudaStream_t st) {
    float *segx = so.fx, *segz = so.fz;
    TmaFwdArgs a;
    a.shots = p->shots_d;
    a.tiles = p->tiles.tiles;
    a.maps = p->fwd_maps;
    a.ntiles = p->tiles.n;
    a.scur = p->scur;
    a.out = state_fields(p, 1 - p->scur);
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
    a.err = p->dev_err;
    a.ofield = 5 * (1 - p->scur);
    a.segf = segx ? (int)((segx - p->seg) / p->fsz_total) : -1;
    a.sw = so.sw;
    a.pf = p->tma_pf;
    const int grid = std::min(p->grid_fwd_override > 0 ? p->grid_fwd_override : p->tma_grid, a.ntiles);
    const int tx = p->tiles.tx, tz = p->tiles.tz, nst = p->tma_stages, vec = p->tma_vec, stg = p->tma_store;
    const int sk = p->snap_store;
#define EFWI_LAUNCH_X(a_, b_, c_, d_, e_) \
    if (tx == a_ && tz == b_ && nst == c_ && vec == d_ && stg == e_) launch_tma<a_, b_, c_, d_, e_>(a, grid, st);
#define EFWI_LAUNCH_SNAP_X(a_, b_, c_, d_, e_)                                                         \
    if (tx == a_ && tz == b_ && nst == c_ && vec == d_ && stg == e_) {                                 \
        if (sk == EFWI_STORE_FP16) launch_tma<a_, b_, c_, d_, e_, EFWI_STORE_FP16>(a, grid, st);       \
        else launch_tma<a_, b_, c_, d_, e_, EFWI_STORE_BF16>(a, grid, st);                             \
    }
    if (sk == EFWI_STORE_FP32) { EFWI_TMA_VARIANTS(EFWI_LAUNCH_X) }
    else { EFWI_TMA_SNAP_VARIANTS(EFWI_LAUNCH_SNAP_X) }
#undef EFWI_LAUNCH_X
#undef EFWI_LAUNCH_SNAP_X
}

}  // namespace efwi

// ===========================================================================
// Adjoint time step with TMA staging: same persistent, pipelined structure.
// Per tile, one thread copies (tile + 4-cell halo boxes) the 5 adjoint fields,
// the 5 materials and the 2 forward velocities of step n into shared memory.
// Then, in place over the staged fields:
//   0. every thread keeps the adjoint stresses of its own tile cells;
//   1. f^ = C sigma^ (+ PML) over the staged adjoint stresses;
//   2. v^ += D^T f^ on the tile + 2-cell halo, e^ = dt b v^ (+ PML) over the
//      staged adjoint velocities; b-imaging on the tile;
//   3. sigma^ += D^T e^ on the tile with the C-imaging.
// Inside CPML strips the four f^ (e^) components differ, and the extra
// components go to a separate shared array.
// ===========================================================================
namespace efwi {
namespace {

struct TmaAdjArgs {
    const ShotDev *shots;
    const int4 *tiles;
    const AdjMaps *maps;
    int ntiles;
    int acur;                   // adjoint buffer read (z offset 5 * acur)
    int slot;                   // segment-buffer step of the forward velocities
    Fields out;                 // adjoint buffer written
    Pml pml;                    // current adjoint PML memory
    float *n1, *n3, *n2, *n4;   // next V block
    float *n5, *n8, *n6, *n7;   // next S block
    float *Glam, *Gmu, *Gmuxz, *Gbx, *Gbz;
    float dt, rdx, rdz;
    int *err;
};

template <int TX, int TZ, int NST>
struct AdjLayout {
    static constexpr int SX = TX + 8, SZ = TZ + 8;
    static constexpr int NS = SX * SZ;
    static constexpr int BUF = 12 * NS;                 // 5 adjoint + 5 materials + 2 forward v
    static constexpr unsigned BYTES = BUF * 4u;
    static constexpr int EXTRA = 3 * NS;                 // f^4, e^2, e^4 inside CPML strips
    static constexpr size_t smem() { return (NST * (size_t)BUF + EXTRA) * 4 + 128; }
    static constexpr int PER = (TX * TZ + 255) / 256;    // own tile cells per thread
};

template <int TX, int TZ, int NST>
__device__ __forceinline__ void issue_adj(const TmaAdjArgs &a, int t, float *buf, uint64_t *bar) {
    using L = AdjLayout<TX, TZ, NST>;
    const int4 tl = a.tiles[t];
    const AdjMaps *m = a.maps + tl.x;
    mbar_expect_tx(bar, L::BYTES);
    tma_load_3d(buf, &m->ad, bar, tl.y, tl.z - 2, 5 * a.acur);
    tma_load_3d(buf + 5 * L::NS, &m->m5, bar, tl.y, tl.z - 2, 0);
    tma_load_3d(buf + 10 * L::NS, &m->sg, bar, tl.y, tl.z - 2, 2 * a.slot);
}

template <int TX, int TZ, int NST>
__global__ void __launch_bounds__(256) k_adj_tma(TmaAdjArgs a) {
    using L = AdjLayout<TX, TZ, NST>;
    constexpr int SX = L::SX, NS = L::NS, PER = L::PER;
    extern __shared__ float4 smem_raw[];
    float *smb = align128(smem_raw);
    float *xf4 = smb + NST * L::BUF, *xe2 = xf4 + NS, *xe4 = xe2 + NS;
    __shared__ __align__(8) uint64_t bar[NST];
    __shared__ int ok_s;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int b = 0; b < NST; ++b) mbar_init(&bar[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int b = 0; b < NST - 1; ++b) {
            const int tb = blockIdx.x + b * gridDim.x;
            if (tb < a.ntiles) issue_adj<TX, TZ, NST>(a, tb, smb + b * L::BUF, &bar[b]);
        }
    uint32_t phase = 0;
    int t = blockIdx.x;
    for (int k = 0; t < a.ntiles; t += gridDim.x, ++k) {
        const int b = k % NST;
        float *buf = smb + b * L::BUF;
        const int tn = t + (NST - 1) * gridDim.x;
        const int bn = (k + NST - 1) % NST;
        if (NST > 1 && tid == 0 && tn < a.ntiles) issue_adj<TX, TZ, NST>(a, tn, smb + bn * L::BUF, &bar[bn]);
        if (NST == 1 && tid == 0) issue_adj<TX, TZ, NST>(a, t, buf, &bar[0]);
        if (tid == 0) ok_s = mbar_wait_bounded(&bar[b], (phase >> b) & 1u);
        __syncthreads();
        if (!ok_s) {
            if (tid == 0) {
                atomicOr(a.err, EFWI_FLAG_TIMEOUT);
                // copies in flight: this tile's and, with a pipeline, the next NST-1 tiles'
                // (their refill precedes the wait); no copy is issued after this point
                int inflight = 0;
                for (int j = 0; j < (NST > 1 ? NST : 1); ++j)
                    if (t + j * (int)gridDim.x < a.ntiles) ++inflight;
                mbar_drain_bounded(bar, phase, k, NST, inflight);
            }
            return;
        }
        mbar_wait_bounded(&bar[b], (phase >> b) & 1u);
        phase ^= 1u << b;

        const int4 tl = a.tiles[t];
        const ShotDev *sp = a.shots + tl.x;
        const int NX = sp->NX, NZ = sp->NZ, PP = sp->P, profx = sp->profx, pitch = sp->pitch, w = sp->w;
        const long long off = sp->off, psx = sp->psx, psz = sp->psz;
        const bool edge = (tl.w & 4) != 0;
        const int i0 = tl.y, j0 = tl.z;
        const float dt = a.dt, rdx = a.rdx, rdz = a.rdz;
        float *hvx = buf, *hvz = buf + NS, *hxx = buf + 2 * NS, *hzz = buf + 3 * NS, *hxz = buf + 4 * NS;
        const float *mlam = buf + 5 * NS, *mmu = buf + 6 * NS, *mmxz = buf + 7 * NS, *mbx = buf + 8 * NS,
                    *mbz = buf + 9 * NS, *fvx = buf + 10 * NS, *fvz = buf + 11 * NS;
        float *f4s = edge ? xf4 : hxz;     // f^4 == f^3 away from the CPML
        float *e2s = edge ? xe2 : hvx;     // e^2 == e^1
        float *e4s = edge ? xe4 : hvz;     // e^4 == e^3

        // 0. own tile cells: adjoint stresses and imaging sums into registers
        float rxx[PER], rzz[PER], rxz[PER], gl[PER], gm[PER], gx[PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int q = tid + r * 256;
            const int y = q / TX, x = q - y * TX;
            const int o = (y + 4) * SX + (x + 4);
            rxx[r] = hxx[o]; rzz[r] = hzz[o]; rxz[r] = hxz[o];
            const int i = i0 + x, j = j0 + y;
            gl[r] = gm[r] = gx[r] = 0.f;
            if (q < TX * TZ && (!edge || (i < NX && j < NZ))) {
                const long long c = off + (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                gl[r] = a.Glam[c]; gm[r] = a.Gmu[c]; gx[r] = a.Gmuxz[c];
            }
        }
        __syncthreads();

        // 1. f^ over the staged adjoint stresses (tile + 4-cell halo)
        for (int q = tid; q < NS; q += 256) {
            const int y = q / SX, x = q - y * SX;
            const int i = i0 - 4 + x, j = j0 - 4 + y;
            const float sxx = hxx[q], szz = hzz[q], sxz = hxz[q];
            const float lam = mlam[q], l2m = lam + 2.f * mmu[q];
            const float Ex = dt * (l2m * sxx + lam * szz);
            const float Ez = dt * (lam * sxx + l2m * szz);
            const float Exz = dt * mmxz[q] * sxz;
            float g1 = Ex, g2 = Ez, g3 = Exz, g4 = Exz;
            if (edge) {
                if (i >= 0 && i < NX && j >= 0 && j < NZ) {
                    const bool own = x >= 4 && x < TX + 4 && y >= 4 && y < TZ + 4;
                    const int xs = i < PP ? i : (i >= NX - PP ? i - NX + 2 * PP : -1);
                    const int zs = j < PP ? j : (j >= NZ - PP ? j - NZ + 2 * PP : -1);
                    if (xs >= 0) {
                        const long long kk = psx + (long long)j * 2 * PP + xs;
                        const int pq = profx + i;
                        const float P5 = a.pml.x[2][kk], P8 = a.pml.x[3][kk];
                        g1 += a.pml.ax_i[pq] * (P5 + Ex);
                        g4 += a.pml.ax_h[pq] * (P8 + Exz);
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
                } else {
                    g1 = g2 = g3 = g4 = 0.f;
                }
                f4s[q] = g4;
            }
            hxx[q] = g1; hzz[q] = g2; hxz[q] = g3;
        }
        __syncthreads();

        // 2. v^ += D^T f^ on the tile + 2-cell halo; e^ over the staged adjoint velocities
        float *__restrict__ gbx = a.Gbx + off;
        float *__restrict__ gbz = a.Gbz + off;
        constexpr int VX = TX + 4, VZ = TZ + 4;
        for (int q = tid; q < VX * VZ; q += 256) {
            const int y = q / VX, x = q - y * VX;
            const int i = i0 - 2 + x, j = j0 - 2 + y;
            const int o = (y + 2) * SX + (x + 2);
            float h1 = 0.f, h2 = 0.f, h3 = 0.f, h4 = 0.f;
            if (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ)) {
                const float inc_x = -(C1 * (hxx[o + 1] - hxx[o]) + C2 * (hxx[o + 2] - hxx[o - 1])) * rdx
                                    - (C1 * (hxz[o] - hxz[o - SX]) + C2 * (hxz[o + SX] - hxz[o - 2 * SX])) * rdz;
                const float inc_z = -(C1 * (hzz[o + SX] - hzz[o]) + C2 * (hzz[o + 2 * SX] - hzz[o - SX])) * rdz
                                    - (C1 * (f4s[o] - f4s[o - 1]) + C2 * (f4s[o + 1] - f4s[o - 2])) * rdx;
                const float vx = hvx[o] + inc_x;
                const float vz = hvz[o] + inc_z;
                const float qx = dt * mbx[o] * vx, qz = dt * mbz[o] * vz;
                h1 = qx; h2 = qx; h3 = qz; h4 = qz;
                const bool own = x >= 2 && x < TX + 2 && y >= 2 && y < TZ + 2 && (!edge || (i < NX && j < NZ));
                if (edge) {
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
                }
                if (own) {
                    const int c = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    a.out.vx[off + c] = vx;
                    a.out.vz[off + c] = vz;
                    if (!edge || (i >= PP - 1 && i <= PP + w && j >= PP - 1 && j <= NZ - PP)) {
                        gbx[c] += fvx[o] * inc_x;
                        gbz[c] += fvz[o] * inc_z;
                    }
                }
            }
            if (edge) { e2s[o] = h2; e4s[o] = h4; }
            hvx[o] = h1;
            hvz[o] = h3;
        }
        __syncthreads();

        // 3. sigma^ += D^T e^ on the tile, with the C-imaging
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int q = tid + r * 256;
            if (q >= TX * TZ) break;
            const int y = q / TX, x = q - y * TX;
            const int i = i0 + x, j = j0 + y;
            if (edge && (i >= NX || j >= NZ)) continue;
            const int c = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
            const int o = (y + 4) * SX + (x + 4);
            const float sxx = rxx[r], szz = rzz[r], sxz = rxz[r];
            if (!edge || (i >= PP && i < PP + w && j >= PP && j < NZ - PP)) {
                const float fx = (C1 * (fvx[o] - fvx[o - 1]) + C2 * (fvx[o + 1] - fvx[o - 2])) * rdx;
                const float fz = (C1 * (fvz[o] - fvz[o - SX]) + C2 * (fvz[o + SX] - fvz[o - 2 * SX])) * rdz;
                a.Glam[off + c] = gl[r] + dt * (sxx + szz) * (fx + fz);
                a.Gmu[off + c] = gm[r] + 2.f * dt * (sxx * fx + szz * fz);
            }
            if (!edge || (i >= PP - 1 && i < PP + w && j >= PP - 1 && j < NZ - PP)) {
                const float fxz = (C1 * (fvx[o + SX] - fvx[o]) + C2 * (fvx[o + 2 * SX] - fvx[o - SX])) * rdz +
                                  (C1 * (fvz[o + 1] - fvz[o]) + C2 * (fvz[o + 2] - fvz[o - 1])) * rdx;
                a.Gmuxz[off + c] = gx[r] + dt * sxz * fxz;
            }
            a.out.sxx[off + c] = sxx - (C1 * (hvx[o] - hvx[o - 1]) + C2 * (hvx[o + 1] - hvx[o - 2])) * rdx;
            a.out.szz[off + c] = szz - (C1 * (e4s[o] - e4s[o - SX]) + C2 * (e4s[o + SX] - e4s[o - 2 * SX])) * rdz;
            a.out.sxz[off + c] = sxz - (C1 * (e2s[o + SX] - e2s[o]) + C2 * (e2s[o + 2 * SX] - e2s[o - SX])) * rdz
                                     - (C1 * (hvz[o + 1] - hvz[o]) + C2 * (hvz[o + 2] - hvz[o - 1])) * rdx;
        }
        __syncthreads();
    }
}

template <int TX, int TZ, int NST>
void launch_adj_tma_t(const TmaAdjArgs &a, int grid, cudaStream_t st) {
    k_adj_tma<TX, TZ, NST><<<grid, 256, AdjLayout<TX, TZ, NST>::smem(), st>>>(a);
}

template <int TX, int TZ, int NST>
int adj_occupancy() {
    cudaFuncSetAttribute(k_adj_tma<TX, TZ, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)AdjLayout<TX, TZ, NST>::smem());
    cudaFuncSetAttribute(k_adj_tma<TX, TZ, NST>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_tma<TX, TZ, NST>, 256, AdjLayout<TX, TZ, NST>::smem());
    return nb;
}

#define EFWI_TMA_ADJ_VARIANTS(X) X(32, 8, 1) X(32, 8, 2) X(32, 16, 1) X(32, 16, 2) X(64, 8, 1) X(64, 8, 2)

}  // namespace

bool tma_adj_shape_ok(int tx, int tz, int nst) {
#define EFWI_OK_X(a_, b_, c_) if (tx == a_ && tz == b_ && nst == c_) return true;
    EFWI_TMA_ADJ_VARIANTS(EFWI_OK_X)
#undef EFWI_OK_X
    return false;
}

// Encode the adjoint maps of every shot for tile shape (tx, tz) into p->adj_maps.
int tma_encode_adj_maps(efwi_plan *p, int tx, int tz) {
    std::vector<AdjMaps> h(p->d.ns);
    const long long F = p->fsz_total;
    for (int s = 0; s < p->d.ns; ++s) {
        const ShotDev &sh = p->shots[s];
        int rc = encode_map(&h[s].ad, p->adj[0], sh, F, 10, tx + 8, tz + 8, 5);
        if (!rc) rc = encode_map(&h[s].m5, p->mat, sh, F, 5, tx + 8, tz + 8, 5);
        if (!rc && p->seg) rc = encode_map(&h[s].sg, p->seg, sh, F, 2 * p->nslots, tx + 8, tz + 8, 2);
        if (!rc) rc = encode_map(&h[s].gi, p->G, sh, F, 5, tx, tz, 5);
        if (rc) {
            p->err = "cuTensorMapEncodeTiled failed for the adjoint maps";
            return rc;
        }
    }
    if (!p->adj_maps && cudaMalloc((void **)&p->adj_maps, sizeof(AdjMaps) * p->d.ns) != cudaSuccess)
        return EFWI_ERR_OOM;
    cudaMemcpy(p->adj_maps, h.data(), sizeof(AdjMaps) * p->d.ns, cudaMemcpyHostToDevice);
    return EFWI_OK;
}

int tma_prepare_adj(efwi_plan *p, int tx, int tz, int nst) {
    const int rc = tma_encode_adj_maps(p, tx, tz);
    if (rc) return rc;
    int nb = 0;
#define EFWI_OCC_X(a_, b_, c_) if (tx == a_ && tz == b_ && nst == c_) nb = adj_occupancy<a_, b_, c_>();
    EFWI_TMA_ADJ_VARIANTS(EFWI_OCC_X)
#undef EFWI_OCC_X
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->tma_adj_grid = std::max(1, nb) * sms;
    p->tma_adj_stages = nst;
    return EFWI_OK;
}

void launch_adj_tma(efwi_plan *p, const float *vfx, cudaStream_t st) {
    TmaAdjArgs a;
    a.shots = p->shots_d;
    a.tiles = p->adj_tiles.tiles;
    a.maps = p->adj_maps;
    a.ntiles = p->adj_tiles.n;
    a.acur = p->acur;
    a.slot = (int)((vfx - p->seg) / (2 * p->fsz_total));
    a.out = adj_fields(p, 1 - p->acur);
    a.pml = adj_pml(p, p->apsi_v, p->apsi_s);
    const long long X = p->psx_total, Z = p->psz_total;
    float *vn = psi_block(p->apsi, p, 1 - p->apsi_v), *sn = psi_block(p->apsi, p, 2 + (1 - p->apsi_s));
    a.n1 = vn; a.n3 = vn + X; a.n2 = vn + 2 * X; a.n4 = vn + 2 * X + Z;
    a.n5 = sn; a.n8 = sn + X; a.n6 = sn + 2 * X; a.n7 = sn + 2 * X + Z;
    a.Glam = G_field(p, 0); a.Gmu = G_field(p, 1); a.Gmuxz = G_field(p, 2);
    a.Gbx = G_field(p, 3); a.Gbz = G_field(p, 4);
    a.dt = (float)p->d.dt;
    a.rdx = (float)(1.0 / p->d.dx);
    a.rdz = (float)(1.0 / p->d.dz);
    a.err = p->dev_err;
    const int grid = std::min(p->grid_adj_override > 0 ? p->grid_adj_override : p->tma_adj_grid, a.ntiles);
    const int tx = p->adj_tiles.tx, tz = p->adj_tiles.tz, nst = p->tma_adj_stages;
#define EFWI_LAUNCH_X(a_, b_, c_) if (tx == a_ && tz == b_ && nst == c_) launch_adj_tma_t<a_, b_, c_>(a, grid, st);
    EFWI_TMA_ADJ_VARIANTS(EFWI_LAUNCH_X)
#undef EFWI_LAUNCH_X
}

}  // namespace efwi

// ===========================================================================
// Self-test of the timeout path: one thread waits, with the bounded wait of the
// TMA kernels, on an mbarrier that expects two arrivals and receives one, so
// the phase never completes; after `budget` clock cycles the wait gives up and
// the plan's device flag records it, exactly as a stalled copy would.  Nothing
// else is issued (no copy, no trap), so the kernel always ends.
// ===========================================================================
namespace {

__global__ void k_selftest_timeout(long long budget, int *err) {
    __shared__ __align__(8) uint64_t bar;
    efwi::mbar_init(&bar, 2);
    efwi::fence_mbar_init();
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(efwi::smem_u32(&bar)) : "memory");
    if (!efwi::mbar_wait_bounded(&bar, 0u, budget)) atomicOr(err, EFWI_FLAG_SELFTEST);
}

}  // namespace

extern "C" int efwi_selftest_timeout(efwi_plan *p, long long budget_cycles, efwi_stream_t stream) {
    if (!p || budget_cycles < 1 || budget_cycles > (1LL << 32)) {
        efwi::set_thread_error("efwi_selftest_timeout: plan NULL or budget outside [1, 2^32] cycles");
        if (p) p->err = "budget outside [1, 2^32] cycles";
        return EFWI_ERR_ARG;
    }
    k_selftest_timeout<<<1, 1, 0, (cudaStream_t)stream>>>(budget_cycles, p->dev_err);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        p->err = std::string("efwi_selftest_timeout: ") + cudaGetErrorString(e);
        return EFWI_ERR_CUDA;
    }
    return EFWI_OK;
}
