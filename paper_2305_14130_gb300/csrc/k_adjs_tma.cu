// Adjoint step in scaled-stress form with TMA staging (k_adj_scaled_tma): the step of
// k_adjs.cu (adjoint stresses carried as F = dt C sigma^) on a persistent grid whose
// CTAs copy every input of a tile into shared memory with cp.async.bulk.tensor, one
// tile ahead (two stages completing on mbarriers):
//   * v^x, v^z, b_x, b_z and the forward v_x, v_z of the step on the tile + 4-cell halo
//     in x and the tile + 2 rows in z, F_xx on the same rows, F_zz and F_xz on the rows
//     the velocity sub-step reads (tile + 3 rows on one side, 4 on the other);
//   * lambda, mu, mu_xz and the five imaging sums on the tile.
// A tile then computes from shared memory only: on tiles whose halo touches a CPML
// strip, the stress-sub-step CPML terms are added to the staged F in place (the tile's
// F kept for its update); v^ += D^T F on the tile + 2-cell halo with e^ = dt b v^ (+
// CPML) written over the staged v^; F += dt C (-D^T e^) on the tile with the imaging.
// Every expression is k_adj_scaled's, so both give bitwise-identical results.
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
};

// One stage (halo-4 coordinates: column x = cell i - i0 + 4, row y = cell j - j0 + 4):
// R2 arrays hold rows 2 .. TZ+5, F_zz rows 1 .. TZ+7, F_xz rows 0 .. TZ+6 (R3 rows each,
// padded to 128 bytes); tile arrays TX x TZ.  Every array starts 128-byte aligned.
template <int TX, int TZ>
struct AdjsLayout {
    static constexpr int SX = TX + 8;
    static constexpr int R2 = TZ + 4, R3 = TZ + 7;
    static constexpr int A2 = SX * R2;
    static constexpr int A3 = SX * R3, A3P = (A3 + 31) & ~31;
    static constexpr int NC = TX * TZ;
    static constexpr int OVX = 0, OVZ = A2, OFXX = 2 * A2, OFZZ = 3 * A2, OFXZ = OFZZ + A3P, OBX = OFXZ + A3P,
                         OBZ = OBX + A2, OWX = OBZ + A2, OWZ = OWX + A2, OLAM = OWZ + A2, OG = OLAM + 3 * NC;
    static constexpr int BUF = (OG + 5 * NC + 31) & ~31;                      // floats per stage
    static constexpr unsigned LOADED = (7u * A2 + 2u * A3 + 8u * NC) * 4u;    // bytes the copies bring
    // per CTA, edge tiles only: F_xz with its x-strip CPML term (g4), e^2, e^4 (R2 rows)
    // and F of the tile before its update
    static constexpr int EXTRA = 3 * A2 + 3 * NC;
    static constexpr size_t smem() { return (2 * (size_t)BUF + EXTRA) * 4 + 128; }
    static_assert(A2 % 32 == 0 && NC % 32 == 0, "arrays must keep 128-byte alignment");
};

template <int TX, int TZ>
__device__ __forceinline__ void issue_adjs(const TmaAdjsArgs &a, int t, float *buf, uint64_t *bar) {
    using L = AdjsLayout<TX, TZ>;
    const int4 tl = a.tiles[t];
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

template <int TX, int TZ>
__global__ void __launch_bounds__(kThreads, 2) k_adj_scaled_tma(TmaAdjsArgs a) {
    using L = AdjsLayout<TX, TZ>;
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
    if (tid == 0 && (int)blockIdx.x < a.ntiles) issue_adjs<TX, TZ>(a, blockIdx.x, smb, &bar[0]);
    uint32_t phase = 0;
    int t = blockIdx.x;
    int4 tl_next = t < a.ntiles ? __ldg(a.tiles + t) : make_int4(0, 0, 0, 0);
    for (int k = 0; t < a.ntiles; t += gridDim.x, ++k) {
        const int b = k & 1;
        float *buf = smb + b * L::BUF;
        const int4 tl = tl_next;
        const ShotDev *sp = a.shots + tl.x;
        const int NX = __ldg(&sp->NX), NZ = __ldg(&sp->NZ), PP = __ldg(&sp->P), profx = __ldg(&sp->profx),
                  pitch = __ldg(&sp->pitch), w = __ldg(&sp->w);
        const long long off = __ldg(&sp->off), psx = __ldg(&sp->psx), psz = __ldg(&sp->psz);
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
        if (tid == 0 && t + (int)gridDim.x < a.ntiles)
            issue_adjs<TX, TZ>(a, t + gridDim.x, smb + (b ^ 1) * L::BUF, &bar[b ^ 1]);

        auto tile = [&](auto edge_c) {
            constexpr bool edge = decltype(edge_c)::value;   // 4-cell halo touches a strip or the grid edge
            const int i0 = tl.y, j0 = tl.z;
            const float dt = a.dt, rdx = a.rdx, rdz = a.rdz;
            // base pointers in halo-4 coordinates (element y * SX + x), offset by each array's first row
            float *svx = buf + L::OVX - 2 * SX, *svz = buf + L::OVZ - 2 * SX;
            float *fxx = buf + L::OFXX - 2 * SX, *fzz = buf + L::OFZZ - SX, *fxz = buf + L::OFXZ;
            const float *sbx = buf + L::OBX - 2 * SX, *sbz = buf + L::OBZ - 2 * SX;
            const float *wvx = buf + L::OWX - 2 * SX, *wvz = buf + L::OWZ - 2 * SX;
            const float *slam = buf + L::OLAM, *smu = slam + NC, *smxz = smu + NC;
            const float *sg = buf + L::OG;                    // [5][NC]: lambda, mu, mu_xz, b_x, b_z sums
            float *g4 = edge ? xg4 - 2 * SX : fxz;            // f^4 == f^3 away from the CPML
            float *e2w = edge ? xe2 - 2 * SX : svx;           // e^2 == e^1, e^4 == e^3 away from the CPML
            float *e4w = edge ? xe4 - 2 * SX : svz;

            // 1. edge tiles: the stress-sub-step CPML terms over the staged F, in place, and the
            //    tile's stress-sub-step adjoint CPML memory; F of the tile kept for its update
            if constexpr (edge) {
                for (int q = tid; q < SX * (TZ + 8); q += kThreads) {
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

            // 2. v^ += D^T f^ on the tile + 2-cell halo; e^ over the staged v^
            constexpr int VX = TX + 4, VZ = TZ + 4;
            for (int q = tid; q < VX * VZ; q += kThreads) {
                const int yv = q / VX, xv = q - yv * VX;
                const int i = i0 - 2 + xv, j = j0 - 2 + yv;
                const int o = (yv + 2) * SX + (xv + 2);
                float h1 = 0.f, h2 = 0.f, h3 = 0.f, h4 = 0.f;
                if (!edge || (i >= 0 && i < NX && j >= 0 && j < NZ)) {
                    const float inc_x = -(C1 * (fxx[o + 1] - fxx[o]) + C2 * (fxx[o + 2] - fxx[o - 1])) * rdx
                                        - (C1 * (fxz[o] - fxz[o - SX]) + C2 * (fxz[o + SX] - fxz[o - 2 * SX])) * rdz;
                    const float inc_z = -(C1 * (fzz[o + SX] - fzz[o]) + C2 * (fzz[o + 2 * SX] - fzz[o - SX])) * rdz
                                        - (C1 * (g4[o] - g4[o - 1]) + C2 * (g4[o + 1] - g4[o - 2])) * rdx;
                    const float vx = svx[o] + inc_x;
                    const float vz = svz[o] + inc_z;
                    const float qx = dt * sbx[o] * vx, qz = dt * sbz[o] * vz;
                    h1 = qx; h2 = qx; h3 = qz; h4 = qz;
                    const bool own = xv >= 2 && xv < TX + 2 && yv >= 2 && yv < TZ + 2 && (!edge || (i < NX && j < NZ));
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
                        const long long c = off + (long long)(j + EFWI_GZ) * pitch + (i + EFWI_GX);
                        a.out.vx[c] = vx;
                        a.out.vz[c] = vz;
                        if (!edge || (i >= PP - 1 && i <= PP + w && j >= PP - 1 && j <= NZ - PP)) {
                            const int u = (yv - 2) * TX + (xv - 2);
                            a.Gbx[c] = sg[3 * NC + u] + wvx[o] * inc_x;
                            a.Gbz[c] = sg[4 * NC + u] + wvz[o] * inc_z;
                        }
                    }
                }
                // each thread reads only its own staged v^ before writing e^ over it
                svx[o] = h1; svz[o] = h3;
                if (edge) { e2w[o] = h2; e4w[o] = h4; }
            }
            __syncthreads();
            const float *e1r = svx, *e3r = svz, *e2r = e2w, *e4r = e4w;

            // 3. F += dt C (-D^T e^) on the tile, with the imaging in F
            for (int q = tid; q < NC; q += kThreads) {
                const int y = q / TX, x = q - y * TX;
                const int i = i0 + x, j = j0 + y;
                if (edge && (i >= NX || j >= NZ)) continue;
                const long long c = off + (long long)(j + EFWI_GZ) * pitch + (i + EFWI_GX);
                const int o = (y + 4) * SX + (x + 4);
                const float Fxx = edge ? txx[q] : fxx[o];
                const float Fzz = edge ? tzz[q] : fzz[o];
                const float Fxz = edge ? txz[q] : fxz[o];
                const float *fvx = wvx + o, *fvz = wvz + o;
                if (!edge || (i >= PP && i < PP + w && j >= PP && j < NZ - PP)) {
                    const float fx = (C1 * (fvx[0] - fvx[-1]) + C2 * (fvx[1] - fvx[-2])) * rdx;
                    const float fz = (C1 * (fvz[0] - fvz[-SX]) + C2 * (fvz[SX] - fvz[-2 * SX])) * rdz;
                    a.Glam[c] = sg[q] + (Fxx + Fzz) * (fx + fz);
                    a.Gmu[c] = sg[NC + q] + (Fxx - Fzz) * (fx - fz);
                }
                if (!edge || (i >= PP - 1 && i < PP + w && j >= PP - 1 && j < NZ - PP)) {
                    const float fxzv = (C1 * (fvx[SX] - fvx[0]) + C2 * (fvx[2 * SX] - fvx[-SX])) * rdz +
                                       (C1 * (fvz[1] - fvz[0]) + C2 * (fvz[2] - fvz[-1])) * rdx;
                    a.Gmuxz[c] = sg[2 * NC + q] + Fxz * fxzv;
                }
                const float dxx = -(C1 * (e1r[o] - e1r[o - 1]) + C2 * (e1r[o + 1] - e1r[o - 2])) * rdx;
                const float dzz = -(C1 * (e4r[o] - e4r[o - SX]) + C2 * (e4r[o + SX] - e4r[o - 2 * SX])) * rdz;
                const float dxz = -(C1 * (e2r[o + SX] - e2r[o]) + C2 * (e2r[o + 2 * SX] - e2r[o - SX])) * rdz
                                  - (C1 * (e3r[o + 1] - e3r[o]) + C2 * (e3r[o + 2] - e3r[o - 1])) * rdx;
                const float lam = slam[q], l2m = lam + 2.f * smu[q];
                a.out.sxx[c] = Fxx + dt * (l2m * dxx + lam * dzz);
                a.out.szz[c] = Fzz + dt * (lam * dxx + l2m * dzz);
                a.out.sxz[c] = Fxz + dt * (smxz[q] * dxz);
            }
        };
        if (tl.w & 4) tile(std::true_type{});
        else tile(std::false_type{});
    }
}

template <int TX, int TZ>
int attrs_and_blocks() {
    constexpr int sm = (int)AdjsLayout<TX, TZ>::smem();
    cudaFuncSetAttribute(k_adj_scaled_tma<TX, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_adj_scaled_tma<TX, TZ>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_scaled_tma<TX, TZ>, kThreads, sm);
    return nb;
}

}  // namespace

bool adj_scaled_tma_shape_ok(int tx, int tz) { return tx == 32 && tz == 16; }

int adj_scaled_tma_prepare(efwi_plan *p, int tx, int tz) {
    if (!adj_scaled_tma_shape_ok(tx, tz) || !p->seg) return EFWI_ERR_ARG;
    std::vector<AdjsMaps> h(p->d.ns);
    const long long F = p->fsz_total;
    for (int s = 0; s < p->d.ns; ++s) {
        const ShotDev &sh = p->shots[s];
        int rc = encode_map(&h[s].a2, p->adj[0], sh, F, 10, tx + 8, tz + 4, 2);
        if (!rc) rc = encode_map(&h[s].a1, p->adj[0], sh, F, 10, tx + 8, tz + 4, 1);
        if (!rc) rc = encode_map(&h[s].a3, p->adj[0], sh, F, 10, tx + 8, tz + 7, 1);
        if (!rc) rc = encode_map(&h[s].mb, p->mat, sh, F, 5, tx + 8, tz + 4, 2);
        if (!rc) rc = encode_map(&h[s].mc, p->mat, sh, F, 5, tx, tz, 3);
        if (!rc) rc = encode_map(&h[s].sv, p->seg, sh, F, 2 * p->nslots, tx + 8, tz + 4, 2);
        if (!rc) rc = encode_map(&h[s].gi, p->G, sh, F, 5, tx, tz, 5);
        if (rc) {
            p->err = "cuTensorMapEncodeTiled failed for the scaled-stress adjoint maps";
            return rc;
        }
    }
    if (!p->adjs_maps && cudaMalloc((void **)&p->adjs_maps, sizeof(AdjsMaps) * p->d.ns) != cudaSuccess)
        return EFWI_ERR_OOM;
    cudaMemcpy(p->adjs_maps, h.data(), sizeof(AdjsMaps) * p->d.ns, cudaMemcpyHostToDevice);
    const int nb = attrs_and_blocks<32, 16>();
    p->tma_adj_grid = std::max(1, nb) * std::max(1, p->n_sms);
    p->tma_adj_stages = 2;
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
    a.vf = (int)(2 * ((si.fx - p->seg) / (2 * p->fsz_total)));
    a.out = f.out;
    a.pml = f.pml;
    a.n1 = f.n1; a.n3 = f.n3; a.n2 = f.n2; a.n4 = f.n4;
    a.n5 = f.n5; a.n8 = f.n8; a.n6 = f.n6; a.n7 = f.n7;
    a.Glam = f.Glam; a.Gmu = f.Gmu; a.Gmuxz = f.Gmuxz; a.Gbx = f.Gbx; a.Gbz = f.Gbz;
    a.dt = f.dt; a.rdx = f.rdx; a.rdz = f.rdz;
    a.err = p->dev_err;
    const int grid = std::min(p->grid_adj_override > 0 ? p->grid_adj_override : p->tma_adj_grid, a.ntiles);
    k_adj_scaled_tma<32, 16><<<grid, kThreads, AdjsLayout<32, 16>::smem(), st>>>(a);
}

}  // namespace efwi
