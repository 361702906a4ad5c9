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
    int nt, n;
    float dt, rdx, rdz;
    int *err;
};

template <int TX, int TZ, int NST>
struct FwdLayout {
    static constexpr int SX = TX + 8, SZ = TZ + 8;
    static constexpr int NS = SX * SZ;              // one halo field
    static constexpr int NC = TX * TZ;              // one tile field
    static constexpr int BUF = 7 * NS + 3 * NC;     // floats per buffer
    static constexpr unsigned BYTES = BUF * 4u;
    static constexpr size_t smem() { return NST * (size_t)BYTES + 128; }
};

template <int TX, int TZ, int NST>
__device__ __forceinline__ void issue_fwd(const TmaFwdArgs &a, int t, float *buf, uint64_t *bar) {
    using L = FwdLayout<TX, TZ, NST>;
    const int4 tl = a.tiles[t];
    const FwdMaps *m = a.maps + tl.x;
    mbar_expect_tx(bar, L::BYTES);
    // element x = cell i + GX, row y = cell j + GZ
    tma_load_3d(buf, &m->st, bar, tl.y, tl.z - 2, 5 * a.scur);
    tma_load_3d(buf + 5 * L::NS, &m->mb, bar, tl.y, tl.z - 2, 3);
    tma_load_3d(buf + 7 * L::NS, &m->mc, bar, tl.y + 4, tl.z + 2, 0);
}

template <int TX, int TZ, int NST>
__global__ void __launch_bounds__(kThreads) k_step_tma(TmaFwdArgs a) {
    using L = FwdLayout<TX, TZ, NST>;
    constexpr int SX = L::SX;
    extern __shared__ float4 smem_raw[];
    float *smb = align128(smem_raw);
    __shared__ __align__(8) uint64_t bar[NST];
    __shared__ int ok_s;
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
            if (tb < a.ntiles) issue_fwd<TX, TZ, NST>(a, tb, smb + b * L::BUF, &bar[b]);
        }
    uint32_t phase = 0;
    int t = blockIdx.x;
    for (int k = 0; t < a.ntiles; t += gridDim.x, ++k) {
        const int b = k % NST;
        float *buf = smb + b * L::BUF;
        // refill the stage consumed in the previous iteration with tile k + NST - 1
        const int tn = t + (NST - 1) * gridDim.x;
        const int bn = (k + NST - 1) % NST;
        if (tid == 0 && tn < a.ntiles) issue_fwd<TX, TZ, NST>(a, tn, smb + bn * L::BUF, &bar[bn]);
        if (tid == 0) ok_s = mbar_wait_bounded(&bar[b], (phase >> b) & 1u);
        __syncthreads();
        if (!ok_s) {
            if (tid == 0) atomicExch(a.err, 1);
            return;
        }
        mbar_wait_bounded(&bar[b], (phase >> b) & 1u);   // completed: acquire for every thread
        phase ^= 1u << b;

        const int4 tl = a.tiles[t];
        const ShotDev *sp = a.shots + tl.x;
        // shot scalars in registers (loaded once per tile, not after every store)
        const int NX = sp->NX, NZ = sp->NZ, P = sp->P, profx = sp->profx, pitch = sp->pitch;
        const long long off = sp->off, psx = sp->psx, psz = sp->psz;
        const bool edge = (tl.w & 2) != 0;
        const int i0 = tl.y, j0 = tl.z;
        float *svx = buf, *svz = buf + L::NS, *sxx = buf + 2 * L::NS, *szz = buf + 3 * L::NS, *sxz = buf + 4 * L::NS;
        const float *sbx = buf + 5 * L::NS, *sbz = buf + 6 * L::NS;
        const float *slam = buf + 7 * L::NS, *smu = slam + L::NC, *smxz = smu + L::NC;
        float *__restrict__ ovx = a.out.vx + off;
        float *__restrict__ ovz = a.out.vz + off;
        const float dt = a.dt, rdx = a.rdx, rdz = a.rdz;

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
                vx = svx[o] + dt * sbx[o] * (e1 + e2);
                vz = svz[o] + dt * sbz[o] * (e3 + e4);
                if (own && (!edge || (i < NX && j < NZ))) {
                    const int c = (j + EFWI_GZ) * pitch + (i + EFWI_GX);
                    ovx[c] = vx;
                    ovz[c] = vz;
                    if (a.segx) { a.segx[off + c] = vx; a.segz[off + c] = vz; }
                }
            }
            svx[o] = vx;
            svz[o] = vz;
        }
        __syncthreads();

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
        __syncthreads();   // this buffer is refilled by the next iteration's prefetch
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

template <int TX, int TZ, int NST>
void launch_tma(const TmaFwdArgs &a, int grid, cudaStream_t st) {
    k_step_tma<TX, TZ, NST><<<grid, kThreads, FwdLayout<TX, TZ, NST>::smem(), st>>>(a);
}

template <int TX, int TZ, int NST>
int occupancy() {
    cudaFuncSetAttribute(k_step_tma<TX, TZ, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)FwdLayout<TX, TZ, NST>::smem());
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_tma<TX, TZ, NST>, kThreads,
                                                  FwdLayout<TX, TZ, NST>::smem());
    return nb;
}

// compiled TMA variants: tile shape x pipeline stages
#define EFWI_TMA_VARIANTS(X) X(32, 8, 2) X(32, 8, 3) X(32, 8, 4) X(32, 16, 2) X(32, 16, 3) X(64, 8, 2) X(64, 8, 3) X(64, 16, 2)

}  // namespace

// 3D tensor map over a stack of nfield arrays (stride F floats) of one shot:
// dims {pitch, rows, nfield}, box {bx, by, bz}.
int encode_map(CUtensorMap *m, float *base, const ShotDev &s, long long F, int nfield, int bx, int by, int bz) {
    auto enc = encode_fn();
    if (!enc) return EFWI_ERR_CUDA;
    cuuint64_t dims[3] = {(cuuint64_t)s.pitch, (cuuint64_t)(s.NZ + 2 * EFWI_GZ), (cuuint64_t)nfield};
    cuuint64_t strides[2] = {(cuuint64_t)s.pitch * 4, (cuuint64_t)F * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base + s.off, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? EFWI_OK : EFWI_ERR_CUDA;
}

bool tma_shape_ok(int tx, int tz, int nst) {
#define EFWI_OK_X(a, b, c) if (tx == a && tz == b && nst == c) return true;
    EFWI_TMA_VARIANTS(EFWI_OK_X)
#undef EFWI_OK_X
    return false;
}

// Encode the forward maps of every shot for tile shape (tx, tz) into p->fwd_maps.
int tma_prepare_fwd(efwi_plan *p, int tx, int tz, int nst) {
    std::vector<FwdMaps> h(p->d.ns);
    const long long F = p->fsz_total;
    for (int s = 0; s < p->d.ns; ++s) {
        const ShotDev &sh = p->shots[s];
        int rc = encode_map(&h[s].st, p->state[0], sh, F, 10, tx + 8, tz + 8, 5);
        if (!rc) rc = encode_map(&h[s].mb, p->mat, sh, F, 5, tx + 8, tz + 8, 2);
        if (!rc) rc = encode_map(&h[s].mc, p->mat, sh, F, 5, tx, tz, 3);
        if (rc) {
            p->err = "cuTensorMapEncodeTiled failed for the forward maps";
            return rc;
        }
    }
    if (!p->fwd_maps && cudaMalloc((void **)&p->fwd_maps, sizeof(FwdMaps) * p->d.ns) != cudaSuccess)
        return EFWI_ERR_OOM;
    cudaMemcpy(p->fwd_maps, h.data(), sizeof(FwdMaps) * p->d.ns, cudaMemcpyHostToDevice);
    int nb = 0;
#define EFWI_OCC_X(a, b, c) if (tx == a && tz == b && nst == c) nb = occupancy<a, b, c>();
    EFWI_TMA_VARIANTS(EFWI_OCC_X)
#undef EFWI_OCC_X
    p->tma_stages = nst;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->tma_grid = std::max(1, nb) * sms;
    return EFWI_OK;
}

void launch_step_tma(efwi_plan *p, int n, float *segx, float *segz, cudaStream_t st) {
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
    a.nt = p->d.nt;
    a.n = n;
    a.dt = (float)p->d.dt;
    a.rdx = (float)(1.0 / p->d.dx);
    a.rdz = (float)(1.0 / p->d.dz);
    a.err = p->dev_err;
    const int grid = std::min(p->tma_grid, a.ntiles);
    const int tx = p->tiles.tx, tz = p->tiles.tz, nst = p->tma_stages;
#define EFWI_LAUNCH_X(a_, b_, c_) if (tx == a_ && tz == b_ && nst == c_) launch_tma<a_, b_, c_>(a, grid, st);
    EFWI_TMA_VARIANTS(EFWI_LAUNCH_X)
#undef EFWI_LAUNCH_X
}

}  // namespace efwi
