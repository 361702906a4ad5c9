// Inline-PTX helpers for TMA (cp.async.bulk.tensor) and mbarriers on sm_103a,
// and the per-shot tensor-map bundles the TMA kernels read.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace efwi {

// Tensor maps of one shot for the forward step, over the state (both buffers, 10
// fields) and the materials: boxes of the tile + 4-cell halo in x and, in z, the
// rows each field's readers use -- s2: vx, vz (2 fields, tile + 2 rows each side),
// s1: sigma_xx (1 field, the same rows), s3: sigma_zz or sigma_xz (1 field, tile +
// 3 rows on one side and 4 on the other), mb: b_x, b_z (2 fields, tile + 2 rows);
// mc: lambda/mu/mu_xz on the tile.  With shared-memory output staging, o2 / o3
// store the new velocities / stresses of a tile (boxes of 2 and 3 fields, tile
// only) and sg the segment-buffer copy of the velocities.
struct __align__(64) FwdMaps {
    CUtensorMap s2, s1, s3, mb, mc, o2, o3, sg;
};

// Tensor maps of one shot for the adjoint step: adjoint state (both buffers,
// 10 fields) and the 5 materials on the halo box, the forward velocities of
// the segment buffer (2 fields per stored step) on the halo box; gi: the 5
// imaging sums on the tile (L2 prefetch of the per-thread-load adjoint).
struct __align__(64) AdjMaps {
    CUtensorMap ad, m5, sg, gi;
};

// Tensor maps of one shot for the TMA adjoint step in scaled-stress form: boxes of the
// tile + 4-cell halo in x and, in z, the rows each field's readers use (as FwdMaps):
// a2: v^x, v^z (tile + 2 rows each side), a1: F_xx (the same rows), a3: F_zz or F_xz
// (tile + 3 rows on one side, 4 on the other), mb: b_x, b_z, sv: the forward v_x, v_z
// of the step (FP32 segment buffer; tile + 2 rows), mc: lambda, mu, mu_xz and gi: the
// five imaging sums on the tile.
struct __align__(64) AdjsMaps {
    CUtensorMap a2, a1, a3, mb, mc, sv, gi;
};

struct ShotDev;
// Encode a 3D map (x, row, field) over nfield arrays of F elements (4-byte floats, or 2-byte
// FP16/BF16 snapshot elements copied as raw 16-bit words) of the shot's block with box
// bx x by x bz (k_tma.cu).
int encode_map(CUtensorMap *m, void *base, const ShotDev &s, long long F, int nfield, int bx, int by, int bz,
               int elem_bytes = 4);

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// The first 128-byte aligned float of a dynamic shared-memory array, as an offset from
// the array itself: the pointer stays derived from the __shared__ symbol, so the
// compiler keeps shared-memory loads and stores (a round trip through an integer would
// leave it generic addresses, which the hardware resolves at every access).
__device__ __forceinline__ float *align128(float4 *p) {
    const uint32_t a = smem_u32(p);
    return reinterpret_cast<float *>(p) + ((((a + 127u) & ~127u) - a) >> 2);
}

__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ void st2g(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity, giving up after `budget` clock cycles
// (default 2^31, about one second): returns false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long budget = 1LL << 31) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

// Failure path of a bounded wait that expired: the stages of the pipeline that still
// have a copy in flight (count of them, the first being stage `b0` of the CTA's k-th
// tile) are each waited for once more with a bounded wait, so that, as far as the
// hardware lets a stalled copy finish, no copy lands in the shared memory of a CTA
// that has exited.  Best effort: a copy that never completes is abandoned after the
// budget.  Called by the thread that issues the copies; the caller issues no copy
// after the first failed wait.
__device__ __forceinline__ void mbar_drain_bounded(uint64_t *bar, uint32_t phase, int k, int nst, int count,
                                                   long long budget = 1LL << 31) {
    for (int j = 0; j < count; ++j) {
        const int b = (k + j) % nst;
        mbar_wait_bounded(&bar[b], (phase >> b) & 1u, budget);
    }
}

// Bring a box of the tensor into L2 (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Tile store shared -> global through the tensor map (bulk-group completion).
// Box elements outside the tensor's extent are not written.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];"
        ::"l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// every committed bulk store has finished reading its shared-memory source
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// every committed bulk store has completed
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// order this thread's generic-proxy shared-memory writes before later async-proxy
// (bulk copy) reads of them
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace efwi
