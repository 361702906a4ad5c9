// Shot groups of an extended problem held on the device.
//
// The model extension gives every source its own component m_s, and each
// component is independent through the forward modelling, the adjoint and the
// imaging (eqs. 1-6 applied per m_s); only the consistency term (eqs. 8, 11, 12)
// couples them, through per-pixel sums over all components.  A problem with
// more sources than one plan holds therefore runs as groups of the plan's
// shape.  efwi_plan_rebind binds a plan to the next group from host memory; a
// group set keeps every group's acquisition-dependent arrays (source and receiver
// weights, adjoint gather, wavelet increments, tile flags) in device memory, so
// that binding group k is a handful of device-to-device copies, which a stream
// capture can record.  The extended objective of all groups is then one
// capturable sequence: the objective that the device-resident l-BFGS iteration
// replays from its graph.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "plan.hpp"

using namespace efwi;

namespace {

__global__ void k_sum_phi(const double *parts, int n, double *out) {
    // one thread, fixed order: the groups' misfits, then the three consistency terms
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += parts[k];
        *out = s;
    }
}

int fail(const std::string &msg, int code = EFWI_ERR_ARG) {
    set_thread_error(msg);
    return code;
}

}  // namespace

struct efwi_groups {
    efwi_plan *p = nullptr;
    int ng = 0;
    // per group, back to back: the plan's device arrays that depend on the acquisition
    ShotDev *shots = nullptr;            // [ng][ns]
    float *dw = nullptr, *wv = nullptr;  // [ng][ns * nt]
    int *tr_off = nullptr;               // [ng][ntr * 16]
    float *tr_w = nullptr;
    int *g_shot = nullptr, *g_field = nullptr, *g_off = nullptr, *g_ptr = nullptr, *g_tr = nullptr;
    float *g_w = nullptr;
    int4 *tiles = nullptr, *adj_tiles = nullptr;
    size_t n_dw = 0, n_trw = 0, n_tgt = 0, n_ptr = 0, n_nnz = 0, n_tiles = 0, n_adj_tiles = 0;
    double *phi_parts = nullptr;         // [ng + 3]: group misfits, consistency terms
    size_t bytes = 0;
};

static void free_groups(efwi_groups *g) {
    if (!g) return;
    for (void *q : {(void *)g->shots, (void *)g->dw, (void *)g->wv, (void *)g->tr_off, (void *)g->tr_w,
                    (void *)g->g_shot, (void *)g->g_field, (void *)g->g_off, (void *)g->g_ptr, (void *)g->g_tr,
                    (void *)g->g_w, (void *)g->tiles, (void *)g->adj_tiles, (void *)g->phi_parts})
        if (q) cudaFree(q);
    delete g;
}

extern "C" int efwi_groups_create(efwi_groups **out, efwi_plan *p, const efwi_plan_desc *descs, int ngroups) {
    if (!out) return fail("out is NULL");
    *out = nullptr;
    if (!p || !descs || ngroups < 1) return fail("efwi_groups_create: plan, descriptions and ngroups >= 1 required");
    if (p->d.exec != EFWI_EXEC_BATCHED) return fail("efwi_groups_create: the plan must use EXEC_BATCHED");
    const int ns = p->d.ns, nt = p->d.nt, ntr = p->d.ntr;
    std::vector<AcqHost> acq(ngroups);
    for (int k = 0; k < ngroups; ++k) {
        std::string err;
        if (check_same_shape(p, &descs[k], err) != EFWI_OK || build_acq(descs[k], p->shots, acq[k], err) != EFWI_OK)
            return fail("efwi_groups_create: group " + std::to_string(k) + ": " + err);
        // every group shares the adjoint gather's launch shape with the plan (its graphs hold it)
        if ((int)acq[k].g_shot.size() != p->gather.n_tgt || acq[k].gather_ptr != p->gather_ptr ||
            (int)acq[k].g_tr.size() != p->gather_nnz)
            return fail("efwi_groups_create: the receivers of group " + std::to_string(k) +
                        " give another adjoint-source gather than the plan's (bind it with efwi_plan_rebind)");
    }
    efwi_groups *g = new efwi_groups();
    g->p = p;
    g->ng = ngroups;
    g->n_dw = (size_t)ns * nt;
    g->n_trw = (size_t)std::max(ntr, 1) * 16;
    g->n_tgt = p->gather.n_tgt;
    g->n_ptr = g->n_tgt + 1;
    g->n_nnz = p->gather_nnz;
    g->n_tiles = p->tiles.n;
    g->n_adj_tiles = p->adj_tiles.n;
    bool ok = true;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (!ok || bytes == 0) return;
        if (cudaMalloc(ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            *ptr = nullptr;
            return;
        }
        g->bytes += bytes;
    };
    const size_t G = ngroups;
    alloc((void **)&g->shots, G * ns * sizeof(ShotDev));
    alloc((void **)&g->dw, G * g->n_dw * 4);
    if (p->has_force) alloc((void **)&g->wv, G * g->n_dw * 4);
    alloc((void **)&g->tr_off, G * g->n_trw * 4);
    alloc((void **)&g->tr_w, G * g->n_trw * 4);
    alloc((void **)&g->g_shot, G * g->n_tgt * 4);
    alloc((void **)&g->g_field, G * g->n_tgt * 4);
    alloc((void **)&g->g_off, G * g->n_tgt * 4);
    alloc((void **)&g->g_ptr, G * g->n_ptr * 4);
    alloc((void **)&g->g_tr, G * g->n_nnz * 4);
    alloc((void **)&g->g_w, G * g->n_nnz * 4);
    alloc((void **)&g->tiles, G * g->n_tiles * sizeof(int4));
    alloc((void **)&g->adj_tiles, G * g->n_adj_tiles * sizeof(int4));
    alloc((void **)&g->phi_parts, (G + 3) * sizeof(double));
    if (!ok) {
        free_groups(g);
        return fail("efwi_groups_create: device allocation failed", EFWI_ERR_OOM);
    }
    auto up = [](void *dst, const void *src, size_t bytes) {
        if (bytes) cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    for (int k = 0; k < ngroups; ++k) {
        const AcqHost &h = acq[k];
        up(g->shots + (size_t)k * ns, h.shots.data(), ns * sizeof(ShotDev));
        up(g->dw + k * g->n_dw, h.h_dw.data(), g->n_dw * 4);
        if (g->wv) up(g->wv + k * g->n_dw, h.h_wv.data(), g->n_dw * 4);
        up(g->tr_off + k * g->n_trw, h.h_off.data(), g->n_trw * 4);
        up(g->tr_w + k * g->n_trw, h.h_w.data(), g->n_trw * 4);
        up(g->g_shot + k * g->n_tgt, h.g_shot.data(), g->n_tgt * 4);
        up(g->g_field + k * g->n_tgt, h.g_field.data(), g->n_tgt * 4);
        up(g->g_off + k * g->n_tgt, h.g_off.data(), g->n_tgt * 4);
        up(g->g_ptr + k * g->n_ptr, h.g_ptr.data(), g->n_ptr * 4);
        up(g->g_tr + k * g->n_nnz, h.g_tr.data(), g->n_nnz * 4);
        up(g->g_w + k * g->n_nnz, h.g_w.data(), g->n_nnz * 4);
        const std::vector<int4> t = tiles_of(h.shots, p->tiles), ta = tiles_of(h.shots, p->adj_tiles);
        if (t.size() != g->n_tiles || ta.size() != g->n_adj_tiles) {
            free_groups(g);
            return fail("efwi_groups_create: tile lists of group " + std::to_string(k) + " differ from the plan's");
        }
        up(g->tiles + k * g->n_tiles, t.data(), t.size() * sizeof(int4));
        up(g->adj_tiles + k * g->n_adj_tiles, ta.data(), ta.size() * sizeof(int4));
    }
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_groups(g);
        return fail(std::string("efwi_groups_create: upload failed: ") + cudaGetErrorString(e), EFWI_ERR_CUDA);
    }
    *out = g;
    return EFWI_OK;
}

extern "C" int efwi_groups_destroy(efwi_groups *g) {
    if (!g) return EFWI_OK;
    cudaDeviceSynchronize();
    free_groups(g);
    return EFWI_OK;
}

extern "C" int efwi_groups_bind(efwi_groups *g, int k, efwi_stream_t stream) {
    if (!g || k < 0 || k >= g->ng) return fail("efwi_groups_bind: group set NULL or k outside [0, ngroups)");
    efwi_plan *p = g->p;
    cudaStream_t st = (cudaStream_t)stream;
    const int ns = p->d.ns;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (bytes && dst) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
    };
    cp(p->shots_d, g->shots + (size_t)k * ns, ns * sizeof(ShotDev));
    cp(p->dw, g->dw + k * g->n_dw, g->n_dw * 4);
    if (g->wv) cp(p->wv, g->wv + k * g->n_dw, g->n_dw * 4);
    if (p->d.ntr > 0) {
        cp(p->tr_off, g->tr_off + k * g->n_trw, g->n_trw * 4);
        cp(p->tr_w, g->tr_w + k * g->n_trw, g->n_trw * 4);
    }
    if (g->n_tgt > 0) {
        cp(p->gather.tgt_shot, g->g_shot + k * g->n_tgt, g->n_tgt * 4);
        cp(p->gather.tgt_field, g->g_field + k * g->n_tgt, g->n_tgt * 4);
        cp(p->gather.tgt_off, g->g_off + k * g->n_tgt, g->n_tgt * 4);
        cp(p->gather.ptr, g->g_ptr + k * g->n_ptr, g->n_ptr * 4);
        cp(p->gather.tr, g->g_tr + k * g->n_nnz, g->n_nnz * 4);
        cp(p->gather.w, g->g_w + k * g->n_nnz, g->n_nnz * 4);
    }
    cp(p->tiles.tiles, g->tiles + k * g->n_tiles, g->n_tiles * sizeof(int4));
    cp(p->adj_tiles.tiles, g->adj_tiles + k * g->n_adj_tiles, g->n_adj_tiles * sizeof(int4));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(std::string("efwi_groups_bind: ") + cudaGetErrorString(e), EFWI_ERR_CUDA);
    return EFWI_OK;
}

extern "C" int efwi_groups_objective(efwi_groups *g, const float *x, const float *d_obs, const double eta[3],
                                     const float *b, const float *bp, const uint8_t *sink, double *phi, float *grad,
                                     efwi_stream_t stream) {
    if (!g || !x || !d_obs || !eta || !phi || !grad)
        return fail("efwi_groups_objective: NULL argument");
    efwi_plan *p = g->p;
    const int ns = p->d.ns, ng = g->ng, nall = ns * ng;
    const long long npix = (long long)p->d.nz * p->d.nx;
    const long long field = (long long)nall * npix;       // one parameter of every component
    const size_t dstride = (size_t)p->d.ntr * p->d.nt;    // observed data of one group
    for (int k = 0; k < ng; ++k) {
        int rc = efwi_groups_bind(g, k, stream);
        if (rc) return rc;
        const long long o = (long long)k * ns * npix;
        rc = efwi_adjoint_gradient(p, x + o, x + field + o, x + 2 * field + o, d_obs + k * dstride, g->phi_parts + k,
                                   grad + o, grad + field + o, grad + 2 * field + o, nullptr, nullptr, stream);
        if (rc) {
            set_thread_error(std::string("efwi_groups_objective: group gradient: ") + efwi_last_error(p));
            return rc;
        }
    }
    for (int q = 0; q < 3; ++q) {
        const int rc = efwi_regularization_grad_n(p, nall, x + q * field, b, bp, sink, eta[q], g->phi_parts + ng + q,
                                                  grad + q * field, stream);
        if (rc) {
            set_thread_error(std::string("efwi_groups_objective: consistency term: ") + efwi_last_error(p));
            return rc;
        }
    }
    k_sum_phi<<<1, 32, 0, (cudaStream_t)stream>>>(g->phi_parts, ng + 3, phi);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(std::string("efwi_groups_objective: ") + cudaGetErrorString(e), EFWI_ERR_CUDA);
    return EFWI_OK;
}

extern "C" int efwi_groups_objective_fn(void *ctx, const float *x, double *phi, float *g, efwi_stream_t stream) {
    const efwi_groups_objective_ctx *o = static_cast<const efwi_groups_objective_ctx *>(ctx);
    if (!o) return EFWI_ERR_ARG;
    return efwi_groups_objective(o->groups, x, o->d_obs, o->eta, o->b, o->bp, o->sink, phi, g, stream);
}
