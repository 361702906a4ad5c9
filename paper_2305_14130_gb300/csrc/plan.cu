// Plan creation and destruction, argument validation, host-side precompute
// (CPML profiles, source and DAS interpolation weights, the deterministic
// adjoint-source gather), workspace allocation, and the plan-level C ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <nvtx3/nvToolsExt.h>
#include <cstring>
#include <map>
#include <tuple>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "plan.hpp"

using namespace efwi;

static thread_local std::string g_thread_err;

static int fail(efwi_plan *p, int code, const std::string &msg) {
    if (p) p->err = msg;
    g_thread_err = msg;
    return code;
}

namespace {

// Workspace allocation of a plan.  EFWI_TEST_FAIL_ALLOC=k makes the k-th allocation
// (1-based) fail without calling cudaMalloc, to test the out-of-memory path.
struct Alloc {
    efwi_plan *p;
    bool ok = true;
    std::string what;
    int count_ = 0;
    int fail_at = [] {
        const char *e = getenv("EFWI_TEST_FAIL_ALLOC");
        return e ? atoi(e) : 0;
    }();
    template <class T>
    void operator()(T **ptr, size_t count, const char *name) {
        if (!ok || count == 0) return;
        size_t bytes = count * sizeof(T);
        if (++count_ == fail_at) {
            ok = false;
            what = std::string("allocation of ") + name + " failed (EFWI_TEST_FAIL_ALLOC)";
            *ptr = nullptr;
            return;
        }
        cudaError_t e = cudaMalloc((void **)ptr, bytes);
        if (e != cudaSuccess) {
            ok = false;
            char buf[256];
            snprintf(buf, sizeof buf, "cudaMalloc of %zu bytes for %s failed: %s", bytes, name, cudaGetErrorString(e));
            what = buf;
            cudaGetLastError();
            *ptr = nullptr;
            return;
        }
        p->bytes += bytes;
        cudaMemset(*ptr, 0, bytes);
    }
};

// CPML (Komatitsch & Martin 2007) with kappa = 1 along one padded axis:
// psi <- b psi + a d(.), b = exp(-(d + alpha) dt), a = d (b - 1) / (d + alpha),
// d = d0 r^2, d0 = -3 vmax ln(R) / (2 L), alpha = pi f0 (1 - r).  The damping
// starts beyond the first padding node: r = distance past index P-1 (left) or
// N-P (right), over L = npml cells, clamped to 1.
void cpml_axis(int N, int P, double h, int npml, double R, double vmax, double f0, double dt, bool half,
               float *a, float *b) {
    const double L = npml * h;
    const double d0 = -3.0 * vmax * std::log(R) / (2.0 * L);
    for (int k = 0; k < N; ++k) {
        const double pos = k + (half ? 0.5 : 0.0);
        const double dist = std::max(std::max((P - 1) - pos, pos - (N - P)), 0.0);
        const double r = std::min(dist * h / L, 1.0);
        const double d = d0 * r * r;
        const double al = M_PI * f0 * (1.0 - r);
        const double bb = std::exp(-(d + al) * dt);
        a[k] = (float)(d > 0.0 ? d * (bb - 1.0) / (d + al) : 0.0);
        b[k] = (float)bb;
    }
}

struct Corner {
    int i, j;
    double w;
};

// Bilinear corners of the point (x, z) on the sub-grid offset by (ox, oz)
// cells, in the padded frame of shot geometry s.  False if the point lies
// outside the shot's physical window.
bool bilinear(const efwi_plan_desc &d, const ShotDev &s, double x, double z, double ox, double oz, Corner out[4]) {
    const double ux = x / d.dx - s.x0, uz = z / d.dz;
    if (!(ux >= 0.0 && ux <= s.w - 1 && uz >= 0.0 && uz <= d.nz - 1)) return false;
    const double fi = ux + s.P - ox, fj = uz + s.P - oz;
    const int i0 = (int)std::floor(fi), j0 = (int)std::floor(fj);
    const double ti = fi - i0, tj = fj - j0;
    out[0] = {i0, j0, (1 - ti) * (1 - tj)};
    out[1] = {i0 + 1, j0, ti * (1 - tj)};
    out[2] = {i0, j0 + 1, (1 - ti) * tj};
    out[3] = {i0 + 1, j0 + 1, ti * tj};
    return true;
}

int local_off(const ShotDev &s, int i, int j) { return (j + EFWI_GZ) * s.pitch + (i + EFWI_GX); }

}  // namespace

namespace efwi {

void set_thread_error(const std::string &msg) { g_thread_err = msg; }

Fields state_fields(efwi_plan *p, int which) {
    const long long F = p->fsz_total;
    float *s = p->state[which];
    return {s, s + F, s + 2 * F, s + 3 * F, s + 4 * F};
}
Fields adj_fields(efwi_plan *p, int which) {
    const long long F = p->fsz_total;
    float *s = p->adj[which];
    return {s, s + F, s + 2 * F, s + 3 * F, s + 4 * F};
}
Mat materials(efwi_plan *p) {
    const long long F = p->fsz_total;
    return {p->mat, p->mat + F, p->mat + 2 * F, p->mat + 3 * F, p->mat + 4 * F};
}
float *psi_block(float *base, efwi_plan *p, int blk) { return base + blk * p->H; }
static Pml make_pml(efwi_plan *p, float *base, int vblk, int sblk) {
    Pml m;
    const long long X = p->psx_total;
    float *v = psi_block(base, p, vblk), *s = psi_block(base, p, 2 + sblk);
    m.x[0] = v; m.x[1] = v + X; m.z[0] = v + 2 * X; m.z[1] = v + 2 * X + p->psz_total;
    m.x[2] = s; m.x[3] = s + X; m.z[2] = s + 2 * X; m.z[3] = s + 2 * X + p->psz_total;
    const int PX = p->prof_x_total;
    m.ax_i = p->prof; m.bx_i = p->prof + PX; m.ax_h = p->prof + 2 * PX; m.bx_h = p->prof + 3 * PX;
    const float *z = p->prof + 4 * PX;
    m.az_i = z; m.bz_i = z + p->nzp; m.az_h = z + 2 * p->nzp; m.bz_h = z + 3 * p->nzp;
    return m;
}
Pml fwd_pml(efwi_plan *p, int vblk, int sblk) { return make_pml(p, p->psi, vblk, sblk); }
Pml adj_pml(efwi_plan *p, int vblk, int sblk) { return make_pml(p, p->apsi, vblk, sblk); }
float *G_field(efwi_plan *p, int k) { return p->G + k * p->fsz_total; }

// Inside a stream capture an event record becomes a graph node (re-recorded by
// every replay) only with cudaEventRecordExternal.
static void record_event(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
}

void prof_begin(efwi_plan *p, cudaStream_t st, int *slot, int kind) {
    *slot = -1;
    if (p->prof_every <= 0) return;
    if ((p->prof_counter[kind]++ % p->prof_every) != 0) return;
    if (p->ev_used + 2 > (int)p->ev.size()) return;
    *slot = p->ev_used;
    p->ev_kind[*slot / 2] = kind;
    p->ev_used += 2;
    record_event(p->ev[*slot], st);
}
void prof_end(efwi_plan *p, cudaStream_t st, int slot) {
    if (slot >= 0) record_event(p->ev[slot + 1], st);
}

}  // namespace efwi

int efwi::build_acq(const efwi_plan_desc &dd, const std::vector<ShotDev> &geom, AcqHost &h, std::string &err) {
    const efwi_plan_desc *d = &dd;
    const int ns = d->ns, nt = d->nt;
    h.shots = geom;
    const double cellA = d->dx * d->dz;
    for (int s = 0; s < ns; ++s) {
        ShotDev &sh = h.shots[s];
        sh.mxx = (float)d->mt[3 * s]; sh.mzz = (float)d->mt[3 * s + 1]; sh.mxz = (float)d->mt[3 * s + 2];
        Corner cn[4], cx[4];
        if (!bilinear(*d, sh, d->src_xz[2 * s], d->src_xz[2 * s + 1], 0.0, 0.0, cn) ||
            !bilinear(*d, sh, d->src_xz[2 * s], d->src_xz[2 * s + 1], 0.5, 0.5, cx)) {
            err = "source " + std::to_string(s) + " outside its window";
            return EFWI_ERR_ARG;
        }
        for (int q = 0; q < 4; ++q) {
            sh.inj_n[q] = local_off(sh, cn[q].i, cn[q].j); sh.inj_nw[q] = (float)(cn[q].w / cellA);
            sh.inj_x[q] = local_off(sh, cx[q].i, cx[q].j); sh.inj_xw[q] = (float)(cx[q].w / cellA);
        }
        // vector force (eq. 2, second case) on the staggered v grids; it replaces the
        // moment tensor (whose injection then adds zeros)
        Corner fxc[4], fzc[4];
        bilinear(*d, sh, d->src_xz[2 * s], d->src_xz[2 * s + 1], 0.5, 0.0, fxc);
        bilinear(*d, sh, d->src_xz[2 * s], d->src_xz[2 * s + 1], 0.0, 0.5, fzc);
        for (int q = 0; q < 4; ++q) {
            sh.inj_vx[q] = local_off(sh, fxc[q].i, fxc[q].j); sh.inj_vxw[q] = (float)fxc[q].w;
            sh.inj_vz[q] = local_off(sh, fzc[q].i, fzc[q].j); sh.inj_vzw[q] = (float)fzc[q].w;
        }
        sh.fx = sh.fz = 0.f;
        if (d->force) {
            sh.fx = (float)d->force[2 * s];
            sh.fz = (float)d->force[2 * s + 1];
            sh.mxx = sh.mzz = sh.mxz = 0.f;
        }
    }
    h.has_force = d->force != nullptr;

    // DAS gauges: 4 components x 4 corners per trace
    const int ntr = d->ntr;
    h.h_off.assign((size_t)std::max(ntr, 1) * 16, 0);
    h.h_w.assign((size_t)std::max(ntr, 1) * 16, 0.f);
    h.trace_shot.assign(ntr, 0);
    // gather: (shot, field, off) -> list of (trace, weight)
    std::map<std::tuple<int, int, int>, std::vector<std::pair<int, float>>> gmap;
    for (int s = 0; s < ns; ++s) {
        const ShotDev &sh = h.shots[s];
        for (int c = d->tr_ptr[s]; c < d->tr_ptr[s + 1]; ++c) {
            h.trace_shot[c] = s;
            const double cx = d->ch_xz[2 * c], cz = d->ch_xz[2 * c + 1];
            const double tx = d->ch_t[2 * c], tz = d->ch_t[2 * c + 1];
            // DAS: gauge ends p+- = c +- (L/2) t with weights +-t/L; particle-velocity
            // receiver: the point c with weight t (the second "end" carries zero weight)
            const bool point = d->das_mode == EFWI_DAS_VELOCITY;
            const double hl = point ? 0.0 : 0.5 * d->gauge;
            const double scale = point ? 1.0 : 1.0 / d->gauge;
            const double ends[2][2] = {{cx + hl * tx, cz + hl * tz}, {cx - hl * tx, cz - hl * tz}};
            for (int k = 0; k < 4; ++k) {
                const int e = k >> 1, field = k & 1;
                const double sgn = e == 0 ? 1.0 : (point ? 0.0 : -1.0);
                const double tcomp = field == 0 ? tx : tz;
                Corner cr[4];
                if (!bilinear(*d, sh, ends[e][0], ends[e][1], field == 0 ? 0.5 : 0.0, field == 0 ? 0.0 : 0.5, cr)) {
                    err = "gauge end of trace " + std::to_string(c) + " outside the window of shot " +
                          std::to_string(s);
                    return EFWI_ERR_ARG;
                }
                for (int q = 0; q < 4; ++q) {
                    const int o = local_off(sh, cr[q].i, cr[q].j);
                    const float wq = (float)(cr[q].w * sgn * tcomp * scale);
                    h.h_off[(size_t)c * 16 + k * 4 + q] = o;
                    h.h_w[(size_t)c * 16 + k * 4 + q] = wq;
                    if (wq != 0.f) gmap[std::make_tuple(s, field, o)].push_back({c, wq});
                }
            }
        }
    }
    h.g_ptr.assign(1, 0);
    for (auto &kv : gmap) {
        h.g_shot.push_back(std::get<0>(kv.first));
        h.g_field.push_back(std::get<1>(kv.first));
        h.g_off.push_back(std::get<2>(kv.first));
        for (auto &e : kv.second) { h.g_tr.push_back(e.first); h.g_w.push_back(e.second); }
        h.g_ptr.push_back((int)h.g_tr.size());
    }
    h.gather_ptr.assign(ns + 1, 0);
    for (int s : h.g_shot) h.gather_ptr[s + 1]++;
    for (int s = 0; s < ns; ++s) h.gather_ptr[s + 1] += h.gather_ptr[s];

    // wavelet increments (moment tensors) and samples / (dx dz) (forces)
    h.h_dw.resize((size_t)ns * nt);
    for (int s = 0; s < ns; ++s)
        for (int n = 0; n < nt; ++n)
            h.h_dw[(size_t)s * nt + n] =
                (float)((double)d->wavelet[(size_t)s * (nt + 1) + n + 1] - (double)d->wavelet[(size_t)s * (nt + 1) + n]);
    h.h_wv.assign(h.has_force ? (size_t)ns * nt : 0, 0.f);
    for (size_t k = 0; k < h.h_wv.size(); ++k) {
        const size_t s = k / nt, n = k % nt;
        h.h_wv[k] = (float)((double)d->wavelet[s * (nt + 1) + n] / cellA);
    }
    return EFWI_OK;
}

// The host-side part of an acquisition becomes the plan's.
static void commit_acq(efwi_plan *p, const AcqHost &h) {
    p->shots = h.shots;
    p->trace_shot = h.trace_shot;
    p->has_force = h.has_force;
    p->gather.n_tgt = (int)h.g_shot.size();
    p->gather_ptr = h.gather_ptr;
    p->gather_nnz = (int)h.g_tr.size();
}

static void free_plan(efwi_plan *p) {
    if (!p) return;
    void *ptrs[] = {p->shots_d, p->state[0], p->mat, p->adj[0], p->fwd_maps, p->adj_maps, p->adjs_maps, p->dev_err, p->G, p->Gtot, p->Gcmp, p->psi, p->apsi,
                    p->prof, p->dw, p->wv, p->ref, p->tr_shot, p->tr_off, p->tr_w, p->tr_acc, p->tr_coef,
                    p->gather.tgt_shot, p->gather.tgt_field, p->gather.tgt_off, p->gather.ptr, p->gather.tr,
                    p->gather.w, p->tiles.tiles, p->adj_tiles.tiles, p->resid, p->dbuf, p->partial, p->seg, p->ck.fields, p->ck.psi,
                    p->ck.scale, p->segh, p->segmax, p->zoi_b, p->zoi_bp, p->zoi_sink};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (GraphCache *g : {&p->g_fwd, &p->g_fwd_ck, &p->g_adj, &p->g_ph})
        if (g->exec) cudaGraphExecDestroy(g->exec);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->cap2) cudaStreamDestroy(p->cap2);
    for (auto &e : p->ovev) cudaEventDestroy(e);
    for (auto &e : p->ev) cudaEventDestroy(e);
    delete p;
}

int efwi_autotune(efwi_plan *p);   // k_fused.cu

extern "C" int efwi_plan_create(efwi_plan **out, const efwi_plan_desc *d) {
    if (!out) return fail(nullptr, EFWI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return fail(nullptr, EFWI_ERR_ARG, "desc is NULL");
    if (d->nx < 1 || d->nz < 1 || !(d->dx > 0) || !(d->dz > 0) || d->nt < 1 || !(d->dt > 0))
        return fail(nullptr, EFWI_ERR_ARG, "grid sizes, spacings, nt and dt must be positive");
    if (d->npml < 1 || d->npml > 200) return fail(nullptr, EFWI_ERR_ARG, "npml must be in [1, 200]");
    if (!(d->pml_R > 0 && d->pml_R < 1)) return fail(nullptr, EFWI_ERR_ARG, "pml_R must be in (0, 1)");
    if (d->ns < 1) return fail(nullptr, EFWI_ERR_ARG, "ns must be >= 1");
    if (d->ntr < 0) return fail(nullptr, EFWI_ERR_ARG, "ntr must be >= 0");
    if (!d->src_xz || !d->mt || !d->wavelet || !d->tr_ptr || !d->ref_vp || !d->ref_vs || !d->ref_rho)
        return fail(nullptr, EFWI_ERR_ARG, "a required host array is NULL");
    if (d->ntr > 0 && (!d->ch_xz || !d->ch_t)) return fail(nullptr, EFWI_ERR_ARG, "channel arrays are NULL");
    if (d->das_mode != EFWI_DAS_STRAIN && d->das_mode != EFWI_DAS_STRAIN_RATE && d->das_mode != EFWI_DAS_VELOCITY)
        return fail(nullptr, EFWI_ERR_ARG, "unknown das_mode");
    if (d->ntr > 0 && d->das_mode != EFWI_DAS_VELOCITY && !(d->gauge > 0))
        return fail(nullptr, EFWI_ERR_ARG, "gauge must be > 0");
    if (d->ckpt_store < EFWI_STORE_FP32 || d->ckpt_store > EFWI_STORE_BF16)
        return fail(nullptr, EFWI_ERR_ARG, "unknown ckpt_store");
    if (d->exec != EFWI_EXEC_PLAIN && d->exec != EFWI_EXEC_BATCHED) return fail(nullptr, EFWI_ERR_ARG, "unknown exec");
    if (d->ckpt_interval < EFWI_CKPT_AUTO)
        return fail(nullptr, EFWI_ERR_ARG, "ckpt_interval must be >= 0 or EFWI_CKPT_AUTO");
    if (d->stored_steps < 0) return fail(nullptr, EFWI_ERR_ARG, "stored_steps must be >= 0");
    if (d->stored_steps > 0 && d->overlap == EFWI_OVERLAP_ON && d->ckpt_interval != EFWI_CKPT_AUTO &&
        d->ckpt_interval < d->nt)
        return fail(nullptr, EFWI_ERR_ARG, "stored_steps > 0 cannot be combined with a forced overlap");
    if (d->snap_store < EFWI_STORE_FP32 || d->snap_store > EFWI_STORE_BF16)
        return fail(nullptr, EFWI_ERR_ARG, "unknown snap_store");
    if (d->snap_store != EFWI_STORE_FP32 && d->exec != EFWI_EXEC_BATCHED)
        return fail(nullptr, EFWI_ERR_ARG, "FP16/BF16 snapshots need EXEC_BATCHED (EXEC_PLAIN keeps FP32)");
    if (d->snap_store != EFWI_STORE_FP32 && d->overlap == EFWI_OVERLAP_ON)
        return fail(nullptr, EFWI_ERR_ARG, "the overlapped recompute schedule keeps FP32 snapshots");
    if (d->tr_ptr[0] != 0 || d->tr_ptr[d->ns] != d->ntr) return fail(nullptr, EFWI_ERR_ARG, "tr_ptr must run 0..ntr");
    for (int s = 0; s < d->ns; ++s)
        if (d->tr_ptr[s + 1] < d->tr_ptr[s]) return fail(nullptr, EFWI_ERR_ARG, "tr_ptr must be non-decreasing");
    if (d->exec == EFWI_EXEC_BATCHED &&
        ((d->tile_x != 0 || d->tile_z != 0) && (d->tile_x <= 0 || d->tile_z <= 0)))
        return fail(nullptr, EFWI_ERR_ARG, "tile_x and tile_z must both be 0 or both positive");
    if (d->stencil < EFWI_STENCIL_AUTO || d->stencil > EFWI_STENCIL_TMA_STAGED ||
        d->adj_stencil < EFWI_STENCIL_AUTO || d->adj_stencil > EFWI_STENCIL_TMA_STAGED)
        return fail(nullptr, EFWI_ERR_ARG, "unknown stencil");
    if (d->exec == EFWI_EXEC_BATCHED &&
        ((d->adj_tile_x != 0 || d->adj_tile_z != 0) && (d->adj_tile_x <= 0 || d->adj_tile_z <= 0)))
        return fail(nullptr, EFWI_ERR_ARG, "adj_tile_x and adj_tile_z must both be 0 or both positive");
    if (d->overlap < EFWI_OVERLAP_AUTO || d->overlap > EFWI_OVERLAP_ON)
        return fail(nullptr, EFWI_ERR_ARG, "unknown overlap");
    if (d->adj_form < EFWI_ADJ_FORM_AUTO || d->adj_form > EFWI_ADJ_FORM_SCALED)
        return fail(nullptr, EFWI_ERR_ARG, "unknown adj_form");
    if (d->adj_form == EFWI_ADJ_FORM_SCALED &&
        (d->exec != EFWI_EXEC_BATCHED || d->adj_stencil > EFWI_STENCIL_TMA))
        return fail(nullptr, EFWI_ERR_ARG, "the scaled-stress adjoint needs EXEC_BATCHED and adj_stencil AUTO, "
                                           "LOADS or TMA");
    if (d->force)
        for (int k = 0; k < 2 * d->ns; ++k)
            if (!std::isfinite(d->force[k])) return fail(nullptr, EFWI_ERR_ARG, "force components must be finite");

    const long long ncell = (long long)d->nx * d->nz;
    double vmax = d->pml_vmax;
    if (!(vmax > 0)) {
        vmax = 0;
        for (long long k = 0; k < ncell; ++k) vmax = std::max(vmax, (double)d->ref_vp[k]);
    }
    for (long long k = 0; k < ncell; ++k)
        if (!(d->ref_vs[k] > 0) || !(d->ref_rho[k] > 0) || !(d->ref_vp[k] > 0))
            return fail(nullptr, EFWI_ERR_ARG, "reference model must have Vp, Vs, rho > 0");
    const double cfl = d->dt * vmax * std::sqrt(2.0) * (9.0 / 8.0 + 1.0 / 24.0) / std::min(d->dx, d->dz);
    if (!(cfl < 1.0)) {
        char b[160];
        snprintf(b, sizeof b, "CFL number %.4f >= 1 (dt=%g, vmax=%g)", cfl, d->dt, vmax);
        return fail(nullptr, EFWI_ERR_CFL, b);
    }

    efwi_plan *p = new (std::nothrow) efwi_plan();
    if (!p) return fail(nullptr, EFWI_ERR_OOM, "host allocation failed");
    p->d = *d;
    p->d.src_xz = nullptr; p->d.mt = nullptr; p->d.wavelet = nullptr; p->d.tr_ptr = nullptr;
    p->d.ch_xz = nullptr; p->d.ch_t = nullptr; p->d.win = nullptr;
    p->d.ref_vp = p->d.ref_vs = p->d.ref_rho = nullptr;
    p->d.force = nullptr;
    p->d.pml_vmax = vmax;
    const int P = d->npml + 1;
    p->P = P;
    const int ns = d->ns, nt = d->nt;
    const int NZ = d->nz + 2 * P;
    p->nzp = NZ;

    // --- per-shot geometry -------------------------------------------------
    p->shots.resize(ns);
    long long off = 0, psx = 0, psz = 0;
    int profx = 0;
    for (int s = 0; s < ns; ++s) {
        int x0 = 0, w = d->nx;
        if (d->win) { x0 = d->win[2 * s]; w = d->win[2 * s + 1]; }
        if (x0 < 0 || w < 1 || x0 + w > d->nx) {
            free_plan(p);
            return fail(nullptr, EFWI_ERR_ARG, "window of shot " + std::to_string(s) + " outside the grid");
        }
        ShotDev &sh = p->shots[s];
        memset(&sh, 0, sizeof sh);
        sh.P = P; sh.x0 = x0; sh.w = w;
        sh.NX = w + 2 * P; sh.NZ = NZ;
        sh.pitch = ((sh.NX + 7) / 8) * 8 + 8;
        sh.off = off;
        off += (((long long)(NZ + 2 * EFWI_GZ) * sh.pitch + 63) / 64) * 64;
        sh.psx = psx; psx += (long long)NZ * 2 * P;
        sh.psz = psz; psz += (long long)2 * P * sh.NX;
        sh.profx = profx; profx += sh.NX;
        sh.tr0 = d->tr_ptr[s]; sh.ntr = d->tr_ptr[s + 1] - d->tr_ptr[s];
        sh.mxx = (float)d->mt[3 * s]; sh.mzz = (float)d->mt[3 * s + 1]; sh.mxz = (float)d->mt[3 * s + 2];
        p->padded_cells += (long long)sh.NX * NZ;
        p->physical_cells += (long long)w * d->nz;
        p->max_nx = std::max(p->max_nx, sh.NX);
        if (off > (1LL << 31) * 8) { free_plan(p); return fail(nullptr, EFWI_ERR_ARG, "problem too large"); }
    }
    p->fsz_total = off;
    p->psx_total = psx; p->psz_total = psz;
    p->H = 2 * psx + 2 * psz;
    p->prof_x_total = profx;

    // --- sources, receivers, adjoint gather, wavelet increments -------------------
    AcqHost acq;
    {
        std::string err;
        if (build_acq(*d, p->shots, acq, err) != EFWI_OK) {
            free_plan(p);
            return fail(nullptr, EFWI_ERR_ARG, err);
        }
        commit_acq(p, acq);
    }
    const int ntr = d->ntr;
    std::vector<int> &h_off = acq.h_off;
    std::vector<float> &h_w = acq.h_w, &h_dw = acq.h_dw, &h_wv = acq.h_wv;
    std::vector<int> &g_shot = acq.g_shot, &g_field = acq.g_field, &g_off = acq.g_off, &g_ptr = acq.g_ptr,
                     &g_tr = acq.g_tr;
    std::vector<float> &g_w = acq.g_w;

    const int X = p->prof_x_total;
    std::vector<float> h_prof(4 * (size_t)X + 4 * (size_t)NZ);
    for (int s = 0; s < ns; ++s) {
        const ShotDev &sh = p->shots[s];
        cpml_axis(sh.NX, P, d->dx, d->npml, d->pml_R, vmax, d->pml_f0, d->dt, false, &h_prof[sh.profx], &h_prof[X + sh.profx]);
        cpml_axis(sh.NX, P, d->dx, d->npml, d->pml_R, vmax, d->pml_f0, d->dt, true, &h_prof[2 * X + sh.profx],
                  &h_prof[3 * X + sh.profx]);
    }
    float *zp = &h_prof[4 * (size_t)X];
    cpml_axis(NZ, P, d->dz, d->npml, d->pml_R, vmax, d->pml_f0, d->dt, false, zp, zp + NZ);
    cpml_axis(NZ, P, d->dz, d->npml, d->pml_R, vmax, d->pml_f0, d->dt, true, zp + 2 * NZ, zp + 3 * NZ);

    // --- device allocation -------------------------------------------------------
    // (the snapshot slots and the checkpoints come last: their number depends on the
    // checkpoint schedule, which EFWI_CKPT_AUTO chooses from the memory left)
    Alloc A{p};
    const long long F = p->fsz_total;
    p->snap_store = d->snap_store;
    p->ck.store = d->ckpt_store;
    A(&p->shots_d, (size_t)ns, "shots");
    const bool batched = d->exec == EFWI_EXEC_BATCHED;
    // the batched path's two state buffers are one allocation (one tensor map covers both)
    A(&p->state[0], (size_t)((batched ? 10 : 5) * F), "state");
    A(&p->mat, (size_t)(5 * F), "materials");
    A(&p->adj[0], (size_t)((batched ? 10 : 5) * F), "adjoint state");
    A(&p->dev_err, (size_t)1, "device error flag");
    A(&p->G, (size_t)(5 * F), "imaging accumulators");
    if (batched) {
        A(&p->Gtot, (size_t)(5 * F), "Kahan totals");
        A(&p->Gcmp, (size_t)(5 * F), "Kahan compensation");
    }
    A(&p->psi, (size_t)(4 * p->H), "psi");
    A(&p->apsi, (size_t)(4 * p->H), "adjoint psi");
    A(&p->prof, h_prof.size(), "profiles");
    A(&p->dw, h_dw.size(), "wavelet increments");
    if (p->has_force) A(&p->wv, h_wv.size(), "wavelet");
    A(&p->ref, (size_t)(3 * ncell), "reference model");
    A(&p->tr_shot, (size_t)std::max(ntr, 1), "trace shots");
    A(&p->tr_off, h_off.size(), "trace offsets");
    A(&p->tr_w, h_w.size(), "trace weights");
    A(&p->tr_acc, (size_t)std::max(ntr, 1), "trace accumulators");
    A(&p->tr_coef, (size_t)std::max(ntr, 1), "trace coefficients");
    if (p->gather.n_tgt > 0) {
        A(&p->gather.tgt_shot, g_shot.size(), "gather");
        A(&p->gather.tgt_field, g_field.size(), "gather");
        A(&p->gather.tgt_off, g_off.size(), "gather");
        A(&p->gather.ptr, g_ptr.size(), "gather");
        A(&p->gather.tr, g_tr.size(), "gather");
        A(&p->gather.w, g_w.size(), "gather");
    }
    A(&p->resid, (size_t)std::max(ntr, 1) * nt, "residual");
    A(&p->dbuf, (size_t)std::max(ntr, 1) * nt, "data buffer");
    A(&p->partial, (size_t)kPartials + 8, "reduction scratch");

    // --- checkpoint schedule ---------------------------------------------------
    const size_t snap_el = p->snap_store == EFWI_STORE_FP32 ? 4 : 2;
    const size_t ck_el = p->ck.store == EFWI_STORE_FP32 ? 4 : 2;
    const size_t slot_bytes = 2 * F * snap_el + (size_t)2 * ns * kMaxPad * 4;
    const size_t ck_bytes = 5 * F * ck_el + 2 * p->H * 4 + 5 * ns * 4;
    // device bytes of a schedule: interval k, the steps before n_split recomputed
    // from checkpoints (k slots), the rest kept by the forward pass
    auto sched_bytes = [&](int k, int split) {
        if (k >= nt) return (size_t)nt * slot_bytes + ck_bytes;
        return (size_t)(k + nt - split) * slot_bytes + (size_t)((split + k - 1) / k) * ck_bytes;
    };
    int K = d->ckpt_interval;
    const int Ksqrt = std::min(nt, (int)std::ceil(std::sqrt((double)nt)));
    int split = nt;
    if (K == EFWI_CKPT_AUTO) {
        size_t fr = 0, tot = 0;
        K = Ksqrt;
        if (A.ok && cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
            const size_t keep = tot / 20 + (2ull << 30);
            const size_t room = fr > keep ? fr - keep : 0;
            if (sched_bytes(nt, 0) <= room) {
                K = nt;
            } else if (K < nt && d->overlap != EFWI_OVERLAP_ON) {
                // fewest recomputed segments whose schedule fits
                for (int m = 1; m * K < nt; ++m)
                    if (sched_bytes(K, m * K) <= room) { split = m * K; break; }
            }
        } else {
            cudaGetLastError();
        }
    } else {
        if (K == 0) K = Ksqrt;
        K = std::min(K, nt);
        if (K < nt && d->stored_steps > 0) {
            const long long first = std::max(0LL, (long long)nt - d->stored_steps);
            split = (int)std::min((long long)nt, (first + K - 1) / K * K);
        }
    }
    if (K < nt && split == 0) K = nt;          // every step kept: the full-storage schedule
    p->K = K;
    p->n_split = K >= nt ? 0 : split;
    p->ck.n = K >= nt ? 1 : (p->n_split + K - 1) / K;
    p->nslots = K >= nt ? nt : K + (nt - p->n_split);
    // the second half of the segment buffer exists only if the autotuner keeps the
    // overlapped recompute/adjoint schedule (or the caller forces it)
    p->seg_double = false;
    if (p->snap_store == EFWI_STORE_FP32) {
        A(&p->seg, (size_t)p->nslots * 2 * F, "snapshot slots");
    } else {
        A((__half **)&p->segh, (size_t)p->nslots * 2 * F, "FP16/BF16 snapshots");
        A(&p->segmax, (size_t)p->nslots * 2 * ns * kMaxPad, "snapshot maxima");
    }
    const size_t nck_el = (size_t)p->ck.n * 5 * F;
    if (p->ck.store == EFWI_STORE_FP32) A((float **)&p->ck.fields, nck_el, "checkpoints");
    else {
        A((__half **)&p->ck.fields, nck_el, "checkpoints");
        A(&p->ck.scale, (size_t)p->ck.n * 5 * ns, "checkpoint scales");
    }
    A(&p->ck.psi, (size_t)p->ck.n * 2 * p->H, "checkpoint psi");
    if (!A.ok) {
        free_plan(p);
        return fail(nullptr, EFWI_ERR_OOM, A.what);
    }
    if (batched) {
        p->state[1] = p->state[0] + 5 * F;
        p->adj[1] = p->adj[0] + 5 * F;
    }

    // --- upload --------------------------------------------------------------------
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (bytes) cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(p->shots_d, p->shots.data(), sizeof(ShotDev) * ns);
    up(p->prof, h_prof.data(), h_prof.size() * 4);
    up(p->dw, h_dw.data(), h_dw.size() * 4);
    if (p->has_force) up(p->wv, h_wv.data(), h_wv.size() * 4);
    up(p->ref, d->ref_vp, ncell * 4);
    up(p->ref + ncell, d->ref_vs, ncell * 4);
    up(p->ref + 2 * ncell, d->ref_rho, ncell * 4);
    if (ntr > 0) {
        up(p->tr_shot, p->trace_shot.data(), 4 * (size_t)ntr);
        up(p->tr_off, h_off.data(), 4 * h_off.size());
        up(p->tr_w, h_w.data(), 4 * h_w.size());
    }
    if (p->gather.n_tgt > 0) {
        up(p->gather.tgt_shot, g_shot.data(), 4 * g_shot.size());
        up(p->gather.tgt_field, g_field.data(), 4 * g_field.size());
        up(p->gather.tgt_off, g_off.data(), 4 * g_off.size());
        up(p->gather.ptr, g_ptr.data(), 4 * g_ptr.size());
        up(p->gather.tr, g_tr.data(), 4 * g_tr.size());
        up(p->gather.w, g_w.data(), 4 * g_w.size());
    }
    p->ev.resize(8192);
    p->ev_kind.assign(4096, 0);
    cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&p->cap2, cudaStreamNonBlocking);
    p->ovev.resize(2 * p->ck.n + 2);   // events of the overlapped schedule (dependency only)
    for (auto &e : p->ovev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&p->n_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    for (auto &e : p->ev) cudaEventCreate(&e);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        std::string m = std::string("plan upload failed: ") + cudaGetErrorString(e);
        free_plan(p);
        return fail(nullptr, EFWI_ERR_CUDA, m);
    }
    if (d->exec == EFWI_EXEC_BATCHED) {
        p->tile_x = d->tile_x; p->tile_z = d->tile_z;
        p->adj_tile_x = d->adj_tile_x; p->adj_tile_z = d->adj_tile_z;
        int rc = efwi_autotune(p);
        if (rc != EFWI_OK) {
            std::string m = p->err;
            free_plan(p);
            return fail(nullptr, rc, m);
        }
    }
    *out = p;
    return EFWI_OK;
}

extern "C" int efwi_plan_destroy(efwi_plan *p) {
    if (!p) return EFWI_OK;
    cudaDeviceSynchronize();
    free_plan(p);
    return EFWI_OK;
}

extern "C" const char *efwi_last_error(const efwi_plan *p) {
    if (p) return p->err.c_str();
    return g_thread_err.c_str();
}

extern "C" int efwi_plan_info(const efwi_plan *p, efwi_plan_info_t *info) {
    if (!p || !info) return fail(nullptr, EFWI_ERR_ARG, "NULL argument");
    info->ckpt_interval = p->K;
    info->n_ckpt = p->ck.n;
    info->stored_steps = p->d.nt - p->n_split;
    info->tile_x = p->tile_x;
    info->tile_z = p->tile_z;
    info->adj_tile_x = p->adj_tile_x;
    info->adj_tile_z = p->adj_tile_z;
    info->stencil = p->stencil;
    info->stages = p->stencil >= EFWI_STENCIL_TMA ? p->tma_stages : 0;
    info->adj_stencil = p->adj_stencil;
    info->adj_stages = p->adj_stencil == EFWI_STENCIL_TMA ? p->tma_adj_stages : 0;
    info->overlap_fwd_blocks = p->ov_fwd;
    info->overlap_adj_blocks = p->ov_adj;
    info->workspace_bytes = p->bytes;
    info->padded_cells = p->padded_cells;
    info->physical_cells = p->physical_cells;
    info->launches = p->launches;
    info->layout = p->stencil >= EFWI_STENCIL_TMA ? p->tma_vec : 0;
    info->staged_stores = p->stencil >= EFWI_STENCIL_TMA ? p->tma_store : 0;
    info->adj_persistent = p->adj_stencil == EFWI_STENCIL_LOADS && p->adj_grid > 0;
    info->snap_store = p->snap_store;
    info->prefetch = (p->stencil >= EFWI_STENCIL_TMA && p->tma_pf ? 1 : 0) | (p->adj_pf ? 2 : 0);
    info->adj_form = p->adj_form;
    info->adj_layout = p->adj_form == EFWI_ADJ_FORM_SCALED && p->adj_stencil == EFWI_STENCIL_TMA ? p->adjs_vec : 0;
    return EFWI_OK;
}

extern "C" int efwi_sync_status(efwi_plan *p, efwi_stream_t stream) {
    if (!p) return fail(nullptr, EFWI_ERR_ARG, "plan is NULL");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail(p, EFWI_ERR_CUDA, std::string("stream sync: ") + cudaGetErrorString(e));
    int flag = 0;
    cudaMemcpy(&flag, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (flag) {
        cudaMemset(p->dev_err, 0, sizeof(int));
        if (flag & EFWI_FLAG_TIMEOUT) {
            // a copy may have stalled in hardware: the workspace and its pipelines are no
            // longer trusted, so every later call on this plan fails until it is recreated
            p->broken = true;
            return fail(p, EFWI_ERR_TIMEOUT, "a kernel gave up a bounded wait; results of that call are invalid "
                                             "and the plan must be destroyed and created again");
        }
        if (flag & EFWI_FLAG_SELFTEST)
            return fail(p, EFWI_ERR_TIMEOUT, "the timeout self-test's bounded wait expired (as intended)");
        if (flag & EFWI_FLAG_SHEAR)
            return fail(p, EFWI_ERR_NAN, "a gradient needs mu > 0 (Vs > 0) on the physical cells, and the scaled-stress "
                                         "adjoint also lambda + mu > 0 (Vp > Vs) there and on the half cells next "
                                         "to them; the gradient of that call is invalid");
        return fail(p, EFWI_ERR_NAN, "the model holds a non-finite value or a non-positive density; results of "
                                     "that call are invalid");
    }
    return EFWI_OK;
}

extern "C" int efwi_prof_enable(efwi_plan *p, int every) {
    if (!p || every < 0) return fail(p, EFWI_ERR_ARG, "bad arguments to efwi_prof_enable");
    cudaDeviceSynchronize();
    for (GraphCache *g : {&p->g_fwd, &p->g_fwd_ck, &p->g_adj, &p->g_ph})
        if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
    p->prof_every = every;
    p->prof_counter[0] = p->prof_counter[1] = 0;
    p->ev_used = 0;
    return EFWI_OK;
}

extern "C" int efwi_prof_read(efwi_plan *p, int kernel, double *total_ms, long long *count) {
    if (!p || !total_ms || !count || kernel < 0 || kernel > 1) return fail(p, EFWI_ERR_ARG, "bad arguments to efwi_prof_read");
    double ms = 0;
    long long c = 0;
    for (int k = 0; k + 1 < p->ev_used; k += 2) {
        if (p->ev_kind[k / 2] != kernel) continue;
        if (cudaEventSynchronize(p->ev[k + 1]) != cudaSuccess) return fail(p, EFWI_ERR_CUDA, "event sync failed");
        float t = 0;
        if (cudaEventElapsedTime(&t, p->ev[k], p->ev[k + 1]) == cudaSuccess) { ms += t; ++c; }
    }
    *total_ms = ms;
    *count = c;
    return EFWI_OK;
}

extern "C" int efwi_zoi_weights(int ns, int nx, int nz, double dx, double dz, const efwi_zoi_desc *z, float *b,
                                float *bp, uint8_t *sink, efwi_stream_t stream) {
    std::string err;
    int rc = launch_zoi(ns, nx, nz, dx, dz, z, b, bp, sink, (cudaStream_t)stream, err);
    if (rc != EFWI_OK) return fail(nullptr, rc, err);
    return EFWI_OK;
}

extern "C" int efwi_collapse(int ns, int nx, int nz, const float *x, const float *b, const float *bp,
                             const uint8_t *sink, float *out, efwi_stream_t stream) {
    if (ns < 1 || nx < 1 || nz < 1) return fail(nullptr, EFWI_ERR_ARG, "ns, nx and nz must be >= 1");
    if (!x || !b || !bp || !sink || !out) return fail(nullptr, EFWI_ERR_ARG, "NULL device pointer");
    launch_collapse(ns, (long long)nx * nz, x, b, bp, sink, out, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, EFWI_ERR_CUDA, cudaGetErrorString(e));
    return EFWI_OK;
}

// b, bp, sink all given, or all NULL for the weights the plan holds (ns components)
int efwi::resolve_zoi(efwi_plan *p, int ns, const float *&b, const float *&bp, const uint8_t *&sink) {
    if (b && bp && sink) return EFWI_OK;
    if (b || bp || sink)
        return fail(p, EFWI_ERR_ARG, "b, bp and sink must all be given, or all be NULL for the plan's weights");
    if (!p->zoi_b)
        return fail(p, EFWI_ERR_ARG, "no zone-of-influence weights: pass b, bp, sink or call efwi_plan_set_zoi");
    if (ns != p->d.ns)
        return fail(p, EFWI_ERR_ARG, "the plan's zone-of-influence weights hold its own ns components");
    b = p->zoi_b;
    bp = p->zoi_bp;
    sink = p->zoi_sink;
    return EFWI_OK;
}

extern "C" int efwi_plan_set_zoi(efwi_plan *p, const efwi_zoi_desc *z, efwi_stream_t stream) {
    if (!p) return fail(nullptr, EFWI_ERR_ARG, "plan is NULL");
    const size_t n = (size_t)p->d.ns * p->d.nz * p->d.nx;
    if (!p->zoi_b) {
        Alloc A{p};
        A(&p->zoi_b, n, "zone-of-influence b");
        A(&p->zoi_bp, n, "zone-of-influence b'");
        A(&p->zoi_sink, n, "sinkhole flags");
        if (!A.ok) {
            for (void *q : {(void *)p->zoi_b, (void *)p->zoi_bp, (void *)p->zoi_sink})
                if (q) cudaFree(q);
            p->zoi_b = p->zoi_bp = nullptr;
            p->zoi_sink = nullptr;
            return fail(p, EFWI_ERR_OOM, A.what);
        }
    }
    std::string err;
    const int rc = launch_zoi(p->d.ns, p->d.nx, p->d.nz, p->d.dx, p->d.dz, z, p->zoi_b, p->zoi_bp, p->zoi_sink,
                              (cudaStream_t)stream, err);
    if (rc != EFWI_OK) return fail(p, rc, err);
    return EFWI_OK;
}

extern "C" int efwi_regularization_grad_n(efwi_plan *p, int ns, const float *m, const float *b, const float *bp,
                                          const uint8_t *sink, double eta, double *phi_reg, float *g,
                                          efwi_stream_t stream) {
    if (!p) return fail(nullptr, EFWI_ERR_ARG, "plan is NULL");
    if (ns < 1) return fail(p, EFWI_ERR_ARG, "ns must be >= 1");
    if (int rc = resolve_zoi(p, ns, b, bp, sink)) return rc;
    if (!m || !phi_reg || !g) return fail(p, EFWI_ERR_ARG, "NULL device pointer");
    if (!std::isfinite(eta)) return fail(p, EFWI_ERR_ARG, "eta must be finite");
    nvtxRangePushA("efwi consistency term");
    launch_reg(p, m, b, bp, sink, eta, phi_reg, g, 0, (cudaStream_t)stream, ns);
    nvtxRangePop();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(p, EFWI_ERR_CUDA, cudaGetErrorString(e));
    return EFWI_OK;
}

extern "C" int efwi_regularization_grad(efwi_plan *p, const float *m, const float *b, const float *bp,
                                        const uint8_t *sink, double eta, double *phi_reg, float *g,
                                        efwi_stream_t stream) {
    if (!p) return fail(nullptr, EFWI_ERR_ARG, "plan is NULL");
    if (int rc = resolve_zoi(p, p->d.ns, b, bp, sink)) return rc;
    if (!m || !phi_reg || !g) return fail(p, EFWI_ERR_ARG, "NULL device pointer");
    if (!std::isfinite(eta)) return fail(p, EFWI_ERR_ARG, "eta must be finite");
    nvtxRangePushA("efwi consistency term");
    launch_reg(p, m, b, bp, sink, eta, phi_reg, g, 0, (cudaStream_t)stream);
    nvtxRangePop();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(p, EFWI_ERR_CUDA, cudaGetErrorString(e));
    return EFWI_OK;
}

int efwi::check_same_shape(efwi_plan *p, const efwi_plan_desc *d, std::string &err) {
    const efwi_plan_desc &o = p->d;
    const bool gauge_used = d->ntr > 0 && d->das_mode != EFWI_DAS_VELOCITY;
    if (d->nx != o.nx || d->nz != o.nz || d->dx != o.dx || d->dz != o.dz || d->nt != o.nt || d->dt != o.dt ||
        d->npml != o.npml || d->ns != o.ns || d->ntr != o.ntr || d->das_mode != o.das_mode ||
        (gauge_used && d->gauge != o.gauge)) {
        err = "grid, time axis, npml, ns, ntr, das_mode and gauge must equal the plan's";
        return EFWI_ERR_ARG;
    }
    if (!d->src_xz || !d->mt || !d->wavelet || !d->tr_ptr || (d->ntr > 0 && (!d->ch_xz || !d->ch_t))) {
        err = "a required host array is NULL";
        return EFWI_ERR_ARG;
    }
    for (int s = 0; s < d->ns; ++s) {
        const ShotDev &sh = p->shots[s];
        const int x0 = d->win ? d->win[2 * s] : 0, w = d->win ? d->win[2 * s + 1] : d->nx;
        if (d->tr_ptr[s] != sh.tr0 || d->tr_ptr[s + 1] - d->tr_ptr[s] != sh.ntr || x0 != sh.x0 || w != sh.w) {
            err = "the windows and traces per shot must equal the plan's (shot " + std::to_string(s) + ")";
            return EFWI_ERR_ARG;
        }
    }
    if ((d->force != nullptr) != p->has_force) {
        err = "force sources must stay force sources (and moment tensors moment tensors)";
        return EFWI_ERR_ARG;
    }
    if (d->force)
        for (int k = 0; k < 2 * d->ns; ++k)
            if (!std::isfinite(d->force[k])) {
                err = "force components must be finite";
                return EFWI_ERR_ARG;
            }
    return EFWI_OK;
}

extern "C" int efwi_plan_rebind(efwi_plan *p, const efwi_plan_desc *d, efwi_stream_t stream) {
    if (!p || !d) return fail(p, EFWI_ERR_ARG, "efwi_plan_rebind: plan and desc must be non-NULL");
    if (p->broken)
        return fail(p, EFWI_ERR_TIMEOUT, "a bounded device wait of an earlier call expired; destroy this plan");
    {
        std::string e;
        if (check_same_shape(p, d, e) != EFWI_OK) return fail(p, EFWI_ERR_ARG, "efwi_plan_rebind: " + e);
    }
    AcqHost h;
    std::string err;
    if (build_acq(*d, p->shots, h, err) != EFWI_OK) return fail(p, EFWI_ERR_ARG, "efwi_plan_rebind: " + err);
    cudaStream_t st = (cudaStream_t)stream;
    const bool same_shape = (int)h.g_shot.size() == p->gather.n_tgt && h.gather_ptr == p->gather_ptr &&
                            (int)h.g_tr.size() == p->gather_nnz;
    if (!same_shape) {
        // the captured time loops hold the gather's launch shape and arrays: drop them
        cudaStreamSynchronize(st);
        cudaDeviceSynchronize();
        for (GraphCache *g : {&p->g_fwd, &p->g_fwd_ck, &p->g_adj, &p->g_ph})
            if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
        GatherCSR &G = p->gather;
        p->bytes -= (size_t)p->gather.n_tgt * 4 * 3 + (size_t)(p->gather.n_tgt + 1) * 4 + (size_t)p->gather_nnz * 8;
        for (void *q : {(void *)G.tgt_shot, (void *)G.tgt_field, (void *)G.tgt_off, (void *)G.ptr, (void *)G.tr,
                        (void *)G.w})
            if (q) cudaFree(q);
        G.tgt_shot = G.tgt_field = G.tgt_off = G.ptr = G.tr = nullptr;
        G.w = nullptr;
        Alloc A{p};
        if (!h.g_shot.empty()) {
            A(&G.tgt_shot, h.g_shot.size(), "gather");
            A(&G.tgt_field, h.g_field.size(), "gather");
            A(&G.tgt_off, h.g_off.size(), "gather");
            A(&G.ptr, h.g_ptr.size(), "gather");
            A(&G.tr, h.g_tr.size(), "gather");
            A(&G.w, h.g_w.size(), "gather");
        }
        if (!A.ok) {
            p->broken = true;
            return fail(p, EFWI_ERR_OOM, "efwi_plan_rebind: " + A.what + "; the plan must be destroyed");
        }
    }
    commit_acq(p, h);
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (bytes && dst) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    up(p->shots_d, p->shots.data(), sizeof(ShotDev) * p->shots.size());
    up(p->dw, h.h_dw.data(), 4 * h.h_dw.size());
    if (p->has_force) up(p->wv, h.h_wv.data(), 4 * h.h_wv.size());
    if (d->ntr > 0) {
        up(p->tr_off, h.h_off.data(), 4 * h.h_off.size());
        up(p->tr_w, h.h_w.data(), 4 * h.h_w.size());
    }
    if (p->gather.n_tgt > 0) {
        up(p->gather.tgt_shot, h.g_shot.data(), 4 * h.g_shot.size());
        up(p->gather.tgt_field, h.g_field.data(), 4 * h.g_field.size());
        up(p->gather.tgt_off, h.g_off.data(), 4 * h.g_off.size());
        up(p->gather.ptr, h.g_ptr.data(), 4 * h.g_ptr.size());
        up(p->gather.tr, h.g_tr.data(), 4 * h.g_tr.size());
        up(p->gather.w, h.g_w.data(), 4 * h.g_w.size());
    }
    int rc = refresh_tiles(p, p->tiles, st);
    if (!rc) rc = refresh_tiles(p, p->adj_tiles, st);
    if (rc) {
        p->broken = true;
        return fail(p, rc, "efwi_plan_rebind: tile list mismatch; the plan must be destroyed");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(p, EFWI_ERR_CUDA, std::string("efwi_plan_rebind: ") + cudaGetErrorString(e));
    return EFWI_OK;
}
