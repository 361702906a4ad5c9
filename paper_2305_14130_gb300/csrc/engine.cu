// Time-loop orchestration behind the C ABI: forward modelling, the
// checkpointed adjoint-state gradient and the extended objective.
//
// Gradient schedule (uniform checkpoints, one recompute pass):
//   forward n = 0..nt-1, saving the state x^n every K steps (FP32 or scaled
//   FP16/BF16); residual r = d - d_obs and phi = 1/2 |r|^2 in FP64;
//   for every segment [n0, n1) from the last: restore x^{n0}, recompute the
//   segment keeping v^{n+1/2} of each step, then run the adjoint steps
//   n1-1 .. n0, each accumulating the zero-lag imaging sums.  With K >= nt the
//   first forward pass already keeps every v^{n+1/2} and nothing is recomputed.
// The kept velocities ("snapshots", one slot per step of a segment) are FP32,
// written by the step that computes them, or scaled FP16/BF16: the step that
// computes v^{n+1/2} accumulates its maxima into the slot's scale, the next
// step writes the 2-byte copy, and a small kernel packs the segment's last step.
// EXEC_PLAIN launches one kernel per half-step and shot; EXEC_BATCHED runs all
// shots in fused launches and replays the time loop from CUDA graphs.
#include <algorithm>
#include <cmath>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "plan.hpp"

using namespace efwi;

namespace {

// NVTX range over a phase of a call (host timeline; no-ops without a profiler).
// Inside CUDA graphs the ranges mark the replay call, not each replayed kernel.
struct Phase {
    explicit Phase(const char *name) { nvtxRangePushA(name); }
    ~Phase() { nvtxRangePop(); }
    Phase(const Phase &) = delete;
    Phase &operator=(const Phase &) = delete;
};

int cuda_status(efwi_plan *p, const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        p->err = std::string(where) + ": " + cudaGetErrorString(e);
        return EFWI_ERR_CUDA;
    }
    return EFWI_OK;
}

int check_model_args(efwi_plan *p, const float *vp, const float *vs, const float *rho) {
    if (p->broken) {
        p->err = "a bounded device wait of an earlier call expired; destroy this plan and create it again";
        return EFWI_ERR_TIMEOUT;
    }
    if (!vp || !vs || !rho) {
        p->err = "model pointers must be non-NULL device pointers";
        return EFWI_ERR_ARG;
    }
    return EFWI_OK;
}

void reset_forward_state(efwi_plan *p, cudaStream_t st) {
    for (int k = 0; k < 2; ++k)
        if (p->state[k]) cudaMemsetAsync(p->state[k], 0, sizeof(float) * 5 * p->fsz_total, st);
    cudaMemsetAsync(p->psi, 0, sizeof(float) * 4 * p->H, st);
    if (p->d.ntr > 0) cudaMemsetAsync(p->tr_acc, 0, sizeof(double) * p->d.ntr, st);
    p->scur = 0;
    p->psi_v = 0;
    p->psi_s = 0;
}

float *seg_x(efwi_plan *p, int slot) { return p->seg + (size_t)slot * 2 * p->fsz_total; }
float *seg_z(efwi_plan *p, int slot) { return p->seg + (size_t)slot * 2 * p->fsz_total + p->fsz_total; }
// slot of the segment buffer half used by segment sgi in the overlapped schedule
int seg_slot(efwi_plan *p, int sgi, int k) { return (p->seg_double ? (sgi & 1) * p->K : 0) + k; }

bool half_snaps(const efwi_plan *p) { return p->snap_store != EFWI_STORE_FP32; }

// maxima of the reduced-precision snapshot slots [k0, k1) start from zero
void clear_snap_max(efwi_plan *p, int k0, int k1, cudaStream_t st) {
    if (half_snaps(p) && k1 > k0)
        cudaMemsetAsync(efwi::snap_max(p, k0), 0, sizeof(float) * (size_t)(k1 - k0) * 2 * p->d.ns * kMaxPad, st);
}

// One forward step of every shot; d == nullptr skips the DAS sampling.
void forward_step(efwi_plan *p, int n, float *d, const SnapOut &so, cudaStream_t st) {
    if (p->d.exec == EFWI_EXEC_PLAIN) {
        Fields F = state_fields(p, 0);
        for (int s = 0; s < p->d.ns; ++s) {
            launch_vel_plain(p, s, so.fx, so.fz, st);
            launch_force(p, F, n, s, so.fx, so.fz, st);
            if (d) launch_das_fwd(p, F, n, d, s, st);
            launch_stress_plain(p, s, st);
            launch_inject(p, F, n, s, st);
        }
    } else {
        launch_step_fused(p, n, so, st);       // leaves v^{n+1/2}, sigma^{n+1} in state[scur]
        if (d) launch_das_fwd(p, state_fields(p, p->scur), n, d, -1, st);
    }
}

// Forward steps n0 .. n1-1 keeping every v^{n+1/2} in slots k0 + (n - n0) (with
// reduced-precision snapshots the last one is packed after the loop).
void forward_keep(efwi_plan *p, int n0, int n1, int k0, float *d, cudaStream_t st) {
    clear_snap_max(p, k0, k0 + (n1 - n0), st);
    for (int n = n0; n < n1; ++n) {
        const int k = k0 + (n - n0);
        forward_step(p, n, d, snap_out(p, k, n > n0 ? k - 1 : -1), st);
    }
    if (half_snaps(p) && n1 > n0) launch_snap_tail(p, snap_out(p, -1, k0 + (n1 - n0) - 1).sw, st);
}

void adjoint_step(efwi_plan *p, int n, const SnapIn &si, cudaStream_t st) {
    if (p->d.exec == EFWI_EXEC_PLAIN) {
        Fields A = adj_fields(p, 0);
        for (int s = 0; s < p->d.ns; ++s) {
            launch_das_adj(p, A, si, G_field(p, 3), G_field(p, 4), n, s, st);
            launch_adj_vel_plain(p, s, si.fx, si.fz, st);
            launch_adj_stress_plain(p, s, si.fx, si.fz, st);
        }
        p->apsi_v ^= 1;
    } else {
        launch_das_adj(p, adj_fields(p, p->acur), si, G_field(p, 3), G_field(p, 4), n, -1, st);
        launch_adj_fused(p, n, si, st);        // flips acur and the adjoint psi blocks
    }
}

}  // namespace

namespace efwi {

float *snap_max(efwi_plan *p, int slot) { return p->segmax + (size_t)slot * 2 * p->d.ns * kMaxPad; }

void *snap_half(efwi_plan *p, int slot) {
    return static_cast<char *>(p->segh) + (size_t)slot * 2 * p->fsz_total * 2;
}

SnapOut snap_out(efwi_plan *p, int slot, int prev) {
    SnapOut so;
    if (!half_snaps(p)) {
        if (slot >= 0) { so.fx = seg_x(p, slot); so.fz = seg_z(p, slot); }
        return so;
    }
    so.sw.F = p->fsz_total;
    so.sw.ns = p->d.ns;
    so.sw.kind = p->snap_store;
    if (slot >= 0) so.sw.amax = snap_max(p, slot);
    if (prev >= 0) { so.sw.h = snap_half(p, prev); so.sw.hmax = snap_max(p, prev); }
    return so;
}

SnapIn snap_in(efwi_plan *p, int slot) {
    SnapIn si;
    if (!half_snaps(p)) {
        si.fx = seg_x(p, slot);
        si.fz = seg_z(p, slot);
        return si;
    }
    si.sr.h = snap_half(p, slot);
    si.sr.hmax = snap_max(p, slot);
    si.sr.F = p->fsz_total;
    si.sr.ns = p->d.ns;
    si.sr.kind = p->snap_store;
    return si;
}

// Forward pass over all steps; when ck, keeps a checkpoint at the start of every
// segment that the adjoint recomputes and every v^{n+1/2}, n >= n_split, in the
// snapshot slots (all steps when the plan stores all of them).
void forward_loop(efwi_plan *p, float *d, bool ck, cudaStream_t st) {
    reset_forward_state(p, st);
    const int nt = p->d.nt;
    if (ck && p->K >= nt) {
        launch_ckpt_save(p, 0, st);
        forward_keep(p, 0, nt, 0, d, st);
        return;
    }
    const int n_keep = ck ? p->n_split : nt;
    for (int n = 0; n < n_keep; ++n) {
        if (ck && n % p->K == 0) launch_ckpt_save(p, n / p->K, st);
        forward_step(p, n, d, SnapOut{}, st);
    }
    if (n_keep < nt) forward_keep(p, n_keep, nt, p->K, d, st);
}

void adjoint_loop(efwi_plan *p, cudaStream_t st) {
    const long long F = p->fsz_total;
    for (int k = 0; k < 2; ++k)
        if (p->adj[k]) cudaMemsetAsync(p->adj[k], 0, sizeof(float) * 5 * F, st);
    cudaMemsetAsync(p->apsi, 0, sizeof(float) * 4 * p->H, st);
    cudaMemsetAsync(p->G, 0, sizeof(float) * 5 * F, st);
    if (p->Gtot) cudaMemsetAsync(p->Gtot, 0, sizeof(float) * 5 * F, st);
    if (p->Gcmp) cudaMemsetAsync(p->Gcmp, 0, sizeof(float) * 5 * F, st);
    if (p->d.ntr > 0) cudaMemsetAsync(p->tr_acc, 0, sizeof(double) * p->d.ntr, st);
    p->acur = 0;
    p->apsi_v = 0;
    p->apsi_s = 0;
    const int nt = p->d.nt, K = p->K;
    const bool full = K >= nt;
    const int nseg = (nt + K - 1) / K;
    if (!full && p->ov_fwd > 0 && p->seg_double && p->n_split >= nt) {
        // recompute of segment s-1 (stream sr) runs concurrently with the adjoint of
        // segment s (stream st); the two alternate between the segment-buffer halves
        cudaStream_t sr = p->cap2;
        cudaEvent_t *evR = &p->ovev[0], *evA = &p->ovev[nseg];
        cudaEvent_t fork = p->ovev[2 * nseg], join = p->ovev[2 * nseg + 1];
        cudaEventRecord(fork, st);
        cudaStreamWaitEvent(sr, fork);
        auto recompute = [&](int s) {
            if (s + 2 < nseg) cudaStreamWaitEvent(sr, evA[s + 2]);
            const int n0 = s * K, n1 = std::min(n0 + K, nt);
            launch_ckpt_load(p, s, sr);
            p->grid_fwd_override = p->ov_fwd * p->n_sms;
            forward_keep(p, n0, n1, seg_slot(p, s, 0), nullptr, sr);   // FP32 snapshots (the overlap needs them)
            p->grid_fwd_override = 0;
            cudaEventRecord(evR[s], sr);
        };
        recompute(nseg - 1);
        for (int sgi = nseg - 1; sgi >= 0; --sgi) {
            if (sgi > 0) recompute(sgi - 1);
            cudaStreamWaitEvent(st, evR[sgi]);
            const int n0 = sgi * K, n1 = std::min(n0 + K, nt);
            p->grid_adj_override = p->ov_adj * p->n_sms;
            for (int n = n1 - 1; n >= n0; --n) adjoint_step(p, n, snap_in(p, seg_slot(p, sgi, n - n0)), st);
            p->grid_adj_override = 0;
            if (p->Gtot) launch_kahan_fold(p, st);
            cudaEventRecord(evA[sgi], st);
        }
        cudaEventRecord(join, sr);
        cudaStreamWaitEvent(st, join);
        return;
    }
    // segments of K steps (recompute, then adjoint; the steps from n_split on were kept
    // by the forward pass); with every step stored, chunks of ceil(sqrt(nt)) steps, so
    // that the imaging sums are Kahan-folded as often
    const int KF = full ? std::min(nt, (int)std::ceil(std::sqrt((double)nt))) : K;
    for (int sgi = (nt + KF - 1) / KF - 1; sgi >= 0; --sgi) {
        const int n0 = sgi * KF, n1 = std::min(n0 + KF, nt);
        const bool kept = full || n0 >= p->n_split;     // n_split is a multiple of K
        if (!kept) {
            launch_ckpt_load(p, sgi, st);
            forward_keep(p, n0, n1, 0, nullptr, st);
        }
        for (int n = n1 - 1; n >= n0; --n)
            adjoint_step(p, n, snap_in(p, full ? n : kept ? K + (n - p->n_split) : n - n0), st);
        if (p->Gtot) launch_kahan_fold(p, st);
    }
}

// Capture body() once into gc (on the plan's capture stream), then replay it on st.
// When the caller's stream is itself being captured (a device-resident optimizer
// iteration that holds whole gradients in its graph), the loop is enqueued in place
// and becomes part of the caller's graph; a graph launch cannot be captured.
template <class Body>
int replay(efwi_plan *p, GraphCache &gc, cudaStream_t st, Body body) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(p, "stream capture query");
    }
    if (cs == cudaStreamCaptureStatusActive) {
        body(st);
        return cuda_status(p, "time loop inside a stream capture");
    }
    if (!gc.exec) {
        const long long l0 = p->launches;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return cuda_status(p, "begin graph capture");
        body(p->cap);
        if (cudaStreamEndCapture(p->cap, &g) != cudaSuccess || !g) return cuda_status(p, "end graph capture");
        cudaError_t e = cudaGraphInstantiate(&gc.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            gc.exec = nullptr;
            return cuda_status(p, "graph instantiate");
        }
        gc.launches = p->launches - l0;
        p->launches = l0;
    }
    if (cudaGraphLaunch(gc.exec, st) != cudaSuccess) return cuda_status(p, "graph launch");
    p->launches += gc.launches;
    return EFWI_OK;
}

int run_forward(efwi_plan *p, float *d, bool ck, cudaStream_t st) {
    Phase ph(ck ? "efwi forward with checkpoints" : "efwi forward");
    if (p->d.exec == EFWI_EXEC_BATCHED && p->use_graphs) {
        int rc = replay(p, ck ? p->g_fwd_ck : p->g_fwd, st,
                        [&](cudaStream_t cs) { forward_loop(p, p->dbuf, ck, cs); });
        if (rc) return rc;
        if (d && d != p->dbuf && p->d.ntr > 0)
            cudaMemcpyAsync(d, p->dbuf, sizeof(float) * (size_t)p->d.ntr * p->d.nt, cudaMemcpyDeviceToDevice, st);
    } else {
        forward_loop(p, d, ck, st);
    }
    return cuda_status(p, "forward time loop");
}

int run_adjoint(efwi_plan *p, cudaStream_t st) {
    Phase ph("efwi adjoint (checkpoint recompute, adjoint steps, imaging)");
    if (p->d.exec == EFWI_EXEC_BATCHED && p->use_graphs) {
        int rc = replay(p, p->g_adj, st, [&](cudaStream_t cs) { adjoint_loop(p, cs); });
        if (rc) return rc;
    } else {
        adjoint_loop(p, st);
    }
    return cuda_status(p, "adjoint time loop");
}

}  // namespace efwi

extern "C" int efwi_forward(efwi_plan *p, const float *vp, const float *vs, const float *rho, float *d_out,
                            efwi_stream_t stream) {
    if (!p) return EFWI_ERR_ARG;
    int rc = check_model_args(p, vp, vs, rho);
    if (rc) return rc;
    if (!d_out && p->d.ntr > 0) {
        p->err = "d_out must be a device pointer";
        return EFWI_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    p->launches = 0;
    launch_materials(p, vp, vs, rho, st);
    rc = run_forward(p, d_out, false, st);
    return rc;
}

extern "C" int efwi_adjoint_gradient(efwi_plan *p, const float *vp, const float *vs, const float *rho,
                                     const float *d_obs, double *phi_data, float *g_vp, float *g_vs, float *g_rho,
                                     const float *mask, float *d_out, efwi_stream_t stream) {
    if (!p) return EFWI_ERR_ARG;
    int rc = check_model_args(p, vp, vs, rho);
    if (rc) return rc;
    if ((!d_obs && p->d.ntr > 0) || !phi_data || !g_vp || !g_vs || !g_rho) {
        p->err = "d_obs, phi_data and gradient pointers must be device pointers";
        return EFWI_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    p->launches = 0;
    float *d = d_out ? d_out : p->dbuf;
    launch_materials(p, vp, vs, rho, st, 1);
    if ((rc = run_forward(p, d, true, st))) return rc;
    {
        Phase ph("efwi residual and misfit");
        if (p->d.ntr > 0) launch_residual(p, d, d_obs, phi_data, st);
        else cudaMemsetAsync(phi_data, 0, sizeof(double), st);
    }
    if ((rc = run_adjoint(p, st))) return rc;
    Phase ph("efwi chain rule");
    float *src = p->Gtot ? p->Gtot : p->G;
    // the scaled-stress adjoint's sums (A, B, C_s) to the stress form's (lambda, mu, mu_xz)
    if (p->adj_form == EFWI_ADJ_FORM_SCALED) launch_imag_unscale(p, src, st);
    const float *G[5];
    for (int k = 0; k < 5; ++k) G[k] = src + k * p->fsz_total;
    launch_chain_rule(p, vp, vs, rho, G, mask, g_vp, g_vs, g_rho, st);
    return cuda_status(p, "gradient epilogue");
}

extern "C" int efwi_pseudo_hessian(efwi_plan *p, const float *vp, const float *vs, const float *rho, double eps,
                                   float *h, float *h_inv, efwi_stream_t stream) {
    if (!p) return EFWI_ERR_ARG;
    int rc = check_model_args(p, vp, vs, rho);
    if (rc) return rc;
    if (!h) {
        p->err = "h must be a device pointer";
        return EFWI_ERR_ARG;
    }
    if (!(eps > 0.0 && eps <= 1.0)) {
        p->err = "eps must lie in (0, 1]";
        return EFWI_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    p->launches = 0;
    launch_materials(p, vp, vs, rho, st);
    // Kahan-compensated FP32 sum and its compensation with the wavefield layout,
    // over the first two fields of the imaging workspace G
    float *acc = p->G, *cmp = p->G + p->fsz_total;
    Phase ph("efwi pseudo-Hessian");
    auto body = [&](cudaStream_t cs) {
        reset_forward_state(p, cs);
        cudaMemsetAsync(acc, 0, sizeof(float) * 2 * p->fsz_total, cs);
        for (int n = 0; n < p->d.nt; ++n) {
            forward_step(p, n, nullptr, SnapOut{}, cs);
            launch_vel_energy(p, state_fields(p, p->d.exec == EFWI_EXEC_PLAIN ? 0 : p->scur), acc, cmp, cs);
        }
    };
    if (p->d.exec == EFWI_EXEC_BATCHED && p->use_graphs) {
        if ((rc = replay(p, p->g_ph, st, body))) return rc;
    } else {
        body(st);
    }
    launch_ph_finish(p, acc, cmp, eps, h, h_inv, st);
    return cuda_status(p, "pseudo-Hessian");
}

extern "C" int efwi_extended_objective(efwi_plan *p, const float *vp, const float *vs, const float *rho,
                                       const float *d_obs, const double eta[3], const float *b, const float *bp,
                                       const uint8_t *sink, double *phi_data, double *phi_reg,
                                       efwi_stream_t stream) {
    if (!p) return EFWI_ERR_ARG;
    int rc = check_model_args(p, vp, vs, rho);
    if (rc) return rc;
    if ((rc = resolve_zoi(p, p->d.ns, b, bp, sink))) return rc;
    if ((!d_obs && p->d.ntr > 0) || !eta || !phi_data || !phi_reg) {
        p->err = "NULL argument to efwi_extended_objective";
        return EFWI_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    p->launches = 0;
    launch_materials(p, vp, vs, rho, st);
    if ((rc = run_forward(p, p->dbuf, false, st))) return rc;
    if (p->d.ntr > 0) launch_residual(p, p->dbuf, d_obs, phi_data, st);
    else cudaMemsetAsync(phi_data, 0, sizeof(double), st);
    const float *ms[3] = {vp, vs, rho};
    for (int k = 0; k < 3; ++k) launch_reg(p, ms[k], b, bp, sink, eta[k], phi_reg, nullptr, k > 0, st);
    return cuda_status(p, "extended objective");
}
