// Host-side plan object and the launchers each translation unit exports.
#pragma once

#include <string>
#include <vector>

#include "efwi_common.cuh"

namespace efwi {

struct FwdMaps;   // tensor maps of one shot (tma.cuh)
struct AdjMaps;
struct AdjsMaps;

// Adjoint-source gather (the transpose of the DAS sampling): for every grid
// cell touched by any gauge end, the list of (trace, weight) contributions,
// summed in a fixed order so the result is deterministic.
struct GatherCSR {
    int n_tgt = 0;
    int *tgt_shot = nullptr;     // [n_tgt]
    int *tgt_field = nullptr;    // [n_tgt] 0 = vx, 1 = vz
    int *tgt_off = nullptr;      // [n_tgt] offset within the shot block
    int *ptr = nullptr;          // [n_tgt + 1]
    int *tr = nullptr;           // [nnz] global trace index
    float *w = nullptr;          // [nnz] bilinear weight * (+-t_k) / L
};

// What a forward step hands to the adjoint besides the state: the FP32 copy of
// its v^{n+1/2} (fx, fz: segment-buffer slots) or, with a reduced-precision
// snapshot store, the snapshot work of SnapW; and what an adjoint step reads.
struct SnapOut {
    float *fx = nullptr, *fz = nullptr;
    SnapW sw{};
};
struct SnapIn {
    const float *fx = nullptr, *fz = nullptr;
    SnapR sr{};
};

// An instantiated CUDA graph of a time loop and the kernels it launches.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
};

struct TileList {
    int n = 0;
    int tx = 0, tz = 0;          // tile shape
    int4 *tiles = nullptr;       // (shot, i0, j0, unused)
};

// Checkpoint of the forward state (wavefields + CPML memory) in FP32 or
// per-snapshot, per-field scaled FP16 / BF16.
struct CkptStore {
    int store = EFWI_STORE_FP32;
    int n = 0;                   // number of checkpoints
    void *fields = nullptr;      // n x 5 x fsz_total elements (float / half / bf16)
    float *psi = nullptr;        // n x 2H floats (V and S blocks, always FP32)
    float *scale = nullptr;      // n x 5 x ns per-field scales (reduced precision only)
};

}  // namespace efwi

struct efwi_plan {
    efwi_plan_desc d;                       // scalars only (pointers cleared)
    int P = 0;
    std::vector<efwi::ShotDev> shots;
    efwi::ShotDev *shots_d = nullptr;
    long long fsz_total = 0;               // floats per field kind, all shots
    long long psx_total = 0, psz_total = 0;
    long long H = 0;                       // 2 * psx_total + 2 * psz_total (one psi block)
    long long padded_cells = 0, physical_cells = 0;
    int prof_x_total = 0;
    int max_nx = 0, nzp = 0;
    std::vector<int> trace_shot;

    // device buffers
    // Wavefields: two buffers of 5 * fsz_total (vx, vz, sxx, szz, sxz).  The plain
    // path updates buffer 0 in place; the batched path reads buffer scur and writes
    // the other one (a tile reads halos that neighbouring tiles overwrite).
    float *state[2] = {nullptr, nullptr};
    int scur = 0;
    float *mat = nullptr;                  // 5 * fsz_total (lambda, mu, mu_xz, b_x, b_z)
    float *adj[2] = {nullptr, nullptr};    // adjoint wavefields, same scheme
    int acur = 0;
    float *G = nullptr;                    // 5 * fsz_total (per-segment or direct accumulators)
    float *Gtot = nullptr, *Gcmp = nullptr;// Kahan totals and compensation (batched)
    // CPML memory, 4 blocks of H = 2 psx_total + 2 psz_total floats:
    //   [V0 | V1 | S0 | S1], V = (psi1, psi3 | psi2, psi4) of the velocity sub-step,
    //   S = (psi5, psi8 | psi6, psi7) of the stress sub-step; x-strip arrays first.
    float *psi = nullptr;
    int psi_v = 0, psi_s = 0;              // current V and S blocks
    float *apsi = nullptr;                 // adjoint CPML memory, same layout
    int apsi_v = 0, apsi_s = 0;
    float *prof = nullptr;                 // 4 * prof_x_total + 4 * nzp
    float *dw = nullptr;                   // [ns][nt] (w_{n+1} - w_n)
    float *wv = nullptr;                   // [ns][nt] w_n / (dx dz), force sources only
    bool has_force = false;
    float *ref = nullptr;                  // [3][nz][nx] reference model
    int *tr_shot = nullptr;                // [ntr]
    int *tr_off = nullptr;                 // [ntr][16] offsets within shot block
    float *tr_w = nullptr;                 // [ntr][16] weights * (+-t) / L
    double *tr_acc = nullptr;              // [ntr] running strain (fwd) / reverse residual sum (adj)
    float *tr_coef = nullptr;              // [ntr] adjoint-source coefficient of the current step
    efwi::GatherCSR gather;
    std::vector<int> gather_ptr;           // [ns+1] per-shot range of gather targets
    int gather_nnz = 0;                    // (trace, weight) entries of the gather
    efwi::TileList tiles;                  // forward fused-step work items
    efwi::TileList adj_tiles;              // adjoint fused-step work items
    float *resid = nullptr;                // [ntr][nt]
    float *dbuf = nullptr;                 // [ntr][nt]
    double *partial = nullptr;             // reduction scratch
    // Snapshot slots, one per kept step v^{n+1/2} (x and z planes): slots 0 .. K-1 hold the
    // segment being recomputed (two such halves with the overlapped schedule), slots
    // K + (n - n_split) the steps n >= n_split that the forward pass keeps; with every
    // step stored (K >= nt) slot n is step n.
    float *seg = nullptr;                  // FP32 snapshots: nslots x 2 x fsz_total
    int snap_store = EFWI_STORE_FP32;      // precision of the stored forward velocities
    void *segh = nullptr;                  // FP16/BF16 snapshots: nslots x 2 x fsz_total elements of 2 bytes
    float *segmax = nullptr;               // their maxima: nslots x [2][ns][kMaxPad] floats
    int nslots = 0;                        // snapshot slots allocated
    int n_split = 0;                       // first step the forward pass keeps (0 with K >= nt, nt for none)
    efwi::CkptStore ck;
    float *zoi_b = nullptr, *zoi_bp = nullptr;   // zone-of-influence weights held by the plan (efwi_plan_set_zoi)
    uint8_t *zoi_sink = nullptr;
    int K = 0;                             // checkpoint interval
    int tile_x = 0, tile_z = 0;            // forward tile
    int stencil = EFWI_STENCIL_LOADS;      // staging of the forward step (after tuning)
    efwi::FwdMaps *fwd_maps = nullptr;     // [ns] tensor maps for EFWI_STENCIL_TMA
    int tma_grid = 0;                      // persistent CTAs of the TMA forward step
    int tma_stages = 2;                    // shared-memory pipeline depth of the TMA forward step
    int tma_vec = 1;                       // cells per thread and shared-memory access (1 or 2)
    int tma_store = 0;                     // forward outputs staged in shared memory, bulk-stored
    int tma_pf = 0;                        // forward step: L2 prefetch of the tile beyond the pipeline
    int adj_pf = 0;                        // per-thread-load adjoint: L2 prefetch of the CTA's next tile
    int adj_stencil = EFWI_STENCIL_LOADS;  // staging of the adjoint step (after tuning)
    int adj_form = EFWI_ADJ_FORM_STRESS;   // adjoint stress variable in use (EFWI_ADJ_FORM_STRESS / _SCALED)
    efwi::AdjMaps *adj_maps = nullptr;
    efwi::AdjsMaps *adjs_maps = nullptr;   // [ns] tensor maps of the TMA scaled-stress adjoint
    int adjs_vec = 1;                      // its layout: 1 = one cell per thread, 2 = cell pairs,
                                           // 3 = cell pairs in 512-thread CTAs
    int tma_adj_grid = 0, tma_adj_stages = 1;
    int adj_grid = 0;                      // per-thread-load adjoint: persistent grid (0 = one CTA per tile)
    int *dev_err = nullptr;                // device flag: a bounded wait expired
    bool broken = false;                   // a real bounded wait expired: the plan is not used again
    int adj_tile_x = 0, adj_tile_z = 0;    // adjoint tile
    size_t bytes = 0;
    long long launches = 0;

    // batched path: time loops captured once and replayed
    cudaStream_t cap = nullptr;            // capture stream (never executes work)
    cudaStream_t cap2 = nullptr;           // second capture stream (recompute branch)
    std::vector<cudaEvent_t> ovev;         // dependency events of the overlapped schedule
    int n_sms = 0;
    // recompute of segment k-1 overlapped with the adjoint of segment k: persistent
    // blocks per SM of the forward and adjoint step kernels (0: run one after the other)
    int ov_fwd = 0, ov_adj = 0;
    int grid_fwd_override = 0, grid_adj_override = 0;   // launch grids in effect (0 = default)
    bool seg_double = false;               // segment buffer holds two halves (overlap)
    efwi::GraphCache g_fwd, g_fwd_ck, g_adj, g_ph;
    bool use_graphs = true;

    // timing of the dominant kernels (event pairs, tagged by kernel kind)
    int prof_every = 0;
    long long prof_counter[2] = {0, 0};
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    int ev_used = 0;

    std::string err;
};

namespace efwi {

constexpr int kPartials = 1024;            // blocks of the FP64 reductions

// --- k_misc.cu ---------------------------------------------------------------
// gradient = 1: the call images (the shear-modulus check of the chain rule and the adjoint applies)
void launch_materials(efwi_plan *p, const float *vp, const float *vs, const float *rho, cudaStream_t st,
                      int gradient = 0);
void launch_inject(efwi_plan *p, Fields F, int n, int shot /* -1 = all */, cudaStream_t st);
void launch_force(efwi_plan *p, Fields F, int n, int shot, float *segx, float *segz, cudaStream_t st);
void launch_das_fwd(efwi_plan *p, Fields F, int n, float *d, int shot, cudaStream_t st);
void launch_das_adj(efwi_plan *p, Fields A, const SnapIn &si, float *Gbx, float *Gbz, int n, int shot,
                    cudaStream_t st);
// packs v of state buffer scur (the last step of a pass) into the snapshot slot sw.h with maxima sw.hmax
void launch_snap_tail(efwi_plan *p, const SnapW &sw, cudaStream_t st);
void launch_residual(efwi_plan *p, const float *d, const float *dobs, double *phi, cudaStream_t st);
void launch_chain_rule(efwi_plan *p, const float *vp, const float *vs, const float *rho, const float *const *G,
                       const float *mask, float *gvp, float *gvs, float *grho, cudaStream_t st);
void launch_kahan_fold(efwi_plan *p, cudaStream_t st);
void launch_ckpt_save(efwi_plan *p, int slot, cudaStream_t st);
void launch_ckpt_load(efwi_plan *p, int slot, cudaStream_t st);
int launch_zoi(int ns, int nx, int nz, double dx, double dz, const efwi_zoi_desc *z, float *b, float *bp,
               uint8_t *sink, cudaStream_t st, std::string &err);
void launch_collapse(int ns, long long npix, const float *x, const float *b, const float *bp, const uint8_t *sink,
                     float *out, cudaStream_t st);
// ns > 0: the arrays hold ns components (default: the plan's shots)
void launch_reg(efwi_plan *p, const float *m, const float *b, const float *bp, const uint8_t *sink, double eta,
                double *phi, float *g, int accumulate_phi, cudaStream_t st, int ns = 0);

// --- k_hessian.cu --------------------------------------------------------------
void launch_vel_energy(efwi_plan *p, Fields F, float *sum, float *cmp, cudaStream_t st);
void launch_ph_finish(efwi_plan *p, const float *sum, const float *cmp, double eps, float *h, float *hinv,
                      cudaStream_t st);

// --- k_plain.cu (shot >= 0: that shot only; shot < 0: all shots in one launch) ---
void launch_vel_plain(efwi_plan *p, int shot, float *segx, float *segz, cudaStream_t st);
void launch_stress_plain(efwi_plan *p, int shot, cudaStream_t st);
void launch_adj_vel_plain(efwi_plan *p, int shot, const float *vfx, const float *vfz, cudaStream_t st);
void launch_adj_stress_plain(efwi_plan *p, int shot, const float *vfx, const float *vfz, cudaStream_t st);

// --- k_tma.cu ----------------------------------------------------------------
bool tma_shape_ok(int tx, int tz, int nst, int vec, int st, int snap);
int tma_prepare_fwd(efwi_plan *p, int tx, int tz, int nst, int vec, int st);
void launch_step_tma(efwi_plan *p, int n, const SnapOut &so, cudaStream_t st);
bool tma_adj_shape_ok(int tx, int tz, int nst);
int tma_prepare_adj(efwi_plan *p, int tx, int tz, int nst);
int tma_encode_adj_maps(efwi_plan *p, int tx, int tz);
void launch_adj_tma(efwi_plan *p, const float *vfx, cudaStream_t st);

// --- k_adjs.cu (adjoint step in scaled-stress form) ----------------------------
bool adj_scaled_shape_ok(int tx, int tz);
void adj_scaled_set_attrs();
int adj_scaled_blocks_per_sm(int tx, int tz, int snap_store);
void launch_adj_scaled(efwi_plan *p, const SnapIn &si, cudaStream_t st);
// G: the plan's 5 imaging fields; converts the first three in place to the stress form's sums
void launch_imag_unscale(efwi_plan *p, float *G, cudaStream_t st);
// --- k_adjs_tma.cu (the same step with TMA staging, FP32 forward velocities) ----
bool adj_scaled_tma_shape_ok(int tx, int tz);
// tensor maps and grid; vec 1 (single cells), 2 (cell pairs), 3 (cell pairs, 512-thread CTAs)
int adj_scaled_tma_prepare(efwi_plan *p, int tx, int tz, int vec);
void launch_adj_scaled_tma(efwi_plan *p, const SnapIn &si, cudaStream_t st);

// --- k_fused.cu --------------------------------------------------------------
void launch_step_fused(efwi_plan *p, int n, const SnapOut &so, cudaStream_t st);
void launch_adj_fused(efwi_plan *p, int n, const SnapIn &si, cudaStream_t st);
int upload_tiles(efwi_plan *p, TileList &tl, int tx, int tz);
// the work items of tile list tl (same shape and order) with the flags of another acquisition
std::vector<int4> tiles_of(const std::vector<ShotDev> &shots, const TileList &tl);
int refresh_tiles(efwi_plan *p, TileList &tl, cudaStream_t st);

// snapshot slots (engine.cu): slot >= 0 this step's slot, prev >= 0 the previous
// step's slot whose reduced-precision copy the step writes (-1: none)
SnapOut snap_out(efwi_plan *p, int slot, int prev);
SnapIn snap_in(efwi_plan *p, int slot);
float *snap_max(efwi_plan *p, int slot);
void *snap_half(efwi_plan *p, int slot);

// Host-side precompute of an acquisition on a plan's shot geometry (plan.cu): source
// injection weights (eq. 2), receiver interpolation weights (eq. 3), the deterministic
// gather of the adjoint source and the wavelet increments.
struct AcqHost {
    std::vector<ShotDev> shots;            // geometry of the plan + the source fields of this acquisition
    std::vector<int> trace_shot;
    std::vector<int> h_off;                // [ntr][16]
    std::vector<float> h_w;
    std::vector<int> g_shot, g_field, g_off, g_ptr, g_tr;
    std::vector<float> g_w;
    std::vector<int> gather_ptr;           // [ns + 1]
    std::vector<float> h_dw, h_wv;
    bool has_force = false;
};
int build_acq(const efwi_plan_desc &d, const std::vector<ShotDev> &geom, AcqHost &h, std::string &err);
// the same checks as efwi_plan_rebind: desc has the plan's shape (grid, time axis, windows, traces)
int check_same_shape(efwi_plan *p, const efwi_plan_desc *d, std::string &err);

// helpers (plan.cu)
// b, bp, sink all given, or all NULL for the plan's own weights (EFWI_ERR_ARG otherwise)
int resolve_zoi(efwi_plan *p, int ns, const float *&b, const float *&bp, const uint8_t *&sink);
void set_thread_error(const std::string &msg);  // message for efwi_last_error(NULL)
Fields state_fields(efwi_plan *p, int which);   // which: 0/1 buffer
Fields adj_fields(efwi_plan *p, int which);
Mat materials(efwi_plan *p);
Pml fwd_pml(efwi_plan *p, int vblk, int sblk);  // profiles + psi blocks
Pml adj_pml(efwi_plan *p, int vblk, int sblk);
float *psi_block(float *base, efwi_plan *p, int blk);  // blk 0,1 = V0,V1; 2,3 = S0,S1
float *G_field(efwi_plan *p, int k);      // k: 0 lam, 1 mu, 2 muxz, 3 bx, 4 bz
void prof_begin(efwi_plan *p, cudaStream_t st, int *slot, int kind);
void prof_end(efwi_plan *p, cudaStream_t st, int slot);

}  // namespace efwi
