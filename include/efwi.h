/*
 * efwi.h -- C ABI of the GB300 (sm_103a) library for source-extended elastic
 * full-waveform inversion with DAS data.
 *
 * The method (Bader, Clapp, Nihei, Biondi, "Source footprint elimination in
 * full-waveform inversion by model extension") extends the model along
 * sources, m~ = (m_1, ..., m_Ns), so that shot s is modelled with its own
 * component m_s, and regularises the components towards a common "useful"
 * model with the operator (I - S^T S_w) W:
 *
 *   phi_ext(m~) = 1/2 sum_s sum_r || d_{s,r}(m_s) - d_obs_{s,r} ||^2
 *               + 1/2 eta^2 || (I - S^T S_w) W m~ ||^2                  (eq. 8)
 *
 * This library computes, on one GPU, every quantity the inversion needs per
 * iteration: modelled DAS data (eqs. 1-3), the data misfit (eq. 4 / first
 * term of eq. 8) and its gradient with respect to every extended component
 * (eq. 6 applied to each m_s), the zone-of-influence weights (eq. 10) and the
 * consistency term with its gradient (eqs. 8, 11, 12); the collapse of the
 * extended model to the final model (eq. 9, and eq. 15 on gradients); the
 * pseudo-Hessian preconditioner of the paper's comparison method; and the
 * optimizer, l-BFGS with a strong-Wolfe line search and the convergence rate
 * of eq. 13.
 *
 * Physics (the paper fixes no scheme): 2D isotropic elastic velocity-stress
 * equations on a Virieux staggered grid, 4th order in space, 2nd order in
 * time, convolutional PML (Komatitsch & Martin 2007), moment-tensor or
 * vector-force sources, DAS gauge-averaged axial strain (or strain rate) or
 * 2-C particle-velocity receivers.  The gradient is the exact
 * discrete adjoint of the forward time stepping.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Row-major arrays, x fastest: a model component is [nz][nx]; an extended
 *    model is [ns][nz][nx]; data are [ntr][nt] (trace-major; the traces of
 *    shot s are tr_ptr[s] .. tr_ptr[s+1]-1).  Node (ix, iz) sits at
 *    (ix*dx, iz*dz) metres.
 *  - Arguments named "device" are device pointers owned by the caller,
 *    16-byte aligned, never freed or retained by the library.  Everything in
 *    efwi_plan_desc / efwi_zoi_desc is host memory, copied at the call.
 *  - Work is enqueued asynchronously on the caller's stream; scalar results
 *    (misfits) are written to device doubles.  No call synchronises the
 *    device except efwi_plan_create / efwi_plan_destroy.
 *  - Every call returns an int status: EFWI_OK (0) or a negative EFWI_ERR_*.
 *    Nothing throws across the ABI.  efwi_last_error() gives the message.
 *  - A plan is not thread-safe: calls on one plan must be serialised (they
 *    share its workspace).  Different plans are independent.
 */
#ifndef EFWI_H
#define EFWI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same underlying type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *efwi_stream_t;
typedef struct efwi_plan efwi_plan;

enum efwi_status {
    EFWI_OK = 0,
    EFWI_ERR_ARG = -1,              /* invalid argument (sizes, positions, NULL pointers) */
    EFWI_ERR_CFL = -2,              /* dt * vmax * sqrt(2) * (9/8 + 1/24) / min(dx, dz) >= 1 */
    EFWI_ERR_OOM = -3,              /* device allocation failed at plan creation */
    EFWI_ERR_CUDA = -4,             /* a CUDA runtime call or kernel launch failed */
    EFWI_ERR_TIMEOUT = -5,          /* a bounded device-side wait expired */
    EFWI_ERR_NAN = -6,              /* a model held a non-finite value or a non-positive density,
                                       or a gradient's model a zero shear modulus where the
                                       gradient divides by it (reported by efwi_sync_status) */
    EFWI_ERR_NOT_IMPLEMENTED = -7
};

/* receiver kind of every trace:
 *  STRAIN       DAS gauge-averaged axial strain t.(u(p+) - u(p-))/L, u the running
 *               time integral of the particle velocity at the gauge ends p+- = c +- (L/2) t
 *  STRAIN_RATE  the same with v instead of u
 *  VELOCITY     particle-velocity receiver (2-C geophones: one trace per component):
 *               t.v(c) at the channel point c; the gauge is not used                */
enum efwi_das_mode { EFWI_DAS_STRAIN = 0, EFWI_DAS_STRAIN_RATE = 1, EFWI_DAS_VELOCITY = 2 };
/* storage precision of the wavefield checkpoints and of the forward-velocity
 * snapshots (the time stepping is FP32).  FP16/BF16 store x as RNE(x 2^k) with
 * s 2^k in [2^14, 2^15), s = max |x| of the snapshot field and shot: per
 * element |x^ - x| <= 2^-11 |x| (FP16; every |x| >= s 2^-28) or 2^-8 |x| (BF16) */
enum efwi_store { EFWI_STORE_FP32 = 0, EFWI_STORE_FP16 = 1, EFWI_STORE_BF16 = 2 };
/* ckpt_interval value: store every step when the snapshots fit the device's
 * free memory at plan creation, else ceil(sqrt(nt)) with as many stored final
 * steps as fit (see stored_steps) */
#define EFWI_CKPT_AUTO (-1)
/* execution strategy:
 *  PLAIN   one shot per launch, one kernel per half-step, no graph, no tuning
 *  BATCHED all shots (any window sizes) in one fused launch per time step,
 *          the time loop captured and replayed as CUDA graphs               */
enum efwi_exec { EFWI_EXEC_PLAIN = 0, EFWI_EXEC_BATCHED = 1 };
/* tile staging of the batched forward and adjoint steps: per-thread loads, or
 * TMA bulk tensor copies into pipelined shared memory (persistent CTAs)     */
enum efwi_overlap { EFWI_OVERLAP_AUTO = 0, EFWI_OVERLAP_OFF = 1, EFWI_OVERLAP_ON = 2 };
enum efwi_stencil { EFWI_STENCIL_AUTO = 0, EFWI_STENCIL_LOADS = 1, EFWI_STENCIL_TMA = 2,
                    EFWI_STENCIL_TMA_PAIRS = 3 /* TMA, two adjacent cells per thread (forward step) */,
                    EFWI_STENCIL_TMA_STAGED = 4 /* TMA_PAIRS with the tile's outputs staged in shared
                                                   memory and written by bulk tensor stores (forward) */ };
/* the variable in which the batched adjoint step carries the adjoint stresses:
 *   STRESS  sigma^ itself (every staging and tile of the adjoint; EXEC_PLAIN always)
 *   SCALED  F = dt C sigma^ (C the cell's stiffness), which the transposed step only
 *           ever uses through C, so a step needs the stiffness on the tile alone and
 *           no pass over the 4-cell halo to form C sigma^ (per-thread loads or TMA
 *           staging; the imaging sums are converted back once per gradient).  Needs lambda + mu > 0
 *           (Vp > Vs) and mu > 0 on the physical cells and the half cells next to
 *           them; a gradient of a model without it is flagged (efwi_sync_status:
 *           EFWI_ERR_NAN).  Either form's chain rule needs mu > 0 on the physical
 *           cells, which every gradient call checks.
 *   AUTO    SCALED with EXEC_BATCHED unless adj_stencil asks for TMA_PAIRS or
 *           TMA_STAGED (stagings of the stress form only), else STRESS
 * The two forms agree up to FP32 rounding (not bit for bit); all tiles of one form
 * give bitwise-identical results.                                                */
enum efwi_adj_form { EFWI_ADJ_FORM_AUTO = 0, EFWI_ADJ_FORM_STRESS = 1, EFWI_ADJ_FORM_SCALED = 2 };

/*
 * Problem description (host memory; copied by efwi_plan_create).
 *
 *   nx, nz, dx, dz     physical grid (cells, metres)
 *   nt, dt             time steps and step (s); data sample n is taken after
 *                      the velocity update of step n, n = 0..nt-1
 *   npml               CPML thickness in cells; the grid is padded by npml+1
 *                      cells per side (the first padding node is undamped)
 *   pml_R, pml_vmax,   CPML reflection target, velocity and frequency used in
 *   pml_f0             d0 = -3 vmax ln R / (2 L) and alpha = pi f0 (1 - r);
 *                      pml_vmax <= 0 takes the maximum of ref_vp
 *   ns                 number of sources = number of extended components
 *   src_xz [ns][2]     source positions (m), inside the shot's window
 *   mt [ns][3]         moment tensor (Mxx, Mzz, Mxz) per source (eq. 2)
 *   wavelet [ns][nt+1] source time function w(t_n), t_n = n dt
 *   ntr, tr_ptr[ns+1]  traces, CSR over sources (the set N_r^s of eq. 4)
 *   ch_xz [ntr][2]     gauge centres / receiver points (m); ch_t [ntr][2] unit
 *                      tangents (DAS) or recorded components (VELOCITY)
 *   gauge              gauge length L (m): d = t.(u(p+) - u(p-)) / L,
 *                      p+- = centre +- (L/2) t, u the displacement (STRAIN)
 *                      or the particle velocity (STRAIN_RATE); unused for
 *                      VELOCITY receivers (d = t.v(centre))
 *   win [ns][2]        optional per-shot window (x0, width) in cells: shot s
 *                      is modelled on columns x0 .. x0+width-1 only (NULL =
 *                      the full grid for every shot)
 *   ref_vp/vs/rho      frozen reference model [nz][nx]; the absorbing padding
 *                      takes its edge values, so only physical cells are
 *                      inversion variables
 *   ckpt_interval      steps between wavefield checkpoints for the gradient:
 *                      0 = ceil(sqrt(nt)); >= nt = store every step (no recompute);
 *                      EFWI_CKPT_AUTO = every step if all nt snapshots (at
 *                      snap_store precision) fit in the free device memory
 *                      after the rest of the workspace, with 5 % + 2 GB left
 *                      over, else ceil(sqrt(nt)) with the largest stored_steps
 *                      that fits (stored_steps is then ignored; 0 when the
 *                      overlapped schedule is forced)
 *   ckpt_store         EFWI_STORE_* precision of the checkpoints
 *   exec               EFWI_EXEC_*
 *   tile_x, tile_z     stencil tile for EXEC_BATCHED (0, 0 = autotune at plan creation)
 *   stencil            EFWI_STENCIL_*: how EXEC_BATCHED stages a tile in shared
 *                      memory (AUTO lets the autotuner choose); every choice gives
 *                      bitwise-identical results
 *   adj_tile_x/_z,     the same two choices for the adjoint step (0, 0, AUTO =
 *   adj_stencil        autotune independently of the forward step)
 *   overlap            EFWI_OVERLAP_*: whether the checkpoint recompute of one
 *                      segment runs concurrently with the adjoint of the next
 *                      (EXEC_BATCHED with ckpt_interval < nt); results are the same
 *   force [ns][2]      optional vector-force sources (Fx, Fz) (eq. 2, second
 *                      case), replacing the moment tensors (mt is then ignored):
 *                      v^{n+1/2} += dt b F w(t_n) delta_h on the staggered v
 *                      grids (bilinear delta_h / (dx dz)); NULL = moment tensors
 *   snap_store         EFWI_STORE_* precision of the forward velocities
 *                      v^{n+1/2} kept for the imaging condition (every step with
 *                      full storage, the steps of one segment otherwise); FP16
 *                      and BF16 halve their memory and traffic and need
 *                      EXEC_BATCHED (and no forced overlap)
 *   stored_steps       with ckpt_interval K < nt: the forward pass also keeps the
 *                      velocities of the final stored_steps steps, rounded down so
 *                      that the steps before them form whole K-step segments; the
 *                      adjoint reads those directly and recomputes only the
 *                      segments before them from their checkpoints (no checkpoints
 *                      are taken inside the stored part).  0 = none (the whole
 *                      sqrt(nt) schedule); results equal those of stored_steps = 0
 *                      bit for bit with FP32 checkpoints (the imaging sums are
 *                      folded at the same segment ends).  Not combinable with a
 *                      forced overlapped schedule.
 *   adj_form           EFWI_ADJ_FORM_*: the adjoint step's stress variable (above)
 */
typedef struct efwi_plan_desc {
    int nx, nz;
    double dx, dz;
    int nt;
    double dt;
    int npml;
    double pml_R, pml_vmax, pml_f0;
    int ns;
    const double *src_xz;
    const double *mt;
    const float *wavelet;
    int ntr;
    const int *tr_ptr;
    const double *ch_xz;
    const double *ch_t;
    double gauge;
    int das_mode;
    const int *win;
    const float *ref_vp, *ref_vs, *ref_rho;
    int ckpt_interval;
    int ckpt_store;
    int exec;
    int tile_x, tile_z;
    int stencil;
    int adj_tile_x, adj_tile_z;
    int adj_stencil;
    int overlap;
    const double *force;
    int snap_store;
    int stored_steps;
    int adj_form;
} efwi_plan_desc;

/* What a plan chose and holds (filled by efwi_plan_info). */
typedef struct efwi_plan_info_t {
    int ckpt_interval;          /* steps per checkpoint segment */
    int n_ckpt;                 /* checkpoints per gradient */
    int tile_x, tile_z;         /* forward stencil tile in use (EXEC_BATCHED) */
    int adj_tile_x, adj_tile_z; /* adjoint stencil tile in use (EXEC_BATCHED) */
    int stencil;                /* EFWI_STENCIL_* used by the forward step */
    int stages;                 /* shared-memory pipeline depth of the TMA forward step */
    int adj_stencil;            /* EFWI_STENCIL_* used by the adjoint step */
    int adj_stages;             /* pipeline depth of the TMA adjoint step */
    int overlap_fwd_blocks;     /* persistent blocks per SM of the recompute step when it
                                   overlaps the adjoint (0: no overlap) */
    int overlap_adj_blocks;     /* and of the adjoint step */
    size_t workspace_bytes;     /* device bytes owned by the plan */
    long long padded_cells;     /* sum over shots of padded (nx_w + 2P)(nz + 2P) */
    long long physical_cells;   /* sum over shots of window width * nz */
    long long launches;         /* kernels launched by the last forward/gradient call */
    int layout;                 /* TMA forward step: cells per thread and shared-memory access
                                   (1, 2 = cell pairs, 3 = pairs on the tile and single cells
                                   on the velocity halo ring); 0 otherwise */
    int staged_stores;          /* TMA forward step writes its outputs by bulk tensor stores */
    int adj_persistent;         /* per-thread-load adjoint step runs on a persistent grid */
    int snap_store;             /* EFWI_STORE_* of the forward-velocity snapshots */
    int prefetch;               /* L2 prefetch one tile ahead: bit 0 forward step, bit 1 adjoint step */
    int stored_steps;           /* final steps whose velocities the forward pass keeps
                                   (nt with every step stored, 0 for the sqrt(nt) schedule) */
    int adj_form;               /* EFWI_ADJ_FORM_STRESS or _SCALED: the adjoint step in use */
    int adj_layout;             /* TMA scaled-stress adjoint: 1 = one cell per thread, 2 = cell
                                   pairs (64-bit shared-memory accesses), 3 = cell pairs in
                                   512-thread CTAs (tile pairs and halo ring on separate
                                   threads); 0 otherwise */
} efwi_plan_info_t;

/* Zone-of-influence description (eq. 10), host memory.  Per source s:
 *   active_x[s][2]  x-span (m) where the outer weight is 1
 *   taper[s]        outer taper width (m): r = distance outside the span / taper
 *   sink_xz[s][2]   sinkhole centre (m); sink_axes[s][2] ellipse semi-axes (m):
 *                   d_M = sqrt((dx/a_x)^2 + (dz/a_z)^2), r = 1 - d_M, inside iff d_M < 1
 *   n, nu           stiffness and height of the transition (0 < nu < 1)     */
typedef struct efwi_zoi_desc {
    const double *active_x;
    const double *taper;
    const double *sink_xz;
    const double *sink_axes;
    double n, nu;
} efwi_zoi_desc;

/* Create a plan: validates the description (positions inside windows, CFL),
 * precomputes CPML profiles, interpolation weights and tile lists, allocates
 * the workspace and, for EXEC_BATCHED with tile 0x0, runs the tile autotuner.
 * Synchronises the device.  Errors: EFWI_ERR_ARG, EFWI_ERR_CFL, EFWI_ERR_OOM,
 * EFWI_ERR_CUDA (*out is then NULL; the message is in efwi_last_error(NULL)).
 * Environment variables read here (all optional; no effect on results, which
 * are bitwise the same for every variant of one adjoint form):
 *   EFWI_TMA_STAGES=n     the autotuner keeps only n-stage TMA forward variants
 *   EFWI_TMA_VEC=v        only forward layout v (1 single cells, 2 cell pairs,
 *                         3 cell pairs with the halo ring as single cells)
 *   EFWI_ADJ_PERSIST=0|1  only the one-CTA-per-tile / persistent-grid adjoint
 *   EFWI_ADJ_VEC=1|2|3    only the single-cell / cell-pair / 512-thread cell-pair TMA
 *                         scaled-stress adjoint
 *   EFWI_PREFETCH=0|1     L2 prefetch one tile ahead off / on (else timed)
 *   EFWI_AUTOTUNE_LOG=1   print every timed variant on stderr
 *   EFWI_TEST_FAIL_ALLOC=k  make the k-th workspace allocation fail with
 *                         EFWI_ERR_OOM (tests of the clean-up path)        */
int efwi_plan_create(efwi_plan **out, const efwi_plan_desc *desc);

/* Free a plan and its workspace (synchronises the device).  NULL is allowed. */
int efwi_plan_destroy(efwi_plan *plan);

/* Last error message of a plan, or of the calling thread when plan is NULL. */
const char *efwi_last_error(const efwi_plan *plan);

int efwi_plan_info(const efwi_plan *plan, efwi_plan_info_t *info);

/* Bind a plan to another acquisition of the same shape: the next group of
 * shots of an extended problem whose sources do not fit one plan (each
 * component is independent through eqs. 1-6, so a group is a slice of the
 * problem).  Source positions, moment tensors or forces, wavelets and
 * receiver positions and tangents are taken from desc; the grid, time axis,
 * CPML, reference model, checkpoint schedule, windows and traces per shot
 * must equal the plan's (EFWI_ERR_ARG otherwise, the plan unchanged).  No
 * workspace is re-allocated and the tile autotuner does not run again; the
 * captured time loops are kept when the adjoint-source gather keeps its
 * shape, else they are captured again on the next call.  The uploads are
 * enqueued on stream after the caller's earlier work there; calls of the
 * plan on other streams must have completed.                               */
int efwi_plan_rebind(efwi_plan *plan, const efwi_plan_desc *desc, efwi_stream_t stream);

/* Synchronise the stream and report device-side failures of earlier calls on
 * this plan: EFWI_ERR_TIMEOUT if a kernel gave up a bounded wait (its results
 * are then invalid), EFWI_ERR_NAN if a model passed to a call held a
 * non-finite velocity or density or a non-positive density (checked on every
 * cell the call's materials read) or, in a gradient call, mu <= 0 (or, with
 * the scaled-stress adjoint, lambda + mu <= 0) where the gradient divides by
 * it (efwi_adj_form), EFWI_ERR_CUDA for an asynchronous CUDA
 * error.  The device flag is cleared.                                        */
int efwi_sync_status(efwi_plan *plan, efwi_stream_t stream);

/* Forward modelling of every shot with its own component (eqs. 1-3; first
 * term of eq. 8).
 *   vp, vs, rho  device [ns][nz][nx] FP32 extended model (Vs > 0 everywhere)
 *   d_out        device [ntr][nt] FP32, overwritten with the DAS data       */
int efwi_forward(efwi_plan *plan, const float *vp, const float *vs, const float *rho,
                 float *d_out, efwi_stream_t stream);

/* Data misfit and its gradient with respect to every extended component
 * (eq. 4 and eq. 6 applied to each m_s, by the adjoint-state method: exact
 * discrete adjoint of the forward time stepping, zero-lag cross-correlation
 * of forward and adjoint wavefields).
 *   d_obs              device [ntr][nt] FP32 observed data
 *   phi_data           device double: 1/2 sum (d - d_obs)^2 (FP64 reduction)
 *   g_vp, g_vs, g_rho  device [ns][nz][nx] FP32, overwritten; zero outside a
 *                      shot's window
 *   mask               device [nz][nx] FP32 multiplier of every gradient, or NULL
 *   d_out              device [ntr][nt] FP32 modelled data, or NULL          */
int efwi_adjoint_gradient(efwi_plan *plan, const float *vp, const float *vs, const float *rho,
                          const float *d_obs, double *phi_data, float *g_vp, float *g_vs,
                          float *g_rho, const float *mask, float *d_out, efwi_stream_t stream);

/* Zone-of-influence weights of every source (eq. 10): b_s, b'_s (= 1 inside
 * the sinkhole of s, b_s outside; eq. 12) and the sinkhole flag.
 *   b, bp  device [ns][nz][nx] FP32; sink device [ns][nz][nx] uint8          */
int efwi_zoi_weights(int ns, int nx, int nz, double dx, double dz, const efwi_zoi_desc *zoi,
                     float *b, float *bp, uint8_t *sink, efwi_stream_t stream);

/* Zone-of-influence weights held by the plan: efwi_zoi_weights of the plan's
 * ns sources on its grid, computed on the device into plan-owned arrays
 * (allocated by the first call, which synchronises the device).  Afterwards
 * efwi_regularization_grad, efwi_regularization_grad_n (with the plan's ns)
 * and efwi_extended_objective take NULL b, bp, sink to mean these weights.
 * Errors as efwi_zoi_weights, EFWI_ERR_OOM.                                 */
int efwi_plan_set_zoi(efwi_plan *plan, const efwi_zoi_desc *zoi, efwi_stream_t stream);

/* Consistency term of eq. 8 for one parameter field and its gradient:
 *   phi_reg = 1/2 eta^2 || (I - S^T S_w) W m~ ||^2,
 *   g      += eta^2 W^T (I - S^T S_w)^T (I - S^T S_w) W m~
 * with W of eq. 11 and S_w of eq. 12, per pixel over the ns components.  The
 * residual (I - S^T S_w) W m~ and its norm are FP64; the gradient increment is
 * FP64 at pixels where some component has its sinkhole and FP32 elsewhere.
 *   m, b, bp   device [ns][nz][nx] FP32; sink device [ns][nz][nx] uint8;
 *              b, bp, sink all NULL: the plan's weights (efwi_plan_set_zoi)
 *   phi_reg    device double (overwritten; FP64 reduction)
 *   g          device [ns][nz][nx] FP32, accumulated into (+=)             */
int efwi_regularization_grad(efwi_plan *plan, const float *m, const float *b, const float *bp,
                             const uint8_t *sink, double eta, double *phi_reg, float *g,
                             efwi_stream_t stream);

/* efwi_regularization_grad over ns components instead of the plan's shots
 * (m, b, bp, sink: device [ns][nz][nx] on the plan's grid).  The plan lends
 * only its grid and reduction scratch, so a plan made for one group of shots
 * evaluates the consistency term (eqs. 8, 11, 12) of every component when the
 * extended problem runs in shot groups that do not fit one plan together.
 * EFWI_ERR_ARG for ns < 1; the rest as efwi_regularization_grad.            */
int efwi_regularization_grad_n(efwi_plan *plan, int ns, const float *m, const float *b, const float *bp,
                               const uint8_t *sink, double eta, double *phi_reg, float *g,
                               efwi_stream_t stream);

/* Allocation-free variant of efwi_regularization_grad (no counterpart in the
 * paper; it exists for callers that cannot let a library allocate device
 * memory, e.g. applications that own all device memory through their own
 * pool or budget, and for callers that want the regularization without
 * creating a plan, whose creation allocates the whole workspace).  Same
 * arguments and results as efwi_regularization_grad but no plan: ns, nx, nz
 * give the sizes of the [ns][nz][nx] arrays.  It calls no cudaMalloc or
 * cudaFree.  Its only scratch (FP64 block partials of phi_reg) is a static
 * 32 KB device array that every GPU loading the library holds until exit.
 * Every call made outside a stream capture looks up that array's address on
 * the current device; a call inside a capture reuses the address found by
 * the last uncaptured call on that device, so call it once before any
 * capture (a captured first call returns EFWI_ERR_CUDA).  A cudaDeviceReset
 * may move the array: later uncaptured calls find it again, graphs captured
 * before the reset must not be replayed.  Limit: nx * nz <= 1048576 pixels,
 * larger sizes return EFWI_ERR_ARG without launching anything.  All calls
 * share the array, so calls that overlap on the GPU race on it.             */
int efwi_regularization_grad_noalloc(int ns, int nx, int nz, const float *m, const float *b,
                                     const float *bp, const uint8_t *sink, double eta,
                                     double *phi_reg, float *g, efwi_stream_t stream);

/* Collapse of an extended field to one physical field, out = S_w W x~
 * (eq. 9: the final model from the extended model; the same operator applied
 * to the per-source gradients is the preconditioned gradient of eq. 15).
 * W of eq. 11 and S_w of eq. 12 act per pixel over the ns components, in FP64.
 *   x, b, bp   device [ns][nz][nx] FP32; sink device [ns][nz][nx] uint8
 *   out        device [nz][nx] FP32 (overwritten)
 * No plan and no workspace; EFWI_ERR_ARG on sizes < 1 or NULL pointers.     */
int efwi_collapse(int ns, int nx, int nz, const float *x, const float *b, const float *bp,
                  const uint8_t *sink, float *out, efwi_stream_t stream);

/* Pseudo-Hessian of the paper's illumination-compensation comparison method
 * (pseudo-Hessian = diagonal of the approximate Hessian, the preconditioning
 * paragraph; built, as the comparison section describes, by auto-correlating
 * the absolute particle velocity in time, summing over shots, clipping and
 * scaling, and given to l-BFGS as the initial inverse Hessian):
 *   h(x)    = sum_s sum_n |v_s(x, t_{n+1/2})|^2   (zero lag, no dt factor),
 *   h_inv(x) = c / max(h(x), c),  c = eps * max_x h   (1 everywhere if h = 0),
 * with |v|^2 at a node from the mean of the two staggered neighbours of each
 * velocity component.  Shot s runs in its own component of the extended
 * model (vp, vs, rho: device [ns][nz][nx]) and contributes inside its window.
 *   eps     clipping level, 0 < eps <= 1 (EFWI_ERR_ARG otherwise)
 *   h       device [nz][nx] FP32 (overwritten); accumulated over time in
 *           Kahan-compensated FP32 per shot, summed over shots in FP64
 *   h_inv   device [nz][nx] FP32 (overwritten), or NULL
 * Runs one forward pass of every shot (no DAS sampling); uses the plan's
 * imaging workspace, so it must not overlap an efwi_adjoint_gradient call
 * of the same plan on the GPU.                                              */
int efwi_pseudo_hessian(efwi_plan *plan, const float *vp, const float *vs, const float *rho, double eps,
                        float *h, float *h_inv, efwi_stream_t stream);

/* ---- Optimizer: limited-memory BFGS with a strong-Wolfe line search -------
 * The paper's inversions run l-BFGS with a step length satisfying the Wolfe
 * conditions and stop when the convergence rate of eq. 13,
 *   rate_{k+1} = (Phi_k - Phi_{k+1}) / Phi_k,
 * drops below a threshold (0.1 %) or when no suitable step is found.
 * A handle owns m pairs (s_i, y_i) of n-element FP32 device vectors plus
 * scratch (about (2m + 5) n floats).  Directions come from the two-loop
 * recursion with H_0 = (s^T y / y^T y) I of the newest pair (I without pairs),
 * or a caller's diagonal guess (efwi_lbfgs_set_h0); inner products are FP64
 * reductions in a fixed order.  The line search (bracketing, then zoom with
 * safeguarded quadratic interpolation) starts at step 1 (1 / ||d|| on the
 * first iteration, d = -H_0 g) and evaluates the objective
 * through the caller's callback:
 *   fn(ctx, x, phi, g, stream): x device [n] (read only), phi HOST double
 *   (written), g device [n] (written); returns 0, or nonzero to abort (a
 *   negative value is passed on as the status).
 * A trial point whose objective or slope is not finite (a step so long that
 * the modelling becomes unstable) counts as failing sufficient decrease: it
 * bounds the bracket from above and the zoom bisects towards shorter steps.
 * A pair is stored only when s^T y > 0.                                     */
typedef struct efwi_lbfgs efwi_lbfgs;
typedef int (*efwi_objective_fn)(void *ctx, const float *x, double *phi, float *g, efwi_stream_t stream);

enum efwi_lbfgs_stop {
    EFWI_LBFGS_STOP_MAX_ITER = 0,  /* max_iter iterations done */
    EFWI_LBFGS_STOP_RATE = 1,      /* rate of eq. 13 below min_rate */
    EFWI_LBFGS_STOP_NO_STEP = 2    /* the line search found no step within max_ls evaluations */
};

typedef struct efwi_lbfgs_info_t {
    double phi;          /* objective after the iteration(s) */
    double phi_prev;     /* objective before the last iteration */
    double rate;         /* eq. 13 of the last iteration */
    double alpha;        /* accepted step length of the last iteration */
    int evals;           /* objective evaluations */
    int iters;           /* iterations done (efwi_lbfgs_run) */
    int pairs;           /* stored (s, y) pairs */
    int ls_failed;       /* 1: no step found (x, g and phi unchanged) */
    int stop;            /* EFWI_LBFGS_STOP_* (efwi_lbfgs_run) */
} efwi_lbfgs_info_t;

/* n vector length, m stored pairs (1..64), 0 < c1 < c2 < 1 (sufficient
 * decrease and curvature constants, e.g. 1e-4 and 0.9), max_ls objective
 * evaluations per line search.  Errors: EFWI_ERR_ARG, EFWI_ERR_OOM.         */
int efwi_lbfgs_create(efwi_lbfgs **out, long long n, int m, double c1, double c2, int max_ls);
int efwi_lbfgs_destroy(efwi_lbfgs *h);
/* Forgets the stored pairs (and the graph of efwi_lbfgs_iterate_device). */
int efwi_lbfgs_reset(efwi_lbfgs *h);
/* Length of the first trial step of an iteration without stored pairs (the
 * first iteration, or after a restart): the trial moves x by len along d
 * (a = len / ||d||).  len = 0, the default, keeps a = min(1, 1 / ||d||).
 * A model in physical units (m/s, kg/m^3) wants a length of the order of
 * the change it should see, e.g. 1e-3 ||x||.  EFWI_ERR_ARG for len < 0.     */
int efwi_lbfgs_set_step0(efwi_lbfgs *h, double len);
/* Stores the pair (s, y) (device [n] each, copied) if s^T y > 0; *accepted
 * (may be NULL) tells whether it was.  Synchronises the stream.             */
int efwi_lbfgs_push(efwi_lbfgs *h, const float *s, const float *y, int *accepted, efwi_stream_t stream);
/* Positive diagonal D (device [n], copied) as the initial inverse Hessian:
 * H_0 = gamma D with gamma = s^T y / y^T D y of the newest pair, H_0 = D
 * without pairs (the paper gives l-BFGS the clipped, scaled inverse
 * pseudo-Hessian of efwi_pseudo_hessian this way).  NULL returns to
 * H_0 = gamma I.  Forgets the stored pairs.                                 */
int efwi_lbfgs_set_h0(efwi_lbfgs *h, const float *diag, efwi_stream_t stream);
/* Saves the history (to resume an inversion later; the paper has no
 * counterpart): *pairs receives the number of stored pairs; when S_out and
 * Y_out (device [pairs][n] each) are given, the pairs are copied there,
 * oldest first (asynchronous).  Restoring is efwi_lbfgs_reset followed by
 * efwi_lbfgs_push of each pair in the same order, which recomputes their
 * scalars with the same reductions, so directions are bit-identical; a
 * diagonal H_0 is set again with efwi_lbfgs_set_h0 before the pushes.       */
int efwi_lbfgs_export(efwi_lbfgs *h, int *pairs, float *S_out, float *Y_out, efwi_stream_t stream);
/* d = -H g (device [n] each) from the stored pairs, asynchronous.          */
int efwi_lbfgs_direction(efwi_lbfgs *h, const float *g, float *d, efwi_stream_t stream);
/* One iteration from x (device [n], updated), *phi (host, updated) and its
 * gradient g (device [n], updated): direction, line search, new pair.  The
 * history restarts from -g when d is not a descent direction.  When no step
 * is found info->ls_failed = 1 and x, phi, g are unchanged.                */
int efwi_lbfgs_iterate(efwi_lbfgs *h, float *x, double *phi, float *g, efwi_objective_fn fn, void *ctx,
                       efwi_lbfgs_info_t *info, efwi_stream_t stream);
/* Evaluates fn at x, then iterates until max_iter iterations, a rate of
 * eq. 13 below min_rate (0.001 in the paper) or a failed line search.
 * x and g (device [n]) hold the final model and its gradient.              */
int efwi_lbfgs_run(efwi_lbfgs *h, float *x, float *g, efwi_objective_fn fn, void *ctx, int max_iter,
                   double min_rate, efwi_lbfgs_info_t *info, efwi_stream_t stream);

/* One efwi_lbfgs_iterate whose strong-Wolfe line search runs on the device
 * (no counterpart in the paper, which gives the optimizer, not where it runs):
 * the bracketing and zoom of efwi_lbfgs_iterate -- the same steps, c1, c2,
 * max_ls and quadratic interpolation, in FP64 -- are a one-thread state
 * machine in device memory, and one CUDA graph repeats, in a conditional
 * while-node, trial point x + a d, objective, phi' = g^T d and search step
 * until a step is accepted or max_ls evaluations are spent: no host
 * synchronisation inside the search.  The direction (with its reads of g^T d
 * and, on a first step, d^T d) precedes the graph; one read of the search
 * state and the pair update of efwi_lbfgs_iterate follow it.
 *   phi  device double: the objective at x on entry, updated
 *   fn(ctx, x, phi, g, stream) enqueues the objective at x (device [n]) into
 *        phi (DEVICE double) and g (device [n]) on stream; it is called only
 *        while the graph is captured (the first call for this fn, ctx, x, phi,
 *        g; later calls replay the graph), so it must enqueue stream-
 *        capturable work only (kernels, device copies and memsets: no
 *        synchronisation, no allocation, no host copies) and return 0.
 *        The graph holds the device arrays the objective used: after any of
 *        them moves (a plan destroyed or re-allocated, e.g. by
 *        efwi_plan_rebind to another gather shape or efwi_prof_enable),
 *        efwi_lbfgs_reset drops it so that the next call captures it again.
 * efwi_groups_objective_fn is such an objective (the extended problem in
 * shot groups).                                                             */
typedef int (*efwi_device_objective_fn)(void *ctx, const float *x, double *phi, float *g, efwi_stream_t stream);
int efwi_lbfgs_iterate_device(efwi_lbfgs *h, float *x, double *phi, float *g, efwi_device_objective_fn fn,
                              void *ctx, efwi_lbfgs_info_t *info, efwi_stream_t stream);

/* ---- Shot groups held on the device ---------------------------------------
 * An extended problem with ngroups x ns sources (ns = the plan's) runs as
 * groups of the plan's shape (each component is independent through eqs.
 * 1-6).  A group set keeps every group's source and receiver weights, adjoint
 * gather, wavelet increments and tile flags in device memory, so that binding
 * the plan to group k (efwi_groups_bind) is device-to-device copies, which a
 * stream capture records (efwi_plan_rebind uploads from the host instead).
 * Every group must have the plan's shape (efwi_plan_rebind's rules) and give
 * the plan's adjoint-gather shape (the same receiver geometry); the plan must
 * use EXEC_BATCHED.  No counterpart in the paper.                          */
typedef struct efwi_groups efwi_groups;
int efwi_groups_create(efwi_groups **out, efwi_plan *plan, const efwi_plan_desc *groups, int ngroups);
int efwi_groups_destroy(efwi_groups *groups);
int efwi_groups_bind(efwi_groups *groups, int k, efwi_stream_t stream);
/* The extended objective of eq. 8 over all ngroups x ns components and its
 * gradient, enqueued on stream (stream-capturable): for every group, bind
 * and efwi_adjoint_gradient; then efwi_regularization_grad_n of Vp, Vs, rho
 * with eta[3]; phi = the groups' misfits + the three consistency terms,
 * summed in that order on the device.
 *   x, grad   device [3][ngroups*ns][nz][nx] (Vp, Vs, rho of every component)
 *   d_obs     device [ngroups][ntr][nt]
 *   b, bp, sink  device [ngroups*ns][nz][nx] (or NULL when ngroups == 1 and
 *             the plan holds its weights)
 *   phi       device double                                                 */
int efwi_groups_objective(efwi_groups *groups, const float *x, const float *d_obs, const double eta[3],
                          const float *b, const float *bp, const uint8_t *sink, double *phi, float *grad,
                          efwi_stream_t stream);
/* efwi_groups_objective as an efwi_device_objective_fn: ctx points to an
 * efwi_groups_objective_ctx (host memory that outlives the graphs using it). */
typedef struct efwi_groups_objective_ctx {
    efwi_groups *groups;
    const float *d_obs;
    double eta[3];
    const float *b, *bp;
    const uint8_t *sink;
} efwi_groups_objective_ctx;
int efwi_groups_objective_fn(void *ctx, const float *x, double *phi, float *g, efwi_stream_t stream);

/* Extended objective of eq. 8: phi_data (as efwi_forward + misfit) and
 * phi_reg summed over the three parameter fields (Vp, Vs, rho) with their
 * own eta[3].  Both results are device doubles (overwritten).  b, bp, sink
 * as in efwi_regularization_grad (all NULL: the plan's weights).            */
int efwi_extended_objective(efwi_plan *plan, const float *vp, const float *vs, const float *rho,
                            const float *d_obs, const double eta[3], const float *b,
                            const float *bp, const uint8_t *sink, double *phi_data,
                            double *phi_reg, efwi_stream_t stream);

/* Self-test of the failure path of bounded device waits (no counterpart in
 * the paper): launches one thread that waits, with the same bounded wait as
 * the TMA kernels, on a barrier that never completes, and gives up after
 * budget_cycles clock cycles (1 .. 2^32; 2^21 is about a millisecond).  The
 * next efwi_sync_status on the plan then returns EFWI_ERR_TIMEOUT and clears
 * the flag.  Nothing faults, traps or hangs.                                */
int efwi_selftest_timeout(efwi_plan *plan, long long budget_cycles, efwi_stream_t stream);

/* Numerics self-tests (no counterpart in the paper): the device routines that
 * the time loops use for reduced-precision snapshots and for the Kahan fold
 * of the imaging sums, applied to caller arrays so that tests can check them
 * against FP64 arithmetic and the stated error bounds.
 *
 * efwi_selftest_store: treats x (device [n] FP32) as one snapshot field,
 *   writes s = max |x| to s_out (device float), encodes x into enc (device
 *   [n] elements of 2 bytes) as checkpoints and stored forward velocities
 *   are encoded -- RNE(x 2^k) with s 2^k in [2^14, 2^15) -- and decodes enc
 *   into y (device [n] FP32).  Per element |y - x| <= 2^-11 |x| (FP16) or
 *   2^-8 |x| (BF16) where x 2^k is a normal number of the format, and
 *   <= 2^-25 2^-k (FP16) below that.  store = EFWI_STORE_FP32 copies x
 *   (enc unused).
 * efwi_selftest_kahan: folds the nterms arrays terms[k] (device
 *   [nterms][n] FP32, consumed: zeroed) one after another into tot (device
 *   [n] FP32) with Kahan (1965) compensation cmp (device [n] FP32); tot and
 *   cmp start from zero.                                                    */
int efwi_selftest_store(int store, long long n, const float *x, void *enc, float *y, float *s_out,
                        efwi_stream_t stream);
int efwi_selftest_kahan(long long n, int nterms, float *terms, float *tot, float *cmp, efwi_stream_t stream);

/* Kernel timing for measurements.  When every > 0 the plan brackets every
 * every-th launch of its two dominant stencil kernels with CUDA events on the
 * launching stream (inside the captured graphs too, where each replay
 * re-records them).  efwi_prof_read synchronises the events of one kernel
 * (EFWI_KERNEL_STEP: the forward time step; EFWI_KERNEL_ADJ: the adjoint time
 * step) and returns their summed elapsed milliseconds and the number of timed
 * launches.  efwi_prof_enable drops the cached graphs.                     */
enum efwi_kernel { EFWI_KERNEL_STEP = 0, EFWI_KERNEL_ADJ = 1 };
int efwi_prof_enable(efwi_plan *plan, int every);
int efwi_prof_read(efwi_plan *plan, int kernel, double *total_ms, long long *count);

#ifdef __cplusplus
}
#endif
#endif /* EFWI_H */
