/*
 * bh.h - C ABI of libbh, the GB300 (sm_103a) hot path of borehole acoustic
 * full-waveform inversion (Tang, Cheng, Li, Fang, "Borehole acoustic
 * full-waveform inversion").
 *
 * The calls follow the five steps of one inversion iteration (Method
 * section, Fig. 1): forward modelling, data residual, adjoint modelling,
 * gradient, model update.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Grid.  Cell (i, j), 0 <= i < nr, 0 <= j < nz, sits at r = (i + 1/2) dr,
 *   z = j dz and carries the normal stresses and lambda, mu, rho.  v_r sits
 *   at (i dr, j dz), v_z at ((i + 1/2) dr, (j + 1/2) dz), tau_rz at
 *   (i dr, (j + 1/2) dz).  v_r and tau_rz vanish on the axis (i = 0).
 *   Space is 4th order (staggered), time 2nd order (leapfrog).  A C-PML
 *   absorbs at the outer radial edge and at the top and bottom of every
 *   shot window; the axis is a symmetry line.
 * - Model arrays are row-major [nr][nz_global] float32, z contiguous.
 * - Every pointer argument is owned by the caller.  Pointers are DEVICE
 *   pointers unless a comment says "host".  libbh owns everything it
 *   allocates (wavefields, C-PML memories, forward history, accumulators)
 *   and frees it in bh_model_destroy.
 * - All device work is enqueued on the CUDA stream given to
 *   bh_model_create, in call order.  A call returns once its work is
 *   enqueued, except where it writes a host scalar (J, alpha): those calls
 *   synchronise the stream before returning.
 * - Every call returns a bh_status; nothing aborts or exits.  On error the
 *   model keeps its previous state where possible and bh_last_error()
 *   describes the failure.
 * - One model must not be used from two host threads at once.
 */
#ifndef BH_H
#define BH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BH_OK = 0,
    BH_ERR_INVALID_ARG = 1, /* NULL pointer, bad size, index out of range   */
    BH_ERR_CFL = 2,         /* dt violates the 4th-order staggered limit    */
    BH_ERR_OOM = 3,         /* device allocation failed or exceeds the cap  */
    BH_ERR_CUDA = 4,        /* a CUDA runtime call failed                   */
    BH_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired           */
    BH_ERR_STATE = 6,       /* calls made in the wrong order                */
    BH_ERR_UNSUPPORTED = 7  /* option not available in this build           */
} bh_status;

typedef struct bh_model bh_model; /* opaque, owned by libbh */

typedef struct {
    int nr;              /* radial cells, outer C-PML included                 */
    int nz;              /* axial cells of the global model (== nz_global)     */
    int nt;              /* time steps per shot                                */
    int npml_r;          /* C-PML cells at the outer radial edge               */
    int npml_z;          /* C-PML cells at the top and at the bottom of a window */
    double dr, dz, dt;   /* m, m, s                                            */
    double f0;           /* Hz; sets the C-PML frequency shift pi f0           */
    double pml_R;        /* target C-PML reflection; <= 0 means 1e-3           */
    int snapshot_precision;      /* checkpoint snapshots: 0 fp32, 1 bf16, 2 fp16, each
                                    plane with its own power-of-two scale        */
    size_t checkpoint_cap_bytes; /* 0: store v_r, v_z of every step; > 0: byte cap
                                    of the history window plus the checkpoints   */
} bh_grid_desc;

typedef struct {
    int z_offset;        /* first global row of the shot's window              */
    int nz;              /* window length in cells (its own top/bottom C-PML)  */
    int src_ir, src_iz;  /* source cell, window coordinates                    */
    int nrec;            /* receivers of this shot                             */
    const int* rec_iz;   /* host [nrec]: receiver cells (i = 0, on the axis)   */
} bh_shot_desc;

/*
 * Build a model: Lame parameters from velocities (Eq. 3, Eq. 4), buoyancy
 * at the velocity nodes, harmonic-mean mu at the shear-stress nodes,
 * C-PML profiles, shot descriptors, and the forward-history store.
 *   grid      host; grid->nz must equal nz_global
 *   vp, vs, rho  device [nr][nz_global] float32 (vs = 0 marks fluid)
 *   shots     host [nshots]; every window must lie inside the model, every
 *             source and receiver inside the window's interior
 *   stream    cudaStream_t (NULL = legacy default stream)
 *   out       host; receives the new model
 * Errors: BH_ERR_INVALID_ARG (bad sizes or indices), BH_ERR_CFL when
 *   dt Vmax sqrt(1/dr^2 + 1/dz^2) (9/8 + 1/24) >= 1, BH_ERR_OOM, BH_ERR_CUDA.
 * Citation: Method section, Eq. 2-4; C-PML and axis conditions as cited
 *   there (finite differences; absorbing layers at the two axial ends and the
 *   outer radius).
 */
bh_status bh_model_create(const bh_grid_desc* grid, int nz_global, const float* vp,
                          const float* vs, const float* rho, const bh_shot_desc* shots,
                          int nshots, void* stream, bh_model** out);

/* Free every device buffer of the model.  NULL is accepted. */
void bh_model_destroy(bh_model* model);

/*
 * Replace the model (velocities and density) without rebuilding the shot
 * plan; invalidates any stored forward history.
 *   vp, vs, rho  device [nr][nz_global] float32
 * Errors: BH_ERR_INVALID_ARG, BH_ERR_CFL.
 */
bh_status bh_set_model(bh_model* model, const float* vp, const float* vs, const float* rho);

/*
 * Shots run together, in groups of up to 32: every kernel launch (or every
 * phase of a cooperative launch) covers the tiles of one group's shots, each
 * shot on its own window state.
 *
 * Forward history.  The adjoint correlation needs v^{n+1/2} of every step.
 * With checkpoint_cap_bytes = 0 every step is stored (nt + 1 slots of v_r,
 * v_z per shot).  With a cap, the history of the last steps (the tail) is
 * stored by the forward sweep itself, and the steps before it are cut into
 * segments of L steps: a binomial (Griewank-Walther) checkpoint schedule
 * over the segments keeps at most s full forward states per shot, and each
 * segment is re-run once into an (L + 1)-slot history window before its
 * adjoint; L, s and the tail are the plan that fits the cap with the fewest
 * recomputed steps (bh_plan_history).  With FP32
 * snapshots the results are bit-identical to storing every step.  With
 * snapshot_precision 1 (BF16) or 2 (FP16) a snapshot takes half the bytes;
 * every plane (each wavefield and each C-PML memory of each shot) is stored
 * as x / s, s a power of two from the plane's max |x|, so the restored
 * trajectory differs from the stored one by the 16-bit rounding and the
 * gradient by the resulting error (the seismograms and J are unaffected:
 * they come from the first, unrounded sweep).
 */

/*
 * Forward modelling (Eq. 2) of every shot: leapfrog steps of the velocity
 * and stress equations; the source rate wavelet[n] (sampled at
 * t = (n + 1/2) dt) is injected as dt * wavelet[n] / V into the three
 * normal stresses of the source cell (V the cell volume); the pressure is
 * recorded as the mean normal stress at the receivers (the Method section
 * records normal stresses at the receiver positions).  Keeps the forward history
 * needed by bh_adjoint_gradient.
 *   wavelet  device [nt] float32; with checkpointing it is read again by
 *            the next bh_adjoint_gradient, so it must stay valid until then
 *   seis     device [nshots][nrec_max][nt] float32, row n = after step n;
 *            entries of receivers a shot does not have are set to 0
 * Errors: BH_ERR_INVALID_ARG, BH_ERR_CUDA.
 */
bh_status bh_forward(bh_model* model, const float* wavelet, float* seis);

/*
 * Data residual Delta p = p_mod - p_mes (Eq. 5) and misfit
 * J = 1/2 ||Delta p||^2 (Eq. 1), summed in FP64 in a fixed order.
 *   seis_mod, seis_obs  device [nshots][nrec_max][nt] float32
 *   resid    device, same shape, float32 (may alias seis_mod)
 *   J        host double; the call synchronises the stream
 * Errors: BH_ERR_INVALID_ARG, BH_ERR_CUDA.
 */
bh_status bh_residual_misfit(bh_model* model, const float* seis_mod, const float* seis_obs,
                             float* resid, double* J);

/*
 * Adjoint modelling driven by the residual (Eq. 6, as the exact transpose
 * of the discrete forward step) and the zero-lag correlations of Eq. 7
 * (lambda) and Eq. 8 (mu), plus the density term through the buoyancy.
 * The gradients of every shot are added, in FP64, into the global model
 * arrays; cells inside the C-PML (radial, and the top/bottom layers of
 * every window that covers them) receive nothing.  Also accumulates the
 * diagonal pseudo-Hessian used by bh_precondition.
 *   resid    device [nshots][nrec_max][nt] float32 (the adjoint source)
 *   g_lam, g_mu  device [nr][nz_global] double, OVERWRITTEN
 *   g_rho    device [nr][nz_global] double or NULL
 * Errors: BH_ERR_STATE without a preceding bh_forward on the same model,
 *   BH_ERR_INVALID_ARG, BH_ERR_CUDA.
 */
bh_status bh_adjoint_gradient(bh_model* model, const float* resid, double* g_lam,
                              double* g_mu, double* g_rho);

/*
 * Copy the pseudo-Hessian diagonals accumulated by the last
 * bh_adjoint_gradient:  H_lam = sum dt (div v)^2,
 * H_mu = sum dt [ (2 e_rr)^2 + (2 e_tt)^2 + (2 e_zz)^2 ] plus a quarter of
 * sum dt (dv_r/dz + dv_z/dr)^2 from each of the cell's four shear nodes.
 *   H_lam, H_mu  device [nr][nz_global] double
 * Errors: BH_ERR_STATE, BH_ERR_INVALID_ARG.
 */
bh_status bh_get_hessian(bh_model* model, double* H_lam, double* H_mu);

/*
 * Diagonal preconditioner (Numerical Examples, Fig. 6: weights the
 * gradient to suppress the borehole guided-wave imprint near the wall; the
 * paper prints no formula): g <- g / (H + eps_rel * max H), with H the
 * pseudo-Hessian of the same parameter and max over the inversion mask;
 * g <- 0 outside the mask (fluid cells and C-PML cells).
 *   g_lam, g_mu  device [nr][nz_global] double, in place
 * Errors: BH_ERR_STATE without a preceding bh_adjoint_gradient,
 *   BH_ERR_INVALID_ARG (eps_rel < 0), BH_ERR_CUDA.
 */
bh_status bh_precondition(bh_model* model, double* g_lam, double* g_mu, double eps_rel);

/*
 * Gradient-descent update (Eq. 9, Eq. 10) with alpha chosen per parameter
 * so that no cell changes by more than kappa times the largest modulus
 * (the Method section has alpha set the largest change of the model):
 * alpha_m = kappa max|m| / max|g_m| over the inversion mask; then mu >= 0,
 * lambda + 2 mu >= rho (1 m/s)^2, and Vp, Vs from Eq. 11, Eq. 12 in the
 * updated cells; cells outside the mask keep the Vp, Vs the model was given
 * bit for bit.  The model's own coefficients are rebuilt; any stored
 * history is invalidated.
 *   g_lam, g_mu  device [nr][nz_global] double
 *   alpha_out    host double[2] (alpha_lambda, alpha_mu) or NULL; when
 *                given, the call synchronises the stream
 *   vp_out, vs_out  device [nr][nz_global] float32 or NULL
 * Errors: BH_ERR_INVALID_ARG (kappa < 0), BH_ERR_CUDA.
 */
bh_status bh_update(bh_model* model, const double* g_lam, const double* g_mu, double kappa,
                    double* alpha_out, float* vp_out, float* vs_out);

/*
 * Gradients with respect to the velocities and density of the current
 * model, by the chain rule through Eq. 3 and Eq. 4:
 * g_Vp = 2 rho Vp g_lambda, g_Vs = 2 rho Vs (g_mu - 2 g_lambda),
 * g_rho|Vp,Vs = g_rho + (Vp^2 - 2 Vs^2) g_lambda + Vs^2 g_mu.
 *   g_lam, g_mu  device [nr][nz_global] double (from bh_adjoint_gradient)
 *   g_rho    device double or NULL (density held fixed)
 *   g_vp, g_vs, g_rho_v  device [nr][nz_global] float32, each may be NULL
 * Errors: BH_ERR_INVALID_ARG, BH_ERR_CUDA.
 */
bh_status bh_velocity_gradient(bh_model* model, const double* g_lam, const double* g_mu,
                               const double* g_rho, float* g_vp, float* g_vs, float* g_rho_v);

/*
 * Gradient-descent update in the velocities, and optionally the density,
 * instead of the Lame parameters (Eq. 9, Eq. 10 applied to Vp, Vs, rho; the
 * Method section derives Vp, Vs from lambda, mu by Eq. 11, Eq. 12 and takes
 * rho from density logs, so stepping rho is optional).  The gradients with
 * respect to (Vp, Vs, rho) follow from g_lam, g_mu, g_rho by the chain rule
 * of bh_velocity_gradient, in FP64; each parameter m steps by
 * alpha_m = kappa max|m| / max|g_m| over the inversion mask; then
 * Vs >= 0, Vp >= 1 m/s, rho >= 1 kg/m^3, and lambda, mu follow from Eq. 3,
 * Eq. 4.  Cells outside the mask keep their values bit for bit.  The
 * model's own coefficients are rebuilt; any stored history is invalidated.
 *   g_lam, g_mu  device [nr][nz_global] double (raw or preconditioned)
 *   g_rho    device [nr][nz_global] double or NULL (no density gradient)
 *   update_rho  0: rho is held fixed; 1: rho steps too
 *   alpha_out   host double[3] (alpha_Vp, alpha_Vs, alpha_rho) or NULL;
 *               when given, the call synchronises the stream
 *   vp_out, vs_out, rho_out  device [nr][nz_global] float32 or NULL
 * Errors: BH_ERR_INVALID_ARG (kappa < 0, update_rho not 0 or 1), BH_ERR_CUDA.
 */
bh_status bh_update_velocity(bh_model* model, const double* g_lam, const double* g_mu,
                             const double* g_rho, int update_rho, double kappa,
                             double* alpha_out, float* vp_out, float* vs_out, float* rho_out);

/* Current model velocities: those given to bh_model_create / bh_set_model,
 * as the updates left them.  vp, vs: device [nr][nz_global] float32. */
bh_status bh_get_model(bh_model* model, float* vp, float* vs);

/* Current model density.  rho: device [nr][nz_global] float32. */
bh_status bh_get_density(bh_model* model, float* rho);

/*
 * Sampled kernel timing (tracing aid; the paper has no counterpart).  With
 * every > 0, CUDA events bracket the launches of every every-th time step
 * of the stepping kernels on the model's stream; every = 0 turns it off.
 * bh_profile_read synchronises the stream and returns, for one kernel, the
 * summed event time in ms and the number of sampled launches since the last
 * bh_profile_reset.  Kernel ids: BH_KERNEL_*.
 * Errors: BH_ERR_INVALID_ARG, BH_ERR_CUDA.
 */
enum {
    BH_KERNEL_FWD_VEL = 0,     /* velocity half-step, Eq. 2 lines 1-2          */
    BH_KERNEL_FWD_STRESS = 1,  /* stress half-step, Eq. 2 lines 3-6            */
    BH_KERNEL_ADJ_STRESS = 2,  /* transposed stress step + Eq. 7 / Eq. 8        */
    BH_KERNEL_ADJ_VEL = 3,     /* transposed velocity step                     */
    BH_KERNEL_FWD_PERSIST = 4, /* cooperative forward: all steps of a run       */
    BH_KERNEL_ADJ_PERSIST = 5, /* cooperative adjoint + correlation of a run    */
    BH_KERNEL_FWD_STEP = 6,    /* one whole forward step of a shot group with
                                  fused interior steps ("split" 3)          */
    BH_KERNEL_COUNT = 7
};
bh_status bh_profile_enable(bh_model* model, int every);
bh_status bh_profile_read(bh_model* model, int kernel, double* total_ms, long* launches);
bh_status bh_profile_reset(bh_model* model);

/*
 * Residual and misfit without any device allocation (the paper has no
 * counterpart; this is a service for callers that may not allocate device
 * memory: processes whose device memory is owned by another allocator or
 * fixed at start-up, and serving paths that forbid allocation, which can
 * synchronise the device, after warm-up).  Computes
 * exactly what bh_residual_misfit computes, Delta p = p_mod - p_mes and
 * J = 1/2 ||Delta p||^2 in FP64, but needs no bh_model: its scratch is a
 * fixed 64 KB array inside the library, present on every GPU that loads
 * the library until the process exits.
 *   seis_mod, seis_obs  device float32 [n]
 *   resid    device float32 [n] (may alias seis_mod)
 *   n        number of samples, at most BH_NOALLOC_MAX_SAMPLES
 *   J        host double; the call synchronises `stream`
 *   stream   cudaStream_t (NULL = legacy default stream)
 * The first call on a device looks up the scratch address on that device
 * (cudaGetSymbolAddress) and keeps it for the life of the process.  A
 * device reset (cudaDeviceReset)
 * after the first call is not supported: the kept address would be stale.
 * All calls share the one scratch array: calls whose work overlaps on the
 * GPU (unordered streams) race and may return a wrong J.
 * Errors: BH_ERR_INVALID_ARG (NULL pointer, n > BH_NOALLOC_MAX_SAMPLES),
 *   BH_ERR_CUDA; bh_last_error(NULL) gives the message.
 */
#define BH_NOALLOC_MAX_SAMPLES 33554432 /* 8192 blocks x 4096 samples */
bh_status bh_residual_misfit_noalloc(const float* seis_mod, const float* seis_obs,
                                     float* resid, size_t n, double* J, void* stream);

/*
 * Execution options (the paper has no counterpart).
 *   "persistent"      1: one cooperative launch runs every time step of a
 *                     shot group, with a bounded grid barrier between half
 *                     steps; 0: one kernel launch per half-step; 2 (default
 *                     where the device supports cooperative launch): 1 for a
 *                     group whose tiles fit the co-resident blocks (one tile
 *                     per block), else 0.  All give bit-identical results.
 *   "tile_code"       forward tile code: 0 (default) one code path that reads
 *                     each tile's C-PML flag, 1 one instantiation per tile
 *                     class (interior tiles without any layer state).  The
 *                     two differ in how the compiler contracts multiply-adds
 *                     (results agree to rounding, not bit for bit).
 *   "split"           0 (default) one launch per half-step covers every tile
 *                     of a shot group; 1: one launch per half-step and tile
 *                     class (interior tiles, C-PML tiles), so that interior
 *                     tiles run more blocks per SM; applies to the adjoint
 *                     and, with "tile_code" 1, to the forward; 2: as 1,
 *                     and with "tile_code" 1 the forward's interior tiles
 *                     run in pipelined kernels (a grid of a few blocks per
 *                     SM, each block copying its next tile while it
 *                     computes the current one).  0, 1 and 2 give bit for
 *                     bit the same results.  BH_ERR_UNSUPPORTED for 2 when
 *                     the pipelined kernels do not fit an SM.  3: as 1,
 *                     and with "tile_code" 1 every forward step of the
 *                     interior tiles is one launch (both half-steps of a
 *                     tile in one block, velocities recomputed on the
 *                     stress stencil's halo); the six forward fields then
 *                     alternate between two buffers (always allocated: 6
 *                     planes per shot).  Its velocity arithmetic is the
 *                     same expressions compiled in another kernel, so
 *                     results agree with 1 to rounding (multiply-add
 *                     contraction), and bit for bit across shot
 *                     groupings.  4: as 3, with the fused step's tiles
 *                     staged by TMA box copies (cp.async.bulk.tensor on
 *                     tensor maps of the field buffers and coefficient
 *                     copies, one issuing thread, a bounded mbarrier wait);
 *                     the same results as 3.  BH_ERR_UNSUPPORTED for 4 when
 *                     the tensor maps could not be encoded; a copy that
 *                     does not complete makes bh_forward /
 *                     bh_adjoint_gradient return BH_ERR_TIMEOUT.
 *   "pipe_grid"       cap on the blocks of a pipelined launch (default 0:
 *                     as many as fit the SMs); a small cap makes every
 *                     block walk many tiles (a test knob).
 *   "tile_order"      order of the tiles within a launch: 0 (default) by
 *                     global column, then row, then shot; 1 by shot, then
 *                     row, then column.  The same results bit for bit.
 *   "group"           shots per launch group, 1 .. min(32, nshots) (default
 *                     the largest): one launch, or one cooperative phase,
 *                     covers the tiles of a group's shots; groups run one
 *                     after the other over a run's steps.  Invalidates any
 *                     stored forward history.  All values give bit-identical
 *                     results.
 *   "barrier_timeout_ms"  wall-clock limit of one barrier wait (default
 *                     2000).  A wait that runs out sets a device error flag,
 *                     every block returns, and bh_forward /
 *                     bh_adjoint_gradient return BH_ERR_TIMEOUT; the CUDA
 *                     context stays usable.
 *   "barrier_extra_arrivals"  test knob: the barrier waits for this many
 *                     arrivals beyond the blocks launched, so every wait
 *                     runs out (default 0).
 * With cooperative launches bh_forward and bh_adjoint_gradient synchronise
 * the stream once per launch to read the barrier status.
 * Errors: BH_ERR_INVALID_ARG (unknown key, value out of range),
 *   BH_ERR_UNSUPPORTED (persistent mode without cooperative launch).
 */
bh_status bh_set_option(bh_model* model, const char* key, double value);

/*
 * Autotuner of the stepping kernels' launch configuration (the paper has no
 * counterpart).  The candidates are both forward tile codes ("tile_code"),
 * the shot group sizes 1, 2, 4, ... up to min(32, nshots) (and nshots
 * itself) and the launch forms of the "persistent" option that differ for
 * that grouping (and, for one launch per half-step, "split" 0 and 1, and 2
 * to 4 with tile code 1, and both "tile_order" values); each
 * is timed four times over `steps` forward and `steps` adjoint steps of
 * every shot (CUDA events on the model's stream, the best of the last three
 * kept) and the fastest is applied (options "tile_code", "group",
 * "persistent", "split" and "tile_order").  With cache_path, a line
 * "<key> <group> <form> <tile code> <split> <tile order> <ms> ..." whose key
 * (GPU name
 * with blanks as '_',
 * nr, window pitch, nshots, as bh_tune_lookup forms it) matches is applied
 * without timing; otherwise the timed choice is appended to the file.  The
 * timed runs overwrite the model's wavefields and history: any stored
 * forward history is invalidated.  Results of later calls do not depend on
 * the group or the form (bit for bit); the tile code changes them at the
 * rounding level (see "tile_code").
 *   steps       >= 1 (clamped to nt and to the history window)
 *   cache_path  host path or NULL
 *   choice      host char[choice_len] or NULL: the choice and the timings
 * Errors: BH_ERR_INVALID_ARG, BH_ERR_STATE (history window below one
 *   step), BH_ERR_OOM, BH_ERR_CUDA.
 */
bh_status bh_tune(bh_model* model, int steps, const char* cache_path, char* choice,
                  int choice_len);

/*
 * The cached launch configuration (group, form, tile code, split, tile
 * order) for a key (host only, no GPU): the last
 * line of cache_path whose key is gpu_name (blanks as '_') | nr |
 * window_pitch (the largest window length rounded up to 32) | nshots.
 * Errors: BH_ERR_INVALID_ARG, BH_ERR_STATE (no such line, or no file).
 */
bh_status bh_tune_lookup(const char* cache_path, const char* gpu_name, int nr,
                         int window_pitch, int nshots, int* group, int* form, int* tile_code,
                         int* split, int* tile_order);

/*
 * Read-only facts about a model (the paper has no counterpart):
 * "history_steps" (L), "snapshots" (s), "tail_steps" (steps whose history
 * the forward sweep stores itself), "recompute_steps" (forward steps
 * re-run by one bh_adjoint_gradient), "tiles", "persistent",
 * "persistent_blocks_fwd", "persistent_blocks_adj", "persistent_runs_per_step"
 * (stepping-kernel launches of the last bh_forward + bh_adjoint_gradient),
 * "history_snapshot_bytes", "device_bytes", "kernel_launches" (kernels the
 * model has launched since it was created, for counting the launches of a
 * timed region), "group" (shots per launch group), "tile_code", "split",
 * "pipe_grid", "tile_order" (the options' values), "tma" (1 when the
 * tensor maps of "split" 4 exist), "pipe_blocks" (blocks of a pipelined
 * launch that fit the SMs), "state_version"
 * (changes whenever the stored forward
 * history is replaced or invalidated: bh_forward, bh_set_model, bh_update,
 * bh_update_velocity; a caller that keeps a forward run for a later
 * bh_adjoint_gradient can check that it is still the stored one).
 *   value  host double
 * Errors: BH_ERR_INVALID_ARG (unknown key).
 */
bh_status bh_get_info(bh_model* model, const char* key, double* value);

/*
 * The checkpoint schedule of the forward history (host only, no GPU; the
 * paper has no counterpart): for nseg segments and nsnap snapshot slots
 * (slot 0 is the zero initial state, slots 1..nsnap are stored), the
 * snapshots taken during the forward sweep, spine[k] = (segment, slot), and
 * the actions of the reversal, actions[k] = (kind, a, b) with kind
 * 0 ADVANCE from segment a to segment b, 1 TAKE slot a at segment b,
 * 2 RESTORE slot a (holding segment b), 3 REVERSE segment a.
 *   actions  host int [max_actions][3];  spine  host int [max_spine][2]
 * Errors: BH_ERR_INVALID_ARG (bad sizes; *n_actions and *n_spine still give
 *   the sizes needed).
 */
bh_status bh_checkpoint_plan(int nseg, int nsnap, int* actions, int max_actions,
                             int* n_actions, int* spine, int max_spine, int* n_spine);

/*
 * Starting model (Numerical Examples, Fig. 3 and Fig. 4): the paper takes
 * the formation velocities at the borehole wall from the semblance of the
 * near-monopole data, those one meter into the formation from the
 * ultra-far-monopole data, and interpolates linearly in r between them.
 * Per depth j: cells whose centre r = (i + 1/2) dr lies inside r_wall get
 * the fluid (vp_fluid, Vs = 0); others get
 * v = v_wall + t (v_far - v_wall), t = (r - r_wall) / (r_far - r_wall)
 * clamped to [0, 1] (the far values beyond r_far).  The semblance analysis
 * itself is not part of this library: the four velocity logs are inputs.
 * Needs no model.
 *   vp_wall, vs_wall, vp_far, vs_far  device [nz] float32
 *   vp, vs   device [nr][nz] float32, written
 *   stream   cudaStream_t (NULL = legacy default stream); the call
 *            returns once the work is enqueued
 * Errors: BH_ERR_INVALID_ARG (sizes, NULL, r_far <= r_wall), BH_ERR_CUDA;
 *   bh_last_error(NULL) gives the message.
 */
bh_status bh_starting_model(int nr, int nz, double dr, double r_wall, double r_far,
                            const float* vp_wall, const float* vs_wall, const float* vp_far,
                            const float* vs_far, float vp_fluid, float* vp, float* vs,
                            void* stream);

/*
 * The forward-history plan bh_model_create picks under a byte cap (host
 * only, no GPU; the paper has no counterpart).  The nt steps split into
 * segments of L steps and a tail of the last `tail` steps, whose history
 * the forward sweep stores as it goes; every segment is re-run once into the
 * history window before its adjoint, from one of nsnap snapshots (binomial
 * schedule when they are fewer than the segments).  Memory:
 * (max(tail, L) + 1) history slots of hist_step_bytes each plus nsnap
 * snapshots of snapshot_bytes each, at most cap_bytes; the plan with the
 * fewest recomputed forward steps wins, then the least memory.  tail = nt
 * (L = nt, nsnap = 0, recompute = 0) stores every step.
 *   hist_step_bytes  v_r, v_z planes of one step of every shot
 *   snapshot_bytes   one full forward state of every shot
 *   L, nsnap, tail, recompute  host outputs
 * Errors: BH_ERR_INVALID_ARG, BH_ERR_OOM (cap below one history window).
 */
bh_status bh_plan_history(int nt, double hist_step_bytes, double snapshot_bytes,
                          size_t cap_bytes, int* L, int* nsnap, int* tail,
                          long long* recompute);

/* Static description of a status code. */
const char* bh_status_string(bh_status status);

/* Text of the last error on this model ("" if none); NULL model: the last
 * error of bh_model_create, bh_residual_misfit_noalloc, bh_starting_model or
 * bh_plan_history on this thread. */
const char* bh_last_error(const bh_model* model);

#ifdef __cplusplus
}
#endif

#endif /* BH_H */
