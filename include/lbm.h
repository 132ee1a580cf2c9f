/*
 * lbm.h -- C ABI of the GB300 fractional-step MRT lattice Boltzmann solver.
 *
 * The library advances the two-phase model of Zhang, Guo & Li, "A fractional
 * step lattice Boltzmann model for two phase flows with large density
 * differences" (arXiv:1812.02459) on one CUDA device:
 *   - Sec. III.A: MRT lattice Boltzmann equation for the Cahn-Hilliard
 *     sub-equation (Eqs. distribution_CH, feq_CH, collison, D2Q9MRT, Fi);
 *   - Sec. III.A: finite-difference TVD-RK3 step for the profile and flux
 *     correction d_t phi = div(lambda J_phi + q) (Eqs. step2, TVD-3order,
 *     fourOrder_FDM);
 *   - Sec. III.B: velocity-based MRT lattice Boltzmann equation for the
 *     incompressible Navier-Stokes equations with the forcing of
 *     Eqs. (reformNS), (Gi), (u), solved by Picard sweeps;
 *   - Sec. III.B: explicit selective filter of (p, u) (Eq. filter, App. B).
 *
 * Conventions shared by every call:
 *   - Host fields are row-major double arrays [ny][nx], x = column i,
 *     y = row j, lattice units (dx = dt = 1).  Population sets are [9][ny][nx]
 *     in the direction order c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1)
 *     c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1) (Sec. III.A Eq. D2Q9).
 *   - Axes with periodic_* = 0 carry halfway bounce-back no-slip walls at
 *     -1/2 and n-1/2; stencils see mirrored ghosts there (phi, mu, p even,
 *     u odd).
 *   - The handle owns every device buffer it allocates (cudaMalloc at
 *     lbm_create, cudaFree at lbm_destroy).  The caller owns every pointer it
 *     passes; no call keeps or aliases a caller pointer after it returns.
 *   - Every call returns an lbm_status; no C++ exception crosses the ABI.
 *     After an error, lbm_last_error() describes it.  CUDA errors from
 *     earlier asynchronous work surface at the next synchronising call.
 *   - Work is issued on the CUDA stream given to lbm_create (NULL = the
 *     legacy default stream).  lbm_step is asynchronous; calls that return
 *     host data synchronise that stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_NDIAG 11
#define LBM_MIN_EXTENT 12   /* smallest nx, ny: the widest stencil halo */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,        /* invalid argument or parameter */
    LBM_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    LBM_ERR_OOM = 3,        /* device allocation failed */
    LBM_ERR_NONFINITE = 4,  /* a field holds NaN or Inf */
    LBM_ERR_RANGE = 5,      /* phi left [-1-delta, 1+delta] */
    LBM_ERR_STATE = 6       /* call not valid for this handle */
} lbm_status;

typedef enum {
    LBM_FP64 = 0,           /* populations and arithmetic in double */
    LBM_FP32 = 1,           /* populations and arithmetic in float */
    LBM_MIX_BF16 = 2,       /* populations stored as bf16, arithmetic in float */
    LBM_MIX_FP16 = 3        /* populations stored as fp16, arithmetic in float */
} lbm_precision;
/* The 16-bit words hold f_1..f_8 and g_q - w_q (3 p_hat + s_q(u^n)), the NS
 * populations less their equilibrium (Sec. III.B Eq. geq) at the node's
 * post-stream p_hat and the velocity u^n they were collided with; the rest
 * populations come from the FP32 moments (phi_bar, p_hat).  lbm_get_state /
 * lbm_set_state decode and encode this form. */

typedef struct {
    int nx, ny;             /* nodes per axis, each >= LBM_MIN_EXTENT */
    int periodic_x;         /* 1 periodic, 0 no-slip walls */
    int periodic_y;
    int precision;          /* an lbm_precision */
} lbm_grid;

typedef struct {
    double M;               /* CH mobility (Sec. II.A Eq. final_mCHE) */
    double eta;             /* CH equilibrium parameter; tau_f = 1/2 + M/(eta cs^2) (Eq. mobility) */
    double W;               /* interface width (Eq. equilibrium_profile) */
    double sigma;           /* surface tension: kappa = 3 sigma W/8, beta = 3 sigma/(4W) (Sec. II.A) */
    double lambda;          /* weight of the profile flux J_phi in J_d = lambda J_phi + q (Sec. IV.B) */
    int flux_correction;    /* 1 includes q = -M (grad mu . n) n, 0 drops it */
    double rho_H, rho_L;    /* densities at phi = +1 and phi = -1 (Eq. rho) */
    double nu_H, nu_L;      /* kinematic viscosities; mu = rho nu interpolated linearly (Eq. dynamic_vis) */
    double s_f[9];          /* CH MRT rates; s_f[3], s_f[5] are replaced by 1/tau_f (Eq. CH_Sf) */
    double s_g[9];          /* NS MRT rates; s_g[7], s_g[8] are replaced by 1/tau_g(x) (Sec. III.B) */
    double gx, gy;          /* gravity, F_g = (rho - g_rho_ref) g (Sec. II.B; see g_rho_ref) */
    double g_rho_ref;       /* 0: F_g = rho g as printed; rho_ref > 0 measures gravity against the
                               hydrostatic pressure of a fluid of density rho_ref, which differs
                               from rho g by the gradient grad(rho_ref g.x) that the pressure absorbs */
    int filter_order;       /* 0 (off), 5, 7, 9 or 11: explicit selective filter SF-n (App. B) */
    double filter_a;        /* filter intensity, 0 < a <= 1 (Eq. filter) */
    int picard_iters;       /* sweeps of u = j + F(u)/(2 rho) per step (Eq. u), >= 1 */
    double picard_zeta;     /* must be 0: fixed sweep count (residual stop is not offered) */
    double grad_eps;        /* eps in n = grad phi / sqrt(|grad phi|^2 + eps^2), > 0 */
    unsigned flags;         /* 0, or LBM_FLAG_STRAIN_MOMENTS */
} lbm_params;

/* flags: the Picard sweeps take the strain rate grad u + grad u^T of F_nu
 * from the non-equilibrium part of the step's post-stream NS populations
 * (Sec. III.B Eq. Fmu, whose sum over f is read as one over g) instead of
 * the isotropic stencils:
 *   S = [(s_7 - s_1)(F0.u) I - s_7 (F0 u + u F0)] / (2 rho cs^2)
 *       - sum_i c_i c_i [M^-1 S^g M (g - g_eq(p_hat, u^k))]_i / cs^2,
 * with F0 the sweep's force without F_nu.  F_m still uses the stencils, as
 * does the collision.  FP64 and FP32 populations only; the sweeps then run
 * the one-node-per-thread kernel. */
#define LBM_FLAG_STRAIN_MOMENTS 1u

typedef struct lbm_handle lbm_handle;

/*
 * lbm_create -- allocate a simulation and initialise it from host fields.
 * phi0, p0, ux0, uy0: host [ny][nx] doubles (order parameter, kinematic
 * pressure p = p'/rho of Sec. II.B, velocity).  Populations start at their
 * equilibria: f = f_eq(phi0, mu(phi0), u0) (Eq. feq_CH), g = g_eq(p0, u0)
 * (Eq. geq).  stream: a cudaStream_t or NULL.  On success *out receives the
 * handle.  Errors: LBM_ERR_ARG for invalid sizes or parameters (tau_f or
 * tau_g <= 1/2, a rate outside [0,2], rho <= 0, W <= 0, a outside (0,1], a
 * filter order other than 0/5/7/9/11, picard_iters < 1, picard_zeta != 0,
 * undefined flags, LBM_FLAG_STRAIN_MOMENTS with 16-bit populations),
 * LBM_ERR_OOM, LBM_ERR_CUDA.
 */
lbm_status lbm_create(const lbm_grid *grid, const lbm_params *params,
                      const double *phi0, const double *p0,
                      const double *ux0, const double *uy0,
                      void *stream, lbm_handle **out);

/*
 * lbm_step -- advance n >= 0 time steps (the whole Sec. III update each
 * step: fields and forces, collision and streaming of both lattices, the
 * RK3 finite-difference correction, the implicit velocity, the filter).
 * Asynchronous on the handle's stream.  Errors: LBM_ERR_ARG for n < 0;
 * LBM_ERR_STATE once a synchronising call has reported that a kernel gave
 * up a bounded wait for a tile copy (see lbm_check): that step left its tile
 * un-updated and a copy landing late may still write the kernel's shared
 * memory, so the handle refuses further steps and must be destroyed.
 */
lbm_status lbm_step(lbm_handle *h, int n);

/*
 * lbm_step_ch -- advance n >= 0 steps of the Cahn-Hilliard part alone under
 * a prescribed velocity, as in the interface-capturing tests of
 * Sec. IV.A-B where the flow is given: each step takes mu from phi
 * (Eq. chemical), collides the CH populations with f_eq(phi, mu, u) and the
 * source F_i of d_t u + u.grad u (Eqs. feq_CH, Fi, with d_t u = u - u of the
 * previous step), streams them and applies the RK3 finite-difference
 * correction (Eq. TVD-3order).  The velocity of step k is
 * tfac[k] * (ux, uy): ux, uy are host [ny][nx] doubles and tfac a host array
 * of n factors, or NULL for 1 (a separable time dependence such as the
 * cos(pi t/T) of the single-vortex field needs no upload per step).  The
 * NS populations, p and u_hat are left as they are; the last step's
 * velocity becomes the state's velocity and its previous one.  Asynchronous
 * after the upload of ux, uy.  Errors: LBM_ERR_ARG (n < 0, NULL ux or uy,
 * reduced-precision populations), LBM_ERR_STATE as lbm_step.
 */
lbm_status lbm_step_ch(lbm_handle *h, int n, const double *ux, const double *uy, const double *tfac);

/*
 * lbm_fields -- copy phi, the filtered kinematic pressure p, and the
 * filtered velocity (ux, uy) into host [ny][nx] double arrays.  A NULL
 * pointer skips that field.  Synchronises the stream.
 */
lbm_status lbm_fields(lbm_handle *h, double *phi, double *p, double *ux, double *uy);

/*
 * lbm_dynamic_pressure -- the dynamic pressure p' = rho(phi) p into the host
 * [ny][nx] double array pd (caller-owned).  The state's p is the kinematic
 * pressure p'/rho (Sec. II.B, below Eq. reformNS); rho(phi) is Eq. (rho)
 * with phi clamped to [-1, 1], as in the step.  The product is formed on the
 * device in FP64 from phi (both floats of an FP32 handle's phi) and the
 * filtered p.  LBM_ERR_ARG for a NULL handle or pd.  Synchronises the
 * stream; like lbm_fields it reports a recorded device error.
 */
lbm_status lbm_dynamic_pressure(lbm_handle *h, double *pd);

/*
 * lbm_fields_device -- same fields into caller-owned device buffers of
 * nx*ny elements; dtype 0 = double, 1 = float.  Asynchronous.
 */
lbm_status lbm_fields_device(lbm_handle *h, void *phi, void *p, void *ux, void *uy, int dtype);

/*
 * lbm_set_fields -- re-initialise an existing handle from host fields, as
 * lbm_create does (no allocation).  Synchronises the stream.
 */
lbm_status lbm_set_fields(lbm_handle *h, const double *phi0, const double *p0,
                          const double *ux0, const double *uy0);

/*
 * lbm_diagnostics -- sums over the nodes (Sec. IV.C volume error,
 * Sec. IV.E Eqs. quantify-yc, quantify-uc), into host out[LBM_NDIAG]; the
 * sums are FP64 over row segments of at most 16 nodes (FP64 handles sum the
 * segments in FP64; FP32 handles form each term exactly as a pair of floats
 * and sum the segment with TwoSum, which matches FP64 sums of the same
 * fields to the order of FP64 rounding; exact counts in [1], [2], [3], [10]):
 *   [0] sum phi   [1] #(phi>0)   [2] #(phi<0)   [3] sum_{phi<0} y
 *   [4] sum_{phi<0} u_y   [5] sum w   [6] sum w y   [7] sum w u_y
 *       (w = (1-phi)/2, y = row index)   [8] max phi   [9] min phi
 *   [10] number of non-finite values among phi, p, ux, uy.
 * Synchronises the stream.
 */
lbm_status lbm_diagnostics(lbm_handle *h, double *out);

/*
 * lbm_diagnostics_async -- the sums of lbm_diagnostics, enqueued on the
 * handle's stream without waiting: the reduction kernels, then a copy of the
 * LBM_NDIAG doubles into host out.  out (caller-owned) must stay valid until
 * the stream has passed the copy (cudaStreamSynchronize or an event recorded
 * after the call); it should be page-locked host memory, otherwise the copy
 * is staged by the driver and may wait.  Calls on one handle are ordered by
 * the stream, so a later call never overwrites an earlier result before it
 * has been copied.  Lets a caller read back every step's sums while the next
 * step already runs.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA.
 */
lbm_status lbm_diagnostics_async(lbm_handle *h, double *out);

/*
 * lbm_check -- LBM_ERR_NONFINITE if any field value is NaN/Inf,
 * LBM_ERR_RANGE if phi leaves [-1-delta, 1+delta], LBM_ERR_CUDA if a kernel
 * of an earlier step gave up a bounded wait for a tile copy (its tile was
 * then not updated), else LBM_OK.  Synchronises the stream.  The device
 * word that records a given-up wait is also read by lbm_fields,
 * lbm_diagnostics, lbm_get_state and the adjoint calls, which then return
 * LBM_ERR_CUDA; from then on lbm_step returns LBM_ERR_STATE.
 */
lbm_status lbm_check(lbm_handle *h, double delta);

/*
 * lbm_set_check -- periodic finite and range check inside lbm_step.  With
 * every = k > 0, lbm_step enqueues the sums of lbm_diagnostics after every
 * k-th step on the handle's stream, into page-locked host memory the handle
 * owns, without waiting for them.  Each later lbm_step call first looks at
 * the last such result the stream has already passed (it never waits): if
 * it counted a non-finite value it returns LBM_ERR_NONFINITE, if phi left
 * [-1-delta, 1+delta] it returns LBM_ERR_RANGE, before issuing any work,
 * and keeps returning it until lbm_set_fields or lbm_set_state.  At most one
 * check is in flight; every = 0 (the default) turns the check off.
 * lbm_check remains the synchronising check.  Errors: LBM_ERR_ARG (every < 0,
 * delta < 0), LBM_ERR_CUDA (page-locked allocation).
 */
lbm_status lbm_set_check(lbm_handle *h, int every, double delta);

/*
 * lbm_get_state / lbm_set_state -- the full state between steps, as host
 * doubles: post-stream populations f, g [9][ny][nx]; phi; filtered p, ux,
 * uy; unfiltered velocity (uhx, uhy) of the last implicit update; filtered
 * velocity of the previous step (upx, upy).  Reduced-precision population
 * storage is decoded on get and encoded on set.  Synchronise the stream.
 */
lbm_status lbm_get_state(lbm_handle *h, double *f, double *g, double *phi, double *p,
                         double *ux, double *uy, double *uhx, double *uhy,
                         double *upx, double *upy);
lbm_status lbm_set_state(lbm_handle *h, const double *f, const double *g, const double *phi,
                         const double *p, const double *ux, const double *uy,
                         const double *uhx, const double *uhy,
                         const double *upx, const double *upy);

/*
 * Per-kernel device timing (a tracing aid, not part of the method).
 * lbm_profile(h, 1) clears the totals and starts recording CUDA events
 * around every kernel launch that lbm_step issues: within one lbm_step call
 * a launch that directly follows another starts at that one's end event, so
 * a step records one event per launch boundary (a launch's time then
 * includes the gap before it); lbm_profile(h, 0) stops.  lbm_profile_read
 * fills ms[k] (total device milliseconds) and
 * launches[k] for each kernel kind k < LBM_NKERNELS, summed since recording
 * started; it synchronises the stream.  Kinds: 0 collide+stream,
 * 1 RK3 stage, 2 Picard sweep, 3 filter.
 */
#define LBM_NKERNELS 4
lbm_status lbm_profile(lbm_handle *h, int on);
lbm_status lbm_profile_read(lbm_handle *h, double *ms, long long *launches);
const char *lbm_kernel_name(int kind);

/*
 * lbm_debug_violations -- in a library built with LBM_DEBUG (liblbm_debug.so,
 * the debug build beside liblbm.so), every paired shared-memory access of the
 * FP32 kernels is checked against the launch's dynamic shared memory; an
 * access outside it is skipped and the first one recorded.  Synchronises
 * the device and returns that record (block index in the high 32 bits,
 * 1 + byte offset in the low ones), or 0 when every access was in bounds,
 * and clears it.  ~0 if the device could not be read.  Always 0 in a
 * release build, which checks nothing.
 */
unsigned long long lbm_debug_violations(void);

/*
 * lbm_kernel_variant -- name of the kernel that lbm_step launches on this
 * handle for kernel kind `kind` (a static string; "none" for a filter of
 * order 0, "unknown" for a NULL handle or a kind outside 0..LBM_NKERNELS-1).
 * Which variant runs depends on the precision, the grid width, the wall
 * configuration and the relaxation rates; every variant computes the same
 * pass.
 */
const char *lbm_kernel_variant(const lbm_handle *h, int kind);

/*
 * Discrete adjoint of lbm_step (reverse mode), for gradients of a loss of the
 * final order parameter with respect to the initial order parameter, the
 * surface tension sigma and the mobility M.
 *   lbm_adjoint_begin(h, nsteps, k): the handle must hold a state freshly set
 *     from fields (lbm_create or lbm_set_fields, no step since) and FP64 or
 *     FP32 populations; axes periodic or walled as in lbm_step (the walls'
 *     bounce-back and mirrored stencil ghosts have their own
 *     vector-Jacobian products).  Advances nsteps steps, keeping
 *     every k-th state as a checkpoint on the device; the handle then holds
 *     the state after nsteps steps.  Errors: LBM_ERR_ARG, LBM_ERR_STATE,
 *     LBM_ERR_OOM, LBM_ERR_CUDA.
 *   lbm_adjoint_end(h, dL_dphi, dL_dphi0, dL_dsigma, dL_dM): dL_dphi is the
 *     host [ny][nx] gradient of the loss with respect to phi after nsteps.
 *     Runs the reverse sweep -- each segment of k steps is regenerated from
 *     its checkpoint and reversed step by step through the hand-written
 *     vector-Jacobian products of the step's plane operations, in the
 *     handle's arithmetic type (FP64 or FP32; the sigma and M gradients are
 *     summed in FP64) -- and writes dL/dphi0 (host [ny][nx], may be NULL),
 *     dL/dsigma and dL/dM (may be NULL).  The handle is left at the state
 *     after nsteps steps.
 *     Synchronises the stream.  Errors: LBM_ERR_STATE (no begin), LBM_ERR_ARG
 *     (also: walls without the compiled level kernels below), LBM_ERR_CUDA.
 * sigma enters through kappa = 3 sigma W/8 and beta = 3 sigma/(4W)
 * (Sec. II.A); M through tau_f (Eq. mobility), the flux q and J (Sec. II).
 */
lbm_status lbm_adjoint_begin(lbm_handle *h, int nsteps, int checkpoint_every);
lbm_status lbm_adjoint_end(lbm_handle *h, const double *dL_dphi, double *dL_dphi0,
                           double *dL_dsigma, double *dL_dM);

/*
 * lbm_adjoint_engine -- how the last lbm_adjoint_end on h ran the
 * vector-Jacobian products of the step: 1 when by level kernels compiled
 * for this tape at run time (the step's plane operations written out as
 * straight-line CUDA C++ and compiled once per tape structure with NVRTC
 * for sm_103a), 0 when by the tape interpreter kernels (NVRTC not found,
 * compilation failed, or LBM_ADJOINT_COMPILED=0 in the environment), -1
 * before any reverse sweep or for a NULL handle.  Both give the same
 * gradients up to rounding order.
 * The reverse sweep runs the tape's forward passes in batches of up to a
 * checkpoint segment's steps, fewer if the value planes would exceed a
 * quarter of the free device memory; LBM_ADJOINT_BATCH=<k> in the
 * environment caps a batch at k steps (same gradients, less memory).
 */
int lbm_adjoint_engine(const lbm_handle *h);

/*
 * lbm_field_sums_noalloc -- the sums of lbm_diagnostics for fields the
 * caller holds on the device, computed without allocating device memory.
 * The paper has no counterpart: this is an operational entry point.  It is
 * for callers that cannot call cudaMalloc -- a host framework that owns all
 * device memory through its own pool, a loop that cannot absorb the
 * device-wide synchronisation of cudaMalloc/cudaFree, a monitor that must
 * keep working after device memory is exhausted.
 *   phi, p, ux, uy: device arrays of nx*ny elements, row-major [ny][nx],
 *     dtype 0 = double, 1 = float (caller-owned, read only).
 *   out: device array of LBM_NDIAG doubles (caller-owned), written with the
 *     layout documented at lbm_diagnostics.
 *   stream: a cudaStream_t or NULL; the call is asynchronous on it.
 * Scratch: the block partial sums live in one file-scope static device
 * array sized for LBM_NOALLOC_MAX_NODES nodes (4096 partials x 11 doubles,
 * 352 KiB), held by every GPU that loads the library until the process
 * exits.  nx*ny above LBM_NOALLOC_MAX_NODES is rejected with LBM_ERR_ARG.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  All calls share the one array: calls that overlap on the
 * GPU (different streams, or different host threads without ordering) race
 * on it.  Nothing accumulates into it -- each call writes every partial it
 * later reads -- so no clearing is needed between calls.
 * Errors: LBM_ERR_ARG (NULL pointer, bad sizes or dtype), LBM_ERR_CUDA; the
 * text is in lbm_noalloc_last_error().  No cudaMalloc, cudaFree or
 * allocating library call is made.
 */
#define LBM_NOALLOC_MAX_NODES 67108864
lbm_status lbm_field_sums_noalloc(const void *phi, const void *p, const void *ux, const void *uy,
                                  int nx, int ny, int dtype, double *out, void *stream);
const char *lbm_noalloc_last_error(void);

/* lbm_device_bytes -- device memory held by the handle, in bytes. */
size_t lbm_device_bytes(const lbm_handle *h);

/* lbm_destroy -- free every device buffer of the handle; NULL is a no-op. */
void lbm_destroy(lbm_handle *h);

/* lbm_last_error -- text of the last error on h (or of the last failed
 * lbm_create when h is NULL); never NULL. */
const char *lbm_last_error(const lbm_handle *h);

#ifdef __cplusplus
}
#endif
#endif
