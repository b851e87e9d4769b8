/*
 * lbm.h - C ABI of the GB300 semiclassical lattice Boltzmann library.
 *
 * The library advances the isothermal semiclassical (Fermi-Dirac,
 * Bose-Einstein or Maxwell-Boltzmann weight) lattice Boltzmann model of
 * Coelho & Doria, "Lattice Boltzmann method for semiclassical fluids",
 * arXiv 1710.09472, Sec. 9.1, on one CUDA device:
 *
 *   f_a(x + e_a, t + 1) = f_a(x, t) - (f_a(x, t) - f^eq_a(x, t)) / tau [+ S_a]
 *
 * with the second-order equilibrium of Sec. 9.1 (equivalently Sec. 5.1),
 * the Lorentz forcing of Sec. 7 (velocity shift or explicit term), halfway
 * bounce-back on links into solid cells, and a hand-written adjoint.
 *
 * Conventions shared by every call:
 *   - dims = {nx, ny, nz}; 2D lattices take nz = 1, 1D ny = nz = 1.  Cells are numbered
 *     cell = (z * ny + y) * nx + x (x fastest); N = nx * ny * nz.
 *   - The box is periodic in every direction; walls and obstacles come
 *     only from the solid mask.
 *   - Velocity-set order (rest vector first, then opposite pairs; a odd
 *     has opposite a + 1):
 *       D2V9 : 0 (0,0) 1 (1,0) 2 (-1,0) 3 (0,1) 4 (0,-1) 5 (1,1) 6 (-1,-1)
 *              7 (1,-1) 8 (-1,1)
 *       D3V19: 0 (0,0,0) 1 (1,0,0) 2 (-1,0,0) 3 (0,1,0) 4 (0,-1,0)
 *              5 (0,0,1) 6 (0,0,-1) 7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0)
 *              10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1)
 *              15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
 *       D3V27: D3V19's 0 .. 18, then 19 (1,1,1) 20 (-1,-1,-1) 21 (1,1,-1)
 *              22 (-1,-1,1) 23 (1,-1,1) 24 (-1,1,-1) 25 (-1,1,1) 26 (1,-1,-1)
 *       D1V3 : 0 (0) 1 (1) 2 (-1)
 *   - Velocities u, currents j = rho u, fields E and B are in the paper's
 *     xi units (velocity / reference speed c_s, Sec. 8; Sec. 9.3 takes the
 *     acceleration a = E).  A lattice-unit velocity is c_s * u.
 *   - Per-cell vector fields are laid out component-major: v[d * N + cell].
 *   - "State at time t": after t calls' worth of steps, f(x, t) is the
 *     post-stream (pre-collision) population field.  Moments are those of
 *     f(x, t): rho = sum_a f_a, rho u = sum_a f_a e_a / c_s (the reading of
 *     Sec. 9.1 Eq. mac-fields-model-sec-eq without the stray w_a).
 *   - Pointer arguments marked "host or device" may point to either; the
 *     library inspects them.  Device pointers must belong to the context's
 *     device.  Caller buffers are only borrowed for the duration of a call.
 *   - Calls are asynchronous on the context's stream unless they return
 *     host values, in which case they synchronise that stream first.
 *   - Every call returns an lbm_status and never aborts; on error the
 *     context keeps a message readable with lbm_last_error().
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1,      /* a bad size, pointer, enum or parameter */
    LBM_ERR_UNSTABLE_LATTICE = 2, /* a weight w_a or c_s is not positive (Sec. 8) */
    LBM_ERR_CUDA = 3,             /* a CUDA runtime call failed; see lbm_last_error */
    LBM_ERR_OOM = 4,              /* device or host allocation failed */
    LBM_ERR_NONFINITE = 5,        /* a NaN/Inf appeared in a reduction */
    LBM_ERR_TIMEOUT = 6,          /* a kernel's bounded wait on its own asynchronous copies ran
                                     out (about 1 s); reported by the next synchronising call
                                     (lbm_moments with totals or host outputs, lbm_get_populations,
                                     lbm_window_totals, lbm_adjoint, lbm_save_state); the state
                                     is then invalid */
    LBM_ERR_STATE = 7             /* call out of order (e.g. step before init) */
} lbm_status;

typedef enum { LBM_D2V9 = 0, LBM_D3V19 = 1, LBM_D3V27 = 2, LBM_D1V3 = 3 } lbm_velset;
    /* D2V9 Sec. 8.2, D1V3 Sec. 8.1, D3V19 and D3V27 Table lattices-tab (App. A) */
typedef enum { LBM_FD = 0, LBM_BE = 1, LBM_MB = 2 } lbm_stat;      /* Sec. 2, Eq. be-fd-dist-eq */
typedef enum { LBM_F32 = 0, LBM_F16_DEV = 1, LBM_BF16_DEV = 2 } lbm_dtype;
typedef enum { LBM_FORCE_SHIFT = 0, LBM_FORCE_TERM = 1 } lbm_force; /* Sec. 7 */

/* Model description.
 *   vel   : lbm_velset
 *   stat  : weight omega(xi) (Sec. 2, 9.1): FD 1/(exp((xi^2-mu)/theta)+1),
 *           BE 1/(exp((xi^2-mu)/theta)-1) with mu < 0,
 *           MB (2 pi theta)^(-D/2) exp(-xi^2 / 2 theta) (theta = 1: Hermite).
 *   theta, mu : weight parameters (the paper's electrons: 1/270 and 1).
 *   force : LBM_FORCE_SHIFT - f^eq evaluated at u + tau (E + u x B)
 *           (Sec. 7, Eq. u-update-force-term-eq);
 *           LBM_FORCE_TERM  - explicit source S_a = a_a . grad_u f^eq_a with
 *           a_a = E + xi_a x B (Sec. 7, Eq. forcing-term-integrals-eq).
 *   rho0  : reference density of the stored deviations (see lbm_create). */
typedef struct {
    int vel;
    int stat;
    double theta;
    double mu;
    int force;
    double rho0;
} lbm_lattice;

/* Create a context and allocate its device buffers.
 *   dims   : {nx, ny, nz}, each >= 1 (nz == 1 for D2V9, ny == nz == 1 for D1V3); N < 2^31 * 16.
 *   tau    : BGK relaxation time, > 1/2.
 *   E, B   : uniform field (3 components each, may be NULL = 0).  In 2D only
 *            E_x, E_y and B_z act.
 *   storage: population storage.  Every storage keeps the deviation
 *            h_a = f_a - rho0 w_a / I_0 from the rest equilibrium at rho0;
 *            LBM_F32 stores h in FP32, LBM_F16_DEV stores 2^12 h in FP16,
 *            LBM_BF16_DEV stores h in BF16.  Collision arithmetic is FP32.
 *   cuda_stream: cudaStream_t to run on (NULL = the legacy default stream).
 * Host-side set-up derives I_0..I_4 (Sec. 3, Eq. i2n-cont2), the EDF
 * coefficients (Sec. 5.1) and the lattice weights and c_s (Sec. 8) in FP64.
 * The new context has no geometry (all fluid) and no state: call
 * lbm_init_equilibrium before lbm_step.  *out receives the handle; the
 * caller releases it with lbm_destroy.
 * Errors: INVALID_ARG, UNSTABLE_LATTICE (a weight or c_s <= 0), OOM, CUDA. */
lbm_status lbm_create(lbm_ctx** out, const lbm_lattice* lat, const int64_t dims[3], double tau,
                      const double E[3], const double B[3], int storage, void* cuda_stream);

/* Release every buffer of the context (synchronises its stream).  NULL is a no-op. */
void lbm_destroy(lbm_ctx* ctx);

/* Copy the host-side constants into out[0..n-1] (FP64):
 *   I0 I2 I4 c0 c1 c2 cbar2 cprime2 thetabar J2 Delta2 cs w[0..Q-1]
 * (Sec. 3 coefficients, Sec. 9.1 thetabar = I2/I0, Sec. 8 weights).
 * n must be >= 12 + Q.  Errors: INVALID_ARG. */
lbm_status lbm_constants(const lbm_ctx* ctx, double* out, int n);

/* Read back sizes: out = {D, Q, nx, ny, nz, N, n_fluid, steps_done,
 * bytes_per_population}.  n must be >= 9.  n_fluid is exact once the
 * geometry is set (synchronises).  Errors: INVALID_ARG. */
lbm_status lbm_info(const lbm_ctx* ctx, int64_t* out, int n);

/* Solid geometry (Sec. 9.3 walls, Sec. 9.4 obstacles): solid_mask[N] bytes,
 * nonzero = solid, host or device.  Links from a fluid cell into a solid cell
 * bounce back halfway.  Resets the state (call lbm_init_equilibrium again).
 * Errors: INVALID_ARG, CUDA. */
lbm_status lbm_set_geometry(lbm_ctx* ctx, const uint8_t* solid_mask);

/* Per-cell electric field E(x) (the acceleration of Sec. 7, a_E = E):
 * E[D * N] FP32, component-major, host or device; copied into the context.
 * NULL switches back to the uniform E of lbm_create / lbm_set_params.
 * Errors: INVALID_ARG, OOM, CUDA. */
lbm_status lbm_set_E_field(lbm_ctx* ctx, const float* E);

/* Rounding of FP16/BF16 stores: stochastic != 0 rounds each stored deviation
 * up or down with probability given by its distance to the two neighbouring
 * representable values (unbiased; the random bits are a hash of the step
 * index, the cell and the direction, so a replayed step is bit-identical);
 * 0 rounds to nearest even.  The default for FP16/BF16 storage is stochastic:
 * with nearest rounding, per-step increments below half an ulp of the stored
 * deviation are lost (for example the force increment of a 1e-6 field on
 * a flow at u ~ 3e-3).  Errors: INVALID_ARG (FP32 storage with stochastic). */
lbm_status lbm_set_rounding(lbm_ctx* ctx, int stochastic);

/* Seed of the stochastic-rounding stream (default 0).  Two runs that differ
 * only in this seed differ only by their rounding noise, which estimates the
 * rounding floor of 16-bit storage on problems too large for an FP64
 * reference.  A replayed step uses the seed in force when it is replayed, so
 * keep it fixed within one lbm_adjoint call.  Errors: INVALID_ARG. */
lbm_status lbm_set_rounding_seed(lbm_ctx* ctx, uint32_t seed);

/* Change tau, the uniform E and B between steps without reallocating.
 * E or B may be NULL (unchanged).  Errors: INVALID_ARG (tau <= 1/2). */
lbm_status lbm_set_params(lbm_ctx* ctx, double tau, const double E[3], const double B[3]);

/* Local chemical-potential model (enable != 0; 0 switches back).  The
 * collision uses the second-order EDF of Sec. 9.1, Eq. feq-exp-2nd-order-eq,
 * with the thetabar terms that Sec. 9.1 freezes at the weight's value taken
 * per cell: thetabar(x) = I_2/I_0 = theta g_{D/2+1}(z) / (2 g_{D/2}(z)) at the
 * chemical potential of the cell's density (Eq. rho-def-eq, inverted as in
 * Sec. 9.1.2), i.e. the weight-equals-EDF choice of Sec. 5, Eq. omega-feq,
 * for the density while the lattice (c_s, w_a) stays the weight's.  Densities
 * are in units where rho0 is the weight's own density I_0(mu): a cell of
 * density rho has I_0(mu(x)) = (rho / rho0) I_0(mu).  thetabar comes from a
 * table over rho / rho0 in [1/4, 4] (3841 nodes, cubic Hermite; outside that
 * range the end value is used), built on the device when the model is
 * enabled (FD weight; with the MB weight thetabar does not depend on mu and
 * the model equals the default one).  Its steps run on the row-staged
 * kernel (an instantiation with a run-time row stride) where the rows
 * qualify, else on the general kernel.  lbm_init_equilibrium keeps the
 * default EDF; the local thetabar enters from the first collision.
 * lbm_adjoint differentiates the model too: its reverse step adds the
 * density derivative of the local terms (thetabar'(rho) from the same table).
 * Errors: INVALID_ARG (D3V27, D1V3 or the BE weight: not built), OOM, CUDA. */
lbm_status lbm_set_local_mu(lbm_ctx* ctx, int enable);

/* Start state f(x, 0) = f^eq(rho(x), u(x)) on fluid cells (Sec. 9.1 EDF, no
 * force shift).  rho[N] FP32 (NULL = rho0 everywhere) and u[D * N] FP32 in
 * xi units (NULL = 0), host or device.  Sets the step counter to 0.
 * Errors: INVALID_ARG, CUDA. */
lbm_status lbm_init_equilibrium(lbm_ctx* ctx, const float* rho, const float* u);

/* Advance n >= 0 time steps (collide, then stream; one fused kernel per
 * step).  Asynchronous.  Errors: STATE (no init), CUDA. */
lbm_status lbm_step(lbm_ctx* ctx, int64_t n);

/* Moments of the current state f(x, t): rho[N] and j[D * N] (FP32, host or
 * device, either may be NULL; solid cells get 0), and the FP64 totals over
 * fluid cells total_rho = sum rho, total_j[3] = sum j (host, either may be
 * NULL; requesting a total or a host output synchronises).  Totals are
 * reduced deterministically (fixed tree order).
 * Errors: STATE, CUDA, NONFINITE (a total is NaN/Inf). */
lbm_status lbm_moments(lbm_ctx* ctx, float* rho, float* j, double* total_rho, double total_j[3]);

/* Populations of the current state as FP32, f[Q * N] (population-major:
 * f[a * N + cell]), host or device; solid cells get 0.  deviation == 0 gives
 * f_a(x, t); deviation != 0 gives the stored deviation h_a = f_a - rho0 w_a / I_0
 * exactly as the kernels see it (decoded from the storage format).
 * Errors: STATE, CUDA. */
lbm_status lbm_get_populations(lbm_ctx* ctx, float* f, int deviation);

/* Advance t_end steps from the current state and return the window sums of
 * the FP64 fluid totals over the states after steps t_begin+1 .. t_end:
 *   out = {sum_t sum_x rho, sum_t sum_x j_x, sum_t sum_x j_y, sum_t sum_x j_z}.
 * t_begin = -1 includes the start state.  Requires -1 <= t_begin <= t_end.
 * Synchronises.  Errors: INVALID_ARG, STATE, CUDA, NONFINITE. */
lbm_status lbm_window_totals(lbm_ctx* ctx, int64_t t_begin, int64_t t_end, double out[4]);

/* Frees the device buffers that lbm_adjoint keeps in the context between
 * calls (forward states, adjoint fields, gradient scratch).  Synchronises the
 * context's stream.  Infrastructure; the paper has no counterpart.  Errors:
 * INVALID_ARG. */
lbm_status lbm_release_workspace(lbm_ctx* ctx);

/* Device bytes that an lbm_adjoint call with checkpoint_every = 0 may spend
 * on kept forward states (0, the default: 95% of the free device memory left
 * after the adjoint fields).  The adjoint fields and gradient scratch come on
 * top.  Infrastructure for the checkpoint schedule; the paper has no
 * counterpart.  Errors: INVALID_ARG. */
lbm_status lbm_set_memory_budget(lbm_ctx* ctx, uint64_t bytes);

/* Schedule of the last lbm_adjoint call and the size of one kept state:
 * out = {0 segment / 1 binomial / 2 every state kept, state buffers held, forward steps run,
 * reverse steps run, bytes per state buffer}.  Errors: INVALID_ARG. */
lbm_status lbm_adjoint_stats(const lbm_ctx* ctx, int64_t out[5]);

/* Failure-path self-check (the paper has no counterpart).  Launches one block
 * that waits on an mbarrier that nothing completes, using the same bounded
 * wait as the row-staged kernels but a limit of `clocks` SM cycles
 * (1 <= clocks <= 2^31).  The wait runs out, the block writes its code into
 * the context's status word and returns, and this call (which synchronises)
 * returns LBM_ERR_TIMEOUT, just as a real timeout would be reported.  The
 * context stays usable.  Errors: INVALID_ARG, CUDA; an earlier unreported
 * timeout is returned first. */
lbm_status lbm_selftest_wait_timeout(lbm_ctx* ctx, int64_t clocks);

/* Reverse-mode gradient of a linear functional of the trajectory that starts
 * at the current state f_0 (this is an addition to the paper's method: a
 * hand-written adjoint of the Sec. 9.1 step, with the Sec. 7 forcing):
 *   L = sum_{t_begin < t <= t_end} sum_x [w_rho(x) rho_t(x) + w_j(x) . j_t(x)],
 * where rho_t, j_t are the moments after t steps (lbm_moments convention).
 * The call leaves the context at step t_end, as lbm_step would.  The reverse
 * step kernel maps lam_{t+1} = dL/df_{t+1} to lam_t and needs the forward
 * state at t; checkpoint_every chooses how those states are kept:
 *   K > 0 : segment schedule: t_end forward steps keeping a copy every K
 *           steps, then each segment is replayed from its copy storing every
 *           state (ceil(t_end / K) + K - 1 states; 2 t_end forward steps);
 *   K = 0 : every state kept during the one forward sweep (t_end - 1 extra
 *           states, no replay) when they fit the memory budget
 *           (lbm_set_memory_budget); else the segment schedule with
 *           K = ceil(sqrt(t_end)) when it fits; else the binomial schedule
 *           with as many snapshots as fit;
 *   K < 0 : binomial schedule with -K snapshots: the recursion of Griewank's
 *           revolve (snapshots placed so that s snapshots and r sweeps cover
 *           C(s + r, s) steps), holding -K + 2 states (the initial state and a
 *           work buffer besides the snapshots).
 * Forward states are recomputed bit for bit (the stochastic-rounding stream
 * depends on the global step index only), so every schedule gives the same
 * gradients.
 *   w_rho[N], w_j[D * N] : FP32 loss weights, host or device, NULL = 0.
 *   t_begin, t_end       : -1 <= t_begin < t_end, t_end >= 1.
 *   dL_dE   : [D * N] FP64 device, per-cell dL/dE(x) (overwritten), or NULL.
 *             With a uniform E, sum_x dL/dE(x) is the uniform-field gradient.
 *   dL_dB   : 3 host doubles, dL/dB (2D: only the z component), or NULL.
 *   dL_dtau : host double, or NULL.   loss : host double (L itself), or NULL.
 *   dL_df0  : [Q * N] FP32 device, dL/df_0 (population-major, [a * N + cell], as
 *             lbm_get_populations), or NULL.
 * Device memory: the schedule's states (populations + bounce-back link
 * buffer each) plus two FP32 adjoint fields (Q N values + one per bounce-back
 * link each), and with dL_dE an FP32 partial of it (D N values).  The
 * context keeps these buffers after the call and reuses them in the next one
 * (buffers it already holds count as free memory when the schedule is
 * chosen); lbm_release_workspace, lbm_set_geometry and lbm_destroy free them.
 * dL/dB, dL/dtau and the loss accumulate in FP64; dL/dE(x) accumulates in the
 * FP32 partial for at most 32 reverse steps at a time, each batch then added
 * into the FP64 dL_dE.  The sweep is deterministic.
 * Synchronises.  Errors: INVALID_ARG, STATE, OOM (with the size needed), CUDA,
 * NONFINITE. */
lbm_status lbm_adjoint(lbm_ctx* ctx, const float* w_rho, const float* w_j, int64_t t_begin, int64_t t_end,
                       int64_t checkpoint_every, double* dL_dE, double dL_dB[3], double* dL_dtau, double* loss,
                       float* dL_df0);

/* FP64 weight integrals I_0, I_2, ..., I_8 of the weight omega (Sec. 3, Eq.
 * i2n-cont2) in dimension D, for stat / theta / mu as in lbm_lattice.
 * Host only; needs no device.  Errors: INVALID_ARG. */
lbm_status lbm_weight_integrals(int D, int stat, double theta, double mu, double I[5]);

/* Serialise / restore the state (raw stored populations, in the library's
 * internal layout, plus a header with lattice, dims, storage, step count and a
 * checksum) to / from host memory.
 * lbm_save_state with host_buf == NULL only reports the size in *used.
 * lbm_load_state checks the header against the context.
 * Errors: INVALID_ARG (short buffer, header mismatch, bad checksum), CUDA. */
lbm_status lbm_save_state(lbm_ctx* ctx, void* host_buf, size_t cap, size_t* used);
lbm_status lbm_load_state(lbm_ctx* ctx, const void* host_buf, size_t len);

/* FP64 fluid totals of the current state, like the totals of lbm_moments, but
 * without any device allocation; the paper has no counterpart (this is a
 * library service).  It is meant for callers that cannot or must not call
 * the CUDA allocator where they read the totals, for example an application
 * that reserves all device memory for its own pool up front, or a
 * time-critical loop in which allocation calls are forbidden.
 *   totals : 4 doubles in device memory, owned by the caller, written
 *            asynchronously on the context's stream with
 *            {sum rho, sum j_x, sum j_y, sum j_z} over fluid cells.
 * The per-block partial sums live in one file-scope device array of 262144
 * x 4 doubles (8 MiB), held by every GPU that loads the library until the
 * process exits; grids needing more partials than that, i.e.
 * ny * nz * ceil(nx / 128) > 262144, are rejected with INVALID_ARG and a
 * message.  Each call overwrites every partial it reads, so nothing needs
 * clearing; but every call in the process shares the one array, so calls
 * whose kernels overlap on the GPU (different streams or contexts running
 * concurrently) race and must be serialised by the caller.  The first call on
 * a device looks up the array's device address once (cudaGetSymbolAddress);
 * make that first call before any stream capture.  That address is kept for
 * the rest of the process: after cudaDeviceReset on a device the module may
 * load at another address, so do not call this entry point on a device that
 * has been reset.  The context's device must be current.  Errors:
 * INVALID_ARG, STATE, CUDA. */
lbm_status lbm_moment_totals_static(lbm_ctx* ctx, double* totals);

/* ------------------------------------------------------------------------- */
/* One-dimensional thermal model with the fourth-order equilibrium.          */
/* The EDF is Eq. feq-4order-01 (Sec. 4): f^eq_a = w_a sum_{N <= order}      */
/* A_N . P_N(xi_a) / N!, with the polynomials and coefficients of Sec. 3      */
/* (c_K up to K = 4, c'_K, cbar_K, d_4, d'_4, dbar_4) and the projections     */
/* A_N(rho, u, thetabar, g) of Sec. 4.  thetabar(x) is local: rho (thetabar   */
/* + u^2) = sum_a f_a xi_a^2, so the collision keeps mass, momentum and       */
/* energy; g is held at the weight's value I0 I4 / I2^2.  The lattice is      */
/* D1V5 (roots a and b of Table lattices-tab) or D1V7 (App. A; root 0 is the  */
/* printed closed form, the largest positive root of its cubic, roots 1 and   */
/* 2 the next smaller positive ones).  A uniform force E acts by the velocity */
/* shift u* = u + tau E (Sec. 7, Eq. u-update-force-term-eq).  The box is     */
/* periodic, with no solid cells.                                             */
/* Populations are stored as the deviation h_a = f_a - rho0 w_a / I0, FP32,   */
/* FP16 (scaled by 2^12) or BF16, direction-major h[a * nx + x]; the         */
/* collision is FP32; FP16/BF16 stores round stochastically by default.      */
/* ------------------------------------------------------------------------- */
typedef struct lbm_thermal lbm_thermal;  /* opaque; owns its device memory */
typedef enum {
    LBM_T_D1V5A = 0,   /* e = 0, +-1, +-3; c_s^2 with the + sign */
    LBM_T_D1V5B = 1,   /* the - sign */
    LBM_T_D1V7 = 2,    /* e = 0, +-1, +-2, +-3; root 0 of the App. A cubic */
    LBM_T_D1V7_R1 = 3, /* root 1 */
    LBM_T_D1V7_R2 = 4  /* root 2 */
} lbm_thermal_lattice;

/* stat, theta, mu: the weight (as lbm_lattice); nx cells; tau > 1/2; E the
 * uniform force (xi units); order 2, 3 or 4 (terms of the EDF kept);
 * storage an lbm_dtype; stream a cudaStream_t or NULL.  Rho0 = 1.  Errors:
 * INVALID_ARG, UNSTABLE_LATTICE (no such root, or a weight or c_s not
 * positive, Sec. 8), OOM, CUDA. */
lbm_status lbm_thermal_create(lbm_thermal** out, int lattice, int stat, double theta, double mu, int64_t nx,
                              double tau, double E, int order, int storage, void* stream);
void lbm_thermal_destroy(lbm_thermal* t);

/* out[0..4] I_0..I_8, out[5] c_s, out[6] g, out[7..11] c_0..c_4,
 * out[12..14] c'_2..c'_4, out[15..17] cbar_2..cbar_4, out[18..20] d_4, d'_4,
 * dbar_4, out[21] thetabar of the weight (I2/I0), out[22] Q, out[23] tau,
 * out[24..24+Q) the weights; n >= 24 + Q.  Errors: INVALID_ARG. */
lbm_status lbm_thermal_constants(const lbm_thermal* t, double* out, int n);

/* Stochastic (default for FP16/BF16) or nearest rounding of the stores, and
 * the seed of the stochastic stream.  Errors: INVALID_ARG (FP32 with
 * stochastic). */
lbm_status lbm_thermal_set_rounding(lbm_thermal* t, int stochastic, uint32_t seed);

/* f(x, 0) = f^eq(rho(x), u(x), thetabar(x)) (no force shift): each of rho,
 * u, thetabar is nx FP32 values, host or device, or NULL (rho0 = 1, u = 0,
 * thetabar = I2/I0).  Asynchronous.  Errors: INVALID_ARG, CUDA. */
lbm_status lbm_thermal_init(lbm_thermal* t, const float* rho, const float* u, const float* thetabar);

/* n collide-and-stream steps (Sec. 9.1 discrete Boltzmann equation),
 * asynchronous on the stream.  Errors: INVALID_ARG, STATE, CUDA. */
lbm_status lbm_thermal_step(lbm_thermal* t, int64_t n);

/* Per-cell rho, j = sum f xi and energy sum f xi^2 = rho (thetabar + u^2)
 * (nx FP32 each, device, any may be NULL), and, when totals is not NULL,
 * their FP64 sums over the box on the host (synchronises).  Errors:
 * INVALID_ARG, STATE, NONFINITE, CUDA. */
lbm_status lbm_thermal_moments(lbm_thermal* t, float* rho, float* j, float* energy, double totals[3]);

/* f_a(x) (or h_a(x) when deviation != 0) into f[Q * nx] FP32, device,
 * direction-major.  Errors: INVALID_ARG, STATE, CUDA. */
lbm_status lbm_thermal_populations(lbm_thermal* t, float* f, int deviation);

const char* lbm_thermal_last_error(const lbm_thermal* t);
int64_t lbm_thermal_launch_count(const lbm_thermal* t);

/* ------------------------------------------------------------------------- */
/* Density <-> chemical potential of the Fermi-Dirac equilibrium, as field   */
/* conversions (the paper uses them to set initial conditions and to report  */
/* fields, Sec. 9.1.2):                                                       */
/*   rho = (pi theta)^{D/2} g_{D/2}(e^{mu/theta})          (Sec. 9.1, Eq. rho-def-eq) */
/*   mu  = theta ln g_{D/2}^{-1}(rho / (pi theta)^{D/2})    (Sec. 9.1.2)      */
/* with the complete FD integral g_nu of Sec. 4 (before Eq. rho-fd-be-eq), in */
/* the non-dimensional units of Eq. fd-dist-non-dim-eq.  mu / rho: n FP32     */
/* values in device memory (the input is only read), computed in FP64 on the  */
/* stream (cudaStream_t or NULL), asynchronous.  A non-positive or infinite   */
/* density gives NaN.  The first call on a device for a dimension D builds a  */
/* 144 KB table of ln g_{D/2} on that device (and synchronises the stream);   */
/* the table stays until the process exits.  D in 1..3, theta > 0.            */
/* Errors: INVALID_ARG (bad D, theta, n or a host pointer), OOM, CUDA.        */
/* ------------------------------------------------------------------------- */
lbm_status lbm_density_from_mu(int D, double theta, const float* mu, float* rho, int64_t n, void* stream);
lbm_status lbm_mu_from_density(int D, double theta, const float* rho, float* mu, int64_t n, void* stream);

/* Message of the last failed call on this context ("" if none). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Static text of a status code. */
const char* lbm_status_string(lbm_status s);

/* Number of kernels this context has launched so far (host-side counter). */
int64_t lbm_launch_count(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
