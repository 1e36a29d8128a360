/*
 * irkgl.h -- C-ABI of the GB300 IRKGL16 library (libirkgl.so).
 *
 * The library integrates batches of separable second-order systems
 *     q'' = g(q),  y = (q, v),  q, v in R^d
 * with IRKGL16, the 8-stage order-16 Gauss-Legendre collocation method in
 * the exactly-symplectic second-order floating-point form of
 * arXiv 2511.03655:
 *   G_i = g(Q_i),  R_i = h b_i G_i                         (Sec. 2.4, Eq. Gi)
 *   Q_i = q_{n-1} + h (c_i v_{n-1} + sum_j eta_ij R_j)    (Eq. Qi2)
 *   v_n = v_{n-1} + sum_i R_i,
 *   q_n = q_{n-1} + h v_n - h sum_i c_i R_i                 (Eq. qnvn2)
 * solved by the stage-wise fixed-point iteration of Eq. IRK_FP2, started
 * from the extrapolated guess of Eq. IRK_init2 (Eq. Pol0), stopped by the
 * roundoff-aware rule of Eqs. Delta_n / stopping (positions only), with the
 * state (q, v) kept as compensated hi + lo pairs (Sec. 5).  Everything is
 * computed in FP64 on the GPU.
 *
 * Conventions for every function:
 *   - Return value: IRKGL_OK (0) or a negative irkgl_error.  Launches are
 *     asynchronous on the given CUDA stream (cudaStream_t passed as void*,
 *     NULL = legacy default stream); a device-side failure surfaces on the
 *     next synchronising call.  Per-trajectory outcomes are written to
 *     status[] (IRKGL_STATUS_*).
 *   - Layout: FP64, trajectory-major, contiguous: positions and velocities
 *     are [batch][dim]; stage increments R are [batch][8][dim].
 *   - Ownership: the caller owns every array passed in; the library owns
 *     only the context and its small device workspace.  Pointers documented
 *     as "device" must be CUDA device (or managed) memory on the current
 *     device; "host" pointers are ordinary host memory.
 *   - A context's calls must not overlap on the device (issue them on one
 *     stream, or synchronise between streams): they share one work counter.
 *   - Thread safety: distinct contexts may be used from distinct host
 *     threads; one context is not re-entrant.
 */
#ifndef IRKGL_H
#define IRKGL_H

#ifdef __cplusplus
extern "C" {
#endif

#define IRKGL_STAGES 8

typedef enum {
  IRKGL_OK = 0,
  IRKGL_ERR_INVALID = -1,     /* an argument is out of range or NULL where required */
  IRKGL_ERR_NOMEM = -2,       /* a host or device allocation failed */
  IRKGL_ERR_CUDA = -3,        /* a CUDA runtime call failed (see irkgl_last_cuda_error) */
  IRKGL_ERR_UNSUPPORTED = -4  /* no compiled kernel for this (rhs kind, dim, tile) */
} irkgl_error;

/* Per-trajectory outcome written to status[]. */
enum {
  IRKGL_STATUS_OK = 0,        /* all requested steps completed */
  IRKGL_STATUS_MAXITER = 1,   /* a step reached the sweep cap without meeting Eq. stopping;
                                 the trajectory stops at the start of that step */
  IRKGL_STATUS_NONFINITE = 2, /* a stage value became Inf/NaN; stops as above */
  IRKGL_STATUS_BAD_INSTANCE = 3 /* ragged batches: the instance descriptor is invalid (kind,
                                   dim > dmax, parameter count); nothing of it was touched */
};

/* Built-in right-hand sides g(q) (device functions; the paper's user
 * function f_ODE! of Sec. 3 is replaced by these compiled kinds). */
typedef enum {
  IRKGL_RHS_KEPLER = 1,        /* d = 2: g = -mu q/|q|^3;            params = {mu} */
  IRKGL_RHS_NBODY = 2,         /* d = 3N: g_a = G sum_b m_b (q_b - q_a)/|q_b - q_a|^3;
                                  params = {G, m_0, ..., m_{N-1}} */
  IRKGL_RHS_FPUT = 3,          /* d = n: FPUT alpha chain, fixed ends; params = {alpha} */
  IRKGL_RHS_HENON_HEILES = 4,  /* d = 2: Henon-Heiles (Sec. 5.1);    params = {lambda} */
  IRKGL_RHS_HARMONIC = 5,      /* any d: g = -omega^2 q;             params = {omega} */
  IRKGL_RHS_HENON_HEILES_FORCED = 6, /* d = 2: the non-autonomous example of Sec. 3,
                                  g(t, q) with lambda + xi sin t in place of lambda;
                                  params = {lambda, xi}.  Evaluated at the stage times
                                  t_n + c_i h.  Time starts at 0 except through
                                  irkgl_advance_t; the energy monitor is off (dH_max = 0) */
  /* First-order systems y' = f(y) (the mu form of Eq. Yi2; use the irkgl_*1 calls,
     dim = D, the full state dimension): */
  IRKGL_RHS_SCHWARZSCHILD = 7, /* D = 4: charged particle near a Schwarzschild black hole in a
                                  magnetic field, Eq. Ham_SBH; y = (r, theta, p_r, p_theta);
                                  params = {E, L, beta} */
  IRKGL_RHS_HARMONIC1 = 8      /* D = 2: q' = p, p' = -omega^2 q; params = {omega} */
} irkgl_rhs_kind;

typedef struct {
  irkgl_rhs_kind kind;
  const double* params;  /* host pointer, copied by irkgl_create */
  int nparams;           /* number of doubles at params */
} irkgl_rhs;

/* Coefficient tables, row-major [i*8 + j] (i: stage being formed). */
typedef struct {
  double c[8], b[8], mu[64], eta[64], nu[64];
} irkgl_coeffs;

/* Optional outputs of irkgl_integrate (device pointers; NULL = not wanted,
 * except q and v which are required). */
typedef struct {
  double* q;          /* [batch][dim] final positions (hi parts of the compensated pairs) */
  double* v;          /* [batch][dim] final velocities (hi parts) */
  double* q_lo;       /* [batch][dim] compensation parts */
  double* v_lo;       /* [batch][dim] */
  double* r_prev;     /* [batch][8][dim] R of the last completed step (for a resumed run) */
  double* dH_max;     /* [batch] max over monitored steps of |(H_n - H_0)/H_0|, Eq. DHglobmax */
  long long* iters;   /* [batch] total fixed-point sweeps (evaluations of g = 8 x iters) */
  long long* steps;   /* [batch] steps completed */
  int* status;        /* [batch] IRKGL_STATUS_* */
} irkgl_outputs;

/* Outputs of irkgl_integrate1 (first-order kinds; device pointers, NULL =
 * not wanted except y). */
typedef struct {
  double* y;          /* [batch][D] final state (hi parts of the compensated pairs) */
  double* y_lo;       /* [batch][D] compensation parts */
  double* l_prev;     /* [batch][8][D] L of the last completed step (for a resumed run) */
  double* dH_max;     /* [batch] max over monitored steps of |(H_n - H_0)/H_0| */
  long long* iters;   /* [batch] total fixed-point sweeps */
  long long* steps;   /* [batch] steps completed */
  int* status;        /* [batch] IRKGL_STATUS_* */
} irkgl_outputs1;

/* One instance of a ragged batch (irkgl_integrate_ragged): its own right-hand
 * side, dimension, step and horizon.  States of all instances are packed
 * one after another: instance k occupies elements [offset, offset + dim) of
 * the packed position/velocity arrays and [8*offset, 8*(offset + dim)) of a
 * packed R array; its parameters are params[param_offset .. + nparams). */
typedef struct {
  int kind;           /* irkgl_rhs_kind: IRKGL_RHS_NBODY, IRKGL_RHS_FPUT or IRKGL_RHS_HARMONIC */
  int dim;            /* position dimension d (N-body: 3 x bodies) */
  long long offset;   /* first packed element of this instance */
  int param_offset;   /* first parameter in the packed parameter array */
  int nparams;        /* N-body: 1 + bodies (G, masses); FPUT: 1 (alpha); harmonic: 1 (omega) */
  double h;           /* step size (finite, nonzero) */
  long long nsteps;   /* steps to take (>= 0) */
} irkgl_instance;

/* Options for irkgl_set_option. */
enum {
  IRKGL_OPT_LANES_PER_TRAJ = 1, /* tile: 1, 2, 4 or 8 lanes share one trajectory's 8 stages
                                   (0 = the built-in default for (kind, dim)) */
  IRKGL_OPT_KMAX = 2,           /* sweep cap per step (default 100); 1..1000 */
  IRKGL_OPT_MONITOR_EVERY = 3,  /* evaluate H every m steps for dH_max (default 1; 0 = off) */
  IRKGL_OPT_BLOCK_THREADS = 4,  /* threads per block: 64, 128 or 256 (default 128) */
  IRKGL_OPT_GRID_BLOCKS = 5,    /* persistent grid size (0 = one full wave, the default) */
  IRKGL_OPT_WIDE_TEAM = 6,      /* ragged batches: threads per instance, 32, 64, 128 or 256
                                   (0 = 256, the default: fastest or within a few per cent of
                                   the fastest for every size measured on GB300) */
  IRKGL_OPT_MONITOR_LOCAL = 7,  /* 1: dH_max reports the local error max_n |(H_n - H_{n-1})/H_{n-1}|
                                   (Eq. DHlocmax) instead of the global one (default 0; not
                                   carried across irkgl_advance calls) */
  IRKGL_OPT_MIX = 8,            /* stage mixing of Eq. Qi2 and the initial guess: 0 = FP64 FMA
                                   chain (default); 1 = exact fixed-point sums on the integer
                                   pipes, rounded once (the one-lane and component-split tiles,
                                   the tiles with the stage rows spread over lanes, the wide
                                   kernel); needs the default tables.  2 = reproducible: every
                                   FP64 operation of the method's plain definition rounded
                                   separately, in that definition's order (the two-matrix
                                   initial guess of Eq. IRK_init2 with nu and mu, sums left to
                                   right from j = 1, g and H with IEEE division and square root,
                                   dH as |(H_n - H_0) / H_0|), one thread per trajectory; any
                                   IEEE-754 binary64 program of the same sequence (no
                                   contraction, no flush to zero) returns the same bits, sweep
                                   counts included.  Uses the context's own tables.  The
                                   second-order calls of the register kinds (Kepler, Henon-Heiles,
                                   harmonic d <= 3, N-body 3..6 bodies) and the ragged calls
                                   (N-body up to 128 bodies, FPUT, harmonic; d <= 1536, every
                                   team size giving the same bits), and the first-order calls of
                                   IRKGL_RHS_HARMONIC1 for every IRKGL_OPT_STAGES; not the
                                   kinds whose sin and cos are not correctly rounded (the
                                   time-dependent kind, Schwarzschild).  A call with no
                                   compiled kernel for the choice returns
                                   IRKGL_ERR_UNSUPPORTED */
  IRKGL_OPT_TILE_LAYOUT = 10,   /* second-order kinds: 1 = the stage-split tiles (LPT lanes per
                                   trajectory share the stages); 2 = the component-split tile for
                                   d = 2 (Kepler, Henon-Heiles): two lanes per trajectory, each
                                   holding one component of all eight stages, so the mixing of
                                   Eq. Qi2 uses compile-time coefficients and no exchange
                                   (IRKGL_ERR_UNSUPPORTED at the call for other kinds); 0 = auto
                                   (default): the component split with the fixed-point mixing where
                                   compiled, else the stage split.  Results are bit-identical
                                   between the layouts (to the two-lane stage split with mix 0, the
                                   one-lane tile with mix 1) */
  IRKGL_OPT_STAGES = 9          /* first-order kinds: s of the s-stage IRKGL scheme, 2, 4, 6 or 8
                                   (default 8 = IRKGL16; s < 8 uses the built-in Gauss tables of
                                   that s, order 2s).  l_prev arrays are then [batch][s][D].  The
                                   second-order calls accept only 8 (IRKGL_ERR_UNSUPPORTED) */
};

/* Fill *out with the default IRKGL16 tables of Sec. 2.4 (nodes c and weights
 * b of the 8-point Gauss rule; mu of Eq. Yi2; eta of Eq. Qi2 satisfying
 * Eq. sympl_cond_2 exactly; nu of Eq. Pol0 scaled to L = h b F).
 * Host-only; needs no GPU.  Returns IRKGL_ERR_INVALID if out is NULL. */
int irkgl_default_coeffs(irkgl_coeffs* out);

/* Create a context for right-hand side f, position dimension dim (>= 1) and
 * default step h (finite, nonzero; negative integrates backwards).
 * coeffs == NULL selects irkgl_default_coeffs.  Allocates the context and a
 * few bytes of device workspace on the current device.  Errors:
 * IRKGL_ERR_INVALID (bad kind/dim/params/h), IRKGL_ERR_NOMEM, IRKGL_ERR_CUDA. */
int irkgl_create(struct irkgl_ctx** out, irkgl_rhs f, int dim, double h,
                 const irkgl_coeffs* coeffs);

/* Set an IRKGL_OPT_* option; IRKGL_ERR_INVALID for an unknown key or value. */
int irkgl_set_option(struct irkgl_ctx* ctx, int option, long long value);

/* Advance `batch` trajectories by `nsteps` steps each, in place (device
 * arrays).  This is the step-by-step form (Eq. IRK_init2 -> Eq. IRK_FP2 ->
 * Eq. qnvn2 per step), used for chunked integration, resumption and the
 * plain one-trajectory-per-launch form (batch = 1, nsteps = 1).
 *   q, v      [batch][dim] in/out hi parts (required)
 *   q_lo,v_lo [batch][dim] in/out compensation parts; NULL = start from 0
 *             and do not write back
 *   r_prev    [batch][8][dim] in/out R of the previous step (zero before the
 *             first step); NULL = zeros, not written back
 *   h         [batch] per-trajectory steps, or NULL for the context's h
 *   iters     [batch][nsteps] sweeps per step, or NULL
 *   status    [batch] outcome, or NULL
 * batch == 0 or nsteps == 0 is a no-op.  Errors: IRKGL_ERR_INVALID,
 * IRKGL_ERR_UNSUPPORTED, IRKGL_ERR_CUDA. */
int irkgl_step(struct irkgl_ctx* ctx, double* q, double* v, double* q_lo, double* v_lo,
               double* r_prev, const double* h, int batch, int nsteps, int* iters,
               int* status, void* cuda_stream);

/* Advance device-resident trajectories by a per-trajectory number of steps,
 * continuing everything a long run carries (the compensated state, R_prev
 * for the extrapolated guess of Eq. IRK_init2, the reference energy H_0 and
 * the running max |dH/H|), so a run split into chunks of any sizes gives the
 * bits of one uninterrupted run.  Used by the serving loop, which advances
 * many requests in interleaved chunks.  Device arrays, [batch] unless noted:
 *   q, v, q_lo, v_lo [batch][dim], r_prev [batch][8][dim]   in/out (required)
 *   h        per-trajectory step, or NULL for the context's h
 *   nsteps   steps to take in this call (0 = leave the trajectory alone)
 *   H0       in/out reference energy (required when dH_max is given)
 *   h0_init  1 on the first call of a run: H0 is computed at the first step
 *            and written; 0 afterwards: H0 is read, except that an entry
 *            holding NaN is computed at that trajectory's first step in this
 *            call (when it takes one) and written
 *   dH_max, iters   in/out running maxima / totals (NULL = not tracked)
 *   status   out: IRKGL_STATUS_* of this call (NULL = not wanted)
 * Errors: IRKGL_ERR_INVALID, IRKGL_ERR_UNSUPPORTED, IRKGL_ERR_CUDA. */
int irkgl_advance(struct irkgl_ctx* ctx, double* q, double* v, double* q_lo, double* v_lo,
                  double* r_prev, const double* h, const long long* nsteps, double* H0,
                  int h0_init, double* dH_max, long long* iters, int* status, int batch,
                  void* cuda_stream);

/* irkgl_advance for a batch that mixes many requests of one right-hand-side
 * kind and dimension (the serving loop's shared state arrays, Sec. 3's
 * driver loop run for many problems at once): every trajectory may carry its
 * own parameters, trajectories join the batch between calls, and idle slots
 * of the arrays are skipped without being touched.
 *   params        [batch][param_stride] device parameters: trajectory b uses
 *                 params[b * param_stride ...] (param_stride >= the kind's
 *                 parameter count, as given to irkgl_create); NULL with
 *                 param_stride = 0 uses the context's parameters for all
 *   order         [batch] device list of the slots to advance, -1 for a slot
 *                 to skip (its arrays are neither read nor written), or NULL
 *                 for 0..batch-1
 *   H0            in/out [batch]: an entry holding NaN (a trajectory that
 *                 joins the batch) is computed at its first step in this call
 *                 and written; the others are read
 *   status        in/out [batch] (NULL = not tracked): zero before a
 *                 trajectory's first call; an entry that is nonzero on entry
 *                 (IRKGL_STATUS_MAXITER / NONFINITE of an earlier call) marks a
 *                 trajectory that stopped, which is not advanced again and
 *                 keeps its status, as in one uninterrupted run
 *   q .. r_prev, h, nsteps, dH_max, iters as in irkgl_advance.
 * A trajectory's bits do not depend on what else is in the batch or on how
 * its steps are split over calls.  Errors: IRKGL_ERR_INVALID (also for
 * param_stride below the kind's count), IRKGL_ERR_UNSUPPORTED, IRKGL_ERR_CUDA. */
int irkgl_advance_multi(struct irkgl_ctx* ctx, double* q, double* v, double* q_lo, double* v_lo,
                        double* r_prev, const double* h, const long long* nsteps,
                        const double* params, int param_stride, const int* order, double* H0,
                        double* dH_max, long long* iters, int* status, int batch,
                        void* cuda_stream);

/* irkgl_advance for a right-hand side that depends on t (IRKGL_RHS_HENON_HEILES_FORCED),
 * with the time carried alongside the state.  Each trajectory starts at
 * t_n = t[b] + t_lo[b]; g is evaluated at the stage times fl(t[b] + fl(h c_i))
 * (Eq. IRK_FP, first line, with the time split off by the paper's
 * compensated-sum device of Sec. 5), and after every step (t, t_lo) gains h
 * by the same TwoSum + Fast2Sum update as q and v, so chunked runs give the
 * bits of one run.  Device arrays, [batch] unless noted:
 *   q, v, q_lo, v_lo [batch][dim], r_prev [batch][8][dim]   in/out (required)
 *   t        in/out time, hi part (required)
 *   t_lo     in/out time, compensation part; NULL = 0, not written back
 *   h        per-trajectory step, or NULL for the context's h
 *   nsteps   steps to take in this call (required)
 *   iters    in/out running total of sweeps (NULL = not tracked)
 *   status   out: IRKGL_STATUS_* of this call (NULL = not wanted)
 * No energy monitor (H(t) is not conserved).  Errors: IRKGL_ERR_INVALID (also
 * for a context whose right-hand side does not read t), IRKGL_ERR_UNSUPPORTED,
 * IRKGL_ERR_CUDA. */
int irkgl_advance_t(struct irkgl_ctx* ctx, double* q, double* v, double* q_lo, double* v_lo,
                    double* r_prev, double* t, double* t_lo, const double* h,
                    const long long* nsteps, long long* iters, int* status, int batch,
                    void* cuda_stream);

/* First-order systems y' = f(y) (IRKGL_RHS_SCHWARZSCHILD, IRKGL_RHS_HARMONIC1), in the
 * exactly-symplectic mu form of Sec. 2.4 (Eq. Yi2): per step the guess
 * Y_i = y + sum_j nu_ij Lprev_j (Eq. IRK_init), sweeps L_i = h b_i f(Y_i),
 * Y_i = y + sum_j mu_ij L_j (Eq. IRK_FP) until Eq. stopping holds on all D
 * components, then y += sum_i L_i with a compensated pair (Eq. yn2, Sec. 5).
 * The context is created by irkgl_create with dim = D.  Second-order calls
 * on such a context, and these calls on a second-order context, return
 * IRKGL_ERR_INVALID.
 *
 * irkgl_integrate1: y0 [batch][D] device, per-trajectory nsteps (or
 * nsteps_all), h (or NULL for the context's), order (or NULL); outputs as in
 * irkgl_outputs1.  Lprev starts at zero. */
int irkgl_integrate1(struct irkgl_ctx* ctx, const double* y0, int batch, const long long* nsteps,
                     long long nsteps_all, const double* h, const int* order,
                     const irkgl_outputs1* out, void* cuda_stream);

/* irkgl_advance1: continue device-resident first-order trajectories in place
 * (y, y_lo [batch][D], l_prev [batch][8][D], all required), carrying H0 /
 * dH_max / iters like irkgl_advance (a NaN entry of H0 included), so chunked
 * runs give the bits of one run. */
int irkgl_advance1(struct irkgl_ctx* ctx, double* y, double* y_lo, double* l_prev, const double* h,
                   const long long* nsteps, double* H0, int h0_init, double* dH_max,
                   long long* iters, int* status, int batch, void* cuda_stream);

/* Explicit symplectic splitting baselines (Sec. 4, not IRKGL): the drift
 * q += (a_j h) v and kick v += (b_j h) g(q) flows of Eq. flowAB in the
 * sequence of Eq. high_order_splitting, with compensated (TwoSum + Fast2Sum)
 * q and v pairs, one thread per trajectory.  For the GPU form of the
 * paper's time-per-g-evaluation comparison (Table tab:overhead).
 *   scheme  IRKGL_SPLIT_STRANG (Eq. Strang, 1 g evaluation per step) or
 *           IRKGL_SPLIT_SUZ90 (Suzuki's fourth-order composition of five Strang
 *           steps, 5 evaluations per step)
 * Compiled for Kepler and Henon-Heiles (dim 2) and the 6-body problem (dim 18);
 * other contexts return IRKGL_ERR_UNSUPPORTED, first-order ones
 * IRKGL_ERR_INVALID.  Arguments as in irkgl_integrate; out->iters receives
 * the number of g evaluations, out->r_prev is not written; out->dH_max
 * follows the context's monitor options (IRKGL_OPT_MONITOR_LOCAL: Eq. DHlocmax). */
enum { IRKGL_SPLIT_STRANG = 1, IRKGL_SPLIT_SUZ90 = 2 };
int irkgl_split_integrate(struct irkgl_ctx* ctx, int scheme, const double* q0, const double* v0,
                          int batch, const long long* nsteps, long long nsteps_all, const double* h,
                          const irkgl_outputs* out, void* cuda_stream);

/* Integrate `batch` independent initial states (device arrays q0, v0
 * [batch][dim], R_prev = 0, lo = 0) in one persistent launch.
 *   nsteps  [batch] steps per trajectory (device), or NULL to use nsteps_all
 *   h       [batch] per-trajectory steps (device), or NULL for the context's h
 *   order   [batch] processing order, a permutation of 0..batch-1 (device),
 *           or NULL for 0..batch-1; grouping similar trajectories next to
 *           each other reduces lock-step waste inside a warp
 *   out     output pointers (see irkgl_outputs)
 * Errors: IRKGL_ERR_INVALID, IRKGL_ERR_UNSUPPORTED, IRKGL_ERR_CUDA. */
int irkgl_integrate(struct irkgl_ctx* ctx, const double* q0, const double* v0, int batch,
                    const long long* nsteps, long long nsteps_all, const double* h,
                    const int* order, const irkgl_outputs* out, void* cuda_stream);

/* Same as irkgl_integrate but every array is a HOST pointer: the inputs are
 * copied to the device, integrated, and the outputs copied back before the
 * call returns (synchronous on cuda_stream).  Device staging buffers are
 * owned by the context and grow on demand.  Errors as irkgl_integrate, plus
 * IRKGL_ERR_NOMEM. */
int irkgl_integrate_host(struct irkgl_ctx* ctx, const double* q0, const double* v0, int batch,
                         const long long* nsteps, long long nsteps_all, const double* h,
                         const int* order, const irkgl_outputs* out, void* cuda_stream);

/* Integrate a ragged batch: `ninst` independent instances of different right-hand
 * sides and dimensions (irkgl_instance, device array) in one persistent launch
 * of the wide kernel: a team of threads (a warp, or a whole block, see
 * IRKGL_OPT_WIDE_TEAM) owns one instance at a time, with its 8 stage values
 * in shared memory.  The step is the same as irkgl_integrate's (Eqs.
 * IRK_init2, IRK_FP2, stopping, qnvn2 with compensated sums), starting from
 * R_prev = 0 and lo = 0.
 *   dmax     the largest inst[k].dim (host value; sizes shared memory), 1..1536
 *            (above 1024 only with 256-thread teams); N-body instances may have
 *            at most 128 bodies (larger ones get IRKGL_STATUS_BAD_INSTANCE)
 *   params   packed parameters (device)
 *   q0, v0   packed initial states (device)
 *   order    processing order (device permutation of 0..ninst-1) or NULL;
 *            costliest first keeps the persistent teams balanced
 *   out      q, v, q_lo, v_lo packed like q0; r_prev packed [.][8][dim];
 *            dH_max, iters, steps, status per instance
 * The context supplies the tables, options and work counter; its own right-
 * hand side and dimension are not used.  Errors: IRKGL_ERR_INVALID,
 * IRKGL_ERR_UNSUPPORTED (dmax beyond the compiled shapes), IRKGL_ERR_CUDA. */
int irkgl_integrate_ragged(struct irkgl_ctx* ctx, const irkgl_instance* inst, int ninst, int dmax,
                           const double* params, const double* q0, const double* v0,
                           const int* order, const irkgl_outputs* out, void* cuda_stream);

/* Continue a ragged batch in place (the wide-kernel counterpart of
 * irkgl_advance): instance k takes nsteps[k] steps (device int64 [ninst];
 * inst[k].nsteps is ignored) from the packed state q, v, q_lo, v_lo, r_prev
 * (all required, in/out), with H0 / h0_init / dH_max / iters as in
 * irkgl_advance (per instance; with h0_init = 0 a NaN entry of H0 is computed
 * at that instance's first step in the call).  status is in/out as in
 * irkgl_advance_multi: zero it before an instance's first call; an instance
 * whose entry is nonzero on entry stopped in an earlier call and is not
 * advanced again.  order (device, [ninst], or NULL for 0..ninst-1) lists the
 * instances to advance; an entry of -1 is skipped without touching that
 * instance's memory, so a serving loop can keep idle descriptors in its
 * arrays.  Errors as irkgl_integrate_ragged. */
int irkgl_advance_ragged(struct irkgl_ctx* ctx, const irkgl_instance* inst, int ninst, int dmax,
                         const double* params, double* q, double* v, double* q_lo, double* v_lo,
                         double* r_prev, const long long* nsteps, double* H0, int h0_init,
                         double* dH_max, long long* iters, int* status, const int* order,
                         void* cuda_stream);

/* Release the context and its device workspace (NULL is ignored). */
void irkgl_destroy(struct irkgl_ctx* ctx);

/* Static text for an irkgl_error or IRKGL_STATUS_* value (never NULL). */
const char* irkgl_strerror(int code);

/* The CUDA error string of the last IRKGL_ERR_CUDA on this host thread. */
const char* irkgl_last_cuda_error(void);

/* Lanes per trajectory that the context would use for its (kind, dim). */
int irkgl_get_tile(struct irkgl_ctx* ctx);

/* The tile layout a call on this context runs: 1 = stage split, 2 = component
 * split (IRKGL_OPT_TILE_LAYOUT resolved), 3 = the reproducible form's one
 * thread per trajectory (IRKGL_OPT_MIX = 2); first-order contexts report 1.
 * Returns IRKGL_ERR_INVALID for a NULL context. */
int irkgl_get_layout(struct irkgl_ctx* ctx);

/* Diagnostic, not part of the method: launch an FP64 fused multiply-add
 * throughput probe (a full grid of independent FMA chains) on cuda_stream
 * and store the number of FMAs it issues in *fma_count (host pointer).
 * scratch is one device double the probe may write.  The caller times the
 * launch with events on the same stream; FMAs / seconds is the FP64 roof
 * used for the roofline fraction.  Errors: IRKGL_ERR_INVALID, IRKGL_ERR_CUDA. */
int irkgl_probe_fp64_fma(double* scratch, long long* fma_count, void* cuda_stream);

/* Diagnostic, not part of the method: the fixed-point stage mixing of
 * IRKGL_OPT_MIX = 1 applied to n columns R[n][8] (device): out[n][8][2]
 * receives sum_j eta_ij R_j and sum_j W_ij R_j for each row i, as the kernel
 * computes them (exact sums rounded once).  Errors: IRKGL_ERR_INVALID,
 * IRKGL_ERR_CUDA. */
int irkgl_diag_fixed_mix(const double* R, double* out, int n, void* cuda_stream);

/* Diagnostic, not part of the method: the same sums as irkgl_diag_fixed_mix
 * (same arguments, layout and errors), formed the way the stage-split tiles
 * that spread the stage rows over several lanes form them: one 128-bit
 * accumulator per row, a negative coefficient applied to the two's
 * complement of the operand, and a per-row constant.  The results must equal
 * irkgl_diag_fixed_mix's bit for bit. */
int irkgl_diag_fixed_mix_rows(const double* R, double* out, int n, void* cuda_stream);

/* Diagnostic, not part of the method: the reciprocal roots the right-hand
 * sides evaluate, for n arguments x[n] (device): out[n][3] (device)
 * receives x^(-3/2) (the gravitational force factor), x^(-1/2) (the
 * potential) and 1/x (the Schwarzschild terms).  Errors: IRKGL_ERR_INVALID,
 * IRKGL_ERR_CUDA. */
int irkgl_diag_rinv(const double* x, double* out, int n, void* cuda_stream);

/* Diagnostic, not part of the method: sin x and cos x as the Schwarzschild
 * right-hand side evaluates them, for n arguments x[n] (device): out[n][2]
 * (device) receives (sin, cos).  Errors: IRKGL_ERR_INVALID, IRKGL_ERR_CUDA. */
int irkgl_diag_sincos(const double* x, double* out, int n, void* cuda_stream);

/* Integration for callers that cannot allocate device memory.  (The paper
 * has no counterpart: this is a deployment entry point.)
 *
 * Some callers cannot call cudaMalloc: applications that reserve nearly all
 * device memory for their own pool up front, real-time or certified code
 * that forbids allocation after start-up, and plug-ins that must not touch
 * the device heap of the host application.  This call does the work of
 * irkgl_create(f, dim, h, NULL) + irkgl_integrate(...) + irkgl_destroy with
 * the default tables and options (default tile, 128 threads per block,
 * sweep cap 100, energy monitor every step), and allocates nothing: no
 * context, no cudaMalloc/cudaFree.  The caller passes every input and output
 * (device pointers, as for irkgl_integrate; f.params is a host pointer).
 *
 * Its scratch (the persistent grid's work counter and a copy of f.params)
 * is a fixed array of 64 doubles (512 bytes) inside the library, held by
 * every GPU that loads the library until the process exits.  All calls
 * share it and it keeps the last call's contents: each call clears the
 * counter and rewrites the parameters before launching, so calls that
 * overlap on the GPU race on it; serialise them (one stream, or ordering
 * between streams).  The first call on a device looks up the array's device
 * address for that device (cudaGetSymbolAddress) and keeps it for the life
 * of the process; make that first call before any stream capture on that
 * device.  The kept address does not survive cudaDeviceReset: do not call
 * this entry point on a device after resetting it.  As with irkgl_integrate,
 * the energy monitor is off for the time-dependent kind
 * IRKGL_RHS_HENON_HEILES_FORCED (dH_max is left at 0).
 *
 * Errors: IRKGL_ERR_INVALID for the same argument errors as irkgl_create /
 * irkgl_integrate (including the first-order kinds, which take the
 * irkgl_*1 calls), and when f.nparams > IRKGL_NOALLOC_MAX_PARAMS (the
 * parameters must fit the fixed scratch); IRKGL_ERR_UNSUPPORTED;
 * IRKGL_ERR_CUDA. */
#define IRKGL_NOALLOC_MAX_PARAMS 63
int irkgl_integrate_noalloc(irkgl_rhs f, int dim, double h, const double* q0, const double* v0,
                            int batch, const long long* nsteps, long long nsteps_all,
                            const double* h_per_traj, const int* order,
                            const irkgl_outputs* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* IRKGL_H */
