/*
 * acopf.h -- C ABI of the GB300 (sm_103a) SQP-ADMM solver for the AC optimal
 * power flow problem of Li, Schanen and Kim, "GPU-Accelerated Sequential
 * Quadratic Programming Algorithm for Solving ACOPF" (arXiv 2310.13143).
 *
 * The solver runs the trust-region SQP method of Algorithm 1 on the
 * rectangular ACOPF (Sec. III-A, eq. acopf).  Each QP subproblem (eq. QPsub,
 * with d_wR and d_wI eliminated as in Sec. III-C, eq. elim) is solved by the
 * component-decomposed ADMM of Algorithm 2: generator updates (eq.
 * gen_kernel), per-branch 4-variable QPs (eq. line_kernel, solved by an
 * augmented Lagrangian with a projected Newton inner solver), bus updates
 * (eq. bus_kernel, closed form) and multiplier updates (eq. multiplier),
 * with the residual test of Sec. IV-B.  Every step runs in CUDA kernels.
 *
 * Conventions
 *  - Every function returns acopf_status; ACOPF_OK is 0.  Nothing throws
 *    across the ABI.  Non-convergence is not an error: it is reported in
 *    acopf_residuals.result.
 *  - Units are per unit on base_mva, angles in radians, costs per MW.
 *  - Pointers marked "host" are read (or written) during the call only; the
 *    caller keeps ownership.  Device memory is owned by the handle.
 *  - Calls are asynchronous on the handle's stream except the acopf_get_*
 *    functions, which synchronise that stream before they return.
 *  - A handle is not thread-safe; calls on different handles are independent.
 *  - No CPU fallback: without a usable CUDA device acopf_create fails with
 *    ACOPF_ECUDA.
 */
#ifndef ACOPF_H
#define ACOPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct acopf_ctx* acopf_handle;

typedef enum {
  ACOPF_OK = 0,
  ACOPF_EINVAL = 1,     /* invalid argument or grid data (message in acopf_last_error) */
  ACOPF_ENOMEM = 2,     /* device or host allocation failed */
  ACOPF_ECUDA = 3,      /* CUDA runtime error */
  ACOPF_ETIMEOUT = 4,   /* a device-wide barrier of the ADMM kernel gave up waiting */
  ACOPF_ENOTREADY = 5   /* the requested data does not exist yet (e.g. no QP built) */
} acopf_status;

typedef enum {
  ACOPF_CONVERGED = 0,      /* primal and dual infeasibility <= tol */
  ACOPF_MAXITER = 1,        /* SQP iteration limit reached */
  ACOPF_STEP_TOO_SMALL = 2, /* accepted step below step_tol, or trust region below delta_min */
  ACOPF_NONFINITE = 3,      /* a non-finite value appeared */
  ACOPF_RUNNING = 4,        /* no solve has finished for this instance */
  ACOPF_INFEASIBLE = 5      /* locally infeasible: the feasibility restoration (sqp_options.restore)
                               stalled with the primal infeasibility above tol */
} acopf_result;

enum { ACOPF_FP64 = 0, ACOPF_MIXED = 1 };

/* One grid (Sec. III-A).  All pointers are host arrays read during
 * acopf_create only.  Branch (i, j) runs from f[l] to t[l] (0-based bus
 * indices).  tap and shift may be NULL (tap 1, shift 0).  rate <= 0 means no
 * line limit; angmin <= -2pi or angmax >= 2pi means no angle limit.
 * Exactly one bus must have bus_type 3 (reference); its angle is fixed at 0. */
typedef struct {
  int32_t nbus;
  const int32_t* bus_type;
  const double *pd, *qd, *gs, *bs, *vmin, *vmax;
  int32_t nbranch;
  const int32_t *f, *t;
  const double *r, *x, *b, *rate, *angmin, *angmax, *tap, *shift;
  int32_t ngen;
  const int32_t* gbus;
  const double *pmin, *pmax, *qmin, *qmax, *c2, *c1, *c0;
  double base_mva;
} acopf_grid;

typedef struct {
  int32_t precision;     /* ACOPF_FP64: ADMM sweep in FP64.  ACOPF_MIXED: ADMM state and
                            component updates in FP32; QP build, residual norms, step
                            acceptance and the iterate stay FP64 */
  int32_t use_angle;     /* 1: angle-difference limits enter the line subproblems */
  int32_t device;        /* CUDA device ordinal */
  int32_t block_threads; /* threads per CTA of the ADMM kernel (0: default 256) */
  int32_t ctas_per_sm;   /* resident CTAs per SM of the ADMM kernel (0: as many as fit) */
} acopf_options;

typedef struct {
  double rho;            /* ADMM penalty for every coupling (Tables I-II: 2e4) */
  double eps;            /* tolerance on the l_inf primal and dual residuals (Sec. IV-B) */
  double eps_dual;       /* separate tolerance on the dual residual s (0: eps).  In the FP32
                            sweep s = rho (z+ - z) has a floor of about rho times the FP32
                            resolution of z, so the mixed path needs a larger value */
  int32_t max_iter;      /* ADMM iteration limit per QP */
  int32_t warm;          /* 0: every QP starts from d = 0, lambda = 0;  1: lambda (and the
                            line multipliers) carry over from the previous QP */
  double alm_beta;       /* augmented-Lagrangian penalty, as a multiple of max_i Q_ii */
  double alm_tol;        /* line-limit feasibility/complementarity tolerance (default 1e-14; the
                            FP32 sweep uses at least 2e-6) */
  int32_t alm_max_outer; /* multiplier updates per line subproblem */
  int32_t newton_max;    /* projected Newton steps per multiplier update */
  int64_t spin_limit;    /* clock cycles a CTA waits at a device-wide barrier before giving up */
  int32_t rb_period;     /* residual balancing every rb_period iterations (0: fixed rho):   */
  double rb_mu, rb_tau;  /* rho *= rb_tau if r > rb_mu s, rho /= rb_tau if s > rb_mu r; the
                            adapted penalties carry over to the next QP when warm = 1     */
  int32_t line_solver;   /* how the FP64 sweep solves each line subproblem (eq. line_kernel):
                            0 (default): exactly, by the dual active-set method of Goldfarb and
                            Idnani, a subproblem with no feasible point falling back to 1;
                            1: the augmented Lagrangian of Sec. IV-B (alm_* and newton_max above).
                            The FP32 sweep always uses the augmented Lagrangian, whose final
                            solves are refined in twice the working precision */
} admm_options;

typedef struct {
  double mu;             /* l1 merit penalty (Sec. V-A: 1e5) */
  double tol;            /* primal and dual infeasibility tolerance */
  double step_tol;       /* stop when an accepted step's l_inf norm is below this */
  double delta0, delta_max, delta_min; /* trust region: initial, cap, failure threshold */
  int32_t max_sqp;
  int32_t merit_linear;  /* 1 (default): h of the l1 merit function also sums the violations of
                            the linear constraints (power balance, bounds, angle limits), which an
                            inexact ADMM step does not satisfy exactly; 0: nonlinear constraints
                            only, as h is defined in Sec. II-C */
  admm_options admm;
  int32_t soc;           /* 1: second-order correction of a rejected step (named as future work
                            in Sec. II-D): the QP is rebuilt at x
                            with every nonlinear constraint's value taken at x + d (linearised
                            at x), solved, and x + d' passes the ratio test against the
                            original step's model reduction; the history marks the outcome */
  int32_t restore;       /* 1: feasibility restoration (likewise future work in the paper): when
                            the SQP stalls (step or radius below its tolerance) or the primal
                            infeasibility, above 10 tol, fails to fall by a tenth over five
                            iterations, the objective is dropped (weight 0, merit mu h) until
                            the infeasibility is within tol, then the SQP resumes from delta0;
                            a stall during restoration ends with ACOPF_INFEASIBLE */
} sqp_options;

typedef struct {         /* caller-allocated host arrays (NULL to skip one) */
  double *pg, *qg;       /* ngen */
  double *vm, *va;       /* nbus: sqrt(w), theta */
  double *wr, *wi;       /* nbranch */
  double obj;            /* objective at the returned point */
} acopf_solution;

typedef struct {
  double primal;         /* l_inf of all constraint violations (p.u.) */
  double dual;           /* l_inf of the projected Lagrangian gradient / max(1, ||grad f||_inf) */
  double r_inf, s_inf;   /* last ADMM primal and dual residuals */
  double obj;
  double delta;          /* trust-region radius */
  int32_t sqp_iter, admm_iter, accepted;
  int32_t result;        /* acopf_result */
} acopf_residuals;

/* defaults: FP64, angle limits on, device 0; rho 2e4, eps 1e-4, 20000 ADMM
 * iterations, warm 1; mu 1e5, tol 1e-4, delta0 1, delta_max 10, 30 SQP steps */
void acopf_default_options(acopf_options* o);
void admm_default_options(admm_options* o);
void sqp_default_options(sqp_options* o);

const char* acopf_status_string(acopf_status s);
/* message of the handle's last error (or of the last failed acopf_create when h is NULL) */
acopf_status acopf_last_error(acopf_handle h, char* buf, size_t n);

/* Build the device model of ngrids independent instances (Sec. III-A): the
 * branch admittances of the pi model, bus/branch/generator adjacency, and all
 * solver state.  Instances are solved together by every later call.
 * Errors: EINVAL for an index out of range, x <= 0 with r = 0, vmin > vmax,
 * pmin > pmax, qmin > qmax, no (or more than one) reference bus, an isolated
 * bus, ngrids < 1, or more components than 32-bit indices hold (all buses,
 * or 2 x branches + generators, at 2^30 or more); ECUDA without a device. */
acopf_status acopf_create(const acopf_grid* grids, int32_t ngrids, const acopf_options* opt,
                          acopf_handle* out);
acopf_status acopf_destroy(acopf_handle h);

/* Stream (a cudaStream_t) on which all later work is queued; NULL = legacy default. */
acopf_status acopf_set_stream(acopf_handle h, void* cuda_stream);

/* Device memory from the caller's allocator (for example a framework's caching
 * allocator, so that the solver's state counts against its pool).  The paper
 * prescribes no memory management; this is plumbing around Algorithms 1-2.
 *
 * alloc(bytes, ctx) returns a block of at least bytes of device memory on the
 * handle's device, 256-byte aligned, or NULL; release(ptr, ctx) returns a
 * block that alloc gave.  Both are called on the calling thread, only from
 * inside calls on this handle.  The call waits for the handle's stream, then
 * moves every block the handle owns (its model, iterate and ADMM state, the
 * QP's export arrays) into new blocks from alloc, copying their contents, and
 * releases the old ones through the allocator that made them.  Every later
 * device allocation of the handle (export arrays, the scratch of
 * acopf_project_linear, the device copy used by acopf_set_warm_start_device)
 * goes through alloc, and acopf_destroy returns the blocks through release.
 * The library calls release only after waiting for the handle's stream, so
 * the blocks are idle when they are returned.  alloc = release = NULL goes
 * back to cudaMalloc / cudaFree, moving the memory back the same way.  A
 * captured SQP graph (sqp_solve_graph) is dropped and captured again.  The
 * scratch of admm_iterate_static is not the handle's and does not move.
 *
 * Errors: EINVAL for a NULL handle, for only one of alloc and release NULL,
 * or when alloc returned a block that is not 256-byte aligned device memory
 * of the handle's device (that block is released again); ENOMEM when alloc
 * returned NULL.  On any error the handle keeps its memory and its previous
 * allocator. */
acopf_status acopf_set_allocator(acopf_handle h, void* (*alloc)(size_t bytes, void* ctx),
                                 void (*release)(void* ptr, void* ctx), void* ctx);

/* Replace the loads p_i^d, q_i^d of instance inst (Sec. III-A, eq. acopf: the
 * right-hand sides of the bus power balances opfc5-opfc6), in p.u.: host
 * arrays of the instance's nbus.  The copies are queued on the handle's
 * stream: pageable arrays are read during the call, page-locked ones must
 * stay unchanged until the stream has reached the copy.  Takes effect at the
 * next QP build.  Errors: EINVAL for a bad handle, instance or NULL array. */
acopf_status acopf_set_loads(acopf_handle h, int32_t inst, const double* pd, const double* qd);

/* Run Algorithm 1 from a flat start (or from the warm start set below) on
 * every instance until each one converges or stops. */
acopf_status sqp_solve(acopf_handle h, const sqp_options* o);

/* One QP at the current iterate: build it (Alg. 1, eq. QPsub) and solve it by
 * ADMM (Alg. 2); the step and the new multipliers become available through
 * acopf_get_step.  The iterate itself is not changed. */
acopf_status admm_solve_qp(acopf_handle h, double delta, const admm_options* o);

/* sqp_solve with the SQP loop replayed from a CUDA graph: the first iteration
 * runs as individual launches (its ADMM start depends on the warm start); one
 * later iteration -- QP build, ADMM reset, the persistent sweep, step, merit
 * test and trust-region update (the loop of Alg. 1, with Alg. 2) -- is captured once
 * per handle and option set and replayed until every instance has stopped.
 * The host reads the number of running instances from pinned memory after
 * every check_every >= 1 replays; replays after the last instance stopped
 * leave every instance unchanged.  Results equal those of sqp_solve.  If the
 * handle has no stream (acopf_set_stream), an internal stream is used and the
 * device is synchronised first.  Returns when the solve is complete. */
acopf_status sqp_solve_graph(acopf_handle h, const sqp_options* o, int32_t check_every);

/* Linear feasibility projection (Sec. II, eq. linfeas; the initial feasibility step of Alg. 1): the
 * current iterate of every instance -- as last set by acopf_set_iterate or a
 * warm start, or left by the last solve -- is replaced by the nearest point
 * (Euclidean norm over [pg | qg | w | theta | wR | wI]) that satisfies the
 * NLP's linear constraints: the bus power balances (eq. opfc5, opfc6, with the
 * branch flows of eq. acopf_pf, linear in w, wR, wI), the bounds of pg, qg,
 * w and theta (opfc1-4) and theta_ref = 0.  Solved in FP64 by component ADMM
 * (generator box projections, a 4-variable box QP per branch over its wR, wI
 * and copies of its end-bus voltages, closed-form bus updates) with penalty
 * rho > 0 (0.5 suits unit-weight objectives) until the l_inf primal and dual
 * residuals of every instance are <= eps, or max_iter iterations; iters and
 * rs[2] (largest r and s) may be NULL.  The next sqp_solve starts from the
 * projected point.  Allocates scratch for the call; synchronises the stream. */
acopf_status acopf_project_linear(acopf_handle h, double rho, double eps, int32_t max_iter, int32_t* iters,
                                  double* rs);

/* Warm start of instance inst: x0 = NLP point in the layout of
 * acopf_set_iterate (may be NULL; pi is reset to 0), lambda0 = ADMM multipliers:
 * the lam array of acopf_admm_state (8 per branch) followed by its lg array
 * (2 per generator) (may be NULL), rho = per-component penalties
 * (nbranch values, then ngen values; may be NULL).  Used by the next
 * sqp_solve. */
acopf_status acopf_set_warm_start(acopf_handle h, int32_t inst, const double* x0, const double* lambda0,
                                  const double* rho);

/* The iterate of instance inst after the last solve, in the variables of
 * Sec. III-A (eq. acopf): generator dispatch p_g, q_g; bus voltage magnitude
 * sqrt(w_i) and angle theta_i; branch products w^R_ij, w^I_ij; and the
 * objective of eq. acopf at that point (costs per MW, c2 (S p)^2 + c1 S p +
 * c0 with S = base_mva).  out's arrays are caller-owned host arrays (NULL to
 * skip one).  Synchronises the handle's stream.  Errors: EINVAL for a bad
 * handle, instance or out. */
acopf_status acopf_get_solution(acopf_handle h, int32_t inst, acopf_solution* out);
/* Termination measures of instance inst (Alg. 1: the SQP stops when the
 * primal and dual infeasibility of eq. acopf are both within tol, or the
 * accepted step is below step_tol; the columns reported in Tables I-II):
 * primal = l_inf of every constraint violation in p.u.; dual = l_inf of the
 * gradient of the Lagrangian (bus balance multipliers, pi and angle-row
 * multipliers of the last QP, projected at active bounds) over max(1,
 * ||grad f||_inf); r_inf, s_inf = the last ADMM residuals of Sec. IV-B;
 * delta = the trust radius; iteration counts and the acopf_result.
 * Synchronises the handle's stream.  Errors: EINVAL for a bad handle,
 * instance or out. */
acopf_status acopf_get_residuals(acopf_handle h, int32_t inst, acopf_residuals* out);

/* Per-SQP-iteration history of the last sqp_solve for instance inst, 14 values
 * per iteration: objective, primal, dual, ADMM iterations (both passes), r, s,
 * accepted (0/1), trust radius after the update, step norm, actual and
 * predicted merit reduction, penalty factor of the last QP, second-order
 * correction (0 none, 1 corrected step rejected, 2 accepted), restoration
 * phase (0/1).  Writes at most cap rows, returns the number of iterations in
 * *n.  At most ACOPF_HIST_MAX rows are kept. */
#define ACOPF_HIST_MAX 64
acopf_status acopf_get_history(acopf_handle h, int32_t inst, double* out, int32_t cap, int32_t* n);

/* ---- lower-level calls used by the parity tests and the benchmark ------- */

/* NLP point of instance inst, host, n = 2*ngen + 2*nbus + 2*nbranch values in
 * the order [pg | qg | w | theta | wR | wI] (w = v^2), and the multipliers pi
 * of eq. lag (4 per branch: pi11 pi12 pi13 pi14, branch-major; may be NULL). */
acopf_status acopf_set_iterate(acopf_handle h, int32_t inst, const double* x, const double* pi);
acopf_status acopf_get_iterate(acopf_handle h, int32_t inst, double* x, double* pi);

/* Build the QP at the current iterate with trust-region radius delta and
 * penalty rho (every coupling), without solving it. */
acopf_status acopf_build_qp(acopf_handle h, double delta, double rho, int32_t use_angle);

/* Host copies of the QP data of instance inst (any pointer may be NULL):
 * per branch (branch-major): flow 4 (p_ij q_ij p_ji q_ji), H 36 (Hessian of
 * L_ij over z = (w_i, th_i, wR, wI, w_j, th_j), row-major), aR 4, aI 4, bR 1,
 * bI 1, QH 16 (A'HA), gH 4 (A'Hb), F 16 (flow-change rows over
 * dbar = (d_wi, d_thi, d_wj, d_thj)), f0 4, lo 4, hi 4, G 8 (line-limit rows),
 * grhs 2, alo 1, ahi 1; per generator: gen 6 (f', f'', lp, up, lq, uq);
 * per bus: bus 2 (p_i^{d,(k)}, q_i^{d,(k)}). */
typedef struct {
  double *flow, *H, *aR, *aI, *bR, *bI, *QH, *gH, *F, *f0, *lo, *hi, *G, *grhs, *alo, *ahi;
  double *gen, *bus;
} acopf_qp_view;
acopf_status acopf_get_qp(acopf_handle h, int32_t inst, acopf_qp_view* out);

/* ADMM state of instance inst (host, any pointer may be NULL).  Couplings of
 * branch l in the order p_ij q_ij p_ji q_ji w_i(ij) th_i(ij) w_j(ji) th_j(ji):
 * x = line side, z = bus side, lam = multipliers (8 per branch); generators:
 * xg, zg, lg (2 per generator: p, q); bus: zb (d_w, d_theta), nu (power-balance
 * multipliers), 2 per bus; ul: line inequality multipliers (lim_ij, lim_ji,
 * ang_hi, ang_lo), 4 per branch. */
typedef struct {
  double *x, *z, *lam, *xg, *zg, *lg, *zb, *nu, *ul;
} acopf_admm_state;
acopf_status acopf_get_admm_state(acopf_handle h, int32_t inst, acopf_admm_state* out);
acopf_status acopf_set_admm_state(acopf_handle h, int32_t inst, const acopf_admm_state* in);

/* Run exactly n ADMM iterations (n >= 1) of Alg. 2 on the QP last built, from
 * the current ADMM state, ignoring the residual test (o->eps unused). */
acopf_status admm_iterate(acopf_handle h, int32_t n, const admm_options* o);

/* Step d of the last QP (layout of acopf_set_iterate: d_wR, d_wI from eq.
 * elim on the bus values) and the multipliers pi recovered from the line
 * subproblems' KKT conditions (Sec. IV-B), host arrays. */
acopf_status acopf_get_step(acopf_handle h, int32_t inst, double* d, double* pi);

/* Kernel launches issued by this handle since it was created. */
acopf_status acopf_launch_count(acopf_handle h, int64_t* n);

/* Device timing of the ADMM sweep kernel: with on = 1, CUDA events are
 * recorded on the handle's stream around every sweep launch; the accumulated
 * device milliseconds, the number of sweep launches and the ADMM iterations
 * they ran (summed over instances' maximum per launch) are returned by
 * acopf_get_profile, which synchronises the stream.  on = 0 stops recording;
 * acopf_profile always resets the totals. */
acopf_status acopf_profile(acopf_handle h, int32_t on);
acopf_status acopf_get_profile(acopf_handle h, double* sweep_ms, int64_t* sweeps, int64_t* admm_iters);
/* While profiling, CTA 0 of the sweep reads the global timer at each phase
 * boundary: ns[0] its own phase A (generators, branches), ns[1] its wait at
 * the first device-wide barrier, ns[2] its phase B (buses), ns[3] the second
 * barrier plus the residual test; summed over iterations since acopf_profile. */
acopf_status acopf_get_profile_phases(acopf_handle h, double* ns);

/* Launch shape of the ADMM sweep (the autotuner's knobs): threads per CTA
 * (32..256, multiple of 32; 0 keeps), resident CTAs per SM (0 = as many as
 * fit; -1 keeps), and how branch records reach the line solves (-1 keeps):
 * 0 = read in place from global memory every iteration; 1 or 2 (FP32 sweep)
 * = shared-memory tile buffers filled by bulk async copies; 3 = loaded once
 * per sweep into registers, together with every other piece of static data
 * (instance ids, bus-task slots, bus loads), which needs a co-resident grid
 * with one thread per generator or branch and at most two bus tasks per
 * warp, and residual balancing off -- otherwise the sweep runs as with 0;
 * 4 = one thread-block cluster of up to 16 CTAs per instance (enough CTAs
 * for one thread per generator or branch of the largest instance), whose
 * barriers are the cluster's hardware barrier and whose residual maxima are
 * combined in distributed shared memory, so instances never wait on one
 * another (residual balancing off -- otherwise as with 0).  With 3 and 4 the
 * FP64 sweep sizes the grid (or cluster) for one bus task per warp where it
 * still fits: FP64 arithmetic issues at a small fraction of the FP32 rate,
 * so two tasks interleaved in a warp take twice as long as one. */
acopf_status acopf_tune(acopf_handle h, int32_t block_threads, int32_t ctas_per_sm, int32_t sweep_stages);

/* Autotuner of the sweep's launch shape.  If cache_path (may be NULL) names a
 * JSON file holding an entry for this handle's key -- SM count, sweep
 * precision and the binary orders of magnitude of the instance, bus and
 * branch counts -- that shape is applied.  Otherwise the QP at the current
 * iterate is built (delta 1, rho 2e4) and every shape of {64, 128, 192, 224, 256}
 * threads x {as many CTAs per SM as fit, 1} x record access {0, 1, 2, 3, 4}
 * (FP32 sweep; FP64: {0, 3, 4}, see acopf_tune) is timed over iters fixed ADMM iterations with CUDA
 * events; the fastest is applied and written to the cache (other keys are
 * kept).  shape_out (3 ints: threads, CTAs per SM, buffers) and us_per_iter
 * (-1 when taken from the cache) may be NULL.  Resets the ADMM state: call it
 * before setting a warm start. */
acopf_status acopf_autotune(acopf_handle h, const char* cache_path, int32_t iters, int32_t* shape_out,
                            double* us_per_iter);

/* ---- allocation-free sweep (the paper has no counterpart) ----------------
 *
 * admm_iterate_static runs exactly the n ADMM iterations admm_iterate runs,
 * on the QP last built and the current ADMM state of the handle, and then
 * assembles the step, but allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library call.  It is meant for callers that may not allocate
 * device memory while they run -- code working inside a pre-sized memory
 * arena, a real-time loop that cannot afford the implicit device
 * synchronisation an allocation can cause, or a thread that has no access to
 * the application's allocator.  (The handle itself is still created, with its
 * allocations, beforehand by acopf_create.)
 *
 * The sweep kernel's scratch -- its device-wide barrier counters, error flag,
 * per-instance residual slots, finished flags and penalty factors -- lives in
 * one fixed array in device memory, sized for ACOPF_STATIC_MAX_INSTANCES
 * instances (about 180 KB).  Every GPU that loads the library holds that
 * array until the process exits.  The first call on a device looks up the
 * array's device address, so make that first call before any stream capture.
 * All calls share the array and each call clears what must start at zero;
 * calls whose work overlaps on the GPU (two handles on different streams, or
 * two threads) race on it and must be serialised by the caller.
 *
 * An instance whose ADMM residual test passed in the handle's last
 * admm_solve_qp is skipped, as admm_iterate skips it.  The sweep is not timed
 * by acopf_profile.
 *
 * n >= 1 iterations, o as for admm_iterate.  rs and iters are caller-owned
 * DEVICE buffers: rs receives 2*K doubles (r of every instance, then s) of
 * the last iteration, iters K int32 iteration counts, K = number of instances;
 * the same values are copied (device to device) into the handle's own record,
 * so acopf_get_residuals reports them afterwards.  The device address of the
 * fixed array is looked up once per device and assumes that the device's
 * primary context lives until the process exits (no cudaDeviceReset).
 * Errors: EINVAL for a NULL buffer, bad options, or a handle with more than
 * ACOPF_STATIC_MAX_INSTANCES instances; ENOTREADY before any QP was built;
 * ETIMEOUT as admm_iterate; ECUDA if the device address cannot be obtained. */
#define ACOPF_STATIC_MAX_INSTANCES 4096
acopf_status admm_iterate_static(acopf_handle h, int32_t n, const admm_options* o, double* rs, int32_t* iters);

#ifdef __cplusplus
}
#endif
#endif /* ACOPF_H */
