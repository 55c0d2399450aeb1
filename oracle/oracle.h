/*
 * Plain, slow FP64 CPU oracle of the trust-region SQP method for ACOPF whose
 * QP subproblems are solved by component-decomposed ADMM (Li, Schanen, Kim,
 * "GPU-Accelerated Sequential Quadratic Programming Algorithm for Solving
 * ACOPF", arXiv 2310.13143).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the package smoke check and the
 * benchmark's CPU-baseline leg are the only code that may load this library.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * Variable vector x of the NLP (Sec. III-A, eq. acopf), flat, in this order:
 *   [ pg(G) | qg(G) | w(B) | theta(B) | wR(L) | wI(L) ].
 * Line coupling slots (Sec. IV-A, eq. cpl), per branch l with from bus i and
 * to bus j, 8 per branch:
 *   0 p_ij, 1 q_ij, 2 p_ji, 3 q_ji, 4 w_i(ij), 5 theta_i(ij), 6 w_j(ji), 7 theta_j(ji)
 * Generator coupling slots: 0 p_g, 1 q_g.
 * dbar (the line's four independent variables) = (d_wi, d_thi, d_wj, d_thj).
 * The 6-vector z of the per-branch Hessian = (w_i, th_i, wR, wI, w_j, th_j).
 */
#ifndef ACOPF_ORACLE_H
#define ACOPF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t nbus, nbranch, ngen;
  const int32_t* bus_type;  /* 3 = reference bus */
  const double *pd, *qd, *gs, *bs, *vmin, *vmax;
  const int32_t *f, *t;
  const double *r, *x, *b, *rate, *angmin, *angmax, *tap, *shift;
  const int32_t* gbus;
  const double *pmin, *pmax, *qmin, *qmax, *c2, *c1, *c0;
  double base_mva;
} og_grid;

/* QP data of one SQP iteration (eq. QPsub with the elimination eq. elim).
 * Every array is caller-allocated with the stated length. */
typedef struct {
  double *flow;        /* 4L  p_ij q_ij p_ji q_ji at x                 */
  double *H;           /* 36L Hessian of L_ij over z, row-major         */
  double *aR, *aI;     /* 4L  elimination coefficients (eq. elim)       */
  double *bR, *bI;     /* L                                             */
  double *QH;          /* 16L A^T H A                                   */
  double *gH;          /* 4L  A^T H b                                   */
  double *F;           /* 16L flow-change rows over dbar                */
  double *f0;          /* 4L  flow-change offsets                       */
  double *lo, *hi;     /* 4L  box on dbar (bounds and trust region)     */
  double *G;           /* 8L  line-limit rows over dbar                 */
  double *grhs;        /* 2L  line-limit right-hand sides               */
  double *alo, *ahi;   /* L   bounds on d_thi - d_thj (angle limits)    */
  double *gd1, *gd2;   /* G   f'(pg), f''(pg)                           */
  double *glp, *gup, *glq, *guq; /* G  generator step boxes              */
  double *pdk, *qdk;   /* B   power-balance right-hand sides            */
} og_qp;

typedef struct {
  double *xl, *zl, *ll; /* 8L line-side value, bus-side value, multiplier */
  double *xg, *zg, *lg; /* 2G                                             */
  double *rl, *rg;      /* 8L, 2G penalty rho per coupling                */
  double *zb;           /* 2B bus d_w, d_theta                            */
  double *nu;           /* 2B bus power-balance multipliers               */
  double *ul;           /* 4L line inequality multipliers: lim_ij, lim_ji, ang_hi, ang_lo */
  int32_t *aset;        /* L  last active set of each line QP (bit mask, -1 none); may be NULL */
} og_admm_state;

typedef struct {
  double eps;          /* tolerance on l_inf primal and dual ADMM residuals */
  int32_t max_iter;
  int32_t use_angle;   /* angle-difference rows in the line subproblem */
  int32_t rb_period;   /* residual balancing every rb_period iterations (0: off) */
  double rb_mu, rb_tau;
} og_admm_opts;

typedef struct {
  int32_t iters;
  double r_inf, s_inf;
  int32_t line_fail;   /* line QPs whose enumeration found no KKT point */
  int32_t line_reg;    /* line QPs that needed a diagonal shift to be convex */
} og_admm_info;

typedef struct {
  double mu;           /* l1 merit penalty */
  double tol;          /* KKT tolerance (primal and dual) */
  double step_tol;     /* stop when the accepted step is below this */
  double delta0, delta_max, delta_min;
  double rho;          /* ADMM penalty for every coupling */
  int32_t max_sqp;
  int32_t warm_lambda; /* carry ADMM multipliers from one QP to the next */
  og_admm_opts admm;
  int32_t soc;         /* second-order correction of rejected steps */
  int32_t restore;     /* feasibility restoration when the SQP stalls infeasible */
} og_sqp_opts;

typedef struct {
  int32_t iters, accepted, status; /* status: 0 converged, 1 max iter, 2 step too small, 3 non-finite,
                                      5 locally infeasible (restoration stalled) */
  int32_t admm_total;
  double obj, primal, dual, delta;
} og_sqp_info;

/* per-iteration history row: obj primal dual admm_iters r s accept delta dnorm ared pred
 * soc (0 none, 1 corrected step rejected, 2 accepted) restoring (0/1) */
#define OG_HIST_W 13

typedef struct og_model og_model;

int  og_model_create(const og_grid* g, og_model** out);
void og_model_destroy(og_model* m);
int  og_n_vars(const og_model* m);

void og_admittance(const og_model* m, double* Y /* 8L: gii bii gij bij gji bji gjj bjj */);
void og_flat_start(const og_model* m, double* x);
void og_flows(const og_model* m, const double* x, double* flow /* 4L */);
/* constraint values: c11 c12 c13 c14 per branch (4L), balance P,Q per bus (2B) */
void og_constraints(const og_model* m, const double* x, double* c4, double* bal2);
double og_objective(const og_model* m, const double* x);

void og_build(const og_model* m, const double* x, const double* pi, double delta, int use_angle, og_qp* qp);

/* single-component updates (for pins) */
void og_gen_update(double gd1, double gd2, double lp, double up, double lq, double uq,
                   const double z[2], const double lam[2], const double rho[2], double out[2]);
/* exact small QP: min 1/2 x'Qx + c'x, lo<=x<=hi, G x <= grhs (2 rows), alo <= x1-x3 <= ahi.
 * returns 0 ok, 1 regularised, 2 no KKT point found (best candidate returned).
 * mult: 4 values for rows lim0, lim1, ang_hi, ang_lo */
int og_line_qp(const double Q[16], const double c[4], const double lo[4], const double hi[4],
               const double G[8], const double grhs[2], double alo, double ahi, int use_angle,
               double x[4], double mult[4]);
int og_line_qp_hint(const double Q[16], const double c[4], const double lo[4], const double hi[4],
                    const double G[8], const double grhs[2], double alo, double ahi, int use_angle,
                    double x[4], double mult[4], int32_t* hint);
int og_line_update(const og_model* m, const og_qp* qp, int l, const double z[8], const double lam[8],
                   const double rho[8], int use_angle, double x[8], double mult[4], int32_t* hint);
void og_bus_update(const og_model* m, const og_qp* qp, int i, og_admm_state* s, double* rmax, double* smax);

/* keep_lambda: multipliers and penalties carry over */
void og_admm_cold(const og_model* m, og_admm_state* s, double rho, int keep_lambda);
int og_admm(const og_model* m, const og_qp* qp, const og_admm_opts* o, og_admm_state* s, og_admm_info* info);

/* step d (flat, same layout as x) from the ADMM state; new line multipliers pi (4L) */
void og_step(const og_model* m, const og_qp* qp, const og_admm_state* s, const double* x, double* d, double* pi);
/* l1 merit pieces: phi = f + mu h, model reduction pred = q(0)-q(d) */
void og_merit(const og_model* m, const og_qp* qp, const double* x, const double* d, double mu, int use_angle,
              double* phi_x, double* phi_xd, double* pred);
void og_kkt(const og_model* m, const double* x, const double* pi, const double* nu, const double* ul,
            int use_angle, double* primal, double* dual);

int og_sqp(const og_model* m, const og_sqp_opts* o, const double* x0, double* x, double* pi,
           og_sqp_info* info, double* hist, int hist_cap);

void og_build_ex(const og_model* m, const double* x, const double* pi, double delta, int use_angle, const double* dsoc,
                 double fscale, og_qp* qp);
void og_merit_ex(const og_model* m, const og_qp* qp, const double* x, const double* d, double mu, int use_angle,
                 double fscale, double* phi_x, double* phi_xd, double* pred);
/* ratio test and trust-region update of Alg. 1: returns the new radius, *accept 0/1 */
double og_tr_update(const og_sqp_opts* o, double delta, double dnorm, double ared, double pred, int* accept);
/* l1 sum and l_inf maximum of every constraint violation at x (h of the merit function) */
void og_violations(const og_model* m, const double* x, int use_angle, double* h1, double* hinf);

#ifdef __cplusplus
}
#endif
#endif
