/*
 * Plain FP64 CPU oracle: trust-region SQP (Alg. 1) for the rectangular ACOPF
 * (eq. acopf), whose QP subproblem (eq. QPsub, with the elimination of
 * Sec. III-C) is solved by component-decomposed ADMM (Alg. 2: generator
 * eq. gen_kernel, line eq. line_kernel, bus eq. bus_kernel, multipliers
 * eq. multiplier).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Single thread, straight loops over
 * components in the paper's order.  The line subproblem is solved exactly by
 * enumerating active sets (its plain definition: the minimiser of a small
 * convex QP), not by the augmented-Lagrangian iteration the paper uses to
 * reach it.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586476925286766559
#define BIG 1e30

struct og_model {
  og_grid g;
  double* Y;            /* 8L */
  int32_t *end_ptr, *end_idx; /* bus -> incident branch ends (2*l+e) */
  int32_t *gen_ptr, *gen_idx; /* bus -> generators */
  int32_t ref;
  int nvar;
};

/* offsets into the flat variable vector */
#define OPG(m) 0
#define OQG(m) ((m)->g.ngen)
#define OW(m) (2 * (m)->g.ngen)
#define OTH(m) (2 * (m)->g.ngen + (m)->g.nbus)
#define OWR(m) (2 * (m)->g.ngen + 2 * (m)->g.nbus)
#define OWI(m) (2 * (m)->g.ngen + 2 * (m)->g.nbus + (m)->g.nbranch)

static double sq(double a) { return a * a; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }
static double neg(double a) { return a < 0 ? -a : 0.0; } /* [a]^- */

/* ------------------------------------------------------------------ model */
int og_model_create(const og_grid* g, og_model** out) {
  int B = g->nbus, L = g->nbranch, G = g->ngen;
  if (B < 1 || L < 0 || G < 1) return 1;
  og_model* m = (og_model*)calloc(1, sizeof(og_model));
  m->g = *g;
  m->nvar = 2 * G + 2 * B + 2 * L;
  m->ref = -1;
  for (int i = 0; i < B; ++i)
    if (g->bus_type[i] == 3) { m->ref = i; break; }
  if (m->ref < 0) { free(m); return 2; }
  for (int l = 0; l < L; ++l)
    if (g->f[l] < 0 || g->f[l] >= B || g->t[l] < 0 || g->t[l] >= B || g->f[l] == g->t[l]) { free(m); return 3; }
  for (int k = 0; k < G; ++k)
    if (g->gbus[k] < 0 || g->gbus[k] >= B) { free(m); return 3; }

  /* pi-model admittance entries per branch (Sec. III-A: g_ij + j b_ij is the
   * (i,j) entry of the branch admittance matrix) */
  m->Y = (double*)malloc(sizeof(double) * 8 * (L > 0 ? L : 1));
  for (int l = 0; l < L; ++l) {
    double r = g->r[l], x = g->x[l], bc = g->b[l];
    double tap = g->tap ? g->tap[l] : 1.0, sh = g->shift ? g->shift[l] : 0.0;
    if (tap == 0.0) tap = 1.0;
    double den = r * r + x * x;
    double ys_re = r / den, ys_im = -x / den;       /* y = 1/(r + jx) */
    double yff_re = ys_re / (tap * tap), yff_im = (ys_im + 0.5 * bc) / (tap * tap);
    double ytt_re = ys_re, ytt_im = ys_im + 0.5 * bc;
    /* Y_ft = -y / (tap e^{-j sh}) = -(y/tap) e^{j sh};  Y_tf = -(y/tap) e^{-j sh} */
    double cs = cos(sh), sn = sin(sh);
    double a_re = -ys_re / tap, a_im = -ys_im / tap;
    double yft_re = a_re * cs - a_im * sn, yft_im = a_re * sn + a_im * cs;
    double ytf_re = a_re * cs + a_im * sn, ytf_im = -a_re * sn + a_im * cs;
    double* Y = m->Y + 8 * l;
    Y[0] = yff_re; Y[1] = yff_im; /* gii bii */
    Y[2] = yft_re; Y[3] = yft_im; /* gij bij */
    Y[4] = ytf_re; Y[5] = ytf_im; /* gji bji */
    Y[6] = ytt_re; Y[7] = ytt_im; /* gjj bjj */
  }
  /* adjacency: ends and generators per bus */
  m->end_ptr = (int32_t*)calloc(B + 1, sizeof(int32_t));
  m->end_idx = (int32_t*)malloc(sizeof(int32_t) * (2 * L > 0 ? 2 * L : 1));
  for (int l = 0; l < L; ++l) { m->end_ptr[g->f[l] + 1]++; m->end_ptr[g->t[l] + 1]++; }
  for (int i = 0; i < B; ++i) m->end_ptr[i + 1] += m->end_ptr[i];
  int32_t* fill = (int32_t*)calloc(B, sizeof(int32_t));
  for (int l = 0; l < L; ++l) {
    int i = g->f[l], j = g->t[l];
    m->end_idx[m->end_ptr[i] + fill[i]++] = 2 * l;
    m->end_idx[m->end_ptr[j] + fill[j]++] = 2 * l + 1;
  }
  m->gen_ptr = (int32_t*)calloc(B + 1, sizeof(int32_t));
  m->gen_idx = (int32_t*)malloc(sizeof(int32_t) * G);
  for (int k = 0; k < G; ++k) m->gen_ptr[g->gbus[k] + 1]++;
  for (int i = 0; i < B; ++i) m->gen_ptr[i + 1] += m->gen_ptr[i];
  memset(fill, 0, sizeof(int32_t) * B);
  for (int k = 0; k < G; ++k) { int i = g->gbus[k]; m->gen_idx[m->gen_ptr[i] + fill[i]++] = k; }
  free(fill);
  for (int i = 0; i < B; ++i)
    if (m->end_ptr[i + 1] == m->end_ptr[i] && B > 1) { og_model_destroy(m); return 4; } /* isolated bus */
  *out = m;
  return 0;
}

void og_model_destroy(og_model* m) {
  if (!m) return;
  free(m->Y); free(m->end_ptr); free(m->end_idx); free(m->gen_ptr); free(m->gen_idx);
  free(m);
}

int og_n_vars(const og_model* m) { return m->nvar; }

void og_admittance(const og_model* m, double* Y) { memcpy(Y, m->Y, sizeof(double) * 8 * m->g.nbranch); }

/* flat start (the starting point of Alg. 1): w = 1, theta = 0, wR = 1, wI = 0, generators mid-box */
void og_flat_start(const og_model* m, double* x) {
  const og_grid* g = &m->g;
  for (int k = 0; k < g->ngen; ++k) {
    x[OPG(m) + k] = 0.5 * (g->pmin[k] + g->pmax[k]);
    x[OQG(m) + k] = 0.5 * (g->qmin[k] + g->qmax[k]);
  }
  for (int i = 0; i < g->nbus; ++i) { x[OW(m) + i] = 1.0; x[OTH(m) + i] = 0.0; }
  for (int l = 0; l < g->nbranch; ++l) { x[OWR(m) + l] = 1.0; x[OWI(m) + l] = 0.0; }
}

/* eq. acopf_pf */
static void branch_flows(const og_model* m, const double* x, int l, double fl[4]) {
  const double* Y = m->Y + 8 * l;
  int i = m->g.f[l], j = m->g.t[l];
  double wi = x[OW(m) + i], wj = x[OW(m) + j], wr = x[OWR(m) + l], wim = x[OWI(m) + l];
  fl[0] = Y[0] * wi + Y[2] * wr + Y[3] * wim;
  fl[1] = -Y[1] * wi - Y[3] * wr + Y[2] * wim;
  fl[2] = Y[6] * wj + Y[4] * wr - Y[5] * wim;
  fl[3] = -Y[7] * wj - Y[5] * wr - Y[4] * wim;
}

void og_flows(const og_model* m, const double* x, double* flow) {
  for (int l = 0; l < m->g.nbranch; ++l) branch_flows(m, x, l, flow + 4 * l);
}

/* gradient rows of the four flows over z = (w_i, th_i, wR, wI, w_j, th_j) */
static void flow_jac(const double* Y, double J[4][6]) {
  memset(J, 0, sizeof(double) * 24);
  J[0][0] = Y[0];  J[0][2] = Y[2];  J[0][3] = Y[3];
  J[1][0] = -Y[1]; J[1][2] = -Y[3]; J[1][3] = Y[2];
  J[2][4] = Y[6];  J[2][2] = Y[4];  J[2][3] = -Y[5];
  J[3][4] = -Y[7]; J[3][2] = -Y[5]; J[3][3] = -Y[4];
}

/* c11..c14 of eq. acopf (sign as written in eq. lag) and bus balances (opfc5, opfc6) */
void og_constraints(const og_model* m, const double* x, double* c4, double* bal2) {
  const og_grid* g = &m->g;
  int B = g->nbus, L = g->nbranch, G = g->ngen;
  for (int i = 0; i < B; ++i) {
    bal2[2 * i] = -g->pd[i] - g->gs[i] * x[OW(m) + i];
    bal2[2 * i + 1] = -g->qd[i] + g->bs[i] * x[OW(m) + i];
  }
  for (int k = 0; k < G; ++k) {
    bal2[2 * g->gbus[k]] += x[OPG(m) + k];
    bal2[2 * g->gbus[k] + 1] += x[OQG(m) + k];
  }
  for (int l = 0; l < L; ++l) {
    int i = g->f[l], j = g->t[l];
    double fl[4];
    branch_flows(m, x, l, fl);
    double wr = x[OWR(m) + l], wim = x[OWI(m) + l];
    double th = x[OTH(m) + i] - x[OTH(m) + j];
    double s2 = g->rate[l] > 0 ? sq(g->rate[l]) : BIG;
    c4[4 * l + 0] = wr * wr + wim * wim - x[OW(m) + i] * x[OW(m) + j];
    c4[4 * l + 1] = wr * sin(th) - wim * cos(th);
    c4[4 * l + 2] = s2 - fl[0] * fl[0] - fl[1] * fl[1];
    c4[4 * l + 3] = s2 - fl[2] * fl[2] - fl[3] * fl[3];
    bal2[2 * i] -= fl[0];
    bal2[2 * i + 1] -= fl[1];
    bal2[2 * j] -= fl[2];
    bal2[2 * j + 1] -= fl[3];
  }
}

/* f_gi(p) = c2 (S p)^2 + c1 (S p) + c0, S = base MVA (costs are per MW) */
double og_objective(const og_model* m, const double* x) {
  const og_grid* g = &m->g;
  double S = g->base_mva, f = 0.0;
  for (int k = 0; k < g->ngen; ++k) {
    double p = S * x[OPG(m) + k];
    f += g->c2[k] * p * p + g->c1[k] * p + g->c0[k];
  }
  return f;
}

static void box_shift(double lb, double ub, double v, double delta, double* lo, double* hi) {
  double l = dmax(lb - v, -delta), u = dmin(ub - v, delta);
  if (l > u) { /* point further than delta outside its bounds: move the full radius back */
    double mv = (ub - v < -delta) ? -delta : delta;
    l = u = mv;
  }
  *lo = l; *hi = u;
}

/* ------------------------------------------------------------ QP build */
/* Hessian of L_ij (eq. lag) over z = (w_i, th_i, wR, wI, w_j, th_j) */
static void branch_hessian(const double* Y, double thi, double thj, double wr, double wim,
                           const double pi[4], double H[36]) {
  memset(H, 0, sizeof(double) * 36);
  double sn = sin(thi - thj), cs = cos(thi - thj);
  /* c11 = wR^2 + wI^2 - w_i w_j */
  H[2 * 6 + 2] += 2 * pi[0];
  H[3 * 6 + 3] += 2 * pi[0];
  H[0 * 6 + 4] += -pi[0];
  H[4 * 6 + 0] += -pi[0];
  /* c12 = wR sin(th_i - th_j) - wI cos(th_i - th_j) */
  double s0 = -wr * sn + wim * cs; /* second derivative in th_i */
  H[1 * 6 + 1] += pi[1] * s0;
  H[5 * 6 + 5] += pi[1] * s0;
  H[1 * 6 + 5] += -pi[1] * s0;
  H[5 * 6 + 1] += -pi[1] * s0;
  H[2 * 6 + 1] += pi[1] * cs; H[1 * 6 + 2] += pi[1] * cs;
  H[2 * 6 + 5] -= pi[1] * cs; H[5 * 6 + 2] -= pi[1] * cs;
  H[3 * 6 + 1] += pi[1] * sn; H[1 * 6 + 3] += pi[1] * sn;
  H[3 * 6 + 5] -= pi[1] * sn; H[5 * 6 + 3] -= pi[1] * sn;
  /* c13 = s^2 - p_ij^2 - q_ij^2, c14 = s^2 - p_ji^2 - q_ji^2 (flows linear in z) */
  double J[4][6];
  flow_jac(Y, J);
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      H[a * 6 + b] += -2.0 * pi[2] * (J[0][a] * J[0][b] + J[1][a] * J[1][b]);
      H[a * 6 + b] += -2.0 * pi[3] * (J[2][a] * J[2][b] + J[3][a] * J[3][b]);
    }
}

/* The QP of eq. QPsub at x.  With dsoc (a step of the same layout as x) it is
 * the second-order correction QP of that step: every nonlinear constraint
 * value c(x) in the linearisation is replaced by c(x + d) - grad c(x)' d, so
 * that the linearised constraints at the corrected step d' read
 * c(x + d) + grad c(x)' (d' - d) (the value at x + d, linearised at x).  For
 * the quadratic opfc11 and the line limits the difference is the step's exact
 * second-order term; opfc12 is evaluated at x + d.  fscale weights the
 * objective (0: the feasibility-restoration QP, which minimises the
 * violation alone). */
void og_build_ex(const og_model* m, const double* x, const double* pi, double delta, int use_angle, const double* dsoc,
                 double fscale, og_qp* qp) {
  const og_grid* g = &m->g;
  int B = g->nbus, L = g->nbranch, G = g->ngen;
  double S = g->base_mva;
  /* generators: gradient and curvature of the cost, shifted boxes (opfqpc1-2 with the trust region) */
  for (int k = 0; k < G; ++k) {
    double p = x[OPG(m) + k], q = x[OQG(m) + k];
    qp->gd1[k] = fscale * (2.0 * g->c2[k] * S * S * p + g->c1[k] * S);
    qp->gd2[k] = fscale * 2.0 * g->c2[k] * S * S;
    box_shift(g->pmin[k], g->pmax[k], p, delta, &qp->glp[k], &qp->gup[k]);
    box_shift(g->qmin[k], g->qmax[k], q, delta, &qp->glq[k], &qp->guq[k]);
  }
  /* buses: p_i^{d,(k)}, q_i^{d,(k)} */
  for (int i = 0; i < B; ++i) {
    qp->pdk[i] = g->pd[i] + g->gs[i] * x[OW(m) + i];
    qp->qdk[i] = g->qd[i] - g->bs[i] * x[OW(m) + i];
  }
  for (int k = 0; k < G; ++k) {
    qp->pdk[g->gbus[k]] -= x[OPG(m) + k];
    qp->qdk[g->gbus[k]] -= x[OQG(m) + k];
  }
  for (int l = 0; l < L; ++l) {
    const double* Y = m->Y + 8 * l;
    int i = g->f[l], j = g->t[l];
    double wi = x[OW(m) + i], wj = x[OW(m) + j], thi = x[OTH(m) + i], thj = x[OTH(m) + j];
    double wr = x[OWR(m) + l], wim = x[OWI(m) + l];
    double* fl = qp->flow + 4 * l;
    branch_flows(m, x, l, fl);
    qp->pdk[i] += fl[0]; qp->qdk[i] += fl[1];
    qp->pdk[j] += fl[2]; qp->qdk[j] += fl[3];

    double* H = qp->H + 36 * l;
    branch_hessian(Y, thi, thj, wr, wim, pi + 4 * l, H);

    /* elimination (eq. elim): solve the linearised opfc11 and opfc12 for (d_wR, d_wI) */
    double sn = sin(thi - thj), cs = cos(thi - thj);
    double D = wr * cs + wim * sn;
    double R0 = wi * wj - wr * wr - wim * wim;
    double S0 = -wr * sn + wim * cs;
    if (dsoc) {
      double dwi = dsoc[OW(m) + i], dwj = dsoc[OW(m) + j];
      double dth = dsoc[OTH(m) + i] - dsoc[OTH(m) + j];
      double dwr = dsoc[OWR(m) + l], dwim = dsoc[OWI(m) + l];
      R0 += dwi * dwj - dwr * dwr - dwim * dwim;
      double s1 = sin(thi - thj + dth), c1 = cos(thi - thj + dth);
      S0 = (-(wr + dwr) * s1 + (wim + dwim) * c1) - (-sn * dwr + cs * dwim - D * dth);
    }
    double* aR = qp->aR + 4 * l;
    double* aI = qp->aI + 4 * l;
    aR[0] = cs * wj / (2 * D); aR[1] = -wim; aR[2] = cs * wi / (2 * D); aR[3] = wim;
    aI[0] = sn * wj / (2 * D); aI[1] = wr;   aI[2] = sn * wi / (2 * D); aI[3] = -wr;
    qp->bR[l] = (cs * R0 + 2 * wim * S0) / (2 * D);
    qp->bI[l] = (sn * R0 - 2 * wr * S0) / (2 * D);

    /* A (6x4) and b (6) of the line subproblem */
    double A[6][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {aR[0], aR[1], aR[2], aR[3]},
                      {aI[0], aI[1], aI[2], aI[3]}, {0, 0, 1, 0}, {0, 0, 0, 1}};
    double bb[6] = {0, 0, qp->bR[l], qp->bI[l], 0, 0};
    double HA[6][4];
    for (int a = 0; a < 6; ++a)
      for (int c = 0; c < 4; ++c) {
        double s = 0;
        for (int k = 0; k < 6; ++k) s += H[a * 6 + k] * A[k][c];
        HA[a][c] = s;
      }
    for (int r = 0; r < 4; ++r) {
      for (int c = 0; c < 4; ++c) {
        double s = 0;
        for (int k = 0; k < 6; ++k) s += A[k][r] * HA[k][c];
        qp->QH[16 * l + 4 * r + c] = s;
      }
      double s = 0;
      for (int k = 0; k < 6; ++k) s += bb[k] * HA[k][r];
      qp->gH[4 * l + r] = s;
    }
    /* flow changes as affine maps of dbar (eq. acopf_qppf with eq. elim) */
    double J[4][6];
    flow_jac(Y, J);
    for (int r = 0; r < 4; ++r) {
      double s0 = 0;
      for (int k = 0; k < 6; ++k) s0 += J[r][k] * bb[k];
      qp->f0[4 * l + r] = s0;
      for (int c = 0; c < 4; ++c) {
        double s = 0;
        for (int k = 0; k < 6; ++k) s += J[r][k] * A[k][c];
        qp->F[16 * l + 4 * r + c] = s;
      }
    }
    /* boxes on dbar = (d_wi, d_thi, d_wj, d_thj); the reference angle stays 0 */
    double* lo = qp->lo + 4 * l;
    double* hi = qp->hi + 4 * l;
    box_shift(sq(g->vmin[i]), sq(g->vmax[i]), wi, delta, &lo[0], &hi[0]);
    box_shift(-TWO_PI, TWO_PI, thi, delta, &lo[1], &hi[1]);
    box_shift(sq(g->vmin[j]), sq(g->vmax[j]), wj, delta, &lo[2], &hi[2]);
    box_shift(-TWO_PI, TWO_PI, thj, delta, &lo[3], &hi[3]);
    if (i == m->ref) lo[1] = hi[1] = -thi;
    if (j == m->ref) lo[3] = hi[3] = -thj;
    /* line limits (line_kernel_1, line_kernel_2) as rows over dbar */
    double s2 = g->rate[l] > 0 ? sq(g->rate[l]) : -1.0;
    for (int e = 0; e < 2; ++e) {
      double p = fl[2 * e], q = fl[2 * e + 1];
      double* Gr = qp->G + 8 * l + 4 * e;
      if (s2 < 0) {
        for (int c = 0; c < 4; ++c) Gr[c] = 0.0;
        qp->grhs[2 * l + e] = BIG;
        continue;
      }
      for (int c = 0; c < 4; ++c) Gr[c] = 2 * p * qp->F[16 * l + 4 * (2 * e) + c] + 2 * q * qp->F[16 * l + 4 * (2 * e + 1) + c];
      double lim = s2 - p * p - q * q;
      if (dsoc) {  /* the flows are linear in (w, wR, wI): their change under d is exact */
        double dz[6] = {dsoc[OW(m) + i], dsoc[OTH(m) + i], dsoc[OWR(m) + l], dsoc[OWI(m) + l], dsoc[OW(m) + j],
                        dsoc[OTH(m) + j]};
        double dp = 0, dq = 0;
        for (int k = 0; k < 6; ++k) { dp += J[2 * e][k] * dz[k]; dq += J[2 * e + 1][k] * dz[k]; }
        lim -= dp * dp + dq * dq;
      }
      qp->grhs[2 * l + e] = lim - 2 * p * qp->f0[4 * l + 2 * e] - 2 * q * qp->f0[4 * l + 2 * e + 1];
    }
    /* angle-difference limits on th_i - th_j */
    if (use_angle && g->angmin[l] > -TWO_PI && g->angmax[l] < TWO_PI) {
      qp->alo[l] = g->angmin[l] - (thi - thj);
      qp->ahi[l] = g->angmax[l] - (thi - thj);
    } else {
      qp->alo[l] = -BIG;
      qp->ahi[l] = BIG;
    }
  }
}

void og_build(const og_model* m, const double* x, const double* pi, double delta, int use_angle, og_qp* qp) {
  og_build_ex(m, x, pi, delta, use_angle, NULL, 1.0, qp);
}

/* ------------------------------------------------------- generator update */
/* eq. gen_kernel: x* = clamp(Q^{-1} c) with Q = f''+rho (p) or rho (q) */
void og_gen_update(double gd1, double gd2, double lp, double up, double lq, double uq,
                   const double z[2], const double lam[2], const double rho[2], double out[2]) {
  double p = (rho[0] * z[0] - lam[0] - gd1) / (gd2 + rho[0]);
  double q = (rho[1] * z[1] - lam[1]) / rho[1];
  out[0] = dmax(lp, dmin(up, p));
  out[1] = dmax(lq, dmin(uq, q));
}

/* ------------------------------------------------------- small exact QP */
/* Dense Gaussian elimination with partial pivoting; returns 0 when singular. */
static int gauss_solve(int n, double* M, double* rhs) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = fabs(M[c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r * n + c]) > best) { best = fabs(M[r * n + c]); p = r; }
    if (!(best > 1e-300)) return 0;
    if (p != c) {
      for (int k = 0; k < n; ++k) { double t = M[c * n + k]; M[c * n + k] = M[p * n + k]; M[p * n + k] = t; }
      double t = rhs[c]; rhs[c] = rhs[p]; rhs[p] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = M[r * n + c] / M[c * n + c];
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) M[r * n + k] -= f * M[c * n + k];
      rhs[r] -= f * rhs[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = rhs[r];
    for (int k = r + 1; k < n; ++k) s -= M[r * n + k] * rhs[k];
    rhs[r] = s / M[r * n + r];
  }
  return 1;
}

static int chol4_ok(const double Q[16]) {
  double Lm[16] = {0};
  for (int j = 0; j < 4; ++j) {
    double s = Q[j * 4 + j];
    for (int k = 0; k < j; ++k) s -= Lm[j * 4 + k] * Lm[j * 4 + k];
    if (!(s > 0)) return 0;
    Lm[j * 4 + j] = sqrt(s);
    for (int i = j + 1; i < 4; ++i) {
      double t = Q[i * 4 + j];
      for (int k = 0; k < j; ++k) t -= Lm[i * 4 + k] * Lm[j * 4 + k];
      Lm[i * 4 + j] = t / Lm[j * 4 + j];
    }
  }
  return 1;
}

/* Rows of the line subproblem's inequalities, a_k' x <= b_k:
 *   0..3 lower bounds (-e_v), 4..7 upper bounds (e_v), 8..9 line limits,
 *   10 angle upper (x1 - x3 <= ahi), 11 angle lower (-(x1 - x3) <= -alo). */
#define NROW 12
typedef struct {
  double Q[16], c[4], A[NROW][4], b[NROW];
  double qsc, csc;
} lqp;

/* Solve the equality-constrained QP on working set W and test it for the KKT
 * conditions of the inequality QP.  Returns -1 if the KKT matrix is singular,
 * else the badness (0 = valid KKT point); W[0..nmust) are equalities. */
static double kkt_try(const lqp* P, const int* W, int nw, int nmust, double x[4], double multW[4]) {
  int n = 4 + nw;
  double M[64], rhs[8];
  memset(M, 0, sizeof(M));
  for (int r = 0; r < 4; ++r) {
    for (int cc = 0; cc < 4; ++cc) M[r * n + cc] = P->Q[4 * r + cc];
    for (int k = 0; k < nw; ++k) M[r * n + 4 + k] = P->A[W[k]][r];
    rhs[r] = -P->c[r];
  }
  for (int k = 0; k < nw; ++k) {
    for (int cc = 0; cc < 4; ++cc) M[(4 + k) * n + cc] = P->A[W[k]][cc];
    rhs[4 + k] = P->b[W[k]];
  }
  if (!gauss_solve(n, M, rhs)) return -1.0;
  for (int k = 0; k < 4; ++k) x[k] = rhs[k];
  for (int k = 0; k < nw; ++k) multW[k] = rhs[4 + k];
  double xs = fabs(x[0]) + fabs(x[1]) + fabs(x[2]) + fabs(x[3]);
  double viol = 0, dviol = 0;
  int inW[NROW] = {0};
  for (int k = 0; k < nw; ++k) inW[W[k]] = 1;
  /* a KKT point satisfies its working set's rows as equalities; a (nearly)
   * singular system can return a point that does not, which is no solution */
  for (int k = 0; k < 4 + nw; ++k)
    if (!isfinite(rhs[k])) return -1.0;
  for (int k = 0; k < nw; ++k) {
    const double* a = P->A[W[k]];
    double an = fabs(a[0]) + fabs(a[1]) + fabs(a[2]) + fabs(a[3]);
    double ax = a[0] * x[0] + a[1] * x[1] + a[2] * x[2] + a[3] * x[3];
    if (fabs(ax - P->b[W[k]]) > 1e-9 * (1.0 + fabs(P->b[W[k]]) + an * xs)) return -1.0;
  }
  for (int k = 0; k < NROW; ++k) {
    if (inW[k] || P->b[k] >= 0.5 * BIG) continue;
    double ax = P->A[k][0] * x[0] + P->A[k][1] * x[1] + P->A[k][2] * x[2] + P->A[k][3] * x[3];
    double an = fabs(P->A[k][0]) + fabs(P->A[k][1]) + fabs(P->A[k][2]) + fabs(P->A[k][3]);
    double tol = 1e-9 * (1.0 + fabs(P->b[k]) + an * xs);
    if (ax - P->b[k] > tol) viol = dmax(viol, (ax - P->b[k]) / (1.0 + fabs(P->b[k]) + an * xs));
  }
  for (int k = nmust; k < nw; ++k) {
    double an = fabs(P->A[W[k]][0]) + fabs(P->A[W[k]][1]) + fabs(P->A[W[k]][2]) + fabs(P->A[W[k]][3]);
    double tol = 1e-9 * (1.0 + P->csc + P->qsc * xs) / an;
    if (rhs[4 + k] < -tol) dviol = dmax(dviol, -rhs[4 + k] * an / (1.0 + P->csc + P->qsc * xs));
  }
  return viol + dviol;
}

static int pair_conflict(const int* W, int nw) {
  for (int a = 0; a < nw; ++a)
    for (int bq = a + 1; bq < nw; ++bq) {
      int ra = W[a], rb = W[bq];
      if ((ra < 8 && rb < 8 && (ra % 4) == (rb % 4)) || (ra >= 10 && rb >= 10)) return 1;
    }
  return 0;
}

/* Exact minimiser of the (strictly convex) line QP.  Its KKT point is unique,
 * so the first working set that passes the KKT test is the answer; the set
 * found at the previous call (*hint, a bit mask over the 12 rows) is tried
 * first, then all sets in order of size. */
int og_line_qp_hint(const double Qin[16], const double c[4], const double lo[4], const double hi[4],
                    const double Gm[8], const double grhs[2], double alo, double ahi, int use_angle,
                    double xout[4], double mult[4], int32_t* hint) {
  lqp P;
  memcpy(P.Q, Qin, sizeof(P.Q));
  int reg = 0;
  /* nonconvex case: shift the diagonal until Q is positive definite */
  if (!chol4_ok(P.Q)) {
    double qmax = 0;
    for (int k = 0; k < 4; ++k) qmax = dmax(qmax, fabs(P.Q[5 * k]));
    double dl = 1e-8 * (qmax > 0 ? qmax : 1.0);
    while (!chol4_ok(P.Q)) {
      for (int k = 0; k < 4; ++k) P.Q[5 * k] = Qin[5 * k] + dl;
      dl *= 2;
    }
    reg = 1;
  }
  memcpy(P.c, c, sizeof(P.c));
  memset(P.A, 0, sizeof(P.A));
  for (int v = 0; v < 4; ++v) {
    P.A[v][v] = -1; P.b[v] = -lo[v];
    P.A[4 + v][v] = 1; P.b[4 + v] = hi[v];
  }
  for (int e = 0; e < 2; ++e) {
    for (int k = 0; k < 4; ++k) P.A[8 + e][k] = Gm[4 * e + k];
    P.b[8 + e] = grhs[e];
  }
  P.A[10][1] = 1; P.A[10][3] = -1; P.b[10] = use_angle ? ahi : BIG;
  P.A[11][1] = -1; P.A[11][3] = 1; P.b[11] = use_angle ? -alo : BIG;
  /* rows that can never be active: disabled limits; fixed variables use the lower row as an equality */
  int must[NROW] = {0}, active_ok[NROW];
  for (int k = 0; k < NROW; ++k) active_ok[k] = P.b[k] < 0.5 * BIG;
  for (int e = 0; e < 2; ++e) {
    double nrm = fabs(Gm[4 * e]) + fabs(Gm[4 * e + 1]) + fabs(Gm[4 * e + 2]) + fabs(Gm[4 * e + 3]);
    if (nrm == 0.0) active_ok[8 + e] = 0;
  }
  for (int v = 0; v < 4; ++v)
    if (lo[v] == hi[v]) { must[v] = 1; active_ok[4 + v] = 0; }
  P.qsc = 0; P.csc = 0;
  for (int k = 0; k < 16; ++k) P.qsc = dmax(P.qsc, fabs(P.Q[k]));
  for (int k = 0; k < 4; ++k) P.csc = dmax(P.csc, fabs(c[k]));

  int nmust = 0, idx_must[4];
  for (int k = 0; k < NROW; ++k)
    if (must[k]) idx_must[nmust++] = k;
  int opt[NROW], nopt = 0;
  for (int k = 0; k < NROW; ++k)
    if (active_ok[k] && !must[k]) opt[nopt++] = k;

  double best_x[4] = {0}, best_mult[NROW] = {0};
  double best_bad = BIG, xv[4], mw[4];
  int found = 0, best_mask = 0;
  int maxs = 4 - nmust;

  /* 1) the previous working set */
  if (hint && *hint >= 0) {
    int W[4], nw = 0, ok = 1;
    for (int k = 0; k < nmust; ++k) W[nw++] = idx_must[k];
    for (int k = 0; k < NROW && ok; ++k)
      if ((*hint >> k) & 1) {
        if (!active_ok[k] || must[k] || nw >= 4) ok = 0;
        else W[nw++] = k;
      }
    if (ok && !pair_conflict(W, nw)) {
      double bad = kkt_try(&P, W, nw, nmust, xv, mw);
      if (bad == 0.0) {
        memcpy(best_x, xv, sizeof(xv));
        for (int k = 0; k < nw; ++k) best_mult[W[k]] = mw[k];
        found = 1;
        best_mask = *hint;
      }
    }
  }
  /* 2) every working set, smallest first */
  for (int s = 0; s <= maxs && !found; ++s) {
    if (s > nopt) break;
    int comb[4];
    for (int k = 0; k < s; ++k) comb[k] = k;
    while (1) {
      int W[4], nw = 0, mask = 0;
      for (int k = 0; k < nmust; ++k) W[nw++] = idx_must[k];
      for (int k = 0; k < s; ++k) { W[nw++] = opt[comb[k]]; mask |= 1 << opt[comb[k]]; }
      if (!pair_conflict(W, nw)) {
        double bad = kkt_try(&P, W, nw, nmust, xv, mw);
        if (bad >= 0.0 && bad < best_bad) {
          best_bad = bad;
          memcpy(best_x, xv, sizeof(xv));
          for (int k = 0; k < NROW; ++k) best_mult[k] = 0;
          for (int k = 0; k < nw; ++k) best_mult[W[k]] = mw[k];
          best_mask = mask;
          if (bad == 0.0) { found = 1; break; }
        }
      }
      if (s == 0) break;
      int k = s - 1;
      while (k >= 0 && comb[k] == nopt - s + k) --k;
      if (k < 0) break;
      comb[k]++;
      for (int q = k + 1; q < s; ++q) comb[q] = comb[q - 1] + 1;
    }
  }
  if (hint) *hint = best_mask;
  memcpy(xout, best_x, sizeof(best_x));
  mult[0] = best_mult[8];
  mult[1] = best_mult[9];
  mult[2] = best_mult[10];
  mult[3] = best_mult[11];
  if (!found) return 2;
  return reg;
}

int og_line_qp(const double Q[16], const double c[4], const double lo[4], const double hi[4],
               const double Gm[8], const double grhs[2], double alo, double ahi, int use_angle,
               double xout[4], double mult[4]) {
  return og_line_qp_hint(Q, c, lo, hi, Gm, grhs, alo, ahi, use_angle, xout, mult, NULL);
}

/* eq. line_kernel: assemble the 4-variable QP of branch l and solve it */
int og_line_update(const og_model* m, const og_qp* qp, int l, const double z[8], const double lam[8],
                   const double rho[8], int use_angle, double xo[8], double mult[4], int32_t* hint) {
  (void)m;
  const double* F = qp->F + 16 * l;
  const double* f0 = qp->f0 + 4 * l;
  double Q[16], c[4];
  memcpy(Q, qp->QH + 16 * l, sizeof(Q));
  memcpy(c, qp->gH + 4 * l, sizeof(c));
  for (int s = 0; s < 4; ++s) {
    /* lambda_f (d_f - z_f) + rho_f/2 (d_f - z_f)^2 with d_f = F_s dbar + f0_s */
    double coef = lam[s] + rho[s] * (f0[s] - z[s]);
    for (int a = 0; a < 4; ++a) {
      c[a] += coef * F[4 * s + a];
      for (int b2 = 0; b2 < 4; ++b2) Q[4 * a + b2] += rho[s] * F[4 * s + a] * F[4 * s + b2];
    }
  }
  for (int v = 0; v < 4; ++v) {
    /* lambda_v (dbar_v - z_v) + rho_v/2 (dbar_v - z_v)^2 */
    Q[5 * v] += rho[4 + v];
    c[v] += lam[4 + v] - rho[4 + v] * z[4 + v];
  }
  double xb[4];
  int rc = og_line_qp_hint(Q, c, qp->lo + 4 * l, qp->hi + 4 * l, qp->G + 8 * l, qp->grhs + 2 * l,
                           qp->alo[l], qp->ahi[l], use_angle, xb, mult, hint);
  for (int s = 0; s < 4; ++s)
    xo[s] = F[4 * s] * xb[0] + F[4 * s + 1] * xb[1] + F[4 * s + 2] * xb[2] + F[4 * s + 3] * xb[3] + f0[s];
  for (int v = 0; v < 4; ++v) xo[4 + v] = xb[v];
  return rc;
}

/* ------------------------------------------------------------ bus update */
/* eq. bus_kernel: min 1/2 x'Qx - c'x s.t. Ax = b, with Q = diag(rho),
 * c = lambda + rho * (component value); lambda* = (AQ^-1A')^-1 (AQ^-1 c - b),
 * x* = Q^-1 (c - A' lambda*).  Rows: active and reactive power balance. */
void og_bus_update(const og_model* m, const og_qp* qp, int i, og_admm_state* s, double* rmax, double* smax) {
  const og_grid* g = &m->g;
  double M11 = 0, M22 = 0, M12 = 0, v1 = 0, v2 = 0;
  double Qw = 0, cw = 0, Qt = 0, ct = 0;
  for (int k = m->gen_ptr[i]; k < m->gen_ptr[i + 1]; ++k) {
    int gk = m->gen_idx[k];
    double rp = s->rg[2 * gk], rq = s->rg[2 * gk + 1];
    double cp = s->lg[2 * gk] + rp * s->xg[2 * gk];
    double cq = s->lg[2 * gk + 1] + rq * s->xg[2 * gk + 1];
    M11 += 1.0 / rp; M22 += 1.0 / rq;
    v1 += cp / rp; v2 += cq / rq;
  }
  for (int k = m->end_ptr[i]; k < m->end_ptr[i + 1]; ++k) {
    int le = m->end_idx[k], l = le >> 1, e = le & 1;
    int sp = 2 * e, sq_ = 2 * e + 1, sw = 4 + 2 * e, st = 5 + 2 * e;
    double rp = s->rl[8 * l + sp], rq = s->rl[8 * l + sq_];
    double cp = s->ll[8 * l + sp] + rp * s->xl[8 * l + sp];
    double cq = s->ll[8 * l + sq_] + rq * s->xl[8 * l + sq_];
    M11 += 1.0 / rp; M22 += 1.0 / rq;
    v1 -= cp / rp; v2 -= cq / rq;
    Qw += s->rl[8 * l + sw]; cw += s->ll[8 * l + sw] + s->rl[8 * l + sw] * s->xl[8 * l + sw];
    Qt += s->rl[8 * l + st]; ct += s->ll[8 * l + st] + s->rl[8 * l + st] * s->xl[8 * l + st];
  }
  double gsh = g->gs[i], bsh = g->bs[i];
  M11 += gsh * gsh / Qw;
  M22 += bsh * bsh / Qw;
  M12 = -gsh * bsh / Qw;
  v1 += -gsh * cw / Qw - qp->pdk[i];
  v2 += bsh * cw / Qw - qp->qdk[i];
  double det = M11 * M22 - M12 * M12;
  double nu1 = (M22 * v1 - M12 * v2) / det;
  double nu2 = (M11 * v2 - M12 * v1) / det;
  s->nu[2 * i] = nu1;
  s->nu[2 * i + 1] = nu2;
  double rm = *rmax, sm = *smax;
  for (int k = m->gen_ptr[i]; k < m->gen_ptr[i + 1]; ++k) {
    int gk = m->gen_idx[k];
    for (int a = 0; a < 2; ++a) {
      double rr = s->rg[2 * gk + a];
      double cc = s->lg[2 * gk + a] + rr * s->xg[2 * gk + a];
      double znew = (cc - (a == 0 ? nu1 : nu2)) / rr;
      sm = dmax(sm, fabs(rr * (znew - s->zg[2 * gk + a])));
      s->zg[2 * gk + a] = znew;
      rm = dmax(rm, fabs(s->xg[2 * gk + a] - znew));
    }
  }
  double dw = (cw + gsh * nu1 - bsh * nu2) / Qw;
  double dth = (i == m->ref) ? 0.0 : ct / Qt;
  for (int k = m->end_ptr[i]; k < m->end_ptr[i + 1]; ++k) {
    int le = m->end_idx[k], l = le >> 1, e = le & 1;
    for (int a = 0; a < 2; ++a) {
      int sl = 2 * e + a;
      double rr = s->rl[8 * l + sl];
      double cc = s->ll[8 * l + sl] + rr * s->xl[8 * l + sl];
      double znew = (cc + (a == 0 ? nu1 : nu2)) / rr;
      sm = dmax(sm, fabs(rr * (znew - s->zl[8 * l + sl])));
      s->zl[8 * l + sl] = znew;
      rm = dmax(rm, fabs(s->xl[8 * l + sl] - znew));
    }
    int sw = 4 + 2 * e, st = 5 + 2 * e;
    sm = dmax(sm, fabs(s->rl[8 * l + sw] * (dw - s->zl[8 * l + sw])));
    sm = dmax(sm, fabs(s->rl[8 * l + st] * (dth - s->zl[8 * l + st])));
    s->zl[8 * l + sw] = dw;
    s->zl[8 * l + st] = dth;
    rm = dmax(rm, fabs(s->xl[8 * l + sw] - dw));
    rm = dmax(rm, fabs(s->xl[8 * l + st] - dth));
  }
  s->zb[2 * i] = dw;
  s->zb[2 * i + 1] = dth;
  *rmax = rm;
  *smax = sm;
}

/* ---------------------------------------------------------------- ADMM */
void og_admm_cold(const og_model* m, og_admm_state* s, double rho, int keep_lambda) {
  int B = m->g.nbus, L = m->g.nbranch, G = m->g.ngen;
  for (int k = 0; k < 8 * L; ++k) {
    s->xl[k] = 0; s->zl[k] = 0;
    if (!keep_lambda) { s->ll[k] = 0; s->rl[k] = rho; }
  }
  for (int k = 0; k < 2 * G; ++k) {
    s->xg[k] = 0; s->zg[k] = 0;
    if (!keep_lambda) { s->lg[k] = 0; s->rg[k] = rho; }
  }
  for (int k = 0; k < 2 * B; ++k) { s->zb[k] = 0; s->nu[k] = 0; }
  if (s->aset)
    for (int k = 0; k < L; ++k) s->aset[k] = -1;
  if (!keep_lambda)
    for (int k = 0; k < 4 * L; ++k) s->ul[k] = 0;
}

/* Alg. 2: generators, lines, buses, multipliers; stop on l_inf residuals */
int og_admm(const og_model* m, const og_qp* qp, const og_admm_opts* o, og_admm_state* s, og_admm_info* info) {
  int B = m->g.nbus, L = m->g.nbranch, G = m->g.ngen;
  int it = 0, nfail = 0, nreg = 0;
  double rmax = 0, smax = 0;
  for (it = 1; it <= o->max_iter; ++it) {
    for (int k = 0; k < G; ++k)
      og_gen_update(qp->gd1[k], qp->gd2[k], qp->glp[k], qp->gup[k], qp->glq[k], qp->guq[k],
                    s->zg + 2 * k, s->lg + 2 * k, s->rg + 2 * k, s->xg + 2 * k);
    for (int l = 0; l < L; ++l) {
      int rc = og_line_update(m, qp, l, s->zl + 8 * l, s->ll + 8 * l, s->rl + 8 * l, o->use_angle,
                              s->xl + 8 * l, s->ul + 4 * l, s->aset ? s->aset + l : NULL);
      if (rc == 2) nfail++;
      if (rc == 1) nreg++;
    }
    rmax = 0; smax = 0;
    for (int i = 0; i < B; ++i) og_bus_update(m, qp, i, s, &rmax, &smax);
    /* eq. multiplier */
    for (int k = 0; k < 8 * L; ++k) s->ll[k] += s->rl[k] * (s->xl[k] - s->zl[k]);
    for (int k = 0; k < 2 * G; ++k) s->lg[k] += s->rg[k] * (s->xg[k] - s->zg[k]);
    if (rmax <= o->eps && smax <= o->eps) break;
    /* residual balancing (Boyd et al., Sec. 3.4.1): scale every penalty of the
     * instance; lambda is not scaled, so nothing else changes */
    if (o->rb_period > 0 && it % o->rb_period == 0) {
      double f = 1.0;
      if (rmax > o->rb_mu * smax) f = o->rb_tau;
      else if (smax > o->rb_mu * rmax) f = 1.0 / o->rb_tau;
      if (f != 1.0) {
        for (int k = 0; k < 8 * L; ++k) s->rl[k] *= f;
        for (int k = 0; k < 2 * G; ++k) s->rg[k] *= f;
      }
    }
  }
  if (it > o->max_iter) it = o->max_iter;
  info->iters = it;
  info->r_inf = rmax;
  info->s_inf = smax;
  info->line_fail = nfail;
  info->line_reg = nreg;
  return (rmax <= o->eps && smax <= o->eps) ? 0 : 1;
}

/* ------------------------------------------------------ step and multipliers */
void og_step(const og_model* m, const og_qp* qp, const og_admm_state* s, const double* x, double* d, double* pi) {
  const og_grid* g = &m->g;
  int B = g->nbus, L = g->nbranch, G = g->ngen;
  for (int k = 0; k < G; ++k) { d[OPG(m) + k] = s->xg[2 * k]; d[OQG(m) + k] = s->xg[2 * k + 1]; }
  for (int i = 0; i < B; ++i) { d[OW(m) + i] = s->zb[2 * i]; d[OTH(m) + i] = s->zb[2 * i + 1]; }
  for (int l = 0; l < L; ++l) {
    int i = g->f[l], j = g->t[l];
    double db[4] = {s->zb[2 * i], s->zb[2 * i + 1], s->zb[2 * j], s->zb[2 * j + 1]};
    const double* aR = qp->aR + 4 * l;
    const double* aI = qp->aI + 4 * l;
    d[OWR(m) + l] = aR[0] * db[0] + aR[1] * db[1] + aR[2] * db[2] + aR[3] * db[3] + qp->bR[l];
    d[OWI(m) + l] = aI[0] * db[0] + aI[1] * db[1] + aI[2] * db[2] + aI[3] * db[3] + qp->bI[l];
  }
  /* multipliers pi of eq. lag from the KKT conditions of the line subproblem:
   * pi13, pi14 = -(line-limit multipliers); (pi11, pi12) from stationarity in (d_wR, d_wI) */
  for (int l = 0; l < L; ++l) {
    int i = g->f[l], j = g->t[l];
    const double* Y = m->Y + 8 * l;
    const double* xl = s->xl + 8 * l;
    double wi = x[OW(m) + i], wj = x[OW(m) + j], thi = x[OTH(m) + i], thj = x[OTH(m) + j];
    double wr = x[OWR(m) + l], wim = x[OWI(m) + l];
    double sn = sin(thi - thj), cs = cos(thi - thj);
    const double* aR = qp->aR + 4 * l;
    const double* aI = qp->aI + 4 * l;
    double db[4] = {xl[4], xl[5], xl[6], xl[7]};
    double z[6];
    z[0] = db[0]; z[1] = db[1];
    z[2] = aR[0] * db[0] + aR[1] * db[1] + aR[2] * db[2] + aR[3] * db[3] + qp->bR[l];
    z[3] = aI[0] * db[0] + aI[1] * db[1] + aI[2] * db[2] + aI[3] * db[3] + qp->bI[l];
    z[4] = db[2]; z[5] = db[3];
    const double* H = qp->H + 36 * l;
    double gR = 0, gI = 0;
    for (int k = 0; k < 6; ++k) { gR += H[2 * 6 + k] * z[k]; gI += H[3 * 6 + k] * z[k]; }
    double J[4][6];
    flow_jac(Y, J);
    const double* lam = s->ll + 8 * l;
    for (int f = 0; f < 4; ++f) { gR += lam[f] * J[f][2]; gI += lam[f] * J[f][3]; }
    const double* fl = qp->flow + 4 * l;
    double u13 = s->ul[4 * l], u14 = s->ul[4 * l + 1];
    /* h = 2p dp + 2q dq - rhs; derivative in dwR: 2p dp/dwR + 2q dq/dwR */
    gR += u13 * (2 * fl[0] * J[0][2] + 2 * fl[1] * J[1][2]) + u14 * (2 * fl[2] * J[2][2] + 2 * fl[3] * J[3][2]);
    gI += u13 * (2 * fl[0] * J[0][3] + 2 * fl[1] * J[1][3]) + u14 * (2 * fl[2] * J[2][3] + 2 * fl[3] * J[3][3]);
    /* J^T pi = -g with J = [[2wR, 2wI], [sin, -cos]] */
    double a11 = 2 * wr, a12 = sn, a21 = 2 * wim, a22 = -cs; /* J^T */
    double det = a11 * a22 - a12 * a21;
    double p11 = (-gR * a22 + gI * a12) / det;
    double p12 = (-gI * a11 + gR * a21) / det;
    pi[4 * l + 0] = p11;
    pi[4 * l + 1] = p12;
    pi[4 * l + 2] = -u13;
    pi[4 * l + 3] = -u14;
    (void)wi; (void)wj;
  }
}

/* sum of l1 violations of every constraint at point x (h of the merit function,
 * with the linear constraints included), and the l_inf maximum */
static void violations(const og_model* m, const double* x, int use_angle, double* h1, double* hinf) {
  const og_grid* g = &m->g;
  int B = g->nbus, L = g->nbranch, G = g->ngen;
  double* c4 = (double*)malloc(sizeof(double) * (4 * L + 1));
  double* bal = (double*)malloc(sizeof(double) * 2 * B);
  og_constraints(m, x, c4, bal);
  double s = 0, mx = 0, v;
#define ACC(val) do { v = (val); s += v; if (v > mx) mx = v; } while (0)
  for (int l = 0; l < L; ++l) {
    ACC(fabs(c4[4 * l])); ACC(fabs(c4[4 * l + 1]));
    ACC(neg(c4[4 * l + 2])); ACC(neg(c4[4 * l + 3]));
    if (use_angle) {
      double th = x[OTH(m) + g->f[l]] - x[OTH(m) + g->t[l]];
      if (g->angmin[l] > -TWO_PI) ACC(neg(th - g->angmin[l]));
      if (g->angmax[l] < TWO_PI) ACC(neg(g->angmax[l] - th));
    }
  }
  for (int i = 0; i < B; ++i) {
    ACC(fabs(bal[2 * i])); ACC(fabs(bal[2 * i + 1]));
    double w = x[OW(m) + i], th = x[OTH(m) + i];
    ACC(neg(w - sq(g->vmin[i]))); ACC(neg(sq(g->vmax[i]) - w));
    if (i == m->ref) ACC(fabs(th));
    else { ACC(neg(th + TWO_PI)); ACC(neg(TWO_PI - th)); }
  }
  for (int k = 0; k < G; ++k) {
    double p = x[OPG(m) + k], q = x[OQG(m) + k];
    ACC(neg(p - g->pmin[k])); ACC(neg(g->pmax[k] - p));
    ACC(neg(q - g->qmin[k])); ACC(neg(g->qmax[k] - q));
  }
#undef ACC
  free(c4); free(bal);
  *h1 = s;
  *hinf = mx;
}

/* phi_1(x) = f + mu h, q(d) = f + grad f'd + 1/2 d'(Hess L)d + mu m(d) (Sec. II-C) */
void og_merit(const og_model* m, const og_qp* qp, const double* x, const double* d, double mu, int use_angle,
              double* phi_x, double* phi_xd, double* pred) {
  og_merit_ex(m, qp, x, d, mu, use_angle, 1.0, phi_x, phi_xd, pred);
}

/* og_merit with the objective weighted by fscale (the QP's own gradient and
 * curvature were built with the same weight) */
void og_merit_ex(const og_model* m, const og_qp* qp, const double* x, const double* d, double mu, int use_angle,
                 double fscale, double* phi_x, double* phi_xd, double* pred) {
  const og_grid* g = &m->g;
  int B = g->nbus, L = g->nbranch, G = g->ngen, n = m->nvar;
  double* xd = (double*)malloc(sizeof(double) * n);
  for (int k = 0; k < n; ++k) xd[k] = x[k] + d[k];
  double h0, hinf0, h1, hinf1;
  violations(m, x, use_angle, &h0, &hinf0);
  violations(m, xd, use_angle, &h1, &hinf1);
  double f0 = fscale * og_objective(m, x), f1 = fscale * og_objective(m, xd);
  *phi_x = f0 + mu * h0;
  *phi_xd = f1 + mu * h1;
  /* model: gradient and curvature */
  double lin = 0, quad = 0;
  for (int k = 0; k < G; ++k) {
    double dp = d[OPG(m) + k];
    lin += qp->gd1[k] * dp;
    quad += qp->gd2[k] * dp * dp;
  }
  /* m(d): linearised nonlinear constraints, exact linear ones at x + d */
  double md = 0;
  double* c4 = (double*)malloc(sizeof(double) * (4 * L + 1));
  double* bal = (double*)malloc(sizeof(double) * 2 * B);
  og_constraints(m, x, c4, bal);
  for (int l = 0; l < L; ++l) {
    int i = g->f[l], j = g->t[l];
    double z[6] = {d[OW(m) + i], d[OTH(m) + i], d[OWR(m) + l], d[OWI(m) + l], d[OW(m) + j], d[OTH(m) + j]};
    const double* H = qp->H + 36 * l;
    for (int a = 0; a < 6; ++a)
      for (int b2 = 0; b2 < 6; ++b2) quad += z[a] * H[6 * a + b2] * z[b2];
    double wi = x[OW(m) + i], wj = x[OW(m) + j], wr = x[OWR(m) + l], wim = x[OWI(m) + l];
    double th = x[OTH(m) + i] - x[OTH(m) + j];
    double sn = sin(th), cs = cos(th), D = wr * cs + wim * sn;
    double l11 = c4[4 * l] + 2 * wr * z[2] + 2 * wim * z[3] - wj * z[0] - wi * z[4];
    double l12 = c4[4 * l + 1] + sn * z[2] - cs * z[3] + D * (z[1] - z[5]);
    double J[4][6];
    flow_jac(m->Y + 8 * l, J);
    double df[4];
    for (int r = 0; r < 4; ++r) {
      df[r] = 0;
      for (int k = 0; k < 6; ++k) df[r] += J[r][k] * z[k];
    }
    const double* fl = qp->flow + 4 * l;
    double l13 = c4[4 * l + 2] - 2 * fl[0] * df[0] - 2 * fl[1] * df[1];
    double l14 = c4[4 * l + 3] - 2 * fl[2] * df[2] - 2 * fl[3] * df[3];
    md += fabs(l11) + fabs(l12) + neg(l13) + neg(l14);
  }
  /* linear constraints: the same terms as h at x + d */
  {
    double* c4d = (double*)malloc(sizeof(double) * (4 * L + 1));
    double* bald = (double*)malloc(sizeof(double) * 2 * B);
    og_constraints(m, xd, c4d, bald);
    double nl = 0;
    for (int l = 0; l < L; ++l) nl += fabs(c4d[4 * l]) + fabs(c4d[4 * l + 1]) + neg(c4d[4 * l + 2]) + neg(c4d[4 * l + 3]);
    md += h1 - nl; /* h1 minus its nonlinear part = linear part at x + d */
    free(c4d); free(bald);
  }
  free(c4); free(bal);
  /* q(0) - q(d) */
  *pred = -lin - 0.5 * quad + mu * (h0 - md);
  free(xd);
}

/* primal infeasibility (l_inf of all violations) and scaled dual infeasibility
 * (projected gradient of the Lagrangian, multipliers from the last QP) */
void og_kkt(const og_model* m, const double* x, const double* pi, const double* nu, const double* ul,
            int use_angle, double* primal, double* dual) {
  const og_grid* g = &m->g;
  int B = g->nbus, L = g->nbranch, G = g->ngen, n = m->nvar;
  double h1, hinf;
  violations(m, x, use_angle, &h1, &hinf);
  *primal = hinf;
  double* gr = (double*)calloc(n, sizeof(double));
  double S = g->base_mva, gfmax = 0;
  for (int k = 0; k < G; ++k) {
    double gf = 2 * g->c2[k] * S * S * x[OPG(m) + k] + g->c1[k] * S;
    gfmax = dmax(gfmax, fabs(gf));
    gr[OPG(m) + k] = gf + nu[2 * g->gbus[k]];
    gr[OQG(m) + k] = nu[2 * g->gbus[k] + 1];
  }
  for (int i = 0; i < B; ++i) gr[OW(m) + i] += -g->gs[i] * nu[2 * i] + g->bs[i] * nu[2 * i + 1];
  for (int l = 0; l < L; ++l) {
    int i = g->f[l], j = g->t[l];
    double J[4][6];
    flow_jac(m->Y + 8 * l, J);
    double fl[4];
    branch_flows(m, x, l, fl);
    double wi = x[OW(m) + i], wj = x[OW(m) + j], wr = x[OWR(m) + l], wim = x[OWI(m) + l];
    double th = x[OTH(m) + i] - x[OTH(m) + j];
    double sn = sin(th), cs = cos(th), D = wr * cs + wim * sn;
    const double* p = pi + 4 * l;
    /* gradient over z = (w_i, th_i, wR, wI, w_j, th_j) */
    double gz[6] = {0};
    /* balance terms: -y_P(end bus) dp_e - y_Q dq_e */
    for (int k = 0; k < 6; ++k) {
      gz[k] += -nu[2 * i] * J[0][k] - nu[2 * i + 1] * J[1][k];
      gz[k] += -nu[2 * j] * J[2][k] - nu[2 * j + 1] * J[3][k];
    }
    /* pi11 c11 */
    gz[0] += p[0] * (-wj); gz[4] += p[0] * (-wi); gz[2] += p[0] * 2 * wr; gz[3] += p[0] * 2 * wim;
    /* pi12 c12 */
    gz[1] += p[1] * D; gz[5] += -p[1] * D; gz[2] += p[1] * sn; gz[3] += -p[1] * cs;
    /* pi13 c13, pi14 c14 */
    for (int k = 0; k < 6; ++k) {
      gz[k] += p[2] * (-2 * fl[0] * J[0][k] - 2 * fl[1] * J[1][k]);
      gz[k] += p[3] * (-2 * fl[2] * J[2][k] - 2 * fl[3] * J[3][k]);
    }
    /* angle rows: angmax - th >= 0 (pi = -u_hi), th - angmin >= 0 (pi = -u_lo) */
    if (use_angle) {
      double uh = ul[4 * l + 2], ulo = ul[4 * l + 3];
      gz[1] += -uh * (-1.0) + -ulo * (1.0);
      gz[5] += -uh * (1.0) + -ulo * (-1.0);
    }
    gr[OW(m) + i] += gz[0]; gr[OTH(m) + i] += gz[1];
    gr[OWR(m) + l] += gz[2]; gr[OWI(m) + l] += gz[3];
    gr[OW(m) + j] += gz[4]; gr[OTH(m) + j] += gz[5];
  }
  /* projection for variables at a bound (bound multipliers absorb the right sign) */
  const double tact = 1e-5;
  double dm = 0;
  for (int k = 0; k < G; ++k) {
    double v;
    double p = x[OPG(m) + k];
    v = gr[OPG(m) + k];
    if (p - g->pmin[k] <= tact && v > 0) v = 0;
    if (g->pmax[k] - p <= tact && v < 0) v = 0;
    dm = dmax(dm, fabs(v));
    double q = x[OQG(m) + k];
    v = gr[OQG(m) + k];
    if (q - g->qmin[k] <= tact && v > 0) v = 0;
    if (g->qmax[k] - q <= tact && v < 0) v = 0;
    dm = dmax(dm, fabs(v));
  }
  for (int i = 0; i < B; ++i) {
    double w = x[OW(m) + i], v = gr[OW(m) + i];
    if (w - sq(g->vmin[i]) <= tact && v > 0) v = 0;
    if (sq(g->vmax[i]) - w <= tact && v < 0) v = 0;
    dm = dmax(dm, fabs(v));
    if (i != m->ref) dm = dmax(dm, fabs(gr[OTH(m) + i]));
  }
  for (int l = 0; l < L; ++l) {
    dm = dmax(dm, fabs(gr[OWR(m) + l]));
    dm = dmax(dm, fabs(gr[OWI(m) + l]));
  }
  free(gr);
  *dual = dm / dmax(1.0, gfmax);
}

/* ------------------------------------------------------------------ SQP */
/* Step acceptance and trust-region update of Alg. 1.
 * Acceptance is the ratio test of Sec. II-C as printed: the actual merit
 * reduction ared = phi_1(x) - phi_1(x + d) must be positive and so must
 * ared / pred, pred = q(0) - q(d); with ared > 0 that is pred > 0 (a zero or
 * non-finite pred rejects).  Alg. 1 prints only Delta+ >= Delta on acceptance
 * and Delta+ <= Delta on rejection; the rules it carries as comments give the
 * constants: an accepted step on the trust-region boundary (|d|_inf >= 0.99
 * Delta, the boundary up to rounding) doubles Delta, capped at delta_max (the
 * commented max{2 Delta, Delta-bar} read as a cap); an accepted interior step
 * keeps Delta; a rejected step sets Delta = 0.5 min(Delta, |d|_inf). */
double og_tr_update(const og_sqp_opts* o, double delta, double dnorm, double ared, double pred, int* accept) {
  int acc = isfinite(ared) && isfinite(pred) && ared > 0 && pred > 0;
  *accept = acc;
  if (acc) return dnorm >= 0.99 * delta ? dmin(2 * delta, o->delta_max) : delta;
  return 0.5 * dmin(delta, dnorm);
}

void og_violations(const og_model* m, const double* x, int use_angle, double* h1, double* hinf) {
  violations(m, x, use_angle, h1, hinf);
}

static int all_finite(const double* v, int n) {
  for (int k = 0; k < n; ++k)
    if (!isfinite(v[k])) return 0;
  return 1;
}

int og_sqp(const og_model* m, const og_sqp_opts* o, const double* x0, double* x, double* pi,
           og_sqp_info* info, double* hist, int hist_cap) {
  const og_grid* g = &m->g;
  int B = g->nbus, L = g->nbranch, G = g->ngen, n = m->nvar;
  /* QP and ADMM storage */
  double* buf = (double*)calloc((size_t)(4 + 36 + 4 + 4 + 1 + 1 + 16 + 4 + 16 + 4 + 4 + 4 + 8 + 2 + 1 + 1) * L + 6 * G + 2 * B + 1,
                                sizeof(double));
  double* p = buf;
  og_qp qp;
#define TAKE(field, cnt) do { qp.field = p; p += (cnt); } while (0)
  TAKE(flow, 4 * L); TAKE(H, 36 * L); TAKE(aR, 4 * L); TAKE(aI, 4 * L); TAKE(bR, L); TAKE(bI, L);
  TAKE(QH, 16 * L); TAKE(gH, 4 * L); TAKE(F, 16 * L); TAKE(f0, 4 * L); TAKE(lo, 4 * L); TAKE(hi, 4 * L);
  TAKE(G, 8 * L); TAKE(grhs, 2 * L); TAKE(alo, L); TAKE(ahi, L);
  TAKE(gd1, G); TAKE(gd2, G); TAKE(glp, G); TAKE(gup, G); TAKE(glq, G); TAKE(guq, G);
  TAKE(pdk, B); TAKE(qdk, B);
#undef TAKE
  double* sbuf = (double*)calloc((size_t)(8 * 4) * L + 2 * 4 * G + 4 * B + 4 * L + 1, sizeof(double));
  og_admm_state st;
  p = sbuf;
  st.xl = p; p += 8 * L; st.zl = p; p += 8 * L; st.ll = p; p += 8 * L; st.rl = p; p += 8 * L;
  st.xg = p; p += 2 * G; st.zg = p; p += 2 * G; st.lg = p; p += 2 * G; st.rg = p; p += 2 * G;
  st.zb = p; p += 2 * B; st.nu = p; p += 2 * B; st.ul = p; p += 4 * L;
  st.aset = (int32_t*)malloc(sizeof(int32_t) * (L > 0 ? L : 1));
  for (int k = 0; k < L; ++k) st.aset[k] = -1;
  double* d = (double*)calloc(n, sizeof(double));
  double* pin = (double*)calloc(4 * L + 1, sizeof(double));
  double* dsoc = (double*)calloc(n, sizeof(double));
  double* pisoc = (double*)calloc(4 * L + 1, sizeof(double));

  memcpy(x, x0, sizeof(double) * n);
  memset(pi, 0, sizeof(double) * 4 * L);
  og_admm_cold(m, &st, o->rho, 0);
  double delta = o->delta0;
  int first_qp = 1;
  int status = 1, k, acc = 0, admm_total = 0;
  int restoring = 0;       /* 1 in the feasibility-restoration phase */
  double fscale = 1.0;     /* objective weight: 0 while restoring */
  enum { kRestoreWindow = 5 };
  double primal_at[kRestoreWindow] = {0};  /* primal infeasibility of the last iterations */
  int since_switch = 0;    /* iterations since the last change of phase */
  double primal = BIG, dual = BIG;
  {
    double h1;
    violations(m, x, o->admm.use_angle, &h1, &primal);
  }
  for (k = 0; k < o->max_sqp; ++k) {
    og_build_ex(m, x, pi, delta, o->admm.use_angle, NULL, fscale, &qp);
    og_admm_cold(m, &st, o->rho, first_qp ? 0 : o->warm_lambda);
    first_qp = 0;
    og_admm_info ai;
    og_admm(m, &qp, &o->admm, &st, &ai);
    int iters = ai.iters;
    og_step(m, &qp, &st, x, d, pin);
    double dn = 0;
    for (int t2 = 0; t2 < 2 * G + 2 * B; ++t2) dn = dmax(dn, fabs(d[t2]));
    double phx, phxd, pred;
    og_merit_ex(m, &qp, x, d, o->mu, o->admm.use_angle, fscale, &phx, &phxd, &pred);
    double ared = phx - phxd;
    int accept = 0, soc = 0;
    og_tr_update(o, delta, dn, ared, pred, &accept);
    if (!accept && o->soc && isfinite(pred) && pred > 0) {
      /* second-order correction: the same QP with the constraint values of
       * x + d (linearised at x); the corrected step passes if it reduces the
       * merit function against the original step's model reduction */
      og_build_ex(m, x, pi, delta, o->admm.use_angle, d, fscale, &qp);
      og_admm_cold(m, &st, o->rho, o->warm_lambda);
      og_admm_info as;
      og_admm(m, &qp, &o->admm, &st, &as);
      iters += as.iters;
      og_step(m, &qp, &st, x, dsoc, pisoc);
      double dns = 0;
      for (int t2 = 0; t2 < 2 * G + 2 * B; ++t2) dns = dmax(dns, fabs(dsoc[t2]));
      double phx2, phxd2, pred2;
      og_merit_ex(m, &qp, x, dsoc, o->mu, o->admm.use_angle, fscale, &phx2, &phxd2, &pred2);
      double ared2 = phx - phxd2;
      int acc2 = 0;
      og_tr_update(o, delta, dns, ared2, pred, &acc2);
      soc = 1;
      if (acc2) {
        memcpy(d, dsoc, sizeof(double) * n);
        memcpy(pin, pisoc, sizeof(double) * 4 * L);
        dn = dns;
        ared = ared2;
        soc = 2;
      }
      ai.r_inf = as.r_inf;
      ai.s_inf = as.s_inf;
    }
    admm_total += iters;
    delta = og_tr_update(o, delta, dn, ared, pred, &accept);
    if (accept) {
      for (int t2 = 0; t2 < n; ++t2) x[t2] += d[t2];
      memcpy(pi, pin, sizeof(double) * 4 * L);
      acc++;
      og_kkt(m, x, pi, st.nu, st.ul, o->admm.use_angle, &primal, &dual);
    }
    if (hist && k < hist_cap) {
      double* hr = hist + OG_HIST_W * k;
      hr[0] = og_objective(m, x); hr[1] = primal; hr[2] = dual; hr[3] = iters;
      hr[4] = ai.r_inf; hr[5] = ai.s_inf; hr[6] = accept; hr[7] = delta; hr[8] = dn; hr[9] = ared; hr[10] = pred;
      hr[11] = soc; hr[12] = restoring;
    }
    if (!all_finite(x, n)) { status = 3; k++; break; }
    int stall = (accept && dn <= o->step_tol) || delta < o->delta_min;
    /* no progress towards feasibility: the violation, above 10 tol, has not
     * fallen by a tenth over the last kRestoreWindow iterations */
    double older = primal_at[k % kRestoreWindow];  /* the value kRestoreWindow iterations ago */
    primal_at[k % kRestoreWindow] = primal;
    int no_progress = k >= kRestoreWindow && primal > 10 * o->tol && primal > 0.9 * older &&
                      since_switch >= kRestoreWindow;
    ++since_switch;
    if (!restoring) {
      if (accept && primal <= o->tol && dual <= o->tol) { status = 0; k++; break; }
      if (stall || (o->restore && no_progress)) {
        if (o->restore && primal > o->tol) {
          /* feasibility restoration: minimise the violation alone (objective
           * weight 0, merit mu h) from the current point and radius delta0 */
          restoring = 1;
          fscale = 0.0;
          delta = o->delta0;
          since_switch = 0;
          continue;
        }
        status = 2; k++; break;
      }
    } else {
      if (accept && primal <= o->tol) {  /* feasible again: back to the SQP on the ACOPF */
        restoring = 0;
        fscale = 1.0;
        delta = o->delta0;
        since_switch = 0;
        continue;
      }
      /* the violation stalls above tol: locally infeasible */
      if (stall || no_progress) { status = 5; k++; break; }
    }
  }
  info->iters = k;
  info->accepted = acc;
  info->status = status;
  info->admm_total = admm_total;
  info->obj = og_objective(m, x);
  info->primal = primal;
  info->dual = dual;
  info->delta = delta;
  free(buf); free(sbuf); free(d); free(pin); free(dsoc); free(pisoc); free(st.aset);
  return status;
}
