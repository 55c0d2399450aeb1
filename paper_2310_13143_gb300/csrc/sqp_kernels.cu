// SQP-side kernels (FP64): model set-up, QP build (Alg. 1, eq. QPsub), step and
// multiplier recovery after the ADMM sweep, l1 merit test with the trust-region
// update (Sec. II-C/D), and the KKT measures used for termination.
//
// One thread per component (branch, generator or bus); per-instance sums use
// per-component term arrays reduced by one CTA per instance in a fixed order,
// so every result is deterministic.
#include <math.h>

#include "common.cuh"

namespace acopf {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ double sq(double a) { return a * a; }
__device__ __forceinline__ double negpart(double a) { return a < 0 ? -a : 0.0; }

struct Br {  // one branch's local data at the current iterate
  int i, j;
  double Y[8];
  double wi, wj, thi, thj, wr, wim;
};

__device__ __forceinline__ void load_branch(const Dev& d, int l, Br& b) {
  b.i = d.f[l];
  b.j = d.t[l];
#pragma unroll
  for (int k = 0; k < 8; ++k) b.Y[k] = d.Y[k * d.L + l];
  b.wi = d.w[b.i];
  b.wj = d.w[b.j];
  b.thi = d.th[b.i];
  b.thj = d.th[b.j];
  b.wr = d.wr[l];
  b.wim = d.wi[l];
}

// flows of eq. acopf_pf as rows over z = (w_i, th_i, wR, wI, w_j, th_j)
__device__ __forceinline__ void flow_jac(const double* Y, double J[4][6]) {
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int k = 0; k < 6; ++k) J[r][k] = 0.0;
  J[0][0] = Y[0];  J[0][2] = Y[2];  J[0][3] = Y[3];
  J[1][0] = -Y[1]; J[1][2] = -Y[3]; J[1][3] = Y[2];
  J[2][4] = Y[6];  J[2][2] = Y[4];  J[2][3] = -Y[5];
  J[3][4] = -Y[7]; J[3][2] = -Y[5]; J[3][3] = -Y[4];
}

__device__ __forceinline__ void flows_at(const double* Y, double wi, double wj, double wr, double wim, double fl[4]) {
  fl[0] = Y[0] * wi + Y[2] * wr + Y[3] * wim;
  fl[1] = -Y[1] * wi - Y[3] * wr + Y[2] * wim;
  fl[2] = Y[6] * wj + Y[4] * wr - Y[5] * wim;
  fl[3] = -Y[7] * wj - Y[5] * wr - Y[4] * wim;
}

// Hessian of L_ij (eq. lag) over z
__device__ void branch_hessian(const Br& b, const double pi[4], double H[6][6]) {
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int k = 0; k < 6; ++k) H[r][k] = 0.0;
  double sn, cs;
  sincos(b.thi - b.thj, &sn, &cs);
  H[2][2] += 2.0 * pi[0];
  H[3][3] += 2.0 * pi[0];
  H[0][4] -= pi[0];
  H[4][0] -= pi[0];
  double s0 = -b.wr * sn + b.wim * cs;
  H[1][1] += pi[1] * s0;
  H[5][5] += pi[1] * s0;
  H[1][5] -= pi[1] * s0;
  H[5][1] -= pi[1] * s0;
  H[2][1] += pi[1] * cs; H[1][2] += pi[1] * cs;
  H[2][5] -= pi[1] * cs; H[5][2] -= pi[1] * cs;
  H[3][1] += pi[1] * sn; H[1][3] += pi[1] * sn;
  H[3][5] -= pi[1] * sn; H[5][3] -= pi[1] * sn;
  double J[4][6];
  flow_jac(b.Y, J);
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int c = 0; c < 6; ++c)
      H[a][c] += -2.0 * pi[2] * (J[0][a] * J[0][c] + J[1][a] * J[1][c]) -
                 2.0 * pi[3] * (J[2][a] * J[2][c] + J[3][a] * J[3][c]);
}

__device__ __forceinline__ void box_shift(double lb, double ub, double v, double delta, double& lo, double& hi) {
  double l = fmax(lb - v, -delta), u = fmin(ub - v, delta);
  if (l > u) {  // further than delta outside its bounds: move the full radius back
    double mv = (ub - v < -delta) ? -delta : delta;
    l = u = mv;
  }
  lo = l;
  hi = u;
}

__device__ bool chol4_pd(const double Q[4][4]) {
  double Lm[4][4] = {};
  for (int j = 0; j < 4; ++j) {
    double s = Q[j][j];
    for (int k = 0; k < j; ++k) s -= Lm[j][k] * Lm[j][k];
    if (!(s > 0)) return false;
    Lm[j][j] = sqrt(s);
    for (int i = j + 1; i < 4; ++i) {
      double t = Q[i][j];
      for (int k = 0; k < j; ++k) t -= Lm[i][k] * Lm[j][k];
      Lm[i][j] = t / Lm[j][j];
    }
  }
  return true;
}

// ------------------------------------------------------------ set-up
// pi-model entries of every branch (Sec. III-A)
__global__ void k_admittance(int L, const double* r, const double* x, const double* bc, const double* tap,
                             const double* shift, double* Y) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  double tp = tap[l] == 0.0 ? 1.0 : tap[l];
  double den = r[l] * r[l] + x[l] * x[l];
  double ys_re = r[l] / den, ys_im = -x[l] / den;
  double sn, cs;
  sincos(shift[l], &sn, &cs);
  double a_re = -ys_re / tp, a_im = -ys_im / tp;
  Y[0 * L + l] = ys_re / (tp * tp);
  Y[1 * L + l] = (ys_im + 0.5 * bc[l]) / (tp * tp);
  Y[2 * L + l] = a_re * cs - a_im * sn;
  Y[3 * L + l] = a_re * sn + a_im * cs;
  Y[4 * L + l] = a_re * cs + a_im * sn;
  Y[5 * L + l] = -a_re * sn + a_im * cs;
  Y[6 * L + l] = ys_re;
  Y[7 * L + l] = ys_im + 0.5 * bc[l];
}

// flat start (the starting point of Alg. 1)
__global__ void k_flat_start(Dev d) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < d.G) {
    d.pg[k] = 0.5 * (d.pmin[k] + d.pmax[k]);
    d.qg[k] = 0.5 * (d.qmin[k] + d.qmax[k]);
  }
  if (k < d.B) {
    d.w[k] = 1.0;
    d.th[k] = 0.0;
  }
  if (k < d.L) {
    d.wr[k] = 1.0;
    d.wi[k] = 0.0;
    for (int r = 0; r < 4; ++r) d.pi[r * d.L + k] = 0.0;
  }
}

// ------------------------------------------------------------ QP build
// One thread per branch: flows, Hessian, elimination (eq. elim), the line
// subproblem's quadratic (with the ADMM penalty folded in), flow maps, boxes
// and line-limit rows.  Optionally exports the FP64 QP data (110 per branch).
template <typename T>
__global__ void k_build_branch(Dev d, int use_angle, double* xbr, int pass) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= d.L) return;
  int k = d.br_inst[l];
  if (!live(d.ctl[k], pass)) return;
  d.wset[l] = 0;  // a new QP: no active set carried over
  double delta = d.ctl[k].delta;
  double rho = d.rho_l[l];
  Br b;
  load_branch(d, l, b);
  double fl[4];
  flows_at(b.Y, b.wi, b.wj, b.wr, b.wim, fl);
  for (int r = 0; r < 4; ++r) d.flow[r * d.L + l] = fl[r];
  double pi[4];
  for (int r = 0; r < 4; ++r) pi[r] = d.pi[r * d.L + l];
  double H[6][6];
  branch_hessian(b, pi, H);

  double sn, cs;
  sincos(b.thi - b.thj, &sn, &cs);
  double D = b.wr * cs + b.wim * sn;
  double R0 = b.wi * b.wj - b.wr * b.wr - b.wim * b.wim;
  double S0 = -b.wr * sn + b.wim * cs;
  // correction pass: the constraint values of x + d (d = the rejected step),
  // linearised at x -- c(x + d) - grad c(x)' d; for the quadratic opfc11 that
  // adds the step's second-order term, opfc12 is evaluated at x + d
  double dz[6] = {0, 0, 0, 0, 0, 0};
  if (pass) {
    dz[0] = d.dw[b.i]; dz[1] = d.dth[b.i]; dz[2] = d.dwr[l]; dz[3] = d.dwi[l]; dz[4] = d.dw[b.j]; dz[5] = d.dth[b.j];
    const double dth = dz[1] - dz[5];
    R0 += dz[0] * dz[4] - dz[2] * dz[2] - dz[3] * dz[3];
    double s1, c1;
    sincos(b.thi - b.thj + dth, &s1, &c1);
    S0 = (-(b.wr + dz[2]) * s1 + (b.wim + dz[3]) * c1) - (-sn * dz[2] + cs * dz[3] - D * dth);
  }
  double aR[4] = {cs * b.wj / (2 * D), -b.wim, cs * b.wi / (2 * D), b.wim};
  double aI[4] = {sn * b.wj / (2 * D), b.wr, sn * b.wi / (2 * D), -b.wr};
  double bR = (cs * R0 + 2 * b.wim * S0) / (2 * D);
  double bI = (sn * R0 - 2 * b.wr * S0) / (2 * D);
  for (int r = 0; r < 4; ++r) {
    d.aR[r * d.L + l] = aR[r];
    d.aI[r * d.L + l] = aI[r];
  }
  d.bR[l] = bR;
  d.bI[l] = bI;

  // A (6x4): rows w_i, th_i <- identity; wR <- aR; wI <- aI; w_j, th_j <- identity
  double A[6][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {aR[0], aR[1], aR[2], aR[3]},
                    {aI[0], aI[1], aI[2], aI[3]}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  double bb[6] = {0, 0, bR, bI, 0, 0};
  double HA[6][4];
  for (int a = 0; a < 6; ++a)
    for (int c = 0; c < 4; ++c) {
      double s = 0;
      for (int q = 0; q < 6; ++q) s += H[a][q] * A[q][c];
      HA[a][c] = s;
    }
  double QH[4][4], gH[4];
  for (int r = 0; r < 4; ++r) {
    for (int c = 0; c < 4; ++c) {
      double s = 0;
      for (int q = 0; q < 6; ++q) s += A[q][r] * HA[q][c];
      QH[r][c] = s;
    }
    double s = 0;
    for (int q = 0; q < 6; ++q) s += bb[q] * HA[q][r];
    gH[r] = s;
  }
  double J[4][6];
  flow_jac(b.Y, J);
  double F[4][4], f0[4];
  for (int r = 0; r < 4; ++r) {
    double s0 = 0;
    for (int q = 0; q < 6; ++q) s0 += J[r][q] * bb[q];
    f0[r] = s0;
    for (int c = 0; c < 4; ++c) {
      double s = 0;
      for (int q = 0; q < 6; ++q) s += J[r][q] * A[q][c];
      F[r][c] = s;
    }
  }
  // line subproblem quadratic: Q = A'HA + rho (F'F + I); made positive definite
  // by a doubling diagonal shift when the Hessian makes it indefinite (Sec. III-B)
  double Q[4][4];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = QH[r][c];
      for (int q = 0; q < 4; ++q) s += rho * F[q][r] * F[q][c];
      Q[r][c] = s + (r == c ? rho : 0.0);
    }
  if (!chol4_pd(Q)) {
    double qmax = 0;
    for (int r = 0; r < 4; ++r) qmax = fmax(qmax, fabs(Q[r][r]));
    double dl = 1e-8 * (qmax > 0 ? qmax : 1.0);
    double Q0[4] = {Q[0][0], Q[1][1], Q[2][2], Q[3][3]};
    for (int it = 0; it < 200 && !chol4_pd(Q); ++it) {
      for (int r = 0; r < 4; ++r) Q[r][r] = Q0[r] + dl;
      dl *= 2;
    }
  }
  double c0[4];
  for (int r = 0; r < 4; ++r) {
    double s = gH[r];
    for (int q = 0; q < 4; ++q) s += rho * F[q][r] * f0[q];
    c0[r] = s;
  }
  // boxes on dbar (bounds and trust region); the reference angle stays 0
  double lo[4], hi[4];
  box_shift(d.wmin[b.i], d.wmax[b.i], b.wi, delta, lo[0], hi[0]);
  box_shift(-kTwoPi, kTwoPi, b.thi, delta, lo[1], hi[1]);
  box_shift(d.wmin[b.j], d.wmax[b.j], b.wj, delta, lo[2], hi[2]);
  box_shift(-kTwoPi, kTwoPi, b.thj, delta, lo[3], hi[3]);
  if (d.isref[b.i]) lo[1] = hi[1] = -b.thi;
  if (d.isref[b.j]) lo[3] = hi[3] = -b.thj;
  // line limits (line_kernel_1, line_kernel_2)
  double G[2][4], grhs[2], gnorm[2];
  double s2 = d.s2[l];
  for (int e = 0; e < 2; ++e) {
    double p = fl[2 * e], q = fl[2 * e + 1];
    if (s2 < 0) {
      for (int c = 0; c < 4; ++c) G[e][c] = 0.0;
      grhs[e] = kBig;
      gnorm[e] = 0.0;
      continue;
    }
    double nn = 0;
    for (int c = 0; c < 4; ++c) {
      G[e][c] = 2 * p * F[2 * e][c] + 2 * q * F[2 * e + 1][c];
      nn += G[e][c] * G[e][c];
    }
    double lim = s2 - p * p - q * q;
    if (pass) {  // the flows are linear in (w, wR, wI): their change under d is exact
      double dp = 0, dq = 0;
      for (int c = 0; c < 6; ++c) {
        dp += J[2 * e][c] * dz[c];
        dq += J[2 * e + 1][c] * dz[c];
      }
      lim -= dp * dp + dq * dq;
    }
    grhs[e] = lim - 2 * p * f0[2 * e] - 2 * q * f0[2 * e + 1];
    gnorm[e] = sqrt(nn);
  }
  double alo = -kBig, ahi = kBig;
  if (use_angle && d.angmin[l] > -kTwoPi && d.angmax[l] < kTwoPi) {
    alo = d.angmin[l] - (b.thi - b.thj);
    ahi = d.angmax[l] - (b.thi - b.thj);
  }

  // sweep record in the sweep precision
  T rec[56];
  rec[0] = (T)Q[0][0]; rec[1] = (T)Q[0][1]; rec[2] = (T)Q[0][2]; rec[3] = (T)Q[0][3];
  rec[4] = (T)Q[1][1]; rec[5] = (T)Q[1][2]; rec[6] = (T)Q[1][3];
  rec[7] = (T)Q[2][2]; rec[8] = (T)Q[2][3]; rec[9] = (T)Q[3][3];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) rec[10 + 4 * r + c] = (T)F[r][c];
  for (int r = 0; r < 4; ++r) {
    rec[26 + r] = (T)f0[r];
    rec[30 + r] = (T)c0[r];
    rec[34 + r] = (T)lo[r];
    rec[38 + r] = (T)hi[r];
  }
  for (int e = 0; e < 2; ++e) {
    double inv = gnorm[e] > 0 ? 1.0 / gnorm[e] : 0.0;
    for (int c = 0; c < 4; ++c) rec[42 + 4 * e + c] = (T)(G[e][c] * inv);
    rec[50 + e] = (T)(gnorm[e] > 0 ? grhs[e] * inv : kBig);
    rec[54 + e] = (T)gnorm[e];
  }
  rec[52] = (T)alo;
  rec[53] = (T)ahi;
  V4<T>* R = (V4<T>*)d.lrec;
  for (int c = 0; c < kRecChunks; ++c) {
    V4<T> v;
    v.x = rec[4 * c];
    v.y = rec[4 * c + 1];
    v.z = rec[4 * c + 2];
    v.w = rec[4 * c + 3];
    R[c * d.L + l] = v;
  }
  ((T*)d.trho_l)[l] = (T)rho;

  if (xbr) {  // FP64 export for the parity tests
    double* o = xbr + (size_t)110 * l;
    for (int r = 0; r < 4; ++r) o[r] = fl[r];
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) o[4 + 6 * r + c] = H[r][c];
    for (int r = 0; r < 4; ++r) { o[40 + r] = aR[r]; o[44 + r] = aI[r]; }
    o[48] = bR;
    o[49] = bI;
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) { o[50 + 4 * r + c] = QH[r][c]; o[70 + 4 * r + c] = F[r][c]; }
    for (int r = 0; r < 4; ++r) { o[66 + r] = gH[r]; o[86 + r] = f0[r]; o[90 + r] = lo[r]; o[94 + r] = hi[r]; }
    for (int e = 0; e < 2; ++e)
      for (int c = 0; c < 4; ++c) o[98 + 4 * e + c] = G[e][c];
    o[106] = grhs[0];
    o[107] = grhs[1];
    o[108] = alo;
    o[109] = ahi;
  }
}

// generators: gradient/curvature of the cost, shifted boxes (opfqpc1-2 with the trust region)
template <typename T>
__global__ void k_build_gen(Dev d, double* xgen, int pass) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= d.G) return;
  int k = d.gen_inst[g];
  if (!live(d.ctl[k], pass)) return;
  double delta = d.ctl[k].delta;
  const double fs = d.ctl[k].fscale;  // objective weight (0 while restoring feasibility)
  double p = d.pg[g], q = d.qg[g];
  double g1 = fs * (2.0 * d.cq[g] * p + d.cl[g]);
  double g2 = fs * 2.0 * d.cq[g];
  double lp, up, lq, uq;
  box_shift(d.pmin[g], d.pmax[g], p, delta, lp, up);
  box_shift(d.qmin[g], d.qmax[g], q, delta, lq, uq);
  d.gd1[g] = g1;
  d.gd2[g] = g2;
  V4<T>* R = (V4<T>*)d.grec;
  V4<T> a, b2;
  a.x = (T)g1; a.y = (T)g2; a.z = (T)lp; a.w = (T)up;
  b2.x = (T)lq; b2.y = (T)uq; b2.z = (T)d.rho_g[g]; b2.w = (T)0;
  R[g] = a;
  R[d.G + g] = b2;
  if (xgen) {
    double* o = xgen + 6 * (size_t)g;
    o[0] = g1; o[1] = g2; o[2] = lp; o[3] = up; o[4] = lq; o[5] = uq;
  }
}

// buses: p_i^{d,(k)}, q_i^{d,(k)} (CSR gather of the branch flows at the bus)
template <typename T>
__global__ void k_build_bus(Dev d, double* xbus, int pass) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.B) return;
  int k = d.bus_inst[i];
  if (!live(d.ctl[k], pass)) return;
  double pk = d.pd[i] + d.gs[i] * d.w[i];
  double qk = d.qd[i] - d.bs[i] * d.w[i];
  for (int g = d.gen_ptr[i]; g < d.gen_ptr[i + 1]; ++g) {
    pk -= d.pg[g];
    qk -= d.qg[g];
  }
  for (int e = d.end_ptr[i]; e < d.end_ptr[i + 1]; ++e) {
    int le = d.end_idx[e], l = le >> 1, s = le & 1;
    pk += d.flow[(2 * s) * d.L + l];
    qk += d.flow[(2 * s + 1) * d.L + l];
  }
  V4<T> v;
  v.x = (T)pk; v.y = (T)qk; v.z = (T)d.gs[i]; v.w = (T)d.bs[i];
  ((V4<T>*)d.brec)[i] = v;
  if (xbus) {
    xbus[2 * (size_t)i] = pk;
    xbus[2 * (size_t)i + 1] = qk;
  }
}

// --------------------------------------------------- step and multipliers
// Step d (eq. elim applied to the bus values) and the multipliers pi of eq. lag
// recovered from the KKT conditions of each line subproblem (Sec. IV-B):
// pi13, pi14 = -(line-limit multipliers); (pi11, pi12) from stationarity in (d_wR, d_wI).
template <typename T>
__global__ void k_step_branch(Dev d, int pass) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= d.L) return;
  int k = d.br_inst[l];
  if (!live(d.ctl[k], pass)) return;
  Br b;
  load_branch(d, l, b);
  const V2<T>* ZB = (const V2<T>*)d.ZB;
  V2<T> zi = ZB[b.i], zj = ZB[b.j];
  double db[4] = {(double)zi.x, (double)zi.y, (double)zj.x, (double)zj.y};
  double aR[4], aI[4];
  for (int r = 0; r < 4; ++r) {
    aR[r] = d.aR[r * d.L + l];
    aI[r] = d.aI[r * d.L + l];
  }
  double bR = d.bR[l], bI = d.bI[l];
  d.dwr[l] = aR[0] * db[0] + aR[1] * db[1] + aR[2] * db[2] + aR[3] * db[3] + bR;
  d.dwi[l] = aI[0] * db[0] + aI[1] * db[1] + aI[2] * db[2] + aI[3] * db[3] + bI;

  // line side dbar, multipliers of the flow couplings, line-limit multipliers
  const V4<T>* X = (const V4<T>*)d.X;
  const V4<T>* LM = (const V4<T>*)d.LAM;
  V4<T> x0 = X[2 * l], x1 = X[2 * l + 1];
  V4<T> l0 = LM[2 * l], l1 = LM[2 * l + 1];
  V4<T> u = ((const V4<T>*)d.U)[l];
  const V4<T>* R = (const V4<T>*)d.lrec;
  V4<T> gsc = R[13 * d.L + l];  // chunk 13: alo ahi |G0| |G1|
  double dl[4] = {(double)x0.z, (double)x0.w, (double)x1.z, (double)x1.w};
  double z[6];
  z[0] = dl[0];
  z[1] = dl[1];
  z[2] = aR[0] * dl[0] + aR[1] * dl[1] + aR[2] * dl[2] + aR[3] * dl[3] + bR;
  z[3] = aI[0] * dl[0] + aI[1] * dl[1] + aI[2] * dl[2] + aI[3] * dl[3] + bI;
  z[4] = dl[2];
  z[5] = dl[3];
  double pi[4];
  for (int r = 0; r < 4; ++r) pi[r] = d.pi[r * d.L + l];
  double H[6][6];
  branch_hessian(b, pi, H);
  double gR = 0, gI = 0;
  for (int q = 0; q < 6; ++q) {
    gR += H[2][q] * z[q];
    gI += H[3][q] * z[q];
  }
  double J[4][6];
  flow_jac(b.Y, J);
  double lam[4] = {(double)l0.x, (double)l0.y, (double)l1.x, (double)l1.y};
  for (int f = 0; f < 4; ++f) {
    gR += lam[f] * J[f][2];
    gI += lam[f] * J[f][3];
  }
  double fl[4];
  for (int r = 0; r < 4; ++r) fl[r] = d.flow[r * d.L + l];
  // normalised rows carry multiplier u_hat = |G| u
  double u13 = (double)gsc.z > 0 ? (double)u.x / (double)gsc.z : 0.0;
  double u14 = (double)gsc.w > 0 ? (double)u.y / (double)gsc.w : 0.0;
  gR += u13 * (2 * fl[0] * J[0][2] + 2 * fl[1] * J[1][2]) + u14 * (2 * fl[2] * J[2][2] + 2 * fl[3] * J[3][2]);
  gI += u13 * (2 * fl[0] * J[0][3] + 2 * fl[1] * J[1][3]) + u14 * (2 * fl[2] * J[2][3] + 2 * fl[3] * J[3][3]);
  double sn, cs;
  sincos(b.thi - b.thj, &sn, &cs);
  double a11 = 2 * b.wr, a12 = sn, a21 = 2 * b.wim, a22 = -cs;
  double det = a11 * a22 - a12 * a21;
  d.pi_new[0 * d.L + l] = (-gR * a22 + gI * a12) / det;
  d.pi_new[1 * d.L + l] = (-gI * a11 + gR * a21) / det;
  d.pi_new[2 * d.L + l] = -u13;
  d.pi_new[3 * d.L + l] = -u14;
}

template <typename T>
__global__ void k_step_nodes(Dev d, int pass) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < d.G) {
    int k = d.gen_inst[n];
    if (live(d.ctl[k], pass)) {
      V2<T> xg = ((const V2<T>*)d.XG)[n];
      d.dpg[n] = (double)xg.x;
      d.dqg[n] = (double)xg.y;
    }
  }
  if (n < d.B) {
    int k = d.bus_inst[n];
    if (live(d.ctl[k], pass)) {
      V2<T> zb = ((const V2<T>*)d.ZB)[n];
      d.dw[n] = (double)zb.x;
      d.dth[n] = (double)zb.y;
    }
  }
}

// ------------------------------------------------------------ merit
// Terms of phi_1 = f + mu h at x and x + d and of the model reduction
// q(0) - q(d) (Sec. II-C).  h sums the l1 violations of all constraints; the
// linear ones (balance, bounds, angle limits) enter h as well because an
// inexact ADMM step does not satisfy them exactly.
//   tbr:  0 nonlinear part of h at x, 1 angle part at x, 2 nonlinear part at x+d,
//         3 angle part at x+d, 4 d'Hd, 5 linearised nonlinear part m, 6 max violation at x+d
//   tbus: 0 h at x, 1 h at x+d, 2 max violation at x+d
//   tgen: 0 h at x, 1 h at x+d, 2 f(x), 3 f(x+d), 4 grad f'd, 5 f'' d^2, 6 max violation at x+d
__device__ __forceinline__ void angle_viol(double th, double amin, double amax, int use, double& s, double& m) {
  if (!use) return;
  if (amin > -kTwoPi) { double v = negpart(th - amin); s += v; m = fmax(m, v); }
  if (amax < kTwoPi) { double v = negpart(amax - th); s += v; m = fmax(m, v); }
}

__global__ void k_merit_branch(Dev d, int use_angle, int pass) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= d.L) return;
  int k = d.br_inst[l];
  if (!live(d.ctl[k], pass)) return;
  Br b;
  load_branch(d, l, b);
  double zs[6] = {d.dw[b.i], d.dth[b.i], d.dwr[l], d.dwi[l], d.dw[b.j], d.dth[b.j]};
  double s2 = d.s2[l] < 0 ? kBig : d.s2[l];
  double fl[4];
  for (int r = 0; r < 4; ++r) fl[r] = d.flow[r * d.L + l];
  double J[4][6];
  flow_jac(b.Y, J);
  double df[4];
  for (int r = 0; r < 4; ++r) {
    double s = 0;
    for (int q = 0; q < 6; ++q) s += J[r][q] * zs[q];
    df[r] = s;
    d.flow_xd[r * d.L + l] = fl[r] + s;
  }
  double sn, cs;
  sincos(b.thi - b.thj, &sn, &cs);
  double D = b.wr * cs + b.wim * sn;
  double c11 = b.wr * b.wr + b.wim * b.wim - b.wi * b.wj;
  double c12 = b.wr * sn - b.wim * cs;
  double c13 = s2 - fl[0] * fl[0] - fl[1] * fl[1];
  double c14 = s2 - fl[2] * fl[2] - fl[3] * fl[3];
  double h0 = fabs(c11) + fabs(c12) + negpart(c13) + negpart(c14);
  double a0s = 0, a0m = 0;
  angle_viol(b.thi - b.thj, d.angmin[l], d.angmax[l], use_angle, a0s, a0m);
  // at x + d
  double wi1 = b.wi + zs[0], wj1 = b.wj + zs[4], wr1 = b.wr + zs[2], wim1 = b.wim + zs[3];
  double th1 = b.thi + zs[1] - b.thj - zs[5];
  double sn1, cs1;
  sincos(th1, &sn1, &cs1);
  double f1[4] = {fl[0] + df[0], fl[1] + df[1], fl[2] + df[2], fl[3] + df[3]};
  double e11 = wr1 * wr1 + wim1 * wim1 - wi1 * wj1;
  double e12 = wr1 * sn1 - wim1 * cs1;
  double e13 = s2 - f1[0] * f1[0] - f1[1] * f1[1];
  double e14 = s2 - f1[2] * f1[2] - f1[3] * f1[3];
  double h1 = fabs(e11) + fabs(e12) + negpart(e13) + negpart(e14);
  double mx = fmax(fmax(fabs(e11), fabs(e12)), fmax(negpart(e13), negpart(e14)));
  double a1s = 0, a1m = 0;
  angle_viol(th1, d.angmin[l], d.angmax[l], use_angle, a1s, a1m);
  mx = fmax(mx, a1m);
  // model: curvature and linearised constraints
  double pi[4];
  for (int r = 0; r < 4; ++r) pi[r] = d.pi[r * d.L + l];
  double H[6][6];
  branch_hessian(b, pi, H);
  double quad = 0;
  for (int a = 0; a < 6; ++a)
    for (int c = 0; c < 6; ++c) quad += zs[a] * H[a][c] * zs[c];
  double l11 = c11 + 2 * b.wr * zs[2] + 2 * b.wim * zs[3] - b.wj * zs[0] - b.wi * zs[4];
  double l12 = c12 + sn * zs[2] - cs * zs[3] + D * (zs[1] - zs[5]);
  double l13 = c13 - 2 * fl[0] * df[0] - 2 * fl[1] * df[1];
  double l14 = c14 - 2 * fl[2] * df[2] - 2 * fl[3] * df[3];
  double ml = fabs(l11) + fabs(l12) + negpart(l13) + negpart(l14);
  double* t = d.tbr;
  int L = d.L;
  t[0 * L + l] = h0;
  t[1 * L + l] = a0s;
  t[2 * L + l] = h1;
  t[3 * L + l] = a1s;
  t[4 * L + l] = quad;
  t[5 * L + l] = ml;
  t[6 * L + l] = mx;
}

__global__ void k_merit_bus(Dev d, int pass) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.B) return;
  int k = d.bus_inst[i];
  if (!live(d.ctl[k], pass)) return;
  double w0 = d.w[i], w1 = d.w[i] + d.dw[i];
  double t0 = d.th[i], t1 = d.th[i] + d.dth[i];
  double p0 = -d.pd[i] - d.gs[i] * w0, q0 = -d.qd[i] + d.bs[i] * w0;
  double p1 = -d.pd[i] - d.gs[i] * w1, q1 = -d.qd[i] + d.bs[i] * w1;
  for (int g = d.gen_ptr[i]; g < d.gen_ptr[i + 1]; ++g) {
    p0 += d.pg[g]; q0 += d.qg[g];
    p1 += d.pg[g] + d.dpg[g]; q1 += d.qg[g] + d.dqg[g];
  }
  for (int e = d.end_ptr[i]; e < d.end_ptr[i + 1]; ++e) {
    int le = d.end_idx[e], l = le >> 1, s = le & 1;
    p0 -= d.flow[(2 * s) * d.L + l];
    q0 -= d.flow[(2 * s + 1) * d.L + l];
    p1 -= d.flow_xd[(2 * s) * d.L + l];
    q1 -= d.flow_xd[(2 * s + 1) * d.L + l];
  }
  double h0 = fabs(p0) + fabs(q0) + negpart(w0 - d.wmin[i]) + negpart(d.wmax[i] - w0);
  double h1 = fabs(p1) + fabs(q1);
  double v1 = negpart(w1 - d.wmin[i]), v2 = negpart(d.wmax[i] - w1);
  h1 += v1 + v2;
  double mx = fmax(fmax(fabs(p1), fabs(q1)), fmax(v1, v2));
  if (d.isref[i]) {
    h0 += fabs(t0);
    h1 += fabs(t1);
    mx = fmax(mx, fabs(t1));
  } else {
    h0 += negpart(t0 + kTwoPi) + negpart(kTwoPi - t0);
    double a = negpart(t1 + kTwoPi), bq = negpart(kTwoPi - t1);
    h1 += a + bq;
    mx = fmax(mx, fmax(a, bq));
  }
  d.tbus[0 * d.B + i] = h0;
  d.tbus[1 * d.B + i] = h1;
  d.tbus[2 * d.B + i] = mx;
}

__global__ void k_merit_gen(Dev d, int pass) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= d.G) return;
  int k = d.gen_inst[g];
  if (!live(d.ctl[k], pass)) return;
  double p0 = d.pg[g], q0 = d.qg[g];
  double p1 = p0 + d.dpg[g], q1 = q0 + d.dqg[g];
  double h0 = negpart(p0 - d.pmin[g]) + negpart(d.pmax[g] - p0) + negpart(q0 - d.qmin[g]) + negpart(d.qmax[g] - q0);
  double a = negpart(p1 - d.pmin[g]), bq = negpart(d.pmax[g] - p1), c = negpart(q1 - d.qmin[g]),
         e = negpart(d.qmax[g] - q1);
  double* t = d.tgen;
  int G = d.G;
  t[0 * G + g] = h0;
  t[1 * G + g] = a + bq + c + e;
  t[2 * G + g] = d.cq[g] * p0 * p0 + d.cl[g] * p0 + d.cc[g];
  t[3 * G + g] = d.cq[g] * p1 * p1 + d.cl[g] * p1 + d.cc[g];
  t[4 * G + g] = d.gd1[g] * d.dpg[g];
  t[5 * G + g] = d.gd2[g] * d.dpg[g] * d.dpg[g];
  t[6 * G + g] = fmax(fmax(a, bq), fmax(c, e));
}

// deterministic per-instance reduction of nt rows of a term array over the
// instance's segment [off[k], off[k+1]); op 0 = sum, 1 = max.  One CTA per instance.
template <int NT>
__device__ void seg_reduce(const double* t, int n, int beg, int end, const int* ops, double* out) {
  __shared__ double sh[NT][256];
  double acc[NT];
  for (int r = 0; r < NT; ++r) acc[r] = 0.0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x)
    for (int r = 0; r < NT; ++r) {
      double v = t[(size_t)r * n + i];
      acc[r] = ops[r] ? fmax(acc[r], v) : acc[r] + v;
    }
  for (int r = 0; r < NT; ++r) sh[r][threadIdx.x] = acc[r];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int r = 0; r < NT; ++r)
        sh[r][threadIdx.x] = ops[r] ? fmax(sh[r][threadIdx.x], sh[r][threadIdx.x + s]) : sh[r][threadIdx.x] + sh[r][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int r = 0; r < NT; ++r) out[r] = sh[r][0];
  __syncthreads();
}

// the ratio test of Sec. II-C: ared > 0 and ared / pred > 0
__device__ __forceinline__ bool ratio_ok(double ared, double pred) {
  return isfinite(ared) && isfinite(pred) && ared > 0 && pred > 0;
}

// l1 merit acceptance (Sec. II-C) and trust-region update (Alg. 1, acceptance
// and radius rules).  Main pass (0): the QP step d.  When d fails the test and
// second-order correction is on (with a positive model reduction), the
// decision waits for the correction pass (1), which judges the corrected step
// against d's model reduction; the radius rule then uses the accepted step's
// norm, or d's on rejection.
__global__ void __launch_bounds__(256) k_decide(Dev d, int pass) {
  int k = blockIdx.x;
  InstCtl& c = d.ctl[k];
  if (!live(c, pass)) return;
  __shared__ double rb[7], rbus[3], rg[7];
  const int opb[7] = {0, 0, 0, 0, 0, 0, 1};
  const int opbus[3] = {0, 0, 1};
  const int opg[7] = {0, 0, 0, 0, 0, 0, 1};
  seg_reduce<7>(d.tbr, d.L, d.br_off[k], d.br_off[k + 1], opb, rb);
  seg_reduce<3>(d.tbus, d.B, d.bus_off[k], d.bus_off[k + 1], opbus, rbus);
  seg_reduce<7>(d.tgen, d.G, d.gen_off[k], d.gen_off[k + 1], opg, rg);
  if (threadIdx.x != 0) return;
  if (pass == 0) {
    c.admm_iter_last = d.admm_iters[k];
  } else {
    c.admm_iter_last += d.admm_iters[k];
  }
  c.admm_iter_total += d.admm_iters[k];
  c.r_inf = d.admm_rs[k];
  c.s_inf = d.admm_rs[d.K + k];
  double mu = c.mu;
  // with merit_linear = 0, h is the paper's literal one: nonlinear constraints only
  double wl = c.merit_linear ? 1.0 : 0.0;
  double h0 = rb[0] + wl * (rb[1] + rbus[0] + rg[0]);
  double lin1 = wl * (rb[3] + rbus[1] + rg[1]);     // linear constraints at x + d
  double h1 = rb[2] + lin1;
  const double fs = c.fscale;                        // objective weight (0 while restoring)
  double f0 = rg[2], f1 = rg[3];
  double phx = fs * f0 + mu * h0, phxd = fs * f1 + mu * h1;
  double md = rb[5] + lin1;
  double pred = -rg[4] - 0.5 * (rg[5] + rb[4]) + mu * (h0 - md);
  double ared = phx - phxd;
  // step norm over the trust-region variables (pg, qg, w, theta)
  double dn = d.red[16 * k + 0];
  if (c.sqp_iter == 0 && pass == 0) {  // objective and infeasibility of the starting point
    c.obj = f0;
    c.primal = fmax(fmax(rb[6], rbus[2]), rg[6]);
  }
  int accept;
  if (pass == 0) {
    accept = ratio_ok(ared, pred);
    c.soc_flag = 0;
    if (!accept && c.soc_on && isfinite(pred) && pred > 0) {
      c.soc_active = 1;
      c.phx_saved = phx;
      c.pred_saved = pred;
      c.dn_saved = dn;
      c.ared_saved = ared;
      return;  // decided by the correction pass
    }
  } else {
    // the corrected step: merit at x + d' against the original model reduction
    const double ared2 = c.phx_saved - phxd;
    pred = c.pred_saved;
    c.soc_active = 0;
    accept = ratio_ok(ared2, pred);
    c.soc_flag = accept ? 2 : 1;
    if (accept) {
      ared = ared2;
    } else {
      ared = c.ared_saved;
      dn = c.dn_saved;
    }
  }
  c.ared = ared;
  c.pred = pred;
  c.dnorm = dn;
  c.accept_last = accept;
  c.sqp_iter += 1;
  if (accept) {
    c.accepted += 1;
    if (dn >= 0.99 * c.delta) c.delta = fmin(2 * c.delta, c.delta_max);
    c.obj = f1;
    c.primal = fmax(fmax(rb[6], rbus[2]), rg[6]);
  } else {
    c.delta = 0.5 * fmin(c.delta, dn);
  }
}

// l_inf norm of the step over (pg, qg, w, theta), per instance
__global__ void __launch_bounds__(256) k_step_norm(Dev d, int pass) {
  int k = blockIdx.x;
  if (!live(d.ctl[k], pass)) return;
  __shared__ double sh[256];
  double m = 0;
  for (int g = d.gen_off[k] + threadIdx.x; g < d.gen_off[k + 1]; g += blockDim.x)
    m = fmax(m, fmax(fabs(d.dpg[g]), fabs(d.dqg[g])));
  for (int i = d.bus_off[k] + threadIdx.x; i < d.bus_off[k + 1]; i += blockDim.x)
    m = fmax(m, fmax(fabs(d.dw[i]), fabs(d.dth[i])));
  if (!isfinite(m)) m = kBig;
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) d.red[16 * k + 0] = sh[0];
}

// x <- x + d and pi <- pi_new on acceptance
__global__ void k_apply(Dev d) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < d.G) {
    const InstCtl& c = d.ctl[d.gen_inst[n]];
    if (c.result == ACOPF_RUNNING && c.accept_last) {
      d.pg[n] += d.dpg[n];
      d.qg[n] += d.dqg[n];
    }
  }
  if (n < d.B) {
    const InstCtl& c = d.ctl[d.bus_inst[n]];
    if (c.result == ACOPF_RUNNING && c.accept_last) {
      d.w[n] += d.dw[n];
      d.th[n] += d.dth[n];
    }
  }
  if (n < d.L) {
    const InstCtl& c = d.ctl[d.br_inst[n]];
    if (c.result == ACOPF_RUNNING && c.accept_last) {
      d.wr[n] += d.dwr[n];
      d.wi[n] += d.dwi[n];
      for (int r = 0; r < 4; ++r) d.pi[r * d.L + n] = d.pi_new[r * d.L + n];
    }
  }
}

// ------------------------------------------------------------ KKT
// Dual infeasibility at the new iterate: gradient of the Lagrangian with the
// QP's multipliers (bus power-balance nu, pi of eq. lag, angle-row
// multipliers), projected at active variable bounds.
//   tbr[7]: max |dL/dwR|, |dL/dwI|;  dend[2][2L]: per-end (w, theta) contributions
template <typename T>
__global__ void k_dual_branch(Dev d, int use_angle) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= d.L) return;
  int k = d.br_inst[l];
  if (d.ctl[k].result != ACOPF_RUNNING || !d.ctl[k].accept_last) return;
  Br b;
  load_branch(d, l, b);
  const V2<T>* NU = (const V2<T>*)d.NU;
  V2<T> ni = NU[b.i], nj = NU[b.j];
  double J[4][6];
  flow_jac(b.Y, J);
  double fl[4];
  flows_at(b.Y, b.wi, b.wj, b.wr, b.wim, fl);
  double sn, cs;
  sincos(b.thi - b.thj, &sn, &cs);
  double D = b.wr * cs + b.wim * sn;
  double p[4];
  for (int r = 0; r < 4; ++r) p[r] = d.pi[r * d.L + l];
  double gz[6];
  for (int q = 0; q < 6; ++q) {
    gz[q] = -(double)ni.x * J[0][q] - (double)ni.y * J[1][q] - (double)nj.x * J[2][q] - (double)nj.y * J[3][q];
    gz[q] += p[2] * (-2 * fl[0] * J[0][q] - 2 * fl[1] * J[1][q]) + p[3] * (-2 * fl[2] * J[2][q] - 2 * fl[3] * J[3][q]);
  }
  gz[0] += -p[0] * b.wj;
  gz[4] += -p[0] * b.wi;
  gz[2] += 2 * p[0] * b.wr;
  gz[3] += 2 * p[0] * b.wim;
  gz[1] += p[1] * D;
  gz[5] -= p[1] * D;
  gz[2] += p[1] * sn;
  gz[3] -= p[1] * cs;
  if (use_angle) {
    V4<T> u = ((const V4<T>*)d.U)[l];
    double uh = (double)u.z, ulo = (double)u.w;
    gz[1] += uh - ulo;
    gz[5] += -uh + ulo;
  }
  int L2 = 2 * d.L;
  d.dend[0 * L2 + 2 * l] = gz[0];
  d.dend[1 * L2 + 2 * l] = gz[1];
  d.dend[0 * L2 + 2 * l + 1] = gz[4];
  d.dend[1 * L2 + 2 * l + 1] = gz[5];
  d.tbr[7 * d.L + l] = fmax(fabs(gz[2]), fabs(gz[3]));
}

__device__ __forceinline__ double project_bound(double v, double x, double lb, double ub) {
  const double tact = 1e-5;
  if (x - lb <= tact && v > 0) v = 0;
  if (ub - x <= tact && v < 0) v = 0;
  return fabs(v);
}

//   tbus[3]: max projected |dL/dw|, |dL/dtheta| at the bus;  tgen[7]: generator residual, tgen[0] reused: |f'|
template <typename T>
__global__ void k_dual_nodes(Dev d) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  const V2<T>* NU = (const V2<T>*)d.NU;
  if (n < d.B) {
    int k = d.bus_inst[n];
    if (d.ctl[k].result == ACOPF_RUNNING && d.ctl[k].accept_last) {
      V2<T> nu = NU[n];
      double gw = -d.gs[n] * (double)nu.x + d.bs[n] * (double)nu.y, gt = 0;
      int L2 = 2 * d.L;
      for (int e = d.end_ptr[n]; e < d.end_ptr[n + 1]; ++e) {
        int le = d.end_idx[e];
        gw += d.dend[0 * L2 + le];
        gt += d.dend[1 * L2 + le];
      }
      double r = project_bound(gw, d.w[n], d.wmin[n], d.wmax[n]);
      if (!d.isref[n]) r = fmax(r, fabs(gt));
      d.tbus[3 * d.B + n] = r;
    }
  }
  if (n < d.G) {
    int k = d.gen_inst[n];
    if (d.ctl[k].result == ACOPF_RUNNING && d.ctl[k].accept_last) {
      V2<T> nu = NU[d.gbus[n]];
      double gf = 2.0 * d.cq[n] * d.pg[n] + d.cl[n];
      double rp = project_bound(gf + (double)nu.x, d.pg[n], d.pmin[n], d.pmax[n]);
      double rq = project_bound((double)nu.y, d.qg[n], d.qmin[n], d.qmax[n]);
      d.tgen[7 * d.G + n] = fmax(rp, rq);
      d.tgen[0 * d.G + n] = fabs(gf);
    }
  }
}

__global__ void __launch_bounds__(256) k_kkt_decide(Dev d) {
  int k = blockIdx.x;
  InstCtl& c = d.ctl[k];
  if (c.result != ACOPF_RUNNING) return;
  __shared__ double a[1], bsh[1], gg[2];
  if (c.accept_last) {
    const int op1[1] = {1};
    seg_reduce<1>(d.tbr + 7 * (size_t)d.L, d.L, d.br_off[k], d.br_off[k + 1], op1, a);
    seg_reduce<1>(d.tbus + 3 * (size_t)d.B, d.B, d.bus_off[k], d.bus_off[k + 1], op1, bsh);
    // rows 0 (|f'|) and 7 (generator residual) of tgen
    seg_reduce<1>(d.tgen, d.G, d.gen_off[k], d.gen_off[k + 1], op1, gg);
    seg_reduce<1>(d.tgen + 7 * (size_t)d.G, d.G, d.gen_off[k], d.gen_off[k + 1], op1, gg + 1);
  }
  if (threadIdx.x != 0) return;
  if (c.accept_last) c.dual = fmax(fmax(a[0], bsh[0]), gg[1]) / fmax(1.0, gg[0]);
  if (c.sqp_iter >= 1 && c.sqp_iter <= ACOPF_HIST_MAX) {
    double* hr = d.hist + ((size_t)k * ACOPF_HIST_MAX + (c.sqp_iter - 1)) * kHistW;
    hr[0] = c.obj; hr[1] = c.primal; hr[2] = c.dual; hr[3] = c.admm_iter_last;
    hr[4] = c.r_inf; hr[5] = c.s_inf; hr[6] = c.accept_last; hr[7] = c.delta;
    hr[8] = c.dnorm; hr[9] = c.ared; hr[10] = c.pred; hr[11] = d.rho_fac[k];
    hr[12] = c.soc_flag; hr[13] = c.restoring;
  }
  // no progress towards feasibility: the infeasibility, above 10 tol, has not
  // fallen by a tenth over the last five iterations (of the current phase)
  const int it = c.sqp_iter - 1;
  const double older = c.primal_ring[it % 5];
  c.primal_ring[it % 5] = c.primal;
  const bool no_progress = it >= 5 && c.primal > 10 * c.tol && c.primal > 0.9 * older && c.since_switch >= 5;
  c.since_switch += 1;
  const bool stall = (c.accept_last && c.dnorm <= c.step_tol) || c.delta < c.delta_min;
  if (!isfinite(c.obj) || !isfinite(c.primal) || !isfinite(c.dual) || !isfinite(c.delta)) {
    c.result = ACOPF_NONFINITE;
  } else if (!c.restoring) {
    if (c.accept_last && c.primal <= c.tol && c.dual <= c.tol) {
      c.result = ACOPF_CONVERGED;
    } else if (stall || (c.restore_on && no_progress)) {
      if (c.restore_on && c.primal > c.tol) {
        // feasibility restoration: the violation alone (objective weight 0,
        // merit mu h) from the current point and radius delta0
        c.restoring = 1;
        c.fscale = 0.0;
        c.delta = c.delta0;
        c.since_switch = 0;
      } else {
        c.result = ACOPF_STEP_TOO_SMALL;
      }
    }
  } else {
    if (c.accept_last && c.primal <= c.tol) {  // feasible again: back to the SQP on the ACOPF
      c.restoring = 0;
      c.fscale = 1.0;
      c.delta = c.delta0;
      c.since_switch = 0;
    } else if (stall || no_progress) {
      c.result = ACOPF_INFEASIBLE;  // the violation stalls above tol: locally infeasible
    }
  }
}

__global__ void k_count_running(Dev d) {
  __shared__ int n;
  if (threadIdx.x == 0) n = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < d.K; k += blockDim.x)
    if (d.ctl[k].result == ACOPF_RUNNING) atomicAdd(&n, 1);
  __syncthreads();
  if (threadIdx.x == 0) *d.n_running = n;
}

__global__ void k_finish(Dev d) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < d.K && d.ctl[k].result == ACOPF_RUNNING) d.ctl[k].result = ACOPF_MAXITER;
}

__global__ void k_fill_rho(Dev d, double rho) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < d.L) d.rho_l[n] = rho;
  if (n < d.G) d.rho_g[n] = rho;
}

// ------------------------------------------------------------ launchers
static inline unsigned cover(const Dev& d) {
  int m = d.L;
  if (d.B > m) m = d.B;
  if (d.G > m) m = d.G;
  return nblk(m, 256);
}

// Warm start of every instance from a prediction row per instance (layout of
// acopf_set_warm_start_device): NLP point clamped into its bounds, line
// multipliers pi, ADMM multipliers in the sweep precision, per-component
// penalties.  Grid (ceil(max(B, L, G) / 256), K).
template <typename T>
__global__ void k_warm_scatter(Dev d, const float* pred, long long ld, const int* gen_iperm, int nb, int nl, int ng,
                               double base_rho, int use_x, int use_pi, int use_lam, int use_rho) {
  const int k = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const float* p = pred + (size_t)k * (size_t)ld;
  const int b0 = d.bus_off[k], l0 = d.br_off[k], g0 = d.gen_off[k];
  const int opi = 2 * ng + 2 * nb + 2 * nl, olam = opi + 4 * nl, orho = olam + 8 * nl + 2 * ng;
  if (use_x) {
    if (j < ng) {
      const int g = gen_iperm[g0 + j];
      d.pg[g] = fmin(fmax((double)p[j], d.pmin[g]), d.pmax[g]);
      d.qg[g] = fmin(fmax((double)p[ng + j], d.qmin[g]), d.qmax[g]);
    }
    if (j < nb) {
      const int i = b0 + j;
      d.w[i] = fmin(fmax((double)p[2 * ng + j], d.wmin[i]), d.wmax[i]);
      d.th[i] = d.isref[i] ? 0.0 : (double)p[2 * ng + nb + j];
    }
    if (j < nl) {
      d.wr[l0 + j] = (double)p[2 * ng + 2 * nb + j];
      d.wi[l0 + j] = (double)p[2 * ng + 2 * nb + nl + j];
      for (int r = 0; r < 4; ++r) d.pi[(size_t)r * d.L + l0 + j] = use_pi ? (double)p[opi + 4 * j + r] : 0.0;
    }
  }
  if (use_lam) {
    if (j < nl) {
      const float* q = p + olam + 8 * j;  // p_ij q_ij p_ji q_ji w_i th_i w_j th_j
      V4<T> e0 = {(T)q[0], (T)q[1], (T)q[4], (T)q[5]};
      V4<T> e1 = {(T)q[2], (T)q[3], (T)q[6], (T)q[7]};
      ((V4<T>*)d.LAM)[2 * (l0 + j)] = e0;
      ((V4<T>*)d.LAM)[2 * (l0 + j) + 1] = e1;
    }
    if (j < ng) {
      const int g = gen_iperm[g0 + j];
      V2<T> v = {(T)p[olam + 8 * nl + 2 * j], (T)p[olam + 8 * nl + 2 * j + 1]};
      ((V2<T>*)d.LG)[g] = v;
    }
  }
  if (use_rho) {
    if (j < nl) d.rho_l[l0 + j] = base_rho * exp(fmin(fmax((double)p[orho + j], -2.3), 2.3));
    if (j < ng) d.rho_g[gen_iperm[g0 + j]] = base_rho * exp(fmin(fmax((double)p[orho + nl + j], -2.3), 2.3));
  }
}

void launch_warm_scatter(Ctx& c, const float* pred, long long ld, int nb, int nl, int ng, double base_rho, int use_x,
                         int use_pi, int use_lam, int use_rho) {
  int m = nb > nl ? nb : nl;
  m = m > ng ? m : ng;
  dim3 grid(nblk(m, 256), c.d.K);
  if (c.precision == ACOPF_MIXED)
    k_warm_scatter<float><<<grid, 256, 0, c.stream>>>(c.d, pred, ld, c.d_gen_iperm, nb, nl, ng, base_rho, use_x,
                                                       use_pi, use_lam, use_rho);
  else
    k_warm_scatter<double><<<grid, 256, 0, c.stream>>>(c.d, pred, ld, c.d_gen_iperm, nb, nl, ng, base_rho, use_x,
                                                        use_pi, use_lam, use_rho);
  c.launches++;
}

void launch_flat_start(Ctx& c) {
  k_flat_start<<<cover(c.d), 256, 0, c.stream>>>(c.d);
  c.launches++;
}

void launch_finish(Ctx& c) {
  k_finish<<<nblk(c.d.K, 256), 256, 0, c.stream>>>(c.d);
  c.launches++;
}

void launch_fill_rho(Ctx& c, double rho) {
  k_fill_rho<<<cover(c.d), 256, 0, c.stream>>>(c.d, rho);
  c.launches++;
}

void launch_build(Ctx& c, bool do_export, int pass) {
  Dev& d = c.d;
  double* xb = do_export ? d.xbr : nullptr;
  double* xg = do_export ? d.xgen : nullptr;
  double* xs = do_export ? d.xbus : nullptr;
  if (c.precision == ACOPF_MIXED) {
    k_build_branch<float><<<nblk(d.L, 128), 128, 0, c.stream>>>(d, c.use_angle, xb, pass);
    k_build_gen<float><<<nblk(d.G, 256), 256, 0, c.stream>>>(d, xg, pass);
    k_build_bus<float><<<nblk(d.B, 256), 256, 0, c.stream>>>(d, xs, pass);
  } else {
    k_build_branch<double><<<nblk(d.L, 128), 128, 0, c.stream>>>(d, c.use_angle, xb, pass);
    k_build_gen<double><<<nblk(d.G, 256), 256, 0, c.stream>>>(d, xg, pass);
    k_build_bus<double><<<nblk(d.B, 256), 256, 0, c.stream>>>(d, xs, pass);
  }
  c.launches += 3;
}

void launch_step(Ctx& c, int pass) {
  Dev& d = c.d;
  if (c.precision == ACOPF_MIXED) {
    k_step_branch<float><<<nblk(d.L, 128), 128, 0, c.stream>>>(d, pass);
    k_step_nodes<float><<<cover(d), 256, 0, c.stream>>>(d, pass);
  } else {
    k_step_branch<double><<<nblk(d.L, 128), 128, 0, c.stream>>>(d, pass);
    k_step_nodes<double><<<cover(d), 256, 0, c.stream>>>(d, pass);
  }
  c.launches += 2;
}

void launch_merit(Ctx& c, int pass) {
  Dev& d = c.d;
  k_merit_branch<<<nblk(d.L, 128), 128, 0, c.stream>>>(d, c.use_angle, pass);
  k_merit_bus<<<nblk(d.B, 256), 256, 0, c.stream>>>(d, pass);
  k_merit_gen<<<nblk(d.G, 256), 256, 0, c.stream>>>(d, pass);
  k_step_norm<<<d.K, 256, 0, c.stream>>>(d, pass);
  k_decide<<<d.K, 256, 0, c.stream>>>(d, pass);
  c.launches += 5;
}

void launch_accept_and_kkt(Ctx& c) {
  Dev& d = c.d;
  k_apply<<<cover(d), 256, 0, c.stream>>>(d);
  if (c.precision == ACOPF_MIXED) {
    k_dual_branch<float><<<nblk(d.L, 128), 128, 0, c.stream>>>(d, c.use_angle);
    k_dual_nodes<float><<<cover(d), 256, 0, c.stream>>>(d);
  } else {
    k_dual_branch<double><<<nblk(d.L, 128), 128, 0, c.stream>>>(d, c.use_angle);
    k_dual_nodes<double><<<cover(d), 256, 0, c.stream>>>(d);
  }
  k_kkt_decide<<<d.K, 256, 0, c.stream>>>(d);
  k_count_running<<<1, 256, 0, c.stream>>>(d);
  c.launches += 5;
}

void launch_admittance(Ctx& c, const double* r, const double* x, const double* b, const double* tap,
                       const double* shift) {
  k_admittance<<<nblk(c.d.L, 256), 256, 0, c.stream>>>(c.d.L, r, x, b, tap, shift, c.d.Y);
  c.launches++;
}

}  // namespace acopf
