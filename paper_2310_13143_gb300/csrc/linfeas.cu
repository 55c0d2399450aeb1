// Linear feasibility projection (Sec. II, eq. linfeas; the initial feasibility step of Alg. 1): the
// current iterate x0 of every instance is replaced by the nearest point, in
// the Euclidean norm, that satisfies the NLP's linear constraints -- the bus
// power balances (eq. opfc5, opfc6 with the flows of eq. acopf_pf, linear in
// w, wR, wI) and the bounds on pg, qg, w and theta (opfc1-4), theta_ref = 0.
//
// It is solved by the same component decomposition as the QP (Alg. 2), in
// FP64:
//   generator g   min (pg - pg0)^2 + (qg - qg0)^2 + ADMM terms, box: closed form;
//   branch l      variables v = (w_i, wR, wI, w_j): its own wR, wI and copies of
//                 the end-bus voltages, flows F v; min (wR - wR0)^2 + (wI - wI0)^2
//                 + ADMM terms on the 4 flows and 2 voltage copies, box on the
//                 copies: a 4-variable box QP solved exactly by the active-set
//                 method of the line subproblem;
//   bus i         the 2x2 system of its balance rows (right-hand side pd, qd)
//                 with its own voltage term (w - w0)^2 added to the voltage row;
//                 multiplier update and residuals.
// theta does not appear in any balance row, so its projection is the clamp
// into [-2 pi, 2 pi] (0 at the reference bus).
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "line_qp.cuh"

namespace acopf {

typedef V4<double> D4;  // 32-byte aligned (p, q, w, -) of a branch end

__device__ __forceinline__ D4 d4(double a, double b, double c, double e) {
  D4 v;
  v.x = a; v.y = b; v.z = c; v.w = e;
  return v;
}

struct LfState {
  D4 *X, *Z, *LAM;     // [2L]: per branch end (p, q, w, -)
  double2 *XG, *ZG, *LG;    // [G]: (p, q)
  double2* own;             // [L]: the branch's (wR, wI)
  double* WB;               // [B]: bus voltage w
  double* x0;               // start point: pg0 [G] | qg0 [G] | w0 [B] | wR0 [L] | wI0 [L]
  unsigned long long* res;  // [2K]: per-instance max r, s (bits of non-negative doubles)
};

// flow rows of branch l over v = (w_i, wR, wI, w_j) (eq. acopf_pf):
//   p_ij = gii w_i + gij wR + bij wI      q_ij = -bii w_i - bij wR + gij wI
//   p_ji = gjj w_j + gji wR - bji wI      q_ji = -bjj w_j - bji wR - gji wI
__device__ __forceinline__ void lf_rows(const Dev& d, int l, double F[4][4]) {
  const size_t L = d.L;
  const double gii = d.Y[l], bii = d.Y[L + l], gij = d.Y[2 * L + l], bij = d.Y[3 * L + l];
  const double gji = d.Y[4 * L + l], bji = d.Y[5 * L + l], gjj = d.Y[6 * L + l], bjj = d.Y[7 * L + l];
  F[0][0] = gii;  F[0][1] = gij;  F[0][2] = bij;  F[0][3] = 0.0;
  F[1][0] = -bii; F[1][1] = -bij; F[1][2] = gij;  F[1][3] = 0.0;
  F[2][0] = 0.0;  F[2][1] = gji;  F[2][2] = -bji; F[2][3] = gjj;
  F[3][0] = 0.0;  F[3][1] = -bji; F[3][2] = -gji; F[3][3] = -bjj;
}

__global__ void k_lf_init(Dev d, LfState s) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int G = d.G, B = d.B, L = d.L;
  double* pg0 = s.x0;
  double* qg0 = s.x0 + G;
  double* w0 = s.x0 + 2 * G;
  double* wr0 = w0 + B;
  double* wi0 = wr0 + L;
  if (n < G) {
    pg0[n] = d.pg[n];
    qg0[n] = d.qg[n];
    s.XG[n] = s.ZG[n] = make_double2(d.pg[n], d.qg[n]);
    s.LG[n] = make_double2(0.0, 0.0);
  }
  if (n < B) {
    w0[n] = d.w[n];
    s.WB[n] = d.w[n];
  }
  if (n < L) {
    wr0[n] = d.wr[n];
    wi0[n] = d.wi[n];
    double F[4][4];
    lf_rows(d, n, F);
    const double v[4] = {d.w[d.f[n]], d.wr[n], d.wi[n], d.w[d.t[n]]};
    double fl[4];
    for (int r = 0; r < 4; ++r) fl[r] = F[r][0] * v[0] + F[r][1] * v[1] + F[r][2] * v[2] + F[r][3] * v[3];
    s.X[2 * n] = s.Z[2 * n] = d4(fl[0], fl[1], v[0], 0.0);
    s.X[2 * n + 1] = s.Z[2 * n + 1] = d4(fl[2], fl[3], v[3], 0.0);
    s.LAM[2 * n] = s.LAM[2 * n + 1] = d4(0.0, 0.0, 0.0, 0.0);
    s.own[n] = make_double2(d.wr[n], d.wi[n]);
  }
}

// generators and branches (one thread each)
__global__ void k_lf_components(Dev d, LfState s, double rho) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int G = d.G, B = d.B, L = d.L;
  if (u < G) {
    const double2 z = s.ZG[u], lm = s.LG[u];
    const double pg0 = s.x0[u], qg0 = s.x0[G + u];
    s.XG[u] = make_double2(clampv((2.0 * pg0 - lm.x + rho * z.x) / (2.0 + rho), d.pmin[u], d.pmax[u]),
                           clampv((2.0 * qg0 - lm.y + rho * z.y) / (2.0 + rho), d.qmin[u], d.qmax[u]));
    return;
  }
  const int l = u - G;
  if (l >= L) return;
  const double wr0 = s.x0[2 * G + B + l], wi0 = s.x0[2 * G + B + L + l];
  double F[4][4];
  lf_rows(d, l, F);
  const D4 z0 = s.Z[2 * l], z1 = s.Z[2 * l + 1], l0 = s.LAM[2 * l], l1 = s.LAM[2 * l + 1];
  const double zf[4] = {z0.x, z0.y, z1.x, z1.y}, lf[4] = {l0.x, l0.y, l1.x, l1.y};
  // Q = rho F'F + diag(rho, 2, 2, rho), packed; c = F'(lambda_f - rho z_f) + (copies, -2 wR0, -2 wI0)
  double h[10], c[4];
  for (int a = 0; a < 4; ++a) {
    for (int b = a; b < 4; ++b) {
      double q = 0.0;
      for (int r = 0; r < 4; ++r) q += F[r][a] * F[r][b];
      h[pk(a, b)] = rho * q;
    }
    double cc = 0.0;
    for (int r = 0; r < 4; ++r) cc += F[r][a] * (lf[r] - rho * zf[r]);
    c[a] = cc;
  }
  h[pk(0, 0)] += rho;
  h[pk(3, 3)] += rho;
  h[pk(1, 1)] += 2.0;
  h[pk(2, 2)] += 2.0;
  c[0] += l0.z - rho * z0.z;
  c[3] += l1.z - rho * z1.z;
  c[1] -= 2.0 * wr0;
  c[2] -= 2.0 * wi0;
  const int fi = d.f[l], ti = d.t[l];
  const double lo[4] = {d.wmin[fi], -kBig, -kBig, d.wmin[ti]};
  const double hi[4] = {d.wmax[fi], kBig, kBig, d.wmax[ti]};
  const double2 ow = s.own[l];
  double v[4] = {clampv(z0.z, lo[0], hi[0]), ow.x, ow.y, clampv(z1.z, lo[3], hi[3])};
  box_qp(h, c, lo, hi, v, 12);
  double fl[4];
  for (int r = 0; r < 4; ++r) fl[r] = F[r][0] * v[0] + F[r][1] * v[1] + F[r][2] * v[2] + F[r][3] * v[3];
  s.X[2 * l] = d4(fl[0], fl[1], v[0], 0.0);
  s.X[2 * l + 1] = d4(fl[2], fl[3], v[3], 0.0);
  s.own[l] = make_double2(v[1], v[2]);
}

// buses (one thread each): balance rows with right-hand side (pd, qd), the
// voltage row with the bus's own term (w - w0)^2, multipliers, residuals
__global__ void k_lf_buses(Dev d, LfState s, double rho) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.B) return;
  const int k = d.bus_inst[i];
  const int g0 = d.gen_ptr[i], g1 = d.gen_ptr[i + 1], e0 = d.end_ptr[i], e1 = d.end_ptr[i + 1];
  double M = 0.0, v1 = 0.0, v2 = 0.0, Qw = 2.0, cw = 2.0 * s.x0[2 * d.G + i];
  for (int g = g0; g < g1; ++g) {
    const double2 x = s.XG[g], lm = s.LG[g];
    M += 1.0 / rho;
    v1 += (lm.x + rho * x.x) / rho;
    v2 += (lm.y + rho * x.y) / rho;
  }
  for (int e = e0; e < e1; ++e) {
    const int le = d.end_idx[e];
    const D4 x = s.X[le], lm = s.LAM[le];
    M += 1.0 / rho;
    v1 -= (lm.x + rho * x.x) / rho;
    v2 -= (lm.y + rho * x.y) / rho;
    Qw += rho;
    cw += lm.z + rho * x.z;
  }
  const double gsh = d.gs[i], bsh = d.bs[i];
  const double M11 = M + gsh * gsh / Qw, M22 = M + bsh * bsh / Qw, M12 = -gsh * bsh / Qw;
  v1 += -gsh * cw / Qw - d.pd[i];
  v2 += bsh * cw / Qw - d.qd[i];
  const double det = M11 * M22 - M12 * M12;
  const double n1 = (M22 * v1 - M12 * v2) / det, n2 = (M11 * v2 - M12 * v1) / det;
  const double w = (cw + gsh * n1 - bsh * n2) / Qw;
  s.WB[i] = w;
  double rm = 0.0, sm = 0.0;
  for (int g = g0; g < g1; ++g) {
    const double2 x = s.XG[g], lm = s.LG[g], zo = s.ZG[g];
    const double2 zn = make_double2((lm.x + rho * x.x - n1) / rho, (lm.y + rho * x.y - n2) / rho);
    rm = fmax(rm, fmax(fabs(x.x - zn.x), fabs(x.y - zn.y)));
    sm = fmax(sm, rho * fmax(fabs(zn.x - zo.x), fabs(zn.y - zo.y)));
    s.ZG[g] = zn;
    s.LG[g] = make_double2(lm.x + rho * (x.x - zn.x), lm.y + rho * (x.y - zn.y));
  }
  for (int e = e0; e < e1; ++e) {
    const int le = d.end_idx[e];
    const D4 x = s.X[le], lm = s.LAM[le], zo = s.Z[le];
    const D4 zn = d4((lm.x + rho * x.x + n1) / rho, (lm.y + rho * x.y + n2) / rho, w, 0.0);
    rm = fmax(rm, fmax(fmax(fabs(x.x - zn.x), fabs(x.y - zn.y)), fabs(x.z - zn.z)));
    sm = fmax(sm, rho * fmax(fmax(fabs(zn.x - zo.x), fabs(zn.y - zo.y)), fabs(zn.z - zo.z)));
    s.Z[le] = zn;
    s.LAM[le] = d4(lm.x + rho * (x.x - zn.x), lm.y + rho * (x.y - zn.y), lm.z + rho * (x.z - zn.z), 0.0);
  }
  if (!(rm == rm)) rm = kBig;
  if (!(sm == sm)) sm = kBig;
  atomicMax(&s.res[k], (unsigned long long)__double_as_longlong(rm));
  atomicMax(&s.res[d.K + k], (unsigned long long)__double_as_longlong(sm));
}

// the projection into the iterate: generators from their (box-feasible)
// update, w from the bus values (clamped), theta clamped, wR and wI from the
// branches
__global__ void k_lf_finish(Dev d, LfState s) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < d.G) {
    d.pg[n] = s.XG[n].x;
    d.qg[n] = s.XG[n].y;
  }
  if (n < d.B) {
    d.w[n] = clampv(s.WB[n], d.wmin[n], d.wmax[n]);
    d.th[n] = d.isref[n] ? 0.0 : clampv(d.th[n], -kTwoPi, kTwoPi);
  }
  if (n < d.L) {
    d.wr[n] = s.own[n].x;
    d.wi[n] = s.own[n].y;
  }
}

template <typename P>
static cudaError_t lf_alloc(Ctx& c, P** p, size_t n) {
  return ctx_alloc(c, (void**)p, sizeof(P) * (n > 0 ? n : 1));
}

acopf_status project_linear(Ctx& c, double rho, double eps, int max_iter, int check, int* iters, double* rs) {
  Dev& d = c.d;
  LfState s;
  std::vector<void*> mem;
  cudaError_t e = cudaSuccess;
#define LA(ptr, n) if (e == cudaSuccess) { e = lf_alloc(c, &(ptr), (n)); if (e == cudaSuccess) mem.push_back((void*)(ptr)); }
  LA(s.X, 2 * (size_t)d.L); LA(s.Z, 2 * (size_t)d.L); LA(s.LAM, 2 * (size_t)d.L);
  LA(s.XG, d.G); LA(s.ZG, d.G); LA(s.LG, d.G); LA(s.own, d.L); LA(s.WB, d.B);
  LA(s.x0, 2 * (size_t)d.G + d.B + 2 * (size_t)d.L); LA(s.res, 2 * (size_t)d.K);
#undef LA
  auto release = [&]() {
    for (void* p : mem) ctx_free(c, p);
  };
  if (e != cudaSuccess) {
    release();
    c.last_error = std::string("acopf_project_linear: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ACOPF_ENOMEM : ACOPF_ECUDA;
  }
  const long m = d.G + d.L > d.B ? d.G + d.L : d.B;
  k_lf_init<<<nblk(m, 256), 256, 0, c.stream>>>(d, s);
  std::vector<double> h(2 * (size_t)d.K, 0.0);
  int it = 0;
  bool done = false;
  while (it < max_iter && !done) {
    const int n = max_iter - it < check ? max_iter - it : check;
    for (int k = 0; k < n; ++k) {
      cudaMemsetAsync(s.res, 0, sizeof(unsigned long long) * 2 * d.K, c.stream);
      k_lf_components<<<nblk(d.G + d.L, 128), 128, 0, c.stream>>>(d, s, rho);
      k_lf_buses<<<nblk(d.B, 128), 128, 0, c.stream>>>(d, s, rho);
      c.launches += 2;
    }
    it += n;
    e = cudaMemcpyAsync(h.data(), s.res, sizeof(double) * 2 * d.K, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) break;
    done = true;
    for (int k = 0; k < 2 * d.K; ++k) done = done && h[k] <= eps;
  }
  if (e == cudaSuccess) {
    k_lf_finish<<<nblk(m, 256), 256, 0, c.stream>>>(d, s);
    c.launches++;
    e = cudaStreamSynchronize(c.stream);
  }
  release();
  if (e != cudaSuccess) {
    c.last_error = std::string("acopf_project_linear: ") + cudaGetErrorString(e);
    return ACOPF_ECUDA;
  }
  if (iters) *iters = it;
  if (rs) {
    double r = 0.0, sv = 0.0;
    for (int k = 0; k < d.K; ++k) {
      r = fmax(r, h[k]);
      sv = fmax(sv, h[d.K + k]);
    }
    rs[0] = r;
    rs[1] = sv;
  }
  return ACOPF_OK;
}

}  // namespace acopf
