// The per-branch line subproblem of eq. line_kernel as a 4-variable QP,
// solved by the augmented Lagrangian method with a projected Newton inner
// solver (Sec. IV-B).  Host and device code: the sweep kernel calls it per
// branch, and the same code compiles on the host for unit checks.
#pragma once

#include <math.h>

#ifndef ACOPF_HD
#define ACOPF_HD __host__ __device__
#endif

namespace acopf {

template <typename T>
struct Tol;
template <>
struct Tol<double> {
  static constexpr double newton = 1e-13;
  static constexpr double alm = 1e-11;
};
template <>
struct Tol<float> {
  static constexpr float newton = 2e-6f;
  static constexpr float alm = 2e-6f;
};

// ---------------------------------------------------- small dense helpers
template <typename T>
ACOPF_HD inline void symv4(const T q[10], const T x[4], T y[4]) {
  y[0] = q[0] * x[0] + q[1] * x[1] + q[2] * x[2] + q[3] * x[3];
  y[1] = q[1] * x[0] + q[4] * x[1] + q[5] * x[2] + q[6] * x[3];
  y[2] = q[2] * x[0] + q[5] * x[1] + q[7] * x[2] + q[8] * x[3];
  y[3] = q[3] * x[0] + q[6] * x[1] + q[8] * x[2] + q[9] * x[3];
}

template <typename T>
ACOPF_HD inline T clampv(T v, T lo, T hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Quotient and reciprocal square root of the line and bus updates.  FP64
// keeps the correctly rounded operations; the FP32 kernel takes the
// special-function unit's approximations (__fdividef, rsqrtf: within a few
// ulp), which shorten the dependent chain of each branch's solve.  The FP32
// box QP refines its final solve with a residual in twice the precision, and
// the ADMM tolerances of the FP32 path lie far above these errors.
ACOPF_HD inline double div_w(double a, double b) { return a / b; }
ACOPF_HD inline float div_w(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
ACOPF_HD inline double rsqrt_w(double a) { return 1.0 / sqrt(a); }
ACOPF_HD inline float rsqrt_w(float a) {
#ifdef __CUDA_ARCH__
  return rsqrtf(a);
#else
  return 1.0f / sqrtf(a);
#endif
}

// ----------------------------------------------------------- line update
// min 1/2 x'Qx + c'x  s.t. lo <= x <= hi,  R_r x <= rb_r for the two
// normalised line-limit rows that are on, and  alo <= x1 - x3 <= ahi  (the
// angle-difference rows, when ang is set).
//
// Augmented Lagrangian (Powell-Hestenes-Rockafellar, penalty beta) on the four
// rows.  Each subproblem  min_{lo<=x<=hi} 1/2 x'Qx + c'x + sum_r psi_r(x),
// psi_r = (max(0, u_r + beta h_r)^2 - u_r^2) / (2 beta), is piecewise
// quadratic; it is solved by a semismooth Newton loop that fixes the pieces
// at the current point and solves the resulting box-constrained QP exactly by
// a primal active-set method (the bounds play the role of TRON's projected
// search; with four variables the active-set method terminates in a few
// factorisations).
template <typename T>
struct LineQP {
  T q[10], c[4], lo[4], hi[4];
  T R[2][4], rb[2];
  T alo, ahi;
  bool on[2], ang;
};

// packed index of (i, j)
ACOPF_HD inline int pk(int i, int j) {
  const int t[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
  return t[i][j];
}

template <typename T>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double v = 2.2204460492503131e-16;
};
template <>
struct Eps<float> {
  static constexpr float v = 1.1920928955078125e-07f;
};

// Solve A p = r, A = h restricted to the free variables (free bit i set) with
// unit rows and columns for the fixed ones, by Cholesky.  False on breakdown.
template <typename T>
ACOPF_HD inline bool chol4_masked(const T h[10], unsigned fr, const T r[4], T p[4]) {
  const bool f0 = fr & 1u, f1 = (fr >> 1) & 1u, f2 = (fr >> 2) & 1u, f3 = (fr >> 3) & 1u;
  T a00 = f0 ? h[0] : T(1), a11 = f1 ? h[4] : T(1), a22 = f2 ? h[7] : T(1), a33 = f3 ? h[9] : T(1);
  T a01 = f0 && f1 ? h[1] : T(0), a02 = f0 && f2 ? h[2] : T(0), a03 = f0 && f3 ? h[3] : T(0);
  T a12 = f1 && f2 ? h[5] : T(0), a13 = f1 && f3 ? h[6] : T(0), a23 = f2 && f3 ? h[8] : T(0);
  if (!(a00 > T(0))) return false;
  T i00 = rsqrt_w(a00);
  T l10 = a01 * i00, l20 = a02 * i00, l30 = a03 * i00;
  T d1 = a11 - l10 * l10;
  if (!(d1 > T(0))) return false;
  T i11 = rsqrt_w(d1);
  T l21 = (a12 - l20 * l10) * i11, l31 = (a13 - l30 * l10) * i11;
  T d2 = a22 - l20 * l20 - l21 * l21;
  if (!(d2 > T(0))) return false;
  T i22 = rsqrt_w(d2);
  T l32 = (a23 - l30 * l20 - l31 * l21) * i22;
  T d3 = a33 - l30 * l30 - l31 * l31 - l32 * l32;
  if (!(d3 > T(0))) return false;
  T i33 = rsqrt_w(d3);
  T y0 = r[0] * i00;
  T y1 = (r[1] - l10 * y0) * i11;
  T y2 = (r[2] - l20 * y0 - l21 * y1) * i22;
  T y3 = (r[3] - l30 * y0 - l31 * y1 - l32 * y2) * i33;
  p[3] = y3 * i33;
  p[2] = (y2 - l32 * p[3]) * i22;
  p[1] = (y1 - l21 * p[2] - l31 * p[3]) * i11;
  p[0] = (y0 - l10 * p[1] - l20 * p[2] - l30 * p[3]) * i00;
  return true;
}

// r - sum_j a_j x_j in twice the working precision (Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005: Dot2 with
// TwoProduct by fused multiply-add and Knuth's TwoSum), rounded once.
template <typename T>
ACOPF_HD inline T resid_dot2(T r, const T a[4], const T x[4]) {
  T s = r, e = T(0);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    T pr = -a[j] * x[j];
    T pe = fma(-a[j], x[j], -pr);  // -a x = pr + pe exactly
    T t = s + pr;
    T z = t - s;
    T se = (s - (t - z)) + (pr - z);  // s + pr = t + se exactly
    s = t;
    e += se + pe;
  }
  return s + e;
}

// Box-constrained strictly convex QP  min 1/2 x'Hx + b'x,  lo <= x <= hi,
// by the primal active-set method from the feasible start x.  Bit i of fx:
// variable i held at a bound (at lo when bit i of hiside is clear).  Returns
// the number of factorisations used.
template <typename T>
ACOPF_HD inline int box_qp(const T h[10], const T b[4], const T lo[4], const T hi[4], T x[4], int maxit) {
  unsigned fx = 0, hs = 0, perm = 0;
  T scale = T(0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (!(lo[i] < hi[i])) { x[i] = lo[i]; fx |= 1u << i; perm |= 1u << i; }
    else if (x[i] <= lo[i]) { x[i] = lo[i]; fx |= 1u << i; }
    else if (x[i] >= hi[i]) { x[i] = hi[i]; fx |= 1u << i; hs |= 1u << i; }
    scale = fmax(scale, fabs(b[i]));
  }
  T hmax = T(0);
#pragma unroll
  for (int k = 0; k < 10; ++k) hmax = fmax(hmax, fabs(h[k]));
  int it = 0;
  for (; it < maxit; ++it) {
    // minimiser over the free variables with the others held at their bounds
    const unsigned fr = ~fx & 15u;
    T rhs[4], y[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T s = -b[i];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((fx >> j) & 1u) s -= h[pk(i, j)] * x[j];
      rhs[i] = ((fx >> i) & 1u) ? T(0) : s;
    }
    if (!chol4_masked(h, fr, rhs, y)) break;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if ((fx >> i) & 1u) y[i] = x[i];
    // longest feasible step towards y
    T alpha = T(1);
    int blk = -1, side = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if ((fx >> i) & 1u) continue;
      T dx = y[i] - x[i];
      if (y[i] < lo[i] && dx < T(0)) {
        T a = div_w(lo[i] - x[i], dx);
        if (a < alpha) { alpha = a; blk = i; side = -1; }
      } else if (y[i] > hi[i] && dx > T(0)) {
        T a = div_w(hi[i] - x[i], dx);
        if (a < alpha) { alpha = a; blk = i; side = 1; }
      }
    }
    if (blk >= 0) {
      alpha = alpha < T(0) ? T(0) : alpha;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (!((fx >> i) & 1u)) x[i] = clampv(x[i] + alpha * (y[i] - x[i]), lo[i], hi[i]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i == blk) {
          x[i] = side < 0 ? lo[i] : hi[i];
          fx |= 1u << i;
          if (side > 0) hs |= 1u << i; else hs &= ~(1u << i);
        }
      continue;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = y[i];
    // multipliers of the bounds held: release the one of wrong sign that is largest
    T g[4];
    symv4(h, x, g);
    T xs = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      g[i] += b[i];
      xs = fmax(xs, fabs(x[i]));
    }
    T tol = T(64) * Eps<T>::v * (scale + hmax * xs);
    int worst = -1;
    T wv = tol;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (!((fx >> i) & 1u) || ((perm >> i) & 1u)) continue;
      T v = ((hs >> i) & 1u) ? g[i] : -g[i];
      if (v > wv) { wv = v; worst = i; }
    }
    if (worst < 0) {
      if (sizeof(T) < sizeof(double)) {
        // final active set: one step of iterative refinement, the residual of
        // the reduced system taken in twice the working precision (the
        // condition number, rho I against rho F'F, reaches 1e4)
        T rr[4], dy[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          T a[4], xf[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            a[j] = h[pk(i, j)];
            xf[j] = ((fx >> j) & 1u) ? T(0) : x[j];
          }
          T ri = resid_dot2(rhs[i], a, xf);
          rr[i] = ((fx >> i) & 1u) ? T(0) : ri;
        }
        if (chol4_masked(h, fr, rr, dy))
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (!((fx >> i) & 1u)) x[i] = clampv(x[i] + dy[i], lo[i], hi[i]);
      }
      return it + 1;
    }
    fx &= ~(1u << worst);
    hs &= ~(1u << worst);
  }
  return it;
}

// row r of the ALM: h_r(x) (<= 0 when satisfied); rows 2, 3 are the angle rows
template <typename T>
ACOPF_HD inline T row_h(const LineQP<T>& P, int r, const T x[4]) {
  if (r < 2) return P.R[r][0] * x[0] + P.R[r][1] * x[1] + P.R[r][2] * x[2] + P.R[r][3] * x[3] - P.rb[r];
  T dth = x[1] - x[3];
  return r == 2 ? dth - P.ahi : P.alo - dth;
}

template <typename T>
ACOPF_HD inline bool row_on(const LineQP<T>& P, int r) {
  return r < 2 ? P.on[r] : P.ang;
}

template <typename T>
ACOPF_HD inline void line_solve(const LineQP<T>& P, T x[4], T u[4], T beta, T alm_tol, int alm_outer, int newton_max,
                                int* work = nullptr) {
  for (int outer = 0; outer < alm_outer; ++outer) {
    if (work) work[1]++;
    unsigned pat = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (row_on(P, r) && u[r] + beta * row_h(P, r, x) > T(0)) pat |= 1u << r;
    for (int it = 0; it < newton_max; ++it) {
      // pieces fixed: quadratic beta R R' and linear (u - beta rb) R on the rows in pat
      T h[10], b[4];
#pragma unroll
      for (int k = 0; k < 10; ++k) h[k] = P.q[k];
#pragma unroll
      for (int i = 0; i < 4; ++i) b[i] = P.c[i];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!((pat >> r) & 1u)) continue;
        const T* Rr = P.R[r];
        T lin = u[r] - beta * P.rb[r];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          b[i] += lin * Rr[i];
#pragma unroll
          for (int j = i; j < 4; ++j) h[pk(i, j)] += beta * Rr[i] * Rr[j];
        }
      }
      // angle rows: R = +-(e1 - e3), right-hand sides ahi and -alo
      if (pat & 12u) {
        T lin = (pat & 4u) ? u[2] - beta * P.ahi : -(u[3] + beta * P.alo);
        T qq = (pat & 4u ? beta : T(0)) + (pat & 8u ? beta : T(0));
        if ((pat & 12u) == 12u) lin = u[2] - beta * P.ahi - (u[3] + beta * P.alo);
        b[1] += lin;
        b[3] -= lin;
        h[4] += qq;
        h[9] += qq;
        h[6] -= qq;
      }
      int nf = box_qp(h, b, P.lo, P.hi, x, 12);
      if (work) work[0] += nf;
      unsigned np = 0;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (row_on(P, r) && u[r] + beta * row_h(P, r, x) > T(0)) np |= 1u << r;
      if (np == pat) break;
      pat = np;
    }
    // multiplier update and feasibility/complementarity test
    T viol = T(0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (!row_on(P, r)) {
        u[r] = T(0);
        continue;
      }
      T hr = row_h(P, r, x);
      T un = u[r] + beta * hr;
      un = un > T(0) ? un : T(0);
      const T mb = div_w(-un, beta);
      T m = hr > mb ? hr : mb;
      viol = fmax(viol, fabs(m));
      u[r] = un;
    }
    if (viol <= alm_tol) break;
  }
}

}  // namespace acopf
