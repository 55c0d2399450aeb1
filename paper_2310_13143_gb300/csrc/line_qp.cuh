// The per-branch line subproblem of eq. line_kernel as a 4-variable QP,
// solved by the augmented Lagrangian method with a projected Newton inner
// solver (Sec. IV-B).  Host and device code: the sweep kernel calls it per
// branch, and the same code compiles on the host for unit checks.
#pragma once

#include <math.h>
#include <string.h>

#ifndef ACOPF_HD
#define ACOPF_HD __host__ __device__
#endif

namespace acopf {

template <typename T>
struct Tol;
template <>
struct Tol<double> {
  static constexpr double newton = 1e-13;
  static constexpr double alm = 1e-14;
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

// FP64 <-> FP32 conversions in integer operations, from the IEEE 754
// binary64 and binary32 formats.  On GB300 a conversion instruction with an
// FP64 operand issues at the FP64 rate, a small fraction of the FP32 and
// integer rates, and the FP64 line solve converts some fifty values per
// branch for its FP32 predictor.
ACOPF_HD inline unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, 8);
  return b;
#endif
}
ACOPF_HD inline double double_of(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}
ACOPF_HD inline float float_of(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
ACOPF_HD inline unsigned bits_of(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
// x rounded toward zero to FP32 (the 52-bit fraction cut to 23 bits);
// magnitudes below the FP32 normal range give a signed zero, above it an
// infinity; a NaN stays a NaN.  For values that seed or predict, where the
// rounding does not matter.
ACOPF_HD inline float f32_trunc(double x) {
  const unsigned long long b = bits_of(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  unsigned out;
  if (e <= 0) out = sign;
  else if (e >= 255) out = sign | 0x7f800000u | (e == 2047 - 1023 + 127 && ((hi & 0xfffffu) | lo) ? 0x400000u : 0u);
  else out = sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return float_of(out);
}
// f as FP64, exactly; an FP32 subnormal gives a signed zero
ACOPF_HD inline double f64_widen(float f) {
  const unsigned u = bits_of(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, frac = u & 0x7fffffu;
  unsigned hi;
  if (e == 0) hi = sign;
  else if (e == 255) hi = sign | 0x7ff00000u | (frac >> 3);
  else hi = sign | ((e - 127u + 1023u) << 20) | (frac >> 3);
  const unsigned lo = e == 0 ? 0u : frac << 29;
  return double_of(((unsigned long long)hi << 32) | lo);
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
// 1/sqrt(a) in FP64 from an estimate y0 by one third-order step: with
// e = 1 - a y0^2 the exact value is y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8
// + 5e^3/16 + ...), and the step keeps the series to e^2.  A relative error d
// of y0 leaves about 5/2 d^3, so an FP32 estimate (|d| <= 2^-21) ends below
// FP64 rounding: five FP64 instructions, against eight for two Newton-Raphson
// steps.  On the device the estimate is the FP32 special-function unit's
// rsqrtf; a correctly rounded square root and division cost many FP64
// instructions on GB300, whose FP64 rate is a small fraction of FP32.
ACOPF_HD inline double rsqrt_newton(double a, double y0) {
  const double t = a * y0;
  const double e = fma(-t, y0, 1.0);
  const double q = e * fma(0.375, e, 0.5);
  return fma(y0, q, y0);
}
ACOPF_HD inline double rsqrt_w(double a) {
#ifdef __CUDA_ARCH__
  // a in [2^-99, 2^101): the FP32 estimate is in range (exponent test in
  // integers, the conversions too; see f32_trunc)
  if ((unsigned)(bits_of(a) >> 52) - (1023u - 99u) < 200u) return rsqrt_newton(a, f64_widen(rsqrtf(f32_trunc(a))));
#endif
  return 1.0 / sqrt(a);
}
// a > 0, false for a NaN; in FP64 on the bit pattern (no FP64 comparison)
ACOPF_HD inline bool pos_w(double a) {
  const long long b = (long long)bits_of(a);
  return b > 0 && b <= 0x7ff0000000000000LL;
}
ACOPF_HD inline bool pos_w(float a) { return a > 0.f; }
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

// Cholesky factor of A = h restricted to the free variables (free bit i set),
// with unit rows and columns for the fixed ones: the strict lower part l and
// the reciprocals of the diagonal i.  False on breakdown.
template <typename T>
struct Chol4 {
  T l10, l20, l30, l21, l31, l32, i00, i11, i22, i33;
};
template <typename T>
ACOPF_HD inline bool chol4_factor(const T h[10], unsigned fr, Chol4<T>& f) {
  const bool f0 = fr & 1u, f1 = (fr >> 1) & 1u, f2 = (fr >> 2) & 1u, f3 = (fr >> 3) & 1u;
  T a00 = f0 ? h[0] : T(1), a11 = f1 ? h[4] : T(1), a22 = f2 ? h[7] : T(1), a33 = f3 ? h[9] : T(1);
  T a01 = f0 && f1 ? h[1] : T(0), a02 = f0 && f2 ? h[2] : T(0), a03 = f0 && f3 ? h[3] : T(0);
  T a12 = f1 && f2 ? h[5] : T(0), a13 = f1 && f3 ? h[6] : T(0), a23 = f2 && f3 ? h[8] : T(0);
  if (!pos_w(a00)) return false;
  f.i00 = rsqrt_w(a00);
  f.l10 = a01 * f.i00; f.l20 = a02 * f.i00; f.l30 = a03 * f.i00;
  T d1 = a11 - f.l10 * f.l10;
  if (!pos_w(d1)) return false;
  f.i11 = rsqrt_w(d1);
  f.l21 = (a12 - f.l20 * f.l10) * f.i11; f.l31 = (a13 - f.l30 * f.l10) * f.i11;
  T d2 = a22 - f.l20 * f.l20 - f.l21 * f.l21;
  if (!pos_w(d2)) return false;
  f.i22 = rsqrt_w(d2);
  f.l32 = (a23 - f.l30 * f.l20 - f.l31 * f.l21) * f.i22;
  T d3 = a33 - f.l30 * f.l30 - f.l31 * f.l31 - f.l32 * f.l32;
  if (!pos_w(d3)) return false;
  f.i33 = rsqrt_w(d3);
  return true;
}
// p = A^-1 r with the factor of chol4_factor
template <typename T>
ACOPF_HD inline void chol4_solve(const Chol4<T>& f, const T r[4], T p[4]) {
  T y0 = r[0] * f.i00;
  T y1 = (r[1] - f.l10 * y0) * f.i11;
  T y2 = (r[2] - f.l20 * y0 - f.l21 * y1) * f.i22;
  T y3 = (r[3] - f.l30 * y0 - f.l31 * y1 - f.l32 * y2) * f.i33;
  p[3] = y3 * f.i33;
  p[2] = (y2 - f.l32 * p[3]) * f.i22;
  p[1] = (y1 - f.l21 * p[2] - f.l31 * p[3]) * f.i11;
  p[0] = (y0 - f.l10 * p[1] - f.l20 * p[2] - f.l30 * p[3]) * f.i00;
}
// Solve A p = r (A as for chol4_factor).  False on breakdown.
template <typename T>
ACOPF_HD inline bool chol4_masked(const T h[10], unsigned fr, const T r[4], T p[4]) {
  Chol4<T> f;
  if (!chol4_factor(h, fr, f)) return false;
  chol4_solve(f, r, p);
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

// A sum of products accumulated in twice the working precision (the same
// Dot2 scheme), rounded once by value().
template <typename T>
struct Dot2Acc {
  T s, e;
  ACOPF_HD inline explicit Dot2Acc(T r) : s(r), e(T(0)) {}
  ACOPF_HD inline void add(T a, T b) {  // s + e += a b
    T pr = a * b;
    T pe = fma(a, b, -pr);
    T t = s + pr;
    T z = t - s;
    T se = (s - (t - z)) + (pr - z);
    s = t;
    e += se + pe;
  }
  ACOPF_HD inline T value() const { return s + e; }
};

// Box-constrained strictly convex QP  min 1/2 x'Hx + b'x,  lo <= x <= hi,
// by the primal active-set method from the feasible start x.  Bit i of fx:
// variable i held at a bound (at lo when bit i of hiside is clear).  Returns
// the number of factorisations used.
template <typename T>
ACOPF_HD inline int box_qp(const T h[10], const T b[4], const T lo[4], const T hi[4], T x[4], int maxit,
                           unsigned* wset = nullptr) {
  unsigned fx = 0, hs = 0, perm = 0;
  T scale = T(0);
  // a warm start: the bounds held at the end of a previous solve (bit 8 set
  // when *wset holds a set: bits 0-3 held, bits 4-7 at the upper bound)
  const unsigned ws = wset ? *wset : 0u;
  const bool warm = (ws >> 8) & 1u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (!(lo[i] < hi[i])) { x[i] = lo[i]; fx |= 1u << i; perm |= 1u << i; }
    else if (warm) {
      if ((ws >> i) & 1u) {
        fx |= 1u << i;
        if ((ws >> (4 + i)) & 1u) { x[i] = hi[i]; hs |= 1u << i; } else { x[i] = lo[i]; }
      } else {
        x[i] = clampv(x[i], lo[i], hi[i]);
      }
    }
    else if (x[i] <= lo[i]) { x[i] = lo[i]; fx |= 1u << i; }
    else if (x[i] >= hi[i]) { x[i] = hi[i]; fx |= 1u << i; hs |= 1u << i; }
    scale = fmax(scale, fabs(b[i]));
  }
  // max |h_k| as a tree (a shorter chain than a running max)
  const T m01 = fmax(fabs(h[0]), fabs(h[1])), m23 = fmax(fabs(h[2]), fabs(h[3])), m45 = fmax(fabs(h[4]), fabs(h[5]));
  const T m67 = fmax(fabs(h[6]), fabs(h[7])), m89 = fmax(fabs(h[8]), fabs(h[9]));
  const T hmax = fmax(fmax(fmax(m01, m23), fmax(m45, m67)), m89);
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
    Chol4<T> fac;
    if (!chol4_factor(h, fr, fac)) break;
    chol4_solve(fac, rhs, y);
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
        chol4_solve(fac, rr, dy);  // the same factor (the active set is unchanged)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (!((fx >> i) & 1u)) x[i] = clampv(x[i] + dy[i], lo[i], hi[i]);
      }
      if (wset) *wset = 0x100u | fx | (hs << 4);
      return it + 1;
    }
    fx &= ~(1u << worst);
    hs &= ~(1u << worst);
  }
  if (wset) *wset = 0x100u | fx | (hs << 4);
  return it;
}

// ------------------------------------------------ exact line QP (dual method)
// The same subproblem solved exactly by the dual active-set method of
// Goldfarb and Idnani ("A numerically stable dual method for solving strictly
// convex quadratic programs", Math. Programming 27, 1983): start from the
// unconstrained minimiser -Q^-1 c, repeatedly add the most violated
// constraint, taking full (primal) steps or partial (dual) steps that drop a
// constraint whose multiplier would turn negative, with Q^-1 and the active
// normals held as J = L^-T (rotated) and the triangular factor R, J'N = [R;0].
// Every step raises the dual objective, so it ends in a few steps at the
// unique KKT point; no feasible start is needed.  Constraint p in the form
// n_p'x >= b_p:
//   0..3  x_v >= lo_v          4..7  -x_v >= -hi_v
//   8, 9  -R_r x >= -rb_r      (line limits, when on)
//   10    -(x1 - x3) >= -ahi   11  x1 - x3 >= alo   (angle rows, when set)
template <typename T>
ACOPF_HD inline bool gi_row(const LineQP<T>& P, int p, T n[4], T& b) {
  bool on = true;
  b = T(0);
#pragma unroll
  for (int i = 0; i < 4; ++i) n[i] = T(0);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    if (p == v) { n[v] = T(1); b = P.lo[v]; }
    if (p == 4 + v) { n[v] = T(-1); b = -P.hi[v]; }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if (p == 8 + r) {
#pragma unroll
      for (int i = 0; i < 4; ++i) n[i] = -P.R[r][i];
      b = -P.rb[r];
      on = P.on[r];
    }
  if (p == 10) { n[1] = T(-1); n[3] = T(1); b = -P.ahi; on = P.ang; }
  if (p == 11) { n[1] = T(1); n[3] = T(-1); b = P.alo; on = P.ang; }
  return on;
}

// Givens rotation of columns a, b of J (applied as J <- J G')
template <typename T>
ACOPF_HD inline void gi_rot_cols(T J[4][4], int a, int b, T c, T s) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T ja = J[i][a], jb = J[i][b];
    J[i][a] = c * ja + s * jb;
    J[i][b] = -s * ja + c * jb;
  }
}

// Returns the number of steps, or -1 - steps when the subproblem has no
// feasible point (it then ends at the last point reached); u (4) receives the
// multipliers of rows lim0, lim1, ang_hi, ang_lo (layout of line_solve's u),
// x the solution.
template <typename T>
ACOPF_HD inline int line_solve_exact(const LineQP<T>& P, T x[4], T u[4], int maxit = 32) {
  // Q = L L' (Q is positive definite by construction of the record)
  const T* q = P.q;
  T l00 = sqrt(q[0]);
  T l10 = q[1] / l00, l20 = q[2] / l00, l30 = q[3] / l00;
  T l11 = sqrt(q[4] - l10 * l10);
  T l21 = (q[5] - l20 * l10) / l11, l31 = (q[6] - l30 * l10) / l11;
  T l22 = sqrt(q[7] - l20 * l20 - l21 * l21);
  T l32 = (q[8] - l30 * l20 - l31 * l21) / l22;
  T l33 = sqrt(q[9] - l30 * l30 - l31 * l31 - l32 * l32);
  // J = L^-T (upper triangular): M = L^-1 by forward substitution, J = M'
  T J[4][4];
  {
    T m00 = T(1) / l00, m11 = T(1) / l11, m22 = T(1) / l22, m33 = T(1) / l33;
    T m10 = -l10 * m00 * m11;
    T m21 = -l21 * m11 * m22;
    T m20 = -(l20 * m00 + l21 * m10) * m22;
    T m32 = -l32 * m22 * m33;
    T m31 = -(l31 * m11 + l32 * m21) * m33;
    T m30 = -(l30 * m00 + l31 * m10 + l32 * m20) * m33;
    J[0][0] = m00; J[0][1] = m10; J[0][2] = m20; J[0][3] = m30;
    J[1][0] = T(0); J[1][1] = m11; J[1][2] = m21; J[1][3] = m31;
    J[2][0] = T(0); J[2][1] = T(0); J[2][2] = m22; J[2][3] = m32;
    J[3][0] = T(0); J[3][1] = T(0); J[3][2] = T(0); J[3][3] = m33;
  }
  // unconstrained minimiser x = -J J' c
  {
    T t[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) t[j] = J[0][j] * P.c[0] + J[1][j] * P.c[1] + J[2][j] * P.c[2] + J[3][j] * P.c[3];
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = -(J[i][0] * t[0] + J[i][1] * t[1] + J[i][2] * t[2] + J[i][3] * t[3]);
  }
  T R[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) R[i][j] = T(0);
  T ua[5] = {T(0), T(0), T(0), T(0), T(0)};  // multipliers of the active constraints (+ the one being added)
  int act[4] = {-1, -1, -1, -1};
  int nq = 0;
  T cs = T(0);
#pragma unroll
  for (int i = 0; i < 4; ++i) cs = fmax(cs, fabs(P.c[i]));
  const T eps = Eps<T>::v;
  int steps = 0;
  bool done = false, infeasible = false;
  while (!done && steps < maxit) {
    // most violated constraint, by its violation relative to its scale
    T xs = fmax(fmax(fabs(x[0]), fabs(x[1])), fmax(fabs(x[2]), fabs(x[3])));
    int p = -1;
    T worst = T(0), sp = T(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      bool in = false;
#pragma unroll
      for (int a = 0; a < 4; ++a) in = in || (a < nq && act[a] == k);
      T n[4], b;
      if (!gi_row(P, k, n, b) || in) continue;
      T sk = n[0] * x[0] + n[1] * x[1] + n[2] * x[2] + n[3] * x[3] - b;
      T nn = fabs(n[0]) + fabs(n[1]) + fabs(n[2]) + fabs(n[3]);
      T v = -sk / (T(1) + fabs(b) + nn * xs);
      if (v > worst) { worst = v; p = k; sp = sk; }
    }
    if (p < 0 || worst <= T(64) * eps) break;
    T np[4], bp;
    gi_row(P, p, np, bp);
#pragma unroll
    for (int a = 0; a < 5; ++a)
      if (a == nq) ua[a] = T(0);
    // add p, with partial steps that drop constraints, until it is active
    for (int inner = 0; inner < 8 && steps < maxit; ++inner) {
      ++steps;
      T d[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) d[j] = J[0][j] * np[0] + J[1][j] * np[1] + J[2][j] * np[2] + J[3][j] * np[3];
      // primal direction z = J2 d2, dual direction r = R^-1 d1
      T z[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j >= nq)
#pragma unroll
          for (int i = 0; i < 4; ++i) z[i] += J[i][j] * d[j];
      T r[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int i = 3; i >= 0; --i) {
        if (i >= nq) continue;
        T sacc = d[i];
#pragma unroll
        for (int j = i + 1; j < 4; ++j)
          if (j < nq) sacc -= R[i][j] * r[j];
        r[i] = sacc / R[i][i];
      }
      // partial step: the active multiplier that reaches zero first
      T t1 = T(0);
      int kd = -1;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j >= nq || !(r[j] > T(0))) continue;
        T tj = ua[j] / r[j];
        if (kd < 0 || tj < t1) { t1 = tj; kd = j; }
      }
      // full step: p becomes active
      T zn = z[0] * np[0] + z[1] * np[1] + z[2] * np[2] + z[3] * np[3];
      T dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3];
      const bool full_ok = zn > T(64) * eps * dd;
      T t2 = full_ok ? -sp / zn : T(0);
      if (!full_ok && kd < 0) { done = infeasible = true; break; }  // no feasible point
      const bool partial = kd >= 0 && (!full_ok || t1 < t2);
      const T t = partial ? t1 : t2;
      if (full_ok) {
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] += t * z[i];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < nq) ua[j] -= t * r[j];
#pragma unroll
      for (int a = 0; a < 5; ++a)
        if (a == nq) ua[a] += t;
      if (!partial) {
        // add p: rotate d[j] (j > nq) into d[nq]; R's new column is d[0..nq]
#pragma unroll
        for (int j = 3; j >= 1; --j) {
          if (j <= nq || d[j] == T(0)) continue;
          T h = sqrt(d[j - 1] * d[j - 1] + d[j] * d[j]);
          T c = d[j - 1] / h, s = d[j] / h;
          d[j - 1] = h;
          d[j] = T(0);
          gi_rot_cols(J, j - 1, j, c, s);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j == nq && i <= nq) R[i][j] = d[i];
#pragma unroll
        for (int a = 0; a < 4; ++a)
          if (a == nq) act[a] = p;
        ++nq;
        break;
      }
      // drop the constraint at position kd: remove its column of R and its
      // multiplier (the entering one moves down with the others), then
      // restore R's triangular form by rotations
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (j >= kd && j < nq - 1) {
#pragma unroll
          for (int i = 0; i < 4; ++i) R[i][j] = R[i][j + 1];
          act[j] = act[j + 1];
        }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j >= kd && j < nq) ua[j] = ua[j + 1];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j == nq - 1) R[i][j] = T(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (j < kd || j >= nq - 1) continue;
        T a0 = R[j][j], b0 = R[j + 1][j];
        if (b0 == T(0)) continue;
        T h = sqrt(a0 * a0 + b0 * b0);
        T c = a0 / h, s = b0 / h;
#pragma unroll
        for (int col = 0; col < 4; ++col) {
          if (col < j || col >= nq - 1) continue;
          T ra = R[j][col], rb = R[j + 1][col];
          R[j][col] = c * ra + s * rb;
          R[j + 1][col] = -s * ra + c * rb;
        }
        gi_rot_cols(J, j, j + 1, c, s);
      }
      --nq;
      sp = np[0] * x[0] + np[1] * x[1] + np[2] * x[2] + np[3] * x[3] - bp;
    }
  }
  (void)cs;
  if (sizeof(T) < sizeof(double)) {
    // one step of iterative refinement on the final active set: residuals of
    // stationarity (Qx + c - N u = 0) and of the active rows (N'x = b) in
    // twice the working precision, the correction from the factors J and R
    // (with dx = J y: R' y1 = r_b, y2 = (J'r_x)_2, R du = y1 - (J'r_x)_1)
    T rx[4], rb[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      Dot2Acc<T> acc(-P.c[i]);
#pragma unroll
      for (int j = 0; j < 4; ++j) acc.add(-q[pk(i, j)], x[j]);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (a >= nq) continue;
        T n[4], b;
        gi_row(P, act[a], n, b);
        acc.add(n[i], ua[a]);
      }
      rx[i] = acc.value();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (a >= nq) continue;
      T n[4], b;
      gi_row(P, act[a], n, b);
      Dot2Acc<T> acc(b);
#pragma unroll
      for (int j = 0; j < 4; ++j) acc.add(-n[j], x[j]);
      rb[a] = acc.value();
    }
    T w[4], y[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = J[0][j] * rx[0] + J[1][j] * rx[1] + J[2][j] * rx[2] + J[3][j] * rx[3];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i >= nq) {
        y[i] = w[i];
        continue;
      }
      T sacc = rb[i];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < i) sacc -= R[k][i] * y[k];
      y[i] = sacc / R[i][i];
    }
    T du[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int i = 3; i >= 0; --i) {
      if (i >= nq) continue;
      T sacc = y[i] - w[i];
#pragma unroll
      for (int k = i + 1; k < 4; ++k)
        if (k < nq) sacc -= R[i][k] * du[k];
      du[i] = sacc / R[i][i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] += J[i][0] * y[0] + J[i][1] * y[1] + J[i][2] * y[2] + J[i][3] * y[3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (a < nq) ua[a] += du[a];
  }
  // bounds hold to rounding; keep x inside the box exactly
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = clampv(x[i], P.lo[i], P.hi[i]);
#pragma unroll
  for (int r = 0; r < 4; ++r) u[r] = T(0);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (a >= nq) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (act[a] == 8 + r) u[r] = ua[a];
  }
  return infeasible ? -1 - steps : steps;
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
                                int* work = nullptr, unsigned* wset = nullptr) {
  // the rows' values at the current x, evaluated once per point
  T hv[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) hv[r] = row_h(P, r, x);
  for (int outer = 0; outer < alm_outer; ++outer) {
    if (work) work[1]++;
    unsigned pat = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (row_on(P, r) && u[r] + beta * hv[r] > T(0)) pat |= 1u << r;
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
      int nf = box_qp(h, b, P.lo, P.hi, x, 12, wset);
      if (work) work[0] += nf;
#pragma unroll
      for (int r = 0; r < 4; ++r) hv[r] = row_h(P, r, x);
      unsigned np = 0;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (row_on(P, r) && u[r] + beta * hv[r] > T(0)) np |= 1u << r;
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
      const T hr = hv[r];
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


// ------------------------------------------ exact FP64 line QP by prediction
// The FP64 line subproblem solved exactly with most of the work in FP32: the
// augmented Lagrangian in FP32 (from the multipliers u and the point x given)
// predicts which bounds and rows are active;
// the equality-constrained QP on that set is solved in FP64 (Cholesky of Q on
// the free variables, then the rows' multipliers from the Schur complement
// S = N Q^-1 N', in closed form for up to two active rows); the KKT
// conditions are checked in FP64: the Lagrangian stationary in the free
// variables, every free variable within its bounds, every row satisfied,
// every multiplier of an active row or bound of the right sign, each up to a
// tolerance of 1e-11 of the problem's scale.  Both solutions are the unique
// KKT point, so they agree up to rounding.  Returns false when the prediction
// fails the check and two corrections of the set; the caller then runs the
// FP64 dual active-set method.  On entry x and u hold a starting point and
// multipliers.  FP64 instructions issue at a small fraction of the FP32 rate
// on GB300, so the FP64 part is written to be short.
ACOPF_HD inline bool line_solve_predicted(const LineQP<double>& P, double x[4], double u[4]) {
  // the FP32 copy for the predictor (truncated: the prediction is checked in FP64)
  LineQP<float> F;
#pragma unroll
  for (int k = 0; k < 10; ++k) F.q[k] = f32_trunc(P.q[k]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    F.c[i] = f32_trunc(P.c[i]);
    F.lo[i] = f32_trunc(P.lo[i]);
    F.hi[i] = f32_trunc(P.hi[i]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int i = 0; i < 4; ++i) F.R[r][i] = f32_trunc(P.R[r][i]);
    F.rb[r] = f32_trunc(P.rb[r]);
    F.on[r] = P.on[r];
  }
  F.alo = f32_trunc(P.alo);
  F.ahi = f32_trunc(P.ahi);
  F.ang = P.ang;
  // the FP32 augmented Lagrangian from the multipliers given and the
  // unconstrained start clamped into the box
  float xf[4], uf[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    xf[i] = clampv(f32_trunc(x[i]), F.lo[i], F.hi[i]);
    uf[i] = f32_trunc(u[i]);
  }
  {
    const float qd = fmax(fmax(F.q[0], F.q[4]), fmax(F.q[7], F.q[9]));
    line_solve(F, xf, uf, 10.0f * qd, Tol<float>::alm, 50, 20);
  }
  // predicted active set: bounds (at hi when the hs bit is set) and rows; a
  // bound counts as active when the FP32 point lies within 1e-6 of the box's
  // width from it (FP32 rounding can leave an active bound a hair inside)
  unsigned fx = 0, hs = 0, act = 0;
  double xb[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    xb[i] = 0.0;
    const float dlt = 1e-6f * (F.hi[i] - F.lo[i]);
    if (!(P.lo[i] < P.hi[i]) || xf[i] <= F.lo[i] + dlt) {
      fx |= 1u << i;
      xb[i] = P.lo[i];
    } else if (xf[i] >= F.hi[i] - dlt) {
      fx |= 1u << i;
      hs |= 1u << i;
      xb[i] = P.hi[i];
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (row_on(P, r) && uf[r] > 0.f) act |= 1u << r;
  // row r: n_r . x <= b_r
  double n[4][4], b[4];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int i = 0; i < 4; ++i) n[r][i] = P.R[r][i];
    b[r] = P.rb[r];
  }
  n[2][0] = 0.0; n[2][1] = 1.0; n[2][2] = 0.0; n[2][3] = -1.0; b[2] = P.ahi;
  n[3][0] = 0.0; n[3][1] = -1.0; n[3][2] = 0.0; n[3][3] = 1.0; b[3] = -P.alo;
  // the scales of the tolerances below, from the FP32 copy (a relative
  // error of 1e-7 in a tolerance does not matter; FP32 costs far less)
  float cmf = 0.f, qmf = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) cmf = fmax(cmf, fabs(F.c[i]));
#pragma unroll
  for (int k = 0; k < 10; ++k) qmf = fmax(qmf, fabs(F.q[k]));
  const double cm = f64_widen(cmf), qm = f64_widen(qmf);
  double xs[4], mu[4];
  bool ok = false;
  // the predicted set, then at most two corrections of it (bounds and rows
  // found violated are added, those with a multiplier of the wrong sign
  // dropped) before giving up
  for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
    // minimiser y over the free variables with the rows left out
    const unsigned fr = ~fx & 15u;
    Chol4<double> fac;
    if (!chol4_factor(P.q, fr, fac)) return false;
    double rhs[4], y[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      double sv = -P.c[i];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((fx >> j) & 1u) sv -= P.q[pk(i, j)] * xb[j];
      rhs[i] = ((fx >> i) & 1u) ? 0.0 : sv;
    }
    chol4_solve(fac, rhs, y);
    // the multipliers of the active rows from the Schur complement S = N W,
    // W = Q_FF^-1 N(F)', t = N y - (b - N xb) (N: the active rows, N(F) on
    // the free variables); then xs = y - W' mu and gm = N' mu
    double gm[4];
    const int na = (int)(act & 1u) + (int)((act >> 1) & 1u) + (int)((act >> 2) & 1u) + (int)((act >> 3) & 1u);
    if (na <= 2) {
      // at most two active rows (the common case): S is 1x1 or 2x2, solved
      // in closed form, and two row slots replace the four rows
      int r0 = -1, r1 = -1;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if ((act >> r) & 1u) {
          if (r0 < 0) r0 = r;
          else r1 = r;
        }
      double m0[4], m1[4], c0 = 0.0, c1 = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) m0[i] = m1[i] = 0.0;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (r == r0) m0[i] = n[r][i];
          if (r == r1) m1[i] = n[r][i];
        }
        if (r == r0) c0 = b[r];
        if (r == r1) c1 = b[r];
      }
      // on the free variables; the fixed ones go to the right-hand side
      // (xb is 0 on the free variables)
      double f0[4], f1[4], W0[4] = {0.0, 0.0, 0.0, 0.0}, W1[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool fixed = (fx >> i) & 1u;
        f0[i] = fixed ? 0.0 : m0[i];
        f1[i] = fixed ? 0.0 : m1[i];
        c0 -= m0[i] * xb[i];
        c1 -= m1[i] * xb[i];
      }
      double mu0 = 0.0, mu1 = 0.0;
      if (r0 >= 0) {
        chol4_solve(fac, f0, W0);
        double t0 = -c0, s00 = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          t0 += f0[i] * y[i];
          s00 += f0[i] * W0[i];
        }
        if (!(s00 > 0.0)) return false;
        if (r1 >= 0) {
          chol4_solve(fac, f1, W1);
          double t1 = -c1, s01 = 0.0, s11 = 0.0;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            t1 += f1[i] * y[i];
            s01 += f0[i] * W1[i];
            s11 += f1[i] * W1[i];
          }
          const double det = s00 * s11 - s01 * s01;
          if (!(det > 0.0)) return false;
          const double id = 1.0 / det;
          mu0 = (s11 * t0 - s01 * t1) * id;
          mu1 = (s00 * t1 - s01 * t0) * id;
        } else {
          mu0 = t0 / s00;
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xs[i] = ((fx >> i) & 1u) ? xb[i] : y[i] - mu0 * W0[i] - mu1 * W1[i];
        gm[i] = mu0 * m0[i] + mu1 * m1[i];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) mu[r] = r == r0 ? mu0 : (r == r1 ? mu1 : 0.0);
    } else {
      // three or four active rows: S by a masked 4x4 Cholesky
      double W[4][4], S[10], t[4];
#pragma unroll
      for (int k = 0; k < 10; ++k) S[k] = 0.0;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        t[r] = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) W[r][i] = 0.0;
        if (!((act >> r) & 1u)) continue;
        double nf[4], bf = b[r];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const bool fixed = (fx >> i) & 1u;
          nf[i] = fixed ? 0.0 : n[r][i];
          if (fixed) bf -= n[r][i] * xb[i];
        }
        chol4_solve(fac, nf, W[r]);
        double ny = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) ny += nf[i] * y[i];
        t[r] = ny - bf;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = r; q < 4; ++q) {
          if (!((act >> r) & 1u) || !((act >> q) & 1u)) continue;
          double v = 0.0;
#pragma unroll
          for (int i = 0; i < 4; ++i) v += ((fx >> i) & 1u) ? 0.0 : n[r][i] * W[q][i];
          S[pk(r, q)] = v;
        }
      Chol4<double> fs;
      if (!chol4_factor(S, act, fs)) return false;
      chol4_solve(fs, t, mu);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        double v = ((fx >> i) & 1u) ? xb[i] : y[i];
        gm[i] = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if ((act >> r) & 1u) {
            v -= mu[r] * W[r][i];
            gm[i] += mu[r] * n[r][i];
          }
        xs[i] = ((fx >> i) & 1u) ? xb[i] : v;
      }
    }
    // KKT check: gradient of the Lagrangian g = Q x + c + sum_r mu_r n_r
    double g[4];
    symv4(P.q, xs, g);
    unsigned long long xmb = 0ull;  // max |xs_i| on the bit patterns (a NaN the largest)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      g[i] += P.c[i] + gm[i];
      const unsigned long long b = bits_of(xs[i]) & 0x7fffffffffffffffull;
      xmb = b > xmb ? b : xmb;
    }
    const double xm = double_of(xmb);
    const double tol = 1e-11 * (cm + qm * xm + 1.0), tx = 1e-11 * (xm + 1.0);
    unsigned nfx = fx, nhs = hs, nact = act;
    ok = true;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (!row_on(P, r)) continue;
      double v = -b[r];
      if (r < 2) {
#pragma unroll
        for (int i = 0; i < 4; ++i) v += n[r][i] * xs[i];
      } else {  // the angle rows: +-(x1 - x3), the same sums without the zero terms
        v = r == 2 ? (v + xs[1]) - xs[3] : (v - xs[1]) + xs[3];
      }
      const bool feas = v <= tx * (1.0 + fabs(b[r]));  // every row, active or not (a singular S shows here)
      if ((act >> r) & 1u) {
        if (!(mu[r] >= -tol)) { ok = false; nact &= ~(1u << r); }
        if (!feas) ok = false;
      } else if (!feas) {
        ok = false;
        nact |= 1u << r;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (!((fx >> i) & 1u)) {
        if (!(fabs(g[i]) <= tol)) ok = false;  // stationary in the free variables
        if (!(xs[i] >= P.lo[i] - tx)) { ok = false; nfx |= 1u << i; nhs &= ~(1u << i); xb[i] = P.lo[i]; }
        else if (!(xs[i] <= P.hi[i] + tx)) { ok = false; nfx |= 1u << i; nhs |= 1u << i; xb[i] = P.hi[i]; }
      } else if (P.lo[i] < P.hi[i]) {
        if (!(((hs >> i) & 1u) ? g[i] <= tol : g[i] >= -tol)) { ok = false; nfx &= ~(1u << i); xb[i] = 0.0; }
      }
    }
    if (!ok && nfx == fx && nhs == hs && nact == act) return false;  // nothing to correct (non-finite values)
    fx = nfx;
    hs = nhs;
    act = nact;
  }
  if (!ok) return false;
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = clampv(xs[i], P.lo[i], P.hi[i]);
#pragma unroll
  for (int r = 0; r < 4; ++r) u[r] = ((act >> r) & 1u) && pos_w(mu[r]) ? mu[r] : 0.0;
  return true;
}

}  // namespace acopf
