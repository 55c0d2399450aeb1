// Host build of the line subproblem's numerical helpers, for the CPU tests:
// the FP64 reciprocal square root by one third-order step from a given
// estimate, the integer FP64 <-> FP32 conversions, and the exact FP64 line solve by a predicted active set against
// the dual active-set method.  Plain C entry points for ctypes.
#define ACOPF_HD
#include <math.h>
#include <algorithm>
using std::fmax;
#include "../../paper_2310_13143_gb300/csrc/line_qp.cuh"
using namespace acopf;

extern "C" double host_rsqrt_newton(double a, double y0) { return rsqrt_newton(a, y0); }

// the integer FP64 <-> FP32 conversions, elementwise
extern "C" void host_f32_trunc(int n, const double* x, float* out) {
  for (int i = 0; i < n; ++i) out[i] = f32_trunc(x[i]);
}
extern "C" void host_f64_widen(int n, const float* x, double* out) {
  for (int i = 0; i < n; ++i) out[i] = f64_widen(x[i]);
}

// in: q10 c4 lo4 hi4 R8 rb2 on2 alo ahi ang x4 (41 values per problem)
static LineQP<double> make(const double* in) {
  LineQP<double> P;
  for (int k = 0; k < 10; ++k) P.q[k] = in[k];
  for (int i = 0; i < 4; ++i) { P.c[i] = in[10 + i]; P.lo[i] = in[14 + i]; P.hi[i] = in[18 + i]; }
  for (int e = 0; e < 2; ++e) {
    for (int i = 0; i < 4; ++i) P.R[e][i] = in[22 + 4 * e + i];
    P.rb[e] = in[30 + e];
    P.on[e] = in[32 + e] > 0;
  }
  P.alo = in[34]; P.ahi = in[35]; P.ang = in[36] > 0;
  return P;
}

// per problem: the predicted solve's flag, x and u, and the dual method's status, x and u
extern "C" void host_line_solves(int n, const double* in, int* ok, double* xp, double* up, int* st, double* xe,
                                 double* ue) {
  for (int b = 0; b < n; ++b) {
    const double* r = in + 41 * b;
    LineQP<double> P = make(r);
    double x[4] = {r[37], r[38], r[39], r[40]}, u[4] = {0, 0, 0, 0};
    ok[b] = line_solve_predicted(P, x, u) ? 1 : 0;
    for (int i = 0; i < 4; ++i) { xp[4 * b + i] = x[i]; up[4 * b + i] = u[i]; }
    double x2[4], u2[4];
    st[b] = line_solve_exact(P, x2, u2);
    for (int i = 0; i < 4; ++i) { xe[4 * b + i] = x2[i]; ue[4 * b + i] = u2[i]; }
  }
}
