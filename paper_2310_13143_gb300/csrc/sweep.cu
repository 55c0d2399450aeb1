// The ADMM sweep of Algorithm 2 fused into one persistent cooperative kernel.
//
// Iteration t:
//   phase A  one thread per generator (eq. gen_kernel, closed form) and per
//            branch (eq. line_kernel: 4-variable QP with box, line-limit and
//            angle rows, solved by an augmented Lagrangian whose subproblems
//            are solved by projected Newton -- Sec. IV-B);
//   barrier
//   phase B  one lane per generator or branch end, one warp per task of
//            consecutive buses (eq. bus_kernel, closed form from the 2x2
//            system of the power-balance rows, per-bus sums by a segmented
//            warp scan), fused with the multiplier update of every coupling
//            (eq. multiplier) and the primal/dual residuals r = x - z,
//            s = rho (z+ - z) (Sec. IV-B), reduced with warp shuffles and one
//            64-bit atomicMax per run of lanes of one instance;
//   barrier
//   every CTA reads the per-instance residual slots and decides, identically,
//   which instances have converged; finished instances are skipped.
//
// The device-wide barrier spins with a clock64 limit: a CTA that waits longer
// than the limit records an error and the kernel returns (no unbounded wait).
#include <cooperative_groups.h>
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "common.cuh"
#include "line_qp.cuh"

namespace acopf {

template <typename T>
struct SweepP {
  Dev d;
  int max_iter;
  int fixed;            // 1: run max_iter iterations, no residual test
  double eps, eps_dual;
  T beta_scale, alm_tol;
  int alm_outer, newton_max;
  long long spin_limit;
  int rb_period;
  double rb_mu, rb_tau;
  int stages;     // FP32 sweep: 0 (branches read their records from global memory), 1 or 2 branch-tile buffers
  int profile;    // accumulate CTA 0's phase times into d.phase_ns
  int smem_res;   // 1: residual maxima accumulated per CTA in shared memory (K <= kSmemResMax)
  int line_exact; // FP64 sweep: 1 = line subproblems by the exact dual active-set method, 0 = ALM
  // the convergence test r <= eps && s <= eps_dual on the bit patterns of
  // the residual maxima (non-negative doubles order as unsigned integers),
  // so that it takes no FP64 instruction: can_stop = !fixed, both
  // tolerances >= 0 (not NaN); their patterns (of +0 for -0)
  int can_stop;
  unsigned long long eps_bits, eps_dual_bits;
  __device__ __forceinline__ bool converged(unsigned long long r, unsigned long long s) const {
    return can_stop && r <= eps_bits && s <= eps_dual_bits;
  }
};

template <typename T>
static void set_stop_test(SweepP<T>& p) {
  p.can_stop = !p.fixed && p.eps >= 0.0 && p.eps_dual >= 0.0;
  const double e = p.eps + 0.0, ed = p.eps_dual + 0.0;
  memcpy(&p.eps_bits, &e, 8);
  memcpy(&p.eps_dual_bits, &ed, 8);
}

// instances up to which the residual maxima are accumulated in shared memory
constexpr int kSmemResMax = 1024;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------- barrier
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Device-wide barrier on one arrival counter that only grows (it is zeroed
// before every launch): at its n-th barrier a CTA adds 1 with release
// semantics and waits, with acquire loads, until the counter reaches
// n * gridDim.x.  One atomic per CTA and no reset, so the last CTA to arrive
// releases the others by its own arrival.  epoch is the calling CTA's target
// (held by thread 0).  Returns false (in every thread of the CTA) when this
// CTA gave up waiting or another CTA reported that it did.
__device__ bool grid_barrier(unsigned* count, unsigned& epoch, int* err, long long spin_limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    epoch += gridDim.x;
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    long long t0 = clock64();
    while ((int)(ld_acquire(count) - epoch) < 0) {
      if (clock64() - t0 > spin_limit) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
    }
    __threadfence();
    // another CTA may have given up: leave together (decided by one thread)
    if (ok && *(volatile int*)err) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// ------------------------------------------------ bulk async tile staging
// Branch tiles are streamed into shared memory by one thread with 1-D bulk
// copies (cp.async.bulk, completion counted on an mbarrier in bytes) while
// the CTA solves the previous tile: memory latency overlaps computation
// without needing high occupancy.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(n) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with the given parity; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, long long limit) {
  long long t0 = clock64();
  while (!mbar_test(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(b))
               : "memory");
}

constexpr int kTileV4 = 19;  // per branch: 14 record chunks, 2 z, 2 lambda, 1 u (4-vectors)

// copies of branch tile [l0, l0 + n) into a stage of kTileV4 * tile 4-vectors
template <typename T>
__device__ __forceinline__ void tile_issue(const Dev& d, int l0, int n, V4<T>* st, int tile, unsigned long long* b) {
  const unsigned one = (unsigned)(n * sizeof(V4<T>));
  mbar_arrive_tx(b, 14u * one + 2u * one + 2u * one + one);
  const V4<T>* R = (const V4<T>*)d.lrec;
  for (int c = 0; c < kRecChunks; ++c) bulk_g2s(st + c * tile, R + (size_t)c * d.L + l0, one, b);
  bulk_g2s(st + 14 * tile, (const V4<T>*)d.Z + 2 * (size_t)l0, 2u * one, b);
  bulk_g2s(st + 16 * tile, (const V4<T>*)d.LAM + 2 * (size_t)l0, 2u * one, b);
  bulk_g2s(st + 18 * tile, (const V4<T>*)d.U + l0, one, b);
}

// ------------------------------------------------------------- phases
// eq. gen_kernel for generator g from its record chunks a = (f', f'', lp, up),
// b = (lq, uq, rho, 0): clamp((rho z - lambda - f') / (f'' + rho)) and
// clamp((rho z - lambda) / rho)
template <typename T>
__device__ __forceinline__ V2<T> gen_value(const V4<T>& a, const V4<T>& b, V2<T> z, V2<T> lam) {
  const T rho = b.z;
  V2<T> x;
  x.x = clampv(div_w(rho * z.x - lam.x - a.x, a.y + rho), a.z, a.w);
  x.y = clampv(div_w(rho * z.y - lam.y, rho), b.x, b.y);
  return x;
}

template <typename T>
__device__ __forceinline__ void gen_compute(const Dev& d, int g, const V4<T>& a, const V4<T>& b) {
  ((V2<T>*)d.XG)[g] = gen_value(a, b, ((const V2<T>*)d.ZG)[g], ((const V2<T>*)d.LG)[g]);
}

template <typename T>
__device__ __forceinline__ void gen_phase(const SweepP<T>& p, int g, float sc) {
  const Dev& d = p.d;
  V4<T>* R = (V4<T>*)d.grec;
  V4<T> a = R[g], b = R[d.G + g];
  if (sc != 1.0f) {  // residual balancing changed this instance's penalty
    b.z = (T)((double)b.z * (double)sc);
    R[d.G + g] = b;
  }
  gen_compute(d, g, a, b);
}

// the FP64 line solves as calls of their own (see line_compute): the
// predicted active set, the dual method when the prediction fails its check,
// and the augmented Lagrangian for a subproblem with no feasible point
__device__ __noinline__ bool line_pred_call(const LineQP<double>& P, double* x, double* u) {
  return line_solve_predicted(P, x, u);
}
__device__ __noinline__ int line_exact_call(const LineQP<double>& P, double* x, double* u) {
  return line_solve_exact(P, x, u);
}
template <typename T>
__device__ __noinline__ void line_alm_call(const LineQP<T>& P, T* x, T* u, T beta, T tol, int outer, int newton) {
  line_solve(P, x, u, beta, tol, outer, newton);
}

// How a line solve reads its branch's sweep record: value e (0..55) of the
// layout in common.cuh, and again(e) for the values read a second time after
// the solve.
template <typename T>
struct GRec {  // in global memory (stride L) or a shared-memory tile (stride TILE)
  const T* rt;
  int rstride;
  __device__ __forceinline__ T operator()(int e) const { return rt[4 * (e >> 2) * rstride + (e & 3)]; }
  // volatile: not held in registers across the solve
  __device__ __forceinline__ T again(int e) const {
    return ((const volatile T*)rt)[4 * (e >> 2) * rstride + (e & 3)];
  }
};
template <typename T>
struct RRec {  // held in registers for the whole sweep (every index is a constant after unrolling)
  const V4<T>* r;
  __device__ __forceinline__ T operator()(int e) const {
    const V4<T>& v = r[e >> 2];
    return (e & 3) == 0 ? v.x : (e & 3) == 1 ? v.y : (e & 3) == 2 ? v.z : v.w;
  }
  __device__ __forceinline__ T again(int e) const { return (*this)(e); }
};

// Residual balancing changed this branch's penalty by the factor sc:
// Q = A'HA + rho (F'F + I) and c0 = gH + rho F'f0 change with rho.  The
// record is updated in place (rs: the branch's chunk 0, stride rstride: global
// memory or a shared-memory tile) and in global memory; returns the new rho.
// Out of line: it runs only every rb_period iterations and must not add to
// the registers of the common path.
template <typename T>
__device__ __noinline__ T rb_rescale(const Dev& d, int l, float sc, V4<T>* rs, int rstride, T rho) {
  T* rt = (T*)rs;
  auto at = [&](int e) -> T& { return rt[4 * (e >> 2) * rstride + (e & 3)]; };
  const double r0 = (double)rho;
  const double dr = r0 * ((double)sc - 1.0);
  for (int a = 0; a < 4; ++a) {
    for (int b = a; b < 4; ++b) {
      double ff = a == b ? 1.0 : 0.0;
      for (int f = 0; f < 4; ++f) ff += (double)at(10 + 4 * f + a) * (double)at(10 + 4 * f + b);
      at(pk(a, b)) = (T)((double)at(pk(a, b)) + dr * ff);
    }
  }
  for (int a = 0; a < 4; ++a) {
    double cf = 0.0;
    for (int f = 0; f < 4; ++f) cf += (double)at(10 + 4 * f + a) * (double)at(26 + f);
    at(30 + a) = (T)((double)at(30 + a) + dr * cf);
  }
  V4<T>* R = (V4<T>*)d.lrec;
  const int chunks[5] = {0, 1, 2, 7, 8};
  for (int k = 0; k < 5; ++k) R[(size_t)chunks[k] * d.L + l] = rs[chunks[k] * rstride];
  T rn = (T)(r0 * (double)sc);
  ((T*)d.trho_l)[l] = rn;
  return rn;
}

// One branch's line subproblem.  rec reads the branch's record (global
// memory, a shared-memory tile or registers); values are read where they are
// used rather than copied to registers, to keep the kernel's register count
// low.  z, lambda, u and rho are passed in.
template <typename T, typename Rec, typename Out>
__device__ __forceinline__ void line_compute_to(const SweepP<T>& p, int l, const Rec& rec, V4<T> z0, V4<T> z1,
                                                V4<T> l0, V4<T> l1, V4<T> uu, T rho, Out out, unsigned* wset = nullptr);

template <typename T, typename Rec>
__device__ __forceinline__ void line_compute(const SweepP<T>& p, int l, const Rec& rec, V4<T> z0, V4<T> z1, V4<T> l0,
                                             V4<T> l1, V4<T> uu, T rho, unsigned* wset = nullptr) {
  line_compute_to(
      p, l, rec, z0, z1, l0, l1, uu, rho,
      [&](const V4<T>& o0, const V4<T>& o1, const V4<T>& ou) {
        V4<T>* X = (V4<T>*)p.d.X;
        X[2 * l] = o0;
        X[2 * l + 1] = o1;
        ((V4<T>*)p.d.U)[l] = ou;
      },
      wset);
}

// the line update of branch l; out(o0, o1, ou) receives the couplings of its
// two ends and its line-limit multipliers
// wset (FP32 sweep, may be null): the box bounds held at the end of this
// branch's previous solve, the start of the next one's (a thread that keeps
// its branch from one ADMM iteration to the next holds it in a register)
template <typename T, typename Rec, typename Out>
__device__ __forceinline__ void line_compute_to(const SweepP<T>& p, int l, const Rec& rec, V4<T> z0, V4<T> z1,
                                                V4<T> l0, V4<T> l1, V4<T> uu, T rho, Out out, unsigned* wset) {
  const Dev& d = p.d;
  // couplings: flows p_ij q_ij p_ji q_ji (F rows 0..3), voltages dbar 0..3
  const T zf[4] = {z0.x, z0.y, z1.x, z1.y}, lf[4] = {l0.x, l0.y, l1.x, l1.y};
  const T zv[4] = {z0.z, z0.w, z1.z, z1.w}, lv[4] = {l0.z, l0.w, l1.z, l1.w};
  LineQP<T> P;
#pragma unroll
  for (int k = 0; k < 10; ++k) P.q[k] = rec(k);
  // c = c0 + F'(lambda_F - rho z_F) + lambda_V - rho z_V
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T s = rec(30 + i) + lv[i] - rho * zv[i];
#pragma unroll
    for (int f = 0; f < 4; ++f) s += rec(10 + 4 * f + i) * (lf[f] - rho * zf[f]);
    P.c[i] = s;
    P.lo[i] = rec(34 + i);
    P.hi[i] = rec(38 + i);
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
#pragma unroll
    for (int i = 0; i < 4; ++i) P.R[e][i] = rec(42 + 4 * e + i);
    P.rb[e] = rec(50 + e);
    P.on[e] = rec(54 + e) > T(0);
  }
  P.alo = rec(52);
  P.ahi = rec(53);
  P.ang = P.ahi < T(1e29);
  T x[4], u[4] = {uu.x, uu.y, uu.z, uu.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = clampv(zv[i], P.lo[i], P.hi[i]);
  if constexpr (sizeof(T) == 8) {
    // FP64 sweep: the exact solution by default -- the active set predicted in
    // FP32 and the KKT point solved and checked in FP64, else the dual
    // active-set method; the augmented Lagrangian for line_solver = 1 and for
    // a subproblem with no feasible point (it treats the rows softly)
    bool alm = !p.line_exact;
    if (p.line_exact && !line_pred_call(P, x, u)) {
      const T u_in[4] = {u[0], u[1], u[2], u[3]};
      if (line_exact_call(P, x, u) < 0) {
        alm = true;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          x[i] = clampv(zv[i], P.lo[i], P.hi[i]);
          u[i] = u_in[i];
        }
      }
    }
    if (alm) {
      const T beta = p.beta_scale * fmax(fmax(P.q[0], P.q[4]), fmax(P.q[7], P.q[9]));
      line_alm_call(P, x, u, beta, p.alm_tol, p.alm_outer, p.newton_max);
    }
  } else {
    // FP32 sweep: the augmented Lagrangian with refinement (Sec. IV-B)
    const T beta = p.beta_scale * fmax(fmax(P.q[0], P.q[4]), fmax(P.q[7], P.q[9]));
    line_solve(P, x, u, beta, p.alm_tol, p.alm_outer, p.newton_max, nullptr, wset);
  }
  // flows at the solution (F and f0 read again)
  T xf[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    T s = rec.again(26 + f);
#pragma unroll
    for (int i = 0; i < 4; ++i) s += rec.again(10 + 4 * f + i) * x[i];
    xf[f] = s;
  }
  V4<T> o0, o1, ou;
  o0.x = xf[0]; o0.y = xf[1]; o0.z = x[0]; o0.w = x[1];
  o1.x = xf[2]; o1.y = xf[3]; o1.z = x[2]; o1.w = x[3];
  ou.x = u[0]; ou.y = u[1]; ou.z = u[2]; ou.w = u[3];
  out(o0, o1, ou);
}

// line update of branch l reading its record from global memory (rs, stride L)
// or a shared-memory tile (stride TILE); applies a residual-balancing change
// of its penalty first
template <typename T>
__device__ __forceinline__ void line_from(const SweepP<T>& p, int l, float sc, V4<T>* rs, int rstride, V4<T> z0,
                                          V4<T> z1, V4<T> l0, V4<T> l1, V4<T> uu, T rho) {
  if (sc != 1.0f) rho = rb_rescale(p.d, l, sc, rs, rstride, rho);
  line_compute(p, l, GRec<T>{(const T*)rs, rstride}, z0, z1, l0, l1, uu, rho);
}

template <typename T>
__device__ __forceinline__ void line_phase(const SweepP<T>& p, int l, float sc) {
  const Dev& d = p.d;
  const V4<T>* Z = (const V4<T>*)d.Z;
  const V4<T>* LM = (const V4<T>*)d.LAM;
  line_from(p, l, sc, (V4<T>*)d.lrec + l, d.L, Z[2 * l], Z[2 * l + 1], LM[2 * l], LM[2 * l + 1],
            ((const V4<T>*)d.U)[l], ((const T*)d.trho_l)[l]);
}

// Where the residual maxima of one iteration go: with acc set, per-instance
// accumulators in the CTA's shared memory (flushed to the global slots by
// res_flush once per iteration, so the number of global atomics per instance
// is one per CTA, not one per warp task); otherwise the global slots of
// iteration parity slot directly.
struct ResDst {
  unsigned long long* acc;  // shared [2][K] or null
  unsigned long long* slots;
  int K, slot;
  int kbase;  // instance of acc[0] (a cluster's one-instance accumulator; 0 otherwise)
  // the maxima as the bit patterns of non-negative doubles (ordered as
  // integers); positive values only
  __device__ __forceinline__ void put_bits(int inst, unsigned long long r, unsigned long long s) const {
    if (acc) {
      if (r) atomicMax(&acc[inst - kbase], r);
      if (s) atomicMax(&acc[K + inst - kbase], s);
    } else {
      if (r) atomicMax(&slots[(slot * 2 + 0) * K + inst], r);
      if (s) atomicMax(&slots[(slot * 2 + 1) * K + inst], s);
    }
  }
  // r, s >= 0 and not NaN.  In FP64 the test takes no FP64 comparison (an
  // FP64 instruction issues at a small fraction of the FP32 rate on GB300):
  // a positive double's pattern is a positive integer.  The FP32 overload
  // widens with the conversion instruction and compares in FP64, which
  // measured faster there than widening in integer operations.
  __device__ __forceinline__ void put(int inst, double r, double s) const {
    const long long br = (long long)bits_of(r), bs = (long long)bits_of(s);
    put_bits(inst, br > 0 ? (unsigned long long)br : 0ull, bs > 0 ? (unsigned long long)bs : 0ull);
  }
  __device__ __forceinline__ void put(int inst, float rf, float sf) const {
    const double r = rf, s = sf;
    if (acc) {
      if (r > 0.0) atomicMax(&acc[inst - kbase], (unsigned long long)__double_as_longlong(r));
      if (s > 0.0) atomicMax(&acc[K + inst - kbase], (unsigned long long)__double_as_longlong(s));
    } else {
      if (r > 0.0) atomicMax(&slots[(slot * 2 + 0) * K + inst], (unsigned long long)__double_as_longlong(r));
      if (s > 0.0) atomicMax(&slots[(slot * 2 + 1) * K + inst], (unsigned long long)__double_as_longlong(s));
    }
  }
};

// the CTA's shared-memory maxima into the global slots, and back to zero
// (every thread of the CTA calls it after a __syncthreads)
__device__ __forceinline__ void res_flush(const ResDst& o) {
  for (int k = threadIdx.x; k < o.K; k += blockDim.x) {
    const unsigned long long r = o.acc[k], s = o.acc[o.K + k];
    if (r) atomicMax(&o.slots[(o.slot * 2 + 0) * o.K + k], r);
    if (s) atomicMax(&o.slots[(o.slot * 2 + 1) * o.K + k], s);
    o.acc[k] = 0ull;
    o.acc[o.K + k] = 0ull;
  }
}

// Residual maxima.  FP64 takes them on the bit patterns as integers, which
// order non-negative doubles alike; a NaN's pattern (sign cleared) exceeds
// every other, so a NaN component always reaches the test.  FP32 uses fmax,
// which passes over a NaN component (a non-finite state is then caught by
// the SQP's finiteness checks).
//   rmax: max of two residuals (non-negative or NaN)
//   amax: max(|a|, |b|)
//   nan_big: a NaN residual as 1e30, so that the test cannot pass on it
template <typename T>
__device__ __forceinline__ T rmax(T a, T b) {
  if constexpr (sizeof(T) == 8) {
    const unsigned long long x = bits_of(a) & 0x7fffffffffffffffull, y = bits_of(b) & 0x7fffffffffffffffull;
    return double_of(x > y ? x : y);
  } else {
    return fmax(a, b);
  }
}
template <typename T>
__device__ __forceinline__ T amax(T a, T b) {
  if constexpr (sizeof(T) == 8) return rmax(a, b);
  else return fmax(fabs(a), fabs(b));
}
template <typename T>
__device__ __forceinline__ T nan_big(T v) {
  if constexpr (sizeof(T) == 8) return (bits_of(v) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull ? T(1e30) : v;
  else return v == v ? v : T(1e30);
}

// Warp-level max of the residuals over runs of lanes that hold the same
// instance (buses are sorted by instance, so runs are contiguous): a segmented
// shuffle-down reduction in the sweep precision, then one 64-bit atomicMax per
// run and residual.  All 32 lanes must call it; lanes without a bus pass inst = -1.
template <typename T>
__device__ __forceinline__ void res_max2(const ResDst& dst, T r, T s, int inst) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T r2 = __shfl_down_sync(FULL, r, o);
    T s2 = __shfl_down_sync(FULL, s, o);
    int k2 = __shfl_down_sync(FULL, inst, o);
    if (lane + o < 32 && k2 == inst) {
      r = rmax(r, r2);
      s = rmax(s, s2);
    }
  }
  int kprev = __shfl_up_sync(FULL, inst, 1);
  bool leader = (lane == 0 || kprev != inst) && inst >= 0;
  if (leader) dst.put(inst, r, s);
}

// res_max2 for two tasks at once
template <typename T>
__device__ __forceinline__ void res_max2_pair(const ResDst& dst, T ra, T sa, int ka, T rb, T sb, int kb) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T ra2 = __shfl_down_sync(FULL, ra, o);
    T sa2 = __shfl_down_sync(FULL, sa, o);
    int ka2 = __shfl_down_sync(FULL, ka, o);
    T rb2 = __shfl_down_sync(FULL, rb, o);
    T sb2 = __shfl_down_sync(FULL, sb, o);
    int kb2 = __shfl_down_sync(FULL, kb, o);
    if (lane + o < 32 && ka2 == ka) {
      ra = rmax(ra, ra2);
      sa = rmax(sa, sa2);
    }
    if (lane + o < 32 && kb2 == kb) {
      rb = rmax(rb, rb2);
      sb = rmax(sb, sb2);
    }
  }
  const int kpa = __shfl_up_sync(FULL, ka, 1), kpb = __shfl_up_sync(FULL, kb, 1);
  if ((lane == 0 || kpa != ka) && ka >= 0) dst.put(ka, ra, sa);
  if ((lane == 0 || kpb != kb) && kb >= 0) dst.put(kb, rb, sb);
}

// ---------------------------------------------------------- bus update
// Bus update (eq. bus_kernel), multiplier update (eq. multiplier) and
// residuals, one warp per task of consecutive whole buses: lane j takes one
// entry -- a generator or a branch end -- of the task's buses and loads its
// couplings; the per-bus sums of the 2x2 system are formed by a segmented
// warp scan over the bus ids (a bus's entries are consecutive lanes); the
// segment's last lane solves its bus and the solution is broadcast back to
// the segment, where every lane updates its own coupling.

struct Slot {
  int bus, code, inst;  // bus -1: empty lane
};

__device__ __forceinline__ Slot load_slot(const Dev& d, int t, int lane) {
  const size_t i = 32 * (size_t)t + lane;
  Slot s;
  s.bus = d.pbus[i];
  s.code = d.pent[i];
  s.inst = d.pinst[i];
  return s;
}

template <typename T>
__device__ __forceinline__ void entry_load(const Dev& d, int c, V4<T>& x, V4<T>& lm, V4<T>& zo, T& r) {
  if (c < 0) {
    const int g = -c - 1;
    V2<T> a = ((const V2<T>*)d.XG)[g], b = ((const V2<T>*)d.LG)[g], z = ((const V2<T>*)d.ZG)[g];
    r = ((const V4<T>*)d.grec)[d.G + g].z;
    x = {a.x, a.y, T(0), T(0)};
    lm = {b.x, b.y, T(0), T(0)};
    zo = {z.x, z.y, T(0), T(0)};
  } else {
    x = ((const V4<T>*)d.X)[c];
    lm = ((const V4<T>*)d.LAM)[c];
    zo = ((const V4<T>*)d.Z)[c];
    r = ((const T*)d.trho_l)[c >> 1];
  }
}

// contributions to the bus sums: c = lambda + rho x per coupling; the 2x2
// matrix sums 1/rho over every coupled flow, generators enter with +, branch
// ends with - (they draw power from the bus)
// a / r: in FP64 the product with one reciprocal of r (a correctly rounded
// division costs many FP64 instructions on GB300, whose FP64 rate is a small
// fraction of FP32); in FP32 the special-function quotient
template <typename T>
__device__ __forceinline__ T over_r(T a, T r, T ir) {
  if constexpr (sizeof(T) == 8) return a * ir;
  else return div_w(a, r);
}

// 1/r of a coupling's penalty, used by entry_sums and (FP64) entry_values:
// the FP64 sweep takes the correctly rounded quotient once per coupling and
// iteration (ir_once) and passes it to both; the FP32 sweep takes the
// special-function quotient where entry_sums uses it (ir_at), as
// entry_values does not need it
template <typename T>
__device__ __forceinline__ T ir_once(T r) {
  if constexpr (sizeof(T) == 8) return div_w(T(1), r);
  else return T(0);
}
template <typename T>
__device__ __forceinline__ T ir_at(T r, T once) {
  if constexpr (sizeof(T) == 8) return once;
  else return div_w(T(1), r);
}

// ir = 1/r (see ir_once)
template <typename T>
__device__ __forceinline__ void entry_sums(int c, const V4<T>& x, const V4<T>& lm, T r, T ir, T* S) {
  S[0] += ir;
  if (c < 0) {
    S[1] += over_r(lm.x + r * x.x, r, ir);
    S[2] += over_r(lm.y + r * x.y, r, ir);
  } else {
    S[1] -= over_r(lm.x + r * x.x, r, ir);
    S[2] -= over_r(lm.y + r * x.y, r, ir);
    S[3] += r;
    S[4] += lm.z + r * x.z;
    S[5] += lm.w + r * x.w;
  }
}

// the 2x2 system (A Q^-1 A') nu = A Q^-1 c - b of the bus's power-balance rows
// with shunts, then d_w and d_theta; writes ZB, NU
template <typename T>
__device__ __forceinline__ void bus_values(V4<T> br, int isref, const T* S, T& n1, T& n2, T& dw, T& dth) {
  const T gsh = br.z, bsh = br.w;
  const T iQw = S[3] > T(0) ? div_w(T(1), S[3]) : T(0);  // a bus without branch ends has no voltage copies
  const T M11 = S[0] + gsh * gsh * iQw;
  const T M22 = S[0] + bsh * bsh * iQw;
  const T M12 = -gsh * bsh * iQw;
  const T v1 = S[1] - gsh * S[4] * iQw - br.x;
  const T v2 = S[2] + bsh * S[4] * iQw - br.y;
  const T det = M11 * M22 - M12 * M12;
  const T idet = sizeof(T) == 8 ? div_w(T(1), det) : T(0);
  n1 = over_r(M22 * v1 - M12 * v2, det, idet);
  n2 = over_r(M11 * v2 - M12 * v1, det, idet);
  dw = (S[4] + gsh * n1 - bsh * n2) * iQw;
  dth = (isref || !(S[3] > T(0))) ? T(0) : over_r(S[5], S[3], iQw);
}

template <typename T>
__device__ __forceinline__ void bus_solve(const Dev& d, int bus, V4<T> br, int isref, const T* S, T& n1, T& n2,
                                          T& dw, T& dth) {
  bus_values(br, isref, S, n1, n2, dw, dth);
  V2<T> zb, nu;
  zb.x = dw; zb.y = dth;
  nu.x = n1; nu.y = n2;
  ((V2<T>*)d.ZB)[bus] = zb;
  ((V2<T>*)d.NU)[bus] = nu;
}

// bus-side value, multiplier update and residuals of one coupling
template <typename T>
__device__ __forceinline__ void entry_store(const Dev& d, int c, const V4<T>& zn, const V4<T>& ln) {
  if (c < 0) {
    const int g = -c - 1;
    ((V2<T>*)d.ZG)[g] = V2<T>{zn.x, zn.y};
    ((V2<T>*)d.LG)[g] = V2<T>{ln.x, ln.y};
  } else {
    ((V4<T>*)d.Z)[c] = zn;
    ((V4<T>*)d.LAM)[c] = ln;
  }
}

// new bus-side value zn and multiplier ln of one coupling, with its residuals
// (generator couplings in the x, y components, z and w zero)
template <typename T>
__device__ __forceinline__ void entry_values(int c, const V4<T>& x, const V4<T>& lm, const V4<T>& zo, T r, T ir, T n1,
                                             T n2, T dw, T dth, T& rm, T& sm, V4<T>& zn, V4<T>& ln) {
  if (c < 0) {
    zn.x = over_r(lm.x + r * x.x - n1, r, ir);
    zn.y = over_r(lm.y + r * x.y - n2, r, ir);
    zn.z = zn.w = T(0);
    sm = rmax(sm, r * amax(zn.x - zo.x, zn.y - zo.y));
    const T rx = x.x - zn.x, ry = x.y - zn.y;
    rm = rmax(rm, amax(rx, ry));
    ln.x = lm.x + r * rx;
    ln.y = lm.y + r * ry;
    ln.z = ln.w = T(0);
  } else {
    zn.x = over_r(lm.x + r * x.x + n1, r, ir);
    zn.y = over_r(lm.y + r * x.y + n2, r, ir);
    zn.z = dw;
    zn.w = dth;
    const T a1 = amax(zn.x - zo.x, zn.y - zo.y);
    const T a2 = amax(zn.z - zo.z, zn.w - zo.w);
    sm = rmax(sm, r * rmax(a1, a2));
    const T rx = x.x - zn.x, ry = x.y - zn.y, rw = x.z - zn.z, rt = x.w - zn.w;
    rm = rmax(rm, rmax(amax(rx, ry), amax(rw, rt)));
    ln.x = lm.x + r * rx;
    ln.y = lm.y + r * ry;
    ln.z = lm.z + r * rw;
    ln.w = lm.w + r * rt;
  }
}

template <typename T>
__device__ __forceinline__ void entry_update(const Dev& d, int c, const V4<T>& x, const V4<T>& lm, const V4<T>& zo, T r,
                                             T ir, T n1, T n2, T dw, T dth, T& rm, T& sm) {
  V4<T> zn, ln;
  entry_values(c, x, lm, zo, r, ir, n1, n2, dw, dth, rm, sm, zn, ln);
  entry_store(d, c, zn, ln);
}

// segmented inclusive scan of the six sums by bus id: the last lane of each
// run of equal ids ends with its bus's totals
template <typename T>
__device__ __forceinline__ void seg_scan(int bus, T* S) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T a[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = __shfl_up_sync(FULL, S[k], o);
    const int bu = __shfl_up_sync(FULL, bus, o);
    if (lane >= o && bu == bus) {
#pragma unroll
      for (int k = 0; k < 6; ++k) S[k] += a[k];
    }
  }
}

// seg_scan over two independent tasks at once (their shuffles interleave)
template <typename T>
__device__ __forceinline__ void seg_scan2(int bus_a, T* Sa, int bus_b, T* Sb) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T a[6], b[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      a[k] = __shfl_up_sync(FULL, Sa[k], o);
      b[k] = __shfl_up_sync(FULL, Sb[k], o);
    }
    const int ua = __shfl_up_sync(FULL, bus_a, o);
    const int ub = __shfl_up_sync(FULL, bus_b, o);
    if (lane >= o && ua == bus_a) {
#pragma unroll
      for (int k = 0; k < 6; ++k) Sa[k] += a[k];
    }
    if (lane >= o && ub == bus_b) {
#pragma unroll
      for (int k = 0; k < 6; ++k) Sb[k] += b[k];
    }
  }
}

// What of one task of at most 32 entries stays fixed during a sweep: this
// lane's slot, whether it is the last lane of its bus, and for that lane the
// bus's load and shunts
template <typename T>
struct TaskStatic {
  Slot s;
  bool last;
  V4<T> br;
  int isref;
};

template <typename T>
__device__ __forceinline__ TaskStatic<T> task_static(const Dev& d, Slot s) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  TaskStatic<T> a;
  a.s = s;
  const int bnext = __shfl_down_sync(FULL, s.bus, 1);
  a.last = s.bus >= 0 && (lane == 31 || bnext != s.bus);
  a.br = {T(0), T(0), T(0), T(0)};
  a.isref = 0;
  if (a.last) {
    a.br = ((const V4<T>*)d.brec)[s.bus];  // pdk qdk gs bs
    a.isref = d.isref[s.bus];
  }
  return a;
}

// the loads of one task: this lane's coupling (lanes of finished instances
// are emptied)
template <typename T>
struct TaskData {
  Slot s;
  bool last;
  V4<T> x, lm, zo, br;
  T r;
  int isref;
};

template <typename T, bool kDone = true>
__device__ __forceinline__ TaskData<T> task_load(const Dev& d, const TaskStatic<T>& st, const int* s_done) {
  TaskData<T> a;
  a.s = st.s;
  a.last = st.last;
  a.br = st.br;
  a.isref = st.isref;
  if (kDone && a.s.bus >= 0 && s_done[a.s.inst]) {
    a.s.bus = a.s.inst = -1;
    a.last = false;
  }
  a.x = a.lm = a.zo = {T(0), T(0), T(0), T(0)};
  a.r = T(1);
  if (a.s.bus >= 0) entry_load(d, a.s.code, a.x, a.lm, a.zo, a.r);
  return a;
}

// two tasks from their loaded data, solved together: the dependent chains of
// the two (scan, 2x2 solve, broadcast, update, residual reduction) interleave
// in one warp.  Tasks never share an entry or a bus, so the order of their
// stores does not matter.  All 32 lanes call it.
template <typename T>
__device__ __forceinline__ void bus_task_pair(const Dev& d, const TaskData<T>& a, const TaskData<T>& b,
                                              const ResDst& dst) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  T Sa[6] = {0, 0, 0, 0, 0, 0}, Sb[6] = {0, 0, 0, 0, 0, 0};
  const T ira = ir_once(a.r), irb = ir_once(b.r);
  if (a.s.bus >= 0) entry_sums(a.s.code, a.x, a.lm, a.r, ir_at(a.r, ira), Sa);
  if (b.s.bus >= 0) entry_sums(b.s.code, b.x, b.lm, b.r, ir_at(b.r, irb), Sb);
  seg_scan2(a.s.bus, Sa, b.s.bus, Sb);
  T n1a = 0, n2a = 0, dwa = 0, dta = 0, n1b = 0, n2b = 0, dwb = 0, dtb = 0;
  if (a.last) bus_solve(d, a.s.bus, a.br, a.isref, Sa, n1a, n2a, dwa, dta);
  if (b.last) bus_solve(d, b.s.bus, b.br, b.isref, Sb, n1b, n2b, dwb, dtb);
  const unsigned ha = __ballot_sync(FULL, a.last) >> lane, hb = __ballot_sync(FULL, b.last) >> lane;
  const int srca = ha ? lane + __ffs(ha) - 1 : lane, srcb = hb ? lane + __ffs(hb) - 1 : lane;
  n1a = __shfl_sync(FULL, n1a, srca);
  n1b = __shfl_sync(FULL, n1b, srcb);
  n2a = __shfl_sync(FULL, n2a, srca);
  n2b = __shfl_sync(FULL, n2b, srcb);
  dwa = __shfl_sync(FULL, dwa, srca);
  dwb = __shfl_sync(FULL, dwb, srcb);
  dta = __shfl_sync(FULL, dta, srca);
  dtb = __shfl_sync(FULL, dtb, srcb);
  T rma = T(0), sma = T(0), rmb = T(0), smb = T(0);
  if (a.s.bus >= 0) {
    entry_update(d, a.s.code, a.x, a.lm, a.zo, a.r, ira, n1a, n2a, dwa, dta, rma, sma);
    rma = nan_big(rma);
    sma = nan_big(sma);
  }
  if (b.s.bus >= 0) {
    entry_update(d, b.s.code, b.x, b.lm, b.zo, b.r, irb, n1b, n2b, dwb, dtb, rmb, smb);
    rmb = nan_big(rmb);
    smb = nan_big(smb);
  }
  res_max2_pair(dst, rma, sma, a.s.inst, rmb, smb, b.s.inst);
}

// one task alone in its warp.  The FP64 sweep gives each warp one task where
// the launch allows it: FP64 arithmetic issues at a small fraction of the
// FP32 rate in each SM partition, so two tasks interleaved in one warp take
// about twice as long as one, where in FP32 they overlap.  The arithmetic is
// that of task a of bus_task_pair.  All 32 lanes call it.
template <typename T>
__device__ __forceinline__ void bus_task_one(const Dev& d, const TaskData<T>& a, const ResDst& dst) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  T S[6] = {0, 0, 0, 0, 0, 0};
  const T ir = ir_once(a.r);
  if (a.s.bus >= 0) entry_sums(a.s.code, a.x, a.lm, a.r, ir_at(a.r, ir), S);
  seg_scan(a.s.bus, S);
  T n1 = 0, n2 = 0, dw = 0, dt = 0;
  if (a.last) bus_solve(d, a.s.bus, a.br, a.isref, S, n1, n2, dw, dt);
  const unsigned h = __ballot_sync(FULL, a.last) >> lane;
  const int src = h ? lane + __ffs(h) - 1 : lane;
  n1 = __shfl_sync(FULL, n1, src);
  n2 = __shfl_sync(FULL, n2, src);
  dw = __shfl_sync(FULL, dw, src);
  dt = __shfl_sync(FULL, dt, src);
  T rm = T(0), sm = T(0);
  if (a.s.bus >= 0) {
    entry_update(d, a.s.code, a.x, a.lm, a.zo, a.r, ir, n1, n2, dw, dt, rm, sm);
    rm = nan_big(rm);
    sm = nan_big(sm);
  }
  res_max2(dst, rm, sm, a.s.inst);
}

// one bus with more than 32 entries (entries [q0, q1) of ent); lanes loop
template <typename T, bool kDone = true>
__device__ void bus_task_big(const SweepP<T>& p, int q0, int q1, const ResDst& dst, const int* s_done) {
  const Dev& d = p.d;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int bus = d.ebus[q0];
  const int inst = d.bus_inst[bus];
  if (kDone && s_done[inst]) {
    res_max2(dst, T(0), T(0), -1);
    return;
  }
  T S[6] = {0, 0, 0, 0, 0, 0};
  for (int q = q0 + lane; q < q1; q += 32) {
    V4<T> x, lm, zo;
    T r;
    const int c = d.ent[q];
    entry_load(d, c, x, lm, zo, r);
    entry_sums(c, x, lm, r, div_w(T(1), r), S);
  }
  seg_scan(bus, S);
  T n1 = 0, n2 = 0, dw = 0, dth = 0;
  if (lane == 31) bus_solve(d, bus, ((const V4<T>*)d.brec)[bus], d.isref[bus], S, n1, n2, dw, dth);
  n1 = __shfl_sync(FULL, n1, 31);
  n2 = __shfl_sync(FULL, n2, 31);
  dw = __shfl_sync(FULL, dw, 31);
  dth = __shfl_sync(FULL, dth, 31);
  T rm = T(0), sm = T(0);
  for (int q = q0 + lane; q < q1; q += 32) {
    V4<T> x, lm, zo;
    T r;
    const int c = d.ent[q];
    entry_load(d, c, x, lm, zo, r);
    entry_update(d, c, x, lm, zo, r, div_w(T(1), r), n1, n2, dw, dth, rm, sm);
  }
  rm = nan_big(rm);
  sm = nan_big(sm);
  res_max2(dst, rm, sm, inst);
}

// RES: every thread has at most one generator or branch and every warp at
// most two bus tasks (checked by the launcher); their static data -- the
// branch record, the generator record, instance ids, task slots and bus data
// -- is loaded once, before the first iteration, and held in registers.
template <typename T, bool RES>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && !RES) ? 2 : 1) k_sweep(SweepP<T> p) {
  const Dev& d = p.d;
  // dynamic shared memory: residual accumulators (2K 64-bit, when smem_res),
  // finished flags (K ints), penalty factors (K floats), branch tiles
  extern __shared__ __align__(128) unsigned long long s_dyn[];
  const int K = d.K;
  unsigned long long* s_acc = p.smem_res ? s_dyn : nullptr;
  int* s_done = (int*)(s_dyn + (p.smem_res ? 2 * K : 0));
  float* s_scale = (float*)(s_done + K);
  const int nthreads = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  // FP32 sweep: branch tiles of blockDim.x are staged in one or two
  // shared-memory buffers (stages 1, 2), or read from global memory (stages 0)
  const bool kTiled = !RES && sizeof(T) == 4 && p.stages > 0;
  const int tile = blockDim.x;
  V4<T>* stage0 = (V4<T>*)(((uintptr_t)(s_scale + K) + 127) & ~(uintptr_t)127);
  const bool two = p.stages > 1;
  V4<T>* stage1 = two ? stage0 + kTileV4 * tile : stage0;
  unsigned long long* tbar = (unsigned long long*)(stage1 + kTileV4 * tile);
  unsigned tph0 = 0, tph1 = 0;
  if (kTiled && threadIdx.x == 0) {
    mbar_init(&tbar[0], 1);
    mbar_init(&tbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    s_done[k] = d.admm_done[k];
    s_scale[k] = 1.0f;
    if (s_acc) s_acc[k] = s_acc[K + k] = 0ull;
  }
  __syncthreads();
  // RES: this thread's phase-A item and its record, this warp's two bus tasks
  const int lane = threadIdx.x & 31, wid = tid >> 5, nw = nthreads >> 5;
  const Slot none = {-1, 0, -1};
  int my_k = -1;
  V4<T> rr[kRecChunks];
  T my_rho = T(0);
  unsigned my_wset = 0u;  // the box bounds held at the end of the branch's last solve
  TaskStatic<T> ta, tb;
  if (RES) {
    if (tid < d.G) {
      my_k = d.gen_inst[tid];
      rr[0] = ((const V4<T>*)d.grec)[tid];
      rr[1] = ((const V4<T>*)d.grec)[d.G + tid];
    } else if (tid < d.G + d.L) {
      const int l = tid - d.G;
      my_k = d.br_inst[l];
#pragma unroll
      for (int c = 0; c < kRecChunks; ++c) rr[c] = ((const V4<T>*)d.lrec)[(size_t)c * d.L + l];
      my_rho = ((const T*)d.trho_l)[l];
      my_wset = d.wset[l];
    }
    ta = task_static<T>(d, wid < d.NT ? load_slot(d, wid, lane) : none);
    tb = task_static<T>(d, wid + nw < d.NT ? load_slot(d, wid + nw, lane) : none);
  }
  unsigned epoch = 0;  // this CTA's barrier target
  int it = 0;
  bool aborted = false;
  unsigned long long tp0 = 0, tp1 = 0;
  const bool prof = p.profile && blockIdx.x == 0 && threadIdx.x == 0;
  for (it = 0; it < p.max_iter; ++it) {
    const int slot = it & 1;
    if (prof) tp0 = gtimer();
    // phase A: generators then branches
    if (RES) {
      if (my_k >= 0 && !s_done[my_k]) {
        if (tid < d.G) {
          gen_compute(d, tid, rr[0], rr[1]);
        } else {
          const int l = tid - d.G;
          const V4<T>* Z = (const V4<T>*)d.Z;
          const V4<T>* LM = (const V4<T>*)d.LAM;
          line_compute(p, l, RRec<T>{rr}, Z[2 * l], Z[2 * l + 1], LM[2 * l], LM[2 * l + 1], ((const V4<T>*)d.U)[l],
                       my_rho, &my_wset);
        }
      }
    } else if (!kTiled) {
      for (int u = tid; u < d.G + d.L; u += nthreads) {
        if (u < d.G) {
          int k = d.gen_inst[u];
          if (!s_done[k]) gen_phase(p, u, s_scale[k]);
        } else {
          int l = u - d.G;
          int k = d.br_inst[l];
          if (!s_done[k]) line_phase(p, l, s_scale[k]);
        }
      }
    } else {
      for (int g = tid; g < d.G; g += nthreads) {
        int k = d.gen_inst[g];
        if (!s_done[k]) gen_phase(p, g, s_scale[k]);
      }
      const int ntiles = (d.L + tile - 1) / tile;
      int t = blockIdx.x;
      int sidx = 0;
      if (t < ntiles && threadIdx.x == 0) {
        asm volatile("fence.proxy.async;" ::: "memory");  // z, lambda were written by generic stores
        int n0 = d.L - t * tile < tile ? d.L - t * tile : tile;
        tile_issue(d, t * tile, n0, stage0, tile, &tbar[0]);
      }
      bool tile_fail = false;
      while (t < ntiles) {
        const int tn = t + gridDim.x;
        V4<T>* cur = sidx ? stage1 : stage0;
        if (two && tn < ntiles && threadIdx.x == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the other stage was read generically
          int n1 = d.L - tn * tile < tile ? d.L - tn * tile : tile;
          tile_issue(d, tn * tile, n1, sidx ? stage0 : stage1, tile, &tbar[sidx ^ 1]);
        }
        bool ok = mbar_wait(&tbar[sidx], sidx ? tph1 : tph0, p.spin_limit);
        if (__syncthreads_or(!ok)) {
          // give the copies in flight a bounded chance to land, then report
          if (threadIdx.x == 0) {
            atomicExch(d.err, 1);
            mbar_wait(&tbar[0], tph0, p.spin_limit);
            mbar_wait(&tbar[1], tph1, p.spin_limit);
          }
          tile_fail = true;
          break;
        }
        if (sidx) tph1 ^= 1u; else tph0 ^= 1u;
        const int l = t * tile + threadIdx.x;
        if (l < d.L) {
          int k = d.br_inst[l];
          if (!s_done[k]) {
            const int j = threadIdx.x;
            line_from(p, l, s_scale[k], cur + j, tile, cur[14 * tile + 2 * j], cur[14 * tile + 2 * j + 1],
                         cur[16 * tile + 2 * j], cur[16 * tile + 2 * j + 1], cur[18 * tile + j],
                         ((const T*)d.trho_l)[l]);
          }
        }
        __syncthreads();  // the stage may be refilled
        t = tn;
        if (two) {
          sidx ^= 1;
        } else if (t < ntiles && threadIdx.x == 0) {  // one buffer: load the next tile now
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          int n1 = d.L - t * tile < tile ? d.L - t * tile : tile;
          tile_issue(d, t * tile, n1, stage0, tile, &tbar[0]);
        }
      }
      (void)tile_fail;
    }
    // reset the slot used two iterations ago (read by every CTA before the last barrier)
    if (blockIdx.x == 0)
      for (int k = threadIdx.x; k < K; k += blockDim.x) {
        d.res_slots[(slot * 2 + 0) * K + k] = 0ull;
        d.res_slots[(slot * 2 + 1) * K + k] = 0ull;
      }
    if (prof) { tp1 = gtimer(); atomicAdd(&d.phase_ns[0], tp1 - tp0); }
    if (!grid_barrier(d.bar, epoch, d.err, p.spin_limit)) { aborted = true; break; }
    if (prof) { tp0 = gtimer(); atomicAdd(&d.phase_ns[1], tp0 - tp1); }
    const ResDst dst = {s_acc, d.res_slots, K, slot, 0};
    // phase B: buses, in warp tasks of consecutive whole buses, two tasks at a
    // time (every entry belongs to one task, so the loads ahead never read
    // what the current tasks write); loop bounds are uniform per warp so that
    // all lanes reduce together
    if (RES) {
      if (sizeof(T) == 8 && nw >= d.NT) {  // FP64, one task per warp
        if (wid < d.NT) bus_task_one(d, task_load<T>(d, ta, s_done), dst);
      } else if (wid < d.NT) {
        bus_task_pair(d, task_load<T>(d, ta, s_done), task_load<T>(d, tb, s_done), dst);
      }
      for (int b = wid; b < d.NBIG; b += nw) bus_task_big(p, d.big[2 * b], d.big[2 * b + 1], dst, s_done);
    } else {
      auto slot_at = [&](int t) { return t < d.NT ? load_slot(d, t, lane) : none; };
      // tasks wid, wid + nw, ... taken two at a time; the slots of the next
      // pair are in flight while a pair is solved
      Slot s1a = slot_at(wid + 2 * nw), s1b = slot_at(wid + 3 * nw);
      TaskData<T> ca = task_load<T>(d, task_static<T>(d, slot_at(wid)), s_done);
      TaskData<T> cb = task_load<T>(d, task_static<T>(d, slot_at(wid + nw)), s_done);
      for (int t = wid; t < d.NT; t += 2 * nw) {
        bus_task_pair(d, ca, cb, dst);
        ca = task_load<T>(d, task_static<T>(d, s1a), s_done);
        cb = task_load<T>(d, task_static<T>(d, s1b), s_done);
        s1a = slot_at(t + 4 * nw);
        s1b = slot_at(t + 5 * nw);
      }
      for (int b = wid; b < d.NBIG; b += nw) bus_task_big(p, d.big[2 * b], d.big[2 * b + 1], dst, s_done);
    }
    if (s_acc) {
      __syncthreads();
      res_flush(dst);
    }
    if (prof) { tp1 = gtimer(); atomicAdd(&d.phase_ns[2], tp1 - tp0); }
    if (!grid_barrier(d.bar, epoch, d.err, p.spin_limit)) { aborted = true; break; }
    // residual test (Sec. IV-B) and residual balancing, evaluated identically by every CTA
    const bool rb_now = p.rb_period > 0 && ((it + 1) % p.rb_period) == 0;
    int all = 1;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      s_scale[k] = 1.0f;
      if (s_done[k]) continue;
      const unsigned long long rbits = d.res_slots[(slot * 2 + 0) * K + k];
      const unsigned long long sbits = d.res_slots[(slot * 2 + 1) * K + k];
      const bool conv = p.converged(rbits, sbits);
      if (!conv && rb_now) {
        const double r = __longlong_as_double((long long)rbits), s = __longlong_as_double((long long)sbits);
        float f = 1.0f;
        if (r > p.rb_mu * s) f = (float)p.rb_tau;
        else if (s > p.rb_mu * r) f = (float)(1.0 / p.rb_tau);
        s_scale[k] = f;
        if (blockIdx.x == 0 && f != 1.0f) d.rho_fac[k] *= (double)f;
      }
      if (p.fixed) { all = 0; continue; }
      if (conv) {
        s_done[k] = 1;
        if (blockIdx.x == 0) {
          d.admm_done[k] = 1;
          d.admm_iters[k] = it + 1;
          d.admm_rs[k] = __longlong_as_double((long long)rbits);
          d.admm_rs[K + k] = __longlong_as_double((long long)sbits);
        }
      } else {
        all = 0;
      }
    }
    all = __syncthreads_and(all);
    if (prof) atomicAdd(&d.phase_ns[3], gtimer() - tp1);
    if (all && !p.fixed) { ++it; break; }
  }
  if (RES && sizeof(T) == 4 && tid >= d.G && tid < d.G + d.L) d.wset[tid - d.G] = (uint16_t)my_wset;
  // record the residuals of unfinished instances
  if (blockIdx.x == 0 && !aborted) {
    int last = (it - 1) & 1;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      if (d.admm_done[k] && !p.fixed) continue;
      d.admm_iters[k] = it;
      d.admm_rs[k] = __longlong_as_double((long long)d.res_slots[(last * 2 + 0) * K + k]);
      d.admm_rs[K + k] = __longlong_as_double((long long)d.res_slots[(last * 2 + 1) * K + k]);
    }
  }
}

// ------------------------------------------------ one cluster per instance
// With sweep_stages 4 every instance is swept by one thread-block cluster of
// its own (up to 16 CTAs): the two barriers of an iteration are the cluster's
// hardware barrier instead of a device-wide one, the residual maxima are
// accumulated in each CTA's shared memory and combined through distributed
// shared memory, and clusters of different instances never wait on one
// another.  There is no spin-wait in this form.
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; memory accesses before it are
// visible to the whole cluster after it
__device__ __forceinline__ void cluster_barrier() {
  __syncwarp();  // the .aligned forms want the whole warp converged
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the 64-bit word at p's offset in the shared memory of the cluster's CTA `rank`
__device__ __forceinline__ unsigned long long ld_cluster_u64(const void* p, unsigned rank) {
  unsigned a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_addr(p)), "r"(rank));
  unsigned long long v;
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
  return v;
}

// RES: the cluster has a thread for every generator and branch of its
// instance and a warp for every two of its bus tasks (checked by the
// launcher); the records, instance data and task slots are then loaded once
// and held in registers, as in the resident form of k_sweep.
template <typename T, bool RES>
__global__ void __launch_bounds__(256, 1) k_sweep_cluster(SweepP<T> p) {
  const Dev& d = p.d;
  const unsigned FULL = 0xffffffffu;
  const int K = d.K;
  const int k = (int)cluster_index();
  const int cs = (int)cluster_nctarank(), rank = (int)cluster_ctarank();
  __shared__ unsigned long long s_res[2][2];  // this CTA's maxima (r, s), by iteration parity
  __shared__ double s_rs[2];
  __shared__ int s_stop;
  if (threadIdx.x < 4) (&s_res[0][0])[threadIdx.x] = 0ull;
  if (d.admm_done[k]) return;  // the whole cluster skips an instance that is not running
  cluster_barrier();  // every CTA has started before any distributed shared memory access
  const int nth = cs * blockDim.x, ct = rank * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, cw = ct >> 5, nwc = nth >> 5;
  const int g0 = d.gen_off[k], nG = d.gen_off[k + 1] - g0, l0 = d.br_off[k], l1 = d.br_off[k + 1];
  const int t0 = d.task_off[k], t1 = d.task_off[k + 1], b0 = d.big_off[k], b1 = d.big_off[k + 1];
  const Slot none = {-1, 0, -1};
  const bool prof = p.profile && blockIdx.x == 0 && threadIdx.x == 0;
  // RES: this thread's generator or branch record, this warp's two tasks
  V4<T> rr[kRecChunks];
  T my_rho = T(0);
  unsigned my_wset = 0u;  // the box bounds held at the end of the branch's last solve
  TaskStatic<T> ta, tb;
  if (RES) {
    if (ct < nG) {
      rr[0] = ((const V4<T>*)d.grec)[g0 + ct];
      rr[1] = ((const V4<T>*)d.grec)[d.G + g0 + ct];
    } else if (l0 + ct - nG < l1) {
      const int l = l0 + ct - nG;
#pragma unroll
      for (int c = 0; c < kRecChunks; ++c) rr[c] = ((const V4<T>*)d.lrec)[(size_t)c * d.L + l];
      my_rho = ((const T*)d.trho_l)[l];
      my_wset = d.wset[l];
    }
    ta = task_static<T>(d, t0 + cw < t1 ? load_slot(d, t0 + cw, lane) : none);
    tb = task_static<T>(d, t0 + cw + nwc < t1 ? load_slot(d, t0 + cw + nwc, lane) : none);
  }
  unsigned long long tp0 = 0, tp1 = 0;
  int it = 0;
  bool conv = false;
  for (it = 0; it < p.max_iter; ++it) {
    const int slot = it & 1;
    if (prof) tp0 = gtimer();
    // this parity's maxima were last read before the first barrier of the previous iteration
    if (threadIdx.x < 2) s_res[slot][threadIdx.x] = 0ull;
    // phase A: the instance's generators, then its branches
    if (RES) {
      if (ct < nG) {
        gen_compute(d, g0 + ct, rr[0], rr[1]);
      } else if (l0 + ct - nG < l1) {
        const int l = l0 + ct - nG;
        const V4<T>* Z = (const V4<T>*)d.Z;
        const V4<T>* LM = (const V4<T>*)d.LAM;
        line_compute(p, l, RRec<T>{rr}, Z[2 * l], Z[2 * l + 1], LM[2 * l], LM[2 * l + 1], ((const V4<T>*)d.U)[l],
                     my_rho, &my_wset);
      }
    } else {
      int u = ct;
      for (; u < nG; u += nth) gen_phase(p, g0 + u, 1.0f);
      for (int l = l0 + u - nG; l < l1; l += nth) line_phase(p, l, 1.0f);
    }
    if (prof) { tp1 = gtimer(); atomicAdd(&d.phase_ns[0], tp1 - tp0); }
    cluster_barrier();
    if (prof) { tp0 = gtimer(); atomicAdd(&d.phase_ns[1], tp0 - tp1); }
    // phase B: the instance's bus tasks, two at a time per warp, one in FP64 (warp-uniform loops)
    const ResDst dst = {&s_res[slot][0], nullptr, 1, slot, k};
    if (RES && sizeof(T) == 8 && nwc >= t1 - t0) {  // FP64, one task per warp
      bus_task_one(d, task_load<T, false>(d, ta, nullptr), dst);
    } else if (RES) {
      bus_task_pair(d, task_load<T, false>(d, ta, nullptr), task_load<T, false>(d, tb, nullptr), dst);
    } else if (sizeof(T) == 8) {
      for (int t = t0 + cw; t < t1; t += nwc)
        bus_task_one(d, task_load<T, false>(d, task_static<T>(d, load_slot(d, t, lane)), nullptr), dst);
    } else {
      for (int t = t0 + cw; t < t1; t += 2 * nwc) {
        const Slot sa = load_slot(d, t, lane);
        const Slot sb = t + nwc < t1 ? load_slot(d, t + nwc, lane) : none;
        bus_task_pair(d, task_load<T, false>(d, task_static<T>(d, sa), nullptr),
                      task_load<T, false>(d, task_static<T>(d, sb), nullptr), dst);
      }
    }
    for (int b = b0 + cw; b < b1; b += nwc) bus_task_big<T, false>(p, d.big[2 * b], d.big[2 * b + 1], dst, nullptr);
    if (prof) { tp1 = gtimer(); atomicAdd(&d.phase_ns[2], tp1 - tp0); }
    cluster_barrier();
    // residual test (Sec. IV-B) on the maxima of all the cluster's CTAs, taken alike by every CTA
    if (threadIdx.x < 32) {
      unsigned long long rm = 0ull, sm = 0ull;
      if (lane < cs) {
        rm = ld_cluster_u64(&s_res[slot][0], lane);
        sm = ld_cluster_u64(&s_res[slot][1], lane);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long r2 = __shfl_xor_sync(FULL, rm, o), s2 = __shfl_xor_sync(FULL, sm, o);
        rm = r2 > rm ? r2 : rm;
        sm = s2 > sm ? s2 : sm;
      }
      if (lane == 0) {
        s_rs[0] = __longlong_as_double((long long)rm);
        s_rs[1] = __longlong_as_double((long long)sm);
        s_stop = p.converged(rm, sm);
      }
    }
    __syncthreads();
    if (prof) atomicAdd(&d.phase_ns[3], gtimer() - tp1);
    if (s_stop) {
      conv = true;
      ++it;
      break;
    }
  }
  if (RES && sizeof(T) == 4 && ct >= nG && l0 + ct - nG < l1) d.wset[l0 + ct - nG] = (uint16_t)my_wset;
  if (rank == 0 && threadIdx.x == 0) {
    if (conv) d.admm_done[k] = 1;
    d.admm_iters[k] = it;
    d.admm_rs[k] = it > 0 ? s_rs[0] : 0.0;
    d.admm_rs[K + k] = it > 0 ? s_rs[1] : 0.0;
  }
  cluster_barrier();  // no CTA leaves while another may still read its shared memory
}

// ---------------------------------- cluster form with its state in shared memory
// Distributed shared memory addresses and stores (shared::cluster window).
__device__ __forceinline__ unsigned cluster_addr(const void* p, unsigned rank) {
  unsigned a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_addr(p)), "r"(rank));
  return a;
}
__device__ __forceinline__ void st_cluster(unsigned a, const V4<float>& v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void st_cluster(unsigned a, const V4<double>& v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a + 16), "d"(v.z), "d"(v.w) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(unsigned a, unsigned v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// One bus-task lane of the shared-memory form: its entry, the coupling's
// multiplier and old bus-side value (held from one iteration to the next),
// the penalty, and where its new bus-side value and multiplier go.
template <typename T>
struct DsmLane {
  TaskStatic<T> st;
  V4<T> lm, zo;
  T r;
  unsigned to;  // shared::cluster address of the owner's (z, lambda) pair
};

// Two tasks of one warp: x from this CTA's receive buffers (xa, xb), the bus
// update of eq. bus_kernel and the multiplier update of eq. multiplier, and
// the new (z, lambda) pushed to the generator's or branch's CTA.
template <typename T>
__device__ __forceinline__ void bus_pair_dsm(DsmLane<T>& a, DsmLane<T>& b, const V4<T>& xa, const V4<T>& xb,
                                             const ResDst& dst, V2<T>& zba, V2<T>& nua, V2<T>& zbb, V2<T>& nub) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool ea = a.st.s.bus >= 0, eb = b.st.s.bus >= 0;
  T Sa[6] = {0, 0, 0, 0, 0, 0}, Sb[6] = {0, 0, 0, 0, 0, 0};
  const T ira = ir_once(a.r), irb = ir_once(b.r);
  if (ea) entry_sums(a.st.s.code, xa, a.lm, a.r, ir_at(a.r, ira), Sa);
  if (eb) entry_sums(b.st.s.code, xb, b.lm, b.r, ir_at(b.r, irb), Sb);
  seg_scan2(a.st.s.bus, Sa, b.st.s.bus, Sb);
  T n1a = 0, n2a = 0, dwa = 0, dta = 0, n1b = 0, n2b = 0, dwb = 0, dtb = 0;
  if (a.st.last) {
    bus_values(a.st.br, a.st.isref, Sa, n1a, n2a, dwa, dta);
    zba = V2<T>{dwa, dta};
    nua = V2<T>{n1a, n2a};
  }
  if (b.st.last) {
    bus_values(b.st.br, b.st.isref, Sb, n1b, n2b, dwb, dtb);
    zbb = V2<T>{dwb, dtb};
    nub = V2<T>{n1b, n2b};
  }
  const unsigned ha = __ballot_sync(FULL, a.st.last) >> lane, hb = __ballot_sync(FULL, b.st.last) >> lane;
  const int srca = ha ? lane + __ffs(ha) - 1 : lane, srcb = hb ? lane + __ffs(hb) - 1 : lane;
  n1a = __shfl_sync(FULL, n1a, srca);
  n1b = __shfl_sync(FULL, n1b, srcb);
  n2a = __shfl_sync(FULL, n2a, srca);
  n2b = __shfl_sync(FULL, n2b, srcb);
  dwa = __shfl_sync(FULL, dwa, srca);
  dwb = __shfl_sync(FULL, dwb, srcb);
  dta = __shfl_sync(FULL, dta, srca);
  dtb = __shfl_sync(FULL, dtb, srcb);
  T rma = T(0), sma = T(0), rmb = T(0), smb = T(0);
  if (ea) {
    V4<T> zn, ln;
    entry_values(a.st.s.code, xa, a.lm, a.zo, a.r, ira, n1a, n2a, dwa, dta, rma, sma, zn, ln);
    st_cluster(a.to, zn);
    st_cluster(a.to + sizeof(V4<T>), ln);
    a.zo = zn;
    a.lm = ln;
    rma = nan_big(rma);
    sma = nan_big(sma);
  }
  if (eb) {
    V4<T> zn, ln;
    entry_values(b.st.s.code, xb, b.lm, b.zo, b.r, irb, n1b, n2b, dwb, dtb, rmb, smb, zn, ln);
    st_cluster(b.to, zn);
    st_cluster(b.to + sizeof(V4<T>), ln);
    b.zo = zn;
    b.lm = ln;
    rmb = nan_big(rmb);
    smb = nan_big(smb);
  }
  res_max2_pair(dst, rma, sma, a.st.s.inst, rmb, smb, b.st.s.inst);
}

// The resident cluster form with the exchanged state in shared memory: the
// cluster has a thread for every generator and branch of its instance and a
// warp for every two of its bus tasks, and the instance has no bus of more
// than 32 entries (checked by the launcher).  Each generator or branch keeps
// its coupling pairs (z, lambda) in its own CTA's shared memory, where the
// bus lanes push them; each bus lane keeps its coupling's x in its CTA's
// shared memory, where the generator or branch pushes it.  Within the sweep
// no state goes through global memory: it is read at the start and written
// back at the end.  Dynamic shared memory: (z, lambda) of both ends of every
// item [4 blockDim], x of this CTA's lanes for two tasks [2 blockDim], and
// the lanes' receive addresses per item end [2 blockDim].
template <typename T>
__global__ void __launch_bounds__(256, 1) k_sweep_cluster_dsm(SweepP<T> p) {
  const Dev& d = p.d;
  const unsigned FULL = 0xffffffffu;
  const int K = d.K;
  const int k = (int)cluster_index();
  const int cs = (int)cluster_nctarank(), rank = (int)cluster_ctarank();
  __shared__ unsigned long long s_res[2][2];  // this CTA's maxima (r, s), by iteration parity
  __shared__ double s_rs[2];
  __shared__ int s_stop;
  extern __shared__ __align__(16) unsigned char s_dyn_c[];
  const int bt = blockDim.x;
  V4<T>* s_zl = (V4<T>*)s_dyn_c;
  V4<T>* s_xin = s_zl + 4 * bt;
  unsigned* s_xcons = (unsigned*)(s_xin + 2 * bt);
  if (threadIdx.x < 4) (&s_res[0][0])[threadIdx.x] = 0ull;
  if (d.admm_done[k]) return;  // the whole cluster skips an instance that is not running
  const int nth = cs * bt, ct = rank * bt + threadIdx.x;
  const int lane = threadIdx.x & 31, cw = ct >> 5, nwc = nth >> 5;
  const int g0 = d.gen_off[k], nG = d.gen_off[k + 1] - g0, l0 = d.br_off[k], l1 = d.br_off[k + 1];
  const int t0 = d.task_off[k], t1 = d.task_off[k + 1];
  const Slot none = {-1, 0, -1};
  const bool prof = p.profile && blockIdx.x == 0 && threadIdx.x == 0;
  // this thread's generator or branch, its record, multipliers and (z, lambda)
  const int j = threadIdx.x;
  const bool is_gen = ct < nG, is_br = !is_gen && l0 + ct - nG < l1;
  const int g = g0 + ct, l = l0 + ct - nG;
  V4<T> rr[kRecChunks];
  T my_rho = T(0);
  unsigned my_wset = 0u;  // the box bounds held at the end of the branch's last solve
  V4<T> uu = {T(0), T(0), T(0), T(0)};
  const V4<T> zero4 = {T(0), T(0), T(0), T(0)};
  if (is_gen) {
    rr[0] = ((const V4<T>*)d.grec)[g];
    rr[1] = ((const V4<T>*)d.grec)[d.G + g];
    const V2<T> z = ((const V2<T>*)d.ZG)[g], lg = ((const V2<T>*)d.LG)[g];
    s_zl[4 * j] = V4<T>{z.x, z.y, T(0), T(0)};
    s_zl[4 * j + 1] = V4<T>{lg.x, lg.y, T(0), T(0)};
  } else if (is_br) {
#pragma unroll
    for (int c = 0; c < kRecChunks; ++c) rr[c] = ((const V4<T>*)d.lrec)[(size_t)c * d.L + l];
    my_rho = ((const T*)d.trho_l)[l];
    my_wset = d.wset[l];
    uu = ((const V4<T>*)d.U)[l];
    s_zl[4 * j] = ((const V4<T>*)d.Z)[2 * l];
    s_zl[4 * j + 1] = ((const V4<T>*)d.LAM)[2 * l];
    s_zl[4 * j + 2] = ((const V4<T>*)d.Z)[2 * l + 1];
    s_zl[4 * j + 3] = ((const V4<T>*)d.LAM)[2 * l + 1];
  }
  // this warp's two tasks; every lane with an entry tells the owner of its
  // coupling where to push x, and keeps where to push (z, lambda)
  DsmLane<T> A, B;
  auto lane_init = [&](DsmLane<T>& e, int t, int w) {
    e.st = task_static<T>(d, t < t1 ? load_slot(d, t, lane) : none);
    e.lm = e.zo = zero4;
    e.r = T(1);
    e.to = 0u;
    if (e.st.s.bus >= 0) {
      V4<T> x;
      entry_load(d, e.st.s.code, x, e.lm, e.zo, e.r);
      const int c = e.st.s.code;
      const int uo = c < 0 ? (-c - 1) - g0 : nG + (c >> 1) - l0;
      const int side = c < 0 ? 0 : (c & 1);
      const unsigned orank = (unsigned)(uo / bt), oj = (unsigned)(uo % bt);
      e.to = cluster_addr(&s_zl[4 * oj + 2 * side], orank);
      st_cluster_u32(cluster_addr(&s_xcons[2 * oj + side], orank), cluster_addr(&s_xin[w * bt + threadIdx.x], rank));
    }
  };
  cluster_barrier();  // every CTA has started before any distributed shared memory access
  lane_init(A, t0 + cw, 0);
  lane_init(B, t0 + cw + nwc, 1);
  cluster_barrier();  // the receive addresses are in place
  unsigned xc0 = 0u, xc1 = 0u;
  if (is_gen || is_br) {
    xc0 = s_xcons[2 * j];
    xc1 = s_xcons[2 * j + 1];
  }
  V4<T> x0 = zero4, x1 = zero4;
  V2<T> xg = {T(0), T(0)}, zba = {T(0), T(0)}, nua = zba, zbb = zba, nub = zba;
  unsigned long long tp0 = 0, tp1 = 0;
  int it = 0;
  bool conv = false;
  for (it = 0; it < p.max_iter; ++it) {
    const int slot = it & 1;
    if (prof) tp0 = gtimer();
    if (threadIdx.x < 2) s_res[slot][threadIdx.x] = 0ull;
    // phase A
    if (is_gen) {
      const V4<T> z = s_zl[4 * j], lm = s_zl[4 * j + 1];
      xg = gen_value(rr[0], rr[1], V2<T>{z.x, z.y}, V2<T>{lm.x, lm.y});
      st_cluster(xc0, V4<T>{xg.x, xg.y, T(0), T(0)});
    } else if (is_br) {
      line_compute_to(p, l, RRec<T>{rr}, s_zl[4 * j], s_zl[4 * j + 2], s_zl[4 * j + 1], s_zl[4 * j + 3], uu, my_rho,
                      [&](const V4<T>& o0, const V4<T>& o1, const V4<T>& ou) {
                        st_cluster(xc0, o0);
                        st_cluster(xc1, o1);
                        x0 = o0;
                        x1 = o1;
                        uu = ou;
                      },
                      &my_wset);
    }
    if (prof) { tp1 = gtimer(); atomicAdd(&d.phase_ns[0], tp1 - tp0); }
    cluster_barrier();
    if (prof) { tp0 = gtimer(); atomicAdd(&d.phase_ns[1], tp0 - tp1); }
    // phase B
    const ResDst dst = {&s_res[slot][0], nullptr, 1, slot, k};
    bus_pair_dsm(A, B, s_xin[threadIdx.x], s_xin[bt + threadIdx.x], dst, zba, nua, zbb, nub);
    if (prof) { tp1 = gtimer(); atomicAdd(&d.phase_ns[2], tp1 - tp0); }
    cluster_barrier();
    // residual test (Sec. IV-B) on the maxima of all the cluster's CTAs, taken alike by every CTA
    if (threadIdx.x < 32) {
      unsigned long long rm = 0ull, sm = 0ull;
      if (lane < cs) {
        rm = ld_cluster_u64(&s_res[slot][0], lane);
        sm = ld_cluster_u64(&s_res[slot][1], lane);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long r2 = __shfl_xor_sync(FULL, rm, o), s2 = __shfl_xor_sync(FULL, sm, o);
        rm = r2 > rm ? r2 : rm;
        sm = s2 > sm ? s2 : sm;
      }
      if (lane == 0) {
        s_rs[0] = __longlong_as_double((long long)rm);
        s_rs[1] = __longlong_as_double((long long)sm);
        s_stop = p.converged(rm, sm);
      }
    }
    __syncthreads();
    if (prof) atomicAdd(&d.phase_ns[3], gtimer() - tp1);
    if (s_stop) {
      conv = true;
      ++it;
      break;
    }
  }
  // the state back to global memory
  if (it > 0) {
    if (is_gen) ((V2<T>*)d.XG)[g] = xg;
    if (is_br) {
      ((V4<T>*)d.X)[2 * l] = x0;
      ((V4<T>*)d.X)[2 * l + 1] = x1;
      ((V4<T>*)d.U)[l] = uu;
      d.wset[l] = (uint16_t)my_wset;
    }
    if (A.st.s.bus >= 0) entry_store(d, A.st.s.code, A.zo, A.lm);
    if (B.st.s.bus >= 0) entry_store(d, B.st.s.code, B.zo, B.lm);
    if (A.st.last) {
      ((V2<T>*)d.ZB)[A.st.s.bus] = zba;
      ((V2<T>*)d.NU)[A.st.s.bus] = nua;
    }
    if (B.st.last) {
      ((V2<T>*)d.ZB)[B.st.s.bus] = zbb;
      ((V2<T>*)d.NU)[B.st.s.bus] = nub;
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    if (conv) d.admm_done[k] = 1;
    d.admm_iters[k] = it;
    d.admm_rs[k] = it > 0 ? s_rs[0] : 0.0;
    d.admm_rs[K + k] = it > 0 ? s_rs[1] : 0.0;
  }
  cluster_barrier();  // no CTA leaves while another may still read its shared memory
}

// ADMM state reset: d = 0, z = 0 (and lambda = 0 unless kept); instances that
// are no longer running keep their state
template <typename T>
__global__ void k_admm_reset(Dev d, int keep_lambda, int pass) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  V4<T> z4 = {T(0), T(0), T(0), T(0)};
  V2<T> z2 = {T(0), T(0)};
  if (n < 2 * d.L) {
    int k = d.br_inst[n >> 1];
    if (live(d.ctl[k], pass)) {
      ((V4<T>*)d.X)[n] = z4;
      ((V4<T>*)d.Z)[n] = z4;
      if (!keep_lambda) ((V4<T>*)d.LAM)[n] = z4;
      if (!keep_lambda && (n & 1) == 0) ((V4<T>*)d.U)[n >> 1] = z4;
    }
  }
  if (n < d.G) {
    int k = d.gen_inst[n];
    if (live(d.ctl[k], pass)) {
      ((V2<T>*)d.XG)[n] = z2;
      ((V2<T>*)d.ZG)[n] = z2;
      if (!keep_lambda) ((V2<T>*)d.LG)[n] = z2;
    }
  }
  if (n < d.B) {
    int k = d.bus_inst[n];
    if (live(d.ctl[k], pass)) {
      ((V2<T>*)d.ZB)[n] = z2;
      ((V2<T>*)d.NU)[n] = z2;
    }
  }
  if (n < d.K) {
    d.admm_done[n] = live(d.ctl[n], pass) ? 0 : 1;
    d.admm_iters[n] = 0;
  }
}

__global__ void k_rho_fac_reset(Dev d) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < d.K) d.rho_fac[k] = 1.0;
}

// carry the penalties adapted by residual balancing into the FP64 master copies
__global__ void k_commit_rho(Dev d) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < d.L) d.rho_l[n] *= d.rho_fac[d.br_inst[n]];
  if (n < d.G) d.rho_g[n] *= d.rho_fac[d.gen_inst[n]];
}

static void launch_rho_fac_reset(Ctx& c) {
  k_rho_fac_reset<<<nblk(c.d.K, 256), 256, 0, c.stream>>>(c.d);
  c.launches++;
}

void launch_commit_rho(Ctx& c) {
  long m = c.d.L > c.d.G ? c.d.L : c.d.G;
  k_commit_rho<<<nblk(m, 256), 256, 0, c.stream>>>(c.d);
  c.launches++;
}

// dynamic shared memory of k_sweep<T>: flags and factors of K instances, and
// for the FP32 sweep two branch-tile stages plus their mbarriers
template <typename T>
static size_t sweep_smem(int K, int threads, int stages) {
  size_t b = (sizeof(int) + sizeof(float)) * (size_t)K + (K <= kSmemResMax ? 16 * (size_t)K : 0);
  if (sizeof(T) == 4 && stages > 0)
    b = ((b + 127) & ~(size_t)127) + (size_t)stages * kTileV4 * threads * sizeof(V4<T>) + 16 + 128;
  return b;
}

// Launch shape of k_sweep<T>.  The resident form (sweep_stages 3) is used when
// residual balancing is off and a co-resident grid gives every generator and
// branch a thread of its own and every warp at most two bus tasks; otherwise
// (and for sweep_stages 0-2) the streaming form, with enough CTAs for one pass
// over the larger of the two phases, capped at the co-resident maximum.
struct SweepShape {
  void* fn;
  int blocks;
  size_t smem;
};

template <typename T>
static acopf_status sweep_shape(Ctx& c, const SweepP<T>& p, SweepShape& sh) {
  const Dev& d = c.d;
  const int threads = c.block_threads;
  if (c.sweep_stages == 3 && p.rb_period == 0) {
    const size_t smem = sweep_smem<T>(d.K, threads, 0);
    cudaFuncSetAttribute(k_sweep<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<T, true>, threads, smem);
    if (c.ctas_per_sm > 0 && c.ctas_per_sm < per_sm) per_sm = c.ctas_per_sm;
    const long cap = (long)per_sm * c.num_sms;
    const long wpb = threads / 32;
    long need = ((long)d.G + d.L + threads - 1) / threads;
    const long need_b = ((long)d.NT + 2 * wpb - 1) / (2 * wpb);
    // the FP64 sweep gives each warp one bus task when the grid still fits
    // (two interleaved FP64 tasks take about twice as long as one)
    const long need_b1 = ((long)d.NT + wpb - 1) / wpb;
    if (sizeof(T) == 8 && need_b1 > need && need_b1 <= cap) need = need_b1;
    if (need_b > need) need = need_b;
    if (need < 1) need = 1;
    if (per_sm >= 1 && need <= cap) {
      sh = {(void*)k_sweep<T, true>, (int)need, smem};
      return ACOPF_OK;
    }
  }
  const size_t smem = sweep_smem<T>(d.K, threads, p.stages);
  cudaFuncSetAttribute(k_sweep<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<T, false>, threads, smem);
  if (per_sm < 1) {
    c.last_error = "sweep: the kernel does not fit on a multiprocessor";
    return ACOPF_ECUDA;
  }
  if (c.ctas_per_sm > 0 && c.ctas_per_sm < per_sm) per_sm = c.ctas_per_sm;
  long work = d.G + d.L;
  if (d.B > work) work = d.B;
  long need = (work + threads - 1) / threads;
  long maxb = (long)per_sm * c.num_sms;
  int blocks = (int)(need < maxb ? need : maxb);
  if (blocks < 1) blocks = 1;
  sh = {(void*)k_sweep<T, false>, blocks, smem};
  return ACOPF_OK;
}

// Cluster size of sweep_stages 4: enough CTAs for one thread per generator or
// branch of the largest instance, at most 16, fewer when a cluster of that
// size cannot be resident.  The FP64 sweep takes one bus task per warp when a
// resident cluster of at most 16 CTAs allows it (as in sweep_shape).
template <typename T>
static int cluster_size(Ctx& c, int threads, cudaLaunchConfig_t& cfg, cudaLaunchAttribute& attr, bool& res) {
  long items = 1, tasks = 0;
  for (int k = 0; k < c.d.K; ++k) {
    long n = (long)(c.h_gen_off[k + 1] - c.h_gen_off[k]) + (c.h_br_off[k + 1] - c.h_br_off[k]);
    items = n > items ? n : items;
  }
  const std::vector<int>& toff = c.h_task_off;
  for (int k = 0; k < c.d.K; ++k) tasks = toff[k + 1] - toff[k] > tasks ? toff[k + 1] - toff[k] : tasks;
  int cs = (int)((items + threads - 1) / threads);
  const long wpb = threads / 32;
  const int cs_b = (int)((tasks + 2 * wpb - 1) / (2 * wpb));
  if (cs_b > cs) cs = cs_b;
  if (cs < 1) cs = 1;
  res = cs <= 16;
  if (cs > 16) cs = 16;
  void* fn = res ? (void*)k_sweep_cluster<T, true> : (void*)k_sweep_cluster<T, false>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  const long cs_b1 = (tasks + wpb - 1) / wpb;
  if (sizeof(T) == 8 && res && cs_b1 > cs && cs_b1 <= 16) {
    cfg.gridDim = dim3((unsigned)cs_b1);
    attr.val.clusterDim.x = (unsigned)cs_b1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n >= 1) return (int)cs_b1;
    cudaGetLastError();
  }
  for (; cs > 1; --cs) {
    cfg.gridDim = dim3(cs);
    attr.val.clusterDim.x = cs;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n >= 1) break;
    cudaGetLastError();
    res = false;  // a smaller cluster no longer covers every component
    fn = (void*)k_sweep_cluster<T, false>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  if (res && (long)cs * threads < items) res = false;
  return cs;
}

template <typename T>
static acopf_status run_sweep_cluster(Ctx& c, const SweepP<T>& p) {
  const int threads = c.block_threads;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = c.stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const size_t dsm_smem = (size_t)threads * (6 * sizeof(V4<T>) + 2 * sizeof(unsigned));
  if (c.cluster_threads != threads) {
    bool res = false;
    c.cluster_cs = cluster_size<T>(c, threads, cfg, attr[0], res);
    c.cluster_res = res;
    c.cluster_threads = threads;
    // the shared-memory form: FP32, resident, and no bus of more than 32 entries
    bool dsm = res && sizeof(T) == 4;
    for (int k = 0; dsm && k < c.d.K; ++k) dsm = c.h_big_off[k + 1] == c.h_big_off[k];
    if constexpr (sizeof(T) == 4) if (dsm) {
      cudaFuncSetAttribute(k_sweep_cluster_dsm<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      cudaFuncSetAttribute(k_sweep_cluster_dsm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm_smem);
      cfg.gridDim = dim3(c.cluster_cs);
      attr[0].val.clusterDim.x = c.cluster_cs;
      cfg.dynamicSmemBytes = dsm_smem;
      int n = 0;
      dsm = cudaOccupancyMaxActiveClusters(&n, (void*)k_sweep_cluster_dsm<T>, &cfg) == cudaSuccess && n >= 1;
      cudaGetLastError();
      cfg.dynamicSmemBytes = 0;
    }
    c.cluster_dsm = dsm;
  }
  const int cs = c.cluster_cs;
  attr[0].val.clusterDim.x = cs;
  if (c.cluster_dsm) cfg.dynamicSmemBytes = dsm_smem;
  if (!c.capturing) cudaMemsetAsync(c.d.err, 0, sizeof(int), c.stream);
  cfg.gridDim = dim3((unsigned)(c.d.K * cs));
  const bool prof = c.profiling && !c.capturing;
  if (prof) cudaEventRecord(c.ev0, c.stream);
  cudaError_t e;
  if constexpr (sizeof(T) == 4) {
    e = c.cluster_dsm   ? cudaLaunchKernelEx(&cfg, k_sweep_cluster_dsm<T>, p)
        : c.cluster_res ? cudaLaunchKernelEx(&cfg, k_sweep_cluster<T, true>, p)
                        : cudaLaunchKernelEx(&cfg, k_sweep_cluster<T, false>, p);
  } else {
    e = c.cluster_res ? cudaLaunchKernelEx(&cfg, k_sweep_cluster<T, true>, p)
                      : cudaLaunchKernelEx(&cfg, k_sweep_cluster<T, false>, p);
  }
  c.launches++;
  if (e != cudaSuccess) {
    c.last_error = std::string("sweep launch (clusters): ") + cudaGetErrorString(e);
    return ACOPF_ECUDA;
  }
  if (prof) {
    cudaEventRecord(c.ev1, c.stream);
    cudaEventSynchronize(c.ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.ev0, c.ev1);
    c.prof_ms += ms;
    c.prof_sweeps += 1;
    int mx = 0;
    std::vector<int> it(c.d.K);
    cudaMemcpy(it.data(), c.d.admm_iters, sizeof(int) * c.d.K, cudaMemcpyDeviceToHost);
    for (int k = 0; k < c.d.K; ++k) mx = it[k] > mx ? it[k] : mx;
    c.prof_iters += mx;
  }
  return ACOPF_OK;
}

template <typename T>
static acopf_status run_sweep(Ctx& c, const admm_options& o, int fixed_iters) {
  Dev& d = c.d;
  SweepP<T> p;
  p.d = d;
  p.max_iter = fixed_iters > 0 ? fixed_iters : o.max_iter;
  p.fixed = fixed_iters > 0;
  p.eps = o.eps;
  p.eps_dual = o.eps_dual > 0 ? o.eps_dual : o.eps;
  p.beta_scale = (T)o.alm_beta;
  p.alm_tol = (T)fmax(o.alm_tol, (double)Tol<T>::alm);
  p.alm_outer = o.alm_max_outer;
  p.newton_max = o.newton_max;
  p.spin_limit = o.spin_limit;
  p.rb_period = o.rb_period;
  p.rb_mu = o.rb_mu;
  p.rb_tau = o.rb_tau;
  p.stages = c.sweep_stages >= 3 ? 0 : c.sweep_stages;
  p.profile = c.profiling ? 1 : 0;
  p.smem_res = d.K <= kSmemResMax;
  p.line_exact = o.line_solver == 0;
  set_stop_test(p);
  const int threads = c.block_threads;
  if (c.sweep_stages == 4 && p.rb_period == 0) return run_sweep_cluster(c, p);
  SweepShape sh;
  acopf_status st = sweep_shape(c, p, sh);
  if (st) return st;
  cudaMemsetAsync(d.bar, 0, 2 * sizeof(unsigned), c.stream);
  // inside a captured SQP iteration the error flag is not cleared: a barrier
  // time-out stays visible to the host and makes every later sweep return at
  // its first barrier
  if (!c.capturing) cudaMemsetAsync(d.err, 0, sizeof(int), c.stream);
  cudaMemsetAsync(d.res_slots, 0, sizeof(unsigned long long) * 4 * d.K, c.stream);
  launch_rho_fac_reset(c);
  void* args[] = {&p};
  const bool prof = c.profiling && !c.capturing;
  if (prof) cudaEventRecord(c.ev0, c.stream);
  cudaError_t e = cudaLaunchCooperativeKernel(sh.fn, dim3(sh.blocks), dim3(threads), args, sh.smem, c.stream);
  c.launches++;
  if (e != cudaSuccess) {
    c.last_error = std::string("sweep launch: ") + cudaGetErrorString(e);
    return ACOPF_ECUDA;
  }
  if (prof) {
    cudaEventRecord(c.ev1, c.stream);
    cudaEventSynchronize(c.ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.ev0, c.ev1);
    c.prof_ms += ms;
    c.prof_sweeps += 1;
    int mx = 0;
    std::vector<int> it(d.K);
    cudaMemcpy(it.data(), d.admm_iters, sizeof(int) * d.K, cudaMemcpyDeviceToHost);
    for (int k = 0; k < d.K; ++k) mx = it[k] > mx ? it[k] : mx;
    c.prof_iters += mx;
  }
  return ACOPF_OK;
}

acopf_status launch_sweep(Ctx& c, const admm_options& o, int fixed_iters) {
  return c.precision == ACOPF_MIXED ? run_sweep<float>(c, o, fixed_iters) : run_sweep<double>(c, o, fixed_iters);
}

void launch_admm_reset(Ctx& c, int keep_lambda, int pass) {
  Dev& d = c.d;
  long m = 2L * d.L;
  if (d.G > m) m = d.G;
  if (d.B > m) m = d.B;
  if (d.K > m) m = d.K;
  if (c.precision == ACOPF_MIXED)
    k_admm_reset<float><<<nblk(m, 256), 256, 0, c.stream>>>(d, keep_lambda, pass);
  else
    k_admm_reset<double><<<nblk(m, 256), 256, 0, c.stream>>>(d, keep_lambda, pass);
  c.launches++;
}

// ----------------------------------------------------------------------------
// admm_iterate_static: the sweep of admm_iterate with the kernel's scratch
// (device-wide barrier counters, error flag, residual slots, per-instance
// finished flags and penalty factors) taken from a fixed device array instead
// of memory the handle allocated.  It allocates nothing, for callers that may
// not allocate device memory while they run (a pre-sized memory arena, a
// real-time loop that cannot afford cudaMalloc's implicit synchronisation, a
// thread without access to the application's allocator).
// ----------------------------------------------------------------------------
namespace {

constexpr int kStaticMaxInstances = ACOPF_STATIC_MAX_INSTANCES;
constexpr size_t kStaticHeader = 256;  // barrier count + generation, error flag (padded)
constexpr size_t kStaticSlots = sizeof(unsigned long long) * 4 * kStaticMaxInstances;
constexpr size_t kStaticDone = sizeof(int) * kStaticMaxInstances;
constexpr size_t kStaticFac = sizeof(double) * kStaticMaxInstances;
constexpr size_t kStaticBytes = kStaticHeader + kStaticSlots + kStaticDone + kStaticFac;

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_sweep_scratch[kStaticBytes];

// Device address of g_sweep_scratch per device ordinal (host-side copies of the
// symbol are only stand-ins, not device addresses).  Looked up once per device
// and published atomically, so concurrent first calls on one device are safe
// (both store the same address).  The address belongs to the device's primary
// context: it assumes that context lives for the whole process (a
// cudaDeviceReset would invalidate it).
static std::atomic<void*> g_scratch_addr[64];

// The finished flags start from the handle's own (handle_done): an instance
// whose ADMM residual test passed in the last admm_solve_qp is skipped here
// exactly as admm_iterate skips it.
__global__ void k_static_init(Dev d, const int* handle_done) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < d.K) {
    d.admm_done[k] = handle_done[k];
    d.rho_fac[k] = 1.0;
  }
}

template <typename T>
acopf_status run_sweep_static(Ctx& c, const admm_options& o, int n, double* rs, int* iters, unsigned char* base) {
  Dev d = c.d;
  const int* handle_done = c.d.admm_done;
  d.bar = (unsigned*)base;
  d.err = (int*)(base + 2 * sizeof(unsigned));
  d.res_slots = (unsigned long long*)(base + kStaticHeader);
  d.admm_done = (int*)(base + kStaticHeader + kStaticSlots);
  d.rho_fac = (double*)(base + kStaticHeader + kStaticSlots + kStaticDone);
  d.admm_rs = rs;
  d.admm_iters = iters;
  SweepP<T> p;
  p.d = d;
  p.max_iter = n;
  p.fixed = 1;
  p.eps = o.eps;
  p.eps_dual = o.eps_dual > 0 ? o.eps_dual : o.eps;
  p.beta_scale = (T)o.alm_beta;
  p.alm_tol = (T)fmax(o.alm_tol, (double)Tol<T>::alm);
  p.alm_outer = o.alm_max_outer;
  p.newton_max = o.newton_max;
  p.spin_limit = o.spin_limit;
  p.rb_period = o.rb_period;
  p.rb_mu = o.rb_mu;
  p.rb_tau = o.rb_tau;
  p.stages = c.sweep_stages >= 3 ? 0 : c.sweep_stages;
  p.profile = 0;  // not timed: acopf_profile covers the handle's own sweeps only
  p.smem_res = d.K <= kSmemResMax;
  p.line_exact = o.line_solver == 0;
  set_stop_test(p);
  const int threads = c.block_threads;
  SweepShape sh;
  acopf_status st = sweep_shape(c, p, sh);
  if (st) return st;
  // what must start at zero: barrier counters, error flag, residual slots
  cudaMemsetAsync(base, 0, kStaticHeader + sizeof(unsigned long long) * 4 * d.K, c.stream);
  k_static_init<<<nblk(d.K, 256), 256, 0, c.stream>>>(d, handle_done);
  void* args[] = {&p};
  cudaError_t e = cudaLaunchCooperativeKernel(sh.fn, dim3(sh.blocks), dim3(threads), args, sh.smem, c.stream);
  c.launches += 2;
  if (e != cudaSuccess) {
    c.last_error = std::string("admm_iterate_static launch: ") + cudaGetErrorString(e);
    return ACOPF_ECUDA;
  }
  // the handle's own residual record follows this sweep too (acopf_get_residuals
  // reads it); device-to-device copies into memory the handle already owns
  cudaMemcpyAsync(c.d.admm_rs, rs, sizeof(double) * 2 * d.K, cudaMemcpyDeviceToDevice, c.stream);
  cudaMemcpyAsync(c.d.admm_iters, iters, sizeof(int) * d.K, cudaMemcpyDeviceToDevice, c.stream);
  if (o.rb_period > 0) {
    long m = d.L > d.G ? d.L : d.G;
    k_commit_rho<<<nblk(m, 256), 256, 0, c.stream>>>(d);
    c.launches++;
  }
  return ACOPF_OK;
}

}  // namespace

}  // namespace acopf

extern "C" acopf_status admm_iterate_static(acopf_handle h, int32_t n, const admm_options* ao, double* rs,
                                            int32_t* iters) {
  using namespace acopf;
  Ctx* c = (Ctx*)h;
  if (!c || n < 1 || !ao || !rs || !iters) {
    if (c) c->last_error = "admm_iterate_static: handle, n >= 1, options and the rs/iters buffers are required";
    return ACOPF_EINVAL;
  }
  const admm_options& o = *ao;
  if (!(o.rho > 0) || !(o.eps >= 0) || !(o.eps_dual >= 0) || o.alm_max_outer < 1 || o.newton_max < 1 ||
      !(o.alm_beta > 0) || o.spin_limit < 1 || o.rb_period < 0 ||
      (o.rb_period > 0 && (!(o.rb_mu > 1) || !(o.rb_tau > 1))) || o.line_solver < 0 || o.line_solver > 1) {
    c->last_error = "admm_iterate_static: admm options out of range";
    return ACOPF_EINVAL;
  }
  if (c->d.K > kStaticMaxInstances) {
    c->last_error = "admm_iterate_static: the handle has " + std::to_string(c->d.K) +
                    " instances; the fixed scratch array holds at most " + std::to_string(kStaticMaxInstances);
    return ACOPF_EINVAL;
  }
  if (!c->qp_built) {
    c->last_error = "admm_iterate_static: no QP has been built";
    return ACOPF_ENOTREADY;
  }
  if (c->device < 0 || c->device >= 64) {
    c->last_error = "admm_iterate_static: device ordinal out of range";
    return ACOPF_EINVAL;
  }
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) {
    c->last_error = std::string("admm_iterate_static: cudaSetDevice: ") + cudaGetErrorString(e);
    return ACOPF_ECUDA;
  }
  // one-time set-up per device, with that device current
  void* ptr = g_scratch_addr[c->device].load(std::memory_order_acquire);
  if (!ptr) {
    e = cudaGetSymbolAddress(&ptr, g_sweep_scratch);
    if (e != cudaSuccess || !ptr) {
      c->last_error = std::string("admm_iterate_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return ACOPF_ECUDA;
    }
    g_scratch_addr[c->device].store(ptr, std::memory_order_release);
  }
  unsigned char* base = (unsigned char*)ptr;
  acopf_status s = c->precision == ACOPF_MIXED ? run_sweep_static<float>(*c, o, n, rs, iters, base)
                                               : run_sweep_static<double>(*c, o, n, rs, iters, base);
  if (s) return s;
  launch_step(*c);
  int err = 0;
  e = cudaMemcpyAsync(&err, base + 2 * sizeof(unsigned), sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->last_error = std::string("admm_iterate_static: ") + cudaGetErrorString(e);
    return ACOPF_ECUDA;
  }
  if (err) {
    c->last_error = "admm_iterate_static: a CTA timed out at a device-wide barrier";
    return ACOPF_ETIMEOUT;
  }
  c->have_step = true;
  return ACOPF_OK;
}
