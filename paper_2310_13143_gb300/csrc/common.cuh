// Internal layout of the GB300 SQP-ADMM solver (not part of the C ABI).
//
// All instances of a handle are concatenated: buses, branches and generators
// carry global indices, and per-instance segments are given by *_off arrays.
// Generators are stored sorted by bus (gen_ptr is the CSR row pointer of
// "generators at bus i"); the user's generator order is restored on output.
//
// ADMM state is end-major: each branch has two ends (from = 0, to = 1) and
// each end carries the four couplings (p, q, w, theta) of eq. cpl as one
// 4-vector, so a bus touches one 16/32-byte vector per incident end and a
// branch reads its 8 couplings as two contiguous vectors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/acopf.h"

namespace acopf {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kBig = 1e30;

// per-branch sweep record: 56 values in 14 chunks of 4, chunk c of branch l
// stored at rec[c * L + l] (coalesced 16/32-byte loads across a warp)
//   0-9   Q (packed upper triangle q00 q01 q02 q03 q11 q12 q13 q22 q23 q33)
//   10-25 F (rows p_ij q_ij p_ji q_ji, columns dbar)
//   26-29 f0        30-33 c0 = gH + rho F^T f0
//   34-37 lo        38-41 hi
//   42-49 line-limit rows, normalised to unit 2-norm
//   50-51 their right-hand sides (normalised)
//   52 alo  53 ahi  (angle-difference bounds on d_thi - d_thj; >= 1e29: none)
//   54-55 2-norms of the two line-limit rows (0: row disabled)
constexpr int kRecChunks = 14;
constexpr int kHistW = 14;  // values per row of the SQP history (acopf_get_history)

template <typename T>
struct alignas(4 * sizeof(T)) V4 {
  T x, y, z, w;
};
template <typename T>
struct alignas(2 * sizeof(T)) V2 {
  T x, y;
};

struct InstCtl {            // per-instance SQP control, device resident
  double delta, mu, tol, step_tol, delta_max, delta_min;
  double obj, primal, dual, r_inf, s_inf;
  double ared, pred, dnorm;
  double rho, eps;
  int32_t sqp_iter, admm_iter_total, admm_iter_last, accepted;
  int32_t result;           // acopf_result
  int32_t accept_last;
  int32_t admm_done;        // 1 once the ADMM residual test passed in the last sweep
  int32_t merit_linear;     // 1: h of the merit function includes the linear constraints
  // second-order correction and feasibility restoration
  int32_t soc_on, restore_on;  // options
  int32_t soc_active;       // this iteration's step was rejected and is being corrected
  int32_t soc_flag;         // last iteration: 0 no correction, 1 corrected step rejected, 2 accepted
  int32_t restoring;        // 1 in the restoration phase (objective weight 0)
  int32_t since_switch;     // iterations since the last change of phase
  double fscale;            // objective weight of QP and merit function (1, or 0 while restoring)
  double delta0;            // initial radius (restored at every change of phase)
  double phx_saved, pred_saved, dn_saved, ared_saved;  // the rejected step's merit data
  double primal_ring[5];    // primal infeasibility of the last five iterations
};

// instance k takes part in a pass of one SQP iteration: every running instance
// in the main pass (0); in the correction pass (1) only those whose step was
// rejected and is being corrected (second-order correction)
__host__ __device__ inline bool live(const InstCtl& c, int pass) {
  return c.result == ACOPF_RUNNING && (pass == 0 || c.soc_active);
}

// raw device pointers shared by all kernels
struct Dev {
  int K, B, L, G;
  int *bus_off, *br_off, *gen_off;
  int *bus_inst, *br_inst, *gen_inst;
  // buses
  double *pd, *qd, *gs, *bs, *wmin, *wmax;
  int* isref;
  int *end_ptr, *end_idx, *gen_ptr;
  // bus update work list: entry q (bus order: the bus's generators, then its
  // branch ends) is ent[q] = -(g + 1) for generator g or the end id 2 l + side,
  // ebus[q] its bus.  Warp tasks of consecutive whole buses with at most 32
  // entries are stored padded: slot 32 t + j holds lane j's entry (pent), bus
  // (pbus, -1: empty) and instance (pinst).  A bus with more than 32 entries
  // is a big task: entries [big[2 b], big[2 b + 1]) of ent/ebus.
  int *ent, *ebus;
  int *pent, *pbus, *pinst;
  int* big;
  int E, NT, NBIG;
  // per branch: the box bounds held at the end of its last FP32 line solve in
  // a resident sweep form (bit 8: set held; bits 0-3 held, 4-7 at the upper
  // bound), the start of the next launch's first solve; cleared when the QP
  // is built.  (The streaming forms start each solve from the clamped point:
  // the extra load and store cost more there than the saved factorisations.)
  uint16_t* wset;
  // first warp task and first big task of every instance (K + 1 each); no
  // task holds buses of two instances
  int *task_off, *big_off;
  // branches
  int *f, *t;
  double* Y;        // [8][L]: gii bii gij bij gji bji gjj bjj
  double* s2;       // rate^2, or -1 (no limit)
  double *angmin, *angmax;
  // generators (sorted by bus)
  int* gbus;
  double *pmin, *pmax, *qmin, *qmax, *cq, *cl, *cc;  // cost = cq p^2 + cl p + cc (p in p.u.)
  // iterate (FP64)
  double *pg, *qg, *w, *th, *wr, *wi;
  double* pi;       // [4][L]
  // step (FP64) and recovered multipliers
  double *dpg, *dqg, *dw, *dth, *dwr, *dwi;
  double* pi_new;   // [4][L]
  // QP data needed in FP64 after the sweep
  double* flow;     // [4][L]
  double *aR, *aI;  // [4][L]
  double *bR, *bI;  // [L]
  double *gd1, *gd2;
  double* rho_l;    // [L] per-branch penalty (FP64 master copy)
  double* rho_g;    // [G]
  // sweep data and state in the sweep precision (float or double)
  void* lrec;       // [14][L] chunks
  void* grec;       // [2][G] chunks: (gd1, gd2, lp, up), (lq, uq, rho, 0)
  void* brec;       // [B] chunk: (pdk, qdk, gs, bs)
  void* trho_l;     // [L]
  void *X, *Z, *LAM;  // V4 [2L]
  void* U;            // V4 [L]
  void *XG, *ZG, *LG; // V2 [G]
  void *ZB, *NU;      // V2 [B]
  // sweep control
  unsigned long long* res_slots; // [2 slots][2 (r,s)][K]
  int* admm_done;     // [K]
  int* admm_iters;    // [K]
  double* admm_rs;    // [2][K]
  unsigned int* bar;  // [2]: count, generation
  int* err;           // [1]
  // merit / KKT scratch
  double* flow_xd;    // [4][L]
  double* tbr;        // [8][L]
  double* tbus;       // [4][B]
  double* tgen;       // [8][G]
  double* dend;       // [2][2L] per-end gradient contributions (w, theta)
  double* red;        // [16][K] per-instance reductions
  double* hist;       // [K][ACOPF_HIST_MAX][kHistW] SQP history
  double* rho_fac;    // [K] penalty factor applied by residual balancing in the last sweep
  unsigned long long* phase_ns;  // [4] (profiling) CTA 0's time in phase A, first wait, phase B, second wait + test
  InstCtl* ctl;       // [K]
  int* n_running;     // [1]
  // export buffers (allocated on demand)
  double *xbr, *xgen, *xbus;
};

// host-side handle
struct Ctx {
  Dev d{};
  int precision = ACOPF_FP64;
  int use_angle = 1;
  int device = 0;
  int block_threads = 256;
  int ctas_per_sm = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  std::string last_error;
  int64_t launches = 0;
  bool qp_built = false;
  bool have_step = false;
  // host copies of the segment offsets and the generator permutation
  int* h_bus_off = nullptr;
  int* h_br_off = nullptr;
  int* h_gen_off = nullptr;
  int* h_gen_perm = nullptr;   // internal index -> user index (global)
  int* h_gen_iperm = nullptr;  // user index -> internal index
  // every device block the handle owns, with the handle field that points to
  // it and the release function of the allocator that made it (null: cudaFree)
  struct Block {
    void* p;
    size_t bytes;
    void** slot;
    void (*release)(void*, void*);
    void* rctx;
  };
  Block blocks[192];
  int nblocks = 0;
  // the caller's device allocator (acopf_set_allocator); null: cudaMalloc / cudaFree
  void* (*ualloc)(size_t, void*) = nullptr;
  void (*ufree)(void*, void*) = nullptr;
  void* uctx = nullptr;
  // sweep timing (acopf_profile)
  bool profiling = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double prof_ms = 0.0;
  int64_t prof_sweeps = 0, prof_iters = 0;
  int sweep_stages = 0;  // record access of the sweep (acopf_tune), 4: one thread-block cluster per instance
  int cluster_cs = 1;         // cluster size of sweep_stages 4, chosen for
  int cluster_threads = -1;   // this CTA size (-1: not chosen yet)
  bool cluster_res = false;   // and whether every component of an instance has a thread (static data in registers)
  bool cluster_dsm = false;   // and whether the state it exchanges stays in distributed shared memory
  std::vector<int> h_task_off, h_big_off;  // host copies of d.task_off, d.big_off
  // warm start staged by acopf_set_warm_start / acopf_set_warm_start_device
  bool warm_x = false, warm_lam = false, warm_rho = false;
  int* d_gen_iperm = nullptr;  // device copy of h_gen_iperm (allocated on first use)
  // CUDA graph of one SQP iteration (sqp_solve_graph)
  bool capturing = false;          // launches are being captured: no host reads, no per-sweep error reset
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  sqp_options gopts{};             // options the graph was captured with
  int gkernels = 0;                // kernel nodes per replay
  int* h_running = nullptr;        // pinned host copy of n_running
  cudaStream_t gstream = nullptr;  // capture stream when the handle has none
};

// kernels, launchers (defined in the .cu files)
void launch_setup(Ctx& c);
void launch_flat_start(Ctx& c);
void launch_build(Ctx& c, bool do_export, int pass = 0);
void launch_admm_reset(Ctx& c, int keep_lambda, int pass = 0);
acopf_status launch_sweep(Ctx& c, const admm_options& o, int fixed_iters);
void launch_step(Ctx& c, int pass = 0);
void launch_merit(Ctx& c, int pass = 0);
void launch_accept_and_kkt(Ctx& c);
void launch_fill_rho(Ctx& c, double rho);
void launch_commit_rho(Ctx& c);
acopf_status project_linear(Ctx& c, double rho, double eps, int max_iter, int check, int* iters, double* rs);
void launch_warm_scatter(Ctx& c, const float* pred, long long ld, int nb, int nl, int ng, double base_rho, int use_x,
                         int use_pi, int use_lam, int use_rho);

// device memory through the handle's allocator (cudaMalloc unless the caller
// set one); ctx_alloc fails on a block that is not 256-byte aligned device
// memory of the handle's device
cudaError_t ctx_alloc(Ctx& c, void** p, size_t bytes);
void ctx_free(Ctx& c, void* p);

inline unsigned nblk(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace acopf
