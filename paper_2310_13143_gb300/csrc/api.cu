// Host implementation of the C ABI declared in include/acopf.h (and of
// acopf_set_warm_start_device from include/acopf_mlp.h).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "../../include/acopf_mlp.h"

namespace acopf {
void launch_admittance(Ctx& c, const double* r, const double* x, const double* b, const double* tap,
                       const double* shift);
void launch_finish(Ctx& c);
}  // namespace acopf

using namespace acopf;

static thread_local std::string g_create_error;

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      c->last_error = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return e_ == cudaErrorMemoryAllocation ? ACOPF_ENOMEM : ACOPF_ECUDA;         \
    }                                                                              \
  } while (0)

static acopf_status fail(Ctx* c, acopf_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

namespace acopf {
cudaError_t ctx_alloc(Ctx& c, void** p, size_t bytes) {
  *p = nullptr;
  if (!c.ualloc) return cudaMalloc(p, bytes);
  void* q = c.ualloc(bytes, c.uctx);
  if (!q) return cudaErrorMemoryAllocation;
  cudaPointerAttributes a{};
  const bool ok = ((uintptr_t)q & 255) == 0 && cudaPointerGetAttributes(&a, q) == cudaSuccess &&
                  (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == c.device;
  if (!ok) {
    cudaGetLastError();
    c.ufree(q, c.uctx);
    return cudaErrorInvalidValue;
  }
  *p = q;
  return cudaSuccess;
}

void ctx_free(Ctx& c, void* p) {
  if (!p) return;
  if (c.ualloc) c.ufree(p, c.uctx);
  else cudaFree(p);
}
}  // namespace acopf

static void release_block(const Ctx::Block& b) {
  if (b.release) b.release(b.p, b.rctx);
  else cudaFree(b.p);
}

// a zeroed block owned by the handle; *slot (a field of the handle) points to it
static cudaError_t dalloc_bytes(Ctx* c, void** slot, size_t bytes) {
  if (c->nblocks >= (int)(sizeof(c->blocks) / sizeof(c->blocks[0]))) return cudaErrorInvalidValue;
  void* v = nullptr;
  cudaError_t e = ctx_alloc(*c, &v, bytes);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(v, 0, bytes, c->stream);
  c->blocks[c->nblocks++] = Ctx::Block{v, bytes, slot, c->ualloc ? c->ufree : nullptr, c->uctx};
  *slot = v;
  return cudaSuccess;
}

template <typename P>
static cudaError_t dalloc(Ctx* c, P** p, size_t count) {
  return dalloc_bytes(c, (void**)p, sizeof(P) * (count > 0 ? count : 1));
}

template <typename P>
static cudaError_t upload(Ctx* c, P* dst, const P* src, size_t count) {
  return cudaMemcpyAsync(dst, src, sizeof(P) * count, cudaMemcpyHostToDevice, c->stream);
}

// ------------------------------------------------------------- read-outs
template <typename TT>
static void to_double(const void* src, double* dst, size_t n) {
  const TT* s = (const TT*)src;
  for (size_t k = 0; k < n; ++k) dst[k] = (double)s[k];
}

static acopf_status fetch(Ctx* c, const void* dev, size_t elems, size_t offset_elems, std::vector<double>& out) {
  size_t es = c->precision == ACOPF_MIXED ? sizeof(float) : sizeof(double);
  std::vector<unsigned char> raw(es * elems);
  CK(cudaMemcpy(raw.data(), (const unsigned char*)dev + es * offset_elems, es * elems, cudaMemcpyDeviceToHost));
  out.resize(elems);
  if (c->precision == ACOPF_MIXED) to_double<float>(raw.data(), out.data(), elems);
  else to_double<double>(raw.data(), out.data(), elems);
  return ACOPF_OK;
}

static acopf_status put(Ctx* c, void* dev, const std::vector<double>& in, size_t offset_elems) {
  size_t es = c->precision == ACOPF_MIXED ? sizeof(float) : sizeof(double);
  std::vector<unsigned char> raw(es * in.size());
  if (c->precision == ACOPF_MIXED)
    for (size_t k = 0; k < in.size(); ++k) ((float*)raw.data())[k] = (float)in[k];
  else
    memcpy(raw.data(), in.data(), es * in.size());
  CK(cudaMemcpy((unsigned char*)dev + es * offset_elems, raw.data(), es * in.size(), cudaMemcpyHostToDevice));
  return ACOPF_OK;
}

static void drop_graph(Ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
}

// oracle slot s of a branch -> (end, component) of the end-major layout
static const int kSlotEnd[8] = {0, 0, 1, 1, 0, 0, 1, 1};
static const int kSlotComp[8] = {0, 1, 0, 1, 2, 3, 2, 3};


extern "C" {

void acopf_default_options(acopf_options* o) {
  o->precision = ACOPF_FP64;
  o->use_angle = 1;
  o->device = 0;
  o->block_threads = 256;
  o->ctas_per_sm = 0;
}

void admm_default_options(admm_options* o) {
  o->rho = 2e4;
  o->eps = 1e-4;
  o->eps_dual = 0.0;
  o->max_iter = 20000;
  o->warm = 1;
  o->alm_beta = 10.0;
  o->alm_tol = 1e-14;
  o->alm_max_outer = 50;
  o->newton_max = 20;
  o->spin_limit = 4000000000LL;
  o->rb_period = 0;
  o->rb_mu = 10.0;
  o->rb_tau = 2.0;
  o->line_solver = 0;
}

void sqp_default_options(sqp_options* o) {
  o->mu = 1e5;
  o->tol = 1e-4;
  o->step_tol = 1e-9;
  o->delta0 = 1.0;
  o->delta_max = 10.0;
  o->delta_min = 1e-8;
  o->max_sqp = 30;
  o->merit_linear = 1;
  o->soc = 0;
  o->restore = 0;
  admm_default_options(&o->admm);
}

const char* acopf_status_string(acopf_status s) {
  switch (s) {
    case ACOPF_OK: return "ok";
    case ACOPF_EINVAL: return "invalid argument";
    case ACOPF_ENOMEM: return "out of memory";
    case ACOPF_ECUDA: return "CUDA error";
    case ACOPF_ETIMEOUT: return "device barrier timed out";
    case ACOPF_ENOTREADY: return "not ready";
  }
  return "unknown status";
}

acopf_status acopf_last_error(acopf_handle h, char* buf, size_t n) {
  const std::string& m = h ? ((Ctx*)h)->last_error : g_create_error;
  if (buf && n > 0) {
    size_t k = m.size() < n - 1 ? m.size() : n - 1;
    memcpy(buf, m.data(), k);
    buf[k] = 0;
  }
  return ACOPF_OK;
}

static std::string validate(const acopf_grid& g, int k) {
  char b[256];
  if (g.nbus < 1 || g.nbranch < 0 || g.ngen < 1) {
    snprintf(b, sizeof b, "grid %d: needs nbus >= 1, ngen >= 1", k);
    return b;
  }
  if (!g.bus_type || !g.pd || !g.qd || !g.gs || !g.bs || !g.vmin || !g.vmax || !g.gbus || !g.pmin || !g.pmax ||
      !g.qmin || !g.qmax || !g.c2 || !g.c1 || !g.c0 ||
      (g.nbranch > 0 && (!g.f || !g.t || !g.r || !g.x || !g.b || !g.rate || !g.angmin || !g.angmax))) {
    snprintf(b, sizeof b, "grid %d: a required array is NULL", k);
    return b;
  }
  int nref = 0;
  for (int i = 0; i < g.nbus; ++i) {
    if (g.bus_type[i] == 3) nref++;
    if (!(g.vmin[i] > 0) || !(g.vmin[i] <= g.vmax[i])) {
      snprintf(b, sizeof b, "grid %d: bus %d has invalid voltage limits", k, i);
      return b;
    }
  }
  if (nref != 1) {
    snprintf(b, sizeof b, "grid %d: needs exactly one reference bus (bus_type 3), found %d", k, nref);
    return b;
  }
  std::vector<int> deg(g.nbus, 0);
  for (int l = 0; l < g.nbranch; ++l) {
    if (g.f[l] < 0 || g.f[l] >= g.nbus || g.t[l] < 0 || g.t[l] >= g.nbus || g.f[l] == g.t[l]) {
      snprintf(b, sizeof b, "grid %d: branch %d has invalid end buses", k, l);
      return b;
    }
    if (g.r[l] * g.r[l] + g.x[l] * g.x[l] <= 0) {
      snprintf(b, sizeof b, "grid %d: branch %d has zero impedance", k, l);
      return b;
    }
    deg[g.f[l]]++;
    deg[g.t[l]]++;
  }
  if (g.nbus > 1)
    for (int i = 0; i < g.nbus; ++i)
      if (deg[i] == 0) {
        snprintf(b, sizeof b, "grid %d: bus %d is isolated", k, i);
        return b;
      }
  for (int q = 0; q < g.ngen; ++q) {
    if (g.gbus[q] < 0 || g.gbus[q] >= g.nbus) {
      snprintf(b, sizeof b, "grid %d: generator %d at invalid bus", k, q);
      return b;
    }
    if (!(g.pmin[q] <= g.pmax[q]) || !(g.qmin[q] <= g.qmax[q])) {
      snprintf(b, sizeof b, "grid %d: generator %d has invalid limits", k, q);
      return b;
    }
  }
  return "";
}

acopf_status acopf_create(const acopf_grid* grids, int32_t ngrids, const acopf_options* opt, acopf_handle* out) {
  g_create_error.clear();
  if (!grids || ngrids < 1 || !out) {
    g_create_error = "acopf_create: grids, ngrids >= 1 and out are required";
    return ACOPF_EINVAL;
  }
  acopf_options o;
  if (opt) o = *opt;
  else acopf_default_options(&o);
  if (o.precision != ACOPF_FP64 && o.precision != ACOPF_MIXED) {
    g_create_error = "acopf_create: precision must be ACOPF_FP64 or ACOPF_MIXED";
    return ACOPF_EINVAL;
  }
  for (int k = 0; k < ngrids; ++k) {
    std::string m = validate(grids[k], k);
    if (!m.empty()) {
      g_create_error = m;
      return ACOPF_EINVAL;
    }
  }
  {
    // component indices are 32-bit: branch ends (2L) and bus-update entries
    // (G + 2L) must stay below 2^30
    long long b = 0, l = 0, gg = 0;
    for (int k = 0; k < ngrids; ++k) { b += grids[k].nbus; l += grids[k].nbranch; gg += grids[k].ngen; }
    if (b >= (1ll << 30) || 2 * l + gg >= (1ll << 30)) {
      g_create_error = "acopf_create: too many components for 32-bit indices (buses, 2 x branches + generators < 2^30)";
      return ACOPF_EINVAL;
    }
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1 || o.device < 0 || o.device >= ndev) {
    cudaGetLastError();
    g_create_error = "acopf_create: no usable CUDA device";
    return ACOPF_ECUDA;
  }
  if (cudaSetDevice(o.device) != cudaSuccess) {
    g_create_error = "acopf_create: cudaSetDevice failed";
    return ACOPF_ECUDA;
  }
  Ctx* c = new Ctx();
  c->precision = o.precision;
  c->use_angle = o.use_angle ? 1 : 0;
  c->device = o.device;
  c->block_threads = o.block_threads > 0 ? o.block_threads : 256;
  if (c->block_threads > 256) c->block_threads = 256;
  c->block_threads = (c->block_threads / 32) * 32;
  if (c->block_threads < 32) c->block_threads = 32;
  c->ctas_per_sm = o.ctas_per_sm;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, o.device);
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, o.device);
  if (!coop) {
    delete c;
    g_create_error = "acopf_create: device lacks cooperative launch";
    return ACOPF_ECUDA;
  }

  // ---- host-side concatenation
  int K = ngrids, B = 0, L = 0, G = 0;
  std::vector<int> bus_off(K + 1), br_off(K + 1), gen_off(K + 1);
  for (int k = 0; k < K; ++k) {
    bus_off[k] = B; br_off[k] = L; gen_off[k] = G;
    B += grids[k].nbus; L += grids[k].nbranch; G += grids[k].ngen;
  }
  bus_off[K] = B; br_off[K] = L; gen_off[K] = G;
  std::vector<double> pd(B), qd(B), gs(B), bs(B), wmin(B), wmax(B);
  std::vector<int> isref(B), bus_inst(B), br_inst(L), gen_inst(G);
  std::vector<int> f(L), t(L);
  std::vector<double> r(L), x(L), bc(L), tap(L), shift(L), s2(L), amin(L), amax(L);
  std::vector<int> gbus_user(G);
  std::vector<double> pmin(G), pmax(G), qmin(G), qmax(G), cq(G), cl(G), cc(G);
  for (int k = 0; k < K; ++k) {
    const acopf_grid& g = grids[k];
    double S = g.base_mva > 0 ? g.base_mva : 100.0;
    for (int i = 0; i < g.nbus; ++i) {
      int I = bus_off[k] + i;
      pd[I] = g.pd[i]; qd[I] = g.qd[i]; gs[I] = g.gs[i]; bs[I] = g.bs[i];
      wmin[I] = g.vmin[i] * g.vmin[i]; wmax[I] = g.vmax[i] * g.vmax[i];
      isref[I] = g.bus_type[i] == 3; bus_inst[I] = k;
    }
    for (int l = 0; l < g.nbranch; ++l) {
      int Lg = br_off[k] + l;
      f[Lg] = bus_off[k] + g.f[l]; t[Lg] = bus_off[k] + g.t[l];
      r[Lg] = g.r[l]; x[Lg] = g.x[l]; bc[Lg] = g.b[l];
      tap[Lg] = g.tap ? g.tap[l] : 1.0; shift[Lg] = g.shift ? g.shift[l] : 0.0;
      s2[Lg] = g.rate[l] > 0 ? g.rate[l] * g.rate[l] : -1.0;
      amin[Lg] = g.angmin[l]; amax[Lg] = g.angmax[l];
      br_inst[Lg] = k;
    }
    for (int q = 0; q < g.ngen; ++q) {
      int Q = gen_off[k] + q;
      gbus_user[Q] = bus_off[k] + g.gbus[q];
      pmin[Q] = g.pmin[q]; pmax[Q] = g.pmax[q]; qmin[Q] = g.qmin[q]; qmax[Q] = g.qmax[q];
      // cost per MW -> per unit: c2 (S p)^2 + c1 S p + c0
      cq[Q] = g.c2[q] * S * S; cl[Q] = g.c1[q] * S; cc[Q] = g.c0[q];
    }
  }
  // generators sorted by (global) bus; perm[internal] = user index
  std::vector<int> perm(G);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return gbus_user[a] < gbus_user[b]; });
  std::vector<int> iperm(G);
  for (int q = 0; q < G; ++q) iperm[perm[q]] = q;
  auto P = [&](const std::vector<double>& v) {
    std::vector<double> o2(G);
    for (int q = 0; q < G; ++q) o2[q] = v[perm[q]];
    return o2;
  };
  std::vector<int> gbus(G), gen_inst_s(G);
  for (int q = 0; q < G; ++q) {
    gbus[q] = gbus_user[perm[q]];
    gen_inst_s[q] = bus_inst[gbus[q]];
  }
  std::vector<int> gen_ptr(B + 1, 0);
  for (int q = 0; q < G; ++q) gen_ptr[gbus[q] + 1]++;
  for (int i = 0; i < B; ++i) gen_ptr[i + 1] += gen_ptr[i];
  std::vector<int> end_ptr(B + 1, 0), end_idx(2 * (size_t)L), fill(B, 0);
  for (int l = 0; l < L; ++l) { end_ptr[f[l] + 1]++; end_ptr[t[l] + 1]++; }
  for (int i = 0; i < B; ++i) end_ptr[i + 1] += end_ptr[i];
  for (int l = 0; l < L; ++l) {
    end_idx[end_ptr[f[l]] + fill[f[l]]++] = 2 * l;
    end_idx[end_ptr[t[l]] + fill[t[l]]++] = 2 * l + 1;
  }
  // bus update work list and its warp tasks (consecutive whole buses, at most
  // 32 entries per task; a bus with more entries is a task of its own)
  const size_t E = (size_t)G + 2 * (size_t)L;
  std::vector<int> ent(E), ebus(E), pent, pbus, pinst, big, task_off, big_off;
  {
    size_t q = 0;
    for (int i = 0; i < B; ++i) {
      for (int g = gen_ptr[i]; g < gen_ptr[i + 1]; ++g) { ent[q] = -(g + 1); ebus[q++] = i; }
      for (int e2 = end_ptr[i]; e2 < end_ptr[i + 1]; ++e2) { ent[q] = end_idx[e2]; ebus[q++] = i; }
    }
    size_t q0 = 0;   // first entry of the open task
    size_t cnt = 0;  // its entries
    auto close = [&]() {
      if (cnt == 0) return;
      for (size_t j = 0; j < 32; ++j) {
        bool in = j < cnt;
        pent.push_back(in ? ent[q0 + j] : 0);
        pbus.push_back(in ? ebus[q0 + j] : -1);
        pinst.push_back(in ? bus_inst[ebus[q0 + j]] : -1);
      }
      q0 += cnt;
      cnt = 0;
    };
    task_off.assign(K + 1, 0);
    big_off.assign(K + 1, 0);
    int kk = 0;
    for (int i = 0; i < B; ++i) {
      // tasks never span two instances (a cluster of the sweep takes whole tasks of its instance)
      while (kk < K && i == bus_off[kk]) {
        close();
        task_off[kk] = (int)(pbus.size() / 32);
        big_off[kk] = (int)(big.size() / 2);
        ++kk;
      }
      size_t n = (size_t)(gen_ptr[i + 1] - gen_ptr[i]) + (size_t)(end_ptr[i + 1] - end_ptr[i]);
      if (n > 32) {
        close();
        big.push_back((int)q0);
        big.push_back((int)(q0 + n));
        q0 += n;
        continue;
      }
      if (cnt + n > 32) close();
      cnt += n;
    }
    close();
    for (; kk <= K; ++kk) {
      task_off[kk] = (int)(pbus.size() / 32);
      big_off[kk] = (int)(big.size() / 2);
    }
  }

  // ---- device allocation
  Dev& d = c->d;
  d.K = K; d.B = B; d.L = L; d.G = G;
  cudaError_t e = cudaSuccess;
  size_t T = c->precision == ACOPF_MIXED ? sizeof(float) : sizeof(double);
#define A(ptr, n) if (e == cudaSuccess) e = dalloc(c, &(ptr), (n))
  A(d.bus_off, K + 1); A(d.br_off, K + 1); A(d.gen_off, K + 1);
  A(d.bus_inst, B); A(d.br_inst, L); A(d.gen_inst, G);
  A(d.pd, B); A(d.qd, B); A(d.gs, B); A(d.bs, B); A(d.wmin, B); A(d.wmax, B); A(d.isref, B);
  A(d.end_ptr, B + 1); A(d.end_idx, 2 * (size_t)L); A(d.gen_ptr, B + 1);
  A(d.ent, E); A(d.ebus, E); A(d.pent, pent.size()); A(d.pbus, pbus.size()); A(d.pinst, pinst.size());
  A(d.big, big.size()); A(d.task_off, K + 1); A(d.big_off, K + 1); A(d.wset, L);
  d.E = (int)E;
  d.NT = (int)(pbus.size() / 32);
  d.NBIG = (int)(big.size() / 2);
  A(d.f, L); A(d.t, L); A(d.Y, 8 * (size_t)L); A(d.s2, L); A(d.angmin, L); A(d.angmax, L);
  A(d.gbus, G); A(d.pmin, G); A(d.pmax, G); A(d.qmin, G); A(d.qmax, G); A(d.cq, G); A(d.cl, G); A(d.cc, G);
  A(d.pg, G); A(d.qg, G); A(d.w, B); A(d.th, B); A(d.wr, L); A(d.wi, L); A(d.pi, 4 * (size_t)L);
  A(d.dpg, G); A(d.dqg, G); A(d.dw, B); A(d.dth, B); A(d.dwr, L); A(d.dwi, L); A(d.pi_new, 4 * (size_t)L);
  A(d.flow, 4 * (size_t)L); A(d.aR, 4 * (size_t)L); A(d.aI, 4 * (size_t)L); A(d.bR, L); A(d.bI, L);
  A(d.gd1, G); A(d.gd2, G); A(d.rho_l, L); A(d.rho_g, G);
#define AR(ptr, bytes) if (e == cudaSuccess) e = dalloc_bytes(c, &(ptr), (bytes))
  AR(d.lrec, T * 4 * kRecChunks * (size_t)L);
  AR(d.grec, T * 8 * (size_t)G);
  AR(d.brec, T * 4 * (size_t)B);
  AR(d.trho_l, T * (size_t)L);
  AR(d.X, T * 4 * 2 * (size_t)L); AR(d.Z, T * 4 * 2 * (size_t)L); AR(d.LAM, T * 4 * 2 * (size_t)L);
  AR(d.U, T * 4 * (size_t)L);
  AR(d.XG, T * 2 * (size_t)G); AR(d.ZG, T * 2 * (size_t)G); AR(d.LG, T * 2 * (size_t)G);
  AR(d.ZB, T * 2 * (size_t)B); AR(d.NU, T * 2 * (size_t)B);
  A(d.res_slots, 4 * (size_t)K); A(d.admm_done, K); A(d.admm_iters, K); A(d.admm_rs, 2 * (size_t)K);
  A(d.bar, 2); A(d.err, 1);
  A(d.flow_xd, 4 * (size_t)L); A(d.tbr, 8 * (size_t)L); A(d.tbus, 4 * (size_t)B); A(d.tgen, 8 * (size_t)G);
  A(d.dend, 2 * 2 * (size_t)L); A(d.red, 16 * (size_t)K); A(d.ctl, K); A(d.n_running, 1);
  A(d.hist, (size_t)K * ACOPF_HIST_MAX * kHistW); A(d.rho_fac, K); A(d.phase_ns, 4);
#undef A
#undef AR
  double *d_r = nullptr, *d_x = nullptr, *d_b = nullptr, *d_tap = nullptr, *d_sh = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_r, sizeof(double) * 5 * (size_t)(L > 0 ? L : 1));
  if (e != cudaSuccess) {
    g_create_error = std::string("acopf_create: device allocation failed: ") + cudaGetErrorString(e);
    acopf_destroy((acopf_handle)c);
    return e == cudaErrorMemoryAllocation ? ACOPF_ENOMEM : ACOPF_ECUDA;
  }
  d_x = d_r + L; d_b = d_r + 2 * (size_t)L; d_tap = d_r + 3 * (size_t)L; d_sh = d_r + 4 * (size_t)L;
  std::vector<int> pd_dummy;
  e = cudaSuccess;
#define U(dst, v) if (e == cudaSuccess && !(v).empty()) e = upload(c, dst, (v).data(), (v).size())
  U(d.bus_off, bus_off); U(d.br_off, br_off); U(d.gen_off, gen_off);
  U(d.bus_inst, bus_inst); U(d.br_inst, br_inst); U(d.gen_inst, gen_inst_s);
  U(d.pd, pd); U(d.qd, qd); U(d.gs, gs); U(d.bs, bs); U(d.wmin, wmin); U(d.wmax, wmax); U(d.isref, isref);
  U(d.end_ptr, end_ptr); U(d.end_idx, end_idx); U(d.gen_ptr, gen_ptr);
  U(d.ent, ent); U(d.ebus, ebus); U(d.pent, pent); U(d.pbus, pbus); U(d.pinst, pinst); U(d.big, big);
  U(d.task_off, task_off); U(d.big_off, big_off);
  c->h_task_off = task_off;
  c->h_big_off = big_off;
  U(d.f, f); U(d.t, t); U(d.s2, s2); U(d.angmin, amin); U(d.angmax, amax);
  U(d.gbus, gbus);
  std::vector<double> v_pmin = P(pmin), v_pmax = P(pmax), v_qmin = P(qmin), v_qmax = P(qmax), v_cq = P(cq),
                      v_cl = P(cl), v_cc = P(cc);
  U(d.pmin, v_pmin); U(d.pmax, v_pmax); U(d.qmin, v_qmin); U(d.qmax, v_qmax);
  U(d.cq, v_cq); U(d.cl, v_cl); U(d.cc, v_cc);
  U(d_r, r); U(d_x, x); U(d_b, bc); U(d_tap, tap); U(d_sh, shift);
#undef U
  if (e != cudaSuccess) {
    g_create_error = std::string("acopf_create: upload failed: ") + cudaGetErrorString(e);
    cudaFree(d_r);
    acopf_destroy((acopf_handle)c);
    return ACOPF_ECUDA;
  }
  if (L > 0) launch_admittance(*c, d_r, d_x, d_b, d_tap, d_sh);
  // control blocks
  std::vector<InstCtl> ctl(K);
  for (int k = 0; k < K; ++k) {
    memset(&ctl[k], 0, sizeof(InstCtl));
    ctl[k].result = ACOPF_RUNNING;
    ctl[k].delta = 1.0;
    ctl[k].primal = ctl[k].dual = kBig;
  }
  e = upload(c, d.ctl, ctl.data(), K);
  launch_flat_start(*c);
  admm_options ao;
  admm_default_options(&ao);
  launch_fill_rho(*c, ao.rho);
  cudaError_t e2 = cudaStreamSynchronize(c->stream);
  cudaFree(d_r);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    g_create_error = std::string("acopf_create: set-up failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
    acopf_destroy((acopf_handle)c);
    return ACOPF_ECUDA;
  }
  c->h_bus_off = (int*)malloc(sizeof(int) * (K + 1));
  c->h_br_off = (int*)malloc(sizeof(int) * (K + 1));
  c->h_gen_off = (int*)malloc(sizeof(int) * (K + 1));
  c->h_gen_perm = (int*)malloc(sizeof(int) * (G > 0 ? G : 1));
  c->h_gen_iperm = (int*)malloc(sizeof(int) * (G > 0 ? G : 1));
  memcpy(c->h_bus_off, bus_off.data(), sizeof(int) * (K + 1));
  memcpy(c->h_br_off, br_off.data(), sizeof(int) * (K + 1));
  memcpy(c->h_gen_off, gen_off.data(), sizeof(int) * (K + 1));
  memcpy(c->h_gen_perm, perm.data(), sizeof(int) * G);
  memcpy(c->h_gen_iperm, iperm.data(), sizeof(int) * G);
  *out = (acopf_handle)c;
  return ACOPF_OK;
}

acopf_status acopf_destroy(acopf_handle h) {
  if (!h) return ACOPF_EINVAL;
  Ctx* c = (Ctx*)h;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (int k = 0; k < c->nblocks; ++k) release_block(c->blocks[k]);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->h_running) cudaFreeHost(c->h_running);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  free(c->h_bus_off); free(c->h_br_off); free(c->h_gen_off); free(c->h_gen_perm); free(c->h_gen_iperm);
  delete c;
  return ACOPF_OK;
}

acopf_status acopf_set_stream(acopf_handle h, void* s) {
  if (!h) return ACOPF_EINVAL;
  ((Ctx*)h)->stream = (cudaStream_t)s;
  return ACOPF_OK;
}

acopf_status acopf_set_allocator(acopf_handle h, void* (*alloc)(size_t bytes, void* ctx),
                                 void (*release)(void* ptr, void* ctx), void* ctx) {
  Ctx* c = (Ctx*)h;
  if (!c) return ACOPF_EINVAL;
  if ((alloc == nullptr) != (release == nullptr))
    return fail(c, ACOPF_EINVAL, "acopf_set_allocator: alloc and free must both be given or both be NULL");
  CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
  drop_graph(c);
  void* (*old_alloc)(size_t, void*) = c->ualloc;
  void (*old_free)(void*, void*) = c->ufree;
  void* old_ctx = c->uctx;
  c->ualloc = alloc;
  c->ufree = release;
  c->uctx = ctx;
  // new blocks first: on any failure the handle keeps its memory and allocator
  std::vector<void*> fresh((size_t)c->nblocks, nullptr);
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < c->nblocks && e == cudaSuccess; ++k) e = ctx_alloc(*c, &fresh[k], c->blocks[k].bytes);
  for (int k = 0; k < c->nblocks && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(fresh[k], c->blocks[k].p, c->blocks[k].bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (void* p : fresh) ctx_free(*c, p);
    c->ualloc = old_alloc;
    c->ufree = old_free;
    c->uctx = old_ctx;
    const acopf_status s = e == cudaErrorMemoryAllocation ? ACOPF_ENOMEM
                           : e == cudaErrorInvalidValue   ? ACOPF_EINVAL
                                                          : ACOPF_ECUDA;
    return fail(c, s,
                std::string("acopf_set_allocator: moving the handle's memory failed: ") +
                    (s == ACOPF_EINVAL ? "a block was not 256-byte aligned device memory of the handle's device"
                                       : cudaGetErrorString(e)));
  }
  for (int k = 0; k < c->nblocks; ++k) {
    Ctx::Block& b = c->blocks[k];
    release_block(b);
    b.p = fresh[k];
    *b.slot = fresh[k];
    b.release = alloc ? release : nullptr;
    b.rctx = ctx;
  }
  return ACOPF_OK;
}

acopf_status acopf_profile(acopf_handle h, int32_t on) {
  Ctx* c = (Ctx*)h;
  if (!c) return ACOPF_EINVAL;
  if (!c->ev0) {
    CK(cudaEventCreate(&c->ev0));
    CK(cudaEventCreate(&c->ev1));
  }
  c->profiling = on != 0;
  c->prof_ms = 0.0;
  c->prof_sweeps = c->prof_iters = 0;
  CK(cudaMemsetAsync(c->d.phase_ns, 0, 4 * sizeof(unsigned long long), c->stream));
  return ACOPF_OK;
}

acopf_status acopf_get_profile(acopf_handle h, double* ms, int64_t* sweeps, int64_t* iters) {
  Ctx* c = (Ctx*)h;
  if (!c) return ACOPF_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  if (ms) *ms = c->prof_ms;
  if (sweeps) *sweeps = c->prof_sweeps;
  if (iters) *iters = c->prof_iters;
  return ACOPF_OK;
}

acopf_status acopf_get_profile_phases(acopf_handle h, double* ns) {
  Ctx* c = (Ctx*)h;
  if (!c || !ns) return ACOPF_EINVAL;
  unsigned long long v[4];
  CK(cudaMemcpyAsync(v, c->d.phase_ns, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 4; ++k) ns[k] = (double)v[k];
  return ACOPF_OK;
}

acopf_status acopf_tune(acopf_handle h, int32_t block_threads, int32_t ctas_per_sm, int32_t sweep_stages) {
  Ctx* c = (Ctx*)h;
  if (!c) return ACOPF_EINVAL;
  if (block_threads > 0) {
    if (block_threads % 32 || block_threads > 256) return fail(c, ACOPF_EINVAL, "acopf_tune: block_threads must be 32..256, a multiple of 32");
    c->block_threads = block_threads;
  }
  if (ctas_per_sm >= 0) c->ctas_per_sm = ctas_per_sm;
  if (sweep_stages >= 0) {
    if (sweep_stages > 4) return fail(c, ACOPF_EINVAL, "acopf_tune: sweep_stages must be 0, 1, 2, 3 or 4");
    c->sweep_stages = sweep_stages;
  }
  drop_graph(c);  // the launch shape is baked into a captured graph
  return ACOPF_OK;
}

acopf_status acopf_launch_count(acopf_handle h, int64_t* n) {
  if (!h || !n) return ACOPF_EINVAL;
  *n = ((Ctx*)h)->launches;
  return ACOPF_OK;
}

static bool inst_ok(Ctx* c, int inst) { return inst >= 0 && inst < c->d.K; }

acopf_status acopf_set_loads(acopf_handle h, int32_t inst, const double* pd, const double* qd) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst) || !pd || !qd) return fail(c, ACOPF_EINVAL, "acopf_set_loads: bad arguments");
  int b0 = c->h_bus_off[inst], nb = c->h_bus_off[inst + 1] - b0;
  CK(cudaMemcpyAsync(c->d.pd + b0, pd, sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d.qd + b0, qd, sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream));
  return ACOPF_OK;
}

// ---------------------------------------------------------------- iterate
acopf_status acopf_set_iterate(acopf_handle h, int32_t inst, const double* x, const double* pi) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst) || !x) return fail(c, ACOPF_EINVAL, "acopf_set_iterate: bad arguments");
  Dev& d = c->d;
  int b0 = c->h_bus_off[inst], nb = c->h_bus_off[inst + 1] - b0;
  int l0 = c->h_br_off[inst], nl = c->h_br_off[inst + 1] - l0;
  int g0 = c->h_gen_off[inst], ng = c->h_gen_off[inst + 1] - g0;
  std::vector<double> pg(ng), qg(ng);
  for (int q = 0; q < ng; ++q) {
    int internal = c->h_gen_iperm[g0 + q] - g0;
    pg[internal] = x[q];
    qg[internal] = x[ng + q];
  }
  const double* w = x + 2 * ng;
  CK(cudaMemcpy(d.pg + g0, pg.data(), sizeof(double) * ng, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d.qg + g0, qg.data(), sizeof(double) * ng, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d.w + b0, w, sizeof(double) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d.th + b0, w + nb, sizeof(double) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d.wr + l0, w + 2 * nb, sizeof(double) * nl, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d.wi + l0, w + 2 * nb + nl, sizeof(double) * nl, cudaMemcpyHostToDevice));
  if (pi) {
    std::vector<double> col(nl);
    for (int r = 0; r < 4; ++r) {
      for (int l = 0; l < nl; ++l) col[l] = pi[4 * l + r];
      CK(cudaMemcpy(d.pi + (size_t)r * d.L + l0, col.data(), sizeof(double) * nl, cudaMemcpyHostToDevice));
    }
  }
  return ACOPF_OK;
}

acopf_status acopf_get_iterate(acopf_handle h, int32_t inst, double* x, double* pi) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst) || !x) return fail(c, ACOPF_EINVAL, "acopf_get_iterate: bad arguments");
  Dev& d = c->d;
  CK(cudaStreamSynchronize(c->stream));
  int b0 = c->h_bus_off[inst], nb = c->h_bus_off[inst + 1] - b0;
  int l0 = c->h_br_off[inst], nl = c->h_br_off[inst + 1] - l0;
  int g0 = c->h_gen_off[inst], ng = c->h_gen_off[inst + 1] - g0;
  std::vector<double> pg(ng), qg(ng);
  CK(cudaMemcpy(pg.data(), d.pg + g0, sizeof(double) * ng, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(qg.data(), d.qg + g0, sizeof(double) * ng, cudaMemcpyDeviceToHost));
  for (int q = 0; q < ng; ++q) {
    int internal = c->h_gen_iperm[g0 + q] - g0;
    x[q] = pg[internal];
    x[ng + q] = qg[internal];
  }
  double* w = x + 2 * ng;
  CK(cudaMemcpy(w, d.w + b0, sizeof(double) * nb, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(w + nb, d.th + b0, sizeof(double) * nb, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(w + 2 * nb, d.wr + l0, sizeof(double) * nl, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(w + 2 * nb + nl, d.wi + l0, sizeof(double) * nl, cudaMemcpyDeviceToHost));
  if (pi) {
    std::vector<double> col(nl);
    for (int r = 0; r < 4; ++r) {
      CK(cudaMemcpy(col.data(), d.pi + (size_t)r * d.L + l0, sizeof(double) * nl, cudaMemcpyDeviceToHost));
      for (int l = 0; l < nl; ++l) pi[4 * l + r] = col[l];
    }
  }
  return ACOPF_OK;
}

// ---------------------------------------------------------------- control
static acopf_status reset_control(Ctx* c, const sqp_options& o, bool fresh) {
  Dev& d = c->d;
  std::vector<InstCtl> ctl(d.K);
  for (int k = 0; k < d.K; ++k) {
    InstCtl& q = ctl[k];
    memset(&q, 0, sizeof(q));
    q.delta = o.delta0;
    q.mu = o.mu;
    q.tol = o.tol;
    q.step_tol = o.step_tol;
    q.delta_max = o.delta_max;
    q.delta_min = o.delta_min;
    q.obj = NAN;
    q.primal = fresh ? kBig : kBig;
    q.dual = kBig;
    q.rho = o.admm.rho;
    q.eps = o.admm.eps;
    q.result = ACOPF_RUNNING;
    q.merit_linear = o.merit_linear ? 1 : 0;
    q.soc_on = o.soc ? 1 : 0;
    q.restore_on = o.restore ? 1 : 0;
    q.fscale = 1.0;
    q.delta0 = o.delta0;
  }
  CK(cudaMemcpyAsync(d.ctl, ctl.data(), sizeof(InstCtl) * d.K, cudaMemcpyHostToDevice, c->stream));
  // copy back: the host vector is about to go out of scope
  CK(cudaStreamSynchronize(c->stream));
  return ACOPF_OK;
}

static acopf_status check_admm(const admm_options& a, Ctx* c) {
  if (!(a.rho > 0) || !(a.eps >= 0) || !(a.eps_dual >= 0) || a.max_iter < 1 || a.alm_max_outer < 1 || a.newton_max < 1 ||
      !(a.alm_beta > 0) || a.spin_limit < 1 || a.rb_period < 0 ||
      (a.rb_period > 0 && (!(a.rb_mu > 1) || !(a.rb_tau > 1))) || a.line_solver < 0 || a.line_solver > 1)
    return fail(c, ACOPF_EINVAL, "admm options out of range");
  return ACOPF_OK;
}

static acopf_status sweep_status(Ctx* c) {
  int err = 0;
  CK(cudaMemcpyAsync(&err, c->d.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (err) return fail(c, ACOPF_ETIMEOUT, "ADMM kernel: a CTA timed out at a device-wide barrier");
  return ACOPF_OK;
}

// The correction pass of an SQP iteration (sqp_options.soc): for the instances
// whose step the merit test rejected, the QP rebuilt with the constraint values
// of x + d, solved by the same sweep, and its step judged against the original
// model reduction; every other instance is skipped by each kernel.  Always
// launched when soc is on, so that a captured iteration has a fixed shape.
static acopf_status launch_soc_pass(Ctx& c, const sqp_options& o) {
  if (!o.soc) return ACOPF_OK;
  launch_build(c, false, 1);
  launch_admm_reset(c, o.admm.warm, 1);
  acopf_status s = launch_sweep(c, o.admm, 0);
  if (s) return s;
  launch_step(c, 1);
  launch_merit(c, 1);
  return ACOPF_OK;
}

acopf_status sqp_solve(acopf_handle h, const sqp_options* op) {
  Ctx* c = (Ctx*)h;
  if (!c) return ACOPF_EINVAL;
  sqp_options o;
  if (op) o = *op;
  else sqp_default_options(&o);
  if (o.max_sqp < 1 || !(o.delta0 > 0) || !(o.mu >= 0) || o.soc < 0 || o.soc > 1 || o.restore < 0 || o.restore > 1)
    return fail(c, ACOPF_EINVAL, "sqp options out of range");
  acopf_status s = check_admm(o.admm, c);
  if (s) return s;
  if (!c->warm_x) launch_flat_start(*c);
  if (!c->warm_rho) launch_fill_rho(*c, o.admm.rho);
  if ((s = reset_control(c, o, true))) return s;
  bool first = true;
  for (int it = 0; it < o.max_sqp; ++it) {
    launch_build(*c, false);
    int keep = first ? (c->warm_lam ? 1 : 0) : o.admm.warm;
    launch_admm_reset(*c, keep);
    first = false;
    if ((s = launch_sweep(*c, o.admm, 0))) return s;
    if (o.admm.warm && o.admm.rb_period > 0) launch_commit_rho(*c);
    launch_step(*c);
    launch_merit(*c);
    if ((s = launch_soc_pass(*c, o))) return s;
    launch_accept_and_kkt(*c);
    int running = 0;
    CK(cudaMemcpyAsync(&running, c->d.n_running, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if ((s = sweep_status(c))) return s;
    CK(cudaGetLastError());
    if (running == 0) break;
  }
  launch_finish(*c);
  CK(cudaGetLastError());
  c->warm_x = c->warm_lam = c->warm_rho = false;
  c->qp_built = true;
  c->have_step = true;
  return ACOPF_OK;
}

// The SQP loop with every iteration after the first replayed from one CUDA
// graph (build, ADMM reset, the persistent sweep, step, merit, acceptance and
// the copy of the running count to pinned host memory).  The host reads the
// running count only every check_every replays; replays after the last
// instance has stopped change nothing (every kernel skips stopped instances).
acopf_status sqp_solve_graph(acopf_handle h, const sqp_options* op, int32_t check_every) {
  Ctx* c = (Ctx*)h;
  if (!c || check_every < 1) return fail(c, ACOPF_EINVAL, "sqp_solve_graph: bad arguments");
  sqp_options o;
  if (op) o = *op;
  else sqp_default_options(&o);
  if (o.max_sqp < 1 || !(o.delta0 > 0) || !(o.mu >= 0) || o.soc < 0 || o.soc > 1 || o.restore < 0 || o.restore > 1)
    return fail(c, ACOPF_EINVAL, "sqp options out of range");
  acopf_status s = check_admm(o.admm, c);
  if (s) return s;
  cudaStream_t user = c->stream;
  if (!user) {
    if (!c->gstream) CK(cudaStreamCreate(&c->gstream));
    CK(cudaDeviceSynchronize());
    c->stream = c->gstream;
  }
  struct Restore {
    Ctx* c;
    cudaStream_t s;
    ~Restore() { c->stream = s; c->capturing = false; }
  } restore{c, user};
  if (!c->h_running) CK(cudaMallocHost(&c->h_running, sizeof(int)));
  if (!c->warm_x) launch_flat_start(*c);
  if (!c->warm_rho) launch_fill_rho(*c, o.admm.rho);
  if ((s = reset_control(c, o, true))) return s;
  // first iteration eagerly: its ADMM start depends on the warm start
  launch_build(*c, false);
  launch_admm_reset(*c, c->warm_lam ? 1 : 0);
  if ((s = launch_sweep(*c, o.admm, 0))) return s;
  if (o.admm.warm && o.admm.rb_period > 0) launch_commit_rho(*c);
  launch_step(*c);
  launch_merit(*c);
  if ((s = launch_soc_pass(*c, o))) return s;
  launch_accept_and_kkt(*c);
  CK(cudaMemcpyAsync(c->h_running, c->d.n_running, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if ((s = sweep_status(c))) return s;
  int running = *c->h_running;
  if (running > 0 && o.max_sqp > 1) {
    if (!c->gexec || memcmp(&c->gopts, &o, sizeof(o)) != 0) {
      drop_graph(c);
      int64_t l0 = c->launches;
      c->capturing = true;
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      launch_build(*c, false);
      launch_admm_reset(*c, o.admm.warm);
      acopf_status cs = launch_sweep(*c, o.admm, 0);
      if (o.admm.warm && o.admm.rb_period > 0) launch_commit_rho(*c);
      launch_step(*c);
      launch_merit(*c);
      if (!cs) cs = launch_soc_pass(*c, o);
      launch_accept_and_kkt(*c);
      cudaMemcpyAsync(c->h_running, c->d.n_running, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
      c->capturing = false;
      c->gkernels = (int)(c->launches - l0);
      c->launches = l0;
      if (cs) {
        if (g) cudaGraphDestroy(g);
        return cs;
      }
      CK(ce);
      c->graph = g;
      CK(cudaGraphInstantiate(&c->gexec, g, 0));
      c->gopts = o;
    }
    for (int it = 1; it < o.max_sqp; ++it) {
      CK(cudaGraphLaunch(c->gexec, c->stream));
      c->launches += c->gkernels;
      if (it % check_every == 0 || it == o.max_sqp - 1) {
        if ((s = sweep_status(c))) return s;
        if (*c->h_running == 0) break;
      }
    }
  }
  launch_finish(*c);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  c->warm_x = c->warm_lam = c->warm_rho = false;
  c->qp_built = true;
  c->have_step = true;
  return ACOPF_OK;
}

// ----------------------------------------------------------------- autotune
// Launch shapes of the ADMM sweep timed on the QP at the current iterate; the
// fastest is applied and remembered in a JSON cache keyed by the GPU's SM
// count, the sweep precision and the binary orders of magnitude of the
// instance, bus and branch counts.
static std::string tune_key(Ctx* c) {
  auto lg = [](long v) {
    int k = 0;
    while (v > 1) { v >>= 1; ++k; }
    return k;
  };
  char buf[128];
  snprintf(buf, sizeof(buf), "v4-sm%d-%s-K%d-B%d-L%d", c->num_sms, c->precision == ACOPF_MIXED ? "mixed" : "fp64",
           lg(c->d.K), lg(c->d.B), lg(c->d.L));
  return buf;
}

static std::vector<std::string> read_lines(const char* path) {
  std::vector<std::string> out;
  FILE* f = path ? fopen(path, "r") : nullptr;
  if (!f) return out;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    std::string l(line);
    while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
    out.push_back(l);
  }
  fclose(f);
  return out;
}

static bool cache_lookup(const char* path, const std::string& key, int shape[3]) {
  for (const std::string& l : read_lines(path)) {
    if (l.find("\"key\": \"" + key + "\"") == std::string::npos) continue;
    int bt = 0, cps = -1, st = 0;
    const char* p = strstr(l.c_str(), "\"block_threads\":");
    const char* q = strstr(l.c_str(), "\"ctas_per_sm\":");
    const char* r = strstr(l.c_str(), "\"stages\":");
    if (!p || !q || !r) continue;
    if (sscanf(p, "\"block_threads\": %d", &bt) != 1 || sscanf(q, "\"ctas_per_sm\": %d", &cps) != 1 ||
        sscanf(r, "\"stages\": %d", &st) != 1)
      continue;
    if (bt < 32 || bt > 256 || bt % 32 || cps < 0 || st < 0 || st > 4) continue;
    shape[0] = bt; shape[1] = cps; shape[2] = st;
    return true;
  }
  return false;
}

static void cache_store(const char* path, const std::string& key, const int shape[3], double us) {
  if (!path) return;
  std::vector<std::string> keep;
  for (const std::string& l : read_lines(path))
    if (l.find("\"key\":") != std::string::npos && l.find("\"key\": \"" + key + "\"") == std::string::npos) {
      std::string e = l;
      while (!e.empty() && (e.back() == ',' || e.back() == ' ')) e.pop_back();
      keep.push_back(e);
    }
  char buf[256];
  snprintf(buf, sizeof(buf),
           "  {\"key\": \"%s\", \"block_threads\": %d, \"ctas_per_sm\": %d, \"stages\": %d, \"us_per_iter\": %.3f}",
           key.c_str(), shape[0], shape[1], shape[2], us);
  keep.push_back(buf);
  std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "[\n");
  for (size_t k = 0; k < keep.size(); ++k) {
    std::string e = keep[k];
    size_t a = e.find('{');
    fprintf(f, "  %s%s\n", a == std::string::npos ? e.c_str() : e.c_str() + a, k + 1 < keep.size() ? "," : "");
  }
  fprintf(f, "]\n");
  fclose(f);
  rename(tmp.c_str(), path);
}

acopf_status acopf_autotune(acopf_handle h, const char* cache_path, int32_t iters, int32_t* shape_out,
                            double* us_per_iter) {
  Ctx* c = (Ctx*)h;
  if (!c || iters < 1) return fail(c, ACOPF_EINVAL, "acopf_autotune: bad arguments");
  const std::string key = tune_key(c);
  int best[3] = {c->block_threads, c->ctas_per_sm, c->sweep_stages};
  double best_us = -1.0;
  if (!cache_lookup(cache_path, key, best)) {
    acopf_status s = acopf_build_qp(h, 1.0, 2e4, c->use_angle);
    if (s) return s;
    admm_options a;
    admm_default_options(&a);
    bool prof = c->profiling;
    c->profiling = false;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int threads[5] = {64, 128, 192, 224, 256};
    // record access: in place (0), staged tiles (1, 2; FP32 sweep only), held
    // in registers (3); one thread-block cluster per instance (4)
    const int modes_mixed[5] = {0, 1, 2, 3, 4}, modes_fp64[3] = {0, 3, 4};
    const int* modes = c->precision == ACOPF_MIXED ? modes_mixed : modes_fp64;
    const int nmodes = c->precision == ACOPF_MIXED ? 5 : 3;
    for (int ti = 0; ti < 5; ++ti)
      for (int cps = 0; cps <= 1; ++cps)
        for (int mi = 0; mi < nmodes; ++mi) {
          const int st = modes[mi];
          c->block_threads = threads[ti];
          c->ctas_per_sm = cps;
          c->sweep_stages = st;
          launch_admm_reset(*c, 0);
          if ((s = launch_sweep(*c, a, iters > 4 ? iters / 4 : 1))) break;
          CK(cudaEventRecord(e0, c->stream));
          if ((s = launch_sweep(*c, a, iters))) break;
          CK(cudaEventRecord(e1, c->stream));
          if ((s = sweep_status(c))) break;
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          double us = 1e3 * ms / iters;
          if (best_us < 0 || us < best_us) {
            best_us = us;
            best[0] = threads[ti]; best[1] = cps; best[2] = st;
          }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->profiling = prof;
    launch_admm_reset(*c, 0);
    if (s) return s;
    cache_store(cache_path, key, best, best_us);
  }
  c->block_threads = best[0];
  c->ctas_per_sm = best[1];
  c->sweep_stages = best[2];
  drop_graph(c);
  if (shape_out) { shape_out[0] = best[0]; shape_out[1] = best[1]; shape_out[2] = best[2]; }
  if (us_per_iter) *us_per_iter = best_us;
  return ACOPF_OK;
}

acopf_status acopf_build_qp(acopf_handle h, double delta, double rho, int32_t use_angle) {
  Ctx* c = (Ctx*)h;
  if (!c || !(delta > 0) || !(rho > 0)) return fail(c, ACOPF_EINVAL, "acopf_build_qp: bad arguments");
  Dev& d = c->d;
  if (!d.xbr) {
    CK(dalloc(c, &d.xbr, 110 * (size_t)d.L));
    CK(dalloc(c, &d.xgen, 6 * (size_t)d.G));
    CK(dalloc(c, &d.xbus, 2 * (size_t)d.B));
  }
  sqp_options o;
  sqp_default_options(&o);
  o.delta0 = delta;
  o.admm.rho = rho;
  acopf_status s = reset_control(c, o, false);
  if (s) return s;
  c->use_angle = use_angle ? 1 : 0;
  launch_fill_rho(*c, rho);
  launch_build(*c, true);
  CK(cudaGetLastError());
  c->qp_built = true;
  return ACOPF_OK;
}

acopf_status admm_solve_qp(acopf_handle h, double delta, const admm_options* ao) {
  Ctx* c = (Ctx*)h;
  if (!c || !(delta > 0)) return fail(c, ACOPF_EINVAL, "admm_solve_qp: bad arguments");
  admm_options a;
  if (ao) a = *ao;
  else admm_default_options(&a);
  acopf_status s = check_admm(a, c);
  if (s) return s;
  if ((s = acopf_build_qp(h, delta, a.rho, c->use_angle))) return s;
  launch_admm_reset(*c, a.warm);
  if ((s = launch_sweep(*c, a, 0))) return s;
  if (a.rb_period > 0) launch_commit_rho(*c);
  launch_step(*c);
  if ((s = sweep_status(c))) return s;
  c->have_step = true;
  return ACOPF_OK;
}

acopf_status admm_iterate(acopf_handle h, int32_t n, const admm_options* ao) {
  Ctx* c = (Ctx*)h;
  if (!c || n < 1) return fail(c, ACOPF_EINVAL, "admm_iterate: n >= 1 required");
  if (!c->qp_built) return fail(c, ACOPF_ENOTREADY, "admm_iterate: no QP has been built");
  admm_options a;
  if (ao) a = *ao;
  else admm_default_options(&a);
  acopf_status s = check_admm(a, c);
  if (s) return s;
  if ((s = launch_sweep(*c, a, n))) return s;
  if (a.rb_period > 0) launch_commit_rho(*c);
  launch_step(*c);
  if ((s = sweep_status(c))) return s;
  c->have_step = true;
  return ACOPF_OK;
}

acopf_status acopf_get_qp(acopf_handle h, int32_t inst, acopf_qp_view* v) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst) || !v) return fail(c, ACOPF_EINVAL, "acopf_get_qp: bad arguments");
  Dev& d = c->d;
  if (!d.xbr) return fail(c, ACOPF_ENOTREADY, "acopf_get_qp: call acopf_build_qp first");
  CK(cudaStreamSynchronize(c->stream));
  int b0 = c->h_bus_off[inst], nb = c->h_bus_off[inst + 1] - b0;
  int l0 = c->h_br_off[inst], nl = c->h_br_off[inst + 1] - l0;
  int g0 = c->h_gen_off[inst], ng = c->h_gen_off[inst + 1] - g0;
  std::vector<double> br((size_t)110 * nl), gn((size_t)6 * ng), bu((size_t)2 * nb);
  if (nl) CK(cudaMemcpy(br.data(), d.xbr + (size_t)110 * l0, sizeof(double) * br.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(gn.data(), d.xgen + (size_t)6 * g0, sizeof(double) * gn.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(bu.data(), d.xbus + (size_t)2 * b0, sizeof(double) * bu.size(), cudaMemcpyDeviceToHost));
  struct F { double* dst; int off, n; } fs[] = {{v->flow, 0, 4}, {v->H, 4, 36}, {v->aR, 40, 4}, {v->aI, 44, 4},
                                                 {v->bR, 48, 1}, {v->bI, 49, 1}, {v->QH, 50, 16}, {v->gH, 66, 4},
                                                 {v->F, 70, 16}, {v->f0, 86, 4}, {v->lo, 90, 4}, {v->hi, 94, 4},
                                                 {v->G, 98, 8}, {v->grhs, 106, 2}, {v->alo, 108, 1}, {v->ahi, 109, 1}};
  for (auto& fld : fs) {
    if (!fld.dst) continue;
    for (int l = 0; l < nl; ++l)
      for (int k = 0; k < fld.n; ++k) fld.dst[(size_t)fld.n * l + k] = br[(size_t)110 * l + fld.off + k];
  }
  if (v->gen)
    for (int q = 0; q < ng; ++q) {
      int internal = c->h_gen_iperm[g0 + q] - g0;
      for (int k = 0; k < 6; ++k) v->gen[6 * q + k] = gn[6 * internal + k];
    }
  if (v->bus) memcpy(v->bus, bu.data(), sizeof(double) * bu.size());
  return ACOPF_OK;
}

acopf_status acopf_get_admm_state(acopf_handle h, int32_t inst, acopf_admm_state* s) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst) || !s) return fail(c, ACOPF_EINVAL, "acopf_get_admm_state: bad arguments");
  Dev& d = c->d;
  CK(cudaStreamSynchronize(c->stream));
  int b0 = c->h_bus_off[inst], nb = c->h_bus_off[inst + 1] - b0;
  int l0 = c->h_br_off[inst], nl = c->h_br_off[inst + 1] - l0;
  int g0 = c->h_gen_off[inst], ng = c->h_gen_off[inst + 1] - g0;
  acopf_status st;
  std::vector<double> tmp;
  double* outs[3] = {s->x, s->z, s->lam};
  void* srcs[3] = {d.X, d.Z, d.LAM};
  for (int a = 0; a < 3; ++a) {
    if (!outs[a]) continue;
    if ((st = fetch(c, srcs[a], (size_t)8 * nl, (size_t)8 * l0, tmp))) return st;
    for (int l = 0; l < nl; ++l)
      for (int sl = 0; sl < 8; ++sl) outs[a][8 * l + sl] = tmp[8 * l + 4 * kSlotEnd[sl] + kSlotComp[sl]];
  }
  double* gouts[3] = {s->xg, s->zg, s->lg};
  void* gsrcs[3] = {d.XG, d.ZG, d.LG};
  for (int a = 0; a < 3; ++a) {
    if (!gouts[a]) continue;
    if ((st = fetch(c, gsrcs[a], (size_t)2 * ng, (size_t)2 * g0, tmp))) return st;
    for (int q = 0; q < ng; ++q) {
      int internal = c->h_gen_iperm[g0 + q] - g0;
      gouts[a][2 * q] = tmp[2 * internal];
      gouts[a][2 * q + 1] = tmp[2 * internal + 1];
    }
  }
  if (s->zb) {
    if ((st = fetch(c, d.ZB, (size_t)2 * nb, (size_t)2 * b0, tmp))) return st;
    memcpy(s->zb, tmp.data(), sizeof(double) * 2 * nb);
  }
  if (s->nu) {
    if ((st = fetch(c, d.NU, (size_t)2 * nb, (size_t)2 * b0, tmp))) return st;
    memcpy(s->nu, tmp.data(), sizeof(double) * 2 * nb);
  }
  if (s->ul) {
    std::vector<double> sc;
    if ((st = fetch(c, d.U, (size_t)4 * nl, (size_t)4 * l0, tmp))) return st;
    if ((st = fetch(c, d.lrec, (size_t)4 * nl, (size_t)4 * (13 * (size_t)d.L + l0), sc))) return st;
    for (int l = 0; l < nl; ++l) {
      double n0 = sc[4 * l + 2], n1 = sc[4 * l + 3];
      s->ul[4 * l + 0] = n0 > 0 ? tmp[4 * l + 0] / n0 : 0.0;
      s->ul[4 * l + 1] = n1 > 0 ? tmp[4 * l + 1] / n1 : 0.0;
      s->ul[4 * l + 2] = tmp[4 * l + 2];
      s->ul[4 * l + 3] = tmp[4 * l + 3];
    }
  }
  return ACOPF_OK;
}

acopf_status acopf_set_admm_state(acopf_handle h, int32_t inst, const acopf_admm_state* s) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst) || !s) return fail(c, ACOPF_EINVAL, "acopf_set_admm_state: bad arguments");
  Dev& d = c->d;
  CK(cudaStreamSynchronize(c->stream));
  int b0 = c->h_bus_off[inst], nb = c->h_bus_off[inst + 1] - b0;
  int l0 = c->h_br_off[inst], nl = c->h_br_off[inst + 1] - l0;
  int g0 = c->h_gen_off[inst], ng = c->h_gen_off[inst + 1] - g0;
  acopf_status st;
  std::vector<double> tmp;
  const double* ins[3] = {s->x, s->z, s->lam};
  void* dsts[3] = {d.X, d.Z, d.LAM};
  for (int a = 0; a < 3; ++a) {
    if (!ins[a]) continue;
    tmp.assign((size_t)8 * nl, 0.0);
    for (int l = 0; l < nl; ++l)
      for (int sl = 0; sl < 8; ++sl) tmp[8 * l + 4 * kSlotEnd[sl] + kSlotComp[sl]] = ins[a][8 * l + sl];
    if ((st = put(c, dsts[a], tmp, (size_t)8 * l0))) return st;
  }
  const double* gins[3] = {s->xg, s->zg, s->lg};
  void* gdsts[3] = {d.XG, d.ZG, d.LG};
  for (int a = 0; a < 3; ++a) {
    if (!gins[a]) continue;
    tmp.assign((size_t)2 * ng, 0.0);
    for (int q = 0; q < ng; ++q) {
      int internal = c->h_gen_iperm[g0 + q] - g0;
      tmp[2 * internal] = gins[a][2 * q];
      tmp[2 * internal + 1] = gins[a][2 * q + 1];
    }
    if ((st = put(c, gdsts[a], tmp, (size_t)2 * g0))) return st;
  }
  if (s->zb) {
    tmp.assign(s->zb, s->zb + 2 * nb);
    if ((st = put(c, d.ZB, tmp, (size_t)2 * b0))) return st;
  }
  if (s->nu) {
    tmp.assign(s->nu, s->nu + 2 * nb);
    if ((st = put(c, d.NU, tmp, (size_t)2 * b0))) return st;
  }
  if (s->ul) {
    std::vector<double> sc;
    if ((st = fetch(c, d.lrec, (size_t)4 * nl, (size_t)4 * (13 * (size_t)d.L + l0), sc))) return st;
    tmp.assign((size_t)4 * nl, 0.0);
    for (int l = 0; l < nl; ++l) {
      tmp[4 * l + 0] = s->ul[4 * l + 0] * sc[4 * l + 2];
      tmp[4 * l + 1] = s->ul[4 * l + 1] * sc[4 * l + 3];
      tmp[4 * l + 2] = s->ul[4 * l + 2];
      tmp[4 * l + 3] = s->ul[4 * l + 3];
    }
    if ((st = put(c, d.U, tmp, (size_t)4 * l0))) return st;
  }
  return ACOPF_OK;
}

acopf_status acopf_get_step(acopf_handle h, int32_t inst, double* dx, double* pi) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst)) return fail(c, ACOPF_EINVAL, "acopf_get_step: bad arguments");
  if (!c->have_step) return fail(c, ACOPF_ENOTREADY, "acopf_get_step: no QP has been solved");
  Dev& d = c->d;
  CK(cudaStreamSynchronize(c->stream));
  int b0 = c->h_bus_off[inst], nb = c->h_bus_off[inst + 1] - b0;
  int l0 = c->h_br_off[inst], nl = c->h_br_off[inst + 1] - l0;
  int g0 = c->h_gen_off[inst], ng = c->h_gen_off[inst + 1] - g0;
  if (dx) {
    std::vector<double> pg(ng), qg(ng);
    CK(cudaMemcpy(pg.data(), d.dpg + g0, sizeof(double) * ng, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(qg.data(), d.dqg + g0, sizeof(double) * ng, cudaMemcpyDeviceToHost));
    for (int q = 0; q < ng; ++q) {
      int internal = c->h_gen_iperm[g0 + q] - g0;
      dx[q] = pg[internal];
      dx[ng + q] = qg[internal];
    }
    double* w = dx + 2 * ng;
    CK(cudaMemcpy(w, d.dw + b0, sizeof(double) * nb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(w + nb, d.dth + b0, sizeof(double) * nb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(w + 2 * nb, d.dwr + l0, sizeof(double) * nl, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(w + 2 * nb + nl, d.dwi + l0, sizeof(double) * nl, cudaMemcpyDeviceToHost));
  }
  if (pi) {
    std::vector<double> col(nl);
    for (int r = 0; r < 4; ++r) {
      CK(cudaMemcpy(col.data(), d.pi_new + (size_t)r * d.L + l0, sizeof(double) * nl, cudaMemcpyDeviceToHost));
      for (int l = 0; l < nl; ++l) pi[4 * l + r] = col[l];
    }
  }
  return ACOPF_OK;
}

acopf_status acopf_get_solution(acopf_handle h, int32_t inst, acopf_solution* out) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst) || !out) return fail(c, ACOPF_EINVAL, "acopf_get_solution: bad arguments");
  int nb = c->h_bus_off[inst + 1] - c->h_bus_off[inst];
  int nl = c->h_br_off[inst + 1] - c->h_br_off[inst];
  int ng = c->h_gen_off[inst + 1] - c->h_gen_off[inst];
  std::vector<double> x(2 * (size_t)ng + 2 * (size_t)nb + 2 * (size_t)nl);
  acopf_status s = acopf_get_iterate(h, inst, x.data(), nullptr);
  if (s) return s;
  const double* v = x.data();
  if (out->pg) memcpy(out->pg, v, sizeof(double) * ng);
  if (out->qg) memcpy(out->qg, v + ng, sizeof(double) * ng);
  const double* w = v + 2 * ng;
  if (out->vm)
    for (int i = 0; i < nb; ++i) out->vm[i] = sqrt(w[i] > 0 ? w[i] : 0.0);
  if (out->va) memcpy(out->va, w + nb, sizeof(double) * nb);
  if (out->wr) memcpy(out->wr, w + 2 * nb, sizeof(double) * nl);
  if (out->wi) memcpy(out->wi, w + 2 * nb + nl, sizeof(double) * nl);
  InstCtl q;
  CK(cudaMemcpy(&q, c->d.ctl + inst, sizeof(q), cudaMemcpyDeviceToHost));
  out->obj = q.obj;
  return ACOPF_OK;
}

acopf_status acopf_get_residuals(acopf_handle h, int32_t inst, acopf_residuals* out) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst) || !out) return fail(c, ACOPF_EINVAL, "acopf_get_residuals: bad arguments");
  CK(cudaStreamSynchronize(c->stream));
  InstCtl q;
  CK(cudaMemcpy(&q, c->d.ctl + inst, sizeof(q), cudaMemcpyDeviceToHost));
  int iters = 0;
  double rs[2] = {0, 0};
  CK(cudaMemcpy(&iters, c->d.admm_iters + inst, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&rs[0], c->d.admm_rs + inst, sizeof(double), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&rs[1], c->d.admm_rs + c->d.K + inst, sizeof(double), cudaMemcpyDeviceToHost));
  out->primal = q.primal;
  out->dual = q.dual;
  out->r_inf = rs[0];
  out->s_inf = rs[1];
  out->obj = q.obj;
  out->delta = q.delta;
  out->sqp_iter = q.sqp_iter;
  out->admm_iter = q.sqp_iter > 0 ? q.admm_iter_total : iters;
  out->accepted = q.accepted;
  out->result = q.result;
  return ACOPF_OK;
}

acopf_status acopf_get_history(acopf_handle h, int32_t inst, double* out, int32_t cap, int32_t* n) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst) || cap < 0 || (cap > 0 && !out)) return fail(c, ACOPF_EINVAL, "acopf_get_history: bad arguments");
  CK(cudaStreamSynchronize(c->stream));
  InstCtl q;
  CK(cudaMemcpy(&q, c->d.ctl + inst, sizeof(q), cudaMemcpyDeviceToHost));
  int rows = q.sqp_iter < ACOPF_HIST_MAX ? q.sqp_iter : ACOPF_HIST_MAX;
  int k = rows < cap ? rows : cap;
  if (k > 0)
    CK(cudaMemcpy(out, c->d.hist + (size_t)inst * ACOPF_HIST_MAX * kHistW, sizeof(double) * kHistW * k,
                  cudaMemcpyDeviceToHost));
  if (n) *n = q.sqp_iter;
  return ACOPF_OK;
}

acopf_status acopf_set_warm_start(acopf_handle h, int32_t inst, const double* x0, const double* lambda0,
                                  const double* rho) {
  Ctx* c = (Ctx*)h;
  if (!c || !inst_ok(c, inst)) return fail(c, ACOPF_EINVAL, "acopf_set_warm_start: bad arguments");
  acopf_status s;
  if (x0) {
    if ((s = acopf_set_iterate(h, inst, x0, nullptr))) return s;
    int l0 = c->h_br_off[inst], nl = c->h_br_off[inst + 1] - l0;
    for (int r = 0; r < 4; ++r) CK(cudaMemset(c->d.pi + (size_t)r * c->d.L + l0, 0, sizeof(double) * nl));
    c->warm_x = true;
  }
  if (lambda0) {
    int nl = c->h_br_off[inst + 1] - c->h_br_off[inst];
    acopf_admm_state st;
    memset(&st, 0, sizeof(st));
    st.lam = (double*)lambda0;
    st.lg = (double*)(lambda0 + 8 * (size_t)nl);
    if ((s = acopf_set_admm_state(h, inst, &st))) return s;
    c->warm_lam = true;
  }
  if (rho) {
    int l0 = c->h_br_off[inst], nl = c->h_br_off[inst + 1] - l0;
    int g0 = c->h_gen_off[inst], ng = c->h_gen_off[inst + 1] - g0;
    for (int l = 0; l < nl; ++l)
      if (!(rho[l] > 0)) return fail(c, ACOPF_EINVAL, "acopf_set_warm_start: rho must be positive");
    CK(cudaMemcpy(c->d.rho_l + l0, rho, sizeof(double) * nl, cudaMemcpyHostToDevice));
    std::vector<double> rg(ng);
    for (int q = 0; q < ng; ++q) {
      if (!(rho[nl + q] > 0)) return fail(c, ACOPF_EINVAL, "acopf_set_warm_start: rho must be positive");
      rg[c->h_gen_iperm[g0 + q] - g0] = rho[nl + q];
    }
    CK(cudaMemcpy(c->d.rho_g + g0, rg.data(), sizeof(double) * ng, cudaMemcpyHostToDevice));
    c->warm_rho = true;
  }
  return ACOPF_OK;
}

acopf_status acopf_set_warm_start_device(acopf_handle h, const float* pred, int64_t ld, double base_rho,
                                         int32_t use_x, int32_t use_pi, int32_t use_lambda, int32_t use_rho) {
  Ctx* c = (Ctx*)h;
  if (!c || !pred || (use_rho && !(base_rho > 0)) || (use_pi && !use_x))
    return fail(c, ACOPF_EINVAL, "acopf_set_warm_start_device: bad arguments");
  const int K = c->d.K;
  const int nb = c->h_bus_off[1] - c->h_bus_off[0];
  const int nl = c->h_br_off[1] - c->h_br_off[0];
  const int ng = c->h_gen_off[1] - c->h_gen_off[0];
  for (int k = 1; k < K; ++k)
    if (c->h_bus_off[k + 1] - c->h_bus_off[k] != nb || c->h_br_off[k + 1] - c->h_br_off[k] != nl ||
        c->h_gen_off[k + 1] - c->h_gen_off[k] != ng)
      return fail(c, ACOPF_EINVAL, "acopf_set_warm_start_device: instances of different sizes");
  const int64_t width = 5LL * ng + 2LL * nb + 15LL * nl;
  if (ld < width) return fail(c, ACOPF_EINVAL, "acopf_set_warm_start_device: ld below the row width 5G + 2B + 15L");
  if (!c->d_gen_iperm) {
    CK(dalloc(c, &c->d_gen_iperm, (size_t)c->d.G));
    CK(upload(c, c->d_gen_iperm, c->h_gen_iperm, (size_t)c->d.G));
  }
  launch_warm_scatter(*c, pred, ld, nb, nl, ng, base_rho, use_x, use_pi, use_lambda, use_rho);
  CK(cudaGetLastError());
  if (use_x) c->warm_x = true;
  if (use_lambda) c->warm_lam = true;
  if (use_rho) c->warm_rho = true;
  return ACOPF_OK;
}

acopf_status acopf_project_linear(acopf_handle h, double rho, double eps, int32_t max_iter, int32_t* iters,
                                  double* rs) {
  Ctx* c = (Ctx*)h;
  if (!c || !(rho > 0) || !(eps > 0) || max_iter < 1)
    return fail(c, ACOPF_EINVAL, "acopf_project_linear: rho > 0, eps > 0, max_iter >= 1 required");
  acopf_status s = project_linear(*c, rho, eps, max_iter, 25, iters, rs);
  if (s) return s;
  c->warm_x = true;  // the next sqp_solve starts from the projected point
  return ACOPF_OK;
}

}  // extern "C"
