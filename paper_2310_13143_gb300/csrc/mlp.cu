// The learned warm start's network on the fifth-generation tensor cores.
//
// A multilayer perceptron (GELU hidden layers, affine output) maps a load
// scenario's per-bus (pd, qd) to an ADMM starting point, multipliers and
// per-component penalties.  Every matrix product of its forward and backward
// passes is one kernel, k_gemm_tc:
//
//   C[M x N] = A[M x K] * B[N x K]^T,   A, B bfloat16, K contiguous,
//
// with 128 x 256 output tiles in a persistent, warp-specialised kernel: one
// CTA per SM loops over tiles; warp 0 streams 128 x 64 and 256 x 64 operand
// tiles into a four-stage shared-memory ring with TMA (cp.async.bulk.tensor,
// 128-byte swizzle, completion counted on mbarriers); warp 1 issues
// tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, 128 x 256 x 16) into one of two
// 256-column tensor-memory accumulators; warps 2-5 read the other accumulator
// back with tcgen05.ld for a fused epilogue (bias, GELU, GELU derivative,
// bfloat16 row-major and transposed stores), so the epilogue of one tile
// overlaps the main loop of the next.  Long contractions are split over K
// into FP32 partial tiles summed by k_splitk.
//
// Layout convention: the backward pass needs every operand with its
// contraction index contiguous, so the forward epilogue stores each hidden
// activation both row-major and transposed, the backward epilogue does the
// same for each pre-activation gradient, and the Adam kernel keeps each
// weight both as [out x in] and as [in x out].  Every product is then the
// K-major x K-major form above.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/acopf.h"
#include "../../include/acopf_mlp.h"

namespace acopf {
namespace nn {

typedef __nv_bfloat16 bf16;

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr uint32_t kABytes = BM * BK * 2;  // A tile: 128 rows x 128 bytes
constexpr uint32_t kBBytes = BN * BK * 2;  // B tile: 256 rows x 128 bytes
constexpr int kGemmThreads = 192;          // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr size_t kGemmSmem = 1024 + (size_t)STAGES * (kABytes + kBBytes) + 256;
constexpr uint32_t kTmemCols = 512;        // two 256-column FP32 accumulators

// Instruction descriptor of tcgen05.mma kind::f16: D in FP32 (bits 4-5 = 1),
// A and B bfloat16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

enum { EPI_F32 = 0, EPI_GELU = 1, EPI_GELU_BWD = 2, EPI_PARTIAL = 3 };

struct Epi {
  int op;
  int M, N;             // output extent
  int rows_valid;       // bf16 outputs of rows >= rows_valid are written as 0
  const float* bias;    // [N] or null
  float* f32;           // FP32 row-major output (EPI_F32, EPI_PARTIAL; EPI_GELU: the pre-activation)
  int ld_f32;
  size_t split_stride;  // EPI_PARTIAL: elements between the partial tiles of consecutive K splits
  bf16* bf;             // bfloat16 row-major output
  int ld_bf;
  bf16* bt;             // bfloat16 transposed output: (m, n) at bt[n * ld_bt + m]
  int ld_bt;
  const float* z;       // EPI_GELU_BWD: saved pre-activation
  int ld_z;
};

// --------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long long limit) {
  long long t0 = clock64();
  while (!mbar_test(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          saddr(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}
// shared-memory matrix descriptor: K-major operand tile of 128-byte rows with
// the 128-byte swizzle, 8-row groups 1024 bytes apart (stride byte offset),
// descriptor version 1 (bit 46), swizzle mode 2 (bits 61-63)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ epilogue
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void epi_one(const Epi& e, int m, int n, float acc, int split) {
  if (m >= e.M || n >= e.N) return;
  switch (e.op) {
    case EPI_F32: {
      e.f32[(size_t)m * e.ld_f32 + n] = acc + (e.bias ? e.bias[n] : 0.0f);
      break;
    }
    case EPI_GELU: {
      float zz = acc + e.bias[n];
      e.f32[(size_t)m * e.ld_f32 + n] = zz;
      bf16 h = __float2bfloat16_rn(m < e.rows_valid ? gelu_f(zz) : 0.0f);
      e.bf[(size_t)m * e.ld_bf + n] = h;
      e.bt[(size_t)n * e.ld_bt + m] = h;
      break;
    }
    case EPI_GELU_BWD: {
      float v = m < e.rows_valid ? acc * gelu_grad_f(e.z[(size_t)m * e.ld_z + n]) : 0.0f;
      bf16 h = __float2bfloat16_rn(v);
      e.bf[(size_t)m * e.ld_bf + n] = h;
      e.bt[(size_t)n * e.ld_bt + m] = h;
      break;
    }
    default:  // EPI_PARTIAL
      e.f32[(size_t)split * e.split_stride + (size_t)m * e.ld_f32 + n] = acc;
      break;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

// 16 consecutive accumulator columns [n, n + 16) of row m: vector stores when
// the whole group is in range, the per-element epilogue otherwise
__device__ __forceinline__ void epi_store16(const Epi& e, int m, int n, const float v[16], int split) {
  if (m >= e.M) return;
  if (n + 16 > e.N) {
#pragma unroll
    for (int j = 0; j < 16; ++j) epi_one(e, m, n + j, v[j], split);
    return;
  }
  switch (e.op) {
    case EPI_F32:
    case EPI_PARTIAL: {
      float* dst = e.op == EPI_PARTIAL ? e.f32 + (size_t)split * e.split_stride + (size_t)m * e.ld_f32 + n
                                       : e.f32 + (size_t)m * e.ld_f32 + n;
      float w[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        w[j] = v[j] + (e.op == EPI_F32 && e.bias ? e.bias[n + j] : 0.0f);
      }
      if (((uintptr_t)dst & 15) == 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 4) *(float4*)(dst + j) = make_float4(w[j], w[j + 1], w[j + 2], w[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) dst[j] = w[j];
      }
      break;
    }
    case EPI_GELU:
    case EPI_GELU_BWD: {
      bf16 h[16];
      if (e.op == EPI_GELU) {
        float* zd = e.f32 + (size_t)m * e.ld_f32 + n;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float zz = v[j] + e.bias[n + j];
          zd[j] = zz;
          h[j] = __float2bfloat16_rn(m < e.rows_valid ? gelu_f(zz) : 0.0f);
        }
      } else {
        const float* zs = e.z + (size_t)m * e.ld_z + n;
#pragma unroll
        for (int j = 0; j < 16; ++j) h[j] = __float2bfloat16_rn(m < e.rows_valid ? v[j] * gelu_grad_f(zs[j]) : 0.0f);
      }
      bf16* dst = e.bf + (size_t)m * e.ld_bf + n;
      if (((uintptr_t)dst & 15) == 0) {
        *(uint4*)dst = *(const uint4*)&h[0];
        *(uint4*)(dst + 8) = *(const uint4*)&h[8];
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) dst[j] = h[j];
      }
      // transposed: lanes hold consecutive rows, so each column's stores coalesce
#pragma unroll
      for (int j = 0; j < 16; ++j) e.bt[(size_t)(n + j) * e.ld_bt + m] = h[j];
      break;
    }
  }
}

// work item w -> (split z, row block mb, column block nb).  Within a split,
// items run through groups of kGroup row blocks, column-block-major inside a
// group, so the tiles in flight at one time share a few A and B blocks in L2.
constexpr int kGroup = 16;
__device__ __forceinline__ void decode_item(int w, int mt, int nt, int& z, int& mb, int& nb) {
  z = w / (mt * nt);
  const int r = w - z * mt * nt;
  const int g = r / (kGroup * nt);
  const int g0 = g * kGroup;
  const int gm = mt - g0 < kGroup ? mt - g0 : kGroup;  // row blocks in this group
  const int rr = r - g0 * nt;
  mb = g0 + rr % gm;
  nb = rr / gm;
}

// -------------------------------------------------------------- GEMM kernel
// Persistent: grid = min(work items, SMs), 192 threads, kGemmSmem bytes of
// dynamic shared memory.  Work item w = (split z, row block, column block);
// split z covers K tiles [z * kts, (z + 1) * kts).  Every wait is bounded:
// on time-out the waiting role records *err and stops.
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int K, int kts,
              int splits, Epi e, int* err, long long spin) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * kABytes;
  uint64_t* full = (uint64_t*)(smem + STAGES * (kABytes + kBBytes));
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;  // accumulator a holds a finished tile
  uint64_t* tempty = tfull + 2;      // accumulator a has been read by the epilogue
  uint32_t* tslot = (uint32_t*)(tempty + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = (e.M + BM - 1) / BM, nt = (e.N + BN - 1) / BN;
  const int items = splits * mt * nt;
  const int kt_total = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {  // producer: operand tiles into the ring of stages
      int i = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < items && ok; w += gridDim.x) {
        int z, mb, nb;
        decode_item(w, mt, nt, z, mb, nb);
        const int kt0 = z * kts, kt1 = kt0 + kts < kt_total ? kt0 + kts : kt_total;
        for (int kt = kt0; kt < kt1; ++kt, ++i) {
          const int s = i % STAGES;
          if (i >= STAGES && !mbar_wait(&empty[s], ((i / STAGES) - 1) & 1, spin)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], kABytes + kBBytes);
          tma_load_2d(sA + s * kABytes, &ta, kt * BK, mb * BM, &full[s]);
          tma_load_2d(sB + s * kBBytes, &tb, kt * BK, nb * BN, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int i = 0, j = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < items && ok; w += gridDim.x, ++j) {
        const int z = w / (mt * nt);  // the MMA issuer only needs the split
        const int kt0 = z * kts, kt1 = kt0 + kts < kt_total ? kt0 + kts : kt_total;
        const int a = j & 1, u = j >> 1;
        if (u >= 1 && !mbar_wait(&tempty[a], (u - 1) & 1, spin)) {
          atomicExch(err, 1);
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(a * BN);
        for (int kt = kt0; kt < kt1; ++kt, ++i) {
          const int s = i % STAGES;
          if (!mbar_wait(&full[s], (i / STAGES) & 1, spin)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t pa = saddr(sA + s * kABytes), pb = saddr(sB + s * kBBytes);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_bf16(acc, sdesc(pa + 32 * kk), sdesc(pb + 32 * kk), (kt > kt0 || kk > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        if (kt1 > kt0) mma_commit(&tfull[a]);  // arrives when this tile's MMAs are done
        else mbar_arrive(&tfull[a]);            // empty K range: nothing to wait for
      }
    }
  } else {
    // epilogue: warp w reads accumulator lanes (rows) 32 (w % 4) .. + 31
    const int q = warp & 3;
    int j = 0;
    for (int w = blockIdx.x; w < items; w += gridDim.x, ++j) {
      int z, mb, nb;
        decode_item(w, mt, nt, z, mb, nb);
      const int kt0 = z * kts, kt1 = kt0 + kts < kt_total ? kt0 + kts : kt_total;
      const int a = j & 1, u = j >> 1;
      bool ok = mbar_wait(&tfull[a], u & 1, spin);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      tc_fence_after();
      const int row = mb * BM + q * 32 + lane;
      const int n0 = nb * BN;
      for (int c = 0; c < BN; c += 16) {
        if (n0 + c >= e.N) break;
        float v[16];
        if (kt1 > kt0) {
          tmem_ld16(tmem + (uint32_t)(a * BN) + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
        } else {
#pragma unroll
          for (int t = 0; t < 16; ++t) v[t] = 0.0f;
        }
        epi_store16(e, row, n0 + c, v, z);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[a]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// sum of the K-split partial tiles, then the epilogue
__global__ void k_splitk(const float* ws, int splits, size_t stride, Epi e) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)e.M * e.N;
  if (i >= total) return;
  int m = (int)(i / e.N), n = (int)(i % e.N);
  float acc = 0.0f;
  for (int z = 0; z < splits; ++z) acc += ws[(size_t)z * stride + i];
  epi_one(e, m, n, acc, 0);
}

// --------------------------------------------------------- other kernels
// layer-0 input: rows idx[r] of the raw data X (ld = d0), standardised,
// rounded to bfloat16, stored row-major and transposed; rows >= rows are 0
__global__ void k_input(const float* X, const int* idx, int rows, int Mb, int d0, const float* mu, const float* sd,
                        bf16* A, bf16* AT) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)Mb * d0) return;
  int r = (int)(i / d0), j = (int)(i % d0);
  float v = 0.0f;
  if (r < rows) {
    size_t src = idx ? (size_t)idx[r] : (size_t)r;
    v = (X[src * d0 + j] - mu[j]) / sd[j];
  }
  bf16 h = __float2bfloat16_rn(v);
  A[i] = h;
  AT[(size_t)j * Mb + r] = h;
}

// mean squared error against standardised targets: dY = 2 (Y - T) / (rows * N)
// in bfloat16, row-major and transposed (32 x 32 tiles transposed through
// shared memory so both stores coalesce), one sum of squares per block.
// Grid (ceil(N / 32), Mb / 32), block 32 x 8.
__global__ void k_mse(const float* Y, const float* T, const int* idx, int rows, int Mb, int N, const float* mu,
                      const float* sd, bf16* D, bf16* DT, double* part) {
  __shared__ bf16 tile[32][34];
  __shared__ double red[256];
  const int n = blockIdx.x * 32 + threadIdx.x;
  const int r0 = blockIdx.y * 32;
  double sq = 0.0;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = r0 + k;
    float g = 0.0f;
    if (n < N && r < rows) {
      const size_t src = idx ? (size_t)idx[r] : (size_t)r;
      const float t = (T[src * N + n] - mu[n]) / sd[n];
      const float d = Y[(size_t)r * N + n] - t;
      sq += (double)d * (double)d;
      g = 2.0f * d / ((float)rows * (float)N);
    }
    const bf16 h = __float2bfloat16_rn(g);
    if (n < N) D[(size_t)r * N + n] = h;
    tile[k][threadIdx.x] = h;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int nn = blockIdx.x * 32 + k;
    if (nn < N) DT[(size_t)nn * Mb + r0 + threadIdx.x] = tile[threadIdx.x][k];
  }
  const int t = threadIdx.y * 32 + threadIdx.x;
  red[t] = sq;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (t < st) red[t] += red[t + st];
    __syncthreads();
  }
  if (t == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// sum of n partial sums in a fixed order (strided per thread, then a tree);
// one block of 1024 threads
__global__ void k_sum(const double* part, int n, double scale, float* out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (float)(red[0] * scale);
}

// column sums of a bfloat16 matrix [rows x N] (bias gradients), fixed order
__global__ void k_colsum(const bf16* D, int rows, int N, float* out) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int r = 0; r < rows; ++r) s += __bfloat162float(D[(size_t)r * N + n]);
  out[n] = s;
}

// Adam (bias-corrected) on FP32 master weights W [out x in] with gradient G;
// writes the bfloat16 copies W16 [out x in] and W16T [in x out] (32 x 32
// tiles transposed through shared memory)
__global__ void k_adam_w(float* W, const float* G, float* Mm, float* Vv, int out, int in, float lr, float b1, float b2,
                         float eps, float c1, float c2, bf16* W16, bf16* W16T) {
  __shared__ bf16 tile[32][33];
  int j = blockIdx.x * 32 + threadIdx.x;  // in
  int i0 = blockIdx.y * 32;               // out
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int i = i0 + k;
    bf16 h = __float2bfloat16_rn(0.0f);
    if (i < out && j < in) {
      size_t p = (size_t)i * in + j;
      float g = G[p];
      float m = b1 * Mm[p] + (1.0f - b1) * g;
      float v = b2 * Vv[p] + (1.0f - b2) * g * g;
      Mm[p] = m;
      Vv[p] = v;
      float w = W[p] - lr * (m / c1) / (sqrtf(v / c2) + eps);
      W[p] = w;
      h = __float2bfloat16_rn(w);
      W16[p] = h;
    }
    tile[k][threadIdx.x] = h;
  }
  __syncthreads();
  int i = i0 + threadIdx.x;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int jj = blockIdx.x * 32 + k;
    if (i < out && jj < in) W16T[(size_t)jj * out + i] = tile[threadIdx.x][k];
  }
}

__global__ void k_adam_b(float* b, const float* G, float* Mm, float* Vv, int n, float lr, float b1, float b2, float eps,
                         float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float g = G[i];
  float m = b1 * Mm[i] + (1.0f - b1) * g;
  float v = b2 * Vv[i] + (1.0f - b2) * g * g;
  Mm[i] = m;
  Vv[i] = v;
  b[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// de-standardised network outputs: out = y sd + mu (y row-major, N columns)
__global__ void k_destd(const float* Y, float* out, size_t total, int N, const float* mu, const float* sd) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int n = (int)(i % N);
  out[i] = Y[i] * sd[n] + mu[n];
}

// bfloat16 copies of FP32 weights (after set_params)
__global__ void k_w16(const float* W, int out, int in, bf16* W16, bf16* W16T) {
  size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (size_t)out * in) return;
  int i = (int)(p / in), j = (int)(p % in);
  bf16 h = __float2bfloat16_rn(W[p]);
  W16[p] = h;
  W16T[(size_t)j * out + i] = h;
}

// column means and population deviations (FP64 accumulation); a column whose
// deviation is at most 1e-12 (1 + |mean|) gets deviation 1
__global__ void k_standardiser(const float* X, int rows, int N, float* mu, float* sd) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s = 0.0;
  for (int r = 0; r < rows; ++r) s += (double)X[(size_t)r * N + n];
  double m = s / rows;
  double q = 0.0;
  for (int r = 0; r < rows; ++r) {
    double d = (double)X[(size_t)r * N + n] - m;
    q += d * d;
  }
  double dev = sqrt(q / rows);
  if (dev <= 1e-12 * (1.0 + fabs(m))) dev = 1.0;
  mu[n] = (float)m;
  sd[n] = (float)dev;
}

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool encode_fn() {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return true;
}

// 2-D bfloat16 operand [rows x cols], row stride ld elements; boxes of box_rows rows x 64 columns
static bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows) {
  if (!encode_fn()) return false;
  if (((uintptr_t)base & 15) || (ld * 2) % 16 || rows < 1 || cols < 1) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

struct Gemm {
  CUtensorMap ta, tb;
  int M, N, K, splits, kts;
  Epi e;
};

static int g_smem_set = -1;

static cudaError_t run_gemm(const Gemm& g, float* ws, int* err, cudaStream_t st, long long spin, int sms) {
  if (g_smem_set < 0) {
    cudaError_t c = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
    if (c != cudaSuccess) return c;
    g_smem_set = 1;
  }
  const int items = g.splits * ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
  const int grid = items < sms ? items : sms;
  if (g.splits == 1) {
    k_gemm_tc<<<grid, kGemmThreads, kGemmSmem, st>>>(g.ta, g.tb, g.K, g.kts, 1, g.e, err, spin);
    return cudaGetLastError();
  }
  Epi p = g.e;
  p.op = EPI_PARTIAL;
  p.f32 = ws;
  p.ld_f32 = g.N;
  p.split_stride = (size_t)g.M * g.N;
  k_gemm_tc<<<grid, kGemmThreads, kGemmSmem, st>>>(g.ta, g.tb, g.K, g.kts, g.splits, p, err, spin);
  size_t total = (size_t)g.M * g.N;
  k_splitk<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(ws, g.splits, p.split_stride, g.e);
  return cudaGetLastError();
}

// K split so that the grid covers the GPU's SMs about once
static void plan_split(Gemm& g, int sms) {
  int tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
  int kt = (g.K + BK - 1) / BK;
  int s = 1;
  while (tiles * s * 2 <= sms && kt / (s * 2) >= 4) s *= 2;
  g.kts = (kt + s - 1) / s;
  g.splits = (kt + g.kts - 1) / g.kts;
}

static size_t ws_need(const Gemm& g) { return g.splits > 1 ? (size_t)g.splits * g.M * g.N : 0; }

// --------------------------------------------------------------- the network
struct Layer {
  int in, out;
  float *W, *b, *mW, *vW, *mb, *vb, *gW, *gb;
  bf16 *W16, *W16T;
};

struct Net {
  int device = 0;
  int nl = 0;
  std::vector<int> dims;
  int Mb = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  std::vector<Layer> L;
  // activations: A[l] / AT[l] layer inputs (l = 0..nl-1), Z[l] pre-activations of hidden layer l (1..nl-1)
  std::vector<bf16*> A, AT;
  std::vector<float*> Z;
  float* Y = nullptr;
  // gradients of layer outputs: D[l] / DT[l], l = 1..nl (D[nl] = dL/dY)
  std::vector<bf16*> D, DT;
  float *mu_x = nullptr, *sd_x = nullptr, *mu_y = nullptr, *sd_y = nullptr;
  float* ws = nullptr;
  size_t ws_elems = 0;
  double* part = nullptr;
  int nparts = 0;
  int* err = nullptr;
  float* loss = nullptr;
  int step = 0;
  std::vector<Gemm> fwd, bwd_w, bwd_x;  // fwd[l], bwd_w[l] (dW_l), bwd_x[l] (dA_l, l >= 1)
  std::vector<void*> allocs;
  std::string last_error;
  long long spin = 1ll << 32;
};

template <typename T>
static bool dalloc(Net* n, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) return false;
  cudaMemset(q, 0, count * sizeof(T) + 16);
  n->allocs.push_back(q);
  *p = (T*)q;
  return true;
}

static void free_net(Net* n) {
  for (void* p : n->allocs) cudaFree(p);
  n->allocs.clear();
}

static acopf_status nfail(Net* n, acopf_status s, const std::string& m) {
  if (n) n->last_error = m;
  return s;
}

static bool plan(Net* n) {
  const int nl = n->nl, Mb = n->Mb;
  n->fwd.assign(nl, Gemm{});
  n->bwd_w.assign(nl, Gemm{});
  n->bwd_x.assign(nl, Gemm{});
  size_t ws = 0;
  for (int l = 0; l < nl; ++l) {
    const int in = n->dims[l], out = n->dims[l + 1];
    Layer& y = n->L[l];
    // forward: [Mb x in] * W[out x in]^T
    Gemm& f = n->fwd[l];
    f.M = Mb; f.N = out; f.K = in;
    if (!make_map(&f.ta, n->A[l], Mb, in, in, BM) || !make_map(&f.tb, y.W16, out, in, in, BN)) return false;
    memset(&f.e, 0, sizeof(Epi));
    f.e.M = Mb; f.e.N = out; f.e.rows_valid = Mb; f.e.bias = y.b;
    if (l < nl - 1) {
      f.e.op = EPI_GELU;
      f.e.f32 = n->Z[l + 1]; f.e.ld_f32 = out;
      f.e.bf = n->A[l + 1]; f.e.ld_bf = out;
      f.e.bt = n->AT[l + 1]; f.e.ld_bt = Mb;
    } else {
      f.e.op = EPI_F32;
      f.e.f32 = n->Y; f.e.ld_f32 = out;
    }
    plan_split(f, n->sms);
    ws = ws > ws_need(f) ? ws : ws_need(f);
    // weight gradient: dW = D^T [out x Mb] * (A^T [in x Mb])^T
    Gemm& w = n->bwd_w[l];
    w.M = out; w.N = in; w.K = Mb;
    if (!make_map(&w.ta, n->DT[l + 1], out, Mb, Mb, BM) || !make_map(&w.tb, n->AT[l], in, Mb, Mb, BN)) return false;
    memset(&w.e, 0, sizeof(Epi));
    w.e.op = EPI_F32; w.e.M = out; w.e.N = in; w.e.rows_valid = out;
    w.e.f32 = y.gW; w.e.ld_f32 = in;
    plan_split(w, n->sms);
    ws = ws > ws_need(w) ? ws : ws_need(w);
    if (l >= 1) {
      // input gradient: D_l = (D_{l+1} [Mb x out] * (W16T [in x out])^T) * GELU'(Z_l)
      Gemm& x = n->bwd_x[l];
      x.M = Mb; x.N = in; x.K = out;
      if (!make_map(&x.ta, n->D[l + 1], Mb, out, out, BM) || !make_map(&x.tb, y.W16T, in, out, out, BN)) return false;
      memset(&x.e, 0, sizeof(Epi));
      x.e.op = EPI_GELU_BWD; x.e.M = Mb; x.e.N = in; x.e.rows_valid = Mb;
      x.e.z = n->Z[l]; x.e.ld_z = in;
      x.e.bf = n->D[l]; x.e.ld_bf = in;
      x.e.bt = n->DT[l]; x.e.ld_bt = Mb;
      plan_split(x, n->sms);
      ws = ws > ws_need(x) ? ws : ws_need(x);
    }
  }
  n->ws_elems = ws;
  return ws == 0 || dalloc(n, &n->ws, ws);
}

static acopf_status check_err(Net* n) {
  int e = 0;
  if (cudaMemcpyAsync(&e, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess)
    return nfail(n, ACOPF_ECUDA, std::string("cuda: ") + cudaGetErrorString(cudaGetLastError()));
  if (e) {
    cudaMemsetAsync(n->err, 0, sizeof(int), n->stream);
    return nfail(n, ACOPF_ETIMEOUT, "tensor-core GEMM: a pipeline wait ran out");
  }
  return ACOPF_OK;
}

#define NCK(x)                                                                          \
  do {                                                                                  \
    cudaError_t _e = (x);                                                               \
    if (_e != cudaSuccess) return nfail(n, ACOPF_ECUDA, std::string("cuda: ") + cudaGetErrorString(_e)); \
  } while (0)

static acopf_status forward(Net* n, int rows) {
  for (int l = 0; l < n->nl; ++l) {
    Gemm g = n->fwd[l];
    g.e.rows_valid = rows;
    NCK(run_gemm(g, n->ws, n->err, n->stream, n->spin, n->sms));
  }
  return ACOPF_OK;
}

}  // namespace nn
}  // namespace acopf

using namespace acopf::nn;

extern "C" {

acopf_status acopf_mlp_create(const int32_t* dims, int32_t nlayers, int32_t max_batch, int32_t device,
                              acopf_mlp_handle* out) {
  if (!dims || !out || nlayers < 1 || nlayers > 16 || max_batch < 1) return ACOPF_EINVAL;
  *out = nullptr;
  for (int l = 0; l <= nlayers; ++l)
    if (dims[l] < 8 || dims[l] % 8) return ACOPF_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ACOPF_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return ACOPF_ECUDA;
  int major = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  if (major < 10) return ACOPF_ECUDA;
  Net* n = new Net();
  n->device = device;
  n->nl = nlayers;
  n->dims.assign(dims, dims + nlayers + 1);
  n->Mb = ((max_batch + BM - 1) / BM) * BM;
  cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, device);
  const int Mb = n->Mb;
  bool ok = true;
  n->L.resize(nlayers);
  for (int l = 0; l < nlayers && ok; ++l) {
    Layer& y = n->L[l];
    y.in = dims[l];
    y.out = dims[l + 1];
    size_t w = (size_t)y.in * y.out;
    ok = dalloc(n, &y.W, w) && dalloc(n, &y.b, y.out) && dalloc(n, &y.mW, w) && dalloc(n, &y.vW, w) &&
         dalloc(n, &y.mb, y.out) && dalloc(n, &y.vb, y.out) && dalloc(n, &y.gW, w) && dalloc(n, &y.gb, y.out) &&
         dalloc(n, &y.W16, w) && dalloc(n, &y.W16T, w);
  }
  n->A.assign(nlayers, nullptr);
  n->AT.assign(nlayers, nullptr);
  n->Z.assign(nlayers, nullptr);
  n->D.assign(nlayers + 1, nullptr);
  n->DT.assign(nlayers + 1, nullptr);
  for (int l = 0; l < nlayers && ok; ++l) {
    ok = dalloc(n, &n->A[l], (size_t)Mb * dims[l]) && dalloc(n, &n->AT[l], (size_t)Mb * dims[l]);
    if (ok && l >= 1) ok = dalloc(n, &n->Z[l], (size_t)Mb * dims[l]);
  }
  for (int l = 1; l <= nlayers && ok; ++l)
    ok = dalloc(n, &n->D[l], (size_t)Mb * dims[l]) && dalloc(n, &n->DT[l], (size_t)Mb * dims[l]);
  ok = ok && dalloc(n, &n->Y, (size_t)Mb * dims[nlayers]) && dalloc(n, &n->mu_x, dims[0]) &&
       dalloc(n, &n->sd_x, dims[0]) && dalloc(n, &n->mu_y, dims[nlayers]) && dalloc(n, &n->sd_y, dims[nlayers]) &&
       dalloc(n, &n->err, 1) && dalloc(n, &n->loss, 1);
  if (ok) {
    n->nparts = (int)(((size_t)dims[nlayers] + 31) / 32 * ((size_t)Mb / 32));
    ok = dalloc(n, &n->part, n->nparts);
  }
  if (ok) {
    // identity standardisation until fitted
    std::vector<float> one((size_t)(dims[0] > dims[nlayers] ? dims[0] : dims[nlayers]), 1.0f);
    ok = cudaMemcpy(n->sd_x, one.data(), sizeof(float) * dims[0], cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(n->sd_y, one.data(), sizeof(float) * dims[nlayers], cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok || !plan(n)) {
    free_net(n);
    delete n;
    cudaGetLastError();
    return ACOPF_ENOMEM;
  }
  *out = (acopf_mlp_handle)n;
  return ACOPF_OK;
}

acopf_status acopf_mlp_destroy(acopf_mlp_handle h) {
  Net* n = (Net*)h;
  if (!n) return ACOPF_EINVAL;
  cudaSetDevice(n->device);
  if (n->stream) cudaStreamSynchronize(n->stream);
  free_net(n);
  delete n;
  return ACOPF_OK;
}

acopf_status acopf_mlp_set_stream(acopf_mlp_handle h, void* stream) {
  Net* n = (Net*)h;
  if (!n) return ACOPF_EINVAL;
  n->stream = (cudaStream_t)stream;
  return ACOPF_OK;
}

acopf_status acopf_mlp_last_error(acopf_mlp_handle h, char* buf, size_t len) {
  Net* n = (Net*)h;
  if (!n || !buf || len == 0) return ACOPF_EINVAL;
  snprintf(buf, len, "%s", n->last_error.c_str());
  return ACOPF_OK;
}

acopf_status acopf_mlp_num_params(acopf_mlp_handle h, int64_t* count) {
  Net* n = (Net*)h;
  if (!n || !count) return ACOPF_EINVAL;
  int64_t c = 0;
  for (auto& y : n->L) c += (int64_t)y.in * y.out + y.out;
  *count = c;
  return ACOPF_OK;
}

static acopf_status copy_params(Net* n, float* host, int64_t count, bool to_device, bool grads) {
  int64_t need = 0;
  acopf_mlp_num_params((acopf_mlp_handle)n, &need);
  if (!host || count != need) return nfail(n, ACOPF_EINVAL, "parameter count mismatch");
  cudaSetDevice(n->device);
  NCK(cudaStreamSynchronize(n->stream));
  size_t off = 0;
  for (auto& y : n->L) {
    size_t w = (size_t)y.in * y.out;
    float* dw = grads ? y.gW : y.W;
    float* db = grads ? y.gb : y.b;
    if (to_device) {
      NCK(cudaMemcpy(dw, host + off, sizeof(float) * w, cudaMemcpyHostToDevice));
      NCK(cudaMemcpy(db, host + off + w, sizeof(float) * y.out, cudaMemcpyHostToDevice));
    } else {
      NCK(cudaMemcpy(host + off, dw, sizeof(float) * w, cudaMemcpyDeviceToHost));
      NCK(cudaMemcpy(host + off + w, db, sizeof(float) * y.out, cudaMemcpyDeviceToHost));
    }
    off += w + y.out;
  }
  return ACOPF_OK;
}

acopf_status acopf_mlp_set_params(acopf_mlp_handle h, const float* params, int64_t count) {
  Net* n = (Net*)h;
  if (!n) return ACOPF_EINVAL;
  acopf_status s = copy_params(n, (float*)params, count, true, false);
  if (s) return s;
  for (auto& y : n->L) {
    size_t w = (size_t)y.in * y.out;
    k_w16<<<(unsigned)((w + 255) / 256), 256, 0, n->stream>>>(y.W, y.out, y.in, y.W16, y.W16T);
    NCK(cudaMemsetAsync(y.mW, 0, sizeof(float) * w, n->stream));
    NCK(cudaMemsetAsync(y.vW, 0, sizeof(float) * w, n->stream));
    NCK(cudaMemsetAsync(y.mb, 0, sizeof(float) * y.out, n->stream));
    NCK(cudaMemsetAsync(y.vb, 0, sizeof(float) * y.out, n->stream));
  }
  n->step = 0;
  NCK(cudaGetLastError());
  NCK(cudaStreamSynchronize(n->stream));
  return ACOPF_OK;
}

acopf_status acopf_mlp_get_params(acopf_mlp_handle h, float* params, int64_t count) {
  Net* n = (Net*)h;
  if (!n) return ACOPF_EINVAL;
  return copy_params(n, params, count, false, false);
}

acopf_status acopf_mlp_get_grads(acopf_mlp_handle h, float* grads, int64_t count) {
  Net* n = (Net*)h;
  if (!n) return ACOPF_EINVAL;
  return copy_params(n, grads, count, false, true);
}

acopf_status acopf_mlp_fit_standardiser(acopf_mlp_handle h, const float* X, const float* Y, int32_t rows) {
  Net* n = (Net*)h;
  if (!n || !X || !Y || rows < 1) return nfail(n, ACOPF_EINVAL, "fit_standardiser: bad arguments");
  cudaSetDevice(n->device);
  const int d0 = n->dims[0], dn = n->dims[n->nl];
  k_standardiser<<<(d0 + 127) / 128, 128, 0, n->stream>>>(X, rows, d0, n->mu_x, n->sd_x);
  k_standardiser<<<(dn + 127) / 128, 128, 0, n->stream>>>(Y, rows, dn, n->mu_y, n->sd_y);
  NCK(cudaGetLastError());
  NCK(cudaStreamSynchronize(n->stream));
  return ACOPF_OK;
}

acopf_status acopf_mlp_get_standardiser(acopf_mlp_handle h, float* mu_x, float* sd_x, float* mu_y, float* sd_y) {
  Net* n = (Net*)h;
  if (!n) return ACOPF_EINVAL;
  cudaSetDevice(n->device);
  NCK(cudaStreamSynchronize(n->stream));
  const int d0 = n->dims[0], dn = n->dims[n->nl];
  if (mu_x) NCK(cudaMemcpy(mu_x, n->mu_x, sizeof(float) * d0, cudaMemcpyDeviceToHost));
  if (sd_x) NCK(cudaMemcpy(sd_x, n->sd_x, sizeof(float) * d0, cudaMemcpyDeviceToHost));
  if (mu_y) NCK(cudaMemcpy(mu_y, n->mu_y, sizeof(float) * dn, cudaMemcpyDeviceToHost));
  if (sd_y) NCK(cudaMemcpy(sd_y, n->sd_y, sizeof(float) * dn, cudaMemcpyDeviceToHost));
  return ACOPF_OK;
}

acopf_status acopf_mlp_forward(acopf_mlp_handle h, const float* X, int32_t rows, float* Y) {
  Net* n = (Net*)h;
  if (!n || !X || !Y || rows < 1) return nfail(n, ACOPF_EINVAL, "mlp_forward: bad arguments");
  cudaSetDevice(n->device);
  const int d0 = n->dims[0], dn = n->dims[n->nl];
  for (int r0 = 0; r0 < rows; r0 += n->Mb) {
    int rr = rows - r0 < n->Mb ? rows - r0 : n->Mb;
    size_t tot = (size_t)n->Mb * d0;
    k_input<<<(unsigned)((tot + 255) / 256), 256, 0, n->stream>>>(X + (size_t)r0 * d0, nullptr, rr, n->Mb, d0,
                                                                   n->mu_x, n->sd_x, n->A[0], n->AT[0]);
    NCK(cudaGetLastError());
    acopf_status s = forward(n, rr);
    if (s) return s;
    // outputs of the valid rows, de-standardised: y = y_std sd + mu
    size_t ty = (size_t)rr * dn;
    k_destd<<<(unsigned)((ty + 255) / 256), 256, 0, n->stream>>>(n->Y, Y + (size_t)r0 * dn, ty, dn, n->mu_y, n->sd_y);
    NCK(cudaGetLastError());
  }
  return check_err(n);
}

acopf_status acopf_mlp_train_step(acopf_mlp_handle h, const float* X, const float* T, const int32_t* idx,
                                  int32_t rows, float lr, float* loss) {
  Net* n = (Net*)h;
  if (!n || !X || !T || rows < 1 || rows > n->Mb || !(lr > 0)) return nfail(n, ACOPF_EINVAL, "mlp_train_step: bad arguments");
  cudaSetDevice(n->device);
  const int nl = n->nl, Mb = n->Mb, d0 = n->dims[0], dn = n->dims[nl];
  size_t tot = (size_t)Mb * d0;
  k_input<<<(unsigned)((tot + 255) / 256), 256, 0, n->stream>>>(X, idx, rows, Mb, d0, n->mu_x, n->sd_x, n->A[0],
                                                                 n->AT[0]);
  NCK(cudaGetLastError());
  acopf_status s = forward(n, rows);
  if (s) return s;
  dim3 mgrid((dn + 31) / 32, Mb / 32);
  k_mse<<<mgrid, dim3(32, 8), 0, n->stream>>>(n->Y, T, idx, rows, Mb, dn, n->mu_y, n->sd_y, n->D[nl], n->DT[nl],
                                              n->part);
  k_sum<<<1, 1024, 0, n->stream>>>(n->part, (int)(mgrid.x * mgrid.y), 1.0 / ((double)rows * dn), n->loss);
  NCK(cudaGetLastError());
  for (int l = nl - 1; l >= 0; --l) {
    NCK(run_gemm(n->bwd_w[l], n->ws, n->err, n->stream, n->spin, n->sms));
    k_colsum<<<(n->dims[l + 1] + 127) / 128, 128, 0, n->stream>>>(n->D[l + 1], Mb, n->dims[l + 1], n->L[l].gb);
    NCK(cudaGetLastError());
    if (l >= 1) NCK(run_gemm(n->bwd_x[l], n->ws, n->err, n->stream, n->spin, n->sms));
  }
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 - pow(0.9, n->step)), c2 = (float)(1.0 - pow(0.999, n->step));
  for (auto& y : n->L) {
    dim3 grid((y.in + 31) / 32, (y.out + 31) / 32);
    k_adam_w<<<grid, dim3(32, 8), 0, n->stream>>>(y.W, y.gW, y.mW, y.vW, y.out, y.in, lr, b1, b2, eps, c1, c2, y.W16,
                                                    y.W16T);
    k_adam_b<<<(y.out + 255) / 256, 256, 0, n->stream>>>(y.b, y.gb, y.mb, y.vb, y.out, lr, b1, b2, eps, c1, c2);
  }
  NCK(cudaGetLastError());
  if (loss) NCK(cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
  return ACOPF_OK;
}

acopf_status acopf_mlp_sync(acopf_mlp_handle h) {
  Net* n = (Net*)h;
  if (!n) return ACOPF_EINVAL;
  cudaSetDevice(n->device);
  return check_err(n);
}

// C[M x N] = A[M x K] B[N x K]^T: bfloat16 operands (row stride K), FP32 output
// (row stride N), all device pointers; on the given stream, synchronised.
acopf_status acopf_gemm_bf16(const void* A, const void* B, float* C, int32_t M, int32_t N, int32_t K, int32_t splits,
                             void* stream, float* ms) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 8 || K % 8) return ACOPF_EINVAL;
  Gemm g;
  memset(&g, 0, sizeof(g));
  g.M = M; g.N = N; g.K = K;
  if (!make_map(&g.ta, A, M, K, K, BM) || !make_map(&g.tb, B, N, K, K, BN)) return ACOPF_EINVAL;
  int kt = (K + BK - 1) / BK;
  int s = splits < 1 ? 1 : (splits > kt ? kt : splits);
  g.kts = (kt + s - 1) / s;
  g.splits = (kt + g.kts - 1) / g.kts;
  g.e.op = EPI_F32; g.e.M = M; g.e.N = N; g.e.rows_valid = M; g.e.f32 = C; g.e.ld_f32 = N;
  cudaStream_t st = (cudaStream_t)stream;
  float* ws = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return ACOPF_ENOMEM;
  cudaMemsetAsync(err, 0, sizeof(int), st);
  if (g.splits > 1 && cudaMalloc(&ws, sizeof(float) * (size_t)g.splits * M * N) != cudaSuccess) {
    cudaFree(err);
    return ACOPF_ENOMEM;
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  cudaError_t e = run_gemm(g, ws, err, st, 1ll << 32, sms);
  if (ms) cudaEventRecord(e1, st);
  int hv = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hv, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (ms) {
    *ms = 0.0f;
    if (e == cudaSuccess) cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (ws) cudaFree(ws);
  cudaFree(err);
  if (e != cudaSuccess) return ACOPF_ECUDA;
  return hv ? ACOPF_ETIMEOUT : ACOPF_OK;
}

}  // extern "C"

