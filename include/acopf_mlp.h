/*
 * acopf_mlp.h -- C ABI of the learned ADMM warm start (GB300, sm_103a).
 *
 * A multilayer perceptron maps a load scenario, the per-bus (pd, qd) of a
 * grid, to a starting point for the SQP-ADMM solver of acopf.h: the NLP
 * point x0, the line multipliers pi, the ADMM multipliers lambda0 and a
 * per-component penalty factor.  The paper warm-starts each QP's ADMM from
 * the previous QP (Sec. IV; abstract); this network extends that to the
 * first QP of a new load scenario.  It is trained on solutions the cold-start
 * solver computes for sampled loads, and the cold-start solver stays the
 * judge of its error: a warm-started solve must reach the same tolerance.
 *
 * Network: nlayers affine layers, dims[0] inputs, hidden widths
 * dims[1..nlayers-1] with the exact GELU x Phi(x) (Hendrycks and Gimpel,
 * 2016), dims[nlayers] outputs (affine).  Inputs and outputs are
 * standardised column by column (mean, population deviation of the training
 * set).  Weights are kept in FP32 (master copy, Adam moments) and used in
 * bfloat16; layer inputs and back-propagated gradients are bfloat16; every
 * product accumulates in FP32 on the tensor cores (tcgen05.mma, operands
 * staged by TMA, accumulator in tensor memory).  Loss: mean squared error over
 * all standardised outputs; optimiser: Adam with bias correction (Kingma and
 * Ba, 2015; beta1 0.9, beta2 0.999, eps 1e-8).
 *
 * Conventions: every call returns acopf_status (0 = ACOPF_OK).  Matrices are
 * row-major FP32.  "Device" pointers must be CUDA device memory of the
 * handle's device; host pointers are plain host memory.  The handle owns its
 * device memory.  Calls are asynchronous on the handle's stream except where
 * stated; handles are not thread-safe.  ACOPF_EINVAL: bad sizes or NULL
 * arguments; ACOPF_ENOMEM: allocation failed; ACOPF_ECUDA: no usable device
 * (compute capability 10 or higher is required) or a CUDA error;
 * ACOPF_ETIMEOUT: a tensor-core pipeline wait in a kernel gave up (the
 * kernel's waits are bounded; the context stays usable).
 */
#ifndef ACOPF_MLP_H
#define ACOPF_MLP_H

#include <stddef.h>
#include <stdint.h>

#include "acopf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct acopf_mlp* acopf_mlp_handle;

/* dims: nlayers + 1 widths, each a positive multiple of 8 (rows of bfloat16
 * operands must be 16-byte multiples); max_batch: rows per training step and
 * per forward chunk (rounded up to a multiple of 128 internally). */
acopf_status acopf_mlp_create(const int32_t* dims, int32_t nlayers, int32_t max_batch, int32_t device,
                              acopf_mlp_handle* out);
acopf_status acopf_mlp_destroy(acopf_mlp_handle h);
acopf_status acopf_mlp_set_stream(acopf_mlp_handle h, void* cuda_stream);
acopf_status acopf_mlp_last_error(acopf_mlp_handle h, char* buf, size_t n);

/* Parameters as one host FP32 array: for each layer l, W_l [dims[l+1] x
 * dims[l]] row-major, then b_l [dims[l+1]].  set_params also resets the Adam
 * moments and step count.  Synchronous.  get_grads returns the gradients of
 * the last training step in the same layout. */
acopf_status acopf_mlp_num_params(acopf_mlp_handle h, int64_t* count);
acopf_status acopf_mlp_set_params(acopf_mlp_handle h, const float* params, int64_t count);
acopf_status acopf_mlp_get_params(acopf_mlp_handle h, float* params, int64_t count);
acopf_status acopf_mlp_get_grads(acopf_mlp_handle h, float* grads, int64_t count);

/* Column statistics of the training inputs X [rows x dims[0]] and targets
 * Y [rows x dims[nlayers]] (device); synchronous.  get_standardiser copies
 * them to host arrays (any may be NULL). */
acopf_status acopf_mlp_fit_standardiser(acopf_mlp_handle h, const float* X, const float* Y, int32_t rows);
acopf_status acopf_mlp_get_standardiser(acopf_mlp_handle h, float* mu_x, float* sd_x, float* mu_y, float* sd_y);

/* Y [rows x dims[nlayers]] = network(X [rows x dims[0]]), raw (de-standardised)
 * outputs; X and Y on the device; any rows >= 1 (processed in chunks of
 * max_batch).  Synchronises the stream to read the kernels' error flag. */
acopf_status acopf_mlp_forward(acopf_mlp_handle h, const float* X, int32_t rows, float* Y);

/* One Adam step on the rows idx[0..rows) (device int32 indices; NULL: rows
 * 0..rows-1) of the data set X [. x dims[0]], T [. x dims[nlayers]] (raw,
 * device), 1 <= rows <= max_batch, learning rate lr > 0.  If loss is not
 * NULL, the batch's mean squared error (before the step, on standardised
 * outputs) is written to that DEVICE float.  Asynchronous. */
acopf_status acopf_mlp_train_step(acopf_mlp_handle h, const float* X, const float* T, const int32_t* idx,
                                  int32_t rows, float lr, float* loss);

/* Wait for the handle's stream and report a pipeline time-out, if any. */
acopf_status acopf_mlp_sync(acopf_mlp_handle h);

/* The tensor-core matrix product alone, for tests and measurement:
 * C [M x N] = A [M x K] * B [N x K]^T with A, B bfloat16 (row stride K, K a
 * multiple of 8, 16-byte aligned) and C FP32 (row stride N), all device
 * memory; the contraction is split into at most `splits` slices summed in
 * FP32.  Allocates scratch, synchronises the stream.  If ms is not NULL it
 * receives the device time of the product's kernels (CUDA events recorded on
 * the stream around them). */
acopf_status acopf_gemm_bf16(const void* A, const void* B, float* C, int32_t M, int32_t N, int32_t K, int32_t splits,
                             void* cuda_stream, float* ms);

/* Warm start of every instance of a solver handle from device predictions:
 * pred [K x ld] FP32 (K = number of instances; ld >= the width below), row k
 * laid out as
 *   x0      2G + 2B + 2L   NLP point in the layout of acopf_set_iterate
 *   pi      4L             line multipliers, branch-major (pi11 pi12 pi13 pi14)
 *   lambda  8L + 2G        ADMM multipliers: the lam array of acopf_admm_state,
 *                          then its lg array
 *   logfac  L + G          natural log of each component's penalty factor:
 *                          rho = base_rho * exp(clamp(logfac, -2.3, 2.3))
 * where B, L, G are that instance's bus, branch and generator counts (the
 * instances must share them).  Any part may be skipped: use_x, use_pi,
 * use_lambda, use_rho select which are applied.  The values are used by the
 * next sqp_solve, as for acopf_set_warm_start.  Voltages are clamped into
 * their bounds and generator outputs into their boxes. */
acopf_status acopf_set_warm_start_device(acopf_handle h, const float* pred, int64_t ld, double base_rho,
                                         int32_t use_x, int32_t use_pi, int32_t use_lambda, int32_t use_rho);

#ifdef __cplusplus
}
#endif

#endif /* ACOPF_MLP_H */
