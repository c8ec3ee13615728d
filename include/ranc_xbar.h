/*
 * ranc_xbar.h - C ABI of the crossbar-product measurement kernels: the
 * integration step of the RANC neuron block (Alg. 1 and Sec. III-C; Sec. II:
 * a binary axon x neuron crossbar and one weight per axon type per neuron)
 * for a batch of samples, computed in three exact tensor-core formulations so
 * that their speed can be compared on the same inputs:
 *
 *   RANC_XBAR_F16_FOLDED   the batched path's own form: W[n][a] = C[a][n] *
 *                          w[type(a)][n] folded once into an fp16 matrix,
 *                          0/1 spikes in fp16, one tcgen05.mma kind::f16
 *                          GEMM with fp32 accumulation in tensor memory
 *                          (exact: |w| <= 2047 and every partial sum is an
 *                          integer below 2^22);
 *   RANC_XBAR_F8_PER_TYPE  0/1 crossbar and 0/1 spikes in e4m3 (exact), axons
 *                          sorted by type with each type's range padded to 32,
 *                          one tcgen05.mma kind::f8f6f4 accumulator per type
 *                          (per-type connection counts, exact in fp32), then
 *                          dV = sum_k w[k][n] * count_k in int32;
 *   RANC_XBAR_I8_MMA_SYNC  the same per-type counts with int8 0/1 operands on
 *                          the warp-level mma.sync.m16n8k32 s8 instruction
 *                          (int32 accumulation), then the same int32 sum.
 *
 * All three give dV[b][c][n] = sum over active axons a of sample b that
 * connect to neuron n of core c of w[type(a)][n], exactly.
 *
 * Conventions as in ranc.h (0 or a negative RANC_E* code; reason in
 * ranc_xbar_last_error; work on the stream given at creation; "device"
 * pointers are caller-owned CUDA memory).  Not thread-safe per handle.
 */
#ifndef RANC_XBAR_H
#define RANC_XBAR_H

#include <stdint.h>

#include "ranc.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { RANC_XBAR_F16_FOLDED = 0, RANC_XBAR_F8_PER_TYPE = 1, RANC_XBAR_I8_MMA_SYNC = 2 };

typedef struct ranc_xbar ranc_xbar;

/* Lays out the crossbars, axon types and weights of `desc` (the other fields
 * are not used beyond validation) for formulation `form` and copies them to
 * the device.  Shapes: axons a multiple of 64 in [64, 512], neurons a
 * multiple of 128 in [128, 512], at most 4 axon types, |weight| <= 2047.
 * Errors: RANC_EINVAL (description, shape or form; an sm_103 device is needed
 * for the tcgen05 forms), RANC_ENOMEM, RANC_ECUDA.  *out is NULL on error. */
int ranc_xbar_create(const ranc_desc *desc, int32_t form, void *cuda_stream, ranc_xbar **out);

/* dV for `batch` samples (a multiple of 128).  spikes: device
 * [batch][axons/32] uint32, bit a%32 of word a/32 = axon a of sample b is
 * active.  dv: device [batch][n_cores][neurons] int32, or NULL; sums: device
 * [batch][n_cores] int64 receiving sum_n (n % 8 + 1) * dV[b][c][n] (an exact
 * digest that moves 1/neurons of dV's bytes, for timing the product rather
 * than its stores), or NULL.  Stream-ordered; errors of the kernel surface at
 * the next ranc_xbar_sync. */
int ranc_xbar_run(ranc_xbar *x, const uint32_t *spikes, int32_t batch, int32_t *dv, int64_t *sums);

/* Synchronises the handle's stream and reports a kernel failure (RANC_ECUDA,
 * or RANC_ETIMEOUT when a bounded device-side wait gave up). */
int ranc_xbar_sync(ranc_xbar *x);

void ranc_xbar_destroy(ranc_xbar *x);
const char *ranc_xbar_last_error(const ranc_xbar *x);

#ifdef __cplusplus
}
#endif
#endif /* RANC_XBAR_H */
