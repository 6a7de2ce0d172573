// Reconstruction of a group of loops that share one bfloat16 reconstructor, as one
// tensor-core product per step: dmodes[:, b] = R s_b for the group's B loops is
// C = R S^T with S = [s_1 ... s_B] (Table 1 modalrec, batched). Used by batches.
#pragma once
#include <cuda_bf16.h>

#include "internal.h"
#include "recon.cuh"

namespace pas {

// Per-loop pointers of one group (device arrays of B entries each).
struct BatchRecState {
  const float* const* slopes = nullptr;   // [B] -> [n_s]
  float* const* ring = nullptr;            // [B] -> [delay_b][n_m] command ring
  const float* const* gain = nullptr;      // [B] -> [n_m]
  float* const* cmd = nullptr;             // [B] -> [n_m] copy of the new command
  float* const* dmodes = nullptr;          // [B] -> [n_m]
  long long* const* step = nullptr;        // [B] -> step counter (advanced after the product)
  const int* delay = nullptr;              // [B]
};

struct BatchRecGroup;  // opaque: the group's buffers and tensor maps

// Set up a group of B loops sharing `rec` (PAS_BF16): allocates the bf16 slope matrix,
// the pointer arrays and the GEMM's tensor maps. Host arrays of B entries.
pas_status batch_rec_create(pas_ctx_t ctx, pas_recon_t rec, int B, const float* const* slopes,
                            float* const* ring, const float* const* gain, float* const* cmd,
                            float* const* dmodes, long long* const* step, const int* delay,
                            BatchRecGroup** out);
// The same for B loops that share one network (pas_mlp_t, B <= its batch size): each step
// one batched forward of their slopes through the tensor-core layers (bf16 activations,
// float32 accumulation), then each loop's integrator on its output, as the single-vector
// chain's last layer applies it.
pas_status batch_mlp_create(pas_ctx_t ctx, pas_mlp_t mlp, int B, const float* const* slopes,
                            float* const* ring, const float* const* gain, float* const* cmd,
                            float* const* dmodes, long long* const* step, const int* delay,
                            BatchRecGroup** out);
// Enqueue on `st`: gather the B slope vectors as bf16, the product with the fused
// integrator (or the network's batched forward and the integrator), then advance the B
// step counters.
pas_status batch_rec_launch(BatchRecGroup* g, cudaStream_t st);
// Error word of the product's (the network's GEMMs') bounded waits (non-zero: a wait gave up).
unsigned int* batch_rec_err(BatchRecGroup* g);
// Kernels one launch enqueues.
int batch_rec_kernels(BatchRecGroup* g);
void batch_rec_destroy(BatchRecGroup* g);

}  // namespace pas
