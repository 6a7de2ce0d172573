// Learned nonlinear reconstructor (multilayer perceptron, slopes -> modal
// coefficients): object layout shared with the loop. The paper's reconstructor
// is linear (Table 1 modalrec); this one replaces the matrix-vector product of
// the loop when attached to it.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.h"
#include "recon.cuh"

#define PAS_MLP_MAX_LAYERS 8

struct pas_mlp_s {
  pas_ctx_t ctx = nullptr;
  int L = 0;                                // weight layers
  int sz[PAS_MLP_MAX_LAYERS + 1] = {};      // layer widths, sz[0] = inputs
  int ld[PAS_MLP_MAX_LAYERS + 1] = {};      // widths rounded up to 8 (16-byte rows in bf16)
  int max_batch = 0, ldb = 0;               // ldb: max_batch rounded up to 8
  size_t n_params = 0;
  size_t offW[PAS_MLP_MAX_LAYERS] = {}, offb[PAS_MLP_MAX_LAYERS] = {};
  // parameters: float32 master copy, gradients, Adam moments (flat, W_l then b_l)
  float* d_p = nullptr;
  float* d_g = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  long long* d_t = nullptr;                  // Adam step count
  __nv_bfloat16* d_W[PAS_MLP_MAX_LAYERS] = {};   // [out][ld in]
  __nv_bfloat16* d_Wt[PAS_MLP_MAX_LAYERS] = {};  // [in][ld out]
  float* d_mean = nullptr;                   // input standardisation
  float* d_istd = nullptr;
  // batched activations (batch <= max_batch)
  __nv_bfloat16* d_X = nullptr;              // [B][ld in]
  __nv_bfloat16* d_Xt = nullptr;             // [in][ldb]
  float* d_Z[PAS_MLP_MAX_LAYERS] = {};       // hidden pre-activations [B][ld]
  __nv_bfloat16* d_H[PAS_MLP_MAX_LAYERS] = {};
  __nv_bfloat16* d_Ht[PAS_MLP_MAX_LAYERS] = {};
  float* d_out = nullptr;                    // [B][ld out]
  __nv_bfloat16* d_dZ[PAS_MLP_MAX_LAYERS] = {};
  __nv_bfloat16* d_dZt[PAS_MLP_MAX_LAYERS] = {};
  float* d_loss_part = nullptr;
  unsigned int* d_done = nullptr;            // last-CTA counters [4]
  int* d_zero = nullptr;                     // a constant 0 (step index of one-off calls)
  int* d_iter = nullptr;                     // step index inside a training run
  float* d_loss1 = nullptr;
  float* d_lr1 = nullptr;
  unsigned int* d_err = nullptr;             // tensor-core pipeline timeouts, bad sample indices
  unsigned int* d_fault = nullptr;           // non-finite output seen by the loop's final layer
  // single-vector inference (the loop)
  float* d_vec[2] = {};
  unsigned int* d_gemv_done = nullptr;
  // captured training step
  cudaGraph_t train_graph = nullptr;
  cudaGraphExec_t train_exec = nullptr;
  const void* train_key[6] = {};
  int train_batch = 0;
};

namespace pas {
// Enqueue the single-vector inference chain with the loop's integrator in the last layer.
pas_status mlp_loop_launch(pas_mlp_t m, const ReconArgs& integ, cudaStream_t st, bool pdl);
// Enqueue the forward pass of B vectors given by device pointers (d_slopes: a device
// array of B pointers to n_in floats), standardised and cast to bf16 on the way in, through
// the tensor-core layers: the outputs land in m->d_out [B][m->ld[m->L]] (float32). A layer
// with fewer output tiles than SMs splits its reduction over K when `part` (part_len
// floats, mlp_split_workspace(m, B) of them) is given: partials, then a kernel that adds
// them in order and applies the bias and activation.
pas_status mlp_batch_forward(pas_mlp_t m, int B, const float* const* d_slopes, float* part, size_t part_len,
                             cudaStream_t st);
size_t mlp_split_workspace(pas_mlp_t m, int B);
// Kernels one mlp_batch_forward launches.
int mlp_batch_forward_kernels(pas_mlp_t m, int B, size_t part_len);
}
