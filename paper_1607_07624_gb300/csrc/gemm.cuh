// BF16 tensor-core GEMM for sm_100-family GPUs: C = A * B^T with A [M][K] and
// B [N][K] both row-major (K contiguous), float32 accumulation in tensor memory.
//
// One CTA computes one 128 x BN tile of C with four warps:
//   warp 0 lane 0  issues TMA tile loads (64-element K slices, 128-byte swizzle)
//                  into a STAGES-deep ring of shared-memory slots;
//   warp 1 lane 0  issues tcgen05.mma (128 x BN x 16 per instruction) into a
//                  128-lane x BN-column float32 accumulator in tensor memory, and
//                  frees each slot with tcgen05.commit once its MMAs complete;
//   all four warps then read the accumulator (warp w owns rows 32w..32w+31)
//                  and hand 16-column pieces to the epilogue functor.
// Out-of-range rows and columns of the operands are zero-filled by the TMA unit,
// so M, N and K need no padding; the epilogue skips rows >= M and columns >= N.
// Every wait is bounded: a pipeline wait gives up after wait_limit tries, sets a bit
// in *err and the CTA unwinds: it waits (bounded by tc::WAIT_LIMIT, far longer than
// any copy or product takes) for its own outstanding TMA copies and for the products
// it issued, so that nothing is in flight when it frees its tensor memory and exits.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.h"
#include "pdl.cuh"
#include "tc.cuh"

namespace pas {

constexpr unsigned GEMM_ERR_PRODUCER = 1u, GEMM_ERR_MMA = 2u, GEMM_ERR_EPILOGUE = 4u, GEMM_ERR_DRAIN = 8u;
constexpr int GEMM_GROUP = 8;  // column tiles per band of the grouped tile order

template <int BN, int STAGES>
struct GemmCfg {
  static constexpr uint32_t A_BYTES = 128u * 64u * 2u;
  static constexpr uint32_t B_BYTES = (uint32_t)BN * 64u * 2u;
  static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;  // + alignment slack
  static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 M=128 needs N in [16,256], N % 16 == 0");
  static_assert((BN & (BN - 1)) == 0, "tensor-memory allocation needs a power of two");
};

template <int BN, int STAGES, class Epi>
__global__ void __launch_bounds__(128, 1)
    gemm_bf16_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M,
                        int N, int K, Epi epi, unsigned int* err, uint32_t wait_limit) {
  using C = GemmCfg<BN, STAGES>;
  extern __shared__ uint8_t gemm_dsm[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gemm_dsm) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped tile order: CTAs are dispatched in linear order; consecutive ones sweep
  // a band of GEMM_GROUP column tiles row by row, so a wave reads a band of B (which
  // stays in L2 while the band is swept) instead of all of it
  int n_tile, m_tile;
  {
    const int tn = gridDim.x, tm = gridDim.y;
    const int lin = blockIdx.y * tn + blockIdx.x;
    const int band = lin / (GEMM_GROUP * tm);
    const int first = band * GEMM_GROUP;
    const int width = min(GEMM_GROUP, tn - first);
    const int in_band = lin - band * GEMM_GROUP * tm;
    n_tile = first + in_band % width;
    m_tile = in_band / width;
  }
  const int n0 = n_tile * BN, m0 = m_tile * 128;
  const int nk = (K + 63) / 64;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    abort_flag = 0;
    tc::fence_barrier_init();
    tc::prefetch_tensormap(&tmA);
    tc::prefetch_tensormap(&tmB);
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, C::TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  // launched programmatically after the producer of A, B or the epilogue inputs:
  // the set-up above overlaps its tail; nothing it wrote is touched before this
  pdl_trigger();
  pdl_wait();

  // last round issued per slot (for the drain after a timeout); producer only
  int last_round[STAGES];
  for (int s = 0; s < STAGES; ++s) last_round[s] = -1;

  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES, round = kb / STAGES;
      if (round > 0 && !tc::mbar_wait(&empty[s], (uint32_t)(round - 1) & 1u, wait_limit)) {
        atomicOr(err, GEMM_ERR_PRODUCER);
        abort_flag = 1;
        break;
      }
      if (abort_flag) break;
      uint8_t* a = sm + (size_t)s * C::STAGE_BYTES;
      tc::mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
      tc::tma_load_2d(a, &tmA, &full[s], kb * 64, m0);
      tc::tma_load_2d(a + C::A_BYTES, &tmB, &full[s], kb * 64, n0);
      last_round[s] = round;
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, BN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!tc::mbar_wait(&full[s], (uint32_t)(kb / STAGES) & 1u, wait_limit)) {
        atomicOr(err, GEMM_ERR_MMA);
        abort_flag = 1;
        break;
      }
      if (abort_flag) break;
      tc::fence_after_sync();
      const uint32_t a = tc::smem_addr(sm + (size_t)s * C::STAGE_BYTES), b = a + C::A_BYTES;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        tc::mma_bf16(tmem, tc::desc_sw128(a + 32u * k), tc::desc_sw128(b + 32u * k), idesc,
                     (kb | k) != 0 ? 1u : 0u);
      tc::mma_commit(&empty[s]);
    }
    // arrives once every MMA issued above has completed (immediately if none)
    tc::mma_commit(&done);
  }
  __syncwarp();

  if (!tc::mbar_wait(&done, 0, wait_limit)) {
    atomicOr(err, GEMM_ERR_EPILOGUE);
    abort_flag = 1;
  }
  tc::fence_after_sync();
  __syncthreads();
  if (!abort_flag && nk > 0) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
      if (n0 + c >= N) break;  // uniform across the CTA
      float v[16];
      tc::tmem_ld16(tmem + lane_base + (uint32_t)c, v);
      if (row < M) epi.store(row, n0 + c, v);
    }
  }
  if (abort_flag && warp == 0 && lane == 0) {
    // copies still in flight land before the CTA's shared memory is released, and
    // the products issued complete before their tensor memory is freed (the MMA
    // thread commits `done` after its loop, aborted or not)
    for (int s = 0; s < STAGES; ++s)
      if (last_round[s] >= 0 && !tc::mbar_wait(&full[s], (uint32_t)last_round[s] & 1u))
        atomicOr(err, GEMM_ERR_DRAIN);
    if (!tc::mbar_wait(&done, 0)) atomicOr(err, GEMM_ERR_DRAIN);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

// Host side ------------------------------------------------------------------

// Tensor map of a row-major bf16 matrix [rows][cols] with leading dimension ld
// (elements; ld * 2 must be a multiple of 16), box 64 columns x box_rows rows,
// 128-byte swizzle, zero fill outside the matrix.
bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                    uint32_t box_rows);

// Operand maps and sizes of one GEMM C[M][N] = A[M][K] * B[N][K]^T.
struct GemmOp {
  CUtensorMap a, b;
  int M = 0, N = 0, K = 0, bn = 128;
};

// Pick the tile width for an M x N output on `sms` SMs (fewest waves of the
// cheapest tile).
int gemm_pick_bn(int M, int N, int sms);

// Build the maps for A (lda) and B (ldb); false if the tensor-map encoder
// rejects them (alignment) or is unavailable.
bool gemm_prepare(GemmOp* op, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                  int sms);

// pdl: launch with programmatic stream serialization (the kernel waits for its
// predecessor after its set-up).
template <int BN, int STAGES, class Epi>
cudaError_t gemm_launch_bn(const GemmOp& op, const Epi& epi, cudaStream_t st, unsigned* err, bool pdl,
                           uint32_t wait_limit) {
  using C = GemmCfg<BN, STAGES>;
  auto kern = gemm_bf16_tc_kernel<BN, STAGES, Epi>;
  cudaError_t e = raise_dyn_smem((const void*)kern, C::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid((op.N + BN - 1) / BN, (op.M + 127) / 128);
  return launch_k(kern, grid, dim3(128), C::SMEM, st, pdl, op.a, op.b, op.M, op.N, op.K, epi, err, wait_limit);
}

// wait_limit: tries of each pipeline wait before it gives up (tc::WAIT_LIMIT by default).
template <class Epi>
cudaError_t gemm_launch(const GemmOp& op, const Epi& epi, cudaStream_t st, unsigned* err, bool pdl = false,
                        uint32_t wait_limit = tc::WAIT_LIMIT) {
  switch (op.bn) {
    case 16:
      return gemm_launch_bn<16, 8>(op, epi, st, err, pdl, wait_limit);
    case 32:
      return gemm_launch_bn<32, 8>(op, epi, st, err, pdl, wait_limit);
    case 64:
      return gemm_launch_bn<64, 6>(op, epi, st, err, pdl, wait_limit);
    case 256:
      return gemm_launch_bn<256, 4>(op, epi, st, err, pdl, wait_limit);
    default:
      return gemm_launch_bn<128, 5>(op, epi, st, err, pdl, wait_limit);
  }
}

}  // namespace pas
