// BF16 tensor-core GEMM for sm_100-family GPUs: C = A * B^T with A [M][K] and
// B [N][K] both row-major (K contiguous), float32 accumulation in tensor memory.
//
// One CTA computes one 128 x BN tile of C (or, with the reduction split into gridDim.z
// ranges of K, one range's partial of it) with four warps:
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
  // split K (gridDim.z > 1): CTA z takes 64-element slices [kb0, kb0 + nk) of the
  // reduction and its epilogue stores a partial product (the epilogue reads blockIdx.z)
  const int nk_all = (K + 63) / 64;
  const int kb0 = (int)(((long long)nk_all * blockIdx.z) / gridDim.z);
  const int nk = (int)(((long long)nk_all * (blockIdx.z + 1)) / gridDim.z) - kb0;

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
      tc::tma_load_2d(a, &tmA, &full[s], (kb0 + kb) * 64, m0);
      tc::tma_load_2d(a + C::A_BYTES, &tmB, &full[s], (kb0 + kb) * 64, n0);
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

// The same product for many tiles, persistent: one CTA per SM walks the tiles
// (tile t, t + gridDim.x, ... in the grouped order above) with six warps:
//   warp 0 lane 0  TMA loads into the STAGES-deep ring, across tile boundaries;
//   warp 1 lane 0  tcgen05.mma into a tile accumulator in tensor memory, waiting
//                  until the epilogue has emptied it; commits it as full;
//   warps 2..5     the epilogue (warp w reads tensor-memory lanes 32 (w mod 4) on).
// A tile is MH x 128 rows by BN columns: with MH = 2 the two 128-row halves share each
// B slice (one 256 x 256 tile reads 0.0078 operand bytes per flop against 0.0117 for
// 128 x 256, the rate at which L2 feeds the SMs being the bound of the smaller tile).
// Two accumulators alternate between tiles where they fit the 512 columns (the
// epilogue of tile i then runs under the products of tile i + 1); one otherwise (the
// ring keeps loading the next tile's slices during the epilogue).
// Waits are bounded as in gemm_bf16_tc_kernel, with the same error bits and unwinding.
template <int BN, int STAGES, int MH>
struct GemmPCfg {
  static constexpr uint32_t A_BYTES = (uint32_t)MH * 128u * 64u * 2u;
  static constexpr uint32_t B_BYTES = (uint32_t)BN * 64u * 2u;
  static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
  static constexpr uint32_t ACC = (uint32_t)MH * BN;            // columns of one tile accumulator
  static constexpr int NBUF = 2 * ACC <= 512 ? 2 : 1;
  static constexpr uint32_t TMEM_COLS = NBUF * ACC;
  static_assert(BN >= 128 && BN <= 256 && (BN & (BN - 1)) == 0, "128- or 256-column tiles");
  static_assert(MH == 1 || MH == 2, "one or two 128-row halves");
  static_assert(TMEM_COLS <= 512 && SMEM <= 227 * 1024, "tensor and shared memory of one SM");
};

template <int BN, int STAGES, int MH, class Epi>
__global__ void __launch_bounds__(192, 1)
    gemm_bf16_tc_persist_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                                int M, int N, int K, Epi epi, unsigned int* err, uint32_t wait_limit) {
  using C = GemmPCfg<BN, STAGES, MH>;
  constexpr int NBUF = C::NBUF;
  extern __shared__ uint8_t gemm_dsm[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gemm_dsm) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[STAGES], empty[STAGES], acc_full[NBUF], acc_empty[NBUF], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int TM_ROWS = 128 * MH;
  const int tn = (N + BN - 1) / BN, tm = (M + TM_ROWS - 1) / TM_ROWS, n_tiles = tn * tm;
  const int nk = (K + 63) / 64;
  auto tile_origin = [&](int lin, int& m0, int& n0) {
    const int band = lin / (GEMM_GROUP * tm);
    const int first = band * GEMM_GROUP;
    const int width = min(GEMM_GROUP, tn - first);
    const int in_band = lin - band * GEMM_GROUP * tm;
    n0 = (first + in_band % width) * BN;
    m0 = (in_band / width) * TM_ROWS;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
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
  pdl_trigger();
  pdl_wait();

  int last_round[STAGES];  // producer: last round issued per slot (for the unwinding)
  for (int s = 0; s < STAGES; ++s) last_round[s] = -1;

  if (warp == 0 && lane == 0) {
    int g = 0;
    for (int t = blockIdx.x; t < n_tiles && !abort_flag; t += gridDim.x) {
      int m0, n0;
      tile_origin(t, m0, n0);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % STAGES, round = g / STAGES;
        if (round > 0 && !tc::mbar_wait(&empty[s], (uint32_t)(round - 1) & 1u, wait_limit)) {
          atomicOr(err, GEMM_ERR_PRODUCER);
          abort_flag = 1;
          break;
        }
        if (abort_flag) break;
        uint8_t* a = sm + (size_t)s * C::STAGE_BYTES;
        tc::mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
#pragma unroll
        for (int h = 0; h < MH; ++h) tc::tma_load_2d(a + h * 16384, &tmA, &full[s], kb * 64, m0 + 128 * h);
        tc::tma_load_2d(a + C::A_BYTES, &tmB, &full[s], kb * 64, n0);
        last_round[s] = round;
      }
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, BN);
    int g = 0, it = 0;
    for (int t = blockIdx.x; t < n_tiles && !abort_flag && nk > 0; t += gridDim.x, ++it) {
      const int buf = it % NBUF, use = it / NBUF;
      if (use > 0 && !tc::mbar_wait(&acc_empty[buf], (uint32_t)(use - 1) & 1u, wait_limit)) {
        atomicOr(err, GEMM_ERR_MMA);
        abort_flag = 1;
        break;
      }
      if (abort_flag) break;
      tc::fence_after_sync();
      const uint32_t acc = tmem + (uint32_t)buf * C::ACC;
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % STAGES;
        if (!tc::mbar_wait(&full[s], (uint32_t)(g / STAGES) & 1u, wait_limit)) {
          atomicOr(err, GEMM_ERR_MMA);
          abort_flag = 1;
          ok = false;
          break;
        }
        if (abort_flag) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t a = tc::smem_addr(sm + (size_t)s * C::STAGE_BYTES), b = a + C::A_BYTES;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int h = 0; h < MH; ++h)
            tc::mma_bf16(acc + (uint32_t)(h * BN), tc::desc_sw128(a + 16384u * h + 32u * k),
                         tc::desc_sw128(b + 32u * k), idesc, (kb | k) != 0 ? 1u : 0u);
        tc::mma_commit(&empty[s]);
      }
      if (!ok) break;
      tc::mma_commit(&acc_full[buf]);
    }
    // arrives once every product issued above has completed (immediately if none)
    tc::mma_commit(&done);
  } else if (warp >= 2) {
    const int q = warp & 3;  // the tensor-memory lane quarter this warp may read
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int it = 0;
    for (int t = blockIdx.x; t < n_tiles && nk > 0; t += gridDim.x, ++it) {
      const int buf = it % NBUF, use = it / NBUF;
      const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&acc_full[buf], (uint32_t)use & 1u, wait_limit));
      if (!ok) {
        if (lane == 0) atomicOr(err, GEMM_ERR_EPILOGUE);
        abort_flag = 1;
        break;
      }
      if (abort_flag) break;
      tc::fence_after_sync();
      int m0, n0;
      tile_origin(t, m0, n0);
#pragma unroll 1
      for (int h = 0; h < MH; ++h) {
        const int row = m0 + 128 * h + q * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
          if (n0 + c >= N) break;  // uniform across the warp
          float v[16];
          tc::tmem_ld16(tmem + (uint32_t)buf * C::ACC + (uint32_t)(h * BN) + lane_base + (uint32_t)c, v);
          if (row < M) epi.store(row, n0 + c, v);
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[buf]);
    }
  }
  __syncwarp();
  // every product issued has completed before the tensor memory is freed
  if (!tc::mbar_wait(&done, 0) && threadIdx.x == 0) atomicOr(err, GEMM_ERR_DRAIN);
  if (abort_flag && warp == 0 && lane == 0) {
    // copies still in flight land before the CTA's shared memory is released
    for (int s = 0; s < STAGES; ++s)
      if (last_round[s] >= 0 && !tc::mbar_wait(&full[s], (uint32_t)last_round[s] & 1u))
        atomicOr(err, GEMM_ERR_DRAIN);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

// Epilogue of a product whose reduction is split over gridDim.z ranges of K: range z
// stores its partial C into part[z][M][N] (float32); a later kernel adds the ranges in
// order.
struct EpiSplitPart {
  float* part;
  int M, N;
  __device__ void store(int row, int col, const float (&v)[16]) const {
    float* o = part + ((size_t)blockIdx.z * M + row) * N + col;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (col + j < N) o[j] = v[j];
  }
};

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
  int persist = 0;  // > 0: this many persistent CTAs (gemm_bf16_tc_persist_kernel)
  int mh = 1;       // persistent tiles of mh x 128 rows
  int splits = 1;   // one CTA per tile: K ranges per tile (gridDim.z), at most ceil(K / 64)
};

// Persistent CTAs for an M x N output in tiles of width bn: one per SM once there
// are at least two tiles per SM (0: one CTA per tile).
inline int gemm_persist_ctas(int M, int N, int bn, int sms, int mh = 1) {
  const long tiles = (long)((M + 128 * mh - 1) / (128 * mh)) * ((N + bn - 1) / bn);
  return (bn >= 128 && sms > 0 && tiles >= (mh == 2 ? 1L : 2L) * sms) ? sms : 0;
}

// Persistent geometry of an op whose tile width is set: 256 x 256 tiles where they
// give at least one tile per SM (their operand traffic per flop is the lower), else
// 128 x bn tiles where there are two per SM, else one CTA per tile.
inline void gemm_set_persist(GemmOp* op, int sms) {
  op->mh = 1;
  op->persist = 0;
  if (op->bn == 256 && gemm_persist_ctas(op->M, op->N, 256, sms, 2) > 0) {
    op->mh = 2;
    op->persist = sms;
  } else {
    op->persist = gemm_persist_ctas(op->M, op->N, op->bn, sms);
  }
}

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
  dim3 grid((op.N + BN - 1) / BN, (op.M + 127) / 128, op.splits > 1 ? op.splits : 1);
  return launch_k(kern, grid, dim3(128), C::SMEM, st, pdl, op.a, op.b, op.M, op.N, op.K, epi, err, wait_limit);
}

template <int BN, int STAGES, int MH, class Epi>
cudaError_t gemm_launch_persist(const GemmOp& op, const Epi& epi, cudaStream_t st, unsigned* err, bool pdl,
                                uint32_t wait_limit) {
  using C = GemmPCfg<BN, STAGES, MH>;
  auto kern = gemm_bf16_tc_persist_kernel<BN, STAGES, MH, Epi>;
  cudaError_t e = raise_dyn_smem((const void*)kern, C::SMEM);
  if (e != cudaSuccess) return e;
  return launch_k(kern, dim3(op.persist), dim3(192), C::SMEM, st, pdl, op.a, op.b, op.M, op.N, op.K, epi, err,
                  wait_limit);
}

// wait_limit: tries of each pipeline wait before it gives up (tc::WAIT_LIMIT by default).
template <class Epi>
cudaError_t gemm_launch(const GemmOp& op, const Epi& epi, cudaStream_t st, unsigned* err, bool pdl = false,
                        uint32_t wait_limit = tc::WAIT_LIMIT) {
  if (op.persist > 0 && op.bn == 256 && op.mh == 2)
    return gemm_launch_persist<256, 3, 2>(op, epi, st, err, pdl, wait_limit);
  if (op.persist > 0 && op.bn == 256) return gemm_launch_persist<256, 4, 1>(op, epi, st, err, pdl, wait_limit);
  if (op.persist > 0 && op.bn == 128) return gemm_launch_persist<128, 5, 1>(op, epi, st, err, pdl, wait_limit);
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
