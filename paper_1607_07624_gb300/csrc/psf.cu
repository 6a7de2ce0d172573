// PSF camera: point-spread function and Strehl ratio of the residual field (Table 1
// camera: wavelengthInNm, nd "padding coefficient for PSF computation"; Table 2
// psf.in_ef, psf.out_sr, psf.out_int_psf; Sec. GPU acceleration, "PSF generation from
// residual wavefront").
//
// E = A exp(2 pi i opd / lambda) on the Np x Np pupil, zero-padded to N = nd Np, and
// PSF(p, q) = |F(p, q)|^2 / (sum A)^2 with F the 2-D DFT of E (-1)^(i+j): the sign
// moves the zero frequency to (N/2, N/2), where a diffraction-limited pupil peaks at
// exactly 1 and where the Strehl ratio is read.
//
// The padding is used, not transformed: a length-N DFT of a sequence that is zero
// beyond Np samples gives at frequency k = nd m + r the length-Np DFT of
// x[n] exp(-2 pi i r n / N) at m. So each padded 1-D transform is nd warp FFTs of
// length Np (fft.cuh), one per residue r: first along axis 0 for the Np pupil
// columns (spectrum written transposed, H[p][j]), then along axis 1 for the N
// frequency rows, whose nd residues meet in shared memory and leave as one
// coalesced row of |F|^2. Pupils of 240 and 480 px run two transforms per warp
// through the four-step engine of fft4.cuh (pair_forward); the others one per warp
// through the pass-by-pass engine.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <vector>

#include "fft.cuh"
#include "fft4.cuh"
#include "fft_host.h"
#include "internal.h"
#include "pdl.cuh"
#include "phasor.cuh"
#include "psf.cuh"

namespace pas {

constexpr int PSF_COLS_WARPS = 8;  // pupil columns per CTA of the first pass (a power of two)
constexpr int PSF_MAX_ND = 16;

struct PsfArgs {
  const float* opd;     // [Np][Np] nm
  const float2* tw;     // per-pass twiddles of the length-Np FFT
  const int* pos;       // [Np] buffer position holding frequency m after fft_forward
  const float2* rot;    // [nd][Np] exp(-2 pi i r n / N)
  float2* H;            // [N][Np] spectra of the pupil columns along axis 0
  float* psf;           // [N][N]
  double* strehl;       // scalar or null (with `step`: a ring of sr_len entries)
  int nd, T_obs, accumulate;
  float inv_hi, inv_lo;  // 1/lambda split in two floats
  float norm;            // 1 / (sum A)^2
  // a camera inside a loop's step: nothing before step `start`; the Strehl ratio of
  // step t goes to strehl[t mod sr_len]
  const long long* step = nullptr;
  long long start = 0;
  int sr_len = 1;
};

template <int NP>
__device__ __forceinline__ void psf_stage_tables(const PsfArgs& a, float2* tw_s, int* pos_s) {
  for (int t = threadIdx.x; t < tw_size(NP); t += blockDim.x) tw_s[t] = a.tw[t];
  for (int t = threadIdx.x; t < NP; t += blockDim.x) pos_s[t] = a.pos[t];
}

// One row of |F|^2 (sum A)^-2 from shared memory to the PSF, written or added: as
// float4 where both rows are 16-byte aligned (every N = nd Np a multiple of 4), the old
// values of an integrated PSF loaded RW at a time before their adds, so that RW memory
// latencies overlap instead of one per element.
__device__ __forceinline__ void psf_write_row(float* out, const float* row, int N, bool acc) {
  constexpr int RW = 4;
  if ((N & 3) == 0 && ((reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(row)) & 15) == 0) {
    const int n4 = N >> 2;
    float4* o4 = reinterpret_cast<float4*>(out);
    const float4* r4 = reinterpret_cast<const float4*>(row);
    for (int q0 = threadIdx.x; q0 < n4; q0 += RW * blockDim.x) {
      float4 old[RW];
#pragma unroll
      for (int u = 0; u < RW; ++u) {
        const int q = q0 + u * blockDim.x;
        old[u] = acc && q < n4 ? o4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < RW; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q < n4) {
          float4 v = r4[q];
          if (acc)
            v = make_float4(__fadd_rn(old[u].x, v.x), __fadd_rn(old[u].y, v.y), __fadd_rn(old[u].z, v.z),
                            __fadd_rn(old[u].w, v.w));
          o4[q] = v;
        }
      }
    }
    return;
  }
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    const float val = row[q];
    out[q] = acc ? __fadd_rn(out[q], val) : val;
  }
}

// The paired rows pass keeps its row padded by one word per 32 (entry q at q + q / 32):
// its lanes store frequencies nd apart, which would otherwise meet in a few banks. The
// write-out reads four consecutive entries (never split by the padding) per float4.
__device__ __forceinline__ int psf_pad(int q) { return q + (q >> 5); }

__device__ __forceinline__ void psf_write_row_padded(float* out, const float* row, int N, bool acc) {
  constexpr int RW = 4;
  const int n4 = N >> 2;  // N = nd Np, Np 240 or 480: a multiple of 4; rows 16-byte aligned
  float4* o4 = reinterpret_cast<float4*>(out);
  for (int q0 = threadIdx.x; q0 < n4; q0 += RW * blockDim.x) {
    float4 old[RW];
#pragma unroll
    for (int u = 0; u < RW; ++u) {
      const int q = q0 + u * blockDim.x;
      old[u] = acc && q < n4 ? o4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < RW; ++u) {
      const int q = q0 + u * blockDim.x;
      if (q < n4) {
        const float* r = row + psf_pad(4 * q);
        float4 v = make_float4(r[0], r[1], r[2], r[3]);
        if (acc)
          v = make_float4(__fadd_rn(old[u].x, v.x), __fadd_rn(old[u].y, v.y), __fadd_rn(old[u].z, v.z),
                          __fadd_rn(old[u].w, v.w));
        o4[q] = v;
      }
    }
  }
}

// Pass 1: CTA (column block, residue r), one warp per pupil column j, transform
// along axis 0 of A e^{i phi} (-1)^(i+j) e^{-2 pi i r i / N}.
template <int NP>
__global__ void __launch_bounds__(PSF_COLS_WARPS * 32) psf_cols_kernel(PsfArgs a) {
  constexpr int TWN = tw_size(NP), PITCH = buf_len(NP) | 1;
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  int* pos_s = reinterpret_cast<int*>(smem + TWN);
  float2* bufs = smem + TWN + (NP + 1) / 2;  // after pos_s (NP ints)
  pdl_trigger();
  if (a.step && *a.step < a.start) return;  // the camera has not started (uniform)
  psf_stage_tables<NP>(a, tw_s, pos_s);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.y, nd = a.nd;
  const int j0 = blockIdx.x * PSF_COLS_WARPS, j = j0 + warp;
  float2* buf = bufs + warp * PITCH;
  const float2* rot = a.rot + (size_t)r * NP;
  if (j < NP) {
    const int bj = 2 * j - NP + 1;
    auto load = [&](int, int, int x) -> float2 {
      const int ai = 2 * x - NP + 1;
      const int d2 = ai * ai + bj * bj;
      if (d2 > NP * NP || d2 < a.T_obs) return make_float2(0.f, 0.f);
      float2 v = opd_phasor(__ldg(a.opd + (size_t)x * NP + j), a.inv_hi, a.inv_lo);
      if ((x + j) & 1) v = make_float2(-v.x, -v.y);
      return cmul(v, __ldg(rot + x));
    };
    fft_forward<NP>(buf, tw_s, lane, load);
  }
  __syncthreads();
  // transposed write H[nd m + r][j0 + w]: 8 x 8 contiguous bytes per frequency
  constexpr int LG = PSF_COLS_WARPS == 8 ? 3 : PSF_COLS_WARPS == 4 ? 2 : PSF_COLS_WARPS == 2 ? 1 : 0;
  static_assert((1 << LG) == PSF_COLS_WARPS, "PSF_COLS_WARPS must be 1, 2, 4 or 8");
  for (int idx = threadIdx.x; idx < NP * PSF_COLS_WARPS; idx += blockDim.x) {
    const int w = idx & (PSF_COLS_WARPS - 1), m = idx >> LG;
    if (j0 + w < NP) a.H[((size_t)nd * m + r) * NP + j0 + w] = bufs[w * PITCH + phys(pos_s[m])];
  }
}

// Pass 2: CTA = one frequency row p, warp r = residue; |F|^2 (sum A)^-2 gathered in
// shared memory at q = nd m + r and written (or added) as one row.
template <int NP>
__global__ void psf_rows_kernel(PsfArgs a) {
  constexpr int TWN = tw_size(NP), PITCH = buf_len(NP) | 1;
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  int* pos_s = reinterpret_cast<int*>(smem + TWN);
  float2* bufs = smem + TWN + (NP + 1) / 2;
  const int nd = a.nd, N = nd * NP;
  float* row = reinterpret_cast<float*>(bufs + nd * PITCH);  // [N]
  pdl_wait();  // H (and the step counter's value) come from the predecessors
  long long t = 0;
  if (a.step) {
    t = *a.step;
    if (t < a.start) return;  // uniform
  }
  psf_stage_tables<NP>(a, tw_s, pos_s);
  __syncthreads();
  const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x;
  float2* buf = bufs + r * PITCH;
  const float2* Hrow = a.H + (size_t)p * NP;
  const float2* rot = a.rot + (size_t)r * NP;
  auto load = [&](int, int, int x) -> float2 { return cmul(__ldg(Hrow + x), __ldg(rot + x)); };
  fft_forward<NP>(buf, tw_s, lane, load);
  for (int m = lane; m < NP; m += 32) {
    const float2 v = buf[phys(pos_s[m])];
    row[nd * m + r] = __fmul_rn(__fmaf_rn(v.x, v.x, __fmul_rn(v.y, v.y)), a.norm);
  }
  __syncthreads();
  psf_write_row(a.psf + (size_t)p * N, row, N, a.accumulate != 0);
  if (a.strehl && p == N / 2 && threadIdx.x == 0) a.strehl[a.step ? t % a.sr_len : 0] = (double)row[N / 2];
}

// Pupils of 240 and 480 px: the same two passes with two transforms per warp
// (pair_forward, fft4.cuh: frequencies in natural order, no position table).
// Pass 1: CTA = PSF_PAIR_COLS pupil column(s) x every residue. The CTA forms the field
// A e^{i phi} (-1)^(i+j) of its columns once in shared memory (one phasor per pixel
// for all nd residues); warp w takes column j0 + w / nw and residues 2 (w % nw) and
// 2 (w % nw) + 1 (nw = ceil(nd / 2); a missing second residue of an odd nd transforms
// zeros and stores nothing); lanes write H[nd m + r][j] directly.
constexpr int PSF_PAIR_COLS = 1;

template <int NP>
__global__ void __launch_bounds__(PSF_PAIR_COLS * 8 * 32) psf_cols_pair_kernel(PsfArgs a) {
  extern __shared__ float2 smem[];
  pdl_trigger();
  if (a.step && *a.step < a.start) return;  // the camera has not started (uniform)
  const int nd = a.nd, nw = (nd + 1) / 2;
  const int j0 = blockIdx.x * PSF_PAIR_COLS;
  // the constant tables the transforms read (L1), fetched under the field's latency
  prefetch_l1_span(a.rot, sizeof(float2) * (size_t)nd * NP);
  prefetch_l1_span(a.tw, sizeof(float2) * pair_tw_size(NP));
  float2* E = smem;                                    // [PSF_PAIR_COLS][NP]
  float2* Tb = smem + PSF_PAIR_COLS * NP;              // [warps][pair_buf]
  for (int e = threadIdx.x; e < PSF_PAIR_COLS * NP; e += blockDim.x) {
    const int c = e / NP, x = e - c * NP, j = j0 + c;
    const int ai = 2 * x - NP + 1, bj = 2 * j - NP + 1;
    const int d2 = ai * ai + bj * bj;
    float2 v = make_float2(0.f, 0.f);
    if (j < NP && d2 <= NP * NP && d2 >= a.T_obs) {
      v = opd_phasor(__ldg(a.opd + (size_t)x * NP + j), a.inv_hi, a.inv_lo);
      if ((x + j) & 1) v = make_float2(-v.x, -v.y);
    }
    E[e] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = warp / nw, rp = warp - c * nw, j = j0 + c;
  float2* T = Tb + warp * pair_buf(NP);
  const float2* Ec = E + c * NP;
  auto load = [&](int t, int x) -> float2 {
    const int r = 2 * rp + t;
    if (r >= nd) return make_float2(0.f, 0.f);
    return cmul(Ec[x], __ldg(a.rot + (size_t)r * NP + x));
  };
  auto store = [&](int t, int m, float2 v) {
    const int r = 2 * rp + t;
    if (r < nd && j < NP) a.H[((size_t)nd * m + r) * NP + j] = v;
  };
  pair_forward<NP>(T, a.tw, lane, load, store);
}

// Pass 2: CTA = one frequency row p, warp w = residues w and w + nw (nw = ceil(nd / 2);
// a missing second residue of an odd nd transforms zeros and stores nothing: with
// residues nw apart the pair's 30 lanes store to 30 distinct banks at nd = 8);
// |F|^2 (sum A)^-2 gathered in shared memory at q = nd m + r (padded) and written (or
// added) as one row.
template <int NP>
__global__ void __launch_bounds__(256) psf_rows_pair_kernel(PsfArgs a) {
  extern __shared__ float2 smem[];
  const int nd = a.nd, N = nd * NP, nw = (nd + 1) / 2;
  float* row = reinterpret_cast<float*>(smem + nw * pair_buf(NP));  // [N]
  // before the wait, for an integrated PSF: this row's old values into L2 (the previous
  // frame's rows pass completed before this frame's columns pass started)
  if (a.accumulate) {
    const char* o = reinterpret_cast<const char*>(a.psf + (size_t)blockIdx.x * N);
    for (int l = threadIdx.x * 128; l < N * 4; l += blockDim.x * 128) prefetch_l2(o + l);
  }
  pdl_wait();  // H (and the step counter's value) come from the predecessors
  long long t = 0;
  if (a.step) {
    t = *a.step;
    if (t < a.start) return;  // uniform
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x;
  float2* T = smem + warp * pair_buf(NP);
  const float2* Hrow = a.H + (size_t)p * NP;
  auto load = [&](int tt, int x) -> float2 {
    const int r = warp + nw * tt;
    if (r >= nd) return make_float2(0.f, 0.f);
    return cmul(__ldg(Hrow + x), __ldg(a.rot + (size_t)r * NP + x));
  };
  auto store = [&](int tt, int m, float2 v) {
    const int r = warp + nw * tt;
    if (r < nd) row[psf_pad(nd * m + r)] = __fmul_rn(__fmaf_rn(v.x, v.x, __fmul_rn(v.y, v.y)), a.norm);
  };
  pair_forward<NP>(T, a.tw, lane, load, store);
  __syncthreads();
  psf_write_row_padded(a.psf + (size_t)p * N, row, N, a.accumulate != 0);
  if (a.strehl && p == N / 2 && threadIdx.x == 0)
    a.strehl[a.step ? t % a.sr_len : 0] = (double)row[psf_pad(N / 2)];
}

struct PsfKernels {
  void (*cols)(PsfArgs);
  void (*rows)(PsfArgs);
  int tw_n, pitch;
  bool pair;  // pair_forward kernels: tw_n = pair_tw_size, pitch = pair_buf per warp
};

#define PAS_PSF_PUPILS(X) X(48) X(64) X(120) X(128) X(256)

static bool lookup_psf_kernels(int Np, PsfKernels* k) {
  switch (Np) {
    case 240:
      *k = PsfKernels{psf_cols_pair_kernel<240>, psf_rows_pair_kernel<240>, pair_tw_size(240), pair_buf(240), true};
      return true;
    case 480:
      *k = PsfKernels{psf_cols_pair_kernel<480>, psf_rows_pair_kernel<480>, pair_tw_size(480), pair_buf(480), true};
      return true;
#define PAS_CASE(n)                                                                             \
  case n:                                                                                       \
    *k = PsfKernels{psf_cols_kernel<n>, psf_rows_kernel<n>, tw_size(n), buf_len(n) | 1, false}; \
    return true;
    PAS_PSF_PUPILS(PAS_CASE)
#undef PAS_CASE
    default:
      return false;
  }
}

// W_N^(n1 k2) = exp(-2 pi i n1 k2 / N) at [(k2 - 1) R + n1], k2 = 1..14, n1 < R = N / 15
// (pair_forward's table), float32 of the double value.
static std::vector<float2> pair_twiddles(int N) {
  const int R = pair_r(N);
  std::vector<float2> tw((size_t)pair_tw_size(N));
  for (int k2 = 1; k2 < 15; ++k2)
    for (int n1 = 0; n1 < R; ++n1) {
      const double a = -2.0 * M_PI * (double)(n1 * k2) / (double)N;
      tw[(size_t)(k2 - 1) * R + n1] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  return tw;
}

}  // namespace pas

struct pas_psf_s {
  pas_ctx_t ctx = nullptr;
  int Np = 0, nd = 0, N = 0, T_obs = 0;
  float inv_hi = 0.f, inv_lo = 0.f, norm = 0.f;
  pas::PsfKernels kern{};
  size_t smem_cols = 0, smem_rows = 0;
  float2* d_tw = nullptr;
  int* d_pos = nullptr;
  float2* d_rot = nullptr;
  float2* d_H = nullptr;
};

extern "C" {

void pas_psf_destroy(pas_psf_t P) {
  if (!P) return;
  pas::dev_free(P->d_tw);
  pas::dev_free(P->d_pos);
  pas::dev_free(P->d_rot);
  pas::dev_free(P->d_H);
  delete P;
}

pas_status pas_psf_create(pas_ctx_t ctx, int32_t Np, int32_t nd, double wavelength_nm, double obs,
                          pas_psf_t* out) {
  if (!ctx || !out) return pas::set_global_error(PAS_EINVAL, "pas_psf_create: NULL argument");
  *out = nullptr;
  PAS_CHECK_ARG(ctx, Np > 0 && nd >= 1 && nd <= pas::PSF_MAX_ND && wavelength_nm > 0 && obs >= 0 && obs < 1,
                "pas_psf_create: need Np > 0, 1 <= nd <= 16, wavelength > 0, 0 <= obs < 1");
  pas::PsfKernels kern;
  if (!pas::lookup_psf_kernels(Np, &kern))
    return pas::set_error(ctx, PAS_EINVAL, "pas_psf_create: pupil of %d px not supported", Np);
  int32_t n_pup = 0;
  pas_pupil_mask(Np, obs, nullptr, &n_pup);
  PAS_CHECK_ARG(ctx, n_pup > 0, "pas_psf_create: empty pupil");
  const int N = Np * nd;

  pas_psf_t P = new pas_psf_s();
  P->ctx = ctx;
  P->Np = Np;
  P->nd = nd;
  P->N = N;
  P->kern = kern;
  P->T_obs = (int)pas::obstruction_threshold(Np, obs);
  const double inv = 1.0 / wavelength_nm;
  P->inv_hi = (float)inv;
  P->inv_lo = (float)(inv - (double)P->inv_hi);
  P->norm = (float)(1.0 / ((double)n_pup * (double)n_pup));
  std::vector<float2> tw;
  std::vector<int> pos(Np, 0);
  if (kern.pair) {
    // no staged tables: per warp one transpose buffer; the rows pass adds its row
    P->smem_cols = sizeof(float2) * ((size_t)pas::PSF_PAIR_COLS * Np +
                                     (size_t)pas::PSF_PAIR_COLS * ((nd + 1) / 2) * kern.pitch);
    P->smem_rows = sizeof(float2) * ((size_t)((nd + 1) / 2) * kern.pitch) + sizeof(float) * ((size_t)N + N / 32 + 1);
    tw = pas::pair_twiddles(Np);
  } else {
    const size_t tables = sizeof(float2) * ((size_t)kern.tw_n + (size_t)(Np + 1) / 2);
    P->smem_cols = tables + sizeof(float2) * (size_t)pas::PSF_COLS_WARPS * kern.pitch;
    P->smem_rows = tables + sizeof(float2) * ((size_t)nd * kern.pitch + (size_t)(N + 1) / 2);
    tw = pas::fft_twiddles(Np);
    for (int p = 0; p < Np; ++p) pos[pas::fft_freq_at(Np, p)] = p;
  }
  std::vector<float2> rot((size_t)nd * Np);
  for (int r = 0; r < nd; ++r)
    for (int n = 0; n < Np; ++n) {
      const double a = -2.0 * M_PI * (double)((long long)r * n % N) / (double)N;
      rot[(size_t)r * Np + n] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  pas_status st = PAS_OK;
  auto A = [&](void** ptr, size_t bytes) {
    if (st == PAS_OK) st = pas::dev_alloc(ctx, ptr, bytes);
  };
  A((void**)&P->d_tw, sizeof(float2) * tw.size());
  A((void**)&P->d_pos, sizeof(int) * Np);
  A((void**)&P->d_rot, sizeof(float2) * rot.size());
  A((void**)&P->d_H, sizeof(float2) * (size_t)N * Np);
  if (st != PAS_OK) {
    pas_psf_destroy(P);
    return st;
  }
  cudaError_t e = cudaMemcpy(P->d_tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P->d_pos, pos.data(), sizeof(int) * Np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P->d_rot, rot.data(), sizeof(float2) * rot.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = pas::raise_dyn_smem((const void*)kern.cols, P->smem_cols);
  if (e == cudaSuccess) e = pas::raise_dyn_smem((const void*)kern.rows, P->smem_rows);
  if (e != cudaSuccess) {
    pas_psf_destroy(P);
    return pas::set_error(ctx, PAS_ECUDA, "pas_psf_create: %s", cudaGetErrorString(e));
  }
  *out = P;
  return PAS_OK;
}

int32_t pas_psf_size(pas_psf_t P) { return P ? P->N : -1; }

}  // extern "C"

namespace pas {

pas_status psf_launch(pas_psf_t P, const float* d_opd, float* d_psf, int accumulate, double* d_strehl,
                      const long long* d_step, long long start, int sr_len, cudaStream_t st) {
  PsfArgs a;
  a.opd = d_opd;
  a.tw = P->d_tw;
  a.pos = P->d_pos;
  a.rot = P->d_rot;
  a.H = P->d_H;
  a.psf = d_psf;
  a.strehl = d_strehl;
  a.nd = P->nd;
  a.T_obs = P->T_obs;
  a.accumulate = accumulate ? 1 : 0;
  a.inv_hi = P->inv_hi;
  a.inv_lo = P->inv_lo;
  a.norm = P->norm;
  a.step = d_step;
  a.start = start;
  a.sr_len = sr_len;
  cudaError_t e;
  if (P->kern.pair) {
    e = launch_k(P->kern.cols, dim3((P->Np + PSF_PAIR_COLS - 1) / PSF_PAIR_COLS),
                 dim3(PSF_PAIR_COLS * ((P->nd + 1) / 2) * 32), P->smem_cols, st, false, a);
    if (e == cudaSuccess)
      e = launch_k(P->kern.rows, dim3(P->N), dim3((P->nd + 1) / 2 * 32), P->smem_rows, st, true, a);
  } else {
    e = launch_k(P->kern.cols, dim3((P->Np + PSF_COLS_WARPS - 1) / PSF_COLS_WARPS, P->nd),
                 dim3(PSF_COLS_WARPS * 32), P->smem_cols, st, false, a);
    if (e == cudaSuccess) e = launch_k(P->kern.rows, dim3(P->N), dim3(P->nd * 32), P->smem_rows, st, true, a);
  }
  if (e != cudaSuccess) return set_error(P->ctx, PAS_ECUDA, "PSF camera launch: %s", cudaGetErrorString(e));
  return PAS_OK;
}

int psf_np(pas_psf_t P) { return P->Np; }

}  // namespace pas

extern "C" {

pas_status pas_psf_compute(pas_psf_t P, const float* d_opd, float* d_psf, int32_t accumulate, double* d_strehl) {
  if (!P || !d_opd || !d_psf) return pas::set_global_error(PAS_EINVAL, "pas_psf_compute: NULL argument");
  return pas::psf_launch(P, d_opd, d_psf, accumulate, d_strehl, nullptr, 0, 1, P->ctx->stream);
}

}  // extern "C"
