// Modulated four-face pyramid WFS, CCD binning/noise and slope computer
// (Table 1 pyramid / detector / slopec; Sec. GPU acceleration, "pyramid
// propagation from wavefront to detector plane").
//
// The centred DFT, the pyramid mask |u~| + |v~| and the modulation tilt are all
// separable, so for modulation point k the pupil-plane field after the pyramid is
//   g_k = A diag(tx_k) E0 diag(ty_k) A^T,   A = IDFT diag(p) DFT  (1-D, N x N),
// with E0 the embedded pupil field. Two passes compute it:
//   rows pass: for each pupil row i and each distinct sin(theta_k):
//              phasor * tilt_y -> FFT -> p(u)/N -> IFFT  => H_s[y][i] (transposed);
//   cols pass: for each column y and each k: H_s(k)[y][:] * tilt_x -> FFT -> p/N ->
//              IFFT -> |.|^2, accumulated over the CTA's k and binned b x b.
// The centring ramps of the DFT reduce to (-1)^x exp(-i pi x / N) on the input
// and a unit-modulus ramp on the output; the output ramp of each pass is a
// per-row/column constant of the next pass and vanishes in |.|^2, so only the
// input ramp is kept (merged into the tilt phases alpha_k, beta_s).
// Modulation points with equal sin(theta) (theta and pi - theta) share a rows pass.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "fft.cuh"
#include "fft4.cuh"
#include "fft_host.h"
#include "internal.h"
#include "noise.cuh"
#include "pdl.cuh"
#include "phasor.cuh"
#include "pyr.cuh"
#include "pyr_host.h"
#include "wfe.cuh"

namespace pas {

constexpr int MAX_ROWS_PER_CTA = 8;  // rows pass: one warp per pupil row
// A rows-pass CTA of 16 rows (512 threads at the 128-register cap: the whole register
// file of an SM), where its shared memory fits: the per-warp phasor row and transpose
// buffer, not the registers, then bound the warps per SM.
constexpr int ROWS_WIDE = 16;
constexpr size_t SMEM_MAX = 227 * 1024;  // opt-in dynamic shared memory of one CTA

struct RowArgs {
  const float* opd;     // [Np][Np]
  const float2* tw;     // [N]
  const float2* mask;   // [N] digit-reversed
  const float2* tw4;    // four-step engine tables (N = 480, 960)
  const float2* mk4;
  const float* beta;    // [n_s] cycles per pixel (tilt_y + input ramp)
  float2* H;            // [n_s][N][Np]
  int Np, off;
  int n_s, s_chunk;     // distinct sin values; at most s_chunk per CTA
  int T_obs;            // obstruction threshold (integer)
  float inv_hi, inv_lo; // 1/lambda split in two floats
};

// Detector frame, noise and slopes, done by the last CTAs of the columns pass.
struct FrameArgs {
  float* frame;                // [nd*nd]
  const unsigned char* vpix;   // [nd*nd] 1: quadrant pixel of a valid sub-aperture
  double* flux_part;           // [nd] per detector column
  unsigned int* done_col;      // [nd] CTA completion counters (0 between launches)
  long long* frame_ctr;
  int ctr_increment;
  int G, np;
  float invK, scale, ron;
  unsigned long long seed;
  const int* valid;
  const float* sn;             // [2nv] or null
  float* slopes;               // [2nv] or null
  int nv, n_sub, local_norm;
  LoopExtra wfe;               // wfe.wfe_part null: no WFE
};

struct ColArgs {
  const float2* H;
  const float2* tw;
  const float2* mask;
  const float2* tw4;    // four-step engine (N = 480, 960): W_N^(n1 k2) [(Q-1)][32]
  const float2* mk4;    // and the mask by natural frequency [Q][33]
  const float2* tilt;   // [K][Np] (-1)^i exp(2 pi i (i - ci) alpha_k): tilt_x + input ramp
  const int* kmap;      // [K] -> rows-pass index
  float* part;          // [G][nd][nd]
  int Np, off, K, kper, nd, b;  // b: fine columns of one detector column (integer binning)
  int split;            // CTAs per detector column and group, each b / split fine columns
  int frac;             // detector pixels of N / nd fine pixels, N / nd not an integer
  FrameArgs fin;
};

// Where one loop's tasks sit in a persistent batched launch's ticket queue, and the
// geometry of its own two passes.
struct BatchLoopGeo {
  int row_base, n_row;  // tickets [row_base, row_base + n_row): rows-pass tasks
  int nbx, rows;        // rows pass: nbx x (n_row / nbx) CTAs of `rows` warps
  int col_base, n_col;  // tickets of the columns-pass tasks
  int nd, bw;           // columns pass: nd x (n_col / nd) CTAs of bw warps
};

struct BatchPyrArgs {
  const RowArgs* ra;             // [L]
  const ColArgs* ca;             // [L]
  const BatchLoopGeo* geo;       // [L]
  unsigned int* ticket;          // next ticket, 0 before the launch
  unsigned int* rows_done;       // [L] completed rows-pass tasks, 0 before the launch
  unsigned int* err;             // bit 0: a columns-pass task's wait gave up
  const long long* wait_limit;   // polls (about 0.3 us each) before a wait gives up
  int n_loops, n_row_tickets, n_tickets, first_ticket;
};



// Register caps per transform length: 72 for N = 480 compiles without spills and
// lets 3 columns-pass CTAs of 8 warps (and 7 rows-pass CTAs of 4 warps) share an SM
// instead of 2 (4); other lengths keep the compiler's choice.
constexpr int rows_max_regs(int N) { return 128; }
constexpr int cols_max_regs(int N) { return 128; }

// One rows-pass task: pupil rows [bx rows, (bx + 1) rows) and the bx-th of nby chunks of
// the distinct sin values, by warps 0 .. rows-1 of the CTA (rows a power of two <= the
// CTA's warps; further warps take part in the barriers only).
template <int N>
__device__ __forceinline__ void rows_task(const RowArgs& a, int bx, int by, int nby, int rows) {
  constexpr bool FOUR = four_step_ok(N);
  constexpr int TWN = FOUR ? four_tw_size(N) : tw_size(N);
  constexpr int MKN = FOUR ? four_mask_size(N) : buf_len(N);
  constexpr int PITCH = FOUR ? four_buf(N) : (buf_len(N) | 1);
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  float2* mk_s = smem + TWN;
  float2* tilt_s = mk_s + MKN;                      // [s_chunk][Np]
  float2* phs = tilt_s + a.s_chunk * a.Np;          // [rows][Np]
  float2* bufs = phs + rows * a.Np;                 // [rows][PITCH]
  const int Np = a.Np, off = a.off;
  const int i0 = bx * rows;
  const int s0 = (by * a.n_s) / nby, s1 = ((by + 1) * a.n_s) / nby;
  pdl_trigger();
  {
    const float2* twg = FOUR ? a.tw4 : a.tw;
    const float2* mkg = FOUR ? a.mk4 : a.mask;
    for (int t = threadIdx.x; t < TWN; t += blockDim.x) tw_s[t] = twg[t];
    for (int t = threadIdx.x; t < MKN; t += blockDim.x) mk_s[t] = mkg[t];
  }
  // tilt along the row (with the input centring ramp and (-1)^j) per sin value
  const float cj = 0.5f * (float)(Np - 1);
  for (int t = threadIdx.x; t < (s1 - s0) * Np; t += blockDim.x) {
    const int sl = t / Np, j = t - sl * Np;
    float sn, cs;
    sincospif(2.0f * ((float)j - cj) * a.beta[s0 + sl], &sn, &cs);
    tilt_s[t] = (j & 1) ? make_float2(-cs, -sn) : make_float2(cs, sn);
  }
  const int warp_raw = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool row_warp = warp_raw < rows;
  const int warp = row_warp ? warp_raw : 0;
  const int i = row_warp ? i0 + warp : Np;      // a warp beyond `rows` owns no row
  float2* buf = bufs + warp * PITCH;
  // pupil phasor A exp(2 pi i opd / lambda) of this warp's row, kept for all s
  float2* phrow = phs + warp * Np;
  pdl_wait();  // the OPD comes from the predecessor
  {
    const int ai = 2 * i - Np + 1;
    const int ai2 = ai * ai;
    const float* orow = a.opd + (size_t)min(i, Np - 1) * Np;
    for (int j = lane; j < Np && row_warp; j += 32) {
      float2 v = make_float2(0.f, 0.f);
      const int bj = 2 * j - Np + 1;
      const int d2 = ai2 + bj * bj;
      if (i < Np && d2 <= Np * Np && d2 >= a.T_obs) v = opd_phasor(__ldg(orow + j), a.inv_hi, a.inv_lo);
      phrow[j] = v;
    }
  }
  __syncthreads();
  const int nr = min(rows, Np - i0);
  const int lg = __ffs(rows) - 1;
  constexpr int TPW = FOUR ? four_tpw(N) : 1;   // sin values per engine call
  for (int s = s0; s < s1; s += TPW) {
    if (i < Np) {
      if constexpr (FOUR) {
        auto load = [&](int t, int jj) -> float2 {
          const int j = lane + 32 * jj - off;
          if ((unsigned)j < (unsigned)Np && s + t < s1) return cmul(phrow[j], tilt_s[(s + t - s0) * Np + j]);
          return make_float2(0.f, 0.f);
        };
        auto store = [&](int t, int jj, float2 v) { buf[t * N + lane + 32 * jj] = v; };
        four_step_mask<N>(buf, tw_s, mk_s, lane, load, store);
      } else {
        const float2* tl = tilt_s + (s - s0) * Np;
        auto load = [&](int, int, int x) -> float2 {
          const int j = x - off;
          if ((unsigned)j < (unsigned)Np) return cmul(phrow[j], tl[j]);
          return make_float2(0.f, 0.f);
        };
        auto store = [&](int, int, int x, float2 v) { buf[phys(x)] = v; };
        fft_mask_ifft<N>(buf, tw_s, mk_s, lane, load, store);
      }
    }
    __syncthreads();
    // transposed write: H[s][y][i0 + r], rows x 8 contiguous bytes per y (rows is a
    // power of two: index split by shift and mask)
    for (int t = 0; t < TPW && s + t < s1; ++t) {
      float2* Hs = a.H + (size_t)(s + t) * N * Np;
      for (int idx = threadIdx.x; idx < N * rows; idx += blockDim.x) {
        const int r = idx & (rows - 1), y = idx >> lg;
        if (r < nr) Hs[(size_t)y * Np + i0 + r] = FOUR ? bufs[r * PITCH + t * N + y] : bufs[r * PITCH + phys(y)];
      }
    }
    __syncthreads();
  }
}

template <int N>
__global__ void __maxnreg__(rows_max_regs(N))
pyr_rows_kernel(RowArgs a) {
  rows_task<N>(a, blockIdx.x, blockIdx.y, gridDim.y, blockDim.x >> 5);
}

// Block sum of one float per thread: float within each warp (fixed shuffle tree),
// the warps' sums added in double in warp order (FP64 is a slow pipe on this GPU,
// so it is kept out of the per-thread work). Result in every thread.
__device__ inline double block_sum_f(float v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = (double)v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    red[0] = t;
  }
  __syncthreads();
  return red[0];
}

// Column q of the detector: sum of the G groups' partials / K, noise, and the
// column's flux over the valid sub-apertures' pixels (run by the column's last CTA,
// on the step's critical path: the partials are fetched 8 at a time and summed in
// group order; g lanes per pixel share the photon-noise rejection loop).
// fidx: the frame counter, read by the caller before the handshake.
// nthreads: the threads that take pixels (the CTA's first nthreads, a multiple of 32;
// the others join the barriers and votes with no pixel).
__device__ __noinline__ void finish_column(const FrameArgs& f, const float* part, int q, int nd, double* red,
                              long long fidx, int nthreads) {
  constexpr int BATCH = 8;
  int g = 1;
  while (g < 8 && nd * g * 2 <= nthreads) g *= 2;
  float flux = 0.f;
  for (int t0 = 0; t0 < nd * g; t0 += nthreads) {  // the same trip count in every thread
    const int t = t0 + threadIdx.x;
    const int p = t / g, sub = t - p * g;
    const bool active = p < nd && (int)threadIdx.x < nthreads;
    const int pix = (active ? p : 0) * nd + q;
    const bool valid_pix = active && f.vpix[pix] != 0;
    float v = 0.f;
    if (active) {
      for (int g0 = 0; g0 < f.G; g0 += BATCH) {
        float tv[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) tv[u] = g0 + u < f.G ? __ldcg(part + (size_t)(g0 + u) * f.np + pix) : 0.f;
#pragma unroll
        for (int u = 0; u < BATCH; ++u) v += tv[u];  // + 0 leaves the partial sums unchanged
      }
    }
    v *= f.invK;
    if (f.wfe.n_int > 1) {  // the same branch in every thread of the CTA
      const float a = active ? __fadd_rn(__ldcg(f.wfe.acc + pix), v) : 0.f;
      if ((fidx + 1) % f.wfe.n_int != 0) {
        if (active && sub == 0) f.wfe.acc[pix] = a;
        continue;
      }
      if (active && sub == 0) f.wfe.acc[pix] = 0.f;
      v = __fdiv_rn(a, (float)f.wfe.n_int);  // the window's mean frame
    }
    v = noisy_pixel_group(v, f.scale, f.ron, f.seed, (uint32_t)pix, (uint64_t)fidx, sub, g, active);
    if (active && sub == 0) {
      f.frame[pix] = v;
      if (valid_pix) flux += v;
    }
  }
  const double col_flux = block_sum_f(flux, red);
  if (threadIdx.x == 0) {
    f.flux_part[q] = col_flux;
    f.done_col[q] = 0u;
  }
}

// Normalised slopes: every CTA forms the global flux from the per-column partials
// (fixed order) and computes its share of the valid sub-apertures; CTA 0 also
// closes the loop step's residual WFE and advances the frame counter.
__global__ void __launch_bounds__(256) slopes_kernel(FrameArgs f, int nd) {
  __shared__ double red[32];
  pdl_trigger();
  // Before the wait for the columns pass: the constants of this thread's slope and
  // the step's residual WFE, whose partials the residual kernel wrote before the
  // rows pass started (that kernel has completed).
  const int ns = f.n_sub;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const bool mine = f.slopes && j < f.nv;
  int i00 = 0, i01 = 0, i10 = 0, i11 = 0;
  float snx = 0.f, sny = 0.f;
  if (mine) {
    const int v = f.valid[j], r = v / ns, c = v - r * ns;
    i00 = r * nd + c;
    i01 = r * nd + ns + c;
    i10 = (ns + r) * nd + c;
    i11 = (ns + r) * nd + ns + c;
    if (f.sn) {
      snx = f.sn[j];
      sny = f.sn[f.nv + j];
    }
  }
  if (blockIdx.x == 0 && f.wfe.wfe_part) wfe_finalize(f.wfe, red);
  // a detector integrating several steps: no frame between read-outs, the slopes keep
  // their value (the step counter was advanced by the previous step's last kernel)
  const bool hold = f.wfe.n_int > 1 && f.frame_ctr && (*f.frame_ctr + 1) % f.wfe.n_int != 0;
  pdl_wait();
  if (hold) return;
  // the frame and the column fluxes: all loads in one round
  double fl = 0.0;
  for (int t = threadIdx.x; t < nd; t += blockDim.x) fl += f.flux_part[t];
  float q00 = 0.f, q01 = 0.f, q10 = 0.f, q11 = 0.f;
  if (mine) {
    q00 = f.frame[i00];
    q01 = f.frame[i01];
    q10 = f.frame[i10];
    q11 = f.frame[i11];
  }
  const float F = (float)(block_sum_f((float)fl, red) / (double)f.nv);
  if (mine) {
    const float den = f.local_norm ? (q00 + q01 + q10 + q11) : F;
    const float inv = 1.0f / den;
    f.slopes[j] = ((q10 + q11) - (q00 + q01)) * inv - snx;
    f.slopes[f.nv + j] = ((q01 + q11) - (q00 + q10)) * inv - sny;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && f.ctr_increment && f.frame_ctr) *f.frame_ctr += 1;
}

// Column tilt phasors of the modulation points, [K][Np]: (-1)^i e^{2 pi i (i - ci) alpha_k}
// (tilt along axis 0 with the input centring ramp). Constant for a geometry: built
// once at creation, in the same float arithmetic the columns pass used inline.
// amp (may be null): per-point amplitudes (an extended source's weights).
__global__ void tilt_table_kernel(const float* alpha, const float* amp, int K, int Np, float2* tilt) {
  const int k = blockIdx.x;
  if (k >= K) return;
  const float ci = 0.5f * (float)(Np - 1);
  const float al = alpha[k];
  const float am = amp ? amp[k] : 1.0f;
  for (int i = threadIdx.x; i < Np; i += blockDim.x) {
    float sn, cs;
    sincospif(2.0f * ((float)i - ci) * al, &sn, &cs);
    if (amp) {
      cs *= am;
      sn *= am;
    }
    tilt[(size_t)k * Np + i] = (i & 1) ? make_float2(-cs, -sn) : make_float2(cs, sn);
  }
}

// One columns-pass task: detector column q, modulation group x column part gh, by
// warps 0 .. bw-1 (the fine columns it transforms; further warps take part in the
// barriers only). skip: transform nothing (a persistent launch whose wait for the
// rows pass gave up still keeps the column handshake in step).
// H through the read-only cache (written by an earlier kernel), or (COH: written by
// other CTAs of the same persistent launch) by plain cached loads, which the task's
// acquire of its loop's rows-pass count (thread 0) and the barrier after it order after
// those writes
template <bool COH>
__device__ __forceinline__ float2 ld_h(const float2* p) {
  if constexpr (COH)
    return __ldca(p);
  else
    return __ldg(p);
}

template <int N, bool COH = false>
__device__ __forceinline__ void cols_task(const ColArgs& a, int q, int gh, int bw, bool skip = false) {
  // per-warp buffers: one transform's padded buffer (pass-by-pass engine) or the
  // four-step engine's transpose buffer; both then hold the warp's column of |g|^2
  constexpr bool FOUR = four_step_ok(N);
  constexpr int TWN = FOUR ? four_tw_size(N) : tw_size(N);
  constexpr int MKN = FOUR ? four_mask_size(N) : buf_len(N);
  constexpr int PITCH = FOUR ? four_buf(N) : (buf_len(N) | 1);
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  float2* mk_s = smem + TWN;
  float2* bufs = mk_s + MKN;                      // [b][PITCH]
  const int Np = a.Np;
  const int g = gh / a.split, h = gh - g * a.split;
  const int k0 = g * a.kper;
  const int kc = skip ? 0 : min(a.kper, a.K - k0);
  pdl_trigger();
  {
    const float2* twg = FOUR ? a.tw4 : a.tw;
    const float2* mkg = FOUR ? a.mk4 : a.mask;
    for (int t = threadIdx.x; t < TWN; t += blockDim.x) tw_s[t] = twg[t];
    for (int t = threadIdx.x; t < MKN; t += blockDim.x) mk_s[t] = mkg[t];
  }
  pdl_wait();  // H, the partial frames and the counters belong to the predecessors
  __syncthreads();  // twiddles and mask staged
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the fine columns overlapping detector column q: [q b, (q+1) b) exactly when b is an
  // integer, of which this CTA takes part h of `split`; [floor(q N/nd), ceil((q+1) N/nd))
  // otherwise (the edge columns are shared with the neighbouring detector columns and
  // transformed by both CTAs)
  const int y0 = a.frac ? (q * N) / a.nd : q * a.b + h * bw;
  const int nw = a.frac ? ((q + 1) * N + a.nd - 1) / a.nd - y0 : bw;
  const int y = y0 + warp;
  float2* buf = bufs + min(warp, bw - 1) * PITCH;  // warps >= bw transform nothing (nw <= bw)
  float* accw = reinterpret_cast<float*>(buf);
  if constexpr (FOUR) {
    // lane l accumulates |g|^2 of rows l + 32 j; TPW modulation points per call (a
    // missing second point of an odd count transforms zeros)
    constexpr int Q = four_q(N), TPW = four_tpw(N);
    float acc[Q];
#pragma unroll
    for (int t = 0; t < Q; ++t) acc[t] = 0.f;
    for (int kk = 0; kk < (warp < nw ? kc : 0); kk += TPW) {
      const float2* Hcol[TPW];
      const float2* tk[TPW];
#pragma unroll
      for (int t = 0; t < TPW; ++t) {
        const int kt = min(kk + t, kc - 1);
        Hcol[t] = a.H + ((size_t)a.kmap[k0 + kt] * N + y) * Np;
        tk[t] = a.tilt + (size_t)(k0 + kt) * Np;
      }
      const int off = a.off;
      auto load = [&](int t, int j) -> float2 {
        const int i = lane + 32 * j - off;
        if ((unsigned)i < (unsigned)Np && kk + t < kc) return cmul(ld_h<COH>(Hcol[t] + i), __ldg(tk[t] + i));
        return make_float2(0.f, 0.f);
      };
      auto store = [&](int, int j, float2 v) { acc[j] = fmaf(v.x, v.x, fmaf(v.y, v.y, acc[j])); };
      four_step_mask<N>(buf, tw_s, mk_s, lane, load, store);
    }
    // stage |g|^2 of this column in natural order
    if (warp < bw) {
#pragma unroll
      for (int j = 0; j < Q; ++j) accw[lane + 32 * j] = acc[j];
    }
  } else {
    using OS = OutShape<N>;
    float acc[OS::PER_LANE];
#pragma unroll
    for (int t = 0; t < OS::PER_LANE; ++t) acc[t] = 0.f;
    for (int kk = 0; kk < (warp < nw ? kc : 0); ++kk) {
      // the tilt row of this k is shared by the CTA's warps through L1; no barrier
      const float2* Hcol = a.H + ((size_t)a.kmap[k0 + kk] * N + y) * Np;
      const float2* tk = a.tilt + (size_t)(k0 + kk) * Np;
      const int off = a.off;
      auto load = [&](int, int, int x) -> float2 {
        const int i = x - off;
        if ((unsigned)i < (unsigned)Np) return cmul(ld_h<COH>(Hcol + i), __ldg(tk + i));
        return make_float2(0.f, 0.f);
      };
      auto store = [&](int jb, int k, int, float2 v) {
        acc[jb * OS::R0 + k] = fmaf(v.x, v.x, fmaf(v.y, v.y, acc[jb * OS::R0 + k]));
      };
      fft_mask_ifft<N>(buf, tw_s, mk_s, lane, load, store);
      __syncwarp();
    }
    // stage |g|^2 of this column (natural order)
#pragma unroll
    for (int jb = 0; jb < OS::NJ0; ++jb) {
      const int bb = lane + 32 * jb;
      if (warp < bw && (OS::NB0 % 32 == 0 || bb < OS::NB0)) {
#pragma unroll
        for (int k = 0; k < OS::R0; ++k) accw[bb + k * OS::NB0] = acc[jb * OS::R0 + k];
      }
    }
  }
  __syncthreads();
  const int nd = a.nd, b = a.b;
  float* out = a.part + (size_t)gh * nd * nd;
  if (!a.frac) {
    // gb adjacent lanes per detector pixel, each over every gb-th column, then a
    // butterfly sum within the lane group
    int gb = 1;
    while (gb < 8 && gb < bw && nd * gb * 2 <= bw * 32) gb *= 2;  // the CTA's own warps decide
    for (int t0 = 0; t0 < nd * gb; t0 += blockDim.x) {  // the same trip count in every thread
      const int t = t0 + threadIdx.x;
      const int p = t / gb, sub = t - p * gb;
      float sum = 0.f;
      if (p < nd)
        for (int w = sub; w < bw; w += gb) {
          const float* col = reinterpret_cast<const float*>(bufs + w * PITCH) + p * b;
          for (int xx = 0; xx < b; ++xx) sum += col[xx];
        }
      for (int o = 1; o < gb; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (p < nd && sub == 0) out[(size_t)p * nd + q] = sum;
    }
  } else {
    // area weights: fine pixel i shares |[i nd, (i+1) nd) & [p N, (p+1) N)| / nd of
    // itself with detector pixel p (integers, exact in float)
    const float inv = 1.0f / ((float)nd * (float)nd);
    for (int p = threadIdx.x; p < nd; p += blockDim.x) {
      const int x0 = (p * N) / nd, x1 = ((p + 1) * N + nd - 1) / nd;
      float sum = 0.f;
      for (int w = 0; w < nw; ++w) {
        const int yy = y0 + w;
        const int oy = min((yy + 1) * nd, (q + 1) * N) - max(yy * nd, q * N);
        const float* col = reinterpret_cast<const float*>(bufs + w * PITCH);
        float cs = 0.f;
        for (int i = x0; i < x1; ++i) {
          const int ox = min((i + 1) * nd, (p + 1) * N) - max(i * nd, p * N);
          cs = fmaf((float)ox, col[i], cs);
        }
        sum = fmaf((float)oy, cs, sum);
      }
      out[(size_t)p * nd + q] = sum * inv;
    }
  }
  // the last of the G x split CTAs of column q builds that detector column; the CTA
  // that completes the last column computes the slopes
  __shared__ double red[32];
  __shared__ bool flag;
  // written by earlier kernels: fetched now, its latency hidden by the handshake
  const long long fidx = a.fin.frame_ctr ? *a.fin.frame_ctr : 0;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) flag = atomicAdd(a.fin.done_col + q, 1u) == (unsigned)a.fin.G - 1;
  __syncthreads();
  if (!flag) return;
  __threadfence();
  finish_column(a.fin, a.part, q, nd, red, fidx, bw * 32);
}




template <int N>
__global__ void __maxnreg__(cols_max_regs(N))
pyr_cols_kernel(ColArgs a) {
  cols_task<N>(a, blockIdx.x, blockIdx.y, blockDim.x >> 5);
}

// ------------------------------------------------- persistent batched launch
// Both passes of several loops' pyramids (one transform length) in one launch: the
// CTAs draw tickets from one queue, every loop's rows-pass tasks first, then every
// loop's columns-pass tasks (detector column x modulation group x column part). A
// task is exactly one CTA of the loop's own launches (its geometry, its warps, its
// arithmetic), so the frames equal those of the loop measured alone, bit for bit.

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int N>
__global__ void __maxnreg__(cols_max_regs(N))
pyr_batch_kernel(BatchPyrArgs a) {
  __shared__ int s_task, s_loop, s_skip;
  int cur_r = 0, cur_c = 0;  // thread 0's cursors: a CTA's tickets increase
  for (;;) {
    __syncthreads();  // the previous task is done with the shared memory
    if (threadIdx.x == 0) {
      const int t = (int)atomicAdd(a.ticket, 1u) + a.first_ticket;
      int l = -1, skip = 0;
      if (t < a.n_row_tickets) {
        while (a.geo[cur_r].row_base + a.geo[cur_r].n_row <= t) ++cur_r;
        l = cur_r;
      } else if (t < a.n_tickets) {
        while (a.geo[cur_c].col_base + a.geo[cur_c].n_col <= t) ++cur_c;
        l = cur_c;
        // the loop's rows pass must be complete. Its tasks hold lower tickets, each
        // claimed by a running CTA that waits for nothing, so the wait ends; a wait
        // that outlasts the limit flags the launch and the task transforms nothing
        // (its column handshake still runs, the counters stay consistent)
        const unsigned int need = (unsigned int)a.geo[l].n_row;
        const long long limit = *a.wait_limit;
        for (long long polls = 0; ld_acquire_u32(a.rows_done + l) < need; ++polls) {
          if (polls >= limit) {
            atomicOr(a.err, 1u);
            skip = 1;
            break;
          }
          __nanosleep(256);
        }
      }
      s_task = t;
      s_loop = l;
      s_skip = skip;
    }
    __syncthreads();
    const int t = s_task, l = s_loop;
    if (l < 0) return;  // the queue is empty
    const BatchLoopGeo g = a.geo[l];
    if (t < a.n_row_tickets) {
      const int r = t - g.row_base;
      const int by = r / g.nbx;
      rows_task<N>(a.ra[l], r - by * g.nbx, by, g.n_row / g.nbx, g.rows);
      // this task's part of H, written by all threads, published by one release: the
      // barrier orders the writes before thread 0's fence (cumulative) and count
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.rows_done + l, 1u);
      }
    } else {
      // thread 0's acquire load of the count, then the barrier after the claim, order
      // this task's reads of H after the rows tasks' writes
      const int c = t - g.col_base;
      const int gh = c / g.nd;
      cols_task<N, true>(a.ca[l], c - gh * g.nd, gh, g.bw, s_skip != 0);
    }
  }
}

__global__ void ccd_noise_kernel(const float* in, float* out, int n, float scale, float ron,
                                 unsigned long long seed, long long fidx) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
    out[p] = noisy_pixel(in[p], scale, ron, seed, (uint32_t)p, (uint64_t)fidx);
}

// ------------------------------------------------------------------ dispatch

struct PyrKernels {
  void (*rows)(RowArgs);
  void (*cols)(ColArgs);
  int tw_n, buf_n, pitch;
  void (*batch)(BatchPyrArgs);
};

template <int N>
PyrKernels kernels_for() {
  return PyrKernels{pyr_rows_kernel<N>, pyr_cols_kernel<N>, tw_size(N), buf_len(N), buf_len(N) | 1,
                    pyr_batch_kernel<N>};
}

#define PAS_PYR_SIZES(X) X(16) X(24) X(32) X(40) X(48) X(64) X(80) X(96) X(120) X(128) X(160) \
  X(192) X(240) X(256) X(320) X(480) X(512) X(640) X(960)

static bool lookup_kernels(int N, PyrKernels* k) {
  switch (N) {
#define PAS_CASE(n) \
  case n:           \
    *k = kernels_for<n>(); \
    return true;
    PAS_PYR_SIZES(PAS_CASE)
#undef PAS_CASE
    default:
      return false;
  }
}

// Digit-reversed frequency of in-place position p for the radix list of N.
}  // namespace pas

struct pas_pyr_s {
  pas_ctx_t ctx = nullptr;
  pas_pyr_params p{};
  pas::PyrKernels kern{};
  int b = 0, nd = 0, n_s = 0, G = 0, kper = 0, n_valid = 0, n_pupil = 0;
  int H = 1, h_max = 1;  // columns-pass CTAs per detector column and group (divides b)
  int frac = 0;  // non-integer fine pixels per detector pixel
  int rows = 4, s_chunk = 1, n_schunks = 1;
  int s_chunk_max = 1;   // largest rows-pass chunk whose shared memory fits a CTA
  int s_chunk_wide = 0;  // the same for a CTA of ROWS_WIDE rows (0: it does not fit)
  int K_mod = 0, n_src = 1;  // modulation points and source points (p.K = K_mod n_src)
  int64_t T_obs = 0;
  float inv_hi = 0.f, inv_lo = 0.f;
  size_t smem_rows = 0, smem_cols = 0;
  int32_t* d_valid = nullptr;
  float* d_sn = nullptr;
  float2* d_tw = nullptr;
  float2* d_mask = nullptr;
  float2* d_tw4 = nullptr;   // four-step columns pass (N = 480, 960)
  float2* d_mk4 = nullptr;
  float* d_alpha = nullptr;
  float2* d_tilt = nullptr;
  float* d_amp = nullptr;  // [K] column-tilt amplitudes of an extended source
  float* d_beta = nullptr;
  int* d_kmap = nullptr;
  float2* d_H = nullptr;
  float* d_part = nullptr;
  float* d_frame = nullptr;
  long long* d_frame_ctr = nullptr;
  unsigned char* d_vpix = nullptr;
  unsigned int* d_done_col = nullptr;
  double* d_flux_part = nullptr;
  float photon_scale = 0.f, ron = 0.f;
  unsigned long long seed = 0;
  bool has_sn = false;
};

namespace pas {

// The dynamic shared-memory limit is a property of the kernel function, shared by
// every object using it: only ever raise it.
cudaError_t raise_dyn_smem(const void* func, size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// columns pass with `warps` fine columns per CTA
size_t cols_smem(pas_pyr_t y, int warps) {
  if (four_step_ok(y->p.N))
    return sizeof(float2) * ((size_t)four_tw_size(y->p.N) + four_mask_size(y->p.N) + (size_t)warps * four_buf(y->p.N));
  return sizeof(float2) * ((size_t)y->kern.tw_n + y->kern.buf_n + (size_t)warps * y->kern.pitch);
}

// Column splits the columns pass accepts: divisors of b up to 8 (1 alone for
// non-integer binning, whose CTAs cover overlapping column ranges).
static bool split_ok(pas_pyr_t y, int H) { return H == 1 || (!y->frac && H >= 1 && H <= 8 && y->b % H == 0); }

size_t rows_smem(pas_pyr_t y, int rows, int s_chunk) {
  if (four_step_ok(y->p.N))
    return sizeof(float2) * ((size_t)four_tw_size(y->p.N) + four_mask_size(y->p.N) + (size_t)s_chunk * y->p.Np +
                             (size_t)rows * (y->p.Np + four_buf(y->p.N)));
  return sizeof(float2) * ((size_t)y->kern.tw_n + y->kern.buf_n + (size_t)s_chunk * y->p.Np +
                           (size_t)rows * (y->p.Np + y->kern.pitch));
}

static RowArgs make_row_args(pas_pyr_t y, const float* d_opd) {
  const pas_pyr_params& p = y->p;
  RowArgs ra;
  ra.opd = d_opd;
  ra.tw = y->d_tw;
  ra.mask = y->d_mask;
  ra.tw4 = y->d_tw4;
  ra.mk4 = y->d_mk4;
  ra.beta = y->d_beta;
  ra.H = y->d_H;
  ra.Np = p.Np;
  ra.off = (p.N - p.Np) / 2;
  ra.T_obs = (int)y->T_obs;
  ra.inv_hi = y->inv_hi;
  ra.inv_lo = y->inv_lo;
  ra.n_s = y->n_s;
  ra.s_chunk = y->s_chunk;
  return ra;
}

static void launch_rows(pas_pyr_t y, const float* d_opd, cudaStream_t st, bool pdl = false) {
  const RowArgs ra = make_row_args(y, d_opd);
  dim3 gr((y->p.Np + y->rows - 1) / y->rows, y->n_schunks);
  launch_k(y->kern.rows, gr, dim3(y->rows * 32), rows_smem(y, y->rows, y->s_chunk), st, pdl, ra);
}

static ColArgs make_col_args(pas_pyr_t y, float* d_frame, float* d_slopes, const LoopExtra* fa_extra,
                             bool increment_ctr) {
  const pas_pyr_params& p = y->p;
  ColArgs ca;
  ca.H = y->d_H;
  ca.tw = y->d_tw;
  ca.mask = y->d_mask;
  ca.tw4 = y->d_tw4;
  ca.mk4 = y->d_mk4;
  ca.tilt = y->d_tilt;
  ca.kmap = y->d_kmap;
  ca.part = y->d_part;
  ca.Np = p.Np;
  ca.off = (p.N - p.Np) / 2;
  ca.K = p.K;
  ca.kper = y->kper;
  ca.nd = y->nd;
  ca.b = y->b;
  ca.split = y->H;
  ca.frac = y->frac;
  long long* ctr = fa_extra ? fa_extra->frame_ctr : y->d_frame_ctr;
  FrameArgs& fa = ca.fin;
  fa.frame = d_frame ? d_frame : y->d_frame;
  fa.vpix = y->d_vpix;
  fa.flux_part = y->d_flux_part;
  fa.done_col = y->d_done_col;
  fa.frame_ctr = ctr;
  fa.ctr_increment = increment_ctr ? 1 : 0;
  fa.G = y->G * y->H;
  fa.np = y->nd * y->nd;
  fa.invK = 1.0f / (float)p.K;
  fa.scale = y->photon_scale;
  fa.ron = y->ron;
  fa.seed = y->seed;
  fa.valid = y->d_valid;
  fa.sn = y->has_sn ? y->d_sn : nullptr;
  fa.slopes = d_slopes;
  fa.nv = y->n_valid;
  fa.n_sub = p.n_sub;
  fa.local_norm = p.local_norm;
  fa.wfe = fa_extra ? *fa_extra : LoopExtra();
  return ca;
}

static void launch_cols(pas_pyr_t y, float* d_frame, float* d_slopes, cudaStream_t st,
                        const LoopExtra* fa_extra, bool increment_ctr) {
  const ColArgs ca = make_col_args(y, d_frame, d_slopes, fa_extra, increment_ctr);
  dim3 gc(y->nd, y->G * y->H);
  const int warps = y->b / y->H;
  // the columns pass starts after the rows pass has finished: launched early, its
  // CTAs (up to 3 per SM) wait on the SMs while the rows pass runs and slow it
  // (measured on the 480 grid: 84 us per loop step this way, 89-99 us with the
  // early launch)
  launch_k(y->kern.cols, gc, dim3(warps * 32), cols_smem(y, warps), st, false, ca);
}

static void launch_slopes(pas_pyr_t y, float* d_frame, float* d_slopes, cudaStream_t st,
                          const LoopExtra* fa_extra, bool increment_ctr, bool pdl = false) {
  FrameArgs f{};
  f.frame = d_frame ? d_frame : y->d_frame;
  f.flux_part = y->d_flux_part;
  f.frame_ctr = fa_extra ? fa_extra->frame_ctr : y->d_frame_ctr;
  f.ctr_increment = increment_ctr ? 1 : 0;
  f.valid = y->d_valid;
  f.sn = y->has_sn ? y->d_sn : nullptr;
  f.slopes = d_slopes;
  f.nv = y->n_valid;
  f.n_sub = y->p.n_sub;
  f.local_norm = y->p.local_norm;
  f.wfe = fa_extra ? *fa_extra : LoopExtra();
  launch_k(slopes_kernel, dim3((y->n_valid + 255) / 256), dim3(256), 0, st, pdl, f, y->nd);
}

// Launch the pyramid kernels (rows pass, columns pass with the detector frame,
// noise and slopes). `fa_extra`: the loop's frame counter and WFE fields.
pas_status pyr_launch(pas_pyr_t y, const float* d_opd, float* d_frame, float* d_slopes,
                      cudaStream_t st, const LoopExtra* fa_extra, bool increment_ctr, cudaEvent_t* ev,
                      bool pdl_first) {
  // the slopes kernel follows the columns pass programmatically (and the rows pass
  // its predecessor when pdl_first) unless events are recorded between the kernels
  const bool pdl = ev == nullptr;
  if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
  launch_rows(y, d_opd, st, pdl && pdl_first);
  if (ev) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
  launch_cols(y, d_frame, d_slopes, st, fa_extra, increment_ctr);
  if (ev) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
  launch_slopes(y, d_frame, d_slopes, st, fa_extra, increment_ctr, pdl);
  return check_launch(y->ctx, "pas_pyr_measure launch");
}

// ------------------------------------------------- persistent batched launch (host)

struct PyrBatchGroup {
  int N = 0;
  void (*kern)(BatchPyrArgs) = nullptr;
  BatchPyrArgs args{};
  int grid = 0, threads = 0;
  size_t smem = 0;
  int rows = 1, row_chunk = 1;  // rows-task geometry chosen for the shared CTA
  size_t counter_off = 0;       // its counters: ticket, rows_done[L]
};

struct PyrBatch {
  pas_ctx_t ctx = nullptr;
  std::vector<pas_pyr_t> pyr;
  std::vector<float*> frame, slopes;
  std::vector<LoopExtra> extra;
  std::vector<PyrBatchGroup> groups;
  std::vector<int> group_of;        // member -> group
  void* d_mem = nullptr;            // argument arrays of every group
  unsigned int* d_counters = nullptr;  // per group: ticket, rows_done[L]; zeroed per launch
  size_t counter_bytes = 0;
  unsigned int* d_err = nullptr;
  long long* d_wait_limit = nullptr;
};

void pyr_batch_destroy(PyrBatch* b) {
  if (!b) return;
  dev_free(b->d_mem);
  dev_free(b->d_counters);
  dev_free(b->d_err);
  dev_free(b->d_wait_limit);
  delete b;
}

pas_status pyr_batch_create(pas_ctx_t ctx, int n, const pas_pyr_t* y, const float* const* opd, float* const* frame,
                            float* const* slopes, const LoopExtra* extra, PyrBatch** out) {
  *out = nullptr;
  PAS_CHECK_ARG(ctx, n >= 1, "persistent pyramid batch: at least one pyramid");
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      PAS_CHECK_ARG(ctx, y[i] != y[j], "persistent pyramid batch: a pyramid object appears twice");
  PyrBatch* b = new PyrBatch();
  b->ctx = ctx;
  b->pyr.assign(y, y + n);
  b->frame.assign(frame, frame + n);
  b->slopes.assign(slopes, slopes + n);
  b->extra.assign(extra, extra + n);
  b->group_of.assign(n, -1);
  // one group per transform length, members in batch order
  std::vector<std::vector<int>> members;
  for (int i = 0; i < n; ++i) {
    int g = -1;
    for (size_t k = 0; k < b->groups.size(); ++k)
      if (b->groups[k].N == y[i]->p.N) g = (int)k;
    if (g < 0) {
      g = (int)b->groups.size();
      b->groups.emplace_back();
      b->groups.back().N = y[i]->p.N;
      b->groups.back().kern = y[i]->kern.batch;
      members.emplace_back();
    }
    members[g].push_back(i);
    b->group_of[i] = g;
  }
  const size_t G = b->groups.size();
  size_t arg_bytes = 0, n_counters = 0;
  for (size_t g = 0; g < G; ++g) {
    const size_t L = members[g].size();
    arg_bytes += L * (sizeof(RowArgs) + sizeof(ColArgs) + sizeof(BatchLoopGeo)) + 3 * 256;
    n_counters += 1 + L;
  }
  b->counter_bytes = sizeof(unsigned int) * n_counters;
  pas_status st = dev_alloc(ctx, &b->d_mem, arg_bytes);
  if (st == PAS_OK) st = dev_alloc(ctx, (void**)&b->d_counters, b->counter_bytes);
  if (st == PAS_OK) st = dev_alloc(ctx, (void**)&b->d_err, sizeof(unsigned int));
  if (st == PAS_OK) st = dev_alloc(ctx, (void**)&b->d_wait_limit, sizeof(long long));
  if (st != PAS_OK) {
    pyr_batch_destroy(b);
    return st;
  }
  std::vector<unsigned char> host(arg_bytes, 0);
  size_t off = 0, ctr = 0;
  auto carve = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) & ~size_t(255);
    return at;
  };
  cudaError_t e = cudaSuccess;
  for (size_t g = 0; g < G && e == cudaSuccess; ++g) {
    PyrBatchGroup& grp = b->groups[g];
    const size_t L = members[g].size();
    const size_t o_ra = carve(L * sizeof(RowArgs)), o_ca = carve(L * sizeof(ColArgs)),
                 o_geo = carve(L * sizeof(BatchLoopGeo));
    RowArgs* ra = reinterpret_cast<RowArgs*>(host.data() + o_ra);
    ColArgs* ca = reinterpret_cast<ColArgs*>(host.data() + o_ca);
    BatchLoopGeo* geo = reinterpret_cast<BatchLoopGeo*>(host.data() + o_geo);
    // The columns tasks keep each loop's own geometry (it fixes the order of the
    // modulation-group sums); the CTA has the widest columns task's warps. The rows
    // tasks' geometry does not change H (each transform is one warp's, whatever the
    // CTA), so it is chosen for the shared CTA: the (rows, sin-chunk) pair with the
    // least modelled time, each phase's work over its working warps per SM (at most
    // 16 of them keep the issue slots busy).
    int warps = 1;
    size_t smem_c = 0;
    double w_rows = 0.0, w_cols = 0.0, bw_sum = 0.0;
    int n_s_max = 1;
    double n_col_tasks = 0.0;
    for (size_t k = 0; k < L; ++k) {
      pas_pyr_t p = y[members[g][k]];
      const int bw = p->b / p->H;
      warps = std::max(warps, bw);
      smem_c = std::max(smem_c, cols_smem(p, bw));
      w_rows += (double)p->n_s * p->p.Np;
      w_cols += (double)p->p.K * p->nd * p->b;
      bw_sum += bw;
      n_s_max = std::max(n_s_max, p->n_s);
      n_col_tasks += (double)p->nd * p->G * p->H;
    }
    int best_rows = 1, best_chunk = 1;
    size_t best_smem = 0;
    double best_t = -1.0;
    // the opt-in shared memory of a CTA less the kernel's static shared memory
    size_t smem_lim = 0;
    {
      cudaFuncAttributes fa;
      int optin = 0;
      e = cudaFuncGetAttributes(&fa, (const void*)grp.kern);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
      if (e == cudaSuccess) smem_lim = std::min(SMEM_MAX, (size_t)optin - fa.sharedSizeBytes);
      if (e == cudaSuccess) e = raise_dyn_smem((const void*)grp.kern, smem_lim);
    }
    for (int rows = 1; rows <= std::min(warps, MAX_ROWS_PER_CTA) && e == cudaSuccess; rows *= 2) {
      for (int c = 1; c <= n_s_max && e == cudaSuccess; ++c) {
        size_t sm = smem_c;
        for (size_t k = 0; k < L; ++k) {
          pas_pyr_t p = y[members[g][k]];
          const int nby = (p->n_s + c - 1) / c;
          sm = std::max(sm, rows_smem(p, rows, (p->n_s + nby - 1) / nby));
        }
        if (sm > smem_lim) continue;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, grp.kern, 32 * warps, sm);
        if (e != cudaSuccess || occ < 1) continue;
        // the OPD phasor is formed once per chunk: n_s / c of them per row; a phase
        // keeps at most as many CTAs busy per SM as it has tasks per SM
        const double rows_work = w_rows * (1.0 + 0.25 / c);
        double n_row_tasks = 0.0;
        for (size_t k = 0; k < L; ++k) {
          pas_pyr_t p = y[members[g][k]];
          n_row_tasks += (double)((p->p.Np + rows - 1) / rows) * ((p->n_s + c - 1) / c);
        }
        const double sms = std::max(1, ctx->sm_count);
        const double ctas_r = std::min((double)occ, n_row_tasks / sms);
        const double ctas_c = std::min((double)occ, n_col_tasks / sms);
        const double t = rows_work / std::min(16.0, ctas_r * rows) +
                         w_cols / std::min(16.0, ctas_c * bw_sum / (double)L);
        if (best_t < 0.0 || t < best_t) {
          best_t = t;
          best_rows = rows;
          best_chunk = c;
          best_smem = sm;
        }
      }
    }
    if (e == cudaSuccess && best_t < 0.0) {
      pyr_batch_destroy(b);
      return set_error(ctx, PAS_EINVAL, "persistent pyramid batch: no CTA shape fits an SM");
    }
    int tickets = 0;
    const size_t smem = best_smem;
    for (size_t k = 0; k < L && e == cudaSuccess; ++k) {
      const int i = members[g][k];
      pas_pyr_t p = y[i];
      ra[k] = make_row_args(p, opd[i]);
      ca[k] = make_col_args(p, frame[i], slopes[i], &extra[i], false);
      const int nby = (p->n_s + best_chunk - 1) / best_chunk;
      ra[k].s_chunk = (p->n_s + nby - 1) / nby;
      BatchLoopGeo& q = geo[k];
      q.rows = best_rows;
      q.nbx = (p->p.Np + best_rows - 1) / best_rows;
      q.row_base = tickets;
      q.n_row = q.nbx * nby;
      tickets += q.n_row;
      q.nd = p->nd;
      q.bw = p->b / p->H;
      q.n_col = p->nd * p->G * p->H;
    }
    const int n_row_tickets = tickets;
    for (size_t k = 0; k < L; ++k) {
      geo[k].col_base = tickets;
      tickets += geo[k].n_col;
    }
    BatchPyrArgs& a = grp.args;
    unsigned char* dm = static_cast<unsigned char*>(b->d_mem);
    a.ra = reinterpret_cast<const RowArgs*>(dm + o_ra);
    a.ca = reinterpret_cast<const ColArgs*>(dm + o_ca);
    a.geo = reinterpret_cast<const BatchLoopGeo*>(dm + o_geo);
    a.ticket = b->d_counters + ctr;
    a.rows_done = b->d_counters + ctr + 1;
    grp.counter_off = ctr;
    ctr += 1 + L;
    a.err = b->d_err;
    a.wait_limit = b->d_wait_limit;
    a.n_loops = (int)L;
    a.n_row_tickets = n_row_tickets;
    a.n_tickets = tickets;
    a.first_ticket = 0;
    grp.threads = 32 * warps;
    grp.smem = smem;
    grp.rows = best_rows;
    grp.row_chunk = best_chunk;
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, grp.kern, grp.threads, smem);
    if (e == cudaSuccess && occ < 1) {
      pyr_batch_destroy(b);
      return set_error(ctx, PAS_EINVAL, "persistent pyramid batch: a CTA of %d threads does not fit an SM",
                       grp.threads);
    }
    grp.grid = std::max(1, std::min(tickets, occ * std::max(1, ctx->sm_count)));
  }
  const long long limit = PAS_BATCH_WAIT_DEFAULT;
  if (e == cudaSuccess) e = cudaMemcpy(b->d_mem, host.data(), arg_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_wait_limit, &limit, sizeof(limit), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, b->counter_bytes);
  if (e != cudaSuccess) {
    pyr_batch_destroy(b);
    return set_error(ctx, PAS_ECUDA, "persistent pyramid batch: %s", cudaGetErrorString(e));
  }
  *out = b;
  return PAS_OK;
}

// Both passes of every member on `st`: the counters are zeroed, then one persistent
// launch per transform length (in group order). columns_only: the queue starts at
// the columns-pass tickets, the rows pass is withheld (a diagnostic of the waits).
pas_status pyr_batch_launch_group(PyrBatch* b, int g, cudaStream_t st, bool columns_only) {
  const PyrBatchGroup& grp = b->groups[g];
  BatchPyrArgs a = grp.args;
  if (columns_only) a.first_ticket = a.n_row_tickets;
  cudaError_t e = cudaMemsetAsync(b->d_counters + grp.counter_off, 0, sizeof(unsigned int) * (1 + a.n_loops), st);
  if (e == cudaSuccess) e = launch_k(grp.kern, dim3(grp.grid), dim3(grp.threads), grp.smem, st, false, a);
  if (e != cudaSuccess) return set_error(b->ctx, PAS_ECUDA, "persistent pyramid batch launch: %s", cudaGetErrorString(e));
  return PAS_OK;
}

pas_status pyr_batch_launch(PyrBatch* b, cudaStream_t st, bool columns_only) {
  for (size_t g = 0; g < b->groups.size(); ++g) {
    const pas_status s = pyr_batch_launch_group(b, (int)g, st, columns_only);
    if (s != PAS_OK) return s;
  }
  return PAS_OK;
}

int pyr_batch_group_of(const PyrBatch* b, int i) { return b->group_of[i]; }

void pyr_batch_geometry(const PyrBatch* b, int g, int* h) {
  const PyrBatchGroup& grp = b->groups[g];
  h[0] = grp.N;
  h[1] = grp.grid;
  h[2] = grp.threads;
  h[3] = (int)grp.smem;
  h[4] = grp.rows;
  h[5] = grp.row_chunk;
  h[6] = grp.args.n_row_tickets;
  h[7] = grp.args.n_tickets - grp.args.n_row_tickets;
}

// Member i's slopes kernel on `st` (after pyr_batch_launch); pdl: it follows a
// kernel of `st` programmatically.
pas_status pyr_batch_slopes(PyrBatch* b, int i, cudaStream_t st, bool pdl) {
  launch_slopes(b->pyr[i], b->frame[i], b->slopes[i], st, &b->extra[i], false, pdl);
  return check_launch(b->ctx, "persistent pyramid batch: slopes launch");
}

int pyr_batch_n_groups(const PyrBatch* b) { return (int)b->groups.size(); }
unsigned int* pyr_batch_err(PyrBatch* b) { return b->d_err; }
long long* pyr_batch_wait_limit(PyrBatch* b) { return b->d_wait_limit; }

int pyr_n_pupil(pas_pyr_t y) { return y->n_pupil; }
int pyr_n_valid(pas_pyr_t y) { return y->n_valid; }

pas_status pyr_measure_noiseless(pas_pyr_t y, const float* d_opd, float* d_frame, float* d_slopes, cudaStream_t st) {
  // launch arguments are taken by value, so the object's noise setting is restored
  // as soon as the kernels are enqueued
  const float scale = y->photon_scale;
  y->photon_scale = 0.f;
  const pas_status s = pyr_launch(y, d_opd, d_frame, d_slopes, st, nullptr, false);
  y->photon_scale = scale;
  return s;
}
int pyr_nd(pas_pyr_t y) { return y->nd; }
int pyr_np(pas_pyr_t y) { return y->p.Np; }

}  // namespace pas

extern "C" {

int pas_pyr_supported(int N) {
  pas::PyrKernels k;
  return pas::lookup_kernels(N, &k) ? 1 : 0;
}

void pas_pyr_destroy(pas_pyr_t y) {
  if (!y) return;
  pas::dev_free(y->d_valid);
  pas::dev_free(y->d_sn);
  pas::dev_free(y->d_tw);
  pas::dev_free(y->d_mask);
  pas::dev_free(y->d_alpha);
  pas::dev_free(y->d_tilt);
  pas::dev_free(y->d_amp);
  pas::dev_free(y->d_beta);
  pas::dev_free(y->d_kmap);
  pas::dev_free(y->d_tw4);
  pas::dev_free(y->d_mk4);
  pas::dev_free(y->d_H);
  pas::dev_free(y->d_part);
  pas::dev_free(y->d_frame);
  pas::dev_free(y->d_frame_ctr);
  pas::dev_free(y->d_vpix);
  pas::dev_free(y->d_done_col);
  pas::dev_free(y->d_flux_part);
  delete y;
}

// Source: n_src = 0 for a point source, else n_src points at (ex, ey) lambda/D with
// weights w (null: equal).
static pas_status pyr_create(pas_ctx_t ctx, const pas_pyr_params* pp, const int32_t* h_valid, int32_t n_valid,
                             const double* ex, const double* ey, const double* w, int n_src, pas_pyr_t* out) {
  if (!ctx || !pp || !out) return pas::set_global_error(PAS_EINVAL, "pas_pyr_create: NULL argument");
  *out = nullptr;
  pas_pyr_params p = *pp;
  PAS_CHECK_ARG(ctx, p.Np > 0 && p.N == 2 * p.Np, "pas_pyr_create: N must equal 2*Np");
  PAS_CHECK_ARG(ctx, p.n_sub > 0 && 2 * p.n_sub <= p.N, "pas_pyr_create: need 1 <= n_sub <= Np");
  PAS_CHECK_ARG(ctx, p.K >= 1 && p.K * std::max(n_src, 1) <= 4096, "pas_pyr_create: K (x source points) out of range");
  const int P = std::max(n_src, 1);
  std::vector<double> src_w(P, 1.0 / P);
  if (n_src > 0) {
    PAS_CHECK_ARG(ctx, ex && ey, "pas_pyr_create_extended: NULL offsets");
    double tot = 0.0;
    for (int q = 0; q < P; ++q) {
      PAS_CHECK_ARG(ctx, std::isfinite(ex[q]) && std::isfinite(ey[q]), "pas_pyr_create_extended: offsets not finite");
      if (w) PAS_CHECK_ARG(ctx, std::isfinite(w[q]) && w[q] >= 0.0, "pas_pyr_create_extended: weights >= 0");
      tot += w ? w[q] : 1.0;
    }
    PAS_CHECK_ARG(ctx, tot > 0.0, "pas_pyr_create_extended: weights sum to zero");
    for (int q = 0; q < P; ++q) src_w[q] = (w ? w[q] : 1.0) / tot;
  }
  PAS_CHECK_ARG(ctx, p.wavelength_nm > 0 && p.mod_radius >= 0 && p.obs >= 0 && p.obs < 1,
                "pas_pyr_create: bad wavelength, modulation radius or obstruction");
  pas::PyrKernels kern;
  if (!pas::lookup_kernels(p.N, &kern))
    return pas::set_error(ctx, PAS_EINVAL, "pas_pyr_create: FFT size N=%d not supported", p.N);
  // warps per columns CTA: b fine columns per detector column, or for a non-integer
  // N / (2 n_sub) the most fine columns any detector column overlaps
  const int nd_ = 2 * p.n_sub, frac = p.N % nd_ != 0;
  int b = p.N / nd_;
  if (frac)
    for (int q = 0; q < nd_; ++q) b = std::max(b, ((q + 1) * p.N + nd_ - 1) / nd_ - (q * p.N) / nd_);
  PAS_CHECK_ARG(ctx, b <= 16, "pas_pyr_create: more than 16 fine pixels per detector pixel");

  pas_pyr_t y = new pas_pyr_s();
  y->ctx = ctx;
  y->p = p;
  y->kern = kern;
  y->b = b;
  y->frac = frac;
  y->nd = 2 * p.n_sub;
  y->T_obs = pas::obstruction_threshold(p.Np, p.obs);
  {
    int32_t n = 0;
    pas_pupil_mask(p.Np, p.obs, nullptr, &n);
    y->n_pupil = n;
  }
  // valid sub-apertures
  std::vector<int32_t> valid;
  if (h_valid) {
    if (n_valid <= 0) {
      delete y;
      return pas::set_error(ctx, PAS_EINVAL, "pas_pyr_create: n_valid must be > 0");
    }
    valid.assign(h_valid, h_valid + n_valid);
    for (int j = 0; j < n_valid; ++j)
      if (valid[j] < 0 || valid[j] >= p.n_sub * p.n_sub || (j > 0 && valid[j] <= valid[j - 1])) {
        delete y;
        return pas::set_error(ctx, PAS_EINVAL, "pas_pyr_create: valid indices must be ascending in [0, n_sub^2)");
      }
  } else {
    int32_t nv = 0;
    pas_valid_subaps(p.Np, p.obs, p.n_sub, nullptr, 0, &nv);
    valid.resize(nv);
    pas_valid_subaps(p.Np, p.obs, p.n_sub, valid.data(), nv, &nv);
  }
  y->n_valid = (int)valid.size();

  // tilt points: modulation point k of source point q at
  // (R cos theta_k + ex_q, R sin theta_k + ey_q), index t = q K + k. One rows pass per
  // distinct (sin theta, ey): theta and pi - theta share one, and so do source points
  // of equal ey. An extended source's weights become column-tilt amplitudes
  // sqrt(w_q P): the frame is (1/(K P)) sum_t |E_t|^2 = sum_q w_q (1/K) sum_k |E_qk|^2.
  const int Km = p.K, Kt = Km * P;
  y->K_mod = Km;
  y->n_src = P;
  std::vector<int> kmap(Kt), key_rep(Kt), key_ey(Kt);
  std::vector<float> alpha(Kt), beta(Kt), amp(Kt);
  y->n_s = pas::pyr_tilt_tables(p.Np, p.N, Km, p.mod_radius, P, n_src > 0 ? ex : nullptr, n_src > 0 ? ey : nullptr,
                                src_w.data(), kmap.data(), alpha.data(), amp.data(), beta.data(), key_rep.data(),
                                key_ey.data());
  // from here on p.K counts all tilt points
  p.K = Kt;
  y->p.K = Kt;
  // per-pass twiddle tables ([k-1][n1] = w_L^{n1 k}) and the digit-reversed
  // pyramid mask (delta = N/4: phase (pi/2)|u~|, divided by N) in padded layout
  std::vector<float2> tw = pas::fft_twiddles(p.N), mk(kern.buf_n);
  pas::pyr_mask_table(p.N, kern.buf_n, mk.data());
  double inv = 1.0 / p.wavelength_nm;
  y->inv_hi = (float)inv;
  y->inv_lo = (float)(inv - (double)y->inv_hi);

  // rows pass default: 4 rows per CTA, chunks of about 4 distinct sin values
  // (pas_pyr_autotune measures the alternatives)
  y->rows = 4;
  y->n_schunks = (y->n_s + 3) / 4;
  y->s_chunk = (y->n_s + y->n_schunks - 1) / y->n_schunks;
  y->s_chunk_max = y->n_s;
  while (y->s_chunk_max > 1 && pas::rows_smem(y, pas::MAX_ROWS_PER_CTA, y->s_chunk_max) > pas::SMEM_MAX)
    --y->s_chunk_max;
  y->smem_rows = pas::rows_smem(y, pas::MAX_ROWS_PER_CTA, y->s_chunk_max);  // largest candidate
  y->s_chunk_wide = std::min(y->n_s, y->s_chunk_max);
  while (y->s_chunk_wide > 0 && pas::rows_smem(y, pas::ROWS_WIDE, y->s_chunk_wide) > pas::SMEM_MAX) --y->s_chunk_wide;
  if (y->s_chunk_wide > 0)
    y->smem_rows = std::max(y->smem_rows, pas::rows_smem(y, pas::ROWS_WIDE, y->s_chunk_wide));
  y->smem_cols = pas::cols_smem(y, b);  // largest: one CTA per detector column and group
  for (int H = 2; H <= 8; ++H)
    if (pas::split_ok(y, H)) y->h_max = H;

  pas_status st = PAS_OK;
  auto A = [&](void** ptr, size_t bytes) {
    if (st == PAS_OK) st = pas::dev_alloc(ctx, ptr, bytes);
  };
  A((void**)&y->d_valid, sizeof(int32_t) * y->n_valid);
  A((void**)&y->d_sn, sizeof(float) * 2 * y->n_valid);
  A((void**)&y->d_tw, sizeof(float2) * kern.tw_n);
  A((void**)&y->d_mask, sizeof(float2) * kern.buf_n);
  if (pas::four_step_ok(p.N)) {
    A((void**)&y->d_tw4, sizeof(float2) * pas::four_tw_size(p.N));
    A((void**)&y->d_mk4, sizeof(float2) * pas::four_mask_size(p.N));
  }
  A((void**)&y->d_alpha, sizeof(float) * p.K);
  A((void**)&y->d_tilt, sizeof(float2) * (size_t)p.K * p.Np);
  if (n_src > 0) A((void**)&y->d_amp, sizeof(float) * p.K);
  A((void**)&y->d_beta, sizeof(float) * y->n_s);
  A((void**)&y->d_kmap, sizeof(int) * p.K);
  A((void**)&y->d_H, sizeof(float2) * (size_t)y->n_s * p.N * p.Np);
  A((void**)&y->d_part, sizeof(float) * (size_t)p.K * y->h_max * y->nd * y->nd);  // G <= K groups x split
  A((void**)&y->d_frame, sizeof(float) * y->nd * y->nd);
  A((void**)&y->d_frame_ctr, sizeof(long long));
  A((void**)&y->d_vpix, (size_t)y->nd * y->nd);
  A((void**)&y->d_flux_part, sizeof(double) * y->nd);
  A((void**)&y->d_done_col, sizeof(unsigned int) * y->nd);
  if (st != PAS_OK) {
    pas_pyr_destroy(y);
    return st;
  }
  cudaError_t e = cudaSuccess;
  auto C = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  C(y->d_valid, valid.data(), sizeof(int32_t) * y->n_valid);
  C(y->d_tw, tw.data(), sizeof(float2) * kern.tw_n);
  C(y->d_mask, mk.data(), sizeof(float2) * kern.buf_n);
  if (pas::four_step_ok(p.N)) {
    std::vector<float2> tw4(pas::four_tw_size(p.N)), mk4(pas::four_mask_size(p.N));
    pas::four_step_tables(p.N, tw4.data(), mk4.data());
    C(y->d_tw4, tw4.data(), sizeof(float2) * tw4.size());
    C(y->d_mk4, mk4.data(), sizeof(float2) * mk4.size());
  }
  C(y->d_alpha, alpha.data(), sizeof(float) * p.K);
  if (y->d_amp) C(y->d_amp, amp.data(), sizeof(float) * p.K);
  if (e == cudaSuccess) {
    pas::tilt_table_kernel<<<p.K, 256>>>(y->d_alpha, y->d_amp, p.K, p.Np, y->d_tilt);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  C(y->d_beta, beta.data(), sizeof(float) * y->n_s);
  C(y->d_kmap, kmap.data(), sizeof(int) * p.K);
  {
    std::vector<unsigned char> vpix((size_t)y->nd * y->nd);
    pas::quadrant_valid_map(p.n_sub, valid.data(), y->n_valid, vpix.data());
    C(y->d_vpix, vpix.data(), vpix.size());
  }
  if (e == cudaSuccess) e = cudaMemset(y->d_sn, 0, sizeof(float) * 2 * y->n_valid);
  if (e == cudaSuccess) e = cudaMemset(y->d_frame_ctr, 0, sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(y->d_done_col, 0, sizeof(unsigned int) * y->nd);
  if (e == cudaSuccess) e = pas::raise_dyn_smem((const void*)kern.rows, y->smem_rows);
  if (e == cudaSuccess) e = pas::raise_dyn_smem((const void*)kern.cols, y->smem_cols);
  // modulation grouping: the columns pass runs nd x G CTAs of b warps, each warp
  // doing kper = ceil(K / G) transforms; pick G minimising waves x kper
  int occ = 1;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern.cols, b * 32, y->smem_cols);
  if (e == cudaSuccess)
    pas::pick_modulation_groups(p.K, y->nd, std::max(1, occ) * std::max(1, ctx->sm_count), &y->kper, &y->G,
                                pas::four_step_ok(p.N) ? pas::four_tpw(p.N) : 1);
  if (e != cudaSuccess) {
    pas_pyr_destroy(y);
    return pas::set_error(ctx, PAS_ECUDA, "pas_pyr_create: %s", cudaGetErrorString(e));
  }
  *out = y;
  return PAS_OK;
}

pas_status pas_pyr_create(pas_ctx_t ctx, const pas_pyr_params* pp, const int32_t* h_valid, int32_t n_valid,
                          pas_pyr_t* out) {
  return pyr_create(ctx, pp, h_valid, n_valid, nullptr, nullptr, nullptr, 0, out);
}

pas_status pas_pyr_create_extended(pas_ctx_t ctx, const pas_pyr_params* pp, const int32_t* h_valid,
                                   int32_t n_valid, const double* h_ex, const double* h_ey, const double* h_w,
                                   int32_t n_points, pas_pyr_t* out) {
  if (!ctx || !out) return pas::set_global_error(PAS_EINVAL, "pas_pyr_create_extended: NULL argument");
  *out = nullptr;
  PAS_CHECK_ARG(ctx, n_points >= 1, "pas_pyr_create_extended: n_points >= 1");
  return pyr_create(ctx, pp, h_valid, n_valid, h_ex, h_ey, h_w, n_points, out);
}

int32_t pas_pyr_n_valid(pas_pyr_t y) { return y ? y->n_valid : -1; }

pas_status pas_pyr_get_valid(pas_pyr_t y, int32_t* h_valid, int32_t cap) {
  if (!y || !h_valid) return pas::set_global_error(PAS_EINVAL, "pas_pyr_get_valid: NULL argument");
  PAS_CHECK_ARG(y->ctx, cap >= y->n_valid, "pas_pyr_get_valid: cap too small");
  PAS_CUDA_TRY(y->ctx, cudaMemcpy(h_valid, y->d_valid, sizeof(int32_t) * y->n_valid, cudaMemcpyDeviceToHost));
  return PAS_OK;
}

pas_status pas_pyr_set_reference(pas_pyr_t y, const float* d_sn) {
  if (!y) return pas::set_global_error(PAS_EINVAL, "pas_pyr_set_reference: NULL pyramid");
  if (!d_sn) {
    y->has_sn = false;
    return PAS_OK;
  }
  PAS_CUDA_TRY(y->ctx, cudaMemcpyAsync(y->d_sn, d_sn, sizeof(float) * 2 * y->n_valid,
                                       cudaMemcpyDeviceToDevice, y->ctx->stream));
  y->has_sn = true;
  return PAS_OK;
}

pas_status pas_pyr_set_noise(pas_pyr_t y, double photons, double ron, uint64_t seed, int64_t frame_index) {
  if (!y) return pas::set_global_error(PAS_EINVAL, "pas_pyr_set_noise: NULL pyramid");
  PAS_CHECK_ARG(y->ctx, ron >= 0.0 && frame_index >= 0, "pas_pyr_set_noise: bad read noise or frame index");
  y->photon_scale = photons > 0.0 ? (float)(photons / (double)y->n_pupil) : 0.f;
  y->ron = (float)ron;
  y->seed = seed;
  long long f = frame_index;
  PAS_CUDA_TRY(y->ctx, cudaMemcpyAsync(y->d_frame_ctr, &f, sizeof(f), cudaMemcpyHostToDevice, y->ctx->stream));
  PAS_CUDA_TRY(y->ctx, cudaStreamSynchronize(y->ctx->stream));
  return PAS_OK;
}

pas_status pas_pyr_measure(pas_pyr_t y, const float* d_opd, float* d_frame, float* d_slopes) {
  if (!y || !d_opd) return pas::set_global_error(PAS_EINVAL, "pas_pyr_measure: NULL argument");
  return pas::pyr_launch(y, d_opd, d_frame, d_slopes, y->ctx->stream, nullptr, true);
}

pas_status pas_pyr_get_tuning(pas_pyr_t y, pas_pyr_tuning* out) {
  if (!y || !out) return pas::set_global_error(PAS_EINVAL, "pas_pyr_get_tuning: NULL argument");
  out->rows_per_cta = y->rows;
  out->row_chunks = y->n_schunks;
  out->col_groups = y->G;
  out->col_split = y->H;
  return PAS_OK;
}

pas_status pas_pyr_set_tuning(pas_pyr_t y, const pas_pyr_tuning* t) {
  if (!y || !t) return pas::set_global_error(PAS_EINVAL, "pas_pyr_set_tuning: NULL argument");
  const int r = t->rows_per_cta;
  const int chunk = t->row_chunks >= 1 ? (y->n_s + t->row_chunks - 1) / t->row_chunks : 0;
  const bool rows_ok = r == 1 || r == 2 || r == 4 || r == 8 || (r == pas::ROWS_WIDE && chunk <= y->s_chunk_wide);
  PAS_CHECK_ARG(y->ctx, rows_ok && t->row_chunks >= 1 &&
                t->row_chunks <= y->n_s && chunk <= y->s_chunk_max &&
                t->col_groups >= 1 && t->col_groups <= y->p.K && pas::split_ok(y, t->col_split),
                "pas_pyr_set_tuning: rows_per_cta in {1,2,4,8} (16 where its chunk's shared memory fits), 1 <= "
                "row_chunks <= distinct sin values (chunks within shared memory), 1 <= col_groups <= K, col_split "
                "1 or a divisor <= 8 of the fine pixels per detector pixel");
  y->rows = r;
  y->s_chunk = (y->n_s + t->row_chunks - 1) / t->row_chunks;
  y->n_schunks = (y->n_s + y->s_chunk - 1) / y->s_chunk;
  y->kper = (y->p.K + t->col_groups - 1) / t->col_groups;
  y->G = (y->p.K + y->kper - 1) / y->kper;
  y->H = t->col_split;
  return PAS_OK;
}

pas_status pas_pyr_autotune(pas_pyr_t y, const float* d_opd, int32_t iters, pas_pyr_tuning* out) {
  if (!y || !d_opd) return pas::set_global_error(PAS_EINVAL, "pas_pyr_autotune: NULL argument");
  PAS_CHECK_ARG(y->ctx, iters >= 1, "pas_pyr_autotune: iters >= 1");
  cudaStream_t st = y->ctx->stream;
  cudaEvent_t e0, e1;
  PAS_CUDA_TRY(y->ctx, cudaStreamSynchronize(st));
  PAS_CUDA_TRY(y->ctx, cudaEventCreate(&e0));
  PAS_CUDA_TRY(y->ctx, cudaEventCreate(&e1));
  // each candidate: `iters` launches captured in a graph, timed on the GPU
  // (host launch latency does not enter the measurement)
  cudaStream_t cs = y->ctx->capture_stream;
  auto time_it = [&](auto&& launch) -> float {
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return 1e30f;
    for (int i = 0; i < iters; ++i) launch(cs);
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess || !g) return 1e30f;
    cudaGraphExec_t ex = nullptr;
    float ms = 1e30f;
    if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
      cudaGraphLaunch(ex, st);
      cudaEventRecord(e0, st);
      cudaGraphLaunch(ex, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      cudaGraphExecDestroy(ex);
    }
    cudaGraphDestroy(g);
    return ms;
  };
  // rows pass
  float best = 1e30f;
  pas_pyr_tuning bt{y->rows, y->n_schunks, y->G, y->H};
  const int rows_c[4] = {2, 4, 8, pas::ROWS_WIDE};
  for (int r : rows_c) {
    int last_chunk = -1;
    const int cmax = r == pas::ROWS_WIDE ? y->s_chunk_wide : y->s_chunk_max;
    for (int nc = 1; nc <= y->n_s; ++nc) {
      const int chunk = (y->n_s + nc - 1) / nc;
      if (chunk == last_chunk || chunk > cmax) continue;
      last_chunk = chunk;
      y->rows = r;
      y->s_chunk = chunk;
      y->n_schunks = (y->n_s + chunk - 1) / chunk;
      const float ms = time_it([&](cudaStream_t q) { pas::launch_rows(y, d_opd, q); });
      if (ms < best) {
        best = ms;
        bt.rows_per_cta = r;
        bt.row_chunks = y->n_schunks;
      }
    }
  }
  pas_pyr_tuning cur = bt;
  cur.col_groups = y->G;
  cur.col_split = y->H;
  pas_pyr_set_tuning(y, &cur);
  pas::launch_rows(y, d_opd, st);
  // columns pass (with the frame/slopes tail, into the internal frame)
  best = 1e30f;
  for (int H = 1; H <= y->h_max; ++H) {
    if (!pas::split_ok(y, H)) continue;
    y->H = H;
    int last_kper = -1;
    for (int G = 1; G <= y->p.K; ++G) {
      const int kper = (y->p.K + G - 1) / G;
      if (kper == last_kper) continue;
      last_kper = kper;
      y->kper = kper;
      y->G = (y->p.K + kper - 1) / kper;
      const float ms = time_it([&](cudaStream_t q) { pas::launch_cols(y, nullptr, nullptr, q, nullptr, false); });
      if (ms < best) {
        best = ms;
        bt.col_groups = y->G;
        bt.col_split = H;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pas_status s = pas::check_launch(y->ctx, "pas_pyr_autotune launches");
  if (s != PAS_OK) return s;
  pas_pyr_set_tuning(y, &bt);
  if (out) *out = bt;
  return PAS_OK;
}

pas_status pas_ccd_noise(pas_ctx_t ctx, const float* d_in, float* d_out, int32_t n, double photons,
                         int32_t n_pupil_pixels, double ron, uint64_t seed, int64_t frame_index) {
  if (!ctx || !d_in || !d_out) return pas::set_global_error(PAS_EINVAL, "pas_ccd_noise: NULL argument");
  PAS_CHECK_ARG(ctx, n >= 0 && n_pupil_pixels > 0 && ron >= 0 && frame_index >= 0, "pas_ccd_noise: bad argument");
  if (n == 0) return PAS_OK;
  const float scale = photons > 0.0 ? (float)(photons / (double)n_pupil_pixels) : 0.f;
  int threads = 256, blocks = (n + threads - 1) / threads;
  pas::ccd_noise_kernel<<<blocks, threads, 0, ctx->stream>>>(d_in, d_out, n, scale, (float)ron, seed, frame_index);
  return pas::check_launch(ctx, "pas_ccd_noise launch");
}

}  // extern "C"

// ------------------------------------------------------------------------------
// Allocation-free pyramid measurement.
//
// For callers that cannot allocate device memory while they run: a simulation
// embedded in a host application whose allocator forbids cudaMalloc after start-up,
// code running while another library owns the device allocator, or a context where
// a cudaMalloc would synchronise the device at the wrong moment. Everything the
// measurement needs besides the caller's input and outputs lives in one fixed array
// of device memory compiled into this library; every GPU that loads the library
// holds it until the process exits.
namespace pas {

constexpr int STATIC_MAX_K = 256;      // modulation points
constexpr int STATIC_MAX_N = 960;      // FFT grid side
constexpr int STATIC_MAX_NSUB = 128;   // sub-apertures across
constexpr int STATIC_TABLE = 1024;     // twiddle / mask entries
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)PAS_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_pyr_scratch[STATIC_SCRATCH_BYTES];

constexpr int STATIC_MAX_DEVICES = 64;
static std::mutex g_static_mutex;
static unsigned char* g_static_ptr[STATIC_MAX_DEVICES] = {};
static int g_static_sms[STATIC_MAX_DEVICES] = {};

// Host tables of one call, filled under g_static_mutex and copied to the scratch
// array before the mutex is released (a copy from pageable memory returns once the
// source has been read), so concurrent callers never share them mid-call and no
// call puts them on its thread's stack.
struct StaticTables {
  int32_t valid[STATIC_MAX_NSUB * STATIC_MAX_NSUB];
  int kmap[STATIC_MAX_K], key_rep[STATIC_MAX_K], key_ey[STATIC_MAX_K];
  float alpha[STATIC_MAX_K], beta[STATIC_MAX_K];
  float2 tw[STATIC_TABLE], mk[STATIC_TABLE];
  float2 tw4[STATIC_TABLE], mk4[STATIC_TABLE];
  unsigned char vpix[(2 * STATIC_MAX_NSUB) * (2 * STATIC_MAX_NSUB)];
};
static_assert(four_tw_size(960) <= STATIC_TABLE && four_mask_size(960) <= STATIC_TABLE, "four-step tables");
static StaticTables g_static_tables;

// Device address of the scratch array for the current device (looked up once per
// device, with that device current). The caller holds g_static_mutex.
static pas_status static_scratch_locked(unsigned char** out, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_global_error(PAS_ECUDA, "pas_pyr_measure_static: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= STATIC_MAX_DEVICES)
    return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: device index %d out of range", dev);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pyr_scratch);
    if (e != cudaSuccess || !p)
      return set_global_error(PAS_ECUDA, "pas_pyr_measure_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_global_error(PAS_ECUDA, "pas_pyr_measure_static: %s", cudaGetErrorString(e));
    g_static_ptr[dev] = static_cast<unsigned char*>(p);
    g_static_sms[dev] = n;
  }
  *out = g_static_ptr[dev];
  *sms = g_static_sms[dev];
  return PAS_OK;
}

}  // namespace pas

extern "C" pas_status pas_pyr_measure_static(const pas_pyr_params* pp, const int32_t* h_valid, int32_t n_valid,
                                             const float* d_sn, const float* d_opd, float* d_frame,
                                             float* d_slopes, void* cuda_stream) {
  using namespace pas;
  if (!pp || !d_opd || !d_frame)
    return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: NULL parameters, input or frame");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  {
    // the table copies below read host memory that is reused by the next call: a
    // graph recorded from them would replay stale tables, so a capturing stream is
    // refused before anything is enqueued
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess)
      return set_global_error(PAS_ECUDA, "pas_pyr_measure_static: %s", cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone)
      return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: the stream is being captured; this call "
                              "copies host tables and cannot be recorded (use pas_pyr_create / pas_pyr_measure)");
  }
  const pas_pyr_params p = *pp;
  if (!(p.Np > 0 && p.N == 2 * p.Np && p.n_sub > 0 && p.N % (2 * p.n_sub) == 0 && p.K >= 1 &&
        p.K <= STATIC_MAX_K && p.wavelength_nm > 0 && p.mod_radius >= 0 && p.obs >= 0 && p.obs < 1))
    return set_global_error(PAS_EINVAL,
                            "pas_pyr_measure_static: need N = 2 Np, N a multiple of 2 n_sub, 1 <= K <= %d", STATIC_MAX_K);
  PyrKernels kern;
  if (!lookup_kernels(p.N, &kern) || p.N > STATIC_MAX_N)
    return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: FFT size N=%d not supported here (max %d)",
                            p.N, STATIC_MAX_N);
  const int b = p.N / (2 * p.n_sub), nd = 2 * p.n_sub;
  if (b > 16 || p.n_sub > STATIC_MAX_NSUB)
    return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: at most 16 fine pixels per detector pixel "
                            "and %d sub-apertures across", STATIC_MAX_NSUB);
  if (kern.tw_n > STATIC_TABLE || kern.buf_n > STATIC_TABLE)
    return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: table size");
  if (h_valid && (n_valid <= 0 || n_valid > p.n_sub * p.n_sub))
    return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: bad n_valid");
  if (!h_valid && p.Np % p.n_sub != 0)
    return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: geometric rule needs Np multiple of n_sub");

  std::lock_guard<std::mutex> lock(g_static_mutex);
  StaticTables& T = g_static_tables;
  // valid sub-apertures
  int32_t nv = 0;
  if (h_valid) {
    for (int j = 0; j < n_valid; ++j) {
      if (h_valid[j] < 0 || h_valid[j] >= p.n_sub * p.n_sub || (j > 0 && h_valid[j] <= h_valid[j - 1]))
        return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: valid indices must be ascending in [0, n_sub^2)");
      T.valid[j] = h_valid[j];
    }
    nv = n_valid;
  } else {
    pas_status s = pas_valid_subaps(p.Np, p.obs, p.n_sub, T.valid, STATIC_MAX_NSUB * STATIC_MAX_NSUB, &nv);
    if (s != PAS_OK) return s;
  }
  if (d_slopes && nv <= 0) return set_global_error(PAS_EINVAL, "pas_pyr_measure_static: no valid sub-aperture");

  // rows passes, tilts, twiddles, mask and the valid-pixel map: the builders of
  // pas_pyr_create, written into the file-scope tables
  const int n_s = pyr_tilt_tables(p.Np, p.N, p.K, p.mod_radius, 1, nullptr, nullptr, nullptr, T.kmap, T.alpha,
                                  nullptr, T.beta, T.key_rep, T.key_ey);
  fft_twiddles_into(p.N, T.tw);
  pyr_mask_table(p.N, kern.buf_n, T.mk);
  quadrant_valid_map(p.n_sub, T.valid, nv, T.vpix);
  if (four_step_ok(p.N)) four_step_tables(p.N, T.tw4, T.mk4);

  // carve the scratch array
  unsigned char* base = nullptr;
  int sms = 0;
  pas_status st0 = static_scratch_locked(&base, &sms);
  if (st0 != PAS_OK) return st0;
  size_t off = 0;
  auto carve = [&](size_t bytes) -> unsigned char* {
    unsigned char* q = base + off;
    off += (bytes + 255) / 256 * 256;
    return q;
  };
  pas_pyr_s y;
  y.p = p;
  y.kern = kern;
  y.b = b;
  y.nd = nd;
  y.n_s = n_s;
  y.n_valid = nv;
  y.T_obs = obstruction_threshold(p.Np, p.obs);
  const double inv = 1.0 / p.wavelength_nm;
  y.inv_hi = (float)inv;
  y.inv_lo = (float)(inv - (double)y.inv_hi);
  y.rows = 4;
  y.n_schunks = (n_s + 3) / 4;
  y.s_chunk = (n_s + y.n_schunks - 1) / y.n_schunks;
  y.smem_cols = cols_smem(&y, b);
  cudaError_t e = cudaSuccess;
  {
    // the columns pass's resident CTAs per SM, as pas_pyr_create counts them
    int occ = 1;
    e = raise_dyn_smem((const void*)kern.cols, y.smem_cols);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern.cols, b * 32, y.smem_cols);
    if (e != cudaSuccess) return set_global_error(PAS_ECUDA, "pas_pyr_measure_static: %s", cudaGetErrorString(e));
    pick_modulation_groups(p.K, nd, std::max(1, occ) * std::max(1, sms), &y.kper, &y.G,
                           four_step_ok(p.N) ? four_tpw(p.N) : 1);
  }
  y.d_H = reinterpret_cast<float2*>(carve(sizeof(float2) * (size_t)n_s * p.N * p.Np));
  y.d_part = reinterpret_cast<float*>(carve(sizeof(float) * (size_t)y.G * nd * nd));
  y.d_tw = reinterpret_cast<float2*>(carve(sizeof(float2) * kern.tw_n));
  y.d_mask = reinterpret_cast<float2*>(carve(sizeof(float2) * kern.buf_n));
  if (four_step_ok(p.N)) {
    y.d_tw4 = reinterpret_cast<float2*>(carve(sizeof(float2) * four_tw_size(p.N)));
    y.d_mk4 = reinterpret_cast<float2*>(carve(sizeof(float2) * four_mask_size(p.N)));
  }
  y.d_alpha = reinterpret_cast<float*>(carve(sizeof(float) * p.K));
  y.d_tilt = reinterpret_cast<float2*>(carve(sizeof(float2) * (size_t)p.K * p.Np));
  y.d_beta = reinterpret_cast<float*>(carve(sizeof(float) * n_s));
  y.d_kmap = reinterpret_cast<int*>(carve(sizeof(int) * p.K));
  y.d_valid = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * std::max(nv, 1)));
  y.d_vpix = carve((size_t)nd * nd);
  y.d_flux_part = reinterpret_cast<double*>(carve(sizeof(double) * nd));
  y.d_done_col = reinterpret_cast<unsigned int*>(carve(sizeof(unsigned int) * nd));
  y.d_frame_ctr = reinterpret_cast<long long*>(carve(sizeof(long long)));
  y.d_frame = d_frame;
  if (off > STATIC_SCRATCH_BYTES)
    return set_global_error(PAS_EINVAL,
                            "pas_pyr_measure_static: this geometry needs %zu bytes of scratch, the library holds %zu "
                            "(use pas_pyr_create / pas_pyr_measure)", off, STATIC_SCRATCH_BYTES);
  y.has_sn = d_sn != nullptr;
  y.d_sn = const_cast<float*>(d_sn);
  const size_t smem_rows = rows_smem(&y, y.rows, y.s_chunk);
  e = raise_dyn_smem((const void*)kern.rows, smem_rows);
  // tables in, counters (and the unused noise frame counter) cleared
  auto H2D = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  H2D(y.d_tw, T.tw, sizeof(float2) * kern.tw_n);
  H2D(y.d_mask, T.mk, sizeof(float2) * kern.buf_n);
  if (four_step_ok(p.N)) {
    H2D(y.d_tw4, T.tw4, sizeof(float2) * four_tw_size(p.N));
    H2D(y.d_mk4, T.mk4, sizeof(float2) * four_mask_size(p.N));
  }
  H2D(y.d_alpha, T.alpha, sizeof(float) * p.K);
  if (e == cudaSuccess) {
    tilt_table_kernel<<<p.K, 256, 0, st>>>(y.d_alpha, nullptr, p.K, p.Np, y.d_tilt);
    e = cudaGetLastError();
  }
  H2D(y.d_beta, T.beta, sizeof(float) * n_s);
  H2D(y.d_kmap, T.kmap, sizeof(int) * p.K);
  H2D(y.d_valid, T.valid, sizeof(int32_t) * std::max(nv, 1));
  H2D(y.d_vpix, T.vpix, (size_t)nd * nd);
  if (e == cudaSuccess) e = cudaMemsetAsync(y.d_done_col, 0, sizeof(unsigned int) * nd, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(y.d_frame_ctr, 0, sizeof(long long), st);
  if (e != cudaSuccess) return set_global_error(PAS_ECUDA, "pas_pyr_measure_static: %s", cudaGetErrorString(e));
  launch_rows(&y, d_opd, st);
  launch_cols(&y, d_frame, d_slopes, st, nullptr, false);
  if (d_slopes) launch_slopes(&y, d_frame, d_slopes, st, nullptr, false);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_global_error(PAS_ECUDA, "pas_pyr_measure_static launch: %s", cudaGetErrorString(e));
  return PAS_OK;
}
