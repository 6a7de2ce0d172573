// Shared-memory mixed-radix FFT -> pointwise mask -> inverse FFT, one warp per
// transform, for the pyramid propagation (Sec. GPU acceleration: "pyramid
// propagation from wavefront to detector plane").
//
// Scheme (in place, length N = R0 R1 ... R_{M-1}, radices 2, 3, 4, 5, 8, 15, 16):
//   forward  : decimation-in-frequency passes 0 .. M-2; pass i works on blocks of
//              length L_i = N / (R0 .. R_{i-1}), stride S_i = L_i / R_i: radix-R_i
//              butterfly, then twiddle w_{L_i}^{n1 k};
//   middle   : pass M-1 (contiguous groups of R_{M-1}) does the last forward
//              butterfly, multiplies by the mask stored in the same digit-reversed
//              position order, and the first inverse butterfly, all in registers;
//   inverse  : decimation-in-time passes M-2 .. 0 (conjugate twiddle, then the
//              inverse butterfly) restore natural order.
// The first pass reads its inputs from a functor (nothing is staged) and the last
// pass hands its outputs to a functor, so callers fuse the phasor/tilt multiply
// and the |.|^2 accumulation into the transform.
//
// Shared-memory layout: element x of a transform lives at x + (x >> 4) (one
// float2 of padding every 16) so that the strided passes spread over the banks.
// Twiddles of pass i live in their own table, entry (k - 1) S_i + n1 = w_{L_i}^{n1 k},
// so lanes of a pass read consecutive or identical entries.
// The radix plan of each size was chosen with a bank-conflict model (fewest
// shared-memory wavefronts at >= 90 % lane use for the large sizes).
#pragma once
#include <cuda_runtime.h>

namespace pas {

__host__ __device__ constexpr int plan_count(int N) {
  switch (N) {
    case 16: case 24: case 32: case 40: case 48: case 64: case 80: case 120: case 128:
    case 240: case 256:
      return 2;
    case 96: case 160: case 192: case 320: case 480: case 512: case 640: case 960:
      return 3;
    default:
      return 0;
  }
}

__host__ __device__ constexpr int plan_radix(int N, int i) {
  switch (N) {
    case 16: { constexpr int r[] = {4, 4}; return r[i]; }
    case 24: { constexpr int r[] = {3, 8}; return r[i]; }
    case 32: { constexpr int r[] = {4, 8}; return r[i]; }
    case 40: { constexpr int r[] = {5, 8}; return r[i]; }
    case 48: { constexpr int r[] = {3, 16}; return r[i]; }
    case 64: { constexpr int r[] = {4, 16}; return r[i]; }
    case 80: { constexpr int r[] = {5, 16}; return r[i]; }
    case 96: { constexpr int r[] = {3, 2, 16}; return r[i]; }
    case 120: { constexpr int r[] = {15, 8}; return r[i]; }
    case 128: { constexpr int r[] = {8, 16}; return r[i]; }
    case 160: { constexpr int r[] = {5, 2, 16}; return r[i]; }
    case 192: { constexpr int r[] = {3, 4, 16}; return r[i]; }
    case 240: { constexpr int r[] = {15, 16}; return r[i]; }
    case 256: { constexpr int r[] = {16, 16}; return r[i]; }
    case 320: { constexpr int r[] = {5, 4, 16}; return r[i]; }
    case 480: { constexpr int r[] = {15, 2, 16}; return r[i]; }
    case 512: { constexpr int r[] = {2, 16, 16}; return r[i]; }
    case 640: { constexpr int r[] = {5, 8, 16}; return r[i]; }
    case 960: { constexpr int r[] = {15, 4, 16}; return r[i]; }
    default: return 0;
  }
}

__host__ __device__ constexpr int block_len(int N, int pass) {
  int l = N;
  for (int j = 0; j < pass; ++j) l /= plan_radix(N, j);
  return l;
}

// Offset of pass i's twiddle table: sum over earlier passes of (R - 1) * S.
__host__ __device__ constexpr int tw_offset(int N, int pass) {
  int o = 0;
  for (int j = 0; j < pass; ++j) o += (plan_radix(N, j) - 1) * (block_len(N, j) / plan_radix(N, j));
  return o;
}

// Total twiddle entries (forward passes 0 .. M-2).
__host__ __device__ constexpr int tw_size(int N) { return tw_offset(N, plan_count(N) - 1); }

__host__ __device__ constexpr int phys(int x) { return x + (x >> 4); }
// float2 slots of one padded transform buffer
__host__ __device__ constexpr int buf_len(int N) { return phys(N - 1) + 1; }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// DFT constants (exact values of the trigonometric numbers involved)
#define PAS_SQRT1_2 0.70710678118654752440f
#define PAS_SQRT3_2 0.86602540378443864676f
#define PAS_C51 0.30901699437494742410f    /* cos(2 pi / 5) */
#define PAS_C52 (-0.80901699437494742410f) /* cos(4 pi / 5) */
#define PAS_S51 0.95105651629515357212f    /* sin(2 pi / 5) */
#define PAS_S52 0.58778525229247312917f    /* sin(4 pi / 5) */
#define PAS_C16 0.92387953251128675613f    /* cos(pi / 8) */
#define PAS_S16 0.38268343236508977173f    /* sin(pi / 8) */

// In-register DFT of R points; forward uses exp(-2 pi i nk/R), inverse exp(+...).
template <int R, bool INV> struct Bfly;

template <bool INV> struct Bfly<2, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV> struct Bfly<4, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = rot90<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV> struct Bfly<8, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 b[4], c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      b[k] = cadd(v[k], v[k + 4]);
      c[k] = csub(v[k], v[k + 4]);
    }
    // c_k *= w8^k, w8 = exp(-+ i pi / 4)
    {
      float2 t = c[1];
      c[1] = INV ? make_float2((t.x - t.y) * PAS_SQRT1_2, (t.x + t.y) * PAS_SQRT1_2)
                 : make_float2((t.x + t.y) * PAS_SQRT1_2, (t.y - t.x) * PAS_SQRT1_2);
      c[2] = rot90<INV>(c[2]);
      t = c[3];
      c[3] = INV ? make_float2((-t.x - t.y) * PAS_SQRT1_2, (t.x - t.y) * PAS_SQRT1_2)
                 : make_float2((t.y - t.x) * PAS_SQRT1_2, (-t.x - t.y) * PAS_SQRT1_2);
    }
    Bfly<4, INV>::run(b);
    Bfly<4, INV>::run(c);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      v[2 * m] = b[m];
      v[2 * m + 1] = c[m];
    }
  }
};

template <bool INV> struct Bfly<3, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 t = cadd(v[1], v[2]);
    float2 d = csub(v[1], v[2]);
    float2 m = make_float2(fmaf(-0.5f, t.x, v[0].x), fmaf(-0.5f, t.y, v[0].y));
    float2 r = rot90<INV>(cscale(d, PAS_SQRT3_2));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};

template <bool INV> struct Bfly<5, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 s1 = cadd(v[1], v[4]), d1 = csub(v[1], v[4]);
    float2 s2 = cadd(v[2], v[3]), d2 = csub(v[2], v[3]);
    float2 a0 = v[0];
    float2 p1 = make_float2(a0.x + PAS_C51 * s1.x + PAS_C52 * s2.x, a0.y + PAS_C51 * s1.y + PAS_C52 * s2.y);
    float2 p2 = make_float2(a0.x + PAS_C52 * s1.x + PAS_C51 * s2.x, a0.y + PAS_C52 * s1.y + PAS_C51 * s2.y);
    float2 q1 = make_float2(PAS_S51 * d1.x + PAS_S52 * d2.x, PAS_S51 * d1.y + PAS_S52 * d2.y);
    float2 q2 = make_float2(PAS_S52 * d1.x - PAS_S51 * d2.x, PAS_S52 * d1.y - PAS_S51 * d2.y);
    q1 = rot90<INV>(q1);
    q2 = rot90<INV>(q2);
    v[0] = make_float2(a0.x + s1.x + s2.x, a0.y + s1.y + s2.y);
    v[1] = cadd(p1, q1);
    v[4] = csub(p1, q1);
    v[2] = cadd(p2, q2);
    v[3] = csub(p2, q2);
  }
};

// 15 = 3 x 5 by the prime-factor (Good-Thomas) mapping: input n = (5 n1 + 3 n2)
// mod 15, output k = (10 k1 + 6 k2) mod 15; no internal twiddles.
template <bool INV> struct Bfly<15, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 y[3][5];
#pragma unroll
    for (int n1 = 0; n1 < 3; ++n1) {
#pragma unroll
      for (int n2 = 0; n2 < 5; ++n2) y[n1][n2] = v[(5 * n1 + 3 * n2) % 15];
      Bfly<5, INV>::run(y[n1]);
    }
#pragma unroll
    for (int k2 = 0; k2 < 5; ++k2) {
      float2 t[3] = {y[0][k2], y[1][k2], y[2][k2]};
      Bfly<3, INV>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 3; ++k1) v[(10 * k1 + 6 * k2) % 15] = t[k1];
    }
  }
};

// 16 = 4 x 4 Cooley-Tukey with the internal twiddles w16^(n2 k1).
template <bool INV> struct Bfly<16, INV> {
  static __device__ __forceinline__ float2 w16(float2 a, int m) {
    // a * exp(-+ 2 pi i m / 16), m in 0..9
    const float c[10] = {1.f, PAS_C16, PAS_SQRT1_2, PAS_S16, 0.f, -PAS_S16, -PAS_SQRT1_2, -PAS_C16, -1.f, -PAS_C16};
    const float s[10] = {0.f, PAS_S16, PAS_SQRT1_2, PAS_C16, 1.f, PAS_C16, PAS_SQRT1_2, PAS_S16, 0.f, -PAS_S16};
    const float sn = INV ? s[m] : -s[m];
    return make_float2(a.x * c[m] - a.y * sn, a.x * sn + a.y * c[m]);
  }
  static __device__ __forceinline__ void run(float2* v) {
    float2 t[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      float2 a[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
      Bfly<4, INV>::run(a);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) t[n2][k1] = (n2 * k1 == 0) ? a[k1] : w16(a[k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 b[4] = {t[0][k1], t[1][k1], t[2][k1], t[3][k1]};
      Bfly<4, INV>::run(b);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
    }
  }
};

// Forward DIF passes I .. M-2. Pass 0 reads through `load(jb, k, x)`: the lane's
// butterfly iteration jb, element k, natural index x (jb and k are compile-time).
template <int N, int I, class Load>
__device__ __forceinline__ void dif_passes(float2* buf, const float2* tw, int lane, Load& load) {
  constexpr int M = plan_count(N);
  constexpr int R = plan_radix(N, I);
  constexpr int L = block_len(N, I);
  constexpr int S = L / R;
  constexpr int NB = N / R;
  constexpr int NJ = (NB + 31) / 32;
  const float2* twp = tw + tw_offset(N, I);
#pragma unroll
  for (int jb = 0; jb < NJ; ++jb) {
    const int b = lane + 32 * jb;
    if (NB % 32 == 0 || b < NB) {
      const int blk = b / S;
      const int n1 = b - blk * S;
      const int base = blk * L + n1;
      float2 v[R];
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = (I == 0) ? load(jb, k, base + k * S) : buf[phys(base + k * S)];
      Bfly<R, false>::run(v);
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], twp[(k - 1) * S + n1]);
#pragma unroll
      for (int k = 0; k < R; ++k) buf[phys(base + k * S)] = v[k];
    }
  }
  __syncwarp();
  if constexpr (I + 2 < M) dif_passes<N, I + 1>(buf, tw, lane, load);
}

// Inverse DIT passes I .. 0. Pass 0 hands (jb, k, x, value) to `store`.
template <int N, int I, class Store>
__device__ __forceinline__ void dit_passes(float2* buf, const float2* tw, int lane, Store& store) {
  constexpr int R = plan_radix(N, I);
  constexpr int L = block_len(N, I);
  constexpr int S = L / R;
  constexpr int NB = N / R;
  constexpr int NJ = (NB + 31) / 32;
  const float2* twp = tw + tw_offset(N, I);
#pragma unroll
  for (int jb = 0; jb < NJ; ++jb) {
    const int b = lane + 32 * jb;
    if (NB % 32 == 0 || b < NB) {
      const int blk = b / S;
      const int n1 = b - blk * S;
      const int base = blk * L + n1;
      float2 v[R];
      v[0] = buf[phys(base)];
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmulc(buf[phys(base + k * S)], twp[(k - 1) * S + n1]);
      Bfly<R, true>::run(v);
      if constexpr (I == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) store(jb, k, base + k * S, v[k]);
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k) buf[phys(base + k * S)] = v[k];
      }
    }
  }
  if constexpr (I > 0) {
    __syncwarp();
    dit_passes<N, I - 1>(buf, tw, lane, store);
  }
}

// Full FFT -> mask -> inverse FFT of one length-N vector by one warp.
// buf: this warp's buf_len(N) float2 of shared memory (padded layout);
// tw: the per-pass twiddle tables (tw_size(N) entries);
// mask[phys(p)] = mask value of the frequency held at digit-reversed position p.
template <int N, class Load, class Store>
__device__ __forceinline__ void fft_mask_ifft(float2* buf, const float2* tw, const float2* mask,
                                              int lane, Load& load, Store& store) {
  constexpr int M = plan_count(N);
  static_assert(M >= 2, "transform needs at least two radix passes");
  dif_passes<N, 0>(buf, tw, lane, load);
  {
    constexpr int R = plan_radix(N, M - 1);
    constexpr int NB = N / R;
    constexpr int NJ = (NB + 31) / 32;
#pragma unroll
    for (int jb = 0; jb < NJ; ++jb) {
      const int b = lane + 32 * jb;
      if (NB % 32 == 0 || b < NB) {
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = buf[phys(b * R + k)];
        Bfly<R, false>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = cmul(v[k], mask[phys(b * R + k)]);
        Bfly<R, true>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) buf[phys(b * R + k)] = v[k];
      }
    }
    __syncwarp();
  }
  dit_passes<N, M - 2>(buf, tw, lane, store);
}

// Forward FFT of one length-N vector by one warp, without mask or inverse: pass 0
// reads through `load` as in fft_mask_ifft; on return buf[phys(p)] holds the
// frequency fft_freq_at(N, p) (digit-reversed order, fft_host.h).
template <int N, class Load>
__device__ __forceinline__ void fft_forward(float2* buf, const float2* tw, int lane, Load& load) {
  constexpr int M = plan_count(N);
  static_assert(M >= 2, "transform needs at least two radix passes");
  dif_passes<N, 0>(buf, tw, lane, load);
  constexpr int R = plan_radix(N, M - 1);
  constexpr int NB = N / R;
  constexpr int NJ = (NB + 31) / 32;
#pragma unroll
  for (int jb = 0; jb < NJ; ++jb) {
    const int b = lane + 32 * jb;
    if (NB % 32 == 0 || b < NB) {
      float2 v[R];
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = buf[phys(b * R + k)];
      Bfly<R, false>::run(v);
#pragma unroll
      for (int k = 0; k < R; ++k) buf[phys(b * R + k)] = v[k];
    }
  }
  __syncwarp();
}

// Outputs a lane receives from the last inverse pass: NJ0 butterflies x R0 values.
template <int N> struct OutShape {
  static constexpr int R0 = plan_radix(N, 0);
  static constexpr int NB0 = N / R0;
  static constexpr int NJ0 = (NB0 + 31) / 32;
  static constexpr int PER_LANE = NJ0 * R0;
};

}  // namespace pas
