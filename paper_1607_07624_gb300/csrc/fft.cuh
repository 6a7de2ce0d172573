// Shared-memory mixed-radix FFT -> pointwise mask -> inverse FFT, one warp per
// transform, for the pyramid propagation (Sec. GPU acceleration: "pyramid
// propagation from wavefront to detector plane").
//
// Scheme (in place, length N = R0 R1 ... R_{M-1}, radices 2, 3, 4, 5, 8):
//   forward  : decimation-in-frequency passes 0 .. M-2; pass i works on blocks of
//              length L_i = N / (R0 .. R_{i-1}), stride S_i = L_i / R_i, radix-R_i
//              butterfly then twiddle w_{L_i}^{n1 k};
//   middle   : pass M-1 (contiguous groups of R_{M-1}) does the last forward
//              butterfly, multiplies by the mask stored in the same digit-reversed
//              position order, and the first inverse butterfly, all in registers;
//   inverse  : decimation-in-time passes M-2 .. 0 (conjugate twiddle, then the
//              inverse butterfly) restore natural order.
// The first pass reads its inputs from a functor (nothing is staged) and the last
// pass hands its outputs to a functor, so callers fuse the phasor/tilt multiply
// and the |.|^2 accumulation into the transform.
#pragma once
#include <cuda_runtime.h>

namespace pas {

__host__ __device__ constexpr int pow2_exponent(int n) {
  int a = 0;
  while (n % 2 == 0) { n /= 2; ++a; }
  return a;
}

// Radix list of N: all 5s, then all 3s, then the power of two split into 8s and
// 4s (a single 2 when N has one factor of two). Returns 0 on unsupported N.
__host__ __device__ constexpr int radix_count(int N) {
  int n = N, c = 0;
  while (n % 5 == 0) { n /= 5; ++c; }
  while (n % 3 == 0) { n /= 3; ++c; }
  int a = pow2_exponent(n);
  for (int i = 0; i < a; ++i) n /= 2;
  if (n != 1) return 0;
  if (a == 1) return c + 1;
  if (a % 3 == 0) return c + a / 3;
  if (a % 3 == 1) return c + 2 + (a - 4) / 3;
  return c + 1 + (a - 2) / 3;
}

__host__ __device__ constexpr int radix_at(int N, int idx) {
  int n = N, c = 0;
  while (n % 5 == 0) { n /= 5; if (c++ == idx) return 5; }
  while (n % 3 == 0) { n /= 3; if (c++ == idx) return 3; }
  int a = pow2_exponent(n);
  int k = idx - c;
  if (a == 1) return 2;
  if (a % 3 == 0) return 8;
  if (a % 3 == 1) return k < 2 ? 4 : 8;
  return k < 1 ? 4 : 8;
}

__host__ __device__ constexpr int block_len(int N, int pass) {
  int l = N;
  for (int j = 0; j < pass; ++j) l /= radix_at(N, j);
  return l;
}

struct cf { float x, y; };

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
#define PAS_C51 0.30901699437494742410f   /* cos(2 pi / 5) */
#define PAS_C52 (-0.80901699437494742410f) /* cos(4 pi / 5) */
#define PAS_S51 0.95105651629515357212f   /* sin(2 pi / 5) */
#define PAS_S52 0.58778525229247312917f   /* sin(4 pi / 5) */

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
      // (x + iy)(1 -+ i)/sqrt2
      c[1] = INV ? make_float2((t.x - t.y) * PAS_SQRT1_2, (t.x + t.y) * PAS_SQRT1_2)
                 : make_float2((t.x + t.y) * PAS_SQRT1_2, (t.y - t.x) * PAS_SQRT1_2);
      c[2] = rot90<INV>(c[2]);
      t = c[3];
      // (x + iy)(-1 -+ i)/sqrt2
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

// Forward DIF passes I .. M-2. Pass 0 reads through `load(x)` (natural index x).
template <int N, int I, class Load>
__device__ __forceinline__ void dif_passes(float2* buf, const float2* tw, int lane, Load& load) {
  constexpr int M = radix_count(N);
  constexpr int R = radix_at(N, I);
  constexpr int L = block_len(N, I);
  constexpr int S = L / R;
  constexpr int NB = N / R;
  constexpr int NJ = (NB + 31) / 32;
#pragma unroll
  for (int jb = 0; jb < NJ; ++jb) {
    const int b = lane + 32 * jb;
    if (NB % 32 == 0 || b < NB) {
      const int blk = b / S;
      const int n1 = b - blk * S;
      const int base = blk * L + n1;
      float2 v[R];
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = (I == 0) ? load(base + k * S) : buf[base + k * S];
      Bfly<R, false>::run(v);
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], tw[(N / L) * n1 * k]);
#pragma unroll
      for (int k = 0; k < R; ++k) buf[base + k * S] = v[k];
    }
  }
  __syncwarp();
  if constexpr (I + 2 < M) dif_passes<N, I + 1>(buf, tw, lane, load);
}

// Inverse DIT passes I .. 0. Pass 0 hands (jb, k, x, value) to `store`.
template <int N, int I, class Store>
__device__ __forceinline__ void dit_passes(float2* buf, const float2* tw, int lane, Store& store) {
  constexpr int R = radix_at(N, I);
  constexpr int L = block_len(N, I);
  constexpr int S = L / R;
  constexpr int NB = N / R;
  constexpr int NJ = (NB + 31) / 32;
#pragma unroll
  for (int jb = 0; jb < NJ; ++jb) {
    const int b = lane + 32 * jb;
    if (NB % 32 == 0 || b < NB) {
      const int blk = b / S;
      const int n1 = b - blk * S;
      const int base = blk * L + n1;
      float2 v[R];
      v[0] = buf[base];
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmulc(buf[base + k * S], tw[(N / L) * n1 * k]);
      Bfly<R, true>::run(v);
      if constexpr (I == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) store(jb, k, base + k * S, v[k]);
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k) buf[base + k * S] = v[k];
      }
    }
  }
  if constexpr (I > 0) {
    __syncwarp();
    dit_passes<N, I - 1>(buf, tw, lane, store);
  }
}

// Full FFT -> mask -> inverse FFT of one length-N vector by one warp.
// buf: this warp's N float2 of shared memory; tw[j] = exp(-2 pi i j / N);
// mask[p] = mask value of the frequency held at digit-reversed position p.
template <int N, class Load, class Store>
__device__ __forceinline__ void fft_mask_ifft(float2* buf, const float2* tw, const float2* mask,
                                              int lane, Load& load, Store& store) {
  constexpr int M = radix_count(N);
  static_assert(M >= 2, "transform needs at least two radix passes");
  dif_passes<N, 0>(buf, tw, lane, load);
  {
    constexpr int R = radix_at(N, M - 1);
    constexpr int NB = N / R;
    constexpr int NJ = (NB + 31) / 32;
#pragma unroll
    for (int jb = 0; jb < NJ; ++jb) {
      const int b = lane + 32 * jb;
      if (NB % 32 == 0 || b < NB) {
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = buf[b * R + k];
        Bfly<R, false>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = cmul(v[k], mask[b * R + k]);
        Bfly<R, true>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) buf[b * R + k] = v[k];
      }
    }
    __syncwarp();
  }
  dit_passes<N, M - 2>(buf, tw, lane, store);
}

// Outputs a lane receives from the last inverse pass: NJ0 butterflies x R0 values.
template <int N> struct OutShape {
  static constexpr int R0 = radix_at(N, 0);
  static constexpr int NB0 = N / R0;
  static constexpr int NJ0 = (NB0 + 31) / 32;
  static constexpr int PER_LANE = NJ0 * R0;
};

}  // namespace pas
