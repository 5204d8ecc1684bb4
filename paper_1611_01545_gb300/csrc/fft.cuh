// Shared-memory batched FFTs for the PM solve (paper Sec. 2.1, Eqs. 2-3;
// the per-tile "Fourier_transforms" stage of Fig. 2).
//
// A length-N transform (N = N1 * N2, N in {16, 32, 48, 64, 96, 128, 192, 256,
// 384}) is done as two register passes with one shared-memory exchange
// (four-step):
//   forward, natural in -> "slot" out:
//     step 1, item (seq, j2): N1-point DFT over x[N2 j1 + j2], times W_N^(j2 k1),
//             written back to the same slots N2 k1 + j2;
//     step 2, item (seq, k1): N2-point DFT over slots N2 k1 + j2, result
//             X[k1 + N1 k2] written back to slot N2 k1 + k2.
//   inverse, slot in -> natural out: the same data flow run backwards.
// Each item writes only the slots it read, so the only barrier is between the
// two steps.  X[k] therefore sits at slot(k) = N2 (k mod N1) + k / N1 after a
// forward transform, which the kernel-multiply stage indexes directly; the
// inverse transform consumes that order and restores natural order.
#pragma once
#include <cuda_runtime.h>

namespace pmfft {

constexpr double kPi = 3.14159265358979323846264338327950288;

// Taylor series, evaluated at compile time for the small in-register DFTs.
constexpr double tcos(double x) {
  double s = 1.0, t = 1.0;
  for (int k = 1; k < 40; ++k) { t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k)); s += t; }
  return s;
}
constexpr double tsin(double x) {
  double s = x, t = x;
  for (int k = 1; k < 40; ++k) { t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0)); s += t; }
  return s;
}
// exp(DIR * 2 pi i j / R) with the angle reduced to (-pi, pi].
constexpr double tw_angle(int j, int R, int dir) {
  int jj = ((j % R) + R) % R;
  double a = 2.0 * kPi * (double)jj / (double)R;
  if (a > kPi) a -= 2.0 * kPi;
  return dir * a;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

template <int R> struct SmallestFactor { static constexpr int value = (R % 2 == 0) ? 2 : 3; };

// Multiplies b[p][k1] by exp(DIR 2 pi i p k1 / (P Q)); the factors are
// compile-time constants (Taylor series above), one (p, k1) per instantiation.
template <int P, int Q, int DIR, int I = 0>
struct TwApply {
  static __device__ __forceinline__ void run(float2 (&b)[P][Q]) {
    constexpr int p = I / Q, k1 = I % Q;
    constexpr int R = P * Q;
    if constexpr (p > 0 && k1 > 0) {
      if constexpr ((4 * p * k1) % R == 0) {
        // quarter turns: exact swaps and sign flips, no multiplies
        constexpr int quarter = ((4 * p * k1) / R) % 4;
        const float2 a = b[p][k1];
        if constexpr (quarter == 1) b[p][k1] = DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
        else if constexpr (quarter == 2) b[p][k1] = make_float2(-a.x, -a.y);
        else if constexpr (quarter == 3) b[p][k1] = DIR < 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
      } else {
        constexpr float c = (float)tcos(tw_angle(p * k1, R, DIR));
        constexpr float s = (float)tsin(tw_angle(p * k1, R, DIR));
        b[p][k1] = cmul(b[p][k1], make_float2(c, s));
      }
    }
    if constexpr (I + 1 < P * Q) TwApply<P, Q, DIR, I + 1>::run(b);
  }
};

// In-register DFT of size R in {1, 2, 3, 4, 6, 8, 12, 16, 24}, direction DIR (-1 forward, +1 inverse).
template <int R, int DIR> struct Dft {
  static __device__ __forceinline__ void run(float2 (&a)[R]) {
    constexpr int P = SmallestFactor<R>::value;
    constexpr int Q = R / P;
    float2 b[P][Q];
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int q = 0; q < Q; ++q) b[p][q] = a[q * P + p];
#pragma unroll
    for (int p = 0; p < P; ++p) Dft<Q, DIR>::run(b[p]);
    TwApply<P, Q, DIR>::run(b);
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) {
      float2 c[P];
#pragma unroll
      for (int p = 0; p < P; ++p) c[p] = b[p][k1];
      Dft<P, DIR>::run(c);
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) a[k1 + Q * k2] = c[k2];
    }
  }
};
template <int DIR> struct Dft<1, DIR> {
  static __device__ __forceinline__ void run(float2 (&)[1]) {}
};
template <int DIR> struct Dft<2, DIR> {
  static __device__ __forceinline__ void run(float2 (&a)[2]) {
    float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};
template <int DIR> struct Dft<3, DIR> {
  static __device__ __forceinline__ void run(float2 (&a)[3]) {
    const float c = -0.5f;
    const float s = (float)(DIR * 0.86602540378443864676);  // sin(2 pi / 3)
    float2 t1 = cadd(a[1], a[2]);
    float2 t2 = csub(a[1], a[2]);
    float2 m = make_float2(a[0].x + c * t1.x, a[0].y + c * t1.y);
    // i * s * t2
    float2 r = make_float2(-s * t2.y, s * t2.x);
    a[0] = cadd(a[0], t1);
    a[1] = cadd(m, r);
    a[2] = csub(m, r);
  }
};

template <int N> struct Factor;
template <> struct Factor<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Factor<32> { static constexpr int N1 = 4, N2 = 8; };
template <> struct Factor<48> { static constexpr int N1 = 6, N2 = 8; };
template <> struct Factor<64> { static constexpr int N1 = 8, N2 = 8; };
#ifndef PM_FFT96_N1
#define PM_FFT96_N1 8
#endif
template <> struct Factor<96> { static constexpr int N1 = PM_FFT96_N1, N2 = 96 / PM_FFT96_N1; };
template <> struct Factor<128> { static constexpr int N1 = 8, N2 = 16; };
// large periodic meshes (row / column passes, solve.cu)
template <> struct Factor<192> { static constexpr int N1 = 16, N2 = 12; };
template <> struct Factor<256> { static constexpr int N1 = 16, N2 = 16; };
template <> struct Factor<384> { static constexpr int N1 = 16, N2 = 24; };

template <int N> __host__ __device__ constexpr int slot_of(int k) {
  return Factor<N>::N2 * (k % Factor<N>::N1) + k / Factor<N>::N1;
}
template <int N> __host__ __device__ constexpr int k_of_slot(int s) {
  return (s / Factor<N>::N2) + Factor<N>::N1 * (s % Factor<N>::N2);
}

// Batched transforms over S sequences held in shared memory: element e of
// sequence q is data[q * SS + e * ES].  tw[j] = exp(-2 pi i j / N) (smem);
// twiddle indices j2 k1 stay below N1 N2 = N, so no reduction is needed.
// S, SS, ES are compile-time so the item decomposition costs no division.
// When ES == 1 items are enumerated element-fastest, otherwise
// sequence-fastest, so a warp touches consecutive addresses.
template <int S, int INNER, bool ELEM_FAST>
__device__ __forceinline__ void item_split(int w, int& q, int& j) {
  if (ELEM_FAST) { q = w / INNER; j = w - q * INNER; }
  else { j = w / S; q = w - j * S; }
}

template <int N, int S, int SS, int ES>
__device__ __forceinline__ void fft_fwd(float2* data, const float2* tw) {
  constexpr int N1 = Factor<N>::N1, N2 = Factor<N>::N2;
  constexpr bool EF = (ES == 1);
  for (int w = threadIdx.x; w < S * N2; w += blockDim.x) {
    int q, j2;
    item_split<S, N2, EF>(w, q, j2);
    float2* base = data + q * SS;
    float2 a[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) a[j1] = base[(N2 * j1 + j2) * ES];
    Dft<N1, -1>::run(a);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) a[k1] = cmul(a[k1], tw[j2 * k1]);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) base[(N2 * k1 + j2) * ES] = a[k1];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < S * N1; w += blockDim.x) {
    int q, k1;
    item_split<S, N1, EF>(w, q, k1);
    float2* base = data + q * SS;
    float2 b[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) b[j2] = base[(N2 * k1 + j2) * ES];
    Dft<N2, -1>::run(b);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) base[(N2 * k1 + k2) * ES] = b[k2];
  }
  __syncthreads();
}

template <int N, int S, int SS, int ES>
__device__ __forceinline__ void fft_inv(float2* data, const float2* tw) {
  constexpr int N1 = Factor<N>::N1, N2 = Factor<N>::N2;
  constexpr bool EF = (ES == 1);
  for (int w = threadIdx.x; w < S * N1; w += blockDim.x) {
    int q, k1;
    item_split<S, N1, EF>(w, q, k1);
    float2* base = data + q * SS;
    float2 b[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) b[k2] = base[(N2 * k1 + k2) * ES];
    Dft<N2, 1>::run(b);
    // b[j2] now holds sum_k2 X[k1 + N1 k2] W_N2^(-j2 k2); apply W_N^(-j2 k1).
#pragma unroll
    for (int j2 = 1; j2 < N2; ++j2) b[j2] = cmul(b[j2], conjf2(tw[j2 * k1]));
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) base[(N2 * k1 + j2) * ES] = b[j2];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < S * N2; w += blockDim.x) {
    int q, j2;
    item_split<S, N2, EF>(w, q, j2);
    float2* base = data + q * SS;
    float2 a[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) a[k1] = base[(N2 * k1 + j2) * ES];
    Dft<N1, 1>::run(a);
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) base[(N2 * j1 + j2) * ES] = a[j1];
  }
  __syncthreads();
}

// Inverse transforms of S contiguous rows (ES == 1, row stride SS) with a
// runtime row count: items are split by the compile-time factors only.
template <int N, int SS>
__device__ __forceinline__ void fft_inv_rows(float2* data, int S, const float2* tw) {
  constexpr int N1 = Factor<N>::N1, N2 = Factor<N>::N2;
  for (int w = threadIdx.x; w < S * N1; w += blockDim.x) {
    const int q = w / N1, k1 = w - q * N1;
    float2* base = data + q * SS;
    float2 b[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) b[k2] = base[N2 * k1 + k2];
    Dft<N2, 1>::run(b);
#pragma unroll
    for (int j2 = 1; j2 < N2; ++j2) b[j2] = cmul(b[j2], conjf2(tw[j2 * k1]));
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) base[N2 * k1 + j2] = b[j2];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < S * N2; w += blockDim.x) {
    const int q = w / N2, j2 = w - q * N2;
    float2* base = data + q * SS;
    float2 a[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) a[k1] = base[N2 * k1 + j2];
    Dft<N1, 1>::run(a);
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) base[N2 * j1 + j2] = a[j1];
  }
  __syncthreads();
}

}  // namespace pmfft
