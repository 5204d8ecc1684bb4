// Reverse mode of the single-mesh PM step (added for differentiable use; the
// paper itself has no adjoint).  Forward, per step: rho = sum m W(x - c),
// a = A rho (Eqs. 1-3), a_p = sum a(c) W(x_p - c), v' = v + c_k a_p,
// x' = x + c_d v'.  With W the CIC weight prod_d (1 - |x_d - c_d|), whose
// derivative along d is -1 on the lower and +1 on the upper corner factor:
//   k_adj_interp:  lam_v += c_d lam_x;  lam_a = c_k lam_v;
//                  lam_A(c) += lam_a W(x - c)  (transpose of interpolation;
//                  one float4 vector reduction per corner when lam_A is
//                  interleaved);
//                  lam_x += sum_c (lam_a . a(c)) grad W(x - c)
//   (A^T on the mesh, solve.cu)
//   k_adj_deposit: lam_x += m sum_c lam_rho(c) grad W(x - c)
#include <cuda_runtime.h>
#include <stdint.h>

#include "particles.cuh"
#include "pm_common.cuh"

namespace pm {

namespace {

struct Cic {
  int i0[3], i1[3];
  float w[2][3], dw[2][3];
};

__device__ __forceinline__ Cic cic_of(const float* x, int n) {
  Cic c;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float f = floorf(x[d]);
    float w1 = __fsub_rn(x[d], f);
    int i0 = (int)f;
    if (i0 >= n) i0 -= n;
    if (i0 < 0) i0 += n;
    c.i0[d] = i0;
    c.i1[d] = (i0 + 1 == n) ? 0 : i0 + 1;
    c.w[0][d] = __fsub_rn(1.0f, w1);
    c.w[1][d] = w1;
    c.dw[0][d] = -1.0f;
    c.dw[1][d] = 1.0f;
  }
  return c;
}

__device__ __forceinline__ int64_t corner_index(const Cic& c, int dx, int dy, int dz, int n) {
  return ((int64_t)(dz ? c.i1[2] : c.i0[2]) * n + (dy ? c.i1[1] : c.i0[1])) * n + (dx ? c.i1[0] : c.i0[0]);
}

__global__ void k_adj_deposit(const float* x, int64_t np, float m, int n, const float* lam_rho, float* lam_x) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const float xp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
    const Cic c = cic_of(xp, n);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
      const float v = __ldg(lam_rho + corner_index(c, dx, dy, dz, n));
      g0 += v * c.dw[dx][0] * c.w[dy][1] * c.w[dz][2];
      g1 += v * c.w[dx][0] * c.dw[dy][1] * c.w[dz][2];
      g2 += v * c.w[dx][0] * c.w[dy][1] * c.dw[dz][2];
    }
    lam_x[3 * p] += m * g0;
    lam_x[3 * p + 1] += m * g1;
    lam_x[3 * p + 2] += m * g2;
  }
}

template <bool V4>
__global__ void k_adj_interp(const float* x, int64_t np, int n, const float* acc, float ck, float cd, float* lam_x,
                             float* lam_v, float* lam_A) {
  const int64_t n3 = (int64_t)n * n * n;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const float xp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
    float la[3], lv[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lv[d] = lam_v[3 * p + d] + cd * lam_x[3 * p + d];
      la[d] = ck * lv[d];
      lam_v[3 * p + d] = lv[d];
    }
    const Cic c = cic_of(xp, n);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
      const int64_t idx = corner_index(c, dx, dy, dz, n);
      const float w = c.w[dx][0] * c.w[dy][1] * c.w[dz][2];
      if (V4) {
        atomicAdd(reinterpret_cast<float4*>(lam_A) + idx, make_float4(la[0] * w, la[1] * w, la[2] * w, 0.f));
      } else {
        atomicAdd(lam_A + idx, la[0] * w);
        atomicAdd(lam_A + n3 + idx, la[1] * w);
        atomicAdd(lam_A + 2 * n3 + idx, la[2] * w);
      }
      const float dot = la[0] * __ldg(acc + idx) + la[1] * __ldg(acc + n3 + idx) + la[2] * __ldg(acc + 2 * n3 + idx);
      g0 += dot * c.dw[dx][0] * c.w[dy][1] * c.w[dz][2];
      g1 += dot * c.w[dx][0] * c.dw[dy][1] * c.w[dz][2];
      g2 += dot * c.w[dx][0] * c.w[dy][1] * c.dw[dz][2];
    }
    lam_x[3 * p] += g0;
    lam_x[3 * p + 1] += g1;
    lam_x[3 * p + 2] += g2;
  }
}

int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_adj_deposit(const float* x, int64_t n, float m, int nf, const float* lam_rho, float* lam_x,
                               cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_adj_deposit<<<grid_of(n), 256, 0, st>>>(x, n, m, nf, lam_rho, lam_x);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_adj_interp(const float* x, int64_t n, int nf, const float* acc, float ck, float cd, float* lam_x,
                              float* lam_v, float* lam_A, bool interleaved, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (interleaved)
    k_adj_interp<true><<<grid_of(n), 256, 0, st>>>(x, n, nf, acc, ck, cd, lam_x, lam_v, lam_A);
  else
    k_adj_interp<false><<<grid_of(n), 256, 0, st>>>(x, n, nf, acc, ck, cd, lam_x, lam_v, lam_A);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace pm
