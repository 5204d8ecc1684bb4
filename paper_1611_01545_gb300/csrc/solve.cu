// Fourier-space PM solve on periodic windows (paper Sec. 2.1, Eqs. 1-3).
//
// One "problem" is an N^3 window of a periodic source mesh whose cell 0 sits
// at origin p*t - b (p = problem coordinates): the whole coarse / single mesh
// (t = N, b = 0), or one buffered fine tile (Fig. 1; N = T = t + 2b).  Three
// kernels per batch of problems:
//   A  per z plane: load the real window plane, real-to-complex along x (two
//      rows packed as one complex row), complex FFT along y -> half spectrum;
//   B  per ky: FFT along z, multiply by the precomputed kernel of each force
//      component (i K_d), inverse FFT along z, keep the output z range;
//   C  per (output z, component): inverse FFT along y, complex-to-real along
//      x (two rows packed), store the output interior into the destination
//      mesh [3][n][n][n].
// The kernel tables already contain the 1/N^3 (tiles) or 1/V (periodic)
// normalisation, so both transform directions are unnormalised.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "fft.cuh"
#include "pm_common.cuh"
#include "tma.cuh"

namespace pm {
using namespace pmfft;

template <int N> struct SolveCfg {
  static constexpr int NH = N / 2 + 1;
  static constexpr int NP = spec_pitch(N);   // row pitch (complex values) of the spectrum buffers
// Threads per block of passes A and C (compile-time tunables; measured on the
// 96^3 tiles: 512 for A, 384 for C).
#ifndef PM_SOLVE_THREADS
#define PM_SOLVE_THREADS 512
#endif
#ifndef PM_SOLVE_C_THREADS
#define PM_SOLVE_C_THREADS 384
#endif
  static constexpr int threads = (N >= 96) ? PM_SOLVE_THREADS : 256;
  static constexpr int threads_c = (N >= 96) ? PM_SOLVE_C_THREADS : 256;
  static constexpr size_t smem_a = sizeof(float2) * (N + (size_t)N * N / 2 + (size_t)N * NP);
};

struct SolveArgs {
  const void* src;
  int src_fixed;
  int src_n;
  int nts;
  int t, b;
  int p0;
  float2* spec;
  float2* spec3;
  const float* kern;
  const float2* tw;
  float* dst;
  int comp_mode;   // pass A only: blockIdx.y selects component pb of a 3-component source at origin 0
  unsigned int* amax;   // pass C: if set, atomicMax of max |output| (float bits; values are >= 0)
  const float* pc;      // pass C: if set, add this coarse force [3][pnc^3] trilinearly prolongated to the fine nodes
  int pnc, prc;         // its edge and the fine cells per coarse cell (a power of two dividing t)
  int* status;          // library status word: ST_TIMEOUT when a bounded copy wait gives up
};

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ void problem_origin(const SolveArgs& a, int p, int& ox, int& oy, int& oz) {
  int px = p % a.nts, py = (p / a.nts) % a.nts, pz = p / (a.nts * a.nts);
  ox = px * a.t - a.b;
  oy = py * a.t - a.b;
  oz = pz * a.t - a.b;
}

// Row loops below give each warp whole rows and each lane strided columns, so
// row indices are computed once per row and no division is needed.
// Global -> shared copies that do not stall the issuing thread (cp.async);
// async_wait() waits for all of the thread's copies (a barrier must follow).
__device__ __forceinline__ void async_copy4(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void async_copy8(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void async_copy16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

#define PM_ROWS(row, nrows) for (int row = threadIdx.x >> 5; row < (nrows); row += (blockDim.x >> 5))
#define PM_COLS(col, ncols) for (int col = threadIdx.x & 31; col < (ncols); col += 32)

template <bool FIXED>
__device__ __forceinline__ float src_value(const void* src, int64_t idx) {
  if (FIXED) return (float)((double)static_cast<const long long*>(src)[idx] * 2.3283064365386963e-10);  // 2^-32
  return __ldg(static_cast<const float*>(src) + idx);
}

__device__ __forceinline__ int wrap1(int g, int n) { return g < 0 ? g + n : (g >= n ? g - n : g); }

// CS > 1 (comp_mode only): the components are interleaved, element i of
// component pb at src[i * CS + pb] (the adjoint's float4 accumulation mesh).
template <int N, bool FIXED, int CS = 1>
__device__ __forceinline__ void solve_a_body(const SolveArgs& a) {
  constexpr int NH = SolveCfg<N>::NH, NP = SolveCfg<N>::NP;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* W = sm + N;               // N/2 packed rows of N
  float2* P = W + N * N / 2;        // N rows (y) of NH, pitch NP
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  const int z = blockIdx.x;
  const int pb = blockIdx.y;
  int ox, oy, oz;
  problem_origin(a, a.p0 + pb, ox, oy, oz);
  const int n = a.src_n;
  const void* src = a.src;
  if (a.comp_mode) {
    ox = oy = oz = 0;
    src = static_cast<const float*>(a.src) + (CS > 1 ? (size_t)pb : (size_t)pb * n * n * n);
  }
  // origins lie in (-n, n) and N <= n, so one conditional wrap suffices
  const int gz = wrap1(oz + z, n);
  PM_ROWS(y, N) {
    const int64_t rowbase = ((int64_t)gz * n + wrap1(oy + y, n)) * n;
    float* w = reinterpret_cast<float*>(W + (y >> 1) * N) + (y & 1);
    if (FIXED) {
      PM_COLS(x, N) w[2 * x] = src_value<FIXED>(src, rowbase + wrap1(ox + x, n));
    } else {
      const float* srow = static_cast<const float*>(src) + rowbase * CS;
      PM_COLS(x, N) async_copy4(w + 2 * x, srow + wrap1(ox + x, n) * CS);
    }
  }
  if (!FIXED) async_wait();
  __syncthreads();
  fft_fwd<N, N / 2, N, 1>(W, tw);
  // Unpack the two real rows of each packed row: A = (Z_k + conj Z_-k)/2, B = (Z_k - conj Z_-k)/(2i).
  PM_ROWS(j, N / 2) {
    const float2* Wj = W + j * N;
    PM_COLS(k, NH) {
      float2 zk = Wj[slot_of<N>(k)];
      float2 zm = Wj[slot_of<N>(k == 0 ? 0 : N - k)];
      P[(2 * j) * NP + k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      P[(2 * j + 1) * NP + k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    }
  }
  __syncthreads();
  fft_fwd<N, NH, 1, NP>(P, tw);
  // N * NP is even for every supported N: copy two complex values per access
  // (the pitch's pad columns are copied too and never read).
  float4* out = reinterpret_cast<float4*>(a.spec + ((size_t)pb * N + z) * N * NP);
  const float4* P4 = reinterpret_cast<const float4*>(P);
  for (int i = threadIdx.x; i < N * NP / 2; i += blockDim.x) out[i] = P4[i];
}

template <int N, bool FIXED, int CS = 1>
__global__ void __launch_bounds__(SolveCfg<N>::threads) k_solve_a(SolveArgs a) {
  solve_a_body<N, FIXED, CS>(a);
}

// The 96^3 tiles' pass A is compiled for 3 resident blocks per SM (40
// registers; 3 blocks fit its shared memory): measured 0.205 -> 0.188 ms.
#ifndef PM_SOLVE_A_MINB
#define PM_SOLVE_A_MINB 3
#endif
template <bool FIXED>
__global__ void __launch_bounds__(SolveCfg<96>::threads, PM_SOLVE_A_MINB) k_solve_a96(SolveArgs a) {
  solve_a_body<96, FIXED>(a);
}

template <int N, bool FIXED>
constexpr auto solve_a_kernel() {
  if constexpr (N == 96) return k_solve_a96<FIXED>;
  else return k_solve_a<N, FIXED>;
}

// Pass B works on one ky row and one chunk of KC kx columns (KC = ceil(NH/2),
// i.e. two chunks, up to N = 128): forward z FFT, the three
// kernel products i K_d F written side by side, then one batched inverse z
// FFT over all 3 KC columns, so a block needs only a few barriers.
// Large meshes (N > 128) take 16 columns per block, so their z columns fit.
template <int N> struct PassB {
  static constexpr int NH = N / 2 + 1;
  static constexpr int KC = N > 128 ? 16 : (NH + 1) / 2;
  static constexpr int nchunk = (NH + KC - 1) / KC;
#ifndef PM_PASSB_THREADS
#define PM_PASSB_THREADS 512
#endif
  static constexpr int threads = N > 128 ? 256 : ((N >= 96) ? PM_PASSB_THREADS : 256);
  // twiddles + [z][3 KC]: the forward transform runs in the first KC columns
  static constexpr size_t smem = sizeof(float2) * (N + 3 * (size_t)N * KC);
};

template <int N>
__device__ __forceinline__ void solve_b_body(const SolveArgs& a) {
  constexpr int NH = PassB<N>::NH, KC = PassB<N>::KC, NP = SolveCfg<N>::NP;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  // [z][3 KC]: component d of the products in columns d KC .. d KC + KC - 1; the
  // density spectrum F is transformed in the columns of component 0 and each
  // thread overwrites its element with the three products (in place for d = 0)
  float2* G = sm + N;
  float2* F = G;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  const int ys = blockIdx.x;      // ky in slot order
  const int half = blockIdx.y;    // which chunk of the kx columns
  const int pb = blockIdx.z;
  const int kx0 = half * KC;
  const int ncol = (NH - kx0) < KC ? (NH - kx0) : KC;
  const float2* in = a.spec + (size_t)pb * N * N * NP + (size_t)ys * NP + kx0;
  for (int i = threadIdx.x; i < N * KC; i += blockDim.x) {
    const int z = i / KC, c = i - z * KC;
    if (c < ncol) async_copy8(F + z * 3 * KC + c, in + (size_t)z * N * NP + c);
    else F[z * 3 * KC + c] = make_float2(0.f, 0.f);
  }
  async_wait();
  __syncthreads();
  fft_fwd<N, KC, 1, 3 * KC>(F, tw);
  const float* K = a.kern + (size_t)ys * NH + kx0;
  const size_t kstride = (size_t)N * N * NH;
  for (int i = threadIdx.x; i < N * KC; i += blockDim.x) {
    const int zs = i / KC, c = i - zs * KC;
    float2* g = G + zs * 3 * KC + c;
    const float2 f = g[0];
    if (c < ncol) {
      const float* Kz = K + (size_t)zs * N * NH + c;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float k = __ldg(Kz + d * kstride);
        g[d * KC] = make_float2(-f.y * k, f.x * k);   // i K f
      }
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) g[d * KC] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  fft_inv<N, 3 * KC, 1, 3 * KC>(G, tw);
  for (int d = 0; d < 3; ++d) {
    float2* out = a.spec3 + ((size_t)pb * 3 + d) * a.t * N * NP + (size_t)ys * NP + kx0;
    for (int i = threadIdx.x; i < a.t * KC; i += blockDim.x) {
      const int zo = i / KC, c = i - zo * KC;
      if (c < ncol) out[(size_t)zo * N * NP + c] = G[(zo + a.b) * 3 * KC + d * KC + c];
    }
  }
}

template <int N>
__global__ void __launch_bounds__(PassB<N>::threads) k_solve_b(SolveArgs a) {
  solve_b_body<N>(a);
}

// The 96^3 tiles' pass B compiled for 3 resident blocks per SM (its shared
// memory allows 3 since the forward transform shares the product buffer).
#ifndef PM_PASSB_MINB
#define PM_PASSB_MINB 3
#endif
__global__ void __launch_bounds__(PassB<96>::threads, PM_PASSB_MINB) k_solve_b96(SolveArgs a) {
  solve_b_body<96>(a);
}

template <int N>
constexpr auto solve_b_kernel() {
  if constexpr (N == 96) return k_solve_b96;
  else return k_solve_b<N>;
}

// Transpose of the solve for one periodic mesh (the adjoint of a_d = K_d * rho):
// the three component spectra (pass A with comp_mode) are z-transformed, each
// multiplied by the conjugate kernel conj(i K_d) = -i K_d and summed, and the
// sum is inverse z-transformed into component slot 0 of spec3; pass C then
// gives the scalar result.
template <int N>
__global__ void __launch_bounds__(PassB<N>::threads) k_solve_b_adj(SolveArgs a) {
  constexpr int NH = PassB<N>::NH, KC = PassB<N>::KC, NP = SolveCfg<N>::NP;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* F = sm + N;             // [z][KC]
  float2* G = F + N * KC;         // [z][KC]
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  const int ys = blockIdx.x, half = blockIdx.y;
  const int kx0 = half * KC;
  const int ncol = (NH - kx0) < KC ? (NH - kx0) : KC;
  const size_t kstride = (size_t)N * N * NH;
  for (int i = threadIdx.x; i < N * KC; i += blockDim.x) G[i] = make_float2(0.f, 0.f);
  for (int d = 0; d < 3; ++d) {
    const float2* in = a.spec + (size_t)d * N * N * NP + (size_t)ys * NP + kx0;
    for (int i = threadIdx.x; i < N * KC; i += blockDim.x) {
      const int z = i / KC, c = i - z * KC;
      F[i] = c < ncol ? in[(size_t)z * N * NP + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_fwd<N, KC, 1, KC>(F, tw);
    const float* K = a.kern + d * kstride + (size_t)ys * NH + kx0;
    for (int i = threadIdx.x; i < N * KC; i += blockDim.x) {
      const int zs = i / KC, c = i - zs * KC;
      if (c < ncol) {
        const float k = __ldg(K + (size_t)zs * N * NH + c);
        const float2 f = F[i];
        G[i] = make_float2(G[i].x + f.y * k, G[i].y - f.x * k);   // += -i K f
      }
    }
    __syncthreads();
  }
  fft_inv<N, KC, 1, KC>(G, tw);
  float2* out = a.spec3 + (size_t)ys * NP + kx0;
  for (int i = threadIdx.x; i < N * KC; i += blockDim.x) {
    const int z = i / KC, c = i - z * KC;
    if (c < ncol) out[(size_t)z * N * NP + c] = G[i];
  }
}

template <int N>
__device__ __forceinline__ void solve_c_body(const SolveArgs& a, float2* tw, float2* P, float2* W);

template <int N>
__global__ void __launch_bounds__(SolveCfg<N>::threads_c) k_solve_c(SolveArgs a) {
  constexpr int NP = SolveCfg<N>::NP;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* P = sm + N;          // [y][kx], pitch NP
  float2* W = P + N * NP;      // t/2 packed rows of N
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  const int zo = blockIdx.x;
  const int d = blockIdx.y;
  const int pb = blockIdx.z;
  const float4* in = reinterpret_cast<const float4*>(a.spec3 + (((size_t)pb * 3 + d) * a.t + zo) * N * NP);
  float4* P4 = reinterpret_cast<float4*>(P);
  for (int i = threadIdx.x; i < N * NP / 2; i += blockDim.x) async_copy16(P4 + i, in + i);
  async_wait();
  __syncthreads();
  solve_c_body<N>(a, tw, P, W);
}

// Pass C after its input plane is in P: inverse y transform, the packed
// inverse x transform of the output rows, the prolongated coarse force, the
// output store and the running max |a|.
template <int N>
__device__ __forceinline__ void solve_c_body(const SolveArgs& a, float2* tw, float2* P, float2* W) {
  constexpr int NH = SolveCfg<N>::NH, NP = SolveCfg<N>::NP;
  const int zo = blockIdx.x;
  const int d = blockIdx.y;
  const int pb = blockIdx.z;
  fft_inv<N, NH, 1, NP>(P, tw);
  const int half_rows = a.t / 2;
  // Inverse x transforms of the output rows, two real rows (b + 2j, b + 2j + 1)
  // packed as one complex row A + i B (A, B their half spectra, extended by
  // conjugate symmetry).  Step 1 forms its inputs from P directly: slot
  // N2 k1 + k2 holds frequency k = k1 + N1 k2.
  {
    constexpr int N1 = Factor<N>::N1, N2 = Factor<N>::N2;
    for (int w = threadIdx.x; w < half_rows * N1; w += blockDim.x) {
      const int j = w / N1, k1 = w - j * N1;
      const float2* Pa = P + (a.b + 2 * j) * NP;
      const float2* Pb = Pa + NP;
      float2 v[N2];
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int k = k1 + N1 * k2;
        float2 A, B;
        if (k <= N / 2) {
          A = Pa[k];
          B = Pb[k];
        } else {
          A = conjf2(Pa[N - k]);
          B = conjf2(Pb[N - k]);
        }
        v[k2] = make_float2(A.x - B.y, A.y + B.x);   // A + i B
      }
      Dft<N2, 1>::run(v);
#pragma unroll
      for (int j2 = 1; j2 < N2; ++j2) v[j2] = cmul(v[j2], conjf2(tw[j2 * k1]));
      float2* base = W + j * N;
#pragma unroll
      for (int j2 = 0; j2 < N2; ++j2) base[N2 * k1 + j2] = v[j2];
    }
    __syncthreads();
    for (int w = threadIdx.x; w < half_rows * N2; w += blockDim.x) {
      const int q = w / N2, j2 = w - q * N2;
      float2* base = W + q * N;
      float2 v[N1];
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) v[k1] = base[N2 * k1 + j2];
      Dft<N1, 1>::run(v);
#pragma unroll
      for (int j1 = 0; j1 < N1; ++j1) base[N2 * j1 + j2] = v[j1];
    }
    __syncthreads();
  }
  int ox, oy, oz;
  problem_origin(a, a.p0 + pb, ox, oy, oz);
  const int n = a.src_n;
  // Prolongation of the coarse force onto this output plane: the coarse values
  // around the tile interior, interpolated in z, staged in P (free by now),
  // then along x onto the output columns (R), so an output cell needs one
  // interpolation in y.
  float* Q = reinterpret_cast<float*>(P);
  const int nq = a.pc ? a.t / a.prc + 1 : 0;
  float* R = Q + nq * nq;   // [nq][t]
  int lr = 0;
  float inv_r = 0.f;
  if (a.pc) {
    lr = __ffs(a.prc) - 1;
    inv_r = 1.0f / (float)a.prc;
    const int gz = oz + a.b + zo;
    const int cz0 = gz >> lr, cz1 = cz0 + 1 == a.pnc ? 0 : cz0 + 1;
    const float wz = (float)(gz & (a.prc - 1)) * inv_r;
    const int cyb = (oy + a.b) >> lr, cxb = (ox + a.b) >> lr;
    const float* c0 = a.pc + ((size_t)d * a.pnc + cz0) * a.pnc * a.pnc;
    const float* c1 = a.pc + ((size_t)d * a.pnc + cz1) * a.pnc * a.pnc;
    PM_ROWS(qy, nq) {
      int cy = cyb + qy;
      if (cy >= a.pnc) cy -= a.pnc;
      PM_COLS(qx, nq) {
        int cx = cxb + qx;
        if (cx >= a.pnc) cx -= a.pnc;
        const size_t o = (size_t)cy * a.pnc + cx;
        Q[qy * nq + qx] = (1.0f - wz) * __ldg(c0 + o) + wz * __ldg(c1 + o);
      }
    }
    __syncthreads();
    PM_ROWS(qy, nq) {
      const float* q = Q + qy * nq;
      PM_COLS(xl, a.t) {
        const int qx = xl >> lr;
        const float fx = (float)(xl & (a.prc - 1)) * inv_r;
        R[qy * a.t + xl] = fmaf(fx, q[qx + 1] - q[qx], q[qx]);
      }
    }
    __syncthreads();
  }
  // Output cells are interior cells: origin + b + local lies inside [0, n) without wrap.
  const int gz = oz + a.b + zo;
  float* dst = a.dst + (size_t)d * n * n * n + ((int64_t)gz * n + oy + a.b) * n + ox + a.b;
  float m = 0.f;
  PM_ROWS(yl, a.t) {
    const float* w = reinterpret_cast<const float*>(W + (yl >> 1) * N + a.b) + (yl & 1);
    float* drow = dst + (int64_t)yl * n;
    PM_COLS(xl, a.t) {
      float val = w[2 * xl];
      m = fmaxf(m, fabsf(val));
      if (a.pc) {
        const int qy = yl >> lr;
        const float fy = (float)(yl & (a.prc - 1)) * inv_r;
        const float lo = R[qy * a.t + xl], hi = R[(qy + 1) * a.t + xl];
        val += fmaf(fy, hi - lo, lo);
      }
      drow[xl] = val;
    }
  }
  if (a.amax) {
    // warp maximum; an atomic only when it raises the running maximum
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > __uint_as_float(*(volatile unsigned int*)a.amax))
      atomicMax(a.amax, __float_as_uint(m));
  }
}

// ---- 96^3 passes staged by the tensor memory accelerator ----------------
//
// The 96^3 transforms (the buffered fine tiles, and a 96^3 periodic mesh)
// move their shared-memory pencils with TMA bulk copies instead of
// per-thread copies:
//   A  the window plane arrives as 36 boxes of 16 x 16 cells (a tensor map
//      of the source mesh; window origins are multiples of 16 cells, so no
//      box crosses the periodic boundary), is repacked into two-row complex
//      rows and transformed as before; the half-spectrum plane leaves as one
//      bulk store;
//   B  the z pencils of KT = 26 kx columns arrive as one 52 x 1 x 96 box of
//      the spectrum (columns past kx = N/2 read as zeros); the second step of
//      the forward z transform, the three kernel products and the first step
//      of each inverse transform run in registers per (column, k1) item; the
//      output z range of each component leaves as one box store;
//   C  the input plane arrives as one bulk copy.
// Spectrum rows are padded to spec_pitch(96) = 50 complex values (400
// bytes), so rows, boxes and planes start on 16-byte boundaries.

constexpr int kTmaAlign = 128;   // shared-memory alignment of every TMA destination and source
constexpr int kBox = 16;         // edge (cells) of the pass-A window boxes

__device__ __forceinline__ unsigned char* tma_align(unsigned char* p) {
  const unsigned a = tma::smem_u32(p);
  return p + ((kTmaAlign - (a & (kTmaAlign - 1))) & (kTmaAlign - 1));
}

// Bounded wait of the whole block for phase 0 of `bar`.  When it gives up
// (the copies did not complete in time) the block records ST_TIMEOUT, waits
// once more (bounded) for copies still in flight, and the caller returns.
__device__ __forceinline__ bool block_wait(uint64_t* bar, int* status) {
  int bad = tma::mbar_wait(bar, 0) ? 0 : 1;
  bad = __syncthreads_or(bad);
  if (bad) {
    if (threadIdx.x == 0 && status) atomicOr(status, ST_TIMEOUT);
    tma::mbar_wait(bar, 0);
  }
  return !bad;
}

template <int N> struct PassAT {
  static constexpr int NH = N / 2 + 1, NP = spec_pitch(N), NB = N / kBox;
  // P [N][NP] (first the staged boxes), W [N/2][N], twiddles
  static constexpr size_t smem = kTmaAlign + sizeof(float2) * ((size_t)N * NP + (size_t)N / 2 * N + N);
};

template <int N>
__global__ void __launch_bounds__(SolveCfg<N>::threads, PM_SOLVE_A_MINB)
    k_solve_a_tma(SolveArgs a, const __grid_constant__ CUtensorMap src_map) {
  using C = PassAT<N>;
  constexpr int NH = C::NH, NP = C::NP, NB = C::NB;
  static_assert((size_t)NB * NB * kBox * kBox <= (size_t)2 * N * NP, "staged window must fit in P");
  extern __shared__ unsigned char smraw_a[];
  __shared__ uint64_t bar;
  float2* P = reinterpret_cast<float2*>(tma_align(smraw_a));   // [y][NP]; first the staged window boxes
  float2* W = P + N * NP;                                        // N/2 packed rows of N
  float2* tw = W + N * N / 2;
  float* S = reinterpret_cast<float*>(P);                        // box (yb, xb) at S + (yb NB + xb) 256
  const int z = blockIdx.x, pb = blockIdx.y;
  int ox, oy, oz;
  problem_origin(a, a.p0 + pb, ox, oy, oz);
  const int n = a.src_n;
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) tma::mbar_arrive_expect_tx(&bar, NB * NB * kBox * kBox * (unsigned)sizeof(float));
    __syncwarp();
    const int gz = wrap1(oz + z, n);
    for (int k = threadIdx.x; k < NB * NB; k += 32) {
      const int yb = k / NB, xb = k - yb * NB;
      tma::tensor_load_3d(S + k * kBox * kBox, &src_map, wrap1(ox + kBox * xb, n), wrap1(oy + kBox * yb, n), gz,
                          &bar);
    }
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  if (!block_wait(&bar, a.status)) return;
  // W[j][x] = (row 2j, row 2j + 1) at x; both rows lie in the same box row pair
  for (int i = threadIdx.x; i < (N / 2) * (N / 4); i += blockDim.x) {
    const int j = i / (N / 4), x = 4 * (i - j * (N / 4));
    const int y0 = 2 * j;
    const float* s0 = S + ((y0 / kBox) * NB + x / kBox) * kBox * kBox + (y0 % kBox) * kBox + x % kBox;
    const float4 r0 = *reinterpret_cast<const float4*>(s0);
    const float4 r1 = *reinterpret_cast<const float4*>(s0 + kBox);
    float4* w = reinterpret_cast<float4*>(W + j * N + x);
    w[0] = make_float4(r0.x, r1.x, r0.y, r1.y);
    w[1] = make_float4(r0.z, r1.z, r0.w, r1.w);
  }
  __syncthreads();
  fft_fwd<N, N / 2, N, 1>(W, tw);
  PM_ROWS(j, N / 2) {
    const float2* Wj = W + j * N;
    PM_COLS(k, NH) {
      float2 zk = Wj[slot_of<N>(k)];
      float2 zm = Wj[slot_of<N>(k == 0 ? 0 : N - k)];
      P[(2 * j) * NP + k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      P[(2 * j + 1) * NP + k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    }
  }
  __syncthreads();
  fft_fwd<N, NH, 1, NP>(P, tw);
  tma::fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    tma::bulk_store(a.spec + ((size_t)pb * N + z) * N * NP, P, (unsigned)(N * NP * sizeof(float2)));
    tma::bulk_commit();
    tma::bulk_wait_all();
  }
}

// Threads and resident blocks per SM of the TMA pass B (compile-time tunables).
#ifndef PM_PASSB_TMA_THREADS
#define PM_PASSB_TMA_THREADS 256
#endif
#ifndef PM_PASSB_TMA_MINB
#define PM_PASSB_TMA_MINB 3
#endif
template <int N> struct PassBT {
  static constexpr int NH = N / 2 + 1, NP = spec_pitch(N);
  static constexpr int KT = 26;                        // kx columns per block: KT * 8 bytes is a multiple of 16
  static constexpr int nchunk = (NH + KT - 1) / KT;
  static constexpr int threads = PM_PASSB_TMA_THREADS;
  // G [3][N][KT] (component, z, column), twiddles
  static constexpr size_t smem = kTmaAlign + sizeof(float2) * (3 * (size_t)N * KT + N);
};

template <int N>
__global__ void __launch_bounds__(PassBT<N>::threads, PM_PASSB_TMA_MINB)
    k_solve_b_tma(SolveArgs a, const __grid_constant__ CUtensorMap spec_map,
                  const __grid_constant__ CUtensorMap spec3_map) {
  using B = PassBT<N>;
  constexpr int NH = B::NH, KT = B::KT;
  constexpr int N1 = Factor<N>::N1, N2 = Factor<N>::N2;
  extern __shared__ unsigned char smraw_b[];
  __shared__ uint64_t bar;
  float2* G = reinterpret_cast<float2*>(tma_align(smraw_b));   // [3][N][KT]
  float2* tw = G + 3 * N * KT;
  const int ys = blockIdx.x, kx0 = blockIdx.y * KT, pb = blockIdx.z;
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    tma::mbar_arrive_expect_tx(&bar, N * KT * (unsigned)sizeof(float2));
    tma::tensor_load_3d(G, &spec_map, 2 * kx0, ys, pb * N, &bar);
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  if (!block_wait(&bar, a.status)) return;
  // forward z transform, step 1 (items (j2, column)), in component 0
  for (int w = threadIdx.x; w < KT * N2; w += blockDim.x) {
    const int j2 = w / KT, c = w - j2 * KT;
    float2* base = G + c;
    float2 v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) v[j1] = base[(N2 * j1 + j2) * KT];
    Dft<N1, -1>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw[j2 * k1]);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) base[(N2 * k1 + j2) * KT] = v[k1];
  }
  __syncthreads();
  // forward step 2, the products i K_d F and step 1 of each inverse
  // transform, per (k1, column) item: F(kz = k1 + N1 k2) sits at slot N2 k1 + k2
  const float* Kb = a.kern + (size_t)ys * NH + kx0;
  const size_t kstride = (size_t)N * N * NH;
  for (int w = threadIdx.x; w < KT * N1; w += blockDim.x) {
    const int k1 = w / KT, c = w - k1 * KT;
    const bool live = kx0 + c < NH;
    float2 f[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) f[j2] = G[(N2 * k1 + j2) * KT + c];
    Dft<N2, -1>::run(f);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float* Kd = Kb + d * kstride + (size_t)(N2 * k1) * N * NH + c;
      float2 g[N2];
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const float k = live ? __ldg(Kd + (size_t)k2 * N * NH) : 0.f;
        g[k2] = make_float2(-f[k2].y * k, f[k2].x * k);   // i K f
      }
      Dft<N2, 1>::run(g);
#pragma unroll
      for (int j2 = 1; j2 < N2; ++j2) g[j2] = cmul(g[j2], conjf2(tw[j2 * k1]));
      float2* gd = G + (size_t)d * N * KT + c;
#pragma unroll
      for (int j2 = 0; j2 < N2; ++j2) gd[(N2 * k1 + j2) * KT] = g[j2];
    }
  }
  __syncthreads();
  // inverse step 2 of the three components -> natural z order
  for (int w = threadIdx.x; w < 3 * KT * N2; w += blockDim.x) {
    const int j2 = w / (3 * KT), q = w - j2 * 3 * KT;
    const int d = q / KT, c = q - d * KT;
    float2* base = G + (size_t)d * N * KT + c;
    float2 v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = base[(N2 * k1 + j2) * KT];
    Dft<N1, 1>::run(v);
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) base[(N2 * j1 + j2) * KT] = v[j1];
  }
  tma::fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int d = 0; d < 3; ++d)
      tma::tensor_store_3d(&spec3_map, 2 * kx0, ys, (pb * 3 + d) * a.t, G + ((size_t)d * N + a.b) * KT);
    tma::bulk_commit();
    tma::bulk_wait_all();
  }
}

template <int N> struct PassCT {
  // P [N][NP], W [N/2][N], twiddles
  static constexpr size_t smem = kTmaAlign + sizeof(float2) * ((size_t)N * spec_pitch(N) + (size_t)N / 2 * N + N);
};

#ifndef PM_SOLVE_C_MINB
#define PM_SOLVE_C_MINB 3
#endif
template <int N>
__global__ void __launch_bounds__(SolveCfg<N>::threads_c, PM_SOLVE_C_MINB) k_solve_c_tma(SolveArgs a) {
  constexpr int NP = SolveCfg<N>::NP;
  extern __shared__ unsigned char smraw_c[];
  __shared__ uint64_t bar;
  float2* P = reinterpret_cast<float2*>(tma_align(smraw_c));   // [y][NP]
  float2* W = P + N * NP;                                        // t/2 packed rows of N
  float2* tw = W + N * N / 2;
  const int zo = blockIdx.x, d = blockIdx.y, pb = blockIdx.z;
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned bytes = N * NP * (unsigned)sizeof(float2);
    tma::mbar_arrive_expect_tx(&bar, bytes);
    tma::bulk_load(P, a.spec3 + (((size_t)pb * 3 + d) * a.t + zo) * N * NP, bytes, &bar);
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  if (!block_wait(&bar, a.status)) return;
  solve_c_body<N>(a, tw, P, W);
}

// Tensor maps (encoded on the host; cuTensorMapEncodeTiled reached through
// the runtime's driver entry point, so the library links no driver library).
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3-D float32 tensor: dims d0 (innermost) .. d2, byte strides s1, s2 of dims 1 and 2, box b0 x b1 x b2.
static bool map_3d(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1, uint64_t s2,
                   uint32_t b0, uint32_t b1, uint32_t b2) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (s1 & 15) || (s2 & 15) || (b0 * 4) % 16 || b0 > 256 ||
      b1 > 256 || b2 > 256)
    return false;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {s1, s2};
  cuuint32_t box[3] = {b0, b1, b2};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---- Large periodic meshes (N > 128: the coarse mesh of the largest
// two-level runs).  A z plane of N^2 complex values no longer fits in shared
// memory, so passes A and C are each split into a row pass along x and a
// column pass along y, in place in the spectrum buffers:
//   AX  per (z, R rows): real-to-complex along x, two rows packed as one
//       complex row -> spec[z][y][kx] (natural order);
//   AY  per (z, KC columns): FFT along y -> spec[z][ky slot][kx], the layout
//       pass B reads;
//   B   the pass above, KC columns per block;
//   CY  per (component, z, KC columns): inverse FFT along y -> natural y;
//   CX  per (component, z, R rows): complex-to-real along x -> dst, with the
//       running max |a| when asked.
// The window is the whole mesh (one problem, origin 0).
template <int N> struct Large {
  static constexpr int NH = N / 2 + 1;
  static constexpr int R = 32;      // rows per block of the x passes
  static constexpr int KC = 16;     // columns per block of the y passes
  static constexpr int threads = 256;
  static constexpr int nchunk = (NH + KC - 1) / KC;
  static constexpr size_t smem_ax = sizeof(float2) * (N + (size_t)(R / 2) * N);
  static constexpr size_t smem_y = sizeof(float2) * (N + (size_t)N * KC);
  static constexpr size_t smem_cx = sizeof(float2) * (N + (size_t)R * NH + (size_t)(R / 2) * N);
};

template <int N, bool FIXED>
__global__ void __launch_bounds__(Large<N>::threads) k_large_ax(SolveArgs a) {
  constexpr int NH = Large<N>::NH, R = Large<N>::R;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* W = sm + N;   // R/2 packed rows of N
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  const int y0 = blockIdx.x * R, z = blockIdx.y;
  PM_ROWS(r, R) {
    const int64_t rowbase = ((int64_t)z * N + y0 + r) * N;
    float* w = reinterpret_cast<float*>(W + (r >> 1) * N) + (r & 1);
    if (FIXED) {
      PM_COLS(x, N) w[2 * x] = src_value<FIXED>(a.src, rowbase + x);
    } else {
      const float* srow = static_cast<const float*>(a.src) + rowbase;
      PM_COLS(x, N) async_copy4(w + 2 * x, srow + x);
    }
  }
  if (!FIXED) async_wait();
  __syncthreads();
  fft_fwd<N, R / 2, N, 1>(W, tw);
  // unpack the two real rows of each packed row (as in pass A), natural kx order
  float2* out = a.spec + ((size_t)z * N + y0) * NH;
  PM_ROWS(j, R / 2) {
    const float2* Wj = W + j * N;
    float2* o0 = out + (size_t)(2 * j) * NH;
    float2* o1 = o0 + NH;
    PM_COLS(k, NH) {
      const float2 zk = Wj[slot_of<N>(k)];
      const float2 zm = Wj[slot_of<N>(k == 0 ? 0 : N - k)];
      o0[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      o1[k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    }
  }
}

// FFT along y of KC columns of plane (blockIdx.z N + blockIdx.y) of buf
// [plane][N][NH], in place: DIR -1 natural -> slot order, +1 slot -> natural.
template <int N, int DIR>
__global__ void __launch_bounds__(Large<N>::threads) k_large_y(float2* buf, const float2* twg) {
  constexpr int NH = Large<N>::NH, KC = Large<N>::KC;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* F = sm + N;   // [y][KC]
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  const int kx0 = blockIdx.x * KC;
  const int ncol = (NH - kx0) < KC ? (NH - kx0) : KC;
  float2* pl = buf + ((size_t)blockIdx.z * N + blockIdx.y) * N * NH + kx0;
  for (int i = threadIdx.x; i < N * KC; i += blockDim.x) {
    const int y = i / KC, c = i - y * KC;
    if (c < ncol) async_copy8(F + i, pl + (size_t)y * NH + c);
    else F[i] = make_float2(0.f, 0.f);
  }
  async_wait();
  __syncthreads();
  if (DIR < 0) fft_fwd<N, KC, 1, KC>(F, tw);
  else fft_inv<N, KC, 1, KC>(F, tw);
  for (int i = threadIdx.x; i < N * KC; i += blockDim.x) {
    const int y = i / KC, c = i - y * KC;
    if (c < ncol) pl[(size_t)y * NH + c] = F[i];
  }
}

template <int N>
__global__ void __launch_bounds__(Large<N>::threads) k_large_cx(SolveArgs a) {
  constexpr int NH = Large<N>::NH, R = Large<N>::R;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* P = sm + N;          // [R][NH], natural order
  float2* W = P + R * NH;      // R/2 packed rows of N
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  const int y0 = blockIdx.x * R, z = blockIdx.y, d = blockIdx.z;
  const float2* in = a.spec3 + (((size_t)d * N + z) * N + y0) * NH;
  for (int i = threadIdx.x; i < R * NH; i += blockDim.x) async_copy8(P + i, in + i);
  async_wait();
  __syncthreads();
  PM_ROWS(j, R / 2) {
    const float2* Pa = P + (2 * j) * NH;
    const float2* Pb = Pa + NH;
    float2* Wj = W + j * N;
    PM_COLS(k, N) {
      float2 A, B;
      if (k <= N / 2) {
        A = Pa[k];
        B = Pb[k];
      } else {
        A = conjf2(Pa[N - k]);
        B = conjf2(Pb[N - k]);
      }
      Wj[slot_of<N>(k)] = make_float2(A.x - B.y, A.y + B.x);   // A + i B
    }
  }
  __syncthreads();
  fft_inv_rows<N, N>(W, R / 2, tw);
  float* dst = a.dst + (size_t)d * N * N * N + ((size_t)z * N + y0) * N;
  float m = 0.f;
  PM_ROWS(yl, R) {
    const float* w = reinterpret_cast<const float*>(W + (yl >> 1) * N) + (yl & 1);
    float* drow = dst + (size_t)yl * N;
    PM_COLS(x, N) {
      const float val = w[2 * x];
      m = fmaxf(m, fabsf(val));
      drow[x] = val;
    }
  }
  if (a.amax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > __uint_as_float(*(volatile unsigned int*)a.amax))
      atomicMax(a.amax, __float_as_uint(m));
  }
}

template <int N>
static cudaError_t solve_large_n(const SolvePlan& p, const void* src, bool fixed, float* dst, cudaStream_t st,
                                 Timer* tm, unsigned int* amax) {
  using L = Large<N>;
  if (p.nts != 1 || p.b != 0 || p.t != N || p.src_n != N) return cudaErrorInvalidValue;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_large_ax<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::smem_ax);
    cudaFuncSetAttribute(k_large_ax<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::smem_ax);
    cudaFuncSetAttribute(k_large_y<N, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::smem_y);
    cudaFuncSetAttribute(k_large_y<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::smem_y);
    cudaFuncSetAttribute(solve_b_kernel<N>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassB<N>::smem);
    cudaFuncSetAttribute(k_large_cx<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::smem_cx);
    attr_done = true;
  }
  SolveArgs a{src, fixed ? 1 : 0, N, 1, N, 0, 0, p.spec, p.spec3, p.kern, p.tw, dst, 0, amax, nullptr, 0, 1, p.status};
  {
    TimedScope ts(tm, "fft_a_mesh", st);
    if (fixed) k_large_ax<N, true><<<dim3(N / L::R, N), L::threads, L::smem_ax, st>>>(a);
    else k_large_ax<N, false><<<dim3(N / L::R, N), L::threads, L::smem_ax, st>>>(a);
    k_large_y<N, -1><<<dim3(L::nchunk, N, 1), L::threads, L::smem_y, st>>>(p.spec, p.tw);
  }
  {
    TimedScope ts(tm, "fft_b_mesh", st);
    solve_b_kernel<N>()<<<dim3(N, PassB<N>::nchunk, 1), PassB<N>::threads, PassB<N>::smem, st>>>(a);
  }
  {
    TimedScope ts(tm, "fft_c_mesh", st);
    k_large_y<N, 1><<<dim3(L::nchunk, N, 3), L::threads, L::smem_y, st>>>(p.spec3, p.tw);
    k_large_cx<N><<<dim3(N / L::R, N, 3), L::threads, L::smem_cx, st>>>(a);
  }
  note_launches(5);
  return cudaGetLastError();
}

template <int N>
__global__ void k_tile_window(const float* src, int src_n, int nts, int t, int b, int64_t tile, float* out) {
  int px = (int)(tile % nts), py = (int)((tile / nts) % nts), pz = (int)(tile / ((int64_t)nts * nts));
  int ox = px * t - b, oy = py * t - b, oz = pz * t - b;
  int64_t total = (int64_t)N * N * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((int64_t)N * N));
    int gx = pmod(ox + x, src_n), gy = pmod(oy + y, src_n), gz = pmod(oz + z, src_n);
    out[i] = src[((int64_t)gz * src_n + gy) * src_n + gx];
  }
}

template <int N>
static cudaError_t solve_n(const SolvePlan& p, const void* src, bool fixed, float* dst, cudaStream_t st, Timer* tm,
                           unsigned int* amax, const Prolong* pro) {
  using C = SolveCfg<N>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(solve_a_kernel<N, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_a);
    cudaFuncSetAttribute(solve_a_kernel<N, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_a);
    cudaFuncSetAttribute(solve_b_kernel<N>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassB<N>::smem);
    cudaFuncSetAttribute(k_solve_c<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_a);
    if constexpr (N == 96) {
      cudaFuncSetAttribute(k_solve_a_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassAT<N>::smem);
      cudaFuncSetAttribute(k_solve_b_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassBT<N>::smem);
      cudaFuncSetAttribute(k_solve_c_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassCT<N>::smem);
    }
    attr_done = true;
  }
  // 96^3 passes staged by TMA: pass A wants window origins and the source
  // mesh on 16-cell boundaries (float source), pass B its output z range on
  // an 8-row boundary; pass C always applies.
  bool tma_a = false, tma_b = false;
  CUtensorMap src_map, spec_map, spec3_map;
  if constexpr (N == 96) {
    const int n = p.src_n;
    tma_a = !fixed && n % kBox == 0 && p.t % kBox == 0 && p.b % kBox == 0 &&
            map_3d(&src_map, src, n, n, n, (uint64_t)n * 4, (uint64_t)n * n * 4, kBox, kBox, 1);
    tma_b = p.b % 8 == 0 &&
            map_3d(&spec_map, p.spec, 2 * C::NH, N, (uint64_t)p.batch * N, (uint64_t)C::NP * 8,
                   (uint64_t)N * C::NP * 8, 2 * PassBT<N>::KT, 1, N) &&
            map_3d(&spec3_map, p.spec3, 2 * C::NH, N, (uint64_t)p.batch * 3 * p.t, (uint64_t)C::NP * 8,
                   (uint64_t)N * C::NP * 8, 2 * PassBT<N>::KT, 1, p.t);
  }
  const int nprob = p.nts * p.nts * p.nts;
  for (int p0 = 0; p0 < nprob; p0 += p.batch) {
    int nb = (nprob - p0 < p.batch) ? (nprob - p0) : p.batch;
    SolveArgs a{src, fixed ? 1 : 0, p.src_n, p.nts, p.t, p.b, p0, p.spec, p.spec3, p.kern, p.tw, dst, 0, amax,
                pro ? pro->coarse : nullptr, pro ? pro->nc : 0, pro ? pro->rc : 1, p.status};
    {
      TimedScope ts(tm, N == p.src_n && p.b == 0 ? "fft_a_mesh" : "fft_a_tiles", st);
      if constexpr (N == 96) {
        if (tma_a) k_solve_a_tma<N><<<dim3(N, nb), C::threads, PassAT<N>::smem, st>>>(a, src_map);
      }
      if (!tma_a) {
        if (fixed) solve_a_kernel<N, true>()<<<dim3(N, nb), C::threads, C::smem_a, st>>>(a);
        else solve_a_kernel<N, false>()<<<dim3(N, nb), C::threads, C::smem_a, st>>>(a);
      }
    }
    {
      TimedScope ts(tm, N == p.src_n && p.b == 0 ? "fft_b_mesh" : "fft_b_tiles", st);
      if constexpr (N == 96) {
        if (tma_b)
          k_solve_b_tma<N><<<dim3(N, PassBT<N>::nchunk, nb), PassBT<N>::threads, PassBT<N>::smem, st>>>(a, spec_map,
                                                                                                       spec3_map);
      }
      if (!tma_b) solve_b_kernel<N>()<<<dim3(N, PassB<N>::nchunk, nb), PassB<N>::threads, PassB<N>::smem, st>>>(a);
    }
    if (pro && pro->ready && p0 == 0) {
      cudaError_t e = cudaStreamWaitEvent(st, pro->ready, 0);   // the coarse force must be complete
      if (e != cudaSuccess) return e;
    }
    {
      TimedScope ts(tm, N == p.src_n && p.b == 0 ? "fft_c_mesh" : "fft_c_tiles", st);
      if constexpr (N == 96) k_solve_c_tma<N><<<dim3(p.t, 3, nb), C::threads_c, PassCT<N>::smem, st>>>(a);
      else k_solve_c<N><<<dim3(p.t, 3, nb), C::threads_c, C::smem_a, st>>>(a);
    }
    note_launches(3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t solve_launch(const SolvePlan& p, const void* src, bool fixed, float* dst, cudaStream_t st, Timer* tm,
                         unsigned int* amax, const Prolong* pro) {
  if (pro && (p.t % pro->rc || (pro->rc & (pro->rc - 1)))) return cudaErrorInvalidValue;
  switch (p.N) {
    case 16: return solve_n<16>(p, src, fixed, dst, st, tm, amax, pro);
    case 32: return solve_n<32>(p, src, fixed, dst, st, tm, amax, pro);
    case 48: return solve_n<48>(p, src, fixed, dst, st, tm, amax, pro);
    case 64: return solve_n<64>(p, src, fixed, dst, st, tm, amax, pro);
    case 96: return solve_n<96>(p, src, fixed, dst, st, tm, amax, pro);
    case 128: return solve_n<128>(p, src, fixed, dst, st, tm, amax, pro);
    case 192: return pro ? cudaErrorInvalidValue : solve_large_n<192>(p, src, fixed, dst, st, tm, amax);
    case 256: return pro ? cudaErrorInvalidValue : solve_large_n<256>(p, src, fixed, dst, st, tm, amax);
    case 384: return pro ? cudaErrorInvalidValue : solve_large_n<384>(p, src, fixed, dst, st, tm, amax);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
static cudaError_t solve_adjoint_n(const SolvePlan& p, const float* lam_acc, bool interleaved, float* lam_rho,
                                   float2* spec3comp, cudaStream_t st) {
  using C = SolveCfg<N>;
  const auto ka = interleaved ? k_solve_a<N, false, 4> : solve_a_kernel<N, false>();
  cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_a);
  cudaFuncSetAttribute(k_solve_b_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float2) * (N + 2 * (size_t)N * PassB<N>::KC)));
  cudaFuncSetAttribute(k_solve_c<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_a);
  SolveArgs a{lam_acc, 0, p.src_n, 1, N, 0, 0, spec3comp, p.spec3, p.kern, p.tw, lam_rho, 1, nullptr, nullptr, 0, 1,
              p.status};
  ka<<<dim3(N, 3), C::threads, C::smem_a, st>>>(a);
  a.comp_mode = 0;
  k_solve_b_adj<N><<<dim3(N, 2, 1), PassB<N>::threads, sizeof(float2) * (N + 2 * (size_t)N * PassB<N>::KC), st>>>(a);
  k_solve_c<N><<<dim3(N, 1, 1), C::threads_c, C::smem_a, st>>>(a);
  note_launches(3);
  return cudaGetLastError();
}

cudaError_t solve_adjoint_launch(const SolvePlan& p, const float* lam_acc, bool interleaved, float* lam_rho,
                                 float2* spec3comp, cudaStream_t st) {
  if (p.nts != 1 || p.b != 0 || p.t != p.N) return cudaErrorInvalidValue;
  switch (p.N) {
    case 16: return solve_adjoint_n<16>(p, lam_acc, interleaved, lam_rho, spec3comp, st);
    case 32: return solve_adjoint_n<32>(p, lam_acc, interleaved, lam_rho, spec3comp, st);
    case 48: return solve_adjoint_n<48>(p, lam_acc, interleaved, lam_rho, spec3comp, st);
    case 64: return solve_adjoint_n<64>(p, lam_acc, interleaved, lam_rho, spec3comp, st);
    case 96: return solve_adjoint_n<96>(p, lam_acc, interleaved, lam_rho, spec3comp, st);
    case 128: return solve_adjoint_n<128>(p, lam_acc, interleaved, lam_rho, spec3comp, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tile_window_launch(const SolvePlan& p, const float* src, int64_t tile, float* out, cudaStream_t st) {
  int blocks = 256;
  switch (p.N) {
    case 16: k_tile_window<16><<<blocks, 256, 0, st>>>(src, p.src_n, p.nts, p.t, p.b, tile, out); break;
    case 32: k_tile_window<32><<<blocks, 256, 0, st>>>(src, p.src_n, p.nts, p.t, p.b, tile, out); break;
    case 48: k_tile_window<48><<<blocks, 256, 0, st>>>(src, p.src_n, p.nts, p.t, p.b, tile, out); break;
    case 64: k_tile_window<64><<<blocks, 256, 0, st>>>(src, p.src_n, p.nts, p.t, p.b, tile, out); break;
    case 96: k_tile_window<96><<<blocks, 256, 0, st>>>(src, p.src_n, p.nts, p.t, p.b, tile, out); break;
    case 128: k_tile_window<128><<<blocks, 256, 0, st>>>(src, p.src_n, p.nts, p.t, p.b, tile, out); break;
    default: return cudaErrorInvalidValue;
  }
  note_launches(1);
  return cudaGetLastError();
}

// Coarse CIC density from the fine one (exact for CIC: the coarse tent is the
// fine-node interpolation of itself): rho_c(C) = sum_k w(kx) w(ky) w(kz)
// rho_f(rc C + k), w(k) = 1 - |k| / rc, k = -(rc-1) .. rc-1, periodic.  One
// block per coarse (y, z) row: threads sum the (2 rc - 1)^2 fine rows with
// their y, z weights along x into shared memory, then the x weights.
template <int RC>   // RC > 0: compile-time ratio (loops unrolled); 0: runtime ratio rc
__global__ void __launch_bounds__(256, 1) k_restrict(const float* rho_f, int nf, int rc_rt, float* rho_c) {
  extern __shared__ float acc[];   // [nf]
  const int rc = RC > 0 ? RC : rc_rt;
  const int nc = nf / rc;
  const int cy = blockIdx.x % nc, cz = blockIdx.x / nc;
  const float inv = 1.0f / (float)rc;
  int zrow[2 * (RC > 0 ? RC : 16) - 1], yrow[2 * (RC > 0 ? RC : 16) - 1];
#pragma unroll
  for (int k = 1 - rc; k < rc; ++k) {
    int z = rc * cz + k, y = rc * cy + k;
    z += z < 0 ? nf : (z >= nf ? -nf : 0);
    y += y < 0 ? nf : (y >= nf ? -nf : 0);
    zrow[k + rc - 1] = z;
    yrow[k + rc - 1] = y;
  }
  for (int x = threadIdx.x; x < nf; x += blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int kz = 1 - rc; kz < rc; ++kz) {
      const float wz = 1.0f - (float)(kz < 0 ? -kz : kz) * inv;
      const float* zp = rho_f + (size_t)zrow[kz + rc - 1] * nf * nf + x;
#pragma unroll
      for (int ky = 1 - rc; ky < rc; ++ky) {
        const float wy = 1.0f - (float)(ky < 0 ? -ky : ky) * inv;
        s = fmaf(wz * wy, __ldg(zp + (size_t)yrow[ky + rc - 1] * nf), s);
      }
    }
    acc[x] = s;
  }
  __syncthreads();
  for (int cx = threadIdx.x; cx < nc; cx += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int kx = 1 - rc; kx < rc; ++kx) {
      int x = rc * cx + kx;
      x += x < 0 ? nf : (x >= nf ? -nf : 0);
      t = fmaf(1.0f - (float)(kx < 0 ? -kx : kx) * inv, acc[x], t);
    }
    rho_c[((size_t)cz * nc + cy) * nc + cx] = t;
  }
}

cudaError_t launch_restrict(const float* rho_f, int nf, int rc, float* rho_c, cudaStream_t st) {
  if (rc < 1 || rc > 16 || nf % rc) return cudaErrorInvalidValue;
  const int nc = nf / rc;
  if (rc == 4) k_restrict<4><<<nc * nc, 256, (size_t)nf * sizeof(float), st>>>(rho_f, nf, rc, rho_c);
  else k_restrict<0><<<nc * nc, 256, (size_t)nf * sizeof(float), st>>>(rho_f, nf, rc, rho_c);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace pm
