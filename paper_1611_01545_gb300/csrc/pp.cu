// Particle-particle force (paper Sec. 2.1, Eq. 4) on the compressed state.
//
// a_i = G sum_{j != i, same fine cell, |x_j - x_i| >= r_soft} m_j (x_j - x_i) / |x_j - x_i|^3
//
// over the particles of both species that share particle i's fine-mesh cell
// [k, k+1)^3.  The fine cells of one compression cell lie inside it, and the
// codes are ordered by compression cell, so one CTA takes one x-row of
// compression cells (PP_RX cells; both species' particles of a cell are
// contiguous ranges of their streams) and walks it in chunks of whole
// compression cells holding at most PP_CAP particles:
//   1. decode the chunk's positions into shared memory and link every
//      particle into the list of its fine cell (head per fine cell of the
//      row, next per particle; atomicExch on the head);
//   2. each particle walks its own list and sums the pairs.
// A compression cell with more than PP_CAP particles (a dense cluster) is
// done alone by the tiled all-pairs path: the particles of the cell pass
// through shared memory PP_CAP at a time and every particle of the cell
// compares fine cells with each of them.
// The result goes to a[t] (float4, w = 0) at the particle's stream index t
// (species 0 first), and the largest |a_d| of the launch to *amax (float
// bits) when amax is set.
#include <cuda_runtime.h>
#include <stdint.h>

#include "particles.cuh"
#include "pm_common.cuh"

namespace pm {

namespace {

constexpr int PP_RX = 16;        // compression cells per CTA row segment
constexpr int PP_CAP = 2048;     // particles per chunk held in shared memory
constexpr int PP_THREADS = 256;

struct PPArgs {
  PCodes c0, c1;
  const int64_t* off0;
  const int64_t* off1;
  Geo g;
  float m0, m1;
  float G, r_soft2;
  float4* acc;
  uint32_t* amax;
  int rx;                         // compression cells per CTA (divides n_cmp)
};

struct Decoded {
  float x, y, z;
  int fine;                       // fine cell index within the CTA's row segment
};

__device__ __forceinline__ Decoded decode_word(const PPArgs& a, uint32_t word, int cx, int cy, int cz, int ix0) {
  const int r = a.g.rcmp;
  const float pscale = (float)r / 256.0f;
  int q[3];
  unpack_pos(word, q);
  Decoded d;
  d.x = decode_pos(cx, q[0], pscale);
  d.y = decode_pos(cy, q[1], pscale);
  d.z = decode_pos(cz, q[2], pscale);
  // decoded positions are c r + (2q + 1) r / 512 exactly: fine offset in the cell
  const int fx = (cx - ix0) * r + (((2 * q[0] + 1) * r) >> 9);
  const int fy = ((2 * q[1] + 1) * r) >> 9;
  const int fz = ((2 * q[2] + 1) * r) >> 9;
  d.fine = (fz * r + fy) * (a.rx * r) + fx;
  return d;
}

__device__ __forceinline__ Decoded decode_one(const PPArgs& a, const PCodes& cs, int64_t p, int cx, int cy, int cz,
                                              int ix0) {
  return decode_word(a, cs.pos[p], cx, cy, cz, ix0);
}

__device__ __forceinline__ void pair_add(float xi, float yi, float zi, float xj, float yj, float zj, float mj,
                                         float r_soft2, float& ax, float& ay, float& az) {
  const float dx = xj - xi, dy = yj - yi, dz = zj - zi;
  const float r2 = dx * dx + dy * dy + dz * dz;
  if (r2 >= r_soft2 && r2 > 0.f) {
    const float inv = rsqrtf(r2);
    const float w = mj * inv * inv * inv;
    ax = fmaf(w, dx, ax);
    ay = fmaf(w, dy, ay);
    az = fmaf(w, dz, az);
  }
}

__device__ __forceinline__ void store_acc(const PPArgs& a, int64_t t, float ax, float ay, float az, float& m) {
  ax *= a.G;
  ay *= a.G;
  az *= a.G;
  a.acc[t] = make_float4(ax, ay, az, 0.f);
  m = fmaxf(m, fmaxf(fabsf(ax), fmaxf(fabsf(ay), fabsf(az))));
}

__global__ void __launch_bounds__(PP_THREADS) k_pp(PPArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int r = a.g.rcmp, n = a.g.ncmp;
  const int nseg = n / a.rx;
  const int seg = blockIdx.x % nseg, row = blockIdx.x / nseg;
  const int cy = row % n, cz = row / n, ix0 = seg * a.rx;
  float4* P = reinterpret_cast<float4*>(smraw);                 // x, y, z, m
  int* nxt = reinterpret_cast<int*>(P + PP_CAP);
  int* fin = nxt + PP_CAP;                                      // fine cell of each chunk particle
  int* head = fin + PP_CAP;                                     // [nfine]
  __shared__ int64_t r0[2][PP_RX + 1];
  for (int i = threadIdx.x; i < 2 * (a.rx + 1); i += blockDim.x) {
    const int s = i / (a.rx + 1), k = i - s * (a.rx + 1);
    const int64_t c = (int64_t)ix0 + k + (int64_t)n * (cy + (int64_t)n * cz);
    const int64_t o = (s ? a.off1 : a.off0)[c];
    const int64_t lim = s ? a.c1.n : a.c0.n;
    r0[s][k] = o < lim ? o : lim;
  }
  __syncthreads();
  float m = 0.f;
  int c0 = 0;
  while (c0 < a.rx) {
    // chunk [c0, c1): whole compression cells, at most PP_CAP particles
    int c1 = c0;
    while (c1 < a.rx) {
      const int64_t cnt = (r0[0][c1 + 1] - r0[0][c0]) + (r0[1][c1 + 1] - r0[1][c0]);
      if (cnt > PP_CAP) break;
      ++c1;
    }
    if (c1 == c0) {
      // one compression cell beyond PP_CAP: tiled all-pairs within the cell
      const int64_t b0 = r0[0][c0], e0 = r0[0][c0 + 1], b1 = r0[1][c0], e1 = r0[1][c0 + 1];
      const int64_t n0 = e0 - b0, ntot = n0 + (e1 - b1);
      for (int64_t ib = 0; ib < ntot; ib += blockDim.x) {
        const int64_t ii = ib + threadIdx.x;
        const bool live = ii < ntot;
        Decoded di{0.f, 0.f, 0.f, -1};
        if (live) di = ii < n0 ? decode_one(a, a.c0, b0 + ii, ix0 + c0, cy, cz, ix0)
                               : decode_one(a, a.c1, b1 + ii - n0, ix0 + c0, cy, cz, ix0);
        float ax = 0.f, ay = 0.f, az = 0.f;
        for (int64_t jb = 0; jb < ntot; jb += PP_CAP) {
          const int64_t jn = ntot - jb < PP_CAP ? ntot - jb : PP_CAP;
          __syncthreads();
          for (int j = threadIdx.x; j < jn; j += blockDim.x) {
            const int64_t jj = jb + j;
            const Decoded dj = jj < n0 ? decode_one(a, a.c0, b0 + jj, ix0 + c0, cy, cz, ix0)
                                       : decode_one(a, a.c1, b1 + jj - n0, ix0 + c0, cy, cz, ix0);
            P[j] = make_float4(dj.x, dj.y, dj.z, jj < n0 ? a.m0 : a.m1);
            fin[j] = dj.fine;
          }
          __syncthreads();
          if (live)
            for (int j = 0; j < jn; ++j)
              if (fin[j] == di.fine && jb + j != ii) pair_add(di.x, di.y, di.z, P[j].x, P[j].y, P[j].z, P[j].w,
                                                             a.r_soft2, ax, ay, az);
        }
        if (live) store_acc(a, ii < n0 ? b0 + ii : a.c0.n + b1 + (ii - n0), ax, ay, az, m);
      }
      __syncthreads();
      c0 += 1;
      continue;
    }
    // linked lists per fine cell of the chunk
    const int64_t b0 = r0[0][c0], e0 = r0[0][c1], b1 = r0[1][c0], e1 = r0[1][c1];
    const int n0 = (int)(e0 - b0), ntot = n0 + (int)(e1 - b1);
    const int f0 = c0 * r, f1 = c1 * r;   // fine x range of the chunk within the segment
    // reset the chunk's list heads: fine rows (z, y) of the segment, x in [f0, f1)
    for (int i = threadIdx.x; i < r * r * (f1 - f0); i += blockDim.x) {
      const int line = i / (f1 - f0), fx = f0 + (i - line * (f1 - f0));
      head[line * (a.rx * r) + fx] = -1;
    }
    __syncthreads();
    // four particles per thread: position words loaded before any is linked
    for (int i0 = threadIdx.x; i0 < ntot; i0 += 4 * blockDim.x) {
      uint32_t w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        const bool s1 = i >= n0;
        w[u] = i < ntot ? (s1 ? a.c1 : a.c0).pos[s1 ? b1 + (i - n0) : b0 + i] : 0u;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i >= ntot) break;
        const bool s1 = i >= n0;
        const int64_t p = s1 ? b1 + (i - n0) : b0 + i;
        const int64_t* ro = r0[s1 ? 1 : 0];
        // compression cell of p within [c0, c1): rows are short, scan them
        int c = c0;
        while (c + 1 < c1 && ro[c + 1] <= p) ++c;
        const Decoded d = decode_word(a, w[u], ix0 + c, cy, cz, ix0);
        P[i] = make_float4(d.x, d.y, d.z, s1 ? a.m1 : a.m0);
        fin[i] = d.fine;
        nxt[i] = atomicExch(&head[d.fine], i);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ntot; i += blockDim.x) {
      const float4 pi = P[i];
      float ax = 0.f, ay = 0.f, az = 0.f;
      for (int j = head[fin[i]]; j >= 0; j = nxt[j])
        if (j != i) pair_add(pi.x, pi.y, pi.z, P[j].x, P[j].y, P[j].z, P[j].w, a.r_soft2, ax, ay, az);
      const bool s1 = i >= n0;
      store_acc(a, s1 ? a.c0.n + b1 + (i - n0) : b0 + i, ax, ay, az, m);
    }
    __syncthreads();
    c0 = c1;
  }
  if (a.amax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > __uint_as_float(*(volatile uint32_t*)a.amax))
      atomicMax(a.amax, __float_as_uint(m));
  }
}

}  // namespace

size_t pp_smem(const Geo& g) {
  const int rx = g.ncmp < PP_RX ? g.ncmp : PP_RX;
  return (size_t)PP_CAP * (sizeof(float4) + 2 * sizeof(int)) + (size_t)rx * g.rcmp * g.rcmp * g.rcmp * sizeof(int);
}

cudaError_t launch_pp(const PCodes& c0, const PCodes& c1, const int64_t* off0, const int64_t* off1, const Geo& g,
                      float m0, float m1, float G, float r_soft, float4* acc, uint32_t* amax, cudaStream_t st) {
  if (c0.n + c1.n == 0) return cudaSuccess;
  const int rx = g.ncmp < PP_RX ? g.ncmp : PP_RX;
  if (g.ncmp % rx) return cudaErrorInvalidValue;
  PPArgs a{c0, c1, off0, off1, g, m0, m1, G, r_soft * r_soft, acc, amax, rx};
  const size_t smem = pp_smem(g);
  cudaFuncSetAttribute(k_pp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long long nblk = (long long)g.ncmp * g.ncmp * (g.ncmp / rx);
  k_pp<<<(unsigned)nblk, PP_THREADS, smem, st>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace pm
