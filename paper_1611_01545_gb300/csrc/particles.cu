// Particle-side kernels of the PM step:
//   * cell-count scans of the cell-ordered codec (Sec. 2.4): count byte with
//     the 255 escape, CSR offsets, escape-list compaction;
//   * decompress / compress of one species (Sec. 2.4);
//   * CIC deposit (Sec. 2.3 density_interpolation; Sec. 2.1 footnote: both
//     species, their own masses, one mesh), float32 or int64 fixed point;
//   * CIC force interpolation, kick and drift;
//   * the fused step passes that read the codes directly: decode + deposit
//     (binned in shared memory per block of compression cells), and decode +
//     interpolate + kick + drift + recompress (count pass, then scatter pass
//     that recomputes the same update bit for bit).
#include <cuda_runtime.h>
#include <stdint.h>

#include "particles.cuh"

namespace pm {

// ------------------------------------------------------------ scan -------

struct V2 {
  long long a;
  int b;
};
__device__ __forceinline__ V2 v2add(V2 x, V2 y) { return V2{x.a + y.a, x.b + y.b}; }

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ V2 warp_incl(V2 v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long a = __shfl_up_sync(0xffffffffu, v.a, o);
    int b = __shfl_up_sync(0xffffffffu, v.b, o);
    if (lane >= o) { v.a += a; v.b += b; }
  }
  return v;
}

// Exclusive block scan of one V2 per thread; returns the exclusive prefix and the block total.
__device__ V2 block_excl(V2 v, V2* total) {
  __shared__ V2 warp_sums[32];
  __shared__ V2 block_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  V2 inc = warp_incl(v);
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    V2 w = lane < nw ? warp_sums[lane] : V2{0, 0};
    V2 wi = warp_incl(w);
    if (lane < nw) warp_sums[lane] = V2{wi.a - w.a, wi.b - w.b};
    if (lane == nw - 1) block_total = wi;
  }
  __syncthreads();
  V2 res = v2add(warp_sums[wid], V2{inc.a - v.a, inc.b - v.b});
  *total = block_total;
  __syncthreads();
  return res;
}

// Count of compression cell c from the count byte and the escape list.
struct CodesCount {
  const uint8_t* cnt;
  const uint32_t* esc;
  const uint32_t* n_esc;
  int64_t esc_cap;
  int* status;
  __device__ V2 operator()(int64_t c) const {
    unsigned k = cnt[c];
    if (k != 255u) return V2{(long long)k, 0};
    long long ne = (long long)*n_esc;
    if (ne > esc_cap) ne = esc_cap;
    long long lo = 0, hi = ne - 1;
    while (lo <= hi) {
      long long mid = (lo + hi) >> 1;
      long long cm = esc[2 * mid];
      if (cm == c) return V2{(long long)esc[2 * mid + 1], 1};
      if (cm < c) lo = mid + 1; else hi = mid - 1;
    }
    atomicOr(status, ST_CORRUPT);
    return V2{0, 1};
  }
};

struct U32Count {
  const uint32_t* cnt;
  __device__ V2 operator()(int64_t c) const {
    unsigned k = cnt[c];
    return V2{(long long)k, k >= 255u ? 1 : 0};
  }
};

// Each scan launch serves one or two species: blockIdx.y (blockIdx.x for the
// one-block kernels) selects the species' getter / output and its partials
// (stride pstride V2 per species).
template <class T> struct Pair { T v[2]; };

template <class Get>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(Pair<Get> gets, int64_t n, V2* partial_all,
                                                            int pstride) {
  const Get& get = gets.v[blockIdx.y];
  V2* partial = partial_all + (size_t)blockIdx.y * pstride;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  V2 s{0, 0};
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
    int64_t j = base + i;
    if (j < n) s = v2add(s, get(j));
  }
  V2 tot;
  block_excl(s, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Exclusive scan of the partials in place (one block per species); partial[nb] = grand total.
__global__ void __launch_bounds__(1024) k_scan_partials(V2* partial_all, int nb, int pstride) {
  V2* partial = partial_all + (size_t)blockIdx.x * pstride;
  __shared__ V2 carry;
  if (threadIdx.x == 0) carry = V2{0, 0};
  __syncthreads();
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    V2 v = i < nb ? partial[i] : V2{0, 0};
    V2 tot;
    V2 ex = block_excl(v, &tot);
    V2 c = carry;
    if (i < nb) partial[i] = v2add(ex, c);
    __syncthreads();
    if (threadIdx.x == 0) carry = v2add(c, tot);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[nb] = carry;
}

// Decompress offsets: off[c] = sum_{c' < c} count(c'), off[n] = total; checks total == expect.
struct PutOffsets {
  int64_t* off;
  __device__ void operator()(int64_t c, V2 excl, V2) const { off[c] = excl.a; }
};

// Compress outputs: CSR offsets, count bytes, ordered escape list.
struct PutCodes {
  int64_t* off;
  uint8_t* cnt;
  uint32_t* esc;
  int64_t esc_cap;
  int* status;
  __device__ void operator()(int64_t c, V2 excl, V2 v) const {
    off[c] = excl.a;
    long long k = v.a;
    cnt[c] = (uint8_t)(k >= 255 ? 255 : k);
    if (k >= 255) {
      if ((int64_t)excl.b < esc_cap) {
        esc[2 * (int64_t)excl.b] = (uint32_t)c;
        esc[2 * (int64_t)excl.b + 1] = (uint32_t)k;
      } else {
        atomicOr(status, ST_OVERFLOW);
      }
    }
  }
};

template <class Get, class Put>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_final(Pair<Get> gets, Pair<Put> puts, int64_t n,
                                                           const V2* partial_all, int pstride) {
  const Get& get = gets.v[blockIdx.y];
  const Put& put = puts.v[blockIdx.y];
  const V2* partial = partial_all + (size_t)blockIdx.y * pstride;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  V2 v[SCAN_ITEMS];
  V2 s{0, 0};
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t j = base + k;
    v[k] = j < n ? get(j) : V2{0, 0};
    s = v2add(s, v[k]);
  }
  V2 tot;
  V2 ex = v2add(block_excl(s, &tot), partial[blockIdx.x]);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t j = base + k;
    if (j < n) put(j, ex, v[k]);
    ex = v2add(ex, v[k]);
  }
}

struct FinishArgs {
  int64_t expect;
  int64_t* off;
  uint32_t* n_esc_out;   // set for compressed outputs
  int64_t esc_cap;
};

// Writes off[n] = total, checks the total, sets n_esc if asked; thread s = species s.
__global__ void k_scan_finish(const V2* partial_all, int nb, int pstride, int64_t n, Pair<FinishArgs> fa, int nsp,
                              int* status) {
  const int s = threadIdx.x;
  if (s >= nsp) return;
  const FinishArgs& f = fa.v[s];
  V2 t = partial_all[(size_t)s * pstride + nb];
  f.off[n] = t.a;
  if (t.a != f.expect) atomicOr(status, ST_CORRUPT);
  if (f.n_esc_out) *f.n_esc_out = (uint32_t)(t.b < f.esc_cap ? t.b : f.esc_cap);
}

struct EscArgs {
  const uint8_t* cnt;
  const uint32_t* esc;
  const uint32_t* n_esc;
  int64_t esc_cap;
  const float* vmax;
};

// Every escape entry must name a cell whose byte is 255, hold >= 255, ascend; blockIdx.y = species.
__global__ void k_check_escapes(Pair<EscArgs> ea, int64_t ncell, int* status) {
  const EscArgs& e = ea.v[blockIdx.y];
  long long ne = *e.n_esc;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float vm = *e.vmax;
    if (!(vm >= 0.f) || isinf(vm)) atomicOr(status, ST_CORRUPT);
    if (ne > e.esc_cap) atomicOr(status, ST_CORRUPT);
  }
  if (ne > e.esc_cap) ne = e.esc_cap;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ne; i += (long long)gridDim.x * blockDim.x) {
    uint32_t c = e.esc[2 * i], k = e.esc[2 * i + 1];
    bool bad = (int64_t)c >= ncell || k < 255u || e.cnt[c] != 255u || (i > 0 && e.esc[2 * (i - 1)] >= c);
    if (bad) atomicOr(status, ST_CORRUPT);
  }
}

static int scan_blocks(int64_t n) { return (int)((n + SCAN_TILE - 1) / SCAN_TILE); }

// Offsets of nsp (1 or 2) species' input codes in one set of launches.
static cudaError_t scan_codes_n(const pm_codes_t* in, int nsp, int64_t ncell, int64_t* const* off, void* partial_ws,
                                int* status, cudaStream_t st) {
  V2* partial = static_cast<V2*>(partial_ws);
  const int nb = scan_blocks(ncell), ps = nb + 1;
  Pair<CodesCount> get{};
  Pair<PutOffsets> put{};
  Pair<FinishArgs> fin{};
  Pair<EscArgs> esc{};
  for (int s = 0; s < nsp; ++s) {
    get.v[s] = CodesCount{in[s].cnt, in[s].esc, in[s].n_esc, in[s].esc_cap, status};
    put.v[s] = PutOffsets{off[s]};
    fin.v[s] = FinishArgs{in[s].n, off[s], nullptr, 0};
    esc.v[s] = EscArgs{in[s].cnt, in[s].esc, in[s].n_esc, in[s].esc_cap, in[s].vmax};
  }
  k_check_escapes<<<dim3(64, nsp), 256, 0, st>>>(esc, ncell, status);
  k_scan_reduce<<<dim3(nb, nsp), SCAN_THREADS, 0, st>>>(get, ncell, partial, ps);
  k_scan_partials<<<nsp, 1024, 0, st>>>(partial, nb, ps);
  k_scan_final<<<dim3(nb, nsp), SCAN_THREADS, 0, st>>>(get, put, ncell, partial, ps);
  k_scan_finish<<<1, 32, 0, st>>>(partial, nb, ps, ncell, fin, nsp, status);
  note_launches(5);
  return cudaGetLastError();
}

cudaError_t scan_codes(const pm_codes_t& in, int64_t ncell, int64_t* off, void* partial_ws, int* status,
                       cudaStream_t st) {
  int64_t* offs[1] = {off};
  return scan_codes_n(&in, 1, ncell, offs, partial_ws, status, st);
}

cudaError_t scan_codes2(const pm_codes_t in[2], int64_t ncell, int64_t* off0, int64_t* off1, void* partial_ws,
                        int* status, cudaStream_t st) {
  int64_t* offs[2] = {off0, off1};
  return scan_codes_n(in, 2, ncell, offs, partial_ws, status, st);
}

static cudaError_t scan_counts_n(const uint32_t* const* counts, int nsp, int64_t ncell, const int64_t* expect,
                                 int64_t* const* off, pm_codes_t* out, void* partial_ws, int* status,
                                 cudaStream_t st) {
  V2* partial = static_cast<V2*>(partial_ws);
  const int nb = scan_blocks(ncell), ps = nb + 1;
  Pair<U32Count> get{};
  Pair<PutCodes> put{};
  Pair<FinishArgs> fin{};
  for (int s = 0; s < nsp; ++s) {
    get.v[s] = U32Count{counts[s]};
    put.v[s] = PutCodes{off[s], out[s].cnt, out[s].esc, out[s].esc_cap, status};
    fin.v[s] = FinishArgs{expect[s], off[s], out[s].n_esc, out[s].esc_cap};
  }
  k_scan_reduce<<<dim3(nb, nsp), SCAN_THREADS, 0, st>>>(get, ncell, partial, ps);
  k_scan_partials<<<nsp, 1024, 0, st>>>(partial, nb, ps);
  k_scan_final<<<dim3(nb, nsp), SCAN_THREADS, 0, st>>>(get, put, ncell, partial, ps);
  k_scan_finish<<<1, 32, 0, st>>>(partial, nb, ps, ncell, fin, nsp, status);
  note_launches(4);
  return cudaGetLastError();
}

cudaError_t scan_counts(const uint32_t* counts, int64_t ncell, int64_t expect, int64_t* off, pm_codes_t& out,
                        void* partial_ws, int* status, cudaStream_t st) {
  const uint32_t* c[1] = {counts};
  int64_t* o[1] = {off};
  return scan_counts_n(c, 1, ncell, &expect, o, &out, partial_ws, status, st);
}

cudaError_t scan_counts2(const uint32_t* counts0, const uint32_t* counts1, int64_t ncell, const int64_t expect[2],
                         int64_t* off0, int64_t* off1, pm_codes_t out[2], void* partial_ws, int* status,
                         cudaStream_t st) {
  const uint32_t* c[2] = {counts0, counts1};
  int64_t* o[2] = {off0, off1};
  return scan_counts_n(c, 2, ncell, expect, o, out, partial_ws, status, st);
}

// Partials of one species; the two-species scans use twice this.
size_t scan_partial_bytes(int64_t ncell) { return sizeof(V2) * (size_t)(scan_blocks(ncell) + 1); }

// ------------------------------------------------- plain per-particle -----

// Cell of stream index p: the last c with off[c] <= p (binary search over all cells).
__device__ __forceinline__ int64_t find_cell(const int64_t* off, int64_t ncell, int64_t p) {
  int64_t lo = 0, hi = ncell - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_decompress(PCodes in, const int64_t* off, Geo g, float* x, float* v) {
  const float pscale = (float)g.rcmp / 256.0f;
  const float vm = *in.vmax;
  const int half = in.vel16 ? 32768 : 128;
  const float step = __fmul_rn(vm, 1.0f / (float)half);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < in.n; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = find_cell(off, g.ncell, p);
    int cx = (int)(c % g.ncmp), cy = (int)((c / g.ncmp) % g.ncmp), cz = (int)(c / ((int64_t)g.ncmp * g.ncmp));
    int q[3], qv[3];
    unpack_pos(in.pos[p], q);
    load_vel(in.vel, in.vel16, p, qv);
    x[3 * p + 0] = decode_pos(cx, q[0], pscale);
    x[3 * p + 1] = decode_pos(cy, q[1], pscale);
    x[3 * p + 2] = decode_pos(cz, q[2], pscale);
#pragma unroll
    for (int d = 0; d < 3; ++d) v[3 * p + d] = decode_vel(qv[d], half, step);
  }
}

// Float32 CIC deposit into global meshes with atomics.
__device__ __forceinline__ void cic_axis(float x, int n, int& i0, int& i1, float& w0, float& w1) {
  float f = floorf(x);
  w1 = __fsub_rn(x, f);
  w0 = __fsub_rn(1.0f, w1);
  i0 = (int)f;
  if (i0 >= n) i0 -= n;
  if (i0 < 0) i0 += n;
  i1 = (i0 + 1 == n) ? 0 : i0 + 1;
}

__global__ void k_deposit_global(const float* x, int64_t n, float m, Geo g, float* rho_c, float* rho_f) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float px = x[3 * p], py = x[3 * p + 1], pz = x[3 * p + 2];
    int ix[2], iy[2], iz[2];
    float wx[2], wy[2], wz[2];
    cic_axis(px, g.nf, ix[0], ix[1], wx[0], wx[1]);
    cic_axis(py, g.nf, iy[0], iy[1], wy[0], wy[1]);
    cic_axis(pz, g.nf, iz[0], iz[1], wz[0], wz[1]);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
      float w = __fmul_rn(__fmul_rn(wx[dx], wy[dy]), wz[dz]);
      atomicAdd(&rho_f[((int64_t)iz[dz] * g.nf + iy[dy]) * g.nf + ix[dx]], __fmul_rn(m, w));
    }
    if (rho_c) {
      float s = 1.0f / (float)g.rc;
      cic_axis(__fmul_rn(px, s), g.nc, ix[0], ix[1], wx[0], wx[1]);
      cic_axis(__fmul_rn(py, s), g.nc, iy[0], iy[1], wy[0], wy[1]);
      cic_axis(__fmul_rn(pz, s), g.nc, iz[0], iz[1], wz[0], wz[1]);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        float w = __fmul_rn(__fmul_rn(wx[dx], wy[dy]), wz[dz]);
        atomicAdd(&rho_c[((int64_t)iz[dz] * g.nc + iy[dy]) * g.nc + ix[dx]], __fmul_rn(m, w));
      }
    }
  }
}

// Periodic CIC deposit of nw per-particle weights (w[p nw + c], c < nw <= 4)
// onto nw fine meshes out[c][nf^3] (float32, the mesh convention of the
// deposit above): number and momentum densities for the power spectra of
// the compression study.
__global__ void k_deposit_weights(const float* x, int64_t n, const float* w, int nw, Geo g, float* out) {
  const int64_t nf3 = (int64_t)g.nf * g.nf * g.nf;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int ix[2], iy[2], iz[2];
    float wx[2], wy[2], wz[2];
    cic_axis(x[3 * p], g.nf, ix[0], ix[1], wx[0], wx[1]);
    cic_axis(x[3 * p + 1], g.nf, iy[0], iy[1], wy[0], wy[1]);
    cic_axis(x[3 * p + 2], g.nf, iz[0], iz[1], wz[0], wz[1]);
    float q[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c = 0; c < nw; ++c) q[c] = w[p * nw + c];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
      const float wt = __fmul_rn(__fmul_rn(wx[dx], wy[dy]), wz[dz]);
      float* cell = out + ((int64_t)iz[dz] * g.nf + iy[dy]) * g.nf + ix[dx];
      for (int c = 0; c < nw; ++c) atomicAdd(cell + c * nf3, __fmul_rn(q[c], wt));
    }
  }
}

// Fixed point: weights a1 = floor(f 2^20), mass split hi = (M a1 + 2^19) >> 20, lo = M - hi.
__device__ __forceinline__ void fixed_axis(float x, int n, int& i0, int& i1, long long& a1) {
  float f = floorf(x);
  float fr = __fsub_rn(x, f);
  a1 = (long long)__fmul_rn(fr, 1048576.0f);
  i0 = (int)f;
  if (i0 >= n) i0 -= n;
  if (i0 < 0) i0 += n;
  i1 = (i0 + 1 == n) ? 0 : i0 + 1;
}
__device__ __forceinline__ void fixed_split(long long M, long long a1, long long& lo, long long& hi) {
  hi = (M * a1 + (1LL << 19)) >> 20;
  lo = M - hi;
}
__device__ __forceinline__ void fixed_corners(long long M, const long long a[3], long long out[8]) {
  long long mx[2], my[2], mz[2];
  fixed_split(M, a[0], mx[0], mx[1]);
#pragma unroll
  for (int dx = 0; dx < 2; ++dx) {
    fixed_split(mx[dx], a[1], my[0], my[1]);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      fixed_split(my[dy], a[2], mz[0], mz[1]);
      out[dx + 2 * dy + 0] = mz[0];
      out[dx + 2 * dy + 4] = mz[1];
    }
  }
}

__global__ void k_deposit_fixed_global(const float* x, int64_t n, long long M, Geo g, long long* rho_c,
                                       long long* rho_f) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float pp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
    for (int level = 0; level < 2; ++level) {
      long long* rho = level == 0 ? rho_f : rho_c;
      if (!rho) continue;
      int nn = level == 0 ? g.nf : g.nc;
      float s = level == 0 ? 1.0f : 1.0f / (float)g.rc;
      int i0[3], i1[3];
      long long a1[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) fixed_axis(__fmul_rn(pp[d], s), nn, i0[d], i1[d], a1[d]);
      long long terms[8];
      fixed_corners(M, a1, terms);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        int gx = dx ? i1[0] : i0[0], gy = dy ? i1[1] : i0[1], gz = dz ? i1[2] : i0[2];
        atomicAdd(reinterpret_cast<unsigned long long*>(&rho[((int64_t)gz * nn + gy) * nn + gx]),
                  (unsigned long long)terms[c]);
      }
    }
  }
}

// CIC gather of a [3][n^3] field; fixed operation order so recomputation is bit-identical.
__device__ __forceinline__ void gather(const float* __restrict__ F, int n, float px, float py, float pz, float a[3]) {
  int ix[2], iy[2], iz[2];
  float wx[2], wy[2], wz[2];
  cic_axis(px, n, ix[0], ix[1], wx[0], wx[1]);
  cic_axis(py, n, iy[0], iy[1], wy[0], wy[1]);
  cic_axis(pz, n, iz[0], iz[1], wz[0], wz[1]);
  const int64_t n3 = (int64_t)n * n * n;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    float w = __fmul_rn(__fmul_rn(wx[dx], wy[dy]), wz[dz]);
    int64_t idx = ((int64_t)iz[dz] * n + iy[dy]) * n + ix[dx];
    s0 = __fmaf_rn(w, __ldg(F + idx), s0);
    s1 = __fmaf_rn(w, __ldg(F + n3 + idx), s1);
    s2 = __fmaf_rn(w, __ldg(F + 2 * n3 + idx), s2);
  }
  a[0] = s0;
  a[1] = s1;
  a[2] = s2;
}

__device__ __forceinline__ void accel_at(const Geo& g, const float* acc_c, const float* acc_f, float px, float py,
                                         float pz, float a[3]) {
  gather(acc_f, g.nf, px, py, pz, a);
  if (g.two) {
    float s = 1.0f / (float)g.rc;
    float b[3];
    gather(acc_c, g.nc, __fmul_rn(px, s), __fmul_rn(py, s), __fmul_rn(pz, s), b);
    a[0] = __fadd_rn(b[0], a[0]);
    a[1] = __fadd_rn(b[1], a[1]);
    a[2] = __fadd_rn(b[2], a[2]);
  }
}

// The same CIC gather from a shared-memory copy S[3][fz][fy][fx] of the mesh
// region whose cell (0,0,0) is the global cell (ox, oy, oz); identical
// arithmetic and order to gather(), so both give the same bits.
__device__ __forceinline__ void gather_local(const float* S, int fx, int fy, int fz, int ox, int oy, int oz, float px,
                                             float py, float pz, float a[3]) {
  float fl[3] = {floorf(px), floorf(py), floorf(pz)};
  float w1[3] = {__fsub_rn(px, fl[0]), __fsub_rn(py, fl[1]), __fsub_rn(pz, fl[2])};
  float w0[3] = {__fsub_rn(1.0f, w1[0]), __fsub_rn(1.0f, w1[1]), __fsub_rn(1.0f, w1[2])};
  const int lx = (int)fl[0] - ox, ly = (int)fl[1] - oy, lz = (int)fl[2] - oz;
  const int plane = fx * fy * fz;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    float w = __fmul_rn(__fmul_rn(dx ? w1[0] : w0[0], dy ? w1[1] : w0[1]), dz ? w1[2] : w0[2]);
    int idx = ((lz + dz) * fy + (ly + dy)) * fx + (lx + dx);
    s0 = __fmaf_rn(w, S[idx], s0);
    s1 = __fmaf_rn(w, S[plane + idx], s1);
    s2 = __fmaf_rn(w, S[2 * plane + idx], s2);
  }
  a[0] = s0;
  a[1] = s1;
  a[2] = s2;
}

// The same CIC gather when the lower corner's local index (lx, ly, lz) and the
// upper weights w1 are already known; same weights and order as gather().
__device__ __forceinline__ void gather_idx(const float* S, int fx, int fy, int fz, int lx, int ly, int lz,
                                           const float w1[3], float a[3]) {
  const float w0[3] = {__fsub_rn(1.0f, w1[0]), __fsub_rn(1.0f, w1[1]), __fsub_rn(1.0f, w1[2])};
  const int plane = fx * fy * fz;
  const float* base = S + (lz * fy + ly) * fx + lx;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    const float w = __fmul_rn(__fmul_rn(dx ? w1[0] : w0[0], dy ? w1[1] : w0[1]), dz ? w1[2] : w0[2]);
    const float* q = base + (dz * fy + dy) * fx + dx;
    s0 = __fmaf_rn(w, q[0], s0);
    s1 = __fmaf_rn(w, q[plane], s1);
    s2 = __fmaf_rn(w, q[2 * plane], s2);
  }
  a[0] = s0;
  a[1] = s1;
  a[2] = s2;
}

// Strides of a staged force region (fx x fy x fz nodes, 3 components) in
// shared memory: rows padded to 4 and planes to 16 banks modulo 32, so that
// the nodes around the particles of one compression cell, which the lanes of
// a warp gather at the same time, fall in different banks.
struct RegionStrides {
  int row, plane, comp;
};
#ifndef PM_IKD_PAD
#define PM_IKD_PAD 1
#endif
__host__ __device__ __forceinline__ RegionStrides region_strides(int fx, int fy, int fz) {
  RegionStrides st;
  st.row = PM_IKD_PAD ? fx + ((4 - fx) & 31) : fx;
  const int p0 = st.row * fy;
  st.plane = PM_IKD_PAD ? p0 + ((16 - p0) & 31) : p0;
  st.comp = st.plane * fz;
  return st;
}

// gather_idx on a region with the strides above; same weights and order.
__device__ __forceinline__ void gather_strided(const float* S, RegionStrides st, int lx, int ly, int lz,
                                               const float w1[3], float a[3]) {
  const float w0[3] = {__fsub_rn(1.0f, w1[0]), __fsub_rn(1.0f, w1[1]), __fsub_rn(1.0f, w1[2])};
  const float* base = S + lz * st.plane + ly * st.row + lx;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    const float w = __fmul_rn(__fmul_rn(dx ? w1[0] : w0[0], dy ? w1[1] : w0[1]), dz ? w1[2] : w0[2]);
    const float* q = base + dz * st.plane + dy * st.row + dx;
    s0 = __fmaf_rn(w, q[0], s0);
    s1 = __fmaf_rn(w, q[st.comp], s1);
    s2 = __fmaf_rn(w, q[2 * st.comp], s2);
  }
  a[0] = s0;
  a[1] = s1;
  a[2] = s2;
}

__device__ __forceinline__ float wrap_pos(float x, float nf) {
  if (x < 0.f) x = __fadd_rn(x, nf);
  if (x >= nf) x = __fsub_rn(x, nf);
  if (!(x >= 0.f && x < nf)) {      // moved more than one box length, or rounding onto nf
    x = __fsub_rn(x, __fmul_rn(nf, floorf(__fdiv_rn(x, nf))));
    if (!(x >= 0.f && x < nf)) x = 0.f;
  }
  return x;
}

// v' = v + c_k a ; x' = wrap(x + c_d v')
__device__ __forceinline__ void kick_drift(float x[3], float v[3], const float a[3], float ck, float cd, float nf) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    v[d] = __fmaf_rn(ck, a[d], v[d]);
    x[d] = wrap_pos(__fmaf_rn(cd, v[d], x[d]), nf);
  }
}

__global__ void k_interpolate(const float* x, int64_t n, Geo g, const float* acc_c, const float* acc_f, float* a) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float r[3];
    accel_at(g, acc_c, acc_f, x[3 * p], x[3 * p + 1], x[3 * p + 2], r);
    a[3 * p] = r[0];
    a[3 * p + 1] = r[1];
    a[3 * p + 2] = r[2];
  }
}

__global__ void k_kick_drift(float* x, float* v, int64_t n, Geo g, const float* acc_c, const float* acc_f, float ck,
                             float cd) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float xx[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
    float vv[3] = {v[3 * p], v[3 * p + 1], v[3 * p + 2]};
    float a[3];
    accel_at(g, acc_c, acc_f, xx[0], xx[1], xx[2], a);
    kick_drift(xx, vv, a, ck, cd, (float)g.nf);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      x[3 * p + d] = xx[d];
      v[3 * p + d] = vv[d];
    }
  }
}

// ------------------------------------------------ recompress passes ------

// Warp-aggregated count / rank of a cell key; key 0xffffffff = inactive lane.
__device__ __forceinline__ void count_cell(uint32_t* counts, uint32_t key) {
  unsigned peers = __match_any_sync(0xffffffffu, key);
  int leader = __ffs(peers) - 1;
  if (key != 0xffffffffu && (threadIdx.x & 31) == leader) atomicAdd(counts + key, (unsigned)__popc(peers));
}
__device__ __forceinline__ uint32_t take_rank(uint32_t* counts, uint32_t key) {
  unsigned peers = __match_any_sync(0xffffffffu, key);
  int lane = threadIdx.x & 31;
  int leader = __ffs(peers) - 1;
  unsigned old = 0;
  if (key != 0xffffffffu && lane == leader) old = atomicSub(counts + key, (unsigned)__popc(peers));
  old = __shfl_sync(0xffffffffu, old, leader);
  unsigned below = __popc(peers & ((1u << lane) - 1u));
  return old - (unsigned)__popc(peers) + below;
}

// Block maximum of values m >= 0, returned to every thread.  Every thread of
// the block must call it.
__device__ __forceinline__ float block_max_all(float m) {
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();   // red may still be read by a previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  float r = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
  return r;
}

// Block maximum of m into *vmax_bits (float bits of a value >= 0): one atomic
// per block, and none when the block's maximum does not exceed the current
// value.  Every thread of the block must call it.
__device__ __forceinline__ void block_vmax(float m, uint32_t* vmax_bits) {
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();   // red may still be read by a previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    if (m > 0.f && m > __uint_as_float(*(volatile uint32_t*)vmax_bits)) atomicMax(vmax_bits, __float_as_uint(m));
  }
}

__device__ __forceinline__ void write_codes(PCodesOut o, int64_t dst, const float x[3], const float v[3], float inv_r,
                                            int ncmp, float s, bool vzero) {
  const int half = o.vel16 ? 32768 : 128;
  int q[3], qv[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int c;
    encode_pos(x[d], inv_r, ncmp, c, q[d]);
    qv[d] = encode_vel(v[d], s, half, vzero);
  }
  o.pos[dst] = (uint32_t)q[0] | ((uint32_t)q[1] << 8) | ((uint32_t)q[2] << 16);
  store_vel(o.vel, o.vel16, dst, qv);
}

__device__ __forceinline__ uint32_t cell_key(const float x[3], float inv_r, int ncmp) {
  int c[3], q;
#pragma unroll
  for (int d = 0; d < 3; ++d) encode_pos(x[d], inv_r, ncmp, c[d], q);
  return (uint32_t)(c[0] + ncmp * (c[1] + ncmp * c[2]));
}

// pm_compress passes over float input.  MODE 0: count cells (+ v_max); MODE 1: scatter codes.
template <int MODE>
__global__ void k_compress_pass(const float* x, const float* v, int64_t n, Geo g, uint32_t* counts,
                                uint32_t* vmax_bits, const float* vmax_in, const int64_t* off, PCodesOut o,
                                int* status) {
  const float inv_r = 1.0f / (float)g.rcmp;
  const float nf = (float)g.nf;
  float vm = 0.f, s = 0.f;
  bool vzero = false;
  if (MODE == 1) {
    vm = *o.vmax;
    vzero = !(vm > 0.f);
    s = vzero ? 0.f : __fdiv_rn(o.vel16 ? 32768.0f : 128.0f, vm);
  }
  float local_max = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nround = ((n + stride - 1) / stride) * stride;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nround; p += stride) {
    uint32_t key = 0xffffffffu;
    float xx[3], vv[3];
    if (p < n) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        xx[d] = x[3 * p + d];
        vv[d] = v[3 * p + d];
        local_max = fmaxf(local_max, fabsf(vv[d]));
      }
      bool ok = xx[0] >= 0.f && xx[0] < nf && xx[1] >= 0.f && xx[1] < nf && xx[2] >= 0.f && xx[2] < nf;
      if (ok) key = cell_key(xx, inv_r, g.ncmp);
      else if (MODE == 0) atomicOr(status, ST_RANGE);
    }
    if (MODE == 0) {
      count_cell(counts, key);
    } else {
      uint32_t r = take_rank(counts, key);
      if (key != 0xffffffffu) {
        int64_t dst = off[key] + r;
        if (dst < n && r < 0x80000000u) write_codes(o, dst, xx, vv, inv_r, g.ncmp, s, vzero);
        else atomicOr(status, ST_CORRUPT);
      }
    }
  }
  if (MODE == 0 && vmax_in == nullptr) block_vmax(local_max, vmax_bits);
}

__global__ void k_set_vmax(const uint32_t* vmax_bits, const float* vmax_in, float* out) {
  *out = vmax_in ? *vmax_in : __uint_as_float(*vmax_bits);
}

// Bound on |v'_d| = |v_d + c_k a_d(x)| before the kick: decoded |v_d| < v_max
// (bin centres) and a CIC-interpolated component never exceeds the largest
// mesh value, so v_max' = v_max + |c_k| (max|a_coarse| + max|a_fine|); every
// operation rounds up, so the float result is not below the exact bound.
__global__ void k_vmax_bound(const float* vin0, const float* vin1, const uint32_t* amax, float ck, float* vout0,
                             float* vout1) {
  const float a = __fadd_ru(__fadd_ru(__uint_as_float(amax[0]), __uint_as_float(amax[1])), __uint_as_float(amax[2]));
  const float ka = __fmul_ru(fabsf(ck), a);
  *vout0 = __fadd_ru(*vin0, ka);
  *vout1 = __fadd_ru(*vin1, ka);
}

// --------------------------------------------- fused passes over codes ----

// Block of compression cells handled by one CTA: x cells [bx*RX, +RX), rows y [by*RY, +RY), z [bz*RZ, +RZ).
struct CellBlock {
  int ix0, iy0, iz0;
};
// Blocks are handed out x fastest, then in bricks of bk.brick x bk.brick
// (y, z) block rows (the host picks bricks for large meshes, see
// block_brick), so that the blocks running at the same time cover a compact
// region: the partial writes that neighbouring blocks make to the same
// cells (new-cell ranges of the recompressed codes, fine density halos)
// then meet in L2 before the lines are evicted.
__device__ __forceinline__ CellBlock block_of(const Blk& bk, int bid) {
  const int nbx = bk.nbx, nby = bk.nby;
  const int bx = bid % nbx, r = bid / nbx;
  int by, bz;
  const int B = bk.brick;
  if (B > 1) {
    const int in = r % (B * B), brick = r / (B * B);
    const int nyb = nby / B;
    by = (brick % nyb) * B + in % B;
    bz = (brick / nyb) * B + in / B;
  } else {
    by = r % nby;
    bz = r / nby;
  }
  return CellBlock{bx * bk.RX, by * bk.RY, bz * bk.RZ};
}

// Runs body(bid) for the cell blocks of this CTA: its own block (one CTA per
// cell block), or, when bk.work is set (persistent launch), blocks drawn one
// at a time from the device counter *bk.work until all are taken, so that
// CTAs that drew light blocks take more of them.  body must use __syncthreads
// uniformly; the barrier before each draw keeps the next block's shared-memory
// set-up from overlapping the previous block's flush.
template <class F>
__device__ __forceinline__ void for_each_block(const Blk& bk, F&& body) {
  if (!bk.work) {
    body((int)blockIdx.x);
    return;
  }
  __shared__ int s_bid;
  const int nblk = bk.nbx * bk.nby * bk.nbz;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_bid = atomicAdd(bk.work, 1);
    __syncthreads();
    const int bid = s_bid;
    if (bid >= nblk) break;
    body(bid);
  }
}

// Loads the CSR offsets of the block's rows into smem: roff[r*(RX+1) + i], r = row (y fastest).
__device__ __forceinline__ void load_row_offsets(const int64_t* off, const Geo& g, const Blk& bk, CellBlock cb,
                                                 int64_t* roff) {
  const int nrow = bk.RY * bk.RZ;
  for (int i = threadIdx.x; i < nrow * (bk.RX + 1); i += blockDim.x) {
    int r = i / (bk.RX + 1), k = i - r * (bk.RX + 1);
    int iy = cb.iy0 + r % bk.RY, iz = cb.iz0 + r / bk.RY;
    int64_t c = (int64_t)cb.ix0 + k + (int64_t)g.ncmp * (iy + (int64_t)g.ncmp * iz);
    roff[i] = off[c];
  }
}

// Index (0..RX-1) of the cell of stream index p within a row's offsets ro[0..RX].
__device__ __forceinline__ int row_cell(const int64_t* ro, int RX, int64_t p) {
  int lo = 0, hi = RX - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (ro[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// 4-byte global -> shared copy that does not stall the issuing thread
// (cp.async); async_copies_wait() waits for all of the thread's copies.
__device__ __forceinline__ void copy_async4(float* smem_dst, const float* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void async_copies_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void smem_acc(long long* a, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(a), (unsigned long long)v);
}
__device__ __forceinline__ void smem_acc(float* a, float v) { atomicAdd(a, v); }
__device__ __forceinline__ void global_add(float* a, float v) { atomicAdd(a, v); }
__device__ __forceinline__ void global_add(long long* a, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(a), (unsigned long long)v);
}

// Sums v[] over runs of consecutive lanes holding the same key (the particle
// stream is cell ordered, so a warp's particles form few runs); returns true
// on the last lane of each run, which then holds the run's totals.
template <int K, typename T>
__device__ __forceinline__ bool run_reduce(unsigned key, T (&v)[K]) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned prev = __shfl_up_sync(FULL, key, 1);
  const unsigned next = __shfl_down_sync(FULL, key, 1);
  const bool head = lane == 0 || prev != key;
  const bool tail = lane == 31 || next != key;
  const unsigned heads = __ballot_sync(FULL, head);
  const int start = 31 - __clz(heads & (FULL >> (31 - lane)));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      T u = __shfl_up_sync(FULL, v[k], o);
      if (lane - start >= o) v[k] += u;
    }
  }
  return tail;
}

// Compile-time cell-block shape: RX_ > 0 fixes RX, RY, RZ and the fine cells per
// compression cell (the shapes the autotuner picks on the benchmark meshes), so
// the staged region's strides and the row search are constants; 0 reads them
// from the arguments.
#ifndef PM_SHAPE_INSTANCES
#define PM_SHAPE_INSTANCES 1
#endif
template <int RX_, int RY_, int RZ_, int R_>
__device__ __forceinline__ void fix_shape(Geo& g, Blk& bk) {
  if (RX_ > 0) {
    bk.RX = RX_;
    bk.RY = RY_;
    bk.RZ = RZ_;
    g.rcmp = R_;
  }
}

// Mass of each CIC corner: float mode m w_x w_y w_z in float32; fixed mode
// the conservative integer split of the fixed-point deposit (2^-32 units).
__device__ __forceinline__ void corner_masses(float m, long long, const float w1[3], float out[8]) {
  float w0[3] = {__fsub_rn(1.f, w1[0]), __fsub_rn(1.f, w1[1]), __fsub_rn(1.f, w1[2])};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    float w = __fmul_rn(__fmul_rn(dx ? w1[0] : w0[0], dy ? w1[1] : w0[1]), dz ? w1[2] : w0[2]);
    out[c] = __fmul_rn(m, w);
  }
}
__device__ __forceinline__ void corner_masses(float, long long M, const float w1[3], long long out[8]) {
  long long a1[3] = {(long long)__fmul_rn(w1[0], 1048576.0f), (long long)__fmul_rn(w1[1], 1048576.0f),
                     (long long)__fmul_rn(w1[2], 1048576.0f)};
  fixed_corners(M, a1, out);
}

// Decode + deposit of both species for one cell block, binned in shared memory
// (32-bit fixed point with a per-block power-of-two scale, converted to
// float32 before the flush; or int64 in units of 2^-32 mass for the
// fixed-point mode) and flushed once per cell.  smem: row offsets (2 species), fine region
// (RX r + 1)(RY r + 1)(RZ r + 1), coarse region (RX + 1)(RY + 1)(RZ + 1).
// Threads per CTA of the deposit.
#ifndef PM_DEPOSIT_THREADS
#define PM_DEPOSIT_THREADS 256
#endif

// Register budget of the deposit: resident CTAs per SM it is compiled for
// (6: 40 registers; measured 0.391 -> 0.347 ms against the compiler's own
// allocation on the 256^3 workload; the int64 mode keeps 4).  0 keeps the
// compiler's allocation.
#ifndef PM_DEPOSIT_MINB
#define PM_DEPOSIT_MINB 6
#endif
#if PM_DEPOSIT_MINB > 0
#define PM_DEPOSIT_BOUNDS __launch_bounds__(PM_DEPOSIT_THREADS, sizeof(Acc) == 4 ? PM_DEPOSIT_MINB : 4)
#else
#define PM_DEPOSIT_BOUNDS
#endif
template <typename Acc, int RX_, int RY_, int RZ_, int R_>
__global__ void PM_DEPOSIT_BOUNDS k_deposit_codes(PCodes c0, PCodes c1, const int64_t* off0, const int64_t* off1, Geo g_arg, Blk bk_arg,
                                float m0, float m1, long long M0, long long M1, Acc* rho_c, Acc* rho_f) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Geo g = g_arg;
  Blk bk = bk_arg;
  fix_shape<RX_, RY_, RZ_, R_>(g, bk);
  for_each_block(bk, [&](const int bid) {
    const int r = g.rcmp;
    const int fx = bk.RX * r + 1, fy = bk.RY * r + 1, fz = bk.RZ * r + 1;
    const int cx = bk.RX + 1, cy = bk.RY + 1, cz = bk.RZ + 1;
    const int nrow = bk.RY * bk.RZ;
    int64_t* roff = reinterpret_cast<int64_t*>(smraw);
    Acc* sf = reinterpret_cast<Acc*>(roff + 2 * nrow * (bk.RX + 1));
    Acc* sc = sf + fx * fy * fz;
    // Coarse density: the int64 mode deposits each particle's 8 coarse corners
    // (exact, order independent); the float mode restricts the block's fine
    // tile onto the coarse cells it touches when it flushes (CIC restriction
    // is exact and linear, so the blocks' partial sums add up to it).
    const bool dep_coarse = g.two && rho_c != nullptr && sizeof(Acc) == 8;
    const bool restr = g.two && rho_c != nullptr && sizeof(Acc) == 4;
    const int nsf = fx * fy * fz, nsc = dep_coarse ? cx * cy * cz : 0;
    for (int i = threadIdx.x; i < nsf + nsc; i += blockDim.x) sf[i] = (Acc)0;
    const CellBlock cb = block_of(bk, bid);
    load_row_offsets(off0, g, bk, cb, roff);
    load_row_offsets(off1, g, bk, cb, roff + nrow * (bk.RX + 1));
    __syncthreads();
    // Float mode: the block bins its corner masses in 32-bit fixed point
    // (integer shared-memory atomics, several times the rate of float ones,
    // and independent of the order of the adds) with a power-of-two scale S.
    // A fine node receives mass only from particles of the (at most 8)
    // compression cells around it, so 8 x the block's heaviest compression
    // cell bounds every node's total; S = 2^floor(log2(2^31 / bound)) keeps
    // the scaled total below 2^31, and the corner roundings below 2^31 more.
    float S = 1.f;
    if constexpr (sizeof(Acc) == 4) {
      float cm = 0.f;
      const int nrx = bk.RX + 1, ncells = nrow * bk.RX;
      for (int i = threadIdx.x; i < ncells; i += blockDim.x) {
        const int row = i / bk.RX, k = i - row * bk.RX;
        const int64_t* r0 = roff + row * nrx + k;
        const int64_t* r1 = r0 + nrow * nrx;
        const int64_t a0 = r0[0] < c0.n ? r0[0] : c0.n, b0 = r0[1] < c0.n ? r0[1] : c0.n;
        const int64_t a1 = r1[0] < c1.n ? r1[0] : c1.n, b1 = r1[1] < c1.n ? r1[1] : c1.n;
        const float w = __fadd_ru(__fmul_ru((float)(b0 - a0), m0), __fmul_ru((float)(b1 - a1), m1));
        cm = fmaxf(cm, w);
      }
      cm = block_max_all(cm);
      if (cm > 0.f) {
        const float x = fminf(__fdiv_rd(268435456.0f, cm), 1.329228e36f);   // 2^31 / (8 cm), at most 2^120
        S = __uint_as_float(__float_as_uint(x) & 0xff800000u);
      }
    }
    const float pscale = (float)r / 256.0f;
    const int bxf = cb.ix0 * r, byf = cb.iy0 * r, bzf = cb.iz0 * r;
    for (int s = 0; s < 2; ++s) {
      const PCodes& cs = s ? c1 : c0;
      // float mode: the species mass times the block's power-of-two scale
      // (exact), so a corner's fixed-point value is rint(m S w)
      const float m = sizeof(Acc) == 4 ? __fmul_rn(s ? m1 : m0, S) : (s ? m1 : m0);
      const long long M = s ? M1 : M0;
      const int64_t* ro_s = roff + s * nrow * (bk.RX + 1);
      for (int row = 0; row < nrow; ++row) {
        const int64_t* ro = ro_s + row * (bk.RX + 1);
        const int iy = cb.iy0 + row % bk.RY, iz = cb.iz0 + row / bk.RY;
        // A corrupt stream (flagged by the scan) may claim more particles than
        // exist; never read past the caller's n records.
        const int64_t p0 = ro[0] < cs.n ? ro[0] : cs.n;
        const int64_t p1 = ro[bk.RX] < cs.n ? ro[bk.RX] : cs.n;
        const int64_t rounds = (p1 - p0 + blockDim.x - 1) / blockDim.x;
        for (int64_t it = 0; it < rounds; ++it) {
          const int64_t p = p0 + it * blockDim.x + threadIdx.x;
          const bool live = p < p1;
          int ixl = 0;
          float px = 0.f, py = 0.f, pz = 0.f;
          if (live) {
            ixl = row_cell(ro, bk.RX, p);
            int q[3];
            unpack_pos(cs.pos[p], q);
            if (dep_coarse) {
              px = decode_pos(cb.ix0 + ixl, q[0], pscale);
              py = decode_pos(iy, q[1], pscale);
              pz = decode_pos(iz, q[2], pscale);
            }
            // fine CIC in local region coordinates (no wrap inside the block).
            // Decoded positions are exact dyadics, x = c r + (2q + 1) r / 512,
            // so the fine cell and the weight come from the codes in integer
            // arithmetic (the same values as floor(x) and x - floor(x)).
            int num[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) num[d] = (2 * q[d] + 1) * r;
            const int lx = ixl * r + (num[0] >> 9), ly = (iy - cb.iy0) * r + (num[1] >> 9),
                      lz = (iz - cb.iz0) * r + (num[2] >> 9);
            float w1[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) w1[d] = __fmul_rn(__int2float_rn(num[d] & 511), 1.0f / 512.0f);
            Acc t8[8];
            corner_masses(m, M, w1, t8);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
              const int idx = ((lz + dz) * fy + (ly + dy)) * fx + (lx + dx);
              if constexpr (sizeof(Acc) == 4)
                atomicAdd(reinterpret_cast<unsigned int*>(sf) + idx, __float2uint_rn((float)t8[c]));
              else
                smem_acc(&sf[idx], t8[c]);
            }
          }
          if (dep_coarse) {
            // Coarse cell == compression cell (coarse_ratio == cmp_ratio), so every
            // particle of a run shares its 8 coarse corners: sum the run in
            // registers and let its last lane do 8 shared-memory adds.
            Acc cv[8];
            if (live) {
              const float sc_inv = 1.0f / (float)g.rc;
              float ux = __fmul_rn(px, sc_inv), uy = __fmul_rn(py, sc_inv), uz = __fmul_rn(pz, sc_inv);
              float v1[3] = {__fsub_rn(ux, floorf(ux)), __fsub_rn(uy, floorf(uy)), __fsub_rn(uz, floorf(uz))};
              corner_masses(m, M, v1, cv);
            } else {
#pragma unroll
              for (int c = 0; c < 8; ++c) cv[c] = (Acc)0;
            }
            const unsigned key = live ? (unsigned)ixl : 0xffffffffu;
            if (run_reduce<8, Acc>(key, cv) && live) {
              const int kx = ixl, ky = row % bk.RY, kz = row / bk.RY;
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
                smem_acc(&sc[((kz + dz) * cy + (ky + dy)) * cx + (kx + dx)], cv[c]);
              }
            }
          }
        }
      }
    }
    __syncthreads();
    if constexpr (sizeof(Acc) == 4) {
      // fixed point -> float32 (S is a power of two: the scaling is exact)
      const float inv_s = 1.0f / S;
      const unsigned int* si = reinterpret_cast<const unsigned int*>(sf);
      for (int i = threadIdx.x; i < nsf; i += blockDim.x) sf[i] = __fmul_rn(__uint2float_rn(si[i]), inv_s);
      __syncthreads();
    }
    const int nf = g.nf;
    // flush: one warp per region row (z, y), lanes along x
    for (int line = threadIdx.x >> 5; line < fy * fz; line += blockDim.x >> 5) {
      const int lz = line / fy, ly = line - lz * fy;
      int gy = byf + ly, gz = bzf + lz;
      if (gy >= nf) gy -= nf;
      if (gz >= nf) gz -= nf;
      Acc* grow = rho_f + ((int64_t)gz * nf + gy) * nf;
      const Acc* srow = sf + line * fx;
      for (int lx = threadIdx.x & 31; lx < fx; lx += 32) {
        const Acc val = srow[lx];
        if (val == (Acc)0) continue;
        int gx = bxf + lx;
        if (gx >= nf) gx -= nf;
        global_add(grow + gx, val);
      }
    }
    const int nc = g.nc;
    for (int i = threadIdx.x; i < nsc; i += blockDim.x) {
      Acc val = sc[i];
      if (val == (Acc)0) continue;
      int lx = i % cx, ly = (i / cx) % cy, lz = i / (cx * cy);
      int gx = cb.ix0 + lx, gy = cb.iy0 + ly, gz = cb.iz0 + lz;
      if (gx >= nc) gx -= nc;
      if (gy >= nc) gy -= nc;
      if (gz >= nc) gz -= nc;
      global_add(&rho_c[((int64_t)gz * nc + gy) * nc + gx], val);
    }
    if (restr) {
      // rho_c(C) += sum_k w(kx) w(ky) w(kz) tile(r C + k), w(k) = 1 - |k| / r, over the
      // tile's part; coarse cells C = block cell + (0 .. RX, 0 .. RY, 0 .. RZ); separable.
      const float* tile = reinterpret_cast<const float*>(sf);
      float* T1 = reinterpret_cast<float*>(sc) + cx * cy * cz;   // [fz][fy][cx]
      float* T2 = T1 + fz * fy * cx;                             // [fz][cy][cx]
      const float inv = 1.0f / (float)r;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
      for (int line = warp; line < fz * fy; line += nwarp) {
        const float* row = tile + line * fx;
        for (int q = lane; q < cx; q += 32) {
          float t = 0.f;
          for (int k = 1 - r; k < r; ++k) {
            const int j = r * q + k;
            if (j >= 0 && j < fx) t = fmaf(1.0f - (float)(k < 0 ? -k : k) * inv, row[j], t);
          }
          T1[line * cx + q] = t;
        }
      }
      __syncthreads();
      for (int line = warp; line < fz * cy; line += nwarp) {
        const int lz = line / cy, qy = line - lz * cy;
        for (int q = lane; q < cx; q += 32) {
          float t = 0.f;
          for (int k = 1 - r; k < r; ++k) {
            const int j = r * qy + k;
            if (j >= 0 && j < fy) t = fmaf(1.0f - (float)(k < 0 ? -k : k) * inv, T1[(lz * fy + j) * cx + q], t);
          }
          T2[line * cx + q] = t;
        }
      }
      __syncthreads();
      for (int line = warp; line < cz * cy; line += nwarp) {
        const int qz = line / cy, qy = line - qz * cy;
        int gy = cb.iy0 + qy, gz = cb.iz0 + qz;
        if (gy >= nc) gy -= nc;
        if (gz >= nc) gz -= nc;
        float* crow = reinterpret_cast<float*>(rho_c) + ((int64_t)gz * nc + gy) * nc;
        for (int q = lane; q < cx; q += 32) {
          float t = 0.f;
          for (int k = 1 - r; k < r; ++k) {
            const int j = r * qz + k;
            if (j >= 0 && j < fz) t = fmaf(1.0f - (float)(k < 0 ? -k : k) * inv, T2[(j * cy + qy) * cx + q], t);
          }
          int gx = cb.ix0 + q;
          if (gx >= nc) gx -= nc;
          if (t != 0.f) atomicAdd(crow + gx, t);
        }
      }
    }
  });
}

// Window of destination compression cells owned by a cell block's histogram:
// the block widened by D cells on each side (clamped to the mesh), periodic.
struct Win {
  int ox, oy, oz, wx, wy, wz;
};
__device__ __forceinline__ Win window_of(const Geo& g, const Blk& bk, CellBlock cb) {
  Win w;
  const int n = g.ncmp, D = bk.D;
  w.wx = bk.RX + 2 * D < n ? bk.RX + 2 * D : n;
  w.wy = bk.RY + 2 * D < n ? bk.RY + 2 * D : n;
  w.wz = bk.RZ + 2 * D < n ? bk.RZ + 2 * D : n;
  w.ox = w.wx == n ? 0 : cb.ix0 - D;
  w.oy = w.wy == n ? 0 : cb.iy0 - D;
  w.oz = w.wz == n ? 0 : cb.iz0 - D;
  return w;
}
// Window slot of compression cell `key`, or -1 outside the window.
__device__ __forceinline__ int window_slot(const Geo& g, const Win& w, uint32_t key) {
  const int n = g.ncmp;
  int cx = (int)(key % (uint32_t)n), cy = (int)((key / (uint32_t)n) % (uint32_t)n), cz = (int)(key / ((uint32_t)n * n));
  int lx = cx - w.ox, ly = cy - w.oy, lz = cz - w.oz;
  if (lx < 0) lx += n;
  if (ly < 0) ly += n;
  if (lz < 0) lz += n;
  if (lx >= w.wx || ly >= w.wy || lz >= w.wz) return -1;
  return (lz * w.wy + ly) * w.wx + lx;
}
// Window slot of the compression cell with coordinates (cx, cy, cz), or -1.
__device__ __forceinline__ int window_slot_xyz(const Win& w, int n, int cx, int cy, int cz) {
  int lx = cx - w.ox, ly = cy - w.oy, lz = cz - w.oz;
  lx += lx < 0 ? n : (lx >= n ? -n : 0);
  ly += ly < 0 ? n : (ly >= n ? -n : 0);
  lz += lz < 0 ? n : (lz >= n ? -n : 0);
  if (lx >= w.wx || ly >= w.wy || lz >= w.wz) return -1;
  return (lz * w.wy + ly) * w.wx + lx;
}
// Scratch key of a particle: its window slot with the top bit set when its new
// cell lies in the block's window, else the new cell index itself.
constexpr uint32_t kInWindow = 0x80000000u;

// Per-particle scratch record of the two recompress passes (stream index t
// of ntot particles, both species).  Exact v_max' mode: one 16-byte record
// {new position word, v'_x, v'_y, v'_z as float bits}.  Bound mode (codes
// final in the count pass): 8-bit codes as one 8-byte record {position
// word, velocity word}; 16-bit codes as a 4-byte position word and, in a
// second array after the first (16-byte aligned), an 8-byte velocity word.
__device__ __forceinline__ unsigned long long* coded_vel16(uint4* tpv, int64_t ntot) {
  return reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(tpv) + ((4 * ntot + 15) & ~15ll));
}
__device__ __forceinline__ uint4 load_record(const uint4* tpv, int64_t t, int coded, bool vel16, int64_t ntot) {
  if (!coded) return tpv[t];
  if (!vel16) {
    const uint2 r = reinterpret_cast<const uint2*>(tpv)[t];
    return make_uint4(r.x, r.y, 0u, 0u);
  }
  const uint32_t pw = reinterpret_cast<const uint32_t*>(tpv)[t];
  const unsigned long long v = coded_vel16(const_cast<uint4*>(tpv), ntot)[t];
  return make_uint4(pw, (uint32_t)v, (uint32_t)(v >> 32), 0u);
}

// Cell index of window row r = lz wy + ly at x = 0 (add window_x for the column).
__device__ __forceinline__ uint32_t window_row(const Geo& g, const Win& w, int r) {
  const int n = g.ncmp;
  const int lz = r / w.wy, ly = r - lz * w.wy;
  int cy = w.oy + ly, cz = w.oz + lz;
  if (cy < 0) cy += n; else if (cy >= n) cy -= n;
  if (cz < 0) cz += n; else if (cz >= n) cz -= n;
  return (uint32_t)(n * (cy + n * cz));
}
__device__ __forceinline__ uint32_t window_x(const Geo& g, const Win& w, int lx) {
  int cx = w.ox + lx;
  if (cx < 0) cx += g.ncmp; else if (cx >= g.ncmp) cx -= g.ncmp;
  return (uint32_t)cx;
}

// Pass 1 of interpolate + kick + drift + recompress, both species of one cell
// block: the block's force region (fine: (RX r + 1)(RY r + 1)(RZ r + 1) cells,
// coarse: (RX + 1)(RY + 1)(RZ + 1), 3 components) is copied to shared memory
// with coalesced row loads; every particle is decoded, gathered, kicked and
// drifted; its new cell, in-cell position bytes and new velocity go to the
// step's scratch arrays in stream order; new-cell counts are histogrammed in
// shared memory over the block's window (far movers: global atomics) and
// flushed once per window cell; per-species max |v'_d| is reduced.
// Threads per CTA of the deposit and of the two kick passes, and the resident
// CTAs per SM the kick passes are compiled for (sets their register budget).
#ifndef PM_IKD_THREADS
#define PM_IKD_THREADS 512
#endif
#ifndef PM_SCATTER_THREADS
#define PM_SCATTER_THREADS 256
#endif
#ifndef PM_IKD_MIN_BLOCKS
#define PM_IKD_MIN_BLOCKS 2
#endif
// Scratch records a scatter thread loads before placing any of them.
#ifndef PM_SCATTER_UNROLL
#define PM_SCATTER_UNROLL 2
#endif
#ifndef PM_SCATTER_MIN_BLOCKS
#define PM_SCATTER_MIN_BLOCKS 5
#endif

template <int RX_, int RY_, int RZ_, int R_>
__global__ void __launch_bounds__(PM_IKD_THREADS, PM_IKD_MIN_BLOCKS) k_ikd_count(PCodes c0, PCodes c1, const int64_t* off0, const int64_t* off1, Geo g_arg, Blk bk_arg,
                            const float* acc_c, const float* acc_f, float ck, float cd, uint32_t* counts0,
                            uint32_t* counts1, uint32_t* vmax_bits, uint32_t* tkey, uint4* tpv,
                            const float* vq0, const float* vq1, const float4* app, int coarse) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Geo g = g_arg;
  Blk bk = bk_arg;
  fix_shape<RX_, RY_, RZ_, R_>(g, bk);
  // coarse: gather the coarse force separately (0 when the fine force mesh
  // already carries the prolongated coarse force)
  const bool two_c = g.two && coarse != 0;
  for_each_block(bk, [&](const int bid) {
    const int r = g.rcmp;
    const int nrow = bk.RY * bk.RZ;
    const int fx = bk.RX * r + 1, fy = bk.RY * r + 1, fz = bk.RZ * r + 1;
    const int cx = bk.RX + 1, cy = bk.RY + 1, cz = bk.RZ + 1;
    const CellBlock cb = block_of(bk, bid);
    const Win win = window_of(g, bk, cb);
    const int W = win.wx * win.wy * win.wz;
    int64_t* roff = reinterpret_cast<int64_t*>(smraw);
    uint32_t* hist = reinterpret_cast<uint32_t*>(roff + 2 * nrow * (bk.RX + 1));
    float* sf = reinterpret_cast<float*>(hist + 2 * W);
    const RegionStrides fst = region_strides(fx, fy, fz);
    float* sc = sf + 3 * fst.comp;
    load_row_offsets(off0, g, bk, cb, roff);
    load_row_offsets(off1, g, bk, cb, roff + nrow * (bk.RX + 1));
    for (int i = threadIdx.x; i < 2 * W; i += blockDim.x) hist[i] = 0;
    const int bxf = cb.ix0 * r, byf = cb.iy0 * r, bzf = cb.iz0 * r;
    {
      const int nf = g.nf;
      const int64_t nf3 = (int64_t)nf * nf * nf;
      const int lines = 3 * fz * fy;
      for (int li = threadIdx.x >> 5; li < lines; li += blockDim.x >> 5) {
        int comp = li / (fz * fy), rem = li - comp * fz * fy;
        int lz = rem / fy, ly = rem - lz * fy;
        int gz = bzf + lz, gy = byf + ly;
        if (gz >= nf) gz -= nf;
        if (gy >= nf) gy -= nf;
        const float* src = acc_f + comp * nf3 + ((int64_t)gz * nf + gy) * nf;
        float* dst = sf + comp * fst.comp + lz * fst.plane + ly * fst.row;
        for (int lx = threadIdx.x & 31; lx < fx; lx += 32) {
          int gx = bxf + lx;
          if (gx >= nf) gx -= nf;
          copy_async4(dst + lx, src + gx);   // all of a thread's copies in flight at once
        }
      }
      async_copies_wait();
      if (two_c) {
        const int nc = g.nc;
        const int64_t nc3 = (int64_t)nc * nc * nc;
        for (int i = threadIdx.x; i < 3 * cx * cy * cz; i += blockDim.x) {
          int comp = i / (cx * cy * cz), rem = i - comp * cx * cy * cz;
          int lz = rem / (cx * cy), rem2 = rem - lz * cx * cy;
          int ly = rem2 / cx, lx = rem2 - ly * cx;
          int gx = cb.ix0 + lx, gy = cb.iy0 + ly, gz = cb.iz0 + lz;
          if (gx >= nc) gx -= nc;
          if (gy >= nc) gy -= nc;
          if (gz >= nc) gz -= nc;
          sc[i] = __ldg(acc_c + comp * nc3 + ((int64_t)gz * nc + gy) * nc + gx);
        }
      }
    }
    __syncthreads();
    const float pscale = (float)r / 256.0f;
    const float inv_r = 1.0f / (float)r;
    const float nf = (float)g.nf;
    for (int s = 0; s < 2; ++s) {
      const PCodes& in = s ? c1 : c0;
      uint32_t* counts = s ? counts1 : counts0;
      uint32_t* hs = hist + s * W;
      const int64_t toff = s ? c0.n : 0;
      const int half = in.vel16 ? 32768 : 128;
      const float step = __fmul_rn(*in.vmax, 1.0f / (float)half);
      float local_max = 0.f;
      // v_max' known before the pass (bound mode): quantise here, the scatter copies codes
      const float* vq = s ? vq1 : vq0;
      const bool coded = vq != nullptr;
      const float vqm = coded ? *vq : 0.f;
      const bool qzero = !(vqm > 0.f);
      const float qs = (coded && !qzero) ? __fdiv_rn(in.vel16 ? 32768.0f : 128.0f, vqm) : 0.f;
      const int64_t* ro_s = roff + s * nrow * (bk.RX + 1);
      for (int row = 0; row < nrow; ++row) {
        const int64_t* ro = ro_s + row * (bk.RX + 1);
        const int iy = cb.iy0 + row % bk.RY, iz = cb.iz0 + row / bk.RY;
        const int64_t p0 = ro[0] < in.n ? ro[0] : in.n;
        const int64_t p1 = ro[bk.RX] < in.n ? ro[bk.RX] : in.n;
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
          const int ixl = row_cell(ro, bk.RX, p);
          int q[3], qv[3];
          unpack_pos(in.pos[p], q);
          load_vel(in.vel, in.vel16, p, qv);
          float x[3], v[3], a[3];
          x[0] = decode_pos(cb.ix0 + ixl, q[0], pscale);
          x[1] = decode_pos(iy, q[1], pscale);
          x[2] = decode_pos(iz, q[2], pscale);
#pragma unroll
          for (int d = 0; d < 3; ++d) v[d] = decode_vel(qv[d], half, step);
          // Decoded positions are exact dyadics, so the CIC cell and weight come
          // from the codes in integer arithmetic: x = c r + (2q + 1) r / 512.
          const int ky = row % bk.RY, kz = row / bk.RY;
          int num[3];
          float w1[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            num[d] = (2 * q[d] + 1) * r;
            w1[d] = __fmul_rn(__int2float_rn(num[d] & 511), 1.0f / 512.0f);
          }
          gather_strided(sf, fst, ixl * r + (num[0] >> 9), ky * r + (num[1] >> 9), kz * r + (num[2] >> 9), w1, a);
          if (two_c) {
            // coarse cell == compression cell: corner (ixl, ky, kz), weight (2q + 1) / 512
            float b[3], u1[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) u1[d] = __fmul_rn(__int2float_rn(2 * q[d] + 1), 1.0f / 512.0f);
            gather_idx(sc, cx, cy, cz, ixl, ky, kz, u1, b);
            a[0] = __fadd_rn(b[0], a[0]);
            a[1] = __fadd_rn(b[1], a[1]);
            a[2] = __fadd_rn(b[2], a[2]);
          }
          if (app) {   // particle-particle term (Eq. 4), precomputed per particle
            const float4 q4 = app[toff + p];
            a[0] = __fadd_rn(a[0], q4.x);
            a[1] = __fadd_rn(a[1], q4.y);
            a[2] = __fadd_rn(a[2], q4.z);
          }
          kick_drift(x, v, a, ck, cd, nf);
          int cc[3], qq[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) encode_pos(x[d], inv_r, g.ncmp, cc[d], qq[d]);
          const uint32_t key = (uint32_t)(cc[0] + g.ncmp * (cc[1] + g.ncmp * cc[2]));
          const int slot = window_slot_xyz(win, g.ncmp, cc[0], cc[1], cc[2]);
          const int64_t t = toff + p;
          tkey[t] = slot >= 0 ? (kInWindow | (uint32_t)slot) : key;
          const uint32_t pw = (uint32_t)qq[0] | ((uint32_t)qq[1] << 8) | ((uint32_t)qq[2] << 16);
          if (coded) {
            int c3[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) c3[d] = encode_vel(v[d], qs, half, qzero);
            if (in.vel16) {
              reinterpret_cast<uint32_t*>(tpv)[t] = pw;
              coded_vel16(tpv, c0.n + c1.n)[t] = (unsigned long long)((uint32_t)c3[0] | ((uint32_t)c3[1] << 16)) |
                                                 ((unsigned long long)c3[2] << 32);
            } else {
              reinterpret_cast<uint2*>(tpv)[t] =
                  make_uint2(pw, (uint32_t)c3[0] | ((uint32_t)c3[1] << 8) | ((uint32_t)c3[2] << 16));
            }
          } else {
            tpv[t] = make_uint4(pw, __float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]));
            local_max = fmaxf(local_max, fmaxf(fabsf(v[0]), fmaxf(fabsf(v[1]), fabsf(v[2]))));
          }
          if (slot >= 0) atomicAdd(hs + slot, 1u);
          else atomicAdd(counts + key, 1u);
        }
      }
      if (!coded) block_vmax(local_max, vmax_bits + s);
    }
    __syncthreads();
    // flush: one warp per window row (species, z, y), lanes along x
    const int wyz = win.wy * win.wz;
    for (int rw = threadIdx.x >> 5; rw < 2 * wyz; rw += blockDim.x >> 5) {
      const int sp = rw >= wyz ? 1 : 0;
      const uint32_t rowcell = window_row(g, win, rw - sp * wyz);
      const uint32_t* hrow = hist + sp * W + (rw - sp * wyz) * win.wx;
      uint32_t* cnt = sp ? counts1 : counts0;
      for (int lx = threadIdx.x & 31; lx < win.wx; lx += 32) {
        const uint32_t k = hrow[lx];
        if (k) atomicAdd(cnt + rowcell + window_x(g, win, lx), k);
      }
    }
  });
}

// Slot countdown of the in-window particles of a warp.  Consecutive lanes
// with the same slot form a run (the particle stream is cell ordered and most
// particles stay in their cell, so a warp's particles fall in one or two
// runs); the run's first lane takes the run's slots with one atomic and
// hands them out, since a shared-memory atomic whose lanes share an address
// and return their values is serialised lane by lane.  All 32 lanes must
// call it; lanes without a slot pass has = false and a slot of their own
// (~0u - lane).  Returns what atomicSub(hist + slot, 1) would have returned.
__device__ __forceinline__ uint32_t run_countdown(uint32_t* hist, uint32_t slot, bool has) {
  const int lane = (int)(threadIdx.x & 31);
  const uint32_t prev = __shfl_up_sync(0xffffffffu, slot, 1);
  const bool head = lane == 0 || prev != slot;
  const uint32_t heads = __ballot_sync(0xffffffffu, head);
  const uint32_t upto = 0xffffffffu >> (31 - lane);   // lanes 0 .. lane
  const int first = 31 - __clz(heads & upto);         // head of this lane's run
  const uint32_t later = heads & ~upto;
  const int end = later ? __ffs(later) - 1 : 32;       // head of the next run
  uint32_t old = 0;
  if (head && has) old = atomicSub(hist + slot, (uint32_t)(end - lane));
  old = __shfl_sync(0xffffffffu, old, first);
  return old - (uint32_t)(lane - first);
}

// Pass 2: place every particle of a cell block in its new cell.  Phase 1
// histograms the block's new cells over its window; phase 2 reserves one
// contiguous range per window cell from the cell's global cursor (counts,
// counted down to zero); phase 3 hands out slots from those ranges with
// shared-memory atomics (far movers take single global slots), quantises the
// velocity with the new v_max and writes the codes.
template <int RX_, int RY_, int RZ_, int R_>
__global__ void __launch_bounds__(PM_SCATTER_THREADS, PM_SCATTER_MIN_BLOCKS) k_ikd_scatter(int64_t n0, int64_t n1, const int64_t* off0, const int64_t* off1, Geo g_arg, Blk bk_arg,
                              uint32_t* counts0, uint32_t* counts1, const int64_t* newoff0, const int64_t* newoff1,
                              PCodesOut o0, PCodesOut o1, const uint32_t* tkey, const uint4* tpv, int coded,
                              int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Geo g = g_arg;
  Blk bk = bk_arg;
  fix_shape<RX_, RY_, RZ_, R_>(g, bk);
  for_each_block(bk, [&](const int bid) {
    const int nrow = bk.RY * bk.RZ;
    const CellBlock cb = block_of(bk, bid);
    const Win win = window_of(g, bk, cb);
    const int W = win.wx * win.wy * win.wz;
    int64_t* roff = reinterpret_cast<int64_t*>(smraw);
    unsigned long long* base = reinterpret_cast<unsigned long long*>(roff + 2 * nrow * (bk.RX + 1));
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + 2 * W);
    load_row_offsets(off0, g, bk, cb, roff);
    load_row_offsets(off1, g, bk, cb, roff + nrow * (bk.RX + 1));
    for (int i = threadIdx.x; i < 2 * W; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int s = 0; s < 2; ++s) {
      const int64_t n = s ? n1 : n0;
      const int64_t toff = s ? n0 : 0;
      for (int row = 0; row < nrow; ++row) {
        const int64_t* ro = roff + (s * nrow + row) * (bk.RX + 1);
        const int64_t p0 = ro[0] < n ? ro[0] : n, p1 = ro[bk.RX] < n ? ro[bk.RX] : n;
        // four keys per thread loaded before any is counted
        for (int64_t p = p0 + threadIdx.x; p < p1; p += 4 * (int64_t)blockDim.x) {
          uint32_t tk[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int64_t q = p + j * (int64_t)blockDim.x;
            tk[j] = q < p1 ? tkey[toff + q] : 0u;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (tk[j] & kInWindow) atomicAdd(hist + s * W + (tk[j] & ~kInWindow), 1u);
        }
      }
    }
    __syncthreads();
    // Reserve the block's range in each window cell.  A thread takes up to
    // RJ slots at a time and issues all their cursor atomics and offset loads
    // before using any result, so their round trips overlap.
    constexpr int RJ = 4;
    for (int i0 = threadIdx.x; i0 < 2 * W; i0 += RJ * blockDim.x) {
      uint32_t cell[RJ], k[RJ], top[RJ];
      int64_t no[RJ];
#pragma unroll
      for (int j = 0; j < RJ; ++j) {
        const int i = i0 + j * blockDim.x;
        k[j] = i < 2 * W ? hist[i] : 0u;
        cell[j] = 0;
        if (k[j]) {
          const int sp = i >= W ? 1 : 0, r = i - sp * W;
          const int row = r / win.wx, lx = r - row * win.wx;
          cell[j] = window_row(g, win, row) + window_x(g, win, lx);
        }
      }
#pragma unroll
      for (int j = 0; j < RJ; ++j) {
        const int i = i0 + j * blockDim.x;
        if (!k[j]) continue;
        const bool sp = i >= W;
        top[j] = atomicSub((sp ? counts1 : counts0) + cell[j], k[j]);
        no[j] = (sp ? newoff1 : newoff0)[cell[j]];
      }
#pragma unroll
      for (int j = 0; j < RJ; ++j)
        if (k[j]) base[i0 + j * blockDim.x] = (unsigned long long)(no[j] + (int64_t)top[j] - (int64_t)k[j]);
    }
    __syncthreads();
    for (int s = 0; s < 2; ++s) {
      const int64_t n = s ? n1 : n0;
      const int64_t toff = s ? n0 : 0;
      const PCodesOut& o = s ? o1 : o0;
      uint32_t* counts = s ? counts1 : counts0;
      const int64_t* newoff = s ? newoff1 : newoff0;
      const int half = o.vel16 ? 32768 : 128;
      const float vm = *o.vmax;
      const bool vzero = !(vm > 0.f);
      const float sv = vzero ? 0.f : __fdiv_rn(o.vel16 ? 32768.0f : 128.0f, vm);
      for (int row = 0; row < nrow; ++row) {
        const int64_t* ro = roff + (s * nrow + row) * (bk.RX + 1);
        const int64_t p0 = ro[0] < n ? ro[0] : n, p1 = ro[bk.RX] < n ? ro[bk.RX] : n;
        // PM_SCATTER_UNROLL particles per thread per iteration, all loaded
        // before any is placed, keep that many independent loads in flight.
        // The trip count is the same for every thread (whole warps take part
        // in the slot countdown).
        for (int64_t pb = p0; pb < p1; pb += PM_SCATTER_UNROLL * (int64_t)blockDim.x) {
          const int64_t p = pb + threadIdx.x;
          int64_t pp[PM_SCATTER_UNROLL];
          uint32_t tk[PM_SCATTER_UNROLL];
          uint4 pv[PM_SCATTER_UNROLL];
#pragma unroll
          for (int u = 0; u < PM_SCATTER_UNROLL; ++u) {
            pp[u] = p + u * (int64_t)blockDim.x;
            tk[u] = 0u;
            if (pp[u] < p1) {
              tk[u] = tkey[toff + pp[u]];
              pv[u] = load_record(tpv, toff + pp[u], coded, o.vel16, n0 + n1);
            }
          }
#pragma unroll
          for (int u = 0; u < PM_SCATTER_UNROLL; ++u) {
            const bool live = pp[u] < p1;
            const bool inw = live && (tk[u] & kInWindow);
            const uint32_t sl = inw ? s * W + (tk[u] & ~kInWindow) : ~0u - (threadIdx.x & 31);
            // rank within the block's range of the cell: count its histogram entry down
            const uint32_t rank = run_countdown(hist, sl, inw);
            if (!live) continue;
            int64_t dst;
            if (inw) {
              dst = (int64_t)base[sl] + (int64_t)rank - 1;
            } else {
              const uint32_t top = atomicSub(counts + tk[u], 1u);
              dst = newoff[tk[u]] + (int64_t)top - 1;
            }
            if (dst < 0 || dst >= n) {
              atomicOr(status, ST_CORRUPT);
              continue;
            }
            o.pos[dst] = pv[u].x;
            if (coded) {
              if (o.vel16)
                reinterpret_cast<unsigned long long*>(o.vel)[dst] =
                    (unsigned long long)pv[u].y | ((unsigned long long)pv[u].z << 32);
              else
                reinterpret_cast<uint32_t*>(o.vel)[dst] = pv[u].y;
              continue;
            }
            int qv[3];
            qv[0] = encode_vel(__uint_as_float(pv[u].y), sv, half, vzero);
            qv[1] = encode_vel(__uint_as_float(pv[u].z), sv, half, vzero);
            qv[2] = encode_vel(__uint_as_float(pv[u].w), sv, half, vzero);
            store_vel(o.vel, o.vel16, dst, qv);
          }
        }
      }
    }
  });
}

// ------------------------------------------------------------ launchers --

// Brick order of the cell blocks (block_of): edge in block rows, and the
// number of (y, z) block rows from which it is used.  Measured on the
// 1536^3 workload (147,456 kick-block rows): scatter 90.1 -> 70.5 ms; on
// the 256^3 workload (4,096 rows, whose new codes fit in L2 anyway) it made
// the scatter 4% slower, so smaller grids keep the row order.
#ifndef PM_BLOCK_BRICK
#define PM_BLOCK_BRICK 16
#endif
#ifndef PM_BRICK_MIN_ROWS
#define PM_BRICK_MIN_ROWS 32768
#endif

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_decompress(const PCodes& in, const int64_t* off, const Geo& g, float* x, float* v, cudaStream_t st) {
  if (in.n == 0) return cudaSuccess;
  k_decompress<<<grid_for(in.n, 256), 256, 0, st>>>(in, off, g, x, v);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_deposit(const float* x, int64_t n, float m, const Geo& g, float* rho_c, float* rho_f, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_deposit_global<<<grid_for(n, 256), 256, 0, st>>>(x, n, m, g, rho_c, rho_f);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_deposit_weights(const float* x, int64_t n, const float* w, int nw, const Geo& g, float* out,
                                  cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_deposit_weights<<<grid_for(n, 256), 256, 0, st>>>(x, n, w, nw, g, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_deposit_fixed(const float* x, int64_t n, long long M, const Geo& g, long long* rho_c,
                                 long long* rho_f, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_deposit_fixed_global<<<grid_for(n, 256), 256, 0, st>>>(x, n, M, g, rho_c, rho_f);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_interpolate(const float* x, int64_t n, const Geo& g, const float* acc_c, const float* acc_f,
                               float* a, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_interpolate<<<grid_for(n, 256), 256, 0, st>>>(x, n, g, acc_c, acc_f, a);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_kick_drift(float* x, float* v, int64_t n, const Geo& g, const float* acc_c, const float* acc_f,
                              float ck, float cd, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_kick_drift<<<grid_for(n, 256), 256, 0, st>>>(x, v, n, g, acc_c, acc_f, ck, cd);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_compress(const float* x, const float* v, int64_t n, const Geo& g, uint32_t* counts,
                            uint32_t* vmax_bits, const float* vmax_in, int64_t* off, pm_codes_t& out, bool vel16,
                            void* partial, int* status, cudaStream_t st) {
  PCodesOut o{reinterpret_cast<uint32_t*>(out.pos), out.vel, out.vmax, vel16};
  cudaMemsetAsync(vmax_bits, 0, sizeof(uint32_t), st);
  int grid = grid_for(n > 0 ? n : 1, 256);
  k_compress_pass<0><<<grid, 256, 0, st>>>(x, v, n, g, counts, vmax_bits, vmax_in, off, o, status);
  k_set_vmax<<<1, 1, 0, st>>>(vmax_bits, vmax_in, out.vmax);
  cudaError_t e = scan_counts(counts, g.ncell, n, off, out, partial, status, st);
  if (e != cudaSuccess) return e;
  k_compress_pass<1><<<grid, 256, 0, st>>>(x, v, n, g, counts, vmax_bits, vmax_in, off, o, status);
  note_launches(3);
  return cudaGetLastError();
}

size_t ikd_count_smem(const Geo& g, const Blk& bk) {
  size_t nrow = (size_t)bk.RY * bk.RZ;
  size_t coarse = g.two ? (size_t)(bk.RX + 1) * (bk.RY + 1) * (bk.RZ + 1) : 0;
  const RegionStrides st = region_strides(bk.RX * g.rcmp + 1, bk.RY * g.rcmp + 1, bk.RZ * g.rcmp + 1);
  return 2 * nrow * (bk.RX + 1) * sizeof(int64_t) + 2 * (size_t)window_cells(g, bk) * 4 +
         3 * ((size_t)st.comp + coarse) * sizeof(float);
}

size_t ikd_scatter_smem(const Geo& g, const Blk& bk) {
  size_t nrow = (size_t)bk.RY * bk.RZ;
  return 2 * nrow * (bk.RX + 1) * sizeof(int64_t) + 2 * (size_t)window_cells(g, bk) * (8 + 4);
}

int block_brick(const Blk& bk) {
  const int B = PM_BLOCK_BRICK;
  return (B > 1 && bk.nby % B == 0 && bk.nbz % B == 0 && (int64_t)bk.nby * bk.nbz >= PM_BRICK_MIN_ROWS) ? B : 1;
}

int window_cells(const Geo& g, const Blk& bk) {
  const int n = g.ncmp;
  int wx = bk.RX + 2 * bk.D < n ? bk.RX + 2 * bk.D : n;
  int wy = bk.RY + 2 * bk.D < n ? bk.RY + 2 * bk.D : n;
  int wz = bk.RZ + 2 * bk.D < n ? bk.RZ + 2 * bk.D : n;
  return wx * wy * wz;
}

size_t deposit_codes_smem(const Geo& g, const Blk& bk, bool fixed) {
  size_t nrow = (size_t)bk.RY * bk.RZ;
  size_t fine = (size_t)(bk.RX * g.rcmp + 1) * (bk.RY * g.rcmp + 1) * (bk.RZ * g.rcmp + 1);
  size_t coarse = g.two ? (size_t)(bk.RX + 1) * (bk.RY + 1) * (bk.RZ + 1) : 0;
  // float two-level: room for the restriction's x and y partial sums
  size_t restr = (g.two && !fixed) ? ((size_t)(bk.RZ * g.rcmp + 1) * ((bk.RY * g.rcmp + 1) + (bk.RY + 1)) *
                                      (bk.RX + 1)) : 0;
  return 2 * nrow * (bk.RX + 1) * sizeof(int64_t) + (fine + coarse) * (fixed ? 8 : 4) + restr * 4;
}

// Grid of a cell-block launch: one CTA per block, or (bk.work set) as many
// CTAs as fit on the device at once, capped by the block count.
template <class K>
static int block_grid(K kernel, const Blk& bk, int threads, size_t smem) {
  const int nblk = bk.nbx * bk.nby * bk.nbz;
  if (!bk.work) return nblk;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  const long long resident = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  return (int)(resident < nblk ? resident : nblk);
}

cudaError_t launch_deposit_codes(const PCodes& c0, const PCodes& c1, const int64_t* off0, const int64_t* off1,
                                 const Geo& g, const Blk& bk, float m0, float m1, long long M0, long long M1,
                                 void* rho_c, void* rho_f, bool fixed, cudaStream_t st) {
  size_t smem = deposit_codes_smem(g, bk, fixed);
  int nblk = bk.nbx * bk.nby * bk.nbz;
  const bool tuned = PM_SHAPE_INSTANCES && bk.RX == 32 && bk.RY == 2 && bk.RZ == 1 && g.rcmp == 4;
  if (fixed) {
    cudaFuncSetAttribute(k_deposit_codes<long long, 0, 0, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    nblk = block_grid(k_deposit_codes<long long, 0, 0, 0, 0>, bk, PM_DEPOSIT_THREADS, smem);
    k_deposit_codes<long long, 0, 0, 0, 0><<<nblk, PM_DEPOSIT_THREADS, smem, st>>>(c0, c1, off0, off1, g, bk, m0, m1, M0, M1,
                                                       static_cast<long long*>(rho_c), static_cast<long long*>(rho_f));
  } else {
    const auto k = tuned ? k_deposit_codes<float, 32, 2, 1, 4> : k_deposit_codes<float, 0, 0, 0, 0>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    nblk = block_grid(k, bk, PM_DEPOSIT_THREADS, smem);
    k<<<nblk, PM_DEPOSIT_THREADS, smem, st>>>(c0, c1, off0, off1, g, bk, m0, m1, M0, M1, static_cast<float*>(rho_c),
                                              static_cast<float*>(rho_f));
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ikd_count(const PCodes& c0, const PCodes& c1, const int64_t* off0, const int64_t* off1,
                             const Geo& g, const Blk& bk, const float* acc_c, const float* acc_f, float ck, float cd,
                             uint32_t* counts0, uint32_t* counts1, uint32_t* vmax_bits, uint32_t* tkey,
                             uint4* tpv, const float* vq0, const float* vq1, const float4* app, bool coarse, cudaStream_t st) {
  size_t smem = ikd_count_smem(g, bk);
  int nblk = bk.nbx * bk.nby * bk.nbz;
  const bool tuned = PM_SHAPE_INSTANCES && bk.RX == 64 && bk.RY == 1 && bk.RZ == 1 && g.rcmp == 4;
  const auto k = tuned ? k_ikd_count<64, 1, 1, 4> : k_ikd_count<0, 0, 0, 0>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  nblk = block_grid(k, bk, PM_IKD_THREADS, smem);
  k<<<nblk, PM_IKD_THREADS, smem, st>>>(c0, c1, off0, off1, g, bk, acc_c, acc_f, ck, cd, counts0, counts1, vmax_bits,
                                       tkey, tpv, vq0, vq1, app, coarse ? 1 : 0);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ikd_scatter(int64_t n0, int64_t n1, const int64_t* off0, const int64_t* off1, const Geo& g,
                               const Blk& bk, uint32_t* counts0, uint32_t* counts1, const int64_t* newoff0,
                               const int64_t* newoff1, const PCodesOut& o0, const PCodesOut& o1, const uint32_t* tkey,
                               const uint4* tpv, bool coded, int* status, cudaStream_t st) {
  size_t smem = ikd_scatter_smem(g, bk);
  int nblk = bk.nbx * bk.nby * bk.nbz;
  const bool tuned = PM_SHAPE_INSTANCES && bk.RX == 64 && bk.RY == 1 && bk.RZ == 1 && g.rcmp == 4;
  const auto k = tuned ? k_ikd_scatter<64, 1, 1, 4> : k_ikd_scatter<0, 0, 0, 0>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  nblk = block_grid(k, bk, PM_SCATTER_THREADS, smem);
  k<<<nblk, PM_SCATTER_THREADS, smem, st>>>(n0, n1, off0, off1, g, bk, counts0, counts1, newoff0, newoff1, o0, o1, tkey,
                                         tpv, coded ? 1 : 0, status);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_vmax_bound(const float* vin0, const float* vin1, const uint32_t* amax, float ck, float* vout0,
                              float* vout1, cudaStream_t st) {
  k_vmax_bound<<<1, 1, 0, st>>>(vin0, vin1, amax, ck, vout0, vout1);
  note_launches(1);
  return cudaGetLastError();
}

__global__ void k_set_vmax2(const uint32_t* vmax_bits, float* out0, float* out1) {
  *out0 = __uint_as_float(vmax_bits[0]);
  *out1 = __uint_as_float(vmax_bits[1]);
}

cudaError_t launch_set_vmax2(const uint32_t* vmax_bits, float* out0, float* out1, cudaStream_t st) {
  k_set_vmax2<<<1, 1, 0, st>>>(vmax_bits, out0, out1);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_set_vmax(const uint32_t* vmax_bits, float* out, cudaStream_t st) {
  k_set_vmax<<<1, 1, 0, st>>>(vmax_bits, nullptr, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace pm
