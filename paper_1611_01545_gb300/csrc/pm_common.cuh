// Internal declarations shared by the libpm translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pm.h"

namespace pm {

enum StatusBits : int { ST_CORRUPT = 1, ST_OVERFLOW = 2, ST_RANGE = 4, ST_TIMEOUT = 8 };

// Mesh / tile / compression-cell geometry derived from pm_config_t.
struct Geom {
  int nf = 0;     // fine cells per side
  int rc = 1;     // fine cells per coarse cell (1 = single mesh)
  int nc = 0;     // coarse cells per side (0 for a single mesh)
  int t = 0;      // tile interior
  int b = 0;      // tile buffer
  int T = 0;      // tile edge t + 2b (single mesh: nf)
  int nts = 1;    // tiles per side
  int rcmp = 4;   // fine cells per compression cell
  int ncmp = 0;   // compression cells per side
  bool two = false;
  int64_t ncell() const { return (int64_t)ncmp * ncmp * ncmp; }
  int64_t nfine3() const { return (int64_t)nf * nf * nf; }
  int64_t ncoarse3() const { return (int64_t)nc * nc * nc; }
  int ntiles() const { return nts * nts * nts; }
};

// Row pitch (complex values) of the spectrum buffers of an N^3 transform:
// N/2 + 1, padded to 50 for N = 96 so that every spectrum row starts on a
// 16-byte boundary (the tensor-map copies of the 96^3 passes need row
// strides that are multiples of 16 bytes).
__host__ __device__ constexpr int spec_pitch(int N) { return N == 96 ? 50 : N / 2 + 1; }

// One periodic-window FFT solve family (coarse mesh, single mesh or fine tiles).
struct SolvePlan {
  int N = 0;          // transform edge
  int NH = 0;         // N/2 + 1
  int NP = 0;         // spectrum row pitch, spec_pitch(N)
  int* status = nullptr;   // library status word (bounded copy waits report ST_TIMEOUT)
  int nts = 1;        // problems per side
  int t = 0, b = 0;   // output interior and offset of the window
  int src_n = 0;      // periodic source / destination mesh edge
  int batch = 1;      // problems per batch
  float* kern = nullptr;   // device [3][N slot][N slot][NH]
  float2* tw = nullptr;    // device [N]
  float2* spec = nullptr;  // device [batch][N][N][NP]
  float2* spec3 = nullptr; // device [batch][3][t][N][NP]
};

// Counts kernel launches made by the library (all handles); read by pm_launch_count.
void note_launches(int k);

// Launch helpers implemented in solve.cu.
// Prolongation added by the last solve pass: the coarse force [3][nc^3] (rc
// fine cells per coarse cell) interpolated onto the written fine nodes, after
// waiting for `ready` (may be null) on the launching stream.
struct Prolong {
  const float* coarse;
  int nc, rc;
  cudaEvent_t ready;
};
// amax (optional): atomicMax of max |a| over the written force values (before
// any prolongation is added), as float bits.
cudaError_t solve_launch(const SolvePlan& p, const void* src, bool src_fixed, float* dst, cudaStream_t st,
                         struct Timer* timer, unsigned int* amax = nullptr, const Prolong* pro = nullptr);
// Coarse density from the fine one (CIC restriction, float32).
cudaError_t launch_restrict(const float* rho_f, int nf, int rc, float* rho_c, cudaStream_t st);
// Transpose of the periodic-mesh solve (adjoint): lam_rho = A^T lam_acc; spec3comp holds
// the three component spectra [3][N][N][N/2+1].  lam_acc is [3][n^3], or float4 [n^3]
// (x, y, z, unused) when interleaved.
cudaError_t solve_adjoint_launch(const SolvePlan& p, const float* lam_acc, bool interleaved, float* lam_rho,
                                 float2* spec3comp, cudaStream_t st);
cudaError_t tile_window_launch(const SolvePlan& p, const float* src, int64_t tile, float* out, cudaStream_t st);

// Per-launch CUDA-event timing, accumulated by kind.
struct Timer {
  bool on = false;
  std::vector<std::string> names;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<double> total_ms;
  std::vector<long> count;
  std::vector<cudaEvent_t> pool;
  int kind(const char* name);
  void begin(int k, cudaStream_t st, cudaEvent_t* out);
  void end(int k, cudaStream_t st, cudaEvent_t start);
  void flush();
  void clear();
};

struct TimedScope {
  Timer* t;
  int k;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  TimedScope(Timer* tm, const char* name, cudaStream_t s) : t(tm), k(-1), st(s) {
    if (t && t->on) { k = t->kind(name); t->begin(k, st, &e0); }
  }
  ~TimedScope() {
    if (t && t->on && k >= 0) t->end(k, st, e0);
  }
};

// ---- codec arithmetic (Sec. 2.4), pinned to one rounding per operation ----

// Decoded coordinate of byte q in compression cell c: ((c 256 + q) + 1/2) * (rcmp / 256).
__device__ __forceinline__ float decode_pos(int c, int q, float scale) {
  return __fmul_rn(__fadd_rn(__int2float_rn(c * 256 + q), 0.5f), scale);
}
// ((q - half) + 1/2) * (vmax / half)
__device__ __forceinline__ float decode_vel(int q, int half, float step) {
  return __fmul_rn(__fadd_rn(__int2float_rn(q - half), 0.5f), step);
}
// floor(v * (half / vmax) + half) clamped to [0, 2 half - 1]; vmax == 0 -> half.
__device__ __forceinline__ int encode_vel(float v, float s, int half, bool zero) {
  if (zero) return half;
  float t = __fadd_rn(__fmul_rn(v, s), (float)half);
  float f = floorf(t);
  int q = (f < 0.f) ? 0 : (f > (float)(2 * half - 1) ? 2 * half - 1 : (int)f);
  return q;
}
// In-memory codes hold one padded word per particle: position bytes
// (px, py, pz, 0) as a uint32; velocity codes (vx, vy, vz, 0) as a uint32
// (8-bit codes) or as four uint16 in a uint64 (16-bit codes).
__device__ __forceinline__ void unpack_pos(uint32_t w, int q[3]) {
  q[0] = (int)(w & 0xffu);
  q[1] = (int)((w >> 8) & 0xffu);
  q[2] = (int)((w >> 16) & 0xffu);
}
__device__ __forceinline__ void load_vel(const void* vel, bool vel16, int64_t p, int q[3]) {
  if (vel16) {
    unsigned long long w = reinterpret_cast<const unsigned long long*>(vel)[p];
    q[0] = (int)(w & 0xffffull);
    q[1] = (int)((w >> 16) & 0xffffull);
    q[2] = (int)((w >> 32) & 0xffffull);
  } else {
    uint32_t w = reinterpret_cast<const uint32_t*>(vel)[p];
    q[0] = (int)(w & 0xffu);
    q[1] = (int)((w >> 8) & 0xffu);
    q[2] = (int)((w >> 16) & 0xffu);
  }
}
__device__ __forceinline__ void store_vel(void* vel, bool vel16, int64_t p, const int q[3]) {
  if (vel16)
    reinterpret_cast<unsigned long long*>(vel)[p] =
        (unsigned long long)q[0] | ((unsigned long long)q[1] << 16) | ((unsigned long long)q[2] << 32);
  else
    reinterpret_cast<uint32_t*>(vel)[p] = (uint32_t)q[0] | ((uint32_t)q[1] << 8) | ((uint32_t)q[2] << 16);
}

// In-cell byte and cell coordinate of x in [0, nf): u = x / rcmp (exact).
__device__ __forceinline__ void encode_pos(float x, float inv_r, int ncmp, int& c, int& q) {
  float u = __fmul_rn(x, inv_r);
  float fc = floorf(u);
  float f = __fsub_rn(u, fc);
  int qq = (int)__fmul_rn(f, 256.0f);
  q = qq > 255 ? 255 : qq;
  int ci = (int)fc;
  c = ci < 0 ? 0 : (ci >= ncmp ? ncmp - 1 : ci);
}

}  // namespace pm
