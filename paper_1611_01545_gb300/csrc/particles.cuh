// Device-side views and launchers of the particle kernels (particles.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pm_common.cuh"

namespace pm {

// Geometry as the particle kernels see it (plain values, passed by value).
struct Geo {
  int nf, rc, nc, rcmp, ncmp;
  int64_t ncell;
  bool two;
};

// Cell-block decomposition of the compression mesh for the fused passes.
struct Blk {
  int RX, RY, RZ;     // cells per block along x, y, z
  int nbx, nby, nbz;  // blocks along x, y, z
  int D;              // half-width (cells) of the new-cell histogram window
  int brick;          // blocks are handed out in bricks of brick x brick (y, z) block rows (1: row order)
  int* work;          // persistent launch: device counter of cell blocks taken (zeroed before the launch); null: one CTA per block
};

struct PCodes {
  const uint32_t* pos;
  const void* vel;
  const float* vmax;
  int64_t n;
  bool vel16;
};

struct PCodesOut {
  uint32_t* pos;
  void* vel;
  float* vmax;
  bool vel16;
};

cudaError_t scan_codes(const pm_codes_t& in, int64_t ncell, int64_t* off, void* partial_ws, int* status,
                       cudaStream_t st);
cudaError_t scan_counts(const uint32_t* counts, int64_t ncell, int64_t expect, int64_t* off, pm_codes_t& out,
                        void* partial_ws, int* status, cudaStream_t st);
// Both species in one set of launches (partials: 2 * scan_partial_bytes).
cudaError_t scan_codes2(const pm_codes_t in[2], int64_t ncell, int64_t* off0, int64_t* off1, void* partial_ws,
                        int* status, cudaStream_t st);
cudaError_t scan_counts2(const uint32_t* counts0, const uint32_t* counts1, int64_t ncell, const int64_t expect[2],
                         int64_t* off0, int64_t* off1, pm_codes_t out[2], void* partial_ws, int* status,
                         cudaStream_t st);
size_t scan_partial_bytes(int64_t ncell);

cudaError_t launch_decompress(const PCodes& in, const int64_t* off, const Geo& g, float* x, float* v, cudaStream_t st);
cudaError_t launch_deposit(const float* x, int64_t n, float m, const Geo& g, float* rho_c, float* rho_f,
                           cudaStream_t st);
cudaError_t launch_deposit_weights(const float* x, int64_t n, const float* w, int nw, const Geo& g, float* out,
                                  cudaStream_t st);
cudaError_t launch_deposit_fixed(const float* x, int64_t n, long long M, const Geo& g, long long* rho_c,
                                 long long* rho_f, cudaStream_t st);
cudaError_t launch_interpolate(const float* x, int64_t n, const Geo& g, const float* acc_c, const float* acc_f,
                               float* a, cudaStream_t st);
cudaError_t launch_kick_drift(float* x, float* v, int64_t n, const Geo& g, const float* acc_c, const float* acc_f,
                              float ck, float cd, cudaStream_t st);
cudaError_t launch_compress(const float* x, const float* v, int64_t n, const Geo& g, uint32_t* counts,
                            uint32_t* vmax_bits, const float* vmax_in, int64_t* off, pm_codes_t& out, bool vel16,
                            void* partial, int* status, cudaStream_t st);
size_t deposit_codes_smem(const Geo& g, const Blk& bk, bool fixed);
size_t ikd_count_smem(const Geo& g, const Blk& bk);
size_t ikd_scatter_smem(const Geo& g, const Blk& bk);
int window_cells(const Geo& g, const Blk& bk);
// Brick edge (block rows) of the block order for a block grid (1: row order).
int block_brick(const Blk& bk);
cudaError_t launch_deposit_codes(const PCodes& c0, const PCodes& c1, const int64_t* off0, const int64_t* off1,
                                 const Geo& g, const Blk& bk, float m0, float m1, long long M0, long long M1,
                                 void* rho_c, void* rho_f, bool fixed, cudaStream_t st);
cudaError_t launch_ikd_count(const PCodes& c0, const PCodes& c1, const int64_t* off0, const int64_t* off1,
                             const Geo& g, const Blk& bk, const float* acc_c, const float* acc_f, float ck, float cd,
                             uint32_t* counts0, uint32_t* counts1, uint32_t* vmax_bits, uint32_t* tkey,
                             uint4* tpv, const float* vq0, const float* vq1, const float4* app, bool coarse,
                             cudaStream_t st);
cudaError_t launch_ikd_scatter(int64_t n0, int64_t n1, const int64_t* off0, const int64_t* off1, const Geo& g,
                               const Blk& bk, uint32_t* counts0, uint32_t* counts1, const int64_t* newoff0,
                               const int64_t* newoff1, const PCodesOut& o0, const PCodesOut& o1, const uint32_t* tkey,
                               const uint4* tpv, bool coded, int* status, cudaStream_t st);
cudaError_t launch_set_vmax(const uint32_t* vmax_bits, float* out, cudaStream_t st);
cudaError_t launch_set_vmax2(const uint32_t* vmax_bits, float* out0, float* out1, cudaStream_t st);
// v_max' bound of both species from v_max and the maxima amax[3] (coarse mesh,
// fine mesh, PP accelerations; float bits).
// PP acceleration (Eq. 4) of every particle of both species into acc[t] (stream index t,
// species 0 first; float4, w = 0); max |a_d| into *amax when set.  pp.cu.
size_t pp_smem(const Geo& g);
cudaError_t launch_pp(const PCodes& c0, const PCodes& c1, const int64_t* off0, const int64_t* off1, const Geo& g,
                      float m0, float m1, float G, float r_soft, float4* acc, uint32_t* amax, cudaStream_t st);
// Packed codes (pack.cu): padded position / velocity words <-> record bytes.
cudaError_t launch_pack(const uint32_t* pos, const void* vel, bool vel16, int64_t n, uint8_t* ppos, uint8_t* pvel,
                        cudaStream_t st);
cudaError_t launch_unpack(const uint8_t* ppos, const uint8_t* pvel, bool vel16, int64_t n, uint32_t* pos, void* vel,
                          cudaStream_t st);
cudaError_t launch_vmax_bound(const float* vin0, const float* vin1, const uint32_t* amax, float ck, float* vout0,
                              float* vout1, cudaStream_t st);
cudaError_t launch_adj_deposit(const float* x, int64_t n, float m, int nf, const float* lam_rho, float* lam_x,
                               cudaStream_t st);
// lam_A is [3][n^3], or float4 [n^3] (x, y, z, unused) when interleaved (one vector
// reduction per corner instead of three).
cudaError_t launch_adj_interp(const float* x, int64_t n, int nf, const float* acc, float ck, float cd, float* lam_x,
                              float* lam_v, float* lam_A, bool interleaved, cudaStream_t st);

}  // namespace pm
