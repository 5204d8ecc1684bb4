// C ABI of libpm (include/pm.h): handle, workspace, precomputed Green's
// functions, entry points and the host serializer of the Sec. 2.4 stream.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "fft.cuh"
#include "particles.cuh"
#include "pm_common.cuh"

using namespace pm;

struct pm_handle {
  pm_config_t cfg;
  Geom gm;
  Geo geo;
  int device = 0;
  std::string err;
  // plans
  SolvePlan plan_mesh;   // coarse mesh (two-level) or the single periodic mesh
  SolvePlan plan_tiles;  // fine tiles (two-level)
  // workspace
  float* rho_f = nullptr;
  float* rho_c = nullptr;
  long long* rho_f_fix = nullptr;
  long long* rho_c_fix = nullptr;
  float* acc_f = nullptr;
  float* acc_c = nullptr;
  int64_t* off[2] = {nullptr, nullptr};
  int64_t* newoff[2] = {nullptr, nullptr};
  uint32_t* counts[2] = {nullptr, nullptr};
  uint32_t* vmax_bits = nullptr;  // [2]
  uint32_t* amax = nullptr;       // [3] max |a| over the coarse / fine force meshes and the PP accelerations (float bits)
  float4* app = nullptr;          // per particle PP acceleration (pp = 1), stream order, species 0 first
  void* partial = nullptr;
  int* status = nullptr;
  Blk blk_dep{}, blk_ikd{};
  bool persist_dep = false, persist_ikd = false;   // persistent launches of the particle passes
  int* work = nullptr;           // [4] device work counters of persistent launches
  int tile_batch_alloc = 1;      // tile workspace capacity (problems per solve batch)
  size_t smem_optin = 0;         // largest dynamic shared memory per block on this device
  // per-particle scratch of the fused step (stream order, both species)
  int64_t scratch_n = 0;
  uint32_t* tkey = nullptr;
  uint4* tpv = nullptr;      // per particle: new in-cell position code, v'_x, v'_y, v'_z (float bits)
  std::vector<void*> allocs;
  Timer timer;
  // adjoint workspace (single mesh): lam_acc float4 [n^3], component spectra [3][N][N][N/2+1]
  float* lam_acc = nullptr;
  float2* adj_spec = nullptr;
  // staging for pm_step_host
  pm_codes_t stage_in[2]{}, stage_out[2]{};
  bool staged = false;
  // packed record bytes for pm_step_packed (pos 3 B, vel 3 or 6 B per particle)
  uint8_t* pk_pos[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [in/out][species]; in and out share buffers
  uint8_t* pk_vel[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool pk_staged = false;
  // pm_step_packed: velocity bytes come over on their own stream while the
  // deposit and the solve run; the count pass waits for them
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t pk_fork = nullptr, pk_vel_ready = nullptr;
  cudaEvent_t pre_count_wait = nullptr;   // set only while a packed step is being enqueued
  // pm_step_packed_async: input copies on copy_stream, output copies on
  // d2h_stream, so consecutive steps overlap their copies with each other's
  // compute; separate packed input buffers (the output ones sit in the scratch)
  cudaStream_t d2h_stream = nullptr;
  cudaEvent_t as_in_free = nullptr, as_pos_ready = nullptr, as_vel_ready = nullptr, as_packed = nullptr,
              as_meta_done = nullptr, as_out_done = nullptr;
  uint8_t* as_pos[2] = {nullptr, nullptr};
  uint8_t* as_vel[2] = {nullptr, nullptr};
  // packed output buffers of their own when device memory allows; otherwise
  // the output shares the step scratch and the next count pass waits for it
  uint8_t* as_opos[2] = {nullptr, nullptr};
  uint8_t* as_ovel[2] = {nullptr, nullptr};
  bool as_sep = false;
  bool as_ready = false;
  cudaEvent_t pre_count_wait2 = nullptr;     // set only while an async packed step is being enqueued
  cudaEvent_t post_count_record = nullptr;   // recorded after the count pass (the staged input is read)
  // pm_step replay: one instantiated graph per (codes descriptors, c_k, c_d)
  struct StepGraph {
    int kind;   // 0: pm_step (device codes); 1: pm_step_packed (host codes)
    pm_codes_t in[2], out[2];
    double ck, cd;
    cudaGraphExec_t exec;
    long long launches;
  };
  bool graphs = false;
  cudaStream_t capture_stream = nullptr;
  // the coarse solve runs beside the tile solve on this stream (fork / join events)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // asynchronous checkpoint: device -> pinned host copies on their own stream
  cudaStream_t ckpt_stream = nullptr;
  cudaEvent_t ckpt_ready = nullptr, ckpt_done = nullptr;
  bool ckpt_pending = false;
  std::vector<StepGraph> step_graphs;
};

namespace {

int fail(pm_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define CK(h, expr)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(h, PM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));      \
  } while (0)

template <class T>
cudaError_t dalloc(pm_handle* h, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();   // an allocation failure must not surface later as a launch error
    return e;
  }
  h->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

bool supported_fft(int n) { return n == 16 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128; }
// The coarse mesh also takes the large sizes (row / column FFT passes).
bool supported_coarse(int n) { return supported_fft(n) || n == 192 || n == 256 || n == 384; }
bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int slot_of_rt(int N, int k) {
  // the same factorisation the device transforms use (fft.cuh)
  switch (N) {
    case 16: return pmfft::slot_of<16>(k);
    case 32: return pmfft::slot_of<32>(k);
    case 48: return pmfft::slot_of<48>(k);
    case 64: return pmfft::slot_of<64>(k);
    case 96: return pmfft::slot_of<96>(k);
    case 128: return pmfft::slot_of<128>(k);
    case 192: return pmfft::slot_of<192>(k);
    case 256: return pmfft::slot_of<256>(k);
    case 384: return pmfft::slot_of<384>(k);
  }
  return k;
}

int mode_number(int j, int n) { return j <= n / 2 ? j : j - n; }

// Periodic-mesh multiplier of i: a_d(k) = i [4 pi G k_d g(k) / (k^2 V)] M(k), k = 2 pi m / (N h),
// g = exp(-k^2 r_s^2) (long range) or 1; k_d -> 0 at the Nyquist index; 0 at k = 0.
std::vector<float> periodic_kernel(int N, double h, double G, double r_s) {
  const int NH = N / 2 + 1;
  std::vector<float> out((size_t)3 * N * N * NH);
  const double V = std::pow(N * h, 3);
  const double two_pi = 2.0 * pmfft::kPi;
  for (int kz = 0; kz < N; ++kz)
    for (int ky = 0; ky < N; ++ky)
      for (int kx = 0; kx < NH; ++kx) {
        int m[3] = {mode_number(kx, N), mode_number(ky, N), mode_number(kz, N)};
        double k[3], kg[3], k2 = 0;
        for (int d = 0; d < 3; ++d) {
          k[d] = two_pi * m[d] / (N * h);
          kg[d] = (2 * std::abs(m[d]) == N) ? 0.0 : k[d];
          k2 += k[d] * k[d];
        }
        double g = 0.0;
        if (k2 > 0) {
          g = 4.0 * pmfft::kPi * G / (k2 * V);
          if (r_s > 0) g *= std::exp(-k2 * r_s * r_s);
        }
        size_t idx = ((size_t)slot_of_rt(N, kz) * N + slot_of_rt(N, ky)) * NH + kx;
        for (int d = 0; d < 3; ++d) out[(size_t)d * N * N * NH + idx] = (float)(kg[d] * g);
      }
  return out;
}

// Fine tile multiplier of i: Im DFT_T[K_d] / T^3 with K_d(r) = -G r_d S(r) / r^3 (0 < r <= R),
// S(r) = erfc(r / 2 r_s) + r / (r_s sqrt(pi)) exp(-r^2 / 4 r_s^2).  K_d is odd along d and even
// along the other axes, so Im DFT = -sum K_d sin(2 pi n_d r_d / T) prod_{e != d} cos(2 pi n_e r_e / T),
// evaluated separably over the (2R+1)^3 support.
std::vector<float> tile_kernel(int T, double G, double r_s, double R) {
  const int NH = T / 2 + 1;
  const int Ri = (int)std::floor(R);
  const int W = 2 * Ri + 1;
  std::vector<float> out((size_t)3 * T * T * NH);
  std::vector<double> cs((size_t)T * W), sn((size_t)T * W);
  for (int n = 0; n < T; ++n)
    for (int j = -Ri; j <= Ri; ++j) {
      double a = 2.0 * pmfft::kPi * n * j / T;
      cs[(size_t)n * W + (j + Ri)] = std::cos(a);
      sn[(size_t)n * W + (j + Ri)] = std::sin(a);
    }
  std::vector<double> K((size_t)W * W * W);
  std::vector<double> A((size_t)W * W * T), B((size_t)W * T * T);
  for (int d = 0; d < 3; ++d) {
    for (int z = -Ri; z <= Ri; ++z)
      for (int y = -Ri; y <= Ri; ++y)
        for (int x = -Ri; x <= Ri; ++x) {
          double r = std::sqrt((double)x * x + (double)y * y + (double)z * z);
          double v = 0.0;
          if (r > 0 && r <= R) {
            double S = std::erfc(r / (2.0 * r_s)) + r / (r_s * std::sqrt(pmfft::kPi)) * std::exp(-r * r / (4.0 * r_s * r_s));
            double rd = d == 0 ? x : (d == 1 ? y : z);
            v = -G * rd * S / (r * r * r);
          }
          K[((size_t)(z + Ri) * W + (y + Ri)) * W + (x + Ri)] = v;
        }
    const std::vector<double>& fz = d == 2 ? sn : cs;
    const std::vector<double>& fy = d == 1 ? sn : cs;
    const std::vector<double>& fx = d == 0 ? sn : cs;
    // A[x][y][nz] = sum_z K[z][y][x] fz(nz, z)
    for (int x = 0; x < W; ++x)
      for (int y = 0; y < W; ++y)
        for (int nz = 0; nz < T; ++nz) {
          double s = 0;
          for (int z = 0; z < W; ++z) s += K[((size_t)z * W + y) * W + x] * fz[(size_t)nz * W + z];
          A[((size_t)x * W + y) * T + nz] = s;
        }
    // B[x][ny][nz] = sum_y A[x][y][nz] fy(ny, y)
    for (int x = 0; x < W; ++x)
      for (int ny = 0; ny < T; ++ny)
        for (int nz = 0; nz < T; ++nz) {
          double s = 0;
          for (int y = 0; y < W; ++y) s += A[((size_t)x * W + y) * T + nz] * fy[(size_t)ny * W + y];
          B[((size_t)x * T + ny) * T + nz] = s;
        }
    const double norm = 1.0 / ((double)T * T * T);
    for (int nz = 0; nz < T; ++nz)
      for (int ny = 0; ny < T; ++ny)
        for (int nx = 0; nx < NH; ++nx) {
          double s = 0;
          for (int x = 0; x < W; ++x) s += B[((size_t)x * T + ny) * T + nz] * fx[(size_t)nx * W + x];
          size_t idx = ((size_t)slot_of_rt(T, nz) * T + slot_of_rt(T, ny)) * NH + nx;
          out[(size_t)d * T * T * NH + idx] = (float)(-s * norm);
        }
  }
  return out;
}

std::vector<float2> twiddles(int N) {
  std::vector<float2> tw(N);
  for (int j = 0; j < N; ++j) {
    double a = 2.0 * pmfft::kPi * j / N;
    tw[j] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  return tw;
}

// Cell-block shapes for the fused passes.  Deposit: full x rows, one row per
// block unless the bins would not fit (small blocks keep many warps per SM).
// Interpolate/recompress: the force region staged per block must stay under
// about 100 KB so two 512-thread blocks share an SM.
Blk choose_blk(const Geom& g, bool fixed, bool deposit) {
  Blk b{};
  b.RX = g.ncmp;
  b.RY = b.RZ = 1;
  b.D = 2;
  Geo geo{g.nf, g.rc, g.nc, g.rcmp, g.ncmp, g.ncell(), g.two};
  if (!deposit) {
    while (b.RX > 1 && b.RX % 2 == 0 && ikd_count_smem(geo, b) > 100 * 1024) b.RX /= 2;
  } else {
    while (b.RX > 1 && b.RX % 2 == 0 && deposit_codes_smem(geo, b, fixed) > 64 * 1024) b.RX /= 2;
  }
  b.nbx = g.ncmp / b.RX;
  b.nby = g.ncmp / b.RY;
  b.nbz = g.ncmp / b.RZ;
  return b;
}

Geo to_geo(const Geom& g) { return Geo{g.nf, g.rc, g.nc, g.rcmp, g.ncmp, g.ncell(), g.two}; }

// Launch copies of the handle's cell-block shapes with their work counters.
Blk dep_blk(const pm_handle* h) {
  Blk b = h->blk_dep;
  b.work = h->persist_dep ? h->work : nullptr;
  b.brick = block_brick(b);
  return b;
}
Blk ikd_blk(const pm_handle* h, int pass) {
  Blk b = h->blk_ikd;
  b.work = h->persist_ikd ? h->work + 1 + pass : nullptr;
  b.brick = block_brick(b);
  return b;
}
cudaError_t zero_work(const pm_handle* h, cudaStream_t st) {
  if (!h->persist_dep && !h->persist_ikd) return cudaSuccess;
  return cudaMemsetAsync(h->work, 0, 4 * sizeof(int), st);
}

PCodes view(const pm_codes_t& c, bool vel16) {
  return PCodes{reinterpret_cast<const uint32_t*>(c.pos), c.vel, c.vmax, c.n, vel16};
}
PCodesOut oview(const pm_codes_t& c, bool vel16) {
  return PCodesOut{reinterpret_cast<uint32_t*>(c.pos), c.vel, c.vmax, vel16};
}

int check_species(pm_handle* h, int s) {
  if (s < 0 || s > 1) return fail(h, PM_ERR_ARG, "species must be 0 or 1");
  return PM_OK;
}

}  // namespace

// ---------------------------------------------------------------- Timer --
namespace pm {
static std::atomic<long long> g_launch_count{0};
void note_launches(int k) { g_launch_count.fetch_add(k, std::memory_order_relaxed); }

int Timer::kind(const char* name) {
  for (size_t i = 0; i < names.size(); ++i)
    if (names[i] == name) return (int)i;
  names.push_back(name);
  total_ms.push_back(0.0);
  count.push_back(0);
  return (int)names.size() - 1;
}
void Timer::begin(int, cudaStream_t st, cudaEvent_t* out) {
  cudaEvent_t e;
  if (!pool.empty()) { e = pool.back(); pool.pop_back(); }
  else cudaEventCreate(&e);
  cudaEventRecord(e, st);
  *out = e;
}
void Timer::end(int k, cudaStream_t st, cudaEvent_t start) {
  cudaEvent_t e;
  if (!pool.empty()) { e = pool.back(); pool.pop_back(); }
  else cudaEventCreate(&e);
  cudaEventRecord(e, st);
  pending.push_back({k, {start, e}});
}
void Timer::flush() {
  for (auto& p : pending) {
    cudaEventSynchronize(p.second.second);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    total_ms[p.first] += ms;
    count[p.first] += 1;
    pool.push_back(p.second.first);
    pool.push_back(p.second.second);
  }
  pending.clear();
}
void Timer::clear() {
  flush();
  for (auto& t : total_ms) t = 0.0;
  for (auto& c : count) c = 0;
}
}  // namespace pm

// ------------------------------------------------------------ entry points --
namespace pm {
cudaError_t launch_wait_probe(int* status, long long limit, cudaStream_t st);   // probe.cu
}

extern "C" {

int64_t pm_launch_count(void) { return (int64_t)pm::g_launch_count.load(); }

const char* pm_error_string(int code) {
  switch (code) {
    case PM_OK: return "ok";
    case PM_ERR_ARG: return "bad argument";
    case PM_ERR_CONFIG: return "unsupported configuration";
    case PM_ERR_CUDA: return "CUDA error";
    case PM_ERR_CORRUPT: return "corrupt compressed stream";
    case PM_ERR_OVERFLOW: return "capacity overflow";
    case PM_ERR_RANGE: return "position out of range";
    case PM_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown error";
  }
}

int pm_init(const pm_config_t* cfg, pm_handle_t** out) {
  if (!cfg || !out) return PM_ERR_ARG;
  *out = nullptr;
  pm_handle* h = new pm_handle();
  h->cfg = *cfg;
  Geom& g = h->gm;
  const pm_config_t& c = *cfg;
  auto bad = [&](const char* m) {
    std::string s = m;
    delete h;
    fprintf(stderr, "pm_init: %s\n", s.c_str());
    return PM_ERR_CONFIG;
  };
  if (c.n_fine <= 0 || c.cmp_ratio <= 0 || !pow2(c.cmp_ratio) || c.n_fine % c.cmp_ratio) return bad("cmp_ratio must be a power of two dividing n_fine");
  if (c.vel_bits != 8 && c.vel_bits != 16) return bad("vel_bits must be 8 or 16");
  if (c.deposit_mode != 0 && c.deposit_mode != 1) return bad("deposit_mode must be 0 or 1");
  if (c.vmax_mode != 0 && c.vmax_mode != 1) return bad("vmax_mode must be 0 or 1");
  if (c.pp != 0 && c.pp != 1) return bad("pp must be 0 or 1");
  if (c.pp && !(c.r_soft >= 0.0 && c.r_soft < 1.0)) return bad("r_soft must lie in [0, 1) fine cells");
  if (c.count[0] < 0 || c.count[1] < 0) return bad("negative particle count");
  g.nf = c.n_fine;
  g.rcmp = c.cmp_ratio;
  g.ncmp = c.n_fine / c.cmp_ratio;
  if ((int64_t)g.ncmp * g.ncmp * g.ncmp >= (int64_t)1 << 32) return bad("too many compression cells");
  if (c.coarse_ratio == 1) {
    g.two = false;
    g.rc = 1;
    g.nc = 0;
    g.t = g.nf;
    g.b = 0;
    g.T = g.nf;
    g.nts = 1;
    if (!supported_fft(g.nf)) return bad("single-mesh n_fine must be 16, 32, 48, 64, 96 or 128");
  } else {
    g.two = true;
    g.rc = c.coarse_ratio;
    if (c.coarse_ratio != c.cmp_ratio) return bad("two-level mode needs coarse_ratio == cmp_ratio");
    if (c.n_fine % c.coarse_ratio) return bad("coarse_ratio must divide n_fine");
    g.nc = c.n_fine / c.coarse_ratio;
    if (!supported_coarse(g.nc)) return bad("coarse mesh edge must be 16, 32, 48, 64, 96, 128, 192, 256 or 384");
    g.t = c.tile;
    g.b = c.buffer;
    g.T = c.tile + 2 * c.buffer;
    if (g.t <= 0 || g.b < 0 || g.nf % g.t || g.t % 2) return bad("tile must be even and divide n_fine");
    if (!supported_fft(g.T)) return bad("tile + 2 buffer must be 16, 32, 48, 64, 96 or 128");
    if (g.T > g.nf) return bad("tile edge exceeds the mesh");
    if (!(c.r_cut > 0) || c.r_cut > g.b - 2) return bad("r_cut must satisfy 0 < R <= buffer - 2");
    if (!(c.r_split > 0)) return bad("r_split must be positive");
    g.nts = g.nf / g.t;
  }
  if (!g.two && g.nf % 2) return bad("n_fine must be even");
  cudaGetDevice(&h->device);
  h->geo = to_geo(g);
  const bool fixed = c.deposit_mode == 1;
  int rc = PM_OK;
  auto A = [&](auto** p, size_t bytes) {
    if (rc != PM_OK) return;
    cudaError_t e = dalloc(h, p, bytes);
    if (e != cudaSuccess) rc = fail(h, PM_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  };
  const size_t nf3 = (size_t)g.nfine3(), nc3 = (size_t)g.ncoarse3();
  A(&h->rho_f, nf3 * 4);
  A(&h->acc_f, 3 * nf3 * 4);
  if (g.two) {
    A(&h->rho_c, nc3 * 4);
    A(&h->acc_c, 3 * nc3 * 4);
  }
  if (fixed) {
    A(&h->rho_f_fix, nf3 * 8);
    if (g.two) A(&h->rho_c_fix, nc3 * 8);
  }
  const size_t ncell = (size_t)g.ncell();
  for (int s = 0; s < 2; ++s) {
    A(&h->off[s], (ncell + 1) * 8);
    A(&h->newoff[s], (ncell + 1) * 8);
    A(&h->counts[s], ncell * 4);
  }
  A(&h->vmax_bits, 2 * 4);
  A(&h->amax, 3 * 4);
  if (c.pp) A(&h->app, (size_t)(c.count[0] + c.count[1]) * sizeof(float4));
  A(&h->work, 4 * 4);
  h->scratch_n = c.count[0] + c.count[1];
  A(&h->tkey, (size_t)h->scratch_n * 4);
  A(&h->tpv, (size_t)h->scratch_n * 16);
  A(&h->partial, 2 * scan_partial_bytes((int64_t)ncell));
  A(&h->status, 4);
  // plans and tables
  auto make_plan = [&](SolvePlan& p, int N, int nts, int t, int b, int src_n, int batch, const std::vector<float>& kern) {
    p.N = N;
    p.NH = N / 2 + 1;
    p.NP = spec_pitch(N);
    p.status = h->status;
    p.nts = nts;
    p.t = t;
    p.b = b;
    p.src_n = src_n;
    p.batch = batch;
    A(&p.kern, kern.size() * 4);
    A(&p.tw, (size_t)N * sizeof(float2));
    A(&p.spec, (size_t)batch * N * N * p.NP * sizeof(float2));
    A(&p.spec3, (size_t)batch * 3 * t * N * p.NP * sizeof(float2));
    if (rc != PM_OK) return;
    std::vector<float2> tw = twiddles(N);
    if (cudaMemcpy(p.kern, kern.data(), kern.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = fail(h, PM_ERR_CUDA, "kernel table upload failed");
  };
  if (g.two) {
    make_plan(h->plan_mesh, g.nc, 1, g.nc, 0, g.nc, 1, periodic_kernel(g.nc, (double)g.rc, c.G, c.r_split));
    int ntiles = g.ntiles();
    // Batches exist only to bound the spectrum workspace (about 11 MB per
    // 96^3 tile): all tiles in one launch per pass when that fits.
    int batch = c.tile_batch > 0 ? c.tile_batch : 1024;
    if (batch > ntiles) batch = ntiles;
    make_plan(h->plan_tiles, g.T, g.nts, g.t, g.b, g.nf, batch, tile_kernel(g.T, c.G, c.r_split, c.r_cut));
  } else {
    make_plan(h->plan_mesh, g.nf, 1, g.nf, 0, g.nf, 1, periodic_kernel(g.nf, 1.0, c.G, 0.0));
  }
  if (rc == PM_OK) {
    for (int s = 0; s < 2; ++s)
      if (cudaMemset(h->counts[s], 0, ncell * 4) != cudaSuccess) rc = fail(h, PM_ERR_CUDA, "memset");
    if (cudaMemset(h->status, 0, 4) != cudaSuccess) rc = fail(h, PM_ERR_CUDA, "memset");
    if (cudaDeviceSynchronize() != cudaSuccess) rc = fail(h, PM_ERR_CUDA, "init sync");
  }
  if (!g.two) {
    A(&h->lam_acc, 4 * nf3 * 4);
    A(&h->adj_spec, (size_t)3 * g.nf * g.nf * spec_pitch(g.nf) * sizeof(float2));
  }
  h->blk_dep = choose_blk(g, fixed, true);
  h->blk_ikd = choose_blk(g, fixed, false);
  h->tile_batch_alloc = g.two ? h->plan_tiles.batch : 1;
  {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    h->smem_optin = optin > 1024 ? (size_t)optin - 1024 : 0;   // room for the kernels' static shared memory
  }
  if (rc != PM_OK) {
    fprintf(stderr, "pm_init: %s\n", h->err.c_str());
    pm_destroy(h);
    return rc;
  }
  *out = h;
  return PM_OK;
}

int pm_destroy(pm_handle_t* h) {
  if (!h) return PM_ERR_ARG;
  cudaDeviceSynchronize();
  for (auto& g : h->step_graphs) cudaGraphExecDestroy(g.exec);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->pk_fork) cudaEventDestroy(h->pk_fork);
  if (h->pk_vel_ready) cudaEventDestroy(h->pk_vel_ready);
  if (h->d2h_stream) cudaStreamDestroy(h->d2h_stream);
  for (cudaEvent_t e : {h->as_in_free, h->as_pos_ready, h->as_vel_ready, h->as_packed, h->as_meta_done,
                        h->as_out_done})
    if (e) cudaEventDestroy(e);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  if (h->join_ev) cudaEventDestroy(h->join_ev);
  if (h->ckpt_stream) cudaStreamDestroy(h->ckpt_stream);
  if (h->ckpt_ready) cudaEventDestroy(h->ckpt_ready);
  if (h->ckpt_done) cudaEventDestroy(h->ckpt_done);
  h->timer.flush();
  for (auto e : h->timer.pool) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
  return PM_OK;
}

int pm_geometry(const pm_handle_t* h, int64_t* n_cmp, int64_t* n_coarse, int64_t* n_tiles, int64_t* tile_edge) {
  if (!h) return PM_ERR_ARG;
  if (n_cmp) *n_cmp = h->gm.ncmp;
  if (n_coarse) *n_coarse = h->gm.nc;
  if (n_tiles) *n_tiles = h->gm.two ? h->gm.ntiles() : 0;
  if (tile_edge) *tile_edge = h->gm.two ? h->gm.T : 0;
  return PM_OK;
}

int pm_decompress(pm_handle_t* h, int species, const pm_codes_t* in, float* x, float* v, void* stream) {
  if (!h || !in || (in->n > 0 && (!x || !v))) return fail(h, PM_ERR_ARG, "null argument");
  if (int r = check_species(h, species)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const bool vel16 = h->cfg.vel_bits == 16;
  CK(h, scan_codes(*in, h->gm.ncell(), h->off[species], h->partial, h->status, st));
  CK(h, launch_decompress(view(*in, vel16), h->off[species], h->geo, x, v, st));
  return PM_OK;
}

int pm_compress(pm_handle_t* h, int species, const float* x, const float* v, const float* vmax_in, pm_codes_t* out,
                void* stream) {
  if (!h || !out || !out->cnt || !out->vmax || !out->n_esc || !out->esc ||
      (out->n > 0 && (!x || !v || !out->pos || !out->vel)))
    return fail(h, PM_ERR_ARG, "null argument");
  if (int r = check_species(h, species)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  CK(h, cudaMemsetAsync(h->counts[species], 0, (size_t)h->gm.ncell() * 4, st));
  CK(h, launch_compress(x, v, out->n, h->geo, h->counts[species], h->vmax_bits + species, vmax_in,
                        h->newoff[species], *out, h->cfg.vel_bits == 16, h->partial, h->status, st));
  return PM_OK;
}

int pm_deposit(pm_handle_t* h, int species, const float* x, int64_t n, float* rho_coarse, float* rho_fine,
               void* stream) {
  if (!h || (!x && n) || !rho_fine || (h->gm.two && !rho_coarse)) return fail(h, PM_ERR_ARG, "null argument");
  if (int r = check_species(h, species)) return r;
  CK(h, launch_deposit(x, n, (float)h->cfg.mass[species], h->geo, h->gm.two ? rho_coarse : nullptr, rho_fine,
                       (cudaStream_t)stream));
  return PM_OK;
}

int pm_deposit_weights(pm_handle_t* h, const float* x, int64_t n, const float* w, int32_t nw, float* out,
                       void* stream) {
  if (!h || !out || (n && (!x || !w))) return fail(h, PM_ERR_ARG, "null argument");
  if (nw < 1 || nw > 4 || n < 0) return fail(h, PM_ERR_ARG, "nw must be 1..4, n >= 0");
  CK(h, launch_deposit_weights(x, n, w, nw, h->geo, out, (cudaStream_t)stream));
  return PM_OK;
}

int pm_deposit_fixed(pm_handle_t* h, int species, const float* x, int64_t n, int64_t* rho_coarse, int64_t* rho_fine,
                     void* stream) {
  if (!h || (!x && n) || !rho_fine || (h->gm.two && !rho_coarse)) return fail(h, PM_ERR_ARG, "null argument");
  if (int r = check_species(h, species)) return r;
  long long M = llrint(h->cfg.mass[species] * 4294967296.0);
  CK(h, launch_deposit_fixed(x, n, M, h->geo, h->gm.two ? (long long*)rho_coarse : nullptr, (long long*)rho_fine,
                             (cudaStream_t)stream));
  return PM_OK;
}

int pm_deposit_codes(pm_handle_t* h, const pm_codes_t in[2], void* rho_coarse, void* rho_fine, void* stream) {
  if (!h || !in || !rho_fine || (h->gm.two && !rho_coarse)) return fail(h, PM_ERR_ARG, "null argument");
  for (int s = 0; s < 2; ++s)
    if (!in[s].cnt || !in[s].vmax || !in[s].n_esc || !in[s].esc || (in[s].n > 0 && (!in[s].pos || !in[s].vel)))
      return fail(h, PM_ERR_ARG, "null codes pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const bool fixed = h->cfg.deposit_mode == 1;
  const bool vel16 = h->cfg.vel_bits == 16;
  CK(h, scan_codes2(in, h->gm.ncell(), h->off[0], h->off[1], h->partial, h->status, st));
  long long M0 = llrint(h->cfg.mass[0] * 4294967296.0), M1 = llrint(h->cfg.mass[1] * 4294967296.0);
  CK(h, zero_work(h, st));
  CK(h, launch_deposit_codes(view(in[0], vel16), view(in[1], vel16), h->off[0], h->off[1], h->geo, dep_blk(h),
                             (float)h->cfg.mass[0], (float)h->cfg.mass[1], M0, M1, h->gm.two ? rho_coarse : nullptr,
                             rho_fine, fixed, st));
  return PM_OK;
}

int pm_pp_accel(pm_handle_t* h, const pm_codes_t in[2], float* acc, void* stream) {
  if (!h || !in) return fail(h, PM_ERR_ARG, "null argument");
  for (int s = 0; s < 2; ++s)
    if (!in[s].cnt || !in[s].vmax || !in[s].n_esc || !in[s].esc || (in[s].n > 0 && (!in[s].pos || !in[s].vel)))
      return fail(h, PM_ERR_ARG, "null codes pointer");
  if (in[0].n + in[1].n > 0 && !acc) return fail(h, PM_ERR_ARG, "null acc");
  if ((reinterpret_cast<uintptr_t>(acc) & 15) != 0) return fail(h, PM_ERR_ARG, "acc must be 16-byte aligned");
  if (!(h->cfg.r_soft >= 0.0 && h->cfg.r_soft < 1.0)) return fail(h, PM_ERR_ARG, "r_soft must lie in [0, 1)");
  cudaStream_t st = (cudaStream_t)stream;
  const bool vel16 = h->cfg.vel_bits == 16;
  CK(h, scan_codes2(in, h->gm.ncell(), h->off[0], h->off[1], h->partial, h->status, st));
  CK(h, launch_pp(view(in[0], vel16), view(in[1], vel16), h->off[0], h->off[1], h->geo, (float)h->cfg.mass[0],
                  (float)h->cfg.mass[1], (float)h->cfg.G, (float)h->cfg.r_soft, reinterpret_cast<float4*>(acc), nullptr,
                  st));
  return PM_OK;
}

int pm_checkpoint_begin(pm_handle_t* h, const pm_codes_t codes[2], pm_host_codes_t host[2], void* stream) {
  if (!h || !codes || !host) return fail(h, PM_ERR_ARG, "null argument");
  if (h->ckpt_pending) return fail(h, PM_ERR_ARG, "a checkpoint is still pending: call pm_checkpoint_wait first");
  const bool vel16 = h->cfg.vel_bits == 16;
  const int64_t ncell = h->gm.ncell();
  for (int s = 0; s < 2; ++s) {
    const pm_codes_t& d = codes[s];
    const pm_host_codes_t& o = host[s];
    if (!d.cnt || !d.esc || !d.n_esc || !d.vmax || !o.cnt || !o.esc || !o.n_esc || !o.vmax ||
        (d.n > 0 && (!d.pos || !d.vel || !o.pos || !o.vel)))
      return fail(h, PM_ERR_ARG, "null codes pointer");
    if (o.n != d.n || o.esc_cap < d.esc_cap) return fail(h, PM_ERR_ARG, "host codes smaller than the device codes");
  }
  if (!h->ckpt_stream) {
    CK(h, cudaStreamCreateWithFlags(&h->ckpt_stream, cudaStreamNonBlocking));
    CK(h, cudaEventCreateWithFlags(&h->ckpt_ready, cudaEventDisableTiming));
    CK(h, cudaEventCreateWithFlags(&h->ckpt_done, cudaEventDisableTiming));
  }
  // the copies start once the caller's stream has produced the codes
  CK(h, cudaEventRecord(h->ckpt_ready, (cudaStream_t)stream));
  CK(h, cudaStreamWaitEvent(h->ckpt_stream, h->ckpt_ready, 0));
  cudaStream_t cs = h->ckpt_stream;
  for (int s = 0; s < 2; ++s) {
    const pm_codes_t& d = codes[s];
    pm_host_codes_t& o = host[s];
    CK(h, cudaMemcpyAsync(o.cnt, d.cnt, (size_t)ncell, cudaMemcpyDeviceToHost, cs));
    CK(h, cudaMemcpyAsync(o.esc, d.esc, (size_t)d.esc_cap * 8, cudaMemcpyDeviceToHost, cs));
    CK(h, cudaMemcpyAsync(o.n_esc, d.n_esc, 4, cudaMemcpyDeviceToHost, cs));
    CK(h, cudaMemcpyAsync(o.vmax, d.vmax, 4, cudaMemcpyDeviceToHost, cs));
    if (d.n > 0) {
      CK(h, cudaMemcpyAsync(o.pos, d.pos, (size_t)d.n * 4, cudaMemcpyDeviceToHost, cs));
      CK(h, cudaMemcpyAsync(o.vel, d.vel, (size_t)d.n * (vel16 ? 8 : 4), cudaMemcpyDeviceToHost, cs));
    }
  }
  CK(h, cudaEventRecord(h->ckpt_done, cs));
  h->ckpt_pending = true;
  return PM_OK;
}

int pm_checkpoint_fence(pm_handle_t* h, void* stream) {
  if (!h) return PM_ERR_ARG;
  if (!h->ckpt_pending) return PM_OK;
  CK(h, cudaStreamWaitEvent((cudaStream_t)stream, h->ckpt_done, 0));
  return PM_OK;
}

int pm_checkpoint_wait(pm_handle_t* h) {
  if (!h) return PM_ERR_ARG;
  if (!h->ckpt_pending) return PM_OK;
  h->ckpt_pending = false;
  CK(h, cudaEventSynchronize(h->ckpt_done));
  return PM_OK;
}

int pm_restrict(pm_handle_t* h, const float* rho_fine, float* rho_coarse, void* stream) {
  if (!h || !rho_fine || !rho_coarse) return fail(h, PM_ERR_ARG, "null argument");
  if (!h->gm.two) return fail(h, PM_ERR_CONFIG, "pm_restrict needs a two-level handle");
  CK(h, launch_restrict(rho_fine, h->gm.nf, h->gm.rc, rho_coarse, (cudaStream_t)stream));
  return PM_OK;
}

int pm_tile_density(pm_handle_t* h, const float* rho_fine, int64_t tile, float* out, void* stream) {
  if (!h || !rho_fine || !out) return fail(h, PM_ERR_ARG, "null argument");
  if (!h->gm.two || tile < 0 || tile >= h->gm.ntiles()) return fail(h, PM_ERR_ARG, "no such tile");
  CK(h, tile_window_launch(h->plan_tiles, rho_fine, tile, out, (cudaStream_t)stream));
  return PM_OK;
}

static int solve_impl(pm_handle_t* h, const void* rho_c, const void* rho_f, bool fixed, float* acc_c, float* acc_f,
                      cudaStream_t st, uint32_t* amax = nullptr, bool prolong = false) {
  Timer* tm = h->timer.on ? &h->timer : nullptr;
  if (h->gm.two && !tm) {
    // The coarse mesh (a few hundred blocks) and the tiles use separate plans,
    // inputs and outputs: solve the coarse mesh on the side stream meanwhile.
    if (!h->side_stream) {
      CK(h, cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
      CK(h, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
      CK(h, cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
    }
    CK(h, cudaEventRecord(h->fork_ev, st));
    CK(h, cudaStreamWaitEvent(h->side_stream, h->fork_ev, 0));
    CK(h, solve_launch(h->plan_mesh, rho_c, fixed, acc_c, h->side_stream, nullptr, amax));
    CK(h, cudaEventRecord(h->join_ev, h->side_stream));
    // with prolongation the tile solve's last pass waits for the coarse force
    const Prolong pro{acc_c, h->gm.nc, h->gm.rc, h->join_ev};
    CK(h, solve_launch(h->plan_tiles, rho_f, fixed, acc_f, st, nullptr, amax ? amax + 1 : nullptr,
                       prolong ? &pro : nullptr));
    CK(h, cudaStreamWaitEvent(st, h->join_ev, 0));
  } else if (h->gm.two) {
    {
      TimedScope ts(tm, "solve_coarse", st);
      CK(h, solve_launch(h->plan_mesh, rho_c, fixed, acc_c, st, nullptr, amax));
    }
    const Prolong pro{acc_c, h->gm.nc, h->gm.rc, nullptr};
    CK(h, solve_launch(h->plan_tiles, rho_f, fixed, acc_f, st, tm, amax ? amax + 1 : nullptr, prolong ? &pro : nullptr));
  } else {
    CK(h, solve_launch(h->plan_mesh, rho_f, fixed, acc_f, st, tm, amax ? amax + 1 : nullptr));
  }
  return PM_OK;
}

int pm_solve(pm_handle_t* h, const float* rho_coarse, const float* rho_fine, float* acc_coarse, float* acc_fine,
             void* stream) {
  if (!h || !rho_fine || !acc_fine || (h->gm.two && (!rho_coarse || !acc_coarse)))
    return fail(h, PM_ERR_ARG, "null argument");
  return solve_impl(h, rho_coarse, rho_fine, false, acc_coarse, acc_fine, (cudaStream_t)stream);
}

int pm_solve_fixed(pm_handle_t* h, const int64_t* rho_coarse, const int64_t* rho_fine, float* acc_coarse,
                   float* acc_fine, void* stream) {
  if (!h || !rho_fine || !acc_fine || (h->gm.two && (!rho_coarse || !acc_coarse)))
    return fail(h, PM_ERR_ARG, "null argument");
  return solve_impl(h, rho_coarse, rho_fine, true, acc_coarse, acc_fine, (cudaStream_t)stream);
}

int pm_interpolate(pm_handle_t* h, const float* x, int64_t n, const float* acc_coarse, const float* acc_fine, float* a,
                   void* stream) {
  if (!h || (n && (!x || !a)) || !acc_fine || (h->gm.two && !acc_coarse)) return fail(h, PM_ERR_ARG, "null argument");
  CK(h, launch_interpolate(x, n, h->geo, acc_coarse, acc_fine, a, (cudaStream_t)stream));
  return PM_OK;
}

int pm_kick_drift(pm_handle_t* h, float* x, float* v, int64_t n, const float* acc_coarse, const float* acc_fine,
                  double c_kick, double c_drift, void* stream) {
  if (!h || (n && (!x || !v)) || !acc_fine || (h->gm.two && !acc_coarse)) return fail(h, PM_ERR_ARG, "null argument");
  CK(h, launch_kick_drift(x, v, n, h->geo, acc_coarse, acc_fine, (float)c_kick, (float)c_drift, (cudaStream_t)stream));
  return PM_OK;
}

namespace {
int step_launch(pm_handle_t* h, const pm_codes_t in[2], pm_codes_t out[2], double c_kick, double c_drift,
                cudaStream_t st);

bool same_codes(const pm_codes_t& a, const pm_codes_t& b) { return memcmp(&a, &b, sizeof(pm_codes_t)) == 0; }

// Replays (capturing on first use) the step's launch sequence as one graph.
// Capture runs on a library stream, since the caller's stream may be the
// legacy default stream, which cannot be captured.
int packed_launch(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2], double c_kick,
                  double c_drift, cudaStream_t st);

int step_graph(pm_handle_t* h, const pm_codes_t in[2], pm_codes_t out[2], double c_kick, double c_drift,
               cudaStream_t st, int kind = 0) {
  for (auto& g : h->step_graphs) {
    if (g.kind == kind && g.ck == c_kick && g.cd == c_drift && same_codes(g.in[0], in[0]) &&
        same_codes(g.in[1], in[1]) && same_codes(g.out[0], out[0]) && same_codes(g.out[1], out[1])) {
      CK(h, cudaGraphLaunch(g.exec, st));
      note_launches((int)g.launches);
      return PM_OK;
    }
  }
  if (!h->capture_stream) CK(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
  const long long before = pm_launch_count();
  CK(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
  const int r = kind == 0 ? step_launch(h, in, out, c_kick, c_drift, h->capture_stream)
                          : packed_launch(h, in, out, c_kick, c_drift, h->capture_stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(h->capture_stream, &graph);
  const long long captured = pm_launch_count() - before;
  note_launches((int)-captured);   // captured launches run only when the graph is launched
  if (r != PM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (ec != cudaSuccess) return fail(h, PM_ERR_CUDA, std::string("step capture: ") + cudaGetErrorString(ec));
  pm_handle::StepGraph g{};
  g.kind = kind;
  for (int s = 0; s < 2; ++s) {
    g.in[s] = in[s];
    g.out[s] = out[s];
  }
  g.ck = c_kick;
  g.cd = c_drift;
  g.launches = captured;
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return fail(h, PM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
  if (h->step_graphs.size() >= 8) {
    cudaGraphExecDestroy(h->step_graphs.front().exec);
    h->step_graphs.erase(h->step_graphs.begin());
  }
  h->step_graphs.push_back(g);
  CK(h, cudaGraphLaunch(g.exec, st));
  note_launches((int)captured);
  return PM_OK;
}
}  // namespace

int pm_set_graphs(pm_handle_t* h, int on) {
  if (!h) return PM_ERR_ARG;
  h->graphs = on != 0;
  if (!h->graphs) {
    cudaDeviceSynchronize();
    for (auto& g : h->step_graphs) cudaGraphExecDestroy(g.exec);
    h->step_graphs.clear();
  }
  return PM_OK;
}

namespace {
// A cell-block shape is usable when it tiles the compression mesh and its
// shared memory fits one block of this device.
bool blk_fits(const pm_handle* h, const Blk& b, bool deposit) {
  const int n = h->gm.ncmp;
  if (b.RX < 1 || b.RY < 1 || b.RZ < 1 || n % b.RX || n % b.RY || n % b.RZ) return false;
  if (b.D < 1 || b.D > 4) return false;
  if (deposit) return deposit_codes_smem(h->geo, b, h->cfg.deposit_mode == 1) <= h->smem_optin;
  return ikd_count_smem(h->geo, b) <= h->smem_optin && ikd_scatter_smem(h->geo, b) <= h->smem_optin;
}

Blk make_blk(const pm_handle* h, const int32_t r[3], int D) {
  Blk b{};
  b.RX = r[0];
  b.RY = r[1];
  b.RZ = r[2];
  b.D = D;
  if (b.RX > 0 && b.RY > 0 && b.RZ > 0) {
    b.nbx = h->gm.ncmp / b.RX;
    b.nby = h->gm.ncmp / b.RY;
    b.nbz = h->gm.ncmp / b.RZ;
  }
  return b;
}

void drop_graphs(pm_handle* h) {
  if (h->step_graphs.empty()) return;
  cudaDeviceSynchronize();
  for (auto& g : h->step_graphs) cudaGraphExecDestroy(g.exec);
  h->step_graphs.clear();
}

int apply_tuning(pm_handle* h, const pm_tuning_t* t) {
  const Blk bd = make_blk(h, t->deposit_block, 2);
  const Blk bi = make_blk(h, t->kick_block, t->kick_window);
  if (!blk_fits(h, bd, true)) return fail(h, PM_ERR_ARG, "deposit_block does not tile the mesh or exceeds shared memory");
  if (!blk_fits(h, bi, false)) return fail(h, PM_ERR_ARG, "kick_block/kick_window invalid or exceeds shared memory");
  if (t->tile_batch < 1 || t->tile_batch > h->tile_batch_alloc)
    return fail(h, PM_ERR_ARG, "tile_batch must lie in [1, the configured tile batch]");
  if ((t->deposit_persistent & ~1) || (t->kick_persistent & ~1)) return fail(h, PM_ERR_ARG, "persistent flags are 0 or 1");
  drop_graphs(h);
  h->blk_dep = bd;
  h->blk_ikd = bi;
  h->persist_dep = t->deposit_persistent != 0;
  h->persist_ikd = t->kick_persistent != 0;
  if (h->gm.two) h->plan_tiles.batch = t->tile_batch;
  return PM_OK;
}
}  // namespace

int pm_get_tuning(const pm_handle_t* h, pm_tuning_t* t) {
  if (!h || !t) return PM_ERR_ARG;
  t->deposit_block[0] = h->blk_dep.RX;
  t->deposit_block[1] = h->blk_dep.RY;
  t->deposit_block[2] = h->blk_dep.RZ;
  t->deposit_persistent = h->persist_dep ? 1 : 0;
  t->kick_block[0] = h->blk_ikd.RX;
  t->kick_block[1] = h->blk_ikd.RY;
  t->kick_block[2] = h->blk_ikd.RZ;
  t->kick_window = h->blk_ikd.D;
  t->kick_persistent = h->persist_ikd ? 1 : 0;
  t->tile_batch = h->gm.two ? h->plan_tiles.batch : 1;
  return PM_OK;
}

int pm_set_tuning(pm_handle_t* h, const pm_tuning_t* t) {
  if (!h || !t) return fail(h, PM_ERR_ARG, "null argument");
  return apply_tuning(h, t);
}

int pm_autotune(pm_handle_t* h, const pm_codes_t in[2], pm_codes_t out[2], double c_kick, double c_drift, int32_t reps,
                void* stream, pm_tuning_t* chosen) {
  if (!h || !in || !out) return fail(h, PM_ERR_ARG, "null argument");
  if (reps < 1 || reps > 1000) return fail(h, PM_ERR_ARG, "reps must lie in [1, 1000]");
  cudaStream_t st = (cudaStream_t)stream;
  const bool timing = h->timer.on, graphs = h->graphs;
  h->timer.on = false;
  h->graphs = false;
  pm_tuning_t best{};
  pm_get_tuning(h, &best);
  const pm_tuning_t start = best;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PM_OK;
  float best_ms = 0.f;
  auto restore = [&](int code) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    h->timer.on = timing;
    h->graphs = graphs;
    return code;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return restore(fail(h, PM_ERR_CUDA, "event create"));
  // mean step time of a tuning: one untimed step, then reps steps between events
  auto time_of = [&](const pm_tuning_t& t, float* ms) -> int {
    if (int r = apply_tuning(h, &t)) return r;
    if (int r = step_launch(h, in, out, c_kick, c_drift, st)) return r;
    if (cudaEventRecord(e0, st) != cudaSuccess) return fail(h, PM_ERR_CUDA, "event record");
    for (int i = 0; i < reps; ++i)
      if (int r = step_launch(h, in, out, c_kick, c_drift, st)) return r;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return fail(h, PM_ERR_CUDA, "event timing");
    *ms /= (float)reps;
    return PM_OK;
  };
  if ((rc = time_of(best, &best_ms))) {
    apply_tuning(h, &start);
    return restore(rc);
  }
  auto consider = [&](const pm_tuning_t& t) -> int {
    const Blk bd = make_blk(h, t.deposit_block, 2), bi = make_blk(h, t.kick_block, t.kick_window);
    if (!blk_fits(h, bd, true) || !blk_fits(h, bi, false)) return PM_OK;   // not a candidate on this mesh
    float ms = 0.f;
    if (int r = time_of(t, &ms)) return r;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
    return PM_OK;
  };
  const int n = h->gm.ncmp;
  const int rx[4] = {n, n / 2, n / 4, n / 8};
  const int ry[3] = {1, 2, 4}, rz[2] = {1, 2};
  // coordinate search: deposit block and launch form, then the kick passes'
  // block, window and launch form, then the tile batch
  for (int pass = 0; pass < 2 && rc == PM_OK; ++pass)
    for (int a = 0; a < 4 && rc == PM_OK; ++a)
      for (int b = 0; b < 3 && rc == PM_OK; ++b)
        for (int c = 0; c < 2 && rc == PM_OK; ++c)
          for (int p = 0; p < 2 && rc == PM_OK; ++p)
            for (int D = (pass ? 1 : 2); D <= 2 && rc == PM_OK; ++D) {
              if (rx[a] < 1) continue;
              pm_tuning_t t = best;
              int32_t* blk = pass ? t.kick_block : t.deposit_block;
              blk[0] = rx[a];
              blk[1] = ry[b];
              blk[2] = rz[c];
              if (pass) {
                t.kick_persistent = p;
                t.kick_window = D;
              } else {
                t.deposit_persistent = p;
              }
              rc = consider(t);
            }
  for (int k = 1; k <= 4 && rc == PM_OK; k *= 2) {
    pm_tuning_t t = best;
    t.tile_batch = h->tile_batch_alloc / k > 0 ? h->tile_batch_alloc / k : 1;
    rc = consider(t);
  }
  if (rc != PM_OK) {
    apply_tuning(h, &start);
    return restore(rc);
  }
  apply_tuning(h, &best);
  if (chosen) *chosen = best;
  return restore(PM_OK);
}

int pm_step(pm_handle_t* h, const pm_codes_t in[2], pm_codes_t out[2], double c_kick, double c_drift, void* stream) {
  if (!h || !in || !out) return fail(h, PM_ERR_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (h->graphs && !h->timer.on) return step_graph(h, in, out, c_kick, c_drift, st);
  return step_launch(h, in, out, c_kick, c_drift, st);
}

namespace {
int step_launch(pm_handle_t* h, const pm_codes_t in[2], pm_codes_t out[2], double c_kick, double c_drift,
                cudaStream_t st) {
  for (int s = 0; s < 2; ++s) {
    if (in[s].n != out[s].n) return fail(h, PM_ERR_ARG, "out[s].n must equal in[s].n");
    if (!in[s].cnt || !in[s].vmax || !in[s].n_esc || !in[s].esc || !out[s].cnt || !out[s].vmax || !out[s].n_esc ||
        !out[s].esc || (in[s].n > 0 && (!in[s].pos || !in[s].vel || !out[s].pos || !out[s].vel)))
      return fail(h, PM_ERR_ARG, "null codes pointer");
    if (in[s].n > 0 && in[s].pos == out[s].pos) return fail(h, PM_ERR_ARG, "in and out codes must not alias");
  }
  if (in[0].n + in[1].n > h->scratch_n)
    return fail(h, PM_ERR_ARG, "particle counts exceed the pm_config_t counts the handle was sized for");
  Timer* tm = h->timer.on ? &h->timer : nullptr;
  const Geom& g = h->gm;
  const bool fixed = h->cfg.deposit_mode == 1;
  const bool vel16 = h->cfg.vel_bits == 16;
  const int64_t ncell = g.ncell();
  {
    TimedScope ts(tm, "scan_in", st);
    CK(h, scan_codes2(in, ncell, h->off[0], h->off[1], h->partial, h->status, st));
  }
  void* rc = fixed ? (void*)h->rho_c_fix : (void*)h->rho_c;
  void* rf = fixed ? (void*)h->rho_f_fix : (void*)h->rho_f;
  // Float two-level step: the coarse mesh comes from the fine one (CIC
  // restriction, exact for CIC), and the coarse force is prolongated onto the
  // fine force mesh as the tile solve writes it, so the particle passes touch
  // only the fine meshes.  The fixed-point mode keeps the direct integer coarse
  // deposit and gathers both meshes (bit-reproducible against the plain calls).
  const bool via_fine = g.two && !fixed;
  {
    TimedScope ts(tm, "deposit", st);
    CK(h, cudaMemsetAsync(rf, 0, (size_t)g.nfine3() * (fixed ? 8 : 4), st));
    if (g.two) CK(h, cudaMemsetAsync(rc, 0, (size_t)g.ncoarse3() * (fixed ? 8 : 4), st));
    long long M0 = llrint(h->cfg.mass[0] * 4294967296.0), M1 = llrint(h->cfg.mass[1] * 4294967296.0);
    CK(h, zero_work(h, st));
    // (float: the coarse density is restricted from each block's fine tile as it flushes)
    CK(h, launch_deposit_codes(view(in[0], vel16), view(in[1], vel16), h->off[0], h->off[1], h->geo, dep_blk(h),
                               (float)h->cfg.mass[0], (float)h->cfg.mass[1], M0, M1, g.two ? rc : nullptr, rf, fixed,
                               st));
  }
  const bool bound = h->cfg.vmax_mode == 1;
  const float ck = (float)c_kick, cd = (float)c_drift;
  if (bound) CK(h, cudaMemsetAsync(h->amax, 0, 12, st));
  if (int r = solve_impl(h, rc, rf, fixed, h->acc_c, h->acc_f, st, bound ? h->amax : nullptr, via_fine)) return r;
  if (h->cfg.pp) {
    TimedScope ts(tm, "pp", st);
    CK(h, launch_pp(view(in[0], vel16), view(in[1], vel16), h->off[0], h->off[1], h->geo, (float)h->cfg.mass[0],
                    (float)h->cfg.mass[1], (float)h->cfg.G, (float)h->cfg.r_soft, h->app, bound ? h->amax + 2 : nullptr,
                    st));
  }
  if (h->pre_count_wait) CK(h, cudaStreamWaitEvent(st, h->pre_count_wait, 0));   // packed step: velocities in
  if (h->pre_count_wait2) CK(h, cudaStreamWaitEvent(st, h->pre_count_wait2, 0)); // async: previous output copied
  // bound mode: v_max' from the mesh maxima, before any particle is kicked
  if (bound) CK(h, launch_vmax_bound(in[0].vmax, in[1].vmax, h->amax, ck, out[0].vmax, out[1].vmax, st));
  {
    TimedScope ts(tm, "ikd_count", st);
    if (!bound) CK(h, cudaMemsetAsync(h->vmax_bits, 0, 8, st));
    for (int s = 0; s < 2; ++s) CK(h, cudaMemsetAsync(h->counts[s], 0, (size_t)ncell * 4, st));
    CK(h, launch_ikd_count(view(in[0], vel16), view(in[1], vel16), h->off[0], h->off[1], h->geo, ikd_blk(h, 0),
                           h->acc_c, h->acc_f, ck, cd, h->counts[0], h->counts[1], h->vmax_bits, h->tkey, h->tpv,
                           bound ? out[0].vmax : nullptr, bound ? out[1].vmax : nullptr, h->cfg.pp ? h->app : nullptr,
                           !via_fine, st));
  }
  if (h->post_count_record) CK(h, cudaEventRecord(h->post_count_record, st));
  {
    TimedScope ts(tm, "scan_out", st);
    if (!bound) CK(h, launch_set_vmax2(h->vmax_bits, out[0].vmax, out[1].vmax, st));
    const int64_t expect[2] = {in[0].n, in[1].n};
    CK(h, scan_counts2(h->counts[0], h->counts[1], ncell, expect, h->newoff[0], h->newoff[1], out, h->partial,
                       h->status, st));
  }
  {
    TimedScope ts(tm, "ikd_scatter", st);
    PCodesOut o0 = oview(out[0], vel16), o1 = oview(out[1], vel16);
    CK(h, launch_ikd_scatter(in[0].n, in[1].n, h->off[0], h->off[1], h->geo, ikd_blk(h, 1), h->counts[0], h->counts[1],
                             h->newoff[0], h->newoff[1], o0, o1, h->tkey, h->tpv, bound, h->status, st));
  }
  return PM_OK;
}
}  // namespace

int pm_deposit_adjoint(pm_handle_t* h, int species, const float* x, int64_t n, const float* lam_rho, float* lam_x,
                       void* stream) {
  if (!h || (n && (!x || !lam_x)) || !lam_rho) return fail(h, PM_ERR_ARG, "null argument");
  if (int r = check_species(h, species)) return r;
  if (h->gm.two) return fail(h, PM_ERR_CONFIG, "adjoints are implemented for the single periodic mesh");
  CK(h, launch_adj_deposit(x, n, (float)h->cfg.mass[species], h->gm.nf, lam_rho, lam_x, (cudaStream_t)stream));
  return PM_OK;
}

int pm_solve_adjoint(pm_handle_t* h, const float* lam_acc, float* lam_rho, void* stream) {
  if (!h || !lam_acc || !lam_rho) return fail(h, PM_ERR_ARG, "null argument");
  if (h->gm.two) return fail(h, PM_ERR_CONFIG, "adjoints are implemented for the single periodic mesh");
  CK(h, solve_adjoint_launch(h->plan_mesh, lam_acc, false, lam_rho, h->adj_spec, (cudaStream_t)stream));
  return PM_OK;
}

int pm_interpolate_adjoint(pm_handle_t* h, const float* x, int64_t n, const float* acc_fine, double c_kick,
                           double c_drift, float* lam_x, float* lam_v, float* lam_acc, void* stream) {
  if (!h || (n && (!x || !lam_x || !lam_v)) || !acc_fine || !lam_acc) return fail(h, PM_ERR_ARG, "null argument");
  if (h->gm.two) return fail(h, PM_ERR_CONFIG, "adjoints are implemented for the single periodic mesh");
  CK(h, launch_adj_interp(x, n, h->gm.nf, acc_fine, (float)c_kick, (float)c_drift, lam_x, lam_v, lam_acc, false,
                          (cudaStream_t)stream));
  return PM_OK;
}

// The reverse step given the step's acceleration mesh acc [3][n^3] at the pre-step positions.
static int step_adjoint_core(pm_handle_t* h, const pm_particles_t state[2], pm_particles_t lam[2], const float* acc,
                             double c_kick, double c_drift, cudaStream_t st) {
  const Geom& g = h->gm;
  const size_t nf3 = (size_t)g.nfine3();
  // interleaved float4 accumulation mesh: one vector reduction per CIC corner
  CK(h, cudaMemsetAsync(h->lam_acc, 0, 4 * nf3 * 4, st));
  for (int s = 0; s < 2; ++s)
    CK(h, launch_adj_interp(state[s].x, state[s].n, g.nf, acc, (float)c_kick, (float)c_drift, lam[s].x, lam[s].v,
                            h->lam_acc, true, st));
  CK(h, solve_adjoint_launch(h->plan_mesh, h->lam_acc, true, h->rho_f, h->adj_spec, st));   // rho_f holds lam_rho
  for (int s = 0; s < 2; ++s)
    CK(h, launch_adj_deposit(state[s].x, state[s].n, (float)h->cfg.mass[s], g.nf, h->rho_f, lam[s].x, st));
  return PM_OK;
}

static int check_adjoint_args(pm_handle_t* h, const pm_particles_t state[2], pm_particles_t lam[2]) {
  if (!h || !state || !lam) return fail(h, PM_ERR_ARG, "null argument");
  if (h->gm.two) return fail(h, PM_ERR_CONFIG, "adjoints are implemented for the single periodic mesh");
  for (int s = 0; s < 2; ++s)
    if (state[s].n != lam[s].n || (state[s].n && (!state[s].x || !lam[s].x || !lam[s].v)))
      return fail(h, PM_ERR_ARG, "state and adjoint particle arrays disagree");
  return PM_OK;
}

int pm_step_adjoint(pm_handle_t* h, const pm_particles_t state[2], pm_particles_t lam[2], double c_kick,
                    double c_drift, void* stream) {
  if (int rc = check_adjoint_args(h, state, lam)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const bool fixed = h->cfg.deposit_mode == 1;
  const size_t nf3 = (size_t)h->gm.nfine3();
  // recompute the step's acceleration mesh at the pre-step positions
  if (fixed) {
    CK(h, cudaMemsetAsync(h->rho_f_fix, 0, nf3 * 8, st));
    for (int s = 0; s < 2; ++s) {
      long long M = llrint(h->cfg.mass[s] * 4294967296.0);
      CK(h, launch_deposit_fixed(state[s].x, state[s].n, M, h->geo, nullptr, h->rho_f_fix, st));
    }
    CK(h, solve_launch(h->plan_mesh, h->rho_f_fix, true, h->acc_f, st, nullptr));
  } else {
    CK(h, cudaMemsetAsync(h->rho_f, 0, nf3 * 4, st));
    for (int s = 0; s < 2; ++s)
      CK(h, launch_deposit(state[s].x, state[s].n, (float)h->cfg.mass[s], h->geo, nullptr, h->rho_f, st));
    CK(h, solve_launch(h->plan_mesh, h->rho_f, false, h->acc_f, st, nullptr));
  }
  return step_adjoint_core(h, state, lam, h->acc_f, c_kick, c_drift, st);
}

int pm_step_adjoint_acc(pm_handle_t* h, const pm_particles_t state[2], pm_particles_t lam[2], const float* acc_fine,
                        double c_kick, double c_drift, void* stream) {
  if (int rc = check_adjoint_args(h, state, lam)) return rc;
  if (!acc_fine) return fail(h, PM_ERR_ARG, "null acceleration mesh");
  return step_adjoint_core(h, state, lam, acc_fine, c_kick, c_drift, (cudaStream_t)stream);
}

static int alloc_codes(pm_handle* h, pm_codes_t& c, int64_t n, int64_t esc_cap) {
  const int vb = h->cfg.vel_bits == 16 ? 2 : 1;
  const size_t ncell = (size_t)h->gm.ncell();
  c.n = n;
  c.esc_cap = esc_cap;
  CK(h, dalloc(h, &c.cnt, ncell));
  CK(h, dalloc(h, &c.esc, (size_t)(esc_cap > 0 ? esc_cap : 1) * 8));
  CK(h, dalloc(h, &c.n_esc, 4));
  CK(h, dalloc(h, &c.pos, (size_t)n * 4));
  void* v = nullptr;
  CK(h, dalloc(h, &v, (size_t)n * 4 * vb));
  c.vel = v;
  CK(h, dalloc(h, &c.vmax, 4));
  return PM_OK;
}

static int copy_codes(pm_handle* h, const pm_codes_t& dst, const pm_codes_t& src, int64_t ncell, int vb,
                      cudaMemcpyKind kind, cudaStream_t st, bool include_esc_all) {
  CK(h, cudaMemcpyAsync(dst.cnt, src.cnt, (size_t)ncell, kind, st));
  CK(h, cudaMemcpyAsync(dst.n_esc, src.n_esc, 4, kind, st));
  int64_t ecap = src.esc_cap < dst.esc_cap ? src.esc_cap : dst.esc_cap;
  if (include_esc_all && ecap > 0) CK(h, cudaMemcpyAsync(dst.esc, src.esc, (size_t)ecap * 8, kind, st));
  CK(h, cudaMemcpyAsync(dst.pos, src.pos, (size_t)src.n * 4, kind, st));
  CK(h, cudaMemcpyAsync(dst.vel, src.vel, (size_t)src.n * 4 * vb, kind, st));
  CK(h, cudaMemcpyAsync(dst.vmax, src.vmax, 4, kind, st));
  return PM_OK;
}

namespace {
bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// Counts, escape list and v_max are the same in both forms.
int copy_meta(pm_handle* h, const pm_codes_t& dst, const pm_codes_t& src, int64_t ncell, cudaMemcpyKind kind,
              cudaStream_t st) {
  CK(h, cudaMemcpyAsync(dst.cnt, src.cnt, (size_t)ncell, kind, st));
  CK(h, cudaMemcpyAsync(dst.n_esc, src.n_esc, 4, kind, st));
  const int64_t ecap = src.esc_cap < dst.esc_cap ? src.esc_cap : dst.esc_cap;
  if (ecap > 0) CK(h, cudaMemcpyAsync(dst.esc, src.esc, (size_t)ecap * 8, kind, st));
  CK(h, cudaMemcpyAsync(dst.vmax, src.vmax, 4, kind, st));
  return PM_OK;
}
}  // namespace

int pm_pack_codes(pm_handle_t* h, const pm_codes_t* in, pm_codes_t* out, void* stream) {
  if (!h || !in || !out) return fail(h, PM_ERR_ARG, "null argument");
  const bool vel16 = h->cfg.vel_bits == 16;
  if (in->n != out->n || out->esc_cap < in->esc_cap) return fail(h, PM_ERR_ARG, "out must hold in's particles and escapes");
  if (in->n > 0 && (!aligned(in->pos, 16) || !aligned(in->vel, 16) || !aligned(out->pos, 4) ||
                    !aligned(out->vel, vel16 ? 8 : 4)))
    return fail(h, PM_ERR_ARG, "pos/vel alignment: padded 16 B, packed 4 B (8 B for 16-bit velocities)");
  cudaStream_t st = (cudaStream_t)stream;
  if (int r = copy_meta(h, *out, *in, h->gm.ncell(), cudaMemcpyDeviceToDevice, st)) return r;
  CK(h, launch_pack(reinterpret_cast<const uint32_t*>(in->pos), in->vel, vel16, in->n,
                    reinterpret_cast<uint8_t*>(out->pos), reinterpret_cast<uint8_t*>(out->vel), st));
  return PM_OK;
}

int pm_unpack_codes(pm_handle_t* h, const pm_codes_t* in, pm_codes_t* out, void* stream) {
  if (!h || !in || !out) return fail(h, PM_ERR_ARG, "null argument");
  const bool vel16 = h->cfg.vel_bits == 16;
  if (in->n != out->n || out->esc_cap < in->esc_cap) return fail(h, PM_ERR_ARG, "out must hold in's particles and escapes");
  if (in->n > 0 && (!aligned(out->pos, 16) || !aligned(out->vel, 16) || !aligned(in->pos, 4) ||
                    !aligned(in->vel, vel16 ? 8 : 4)))
    return fail(h, PM_ERR_ARG, "pos/vel alignment: padded 16 B, packed 4 B (8 B for 16-bit velocities)");
  cudaStream_t st = (cudaStream_t)stream;
  if (int r = copy_meta(h, *out, *in, h->gm.ncell(), cudaMemcpyDeviceToDevice, st)) return r;
  CK(h, launch_unpack(reinterpret_cast<const uint8_t*>(in->pos), reinterpret_cast<const uint8_t*>(in->vel), vel16,
                      in->n, reinterpret_cast<uint32_t*>(out->pos), out->vel, st));
  return PM_OK;
}

namespace {
// Enqueues one packed step: counts, escapes, v_max and position bytes on st,
// unpacked there; velocity bytes on the copy stream (forked from st), needed
// only by the count pass; the step; then pack and device -> host copies.
int packed_launch(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2], double c_kick,
                  double c_drift, cudaStream_t st) {
  const bool vel16 = h->cfg.vel_bits == 16;
  const int64_t ncell = h->gm.ncell();
  const size_t vbytes = vel16 ? 6 : 3;
  for (int s = 0; s < 2; ++s) {
    const int64_t n = in[s].n;
    if (int r = copy_meta(h, h->stage_in[s], in[s], ncell, cudaMemcpyHostToDevice, st)) return r;
    if (n > 0) CK(h, cudaMemcpyAsync(h->pk_pos[0][s], in[s].pos, (size_t)n * 3, cudaMemcpyHostToDevice, st));
    CK(h, launch_unpack(h->pk_pos[0][s], nullptr, vel16, n, reinterpret_cast<uint32_t*>(h->stage_in[s].pos), nullptr,
                        st));
  }
  CK(h, cudaEventRecord(h->pk_fork, st));
  CK(h, cudaStreamWaitEvent(h->copy_stream, h->pk_fork, 0));
  for (int s = 0; s < 2; ++s) {
    const int64_t n = in[s].n;
    if (n > 0)
      CK(h, cudaMemcpyAsync(h->pk_vel[0][s], in[s].vel, (size_t)n * vbytes, cudaMemcpyHostToDevice, h->copy_stream));
    CK(h, launch_unpack(nullptr, h->pk_vel[0][s], vel16, n, nullptr, h->stage_in[s].vel, h->copy_stream));
  }
  CK(h, cudaEventRecord(h->pk_vel_ready, h->copy_stream));
  h->pre_count_wait = h->pk_vel_ready;
  const int r = step_launch(h, h->stage_in, h->stage_out, c_kick, c_drift, st);
  h->pre_count_wait = nullptr;
  if (r != PM_OK) return r;
  for (int s = 0; s < 2; ++s) {
    const int64_t n = in[s].n;
    CK(h, launch_pack(reinterpret_cast<const uint32_t*>(h->stage_out[s].pos), h->stage_out[s].vel, vel16, n,
                      h->pk_pos[1][s], h->pk_vel[1][s], st));
    if (int r2 = copy_meta(h, out[s], h->stage_out[s], ncell, cudaMemcpyDeviceToHost, st)) return r2;
    if (n > 0) {
      CK(h, cudaMemcpyAsync(out[s].pos, h->pk_pos[1][s], (size_t)n * 3, cudaMemcpyDeviceToHost, st));
      CK(h, cudaMemcpyAsync(out[s].vel, h->pk_vel[1][s], (size_t)n * vbytes, cudaMemcpyDeviceToHost, st));
    }
  }
  return PM_OK;
}
}  // namespace

namespace {
int packed_setup(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2]);
}

int pm_step_packed(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2], double c_kick,
                   double c_drift, void* stream) {
  if (!h || !in || !out) return fail(h, PM_ERR_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (int r = packed_setup(h, in, out)) return r;
  const int r = (h->graphs && !h->timer.on) ? step_graph(h, in, out, c_kick, c_drift, st, 1)
                                            : packed_launch(h, in, out, c_kick, c_drift, st);
  if (r != PM_OK) return r;
  return pm_check(h, stream);
}

int pm_step_packed_async(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2], double c_kick,
                         double c_drift, void* stream) {
  if (!h || !in || !out) return fail(h, PM_ERR_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (int r = packed_setup(h, in, out)) return r;
  const bool vel16 = h->cfg.vel_bits == 16;
  const int64_t ncell = h->gm.ncell();
  const size_t vbytes = vel16 ? 6 : 3;
  if (!h->as_ready) {
    for (int s = 0; s < 2; ++s) {
      const size_t n = (size_t)h->stage_in[s].n;
      CK(h, dalloc(h, &h->as_pos[s], 3 * n + 16));
      CK(h, dalloc(h, &h->as_vel[s], vbytes * n + 16));
    }
    // separate packed output buffers when they fit with 2 GB to spare
    // (otherwise the output shares the step scratch)
    size_t need = 0, free_b = 0, total_b = 0;
    for (int s = 0; s < 2; ++s) need += (3 + vbytes) * (size_t)h->stage_in[s].n + 512;
    CK(h, cudaMemGetInfo(&free_b, &total_b));
    h->as_sep = free_b > need + ((size_t)2 << 30);
    for (int s = 0; s < 2 && h->as_sep; ++s) {
      const size_t n = (size_t)h->stage_in[s].n;
      CK(h, dalloc(h, &h->as_opos[s], 3 * n + 16));
      CK(h, dalloc(h, &h->as_ovel[s], vbytes * n + 16));
    }
    CK(h, cudaStreamCreateWithFlags(&h->d2h_stream, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&h->as_in_free, &h->as_pos_ready, &h->as_vel_ready, &h->as_packed, &h->as_meta_done,
                           &h->as_out_done})
      CK(h, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    CK(h, cudaEventRecord(h->as_in_free, st));
    CK(h, cudaEventRecord(h->as_meta_done, h->d2h_stream));
    CK(h, cudaEventRecord(h->as_out_done, h->d2h_stream));
    h->as_ready = true;
  }
  uint8_t* const* opos = h->as_sep ? h->as_opos : h->pk_pos[1];
  uint8_t* const* ovel = h->as_sep ? h->as_ovel : h->pk_vel[1];
  // Position records into the packed staging, which the previous call's
  // unpacking (earlier on the same stream) has finished reading, so they run
  // beside the previous step; then, once that step's count pass has read its
  // input, counts, escapes, v_max and the unpacked positions (the deposit
  // needs no more); then the velocity records, which only the count pass
  // needs (they run beside the previous scatter and this deposit and solve).
  for (int s = 0; s < 2; ++s) {
    const int64_t n = in[s].n;
    if (n > 0) CK(h, cudaMemcpyAsync(h->as_pos[s], in[s].pos, (size_t)n * 3, cudaMemcpyHostToDevice, h->copy_stream));
  }
  CK(h, cudaStreamWaitEvent(h->copy_stream, h->as_in_free, 0));
  for (int s = 0; s < 2; ++s) {
    if (int r = copy_meta(h, h->stage_in[s], in[s], ncell, cudaMemcpyHostToDevice, h->copy_stream)) return r;
    CK(h, launch_unpack(h->as_pos[s], nullptr, vel16, in[s].n, reinterpret_cast<uint32_t*>(h->stage_in[s].pos),
                        nullptr, h->copy_stream));
  }
  CK(h, cudaEventRecord(h->as_pos_ready, h->copy_stream));
  for (int s = 0; s < 2; ++s) {
    const int64_t n = in[s].n;
    if (n > 0)
      CK(h, cudaMemcpyAsync(h->as_vel[s], in[s].vel, (size_t)n * vbytes, cudaMemcpyHostToDevice, h->copy_stream));
    CK(h, launch_unpack(nullptr, h->as_vel[s], vel16, n, nullptr, h->stage_in[s].vel, h->copy_stream));
  }
  CK(h, cudaEventRecord(h->as_vel_ready, h->copy_stream));
  // the step: positions first; velocities, and the previous step's output
  // copies out of what this step overwrites, before the count pass (its
  // counts and v_max always; its packed records too when they share the
  // step scratch)
  CK(h, cudaStreamWaitEvent(st, h->as_pos_ready, 0));
  h->pre_count_wait = h->as_vel_ready;
  h->pre_count_wait2 = h->as_sep ? h->as_meta_done : h->as_out_done;
  h->post_count_record = h->as_in_free;
  const int r = step_launch(h, h->stage_in, h->stage_out, c_kick, c_drift, st);
  h->pre_count_wait = h->pre_count_wait2 = h->post_count_record = nullptr;
  if (r != PM_OK) return r;
  if (h->as_sep) CK(h, cudaStreamWaitEvent(st, h->as_out_done, 0));   // previous packed output copied out
  for (int s = 0; s < 2; ++s)
    CK(h, launch_pack(reinterpret_cast<const uint32_t*>(h->stage_out[s].pos), h->stage_out[s].vel, vel16,
                      in[s].n, opos[s], ovel[s], st));
  CK(h, cudaEventRecord(h->as_packed, st));
  // output copies: counts, escapes and v_max first (the next step rewrites them)
  CK(h, cudaStreamWaitEvent(h->d2h_stream, h->as_packed, 0));
  for (int s = 0; s < 2; ++s)
    if (int r2 = copy_meta(h, out[s], h->stage_out[s], ncell, cudaMemcpyDeviceToHost, h->d2h_stream)) return r2;
  CK(h, cudaEventRecord(h->as_meta_done, h->d2h_stream));
  for (int s = 0; s < 2; ++s) {
    const int64_t n = in[s].n;
    if (n > 0) {
      CK(h, cudaMemcpyAsync(out[s].pos, opos[s], (size_t)n * 3, cudaMemcpyDeviceToHost, h->d2h_stream));
      CK(h, cudaMemcpyAsync(out[s].vel, ovel[s], (size_t)n * vbytes, cudaMemcpyDeviceToHost, h->d2h_stream));
    }
  }
  CK(h, cudaEventRecord(h->as_out_done, h->d2h_stream));
  return PM_OK;
}

namespace {
// Checks and first-use allocations shared by the packed steps: staging codes,
// packed buffers (in and out share the step scratch), copy stream and events.
int packed_setup(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2]) {
  const bool vel16 = h->cfg.vel_bits == 16;
  for (int s = 0; s < 2; ++s) {
    if (out[s].n != in[s].n) return fail(h, PM_ERR_ARG, "out[s].n must equal in[s].n");
    if (!in[s].cnt || !in[s].esc || !in[s].n_esc || !in[s].vmax || !out[s].cnt || !out[s].esc || !out[s].n_esc ||
        !out[s].vmax || (in[s].n > 0 && (!in[s].pos || !in[s].vel || !out[s].pos || !out[s].vel)))
      return fail(h, PM_ERR_ARG, "null codes pointer");
  }
  if (!h->staged) {
    for (int s = 0; s < 2; ++s) {
      int64_t cap = in[s].esc_cap > out[s].esc_cap ? in[s].esc_cap : out[s].esc_cap;
      if (int r = alloc_codes(h, h->stage_in[s], in[s].n, cap)) return r;
      if (int r = alloc_codes(h, h->stage_out[s], in[s].n, cap)) return r;
    }
    h->staged = true;
  }
  if (!h->pk_staged) {
    // The packed input bytes are dead once the count pass starts (positions
    // are unpacked before the deposit, velocities before the count pass,
    // which waits for them), and the packed output is written after the
    // scatter has read the step's scratch for the last time.  So input and
    // output share one set of buffers, carved from the per-particle scratch
    // when it is large enough (it is 16 B per particle, the records 9 B at
    // most): a packed step then needs no device memory beyond the padded
    // staging codes.
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t need = 0;
    for (int s = 0; s < 2; ++s) {
      const size_t n = (size_t)h->stage_in[s].n;
      need += up(3 * n + 16) + up(3 * n * (vel16 ? 2 : 1) + 16);
    }
    uint8_t* carve = reinterpret_cast<uint8_t*>(h->tpv);
    if (need <= (size_t)h->scratch_n * sizeof(uint4)) {
      for (int s = 0; s < 2; ++s) {
        const size_t n = (size_t)h->stage_in[s].n;
        h->pk_pos[0][s] = h->pk_pos[1][s] = carve;
        carve += up(3 * n + 16);
        h->pk_vel[0][s] = h->pk_vel[1][s] = carve;
        carve += up(3 * n * (vel16 ? 2 : 1) + 16);
      }
    } else {
      for (int s = 0; s < 2; ++s) {
        const size_t n = (size_t)h->stage_in[s].n;
        CK(h, dalloc(h, &h->pk_pos[0][s], 3 * n + 16));
        CK(h, dalloc(h, &h->pk_vel[0][s], 3 * n * (vel16 ? 2 : 1) + 16));
        h->pk_pos[1][s] = h->pk_pos[0][s];
        h->pk_vel[1][s] = h->pk_vel[0][s];
      }
    }
    h->pk_staged = true;
  }
  if (!h->copy_stream) {
    CK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    CK(h, cudaEventCreateWithFlags(&h->pk_fork, cudaEventDisableTiming));
    CK(h, cudaEventCreateWithFlags(&h->pk_vel_ready, cudaEventDisableTiming));
  }
  for (int s = 0; s < 2; ++s) {
    if (h->stage_in[s].n != in[s].n) return fail(h, PM_ERR_ARG, "particle counts changed");
    if (in[s].esc_cap > h->stage_in[s].esc_cap)
      return fail(h, PM_ERR_ARG, "input escape capacity larger than at the first call");
  }
  return PM_OK;
}
}  // namespace

int pm_step_host(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2], double c_kick, double c_drift,
                 void* stream) {
  if (!h || !in || !out) return fail(h, PM_ERR_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int vb = h->cfg.vel_bits == 16 ? 2 : 1;
  const int64_t ncell = h->gm.ncell();
  if (!h->staged) {
    for (int s = 0; s < 2; ++s) {
      int64_t cap = in[s].esc_cap > out[s].esc_cap ? in[s].esc_cap : out[s].esc_cap;
      if (int r = alloc_codes(h, h->stage_in[s], in[s].n, cap)) return r;
      if (int r = alloc_codes(h, h->stage_out[s], in[s].n, cap)) return r;
    }
    h->staged = true;
  }
  for (int s = 0; s < 2; ++s)
    if (h->stage_in[s].n != in[s].n || out[s].n != in[s].n) return fail(h, PM_ERR_ARG, "particle counts changed");
  for (int s = 0; s < 2; ++s)
    if (int r = copy_codes(h, h->stage_in[s], in[s], ncell, vb, cudaMemcpyHostToDevice, st, true)) return r;
  if (int r = pm_step(h, h->stage_in, h->stage_out, c_kick, c_drift, stream)) return r;
  for (int s = 0; s < 2; ++s)
    if (int r = copy_codes(h, out[s], h->stage_out[s], ncell, vb, cudaMemcpyDeviceToHost, st, true)) return r;
  return pm_check(h, stream);
}

int pm_check(pm_handle_t* h, void* stream) {
  if (!h) return PM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(h, cudaStreamSynchronize(st));
  if (h->d2h_stream) CK(h, cudaStreamSynchronize(h->d2h_stream));   // copies queued by pm_step_packed_async
  if (h->copy_stream) CK(h, cudaStreamSynchronize(h->copy_stream));
  int s = 0;
  CK(h, cudaMemcpy(&s, h->status, 4, cudaMemcpyDeviceToHost));
  CK(h, cudaMemset(h->status, 0, 4));
  if (s & ST_RANGE) return fail(h, PM_ERR_RANGE, "device validation: position outside [0, n_fine)");
  if (s & ST_OVERFLOW) return fail(h, PM_ERR_OVERFLOW, "device validation: escape list capacity exceeded");
  if (s & ST_CORRUPT) return fail(h, PM_ERR_CORRUPT, "device validation: corrupt compressed stream");
  if (s & ST_TIMEOUT) return fail(h, PM_ERR_TIMEOUT, "device wait timed out");
  return PM_OK;
}

int pm_wait_probe(pm_handle_t* h, int64_t limit_cycles, void* stream) {
  if (!h) return PM_ERR_ARG;
  if (limit_cycles < 1000 || limit_cycles > 2000000000LL) return fail(h, PM_ERR_ARG, "limit_cycles outside [1e3, 2e9]");
  CK(h, launch_wait_probe(h->status, (long long)limit_cycles, (cudaStream_t)stream));
  note_launches(1);
  return PM_OK;
}

int pm_last_error(const pm_handle_t* h, char* buf, size_t n) {
  if (!h || !buf || n == 0) return PM_ERR_ARG;
  snprintf(buf, n, "%s", h->err.c_str());
  return PM_OK;
}

int pm_set_timing(pm_handle_t* h, int on) {
  if (!h) return PM_ERR_ARG;
  h->timer.clear();
  h->timer.on = on != 0;
  return PM_OK;
}

int pm_stage_times(pm_handle_t* h, float* ms, int cap, int* n_stages, char* names, size_t names_cap) {
  if (!h) return PM_ERR_ARG;
  h->timer.flush();
  int n = (int)h->timer.names.size();
  if (n_stages) *n_stages = n;
  std::string joined;
  for (int i = 0; i < n; ++i) {
    if (ms && i < cap) ms[i] = h->timer.count[i] ? (float)(h->timer.total_ms[i] / h->timer.count[i]) : 0.f;
    if (i) joined += ";";
    joined += h->timer.names[i];
    joined += "#" + std::to_string(h->timer.count[i]);
  }
  if (names && names_cap) snprintf(names, names_cap, "%s", joined.c_str());
  return PM_OK;
}

int pm_serialize(const pm_host_codes_t* c, int32_t n_cmp, int32_t vel_bits, uint8_t* buf, size_t cap, size_t* len) {
  if (!c || !len || (vel_bits != 8 && vel_bits != 16) || n_cmp <= 0) return PM_ERR_ARG;
  const int64_t ncell = (int64_t)n_cmp * n_cmp * n_cmp;
  const int vb = vel_bits == 16 ? 2 : 1;
  const uint32_t ne = c->n_esc ? *c->n_esc : 0;
  // size
  size_t total = 32;
  uint32_t ei = 0;
  int64_t np = 0;
  std::vector<int64_t> counts((size_t)ncell);
  for (int64_t cell = 0; cell < ncell; ++cell) {
    int64_t k = c->cnt[cell];
    if (k == 255) {
      if (ei >= ne || c->esc[2 * ei] != (uint32_t)cell) return PM_ERR_CORRUPT;
      k = c->esc[2 * ei + 1];
      ++ei;
      total += 5;
    } else {
      total += 1;
    }
    counts[(size_t)cell] = k;
    np += k;
  }
  if (np != c->n || ei != ne) return PM_ERR_CORRUPT;
  total += (size_t)np * (3 + 3 * vb);
  *len = total;
  if (!buf) return PM_OK;
  if (cap < total) return PM_ERR_OVERFLOW;
  uint8_t* o = buf;
  const uint32_t ver = 1, ncu = (uint32_t)n_cmp, vbits = (uint32_t)vel_bits, zero = 0;
  const uint64_t n64 = (uint64_t)c->n;
  const float vm = *c->vmax;
  memcpy(o, "PMNU", 4); o += 4;
  memcpy(o, &ver, 4); o += 4;
  memcpy(o, &ncu, 4); o += 4;
  memcpy(o, &vbits, 4); o += 4;
  memcpy(o, &n64, 8); o += 8;
  memcpy(o, &vm, 4); o += 4;
  memcpy(o, &zero, 4); o += 4;
  int64_t p = 0;
  for (int64_t cell = 0; cell < ncell; ++cell) {
    int64_t k = counts[(size_t)cell];
    if (k >= 255) {
      *o++ = 255;
      int32_t k32 = (int32_t)k;
      memcpy(o, &k32, 4);
      o += 4;
    } else {
      *o++ = (uint8_t)k;
    }
    for (int64_t j = 0; j < k; ++j, ++p) {
      memcpy(o, c->pos + 4 * p, 3);
      o += 3;
      for (int d = 0; d < 3; ++d) {
        if (vb == 2) {
          uint16_t q = static_cast<const uint16_t*>(c->vel)[4 * p + d];
          o[0] = (uint8_t)(q & 0xff);
          o[1] = (uint8_t)(q >> 8);
          o += 2;
        } else {
          *o++ = static_cast<const uint8_t*>(c->vel)[4 * p + d];
        }
      }
    }
  }
  return PM_OK;
}

int pm_deserialize(const uint8_t* buf, size_t len, int32_t n_cmp, int32_t vel_bits, pm_host_codes_t* c) {
  if (!buf || !c || len < 32) return PM_ERR_ARG;
  if (memcmp(buf, "PMNU", 4) != 0) return PM_ERR_CORRUPT;
  uint32_t ver, ncu, vbits;
  uint64_t n64;
  float vm;
  memcpy(&ver, buf + 4, 4);
  memcpy(&ncu, buf + 8, 4);
  memcpy(&vbits, buf + 12, 4);
  memcpy(&n64, buf + 16, 8);
  memcpy(&vm, buf + 24, 4);
  if (ver != 1 || (int32_t)ncu != n_cmp || (int32_t)vbits != vel_bits) return PM_ERR_CORRUPT;
  if ((int64_t)n64 != c->n) return PM_ERR_ARG;
  const int vb = vel_bits == 16 ? 2 : 1;
  const int64_t ncell = (int64_t)n_cmp * n_cmp * n_cmp;
  size_t off = 32;
  int64_t p = 0;
  uint32_t ne = 0;
  for (int64_t cell = 0; cell < ncell; ++cell) {
    if (off >= len) return PM_ERR_CORRUPT;
    int64_t k = buf[off++];
    c->cnt[cell] = (uint8_t)k;
    if (k == 255) {
      if (off + 4 > len) return PM_ERR_CORRUPT;
      int32_t k32;
      memcpy(&k32, buf + off, 4);
      off += 4;
      if (k32 < 255) return PM_ERR_CORRUPT;
      if ((int64_t)ne >= c->esc_cap) return PM_ERR_OVERFLOW;
      c->esc[2 * ne] = (uint32_t)cell;
      c->esc[2 * ne + 1] = (uint32_t)k32;
      ++ne;
      k = k32;
    }
    if (p + k > c->n) return PM_ERR_CORRUPT;
    size_t rec = (size_t)(3 + 3 * vb);
    if (off + (size_t)k * rec > len) return PM_ERR_CORRUPT;
    for (int64_t j = 0; j < k; ++j, ++p) {
      memcpy(c->pos + 4 * p, buf + off, 3);
      c->pos[4 * p + 3] = 0;
      off += 3;
      for (int d = 0; d < 3; ++d) {
        if (vb == 2) {
          static_cast<uint16_t*>(c->vel)[4 * p + d] = (uint16_t)(buf[off] | (buf[off + 1] << 8));
          off += 2;
        } else {
          static_cast<uint8_t*>(c->vel)[4 * p + d] = buf[off++];
        }
      }
      if (vb == 2) static_cast<uint16_t*>(c->vel)[4 * p + 3] = 0;
      else static_cast<uint8_t*>(c->vel)[4 * p + 3] = 0;
    }
  }
  if (off != len || p != c->n) return PM_ERR_CORRUPT;
  if (c->n_esc) *c->n_esc = ne;
  if (c->vmax) *c->vmax = vm;
  return PM_OK;
}

}  // extern "C"
