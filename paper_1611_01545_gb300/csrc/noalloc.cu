// Decompression without any device allocation.
//
// pm_decompress needs a handle, and pm_init allocates the handle's workspace
// with cudaMalloc.  Some callers cannot allow that: an application that owns
// the device's whole memory budget and hands libraries only the buffers they
// are given, or a host thread that must not pay the device-wide
// synchronisation that cudaMalloc / cudaFree can cause.  pm_decompress_noalloc
// serves them: its only scratch (the per-cell CSR offsets, the scan partials
// and a status word) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads the library keeps until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "particles.cuh"
#include "pm_common.cuh"

namespace {

constexpr int64_t kMaxCells = (int64_t)64 * 64 * 64;   // n_cmp <= 64
constexpr size_t kOffBytes = (size_t)(kMaxCells + 1) * sizeof(int64_t);
constexpr size_t kPartialOffset = (kOffBytes + 255) / 256 * 256;
constexpr size_t kPartialBytes = 4096;                  // >= pm::scan_partial_bytes(kMaxCells)
constexpr size_t kStatusOffset = kPartialOffset + kPartialBytes;
constexpr size_t kScratchBytes = kStatusOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code may not use the symbol itself as a device pointer).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int pm_decompress_noalloc(int32_t n_fine, int32_t cmp_ratio, int32_t vel_bits, const pm_codes_t* in,
                                     float* x, float* v, void* stream) {
  if (!in || (in->n > 0 && (!x || !v || !in->pos || !in->vel)) || !in->cnt || !in->esc || !in->n_esc ||
      !in->vmax)
    return PM_ERR_ARG;
  if (vel_bits != 8 && vel_bits != 16) return PM_ERR_ARG;
  if (n_fine <= 0 || cmp_ratio <= 0 || (cmp_ratio & (cmp_ratio - 1)) || n_fine % cmp_ratio) return PM_ERR_ARG;
  const int ncmp = n_fine / cmp_ratio;
  const int64_t ncell = (int64_t)ncmp * ncmp * ncmp;
  if (ncell > kMaxCells || pm::scan_partial_bytes(ncell) > kPartialBytes) return PM_ERR_ARG;
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return PM_ERR_CUDA;
  int64_t* off = reinterpret_cast<int64_t*>(base);
  void* partial = base + kPartialOffset;
  int* status = reinterpret_cast<int*>(base + kStatusOffset);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return PM_ERR_CUDA;
  pm::Geo g{n_fine, 1, 0, cmp_ratio, ncmp, ncell, false};
  if (pm::scan_codes(*in, ncell, off, partial, status, st) != cudaSuccess) return PM_ERR_CUDA;
  pm::PCodes view{reinterpret_cast<const uint32_t*>(in->pos), in->vel, in->vmax, in->n, vel_bits == 16};
  if (pm::launch_decompress(view, off, g, x, v, st) != cudaSuccess) return PM_ERR_CUDA;
  int host_status = 0;
  if (cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PM_ERR_CUDA;
  if (host_status & pm::ST_CORRUPT) return PM_ERR_CORRUPT;
  return PM_OK;
}
