// Packed codes: the Sec. 2.4 record fields without the in-memory padding.
//
// In device memory every particle's position codes occupy one 4-byte word
// (px, py, pz, 0) and its velocity codes one 4-byte (8-bit codes) or 8-byte
// (16-bit codes, little-endian u16 each) word, so that decode and placement
// are one aligned access per particle.  The packed form keeps exactly the
// record bytes: pos u8[n][3] and vel u8[n][3] or u16[n][3] (little-endian),
// i.e. 6 or 9 bytes per particle instead of 8 or 12 -- the form to move over
// the host link.  A thread packs or unpacks four consecutive particles at a
// time (12 / 24 byte groups, word aligned); the last, incomplete group is
// done byte by byte.  Unpacking takes positions only (pvel null) or
// velocities only (ppos null) when asked.
#include <cuda_runtime.h>
#include <stdint.h>

#include "particles.cuh"
#include "pm_common.cuh"

namespace pm {

namespace {

constexpr unsigned long long kM48 = 0xFFFFFFFFFFFFull;

__global__ void k_pack(const uint32_t* pos, const void* vel, int vel16, int64_t n, uint8_t* ppos, uint8_t* pvel) {
  const int64_t ngroups = n / 4;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g <= ngroups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = 4 * g;
    if (g < ngroups) {
      const uint4 w = *reinterpret_cast<const uint4*>(pos + p);
      uint32_t* o = reinterpret_cast<uint32_t*>(ppos + 3 * p);
      o[0] = (w.x & 0xFFFFFFu) | (w.y << 24);
      o[1] = ((w.y >> 8) & 0xFFFFu) | (w.z << 16);
      o[2] = ((w.z >> 16) & 0xFFu) | ((w.w & 0xFFFFFFu) << 8);
      if (vel16) {
        const unsigned long long* v = reinterpret_cast<const unsigned long long*>(vel) + p;
        const unsigned long long v0 = v[0] & kM48, v1 = v[1] & kM48, v2 = v[2] & kM48, v3 = v[3] & kM48;
        unsigned long long* q = reinterpret_cast<unsigned long long*>(pvel + 6 * p);
        q[0] = v0 | (v1 << 48);
        q[1] = (v1 >> 16) | (v2 << 32);
        q[2] = (v2 >> 32) | (v3 << 16);
      } else {
        const uint4 u = *reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(vel) + p);
        uint32_t* q = reinterpret_cast<uint32_t*>(pvel + 3 * p);
        q[0] = (u.x & 0xFFFFFFu) | (u.y << 24);
        q[1] = ((u.y >> 8) & 0xFFFFu) | (u.z << 16);
        q[2] = ((u.z >> 16) & 0xFFu) | ((u.w & 0xFFFFFFu) << 8);
      }
    } else {
      for (int64_t i = p; i < n; ++i) {
        const uint32_t w = pos[i];
        for (int b = 0; b < 3; ++b) ppos[3 * i + b] = (uint8_t)(w >> (8 * b));
        if (vel16) {
          const unsigned long long v = reinterpret_cast<const unsigned long long*>(vel)[i];
          for (int b = 0; b < 6; ++b) pvel[6 * i + b] = (uint8_t)(v >> (8 * b));
        } else {
          const uint32_t u = reinterpret_cast<const uint32_t*>(vel)[i];
          for (int b = 0; b < 3; ++b) pvel[3 * i + b] = (uint8_t)(u >> (8 * b));
        }
      }
    }
  }
}

__global__ void k_unpack(const uint8_t* ppos, const uint8_t* pvel, int vel16, int64_t n, uint32_t* pos, void* vel) {
  const int64_t ngroups = n / 4;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g <= ngroups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = 4 * g;
    if (g < ngroups) {
      if (ppos) {
        const uint32_t* i = reinterpret_cast<const uint32_t*>(ppos + 3 * p);
        const uint32_t i0 = i[0], i1 = i[1], i2 = i[2];
        *reinterpret_cast<uint4*>(pos + p) =
            make_uint4(i0 & 0xFFFFFFu, (i0 >> 24) | ((i1 & 0xFFFFu) << 8), (i1 >> 16) | ((i2 & 0xFFu) << 16), i2 >> 8);
      }
      if (!pvel) {
      } else if (vel16) {
        const unsigned long long* q = reinterpret_cast<const unsigned long long*>(pvel + 6 * p);
        const unsigned long long o0 = q[0], o1 = q[1], o2 = q[2];
        unsigned long long* v = reinterpret_cast<unsigned long long*>(vel) + p;
        v[0] = o0 & kM48;
        v[1] = (o0 >> 48) | ((o1 & 0xFFFFFFFFull) << 16);
        v[2] = (o1 >> 32) | ((o2 & 0xFFFFull) << 32);
        v[3] = o2 >> 16;
      } else {
        const uint32_t* q = reinterpret_cast<const uint32_t*>(pvel + 3 * p);
        const uint32_t u0 = q[0], u1 = q[1], u2 = q[2];
        *reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(vel) + p) =
            make_uint4(u0 & 0xFFFFFFu, (u0 >> 24) | ((u1 & 0xFFFFu) << 8), (u1 >> 16) | ((u2 & 0xFFu) << 16), u2 >> 8);
      }
    } else {
      for (int64_t k = p; k < n; ++k) {
        if (ppos) {
          uint32_t w = 0;
          for (int b = 0; b < 3; ++b) w |= (uint32_t)ppos[3 * k + b] << (8 * b);
          pos[k] = w;
        }
        if (!pvel) {
        } else if (vel16) {
          unsigned long long v = 0;
          for (int b = 0; b < 6; ++b) v |= (unsigned long long)pvel[6 * k + b] << (8 * b);
          reinterpret_cast<unsigned long long*>(vel)[k] = v;
        } else {
          uint32_t u = 0;
          for (int b = 0; b < 3; ++b) u |= (uint32_t)pvel[3 * k + b] << (8 * b);
          reinterpret_cast<uint32_t*>(vel)[k] = u;
        }
      }
    }
  }
}

int pack_grid(int64_t n) {
  int64_t b = (n / 4 + 1 + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_pack(const uint32_t* pos, const void* vel, bool vel16, int64_t n, uint8_t* ppos, uint8_t* pvel,
                        cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_pack<<<pack_grid(n), 256, 0, st>>>(pos, vel, vel16 ? 1 : 0, n, ppos, pvel);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint8_t* ppos, const uint8_t* pvel, bool vel16, int64_t n, uint32_t* pos, void* vel,
                          cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_unpack<<<pack_grid(n), 256, 0, st>>>(ppos, pvel, vel16 ? 1 : 0, n, pos, vel);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace pm
