// gc_device.cuh -- device-side helpers shared by the decode, index and
// encode kernels of the Group-codec library (arXiv 1502.01916).
//
// Layout facts used everywhere (Sec 2.1.2, Sec 3.1; k = 4 is the paper's
// 4-way vertical layout, k = 32 is the same rule with 32 lanes):
//   - int i of a list is lane i % k of row i / k;
//   - lane j's data bit t is bit t % 32 of word (t / 32) * k + j;
//   - control bit t is bit t % 8 of byte t / 8.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gc.h"

namespace gcdev {

constexpr int kTileInts = 1024;  // ints per decoding tile (one warp)
constexpr uint32_t kPfdFrameRows = 32;
constexpr unsigned kFull = 0xffffffffu;

// Table III, one 6-bit field per selector: BW and NUM (NUM * BW <= 32).
constexpr uint64_t pack6(const int (&v)[10]) {
  uint64_t r = 0;
  for (int i = 0; i < 10; ++i) r |= (uint64_t)v[i] << (6 * i);
  return r;
}
constexpr int kSelBw[10] = {1, 2, 3, 4, 5, 6, 8, 10, 16, 32};
constexpr int kSelNum[10] = {32, 16, 10, 8, 6, 5, 4, 3, 2, 1};
constexpr uint64_t kBwPack = pack6(kSelBw);
constexpr uint64_t kNumPack = pack6(kSelNum);

__device__ __forceinline__ uint32_t sel_bw(uint32_t s) { return (uint32_t)(kBwPack >> (6 * s)) & 63u; }
__device__ __forceinline__ uint32_t sel_num(uint32_t s) { return (uint32_t)(kNumPack >> (6 * s)) & 63u; }

__host__ __device__ __forceinline__ uint64_t min64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t low_mask(uint32_t w) { return w >= 32 ? 0xffffffffu : ((1u << w) - 1u); }

// Effective bit width (Sec 2.1.2): 0 for 0.
__device__ __forceinline__ uint32_t eff_bits(uint32_t x) { return 32u - (uint32_t)__clz(x); }

__device__ __forceinline__ uint32_t log2_cg(uint32_t cg) { return cg == 1 ? 0u : cg == 2 ? 1u : cg == 4 ? 2u : 3u; }

// Binary length descriptors are aligned (Sec 5.2.1(b)): 3 per 16 bits at
// CG 1, 2 per byte at CG 2 and 4, 4 per byte at CG 8.
__device__ __forceinline__ uint64_t bin_ld_pos(uint64_t r, uint32_t cg) {
  switch (cg) {
    case 1: return (r / 3) * 16 + (r % 3) * 5;
    case 2: return (r >> 1) * 8 + (r & 1) * 4;
    case 4: return (r >> 1) * 8 + (r & 1) * 3;
    default: return (r >> 2) * 8 + (r & 3) * 2;
  }
}
__host__ __device__ __forceinline__ uint64_t bin_ld_bytes(uint64_t R, uint32_t cg) {
  return cg == 1 ? 2 * ((R + 2) / 3) : cg == 8 ? (R + 3) / 4 : (R + 1) / 2;
}

// ------------------------------------------------------------ warp scans

template <class T>
__device__ __forceinline__ T warp_incl_sum(T v) {
  const uint32_t l = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, v, o);
    if (l >= (uint32_t)o) v += y;
  }
  return v;
}

template <class T>
__device__ __forceinline__ T warp_incl_max(T v) {
  const uint32_t l = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, v, o);
    if (l >= (uint32_t)o && y > v) v = y;
  }
  return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ------------------------------------------------------------ status

// First error wins; the second word records where (tile or list).
// (kept out of line: it sits on many paths that almost never run)
static __device__ __noinline__ void report(uint32_t* status, uint32_t code, uint32_t where) {
  if (status && atomicCAS(status, 0u, code) == 0u) atomicExch(status + 1, where);
}

// ------------------------------------------------------------ memory

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Little-endian read of `nb` (1..4) bytes at byte offset `off`, or `fill`
// bytes past `size` (the caller decides whether that is an error).
__device__ __forceinline__ uint32_t read_le(const uint8_t* p, uint64_t size, uint64_t off, uint32_t nb,
                                            uint32_t fill = 0) {
  uint32_t v = 0;
  for (uint32_t t = 0; t < nb; ++t) {
    const uint32_t byte = (off + t < size) ? (uint32_t)__ldg(p + off + t) : fill;
    v |= byte << (8 * t);
  }
  return v;
}

// `width` (<= 25) control bits from bit position `pos`.
__device__ __forceinline__ uint32_t read_ctrl_bits(const uint8_t* c, uint64_t size, uint64_t pos,
                                                   uint32_t width) {
  const uint32_t w = read_le(c, size, pos >> 3, 4);
  return (w >> (pos & 7)) & low_mask(width);
}

}  // namespace gcdev
