// gc_vb.cu -- Variable Byte for the short posting lists of an index.
//
// Sec 2.3 defines Variable Byte: a number in whole bytes, 7 bits of its
// binary representation per byte, the remaining bit of each byte marking
// the number's last byte. Sec 7.5 keeps it for posting lists shorter than
// 64, where the vertical group codecs spend at least a whole vector. Groups
// go most significant first and the last byte carries the set bit (the form
// of the book the paper cites). A list of n < 64 numbers is a few dozen
// bytes, so one thread encodes or decodes one list.

#include <cstdint>
#include <cuda_runtime.h>

#include "gc.h"
#include "gc_device.cuh"
#include "gc_host.h"

namespace gcvb {

using gcdev::report;
constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kScan = 1024;  // lists per scan block

__device__ __forceinline__ uint32_t vb_size(uint32_t x) {
  return x < (1u << 7) ? 1u : x < (1u << 14) ? 2u : x < (1u << 21) ? 3u : x < (1u << 28) ? 4u : 5u;
}

struct Enc {
  const uint32_t* gaps;
  const uint64_t* in_off;
  const uint32_t* n;
  uint64_t nlists;
  uint64_t* offs;        // per list: bytes, then their exclusive prefix sums
  uint64_t* block_sums;  // per scan block
  uint64_t nblocks;
  gc_vb_list* lists;
  uint8_t* bytes;
  uint64_t cap;
  uint64_t* total;
  uint32_t* status;
};

// bytes of each list
__global__ void k_vb_sizes(Enc e) {
  const uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= e.nlists) return;
  const uint32_t* g = e.gaps + e.in_off[l];
  uint64_t b = 0;
  for (uint32_t i = 0; i < e.n[l]; ++i) b += vb_size(g[i]);
  e.offs[l] = b;
}

// exclusive scan of a block of kScan values in place; the block's sum to
// block_sums
__global__ void k_vb_scan_blocks(Enc e) {
  __shared__ uint64_t warp_sums[kScan / 32];
  const uint64_t i = (uint64_t)blockIdx.x * kScan + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const uint64_t v = i < e.nlists ? e.offs[i] : 0;
  uint64_t s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, s, o);
    if (lane >= (uint32_t)o) s += y;
  }
  if (lane == 31) warp_sums[wid] = s;
  __syncthreads();
  if (wid == 0) {
    uint64_t w = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, w, o);
      if (lane >= (uint32_t)o) w += y;
    }
    warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const uint64_t before = wid ? warp_sums[wid - 1] : 0;
  if (i < e.nlists) e.offs[i] = before + s - v;
  if (threadIdx.x == kScan - 1) e.block_sums[blockIdx.x] = warp_sums[kScan / 32 - 1];
}

// exclusive scan of the block sums (one block, in rounds of kScan); the
// total to *total
__global__ void k_vb_scan_top(Enc e) {
  __shared__ uint64_t warp_sums[kScan / 32];
  __shared__ uint64_t carry;
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t r = 0; r < e.nblocks; r += kScan) {
    const uint64_t i = r + threadIdx.x;
    const uint64_t v = i < e.nblocks ? e.block_sums[i] : 0;
    uint64_t s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, s, o);
      if (lane >= (uint32_t)o) s += y;
    }
    if (lane == 31) warp_sums[wid] = s;
    __syncthreads();
    if (wid == 0) {
      uint64_t w = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(kFull, w, o);
        if (lane >= (uint32_t)o) w += y;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    const uint64_t c = carry;
    if (i < e.nblocks) e.block_sums[i] = c + (wid ? warp_sums[wid - 1] : 0) + s - v;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + warp_sums[kScan / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *e.total = carry;
}

// each list's bytes at its offset (the whole batch must fit)
__global__ void k_vb_write(Enc e) {
  const uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= e.nlists) return;
  if (*e.total > e.cap) {
    if (l == 0) report(e.status, GC_ERR_NOSPACE, 0);
    return;
  }
  const uint64_t off = e.offs[l] + e.block_sums[l / kScan];
  const uint32_t n = e.n[l];
  const uint32_t* g = e.gaps + e.in_off[l];
  uint8_t* p = e.bytes + off;
  uint64_t pos = 0;
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t x = g[i];
    const uint32_t sz = vb_size(x);
    for (uint32_t j = 0; j < sz; ++j) {  // group j (least significant first) to byte sz - 1 - j
      p[pos + sz - 1 - j] = (uint8_t)((x & 0x7fu) | (j == 0 ? 0x80u : 0u));
      x >>= 7;
    }
    pos += sz;
  }
  gc_vb_list d;
  d.byte_off = off;
  d.out_off = e.in_off[l];
  d.n = n;
  d.nbytes = (uint32_t)pos;
  e.lists[l] = d;
}

struct Dec {
  const gc_vb_list* lists;
  uint64_t nlists;
  const uint8_t* bytes;
  uint64_t bytes_len;
  uint32_t* out;
  uint64_t out_len;
  int restore;
  uint32_t* status;
};

// each list's numbers (its docIDs when restoring: the list's own prefix
// sum, modulo 2^32)
__global__ void k_vb_decode(Dec d) {
  for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < d.nlists;
       l += (uint64_t)gridDim.x * blockDim.x) {
    const gc_vb_list L = d.lists[l];
    if (L.byte_off + L.nbytes > d.bytes_len || L.out_off + L.n > d.out_len) {
      report(d.status, GC_ERR_INVALID, (uint32_t)l);
      continue;
    }
    const uint8_t* p = d.bytes + L.byte_off;
    uint32_t* o = d.out + L.out_off;
    uint32_t pos = 0, sum = 0;
    bool ok = true;
    for (uint32_t i = 0; i < L.n && ok; ++i) {
      uint64_t v = 0;
      for (;;) {
        if (pos >= L.nbytes) {
          ok = false;
          break;
        }
        const uint32_t b = p[pos++];
        v = v * 128u + (b & 0x7fu);
        if (v > 0xffffffffull) {
          ok = false;
          break;
        }
        if (b & 0x80u) break;
      }
      if (!ok) break;
      sum += (uint32_t)v;
      o[i] = d.restore ? sum : (uint32_t)v;
    }
    if (!ok || pos != L.nbytes) report(d.status, GC_ERR_CORRUPT, (uint32_t)l);
  }
}

}  // namespace gcvb

extern "C" {

gc_status gc_vb_encode_batch_scratch_size(uint64_t nlists, uint64_t* bytes) {
  if (!bytes) return GC_ERR_INVALID;
  const uint64_t nb = (nlists + gcvb::kScan - 1) / gcvb::kScan;
  *bytes = gc_host::align_up(nlists * 8, 256) + gc_host::align_up((nb ? nb : 1) * 8, 256);
  return GC_OK;
}

gc_status gc_vb_encode_batch(const uint32_t* d_gaps, const uint64_t* d_in_off, const uint32_t* d_n, uint64_t nlists,
                             gc_vb_list* d_lists, uint8_t* d_bytes, uint64_t bytes_cap, uint64_t* d_total,
                             void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  if (!d_total) return GC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (nlists == 0) return cudaMemsetAsync(d_total, 0, 8, s) == cudaSuccess ? GC_OK : GC_ERR_CUDA;
  if (!d_gaps || !d_in_off || !d_n || !d_lists || !d_scratch || (!d_bytes && bytes_cap)) return GC_ERR_INVALID;
  uint64_t need = 0;
  gc_vb_encode_batch_scratch_size(nlists, &need);
  if (scratch_bytes < need) return GC_ERR_NOSPACE;
  gcvb::Enc e = {};
  e.gaps = d_gaps;
  e.in_off = d_in_off;
  e.n = d_n;
  e.nlists = nlists;
  e.offs = reinterpret_cast<uint64_t*>(d_scratch);
  e.block_sums = reinterpret_cast<uint64_t*>((unsigned char*)d_scratch + gc_host::align_up(nlists * 8, 256));
  e.nblocks = (nlists + gcvb::kScan - 1) / gcvb::kScan;
  e.lists = d_lists;
  e.bytes = d_bytes;
  e.cap = bytes_cap;
  e.total = d_total;
  e.status = d_status;
  const unsigned g = (unsigned)((nlists + 255) / 256);
  gcvb::k_vb_sizes<<<g, 256, 0, s>>>(e);
  gcvb::k_vb_scan_blocks<<<(unsigned)e.nblocks, gcvb::kScan, 0, s>>>(e);
  gcvb::k_vb_scan_top<<<1, gcvb::kScan, 0, s>>>(e);
  gcvb::k_vb_write<<<g, 256, 0, s>>>(e);
  gc_host::count_launch(4);
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

gc_status gc_vb_decode_batch(const gc_vb_list* d_lists, uint64_t nlists, const uint8_t* d_bytes, uint64_t bytes_len,
                             uint32_t* d_out, uint64_t out_len, int restore_docids, uint32_t* d_status,
                             void* stream) {
  gc_host::reset_launches();
  if (nlists == 0) return GC_OK;
  if (!d_lists || !d_out || (!d_bytes && bytes_len)) return GC_ERR_INVALID;
  gcvb::Dec d = {};
  d.lists = d_lists;
  d.nlists = nlists;
  d.bytes = d_bytes;
  d.bytes_len = bytes_len;
  d.out = d_out;
  d.out_len = out_len;
  d.restore = restore_docids;
  d.status = d_status;
  const uint64_t want = (nlists + 255) / 256;
  const unsigned g = (unsigned)(want < 65536 ? want : 65536);
  gcvb::k_vb_decode<<<g, 256, 0, (cudaStream_t)stream>>>(d);
  gc_host::count_launch(1);
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

}  // extern "C"
