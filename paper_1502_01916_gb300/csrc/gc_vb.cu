// gc_vb.cu -- Variable Byte for the short posting lists of an index.
//
// Sec 2.3 defines Variable Byte: a number in whole bytes, 7 bits of its
// binary representation per byte, the remaining bit of each byte marking
// the number's last byte. Sec 7.5 keeps it for posting lists shorter than
// 64, where the vertical group codecs spend at least a whole vector. Groups
// go most significant first and the last byte carries the set bit (the form
// of the book the paper cites). A list of n < 64 numbers is a few dozen
// bytes: one thread encodes one list. A warp decodes 32 lists whose bytes
// lie back to back as one stream cut into 32 equal segments, a lane each,
// so that no lane waits for the longest list.

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

// The numbers of one list from its bytes p[0 .. nbytes) into o[0 .. n),
// or its docIDs when restoring (the list's own prefix sum, modulo 2^32);
// false when the bytes do not hold exactly n numbers of at most 32 bits.
__device__ __forceinline__ bool vb_list(const uint8_t* p, uint32_t nbytes, uint32_t n, bool restore, uint32_t* o) {
  uint32_t pos = 0, sum = 0;
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t v = 0;
    for (;;) {
      if (pos >= nbytes || (v >> 25)) return false;  // (v * 128 + 127 would not fit)
      const uint32_t b = p[pos++];
      v = (v << 7) | (b & 0x7fu);
      if (b & 0x80u) break;
    }
    sum += v;
    o[i] = restore ? sum : v;
  }
  return pos == nbytes;
}

// What a warp keeps of its group of 32 lists, per list j.
struct GroupTab {
  uint32_t s[33];   // its first byte in the group (past the group's lists: the group's length)
  uint32_t n[32];   // its numbers
  uint32_t m[32];   // number ends in the group before its first byte
  uint32_t mp[32];  // ... within the segment that holds that byte
  uint32_t b[32];   // running sum of the group's numbers before its first number
  uint32_t bp[32];  // ... within the segment that holds its first byte
  uint64_t oo[32];  // its output offset
};

// Lane t's part of a group whose bytes p[0 .. len) lie back to back: the
// numbers that end (their byte with the high bit set) in its segment
// [a, b). A number belongs to the list holding its last byte; its bytes
// start after the number end before it, but not before its list's first
// byte (what a list's bytes leave unended at its last byte is dropped).
// Counts the segment's numbers (k) and sums their values (sum; a number
// wider than 32 bits counts as 0). The first pass records, for each list
// starting in the segment, k and sum before its first number; the second
// writes each number to its list's output, at its index in the group (C +
// k) less the number ends before the list, as a docID the running sum (E +
// sum) less the sum before the list.
template <bool WRITE>
__device__ __forceinline__ void vb_segment(const Dec& d, uint64_t g0, const uint8_t* p, uint32_t nm, GroupTab& T,
                                           uint32_t a, uint32_t b, uint32_t C, uint32_t E, uint32_t& k,
                                           uint32_t& sum) {
  k = 0;
  sum = 0;
  if (a >= b) return;
  // the list holding byte a (the last one starting at or before a) and the
  // first list starting at or after a
  uint32_t lst = 0, jn = 0;
#pragma unroll
  for (uint32_t step = 16; step; step >>= 1)
    if (lst + step < nm && T.s[lst + step] <= a) lst += step;
#pragma unroll
  for (uint32_t step = 32; step; step >>= 1)
    if (jn + step <= nm && T.s[jn + step - 1] < a) jn += step;
  uint32_t nxt = T.s[lst + 1];
  uint32_t sjn = jn < nm ? T.s[jn] : 0xffffffffu;
  uint32_t m_l = 0, n_l = 0, b_l = 0;
  uint64_t o_l = 0;
  if (WRITE) m_l = T.m[lst], n_l = T.n[lst], b_l = T.b[lst], o_l = T.oo[lst];
  // the first byte of the number holding byte a
  uint32_t q = a;
  const uint32_t s0 = T.s[lst];
  while (q > s0 && !(p[q - 1] & 0x80u)) --q;
  uint32_t v = 0;
  bool wide = false;
  for (uint32_t pos = q; pos < b; ++pos) {
    if (pos == nxt) {  // a list starts here
      v = 0;
      wide = false;
      do {
        ++lst;
        nxt = T.s[lst + 1];
      } while (nxt <= pos);
      if (WRITE) m_l = T.m[lst], n_l = T.n[lst], b_l = T.b[lst], o_l = T.oo[lst];
    }
    const uint32_t x = p[pos];
    if (v >> 25) wide = true;  // (v * 128 + 127 would not fit)
    v = (v << 7) | (x & 0x7fu);
    if (x & 0x80u) {
      if (!WRITE) {
        while (sjn <= pos && sjn < b) {
          T.mp[jn] = k;
          T.bp[jn] = sum;
          ++jn;
          sjn = jn < nm ? T.s[jn] : 0xffffffffu;
        }
      }
      sum += wide ? 0u : v;
      if (WRITE) {
        const uint32_t idx = C + k - m_l;
        if (!wide && idx < n_l) d.out[o_l + idx] = d.restore ? E + sum - b_l : v;
        else report(d.status, GC_ERR_CORRUPT, (uint32_t)(g0 + lst));
      }
      ++k;
      v = 0;
      wide = false;
    }
  }
  if (!WRITE) {
    while (sjn < b) {
      T.mp[jn] = k;
      T.bp[jn] = sum;
      ++jn;
      sjn = jn < nm ? T.s[jn] : 0xffffffffu;
    }
  }
}

// A warp takes lists 32 g .. 32 g + 31, lane j holding list j. When their
// bytes lie back to back, they are cut into 32 equal segments, lane t
// taking segment t (vb_segment), so that every lane has the same bytes to
// walk whatever the lists' lengths: a first pass counts and sums each
// segment's numbers, two warp scans give every segment its numbers and sum
// before it, and a second pass writes. A list is accepted exactly as by
// the one-thread loop: its bytes hold n number ends (the segments' counts),
// its last byte ends a number and every number fits 32 bits; a number that
// is not accepted is not written, so a malformed list writes only inside
// its own output. Lists whose bytes do not lie back to back go one per
// thread.
__device__ void vb_group(const Dec& d, uint64_t g, const gc_vb_list& L, bool mine, bool in, GroupTab& T) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t l = g * 32 + lane;
  if (g * 32 >= d.nlists) return;
  // back to back: each list starts where the one before ends
  const uint64_t end = L.byte_off + L.nbytes;
  const uint64_t prev_end = __shfl_up_sync(kFull, end, 1);
  const uint64_t first = __shfl_sync(kFull, L.byte_off, 0);
  const uint32_t nm = (uint32_t)min((uint64_t)32, d.nlists - g * 32);
  const uint64_t last_end = __shfl_sync(kFull, end, nm - 1);
  const bool joined = !mine || lane == 0 || L.byte_off == prev_end;
  if (__ballot_sync(kFull, in && joined) != kFull || last_end - first >= (1ull << 31)) {
    if (mine && in && !vb_list(d.bytes + L.byte_off, L.nbytes, L.n, d.restore, d.out + L.out_off))
      report(d.status, GC_ERR_CORRUPT, (uint32_t)l);
    return;
  }
  const uint8_t* p = d.bytes + first;
  const uint32_t len = (uint32_t)(last_end - first);
  const uint32_t sj = mine ? (uint32_t)(L.byte_off - first) : len;
  __syncwarp();  // (the group before is written out)
  T.s[lane] = sj;
  if (lane == 0) T.s[32] = len;
  if (mine) {
    T.n[lane] = L.n;
    T.oo[lane] = L.out_off;
  }
  __syncwarp();
  const uint32_t S = (len + 31) / 32;  // bytes per segment
  const uint32_t a = min(lane * S, len), b = min(a + S, len);
  uint32_t k, sum;
  vb_segment<false>(d, g * 32, p, nm, T, a, b, 0, 0, k, sum);
  uint32_t C = k, E = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, C, o), z = __shfl_up_sync(kFull, E, o);
    if (lane >= (uint32_t)o) C += y, E += z;
  }
  const uint32_t ends = __shfl_sync(kFull, C, 31);  // number ends in the group
  C -= k;
  E -= sum;
  __syncwarp();
  const uint32_t u = S && sj < len ? min(sj / S, 31u) : 0u;  // the segment holding list j's first byte
  const uint32_t Cu = __shfl_sync(kFull, C, u), Eu = __shfl_sync(kFull, E, u);
  const uint32_t mj = sj < len ? Cu + T.mp[lane] : ends;
  T.m[lane] = mj;
  T.b[lane] = sj < len ? Eu + T.bp[lane] : 0u;
  const uint32_t m_next = __shfl_down_sync(kFull, mj, 1);
  if (mine && ((lane + 1 < nm ? m_next : ends) - mj != L.n || (L.nbytes && !(p[sj + L.nbytes - 1] & 0x80u))))
    report(d.status, GC_ERR_CORRUPT, (uint32_t)l);
  __syncwarp();
  vb_segment<true>(d, g * 32, p, nm, T, a, b, C, E, k, sum);
}

// Warp w takes lists 32 w .. 32 w + 31 as a group (vb_group).
__global__ void __launch_bounds__(256) k_vb_decode(Dec d) {
  __shared__ GroupTab tabs[8];
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t groups = (d.nlists + 31) / 32;
  for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; g < groups;
       g += (uint64_t)gridDim.x * blockDim.x / 32) {
    const uint64_t l = g * 32 + lane;
    const bool mine = l < d.nlists;
    gc_vb_list L = {};
    if (mine) L = d.lists[l];
    const bool in = !mine || (L.byte_off <= d.bytes_len && L.nbytes <= d.bytes_len - L.byte_off &&
                              L.out_off <= d.out_len && L.n <= d.out_len - L.out_off);
    if (!in) report(d.status, GC_ERR_INVALID, (uint32_t)l);
    vb_group(d, g, L, mine, in, tabs[threadIdx.x >> 5]);
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
  if (nlists > 0xffffffffull) return GC_ERR_UNSUPPORTED;  // (list indices are reported as uint32)
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
  if (nlists > 0xffffffffull) return GC_ERR_UNSUPPORTED;  // (list indices are reported as uint32)
  gcvb::Dec d = {};
  d.lists = d_lists;
  d.nlists = nlists;
  d.bytes = d_bytes;
  d.bytes_len = bytes_len;
  d.out = d_out;
  d.out_len = out_len;
  d.restore = restore_docids;
  d.status = d_status;
  const uint64_t want = (nlists + 255) / 256;  // a warp per 32 lists, 8 warps per block
  const unsigned g = (unsigned)(want < 65536 ? want : 65536);
  gcvb::k_vb_decode<<<g, 256, 0, (cudaStream_t)stream>>>(d);
  gc_host::count_launch(1);
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

}  // extern "C"
