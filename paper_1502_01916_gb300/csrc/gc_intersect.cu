// gc_intersect.cu -- AND queries over a resident index: the docIDs of one
// list that are also in another, decoding all of the first list and, of
// the second, only the tiles whose docID range (from their skip entries)
// can hold one of the first list's docIDs.
//
// The paper decodes the lists of a query and intersects them with skip
// pointers (Sec 7.4): a skip entry gives the docID before a block, so a
// block that cannot hold the docID looked for is never decoded. Here the
// blocks are the 1024-int tiles of the tile index, whose records carry the
// docID before the tile (gc_tile.base with GC_TILE_BASE).
//
// Steps, all on the caller's stream: (1) plan and decode every query's
// list a (gc_plan_select + gc_decode_plan); (2) for each docID x of a, the
// tile of list b that could hold it: the number of b's tiles t >= 1 whose
// base (the docID before tile t) is below x; mark it; (3) one plan record
// per marked tile, its 1024 ints to their own slot; (4) decode those
// tiles; (5) look x up in its tile by binary search; (6) per query, the
// hits in order: every docID of a gets the number of hits before it in
// all of a (a scan over spans of 4096 docIDs), so that a hit's place in
// its query's results is its rank minus the rank of the query's first
// docID -- the time does not hang on the longest query.

#include <cstdint>
#include <cuda_runtime.h>

#include "gc.h"
#include "gc_device.cuh"
#include "gc_host.h"

namespace gcisect {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kTile = 1024;           // ints per tile
constexpr uint32_t kUnmarked = 0xffffffffu;
constexpr uint32_t kMarked = 0xfffffffeu;
constexpr uint32_t kSpanThreads = 256;
constexpr uint32_t kSpan = 16 * kSpanThreads;  // docIDs of a per span of the rank scan
constexpr uint32_t kScan = 1024;               // span sums per round of their scan

struct Args {
  const gc_list* lists;
  uint64_t nlists;
  const gc_tile* tiles;
  uint64_t ntiles;
  const uint32_t* qa;      // per query: list a (decoded whole)
  const uint32_t* qb;      // per query: list b (decoded by tile)
  const uint64_t* aoff;    // per query: first int of a's docIDs (and of its results)
  const uint64_t* boff;    // per query: first of b's tiles in the marks
  uint64_t nq;
  uint64_t a_ints;         // sum of the a lists' lengths
  uint64_t b_tiles;        // sum of the b lists' tiles
  uint32_t k;              // codec lanes (tile rows = 1024 / k)
  uint32_t* adoc;          // decoded a docIDs (a_ints)
  uint32_t* at;            // per a docID: its tile of b
  uint32_t* mark;          // per tile of b: kUnmarked, kMarked, or its plan record
  uint8_t* hit;            // per a docID: found in b
  gc_work* work;           // plan records of the marked tiles
  uint32_t* sel;           // per record: list b
  uint64_t* outs;          // per record: output offset - 1024 * tile
  unsigned long long* count;  // [0] records
  uint64_t rec_cap;
  uint32_t* bdoc;          // decoded tiles, 1024 ints per record
  uint32_t* span;          // per span: its hits, then the hits before it
  uint64_t nspans;
  uint32_t* total;         // hits in all of a
  uint32_t* rank;          // per a docID: the hits before it in all of a (reuses at)
  uint32_t* out;           // results at aoff[q]
  uint32_t* counts;        // per query: results
  uint32_t* status;
};

using gcdev::report;

// query q of flat index i: the last q with off[q] <= i
__device__ __forceinline__ uint64_t query_of(const uint64_t* off, uint64_t nq, uint64_t i) {
  uint64_t lo = 0, hi = nq;  // off[lo] <= i < off[hi] (off[nq] taken as infinite)
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) / 2;
    if (off[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint64_t tiles_of(uint64_t n, uint32_t k) {
  const uint64_t rows = (n + k - 1) / k;
  const uint64_t tr = kTile / k;
  return (rows + tr - 1) / tr;
}

// (2) each docID of a: its tile of b, marked
__global__ void k_isect_mark(Args a) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.a_ints) return;
  const uint64_t q = query_of(a.aoff, a.nq, i);
  const uint32_t lb = a.qb[q];
  a.at[i] = kUnmarked;
  if (a.qa[q] >= a.nlists || lb >= a.nlists) return;  // reported by k_isect_check
  const gc_list B = a.lists[lb];
  const uint64_t nt = tiles_of(B.n, a.k);
  if (nt == 0) return;
  const uint32_t x = a.adoc[i];
  // tiles t >= 1 whose base (the docID before the tile) is below x
  uint64_t lo = 0, hi = nt - 1;  // the answer is in [lo, hi]
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) / 2;  // tile mid >= 1
    const uint64_t ti = (uint64_t)B.tile_off + mid - 1;
    if (ti >= a.ntiles) {
      report(a.status, GC_ERR_CORRUPT, lb);
      return;
    }
    const gc_tile r = a.tiles[ti];
    if (!(r.flags & GC_TILE_BASE)) {
      report(a.status, GC_ERR_UNSUPPORTED, lb);  // an index without skip entries
      return;
    }
    if (r.base < x) lo = mid;
    else hi = mid - 1;
  }
  a.at[i] = (uint32_t)lo;
  const uint64_t g = a.boff[q] + lo;
  if (g < a.b_tiles) a.mark[g] = kMarked;
}

// (3) one plan record per marked tile: (record, tile), list b, its ints
// at 1024 * record
__global__ void k_isect_reserve(Args a) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31u;
  bool want = false;
  uint64_t q = 0, t = 0;
  if (g < a.b_tiles && a.mark[g] == kMarked) {
    q = query_of(a.boff, a.nq, g);
    t = g - a.boff[q];
    want = true;
  }
  const uint32_t m = __ballot_sync(kFull, want);
  unsigned long long base = 0;
  if (lane == 0 && m) base = atomicAdd(a.count, (unsigned long long)__popc(m));
  base = __shfl_sync(kFull, base, 0);
  if (!want) return;
  const uint64_t r = base + __popc(m & ((1u << lane) - 1u));
  if (r >= a.rec_cap) {
    report(a.status, GC_ERR_NOSPACE, (uint32_t)q);
    a.mark[g] = kUnmarked;
    return;
  }
  gc_work w = {};
  w.list = (uint32_t)r;
  w.tile = (uint32_t)t;
  a.work[r] = w;
  a.sel[r] = a.qb[q];
  a.outs[r] = (uint64_t)kTile * r - (uint64_t)kTile * t;  // (modulo 2^64: the tile lands at 1024 r)
  a.mark[g] = (uint32_t)r;
}

// (5) each docID of a looked up in its tile of b
__global__ void k_isect_probe(Args a) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.a_ints) return;
  const uint64_t q = query_of(a.aoff, a.nq, i);
  const uint32_t lb = a.qb[q];
  bool found = false;
  if (a.qa[q] < a.nlists && lb < a.nlists) {
    const gc_list B = a.lists[lb];
    const uint32_t t = a.at[i];
    const uint64_t g = a.boff[q] + t;
    const uint32_t r = t < tiles_of(B.n, a.k) && g < a.b_tiles ? a.mark[g] : kUnmarked;
    if (r < a.rec_cap && r < a.count[0]) {
      const uint64_t first = (uint64_t)t * kTile;
      const uint32_t n = first < B.n ? (uint32_t)min((uint64_t)kTile, B.n - first) : 0u;
      const uint32_t* d = a.bdoc + (uint64_t)kTile * r;
      const uint32_t x = a.adoc[i];
      uint32_t lo = 0, hi = n;  // first position with d[pos] >= x
      while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (d[mid] < x) lo = mid + 1;
        else hi = mid;
      }
      found = lo < n && d[lo] == x;
    }
  }
  a.hit[i] = found ? 1 : 0;
}

// the hit flags (0 or 1 a byte) of a's docIDs i0 .. i0 + 15 as four words
// and their sum (i0 a multiple of 16: whole groups are one 16-byte load)
__device__ __forceinline__ uint32_t hits16(const Args& a, uint64_t i0, uint32_t w[4]) {
  if (i0 + 16 <= a.a_ints) {
    const uint4 v = *reinterpret_cast<const uint4*>(a.hit + i0);
    w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
  } else {
    w[0] = w[1] = w[2] = w[3] = 0;
    for (uint32_t j = 0; i0 + j < a.a_ints && j < 16; ++j) w[j / 4] |= (uint32_t)a.hit[i0 + j] << (8 * (j % 4));
  }
  return __popc(w[0]) + __popc(w[1]) + __popc(w[2]) + __popc(w[3]);
}

// exclusive scan of one value per thread over a block of kSpanThreads;
// the block's sum to *sum
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t* sum) {
  __shared__ uint32_t warp_sums[kSpanThreads / 32];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (uint32_t w = 0; w < kSpanThreads / 32; ++w) {
    before += w < wid ? warp_sums[w] : 0u;
    all += warp_sums[w];
  }
  *sum = all;
  return before + x - v;
}

// (6a) the hits of each span
__global__ void __launch_bounds__(kSpanThreads) k_isect_span_sums(Args a) {
  uint32_t w[4], all;
  block_scan(hits16(a, (uint64_t)blockIdx.x * kSpan + 16u * threadIdx.x, w), &all);
  if (threadIdx.x == 0) a.span[blockIdx.x] = all;
}

// (6b) exclusive scan of the span sums (one block, rounds of kScan); the
// total to *total
__global__ void __launch_bounds__(kScan) k_isect_span_scan(Args a) {
  __shared__ uint32_t warp_sums[kScan / 32];
  __shared__ uint32_t carry;
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t r = 0; r < a.nspans; r += kScan) {
    const uint64_t i = r + threadIdx.x;
    const uint32_t v = i < a.nspans ? a.span[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint32_t y = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t z = __shfl_up_sync(kFull, y, o);
        if (lane >= (uint32_t)o) y += z;
      }
      warp_sums[lane] = y;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t c = carry;
    if (i < a.nspans) a.span[i] = c + (wid ? warp_sums[wid - 1] : 0u) + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + warp_sums[kScan / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.total = carry;
}

// (6c) each docID of a: the hits before it in all of a
__global__ void __launch_bounds__(kSpanThreads) k_isect_rank(Args a) {
  const uint64_t i0 = (uint64_t)blockIdx.x * kSpan + 16u * threadIdx.x;
  uint32_t w[4], all;
  uint32_t r = a.span[blockIdx.x] + block_scan(hits16(a, i0, w), &all);
  uint32_t rk[16];
#pragma unroll
  for (uint32_t j = 0; j < 16; ++j) {
    rk[j] = r;
    r += (w[j / 4] >> (8 * (j % 4))) & 1u;
  }
  if (i0 + 16 <= a.a_ints) {
    uint4* d = reinterpret_cast<uint4*>(a.rank + i0);
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) d[j] = make_uint4(rk[4 * j], rk[4 * j + 1], rk[4 * j + 2], rk[4 * j + 3]);
  } else {
#pragma unroll
    for (uint32_t j = 0; j < 16; ++j)
      if (i0 + j < a.a_ints) a.rank[i0 + j] = rk[j];
  }
}

// (6d) each hit to its query's results, in order; each query's count
__global__ void k_isect_place(Args a) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.a_ints && a.hit[i]) {
    const uint64_t q = query_of(a.aoff, a.nq, i);
    const uint64_t p = a.aoff[q];
    if (p > i) report(a.status, GC_ERR_INVALID, (uint32_t)q);
    else a.out[p + (a.rank[i] - a.rank[p])] = a.adoc[i];
  }
  if (i < a.nq) {
    const uint64_t p = a.aoff[i], e = i + 1 < a.nq ? a.aoff[i + 1] : a.a_ints;
    if (p > e || e > a.a_ints) {
      report(a.status, GC_ERR_INVALID, (uint32_t)i);
      a.counts[i] = 0;
    } else {
      const uint32_t rp = p < a.a_ints ? a.rank[p] : *a.total, re = e < a.a_ints ? a.rank[e] : *a.total;
      a.counts[i] = re - rp;
    }
  }
}

// the queries' lists exist
__global__ void k_isect_check(Args a) {
  const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nq) return;
  if (a.qa[q] >= a.nlists || a.qb[q] >= a.nlists) report(a.status, GC_ERR_INVALID, (uint32_t)q);
}

}  // namespace gcisect

namespace {

using namespace gcisect;

struct Layout {
  uint64_t hdr, work_a, dec_a, adoc, at, hit, span, mark, work_b, sel, outs, dec_b, bdoc, total;
};

Layout layout(uint64_t a_tiles, uint64_t a_ints, uint64_t b_tiles) {
  using gc_host::align_up;
  const uint64_t rec = a_ints < b_tiles ? a_ints : b_tiles;
  uint64_t dec_a = 0, dec_b = 0;
  gc_decode_plan_scratch_size(a_tiles ? a_tiles : 1, &dec_a);
  gc_decode_plan_scratch_size(rec ? rec : 1, &dec_b);
  Layout L;
  uint64_t o = 0;
  L.hdr = o;
  o += 256;  // plan counts of a (2 uint64) and of b (2 uint64); hits in all of a (uint32)
  L.work_a = o;
  o += align_up(a_tiles * sizeof(gc_work), 256);
  L.dec_a = o;
  o += align_up(dec_a, 256);
  L.adoc = o;
  o += align_up(a_ints * 4, 256);
  L.at = o;
  o += align_up(a_ints * 4, 256);
  L.hit = o;
  o += align_up(a_ints, 256);
  L.span = o;
  o += align_up((a_ints + kSpan - 1) / kSpan * 4, 256);
  L.mark = o;
  o += align_up(b_tiles * 4, 256);
  L.work_b = o;
  o += align_up(rec * sizeof(gc_work), 256);
  L.sel = o;
  o += align_up(rec * 4, 256);
  L.outs = o;
  o += align_up(rec * 8, 256);
  L.dec_b = o;
  o += align_up(dec_b, 256);
  L.bdoc = o;
  o += align_up(rec * (uint64_t)kTile * 4, 256);
  L.total = o;
  return L;
}

unsigned grid(uint64_t n, unsigned per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

extern "C" {

gc_status gc_intersect_scratch_size(uint64_t a_ints, uint64_t a_tiles, uint64_t b_tiles, uint64_t* bytes) {
  if (!bytes) return GC_ERR_INVALID;
  *bytes = layout(a_tiles, a_ints, b_tiles).total;
  return GC_OK;
}

gc_status gc_intersect(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists, const gc_tile* d_tile_pool,
                       uint64_t tile_pool_len, const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes,
                       const uint32_t* d_data_pool, uint64_t data_pool_words, const uint32_t* d_a,
                       const uint32_t* d_b, const uint64_t* d_a_offs, const uint64_t* d_b_tile_offs, uint64_t nqueries,
                       uint64_t a_ints, uint64_t a_tiles, uint64_t b_tiles, uint32_t* d_out, uint32_t* d_counts,
                       void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (nqueries == 0) return GC_OK;
  if (!d_lists || !d_tile_pool || !d_a || !d_b || !d_a_offs || !d_b_tile_offs || !d_counts || !d_scratch ||
      (!d_ctrl_pool && ctrl_pool_bytes) || (!d_data_pool && data_pool_words) || (a_ints && !d_out))
    return GC_ERR_INVALID;
  if (((uintptr_t)d_data_pool & 15) != 0 || ((uintptr_t)d_ctrl_pool & 15) != 0 ||
      ((uintptr_t)d_scratch & 255) != 0)
    return GC_ERR_INVALID;
  if (nlists > 0xffffffffull || nqueries > 0xffffffffull || a_tiles > 0xffffffffull - 1024 ||
      b_tiles > 0xffffffffull - 1024 || a_ints > 0xffffffffull)
    return GC_ERR_UNSUPPORTED;
  const Layout L = layout(a_tiles, a_ints, b_tiles);
  if (scratch_bytes < L.total) return GC_ERR_NOSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = (unsigned char*)d_scratch;
  uint64_t* count_a = reinterpret_cast<uint64_t*>(base + L.hdr);
  uint64_t* count_b = count_a + 2;
  const uint64_t rec = a_ints < b_tiles ? a_ints : b_tiles;
  uint32_t launches = 0;

  Args g = {};
  g.lists = d_lists;
  g.nlists = nlists;
  g.tiles = d_tile_pool;
  g.ntiles = tile_pool_len;
  g.qa = d_a;
  g.qb = d_b;
  g.aoff = d_a_offs;
  g.boff = d_b_tile_offs;
  g.nq = nqueries;
  g.a_ints = a_ints;
  g.b_tiles = b_tiles;
  g.k = codec->k;
  g.adoc = reinterpret_cast<uint32_t*>(base + L.adoc);
  g.at = reinterpret_cast<uint32_t*>(base + L.at);
  g.mark = reinterpret_cast<uint32_t*>(base + L.mark);
  g.hit = base + L.hit;
  g.work = reinterpret_cast<gc_work*>(base + L.work_b);
  g.sel = reinterpret_cast<uint32_t*>(base + L.sel);
  g.outs = reinterpret_cast<uint64_t*>(base + L.outs);
  g.count = reinterpret_cast<unsigned long long*>(count_b);
  g.rec_cap = rec;
  g.bdoc = reinterpret_cast<uint32_t*>(base + L.bdoc);
  g.span = reinterpret_cast<uint32_t*>(base + L.span);
  g.nspans = (a_ints + kSpan - 1) / kSpan;
  g.total = reinterpret_cast<uint32_t*>(base + L.hdr + 32);
  g.rank = g.at;  // the tiles of b are looked up by then
  g.out = d_out;
  g.counts = d_counts;
  g.status = d_status;

  k_isect_check<<<grid(nqueries, 256), 256, 0, s>>>(g);
  ++launches;
  // (1) every list a, whole, its docIDs at a_offs
  if (a_ints) {
    st = gc_plan_select(codec, d_lists, nlists, d_a, d_a_offs, nqueries, d_tile_pool, tile_pool_len, d_ctrl_pool,
                        ctrl_pool_bytes, reinterpret_cast<gc_work*>(base + L.work_a), a_tiles, count_a, d_status,
                        stream);
    if (st != GC_OK) return st;
    launches += gc_host::launches();
    uint64_t dec_a = 0;
    gc_decode_plan_scratch_size(a_tiles, &dec_a);
    st = gc_decode_plan(codec, reinterpret_cast<gc_work*>(base + L.work_a), count_a, a_tiles, d_ctrl_pool,
                        ctrl_pool_bytes, d_data_pool, data_pool_words, g.adoc, a_ints, 1, nullptr, base + L.dec_a,
                        dec_a, d_status, stream);
    if (st != GC_OK) return st;
    launches += gc_host::launches();
  }
  // (2) the tiles of b that can hold a docID of a
  if (cudaMemsetAsync(count_b, 0, 16, s) != cudaSuccess) return GC_ERR_CUDA;
  if (b_tiles && cudaMemsetAsync(g.mark, 0xff, b_tiles * 4, s) != cudaSuccess) return GC_ERR_CUDA;
  if (a_ints) {
    k_isect_mark<<<grid(a_ints, 256), 256, 0, s>>>(g);
    ++launches;
  }
  // (3) their plan records, (4) their decode
  if (b_tiles && rec) {
    k_isect_reserve<<<grid(b_tiles, 256), 256, 0, s>>>(g);
    ++launches;
    gc_host::reset_launches();
    st = gc_host::plan_fill(*codec, d_lists, nlists, g.sel, g.outs, rec, d_tile_pool, tile_pool_len, d_ctrl_pool,
                            ctrl_pool_bytes, g.work, rec, count_b, d_status, s);
    if (st != GC_OK) return st;
    launches += gc_host::launches();
    uint64_t dec_b = 0;
    gc_decode_plan_scratch_size(rec, &dec_b);
    st = gc_decode_plan(codec, g.work, count_b, rec, d_ctrl_pool, ctrl_pool_bytes, d_data_pool, data_pool_words,
                        g.bdoc, rec * kTile, 1, nullptr, base + L.dec_b, dec_b, d_status,
                        stream);
    if (st != GC_OK) return st;
    launches += gc_host::launches();
  }
  // (5) lookups, (6) results in order
  if (a_ints) {
    k_isect_probe<<<grid(a_ints, 256), 256, 0, s>>>(g);
    k_isect_span_sums<<<(unsigned)g.nspans, kSpanThreads, 0, s>>>(g);
    k_isect_span_scan<<<1, kScan, 0, s>>>(g);
    k_isect_rank<<<(unsigned)g.nspans, kSpanThreads, 0, s>>>(g);
    launches += 4;
  } else if (cudaMemsetAsync(g.total, 0, 4, s) != cudaSuccess) {
    return GC_ERR_CUDA;
  }
  k_isect_place<<<grid(a_ints > nqueries ? a_ints : nqueries, 256), 256, 0, s>>>(g);
  ++launches;
  gc_host::reset_launches();
  gc_host::count_launch(launches);
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

}  // extern "C"
