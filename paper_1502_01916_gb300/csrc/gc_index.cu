// gc_index.cu -- the tile index of one list, built from its control area.
//
// The paper's format stores no position records inside a list (Sec 4.3 reads
// the control patterns from the start). Decoding tile t of a list in
// parallel needs where the unit that holds the tile's first row starts: its
// lane bit, its control bit, its Group-PFD exception offset, and how many of
// its rows precede the tile. Those follow from the control area alone: split
// it into chunks, sum (rows, lane bits, exception bytes) per chunk, scan the
// chunk sums, and walk each chunk again from its prefix, writing a record
// for every tile whose first row falls in a unit. No data word is read, so
// no record but tile 0's carries a docID base.
#include <cstdint>
#include <cuda_runtime.h>

#include "gc_device.cuh"
#include "gc_host.h"

namespace gcidx {

using namespace gcdev;


struct UnitAgg {
  uint64_t rows, lbits, xbytes;
};

struct IndexArgs {
  uint32_t kind, k, cg, ld;
  const uint8_t* ctrl;
  uint64_t ctrl_bytes;
  uint64_t n, R;
  uint64_t nunits;   // units (fixed-size control) or control bytes (unary)
  uint64_t nchunks;
  gc_tile* tiles;
  uint64_t ntiles;
  UnitAgg* block_sums;
  uint32_t* status;
};

constexpr int kChunkUnits = 64;  // units per chunk (fixed-size control)
constexpr int kChunkBytes = 8;   // control bytes per chunk (unary)
constexpr int kIndexThreads = 256;

// Walk one chunk. With emit = false only the sums; with emit = true starting
// from `base`, write the tile records.
__device__ UnitAgg walk_chunk(const IndexArgs& a, uint64_t c, bool emit, UnitAgg base) {
  UnitAgg s = {0, 0, 0};
  const uint64_t tr = kTileInts / a.k;
  auto put = [&](uint64_t row, uint64_t urows, uint64_t lbit, uint64_t cbit, uint64_t xoff) {
    // tiles whose first row lies in [row, row + urows)
    uint64_t t = (row + tr - 1) / tr;
    for (; t * tr < row + urows && t < a.ntiles; ++t) {
      gc_tile g;
      g.lane_bit = lbit;
      g.ctrl_bit = cbit;
      g.exc_off = (uint32_t)xoff;
      g.row_skip = (uint32_t)(t * tr - row);
      g.base = 0;
      g.flags = t == 0 ? GC_TILE_BASE : 0u;  // the docID before a list is 0
      a.tiles[t] = g;
    }
  };
  if (a.kind == GC_SCHEME && a.ld != GC_LD_BINARY) {
    // unary: units are zeros; a chunk owns the descriptors whose closing
    // zero lies in its bytes
    const uint64_t b0 = c * kChunkBytes;
    const uint64_t b1 = (b0 + kChunkBytes) < a.ctrl_bytes ? (b0 + kChunkBytes) : a.ctrl_bytes;
    const bool iu = a.ld == GC_LD_IU;
    // previous zero before the chunk (CU only; within 32 bits unless at 0)
    int64_t prev = -1;
    if (!iu && b0 > 0) {
      for (int64_t p = (int64_t)b0 * 8 - 1; p >= 0 && p >= (int64_t)b0 * 8 - 40; --p)
        if (!((a.ctrl[p >> 3] >> (p & 7)) & 1)) { prev = p; break; }
    }
    uint64_t row = base.rows, lb = base.lbits;
    for (uint64_t by = b0; by < b1; ++by) {
      const uint32_t byte = a.ctrl[by];
      if (iu) prev = (int64_t)by * 8 - 1;
      for (uint32_t bit = 0; bit < 8; ++bit) {
        if ((byte >> bit) & 1u) continue;
        const int64_t p = (int64_t)by * 8 + bit;
        const uint64_t u = (uint64_t)(p - prev);
        if (emit && row < a.R) put(row, 1, lb, (uint64_t)(prev + 1), 0);
        ++row;
        lb += a.cg * u;
        s.rows += 1;
        s.lbits += a.cg * u;
        prev = p;
      }
    }
    return s;
  }
  const uint64_t u0 = c * kChunkUnits;
  const uint64_t u1 = (u0 + kChunkUnits) < a.nunits ? (u0 + kChunkUnits) : a.nunits;
  uint64_t row = base.rows, lb = base.lbits, xo = base.xbytes;
  const uint64_t nf = (a.R + kPfdFrameRows - 1) / kPfdFrameRows;
  const uint32_t pb = (kPfdFrameRows * a.k) <= 256 ? 1u : 2u;
  for (uint64_t u = u0; u < u1; ++u) {
    uint64_t urows, lbits, xb = 0, cbit;
    if (a.kind == GC_SIMPLE) {
      const uint32_t sel = (a.ctrl[u >> 1] >> ((u & 1) * 4)) & 15u;
      if (sel > 9) {
        if (emit && row < a.R) report(a.status, GC_ERR_CORRUPT, (uint32_t)u);
        urows = 32;
        lbits = 32;
      } else {
        urows = sel_num(sel);
        lbits = 32;
      }
      cbit = 4 * u;
    } else if (a.kind == GC_SCHEME) {
      const uint32_t width = 5 - log2_cg(a.cg);
      cbit = bin_ld_pos(u, a.cg);
      const uint32_t v = read_ctrl_bits(a.ctrl, a.ctrl_bytes, cbit, width) + 1;
      urows = 1;
      lbits = (uint64_t)a.cg * v;
    } else if (a.kind == GC_AFOR) {
      const uint32_t byte = a.ctrl[u];
      const uint32_t code = byte >> 6, b = byte & 63u;
      if (code > 2 || b > 32) {
        if (emit && row < a.R) report(a.status, GC_ERR_CORRUPT, (uint32_t)u);
        urows = 32;
        lbits = 0;
      } else {
        urows = 8u << code;
        lbits = urows * b;
      }
      cbit = 8 * u;
    } else {
      const uint32_t hdr = read_le(a.ctrl, a.ctrl_bytes, 4 * u, 4);
      const uint32_t b = hdr & 63u, wc = (hdr >> 6) & 3u, e = hdr >> 8;
      urows = kPfdFrameRows;
      lbits = (uint64_t)kPfdFrameRows * (b > 32 ? 0 : b);
      xb = (uint64_t)e * (pb + (1u << (wc > 2 ? 2 : wc)));
      cbit = 32 * u;
      (void)nf;
    }
    if (emit && row < a.R) put(row, urows, lb, cbit, xo);
    row += urows;
    lb += lbits;
    xo += xb;
    s.rows += urows;
    s.lbits += lbits;
    s.xbytes += xb;
  }
  return s;
}

__device__ __forceinline__ UnitAgg agg_add(UnitAgg x, UnitAgg y) {
  return UnitAgg{x.rows + y.rows, x.lbits + y.lbits, x.xbytes + y.xbytes};
}

// Block-wide exclusive scan of UnitAgg (256 threads); returns the exclusive
// value and writes the block total.
__device__ UnitAgg block_excl_scan(UnitAgg v, UnitAgg* total) {
  __shared__ UnitAgg warp_tot[kIndexThreads / 32];
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  UnitAgg inc;
  inc.rows = warp_incl_sum(v.rows);
  inc.lbits = warp_incl_sum(v.lbits);
  inc.xbytes = warp_incl_sum(v.xbytes);
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  UnitAgg wbase = {0, 0, 0}, tot = {0, 0, 0};
  for (int i = 0; i < kIndexThreads / 32; ++i) {
    if (i < (int)w) wbase = agg_add(wbase, warp_tot[i]);
    tot = agg_add(tot, warp_tot[i]);
  }
  __syncthreads();
  *total = tot;
  return UnitAgg{wbase.rows + inc.rows - v.rows, wbase.lbits + inc.lbits - v.lbits,
                 wbase.xbytes + inc.xbytes - v.xbytes};
}

__global__ void __launch_bounds__(kIndexThreads) k_index_sums(IndexArgs a) {
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  UnitAgg v = {0, 0, 0};
  if (c < a.nchunks) v = walk_chunk(a, c, false, v);
  UnitAgg tot;
  block_excl_scan(v, &tot);
  if (threadIdx.x == 0) a.block_sums[blockIdx.x] = tot;
}

// One block: exclusive scan of the block sums in place.
__global__ void __launch_bounds__(kIndexThreads) k_index_scan(UnitAgg* sums, uint64_t nblocks) {
  UnitAgg carry = {0, 0, 0};
  for (uint64_t b0 = 0; b0 < nblocks; b0 += kIndexThreads) {
    const uint64_t i = b0 + threadIdx.x;
    UnitAgg v = i < nblocks ? sums[i] : UnitAgg{0, 0, 0};
    UnitAgg tot;
    UnitAgg ex = block_excl_scan(v, &tot);
    if (i < nblocks) sums[i] = agg_add(carry, ex);
    carry = agg_add(carry, tot);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kIndexThreads) k_index_emit(IndexArgs a) {
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0) a.tiles[0] = gc_tile{0, 0, 0, 0, 0, GC_TILE_BASE};  // tile 0 starts at unit 0
  UnitAgg v = {0, 0, 0};
  if (c < a.nchunks) v = walk_chunk(a, c, false, v);
  UnitAgg tot;
  UnitAgg ex = block_excl_scan(v, &tot);
  if (c < a.nchunks) walk_chunk(a, c, true, agg_add(a.block_sums[blockIdx.x], ex));
}

// The head of the paper's single buffer (Sec 4.3 step 1): the data area's
// offset in 4-byte words, then, after the control area, zeros up to the
// data area's 16-byte boundary. One thread per byte of the padding.
__global__ void k_paper_head(uint8_t* buf, uint64_t ctrl_bytes, uint32_t off_words) {
  const uint32_t i = threadIdx.x;
  if (i == 0) *reinterpret_cast<uint32_t*>(buf) = off_words;
  const uint64_t pad0 = 4 + ctrl_bytes, pad1 = 4ull * off_words;
  if (pad0 + i < pad1) buf[pad0 + i] = 0;
}

}  // namespace gcidx

namespace gc_host {

using namespace gcidx;

uint64_t index_nunits(const gc_codec& c, uint64_t R, uint64_t ctrl_bytes) {
  switch (c.kind) {
    case GC_SIMPLE: return 2 * ctrl_bytes;
    case GC_SCHEME: return c.ld == GC_LD_BINARY ? R : ctrl_bytes;
    case GC_AFOR: return ctrl_bytes;
    default: return (R + kPfdFrameRows - 1) / kPfdFrameRows;
  }
}

uint64_t index_chunks(const gc_codec& c, uint64_t nunits) {
  if (c.kind == GC_SCHEME && c.ld != GC_LD_BINARY) return (nunits + kChunkBytes - 1) / kChunkBytes;
  return (nunits + kChunkUnits - 1) / kChunkUnits;
}

uint64_t index_sums_bytes(const gc_codec& c, uint64_t n) {
  // bound the control bytes by the encoder's maximum
  uint64_t cc = 0, dc = 0, nt = 0;
  gc_max_encoded_size(&c, n, &cc, &dc, &nt);
  const uint64_t R = (n + c.k - 1) / c.k;
  const uint64_t chunks = index_chunks(c, index_nunits(c, R, cc));
  const uint64_t blocks = (chunks + kIndexThreads - 1) / kIndexThreads;
  (void)dc;
  (void)nt;
  return gc_host::align_up(blocks * sizeof(UnitAgg) + 64, 256);
}

gc_status build_tiles(const gc_codec& c, const uint8_t* ctrl, uint64_t ctrl_bytes, uint64_t n, gc_tile* tiles,
                      void* d_sums, uint32_t* status, cudaStream_t s) {
  UnitAgg* sums = (UnitAgg*)d_sums;
  const uint64_t R = (n + c.k - 1) / c.k;
  const uint64_t tr = kTileInts / c.k;
  const uint64_t nt = (R + tr - 1) / tr;
  if (nt == 0) return GC_OK;
  IndexArgs a;
  a.kind = c.kind;
  a.k = c.k;
  a.cg = c.cg;
  a.ld = c.ld;
  a.ctrl = ctrl;
  a.ctrl_bytes = ctrl_bytes;
  a.n = n;
  a.R = R;
  a.nunits = index_nunits(c, R, ctrl_bytes);
  if (c.kind == GC_PFD && 4 * a.nunits > ctrl_bytes) return GC_ERR_INVALID;
  if (c.kind == GC_SCHEME && c.ld == GC_LD_BINARY && bin_ld_bytes(R, c.cg) > ctrl_bytes) return GC_ERR_INVALID;
  a.nchunks = index_chunks(c, a.nunits);
  a.tiles = tiles;
  a.ntiles = nt;
  a.block_sums = sums;
  a.status = status;
  const uint64_t blocks = (a.nchunks + kIndexThreads - 1) / kIndexThreads;
  if (blocks == 0) return GC_ERR_INVALID;
  k_index_sums<<<(unsigned)blocks, kIndexThreads, 0, s>>>(a);
  k_index_scan<<<1, kIndexThreads, 0, s>>>(sums, blocks);
  k_index_emit<<<(unsigned)blocks, kIndexThreads, 0, s>>>(a);
  gc_host::count_launch(3);
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

}  // namespace gc_host

extern "C" {

gc_status gc_build_tiles(const gc_codec* codec, const uint8_t* d_ctrl, uint64_t ctrl_bytes, uint64_t n,
                         gc_tile* d_tiles, void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status,
                         void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (n == 0) return GC_OK;
  if ((!d_ctrl && ctrl_bytes) || !d_tiles || !d_scratch) return GC_ERR_INVALID;
  if (scratch_bytes < gc_host::index_sums_bytes(*codec, n)) return GC_ERR_NOSPACE;
  return gc_host::build_tiles(*codec, d_ctrl, ctrl_bytes, n, d_tiles, d_scratch, d_status, (cudaStream_t)stream);
}

uint64_t gc_paper_bytes(uint64_t ctrl_bytes, uint64_t data_words) {
  return gc_host::align_up(4 + ctrl_bytes, 16) + 4 * data_words;
}

gc_status gc_pack_paper(const uint8_t* d_ctrl, uint64_t ctrl_bytes, const uint32_t* d_data, uint64_t data_words,
                        uint8_t* d_buf, uint64_t buf_bytes, void* stream) {
  gc_host::reset_launches();
  if ((!d_ctrl && ctrl_bytes) || (!d_data && data_words) || !d_buf) return GC_ERR_INVALID;
  if (((uintptr_t)d_buf & 15) != 0) return GC_ERR_INVALID;
  const uint64_t doff = gc_host::align_up(4 + ctrl_bytes, 16);
  if (doff / 4 > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  if (buf_bytes < gc_paper_bytes(ctrl_bytes, data_words)) return GC_ERR_NOSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  gcidx::k_paper_head<<<1, 16, 0, s>>>(d_buf, ctrl_bytes, (uint32_t)(doff / 4));
  gc_host::count_launch();
  if (cudaGetLastError() != cudaSuccess) return GC_ERR_CUDA;
  if (ctrl_bytes && cudaMemcpyAsync(d_buf + 4, d_ctrl, ctrl_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GC_ERR_CUDA;
  if (data_words && cudaMemcpyAsync(d_buf + doff, d_data, 4 * data_words, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GC_ERR_CUDA;
  return GC_OK;
}

gc_status gc_unpack_paper(const uint8_t* d_buf, uint64_t buf_bytes, uint8_t* d_ctrl, uint64_t ctrl_cap,
                          uint32_t* d_data, uint64_t data_cap, uint64_t* ctrl_bytes, uint64_t* data_words,
                          void* stream) {
  gc_host::reset_launches();
  if (!d_buf || buf_bytes < 4 || !ctrl_bytes || !data_words) return GC_ERR_INVALID;
  if (((uintptr_t)d_buf & 15) != 0) return GC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t off_words = 0;
  if (cudaMemcpyAsync(&off_words, d_buf, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GC_ERR_CUDA;
  const uint64_t doff = 4ull * off_words;
  if (doff < 4 || doff > buf_bytes || (doff & 15)) return GC_ERR_CORRUPT;
  const uint64_t cb = doff - 4, dw = (buf_bytes - doff) / 4;
  *ctrl_bytes = cb;
  *data_words = dw;
  if (cb > ctrl_cap || dw > data_cap) return GC_ERR_NOSPACE;
  if ((!d_ctrl && cb) || (!d_data && dw)) return GC_ERR_INVALID;
  if (cb && cudaMemcpyAsync(d_ctrl, d_buf + 4, cb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GC_ERR_CUDA;
  if (dw && cudaMemcpyAsync(d_data, d_buf + doff, 4 * dw, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GC_ERR_CUDA;
  return GC_OK;
}

}  // extern "C"
