// gc_encode.cu -- GPU encoders of the Group-codec library.
//
// Every list of a batch is encoded on the device, and the streams equal
// the paper's procedures bit for bit:
//   - Group-Simple (Sec 4.2): Algorithm 1's choice at every row is computed
//     in parallel (the pattern that would start there); the chain of
//     choices from row 0 is found per 1024-row segment for all 32 possible
//     entry rows, composed per list, and replayed, so the selectors are
//     exactly those of the sequential greedy loop.
//   - Group-Scheme (Sec 5.2.2, Eq. 1): descriptor and width per row; scans
//     give every row's control and lane bit positions (the incomplete-unary
//     byte rule is a short sequential walk per list).
//   - Group-AFOR (Sec 6.1): the size-minimising partition into frames of
//     8/16/32 rows by dynamic programming, one thread per list.
//   - Group-PFD (Sec 6.2, Steps 1-4): one warp per 32-row frame finds b,
//     the exceptions and their width.
// Tile records also carry skip entries (Sec 7.5 keeps a docID every so many
// postings): the docID before each tile, from per-tile gap sums and a scan.
// Row maxima are the effective widths of the k ints of each row (Sec 4.2).
// Lists are laid out back to back; tile records for tiles >= 1 (or all
// tiles, for a single list) are written by the same passes.
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "gc_device.cuh"
#include "gc_host.h"

namespace gcenc {

using namespace gcdev;

constexpr int kSeg = 1024;  // Group-Simple chain segment, rows
constexpr int kT = 256;     // threads per block

struct Enc {
  uint32_t kind, k, cg, ld, T, tr;
  uint32_t include_tile0;
  uint64_t nlists, Rtot, Utot;  // Utot: codec units index space
  uint64_t Atot;                // tiles of all lists, tile 0 included
  const uint32_t* gaps;
  // per list
  const uint32_t* n;
  const uint64_t* in_off;
  const uint64_t* rowbase;   // nlists + 1
  const uint64_t* tilebase;  // nlists + 1
  const uint64_t* ubase;     // nlists + 1 (PFD frames, AFOR blocks + 1, GS segments)
  const uint64_t* abase;     // nlists + 1: first tile of each list, tile 0 included
  uint64_t* tsum;            // Atot + 1: gap sum per tile, then its exclusive scan
  uint64_t* csize;           // nlists + 1: control bytes, then exclusive offsets
  uint64_t* dsize;           // nlists + 1: data words, then exclusive offsets
  uint64_t* aux;             // nlists + 1: GS selectors / AFOR frames per list, then offsets
  // per row
  uint8_t* eb;
  uint32_t* rlist;
  // per unit / per row, codec specific
  uint64_t* s0;  // scan buffer (Utot + 1 or Rtot + 1)
  uint64_t* s1;  // second scan buffer
  uint8_t* u8a;
  uint8_t* u8b;
  uint32_t* u32a;
  uint32_t* u32b;
  // outputs
  uint8_t* ctrl;
  uint32_t* data;
  gc_tile* tiles;
  gc_list* lists;
  uint64_t* totals;  // ctrl bytes, data words, tile records
  uint32_t* status;
};

__device__ __forceinline__ uint64_t find_list(const uint64_t* base, uint64_t nlists, uint64_t g) {
  // largest i with base[i] <= g (base is nondecreasing, base[0] = 0)
  uint64_t lo = 0, hi = nlists;  // invariant: base[lo] <= g < base[hi] (base[nlists] = total)
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (base[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t gap_at(const Enc& e, uint64_t list, uint64_t i) {
  return i < e.n[list] ? e.gaps[e.in_off[list] + i] : 0u;
}

__device__ __forceinline__ uint64_t tile_slot(const Enc& e, uint64_t list, uint64_t t) {
  return e.tilebase[list] + t - (e.include_tile0 ? 0 : 1);
}

__device__ __forceinline__ void put_tile(const Enc& e, uint64_t list, uint64_t t, uint64_t lane_bit,
                                         uint64_t ctrl_bit, uint64_t exc, uint64_t skip) {
  if (!e.tiles || (t == 0 && !e.include_tile0)) return;
  gc_tile g;
  g.lane_bit = lane_bit;
  g.ctrl_bit = ctrl_bit;
  g.exc_off = (uint32_t)exc;
  g.row_skip = (uint32_t)skip;
  g.base = 0;  // written by k_put_bases
  g.flags = t == 0 ? GC_TILE_BASE : 0u;
  e.tiles[tile_slot(e, list, t)] = g;
}

// tiles whose first row lies in [row, row + rows) of a list with R rows
__device__ __forceinline__ void put_tiles_in(const Enc& e, uint64_t list, uint64_t R, uint64_t row,
                                             uint64_t rows, uint64_t lane_bit, uint64_t ctrl_bit,
                                             uint64_t exc) {
  for (uint64_t t = (row + e.tr - 1) / e.tr; t * e.tr < row + rows && t * e.tr < R; ++t)
    put_tile(e, list, t, lane_bit, ctrl_bit, exc, t * e.tr - row);
}

// OR `width` (<= 32) bits of v into bit position `bit` of a byte stream kept
// as aligned 32-bit words (the stream base is 4-byte aligned).
__device__ __forceinline__ void or_bits(uint8_t* base, uint64_t bit, uint32_t v, uint32_t width) {
  if (width == 0) return;
  uint32_t* w = reinterpret_cast<uint32_t*>(base);
  v &= low_mask(width);
  const uint64_t wi = bit >> 5;
  const uint32_t off = (uint32_t)bit & 31u;
  if (v << off) atomicOr(w + wi, v << off);
  if (off + width > 32 && (v >> (32 - off))) atomicOr(w + wi + 1, v >> (32 - off));
}

// OR the low `width` bits of v into lane j's stream at lane bit `lbit`.
__device__ __forceinline__ void or_lane(uint32_t* data, uint32_t k, uint32_t j, uint64_t lbit, uint32_t v,
                                        uint32_t width) {
  if (width == 0) return;
  v &= low_mask(width);
  const uint64_t wi = lbit >> 5;
  const uint32_t off = (uint32_t)lbit & 31u;
  if (v << off) atomicOr(data + wi * k + j, v << off);
  if (off + width > 32 && (v >> (32 - off))) atomicOr(data + (wi + 1) * k + j, v >> (32 - off));
}

// ----------------------------------------------------------- u64 scan
// In place: buf[0..n) becomes its exclusive prefix sum, buf[n] the total.

constexpr int kScanItems = 4;
constexpr uint64_t kScanBlock = (uint64_t)kT * kScanItems;

__device__ uint64_t block_excl_u64(uint64_t v, uint64_t* total) {
  __shared__ uint64_t wt[kT / 32];
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const uint64_t inc = warp_incl_sum(v);
  if (lane == 31) wt[w] = inc;
  __syncthreads();
  uint64_t base = 0, tot = 0;
  for (int i = 0; i < kT / 32; ++i) {
    if (i < (int)w) base += wt[i];
    tot += wt[i];
  }
  __syncthreads();
  *total = tot;
  return base + inc - v;
}

__global__ void k_scan_sums(const uint64_t* buf, uint64_t n, uint64_t* sums) {
  const uint64_t b0 = (uint64_t)blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * kScanItems;
  uint64_t v = 0;
  for (int i = 0; i < kScanItems; ++i)
    if (b0 + i < n) v += buf[b0 + i];
  uint64_t tot;
  block_excl_u64(v, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(uint64_t* sums, uint64_t nb) {
  uint64_t carry = 0;
  for (uint64_t b0 = 0; b0 < nb; b0 += kT) {
    const uint64_t i = b0 + threadIdx.x;
    const uint64_t v = i < nb ? sums[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_excl_u64(v, &tot);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_down(uint64_t* buf, uint64_t n, const uint64_t* sums) {
  const uint64_t b0 = (uint64_t)blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * kScanItems;
  uint64_t x[kScanItems];
  uint64_t v = 0;
  for (int i = 0; i < kScanItems; ++i) {
    x[i] = (b0 + i < n) ? buf[b0 + i] : 0;
    v += x[i];
  }
  uint64_t tot;
  uint64_t run = block_excl_u64(v, &tot) + sums[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    if (b0 + i < n) buf[b0 + i] = run;
    run += x[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kT - 1) buf[n] = sums[gridDim.x];
}

uint64_t scan_tmp_words(uint64_t n) { return (n + kScanBlock - 1) / kScanBlock + 2; }

void scan_u64(uint64_t* buf, uint64_t n, uint64_t* tmp, cudaStream_t s) {
  const uint64_t nb = (n + kScanBlock - 1) / kScanBlock;
  if (nb == 0) {
    cudaMemsetAsync(buf, 0, 8, s);
    return;
  }
  k_scan_sums<<<(unsigned)nb, kT, 0, s>>>(buf, n, tmp);
  k_scan_top<<<1, kT, 0, s>>>(tmp, nb);
  k_scan_down<<<(unsigned)nb, kT, 0, s>>>(buf, n, tmp);
  gc_host::count_launch(3);
}

// ------------------------------------------------------------- rows

__global__ void k_rows(Enc e) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= e.Rtot) return;
  const uint64_t L = find_list(e.rowbase, e.nlists, g);
  const uint64_t r = g - e.rowbase[L];
  uint32_t m = 0;
  for (uint32_t j = 0; j < e.k; ++j) m = max(m, gap_at(e, L, r * e.k + j));
  e.eb[g] = (uint8_t)eff_bits(m);
  e.rlist[g] = (uint32_t)L;
}

// Per list: csize/dsize -> offsets (after the scans), then the descriptor.
__global__ void k_lists_out(Enc e) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < e.nlists) {
    gc_list d;
    d.ctrl_off = e.csize[i];
    d.data_off = e.dsize[i];
    d.out_off = e.in_off[i];
    d.n = e.n[i];
    d.tile_off = (uint32_t)e.tilebase[i];
    d.ctrl_bytes = (uint32_t)(e.csize[i + 1] - e.csize[i]);
    d.data_words = (uint32_t)(e.dsize[i + 1] - e.dsize[i]);
    e.lists[i] = d;
  }
  if (i == 0) {
    e.totals[0] = e.csize[e.nlists];
    e.totals[1] = e.dsize[e.nlists];
    e.totals[2] = e.tilebase[e.nlists];
  }
}

// Skip entries: one warp per tile (tile 0 included) sums the tile's gaps;
// after an exclusive scan of the sums over all tiles, the base of tile t of
// list L is its scanned value minus that of the list's tile 0 (sums of
// uint32 gaps modulo 2^32, the docID before the tile, Sec 2.1.1).
__global__ void k_tile_sums(Enc e) {
  const uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (g >= e.Atot) return;  // uniform per warp
  const uint64_t L = find_list(e.abase, e.nlists, g);
  const uint64_t i0 = (g - e.abase[L]) * 1024;
  const uint64_t i1 = min64(e.n[L], i0 + 1024);
  uint32_t s = 0;
  for (uint64_t i = i0 + lane_id(); i < i1; i += 32) s += e.gaps[e.in_off[L] + i];
  s = warp_sum(s);
  if (lane_id() == 0) e.tsum[g] = s;
}

__global__ void k_put_bases(Enc e) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= e.Atot || !e.tiles) return;
  const uint64_t L = find_list(e.abase, e.nlists, g);
  const uint64_t t = g - e.abase[L];
  if (t == 0 && !e.include_tile0) return;
  gc_tile* r = e.tiles + tile_slot(e, L, t);
  r->base = (uint32_t)(e.tsum[g] - e.tsum[e.abase[L]]);
  r->flags = GC_TILE_BASE;
}

// ------------------------------------------------------- Group-PFD

// One warp per frame (32 rows): b (Step 2), exceptions (Step 3), sizes.
// u8a = b, u8b = width code, u32a = e; s0 = exception bytes, s1 = lane bits.
__global__ void k_pfd_frames(Enc e) {
  const uint64_t F = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (F >= e.Utot) return;
  const uint32_t lane = lane_id();
  const uint64_t L = find_list(e.ubase, e.nlists, F);
  const uint64_t f = F - e.ubase[L];
  const uint64_t R = e.rowbase[L + 1] - e.rowbase[L];
  const uint64_t r0 = f * kPfdFrameRows;
  const uint32_t frows = (uint32_t)min64(kPfdFrameRows, R - r0);
  const uint32_t myb = lane < frows ? e.eb[e.rowbase[L] + r0 + lane] : 0u;
  // the frame's own exception ratio: a list's last frame of fewer rows may
  // have the 32-row budget scaled to its rows (rounded down)
  const uint32_t budget = e.T * frows / kPfdFrameRows;
  uint32_t b = 0;
  for (; b < 32; ++b)
    if ((uint32_t)__popc(__ballot_sync(kFull, myb > b)) <= budget) break;
  // exceptions: ints above 2^b - 1 in rows whose max is above it
  uint32_t rowsx = __ballot_sync(kFull, myb > b);
  uint32_t cnt = 0, vmax = 0;
  while (rowsx) {
    const uint32_t q = __ffs(rowsx) - 1;
    rowsx &= rowsx - 1;
    for (uint32_t j0 = 0; j0 < e.k; j0 += 32) {
      const uint32_t j = j0 + lane;
      const uint32_t v = j < e.k ? gap_at(e, L, (r0 + q) * e.k + j) : 0u;
      const bool x = j < e.k && eff_bits(v) > b;
      cnt += __popc(__ballot_sync(kFull, x));
      uint32_t m = x ? v : 0u;
      for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
      vmax = max(vmax, m);
    }
  }
  if (lane == 0) {
    const uint32_t wc = cnt == 0 ? 0u : vmax < 256u ? 0u : vmax < 65536u ? 1u : 2u;
    const uint32_t pb = (kPfdFrameRows * e.k) <= 256 ? 1u : 2u;
    e.u8a[F] = (uint8_t)b;
    e.u8b[F] = (uint8_t)wc;
    e.u32a[F] = cnt;
    e.s0[F] = (uint64_t)cnt * (pb + (1u << wc));
    e.s1[F] = (uint64_t)frows * b;
  }
}

__global__ void k_pfd_sizes(Enc e) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.nlists) return;
  const uint64_t f0 = e.ubase[i], f1 = e.ubase[i + 1];
  const uint64_t nf = f1 - f0;
  e.csize[i] = 4 * nf + (e.s0[f1] - e.s0[f0]);
  e.dsize[i] = e.k * ((e.s1[f1] - e.s1[f0] + 31) / 32);
}

// Step 4: one warp per frame writes the header, the exception record and
// the frame's lane words (each frame owns whole words of every lane).
__global__ void k_pfd_pack(Enc e) {
  const uint64_t F = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (F >= e.Utot) return;
  const uint32_t lane = lane_id();
  const uint64_t L = find_list(e.ubase, e.nlists, F);
  const uint64_t f0 = e.ubase[L];
  const uint64_t f = F - f0;
  const uint64_t nf = e.ubase[L + 1] - f0;
  const uint64_t R = e.rowbase[L + 1] - e.rowbase[L];
  const uint64_t r0 = f * kPfdFrameRows;
  const uint32_t frows = (uint32_t)min64(kPfdFrameRows, R - r0);
  const uint32_t b = e.u8a[F], wc = e.u8b[F], cnt = e.u32a[F];
  const uint32_t pb = (kPfdFrameRows * e.k) <= 256 ? 1u : 2u;
  const uint32_t wb = 1u << wc;
  uint8_t* ctrl = e.ctrl + e.csize[L];
  uint32_t* data = e.data + e.dsize[L];
  const uint64_t xoff = e.s0[F] - e.s0[f0];
  const uint64_t lbit = e.s1[F] - e.s1[f0];
  if (lane < 4) ctrl[4 * f + lane] = (uint8_t)((b | (wc << 6) | (cnt << 8)) >> (8 * lane));
  // exception record, in position order
  uint8_t* rec = ctrl + 4 * nf + xoff;
  const uint32_t myb = lane < frows ? e.eb[e.rowbase[L] + r0 + lane] : 0u;
  uint32_t rowsx = __ballot_sync(kFull, myb > b);
  uint32_t x0 = 0;
  while (rowsx) {
    const uint32_t q = __ffs(rowsx) - 1;
    rowsx &= rowsx - 1;
    for (uint32_t j0 = 0; j0 < e.k; j0 += 32) {
      const uint32_t j = j0 + lane;
      const uint32_t v = j < e.k ? gap_at(e, L, (r0 + q) * e.k + j) : 0u;
      const bool x = j < e.k && eff_bits(v) > b;
      const uint32_t m = __ballot_sync(kFull, x);
      if (x) {
        const uint32_t idx = x0 + __popc(m & ((1u << lane) - 1u));
        const uint32_t pos = q * e.k + j;
        for (uint32_t t = 0; t < pb; ++t) rec[(uint64_t)idx * pb + t] = (uint8_t)(pos >> (8 * t));
        for (uint32_t t = 0; t < wb; ++t) rec[(uint64_t)cnt * pb + (uint64_t)idx * wb + t] = (uint8_t)(v >> (8 * t));
      }
      x0 += __popc(m);
    }
  }
  // slots: lane j packs its rows into whole words
  const uint32_t msk = low_mask(b);
  for (uint32_t j = lane; j < e.k; j += 32) {
    if (b == 0) break;
    uint64_t acc = 0;
    uint32_t nb = 0;
    uint64_t wi = lbit >> 5;  // lbit is a multiple of 32 here
    for (uint32_t q = 0; q < frows; ++q) {
      acc |= (uint64_t)(gap_at(e, L, (r0 + q) * e.k + j) & msk) << nb;
      nb += b;
      if (nb >= 32) {
        data[wi * e.k + j] = (uint32_t)acc;
        ++wi;
        acc >>= 32;
        nb -= 32;
      }
    }
    if (nb) data[wi * e.k + j] = (uint32_t)acc;
  }
  if (lane == 0) {
    // a tile starts at every (1024/k)-row boundary, which is a frame start
    if (r0 % e.tr == 0) put_tile(e, L, r0 / e.tr, lbit, 32 * f, xoff, 0);
  }
}

// ---------------------------------------------------- Group-Scheme

// Per row: unit count (Eq. 1) in u8a; width into s1 (scan -> lane bit
// offsets); unary descriptor length into s0 (scan -> control offsets, CU).
__global__ void k_gsc_rows(Enc e) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= e.Rtot) return;
  uint32_t u = (e.eb[g] + e.cg - 1) / e.cg;
  if (u == 0) u = 1;
  e.u8a[g] = (uint8_t)u;
  e.s1[g] = (uint64_t)e.cg * u;
  e.s0[g] = u;
}

// Incomplete unary: descriptors never straddle a byte (Sec 5.2.1(a)). A
// walk per list gives each row's control bit (relative to the list) in s0
// and the list's control bytes.
__global__ void k_gsc_iu_walk(Enc e) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.nlists) return;
  uint64_t pos = 0;
  for (uint64_t g = e.rowbase[i]; g < e.rowbase[i + 1]; ++g) {
    const uint32_t u = e.u8a[g];
    if ((pos & 7) + u > 8) pos = (pos + 7) & ~7ull;
    e.s0[g] = pos;
    pos += u;
  }
  e.csize[i] = (pos + 7) / 8;
}

__global__ void k_gsc_sizes(Enc e) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.nlists) return;
  const uint64_t g0 = e.rowbase[i], g1 = e.rowbase[i + 1];
  const uint64_t R = g1 - g0;
  if (e.ld == GC_LD_BINARY) e.csize[i] = bin_ld_bytes(R, e.cg);
  else if (e.ld == GC_LD_CU) e.csize[i] = (e.s0[g1] - e.s0[g0] + 7) / 8;
  // IU: set by the walk
  e.dsize[i] = e.k * ((e.s1[g1] - e.s1[g0] + 31) / 32);
}

// Per row: descriptor bits, padding ones after it (unary), tile record.
__global__ void k_gsc_ctrl(Enc e) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= e.Rtot) return;
  const uint64_t L = e.rlist[g];
  const uint64_t g0 = e.rowbase[L], g1 = e.rowbase[L + 1];
  const uint64_t r = g - g0;
  const uint32_t u = e.u8a[g];
  const uint64_t cbase = 8 * e.csize[L];  // list's first control bit in the pool
  uint64_t cpos;
  if (e.ld == GC_LD_BINARY) {
    cpos = bin_ld_pos(r, e.cg);
    or_bits(e.ctrl, cbase + cpos, u - 1, 5 - log2_cg(e.cg));
  } else {
    cpos = e.ld == GC_LD_CU ? e.s0[g] - e.s0[g0] : e.s0[g];
    or_bits(e.ctrl, cbase + cpos, low_mask(u - 1), u - 1);  // (u-1) ones, the zero is implicit
    // padding ones up to the next descriptor (IU) or to the end of the last byte
    uint64_t next;
    if (g + 1 < g1) next = e.ld == GC_LD_CU ? e.s0[g + 1] - e.s0[g0] : e.s0[g + 1];
    else next = (cpos + u + 7) & ~7ull;
    for (uint64_t p = cpos + u; p < next; p += 32) {
      const uint32_t w = (uint32_t)min64(32, next - p);
      or_bits(e.ctrl, cbase + p, 0xffffffffu, w);
    }
  }
  if (r % e.tr == 0) put_tile(e, L, r / e.tr, e.s1[g] - e.s1[g0], cpos, 0, 0);
}

// Per (row, lane): the value at its width into the lane stream.
__global__ void k_gsc_data(Enc e) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= e.Rtot * e.k) return;
  const uint64_t g = t / e.k;
  const uint32_t j = (uint32_t)(t % e.k);
  const uint64_t L = e.rlist[g];
  const uint64_t g0 = e.rowbase[L];
  const uint32_t v = gap_at(e, L, (g - g0) * e.k + j);
  or_lane(e.data + e.dsize[L], e.k, j, e.s1[g] - e.s1[g0], v, e.cg * e.u8a[g]);
}

// ------------------------------------------------------- Group-AFOR
// Blocks of 8 rows; unit index space per list: nb + 1 slots.
// u8a[B] = max width of the block's rows.

__global__ void k_afor_blocks(Enc e) {
  const uint64_t B = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (B >= e.Utot) return;
  const uint64_t L = find_list(e.ubase, e.nlists, B);
  const uint64_t p = B - e.ubase[L];
  const uint64_t R = e.rowbase[L + 1] - e.rowbase[L];
  uint32_t m = 0;
  for (uint64_t r = 8 * p; r < 8 * p + 8 && r < R; ++r) m = max(m, (uint32_t)e.eb[e.rowbase[L] + r]);
  e.u8a[B] = (uint8_t)m;
}

// Dynamic programming from the end: best[p] = min over F in {32,16,8} of
// 8 + k*F*b(p, F) + best[p + F/8]; ties go to the larger frame. Then the
// partition from row 0. Frames go to the list's slots: u8b = size code,
// u32a = first block, s1 = lane bits (F*b) for the scan; u32b[B] = frame
// index of block B.
__global__ void k_afor_dp(Enc e) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.nlists) return;
  const uint64_t B0 = e.ubase[i];
  const uint64_t nb = e.ubase[i + 1] - B0 - 1;
  uint64_t* best = e.s0 + B0;  // nb + 1 slots
  best[nb] = 0;
  for (uint64_t p = nb; p-- > 0;) {
    uint64_t bb = ~0ull;
    uint32_t choice = 0;
    uint32_t w = 0;
    const uint32_t sizes[3] = {8, 16, 32};
    uint64_t cand[3] = {~0ull, ~0ull, ~0ull};
    for (int s = 0; s < 3; ++s) {
      const uint32_t nbk = sizes[s] / 8;
      if (p + nbk > nb) break;
      for (uint32_t q = (s == 0 ? 0 : sizes[s - 1] / 8); q < nbk; ++q) w = max(w, (uint32_t)e.u8a[B0 + p + q]);
      cand[s] = 8 + (uint64_t)e.k * sizes[s] * w + best[p + nbk];
    }
    for (int s = 2; s >= 0; --s)
      if (cand[s] < bb) { bb = cand[s]; choice = (uint32_t)s; }
    best[p] = bb;
    e.u8b[B0 + p] = (uint8_t)choice;  // temporarily: choice per block
  }
  // walk: frames written to slots [B0, B0 + nfr)
  uint64_t nfr = 0;
  for (uint64_t p = 0; p < nb;) {
    const uint32_t code = e.u8b[B0 + p];
    const uint32_t nbk = 1u << code;
    uint32_t w = 0;
    for (uint32_t q = 0; q < nbk; ++q) w = max(w, (uint32_t)e.u8a[B0 + p + q]);
    for (uint32_t q = 0; q < nbk; ++q) e.u32b[B0 + p + q] = (uint32_t)nfr;
    e.u32a[B0 + nfr] = (uint32_t)p;
    e.s1[B0 + nfr] = (uint64_t)(8u << code) * w;
    // the frame's control byte goes to slot nfr of u8a: nfr <= p, so every
    // block max still to be read (blocks >= p + nbk) is intact
    e.u8a[B0 + nfr] = (uint8_t)((code << 6) | w);
    ++nfr;
    p += nbk;
  }
  for (uint64_t q = nfr; q <= nb; ++q) e.s1[B0 + q] = 0;
  e.aux[i] = nfr;
}

__global__ void k_afor_sizes(Enc e) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.nlists) return;
  const uint64_t B0 = e.ubase[i], B1 = e.ubase[i + 1];
  e.csize[i] = e.aux[i];
  e.dsize[i] = e.k * ((e.s1[B1] - e.s1[B0] + 31) / 32);
}

// Per frame slot: control byte and tile records.
__global__ void k_afor_ctrl(Enc e) {
  const uint64_t B = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (B >= e.Utot) return;
  const uint64_t L = find_list(e.ubase, e.nlists, B);
  const uint64_t B0 = e.ubase[L];
  const uint64_t fi = B - B0;
  if (fi >= e.aux[L]) return;
  const uint32_t byte = e.u8a[B];
  e.ctrl[e.csize[L] + fi] = (uint8_t)byte;
  const uint64_t R = e.rowbase[L + 1] - e.rowbase[L];
  const uint64_t row = 8ull * e.u32a[B];
  put_tiles_in(e, L, R, row, 8u << (byte >> 6), e.s1[B] - e.s1[B0], 8 * fi, 0);
}

// Per (row, lane): value at the frame's width.
__global__ void k_afor_data(Enc e) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= e.Rtot * e.k) return;
  const uint64_t g = t / e.k;
  const uint32_t j = (uint32_t)(t % e.k);
  const uint64_t L = e.rlist[g];
  const uint64_t r = g - e.rowbase[L];
  const uint64_t B0 = e.ubase[L];
  const uint64_t fi = e.u32b[B0 + r / 8];
  const uint32_t byte = e.u8a[B0 + fi];
  const uint32_t b = byte & 63u;
  const uint64_t frow = 8ull * e.u32a[B0 + fi];
  const uint64_t lbit = e.s1[B0 + fi] - e.s1[B0] + (r - frow) * b;
  or_lane(e.data + e.dsize[L], e.k, j, lbit, gap_at(e, L, r * e.k + j), b);
}

// ---------------------------------------------------- Group-Simple
// u8a[g] = Algorithm 1's selector for a run starting at row g, u8b[g] = the
// rows it takes (pos).

__global__ void k_gs_choice(Enc e) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= e.Rtot) return;
  const uint64_t L = e.rlist[g];
  const uint64_t l = e.rowbase[L + 1] - g;  // rows left in the list
  uint32_t sel = 9, pos = 1;
  for (uint32_t i = 0; i < 10; ++i) {
    const uint32_t num = sel_num(i), bw = sel_bw(i);
    const uint64_t lim = num < l ? num : l;
    uint32_t p = 0;
    while (p < lim && e.eb[g + p] <= bw) ++p;
    if (p == num || p == l) { sel = i; pos = p; break; }
  }
  e.u8a[g] = (uint8_t)sel;
  e.u8b[g] = (uint8_t)pos;
}

// Per (segment, entry row 0..31): follow the chain inside the segment;
// u32a = selectors taken, u8... exit offset packed in the high byte.
__global__ void k_gs_segments(Enc e) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t S = t >> 5;
  if (S >= e.Utot) return;
  const uint32_t ent = (uint32_t)(t & 31);
  const uint64_t L = find_list(e.ubase, e.nlists, S);
  const uint64_t s = S - e.ubase[L];
  const uint64_t R = e.rowbase[L + 1] - e.rowbase[L];
  const uint64_t seg_end = min64((s + 1) * kSeg, R);
  uint64_t r = s * kSeg + ent;
  uint32_t cnt = 0;
  while (r < seg_end) {
    r += e.u8b[e.rowbase[L] + r];
    ++cnt;
  }
  const uint32_t exit = r >= R ? 0u : (uint32_t)(r - seg_end);
  e.u32b[t] = cnt | (exit << 24);
}

// Per list: compose the segments from entry 0; s0[S] = selectors before
// segment S (in the list), u8a-like entry kept in u32a[S].
__global__ void k_gs_compose(Enc e) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.nlists) return;
  uint32_t ent = 0;
  uint64_t run = 0;
  for (uint64_t S = e.ubase[i]; S < e.ubase[i + 1]; ++S) {
    const uint32_t v = e.u32b[S * 32 + ent];
    e.s0[S] = run;
    e.u32a[S] = ent;
    run += v & 0xffffffu;
    ent = v >> 24;
  }
  e.aux[i] = run;
}

__global__ void k_gs_sizes(Enc e) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.nlists) return;
  e.csize[i] = (e.aux[i] + 1) / 2;
  e.dsize[i] = e.k * e.aux[i];
}

// Per segment: replay the chain from the actual entry; each selector writes
// its nibble (atomically: two selectors share a byte), its data vector and
// any tile records.
__global__ void k_gs_emit(Enc e) {
  const uint64_t S = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (S >= e.Utot) return;
  const uint64_t L = find_list(e.ubase, e.nlists, S);
  const uint64_t s = S - e.ubase[L];
  const uint64_t R = e.rowbase[L + 1] - e.rowbase[L];
  const uint64_t g0 = e.rowbase[L];
  const uint64_t seg_end = min64((s + 1) * kSeg, R);
  uint64_t r = s * kSeg + e.u32a[S];
  uint64_t idx = e.s0[S];
  const uint64_t cb = 8 * e.csize[L];
  while (r < seg_end) {
    const uint32_t sel = e.u8a[g0 + r];
    const uint32_t pos = e.u8b[g0 + r];
    or_bits(e.ctrl, cb + 4 * idx, sel, 4);
    put_tiles_in(e, L, R, r, pos, 32 * idx, 4 * idx, 0);
    r += pos;
    ++idx;
  }
}

// Per (selector slot, lane): pack the selector's rows into its word. The
// selector of a vector is found from its row via the emitted nibbles, so
// this runs per row instead: row r of the list belongs to the selector
// whose chain position covers it; u32b (reused) holds, per row, the
// selector index of the run containing it, set by k_gs_mark.
__global__ void k_gs_mark(Enc e) {
  const uint64_t S = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (S >= e.Utot) return;
  const uint64_t L = find_list(e.ubase, e.nlists, S);
  const uint64_t s = S - e.ubase[L];
  const uint64_t R = e.rowbase[L + 1] - e.rowbase[L];
  const uint64_t g0 = e.rowbase[L];
  const uint64_t seg_end = min64((s + 1) * kSeg, R);
  uint64_t r = s * kSeg + e.u32a[S];
  uint64_t idx = e.s0[S];
  while (r < seg_end) {
    const uint32_t pos = e.u8b[g0 + r];
    for (uint32_t q = 0; q < pos; ++q) e.s1[g0 + r + q] = (idx << 6) | q;  // selector, row in it
    r += pos;
    ++idx;
  }
}

__global__ void k_gs_data(Enc e) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= e.Rtot * e.k) return;
  const uint64_t g = t / e.k;
  const uint32_t j = (uint32_t)(t % e.k);
  const uint64_t L = e.rlist[g];
  const uint64_t r = g - e.rowbase[L];
  const uint64_t m = e.s1[g];
  const uint64_t idx = m >> 6;
  const uint32_t q = (uint32_t)(m & 63);
  const uint32_t sel = e.u8a[g - q];  // the selector chosen at the run's first row
  const uint32_t bw = sel_bw(sel);
  or_lane(e.data + e.dsize[L], e.k, j, 32 * idx + q * bw, gap_at(e, L, r * e.k + j), bw);
}

// ---------------------------------------------------------------- host

struct Bump {
  unsigned char* base;
  uint64_t off = 0;
  template <class T>
  T* take(uint64_t count) {
    off = gc_host::align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct Plan {
  uint64_t nlists = 0, Rtot = 0, Utot = 0, tiles = 0, ctrl_cap = 0, data_cap = 0, Atot = 0;
  std::vector<uint64_t> rowbase, tilebase, ubase, abase;
};

Plan make_plan(const gc_codec& c, const uint32_t* h_n, uint64_t nlists, bool include0) {
  Plan p;
  p.nlists = nlists;
  p.rowbase.resize(nlists + 1);
  p.tilebase.resize(nlists + 1);
  p.ubase.resize(nlists + 1);
  p.abase.resize(nlists + 1);
  const uint64_t k = c.k, tr = 1024 / k;
  uint64_t rb = 0, tb = 0, ub = 0, ab = 0;
  for (uint64_t i = 0; i < nlists; ++i) {
    p.rowbase[i] = rb;
    p.tilebase[i] = tb;
    p.ubase[i] = ub;
    p.abase[i] = ab;
    const uint64_t R = (h_n[i] + k - 1) / k;
    const uint64_t nt = (R + tr - 1) / tr;
    ab += nt;
    rb += R;
    tb += include0 ? nt : (nt ? nt - 1 : 0);
    switch (c.kind) {
      case GC_PFD: ub += (R + 31) / 32; break;
      case GC_AFOR: ub += (R + 7) / 8 + 1; break;
      case GC_SIMPLE: ub += (R + kSeg - 1) / kSeg; break;
      default: break;
    }
    uint64_t cc = 0, dc = 0;
    gc_max_encoded_size(&c, h_n[i], &cc, &dc, nullptr);
    p.ctrl_cap += cc;
    p.data_cap += dc;
  }
  p.rowbase[nlists] = rb;
  p.tilebase[nlists] = tb;
  p.ubase[nlists] = ub;
  p.abase[nlists] = ab;
  p.Atot = ab;
  p.Rtot = rb;
  p.Utot = ub;
  p.tiles = tb;
  return p;
}

// Lay out the scratch (base == nullptr: size only).
uint64_t layout(const gc_codec& c, const Plan& p, unsigned char* base, Enc& e, uint64_t** tmp,
                uint32_t** d_n, uint64_t** d_in_off, uint64_t** d_rowbase, uint64_t** d_tilebase,
                uint64_t** d_ubase, uint64_t** d_abase) {
  Bump b{base};
  const uint64_t L = p.nlists;
  *d_n = b.take<uint32_t>(L);
  *d_in_off = b.take<uint64_t>(L);
  *d_rowbase = b.take<uint64_t>(L + 1);
  *d_tilebase = b.take<uint64_t>(L + 1);
  *d_ubase = b.take<uint64_t>(L + 1);
  *d_abase = b.take<uint64_t>(L + 1);
  e.tsum = b.take<uint64_t>(p.Atot + 1);
  e.csize = b.take<uint64_t>(L + 1);
  e.dsize = b.take<uint64_t>(L + 1);
  e.aux = b.take<uint64_t>(L + 1);
  e.eb = b.take<uint8_t>(p.Rtot + 1);
  e.rlist = b.take<uint32_t>(p.Rtot + 1);
  const uint64_t R1 = p.Rtot + 1, U1 = p.Utot + 1;
  uint64_t scan_n = std::max(L + 1, p.Atot + 1);
  switch (c.kind) {
    case GC_PFD:
      e.s0 = b.take<uint64_t>(U1);
      e.s1 = b.take<uint64_t>(U1);
      e.u8a = b.take<uint8_t>(U1);
      e.u8b = b.take<uint8_t>(U1);
      e.u32a = b.take<uint32_t>(U1);
      scan_n = std::max(scan_n, U1);
      break;
    case GC_SCHEME:
      e.s0 = b.take<uint64_t>(R1);
      e.s1 = b.take<uint64_t>(R1);
      e.u8a = b.take<uint8_t>(R1);
      scan_n = std::max(scan_n, R1);
      break;
    case GC_AFOR:
      e.s0 = b.take<uint64_t>(U1);
      e.s1 = b.take<uint64_t>(U1);
      e.u8a = b.take<uint8_t>(U1);
      e.u8b = b.take<uint8_t>(U1);
      e.u32a = b.take<uint32_t>(U1);
      e.u32b = b.take<uint32_t>(U1);
      scan_n = std::max(scan_n, U1);
      break;
    default:  // simple
      e.s0 = b.take<uint64_t>(U1);
      e.s1 = b.take<uint64_t>(R1);
      e.u8a = b.take<uint8_t>(R1);
      e.u8b = b.take<uint8_t>(R1);
      e.u32a = b.take<uint32_t>(U1);
      e.u32b = b.take<uint32_t>(32 * U1);
      scan_n = std::max(scan_n, U1);
      break;
  }
  *tmp = b.take<uint64_t>(scan_tmp_words(scan_n) + 2);
  return b.off + 256;
}

unsigned blocks_for(uint64_t n, uint64_t per = kT) { return (unsigned)std::max<uint64_t>(1, (n + per - 1) / per); }

gc_status encode_impl(const gc_codec& c, const uint32_t* d_gaps, const uint32_t* h_n, const uint64_t* h_in_off,
                      uint64_t nlists, bool single, gc_list* d_lists, uint8_t* d_ctrl, uint64_t ctrl_cap,
                      uint32_t* d_data, uint64_t data_cap, gc_tile* d_tiles, uint64_t tiles_cap,
                      uint64_t* d_totals, void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status,
                      cudaStream_t s) {
  gc_host::reset_launches();
  const Plan p = make_plan(c, h_n, nlists, single);
  if (p.ctrl_cap > ctrl_cap || p.data_cap > data_cap) return GC_ERR_NOSPACE;
  if (d_tiles && p.tiles > tiles_cap) return GC_ERR_NOSPACE;
  if (((uintptr_t)d_ctrl & 3) || ((uintptr_t)d_data & 15)) return GC_ERR_INVALID;
  Enc e = {};
  uint64_t* tmp;
  uint32_t* dn;
  uint64_t *din, *drb, *dtb, *dub, *dab;
  const uint64_t need = layout(c, p, nullptr, e, &tmp, &dn, &din, &drb, &dtb, &dub, &dab);
  if (scratch_bytes < need) return GC_ERR_NOSPACE;
  layout(c, p, (unsigned char*)d_scratch, e, &tmp, &dn, &din, &drb, &dtb, &dub, &dab);
  e.kind = c.kind;
  e.k = c.k;
  e.cg = c.cg;
  e.ld = c.ld;
  e.T = c.pfd_exc_rows;
  e.tr = 1024 / c.k;
  e.include_tile0 = single ? 1 : 0;
  e.nlists = nlists;
  e.Rtot = p.Rtot;
  e.Utot = p.Utot;
  e.gaps = d_gaps;
  e.n = dn;
  e.in_off = din;
  e.rowbase = drb;
  e.tilebase = dtb;
  e.ubase = dub;
  e.abase = dab;
  e.Atot = p.Atot;
  e.ctrl = d_ctrl;
  e.data = d_data;
  e.tiles = d_tiles;
  e.lists = d_lists;
  e.totals = d_totals;
  e.status = d_status;
  if (!d_tiles) e.include_tile0 = 0;
  // host arrays to the device (pageable copies; the encoder is not timed)
  cudaMemcpyAsync(dn, h_n, nlists * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(din, h_in_off, nlists * 8, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(drb, p.rowbase.data(), (nlists + 1) * 8, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dtb, p.tilebase.data(), (nlists + 1) * 8, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dub, p.ubase.data(), (nlists + 1) * 8, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dab, p.abase.data(), (nlists + 1) * 8, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(d_ctrl, 0, gc_host::align_up(p.ctrl_cap, 4) < ctrl_cap ? gc_host::align_up(p.ctrl_cap, 4) : ctrl_cap, s);
  cudaMemsetAsync(d_data, 0, p.data_cap * 4, s);
  if (p.Rtot) {
    k_rows<<<blocks_for(p.Rtot), kT, 0, s>>>(e);
    gc_host::count_launch();
  }
  const unsigned lb = blocks_for(nlists);
  if (!d_tiles) e.tiles = nullptr;
  // put_tile must not write when there is no tile output
  switch (c.kind) {
    case GC_PFD:
      if (p.Utot) {
        k_pfd_frames<<<blocks_for(p.Utot * 32), kT, 0, s>>>(e);
        gc_host::count_launch();
      }
      scan_u64(e.s0, p.Utot, tmp, s);
      scan_u64(e.s1, p.Utot, tmp, s);
      k_pfd_sizes<<<lb, kT, 0, s>>>(e);
      scan_u64(e.csize, nlists, tmp, s);
      scan_u64(e.dsize, nlists, tmp, s);
      gc_host::count_launch();
      if (p.Utot) {
        k_pfd_pack<<<blocks_for(p.Utot * 32), kT, 0, s>>>(e);
        gc_host::count_launch();
      }
      break;
    case GC_SCHEME:
      if (p.Rtot) {
        k_gsc_rows<<<blocks_for(p.Rtot), kT, 0, s>>>(e);
        gc_host::count_launch();
      }
      if (c.ld == GC_LD_IU) {
        k_gsc_iu_walk<<<lb, kT, 0, s>>>(e);
        gc_host::count_launch();
      } else {
        scan_u64(e.s0, p.Rtot, tmp, s);
      }
      scan_u64(e.s1, p.Rtot, tmp, s);
      k_gsc_sizes<<<lb, kT, 0, s>>>(e);
      scan_u64(e.csize, nlists, tmp, s);
      scan_u64(e.dsize, nlists, tmp, s);
      gc_host::count_launch();
      if (p.Rtot) {
        k_gsc_ctrl<<<blocks_for(p.Rtot), kT, 0, s>>>(e);
        k_gsc_data<<<blocks_for(p.Rtot * c.k), kT, 0, s>>>(e);
        gc_host::count_launch(2);
      }
      break;
    case GC_AFOR:
      if (p.Utot) {
        k_afor_blocks<<<blocks_for(p.Utot), kT, 0, s>>>(e);
        gc_host::count_launch();
      }
      k_afor_dp<<<blocks_for(nlists, 64), 64, 0, s>>>(e);
      gc_host::count_launch();
      scan_u64(e.s1, p.Utot, tmp, s);
      k_afor_sizes<<<lb, kT, 0, s>>>(e);
      scan_u64(e.csize, nlists, tmp, s);
      scan_u64(e.dsize, nlists, tmp, s);
      gc_host::count_launch();
      if (p.Utot) {
        k_afor_ctrl<<<blocks_for(p.Utot), kT, 0, s>>>(e);
        gc_host::count_launch();
      }
      if (p.Rtot) {
        k_afor_data<<<blocks_for(p.Rtot * c.k), kT, 0, s>>>(e);
        gc_host::count_launch();
      }
      break;
    default:
      if (p.Rtot) {
        k_gs_choice<<<blocks_for(p.Rtot), kT, 0, s>>>(e);
        k_gs_segments<<<blocks_for(p.Utot * 32), kT, 0, s>>>(e);
        gc_host::count_launch(2);
      }
      k_gs_compose<<<blocks_for(nlists, 64), 64, 0, s>>>(e);
      k_gs_sizes<<<lb, kT, 0, s>>>(e);
      gc_host::count_launch(2);
      scan_u64(e.csize, nlists, tmp, s);
      scan_u64(e.dsize, nlists, tmp, s);
      if (p.Utot) {
        k_gs_emit<<<blocks_for(p.Utot), kT, 0, s>>>(e);
        k_gs_mark<<<blocks_for(p.Utot), kT, 0, s>>>(e);
        k_gs_data<<<blocks_for(p.Rtot * c.k), kT, 0, s>>>(e);
        gc_host::count_launch(3);
      }
      break;
  }
  if (d_tiles && p.Atot) {
    e.tiles = d_tiles;
    k_tile_sums<<<blocks_for(p.Atot * 32), kT, 0, s>>>(e);
    gc_host::count_launch();
    scan_u64(e.tsum, p.Atot, tmp, s);
    k_put_bases<<<blocks_for(p.Atot), kT, 0, s>>>(e);
    gc_host::count_launch();
  }
  if (d_lists) {
    k_lists_out<<<lb, kT, 0, s>>>(e);
    gc_host::count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

__global__ void k_single_sizes(const uint64_t* csize, const uint64_t* dsize, uint64_t* out) {
  out[0] = csize[1];
  out[1] = dsize[1];
}

}  // namespace gcenc

using namespace gcenc;

extern "C" {

gc_status gc_encode_batch_scratch_size(const gc_codec* codec, const uint32_t* h_n, uint64_t nlists,
                                       uint64_t* bytes) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!bytes || (nlists && !h_n)) return GC_ERR_INVALID;
  const Plan p = make_plan(*codec, h_n, nlists, false);
  Enc e = {};
  uint64_t* tmp;
  uint32_t* dn;
  uint64_t *din, *drb, *dtb, *dub, *dab;
  *bytes = layout(*codec, p, nullptr, e, &tmp, &dn, &din, &drb, &dtb, &dub, &dab);
  return GC_OK;
}

gc_status gc_encode_scratch_size(const gc_codec* codec, uint64_t n, uint64_t* bytes) {
  if (n > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  const uint32_t n32 = (uint32_t)n;
  return gc_encode_batch_scratch_size(codec, &n32, 1, bytes);
}

gc_status gc_encode_batch(const gc_codec* codec, const uint32_t* d_gaps, const uint32_t* h_n,
                          const uint64_t* h_in_off, uint64_t nlists, gc_list* d_lists, uint8_t* d_ctrl,
                          uint64_t ctrl_cap, uint32_t* d_data, uint64_t data_cap, gc_tile* d_tiles,
                          uint64_t tiles_cap, uint64_t* d_totals, void* d_scratch, uint64_t scratch_bytes,
                          void* stream) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (nlists == 0) return GC_OK;
  if (!d_gaps || !h_n || !h_in_off || !d_lists || !d_ctrl || !d_data || !d_totals || !d_scratch)
    return GC_ERR_INVALID;
  if (nlists > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  return encode_impl(*codec, d_gaps, h_n, h_in_off, nlists, false, d_lists, d_ctrl, ctrl_cap, d_data, data_cap,
                     d_tiles, tiles_cap, d_totals, d_scratch, scratch_bytes, nullptr, (cudaStream_t)stream);
}

gc_status gc_encode(const gc_codec* codec, const uint32_t* d_gaps, uint64_t n, uint8_t* d_ctrl, uint64_t ctrl_cap,
                    uint32_t* d_data, uint64_t data_cap, gc_tile* d_tiles, uint64_t* d_sizes, void* d_scratch,
                    uint64_t scratch_bytes, void* stream) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!d_sizes || !d_scratch) return GC_ERR_INVALID;
  if (n > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    return cudaMemsetAsync(d_sizes, 0, 16, s) == cudaSuccess ? GC_OK : GC_ERR_CUDA;
  }
  if (!d_gaps || !d_ctrl || !d_data) return GC_ERR_INVALID;
  const uint32_t n32 = (uint32_t)n;
  const uint64_t off = 0;
  uint64_t nt = 0;
  gc_max_encoded_size(codec, n, nullptr, nullptr, &nt);
  st = encode_impl(*codec, d_gaps, &n32, &off, 1, true, nullptr, d_ctrl, ctrl_cap, d_data, data_cap, d_tiles,
                   nt, nullptr, d_scratch, scratch_bytes, nullptr, s);
  if (st != GC_OK) return st;
  // the per-list sizes were scanned into offsets; offsets[1] is the total
  Enc e = {};
  uint64_t* tmp;
  uint32_t* dn;
  uint64_t *din, *drb, *dtb, *dub, *dab;
  const Plan p = make_plan(*codec, &n32, 1, true);
  layout(*codec, p, (unsigned char*)d_scratch, e, &tmp, &dn, &din, &drb, &dtb, &dub, &dab);
  k_single_sizes<<<1, 1, 0, s>>>(e.csize, e.dsize, d_sizes);
  gc_host::count_launch();
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

}  // extern "C"
