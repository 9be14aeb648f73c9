// gc_decode.cu -- decoding kernels of the Group-codec library.
//
// One warp decodes one tile of 1024 ints (1024/k rows) of one list:
//   1. parse the tile's control patterns into a per-row table (lane-bit
//      offset, bit width): Group-Simple selectors (Table III, Sec 4.3),
//      Group-Scheme length descriptors (Eq. 2; binary, complete unary and
//      incomplete unary, Sec 5.2.1 and 5.3.1), Group-AFOR frame bytes
//      (Sec 6.1), Group-PFD frame headers (Sec 6.2 decoding Step 1);
//   2. extract every int with a funnel shift from its lane's stream (the
//      k-way vertical layout: at k = 32 a warp reads one 128-byte vector per
//      row, fully coalesced);
//   3. Group-PFD: write the frame's exceptions over their slots (Step 3);
//   4. optionally restore docIDs (Sec 2.1.1): per-lane sequential sums, a
//      warp scan, and a decoupled look-back across the tiles of the list
//      (bounded waits: a wait that runs out reports GC_ERR_TIMEOUT);
//   5. store the 1024 ints with coalesced 128-byte stores.
// Warps claim tiles in increasing order from a global counter, so the tile
// a warp waits on has always been claimed by a running warp.
#include <cstdint>
#include <cuda_runtime.h>

#include "gc_device.cuh"
#include "gc_host.h"

namespace gcdev {

constexpr unsigned long long kFlagAgg = 1ull << 32;
constexpr unsigned long long kFlagPrefix = 2ull << 32;
constexpr uint32_t kSpinLimit = 1u << 22;  // ~0.5 s of polling

template <int K>
struct __align__(16) WarpSmem {
  static constexpr int TR = kTileInts / K;  // rows per tile
  static constexpr int FPT = TR / 32;       // PFD frames per tile
  // the tile's data words, staged (TR rows of at most 32 bits per lane and
  // a start offset below 32 span at most TR + 1 words per lane)
  static constexpr int DW = (TR + 1) * K;
  uint32_t d[DW];
  uint32_t outs[kTileInts + kTileInts / 32];  // padded: int i at i + i/32
  uint64_t fx[FPT];                           // PFD: byte offset of each frame's exception record
  uint32_t rb[TR];                            // lane-bit offset of each row (from the tile's unit)
  uint32_t fe[FPT], fw[FPT], fr[FPT];         // PFD: exceptions, width code, rows of each frame
  uint8_t rw[TR];                             // bit width of each row
};

struct ListRef {
  const uint8_t* ctrl;
  uint64_t ctrl_bytes;
  const uint32_t* data;
  uint64_t data_words;
  uint32_t* out;
  uint64_t n;
};

struct DecodeArgs {
  ListRef one;  // single-list launch
  const gc_tile* one_tiles;
  uint64_t one_ntiles;
  const gc_work* work;  // batched launch: one record per tile
  const unsigned long long* work_count;
  uint64_t work_cap;
  const uint8_t* ctrl_pool;
  uint64_t ctrl_pool_bytes;
  const uint32_t* data_pool;
  uint64_t data_pool_words;
  uint32_t* out_pool;
  uint64_t out_pool_len;
  uint32_t* counters;       // [0] claim counter
  unsigned long long* lb;   // look-back word per work item
  uint32_t cg, ld;
  uint32_t claim;           // work items per claim
  int restore;
  uint32_t* status;
};

__device__ __forceinline__ uint32_t pad_idx(uint32_t i) { return i + (i >> 5); }

// ---------------------------------------------------------------- parse
// Each parser fills rb[0..rows) and rw[0..rows) for rows row0.. of the list,
// starting from the tile record `rec`. Returns false on a malformed stream.

template <int K>
__device__ bool parse_simple(const ListRef& L, const gc_tile& rec, uint64_t row0, uint32_t rows,
                             WarpSmem<K>& ws) {
  const uint32_t lane = lane_id();
  const uint64_t u0 = rec.ctrl_bit >> 2;
  const uint64_t tile_end = row0 + rows;
  uint64_t cov = row0 - rec.row_skip;  // first row of the next unit to read
  bool ok = true;
  for (uint32_t c = 0; cov < tile_end; c += 32) {
    const uint64_t u = u0 + c + lane;
    uint32_t sel = 15;
    if ((u >> 1) < L.ctrl_bytes) sel = (__ldg(L.ctrl + (u >> 1)) >> ((u & 1) * 4)) & 15u;
    const bool bad = sel > 9;
    const uint32_t num = bad ? 32u : sel_num(sel);
    const uint32_t bw = bad ? 0u : sel_bw(sel);
    const uint32_t incl = warp_incl_sum(num);
    const uint64_t start = cov + incl - num;
    if (start < tile_end) {
      if (bad) ok = false;
      const uint64_t a = start > row0 ? start : row0;
      const uint64_t b = (start + num) < tile_end ? (start + num) : tile_end;
      for (uint64_t q = a; q < b; ++q) {
        ws.rb[q - row0] = 32u * (c + lane) + (uint32_t)(q - start) * bw;
        ws.rw[q - row0] = (uint8_t)bw;
      }
    }
    cov += __shfl_sync(kFull, incl, 31);
  }
  return __all_sync(kFull, ok);
}

template <int K>
__device__ bool parse_scheme_binary(const ListRef& L, uint64_t row0, uint32_t rows, uint32_t cg,
                                    WarpSmem<K>& ws) {
  const uint32_t lane = lane_id();
  const uint32_t width = 5 - log2_cg(cg);
  const uint32_t maxu = 32 / cg;
  uint32_t carry = 0;
  bool ok = true;
  for (uint32_t c = 0; c < rows; c += 32) {
    const uint32_t q = c + lane;
    uint32_t bw = 0;
    if (q < rows) {
      const uint64_t pos = bin_ld_pos(row0 + q, cg);
      if (((pos + width + 7) >> 3) > L.ctrl_bytes) ok = false;
      const uint32_t u = read_ctrl_bits(L.ctrl, L.ctrl_bytes, pos, width) + 1;
      if (u > maxu) ok = false;
      bw = cg * u;
    }
    const uint32_t incl = warp_incl_sum(bw);
    if (q < rows) {
      ws.rb[q] = carry + incl - bw;
      ws.rw[q] = (uint8_t)bw;
    }
    carry += __shfl_sync(kFull, incl, 31);
  }
  return __all_sync(kFull, ok);
}

// Unary descriptors (Sec 5.2.1(a), 5.3.1): (u - 1) ones closed by a zero.
// Lanes take byte-aligned 32-bit windows of the control stream; each zero
// closes one descriptor. CU: a descriptor starts right after the previous
// zero (possibly in an earlier window). IU: descriptors never straddle a
// byte, so one starts after the previous zero of its byte or at the byte's
// first bit; trailing ones of a byte are padding.
template <int K>
__device__ bool parse_scheme_unary(const ListRef& L, const gc_tile& rec, uint32_t rows, uint32_t cg,
                                   bool iu, WarpSmem<K>& ws) {
  const uint32_t lane = lane_id();
  const uint64_t P0 = rec.ctrl_bit;
  const uint64_t A = P0 & ~7ull;
  const uint32_t maxu = 32 / cg;
  uint32_t found = 0, ubase = 0;
  int64_t prev_last = (int64_t)P0 - 1;  // last zero before the current window group
  bool ok = true;
  for (uint64_t w = 0; found < rows; w += 32) {
    const uint64_t wbit = A + 32 * (w + lane);
    if ((A >> 3) + 4 * w >= L.ctrl_bytes) { ok = false; break; }  // ran off the control area
    uint32_t win = read_le(L.ctrl, L.ctrl_bytes, wbit >> 3, 4, 0xffu);
    if (wbit < P0) win |= (1u << (uint32_t)(P0 - wbit)) - 1u;
    const uint32_t zeros = ~win;
    const uint32_t nz = __popc(zeros);
    const int64_t lastz = nz ? (int64_t)(wbit + 31 - __clz(zeros)) : INT64_MIN;
    const int64_t incl_last = warp_incl_max(lastz);
    int64_t prev = __shfl_up_sync(kFull, incl_last, 1);
    if (lane == 0 || prev < prev_last) prev = prev_last;
    // pass 1: sum of descriptor values in this window
    uint32_t usum = 0;
    {
      uint32_t z = zeros;
      int64_t pv = prev;
      while (z) {
        const uint32_t b = __ffs(z) - 1;
        z &= z - 1;
        const int64_t p = (int64_t)wbit + b;
        int64_t start = pv + 1;
        if (iu) {
          const int64_t bs = p & ~7ll;
          if (pv < bs) start = bs > (int64_t)P0 ? bs : (int64_t)P0;
        }
        usum += (uint32_t)(p - start + 1);
        pv = p;
      }
    }
    const uint32_t incl_nz = warp_incl_sum(nz);
    const uint32_t incl_us = warp_incl_sum(usum);
    uint32_t q = found + incl_nz - nz;
    uint32_t ub = ubase + incl_us - usum;
    {
      uint32_t z = zeros;
      int64_t pv = prev;
      while (z && q < rows) {
        const uint32_t b = __ffs(z) - 1;
        z &= z - 1;
        const int64_t p = (int64_t)wbit + b;
        int64_t start = pv + 1;
        if (iu) {
          const int64_t bs = p & ~7ll;
          if (pv < bs) start = bs > (int64_t)P0 ? bs : (int64_t)P0;
        }
        const uint32_t u = (uint32_t)(p - start + 1);
        if (u > maxu) ok = false;
        ws.rb[q] = cg * ub;
        ws.rw[q] = (uint8_t)(cg * u);
        ub += u;
        ++q;
        pv = p;
      }
    }
    found += __shfl_sync(kFull, incl_nz, 31);
    ubase += __shfl_sync(kFull, incl_us, 31);
    const int64_t gl = __shfl_sync(kFull, incl_last, 31);
    if (gl > prev_last) prev_last = gl;
  }
  return __all_sync(kFull, ok);
}

template <int K>
__device__ bool parse_afor(const ListRef& L, const gc_tile& rec, uint64_t row0, uint32_t rows,
                           WarpSmem<K>& ws) {
  const uint32_t lane = lane_id();
  const uint64_t f0 = rec.ctrl_bit >> 3;
  const uint64_t tile_end = row0 + rows;
  uint64_t cov = row0 - rec.row_skip;
  uint32_t lcarry = 0;
  bool ok = true;
  for (uint32_t c = 0; cov < tile_end; c += 32) {
    const uint64_t f = f0 + c + lane;
    const uint32_t byte = f < L.ctrl_bytes ? (uint32_t)__ldg(L.ctrl + f) : 0xffu;
    const uint32_t code = byte >> 6, b = byte & 63u;
    const bool bad = code > 2 || b > 32;
    const uint32_t F = bad ? 32u : (8u << code);
    const uint32_t lbits = bad ? 0u : F * b;
    const uint32_t inclF = warp_incl_sum(F);
    const uint32_t inclL = warp_incl_sum(lbits);
    const uint64_t start = cov + inclF - F;
    const uint32_t lstart = lcarry + inclL - lbits;
    if (start < tile_end) {
      if (bad) ok = false;
      const uint64_t a = start > row0 ? start : row0;
      const uint64_t e = (start + F) < tile_end ? (start + F) : tile_end;
      for (uint64_t q = a; q < e; ++q) {
        ws.rb[q - row0] = lstart + (uint32_t)(q - start) * b;
        ws.rw[q - row0] = (uint8_t)(bad ? 0 : b);
      }
    }
    cov += __shfl_sync(kFull, inclF, 31);
    lcarry += __shfl_sync(kFull, inclL, 31);
  }
  return __all_sync(kFull, ok);
}

// Group-PFD decoding Step 1: per frame, the header (b, exception width, e).
// The exception records follow the headers, frame after frame; the tile
// record gives the offset of the tile's first frame's record.
template <int K>
__device__ bool parse_pfd(const ListRef& L, const gc_tile& rec, uint64_t row0, uint32_t rows,
                          uint64_t R, WarpSmem<K>& ws) {
  constexpr int FPT = WarpSmem<K>::FPT;
  constexpr uint32_t pb = (kPfdFrameRows * K) <= 256 ? 1u : 2u;
  const uint32_t lane = lane_id();
  const uint64_t nf = (R + kPfdFrameRows - 1) / kPfdFrameRows;
  const uint64_t f0 = row0 / kPfdFrameRows;
  const uint32_t nfr = (rows + kPfdFrameRows - 1) / kPfdFrameRows;
  bool ok = true;
  uint32_t b = 0, wcode = 0, e = 0, xb = 0, frows = 0;
  if (lane < (uint32_t)FPT && lane < nfr) {
    const uint64_t f = f0 + lane;
    if (4 * f + 4 > L.ctrl_bytes) ok = false;
    const uint32_t hdr = read_le(L.ctrl, L.ctrl_bytes, 4 * f, 4);
    b = hdr & 63u;
    wcode = (hdr >> 6) & 3u;
    e = hdr >> 8;
    if (b > 32 || wcode > 2) { ok = false; b = 0; e = 0; }
    frows = (uint32_t)((R - f * kPfdFrameRows) < kPfdFrameRows ? (R - f * kPfdFrameRows) : kPfdFrameRows);
    if (e > frows * K) { ok = false; e = 0; }
    xb = e * (pb + (1u << wcode));
  }
  const uint32_t inclL = warp_incl_sum(32u * b);
  const uint32_t inclX = warp_incl_sum(xb);
  if (lane < (uint32_t)FPT) {
    ws.fx[lane] = 4 * nf + rec.exc_off + (inclX - xb);
    ws.fe[lane] = e;
    ws.fw[lane] = wcode;
    ws.fr[lane] = frows;
    if (e && ws.fx[lane] + xb > L.ctrl_bytes) ok = false;
  }
  const uint32_t lstart = inclL - 32u * b;
  // rows: frame fl = q / 32
  for (uint32_t fl = 0; fl < nfr; ++fl) {
    const uint32_t bf = __shfl_sync(kFull, b, fl);
    const uint32_t ls = __shfl_sync(kFull, lstart, fl);
    const uint32_t q = fl * 32 + lane;
    if (q < rows) {
      ws.rb[q] = ls + lane * bf;
      ws.rw[q] = (uint8_t)bf;
    }
  }
  return __all_sync(kFull, ok);
}

// Step 3: write each exception over its slot.
template <int K>
__device__ bool patch_pfd(const ListRef& L, uint32_t rows, uint32_t nints, WarpSmem<K>& ws) {
  constexpr uint32_t pb = (kPfdFrameRows * K) <= 256 ? 1u : 2u;
  const uint32_t lane = lane_id();
  const uint32_t nfr = (rows + kPfdFrameRows - 1) / kPfdFrameRows;
  bool ok = true;
  for (uint32_t fl = 0; fl < nfr; ++fl) {
    const uint32_t e = ws.fe[fl];
    if (e == 0) continue;
    const uint32_t wb = 1u << ws.fw[fl];
    const uint64_t base = ws.fx[fl];
    const uint32_t lim = ws.fr[fl] * K;
    for (uint32_t x = lane; x < e; x += 32) {
      const uint32_t pos = read_le(L.ctrl, L.ctrl_bytes, base + (uint64_t)x * pb, pb);
      const uint32_t val = read_le(L.ctrl, L.ctrl_bytes, base + (uint64_t)e * pb + (uint64_t)x * wb, wb);
      const uint32_t i = fl * kPfdFrameRows * K + pos;
      if (pos < lim && i < nints) ws.outs[pad_idx(i)] = val;
      else if (pos >= lim) ok = false;
    }
  }
  return __all_sync(kFull, ok);
}

// ------------------------------------------------------------ look-back

// Decoupled look-back over the tiles of one list, a warp at a time: publish
// this tile's aggregate, then read the 32 nearest predecessors at once; the
// nearest one that carries an inclusive prefix ends the walk, otherwise the
// window moves 32 tiles back. Tile 0 of a list always carries a prefix, so
// the walk ends inside the list. Returns the exclusive prefix (all lanes).
// Every wait is bounded; a wait that runs out reports GC_ERR_TIMEOUT.
__device__ uint32_t look_back(unsigned long long* lb, uint64_t item, uint64_t t, uint32_t agg, uint32_t* status,
                              uint32_t where) {
  const uint32_t lane = lane_id();
  if (t == 0) {
    if (lane == 0) st_release(lb + item, kFlagPrefix | agg);
    return 0;
  }
  if (lane == 0) st_release(lb + item, kFlagAgg | agg);
  uint32_t excl = 0;
  bool timed_out = false;
  for (uint64_t d = 1;; d += 32) {
    const uint64_t dist = d + lane;  // predecessor tile t - dist
    unsigned long long s = kFlagPrefix;
    if (dist <= t) {
      s = ld_acquire(lb + item - dist);
      uint32_t spins = 0;
      while ((s >> 32) == 0) {
        if (++spins > kSpinLimit) {
          timed_out = true;
          break;
        }
        __nanosleep(32);
        s = ld_acquire(lb + item - dist);
      }
    }
    if (__any_sync(kFull, timed_out)) {
      if (lane == 0) report(status, GC_ERR_TIMEOUT, where);
      break;
    }
    const uint32_t pm = __ballot_sync(kFull, (s & ~0xffffffffull) == kFlagPrefix);
    uint32_t v = (uint32_t)s;
    if (pm) {
      if (lane > (uint32_t)(__ffs(pm) - 1)) v = 0;
      excl += warp_sum(v);
      break;
    }
    excl += warp_sum(v);
  }
  if (lane == 0) st_release(lb + item, kFlagPrefix | (uint32_t)(excl + agg));
  return excl;
}

__device__ __forceinline__ uint4 ldg_v4(const uint32_t* p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// ---------------------------------------------------------------- tile

// Decode tile t of list L (work item `item`). `chained`: the previous tile
// of the list was decoded by this warp, and `carry` is its inclusive prefix.
// Returns the tile's inclusive prefix (docIDs modulo 2^32).
template <int KIND, int K>
__device__ uint32_t decode_tile(const DecodeArgs& a, const ListRef& L, const gc_tile& rec, uint64_t t,
                                uint64_t item, uint32_t where, bool chained, uint32_t carry, WarpSmem<K>& ws) {
  constexpr uint32_t TR = kTileInts / K;
  constexpr uint32_t DW = WarpSmem<K>::DW;
  const uint32_t lane = lane_id();
  const uint64_t R = (L.n + K - 1) / K;
  const uint64_t row0 = t * TR;
  const uint32_t rows = (uint32_t)((R - row0) < TR ? (R - row0) : TR);
  const uint32_t nints = (uint32_t)((L.n - row0 * K) < (uint64_t)kTileInts ? (L.n - row0 * K) : kTileInts);

  // 1. control patterns -> per-row (lane-bit offset, width)
  bool ok;
  if (KIND == GC_SIMPLE) ok = parse_simple<K>(L, rec, row0, rows, ws);
  else if (KIND == GC_SCHEME) {
    if (a.ld == GC_LD_BINARY) ok = parse_scheme_binary<K>(L, row0, rows, a.cg, ws);
    else ok = parse_scheme_unary<K>(L, rec, rows, a.cg, a.ld == GC_LD_IU, ws);
  } else if (KIND == GC_AFOR) ok = parse_afor<K>(L, rec, row0, rows, ws);
  else ok = parse_pfd<K>(L, rec, row0, rows, R, ws);
  __syncwarp();

  // 2. stage the tile's data words in shared memory: whole k-word vectors
  // from the first row's word to the last row's, with 16-byte loads that
  // are all in flight at once
  const uint32_t rb0 = ws.rb[0];
  const uint64_t base = rec.lane_bit + rb0;
  const uint32_t off0 = (uint32_t)base & 31u;
  const uint32_t tbits = ws.rb[rows - 1] - rb0 + ws.rw[rows - 1];
  uint32_t nwr = (off0 + tbits + 31) >> 5;
  if (nwr * K > DW) {
    nwr = DW / K;
    ok = false;
  }
  const uint64_t g0 = (base >> 5) * K;
  bool dok = true;
  for (uint32_t c = lane; c < nwr * K / 4; c += 32) {
    const uint64_t gw = g0 + 4ull * c;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (gw + 4 <= L.data_words) v = ldg_v4(L.data + gw);
    else dok = false;
    *reinterpret_cast<uint4*>(ws.d + 4 * c) = v;
  }
  __syncwarp();

  // 3. extract: int i of the tile is lane i % K of row i / K
#pragma unroll 4
  for (uint32_t m = 0; m < 32; ++m) {
    const uint32_t i = lane + 32 * m;
    uint32_t v = 0;
    if (i < nints) {
      const uint32_t r = i / K, j = i % K;
      const uint32_t w = ws.rw[r];
      const uint32_t bit = off0 + ws.rb[r] - rb0;
      const uint32_t o = bit & 31u;
      uint32_t wi = (bit >> 5) * K + j;
      wi = wi < DW ? wi : DW - 1;
      const uint32_t lo = ws.d[wi];
      uint32_t hi = 0;
      if (o + w > 32) hi = ws.d[wi + K < DW ? wi + K : DW - 1];
      v = __funnelshift_r(lo, hi, o) & low_mask(w);
      if (w == 0) v = 0;
    }
    ws.outs[pad_idx(i)] = v;
  }
  __syncwarp();
  if (KIND == GC_PFD) {
    ok = patch_pfd<K>(L, rows, nints, ws) && ok;
    __syncwarp();
  }
  if (!__all_sync(kFull, dok)) ok = false;
  if (!ok && lane == 0) report(a.status, GC_ERR_CORRUPT, where);

  // 4. docIDs: lane l sums ints 32l..32l+31, a warp scan joins the lanes, the
  // previous tile's prefix comes from this warp (chained) or by look-back
  uint32_t incl_tile = 0;
  if (a.restore) {
    uint32_t v[32];
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      s += ws.outs[lane * 33 + c];
      v[c] = s;
    }
    const uint32_t incl = warp_incl_sum(s);
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    uint32_t pre;
    if (chained) {
      pre = carry;
      if (lane == 0) st_release(a.lb + item, kFlagPrefix | (uint32_t)(carry + total));
    } else {
      pre = look_back(a.lb, item, t, total, a.status, where);
    }
    incl_tile = pre + total;
    pre += incl - s;
#pragma unroll
    for (int c = 0; c < 32; ++c) ws.outs[lane * 33 + c] = v[c] + pre;
    __syncwarp();
  }

  // 5. coalesced stores
  uint32_t* out = L.out + row0 * K;
#pragma unroll 8
  for (uint32_t m = 0; m < 32; ++m) {
    const uint32_t i = lane + 32 * m;
    if (i < nints) out[i] = ws.outs[pad_idx(i)];
  }
  __syncwarp();
  return incl_tile;
}

// Persistent decoder. A block claims chunks of C = warps * G consecutive
// work items from the global counter (one atomic per chunk); its warps take
// the chunk's items one at a time, in order, through a shared-memory word
// (base << 32 | items taken). Items are thus handed out in increasing
// order: every item below a handed-out item has been handed out too, and a
// warp holds only items below those still in its block's chunk. A look-back
// waits on lower items only, so the lowest unfinished item always belongs
// to a running warp and decoding always progresses. When one warp happens
// to take consecutive tiles of a list, it passes the prefix in registers.
__device__ uint64_t take_item(unsigned long long* sq, uint32_t* counter, uint64_t total, uint32_t C,
                              uint32_t* status) {
  // The word starts as (no chunk, C taken), so the first taker refills. A
  // returned item at or past `total` ends the caller's loop.
  for (;;) {
    const unsigned long long old = atomicAdd(sq, 1ull);
    const uint64_t base = old >> 32;
    const uint32_t taken = (uint32_t)old;
    if (taken < C) return base + taken < total ? base + taken : total;
    if (taken == C) {
      uint64_t nb = atomicAdd(counter, C);
      if (nb > total) nb = total;
      atomicExch(sq, ((unsigned long long)nb << 32) | 1ull);
      return nb;
    }
    // another warp is refilling the chunk
    uint32_t spins = 0;
    while ((*(volatile unsigned long long*)sq >> 32) == base) {
      if (++spins > kSpinLimit) {
        report(status, GC_ERR_TIMEOUT, 0xffffffffu);
        return total;
      }
      __nanosleep(20);
    }
  }
}

template <int KIND, int K, bool BATCH>
__global__ void __launch_bounds__(512) k_decode(DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long s_queue;
  WarpSmem<K>& ws = reinterpret_cast<WarpSmem<K>*>(smem_raw)[threadIdx.x >> 5];
  const uint32_t lane = lane_id();
  uint64_t total = a.one_ntiles;
  if (BATCH) {
    total = *(volatile const unsigned long long*)a.work_count;
    if (total > a.work_cap) total = a.work_cap;
  }
  const uint32_t C = a.claim * (blockDim.x >> 5);
  if (threadIdx.x == 0) s_queue = (0xffffffffull << 32) | C;  // empty: the first taker refills
  __syncthreads();
  uint64_t prev_list = ~0ull, prev_t = ~0ull;
  uint32_t prev_incl = 0;
  for (;;) {
    uint64_t item = 0;
    if (lane == 0) item = take_item(&s_queue, a.counters, total, C, a.status);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    ListRef L;
    uint64_t t, list;
    gc_tile rec = {0, 0, 0, 0};
    uint32_t where;
    bool skip = false;
    if (!BATCH) {
      L = a.one;
      t = item;
      list = 0;
      where = (uint32_t)item;
      if (t > 0) {
        const gc_tile* p = a.one_tiles + t;
        rec.lane_bit = p->lane_bit;
        rec.ctrl_bit = p->ctrl_bit;
        rec.exc_off = p->exc_off;
        rec.row_skip = p->row_skip;
      }
    } else {
      const uint4* wp = reinterpret_cast<const uint4*>(a.work + item);
      const uint4 q0 = __ldg(wp), q1 = __ldg(wp + 1), q2 = __ldg(wp + 2), q3 = __ldg(wp + 3);
      const uint64_t ctrl_off = q0.x | ((uint64_t)q0.y << 32);
      const uint64_t data_off = q0.z | ((uint64_t)q0.w << 32);
      const uint64_t out_off = q1.x | ((uint64_t)q1.y << 32);
      const uint32_t n = q1.z;
      t = q1.w;
      rec.lane_bit = q2.x | ((uint64_t)q2.y << 32);
      rec.ctrl_bit = q2.z | ((uint64_t)q2.w << 32);
      rec.exc_off = q3.x;
      rec.row_skip = q3.y;
      list = q3.z;
      where = q3.z;
      L.ctrl = a.ctrl_pool + ctrl_off;
      L.ctrl_bytes = ctrl_off < a.ctrl_pool_bytes ? a.ctrl_pool_bytes - ctrl_off : 0;
      L.data = a.data_pool + data_off;
      L.data_words = data_off < a.data_pool_words ? a.data_pool_words - data_off : 0;
      L.out = a.out_pool + out_off;
      L.n = n;
      if (q3.z == 0xffffffffu) {
        skip = true;  // an empty slot (the plan overflowed its table)
      } else if (out_off + n > a.out_pool_len || (data_off % K) != 0) {
        if (lane == 0) report(a.status, GC_ERR_INVALID, where);
        skip = true;
      }
    }
    if (skip || t * kTileInts >= L.n) {
      // nothing to decode; keep the chain of prefixes alive
      if (a.restore && lane == 0) st_release(a.lb + item, kFlagPrefix);
      prev_list = ~0ull;
      continue;
    }
    const bool chained = (list == prev_list) && (t == prev_t + 1);
    prev_incl = decode_tile<KIND, K>(a, L, rec, t, item, where, chained, prev_incl, ws);
    prev_list = list;
    prev_t = t;
  }
}

// Batched plan, pass 1: one thread per list reserves a contiguous range of
// work items for the list's tiles (one atomic per warp) and writes (list,
// tile) into each record. A list's tiles are consecutive items, so a tile's
// predecessor is always claimed before it.
__global__ void k_plan_reserve(const gc_list* lists, uint64_t nlists, uint32_t k, gc_work* work, uint64_t cap,
                               unsigned long long* count, uint32_t* status) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = lane_id();
  uint64_t nt = 0;
  if (i < nlists) {
    const uint64_t n = lists[i].n;
    const uint64_t R = (n + k - 1) / k;
    const uint64_t tr = kTileInts / k;
    nt = (R + tr - 1) / tr;
  }
  const uint64_t incl = warp_incl_sum(nt);
  unsigned long long b = 0;
  if (lane == 31) b = atomicAdd(count, (unsigned long long)incl);
  const uint64_t base = __shfl_sync(kFull, b, 31) + incl - nt;
  if (i >= nlists) return;
  const bool fits = base + nt <= cap;
  if (!fits) report(status, GC_ERR_NOSPACE, (uint32_t)i);
  for (uint64_t t = 0; t < nt && base + t < cap; ++t) {
    gc_work* w = work + base + t;
    w->tile = (uint32_t)t;
    w->list = fits ? (uint32_t)i : 0xffffffffu;
  }
}

// Pass 2: one thread per work item fills in the list's descriptor and the
// tile's record (tile 0 starts at the list's first unit).
__global__ void k_plan_fill(const gc_list* lists, uint64_t nlists, const gc_tile* tiles, uint64_t ntiles,
                            gc_work* work, uint64_t cap, const unsigned long long* count, uint32_t* status) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t total = *count;
  if (total > cap) total = cap;
  if (i >= total) return;
  gc_work w = work[i];
  if (w.list >= nlists) {
    w = gc_work{0, 0, 0, 0, 0, 0, 0, 0, 0, 0xffffffffu, 0};
    work[i] = w;
    return;
  }
  const gc_list d = lists[w.list];
  w.ctrl_off = d.ctrl_off;
  w.data_off = d.data_off;
  w.out_off = d.out_off;
  w.n = d.n;
  w.lane_bit = w.ctrl_bit = 0;
  w.exc_off = w.row_skip = 0;
  w.reserved = 0;
  if (w.tile > 0) {
    const uint64_t ti = (uint64_t)d.tile_off + w.tile - 1;
    if (ti < ntiles) {
      const gc_tile r = tiles[ti];
      w.lane_bit = r.lane_bit;
      w.ctrl_bit = r.ctrl_bit;
      w.exc_off = r.exc_off;
      w.row_skip = r.row_skip;
    } else {
      report(status, GC_ERR_CORRUPT, w.list);
      w.n = 0;  // decodes nothing
    }
  }
  work[i] = w;
}

// ------------------------------------------------------- tile index build
// The paper's format stores no tile records. They follow from the control
// area alone: split it into chunks, sum (rows, lane bits, exception bytes)
// per chunk, scan the chunk sums, and walk each chunk again from its prefix,
// writing a record for every tile whose first row falls in a unit.

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
  UnitAgg v = {0, 0, 0};
  if (c < a.nchunks) v = walk_chunk(a, c, false, v);
  UnitAgg tot;
  UnitAgg ex = block_excl_scan(v, &tot);
  if (c < a.nchunks) walk_chunk(a, c, true, agg_add(a.block_sums[blockIdx.x], ex));
}

}  // namespace gcdev

// ====================================================================== host

using namespace gcdev;

namespace {

template <int K>
size_t warp_smem() { return sizeof(WarpSmem<K>); }

constexpr uint32_t kMaxWarps = 16;     // warps per block (launch bounds: 512 threads)
constexpr uint32_t kDefaultWarps = 8;
constexpr uint32_t kMaxClaim = 64;     // work items per claim
constexpr uint32_t kDefaultClaim = 4;

template <int KIND, int K, bool BATCH>
cudaError_t launch_decode_t(const DecodeArgs& a, uint32_t warps, uint32_t blocks_per_sm, uint64_t work,
                            cudaStream_t s) {
  auto fn = k_decode<KIND, K, BATCH>;
  const size_t smem = warps * warp_smem<K>();
  // the shared-memory limit only grows, and the occupancy is fixed per
  // (device, warps): both are cached so a launch costs one API call
  static size_t smem_limit[64] = {};
  static int cached_occ[64][kMaxWarps + 1] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cache = dev >= 0 && dev < 64;
  if (!cache || smem > smem_limit[dev]) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cache) smem_limit[dev] = smem;
  }
  int occ = cache ? cached_occ[dev][warps] : 0;
  if (occ == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, (int)(warps * 32), smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (cache) cached_occ[dev][warps] = occ;
  }
  const int sms = gc_host::sm_count();
  uint32_t bps = blocks_per_sm ? blocks_per_sm : (uint32_t)occ;
  if (bps > (uint32_t)occ) bps = (uint32_t)occ;
  uint64_t grid = (uint64_t)bps * sms;
  const uint64_t need = (work + (uint64_t)warps * a.claim - 1) / ((uint64_t)warps * a.claim);
  if (!BATCH && grid > need) grid = need ? need : 1;
  fn<<<(unsigned)grid, warps * 32, smem, s>>>(a);
  gc_host::count_launch();
  return cudaGetLastError();
}

template <bool BATCH>
cudaError_t launch_decode(uint32_t kind, uint32_t k, const DecodeArgs& a, uint32_t warps, uint32_t bps,
                          uint64_t work, cudaStream_t s) {
#define GC_DISPATCH(KIND)                                                           \
  if (kind == KIND) {                                                                \
    if (k == 4) return launch_decode_t<KIND, 4, BATCH>(a, warps, bps, work, s);      \
    return launch_decode_t<KIND, 32, BATCH>(a, warps, bps, work, s);                 \
  }
  GC_DISPATCH(GC_SIMPLE)
  GC_DISPATCH(GC_SCHEME)
  GC_DISPATCH(GC_AFOR)
  GC_DISPATCH(GC_PFD)
#undef GC_DISPATCH
  return cudaErrorInvalidValue;
}

// Launch shape from the caller's request (NULL = defaults); GC_ERR_INVALID
// for a shape out of range.
gc_status launch_shape(const gc_launch* l, uint32_t* warps, uint32_t* bps, uint32_t* claim) {
  *warps = kDefaultWarps;
  *bps = 0;
  *claim = kDefaultClaim;
  if (!l) return GC_OK;
  if (l->warps_per_block < 1 || l->warps_per_block > kMaxWarps) return GC_ERR_INVALID;
  if (l->items_per_claim > kMaxClaim) return GC_ERR_INVALID;
  *warps = l->warps_per_block;
  *bps = l->blocks_per_sm;
  if (l->items_per_claim) *claim = l->items_per_claim;
  return GC_OK;
}

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

uint64_t index_scratch(const gc_codec& c, uint64_t n) {
  // bound the control bytes by the encoder's maximum
  uint64_t cc = 0, dc = 0, nt = 0;
  gc_max_encoded_size(&c, n, &cc, &dc, &nt);
  const uint64_t R = (n + c.k - 1) / c.k;
  const uint64_t chunks = index_chunks(c, index_nunits(c, R, cc));
  const uint64_t blocks = (chunks + kIndexThreads - 1) / kIndexThreads;
  return gc_host::align_up(blocks * sizeof(UnitAgg) + 64, 256) + gc_host::align_up(nt * sizeof(gc_tile), 256);
}

gc_status build_tiles_impl(const gc_codec& c, const uint8_t* ctrl, uint64_t ctrl_bytes, uint64_t n,
                           gc_tile* tiles, UnitAgg* sums, uint32_t* status, cudaStream_t s) {
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
  // tile 0 is always all zeros; emit writes it too when unit 0 exists
  cudaMemsetAsync(tiles, 0, sizeof(gc_tile), s);
  k_index_sums<<<(unsigned)blocks, kIndexThreads, 0, s>>>(a);
  k_index_scan<<<1, kIndexThreads, 0, s>>>(sums, blocks);
  k_index_emit<<<(unsigned)blocks, kIndexThreads, 0, s>>>(a);
  gc_host::count_launch(3);
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

}  // namespace

extern "C" {

gc_status gc_decode_scratch_size(const gc_codec* codec, uint64_t n, int have_tiles, uint64_t* bytes) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!bytes) return GC_ERR_INVALID;
  const uint64_t R = (n + codec->k - 1) / codec->k;
  const uint64_t tr = kTileInts / codec->k;
  const uint64_t nt = (R + tr - 1) / tr;
  uint64_t b = gc_host::align_up(64, 256) + gc_host::align_up(nt * 8, 256);  // counters + look-back
  if (!have_tiles) b += index_scratch(*codec, n);
  *bytes = b;
  return GC_OK;
}

gc_status gc_build_tiles(const gc_codec* codec, const uint8_t* d_ctrl, uint64_t ctrl_bytes, uint64_t n,
                         gc_tile* d_tiles, void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status,
                         void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (n == 0) return GC_OK;
  if ((!d_ctrl && ctrl_bytes) || !d_tiles || !d_scratch) return GC_ERR_INVALID;
  if (scratch_bytes < index_scratch(*codec, n)) return GC_ERR_NOSPACE;
  return build_tiles_impl(*codec, d_ctrl, ctrl_bytes, n, d_tiles, (UnitAgg*)d_scratch, d_status,
                          (cudaStream_t)stream);
}

gc_status gc_decode(const gc_codec* codec, const uint8_t* d_ctrl, uint64_t ctrl_bytes,
                    const uint32_t* d_data, uint64_t data_words, uint64_t n, const gc_tile* d_tiles,
                    uint32_t* d_out, int restore_docids, void* d_scratch, uint64_t scratch_bytes,
                    uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (n == 0) return GC_OK;
  // an area may be empty (a Group-PFD or AFOR list of zeros has no data
  // words); a non-empty one needs a pointer
  if ((!d_ctrl && ctrl_bytes) || (!d_data && data_words) || !d_out || !d_scratch) return GC_ERR_INVALID;
  if (((uintptr_t)d_data & 15) != 0) return GC_ERR_INVALID;
  uint64_t need = 0;
  gc_decode_scratch_size(codec, n, d_tiles != nullptr, &need);
  if (scratch_bytes < need) return GC_ERR_NOSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t R = (n + codec->k - 1) / codec->k;
  const uint64_t tr = kTileInts / codec->k;
  const uint64_t nt = (R + tr - 1) / tr;
  if (nt > 0xffffffffull - kMaxClaim * kMaxWarps) return GC_ERR_UNSUPPORTED;
  unsigned char* base = (unsigned char*)d_scratch;
  uint32_t* counters = (uint32_t*)base;
  unsigned long long* lb = (unsigned long long*)(base + gc_host::align_up(64, 256));
  unsigned char* rest = base + gc_host::align_up(64, 256) + gc_host::align_up(nt * 8, 256);
  const gc_tile* tiles = d_tiles;
  uint32_t launches = 0;
  if (!tiles) {
    const uint64_t chunks_bytes = index_scratch(*codec, n) - gc_host::align_up(nt * sizeof(gc_tile), 256);
    gc_tile* built = (gc_tile*)(rest + chunks_bytes);
    st = build_tiles_impl(*codec, d_ctrl, ctrl_bytes, n, built, (UnitAgg*)rest, d_status, s);
    if (st != GC_OK) return st;
    launches += gc_host::launches();
    tiles = built;
  }
  if (cudaMemsetAsync(base, 0, gc_host::align_up(64, 256) + (restore_docids ? nt * 8 : 0), s) != cudaSuccess)
    return GC_ERR_CUDA;
  DecodeArgs a = {};
  a.one = ListRef{d_ctrl, ctrl_bytes, d_data, data_words, d_out, n};
  a.one_tiles = tiles;
  a.one_ntiles = nt;
  a.counters = counters;
  a.lb = lb;
  a.cg = codec->cg;
  a.ld = codec->ld;
  a.restore = restore_docids;
  a.status = d_status;
  a.claim = kDefaultClaim;
  gc_host::reset_launches();
  cudaError_t e = launch_decode<false>(codec->kind, codec->k, a, kDefaultWarps, 0, nt, s);
  gc_host::count_launch(launches);
  return e == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

gc_status gc_decode_paper(const gc_codec* codec, const uint8_t* d_buf, uint64_t buf_bytes, uint64_t n,
                          uint32_t* d_out, int restore_docids, void* d_scratch, uint64_t scratch_bytes,
                          uint32_t* d_status, void* stream) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!d_buf || buf_bytes < 4) return GC_ERR_INVALID;
  uint32_t off_words = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&off_words, d_buf, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GC_ERR_CUDA;
  const uint64_t doff = 4ull * off_words;
  if (doff < 4 || doff > buf_bytes || (doff & 15)) return GC_ERR_CORRUPT;
  return gc_decode(codec, d_buf + 4, doff - 4, (const uint32_t*)(d_buf + doff), (buf_bytes - doff) / 4, n,
                   nullptr, d_out, restore_docids, d_scratch, scratch_bytes, d_status, stream);
}

gc_status gc_plan_batch(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists, const gc_tile* d_tile_pool,
                        uint64_t tile_pool_len, gc_work* d_work, uint64_t work_cap, uint64_t* d_count,
                        uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!d_count || (nlists && (!d_lists || !d_work))) return GC_ERR_INVALID;
  if (nlists > 0xffffffffull || work_cap > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_count, 0, 8, s) != cudaSuccess) return GC_ERR_CUDA;
  if (nlists == 0) return GC_OK;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(d_count);
  k_plan_reserve<<<(unsigned)((nlists + 255) / 256), 256, 0, s>>>(d_lists, nlists, codec->k, d_work, work_cap, cnt,
                                                                  d_status);
  if (work_cap)
    k_plan_fill<<<(unsigned)((work_cap + 255) / 256), 256, 0, s>>>(d_lists, nlists, d_tile_pool,
                                                                   d_tile_pool ? tile_pool_len : 0, d_work,
                                                                   work_cap, cnt, d_status);
  gc_host::count_launch(work_cap ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

gc_status gc_decode_plan_scratch_size(uint64_t work_cap, uint64_t* bytes) {
  if (!bytes) return GC_ERR_INVALID;
  *bytes = gc_host::align_up(64, 256) + gc_host::align_up(work_cap * 8, 256);
  return GC_OK;
}

gc_status gc_decode_plan(const gc_codec* codec, const gc_work* d_work, const uint64_t* d_count, uint64_t work_cap,
                         const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes, const uint32_t* d_data_pool,
                         uint64_t data_pool_words, uint32_t* d_out_pool, uint64_t out_pool_len, int restore_docids,
                         const gc_launch* launch, void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status,
                         void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (work_cap == 0) return GC_OK;
  if (!d_work || !d_count || (!d_ctrl_pool && ctrl_pool_bytes) || (!d_data_pool && data_pool_words) ||
      !d_out_pool || !d_scratch)
    return GC_ERR_INVALID;
  if (((uintptr_t)d_data_pool & 15) != 0 || ((uintptr_t)d_work & 15) != 0) return GC_ERR_INVALID;
  if (work_cap > 0xffffffffull - kMaxClaim * kMaxWarps) return GC_ERR_UNSUPPORTED;
  uint64_t need = 0;
  gc_decode_plan_scratch_size(work_cap, &need);
  if (scratch_bytes < need) return GC_ERR_NOSPACE;
  uint32_t warps, bps, claim;
  st = launch_shape(launch, &warps, &bps, &claim);
  if (st != GC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = (unsigned char*)d_scratch;
  uint32_t* counters = (uint32_t*)base;
  unsigned long long* lb = (unsigned long long*)(base + gc_host::align_up(64, 256));
  if (cudaMemsetAsync(base, 0, 64, s) != cudaSuccess) return GC_ERR_CUDA;
  if (restore_docids && cudaMemsetAsync(lb, 0, work_cap * 8, s) != cudaSuccess) return GC_ERR_CUDA;
  DecodeArgs a = {};
  a.work = d_work;
  a.work_count = reinterpret_cast<const unsigned long long*>(d_count);
  a.work_cap = work_cap;
  a.ctrl_pool = d_ctrl_pool;
  a.ctrl_pool_bytes = ctrl_pool_bytes;
  a.data_pool = d_data_pool;
  a.data_pool_words = data_pool_words;
  a.out_pool = d_out_pool;
  a.out_pool_len = out_pool_len;
  a.counters = counters;
  a.lb = lb;
  a.cg = codec->cg;
  a.ld = codec->ld;
  a.claim = claim;
  a.restore = restore_docids;
  a.status = d_status;
  cudaError_t e = launch_decode<true>(codec->kind, codec->k, a, warps, bps, work_cap, s);
  return e == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

gc_status gc_decode_batch_scratch_size(uint64_t nlists, uint64_t max_tiles, uint64_t* bytes) {
  (void)nlists;
  if (!bytes) return GC_ERR_INVALID;
  uint64_t dec = 0;
  gc_decode_plan_scratch_size(max_tiles, &dec);
  *bytes = gc_host::align_up(64, 256) + gc_host::align_up(max_tiles * sizeof(gc_work), 256) + dec;
  return GC_OK;
}

gc_status gc_decode_batch(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists,
                          const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes, const uint32_t* d_data_pool,
                          uint64_t data_pool_words, const gc_tile* d_tile_pool, uint64_t tile_pool_len,
                          uint32_t* d_out_pool, uint64_t out_pool_len, int restore_docids, uint64_t max_tiles,
                          const gc_launch* launch, void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status,
                          void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (nlists == 0 || max_tiles == 0) return GC_OK;
  if (!d_lists || (!d_ctrl_pool && ctrl_pool_bytes) || (!d_data_pool && data_pool_words) || !d_out_pool ||
      !d_scratch)
    return GC_ERR_INVALID;
  if (((uintptr_t)d_data_pool & 15) != 0) return GC_ERR_INVALID;
  if (max_tiles > 0xffffffffull - kMaxClaim * kMaxWarps || nlists > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  uint64_t need = 0;
  gc_decode_batch_scratch_size(nlists, max_tiles, &need);
  if (scratch_bytes < need) return GC_ERR_NOSPACE;
  uint32_t warps, bps, claim;
  st = launch_shape(launch, &warps, &bps, &claim);
  if (st != GC_OK) return st;
  unsigned char* base = (unsigned char*)d_scratch;
  uint64_t* count = (uint64_t*)base;
  gc_work* work = (gc_work*)(base + gc_host::align_up(64, 256));
  unsigned char* rest = base + gc_host::align_up(64, 256) + gc_host::align_up(max_tiles * sizeof(gc_work), 256);
  st = gc_plan_batch(codec, d_lists, nlists, d_tile_pool, tile_pool_len, work, max_tiles, count, d_status, stream);
  if (st != GC_OK) return st;
  const uint32_t planned = gc_host::launches();
  uint64_t dec = 0;
  gc_decode_plan_scratch_size(max_tiles, &dec);
  st = gc_decode_plan(codec, work, count, max_tiles, d_ctrl_pool, ctrl_pool_bytes, d_data_pool, data_pool_words,
                      d_out_pool, out_pool_len, restore_docids, launch, rest, dec, d_status, stream);
  gc_host::count_launch(planned);
  return st;
}

}  // extern "C"
