// gc_decode.cu -- the decoder of the Group-codec library.
//
// Decoding runs a plan: one 64-byte record (gc_work) per 1024-int tile of
// every list, giving the unit that holds the tile's first row and the exact
// byte ranges of the tile's control and data streams. The persistent kernel
// gives each block one staging warp and several decoding warps that share a
// shared-memory ring:
//   - the staging warp claims up to 32 records at a time from a shared
//     counter (one bulk copy brings them into shared memory, the next
//     claim's copy in flight while the current one is placed), sizes every
//     tile's staging in parallel (one lane per record), groups the records
//     into packs of up to 32 lines of 32 consecutive ints (one whole tile,
//     or several small tiles together), places each pack in the ring and
//     hands it to its decoding warp through the pack slot's mbarrier;
//   - decoding warp w takes packs w, w + W, w + 2W, ...; it copies the next
//     pack's bytes into the ring (16-byte cp.async per lane, one commit
//     group per pack) while it decodes the current one. At k = 32 every
//     128-byte data vector lands at a 144-byte pitch, so that the lanes of a
//     warp reading 32 different rows hit different banks. The control
//     patterns become one (word, shift, width) entry per row -- Table III
//     selectors (Sec 4.3), Eq. 2 length descriptors (Sec 5.2.3, 5.3.1),
//     AFOR frame bytes (Sec 6.1), PFD frame headers (Sec 6.2 decoding
//     Step 1) -- lane l extracts the 32 ints of line l with funnel shifts,
//     Group-PFD exceptions are patched over their slots (Step 3), the
//     running sum of the line goes to a per-warp transpose buffer, and the
//     pack's ring bytes are given back;
//   - docIDs (Sec 2.1.1): a warp scan joins the line sums of each tile, and
//     a tile starts from its base (a skip entry of the index) or, without
//     one, from the tiles before it by a bounded decoupled look-back;
//   - 16-byte chunks of the transpose buffer, plus each line's base, go out
//     as coalesced 16-byte stores.
#include <cstdint>
#include <mutex>
#include <type_traits>
#include <cuda_runtime.h>

#include "gc_device.cuh"
#include "gc_host.h"

namespace gcdev {

constexpr unsigned long long kFlagAgg = 1ull << 32;
constexpr unsigned long long kFlagPrefix = 2ull << 32;
constexpr uint64_t kWaitNs = 1000000000ull;  // a wait gives up after 1 s

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kChunk = 32;               // plan records per claim (one per lane of the staging warp)
constexpr int kNRec = 96;                // record slots per block
constexpr int kNChunk = kNRec / kChunk;  // claims whose records a block holds at once
constexpr int kMaxSlots = 64;            // pack slots per block (one mbarrier pair each)
constexpr int kCtrlCap = 512;            // control bytes staged per tile at most
constexpr int kExcCap = 1024;            // exception bytes staged per tile (all or none)
constexpr int kVecPitch = 144;           // k = 32: ring bytes per staged 128-byte data vector
constexpr int kVecWords = kVecPitch / 4;
constexpr int kPackCap = 12288;          // ring bytes one pack may take at most
constexpr int kPadVec4 = 272;            // k = 4: data vectors of a pack, re-laid at 4 words each plus one per 8

static_assert(kNRec % kChunk == 0, "record slots hold whole claims");

// A record slot taken from a warp's buffers or a pack's first slot plus a
// lane: kept inside the record arrays (a pack's records lie in one claim's
// buffer, so for the pack's own lanes this is the identity).
__device__ __forceinline__ uint32_t rslot(uint32_t x) { return x < (uint32_t)kNRec ? x : (uint32_t)kNRec - 1; }

template <int K>
struct Geo {
  static constexpr int TR = kTileInts / K;   // rows per tile
  static constexpr int RPL = 32 / K;         // rows per 32-int line (K = 4: 8, K = 32: 1)
  static constexpr int PROWS = 32 * RPL;     // row entries of a pack
  static constexpr int MAXVEC = TR + 1;      // data vectors a tile spans at most
  // k = 32: the pack's 32 lines (transpose buffer); k = 4: the pack's data
  // re-laid, then the transpose buffer
  static constexpr int TBW = K == 32 ? 32 * 32 : 4 * kPadVec4 + kPadVec4 / 8;
  static constexpr int VB = K == 32 ? kVecPitch : 16;  // ring bytes per staged data vector
  static constexpr int THREADS = K == 32 ? 768 : 512;  // launch bound of the kernel
};

// What the staging warp and the decoding warps of a block share.
struct __align__(128) BlockSmem {
  uint4 rec[kNRec][4];        // claimed plan records
  uint32_t item[kNRec];       // plan index of each
  uint32_t at[kNRec];         // ring offset of its staged bytes (its decoding warp writes it)
  uint32_t rrel[kNRec];       // the same, from its pack's start
  uint16_t fvecs[kNRec];      // data vectors staged for it
  uint16_t cst[kNRec];        // control bytes staged
  uint16_t xst[kNRec];        // exception bytes staged
  uint8_t flines[kNRec];      // its 32-int lines (0: not decoded)
  uint32_t pk[kMaxSlots];     // pack: first record slot | records << 8 | lines << 16 (0 records: stop)
  uint32_t prel[kMaxSlots];   // ring bytes the pack gives back
  uint32_t ppos[kMaxSlots];   // ring offset of the pack
  unsigned long long full[kMaxSlots];   // pack staged
  unsigned long long empty[kMaxSlots];  // pack decoded
  unsigned long long recbar[kNChunk];   // records of a claim copied
};

// One decoding warp's own buffers.
template <int K>
struct __align__(128) WarpSmem {
  uint32_t tb[Geo<K>::TBW];              // transpose buffer (k = 4: re-laid data first)
  uint32_t rw[Geo<K>::PROWS];            // row: word of its first word (lane 0)
  uint32_t rs[Geo<K>::PROWS];            // row: shift | width << 8
  unsigned long long iout[32];           // pack item (by rank among decoded ones): first output int
  unsigned long long lout[32];           // line: output index of its first int
  uint32_t inint[32];                    // item: its ints
  uint32_t ibase[32];                    // item: its docID base
  uint32_t irec[32];                     // item: its record slot
  uint32_t lnv[32];                      // line: ints it holds
  uint32_t emask[32];                    // (Group-PFD, k = 32) line: its exception columns
};

struct DecodeArgs {
  const gc_work* work;
  const unsigned long long* count;  // [0] records, [1] records that need look-back
  uint64_t work_cap;
  const uint8_t* ctrl_pool;
  uint64_t ctrl_pool_bytes;
  const uint32_t* data_pool;
  uint64_t data_pool_words;
  uint32_t* out_pool;
  uint64_t out_pool_len;
  uint32_t* counter;        // claim counter (zeroed before the launch)
  unsigned long long* lb;   // look-back word per record (zeroed when restoring)
  uint32_t cg, ld;
  uint32_t claim;           // records per claim (1..32)
  uint32_t ring_bytes;      // staging ring of a block
  uint32_t* status;
};

// ------------------------------------------------------------- async copy

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 16 bytes global -> shared through the load path (not the bulk-copy unit:
// a 16-byte copy costs the issuing warp about as much as a load)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// whether the phase of `bar` with this parity has completed (no waiting)
__device__ __forceinline__ bool mbar_test_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of `bar` with this parity; the thread is suspended
// (it issues nothing) until the phase completes or about 0.1 ms passes.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}
// Every lane of the warp waits for the phase of `bar` with this parity to
// complete; false (in every lane) when it has not after kWaitNs.
__device__ __forceinline__ bool wait_warp(unsigned long long* bar, uint32_t parity) {
  bool ok = mbar_try_wait(bar, parity);
  if (__all_sync(kFull, ok)) return true;
  const uint64_t t0 = now_ns();
  for (;;) {
    if (!ok) ok = mbar_try_wait(bar, parity);
    if (__all_sync(kFull, ok)) return true;
    if (__any_sync(kFull, now_ns() - t0 > kWaitNs)) return false;
  }
}

// ------------------------------------------------------------ control view

// The control bytes of one list, as the parsers see them: byte `off` (from
// the list's control area) comes from the staged control window, the staged
// exception window or global memory, and past the list's end reads `fill`.
struct CtrlView {
  const uint8_t* g;
  uint64_t size;
  const uint8_t* s1;  // staged control window
  int64_t lo1;
  uint32_t len1;
  const uint8_t* s2;  // staged exception window
  int64_t lo2;
  uint32_t len2;

  __device__ __forceinline__ uint32_t byte(uint64_t off, uint32_t fill) const {
    if (off >= size) return fill;
    uint64_t r = off - (uint64_t)lo1;
    if (r < len1) return s1[r];
    r = off - (uint64_t)lo2;
    if (r < len2) return s2[r];
    return __ldg(g + off);
  }
  // little-endian read of nb (1..4) bytes
  __device__ __forceinline__ uint32_t le(uint64_t off, uint32_t nb, uint32_t fill = 0) const {
    uint32_t v = 0;
    for (uint32_t t = 0; t < nb; ++t) v |= byte(off + t, fill) << (8 * t);
    return v;
  }
  __device__ __forceinline__ uint32_t bits(uint64_t pos, uint32_t width) const {
    return (le(pos >> 3, 4) >> (pos & 7)) & low_mask(width);
  }
  // whether bytes lo..hi (inclusive) of the list are all in the staged
  // control window (then s1[off - lo1] reads them)
  __device__ __forceinline__ bool in_win1(uint64_t lo, uint64_t hi) const {
    return hi < size && (int64_t)lo >= lo1 && hi - (uint64_t)lo1 < len1;
  }
  // 4 little-endian bytes at off (off + 4 <= size)
  __device__ __forceinline__ uint32_t le4(uint64_t off) const {
    if (in_win1(off, off + 3)) {
      const uint8_t* p = s1 + (off - (uint64_t)lo1);
      return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
    }
    return le(off, 4);
  }
  // generic address of bytes [off, off + n) (in a staged window when all
  // of them are there, else in global memory; the caller keeps them inside
  // the list)
  __device__ __forceinline__ const uint8_t* addr(uint64_t off, uint64_t n) const {
    uint64_t r = off - (uint64_t)lo2;
    if (r < len2 && r + n <= len2) return s2 + r;
    r = off - (uint64_t)lo1;
    if (r < len1 && r + n <= len1) return s1 + r;
    return g + off;
  }
};

// Where a parser puts row q of the tile: the ring word of the row's first
// word in lane 0's stream, and (shift, width). A row that would run past the
// staged data vectors is an error (its width becomes 0).
template <int K>
struct RowSink {
  uint32_t* rw;
  uint32_t* rs;
  uint32_t word0;     // buffer word of the tile's first staged word
  uint32_t stride;    // buffer words per data vector (K staged, 33 re-laid)
  uint32_t bit0;      // lane bit of the tile's first row in that word
  uint32_t vec_bits;  // 32 * staged vectors

  __device__ __forceinline__ void put(uint32_t q, uint32_t rb, uint32_t w, bool& ok) const {
    const uint32_t b = bit0 + rb;
    const bool bad = b + w > vec_bits;
    ok = ok && !bad;
    rw[q] = word0 + (bad ? 0u : (b >> 5) * stride);
    rs[q] = bad ? 0u : ((b & 31u) | (w << 8));
  }
};

// Rows [lo, hi) of a tile that a batch of up to 32 units covers, one unit
// per lane in order: the unit of lane u starts at row `start` (tile-relative,
// may be negative), its rows are `w` bits wide, and its first row is at lane
// bit `lb` (from the tile's first row). Lane q takes row r0 + q of each
// chunk of 32 rows: the units that start before the chunk, plus those that
// start in it at or before row r0 + q (a bit set over the chunk), give its
// unit, whose start, width and first bit come by shuffle.
template <int K>
__device__ __forceinline__ void emit_rows(int32_t start, uint32_t w, uint32_t lb, int32_t lo, int32_t hi,
                                          const RowSink<K>& out, bool& ok) {
  const uint32_t lane = lane_id();
  for (int32_t r0 = lo; r0 < hi; r0 += 32) {
    const uint32_t before = __popc(__ballot_sync(kFull, start < r0));
    const int32_t d = start - r0;
    const uint32_t M = __reduce_or_sync(kFull, (d >= 0 && d < 32) ? 1u << d : 0u);
    const int32_t r = r0 + (int32_t)lane;
    const uint32_t u = before + __popc(M & (0xffffffffu >> (31u - lane))) - 1u;
    const int32_t st = __shfl_sync(kFull, start, u & 31u);
    const uint32_t wu = __shfl_sync(kFull, w, u & 31u);
    const uint32_t lbu = __shfl_sync(kFull, lb, u & 31u);
    if (r < hi) out.put((uint32_t)r, lbu + (uint32_t)(r - st) * wu, wu, ok);
  }
}

// ---------------------------------------------------------------- parsers
// Each fills rows 0..rows-1 of the tile (tile-relative) and returns false
// (in every lane) for a malformed stream.

// Table III selectors, 4 bits each, low nibble first; selector u holds NUM
// rows of BW bits in one 32-bit word of every lane (Sec 4.1.1, 4.3).
template <int K>
__device__ __forceinline__ bool parse_simple(const CtrlView& C, uint64_t ctrl_bit, uint32_t skip, uint32_t rows,
                             const RowSink<K>& out) {
  const uint32_t lane = lane_id();
  const uint64_t u0 = ctrl_bit >> 2;
  int32_t cov = -(int32_t)skip;  // first row (tile-relative) of the next selector
  bool ok = true;
  for (uint32_t c = 0; cov < (int32_t)rows; c += 32) {
    const uint64_t u = u0 + c + lane;
    const uint32_t sel = (C.byte(u >> 1, 0xffu) >> ((u & 1) * 4)) & 15u;
    const bool bad = sel > 9;
    const uint32_t num = bad ? 32u : sel_num(sel);
    const uint32_t bw = bad ? 0u : sel_bw(sel);
    const uint32_t incl = warp_incl_sum(num);
    const int32_t start = cov + (int32_t)(incl - num);
    if (bad && start < (int32_t)rows) ok = false;
    const int32_t end = cov + (int32_t)__shfl_sync(kFull, incl, 31);
    emit_rows<K>(start, bw, 32u * (c + lane), cov > 0 ? cov : 0, end < (int32_t)rows ? end : (int32_t)rows, out,
                 ok);
    cov = end;
  }
  return __all_sync(kFull, ok);
}

// Binary length descriptors at fixed positions (Sec 5.2.1(b)); the width of
// row r is CG * (descriptor + 1) (Eq. 2).
template <int K>
__device__ __forceinline__ bool parse_scheme_binary(const CtrlView& C, uint64_t row0, uint32_t rows, uint32_t cg,
                                    const RowSink<K>& out) {
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
      if (((pos + width + 7) >> 3) > C.size) ok = false;
      const uint32_t u = C.bits(pos, width) + 1;
      if (u > maxu) ok = false;
      bw = cg * u;
    }
    const uint32_t incl = warp_incl_sum(bw);
    if (q < rows) out.put(q, carry + incl - bw, bw, ok);
    carry += __shfl_sync(kFull, incl, 31);
  }
  return __all_sync(kFull, ok);
}

// Unary descriptors (Sec 5.2.1(a), 5.3.1): (u - 1) ones closed by a zero.
// Lanes take byte-aligned 32-bit windows of the control stream; each zero
// closes one descriptor. CU: a descriptor starts right after the previous
// zero (possibly in an earlier window). IU: descriptors never straddle a
// byte, so one starts after the previous zero of its byte or at the byte's
// first bit; trailing ones of a byte are padding. While the windows lie in
// the staged control bytes only those are read; past them, 32 at a time.
template <int K>
__device__ __forceinline__ bool parse_scheme_unary(const CtrlView& C, uint64_t P0, uint32_t rows, uint32_t cg, bool iu,
                                   const RowSink<K>& out) {
  const uint32_t lane = lane_id();
  const uint64_t A = P0 & ~7ull;
  const uint32_t maxu = 32 / cg;
  // staged windows from A on (the staged range ends at lo1 + len1)
  const int64_t sh_end = C.lo1 + (int64_t)C.len1;
  uint32_t found = 0, ubase = 0;
  int64_t prev_last = (int64_t)P0 - 1;  // last zero before the current window group
  bool ok = true;
  for (uint64_t w = 0; found < rows;) {
    const uint64_t gbyte = (A >> 3) + 4 * w;  // first byte of this window group
    if (gbyte >= C.size) {
      ok = false;  // ran off the control area
      break;
    }
    uint32_t lim = 32;
    if ((int64_t)gbyte < sh_end && (int64_t)gbyte >= C.lo1) {
      const uint64_t nst = ((uint64_t)(sh_end - (int64_t)gbyte) + 3) / 4;
      lim = nst < 32 ? (uint32_t)nst : 32u;
    }
    const bool act = lane < lim;
    const uint64_t wbit = A + 32 * (w + lane);
    uint32_t win = act ? C.le(wbit >> 3, 4, 0xffu) : 0xffffffffu;
    if (act && wbit < P0) win |= (1u << (uint32_t)(P0 - wbit)) - 1u;
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
        out.put(q, cg * ub, cg * u, ok);
        ub += u;
        ++q;
        pv = p;
      }
    }
    found += __shfl_sync(kFull, incl_nz, 31);
    ubase += __shfl_sync(kFull, incl_us, 31);
    const int64_t gl = __shfl_sync(kFull, incl_last, 31);
    if (gl > prev_last) prev_last = gl;
    w += lim;
  }
  return __all_sync(kFull, ok);
}

// Group-AFOR frame bytes: (size code << 6) | b; a frame is 8 << code rows of
// b bits in every lane (Sec 6.1). A frame may start before the tile; the
// staged data starts at the tile's first row, so offsets are taken from
// there (the frame's first `skip` rows, skip * b bits, are not staged).
template <int K>
__device__ __forceinline__ bool parse_afor(const CtrlView& C, uint64_t ctrl_bit, uint32_t skip, uint32_t rows,
                           const RowSink<K>& out) {
  const uint32_t lane = lane_id();
  const uint64_t f0 = ctrl_bit >> 3;
  int32_t cov = -(int32_t)skip;
  const uint32_t b_first = C.byte(f0, 0xffu) & 63u;
  uint32_t lcarry = 0u - skip * (b_first <= 32 ? b_first : 0u);
  bool ok = true;
  for (uint32_t c = 0; cov < (int32_t)rows; c += 32) {
    const uint32_t byte = C.byte(f0 + c + lane, 0xffu);
    const uint32_t code = byte >> 6, b = byte & 63u;
    const bool bad = code > 2 || b > 32;
    const uint32_t F = bad ? 32u : (8u << code);
    const uint32_t bb = bad ? 0u : b;
    const uint32_t lbits = F * bb;
    const uint32_t inclF = warp_incl_sum(F);
    const uint32_t inclL = warp_incl_sum(lbits);
    const int32_t start = cov + (int32_t)(inclF - F);
    if (bad && start < (int32_t)rows) ok = false;
    const int32_t end = cov + (int32_t)__shfl_sync(kFull, inclF, 31);
    emit_rows<K>(start, bb, lcarry + inclL - lbits, cov > 0 ? cov : 0, end < (int32_t)rows ? end : (int32_t)rows,
                 out, ok);
    cov = end;
    lcarry += __shfl_sync(kFull, inclL, 31);
  }
  return __all_sync(kFull, ok);
}

// Group-PFD at k = 4, decoding Step 3: every exception of a tile's frames
// overwrites its slot in the pack's line-major buffer (line l at words
// 32 l .., 16-byte chunk c at chunk c ^ (l & 7)); the tile's first line is
// line0. Headers and records were checked by pfd_line4; a position outside
// its frame, or one that does not increase on the one before, is reported
// (and not patched).
__device__ __forceinline__ void pfd_patch4(const DecodeArgs& a, uint32_t* tb, const CtrlView& C, uint64_t f0,
                                           uint64_t exc_at, uint32_t rows, uint32_t line0, uint32_t list) {
  const uint32_t lane = lane_id();
  const uint32_t nfr = (rows + kPfdFrameRows - 1) / kPfdFrameRows;
  uint32_t e = 0, wb = 1, xb = 0, lim = 0;
  if (lane < nfr) {
    const uint64_t f = f0 + lane;
    const uint32_t hdr = 4 * f + 4 <= C.size ? C.le(4 * f, 4) : 0u;
    const uint32_t wcode = (hdr >> 6) & 3u;
    const uint32_t frows = rows - 32 * lane < 32 ? rows - 32 * lane : 32;
    lim = frows * 4;
    e = hdr >> 8;
    if ((hdr & 63u) > 32 || wcode > 2 || e > lim) e = 0;
    wb = 1u << wcode;
    xb = e * (1u + wb);
  }
  const uint64_t rec = exc_at + (warp_incl_sum(xb) - xb);
  if (lane < nfr && xb && rec + xb > C.size) e = 0;
  // the tile's exceptions, numbered frame after frame, 32 at a time: a
  // lane's frame is the first whose running count passes its number
  const uint32_t Ei = warp_incl_sum(lane < nfr ? e : 0u);
  const uint32_t E = __shfl_sync(kFull, Ei, 31);
#pragma unroll 1
  for (uint32_t x0 = 0; x0 < E; x0 += 32) {
    const uint32_t xg = x0 + lane;
    uint32_t fl = 0;
#pragma unroll
    for (uint32_t step = 4; step; step >>= 1)  // (a tile has at most 8 frames)
      if (__shfl_sync(kFull, Ei, fl + step - 1) <= xg) fl += step;
    fl &= 7u;
    const uint32_t ef = __shfl_sync(kFull, e, fl), wbf = __shfl_sync(kFull, wb, fl);
    const uint32_t limf = __shfl_sync(kFull, lim, fl), ei = __shfl_sync(kFull, Ei, fl);
    const uint64_t rf = __shfl_sync(kFull, rec, fl);
    if (xg >= E) continue;
    const uint32_t x = xg - (ei - ef);  // its number in its frame
    const uint8_t* rp = C.addr(rf, (uint64_t)ef * (1 + wbf));
    const uint32_t pos = rp[x];
    if (pos >= limf || (x && rp[x - 1] >= pos)) {
      report(a.status, GC_ERR_CORRUPT, list);
      continue;
    }
    const uint8_t* v8 = rp + ef + (size_t)x * wbf;
    uint32_t v = v8[0];
    if (wbf > 1) v |= (uint32_t)v8[1] << 8;
    if (wbf > 2) v |= ((uint32_t)v8[2] << 16) | ((uint32_t)v8[3] << 24);
    const uint32_t i = fl * 128 + pos;  // int of the tile
    const uint32_t line = line0 + (i >> 5), col = i & 31u;
    tb[line * 32 + ((4u * (col >> 2)) ^ (4u * (line & 7u))) + (col & 3u)] = v;
  }
}
// ------------------------------------------------------------ look-back

// Decoupled look-back over the tiles of one list, a warp at a time: the
// tile's aggregate is already published; read the 32 nearest predecessors
// at once; the nearest one that carries an inclusive prefix ends the walk,
// otherwise the window moves 32 tiles back. Tile 0 of a list always carries
// a prefix, so the walk ends inside the list. Returns the exclusive prefix
// (all lanes). Every wait is bounded; one that runs out reports
// GC_ERR_TIMEOUT and the walk stops.
__device__ __noinline__ uint32_t look_back(const unsigned long long* lb, uint64_t item, uint64_t t, uint32_t* status,
                              uint32_t where) {
  const uint32_t lane = lane_id();
  uint32_t excl = 0;
  for (uint64_t d = 1; d <= t; d += 32) {
    const uint64_t dist = d + lane;  // predecessor tile t - dist
    unsigned long long s = kFlagPrefix;
    bool timed_out = false;
    if (dist <= t && dist <= item) {
      s = ld_acquire(lb + item - dist);
      if ((s >> 32) == 0) {
        const uint64_t t0 = now_ns();
        uint32_t nap = 32;  // ns, doubling up to 1 us
        while ((s >> 32) == 0) {
          if (now_ns() - t0 > kWaitNs) {
            timed_out = true;
            break;
          }
          __nanosleep(nap);
          nap = nap < 1024u ? 2 * nap : 1024u;
          s = ld_acquire(lb + item - dist);
        }
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
  return excl;
}

// ------------------------------------------------------------------ pack

__device__ __forceinline__ const gc_work& rec_of(const BlockSmem& h, uint32_t s) {
  return *reinterpret_cast<const gc_work*>(h.rec[s]);
}

__device__ __forceinline__ uint32_t w_nint(uint32_t shape) { return (shape & 1023u) + 1; }
__device__ __forceinline__ uint32_t w_vecs(uint32_t shape) { return (shape >> GC_WORK_VEC_SHIFT) & 511u; }
__device__ __forceinline__ uint32_t w_bit0(uint32_t shape) { return (shape >> GC_WORK_BIT_SHIFT) & 31u; }
__device__ __forceinline__ uint32_t w_skip(uint32_t shape) { return (shape >> GC_WORK_SKIP_SHIFT) & 31u; }

// A record the pack decodes: not empty, its tile fits the output pool, and
// its control area and staged data vectors lie inside their pools.
template <int K>
__device__ __forceinline__ bool w_live(const gc_work& w, const DecodeArgs& a) {
  const uint32_t vecs = w_vecs(w.shape);
  return w.list != 0xffffffffu && w.out_at + w_nint(w.shape) <= a.out_pool_len &&
         (uint64_t)w.ctrl_at + w.ctrl_bytes <= a.ctrl_pool_bytes && vecs <= (uint32_t)Geo<K>::MAXVEC &&
         w.data_at % K == 0 && w.data_at + (uint64_t)vecs * K <= a.data_pool_words;
}

// The records of a pack, one per lane p < np (record slot s0 + p): each
// one's lines and data vectors and where they start in the pack, whether
// it is decoded (live) or only reported (dead: it failed its checks), and
// its rank among the live ones. The live ones' output offsets, sizes and
// record slots go to the warp's buffers by rank.
struct Items {
  uint32_t s, lines, line0, vecs, vec0;
  bool live, dead;
  uint32_t live_mask, heads, rank;
  uint32_t item, tile, base, shape, list;
  uint64_t out;
};

template <int K>
__device__ __forceinline__ Items load_items(const BlockSmem& h, WarpSmem<K>& ws, uint32_t s0, uint32_t np) {
  Items t;
  const uint32_t lane = lane_id();
  const bool inp = lane < np;
  t.s = rslot(s0 + lane);
  const uint32_t lv = inp ? (uint32_t)h.flines[t.s] | (uint32_t)h.fvecs[t.s] << 16 : 0u;
  const uint32_t lvi = np == 1 ? lv : warp_incl_sum(lv);
  t.lines = lv & 0xffffu;
  t.vecs = lv >> 16;
  t.line0 = (lvi & 0xffffu) - t.lines;
  t.vec0 = (lvi >> 16) - t.vecs;
  t.live = t.lines > 0;
  t.live_mask = __ballot_sync(kFull, t.live);
  t.heads = np == 1 ? (t.live_mask & 1u) : __reduce_or_sync(kFull, t.live ? 1u << t.line0 : 0u);
  t.item = 0;
  t.tile = 0;
  t.base = 0;
  t.shape = 0;
  t.list = 0xffffffffu;
  t.out = 0;
  if (inp) {
    const gc_work& w = rec_of(h, t.s);
    t.item = h.item[t.s];
    t.tile = w.tile;
    t.base = w.base;
    t.shape = w.shape;
    t.list = w.list;
    t.out = w.out_at;
  }
  t.dead = inp && !t.live && t.list != 0xffffffffu;
  t.rank = __popc(t.live_mask & ((1u << lane) - 1u));
  if (t.live) {
    ws.iout[t.rank] = t.out;
    ws.inint[t.rank] = w_nint(t.shape);
    ws.irec[t.rank] = t.s;
  }
  return t;
}

// docIDs (Sec 2.1.1), the general case of line_bases: each item's base is
// its skip entry or, without one, the sum of the list's tiles before it by
// look-back (every item publishes its aggregate, then its inclusive
// prefix, for the tiles after it). Lane p holds item p's facts; V is the
// plain warp scan of the line totals T. Returns each line's base. (Kept
// out of line: packs of one tile with a skip entry, most of the work, do
// not need it.)
template <int K>
__device__ __noinline__ uint32_t line_bases_chain(const DecodeArgs& a, WarpSmem<K>& ws, uint32_t V, uint32_t T, bool act,
                                                  uint32_t rank, uint32_t lhead, bool live, bool dead, uint32_t line0,
                                                  uint32_t lines, uint32_t shape, uint32_t tile, uint32_t base_in,
                                                  uint32_t item, uint32_t list, uint32_t irank) {
  const uint32_t lane = lane_id();
  const uint32_t Vb = __shfl_sync(kFull, V, (lhead - 1u) & 31u);
  const uint32_t v = V - (lhead ? Vb : 0u);  // inclusive within the item
  const uint32_t E = v - T;
  const uint32_t lastl = live ? line0 + lines - 1 : 0u;
  const uint32_t tot = __shfl_sync(kFull, v, lastl);
  const bool has_base = (shape & GC_WORK_HAS_BASE) != 0;
  const bool needs_lb = live && tile > 0 && !has_base;
  uint32_t base = has_base ? base_in : 0u;
  if (a.lb) {
    if (live && !needs_lb && (shape & GC_WORK_PUBLISH)) st_release(a.lb + item, kFlagPrefix | (uint32_t)(base + tot));
    if (dead) st_release(a.lb + item, kFlagPrefix);  // its error is reported
    if (needs_lb) st_release(a.lb + item, kFlagAgg | tot);
  }
  // every item whose tile just before has its inclusive prefix already
  // takes it at once (one lane each); the others walk back together
  bool walk = needs_lb;
  if (needs_lb && a.lb) {
    const unsigned long long sp = ld_acquire(a.lb + item - 1);
    if ((sp & ~0xffffffffull) == kFlagPrefix) {
      base = (uint32_t)sp;
      st_release(a.lb + item, kFlagPrefix | (uint32_t)(base + tot));
      walk = false;
    }
  }
  for (uint32_t pend = __ballot_sync(kFull, walk); pend; pend &= pend - 1) {
    const uint32_t p = __ffs(pend) - 1;
    const uint32_t it = __shfl_sync(kFull, item, p);
    const uint32_t tl = __shfl_sync(kFull, tile, p);
    const uint32_t lst = __shfl_sync(kFull, list, p);
    const uint32_t ex = a.lb ? look_back(a.lb, it, tl, a.status, lst) : 0u;
    if (lane == p) {
      base = ex;
      if (a.lb) st_release(a.lb + item, kFlagPrefix | (uint32_t)(ex + tot));
    }
  }
  if (live) ws.ibase[irank] = base;
  __syncwarp();
  return E + (act ? ws.ibase[rank] : 0u);
}

// docIDs (Sec 2.1.1): line l holds the running sum R of its own ints; a
// plain warp scan of the line totals, less the scan before the first line
// of the line's item, is the sum of the item's ints before the line, plus
// the item's base. Returns each line's base.
template <int K>
__device__ __forceinline__ uint32_t line_bases(const DecodeArgs& a, WarpSmem<K>& ws, const Items& t, uint32_t np,
                                               bool act, uint32_t R, uint32_t rank, uint32_t lhead) {
  const uint32_t T = act ? R : 0u;
  const uint32_t V = warp_incl_sum(T);
  const uint32_t shape0 = __shfl_sync(kFull, t.shape, 0);
  if (np == 1 && t.heads == 1u && (shape0 & (GC_WORK_HAS_BASE | GC_WORK_PUBLISH)) == GC_WORK_HAS_BASE) {
    // a pack of one live tile with its skip entry, which no other tile
    // waits for
    return V - T + __shfl_sync(kFull, t.base, 0);
  }
  return line_bases_chain<K>(a, ws, V, T, act, rank, lhead, t.live, t.dead, t.line0, t.lines, t.shape, t.tile, t.base,
                             t.item, t.list, t.rank);
}

// Group-PFD at k = 4 (Sec 6.2 decoding Step 1, pack-wide): line l of the
// pack is rows 8 q .. 8 q + 7 of its tile (q = l - its tile's first line),
// which lie in frame q / 4 (a frame is 32 rows, a tile 8 whole frames).
// Every line reads its frame's header; one scan of 32 b over the lines that
// begin a frame, less the scan before the tile's first line, gives where
// each frame's rows start in the tile's lane streams, so row r of the frame
// is at that start + r b. A malformed header, an exception record past the
// control area or rows past the staged vectors are reported. Returns
// whether a frame of the pack has exceptions.
struct Pfd4Line {
  uint32_t rb0;    // lane bit of the line's first row (from the tile's first staged word)
  uint32_t b;      // its frame's width
  uint32_t v0;     // the tile's first vector in the pack's re-laid buffer
  uint32_t q0;     // the line's first row in the tile
  uint32_t rows;   // rows of the tile
  uint32_t vbits;  // 32 * the tile's staged vectors
};

__device__ __forceinline__ bool pfd_line4(const DecodeArgs& a, const BlockSmem& h, const WarpSmem<4>& ws,
                                          const uint8_t* ring, const Items& t, uint32_t s0, bool act,
                                          uint32_t lane, uint32_t rank, uint32_t lhead, Pfd4Line& pl) {
  const uint32_t sp = rslot(ws.irec[act ? rank : 0u]);
  const gc_work& w = rec_of(h, sp);
  const uint32_t vecs = h.fvecs[sp];
  const uint32_t lq = act ? lane - lhead : 0u;  // line in the tile
  const uint32_t f = lq >> 2;                    // frame in the tile
  const uint32_t rows = (w_nint(w.shape) + 3) / 4;
  const uint32_t at = h.at[sp];
  CtrlView C;
  C.g = a.ctrl_pool + w.ctrl_at;
  C.size = w.ctrl_bytes;
  C.s1 = ring + at + vecs * 16;
  C.lo1 = w.win_at;
  C.len1 = h.cst[sp];
  C.s2 = C.s1 + h.cst[sp];
  C.lo2 = (int64_t)((w.ctrl_at + w.exc_at) & ~15ull) - (int64_t)w.ctrl_at;
  C.len2 = h.xst[sp];
  const uint64_t hp = 4ull * ((uint64_t)w.tile * (Geo<4>::TR / kPfdFrameRows) + f);
  bool ok = hp + 4 <= C.size;
  const uint32_t hdr = act && ok ? C.le4(hp) : 0u;
  uint32_t b = hdr & 63u, wcode = (hdr >> 6) & 3u, e = hdr >> 8;
  const uint32_t frows = rows > 32u * f ? min(32u, rows - 32u * f) : 0u;
  if (b > 32 || wcode > 2 || e > frows * 4) {
    ok = false;
    b = 0;
    e = 0;
  }
  const bool fh = act && (lq & 3u) == 0;  // the line begins its frame
  const uint32_t Vb = warp_incl_sum(fh ? 32u * b : 0u);
  const uint32_t xb = fh ? e * (1u + (1u << wcode)) : 0u;
  const uint32_t Vx = warp_incl_sum(xb);
  const uint32_t fl = lhead + 4 * f;  // the frame's first line
  const uint32_t bF = __shfl_sync(kFull, Vb, (fl - 1u) & 31u), bT = __shfl_sync(kFull, Vb, (lhead - 1u) & 31u);
  const uint32_t xF = __shfl_sync(kFull, Vx, (fl - 1u) & 31u), xT = __shfl_sync(kFull, Vx, (lhead - 1u) & 31u);
  const uint32_t start = (fl ? bF : 0u) - (lhead ? bT : 0u);  // the frame's first lane bit in the tile
  if (fh && xb && w.exc_at + (uint64_t)((fl ? xF : 0u) - (lhead ? xT : 0u)) + xb > C.size) ok = false;
  pl.q0 = 8 * lq;
  pl.rows = rows;
  pl.b = b;
  pl.rb0 = w_bit0(w.shape) + start + 8 * (lq & 3u) * b;
  pl.vbits = 32 * vecs;
  pl.v0 = __shfl_sync(kFull, t.vec0, (sp - s0) & 31u);
  // rows that lie past the staged vectors
  const uint32_t nr = act && pl.q0 < rows ? min(8u, rows - pl.q0) : 0u;
  if (nr && pl.rb0 + nr * b > pl.vbits) ok = false;
  if (act && !ok) report(a.status, GC_ERR_CORRUPT, w.list);
  return __any_sync(kFull, act && e != 0);
}

// The k = 4 pack decoder (the paper's own layout): records s0 .. s0 + np - 1
// of the block (staged, the pack's mbarrier complete), `nl` lines in all.
// Each staged tile's 16-byte vectors are re-laid in the warp's buffer,
// vector v of the pack at word 4 v + v / 8 (one spare word per 8 vectors,
// so that lanes reading different rows mostly hit different banks); every
// tile's control patterns become one (vector, shift, width) entry per row;
// lane l then reads line l (32 ints: rows 8 l .. 8 l + 7 of the pack, 4
// components each) in natural order. Group-PFD exceptions are patched into
// the line-major buffer before the running sum. The pack's ring bytes are
// given back (`empty`) once the data and control bytes are read.
template <int KIND, bool RESTORE, bool PER = false>
__device__ void decode_pack4(const DecodeArgs& a, const BlockSmem& h, WarpSmem<4>& ws, const uint8_t* ring,
                             uint32_t s0, uint32_t np, uint32_t nl, unsigned long long* empty) {
  constexpr uint32_t RPL = Geo<4>::RPL;  // rows per line (8)
  const uint32_t lane = lane_id();
  const Items t = load_items<4>(h, ws, s0, np);

  // 1. per tile: re-lay its vectors, and turn its control patterns into one
  // (vector, shift, width) entry per row
  bool exc = false;  // (Group-PFD) a tile of the pack has exceptions
  for (uint32_t lm = t.live_mask; lm; lm &= lm - 1) {
    const uint32_t p = __ffs(lm) - 1;
    const uint32_t line0 = __shfl_sync(kFull, t.line0, p);
    const uint32_t lines = __shfl_sync(kFull, t.lines, p);
    const uint32_t v0 = __shfl_sync(kFull, t.vec0, p);
    const uint32_t sp = rslot(s0 + p);
    const gc_work& w = rec_of(h, sp);
    const uint32_t at = h.at[sp];
    const uint32_t vecs = h.fvecs[sp];
    {
      // lane l moves vector 32 i + l (one 16-byte load, four stores; the
      // stores of a step hit 32 different banks)
      const uint4* src = reinterpret_cast<const uint4*>(ring + at);
      for (uint32_t v = lane; v < vecs; v += 32) {
        const uint4 x = src[v];
        const uint32_t g = v0 + v;
        uint32_t* d = ws.tb + 4 * g + (g >> 3);
        d[0] = x.x;
        d[1] = x.y;
        d[2] = x.z;
        d[3] = x.w;
      }
    }
    if constexpr (KIND == GC_PFD) continue;  // (its rows come from the frame headers in step 2)
    const uint32_t dbytes = vecs * 16;
    CtrlView C;
    C.g = a.ctrl_pool + w.ctrl_at;
    C.size = w.ctrl_bytes;
    C.s1 = ring + at + dbytes;
    C.lo1 = w.win_at;
    C.len1 = h.cst[sp];
    C.s2 = ring + at + dbytes + h.cst[sp];
    C.lo2 = (int64_t)((w.ctrl_at + w.exc_at) & ~15ull) - (int64_t)w.ctrl_at;
    C.len2 = h.xst[sp];
    RowSink<4> out;
    out.rw = ws.rw + line0 * RPL;
    out.rs = ws.rs + line0 * RPL;
    out.word0 = v0;  // entries hold the row's first vector
    out.stride = 1;
    out.bit0 = w_bit0(w.shape);
    out.vec_bits = 32 * vecs;
    const uint32_t rows = (w_nint(w.shape) + 3) / 4;
    const uint64_t row0 = (uint64_t)w.tile * Geo<4>::TR;
    bool ok;
    if (KIND == GC_SIMPLE) {
      ok = parse_simple<4>(C, w.ctrl_bit, w_skip(w.shape), rows, out);
    } else if (KIND == GC_SCHEME) {
      if (a.ld == GC_LD_BINARY) ok = parse_scheme_binary<4>(C, row0, rows, a.cg, out);
      else ok = parse_scheme_unary<4>(C, w.ctrl_bit, rows, a.cg, a.ld == GC_LD_IU, out);
    } else if (KIND == GC_AFOR) {
      ok = parse_afor<4>(C, w.ctrl_bit, w_skip(w.shape), rows, out);
    } else {
      ok = true;
    }
    // rows of the last line past the tile's end read nothing
    if (lane < lines * RPL - rows) {
      ws.rw[line0 * RPL + rows + lane] = v0;
      ws.rs[line0 * RPL + rows + lane] = 0;
    }
    if (!ok && lane == 0) report(a.status, GC_ERR_CORRUPT, w.list);
  }
  __syncwarp();

  // 2. lane l reads line l: rows 8 l .. 8 l + 7, four components each
  const bool act = lane < nl;
  const uint32_t upto = t.heads & (0xffffffffu >> (31u - lane));  // item heads at lines <= l
  const uint32_t rank = act ? (uint32_t)__popc(upto) - 1u : 0u;    // its item among the decoded ones
  const uint32_t lhead = act ? 31u - __clz(upto) : 0u;            // the item's first line
  // (per-record mode) a line of a GC_WORK_RAW record is written without the
  // running sum; its total then counts 0, and the record's base is 0
  bool sum = RESTORE;
  if constexpr (PER) sum = !act || !(rec_of(h, rslot(ws.irec[rank])).shape & GC_WORK_RAW);
  // Group-PFD: the line's rows straight from its frame's header
  Pfd4Line pl;
  if constexpr (KIND == GC_PFD) exc = pfd_line4(a, h, ws, ring, t, s0, act, lane, rank, lhead, pl);
  uint32_t r[32];
  uint32_t R = 0;
#pragma unroll
  for (int rr = 0; rr < (int)RPL; ++rr) {
    uint32_t vi, sw;
    if constexpr (KIND == GC_PFD) {
      const uint32_t rb = pl.rb0 + (uint32_t)rr * pl.b;
      const bool live = act && pl.q0 + (uint32_t)rr < pl.rows && rb + pl.b <= pl.vbits;
      vi = pl.v0 + (live ? rb >> 5 : 0u);
      sw = live ? (rb & 31u) | (pl.b << 8) : 0u;
    } else {
      const uint32_t row = act ? lane * RPL + rr : 0u;
      vi = act ? ws.rw[row] : 0u;
      sw = act ? ws.rs[row] : 0u;
    }
    const uint32_t sh = sw & 31u, wd = sw >> 8;
    const uint32_t msk = low_mask(wd);
    const bool cross = sh + wd > 32;
    const uint32_t* P0 = ws.tb + 4 * vi + (vi >> 3);
    const uint32_t* P1 = ws.tb + 4 * (vi + 1) + ((vi + 1) >> 3);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t lo = P0[c];
      uint32_t hi = 0;
      if (KIND != GC_SIMPLE && cross) hi = P1[c];  // Group-Simple values never cross a word
      r[4 * rr + c] = __funnelshift_r(lo, hi, sh) & msk;
    }
  }
  if (KIND == GC_PFD && exc) {
    // the values over the exception slots, in the line-major buffer (when
    // a tile of the pack has exceptions)
    uint4* T = reinterpret_cast<uint4*>(ws.tb + lane * 32);
    const uint32_t swz = lane & 7u;
    __syncwarp();  // (the re-laid data is read)
    if (act) {
#pragma unroll
      for (int c = 0; c < 8; ++c) T[c ^ swz] = make_uint4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
    }
    __syncwarp();
    for (uint32_t lm = t.live_mask; lm; lm &= lm - 1) {
      const uint32_t p = __ffs(lm) - 1;
      const uint32_t line0 = __shfl_sync(kFull, t.line0, p);
      const uint32_t sp = rslot(s0 + p);
      const gc_work& w = rec_of(h, sp);
      const uint32_t at = h.at[sp];
      const uint32_t dbytes = h.fvecs[sp] * 16;
      CtrlView C;
      C.g = a.ctrl_pool + w.ctrl_at;
      C.size = w.ctrl_bytes;
      C.s1 = ring + at + dbytes;
      C.lo1 = w.win_at;
      C.len1 = h.cst[sp];
      C.s2 = ring + at + dbytes + h.cst[sp];
      C.lo2 = (int64_t)((w.ctrl_at + w.exc_at) & ~15ull) - (int64_t)w.ctrl_at;
      C.len2 = h.xst[sp];
      const uint64_t row0 = (uint64_t)w.tile * Geo<4>::TR;
      pfd_patch4(a, ws.tb, C, row0 / kPfdFrameRows, w.exc_at, (w_nint(w.shape) + 3) / 4, line0, w.list);
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint4 v = T[c ^ swz];
        r[4 * c] = v.x;
        r[4 * c + 1] = v.y;
        r[4 * c + 2] = v.z;
        r[4 * c + 3] = v.w;
      }
    }
  }
  // the pack's staged bytes are read: give its ring bytes back
  __syncwarp();
  if (lane == 0) mbar_arrive(empty);
  if (sum) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      R += r[j];
      r[j] = R;
    }
  }

  // 3. docIDs: each line's base
  const uint32_t k0 = RESTORE ? line_bases<4>(a, ws, t, np, act, R, rank, lhead) : 0u;

  // the re-laid data is read: its buffer takes the results, line l at words
  // 32 l .. 32 l + 31 with its 16-byte chunk c at chunk c ^ (l & 7), so that
  // the eight lanes of each quarter-warp touch eight different chunks both
  // here (a line per lane) and when reading (a chunk per lane, below)
  __syncwarp();
  const bool whole = t.heads == 1u && ws.inint[0] == (uint32_t)kTileInts;  // one whole tile
  if (act) {
    uint4* T = reinterpret_cast<uint4*>(ws.tb + lane * 32);
    const uint32_t sw = lane & 7u;
#pragma unroll
    for (int c = 0; c < 8; ++c)
      T[c ^ sw] = make_uint4(r[4 * c] + k0, r[4 * c + 1] + k0, r[4 * c + 2] + k0, r[4 * c + 3] + k0);
    if (!whole) {
      ws.lout[lane] = ws.iout[rank] + 32ull * (lane - lhead);
      const uint32_t left = ws.inint[rank] - 32u * (lane - lhead);
      ws.lnv[lane] = left < 32u ? left : 32u;
    }
  }
  __syncwarp();

  // 4. stores. Lane j takes chunk c = j % 8 of lines 4 q + j / 8 and stores
  // it with one 16-byte store where the chunk is whole and its output
  // 16-byte aligned, else word by word. A whole tile whose output is not
  // aligned goes out line by line instead, lane j storing word j (word j of
  // line l sits at word 32 l + 4 ((j / 4) ^ (l & 7)) + j % 4).
  const uint32_t c = lane & 7u;
  uint32_t* o1 = a.out_pool + ws.iout[0];
  if (whole) {
    if ((reinterpret_cast<uintptr_t>(o1) & 15u) == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint32_t rr = 4u * q + (lane >> 3);
        const uint4 v = reinterpret_cast<const uint4*>(ws.tb + rr * 32)[c ^ (rr & 7u)];
        reinterpret_cast<uint4*>(o1 + rr * 32)[c] = v;
      }
    } else {
      const uint32_t wsw = 4u * (lane >> 2), wlo = lane & 3u;
#pragma unroll 1
      for (int rr = 0; rr < 32; ++rr) o1[rr * 32 + lane] = ws.tb[rr * 32 + (wsw ^ (4u * (rr & 7))) + wlo];
    }
  } else {
    for (uint32_t q = 0; 4 * q < nl; ++q) {
      const uint32_t ln = 4 * q + (lane >> 3);
      if (ln < nl) {
        const uint32_t n = ws.lnv[ln];
        const uint4 v = reinterpret_cast<const uint4*>(ws.tb + ln * 32)[c ^ (ln & 7u)];
        uint32_t* o = a.out_pool + ws.lout[ln] + 4 * c;
        if (4 * c + 4 <= n && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
          *reinterpret_cast<uint4*>(o) = v;
        } else {
          if (4 * c < n) o[0] = v.x;
          if (4 * c + 1 < n) o[1] = v.y;
          if (4 * c + 2 < n) o[2] = v.z;
          if (4 * c + 3 < n) o[3] = v.w;
        }
      }
    }
  }
  __syncwarp();
}

// One line (32 ints) of the k = 32 decoder: lane l reads its row's 32 words
// (and, for values that cross a word, the next vector's) as eight 16-byte
// chunks from the ring, where vectors sit 144 bytes apart: the eight lanes
// of a quarter-warp read rows at most one vector apart each, so their
// chunks fall in eight different 16-byte bank groups. Each value is a
// funnel shift and a mask; with SUM the running sum (the prefix within the
// line) replaces it, and R ends as the line's total. The results go to the
// line's 16-byte chunks in the transpose buffer, chunk c at c ^ swz. With
// PATCH, the Group-PFD exceptions of the line are already in the buffer at
// their own places and column j's value is taken from there where bit j of
// em is set (Sec 6.2 decoding Step 3), before the running sum.
template <int KIND, bool SUM, bool PATCH = false>
__device__ __forceinline__ void extract_line32(const uint4* P, uint32_t sh, uint32_t msk, bool cross, uint4* T,
                                               uint32_t swz, uint32_t& R, uint32_t em = 0, bool rsum = true) {
  R = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint4 lo = P[c];
    uint4 hi = make_uint4(0u, 0u, 0u, 0u);
    if (KIND != GC_SIMPLE && cross) hi = P[kVecPitch / 16 + c];  // Group-Simple values never cross a word
    uint32_t v0 = __funnelshift_r(lo.x, hi.x, sh) & msk;
    uint32_t v1 = __funnelshift_r(lo.y, hi.y, sh) & msk;
    uint32_t v2 = __funnelshift_r(lo.z, hi.z, sh) & msk;
    uint32_t v3 = __funnelshift_r(lo.w, hi.w, sh) & msk;
    if (PATCH) {
      const uint32_t m4 = (em >> (4 * c)) & 15u;
      if (m4) {
        const uint4 x = T[c ^ swz];
        v0 = (m4 & 1u) ? x.x : v0;
        v1 = (m4 & 2u) ? x.y : v1;
        v2 = (m4 & 4u) ? x.z : v2;
        v3 = (m4 & 8u) ? x.w : v3;
      }
    }
    if (SUM && rsum) {
      v0 += R;
      v1 += v0;
      v2 += v1;
      v3 += v2;
      R = v3;
    }
    T[c ^ swz] = make_uint4(v0, v1, v2, v3);
  }
}

// Group-Simple, k = 32: the rows of all of a pack's tiles at once. Line l of
// the pack is row q = l - lhead of its tile, and lane l also reads its
// tile's selector q (a tile of R rows needs at most R selectors: each
// covers at least one of its rows, the first one too, since fewer than
// its own rows lie in the tile before). One scan of the selectors' row
// counts (less the scan before the tile's first lane) gives each
// selector's first row; a line then takes the last of its tile's
// selectors that starts at or before it. Returns the line's row entry in
// registers (ring word of the row's word in lane 0's stream, shift | width
// << 8) and reports a tile whose selectors are malformed or do not cover
// its rows.
__device__ __forceinline__ void parse_simple_pack32(const DecodeArgs& a, const BlockSmem& h, const WarpSmem<32>& ws,
                                                    const uint8_t* ring, bool act, uint32_t lane, uint32_t heads,
                                                    uint32_t nl, uint32_t rank, uint32_t lhead, uint32_t& ent,
                                                    uint32_t& sw) {
  // this line's tile (a lane past the pack's lines takes the first tile's)
  const uint32_t s = rslot(ws.irec[act ? rank : 0u]);
  const gc_work& w = rec_of(h, s);
  const uint32_t at = h.at[s], vecs = h.fvecs[s];
  const uint32_t after = heads & ~(0xffffffffu >> (31u - lane));  // heads of later tiles
  const uint32_t rows = (after ? __ffs(after) - 1 : nl) - lhead;
  const uint32_t q = lane - lhead;
  CtrlView C;
  C.g = a.ctrl_pool + w.ctrl_at;
  C.size = w.ctrl_bytes;
  C.s1 = ring + at + vecs * kVecPitch;
  C.lo1 = w.win_at;
  C.len1 = h.cst[s];
  C.s2 = nullptr;
  C.lo2 = 0;
  C.len2 = 0;
  // selector q of the tile (Table III; 4 bits each, low nibble first)
  const uint64_t u = (w.ctrl_bit >> 2) + q;
  const uint32_t sel = act ? (C.byte(u >> 1, 0xffu) >> ((u & 1) * 4)) & 15u : 0u;
  const bool bad = sel > 9;
  const uint32_t num = !act ? 0u : bad ? 32u : sel_num(sel);
  const uint32_t bw = bad ? 0u : sel_bw(sel);
  const uint32_t V = warp_incl_sum(num);
  const uint32_t Vb = __shfl_sync(kFull, V, (lhead - 1u) & 31u);
  const int32_t start = (int32_t)(V - (lhead ? Vb : 0u) - num) - (int32_t)w_skip(w.shape);  // its first row
  const bool valid = act && start < (int32_t)rows;
  bool ok = !(valid && bad);
  const uint32_t M = __reduce_or_sync(kFull, valid ? 1u << (lhead + (start > 0 ? (uint32_t)start : 0u)) : 0u);
  // this line's selector: the k-th of its tile's (the valid ones are a prefix of the tile's lanes)
  const uint32_t k = __popc(M & (0xffffffffu >> (31u - lane)) & ~((1u << lhead) - 1u));
  const uint32_t us = (lhead + k - 1u) & 31u;
  const int32_t st = __shfl_sync(kFull, start, us);
  const uint32_t wu = __shfl_sync(kFull, bw, us);
  const uint32_t nu = __shfl_sync(kFull, num, us);
  const uint32_t b = w_bit0(w.shape) + 32u * (us - lhead) + (uint32_t)((int32_t)q - st) * wu;
  // (a row past its selector's rows means the tile's skip entry and its
  // selectors disagree)
  const bool out_of_range = k == 0 || (uint32_t)((int32_t)q - st) >= nu || b + wu > 32u * vecs;
  if (act && out_of_range) ok = false;
  ent = (at >> 2) + (act && !out_of_range ? (b >> 5) * kVecWords : 0u);
  sw = act && !out_of_range ? (b & 31u) | (wu << 8) : 0u;
  if (!ok) report(a.status, GC_ERR_CORRUPT, w.list);
}

// Group-PFD, k = 32: one tile's exceptions go to their slots' places in the
// pack's line-major buffer (line l at words 32 l .. 32 l + 31, its 16-byte
// chunk c at chunk c ^ (l & 7)), and each one's column to its line's mask
// in em: e 16-bit positions at rp, then e values of wb bytes (Sec 6.2,
// decoding Step 3); the tile's first line is hl, its frame holds lim ints.
// A position outside the frame, or one that does not increase on the one
// before, is reported (and not patched).
__device__ __forceinline__ void pfd_patch(const DecodeArgs& a, uint32_t* tb, uint32_t* em, uint32_t lane, uint32_t hl,
                                          uint32_t e, uint32_t lim, uint32_t wb, const uint8_t* rp, uint32_t list) {
  const uint8_t* vp = rp + (size_t)e * 2;
  uint32_t last = 0;  // the position before this round's first
#pragma unroll 1
  for (uint32_t x0 = 0; x0 < e; x0 += 32) {
    const uint32_t x = x0 + lane;
    const uint32_t pos = x < e ? (uint32_t)rp[2 * x] | ((uint32_t)rp[2 * x + 1] << 8) : 0xffffu;
    const uint32_t up = __shfl_up_sync(kFull, pos, 1);
    const uint32_t before = lane ? up : last;
    last = __shfl_sync(kFull, pos, 31);
    if (x >= e) continue;
    if (pos >= lim || (x && before >= pos)) {
      report(a.status, GC_ERR_CORRUPT, list);
      continue;
    }
    const uint8_t* v8 = vp + (size_t)x * wb;
    uint32_t v = v8[0];
    if (wb > 1) v |= (uint32_t)v8[1] << 8;
    if (wb > 2) v |= ((uint32_t)v8[2] << 16) | ((uint32_t)v8[3] << 24);
    const uint32_t line = hl + (pos >> 5), col = pos & 31u;
    tb[line * 32 + ((4u * (col >> 2)) ^ (4u * (line & 7u))) + (col & 3u)] = v;
    atomicOr(em + line, 1u << col);
  }
}

// The facts of a Group-PFD tile's exceptions that the patch step needs.
struct PfdExc {
  const uint8_t* rp;  // the exception record (positions, then values)
  uint32_t e, wb, lim, list;
};

// Group-PFD, k = 32: the headers and rows of all of a pack's tiles at once
// (a tile is one frame, Sec 6). Line l is row q = l - lhead of its tile:
// every line reads its tile's header (b, exception width code, exception
// count e) and takes row q at q * b bits (lanes past the pack's lines read
// the first tile's). Returns the line's row entry in registers and its
// tile's exception record; reports a tile whose header, row widths or
// exception record are malformed.
__device__ __forceinline__ void parse_pfd_pack32(const DecodeArgs& a, const BlockSmem& h, const WarpSmem<32>& ws,
                                                 const uint8_t* ring, bool act, uint32_t lane, uint32_t heads,
                                                 uint32_t nl, uint32_t rank, uint32_t lhead, uint32_t& ent,
                                                 uint32_t& sw, PfdExc& x) {
  // this line's tile (a lane past the pack's lines takes the first tile's)
  const uint32_t s = rslot(ws.irec[heads ? rank : 0u]);
  const gc_work& w = rec_of(h, s);
  const uint32_t at = h.at[s], vecs = h.fvecs[s];
  const uint32_t after = heads & ~(0xffffffffu >> (31u - lane));  // heads of later tiles
  const uint32_t rows = (after ? __ffs(after) - 1 : nl) - lhead;
  const uint32_t q = lane - lhead;
  CtrlView C;
  C.g = a.ctrl_pool + w.ctrl_at;
  C.size = w.ctrl_bytes;
  C.s1 = ring + at + vecs * kVecPitch;
  C.lo1 = w.win_at;
  C.len1 = h.cst[s];
  C.s2 = C.s1 + h.cst[s];
  C.lo2 = (int64_t)((w.ctrl_at + w.exc_at) & ~15ull) - (int64_t)w.ctrl_at;
  C.len2 = h.xst[s];
  // the header
  const uint64_t hp = 4ull * w.tile;
  bool ok = hp + 4 <= C.size;
  const uint32_t hdr = heads && ok ? C.le4(hp) : 0u;
  uint32_t b = hdr & 63u, wcode = (hdr >> 6) & 3u, e = hdr >> 8;
  if (b > 32 || wcode > 2) {
    ok = false;
    b = 0;
    wcode = 0;
    e = 0;
  }
  const uint32_t lim = rows * 32;  // ints of the frame in this tile
  if (e > lim) {
    ok = false;
    e = 0;
  }
  const uint32_t wb = 1u << wcode;
  if (e && w.exc_at + (uint64_t)e * (2 + wb) > C.size) {
    ok = false;
    e = 0;
  }
  // this line's row
  const uint32_t rb = w_bit0(w.shape) + q * b;
  const bool oor = rb + b > 32u * vecs;
  if (oor) ok = false;
  ent = (at >> 2) + (act && !oor ? (rb >> 5) * kVecWords : 0u);
  sw = act && !oor ? (rb & 31u) | (b << 8) : 0u;
  if (act && !ok) report(a.status, GC_ERR_CORRUPT, w.list);
  x.rp = C.addr(w.exc_at, (uint64_t)e * (2 + wb));
  x.e = e;
  x.wb = wb;
  x.lim = lim;
  x.list = w.list;
}

// Group-PFD, k = 32: the exceptions of every tile of the pack at their
// slots' places, and every line's exception columns.
__device__ __forceinline__ void pfd_patch_pack32(const DecodeArgs& a, uint32_t* tb, uint32_t* em, uint32_t lane,
                                                 uint32_t heads, const PfdExc& x) {
  for (uint32_t hm = heads; hm; hm &= hm - 1) {
    const uint32_t hl = __ffs(hm) - 1;  // the tile's first line
    const uint32_t e = __shfl_sync(kFull, x.e, hl);
    const uint32_t lim = __shfl_sync(kFull, x.lim, hl);
    const uint32_t wb = __shfl_sync(kFull, x.wb, hl);
    const uint32_t list = __shfl_sync(kFull, x.list, hl);
    const uint8_t* rp = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, (unsigned long long)x.rp, hl));
    pfd_patch(a, tb, em, lane, hl, e, lim, wb, rp, list);
  }
}

// The k = 32 pack decoder. Lane l decodes line l (row l of the pack) from
// the ring, where the staging warp put every data vector 144 bytes apart,
// and writes its running sums to line l of the transpose buffer; the scan
// of the line totals gives each line's base, which is added as the buffer
// goes out in 16-byte chunks. The pack's ring bytes are given back
// (`empty`) once they are read.
template <int KIND, bool RESTORE, bool PER = false>
__device__ void decode_pack32(const DecodeArgs& a, const BlockSmem& h, WarpSmem<32>& ws, const uint8_t* ring,
                              uint32_t s0, uint32_t np, uint32_t nl, unsigned long long* empty) {
  const uint32_t lane = lane_id();
  const Items t = load_items<32>(h, ws, s0, np);

  // 1. Group-Scheme, Group-AFOR: per tile, the control patterns become one
  // (word, shift, width) entry per row
  if (KIND == GC_SCHEME || KIND == GC_AFOR) {
    for (uint32_t lm = t.live_mask; lm; lm &= lm - 1) {
      const uint32_t p = __ffs(lm) - 1;
      // (a pack of one: line 0, its nl lines)
      const uint32_t line0 = np == 1 ? 0u : __shfl_sync(kFull, t.line0, p);
      const uint32_t rows = np == 1 ? nl : __shfl_sync(kFull, t.lines, p);
      const uint32_t sp = rslot(s0 + p);
      const gc_work& w = rec_of(h, sp);
      const uint32_t at = h.at[sp];
      const uint32_t vecs = h.fvecs[sp];
      const uint32_t dbytes = vecs * kVecPitch;
      CtrlView C;
      C.g = a.ctrl_pool + w.ctrl_at;
      C.size = w.ctrl_bytes;
      C.s1 = ring + at + dbytes;
      C.lo1 = w.win_at;
      C.len1 = h.cst[sp];
      C.s2 = nullptr;
      C.lo2 = 0;
      C.len2 = 0;
      RowSink<32> out;
      out.rw = ws.rw + line0;
      out.rs = ws.rs + line0;
      out.word0 = at >> 2;
      out.stride = kVecWords;
      out.bit0 = w_bit0(w.shape);
      out.vec_bits = 32 * vecs;
      bool ok;
      if (KIND == GC_SCHEME) {
        const uint64_t row0 = (uint64_t)w.tile * Geo<32>::TR;
        if (a.ld == GC_LD_BINARY) ok = parse_scheme_binary<32>(C, row0, rows, a.cg, out);
        else ok = parse_scheme_unary<32>(C, w.ctrl_bit, rows, a.cg, a.ld == GC_LD_IU, out);
      } else {
        ok = parse_afor<32>(C, w.ctrl_bit, w_skip(w.shape), rows, out);
      }
      if (!ok && lane == 0) report(a.status, GC_ERR_CORRUPT, w.list);
    }
  }
  __syncwarp();

  // 2. lane l extracts line l (row l of the pack)
  const bool act = lane < nl;
  const uint32_t upto = t.heads & (0xffffffffu >> (31u - lane));  // item heads at lines <= l
  const uint32_t rank = act ? (uint32_t)__popc(upto) - 1u : 0u;    // its item among the decoded ones
  const uint32_t lhead = act ? 31u - __clz(upto) : 0u;            // the item's first line
  // (per-record mode) a line of a GC_WORK_RAW record is written without the
  // running sum; its total then counts 0, and the record's base is 0
  bool sum = RESTORE;
  if constexpr (PER) sum = !act || !(rec_of(h, rslot(ws.irec[rank])).shape & GC_WORK_RAW);
  uint32_t ent, sw;
  PfdExc px;
  if (KIND == GC_SIMPLE) {
    parse_simple_pack32(a, h, ws, ring, act, lane, t.heads, nl, rank, lhead, ent, sw);
  } else if (KIND == GC_PFD) {
    parse_pfd_pack32(a, h, ws, ring, act, lane, t.heads, nl, rank, lhead, ent, sw, px);
  } else {
    ent = ws.rw[lane];
    sw = act ? ws.rs[lane] : 0u;
  }
  const uint32_t sh = sw & 31u, wd = sw >> 8;
  const uint32_t msk = low_mask(wd);
  const bool cross = sh + wd > 32;
  // A row of no bits (Group-PFD b = 0, Group-AFOR's all-zero frames, an
  // entry left by a malformed stream) may lie past the tile's staged data,
  // which need not hold even one vector: such rows, and lanes past the
  // pack's lines, read their own line of the buffer instead (the mask
  // makes every value 0).
  const uint4* P = act && wd != 0 ? reinterpret_cast<const uint4*>(ring + 4ull * ent)
                                  : reinterpret_cast<const uint4*>(ws.tb + 32 * lane);
  uint4* T = reinterpret_cast<uint4*>(ws.tb + 32 * lane);
  const uint32_t swz = lane & 7u;
  uint32_t R = 0;
  if (KIND != GC_PFD) {
    extract_line32<KIND, RESTORE>(P, sh, msk, cross, T, swz, R, 0u, sum);
  } else {
    // Group-PFD: when a tile of the pack has exceptions, they first go to
    // their places in the buffer and their columns to each line's mask;
    // one extraction then takes a masked column's value from the buffer
    // instead of its slot (no mask: every value from its slot)
    const bool pp = (__ballot_sync(kFull, px.e != 0) & t.heads) != 0;
    uint32_t em = 0;
    if (pp) {
      ws.emask[lane] = 0;
      __syncwarp();
      pfd_patch_pack32(a, ws.tb, ws.emask, lane, t.heads, px);
      __syncwarp();
      em = ws.emask[lane];
    }
    extract_line32<KIND, RESTORE, true>(P, sh, msk, cross, T, swz, R, em, sum);
  }
  // the pack's staged bytes are read: give its ring bytes back
  __syncwarp();
  if (lane == 0) mbar_arrive(empty);

  // 3. docIDs: each line's base
  const uint32_t k0 = RESTORE ? line_bases<32>(a, ws, t, np, act, R, rank, lhead) : 0u;
  const bool whole = t.heads == 1u && ws.inint[0] == (uint32_t)kTileInts;  // one whole tile
  if (act && !whole) {
    ws.lout[lane] = ws.iout[rank] + 32ull * (lane - lhead);
    const uint32_t left = ws.inint[rank] - 32u * (lane - lhead);
    ws.lnv[lane] = left < 32u ? left : 32u;
  }
  __syncwarp();

  // 4. stores. Lane j takes chunk c = j % 8 of lines 4 q + j / 8, adds the
  // line's base, and stores it with one 16-byte store where the chunk is
  // whole and its output 16-byte aligned, else word by word. A whole tile
  // whose output is not aligned goes out line by line instead, lane j
  // storing word j (word j of line l sits at word 32 l + 4 ((j / 4) ^ (l &
  // 7)) + j % 4).
  const uint32_t c = lane & 7u;
  uint32_t* o1 = a.out_pool + ws.iout[0];
  if (whole) {
    if ((reinterpret_cast<uintptr_t>(o1) & 15u) == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint32_t rr = 4u * q + (lane >> 3);
        uint4 v = reinterpret_cast<const uint4*>(ws.tb + rr * 32)[c ^ (rr & 7u)];
        if (RESTORE) {
          const uint32_t kk = __shfl_sync(kFull, k0, rr);
          v.x += kk;
          v.y += kk;
          v.z += kk;
          v.w += kk;
        }
        reinterpret_cast<uint4*>(o1 + rr * 32)[c] = v;
      }
    } else {
      const uint32_t wsw = 4u * (lane >> 2), wlo = lane & 3u;
#pragma unroll 1
      for (int rr = 0; rr < 32; ++rr) {
        const uint32_t kk = RESTORE ? __shfl_sync(kFull, k0, rr) : 0u;
        o1[rr * 32 + lane] = ws.tb[rr * 32 + (wsw ^ (4u * (rr & 7))) + wlo] + kk;
      }
    }
  } else {
    for (uint32_t q = 0; 4 * q < nl; ++q) {
      const uint32_t ln = 4 * q + (lane >> 3);
      const uint32_t kk = RESTORE ? __shfl_sync(kFull, k0, ln & 31u) : 0u;
      if (ln < nl) {
        const uint32_t n = ws.lnv[ln];
        uint4 v = reinterpret_cast<const uint4*>(ws.tb + ln * 32)[c ^ (ln & 7u)];
        v.x += kk;
        v.y += kk;
        v.z += kk;
        v.w += kk;
        uint32_t* o = a.out_pool + ws.lout[ln] + 4 * c;
        if (4 * c + 4 <= n && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
          *reinterpret_cast<uint4*>(o) = v;
        } else {
          if (4 * c < n) o[0] = v.x;
          if (4 * c + 1 < n) o[1] = v.y;
          if (4 * c + 2 < n) o[2] = v.z;
          if (4 * c + 3 < n) o[3] = v.w;
        }
      }
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------- staging warp

// What staging a claimed record takes, found when its claim arrives: its
// 32-int lines, data vectors, control window and (Group-PFD) exception
// window; a record that fails its checks stages nothing and decodes to
// nothing (its error is reported here).
template <int KIND, int K>
__device__ __forceinline__ void stage_sizes(const gc_work& w, const DecodeArgs& a, uint32_t& lines, uint32_t& nv,
                                            uint32_t& cb, uint32_t& xb) {
  lines = 0;
  nv = 0;
  cb = 0;
  xb = 0;
  const bool live = w_live<K>(w, a);
  if (!live && w.list != 0xffffffffu)
    report(a.status, w.out_at + w_nint(w.shape) > a.out_pool_len ? GC_ERR_INVALID : GC_ERR_CORRUPT, w.list);
  if (!live) return;
  lines = (w_nint(w.shape) + 31) / 32;
  nv = w_vecs(w.shape);
  const int64_t ws0 = (int64_t)w.ctrl_at + w.win_at;
  cb = w.win_len < kCtrlCap ? w.win_len : (uint32_t)kCtrlCap;
  if (ws0 < 0 || (ws0 & 15) || (uint64_t)ws0 + cb > a.ctrl_pool_bytes) cb = 0;
  if (KIND == GC_PFD) {
    const uint64_t xs = (w.ctrl_at + w.exc_at) & ~15ull;
    xb = w.exc_len;
    if (xb > (uint32_t)kExcCap || xs + xb > a.ctrl_pool_bytes) xb = 0;
  }
}

// The staging warp's side of the ring: the bytes it holds (padding
// included), where the next pack goes, and the packs issued and given back.
struct Ring {
  uint32_t bytes, head, used;
  uint32_t issued, tail;     // packs issued / given back
  uint32_t ps;               // slot of the next pack
  uint32_t ts, tph;          // slot and phase of the oldest pack not given back
};

// Wait until the oldest pack not given back is decoded, and take its bytes
// back. False (every lane) when the wait runs out.
__device__ __forceinline__ void ring_take(BlockSmem& h, Ring& r, uint32_t S) {
  r.used -= h.prel[r.ts];
  ++r.tail;
  if (++r.ts == S) {
    r.ts = 0;
    r.tph ^= 1u;
  }
}
// (and every later pack that is decoded already, without waiting)
__device__ __forceinline__ bool ring_drain(BlockSmem& h, Ring& r, uint32_t S) {
  if (!wait_warp(&h.empty[r.ts], r.tph)) return false;
  ring_take(h, r, S);
  while (r.tail < r.issued && __all_sync(kFull, mbar_test_wait(&h.empty[r.ts], r.tph))) ring_take(h, r, S);
  return true;
}

// Claim up to `claim` records for record buffer b and start the bulk copy
// that brings them in; returns their first plan index and count (x, y;
// lane-uniform).
__device__ __noinline__ uint2 claim_records(const DecodeArgs& a, BlockSmem& h, uint32_t b, uint32_t claim,
                                            uint64_t total) {
  const uint32_t lane = lane_id();
  uint32_t v = 0;
  if (lane == 0) v = atomicAdd(a.counter, claim);
  const uint32_t x = __shfl_sync(kFull, v, 0);
  const uint32_t cnt = (uint64_t)x < total ? (uint32_t)min64(claim, total - x) : 0u;
  if (lane == 0 && cnt) {
    mbar_expect_tx(&h.recbar[b], cnt * (uint32_t)sizeof(gc_work));
    bulk_g2s(h.rec[b * kChunk], a.work + x, cnt * (uint32_t)sizeof(gc_work), &h.recbar[b]);
  }
  return make_uint2(x, cnt);
}

// A plan with look-back records: the block's c-th claim is records
// blockIdx.x + gridDim.x * (32 c + j), j = 0 .. 31 (the blocks take the
// records in turn, so a tile's predecessor is decoded by the block before,
// at about the same time), loaded by the lanes into record buffer b.
// Returns the claim's first record and count (x, y; lane-uniform).
__device__ __noinline__ uint2 claim_strided(const DecodeArgs& a, BlockSmem& h, uint32_t b, uint32_t c,
                                            uint64_t total) {
  const uint32_t lane = lane_id();
  const uint64_t r = blockIdx.x + (uint64_t)gridDim.x * (32ull * c + lane);
  const bool valid = r < total;
  if (valid) {
    const uint4* src = reinterpret_cast<const uint4*>(a.work + r);
    uint4* dst = h.rec[b * kChunk + lane];
    const uint4 q0 = src[0], q1 = src[1], q2 = src[2], q3 = src[3];
    dst[0] = q0;
    dst[1] = q1;
    dst[2] = q2;
    dst[3] = q3;
  }
  __syncwarp();
  const uint32_t cnt = __popc(__ballot_sync(kFull, valid));
  return make_uint2((uint32_t)(blockIdx.x + (uint64_t)gridDim.x * 32ull * c), cnt);
}

// Group the claim's records (lanes 0 .. cnt - 1) into packs: a pack is a run
// of consecutive records whose lines fit 32, whose ring bytes fit kPackCap
// and, at k = 4, whose data vectors fit the re-lay buffer; packs are formed
// greedily from the first record (a whole tile is a pack by itself). Lane i
// finds by binary search how many records from i on fit one pack (next_i
// is the first record after them); the packs start at the records reached
// from record 0 by following next, found by pointer doubling in five
// rounds. v packs (lines | ring bytes / 16 << 11 | vectors << 32, the
// vectors only at k = 4, whose sums then need 64 bits); returns the mask of
// pack starts, P is each lane's inclusive sum of v and nxt its next_i.
template <int K, class U>
__device__ __forceinline__ uint32_t pack_starts(U v, uint32_t cnt, U& P, uint32_t& nxt) {
  const uint32_t lane = lane_id();
  P = warp_incl_sum(v);
  const U Pex = P - v;
  uint32_t len = 0;
#pragma unroll
  for (uint32_t step = 16; step; step >>= 1) {
    const uint32_t j = lane + len + step - 1;  // the last record of the candidate
    const U s = __shfl_sync(kFull, P, j < 32 ? j : 31u) - Pex;
    bool fits = j < cnt && (uint32_t)(s & 2047u) <= 32u && (uint32_t)((s >> 11) & 0x1fffffu) * 16u <= (uint32_t)kPackCap;
    if constexpr (K == 4) fits = fits && (uint64_t)(s >> 32) <= (uint64_t)kPadVec4;
    if (fits) len += step;
  }
  nxt = lane < cnt ? lane + (len ? len : 1u) : 32u;
  uint32_t g = nxt, reach = cnt ? 1u : 0u;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    reach |= __reduce_or_sync(kFull, ((reach >> lane) & 1u) && g < 32u ? 1u << g : 0u);
    const uint32_t gg = __shfl_sync(kFull, g, g & 31u);
    g = g < 32u ? gg : 32u;
  }
  // (the last pack's next is record cnt, which is not the claim's)
  return cnt >= 32u ? reach : reach & ((1u << cnt) - 1u);
}

// The staging warp. Claims records (the next claim's copy in flight while
// the current one is placed), sizes them one per lane, groups them into
// packs (pack_starts) and places the packs in the ring in order, as many at
// once as the ring and the pack slots allow: a pack never wraps (one that
// would cross the ring's end starts at 0, and the bytes it skips are held
// with it), and the ring's bytes come back in pack order as the decoding
// warps finish. Each placed pack's records get their ring offsets and the
// pack its slot descriptor, then one arrival on the slot's mbarrier tells
// its decoding warp, which copies the pack's bytes in itself. After the
// last record, one empty pack per decoding warp tells it to stop.
template <int KIND, int K>
__device__ void produce(const DecodeArgs& a, BlockSmem& h, uint32_t W, uint32_t S) {
  const uint32_t lane = lane_id();
  uint64_t total = a.count[0];
  if (total > a.work_cap) total = a.work_cap;
  // With tiles that take their prefix by look-back, the blocks take the
  // records in turn (claim_strided) and a claim is made only once the one
  // before is placed: a tile's predecessor is then decoded by another block
  // at about the same time, so a decoding warp seldom waits for it.
  const bool ahead = a.count[1] == 0;
  const uint32_t claim = a.claim < 1u ? 1u : a.claim > (uint32_t)kChunk ? (uint32_t)kChunk : a.claim;
  const uint32_t stride = ahead ? 1u : gridDim.x;  // between the records of a claim
  Ring r = {a.ring_bytes, 0, 0, 0, 0, 0, 0, 0};
  bool failed = false;
  uint32_t busy = 0;  // lane b < kNChunk: record buffer b is free once this many packs are given back
  const uint2 c0 = ahead ? claim_records(a, h, 0, claim, total) : claim_strided(a, h, 0, 0, total);
  uint32_t x = c0.x, cnt = c0.y;
  for (uint32_t c = 0; cnt && !failed; ++c) {
    const uint32_t b = c % kNChunk;
    // the next claim goes to the next buffer once that buffer's packs are given back
    const uint32_t nb = (c + 1) % kNChunk;
    uint32_t nx = 0, ncnt = 0;
    if (ahead) {
      const uint32_t nbusy = __shfl_sync(kFull, busy, nb);
      while (!failed && r.tail < nbusy) failed = !ring_drain(h, r, S);
      if (failed) break;
      const uint2 cn = claim_records(a, h, nb, claim, total);
      nx = cn.x;
      ncnt = cn.y;
    }
    if (ahead && !wait_warp(&h.recbar[b], (c / kNChunk) & 1u)) {
      failed = true;
      break;
    }
    // sizes, one record per lane
    const bool valid = lane < cnt;
    const uint32_t rs = b * kChunk + lane;
    uint32_t lines = 0, nv = 0, cb = 0, xb = 0;
    if (valid) {
      h.item[rs] = x + lane * stride;
      stage_sizes<KIND, K>(rec_of(h, rs), a, lines, nv, cb, xb);
      h.fvecs[rs] = (uint16_t)nv;
      h.cst[rs] = (uint16_t)cb;
      h.xst[rs] = (uint16_t)xb;
      h.flines[rs] = (uint8_t)lines;
    }
    const uint32_t need16 = (nv * (uint32_t)Geo<K>::VB + cb + xb) / 16;  // ring bytes / 16
    using U = typename std::conditional<K == 4, uint64_t, uint32_t>::type;
    const U v = valid ? (U)lines | (U)need16 << 11 | (K == 4 ? (U)((uint64_t)nv << 32) : (U)0) : (U)0;
    U P;
    uint32_t nxt;
    const uint32_t starts = pack_starts<K, U>(v, cnt, P, nxt);
    const U Pex = P - v;
    // each record's offset from its pack's start; at a pack's first record,
    // the pack's ring bytes / 16, records and lines
    const uint32_t le = 0xffffffffu >> (31u - lane);  // lanes <= this one
    const uint32_t s0 = (31u - __clz(starts & le)) & 31u;
    const uint32_t ex16 = (uint32_t)((Pex >> 11) & 0x1fffffu);  // ring bytes / 16 before this record
    const uint32_t sex16 = __shfl_sync(kFull, ex16, s0);
    if (valid) h.rrel[rs] = (ex16 - sex16) * 16;
    const U Pl = __shfl_sync(kFull, P, (nxt - 1u) & 31u);
    const uint32_t pinfo = ((uint32_t)((Pl >> 11) & 0x1fffffu) - ex16) | (nxt - lane) << 16 |
                           ((uint32_t)(Pl & 2047u) - (uint32_t)(Pex & 2047u)) << 24;
    __threadfence_block();
    __syncwarp();
    // place the packs in order
    for (uint32_t m = starts; m && !failed; m &= m - 1) {
      const uint32_t sp = __ffs(m) - 1;
      const uint32_t pi = __shfl_sync(kFull, pinfo, sp);
      const uint32_t B = (pi & 0xffffu) * 16;
      uint32_t off, pad;
      for (;;) {
        if (r.used == 0) r.head = 0;
        off = r.head;
        pad = 0;
        if (off + B > r.bytes) {
          pad = r.bytes - off;
          off = 0;
        }
        if (r.used + pad + B <= r.bytes && r.issued - r.tail < S) break;
        if (!ring_drain(h, r, S)) {
          failed = true;
          break;
        }
      }
      if (failed) break;
      if (lane == 0) {
        h.pk[r.ps] = (b * kChunk + sp) | ((pi >> 16) & 255u) << 8 | (pi >> 24) << 16;
        h.prel[r.ps] = pad + B;
        h.ppos[r.ps] = off;
        mbar_arrive(&h.full[r.ps]);
      }
      r.head = off + B;
      r.used += pad + B;
      ++r.issued;
      if (++r.ps == S) r.ps = 0;
    }
    if (lane == b) busy = r.issued;
    if (!ahead && !failed) {
      const uint32_t nbusy = __shfl_sync(kFull, busy, nb);
      while (!failed && r.tail < nbusy) failed = !ring_drain(h, r, S);
      if (failed) break;
      const uint2 cn = claim_strided(a, h, nb, c + 1, total);
      nx = cn.x;
      ncnt = cn.y;
    }
    x = nx;
    cnt = ncnt;
  }
  if (failed) {
    if (lane == 0) report(a.status, GC_ERR_TIMEOUT, 0xfffffffdu);
    return;
  }
  // one stop per decoding warp
  while (r.issued + W - r.tail > S) {
    if (!ring_drain(h, r, S)) {
      if (lane == 0) report(a.status, GC_ERR_TIMEOUT, 0xfffffffdu);
      return;
    }
  }
  const uint32_t slot = (r.ps + lane) % S;
  if (lane < W) {
    h.pk[slot] = 0;
    h.prel[slot] = 0;
  }
  __threadfence_block();
  __syncwarp();
  if (lane < W) mbar_arrive(&h.full[slot]);
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// A decoding warp copies a pack's bytes into the ring (the places the
// staging warp gave its records), tile by tile: lane j takes 16-byte chunk
// j % C of data vectors j / C, j / C + 32 / C, ... (C chunks per vector,
// each vector at the ring's pitch), then chunks j, j + 32, ... of the
// tile's control window and exception window, which lie back to back after
// its vectors. Each lane's copies are its own cp.async group once
// committed.
template <int K>
__device__ __forceinline__ void copy_pack(const DecodeArgs& a, BlockSmem& h, uint8_t* ring, uint32_t d, uint32_t slot) {
  const uint32_t lane = lane_id();
  const uint32_t s0 = d & 255u, np = (d >> 8) & 255u;
  // the records' ring offsets: the pack's, plus each one's from the pack's start
  if (lane < np) {
    const uint32_t s = rslot(s0 + lane);
    h.at[s] = h.ppos[slot] + h.rrel[s];
  }
  __syncwarp();
  constexpr uint32_t CPV = K * 4 / 16;  // 16-byte chunks per data vector
  constexpr uint32_t VPS = 32 / CPV;    // vectors per step of the warp
  for (uint32_t p = 0; p < np; ++p) {
    const uint32_t s = rslot(s0 + p);
    const uint32_t nvp = h.fvecs[s], ch = (h.cst[s] + h.xst[s]) >> 4;
    const gc_work& w = rec_of(h, s);
    const uint32_t atp = h.at[s];
    uint32_t v = lane / CPV;
    const uint32_t c16 = 16 * (lane % CPV);
    uint8_t* dst = ring + atp + v * (uint32_t)Geo<K>::VB + c16;
    const uint8_t* src = reinterpret_cast<const uint8_t*>(a.data_pool + w.data_at) + (size_t)v * (K * 4) + c16;
#pragma unroll 1
    for (; v < nvp; v += VPS, dst += VPS * Geo<K>::VB, src += VPS * K * 4) cp_async16(dst, src);
    if (ch) {
      const uint32_t cch = h.cst[s] >> 4;
      const uint8_t* csrc = a.ctrl_pool + (w.ctrl_at + w.win_at);
      const uint8_t* xsrc = a.ctrl_pool + ((w.ctrl_at + w.exc_at) & ~15ull) - 16ull * cch;
      uint8_t* cdst = ring + atp + nvp * (uint32_t)Geo<K>::VB;
#pragma unroll 1
      for (uint32_t j = lane; j < ch; j += 32) cp_async16(cdst + 16 * j, (j < cch ? csrc : xsrc) + 16 * j);
    }
  }
}

// A decoding warp: packs w, w + W, w + 2W, ... (slot w + (t mod S/W) W of
// the block's S = W * (kMaxSlots / W) slots), until an empty one. It copies
// the next pack in while it decodes the current one when the staging warp
// has placed it already; it never waits for the next pack before decoding
// the current one (the staging warp may need the current pack's ring bytes
// back first).
template <int KIND, int K, bool RESTORE, bool PER>
__device__ void consume(const DecodeArgs& a, BlockSmem& h, WarpSmem<K>& ws, uint8_t* ring, uint32_t w,
                        uint32_t W, uint32_t S) {
  const uint32_t lane = lane_id();
  // row entries start in range (a parser stopped by a corrupt stream leaves
  // earlier, in-range entries behind, never garbage)
  for (uint32_t i = lane; i < (uint32_t)Geo<K>::PROWS; i += 32) {
    ws.rw[i] = 0;
    ws.rs[i] = 0;
  }
  ws.irec[lane] = 0;
  __syncwarp();
  uint32_t slot = w, par = 0;
  if (!wait_warp(&h.full[slot], par)) {
    if (lane == 0) report(a.status, GC_ERR_TIMEOUT, 0xfffffffeu);
    return;
  }
  uint32_t d = h.pk[slot];
  if (((d >> 8) & 255u) == 0) return;
  copy_pack<K>(a, h, ring, d, slot);
  cp_async_commit();
  for (;;) {
    uint32_t nslot = slot + W, npar = par;
    if (nslot >= S) {
      nslot -= S;
      npar ^= 1u;
    }
    // the next pack's copies, when it is placed already
    const bool pre = __all_sync(kFull, mbar_test_wait(&h.full[nslot], npar));
    uint32_t nd = 0;
    if (pre) {
      nd = h.pk[nslot];
      if ((nd >> 8) & 255u) copy_pack<K>(a, h, ring, nd, nslot);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const uint32_t s0 = d & 255u, np = (d >> 8) & 255u;
    if constexpr (PER) {
      // GC_WORK_RAW records' lines decode without the prefix sum
      const uint32_t nl = d >> 16;
      if constexpr (K == 32) decode_pack32<KIND, true, true>(a, h, ws, ring, s0, np, nl, &h.empty[slot]);
      else decode_pack4<KIND, true, true>(a, h, ws, ring, s0, np, nl, &h.empty[slot]);
    } else {
      const uint32_t nl = d >> 16;
      if constexpr (K == 32) decode_pack32<KIND, RESTORE>(a, h, ws, ring, s0, np, nl, &h.empty[slot]);
      else decode_pack4<KIND, RESTORE>(a, h, ws, ring, s0, np, nl, &h.empty[slot]);
    }
    slot = nslot;
    par = npar;
    if (!pre) {
      if (!wait_warp(&h.full[slot], par)) {
        if (lane == 0) report(a.status, GC_ERR_TIMEOUT, 0xfffffffeu);
        break;
      }
      nd = h.pk[slot];
      if ((nd >> 8) & 255u) {
        copy_pack<K>(a, h, ring, nd, slot);
        cp_async_commit();
      }
    }
    if (((nd >> 8) & 255u) == 0) break;
    d = nd;
  }
  cp_async_wait<0>();
}

// The persistent decoder: warp 0 stages, warps 1 .. W decode. Dynamic
// shared memory: BlockSmem, W WarpSmem<K>, then the ring (a.ring_bytes).
template <int KIND, int K, bool RESTORE, bool PER>
__global__ void __launch_bounds__(Geo<K>::THREADS, 1) k_decode(DecodeArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  BlockSmem& h = *reinterpret_cast<BlockSmem*>(smem_raw);
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t W = (blockDim.x >> 5) - 1;
  const uint32_t S = (kMaxSlots / W) * W;
  WarpSmem<K>* ws = reinterpret_cast<WarpSmem<K>*>(smem_raw + sizeof(BlockSmem));
  uint8_t* ring = smem_raw + sizeof(BlockSmem) + W * sizeof(WarpSmem<K>);
  if (warp == 0) {
    for (uint32_t i = lane; i < S; i += 32) {
      mbar_init(&h.full[i], 1);
      mbar_init(&h.empty[i], 1);
    }
    if (lane < kNChunk) mbar_init(&h.recbar[lane], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (warp == 0) produce<KIND, K>(a, h, W, S);
  else consume<KIND, K, RESTORE, PER>(a, h, ws[warp - 1], ring, warp - 1, W, S);
}

// --------------------------------------------------------------- the plan

struct PlanArgs {
  uint32_t kind, k, cg, ld;
  const gc_list* lists;  // NULL: the single list `one`
  gc_list one;
  uint64_t nlists;       // lists planned (the selection's length when sel is set)
  const uint32_t* sel;   // optional: plan lists[sel[i]] for i < nlists ...
  const uint64_t* outs;  // ... with their ints at outs[i] of the output pool
  uint64_t nall;         // lists in `lists` (bounds the selection)
  const gc_tile* tiles;  // batch: tile t >= 1 of a list at tile_off + t - 1; single: tile t at t
  uint64_t ntiles;
  const uint8_t* ctrl_pool;
  uint64_t ctrl_pool_bytes;
  gc_work* work;
  uint64_t cap;
  unsigned long long* count;  // [0] records, [1] records needing look-back
  uint32_t* status;
  uint32_t pairs;             // interleaved plan: entries 2i (docIDs) and 2i + 1 (raw) tile by tile
};

// The descriptor of planned list i (a selected list takes its output offset
// from the selection); a selection index out of range gives an empty list.
__device__ __forceinline__ gc_list plan_list(const PlanArgs& a, uint64_t i) {
  if (!a.lists) return a.one;
  if (!a.sel) return a.lists[i];
  const uint32_t li = a.sel[i];
  if (li >= a.nall) return gc_list{0, 0, 0, 0, 0, 0, 0};
  gc_list d = a.lists[li];
  d.out_off = a.outs[i];
  return d;
}

// Pass 1: one thread per list reserves a contiguous range of records for the
// list's tiles (one atomic per warp); then the warp writes (list, tile) into
// the records of its lists, one list after another, 32 records per step. A
// list's tiles are consecutive records. (A single list needs no writes: pass
// 2 knows record i is its tile i.)
__global__ void k_plan_reserve(PlanArgs a) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = lane_id();
  // an interleaved plan reserves per pair of entries (2i, 2i + 1), two
  // records per tile
  const uint64_t units = a.pairs ? a.nlists / 2 : a.nlists;
  const uint32_t per = a.pairs ? 2u : 1u;
  uint64_t nt = 0;
  if (i < units) {
    const uint64_t n = plan_list(a, per * i).n;
    const uint64_t R = (n + a.k - 1) / a.k;
    const uint64_t tr = kTileInts / a.k;
    nt = per * ((R + tr - 1) / tr);
    if (a.pairs && plan_list(a, per * i + 1).n != n) {
      report(a.status, GC_ERR_INVALID, (uint32_t)i);
      nt = 0;
    }
  }
  const uint64_t incl = warp_incl_sum(nt);
  unsigned long long b = 0;
  if (lane == 31) b = atomicAdd(a.count, (unsigned long long)incl);
  const uint64_t base = __shfl_sync(kFull, b, 31) + incl - nt;
  const bool fits = base + nt <= a.cap;
  if (i < units && !fits) report(a.status, GC_ERR_NOSPACE, (uint32_t)i);
  if (!a.lists) return;
  for (uint32_t m = __ballot_sync(kFull, i < units && nt > 0); m; m &= m - 1) {
    const uint32_t src = __ffs(m) - 1;
    const uint64_t lb0 = __shfl_sync(kFull, base, src);
    const uint64_t ln = __shfl_sync(kFull, nt, src);
    const uint32_t lid = __shfl_sync(kFull, (uint32_t)i, src);
    const bool lf = __shfl_sync(kFull, fits, src);
    for (uint64_t t = lane; t < ln && lb0 + t < a.cap; t += 32) {
      gc_work* w = a.work + lb0 + t;
      w->tile = (uint32_t)(t / per);
      w->list = lf ? per * lid + (uint32_t)(t % per) : 0xffffffffu;
    }
  }
}

__device__ __forceinline__ bool plan_tile(const PlanArgs& a, const gc_list& d, uint64_t t, gc_tile* r) {
  if (t == 0) {
    *r = gc_tile{0, 0, 0, 0, 0, GC_TILE_BASE};
    return true;
  }
  const uint64_t ti = a.lists ? (uint64_t)d.tile_off + t - 1 : t;
  if (!a.tiles || ti >= a.ntiles) return false;
  *r = a.tiles[ti];
  return true;
}

__device__ __forceinline__ uint64_t al16(uint64_t x) { return x & ~15ull; }

// Pass 2: one thread per record fills in the list's areas, the tile's first
// unit and skip entry, and the exact ranges of the tile's streams: data
// vectors from the unit's first word to the word holding the tile's last
// row (the next tile's first unit, plus the part of it before that tile
// when the unit straddles the two); control bytes per codec.
__global__ void k_plan_fill(PlanArgs a) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t total = a.count[0];
  if (total > a.cap) total = a.cap;
  if (i >= total) return;
  const gc_work empty = {0, 0, 0, 0, 0, 0, 0xffffffffu, 0, 0, 0, 0, 0, 0};
  gc_work w = empty;
  if (a.lists) {
    w = a.work[i];
  } else if (a.count[0] <= a.cap) {  // (a single list that does not fit is not planned)
    w.tile = (uint32_t)i;
    w.list = 0;
  }
  if (w.list == 0xffffffffu || w.list >= a.nlists) {
    a.work[i] = empty;
    return;
  }
  const gc_list d = plan_list(a, w.list);
  const uint64_t k = a.k, TR = kTileInts / k;
  const uint64_t t = w.tile;
  const uint64_t n = d.n;
  const uint64_t R = (n + k - 1) / k;
  const uint64_t nt = (R + TR - 1) / TR;
  const uint64_t row0 = t * TR;
  const uint64_t rows = min64(TR, R - row0);
  gc_tile r0, r1;
  const bool last = t + 1 >= nt;
  bool ok = plan_tile(a, d, t, &r0);
  if (!last) ok = ok && plan_tile(a, d, t + 1, &r1);
  const uint64_t cbytes = d.ctrl_bytes;
  // data vectors, from the word that holds the tile's first row (a Group-AFOR
  // frame may start rows before the tile)
  uint64_t first_bit = r0.lane_bit;
  if (a.kind == GC_AFOR && r0.row_skip) {
    const uint64_t fb = r0.ctrl_bit >> 3;
    const uint64_t at = d.ctrl_off + fb;
    const uint32_t byte = (fb < cbytes && at < a.ctrl_pool_bytes) ? a.ctrl_pool[at] : 0xffu;
    first_bit += (uint64_t)r0.row_skip * ((byte & 63u) <= 32 ? (byte & 63u) : 32u);
  }
  const uint64_t v0 = first_bit >> 5;
  uint64_t v1 = d.data_words / k;
  if (!last) {
    uint64_t straddle = 0;
    if (r1.row_skip) {
      if (a.kind == GC_SIMPLE) {
        straddle = 32;
      } else if (a.kind == GC_AFOR) {
        const uint64_t fb = r1.ctrl_bit >> 3;
        const uint64_t at = d.ctrl_off + fb;
        const uint32_t byte = (fb < cbytes && at < a.ctrl_pool_bytes) ? a.ctrl_pool[at] : 0xffu;
        straddle = (uint64_t)r1.row_skip * ((byte & 63u) <= 32 ? (byte & 63u) : 32u);
      } else {
        straddle = 32ull * r1.row_skip;
      }
    }
    const uint64_t e = r1.lane_bit + straddle;
    v1 = min64((e + 31) >> 5, v1);
  }
  if (v1 < v0 || v1 - v0 > TR + 1 || (d.data_off % k) != 0) ok = false;
  // control bytes [cs, ce) of the tile (and the PFD exception records)
  uint64_t cs = 0, ce = cbytes, xs = 0, xe = 0;
  const uint64_t nf = (R + kPfdFrameRows - 1) / kPfdFrameRows;
  switch (a.kind) {
    case GC_SIMPLE:
      cs = r0.ctrl_bit >> 3;
      if (!last) ce = (r1.ctrl_bit >> 3) + 1;
      break;
    case GC_SCHEME:
      if (a.ld == GC_LD_BINARY) {
        cs = bin_ld_pos(row0, a.cg) >> 3;
        ce = bin_ld_bytes(row0 + rows, a.cg);
      } else {
        cs = r0.ctrl_bit >> 3;
        if (!last) ce = (r1.ctrl_bit + 7) >> 3;
      }
      break;
    case GC_AFOR:
      cs = r0.ctrl_bit >> 3;
      if (!last) ce = (r1.ctrl_bit >> 3) + 1;
      break;
    default:
      cs = 4 * (row0 / kPfdFrameRows);
      ce = 4 * ((row0 + rows + kPfdFrameRows - 1) / kPfdFrameRows);
      xs = 4 * nf + r0.exc_off;
      xe = last ? cbytes : 4 * nf + r1.exc_off;
      break;
  }
  ce = min64(ce, cbytes);
  if (cs > ce) ok = false;
  const uint64_t pool_end = al16(a.ctrl_pool_bytes);
  const uint64_t wlo = al16(d.ctrl_off + cs);
  uint64_t whi = min64(al16(d.ctrl_off + ce + 15), pool_end);
  if (whi < wlo) whi = wlo;
  uint64_t xlen = 0;
  if (a.kind == GC_PFD && xe > xs) {
    const uint64_t xlo = al16(d.ctrl_off + xs);
    const uint64_t xhi = al16(d.ctrl_off + xe + 15);
    xlen = xhi <= pool_end ? xhi - xlo : 0;  // all of the tile's records, or none
    if (xlen > 0xfff0) xlen = 0;
  }
  if (xe < xs || xe > cbytes) ok = false;
  if (d.ctrl_off + cbytes > a.ctrl_pool_bytes) ok = false;
  if (!ok) {
    report(a.status, GC_ERR_CORRUPT, w.list);
    a.work[i] = empty;
    return;
  }
  // an interleaved plan: odd entries are written raw (with base 0: their
  // lines' totals count 0); an even entry's tiles are not consecutive
  // records, so each one after the first needs its base
  const bool raw = a.pairs && (w.list & 1u);
  const bool has_base = raw || (r0.flags & GC_TILE_BASE) != 0;
  const bool publish = !a.pairs && !last && !(r1.flags & GC_TILE_BASE);
  if (a.pairs && !raw && t > 0 && !has_base) {
    report(a.status, GC_ERR_UNSUPPORTED, a.sel ? a.sel[w.list] : w.list);
    a.work[i] = empty;
    return;
  }
  if (!raw && t > 0 && !has_base) {
    // warp-aggregated count of records that take their prefix by look-back
    atomicAdd(a.count + 1, 1ull);
  }
  const uint32_t nint = (uint32_t)min64(kTileInts, n - t * kTileInts);
  w.ctrl_at = d.ctrl_off;
  w.data_at = d.data_off + v0 * k;
  w.out_at = d.out_off + t * kTileInts;
  w.ctrl_bit = r0.ctrl_bit;
  w.ctrl_bytes = (uint32_t)cbytes;
  w.base = has_base && !raw ? r0.base : 0;
  w.exc_at = (uint32_t)xs;
  w.win_at = (int32_t)((int64_t)wlo - (int64_t)d.ctrl_off);
  w.win_len = (uint16_t)min64(whi - wlo, 0xfff0);
  w.exc_len = (uint16_t)xlen;
  if (a.sel) w.list = a.sel[w.list];  // records name the index's list
  w.shape = (nint - 1) | ((uint32_t)(v1 - v0) << GC_WORK_VEC_SHIFT) | ((uint32_t)(first_bit & 31) << GC_WORK_BIT_SHIFT) |
            ((r0.row_skip & 31u) << GC_WORK_SKIP_SHIFT) | (has_base ? (uint32_t)GC_WORK_HAS_BASE : 0u) |
            (publish ? (uint32_t)GC_WORK_PUBLISH : 0u) | (raw ? (uint32_t)GC_WORK_RAW : 0u);
  a.work[i] = w;
}

// The counts of a plan copied in from the host: [0] its records, [1] the
// records that take their prefix by look-back (count zeroed before).
__global__ void k_count_records(const gc_work* work, uint64_t nwork, unsigned long long* count) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) count[0] = nwork;
  bool lb = false;
  if (i < nwork) {
    const gc_work& w = work[i];
    lb = w.list != 0xffffffffu && w.tile > 0 && !(w.shape & GC_WORK_HAS_BASE);
  }
  const uint32_t m = __ballot_sync(kFull, lb);
  if (m && lane_id() == (uint32_t)(__ffs(m) - 1)) atomicAdd(count + 1, (unsigned long long)__popc(m));
}

}  // namespace gcdev

// ====================================================================== host

using namespace gcdev;

namespace {

constexpr uint32_t kMaxClaim = kChunk;  // records per claim
constexpr uint64_t kHdr = 256;           // scratch header: claim counter, record counts
// plans the 32-bit claim counter serves: every block may claim twice past
// the end, with up to 8 blocks on each of up to 512 SMs
constexpr uint64_t kMaxWork = 0xffffffffull - 2ull * kMaxClaim * 8 * 512;

// A launch shape of the persistent decoder: decoding warps per block (plus
// the staging warp), blocks per SM, records per claim, ring bytes per block
// (0: all the shared memory the block's share of the SM leaves).
struct Shape {
  uint32_t warps, bps, claim, stage;
};

Shape default_shape(uint32_t k) { return k == 32 ? Shape{7, 3, kMaxClaim, 0} : Shape{7, 2, kMaxClaim, 0}; }

// Device facts the launches need, looked up once per device.
struct DevInfo {
  int optin = 0;      // shared memory a block may opt in to
  int per_sm = 0;     // shared memory of an SM
};

std::mutex g_launch_mu;
DevInfo g_dev[64];
uint32_t g_epoch = 1;  // advanced by gc_shutdown: per-kernel facts are looked up again

// Launch shapes registered with gc_set_launch: per device, codec kind, k
// (0: 4, 1: 32) and restore flag.
struct Registered {
  bool set = false;
  Shape sh = {};
};
Registered g_reg[64][4][2][2];

template <int KIND, int K, bool RESTORE, bool PER>
gc_status launch_t(DecodeArgs a, Shape sh, uint64_t work, cudaStream_t s) {
  auto fn = k_decode<KIND, K, RESTORE, PER>;
  // per device: the opted-in shared-memory size of this kernel (it only
  // grows) and the occupancy of the last shape asked for
  static size_t smem_set[64] = {};
  static uint32_t occ_key[64][2] = {};
  static int occ_val[64] = {};
  static uint32_t seen[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GC_ERR_CUDA;
  if (dev < 0 || dev >= 64) return GC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_launch_mu);
  if (seen[dev] != g_epoch) {
    smem_set[dev] = 0;
    occ_val[dev] = 0;
    seen[dev] = g_epoch;
  }
  DevInfo& di = g_dev[dev];
  if (di.optin == 0) {
    if (cudaDeviceGetAttribute(&di.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&di.per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
      return GC_ERR_CUDA;
  }
  const uint32_t max_warps = Geo<K>::THREADS / 32 - 1;
  const uint32_t W = sh.warps < 1 ? 1u : sh.warps > max_warps ? max_warps : sh.warps;
  const uint32_t bps = sh.bps ? sh.bps : default_shape(K).bps;
  // the block's share of the SM's shared memory (1 KB of it is reserved per block)
  int64_t budget = (int64_t)di.per_sm / bps - 1024;
  if (budget > di.optin) budget = di.optin;
  const int64_t fixed = (int64_t)sizeof(BlockSmem) + (int64_t)W * sizeof(WarpSmem<K>);
  int64_t ring = (budget - fixed) & ~127ll;
  if (sh.stage && (int64_t)sh.stage < ring) ring = (int64_t)sh.stage & ~127ll;
  if (ring < kPackCap) return GC_ERR_INVALID;  // the shape leaves no room for a pack
  const size_t smem = (size_t)(fixed + ring);
  if (smem > smem_set[dev]) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return GC_ERR_CUDA;
    smem_set[dev] = smem;
  }
  const uint32_t threads = 32 * (W + 1);
  if (occ_key[dev][0] != threads || occ_key[dev][1] != (uint32_t)smem || occ_val[dev] == 0) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, (int)threads, smem) != cudaSuccess) return GC_ERR_CUDA;
    if (occ < 1) return GC_ERR_INVALID;
    occ_key[dev][0] = threads;
    occ_key[dev][1] = (uint32_t)smem;
    occ_val[dev] = occ;
  }
  const uint32_t fit = bps < (uint32_t)occ_val[dev] ? bps : (uint32_t)occ_val[dev];
  uint64_t grid = (uint64_t)fit * gc_host::sm_count();
  a.claim = sh.claim < 1 ? 1u : sh.claim > kMaxClaim ? kMaxClaim : sh.claim;
  a.ring_bytes = (uint32_t)ring;
  const uint64_t chunks = (work + a.claim - 1) / a.claim;  // at least one claim per block
  if (grid > chunks) grid = chunks ? chunks : 1;
  fn<<<(unsigned)grid, threads, smem, s>>>(a);
  gc_host::count_launch();
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

template <bool RESTORE, bool PER>
gc_status launch_r(uint32_t kind, uint32_t k, const DecodeArgs& a, Shape sh, uint64_t work, cudaStream_t s) {
#define GC_DISPATCH(KIND)                                                 \
  if (kind == KIND) {                                                      \
    if (k == 4) return launch_t<KIND, 4, RESTORE, PER>(a, sh, work, s);    \
    return launch_t<KIND, 32, RESTORE, PER>(a, sh, work, s);               \
  }
  GC_DISPATCH(GC_SIMPLE)
  GC_DISPATCH(GC_SCHEME)
  GC_DISPATCH(GC_AFOR)
  GC_DISPATCH(GC_PFD)
#undef GC_DISPATCH
  return GC_ERR_INVALID;
}

// restore: 0 values, 1 docIDs, GC_RESTORE_PER_RECORD docIDs except GC_WORK_RAW records
gc_status launch_decode(uint32_t kind, uint32_t k, int restore, const DecodeArgs& a, Shape sh, uint64_t work,
                        cudaStream_t s) {
  if (restore == GC_RESTORE_PER_RECORD) return launch_r<true, true>(kind, k, a, sh, work, s);
  return restore ? launch_r<true, false>(kind, k, a, sh, work, s) : launch_r<false, false>(kind, k, a, sh, work, s);
}

// A caller's shape over the library default for this k (every field 0 =
// its default); GC_ERR_INVALID for a shape out of range.
gc_status fill_shape(const gc_codec& c, const gc_launch& l, Shape* sh) {
  *sh = default_shape(c.k);
  const uint32_t max_warps = (c.k == 32 ? Geo<32>::THREADS : Geo<4>::THREADS) / 32 - 1;
  if (l.warps_per_block > max_warps || l.items_per_claim > kMaxClaim || l.blocks_per_sm > 8) return GC_ERR_INVALID;
  if (l.warps_per_block) sh->warps = l.warps_per_block;
  if (l.blocks_per_sm) sh->bps = l.blocks_per_sm;
  if (l.items_per_claim) sh->claim = l.items_per_claim;
  sh->stage = l.stage_bytes;
  return GC_OK;
}

Registered* registered(const gc_codec& c, int restore) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  return &g_reg[dev][c.kind & 3u][c.k == 32 ? 1 : 0][restore ? 1 : 0];
}

// Launch shape from the caller's request: NULL = the shape registered for
// this codec (gc_set_launch), else the library default for this k.
gc_status launch_shape(const gc_codec& c, const gc_launch* l, Shape* sh, int restore) {
  if (l) return fill_shape(c, *l, sh);
  *sh = default_shape(c.k);
  std::lock_guard<std::mutex> lock(g_launch_mu);
  const Registered* r = registered(c, restore);
  if (r && r->set) *sh = r->sh;
  return GC_OK;
}

gc_status plan_impl(const gc_codec& c, const gc_list* lists, const gc_list* one, uint64_t nlists,
                    const gc_tile* tiles, uint64_t ntiles, const uint8_t* ctrl_pool, uint64_t ctrl_pool_bytes,
                    gc_work* work, uint64_t cap, uint64_t* count, uint32_t* status, cudaStream_t s,
                    const uint32_t* sel = nullptr, const uint64_t* outs = nullptr, uint64_t nall = 0,
                    bool pairs = false) {
  if (cudaMemsetAsync(count, 0, 16, s) != cudaSuccess) return GC_ERR_CUDA;
  if (nlists == 0) return GC_OK;
  PlanArgs a = {};
  a.kind = c.kind;
  a.k = c.k;
  a.cg = c.cg;
  a.ld = c.ld;
  a.lists = lists;
  if (one) a.one = *one;
  a.nlists = nlists;
  a.sel = sel;
  a.outs = outs;
  a.nall = sel ? nall : nlists;
  a.tiles = tiles;
  a.ntiles = tiles ? ntiles : 0;
  a.ctrl_pool = ctrl_pool;
  a.ctrl_pool_bytes = ctrl_pool ? ctrl_pool_bytes : 0;
  a.work = work;
  a.cap = cap;
  a.count = reinterpret_cast<unsigned long long*>(count);
  a.status = status;
  a.pairs = pairs ? 1u : 0u;
  k_plan_reserve<<<(unsigned)((nlists + 255) / 256), 256, 0, s>>>(a);
  gc_host::count_launch();
  if (cap) {
    k_plan_fill<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(a);
    gc_host::count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

}  // namespace

gc_status gc_host::plan_fill(const gc_codec& c, const gc_list* d_lists, uint64_t nlists, const uint32_t* d_sel,
                             const uint64_t* d_outs, uint64_t nsel, const gc_tile* d_tiles, uint64_t ntiles,
                             const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes, gc_work* d_work, uint64_t cap,
                             uint64_t* d_count, uint32_t* d_status, cudaStream_t s) {
  if (cap == 0) return GC_OK;
  PlanArgs a = {};
  a.kind = c.kind;
  a.k = c.k;
  a.cg = c.cg;
  a.ld = c.ld;
  a.lists = d_lists;
  a.nlists = nsel;
  a.sel = d_sel;
  a.outs = d_outs;
  a.nall = nlists;
  a.tiles = d_tiles;
  a.ntiles = d_tiles ? ntiles : 0;
  a.ctrl_pool = d_ctrl_pool;
  a.ctrl_pool_bytes = d_ctrl_pool ? ctrl_pool_bytes : 0;
  a.work = d_work;
  a.cap = cap;
  a.count = reinterpret_cast<unsigned long long*>(d_count);
  a.status = d_status;
  k_plan_fill<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(a);
  gc_host::count_launch();
  return cudaGetLastError() == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

namespace {

gc_status decode_plan_impl(const gc_codec& c, const gc_work* work, const uint64_t* count, uint64_t work_cap,
                           const uint8_t* ctrl_pool, uint64_t ctrl_pool_bytes, const uint32_t* data_pool,
                           uint64_t data_pool_words, uint32_t* out_pool, uint64_t out_pool_len, int restore,
                           Shape sh, unsigned char* scratch, uint32_t* status, cudaStream_t s) {
  uint32_t* counter = reinterpret_cast<uint32_t*>(scratch);
  unsigned long long* lb = reinterpret_cast<unsigned long long*>(scratch + kHdr);
  if (cudaMemsetAsync(scratch, 0, 64, s) != cudaSuccess) return GC_ERR_CUDA;
  if (restore && cudaMemsetAsync(lb, 0, work_cap * 8, s) != cudaSuccess) return GC_ERR_CUDA;
  DecodeArgs a = {};
  a.work = work;
  a.count = reinterpret_cast<const unsigned long long*>(count);
  a.work_cap = work_cap;
  a.ctrl_pool = ctrl_pool;
  a.ctrl_pool_bytes = ctrl_pool_bytes;
  a.data_pool = data_pool;
  a.data_pool_words = data_pool_words;
  a.out_pool = out_pool;
  a.out_pool_len = out_pool_len;
  a.counter = counter;
  a.lb = restore ? lb : nullptr;
  a.cg = c.cg;
  a.ld = c.ld;
  a.status = status;
  return launch_decode(c.kind, c.k, restore, a, sh, work_cap, s);
}

uint64_t tiles_of(const gc_codec& c, uint64_t n) {
  const uint64_t R = (n + c.k - 1) / c.k;
  const uint64_t tr = kTileInts / c.k;
  return (R + tr - 1) / tr;
}

}  // namespace

extern "C" {

gc_status gc_decode_scratch_size(const gc_codec* codec, uint64_t n, int have_tiles, uint64_t* bytes) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!bytes) return GC_ERR_INVALID;
  const uint64_t nt = tiles_of(*codec, n);
  // header (counter, counts) | plan | look-back words | [tile index, its scratch]
  uint64_t b = kHdr + gc_host::align_up(nt * sizeof(gc_work), 256) + gc_host::align_up(nt * 8, 256);
  if (!have_tiles)
    b += gc_host::align_up(nt * sizeof(gc_tile), 256) + gc_host::align_up(gc_host::index_sums_bytes(*codec, n), 256);
  *bytes = b;
  return GC_OK;
}

gc_status gc_decode(const gc_codec* codec, const uint8_t* d_ctrl, uint64_t ctrl_bytes, const uint32_t* d_data,
                    uint64_t data_words, uint64_t n, const gc_tile* d_tiles, uint32_t* d_out, int restore_docids,
                    void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (n == 0) return GC_OK;
  // an area may be empty (a Group-PFD or AFOR list of zeros has no data
  // words); a non-empty one needs a pointer
  if ((!d_ctrl && ctrl_bytes) || (!d_data && data_words) || !d_out || !d_scratch) return GC_ERR_INVALID;
  if (((uintptr_t)d_data & 15) != 0) return GC_ERR_INVALID;
  if (n > 0xffffffffull || ctrl_bytes > 0xffffffffull || data_words > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  uint64_t need = 0;
  gc_decode_scratch_size(codec, n, d_tiles != nullptr, &need);
  if (scratch_bytes < need) return GC_ERR_NOSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t nt = tiles_of(*codec, n);
  unsigned char* base = (unsigned char*)d_scratch;
  uint64_t* count = reinterpret_cast<uint64_t*>(base + 64);
  gc_work* work = reinterpret_cast<gc_work*>(base + kHdr + gc_host::align_up(nt * 8, 256));
  unsigned char* rest = base + kHdr + gc_host::align_up(nt * 8, 256) + gc_host::align_up(nt * sizeof(gc_work), 256);
  uint32_t launches = 0;
  const gc_tile* tiles = d_tiles;
  if (!tiles) {
    gc_tile* built = reinterpret_cast<gc_tile*>(rest);
    void* sums = rest + gc_host::align_up(nt * sizeof(gc_tile), 256);
    st = gc_host::build_tiles(*codec, d_ctrl, ctrl_bytes, n, built, sums, d_status, s);
    if (st != GC_OK) return st;
    launches += gc_host::launches();
    tiles = built;
  }
  // control bytes are staged from 16-byte boundaries: the pool starts at the
  // boundary at or below d_ctrl (never below the allocation that holds it)
  const uint8_t* pool = reinterpret_cast<const uint8_t*>((uintptr_t)d_ctrl & ~(uintptr_t)15);
  const uint64_t lead = d_ctrl ? (uint64_t)(d_ctrl - pool) : 0;
  gc_list one;
  one.ctrl_off = lead;
  one.data_off = 0;
  one.out_off = 0;
  one.n = (uint32_t)n;
  one.tile_off = 0;
  one.ctrl_bytes = (uint32_t)ctrl_bytes;
  one.data_words = (uint32_t)data_words;
  gc_host::reset_launches();
  st = plan_impl(*codec, nullptr, &one, 1, tiles, nt, pool, lead + ctrl_bytes, work, nt, count, d_status, s);
  if (st != GC_OK) return st;
  launches += gc_host::launches();
  // the look-back words sit right after the header, as gc_decode_plan expects
  gc_host::reset_launches();
  st = decode_plan_impl(*codec, work, count, nt, pool, lead + ctrl_bytes, d_data, data_words, d_out, n,
                        restore_docids, default_shape(codec->k), base, d_status, s);
  gc_host::count_launch(launches);
  return st;
}

gc_status gc_decode_paper(const gc_codec* codec, const uint8_t* d_buf, uint64_t buf_bytes, uint64_t n,
                          uint32_t* d_out, int restore_docids, void* d_scratch, uint64_t scratch_bytes,
                          uint32_t* d_status, void* stream) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!d_buf || buf_bytes < 4) return GC_ERR_INVALID;
  if (((uintptr_t)d_buf & 15) != 0) return GC_ERR_INVALID;
  uint32_t off_words = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&off_words, d_buf, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GC_ERR_CUDA;
  const uint64_t doff = 4ull * off_words;
  if (doff < 4 || doff > buf_bytes || (doff & 15)) return GC_ERR_CORRUPT;
  // the control area starts at byte 4 of the buffer: decode from a view
  // whose control pool is the buffer itself (16-byte aligned) and whose list
  // control area starts at offset 4
  gc_host::reset_launches();
  if (n == 0) return GC_OK;
  if (!d_out || !d_scratch) return GC_ERR_INVALID;
  if (n > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  uint64_t need = 0;
  gc_decode_scratch_size(codec, n, 0, &need);
  if (scratch_bytes < need) return GC_ERR_NOSPACE;
  const uint64_t ctrl_bytes = doff - 4;
  const uint32_t* data = reinterpret_cast<const uint32_t*>(d_buf + doff);
  const uint64_t data_words = (buf_bytes - doff) / 4;
  const uint64_t nt = tiles_of(*codec, n);
  unsigned char* base = (unsigned char*)d_scratch;
  uint64_t* count = reinterpret_cast<uint64_t*>(base + 64);
  gc_work* work = reinterpret_cast<gc_work*>(base + kHdr + gc_host::align_up(nt * 8, 256));
  unsigned char* rest = base + kHdr + gc_host::align_up(nt * 8, 256) + gc_host::align_up(nt * sizeof(gc_work), 256);
  gc_tile* built = reinterpret_cast<gc_tile*>(rest);
  void* sums = rest + gc_host::align_up(nt * sizeof(gc_tile), 256);
  st = gc_host::build_tiles(*codec, d_buf + 4, ctrl_bytes, n, built, sums, d_status, s);
  if (st != GC_OK) return st;
  uint32_t launches = gc_host::launches();
  gc_list one;
  one.ctrl_off = 4;
  one.data_off = 0;
  one.out_off = 0;
  one.n = (uint32_t)n;
  one.tile_off = 0;
  one.ctrl_bytes = (uint32_t)ctrl_bytes;
  one.data_words = (uint32_t)data_words;
  gc_host::reset_launches();
  st = plan_impl(*codec, nullptr, &one, 1, built, nt, d_buf, doff, work, nt, count, d_status, s);
  if (st != GC_OK) return st;
  launches += gc_host::launches();
  gc_host::reset_launches();
  st = decode_plan_impl(*codec, work, count, nt, d_buf, doff, data, data_words, d_out, n, restore_docids,
                        default_shape(codec->k), base, d_status, s);
  gc_host::count_launch(launches);
  return st;
}

gc_status gc_plan_batch(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists, const gc_tile* d_tile_pool,
                        uint64_t tile_pool_len, const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes,
                        gc_work* d_work, uint64_t work_cap, uint64_t* d_count, uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!d_count || (nlists && (!d_lists || !d_work))) return GC_ERR_INVALID;
  if (nlists > 0xffffffffull || work_cap > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  if (((uintptr_t)d_work & 15) != 0) return GC_ERR_INVALID;
  return plan_impl(*codec, d_lists, nullptr, nlists, d_tile_pool, tile_pool_len, d_ctrl_pool, ctrl_pool_bytes, d_work,
                   work_cap, d_count, d_status, (cudaStream_t)stream);
}

gc_status gc_plan_select(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists, const uint32_t* d_sel,
                         const uint64_t* d_out_offs, uint64_t nsel, const gc_tile* d_tile_pool, uint64_t tile_pool_len,
                         const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes, gc_work* d_work, uint64_t work_cap,
                         uint64_t* d_count, uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!d_count || (nsel && (!d_lists || !d_sel || !d_out_offs || !d_work))) return GC_ERR_INVALID;
  if (nlists > 0xffffffffull || nsel > 0xffffffffull || work_cap > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  if (((uintptr_t)d_work & 15) != 0) return GC_ERR_INVALID;
  return plan_impl(*codec, d_lists, nullptr, nsel, d_tile_pool, tile_pool_len, d_ctrl_pool, ctrl_pool_bytes, d_work,
                   work_cap, d_count, d_status, (cudaStream_t)stream, d_sel, d_out_offs, nlists);
}

gc_status gc_plan_interleave(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists,
                             const uint32_t* d_sel_pairs, const uint64_t* d_out_pairs, uint64_t npairs,
                             const gc_tile* d_tile_pool, uint64_t tile_pool_len, const uint8_t* d_ctrl_pool,
                             uint64_t ctrl_pool_bytes, gc_work* d_work, uint64_t work_cap, uint64_t* d_count,
                             uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!d_count || (npairs && (!d_lists || !d_sel_pairs || !d_out_pairs || !d_work))) return GC_ERR_INVALID;
  if (nlists > 0xffffffffull || npairs > 0x7fffffffull || work_cap > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  if (((uintptr_t)d_work & 15) != 0) return GC_ERR_INVALID;
  return plan_impl(*codec, d_lists, nullptr, 2 * npairs, d_tile_pool, tile_pool_len, d_ctrl_pool, ctrl_pool_bytes,
                   d_work, work_cap, d_count, d_status, (cudaStream_t)stream, d_sel_pairs, d_out_pairs, nlists, true);
}

gc_status gc_decode_plan_scratch_size(uint64_t work_cap, uint64_t* bytes) {
  if (!bytes) return GC_ERR_INVALID;
  *bytes = kHdr + gc_host::align_up(work_cap * 8, 256);
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
  if (((uintptr_t)d_data_pool & 15) != 0 || ((uintptr_t)d_ctrl_pool & 15) != 0 || ((uintptr_t)d_work & 15) != 0)
    return GC_ERR_INVALID;
  if (work_cap > kMaxWork) return GC_ERR_UNSUPPORTED;
  uint64_t need = 0;
  gc_decode_plan_scratch_size(work_cap, &need);
  if (scratch_bytes < need) return GC_ERR_NOSPACE;
  Shape sh;
  st = launch_shape(*codec, launch, &sh, restore_docids);
  if (st != GC_OK) return st;
  return decode_plan_impl(*codec, d_work, d_count, work_cap, d_ctrl_pool, ctrl_pool_bytes, d_data_pool,
                          data_pool_words, d_out_pool, out_pool_len, restore_docids, sh, (unsigned char*)d_scratch,
                          d_status, (cudaStream_t)stream);
}

gc_status gc_decode_batch_scratch_size(uint64_t nlists, uint64_t max_tiles, uint64_t* bytes) {
  (void)nlists;
  if (!bytes) return GC_ERR_INVALID;
  uint64_t dec = 0;
  gc_decode_plan_scratch_size(max_tiles, &dec);
  *bytes = kHdr + gc_host::align_up(max_tiles * sizeof(gc_work), 256) + dec;
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
  if (((uintptr_t)d_data_pool & 15) != 0 || ((uintptr_t)d_ctrl_pool & 15) != 0) return GC_ERR_INVALID;
  if (max_tiles > kMaxWork || nlists > 0xffffffffull) return GC_ERR_UNSUPPORTED;
  uint64_t need = 0;
  gc_decode_batch_scratch_size(nlists, max_tiles, &need);
  if (scratch_bytes < need) return GC_ERR_NOSPACE;
  Shape sh;
  st = launch_shape(*codec, launch, &sh, restore_docids);
  if (st != GC_OK) return st;
  unsigned char* base = (unsigned char*)d_scratch;
  uint64_t* count = reinterpret_cast<uint64_t*>(base + 64);
  gc_work* work = reinterpret_cast<gc_work*>(base + kHdr);
  unsigned char* rest = base + kHdr + gc_host::align_up(max_tiles * sizeof(gc_work), 256);
  cudaStream_t s = (cudaStream_t)stream;
  st = plan_impl(*codec, d_lists, nullptr, nlists, d_tile_pool, tile_pool_len, d_ctrl_pool, ctrl_pool_bytes, work,
                 max_tiles, count, d_status, s);
  if (st != GC_OK) return st;
  const uint32_t planned = gc_host::launches();
  gc_host::reset_launches();
  st = decode_plan_impl(*codec, work, count, max_tiles, d_ctrl_pool, ctrl_pool_bytes, d_data_pool, data_pool_words,
                        d_out_pool, out_pool_len, restore_docids, sh, rest, d_status, s);
  gc_host::count_launch(planned);
  return st;
}

// ------------------------------------------------ launch shapes, host buffers

gc_status gc_set_launch(const gc_codec* codec, int restore_docids, const gc_launch* launch) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  Shape sh = default_shape(codec->k);
  if (launch) {
    st = fill_shape(*codec, *launch, &sh);
    if (st != GC_OK) return st;
  }
  std::lock_guard<std::mutex> lock(g_launch_mu);
  Registered* r = registered(*codec, restore_docids);
  if (!r) return GC_ERR_CUDA;
  r->set = launch != nullptr;
  r->sh = sh;
  return GC_OK;
}

gc_status gc_get_launch(const gc_codec* codec, int restore_docids, gc_launch* launch) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (!launch) return GC_ERR_INVALID;
  Shape sh;
  st = launch_shape(*codec, nullptr, &sh, restore_docids);
  if (st != GC_OK) return st;
  launch->warps_per_block = sh.warps;
  launch->blocks_per_sm = sh.bps;
  launch->items_per_claim = sh.claim;
  launch->stage_bytes = sh.stage;
  return GC_OK;
}

}  // extern "C"

namespace {

// Where gc_decode_plan_host puts things in the caller's device buffer.
struct HostLayout {
  uint64_t scratch, count, work, ctrl, data, out, total;
};

HostLayout host_layout(uint64_t nwork, uint64_t ctrl_pool_bytes, uint64_t data_pool_words, uint64_t out_pool_len) {
  HostLayout L;
  uint64_t dec = 0;
  gc_decode_plan_scratch_size(nwork, &dec);
  L.scratch = 0;
  L.count = gc_host::align_up(dec, 256);
  L.work = L.count + 256;
  L.ctrl = L.work + gc_host::align_up(nwork * sizeof(gc_work), 256);
  L.data = L.ctrl + gc_host::align_up(ctrl_pool_bytes, 256);
  L.out = L.data + gc_host::align_up(data_pool_words * 4, 256);
  L.total = L.out + gc_host::align_up(out_pool_len * 4, 256);
  return L;
}

}  // namespace

extern "C" {

gc_status gc_decode_plan_host_buffer_size(uint64_t nwork, uint64_t ctrl_pool_bytes, uint64_t data_pool_words,
                                          uint64_t out_pool_len, uint64_t* bytes) {
  if (!bytes) return GC_ERR_INVALID;
  *bytes = host_layout(nwork, ctrl_pool_bytes, data_pool_words, out_pool_len).total;
  return GC_OK;
}

gc_status gc_decode_plan_host(const gc_codec* codec, const gc_work* h_work, uint64_t nwork, const uint8_t* h_ctrl_pool,
                              uint64_t ctrl_pool_bytes, const uint32_t* h_data_pool, uint64_t data_pool_words,
                              uint32_t* h_out_pool, uint64_t out_pool_len, int restore_docids, const gc_launch* launch,
                              void* d_buffers, uint64_t buffer_bytes, uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (nwork == 0) return GC_OK;
  if (!h_work || (!h_ctrl_pool && ctrl_pool_bytes) || (!h_data_pool && data_pool_words) ||
      (!h_out_pool && out_pool_len) || !d_buffers)
    return GC_ERR_INVALID;
  if (((uintptr_t)d_buffers & 255) != 0) return GC_ERR_INVALID;
  if (nwork > kMaxWork) return GC_ERR_UNSUPPORTED;
  const HostLayout L = host_layout(nwork, ctrl_pool_bytes, data_pool_words, out_pool_len);
  if (buffer_bytes < L.total) return GC_ERR_NOSPACE;
  Shape sh;
  st = launch_shape(*codec, launch, &sh, restore_docids);
  if (st != GC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* b = (unsigned char*)d_buffers;
  gc_work* work = reinterpret_cast<gc_work*>(b + L.work);
  uint64_t* count = reinterpret_cast<uint64_t*>(b + L.count);
  uint8_t* ctrl = b + L.ctrl;
  uint32_t* data = reinterpret_cast<uint32_t*>(b + L.data);
  uint32_t* out = reinterpret_cast<uint32_t*>(b + L.out);
  if (cudaMemcpyAsync(work, h_work, nwork * sizeof(gc_work), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (ctrl_pool_bytes && cudaMemcpyAsync(ctrl, h_ctrl_pool, ctrl_pool_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      (data_pool_words &&
       cudaMemcpyAsync(data, h_data_pool, data_pool_words * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMemsetAsync(count, 0, 16, s) != cudaSuccess ||
      (out_pool_len && cudaMemsetAsync(out, 0, out_pool_len * 4, s) != cudaSuccess))
    return GC_ERR_CUDA;
  k_count_records<<<(unsigned)((nwork + 255) / 256), 256, 0, s>>>(work, nwork,
                                                                  reinterpret_cast<unsigned long long*>(count));
  if (cudaGetLastError() != cudaSuccess) return GC_ERR_CUDA;
  st = decode_plan_impl(*codec, work, count, nwork, ctrl, ctrl_pool_bytes, data, data_pool_words, out, out_pool_len,
                        restore_docids, sh, b + L.scratch, d_status, s);
  gc_host::count_launch(1);
  if (st != GC_OK) return st;
  if (out_pool_len && cudaMemcpyAsync(h_out_pool, out, out_pool_len * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return GC_ERR_CUDA;
  return GC_OK;
}

void gc_shutdown(void) {
  std::lock_guard<std::mutex> lock(g_launch_mu);
  for (auto& d : g_reg)
    for (auto& kd : d)
      for (auto& kk : kd)
        for (auto& r : kk) r = Registered{};
  for (auto& d : g_dev) d = DevInfo{};
  ++g_epoch;
  gc_host::forget_devices();
}

// ------------------------------------------------- decoding without scratch

}  // extern "C"

namespace {

// The scratch of gc_decode_static: one fixed array that every device which
// loads the library holds until the process exits. 128 KiB covers the
// scratch of gc_decode for GC_DECODE_STATIC_MAX_INTS ints of any codec, with
// or without a tile index.
constexpr uint64_t kStaticScratchBytes = 128ull << 10;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[64] = {};

// The device address of g_static_scratch on the current device (in host code
// the array's name is only a host-side stand-in). Looked up once per device.
gc_status static_scratch(void** addr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GC_ERR_CUDA;
  if (dev < 0 || dev >= 64) return GC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return GC_ERR_CUDA;
    g_static_addr[dev] = p;
  }
  *addr = g_static_addr[dev];
  return GC_OK;
}

}  // namespace

extern "C" {

gc_status gc_decode_static(const gc_codec* codec, const uint8_t* d_ctrl, uint64_t ctrl_bytes,
                           const uint32_t* d_data, uint64_t data_words, uint64_t n, const gc_tile* d_tiles,
                           uint32_t* d_out, int restore_docids, uint32_t* d_status, void* stream) {
  gc_host::reset_launches();
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  if (n > GC_DECODE_STATIC_MAX_INTS) return GC_ERR_NOSPACE;
  uint64_t need = 0;
  gc_decode_scratch_size(codec, n, d_tiles != nullptr, &need);
  if (need > kStaticScratchBytes) return GC_ERR_NOSPACE;
  if (n == 0) return GC_OK;
  void* scratch = nullptr;
  st = static_scratch(&scratch);
  if (st != GC_OK) return st;
  // gc_decode clears what must start at zero (the claim counter, the
  // look-back words, the plan's counts) before its kernels read them
  return gc_decode(codec, d_ctrl, ctrl_bytes, d_data, data_words, n, d_tiles, d_out, restore_docids, scratch,
                   kStaticScratchBytes, d_status, stream);
}

}  // extern "C"
