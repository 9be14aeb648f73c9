/*
 * gc_oracle.c -- plain, slow, single-threaded CPU oracle for the Group codecs
 * of "A General SIMD-based Approach to Accelerating Compression Algorithms"
 * (arXiv 1502.01916).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code. The product (the CUDA
 * library) shares no code, header, table or helper with it.
 *
 * What it computes, and where the paper defines it:
 *   - d-gaps and their inverse, the prefix sum that restores docIDs (Sec 2.1.1)
 *   - k-way vertical layout: int i of a list goes to component i mod k of
 *     row i / k (Sec 2.1.2, Sec 3.1; the paper fixes k = 4, k = 32 is the
 *     same rule with 32 components)
 *   - the row ("quad") max array (Sec 4.2)
 *   - Group-Simple: Table III selectors, Algorithm 1 selection, packing and
 *     decoding (Sec 4.1-4.3)
 *   - Group-Scheme: length descriptors from Eq. 1, bit widths from Eq. 2,
 *     binary / complete-unary / incomplete-unary control areas (Sec 5.1-5.3)
 *   - Group-AFOR: frames of {8,16,32} rows chosen by dynamic programming
 *     (Sec 6.1)
 *   - Group-PFD: per-frame b from the exception-ratio rule, exceptions stored
 *     apart at 8/16/32 bits (Sec 6.2, Steps 1-4 of encoding, 1-3 of decoding)
 *   - Variable Byte, the code the paper keeps for posting lists shorter than
 *     64 (Sec 2.3, Sec 7.5), in the form of the book the paper cites for it:
 *     7-bit groups, most significant first, the high bit set on a number's
 *     last byte
 *
 * Byte-level conventions where the paper's figures are missing (Figs 1-5):
 *   - every bit stream is LSB-first: control bit t is bit t%8 of byte t/8;
 *     lane j's data bit t is bit t%32 of word data[(t/32)*k + j];
 *   - the Group-Simple selector s is the nibble s of the control area, low
 *     nibble first.
 * These are readings, not facts printed by the paper; parity with the
 * paper's own binaries is unpinned (no bytes of them are printed).
 *
 * Every function is written for a reader checking it against the paper:
 * values are moved one bit at a time and nothing is blocked or fused.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { ORC_SIMPLE = 0, ORC_SCHEME = 1, ORC_AFOR = 2, ORC_PFD = 3 };
enum { ORC_LD_BINARY = 0, ORC_LD_CU = 1, ORC_LD_IU = 2 };
enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_NOSPACE = 2, ORC_ERR_CORRUPT = 3 };

/* Table III: the ten Group-Simple patterns (SEL = index). */
static const uint32_t TABLE3_NUM[10] = {32, 16, 10, 8, 6, 5, 4, 3, 2, 1};
static const uint32_t TABLE3_BW[10] = {1, 2, 3, 4, 5, 6, 8, 10, 16, 32};

/* Group-PFD frame: 32 rows, i.e. 128 ints at k = 4 (the paper's frame) and
 * 1024 ints at k = 32. */
#define PFD_FRAME_ROWS 32u

/* One decoding tile of the GPU layout covers 1024 ints = 1024/k rows. */
#define TILE_INTS 1024u

void orc_table3(uint32_t* num, uint32_t* bw) {
  for (int i = 0; i < 10; ++i) { num[i] = TABLE3_NUM[i]; bw[i] = TABLE3_BW[i]; }
}

/* Effective bit width (Sec 2.1.2): the minimum number of bits that hold x,
 * i.e. ceil(log2(x + 1)); 0 for x = 0. */
uint32_t orc_effective_bits(uint32_t x) {
  uint32_t b = 0;
  while (x) { ++b; x >>= 1; }
  return b;
}

/* 2^b - 1 computed in 64 bits so that b = 32 does not overflow. */
static uint64_t mask64(uint32_t b) { return (b >= 64) ? ~0ull : ((1ull << b) - 1ull); }

static uint64_t rows_of(uint64_t n, uint32_t k) { return (n + k - 1) / k; }

/* Element i of the list, or 0 past its end (rows are zero padded). */
static uint32_t at(const uint32_t* g, uint64_t n, uint64_t i) { return i < n ? g[i] : 0u; }

/* ------------------------------------------------------------------ bits */

/* Set one bit of lane j's stream in the k-way vertical data area. */
static void lane_put_bit(uint32_t* data, uint32_t k, uint32_t lane, uint64_t t, uint32_t bit) {
  if (bit) data[(t / 32) * k + lane] |= (1u << (t % 32));
}

static uint32_t lane_get_bit(const uint32_t* data, uint32_t k, uint32_t lane, uint64_t t) {
  return (data[(t / 32) * k + lane] >> (t % 32)) & 1u;
}

/* Write the low `width` bits of v into lane j at bit position t, low bit
 * first: a value that crosses a word keeps its low part in the current word
 * and its high part in the next one. */
static void lane_put(uint32_t* data, uint32_t k, uint32_t lane, uint64_t t, uint32_t v,
                     uint32_t width) {
  for (uint32_t b = 0; b < width; ++b) lane_put_bit(data, k, lane, t + b, (v >> b) & 1u);
}

static uint32_t lane_get(const uint32_t* data, uint32_t k, uint32_t lane, uint64_t t,
                         uint32_t width) {
  uint32_t v = 0;
  for (uint32_t b = 0; b < width; ++b) v |= lane_get_bit(data, k, lane, t + b) << b;
  return v;
}

static void ctrl_put_bit(uint8_t* ctrl, uint64_t t, uint32_t bit) {
  if (bit) ctrl[t / 8] |= (uint8_t)(1u << (t % 8));
  else ctrl[t / 8] &= (uint8_t)~(1u << (t % 8));
}

static uint32_t ctrl_get_bit(const uint8_t* ctrl, uint64_t t) { return (ctrl[t / 8] >> (t % 8)) & 1u; }

static void ctrl_put(uint8_t* ctrl, uint64_t t, uint32_t v, uint32_t width) {
  for (uint32_t b = 0; b < width; ++b) ctrl_put_bit(ctrl, t + b, (v >> b) & 1u);
}

static uint32_t ctrl_get(const uint8_t* ctrl, uint64_t t, uint32_t width) {
  uint32_t v = 0;
  for (uint32_t b = 0; b < width; ++b) v |= ctrl_get_bit(ctrl, t + b) << b;
  return v;
}

/* ------------------------------------------------------- shared pieces */

/* Sec 4.2: quadmax[i] = max(input[4i..4i+3]); here the maximum of the k ints
 * of row i, zero padded past n. */
void orc_rowmax(const uint32_t* g, uint64_t n, uint32_t k, uint32_t* out) {
  const uint64_t R = rows_of(n, k);
  for (uint64_t r = 0; r < R; ++r) {
    uint32_t m = 0;
    for (uint32_t j = 0; j < k; ++j) {
      uint32_t v = at(g, n, r * k + j);
      if (v > m) m = v;
    }
    out[r] = m;
  }
}

/* Sec 2.1.1: d_1 is kept, d_i = d_{i-1} + gap_i; arithmetic modulo 2^32. */
void orc_prefix_sum(const uint32_t* gaps, uint64_t n, uint32_t* docids) {
  uint32_t acc = 0;
  for (uint64_t i = 0; i < n; ++i) {
    acc += gaps[i];
    docids[i] = acc;
  }
}

/* The inverse: d-gaps of a docID sequence (d_1 kept as is). */
void orc_dgaps(const uint32_t* docids, uint64_t n, uint32_t* gaps) {
  for (uint64_t i = 0; i < n; ++i) gaps[i] = (i == 0) ? docids[0] : docids[i] - docids[i - 1];
}

/* --------------------------------------------------------- Group-Simple */

/* Algorithm 1, step by step: for each position pick the first SEL in
 * ascending order whose pattern takes NUM rows, or all remaining rows, with
 * every row max <= 2^BW - 1. Returns the number of selectors. */
uint64_t orc_gs_select(const uint32_t* maxarr, uint64_t L, uint8_t* mode_arr) {
  uint64_t total = 0;
  uint64_t l = L;
  uint64_t j = 0;
  while (l > 0) {
    uint32_t i;
    uint64_t pos = 0;
    for (i = 0; i < 10; ++i) {
      const uint64_t n = TABLE3_NUM[i];
      const uint32_t b = TABLE3_BW[i];
      const uint64_t mask = mask64(b);
      const uint64_t lim = n < l ? n : l;
      pos = 0;
      while (pos < lim && (uint64_t)maxarr[j + pos] <= mask) ++pos;
      if (pos == n || pos == l) break;
    }
    l -= pos;
    j += pos;
    mode_arr[total++] = (uint8_t)i;
  }
  return total;
}

/* Pack a given selector sequence (Sec 4.2, "packing"): selector s owns data
 * vector s; row q of the selector sits at bits [q*BW, (q+1)*BW) of each
 * component. The selector goes to nibble s of the control area. Returns
 * ORC_ERR_INVALID if a selector does not fit its rows. */
int orc_gs_pack(const uint32_t* g, uint64_t n, uint32_t k, const uint8_t* sel, uint64_t S,
                uint8_t* ctrl, uint64_t* ctrl_bytes, uint32_t* data, uint64_t* data_words) {
  const uint64_t R = rows_of(n, k);
  memset(ctrl, 0, (size_t)((S + 1) / 2));
  memset(data, 0, (size_t)(S * k) * sizeof(uint32_t));
  uint64_t row = 0;
  for (uint64_t s = 0; s < S; ++s) {
    if (sel[s] > 9 || row >= R) return ORC_ERR_INVALID;
    const uint32_t num = TABLE3_NUM[sel[s]], bw = TABLE3_BW[sel[s]];
    const uint64_t rows = (R - row) < num ? (R - row) : num;
    ctrl_put(ctrl, 4 * s, sel[s], 4);
    for (uint64_t q = 0; q < rows; ++q)
      for (uint32_t j = 0; j < k; ++j) {
        const uint32_t v = at(g, n, (row + q) * k + j);
        if ((uint64_t)v > mask64(bw)) return ORC_ERR_INVALID;
        lane_put(data, k, j, 32 * s + q * bw, v, bw);
      }
    row += rows;
  }
  if (row != R) return ORC_ERR_INVALID;
  *ctrl_bytes = (S + 1) / 2;
  *data_words = S * k;
  return ORC_OK;
}

static int gs_encode(const uint32_t* g, uint64_t n, uint32_t k, uint8_t* ctrl, uint64_t* cb,
                     uint32_t* data, uint64_t* dw) {
  const uint64_t R = rows_of(n, k);
  uint32_t* mx = (uint32_t*)malloc((size_t)(R ? R : 1) * sizeof(uint32_t));
  uint8_t* sel = (uint8_t*)malloc((size_t)(R ? R : 1));
  orc_rowmax(g, n, k, mx);
  const uint64_t S = orc_gs_select(mx, R, sel);
  int st = orc_gs_pack(g, n, k, sel, S, ctrl, cb, data, dw);
  free(mx);
  free(sel);
  return st;
}

/* Sec 4.3: read a selector, unpack NUM rows of its vector, advance by 4 bits
 * and one vector, until n ints are out. */
static int gs_decode(const uint8_t* ctrl, uint64_t cb, const uint32_t* data, uint64_t dw,
                     uint64_t n, uint32_t k, uint32_t* out) {
  const uint64_t R = rows_of(n, k);
  uint64_t row = 0, s = 0;
  while (row < R) {
    if (4 * s + 4 > 8 * cb) return ORC_ERR_CORRUPT;
    const uint32_t sel = ctrl_get(ctrl, 4 * s, 4);
    if (sel > 9) return ORC_ERR_CORRUPT;
    if ((s + 1) * k > dw) return ORC_ERR_CORRUPT;
    const uint32_t num = TABLE3_NUM[sel], bw = TABLE3_BW[sel];
    const uint64_t rows = (R - row) < num ? (R - row) : num;
    for (uint64_t q = 0; q < rows; ++q)
      for (uint32_t j = 0; j < k; ++j) {
        const uint64_t i = (row + q) * k + j;
        const uint32_t v = lane_get(data, k, j, 32 * s + q * bw, bw);
        if (i < n) out[i] = v;
      }
    row += rows;
    ++s;
  }
  return ORC_OK;
}

/* --------------------------------------------------------- Group-Scheme */

/* Eq. 1 on the row max: the number of CG-bit units, ceil(bits/CG), with a
 * zero row taking one unit (Table IV lists unary values from 1). The binary
 * descriptor stores units - 1, the unary one stores units. */
uint32_t orc_gsc_units(uint32_t rowmax, uint32_t cg) {
  const uint32_t bits = orc_effective_bits(rowmax);
  uint32_t u = (bits + cg - 1) / cg;
  return u == 0 ? 1 : u;
}

static uint32_t log2_cg(uint32_t cg) { return cg == 1 ? 0 : cg == 2 ? 1 : cg == 4 ? 2 : 3; }

/* Binary descriptors are 5 - log2(CG) bits wide (Table IV) and aligned:
 * CG 1 puts 3 per 16-bit unit, CG 2 and CG 4 put 2 per byte, CG 8 puts 4 per
 * byte (Sec 5.2.1(b); Sec 7 counts 12, 8, 8 and 16 ints per pattern
 * sequence at k = 4). Returns the control bit where row r's descriptor sits
 * and the control bytes that R rows take. */
static uint64_t gsc_bin_pos(uint64_t r, uint32_t cg) {
  switch (cg) {
    case 1: return (r / 3) * 16 + (r % 3) * 5;
    case 2: return (r / 2) * 8 + (r % 2) * 4;
    case 4: return (r / 2) * 8 + (r % 2) * 3;
    default: return (r / 4) * 8 + (r % 4) * 2;
  }
}

static uint64_t gsc_bin_bytes(uint64_t R, uint32_t cg) {
  switch (cg) {
    case 1: return 2 * ((R + 2) / 3);
    case 2: return (R + 1) / 2;
    case 4: return (R + 1) / 2;
    default: return (R + 3) / 4;
  }
}

static int gsc_valid(uint32_t cg, uint32_t ld) {
  if (cg != 1 && cg != 2 && cg != 4 && cg != 8) return 0;
  if (ld > ORC_LD_IU) return 0;
  if (ld == ORC_LD_IU && cg < 4) return 0; /* Sec 5.2.1(a): IU only for CG 4 and 8 */
  return 1;
}

/* Sec 5.2.2: per row, the descriptor goes to the control area and the k ints
 * go, each at BW = CG * units bits, to the k lane streams (values cross words,
 * low part first). Unary descriptors are (units - 1) ones and a closing zero;
 * IU never lets a descriptor straddle a byte and pads the rest with ones; the
 * last control byte is padded with ones (CU, IU) or zeros (binary). */
static int gsc_encode(const uint32_t* g, uint64_t n, uint32_t k, uint32_t cg, uint32_t ld,
                      uint8_t* ctrl, uint64_t ctrl_cap, uint64_t* cb, uint32_t* data,
                      uint64_t data_cap, uint64_t* dw) {
  const uint64_t R = rows_of(n, k);
  uint32_t* mx = (uint32_t*)malloc((size_t)(R ? R : 1) * sizeof(uint32_t));
  orc_rowmax(g, n, k, mx);
  memset(ctrl, 0, (size_t)ctrl_cap);
  memset(data, 0, (size_t)data_cap * sizeof(uint32_t));
  uint64_t cbit = 0, lbit = 0;
  for (uint64_t r = 0; r < R; ++r) {
    const uint32_t u = orc_gsc_units(mx[r], cg);
    const uint32_t bw = cg * u;
    if (ld == ORC_LD_BINARY) {
      ctrl_put(ctrl, gsc_bin_pos(r, cg), u - 1, 5 - log2_cg(cg));
    } else {
      if (ld == ORC_LD_IU && (cbit % 8) + u > 8) {
        while (cbit % 8) ctrl_put_bit(ctrl, cbit++, 1);
      }
      for (uint32_t t = 0; t + 1 < u; ++t) ctrl_put_bit(ctrl, cbit++, 1);
      ctrl_put_bit(ctrl, cbit++, 0);
    }
    for (uint32_t j = 0; j < k; ++j) lane_put(data, k, j, lbit, at(g, n, r * k + j), bw);
    lbit += bw;
  }
  if (ld == ORC_LD_BINARY) {
    *cb = gsc_bin_bytes(R, cg);
  } else {
    while (cbit % 8) ctrl_put_bit(ctrl, cbit++, 1);
    *cb = cbit / 8;
  }
  *dw = ((lbit + 31) / 32) * k;
  free(mx);
  return ORC_OK;
}

/* Sec 5.2.3 / 5.3.1: read the descriptors back, one row at a time. Writes the
 * unit count of each of the first `rows` rows to units[] and returns the
 * control bits consumed up to the end of the last descriptor read, or
 * UINT64_MAX on a malformed stream. */
uint64_t orc_gsc_parse(const uint8_t* ctrl, uint64_t cb, uint32_t cg, uint32_t ld, uint64_t rows,
                       uint32_t* units) {
  uint64_t cbit = 0;
  const uint64_t nbits = 8 * cb;
  const uint32_t maxu = 32 / cg;
  for (uint64_t r = 0; r < rows; ++r) {
    uint32_t u;
    if (ld == ORC_LD_BINARY) {
      const uint64_t p = gsc_bin_pos(r, cg);
      const uint32_t w = 5 - log2_cg(cg);
      if (p + w > nbits) return UINT64_MAX;
      u = ctrl_get(ctrl, p, w) + 1;
      cbit = p + w;
    } else {
      /* IU: a run of ones reaching the end of a byte is padding. */
      for (;;) {
        u = 1;
        uint64_t t = cbit;
        while (t < nbits && ctrl_get_bit(ctrl, t)) { ++u; ++t; }
        if (t >= nbits) return UINT64_MAX;
        if (ld == ORC_LD_IU && (t / 8) != (cbit / 8)) {
          cbit = (cbit / 8 + 1) * 8; /* skip the padding of this byte */
          continue;
        }
        cbit = t + 1;
        break;
      }
    }
    if (u > maxu) return UINT64_MAX;
    units[r] = u;
  }
  return cbit;
}

static int gsc_decode(const uint8_t* ctrl, uint64_t cb, const uint32_t* data, uint64_t dw,
                      uint64_t n, uint32_t k, uint32_t cg, uint32_t ld, uint32_t* out) {
  const uint64_t R = rows_of(n, k);
  uint32_t* units = (uint32_t*)malloc((size_t)(R ? R : 1) * sizeof(uint32_t));
  if (orc_gsc_parse(ctrl, cb, cg, ld, R, units) == UINT64_MAX) { free(units); return ORC_ERR_CORRUPT; }
  uint64_t lbit = 0;
  for (uint64_t r = 0; r < R; ++r) {
    const uint32_t bw = cg * units[r]; /* Eq. 2 */
    if (((lbit + bw + 31) / 32) * k > dw) { free(units); return ORC_ERR_CORRUPT; }
    for (uint32_t j = 0; j < k; ++j) {
      const uint64_t i = r * k + j;
      const uint32_t v = lane_get(data, k, j, lbit, bw);
      if (i < n) out[i] = v;
    }
    lbit += bw;
  }
  free(units);
  return ORC_OK;
}

/* ----------------------------------------------------------- Group-AFOR */

/* Sec 6.1: frames of 8, 16 or 32 rows (AFOR's {8,16,32} ints times the k of
 * the vertical layout), one bit width b per frame (the effective width of the
 * frame's largest row max). The partition minimises the total size, 8
 * control bits plus k*F*b data bits per frame, by dynamic programming over
 * row positions; rows are zero padded to a multiple of 8; among equal costs
 * the larger frame wins. Writes the frame sizes (in rows) and returns how
 * many frames there are. */
uint64_t orc_afor_partition(const uint32_t* rowmax, uint64_t R, uint32_t k, uint32_t* frame_rows) {
  const uint64_t R8 = (R + 7) / 8 * 8;
  const uint64_t nb = R8 / 8;
  uint64_t* best = (uint64_t*)malloc((size_t)(nb + 1) * sizeof(uint64_t));
  uint32_t* choice = (uint32_t*)malloc((size_t)(nb + 1) * sizeof(uint32_t));
  static const uint32_t sizes[3] = {32, 16, 8};
  best[nb] = 0;
  for (uint64_t p = nb; p-- > 0;) {
    const uint64_t i = p * 8;
    best[p] = UINT64_MAX;
    choice[p] = 0;
    for (int s = 0; s < 3; ++s) {
      const uint32_t F = sizes[s];
      if (i + F > R8) continue;
      uint32_t b = 0;
      for (uint64_t r = i; r < i + F; ++r) {
        const uint32_t e = orc_effective_bits(r < R ? rowmax[r] : 0u);
        if (e > b) b = e;
      }
      const uint64_t cost = 8 + (uint64_t)k * F * b + best[p + F / 8];
      if (cost < best[p]) { best[p] = cost; choice[p] = F; }
    }
  }
  uint64_t nf = 0;
  for (uint64_t p = 0; p < nb;) {
    frame_rows[nf++] = choice[p];
    p += choice[p] / 8;
  }
  free(best);
  free(choice);
  return nf;
}

static uint32_t afor_code(uint32_t F) { return F == 8 ? 0u : F == 16 ? 1u : 2u; }

static int afor_encode(const uint32_t* g, uint64_t n, uint32_t k, uint8_t* ctrl, uint64_t ctrl_cap,
                       uint64_t* cb, uint32_t* data, uint64_t data_cap, uint64_t* dw) {
  const uint64_t R = rows_of(n, k);
  const uint64_t R8 = (R + 7) / 8 * 8;
  uint32_t* mx = (uint32_t*)malloc((size_t)(R ? R : 1) * sizeof(uint32_t));
  uint32_t* fr = (uint32_t*)malloc((size_t)(R8 / 8 + 1) * sizeof(uint32_t));
  orc_rowmax(g, n, k, mx);
  const uint64_t nf = orc_afor_partition(mx, R, k, fr);
  memset(ctrl, 0, (size_t)ctrl_cap);
  memset(data, 0, (size_t)data_cap * sizeof(uint32_t));
  uint64_t row = 0, lbit = 0;
  for (uint64_t f = 0; f < nf; ++f) {
    const uint32_t F = fr[f];
    uint32_t b = 0;
    for (uint64_t r = row; r < row + F; ++r) {
      const uint32_t e = orc_effective_bits(r < R ? mx[r] : 0u);
      if (e > b) b = e;
    }
    ctrl[f] = (uint8_t)((afor_code(F) << 6) | b);
    for (uint64_t r = row; r < row + F; ++r) {
      for (uint32_t j = 0; j < k; ++j) lane_put(data, k, j, lbit, at(g, n, r * k + j), b);
      lbit += b;
    }
    row += F;
  }
  *cb = nf;
  *dw = ((lbit + 31) / 32) * k;
  free(mx);
  free(fr);
  return ORC_OK;
}

static int afor_decode(const uint8_t* ctrl, uint64_t cb, const uint32_t* data, uint64_t dw,
                       uint64_t n, uint32_t k, uint32_t* out) {
  const uint64_t R = rows_of(n, k);
  uint64_t row = 0, lbit = 0, f = 0;
  while (row < R) {
    if (f >= cb) return ORC_ERR_CORRUPT;
    const uint32_t code = ctrl[f] >> 6, b = ctrl[f] & 63u;
    if (code > 2 || b > 32) return ORC_ERR_CORRUPT;
    const uint32_t F = 8u << code;
    if (((lbit + (uint64_t)F * b + 31) / 32) * k > dw) return ORC_ERR_CORRUPT;
    for (uint64_t r = row; r < row + F; ++r) {
      for (uint32_t j = 0; j < k; ++j) {
        const uint64_t i = r * k + j;
        const uint32_t v = lane_get(data, k, j, lbit, b);
        if (i < n) out[i] = v;
      }
      lbit += b;
    }
    row += F;
    ++f;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------ Group-PFD */

/* The exception ratio of Sec 6.2, Step 2 ("below zeta") fixed as an integer
 * once: at most floor-below(zeta * 32) exception rows out of a frame's 32,
 * i.e. the largest count c with c < zeta * 32. */
uint32_t orc_pfd_rows_for_zeta(double zeta) {
  const double lim = zeta * (double)PFD_FRAME_ROWS;
  double c = ceil(lim) - 1.0;
  if (c < 0.0) c = 0.0;
  if (c > (double)(PFD_FRAME_ROWS - 1)) c = (double)(PFD_FRAME_ROWS - 1);
  return (uint32_t)c;
}

/* Step 2 for one frame: the minimum b in 0..32 such that at most max_rows
 * row maxima of the frame exceed 2^b - 1 (b = 32 has none). */
uint32_t orc_pfd_frame_b(const uint32_t* rowmax, uint64_t rows, uint32_t max_rows) {
  for (uint32_t b = 0; b <= 32; ++b) {
    uint64_t cnt = 0;
    for (uint64_t r = 0; r < rows; ++r)
      if ((uint64_t)rowmax[r] > mask64(b)) ++cnt;
    if (cnt <= max_rows) return b;
  }
  return 32;
}

static uint32_t pfd_pos_bytes(uint32_t k) { return (PFD_FRAME_ROWS * k) <= 256 ? 1u : 2u; }

/* Steps 1-4: row max array, b per frame, exceptions found first on the row
 * maxima and then among the k ints of each exception row, normal slots at b
 * bits (an exception's slot keeps its low b bits), and the exception array at
 * the most economical of 8, 16 and 32 bits (the Zhang et al. rule the paper
 * follows).
 *
 * Control area: one 32-bit little-endian header per frame
 *   bits 0-5 b, bits 6-7 exception width code (0: 8, 1: 16, 2: 32 bits),
 *   bits 8-31 exception count e,
 * then, frame after frame, each frame's exception record: e positions in the
 * frame (1 byte each when a frame has at most 256 ints, else 2 bytes LE),
 * then e full values at the frame's width (LE). The data of frame f are its
 * rows at b bits in each lane stream. */
static int pfd_encode(const uint32_t* g, uint64_t n, uint32_t k, uint32_t max_rows, uint8_t* ctrl,
                      uint64_t ctrl_cap, uint64_t* cb, uint32_t* data, uint64_t data_cap,
                      uint64_t* dw) {
  const uint64_t R = rows_of(n, k);
  const uint64_t nf = (R + PFD_FRAME_ROWS - 1) / PFD_FRAME_ROWS;
  uint32_t* mx = (uint32_t*)malloc((size_t)(R ? R : 1) * sizeof(uint32_t));
  orc_rowmax(g, n, k, mx);
  memset(ctrl, 0, (size_t)ctrl_cap);
  memset(data, 0, (size_t)data_cap * sizeof(uint32_t));
  const uint32_t pb = pfd_pos_bytes(k);
  uint64_t xbyte = 4 * nf; /* exception records follow the headers */
  uint64_t lbit = 0;
  uint32_t* xpos = (uint32_t*)malloc(PFD_FRAME_ROWS * k * sizeof(uint32_t));
  uint32_t* xval = (uint32_t*)malloc(PFD_FRAME_ROWS * k * sizeof(uint32_t));
  for (uint64_t f = 0; f < nf; ++f) {
    const uint64_t r0 = f * PFD_FRAME_ROWS;
    const uint64_t rows = (R - r0) < PFD_FRAME_ROWS ? (R - r0) : PFD_FRAME_ROWS;
    /* the exception ratio is the frame's own: a list's last frame of fewer
     * than 32 rows may have the whole frame's budget scaled to its rows */
    const uint32_t b = orc_pfd_frame_b(mx + r0, rows, (uint32_t)((uint64_t)max_rows * rows / PFD_FRAME_ROWS));
    uint32_t e = 0, vmax = 0;
    for (uint64_t r = r0; r < r0 + rows; ++r) {
      if ((uint64_t)mx[r] <= mask64(b)) continue;
      for (uint32_t j = 0; j < k; ++j) {
        const uint32_t v = at(g, n, r * k + j);
        if ((uint64_t)v > mask64(b)) {
          xpos[e] = (uint32_t)((r - r0) * k + j);
          xval[e] = v;
          if (v > vmax) vmax = v;
          ++e;
        }
      }
    }
    const uint32_t wcode = e == 0 ? 0u : vmax < 256u ? 0u : vmax < 65536u ? 1u : 2u;
    const uint32_t wbytes = 1u << wcode;
    const uint32_t hdr = b | (wcode << 6) | (e << 8);
    if (xbyte + (uint64_t)e * (pb + wbytes) > ctrl_cap) { free(mx); free(xpos); free(xval); return ORC_ERR_NOSPACE; }
    for (int t = 0; t < 4; ++t) ctrl[4 * f + t] = (uint8_t)(hdr >> (8 * t));
    for (uint32_t x = 0; x < e; ++x)
      for (uint32_t t = 0; t < pb; ++t) ctrl[xbyte++] = (uint8_t)(xpos[x] >> (8 * t));
    for (uint32_t x = 0; x < e; ++x)
      for (uint32_t t = 0; t < wbytes; ++t) ctrl[xbyte++] = (uint8_t)(xval[x] >> (8 * t));
    for (uint64_t r = r0; r < r0 + rows; ++r) {
      for (uint32_t j = 0; j < k; ++j) {
        const uint32_t v = at(g, n, r * k + j);
        lane_put(data, k, j, lbit, (uint32_t)((uint64_t)v & mask64(b)), b);
      }
      lbit += b;
    }
  }
  *cb = xbyte;
  *dw = ((lbit + 31) / 32) * k;
  free(mx);
  free(xpos);
  free(xval);
  return ORC_OK;
}

/* Decoding Steps 1-3: read b and the frame's exceptions, unpack the normal
 * slots, then write each exception over its slot. */
static int pfd_decode(const uint8_t* ctrl, uint64_t cb, const uint32_t* data, uint64_t dw,
                      uint64_t n, uint32_t k, uint32_t* out) {
  const uint64_t R = rows_of(n, k);
  const uint64_t nf = (R + PFD_FRAME_ROWS - 1) / PFD_FRAME_ROWS;
  const uint32_t pb = pfd_pos_bytes(k);
  if (4 * nf > cb) return ORC_ERR_CORRUPT;
  uint64_t xbyte = 4 * nf, lbit = 0;
  for (uint64_t f = 0; f < nf; ++f) {
    const uint32_t hdr = (uint32_t)ctrl[4 * f] | ((uint32_t)ctrl[4 * f + 1] << 8) |
                         ((uint32_t)ctrl[4 * f + 2] << 16) | ((uint32_t)ctrl[4 * f + 3] << 24);
    const uint32_t b = hdr & 63u, wcode = (hdr >> 6) & 3u, e = hdr >> 8;
    if (b > 32 || wcode > 2) return ORC_ERR_CORRUPT;
    const uint64_t r0 = f * PFD_FRAME_ROWS;
    const uint64_t rows = (R - r0) < PFD_FRAME_ROWS ? (R - r0) : PFD_FRAME_ROWS;
    if (((lbit + rows * b + 31) / 32) * k > dw) return ORC_ERR_CORRUPT;
    for (uint64_t r = r0; r < r0 + rows; ++r) {
      for (uint32_t j = 0; j < k; ++j) {
        const uint64_t i = r * k + j;
        const uint32_t v = lane_get(data, k, j, lbit, b);
        if (i < n) out[i] = v;
      }
      lbit += b;
    }
    const uint32_t wbytes = 1u << wcode;
    if (xbyte + (uint64_t)e * (pb + wbytes) > cb) return ORC_ERR_CORRUPT;
    for (uint32_t x = 0; x < e; ++x) {
      uint32_t pos = 0, val = 0;
      for (uint32_t t = 0; t < pb; ++t) pos |= (uint32_t)ctrl[xbyte + (uint64_t)x * pb + t] << (8 * t);
      for (uint32_t t = 0; t < wbytes; ++t)
        val |= (uint32_t)ctrl[xbyte + (uint64_t)e * pb + (uint64_t)x * wbytes + t] << (8 * t);
      if (pos >= rows * k) return ORC_ERR_CORRUPT;
      const uint64_t i = r0 * k + pos;
      if (i < n) out[i] = val;
    }
    xbyte += (uint64_t)e * (pb + wbytes);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------ dispatch */

/* Upper bounds on the control bytes and data words that encoding n ints can
 * take, so that callers can allocate. */
int orc_max_sizes(uint32_t kind, uint32_t k, uint32_t cg, uint32_t ld, uint32_t max_rows, uint64_t n,
                  uint64_t* ctrl_cap, uint64_t* data_cap) {
  if (k != 4 && k != 32) return ORC_ERR_INVALID;
  const uint64_t R = rows_of(n, k);
  switch (kind) {
    case ORC_SIMPLE:
      *ctrl_cap = (R + 1) / 2;
      *data_cap = R * k;
      return ORC_OK;
    case ORC_SCHEME:
      if (!gsc_valid(cg, ld)) return ORC_ERR_INVALID;
      *ctrl_cap = ld == ORC_LD_BINARY ? gsc_bin_bytes(R, cg) : ld == ORC_LD_CU ? (R * (32 / cg) + 7) / 8 : R;
      *data_cap = R * k;
      return ORC_OK;
    case ORC_AFOR: {
      const uint64_t R8 = (R + 7) / 8 * 8;
      *ctrl_cap = R8 / 8;
      *data_cap = R8 * k;
      return ORC_OK;
    }
    case ORC_PFD: {
      if (max_rows >= PFD_FRAME_ROWS) return ORC_ERR_INVALID;
      const uint64_t nf = (R + PFD_FRAME_ROWS - 1) / PFD_FRAME_ROWS;
      *ctrl_cap = 4 * nf + nf * (uint64_t)max_rows * k * (pfd_pos_bytes(k) + 4);
      *data_cap = R * k;
      return ORC_OK;
    }
    default:
      return ORC_ERR_INVALID;
  }
}

int orc_encode(uint32_t kind, uint32_t k, uint32_t cg, uint32_t ld, uint32_t max_rows,
               const uint32_t* g, uint64_t n, uint8_t* ctrl, uint64_t ctrl_cap, uint64_t* ctrl_bytes,
               uint32_t* data, uint64_t data_cap, uint64_t* data_words) {
  uint64_t cc, dc;
  int st = orc_max_sizes(kind, k, cg, ld, max_rows, n, &cc, &dc);
  if (st) return st;
  if (ctrl_cap < cc || data_cap < dc) return ORC_ERR_NOSPACE;
  switch (kind) {
    case ORC_SIMPLE: return gs_encode(g, n, k, ctrl, ctrl_bytes, data, data_words);
    case ORC_SCHEME: return gsc_encode(g, n, k, cg, ld, ctrl, ctrl_cap, ctrl_bytes, data, data_cap, data_words);
    case ORC_AFOR: return afor_encode(g, n, k, ctrl, ctrl_cap, ctrl_bytes, data, data_cap, data_words);
    case ORC_PFD: return pfd_encode(g, n, k, max_rows, ctrl, ctrl_cap, ctrl_bytes, data, data_cap, data_words);
    default: return ORC_ERR_INVALID;
  }
}

int orc_decode(uint32_t kind, uint32_t k, uint32_t cg, uint32_t ld, const uint8_t* ctrl,
               uint64_t ctrl_bytes, const uint32_t* data, uint64_t data_words, uint64_t n,
               uint32_t* out) {
  if (k != 4 && k != 32) return ORC_ERR_INVALID;
  switch (kind) {
    case ORC_SIMPLE: return gs_decode(ctrl, ctrl_bytes, data, data_words, n, k, out);
    case ORC_SCHEME:
      if (!gsc_valid(cg, ld)) return ORC_ERR_INVALID;
      return gsc_decode(ctrl, ctrl_bytes, data, data_words, n, k, cg, ld, out);
    case ORC_AFOR: return afor_decode(ctrl, ctrl_bytes, data, data_words, n, k, out);
    case ORC_PFD: return pfd_decode(ctrl, ctrl_bytes, data, data_words, n, k, out);
    default: return ORC_ERR_INVALID;
  }
}

/* ---------------------------------------------------- paper's one buffer */

/* Sec 4.3 step 1: the decoder reads the start offset of the data area from
 * the head of the buffer. Layout: u32 offset (in 4-byte words from the
 * buffer start) | control area | zero padding to a 16-byte boundary (the
 * data vectors are read with aligned 128-bit loads, Sec 3.2) | data area.
 * Returns the buffer size in bytes (call with buf = NULL to size it). */
uint64_t orc_paper_pack(const uint8_t* ctrl, uint64_t cb, const uint32_t* data, uint64_t dw,
                        uint8_t* buf) {
  const uint64_t doff = (4 + cb + 15) / 16 * 16;
  const uint64_t total = doff + 4 * dw;
  if (!buf) return total;
  memset(buf, 0, (size_t)total);
  const uint32_t w = (uint32_t)(doff / 4);
  for (int t = 0; t < 4; ++t) buf[t] = (uint8_t)(w >> (8 * t));
  memcpy(buf + 4, ctrl, (size_t)cb);
  memcpy(buf + doff, data, (size_t)(4 * dw));
  return total;
}

/* ------------------------------------------------------------ tile index */

/* Where decoding can start at row t*TR (TR = 1024/k rows): the unit (a
 * Group-Simple selector, a Group-Scheme row, an AFOR or PFD frame) that holds
 * that row, given by its first lane bit, its first control bit, the PFD
 * exception byte offset of its frame (from the start of the exception
 * records), and how many of its rows precede the tile. A record may also
 * hold a skip entry in the sense of Sec 7.5: base, the docID just before
 * the tile, valid when flags is 1. One record of 32 bytes per tile: u64
 * lane_bit, u64 ctrl_bit, u32 exc_off, u32 row_skip, u32 base, u32 flags.
 * orc_tile_index fills the positions from the control area alone, which
 * gives no base but the first (the docID before the list is 0);
 * orc_tile_bases adds every base from the gaps. */
typedef struct {
  uint64_t lane_bit;
  uint64_t ctrl_bit;
  uint32_t exc_off;
  uint32_t row_skip;
  uint32_t base;
  uint32_t flags;
} orc_tile;

uint64_t orc_tile_count(uint64_t n, uint32_t k) {
  const uint64_t tr = TILE_INTS / k;
  return (rows_of(n, k) + tr - 1) / tr;
}

int orc_tile_index(uint32_t kind, uint32_t k, uint32_t cg, uint32_t ld, const uint8_t* ctrl,
                   uint64_t cb, uint64_t n, orc_tile* tiles) {
  const uint64_t R = rows_of(n, k);
  const uint64_t tr = TILE_INTS / k;
  const uint64_t nt = orc_tile_count(n, k);
  uint64_t t = 0;               /* next tile to place */
  uint64_t row = 0;             /* first row of the current unit */
  uint64_t lbit = 0, cbit = 0;  /* its first lane bit and control bit */
  uint64_t xoff = 0;            /* PFD: exception byte offset of the frame */
  uint64_t u = 0;               /* unit index */
  uint32_t* units = NULL;
  if (kind == ORC_SCHEME) {
    units = (uint32_t*)malloc((size_t)(R ? R : 1) * sizeof(uint32_t));
    if (orc_gsc_parse(ctrl, cb, cg, ld, R, units) == UINT64_MAX) { free(units); return ORC_ERR_CORRUPT; }
  }
  const uint32_t pb = pfd_pos_bytes(k);
  while (t < nt) {
    uint64_t rows, lbits, cbits_next, xbytes = 0;
    uint64_t cstart = cbit;
    switch (kind) {
      case ORC_SIMPLE: {
        const uint32_t sel = ctrl_get(ctrl, 4 * u, 4);
        if (sel > 9) return ORC_ERR_CORRUPT;
        rows = TABLE3_NUM[sel];
        lbits = 32;
        cbits_next = 4 * (u + 1);
        break;
      }
      case ORC_SCHEME: {
        rows = 1;
        lbits = (uint64_t)cg * units[u];
        if (ld == ORC_LD_BINARY) {
          cstart = gsc_bin_pos(u, cg);
          cbits_next = gsc_bin_pos(u + 1, cg);
        } else {
          if (ld == ORC_LD_IU && (cbit % 8) + units[u] > 8) cstart = (cbit / 8 + 1) * 8;
          cbits_next = cstart + units[u];
        }
        break;
      }
      case ORC_AFOR: {
        const uint32_t code = ctrl[u] >> 6, b = ctrl[u] & 63u;
        if (code > 2 || b > 32) return ORC_ERR_CORRUPT;
        rows = 8u << code;
        lbits = rows * b;
        cbits_next = 8 * (u + 1);
        break;
      }
      case ORC_PFD: {
        const uint32_t hdr = (uint32_t)ctrl[4 * u] | ((uint32_t)ctrl[4 * u + 1] << 8) |
                             ((uint32_t)ctrl[4 * u + 2] << 16) | ((uint32_t)ctrl[4 * u + 3] << 24);
        rows = PFD_FRAME_ROWS;
        lbits = rows * (hdr & 63u);
        cbits_next = 32 * (u + 1);
        xbytes = (uint64_t)(hdr >> 8) * (pb + (1u << ((hdr >> 6) & 3u)));
        break;
      }
      default:
        return ORC_ERR_INVALID;
    }
    while (t < nt && t * tr < row + rows) {
      tiles[t].lane_bit = lbit;
      tiles[t].ctrl_bit = cstart;
      tiles[t].exc_off = (uint32_t)xoff;
      tiles[t].row_skip = (uint32_t)(t * tr - row);
      tiles[t].base = 0;
      tiles[t].flags = t == 0 ? 1u : 0u;
      ++t;
    }
    row += rows;
    lbit += lbits;
    cbit = cbits_next;
    xoff += xbytes;
    ++u;
    if (row > R + 32 && t < nt) { free(units); return ORC_ERR_CORRUPT; }
  }
  free(units);
  return ORC_OK;
}

/* Skip entries: the docID before tile t is the prefix sum of Sec 2.1.1 up
 * to int t*1024 - 1, i.e. the sum of the gaps before the tile modulo 2^32
 * (0 for tile 0). Sets base and flags = 1 in each of the nt records. */
void orc_tile_bases(const uint32_t* gaps, uint64_t n, uint32_t k, orc_tile* tiles) {
  const uint64_t nt = orc_tile_count(n, k);
  uint32_t sum = 0;
  uint64_t i = 0;
  for (uint64_t t = 0; t < nt; ++t) {
    for (; i < t * TILE_INTS; ++i) sum += gaps[i];
    tiles[t].base = sum;
    tiles[t].flags = 1u;
  }
}

/* ------------------------------------------------------------ Variable Byte
 * Sec 2.3: a non-negative integer in whole bytes, 7 bits of its binary
 * representation per byte, the remaining (most significant) bit of each
 * byte telling whether it is the number's last byte. Groups go most
 * significant first and the last byte carries the set bit (the form of the
 * book the paper cites). Sec 7.5 codes posting lists shorter than 64 so. */

/* bytes Variable Byte takes for x: one per started group of 7 bits, at
 * least one */
uint32_t orc_vb_size(uint32_t x) {
  uint32_t bytes = 1;
  while (x >= 128u) {
    x /= 128u;
    bytes += 1;
  }
  return bytes;
}

/* encode n ints to out (capacity cap bytes); returns the bytes written, or
 * (uint64_t)-1 when they do not fit */
uint64_t orc_vb_encode(const uint32_t* g, uint64_t n, uint8_t* out, uint64_t cap) {
  uint64_t pos = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint32_t x = g[i];
    const uint32_t bytes = orc_vb_size(x);
    if (pos + bytes > cap) return (uint64_t)-1;
    /* group j (0 = least significant) goes to byte pos + bytes - 1 - j */
    uint32_t v = x;
    for (uint32_t j = 0; j < bytes; ++j) {
      out[pos + bytes - 1 - j] = (uint8_t)(v % 128u);
      v /= 128u;
    }
    out[pos + bytes - 1] |= 0x80u; /* the last byte */
    pos += bytes;
  }
  return pos;
}

/* decode n ints from the first nbytes bytes of in; returns 0, or
 * ORC_ERR_CORRUPT when the bytes end before n numbers do, a number needs
 * more than 32 bits, or bytes are left over */
int orc_vb_decode(const uint8_t* in, uint64_t nbytes, uint64_t n, uint32_t* out) {
  uint64_t pos = 0;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t v = 0;
    for (;;) {
      if (pos >= nbytes) return ORC_ERR_CORRUPT;
      const uint8_t b = in[pos++];
      v = v * 128u + (b & 0x7fu);
      if (v > 0xffffffffull) return ORC_ERR_CORRUPT;
      if (b & 0x80u) break;
    }
    out[i] = (uint32_t)v;
  }
  return pos == nbytes ? ORC_OK : ORC_ERR_CORRUPT;
}

