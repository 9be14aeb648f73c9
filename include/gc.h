/*
 * gc.h -- C ABI of the GB300 Group-codec library (decode hot path of
 * "A General SIMD-based Approach to Accelerating Compression Algorithms",
 * arXiv 1502.01916).
 *
 * The library compresses and decompresses the d-gaps of posting lists
 * (Sec 2.1.1) with the paper's four Group codecs: Group-Simple (Sec 4),
 * Group-Scheme (Sec 5), Group-AFOR (Sec 6.1) and Group-PFD (Sec 6.2). Every
 * codec keeps its control patterns in a control area apart from the data
 * area (Sec 3.1), and the data area uses the k-way vertical layout
 * (Sec 2.1.2): int i of a list goes to component i mod k of row i / k. k = 4
 * is the paper's layout (128-bit vectors); k = 32 is the same rule with
 * 128-byte vectors, one component per lane of a warp.
 *
 * Conventions for every call:
 *   - All buffers are owned by the caller. Pointers named d_* are device
 *     pointers (cudaMalloc / torch CUDA tensors); h_* are host pointers.
 *   - Calls that take a `stream` (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream) are asynchronous: argument errors that the host
 *     can see are returned at once; errors found by the GPU (a corrupt
 *     stream, a look-back wait that ran out) are written to the caller's
 *     d_status (two uint32: error code, then the failing tile or list), which
 *     the caller reads after synchronising. d_status is never cleared by the
 *     library: zero it before a call whose errors you want to see.
 *   - The library allocates no device memory: scratch is passed in, sized by
 *     the matching *_scratch_size call.
 *   - Bit order is LSB-first everywhere: control bit t is bit t%8 of byte
 *     t/8; lane j's data bit t is bit t%32 of data word (t/32)*k + j.
 */
#ifndef GC_H
#define GC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GC_OK = 0,
  GC_ERR_INVALID = 1,     /* bad argument (codec, size, alignment, NULL) */
  GC_ERR_NOSPACE = 2,     /* an output or scratch buffer is too small */
  GC_ERR_CORRUPT = 3,     /* a control or data stream is malformed (device) */
  GC_ERR_CUDA = 4,        /* a CUDA call failed */
  GC_ERR_TIMEOUT = 5,     /* a bounded wait between tiles gave up (device) */
  GC_ERR_UNSUPPORTED = 6  /* a valid request that this library does not serve */
} gc_status;

enum { GC_SIMPLE = 0, GC_SCHEME = 1, GC_AFOR = 2, GC_PFD = 3 };
enum { GC_LD_BINARY = 0, GC_LD_CU = 1, GC_LD_IU = 2 };

/* A codec.
 *   kind: GC_SIMPLE (Table III selectors, Algorithm 1), GC_SCHEME (Eq. 1/2),
 *         GC_AFOR (frames of 8/16/32 rows by dynamic programming), GC_PFD
 *         (32-row frames with exceptions).
 *   k:    4 or 32 ints per row.
 *   cg, ld: Group-Scheme compression granularity (1, 2, 4, 8 bits) and
 *         length descriptor (binary, complete unary, incomplete unary; IU
 *         only with cg 4 or 8, Sec 5.2.1(a)).
 *   pfd_exc_rows: Group-PFD, the most rows of a 32-row frame that may hold
 *         exceptions (the ratio threshold zeta of Sec 6.2 Step 2 as an
 *         integer; gc_pfd_rows_for_zeta converts). A list's last frame of
 *         r < 32 rows may hold floor(pfd_exc_rows * r / 32) (its own
 *         exception ratio stays below zeta). */
typedef struct gc_codec {
  uint32_t kind;
  uint32_t k;
  uint32_t cg;
  uint32_t ld;
  uint32_t pfd_exc_rows;
  uint32_t reserved; /* must be 0 */
} gc_codec;

/* Where decoding of one 1024-int tile (1024/k rows) starts: the unit (a
 * selector, a Group-Scheme row, an AFOR or PFD frame) that holds the tile's
 * first row. lane_bit: first bit of the unit in every lane stream; ctrl_bit:
 * first control bit of the unit; exc_off: Group-PFD, byte offset of the
 * unit's exception record from the start of the exception records (0 for
 * other codecs); row_skip: rows of the unit before the tile.
 *
 * A record may also carry a skip entry in the sense of Sec 7.5 (the index
 * keeps a docID every so many postings): base is the docID just before the
 * tile, i.e. the sum of the list's gaps before the tile modulo 2^32, valid
 * when flags has GC_TILE_BASE. A tile with a base decodes without waiting
 * for the tiles before it; one without a base takes its prefix from them
 * by look-back. The GPU encoders write bases; a tile index built from the
 * control area alone (gc_build_tiles, the paper's format) has none. Tile 0
 * of any list is (0, 0, 0, 0, base 0, GC_TILE_BASE). 32 bytes. */
typedef struct gc_tile {
  uint64_t lane_bit;
  uint64_t ctrl_bit;
  uint32_t exc_off;
  uint32_t row_skip;
  uint32_t base;
  uint32_t flags;
} gc_tile;

enum { GC_TILE_BASE = 1u };

/* One posting list in a batch (40 bytes). ctrl_off: byte offset of its
 * control area in the control pool; data_off: word offset of its data area
 * in the data pool (the data of every list starts on a vector boundary,
 * i.e. data_off is a multiple of k); out_off: index of its first output int;
 * n: ints in the list; tile_off: index in the tile pool of the record of its
 * tile 1 (lists of one tile need no record); ctrl_bytes, data_words: the
 * sizes of its two areas. */
typedef struct gc_list {
  uint64_t ctrl_off;
  uint64_t data_off;
  uint64_t out_off;
  uint32_t n;
  uint32_t tile_off;
  uint32_t ctrl_bytes;
  uint32_t data_words;
} gc_list;

/* One unit of work of the decoder: one tile of one list, with what a warp
 * needs to stage the tile's streams in shared memory and decode it (64
 * bytes, 16-byte aligned). gc_plan_batch writes them.
 *   ctrl_at:  byte offset of the list's control area in the control pool.
 *   data_at:  word offset in the data pool of the vector that holds the
 *             tile's first row (a Group-AFOR frame may start rows earlier).
 *   out_at:   index of the tile's first output int in the output pool.
 *   ctrl_bit: first control bit of the tile's first unit, from ctrl_at.
 *   ctrl_bytes: control bytes of the list.
 *   tile:     tile index within the list.
 *   list:     list index; 0xffffffff marks an empty record.
 *   base:     docID just before the tile (GC_WORK_HAS_BASE).
 *   exc_at:   Group-PFD: first byte of the tile's exception records, from
 *             ctrl_at.
 *   win_at, win_len: the control bytes to stage, from ctrl_at (win_at may
 *             be negative: the window starts on a 16-byte boundary of the
 *             pool); win_len is a multiple of 16.
 *   shape:    GC_WORK_* fields below.
 *   exc_len:  Group-PFD exception bytes to stage, from exc_at rounded down
 *             to a 16-byte boundary of the pool; a multiple of 16. */
typedef struct gc_work {
  uint64_t ctrl_at;
  uint64_t data_at;
  uint64_t out_at;
  uint64_t ctrl_bit;
  uint32_t ctrl_bytes;
  uint32_t tile;
  uint32_t list;
  uint32_t base;
  uint32_t exc_at;
  int32_t win_at;
  uint32_t shape;
  uint16_t win_len;
  uint16_t exc_len;
} gc_work;

/* gc_work.shape: bits 0-9 the tile's ints minus one; 10-18 data vectors
 * (k words each) to stage from data_at; 19-23 the lane bit of the tile's
 * first row within the first staged word; 24-28 rows of the tile's first
 * unit before the tile; bit 29 base is valid; bit 30 a later tile without
 * a base takes its prefix from this tile; bit 31 (GC_WORK_RAW) the tile's
 * values are written as they are, without the prefix sum, by a decode with
 * restore_docids = GC_RESTORE_PER_RECORD. */
enum {
  GC_WORK_VEC_SHIFT = 10,
  GC_WORK_BIT_SHIFT = 19,
  GC_WORK_SKIP_SHIFT = 24,
  GC_WORK_HAS_BASE = 1u << 29,
  GC_WORK_PUBLISH = 1u << 30
};
#define GC_WORK_RAW 0x80000000u

/* restore_docids of gc_decode_plan: 0 writes every tile's values (d-gaps,
 * TFs), 1 restores docIDs (Sec 2.1.1) for every tile, and
 * GC_RESTORE_PER_RECORD restores docIDs except in tiles whose record carries
 * GC_WORK_RAW (the TF tiles of an interleaved plan, gc_plan_interleave). */
#define GC_RESTORE_PER_RECORD 2

/* Launch shape of the persistent decoder (NULL = the shape registered with
 * gc_set_launch, else the library default; a field left 0 takes its
 * default). A block has one staging warp, which claims plan records, groups
 * them into packs of up to 32 lines of 32 ints and places each pack in a
 * shared-memory ring, and warps_per_block decoding warps, which copy the
 * packs' bytes into the ring and decode them in turn.
 *   warps_per_block: decoding warps per block, 1..23 at k = 32 (default
 *     7), 1..15 at k = 4 (default 7).
 *   blocks_per_sm: resident blocks per SM, 1..8 (default 3 at k = 32, 2
 *     at k = 4); the
 *     persistent grid is blocks_per_sm * SMs (fewer when fewer fit). A
 *     block takes 1/blocks_per_sm of the SM's shared memory.
 *   items_per_claim: 1..32 plan records a block takes from the shared
 *     counter per atomic (default 32). A plan with records that take their
 *     prefix by look-back (its count[1] > 0) is dealt to the blocks in turn
 *     instead (block b takes records b, b + G, b + 2G, ... of a grid of G
 *     blocks), whatever this says: records claimed from the counter and
 *     queued in one block would hold back the later tiles of their lists in
 *     the others.
 *   stage_bytes: bytes of the block's staging ring (the staging depth:
 *     how much compressed data is in flight per block); 0 = all the
 *     shared memory the block's share leaves. A shape whose ring would be
 *     smaller than 12 KB is refused with GC_ERR_INVALID. */
typedef struct gc_launch {
  uint32_t warps_per_block;
  uint32_t blocks_per_sm;
  uint32_t items_per_claim;
  uint32_t stage_bytes;
} gc_launch;

/* ------------------------------------------------------------- sizes */

/* The exception ratio threshold zeta of Group-PFD (Sec 6.2 Step 2: the
 * ratio must stay below zeta) as the largest row count c with c/32 < zeta,
 * clamped to 0..31. */
uint32_t gc_pfd_rows_for_zeta(double zeta);

/* Upper bounds on the control bytes and data words of n ints, and the number
 * of 1024-int tiles. Returns GC_ERR_INVALID for a bad codec. */
gc_status gc_max_encoded_size(const gc_codec* codec, uint64_t n, uint64_t* ctrl_cap,
                              uint64_t* data_cap, uint64_t* ntiles);

/* ----------------------------------------------------------- encoding */

/* Scratch bytes gc_encode needs for n ints. */
gc_status gc_encode_scratch_size(const gc_codec* codec, uint64_t n, uint64_t* bytes);

/* Encode n uint32 (d-gaps, or any values) on the GPU. Output streams are
 * byte-identical to the paper's procedures: Algorithm 1 for Group-Simple,
 * Eq. 1 for Group-Scheme, the size-minimising partition for Group-AFOR,
 * Steps 1-4 of Sec 6.2 for Group-PFD.
 *   d_gaps: n uint32 on the device.
 *   d_ctrl / ctrl_cap, d_data / data_cap: output areas on the device, at
 *     least gc_max_encoded_size; d_ctrl must be 4-byte aligned, d_data
 *     16-byte aligned.
 *   d_tiles: NULL, or gc_max_encoded_size's ntiles records to receive the
 *     tile index, every record with its base (GC_TILE_BASE).
 *   d_sizes: two uint64 on the device, receive (control bytes, data words).
 * Asynchronous on `stream`. */
gc_status gc_encode(const gc_codec* codec, const uint32_t* d_gaps, uint64_t n, uint8_t* d_ctrl,
                    uint64_t ctrl_cap, uint32_t* d_data, uint64_t data_cap, gc_tile* d_tiles,
                    uint64_t* d_sizes, void* d_scratch, uint64_t scratch_bytes, void* stream);

/* Encode many lists at once (an index). h_n[i] ints of list i start at
 * h_in_off[i] of d_gaps; the caller guarantees h_in_off[i] + h_n[i] <= the
 * length of d_gaps (the library does not know it and reads those ranges as
 * given). h_in_off[i] is also list i's output offset (gc_list.out_off).
 * The library lays the lists' encodings out back to back and
 * writes, on the device: d_lists (one gc_list per list), d_ctrl, d_data,
 * d_tiles (tile records of tiles >= 1, with bases), and d_totals = (control
 * bytes, data words, tile records). Capacities are checked on the host from the
 * gc_max_encoded_size bounds of each list. */
gc_status gc_encode_batch_scratch_size(const gc_codec* codec, const uint32_t* h_n, uint64_t nlists,
                                       uint64_t* bytes);
gc_status gc_encode_batch(const gc_codec* codec, const uint32_t* d_gaps, const uint32_t* h_n,
                          const uint64_t* h_in_off, uint64_t nlists, gc_list* d_lists,
                          uint8_t* d_ctrl, uint64_t ctrl_cap, uint32_t* d_data, uint64_t data_cap,
                          gc_tile* d_tiles, uint64_t tiles_cap, uint64_t* d_totals, void* d_scratch,
                          uint64_t scratch_bytes, void* stream);

/* ----------------------------------------------------------- decoding */

/* Scratch bytes gc_decode needs for n ints; have_tiles = 0 when the caller
 * passes no tile index (the paper's format) and the library must build one. */
gc_status gc_decode_scratch_size(const gc_codec* codec, uint64_t n, int have_tiles,
                                 uint64_t* bytes);

/* Build the tile index of one encoded list from its control area alone
 * (one pass over control bytes, no data read). d_tiles receives
 * gc_max_encoded_size's ntiles records; none but tile 0 carries a base. */
gc_status gc_build_tiles(const gc_codec* codec, const uint8_t* d_ctrl, uint64_t ctrl_bytes,
                         uint64_t n, gc_tile* d_tiles, void* d_scratch, uint64_t scratch_bytes,
                         uint32_t* d_status, void* stream);

/* Decode one list of n ints (Sec 4.3, Sec 5.2.3, Sec 6.2 decoding Steps 1-3)
 * and, when restore_docids != 0, restore docIDs with the inclusive prefix
 * sum of the gaps modulo 2^32 (Sec 2.1.1) in the same kernel.
 *   d_ctrl / ctrl_bytes, d_data / data_words: the list's areas; d_data
 *     16-byte aligned. Control bytes are staged from the 16-byte boundary
 *     at or below d_ctrl, inside the allocation that holds d_ctrl.
 *   d_tiles: the list's tile index (as written by gc_encode or
 *     gc_build_tiles), or NULL to build it into scratch first.
 *   d_out: n uint32.
 * One launch decodes every tile: a plan of the list's tiles is built in
 * scratch, then the decoder of gc_decode_plan runs it. Tiles whose records
 * carry a base (GC_TILE_BASE) start from it; the others chain their prefix
 * sums to the tiles before them with a bounded decoupled look-back. */
gc_status gc_decode(const gc_codec* codec, const uint8_t* d_ctrl, uint64_t ctrl_bytes,
                    const uint32_t* d_data, uint64_t data_words, uint64_t n, const gc_tile* d_tiles,
                    uint32_t* d_out, int restore_docids, void* d_scratch, uint64_t scratch_bytes,
                    uint32_t* d_status, void* stream);

/* Paper's single buffer (Sec 4.3 step 1): u32 offset of the data area in
 * 4-byte words | control area | zero padding to 16 bytes | data area.
 * gc_decode_paper reads the offset from the head of the buffer (a device
 * buffer: the offset is copied to the host, so this call synchronises
 * `stream` once) and decodes as gc_decode with no tile index. d_buf must be
 * 16-byte aligned. */
gc_status gc_decode_paper(const gc_codec* codec, const uint8_t* d_buf, uint64_t buf_bytes,
                          uint64_t n, uint32_t* d_out, int restore_docids, void* d_scratch,
                          uint64_t scratch_bytes, uint32_t* d_status, void* stream);

/* Bytes of the paper's single buffer (Sec 4.3 step 1) for a control area of
 * ctrl_bytes and a data area of data_words: the data area starts at the
 * first 16-byte boundary after the 4-byte head and the control area. */
uint64_t gc_paper_bytes(uint64_t ctrl_bytes, uint64_t data_words);

/* Build the paper's single buffer (Sec 4.3 step 1) from a list's control
 * and data areas (as gc_encode wrote them), all on the device: d_buf (16-byte
 * aligned, buf_bytes >= gc_paper_bytes) receives the data offset in words,
 * the control bytes, zeros to the 16-byte boundary, and the data words.
 * Asynchronous on `stream` (one small kernel and two device copies).
 * GC_ERR_NOSPACE when the buffer is too small, GC_ERR_INVALID for a missing
 * or misaligned pointer. */
gc_status gc_pack_paper(const uint8_t* d_ctrl, uint64_t ctrl_bytes, const uint32_t* d_data, uint64_t data_words,
                        uint8_t* d_buf, uint64_t buf_bytes, void* stream);

/* Split the paper's single buffer (d_buf, buf_bytes, 16-byte aligned) back
 * into a control area and a data area. The head is copied to the host, so
 * the call synchronises `stream` once. *ctrl_bytes receives the control
 * area's length as the buffer gives it (up to its 16-byte boundary: the
 * padding zeros are included, which decode as they did inside the buffer)
 * and *data_words the words after it; both are set before the capacity
 * check, so a call that returns GC_ERR_NOSPACE tells the sizes it needs. A
 * head that points outside the buffer or off a 16-byte boundary returns
 * GC_ERR_CORRUPT. The copies are asynchronous on `stream`. */
gc_status gc_unpack_paper(const uint8_t* d_buf, uint64_t buf_bytes, uint8_t* d_ctrl, uint64_t ctrl_cap,
                          uint32_t* d_data, uint64_t data_cap, uint64_t* ctrl_bytes, uint64_t* data_words,
                          void* stream);

/* The work plan of a batch: one gc_work per tile of every list, a list's
 * tiles in order at consecutive records, built on the device from the
 * descriptors, the tile pool and the control pool (read only where a
 * Group-AFOR frame straddles two tiles). A plan depends only on the index,
 * so a caller that decodes the same resident index many times builds it
 * once.
 *   d_lists / nlists, d_tile_pool / tile_pool_len, d_ctrl_pool /
 *     ctrl_pool_bytes: as for gc_decode_batch.
 *   d_work / work_cap: output records (16-byte aligned). A batch with more
 *     tiles reports GC_ERR_NOSPACE in d_status.
 *   d_count: two uint64 on the device, receive the number of tiles and the
 *     number of tiles that have no base and take their prefix by look-back.
 * A descriptor or tile record that points outside its list reports
 * GC_ERR_CORRUPT (the record is emptied). Asynchronous on `stream`;
 * graph-capturable. */
gc_status gc_plan_batch(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists,
                        const gc_tile* d_tile_pool, uint64_t tile_pool_len, const uint8_t* d_ctrl_pool,
                        uint64_t ctrl_pool_bytes, gc_work* d_work, uint64_t work_cap, uint64_t* d_count,
                        uint32_t* d_status, void* stream);

/* The work plan of a selection of an index's lists: what gc_plan_batch
 * gives for the lists d_lists[d_sel[i]], i < nsel, each decoded to
 * d_out_offs[i] of the output pool instead of its descriptor's out_off. A
 * server builds one per batch of requests over a resident index (the
 * selected lists' tiles are consecutive records, in selection order). A
 * selection index >= nlists plans nothing for that entry. Records name the
 * index's list (d_sel[i]). Other arguments, results and errors as for
 * gc_plan_batch; asynchronous on `stream`, graph-capturable. */
gc_status gc_plan_select(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists, const uint32_t* d_sel,
                         const uint64_t* d_out_offs, uint64_t nsel, const gc_tile* d_tile_pool,
                         uint64_t tile_pool_len, const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes,
                         gc_work* d_work, uint64_t work_cap, uint64_t* d_count, uint32_t* d_status, void* stream);

/* The interleaved plan of a list's docID and term-frequency streams (the
 * paper's TF columns, Sec 7.3, Tables VII and IX): for each pair p < npairs,
 * index list d_sel_pairs[2p] holds a list's d-gaps and list
 * d_sel_pairs[2p + 1] its TFs (the same number of ints). Their tiles are
 * planned alternately -- d-gap tile 0, TF tile 0, d-gap tile 1, ... -- so one
 * decode of the plan with restore_docids = GC_RESTORE_PER_RECORD writes the
 * pair's docIDs to d_out_pairs[2p] and its TFs, without the prefix sum (the
 * TF records carry GC_WORK_RAW), to d_out_pairs[2p + 1]: the two streams of
 * a posting share the launch, the claim and, mostly, the block that decodes
 * them. The d-gap tiles of a pair are not consecutive records, so none of
 * them can take its prefix by look-back: every d-gap tile after a list's
 * first must carry its skip entry (GC_TILE_BASE, which gc_encode_batch
 * writes), else GC_ERR_UNSUPPORTED in d_status and the record is emptied. A
 * pair whose lists differ in length reports GC_ERR_INVALID and plans
 * nothing. Other arguments, results and errors as for gc_plan_select (2 *
 * npairs entries); asynchronous on `stream`, graph-capturable. */
gc_status gc_plan_interleave(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists,
                             const uint32_t* d_sel_pairs, const uint64_t* d_out_pairs, uint64_t npairs,
                             const gc_tile* d_tile_pool, uint64_t tile_pool_len, const uint8_t* d_ctrl_pool,
                             uint64_t ctrl_pool_bytes, gc_work* d_work, uint64_t work_cap, uint64_t* d_count,
                             uint32_t* d_status, void* stream);

/* Scratch bytes gc_decode_plan needs for a plan of up to work_cap tiles. */
gc_status gc_decode_plan_scratch_size(uint64_t work_cap, uint64_t* bytes);

/* Decode every tile of a plan in one persistent launch (Sec 4.3, 5.2.3,
 * 6.2 decoding per tile; docIDs by Sec 2.1.1 when restore_docids != 0).
 * Each block's staging warp claims tiles from a shared counter in plan
 * order and groups them into packs of up to 32 lines of 32 ints (several
 * small tiles together); its decoding warps copy each pack's control and
 * data bytes into a shared-memory ring one pack ahead and decode it. A tile
 * with a base starts from it; one without takes its prefix from the tiles
 * before it by a bounded decoupled look-back. The pools are those the
 * plan's records point into (16-byte aligned); every read is bounds-checked
 * against these sizes, and a record whose tile does not fit out_pool_len
 * reports GC_ERR_INVALID. launch = NULL takes the shape registered with
 * gc_set_launch for this codec, else the library default (gc_launch).
 * Asynchronous on `stream`; graph-capturable (memsets and one kernel). */
gc_status gc_decode_plan(const gc_codec* codec, const gc_work* d_work, const uint64_t* d_count,
                         uint64_t work_cap, const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes,
                         const uint32_t* d_data_pool, uint64_t data_pool_words, uint32_t* d_out_pool,
                         uint64_t out_pool_len, int restore_docids, const gc_launch* launch,
                         void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status, void* stream);

/* Scratch bytes gc_decode_batch needs for a batch of up to max_tiles tiles
 * (the sum over its lists of gc_max_encoded_size's ntiles). */
gc_status gc_decode_batch_scratch_size(uint64_t nlists, uint64_t max_tiles, uint64_t* bytes);

/* Decode many lists in one call: gc_plan_batch into scratch, then
 * gc_decode_plan.
 *   d_lists: nlists descriptors on the device (see gc_list).
 *   d_ctrl_pool / ctrl_pool_bytes, d_data_pool / data_pool_words,
 *   d_tile_pool / tile_pool_len: the index areas (control and data pools
 *     16-byte aligned); every read is bounds-checked against these sizes.
 *   d_out_pool / out_pool_len: outputs; list i goes to out_off.
 *   max_tiles: the scratch was sized for this many tiles; a batch with more
 *     reports GC_ERR_NOSPACE in d_status.
 *   launch: as for gc_decode_plan (NULL = the registered shape, else the
 *     library default).
 * The call is graph-capturable (no host synchronisation). */
gc_status gc_decode_batch(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists,
                          const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes,
                          const uint32_t* d_data_pool, uint64_t data_pool_words,
                          const gc_tile* d_tile_pool, uint64_t tile_pool_len, uint32_t* d_out_pool,
                          uint64_t out_pool_len, int restore_docids, uint64_t max_tiles,
                          const gc_launch* launch, void* d_scratch, uint64_t scratch_bytes,
                          uint32_t* d_status, void* stream);

/* gc_decode for callers that cannot allocate device memory: a plug-in or
 * service embedded in a host application that owns all of the device's
 * memory through its own allocator (a search server that reserves the GPU's
 * memory at start-up), or latency-critical code that cannot afford the
 * implicit device-wide synchronisation of cudaMalloc / cudaFree. The paper
 * has no counterpart: this is a service of the library, not a step of the
 * method.
 *
 * Same arguments and results as gc_decode, without d_scratch: the scratch is
 * a fixed 128 KiB array inside the library, which every GPU that loads the
 * library holds until the process exits. It serves lists of at most
 * GC_DECODE_STATIC_MAX_INTS ints; a longer list returns GC_ERR_NOSPACE at
 * once (use gc_decode with caller scratch). The call allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the
 * life of the process; make that first call before any stream capture.
 * cudaDeviceReset unloads the library's device code, so the kept address is
 * no longer valid after it: do not call gc_decode_static on a device after
 * resetting it. Every call on a device shares the one array, and each call
 * clears what must start at zero before use: calls that overlap on the GPU
 * (on two streams, or from two threads) race and must be ordered by the
 * caller. */
#define GC_DECODE_STATIC_MAX_INTS (1u << 20)
gc_status gc_decode_static(const gc_codec* codec, const uint8_t* d_ctrl, uint64_t ctrl_bytes,
                           const uint32_t* d_data, uint64_t data_words, uint64_t n, const gc_tile* d_tiles,
                           uint32_t* d_out, int restore_docids, uint32_t* d_status, void* stream);

/* ----------------------------------------------- Variable Byte lists */

/* One list of Variable Byte bytes in a batch: its bytes at byte_off of the
 * byte pool (nbytes of them), its n numbers decoding to out_off of the
 * output. 24 bytes. */
typedef struct {
  uint64_t byte_off;
  uint64_t out_off;
  uint32_t n;
  uint32_t nbytes;
} gc_vb_list;

/* Scratch bytes gc_vb_encode_batch needs for nlists lists. */
gc_status gc_vb_encode_batch_scratch_size(uint64_t nlists, uint64_t* bytes);

/* Variable Byte (Sec 2.3), which the paper keeps for posting lists shorter
 * than 64 (Sec 7.5): each number in whole bytes, 7 bits per byte, most
 * significant group first, the high bit set on the number's last byte.
 * Encodes nlists lists at once: list i's d_n[i] gaps start at d_in_off[i]
 * of d_gaps (the caller guarantees they lie inside it); the lists' bytes go
 * back to back to d_bytes (bytes_cap bytes; at most 5 per number), their
 * records to d_lists (out_off = d_in_off[i]), and the total byte count to
 * *d_total (device). A batch larger than bytes_cap writes no list and
 * reports GC_ERR_NOSPACE in d_status. All arguments but the sizes are
 * device pointers; asynchronous on `stream`; the paper has no batch form. */
gc_status gc_vb_encode_batch(const uint32_t* d_gaps, const uint64_t* d_in_off, const uint32_t* d_n, uint64_t nlists,
                             gc_vb_list* d_lists, uint8_t* d_bytes, uint64_t bytes_cap, uint64_t* d_total,
                             void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status, void* stream);

/* Decodes the nlists lists of d_lists from the byte pool d_bytes
 * (bytes_len bytes) into d_out (out_len uint32): raw numbers, or each
 * list's docIDs (its own prefix sum, modulo 2^32) when restore_docids. A
 * record that points outside the pools reports GC_ERR_INVALID, a list whose
 * bytes end inside a number, hold a number wider than 32 bits or are left
 * over reports GC_ERR_CORRUPT (the list's list index in d_status[1]);
 * leading zero groups are accepted. A malformed list writes only inside its
 * own output range; the other lists decode as if it were absent. Lists
 * whose bytes lie back to back (as gc_vb_encode_batch writes them) decode
 * fastest: their warp splits their bytes evenly over its lanes. Asynchronous
 * on `stream`. */
gc_status gc_vb_decode_batch(const gc_vb_list* d_lists, uint64_t nlists, const uint8_t* d_bytes, uint64_t bytes_len,
                             uint32_t* d_out, uint64_t out_len, int restore_docids, uint32_t* d_status,
                             void* stream);

/* ------------------------------------------------------ AND queries */

/* Scratch bytes gc_intersect needs: a_ints = the sum of the a lists'
 * lengths, a_tiles and b_tiles = the sums of the a and b lists' tiles
 * (ceil(n / k) rows in tiles of 1024 / k rows). */
gc_status gc_intersect_scratch_size(uint64_t a_ints, uint64_t a_tiles, uint64_t b_tiles, uint64_t* bytes);

/* AND queries over a batch index (Sec 7.4: the lists of a query are decoded
 * and intersected, skip pointers letting the intersection pass over blocks
 * that cannot match). Query q returns the docIDs of list d_a[q] that are
 * also in list d_b[q], in increasing order. List a is decoded whole; of
 * list b only the tiles that can hold one of a's docIDs are decoded: tile
 * t >= 1 holds the docIDs above its skip entry (gc_tile.base, the docID
 * before the tile), so a docID x can only be in the last tile whose entry
 * is below x. Put the shorter list of a query in d_a.
 *   d_lists / nlists, d_tile_pool / tile_pool_len, d_ctrl_pool /
 *     ctrl_pool_bytes, d_data_pool / data_pool_words: the index, as for
 *     gc_decode_batch; every tile record of a b list must carry its skip
 *     entry (GC_TILE_BASE, which gc_encode_batch writes), else
 *     GC_ERR_UNSUPPORTED in d_status.
 *   d_a, d_b: nqueries list indices each, on the device.
 *   d_a_offs: nqueries uint64, exclusive prefix sums of the a lists'
 *     lengths: a's docIDs, and query q's results, start there.
 *   d_b_tile_offs: nqueries uint64, exclusive prefix sums of the b lists'
 *     tiles.
 *   a_ints, a_tiles, b_tiles: the totals gc_intersect_scratch_size takes.
 *   d_out: a_ints uint32, receives query q's results from d_a_offs[q] on.
 *   d_counts: nqueries uint32, receives each query's result count.
 *   d_scratch: gc_intersect_scratch_size bytes, 256-byte aligned. After
 *     the call its first 32 bytes hold four uint64: the a tiles decoded,
 *     those of them that took their prefix by look-back, the b tiles
 *     decoded, and those of them that took it by look-back.
 * A list index >= nlists gives GC_ERR_INVALID in d_status (and no results
 * for that query). Asynchronous on `stream`; no host synchronisation, so it
 * is graph-capturable. The paper's queries also rank; this call returns the
 * matching docIDs only. */
gc_status gc_intersect(const gc_codec* codec, const gc_list* d_lists, uint64_t nlists, const gc_tile* d_tile_pool,
                       uint64_t tile_pool_len, const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes,
                       const uint32_t* d_data_pool, uint64_t data_pool_words, const uint32_t* d_a,
                       const uint32_t* d_b, const uint64_t* d_a_offs, const uint64_t* d_b_tile_offs, uint64_t nqueries,
                       uint64_t a_ints, uint64_t a_tiles, uint64_t b_tiles, uint32_t* d_out, uint32_t* d_counts,
                       void* d_scratch, uint64_t scratch_bytes, uint32_t* d_status, void* stream);

/* ------------------------------------------- launch shapes and host buffers */

/* Register the launch shape that decode calls given launch = NULL use for
 * this codec kind and k, with or without docIDs, on the current device (the
 * autotuner does this after timing its candidates on an index); launch =
 * NULL clears it. Without one, NULL means the library default. A shape out
 * of range returns GC_ERR_INVALID. Not a step of the paper's method: a
 * service of the library. */
gc_status gc_set_launch(const gc_codec* codec, int restore_docids, const gc_launch* launch);

/* The shape a decode call with launch = NULL uses now on the current
 * device (registered, or the library default), every field filled in
 * (stage_bytes 0 = all the shared memory the block's share leaves). */
gc_status gc_get_launch(const gc_codec* codec, int restore_docids, gc_launch* launch);

/* Device bytes gc_decode_plan_host needs for a plan of nwork records over
 * pools of these sizes and an output pool of out_pool_len ints. */
gc_status gc_decode_plan_host_buffer_size(uint64_t nwork, uint64_t ctrl_pool_bytes, uint64_t data_pool_words,
                                          uint64_t out_pool_len, uint64_t* bytes);

/* gc_decode_plan for a caller whose plan, pools and output are in host
 * memory (the decode of Sec 4.3, 5.2.3, 6.2 and the prefix sum of Sec 2.1.1,
 * as gc_decode_plan). On `stream`: the nwork records of h_work (a plan
 * gc_plan_batch or gc_plan_select made, copied to the host) and both pools
 * are copied into d_buffers, the plan's counts are rebuilt there, the
 * output area is zeroed and decoded, and all out_pool_len ints of it are
 * copied back to h_out_pool (ints no record writes come back as 0).
 *   d_buffers / buffer_bytes: device memory, 256-byte aligned, at least
 *     gc_decode_plan_host_buffer_size bytes, owned by the caller; the call
 *     only uses it while the stream runs the call's work.
 *   launch: as for gc_decode_plan.
 *   d_status: device pointer, as for every decode call.
 * Asynchronous: the host buffers must stay alive and unchanged until the
 * stream reaches the end of the call's work, and copies overlap other work
 * only when the host buffers are page-locked (cudaHostAlloc). Errors as for
 * gc_decode_plan; GC_ERR_NOSPACE when buffer_bytes is too small. */
gc_status gc_decode_plan_host(const gc_codec* codec, const gc_work* h_work, uint64_t nwork, const uint8_t* h_ctrl_pool,
                              uint64_t ctrl_pool_bytes, const uint32_t* h_data_pool, uint64_t data_pool_words,
                              uint32_t* h_out_pool, uint64_t out_pool_len, int restore_docids, const gc_launch* launch,
                              void* d_buffers, uint64_t buffer_bytes, uint32_t* d_status, void* stream);

/* Drop the library's host-side state: the registered launch shapes and the
 * device facts and kernel attributes it looked up (call it after
 * cudaDeviceReset, before the next gc_* call). Safe whenever no other gc_*
 * call is running; later calls look up again what they need. The fixed
 * scratch of gc_decode_static is device memory of the library's code: it is
 * not released. */
void gc_shutdown(void);

/* Number of kernels the last gc_* call on this host thread launched (for
 * launch accounting). */
uint32_t gc_last_launch_count(void);

/* Library version string. */
const char* gc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GC_H */
