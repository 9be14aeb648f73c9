// gc_host.h -- host-side helpers of the Group-codec library (validation,
// sizes, launch accounting, the tile-index build shared by the decoders).
// Internal; the public ABI is include/gc.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gc.h"

namespace gc_host {

inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// GC_OK for a codec the library serves, GC_ERR_INVALID otherwise.
gc_status check_codec(const gc_codec* c);

// Multiprocessors of the current device (cached per device).
int sm_count();
// Forget the device facts looked up so far (gc_shutdown).
void forget_devices();

// Kernel launches made by the current gc_* call on this thread.
void reset_launches();
void count_launch(uint32_t n = 1);
uint32_t launches();

// Scratch bytes (chunk sums) of the tile-index build of a list of n ints.
uint64_t index_sums_bytes(const gc_codec& c, uint64_t n);

// The tile index of one list from its control area (gc_index.cu): writes
// the list's ntiles records to d_tiles, using d_sums as scratch.
gc_status build_tiles(const gc_codec& c, const uint8_t* d_ctrl, uint64_t ctrl_bytes, uint64_t n, gc_tile* d_tiles,
                      void* d_sums, uint32_t* d_status, cudaStream_t s);

// The rest of a work plan whose records the caller has written, (list,
// tile) each, `list` an index into d_sel / d_outs: fills every record
// below count[0] as gc_plan_select fills its own (list d_lists[d_sel[list]],
// output at d_outs[list] + 1024 * tile; records past count[0] are left).
gc_status plan_fill(const gc_codec& c, const gc_list* d_lists, uint64_t nlists, const uint32_t* d_sel,
                    const uint64_t* d_outs, uint64_t nsel, const gc_tile* d_tiles, uint64_t ntiles,
                    const uint8_t* d_ctrl_pool, uint64_t ctrl_pool_bytes, gc_work* d_work, uint64_t cap,
                    uint64_t* d_count, uint32_t* d_status, cudaStream_t s);

}  // namespace gc_host
