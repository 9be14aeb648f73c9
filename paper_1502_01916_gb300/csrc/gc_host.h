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

}  // namespace gc_host
