// gc_host.h -- host-side helpers of the Group-codec library (validation,
// sizes, launch accounting). Internal; the public ABI is include/gc.h.
#pragma once

#include <cstdint>

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

}  // namespace gc_host
