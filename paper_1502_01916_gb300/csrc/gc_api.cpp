// gc_api.cpp -- host entry points of the Group-codec library that launch no
// kernel: codec validation, size bounds, the zeta rule of Group-PFD.
#include <cmath>
#include <cuda_runtime.h>

#include "gc.h"
#include "gc_host.h"

namespace gc_host {

namespace {
thread_local uint32_t t_launches = 0;
int g_sms[64] = {0};
}  // namespace

gc_status check_codec(const gc_codec* c) {
  if (!c) return GC_ERR_INVALID;
  if (c->k != 4 && c->k != 32) return GC_ERR_INVALID;
  if (c->reserved != 0) return GC_ERR_INVALID;
  switch (c->kind) {
    case GC_SIMPLE:
    case GC_AFOR:
      return GC_OK;
    case GC_SCHEME:
      if (c->cg != 1 && c->cg != 2 && c->cg != 4 && c->cg != 8) return GC_ERR_INVALID;
      if (c->ld > GC_LD_IU) return GC_ERR_INVALID;
      if (c->ld == GC_LD_IU && c->cg < 4) return GC_ERR_INVALID;  // Sec 5.2.1(a)
      return GC_OK;
    case GC_PFD:
      return c->pfd_exc_rows < 32 ? GC_OK : GC_ERR_INVALID;
    default:
      return GC_ERR_INVALID;
  }
}

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (g_sms[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_sms[dev] = v > 0 ? v : 1;
  }
  return g_sms[dev];
}

void forget_devices() {
  for (int& v : g_sms) v = 0;
}

void reset_launches() { t_launches = 0; }
void count_launch(uint32_t n) { t_launches += n; }
uint32_t launches() { return t_launches; }

}  // namespace gc_host

extern "C" {

uint32_t gc_pfd_rows_for_zeta(double zeta) {
  // the largest c with c / 32 < zeta
  double c = std::ceil(zeta * 32.0) - 1.0;
  if (c < 0.0) c = 0.0;
  if (c > 31.0) c = 31.0;
  return (uint32_t)c;
}

gc_status gc_max_encoded_size(const gc_codec* codec, uint64_t n, uint64_t* ctrl_cap, uint64_t* data_cap,
                              uint64_t* ntiles) {
  gc_status st = gc_host::check_codec(codec);
  if (st != GC_OK) return st;
  const uint64_t k = codec->k;
  const uint64_t R = (n + k - 1) / k;
  const uint64_t tr = 1024 / k;
  uint64_t cc = 0, dc = 0;
  switch (codec->kind) {
    case GC_SIMPLE:  // at most one selector (one vector) per row
      cc = (R + 1) / 2;
      dc = R * k;
      break;
    case GC_SCHEME: {
      const uint64_t cg = codec->cg;
      if (codec->ld == GC_LD_BINARY) cc = cg == 1 ? 2 * ((R + 2) / 3) : cg == 8 ? (R + 3) / 4 : (R + 1) / 2;
      else if (codec->ld == GC_LD_CU) cc = (R * (32 / cg) + 7) / 8;
      else cc = R;  // IU: at worst one descriptor per byte
      dc = R * k;
      break;
    }
    case GC_AFOR: {
      const uint64_t R8 = (R + 7) / 8 * 8;
      cc = R8 / 8;
      dc = R8 * k;
      break;
    }
    default: {
      const uint64_t nf = (R + 31) / 32;
      const uint64_t pb = (32 * k) <= 256 ? 1 : 2;
      cc = 4 * nf + nf * (uint64_t)codec->pfd_exc_rows * k * (pb + 4);
      dc = R * k;
      break;
    }
  }
  // the encoders OR bits into the control area with aligned 32-bit atomics,
  // so the bound is kept a multiple of 4 bytes
  if (ctrl_cap) *ctrl_cap = gc_host::align_up(cc, 4);
  if (data_cap) *data_cap = dc;
  if (ntiles) *ntiles = (R + tr - 1) / tr;
  return GC_OK;
}

uint32_t gc_last_launch_count(void) { return gc_host::launches(); }

const char* gc_version(void) { return "gc 0.1 (sm_103a)"; }

}  // extern "C"
