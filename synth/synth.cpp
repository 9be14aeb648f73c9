// Seeded synthetic posting-list generators.
//
// This module produces the inputs (d-gap sequences) that both the CPU oracle
// and the CUDA decode path consume. It contains none of the compression
// method's arithmetic: only random number generation, sampling and the d-gap
// transform of sorted docID lists (d-gap: Section 2.1.1).
//
// Random numbers: splitmix64 (seeding) and xoshiro256** (streams), both
// written from their published definitions (Steele/Lea/Flood 2014; Blackman &
// Vigna 2018). Bounded integers use Lemire's multiply-shift with rejection, so
// every integer draw is exact and platform independent. Draws that go through
// floating point (geometric, log-normal, Zipf lengths) use IEEE double and the
// C library's log/exp; they are reproducible on one machine, and no stored
// expected value depends on them.
//
// Per-list streams are seeded with splitmix64(seed ^ list_id), so the output
// never depends on the number of threads.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

inline uint64_t splitmix64_next(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

inline uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

struct Rng {
  uint64_t s[4];
  explicit Rng(uint64_t seed) {
    uint64_t sm = seed;
    for (int i = 0; i < 4; ++i) s[i] = splitmix64_next(sm);
  }
  uint64_t next() {
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
  }
  // Uniform integer in [0, range), range >= 1 (Lemire 2019, exact).
  uint64_t below(uint64_t range) {
    if (range <= 1) return 0;
    if (range <= 0xFFFFFFFFull) {
      uint32_t r = (uint32_t)range;
      uint64_t m = (uint64_t)(uint32_t)(next() >> 32) * r;
      uint32_t l = (uint32_t)m;
      if (l < r) {
        uint32_t t = (uint32_t)(-r) % r;
        while (l < t) {
          m = (uint64_t)(uint32_t)(next() >> 32) * r;
          l = (uint32_t)m;
        }
      }
      return m >> 32;
    }
    // 64-bit ranges: plain rejection on the next power of two.
    uint64_t mask = range - 1;
    mask |= mask >> 1; mask |= mask >> 2; mask |= mask >> 4;
    mask |= mask >> 8; mask |= mask >> 16; mask |= mask >> 32;
    uint64_t x;
    do { x = next() & mask; } while (x >= range);
    return x;
  }
  // Uniform double in (0, 1].
  double unit_open0() { return ((double)(next() >> 11) + 1.0) * (1.0 / 9007199254740992.0); }
  // Geometric on {1, 2, ...} with the given mean (p = 1/mean), by inversion.
  uint32_t geometric(double mean) {
    if (mean <= 1.0) return 1;
    const double p = 1.0 / mean;
    const double u = unit_open0();
    double g = std::floor(std::log(u) / std::log1p(-p));
    if (g > 4.0e9) g = 4.0e9;
    return 1u + (uint32_t)g;
  }
  // Standard normal (Box-Muller, cosine branch).
  double normal() {
    const double u1 = unit_open0();
    const double u2 = unit_open0();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

uint64_t list_seed(uint64_t seed, uint64_t list_id) {
  uint64_t s = seed ^ (list_id * 0xD1B54A32D192ED03ull + 0x8CB92BA72F3D8DD7ull);
  return splitmix64_next(s);
}

// Run fn(i) for i in [0, count) on nthreads workers, dynamic chunks.
template <class F>
void parallel_for(uint64_t count, int nthreads, uint64_t chunk, F fn) {
  if (nthreads <= 1 || count <= chunk) {
    for (uint64_t i = 0; i < count; ++i) fn(i);
    return;
  }
  std::atomic<uint64_t> next{0};
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) {
    pool.emplace_back([&]() {
      for (;;) {
        uint64_t b = next.fetch_add(chunk);
        if (b >= count) break;
        uint64_t e = std::min(count, b + chunk);
        for (uint64_t i = b; i < e; ++i) fn(i);
      }
    });
  }
  for (auto& th : pool) th.join();
}

// Sorted uniform sample of L distinct values from [0, U), written as d-gaps
// (first element kept as is). The set is the first L distinct values of an
// i.i.d. uniform sequence, which is a uniform L-subset.
void sorted_sample_gaps(Rng& rng, uint64_t L, uint64_t U, uint32_t* out) {
  if (L == 0) return;
  if (L > U) L = U;
  std::vector<uint32_t> v;
  if (L * 64 >= U) {
    // Dense: bitmap over the universe. Pick the complement when L > U/2.
    const bool complement = L * 2 > U;
    const uint64_t want = complement ? U - L : L;
    std::vector<uint64_t> bm((U + 63) / 64, 0);
    uint64_t have = 0;
    while (have < want) {
      uint64_t x = rng.below(U);
      uint64_t& w = bm[x >> 6];
      uint64_t bit = 1ull << (x & 63);
      if (!(w & bit)) { w |= bit; ++have; }
    }
    v.reserve(L);
    for (uint64_t i = 0; i < bm.size(); ++i) {
      uint64_t w = complement ? ~bm[i] : bm[i];
      if (i == bm.size() - 1 && (U & 63)) w &= (1ull << (U & 63)) - 1;
      while (w) {
        int b = __builtin_ctzll(w);
        v.push_back((uint32_t)(i * 64 + b));
        w &= w - 1;
      }
    }
  } else {
    v.reserve(L + 16);
    for (uint64_t i = 0; i < L; ++i) v.push_back((uint32_t)rng.below(U));
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    while (v.size() < L) {
      const uint64_t missing = L - v.size();
      for (uint64_t i = 0; i < missing; ++i) v.push_back((uint32_t)rng.below(U));
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
    }
  }
  uint32_t prev = 0;
  for (uint64_t i = 0; i < L; ++i) {
    out[i] = (i == 0) ? v[0] : v[i] - prev;
    prev = v[i];
  }
}

// Clustered docIDs: runs of consecutive documents (run length geometric with
// mean run_mean) separated by geometric jumps (mean jump_mean). Starts at
// docID jump-1. Stops before a docID would reach U. Returns the count written.
uint64_t clustered_gaps(Rng& rng, uint64_t L, uint64_t U, double run_mean, double jump_mean,
                        uint32_t* out) {
  uint64_t written = 0;
  uint64_t doc = (uint64_t)rng.geometric(jump_mean) - 1;
  uint64_t prev = 0;
  bool first = true;
  while (written < L && doc < U) {
    uint64_t run = rng.geometric(run_mean);
    for (uint64_t r = 0; r < run && written < L && doc < U; ++r) {
      out[written++] = first ? (uint32_t)doc : (uint32_t)(doc - prev);
      first = false;
      prev = doc;
      doc += 1;
    }
    doc += rng.geometric(jump_mean) - 1;
  }
  return written;
}

}  // namespace

extern "C" {

// Raw xoshiro256** outputs (lets tests check the generator against its
// published definition).
void synth_raw_u64(uint64_t seed, uint64_t count, uint64_t* out) {
  Rng rng(seed);
  for (uint64_t i = 0; i < count; ++i) out[i] = rng.next();
}

// n gaps, each geometric on {1,2,...} with the given mean.
void synth_geometric_gaps(uint64_t seed, uint64_t n, double mean, uint32_t* out) {
  Rng rng(seed);
  for (uint64_t i = 0; i < n; ++i) out[i] = rng.geometric(mean);
}

// n gaps in runs of run_len: a fraction frac_uniform of the runs (chosen by a
// Fisher-Yates shuffle of run kinds) is uniform in [1, umax], the rest is
// geometric with mean geo_mean.
void synth_mixed_runs(uint64_t seed, uint64_t n, uint32_t run_len, double geo_mean,
                      double frac_uniform, uint32_t umax, uint32_t* out) {
  Rng rng(seed);
  const uint64_t nruns = (n + run_len - 1) / run_len;
  std::vector<uint8_t> kind(nruns, 0);
  const uint64_t nuni = (uint64_t)std::llround(frac_uniform * (double)nruns);
  for (uint64_t i = 0; i < nuni && i < nruns; ++i) kind[i] = 1;
  for (uint64_t i = nruns; i > 1; --i) {
    uint64_t j = rng.below(i);
    std::swap(kind[i - 1], kind[j]);
  }
  for (uint64_t r = 0; r < nruns; ++r) {
    const uint64_t b = r * run_len, e = std::min<uint64_t>(n, b + run_len);
    for (uint64_t i = b; i < e; ++i)
      out[i] = kind[r] ? (uint32_t)(1 + rng.below(umax)) : rng.geometric(geo_mean);
  }
}

// Rank-law list lengths L_r = clamp(round(C * r^-s), 1, cap), r = 1..nlists,
// then shuffled (Fisher-Yates). Returns the sum.
uint64_t synth_zipf_lengths(uint64_t seed, uint64_t nlists, double C, double s, uint64_t cap,
                            uint32_t* out) {
  uint64_t total = 0;
  for (uint64_t r = 1; r <= nlists; ++r) {
    double x = std::nearbyint(C * std::pow((double)r, -s));
    uint64_t L = x < 1.0 ? 1 : (x > (double)cap ? cap : (uint64_t)x);
    out[r - 1] = (uint32_t)L;
    total += L;
  }
  Rng rng(seed);
  for (uint64_t i = nlists; i > 1; --i) {
    uint64_t j = rng.below(i);
    std::swap(out[i - 1], out[j]);
  }
  return total;
}

// Log-normal lengths round(exp(ln(median) + sigma * Z)), at least 1.
uint64_t synth_lognormal_lengths(uint64_t seed, uint64_t nlists, double median, double sigma,
                                 uint64_t cap, uint32_t* out) {
  uint64_t total = 0;
  for (uint64_t i = 0; i < nlists; ++i) {
    Rng rng(list_seed(seed, i));
    double x = std::nearbyint(std::exp(std::log(median) + sigma * rng.normal()));
    uint64_t L = x < 1.0 ? 1 : (x > (double)cap ? cap : (uint64_t)x);
    out[i] = (uint32_t)L;
    total += L;
  }
  return total;
}

// Index of uniform lists: list i is a sorted uniform sample without
// replacement of lengths[i] docIDs from [0, U), written as d-gaps at
// out + offsets[i].
void synth_uniform_index(uint64_t seed, uint64_t nlists, const uint32_t* lengths,
                         const uint64_t* offsets, uint64_t U, uint32_t* out, int nthreads) {
  parallel_for(nlists, nthreads, 256, [&](uint64_t i) {
    Rng rng(list_seed(seed, i));
    sorted_sample_gaps(rng, lengths[i], U, out + offsets[i]);
  });
}

// Clustered index: list i draws up to max_len[i] docIDs (clustered runs) and
// stops early at the universe end. Pass out == nullptr to only compute the
// actual lengths (written to actual[i]); otherwise gaps go to out + offsets[i].
void synth_clustered_index(uint64_t seed, uint64_t nlists, const uint32_t* max_len,
                           const uint64_t* offsets, uint64_t U, double run_mean,
                           double jump_mean, uint32_t* actual, uint32_t* out, int nthreads) {
  parallel_for(nlists, nthreads, 1024, [&](uint64_t i) {
    Rng rng(list_seed(seed, i) ^ 0x5bd1e995ull);
    std::vector<uint32_t> tmp;
    uint32_t* dst;
    if (out) {
      dst = out + offsets[i];
    } else {
      tmp.resize(max_len[i]);
      dst = tmp.data();
    }
    uint64_t w = clustered_gaps(rng, max_len[i], U, run_mean, jump_mean, dst);
    if (actual) actual[i] = (uint32_t)w;
  });
}

// Uniform integers in [lo, hi] (inclusive), for random-stream tests.
void synth_uniform_u32(uint64_t seed, uint64_t n, uint32_t lo, uint32_t hi, uint32_t* out) {
  Rng rng(seed);
  const uint64_t range = (uint64_t)hi - lo + 1;
  for (uint64_t i = 0; i < n; ++i) out[i] = lo + (uint32_t)rng.below(range);
}

// Values with a controlled bit-width mix: each value has a width drawn
// uniformly from [wlo, whi] (0 allowed) and is uniform below 2^width.
void synth_width_mix(uint64_t seed, uint64_t n, uint32_t wlo, uint32_t whi, uint32_t* out) {
  Rng rng(seed);
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t w = wlo + (uint32_t)rng.below((uint64_t)whi - wlo + 1);
    out[i] = w == 0 ? 0u : (w >= 32 ? (uint32_t)rng.next() : (uint32_t)rng.below(1ull << w));
  }
}

// Term frequencies of an index: list i's lengths[i] values, each >= 1 and
// geometric with the given mean, at out + offsets[i] (one stream per list,
// so the values do not depend on the layout or the thread count).
void synth_tf_index(uint64_t seed, uint64_t nlists, const uint32_t* lengths, const uint64_t* offsets,
                    double mean, uint32_t* out, int nthreads) {
  parallel_for(nlists, nthreads, 256, [&](uint64_t i) {
    Rng rng(list_seed(seed, i) ^ 0x2545f491ull);
    uint32_t* dst = out + offsets[i];
    for (uint32_t t = 0; t < lengths[i]; ++t) dst[t] = rng.geometric(mean);
  });
}

}  // extern "C"
