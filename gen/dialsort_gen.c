/*
 * Seeded synthetic key generators shared by the CPU oracle tests, the GPU
 * parity tests and the benchmark.  Nothing here counts, scans or expands a
 * histogram: this file only draws keys.
 *
 * Randomness: a counter-based SplitMix64 stream (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014).  Draw i of
 * stream (seed, stream) is mix(key + (i + 1) * gamma), so any element can be
 * produced independently of the others.
 *
 * Distributions (the shapes of the paper's workloads, Sec. "Distributions",
 * plus the Zipf and run shapes of the scale workloads):
 *   GEN_UNIFORM     i.i.d. uniform on [0, U)
 *   GEN_ZIPF        P(k) proportional to (k + 1)^(-s), hot bin = key 0
 *   GEN_ALL_EQUAL   every key equals `value`
 *   GEN_SORTED      a sorted uniform sample, drawn directly as uniform order
 *                   statistics (normalised prefix sums of exponential
 *                   spacings), so no sort is needed to make it
 *   GEN_REVERSE     GEN_SORTED reversed
 *   GEN_RUNS        consecutive blocks of `run_len` keys, each an independent
 *                   sorted sample, ascending and descending in turn
 *   GEN_PAPER_SKEW  80 % uniform on [0, floor(0.05 U)] (inclusive), 20 %
 *                   uniform on [0, U)
 *   GEN_ZIPF_PERM   GEN_ZIPF with ranks mapped through a seeded bijection of
 *                   [0, U), so hot keys are scattered over the universe
 *
 * Floating point is used only to shape distributions.  Build with
 * -ffp-contract=off; results are reproducible on one machine, and the tests
 * never compare generator output across machines.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  GEN_UNIFORM = 0,
  GEN_ZIPF = 1,
  GEN_ALL_EQUAL = 2,
  GEN_SORTED = 3,
  GEN_REVERSE = 4,
  GEN_RUNS = 5,
  GEN_PAPER_SKEW = 6,
  GEN_ZIPF_PERM = 7,
};

static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static const uint64_t GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t gen_stream_key(uint64_t seed, uint64_t stream) {
  return sm64_mix(seed ^ sm64_mix(stream * GAMMA + 0x632BE59BD9B4E019ULL));
}

static inline uint64_t draw64(uint64_t key, uint64_t i) { return sm64_mix(key + (i + 1) * GAMMA); }

/* uniform integer in [0, m) from the high 32 bits (multiply-shift), m <= 2^32 */
static inline uint64_t below(uint64_t r, uint64_t m) { return ((r >> 32) * m) >> 32; }

/* uniform double in [0, 1) with 53 random bits */
static inline double unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* raw 64-bit draws, for callers that need plain random words */
void gen_u64(uint64_t* out, uint64_t n, uint64_t seed, uint64_t stream) {
  uint64_t key = gen_stream_key(seed, stream);
  for (uint64_t i = 0; i < n; ++i) out[i] = draw64(key, i);
}

/* uniform doubles in [0, 1) */
void gen_unit(double* out, uint64_t n, uint64_t seed, uint64_t stream) {
  uint64_t key = gen_stream_key(seed, stream);
  for (uint64_t i = 0; i < n; ++i) out[i] = unit(draw64(key, i));
}

/* ---- Zipf by table inversion with a guide table (Chen and Asau, 1974) ---- */
typedef struct {
  double* cdf;     /* cdf[k] = P(key <= k), cdf[U-1] = 1 */
  uint32_t* guide; /* guide[j] = smallest k with cdf[k] > j / m */
  uint64_t m;
  uint32_t U;
} zipf_table;

static int zipf_build(zipf_table* t, uint32_t U, double s) {
  t->U = U;
  t->m = U;
  t->cdf = (double*)malloc(sizeof(double) * (size_t)U);
  t->guide = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(t->m + 1));
  if (!t->cdf || !t->guide) {
    free(t->cdf);
    free(t->guide);
    return -1;
  }
  double acc = 0.0;
  for (uint32_t k = 0; k < U; ++k) {
    acc += pow((double)k + 1.0, -s);
    t->cdf[k] = acc;
  }
  for (uint32_t k = 0; k < U; ++k) t->cdf[k] /= acc;
  t->cdf[U - 1] = 1.0;
  uint32_t k = 0;
  for (uint64_t j = 0; j <= t->m; ++j) {
    double u = (double)j / (double)t->m;
    while (k < U - 1 && t->cdf[k] <= u) ++k;
    t->guide[j] = k;
  }
  return 0;
}

static inline uint32_t zipf_draw(const zipf_table* t, double u) {
  uint64_t j = (uint64_t)(u * (double)t->m);
  if (j > t->m) j = t->m;
  uint32_t k = t->guide[j];
  while (t->cdf[k] <= u) ++k; /* cdf[U-1] = 1 > u stops the walk */
  return k;
}

static void zipf_free(zipf_table* t) {
  free(t->cdf);
  free(t->guide);
}

/* a seeded bijection of [0, U): x -> (a * x + b) mod U with gcd(a, U) = 1 */
static uint64_t gcd64(uint64_t a, uint64_t b) {
  while (b) {
    uint64_t r = a % b;
    a = b;
    b = r;
  }
  return a;
}

/* sorted uniform sample of length len on [0, U), via exponential spacings */
static void sorted_block(uint64_t len, uint32_t U, uint64_t key, uint64_t first_draw, int descending,
                         void* out, int key_bytes) {
  double total = 0.0;
  for (uint64_t i = 0; i <= len; ++i) total += -log1p(-unit(draw64(key, first_draw + i)));
  double acc = 0.0;
  for (uint64_t i = 0; i < len; ++i) {
    acc += -log1p(-unit(draw64(key, first_draw + i)));
    double c = acc / total;
    uint64_t v = (uint64_t)(c * (double)U);
    if (v >= U) v = U - 1;
    uint64_t pos = descending ? (len - 1 - i) : i;
    if (key_bytes == 4)
      ((uint32_t*)out)[pos] = (uint32_t)v;
    else
      ((uint16_t*)out)[pos] = (uint16_t)v;
  }
}

/*
 * Fill out[0..n) (uint32 when key_bytes == 4, uint16 when 2) with keys in
 * [0, U).  param: Zipf exponent for GEN_ZIPF / GEN_ZIPF_PERM, the key for
 * GEN_ALL_EQUAL, the block length for GEN_RUNS (0 means 2^20).
 * Returns 0 on success, -1 on bad arguments, -2 when out of host memory.
 */
int gen_keys(void* out, uint64_t n, uint32_t U, int key_bytes, int dist, double param, uint64_t seed,
             uint64_t stream) {
  if (U == 0 || (key_bytes != 4 && key_bytes != 2)) return -1;
  if (key_bytes == 2 && U > 65536u) return -1;
  uint64_t key = gen_stream_key(seed, stream);
#define PUT(i, v)                                  \
  do {                                             \
    if (key_bytes == 4)                            \
      ((uint32_t*)out)[i] = (uint32_t)(v);         \
    else                                           \
      ((uint16_t*)out)[i] = (uint16_t)(v);         \
  } while (0)
  switch (dist) {
    case GEN_UNIFORM:
      for (uint64_t i = 0; i < n; ++i) PUT(i, below(draw64(key, i), U));
      return 0;
    case GEN_ALL_EQUAL: {
      uint64_t v = (uint64_t)param;
      if (param < 0 || v >= U) return -1;
      for (uint64_t i = 0; i < n; ++i) PUT(i, v);
      return 0;
    }
    case GEN_PAPER_SKEW: {
      uint64_t hot = (uint64_t)floor(0.05 * (double)U) + 1; /* [0, floor(0.05U)] inclusive */
      if (hot > U) hot = U;
      for (uint64_t i = 0; i < n; ++i) {
        uint64_t r = draw64(key, i);
        uint64_t pick = draw64(key ^ 0xA5A5A5A5A5A5A5A5ULL, i);
        PUT(i, (below(pick, 10) < 8) ? below(r, hot) : below(r, U));
      }
      return 0;
    }
    case GEN_ZIPF:
    case GEN_ZIPF_PERM: {
      if (!(param > 0.0)) return -1;
      zipf_table t;
      if (zipf_build(&t, U, param) != 0) return -2;
      uint64_t a = 1, b = 0;
      if (dist == GEN_ZIPF_PERM && U > 1) {
        uint64_t r = draw64(key ^ 0x5EEDULL, 0);
        a = (r % U) | 1;
        while (gcd64(a, U) != 1) a = (a + 2) % U;
        b = draw64(key ^ 0x5EEDULL, 1) % U;
      }
      for (uint64_t i = 0; i < n; ++i) {
        uint64_t k = zipf_draw(&t, unit(draw64(key, i)));
        if (dist == GEN_ZIPF_PERM) k = (a * k + b) % U;
        PUT(i, k);
      }
      zipf_free(&t);
      return 0;
    }
    case GEN_SORTED:
    case GEN_REVERSE:
      sorted_block(n, U, key, 0, dist == GEN_REVERSE, out, key_bytes);
      return 0;
    case GEN_RUNS: {
      uint64_t run = param > 0 ? (uint64_t)param : (1ULL << 20);
      uint64_t b = 0;
      for (uint64_t s = 0; s < n; s += run, ++b) {
        uint64_t len = (n - s < run) ? n - s : run;
        char* base = (char*)out + s * (uint64_t)key_bytes;
        sorted_block(len, U, key, s + b, (int)(b & 1), base, key_bytes);
      }
      return 0;
    }
    default:
      return -1;
  }
#undef PUT
}

/* log-uniform integers: floor(2^(lo + (hi - lo) u)), clamped to [2^lo, 2^hi] */
void gen_loguniform(uint64_t* out, uint64_t count, double lo, double hi, uint64_t seed, uint64_t stream) {
  uint64_t key = gen_stream_key(seed, stream);
  double vlo = ldexp(1.0, (int)lo), vhi = ldexp(1.0, (int)hi);
  for (uint64_t i = 0; i < count; ++i) {
    double v = floor(pow(2.0, lo + (hi - lo) * unit(draw64(key, i))));
    if (v < vlo) v = vlo;
    if (v > vhi) v = vhi;
    out[i] = (uint64_t)v;
  }
}
