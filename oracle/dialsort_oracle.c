/*
 * DialSort CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of what the DialSort hot path
 * computes, written from the paper's definitions.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Paper: A. Narvaez, "DialSort: Non-Comparative Integer Sorting via the
 * Self-Indexing Principle" (2026).
 *
 *   oracle_histogram_*   Eq. (1), ingestion: H initialised to zero, then
 *                        H[x] <- H[x] + 1 for every key x of K
 *                        (Sec. "Mathematical Formulation, Correctness, and
 *                        Ordered Projection"; zeroing is the Theta(U) term of
 *                        Theorem "Sequential complexity").
 *   oracle_reconstruct_* Eq. (2), ordered projection: for k = 0..U-1 emit k
 *                        exactly H[k] times.
 *   oracle_offsets       where each k's run starts in the projection of
 *                        Eq. (2): O[k] = sum_{j<k} H[j] (the cursor position
 *                        of the sequential projection when it reaches k).
 *   oracle_crn_level     one level of Definition "CRN level transition"
 *                        (node rule Eqs. (3)-(4)): adjacent items paired,
 *                        equal keys merged additively, distinct keys and an
 *                        odd residual forwarded unchanged.
 *   oracle_crn           ceil(log2 k) such levels applied in turn.
 *   oracle_accumulate_*  Eq. (1) without the zeroing: H[x] <- H[x] + 1 on an
 *                        H that already holds counts (ingesting a stream of
 *                        batches into one histogram).
 *   oracle_sort_mapped   Prop. "General Self-Indexing Principle": count
 *                        each key at index phi(key), then emit
 *                        phi_inv(i) H[i] times for i = 0..U-1.
 *   oracle_radix_sort    DialSort-Radix (Sec. "Full int32 range"): four
 *                        stable counting passes over the base-256 digits,
 *                        least significant first.
 *   oracle_frequency,    the queries of Sec. "Canonical ordered state",
 *   oracle_presence,     answered from H alone: frequency(k) = H[k],
 *   oracle_range_count   presence(k) = [H[k] > 0], range-count(a, b) =
 *                        sum of H[k] for a <= k <= b.
 *
 * Keys outside [0, U) are not defined by the paper; the oracle does not count
 * them and returns how many it skipped.
 */
#include <stdint.h>
#include <stddef.h>

/* Eq. (1): zero H, then one increment per key. Returns the number of keys >= U. */
uint64_t oracle_histogram_u32(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H) {
  for (uint64_t k = 0; k < U; ++k) H[k] = 0;
  uint64_t skipped = 0;
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t x = keys[i];
    if (x < U)
      H[x] = H[x] + 1;
    else
      skipped = skipped + 1;
  }
  return skipped;
}

uint64_t oracle_histogram_u16(const uint16_t* keys, uint64_t n, uint32_t U, uint32_t* H) {
  for (uint64_t k = 0; k < U; ++k) H[k] = 0;
  uint64_t skipped = 0;
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t x = keys[i];
    if (x < U)
      H[x] = H[x] + 1;
    else
      skipped = skipped + 1;
  }
  return skipped;
}

/*
 * Eq. (2): for k = 0, 1, ..., U-1 emit k exactly H[k] times.  Writes at most
 * `cap` keys into out and returns the total number emitted (sum of H), so a
 * caller can tell when out was too small.
 */
uint64_t oracle_reconstruct_u32(const uint32_t* H, uint32_t U, uint32_t* out, uint64_t cap) {
  uint64_t pos = 0;
  for (uint64_t k = 0; k < U; ++k) {
    for (uint64_t j = 0; j < H[k]; ++j) {
      if (pos < cap) out[pos] = (uint32_t)k;
      pos = pos + 1;
    }
  }
  return pos;
}

uint64_t oracle_reconstruct_u16(const uint32_t* H, uint32_t U, uint16_t* out, uint64_t cap) {
  uint64_t pos = 0;
  for (uint64_t k = 0; k < U; ++k) {
    for (uint64_t j = 0; j < H[k]; ++j) {
      if (pos < cap) out[pos] = (uint16_t)k;
      pos = pos + 1;
    }
  }
  return pos;
}

/* The cursor of the sequential projection on reaching k: O[k] = sum_{j<k} H[j], O[U] = sum H. */
void oracle_offsets(const uint32_t* H, uint32_t U, uint64_t* O) {
  uint64_t cursor = 0;
  for (uint64_t k = 0; k < U; ++k) {
    O[k] = cursor;
    cursor = cursor + H[k];
  }
  O[U] = cursor;
}

/*
 * One CRN level (Definition "CRN level transition"): the m items
 * (key_in[i], cnt_in[i]) are grouped into consecutive pairs (0,1), (2,3), ...
 * A pair with equal keys becomes one item (key, c1 + c2) (Eq. (3)); a pair
 * with distinct keys is forwarded unchanged (Eq. (4)); when m is odd the last
 * item is forwarded unchanged.  Returns the number of items written to the
 * output arrays (at most m).  Only equality between keys is evaluated.
 */
size_t oracle_crn_level(const uint32_t* key_in, const uint64_t* cnt_in, size_t m, uint32_t* key_out,
                        uint64_t* cnt_out) {
  size_t w = 0;
  size_t i = 0;
  for (; i + 1 < m; i += 2) {
    if (key_in[i] == key_in[i + 1]) {
      key_out[w] = key_in[i];
      cnt_out[w] = cnt_in[i] + cnt_in[i + 1];
      w = w + 1;
    } else {
      key_out[w] = key_in[i];
      cnt_out[w] = cnt_in[i];
      w = w + 1;
      key_out[w] = key_in[i + 1];
      cnt_out[w] = cnt_in[i + 1];
      w = w + 1;
    }
  }
  if (i < m) { /* odd residual */
    key_out[w] = key_in[i];
    cnt_out[w] = cnt_in[i];
    w = w + 1;
  }
  return w;
}

/*
 * The whole network for k = m lanes: L = ceil(log2 m) levels applied in turn.
 * key/cnt hold the lane states on entry and the surviving items on return;
 * scratch_key/scratch_cnt must hold m entries.  Returns the number of
 * surviving items.
 */
size_t oracle_crn(uint32_t* key, uint64_t* cnt, size_t m, uint32_t* scratch_key, uint64_t* scratch_cnt) {
  size_t levels = 0;
  while (((size_t)1 << levels) < m) levels = levels + 1;
  size_t cur = m;
  for (size_t l = 0; l < levels; ++l) {
    size_t next = oracle_crn_level(key, cnt, cur, scratch_key, scratch_cnt);
    for (size_t i = 0; i < next; ++i) {
      key[i] = scratch_key[i];
      cnt[i] = scratch_cnt[i];
    }
    cur = next;
  }
  return cur;
}

/* Eq. (1) without the zeroing: one increment per key into an H that already holds counts. */
uint64_t oracle_accumulate_u32(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H) {
  uint64_t skipped = 0;
  for (uint64_t i = 0; i < n; ++i) {
    if (keys[i] < U)
      H[keys[i]] = H[keys[i]] + 1;
    else
      skipped = skipped + 1;
  }
  return skipped;
}

uint64_t oracle_accumulate_u16(const uint16_t* keys, uint64_t n, uint32_t U, uint32_t* H) {
  uint64_t skipped = 0;
  for (uint64_t i = 0; i < n; ++i) {
    if (keys[i] < U)
      H[keys[i]] = H[keys[i]] + 1;
    else
      skipped = skipped + 1;
  }
  return skipped;
}

/* frequency(k) = H[k]; a k outside [0, U) was never counted, so its frequency is 0. */
void oracle_frequency(const uint32_t* H, uint32_t U, const uint32_t* q, uint64_t m, uint32_t* freq) {
  for (uint64_t i = 0; i < m; ++i) freq[i] = q[i] < U ? H[q[i]] : 0;
}

/* presence(k) = 1 when k occurs at least once, else 0. */
void oracle_presence(const uint32_t* H, uint32_t U, const uint32_t* q, uint64_t m, uint8_t* present) {
  for (uint64_t i = 0; i < m; ++i) present[i] = (q[i] < U && H[q[i]] > 0) ? 1 : 0;
}

/* range-count(a, b) = sum of H[k] over a <= k <= b, k < U; one pass over the b - a + 1 cells. */
void oracle_range_count(const uint32_t* H, uint32_t U, const uint32_t* a, const uint32_t* b, uint64_t m,
                        uint64_t* count) {
  for (uint64_t i = 0; i < m; ++i) {
    uint64_t sum = 0;
    for (uint64_t k = a[i]; k <= b[i] && k < U; ++k) sum = sum + H[k];
    count[i] = sum;
  }
}

/*
 * DialSort-Radix (Sec. "Full int32 range"): LSD radix sort in base 256.  Pass
 * p = 0..3 looks at digit d = (x >> 8p) & 255 only: H = histogram of the digit
 * (Eq. (1) with U = 256), the cursor of digit d starts at the sum of H below d
 * (the cursor of the projection of Eq. (2)), and keys are placed at
 * cursor[d]++ in their current order, so each pass is stable and after the
 * fourth the keys are sorted.  With is_signed the keys are two's complement
 * int32: the top digit's sign bit is flipped, putting negative keys first.
 * out and tmp hold n keys each; out may equal keys.
 */
void oracle_radix_sort(const uint32_t* keys, uint64_t n, int is_signed, uint32_t* out, uint32_t* tmp) {
  const uint32_t* src = keys;
  for (int pass = 0; pass < 4; ++pass) {
    uint32_t* dst = (pass % 2 == 0) ? tmp : out;
    uint64_t H[256];
    uint64_t cursor[256];
    for (int d = 0; d < 256; ++d) H[d] = 0;
    for (uint64_t i = 0; i < n; ++i) {
      uint32_t d = (src[i] >> (8 * pass)) & 255u;
      if (is_signed && pass == 3) d = d ^ 0x80u;
      H[d] = H[d] + 1;
    }
    uint64_t c = 0;
    for (int d = 0; d < 256; ++d) {
      cursor[d] = c;
      c = c + H[d];
    }
    for (uint64_t i = 0; i < n; ++i) {
      uint32_t d = (src[i] >> (8 * pass)) & 255u;
      if (is_signed && pass == 3) d = d ^ 0x80u;
      dst[cursor[d]] = src[i];
      cursor[d] = cursor[d] + 1;
    }
    src = dst;
  }
}

/*
 * Prop. "General Self-Indexing Principle", constructive proof: step 1, for
 * every key x compute i = phi(x) and add one to H[i]; step 2, for i = 0..U-1
 * emit phi_inv(i) exactly H[i] times.  phi == NULL means phi(x) = x, and
 * phi_inv == NULL means phi_inv(i) = i.  A key with x >= M (when phi is
 * given), phi[x] == 0xffffffff, or index >= U is not in the domain: it is not
 * counted.  Keys and output are passed widened to uint32.  H has U entries.
 * Returns the number of keys not counted; out receives sum(H) keys.
 */
uint64_t oracle_sort_mapped(const uint32_t* keys, uint64_t n, const uint32_t* phi, uint32_t M,
                            const uint32_t* phi_inv, uint32_t U, uint32_t* out, uint32_t* H) {
  uint64_t skipped = 0;
  for (uint64_t k = 0; k < U; ++k) H[k] = 0;
  for (uint64_t j = 0; j < n; ++j) {
    uint32_t i = keys[j];
    if (phi != 0) i = keys[j] < M ? phi[keys[j]] : 0xffffffffu;
    if (i < U)
      H[i] = H[i] + 1;
    else
      skipped = skipped + 1;
  }
  uint64_t pos = 0;
  for (uint64_t i = 0; i < U; ++i) {
    const uint32_t value = phi_inv != 0 ? phi_inv[i] : (uint32_t)i;
    for (uint32_t c = 0; c < H[i]; ++c) {
      out[pos] = value;
      pos = pos + 1;
    }
  }
  return skipped;
}
