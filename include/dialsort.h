/*
 * dialsort.h -- C ABI of libdialsort.so, a GB300 (sm_103a) implementation of
 * the data-parallel hot path of DialSort (A. Narvaez, "DialSort:
 * Non-Comparative Integer Sorting via the Self-Indexing Principle", 2026).
 *
 * The path has two steps:
 *   1. Ingestion, Eq. (1): H[0..U) is zeroed and H[x] += 1 for every key x.
 *      Concurrent equal keys are merged before they reach memory, as the
 *      Conflict Resolution Network of Sec. "Conflict Resolution Network (CRN)"
 *      does (node rule Eqs. (3)-(4), Definition "CRN level transition"): on the
 *      GPU a warp groups equal keys with match.any, sums their counts with
 *      redux.add, and one leader lane applies the sum.  Only equality between
 *      keys is evaluated (Definition "Order comparison").
 *   2. Ordered projection, Eq. (2): for k = 0..U-1, emit k exactly H[k] times.
 *      Placing runs in parallel needs each run's start (the cursor of the
 *      sequential projection); a chunk-level offset scan provides it.
 *
 * Conventions for every entry point:
 *   - Pointers named keys, H, out, ws are DEVICE pointers owned by the caller.
 *     Descriptor arrays passed to the batched entry points are HOST pointers.
 *     Exception: dialsort_histogram*, dialsort_reconstruct(_u16) and
 *     dialsort_sort(_u16) also take keys, H and out in page-locked host
 *     memory (cudaHostAlloc / cudaHostRegister, whole range registered), and
 *     in pageable host memory where the device reads host page tables
 *     (cudaDevAttrPageableMemoryAccess).  The kernels then read and write it
 *     across the CPU-GPU link themselves, with no staging copy; ws is device
 *     memory always.  Memory of another device, or host memory the device
 *     cannot reach, is DIALSORT_ERR_INVALID_ARG.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are asynchronous on that stream; nothing is synchronised unless the
 *     entry point says so.
 *   - The library allocates no device memory on these paths: scratch lives in
 *     the caller's workspace (`ws`, `ws_bytes`), sized by the *_workspace_size
 *     queries.  Workspace must be 256-byte aligned and must not be shared by
 *     calls that may run concurrently.
 *   - Argument errors are found on the host, before any launch, and returned
 *     synchronously.  Errors found by kernels (a key >= U, a scan that gave up
 *     waiting, a histogram whose total exceeds the output) set bits in a
 *     per-device error word, read and cleared by dialsort_stream_status().
 *   - Keys must be aligned to their own width; H must be 16-byte aligned.
 *     keys and out may be at any such alignment (unaligned heads and tails are
 *     handled).  n < 2^32 and 1 <= U < 2^32.
 */
#ifndef DIALSORT_H
#define DIALSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DIALSORT_OK = 0,
  DIALSORT_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or width */
  DIALSORT_ERR_KEY_RANGE = 2,   /* a kernel saw a key >= U; that key was not counted */
  DIALSORT_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  DIALSORT_ERR_BUDGET = 4,      /* a served request cannot fit the server's HBM budget */
  DIALSORT_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  DIALSORT_ERR_BUSY = 6,        /* a served request is not finished yet */
  DIALSORT_ERR_OVERFLOW = 7,    /* sum(H) exceeds the output capacity n; output truncated to n */
  DIALSORT_ERR_WORKSPACE = 8,   /* workspace too small or misaligned */
} dialsort_status_t;

/* How step 1 privatises H (the autotuner picks one when AUTO is given). */
typedef enum {
  DIALSORT_REGIME_AUTO = 0,
  DIALSORT_REGIME_SMEM32 = 1,     /* per-CTA 32-bit sub-histograms in shared memory, merged into H */
  DIALSORT_REGIME_SMEM16 = 2,     /* per-CTA packed 16-bit sub-histograms with exact carry spill */
  DIALSORT_REGIME_CLUSTER = 3,    /* reserved: a sub-histogram spread over a cluster's shared memory; not
                                     built (remote shared-memory atomics measured slower than L2 ones),
                                     refused with DIALSORT_ERR_INVALID_ARG */
  DIALSORT_REGIME_GLOBAL_CRN = 4, /* warp CRN, then one L2 atomic per distinct key of the warp */
  DIALSORT_REGIME_GLOBAL = 5,     /* one L2 atomic per key run of a thread (no cross-lane merge) */
  DIALSORT_REGIME_TWO_LEVEL = 6,  /* large U: partition keys by high bits, then count low bits in shared
                                     memory per bucket (needs workspace; uint32 keys in device memory,
                                     16-byte aligned) */
} dialsort_regime_t;

/* Skew classes of a key sequence (dialsort_probe_skew; the autotuner's table
 * is keyed by them).  How often equal keys meet decides what the CRN's merge
 * saves and how contended the counters get (Sec. "Conflict Resolution
 * Network (CRN)", subsection "Performance consequence under skewed input"). */
typedef enum {
  DIALSORT_SKEW_UNKNOWN = 0,
  DIALSORT_SKEW_LOW = 1,    /* few equal keys meet: near uniform over a large universe */
  DIALSORT_SKEW_HOT = 2,    /* a few keys hold a large share (Zipf-like) */
  DIALSORT_SKEW_RUNS = 3,   /* most neighbours are equal (sorted input, long runs, all equal) */
} dialsort_skew_class_t;

/* Launch choices for step 1.  Zero in any field means "pick automatically". */
typedef struct {
  uint32_t regime;   /* dialsort_regime_t */
  uint32_t crn;      /* 0 = auto, 1 = warp CRN on, 2 = off, 3 = adaptive per warp (the per-thread run
                        merge always runs; auto = adaptive, or off for REGIME_GLOBAL) */
  uint32_t blocks;   /* grid size */
  uint32_t threads;  /* CTA size: 256, 512 or 1024 */
  uint32_t replicas; /* shared-memory sub-histogram copies per CTA (SMEM32 / SMEM16) */
  uint32_t cluster;  /* CTAs per cluster (CLUSTER regime): 2, 4, 8 or 16 */
  uint32_t skew;     /* dialsort_skew_class_t of the keys, when known: with every other field zero the
                        autotuner takes its measured table's entry for this class (0 = unknown) */
} dialsort_hist_config_t;

/* ---------------------------------------------------------------- step 1: ingestion, Eq. (1) */

/*
 * H[0..U) := multiplicity of each k among keys[0..n) (uint32 keys).  H is
 * overwritten (zeroed, then counted).  Keys >= U are skipped and raise
 * DIALSORT_ERR_KEY_RANGE in the error word.  n may be 0 (H is zeroed).
 */
dialsort_status_t dialsort_histogram(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H, void* stream);

/* As dialsort_histogram for uint16 keys; requires U <= 65536. */
dialsort_status_t dialsort_histogram_u16(const uint16_t* keys, uint64_t n, uint32_t U, uint32_t* H, void* stream);

/*
 * As dialsort_histogram with explicit launch choices (key_bytes = 4 or 2).
 * cfg may be NULL (= all automatic).  Invalid combinations (e.g. a shared
 * memory regime whose sub-histogram does not fit) return INVALID_ARG.
 */
dialsort_status_t dialsort_histogram_ex(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H,
                                        const dialsort_hist_config_t* cfg, void* stream);

/*
 * Workspace bytes that dialsort_histogram_ws may use for (n, U, key_bytes):
 * the scratch of the two-level regime when it can apply, else 0.
 */
size_t dialsort_histogram_workspace_size(uint64_t n, uint32_t U, uint32_t key_bytes);

/*
 * As dialsort_histogram_ex with a workspace (256-byte aligned device memory,
 * not shared with concurrent calls).  With enough workspace the automatic
 * plan uses the two-level regime for large universes (uint32 keys in device
 * memory, 16-byte aligned, n >= 2^20); ws may be NULL (then it never does).
 * Forcing DIALSORT_REGIME_TWO_LEVEL on keys that do not qualify returns
 * DIALSORT_ERR_INVALID_ARG (DIALSORT_ERR_WORKSPACE if only ws is short).
 */
dialsort_status_t dialsort_histogram_ws(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H,
                                        const dialsort_hist_config_t* cfg, void* ws, size_t ws_bytes,
                                        void* stream);

/*
 * Accumulating ingestion: H[x] += 1 for every key x, without zeroing H first,
 * so H ends as the histogram of every batch ingested into it since it was
 * last zeroed (Eq. (1) applied to a stream of batches; the paper's remark on
 * streaming ingestion after Thm. "Parallel DialSort with pipelined CRN").  Keys arriving in
 * chunks can be ingested as each chunk lands, and the projection runs once at
 * the end.  Arguments as dialsort_histogram_ws (ws may be NULL); H must
 * already hold valid counts (zero it once before the first batch).  The
 * caller keeps the total below 2^32 per bin.
 */
dialsort_status_t dialsort_histogram_accumulate(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U,
                                               uint32_t* H, void* ws, size_t ws_bytes, void* stream);

/*
 * Chunked ingestion from host memory, overlapped with the copies: the
 * streaming form of Eq. (1) (the remark after Thm. "Parallel DialSort with
 * pipelined CRN": H is a sum over keys, so it can absorb each batch as it
 * lands).  host_keys (n keys of key_bytes = 4 or 2; page-locked host memory,
 * else the copies do not overlap) is copied chunk_keys keys at a time into
 * two device staging buffers in ws on copy_stream, while `stream` ingests
 * the previous chunk into H; a staging buffer is refilled only once the
 * ingestion that read it has finished.  Both streams must be distinct and
 * non-NULL; the copies first wait for the work already queued on `stream`.
 *   dialsort_histogram_chunked: H (device, U counters, 16-byte aligned)
 *     += histogram of the keys (H must hold valid counts: zero it once first,
 *     as for dialsort_histogram_accumulate).
 *   dialsort_sort_chunked: H in ws from 0, then Eq. (2) into out (device or
 *     page-locked host memory, n keys) on `stream`.
 * ws: device memory, 256-byte aligned, dialsort_chunked_workspace_size bytes
 * (sort != 0 for the sort).  Asynchronous; kernel-side errors go to the
 * error word.
 */
size_t dialsort_chunked_workspace_size(uint64_t n, uint32_t U, uint32_t key_bytes, uint64_t chunk_keys, int sort);
dialsort_status_t dialsort_histogram_chunked(const void* host_keys, uint32_t key_bytes, uint64_t n, uint32_t U,
                                             uint64_t chunk_keys, uint32_t* H, void* ws, size_t ws_bytes,
                                             void* stream, void* copy_stream);
dialsort_status_t dialsort_sort_chunked(const void* host_keys, uint32_t key_bytes, uint64_t n, uint32_t U,
                                        uint64_t chunk_keys, void* out, void* ws, size_t ws_bytes, void* stream,
                                        void* copy_stream);

/*
 * The autotuner's choice for a histogram of n keys of key_bytes over [0,U)
 * with the given skew hint (a dialsort_skew_class_t, 0..3).  Host only;
 * writes *cfg with every field filled in.  With every field of *cfg zero on
 * input the choice comes from the measured tuning table (see
 * dialsort_tune_table_load) when it has an entry near (n, U) for this key
 * width and skew class, else from the built-in cost model.  With regime AUTO
 * on input, DIALSORT_REGIME_TWO_LEVEL is reported where dialsort_histogram_ws
 * and dialsort_sort choose it (16-byte aligned keys, workspace given); the
 * other fields then describe the single-pass plan that dialsort_histogram
 * (no workspace) runs instead.
 */
dialsort_status_t dialsort_plan_histogram(uint64_t n, uint32_t U, uint32_t key_bytes, uint32_t skew_hint,
                                          dialsort_hist_config_t* cfg);

/* What the skew probe saw (dialsort_probe_skew). */
typedef struct {
  uint32_t samples;          /* sampled keys below U */
  uint32_t equal_neighbours; /* sampled neighbour pairs holding equal keys */
  uint32_t neighbour_pairs;  /* sampled neighbour pairs */
  uint32_t top_multiplicity; /* largest count of one key among the samples */
  uint32_t skew_class;       /* dialsort_skew_class_t derived from the above */
  uint32_t reserved;
} dialsort_skew_t;

/*
 * Skew probe: one CTA reads 128 windows of 32 consecutive keys spread evenly
 * over keys[0..n) (4096 keys; fewer when n is small) and measures, with
 * equality tests between keys only (Definition "Order comparison"), how many
 * neighbours are equal and the largest multiplicity of one key (a hash table
 * in shared memory whose probes compare keys for equality).  The class is
 * RUNS when at least half of the neighbour pairs are equal, HOT when one key
 * holds at least max(4 x samples / U, samples / 64) samples, else LOW;
 * UNKNOWN below 64 samples.  keys: device (or page-locked host) memory,
 * key_bytes 4 or 2, aligned to its width.  Synchronous: waits for `stream`
 * and fills *out.  Keys >= U are not counted (and raise no error).
 */
dialsort_status_t dialsort_probe_skew(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U,
                                      dialsort_skew_t* out, void* stream);

/*
 * The tuning table: text lines "log2n log2U key_bytes skew regime crn
 * replicas threads blocks_per_sm" ('#' starts a comment; crn in the
 * dialsort_hist_config_t coding; 0 in a field = automatic), measured on the
 * device by the package's tuning script.  The planner takes the entry with
 * the same key width and skew class nearest to (log2 n, log2 U), distance
 * 2|dU| + |dn| at most 6, and uses the cost model where there is none or
 * the entry does not apply (e.g. TWO_LEVEL without workspace).  Loaded at
 * the first plan from the file named by the environment variable
 * DIALSORT_TUNE_CACHE (set but empty: no table), else from tune_table.txt in
 * the library's directory.  dialsort_tune_table_load replaces the table by
 * the file at `path` (NULL: an empty table, the cost model alone); an
 * unreadable file returns INVALID_ARG and keeps the old table.
 */
dialsort_status_t dialsort_tune_table_load(const char* path);
/* Number of entries in the table in use (loads it first if needed). */
uint32_t dialsort_tune_table_size(void);

/* ---------------------------------------------------------------- step 2: ordered projection, Eq. (2) */

/* Bytes of workspace dialsort_reconstruct / dialsort_offsets need for (U, n). */
size_t dialsort_reconstruct_workspace_size(uint32_t U, uint64_t n);

/*
 * out[0..sum(H)) := k repeated H[k] times for k = 0..U-1 (Eq. (2)).  n is
 * the capacity of out (normally the n the histogram was built from, which
 * equals sum(H)).  If sum(H) > n only n keys are written and
 * DIALSORT_ERR_OVERFLOW is raised in the error word; if sum(H) < n,
 * out[sum(H)..n) is left untouched.  out may alias the keys that H was built
 * from (the in-place projection of Sec. "DialSort vs. Classic Counting
 * Sort"); it must not overlap H or ws.
 */
dialsort_status_t dialsort_reconstruct(const uint32_t* H, uint32_t U, uint32_t* out, uint64_t n, void* ws,
                                       size_t ws_bytes, void* stream);

/* As dialsort_reconstruct writing uint16 keys; requires U <= 65536. */
dialsort_status_t dialsort_reconstruct_u16(const uint32_t* H, uint32_t U, uint16_t* out, uint64_t n, void* ws,
                                           size_t ws_bytes, void* stream);

/*
 * The offset scan of step 2 alone (it is the first kernel of
 * dialsort_reconstruct): writes, into ws, the start of every 1024-bin chunk's
 * run in the output and the first chunk of every 8192-key output tile.  Exposed
 * so the scan can be timed and checked separately.  dialsort_read_chunk_offsets
 * copies the chunk starts (ceil(U/1024) + 1 uint64 values, the last = sum(H))
 * to a device array.
 */
dialsort_status_t dialsort_offsets(const uint32_t* H, uint32_t U, uint64_t n, void* ws, size_t ws_bytes,
                                   void* stream);
dialsort_status_t dialsort_read_chunk_offsets(const void* ws, uint32_t U, uint64_t n, uint64_t* chunk_offsets,
                                              void* stream);

/*
 * Allocation-free variant of dialsort_reconstruct (uint32 output).  The paper
 * has no counterpart: this exists for callers that cannot allocate device
 * memory at call time -- e.g. a plugin that a host framework hands only its
 * input and output buffers, or a latency-critical loop that must not take an
 * allocator's locks or risk running out of memory mid-run.  The caller passes
 * H and out exactly as for dialsort_reconstruct but no workspace.
 *
 * Scratch lives in a library-owned device array of
 * DIALSORT_NOALLOC_SCRATCH_BYTES (2 MiB) on every device that loads the
 * library, held until the process exits.  Sizes whose scratch would exceed it
 * (dialsort_reconstruct_workspace_size(U, n) > DIALSORT_NOALLOC_SCRATCH_BYTES;
 * every U <= 2^26 with n <= 2^30 fits) are rejected with
 * DIALSORT_ERR_WORKSPACE before anything is launched.  The call allocates
 * nothing (no cudaMalloc, no allocating library routine).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it; make that
 * first call before any stream capture.  All calls on a device share the
 * array: each call clears the parts that must start at zero, in stream order,
 * but calls whose kernels overlap on the GPU (other streams or threads) race
 * on it and must be serialised by the caller.
 */
#define DIALSORT_NOALLOC_SCRATCH_BYTES ((size_t)2 << 20)
dialsort_status_t dialsort_reconstruct_noalloc(const uint32_t* H, uint32_t U, uint32_t* out, uint64_t n,
                                               void* stream);

/* ---------------------------------------------------------------- both steps */

/* Bytes of workspace dialsort_sort needs: H (4U bytes), the scan scratch and,
 * for large universes, the two-level ingestion scratch. */
size_t dialsort_sort_workspace_size(uint64_t n, uint32_t U);

/*
 * Sorts keys[0..n) into out[0..n) by Eq. (1) then Eq. (2).  H is kept at the
 * start of ws (dialsort_sort_histogram(ws) returns it).  out may equal keys
 * (in place).
 */
dialsort_status_t dialsort_sort(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* out, void* ws,
                                size_t ws_bytes, void* stream);
dialsort_status_t dialsort_sort_u16(const uint16_t* keys, uint64_t n, uint32_t U, uint16_t* out, void* ws,
                                    size_t ws_bytes, void* stream);
/*
 * Runs dialsort_sort (key_bytes 4 or 2, automatic choices) once with CUDA
 * events between its stages and waits for it; for measuring kernels inside
 * a sort.  Writes the stage durations in milliseconds to ms[0 .. *stages):
 * for the two-level form 4 stages (pass 1 partition; split and schedule;
 * counting fused with the projection; painting of long runs), otherwise 1
 * (the whole sort).  ms needs room for 4 values.  Arguments otherwise as
 * dialsort_sort; synchronous.
 */
dialsort_status_t dialsort_sort_stage_times(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, void* out,
                                            void* ws, size_t ws_bytes, void* stream, float* ms, uint32_t* stages);

/*
 * As dialsort_sort (key_bytes 4 or 2) with explicit launch choices for step 1
 * (cfg as for dialsort_histogram_ws, NULL = automatic; its skew field feeds
 * the autotuner).  ws as for dialsort_sort.
 */
dialsort_status_t dialsort_sort_ex(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, void* out,
                                   const dialsort_hist_config_t* cfg, void* ws, size_t ws_bytes, void* stream);
/* Device pointer to the histogram that dialsort_sort leaves in ws. */
uint32_t* dialsort_sort_histogram(void* ws);

/* ---------------------------------------------------------------- mapped domains */

/*
 * Sorting a finite ordered domain through an order-preserving map onto
 * [0, U) (Prop. "General Self-Indexing Principle"): every key x is counted
 * at index phi(x) (Eq. (1) over [0, U)), then for every index i in
 * ascending order phi_inv(i) is emitted H[i] times (Eq. (2)).  When phi
 * preserves order the output is the keys sorted in the domain's order; the
 * library does not check that it does.
 *   keys, out  n raw keys of key_bytes (1, 2 or 4) each, aligned to their
 *              width; out may equal keys.
 *   phi, M     uint32[M] index of every raw value below M; 0xffffffff marks
 *              a value outside the domain.  NULL: the raw value is its own
 *              index (M ignored).  A raw key >= M, or marked outside the
 *              domain, or whose index is >= U, is not counted and sets
 *              DIALSORT_ERR_KEY_RANGE in the error word.
 *   phi_inv    U raw values of key_bytes each, the key emitted for each
 *              index.  NULL: the index itself is emitted.
 *   ws         dialsort_sort_mapped_workspace_size(n, U) bytes, 256-byte
 *              aligned; H is kept at its start.
 * Examples: 8-bit pixels (key_bytes 1, phi = phi_inv = NULL, U = 256);
 * a dictionary of sparse 32-bit codes compacted to their ranks.
 */
size_t dialsort_sort_mapped_workspace_size(uint64_t n, uint32_t U);
dialsort_status_t dialsort_sort_mapped(const void* keys, uint32_t key_bytes, uint64_t n, const uint32_t* phi,
                                       uint32_t M, const void* phi_inv, uint32_t U, void* out, void* ws,
                                       size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- DialSort-Radix */

/*
 * DialSort-Radix (Sec. "Full int32 range"): sorts keys of the full 32-bit
 * range by four stable DialSort passes over base-256 digits, least
 * significant first (each pass: Eq. (1) on the digit with U = 256, then every
 * key placed at its digit's cursor in input order).  _i32 sorts two's
 * complement int32 (negative keys first); _u32 sorts unsigned.
 * keys, out: n keys, 4-byte aligned, device memory (or host memory per the
 * rules above); out may equal keys.  ws: dialsort_radix_workspace_size(n)
 * bytes, 256-byte aligned (n keys of ping-pong space, the digit histograms
 * and the look-back descriptors, which are zeroed by the call).  n < 2^32.
 * A look-back wait that gives up (it should never) records
 * DIALSORT_ERR_TIMEOUT in the error word; no write leaves out[0..n).
 */
size_t dialsort_radix_workspace_size(uint64_t n);
dialsort_status_t dialsort_radix_sort_i32(const int32_t* keys, uint64_t n, int32_t* out, void* ws, size_t ws_bytes,
                                          void* stream);
dialsort_status_t dialsort_radix_sort_u32(const uint32_t* keys, uint64_t n, uint32_t* out, void* ws,
                                          size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- queries on H */

/*
 * H is the canonical ordered state of the data (Sec. "Canonical ordered
 * state"): point and range queries read it directly, with no projection.
 * H: uint32[U], 16-byte aligned, as written by step 1.  Query and result
 * arrays hold m entries, 4-byte aligned (present: 1 byte per entry).  A query
 * key outside [0, U) has frequency 0 and is absent (no key there was
 * counted); it is not an error.  Asynchronous on `stream`; m = 0 launches
 * nothing.  Pointers follow the memory rules of dialsort_histogram.
 */

/* freq[i] = H[q[i]] (Sec. "Canonical ordered state", frequency(k)). */
dialsort_status_t dialsort_frequency(const uint32_t* H, uint32_t U, const uint32_t* q, uint64_t m, uint32_t* freq,
                                     void* stream);

/* present[i] = 1 if H[q[i]] > 0 else 0 (presence(k)). */
dialsort_status_t dialsort_presence(const uint32_t* H, uint32_t U, const uint32_t* q, uint64_t m, uint8_t* present,
                                    void* stream);

/*
 * count[i] = sum of H[k] over a[i] <= k <= b[i] (range-count(a, b), bounds
 * inclusive, clipped to [0, U)); 0 when a[i] > b[i].  Cost O(b - a) per
 * query, as in the paper; one warp sums one range.  Exact while sum(H) <
 * 2^32, which every histogram of n < 2^32 keys satisfies.
 */
dialsort_status_t dialsort_range_count(const uint32_t* H, uint32_t U, const uint32_t* a, const uint32_t* b,
                                       uint64_t m, uint32_t* count, void* stream);

/* ---------------------------------------------------------------- batched form */

/*
 * One independent instance of a batch.  keys (n keys of key_bytes = 4 or 2),
 * H (U uint32 counters, 16-byte aligned, overwritten) and out (n keys, or
 * NULL for histogram only) are device pointers owned by the caller.  The same
 * rules as for dialsort_histogram / dialsort_sort apply to each instance.
 */
typedef struct {
  const void* keys;
  uint32_t* H;
  void* out;
  uint64_t n;
  uint32_t U;
  uint32_t key_bytes;
  uint32_t skew;     /* dialsort_skew_class_t of the keys, 0 = unknown (dialsort_probe_skew_batched) */
  uint32_t regime;   /* 0 = automatic; else the dialsort_regime_t step 1 must use (SMEM32, SMEM16,
                        GLOBAL_CRN, GLOBAL, or TWO_LEVEL for U <= 2^22); one that cannot apply makes
                        dialsort_batch_create return INVALID_ARG */
} dialsort_instance_t;

/*
 * The skew probe of dialsort_probe_skew for every instance of an array in one
 * launch (one CTA per instance); writes instances[i].skew.  Synchronous.
 */
dialsort_status_t dialsort_probe_skew_batched(dialsort_instance_t* instances, uint32_t count, void* stream);

/* A planned batch (host object).  Planning picks, per instance, how step 1
 * privatises H (shared-memory 32-bit, packed 16-bit, or L2 atomics with the
 * adaptive warp CRN), the keys per work item and the item counts of every
 * phase, and orders instances largest first. */
typedef struct dialsort_batch_s* dialsort_batch_t;

/*
 * Plans a batch of `count` instances.  With sort != 0 every instance with
 * n > 0 needs out; with sort == 0 out is ignored (histograms only).  The
 * instance array is copied; the device buffers it names must stay valid until
 * the last launch of the batch has finished.
 */
dialsort_status_t dialsort_batch_create(const dialsort_instance_t* instances, uint32_t count, int sort,
                                        dialsort_batch_t* batch);
/* Workspace bytes (256-byte aligned device memory) a launch of the batch needs. */
size_t dialsort_batch_workspace_size(dialsort_batch_t batch);
/*
 * Runs the whole batch on `stream`: two host-to-device copies of the plan
 * tables (from pinned memory owned by the batch), one memset and ONE
 * persistent kernel whose CTAs pull work items of all instances.  Every call
 * is asynchronous and can be captured into a CUDA graph (the graph reads the
 * batch's pinned tables when it runs, so the batch must outlive the graph).
 * Kernel-side errors (a key >= U, a wait that timed out) go to the error word.
 */
dialsort_status_t dialsort_batch_launch(dialsort_batch_t batch, void* ws, size_t ws_bytes, void* stream);
/* Frees the batch's host tables (after its launches have finished). */
dialsort_status_t dialsort_batch_destroy(dialsort_batch_t batch);
/* The plan of instance `index` (caller's order): regime etc. in *cfg, and the
 * item counts of the zero / histogram / offsets / expand phases in items[4]. */
dialsort_status_t dialsort_batch_describe(dialsort_batch_t batch, uint32_t index, dialsort_hist_config_t* cfg,
                                          uint32_t* items);

/* One-shot forms: plan, launch, synchronise `stream`, free the plan. */
size_t dialsort_batched_workspace_size(const dialsort_instance_t* instances, uint32_t count, int sort);
dialsort_status_t dialsort_batched(const dialsort_instance_t* instances, uint32_t count, int sort, void* ws,
                                   size_t ws_bytes, void* stream);
dialsort_status_t dialsort_histogram_batched(const dialsort_instance_t* instances, uint32_t count, void* ws,
                                             size_t ws_bytes, void* stream);
dialsort_status_t dialsort_sort_batched(const dialsort_instance_t* instances, uint32_t count, void* ws,
                                        size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- served form */

/* Server configuration.  The server allocates, once at creation, an arena of
 * hbm_budget_bytes of device memory for the H, output and scan scratch of
 * admitted requests, plus small tables; nothing is allocated per request. */
typedef struct {
  uint64_t hbm_budget_bytes; /* arena size: admitted requests must fit in it together */
  uint32_t max_slots;        /* requests on the device at once, 1..256 */
  uint32_t reserved;
  uint64_t idle_timeout_ns;  /* the device loop leaves after this long without work (0 = 20 ms) */
} dialsort_server_cfg_t;

/* A request: keys are a device pointer owned by the caller and must stay
 * valid and unchanged until the request has finished. */
typedef struct {
  const void* keys;
  uint64_t n;
  uint32_t U;
  uint32_t key_bytes; /* 4 or 2 */
  uint32_t kind;      /* 0 = histogram (step 1), 1 = sort (steps 1 and 2) */
  uint32_t skew;      /* dialsort_skew_class_t of the keys if known, else 0 */
} dialsort_request_t;

/* A finished request.  H (U counters) and out (n sorted keys, kind 1 only)
 * are device pointers into the server arena, valid until the ticket is
 * released.  Times are CLOCK_MONOTONIC nanoseconds on the host: submission,
 * admission to a device slot, and the moment the server saw it finish. */
typedef struct {
  uint32_t* H;
  void* out;
  uint64_t submit_ns, admit_ns, done_ns;
  uint32_t status; /* DIALSORT_OK or a kernel-side error of this request */
  uint32_t reserved;
} dialsort_result_t;

typedef struct dialsort_server_s dialsort_server_t;

/* Starts a server on the current device: allocates the arena and tables,
 * starts the scheduler thread.  The device loop is launched on demand. */
dialsort_status_t dialsort_server_create(const dialsort_server_cfg_t* cfg, dialsort_server_t** server);
/* Queues a request (admission is in arrival order, as slots and arena space
 * free up).  DIALSORT_ERR_BUDGET if the request alone exceeds the arena. */
dialsort_status_t dialsort_server_submit(dialsort_server_t* server, const dialsort_request_t* request,
                                         uint64_t* ticket);
/* DIALSORT_ERR_BUSY until the request has finished; then fills *result. */
dialsort_status_t dialsort_server_poll(dialsort_server_t* server, uint64_t ticket, dialsort_result_t* result);
/* As poll, blocking up to timeout_ns (DIALSORT_ERR_BUSY on timeout). */
dialsort_status_t dialsort_server_wait(dialsort_server_t* server, uint64_t ticket, uint64_t timeout_ns,
                                       dialsort_result_t* result);
/* Returns a finished (or still pending) request's memory to the arena. */
dialsort_status_t dialsort_server_release(dialsort_server_t* server, uint64_t ticket);
/* Stops the scheduler, lets the device loop finish, frees everything. */
dialsort_status_t dialsort_server_destroy(dialsort_server_t* server);

/* A timed request stream, for comparing the served form with per-request
 * plain launches on the same arrival trace. */
typedef struct {
  const void* keys;
  uint64_t n;
  uint32_t U;
  uint32_t key_bytes;
  uint32_t kind;
  uint32_t reserved;
  uint64_t arrival_ns; /* offset from the start of the replay */
} dialsort_trace_entry_t;

typedef struct {
  uint64_t arrival_ns; /* as given */
  uint64_t done_ns;    /* when the request was seen finished, same clock */
  uint32_t status;
  uint32_t reserved;
} dialsort_trace_result_t;

/*
 * Replays `trace` in real time from the calling thread: with use_server != 0
 * through a server created with *cfg (submit at each arrival, results
 * released as they finish); otherwise with per-request plain launches
 * (dialsort_histogram / dialsort_reconstruct on one stream at each arrival,
 * memory from an arena of cfg->hbm_budget_bytes).  Fills results[i] and the
 * replay's wall time.  Blocks until every request has finished.
 */
dialsort_status_t dialsort_replay(const dialsort_trace_entry_t* trace, uint32_t count, int use_server,
                                  const dialsort_server_cfg_t* cfg, dialsort_trace_result_t* results,
                                  uint64_t* wall_ns);

/* ---------------------------------------------------------------- status */

/*
 * Reads and clears the error word of the current device.  With sync != 0 the
 * stream is synchronised first, so every kernel launched on it so far has
 * reported.  The word is per device, not per stream: errors from work on
 * other streams of the same device show up here too.
 */
dialsort_status_t dialsort_stream_status(void* stream, int sync);

/* A short English description of a status code (static storage). */
const char* dialsort_status_string(dialsort_status_t status);

/* Number of SMs of the current device (0 if there is no usable device). */
int dialsort_device_sm_count(void);

/* 1 if kernels on the current device may read and write pageable host memory
 * (so keys/H/out may be plain malloc'd memory), 0 if only page-locked host
 * memory is reachable, -1 if there is no usable device. */
int dialsort_pageable_host_access(void);

/*
 * Self-test of the bounded device-side waits.  which = 0: one CTA of the
 * offset scan; which = 1: one CTA of a DialSort-Radix pass.  Each is started
 * on a work item whose predecessor is never published, so its look-back wait
 * runs out (about one to two seconds) and records DIALSORT_ERR_TIMEOUT in the
 * error word; the kernel then returns and the context stays usable.  Read the
 * result with dialsort_stream_status(stream, 1).  ws: 256-byte aligned,
 * dialsort_selftest_workspace_size() bytes.  The paper has no counterpart.
 */
size_t dialsort_selftest_workspace_size(void);
dialsort_status_t dialsort_selftest_wait_timeout(int which, void* ws, size_t ws_bytes, void* stream);

/* Library version string, e.g. "dialsort-gb300 0.1.0 sm_103a". */
const char* dialsort_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DIALSORT_H */
