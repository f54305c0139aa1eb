// DialSort-Radix (Sec. "Full int32 range"): LSD radix sort in base 256, four
// passes, each pass a DialSort step on one 8-bit digit -- count the digit
// (Eq. (1) with U = 256) and place every key at its digit's cursor (Eq. (2)'s
// projection, carrying the key instead of the digit).  LSD needs each pass to
// be stable, so placement keeps input order among equal digits.  Signed keys
// sort as unsigned words with the sign bit flipped (two's complement order).
// Keys are only ever split into digits; no two keys are compared by magnitude.
//
// GPU layout of one pass (one kernel per pass with the digit fixed at compile
// time; 512-thread CTAs, two per SM; tiles of 8192 keys taken in ticket order):
//   * warp w of the CTA holds keys [512 w, 512 w + 512) of the tile in
//     registers, lane l key 32 i + l in step i, so the order (step, lane) is
//     input order;
//   * in each step every lane ORs its bit into a per-warp shared-memory table
//     entry of its digit and reads the entry back: the lanes holding the same
//     digit, found by equality alone (the digit indexes the table); the
//     rank is the number of lower lanes among them plus a per-warp digit
//     counter that carries it across steps (a warp whose 32 keys share the
//     digit skips the table);
//   * a scan over (digit, warp) gives each key its slot in the tile's stable
//     digit order; keys are staged there in shared memory;
//   * the tile's per-digit counts are published as soon as they are known and
//     chained to the earlier tiles' by a decoupled look-back (one thread per
//     digit, four earlier tiles read per round with relaxed loads), giving
//     every digit run of the tile its global start = digit base + keys of
//     that digit in earlier tiles;
//   * the staged keys are written out, runs of one digit to consecutive
//     addresses.
// The global digit bases come from a histogram of the pass's digit over all
// keys: the first digit's from a separate counting kernel, the others counted
// by the previous pass while it has the keys in hand.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace dialsort {
namespace {

constexpr uint32_t kRxThreads = 512;                    // two CTAs per SM
constexpr uint32_t kRxWarps = kRxThreads / 32;
constexpr uint32_t kRxSteps = 16;                       // keys per thread
constexpr uint32_t kRxTile = kRxThreads * kRxSteps;     // 8192 keys per tile
constexpr uint32_t kRxWindow = 4;                       // earlier tiles read per look-back round
constexpr uint32_t kRxDigits = 256;
constexpr uint32_t kRxPasses = 4;

// Look-back descriptors: (state << 32) | value.  Pass p publishes state 2p+1
// (the tile's own count of the digit) and 2p+2 (count of the digit in tiles
// 0..t); anything else is "not yet" for pass p, so one zeroing per sort
// serves all four passes.
__device__ __forceinline__ uint64_t rx_desc(uint32_t state, uint32_t value) {
  return ((uint64_t)state << 32) | value;
}

// A descriptor word carries its state and its count together, and the look-back reads nothing else that
// the tile it describes wrote, so relaxed accesses suffice -- and, unlike acquire loads, a window of them
// can be in flight at once.
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Signed keys are sorted as unsigned words with the sign bit flipped (two's complement order): the
// first pass flips it on the way in, the last flips it back on the way out, so every digit is a byte.
template <uint32_t PASS>
__device__ __forceinline__ uint32_t rx_byte(uint32_t x) {
  return (x >> (8u * PASS)) & 0xffu;
}

__device__ __forceinline__ void red_or_shared(uint32_t* p, uint32_t v) {
  asm volatile("red.shared.or.b32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(uint32_t* p, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}

// Add 1 to h[d] for every lane; when all 32 lanes hold the same digit (keys
// that share a byte: small keys, a constant top byte) one lane adds 32.
__device__ __forceinline__ void rx_count(uint32_t* h, uint32_t d, uint32_t lane) {
  const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
  if (__all_sync(0xffffffffu, d == d0)) {
    if (lane == 0) red_add_shared(h + d, 32u);
  } else {
    red_add_shared(h + d, 1u);
  }
}

// Digit-0 histogram of all keys: shared counters (one copy per group of four
// warps), merged into ghist[0].
__global__ void __launch_bounds__(kRxThreads) rx_count_kernel(const uint32_t* __restrict__ keys, uint64_t n,
                                                               uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[4][kRxDigits];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  for (uint32_t i = tid; i < 4 * kRxDigits; i += kRxThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  uint32_t* mine = h[warp & 3u];
  // scalar head up to the first 16-byte boundary, 16-byte body, scalar tail
  const uint64_t mis = (reinterpret_cast<uintptr_t>(keys) & 15u) / 4u;
  const uint64_t head = mis ? ((4u - mis) < n ? (4u - mis) : n) : 0u;
  const uint64_t nvec = (n - head) / 4;
  const uint4* k4 = reinterpret_cast<const uint4*>(keys + head);
  const uint64_t stride = (uint64_t)gridDim.x * kRxThreads;
  const uint64_t vend = (nvec + 31u) & ~31ull;  // whole warps iterate together
  for (uint64_t v = (uint64_t)blockIdx.x * kRxThreads + tid; v < vend; v += stride) {
    const bool ok = v < nvec;  // (the loop bound is warp-uniform: vend and the stride are multiples of 32)
    const uint4 q = ok ? ld_stream_v4(k4 + v) : make_uint4(0u, 0u, 0u, 0u);
    if (__all_sync(0xffffffffu, ok)) {
      rx_count(mine, q.x & 0xffu, lane);
      rx_count(mine, q.y & 0xffu, lane);
      rx_count(mine, q.z & 0xffu, lane);
      rx_count(mine, q.w & 0xffu, lane);
    } else if (ok) {
      red_add_shared(mine + (q.x & 0xffu), 1u);
      red_add_shared(mine + (q.y & 0xffu), 1u);
      red_add_shared(mine + (q.z & 0xffu), 1u);
      red_add_shared(mine + (q.w & 0xffu), 1u);
    }
  }
  if (blockIdx.x == 0) {
    const uint64_t tail0 = head + nvec * 4;
    for (uint64_t i = tid; i < head + (n - tail0); i += kRxThreads)
      red_add_shared(mine + (keys[i < head ? i : tail0 + (i - head)] & 0xffu), 1u);
  }
  __syncthreads();
  for (uint32_t d = tid; d < kRxDigits; d += kRxThreads) {
    const uint32_t c = h[0][d] + h[1][d] + h[2][d] + h[3][d];
    if (c) red_add_global(ghist + d, c);
  }
}

struct RxSmem {
  uint32_t stage[kRxTile];               // the tile's keys in stable digit order
  uint32_t peer[kRxWarps][2][kRxDigits]; // per warp, two alternating tables: lanes (bit masks) holding each digit
  uint16_t wcnt[kRxWarps][kRxDigits];    // per-warp digit counters, then per-warp digit slots in the tile
  uint32_t gpos[kRxDigits];              // global position of the tile's first key of each digit
  uint32_t gbase[kRxDigits];             // global start of each digit
  uint32_t next[kRxDigits];              // histogram of the next pass's digit (this CTA)
  uint32_t red[32];
  uint32_t tile;
};

// Exclusive scan of v over the first 256 threads (the others pass through); returns the prefix.
__device__ __forceinline__ uint32_t scan256(uint32_t v, uint32_t* red, uint32_t* total) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31 && warp < kRxDigits / 32) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w0 = lane < kRxDigits / 32 ? red[lane] : 0u;
    uint32_t s = w0;
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= (uint32_t)d) s += y;
    }
    if (lane < kRxDigits / 32) red[lane] = s - w0;
    if (lane == kRxDigits / 32 - 1) red[kRxDigits / 32] = s;
  }
  __syncthreads();
  const uint32_t r = warp < kRxDigits / 32 ? red[warp] + (x - v) : 0u;
  *total = red[kRxDigits / 32];
  __syncthreads();
  return r;
}

// Load this thread's keys of a tile (step i, lane l -> key 32 i + l of the warp's 512; FLIP is xored in)
// and rank each among the warp's keys of the same digit in (step, lane) order, i.e. input order.
// The lanes holding a digit are found with equality only: each lane sets its bit in the step's table
// entry of its digit, then reads the entry back (one table per step parity; each step clears the
// previous step's entries).  A warp whose keys all share the digit skips the table.  Ranks go to rk as
// 16-bit pairs; wcnt[warp][d] ends as the warp's count of digit d.  FULL: the whole tile lies below n.
template <uint32_t PASS, bool FULL>
__device__ __forceinline__ void rx_load_rank(const uint32_t* __restrict__ src, uint32_t lim, uint32_t flip,
                                             uint32_t (&kv)[kRxSteps], uint32_t (&rk)[kRxSteps / 2], RxSmem& S) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t off = warp * (kRxSteps * 32u) + lane;  // this lane's key 0 in the tile
  const uint32_t* q = src + off;
#pragma unroll
  for (uint32_t i = 0; i < kRxSteps; ++i) kv[i] = (FULL || off + 32u * i < lim) ? q[32u * i] ^ flip : 0u;
  const uint32_t lt = lanemask_lt(), bit = 1u << lane;
  uint16_t* wc = S.wcnt[warp];
  uint32_t* tab = S.peer[warp][0];
  uint32_t dprev = 0;
  bool prev_used = false;
#pragma unroll
  for (uint32_t i = 0; i < kRxSteps; ++i) {
    const bool valid = FULL || off + 32u * i < lim;
    const uint32_t d = rx_byte<PASS>(kv[i]);
    const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);  // every lane takes part, keys or not
    const bool uni = __all_sync(0xffffffffu, valid && d == d0);
    uint32_t* cur = tab + (i & 1u) * kRxDigits;
    if (!uni && valid) red_or_shared(cur + d, bit);
    __syncwarp();  // every lane's bit is in; the previous step's leader update of wc is visible
    const uint32_t peers = uni ? 0xffffffffu : (valid ? cur[d] : 0u);
    if (prev_used) tab[((i + 1u) & 1u) * kRxDigits + dprev] = 0u;  // the previous step's table was read
    prev_used = !uni;
    dprev = d;
    const uint32_t before = wc[d];
    const uint32_t r = before + __popc(peers & lt);
    __syncwarp();  // every lane has read wc and the previous table before they change
    if (valid && (peers & lt) == 0) wc[d] = (uint16_t)(before + __popc(peers));
    if (i % 2 == 0)
      rk[i / 2] = r;
    else
      rk[i / 2] |= r << 16;
  }
  if (prev_used) tab[((kRxSteps - 1u) & 1u) * kRxDigits + dprev] = 0u;
  __syncwarp();
}

// One LSD pass on byte PASS.  Tiles of kRxTile keys are taken in ticket order; each is ranked stably in
// registers, its per-digit count published at once (so that later tiles can add it without waiting),
// its per-digit prefix over earlier tiles found by a decoupled look-back, and its keys staged in stable
// digit order and written out, runs of one digit to consecutive addresses.  The next pass's digit is
// counted on the way out.  kSigned: the sign bit is flipped in pass 0 and flipped back in pass 3.
template <bool kSigned, uint32_t PASS>
__global__ void __launch_bounds__(kRxThreads, 2) rx_pass_kernel(const uint32_t* __restrict__ src,
                                                                uint32_t* __restrict__ dst, uint64_t n,
                                                                uint64_t num_tiles, uint32_t* __restrict__ ghist,
                                                                uint64_t* __restrict__ desc,
                                                                uint32_t* __restrict__ tickets, uint32_t* err) {
  extern __shared__ __align__(16) unsigned char rx_raw[];
  RxSmem& S = *reinterpret_cast<RxSmem*>(rx_raw);
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  constexpr bool count_next = PASS + 1 < kRxPasses;
  constexpr uint32_t agg_state = 2u * PASS + 1u, inc_state = 2u * PASS + 2u;
  const uint32_t flip_in = (kSigned && PASS == 0) ? 0x80000000u : 0u;
  const uint32_t flip_out = (kSigned && PASS == kRxPasses - 1) ? 0x80000000u : 0u;

  // global digit starts of this pass: exclusive scan of its histogram
  {
    uint32_t total;
    const uint32_t c = tid < kRxDigits ? ghist[PASS * kRxDigits + tid] : 0u;
    const uint32_t ex = scan256(c, S.red, &total);
    if (tid < kRxDigits) {
      S.gbase[tid] = ex;
      S.next[tid] = 0;
    }
  }
  for (uint32_t i = tid; i < kRxWarps * 2 * kRxDigits; i += kRxThreads) (&S.peer[0][0][0])[i] = 0;
  bool timed_out = false;

  for (;;) {
    if (tid == 0) S.tile = atomicAdd(tickets + PASS, 1u);
    for (uint32_t i = tid; i < kRxWarps * kRxDigits / 2; i += kRxThreads)
      reinterpret_cast<uint32_t*>(&S.wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t t = S.tile;
    if (t >= num_tiles) break;
    const uint64_t tbase = t * kRxTile;
    const bool full = tbase + kRxTile <= n;
    const uint32_t lim = full ? kRxTile : (uint32_t)(n - tbase);
    uint32_t kv[kRxSteps], rk[kRxSteps / 2];
    if (full)
      rx_load_rank<PASS, true>(src + tbase, lim, flip_in, kv, rk, S);
    else
      rx_load_rank<PASS, false>(src + tbase, lim, flip_in, kv, rk, S);
    __syncthreads();

    // per digit: the warps' counts become their slots within the digit; publish the tile's count
    uint32_t cnt = 0;
    uint64_t* my = desc + t * kRxDigits + tid;
    if (tid < kRxDigits) {
#pragma unroll
      for (uint32_t w = 0; w < kRxWarps; ++w) {
        const uint32_t c = S.wcnt[w][tid];
        S.wcnt[w][tid] = (uint16_t)cnt;
        cnt += c;
      }
      st_relaxed_u64(my, rx_desc(t == 0 ? inc_state : agg_state, cnt));
    }
    uint32_t tile_valid;
    const uint32_t start = scan256(cnt, S.red, &tile_valid);
    if (tid < kRxDigits) {
#pragma unroll
      for (uint32_t w = 0; w < kRxWarps; ++w) S.wcnt[w][tid] = (uint16_t)(S.wcnt[w][tid] + start);
    }
    __syncthreads();  // every key's slot is known: warps past the first 256 threads stage during the look-back
    if (tid < kRxDigits) {
      // look back over earlier tiles for the digit's prefix, kRxWindow tiles per round: the counts of a
      // run of published tiles add up until one that carries its inclusive prefix
      uint32_t prefix = 0;
      if (t > 0) {
        uint64_t tt = t - 1;  // the next earlier tile not yet added
        uint32_t spins = 0;
        for (;;) {
          uint64_t v[kRxWindow];
#pragma unroll
          for (uint32_t j = 0; j < kRxWindow; ++j) v[j] = j <= tt ? ld_relaxed_u64(desc + (tt - j) * kRxDigits + tid) : 0ull;
          uint32_t used = 0;
          bool done = false;
#pragma unroll
          for (uint32_t j = 0; j < kRxWindow; ++j) {
            if (done || used != j || j > tt) continue;
            const uint32_t state = (uint32_t)(v[j] >> 32);
            if (state == inc_state) {
              prefix += (uint32_t)v[j];
              done = true;
            } else if (state == agg_state) {
              prefix += (uint32_t)v[j];
              used = j + 1;
            }
          }
          if (done) break;
          if (used > 0) {  // tile 0 always publishes its inclusive count, so tt stays >= 0 here
            tt -= used;
            continue;
          }
          if (++spins >= kSpinLimit) {  // tile tt never published: give up, report
            timed_out = true;
            break;
          }
          __nanosleep(64);
        }
        st_relaxed_u64(my, rx_desc(inc_state, prefix + cnt));
      }
      S.gpos[tid] = S.gbase[tid] + prefix - start;
    }

    // stage every key at its slot in the tile's stable digit order
    {
      const uint32_t off = warp * (kRxSteps * 32u) + lane;
      const uint16_t* wc = S.wcnt[warp];
#pragma unroll
      for (uint32_t i = 0; i < kRxSteps; ++i) {
        if (full || off + 32u * i < lim) {
          const uint32_t r = (rk[i / 2] >> (16 * (i & 1))) & 0xffffu;
          S.stage[wc[rx_byte<PASS>(kv[i])] + r] = kv[i];
        }
      }
    }
    __syncthreads();
    // write out: consecutive slots of one digit go to consecutive addresses; the next pass's digit is
    // counted on the way (gpos[d] holds the digit's global start minus its start in the tile)
#pragma unroll 4
    for (uint32_t j0 = warp * 32u; j0 < tile_valid; j0 += kRxThreads) {  // warp-uniform bound
      const uint32_t j = j0 + lane;
      const bool valid = j < tile_valid;
      const uint32_t x = valid ? S.stage[j] : 0u;
      if (valid) {
        const uint32_t pos = S.gpos[rx_byte<PASS>(x)] + j;  // mod 2^32: exact, since n < 2^32
        if (pos < n) dst[pos] = x ^ flip_out;  // always true unless a look-back timed out
      }
      if (count_next) {
        const uint32_t dn = rx_byte<(PASS + 1) % kRxPasses>(x);
        const uint32_t d0 = __shfl_sync(0xffffffffu, dn, 0);  // every lane takes part, keys or not
        if (__all_sync(0xffffffffu, valid && dn == d0)) {
          if (lane == 0) red_add_shared(&S.next[dn], 32u);
        } else if (valid) {
          red_add_shared(&S.next[dn], 1u);
        }
      }
    }
    // (the next tile's first barrier orders these reads of stage and gpos before their next writes)
  }
  if (timed_out) raise_error(err, ERRBIT_TIMEOUT);
  if (count_next) {
    __syncthreads();
    for (uint32_t d = tid; d < kRxDigits; d += kRxThreads)
      if (S.next[d]) red_add_global(ghist + (PASS + 1) * kRxDigits + d, S.next[d]);
  }
}

template <bool kSigned>
const void* rx_pass_fn(uint32_t pass) {
  switch (pass) {
    case 0: return reinterpret_cast<const void*>(&rx_pass_kernel<kSigned, 0>);
    case 1: return reinterpret_cast<const void*>(&rx_pass_kernel<kSigned, 1>);
    case 2: return reinterpret_cast<const void*>(&rx_pass_kernel<kSigned, 2>);
    default: return reinterpret_cast<const void*>(&rx_pass_kernel<kSigned, 3>);
  }
}

struct RxLayout {
  uint64_t num_tiles = 0;
  size_t off_ghist = 0, off_tickets = 0, off_desc = 0, clear_bytes = 0, off_tmp = 0, total = 0;
};

RxLayout rx_layout(uint64_t n) {
  RxLayout R;
  R.num_tiles = (n + kRxTile - 1) / kRxTile;
  size_t o = 0;
  R.off_ghist = o;
  o += 4 * (size_t)kRxPasses * kRxDigits;
  R.off_tickets = o;
  o = align_up(o + 4 * kRxPasses, 256);
  R.off_desc = o;
  o = align_up(o + 8 * (size_t)R.num_tiles * kRxDigits, 256);
  R.clear_bytes = o;
  R.off_tmp = o;
  o = align_up(o + 4 * (size_t)n, 256);
  R.total = o;
  return R;
}

dialsort_status_t radix_impl(const uint32_t* keys, uint64_t n, uint32_t* out, void* ws, size_t ws_bytes,
                             bool is_signed, cudaStream_t st) {
  if (n >= (1ull << 32)) return DIALSORT_ERR_INVALID_ARG;
  if (n > 0 && (keys == nullptr || out == nullptr)) return DIALSORT_ERR_INVALID_ARG;
  if (((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(out)) & 3u) != 0)
    return DIALSORT_ERR_INVALID_ARG;
  const RxLayout R = rx_layout(n);
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < R.total)
    return DIALSORT_ERR_WORKSPACE;
  if (n == 0) return DIALSORT_OK;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  const void* kp;
  const void* op;
  dialsort_status_t s = kernel_address(keys, *dev, &kp);
  if (s == DIALSORT_OK) s = kernel_address(out, *dev, &op);
  if (s != DIALSORT_OK) return s;
  keys = static_cast<const uint32_t*>(kp);
  out = static_cast<uint32_t*>(const_cast<void*>(op));

  char* base = static_cast<char*>(ws);
  uint32_t* ghist = reinterpret_cast<uint32_t*>(base + R.off_ghist);
  uint32_t* tickets = reinterpret_cast<uint32_t*>(base + R.off_tickets);
  uint64_t* desc = reinterpret_cast<uint64_t*>(base + R.off_desc);
  uint32_t* tmp = reinterpret_cast<uint32_t*>(base + R.off_tmp);
  cudaError_t e = cudaMemsetAsync(base, 0, R.clear_bytes, st);
  if (e != cudaSuccess) return DIALSORT_ERR_CUDA;
  const unsigned cgrid = (unsigned)std::min<uint64_t>((n / 4 + kRxThreads - 1) / kRxThreads + 1,
                                                      (uint64_t)dev->sms * 4);
  rx_count_kernel<<<cgrid, kRxThreads, 0, st>>>(keys, n, ghist);
  if (cudaGetLastError() != cudaSuccess) return DIALSORT_ERR_CUDA;

  const size_t smem = sizeof(RxSmem);
  int per_sm = 0;
  // tiles go out in ticket order, so a tile waits only on tiles whose CTAs are already running
  // ping-pong: keys -> tmp -> out -> tmp -> out (out may be keys: pass 0 and the count read keys first)
  const uint32_t* srcs[kRxPasses] = {keys, tmp, out, tmp};
  uint32_t* dsts[kRxPasses] = {tmp, out, tmp, out};
  uint64_t num_tiles = R.num_tiles;
  for (uint32_t p = 0; p < kRxPasses; ++p) {
    const void* fn = is_signed ? rx_pass_fn<true>(p) : rx_pass_fn<false>(p);
    if (kernel_config(fn, kRxThreads, smem, false, &per_sm) != cudaSuccess) return DIALSORT_ERR_CUDA;
    const unsigned grid = (unsigned)std::min<uint64_t>(R.num_tiles, (uint64_t)dev->sms * std::max(per_sm, 1));
    const uint32_t* sp = srcs[p];
    uint32_t* dp = dsts[p];
    uint64_t nn = n;
    uint32_t* err = dev->err;
    void* args[] = {&sp, &dp, &nn, &num_tiles, &ghist, &desc, &tickets, &err};
    if (cudaLaunchKernel(fn, dim3(grid), dim3(kRxThreads), args, smem, st) != cudaSuccess) return DIALSORT_ERR_CUDA;
  }
  return DIALSORT_OK;
}

}  // namespace

// Self-test of the bounded look-back wait: one CTA runs pass 0 on tile 1 of
// two tiles of keys (the ticket starts at 1), so tile 0 never publishes and the wait
// for it runs out, recording ERRBIT_TIMEOUT.  Every write stays inside tmp.
size_t radix_selftest_bytes() { return rx_layout(2 * kRxTile).total; }

cudaError_t launch_radix_selftest(void* ws, uint32_t* err, cudaStream_t stream) {
  const uint64_t n = 2 * kRxTile;
  const RxLayout R = rx_layout(n);
  char* base = static_cast<char*>(ws);
  cudaError_t e = cudaMemsetAsync(base, 0, R.total, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + R.off_tickets, 1, 1, stream);  // pass 0's ticket = 1
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(RxSmem);
  e = kernel_config(reinterpret_cast<const void*>(&rx_pass_kernel<false, 0>), kRxThreads, smem, false, nullptr);
  if (e != cudaSuccess) return e;
  uint32_t* tmp = reinterpret_cast<uint32_t*>(base + R.off_tmp);
  rx_pass_kernel<false, 0><<<1, kRxThreads, smem, stream>>>(tmp, tmp, n, R.num_tiles,
                                                             reinterpret_cast<uint32_t*>(base + R.off_ghist),
                                                             reinterpret_cast<uint64_t*>(base + R.off_desc),
                                                             reinterpret_cast<uint32_t*>(base + R.off_tickets), err);
  return cudaGetLastError();
}

namespace {
}  // namespace
}  // namespace dialsort

using namespace dialsort;

extern "C" {

size_t dialsort_radix_workspace_size(uint64_t n) { return rx_layout(n).total; }

dialsort_status_t dialsort_radix_sort_i32(const int32_t* keys, uint64_t n, int32_t* out, void* ws, size_t ws_bytes,
                                          void* stream) {
  return radix_impl(reinterpret_cast<const uint32_t*>(keys), n, reinterpret_cast<uint32_t*>(out), ws, ws_bytes,
                    true, static_cast<cudaStream_t>(stream));
}

dialsort_status_t dialsort_radix_sort_u32(const uint32_t* keys, uint64_t n, uint32_t* out, void* ws,
                                          size_t ws_bytes, void* stream) {
  return radix_impl(keys, n, out, ws, ws_bytes, false, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
