/*
 * A multi-threaded CPU DialSort, used only as a throughput line for the
 * benchmark's host cores.  It is not the oracle (which stays single-threaded
 * and plain) and shares nothing with the GPU path.
 *
 * Eq. (1) on T threads: each thread counts its slice of the keys into a
 * private histogram; the histograms are summed bin-parallel.  Eq. (2): the
 * run starts are a prefix sum over H, and each thread writes the runs of a
 * range of bins chosen so that every thread writes about n / T keys.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_get_max_threads(void) { return 1; }
static int omp_get_thread_num(void) { return 0; }
static int omp_get_num_threads(void) { return 1; }
#endif

/* Threads a call with threads = 0 uses (1 when built without OpenMP). */
int cpu_dialsort_threads(void) { return omp_get_max_threads(); }

/* Sorts keys[0..n) over [0, U) into out; keys >= U are skipped.  Returns the
 * number of keys written, or -1 if memory for the per-thread histograms is
 * not available. */
int64_t cpu_dialsort(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* out, int threads) {
  if (threads < 1 || threads > omp_get_max_threads()) threads = omp_get_max_threads();
  uint32_t* Ht = (uint32_t*)calloc((size_t)threads * U, sizeof(uint32_t));
  uint64_t* start = (uint64_t*)malloc(((size_t)U + 1) * sizeof(uint64_t));
  uint64_t* cut = (uint64_t*)malloc(((size_t)threads + 1) * sizeof(uint64_t));
  if (!Ht || !start || !cut) {
    free(Ht);
    free(start);
    free(cut);
    return -1;
  }
#pragma omp parallel num_threads(threads)
  {
    const int t = omp_get_thread_num();
    const int T = omp_get_num_threads();  /* the threads actually running (at most `threads`) */
    uint32_t* h = Ht + (size_t)t * U;
    const uint64_t lo = n * (uint64_t)t / T, hi = n * (uint64_t)(t + 1) / T;
    for (uint64_t i = lo; i < hi; ++i)
      if (keys[i] < U) h[keys[i]]++;
#pragma omp barrier
    /* sum the private histograms into the first one, bins split among the threads */
    const uint64_t b0 = (uint64_t)U * t / T, b1 = (uint64_t)U * (t + 1) / T;
    for (uint64_t b = b0; b < b1; ++b) {
      uint32_t s = 0;
      for (int j = 0; j < T; ++j) s += Ht[(size_t)j * U + b];
      Ht[b] = s;
    }
#pragma omp barrier
#pragma omp single
    {
      uint64_t c = 0;
      for (uint64_t b = 0; b < U; ++b) {
        start[b] = c;
        c += Ht[b];
      }
      start[U] = c;
      /* thread j writes the runs of bins [cut[j], cut[j+1]): about total / threads keys each */
      uint64_t b = 0;
      for (int j = 0; j <= T; ++j) {
        const uint64_t target = c * (uint64_t)j / T;
        while (b < U && start[b + 1] <= target && j < T) ++b;
        cut[j] = j == T ? U : b;
      }
      cut[0] = 0;
    }
    for (uint64_t k = cut[t]; k < cut[t + 1]; ++k) {
      uint32_t* o = out + start[k];
      for (uint32_t r = 0; r < Ht[k]; ++r) o[r] = (uint32_t)k;
    }
  }
  const int64_t total = (int64_t)start[U];
  free(Ht);
  free(start);
  free(cut);
  return total;
}
