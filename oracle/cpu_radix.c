/* Not the oracle: the stronger CPU baseline that bench.py times beside it.
 *
 * Test infrastructure, like the rest of this folder: only the tests and
 * bench.py's CPU-baseline leg load it; the library never does.
 *
 * An LSD radix sort of uint32 keys on all host threads (Sec. 3.3.1: low
 * digit first, each pass keeping the order of the one before): four passes
 * of 8-bit digits.  Per pass, every thread counts the digits of its chunk,
 * one serial sweep turns the counts into each (digit, thread) start in
 * digit-major order, and every thread moves its chunk to those starts in
 * order, so equal digits keep their input order.  The passes ping-pong
 * between `tmp` and `out`, the last one writing `out`.  Plain C and POSIX
 * threads; the tests check it against the oracle.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { RADIX = 256, MAX_THREADS = 256 };

typedef struct {
  const uint32_t* src;
  uint32_t* dst;
  size_t lo, hi;
  unsigned shift;
  size_t* count; /* [RADIX]: this thread's digit counts, then its starts */
} chunk_t;

static void* count_chunk(void* arg) {
  chunk_t* c = (chunk_t*)arg;
  memset(c->count, 0, RADIX * sizeof(size_t));
  for (size_t i = c->lo; i < c->hi; ++i) c->count[(c->src[i] >> c->shift) & (RADIX - 1)]++;
  return NULL;
}

static void* move_chunk(void* arg) {
  chunk_t* c = (chunk_t*)arg;
  for (size_t i = c->lo; i < c->hi; ++i) {
    const uint32_t k = c->src[i];
    c->dst[c->count[(k >> c->shift) & (RADIX - 1)]++] = k;
  }
  return NULL;
}

static int run_all(void* (*fn)(void*), chunk_t* chunks, int threads) {
  pthread_t tid[MAX_THREADS];
  int started = 0, rc = 0;
  for (int t = 1; t < threads; ++t) {
    if (pthread_create(&tid[t], NULL, fn, &chunks[t]) != 0) {
      rc = -1;
      break;
    }
    started = t;
  }
  if (rc == 0) fn(&chunks[0]);
  for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
  return rc;
}

/* Sorts n keys of `in` into `out` (tmp: n words of scratch; in, out and tmp
 * must not overlap) on `threads` threads (1..256).  Returns 0, or -1 on bad
 * arguments or when a thread could not be started (out is then undefined). */
int cpu_radix_sort_u32(const uint32_t* in, uint32_t* out, uint32_t* tmp, size_t n, int threads) {
  if (threads < 1 || threads > MAX_THREADS || (n && (!in || !out || !tmp))) return -1;
  if ((size_t)threads > n / 4096 + 1) threads = (int)(n / 4096 + 1);
  size_t* counts = (size_t*)malloc((size_t)threads * RADIX * sizeof(size_t));
  chunk_t* chunks = (chunk_t*)malloc((size_t)threads * sizeof(chunk_t));
  if (!counts || !chunks) {
    free(counts);
    free(chunks);
    return -1;
  }
  const uint32_t* src = in;
  int rc = 0;
  for (unsigned pass = 0; pass < 4 && rc == 0; ++pass) {
    uint32_t* dst = (pass & 1) ? out : tmp; /* passes 0, 2 -> tmp; 1, 3 -> out */
    for (int t = 0; t < threads; ++t) {
      chunks[t].src = src;
      chunks[t].dst = dst;
      chunks[t].lo = n * (size_t)t / (size_t)threads;
      chunks[t].hi = n * (size_t)(t + 1) / (size_t)threads;
      chunks[t].shift = 8u * pass;
      chunks[t].count = counts + (size_t)t * RADIX;
    }
    rc = run_all(count_chunk, chunks, threads);
    if (rc) break;
    size_t start = 0; /* digit-major: digit d of thread t follows digit d of threads < t */
    for (int d = 0; d < RADIX; ++d)
      for (int t = 0; t < threads; ++t) {
        const size_t c = chunks[t].count[d];
        chunks[t].count[d] = start;
        start += c;
      }
    rc = run_all(move_chunk, chunks, threads);
    src = dst;
  }
  free(counts);
  free(chunks);
  return rc;
}
