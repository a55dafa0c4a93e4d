/*
 * rsort.h: C ABI of librsort, a GB300 (sm_103a) radix distribution sort of
 * 32-bit unsigned keys, after Weaver & Lynes, "Sorting Integers on the
 * AP1000" (1994).
 *
 * What is computed (the paper's contract and method):
 *  - Sec. 1.1: the keys end up in ascending order, split evenly into
 *    num_parts (the contest used 64) contiguous partitions, partition 0
 *    holding the lowest values.  When num_parts does not divide n the lower
 *    partitions take the extra element (footnote 7 of Sec. 3.4.2), so
 *    partition p starts at  off[p] = p * floor(n / P) + min(p, n mod P).
 *  - Sec. 3.2 / 3.3.1 / 5: the sort is a radix distribution: per digit, a
 *    histogram of the digit (one count per key in its bucket), its cumulative
 *    totals, and a stable partial sort that groups keys by bucket in ascending
 *    bucket order, repeated from the low digit to the high one with the
 *    earlier order kept.  Pairs are therefore sorted STABLY by key.
 *
 * Conventions shared by every entry point:
 *  - Device pointers ("d_" or unprefixed key/value buffers) must be device
 *    memory of the current CUDA device, 4-byte aligned.  Host pointers are
 *    prefixed "h_".
 *  - The caller owns all memory.  The library never allocates: scratch comes
 *    in through (temp, temp_bytes).  Passing temp == NULL is a size query:
 *    *temp_bytes is set to the bytes needed and RS_OK is returned, nothing
 *    else happens.  temp must be 256-byte aligned.  The size needed depends
 *    only on the entry point, n (or total_n), the payload flag and the plan.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default) and
 *    is asynchronous: a return of RS_OK means the arguments were valid and
 *    the launches were enqueued.  Errors raised on the device (a bounded
 *    wait that gave up) are reported by rs_check_device_error().
 *  - Inputs are never modified; outputs must not overlap inputs or temp
 *    (RS_ERR_INVALID).  n = 0 is valid.  n must be below 2^32.
 *  - On any error the thread-local message of rs_last_error() says why.
 */
#ifndef RSORT_H
#define RSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, so callers need no CUDA header. */
typedef struct CUstream_st* rs_stream_t;

typedef enum rs_status {
  RS_OK = 0,
  RS_ERR_INVALID = 1,        /* bad pointer, size, alignment or overlap */
  RS_ERR_TEMP_TOO_SMALL = 2, /* *temp_bytes below the queried size */
  RS_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  RS_ERR_TIMEOUT = 4,        /* a device-side bounded wait gave up */
  RS_ERR_UNSUPPORTED = 5     /* a plan field this build does not offer */
} rs_status;

/* Radix plan.  Zero fields mean "choose automatically" (the library's
 * defaults, measured per size class) or, for key_kind, unsigned keys.
 *   digit_bits: 8 (four passes over 32-bit keys) or 11 (three passes,
 *               11 + 11 + 10 bits).  The paper's bucketing used 12-13 bit
 *               buckets (Sec. 3.2, Sec. 4.7) and planned a 16 + 15-bit
 *               global radix (Sec. 5).
 *   mode:       RS_MODE_LSD = least significant digit first (Sec. 3.3.1);
 *               RS_MODE_MSD = bucket by the top digit first, then sort each
 *               bucket locally (the bucketing + local sort pipeline of
 *               Sec. 3 / Sec. 4.6).
 *   tile:       1 + index of the kernel tile shape (0 = automatic).  8-bit
 *               digits: 1 = 512 threads x 16 keys and 3 = 512 x 24, ranked
 *               per warp through lane-mask tables (every payload layout);
 *               2 = 384 x 24, 5 = 512 x 24, 6 = 512 x 16 and 7 = 256 x 24,
 *               ranked per half-warp with early digit counts (keys and
 *               key + uint32 payload); 4 = 1024 x 16 and 8 = 384 x 24,
 *               lane-mask tables (keys and key + uint32 payload).
 *               11-bit digits: 1 to 4.  Automatic: 2 for keys; for
 *               key+payload sorts 1 up to 2^21 keys, then 8.
 *   key_kind:   how the 32-bit key words are ordered.  RS_KEY_U32: unsigned
 *               (the paper's integers, Sec. 1.1); RS_KEY_I32: two's-complement
 *               signed; RS_KEY_F32: IEEE-754 binary32 in the totalOrder of
 *               IEEE 754-2008 Sec. 5.10 (-NaN < -inf < ... < -0 < +0 < ... <
 *               +inf < +NaN, NaNs by payload).  Every entry point that takes
 *               a plan honours it; the output holds the input's words, only
 *               their order depends on the kind.  The passes run on an
 *               order-preserving unsigned map of each word (sign bit flipped;
 *               for negative binary32 values every bit) taken when a key is
 *               read from the input and undone when it is written to the
 *               output, so the work and traffic are those of unsigned keys. */
enum { RS_MODE_AUTO = 0, RS_MODE_LSD = 1, RS_MODE_MSD = 2 };
enum { RS_KEY_U32 = 0, RS_KEY_I32 = 1, RS_KEY_F32 = 2 };
typedef struct rs_plan {
  uint32_t digit_bits;
  uint32_t mode;
  uint32_t tile;
  uint32_t key_kind;
} rs_plan;

/* Sort n keys ascending into keys_out and write the num_parts + 1 partition
 * offsets (Sec. 1.1, footnote 7) to the HOST array h_part_offsets (may be
 * NULL if not wanted).  num_parts >= 1.  plan may be NULL (automatic).      */
rs_status rs_sort_u32(const uint32_t* keys_in, uint32_t* keys_out, uint64_t n,
                      uint32_t num_parts, uint64_t* h_part_offsets,
                      const rs_plan* plan, void* temp, size_t* temp_bytes,
                      rs_stream_t stream);

/* Stable sort of (key, value) pairs by key (Sec. 3.3.1: the earlier digits'
 * order is kept; Sec. 5: the order inside a bucket survives distribution).
 * Equal keys keep their input order.  Otherwise as rs_sort_u32.             */
rs_status rs_sort_u32_pairs(const uint32_t* keys_in, const uint32_t* vals_in,
                            uint32_t* keys_out, uint32_t* vals_out, uint64_t n,
                            uint32_t num_parts, uint64_t* h_part_offsets,
                            const rs_plan* plan, void* temp, size_t* temp_bytes,
                            rs_stream_t stream);

/* Many independent sorts in one call.  Segment s is
 * [d_seg_offsets[s], d_seg_offsets[s+1]) of the concatenated arrays
 * (DEVICE array of num_segs + 1 uint64, non-decreasing, last = total_n).
 * Each segment is sorted on its own (stably when vals_in != NULL; with
 * vals_in == NULL, vals_out must be NULL too).  d_part_offsets (DEVICE,
 * num_segs * (num_parts + 1) uint64, may be NULL) receives each segment's
 * partition offsets made absolute by adding the segment start.
 * h_seg_offsets is a HOST copy of the same offsets, used to plan the
 * launches (segment classes by size) without reading device memory.
 * plan: digit_bits 0 or 8; tile 1 (512 x 16 tiled passes), 2 (512 x 24
 * for keys, 512 x 22 with payloads) or 3 (384 x 20, three blocks per SM);
 * mode MSD or automatic (every segment
 * of up to 16,384 keys is sorted by one block in shared memory, larger ones
 * by tiled passes) or LSD (only segments of up to 4,096 keys go to the
 * one-block sort); key_kind as for rs_sort_u32.  Zero fields take the plan
 * installed for the batch's size class (rs_set_default_plan), else the
 * compiled defaults (tile 3, automatic).                                    */
rs_status rs_sort_u32_segmented(const uint32_t* keys_in, const uint32_t* vals_in,
                                uint32_t* keys_out, uint32_t* vals_out,
                                const uint64_t* d_seg_offsets,
                                const uint64_t* h_seg_offsets, uint32_t num_segs,
                                uint64_t total_n, uint32_t num_parts,
                                uint64_t* d_part_offsets, const rs_plan* plan,
                                void* temp, size_t* temp_bytes, rs_stream_t stream);

/* ---- single steps of the method, for step-by-step checking ------------- */

/* The count loop of Sec. 3.2 for every digit of a digit_bits-wide plan in
 * one read of the keys, plus the exclusive cumulative totals (Sec. 3.2,
 * Sec. 4.4).  With D = ceil(32 / digit_bits) digits and B = 2^digit_bits:
 *   d_hist [D][B] (DEVICE uint32): keys per bucket of each digit;
 *   d_bases[D][B] (DEVICE uint32, may be NULL): keys with a smaller digit;
 *   d_skip [D]    (DEVICE uint32, may be NULL): 1 when one bucket of that
 *                 digit holds all n keys (the pass would move nothing).
 * Digit j covers bits [j * digit_bits, min(32, (j + 1) * digit_bits)).
 * digit_bits must be 8 or 11.  Needs no temp.                               */
rs_status rs_digit_histograms(const uint32_t* keys, uint64_t n, uint32_t digit_bits,
                              uint32_t* d_hist, uint32_t* d_bases, uint32_t* d_skip,
                              rs_stream_t stream);

/* One stable distribution of (keys, vals) by the digit of `width` bits at
 * `shift` (the partial sort of Sec. 3.2; one pass of Sec. 3.3.1):
 * keys grouped by digit value, in ascending order, input order kept within
 * a digit value.  vals_in/vals_out may both be NULL.  width must be 1..11
 * and shift + width <= 32.  Temp as for the sorts.                          */
rs_status rs_radix_pass(const uint32_t* keys_in, const uint32_t* vals_in,
                        uint32_t* keys_out, uint32_t* vals_out, uint64_t n,
                        uint32_t shift, uint32_t width, void* temp,
                        size_t* temp_bytes, rs_stream_t stream);

/* rs_sort_u32_pairs with 64-bit values (vals_in, vals_out: DEVICE, n uint64
 * each, 8-byte aligned): stable by key.  Every pass carries the value's low
 * and high 32-bit words as two payload words per key (word planes in temp
 * between passes); the first pass reads the interleaved values and the last
 * writes them.  plan: LSD with 8-bit digits (0 fields are fine); key_kind as
 * for the other sorts.  Temp: the key+payload temp plus three n-word planes. */
rs_status rs_sort_u32_pairs64(const uint32_t* keys_in, const uint64_t* vals_in,
                              uint32_t* keys_out, uint64_t* vals_out, uint64_t n,
                              uint32_t num_parts, uint64_t* h_part_offsets,
                              const rs_plan* plan, void* temp, size_t* temp_bytes,
                              rs_stream_t stream);

/* ---- 64-bit keys ------------------------------------------------------- */

/* Sort n 64-bit keys ascending (keys_in, keys_out: DEVICE, n uint64 each,
 * 8-byte aligned, not overlapping) and write the partition offsets as for
 * rs_sort_u32.  No counterpart in the paper, whose keys are 32-bit (Sec. 1.1);
 * the method is the same LSD radix distribution (Sec. 3.3.1) with eight
 * 8-bit digits.  Between passes the keys are held as planes of low and
 * high 32-bit words; each pass moves both words, the low word serving as the
 * key for digits 0-3 and the high word for digits 4-7.  plan: digit_bits must be 0
 * or 8, mode LSD (or 0), tile selects the key+payload tile shape, and
 * key_kind orders the 64-bit words as unsigned (RS_KEY_U32), two's-complement
 * signed (RS_KEY_I32) or IEEE-754 binary64 totalOrder (RS_KEY_F32).  Temp:
 * four n-word planes (six with the tile shapes other than 1 and 3, which
 * split the keys into planes first) plus histograms and status.  The
 * default tile is 3 above 2^22 keys (below 2^30 - 2^16), else 1.           */
rs_status rs_sort_u64(const uint64_t* keys_in, uint64_t* keys_out, uint64_t n,
                      uint32_t num_parts, uint64_t* h_part_offsets,
                      const rs_plan* plan, void* temp, size_t* temp_bytes,
                      rs_stream_t stream);

/* ---- merging sorted runs ------------------------------------------------- */

/* Stable merge of two runs already sorted in the order of plan->key_kind
 * (plan may be NULL: unsigned): out[0, na + nb) receives a[0, na) and
 * b[0, nb) in ascending order, an element of a before an equal one of b, and
 * the partition offsets of the merged array go to h_part_offsets as for
 * rs_sort_u32.  The merge at the heart of the paper's cleanup merge-exchange
 * (Sec. 3.4.2, Sec. 4.6).  a, b, out (and va, vb, vout: all three or none;
 * an empty run may pass NULL) are DEVICE arrays of uint32 words; outputs must
 * not overlap inputs.
 * plan->tile picks the merge tile shape (1..4; 0 = automatic); other plan
 * fields are ignored.  Runs that are not sorted give an
 * unspecified order; a tile whose merge path comes out inconsistent is left
 * unwritten and rs_check_device_error() reports it.  Temp: 4 bytes per tile
 * of 2816 to 5888 outputs.                                                  */
rs_status rs_merge_u32(const uint32_t* a, const uint32_t* va, uint64_t na,
                       const uint32_t* b, const uint32_t* vb, uint64_t nb,
                       uint32_t* out, uint32_t* vout, uint32_t num_parts,
                       uint64_t* h_part_offsets, const rs_plan* plan, void* temp,
                       size_t* temp_bytes, rs_stream_t stream);

/* rs_sort_u64 with a uint32 value per key (vals_in, vals_out: DEVICE, n
 * each): stable by key.  Each pass moves three words per key (both key words
 * and the value); the values go straight from vals_in to vals_out.         */
rs_status rs_sort_u64_pairs(const uint64_t* keys_in, const uint32_t* vals_in,
                            uint64_t* keys_out, uint32_t* vals_out, uint64_t n,
                            uint32_t num_parts, uint64_t* h_part_offsets,
                            const rs_plan* plan, void* temp, size_t* temp_bytes,
                            rs_stream_t stream);

/* rs_sort_u64 with a uint64 value per key (vals_in, vals_out: DEVICE, n
 * each, 8-byte aligned, not overlapping the keys or each other): stable by
 * key.  The passes carry each key's input index in place of its value (the
 * first pass makes it, the last reads vals_in at it and writes the value to
 * vals_out), so each pass moves three words per key as in rs_sort_u64_pairs.
 * plan as for rs_sort_u64; tile shapes without an interleaved
 * two-payload-word kernel (all but the default, 1) give RS_ERR_UNSUPPORTED.  Temp:
 * rs_sort_u64_pairs's plus one n-word plane.                                */
rs_status rs_sort_u64_pairs64(const uint64_t* keys_in, const uint64_t* vals_in,
                              uint64_t* keys_out, uint64_t* vals_out, uint64_t n,
                              uint32_t num_parts, uint64_t* h_part_offsets,
                              const rs_plan* plan, void* temp, size_t* temp_bytes,
                              rs_stream_t stream);

/* ---- host buffers ------------------------------------------------------- */

/* rs_sort_u32 / rs_sort_u32_pairs on HOST arrays: the keys (and values) are
 * copied into device buffers carved from temp, sorted there, and copied back
 * into h_keys_out (and h_vals_out), all enqueued on `stream` in that order.
 * No counterpart in the paper (its keys were already in the cells' memory).
 *   h_keys_in, h_keys_out: HOST, n uint32 each; h_vals_in, h_vals_out: HOST,
 *     n uint32 each, or both NULL for a keys-only sort.  The host outputs
 *     must not overlap the host inputs.
 *   temp: DEVICE; its size (query with temp == NULL) is that of the device
 *     sort plus 2 (keys only) or 4 (pairs) buffers of n uint32.
 * Page-locked host memory (cudaHostAlloc, cudaHostRegister) makes the
 * copies asynchronous; with pageable memory they still run in stream order,
 * but the CUDA runtime may block the caller during them.  The host outputs
 * are complete once the stream has passed the call's work (synchronise it or
 * wait on an event recorded after the call).  Calls on different streams,
 * each with its own temp, overlap on the GPU: one call's device-to-host copy
 * runs while the next one copies in and sorts, which keeps the host link
 * busy in both directions when a stream of host arrays is sorted.          */
rs_status rs_sort_u32_host(const uint32_t* h_keys_in, const uint32_t* h_vals_in,
                           uint32_t* h_keys_out, uint32_t* h_vals_out, uint64_t n,
                           uint32_t num_parts, uint64_t* h_part_offsets,
                           const rs_plan* plan, void* temp, size_t* temp_bytes,
                           rs_stream_t stream);

/* ---- sorting without any device allocation ------------------------------ */

/* Largest n accepted by rs_sort_u32_noalloc. */
#define RS_NOALLOC_MAX_KEYS (1u << 20)

/* The keys-only sort of rs_sort_u32 for callers that cannot allocate device
 * memory: code inside a host program that owns every allocation and offers
 * no allocator, latency-critical code that cannot afford cudaMalloc's
 * possible device-wide synchronisation, code that must not hit
 * out-of-memory once running.  No counterpart in the paper.
 *
 * The caller still owns keys_in and keys_out (device, n keys each) and
 * h_part_offsets (host, num_parts + 1, may be NULL).  Scratch comes from a
 * fixed array of about 4.5 MiB inside the library's device memory, held on
 * every GPU that uses it until the process exits; nothing is allocated or
 * freed by the call.  n above RS_NOALLOC_MAX_KEYS is rejected with
 * RS_ERR_INVALID before any work.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); under CUDA's lazy module
 * loading (the default) that lookup is also what loads the array onto the
 * device, so the first call can still fail for lack of device memory.  Make
 * that first call during set-up (n = 0 does the set-up and sorts nothing)
 * and before any stream capture.  All calls on a device share the array:
 * calls whose work overlaps on the GPU (e.g. on two streams) race and must
 * be serialised by the caller.  Results are identical to rs_sort_u32's.   */
rs_status rs_sort_u32_noalloc(const uint32_t* keys_in, uint32_t* keys_out, uint64_t n,
                              uint32_t num_parts, uint64_t* h_part_offsets,
                              rs_stream_t stream);

/* ---- data-adaptive plan choice (Sec. 4.2.1) ------------------------------- */

/* The selection step of Sec. 4.2.1 on DEVICE keys (n of them, key words of
 * key_kind): an evenly spaced sample of s = min(sample, n) keys (positions
 * floor(i * n / s); the paper used 1000 points, footnote 8), each bucketed
 * by the top `bits` bits of the sample's significant width (in the order of
 * key_kind); the sorted sample buckets stand for the bucketed output and are
 * split into `cells` equal ranges of sample ranks (cell c: [c*s/cells,
 * (c+1)*s/cells)).  A cell whose sampled elements are not above its left
 * neighbour's maximum bucket for 65 % or more of them (100 * overlap >=
 * 65 * size) is a problem cell.  h_out (HOST, 4 words): problem cells,
 * 1 if they are more than max_problem (clustered data), the bucket shift,
 * s.  d_buckets (DEVICE, s words, may be NULL) receives the sorted sample
 * buckets.  Limits: 1 <= sample <= 1024, 1 <= cells <= 1024, 1 <= bits <=
 * 32.  Synchronises `stream`.  One selection runs at a time per process.  */
rs_status rs_sample_overlap(const uint32_t* keys, uint64_t n, uint32_t key_kind, uint32_t bits,
                            uint32_t sample, uint32_t cells, uint32_t max_problem,
                            uint32_t* d_buckets, uint32_t* h_out, rs_stream_t stream);

/* The plan rs_sort_u32 would run for these keys, chosen from the data: the
 * caller's plan `base` resolved like rs_sort_u32's (installed or compiled
 * defaults for zero fields), then the selection of Sec. 4.2.1 with the
 * paper's parameters (1000-point sample, 64 cells, 65 %, more than two
 * problem cells; buckets of the top 13 significant bits).  Clustered data
 * turns a bucketing (MSD) plan into LSD, as the paper abandoned its
 * bucketing algorithm for the clustered data set; other plans are kept.
 * *out receives the plan, h_stats (HOST, 4 words, may be NULL) the
 * selection's words as for rs_sample_overlap.  Synchronises `stream`.     */
rs_status rs_choose_plan(const uint32_t* keys, uint64_t n, const rs_plan* base, rs_plan* out,
                         uint32_t* h_stats, rs_stream_t stream);

/* ---- default plans (autotuning) ------------------------------------------ */

/* Entry points whose plan can be installed per size class. */
enum {
  RS_ENTRY_SORT_U32 = 0,         /* rs_sort_u32 and rs_sort_u32_host without payloads */
  RS_ENTRY_SORT_U32_PAIRS = 1,   /* rs_sort_u32_pairs and rs_sort_u32_host with payloads */
  RS_ENTRY_SEGMENTED = 2,        /* rs_sort_u32_segmented, keys only */
  RS_ENTRY_SEGMENTED_PAIRS = 3   /* rs_sort_u32_segmented with payloads */
};

/* Installs the plan that `entry` uses for size class `size_class` (0..32)
 * when the caller passes plan = NULL or leaves a field zero: the class of a
 * plain sort of n keys is ceil(log2(n)), that of a segmented sort
 * ceil(log2(mean segment size)).  plan = NULL removes the entry (the
 * compiled defaults apply again).  key_kind must be RS_KEY_U32 (the kind
 * always comes from the caller).  This is how the project's autotuner
 * (paper_cs_0004013_gb300/tune.py, which times the candidates on the GPU in
 * use) hands its choices of digit width, tile shape and MSD or LSD to the
 * library; the paper chose its algorithm per data set by measurement too
 * (Sec. 4.2).  Host-only; thread-safe.  For rs_sort_u32_segmented, tile is
 * 1 (512 x 16 tiled passes), 2 (512 x 24 for keys, 512 x 22 with
 * payloads) or 3 (384 x 20, the default) and mode LSD sends only segments
 * of up to 4,096
 * keys to the one-block sort, MSD or automatic every segment up to 16,384. */
rs_status rs_set_default_plan(uint32_t entry, uint32_t size_class, const rs_plan* plan);

/* The installed plan of (entry, size_class): *is_set = 1 and *out = the plan,
 * or *is_set = 0 and *out zeroed.                                          */
rs_status rs_get_default_plan(uint32_t entry, uint32_t size_class, rs_plan* out, int* is_set);

/* ---- errors ------------------------------------------------------------- */

/* Message for the last error raised on the calling thread ("" if none). */
const char* rs_last_error(void);

/* After the work already enqueued on `stream`, takes and clears the device
 * error word of the current device in one atomic step (a one-thread kernel
 * on the stream), waits for the stream and reports what it took:
 * RS_ERR_TIMEOUT if a kernel's bounded wait (the cross-tile lookback) gave
 * up since the last check; RS_ERR_CUDA if the stream failed or a kernel's
 * output-index check fired (the write was skipped); else RS_OK.  The error
 * word is shared by all streams of the device: a bit raised by a kernel on
 * another stream is reported by whichever check takes it first, and a bit
 * raised after this check's take is kept for the next one.                 */
rs_status rs_check_device_error(rs_stream_t stream);

/* Enqueues on `stream`, after its earlier work, a copy of the current
 * device's error word into *h_word (HOST, 4 bytes; pinned memory keeps the
 * copy asynchronous) without clearing it, and returns at once: no kernel,
 * no wait.  *h_word is valid once the stream's later events complete.  A
 * nonzero word says that some kernel of the device raised an error bit
 * since the last rs_check_device_error() (which takes and clears it): bit 0
 * (1) a bounded wait gave up, bit 1 (2) an output-index check fired.  Zero
 * says that none had by the time of the copy.  Meant for callers that keep
 * many streams busy and must not wait on each one.                        */
rs_status rs_peek_device_error_async(uint32_t* h_word, rs_stream_t stream);

/* ---- tracing ------------------------------------------------------------ */

/* Per-kernel timing.  While enabled, every kernel the library launches is
 * bracketed by two CUDA events recorded on the launch's stream (the events
 * are created on first use and kept for reuse; enabling costs two event
 * records per launch and no synchronisation).                              */
typedef struct rs_trace_entry {
  char name[32];      /* kernel kind: "upfront_hist", "digit_scan",
                         "onesweep_r8", "onesweep_r11", "clear", ...        */
  uint32_t launches;  /* launches of this kind since the last read         */
  uint32_t reserved;
  double total_ms;    /* sum of their event-to-event times                 */
  double keys;        /* sum of the keys each launch processed             */
} rs_trace_entry;

rs_status rs_trace_enable(int on);

/* Waits for every traced launch, writes up to `capacity` entries (one per
 * kernel kind seen) and resets the trace.  *count = entries written.       */
rs_status rs_trace_read(rs_trace_entry* out, uint32_t capacity, uint32_t* count);

/* Self-test of failure detection: runs the pass kernels' cross-tile wait
 * (the lookback) against a status row that nothing ever publishes, in
 * temp (DEVICE, >= 4096 bytes, 256-byte aligned; cleared here).  The wait
 * gives up after its bounded number of rounds (tens of milliseconds), raises
 * the device error word and returns, so the next rs_check_device_error()
 * reports RS_ERR_TIMEOUT and the context stays usable.                     */
rs_status rs_selftest_wait_timeout(void* temp, size_t temp_bytes, rs_stream_t stream);

/* Library version as MAJOR * 10000 + MINOR * 100 + PATCH. */
uint32_t rs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RSORT_H */
