/*
 * ss.h -- C ABI of the GB300 string sample sorter (libss_gb300.so).
 *
 * Sorts n byte strings lexicographically and returns the sorted permutation
 * and the LCP array, following the problem statement of Section 2 of
 * Bingmann, Eberle, Sanders, "Engineering Parallel String Sorting": strings
 * over the alphabet {1..255} (unsigned bytes, no 0 byte inside a string),
 * ordered character by character with the end of a string below every
 * character.  The method is super scalar string sample sort (Section 4.3,
 * Algorithm 1) with LCP saving (Section 5.4) and LCP-aware merging of sorted
 * runs (Section 5.1-5.3, Algorithms 2-4), run on one GPU.
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are DEVICE pointers owned by the caller; the
 *     library never frees or retains them past the call.  Pointers named
 *     *_host are host pointers.
 *   - `stream` is a cudaStream_t (may be NULL for the legacy default stream).
 *     Work is ordered on that stream.  ss_sort_batch_async only queues its
 *     sort on `stream` and returns: the recursion is driven on the device (a
 *     scheduler kernel launches every level's kernels from the device, the
 *     paper's job queue of Section 4.5 kept in device memory), outputs are
 *     complete when `stream` reaches that point, and a device-side failure is
 *     written to each request's status_out and recorded for ss_device_error.
 *     The other sort entry points drive the levels from the host, reading a
 *     few counters back between levels, and return when the sort is done: on
 *     GB300 that measured faster at every size (kernels launched from the
 *     device start about 12 us after the one before).  ss_merge, ss_merge_ex,
 *     ss_autotune and the single-step entry points return when done.
 *   - Scratch memory comes from a stream-ordered pool owned by the library
 *     (one per device, kept between calls); it is returned to the pool at the
 *     end of each call.
 *   - Output conventions (the reading taken where the paper is silent):
 *     perm_out[i] = input index of the i-th smallest string; equal strings
 *     appear in ascending input index; lcp_out[0] = 0 and lcp_out[i] =
 *     lcp(s_{perm[i-1]}, s_{perm[i]}) for i >= 1, the LCP stopping at the end
 *     of the shorter string.
 *   - Return value: SS_OK, or a negative ss_status.  On error
 *     ss_last_error_detail() gives a message for the calling thread.  Outputs
 *     are unspecified after an error.
 *   - Reads of string bytes are aligned 8-byte words in a 4 KiB page that
 *     holds at least one byte of the string being read (or of its
 *     terminator), so no read touches a page the strings do not touch.
 *     A 16-byte aligned offsets array may be read in whole 16-byte blocks
 *     (at most 8 bytes past its last entry, in the same block).
 */
#ifndef SS_GB300_H
#define SS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *ss_stream_t; /* identical to cudaStream_t */

typedef enum {
    SS_OK = 0,
    SS_ERR_INVALID = -1,       /* bad argument (NULL pointer with n > 0, bad K, ...) */
    SS_ERR_OOM = -2,           /* scratch allocation failed */
    SS_ERR_CUDA = -3,          /* a CUDA call or launch failed */
    SS_ERR_TIMEOUT = -4,       /* a bounded device-side wait gave up */
    SS_ERR_TOO_LARGE = -5,     /* n or a total beyond 2^32 - 2 */
    SS_ERR_UNIMPLEMENTED = -6, /* feature not available in this build */
    SS_ERR_INTERNAL = -7,      /* a device-side consistency check failed */
    SS_ERR_CANCELLED = -8      /* a queued server request was cancelled before it started */
} ss_status;

/*
 * ss_sort -- sort n NUL-terminated strings (Section 2; Algorithm 1 applied
 * recursively, Section 4.5; LCP saving, Section 5.4).
 *   chars_dev   : string bytes; string i starts at chars_dev[offsets_dev[i]]
 *                 and ends at the first 0 byte (the terminator).
 *   offsets_dev : uint64[n], byte offset of each string.
 *   n           : number of strings, 0 <= n <= 2^32 - 2; n = 0 is a no-op.
 *   perm_out_dev: uint32[n] output, sorted permutation.
 *   lcp_out_dev : uint32[n] output, LCP array.
 * Strings must be shorter than 2^32 - 16 bytes.
 */
int ss_sort(const uint8_t *chars_dev, const uint64_t *offsets_dev, uint32_t n,
            uint32_t *perm_out_dev, uint32_t *lcp_out_dev, ss_stream_t stream);

/*
 * ss_sort_ex -- as ss_sort for strings delimited by length instead of a
 * terminator (for example overlapping windows of one text).
 *   lengths_dev : uint32[n] string lengths, or NULL;
 *   fixed_len   : when lengths_dev is NULL and fixed_len > 0, every string
 *                 has exactly fixed_len bytes; when both are 0/NULL the
 *                 strings are NUL-terminated as in ss_sort.
 * Strings must not contain the byte 0 (the paper's alphabet is {1..sigma}).
 */
int ss_sort_ex(const uint8_t *chars_dev, const uint64_t *offsets_dev, const uint32_t *lengths_dev,
               uint32_t fixed_len, uint32_t n, uint32_t *perm_out_dev, uint32_t *lcp_out_dev,
               ss_stream_t stream);

/*
 * ss_sort_host -- ss_sort_ex for HOST buffers: copies the strings to the
 * device, sorts, copies perm and lcp back, and returns when they are in the
 * host arrays.  chars_len_host is the number of bytes of chars_host to copy
 * (every string and terminator must lie inside it).  Host buffers may be
 * pageable or pinned; pinned buffers copy faster.
 *   runs : 0 or 1 sorts the set in one piece.  runs = K > 1 sorts K
 *          index-contiguous runs together (as one ss_sort_batch) and merges
 *          them with ss_merge, the paper's "independent sorters, then LCP
 *          merge" structure (Section 5); the result is the same.
 */
int ss_sort_host(const uint8_t *chars_host, uint64_t chars_len_host, const uint64_t *offsets_host,
                 const uint32_t *lengths_host, uint32_t fixed_len, uint32_t n, uint32_t runs,
                 uint32_t *perm_out_host, uint32_t *lcp_out_host, ss_stream_t stream);

/*
 * One independent sort request of a batch.  Fields as in ss_sort_ex; all
 * pointers are device pointers.  status_out may be NULL; otherwise the
 * library writes an int32 ss_status there on the device, in stream order:
 * SS_OK when the request's outputs are complete, SS_ERR_TIMEOUT when a
 * bounded device-side wait of the batch gave up, SS_ERR_INTERNAL when a
 * device-side check of the batch failed.  Argument errors are reported by
 * the return value alone, before anything is written.
 */
typedef struct {
    const uint8_t *chars;
    const uint64_t *offsets;
    const uint32_t *lengths;
    uint32_t fixed_len;
    uint32_t n;
    uint32_t *perm_out;
    uint32_t *lcp_out;
    int32_t *status_out;
} ss_request;

/*
 * ss_sort_batch -- sort `count` independent requests together (host array
 * reqs_host).  All requests advance through the same recursion levels in
 * the same kernel launches (the paper's job queue of independent
 * subproblems, Section 4.5, moved onto the device).  The sum of all n must
 * not exceed 2^32 - 2.  Results equal those of one ss_sort_ex per request.
 */
int ss_sort_batch(const ss_request *reqs_host, uint32_t count, ss_stream_t stream);

/*
 * Classifiers: how each key finds its bucket in the splitter tree (Section
 * 4.4 weighs where the equality test goes; Section 8.1 proposes jump tables).
 *   SS_CLASSIFIER_UNROLL  descents with > only, four interleaved per thread,
 *                         then one equality test against the in-order
 *                         splitters (S5-Unroll, the paper's choice; default)
 *   SS_CLASSIFIER_EQUAL   one descent per key testing equality at every node
 *                         and leaving the tree at the first equal splitter
 *                         (S5-Equal)
 *   SS_CLASSIFIER_JUMP    a table over the 10 key bits after the splitters'
 *                         common prefix gives the node where the descent
 *                         starts to depend on later bits; the descent goes on
 *                         from there as SS_CLASSIFIER_UNROLL
 * All three give the bucket 2r + [x_r = c], r = #{j : x_j < c}, except that
 * S5-Equal puts a key equal to a repeated splitter value into the equality
 * bucket of the copy highest in the tree; no sort result depends on it.
 */
#define SS_CLASSIFIER_UNROLL 0u
#define SS_CLASSIFIER_EQUAL 1u
#define SS_CLASSIFIER_JUMP 2u

/*
 * Tuning of one request (0 fields: the library's defaults).  child_target:
 * the segment size the splitter tree aims its children at (a power of two in
 * [32, 65536]; the tree has about size / child_target leaves, at most 256);
 * min_step: the smallest depth step an even bucket takes (in [1, 9]; 9: it
 * never steps and keeps its key); classifier: one of SS_CLASSIFIER_*.
 * alphabet: alphabet compression (Section 8.1) for a request of fixed-length
 * strings (lengths NULL, fixed_len > 0) whose characters all belong to an
 * alphabet of at most four bytes: SS_ALPHABET(a0, a1, a2, a3) with
 * 1 <= a0 <= a1 <= a2 <= a3 (repeat the last byte for fewer), e.g.
 * SS_ALPHABET('A', 'C', 'G', 'T').  Keys then hold 32 characters of 2 bits
 * instead of 8 bytes; depths and LCPs stay in characters.  The library does
 * not check the strings' bytes: a byte outside the alphabet gives an
 * unspecified order.  0: bytes.  max_depth: the largest splitter-tree depth
 * of one distribution level (v = 2^max_depth - 1 splitters), in [2, 8];
 * 0: 8.  small_max: segments of at most this many strings go to the base
 * case, larger ones to another distribution level; a power of two in
 * [64, 2048]; 0: 2048.  The sort's scratch holds about 10 KiB (a segment's
 * splitters, jump table and records) per small_max + 1 strings of the batch's
 * smallest small_max.
 * None of the fields changes any result.
 */
typedef struct {
    uint32_t child_target;
    uint32_t min_step;
    uint32_t classifier;
    uint32_t alphabet;
    uint32_t max_depth;
    uint32_t small_max;
} ss_tuning;

#define SS_ALPHABET(a0, a1, a2, a3) \
    ((uint32_t)(uint8_t)(a0) | ((uint32_t)(uint8_t)(a1) << 8) | ((uint32_t)(uint8_t)(a2) << 16) | \
     ((uint32_t)(uint8_t)(a3) << 24))

/*
 * ss_sort_batch_tuned -- ss_sort_batch with one tuning per request
 * (tunings_host: `count` entries, or NULL for the defaults).  SS_ERR_INVALID
 * for a tuning outside the ranges above.
 */
int ss_sort_batch_tuned(const ss_request *reqs_host, const ss_tuning *tunings_host, uint32_t count,
                        ss_stream_t stream);

/*
 * ss_sort_batch_async -- ss_sort_batch_tuned (tunings_host may be NULL) that
 * returns as soon as the sort is queued on `stream`, with no host wait inside:
 * every recursion level is launched from the device by a scheduler kernel,
 * from the segment and task lists in device memory.  Results are those of
 * ss_sort_batch.  Each request's status_out (if given) receives SS_OK,
 * SS_ERR_TIMEOUT or SS_ERR_INTERNAL in stream order; ss_device_error reports
 * a failure of any request afterwards.  While kernel timing is on
 * (ss_profile_enable) it behaves as ss_sort_batch_tuned.
 */
int ss_sort_batch_async(const ss_request *reqs_host, const ss_tuning *tunings_host, uint32_t count,
                        ss_stream_t stream);

/*
 * Distinguishing characters a sort hands to a later LCP merge (Section 5.4:
 * the merge caches characters at each string's LCP; the sorter has already
 * loaded them).  Device arrays of a request's n entries, written by the
 * sort, per sorted position p:
 *   off_out[p] = offsets[perm_out[p]];
 *   ck_out[p]  = 8 characters of that string from depth ckd_out[p]
 *                (big-endian, zero past its end), where
 *                ckd_out[p] <= lcp_out[p] < ckd_out[p] + 8 or the string
 *                ends before ckd_out[p] + 8 (position 0: depth 0).
 * All three NULL: not written.
 */
typedef struct {
    uint64_t *off_out;
    uint64_t *ck_out;
    uint32_t *ckd_out;
} ss_sort_cache;

/*
 * ss_sort_batch_cached -- ss_sort_batch_tuned (tunings_host may be NULL)
 * that also writes each request's caches (caches_host: `count` entries, or
 * NULL for none) for ss_merge_cached.  Results and completion as
 * ss_sort_batch_tuned.  SS_ERR_INVALID for a cache with only some of its
 * arrays, or on a request with alphabet compression (caches hold bytes).
 */
int ss_sort_batch_cached(const ss_request *reqs_host, const ss_tuning *tunings_host,
                         const ss_sort_cache *caches_host, uint32_t count, ss_stream_t stream);

/*
 * ss_autotune -- picks a tuning for inputs like `req`'s: sorts its first
 * min(n, sample_n) strings (sample_n = 0: 2,000,000) with each of 22 or 23
 * candidate tunings, each step keeping the fastest so far: child_target
 * 256..2048 x min_step 1, 3, 5, 9 with the default classifier; that shape
 * with SS_CLASSIFIER_EQUAL and SS_CLASSIFIER_JUMP; max_depth 6 and 7;
 * small_max 512 and 1024; and, for fixed-length strings whose sampled bytes
 * are at most four non-zero values, the alphabet of those bytes (keys of 32
 * two-bit characters instead of 8 bytes).  Each runs once to warm and once
 * timed with CUDA events on
 * `stream`, into scratch it allocates (req's outputs are not touched), and
 * writes the fastest to *best_out and its time in ms to *best_ms_out (may be
 * NULL).  Returns when done.
 */
int ss_autotune(const ss_request *req_host, uint32_t sample_n, ss_tuning *best_out, double *best_ms_out,
                ss_stream_t stream);

/*
 * ss_merge -- LCP-aware merge of K sorted runs of one string set
 * (Sections 5.1-5.3: LCP-Compare, Algorithm 2; binary LCP-merge,
 * Algorithm 3; the K-way merge is done as ceil(log2 K) rounds of pairwise
 * merges partitioned by merge path).
 *   chars_dev/offsets_dev/lengths_dev/fixed_len : the string set, as ss_sort_ex.
 *   run_perm_dev : uint32[total]; run k is positions
 *                  [run_begin_host[k], run_begin_host[k+1]), sorted.  Its
 *                  entries plus run_base_host[k] are string indices of the set.
 *   run_lcp_dev  : uint32[total] LCP array of each run (entry at a run's
 *                  first position is ignored).
 *   run_begin_host : uint32[K+1] on the host, non-decreasing, [0] = 0.
 *   run_base_host  : uint32[K] on the host, or NULL for all zero (for runs
 *                  sorted by ss_sort_batch with request-local indices: the
 *                  index of each run's first string).
 *   K            : number of runs, 1 <= K.
 *   perm_out_dev/lcp_out_dev : uint32[total] merged order (string indices of
 *                  the set) and its LCP array; must not overlap the inputs.
 * Equal strings from different runs are ordered by run number.  The input
 * arrays are not modified.
 */
int ss_merge(const uint8_t *chars_dev, const uint64_t *offsets_dev, const uint32_t *lengths_dev,
             uint32_t fixed_len, const uint32_t *run_perm_dev, const uint32_t *run_lcp_dev,
             const uint32_t *run_begin_host, const uint32_t *run_base_host, uint32_t K,
             uint32_t *perm_out_dev, uint32_t *lcp_out_dev, ss_stream_t stream);

/* merge methods of ss_merge_ex */
#define SS_MERGE_PAIRWISE 0u    /* ceil(log2 K) rounds of pairwise LCP merges (ss_merge's method) */
#define SS_MERGE_LOSER_TREE 1u  /* one pass with an LCP loser tree per job, up to 8 runs */

/*
 * ss_merge_ex -- ss_merge with the merge method chosen (same arguments,
 * order, results and completion; the output is the same for every method).
 *   method : SS_MERGE_PAIRWISE -- as ss_merge.
 *            SS_MERGE_LOSER_TREE -- the K-way LCP-merge of Algorithm 4
 *            (Section 5.2) in one pass: the output is cut into jobs at
 *            splitter strings taken from the runs (every 128th string of
 *            every run, placed in the other runs by binary search, Section
 *            5.3), and each job is merged by one thread with an LCP-aware
 *            tournament tree (LCP-Compare, Algorithm 2, with the cached
 *            characters of Section 5.4).  Applies to 2..8 non-empty runs;
 *            with more, the pairwise rounds are used.
 *   Errors: as ss_merge; an unknown method returns SS_ERR_INVALID.
 */
int ss_merge_ex(const uint8_t *chars_dev, const uint64_t *offsets_dev, const uint32_t *lengths_dev,
                uint32_t fixed_len, const uint32_t *run_perm_dev, const uint32_t *run_lcp_dev,
                const uint32_t *run_begin_host, const uint32_t *run_base_host, uint32_t K, uint32_t method,
                uint32_t *perm_out_dev, uint32_t *lcp_out_dev, ss_stream_t stream);

/*
 * ss_merge_cached -- ss_merge (pairwise rounds) of runs that a sort wrote
 * with their caches (ss_sort_batch_cached, one request per run): run_off,
 * run_ck, run_ckd are the runs' caches laid out as run_perm (run k at
 * run_begin_host[k]).  The merge starts from them instead of loading every
 * entry's string offset and characters itself.  Same results, completion
 * and errors as ss_merge; NULL cache arrays return SS_ERR_INVALID.
 */
int ss_merge_cached(const uint8_t *chars_dev, const uint64_t *offsets_dev, const uint32_t *lengths_dev,
                    uint32_t fixed_len, const uint32_t *run_perm_dev, const uint32_t *run_lcp_dev,
                    const uint64_t *run_off_dev, const uint64_t *run_ck_dev, const uint32_t *run_ckd_dev,
                    const uint32_t *run_begin_host, const uint32_t *run_base_host, uint32_t K,
                    uint32_t *perm_out_dev, uint32_t *lcp_out_dev, ss_stream_t stream);

/*
 * ss_merge_noalloc -- ss_merge that allocates nothing, for callers that
 * cannot let a library allocate: a process whose device memory is reserved
 * up front by its own arena, code held to a hard memory budget, or a
 * latency-critical path that must not pay for cudaMalloc/cudaFree or pinned
 * host allocations.  The paper has no counterpart; this is a deployment
 * variant of the merge above, with the same arguments, order and results.
 *   Limits: at most 1,048,576 strings in total and at most 64 runs; larger
 *   requests return SS_ERR_TOO_LARGE with a message (use ss_merge).
 *   Memory: its temporary arrays live in a fixed device array of about
 *   8 MiB inside the library image, held by every GPU that loads the
 *   library until the process exits.  Every call on a device shares that
 *   array: calls that overlap on the GPU (unordered streams or threads)
 *   race and give wrong results, so order them on one stream.
 *   Set-up: every call looks up the array's device address with the
 *   current device (a lookup, no allocation); the first call on a device
 *   may load the library's module there, so make that first call before
 *   any stream capture.
 *   Completion: the call only queues work on `stream` and returns; results
 *   are complete when the stream reaches that point.
 */
int ss_merge_noalloc(const uint8_t *chars_dev, const uint64_t *offsets_dev, const uint32_t *lengths_dev,
                     uint32_t fixed_len, const uint32_t *run_perm_dev, const uint32_t *run_lcp_dev,
                     const uint32_t *run_begin_host, const uint32_t *run_base_host, uint32_t K,
                     uint32_t *perm_out_dev, uint32_t *lcp_out_dev, ss_stream_t stream);

/*
 * ss_gather_keys -- chars_h (Section 4.4): for each string i, the 8 bytes at
 * depth depth_dev[i] as a big-endian uint64 (first character in the most
 * significant byte), bytes past the end of the string zero.
 *   depth_dev : uint32[n] depths (each at most the string's length).
 *   keys_out_dev : uint64[n].
 */
int ss_gather_keys(const uint8_t *chars_dev, const uint64_t *offsets_dev, const uint32_t *lengths_dev,
                   uint32_t fixed_len, uint32_t n, const uint32_t *depth_dev, uint64_t *keys_out_dev,
                   ss_stream_t stream);

/*
 * ss_splitters -- splitter selection of Section 4.4 on the device: sort the
 * sample (a keys) and pick v = 2^d - 1 in-order splitters with the recursive
 * scheme that skips samples equal to the chosen middle splitter.
 *   sample_dev : uint64[a], 1 <= a <= 2047; d in [1, 10].
 *   x_out_dev  : uint64[2^d - 1], sorted splitters.
 */
int ss_splitters(const uint64_t *sample_dev, uint32_t a, uint32_t d, uint64_t *x_out_dev,
                 ss_stream_t stream);

/*
 * ss_classify -- one S5 step over n 8-byte keys with given splitters
 * (Algorithm 1: tree descent, equality test, bucket counts, prefix sum,
 * stable redistribution), run by the same kernels the sort uses.
 *   keys_dev     : uint64[n].
 *   x_dev        : uint64[2^d - 1] in-order splitters, non-decreasing; d in [1, 10].
 *   bucket_out_dev : uint16[n]; bucket 2r + [x_r == c] where r = #{j: x_j < c}.
 *   bucket_begin_out_dev : uint32[2^(d+1)] start of each bucket, last = n.
 *   order_out_dev  : uint32[n]; order_out[p] = input position placed at p
 *                    (stable: input order inside a bucket).
 */
int ss_classify(const uint64_t *keys_dev, uint32_t n, const uint64_t *x_dev, uint32_t d,
                uint16_t *bucket_out_dev, uint32_t *bucket_begin_out_dev, uint32_t *order_out_dev,
                ss_stream_t stream);

/*
 * ss_classify_ex -- ss_classify with the classifier chosen (one of
 * SS_CLASSIFIER_*; SS_ERR_INVALID otherwise).  With SS_CLASSIFIER_EQUAL and a
 * repeated splitter value, keys equal to it go to the equality bucket of the
 * copy highest in the tree (in-order index k with the most trailing one bits
 * of k, i.e. trailing zero bits of k + 1), and order_out follows those buckets.
 */
int ss_classify_ex(const uint64_t *keys_dev, uint32_t n, const uint64_t *x_dev, uint32_t d,
                   uint32_t classifier, uint16_t *bucket_out_dev, uint32_t *bucket_begin_out_dev,
                   uint32_t *order_out_dev, ss_stream_t stream);

/*
 * Sort server -- continuous batching of independent requests (the paper's
 * job queue of independent subproblems, Section 4.5, one level up: requests
 * arriving over time).  The server admits submitted requests in arrival order
 * while the scratch memory of the admitted, unfinished ones fits
 * budget_bytes; each of `workers` host threads drives its own CUDA stream and,
 * when idle, takes every admitted request waiting at that moment (at most
 * max_batch, 0 = no limit) as one batch with the launches of ss_sort_batch.
 * Batches formed while others run overlap on the device.  Results equal those
 * of one ss_sort_ex per request.
 *
 * Ownership: the caller keeps every buffer a request points to alive and
 * unchanged (the strings) or untouched (the outputs) until ss_server_wait has
 * returned for its ticket.  Pointers are device pointers, as for ss_request.
 *
 * ss_server_create: budget_bytes > 0, 1 <= workers <= 64; *out receives the
 *   server (SS_ERR_INVALID otherwise; SS_ERR_CUDA if a stream cannot be made).
 *   The server works on the device current at creation.
 * ss_server_submit: queues one request without blocking and returns its
 *   ticket.  SS_ERR_TOO_LARGE if the request alone needs more scratch than the
 *   budget (ss_scratch_bytes); SS_ERR_INVALID for NULL pointers with n > 0 or
 *   after ss_server_destroy has begun.
 * ss_server_wait: blocks until the ticket's request is done, then writes its
 *   status (an ss_status) and, if times_ms_out is not NULL, three times in ms
 *   on the server's clock: submitted, batch started, batch finished.  Each
 *   ticket is waited for once; an unknown ticket gives SS_ERR_INVALID.
 * ss_server_cancel: withdraws a request that is still queued: *cancelled_out
 *   = 1, and its ss_server_wait reports SS_ERR_CANCELLED with its outputs
 *   untouched.  A request a worker has already taken runs to the end:
 *   *cancelled_out = 0.  SS_ERR_INVALID for an unknown ticket.
 * ss_server_destroy: finishes every submitted request, stops the workers and
 *   frees the server.
 * ss_scratch_bytes: scratch bytes one request of n strings is charged.
 */
typedef struct ss_server ss_server;
int ss_server_create(uint64_t budget_bytes, uint32_t workers, uint32_t max_batch, ss_server **out);
int ss_server_submit(ss_server *server, const ss_request *req, uint64_t *ticket_out);

/*
 * A request on host buffers: the arguments of ss_sort_host.  The server runs
 * it alone on one worker (copies in, the sort, the merge of `runs` runs when
 * runs > 1, copies out), so its copies overlap the sorts of other workers:
 * a stream of host requests through a 2-worker server overlaps the transfers
 * of one with the sort of the next.  Pinned host buffers copy faster.  It is
 * charged its device copies, outputs and scratch against the budget.
 */
typedef struct {
    const uint8_t *chars;
    uint64_t chars_len;
    const uint64_t *offsets;
    const uint32_t *lengths;
    uint32_t fixed_len;
    uint32_t n;
    uint32_t runs;
    uint32_t *perm_out;
    uint32_t *lcp_out;
} ss_host_request;
int ss_server_submit_host(ss_server *server, const ss_host_request *req, uint64_t *ticket_out);
int ss_server_wait(ss_server *server, uint64_t ticket, int32_t *status_out, double *times_ms_out);
int ss_server_cancel(ss_server *server, uint64_t ticket, int32_t *cancelled_out);
int ss_server_destroy(ss_server *server);
uint64_t ss_scratch_bytes(uint32_t n);

/*
 * ss_debug_fail_allocs -- fault injection on the host for tests: of the
 * library's next scratch allocations (any thread), the first `skip` succeed
 * and the `count` after them fail as an exhausted pool would, so the calls
 * that make them return SS_ERR_OOM (a server request gets it as its status).
 * count = 0 switches injection off.  Nothing is injected on the device.
 */
int ss_debug_fail_allocs(uint32_t skip, uint32_t count);

/*
 * ss_device_error -- the first device-side failure (SS_ERR_TIMEOUT or
 * SS_ERR_INTERNAL) of any asynchronous sort since the last call, or SS_OK;
 * the record is cleared.  Synchronize the sorts' streams first.  One record
 * for the whole process: with sorts on several streams or threads it tells
 * that one of them failed, each request's status_out tells which.
 */
int ss_device_error(int32_t *status_out_host);

/*
 * ss_debug_copy_wait -- for tests of the timeout path: the budget of every
 * bounded wait for a bulk copy into shared memory in the distribution step
 * (SM clock cycles; 0 restores the default of about a second), and, with
 * withhold != 0, those copies are not issued at all, so every such wait runs
 * out, the tile writes nothing, the sort stops after that level, the call
 * returns SS_ERR_TIMEOUT (ss_sort_batch_async: its requests' status_out does)
 * and each request's status_out reads it.  Nothing faults or hangs: no later
 * kernel reads what the tile did not write.  Affects every sort of the
 * process.
 */
int ss_debug_copy_wait(uint64_t budget_cycles, uint32_t withhold);

/* Kernel timing: when enabled, the library records CUDA events around each of
 * its kernel launches (on the launch stream) and accumulates per-kernel time.
 * ss_profile_read fills up to `cap` entries: name (NUL-terminated, 48 bytes
 * each), launches, total milliseconds and units (strings or records the
 * launches processed); returns the number of kernels.  Any output pointer
 * may be NULL. */
int ss_profile_enable(int on);
int ss_profile_reset(void);
int ss_profile_read(char *names48, uint64_t *launches, double *total_ms, uint64_t *units, int cap);

/* Number of kernel launches issued by the library since the last reset. */
uint64_t ss_launch_count(void);

/* Copies the calling thread's last error message into buf (NUL-terminated);
 * returns its full length. */
int ss_last_error_detail(char *buf, size_t len);

/* ABI version (major * 100 + minor). */
int ss_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SS_GB300_H */
