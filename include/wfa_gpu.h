/*
 * wfa_gpu.h -- C ABI of libwfa_gpu.so: batched exact gap-affine pairwise
 * alignment with the wavefront algorithm (WFA) on one NVIDIA GB300 (sm_103a).
 *
 * The operation (paper, Sec. I "Introduction and Methods"): align a large
 * number of independent read pairs, each one on its own with no
 * communication between pairs, using the original gap-affine WFA with no
 * algorithmic change (Sec. I, "we apply no optimizations"); every pair
 * yields its result (Sec. I: "aligns the reads using WFA, and writes the
 * result").  Here the result is the optimal score and one canonical optimal
 * alignment as a run-length CIGAR.
 *
 * Scoring (gap-affine, match = 0):
 *   score = min over global alignments of
 *           x * (#mismatches) + sum over maximal gap runs of (o + len * e)
 *   I consumes one text character, D one pattern character; an I run next to
 *   a D run counts as two runs.
 *
 * Canonical alignment (the paper is silent on ties; this library fixes one
 * rule): walking back from the end of both sequences, each operation is
 * placed at the largest text offset it can take (fewest trailing matches);
 * among operations at the same offset a mismatch (X) is preferred over an
 * insertion (I) over a deletion (D); inside a gap, extending it is preferred
 * over opening it.
 *
 * CIGAR word: (run_length << 4) | op, op 0 = M (match), 1 = X (mismatch),
 * 2 = I (text only), 3 = D (pattern only).  Runs of one op never touch.
 * SAM users: this library's I/D are from the text's point of view; with the
 * pattern as the query and the text as the reference, swap I and D.
 *
 * Threading: a context may be used by one host thread at a time.  All calls
 * are synchronous unless stated otherwise.
 */
#ifndef WFA_GPU_H
#define WFA_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wfa_gpu_ctx wfa_gpu_ctx;

/* Penalties: mismatch x >= 1, gap open o >= 0, gap extend e >= 1, each at
 * most WFA_GPU_MAX_PENALTY.  A gap of length L costs o + L*e. */
typedef struct {
  int32_t x, o, e;
} wfa_gpu_penalties;

#define WFA_GPU_MAX_PENALTY (1 << 16)
/* Longest accepted sequence.  Run lengths fit the 28-bit CIGAR field. */
#define WFA_GPU_MAX_SEQ_LEN ((1 << 28) - 1)

/* Return codes.  Negative: the call failed and no output is valid. */
enum {
  WFA_GPU_OK = 0,
  WFA_GPU_EINVAL = -1,          /* bad argument (NULL, negative size, bad penalty, bad length) */
  WFA_GPU_ENOMEM = -2,          /* device or host allocation failed, or the scratch arena is
                                   too small for some pair's wavefronts */
  WFA_GPU_ECUDA = -3,           /* a CUDA runtime call failed (no device, launch failure) */
  WFA_GPU_ECIGAR_CAPACITY = -4, /* CIGAR words exceed cigar_capacity_words; scores, status
                                   and out_cigar_offsets are still valid, out_cigar_offsets[n]
                                   is the size needed, the CIGAR buffer holds no valid
                                   alignment (its contents are unspecified) */
  WFA_GPU_ETIMEOUT = -5         /* a bounded device-side wait gave up */
};

/* Per-pair status (out_status). */
enum {
  WFA_PAIR_OK = 0,
  WFA_PAIR_SCORE_LIMIT = 1,  /* optimal score > max_score (max_score > 0) */
  WFA_PAIR_INVALID_CHAR = 2  /* a byte other than A/C/G/T (either case) */
};

/* Flags for wfa_gpu_align_batch. */
enum {
  WFA_GPU_SCORE_ONLY = 1u,  /* compute scores only; out_cigars may be NULL */
  WFA_GPU_DEVICE_PTRS = 2u, /* every input and output pointer is device memory on the
                               context's device (default: host memory) */
  WFA_GPU_TIMING = 4u,      /* record per-phase device times for wfa_gpu_last_timing */
  WFA_GPU_PLAIN = 8u,       /* the plain baseline for comparisons: the same kernels launched
                               call by call with one fixed short-read variant (the largest
                               store of the call's length class and penalty model), no
                               sampling autotuner, pairs in call order (no ordering pass),
                               the arena kernels' work lists in pair order, and no graph
                               replay (WFA_GPU_GRAPH is ignored); same results */
  WFA_GPU_GRAPH = 16u,      /* with WFA_GPU_DEVICE_PTRS: for batches repeated with the same
                               arguments (same sizes and buffers, new contents), the first
                               call runs as usual and records the device work into a CUDA
                               graph; identical later calls replay it with a single host
                               synchronisation (one graph per context) */
  WFA_GPU_ARENA_ONLY = 32u  /* every pair on one-warp (or, above 2,048 bases, one-CTA)
                               arena teams from a work queue in pair order, without the
                               short-read kernels, launched call by call (WFA_GPU_GRAPH is
                               ignored); same results */
};

/* Device-side times of the last wfa_gpu_align_batch call on a context,
 * measured with CUDA events on the context's stream (only with
 * WFA_GPU_TIMING; otherwise zero). */
typedef struct {
  float h2d_ms;      /* host -> device copies of inputs (host-pointer mode) */
  float align_ms;    /* the short-read phase: ordering pass and short-read kernel */
  float general_ms;  /* the scratch-arena wavefront kernel (pairs it took over) */
  float cigar_ms;    /* CIGAR offset scan and compaction */
  float d2h_ms;      /* device -> host copies of outputs (host-pointer mode) */
  float total_ms;    /* whole call, first to last event */
  int32_t kernel_launches; /* kernels this library launched during the call */
  int32_t short_variant;   /* index of the short-read kernel variant that ran (-1: none) */
  int64_t deferred_pairs;  /* pairs handed from the short-read kernel to the arena kernel */
} wfa_gpu_timing;

/* Create a context on CUDA device `device`.
 * scratch_bytes: size of the device scratch arena holding wavefronts of
 * pairs that do not fit the short-read kernel's shared memory (long reads,
 * high scores); 0 selects 1 GiB.  The context owns the arena, its internal
 * buffers (grown on demand) and a CUDA stream.
 * Returns WFA_GPU_OK and *out, or EINVAL (out NULL, device < 0), ECUDA (no
 * such device / CUDA unavailable) or ENOMEM; *out is NULL on failure. */
int wfa_gpu_create(wfa_gpu_ctx **out, int device, size_t scratch_bytes);

/* Make the context launch its work on `stream` (a cudaStream_t of the
 * context's device, e.g. a framework's current stream) instead of its own;
 * NULL restores the context's own stream.  The caller keeps ownership of the
 * stream and must keep it alive while the context uses it. */
int wfa_gpu_set_stream(wfa_gpu_ctx *ctx, void *stream);

/* Ends-free alignment for the context's later wfa_gpu_align_batch calls
 * (the paper aligns reads end to end, Sec. I; this is a variant of the
 * method it cites): up to pattern_begin_free leading and pattern_end_free
 * trailing pattern characters, and up to text_begin_free leading and
 * text_end_free trailing text characters, may stay unaligned at no cost.
 * The alignment starts at (v, 0), v <= pattern_begin_free, or (0, h),
 * h <= text_begin_free, and ends at (n, h), h >= m - text_end_free, or
 * (v, m), v >= n - pattern_end_free; a gap after the start or before the
 * end is paid as usual.  The CIGAR still covers both sequences: skipped
 * characters are its leading / trailing D (pattern) or I (text) runs.  Of
 * the optimal end cells, the one on the diagonal k = h - v nearest m - n is
 * taken, the larger k on a tie.  Example: pattern_* = 0 and text_* >= m
 * aligns the whole pattern to its best-matching stretch of the text.
 * All four 0 (the default) is the global alignment.  A CIGAR may take two
 * runs more than wfa_gpu_cigar_bound() states.  Returns OK, or EINVAL (ctx
 * NULL, a length negative or above WFA_GPU_MAX_SEQ_LEN).  Host-only. */
int wfa_gpu_set_ends_free(wfa_gpu_ctx *ctx, int32_t pattern_begin_free, int32_t pattern_end_free,
                          int32_t text_begin_free, int32_t text_end_free);

/* Align n_pairs independent pairs (paper Sec. I: many read pairs aligned
 * independently, each producing its result; Sec. II workload: 100 bp reads).
 *
 * Inputs, for pair i:
 *   pattern = patterns[pattern_offsets[i] .. + pattern_lengths[i])
 *   text    = texts[text_offsets[i] .. + text_lengths[i])
 * ASCII bytes; A/C/G/T in either case.  An offsets array may be NULL, which
 * means the sequences lie back to back in pair order starting at byte 0.
 * Lengths are 0 .. WFA_GPU_MAX_SEQ_LEN.  Offsets must be >= 0.
 * pen: penalties (see wfa_gpu_penalties).
 * max_score: if > 0, pairs whose optimal score exceeds it get status
 *   WFA_PAIR_SCORE_LIMIT (a score equal to max_score is reported); <= 0 means
 *   no bound.
 * flags: WFA_GPU_SCORE_ONLY | WFA_GPU_DEVICE_PTRS | WFA_GPU_TIMING |
 *   WFA_GPU_PLAIN | WFA_GPU_GRAPH | WFA_GPU_ARENA_ONLY.
 *
 * Outputs (caller-owned):
 *   out_scores[n]   int32 optimal score, -1 if status != OK
 *   out_status[n]   int8 WFA_PAIR_*
 *   out_cigar_offsets[n+1]  int64; pair i's CIGAR is
 *       out_cigars[out_cigar_offsets[i] .. out_cigar_offsets[i+1]); empty if
 *       status != OK; out_cigar_offsets[0] = 0.  May be NULL with SCORE_ONLY.
 *   out_cigars[cigar_capacity_words]  uint32 CIGAR words (see above).  May be
 *       NULL with SCORE_ONLY or when cigar_capacity_words == 0.
 * With WFA_GPU_DEVICE_PTRS every pointer above (inputs and outputs) is device
 * memory; otherwise all are host memory (page-locked memory copies fastest).
 * Sizing: wfa_gpu_cigar_bound() per pair gives a safe capacity.
 *
 * Returns WFA_GPU_OK (every pair has a status), or EINVAL, ENOMEM, ECUDA,
 * ECIGAR_CAPACITY (see the enum).  The call returns after all outputs are
 * in the caller's buffers.  Host-pointer calls of 2^21 pairs or more whose
 * outputs are page-locked run in chunks of 2^19 pairs, each chunk's outputs
 * copied back while the next one computes; when in addition both sequence
 * arrays are page-locked and stored back to back (both offset arrays NULL),
 * each chunk's bases (and its lengths, if page-locked) are copied into a
 * device ring two chunks ahead of the computation instead of being read in
 * place.  Same results either way. */
int wfa_gpu_align_batch(wfa_gpu_ctx *ctx, int64_t n_pairs,
                        const char *patterns, const int64_t *pattern_offsets,
                        const int32_t *pattern_lengths,
                        const char *texts, const int64_t *text_offsets,
                        const int32_t *text_lengths,
                        wfa_gpu_penalties pen, int32_t max_score, uint32_t flags,
                        int32_t *out_scores, int8_t *out_status,
                        uint32_t *out_cigars, int64_t cigar_capacity_words,
                        int64_t *out_cigar_offsets);

/* Pack sequences into the 2-bit format the wavefront kernels extend with
 * (the per-pair fetch of Sec. I, "fetches the read pair ... aligns"):
 * A=0 C=1 G=2 T=3 (either case), 32 bases per uint64 word, base j of a word
 * in bits (63-2j):(62-2j), bits past the end zero, then one zero pad word;
 * sequence i takes ceil(len/32) + 1 words starting at out_word_offsets[i].
 * Inputs as in wfa_gpu_align_batch (offsets may be NULL = back to back).
 * Outputs: out_word_offsets[n_seqs+1] int64 (exclusive prefix sum of the
 * word counts; [n_seqs] = total), out_words[words_capacity] uint64,
 * out_invalid[n_seqs] int8 (1 if the sequence holds a byte other than
 * A/C/G/T; its words are then unspecified).
 * All pointers are device memory when flags has WFA_GPU_DEVICE_PTRS, else
 * host memory.  Returns OK, EINVAL, ENOMEM, ECUDA, or ECIGAR_CAPACITY when
 * the total word count exceeds words_capacity (offsets still valid, words
 * untouched). */
int wfa_gpu_pack2bit(wfa_gpu_ctx *ctx, int64_t n_seqs, const char *seqs,
                     const int64_t *offsets, const int32_t *lengths, uint32_t flags,
                     uint64_t *out_words, int64_t words_capacity,
                     int64_t *out_word_offsets, int8_t *out_invalid);

/* Size of the device scratch array behind wfa_gpu_align_short_noalloc, and
 * the limits it implies. */
#define WFA_GPU_NOALLOC_SCRATCH_BYTES ((size_t)4 << 20)
#define WFA_GPU_NOALLOC_MAX_PAIRS 32768
#define WFA_GPU_NOALLOC_MAX_LEN 127

/* Align short read pairs without allocating any memory.  (The paper has no
 * counterpart to this entry point; it exists for callers of this library.)
 *
 * Who needs it: callers that cannot call cudaMalloc -- applications whose
 * device memory belongs to a pool or framework that forbids allocations
 * made behind its back, and latency-critical paths that must not risk the
 * device-wide synchronisation cudaMalloc and cudaFree can bring.
 * wfa_gpu_create allocates a scratch arena and buffers; this entry point
 * instead keeps its scratch (control block, offset scans, per-pair CIGAR
 * slots, work lists) in one file-scope device array of
 * WFA_GPU_NOALLOC_SCRATCH_BYTES that every GPU which loads the library
 * holds until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.  It is not for use while `stream` is being captured
 * into a CUDA graph: it synchronises `stream` (up to four times) to read its
 * control block back and return its error codes.
 *
 * Same operation, inputs and outputs as wfa_gpu_align_batch with
 * WFA_GPU_DEVICE_PTRS (every pointer is device memory on the current device;
 * offsets may be NULL = back to back), without flags, and limited to:
 *   n_pairs <= WFA_GPU_NOALLOC_MAX_PAIRS, every sequence
 *   <= WFA_GPU_NOALLOC_MAX_LEN bases -- otherwise WFA_GPU_EINVAL;
 *   pairs whose wavefronts fit the short-read kernel's shared memory (for
 *   penalties 4/6/2: an optimal score up to 32), and whose CIGAR has at most
 *   16 runs (a 127-base pair with 8 isolated mismatches scores 32 but needs
 *   17 runs: 9 M and 8 X) -- if a pair breaks either, WFA_GPU_ENOMEM
 *   (wfa_gpu_align_batch handles such pairs in its arena).
 * stream: the cudaStream_t to run on (NULL: the legacy default stream).
 *
 * The first call on a device sets that device up (looks up the scratch
 * array's device address, configures the kernel).  Every call shares the
 * one scratch array, which keeps the previous call's contents; calls whose
 * work overlaps on the GPU (other streams, other host threads) race on it
 * and must be serialised by the caller.  Returns after the outputs are
 * written.  Returns OK, EINVAL, ENOMEM, ECUDA or ECIGAR_CAPACITY as
 * wfa_gpu_align_batch does. */
int wfa_gpu_align_short_noalloc(void *stream, int64_t n_pairs,
                                const char *patterns, const int64_t *pattern_offsets,
                                const int32_t *pattern_lengths,
                                const char *texts, const int64_t *text_offsets,
                                const int32_t *text_lengths,
                                wfa_gpu_penalties pen, int32_t max_score,
                                int32_t *out_scores, int8_t *out_status,
                                uint32_t *out_cigars, int64_t cigar_capacity_words,
                                int64_t *out_cigar_offsets);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of alignment requests.
 *
 * Requests (batches of pairs, of any size, arriving at any time) are queued
 * and admitted onto `workers` slots, each a context with its own stream and
 * buffers; at most two slots run a call at once (a call's device work
 * overlaps another's gathering and scattering on the host; more calls at
 * once only queue behind one another on the GPU and split the queue into
 * smaller batches), three when the third passes an older request whose
 * slice does not fit the free arena yet; further slots wait for a turn.
 * The server
 * owns one scratch arena (the memory budget); every call runs on a slice of
 * it sized to the call's estimated wavefront need (see
 * wfa_gpu_request_bytes; at least 64 MiB, at most half the arena: on a
 * smaller slice than they would like, the arena kernels run fewer pairs at
 * once).  A request is admitted when a
 * slot is free and its slice fits the free arena: the oldest that fits goes
 * first (a later request may pass one that does not fit yet, until that one
 * has waited 50 ms; then the slots drain until it fits; a request alone
 * always fits, on the whole arena at most).  A slot that admits a request
 * also takes the requests queued right behind it that have the same
 * penalties, max_score and flags, up to WFA_GPU_SERVER_MERGE_PAIRS pairs in
 * all, when their slice fits too: it gathers their pairs into one batch,
 * copies it to the device, aligns it with one device-pointer call and copies
 * each request's results back into its own buffers.  A call in which a pair
 * outgrew its slice runs once more on the whole arena.
 * Every request's outputs and result code are the ones wfa_gpu_align_batch
 * gives for it alone (pairs are independent: paper Sec. I; a request whose
 * CIGAR words exceed its capacity gets WFA_GPU_ECIGAR_CAPACITY as alone, and
 * a merged call that fails is re-run one request at a time); only the timing
 * depends on the mix.
 * --------------------------------------------------------------------------- */
#define WFA_GPU_SERVER_MERGE_PAIRS 65536
/* the edit rate (edits per base) the arena need of a request is estimated for */
#define WFA_GPU_SERVER_EDIT_RATE 0.10
typedef struct wfa_gpu_server wfa_gpu_server;

/* One request: the arguments of wfa_gpu_align_batch, host memory only
 * (flags may hold WFA_GPU_SCORE_ONLY and WFA_GPU_PLAIN).  The caller keeps
 * every buffer alive and untouched until wfa_gpu_server_wait returns for it. */
typedef struct {
  int64_t n_pairs;
  const char *patterns;
  const int64_t *pattern_offsets;
  const int32_t *pattern_lengths;
  const char *texts;
  const int64_t *text_offsets;
  const int32_t *text_lengths;
  wfa_gpu_penalties pen;
  int32_t max_score;
  uint32_t flags;
  int32_t *out_scores;
  int8_t *out_status;
  uint32_t *out_cigars;
  int64_t cigar_capacity_words;
  int64_t *out_cigar_offsets;
} wfa_gpu_request;

/* Times of a finished request, in seconds on the server's clock (a steady
 * clock started by wfa_gpu_server_create), and its result code. */
typedef struct {
  double submit_s, start_s, end_s;
  int32_t result;  /* what wfa_gpu_align_batch returned for it */
  int32_t worker;  /* slot that ran it */
} wfa_gpu_request_stats;

/* Create a server on `device` with `workers` slots (1..64) and a device
 * memory budget (0: 8 GiB; at least 64 MiB): the scratch arena the calls
 * share (the slots' gather and result buffers come on top, grown to the
 * largest batch they ran).  Returns OK, EINVAL, ECUDA or ENOMEM; *out is
 * NULL on failure. */
int wfa_gpu_server_create(wfa_gpu_server **out, int device, int workers, size_t memory_budget_bytes);

/* Queue a request; returns its id (>= 0) or a negative WFA_GPU_* code
 * (EINVAL for a malformed request).  Never blocks on the GPU. */
int64_t wfa_gpu_server_submit(wfa_gpu_server *server, const wfa_gpu_request *req);

/* Wait until request `id` has finished (timeout_s < 0: no limit) and return
 * its result code, filling *stats if not NULL; the id is then forgotten.
 * Returns WFA_GPU_ETIMEOUT if the wait ran out (the request stays queued or
 * running; wait again later), EINVAL for an unknown id. */
int wfa_gpu_server_wait(wfa_gpu_server *server, int64_t id, double timeout_s, wfa_gpu_request_stats *stats);

/* Estimated device bytes a request holds while it runs: its sequence
 * bytes, 150 bytes a pair (lengths, offsets, outputs, work buffers, CIGAR
 * slots), 4 bytes a word of CIGAR capacity, and the arena its wavefronts
 * take -- for pairs longer than 127 bases (the short-read kernels keep
 * theirs in shared memory), 3 offsets of 2 bytes (4 from 32,000 bases) on
 * about (s'/e' + 1)^2 cells plus 16 (s' + 1) bytes of per-score records,
 * s' = WFA_GPU_SERVER_EDIT_RATE x max(n, m) x max(x, o + e) / g and
 * e' = e / g (g = gcd(x, o, e)), summed over the 4,096 largest such pairs
 * (no more run at once).  The arena part is what the server admits
 * requests by.  Returns -1 for a NULL or malformed request (n_pairs < 0,
 * or missing length arrays).  Host-only. */
int64_t wfa_gpu_request_bytes(const wfa_gpu_request *req);

/* Finish the admitted requests, drop the queued ones (their waits return
 * ECUDA) and release the server.  NULL-safe. */
void wfa_gpu_server_destroy(wfa_gpu_server *server);

/* Name of short-kernel variant `index` of the context (the index that
 * wfa_gpu_timing.short_variant reports): "lane_l127_c197" (one lane per
 * pair, sequences up to 127 bases, 197 stored cells per pair, one byte per
 * offset), "lane_ct241_l127_c40" (the same with the geometry of scaled
 * penalties x = 2, o + e = 4, e = 1 compiled in), "g2_l127_c197_i8" (the
 * cells of the running pairs spread over the warp's lanes, 2 lanes a pair,
 * int8 offsets), "..._lin" (gap-linear model, M only) or "..._ef"
 * (ends-free calls); NULL if there is no such variant.  The string is
 * static.  Host-only. */
const char *wfa_gpu_short_variant_name(const wfa_gpu_ctx *ctx, int index);

/* Upper bound on the CIGAR words of one pair of lengths plen, tlen under pen
 * and max_score (<= 0: unbounded): with s the largest score the pair can
 * report, at most 2*floor(s / min(x, o+e)) + 1 runs, and never more than
 * plen + tlen.  Returns -1 on invalid arguments.  Host-only; no device work. */
int64_t wfa_gpu_cigar_bound(int32_t plen, int32_t tlen, wfa_gpu_penalties pen,
                            int32_t max_score);

/* Per-phase times of the last align call (see wfa_gpu_timing).  Returns OK
 * or EINVAL. */
int wfa_gpu_last_timing(const wfa_gpu_ctx *ctx, wfa_gpu_timing *out);

/* Static description of a return code.  Never NULL. */
const char *wfa_gpu_strerror(int code);

/* Release the context, its arena, buffers and own stream.  NULL-safe. */
void wfa_gpu_destroy(wfa_gpu_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* WFA_GPU_H */
