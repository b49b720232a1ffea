/*
 * anyseq.h - C ABI of the GB300 pairwise alignment library.
 *
 * The operation is the DP alignment of Sec. III-A of the AnySeq paper
 * (arXiv 2002.04561): for a query Q = q_1..q_n (rows i) and a subject
 * S = s_1..s_m (columns j),
 *
 *   E(i,j) = max(E(i-1,j) + extend, H(i-1,j) + open + extend)   Eq. 4
 *   F(i,j) = max(F(i,j-1) + extend, H(i,j-1) + open + extend)   Eq. 5
 *   H(i,j) = max(H(i-1,j-1) + sigma(q_i,s_j), E(i,j), F(i,j), nu) Eq. 1
 *
 * with the global (nu = -inf, optimum at (n,m)), local (nu = 0, optimum
 * anywhere) and semi-global (row 0 and column 0 free, optimum in the last
 * row or column) initialisations of Sec. III-A. A linear gap g (Eqs. 2, 3)
 * is open = 0, extend = g. Scores are SIGNED: open, extend <= 0, and a gap
 * of length k adds open + k*extend (the paper writes G_o = -open,
 * G_e = -extend). The paper's one-pair interface construct_global_alignment
 * (Sec. III-C) becomes a batch call and a long-pair call here.
 *
 * Conventions fixed by this library where the paper is silent:
 *  - optimum cell on ties: the smallest i, then the smallest j;
 *  - predecessor on ties: diagonal, then E (CIGAR I), then F (CIGAR D); a
 *    local cell of value 0 ends the alignment; inside E/F opening is
 *    preferred over extending;
 *  - CIGAR words are BAM style (length << 4 | op) with op M = 0 (q_i with
 *    s_j), I = 1 (q_i against a gap), D = 2 (s_j against a gap);
 *  - beg_q/beg_s is the DP cell where the path starts (the alignment covers
 *    q[beg_q+1 .. end_q] and s[beg_s+1 .. end_s]); an empty local alignment
 *    has beg = end = (0,0).
 *
 * Pointers: every array argument may be host or device memory (the library
 * asks the driver). Calls are asynchronous on the given CUDA stream when all
 * arrays are device memory; when any output is host memory the call returns
 * after the stream has finished. Inputs and outputs are owned by the caller
 * and never freed by the library; scratch comes from the context, capped by
 * its memory budget. All functions return an anyseq_status_t and never throw;
 * anyseq_last_error() describes the last failure of the calling thread.
 */
#ifndef ANYSEQ_H
#define ANYSEQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ANYSEQ_GLOBAL = 0,      /* Needleman-Wunsch: nu = -inf, optimum H(n,m) */
    ANYSEQ_LOCAL = 1,       /* Smith-Waterman: nu = 0, optimum anywhere */
    ANYSEQ_SEMIGLOBAL = 2   /* free end gaps: local initialisation, nu = -inf, optimum in last row/column */
} anyseq_mode_t;

typedef enum {
    ANYSEQ_OK = 0,
    ANYSEQ_ERR_ARG = 1,       /* bad pointer, size, scoring or mode */
    ANYSEQ_ERR_ALPHABET = 2,  /* a code >= alphabet, or a non-ACGT letter */
    ANYSEQ_ERR_BUDGET = 3,    /* scratch would exceed the context's memory budget */
    ANYSEQ_ERR_CUDA = 4,      /* a CUDA runtime call failed */
    ANYSEQ_ERR_TIMEOUT = 5,   /* a device-side wait exceeded its iteration limit */
    ANYSEQ_ERR_CAPACITY = 6   /* the caller's CIGAR buffer is too small (*cigar_used = words needed) */
} anyseq_status_t;

enum {
    ANYSEQ_WANT_SCORE = 1,    /* score (always computed) */
    ANYSEQ_WANT_END = 2,      /* optimum cell (always computed) */
    ANYSEQ_WANT_CIGAR = 4,    /* traceback to a CIGAR and the start cell */
    ANYSEQ_BAND_LEARNED = 8   /* long/global pairs: try a learned band under a certificate first */
};

/* result flags */
enum {
    ANYSEQ_FLAG_INT32 = 1,        /* computed in 32-bit lanes (did not pass the int16 range test) */
    ANYSEQ_FLAG_BAND_ACCEPTED = 2,/* a banded result was accepted by the certificate */
    ANYSEQ_FLAG_FULL_FALLBACK = 4 /* band certificate failed at every width: full DP */
    /* bits 8..15: number of band doublings */
};

typedef struct {
    int32_t alphabet;        /* 4 for DNA (codes 0..3 = A,C,G,T) up to 32; codes must be < alphabet */
    const int8_t *matrix;    /* alphabet x alphabet row-major, row = query letter (host memory); NULL: match/mismatch */
    int32_t match, mismatch; /* used when matrix == NULL */
    int32_t gap_open;        /* <= 0 */
    int32_t gap_extend;      /* <= 0 */
} anyseq_scoring_t;

typedef struct {
    int32_t score;
    int32_t beg_q, beg_s;    /* start cell (WANT_CIGAR), else -1 */
    int32_t end_q, end_s;    /* optimum cell */
    uint32_t flags;
    uint64_t cigar_off;      /* first word of this pair in the caller's CIGAR buffer */
    uint32_t cigar_len;      /* number of words */
    uint32_t reserved;
} anyseq_result_t;

typedef struct anyseq_ctx anyseq_ctx;

/* Create a context on CUDA device 'device'. Scratch is allocated lazily and
 * reused; its total never exceeds mem_budget_bytes (0 = 90% of free memory). */
anyseq_status_t anyseq_create(anyseq_ctx **ctx, int device, size_t mem_budget_bytes);
anyseq_status_t anyseq_destroy(anyseq_ctx *ctx);

/*
 * Align n_pairs independent pairs (inter-sequence parallelism, Sec. VI).
 *   q, s          concatenated letter codes (uint8), pair p at q[q_off[p] .. q_off[p+1])
 *   q_off, s_off  n_pairs + 1 non-decreasing offsets (int64)
 *   sc            scoring (host struct); mode: anyseq_mode_t; want: ANYSEQ_WANT_* bits
 *   out           n_pairs results (caller-owned)
 *   cigar         with ANYSEQ_WANT_CIGAR: buffer of cigar_cap words; pair p's words start at
 *                 out[p].cigar_off; *cigar_used (host) receives the total. Too small a buffer
 *                 returns ANYSEQ_ERR_CAPACITY with *cigar_used = words needed; NULL/0 allowed otherwise.
 *   cuda_stream   cudaStream_t (NULL = legacy default stream)
 * Any pointer may be host or device memory. Host letters in pinned memory of a
 * 2-bit alphabet (at most 4 letters) are read in place by the device over the
 * host link (option "host_in_place", default 1; 0 copies them first); other host
 * letters are copied. Either way the host buffers must stay unchanged until the
 * call's work on cuda_stream has finished, as with any asynchronous copy.
 * Errors: ERR_ARG (null pointers, decreasing offsets, open/extend > 0, alphabet out of
 * range, mode unknown, a pair of 2^21 letters or more, and in local and
 * semi-global mode a pair whose score could reach 2^21: largest positive
 * substitution score times min(n, m)), ERR_ALPHABET (a code >= alphabet),
 * ERR_BUDGET, ERR_CUDA.
 */
anyseq_status_t anyseq_align_batch(anyseq_ctx *ctx,
                                   const uint8_t *q, const int64_t *q_off,
                                   const uint8_t *s, const int64_t *s_off,
                                   int64_t n_pairs, const anyseq_scoring_t *sc,
                                   int32_t mode, uint32_t want,
                                   anyseq_result_t *out,
                                   uint32_t *cigar, uint64_t cigar_cap, uint64_t *cigar_used,
                                   void *cuda_stream);

/*
 * Align one long pair (intra-sequence parallelism: anti-diagonal wavefront of
 * row stripes, Sec. IV-C), score in linear space, and with ANYSEQ_WANT_CIGAR
 * the divide-and-conquer traceback of Sec. III-A (Myers-Miller for affine
 * gaps). Global: the CIGAR of the whole pair. ANYSEQ_LOCAL and
 * ANYSEQ_SEMIGLOBAL (lengths below 2^21): the alignment ends at the optimum
 * cell; its start (beg_q, beg_s) is the start of largest beg_q, then largest
 * beg_s, among the optimal alignments ending there (any cell for local, row 0
 * or column 0 for semi-global), found by one more wavefront pass over the
 * reversed prefixes; the CIGAR is the global divide-and-conquer CIGAR of
 * q[beg_q .. end_q) against s[beg_s .. end_s). An empty optimum (score 0) has
 * no CIGAR words and begins at its end. Alphabets of up to 4 letters use 2-bit
 * letters and row profiles; larger alphabets (a substitution matrix, up to 32
 * letters) use byte letters and per-stripe query profiles in shared memory.
 * Arguments as for anyseq_align_batch with one pair of lengths n and m:
 * below 2^23 letters each for global alignment, below 2^21 for local and
 * semi-global (the optimum cell's fields). Errors as there, and ERR_ARG for a
 * length at or above those limits, for local and semi-global pairs whose
 * score could reach 2^21 (largest positive substitution score times
 * min(n, m)), for a pair whose scores could leave the 32-bit range, and for a
 * scoring with sigma - open - extend (or extend - open - extend) outside
 * [-128, 127].
 */
anyseq_status_t anyseq_align_long(anyseq_ctx *ctx,
                                  const uint8_t *q, int64_t n,
                                  const uint8_t *s, int64_t m,
                                  const anyseq_scoring_t *sc, int32_t mode, uint32_t want,
                                  anyseq_result_t *out,
                                  uint32_t *cigar, uint64_t cigar_cap, uint64_t *cigar_used,
                                  void *cuda_stream);

/*
 * Learned band (an extension of the global alignment that keeps results exact).
 * With ANYSEQ_BAND_LEARNED, anyseq_align_batch (global mode, scores) first runs
 * a banded DP around a band proposed by a small network from k-mer diagonal
 * features, accepts the banded score only under an exit certificate (no path
 * that leaves the band can score more), doubles the band otherwise, and falls
 * back to the full DP when the band would cover half of the matrix. Results are
 * identical to the full DP; flags tell which route each pair took. The context
 * must hold a model (anyseq_band_train or anyseq_band_model_load/set).
 */
#define ANYSEQ_BAND_FEATURES 64
#define ANYSEQ_BAND_PARAMS 25090   /* W1 64x128, b1 128, W2 128x128, b2 128, W3 128x2, b3 2 (row-major, float) */

/* 64 k-mer diagonal features per pair (k = 12, DNA codes 0..3): hits of sampled
 * query k-mers in the subject binned by their offset from the straight line
 * (0,0)-(n,m), divided by the number of sampled query k-mers. features: n_pairs x 64 floats. */
anyseq_status_t anyseq_band_features(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off, const uint8_t *s,
                                     const int64_t *s_off, int64_t n_pairs, float *features, void *cuda_stream);
/* Network parameters (float master copy; compute uses their bfloat16 rounding). */
anyseq_status_t anyseq_band_model_get(anyseq_ctx *ctx, float *params, int64_t count);
anyseq_status_t anyseq_band_model_set(anyseq_ctx *ctx, const float *params, int64_t count);
anyseq_status_t anyseq_band_model_save(anyseq_ctx *ctx, const char *path);
anyseq_status_t anyseq_band_model_load(anyseq_ctx *ctx, const char *path);
/* Network outputs y (B x 2: band centre in columns, log of the half-width relative
 * to the longer sequence of the pair) for features x (B x 64). */
anyseq_status_t anyseq_band_forward(anyseq_ctx *ctx, const float *x, int64_t B, float *y, void *cuda_stream);
/* Mean loss and its gradient (ANYSEQ_BAND_PARAMS floats) for targets (B x 2). */
anyseq_status_t anyseq_band_gradient(anyseq_ctx *ctx, const float *x, const float *targets, int64_t B,
                                     float *grad, float *loss, void *cuda_stream);
/* Train the network on the GPU from example pairs: targets are the centre of
 * the optimal path (full DP traceback) and the log of the smallest doubling
 * width whose band passes the certificate, divided by the longer sequence's
 * length. epochs over the pairs in batches of 1024 with
 * Adam at learning rate lr; the final mean loss goes to *loss (may be NULL). */
anyseq_status_t anyseq_band_train(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off, const uint8_t *s,
                                  const int64_t *s_off, int64_t n_pairs, const anyseq_scoring_t *sc, int32_t epochs,
                                  float lr, float *loss, void *cuda_stream);

/* Tuning and test switches of a context: "force_int32" (0/1) routes every pair
 * to 32-bit lanes; "force_matrix_path" (0/1) scores every alphabet through the
 * shared-memory profile kernels (as used above 4 letters); "profile" (0/1) times
 * the DP kernels of each call with CUDA events on the call's stream;
 * "hirschberg_base_cells" (default 65536) is the subproblem size below which the
 * divide-and-conquer traceback switches to a full matrix; "spin_limit" (default
 * 2^24) bounds every device-side wait of the wavefront (ANYSEQ_ERR_TIMEOUT);
 * "band_max_doublings" (default 0) is how often ANYSEQ_BAND_LEARNED doubles a
 * band that fails its certificate before the full DP; "band_area_pct" (default
 * 60) sends a pair whose band would exceed that share of its matrix to the full
 * DP, "band_area16_pct" (default 15) the same for pairs that pass the int16
 * range test (the full DP runs those two per 32-bit lane); "band_margin_pct"
 * (default 65) multiplies the network's half-width by that percentage before
 * the band is planned (a width just below the certifying one fails and pays
 * for the full DP too); "band_floor_pct" (default 30) makes every planned
 * half-width at least that share of the pair's longer sequence (the network
 * then widens bands and picks the pairs that go straight to the full DP);
 * "wave_cell"
 * (default 0) picks the wavefront's cell update in global passes: 0 by the
 * number of stripes side by side, 1 always the three-input maximum, 2 always
 * the two-step form (results are the same); "wave_split" (default 0) runs
 * global three-input-maximum passes with split steps (each lane's upper 8
 * rows one column ahead of its lower 8: two dependency chains per step): 0
 * from 12 stripes per SM, 1 always, 2 never (results are the same);
 * "wave_rows" (default 0) sets the
 * wavefront's rows per lane (4, 8 or 16; 0 chooses by the number of stripes,
 * within what each mode has: local passes at most 8, semi-global 4 or 16,
 * traceback passes 4, 8 or 16; results are the same); "wave_ctas_per_sm"
 * (default 0: as many as fit) caps the wavefront's CTAs per SM, leaving room
 * for other kernels beside a long pair (results are the same);
 * "batch_ctas_per_sm" (default 0: as many as fit) caps the batched DP kernel's
 * persistent CTAs per SM likewise (results are the same); "wave_spread"
 * (default 1) holds back the first stripe draws of a wavefront launch so that
 * its first stripes land on distinct SMs, 0 takes them in plain draw order
 * (results are the same); "host_in_place" (default 1) lets 2-bit batches read
 * pinned host letters in place, 0 copies them to the device first (results are
 * the same); "tb_walker"
 * (default 0) picks the
 * batched traceback walk: 0 by batch size, 1 a warp per pair (staged windows),
 * 2 a thread per pair (results are the same). Unknown keys: ANYSEQ_ERR_ARG. */
anyseq_status_t anyseq_set_option(anyseq_ctx *ctx, const char *key, int64_t value);

/* Statistics of the context's last call (host values, valid after the call's
 * stream has finished): "launches" (kernels launched), "dp_ms" (time of the
 * int16x2 DP kernel, needs "profile"), "dp32_ms" (32-bit lanes), "pairs16",
 * "pairs32" (pairs per lane width); with ANYSEQ_BAND_LEARNED also "band_cells"
 * (cells relaxed by banded passes), "band_accepted", "band_fallback" (pairs),
 * "band_rounds", and the host time of its phases "band_plan_ms" (packing,
 * features, network, band plan), "band_pass_ms" (banded passes with the
 * certificate), "band_full_ms" (full DP of the rest). Of the context, not the
 * call: "tuned_bins" (length bins with a tuned cap), "autotune_gain" (default
 * time / tuned time on the tuning sample; 1 when untuned). Unknown keys:
 * ANYSEQ_ERR_ARG. */
anyseq_status_t anyseq_get_stat(anyseq_ctx *ctx, const char *key, double *value);

/*
 * Global score of one long pair, allocating no device memory. The paper has
 * no counterpart: this is for callers that cannot let the library call
 * cudaMalloc/cudaFree, such as a process whose framework owns all device
 * memory through its own pool, or a latency-bound service that cannot accept
 * the synchronisation those calls imply. It runs the same wavefront pass as
 * anyseq_align_long, with all scratch in one fixed device array of the library
 * (about 21 MB on every GPU that loads it, held until the process exits).
 *   q, s    device arrays of codes 0..3 on the current device, lengths
 *           1 <= n, m <= ANYSEQ_NOALLOC_MAX_LEN
 *   score   device int32 on the current device receiving the optimal global score
 * ANYSEQ_ERR_ARG: a length outside those limits, a pointer that is not device
 * memory of the current device, or a scoring whose values could leave the
 * 32-bit range on this pair (the same bound as anyseq_align_long).
 * No context is needed. The first call on a device resolves the array's device
 * address (once per device). The call returns after its stream has finished
 * (it reads the error flags).
 * All calls share the array: calls that overlap on the GPU race on it.
 */
#define ANYSEQ_NOALLOC_MAX_LEN 1048576
anyseq_status_t anyseq_align_long_noalloc(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m,
                                          const anyseq_scoring_t *sc, int32_t *score, void *cuda_stream);

/* Map ASCII A/C/G/T (either case) to codes 0..3; any other byte: ANYSEQ_ERR_ALPHABET.
 * Host pointers only; synchronous. */
anyseq_status_t anyseq_encode_dna(const char *ascii, uint8_t *codes, int64_t len);

/* Description of the calling thread's last error (static storage, never NULL). */
const char *anyseq_last_error(void);

/* Library version string. */
const char *anyseq_version(void);

/* Autotuner of the batched path (not in the paper). The sample (arguments as
 * for anyseq_align_batch, score only; synchronous) is aligned once per
 * candidate tile shape (rows per lane capped at 4, 8, 12 or 16) while the
 * kernel counts SM cycles and cells per length bin (the 8-bit logarithmic
 * bucket of a work item's longest query); each bin takes the cap with the
 * fewest cycles per cell. Then the whole sample is timed (CUDA events, median
 * of five) under the default shape, each smaller uniform cap and the per-bin
 * table; the fastest is kept if it beats the default by 3 %, else the context
 * stays untuned. Later calls of the context use the table for the kernels
 * without traceback and substitution matrix; results do not change.
 * anyseq_set_option(ctx, "autotune_reset", 0) drops it; anyseq_autotune_table
 * copies the 256 caps (0 = default) to the host, and anyseq_autotune_set_table
 * installs a saved table (host array of 256 caps, each 0, 4, 8, 12 or 16,
 * else ERR_ARG; synchronous). */
anyseq_status_t anyseq_autotune(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off,
                                const uint8_t *s, const int64_t *s_off, int64_t n_pairs,
                                const anyseq_scoring_t *sc, int32_t mode, void *cuda_stream);
anyseq_status_t anyseq_autotune_table(anyseq_ctx *ctx, uint8_t *caps);
anyseq_status_t anyseq_autotune_set_table(anyseq_ctx *ctx, const uint8_t *caps);

/* Gapped strings of one alignment (the output form of the paper's one-pair
 * interface, Sec. III-C listing): from the letter codes q[0..n), s[0..m), the
 * start cell (beg_q, beg_s) and cigar_len CIGAR words of a result, write the
 * aligned letters to q_out and s_out (host buffers of cap characters),
 * '-' against a gap, code c printed as letters[c] (e.g. "ACGT"), each string
 * NUL-terminated; *len = columns. Host-only. Errors: ERR_ARG (a CIGAR op other
 * than M/I/D or running past a sequence), ERR_ALPHABET, ERR_CAPACITY (*len set). */
anyseq_status_t anyseq_gapped(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m,
                              int32_t beg_q, int32_t beg_s, const uint32_t *cigar, uint32_t cigar_len,
                              const char *letters, int32_t alphabet, char *q_out, char *s_out,
                              int64_t cap, int64_t *len);

/* Share of one batch for rank `rank` of a data-parallel job of `world` ranks
 * (the paper's inter-sequence parallelism, Sec. VI, spread over GPUs: pairs
 * are independent, so the only exchange is a gather of the results). Pairs go
 * by length-balanced round-robin of bins: the 8-bit logarithmic bins of their
 * cell counts n * m, largest first, index order inside a bin, dealt to the
 * ranks in snake order (0..W-1, W-1..0, ...). Pair counts per rank differ by
 * at most one. q_off, s_off: host arrays of n_pairs + 1 offsets (as for
 * anyseq_align_batch). idx: host array of cap entries receiving the rank's
 * pair indices in increasing order; *count = their number. Host-only and
 * deterministic: every rank computes every rank's share without
 * communication. Errors: ERR_ARG (NULL pointers, rank outside [0, world),
 * decreasing offsets), ERR_CAPACITY (cap < *count; at most ceil(n_pairs /
 * world) entries are ever needed). */
anyseq_status_t anyseq_shard_plan(const int64_t *q_off, const int64_t *s_off, int64_t n_pairs, int32_t world,
                                  int32_t rank, int64_t *idx, int64_t cap, int64_t *count);

/* ------------------------------------------------------------------------
 * Graph plans (batching, not in the paper): one batch shape of
 * anyseq_align_batch (offsets, scoring, mode; score and optimum cell) whose
 * whole launch sequence is captured once in a CUDA graph and replayed. The
 * plan owns device buffers for the letters and the results and a private
 * context, so nothing else can move the scratch the graph points at.
 *   1. anyseq_plan_create: host offsets (copied), scoring (copied), mode.
 *   2. anyseq_plan_buffers: device pointers of the plan's letter arrays
 *      (q_off[n_pairs] and s_off[n_pairs] bytes) and of its n_pairs results.
 *      Fill the letters (any stream, ordered before the run) before each run,
 *      or with anyseq_plan_upload: an asynchronous copy of q_off[n_pairs] and
 *      s_off[n_pairs] bytes from q and s (host or device memory; pinned host
 *      memory keeps the copy asynchronous) on cuda_stream.
 *   After a run, anyseq_plan_download copies the n_pairs result records to
 *   out (host or device) asynchronously on cuda_stream; they are valid after
 *   anyseq_plan_wait. Two plans of one shape on two streams let one batch's
 *   copies overlap the other's run.
 *   3. anyseq_plan_run: enqueue one run on cuda_stream. The first run executes
 *      the batched path once (sizing the scratch; it synchronises), then
 *      captures it; every later run is one graph launch and does not
 *      synchronise.
 *   4. anyseq_plan_wait: synchronise cuda_stream and report the run's letter
 *      check (ERR_ALPHABET if a code was >= alphabet).
 * Runs of one plan must not overlap. Errors: ERR_ARG, ERR_ALPHABET, ERR_CUDA.
 * ------------------------------------------------------------------------ */
typedef struct anyseq_plan anyseq_plan;

anyseq_status_t anyseq_plan_create(anyseq_plan **plan, int device, const int64_t *q_off,
                                   const int64_t *s_off, int64_t n_pairs,
                                   const anyseq_scoring_t *sc, int32_t mode);
anyseq_status_t anyseq_plan_buffers(anyseq_plan *plan, uint8_t **q, uint8_t **s,
                                    anyseq_result_t **out);
anyseq_status_t anyseq_plan_upload(anyseq_plan *plan, const uint8_t *q, const uint8_t *s, void *cuda_stream);
anyseq_status_t anyseq_plan_run(anyseq_plan *plan, void *cuda_stream);
anyseq_status_t anyseq_plan_download(anyseq_plan *plan, anyseq_result_t *out, void *cuda_stream);
anyseq_status_t anyseq_plan_wait(anyseq_plan *plan, void *cuda_stream);
anyseq_status_t anyseq_plan_destroy(anyseq_plan *plan);

/* ------------------------------------------------------------------------
 * Serving (not in the paper, whose interface aligns one pair per call):
 * request queues drained by two service lanes, each a worker thread that owns
 * a context and a CUDA stream. Pairs are submitted one at a time from any
 * thread; a pair of at least long_cells cells goes to the long lane, any other
 * to the short lane. Each lane aligns in micro-batches: it waits at most
 * max_wait_us after its oldest queued request (or until max_batch_pairs are
 * queued). The short lane aligns a batch with one anyseq_align_batch call;
 * the long lane runs its pairs side by side in one wavefront launch of
 * anyseq_align_long's kind. The lanes' kernels are capped so that both fit on
 * every SM at once (the long lane's wavefront at one CTA per SM, the short
 * lane's batched kernel at two and its wavefront launches at one), and a
 * short batch never waits for a long launch to leave the SMs. Results carry
 * score and optimum cell.
 * Admission: the letters of queued and running requests never exceed
 * mem_budget_bytes; a submit beyond it returns ANYSEQ_ERR_BUDGET and queues
 * nothing (the caller may retry later). Device scratch is the context's,
 * grown on demand within 90% of free device memory.
 * ------------------------------------------------------------------------ */
typedef struct anyseq_server anyseq_server;

typedef struct {
    int32_t device;               /* CUDA device of the worker */
    int32_t mode;                 /* anyseq_mode_t of every request */
    anyseq_scoring_t scoring;     /* copied, including the matrix */
    int64_t max_batch_pairs;      /* 0: 65536 */
    int64_t max_wait_us;          /* batching window after the oldest queued request; 0: 200 */
    int64_t long_cells;           /* n*m from which a global pair takes the wavefront path; 0: 2^22 */
    size_t mem_budget_bytes;      /* letters held by queued and running requests; 0: 1 GiB */
} anyseq_server_config_t;

/* Start the worker. Errors: ERR_ARG (bad scoring or limits), ERR_CUDA. */
anyseq_status_t anyseq_server_create(anyseq_server **srv, const anyseq_server_config_t *cfg);
/* Queue one pair (host letter codes, copied before return); *ticket names it.
 * Errors: ERR_ARG, ERR_BUDGET (admission refused). Thread-safe. */
anyseq_status_t anyseq_server_submit(anyseq_server *srv, const uint8_t *q, int64_t n,
                                     const uint8_t *s, int64_t m, uint64_t *ticket);
/* Wait for a ticket (timeout_us < 0: no limit). On return other than
 * ERR_TIMEOUT the ticket is released: *out holds its result and *latency_ns
 * (optional) the time from submit to completion. ERR_TIMEOUT keeps the ticket;
 * an alignment error of the pair is returned as its status. Thread-safe. */
anyseq_status_t anyseq_server_wait(anyseq_server *srv, uint64_t ticket, int64_t timeout_us,
                                   anyseq_result_t *out, int64_t *latency_ns);
/* "completed", "batches", "long_pairs", "rejected", "queued", "held_bytes", "busy_ms". */
anyseq_status_t anyseq_server_stat(anyseq_server *srv, const char *key, double *value);
/* Finish every queued request, stop the worker, free the context; tickets not
 * yet waited for are dropped. */
anyseq_status_t anyseq_server_destroy(anyseq_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* ANYSEQ_H */
