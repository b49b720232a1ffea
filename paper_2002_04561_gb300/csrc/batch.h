// Arguments and launchers of the batched kernels (host and device side).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace anyseq {

// Range test for exact int16 lanes: every H, E, F, Hoe and diagonal term of
// the pair stays inside [-16000, 16000] (bounds from the recurrences: H is at
// most max(sigma,0) * min(n,m); below, global H(i,j) is at least two gaps,
// semi-global at least one, local at least 0; E/F add one more open+extend).
__host__ __device__ __forceinline__ bool fits_int16(int64_t n, int64_t m, int32_t smax, int32_t smin, int32_t o, int32_t e,
                                           int32_t mode) {
    int64_t mn = n < m ? n : m;
    int64_t hi = (int64_t)(smax > 0 ? smax : 0) * (mn + 1) + (smax > 0 ? smax : 0);
    int64_t lo;
    int64_t ox = o, ex = e, sm = smin < 0 ? smin : 0;
    if (mode == GLOBAL) lo = 3 * ox + (n + m + 2) * ex + sm;
    else if (mode == SEMIGLOBAL) lo = 2 * ox + (mn + 2) * ex + sm;
    else lo = ox + 2 * ex + sm;
    // local mode packs the optimum column of both halves into 16 bits each
    return hi <= 16000 && lo >= -16000 && (mode != LOCAL || m < 65535);
}

// 8-bit logarithmic length bucket, 8 sub-steps per octave.
__host__ __device__ __forceinline__ uint32_t lbucket(int64_t x) {
    if (x < 16) return (uint32_t)x;
#ifdef __CUDA_ARCH__
    const int lg = 63 - __clzll(x);
#else
    const int lg = 63 - __builtin_clzll((unsigned long long)x);
#endif
    uint32_t q = 16u + (uint32_t)(lg - 4) * 8u + (uint32_t)((x >> (lg - 3)) & 7);
    return q > 255u ? 255u : q;
}

struct BatchArgs {
    const uint32_t *q2, *s2;        // 2-bit packed letters, 16 per word, global positions
    const int64_t *q_off, *s_off;   // n_pairs + 1 offsets
    const int32_t *list;            // pairs to process, sorted longest first
    const int64_t *n_list;          // device: number of entries in list
    int32_t *counter;               // device: work-item counter (zeroed before launch)
    uint32_t rowprof[5];            // profile word per query letter 0..3 and padding (4)
    int32_t o, e;                   // gap open, extend (<= 0)
    int32_t *scratch;               // border rows of multi-chunk slots: per group 2 * scratch_cols
    int64_t scratch_cols;
    int32_t *score, *end_q, *end_s; // outputs per pair
    uint32_t *flags;
    // substitution matrix path (alphabet > 4): letters as bytes and the table
    // sigma'(a, b) = sigma(a, b) - open - extend (alphabet x alphabet int8, >= 0)
    const uint8_t *q8, *s8;
    const int8_t *sig_tab;
    int32_t alphabet;
    int32_t sig_pad;                // sigma' of the padding rows
    // traceback (direction words, see tb.cu): per pair base word, padding rows, first chunk
    uint32_t *dirs;
    const int64_t *dir_base;
    int32_t *lay_pad, *lay_ch0;
    // autotuning (row-profile kernels without traceback): the rows-per-lane cap
    // per length bin of a work item's longest query (0: the kernel's own), and
    // optional per-bin statistics (SM cycles, cells) of the items
    const uint8_t *rmax_tab;
    unsigned long long *bin_stats;
};

// Work item of the persistent batched kernels: per_item consecutive pairs of a
// sorted list, their row chunking (nch chunks of 16*R rows) and column count.
struct ItemPlan {
    int32_t pid[4];
    int32_t n[4], m[4];
    int32_t nch, R, Mit, count;
};

__device__ __forceinline__ ItemPlan plan_item(const int32_t *list, int64_t n_list, int64_t item, int per_item,
                                              const int64_t *q_off, const int64_t *s_off, int rmax) {
    ItemPlan P;
    int32_t nmax = 0;
    P.Mit = 0;
    P.count = 0;
    for (int k = 0; k < 4; k++) {
        P.pid[k] = -1;
        P.n[k] = 0;
        P.m[k] = 0;
    }
    for (int k = 0; k < per_item; k++) {
        int64_t idx = item * per_item + k;
        if (idx < n_list) {
            int32_t p = list[idx];
            P.pid[k] = p;
            P.n[k] = (int32_t)(q_off[p + 1] - q_off[p]);
            P.m[k] = (int32_t)(s_off[p + 1] - s_off[p]);
            nmax = max(nmax, P.n[k]);
            P.Mit = max(P.Mit, P.m[k]);
            P.count++;
        }
    }
    P.nch = (nmax + 16 * rmax - 1) / (16 * rmax);
    if (P.nch < 1) P.nch = 1;
    int R = (nmax + 16 * P.nch - 1) / (16 * P.nch);
    if (R < 2) R = 2;
    if (R > rmax) R = rmax;
    P.R = R;
    return P;
}

// sigp: 0 = row-profile words (alphabet <= 4), 1 = shared-memory query profile (matrix, alphabet <= 32)
cudaError_t launch_batch(const BatchArgs &A, int cell32, int mode, int tb, int sigp, int grid, cudaStream_t st);
int batch_blocks_per_sm(int cell32, int mode, int tb, int sigp, int alphabet);
constexpr int QP_ROWS = 128;        // rows of the shared-memory query profile (chunk of 16 lanes x 8 rows)
// Threads per CTA of the batched kernel and the CTAs per SM its register
// budget is compiled for: 4-warp CTAs, four per SM (16 warps at 128
// registers). Measured on short reads: 2 % faster than 8-warp CTAs at the same
// occupancy; 20 or 24 warps at 12 rows per lane (80-96 registers) were slower.
__host__ __device__ constexpr int batch_threads(int sigp) { return sigp ? 128 : 128; }
__host__ __device__ constexpr int batch_min_ctas(int sigp) { return sigp ? 4 : 4; }
// Rows per lane of the matrix-path kernels: at most TB_R (their query profile
// has a TB_R-byte slot per lane), exactly TB_R with traceback. The row-profile
// kernels pick R per work item up to row_rmax: 16, or for local int16x2, which
// also keeps per-row maxima and columns, 12 (10 with traceback flags: at 12
// that variant spills).
constexpr int TB_R = 8;
__host__ __device__ constexpr int row_rmax(int mode, int pairs, bool tb) {
    return (mode == LOCAL && pairs == 2) ? (tb ? 10 : 12) : 16;
}
// Smallest rows-per-lane cap a tuned table may set (a chunk of GROUP * 4 rows).
constexpr int TUNE_MIN_R = 4;

// Packing, range tests and length binning (pack.cu).
struct PrepArgs {
    const uint8_t *q, *s;           // letter codes (device)
    const int64_t *q_off, *s_off;
    int64_t n_pairs, q_len, s_len;
    int32_t alphabet;
    uint32_t *q2, *s2;              // 2-bit packed outputs (alphabet <= 4)
    int32_t *bad_code;              // device flag: a code >= alphabet was seen
    // range-test inputs
    int32_t smax, smin, o, e, mode;
    // binning
    uint32_t *hist;                 // 2 * 65536 bucket counters
    uint32_t *tile_sum;             // 128 per-tile sums of the bucket scan
    uint32_t *key;                  // per pair bucket (or 0xFFFFFFFF: trivial pair)
    int32_t *list16, *list32;       // sorted outputs
    int64_t *counts;                // [0] int16 pairs, [1] int32 pairs, [2] trivial pairs
    int32_t *trivial;               // pairs with n == 0 or m == 0
    int32_t *score, *end_q, *end_s; // for trivial pairs
    uint32_t *flags;
    int32_t force32;                // route every pair to 32-bit lanes
    const uint8_t *select;          // optional: only pairs with select[p] != 0 are touched
};

cudaError_t launch_prep(const PrepArgs &P, cudaStream_t st);
cudaError_t launch_pack2bit(const uint8_t *codes, int64_t len, uint32_t *out, int32_t alphabet, int32_t *bad,
                            cudaStream_t st);

}  // namespace anyseq
