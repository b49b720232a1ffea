// Arguments and launchers of the batched kernels (host and device side).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace anyseq {

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
};

cudaError_t launch_batch(const BatchArgs &A, int cell32, int mode, int grid, cudaStream_t st);
int batch_blocks_per_sm(int cell32, int mode);

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
};

cudaError_t launch_prep(const PrepArgs &P, cudaStream_t st);

}  // namespace anyseq
