// Long-pair wavefront kernel (wave.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace anyseq {

// One global pass over q[q0 .. q0+n) x s[s0 .. s0+m) (read reversed when rev),
// column-0 open tb. Its stripes are numbered stripe0 .. stripe0 + ceil(n/512) - 1
// in the launch; border rows at border + border_off (2 x m), progress counters
// at prog + stripe0, last row written at last_H/last_E + out_off (m + 1 values).
struct WavePass {
    int64_t q0, s0;
    int32_t n, m;
    int32_t tb, rev;
    int64_t border_off;
    int64_t out_off;
    int32_t stripe0, pad_;
    int64_t dir_off;              // traceback: first direction word of the pass
};

struct WaveArgs {
    const uint32_t *q2, *s2;      // 2-bit packed letters (global positions)
    const WavePass *passes;       // device table, sorted by stripe0
    int32_t n_passes, n_stripes;
    int32_t o, e;                 // gap open, extend
    uint32_t rowprof[5];          // profile words (global padding in word 4)
    int2 *border;
    int32_t *prog;                // per stripe: border blocks published (zeroed)
    int32_t *stripe_counter;      // zeroed
    int32_t *err;                 // zeroed; 1 after a wait gave up
    int32_t *last_H, *last_E;     // optional outputs
    int64_t spin_limit;           // iterations of one wait
    int32_t rows_per_lane;        // 4, 8 or 16 (stripes of 32 lanes x rows_per_lane rows; traceback 8 or 16)
    uint32_t *dirs;               // optional: traceback direction words (global mode)
    int32_t mode;                 // GLOBAL, LOCAL, SEMIGLOBAL or an anchored mode (every pass)
    uint64_t *best;               // local / semi-global: per pass the best cell's key (initialised)
    int32_t cell;                 // global passes: 0 = by stripe count, 1 = 3-input maximum, 2 = two-step
    // substitution matrix (alphabets above 4 letters): letter codes one byte
    // each, and sigma - open - extend per (query, subject) letter pair
    int32_t mat;                  // 0: 2-bit letters and row profiles; 1: the matrix path
    int32_t ctas_per_sm;          // 0: as many CTAs per SM as fit; else at most this many
    int32_t split;                // global three-input-maximum passes: 0 by stripe count, 1 split steps, 2 plain
    int32_t alphabet;
    const uint8_t *q8, *s8;
    const int8_t *sig;            // alphabet x alphabet bytes (device)
    int32_t sig_pad;              // sigma' of the padding rows above a pass
    int32_t no_spread;            // 0: hold back first draws so that the first stripes land on distinct SMs
    int32_t grid_sms;             // set by launch_wave: the SMs the grid was sized for
};

// Wavefront-only modes of the start-cell pass of a local or semi-global
// long-pair traceback. The pass runs over the reversed prefixes that end at
// the optimum cell, so its values are the global scores of the substrings
// ending there: global initialisation, no clamp at 0, and the best cell
// (largest score, then smallest reversed row, then smallest reversed column)
// over every cell (ANCHORED_LOCAL) or over the last row and column
// (ANCHORED_SEMIGLOBAL, whose cells are the starts in row 0 or column 0).
constexpr int32_t ANCHORED_LOCAL = 3, ANCHORED_SEMIGLOBAL = 4;
// The initialisation (column 0, row 0, padding rows) of a mode.
__host__ __device__ constexpr int32_t wave_init_mode(int32_t mode) {
    return (mode == LOCAL || mode == SEMIGLOBAL) ? mode : GLOBAL;
}

// Rows per lane of a launch over total_rows rows (the sum of the passes' row
// counts) in n_passes passes: the tallest stripes (16, 8, then 4 rows per lane)
// that still give about three stripes for every four SMs; local passes always 8,
// semi-global passes 16 or 4. forced (4, 8 or 16; 0: automatic) overrides the
// choice within what each mode has; min8 keeps at least 8 (the allocation-free
// scratch is sized for 8-row stripes). The stripe table of a launch
// must be built with this value, and WaveArgs.rows_per_lane set to it.
int wave_rows_per_lane(int64_t total_rows, int num_sms, int64_t n_passes, int mode, int forced = 0, bool min8 = false);
cudaError_t launch_wave(const WaveArgs &A, int num_sms, cudaStream_t st);
constexpr int WAVE_LANES = 32;    // lanes per stripe
constexpr int WAVE_SIG_BYTES = 1024;  // shared copy of the sigma' table (alphabets up to 32)
constexpr int WAVE_MIN_ROWS = 256;  // rows of the shortest stripe (8 rows per lane)

}  // namespace anyseq
