// Traceback launchers of the batched path (tb.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace anyseq {

struct TbWalkArgs {
    int64_t n_pairs;
    int32_t mode;
    const int64_t *q_off, *s_off;
    const int32_t *end_q, *end_s;
    const uint32_t *dirs;
    const int64_t *dir_base;
    const int32_t *lay_pad, *lay_ch0;
    const int32_t *lay_r;  // rows per lane of each pair (nullptr: rows_per_lane for all)
    uint32_t *tmp;        // per pair n + m + 1 words at q_off[p] + s_off[p] + p
    int64_t *cig_len;
    int32_t *beg_q, *beg_s;
    // layout of the direction words: chunks of lanes_per_chunk lanes x R rows,
    // steps = m + lanes_per_chunk - 1 per chunk, ceil(R / 8) words per lane and
    // step (byte planes of 8 rows each)
    int32_t lanes_per_chunk, rows_per_lane;
    int32_t walker;       // 0: by batch size, 1: a warp per pair, 2: a thread per pair
};

// Sizes each pair's direction words with the DP kernel's own item plan (rows
// per lane up to rmax, or fixed_r when nonzero) and records its layout.
cudaError_t launch_tb_plan(const int32_t *list, const int64_t *n_list, int per_item, int64_t max_items,
                           const int64_t *q_off, const int64_t *s_off, int64_t *words, int32_t *lay_pad,
                           int32_t *lay_ch0, int32_t *lay_r, int rmax, int fixed_r, cudaStream_t st);
cudaError_t launch_tb_walk(const TbWalkArgs &W, cudaStream_t st);
cudaError_t launch_tb_compact(int64_t n_pairs, const int64_t *q_off, const int64_t *s_off, const uint32_t *tmp,
                              const int64_t *cig_len, const int64_t *cig_off, uint32_t *out, cudaStream_t st);

}  // namespace anyseq
