// Learned band: features, path extents, banded DP with certificate (band.cu)
// and the band network (mlp.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/anyseq.h"

namespace anyseq {

struct BandArgs {
    const uint32_t *q2, *s2;        // 2-bit packed letters
    const int64_t *q_off, *s_off;
    const int32_t *list;            // pairs to try
    int64_t n_list;
    int32_t *counter;               // zeroed work counter
    const int32_t *centre, *width;  // band per pair (diagonals)
    uint32_t rowprof[5];
    int32_t o, e, mmax;
    int32_t strict;                 // 1: accept only S > X
    int32_t *scratch;               // per slot 2 * scratch_cols
    int64_t scratch_cols;
    int32_t *score;                 // per pair
    int32_t *accept;                // per pair: 1 if the certificate holds
    unsigned long long *cells;      // device: cells relaxed by the pass (optional)
};

cudaError_t launch_band(const BandArgs &A, int grid, cudaStream_t st);
int band_blocks_per_sm();
cudaError_t launch_kmer_hist(const uint32_t *q2, const uint32_t *s2, const int64_t *q_off, const int64_t *s_off,
                             const int32_t *pairs, int64_t n_pairs, float *feat, cudaStream_t st);
cudaError_t launch_path_extent(const int64_t *q_off, const int64_t *s_off, const anyseq_result_t *res,
                               const uint32_t *cigar, int64_t n_pairs, int32_t *dmin, int32_t *dmax, cudaStream_t st);

// Band network 64 -> 128 -> 128 -> 2 (ReLU), bfloat16 weights, float32 accumulation.
constexpr int MLP_IN = 64, MLP_H = 128, MLP_OUT = 2;
constexpr int MLP_NPARAM = MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H * MLP_OUT + MLP_OUT;

// Parameter layout in a flat float array: W1 (64x128 row-major), b1, W2, b2, W3 (128x2), b3.
struct MlpDev {
    float *master;      // float32 master copy (training)
    uint16_t *w16;      // bfloat16 copies of W1, W2, W3 (same offsets as master for the weights)
    float *grad;        // float32 gradients
    float *m, *v;       // Adam moments
};

cudaError_t launch_mlp_forward(const MlpDev &P, const float *x, int64_t B, float *y, cudaStream_t st);
// Loss of a batch (sum over pairs, written to *loss) and gradients accumulated into P.grad (zeroed by the caller).
cudaError_t launch_mlp_grad(const MlpDev &P, const float *x, const float *target, int64_t B, float *loss,
                            cudaStream_t st);
cudaError_t launch_mlp_adam(const MlpDev &P, int64_t step, float lr, cudaStream_t st);
cudaError_t launch_mlp_round(const MlpDev &P, cudaStream_t st);

}  // namespace anyseq
