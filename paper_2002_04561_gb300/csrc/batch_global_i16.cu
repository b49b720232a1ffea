// Instantiations of the batched DP kernel for global alignment in int16x2 lanes
// (with and without traceback, row profile or substitution matrix).
#include "batch_kernel.cuh"

namespace anyseq {

int batch_run_global_i16(const BatchArgs *A, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
                         cudaError_t *err) {
    return run_mode<CellI16x2, GLOBAL>(A, tb, sigp, alphabet, grid, st, occ, err);
}

}  // namespace anyseq
