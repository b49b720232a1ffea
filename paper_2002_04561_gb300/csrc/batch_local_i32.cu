// Instantiations of the batched DP kernel for local alignment in int32 lanes
// (with and without traceback, row profile or substitution matrix).
#include "batch_kernel.cuh"

namespace anyseq {

int batch_run_local_i32(const BatchArgs *A, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
                        cudaError_t *err) {
    return run_mode<CellI32, LOCAL>(A, tb, sigp, alphabet, grid, st, occ, err);
}

}  // namespace anyseq
