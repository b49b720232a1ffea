// Instantiations of the batched DP kernel for local alignment (every lane type,
// with and without traceback, row profile or substitution matrix).
#include "batch_kernel.cuh"

namespace anyseq {

int batch_run_local(const BatchArgs *A, int cell32, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
                   cudaError_t *err) {
    return run_mode<LOCAL>(A, cell32, tb, sigp, alphabet, grid, st, occ, err);
}

}  // namespace anyseq
