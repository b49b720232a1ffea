// Launchers of the batched DP kernel: dispatch by alignment mode to the
// per-mode instantiations (batch_global.cu, batch_local.cu, batch_semiglobal.cu).
#include "batch.h"

namespace anyseq {

int batch_run_global(const BatchArgs *A, int cell32, int tb, int sigp, int alphabet, int grid, cudaStream_t st,
                     bool occ, cudaError_t *err);
int batch_run_local(const BatchArgs *A, int cell32, int tb, int sigp, int alphabet, int grid, cudaStream_t st,
                    bool occ, cudaError_t *err);
int batch_run_semiglobal(const BatchArgs *A, int cell32, int tb, int sigp, int alphabet, int grid, cudaStream_t st,
                         bool occ, cudaError_t *err);

static int dispatch(const BatchArgs *A, int cell32, int mode, int tb, int sigp, int alphabet, int grid,
                    cudaStream_t st, bool occ, cudaError_t *err) {
    switch (mode) {
        case GLOBAL: return batch_run_global(A, cell32, tb, sigp, alphabet, grid, st, occ, err);
        case LOCAL: return batch_run_local(A, cell32, tb, sigp, alphabet, grid, st, occ, err);
        default: return batch_run_semiglobal(A, cell32, tb, sigp, alphabet, grid, st, occ, err);
    }
}

cudaError_t launch_batch(const BatchArgs &A, int cell32, int mode, int tb, int sigp, int grid, cudaStream_t st) {
    cudaError_t err = cudaSuccess;
    dispatch(&A, cell32, mode, tb, sigp, A.alphabet, grid, st, false, &err);
    return err;
}

int batch_blocks_per_sm(int cell32, int mode, int tb, int sigp, int alphabet) {
    cudaError_t err = cudaSuccess;
    return dispatch(nullptr, cell32, mode, tb, sigp, alphabet, 0, nullptr, true, &err);
}

}  // namespace anyseq
