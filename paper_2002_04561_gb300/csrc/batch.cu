// Launchers of the batched DP kernel: dispatch by alignment mode and lane type
// to the instantiations in batch_{global,local,semiglobal}_{i16,i32}.cu.
#include "batch.h"

namespace anyseq {

int batch_run_global_i16(const BatchArgs *A, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
                         cudaError_t *err);
int batch_run_global_i32(const BatchArgs *A, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
                         cudaError_t *err);
int batch_run_local_i16(const BatchArgs *A, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
                        cudaError_t *err);
int batch_run_local_i32(const BatchArgs *A, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
                        cudaError_t *err);
int batch_run_semiglobal_i16(const BatchArgs *A, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
                             cudaError_t *err);
int batch_run_semiglobal_i32(const BatchArgs *A, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
                             cudaError_t *err);

static int dispatch(const BatchArgs *A, int cell32, int mode, int tb, int sigp, int alphabet, int grid,
                    cudaStream_t st, bool occ, cudaError_t *err) {
    switch (mode) {
        case GLOBAL:
            return cell32 ? batch_run_global_i32(A, tb, sigp, alphabet, grid, st, occ, err)
                          : batch_run_global_i16(A, tb, sigp, alphabet, grid, st, occ, err);
        case LOCAL:
            return cell32 ? batch_run_local_i32(A, tb, sigp, alphabet, grid, st, occ, err)
                          : batch_run_local_i16(A, tb, sigp, alphabet, grid, st, occ, err);
        default:
            return cell32 ? batch_run_semiglobal_i32(A, tb, sigp, alphabet, grid, st, occ, err)
                          : batch_run_semiglobal_i16(A, tb, sigp, alphabet, grid, st, occ, err);
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
