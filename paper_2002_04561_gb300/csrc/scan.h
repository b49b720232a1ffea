// Device prefix sums (scan.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace anyseq {
// out[i] = sum of in[0..i); *total (device, may be null) = sum of all; tmp has scan_tmp_words(n) words.
cudaError_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, int64_t *total,
                               cudaStream_t st);
int64_t scan_tmp_words(int64_t n);
}  // namespace anyseq
