// Exclusive prefix sum of int64 counts on the device (tile scan, scan of the
// tile sums, add-back), used to lay out per-pair variable-size outputs.
#include "scan.h"

namespace anyseq {

constexpr int SCAN_T = 1024;

__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t *warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = v;
    for (int off = 1; off < 32; off <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t t = warp_tot[lane], ti = t;
        for (int off = 1; off < 32; off <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, ti, off);
            if (lane >= off) ti += y;
        }
        warp_tot[lane] = ti - t;
    }
    __syncthreads();
    int64_t r = inc + warp_tot[w];
    __syncthreads();
    return r;
}

__global__ void scan_tiles_kernel(const int64_t *in, int64_t *out, int64_t n, int64_t *tile_sums) {
    __shared__ int64_t warp_tot[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    int64_t inc = block_incl_scan(v, warp_tot);
    if (i < n) out[i] = inc - v;
    if (threadIdx.x == SCAN_T - 1) tile_sums[blockIdx.x] = inc;
}

// single block: exclusive scan of the tile sums in place, total at tile_sums[ntiles]
__global__ void scan_sums_kernel(int64_t *tile_sums, int64_t ntiles, int64_t *total) {
    __shared__ int64_t warp_tot[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < ntiles; base += SCAN_T) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < ntiles ? tile_sums[i] : 0;
        int64_t inc = block_incl_scan(v, warp_tot);
        if (i < ntiles) tile_sums[i] = carry + inc - v;
        __shared__ int64_t last;
        if (threadIdx.x == SCAN_T - 1) last = inc;
        __syncthreads();
        carry += last;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_add_kernel(int64_t *out, int64_t n, const int64_t *tile_sums) {
    int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
    if (i < n) out[i] += tile_sums[blockIdx.x];
}

cudaError_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, int64_t *total,
                               cudaStream_t st) {
    int64_t ntiles = (n + SCAN_T - 1) / SCAN_T;
    if (ntiles < 1) ntiles = 1;
    scan_tiles_kernel<<<(unsigned)ntiles, SCAN_T, 0, st>>>(in, out, n, tmp);
    scan_sums_kernel<<<1, SCAN_T, 0, st>>>(tmp, ntiles, total);
    scan_add_kernel<<<(unsigned)ntiles, SCAN_T, 0, st>>>(out, n, tmp);
    return cudaGetLastError();
}

int64_t scan_tmp_words(int64_t n) { return (n + SCAN_T - 1) / SCAN_T + 2; }

}  // namespace anyseq
