// Input staging of the batched path: letter validation, 2-bit packing with
// 128-bit loads, the int16 range test, and a counting sort of the pairs into
// length buckets (longest first) that the persistent kernel consumes as its
// work queue. Pairs with an empty sequence get their closed-form result here.
#include "batch.h"
#include "common.cuh"

namespace anyseq {

constexpr int NBUCKET = 65536;

// one thread per output word: 16 letters (one 16-byte load when aligned)
__global__ void pack2bit_kernel(const uint8_t *codes, int64_t len, uint32_t *out, int32_t alphabet,
                                int32_t *bad) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nw = (len + 15) >> 4;
    for (; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        int64_t k0 = w << 4;
        uint8_t b[16];
        if (k0 + 16 <= len && ((reinterpret_cast<uintptr_t>(codes + k0) & 15u) == 0)) {
            uint4 v = *reinterpret_cast<const uint4 *>(codes + k0);
            *reinterpret_cast<uint4 *>(b) = v;
        } else {
#pragma unroll
            for (int t = 0; t < 16; t++) b[t] = (k0 + t < len) ? codes[k0 + t] : 0;
        }
        uint32_t word = 0;
        int badv = 0;
#pragma unroll
        for (int t = 0; t < 16; t++) {
            badv |= (b[t] >= alphabet);
            word |= (uint32_t)(b[t] & 3u) << (2 * t);
        }
        if (out) out[w] = word;
        if (badv) *bad = 1;
    }
}

// bytes only (alphabets above 4): validation
__global__ void validate_kernel(const uint8_t *codes, int64_t len, int32_t alphabet, int32_t *bad) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; k < len; k += (int64_t)gridDim.x * blockDim.x)
        if (codes[k] >= alphabet) *bad = 1;
}



__global__ void bin_kernel(PrepArgs P) {
    // grid-stride loop with a warp-uniform trip count (the shuffles below need the whole warp)
    unsigned long long local[2] = {0, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < P.n_pairs; p0 += stride) {
        const int64_t p = p0 + (base - (int64_t)blockIdx.x * blockDim.x);
        if (p >= P.n_pairs) continue;
        if (P.select && !P.select[p]) { P.key[p] = 0xFFFFFFFFu; continue; }
        int64_t n = P.q_off[p + 1] - P.q_off[p];
        int64_t m = P.s_off[p + 1] - P.s_off[p];
        if (n == 0 || m == 0) {
            int32_t sc = 0;
            if (P.mode == GLOBAL) sc = (n + m == 0) ? 0 : P.o + (int32_t)(n + m) * P.e;
            P.score[p] = sc;
            P.end_q[p] = P.mode == GLOBAL ? (int32_t)n : 0;
            P.end_s[p] = P.mode == GLOBAL ? (int32_t)m : 0;
            P.flags[p] = 0;
            P.key[p] = 0xFFFFFFFFu;
            unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long *>(&P.counts[2]), 1ull);
            if (P.trivial) P.trivial[pos] = (int32_t)p;
            continue;
        }
        uint32_t prec = (P.force32 || !fits_int16(n, m, P.smax, P.smin, P.o, P.e, P.mode)) ? 1u : 0u;
        uint32_t k = prec * NBUCKET + (lbucket(n) << 8) + lbucket(m);
        P.key[p] = k;
        atomicAdd(&P.hist[k], 1u);
        local[prec]++;
    }
    // one counter update per warp and class
#pragma unroll
    for (int c = 0; c < 2; c++) {
        unsigned long long v = local[c];
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(reinterpret_cast<unsigned long long *>(&P.counts[c]), v);
    }
}

// Exclusive offsets in DESCENDING key order within each precision class, in
// place: hist[k] becomes the first list position of bucket k. Two passes over
// tiles of 1024 buckets (reversed order inside a class): tile sums, then a
// block scan per tile offset by the sums of the earlier tiles of its class.
constexpr int SCAN_TILE = 1024;
constexpr int TILES_PER_CLASS = NBUCKET / SCAN_TILE;

__device__ __forceinline__ uint32_t *tile_bucket(uint32_t *hist, int tile, int x) {
    int cls = tile / TILES_PER_CLASS, t = tile % TILES_PER_CLASS;
    return hist + cls * NBUCKET + (NBUCKET - 1 - (t * SCAN_TILE + x));
}

__global__ void tile_sum_kernel(uint32_t *hist, uint32_t *tile_sum) {
    __shared__ uint32_t red[32];
    uint32_t v = *tile_bucket(hist, blockIdx.x, threadIdx.x);
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w = red[threadIdx.x];
        for (int off = 16; off; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
        if (threadIdx.x == 0) tile_sum[blockIdx.x] = w;
    }
}

__global__ void tile_scan_kernel(uint32_t *hist, const uint32_t *tile_sum) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t base;
    const int tile = blockIdx.x, x = threadIdx.x, lane = x & 31, w = x >> 5;
    if (x == 0) {
        uint32_t b = 0;
        int first = (tile / TILES_PER_CLASS) * TILES_PER_CLASS;
        for (int t = first; t < tile; t++) b += tile_sum[t];
        base = b;
    }
    uint32_t *cell = tile_bucket(hist, tile, x);
    uint32_t v = *cell, inc = v;
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = warp_tot[lane], ti = t;
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ti, off);
            if (lane >= off) ti += y;
        }
        warp_tot[lane] = ti - t;
    }
    __syncthreads();
    *cell = base + warp_tot[w] + inc - v;
}

__global__ void scatter_kernel(PrepArgs P) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; p < P.n_pairs; p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t k = P.key[p];
        if (k == 0xFFFFFFFFu) continue;
        uint32_t pos = atomicAdd(&P.hist[k], 1u);
        if (k < NBUCKET) P.list16[pos] = (int32_t)p;
        else P.list32[pos] = (int32_t)p;
    }
}

cudaError_t launch_pack2bit(const uint8_t *codes, int64_t len, uint32_t *out, int32_t alphabet, int32_t *bad,
                            cudaStream_t st) {
    int64_t b = ((len + 15) / 16 + 255) / 256;
    pack2bit_kernel<<<(int)(b < 1 ? 1 : (b > 65535 ? 65535 : b)), 256, 0, st>>>(codes, len, out, alphabet, bad);
    return cudaGetLastError();
}

cudaError_t launch_prep(const PrepArgs &P, cudaStream_t st) {
    const int T = 256;
    auto blocks = [](int64_t work) { int64_t b = (work + 255) / 256; return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b)); };
    cudaMemsetAsync(P.hist, 0, 2 * NBUCKET * sizeof(uint32_t), st);
    cudaMemsetAsync(P.counts, 0, 3 * sizeof(int64_t), st);
    cudaMemsetAsync(P.bad_code, 0, sizeof(int32_t), st);
    if (P.alphabet <= 4) {
        pack2bit_kernel<<<blocks((P.q_len + 15) / 16), T, 0, st>>>(P.q, P.q_len, P.q2, P.alphabet, P.bad_code);
        pack2bit_kernel<<<blocks((P.s_len + 15) / 16), T, 0, st>>>(P.s, P.s_len, P.s2, P.alphabet, P.bad_code);
    } else {
        validate_kernel<<<blocks(P.q_len), T, 0, st>>>(P.q, P.q_len, P.alphabet, P.bad_code);
        validate_kernel<<<blocks(P.s_len), T, 0, st>>>(P.s, P.s_len, P.alphabet, P.bad_code);
    }
    bin_kernel<<<blocks(P.n_pairs), T, 0, st>>>(P);
    tile_sum_kernel<<<2 * TILES_PER_CLASS, SCAN_TILE, 0, st>>>(P.hist, P.tile_sum);
    tile_scan_kernel<<<2 * TILES_PER_CLASS, SCAN_TILE, 0, st>>>(P.hist, P.tile_sum);
    scatter_kernel<<<blocks(P.n_pairs), T, 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace anyseq
