// Traceback of the batched path: layout of the direction words, the walk from
// the optimum cell back to the start (predecessor rule of the relaxation
// function, Sec. III-B), run-length CIGAR, and compaction into the caller's
// buffer.
//
// Direction words: for every pair, row chunk (from the first chunk holding a
// real row), step s and lane g, one 32-bit word for the lane's 8 rows:
//   byte 0: s0, byte 1: s1, byte 2: E opened, byte 3: F opened  (bit r = row r)
// H-source from (s0, s1): global/semi-global (1,x) DIAG, (0,1) E, (0,0) F;
// local (1,0) DIAG, (0,1) E, (0,0) F, (1,1) ZERO (H = 0 ends the alignment).
#include "batch.h"
#include "common.cuh"
#include "tb.h"

namespace anyseq {

__global__ void tb_plan_kernel(const int32_t *list, const int64_t *n_list_p, int per_item, const int64_t *q_off,
                               const int64_t *s_off, int64_t *words, int32_t *lay_pad, int32_t *lay_ch0) {
    const int64_t n_list = *n_list_p;
    const int64_t n_items = (n_list + per_item - 1) / per_item;
    for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < n_items;
         item += (int64_t)gridDim.x * blockDim.x) {
        ItemPlan P = plan_item(list, n_list, item, per_item, q_off, s_off, TB_R, false);
        const int32_t CH = GROUP * TB_R;
        for (int k = 0; k < per_item; k++) {
            int32_t p = P.pid[k];
            if (p < 0) continue;
            int32_t pad = P.nch * CH - P.n[k];
            int32_t ch0 = pad / CH;
            words[p] = (int64_t)(P.nch - ch0) * (P.m[k] + GROUP - 1) * GROUP;
            lay_pad[p] = pad;
            lay_ch0[p] = ch0;
        }
    }
}

struct Runs {
    uint32_t *out;
    int64_t k;
    uint32_t op, len;
    __device__ void push(uint32_t o, uint32_t count) {
        if (count == 0) return;
        if (len && o != op) {
            out[k++] = (len << 4) | op;
            len = 0;
        }
        op = o;
        len += count;
    }
    __device__ void flush() {
        if (len) out[k++] = (len << 4) | op;
        len = 0;
    }
};

// One thread per pair: walk the direction words from the optimum cell.
__global__ void tb_walk_kernel(TbWalkArgs W) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < W.n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = (int32_t)(W.q_off[p + 1] - W.q_off[p]);
        const int32_t m = (int32_t)(W.s_off[p + 1] - W.s_off[p]);
        Runs rl;
        rl.out = W.tmp + W.q_off[p] + W.s_off[p] + p;
        rl.k = 0;
        rl.op = 0;
        rl.len = 0;
        int32_t i = W.end_q[p], j = W.end_s[p];
        if (n == 0 || m == 0) {
            if (W.mode == GLOBAL) {
                rl.push(2u, (uint32_t)m);
                rl.push(1u, (uint32_t)n);
                i = 0;
                j = 0;
            }
        } else {
            const uint32_t *dw = W.dirs + W.dir_base[p];
            const int32_t pad = W.lay_pad[p], ch0 = W.lay_ch0[p];
            const int64_t S = m + GROUP - 1;
            auto word = [&](int32_t ii, int32_t jj, int32_t &r) -> uint32_t {
                int32_t ip = ii + pad - 1;
                int32_t ch = ip / (GROUP * TB_R);
                int32_t gl = (ip % (GROUP * TB_R)) / TB_R;
                r = ip % TB_R;
                int64_t s = (int64_t)(jj - 1) + gl;
                return dw[((int64_t)(ch - ch0) * S + s) * GROUP + gl];
            };
            int state = 0;  // 0: H, 1: E, 2: F
            // every step moves up or left within two iterations; the bound and the
            // boundary checks keep a corrupt word from leaving the pair's words
            for (int64_t guard = 2 * ((int64_t)n + m) + 4; guard > 0; guard--) {
                if (state != 0 && (i <= 0 || j <= 0)) break;
                if (state == 0) {
                    if (i == 0 && j == 0) break;
                    if (W.mode != GLOBAL) {
                        if (i == 0 || j == 0) break;
                    } else {
                        if (j == 0) { rl.push(1u, (uint32_t)i); i = 0; break; }
                        if (i == 0) { rl.push(2u, (uint32_t)j); j = 0; break; }
                    }
                    int32_t r;
                    uint32_t w = word(i, j, r);
                    uint32_t s0 = (w >> r) & 1u, s1 = (w >> (8 + r)) & 1u;
                    if (W.mode == LOCAL) {
                        if (s0 && s1) break;  // H = 0: the local alignment starts here
                        if (s0) { rl.push(0u, 1u); i--; j--; }
                        else state = s1 ? 1 : 2;
                    } else {
                        if (s0) { rl.push(0u, 1u); i--; j--; }
                        else state = s1 ? 1 : 2;
                    }
                } else if (state == 1) {
                    int32_t r;
                    uint32_t w = word(i, j, r);
                    rl.push(1u, 1u);
                    if ((w >> (16 + r)) & 1u) state = 0;
                    i--;
                } else {
                    int32_t r;
                    uint32_t w = word(i, j, r);
                    rl.push(2u, 1u);
                    if ((w >> (24 + r)) & 1u) state = 0;
                    j--;
                }
            }
        }
        rl.flush();
        W.cig_len[p] = rl.k;
        W.beg_q[p] = i;
        W.beg_s[p] = j;
    }
}

// Reverse each pair's runs into the output buffer at its offset.
__global__ void tb_compact_kernel(int64_t n_pairs, const int64_t *q_off, const int64_t *s_off, const uint32_t *tmp,
                                  const int64_t *cig_len, const int64_t *cig_off, uint32_t *out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t *src = tmp + q_off[p] + s_off[p] + p;
        const int64_t len = cig_len[p], off = cig_off[p];
        for (int64_t t = 0; t < len; t++) out[off + t] = src[len - 1 - t];
    }
}

static int grid_of(int64_t work) {
    int64_t b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

cudaError_t launch_tb_plan(const int32_t *list, const int64_t *n_list, int per_item, int64_t max_items,
                           const int64_t *q_off, const int64_t *s_off, int64_t *words, int32_t *lay_pad,
                           int32_t *lay_ch0, cudaStream_t st) {
    tb_plan_kernel<<<grid_of(max_items), 256, 0, st>>>(list, n_list, per_item, q_off, s_off, words, lay_pad, lay_ch0);
    return cudaGetLastError();
}

cudaError_t launch_tb_walk(const TbWalkArgs &W, cudaStream_t st) {
    tb_walk_kernel<<<grid_of(W.n_pairs), 256, 0, st>>>(W);
    return cudaGetLastError();
}

cudaError_t launch_tb_compact(int64_t n_pairs, const int64_t *q_off, const int64_t *s_off, const uint32_t *tmp,
                              const int64_t *cig_len, const int64_t *cig_off, uint32_t *out, cudaStream_t st) {
    tb_compact_kernel<<<grid_of(n_pairs), 256, 0, st>>>(n_pairs, q_off, s_off, tmp, cig_len, cig_off, out);
    return cudaGetLastError();
}

}  // namespace anyseq
