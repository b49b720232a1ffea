// Traceback of the batched path: layout of the direction words, the walk from
// the optimum cell back to the start (predecessor rule of the relaxation
// function, Sec. III-B), run-length CIGAR, and compaction into the caller's
// buffer.
//
// Direction words: for every pair, row chunk (from the first chunk holding a
// real row), step s, lane g and k < ceil(R / 8), one 32-bit word for rows
// 8k..8k+7 of the lane's R rows:
//   byte 0: s0, byte 1: s1, byte 2: E opened, byte 3: F opened  (bit t = row 8k+t)
// H-source from (s0, s1): global/semi-global (1,x) DIAG, (0,1) E, (0,0) F;
// local (1,0) DIAG, (0,1) E, (0,0) F, (1,1) ZERO (H = 0 ends the alignment).
#include "batch.h"
#include "common.cuh"
#include "tb.h"

namespace anyseq {

// Direction-word layout of one pair: lpc lanes of R rows per chunk, S steps
// per chunk, wpl = ceil(R / 8) words per lane and step.
struct TbLayout {
    int32_t pad, ch0, R, wpl, lpc;
    int64_t S;
};

__device__ __forceinline__ TbLayout tb_layout(const TbWalkArgs &W, int64_t p, int32_t m) {
    TbLayout L;
    L.pad = W.lay_pad[p];
    L.ch0 = W.lay_ch0[p];
    L.R = W.lay_r ? W.lay_r[p] : W.rows_per_lane;
    L.wpl = (L.R + 7) / 8;
    L.lpc = W.lanes_per_chunk;
    L.S = (int64_t)m + L.lpc - 1;
    return L;
}

// Position of a DP row in the layout: chunk, lane, row of the lane. The walks
// move up one row at a time, so after one division the position follows by
// decrements (tb_up).
struct TbCursor {
    int32_t ch, gl, rr;
};

__device__ __forceinline__ TbCursor tb_cursor(const TbLayout &L, int32_t ii) {
    const int32_t ip = ii + L.pad - 1, chr = L.lpc * L.R;
    const int32_t within = ip % chr;
    return TbCursor{ip / chr, within / L.R, within % L.R};
}

__device__ __forceinline__ void tb_up(const TbLayout &L, TbCursor &c) {
    if (--c.rr < 0) {
        c.rr = L.R - 1;
        if (--c.gl < 0) {
            c.gl = L.lpc - 1;
            c.ch--;
        }
    }
}

// The word unit (chunk, lane, word of the lane) of a position, numbered in
// increasing row order; the row's bit in the word is rr & 7.
__device__ __forceinline__ int32_t tb_unit(const TbLayout &L, const TbCursor &c) {
    return (c.ch * L.lpc + c.gl) * L.wpl + (c.rr >> 3);
}

// Index of the word of a position at column jj (step jj - 1 + lane).
__device__ __forceinline__ int64_t tb_word_index(const TbLayout &L, int32_t ch, int32_t gl, int32_t sub, int32_t jj) {
    return (((int64_t)(ch - L.ch0) * L.S + (jj - 1) + gl) * L.lpc + gl) * L.wpl + sub;
}

__global__ void tb_plan_kernel(const int32_t *list, const int64_t *n_list_p, int per_item, const int64_t *q_off,
                               const int64_t *s_off, int64_t *words, int32_t *lay_pad, int32_t *lay_ch0,
                               int32_t *lay_r, int rmax, int fixed_r) {
    const int64_t n_list = *n_list_p;
    const int64_t n_items = (n_list + per_item - 1) / per_item;
    for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < n_items;
         item += (int64_t)gridDim.x * blockDim.x) {
        // the DP kernel's own plan of the item
        ItemPlan P = plan_item(list, n_list, item, per_item, q_off, s_off, rmax);
        if (fixed_r) P.R = fixed_r;
        const int32_t CH = GROUP * P.R;
        for (int k = 0; k < per_item; k++) {
            int32_t p = P.pid[k];
            if (p < 0) continue;
            int32_t pad = P.nch * CH - P.n[k];
            int32_t ch0 = pad / CH;
            words[p] = (int64_t)(P.nch - ch0) * (P.m[k] + GROUP - 1) * GROUP * ((P.R + 7) / 8);
            lay_pad[p] = pad;
            lay_ch0[p] = ch0;
            lay_r[p] = P.R;
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

// One warp per pair: the walk from the optimum cell is sequential and every
// step moves up or left, so the warp stages a window of direction words ahead of
// the walker into shared memory (rows i-63..i, columns j-63..j: each lane loads
// the words of two columns, all issued before the first is stored, so a window
// costs one global latency) and lane 0 walks inside it; leaving the window
// triggers the next load. This turns one dependent global load per step into
// one per window. (A 1,000 x 1,100 pair: 32 x 32 windows filled one word at a
// time took 313 us.)
constexpr int TBW = 64;                  // window height and width (cells)
constexpr int TBG = TBW / 2 + 1;         // word units a window can touch (lanes of 2 rows at least)
constexpr int TB_WARPS = 4;              // warps per block of the walk

// Stage one window: each lane loads units 0..nu-1 (from the window's top row up)
// of its two columns j - lane and j - lane - 32, all loads before any store.
template <int MU>
__device__ __forceinline__ void stage_window(const TbLayout &L, const uint32_t *dw, const TbCursor &c0, int32_t nu,
                                             int32_t j, int32_t j_lo, int lane, uint32_t (*wn)[TBW]) {
#pragma unroll
    for (int half = 0; half < TBW / 32; half++) {
        const int32_t col = lane + 32 * half, jj = j - col;
        uint32_t v[MU];
        int32_t ch = c0.ch, gl = c0.gl, sub = c0.rr >> 3;  // the window's first unit, then upwards
#pragma unroll
        for (int u = 0; u < MU; u++) {
            v[u] = (u < nu && jj >= j_lo) ? dw[tb_word_index(L, ch, gl, sub, jj)] : 0u;
            if (++sub == L.wpl) {
                sub = 0;
                if (++gl == L.lpc) {
                    gl = 0;
                    ch++;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < MU; u++)
            if (u < nu) wn[u][col] = v[u];
    }
}

__global__ void __launch_bounds__(TB_WARPS * 32) tb_walk_kernel(TbWalkArgs W) {
    __shared__ uint32_t win[TB_WARPS][TBG][TBW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t(*wn)[TBW] = win[wid];
    const int64_t nw = (int64_t)gridDim.x * TB_WARPS;
    for (int64_t p = (int64_t)blockIdx.x * TB_WARPS + wid; p < W.n_pairs; p += nw) {
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
            const TbLayout L = tb_layout(W, p, m);
            int state = 0;  // 0: H, 1: E, 2: F
            bool done = false;
            // every step moves up or left within two iterations; the bound and the
            // boundary checks keep a corrupt word from leaving the pair's words
            int64_t guard = 2 * ((int64_t)n + m) + 4;
            while (!done) {
                // stage the window below-right of (i, j): rows i_lo..i, columns j_lo..j
                const int32_t i_lo = max(1, i - TBW + 1), j_lo = max(1, j - TBW + 1);
                const int32_t rg_lo = tb_unit(L, tb_cursor(L, i_lo));  // word unit of the window's top row
                if (i >= 1 && j >= 1) {
                    const int32_t nu = tb_unit(L, tb_cursor(L, i)) - rg_lo + 1;  // units of the window (<= TBG)
                    const TbCursor c0 = tb_cursor(L, i_lo);
                    // lanes of 8 rows or more (most batched items, the wavefront's 8- and
                    // 16-row layouts) touch at most TBW / 8 + 1 units, lanes of 4 rows
                    // TBW / 4 + 1: shorter unrolled copies for them
                    if (nu <= TBW / 8 + 1) stage_window<TBW / 8 + 1>(L, dw, c0, nu, j, j_lo, lane, wn);
                    else if (nu <= TBW / 4 + 1) stage_window<TBW / 4 + 1>(L, dw, c0, nu, j, j_lo, lane, wn);
                    else stage_window<TBG>(L, dw, c0, nu, j, j_lo, lane, wn);
                }
                __syncwarp();
                if (lane == 0) {
                    // row i's word unit (as a window row), its bit, and the window column of j,
                    // all followed by increments: a move up leaves the unit only from a word's
                    // first row, and units are numbered in row order
                    TbCursor cur = tb_cursor(L, i);
                    int32_t urow = tb_unit(L, cur) - rg_lo, r = cur.rr & 7, col = 0;
                    auto up = [&]() {
                        if (r == 0) {
                            tb_up(L, cur);
                            urow--;
                            r = cur.rr & 7;
                        } else {
                            cur.rr--;
                            r--;
                        }
                        i--;
                    };
                    // the matrix's first row or column ends the walk; a window starts at
                    // rows and columns from 1, so inside one only its edges need a test
                    if (state != 0 && (i <= 0 || j <= 0)) {
                        done = true;
                    } else if (state == 0) {
                        if (i == 0 && j == 0) {
                            done = true;
                        } else if (W.mode != GLOBAL) {
                            if (i == 0 || j == 0) done = true;
                        } else if (j == 0) {
                            rl.push(1u, (uint32_t)i);
                            i = 0;
                            done = true;
                        } else if (i == 0) {
                            rl.push(2u, (uint32_t)j);
                            j = 0;
                            done = true;
                        }
                    }
                    for (; !done && guard > 0; guard--) {
                        if (i < i_lo || j < j_lo) break;  // next window (or the first row or column)
                        // (i, j)'s bits at positions 0 (s0), 8 (s1), 16 (E opened), 24 (F opened)
                        const uint32_t w = wn[urow][col] >> r;
                        if (state == 0) {
                            if (W.mode == LOCAL && (w & 0x101u) == 0x101u) { done = true; break; }  // H = 0: the start
                            if (w & 1u) {
                                rl.push(0u, 1u);
                                up();
                                j--;
                                col++;
                                continue;
                            }
                            // H from E or F: take that gap's step from the same cell now
                            state = (w & 0x100u) ? 1 : 2;
                        }
                        if (state == 1) {
                            rl.push(1u, 1u);
                            if ((w >> 16) & 1u) state = 0;
                            up();
                        } else {
                            rl.push(2u, 1u);
                            if ((w >> 24) & 1u) state = 0;
                            j--;
                            col++;
                        }
                    }
                    if (!done && guard <= 0) done = true;
                }
                __syncwarp();
                i = __shfl_sync(0xffffffffu, i, 0);
                j = __shfl_sync(0xffffffffu, j, 0);
                state = __shfl_sync(0xffffffffu, state, 0);
                done = __shfl_sync(0xffffffffu, (int)done, 0) != 0;
                guard = __shfl_sync(0xffffffffu, guard, 0);
            }
        }
        if (lane == 0) {
            rl.flush();
            W.cig_len[p] = rl.k;
            W.beg_q[p] = i;
            W.beg_s[p] = j;
        }
    }
}

// One thread per pair: the same walk, reading each direction word from global
// memory (the last word stays in a register, so vertical steps inside a lane's
// 8 rows reuse it). A walk is a chain of dependent loads; with one walker per
// thread a whole batch keeps tens of thousands of them in flight, where the
// warp walk keeps one per warp. Used for large batches (launch_tb_walk).
__global__ void __launch_bounds__(256) tb_walk_thread_kernel(TbWalkArgs W) {
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
            const TbLayout L = tb_layout(W, p, m);
            int64_t cached = -1;
            uint32_t w = 0;
            TbCursor cur = tb_cursor(L, i > 0 ? i : 1);  // row i; follows i downwards
            // the word of cell (i, jj) and its row bit r
            auto word = [&](int32_t jj, int32_t &r) -> uint32_t {
                r = cur.rr & 7;
                const int64_t idx = tb_word_index(L, cur.ch, cur.gl, cur.rr >> 3, jj);
                if (idx != cached) {
                    cached = idx;
                    w = dw[idx];
                }
                return w;
            };
            int state = 0;  // 0: H, 1: E, 2: F
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
                    const uint32_t x = word(j, r);
                    const uint32_t s0 = (x >> r) & 1u, s1 = (x >> (8 + r)) & 1u;
                    if (W.mode == LOCAL && s0 && s1) break;  // H = 0: the alignment starts here
                    if (s0) { rl.push(0u, 1u); i--; j--; tb_up(L, cur); }
                    else state = s1 ? 1 : 2;
                } else {
                    int32_t r;
                    const uint32_t x = word(j, r);
                    if (state == 1) {
                        rl.push(1u, 1u);
                        if ((x >> (16 + r)) & 1u) state = 0;
                        i--;
                        tb_up(L, cur);
                    } else {
                        rl.push(2u, 1u);
                        if ((x >> (24 + r)) & 1u) state = 0;
                        j--;
                    }
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
                           int32_t *lay_ch0, int32_t *lay_r, int rmax, int fixed_r, cudaStream_t st) {
    tb_plan_kernel<<<grid_of(max_items), 256, 0, st>>>(list, n_list, per_item, q_off, s_off, words, lay_pad, lay_ch0,
                                                        lay_r, rmax, fixed_r);
    return cudaGetLastError();
}

// Pairs from which a batch walks one thread per pair. Below it, the warp walk's
// staged windows keep a single long walk short; above it, there are enough
// walks to keep memory busy with one dependent load each.
constexpr int64_t TB_THREAD_WALK_PAIRS = 4096;

cudaError_t launch_tb_walk(const TbWalkArgs &W, cudaStream_t st) {
    const bool per_thread = W.walker == 2 || (W.walker == 0 && W.n_pairs >= TB_THREAD_WALK_PAIRS);
    if (per_thread) {
        tb_walk_thread_kernel<<<grid_of(W.n_pairs), 256, 0, st>>>(W);
        return cudaGetLastError();
    }
    int64_t blocks = (W.n_pairs + TB_WARPS - 1) / TB_WARPS;
    blocks = blocks < 1 ? 1 : (blocks > 65535 ? 65535 : blocks);
    tb_walk_kernel<<<(int)blocks, TB_WARPS * 32, 0, st>>>(W);
    return cudaGetLastError();
}

cudaError_t launch_tb_compact(int64_t n_pairs, const int64_t *q_off, const int64_t *s_off, const uint32_t *tmp,
                              const int64_t *cig_len, const int64_t *cig_off, uint32_t *out, cudaStream_t st) {
    tb_compact_kernel<<<grid_of(n_pairs), 256, 0, st>>>(n_pairs, q_off, s_off, tmp, cig_len, cig_off, out);
    return cudaGetLastError();
}

}  // namespace anyseq
