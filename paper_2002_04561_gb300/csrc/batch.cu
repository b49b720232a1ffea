// Batched inter-sequence DP kernel (Sec. VI: inter-sequence parallelism):
// score and optimum cell of many independent pairs, one slot per 16-lane
// group, persistent warps pulling work items from a length-sorted queue.
#include "engine.cuh"
#include "batch.h"

namespace anyseq {

__device__ __forceinline__ uint32_t letter(const uint32_t *packed, int64_t base, int32_t len, int32_t idx, bool rev) {
    // idx is 0-based inside the sequence
    return code2(packed, base + (rev ? (int64_t)(len - 1 - idx) : (int64_t)idx));
}

template <class C, int MODE, int R>
__device__ __noinline__ void run_slot(const BatchArgs &A, GroupSmem *sm, const Slot &sl,
                                      int nch, int Mit, int g, int64_t gslot, int32_t *res) {
    typedef typename C::T T;
    const int32_t o = A.o, e = A.e, oe = A.o + A.e;
    const T e2 = C::make(e, e), oe2 = C::make(oe, oe);
    const T NEGv = C::make(C::NEG, C::NEG);
    const int CH = GROUP * R;
    const int S = Mit + GROUP - 1;
    int32_t *scr = A.scratch ? A.scratch + gslot * 2 * (int64_t)A.scratch_cols : nullptr;

    // optimum candidates per half, as keys (larger wins)
    uint64_t best[2];
#pragma unroll
    for (int h = 0; h < 2; h++) best[h] = end_key(0, 0, MODE == SEMIGLOBAL ? sl.m[h] : 0);
    int32_t gscore[2] = {0, 0};

    for (int ch = 0; ch < nch; ch++) {
        const bool last = (ch == nch - 1);
        const int32_t rb = ch * CH + g * R + 1;  // padded row of register 0
        uint32_t profA[R], profB[R];
        T Hoe[R], F[R];
        T rowmax[R];
        uint32_t rowj[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            int32_t h0[2];
            uint32_t pw[2];
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
                int32_t i = rb + r - sl.pad[h];
                pw[h] = A.rowprof[4];
                if (i >= 1 && sl.n[h] > 0) pw[h] = A.rowprof[letter(A.q2, sl.q0[h], sl.n[h], i - 1, sl.rev[h])];
                h0[h] = col0(MODE, i, o, e, sl.tb[h]) + oe;
            }
            profA[r] = pw[0];
            profB[r] = C::PAIRS == 2 ? pw[1] : pw[0];
            Hoe[r] = C::make(h0[0], C::PAIRS == 2 ? h0[1] : h0[0]);
            F[r] = NEGv;
            rowmax[r] = C::make(0, 0);
            rowj[r] = 0;
        }
        T diag0;
        {
            int32_t d[2];
#pragma unroll
            for (int h = 0; h < 2; h++) d[h] = col0(MODE, rb - 1 - sl.pad[h], o, e, sl.tb[h]) + oe;
            diag0 = C::make(d[0], d[1]);
        }
        // semi-global last-row tracking (lane 15, last chunk)
        T lr_best = C::make(0, 0);
        uint32_t lr_j = 0;

        // --- ring fill / flush helpers (warp-cooperative, 16 lanes per group)
        auto fill = [&](int blk) {
#pragma unroll
            for (int k = 0; k < 2; k++) {
                int c = blk * BLOCK + g + 16 * k;
                if (c < Mit) {
                    uint32_t ca = 0, cb = 0;
                    if (c < sl.m[0]) ca = letter(A.s2, sl.s0[0], sl.m[0], c, sl.rev[0]);
                    if (C::PAIRS == 2 && c < sl.m[1]) cb = letter(A.s2, sl.s0[1], sl.m[1], c, sl.rev[1]);
                    sm->sel[c & (RING - 1)] = C::selector(ca, cb);
                    if (ch > 0) {
                        sm->top[2 * (c & (RING - 1))] = scr[2 * c];
                        sm->top[2 * (c & (RING - 1)) + 1] = scr[2 * c + 1];
                    }
                }
            }
        };
        auto flush = [&](int blk) {
#pragma unroll
            for (int k = 0; k < 2; k++) {
                int c = blk * BLOCK + g + 16 * k;
                if (blk >= 0 && c < Mit) {
                    scr[2 * c] = sm->bot[2 * (c & (RING - 1))];
                    scr[2 * c + 1] = sm->bot[2 * (c & (RING - 1)) + 1];
                }
            }
        };

        __syncwarp();
        fill(0);
        __syncwarp();
        int flushed = 0;  // next bottom block to flush

        T last_hoe = NEGv, last_e = NEGv, prev_up = diag0;
        for (int s = 0; s < S; s++) {
            if ((s & (BLOCK - 1)) == 0) {
                __syncwarp();
                int k = s / BLOCK;
                fill(k + 1);
                if (!last && k - 2 >= flushed) { flush(k - 2); flushed = k - 1; }
                __syncwarp();
            }
            const int c = s - g;
            T up_hoe = C::from_u(__shfl_up_sync(0xffffffffu, C::as_u(last_hoe), 1, GROUP));
            T up_e = C::from_u(__shfl_up_sync(0xffffffffu, C::as_u(last_e), 1, GROUP));
            if (g == 0) {
                if (ch == 0) {
                    int32_t v = (MODE == GLOBAL ? o + (c + 1) * e : 0) + oe;
                    up_hoe = C::make(v, v);
                    up_e = NEGv;
                } else if (c >= 0 && c < Mit) {
                    up_hoe = C::from_u((uint32_t)sm->top[2 * (c & (RING - 1))]);
                    up_e = C::from_u((uint32_t)sm->top[2 * (c & (RING - 1)) + 1]);
                }
            }
            if (c >= 0 && c < Mit) {
                const uint32_t sel = sm->sel[c & (RING - 1)];
                T diag = (c == 0) ? diag0 : prev_up;
                prev_up = up_hoe;
                T hu = up_hoe, eu = up_e;
                uint32_t valid = 0, jj = 0;
                if (MODE == LOCAL) {
                    valid = C::PAIRS == 2 ? ((c < sl.m[0] ? 0xFFFFu : 0u) | (c < sl.m[1] ? 0xFFFF0000u : 0u))
                                          : (c < sl.m[0] ? 0xFFFFFFFFu : 0u);
                    jj = C::PAIRS == 2 ? ((uint32_t)(c + 1) | ((uint32_t)(c + 1) << 16)) : (uint32_t)(c + 1);
                }
#pragma unroll
                for (int r = 0; r < R; r++) {
                    T sg = C::sigma(profA[r], profB[r], sel);
                    T En = C::addmax(eu, e2, hu);
                    T Fn = C::addmax(F[r], e2, Hoe[r]);
                    T Hd = C::add(diag, sg);
                    T H = (MODE == LOCAL) ? C::max3relu(Hd, En, Fn) : C::max3(Hd, En, Fn);
                    diag = Hoe[r];
                    T Hn = C::add(H, oe2);
                    Hoe[r] = Hn;
                    F[r] = Fn;
                    hu = Hn;
                    eu = En;
                    if (MODE == LOCAL) {
                        T Hm = C::from_u(C::as_u(H) & valid);
                        uint32_t gm = C::gt(Hm, rowmax[r]);
                        rowmax[r] = C::vmax(rowmax[r], Hm);
                        rowj[r] = (jj & gm) | (rowj[r] & ~gm);
                    }
                }
                last_hoe = hu;
                last_e = eu;
                // last row of the query: lane 15, last register, last chunk
                if (MODE != LOCAL && last && g == GROUP - 1) {
                    T H = C::add(hu, C::make(-oe, -oe));
                    if (MODE == SEMIGLOBAL) {
                        uint32_t v = C::PAIRS == 2 ? ((c < sl.m[0] ? 0xFFFFu : 0u) | (c < sl.m[1] ? 0xFFFF0000u : 0u))
                                                   : (c < sl.m[0] ? 0xFFFFFFFFu : 0u);
                        uint32_t gm = C::gt(H, lr_best) & v;
                        lr_best = C::from_u((C::as_u(H) & gm) | (C::as_u(lr_best) & ~gm));
                        uint32_t j2 = C::PAIRS == 2 ? ((uint32_t)(c + 1) | ((uint32_t)(c + 1) << 16)) : (uint32_t)(c + 1);
                        lr_j = (j2 & gm) | (lr_j & ~gm);
                    } else {
                        if (c == sl.m[0] - 1) gscore[0] = C::get(H, 0);
                        if (C::PAIRS == 2 && c == sl.m[1] - 1) gscore[1] = C::get(H, 1);
                    }
                }
                if (!last && g == GROUP - 1) {
                    sm->bot[2 * (c & (RING - 1))] = (int32_t)C::as_u(last_hoe);
                    sm->bot[2 * (c & (RING - 1)) + 1] = (int32_t)C::as_u(last_e);
                }
                // semi-global: last column candidates at c == m-1
                if (MODE == SEMIGLOBAL) {
#pragma unroll
                    for (int h = 0; h < C::PAIRS; h++) {
                        if (c == sl.m[h] - 1) {
#pragma unroll
                            for (int r = 0; r < R; r++) {
                                int32_t i = rb + r - sl.pad[h];
                                if (i >= 1) {
                                    int32_t hv = C::get(Hoe[r], h) - oe;
                                    uint64_t k = end_key(hv, i, sl.m[h]);
                                    best[h] = k > best[h] ? k : best[h];
                                }
                            }
                        }
                    }
                }
            }
        }
        if (!last) {
            __syncwarp();
            int kend = (Mit - 1) / BLOCK;
            for (int b = flushed; b <= kend; b++) flush(b);
            __syncwarp();
        }
        if (MODE == LOCAL) {
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
#pragma unroll
                for (int r = 0; r < R; r++) {
                    int32_t i = rb + r - sl.pad[h];
                    if (i >= 1) {
                        int32_t v = C::get(rowmax[r], h);
                        int32_t j = C::PAIRS == 2 ? (int32_t)((rowj[r] >> (16 * h)) & 0xFFFFu) : (int32_t)rowj[r];
                        if (v > 0) {
                            uint64_t k = end_key(v, i, j);
                            best[h] = k > best[h] ? k : best[h];
                        }
                    }
                }
            }
        }
        if (MODE == SEMIGLOBAL && last && g == GROUP - 1) {
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
                int32_t v = C::get(lr_best, h);
                int32_t j = C::PAIRS == 2 ? (int32_t)((lr_j >> (16 * h)) & 0xFFFFu) : (int32_t)lr_j;
                uint64_t k = end_key(v, sl.n[h], j);
                best[h] = k > best[h] ? k : best[h];
            }
        }
    }
    // reduce across the 16 lanes of the group
#pragma unroll
    for (int h = 0; h < 2; h++) {
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) {
            uint64_t other = __shfl_xor_sync(0xffffffffu, best[h], off, GROUP);
            best[h] = other > best[h] ? other : best[h];
        }
        int32_t gs = __shfl_sync(0xffffffffu, gscore[h], GROUP - 1, GROUP);
        if (MODE == GLOBAL) {
            res[3 * h] = gs;
            res[3 * h + 1] = sl.n[h];
            res[3 * h + 2] = sl.m[h];
        } else {
            res[3 * h] = key_score(best[h]);
            res[3 * h + 1] = key_i(best[h]);
            res[3 * h + 2] = key_j(best[h]);
        }
    }
}

template <class C, int MODE>
__global__ void __launch_bounds__(256, 2) batch_kernel(BatchArgs A) {
    __shared__ GroupSmem smem[16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane >> 4, g = lane & 15;
    GroupSmem *sm = &smem[warp * 2 + grp];
    const int64_t gslot = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 2 + grp;
    const int per_item = 2 * C::PAIRS;
    const int32_t n_items = (int32_t)((*A.n_list + per_item - 1) / per_item);
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(A.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        // pairs of the item: per_item consecutive entries of the sorted list
        int32_t nmax = 0, Mit = 0;
        int32_t pid[2] = {-1, -1};
        Slot sl;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            sl.n[h] = 0; sl.m[h] = 0; sl.q0[h] = 0; sl.s0[h] = 0; sl.rev[h] = false;
            sl.tb[h] = A.o;
        }
        for (int k = 0; k < per_item; k++) {
            int64_t idx = (int64_t)item * per_item + k;
            if (idx < *A.n_list) {
                int32_t p = A.list[idx];
                int32_t n = (int32_t)(A.q_off[p + 1] - A.q_off[p]);
                int32_t m = (int32_t)(A.s_off[p + 1] - A.s_off[p]);
                nmax = max(nmax, n);
                Mit = max(Mit, m);
                if (k / C::PAIRS == grp) {
                    int h = k % C::PAIRS;
                    pid[h] = p;
                    sl.n[h] = n; sl.m[h] = m;
                    sl.q0[h] = A.q_off[p]; sl.s0[h] = A.s_off[p];
                }
            }
        }
        int nch = (nmax + 255) / 256;
        int R = (nmax + GROUP * nch - 1) / (GROUP * nch);
        R += R & 1;
        if (R < 2) R = 2;
        const int rows = nch * GROUP * R;
#pragma unroll
        for (int h = 0; h < 2; h++) sl.pad[h] = rows - sl.n[h];
        int32_t res[6];
        switch (R) {
            case 2: run_slot<C, MODE, 2>(A, sm, sl, nch, Mit, g, gslot, res); break;
            case 4: run_slot<C, MODE, 4>(A, sm, sl, nch, Mit, g, gslot, res); break;
            case 6: run_slot<C, MODE, 6>(A, sm, sl, nch, Mit, g, gslot, res); break;
            case 8: run_slot<C, MODE, 8>(A, sm, sl, nch, Mit, g, gslot, res); break;
            case 10: run_slot<C, MODE, 10>(A, sm, sl, nch, Mit, g, gslot, res); break;
            case 12: run_slot<C, MODE, 12>(A, sm, sl, nch, Mit, g, gslot, res); break;
            case 14: run_slot<C, MODE, 14>(A, sm, sl, nch, Mit, g, gslot, res); break;
            default: run_slot<C, MODE, 16>(A, sm, sl, nch, Mit, g, gslot, res); break;
        }
        if (g == 0) {
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
                if (pid[h] >= 0) {
                    A.score[pid[h]] = res[3 * h];
                    A.end_q[pid[h]] = res[3 * h + 1];
                    A.end_s[pid[h]] = res[3 * h + 2];
                    A.flags[pid[h]] = C::PAIRS == 1 ? 1u : 0u;
                }
            }
        }
    }
}

template <class C, int MODE>
static cudaError_t launch_one(const BatchArgs &A, int grid, cudaStream_t st) {
    batch_kernel<C, MODE><<<grid, 256, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs &A, int cell32, int mode, int grid, cudaStream_t st) {
    if (cell32) {
        switch (mode) {
            case GLOBAL: return launch_one<CellI32, GLOBAL>(A, grid, st);
            case LOCAL: return launch_one<CellI32, LOCAL>(A, grid, st);
            default: return launch_one<CellI32, SEMIGLOBAL>(A, grid, st);
        }
    }
    switch (mode) {
        case GLOBAL: return launch_one<CellI16x2, GLOBAL>(A, grid, st);
        case LOCAL: return launch_one<CellI16x2, LOCAL>(A, grid, st);
        default: return launch_one<CellI16x2, SEMIGLOBAL>(A, grid, st);
    }
}

int batch_blocks_per_sm(int cell32, int mode) {
    int nb = 0;
    cudaError_t err;
    if (cell32) {
        err = mode == GLOBAL ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<CellI32, GLOBAL>, 256, 0)
            : mode == LOCAL  ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<CellI32, LOCAL>, 256, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<CellI32, SEMIGLOBAL>, 256, 0);
    } else {
        err = mode == GLOBAL ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<CellI16x2, GLOBAL>, 256, 0)
            : mode == LOCAL  ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<CellI16x2, LOCAL>, 256, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<CellI16x2, SEMIGLOBAL>, 256, 0);
    }
    if (err != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

}  // namespace anyseq
