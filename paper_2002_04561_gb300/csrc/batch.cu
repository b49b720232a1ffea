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
    const uint32_t e_raw = C::raw(e), oe_raw = C::raw(oe);   // per-half constants of DPX add-max
    const uint32_t oe_c = C::cst(oe);                        // packed constant of IADD
    const T NEGv = C::make(C::NEG, C::NEG);
    const int CH = GROUP * R;
    const int S = Mit + GROUP - 1;
    int32_t *scr = A.scratch ? A.scratch + gslot * 2 * (int64_t)A.scratch_cols : nullptr;

    // optimum candidates per half as keys (larger wins)
    uint64_t best[2];
#pragma unroll
    for (int h = 0; h < 2; h++) best[h] = end_key(0, 0, MODE == SEMIGLOBAL ? sl.m[h] : 0);
    int32_t gscore[2] = {0, 0};

    for (int ch = 0; ch < nch; ch++) {
        const bool last = (ch == nch - 1);
        const int32_t rb = ch * CH + g * R + 1;  // padded row of register 0
        uint32_t profA[R], profB[R];
        T Hoe[R], F[R];
        T rowmax[MODE == LOCAL ? R : 1];
        uint32_t rowj[MODE == LOCAL ? R : 1];   // first column of the row maximum (int16x2: one per half)
#pragma unroll
        for (int r = 0; r < R; r++) {
            int32_t h0[2] = {0, 0};
            uint32_t pw[2] = {A.rowprof[4], A.rowprof[4]};
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
                int32_t i = rb + r - sl.pad[h];
                if (i >= 1 && sl.n[h] > 0) pw[h] = A.rowprof[letter(A.q2, sl.q0[h], sl.n[h], i - 1, sl.rev[h])];
                h0[h] = col0(MODE, i, o, e, sl.tb[h]) + oe;
            }
            profA[r] = pw[0];
            profB[r] = pw[1];
            Hoe[r] = C::make(h0[0], h0[1]);
            F[r] = NEGv;
            if (MODE == LOCAL) {
                rowmax[r] = C::make(oe, oe);  // Hoe of H = 0
                rowj[r] = 0;
            }
        }
        T diag0;
        {
            int32_t d[2];
#pragma unroll
            for (int h = 0; h < 2; h++) d[h] = col0(MODE, rb - 1 - sl.pad[h], o, e, sl.tb[h]) + oe;
            diag0 = C::make(d[0], d[1]);
        }

        // --- ring fill (selectors, border of the previous chunk) and drain of
        //     the bottom ring (border of this chunk, or the query's last row)
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
        auto drain = [&](int blk) {
#pragma unroll
            for (int k = 0; k < 2; k++) {
                int c = blk * BLOCK + g + 16 * k;
                if (blk >= 0 && c < Mit) {
                    int32_t hv = sm->bot[2 * (c & (RING - 1))];
                    if (!last) {
                        scr[2 * c] = hv;
                        scr[2 * c + 1] = sm->bot[2 * (c & (RING - 1)) + 1];
                    } else if (MODE != LOCAL) {
                        // H(n, c+1) of each half: semi-global last-row candidate / global score
#pragma unroll
                        for (int h = 0; h < C::PAIRS; h++) {
                            int32_t H = C::get(C::from_u((uint32_t)hv), h) - oe;
                            if (MODE == SEMIGLOBAL && c < sl.m[h]) {
                                uint64_t key = end_key(H, sl.n[h], c + 1);
                                best[h] = key > best[h] ? key : best[h];
                            }
                            if (MODE == GLOBAL && c == sl.m[h] - 1) gscore[h] = H;
                        }
                    }
                }
            }
        };

        __syncwarp();
        fill(0);
        __syncwarp();
        int drained = 0;  // next bottom block to drain

        T last_hoe = NEGv, last_e = NEGv, prev_up = diag0;
        for (int s = 0; s < S; s++) {
            if ((s & (BLOCK - 1)) == 0) {
                __syncwarp();
                int k = s / BLOCK;
                fill(k + 1);
                if (k - 2 >= drained) { drain(k - 2); drained = k - 1; }
                __syncwarp();
            }
            const int c = s - g;
            // from lane g-1: Hoe of its last row and E of this lane's first row, column c
            T up_hoe = C::from_u(__shfl_up_sync(0xffffffffu, C::as_u(last_hoe), 1, GROUP));
            T up_e = C::from_u(__shfl_up_sync(0xffffffffu, C::as_u(last_e), 1, GROUP));
            if (g == 0) {
                if (ch == 0) {
                    // row 0: H(0, c+1); E below row 0 comes from H only (E(0, .) = -inf)
                    int32_t v = (MODE == GLOBAL ? o + (c + 1) * e : 0) + oe;
                    up_hoe = C::make(v, v);
                    up_e = up_hoe;
                } else if (c >= 0 && c < Mit) {
                    up_hoe = C::from_u((uint32_t)sm->top[2 * (c & (RING - 1))]);
                    up_e = C::from_u((uint32_t)sm->top[2 * (c & (RING - 1)) + 1]);
                }
            }
            if (c >= 0 && c < Mit) {
                const uint32_t sel = sm->sel[c & (RING - 1)];
                T diag = (c == 0) ? diag0 : prev_up;
                prev_up = up_hoe;
                T E = up_e;
                uint32_t valid = 0, jj = 0;
                if (MODE == LOCAL) {
                    valid = C::PAIRS == 2 ? ((c < sl.m[0] ? 0xFFFFu : 0u) | (c < sl.m[1] ? 0xFFFF0000u : 0u))
                                          : (c < sl.m[0] ? 0xFFFFFFFFu : 0u);
                    jj = C::PAIRS == 2 ? (uint32_t)(c + 1) * 65537u : (uint32_t)(c + 1);
                }
#pragma unroll
                for (int r = 0; r < R; r++) {
                    // H(i,j) = max(H(i-1,j-1)+sigma, E(i,j), F(i,j) [,0]) kept as Hoe = H + o + e
                    T sg = C::sigma(profA[r], profB[r], sel);
                    T Ad = C::addc(diag, C::as_u(sg));                 // H(i-1,j-1) + sigma
                    F[r] = C::addmax(F[r], e_raw, Hoe[r]);             // Eq. 5
                    T M = (MODE == LOCAL) ? C::maxrelu(Ad, F[r]) : C::vmax(Ad, F[r]);
                    T X = C::addc(M, oe_c);                           // max(diag, F) + o + e
                    diag = Hoe[r];
                    Hoe[r] = C::addmax(E, oe_raw, X);                  // H + o + e
                    E = C::addmax(E, e_raw, X);                        // Eq. 4 for row i+1
                    if (MODE == LOCAL) {
                        // strict improvement of the row maximum at a valid column
                        uint32_t gm;
                        if (C::PAIRS == 2) {
                            // invalid columns read -16000 (biased 16768): within 2^15 of every row maximum
                            uint32_t Hm = (C::as_u(Hoe[r]) & valid) | (0x41804180u & ~valid);
                            // per half: Hm - rowmax - 1 + 2^15 keeps bit 15 iff Hm > rowmax
                            uint32_t d = Hm + 0x7FFF7FFFu - C::as_u(rowmax[r]);
                            gm = prmt(d, 0u, 0xBB99u);                        // sign of bytes 1, 3 -> halves
                            rowmax[r] = C::vmax(rowmax[r], C::from_u(Hm));
                        } else {
                            int32_t Hm = valid ? (int32_t)C::as_u(Hoe[r]) : (int32_t)C::NEG;
                            gm = Hm > (int32_t)C::as_u(rowmax[r]) ? 0xFFFFFFFFu : 0u;
                            rowmax[r] = C::vmax(rowmax[r], C::from_u((uint32_t)Hm));
                        }
                        rowj[r] = (jj & gm) | (rowj[r] & ~gm);
                    }
                }
                last_hoe = Hoe[R - 1];
                last_e = E;
                if (g == GROUP - 1) {
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
                                    uint64_t k = end_key(C::get(Hoe[r], h) - oe, i, sl.m[h]);
                                    best[h] = k > best[h] ? k : best[h];
                                }
                            }
                        }
                    }
                }
            }
        }
        __syncwarp();
        for (int b = drained; b <= (Mit - 1) / BLOCK; b++) drain(b);
        __syncwarp();
        if (MODE == LOCAL) {
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
#pragma unroll
                for (int r = 0; r < R; r++) {
                    int32_t i = rb + r - sl.pad[h];
                    if (i >= 1) {
                        int32_t v = C::get(rowmax[r], h) - oe;
                        int32_t j = C::PAIRS == 2 ? (int32_t)((rowj[r] >> (16 * h)) & 0xFFFFu) : (int32_t)rowj[r];
                        if (v > 0) {
                            uint64_t k = end_key(v, i, j);
                            best[h] = k > best[h] ? k : best[h];
                        }
                    }
                }
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
        int32_t gs = gscore[h];
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) gs |= __shfl_xor_sync(0xffffffffu, gs, off, GROUP);
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
        // rows per lane: at most 16 (12 for local int16x2, which also keeps per-row maxima)
        constexpr int RMAX = (MODE == LOCAL && C::PAIRS == 2) ? 12 : 16;
        int nch = (nmax + GROUP * RMAX - 1) / (GROUP * RMAX);
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
            case 14: run_slot<C, MODE, (RMAX < 14 ? RMAX : 14)>(A, sm, sl, nch, Mit, g, gslot, res); break;
            default: run_slot<C, MODE, RMAX>(A, sm, sl, nch, Mit, g, gslot, res); break;
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
