// Batched inter-sequence DP kernel (Sec. VI: inter-sequence parallelism):
// score and optimum cell of many independent pairs, one slot per 16-lane
// group, persistent warps pulling work items from a length-sorted queue.
// The templates are instantiated per alignment mode and lane type in
// batch_{global,local,semiglobal}_{i16,i32}.cu (six translation units that
// compile in parallel); batch.cu dispatches to them.
#pragma once
#include "engine.cuh"
#include "batch.h"

namespace anyseq {

// Byte offset of the last-column buffers inside the dynamic shared memory.
__host__ __device__ __forceinline__ size_t lc_offset(int sigp, int alphabet) {
    return sigp ? 1024 + (size_t)(128 / GROUP) * 2 * (alphabet + 1) * QP_ROWS : 0;
}

__device__ __forceinline__ uint32_t letter(const uint32_t *packed, int64_t base, int32_t len, int32_t idx, bool rev) {
    // idx is 0-based inside the sequence
    return code2(packed, base + (rev ? (int64_t)(len - 1 - idx) : (int64_t)idx));
}

// Query profile of one group for the matrix path: byte [h][a][8 * lane + r] =
// sigma'(q_row, a) for row r of the lane's R rows in the chunk (padding rows:
// sig_pad). Each lane has an 8-byte slot whatever R is, so its profile words load
// aligned. Built by the 16 lanes together. Letter a = alphabet is a null letter
// with sigma' = 0 (sigma = open + extend), read by the columns past the end of a
// pair.
template <class C, int R>
__device__ __forceinline__ void build_qprofile(const BatchArgs &A, const Slot &sl, int ch, int g, uint32_t *qp,
                                               const int8_t *tab) {
    const int alpha = A.alphabet;
    const int words_per_letter = QP_ROWS / 4;
    for (int task = g; task < 2 * words_per_letter; task += GROUP) {
        const int h = task / words_per_letter, w = task % words_per_letter;
        int32_t code[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int lane = (w * 4 + k) >> 3, r = (w * 4 + k) & 7;
            int32_t i = ch * GROUP * R + lane * R + r + 1 - sl.pad[h];
            // codes >= alphabet (an ANYSEQ_ERR_ALPHABET call) are clamped inside the table
            code[k] = (h < C::PAIRS && r < R && i >= 1 && sl.n[h] > 0)
                          ? min((int32_t)A.q8[sl.q0[h] + (sl.rev[h] ? sl.n[h] - i : i - 1)], alpha - 1) : -1;
        }
        for (int a = 0; a <= alpha; a++) {
            uint32_t word = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                int32_t v = a == alpha ? 0 : code[k] >= 0 ? (int32_t)tab[code[k] * alpha + a] : A.sig_pad;
                word |= ((uint32_t)v & 0xFFu) << (8 * k);
            }
            qp[(h * (alpha + 1) + a) * words_per_letter + w] = word;
        }
    }
}

// lc (semi-global only): the group's last-column buffer, 2 x GROUP x R words.
// At the step where lane g reaches column m_h - 1 of half h it stores its R
// row words there; the candidates H(i, m_h) are ranked after the chunk, so
// the step loop carries no per-row work for them.
// Local mode keeps, per row, the running maximum and the first column where it
// occurs (a DPX maximum whose predicates flag a strict improvement per half,
// and a select per half); the optimum is ranked after each chunk.
// Refill block (columns) of a variant: 32, or 16 for the matrix path, whose
// query profile leaves less shared memory for the rings (16-column blocks
// halve them, so four 4-warp CTAs fit on an SM instead of three).
__host__ __device__ constexpr int block_cols(int sigp) { return sigp ? 16 : 32; }

template <class C, int MODE, int R, bool TB, int SIGP>
__device__ __noinline__ void run_slot(const BatchArgs &A, GroupSmemT<4 * block_cols(SIGP), block_cols(SIGP)> *sm,
                                      const Slot &sl,
                                      int nch, int Mit, int g, int64_t gslot, int32_t *res, const int32_t *pid,
                                      uint32_t *qp, const int8_t *tab, uint32_t *lc) {
    typedef typename C::T T;
    constexpr int BLOCK = block_cols(SIGP), RING = 4 * BLOCK;
    const int32_t o = A.o, e = A.e, oe = A.o + A.e;
    const uint32_t e_raw = C::raw(e), oe_raw = C::raw(oe);   // per-half constants of DPX add-max
    const uint32_t oe_c = C::cst(oe), e_c = C::cst(e);       // packed constants of IADD
    const T zero = C::make(0, 0);                            // H = 0 in both halves
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
        T rowmax[MODE == LOCAL ? R : 1];   // the row maximum of H so far
        uint32_t rowj0[MODE == LOCAL ? R : 1], rowj1[MODE == LOCAL ? R : 1];  // its first column per half
#pragma unroll
        for (int r = 0; r < R; r++) {
            int32_t h0[2] = {0, 0};
            uint32_t pw[2] = {A.rowprof[4], A.rowprof[4]};
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
                int32_t i = rb + r - sl.pad[h];
                if (SIGP == 0 && i >= 1 && sl.n[h] > 0) pw[h] = A.rowprof[letter(A.q2, sl.q0[h], sl.n[h], i - 1, sl.rev[h])];
                h0[h] = col0(MODE, i, o, e, sl.tb[h]) + oe;
            }
            profA[r] = pw[0];
            profB[r] = pw[1];
            Hoe[r] = C::make(h0[0], h0[1]);
            F[r] = NEGv;
            if (MODE == LOCAL) {
                rowmax[r] = zero;
                rowj0[r] = rowj1[r] = 0;
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
            for (int k = 0; k < BLOCK / 16; k++) {
                int c = blk * BLOCK + g + 16 * k;
                if (c < Mit) {
                    // columns past the end of a pair read a zero sigma' (sigma = open + extend):
                    // their values stay below the pair's optimum (only the local kernel looks at them)
                    if (SIGP == 0) {
                        uint32_t ca = 0, cb = 0;
                        if (c < sl.m[0]) ca = letter(A.s2, sl.s0[0], sl.m[0], c, sl.rev[0]);
                        if (C::PAIRS == 2 && c < sl.m[1]) cb = letter(A.s2, sl.s0[1], sl.m[1], c, sl.rev[1]);
                        sm->sel[c & (RING - 1)] = C::null_past_end(C::selector(ca, cb), c < sl.m[0], c < sl.m[1]);
                    } else {
                        const uint32_t alpha = (uint32_t)A.alphabet;
                        uint32_t ca = alpha, cb = alpha;
                        // a code >= alphabet (the call then fails with ANYSEQ_ERR_ALPHABET)
                        // reads the null letter's row, inside the shared profile
                        if (c < sl.m[0]) ca = min((uint32_t)A.s8[sl.s0[0] + (sl.rev[0] ? sl.m[0] - 1 - c : c)], alpha);
                        if (C::PAIRS == 2 && c < sl.m[1]) cb = min((uint32_t)A.s8[sl.s0[1] + (sl.rev[1] ? sl.m[1] - 1 - c : c)], alpha);
                        // byte offsets of the two letters' profile rows for this lane
                        sm->sel[c & (RING - 1)] = (ca * QP_ROWS) | (((alpha + 1 + cb) * QP_ROWS) << 16);
                    }
                    int2 tv;
                    if (ch > 0) {
                        tv = make_int2(scr[2 * c], scr[2 * c + 1]);
                    } else {
                        // row 0: H(0, c+1); E below row 0 comes from H only (E(0, .) = -inf)
                        const int32_t v = (MODE == GLOBAL ? o + (c + 1) * e : 0) + oe;
                        tv.x = tv.y = (int32_t)C::as_u(C::make(v, v));
                    }
                    reinterpret_cast<int2 *>(sm->top)[c & (RING - 1)] = tv;
                }
            }
        };
        auto drain = [&](int blk) {
#pragma unroll
            for (int k = 0; k < BLOCK / 16; k++) {
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
        if (SIGP) build_qprofile<C, R>(A, sl, ch, g, qp, tab);
        fill(0);
        __syncwarp();
        int drained = 0;  // next bottom block to drain

        // traceback: this chunk's direction words of each half, WPL words per lane
        // and step (rows 8k..8k+7 of the lane in word k; row chunks before the
        // pair's first real row are not stored)
        constexpr int WPL = (R + 7) / 8;
        uint32_t *dptr[2] = {nullptr, nullptr};
        int32_t Sh[2] = {0, 0};
        if (TB) {
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
                int32_t ch0 = sl.pad[h] / CH;
                Sh[h] = sl.m[h] + GROUP - 1;
                if (pid[h] >= 0 && ch >= ch0)
                    dptr[h] = A.dirs + A.dir_base[pid[h]] + ((int64_t)(ch - ch0) * Sh[h] * GROUP + g) * WPL;
            }
        }
        // diag starts as H(i0-1, 0) and afterwards is the Hoe that came down at the
        // previous column (prev_up changes only at valid columns)
        T last_hoe = NEGv, last_e = NEGv, prev_up = diag0;
        const int ev0 = sl.m[0] - 1, ev1 = C::PAIRS == 2 ? sl.m[1] - 1 : -1;  // last-column steps (+g)
        for (int s0 = 0; s0 < S; s0 += BLOCK) {
          __syncwarp();
          {
            const int k = s0 / BLOCK;
            fill(k + 1);
            if (k - 2 >= drained) { drain(k - 2); drained = k - 1; }
          }
          __syncwarp();
          const int s1 = min(S, s0 + BLOCK);
          for (int s = s0; s < s1; s++) {
            const int c = s - g;
            // from lane g-1: Hoe of its last row and E of this lane's first row, column c;
            // lane 0 reads the row above the chunk from the top ring (any column: the
            // ring index is masked, and invalid columns are not used)
            T up_hoe = C::from_u(__shfl_up_sync(0xffffffffu, C::as_u(last_hoe), 1, GROUP));
            T up_e = C::from_u(__shfl_up_sync(0xffffffffu, C::as_u(last_e), 1, GROUP));
            if (g == 0) {
                const int2 tv = reinterpret_cast<const int2 *>(sm->top)[c & (RING - 1)];
                up_hoe = C::from_u((uint32_t)tv.x);
                up_e = C::from_u((uint32_t)tv.y);
            }
            if ((unsigned)c < (unsigned)Mit) {
                const uint32_t sel = sm->sel[c & (RING - 1)];
                uint2 qa = make_uint2(0, 0), qb = make_uint2(0, 0);
                if (SIGP) {
                    const uint8_t *qpb = reinterpret_cast<const uint8_t *>(qp) + g * 8;  // the lane's slot
                    qa = *reinterpret_cast<const uint2 *>(qpb + (sel & 0xFFFFu));
                    if (C::PAIRS == 2) qb = *reinterpret_cast<const uint2 *>(qpb + (sel >> 16));
                }
                // sigma' of row r at this column
                auto sigma_r = [&](int r) -> uint32_t {
                    if (SIGP == 0) return C::as_u(C::sigma(profA[r], profB[r], sel));
                    // byte r of this lane's profile row, per half (bytes are >= 0)
                    const uint32_t wa = (r & 4) ? qa.y : qa.x, wb = (r & 4) ? qb.y : qb.x;
                    const uint32_t b = (uint32_t)(r & 3);
                    return C::PAIRS == 2 ? prmt(wa, wb, b | ((b | 8u) << 4) | ((b + 4u) << 8) | (((b + 4u) | 8u) << 12))
                                         : prmt(wa, wa, b | ((b | 8u) << 4) | ((b | 8u) << 8) | ((b | 8u) << 12));
                };
                // H(i-1,j-1) + sigma of row 0; every later row takes the old Hoe of the row
                // above (its upper-left neighbour) before that register is overwritten, so
                // the row registers update in place
                T Ad = C::addc(prev_up, sigma_r(0));
                prev_up = up_hoe;
                T E = up_e;
                const uint32_t jj = (uint32_t)(c + 1);
                // direction bit planes (traceback): bit 8+r / 24+r of each accumulator
                uint32_t pl_s0 = 0, pl_s1 = 0, pl_eo = 0, pl_fo = 0;
                T hup = up_hoe;  // Hoe of the row above, this column
#pragma unroll
                for (int r = 0; r < R; r++) {
                    // H(i,j) = max(H(i-1,j-1)+sigma, E(i,j), F(i,j) [,0]) kept as Hoe = H + o + e
                    T Adn = Ad;
                    if (r + 1 < R) Adn = C::addc(Hoe[r], sigma_r(r + 1));  // old Hoe[r]: next row's diagonal
                    if (!TB) {
                        // one 3-input maximum for H; local mode keeps F >= 0 (exact for H:
                        // max(F, 0) follows the same recurrence), which makes H >= 0 without
                        // a separate clamp
                        if (MODE == LOCAL) F[r] = C::vmax3(C::addc(F[r], e_c), Hoe[r], zero);  // Eq. 5
                        else F[r] = C::addmax(F[r], e_raw, Hoe[r]);                            // Eq. 5
                        const T Hn = C::vmax3(Ad, F[r], E);                                    // Eq. 1
                        Hoe[r] = C::addc(Hn, oe_c);
                        E = C::addmax(E, e_raw, Hoe[r]);                                       // Eq. 4, row i+1
                        // strict improvement of the row maximum: the column of its first occurrence
                        if (MODE == LOCAL) C::track(rowmax[r], rowj0[r], rowj1[r], Hn, jj);
                    } else {
                        // the same cell, and the predecessor flags of the traceback: each
                        // is the sign bit (bit 15 / 31 per lane) of a biased difference
                        if (MODE == LOCAL) F[r] = C::vmax3(C::addc(F[r], e_c), Hoe[r], zero);  // Eq. 5
                        else F[r] = C::addmax(F[r], e_raw, Hoe[r]);                            // Eq. 5
                        const uint32_t fFo = C::ge(Hoe[r], F[r]);          // F(i,j) opened from H(i,j-1)
                        const T Ein = E;                                   // E(i,j)
                        const T Hn = C::vmax3(Ad, F[r], E);                // Eq. 1
                        Hoe[r] = C::addc(Hn, oe_c);
                        E = C::addmax(E, e_raw, Hoe[r]);                   // Eq. 4, row i+1
                        const uint32_t fD = C::ge(Ad, Hn);                 // diagonal reaches H
                        const uint32_t fE = C::ge(Ein, Hn);                // E reaches H
                        const uint32_t fEo = C::ge(hup, Ein);              // E(i,j) opened from H(i-1,j)
                        uint32_t s0 = fD, s1 = fE;
                        if (MODE == LOCAL) {
                            const uint32_t fZ = C::ge(zero, Hn);           // H == 0 (H >= 0 here)
                            s0 = fZ | fD;
                            s1 = fZ | (fE & ~fD);
                        }
                        const uint32_t FM = C::flag_mask();
                        pl_s0 = (pl_s0 >> 1) | (s0 & FM);
                        pl_s1 = (pl_s1 >> 1) | (s1 & FM);
                        pl_eo = (pl_eo >> 1) | (fEo & FM);
                        pl_fo = (pl_fo >> 1) | (fFo & FM);
                        hup = Hoe[r];
                        if (MODE == LOCAL) C::track(rowmax[r], rowj0[r], rowj1[r], Hn, jj);
                    }
                    Ad = Adn;
                }
                last_hoe = Hoe[R - 1];
                last_e = E;
                if (TB) {
                    // each plane holds R rows per half, the last row in the half's top bit:
                    // one shift brings rows 0..7 / 8..15 of the low half to bytes 0 / 1 and
                    // those of the high half (int16x2) to bytes 2 / 3; the bits between
                    // are zero. Word k of a half: bytes s0, s1, E opened, F opened of rows
                    // 8k..8k+7.
                    constexpr int SH = C::PAIRS == 2 ? 16 - R : 32 - R;
                    const uint32_t x0 = pl_s0 >> SH, x1 = pl_s1 >> SH, x2 = pl_eo >> SH, x3 = pl_fo >> SH;
#pragma unroll
                    for (int k = 0; k < WPL; k++) {
                        const uint32_t a = prmt(x0, x1, (uint32_t)(k | ((4 + k) << 4) | ((2 + k) << 8) | ((6 + k) << 12)));
                        const uint32_t b = prmt(x2, x3, (uint32_t)(k | ((4 + k) << 4) | ((2 + k) << 8) | ((6 + k) << 12)));
                        // a: s0/s1 bytes of the low half, then of the high half; b likewise
                        if (dptr[0] && s < Sh[0]) dptr[0][(int64_t)s * GROUP * WPL + k] = prmt(a, b, 0x5410u);
                        if (C::PAIRS == 2 && dptr[1] && s < Sh[1])
                            dptr[1][(int64_t)s * GROUP * WPL + k] = prmt(a, b, 0x7632u);
                    }
                }
                if (g == GROUP - 1)
                    reinterpret_cast<int2 *>(sm->bot)[c & (RING - 1)] =
                        make_int2((int32_t)C::as_u(last_hoe), (int32_t)C::as_u(last_e));
                // semi-global: this lane's rows of the last column of a half (once per chunk)
                if (MODE == SEMIGLOBAL && (c == ev0 || c == ev1)) {
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        if (c == ev0) lc[g * R + r] = C::as_u(Hoe[r]);
                        if (c == ev1) lc[(GROUP + g) * R + r] = C::as_u(Hoe[r]);
                    }
                }
            }
          }
        }
        __syncwarp();
        for (int b = drained; b <= (Mit - 1) / BLOCK; b++) drain(b);
        __syncwarp();
        if (MODE == SEMIGLOBAL) {
            // last-column candidates H(i, m_h) of this lane's rows
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
                if (sl.m[h] > 0) {
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int32_t i = rb + r - sl.pad[h];
                        if (i >= 1) {
                            const uint64_t k = end_key(C::get(C::from_u(lc[(h * GROUP + g) * R + r]), h) - oe, i, sl.m[h]);
                            best[h] = k > best[h] ? k : best[h];
                        }
                    }
                }
            }
        }
        if (MODE == LOCAL) {
            // every row's maximum, at the first column it occurs (columns past the end of a
            // half never win: their values do not exceed a real cell earlier in row-major order)
#pragma unroll
            for (int h = 0; h < C::PAIRS; h++) {
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int32_t i = rb + r - sl.pad[h], v = C::get(rowmax[r], h);
                    const int32_t j = (int32_t)(h == 0 ? rowj0[r] : rowj1[r]);
                    if (i >= 1 && v > 0) {
                        const uint64_t k = end_key(v, i, j);
                        best[h] = k > best[h] ? k : best[h];
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

}  // namespace anyseq

#include "batch_score.cuh"

namespace anyseq {

// Persistent kernel: each warp pulls work items (2 slots of 16 lanes) from the
// sorted list until it is empty. THREADS = batch_threads (batch.h); the matrix
// path's per-group query profile lives in dynamic shared memory after a copy
// of the sigma' table.
// The run_slot instantiation of a planned R: R itself, at most RMAX.
template <int RMAX>
__host__ __device__ constexpr int rsel(int r) { return r < RMAX ? r : RMAX; }

template <class C, int MODE, bool TB, int SIGP>
__global__ void __launch_bounds__(batch_threads(SIGP), batch_min_ctas(SIGP)) batch_kernel(BatchArgs A) {
    constexpr int THREADS = batch_threads(SIGP);
    __shared__ GroupSmemT<4 * block_cols(SIGP), block_cols(SIGP)> smem[THREADS / 16];
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane >> 4, g = lane & 15;
    GroupSmemT<4 * block_cols(SIGP), block_cols(SIGP)> *sm = &smem[warp * 2 + grp];
    int8_t *tab = nullptr;
    uint32_t *qp = nullptr;
    if (SIGP) {
        tab = reinterpret_cast<int8_t *>(dyn_smem);
        for (int k = threadIdx.x; k < A.alphabet * A.alphabet; k += THREADS) tab[k] = A.sig_tab[k];
        qp = reinterpret_cast<uint32_t *>(dyn_smem + 1024) + (warp * 2 + grp) * (2 * (A.alphabet + 1) * QP_ROWS / 4);
        __syncthreads();
    }
    const int64_t gslot = ((int64_t)blockIdx.x * (THREADS >> 5) + warp) * 2 + grp;
    // rows per lane: at most 16 (12 for local int16x2, which also keeps per-row
    // maxima and columns); at most TB_R for the matrix kernels, whose query
    // profile has an 8-byte slot per lane (exactly TB_R with traceback, the
    // direction-word layout of tb.cu)
    constexpr int RMAX = SIGP ? TB_R : row_rmax(MODE, C::PAIRS, TB);
    uint32_t *lc = nullptr;
    if (MODE == SEMIGLOBAL)
        lc = reinterpret_cast<uint32_t *>(dyn_smem + lc_offset(SIGP, A.alphabet)) + (warp * 2 + grp) * 2 * GROUP * RMAX;
    const int per_item = 2 * C::PAIRS;
    const int64_t n_list = *A.n_list;
    const int64_t n_items = (n_list + per_item - 1) / per_item;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(A.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        // rows per lane: the least R that covers the longest query in its chunks (the
        // direction-word layout of tb.cu plans the same R)
        ItemPlan P = plan_item(A.list, n_list, item, per_item, A.q_off, A.s_off, RMAX);
        if (SIGP && TB) P.R = TB_R;
        uint32_t tbin = 0;
        if (!(TB || SIGP) && (A.rmax_tab || A.bin_stats)) {
            // the tuned tile shape of this item's length bin (rows per lane cap)
            int32_t nmax = 0;
            for (int kk = 0; kk < per_item; kk++) nmax = max(nmax, P.n[kk]);
            tbin = lbucket(nmax);
            const int cap = A.rmax_tab ? (int)A.rmax_tab[tbin] : 0;
            if (cap > 0 && cap < RMAX)
                P = plan_item(A.list, n_list, item, per_item, A.q_off, A.s_off, cap);
        }
        long long t_item = 0;
        if (A.bin_stats && lane == 0) t_item = clock64();
        Slot sl;
        int32_t pid[2] = {-1, -1};
#pragma unroll
        for (int h = 0; h < 2; h++) {
            int k = grp * C::PAIRS + h;
            bool ok = h < C::PAIRS && P.pid[k] >= 0;
            pid[h] = ok ? P.pid[k] : -1;
            sl.n[h] = ok ? P.n[k] : 0;
            sl.m[h] = ok ? P.m[k] : 0;
            sl.q0[h] = ok ? A.q_off[P.pid[k]] : 0;
            sl.s0[h] = ok ? A.s_off[P.pid[k]] : 0;
            sl.rev[h] = false;
            sl.tb[h] = A.o;
            sl.pad[h] = P.nch * GROUP * P.R - sl.n[h];
        }
        int32_t res[6];
        if (P.nch > 1 && A.scratch == nullptr) {
            // the host sizes the border scratch for every multi-chunk query; never reached
            continue;
        }
        // the traceback kernels and the local row-profile kernels (whose per-row maxima
        // and columns leave no registers for the inlined walk) take run_slot
        if constexpr (TB || (MODE == LOCAL && SIGP == 0)) {
            if (SIGP && TB) {
                run_slot<C, MODE, TB_R, TB, SIGP>(A, sm, sl, P.nch, P.Mit, g, gslot, res, pid, qp, tab, lc);
            } else {
                switch (P.R) {
#define ANYSEQ_TB_CASE(RR) \
    case RR: run_slot<C, MODE, rsel<RMAX>(RR), TB, SIGP>(A, sm, sl, P.nch, P.Mit, g, gslot, res, pid, qp, tab, lc); break;
                    ANYSEQ_TB_CASE(2) ANYSEQ_TB_CASE(3) ANYSEQ_TB_CASE(4) ANYSEQ_TB_CASE(5) ANYSEQ_TB_CASE(6)
                    ANYSEQ_TB_CASE(7) ANYSEQ_TB_CASE(8) ANYSEQ_TB_CASE(9) ANYSEQ_TB_CASE(10) ANYSEQ_TB_CASE(11)
                    ANYSEQ_TB_CASE(12) ANYSEQ_TB_CASE(13) ANYSEQ_TB_CASE(14) ANYSEQ_TB_CASE(15)
#undef ANYSEQ_TB_CASE
                    default: run_slot<C, MODE, RMAX, TB, SIGP>(A, sm, sl, P.nch, P.Mit, g, gslot, res, pid, qp, tab, lc); break;
                }
            }
        } else {
            // score only: the lean step loop (batch_score.cuh), one copy per rows-per-lane count
            switch (P.R) {
#define ANYSEQ_SC_CASE(RR) \
    case RR: score_slot<C, MODE, rsel<RMAX>(RR), SIGP, RMAX>(A, sm, sl, P.nch, P.Mit, g, lane, gslot, res, qp, tab, lc); break;
                ANYSEQ_SC_CASE(2) ANYSEQ_SC_CASE(3) ANYSEQ_SC_CASE(4) ANYSEQ_SC_CASE(5) ANYSEQ_SC_CASE(6)
                ANYSEQ_SC_CASE(7) ANYSEQ_SC_CASE(8) ANYSEQ_SC_CASE(9) ANYSEQ_SC_CASE(10) ANYSEQ_SC_CASE(11)
                ANYSEQ_SC_CASE(12) ANYSEQ_SC_CASE(13) ANYSEQ_SC_CASE(14) ANYSEQ_SC_CASE(15)
#undef ANYSEQ_SC_CASE
                default: score_slot<C, MODE, RMAX, SIGP, RMAX>(A, sm, sl, P.nch, P.Mit, g, lane, gslot, res, qp, tab, lc); break;
            }
        }
        if (A.bin_stats && lane == 0) {
            // SM cycles of the item and its cells, per length bin (autotuning)
            unsigned long long cells = 0;
            for (int kk = 0; kk < per_item; kk++) cells += (unsigned long long)P.n[kk] * (unsigned long long)P.m[kk];
            atomicAdd(&A.bin_stats[2 * tbin], (unsigned long long)(clock64() - t_item));
            atomicAdd(&A.bin_stats[2 * tbin + 1], cells);
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

// Dynamic shared memory: [sigma table (1 KB) + per-group query profiles] for the
// matrix path, then the per-group last-column buffers of the semi-global kernels.
static size_t dyn_smem_bytes(int sigp, int alphabet, int mode, bool tb) {
    const int groups = batch_threads(sigp) / GROUP;
    const int rmax = sigp ? TB_R : 16;
    return lc_offset(sigp, alphabet) + (mode == SEMIGLOBAL ? (size_t)groups * 2 * GROUP * rmax * 4 : 0);
}

// One instantiation: launch (occupancy == false) or blocks per SM (occupancy == true).
template <class C, int MODE, bool TB, int SIGP>
static int run_one(const BatchArgs *A, int alphabet, int grid, cudaStream_t st, bool occupancy, cudaError_t *err) {
    auto kern = batch_kernel<C, MODE, TB, SIGP>;
    const size_t dyn = dyn_smem_bytes(SIGP, alphabet, MODE, TB);
    // static rings + dynamic buffers may exceed the 48 KB default: opt in explicitly
    if (dyn) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (occupancy) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, batch_threads(SIGP), dyn) != cudaSuccess) {
            cudaGetLastError();
            nb = 1;
        }
        return nb < 1 ? 1 : nb;
    }
    kern<<<grid, batch_threads(SIGP), dyn, st>>>(*A);
    *err = cudaGetLastError();
    return 0;
}

// Every variant of one mode and lane type: launch (occupancy == false) or
// blocks per SM.
template <class C, int MODE>
int run_mode(const BatchArgs *A, int tb, int sigp, int alphabet, int grid, cudaStream_t st, bool occ,
             cudaError_t *err) {
    if (sigp) return tb ? run_one<C, MODE, true, 1>(A, alphabet, grid, st, occ, err)
                        : run_one<C, MODE, false, 1>(A, alphabet, grid, st, occ, err);
    return tb ? run_one<C, MODE, true, 0>(A, alphabet, grid, st, occ, err)
              : run_one<C, MODE, false, 0>(A, alphabet, grid, st, occ, err);
}

}  // namespace anyseq
