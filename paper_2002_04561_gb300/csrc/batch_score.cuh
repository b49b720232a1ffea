// Score-only walk of one slot (score and optimum cell, no traceback): the
// kernels' hot loop. Same cell, chunking and results as run_slot (engine.cuh,
// batch_kernel.cuh); the step loop carries only the recurrence and the
// exchange between lanes:
//
// * Lane g takes Hoe and E of its first row's upper neighbour from lane g-1 by
//   one shuffle each. Lane 0 takes them from lane 15 too: lane 15 stores its
//   last row to the bottom ring and then loads, into the registers it exports,
//   the border value lane 0 needs at the next step (the row above the chunk,
//   one column ahead). No lane-0 select.
// * Steps run in refill blocks of B columns. Each lane holds a base address
//   into the rings at the block start and reads column s - g as base + j with
//   a constant offset; the rings keep a copy of their first block after their
//   end, so no index wraps inside a block.
// * Only the first block of a chunk (the 15-step ramp, where lane g has no
//   column before step g) and, in semi-global mode, the blocks where a lane
//   reaches the last column of a pair take the checked step. Columns past the
//   longest subject of the slot are null columns (sigma' = 0, border values
//   -inf or row 0) whose cells stay below earlier cells, so the tail needs no
//   guard: the last block just runs on to a multiple of the unroll.
// * The semi-global last column is stored with 128-bit shared stores.
#pragma once
#include <type_traits>

#include "engine.cuh"
#include "batch.h"

namespace anyseq {

template <class C, int MODE, int R, int SIGP, int RS>
__device__ __forceinline__ void score_slot(const BatchArgs &A, GroupSmemT<4 * block_cols(SIGP), block_cols(SIGP)> *sm,
                                           const Slot &sl, int nch, int Mit, int g, int lane, int64_t gslot,
                                           int32_t *res, uint32_t *qp, const int8_t *tab, uint32_t *lc) {
    typedef typename C::T T;
    constexpr int B = block_cols(SIGP), RING = 4 * B;
    constexpr int U = 2;  // unroll of the step loop
    const int32_t o = A.o, e = A.e, oe = A.o + A.e;
    const uint32_t e_raw = C::raw(e);
    const uint32_t oe_c = C::cst(oe), e_c = C::cst(e);
    const T zero = C::make(0, 0);
    const T NEGv = C::make(C::NEG, C::NEG);
    const int CH = GROUP * R;
    const int S = Mit + GROUP - 1;
    const int src = (lane & 16) | ((lane + 15) & 15);  // lane g-1; lane 0 reads lane 15
    int32_t *scr = A.scratch ? A.scratch + gslot * 2 * (int64_t)A.scratch_cols : nullptr;
    const int32_t m0 = sl.m[0], m1 = C::PAIRS == 2 ? sl.m[1] : 0;
    const int ev0 = m0 - 1, ev1 = C::PAIRS == 2 ? m1 - 1 : -1;  // last-column steps (+g)
    // the warp's window of steps where some lane reaches a last column
    int evlo = 1 << 30, evhi = -1;
    if (MODE == SEMIGLOBAL) {
        evlo = m0 > 0 ? ev0 : evlo;
        evhi = ev0;
        if (C::PAIRS == 2 && m1 > 0) {
            evlo = min(evlo, ev1);
            evhi = max(evhi, ev1);
        }
        evlo = min(evlo, __shfl_xor_sync(0xffffffffu, evlo, 16));
        evhi = max(evhi, __shfl_xor_sync(0xffffffffu, evhi, 16)) + GROUP - 1;
    }
    int2 *top2 = reinterpret_cast<int2 *>(sm->top);
    int2 *bot2 = reinterpret_cast<int2 *>(sm->bot);

    uint64_t best[2];
#pragma unroll
    for (int h = 0; h < 2; h++) best[h] = end_key(0, 0, MODE == SEMIGLOBAL ? sl.m[h] : 0);
    int32_t gscore[2] = {0, 0};

    for (int ch = 0; ch < nch; ch++) {
        const bool last = (ch == nch - 1);
        const int32_t rb = ch * CH + g * R + 1;  // padded row of register 0
        uint32_t profA[SIGP ? 1 : R], profB[SIGP ? 1 : R];
        T Hoe[R], F[R];
        T rowmax[MODE == LOCAL ? R : 1];  // the row maximum of H so far
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
            if (SIGP == 0) {
                profA[r] = pw[0];
                profB[r] = pw[1];
            }
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

        // ring fill of refill block blk: every column, null past the slot's longest
        // subject; ring block 0 is also written to the copy after the ring's end
        auto fill = [&](int blk) {
            const bool copy = (blk & 3) == 0;
#pragma unroll
            for (int k = 0; k < B / 16; k++) {
                const int c = blk * B + g + 16 * k;
                const int idx = c & (RING - 1);
                uint32_t selv;
                if (SIGP == 0) {
                    uint32_t ca = 0, cb = 0;
                    if (c < m0) ca = letter(A.s2, sl.s0[0], m0, c, sl.rev[0]);
                    if (C::PAIRS == 2 && c < m1) cb = letter(A.s2, sl.s0[1], m1, c, sl.rev[1]);
                    selv = C::null_past_end(C::selector(ca, cb), c < m0, c < m1);
                } else {
                    const uint32_t alpha = (uint32_t)A.alphabet;
                    uint32_t ca = alpha, cb = alpha;
                    // a code >= alphabet (the call then fails with ANYSEQ_ERR_ALPHABET) reads
                    // the null letter's row, so every profile read stays in shared memory
                    if (c < m0) ca = min((uint32_t)A.s8[sl.s0[0] + (sl.rev[0] ? m0 - 1 - c : c)], alpha);
                    if (C::PAIRS == 2 && c < m1) cb = min((uint32_t)A.s8[sl.s0[1] + (sl.rev[1] ? m1 - 1 - c : c)], alpha);
                    selv = (ca * QP_ROWS) | (((alpha + 1 + cb) * QP_ROWS) << 16);
                }
                int2 tv;
                if (ch > 0) {
                    tv = c < Mit ? make_int2(scr[2 * c], scr[2 * c + 1])
                                 : make_int2((int32_t)C::as_u(NEGv), (int32_t)C::as_u(NEGv));
                } else {
                    // row 0: H(0, c+1); E below row 0 comes from H only (E(0, .) = -inf)
                    const int32_t v = (MODE == GLOBAL ? o + (c + 1) * e : 0) + oe;
                    tv.x = tv.y = (int32_t)C::as_u(C::make(v, v));
                }
                sm->sel[idx] = selv;
                top2[idx] = tv;
                if (copy) {
                    sm->sel[RING + idx] = selv;
                    top2[RING + idx] = tv;
                }
            }
        };
        // drain of refill block blk of the bottom ring: lane 15 stored column c at
        // step c + 15, at its block's base (column of the block start - 15) + offset
        auto drain = [&](int blk) {
#pragma unroll
            for (int k = 0; k < B / 16; k++) {
                const int c = blk * B + g + 16 * k;
                if (c < Mit) {
                    const int sw = (c + GROUP - 1) & ~(B - 1);
                    const int idx = ((sw - (GROUP - 1)) & (RING - 1)) + (c + GROUP - 1 - sw);
                    const int2 hv2 = bot2[idx];
                    if (!last) {
                        scr[2 * c] = hv2.x;
                        scr[2 * c + 1] = hv2.y;
                    } else if (MODE != LOCAL) {
#pragma unroll
                        for (int h = 0; h < C::PAIRS; h++) {
                            const int32_t H = C::get(C::from_u((uint32_t)hv2.x), h) - oe;
                            if (MODE == SEMIGLOBAL && c < sl.m[h]) {
                                const uint64_t key = end_key(H, sl.n[h], c + 1);
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
        // exported values: own last row (Hoe, E of the next row); lane 15: lane 0's border
        T xh, xe;
        {
            const int2 tv = top2[0];
            xh = C::from_u((uint32_t)tv.x);
            xe = C::from_u((uint32_t)tv.y);
        }
        T prev_up = diag0;  // Hoe of the row above at the previous column (diagonal of row 0)
        const uint8_t *qpb = SIGP ? reinterpret_cast<const uint8_t *>(qp) + g * 8 : nullptr;
        int drained = 0;
        const int nblk = (S + B - 1) / B;
        for (int kb = 0; kb < nblk; kb++) {
            const int s0 = kb * B;
            __syncwarp();
            fill(kb + 1);
            if (kb - 2 >= drained) {
                drain(kb - 2);
                drained = kb - 1;
            }
            __syncwarp();
            const int nst = min(S - s0, B);
            const uint32_t *selp = &sm->sel[(s0 - g) & (RING - 1)];
            // shared-space addresses of lane 15's top load and bottom store at the block's first step
            const uint32_t topa = (uint32_t)__cvta_generic_to_shared(&top2[(s0 + 1) & (RING - 1)]);
            const uint32_t bota = (uint32_t)__cvta_generic_to_shared(&bot2[(s0 - (GROUP - 1)) & (RING - 1)]);
            const int c0 = s0 - g;  // this lane's column at the block's first step

            auto run = [&](auto careful_tag) {
                constexpr bool CAREFUL = decltype(careful_tag)::value;
                for (int j0 = 0; j0 < nst; j0 += U) {
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int j = j0 + u;
                        const int c = c0 + j;
                        const T up_hoe = C::from_u(__shfl_sync(0xffffffffu, C::as_u(xh), src));
                        const T up_e = C::from_u(__shfl_sync(0xffffffffu, C::as_u(xe), src));
                        const uint32_t sel = selp[j];
                        if (!CAREFUL || c >= 0) {
                            uint2 qa = make_uint2(0, 0), qb = make_uint2(0, 0);
                            if (SIGP) {
                                qa = *reinterpret_cast<const uint2 *>(qpb + (sel & 0xFFFFu));
                                if (C::PAIRS == 2) qb = *reinterpret_cast<const uint2 *>(qpb + (sel >> 16));
                            }
                            auto sigma_r = [&](int r) -> uint32_t {
                                if (SIGP == 0) return C::as_u(C::sigma(profA[r], profB[r], sel));
                                const uint32_t wa = (r & 4) ? qa.y : qa.x, wb = (r & 4) ? qb.y : qb.x;
                                const uint32_t b = (uint32_t)(r & 3);
                                return C::PAIRS == 2
                                           ? prmt(wa, wb, b | ((b | 8u) << 4) | ((b + 4u) << 8) | (((b + 4u) | 8u) << 12))
                                           : prmt(wa, wa, b | ((b | 8u) << 4) | ((b | 8u) << 8) | ((b | 8u) << 12));
                            };
                            T Ad = C::addc(prev_up, sigma_r(0));
                            prev_up = up_hoe;
                            T E = up_e;
                            const uint32_t jj = (uint32_t)(c + 1);
#pragma unroll
                            for (int r = 0; r < R; r++) {
                                T Adn = Ad;
                                if (r + 1 < R) Adn = C::addc(Hoe[r], sigma_r(r + 1));  // next row's diagonal
                                if (MODE == LOCAL) F[r] = C::vmax3(C::addc(F[r], e_c), Hoe[r], zero);  // Eq. 5
                                else F[r] = C::addmax(F[r], e_raw, Hoe[r]);                            // Eq. 5
                                const T Hn = C::vmax3(Ad, F[r], E);                                    // Eq. 1
                                Hoe[r] = C::addc(Hn, oe_c);
                                E = C::addmax(E, e_raw, Hoe[r]);                                       // Eq. 4
                                if (MODE == LOCAL) C::track(rowmax[r], rowj0[r], rowj1[r], Hn, jj);
                                Ad = Adn;
                            }
                            xh = Hoe[R - 1];
                            xe = E;
                            if (MODE == SEMIGLOBAL && CAREFUL) {
                                // this lane's rows of the last column of a half, 16 bytes per store
#pragma unroll
                                for (int h = 0; h < C::PAIRS; h++) {
                                    if (c == (h ? ev1 : ev0)) {
                                        uint32_t *dst = lc + (h * GROUP + g) * RS;
#pragma unroll
                                        for (int r = 0; r < R; r += 4) {
                                            if (r + 3 < R)
                                                *reinterpret_cast<uint4 *>(dst + r) =
                                                    make_uint4(C::as_u(Hoe[r]), C::as_u(Hoe[r + 1]), C::as_u(Hoe[r + 2]),
                                                               C::as_u(Hoe[r + 3]));
                                            else if (r + 1 < R)
                                                *reinterpret_cast<uint2 *>(dst + r) =
                                                    make_uint2(C::as_u(Hoe[r]), C::as_u(Hoe[r + 1]));
                                            if ((R & 1) && r + 2 == R - 1) dst[r + 2] = C::as_u(Hoe[r + 2]);
                                            if ((R & 1) && r == R - 1) dst[r] = C::as_u(Hoe[r]);
                                        }
                                    }
                                }
                            }
                        }
                        {
                            // lane 15: its last row to the bottom ring, lane 0's next border value in;
                            // predicated shared-memory accesses rather than a branch around them
                            uint32_t hx = C::as_u(xh), ex = C::as_u(xe);
                            asm volatile(
                                "{ .reg .pred p;\n\t"
                                "setp.eq.u32 p, %4, 15;\n\t"
                                "@p st.shared.v2.u32 [%2], {%0, %1};\n\t"
                                "@p ld.shared.v2.u32 {%0, %1}, [%3]; }"
                                : "+r"(hx), "+r"(ex)
                                : "r"(bota + 8u * (uint32_t)j), "r"(topa + 8u * (uint32_t)j), "r"(g)
                                : "memory");
                            xh = C::from_u(hx);
                            xe = C::from_u(ex);
                        }
                    }
                }
            };
            // local mode keeps one copy of the step loop (the checked one): its code is the
            // largest, and the second copy cost more in instruction fetch than it saved
            const bool careful = MODE == LOCAL || kb == 0 || (MODE == SEMIGLOBAL && s0 <= evhi && s0 + B > evlo);
            if (careful) run(std::true_type{});
            else run(std::false_type{});
        }
        __syncwarp();
        for (int b = drained; b <= (Mit - 1) / B; b++) drain(b);
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
                            const uint64_t k = end_key(C::get(C::from_u(lc[(h * GROUP + g) * RS + r]), h) - oe, i, sl.m[h]);
                            best[h] = k > best[h] ? k : best[h];
                        }
                    }
                }
            }
        }
        if (MODE == LOCAL) {
            // every row's maximum, at the first column it occurs (columns past the end of a
            // half never win: their values stay below an earlier real cell)
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
