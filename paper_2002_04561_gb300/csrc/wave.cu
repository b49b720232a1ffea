// Intra-sequence wavefront for one long pair (Sec. IV-C, Sec. VI): global
// alignment of q[1..n] against s[1..m] in linear space, 32-bit lanes.
//
// The rows are cut into stripes of 32 lanes x WR rows (WR = 16, or 8 for local
// passes and for problems too small to fill the GPU with 16-row stripes). A
// warp owns a stripe and walks all m columns; lane l is one step behind lane l-1 and gets
// its upper neighbours by shfl.up (the anti-diagonal dependency of Sec. III-A).
// Stripe k reads the last row of stripe k-1 from a border row in global memory
// and writes its own for stripe k+1 (two border rows, alternating): the first
// row and column of a submatrix come in, its last row goes out (Sec. III-A,
// Fig. submatrix). A border block of 32 columns is published with a release
// store of the stripe's progress counter and consumed after an acquire load;
// persistent warps take stripes in increasing order from an atomic counter, so
// a waiting stripe only waits for a stripe that a running warp already owns.
// Every wait has an iteration limit; on expiry the kernel raises an error flag
// that makes every other waiter give up too, and the host returns
// ANYSEQ_ERR_TIMEOUT.
//
// Per cell: the batched kernel's cell (engine.cuh) in one of two forms, H as a
// three-input maximum (six instructions) or as max(diagonal, F) followed by an
// add-max with E (seven, with a one-instruction chain through the rows);
// launch_wave picks the form by the number of stripes per SM.
#include <type_traits>

#include "common.cuh"
#include "engine.cuh"
#include "wave.h"

namespace anyseq {

constexpr int WG = WAVE_LANES;
constexpr int WRING = 128;

__device__ __forceinline__ uint32_t wletter(const uint32_t *packed, int64_t base, int32_t len, int32_t idx, bool rev) {
    return code2(packed, base + (rev ? (int64_t)(len - 1 - idx) : (int64_t)idx));
}

__device__ __forceinline__ int32_t ld_acquire(const int32_t *p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int32_t *p, int32_t v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t ld_relaxed(const int32_t *p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Rings of WRING columns plus one more block: the selectors and the top row keep
// a copy of ring block 0 after the ring's end, and lane 31's bottom stores run
// on past it, so a lane walks one block from one base address without wrapping.
struct __align__(16) WaveSmem {
    uint32_t sel[WRING + BLOCK];
    int32_t top[2 * (WRING + BLOCK)];
    int32_t bot[2 * (WRING + BLOCK)];
};

// Best-cell searches of a mode: over every cell, or over the last row and column.
__host__ __device__ constexpr bool best_all(int mode) { return mode == LOCAL || mode == ANCHORED_LOCAL; }
__host__ __device__ constexpr bool best_edge(int mode) { return mode == SEMIGLOBAL || mode == ANCHORED_SEMIGLOBAL; }

// TB: also write the traceback direction words of every cell (the layout of the
// batched traceback with 32 lanes x WR rows per chunk, see tb.h), global only.
// MODE: the initialisation and optimum of Sec. III-A, or an anchored mode of
// the start-cell pass (wave.h). Passes with a best-cell search keep their best
// cell as a key (score, then smaller i, then smaller j) merged per pass by a
// 64-bit atomic maximum: over every cell from each row's running maximum and
// its first column (rows per lane 8 there, the extra registers), over the edge
// from the last column (at each lane's last-column step) and the last row (the
// last stripe's bottom row).
//
// MAT: the substitution-matrix path (alphabets above 4 letters). Each warp
// builds the query profile of its stripe in shared memory, byte [a][row] =
// sigma'(q_row, a) for the stripe's 32 x WR rows; the subject ring holds the
// byte offset of the column letter's plane, and a lane reads its WR bytes of
// that plane in one vector load. sigma' of row r is then one byte permute, as
// on the row-profile path.
// Two CTAs of 8 warps per SM (up to 128 registers a thread): 4- and 8-row stripes are
// picked only when a launch has few stripes per SM, so more resident warps would
// not run, and at 64 registers those variants spilled.
template <int WR, bool TB, int MODE, bool TRI, bool MAT, bool SPLIT = false>
__global__ void __launch_bounds__(256, 2) wave_kernel(WaveArgs A) {
    constexpr int INIT = wave_init_mode(MODE);
    constexpr bool ALL = best_all(MODE), EDGE = best_edge(MODE);
    constexpr int WCH = WG * WR;  // rows per stripe
    static_assert(!TB || WR == 4 || WR % 8 == 0, "direction words hold 8 rows (4 in the low half of each byte)");
    constexpr int WPL = (WR + 7) / 8;  // direction words per lane and step
    static_assert(!TB || MODE == GLOBAL, "traceback on the wavefront is global");
    static_assert(!(TB && MAT), "the wavefront's traceback variant takes 2-bit letters");
    static_assert(!SPLIT || (WR == 16 && TRI && MODE == GLOBAL && !TB && !MAT),
                  "split steps: global three-input-maximum score passes with 16 rows per lane");
    // steps from lane 0's column to lane 31's last row at that column: each lane is one
    // column behind the previous, two with split steps (whose lower half runs one more behind)
    constexpr int RAMP = SPLIT ? 2 * (WG - 1) + 1 : WG - 1;
    // refill blocks between a block's first step and the drain of its bottom row
    constexpr int DLAG = SPLIT ? 3 : 2;
    __shared__ WaveSmem smem[8];
    extern __shared__ __align__(16) uint8_t wdyn[];
    const int warp = threadIdx.x >> 5, g = threadIdx.x & 31;
    WaveSmem *sm = &smem[warp];
    int8_t *stab = reinterpret_cast<int8_t *>(wdyn);
    uint8_t *qp = wdyn + WAVE_SIG_BYTES + (size_t)warp * A.alphabet * WCH;
    if (MAT) {
        for (int x = threadIdx.x; x < A.alphabet * A.alphabet; x += blockDim.x) stab[x] = A.sig[x];
        // selectors are read one step ahead, also at ring slots no column of the stripe
        // has filled yet: every slot holds a valid plane offset from the start
        for (int x = g; x < WRING + BLOCK; x += WG) sm->sel[x] = 0;
        __syncthreads();
    }
    typedef CellI32 C;
    typedef int32_t T;
    const int32_t o = A.o, e = A.e, oe = A.o + A.e;
    const uint32_t e_raw = C::raw(e), oe_raw = C::raw(oe), oe_c = C::cst(oe), e_c = C::cst(e);
    // Stripes go to warps in the order they draw them. Consecutive stripes on one SM
    // compete for its issue slots and shared-memory pipe while other SMs idle, so a
    // warp holds back its first draw by its rank (1 us each): the warp index times the
    // CTAs per SM, plus its CTA's launch wave (blockIdx / SMs). With CTAs dispatched
    // breadth-first over the SMs, the warps of one rank sit on distinct SMs. A warp
    // stops waiting once every stripe is taken. (A 35,000-residue protein pair, 137
    // stripes: 14.2 -> 7.3 ms; 100 kbp global, 781 stripes: 32.6 -> 25.9 ms.)
    if (!A.no_spread && A.grid_sms > 0 && g == 0) {
        const int rank = warp * (int)(gridDim.x / (unsigned)A.grid_sms) + (int)(blockIdx.x / (unsigned)A.grid_sms);
        for (int z = 0; z < rank && ld_relaxed(A.stripe_counter) < A.n_stripes; z++) __nanosleep(1000);
    }
    __syncwarp();
    for (;;) {
        int32_t t = 0;
        if (g == 0) t = atomicAdd(A.stripe_counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= A.n_stripes) break;
        // the pass owning global stripe t (binary search over stripe0)
        int lo = 0, hi = A.n_passes - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (A.passes[mid].stripe0 <= t) lo = mid; else hi = mid - 1;
        }
        const WavePass ps = A.passes[lo];
        const int32_t n = ps.n, m = ps.m;
        const int32_t nstripes = (n + WCH - 1) / WCH;
        const int32_t pad = nstripes * WCH - n;
        const int S = m + RAMP;
        const int32_t k = t - ps.stripe0;
        const bool last = (k == nstripes - 1);
        const bool rev = ps.rev != 0;
        int32_t *outH = A.last_H ? A.last_H + ps.out_off : nullptr;
        int32_t *outE = A.last_E ? A.last_E + ps.out_off : nullptr;
        const int32_t rb = k * WCH + g * WR + 1;
        uint32_t prof[WR];  // row profiles (unused on the matrix path)
        T Hoe[WR], F[WR];
#pragma unroll
        for (int r = 0; r < WR; r++) {
            int32_t i = rb + r - pad;
            if constexpr (!MAT) prof[r] = (i >= 1) ? A.rowprof[wletter(A.q2, ps.q0, n, i - 1, rev)] : A.rowprof[4];
            else prof[r] = 0;
            Hoe[r] = col0(INIT, i, o, e, ps.tb) + oe;
            F[r] = C::NEG;
        }
        if (MAT) {
            // this lane's rows of the stripe's query profile (the warp's previous
            // stripe is finished: its last step ended with a warp barrier)
            __syncwarp();
            int32_t qa[WR];
#pragma unroll
            for (int r = 0; r < WR; r++) {
                const int32_t i = rb + r - pad;
                // codes >= alphabet (an ANYSEQ_ERR_ALPHABET call) are clamped inside the table
                qa[r] = i >= 1 ? min((int32_t)A.q8[ps.q0 + (rev ? (int64_t)(n - i) : (int64_t)(i - 1))], A.alphabet - 1) : -1;
            }
            for (int a = 0; a < A.alphabet; a++) {
#pragma unroll
                for (int w4 = 0; w4 < WR / 4; w4++) {
                    uint32_t word = 0;
#pragma unroll
                    for (int b = 0; b < 4; b++) {
                        const int32_t q = qa[4 * w4 + b];
                        const int32_t v = q >= 0 ? (int32_t)stab[q * A.alphabet + a] : A.sig_pad;
                        word |= ((uint32_t)v & 0xFFu) << (8 * b);
                    }
                    *reinterpret_cast<uint32_t *>(qp + (size_t)a * WCH + g * WR + 4 * w4) = word;
                }
            }
            __syncwarp();
        }
        const T diag0 = col0(INIT, rb - 1 - pad, o, e, ps.tb) + oe;
        // best-cell searches: this lane's best cell as a key (the pass's floor is
        // set by the host); rows' running maxima (Hoe) and their first columns
        uint64_t best = 0;
        T rowmax[ALL ? WR : 1];
        int32_t rowj[ALL ? WR : 1];
        if (ALL) {
#pragma unroll
            for (int r = 0; r < WR; r++) {
                rowmax[r] = oe;  // Hoe of H = 0
                rowj[r] = 0;
            }
        }
        const int2 *bin = A.border + ps.border_off + (int64_t)((k - 1) & 1) * m;
        int2 *bout = A.border + ps.border_off + (int64_t)(k & 1) * m;
        int32_t *prog_prev = A.prog + ps.stripe0 + (k > 0 ? k - 1 : 0);
        int32_t *prog_mine = A.prog + t;
        bool failed = false;
        // this stripe's direction words: [step][lane][WR / 8]
        uint32_t *dw = TB ? A.dirs + ps.dir_off + (int64_t)k * S * WG * WPL + g * WPL : nullptr;

        // wait until the previous stripe published border block blk (bounded)
        // The previous stripe's progress last seen (warp-uniform): blocks below it were
        // published before the release that the acquire observed, so the warp polls only
        // when it has caught up (the previous stripe usually runs several blocks ahead).
        int32_t seen_prog = 0;
        auto wait_for = [&](int blk) {
            if (k == 0 || failed || seen_prog >= blk + 1) return;
            int ok = 1;
            int32_t v = 0;
            if (g == 0) {
                int64_t spins = 0;
                while ((v = ld_acquire(prog_prev)) < blk + 1) {
                    if (++spins > A.spin_limit || *((volatile int32_t *)A.err)) {
                        atomicExch(A.err, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            seen_prog = __shfl_sync(0xffffffffu, v, 0);
            failed = !ok;
            __syncwarp();
        };
        // ring refill in two halves: fetch issues this lane's global loads of a block
        // (packed subject word, border of the previous stripe) into registers, put
        // writes them to the rings; in between, the warp computes, so the loads'
        // latency overlaps half a block of cells
        auto fetch = [&](int blk, uint32_t &fw, int32_t &fsh, int2 &ft) {
            const int c = blk * BLOCK + g;
            if (c < m) {
                const int64_t pos = ps.s0 + (rev ? (int64_t)(m - 1 - c) : (int64_t)c);
                if (MAT) {
                    // a code >= alphabet (an ANYSEQ_ERR_ALPHABET call) is clamped, so that
                    // the profile read it selects stays in shared memory
                    fw = min((uint32_t)A.s8[pos], (uint32_t)A.alphabet - 1u);
                } else {
                    fw = A.s2[pos >> 4];
                    fsh = 2 * (int32_t)(pos & 15);
                }
                if (k == 0) {
                    // row 0: H(0, c+1); E below row 0 comes from H only (E(0, .) = -inf)
                    const int32_t v = (INIT == GLOBAL ? o + (c + 1) * e : 0) + oe;
                    ft = make_int2(v, v);
                } else if (!failed) {
                    ft = bin[c];
                }
            }
        };
        auto put = [&](int blk, uint32_t fw, int32_t fsh, int2 ft) {
            const int c = blk * BLOCK + g;
            if (c < m) {
                const uint32_t sv = MAT ? fw * (uint32_t)WCH : C::selector((fw >> fsh) & 3u, 0);
                sm->sel[c & (WRING - 1)] = sv;
                reinterpret_cast<int2 *>(sm->top)[c & (WRING - 1)] = ft;
                if ((blk & 3) == 0) {
                    sm->sel[WRING + (c & (WRING - 1))] = sv;
                    reinterpret_cast<int2 *>(sm->top)[WRING + (c & (WRING - 1))] = ft;
                }
            }
        };
        auto fill = [&](int blk) {
            uint32_t fw = 0;
            int32_t fsh = 0;
            int2 ft = make_int2(C::NEG, C::NEG);
            fetch(blk, fw, fsh, ft);
            put(blk, fw, fsh, ft);
        };
        // drain in two halves too: the stores of a finished bottom block, and (after a
        // warp barrier) the release of the progress counter
        // lane 31 stored column c at step c + 31, at (its block's base column - 31) + offset
        auto bot_index = [&](int c) {
            const int sw = (c + RAMP) & ~(BLOCK - 1);
            return ((sw - RAMP) & (WRING - 1)) + (c + RAMP - sw);
        };
        auto drain_stores = [&](int blk) {
            int c = blk * BLOCK + g;
            if (blk >= 0 && c < m) {
                const int2 b2 = reinterpret_cast<const int2 *>(sm->bot)[bot_index(c)];
                const int32_t hv = b2.x, ev = b2.y;
                if (!last) {
                    bout[c] = make_int2(hv, ev);
                } else {
                    if (outH) outH[c + 1] = hv - oe;
                    if (outE) outE[c + 1] = ev;
                    if (EDGE) {
                        const uint64_t key = end_key(hv - oe, n, c + 1);
                        best = key > best ? key : best;
                    }
                }
            }
        };
        auto drain = [&](int blk) {
            int c = blk * BLOCK + g;
            if (blk >= 0 && c < m) {
                const int2 b2 = reinterpret_cast<const int2 *>(sm->bot)[bot_index(c)];
                const int32_t hv = b2.x, ev = b2.y;
                if (!last) {
                    bout[c] = make_int2(hv, ev);
                } else {
                    if (outH) outH[c + 1] = hv - oe;
                    if (outE) outE[c + 1] = ev;
                    if (EDGE) {
                        const uint64_t key = end_key(hv - oe, n, c + 1);
                        best = key > best ? key : best;
                    }
                }
            }
            __syncwarp();
            if (!last && g == 0 && blk >= 0) st_release(prog_mine, blk + 1);
        };

        wait_for(0);
        fill(0);
        __syncwarp();
        int drained = 0;
        // exported values: this lane's last row (Hoe, and E of the row below); lane 31,
        // whose last row goes to the bottom ring, exports lane 0's border value for its
        // next column instead (the row above the stripe, one column ahead)
        T xh, xe, prev_up = diag0;
        {
            const int2 tv = reinterpret_cast<const int2 *>(sm->top)[0];
            xh = tv.x;
            xe = tv.y;
        }
        const int src = (g + WG - 1) & (WG - 1);  // lane g-1; lane 0 reads lane 31
        // base addresses of the current block: this lane's selectors (column s - g at
        // offset s - s0), lane 31's top loads and bottom stores
        const uint32_t *selp = sm->sel;
        uint32_t topa = 0, bota = 0;
        // loaded one step ahead, so that no shared-memory latency sits in a step's chain:
        // the next step's selector (and on the matrix path this lane's sigma' bytes of
        // its letter), and on lane 31 the top value lane 0 takes after the next step
        uint32_t nsel = sm->sel[(0 - (SPLIT ? 2 : 1) * g) & (WRING - 1)];
        uint32_t nwq[MAT ? WR / 4 : 1];
        auto load_wq = [&](uint32_t sv, uint32_t (&w)[MAT ? WR / 4 : 1]) {
            if constexpr (MAT) {
                const uint8_t *p = qp + sv + g * WR;
                if constexpr (WR == 16) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(p);
                    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
                } else if constexpr (WR == 8) {
                    const uint2 v = *reinterpret_cast<const uint2 *>(p);
                    w[0] = v.x; w[1] = v.y;
                } else {
                    w[0] = *reinterpret_cast<const uint32_t *>(p);
                }
            } else {
                w[0] = 0;
            }
        };
        load_wq(nsel, nwq);
        uint32_t ph, pe;
        {
            const int2 tv = reinterpret_cast<const int2 *>(sm->top)[1];
            ph = (uint32_t)tv.x;
            pe = (uint32_t)tv.y;
        }
        // one step: column s - g of this lane's rows (j = s - s0). Checked steps (the first
        // block, where lane g has no column before step g, and the blocks that reach the
        // last column) skip columns outside the pair and look for the last column's cells.
        auto step = [&](const int s, const int j, auto careful_tag) {
            constexpr bool CAREFUL = decltype(careful_tag)::value;
            const int c = s - g;
            const T up_hoe = (T)__shfl_sync(0xffffffffu, (uint32_t)xh, src);
            const T up_e = (T)__shfl_sync(0xffffffffu, (uint32_t)xe, src);
            T stE = xe;  // E stored by lane 31: of the row below, or its own in the last stripe
            // this step's selector and sigma' bytes (matrix path); the next step's are
            // loaded now (selp[j + 1] stays inside the ring's extra block)
            const uint32_t sel = nsel;
            (void)sel;  // the matrix path reads its sigma' bytes instead
            uint32_t wq[MAT ? WR / 4 : 1];
#pragma unroll
            for (int w = 0; w < (MAT ? WR / 4 : 1); w++) wq[w] = nwq[w];
            nsel = selp[j + 1];
            load_wq(nsel, nwq);
            if (!CAREFUL || (unsigned)c < (unsigned)m) {
                auto sigma_r = [&](int r) -> uint32_t {
                    if constexpr (MAT) {
                        const uint32_t b = (uint32_t)(r & 3);  // byte b, sign-extended
                        return prmt(wq[r >> 2], 0u, b | ((b | 8u) << 4) | ((b | 8u) << 8) | ((b | 8u) << 12));
                    }
                    else return (uint32_t)C::sigma(prof[r], prof[r], sel);
                };
                // prev_up is diag0 until the first valid column; each later row takes the
                // old Hoe of the row above before that register is overwritten
                T Ad = C::addc(prev_up, sigma_r(0));
                prev_up = up_hoe;
                T E = up_e, Ein = up_e;
                T hup = up_hoe;  // Hoe of the row above, this column (traceback)
                uint32_t pl_s0 = 0, pl_s1 = 0, pl_eo = 0, pl_fo = 0;
#pragma unroll
                for (int r = 0; r < WR; r++) {
                    const T Adr = Ad;
                    if (r + 1 < WR) Ad = C::addc(Hoe[r], sigma_r(r + 1));
                    uint32_t fFo = 0;
                    Ein = E;
                    if (TRI) {
                        // H by one 3-input maximum: fewer instructions, but a chain of three
                        // through the rows instead of one, so the launch picks it only when
                        // enough stripes run side by side to hide the latency. Local mode
                        // keeps F >= 0 instead of clamping H (exact for H: max(F, 0)
                        // follows the same recurrence)
                        if (MODE == LOCAL) F[r] = C::vmax3(C::addc(F[r], e_c), Hoe[r], 0);  // Eq. 5
                        else F[r] = C::addmax(F[r], e_raw, Hoe[r]);                        // Eq. 5
                        Hoe[r] = C::addc(C::vmax3(Adr, F[r], E), oe_c);                    // Eq. 1
                        E = C::addmax(E, e_raw, Hoe[r]);                                   // Eq. 4, row i+1
                    } else {
                        F[r] = C::addmax(F[r], e_raw, Hoe[r]);                             // Eq. 5
                        const T M = (MODE == LOCAL) ? C::maxrelu(Adr, F[r]) : C::vmax(Adr, F[r]);  // the clamp at 0
                        const T X = C::addc(M, oe_c);
                        if (TB) fFo = C::ge(Hoe[r], F[r]);         // F(i,j) opened from H(i,j-1)
                        Hoe[r] = C::addmax(E, oe_raw, X);                                  // Eq. 1
                        E = C::addmax(E, e_raw, X);                                        // Eq. 4, row i+1
                    }
                    if (ALL) {
                        // strict improvement of the row maximum: the column of its first occurrence
                        uint32_t unused = 0, jr = (uint32_t)rowj[r];
                        C::track(rowmax[r], jr, unused, Hoe[r], (uint32_t)(c + 1));
                        rowj[r] = (int32_t)jr;
                    }
                    if (TB) {
                        // the predecessor planes of the batched traceback (global mode)
                        const uint32_t fD = C::ge(C::addc(Adr, oe_c), Hoe[r]);  // diagonal reaches H
                        const uint32_t fE = C::ge(C::addc(Ein, oe_c), Hoe[r]);  // E reaches H
                        const uint32_t fEo = C::ge(hup, Ein);                  // E(i,j) opened from H(i-1,j)
                        const uint32_t FM = C::flag_mask();
                        pl_s0 = (pl_s0 >> 1) | (fD & FM);
                        pl_s1 = (pl_s1 >> 1) | (fE & FM);
                        pl_eo = (pl_eo >> 1) | (fEo & FM);
                        pl_fo = (pl_fo >> 1) | (fFo & FM);
                        hup = Hoe[r];
                        if ((r & 7) == 7 || r == WR - 1) {
                            // rows (r & ~7)..r: bytes s0, s1, E opened, F opened (bit k = row
                            // (r & ~7) + k); a word of fewer than 8 rows shifts them down to bit 0
                            const int sh = 7 - (r & 7);
                            dw[(int64_t)s * WG * WPL + (r >> 3)] =
                                prmt(prmt(pl_s0 >> sh, pl_s1 >> sh, 0x7351u), prmt(pl_eo >> sh, pl_fo >> sh, 0x7351u), 0x7632u);
                        }
                    }
                }
                if (EDGE && CAREFUL && c == m - 1) {
#pragma unroll
                    for (int r = 0; r < WR; r++) {
                        const int32_t i = rb + r - pad;
                        if (i >= 1) {
                            const uint64_t key = end_key(Hoe[r] - oe, i, m);
                            best = key > best ? key : best;
                        }
                    }
                }
                xh = Hoe[WR - 1];
                xe = E;
                // border for the next stripe: (Hoe, E of the row below); the last stripe
                // keeps E of its own last row for the Hirschberg join
                stE = last ? Ein : E;
            }
            {
                // lane 31: its last row to the bottom ring; it then exports lane 0's next
                // border value (loaded a step ago) and loads the one after. Predicated
                // shared-memory accesses rather than a branch around them
                uint32_t hx = (uint32_t)xh, ex = (uint32_t)xe;
                asm volatile(
                    "{ .reg .pred p;\n\t"
                    "setp.eq.u32 p, %7, 31;\n\t"
                    "@p st.shared.v2.u32 [%4], {%0, %6};\n\t"
                    "@p mov.b32 %0, %2;\n\t"
                    "@p mov.b32 %1, %3;\n\t"
                    "@p ld.shared.v2.u32 {%2, %3}, [%5]; }"
                    : "+r"(hx), "+r"(ex), "+r"(ph), "+r"(pe)
                    : "r"(bota + 8u * (uint32_t)j), "r"(topa + 8u * (uint32_t)(j + 1)), "r"((uint32_t)stE), "r"(g)
                    : "memory");
                xh = (T)hx;
                xe = (T)ex;
            }
        };
        // Split step (SPLIT): rows 0..7 (half A) at column s - 2g, rows 8..15 (half B) one
        // column behind. The halves are two independent dependency chains of 8 rows in one
        // step instead of one of 16. Half B takes its diagonal, the E entering row 8 and the
        // column's selector from the previous step.
        constexpr int HR = WR / 2;
        T midD = 0, midE = C::NEG;
        uint32_t sel_prev = 0;
        if (SPLIT) midD = col0(INIT, rb + HR - 1 - pad, o, e, ps.tb) + oe;
        auto step2 = [&](const int s, const int j, auto careful_tag) {
            constexpr bool CAREFUL = decltype(careful_tag)::value;
            const int cA = s - 2 * g, cB = cA - 1;
            const T up_hoe = (T)__shfl_sync(0xffffffffu, (uint32_t)xh, src);
            const T up_e = (T)__shfl_sync(0xffffffffu, (uint32_t)xe, src);
            const uint32_t sel = nsel;
            nsel = selp[j + 1];  // the next step's, one step ahead
            const T h7 = Hoe[HR - 1];  // row 7 before this step (half B's diagonal next step)
            T EA = C::NEG, stE = xe;
            const bool okA = !CAREFUL || (unsigned)cA < (unsigned)m;
            const bool okB = !CAREFUL || (unsigned)cB < (unsigned)m;
            if (okA && okB) {
                // both halves, interleaved row by row (two independent chains)
                T AdA = C::addc(prev_up, (uint32_t)C::sigma(prof[0], prof[0], sel));
                T AdB = C::addc(midD, (uint32_t)C::sigma(prof[HR], prof[HR], sel_prev));
                prev_up = up_hoe;
                T E = up_e, EB = midE, EinB = midE;
#pragma unroll
                for (int k = 0; k < HR; k++) {
                    const int ra = k, rb2 = HR + k;
                    const T Ara = AdA, Arb = AdB;
                    if (k + 1 < HR) {
                        AdA = C::addc(Hoe[ra], (uint32_t)C::sigma(prof[ra + 1], prof[ra + 1], sel));
                        AdB = C::addc(Hoe[rb2], (uint32_t)C::sigma(prof[rb2 + 1], prof[rb2 + 1], sel_prev));
                    }
                    F[ra] = C::addmax(F[ra], e_raw, Hoe[ra]);                          // Eq. 5
                    F[rb2] = C::addmax(F[rb2], e_raw, Hoe[rb2]);
                    Hoe[ra] = C::addc(C::vmax3(Ara, F[ra], E), oe_c);                  // Eq. 1
                    Hoe[rb2] = C::addc(C::vmax3(Arb, F[rb2], EB), oe_c);
                    E = C::addmax(E, e_raw, Hoe[ra]);                                  // Eq. 4
                    EinB = EB;
                    EB = C::addmax(EB, e_raw, Hoe[rb2]);
                }
                EA = E;
                xh = Hoe[WR - 1];
                xe = EB;
                stE = last ? EinB : EB;
            } else {
                if (okA) {
                    T Ad = C::addc(prev_up, (uint32_t)C::sigma(prof[0], prof[0], sel));
                    prev_up = up_hoe;
                    T E = up_e;
#pragma unroll
                    for (int r = 0; r < HR; r++) {
                        const T Adr = Ad;
                        if (r + 1 < HR) Ad = C::addc(Hoe[r], (uint32_t)C::sigma(prof[r + 1], prof[r + 1], sel));
                        F[r] = C::addmax(F[r], e_raw, Hoe[r]);
                        Hoe[r] = C::addc(C::vmax3(Adr, F[r], E), oe_c);
                        E = C::addmax(E, e_raw, Hoe[r]);
                    }
                    EA = E;
                }
                if (okB) {
                    T Ad = C::addc(midD, (uint32_t)C::sigma(prof[HR], prof[HR], sel_prev));
                    T E = midE, Ein = midE;
#pragma unroll
                    for (int r = HR; r < WR; r++) {
                        const T Adr = Ad;
                        if (r + 1 < WR) Ad = C::addc(Hoe[r], (uint32_t)C::sigma(prof[r + 1], prof[r + 1], sel_prev));
                        F[r] = C::addmax(F[r], e_raw, Hoe[r]);
                        Hoe[r] = C::addc(C::vmax3(Adr, F[r], E), oe_c);
                        Ein = E;
                        E = C::addmax(E, e_raw, Hoe[r]);
                    }
                    xh = Hoe[WR - 1];
                    xe = E;
                    stE = last ? Ein : E;
                }
            }
            midD = h7;
            midE = EA;
            sel_prev = sel;
            {
                // lane 31: its last row (half B's column) to the bottom ring; it then
                // exports lane 0's next border value (loaded a step ago) and loads the
                // one after
                uint32_t hx = (uint32_t)xh, ex = (uint32_t)xe;
                asm volatile(
                    "{ .reg .pred p;\n\t"
                    "setp.eq.u32 p, %7, 31;\n\t"
                    "@p st.shared.v2.u32 [%4], {%0, %6};\n\t"
                    "@p mov.b32 %0, %2;\n\t"
                    "@p mov.b32 %1, %3;\n\t"
                    "@p ld.shared.v2.u32 {%2, %3}, [%5]; }"
                    : "+r"(hx), "+r"(ex), "+r"(ph), "+r"(pe)
                    : "r"(bota + 8u * (uint32_t)j), "r"(topa + 8u * (uint32_t)(j + 1)), "r"((uint32_t)stE), "r"(g)
                    : "memory");
                xh = (T)hx;
                xe = (T)ex;
            }
        };
        for (int s0 = 0; s0 < S && !failed; s0 += BLOCK) {
            const int kb = s0 / BLOCK;
            if ((kb + 1) * BLOCK < m) wait_for(kb + 1);
            uint32_t fw = 0;
            int32_t fsh = 0;
            int2 ft = make_int2(C::NEG, C::NEG);
            fetch(kb + 1, fw, fsh, ft);
            int released = -1;
            if (kb - DLAG >= drained) {
                drain_stores(kb - DLAG);
                released = kb - DLAG;
                drained = kb - DLAG + 1;
            }
            const int s1 = min(S, s0 + BLOCK), sm_ = min(s1, s0 + BLOCK / 2);
            selp = &sm->sel[(s0 - (SPLIT ? 2 : 1) * g) & (WRING - 1)];
            topa = (uint32_t)__cvta_generic_to_shared(&sm->top[2 * ((s0 + 1) & (WRING - 1))]);
            bota = (uint32_t)__cvta_generic_to_shared(&sm->bot[2 * ((s0 - RAMP) & (WRING - 1))]);
            const bool careful = s0 < RAMP || s0 + BLOCK >= m;
            auto run_half = [&](int sa, int sb) {
                if constexpr (SPLIT) {
                    if (careful) {
                        for (int s = sa; s < sb; s++) step2(s, s - s0, std::true_type{});
                    } else {
                        for (int s = sa; s < sb; s++) step2(s, s - s0, std::false_type{});
                    }
                } else {
                    if (careful) {
                        for (int s = sa; s < sb; s++) step(s, s - s0, std::true_type{});
                    } else {
                        for (int s = sa; s < sb; s++) step(s, s - s0, std::false_type{});
                    }
                }
            };
            run_half(s0, sm_);
            put(kb + 1, fw, fsh, ft);
            __syncwarp();
            if (released >= 0 && !last && g == 0) st_release(prog_mine, released + 1);
            run_half(sm_, s1);
        }
        __syncwarp();
        for (int b = drained; b <= (m - 1) / BLOCK; b++) drain(b);
        if (!last && g == 0) st_release(prog_mine, (m + BLOCK - 1) / BLOCK + 1);
        if (last && g == 0) {
            if (outH) outH[0] = col0(INIT, n, o, e, ps.tb);
            if (outE) outE[0] = col0(INIT, n, o, e, ps.tb);
        }
        if (ALL || EDGE) {
            if (ALL) {
#pragma unroll
                for (int r = 0; r < WR; r++) {
                    const int32_t i = rb + r - pad, v = rowmax[r] - oe;
                    if (i >= 1 && v > 0) {
                        const uint64_t key = end_key(v, i, rowj[r]);
                        best = key > best ? key : best;
                    }
                }
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const uint64_t ox = __shfl_xor_sync(0xffffffffu, best, off);
                best = ox > best ? ox : best;
            }
            if (g == 0) atomicMax(reinterpret_cast<unsigned long long *>(A.best) + lo,
                                  (unsigned long long)best);
        }
    }
}

// Dynamic shared memory of a launch: none on the row-profile path; the sigma'
// table and one query profile per warp (alphabet x 32 x WR bytes) on the
// matrix path.
static size_t wave_dyn_smem(bool mat, int wr, int alphabet) {
    return mat ? (size_t)WAVE_SIG_BYTES + 8 * (size_t)alphabet * WG * wr : 0;
}

// Stripes for every four SMs from which a launch takes a taller stripe.
constexpr int WAVE_MIN_STRIPES_PER_4_SMS = 3;

template <int WR, bool TB, int MODE, bool TRI = false, bool MAT = false, bool SPLIT = false>
static int blocks_per_sm(size_t dyn = 0) {
    auto kern = wave_kernel<WR, TB, MODE, TRI, MAT, SPLIT>;
    if (dyn) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, dyn) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return nb < 1 ? 1 : nb;
}

int wave_rows_per_lane(int64_t total_rows, int num_sms, int64_t n_passes, int mode, int forced, bool min8) {
    // stripes of a launch at wr rows per lane (an upper bound of sum(ceil(n / (32 wr))))
    auto stripes = [&](int wr) { return total_rows / (WG * wr) + n_passes; };
    int wr;
    if (forced == 4 || forced == 8 || forced == 16) {
        wr = forced;
        if (best_all(mode) && wr == 16) wr = 8;   // the rows' maxima and columns take registers
        if (best_edge(mode) && wr == 8) wr = 16;  // its 8-row variant would spill
    } else if (best_all(mode)) {
        // local passes: the rows' maxima and columns make a short step cost relatively
        // more (35,000-residue local pair: 6.5 ms at 8 rows, 7.2 at 4)
        wr = 8;
    } else {
        // the tallest stripes that still give about three stripes for every four SMs:
        // a stripe moves at the speed of its warp's chain, so taller stripes do more
        // per step, and too few leave SMs idle (global pairs, ms at 16 / 8 / 4 rows:
        // 35 kbp 5.65 / 5.05 / 5.91, 100 kbp 16.2 / 18.9 / 20.5)
        const int64_t want = (int64_t)num_sms * WAVE_MIN_STRIPES_PER_4_SMS / 4;
        if (stripes(16) >= want) wr = 16;
        else if (!best_edge(mode) && stripes(8) >= want) wr = 8;
        else wr = 4;
    }
    // the allocation-free scratch is sized for 8-row stripes
    if (min8 && wr < 8) wr = 8;
    return wr;
}

template <int WR, bool TB, int MODE, bool TRI = false, bool MAT = false, bool SPLIT = false>
static void launch_one(const WaveArgs &A, int num_sms, cudaStream_t st) {
    const size_t dyn = wave_dyn_smem(MAT, WR, A.alphabet);
    int per_sm = blocks_per_sm<WR, TB, MODE, TRI, MAT, SPLIT>(dyn);
    if (A.ctas_per_sm > 0 && A.ctas_per_sm < per_sm) per_sm = A.ctas_per_sm;
    WaveArgs B = A;
    B.grid_sms = num_sms;
    wave_kernel<WR, TB, MODE, TRI, MAT, SPLIT><<<num_sms * per_sm, 256, dyn, st>>>(B);
}

// 16-row stripes side by side per SM from which global passes take the
// 3-input-maximum cell with split steps (two chains per step, one more block of
// skew per stripe). Measured on single pairs, ms, two-step cell / 3-input cell /
// 3-input cell with split steps: 100 kbp (1.3 stripes per SM) 17 / 23 / 19, 300 kbp
// (3.9) 76 / 85 / 74, 500 kbp (6.4) 142-146 / 146-152 / 135-136, 700 kbp (9.0)
// - / 275-293 / 238-254, 1 Mbp (12.9) - / 460-470 / 403-405. The 3-input cell
// without split steps no longer wins anywhere; in semi-global passes, where it
// spills, it is never taken.
constexpr int WAVE_TRI_STRIPES_PER_SM = 3;
constexpr int WAVE_SPLIT_STRIPES_PER_SM = 3;
// Launches capped below the CTAs that fit (the serving lanes: one CTA per SM) run
// many small passes side by side on at most 8 warps per SM; there the lower
// thresholds cut the serving sweep's capacity from about 3,800 to 2,680 requests/s,
// so they keep the earlier ones.
constexpr int WAVE_TRI_STRIPES_PER_SM_CAPPED = 8;
constexpr int WAVE_SPLIT_STRIPES_PER_SM_CAPPED = 12;

cudaError_t launch_wave(const WaveArgs &A, int num_sms, cudaStream_t st) {
    const bool tb = A.dirs != nullptr;
    const bool capped = A.ctas_per_sm > 0;
    const int64_t tri_from = capped ? WAVE_TRI_STRIPES_PER_SM_CAPPED : WAVE_TRI_STRIPES_PER_SM;
    const int64_t split_from = capped ? WAVE_SPLIT_STRIPES_PER_SM_CAPPED : WAVE_SPLIT_STRIPES_PER_SM;
    const bool tri = A.mode == GLOBAL && A.rows_per_lane >= 16 && !A.mat &&
                     (A.cell == 1 || (A.cell == 0 && (int64_t)A.n_stripes >= tri_from * num_sms));
    // the stripe table was built for A.rows_per_lane (from wave_rows_per_lane)
    const int wr = A.rows_per_lane;
    if (tb && wr != 4 && wr != 8 && wr != 16) return cudaErrorInvalidValue;
    if (A.mode != GLOBAL && (tb || (wr != 4 && wr != (best_all(A.mode) ? 8 : 16)))) return cudaErrorInvalidValue;
    if (A.mode == GLOBAL && wr != 4 && wr != 8 && wr != 16) return cudaErrorInvalidValue;
    if (A.mat) {
        // the matrix path: letters one byte each, sigma' from shared query profiles
        if (tb || A.alphabet < 1 || A.alphabet > 32 || !A.q8 || !A.s8 || !A.sig) return cudaErrorInvalidValue;
        if (wr == 4) {
            if (A.mode == LOCAL) launch_one<4, false, LOCAL, false, true>(A, num_sms, st);
            else if (A.mode == ANCHORED_LOCAL) launch_one<4, false, ANCHORED_LOCAL, false, true>(A, num_sms, st);
            else if (A.mode == SEMIGLOBAL) launch_one<4, false, SEMIGLOBAL, false, true>(A, num_sms, st);
            else if (A.mode == ANCHORED_SEMIGLOBAL) launch_one<4, false, ANCHORED_SEMIGLOBAL, false, true>(A, num_sms, st);
            else if (A.mode == GLOBAL) launch_one<4, false, GLOBAL, false, true>(A, num_sms, st);
            else return cudaErrorInvalidValue;
            return cudaGetLastError();
        }
        if (A.mode == LOCAL) launch_one<8, false, LOCAL, false, true>(A, num_sms, st);
        else if (A.mode == ANCHORED_LOCAL) launch_one<8, false, ANCHORED_LOCAL, false, true>(A, num_sms, st);
        else if (A.mode == SEMIGLOBAL) launch_one<16, false, SEMIGLOBAL, false, true>(A, num_sms, st);
        else if (A.mode == ANCHORED_SEMIGLOBAL) launch_one<16, false, ANCHORED_SEMIGLOBAL, false, true>(A, num_sms, st);
        else if (A.mode != GLOBAL) return cudaErrorInvalidValue;
        else if (A.rows_per_lane == 8) launch_one<8, false, GLOBAL, false, true>(A, num_sms, st);
        else launch_one<16, false, GLOBAL, false, true>(A, num_sms, st);
        return cudaGetLastError();
    }
    if (wr == 4) {
        if (A.mode == LOCAL) launch_one<4, false, LOCAL>(A, num_sms, st);
        else if (A.mode == ANCHORED_LOCAL) launch_one<4, false, ANCHORED_LOCAL>(A, num_sms, st);
        else if (A.mode == SEMIGLOBAL) launch_one<4, false, SEMIGLOBAL>(A, num_sms, st);
        else if (A.mode == ANCHORED_SEMIGLOBAL) launch_one<4, false, ANCHORED_SEMIGLOBAL>(A, num_sms, st);
        else if (A.mode == GLOBAL && tb) launch_one<4, true, GLOBAL>(A, num_sms, st);
        else if (A.mode == GLOBAL) launch_one<4, false, GLOBAL>(A, num_sms, st);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    if (A.mode == LOCAL) {
        launch_one<8, false, LOCAL>(A, num_sms, st);
    } else if (A.mode == ANCHORED_LOCAL) {
        launch_one<8, false, ANCHORED_LOCAL>(A, num_sms, st);
    } else if (A.mode == SEMIGLOBAL) {
        launch_one<16, false, SEMIGLOBAL>(A, num_sms, st);
    } else if (A.mode == ANCHORED_SEMIGLOBAL) {
        launch_one<16, false, ANCHORED_SEMIGLOBAL>(A, num_sms, st);
    } else if (A.mode != GLOBAL) {
        return cudaErrorInvalidValue;
    } else if (A.rows_per_lane == 8) {
        if (tb) launch_one<8, true, GLOBAL>(A, num_sms, st);
        else launch_one<8, false, GLOBAL>(A, num_sms, st);
    } else {
        if (tb) launch_one<16, true, GLOBAL>(A, num_sms, st);
        else if (tri && (A.split == 1 || (A.split == 0 && (int64_t)A.n_stripes >= split_from * num_sms)))
            launch_one<16, false, GLOBAL, true, false, true>(A, num_sms, st);
        else if (tri) launch_one<16, false, GLOBAL, true>(A, num_sms, st);
        else launch_one<16, false, GLOBAL>(A, num_sms, st);
    }
    return cudaGetLastError();
}

}  // namespace anyseq
