// Learned band for global alignment (an extension that keeps results exact):
// k-mer diagonal features, banded DP restricted to a staircase of row chunks,
// and an exit certificate that proves the banded score is the full optimum.
//
// Band of centre c and half-width w (integers): row i keeps the columns j with
// |j*n - i*m - c*n| <= w*n, i.e. within w of the straight line from (0,0) to
// (n,m) shifted by c. The kernel relaxes, for each chunk of 128 rows, the
// column interval covering its rows' bands (the staircase B); (0,0) and (n,m)
// are always inside.
//
// Certificate: every path from (0,0) to (n,m) that leaves B has a first step
// p -> x from a cell p in B to a cell x outside B, and the part up to p scores
// at most the banded value at p. From x the rest scores at most
//   U(x) = Mmax * min(n - i, m - j) + extend * |(n - i) - (m - j)|
// (all letters matched where possible, the length difference as gap
// extensions, no opens). With X the largest exit value
//   right: F(i, j+1) + U(i, j+1) and H(i, j) + Mmax + U(i+1, j+1),
//   down:  E(i+1, j) + U(i+1, j) and H(i, j) + Mmax + U(i+1, j+1),
// the banded score S is the optimum whenever S >= X (S > X when a CIGAR must
// also be unique). Otherwise the caller widens the band or runs the full DP.
#include <type_traits>

#include "band.h"
#include "batch.h"
#include "common.cuh"
#include "engine.cuh"

namespace anyseq {

// ------------------------------------------------------------------ features

constexpr int KMER = 12;
constexpr int HT = 8192;  // shared hash slots (sampled query k-mers <= 4097)

__device__ __forceinline__ uint32_t fbucket(int64_t x) {
    if (x == 0) return 0;
    int lg = 63 - __clzll(x);
    uint32_t second = lg >= 1 ? (uint32_t)((x >> (lg - 1)) & 1) : 0u;
    uint32_t b = 1u + 2u * (uint32_t)lg + second;
    return b > 31u ? 31u : b;
}

__device__ __forceinline__ uint32_t kmer_at(const uint32_t *packed, int64_t pos) {
    return codes16(packed, pos, (int64_t)1 << 40) & 0xFFFFFFu;
}

// One block per pair: sampled query k-mers into a shared hash table (smallest
// position per key), then every subject k-mer votes for the bin of its hit.
__global__ void kmer_hist_kernel(const uint32_t *q2, const uint32_t *s2, const int64_t *q_off, const int64_t *s_off,
                                 const int32_t *pairs, int64_t n_pairs, float *feat) {
    extern __shared__ __align__(16) uint32_t fsm[];  // keys[HT], pos[HT], hist[64]
    uint32_t *keys = fsm;
    int32_t *pos = reinterpret_cast<int32_t *>(fsm + HT);
    uint32_t *hist = fsm + 2 * HT;
    for (int64_t t = blockIdx.x; t < n_pairs; t += gridDim.x) {
        const int64_t p = pairs ? pairs[t] : t;
        const int64_t q0 = q_off[p], s0 = s_off[p];
        const int64_t n = q_off[p + 1] - q0, m = s_off[p + 1] - s0;
        for (int k = threadIdx.x; k < HT; k += blockDim.x) { keys[k] = 0xFFFFFFFFu; pos[k] = 0x7FFFFFFF; }
        if (threadIdx.x < 64) hist[threadIdx.x] = 0;
        __syncthreads();
        if (n >= KMER && m >= KMER) {
            const int64_t stride = 4 * ((n + 16383) / 16384);
            const int64_t nk = (n - KMER) / stride + 1;
            for (int64_t u = threadIdx.x; u < nk; u += blockDim.x) {
                const int32_t i = (int32_t)(u * stride);
                const uint32_t key = kmer_at(q2, q0 + i);
                uint32_t h = (key * 0x9E3779B1u) >> (32 - 13);
                for (;;) {
                    uint32_t prev = atomicCAS(&keys[h], 0xFFFFFFFFu, key);
                    if (prev == 0xFFFFFFFFu || prev == key) { atomicMin(&pos[h], i); break; }
                    h = (h + 1) & (HT - 1);
                }
            }
            __syncthreads();
            for (int64_t j = threadIdx.x; j <= m - KMER; j += blockDim.x) {
                const uint32_t key = kmer_at(s2, s0 + j);
                uint32_t h = (key * 0x9E3779B1u) >> (32 - 13);
                while (keys[h] != 0xFFFFFFFFu) {
                    if (keys[h] == key) {
                        const int64_t i = pos[h];
                        const int64_t d = (j - i) * n - (m - n) * i;
                        const uint32_t b = fbucket((d < 0 ? -d : d) / n);
                        atomicAdd(&hist[d >= 0 ? 32 + b : 31 - b], 1u);
                        break;
                    }
                    h = (h + 1) & (HT - 1);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < 64) {
            // hits per sampled query k-mer: the mass carries the similarity of the pair
            const int64_t nk = (n >= KMER && m >= KMER) ? (n - KMER) / (4 * ((n + 16383) / 16384)) + 1 : 0;
            feat[t * 64 + threadIdx.x] = nk ? (float)hist[threadIdx.x] / (float)nk : 0.0f;
        }
        __syncthreads();
    }
}

cudaError_t launch_kmer_hist(const uint32_t *q2, const uint32_t *s2, const int64_t *q_off, const int64_t *s_off,
                             const int32_t *pairs, int64_t n_pairs, float *feat, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    int64_t g = n_pairs < 65535 ? n_pairs : 65535;
    const int smem = (2 * HT + 64) * 4;
    cudaFuncSetAttribute(kmer_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    kmer_hist_kernel<<<(unsigned)g, 256, smem, st>>>(q2, s2, q_off, s_off, pairs, n_pairs, feat);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- targets

// One thread per pair: offsets D = j*n - i*m of every cell on the path of a
// CIGAR (starting at (0,0)), as min and max divided by n (floor / ceil).
__global__ void path_extent_kernel(const int64_t *q_off, const int64_t *s_off, const anyseq_result_t *res,
                                   const uint32_t *cigar, int64_t n_pairs, int32_t *dmin, int32_t *dmax) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = q_off[p + 1] - q_off[p], m = s_off[p + 1] - s_off[p];
        int64_t i = 0, j = 0, lo = 0, hi = 0;
        const uint32_t *c = cigar + res[p].cigar_off;
        for (uint32_t k = 0; k < res[p].cigar_len; k++) {
            const uint32_t len = c[k] >> 4, op = c[k] & 15u;
            for (uint32_t t = 0; t < len; t++) {
                if (op != 2u) i++;
                if (op != 1u) j++;
                const int64_t d = j * n - i * m;
                lo = d < lo ? d : lo;
                hi = d > hi ? d : hi;
            }
        }
        const int64_t nn = n > 0 ? n : 1;
        dmin[p] = (int32_t)((lo - (nn - 1)) / nn);  // floor for lo <= 0
        dmax[p] = (int32_t)((hi + nn - 1) / nn);    // ceil for hi >= 0
    }
}

cudaError_t launch_path_extent(const int64_t *q_off, const int64_t *s_off, const anyseq_result_t *res,
                               const uint32_t *cigar, int64_t n_pairs, int32_t *dmin, int32_t *dmax, cudaStream_t st) {
    int64_t b = (n_pairs + 255) / 256;
    path_extent_kernel<<<(unsigned)(b < 1 ? 1 : (b > 65535 ? 65535 : b)), 256, 0, st>>>(q_off, s_off, res, cigar,
                                                                                       n_pairs, dmin, dmax);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- banded DP


__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Band of a pair: around the line from (0,0) to (n,m), row i keeps the
// columns within w(i) of the line shifted by c(i), with c(i) = c (n-i)/n and
// w(i) = wm + (w - wm) (n-i)/n, wm = min(w, BAND_WMIN): both taper linearly to
// the end cell. An exit at row i must beat the banded score by about the
// shortfall of the remaining n - i rows against all-match scoring (the
// certificate's bound), so the margin the band needs shrinks with the rows left;
// the optimal path starts and ends on the line, so the shift tapers too.
constexpr int32_t BAND_WMIN = 16;

// DP-column interval [lo, hi] of the chunk holding real rows [ilo, ihi]
// (rows <= 0 stand for row 0); the first chunk starts at column 0 and the last
// one ends at column m so that (0,0) and (n,m) are inside. The left edge is the
// smallest left edge of the rows from ilo to n and the right edge the largest
// right edge of the rows up to ihi, so consecutive chunks form a staircase.
__device__ __forceinline__ void chunk_cols(int64_t n, int64_t m, int32_t c, int32_t w, int64_t ilo, int64_t ihi,
                                           bool first, bool last, int32_t &lo, int32_t &hi) {
    // a chunk that holds padding rows (copies of row 0) starts at column 0
    if (ilo <= 0) first = true;
    ilo = ilo < 0 ? 0 : ilo;
    ihi = ihi < 0 ? 0 : ihi;
    const int64_t nn = n > 0 ? n : 1;
    const int64_t wm = w < BAND_WMIN ? w : BAND_WMIN;
    // n * (left edge + wm) and n * (right edge - wm) of row i are linear in i
    auto left_num = [&](int64_t i) { return i * m + ((int64_t)c - w + wm) * (n - i); };
    auto right_num = [&](int64_t i) { return i * m + ((int64_t)c + w - wm) * (n - i); };
    const int64_t ln = min(left_num(ilo), left_num(n)), rn = max(right_num(0), right_num(ihi));
    int64_t l = -floor_div(-ln, nn) - wm;  // ceil
    int64_t h = floor_div(rn, nn) + wm;
    if (first || l < 0) l = 0;
    if (last || h > m) h = m;
    if (l > m) l = m;
    if (h < l) h = l;
    lo = (int32_t)l;
    hi = (int32_t)h;
}

// Bound of the certificate from cell (i, j) to (n, m). In 32-bit arithmetic:
// pairs of the banded route run in 32-bit lanes (|values| < 2^28), and the
// bound is at most Mmax * 2^21 < 2^28.
__device__ __forceinline__ int32_t ubound(int32_t n, int32_t m, int32_t i, int32_t j, int32_t mmax, int32_t e) {
    const int32_t di = n - i, dj = m - j;
    const int32_t mn = di < dj ? di : dj, df = di > dj ? di - dj : dj - di;
    return mmax * mn + e * df;
}

// Rings of RING columns plus one more block (the step loop's layout of the
// batched kernel: a copy of ring block 0 after the ring's end for the selectors
// and the top row, room for lane 15's stores past the end in the bottom ring).
struct __align__(16) BandSmem {
    uint32_t sel[RING + BLOCK];
    int32_t top[2 * (RING + BLOCK)];
    int32_t bot[2 * (RING + BLOCK)];
};

// One pair per 16-lane slot (32-bit lanes, global mode), chunks of GROUP * BR
// rows over the band's column window; both slots of a warp run the same BR.
template <int BR>
__device__ __noinline__ void band_slot(const BandArgs &A, BandSmem *sm, int32_t *scr, int g, bool have, int32_t p) {
    typedef CellI32 C;
    typedef int32_t T;
    constexpr int BCH = GROUP * BR;  // rows per chunk
    const int32_t o = A.o, e = A.e, oe = o + e;
    const uint32_t e_raw = C::raw(e), oe_raw = C::raw(oe), oe_c = C::cst(oe);
        const int64_t q0 = have ? A.q_off[p] : 0, s0 = have ? A.s_off[p] : 0;
        const int32_t n = have ? (int32_t)(A.q_off[p + 1] - q0) : 0;
        const int32_t m = have ? (int32_t)(A.s_off[p + 1] - s0) : 0;
        const int32_t bc = have ? A.centre[p] : 0, bw = have ? A.width[p] : 0;
        // chunking shared by the warp: enough chunks for the longer query
        int32_t nmax = max(n, __shfl_xor_sync(0xffffffffu, n, 16));
        const int32_t nch = nmax > 0 ? (nmax + BCH - 1) / BCH : 1;
        const int32_t pad = nch * BCH - n;
        int32_t best_exit = INT32_MIN / 2;  // X, per lane
        int32_t score = 0;
        int64_t cells = 0;                  // relaxed cells of this pair (lane 0)
        int32_t pa = 0, pb = 0;  // previous chunk's computed columns (c in [pa, pb))
        for (int ch = 0; ch < nch; ch++) {
            const bool last = ch == nch - 1;
            const int32_t rb = ch * BCH + g * BR + 1;
            // DP columns [lo, hi] of this chunk and [nlo, nhi] of the next; computed
            // columns c = j - 1 in [a, b) and the left boundary column j = a
            int32_t lo = 0, hi = 0, nlo = 0, nhi = 0;
            if (have && n > 0) {
                chunk_cols(n, m, bc, bw, (int64_t)ch * BCH + 1 - pad, (int64_t)(ch + 1) * BCH - pad, ch == 0, last, lo, hi);
                if (!last)
                    chunk_cols(n, m, bc, bw, (int64_t)(ch + 1) * BCH + 1 - pad, (int64_t)(ch + 2) * BCH - pad, false,
                               ch + 1 == nch - 1, nlo, nhi);
            }
            int32_t a = lo >= 1 ? lo - 1 : 0, b = hi;
            const bool left_in = lo == 0;
            if (!have) { a = 0; b = 0; }
            const int32_t W = b - a;
            const int32_t Wmax = max(W, __shfl_xor_sync(0xffffffffu, W, 16));
            cells += (int64_t)W * BCH;
            const int S = Wmax + GROUP - 1;
            uint32_t prof[BR];
            T Hoe[BR], F[BR];
#pragma unroll
            for (int r = 0; r < BR; r++) {
                int32_t i = rb + r - pad;
                prof[r] = (i >= 1) ? A.rowprof[code2(A.q2, q0 + i - 1)] : A.rowprof[4];
                Hoe[r] = left_in ? col0(GLOBAL, i, o, e, o) + oe : C::NEG;
                F[r] = C::NEG;
            }
            // diagonal of the first computed cell: H(row above, j = a)
            T diag0 = C::NEG;
            if (left_in) diag0 = col0(GLOBAL, rb - 1 - pad, o, e, o) + oe;
            else if (g == 0 && ch > 0 && a - 1 >= pa && a - 1 < pb) diag0 = scr[2 * (a - 1)];
            if (g == 0 && have) {
                // exits along the boundary row and column (H values are closed forms there);
                // row 0 is padded row `pad` (or the virtual row above chunk 0 when pad == 0)
                const bool holds_row0 = pad == 0 ? ch == 0 : (ch * BCH < pad && (ch + 1) * BCH >= pad);
                if (holds_row0 && hi < m) {
                    int64_t h0 = hi == 0 ? 0 : o + (int64_t)hi * e;
                    int32_t v = o + (hi + 1) * e + ubound(n, m, 0, hi + 1, A.mmax, e);
                    best_exit = max(best_exit, v);
                    // diagonal into (1, hi+1): inside only if row 1 opens the next chunk and keeps that column
                    const bool row1_next = (ch + 1) * BCH < pad + 1;
                    const bool inside = row1_next && !last && hi + 1 >= nlo && hi + 1 <= nhi;
                    if (n >= 1 && !inside) best_exit = max(best_exit, (int32_t)h0 + A.mmax + ubound(n, m, 1, hi + 1, A.mmax, e));
                }
                int64_t ir = (int64_t)(ch + 1) * BCH - pad;  // last row of this chunk
                if (!last && left_in && nlo >= 1 && ir >= 0 && ir < n) {
                    int64_t hd = col0(GLOBAL, (int32_t)(ir + 1), o, e, o);  // H(ir+1, 0) via column 0
                    best_exit = max(best_exit, (int32_t)hd + ubound(n, m, (int32_t)ir + 1, 0, A.mmax, e));
                    if (nlo >= 2) {
                        int64_t hr = col0(GLOBAL, (int32_t)ir, o, e, o);
                        best_exit = max(best_exit, (int32_t)hr + A.mmax + ubound(n, m, (int32_t)ir + 1, 1, A.mmax, e));
                    }
                }
            }

            auto fill = [&](int blk) {
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    int cr = blk * BLOCK + g + 16 * k;
                    if (cr < W) {
                        int c = a + cr;
                        const uint32_t sv = C::selector(code2(A.s2, s0 + c), 0);
                        sm->sel[cr & (RING - 1)] = sv;
                        if ((blk & 3) == 0) sm->sel[RING + (cr & (RING - 1))] = sv;
                        int2 tv;
                        if (ch > 0) {
                            const bool in = c >= pa && c < pb;
                            tv = in ? make_int2(scr[2 * c], scr[2 * c + 1]) : make_int2(C::NEG, C::NEG);
                        } else {
                            // row 0: H(0, c+1); E below row 0 comes from H only
                            tv.x = tv.y = o + (c + 1) * e + oe;
                        }
                        reinterpret_cast<int2 *>(sm->top)[cr & (RING - 1)] = tv;
                        if ((blk & 3) == 0) reinterpret_cast<int2 *>(sm->top)[RING + (cr & (RING - 1))] = tv;
                    }
                }
            };
            // lane 15 stored column cr at step cr + 15, at (its block's base - 15) + offset
            auto bot_index = [&](int cr) {
                const int sw = (cr + GROUP - 1) & ~(BLOCK - 1);
                return ((sw - (GROUP - 1)) & (RING - 1)) + (cr + GROUP - 1 - sw);
            };
            auto drain = [&](int blk) {
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    int cr = blk * BLOCK + g + 16 * k;
                    if (blk >= 0 && cr < W) {
                        int c = a + cr;
                        const int2 b2 = reinterpret_cast<const int2 *>(sm->bot)[bot_index(cr)];
                        const int32_t hv = b2.x, ev = b2.y;
                        if (!last) {
                            scr[2 * c] = hv;
                            scr[2 * c + 1] = ev;
                            // down exits: cell (ir, j = c + 1) below which the next chunk
                            // keeps only the DP columns >= nlo
                            int64_t ir = (int64_t)(ch + 1) * BCH - pad;  // this chunk's last row
                            const int64_t j = c + 1;
                            if (j < nlo && ir >= 0 && ir < n) {
                                int32_t v = ev + ubound(n, m, (int32_t)ir + 1, (int32_t)j, A.mmax, e);
                                best_exit = v > best_exit ? v : best_exit;
                                if (j + 1 < nlo) {
                                    int32_t v2 = (hv - oe) + A.mmax + ubound(n, m, (int32_t)ir + 1, (int32_t)j + 1, A.mmax, e);
                                    best_exit = v2 > best_exit ? v2 : best_exit;
                                }
                            }
                        } else if (c == m - 1) {
                            score = hv - oe;
                        }
                    }
                }
            };
            __syncwarp();
            fill(0);
            __syncwarp();
            int drained = 0;
            // prev_up is diag0 until the first valid column
            // exported values: this lane's last row (Hoe, E of the row below); lane 15, whose
            // last row goes to the bottom ring, exports lane 0's border value for its next
            // column instead. prev_up is diag0 until the first valid column.
            T xh, xe, prev_up = diag0;
            {
                const int2 tv = reinterpret_cast<const int2 *>(sm->top)[0];
                xh = tv.x;
                xe = tv.y;
            }
            const int lane = (int)(threadIdx.x & 31);
            const int src = (lane & 16) | ((lane + GROUP - 1) & (GROUP - 1));  // lane g-1; lane 0 reads lane 15
            // the warp's steps where a lane reaches the last computed column of its window
            int wlo = W > 0 ? W - 1 : (1 << 30), whi = W - 1;
            wlo = min(wlo, __shfl_xor_sync(0xffffffffu, wlo, 16));
            whi = max(whi, __shfl_xor_sync(0xffffffffu, whi, 16)) + GROUP - 1;
            for (int s0b = 0; s0b < S; s0b += BLOCK) {
              __syncwarp();
              {
                const int kb = s0b / BLOCK;
                fill(kb + 1);
                if (kb - 2 >= drained) { drain(kb - 2); drained = kb - 1; }
              }
              __syncwarp();
              const int nst = min(S, s0b + BLOCK) - s0b;
              const uint32_t *selp = &sm->sel[(s0b - g) & (RING - 1)];
              const uint32_t topa = (uint32_t)__cvta_generic_to_shared(&sm->top[2 * ((s0b + 1) & (RING - 1))]);
              const uint32_t bota = (uint32_t)__cvta_generic_to_shared(&sm->bot[2 * ((s0b - (GROUP - 1)) & (RING - 1))]);
              // checked steps: the ramp (no column before step g) and the window's right edge
              // (the columns past it are left alone, the right exits are taken there); in
              // between, columns past a narrower window only feed values nobody reads
              auto run = [&](auto careful_tag) {
                constexpr bool CAREFUL = decltype(careful_tag)::value;
                for (int j = 0; j < nst; j++) {
                  const int cr = s0b + j - g;
                  const T up_hoe = (T)__shfl_sync(0xffffffffu, (uint32_t)xh, src);
                  const T up_e = (T)__shfl_sync(0xffffffffu, (uint32_t)xe, src);
                  if (!CAREFUL || (unsigned)cr < (unsigned)W) {
                    const uint32_t sel = selp[j];
                    T Ad = C::addc(prev_up, (uint32_t)C::sigma(prof[0], prof[0], sel));
                    prev_up = up_hoe;
                    T E = up_e;
#pragma unroll
                    for (int r = 0; r < BR; r++) {
                        F[r] = C::addmax(F[r], e_raw, Hoe[r]);                 // Eq. 5
                        const T Hn = C::vmax3(Ad, F[r], E);                    // Eq. 1, one 3-input maximum
                        if (r + 1 < BR) Ad = C::addc(Hoe[r], (uint32_t)C::sigma(prof[r + 1], prof[r + 1], sel));
                        Hoe[r] = C::addc(Hn, oe_c);
                        E = C::addmax(E, e_raw, Hoe[r]);                       // Eq. 4, row i+1
                    }
                    xh = Hoe[BR - 1];
                    xe = E;
                    // right exits from DP column hi = b (the chunk's last computed column)
                    if (CAREFUL && cr == W - 1 && b < m) {
#pragma unroll
                        for (int r = 0; r < BR; r++) {
                            int64_t i = (int64_t)rb + r - pad;
                            if (i >= 1) {
                                int32_t H = Hoe[r] - oe;
                                int32_t Fn = max(F[r] + e, Hoe[r]);  // F(i, hi + 1)
                                int32_t v = Fn + ubound(n, m, (int32_t)i, b + 1, A.mmax, e);
                                best_exit = v > best_exit ? v : best_exit;
                                // diagonal to (i+1, hi+1): outside unless row i+1 opens the next chunk
                                bool next_row_in_next = (r == BR - 1 && g == GROUP - 1);
                                bool inside = next_row_in_next && !last && b + 1 >= nlo && b + 1 <= nhi;
                                if (i + 1 <= n && !inside) {
                                    int32_t v2 = H + A.mmax + ubound(n, m, (int32_t)i + 1, b + 1, A.mmax, e);
                                    best_exit = v2 > best_exit ? v2 : best_exit;
                                }
                            }
                        }
                    }
                  }
                  {
                    // lane 15: its last row to the bottom ring, then lane 0's next border value in
                    uint32_t hx = (uint32_t)xh, ex = (uint32_t)xe;
                    asm volatile(
                        "{ .reg .pred p;\n\t"
                        "setp.eq.u32 p, %4, 15;\n\t"
                        "@p st.shared.v2.u32 [%2], {%0, %1};\n\t"
                        "@p ld.shared.v2.u32 {%0, %1}, [%3]; }"
                        : "+r"(hx), "+r"(ex)
                        : "r"(bota + 8u * (uint32_t)j), "r"(topa + 8u * (uint32_t)j), "r"(g)
                        : "memory");
                    xh = (T)hx;
                    xe = (T)ex;
                  }
                }
              };
              const bool careful = s0b == 0 || (s0b <= whi && s0b + BLOCK > wlo);
              if (careful) run(std::true_type{});
              else run(std::false_type{});
            }
            __syncwarp();
            for (int bk = drained; bk <= (Wmax - 1) / BLOCK; bk++) drain(bk);
            __syncwarp();
            pa = a;
            pb = b;
        }
        // reduce over the 16 lanes
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) {
            int32_t ox = __shfl_xor_sync(0xffffffffu, best_exit, off, GROUP);
            best_exit = ox > best_exit ? ox : best_exit;
            score |= __shfl_xor_sync(0xffffffffu, score, off, GROUP);
        }
        if (g == 0 && have) {
            if (A.cells) atomicAdd(A.cells, (unsigned long long)cells);
            A.score[p] = score;
            const bool ok = A.strict ? score > best_exit : score >= best_exit;
            A.accept[p] = ok ? 1 : 0;
        }
}

// Two slots of 16 lanes per warp, one pair per slot. Rows per lane follow the
// warp's wider band: a chunk's column window spans the band plus the band's
// drift over the chunk's rows, so tall chunks suit wide bands and short chunks
// narrow ones.
__global__ void __launch_bounds__(256, 2) band_kernel(BandArgs A) {
    __shared__ BandSmem smem[16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane >> 4, g = lane & 15;
    BandSmem *sm = &smem[warp * 2 + grp];
    const int64_t gslot = ((int64_t)blockIdx.x * 8 + warp) * 2 + grp;
    int32_t *scr = A.scratch + gslot * 2 * (int64_t)A.scratch_cols;
    const int64_t n_items = (A.n_list + 1) / 2;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(A.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const int64_t li = (int64_t)item * 2 + grp;
        const bool have = li < A.n_list;
        const int32_t p = have ? A.list[li] : -1;
        int32_t bw = have ? A.width[p] : 0;
        bw = max(bw, __shfl_xor_sync(0xffffffffu, bw, 16));
        if (bw >= 192) band_slot<12>(A, sm, scr, g, have, p);
        else if (bw >= 96) band_slot<8>(A, sm, scr, g, have, p);
        else band_slot<4>(A, sm, scr, g, have, p);
    }
}

cudaError_t launch_band(const BandArgs &A, int grid, cudaStream_t st) {
    band_kernel<<<grid, 256, 0, st>>>(A);
    return cudaGetLastError();
}

int band_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, band_kernel, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return nb < 1 ? 1 : nb;
}

}  // namespace anyseq
