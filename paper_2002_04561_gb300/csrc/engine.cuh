// Row-chunk DP engine shared by the batched, traceback and long-pair kernels.
//
// A group of GROUP = 16 lanes relaxes one "slot" (one pair in 32-bit lanes,
// two pairs in the two int16 halves) chunk by chunk. A chunk is 16*R rows;
// lane g owns rows g*R+1 .. g*R+R of the chunk in registers and walks the
// subject column by column, one step behind lane g-1 (the anti-diagonal
// dependency of Sec. III-A: a cell needs its left, upper and upper-left
// neighbours). The last row of lane g-1 reaches lane g by a warp shuffle; the
// first row of a chunk reads the last row of the previous chunk, which goes
// through global memory (the border stripes of Sec. IV-B/C).
//
// Values kept per row: Hoe = H + open + extend (the value a gap opened from H
// starts with; Eq. 4/5) and F. The diagonal term H(i-1,j-1) + sigma is
// Hoe(i-1,j-1) + sigma' with sigma' = sigma - open - extend stored in the row
// profile bytes, so a cell costs six integer instructions:
//   sigma' = prmt(profile, selector)            substitution (Sec. III-C)
//   E      = max(E_up + e, Hoe_up)               Eq. 4
//   F      = max(F_left + e, Hoe_left)           Eq. 5
//   H      = max(Hoe_diag + sigma', E, F [, 0])  Eq. 1 (relu = nu 0, local)
//   Hoe    = H + open + extend
//
// Rows are padded at the TOP so that the query's last row is always the last
// register of lane 15 in the last chunk. Padding rows reproduce row 0 exactly:
// local/semi-global row 0 is all zero (sigma_pad = 0, column 0 = 0); global
// row 0 is open + j*extend (sigma_pad = extend, column 0 = open except the
// last padding row, which holds H(0,0) = 0).
#pragma once
#include "common.cuh"

namespace anyseq {

// Per-group shared memory: subject selectors, top and bottom border rings of
// RG columns (four refill blocks: the one being filled, the one being
// computed, the one the last lanes still finish, the one being drained).
// Each ring has MB entries more: the score kernels keep a copy of ring block 0
// there (selectors, top) or let the last lane's stores run on past the ring's
// end (bottom), so a lane walks one refill block with constant offsets from
// one base address and never wraps.
template <int RG, int MB = 0>
struct __align__(16) GroupSmemT {
    uint32_t sel[RG + MB];
    int32_t top[2 * (RG + MB)];  // (Hoe, E) of the row above the chunk
    int32_t bot[2 * (RG + MB)];  // (Hoe, E) of the chunk's last row
};

// Column-0 value H(i, 0) of padded row with real index i (i <= 0: padding).
__device__ __forceinline__ int32_t col0(int mode, int32_t i, int32_t o, int32_t e, int32_t tb) {
    if (mode != GLOBAL) return 0;
    if (i >= 1) return tb + i * e;
    return i == 0 ? 0 : o;
}

// Description of one slot as seen by one lane.
struct Slot {
    int64_t q0[2], s0[2];   // start positions of query/subject in the packed arrays
    int32_t n[2], m[2];     // lengths (0 for an empty half)
    int32_t pad[2];         // padding rows at the top
    int32_t tb[2];          // column-0 gap open (global), usually the gap open
    bool rev[2];            // read both sequences from their ends
};

}  // namespace anyseq
