// Shared device helpers of the alignment kernels: score lanes (int32 or two
// int16 halves), byte permutes for substitution scores, 2-bit sequence access.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace anyseq {

constexpr int GROUP = 16;        // lanes cooperating on one slot (one row chunk)
constexpr int RING = 128;        // columns held by the per-group shared-memory rings
constexpr int BLOCK = 32;        // ring refill / flush granularity in columns

// Minus infinity of the recurrences (Sec. III-A). Far enough from the
// representable minimum that adding one gap extension cannot wrap, and below
// every real value allowed by the range tests of the host.
constexpr int32_t NEG32 = -(1 << 29);
constexpr int32_t NEG16 = -20000;

enum Mode { GLOBAL = 0, LOCAL = 1, SEMIGLOBAL = 2 };

// prmt.b32 in its default mode: selector nibbles 8..15 replicate the sign
// bit of the selected byte, which turns an int8 into an int16/int32.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Score lanes. Both traits keep the same six-step cell (see engine.cuh) and
// split it between the two integer pipes of the SM: the additions of a
// constant go to full-rate 32-bit IADD, the maxima to the half-rate DPX/VIMNMX
// instructions (measured on sm_103: every max-type integer instruction issues
// at 64 lanes per clock per SM, IADD at 128).

// One signed 32-bit lane per pair.
struct CellI32 {
    typedef int32_t T;
    static constexpr int PAIRS = 1;
    static constexpr int32_t NEG = NEG32;
    __device__ __forceinline__ static T make(int32_t lo, int32_t hi) { (void)hi; return lo; }
    __device__ __forceinline__ static int32_t get(T v, int h) { (void)h; return v; }
    // packed constant for addc (a plain signed 32-bit value here)
    __host__ __device__ __forceinline__ static uint32_t cst(int32_t c) { return (uint32_t)c; }
    __device__ __forceinline__ static T addc(T a, uint32_t c) { return a + (int32_t)c; }
    // raw per-lane constant for addmax
    __device__ __forceinline__ static uint32_t raw(int32_t c) { return (uint32_t)c; }
    __device__ __forceinline__ static T addmax(T a, uint32_t b, T c) { return __viaddmax_s32(a, (int32_t)b, c); }
    __device__ __forceinline__ static T vmax(T a, T b) { return max(a, b); }
    // row maximum with the first column of a strict improvement (j0: the column):
    // keep the column unless v > mx
    __device__ __forceinline__ static void track(T &mx, uint32_t &j0, uint32_t &, T v, uint32_t j) {
        asm("{ .reg .pred k;\n\t"
            "setp.ge.s32 k, %0, %2;\n\t"
            "max.s32 %0, %0, %2;\n\t"
            "selp.b32 %1, %1, %3, k; }"
            : "+r"(mx), "+r"(j0) : "r"(v), "r"(j));
    }
    __device__ __forceinline__ static T maxrelu(T a, T b) { return __vimax_s32_relu(a, b); }
    __device__ __forceinline__ static T vmax3(T a, T b, T c) { return __vimax3_s32(a, b, c); }
    // sigma' >= 0 from a row profile word (4 bytes indexed by subject letter)
    __device__ __forceinline__ static T sigma(uint32_t pa, uint32_t pb, uint32_t sel) {
        (void)pb; return (int32_t)prmt(pa, pa, sel);
    }
    __device__ __forceinline__ static uint32_t selector(uint32_t ca, uint32_t cb) {
        (void)cb;
        uint32_t sgn = ca | 8u;
        return ca | (sgn << 4) | (sgn << 8) | (sgn << 12);
    }
    __device__ __forceinline__ static uint32_t as_u(T v) { return (uint32_t)v; }
    __device__ __forceinline__ static T from_u(uint32_t v) { return (int32_t)v; }
    // flag word: bit 31 set iff a >= b (sign of b - a - 1; |a - b| < 2^31)
    __device__ __forceinline__ static uint32_t ge(T a, T b) { return (uint32_t)(b - a - 1); }
    __device__ __forceinline__ static uint32_t flag_mask() { return 0x80000000u; }
    // selector of a column past the end of the pair: the sign byte of profile byte 0
    // in all four bytes (sigma' = 0 or -1)
    __device__ __forceinline__ static uint32_t null_past_end(uint32_t sel, bool va, bool vb) {
        (void)vb; return va ? sel : 0x8888u;
    }
};

// Two int16 halves per 32-bit word (low: pair A, high: pair B), each stored
// with a bias of 2^15 as an unsigned 16-bit number. With every value inside
// [-32768, 32767] a 32-bit IADD of a packed constant never carries or borrows
// across the halves, so constant additions run on the full-rate adder while
// the unsigned per-half maxima use VIMNMX/DPX.
struct CellI16x2 {
    typedef uint32_t T;
    static constexpr int PAIRS = 2;
    static constexpr int32_t NEG = NEG16;
    __device__ __forceinline__ static T make(int32_t lo, int32_t hi) {
        return ((uint32_t)(lo + 32768) & 0xFFFFu) | (((uint32_t)(hi + 32768) & 0xFFFFu) << 16);
    }
    __device__ __forceinline__ static int32_t get(T v, int h) { return (int32_t)((v >> (16 * h)) & 0xFFFFu) - 32768; }
    __host__ __device__ __forceinline__ static uint32_t cst(int32_t c) { return (uint32_t)(c * 65537); }
    __device__ __forceinline__ static T addc(T a, uint32_t c) { return a + c; }
    __device__ __forceinline__ static uint32_t raw(int32_t c) { return ((uint32_t)c & 0xFFFFu) * 65537u; }
    __device__ __forceinline__ static T addmax(T a, uint32_t b, T c) { return __viaddmax_u16x2(a, b, c); }
    __device__ __forceinline__ static T vmax(T a, T b) { return __vmaxu2(a, b); }
    // row maxima of both halves with the first column of a strict improvement
    // (j0: low half, j1: high half): a packed maximum, a per-half test that it
    // kept the old value, and a select per half. Written out in PTX with the
    // old maximum unpacked before it is overwritten (a read-write operand), so
    // no register assignment can make the test compare the new maximum with
    // itself.
    __device__ __forceinline__ static void track(T &mx, uint32_t &j0, uint32_t &j1, T v, uint32_t j) {
        asm("{ .reg .pred kl, kh;\n\t"
            ".reg .u16 a0, a1, m0, m1;\n\t"
            "mov.b32 {a0, a1}, %0;\n\t"
            "max.u16x2 %0, %0, %3;\n\t"
            "mov.b32 {m0, m1}, %0;\n\t"
            "setp.eq.u16 kl, m0, a0;\n\t"
            "setp.eq.u16 kh, m1, a1;\n\t"
            "selp.b32 %1, %1, %4, kl;\n\t"
            "selp.b32 %2, %2, %4, kh; }"
            : "+r"(mx), "+r"(j0), "+r"(j1) : "r"(v), "r"(j));
    }
    __device__ __forceinline__ static T maxrelu(T a, T b) { return __vimax3_u16x2(a, b, 0x80008000u); }
    __device__ __forceinline__ static T vmax3(T a, T b, T c) { return __vimax3_u16x2(a, b, c); }
    __device__ __forceinline__ static T sigma(uint32_t pa, uint32_t pb, uint32_t sel) { return prmt(pa, pb, sel); }
    // low half: byte ca of pa, high half: byte cb of pb; bytes are >= 0 so the
    // sign replication fills zeros
    __device__ __forceinline__ static uint32_t selector(uint32_t ca, uint32_t cb) {
        uint32_t b4 = cb + 4u;
        return ca | ((ca | 8u) << 4) | (b4 << 8) | ((b4 | 8u) << 12);
    }
    __device__ __forceinline__ static uint32_t as_u(T v) { return v; }
    __device__ __forceinline__ static T from_u(uint32_t v) { return v; }
    // flag word: bit 15 (low half) / 31 (high half) set iff a >= b; one full-rate
    // add because a - b + 2^15 stays inside [0, 2^16) when |a - b| < 2^15
    __device__ __forceinline__ static uint32_t ge(T a, T b) { return a + 0x80008000u - b; }
    __device__ __forceinline__ static uint32_t flag_mask() { return 0x80008000u; }
    // selector nibbles 8 of a half past the end of its pair: the sign of profile
    // byte 0, which is >= 0, in both bytes (sigma' = 0)
    __device__ __forceinline__ static uint32_t null_past_end(uint32_t sel, bool va, bool vb) {
        return (va ? (sel & 0x00FFu) : 0x0088u) | (vb ? (sel & 0xFF00u) : 0x8800u);
    }
};

// Letter at global position k of a 2-bit packed array (16 letters per word).
__device__ __forceinline__ uint32_t code2(const uint32_t *packed, int64_t k) {
    return (packed[k >> 4] >> (2 * (k & 15))) & 3u;
}

// 16 consecutive letters starting at global position k, as one 32-bit word
// (letter t in bits 2t..2t+1). Reads two words and funnel-shifts.
__device__ __forceinline__ uint32_t codes16(const uint32_t *packed, int64_t k, int64_t limit_words) {
    int64_t w = k >> 4;
    uint32_t lo = packed[w];
    uint32_t hi = (w + 1 < limit_words) ? packed[w + 1] : 0u;
    return __funnelshift_r(lo, hi, 2 * (uint32_t)(k & 15));
}

// Lexicographic key of an optimum candidate: larger score, then smaller i,
// then smaller j wins (the tie rule of the optimum cell). Fields: score + 2^21
// in 22 bits, 2^21 - 1 - i and 2^21 - 1 - j in 21 bits each. A score below -1
// is stored as -1: every search starts from a candidate of score 0 (the empty
// alignment) or looks for a positive optimum, so such a candidate never wins,
// and the clamp keeps it inside its field. Callers keep scores below 2^21
// (key_range_ok on the host).
__host__ __device__ __forceinline__ uint64_t end_key(int32_t score, int32_t i, int32_t j) {
    score = score < -1 ? -1 : score;
    return ((uint64_t)(uint32_t)(score + (1 << 21)) << 42) |
           ((uint64_t)(uint32_t)((1 << 21) - 1 - i) << 21) |
           (uint64_t)(uint32_t)((1 << 21) - 1 - j);
}
__host__ __device__ __forceinline__ int32_t key_score(uint64_t k) { return (int32_t)(k >> 42) - (1 << 21); }
__host__ __device__ __forceinline__ int32_t key_i(uint64_t k) { return (1 << 21) - 1 - (int32_t)((k >> 21) & 0x1FFFFF); }
__host__ __device__ __forceinline__ int32_t key_j(uint64_t k) { return (1 << 21) - 1 - (int32_t)(k & 0x1FFFFF); }

}  // namespace anyseq
