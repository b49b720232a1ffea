// C ABI of the library: context, argument validation, staging of host
// buffers, dispatch of the batched path. See include/anyseq.h.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/anyseq.h"
#include "api_internal.h"
#include "batch.h"
#include "common.cuh"

using namespace anyseq;

static thread_local char g_err[512] = "no error";

anyseq_status_t anyseq::fail(anyseq_status_t st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

extern "C" const char *anyseq_last_error(void) { return g_err; }
extern "C" const char *anyseq_version(void) { return "anyseq-gb300 0.1 (sm_103a)"; }

// ------------------------------------------------------------------ arena

void *anyseq_ctx::get(const char *name, size_t bytes, anyseq_status_t *st) {
    for (auto &b : bufs) {
        if (b.name == name) {
            if (b.cap >= bytes) return b.p;
            cudaFree(b.p);
            used -= b.cap;
            b.p = nullptr;
            b.cap = 0;
            size_t want = bytes + bytes / 4;
            if (used + want > budget) want = bytes;
            if (used + want > budget) {
                *st = fail(ANYSEQ_ERR_BUDGET, "scratch '%s' of %zu bytes exceeds the memory budget (%zu of %zu used)",
                           name, bytes, used, budget);
                return nullptr;
            }
            if (cudaMalloc(&b.p, want) != cudaSuccess) {
                cudaGetLastError();
                *st = fail(ANYSEQ_ERR_BUDGET, "cudaMalloc of %zu bytes for '%s' failed", want, name);
                return nullptr;
            }
            b.cap = want;
            used += want;
            return b.p;
        }
    }
    bufs.push_back(Buf{name, nullptr, 0});
    return get(name, bytes, st);
}

extern "C" anyseq_status_t anyseq_create(anyseq_ctx **ctx, int device, size_t mem_budget_bytes) {
    if (!ctx) return fail(ANYSEQ_ERR_ARG, "ctx is NULL");
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(ANYSEQ_ERR_CUDA, "CUDA device %d not available", device);
    }
    if (cudaSetDevice(device) != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    anyseq_ctx *c = new anyseq_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)(fr * 0.9);
    *ctx = c;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_destroy(anyseq_ctx *ctx) {
    if (!ctx) return ANYSEQ_OK;
    cudaSetDevice(ctx->device);
    for (auto &b : ctx->bufs) cudaFree(b.p);
    for (auto &h : ctx->pinned) cudaFreeHost(h.p);
    for (auto &e : ctx->ev) if (e) cudaEventDestroy(e);
    delete ctx;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_set_option(anyseq_ctx *ctx, const char *key, int64_t value) {
    if (!ctx || !key) return fail(ANYSEQ_ERR_ARG, "ctx or key is NULL");
    if (!strcmp(key, "force_int32")) { ctx->force32 = value != 0; return ANYSEQ_OK; }
    if (!strcmp(key, "profile")) {
        ctx->profile = value != 0;
        if (ctx->profile && !ctx->ev[0])
            for (auto &e : ctx->ev) cudaEventCreate(&e);
        return ANYSEQ_OK;
    }
    return fail(ANYSEQ_ERR_ARG, "unknown option '%s'", key);
}

extern "C" anyseq_status_t anyseq_get_stat(anyseq_ctx *ctx, const char *key, double *value) {
    if (!ctx || !key || !value) return fail(ANYSEQ_ERR_ARG, "ctx, key or value is NULL");
    if (!strcmp(key, "launches")) *value = (double)ctx->launches;
    else if (!strcmp(key, "dp_ms")) *value = ctx->dp_ms;
    else if (!strcmp(key, "dp32_ms")) *value = ctx->dp32_ms;
    else if (!strcmp(key, "pairs16")) *value = (double)ctx->pairs16;
    else if (!strcmp(key, "pairs32")) *value = (double)ctx->pairs32;
    else return fail(ANYSEQ_ERR_ARG, "unknown statistic '%s'", key);
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_encode_dna(const char *ascii, uint8_t *codes, int64_t len) {
    if (len < 0 || (len > 0 && (!ascii || !codes))) return fail(ANYSEQ_ERR_ARG, "bad arguments");
    for (int64_t k = 0; k < len; k++) {
        switch (ascii[k]) {
            case 'A': case 'a': codes[k] = 0; break;
            case 'C': case 'c': codes[k] = 1; break;
            case 'G': case 'g': codes[k] = 2; break;
            case 'T': case 't': codes[k] = 3; break;
            default: return fail(ANYSEQ_ERR_ALPHABET, "letter %d at position %lld is not A/C/G/T", (int)(unsigned char)ascii[k], (long long)k);
        }
    }
    return ANYSEQ_OK;
}

// ---------------------------------------------------------------- helpers

bool anyseq::is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

anyseq_status_t anyseq::check_scoring(const anyseq_scoring_t *sc, int32_t mode) {
    if (!sc) return fail(ANYSEQ_ERR_ARG, "scoring is NULL");
    if (mode < 0 || mode > 2) return fail(ANYSEQ_ERR_ARG, "unknown mode %d", mode);
    if (sc->alphabet < 1 || sc->alphabet > 32) return fail(ANYSEQ_ERR_ARG, "alphabet %d outside 1..32", sc->alphabet);
    if (sc->gap_open > 0 || sc->gap_extend > 0)
        return fail(ANYSEQ_ERR_ARG, "gap open/extend must be <= 0 (signed scores), got %d/%d", sc->gap_open, sc->gap_extend);
    if (sc->gap_open < -(1 << 20) || sc->gap_extend < -(1 << 20)) return fail(ANYSEQ_ERR_ARG, "gap scores too large");
    if (!sc->matrix && (sc->match > (1 << 20) || sc->mismatch < -(1 << 20)))
        return fail(ANYSEQ_ERR_ARG, "match/mismatch too large");
    return ANYSEQ_OK;
}

int32_t anyseq::sigma_host(const anyseq_scoring_t *sc, int a, int b) {
    if (sc->matrix) return sc->matrix[a * sc->alphabet + b];
    return a == b ? sc->match : sc->mismatch;
}

// Row-profile words: byte c of word q is sigma(q, c) - open - extend; word 4
// is the padding row (sigma = extend for global, 0 otherwise).
anyseq_status_t anyseq::make_rowprof(const anyseq_scoring_t *sc, int32_t mode, uint32_t prof[5]) {
    const int32_t oe = sc->gap_open + sc->gap_extend;
    for (int a = 0; a < 5; a++) {
        uint32_t w = 0;
        for (int b = 0; b < 4; b++) {
            int32_t sg;
            if (a < 4) sg = (a < sc->alphabet && b < sc->alphabet) ? sigma_host(sc, a, b) : 0;
            else sg = mode == ANYSEQ_GLOBAL ? sc->gap_extend : 0;
            int32_t v = sg - oe;
            if (v < -128 || v > 127)
                return fail(ANYSEQ_ERR_ARG, "sigma - open - extend = %d does not fit the int8 row profile", v);
            w |= (uint32_t)(uint8_t)(int8_t)v << (8 * b);
        }
        prof[a] = w;
    }
    return ANYSEQ_OK;
}

__global__ void len_stats_kernel(const int64_t *q_off, const int64_t *s_off, int64_t n_pairs, int64_t *stats) {
    // stats: [0] max n, [1] max m, [2] bad-offset flag; one atomic per block
    __shared__ unsigned long long red[3][32];
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long mn = 0, mm = 0, bad = 0;
    for (; p < n_pairs; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t n = q_off[p + 1] - q_off[p], m = s_off[p + 1] - s_off[p];
        if (n < 0 || m < 0 || n >= (1 << 21) || m >= (1 << 21)) bad = 1;
        if (n > (int64_t)mn) mn = (unsigned long long)n;
        if (m > (int64_t)mm) mm = (unsigned long long)m;
    }
    for (int off = 16; off; off >>= 1) {
        mn = max(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        mm = max(mm, __shfl_xor_sync(0xffffffffu, mm, off));
        bad |= __shfl_xor_sync(0xffffffffu, bad, off);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { red[0][w] = mn; red[1][w] = mm; red[2][w] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; k++) { mn = max(mn, red[0][k]); mm = max(mm, red[1][k]); bad |= red[2][k]; }
        if (bad) atomicOr(reinterpret_cast<unsigned long long *>(&stats[2]), 1ull);
        atomicMax(reinterpret_cast<unsigned long long *>(&stats[0]), mn);
        atomicMax(reinterpret_cast<unsigned long long *>(&stats[1]), mm);
    }
}

__global__ void write_results_kernel(int64_t n, const int32_t *score, const int32_t *eq, const int32_t *es,
                                     const uint32_t *flags, anyseq_result_t *out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        anyseq_result_t r;
        r.score = score[p];
        r.beg_q = -1;
        r.beg_s = -1;
        r.end_q = eq[p];
        r.end_s = es[p];
        r.flags = flags[p];
        r.cigar_off = 0;
        r.cigar_len = 0;
        r.reserved = 0;
        out[p] = r;
    }
}

static int grid_for(int64_t work) {
    int64_t b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

// --------------------------------------------------------------- batch path

anyseq_status_t anyseq::stage_input(anyseq_ctx *ctx, const char *name, const void *src, size_t bytes,
                                    cudaStream_t st, const void **dev) {
    if (bytes == 0) {
        anyseq_status_t s2 = ANYSEQ_OK;
        *dev = ctx->get(name, 16, &s2);
        return s2;
    }
    if (is_device_ptr(src)) {
        *dev = src;
        return ANYSEQ_OK;
    }
    anyseq_status_t s2 = ANYSEQ_OK;
    void *d = ctx->get(name, bytes, &s2);
    if (!d) return s2;
    if (cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(ANYSEQ_ERR_CUDA, "copy of %s to the device failed: %s", name, cudaGetErrorString(cudaGetLastError()));
    *dev = d;
    return ANYSEQ_OK;
}

#define TRY(x)                              \
    do {                                    \
        anyseq_status_t _s = (x);           \
        if (_s != ANYSEQ_OK) return _s;     \
    } while (0)
#define CUDA_TRY(x)                                                                             \
    do {                                                                                        \
        cudaError_t _e = (x);                                                                   \
        if (_e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(_e)); \
    } while (0)

template <class T>
static T *arena(anyseq_ctx *ctx, const char *name, size_t count, anyseq_status_t *st) {
    return static_cast<T *>(ctx->get(name, count * sizeof(T) + 16, st));
}

anyseq_status_t anyseq::batch_scores(anyseq_ctx *ctx, const BatchInput &in, const anyseq_scoring_t *sc, int32_t mode,
                                     int32_t *score, int32_t *eq, int32_t *es, uint32_t *flags, cudaStream_t st) {
    anyseq_status_t s2 = ANYSEQ_OK;
    const int64_t n = in.n_pairs;
    if (sc->alphabet > 4) return fail(ANYSEQ_ERR_ARG, "alphabets above 4 letters need the profile path (not built)");
    PrepArgs P;
    memset(&P, 0, sizeof(P));
    P.q = in.q; P.s = in.s; P.q_off = in.q_off; P.s_off = in.s_off;
    P.n_pairs = n; P.q_len = in.q_len; P.s_len = in.s_len;
    P.alphabet = sc->alphabet;
    P.q2 = arena<uint32_t>(ctx, "q2", (in.q_len + 15) / 16 + 2, &s2);
    P.s2 = arena<uint32_t>(ctx, "s2", (in.s_len + 15) / 16 + 2, &s2);
    P.bad_code = arena<int32_t>(ctx, "bad", 4, &s2);
    P.hist = arena<uint32_t>(ctx, "hist", 2 * 65536, &s2);
    P.tile_sum = arena<uint32_t>(ctx, "tile_sum", 256, &s2);
    P.key = arena<uint32_t>(ctx, "key", n + 1, &s2);
    P.list16 = arena<int32_t>(ctx, "list16", n + 1, &s2);
    P.list32 = arena<int32_t>(ctx, "list32", n + 1, &s2);
    P.counts = arena<int64_t>(ctx, "counts", 4, &s2);
    P.trivial = nullptr;
    if (s2 != ANYSEQ_OK) return s2;
    int32_t smax = -(1 << 30), smin = 1 << 30;
    for (int a = 0; a < sc->alphabet; a++)
        for (int b = 0; b < sc->alphabet; b++) {
            int32_t v = sigma_host(sc, a, b);
            smax = v > smax ? v : smax;
            smin = v < smin ? v : smin;
        }
    P.smax = smax; P.smin = smin; P.o = sc->gap_open; P.e = sc->gap_extend; P.mode = mode;
    P.score = score; P.end_q = eq; P.end_s = es; P.flags = flags;
    P.force32 = ctx->force32;
    CUDA_TRY(launch_prep(P, st));
    ctx->launches += 6;  // pack/validate x2, bin, tile sums, tile scan, scatter

    BatchArgs A;
    memset(&A, 0, sizeof(A));
    A.q2 = P.q2; A.s2 = P.s2; A.q_off = in.q_off; A.s_off = in.s_off;
    TRY(make_rowprof(sc, mode, A.rowprof));
    A.o = sc->gap_open; A.e = sc->gap_extend;
    A.score = score; A.end_q = eq; A.end_s = es; A.flags = flags;
    A.counter = arena<int32_t>(ctx, "counter", 4, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    for (int cell32 = 0; cell32 < 2; cell32++) {
        int bps = batch_blocks_per_sm(cell32, mode);
        int grid = ctx->num_sms * bps;
        A.list = cell32 ? P.list32 : P.list16;
        A.n_list = P.counts + cell32;
        A.scratch = nullptr;
        A.scratch_cols = 0;
        if (in.max_n > 256) {
            A.scratch_cols = in.max_m + 1;
            A.scratch = arena<int32_t>(ctx, "border", (size_t)grid * 16 * 2 * (size_t)A.scratch_cols, &s2);
            if (s2 != ANYSEQ_OK) return s2;
        }
        CUDA_TRY(cudaMemsetAsync(A.counter, 0, sizeof(int32_t), st));
        if (ctx->profile) cudaEventRecord(ctx->ev[2 * cell32], st);
        CUDA_TRY(launch_batch(A, cell32, mode, grid, st));
        if (ctx->profile) cudaEventRecord(ctx->ev[2 * cell32 + 1], st);
        ctx->launches += 1;
    }
    // letter check (read after the kernels; an invalid code only affects its own scores)
    int32_t bad = 0;
    int64_t hc[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(&bad, P.bad_code, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hc, P.counts, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    ctx->pairs16 = hc[0];
    ctx->pairs32 = hc[1];
    if (ctx->profile) {
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]);
        cudaEventElapsedTime(&b, ctx->ev[2], ctx->ev[3]);
        ctx->dp_ms = a;
        ctx->dp32_ms = b;
    }
    if (bad) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", sc->alphabet);
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_align_batch(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off,
                                              const uint8_t *s, const int64_t *s_off, int64_t n_pairs,
                                              const anyseq_scoring_t *sc, int32_t mode, uint32_t want,
                                              anyseq_result_t *out, uint32_t *cigar, uint64_t cigar_cap,
                                              uint64_t *cigar_used, void *cuda_stream) {
    if (!ctx) return fail(ANYSEQ_ERR_ARG, "ctx is NULL");
    if (n_pairs < 0) return fail(ANYSEQ_ERR_ARG, "n_pairs < 0");
    if (n_pairs == 0) { if (cigar_used) *cigar_used = 0; return ANYSEQ_OK; }
    if (!q_off || !s_off || !out) return fail(ANYSEQ_ERR_ARG, "q_off, s_off and out must not be NULL");
    if (n_pairs >= (1ll << 31) - 2) return fail(ANYSEQ_ERR_ARG, "n_pairs too large");
    TRY(check_scoring(sc, mode));
    if (want & ANYSEQ_WANT_CIGAR) return fail(ANYSEQ_ERR_ARG, "CIGAR output of the batch path is not built");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "cudaSetDevice failed");
    anyseq_status_t s2 = ANYSEQ_OK;

    // offsets: stage, then read totals and maxima
    ctx->launches = 0;
    BatchInput in;
    in.n_pairs = n_pairs;
    const void *dq_off, *ds_off;
    TRY(stage_input(ctx, "in_qoff", q_off, (n_pairs + 1) * sizeof(int64_t), st, &dq_off));
    TRY(stage_input(ctx, "in_soff", s_off, (n_pairs + 1) * sizeof(int64_t), st, &ds_off));
    in.q_off = (const int64_t *)dq_off;
    in.s_off = (const int64_t *)ds_off;
    int64_t *stats = arena<int64_t>(ctx, "stats", 8, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    int64_t hstats[5];
    CUDA_TRY(cudaMemsetAsync(stats, 0, 3 * sizeof(int64_t), st));
    len_stats_kernel<<<grid_for(n_pairs) > 304 ? 304 : grid_for(n_pairs), 256, 0, st>>>(in.q_off, in.s_off, n_pairs, stats);
    CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    CUDA_TRY(cudaMemcpyAsync(hstats, stats, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&hstats[3], in.q_off + n_pairs, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&hstats[4], in.s_off + n_pairs, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    int64_t q0 = 0, s0 = 0;
    CUDA_TRY(cudaMemcpyAsync(&q0, in.q_off, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&s0, in.s_off, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hstats[2] || q0 != 0 || s0 != 0)
        return fail(ANYSEQ_ERR_ARG, "offsets must start at 0, be non-decreasing and give lengths below 2^21");
    in.max_n = hstats[0];
    in.max_m = hstats[1];
    in.q_len = hstats[3];
    in.s_len = hstats[4];
    if ((in.q_len > 0 && !q) || (in.s_len > 0 && !s)) return fail(ANYSEQ_ERR_ARG, "q or s is NULL");
    const void *dq, *ds;
    TRY(stage_input(ctx, "in_q", q, (size_t)in.q_len, st, &dq));
    TRY(stage_input(ctx, "in_s", s, (size_t)in.s_len, st, &ds));
    in.q = (const uint8_t *)dq;
    in.s = (const uint8_t *)ds;

    int32_t *score = arena<int32_t>(ctx, "r_score", n_pairs, &s2);
    int32_t *eq = arena<int32_t>(ctx, "r_eq", n_pairs, &s2);
    int32_t *es = arena<int32_t>(ctx, "r_es", n_pairs, &s2);
    uint32_t *flags = arena<uint32_t>(ctx, "r_flags", n_pairs, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    TRY(batch_scores(ctx, in, sc, mode, score, eq, es, flags, st));

    bool out_dev = is_device_ptr(out);
    anyseq_result_t *dout = out;
    if (!out_dev) {
        dout = arena<anyseq_result_t>(ctx, "r_out", n_pairs, &s2);
        if (s2 != ANYSEQ_OK) return s2;
    }
    write_results_kernel<<<grid_for(n_pairs), 256, 0, st>>>(n_pairs, score, eq, es, flags, dout);
    CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    if (!out_dev) {
        CUDA_TRY(cudaMemcpyAsync(out, dout, n_pairs * sizeof(anyseq_result_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (cigar_used) *cigar_used = 0;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_align_long(anyseq_ctx *ctx, const uint8_t *q, int64_t n, const uint8_t *s,
                                             int64_t m, const anyseq_scoring_t *sc, int32_t mode, uint32_t want,
                                             anyseq_result_t *out, uint32_t *cigar, uint64_t cigar_cap,
                                             uint64_t *cigar_used, void *cuda_stream) {
    (void)ctx; (void)q; (void)n; (void)s; (void)m; (void)sc; (void)mode; (void)want; (void)out;
    (void)cigar; (void)cigar_cap; (void)cigar_used; (void)cuda_stream;
    return fail(ANYSEQ_ERR_ARG, "the long-pair path is not built");
}
