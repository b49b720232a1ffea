// C ABI of the library: context, argument validation, staging of host
// buffers, dispatch of the batched path. See include/anyseq.h.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/anyseq.h"
#include "api_internal.h"
#include "batch.h"
#include "common.cuh"
#include "scan.h"
#include "tb.h"
#include "wave.h"

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
            // The old buffer may still be read by this context's queued work, and
            // cudaFree would wait for every stream of the device (another context's
            // long kernel included), so it is retired rather than freed; the retired
            // buffers are freed when the budget needs their room, and at destroy.
            if (b.p) retired.push_back(b);
            b.p = nullptr;
            b.cap = 0;
            size_t want = bytes + bytes / 2;
            if (used + want > budget) want = bytes;
            if (used + want > budget && !retired.empty()) {
                for (auto &r : retired) {
                    cudaFree(r.p);
                    used -= r.cap;
                }
                retired.clear();
                want = bytes + bytes / 2;
                if (used + want > budget) want = bytes;
            }
            if (used + want > budget) {
                *st = fail(ANYSEQ_ERR_BUDGET, "scratch '%s' of %zu bytes exceeds the memory budget (%zu of %zu used)",
                           name, bytes, used, budget);
                return nullptr;
            }
            if (cudaMalloc(&b.p, want) != cudaSuccess) {
                cudaGetLastError();
                b.p = nullptr;
                // the device is full: give back the retired buffers and try once more
                for (auto &r : retired) {
                    cudaFree(r.p);
                    used -= r.cap;
                }
                const bool had_retired = !retired.empty();
                retired.clear();
                if (!had_retired || cudaMalloc(&b.p, want) != cudaSuccess) {
                    cudaGetLastError();
                    b.p = nullptr;
                    *st = fail(ANYSEQ_ERR_BUDGET, "cudaMalloc of %zu bytes for '%s' failed", want, name);
                    return nullptr;
                }
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
    for (auto &b : ctx->retired) cudaFree(b.p);
    for (auto &h : ctx->pinned) cudaFreeHost(h.p);
    for (auto &e : ctx->ev) if (e) cudaEventDestroy(e);
    if (ctx->mlp) cudaFree(ctx->mlp);
    delete ctx;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_set_option(anyseq_ctx *ctx, const char *key, int64_t value) {
    if (!ctx || !key) return fail(ANYSEQ_ERR_ARG, "ctx or key is NULL");
    if (!strcmp(key, "force_int32")) { ctx->force32 = value != 0; return ANYSEQ_OK; }
    if (!strcmp(key, "force_matrix_path")) { ctx->force_matrix = value != 0; return ANYSEQ_OK; }
    if (!strcmp(key, "hirschberg_base_cells")) {
        if (value < 1) return fail(ANYSEQ_ERR_ARG, "hirschberg_base_cells must be >= 1");
        ctx->base_cells = value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "band_max_doublings")) {
        if (value < 0 || value > 16) return fail(ANYSEQ_ERR_ARG, "band_max_doublings must be in 0..16");
        ctx->band_max_doublings = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "band_area_pct")) {
        if (value < 1 || value > 100) return fail(ANYSEQ_ERR_ARG, "band_area_pct must be in 1..100");
        ctx->band_area_pct = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "band_margin_pct")) {
        if (value < 50 || value > 1000) return fail(ANYSEQ_ERR_ARG, "band_margin_pct must be in 50..1000");
        ctx->band_margin_pct = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "band_floor_pct")) {
        if (value < 0 || value > 100) return fail(ANYSEQ_ERR_ARG, "band_floor_pct must be in 0..100");
        ctx->band_floor_pct = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "band_area16_pct")) {
        if (value < 1 || value > 100) return fail(ANYSEQ_ERR_ARG, "band_area16_pct must be in 1..100");
        ctx->band_area16_pct = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "tb_walker")) {
        if (value < 0 || value > 2) return fail(ANYSEQ_ERR_ARG, "tb_walker must be 0, 1 or 2");
        ctx->tb_walker = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "wave_split")) {
        if (value < 0 || value > 2) return fail(ANYSEQ_ERR_ARG, "wave_split must be 0, 1 or 2");
        ctx->wave_split = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "host_in_place")) {
        if (value != 0 && value != 1) return fail(ANYSEQ_ERR_ARG, "host_in_place must be 0 or 1");
        ctx->host_in_place = (int)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "wave_spread")) {
        if (value != 0 && value != 1) return fail(ANYSEQ_ERR_ARG, "wave_spread must be 0 or 1");
        ctx->wave_spread = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "batch_ctas_per_sm")) {
        if (value < 0 || value > 16) return fail(ANYSEQ_ERR_ARG, "batch_ctas_per_sm must be in 0..16");
        ctx->batch_ctas_per_sm = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "wave_ctas_per_sm")) {
        if (value < 0 || value > 8) return fail(ANYSEQ_ERR_ARG, "wave_ctas_per_sm must be in 0..8");
        ctx->wave_ctas_per_sm = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "wave_rows")) {
        if (value != 0 && value != 4 && value != 8 && value != 16)
            return fail(ANYSEQ_ERR_ARG, "wave_rows must be 0, 4, 8 or 16");
        ctx->wave_rows = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "wave_cell")) {
        if (value < 0 || value > 2) return fail(ANYSEQ_ERR_ARG, "wave_cell must be 0, 1 or 2");
        ctx->wave_cell = (int32_t)value;
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "autotune_reset")) {
        ctx->tuned = false;
        ctx->tune_gain = 1.0;
        memset(ctx->tune_tab, 0, sizeof(ctx->tune_tab));
        return ANYSEQ_OK;
    }
    if (!strcmp(key, "spin_limit")) {
        if (value < 1) return fail(ANYSEQ_ERR_ARG, "spin_limit must be >= 1");
        ctx->spin_limit = value;
        return ANYSEQ_OK;
    }
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
    else if (!strcmp(key, "band_cells")) *value = (double)ctx->band_cells;
    else if (!strcmp(key, "band_accepted")) *value = (double)ctx->band_accepted;
    else if (!strcmp(key, "band_fallback")) *value = (double)ctx->band_fallback;
    else if (!strcmp(key, "band_rounds")) *value = (double)ctx->band_rounds;
    else if (!strcmp(key, "tuned_bins")) {
        int64_t k = 0;
        for (int b = 0; b < 256; b++) k += ctx->tuned && ctx->tune_tab[b] != 0;
        *value = (double)k;
    }
    else if (!strcmp(key, "autotune_gain")) *value = ctx->tune_gain;
    else if (!strcmp(key, "band_plan_ms")) *value = ctx->band_plan_ms;
    else if (!strcmp(key, "band_pass_ms")) *value = ctx->band_pass_ms;
    else if (!strcmp(key, "band_full_ms")) *value = ctx->band_full_ms;
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
            int32_t v = sg - oe;  // range checked by the caller
            w |= (uint32_t)(uint8_t)(int8_t)v << (8 * b);
        }
        prof[a] = w;
    }
    return ANYSEQ_OK;
}

__global__ void len_stats_kernel(const int64_t *q_off, const int64_t *s_off, int64_t n_pairs, int64_t *stats) {
    // stats: [0] max n, [1] max m, [2] bad-offset flag, [3] max of min(n, m);
    // one atomic per block and value
    __shared__ unsigned long long red[4][32];
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long mn = 0, mm = 0, bad = 0, mmin = 0;
    for (; p < n_pairs; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t n = q_off[p + 1] - q_off[p], m = s_off[p + 1] - s_off[p];
        if (n < 0 || m < 0 || n >= (1 << 21) || m >= (1 << 21)) bad = 1;
        if (n > (int64_t)mn) mn = (unsigned long long)n;
        if (m > (int64_t)mm) mm = (unsigned long long)m;
        const int64_t lo = n < m ? n : m;
        if (lo > (int64_t)mmin) mmin = (unsigned long long)lo;
    }
    for (int off = 16; off; off >>= 1) {
        mn = max(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        mm = max(mm, __shfl_xor_sync(0xffffffffu, mm, off));
        mmin = max(mmin, __shfl_xor_sync(0xffffffffu, mmin, off));
        bad |= __shfl_xor_sync(0xffffffffu, bad, off);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { red[0][w] = mn; red[1][w] = mm; red[2][w] = bad; red[3][w] = mmin; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; k++) {
            mn = max(mn, red[0][k]); mm = max(mm, red[1][k]); bad |= red[2][k]; mmin = max(mmin, red[3][k]);
        }
        if (bad) atomicOr(reinterpret_cast<unsigned long long *>(&stats[2]), 1ull);
        atomicMax(reinterpret_cast<unsigned long long *>(&stats[0]), mn);
        atomicMax(reinterpret_cast<unsigned long long *>(&stats[1]), mm);
        atomicMax(reinterpret_cast<unsigned long long *>(&stats[3]), mmin);
    }
}

__global__ void write_results_kernel(int64_t n, const int32_t *score, const int32_t *eq, const int32_t *es,
                                     const uint32_t *flags, const int32_t *bq, const int32_t *bs,
                                     const int64_t *coff, const int64_t *clen, anyseq_result_t *out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        anyseq_result_t r;
        r.score = score[p];
        r.beg_q = bq ? bq[p] : -1;
        r.beg_s = bs ? bs[p] : -1;
        r.end_q = eq[p];
        r.end_s = es[p];
        r.flags = flags[p];
        r.cigar_off = coff ? (uint64_t)coff[p] : 0;
        r.cigar_len = clen ? (uint32_t)clen[p] : 0;
        r.reserved = 0;
        out[p] = r;
    }
}

static int grid_for(int64_t work) {
    int64_t b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

cudaError_t anyseq::launch_write_results(int64_t n, const int32_t *score, const int32_t *eq, const int32_t *es,
                                         const uint32_t *flags, anyseq_result_t *out, cudaStream_t st) {
    write_results_kernel<<<grid_for(n), 256, 0, st>>>(n, score, eq, es, flags, nullptr, nullptr, nullptr, nullptr, out);
    return cudaGetLastError();
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
                                     int32_t *score, int32_t *eq, int32_t *es, uint32_t *flags, cudaStream_t st,
                                     TbOut *tb, bool capture) {
    anyseq_status_t s2 = ANYSEQ_OK;
    const int64_t n = in.n_pairs;
    if (mode != ANYSEQ_GLOBAL && !key_range_ok(sc, in.max_min))
        return fail(ANYSEQ_ERR_ARG, "local / semi-global scores of a pair may reach 2^21 (the optimum key's range)");
    const int sigp = (sc->alphabet > 4 || ctx->force_matrix) ? 1 : 0;
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
    // sigma' = sigma - open - extend must be an int8; int16x2 lanes also need it >= 0
    int32_t sp_min = 1 << 30, sp_max = -(1 << 30);
    const int32_t oe = sc->gap_open + sc->gap_extend;
    const int32_t sig_pad = (mode == ANYSEQ_GLOBAL ? sc->gap_extend : 0) - oe;
    for (int a = 0; a < sc->alphabet; a++)
        for (int b = 0; b < sc->alphabet; b++) {
            int32_t v = sigma_host(sc, a, b) - oe;
            sp_min = v < sp_min ? v : sp_min;
            sp_max = v > sp_max ? v : sp_max;
        }
    sp_min = sig_pad < sp_min ? sig_pad : sp_min;
    sp_max = sig_pad > sp_max ? sig_pad : sp_max;
    if (sp_min < -128 || sp_max > 127)
        return fail(ANYSEQ_ERR_ARG, "sigma - open - extend spans [%d, %d], outside the int8 profile", sp_min, sp_max);
    P.force32 = ctx->force32 || sp_min < 0;
    P.select = in.select;
    CUDA_TRY(launch_prep(P, st));
    ctx->launches += 6;  // pack/validate x2, bin, tile sums, tile scan, scatter

    BatchArgs A;
    memset(&A, 0, sizeof(A));
    A.q2 = P.q2; A.s2 = P.s2; A.q_off = in.q_off; A.s_off = in.s_off;
    if (!sigp) TRY(make_rowprof(sc, mode, A.rowprof));
    A.q8 = in.q;
    A.s8 = in.s;
    A.alphabet = sc->alphabet;
    A.sig_pad = sig_pad;
    if (sigp) {
        int8_t htab[32 * 32];
        for (int a = 0; a < sc->alphabet; a++)
            for (int b = 0; b < sc->alphabet; b++) htab[a * sc->alphabet + b] = (int8_t)(sigma_host(sc, a, b) - oe);
        int8_t *dtab = arena<int8_t>(ctx, "sig_tab", 32 * 32, &s2);
        if (s2 != ANYSEQ_OK) return s2;
        // a graph capture re-uses the table an uncaptured run of the same plan left in place
        if (!capture) CUDA_TRY(cudaMemcpyAsync(dtab, htab, sc->alphabet * sc->alphabet, cudaMemcpyHostToDevice, st));
        A.sig_tab = dtab;
    }
    A.o = sc->gap_open; A.e = sc->gap_extend;
    A.score = score; A.end_q = eq; A.end_s = es; A.flags = flags;
    A.rmax_tab = ctx->tuned ? ctx->d_tune_tab : nullptr;
    A.bin_stats = ctx->d_bin_stats;
    A.counter = arena<int32_t>(ctx, "counter", 4, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    if (tb) {
        // direction-word layout: per pair size from the item plan, then a prefix sum
        int64_t *words = arena<int64_t>(ctx, "tb_words", n + 1, &s2);
        int64_t *base = arena<int64_t>(ctx, "tb_base", n + 1, &s2);
        int64_t *stmp = arena<int64_t>(ctx, "scan_tmp", scan_tmp_words(n) + 2, &s2);
        A.lay_pad = arena<int32_t>(ctx, "tb_pad", n + 1, &s2);
        A.lay_ch0 = arena<int32_t>(ctx, "tb_ch0", n + 1, &s2);
        int32_t *lay_r = arena<int32_t>(ctx, "tb_rows", n + 1, &s2);
        if (s2 != ANYSEQ_OK) return s2;
        CUDA_TRY(cudaMemsetAsync(words, 0, n * sizeof(int64_t), st));
        // the DP kernels' row caps: TB_R fixed on the matrix path, else any R up to row_rmax
        CUDA_TRY(launch_tb_plan(P.list16, P.counts + 0, 4, (n + 3) / 4 + 1, in.q_off, in.s_off, words, A.lay_pad,
                                A.lay_ch0, lay_r, sigp ? TB_R : row_rmax(mode, 2, true), sigp ? TB_R : 0, st));
        CUDA_TRY(launch_tb_plan(P.list32, P.counts + 1, 2, (n + 1) / 2 + 1, in.q_off, in.s_off, words, A.lay_pad,
                                A.lay_ch0, lay_r, sigp ? TB_R : row_rmax(mode, 1, true), sigp ? TB_R : 0, st));
        tb->lay_r = lay_r;
        CUDA_TRY(scan_exclusive_i64(words, base, n, stmp, stmp + scan_tmp_words(n), st));
        int64_t total = 0;
        CUDA_TRY(cudaMemcpyAsync(&total, stmp + scan_tmp_words(n), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        A.dirs = arena<uint32_t>(ctx, "tb_dirs", (size_t)total + 1, &s2);
        if (s2 != ANYSEQ_OK) return s2;
        A.dir_base = base;
        ctx->launches += 5;
        tb->dirs = A.dirs;
        tb->dir_base = base;
        tb->lay_pad = A.lay_pad;
        tb->lay_ch0 = A.lay_ch0;
        tb->dir_words = total;
    }
    for (int cell32 = 0; cell32 < 2; cell32++) {
        int per_sm = batch_blocks_per_sm(cell32, mode, tb != nullptr, sigp, sc->alphabet);
        if (ctx->batch_ctas_per_sm > 0 && ctx->batch_ctas_per_sm < per_sm) per_sm = ctx->batch_ctas_per_sm;
        const int grid = ctx->num_sms * per_sm;
        A.list = cell32 ? P.list32 : P.list16;
        A.n_list = P.counts + cell32;
        A.scratch = nullptr;
        A.scratch_cols = 0;
        // border rows between row chunks: the smallest chunk of any untuned
        // variant is GROUP * TB_R = 128 rows (traceback); a tuned table can
        // cap a chunk at GROUP * 4 rows. Longer queries need scratch.
        const int32_t min_chunk = GROUP * (A.rmax_tab ? TUNE_MIN_R : TB_R);
        if (in.max_n > min_chunk) {
            A.scratch_cols = in.max_m + 1;
            A.scratch = arena<int32_t>(ctx, "border", (size_t)grid * (batch_threads(sigp) / GROUP) * 2 * (size_t)A.scratch_cols, &s2);
            if (s2 != ANYSEQ_OK) return s2;
        }
        CUDA_TRY(cudaMemsetAsync(A.counter, 0, sizeof(int32_t), st));
        if (ctx->profile && !capture) cudaEventRecord(ctx->ev[2 * cell32], st);
        CUDA_TRY(launch_batch(A, cell32, mode, tb != nullptr, sigp, grid, st));
        if (ctx->profile && !capture) cudaEventRecord(ctx->ev[2 * cell32 + 1], st);
        ctx->launches += 1;
    }
    // a graph capture ends here: the caller reads the letter check after the replay
    if (capture) {
        ctx->bad_code = P.bad_code;
        return ANYSEQ_OK;
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

// The device address of pinned host memory that kernels can read in place (a
// mapped allocation in the unified address space), or nullptr.
static const void *mapped_host_ptr(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

anyseq_status_t anyseq::stage_batch(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off, const uint8_t *s,
                                    const int64_t *s_off, int64_t n_pairs, BatchInput &in, cudaStream_t st,
                                    bool read_in_place) {
    anyseq_status_t s2 = ANYSEQ_OK;
    in.n_pairs = n_pairs;
    const void *dq_off, *ds_off;
    TRY(stage_input(ctx, "in_qoff", q_off, (n_pairs + 1) * sizeof(int64_t), st, &dq_off));
    TRY(stage_input(ctx, "in_soff", s_off, (n_pairs + 1) * sizeof(int64_t), st, &ds_off));
    in.q_off = (const int64_t *)dq_off;
    in.s_off = (const int64_t *)ds_off;
    int64_t *stats = arena<int64_t>(ctx, "stats", 8, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    int64_t hstats[6];
    CUDA_TRY(cudaMemsetAsync(stats, 0, 4 * sizeof(int64_t), st));
    len_stats_kernel<<<grid_for(n_pairs) > 304 ? 304 : grid_for(n_pairs), 256, 0, st>>>(in.q_off, in.s_off, n_pairs, stats);
    CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    CUDA_TRY(cudaMemcpyAsync(hstats, stats, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&hstats[4], in.q_off + n_pairs, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&hstats[5], in.s_off + n_pairs, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    int64_t q0 = 0, s0 = 0;
    CUDA_TRY(cudaMemcpyAsync(&q0, in.q_off, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&s0, in.s_off, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hstats[2] || q0 != 0 || s0 != 0)
        return fail(ANYSEQ_ERR_ARG, "offsets must start at 0, be non-decreasing and give lengths below 2^21");
    in.max_n = hstats[0];
    in.max_m = hstats[1];
    in.max_min = hstats[3];
    in.q_len = hstats[4];
    in.s_len = hstats[5];
    if ((in.q_len > 0 && !q) || (in.s_len > 0 && !s)) return fail(ANYSEQ_ERR_ARG, "q or s is NULL");
    // Letters in pinned host memory whose only reader is the 2-bit packing kernel stay
    // where they are: the kernel reads them over the host link as it packs them, in
    // place of a separate copy followed by a pass over device memory.
    const void *dq = read_in_place && in.q_len > 0 ? mapped_host_ptr(q) : nullptr;
    const void *ds = read_in_place && in.s_len > 0 ? mapped_host_ptr(s) : nullptr;
    if (!dq) TRY(stage_input(ctx, "in_q", q, (size_t)in.q_len, st, &dq));
    if (!ds) TRY(stage_input(ctx, "in_s", s, (size_t)in.s_len, st, &ds));
    in.q = (const uint8_t *)dq;
    in.s = (const uint8_t *)ds;

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
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "cudaSetDevice failed");
    anyseq_status_t s2 = ANYSEQ_OK;

    // offsets: stage, then read totals and maxima
    ctx->launches = 0;
    BatchInput in;
    TRY(stage_batch(ctx, q, q_off, s, s_off, n_pairs, in, st,
                    ctx->host_in_place && sc->alphabet <= 4 && !ctx->force_matrix));
    if (mode != ANYSEQ_GLOBAL && !key_range_ok(sc, in.max_min))
        return fail(ANYSEQ_ERR_ARG, "local / semi-global scores of a pair may reach 2^21 (the optimum key's range)");

    int32_t *score = arena<int32_t>(ctx, "r_score", n_pairs, &s2);
    int32_t *eq = arena<int32_t>(ctx, "r_eq", n_pairs, &s2);
    int32_t *es = arena<int32_t>(ctx, "r_es", n_pairs, &s2);
    uint32_t *flags = arena<uint32_t>(ctx, "r_flags", n_pairs, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    const bool want_cigar = (want & ANYSEQ_WANT_CIGAR) != 0;
    TbOut tbo;
    bool on_wave = false;
    if ((want & ANYSEQ_BAND_LEARNED) && !want_cigar && mode == ANYSEQ_GLOBAL && sc->alphabet <= 4) {
        TRY(band_scores(ctx, in, sc, score, eq, es, flags, st));
    } else {
        BatchInput rest = in;
        if (!ctx->force32 && want_cigar && mode == ANYSEQ_GLOBAL)
            TRY(wave_batch(ctx, in, sc, mode, score, eq, es, flags, st, &tbo, &on_wave));
        else if (!ctx->force32 && !want_cigar)
            TRY(long_pairs_split(ctx, in, sc, mode, score, eq, es, flags, st, rest, &on_wave));
        if (!on_wave) TRY(batch_scores(ctx, rest, sc, mode, score, eq, es, flags, st, want_cigar ? &tbo : nullptr));
    }

    int32_t *bq = nullptr, *bs = nullptr;
    int64_t *clen = nullptr, *coff = nullptr;
    uint64_t used = 0;
    if (want_cigar) {
        // walk back, then lay the runs out contiguously in the caller's buffer
        TbWalkArgs W;
        W.n_pairs = n_pairs; W.mode = mode; W.q_off = in.q_off; W.s_off = in.s_off;
        W.end_q = eq; W.end_s = es;
        W.dirs = tbo.dirs; W.dir_base = tbo.dir_base; W.lay_pad = tbo.lay_pad; W.lay_ch0 = tbo.lay_ch0;
        W.lanes_per_chunk = tbo.lanes_per_chunk;
        W.rows_per_lane = tbo.rows_per_lane;
        W.lay_r = tbo.lay_r;
        W.walker = ctx->tb_walker;
        W.tmp = arena<uint32_t>(ctx, "tb_tmp", (size_t)(in.q_len + in.s_len + n_pairs + 1), &s2);
        clen = W.cig_len = arena<int64_t>(ctx, "tb_clen", n_pairs + 1, &s2);
        coff = arena<int64_t>(ctx, "tb_coff", n_pairs + 1, &s2);
        bq = W.beg_q = arena<int32_t>(ctx, "tb_bq", n_pairs + 1, &s2);
        bs = W.beg_s = arena<int32_t>(ctx, "tb_bs", n_pairs + 1, &s2);
        int64_t *stmp = arena<int64_t>(ctx, "scan_tmp", scan_tmp_words(n_pairs) + 2, &s2);
        if (s2 != ANYSEQ_OK) return s2;
        CUDA_TRY(launch_tb_walk(W, st));
        CUDA_TRY(scan_exclusive_i64(clen, coff, n_pairs, stmp, stmp + scan_tmp_words(n_pairs), st));
        int64_t total = 0;
        CUDA_TRY(cudaMemcpyAsync(&total, stmp + scan_tmp_words(n_pairs), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        ctx->launches += 4;
        used = (uint64_t)total;
        if (cigar_used) *cigar_used = used;
        if (!cigar || cigar_cap < used)
            return fail(ANYSEQ_ERR_CAPACITY, "CIGAR buffer holds %llu words, %llu needed",
                        (unsigned long long)cigar_cap, (unsigned long long)used);
        bool cig_dev = is_device_ptr(cigar);
        uint32_t *dcig = cigar;
        if (!cig_dev) {
            dcig = arena<uint32_t>(ctx, "r_cigar", used + 1, &s2);
            if (s2 != ANYSEQ_OK) return s2;
        }
        CUDA_TRY(launch_tb_compact(n_pairs, in.q_off, in.s_off, W.tmp, clen, coff, dcig, st));
        ctx->launches += 1;
        if (!cig_dev && used)
            CUDA_TRY(cudaMemcpyAsync(cigar, dcig, used * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    }

    bool out_dev = is_device_ptr(out);
    anyseq_result_t *dout = out;
    if (!out_dev) {
        dout = arena<anyseq_result_t>(ctx, "r_out", n_pairs, &s2);
        if (s2 != ANYSEQ_OK) return s2;
    }
    write_results_kernel<<<grid_for(n_pairs), 256, 0, st>>>(n_pairs, score, eq, es, flags, bq, bs, coff, clen, dout);
    CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    if (!out_dev) {
        CUDA_TRY(cudaMemcpyAsync(out, dout, n_pairs * sizeof(anyseq_result_t), cudaMemcpyDeviceToHost, st));
    }
    if (!out_dev || (want_cigar && !is_device_ptr(cigar))) CUDA_TRY(cudaStreamSynchronize(st));
    if (cigar_used) *cigar_used = used;
    return ANYSEQ_OK;
}

// 32-bit range of the wavefront: every |value| of the pair stays below 2^28.
// Local and semi-global optima are searched by 64-bit keys whose score field
// holds values below 2^21 (end_key): the best score of a pair is at most the
// largest positive substitution score times min(n, m).
bool anyseq::key_range_ok(const anyseq_scoring_t *sc, int64_t min_nm) {
    int64_t pmax = 0;
    for (int a = 0; a < sc->alphabet; a++)
        for (int b = 0; b < sc->alphabet; b++) {
            const int64_t v = sigma_host(sc, a, b);
            pmax = v > pmax ? v : pmax;
        }
    return pmax * min_nm < (1ll << 21) - 1;
}

// The wavefront's profiles hold sigma - open - extend (and the padding rows'
// value) in signed bytes.
bool anyseq::long_profile_ok(const anyseq_scoring_t *sc) {
    const int32_t oe = sc->gap_open + sc->gap_extend;
    bool ok = sc->gap_extend - oe <= 127 && -oe <= 127;
    for (int a = 0; a < sc->alphabet; a++)
        for (int b = 0; b < sc->alphabet; b++) {
            const int32_t v = sigma_host(sc, a, b) - oe;
            ok = ok && v >= -128 && v <= 127;
        }
    return ok;
}

bool anyseq::long_range_ok(const anyseq_scoring_t *sc, int64_t n, int64_t m) {
    int64_t smax = 0;
    for (int a = 0; a < sc->alphabet; a++)
        for (int b = 0; b < sc->alphabet; b++) {
            int64_t v = sigma_host(sc, a, b);
            smax = v > smax ? v : (-v > smax ? -v : smax);
        }
    const int64_t bound = 3 * (int64_t)(-sc->gap_open) + (n + m + 2) * (int64_t)(-sc->gap_extend) + smax * ((n < m ? n : m) + 1);
    return bound < (1ll << 28);
}

// Batches of at most this many pairs, the largest of at least WAVE_BATCH_CELLS
// cells, run on the wavefront (scores: long_pairs_split; CIGAR: wave_batch).
constexpr int64_t WAVE_BATCH_PAIRS = 8;
constexpr double WAVE_BATCH_CELLS = 262144.0;

__global__ void scatter_results_kernel(int64_t k, const int64_t *idx, const int32_t *vals, int32_t *score,
                                       int32_t *eq, int32_t *es, uint32_t *flags) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = idx[t];
        score[p] = vals[3 * t];
        eq[p] = vals[3 * t + 1];
        es[p] = vals[3 * t + 2];
        flags[p] = ANYSEQ_FLAG_INT32;
    }
}

// Pairs far larger than the rest of a batch leave the batched kernel waiting on
// one 16-lane group per pair, each walking its row chunks in sequence (9
// protein pairs of 20,000 residues: 521 ms, against 10 ms on the wavefront). So
// the long pairs of a score-only batch run as one multi-pass wavefront launch,
// their stripes side by side, and the batched kernel takes the rest through
// its pair selection. A pair is long from 2^18 cells in a batch of at most
// WAVE_BATCH_PAIRS pairs, otherwise from max(2^24, tail_factor x the batch's
// cells / the resident 16-lane groups); it must also pass the wavefront's range
// tests. With in.select, only the selected pairs count and move.
// *all_done: every pair ran on the wavefront; rest: the batch with the other
// pairs selected.
anyseq_status_t anyseq::long_pairs_split(anyseq_ctx *ctx, const BatchInput &in, const anyseq_scoring_t *sc,
                                         int32_t mode, int32_t *score, int32_t *eq, int32_t *es, uint32_t *flags,
                                         cudaStream_t st, BatchInput &rest, bool *all_done, double tail_factor) {
    *all_done = false;
    rest = in;
    const int64_t n = in.n_pairs;
    if (n < 1 || !long_profile_ok(sc)) return ANYSEQ_OK;
    const double small_batch_cells = WAVE_BATCH_CELLS, big_batch_cells = 16777216.0;
    if ((double)in.max_n * (double)in.max_m < (n <= WAVE_BATCH_PAIRS ? small_batch_cells : big_batch_cells))
        return ANYSEQ_OK;
    std::vector<int64_t> hq((size_t)n + 1), hs((size_t)n + 1);
    std::vector<uint8_t> hsel(in.select ? (size_t)n : 0);
    CUDA_TRY(cudaMemcpyAsync(hq.data(), in.q_off, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hs.data(), in.s_off, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (in.select) CUDA_TRY(cudaMemcpyAsync(hsel.data(), in.select, (size_t)n, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    auto taken = [&](int64_t p) { return !in.select || hsel[(size_t)p] != 0; };
    double total = 0;
    int64_t n_taken = 0;
    for (int64_t p = 0; p < n; p++)
        if (taken(p)) {
            total += (double)(hq[p + 1] - hq[p]) * (double)(hs[p + 1] - hs[p]);
            n_taken++;
        }
    const double groups = (double)ctx->num_sms * batch_min_ctas(0) * (batch_threads(0) / GROUP);
    const double thr =
        n_taken <= WAVE_BATCH_PAIRS ? small_batch_cells : std::max(big_batch_cells, tail_factor * total / groups);
    std::vector<int64_t> idx;
    for (int64_t p = 0; p < n; p++) {
        const int64_t qn = hq[p + 1] - hq[p], sm = hs[p + 1] - hs[p];
        if (!taken(p) || qn == 0 || sm == 0 || (double)qn * (double)sm < thr) continue;
        if (!long_range_ok(sc, qn, sm) || (mode != ANYSEQ_GLOBAL && !key_range_ok(sc, qn < sm ? qn : sm))) continue;
        idx.push_back(p);
    }
    if (idx.empty()) return ANYSEQ_OK;
    const int64_t k = (int64_t)idx.size();
    anyseq_status_t s2 = ANYSEQ_OK;
    uint32_t *q2 = arena<uint32_t>(ctx, "wb_q2", (size_t)(in.q_len + 15) / 16 + 2, &s2);
    uint32_t *s2p = arena<uint32_t>(ctx, "wb_s2", (size_t)(in.s_len + 15) / 16 + 2, &s2);
    int32_t *bad = arena<int32_t>(ctx, "wb_bad", 4, &s2);
    int32_t *H = nullptr;
    if (s2 != ANYSEQ_OK) return s2;
    CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
    CUDA_TRY(launch_pack2bit(in.q, in.q_len, q2, sc->alphabet, bad, st));
    CUDA_TRY(launch_pack2bit(in.s, in.s_len, s2p, sc->alphabet, bad, st));
    ctx->launches += 2;
    std::vector<WavePass> passes((size_t)k);
    int64_t out = 0;
    for (int64_t t = 0; t < k; t++) {
        const int64_t p = idx[(size_t)t];
        WavePass &w = passes[(size_t)t];
        memset(&w, 0, sizeof(w));
        w.q0 = hq[p];
        w.s0 = hs[p];
        w.n = (int32_t)(hq[p + 1] - hq[p]);
        w.m = (int32_t)(hs[p + 1] - hs[p]);
        w.tb = sc->gap_open;
        w.out_off = out;
        out += w.m + 1;
    }
    H = arena<int32_t>(ctx, "wb_H", (size_t)out + 2, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    MatLetters ml;
    ml.q8 = in.q;
    ml.s8 = in.s;
    const bool use_mat = sc->alphabet > 4 || ctx->force_matrix;
    std::vector<uint64_t> keys;
    TRY(run_wave_passes(ctx, q2, s2p, passes, sc, H, nullptr, st, nullptr, mode, &keys, use_mat ? &ml : nullptr));
    std::vector<int32_t> vals((size_t)(3 * k));
    for (int64_t t = 0; t < k; t++) {
        const WavePass &w = passes[(size_t)t];
        if (mode == ANYSEQ_GLOBAL) {
            CUDA_TRY(cudaMemcpyAsync(&vals[(size_t)(3 * t)], H + w.out_off + w.m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            vals[(size_t)(3 * t + 1)] = w.n;
            vals[(size_t)(3 * t + 2)] = w.m;
        } else {
            vals[(size_t)(3 * t)] = key_score(keys[(size_t)t]);
            vals[(size_t)(3 * t + 1)] = key_i(keys[(size_t)t]);
            vals[(size_t)(3 * t + 2)] = key_j(keys[(size_t)t]);
        }
    }
    int32_t hb = 0;
    CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hb) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", sc->alphabet);
    int64_t *didx = arena<int64_t>(ctx, "wb_idx", (size_t)k + 1, &s2);
    int32_t *dvals = arena<int32_t>(ctx, "wb_vals", (size_t)(3 * k) + 1, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    CUDA_TRY(cudaMemcpyAsync(didx, idx.data(), (size_t)k * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(dvals, vals.data(), (size_t)(3 * k) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    scatter_results_kernel<<<(unsigned)std::min<int64_t>((k + 255) / 256, 1024), 256, 0, st>>>(k, didx, dvals, score, eq,
                                                                                             es, flags);
    CUDA_TRY(cudaGetLastError());
    ctx->launches += 1;
    if (k == n_taken) {
        *all_done = true;
        ctx->pairs16 = 0;
        ctx->pairs32 = k;
    } else {
        // the batched kernel takes the other pairs
        std::vector<uint8_t> sel((size_t)n, 1);
        if (in.select) sel = hsel;
        for (int64_t p : idx) sel[(size_t)p] = 0;
        uint8_t *dsel = arena<uint8_t>(ctx, "wb_sel", (size_t)n + 16, &s2);
        if (s2 != ANYSEQ_OK) return s2;
        CUDA_TRY(cudaMemcpyAsync(dsel, sel.data(), (size_t)n, cudaMemcpyHostToDevice, st));
        rest.select = dsel;
    }
    // the host vectors must outlive the copies
    CUDA_TRY(cudaStreamSynchronize(st));
    return ANYSEQ_OK;
}

// CIGAR of a batch of a few large global pairs: the wavefront's traceback
// variant runs each pair's stripes side by side, where the batched kernel would
// give each pair one 16-lane group. Qualifies: at most WAVE_BATCH_PAIRS pairs,
// 2-bit letters, every pair inside the wavefront's 32-bit range, and the
// largest pair of at least WAVE_BATCH_CELLS cells.

anyseq_status_t anyseq::wave_batch(anyseq_ctx *ctx, const BatchInput &in, const anyseq_scoring_t *sc,
                                   int32_t mode, int32_t *score, int32_t *eq, int32_t *es, uint32_t *flags,
                                   cudaStream_t st, TbOut *tb, bool *used) {
    *used = false;
    const int64_t n = in.n_pairs;
    // the traceback variant reads 2-bit letters and row profiles
    if (n > WAVE_BATCH_PAIRS || mode != ANYSEQ_GLOBAL || sc->alphabet > 4 || ctx->force_matrix || !long_profile_ok(sc))
        return ANYSEQ_OK;
    if ((double)in.max_n * (double)in.max_m < WAVE_BATCH_CELLS) return ANYSEQ_OK;
    std::vector<int64_t> hq((size_t)n + 1), hs((size_t)n + 1);
    CUDA_TRY(cudaMemcpyAsync(hq.data(), in.q_off, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hs.data(), in.s_off, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t p = 0; p < n; p++)
        if (!long_range_ok(sc, hq[p + 1] - hq[p], hs[p + 1] - hs[p])) return ANYSEQ_OK;
    if (mode != ANYSEQ_GLOBAL && !key_range_ok(sc, in.max_min)) return ANYSEQ_OK;
    std::vector<uint64_t> keys;
    *used = true;
    anyseq_status_t s2 = ANYSEQ_OK;
    uint32_t *q2 = arena<uint32_t>(ctx, "wb_q2", (size_t)(in.q_len + 15) / 16 + 2, &s2);
    uint32_t *s2p = arena<uint32_t>(ctx, "wb_s2", (size_t)(in.s_len + 15) / 16 + 2, &s2);
    int32_t *bad = arena<int32_t>(ctx, "wb_bad", 4, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
    CUDA_TRY(launch_pack2bit(in.q, in.q_len, q2, sc->alphabet, bad, st));
    CUDA_TRY(launch_pack2bit(in.s, in.s_len, s2p, sc->alphabet, bad, st));
    ctx->launches += 2;
    // one pass per non-empty pair; empty pairs take the closed forms of the recurrences
    std::vector<WavePass> passes;
    std::vector<int64_t> pass_of((size_t)n, -1);
    int64_t out = 0;
    for (int64_t p = 0; p < n; p++) {
        const int64_t qn = hq[p + 1] - hq[p], sm = hs[p + 1] - hs[p];
        if (qn == 0 || sm == 0) continue;
        WavePass w;
        memset(&w, 0, sizeof(w));
        w.q0 = hq[p];
        w.s0 = hs[p];
        w.n = (int32_t)qn;
        w.m = (int32_t)sm;
        w.tb = sc->gap_open;
        w.out_off = out;
        out += sm + 1;
        pass_of[(size_t)p] = (int64_t)passes.size();
        passes.push_back(w);
    }
    std::vector<int32_t> hscore((size_t)n), heq((size_t)n), hes((size_t)n), hpad((size_t)n, 0), hch0((size_t)n, 0);
    std::vector<uint32_t> hflags((size_t)n, ANYSEQ_FLAG_INT32);
    std::vector<int64_t> hbase((size_t)n, 0);
    WaveTb wtb;
    if (!passes.empty()) {
        int32_t *H = arena<int32_t>(ctx, "wb_H", (size_t)out + 2, &s2);
        if (s2 != ANYSEQ_OK) return s2;
        TRY(run_wave_passes(ctx, q2, s2p, passes, sc, H, nullptr, st, tb ? &wtb : nullptr, mode, &keys));
        for (int64_t p = 0; p < n; p++) {
            const int64_t k = pass_of[(size_t)p];
            if (k < 0) continue;
            const WavePass &w = passes[(size_t)k];
            if (mode == ANYSEQ_GLOBAL)
                CUDA_TRY(cudaMemcpyAsync(&hscore[(size_t)p], H + w.out_off + w.m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            hbase[(size_t)p] = w.dir_off;
            const int32_t rows = WAVE_LANES * (tb ? wtb.rows_per_lane : 8);
            hpad[(size_t)p] = ((w.n + rows - 1) / rows) * rows - w.n;
        }
    }
    int32_t hb = 0;
    CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hb) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", sc->alphabet);
    for (int64_t p = 0; p < n; p++) {
        const int64_t qn = hq[p + 1] - hq[p], sm = hs[p + 1] - hs[p];
        const int64_t k = pass_of[(size_t)p];
        if (mode == ANYSEQ_GLOBAL) {
            if (qn == 0 || sm == 0) hscore[(size_t)p] = (qn + sm == 0) ? 0 : sc->gap_open + (int32_t)(qn + sm) * sc->gap_extend;
            heq[(size_t)p] = (int32_t)qn;
            hes[(size_t)p] = (int32_t)sm;
        } else if (k < 0) {
            // an empty sequence: the empty alignment at (0, 0)
            hscore[(size_t)p] = heq[(size_t)p] = hes[(size_t)p] = 0;
        } else {
            hscore[(size_t)p] = key_score(keys[(size_t)k]);
            heq[(size_t)p] = key_i(keys[(size_t)k]);
            hes[(size_t)p] = key_j(keys[(size_t)k]);
        }
    }
    CUDA_TRY(cudaMemcpyAsync(score, hscore.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(eq, heq.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(es, hes.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(flags, hflags.data(), (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    if (tb) {
        tb->dirs = wtb.dirs;
        tb->dir_base = arena<int64_t>(ctx, "wb_base", (size_t)n + 1, &s2);
        tb->lay_pad = arena<int32_t>(ctx, "wb_pad", (size_t)n + 1, &s2);
        tb->lay_ch0 = arena<int32_t>(ctx, "wb_ch0", (size_t)n + 1, &s2);
        if (s2 != ANYSEQ_OK) return s2;
        CUDA_TRY(cudaMemcpyAsync(tb->dir_base, hbase.data(), (size_t)n * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(tb->lay_pad, hpad.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(tb->lay_ch0, hch0.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        tb->lanes_per_chunk = WAVE_LANES;
        tb->rows_per_lane = wtb.rows_per_lane;
    }
    // the host vectors must outlive the copies
    CUDA_TRY(cudaStreamSynchronize(st));
    ctx->pairs16 = 0;
    ctx->pairs32 = n;
    return ANYSEQ_OK;
}

// Global scores of several long pairs in one wavefront launch (one pass per
// pair; their stripes run side by side). Host letters and offsets; every pair
// non-empty and inside the 32-bit range test of anyseq_align_long.
anyseq_status_t anyseq::long_scores(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off, const uint8_t *s,
                                    const int64_t *s_off, int64_t count, const anyseq_scoring_t *sc, int32_t *scores,
                                    cudaStream_t st, int32_t mode, int32_t *end_q, int32_t *end_s) {
    if (count <= 0) return ANYSEQ_OK;
    anyseq_status_t s2 = ANYSEQ_OK;
    const int64_t nq = q_off[count], ns = s_off[count];
    std::vector<WavePass> passes((size_t)count);
    int64_t out = 0;
    for (int64_t k = 0; k < count; k++) {
        WavePass &p = passes[(size_t)k];
        memset(&p, 0, sizeof(p));
        p.q0 = q_off[k];
        p.s0 = s_off[k];
        p.n = (int32_t)(q_off[k + 1] - q_off[k]);
        p.m = (int32_t)(s_off[k + 1] - s_off[k]);
        if (p.n <= 0 || p.m <= 0) return fail(ANYSEQ_ERR_ARG, "long_scores: empty pair %lld", (long long)k);
        if (mode != ANYSEQ_GLOBAL && !key_range_ok(sc, p.n < p.m ? p.n : p.m))
            return fail(ANYSEQ_ERR_ARG, "long_scores: scores of pair %lld may reach 2^21", (long long)k);
        p.tb = sc->gap_open;
        p.out_off = out;
        out += p.m + 1;
    }
    const void *dq, *ds;
    TRY(stage_input(ctx, "ls_q", q, (size_t)nq, st, &dq));
    TRY(stage_input(ctx, "ls_s", s, (size_t)ns, st, &ds));
    uint32_t *q2 = arena<uint32_t>(ctx, "ls_q2", (size_t)(nq + 15) / 16 + 2, &s2);
    uint32_t *s2p = arena<uint32_t>(ctx, "ls_s2", (size_t)(ns + 15) / 16 + 2, &s2);
    int32_t *bad = arena<int32_t>(ctx, "ls_bad", 4, &s2);
    int32_t *H = arena<int32_t>(ctx, "ls_H", (size_t)out + 2, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
    CUDA_TRY(launch_pack2bit((const uint8_t *)dq, nq, q2, sc->alphabet, bad, st));
    CUDA_TRY(launch_pack2bit((const uint8_t *)ds, ns, s2p, sc->alphabet, bad, st));
    ctx->launches += 2;
    std::vector<uint64_t> keys;
    TRY(run_wave_passes(ctx, q2, s2p, passes, sc, H, nullptr, st, nullptr, mode, &keys));
    int32_t hb = 0;
    CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (mode == ANYSEQ_GLOBAL) {
        for (int64_t k = 0; k < count; k++) {
            const WavePass &p = passes[(size_t)k];
            CUDA_TRY(cudaMemcpyAsync(&scores[k], H + p.out_off + p.m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        }
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hb) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", sc->alphabet);
    for (int64_t k = 0; k < count; k++) {
        const WavePass &p = passes[(size_t)k];
        if (mode != ANYSEQ_GLOBAL) scores[k] = key_score(keys[(size_t)k]);
        if (end_q) end_q[k] = mode == ANYSEQ_GLOBAL ? p.n : key_i(keys[(size_t)k]);
        if (end_s) end_s[k] = mode == ANYSEQ_GLOBAL ? p.m : key_j(keys[(size_t)k]);
    }
    return ANYSEQ_OK;
}

// Last row (H, E) of one global pass (wavefront kernel, see hb.cu for the
// multi-pass form used by the divide-and-conquer traceback).
anyseq_status_t anyseq::long_last_row(anyseq_ctx *ctx, const uint32_t *q2, int64_t q0, int32_t n, const uint32_t *s2,
                                      int64_t s0, int32_t m, bool rev, int32_t tb, const anyseq_scoring_t *sc,
                                      int32_t *H, int32_t *E, cudaStream_t st, const MatLetters *mat) {
    std::vector<WavePass> passes(1);
    memset(passes.data(), 0, sizeof(WavePass));
    passes[0].q0 = q0; passes[0].s0 = s0; passes[0].n = n; passes[0].m = m;
    passes[0].tb = tb; passes[0].rev = rev ? 1 : 0; passes[0].out_off = 0;
    return run_wave_passes(ctx, q2, s2, passes, sc, H, E, st, nullptr, ANYSEQ_GLOBAL, nullptr, mat);
}

// Start cell of a local or semi-global long-pair traceback (r holds the score
// and the optimum cell). The alignment ends at the optimum cell (ei, ej); its
// score S is the largest global score of q[i .. ei) against s[j .. ej) over the
// starts (i, j) the mode allows: any cell (local), row 0 or column 0
// (semi-global). One anchored wavefront pass over the reversed prefixes gives
// those global scores; its best cell, largest score and then smallest reversed
// row and column, is the start with the largest i and then the largest j. An
// empty optimum (S = 0) starts where it ends.
anyseq_status_t anyseq::long_start_cell(anyseq_ctx *ctx, const uint32_t *q2, const uint32_t *s2p,
                                        const anyseq_scoring_t *sc, int32_t mode, anyseq_result_t &r,
                                        cudaStream_t st, const MatLetters *mat) {
    r.beg_q = r.end_q;
    r.beg_s = r.end_s;
    if (r.score <= 0 || r.end_q == 0 || r.end_s == 0) return ANYSEQ_OK;
    anyseq_status_t s2 = ANYSEQ_OK;
    int32_t *H = arena<int32_t>(ctx, "ls_start_H", (size_t)r.end_s + 2, &s2);
    if (s2 != ANYSEQ_OK) return s2;
    std::vector<WavePass> passes(1);
    memset(passes.data(), 0, sizeof(WavePass));
    passes[0].n = r.end_q;
    passes[0].m = r.end_s;
    passes[0].tb = sc->gap_open;
    passes[0].rev = 1;
    std::vector<uint64_t> keys;
    TRY(run_wave_passes(ctx, q2, s2p, passes, sc, H, nullptr, st, nullptr,
                        mode == ANYSEQ_LOCAL ? ANCHORED_LOCAL : ANCHORED_SEMIGLOBAL, &keys, mat));
    if (keys[0] == 0 || key_score(keys[0]) != r.score)
        return fail(ANYSEQ_ERR_CUDA, "start-cell pass found score %d, the optimum is %d",
                    keys[0] ? key_score(keys[0]) : -1, r.score);
    r.beg_q = r.end_q - key_i(keys[0]);
    r.beg_s = r.end_s - key_j(keys[0]);
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_align_long(anyseq_ctx *ctx, const uint8_t *q, int64_t n, const uint8_t *s,
                                             int64_t m, const anyseq_scoring_t *sc, int32_t mode, uint32_t want,
                                             anyseq_result_t *out, uint32_t *cigar, uint64_t cigar_cap,
                                             uint64_t *cigar_used, void *cuda_stream) {
    if (!ctx) return fail(ANYSEQ_ERR_ARG, "ctx is NULL");
    if (n < 0 || m < 0 || n >= (1ll << 23) || m >= (1ll << 23)) return fail(ANYSEQ_ERR_ARG, "lengths out of range (below 2^23)");
    if (!out) return fail(ANYSEQ_ERR_ARG, "out is NULL");
    if ((n > 0 && !q) || (m > 0 && !s)) return fail(ANYSEQ_ERR_ARG, "q or s is NULL");
    TRY(check_scoring(sc, mode));
    if (mode != ANYSEQ_GLOBAL && (n >= (1ll << 21) || m >= (1ll << 21)))
        return fail(ANYSEQ_ERR_ARG, "local and semi-global long pairs below 2^21 letters");
    if (mode != ANYSEQ_GLOBAL && !key_range_ok(sc, n < m ? n : m))
        return fail(ANYSEQ_ERR_ARG, "local / semi-global scores of this pair may reach 2^21 (the optimum key's range)");
    if (!long_range_ok(sc, n, m)) return fail(ANYSEQ_ERR_ARG, "scores of this pair may leave the 32-bit range");
    if (!long_profile_ok(sc))
        return fail(ANYSEQ_ERR_ARG, "sigma - open - extend leaves the signed byte range on the long-pair path");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "cudaSetDevice failed");
    ctx->launches = 0;
    anyseq_status_t s2 = ANYSEQ_OK;
    anyseq_result_t r;
    memset(&r, 0, sizeof(r));
    r.beg_q = r.beg_s = -1;
    r.end_q = (int32_t)n;
    r.end_s = (int32_t)m;
    r.flags = ANYSEQ_FLAG_INT32;
    const bool want_cigar = (want & ANYSEQ_WANT_CIGAR) != 0;
    std::vector<uint32_t> hcig;
    if (n == 0 || m == 0) {
        if (mode == ANYSEQ_GLOBAL) {
            r.score = (n + m == 0) ? 0 : sc->gap_open + (int32_t)(n + m) * sc->gap_extend;
            if (m) hcig.push_back(((uint32_t)m << 4) | 2u);
            if (n) hcig.push_back(((uint32_t)n << 4) | 1u);
        } else {
            r.score = r.end_q = r.end_s = 0;  // the empty alignment at (0, 0)
        }
    } else {
        const void *dq, *ds;
        TRY(stage_input(ctx, "l_q", q, (size_t)n, st, &dq));
        TRY(stage_input(ctx, "l_s", s, (size_t)m, st, &ds));
        uint32_t *q2 = arena<uint32_t>(ctx, "l_q2", (size_t)(n + 15) / 16 + 2, &s2);
        uint32_t *s2p = arena<uint32_t>(ctx, "l_s2", (size_t)(m + 15) / 16 + 2, &s2);
        int32_t *bad = arena<int32_t>(ctx, "l_bad", 4, &s2);
        int32_t *H = arena<int32_t>(ctx, "l_H", (size_t)m + 2, &s2);
        if (s2 != ANYSEQ_OK) return s2;
        CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
        // letter check (and the 2-bit letters of alphabets up to 4)
        CUDA_TRY(launch_pack2bit((const uint8_t *)dq, n, q2, sc->alphabet, bad, st));
        CUDA_TRY(launch_pack2bit((const uint8_t *)ds, m, s2p, sc->alphabet, bad, st));
        ctx->launches += 2;
        // alphabets above 4 letters (or the forced matrix path): byte letters and a sigma table
        MatLetters ml;
        ml.q8 = (const uint8_t *)dq;
        ml.s8 = (const uint8_t *)ds;
        const MatLetters *mat = (sc->alphabet > 4 || ctx->force_matrix) ? &ml : nullptr;
        if (mode == ANYSEQ_GLOBAL) {
            TRY(long_last_row(ctx, q2, 0, (int32_t)n, s2p, 0, (int32_t)m, false, sc->gap_open, sc, H, nullptr, st, mat));
        } else {
            std::vector<WavePass> passes(1);
            memset(passes.data(), 0, sizeof(WavePass));
            passes[0].n = (int32_t)n;
            passes[0].m = (int32_t)m;
            passes[0].tb = sc->gap_open;
            std::vector<uint64_t> keys;
            TRY(run_wave_passes(ctx, q2, s2p, passes, sc, H, nullptr, st, nullptr, mode, &keys, mat));
            r.score = key_score(keys[0]);
            r.end_q = key_i(keys[0]);
            r.end_s = key_j(keys[0]);
        }
        int32_t hb = 0;
        CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (hb) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", sc->alphabet);
        if (mode == ANYSEQ_GLOBAL) {
            CUDA_TRY(cudaMemcpyAsync(&r.score, H + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
        }
        if (want_cigar && mode == ANYSEQ_GLOBAL) {
            TRY(hirschberg_cigar(ctx, q2, 0, (int32_t)n, s2p, 0, (int32_t)m, sc, hcig, st, mat));
            r.beg_q = r.beg_s = 0;
        } else if (want_cigar) {
            TRY(long_start_cell(ctx, q2, s2p, sc, mode, r, st, mat));
            if (r.end_q > r.beg_q || r.end_s > r.beg_s)
                TRY(hirschberg_cigar(ctx, q2, r.beg_q, r.end_q, s2p, r.beg_s, r.end_s, sc, hcig, st, mat));
        }
    }
    if (want_cigar) {
        if (n == 0 || m == 0) {
            r.beg_q = mode == ANYSEQ_GLOBAL ? 0 : r.end_q;
            r.beg_s = mode == ANYSEQ_GLOBAL ? 0 : r.end_s;
        }
        r.cigar_off = 0;
        r.cigar_len = (uint32_t)hcig.size();
        if (cigar_used) *cigar_used = hcig.size();
        if (!cigar || cigar_cap < hcig.size())
            return fail(ANYSEQ_ERR_CAPACITY, "CIGAR buffer holds %llu words, %zu needed",
                        (unsigned long long)cigar_cap, hcig.size());
        if (!hcig.empty())
            CUDA_TRY(cudaMemcpyAsync(cigar, hcig.data(), hcig.size() * sizeof(uint32_t), cudaMemcpyDefault, st));
    } else if (cigar_used) {
        *cigar_used = 0;
    }
    CUDA_TRY(cudaMemcpyAsync(out, &r, sizeof(r), cudaMemcpyDefault, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return ANYSEQ_OK;
}
