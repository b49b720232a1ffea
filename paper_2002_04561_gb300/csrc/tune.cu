// Autotuner of the batched kernel's tile shape per length bin (not in the
// paper; its tiles are fixed per target). A 16-lane slot relaxes a row chunk
// of 16 x R rows, R chosen per work item from the longest query under a cap:
// tall chunks (large R) spread each step's fixed work over more cells, short
// ones waste fewer padding rows. A tuning run first aligns the sample once per
// candidate cap while the kernel adds up, per length bin of the item's longest
// query, the SM cycles of its items and their cells; each bin takes the cap
// with the fewest cycles per cell. Cycles per item measure a warp's latency
// beside its neighbours, not the launch's throughput, so the run then times
// the whole sample (CUDA events, median of five) under the default shape,
// each uniform cap and the per-bin table, and keeps the fastest; a table must
// beat the default by 3 % (run-to-run variation of a whole batch is about
// 1 %). Later calls of the context read the table. Results do not depend on
// it, only the tile shape does.
#include <algorithm>
#include <cstring>

#include "../../include/anyseq.h"
#include "api_internal.h"
#include "batch.h"

using anyseq::fail;

namespace {
constexpr int CAPS[] = {anyseq::TUNE_MIN_R, 8, 12, 16};
constexpr int NCAPS = 4;
// a bin moves off the kernel's own cap only for a gain above this fraction
constexpr double MIN_GAIN = 0.03;
// a table replaces the default shape only for a whole-sample gain above this
constexpr double MIN_TOTAL_GAIN = 0.03;
constexpr int TIMED_RUNS = 5;
}  // namespace

extern "C" anyseq_status_t anyseq_autotune(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off,
                                           const uint8_t *s, const int64_t *s_off, int64_t n_pairs,
                                           const anyseq_scoring_t *sc, int32_t mode, void *cuda_stream) {
    if (!ctx) return fail(ANYSEQ_ERR_ARG, "ctx is NULL");
    if (n_pairs < 1) return fail(ANYSEQ_ERR_ARG, "the tuning sample needs at least one pair");
    anyseq_status_t st = anyseq::check_scoring(sc, mode);
    if (st != ANYSEQ_OK) return st;
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "cudaSetDevice failed");
    anyseq::BatchInput in;
    st = anyseq::stage_batch(ctx, q, q_off, s, s_off, n_pairs, in, cs);
    if (st != ANYSEQ_OK) return st;
    uint8_t *d_tab = static_cast<uint8_t *>(ctx->get("tune_tab", 256, &st));
    auto *d_stats = static_cast<unsigned long long *>(ctx->get("tune_stats", 512 * sizeof(unsigned long long), &st));
    int32_t *score = static_cast<int32_t *>(ctx->get("tune_score", (size_t)n_pairs * 4 + 16, &st));
    int32_t *eq = static_cast<int32_t *>(ctx->get("tune_eq", (size_t)n_pairs * 4 + 16, &st));
    int32_t *es = static_cast<int32_t *>(ctx->get("tune_es", (size_t)n_pairs * 4 + 16, &st));
    uint32_t *flags = static_cast<uint32_t *>(ctx->get("tune_flags", (size_t)n_pairs * 4 + 16, &st));
    if (st != ANYSEQ_OK) return st;
    ctx->d_tune_tab = d_tab;
    // the context is untuned while the run measures; a failure leaves it so
    ctx->tuned = false;
    memset(ctx->tune_tab, 0, sizeof(ctx->tune_tab));
    ctx->tune_gain = 1.0;

    // runs the sample once with table tab (nullptr: the default shape);
    // stats != nullptr also collects the per-bin cycles and cells
    auto run_with = [&](const uint8_t *tab, unsigned long long *stats) -> anyseq_status_t {
        if (tab) {
            const cudaError_t e = cudaMemcpyAsync(d_tab, tab, 256, cudaMemcpyHostToDevice, cs);
            if (e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
        }
        ctx->tuned = tab != nullptr;
        ctx->d_bin_stats = stats;
        const anyseq_status_t r = anyseq::batch_scores(ctx, in, sc, mode, score, eq, es, flags, cs);
        ctx->d_bin_stats = nullptr;
        ctx->tuned = false;
        return r;
    };

    // 1. per-bin cycles per cell of each cap
    double cpc[NCAPS][256];  // negative: no items in the bin
    for (int k = 0; k < NCAPS; k++) {
        uint8_t tab[256];
        memset(tab, CAPS[k], sizeof(tab));
        unsigned long long hs[512];
        cudaError_t e = cudaMemsetAsync(d_stats, 0, sizeof(hs), cs);
        if (e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
        st = run_with(tab, d_stats);
        if (st != ANYSEQ_OK) return st;
        e = cudaMemcpyAsync(hs, d_stats, sizeof(hs), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
        for (int b = 0; b < 256; b++) cpc[k][b] = hs[2 * b + 1] ? (double)hs[2 * b] / (double)hs[2 * b + 1] : -1.0;
    }
    uint8_t per_bin[256];
    for (int b = 0; b < 256; b++) {
        int best = NCAPS - 1;
        for (int k = 0; k < NCAPS - 1; k++)
            if (cpc[k][b] >= 0 && cpc[NCAPS - 1][b] >= 0 && cpc[k][b] < cpc[best][b] * (1.0 - MIN_GAIN)) best = k;
        per_bin[b] = (best == NCAPS - 1 || cpc[best][b] < 0) ? 0 : (uint8_t)CAPS[best];
    }

    // 2. whole-sample time of each candidate table
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(ANYSEQ_ERR_CUDA, "autotune: cudaEventCreate failed");
    }
    auto time_with = [&](const uint8_t *tab, double *ms) -> anyseq_status_t {
        anyseq_status_t r = run_with(tab, nullptr);  // warm-up
        float t[TIMED_RUNS];
        for (int k = 0; k < TIMED_RUNS && r == ANYSEQ_OK; k++) {
            cudaEventRecord(e0, cs);
            r = run_with(tab, nullptr);
            cudaEventRecord(e1, cs);
            if (r == ANYSEQ_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[k], e0, e1) != cudaSuccess))
                r = fail(ANYSEQ_ERR_CUDA, "autotune: event timing failed");
        }
        if (r == ANYSEQ_OK) {
            std::sort(t, t + TIMED_RUNS);
            *ms = t[TIMED_RUNS / 2];
        }
        return r;
    };
    double t_default = 0, t_best = 0;
    uint8_t best_tab[256] = {0};
    bool best_is_default = true;
    st = time_with(nullptr, &t_default);
    t_best = t_default;
    for (int k = 0; k <= NCAPS && st == ANYSEQ_OK; k++) {
        uint8_t tab[256];
        if (k < NCAPS - 1) memset(tab, CAPS[k], sizeof(tab));   // uniform caps below the default
        else if (k == NCAPS) memcpy(tab, per_bin, sizeof(tab));  // the per-bin pick
        else continue;                                           // the largest cap is the default
        double ms = 0;
        st = time_with(tab, &ms);
        if (st == ANYSEQ_OK && ms < t_best && ms < t_default * (1.0 - MIN_TOTAL_GAIN)) {
            t_best = ms;
            memcpy(best_tab, tab, sizeof(tab));
            best_is_default = false;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != ANYSEQ_OK) return st;
    if (!best_is_default) {
        memcpy(ctx->tune_tab, best_tab, sizeof(best_tab));
        const cudaError_t e = cudaMemcpyAsync(d_tab, ctx->tune_tab, sizeof(ctx->tune_tab), cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess || cudaStreamSynchronize(cs) != cudaSuccess)
            return fail(ANYSEQ_ERR_CUDA, "autotune: copying the table failed");
        ctx->tuned = true;
        ctx->tune_gain = t_default / t_best;
    }
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_autotune_table(anyseq_ctx *ctx, uint8_t *caps) {
    if (!ctx || !caps) return fail(ANYSEQ_ERR_ARG, "ctx and caps must not be NULL");
    for (int b = 0; b < 256; b++) caps[b] = ctx->tuned ? ctx->tune_tab[b] : 0;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_autotune_set_table(anyseq_ctx *ctx, const uint8_t *caps) {
    if (!ctx || !caps) return fail(ANYSEQ_ERR_ARG, "ctx and caps must not be NULL");
    for (int b = 0; b < 256; b++) {
        bool ok = caps[b] == 0;
        for (int k = 0; k < NCAPS; k++) ok = ok || caps[b] == CAPS[k];
        if (!ok) return fail(ANYSEQ_ERR_ARG, "cap %d of bin %d is not 0, 4, 8, 12 or 16", (int)caps[b], b);
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "cudaSetDevice failed");
    anyseq_status_t st = ANYSEQ_OK;
    uint8_t *d_tab = static_cast<uint8_t *>(ctx->get("tune_tab", 256, &st));
    if (st != ANYSEQ_OK) return st;
    memcpy(ctx->tune_tab, caps, sizeof(ctx->tune_tab));
    if (cudaMemcpy(d_tab, ctx->tune_tab, sizeof(ctx->tune_tab), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(ANYSEQ_ERR_CUDA, "autotune: copying the table failed");
    ctx->d_tune_tab = d_tab;
    ctx->tuned = true;
    return ANYSEQ_OK;
}
