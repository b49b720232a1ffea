// Learned band: C ABI entry points, training driver and the banded route of
// anyseq_align_batch (features -> network -> banded DP with certificate ->
// doubling -> full DP). See band.cu for the band and the certificate.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/anyseq.h"
#include "api_internal.h"
#include "band.h"
#include "batch.h"
#include "common.cuh"

using namespace anyseq;

#define BTRY(x)                             \
    do {                                    \
        anyseq_status_t _s = (x);           \
        if (_s != ANYSEQ_OK) return _s;     \
    } while (0)
#define BCUDA(x)                                                                                \
    do {                                                                                        \
        cudaError_t _e = (x);                                                                   \
        if (_e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(_e)); \
    } while (0)

template <class T>
static T *arena_b(anyseq_ctx *ctx, const char *name, size_t count, anyseq_status_t *st) {
    return static_cast<T *>(ctx->get(name, count * sizeof(T) + 16, st));
}

static constexpr int64_t NP = MLP_NPARAM;
static constexpr int32_t MIN_W = 16;

// Cells of a band of top half-width w over n rows (the half-width tapers
// linearly to min(w, 16) at the last row, see chunk_cols).
__host__ __device__ inline double band_area(int64_t n, int32_t w) {
    const double wm = w < 16 ? (double)w : 16.0;
    return ((double)w + wm + 1.0) * (double)n;
}

static MlpDev mlp_dev(anyseq_ctx *ctx) {
    MlpDev P;
    P.master = ctx->mlp;
    P.grad = ctx->mlp + NP;
    P.m = ctx->mlp + 2 * NP;
    P.v = ctx->mlp + 3 * NP;
    P.w16 = reinterpret_cast<uint16_t *>(ctx->mlp + 4 * NP);
    return P;
}

static anyseq_status_t mlp_alloc(anyseq_ctx *ctx) {
    if (ctx->mlp) return ANYSEQ_OK;
    size_t bytes = (size_t)NP * (4 * sizeof(float) + sizeof(uint16_t)) + 64;
    if (cudaMalloc(&ctx->mlp, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ANYSEQ_ERR_BUDGET, "cudaMalloc of the band network failed");
    }
    cudaMemset(ctx->mlp, 0, bytes);
    return ANYSEQ_OK;
}

// Deterministic initial weights: uniform(-1,1) * sqrt(6 / fan_in) from SplitMix64.
static void init_params(std::vector<float> &w, uint64_t seed) {
    w.assign(NP, 0.0f);
    uint64_t z = seed;
    auto next = [&]() {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        return (double)(x >> 11) * (1.0 / 9007199254740992.0);
    };
    const int sizes[4] = {MLP_IN, MLP_H, MLP_H, MLP_OUT};
    int64_t off = 0;
    for (int l = 0; l < 3; l++) {
        const double lim = std::sqrt(6.0 / sizes[l]);
        for (int64_t k = 0; k < (int64_t)sizes[l] * sizes[l + 1]; k++) w[off + k] = (float)((2.0 * next() - 1.0) * lim);
        off += (int64_t)sizes[l] * sizes[l + 1] + sizes[l + 1];  // biases stay 0
    }
    // output bias: centre 0, half-width a quarter of the longer sequence
    w[NP - 1] = -1.386294f;
}

static anyseq_status_t set_params(anyseq_ctx *ctx, const float *h, cudaStream_t st) {
    BTRY(mlp_alloc(ctx));
    MlpDev P = mlp_dev(ctx);
    BCUDA(cudaMemcpyAsync(P.master, h, NP * sizeof(float), cudaMemcpyDefault, st));
    BCUDA(cudaMemsetAsync(P.m, 0, 2 * NP * sizeof(float), st));
    BCUDA(launch_mlp_round(P, st));
    BCUDA(cudaStreamSynchronize(st));
    ctx->mlp_ready = true;
    return ANYSEQ_OK;
}

// ------------------------------------------------------------------ kernels

// Band proposal from the network output; pairs whose band would cover half of
// the matrix (or with an empty sequence) go straight to the full DP.
// Largest band (share of the pair's matrix) worth a banded pass: the full DP
// runs pairs that pass the int16 range test two per 32-bit lane, the banded
// kernel always one, so their bands must be narrower to pay off.
struct BandCaps {
    double area32, area16;
    int32_t smax, smin, o, e;
    float margin;  // the network's half-width is multiplied by this before use
    float floor;   // and is at least this share of the longer sequence
};
__device__ __forceinline__ double band_cap(const BandCaps &K, int64_t n, int64_t m) {
    return fits_int16(n, m, K.smax, K.smin, K.o, K.e, GLOBAL) ? K.area16 : K.area32;
}

__global__ void band_plan_kernel(const float *y, const int64_t *q_off, const int64_t *s_off, int64_t n_pairs,
                                 BandCaps caps, int32_t *centre, int32_t *width, uint8_t *full, int32_t *list,
                                 int64_t *count) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = q_off[p + 1] - q_off[p], m = s_off[p + 1] - s_off[p];
        float c = y[2 * p], lw = y[2 * p + 1];
        c = fminf(fmaxf(c, -1e6f), 1e6f);
        // the network gives the half-width relative to the longer sequence (the
        // certificate's margin grows with the length times the divergence, and the
        // features see the divergence, not the length)
        lw = fminf(fmaxf(lw, -16.0f), 1.0f);
        const float L = (float)(n > m ? n : m);
        // the target is the narrowest certifying width of a doubling series, so a width
        // just below it fails the certificate and pays for the full DP too: a margin
        const float wf = fminf(fmaxf(expf(lw) * caps.margin, caps.floor) * L, 1.0e9f);
        int32_t w = (int32_t)ceilf(wf);
        w = w < MIN_W ? MIN_W : w;
        // the path starts on the line: a shift beyond the top half-width cannot hold it
        c = fminf(fmaxf(c, -(float)w), (float)w);
        centre[p] = (int32_t)rintf(c);
        width[p] = w;
        const bool too_wide = band_area(n, w) > band_cap(caps, n, m) * (double)n * (double)m;
        if (n == 0 || m == 0 || too_wide) {
            full[p] = 1;
        } else {
            full[p] = 0;
            unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long *>(count), 1ull);
            list[pos] = (int32_t)p;
        }
    }
}

// After a banded round: accepted pairs get their result, the others double
// their band or move to the full DP.
__global__ void band_round_kernel(const int32_t *list, int64_t n_list, const int64_t *q_off, const int64_t *s_off,
                                  const int32_t *bscore, const int32_t *accept, int32_t *width, uint8_t *full,
                                  int32_t *next, int64_t *next_count, int32_t round, int32_t last_round,
                                  BandCaps caps, int32_t *score, int32_t *eq, int32_t *es, uint32_t *flags) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_list;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = list[k];
        const int64_t n = q_off[p + 1] - q_off[p], m = s_off[p + 1] - s_off[p];
        if (accept[p]) {
            score[p] = bscore[p];
            eq[p] = (int32_t)n;
            es[p] = (int32_t)m;
            flags[p] = ANYSEQ_FLAG_INT32 | ANYSEQ_FLAG_BAND_ACCEPTED | ((uint32_t)round << 8);
        } else {
            const int32_t w = width[p] * 2;
            width[p] = w;
            if (last_round || band_area(n, w) > band_cap(caps, n, m) * (double)n * (double)m) {
                full[p] = 1;
            } else {
                unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long *>(next_count), 1ull);
                next[pos] = p;
            }
        }
    }
}

__global__ void mark_full_kernel(const uint8_t *full, int64_t n_pairs, uint32_t *flags, int32_t rounds) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += (int64_t)gridDim.x * blockDim.x)
        if (full[p]) flags[p] |= ANYSEQ_FLAG_FULL_FALLBACK | ((uint32_t)rounds << 8);
}

// training targets: centre of the path and log of the certified half-width
// relative to the longer sequence
__global__ void band_targets_kernel(const int32_t *dmin, const int32_t *dmax, const int32_t *wcert, int64_t n,
                                    const int64_t *q_off, const int64_t *s_off, float *target) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t qn = q_off[p + 1] - q_off[p], sm = s_off[p + 1] - s_off[p];
        const float L = (float)(qn > sm ? qn : sm);
        target[2 * p] = 0.5f * (float)(dmin[p] + dmax[p]);
        target[2 * p + 1] = logf((float)wcert[p] / (L > 1.0f ? L : 1.0f));
    }
}

// host wall clock in ms (the banded route synchronises between its phases)
static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int grid_of(int64_t work) {
    int64_t b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

// ------------------------------------------------------------ shared helpers

static anyseq_status_t pack_batch(anyseq_ctx *ctx, const BatchInput &in, int32_t alphabet, uint32_t **q2, uint32_t **s2,
                                  cudaStream_t st) {
    anyseq_status_t s2st = ANYSEQ_OK;
    *q2 = arena_b<uint32_t>(ctx, "b_q2", (size_t)(in.q_len + 15) / 16 + 2, &s2st);
    *s2 = arena_b<uint32_t>(ctx, "b_s2", (size_t)(in.s_len + 15) / 16 + 2, &s2st);
    int32_t *bad = arena_b<int32_t>(ctx, "b_bad", 4, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    BCUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
    BCUDA(launch_pack2bit(in.q, in.q_len, *q2, alphabet, bad, st));
    BCUDA(launch_pack2bit(in.s, in.s_len, *s2, alphabet, bad, st));
    ctx->launches += 2;
    int32_t hb = 0;
    BCUDA(cudaMemcpyAsync(&hb, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    if (hb) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", alphabet);
    return ANYSEQ_OK;
}

// Order a pass's pairs so that the two slots of a warp hold pairs of one chunk
// count and similar band: the warp runs as many chunks as its longer query needs
// and as many steps per chunk as its wider window, and the other slot computes
// columns nobody reads meanwhile. So: queries in 64-row classes (the shortest
// chunk) longest first, then within a class the band width, widest first, then
// the lengths. (Sorted by lengths alone, two pairs of one length could differ
// several-fold in band width.)
static anyseq_status_t sort_pass(const std::vector<int64_t> &hq, const std::vector<int64_t> &hs, const int32_t *width,
                                 int64_t n_pairs, int32_t *list, int64_t n_list, cudaStream_t st) {
    if (n_list < 2) return ANYSEQ_OK;
    std::vector<int32_t> h((size_t)n_list), hw((size_t)n_pairs);
    BCUDA(cudaMemcpyAsync(h.data(), list, (size_t)n_list * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaMemcpyAsync(hw.data(), width, (size_t)n_pairs * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    std::stable_sort(h.begin(), h.end(), [&](int32_t a, int32_t b) {
        const int64_t na = hq[a + 1] - hq[a], nb = hq[b + 1] - hq[b];
        if (na / 64 != nb / 64) return na > nb;
        if (hw[a] != hw[b]) return hw[a] > hw[b];
        if (na != nb) return na > nb;
        return hs[a + 1] - hs[a] > hs[b + 1] - hs[b];
    });
    BCUDA(cudaMemcpyAsync(list, h.data(), (size_t)n_list * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    BCUDA(cudaStreamSynchronize(st));
    return ANYSEQ_OK;
}

// One banded pass over list (centre, width per pair): scores and accept flags.
static anyseq_status_t banded_pass(anyseq_ctx *ctx, const BatchInput &in, const anyseq_scoring_t *sc,
                                   const uint32_t *q2, const uint32_t *s2, const int32_t *list, int64_t n_list,
                                   const int32_t *centre, const int32_t *width, bool strict, int32_t *bscore,
                                   int32_t *accept, cudaStream_t st) {
    anyseq_status_t s2st = ANYSEQ_OK;
    BandArgs A;
    memset(&A, 0, sizeof(A));
    A.q2 = q2; A.s2 = s2; A.q_off = in.q_off; A.s_off = in.s_off;
    A.list = list; A.n_list = n_list;
    A.centre = centre; A.width = width;
    BTRY(make_rowprof(sc, ANYSEQ_GLOBAL, A.rowprof));
    A.o = sc->gap_open; A.e = sc->gap_extend;
    int32_t mmax = -(1 << 30);
    for (int a = 0; a < sc->alphabet; a++)
        for (int b = 0; b < sc->alphabet; b++) mmax = std::max(mmax, sigma_host(sc, a, b));
    A.mmax = mmax;
    A.strict = strict ? 1 : 0;
    const int grid = ctx->num_sms * band_blocks_per_sm();
    A.scratch_cols = in.max_m + 1;
    A.scratch = arena_b<int32_t>(ctx, "b_border", (size_t)grid * 16 * 2 * (size_t)A.scratch_cols, &s2st);
    A.counter = arena_b<int32_t>(ctx, "b_counter", 4, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    A.score = bscore;
    A.accept = accept;
    A.cells = reinterpret_cast<unsigned long long *>(arena_b<int64_t>(ctx, "b_cells", 2, &s2st));
    if (s2st != ANYSEQ_OK) return s2st;
    BCUDA(cudaMemsetAsync(A.cells, 0, sizeof(int64_t), st));
    BCUDA(cudaMemsetAsync(A.counter, 0, sizeof(int32_t), st));
    BCUDA(launch_band(A, grid, st));
    ctx->launches += 1;
    int64_t hc = 0;
    BCUDA(cudaMemcpyAsync(&hc, A.cells, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    ctx->band_cells += hc;
    return ANYSEQ_OK;
}

// --------------------------------------------------------------- inference

anyseq_status_t anyseq::band_scores(anyseq_ctx *ctx, const BatchInput &in, const anyseq_scoring_t *sc, int32_t *score,
                                    int32_t *eq, int32_t *es, uint32_t *flags, cudaStream_t st) {
    if (!ctx->mlp_ready) return fail(ANYSEQ_ERR_ARG, "ANYSEQ_BAND_LEARNED needs a band model (train, load or set one)");
    anyseq_status_t s2st = ANYSEQ_OK;
    const int64_t n = in.n_pairs;
    BCUDA(cudaStreamSynchronize(st));
    const double t_start = now_ms();
    uint32_t *q2, *s2;
    BTRY(pack_batch(ctx, in, sc->alphabet, &q2, &s2, st));
    float *feat = arena_b<float>(ctx, "b_feat", (size_t)n * MLP_IN + 1, &s2st);
    float *y = arena_b<float>(ctx, "b_y", (size_t)n * 2 + 1, &s2st);
    int32_t *centre = arena_b<int32_t>(ctx, "b_centre", n + 1, &s2st);
    int32_t *width = arena_b<int32_t>(ctx, "b_width", n + 1, &s2st);
    uint8_t *full = arena_b<uint8_t>(ctx, "b_full", n + 16, &s2st);
    int32_t *listA = arena_b<int32_t>(ctx, "b_listA", n + 1, &s2st);
    int32_t *listB = arena_b<int32_t>(ctx, "b_listB", n + 1, &s2st);
    int32_t *bscore = arena_b<int32_t>(ctx, "b_bscore", n + 1, &s2st);
    int32_t *accept = arena_b<int32_t>(ctx, "b_accept", n + 1, &s2st);
    int64_t *cnt = arena_b<int64_t>(ctx, "b_cnt", 4, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    BCUDA(launch_kmer_hist(q2, s2, in.q_off, in.s_off, nullptr, n, feat, st));
    BCUDA(launch_mlp_forward(mlp_dev(ctx), feat, n, y, st));
    BCUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(int64_t), st));
    BandCaps caps;
    caps.area32 = ctx->band_area_pct / 100.0;
    caps.area16 = ctx->band_area16_pct / 100.0;
    caps.margin = (float)ctx->band_margin_pct / 100.0f;
    caps.floor = (float)ctx->band_floor_pct / 100.0f;
    caps.smax = -(1 << 30);
    caps.smin = 1 << 30;
    for (int a = 0; a < sc->alphabet; a++)
        for (int b = 0; b < sc->alphabet; b++) {
            caps.smax = std::max(caps.smax, sigma_host(sc, a, b));
            caps.smin = std::min(caps.smin, sigma_host(sc, a, b));
        }
    caps.o = sc->gap_open;
    caps.e = sc->gap_extend;
    if (ctx->force32) caps.area16 = caps.area32;
    band_plan_kernel<<<grid_of(n), 256, 0, st>>>(y, in.q_off, in.s_off, n, caps, centre, width, full, listA, cnt);
    BCUDA(cudaGetLastError());
    ctx->launches += 3;
    int64_t n_list = 0;
    BCUDA(cudaMemcpyAsync(&n_list, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    const double t_plan = now_ms();
    ctx->band_plan_ms = t_plan - t_start;
    ctx->band_cells = 0;
    ctx->band_rounds = 0;
    ctx->band_accepted = 0;
    int32_t round = 0;
    const int64_t n_first = n_list;
    std::vector<int64_t> hq((size_t)n + 1), hs((size_t)n + 1);
    BCUDA(cudaMemcpyAsync(hq.data(), in.q_off, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaMemcpyAsync(hs.data(), in.s_off, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    while (n_list > 0) {
        BTRY(sort_pass(hq, hs, width, n, listA, n_list, st));
        BTRY(banded_pass(ctx, in, sc, q2, s2, listA, n_list, centre, width, false, bscore, accept, st));
        BCUDA(cudaMemsetAsync(cnt + 1, 0, sizeof(int64_t), st));
        band_round_kernel<<<grid_of(n_list), 256, 0, st>>>(listA, n_list, in.q_off, in.s_off, bscore, accept, width,
                                                           full, listB, cnt + 1, round,
                                                           round >= ctx->band_max_doublings ? 1 : 0, caps, score,
                                                           eq, es, flags);
        BCUDA(cudaGetLastError());
        ctx->launches += 1;
        int64_t next = 0;
        BCUDA(cudaMemcpyAsync(&next, cnt + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        BCUDA(cudaStreamSynchronize(st));
        ctx->band_rounds++;
        std::swap(listA, listB);
        n_list = next;
        round++;
    }
    const double t_bands = now_ms();
    ctx->band_pass_ms = t_bands - t_plan;
    // everything not accepted: the full DP, restricted to the marked pairs. The few
    // fallback pairs far above the others' size would each hold one 16-lane group
    // for longer than the rest of the launch takes, so pairs above the selection's
    // cells per resident group run on the wavefront first.
    BatchInput sub = in;
    sub.select = full;
    BatchInput rest = sub;
    bool all_wave = false;
    if (!ctx->force32)
        BTRY(long_pairs_split(ctx, sub, sc, ANYSEQ_GLOBAL, score, eq, es, flags, st, rest, &all_wave, 1.0));
    if (!all_wave) BTRY(batch_scores(ctx, rest, sc, ANYSEQ_GLOBAL, score, eq, es, flags, st));
    mark_full_kernel<<<grid_of(n), 256, 0, st>>>(full, n, flags, round);
    BCUDA(cudaGetLastError());
    ctx->launches += 1;
    std::vector<uint8_t> hfull(n);
    BCUDA(cudaMemcpyAsync(hfull.data(), full, n, cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    int64_t nf = 0;
    for (int64_t p = 0; p < n; p++) nf += hfull[p] != 0;
    ctx->band_fallback = nf;
    ctx->band_accepted = n - nf;
    ctx->band_full_ms = now_ms() - t_bands;
    (void)n_first;
    return ANYSEQ_OK;
}

// -------------------------------------------------------------- entry points

extern "C" anyseq_status_t anyseq_band_features(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off,
                                                const uint8_t *s, const int64_t *s_off, int64_t n_pairs,
                                                float *features, void *cuda_stream) {
    if (!ctx || !features || n_pairs < 0) return fail(ANYSEQ_ERR_ARG, "bad arguments");
    if (n_pairs == 0) return ANYSEQ_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    anyseq_status_t s2st = ANYSEQ_OK;
    ctx->launches = 0;
    BatchInput in;
    BTRY(stage_batch(ctx, q, q_off, s, s_off, n_pairs, in, st));
    uint32_t *q2, *s2;
    BTRY(pack_batch(ctx, in, 4, &q2, &s2, st));
    const bool dev = is_device_ptr(features);
    float *f = dev ? features : arena_b<float>(ctx, "b_feat_out", (size_t)n_pairs * MLP_IN, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    BCUDA(launch_kmer_hist(q2, s2, in.q_off, in.s_off, nullptr, n_pairs, f, st));
    ctx->launches += 1;
    if (!dev) BCUDA(cudaMemcpyAsync(features, f, (size_t)n_pairs * MLP_IN * sizeof(float), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_band_model_get(anyseq_ctx *ctx, float *params, int64_t count) {
    if (!ctx || !params || count != NP) return fail(ANYSEQ_ERR_ARG, "expected %lld parameters", (long long)NP);
    if (!ctx->mlp_ready) return fail(ANYSEQ_ERR_ARG, "no band model");
    BCUDA(cudaMemcpy(params, ctx->mlp, NP * sizeof(float), cudaMemcpyDefault));
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_band_model_set(anyseq_ctx *ctx, const float *params, int64_t count) {
    if (!ctx || !params || count != NP) return fail(ANYSEQ_ERR_ARG, "expected %lld parameters", (long long)NP);
    return set_params(ctx, params, nullptr);
}

extern "C" anyseq_status_t anyseq_band_model_save(anyseq_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(ANYSEQ_ERR_ARG, "bad arguments");
    if (!ctx->mlp_ready) return fail(ANYSEQ_ERR_ARG, "no band model");
    std::vector<float> h(NP);
    BCUDA(cudaMemcpy(h.data(), ctx->mlp, NP * sizeof(float), cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ANYSEQ_ERR_ARG, "cannot write %s", path);
    const char magic[8] = {'A', 'N', 'Y', 'S', 'E', 'Q', 'B', '1'};
    int64_t cnt = NP;
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&cnt, sizeof(cnt), 1, f) == 1 &&
              fwrite(h.data(), sizeof(float), NP, f) == (size_t)NP;
    fclose(f);
    return ok ? ANYSEQ_OK : fail(ANYSEQ_ERR_ARG, "short write to %s", path);
}

extern "C" anyseq_status_t anyseq_band_model_load(anyseq_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(ANYSEQ_ERR_ARG, "bad arguments");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ANYSEQ_ERR_ARG, "cannot read %s", path);
    char magic[8];
    int64_t cnt = 0;
    std::vector<float> h(NP);
    bool ok = fread(magic, 1, 8, f) == 8 && !memcmp(magic, "ANYSEQB1", 8) && fread(&cnt, sizeof(cnt), 1, f) == 1 &&
              cnt == NP && fread(h.data(), sizeof(float), NP, f) == (size_t)NP;
    fclose(f);
    if (!ok) return fail(ANYSEQ_ERR_ARG, "%s is not a band model", path);
    return set_params(ctx, h.data(), nullptr);
}

extern "C" anyseq_status_t anyseq_band_forward(anyseq_ctx *ctx, const float *x, int64_t B, float *y, void *cuda_stream) {
    if (!ctx || !x || !y || B < 0) return fail(ANYSEQ_ERR_ARG, "bad arguments");
    if (!ctx->mlp_ready) return fail(ANYSEQ_ERR_ARG, "no band model");
    if (B == 0) return ANYSEQ_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const void *dx;
    BTRY(stage_input(ctx, "bf_x", x, (size_t)B * MLP_IN * sizeof(float), st, &dx));
    anyseq_status_t s2st = ANYSEQ_OK;
    const bool dev = is_device_ptr(y);
    float *dy = dev ? y : arena_b<float>(ctx, "bf_y", (size_t)B * 2, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    BCUDA(launch_mlp_forward(mlp_dev(ctx), (const float *)dx, B, dy, st));
    if (!dev) BCUDA(cudaMemcpyAsync(y, dy, (size_t)B * 2 * sizeof(float), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_band_gradient(anyseq_ctx *ctx, const float *x, const float *targets, int64_t B,
                                                float *grad, float *loss, void *cuda_stream) {
    if (!ctx || !x || !targets || !grad || B <= 0) return fail(ANYSEQ_ERR_ARG, "bad arguments");
    if (!ctx->mlp_ready) return fail(ANYSEQ_ERR_ARG, "no band model");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const void *dx, *dt;
    BTRY(stage_input(ctx, "bg_x", x, (size_t)B * MLP_IN * sizeof(float), st, &dx));
    BTRY(stage_input(ctx, "bg_t", targets, (size_t)B * 2 * sizeof(float), st, &dt));
    anyseq_status_t s2st = ANYSEQ_OK;
    float *dl = arena_b<float>(ctx, "bg_loss", 4, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    MlpDev P = mlp_dev(ctx);
    BCUDA(cudaMemsetAsync(P.grad, 0, NP * sizeof(float), st));
    BCUDA(cudaMemsetAsync(dl, 0, sizeof(float), st));
    BCUDA(launch_mlp_grad(P, (const float *)dx, (const float *)dt, B, dl, st));
    BCUDA(cudaMemcpyAsync(grad, P.grad, NP * sizeof(float), cudaMemcpyDefault, st));
    float hl = 0;
    BCUDA(cudaMemcpyAsync(&hl, dl, sizeof(float), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    if (loss) *loss = hl / (float)B;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_band_train(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off,
                                             const uint8_t *s, const int64_t *s_off, int64_t n_pairs,
                                             const anyseq_scoring_t *sc, int32_t epochs, float lr, float *loss,
                                             void *cuda_stream) {
    if (!ctx || n_pairs <= 0 || epochs < 0 || !(lr > 0)) return fail(ANYSEQ_ERR_ARG, "bad arguments");
    BTRY(check_scoring(sc, ANYSEQ_GLOBAL));
    if (sc->alphabet > 4) return fail(ANYSEQ_ERR_ARG, "the band model is for DNA (alphabet <= 4)");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    anyseq_status_t s2st = ANYSEQ_OK;
    BatchInput in;
    BTRY(stage_batch(ctx, q, q_off, s, s_off, n_pairs, in, st));
    const int64_t n = n_pairs;
    // 1. optimal paths by the full DP with traceback
    anyseq_result_t *res = arena_b<anyseq_result_t>(ctx, "bt_res", n + 1, &s2st);
    const uint64_t cap = (uint64_t)(in.q_len + in.s_len + n + 16);
    uint32_t *cig = arena_b<uint32_t>(ctx, "bt_cig", cap, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    uint64_t used = 0;
    BTRY(anyseq_align_batch(ctx, in.q, in.q_off, in.s, in.s_off, n, sc, ANYSEQ_GLOBAL,
                            ANYSEQ_WANT_SCORE | ANYSEQ_WANT_CIGAR, res, cig, cap, &used, cuda_stream));
    // 2. path extents and centres
    int32_t *dmin = arena_b<int32_t>(ctx, "bt_dmin", n + 1, &s2st);
    int32_t *dmax = arena_b<int32_t>(ctx, "bt_dmax", n + 1, &s2st);
    int32_t *centre = arena_b<int32_t>(ctx, "bt_centre", n + 1, &s2st);
    int32_t *width = arena_b<int32_t>(ctx, "bt_width", n + 1, &s2st);
    int32_t *list = arena_b<int32_t>(ctx, "bt_list", n + 1, &s2st);
    int32_t *bscore = arena_b<int32_t>(ctx, "bt_bscore", n + 1, &s2st);
    int32_t *accept = arena_b<int32_t>(ctx, "bt_accept", n + 1, &s2st);
    float *feat = arena_b<float>(ctx, "bt_feat", (size_t)n * MLP_IN + 1, &s2st);
    float *target = arena_b<float>(ctx, "bt_target", (size_t)n * 2 + 1, &s2st);
    float *dl = arena_b<float>(ctx, "bt_loss", 4, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    BCUDA(launch_path_extent(in.q_off, in.s_off, res, cig, n, dmin, dmax, st));
    std::vector<int32_t> hmin(n), hmax(n), hc(n), hw(n), wcert(n);
    std::vector<int64_t> qo(n + 1), so(n + 1);
    BCUDA(cudaMemcpyAsync(hmin.data(), dmin, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaMemcpyAsync(hmax.data(), dmax, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaMemcpyAsync(qo.data(), in.q_off, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaMemcpyAsync(so.data(), in.s_off, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BCUDA(cudaStreamSynchronize(st));
    // 3. smallest doubling width at which the band around the path centre passes the certificate
    uint32_t *q2, *s2;
    BTRY(pack_batch(ctx, in, sc->alphabet, &q2, &s2, st));
    std::vector<int32_t> pending;
    for (int64_t p = 0; p < n; p++) {
        hc[p] = (int32_t)std::lround(0.5 * (hmin[p] + hmax[p]));
        hw[p] = std::max(MIN_W, (hmax[p] - hmin[p] + 1) / 2 + 4);
        const int64_t qn = qo[p + 1] - qo[p], sm = so[p + 1] - so[p];
        wcert[p] = (int32_t)std::max<int64_t>(std::max(qn, sm), MIN_W);
        if (qn > 0 && sm > 0) pending.push_back((int32_t)p);
    }
    std::vector<int32_t> hacc(n);
    BCUDA(cudaMemcpyAsync(centre, hc.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    for (int round = 0; !pending.empty() && round < 12; round++) {
        BCUDA(cudaMemcpyAsync(width, hw.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        BCUDA(cudaMemcpyAsync(list, pending.data(), pending.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        BTRY(banded_pass(ctx, in, sc, q2, s2, list, (int64_t)pending.size(), centre, width, false, bscore, accept, st));
        BCUDA(cudaMemcpyAsync(hacc.data(), accept, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        BCUDA(cudaStreamSynchronize(st));
        std::vector<int32_t> next;
        for (int32_t p : pending) {
            const int64_t qn = qo[p + 1] - qo[p], sm = so[p + 1] - so[p];
            if (hacc[p]) {
                wcert[p] = hw[p];
            } else {
                hw[p] *= 2;
                if (band_area(qn, hw[p]) <= 0.5 * (double)qn * (double)sm) next.push_back(p);
            }
        }
        pending.swap(next);
    }
    // 4. features and targets (centre of the path, log of the certified width)
    BCUDA(cudaMemcpyAsync(width, wcert.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    BCUDA(launch_kmer_hist(q2, s2, in.q_off, in.s_off, nullptr, n, feat, st));
    band_targets_kernel<<<grid_of(n), 256, 0, st>>>(dmin, dmax, width, n, in.q_off, in.s_off, target);
    BCUDA(cudaGetLastError());
    // 5. Adam over mini-batches
    if (!ctx->mlp_ready) {
        std::vector<float> w0;
        init_params(w0, 0x5EEDBA4Dull);
        BTRY(set_params(ctx, w0.data(), st));
    }
    MlpDev P = mlp_dev(ctx);
    BCUDA(cudaMemsetAsync(P.m, 0, 2 * NP * sizeof(float), st));
    const int64_t MB = 1024;
    int64_t step = 0;
    float last = 0;
    for (int32_t ep = 0; ep < epochs; ep++) {
        BCUDA(cudaMemsetAsync(dl, 0, sizeof(float), st));
        for (int64_t b0 = 0; b0 < n; b0 += MB) {
            const int64_t B = std::min(MB, n - b0);
            BCUDA(cudaMemsetAsync(P.grad, 0, NP * sizeof(float), st));
            BCUDA(launch_mlp_grad(P, feat + b0 * MLP_IN, target + b0 * 2, B, dl, st));
            BCUDA(launch_mlp_adam(P, ++step, lr, st));
        }
        if (ep == epochs - 1) {
            BCUDA(cudaMemcpyAsync(&last, dl, sizeof(float), cudaMemcpyDeviceToHost, st));
            BCUDA(cudaStreamSynchronize(st));
        }
    }
    BCUDA(cudaStreamSynchronize(st));
    if (loss) *loss = last / (float)n;
    return ANYSEQ_OK;
}
