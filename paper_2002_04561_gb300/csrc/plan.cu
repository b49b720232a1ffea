// Graph plans: one batch shape (offsets, scoring, mode) whose whole launch
// sequence of the batched path (pack and validate, range test and length
// binning, the persistent DP kernels, result records) is captured once in a
// CUDA graph and replayed. For callers that align batches of the same shape
// again and again (a benchmark loop, a serving tier with fixed batch slots),
// a replay costs one graph launch instead of ten kernel launches and the host
// work between them.
//
// A plan owns its device buffers and a private context, so no other call can
// move the scratch the graph points at. The first run executes the sequence
// once without capture (sizing every scratch buffer), then captures it; later
// runs launch the graph. Letters are checked on every run: the flag is copied
// to pinned host memory inside the graph and read by anyseq_plan_wait.
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/anyseq.h"
#include "api_internal.h"

struct anyseq_plan {
    anyseq_ctx *ctx = nullptr;
    anyseq::BatchInput in;
    anyseq_scoring_t sc{};
    std::vector<int8_t> matrix;
    int32_t mode = 0;
    uint8_t *q = nullptr, *s = nullptr;
    int64_t *q_off = nullptr, *s_off = nullptr;
    anyseq_result_t *out = nullptr;
    int32_t *score = nullptr, *eq = nullptr, *es = nullptr;
    uint32_t *flags = nullptr;
    int32_t *h_bad = nullptr;  // pinned
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t runs = 0;
};

using anyseq::fail;

namespace {

// The launch sequence of one run (capturable: no host synchronisation).
anyseq_status_t enqueue(anyseq_plan *P, cudaStream_t st, bool capture) {
    const anyseq_status_t s2 = anyseq::batch_scores(P->ctx, P->in, &P->sc, P->mode, P->score, P->eq, P->es,
                                                    P->flags, st, nullptr, capture);
    if (s2 != ANYSEQ_OK) return s2;
    cudaError_t e = anyseq::launch_write_results(P->in.n_pairs, P->score, P->eq, P->es, P->flags, P->out, st);
    if (e == cudaSuccess && capture)
        e = cudaMemcpyAsync(P->h_bad, P->ctx->bad_code, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "plan launch: %s", cudaGetErrorString(e));
    return ANYSEQ_OK;
}

void release(anyseq_plan *P) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    cudaFree(P->q);
    cudaFree(P->s);
    cudaFree(P->q_off);
    cudaFree(P->s_off);
    cudaFree(P->out);
    cudaFree(P->score);
    cudaFree(P->eq);
    cudaFree(P->es);
    cudaFree(P->flags);
    if (P->h_bad) cudaFreeHost(P->h_bad);
    if (P->ctx) anyseq_destroy(P->ctx);
    delete P;
}

}  // namespace

extern "C" anyseq_status_t anyseq_plan_create(anyseq_plan **out, int device, const int64_t *q_off,
                                              const int64_t *s_off, int64_t n_pairs, const anyseq_scoring_t *sc,
                                              int32_t mode) {
    if (!out || !q_off || !s_off) return fail(ANYSEQ_ERR_ARG, "plan, q_off and s_off must not be NULL");
    *out = nullptr;
    if (n_pairs < 1 || n_pairs >= (1ll << 31) - 2) return fail(ANYSEQ_ERR_ARG, "n_pairs out of range");
    const anyseq_status_t sst = anyseq::check_scoring(sc, mode);
    if (sst != ANYSEQ_OK) return sst;
    if (anyseq::is_device_ptr(q_off) || anyseq::is_device_ptr(s_off))
        return fail(ANYSEQ_ERR_ARG, "plan offsets are host arrays");
    anyseq::BatchInput in;
    in.n_pairs = n_pairs;
    if (q_off[0] != 0 || s_off[0] != 0) return fail(ANYSEQ_ERR_ARG, "offsets must start at 0");
    for (int64_t p = 0; p < n_pairs; p++) {
        const int64_t n = q_off[p + 1] - q_off[p], m = s_off[p + 1] - s_off[p];
        if (n < 0 || m < 0 || n >= (1 << 21) || m >= (1 << 21))
            return fail(ANYSEQ_ERR_ARG, "offsets must be non-decreasing and give lengths below 2^21");
        in.max_n = n > in.max_n ? n : in.max_n;
        in.max_m = m > in.max_m ? m : in.max_m;
    }
    in.q_len = q_off[n_pairs];
    in.s_len = s_off[n_pairs];
    anyseq_plan *P = new anyseq_plan();
    P->mode = mode;
    P->sc = *sc;
    if (sc->matrix) {
        P->matrix.assign(sc->matrix, sc->matrix + (size_t)sc->alphabet * sc->alphabet);
        P->sc.matrix = P->matrix.data();
    }
    anyseq_status_t st = anyseq_create(&P->ctx, device, 0);
    if (st != ANYSEQ_OK) {
        delete P;
        return st;
    }
    const size_t n1 = (size_t)n_pairs + 1;
    cudaError_t e = cudaMalloc(&P->q, (size_t)in.q_len + 16);
    if (e == cudaSuccess) e = cudaMalloc(&P->s, (size_t)in.s_len + 16);
    if (e == cudaSuccess) e = cudaMalloc(&P->q_off, n1 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&P->s_off, n1 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&P->out, (size_t)n_pairs * sizeof(anyseq_result_t));
    if (e == cudaSuccess) e = cudaMalloc(&P->score, (size_t)n_pairs * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&P->eq, (size_t)n_pairs * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&P->es, (size_t)n_pairs * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&P->flags, (size_t)n_pairs * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&P->h_bad, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemcpy(P->q_off, q_off, n1 * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->s_off, s_off, n1 * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(P->q, 0, (size_t)in.q_len + 16);
    if (e == cudaSuccess) e = cudaMemset(P->s, 0, (size_t)in.s_len + 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(P);
        return fail(ANYSEQ_ERR_CUDA, "plan buffers: %s", cudaGetErrorString(e));
    }
    *P->h_bad = 0;
    in.q = P->q;
    in.s = P->s;
    in.q_off = P->q_off;
    in.s_off = P->s_off;
    P->in = in;
    *out = P;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_plan_buffers(anyseq_plan *P, uint8_t **q, uint8_t **s, anyseq_result_t **out) {
    if (!P) return fail(ANYSEQ_ERR_ARG, "plan is NULL");
    if (q) *q = P->q;
    if (s) *s = P->s;
    if (out) *out = P->out;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_plan_run(anyseq_plan *P, void *cuda_stream) {
    if (!P) return fail(ANYSEQ_ERR_ARG, "plan is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(P->ctx->device) != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "cudaSetDevice failed");
    if (!P->exec) {
        // first run: execute (sizing every scratch buffer; the batched path checks the
        // letters and synchronises), then capture the same sequence
        anyseq_status_t s2 = enqueue(P, st, false);
        if (s2 != ANYSEQ_OK) return s2;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "plan warm-up: %s", cudaGetErrorString(e));
        *P->h_bad = 0;
        cudaStream_t cap = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            if (cap) cudaStreamDestroy(cap);
            return fail(ANYSEQ_ERR_CUDA, "plan capture: %s", cudaGetErrorString(e));
        }
        s2 = enqueue(P, cap, true);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (s2 != ANYSEQ_OK) {
            if (g) cudaGraphDestroy(g);
            return s2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, g, 0);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return fail(ANYSEQ_ERR_CUDA, "plan graph: %s", cudaGetErrorString(e));
        }
        P->graph = g;
        P->runs = 1;
        return ANYSEQ_OK;  // the warm-up produced this run's results
    }
    const cudaError_t e = cudaGraphLaunch(P->exec, st);
    if (e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "plan replay: %s", cudaGetErrorString(e));
    P->runs++;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_plan_upload(anyseq_plan *P, const uint8_t *q, const uint8_t *s,
                                              void *cuda_stream) {
    if (!P) return fail(ANYSEQ_ERR_ARG, "plan is NULL");
    if ((P->in.q_len > 0 && !q) || (P->in.s_len > 0 && !s)) return fail(ANYSEQ_ERR_ARG, "q or s is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(P->ctx->device) != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "cudaSetDevice failed");
    cudaError_t e = cudaSuccess;
    if (P->in.q_len > 0) e = cudaMemcpyAsync(P->q, q, (size_t)P->in.q_len, cudaMemcpyDefault, st);
    if (e == cudaSuccess && P->in.s_len > 0) e = cudaMemcpyAsync(P->s, s, (size_t)P->in.s_len, cudaMemcpyDefault, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ANYSEQ_ERR_CUDA, "plan upload: %s", cudaGetErrorString(e));
    }
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_plan_download(anyseq_plan *P, anyseq_result_t *out, void *cuda_stream) {
    if (!P || !out) return fail(ANYSEQ_ERR_ARG, "plan or out is NULL");
    if (cudaSetDevice(P->ctx->device) != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "cudaSetDevice failed");
    const cudaError_t e = cudaMemcpyAsync(out, P->out, (size_t)P->in.n_pairs * sizeof(anyseq_result_t),
                                          cudaMemcpyDefault, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ANYSEQ_ERR_CUDA, "plan download: %s", cudaGetErrorString(e));
    }
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_plan_wait(anyseq_plan *P, void *cuda_stream) {
    if (!P) return fail(ANYSEQ_ERR_ARG, "plan is NULL");
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "plan wait: %s", cudaGetErrorString(e));
    if (*P->h_bad) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", P->sc.alphabet);
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_plan_destroy(anyseq_plan *P) {
    if (!P) return ANYSEQ_OK;
    cudaDeviceSynchronize();
    release(P);
    return ANYSEQ_OK;
}
