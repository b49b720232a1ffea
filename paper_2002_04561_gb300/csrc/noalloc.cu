// Global score of one long pair without any device memory allocation.
//
// Some callers cannot let this library allocate device memory: a host process
// whose framework owns all device memory through its own pool, or a
// latency-bound service that cannot accept the implicit synchronisation of
// cudaMalloc/cudaFree. For them this entry point runs the wavefront pass of
// anyseq_align_long on scratch that lives in one file-scope device array,
// sized for sequences of up to ANYSEQ_NOALLOC_MAX_LEN letters. Every GPU that
// loads the library holds that array (about 21 MB) until the process exits.
//
// The array is shared by every call: calls that overlap on the GPU (on two
// streams, or from two host threads) race on it. Each call clears the parts
// that must start at zero (progress counters, error flags) itself.
#include <cstring>
#include <mutex>

#include "../../include/anyseq.h"
#include "api_internal.h"
#include "batch.h"
#include "common.cuh"
#include "wave.h"

namespace anyseq {

constexpr int64_t NA_MAX = ANYSEQ_NOALLOC_MAX_LEN;
constexpr int64_t NA_PACKED = NA_MAX / 16 + 4;                   // uint32 words per packed sequence
constexpr int64_t NA_STRIPES = (NA_MAX + WAVE_MIN_ROWS - 1) / WAVE_MIN_ROWS;  // the shortest stripes
constexpr int64_t NA_CTL = NA_STRIPES + 8;                       // counter, error flag, progress counters
// byte offsets inside the array (each 256-byte aligned)
constexpr int64_t al(int64_t x) { return (x + 255) / 256 * 256; }
constexpr int64_t NA_OFF_Q2 = 0;
constexpr int64_t NA_OFF_S2 = al(NA_OFF_Q2 + NA_PACKED * 4);
constexpr int64_t NA_OFF_BORDER = al(NA_OFF_S2 + NA_PACKED * 4);
constexpr int64_t NA_OFF_H = al(NA_OFF_BORDER + 2 * NA_MAX * 8);
constexpr int64_t NA_OFF_CTL = al(NA_OFF_H + (NA_MAX + 1) * 4);
constexpr int64_t NA_OFF_PASS = al(NA_OFF_CTL + NA_CTL * 4);
constexpr int64_t NA_OFF_BAD = al(NA_OFF_PASS + (int64_t)sizeof(WavePass));
constexpr int64_t NA_BYTES = al(NA_OFF_BAD + 16);

static __device__ __align__(256) uint8_t g_noalloc_scratch[NA_BYTES];

__global__ void noalloc_init_kernel(WavePass *pass, WavePass value, int32_t *ctl, int64_t nctl, int32_t *bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        *pass = value;
        *bad = 0;
    }
    for (int64_t k = t; k < nctl; k += (int64_t)gridDim.x * blockDim.x) ctl[k] = 0;
}

// True when p is device (or managed) memory of device dev.
static bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

__global__ void noalloc_finish_kernel(const int32_t *H, int32_t m, int32_t *score) { *score = H[m]; }

// Device address of the array on the current device, resolved once per device.
static anyseq_status_t scratch_address(uint8_t **out) {
    static std::mutex mu;
    static uint8_t *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail(ANYSEQ_ERR_CUDA, "no current CUDA device");
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (rc != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(ANYSEQ_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(rc));
        }
        addr[dev] = static_cast<uint8_t *>(p);
    }
    *out = addr[dev];
    return ANYSEQ_OK;
}

}  // namespace anyseq

using namespace anyseq;

extern "C" anyseq_status_t anyseq_align_long_noalloc(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m,
                                                     const anyseq_scoring_t *sc, int32_t *score, void *cuda_stream) {
    anyseq_status_t st2 = check_scoring(sc, ANYSEQ_GLOBAL);
    if (st2 != ANYSEQ_OK) return st2;
    if (sc->alphabet > 4) return fail(ANYSEQ_ERR_ARG, "alphabets of at most 4 letters");
    if (n < 1 || m < 1) return fail(ANYSEQ_ERR_ARG, "both sequences must be non-empty");
    if (n > NA_MAX || m > NA_MAX)
        return fail(ANYSEQ_ERR_ARG, "sequences longer than %lld letters do not fit the fixed scratch array",
                    (long long)NA_MAX);
    if (!q || !s || !score) return fail(ANYSEQ_ERR_ARG, "q, s and score must be device pointers");
    if (!long_range_ok(sc, n, m)) return fail(ANYSEQ_ERR_ARG, "scores of this pair may leave the 32-bit range");
    // the scratch array and the launches belong to the current device: inputs and
    // output must live there too
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return fail(ANYSEQ_ERR_CUDA, "no current CUDA device");
    }
    if (!on_device(q, cur) || !on_device(s, cur) || !on_device(score, cur))
        return fail(ANYSEQ_ERR_ARG, "q, s and score must be device memory of the current device (%d)", cur);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint8_t *base = nullptr;
    st2 = scratch_address(&base);
    if (st2 != ANYSEQ_OK) return st2;
    uint32_t *q2 = reinterpret_cast<uint32_t *>(base + NA_OFF_Q2);
    uint32_t *s2 = reinterpret_cast<uint32_t *>(base + NA_OFF_S2);
    int32_t *ctl = reinterpret_cast<int32_t *>(base + NA_OFF_CTL);
    int32_t *H = reinterpret_cast<int32_t *>(base + NA_OFF_H);
    int32_t *bad = reinterpret_cast<int32_t *>(base + NA_OFF_BAD);
    WavePass *pass = reinterpret_cast<WavePass *>(base + NA_OFF_PASS);

    WavePass ps;
    memset(&ps, 0, sizeof(ps));
    ps.n = (int32_t)n;
    ps.m = (int32_t)m;
    ps.tb = sc->gap_open;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur);
    const int wr = wave_rows_per_lane(n, sms, 1, GLOBAL, 0, true);  // the array is sized for 8-row stripes
    const int64_t stripes = (n + WAVE_LANES * wr - 1) / (WAVE_LANES * wr);
    noalloc_init_kernel<<<8, 256, 0, st>>>(pass, ps, ctl, stripes + 2, bad);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_pack2bit(q, n, q2, sc->alphabet, bad, st);
    if (e == cudaSuccess) e = launch_pack2bit(s, m, s2, sc->alphabet, bad, st);
    WaveArgs W;
    memset(&W, 0, sizeof(W));
    W.q2 = q2;
    W.s2 = s2;
    W.passes = pass;
    W.n_passes = 1;
    W.n_stripes = (int32_t)stripes;
    W.o = sc->gap_open;
    W.e = sc->gap_extend;
    st2 = make_rowprof(sc, ANYSEQ_GLOBAL, W.rowprof);
    if (st2 != ANYSEQ_OK) return st2;
    W.border = reinterpret_cast<int2 *>(base + NA_OFF_BORDER);
    W.stripe_counter = ctl;
    W.err = ctl + 1;
    W.prog = ctl + 2;
    W.last_H = H;
    W.last_E = nullptr;
    W.spin_limit = 1ll << 24;
    W.rows_per_lane = wr;
    if (e == cudaSuccess) e = launch_wave(W, sms, st);
    if (e == cudaSuccess) {
        noalloc_finish_kernel<<<1, 1, 0, st>>>(H, (int32_t)m, score);
        e = cudaGetLastError();
    }
    int32_t flags[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags[0], ctl + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags[1], bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "no-allocation long pair: %s", cudaGetErrorString(e));
    if (flags[1]) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", sc->alphabet);
    if (flags[0]) return fail(ANYSEQ_ERR_TIMEOUT, "a stripe of the wavefront waited past its limit");
    return ANYSEQ_OK;
}
