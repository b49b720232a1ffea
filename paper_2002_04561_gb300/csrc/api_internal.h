// Internal declarations of the host side: the context and its scratch arena.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/anyseq.h"
#include "wave.h"

struct anyseq_ctx {
    struct Buf {
        std::string name;
        void *p;
        size_t cap;
    };
    int device = 0;
    int num_sms = 1;
    size_t budget = 0;
    size_t used = 0;
    int force32 = 0;              // route every pair to 32-bit lanes (testing)
    int force_matrix = 0;         // use the shared-memory profile path for any alphabet (testing)
    int64_t spin_limit = 1ll << 24;  // iterations of one device-side wait (x ~64 ns)
    int64_t base_cells = 1 << 16;    // Hirschberg base-case size
    // band network (device): float master, bfloat16 copies, gradients, Adam moments
    float *mlp = nullptr;
    bool mlp_ready = false;
    int64_t band_cells = 0, band_accepted = 0, band_fallback = 0, band_rounds = 0;
    double band_plan_ms = 0, band_pass_ms = 0, band_full_ms = 0;  // phases of the last banded call
    int32_t band_max_doublings = 0;  // doublings after the predicted width before the full DP
    int32_t band_area_pct = 60;      // a band above this share of the matrix goes to the full DP
    int32_t band_area16_pct = 15;    // the same for pairs the full DP runs in int16x2 lanes
    int32_t band_margin_pct = 65;    // the network's half-width times this / 100 is the band used
    int32_t band_floor_pct = 30;     // ... but at least this share (%) of the longer sequence
    int profile = 0;              // time the DP kernels with events
    int host_in_place = 1;        // 2-bit batches: pinned host letters read in place by the packing kernel
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // statistics of the last call
    int64_t launches = 0;
    double dp_ms = 0, dp32_ms = 0;
    int64_t pairs16 = 0, pairs32 = 0;
    int32_t *bad_code = nullptr;  // letter-check flag of the last captured batch (graph plans)
    // autotuning: rows-per-lane cap per length bin (0 = the kernel's own), its
    // device copy (when tuned), and the per-bin statistics buffer of a tuning run
    uint8_t tune_tab[256] = {0};
    uint8_t *d_tune_tab = nullptr;
    unsigned long long *d_bin_stats = nullptr;
    bool tuned = false;
    double tune_gain = 1.0;       // default time / tuned time on the tuning sample
    int32_t tb_walker = 0;  // traceback walk: 0 by batch size, 1 a warp per pair, 2 a thread per pair
    int32_t wave_split = 0;  // global three-input-maximum wavefront: 0 by stripe count, 1 split steps, 2 plain
    int32_t wave_spread = 1;       // wavefront: first stripes of a launch on distinct SMs
    int32_t wave_ctas_per_sm = 0;  // wavefront CTAs per SM: 0 as many as fit (the serving lanes use 1)
    int32_t batch_ctas_per_sm = 0;  // batched DP CTAs per SM: 0 as many as fit (the serving short lane uses 2)
    int32_t wave_rows = 0;  // wavefront rows per lane: 0 automatic, or 4, 8, 16 (within what each mode has)
    int32_t wave_cell = 0;  // wavefront cell of global passes: 0 by stripe count, 1 three-input max, 2 two-step
    std::vector<Buf> bufs;        // device scratch, grown on demand, reused across calls
    // buffers replaced by larger ones, freed only under budget pressure or at
    // destroy: cudaFree waits for the whole device, including other contexts' work
    std::vector<Buf> retired;
    std::vector<Buf> pinned;      // pinned host staging
    // Named device buffer of at least 'bytes'; contents are not preserved on growth.
    void *get(const char *name, size_t bytes, anyseq_status_t *st);
};

namespace anyseq {

struct BatchInput {
    const uint8_t *q = nullptr, *s = nullptr;          // device
    const int64_t *q_off = nullptr, *s_off = nullptr;  // device
    int64_t n_pairs = 0, q_len = 0, s_len = 0, max_n = 0, max_m = 0;
    int64_t max_min = 0;  // largest min(n, m) of a pair
    const uint8_t *select = nullptr;                   // optional subset of pairs (device)
};

// 40-byte result records from the per-pair score and optimum-cell arrays (no CIGAR)
cudaError_t launch_write_results(int64_t n, const int32_t *score, const int32_t *eq, const int32_t *es,
                                 const uint32_t *flags, anyseq_result_t *out, cudaStream_t st);
anyseq_status_t fail(anyseq_status_t st, const char *fmt, ...);
bool is_device_ptr(const void *p);
anyseq_status_t check_scoring(const anyseq_scoring_t *sc, int32_t mode);
int32_t sigma_host(const anyseq_scoring_t *sc, int a, int b);
anyseq_status_t make_rowprof(const anyseq_scoring_t *sc, int32_t mode, uint32_t prof[5]);
anyseq_status_t stage_input(anyseq_ctx *ctx, const char *name, const void *src, size_t bytes, cudaStream_t st,
                            const void **dev);
// Direction words of a traceback run (see tb.cu).
struct TbOut {
    uint32_t *dirs = nullptr;
    int64_t *dir_base = nullptr;
    int32_t *lay_pad = nullptr, *lay_ch0 = nullptr;
    int32_t *lay_r = nullptr;                         // rows per lane of each pair (batched kernel)
    int64_t dir_words = 0;
    int32_t lanes_per_chunk = 16, rows_per_lane = 8;  // layout when lay_r is null (wavefront: 32 x 8 or 16)
};

// Letters of the long-pair path with a substitution matrix (alphabets above 4):
// device codes one byte each, at the same positions as the 2-bit arrays.
struct MatLetters {
    const uint8_t *q8 = nullptr, *s8 = nullptr;
};
// Small global batches with CIGAR on the wavefront: scores, end cells and the
// direction words of every pair; false in *used when the batch does not qualify.
anyseq_status_t wave_batch(anyseq_ctx *ctx, const BatchInput &in, const anyseq_scoring_t *sc, int32_t mode,
                           int32_t *score, int32_t *eq, int32_t *es, uint32_t *flags, cudaStream_t st, TbOut *tb,
                           bool *used);
// Long pairs of a score-only batch on the wavefront (see api.cu); rest: the
// batch with the other pairs selected, *all_done when none is left. Only pairs
// that in.select keeps (all without one) take part; tail_factor: a pair is long
// from this many times the batch's cells per resident 16-lane group.
anyseq_status_t long_pairs_split(anyseq_ctx *ctx, const BatchInput &in, const anyseq_scoring_t *sc, int32_t mode,
                                 int32_t *score, int32_t *eq, int32_t *es, uint32_t *flags, cudaStream_t st,
                                 BatchInput &rest, bool *all_done, double tail_factor = 4.0);
// read_in_place: letters in pinned (mapped) host memory are left there for the
// device to read through the host link (callers whose only letter reader is the
// 2-bit packing kernel)
anyseq_status_t stage_batch(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off, const uint8_t *s,
                            const int64_t *s_off, int64_t n_pairs, BatchInput &in, cudaStream_t st,
                            bool read_in_place = false);
anyseq_status_t band_scores(anyseq_ctx *ctx, const BatchInput &in, const anyseq_scoring_t *sc, int32_t *score,
                            int32_t *eq, int32_t *es, uint32_t *flags, cudaStream_t st);
bool long_range_ok(const anyseq_scoring_t *sc, int64_t n, int64_t m);
bool long_profile_ok(const anyseq_scoring_t *sc);
// local / semi-global: the best score of a pair with min(n, m) <= min_nm fits the optimum key
bool key_range_ok(const anyseq_scoring_t *sc, int64_t min_nm);
// Scores (and, with end_q/end_s, optimum cells) of several long pairs in one
// wavefront launch, in the given mode (host arrays).
anyseq_status_t long_scores(anyseq_ctx *ctx, const uint8_t *q, const int64_t *q_off, const uint8_t *s,
                            const int64_t *s_off, int64_t count, const anyseq_scoring_t *sc, int32_t *scores,
                            cudaStream_t st, int32_t mode = ANYSEQ_GLOBAL, int32_t *end_q = nullptr,
                            int32_t *end_s = nullptr);
anyseq_status_t long_last_row(anyseq_ctx *ctx, const uint32_t *q2, int64_t q0, int32_t n, const uint32_t *s2,
                              int64_t s0, int32_t m, bool rev, int32_t tb, const anyseq_scoring_t *sc, int32_t *H,
                              int32_t *E, cudaStream_t st, const MatLetters *mat = nullptr);
// Traceback output of a wavefront launch: direction words in the layout of the
// batched traceback with 32 lanes x rows_per_lane rows per chunk (see tb.h);
// each pass's first word is its dir_off.
struct WaveTb {
    uint32_t *dirs = nullptr;
    int32_t rows_per_lane = 0;
};
anyseq_status_t run_wave_passes(anyseq_ctx *ctx, const uint32_t *q2, const uint32_t *s2,
                                std::vector<WavePass> &passes, const anyseq_scoring_t *sc, int32_t *H, int32_t *E,
                                cudaStream_t st, WaveTb *tb = nullptr, int32_t mode = ANYSEQ_GLOBAL,
                                std::vector<uint64_t> *keys = nullptr, const MatLetters *mat = nullptr);
// Start cell of a local / semi-global long-pair traceback from r's score and
// optimum cell (sets r.beg_q, r.beg_s).
anyseq_status_t long_start_cell(anyseq_ctx *ctx, const uint32_t *q2, const uint32_t *s2, const anyseq_scoring_t *sc,
                                int32_t mode, anyseq_result_t &r, cudaStream_t st, const MatLetters *mat = nullptr);
// Global divide-and-conquer CIGAR of q[i0 .. i1) against s[j0 .. j1) (positions
// in the packed arrays q2, s2).
anyseq_status_t hirschberg_cigar(anyseq_ctx *ctx, const uint32_t *q2, int32_t i0, int32_t i1, const uint32_t *s2,
                                 int32_t j0, int32_t j1, const anyseq_scoring_t *sc, std::vector<uint32_t> &cigar,
                                 cudaStream_t st, const MatLetters *mat = nullptr);

// Scores and optimum cells of a batch; with tb != null also the direction words.
anyseq_status_t batch_scores(anyseq_ctx *ctx, const BatchInput &in, const anyseq_scoring_t *sc, int32_t mode,
                             int32_t *score, int32_t *eq, int32_t *es, uint32_t *flags, cudaStream_t st,
                             TbOut *tb = nullptr, bool capture = false);

}  // namespace anyseq
