// Divide-and-conquer traceback of a long global alignment in linear space
// (Sec. III-A: Hirschberg's method, at most doubling the relaxed cells; half of
// every subproblem relaxed in reverse, Sec. III-B/C), for affine gaps in the
// form of Myers & Miller (1988):
//
//   HB(i0, i1, j0, j1, tb, te): align q[i0+1..i1] with s[j0+1..j1]; a vertical
//   gap that starts in the top-left corner opens with tb, one that ends in the
//   bottom-right corner with te (open, or 0 when the gap continues from a
//   neighbouring subproblem).
//   - base case: at most one row, or at most base_cells cells -> full-matrix
//     traceback with the tie rules of the batched path;
//   - otherwise mid = floor((i0+i1)/2); forward pass over rows i0+1..mid gives
//     CC[j] = H(mid, j), DD[j] = E(mid, j); the reverse pass over rows
//     i1..mid+1 gives RR, SS; type 1 joins CC[j] + RR[j], type 2 joins
//     DD[j] + SS[j] - open (a vertical gap through rows mid and mid+1); the
//     largest value wins, then the smallest j, then type 1;
//   - type 1: HB(i0,mid,j0,j*,tb,open) ++ HB(mid,i1,j*,j1,open,te)
//     type 2: HB(i0,mid-1,j0,j*,tb,0) ++ II ++ HB(mid+1,i1,j*,j1,0,te).
//
// The host walks the recursion level by level: all passes of a level run in one
// launch of the wavefront kernel, one launch picks every midpoint, and all base
// cases run in one launch at the end; the pieces are joined in order.
#include <algorithm>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "common.cuh"
#include "wave.h"

namespace anyseq {

// ------------------------------------------------------------------ midpoints

struct MidArgs {
    const int32_t *H, *E;          // pass outputs
    const int64_t *fwd_off, *rev_off;
    const int32_t *cols;
    int32_t o;
    int32_t *jstar, *type;
};

__global__ void midpoint_kernel(MidArgs M) {
    const int b = blockIdx.x;
    const int32_t cols = M.cols[b];
    const int32_t *CC = M.H + M.fwd_off[b], *DD = M.E + M.fwd_off[b];
    const int32_t *RR = M.H + M.rev_off[b], *SS = M.E + M.rev_off[b];
    // key: value, then smaller j, then type 1 (t = 2j + type - 1, smaller wins)
    unsigned long long best = 0;
    for (int32_t j = threadIdx.x; j <= cols; j += blockDim.x) {
        int64_t v1 = (int64_t)CC[j] + RR[cols - j];
        int64_t v2 = (int64_t)DD[j] + SS[cols - j] - M.o;
        uint32_t t1 = 2u * (uint32_t)j, t2 = t1 + 1u;
        unsigned long long k1 = ((unsigned long long)(v1 + (1ll << 38)) << 24) | (0xFFFFFFu - (t1 & 0xFFFFFFu));
        unsigned long long k2 = ((unsigned long long)(v2 + (1ll << 38)) << 24) | (0xFFFFFFu - (t2 & 0xFFFFFFu));
        unsigned long long k = k1 > k2 ? k1 : k2;
        best = k > best ? k : best;
    }
    __shared__ unsigned long long red[32];
    for (int off = 16; off; off >>= 1) {
        unsigned long long x = __shfl_xor_sync(0xffffffffu, best, off);
        best = x > best ? x : best;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) best = red[w] > best ? red[w] : best;
        uint32_t t = 0xFFFFFFu - (uint32_t)(best & 0xFFFFFFu);
        M.jstar[b] = (int32_t)(t >> 1);
        M.type[b] = (int32_t)(t & 1u) + 1;
    }
}

// ---------------------------------------------------------------- base cases

struct BaseCase {
    int64_t q0, s0;                // first letters (packed positions)
    int32_t n, m;
    int32_t tb, te;
    int64_t dir_off;               // n * m direction bytes
    int64_t row_off;               // 2 * (m + 1) ints of row scratch
    int64_t piece_off;             // n + m + 1 words of reversed runs
};

struct BaseArgs {
    const uint32_t *q2, *s2;
    const BaseCase *cases;
    int32_t n_cases;
    uint32_t rowprof[5];           // sigma' bytes (sigma - open - extend)
    int32_t o, e;
    uint8_t *dirs;
    int32_t *rows;
    uint32_t *pieces;
    int32_t *piece_len;
    // substitution matrix: byte letter codes and sigma' per letter pair
    const uint8_t *q8, *s8;
    const int8_t *sig;
    int32_t alphabet;
};

__device__ __forceinline__ int32_t sig(const BaseArgs &A, uint32_t a, uint32_t b, int32_t oe) {
    if (A.sig) return (int32_t)A.sig[a * A.alphabet + b] + oe;
    return (int32_t)(int8_t)((A.rowprof[a] >> (8 * b)) & 0xFFu) + oe;
}
__device__ __forceinline__ uint32_t base_letter(const uint32_t *p2, const uint8_t *p8, int64_t k) {
    return p8 ? (uint32_t)p8[k] : code2(p2, k);
}

// One thread per base case: the full-matrix global alignment with column-0
// open tb and corner open te, direction byte per cell (bits 0-1: H from
// DIAG 0 / E 1 / F 2; bit 2: E opened; bit 3: F opened), then the walk back.
__global__ void hb_base_kernel(BaseArgs A) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= A.n_cases) return;
    const BaseCase bc = A.cases[b];
    const int32_t n = bc.n, m = bc.m, o = A.o, e = A.e, oe = o + e;
    uint32_t *out = A.pieces + bc.piece_off;
    int64_t k = 0;
    uint32_t cur_op = 0, cur_len = 0;
    auto push = [&](uint32_t op, uint32_t cnt) {
        if (!cnt) return;
        if (cur_len && op != cur_op) { out[k++] = (cur_len << 4) | cur_op; cur_len = 0; }
        cur_op = op;
        cur_len += cnt;
    };
    if (n == 0 || m == 0) {
        push(2u, (uint32_t)m);
        push(1u, (uint32_t)n);
    } else {
        uint8_t *dir = A.dirs + bc.dir_off;
        int32_t *Hrow = A.rows + bc.row_off, *Erow = Hrow + (m + 1);
        Hrow[0] = 0;
        for (int32_t j = 1; j <= m; j++) { Hrow[j] = o + j * e; Erow[j] = NEG32; }
        int32_t cornerD = 0, cornerE = 0, cornerF = 0;
        for (int32_t i = 1; i <= n; i++) {
            const uint32_t qi = base_letter(A.q2, A.q8, bc.q0 + i - 1);
            int32_t diag = Hrow[0];
            Hrow[0] = bc.tb + i * e;
            int32_t F = NEG32, Hleft = Hrow[0];
            for (int32_t j = 1; j <= m; j++) {
                const uint32_t sj = base_letter(A.s2, A.s8, bc.s0 + j - 1);
                int32_t Eo = Hrow[j] + oe, Ee = Erow[j] + e;
                int32_t Ev = Ee > Eo ? Ee : Eo;
                int32_t Fo = Hleft + oe, Fe = F + e;
                int32_t Fv = Fe > Fo ? Fe : Fo;
                int32_t Dv = diag + sig(A, qi, sj, oe);
                uint32_t src = 0;
                int32_t Hv = Dv;
                if (Ev > Hv) { Hv = Ev; src = 1; }
                if (Fv > Hv) { Hv = Fv; src = 2; }
                dir[(int64_t)(i - 1) * m + (j - 1)] =
                    (uint8_t)(src | (Ee > Eo ? 0u : 4u) | (Fe > Fo ? 0u : 8u));
                if (i == n && j == m) { cornerD = Dv; cornerE = Ev; cornerF = Fv; }
                diag = Hrow[j];
                Hrow[j] = Hv;
                Erow[j] = Ev;
                F = Fv;
                Hleft = Hv;
            }
        }
        // the corner: a vertical gap that ends here re-opens at te
        int state;  // 0 H via DIAG, 1 E, 2 F
        {
            int32_t best = cornerD;
            state = 0;
            int32_t Ea = cornerE - o + bc.te;
            if (Ea > best) { best = Ea; state = 1; }
            if (cornerF > best) { best = cornerF; state = 2; }
        }
        int32_t i = n, j = m;
        if (state == 0) { push(0u, 1u); i--; j--; }
        // walk (state 3 = H at (i, j))
        int st = state == 0 ? 3 : state;
        for (int64_t guard = 2 * ((int64_t)n + m) + 4; guard > 0; guard--) {
            if (st == 3) {
                if (i == 0 && j == 0) break;
                if (j == 0) { push(1u, (uint32_t)i); break; }
                if (i == 0) { push(2u, (uint32_t)j); break; }
                uint32_t d = dir[(int64_t)(i - 1) * m + (j - 1)] & 3u;
                if (d == 0) { push(0u, 1u); i--; j--; }
                else st = (int)d;
            } else if (st == 1) {
                if (i <= 0 || j <= 0) break;
                uint32_t d = dir[(int64_t)(i - 1) * m + (j - 1)];
                push(1u, 1u);
                i--;
                if (d & 4u) st = 3;
            } else {
                if (i <= 0 || j <= 0) break;
                uint32_t d = dir[(int64_t)(i - 1) * m + (j - 1)];
                push(2u, 1u);
                j--;
                if (d & 8u) st = 3;
            }
        }
    }
    if (cur_len) out[k++] = (cur_len << 4) | cur_op;
    A.piece_len[b] = (int32_t)k;
}

// ------------------------------------------------------------------- driver

#define HB_TRY(x)                           \
    do {                                    \
        anyseq_status_t _s = (x);           \
        if (_s != ANYSEQ_OK) return _s;     \
    } while (0)
#define HB_CUDA(x)                                                                              \
    do {                                                                                        \
        cudaError_t _e = (x);                                                                   \
        if (_e != cudaSuccess) return fail(ANYSEQ_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(_e)); \
    } while (0)

namespace {
struct Sub {
    int32_t i0, i1, j0, j1, tb, te;
};
struct Node {
    Sub sub;
    int kind = 0;      // 0 undecided, 1 base, 2 split type 1, 3 split type 2
    int left = -1, right = -1;
    int base = -1;
};
}  // namespace

template <class T>
static T *arena_t(anyseq_ctx *ctx, const char *name, size_t count, anyseq_status_t *st) {
    return static_cast<T *>(ctx->get(name, count * sizeof(T) + 16, st));
}

// The sigma' table (sigma - open - extend per letter pair) of the matrix path on
// the device; nullptr when the letters are 2-bit.
static const int8_t *device_sig_table(anyseq_ctx *ctx, const anyseq_scoring_t *sc, const MatLetters *mat,
                                      cudaStream_t st, anyseq_status_t *s) {
    if (!mat) return nullptr;
    const int32_t a = sc->alphabet, oe = sc->gap_open + sc->gap_extend;
    int8_t h[WAVE_SIG_BYTES];
    for (int x = 0; x < a; x++)
        for (int y = 0; y < a; y++) h[x * a + y] = (int8_t)(sigma_host(sc, x, y) - oe);
    int8_t *d = arena_t<int8_t>(ctx, "w_sig", WAVE_SIG_BYTES, s);
    if (*s != ANYSEQ_OK) return nullptr;
    if (cudaMemcpyAsync(d, h, (size_t)a * a, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        *s = fail(ANYSEQ_ERR_CUDA, "copying the sigma table failed");
        return nullptr;
    }
    return d;
}

anyseq_status_t run_wave_passes(anyseq_ctx *ctx, const uint32_t *q2, const uint32_t *s2,
                                std::vector<WavePass> &passes, const anyseq_scoring_t *sc, int32_t *H, int32_t *E,
                                cudaStream_t st, WaveTb *tb, int32_t mode, std::vector<uint64_t> *keys,
                                const MatLetters *mat) {
    anyseq_status_t s2st = ANYSEQ_OK;
    int64_t border = 0, rows = 0;
    for (const auto &p : passes) rows += p.n;
    const int wr = wave_rows_per_lane(rows, ctx->num_sms, (int64_t)passes.size(), mode, ctx->wave_rows, false);
    const int stripe_rows = WAVE_LANES * wr;
    int32_t stripes = 0;
    int64_t dir_words = 0;
    for (auto &p : passes) {
        p.border_off = border;
        border += 2 * (int64_t)p.m + 2;
        p.stripe0 = stripes;
        const int32_t ns = (p.n + stripe_rows - 1) / stripe_rows;
        stripes += ns;
        p.dir_off = dir_words;
        if (tb) dir_words += (int64_t)ns * (p.m + WAVE_LANES - 1) * WAVE_LANES * ((wr + 7) / 8);
    }
    WaveArgs W;
    memset(&W, 0, sizeof(W));
    W.q2 = q2;
    W.s2 = s2;
    W.n_passes = (int32_t)passes.size();
    W.n_stripes = stripes;
    W.o = sc->gap_open;
    W.e = sc->gap_extend;
    HB_TRY(make_rowprof(sc, wave_init_mode(mode), W.rowprof));
    W.mode = mode;
    W.best = nullptr;
    std::vector<uint64_t> hkeys;
    if (mode != ANYSEQ_GLOBAL) {
        // best cell per pass, starting from the empty alignment's cell (local,
        // semi-global) or from no candidate (anchored passes look for a
        // positive optimum)
        hkeys.resize(passes.size());
        for (size_t k = 0; k < passes.size(); k++)
            hkeys[k] = mode == ANYSEQ_LOCAL        ? end_key(0, 0, 0)
                       : mode == ANYSEQ_SEMIGLOBAL ? end_key(0, 0, passes[k].m)
                                                   : 0;
        W.best = arena_t<uint64_t>(ctx, "w_best", passes.size() + 1, &s2st);
        if (s2st != ANYSEQ_OK) return s2st;
        HB_CUDA(cudaMemcpyAsync(W.best, hkeys.data(), hkeys.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    }
    WavePass *dpass = arena_t<WavePass>(ctx, "w_pass", passes.size() + 1, &s2st);
    W.border = arena_t<int2>(ctx, "w_border", (size_t)border + 2, &s2st);
    int32_t *ctl = arena_t<int32_t>(ctx, "w_ctl", (size_t)stripes + 8, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    W.passes = dpass;
    W.stripe_counter = ctl;
    W.err = ctl + 1;
    W.prog = ctl + 2;
    W.last_H = H;
    W.last_E = E;
    W.spin_limit = ctx->spin_limit;
    W.cell = ctx->wave_cell;
    W.ctas_per_sm = ctx->wave_ctas_per_sm;
    W.no_spread = ctx->wave_spread ? 0 : 1;
    W.split = ctx->wave_split;
    if (mat) {
        W.mat = 1;
        W.alphabet = sc->alphabet;
        W.q8 = mat->q8;
        W.s8 = mat->s8;
        W.sig = device_sig_table(ctx, sc, mat, st, &s2st);
        if (s2st != ANYSEQ_OK) return s2st;
        W.sig_pad = (wave_init_mode(mode) == GLOBAL ? sc->gap_extend : 0) - (sc->gap_open + sc->gap_extend);
    }
    W.rows_per_lane = wr;
    W.dirs = nullptr;
    if (tb) {
        tb->rows_per_lane = wr;
        tb->dirs = arena_t<uint32_t>(ctx, "w_dirs", (size_t)dir_words + 1, &s2st);
        if (s2st != ANYSEQ_OK) return s2st;
        W.dirs = tb->dirs;
    }
    HB_CUDA(cudaMemcpyAsync(dpass, passes.data(), passes.size() * sizeof(WavePass), cudaMemcpyHostToDevice, st));
    HB_CUDA(cudaMemsetAsync(ctl, 0, ((size_t)stripes + 2) * sizeof(int32_t), st));
    HB_CUDA(launch_wave(W, ctx->num_sms, st));
    ctx->launches += 1;
    int32_t err = 0;
    HB_CUDA(cudaMemcpyAsync(&err, W.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (W.best) HB_CUDA(cudaMemcpyAsync(hkeys.data(), W.best, hkeys.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    HB_CUDA(cudaStreamSynchronize(st));
    if (keys) *keys = hkeys;
    if (err) return fail(ANYSEQ_ERR_TIMEOUT, "a stripe of the wavefront waited past its limit");
    return ANYSEQ_OK;
}

anyseq_status_t hirschberg_cigar(anyseq_ctx *ctx, const uint32_t *q2, int32_t i0, int32_t i1, const uint32_t *s2,
                                 int32_t j0, int32_t j1, const anyseq_scoring_t *sc, std::vector<uint32_t> &cigar,
                                 cudaStream_t st, const MatLetters *mat) {
    anyseq_status_t s2st = ANYSEQ_OK;
    const int32_t o = sc->gap_open;
    std::vector<Node> nodes;
    nodes.push_back(Node{Sub{i0, i1, j0, j1, o, o}});
    std::vector<int> level{0}, bases;
    while (!level.empty()) {
        std::vector<int> splits;
        for (int id : level) {
            const Sub &u = nodes[id].sub;
            int64_t rows = u.i1 - u.i0, cols = u.j1 - u.j0;
            if (rows <= 1 || rows * cols <= ctx->base_cells) {
                nodes[id].kind = 1;
                nodes[id].base = (int)bases.size();
                bases.push_back(id);
            } else {
                splits.push_back(id);
            }
        }
        if (splits.empty()) break;
        // forward and reverse pass of every split, outputs side by side
        std::vector<WavePass> passes;
        std::vector<int64_t> fo(splits.size()), ro(splits.size());
        std::vector<int32_t> colv(splits.size());
        int64_t out = 0;
        for (size_t t = 0; t < splits.size(); t++) {
            const Sub &u = nodes[splits[t]].sub;
            const int32_t mid = (u.i0 + u.i1) / 2, cols = u.j1 - u.j0;
            WavePass f;
            memset(&f, 0, sizeof(f));
            f.q0 = u.i0; f.s0 = u.j0; f.n = mid - u.i0; f.m = cols; f.tb = u.tb; f.rev = 0;
            f.out_off = out; fo[t] = out; out += cols + 1;
            WavePass r = f;
            r.q0 = mid; r.n = u.i1 - mid; r.tb = u.te; r.rev = 1;
            r.out_off = out; ro[t] = out; out += cols + 1;
            passes.push_back(f);
            passes.push_back(r);
            colv[t] = cols;
        }
        int32_t *H = arena_t<int32_t>(ctx, "hb_H", (size_t)out + 1, &s2st);
        int32_t *E = arena_t<int32_t>(ctx, "hb_E", (size_t)out + 1, &s2st);
        if (s2st != ANYSEQ_OK) return s2st;
        HB_TRY(run_wave_passes(ctx, q2, s2, passes, sc, H, E, st, nullptr, ANYSEQ_GLOBAL, nullptr, mat));
        // midpoints
        const size_t ns = splits.size();
        int64_t *dmeta = arena_t<int64_t>(ctx, "hb_meta", 2 * ns + 1, &s2st);
        int32_t *dint = arena_t<int32_t>(ctx, "hb_int", 3 * ns + 1, &s2st);
        if (s2st != ANYSEQ_OK) return s2st;
        std::vector<int64_t> meta(2 * ns);
        std::copy(fo.begin(), fo.end(), meta.begin());
        std::copy(ro.begin(), ro.end(), meta.begin() + ns);
        HB_CUDA(cudaMemcpyAsync(dmeta, meta.data(), 2 * ns * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        HB_CUDA(cudaMemcpyAsync(dint, colv.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        MidArgs M;
        M.H = H; M.E = E; M.fwd_off = dmeta; M.rev_off = dmeta + ns; M.cols = dint; M.o = o;
        M.jstar = dint + ns; M.type = dint + 2 * ns;
        midpoint_kernel<<<(unsigned)ns, 256, 0, st>>>(M);
        HB_CUDA(cudaGetLastError());
        ctx->launches += 1;
        std::vector<int32_t> jt(2 * ns);
        HB_CUDA(cudaMemcpyAsync(jt.data(), dint + ns, 2 * ns * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HB_CUDA(cudaStreamSynchronize(st));
        std::vector<int> next;
        for (size_t t = 0; t < ns; t++) {
            const int id = splits[t];
            const Sub u = nodes[id].sub;
            const int32_t mid = (u.i0 + u.i1) / 2, js = u.j0 + jt[t], type = jt[ns + t];
            Sub a, b;
            if (type == 1) {
                a = Sub{u.i0, mid, u.j0, js, u.tb, o};
                b = Sub{mid, u.i1, js, u.j1, o, u.te};
            } else {
                a = Sub{u.i0, mid - 1, u.j0, js, u.tb, 0};
                b = Sub{mid + 1, u.i1, js, u.j1, 0, u.te};
            }
            nodes[id].kind = type == 1 ? 2 : 3;
            nodes[id].left = (int)nodes.size();
            nodes.push_back(Node{a});
            nodes[id].right = (int)nodes.size();
            nodes.push_back(Node{b});
            next.push_back(nodes[id].left);
            next.push_back(nodes[id].right);
        }
        level.swap(next);
    }
    // base cases in one launch
    const size_t nb = bases.size();
    std::vector<BaseCase> bc(nb);
    int64_t dir_total = 0, row_total = 0, piece_total = 0;
    for (size_t t = 0; t < nb; t++) {
        const Sub &u = nodes[bases[t]].sub;
        BaseCase &c = bc[t];
        c.q0 = u.i0; c.s0 = u.j0; c.n = u.i1 - u.i0; c.m = u.j1 - u.j0; c.tb = u.tb; c.te = u.te;
        c.dir_off = dir_total; dir_total += (int64_t)c.n * c.m;
        c.row_off = row_total; row_total += 2 * ((int64_t)c.m + 1);
        c.piece_off = piece_total; piece_total += (int64_t)c.n + c.m + 1;
    }
    BaseArgs B;
    memset(&B, 0, sizeof(B));
    B.q2 = q2; B.s2 = s2; B.n_cases = (int32_t)nb; B.o = o; B.e = sc->gap_extend;
    HB_TRY(make_rowprof(sc, ANYSEQ_GLOBAL, B.rowprof));  // bytes hold sigma - open - extend
    if (mat) {
        B.q8 = mat->q8;
        B.s8 = mat->s8;
        B.alphabet = sc->alphabet;
        B.sig = device_sig_table(ctx, sc, mat, st, &s2st);
        if (s2st != ANYSEQ_OK) return s2st;
    }
    BaseCase *dbc = arena_t<BaseCase>(ctx, "hb_cases", nb + 1, &s2st);
    B.dirs = arena_t<uint8_t>(ctx, "hb_dirs", (size_t)dir_total + 16, &s2st);
    B.rows = arena_t<int32_t>(ctx, "hb_rows", (size_t)row_total + 16, &s2st);
    B.pieces = arena_t<uint32_t>(ctx, "hb_pieces", (size_t)piece_total + 16, &s2st);
    B.piece_len = arena_t<int32_t>(ctx, "hb_plen", nb + 1, &s2st);
    if (s2st != ANYSEQ_OK) return s2st;
    B.cases = dbc;
    HB_CUDA(cudaMemcpyAsync(dbc, bc.data(), nb * sizeof(BaseCase), cudaMemcpyHostToDevice, st));
    hb_base_kernel<<<(unsigned)((nb + 63) / 64), 64, 0, st>>>(B);
    HB_CUDA(cudaGetLastError());
    ctx->launches += 1;
    std::vector<uint32_t> pieces((size_t)piece_total + 1);
    std::vector<int32_t> plen(nb + 1);
    HB_CUDA(cudaMemcpyAsync(pieces.data(), B.pieces, (size_t)piece_total * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    HB_CUDA(cudaMemcpyAsync(plen.data(), B.piece_len, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HB_CUDA(cudaStreamSynchronize(st));
    // in-order join, merging runs across piece boundaries
    cigar.clear();
    auto emit = [&](uint32_t w) {
        if (!cigar.empty() && (cigar.back() & 15u) == (w & 15u))
            cigar.back() += w & ~15u;
        else
            cigar.push_back(w);
    };
    std::vector<int> stack{0};
    while (!stack.empty()) {
        int id = stack.back();
        stack.pop_back();
        if (id < 0) {  // the two query letters against a gap of a type-2 split
            emit((2u << 4) | 1u);
            continue;
        }
        const Node &nd = nodes[id];
        if (nd.kind == 1) {
            const BaseCase &c = bc[nd.base];
            for (int32_t t = plen[nd.base] - 1; t >= 0; t--) emit(pieces[c.piece_off + t]);
        } else {
            stack.push_back(nd.right);
            if (nd.kind == 3) stack.push_back(-1);
            stack.push_back(nd.left);
        }
    }
    return ANYSEQ_OK;
}

}  // namespace anyseq
