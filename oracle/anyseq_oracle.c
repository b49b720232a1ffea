/*
 * CPU oracle for pairwise DP alignment: TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg call
 * this file. It is a plain, slow, scalar restatement of the recurrences of the
 * AnySeq paper (Sec. III-A, Eqs. 1-5 and the initialisations of the local,
 * global and semi-global cases), written with 64-bit integers so that no
 * overflow can occur, with full matrices wherever a traceback is needed. It
 * shares no code with the CUDA library.
 *
 * Scoring is signed: sigma(a,b) from a matrix or match/mismatch, a gap of
 * length k adds  open + k*extend  (open, extend <= 0). This is Eq. 4/5 with
 * G_o = -open, G_e = -extend; a linear gap g (Eqs. 2/3) is open = 0,
 * extend = g.
 *
 * Conventions that the paper leaves open (each is also written down in the
 * design notes):
 *  - nu = -inf for semi-global (the paper gives it the local initialisation,
 *    H(i,0) = H(0,j) = 0, and the optimum in the last row or column).
 *  - The optimum cell on ties: the smallest i, then the smallest j.
 *  - Predecessor priority on ties follows the order in which the paper's
 *    relaxation function considers its candidates (diagonal first, a gap only
 *    when strictly better): DIAG, then E (q_i against a gap, CIGAR I), then
 *    F (s_j against a gap, CIGAR D). In local mode a cell whose value is 0
 *    ends the alignment. Inside E and F a tie prefers opening over extending.
 *  - Hirschberg (Sec. III-A: divide and conquer, at most doubling the cells)
 *    for affine gaps follows Myers & Miller (1988): midpoint row
 *    floor((i0+i1)/2), type-1 join CC+RR, type-2 join DD+SS-open, largest
 *    value, then smallest j, then type 1; base case when a subproblem has at
 *    most one row or at most base_cells cells.
 *
 * Parity of this oracle is pinned by the tests (brute-force enumeration of
 * all alignments of short sequences, textbook special cases, invariants),
 * not by the CUDA path.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t sc_t;
#define NEG_INF (INT64_MIN / 4)

typedef struct {
    int32_t alphabet;
    const int8_t *matrix;   /* alphabet x alphabet, row = query letter; NULL: match/mismatch */
    int32_t match, mismatch;
    int32_t gap_open, gap_extend;
} orc_scoring;

typedef struct {
    int64_t score;
    int64_t beg_q, beg_s;   /* DP cell where the alignment path starts */
    int64_t end_q, end_s;   /* DP cell where it ends (the optimum cell) */
} orc_result;

enum { ORC_GLOBAL = 0, ORC_LOCAL = 1, ORC_SEMIGLOBAL = 2 };
enum { ORC_OK = 0, ORC_ERR_CAP = -1, ORC_ERR_MEM = -2, ORC_ERR_ARG = -3 };

static sc_t sigma(const orc_scoring *sc, uint8_t a, uint8_t b) {
    if (sc->matrix) return (sc_t)sc->matrix[(int)a * sc->alphabet + (int)b];
    return a == b ? (sc_t)sc->match : (sc_t)sc->mismatch;
}

static sc_t max2(sc_t a, sc_t b) { return a > b ? a : b; }

/* ------------------------------------------------------------------ op lists */

typedef struct { char *ops; int64_t len, cap; int err; } oplist;

static void op_push(oplist *l, char op) {
    if (l->len == l->cap) {
        int64_t nc = l->cap ? l->cap * 2 : 256;
        char *p = (char *)realloc(l->ops, (size_t)nc);
        if (!p) { l->err = 1; return; }
        l->ops = p; l->cap = nc;
    }
    l->ops[l->len++] = op;
}

static void op_reverse(char *ops, int64_t a, int64_t b) { /* reverse ops[a..b) */
    for (b--; a < b; a++, b--) { char t = ops[a]; ops[a] = ops[b]; ops[b] = t; }
}

/* run-length encode 'M','I','D' ops into BAM-style words (len << 4 | op), op M=0 I=1 D=2 */
static int64_t ops_to_cigar(const char *ops, int64_t len, uint32_t *cigar, int64_t cap) {
    int64_t n = 0;
    for (int64_t k = 0; k < len;) {
        int64_t r = k;
        while (r < len && ops[r] == ops[k]) r++;
        uint32_t code = ops[k] == 'M' ? 0u : ops[k] == 'I' ? 1u : 2u;
        if (cigar && n < cap) cigar[n] = ((uint32_t)(r - k) << 4) | code;
        n++;
        k = r;
    }
    return n;
}

/* ------------------------------------------------------- full-matrix alignment */

/*
 * Full matrices H, E, F of size (n+1) x (m+1) (Eqs. 1, 4, 5).
 * E(i,j): q_i aligned to a gap (vertical move), F(i,j): s_j aligned to a gap.
 * For the global case the column-0 run uses open 'tb' and a vertical run that
 * ends in the corner (n,m) uses open 'te'; tb = te = open is the plain global
 * alignment, other values serve the Hirschberg subproblems.
 */
typedef struct { int64_t n, m; sc_t *H, *E, *F; } mats;

#define AT(M_, i, j) ((M_)[(size_t)(i) * (size_t)(mm.m + 1) + (size_t)(j)])

static int fill_full(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m,
                     const orc_scoring *sc, int mode, sc_t tb, mats *out) {
    mats mm = { n, m, NULL, NULL, NULL };
    size_t cells = (size_t)(n + 1) * (size_t)(m + 1);
    mm.H = (sc_t *)malloc(cells * sizeof(sc_t));
    mm.E = (sc_t *)malloc(cells * sizeof(sc_t));
    mm.F = (sc_t *)malloc(cells * sizeof(sc_t));
    if (!mm.H || !mm.E || !mm.F) { free(mm.H); free(mm.E); free(mm.F); return ORC_ERR_MEM; }
    const sc_t o = sc->gap_open, e = sc->gap_extend;
    const sc_t nu = mode == ORC_LOCAL ? 0 : NEG_INF;
    /* initialisation (Sec. III-A): row 0 and column 0 */
    AT(mm.H, 0, 0) = 0; AT(mm.E, 0, 0) = NEG_INF; AT(mm.F, 0, 0) = NEG_INF;
    for (int64_t j = 1; j <= m; j++) {
        AT(mm.H, 0, j) = mode == ORC_GLOBAL ? o + j * e : 0;
        AT(mm.F, 0, j) = mode == ORC_GLOBAL ? AT(mm.H, 0, j) : NEG_INF;
        AT(mm.E, 0, j) = NEG_INF;
    }
    for (int64_t i = 1; i <= n; i++) {
        AT(mm.H, i, 0) = mode == ORC_GLOBAL ? tb + i * e : 0;
        AT(mm.E, i, 0) = mode == ORC_GLOBAL ? AT(mm.H, i, 0) : NEG_INF;
        AT(mm.F, i, 0) = NEG_INF;
    }
    /* recurrences */
    for (int64_t i = 1; i <= n; i++) {
        for (int64_t j = 1; j <= m; j++) {
            sc_t Ev = max2(AT(mm.E, i - 1, j) + e, AT(mm.H, i - 1, j) + o + e);  /* Eq. 4 */
            sc_t Fv = max2(AT(mm.F, i, j - 1) + e, AT(mm.H, i, j - 1) + o + e);  /* Eq. 5 */
            sc_t Dv = AT(mm.H, i - 1, j - 1) + sigma(sc, q[i - 1], s[j - 1]);
            sc_t Hv = max2(max2(Dv, Ev), max2(Fv, nu));                         /* Eq. 1 */
            AT(mm.H, i, j) = Hv; AT(mm.E, i, j) = Ev; AT(mm.F, i, j) = Fv;
        }
    }
    *out = mm;
    return ORC_OK;
}

static void free_mats(mats *mm) { free(mm->H); free(mm->E); free(mm->F); }

/* optimum cell per mode, ties: smallest i then smallest j */
static void find_end(const mats *pm, int mode, int64_t *ei, int64_t *ej) {
    mats mm = *pm;
    int64_t n = mm.n, m = mm.m, bi = n, bj = m;
    if (mode == ORC_LOCAL) {
        sc_t best = NEG_INF;
        for (int64_t i = 0; i <= n; i++)
            for (int64_t j = 0; j <= m; j++)
                if (AT(mm.H, i, j) > best) { best = AT(mm.H, i, j); bi = i; bj = j; }
    } else if (mode == ORC_SEMIGLOBAL) {
        sc_t best = NEG_INF;
        for (int64_t i = 0; i <= n; i++) {
            if (i < n) {
                if (AT(mm.H, i, m) > best) { best = AT(mm.H, i, m); bi = i; bj = m; }
            } else {
                for (int64_t j = 0; j <= m; j++)
                    if (AT(mm.H, n, j) > best) { best = AT(mm.H, n, j); bi = n; bj = j; }
            }
        }
    }
    *ei = bi; *ej = bj;
}

/*
 * Walk the predecessors from (ei, ej) back to the start, appending ops in
 * reverse order to 'l'. 'start' is the state at the end cell: 'H', or 'E'
 * when the corner value of a global subproblem came from its te-adjusted E.
 * Returns the start cell.
 */
static void traceback(const mats *pm, const uint8_t *q, const uint8_t *s, const orc_scoring *sc,
                      int mode, sc_t tb, int64_t ei, int64_t ej, char start, oplist *l,
                      int64_t *bi, int64_t *bj) {
    mats mm = *pm;
    const sc_t o = sc->gap_open, e = sc->gap_extend;
    int64_t i = ei, j = ej;
    char state = start;
    (void)tb;
    for (;;) {
        if (state == 'H') {
            if (i == 0 && j == 0) break;
            if (mode != ORC_GLOBAL) {
                if (i == 0 || j == 0) break;
                if (mode == ORC_LOCAL && AT(mm.H, i, j) == 0) break;
            } else {
                if (j == 0) { while (i > 0) { op_push(l, 'I'); i--; } break; }
                if (i == 0) { while (j > 0) { op_push(l, 'D'); j--; } break; }
            }
            sc_t Hv = AT(mm.H, i, j);
            if (Hv == AT(mm.H, i - 1, j - 1) + sigma(sc, q[i - 1], s[j - 1])) {
                op_push(l, 'M'); i--; j--;
            } else if (Hv == AT(mm.E, i, j)) {
                state = 'E';
            } else {
                state = 'F';
            }
        } else if (state == 'E') {
            /* E(i,j) = max(E(i-1,j)+e, H(i-1,j)+o+e); a tie opens */
            int from_h = AT(mm.E, i, j) == AT(mm.H, i - 1, j) + o + e;
            op_push(l, 'I');
            i--;
            if (from_h) state = 'H';
        } else {
            int from_h = AT(mm.F, i, j) == AT(mm.H, i, j - 1) + o + e;
            op_push(l, 'D');
            j--;
            if (from_h) state = 'H';
        }
    }
    *bi = i; *bj = j;
}

/*
 * Global alignment of q[0..n) and s[0..m) with column-0 open tb and corner
 * open te (see fill_full). Appends the ops in forward order; returns the score.
 */
static int global_sub(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m,
                      const orc_scoring *sc, sc_t tb, sc_t te, oplist *l, sc_t *score) {
    const sc_t o = sc->gap_open, e = sc->gap_extend;
    if (n == 0) { for (int64_t j = 0; j < m; j++) op_push(l, 'D'); *score = m ? o + m * e : 0; return ORC_OK; }
    if (m == 0) { for (int64_t i = 0; i < n; i++) op_push(l, 'I'); *score = max2(tb, te) + n * e; return ORC_OK; }
    mats mm;
    int rc = fill_full(q, n, s, m, sc, ORC_GLOBAL, tb, &mm);
    if (rc) return rc;
    /* the corner: Eq. 1 with the vertical candidate re-opened at te */
    sc_t Dv = AT(mm.H, n - 1, m - 1) + sigma(sc, q[n - 1], s[m - 1]);
    sc_t Ev = AT(mm.E, n, m) - o + te;
    sc_t Fv = AT(mm.F, n, m);
    char start;
    sc_t best = Dv; start = 'D';
    if (Ev > best) { best = Ev; start = 'E'; }
    if (Fv > best) { best = Fv; start = 'F'; }
    int64_t from = l->len, bi, bj;
    if (start == 'D') {
        op_push(l, 'M');
        traceback(&mm, q, s, sc, ORC_GLOBAL, tb, n - 1, m - 1, 'H', l, &bi, &bj);
    } else {
        traceback(&mm, q, s, sc, ORC_GLOBAL, tb, n, m, start, l, &bi, &bj);
    }
    op_reverse(l->ops, from, l->len);
    *score = best;
    free_mats(&mm);
    return l->err ? ORC_ERR_MEM : ORC_OK;
}

/* ------------------------------------------------------ linear-space scoring */

/*
 * Score and optimum cell in O(m) memory: rows of H and E are kept, F runs
 * along the row (the score-only case of Sec. III-A, Fig. 1 right).
 */
int orc_score(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m,
              const orc_scoring *sc, int mode, orc_result *res) {
    const sc_t o = sc->gap_open, e = sc->gap_extend;
    const sc_t nu = mode == ORC_LOCAL ? 0 : NEG_INF;
    sc_t *H = (sc_t *)malloc((size_t)(m + 1) * sizeof(sc_t));
    sc_t *E = (sc_t *)malloc((size_t)(m + 1) * sizeof(sc_t));
    if (!H || !E) { free(H); free(E); return ORC_ERR_MEM; }
    sc_t best = NEG_INF; int64_t bi = 0, bj = 0;
    H[0] = 0; E[0] = NEG_INF;
    for (int64_t j = 1; j <= m; j++) { H[j] = mode == ORC_GLOBAL ? o + j * e : 0; E[j] = NEG_INF; }
    /* row 0 candidates */
    if (mode == ORC_LOCAL) {
        for (int64_t j = 0; j <= m; j++) if (H[j] > best) { best = H[j]; bi = 0; bj = j; }
    } else if (mode == ORC_SEMIGLOBAL) {
        if (n > 0) { if (H[m] > best) { best = H[m]; bi = 0; bj = m; } }
        else for (int64_t j = 0; j <= m; j++) if (H[j] > best) { best = H[j]; bi = 0; bj = j; }
    }
    for (int64_t i = 1; i <= n; i++) {
        sc_t diag = H[0];
        H[0] = mode == ORC_GLOBAL ? o + i * e : 0;
        sc_t Fv = NEG_INF;
        if (mode == ORC_LOCAL && H[0] > best) { best = H[0]; bi = i; bj = 0; }
        for (int64_t j = 1; j <= m; j++) {
            sc_t Ev = max2(E[j] + e, H[j] + o + e);
            Fv = max2(Fv + e, H[j - 1] + o + e);
            sc_t Dv = diag + sigma(sc, q[i - 1], s[j - 1]);
            sc_t Hv = max2(max2(Dv, Ev), max2(Fv, nu));
            diag = H[j];
            H[j] = Hv; E[j] = Ev;
            if (mode == ORC_LOCAL && Hv > best) { best = Hv; bi = i; bj = j; }
        }
        if (mode == ORC_SEMIGLOBAL) {
            if (i < n) { if (H[m] > best) { best = H[m]; bi = i; bj = m; } }
            else for (int64_t j = 0; j <= m; j++) if (H[j] > best) { best = H[j]; bi = n; bj = j; }
        }
    }
    if (mode == ORC_GLOBAL) { best = H[m]; bi = n; bj = m; }
    res->score = best; res->end_q = bi; res->end_s = bj;
    res->beg_q = res->beg_s = -1;  /* unknown without a traceback */
    free(H); free(E);
    return ORC_OK;
}

/* ----------------------------------------------------- alignment with CIGAR */

int orc_align(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m,
              const orc_scoring *sc, int mode, orc_result *res,
              uint32_t *cigar, int64_t cap, int64_t *cigar_len) {
    oplist l = { NULL, 0, 0, 0 };
    int rc = ORC_OK;
    if (mode == ORC_GLOBAL) {
        sc_t score;
        rc = global_sub(q, n, s, m, sc, sc->gap_open, sc->gap_open, &l, &score);
        if (rc) { free(l.ops); return rc; }
        res->score = score; res->beg_q = 0; res->beg_s = 0; res->end_q = n; res->end_s = m;
    } else {
        mats mm;
        rc = fill_full(q, n, s, m, sc, mode, 0, &mm);
        if (rc) return rc;
        int64_t ei, ej, bi, bj;
        find_end(&mm, mode, &ei, &ej);
        traceback(&mm, q, s, sc, mode, 0, ei, ej, 'H', &l, &bi, &bj);
        op_reverse(l.ops, 0, l.len);
        res->score = AT(mm.H, ei, ej);
        res->end_q = ei; res->end_s = ej; res->beg_q = bi; res->beg_s = bj;
        free_mats(&mm);
    }
    if (l.err) { free(l.ops); return ORC_ERR_MEM; }
    int64_t nc = ops_to_cigar(l.ops, l.len, cigar, cap);
    *cigar_len = nc;
    free(l.ops);
    return nc > cap ? ORC_ERR_CAP : ORC_OK;
}

/* -------------------------------------------------------------- Hirschberg */

/*
 * Forward pass over rows 1..n of a global subproblem with column-0 open tb:
 * CC[j] = H(n, j), DD[j] = E(n, j) for j = 0..m (Sec. III-A linear space).
 * 'rev' reads both sequences from their ends (the reversed relaxation order
 * of the divide-and-conquer traceback).
 */
int orc_last_row(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m,
                 const orc_scoring *sc, int64_t tb, int rev, int64_t *CC, int64_t *DD) {
    const sc_t o = sc->gap_open, e = sc->gap_extend;
    CC[0] = 0; DD[0] = NEG_INF;
    for (int64_t j = 1; j <= m; j++) { CC[j] = o + j * e; DD[j] = NEG_INF; }
    for (int64_t i = 1; i <= n; i++) {
        uint8_t qi = rev ? q[n - i] : q[i - 1];
        sc_t diag = CC[0];
        CC[0] = tb + i * e;
        DD[0] = CC[0];
        sc_t Fv = NEG_INF;
        for (int64_t j = 1; j <= m; j++) {
            uint8_t sj = rev ? s[m - j] : s[j - 1];
            sc_t Ev = max2(DD[j] + e, CC[j] + o + e);
            Fv = max2(Fv + e, CC[j - 1] + o + e);
            sc_t Dv = diag + sigma(sc, qi, sj);
            sc_t Hv = max2(max2(Dv, Ev), Fv);
            diag = CC[j];
            CC[j] = Hv; DD[j] = Ev;
        }
    }
    return ORC_OK;
}

typedef struct {
    const uint8_t *q, *s;
    const orc_scoring *sc;
    int64_t base_cells;
    oplist ops;
    sc_t *CC, *DD, *RR, *SS;
    int err;
    int64_t cells;      /* DP cells relaxed, for the at-most-doubling check */
} hb_ctx;

static void hb(hb_ctx *c, int64_t i0, int64_t i1, int64_t j0, int64_t j1, sc_t tb, sc_t te) {
    if (c->err) return;
    const sc_t o = c->sc->gap_open;
    int64_t rows = i1 - i0, cols = j1 - j0;
    if (rows <= 1 || rows * cols <= c->base_cells) {
        sc_t score;
        c->cells += rows * cols;
        if (global_sub(c->q + i0, rows, c->s + j0, cols, c->sc, tb, te, &c->ops, &score)) c->err = 1;
        return;
    }
    int64_t mid = (i0 + i1) / 2;
    /* forward over rows i0+1..mid, reverse over rows i1..mid+1 */
    orc_last_row(c->q + i0, mid - i0, c->s + j0, cols, c->sc, tb, 0, c->CC, c->DD);
    orc_last_row(c->q + mid, i1 - mid, c->s + j0, cols, c->sc, te, 1, c->RR, c->SS);
    c->cells += rows * cols;
    sc_t best = NEG_INF; int64_t bj = j0; int btype = 1;
    for (int64_t j = j0; j <= j1; j++) {
        int64_t k = j - j0, kr = j1 - j;
        sc_t v1 = c->CC[k] + c->RR[kr];
        sc_t v2 = c->DD[k] + c->SS[kr] - o;
        if (v1 > best) { best = v1; bj = j; btype = 1; }
        if (v2 > best) { best = v2; bj = j; btype = 2; }
    }
    if (btype == 1) {
        hb(c, i0, mid, j0, bj, tb, o);
        hb(c, mid, i1, bj, j1, o, te);
    } else {
        hb(c, i0, mid - 1, j0, bj, tb, 0);
        op_push(&c->ops, 'I'); op_push(&c->ops, 'I');
        hb(c, mid + 1, i1, bj, j1, 0, te);
    }
}

/* Global alignment with the linear-space divide-and-conquer traceback. */
int orc_hirschberg(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m,
                   const orc_scoring *sc, int64_t base_cells, uint32_t *cigar, int64_t cap,
                   int64_t *cigar_len, int64_t *cells_relaxed) {
    hb_ctx c;
    memset(&c, 0, sizeof(c));
    c.q = q; c.s = s; c.sc = sc; c.base_cells = base_cells;
    c.CC = (sc_t *)malloc((size_t)(m + 1) * sizeof(sc_t));
    c.DD = (sc_t *)malloc((size_t)(m + 1) * sizeof(sc_t));
    c.RR = (sc_t *)malloc((size_t)(m + 1) * sizeof(sc_t));
    c.SS = (sc_t *)malloc((size_t)(m + 1) * sizeof(sc_t));
    int rc = ORC_OK;
    if (!c.CC || !c.DD || !c.RR || !c.SS) rc = ORC_ERR_MEM;
    else {
        hb(&c, 0, n, 0, m, sc->gap_open, sc->gap_open);
        if (c.err || c.ops.err) rc = ORC_ERR_MEM;
    }
    if (rc == ORC_OK) {
        int64_t nc = ops_to_cigar(c.ops.ops, c.ops.len, cigar, cap);
        *cigar_len = nc;
        if (cells_relaxed) *cells_relaxed = c.cells;
        if (nc > cap) rc = ORC_ERR_CAP;
    }
    free(c.CC); free(c.DD); free(c.RR); free(c.SS); free(c.ops.ops);
    return rc;
}

/* ------------------------------------------- start of a long-pair traceback */

/*
 * Local and semi-global long pairs are traced back in linear space: the
 * alignment ends at the optimum cell (ei, ej) of score S (orc_score), and
 * between its start and that cell it is a global alignment (Eq. 1 with global
 * initialisation) of the two substrings. For every start (i, j), i <= ei and
 * j <= ej, G(i, j) = global score of q[i..ei) against s[j..ej); the optimal
 * alignments ending at (ei, ej) are those whose start has G = S, among the
 * starts the mode allows (local: any cell; semi-global: row 0 or column 0,
 * where its free leading gaps end). The start taken is the allowed cell of
 * largest G, ties: largest i, then largest j.
 *
 * G over all starts is one DP over the reversed prefixes (the recurrences of
 * orc_last_row, reading q and s from ei and ej backwards): cell (r, c) is the
 * start (ei - r, ej - c). Scanning r and then c upwards and keeping strict
 * improvements gives the tie rule.
 */
int orc_start_cell(const uint8_t *q, int64_t ei, const uint8_t *s, int64_t ej,
                   const orc_scoring *sc, int mode, int64_t *best, int64_t *bi, int64_t *bj) {
    const sc_t o = sc->gap_open, e = sc->gap_extend;
    sc_t *CC = (sc_t *)malloc((size_t)(ej + 1) * sizeof(sc_t));
    sc_t *DD = (sc_t *)malloc((size_t)(ej + 1) * sizeof(sc_t));
    if (!CC || !DD) { free(CC); free(DD); return ORC_ERR_MEM; }
    sc_t bv = NEG_INF; int64_t br = 0, bc = 0;
#define ORC_START_CAND(r, c, v)                                                        \
    do {                                                                               \
        int ok = mode == ORC_LOCAL || (r) == ei || (c) == ej;                          \
        if (ok && (v) > bv) { bv = (v); br = (r); bc = (c); }                           \
    } while (0)
    CC[0] = 0; DD[0] = NEG_INF;
    for (int64_t c = 1; c <= ej; c++) { CC[c] = o + c * e; DD[c] = NEG_INF; }
    for (int64_t c = 0; c <= ej; c++) ORC_START_CAND(0, c, CC[c]);
    for (int64_t r = 1; r <= ei; r++) {
        uint8_t qi = q[ei - r];
        sc_t diag = CC[0];
        CC[0] = o + r * e;
        DD[0] = CC[0];
        ORC_START_CAND(r, 0, CC[0]);
        sc_t Fv = NEG_INF;
        for (int64_t c = 1; c <= ej; c++) {
            uint8_t sj = s[ej - c];
            sc_t Ev = max2(DD[c] + e, CC[c] + o + e);
            Fv = max2(Fv + e, CC[c - 1] + o + e);
            sc_t Hv = max2(max2(diag + sigma(sc, qi, sj), Ev), Fv);
            diag = CC[c];
            CC[c] = Hv; DD[c] = Ev;
            ORC_START_CAND(r, c, Hv);
        }
    }
#undef ORC_START_CAND
    free(CC); free(DD);
    *best = bv; *bi = ei - br; *bj = ej - bc;
    return ORC_OK;
}

/* --------------------------------------------------------------- batches */

/* Score-only over pairs [p0, p1) of a batch (offsets index the code arrays). */
int orc_score_batch(const uint8_t *q, const int64_t *q_off, const uint8_t *s, const int64_t *s_off,
                    int64_t p0, int64_t p1, const orc_scoring *sc, int mode, orc_result *res) {
    for (int64_t p = p0; p < p1; p++) {
        int rc = orc_score(q + q_off[p], q_off[p + 1] - q_off[p], s + s_off[p], s_off[p + 1] - s_off[p],
                           sc, mode, &res[p]);
        if (rc) return rc;
    }
    return ORC_OK;
}

/* Alignment with CIGAR over pairs [p0, p1); pair p writes at cigar + cig_off[p], at most cig_cap[p] words. */
int orc_align_batch(const uint8_t *q, const int64_t *q_off, const uint8_t *s, const int64_t *s_off,
                    int64_t p0, int64_t p1, const orc_scoring *sc, int mode, orc_result *res,
                    uint32_t *cigar, const int64_t *cig_off, int64_t *cig_len) {
    for (int64_t p = p0; p < p1; p++) {
        int64_t cap = cig_off[p + 1] - cig_off[p];
        int rc = orc_align(q + q_off[p], q_off[p + 1] - q_off[p], s + s_off[p], s_off[p + 1] - s_off[p],
                           sc, mode, &res[p], cigar + cig_off[p], cap, &cig_len[p]);
        if (rc) return rc;
    }
    return ORC_OK;
}
