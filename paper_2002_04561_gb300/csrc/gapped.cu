// Gapped strings of an alignment, the output form of the paper's one-pair
// interface (construct_global_alignment, Sec. III-C listing): the aligned part
// of each sequence with '-' where the other sequence has a letter against a
// gap. Host code: it reads a CIGAR and the two sequences and writes characters.
#include <cstring>

#include "../../include/anyseq.h"
#include "api_internal.h"

using anyseq::fail;

extern "C" anyseq_status_t anyseq_gapped(const uint8_t *q, int64_t n, const uint8_t *s, int64_t m, int32_t beg_q,
                                         int32_t beg_s, const uint32_t *cigar, uint32_t cigar_len,
                                         const char *letters, int32_t alphabet, char *q_out, char *s_out, int64_t cap,
                                         int64_t *len) {
    if (!len || (cigar_len && !cigar) || !letters || alphabet < 1)
        return fail(ANYSEQ_ERR_ARG, "len, cigar and letters must not be NULL");
    if ((int64_t)strlen(letters) < alphabet) return fail(ANYSEQ_ERR_ARG, "letters holds fewer than alphabet characters");
    if (beg_q < 0 || beg_s < 0 || beg_q > n || beg_s > m) return fail(ANYSEQ_ERR_ARG, "start cell outside the pair");
    // columns and consumed letters
    int64_t cols = 0, i = beg_q, j = beg_s;
    for (uint32_t k = 0; k < cigar_len; k++) {
        const int64_t l = cigar[k] >> 4;
        const uint32_t op = cigar[k] & 15u;
        if (op > 2) return fail(ANYSEQ_ERR_ARG, "CIGAR op %u is not M, I or D", op);
        cols += l;
        if (op != 2) i += l;
        if (op != 1) j += l;
    }
    if (i > n || j > m) return fail(ANYSEQ_ERR_ARG, "the CIGAR runs past the end of a sequence");
    *len = cols;
    if (cap < cols + 1) return fail(ANYSEQ_ERR_CAPACITY, "buffers hold %lld characters, %lld needed", (long long)cap,
                                    (long long)(cols + 1));
    if (!q_out || !s_out) return fail(ANYSEQ_ERR_ARG, "q_out and s_out must not be NULL");
    i = beg_q;
    j = beg_s;
    int64_t c = 0;
    for (uint32_t k = 0; k < cigar_len; k++) {
        const int64_t l = cigar[k] >> 4;
        const uint32_t op = cigar[k] & 15u;
        for (int64_t t = 0; t < l; t++, c++) {
            if (op != 2 && q[i] >= alphabet) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", alphabet);
            if (op != 1 && s[j] >= alphabet) return fail(ANYSEQ_ERR_ALPHABET, "a letter code is >= alphabet (%d)", alphabet);
            q_out[c] = op != 2 ? letters[q[i++]] : '-';
            s_out[c] = op != 1 ? letters[s[j++]] : '-';
        }
    }
    q_out[cols] = 0;
    s_out[cols] = 0;
    return ANYSEQ_OK;
}
