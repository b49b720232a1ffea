// Partition of one batch over the ranks of a data-parallel job. Pairs are
// independent (the inter-sequence parallelism of Sec. VI), so each rank aligns
// a share of them and the only exchange is a gather of the results.
//
// Length-balanced round-robin of bins: every pair falls into the 8-bit
// logarithmic bin of its cell count n * m (8 bins per octave, lbucket of
// batch.h). Bins are taken from the largest down, pairs inside a bin in index
// order, and the whole sequence is dealt to the ranks in snake order (0, 1,
// ..., W-1, W-1, ..., 1, 0, 0, 1, ...). Every rank thus gets its turn in every
// length class, the pair counts differ by at most one, and the cell counts by
// about the largest pair. Host code, no GPU work.
#include <algorithm>
#include <vector>

#include "../../include/anyseq.h"
#include "api_internal.h"
#include "batch.h"

using anyseq::fail;

extern "C" anyseq_status_t anyseq_shard_plan(const int64_t *q_off, const int64_t *s_off, int64_t n_pairs, int32_t world,
                                             int32_t rank, int64_t *idx, int64_t cap, int64_t *count) {
    if (!count || (n_pairs > 0 && (!q_off || !s_off))) return fail(ANYSEQ_ERR_ARG, "offsets and count must not be NULL");
    if (n_pairs < 0 || world < 1 || rank < 0 || rank >= world)
        return fail(ANYSEQ_ERR_ARG, "need n_pairs >= 0 and 0 <= rank < world (got %d of %d)", rank, world);
    // pairs per bin, bins from the largest cell count down
    std::vector<int64_t> start(257, 0);
    std::vector<uint8_t> bin((size_t)n_pairs);
    for (int64_t p = 0; p < n_pairs; p++) {
        const int64_t n = q_off[p + 1] - q_off[p], m = s_off[p + 1] - s_off[p];
        if (n < 0 || m < 0) return fail(ANYSEQ_ERR_ARG, "offsets of pair %lld decrease", (long long)p);
        bin[p] = (uint8_t)(255u - anyseq::lbucket(n * m));
        start[bin[p] + 1]++;
    }
    for (int b = 0; b < 256; b++) start[b + 1] += start[b];
    std::vector<int64_t> order((size_t)n_pairs);
    for (int64_t p = 0; p < n_pairs; p++) order[start[bin[p]]++] = p;  // stable: index order inside a bin
    // snake deal: position t goes to rank t mod W, or W-1 - (t mod W) on odd rounds
    int64_t k = 0;
    const int64_t need = (n_pairs + world - 1) / world;
    for (int64_t t = 0; t < n_pairs; t++) {
        const int64_t round = t / world, pos = t % world;
        const int64_t r = (round & 1) ? world - 1 - pos : pos;
        if (r != rank) continue;
        if (idx && k < cap) idx[k] = order[t];
        k++;
    }
    *count = k;
    if (k > cap || (k > 0 && !idx)) return fail(ANYSEQ_ERR_CAPACITY, "the index buffer holds %lld entries, %lld needed",
                                                (long long)cap, (long long)need);
    std::sort(idx, idx + k);
    return ANYSEQ_OK;
}
