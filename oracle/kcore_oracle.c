/*
 * k-core ORACLE -- test infrastructure, not part of the library.
 *
 * Plain, slow-but-linear, single-threaded CPU code that states what the GPU
 * path must compute.  Only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header or table with the CUDA library.
 *
 * Contents (each function cites the passage it follows):
 *   orc_csr_build      undirected simple CSR from raw edge samples: both
 *                      directions, self-loops dropped, rows sorted ascending,
 *                      duplicates removed (Sec. IV-A: inputs treated as
 *                      undirected with self-loops removed; Sec. III-B "Sorted
 *                      Vectors": neighbour lists kept as sorted vectors).
 *   orc_hindex         the capped h-index used as computeCoreness in Alg. 1
 *                      (the body is not printed in the paper; reading: the
 *                      largest h <= cap such that at least h of the values are
 *                      >= h).
 *   orc_bz             coreness by Batagelj-Zaversnik bucket peeling (the O(m)
 *                      sequential algorithm cited in Sec. II): repeatedly take a
 *                      vertex of minimum current degree; that degree is its
 *                      coreness (Def. 1 and the coreness definition after it).
 *   orc_montresor_sync the synchronous round structure of Alg. 3 (FastK worker):
 *                      active vertices recompute against a snapshot of est,
 *                      updates and activations are applied after the round;
 *                      activation by the selective-sending rule of Sec. III-B
 *                      (new_u < est[v]) or, optionally, the refined rule of
 *                      Sec. IV "Further Optimizations" read as the conjunction
 *                      new_u < est[v] <= old_u, decided after the update phase
 *                      (the extra barrier that passage mentions).
 *
 * Pins: see tests/test_oracle.py (brute force over vertex subsets from Def. 1,
 * repeated min-degree deletion, closed forms, invariants, networkx).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void orc_free(void* p) { free(p); }

/*
 * Build the cleaned CSR.  Every sample (s, d) with s != d contributes the
 * ordered pairs (s, d) and (d, s).  The pairs are put in (row, col) order by
 * two stable counting sorts (first by col, then by row), and repeated pairs
 * are dropped.  Outputs are malloc'd: *row_ptr has n+1 entries, *col has
 * row_ptr[n] entries.  Returns row_ptr[n] (= 2m), or -1 on bad input / no
 * memory.
 */
int64_t orc_csr_build(int64_t n, int64_t samples, const int32_t* src, const int32_t* dst,
                      int64_t** row_ptr_out, int32_t** col_out) {
    *row_ptr_out = NULL;
    *col_out = NULL;
    if (n < 0 || samples < 0) return -1;
    int64_t pairs = 0;
    for (int64_t i = 0; i < samples; i++) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return -1;
        if (src[i] != dst[i]) pairs += 2;
    }
    int32_t* ra = (int32_t*)malloc((size_t)(pairs ? pairs : 1) * sizeof(int32_t));
    int32_t* ca = (int32_t*)malloc((size_t)(pairs ? pairs : 1) * sizeof(int32_t));
    int32_t* rb = (int32_t*)malloc((size_t)(pairs ? pairs : 1) * sizeof(int32_t));
    int32_t* cb = (int32_t*)malloc((size_t)(pairs ? pairs : 1) * sizeof(int32_t));
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* row_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!ra || !ca || !rb || !cb || !cnt || !row_ptr) {
        free(ra); free(ca); free(rb); free(cb); free(cnt); free(row_ptr);
        return -1;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < samples; i++) {
        if (src[i] == dst[i]) continue;
        ra[k] = src[i]; ca[k] = dst[i]; k++;
        ra[k] = dst[i]; ca[k] = src[i]; k++;
    }
    /* stable counting sort by column: (ra, ca) -> (rb, cb) */
    memset(cnt, 0, (size_t)(n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < pairs; i++) cnt[ca[i] + 1]++;
    for (int64_t v = 0; v < n; v++) cnt[v + 1] += cnt[v];
    for (int64_t i = 0; i < pairs; i++) {
        int64_t p = cnt[ca[i]]++;
        rb[p] = ra[i]; cb[p] = ca[i];
    }
    /* stable counting sort by row: (rb, cb) -> (ra, ca); now (row, col) ordered */
    memset(cnt, 0, (size_t)(n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < pairs; i++) cnt[rb[i] + 1]++;
    for (int64_t v = 0; v < n; v++) cnt[v + 1] += cnt[v];
    for (int64_t i = 0; i < pairs; i++) {
        int64_t p = cnt[rb[i]]++;
        ra[p] = rb[i]; ca[p] = cb[i];
    }
    /* drop repeats, count kept entries per row */
    int64_t kept = 0;
    for (int64_t i = 0; i < pairs; i++) {
        if (i > 0 && ra[i] == ra[i - 1] && ca[i] == ca[i - 1]) continue;
        ca[kept] = ca[i];
        row_ptr[ra[i] + 1]++;
        kept++;
    }
    for (int64_t v = 0; v < n; v++) row_ptr[v + 1] += row_ptr[v];
    free(ra); free(rb); free(cb); free(cnt);
    int32_t* col = (int32_t*)realloc(ca, (size_t)(kept ? kept : 1) * sizeof(int32_t));
    if (!col) col = ca;
    *row_ptr_out = row_ptr;
    *col_out = col;
    return kept;
}

/*
 * Capped h-index: the largest h in [0, cap] such that at least h of the
 * `count` values are >= h.  Counted directly: c[j] = number of values >= j,
 * taken from a histogram of min(value, cap) summed from the top.
 * Returns -1 on bad input.
 */
int32_t orc_hindex(const int32_t* values, int64_t count, int32_t cap) {
    if (cap < 0 || count < 0) return -1;
    if (cap > count) cap = (int32_t)count;   /* h can never exceed the count */
    int64_t* hist = (int64_t*)calloc((size_t)cap + 1, sizeof(int64_t));
    if (!hist) return -1;
    for (int64_t i = 0; i < count; i++) {
        int32_t x = values[i];
        if (x < 0) x = 0;
        hist[x < cap ? x : cap]++;
    }
    int64_t at_least = 0;  /* number of values >= h */
    int32_t h = 0;
    for (int32_t j = cap; j >= 1; j--) {
        at_least += hist[j];
        if (at_least >= j) { h = j; break; }
    }
    free(hist);
    return h;
}

/*
 * Batagelj-Zaversnik peeling.  Vertices are kept in an array ordered by
 * current degree (bucket starts bin[d], position pos[v]).  Scanning that array
 * left to right, the vertex v reached has minimum current degree among those
 * not yet scanned; its coreness is that degree.  Each neighbour u with a
 * larger current degree loses one: it is swapped with the first vertex of its
 * bucket, the bucket start advances, and deg[u] decreases.
 * Returns 0, or -1 on no memory.
 */
int orc_bz(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t* core) {
    if (n == 0) return 0;
    int64_t* deg = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* pos = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* vert = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t maxd = 0;
    if (!deg || !pos || !vert) { free(deg); free(pos); free(vert); return -1; }
    for (int64_t v = 0; v < n; v++) {
        deg[v] = row_ptr[v + 1] - row_ptr[v];
        if (deg[v] > maxd) maxd = deg[v];
    }
    int64_t* bin = (int64_t*)calloc((size_t)maxd + 2, sizeof(int64_t));
    if (!bin) { free(deg); free(pos); free(vert); return -1; }
    for (int64_t v = 0; v < n; v++) bin[deg[v]]++;
    int64_t start = 0;
    for (int64_t d = 0; d <= maxd; d++) {
        int64_t num = bin[d];
        bin[d] = start;
        start += num;
    }
    for (int64_t v = 0; v < n; v++) {
        pos[v] = bin[deg[v]];
        vert[pos[v]] = v;
        bin[deg[v]]++;
    }
    for (int64_t d = maxd; d >= 1; d--) bin[d] = bin[d - 1];
    bin[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t v = vert[i];
        core[v] = (int32_t)deg[v];
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            int64_t u = col[e];
            if (deg[u] > deg[v]) {
                int64_t du = deg[u];
                int64_t pu = pos[u];
                int64_t pw = bin[du];
                int64_t w = vert[pw];
                if (u != w) {
                    pos[u] = pw; vert[pu] = w;
                    pos[w] = pu; vert[pw] = u;
                }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    free(deg); free(pos); free(vert); free(bin);
    return 0;
}

/*
 * Synchronous Montresor rounds (Alg. 3 semantics).
 *   est[v] starts at deg(v); every vertex starts active.
 *   Round s: each active u is deactivated and computes
 *   t = orc_hindex(est[N(u)], cap = est[u]) against the est of the previous
 *   round.  If t < est[u], the update (u, t) is recorded, and each neighbour
 *   v with t < est[v] (and, when refined != 0, also est[v] <= est[u]) is
 *   recorded for activation.  After all active vertices are done, updates are
 *   written and activations applied.
 *   The refined rule costs an extra barrier (Sec. IV, Further Optimizations):
 *   it is decided after the updates are written, so est[v] there is v's value
 *   after this round.  Checked against the pre-round snapshot it is wrong: v
 *   may have lowered in the same round to a value that u's old estimate
 *   supported.
 * Stops when no vertex is active (returns the number of rounds run) or after
 * max_rounds rounds with vertices still active (returns -1).  est_out gets
 * the estimates after the last round run.  If frontier_out is non-NULL,
 * frontier_out[s] = active count at the start of round s and changed_out[s] =
 * number of updates in round s, for s < max_record.
 */
int64_t orc_montresor_sync(int64_t n, const int64_t* row_ptr, const int32_t* col,
                           int64_t max_rounds, int refined, int32_t* est_out,
                           int64_t* frontier_out, int64_t* changed_out, int64_t max_record) {
    int32_t* est = est_out;
    uint8_t* active = (uint8_t*)malloc((size_t)(n ? n : 1));
    uint8_t* next_active = (uint8_t*)calloc((size_t)(n ? n : 1), 1);
    int32_t* upd_val = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int64_t* upd_id = (int64_t*)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t maxd = 1;
    for (int64_t v = 0; v < n; v++)
        if (row_ptr[v + 1] - row_ptr[v] > maxd) maxd = row_ptr[v + 1] - row_ptr[v];
    int32_t* vals = (int32_t*)malloc((size_t)maxd * sizeof(int32_t));
    if (!active || !next_active || !upd_val || !upd_id || !vals) {
        free(active); free(next_active); free(upd_val); free(upd_id); free(vals);
        return -2;
    }
    for (int64_t v = 0; v < n; v++) {
        est[v] = (int32_t)(row_ptr[v + 1] - row_ptr[v]);
        active[v] = 1;
    }
    int64_t rounds = 0;
    for (;;) {
        int64_t nactive = 0;
        for (int64_t v = 0; v < n; v++) nactive += active[v];
        if (nactive == 0) break;
        if (rounds >= max_rounds) { rounds = -1; break; }
        int64_t nupd = 0;
        for (int64_t u = 0; u < n; u++) {
            if (!active[u]) continue;
            active[u] = 0;
            int64_t d = row_ptr[u + 1] - row_ptr[u];
            for (int64_t j = 0; j < d; j++) vals[j] = est[col[row_ptr[u] + j]];
            int32_t t = orc_hindex(vals, d, est[u]);
            if (t < est[u]) {
                upd_id[nupd] = u; upd_val[nupd] = t; nupd++;
                if (!refined)
                    for (int64_t j = 0; j < d; j++)
                        if (t < vals[j]) next_active[col[row_ptr[u] + j]] = 1;
            }
        }
        for (int64_t i = 0; i < nupd; i++) {   /* write updates; keep old values */
            int64_t u = upd_id[i];
            int32_t t = upd_val[i];
            upd_val[i] = est[u];
            est[u] = t;
        }
        if (refined) {                          /* activation after the updates */
            for (int64_t i = 0; i < nupd; i++) {
                int64_t u = upd_id[i];
                int32_t old_u = upd_val[i], new_u = est[u];
                for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
                    int32_t x = est[col[e]];
                    if (new_u < x && x <= old_u) next_active[col[e]] = 1;
                }
            }
        }
        for (int64_t v = 0; v < n; v++) {
            active[v] = next_active[v];
            next_active[v] = 0;
        }
        if (frontier_out && rounds < max_record) {
            frontier_out[rounds] = nactive;
            changed_out[rounds] = nupd;
        }
        rounds++;
    }
    free(active); free(next_active); free(upd_val); free(upd_id); free(vals);
    return rounds;
}
