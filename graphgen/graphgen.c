/*
 * Seeded synthetic graph generators.
 *
 * These produce the directed edge samples (src[i], dst[i]) that both the GPU
 * library and the CPU oracle consume.  They hold none of the k-core arithmetic:
 * no symmetrisation, no deduplication of the output, no degrees, no coreness.
 * Edges may contain self-loops, both directions of a pair, and repeats, exactly
 * as a raw edge file would (the paper's inputs are treated as undirected with
 * self-loops removed, Sec. IV-A); cleaning them is the consumer's job.
 *
 * Randomness: one counter-based generator, the SplitMix64 output function
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014).  Output i of the stream keyed by (seed, stream) is
 * mix(key + (i + 1) * GAMMA), so any sample can be computed independently and
 * the result does not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of one named stream under one seed. */
static inline uint64_t gg_key(uint64_t seed, uint64_t stream) {
    return gg_mix(seed * GG_GAMMA + gg_mix(stream + 0x632BE59BD9B4E019ULL));
}

static inline uint64_t gg_at(uint64_t key, uint64_t i) {
    return gg_mix(key + (i + 1) * GG_GAMMA);
}

/* Uniform double in [0, 1) from the top 53 bits. */
static inline double gg_unit(uint64_t r) {
    return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

/* Integer in [0, n) by the multiply-shift map (Lemire 2019). */
static inline uint64_t gg_below(uint64_t r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)r * n) >> 64);
}

enum { S_ER = 1, S_GRID_H, S_GRID_V, S_DIAG, S_DIAG_PICK, S_RMAT, S_PERM,
       S_PLANT_PICK, S_PLANT_EDGE, S_STREAM };

uint64_t gg_random(uint64_t seed, uint64_t stream, uint64_t i) {
    return gg_at(gg_key(seed, stream), i);
}

/*
 * Erdos-Renyi G(n, m): uniform vertex pairs are drawn until m distinct
 * non-loop unordered pairs have been accepted.  Writes exactly m edges, each
 * pair once, in acceptance order.  Returns m, or -1 if m exceeds n(n-1)/2 or
 * memory runs out.
 */
int64_t gg_er(int64_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst) {
    if (n < 0 || m < 0) return -1;
    if (m == 0) return 0;
    if (n < 2 || (double)m > (double)n * (double)(n - 1) / 2.0) return -1;
    uint64_t cap = 1;
    while (cap < (uint64_t)m * 2 + 16) cap <<= 1;
    uint64_t* table = (uint64_t*)calloc(cap, sizeof(uint64_t));
    if (!table) return -1;
    uint64_t key = gg_key(seed, S_ER);
    int64_t got = 0;
    for (uint64_t i = 0; got < m; i += 2) {
        uint64_t a = gg_below(gg_at(key, i), (uint64_t)n);
        uint64_t b = gg_below(gg_at(key, i + 1), (uint64_t)n);
        if (a == b) continue;
        uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
        uint64_t k = ((lo << 32) | hi) + 1;
        uint64_t h = gg_mix(k) & (cap - 1);
        int dup = 0;
        while (table[h]) {
            if (table[h] == k) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        table[h] = k;
        src[got] = (int32_t)a;
        dst[got] = (int32_t)b;
        got++;
    }
    free(table);
    return got;
}

/*
 * Damaged L x L grid: the 4-neighbour grid (vertex r*L + c), each grid edge
 * deleted independently with probability p_del, then each vertex, with
 * probability p_diag, adds one edge to a uniformly chosen in-bounds diagonal
 * neighbour.  Capacity needed: 2L(L-1) + L*L.  Returns the edge count.
 */
int64_t gg_damaged_grid(int64_t L, double p_del, double p_diag, uint64_t seed,
                        int32_t* src, int32_t* dst) {
    if (L < 1 || L > 46340) return -1;
    uint64_t kh = gg_key(seed, S_GRID_H), kv = gg_key(seed, S_GRID_V);
    uint64_t kd = gg_key(seed, S_DIAG), kp = gg_key(seed, S_DIAG_PICK);
    int64_t e = 0;
    for (int64_t r = 0; r < L; r++)
        for (int64_t c = 0; c + 1 < L; c++) {
            uint64_t idx = (uint64_t)(r * (L - 1) + c);
            if (gg_unit(gg_at(kh, idx)) >= p_del) {
                src[e] = (int32_t)(r * L + c); dst[e] = (int32_t)(r * L + c + 1); e++;
            }
        }
    for (int64_t r = 0; r + 1 < L; r++)
        for (int64_t c = 0; c < L; c++) {
            uint64_t idx = (uint64_t)(r * L + c);
            if (gg_unit(gg_at(kv, idx)) >= p_del) {
                src[e] = (int32_t)(r * L + c); dst[e] = (int32_t)((r + 1) * L + c); e++;
            }
        }
    for (int64_t r = 0; r < L; r++)
        for (int64_t c = 0; c < L; c++) {
            uint64_t v = (uint64_t)(r * L + c);
            if (gg_unit(gg_at(kd, v)) >= p_diag) continue;
            int64_t cand[4]; int nc = 0;
            for (int dr = -1; dr <= 1; dr += 2)
                for (int dc = -1; dc <= 1; dc += 2) {
                    int64_t rr = r + dr, cc = c + dc;
                    if (rr >= 0 && rr < L && cc >= 0 && cc < L) cand[nc++] = rr * L + cc;
                }
            if (nc == 0) continue;
            int64_t w = cand[gg_below(gg_at(kp, v), (uint64_t)nc)];
            src[e] = (int32_t)v; dst[e] = (int32_t)w; e++;
        }
    return e;
}

/*
 * Seeded uniform permutation of [0, n) by Fisher-Yates, drawing from the
 * stream `stream`.
 */
static void gg_perm(int64_t n, uint64_t seed, uint64_t stream, int32_t* perm) {
    uint64_t key = gg_key(seed, stream);
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; i--) {
        int64_t j = (int64_t)gg_below(gg_at(key, (uint64_t)i), (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/*
 * R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004) on n vertices with
 * scale = ceil(log2 n): `samples` directed edges, each chosen by `scale`
 * recursive quadrant draws with probabilities (a, b, c, 1-a-b-c), no noise.
 * Endpoints >= n are rejected and the edge is redrawn (up to 64 attempts; then
 * the endpoints are reduced modulo n).  With relabel != 0 a seeded uniform
 * vertex permutation is applied.  Writes exactly `samples` edges.
 */
int64_t gg_rmat(int64_t n, int64_t samples, double a, double b, double c,
                int relabel, uint64_t seed, int32_t* src, int32_t* dst) {
    if (n < 1 || samples < 0 || n > 2147483647LL) return -1;
    int scale = 0;
    while ((1LL << scale) < n) scale++;
    uint64_t key = gg_key(seed, S_RMAT);
    int32_t* perm = NULL;
    if (relabel) {
        perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        if (!perm) return -1;
        gg_perm(n, seed, S_PERM, perm);
    }
    const double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < samples; i++) {
        uint64_t s = 0, d = 0;
        for (int attempt = 0; attempt < 64; attempt++) {
            s = 0; d = 0;
            uint64_t base = ((uint64_t)i * 64 + (uint64_t)attempt) * (uint64_t)(scale > 0 ? scale : 1);
            for (int l = 0; l < scale; l++) {
                double r = gg_unit(gg_at(key, base + (uint64_t)l));
                uint64_t bit = 1ULL << (scale - 1 - l);
                if (r < a) { }
                else if (r < ab) d |= bit;
                else if (r < abc) s |= bit;
                else { s |= bit; d |= bit; }
            }
            if ((int64_t)s < n && (int64_t)d < n) break;
        }
        s %= (uint64_t)n; d %= (uint64_t)n;
        if (perm) { s = (uint64_t)perm[s]; d = (uint64_t)perm[d]; }
        src[i] = (int32_t)s; dst[i] = (int32_t)d;
    }
    free(perm);
    return samples;
}

/*
 * Planted dense block: k vertices drawn uniformly without replacement from
 * [0, n), and each of their k(k-1)/2 pairs kept independently with
 * probability p (a G(k, p) on that subset).  Capacity k(k-1)/2.  Returns the
 * edge count.
 */
int64_t gg_planted(int64_t n, int64_t k, double p, uint64_t seed, int32_t* src, int32_t* dst) {
    if (k < 0 || k > n) return -1;
    if (k < 2) return 0;
    int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!perm) return -1;
    uint64_t kpick = gg_key(seed, S_PLANT_PICK);
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    for (int64_t i = 0; i < k; i++) {  /* partial Fisher-Yates: first k slots */
        int64_t j = i + (int64_t)gg_below(gg_at(kpick, (uint64_t)i), (uint64_t)(n - i));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    uint64_t kedge = gg_key(seed, S_PLANT_EDGE);
    int64_t e = 0;
    for (int64_t i = 0; i < k; i++)
        for (int64_t j = i + 1; j < k; j++)
            if (gg_unit(gg_at(kedge, (uint64_t)(i * k + j))) < p) {
                src[e] = perm[i]; dst[e] = perm[j]; e++;
            }
    free(perm);
    return e;
}

/*
 * Parameters of graph `index` of the batch stream: vertex count log-uniform
 * in [nmin, nmax], and a family uniform over {0: ER, 1: R-MAT, 2: damaged
 * grid}.  For the grid the vertex count becomes side^2, side = round(sqrt(n)).
 */
void gg_stream_params(uint64_t seed, int64_t index, int64_t nmin, int64_t nmax,
                      int64_t* n_out, int32_t* family_out) {
    uint64_t key = gg_key(seed, S_STREAM);
    double u = gg_unit(gg_at(key, (uint64_t)index * 2));
    double ln = log((double)nmin) + u * (log((double)nmax) - log((double)nmin));
    int64_t n = (int64_t)llround(exp(ln));
    if (n < nmin) n = nmin;
    if (n > nmax) n = nmax;
    int32_t fam = (int32_t)gg_below(gg_at(key, (uint64_t)index * 2 + 1), 3);
    if (fam == 2) {
        int64_t side = (int64_t)llround(sqrt((double)n));
        if (side < 1) side = 1;
        n = side * side;
    }
    *n_out = n;
    *family_out = fam;
}
