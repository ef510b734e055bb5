/*
 * Seeded synthetic inputs for the SKIS workloads: directed Erdos-Renyi,
 * directed Chung-Lu (power-law expected degrees), R-MAT, and trivalency
 * (TRI) edge probabilities.
 *
 * This module holds none of the method's arithmetic. It only produces edge
 * lists (src, dst) and, for TRI, one probability per input edge, so that the
 * CUDA path and the CPU oracle can be fed the same input. Its randomness is a
 * counter-based hash built on the SplitMix64 finaliser (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014); it is
 * unrelated to the Philox generator that the method itself uses.
 *
 * Edge generation is parallel over edge indices (OpenMP); every edge is a
 * pure function of (seed, edge index, redraw counter), so the output does not
 * depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN64 0x9E3779B97F4A7C15ull

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Counter-based draw: a 64-bit word that depends on (seed, stream, a, b). */
static inline uint64_t draw64(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b)
{
    uint64_t z = mix64(seed + GOLDEN64 * (stream + 1));
    z = mix64(z + GOLDEN64 * (a + 1));
    return mix64(z ^ (b * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull));
}

/* Uniform integer in [0, bound) by the high half of a 64x64 product. */
static inline uint64_t below(uint64_t x, uint64_t bound)
{
    return (uint64_t)(((unsigned __int128)x * bound) >> 64);
}

/* ---------------------------------------------------------------- ER -- */

/* m distinct ordered pairs (u, v), u != v, uniform over all such pairs.
 * Sequential with an open-addressing set of taken pairs; duplicates and
 * self-loops are redrawn with a per-edge redraw counter. Returns 0, or -1 if
 * m exceeds half of the n(n-1) available pairs or memory runs out. */
int synth_er(int64_t n, int64_t m, uint64_t seed, int32_t *src, int32_t *dst)
{
    if (n < 2 || m < 0 || (double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
    uint64_t cap = 1;
    while (cap < (uint64_t)(2 * m + 2)) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(cap * sizeof(uint64_t));
    if (!set) return -1;
    memset(set, 0xFF, cap * sizeof(uint64_t));
    for (int64_t e = 0; e < m; e++) {
        for (uint64_t redraw = 0;; redraw++) {
            uint64_t x = draw64(seed, 11, (uint64_t)e, redraw);
            uint64_t y = draw64(seed, 12, (uint64_t)e, redraw);
            uint64_t u = below(x, (uint64_t)n), v = below(y, (uint64_t)n);
            if (u == v) continue;
            uint64_t key = u * (uint64_t)n + v;
            uint64_t h = mix64(key) & (cap - 1);
            int dup = 0;
            while (set[h] != ~0ull) {
                if (set[h] == key) { dup = 1; break; }
                h = (h + 1) & (cap - 1);
            }
            if (dup) continue;
            set[h] = key;
            src[e] = (int32_t)u;
            dst[e] = (int32_t)v;
            break;
        }
    }
    free(set);
    return 0;
}

/* ------------------------------------------------------ alias (input) -- */

typedef struct {
    double *prob;
    int64_t *alias;
    int64_t n;
} gen_alias;

/* Walker/Vose alias table over double weights (input generation only). */
static int gen_alias_build(gen_alias *t, const double *wt, int64_t n)
{
    t->n = n;
    t->prob = (double *)malloc((size_t)n * sizeof(double));
    t->alias = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *small = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *large = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    double *sc = (double *)malloc((size_t)n * sizeof(double));
    if (!t->prob || !t->alias || !small || !large || !sc) return -1;
    double tot = 0.0;
    for (int64_t i = 0; i < n; i++) tot += wt[i];
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; i++) {
        sc[i] = wt[i] * (double)n / tot;
        if (sc[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        int64_t s = small[--ns], l = large[--nl];
        t->prob[s] = sc[s];
        t->alias[s] = l;
        sc[l] = (sc[l] + sc[s]) - 1.0;
        if (sc[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int64_t l = large[--nl]; t->prob[l] = 1.0; t->alias[l] = l; }
    while (ns > 0) { int64_t s = small[--ns]; t->prob[s] = 1.0; t->alias[s] = s; }
    free(small); free(large); free(sc);
    return 0;
}

static inline int64_t gen_alias_draw(const gen_alias *t, uint64_t x, uint64_t y)
{
    int64_t c = (int64_t)below(x, (uint64_t)t->n);
    double u = (double)(y >> 11) * (1.0 / 9007199254740992.0);
    return u < t->prob[c] ? c : t->alias[c];
}

static void gen_alias_free(gen_alias *t) { free(t->prob); free(t->alias); }

/* Fisher-Yates permutation of 0..n-1 driven by the counter hash. */
static void gen_permutation(int64_t *perm, int64_t n, uint64_t seed, uint64_t stream)
{
    for (int64_t i = 0; i < n; i++) perm[i] = i;
    for (int64_t i = n - 1; i > 0; i--) {
        int64_t j = (int64_t)below(draw64(seed, stream, (uint64_t)i, 0), (uint64_t)(i + 1));
        int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* ----------------------------------------------------------- Chung-Lu -- */

/* Sum of (i + i0 + 1)^ex over i = 0..n-1: the first 2^16 terms exactly, the
 * tail by the midpoint integral (input generation only; a relative error of
 * ~1e-9 in the normaliser is irrelevant here). */
static double chunglu_weight_sum(int64_t n, double i0, double ex)
{
    const int64_t head = n < 65536 ? n : 65536;
    double tot = 0.0;
    for (int64_t i = 0; i < head; i++) tot += pow((double)i + i0 + 1.0, ex);
    if (head < n) {
        double a = (double)head - 0.5 + i0 + 1.0, b = (double)n - 0.5 + i0 + 1.0;
        tot += (pow(b, ex + 1.0) - pow(a, ex + 1.0)) / (ex + 1.0);
    }
    return tot;
}

/* Expected-degree weight of rank i: (i + i0 + 1)^(-1/(beta-1)). The offset
 * i0 is found by bisection so that the largest expected degree,
 * m * w_0 / sum(w), equals sqrt(m) (i0 = 0 if that is already below). */
static double chunglu_offset(int64_t n, int64_t m, double beta)
{
    double ex = -1.0 / (beta - 1.0);
    double target = sqrt((double)m);
    if ((double)m / chunglu_weight_sum(n, 0.0, ex) <= target) return 0.0;
    double lo = 0.0, hi = (double)n;
    for (int it = 0; it < 100 && hi - lo > 1e-9 * (1.0 + lo); it++) {
        double i0 = 0.5 * (lo + hi);
        double maxdeg = (double)m * pow(i0 + 1.0, ex) / chunglu_weight_sum(n, i0, ex);
        if (maxdeg > target) lo = i0; else hi = i0;
    }
    return 0.5 * (lo + hi);
}

/* Directed Chung-Lu: m edges, each endpoint drawn independently by an alias
 * table over the expected-degree weights; in- and out-weights are attached
 * to vertices through two independent random permutations. Self-loops are
 * redrawn; parallel edges are kept. */
int synth_chunglu(int64_t n, int64_t m, double beta, uint64_t seed, int32_t *src, int32_t *dst)
{
    if (n < 2 || m < 0 || !(beta > 1.0)) return -1;
    double i0 = chunglu_offset(n, m, beta);
    double ex = -1.0 / (beta - 1.0);
    double *wt = (double *)malloc((size_t)n * sizeof(double));
    double *wo = (double *)malloc((size_t)n * sizeof(double));
    double *wi = (double *)malloc((size_t)n * sizeof(double));
    int64_t *perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!wt || !wo || !wi || !perm) return -1;
    for (int64_t i = 0; i < n; i++) wt[i] = pow((double)i + i0 + 1.0, ex);
    gen_permutation(perm, n, seed, 21);
    for (int64_t i = 0; i < n; i++) wo[perm[i]] = wt[i];
    gen_permutation(perm, n, seed, 22);
    for (int64_t i = 0; i < n; i++) wi[perm[i]] = wt[i];
    gen_alias ao, ai;
    if (gen_alias_build(&ao, wo, n) || gen_alias_build(&ai, wi, n)) return -1;
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        for (uint64_t redraw = 0;; redraw++) {
            int64_t u = gen_alias_draw(&ao, draw64(seed, 23, (uint64_t)e, redraw),
                                       draw64(seed, 24, (uint64_t)e, redraw));
            int64_t v = gen_alias_draw(&ai, draw64(seed, 25, (uint64_t)e, redraw),
                                       draw64(seed, 26, (uint64_t)e, redraw));
            if (u == v) continue;
            src[e] = (int32_t)u;
            dst[e] = (int32_t)v;
            break;
        }
    }
    gen_alias_free(&ao); gen_alias_free(&ai);
    free(wt); free(wo); free(wi); free(perm);
    return 0;
}

/* -------------------------------------------------------------- R-MAT -- */

/* R-MAT with quadrant probabilities (a, b, c, 1-a-b-c) over 2^scale
 * vertices: each level picks a quadrant from 32 fresh random bits (two
 * levels per 64-bit draw). Quadrant b sets the destination bit, c the source
 * bit, d both. Self-loops are redrawn. */
int synth_rmat(int scale, int64_t m, double a, double b, double c, uint64_t seed,
               int32_t *src, int32_t *dst)
{
    if (scale < 1 || scale > 31 || m < 0) return -1;
    uint64_t ta = (uint64_t)(a * 4294967296.0);
    uint64_t tb = (uint64_t)((a + b) * 4294967296.0);
    uint64_t tc = (uint64_t)((a + b + c) * 4294967296.0);
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        for (uint64_t redraw = 0;; redraw++) {
            uint64_t u = 0, v = 0, x = 0;
            for (int lvl = 0; lvl < scale; lvl++) {
                if ((lvl & 1) == 0) x = draw64(seed, 31 + redraw, (uint64_t)e, (uint64_t)lvl);
                uint64_t r = (lvl & 1) ? (x >> 32) : (x & 0xFFFFFFFFull);
                uint64_t bu = 0, bv = 0;
                if (r < ta) { bu = 0; bv = 0; }
                else if (r < tb) { bu = 0; bv = 1; }
                else if (r < tc) { bu = 1; bv = 0; }
                else { bu = 1; bv = 1; }
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            if (u == v) continue;
            src[e] = (int32_t)u;
            dst[e] = (int32_t)v;
            break;
        }
    }
    return 0;
}

/* ------------------------------------------------------------ weights -- */

/* Trivalency probabilities: each input edge independently and uniformly one
 * of {0.1, 0.01, 0.001}. */
int synth_tri(int64_t m, uint64_t seed, double *p)
{
    static const double levels[3] = {0.1, 0.01, 0.001};
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) p[e] = levels[below(draw64(seed, 41, (uint64_t)e, 0), 3)];
    return 0;
}

/* Uniform random probabilities in [lo, hi) per input edge (tests only). */
int synth_uniform_p(int64_t m, uint64_t seed, double lo, double hi, double *p)
{
    for (int64_t e = 0; e < m; e++) {
        double u = (double)(draw64(seed, 51, (uint64_t)e, 0) >> 11) * (1.0 / 9007199254740992.0);
        p[e] = lo + (hi - lo) * u;
    }
    return 0;
}

/* ---------------------------------------------------------- seed sets -- */

/* q seed sets; query b has size[b] distinct vertices drawn uniformly without
 * replacement by a partial Fisher-Yates shuffle over a scratch permutation,
 * whose swaps are undone afterwards so every query starts from the identity.
 * offsets must have q+1 entries; seeds receives sum(size) vertices. */
int synth_seed_sets(int64_t n, int32_t q, const int32_t *size, uint64_t seed,
                    int64_t *offsets, int32_t *seeds)
{
    int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *swp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!perm || !swp) { free(perm); free(swp); return -1; }
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    offsets[0] = 0;
    for (int32_t b = 0; b < q; b++) {
        int64_t s = size[b];
        if (s < 0 || s > n) { free(perm); free(swp); return -1; }
        for (int64_t i = 0; i < s; i++) {
            int64_t j = i + (int64_t)below(draw64(seed, 61, (uint64_t)b, (uint64_t)i), (uint64_t)(n - i));
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
            swp[i] = j;
            seeds[offsets[b] + i] = perm[i];
        }
        for (int64_t i = s - 1; i >= 0; i--) {
            int64_t j = swp[i];
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
        offsets[b + 1] = offsets[b] + s;
    }
    free(perm);
    free(swp);
    return 0;
}
