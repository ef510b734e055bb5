/*
 * SKIS ORACLE — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the method of
 * Nguyen, Dinh, Thai, "Importance Sketching of Influence Dynamics in
 * Billion-scale Networks" (arXiv 1709.03565):
 *   - Eq. gamma_v (Sec. III-A, component 1): gamma_v = 1 - prod(1 - w(u,v));
 *   - Eq. probu   (Sec. III-A, component 2): Pr[src = v] = gamma_v / Gamma;
 *   - Alg. 1 (IIS sampler): conditioned first step, then reverse BFS;
 *   - Eq. 21 / Eq. compute_inf (Sec. IV, Sec. V): the SKIS estimator
 *     I_R(S) = Cov_R(S)/|R| * Gamma + sum_{v in S} (1 - gamma_v);
 *   - Alg. 3 and Eq. margin (Sec. V-A): greedy max-coverage.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file. It shares no code with the CUDA library: its Philox
 * generator, CSR construction, fixed-point arithmetic, alias table, sampler,
 * coverage and greedy are all written here independently.
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *   R1 Edge probabilities are integer thresholds tau = floor(p * 2^32); an
 *      edge is live iff its 32-bit coin word x < tau. tau = 2^32 - 1 is a
 *      sentinel for "always live" (p >= 1 - 2^-32, including WC with
 *      in-degree 1). The effective probability is p' = tau / 2^32 (or 1).
 *   R2 WC: tau = floor(2^32 / d_in(v)) in integer arithmetic (Sec. VI,
 *      "Weight Settings"); TRI draws p uniformly from {0.1, 0.01, 0.001} per
 *      edge.
 *   R3 gamma_v is evaluated in fixed point: Q starts at 2^62 and is replaced
 *      by floor(Q * (2^32 - tau) / 2^32) for each in-edge in canonical order
 *      (tau = sentinel sets Q = 0); g_v = 2^62 - Q; with s = ceil(log2 n) + 1
 *      and f = 62 - s, w_v = g_v >> s, and gamma~_v = w_v / 2^f,
 *      Gamma~ = W / 2^f where W = sum_v w_v. These are the values every later
 *      step uses, so the source law and the estimator agree exactly.
 *   R4 The source law w_v / W is drawn from an alias table built by the
 *      sweeping construction of Huebschle-Schneider and Sanders ("Parallel
 *      Weighted Random Sampling", ESA 2019) in integer arithmetic: column
 *      capacity W, item mass w_v * n, light items (mass < W) and heavy items
 *      in ascending vertex order.
 *   R5 The conditioned first step (Alg. 1, Eq. probn) is taken in
 *      rejection form: all in-edge coins of the source are redrawn, round
 *      r = 0, 1, ..., until at least one is live. This has the law of the
 *      bucket choice of Eq. probn followed by independent coins on the
 *      in-neighbours after the chosen one (the bucket definition excludes
 *      those before it, although Alg. 1's first-step loop writes "t != i").
 *   R6 Every coin is a Philox4x32-10 word keyed by the sketch seed, with the
 *      counter (edge-quad e>>2, domain, retry, sample id); see coin_word().
 *      The BFS coin of edge e in sample j is fixed, so R_j is the reverse
 *      reachable set of the source in one live-edge world and does not
 *      depend on the order of the queue.
 *   R7 Work counter "coins" = d_in(src) * (retries + 1) + sum of d_in(u) over
 *      the other members: every in-edge of every popped vertex, which does
 *      not depend on the order of the queue.
 *   R8 Self-loops are rejected; parallel edges are independent coins.
 *
 * Variant (graph flag `lt`): the Linear Threshold model (Sec. "Extensions to
 * other diffusion models"). Thresholds as R1/R2, read as edge weights with
 * w' = tau / 2^32 (2^32 for the sentinel); every row must satisfy
 * sum tau' <= 2^32 (the model's sum_u w(u,v) <= 1).
 *   L1 gamma_v = sum of the row's tau' over 2^32, exactly: w_v = sum tau',
 *      f = 32, W = sum w_v; the source law and alias table are as R4.
 *   L2 In a live-edge world of LT each vertex keeps at most one in-edge: the
 *      edge i of its row (canonical order) with P_{i-1} <= y < P_i, where P
 *      is the running sum of tau', or none if y >= P_d, for a uniform y.
 *   L3 An LT IIS sample: source v by Eq. probu with these gamma; the first
 *      step picks exactly one in-neighbour with probability tau'_i / w_v
 *      (z = floor(U w_v / 2^64) for the 64-bit word U of step 0, then the
 *      row position as L2); then the reverse walk of RIS for LT: from the
 *      last member x, word y of step t picks x's in-edge as L2 (t = 1, 2,
 *      ...); the walk stops when none is picked or the picked vertex is
 *      already in R_j. Step t uses the Philox block (q = t, retry 0,
 *      domain LT = 5, sample j).
 *   L4 Work counter coins = the sum of d_in over all members (each member's
 *      row is examined once); retries = 0.
 *   With `ris`, the source is uniform and step 0 is an ordinary walk step.
 *
 * Variant (flag ORC_F_BUCKET): the first step of Alg. 1 in its bucket form
 * (Eq. probn) instead of rejection (R5):
 *   B1 bucket i of the source's row (canonical order) is "in-edges before i
 *      dead, edge i live"; its mass is Q_{i-1} - Q_i in the fixed-point
 *      chain of R3 (Q_0 = 2^62), which is w_i prod_{t<i} (1 - w_t) 2^62 up to
 *      the chain's floors, of total 2^62 - Q_d. z = floor(U (2^62 - Q_d) /
 *      2^64) for the 64-bit word U of the Philox block (q = 0, retry 0,
 *      domain BUCKET = 6, sample j) picks the first i with 2^62 - Q_i > z;
 *      u_i joins R_j and the in-edges after i get their FIRST coins of round
 *      0; retries = 0.
 *
 * Variant (flag `ris`): plain reverse influence sampling (RIS, Borgs et al.;
 * Sec. II-C): the source is uniform (the column draw alone), the source's
 * in-edges get one unconditioned round (FIRST coins, round 0), so a sample
 * may be singular; the estimator is n Cov / T (Lemma 1) and greedy maximises
 * coverage alone.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ERETRY 4

#define ORC_SENT 0xFFFFFFFFu

enum { ORC_W_P = 0, ORC_W_TAU = 1, ORC_W_WC = 2, ORC_W_TRI = 3 };
enum { DOM_SRC = 1, DOM_FIRST = 2, DOM_BFS = 3, DOM_WEIGHT = 4, DOM_LT = 5, DOM_BUCKET = 6 };
enum { ORC_F_RIS = 1, ORC_F_BUCKET = 2 };  /* sampler flags */

/* ------------------------------------------------------------ Philox -- */

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11). Each round multiplies words 0 and 2
 * by the two round multipliers, recombines the halves with words 1 and 3 and
 * the round key, and the key is advanced by the two Weyl constants. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(pb >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)pb;
        uint32_t y2 = (uint32_t)(pa >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)pa;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One Philox block for (key = seed, edge quad q, retry, domain, sample j):
 *   counter word 0 = q mod 2^32
 *   counter word 1 = (q >> 32) & 0xF | (retry & 0xFFFFFF) << 4 | domain << 28
 *   counter words 2, 3 = j mod 2^32, j >> 32. */
static void philox_block(uint64_t seed, uint64_t q, uint32_t retry, int domain, uint64_t j,
                         uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = (uint32_t)q;
    ctr[1] = (uint32_t)((q >> 32) & 0xFu) | ((retry & 0xFFFFFFu) << 4) | ((uint32_t)domain << 28);
    ctr[2] = (uint32_t)j;
    ctr[3] = (uint32_t)(j >> 32);
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, out);
}

/* The 32-bit coin word of edge e: word (e mod 4) of the block of quad e/4. */
static uint32_t coin_word(uint64_t seed, int domain, uint32_t retry, uint64_t j, uint64_t e)
{
    uint32_t out[4];
    philox_block(seed, e >> 2, retry, domain, j, out);
    return out[e & 3];
}

/* R1: an edge is live iff its coin word is below its threshold. */
static int is_live(uint32_t x, uint32_t tau)
{
    return tau == ORC_SENT || x < tau;
}

/* R1: tau = floor(p * 2^32), clamped to the sentinel. p * 2^32 is exact. */
static uint32_t tau_of_p(double p)
{
    if (p >= 1.0) return ORC_SENT;
    double t = p * 4294967296.0;
    uint64_t ti = (uint64_t)t; /* truncation = floor for t >= 0 */
    return ti >= ORC_SENT ? ORC_SENT : (uint32_t)ti;
}

/* ------------------------------------------------------------- graph -- */

typedef struct orc_graph {
    int64_t n, m;
    int lt;          /* Linear Threshold model (L1-L4) instead of IC */
    int64_t *off;    /* n+1 row offsets of the in-CSR (rows = destinations) */
    int32_t *src;    /* m sources in CSR order */
    uint32_t *tau;   /* m thresholds in CSR order */
    int64_t *perm;   /* m: CSR position -> input edge index */
    uint64_t *w;     /* n fixed-point gamma numerators (R3) */
    uint64_t W;      /* sum of w */
    int32_t f, s;    /* gamma~ = w / 2^f; s = 62 - f */
    uint64_t *prob;  /* n alias thresholds in [0, W] */
    uint32_t *alias; /* n alias targets */
} orc_graph;

static int ceil_log2(int64_t n)
{
    int c = 0;
    while (((int64_t)1 << c) < n) c++;
    return c;
}

void orc_graph_free(orc_graph *g)
{
    if (!g) return;
    free(g->off); free(g->src); free(g->tau); free(g->perm);
    free(g->w); free(g->prob); free(g->alias);
    free(g);
}

/* R4: the sweeping alias construction, sequentially. The current heavy item
 * h has residual mass r; while r < W the heavy item's own column is closed
 * with prob r and alias the next heavy item, which pays the deficit W - r;
 * otherwise the next light item l gets prob mass_l and alias h, and h pays
 * W - mass_l. When the light items run out, every remaining heavy item holds
 * exactly W and aliases itself. Returns -1 if the integer balance fails
 * (it cannot when sum(mass) = n * W). */
static int alias_sweep(orc_graph *g)
{
    int64_t n = g->n;
    uint64_t W = g->W;
    uint64_t *mass = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int64_t *light = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *heavy = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!mass || !light || !heavy) { free(mass); free(light); free(heavy); return -2; }
    int64_t nl = 0, nh = 0;
    for (int64_t v = 0; v < n; v++) {
        mass[v] = g->w[v] * (uint64_t)n;
        if (mass[v] < W) light[nl++] = v; else heavy[nh++] = v;
    }
    int rc = 0;
    if (W == 0) {
        for (int64_t v = 0; v < n; v++) { g->prob[v] = 0; g->alias[v] = (uint32_t)v; }
        goto done;
    }
    int64_t li = 0, hi = 0;
    uint64_t r = mass[heavy[0]];
    for (;;) {
        if (r < W) {
            if (hi + 1 >= nh) { rc = -1; goto done; }
            g->prob[heavy[hi]] = r;
            g->alias[heavy[hi]] = (uint32_t)heavy[hi + 1];
            r = mass[heavy[hi + 1]] - (W - r);
            hi++;
        } else if (li < nl) {
            int64_t l = light[li++];
            g->prob[l] = mass[l];
            g->alias[l] = (uint32_t)heavy[hi];
            r -= W - mass[l];
        } else {
            break;
        }
    }
    if (r != W) { rc = -1; goto done; }
    for (int64_t t = hi; t < nh; t++) {
        if (t > hi && mass[heavy[t]] != W) { rc = -1; goto done; }
        g->prob[heavy[t]] = W;
        g->alias[heavy[t]] = (uint32_t)heavy[t];
    }
done:
    free(mass); free(light); free(heavy);
    return rc;
}

/* Build the probabilistic graph G = (V, E, w) of Sec. II-A: the canonical
 * in-CSR (rows by destination, each row by (source, input index)), the
 * thresholds (R1, R2), gamma in fixed point (R3, Eq. gamma_v) and the alias
 * table of the source law (R4, Eq. probu).
 *   weights: double p[m] (ORC_W_P), uint32 tau[m] (ORC_W_TAU), or NULL. */
int orc_graph_build_model(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                          const void *weights, int model, uint64_t weight_seed, int lt, orc_graph **out)
{
    *out = NULL;
    if (n < 1 || n > ((int64_t)1 << 31) || m < 0) return ORC_EINVAL;
    if ((model == ORC_W_P || model == ORC_W_TAU) && m > 0 && !weights) return ORC_EINVAL;
    if (model < ORC_W_P || model > ORC_W_TRI) return ORC_EINVAL;
    for (int64_t e = 0; e < m; e++) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return ORC_EINVAL;
        if (src[e] == dst[e]) return ORC_EINVAL; /* R8 */
        if (model == ORC_W_P) {
            double p = ((const double *)weights)[e];
            if (!(p >= 0.0 && p <= 1.0)) return ORC_EINVAL; /* also rejects NaN */
        }
    }
    orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
    if (!g) return ORC_ENOMEM;
    g->n = n; g->m = m; g->lt = lt ? 1 : 0;
    size_t mm = (size_t)(m > 0 ? m : 1);
    g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->src = (int32_t *)malloc(mm * sizeof(int32_t));
    g->tau = (uint32_t *)malloc(mm * sizeof(uint32_t));
    g->perm = (int64_t *)malloc(mm * sizeof(int64_t));
    g->w = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    g->prob = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    g->alias = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t *key = (uint64_t *)malloc(mm * sizeof(uint64_t));
    uint64_t *key2 = (uint64_t *)malloc(mm * sizeof(uint64_t));
    int64_t *idx = (int64_t *)malloc(mm * sizeof(int64_t));
    int64_t *idx2 = (int64_t *)malloc(mm * sizeof(int64_t));
    if (!g->off || !g->src || !g->tau || !g->perm || !g->w || !g->prob || !g->alias || !key || !key2 || !idx ||
        !idx2) {
        free(key); free(key2); free(idx); free(idx2); orc_graph_free(g); return ORC_ENOMEM;
    }

    /* canonical in-CSR: rows by destination, each row by (source, input
     * index). The key dst * n + src of every input edge is sorted with a
     * stable least-significant-digit radix sort (11-bit digits) that carries
     * the input index; stability keeps equal keys in input order. */
    for (int64_t e = 0; e < m; e++) { key[e] = (uint64_t)dst[e] * (uint64_t)n + (uint64_t)src[e]; idx[e] = e; }
    int key_bits = 0;
    while (key_bits < 64 && ((uint64_t)n * (uint64_t)n - 1) >> key_bits) key_bits++;
    for (int shift = 0; shift < key_bits; shift += 11) {
        int64_t count[2049];
        memset(count, 0, sizeof(count));
        for (int64_t e = 0; e < m; e++) count[((key[e] >> shift) & 2047) + 1]++;
        for (int d = 0; d < 2048; d++) count[d + 1] += count[d];
        for (int64_t e = 0; e < m; e++) {
            int64_t pos = count[(key[e] >> shift) & 2047]++;
            key2[pos] = key[e];
            idx2[pos] = idx[e];
        }
        uint64_t *tk = key; key = key2; key2 = tk;
        int64_t *ti = idx; idx = idx2; idx2 = ti;
    }
    for (int64_t e = 0; e < m; e++) {
        g->src[e] = (int32_t)(key[e] % (uint64_t)n);
        g->perm[e] = idx[e];
        g->off[key[e] / (uint64_t)n + 1]++;
    }
    for (int64_t v = 0; v < n; v++) g->off[v + 1] += g->off[v];
    free(key); free(key2); free(idx); free(idx2);

    /* thresholds (R1, R2) */
    static const double tri_levels[3] = {0.1, 0.01, 0.001};
    for (int64_t v = 0; v < n; v++) {
        int64_t d = g->off[v + 1] - g->off[v];
        for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) {
            uint32_t t;
            if (model == ORC_W_P) t = tau_of_p(((const double *)weights)[g->perm[e]]);
            else if (model == ORC_W_TAU) t = ((const uint32_t *)weights)[g->perm[e]];
            else if (model == ORC_W_WC) t = (d == 1) ? ORC_SENT : (uint32_t)(((uint64_t)1 << 32) / (uint64_t)d);
            else {
                uint32_t x = coin_word(weight_seed, DOM_WEIGHT, 0, 0, (uint64_t)e);
                t = tau_of_p(tri_levels[((uint64_t)x * 3u) >> 32]);
            }
            g->tau[e] = t;
        }
    }

    if (g->lt) {
        /* L1: gamma_v = sum of the row's weights, exactly; rows above 1 are
         * not an LT instance */
        g->s = 0;
        g->f = 32;
        g->W = 0;
        for (int64_t v = 0; v < n; v++) {
            uint64_t S = 0;
            for (int64_t e = g->off[v]; e < g->off[v + 1]; e++)
                S += g->tau[e] == ORC_SENT ? ((uint64_t)1 << 32) : (uint64_t)g->tau[e];
            if (S > ((uint64_t)1 << 32)) { orc_graph_free(g); return ORC_EINVAL; }
            g->w[v] = S;
            g->W += S;
        }
        int rc_lt = alias_sweep(g);
        if (rc_lt != 0) { orc_graph_free(g); return rc_lt == -2 ? ORC_ENOMEM : ORC_EINVAL; }
        *out = g;
        return ORC_OK;
    }

    /* gamma in fixed point (R3, Eq. gamma_v) */
    g->s = ceil_log2(n) + 1;
    g->f = 62 - g->s;
    g->W = 0;
    const uint64_t one62 = (uint64_t)1 << 62;
    for (int64_t v = 0; v < n; v++) {
        uint64_t Q = one62;
        for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) {
            if (g->tau[e] == ORC_SENT) Q = 0;
            else Q = (uint64_t)(((u128)Q * (u128)(((uint64_t)1 << 32) - g->tau[e])) >> 32);
        }
        g->w[v] = (one62 - Q) >> g->s;
        g->W += g->w[v];
    }

    int rc = alias_sweep(g);
    if (rc != 0) { orc_graph_free(g); return rc == -2 ? ORC_ENOMEM : ORC_EINVAL; }
    *out = g;
    return ORC_OK;
}

int orc_graph_build(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                    const void *weights, int model, uint64_t weight_seed, orc_graph **out)
{
    return orc_graph_build_model(n, m, src, dst, weights, model, weight_seed, 0, out);
}

void orc_graph_scalars(const orc_graph *g, int64_t *n, int64_t *m, uint64_t *W, int32_t *f)
{
    *n = g->n; *m = g->m; *W = g->W; *f = g->f;
}

/* Copy the graph's arrays out (any pointer may be NULL). */
void orc_graph_arrays(const orc_graph *g, int64_t *off, int32_t *src, uint32_t *tau, int64_t *perm,
                      uint64_t *w, uint64_t *prob, uint32_t *alias)
{
    if (off) memcpy(off, g->off, (size_t)(g->n + 1) * sizeof(int64_t));
    if (src) memcpy(src, g->src, (size_t)g->m * sizeof(int32_t));
    if (tau) memcpy(tau, g->tau, (size_t)g->m * sizeof(uint32_t));
    if (perm) memcpy(perm, g->perm, (size_t)g->m * sizeof(int64_t));
    if (w) memcpy(w, g->w, (size_t)g->n * sizeof(uint64_t));
    if (prob) memcpy(prob, g->prob, (size_t)g->n * sizeof(uint64_t));
    if (alias) memcpy(alias, g->alias, (size_t)g->n * sizeof(uint32_t));
}

/* ----------------------------------------------------------- sampler -- */

/* Eq. probu with R4: column col = floor(U1 * n), y = floor(U2 * W) from the
 * SRC-domain Philox block of sample j; the source is col if y < prob[col],
 * else alias[col]. */
static int64_t draw_source(const orc_graph *g, uint64_t seed, uint64_t j)
{
    uint32_t x[4];
    philox_block(seed, 0, 0, DOM_SRC, j, x);
    uint64_t u1 = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
    uint64_t u2 = (uint64_t)x[2] | ((uint64_t)x[3] << 32);
    int64_t col = (int64_t)(((u128)u1 * (u128)(uint64_t)g->n) >> 64);
    uint64_t y = (uint64_t)(((u128)u2 * (u128)g->W) >> 64);
    return y < g->prob[col] ? col : (int64_t)g->alias[col];
}

/* One IIS sample R_j (Alg. 1). visited must be all-zero on entry and is
 * restored before returning; members receives R_j in insertion order (the
 * source first); it must hold n entries. Returns ORC_OK or ORC_ERETRY. */
/* RIS source: uniform over V, the column draw of the SRC block alone. */
static int64_t draw_source_uniform(const orc_graph *g, uint64_t seed, uint64_t j)
{
    uint32_t x[4];
    philox_block(seed, 0, 0, DOM_SRC, j, x);
    uint64_t u1 = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
    return (int64_t)(((u128)u1 * (u128)(uint64_t)g->n) >> 64);
}

/* B1: the bucket (in-edge position in [b, e_end)) of the source's row. */
static int64_t bucket_pick(const orc_graph *g, uint64_t seed, uint64_t j, int64_t b, int64_t e_end)
{
    const uint64_t one62 = (uint64_t)1 << 62;
    uint64_t Q = one62;
    for (int64_t e = b; e < e_end; e++) {
        if (g->tau[e] == ORC_SENT) Q = 0;
        else Q = (uint64_t)(((u128)Q * (u128)(((uint64_t)1 << 32) - g->tau[e])) >> 32);
    }
    uint64_t G = one62 - Q;
    uint32_t x[4];
    philox_block(seed, 0, 0, DOM_BUCKET, j, x);
    uint64_t U = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
    uint64_t z = (uint64_t)(((u128)U * (u128)G) >> 64);
    Q = one62;
    for (int64_t e = b; e < e_end; e++) {
        if (g->tau[e] == ORC_SENT) Q = 0;
        else Q = (uint64_t)(((u128)Q * (u128)(((uint64_t)1 << 32) - g->tau[e])) >> 32);
        if (one62 - Q > z) return e;
    }
    return e_end - 1; /* not reached: z < G = 2^62 - Q_d */
}

static int sample_one(const orc_graph *g, uint64_t seed, uint64_t j, uint32_t retry_cap, int flags,
                      char *visited, int32_t *members, int64_t *len_out, int32_t *src_out,
                      uint32_t *retries_out, uint64_t *coins_out)
{
    const int ris = flags & ORC_F_RIS;
    const int bucket = (flags & ORC_F_BUCKET) && !ris;
    /* the source, Eq. probu (RIS: uniform) */
    int64_t v = ris ? draw_source_uniform(g, seed, j) : draw_source(g, seed, j);
    int64_t b = g->off[v], e_end = g->off[v + 1];
    *src_out = (int32_t)v;

    /* the conditioned first step in rejection form (R5): round r flips every in-edge of v
     * (RIS: round 0 only, accepted whatever its coins) */
    uint32_t r = 0;
    int64_t picked = -1; /* B1: the bucket's live in-edge */
    if (bucket) picked = bucket_pick(g, seed, j, b, e_end);
    for (;; r++) {
        if (ris || bucket) break;
        if (r >= retry_cap) {
            *retries_out = r;
            *len_out = 0;
            *coins_out = (uint64_t)(e_end - b) * r;
            return ORC_ERETRY;
        }
        int any = 0;
        for (int64_t e = b; e < e_end; e++)
            if (is_live(coin_word(seed, DOM_FIRST, r, j, (uint64_t)e), g->tau[e])) { any = 1; break; }
        if (any) break;
    }
    *retries_out = r;

    /* R_j = {v} plus the live in-neighbours of the accepted round;
     * the queue Q is members[head .. len) */
    int64_t len = 0;
    visited[v] = 1;
    members[len++] = (int32_t)v;
    for (int64_t e = (bucket ? picked : b); e < e_end; e++) {
        if (e != picked && !is_live(coin_word(seed, DOM_FIRST, r, j, (uint64_t)e), g->tau[e])) continue;
        int32_t u = g->src[e];
        if (!visited[u]) { visited[u] = 1; members[len++] = u; }
    }

    /* reverse BFS, FIFO, one coin per in-edge from outside R_j */
    uint64_t coins = (uint64_t)(e_end - b) * (r + 1);
    for (int64_t head = 1; head < len; head++) {
        int32_t w = members[head];
        coins += (uint64_t)(g->off[w + 1] - g->off[w]);
        for (int64_t e = g->off[w]; e < g->off[w + 1]; e++) {
            int32_t u = g->src[e];
            if (visited[u]) continue;
            if (is_live(coin_word(seed, DOM_BFS, 0, j, (uint64_t)e), g->tau[e])) {
                visited[u] = 1;
                members[len++] = u;
            }
        }
    }
    for (int64_t i = 0; i < len; i++) visited[members[i]] = 0;
    *len_out = len;
    *coins_out = coins;
    return ORC_OK;
}

/* L2: the in-edge of row [b, e_end) that a draw y in [0, sum tau') picks:
 * the first position whose running sum of tau' exceeds y. */
static int64_t lt_pick(const orc_graph *g, int64_t b, int64_t e_end, uint64_t y)
{
    uint64_t P = 0;
    for (int64_t e = b; e < e_end; e++) {
        P += g->tau[e] == ORC_SENT ? ((uint64_t)1 << 32) : (uint64_t)g->tau[e];
        if (P > y) return e;
    }
    return -1;
}

/* One LT IIS sample (L3): the source, its one conditioned in-neighbour, then
 * the reverse walk until no in-edge is picked or the walk meets R_j again.
 * With ris: uniform source, and step 0 is an ordinary walk step. */
static int sample_one_lt(const orc_graph *g, uint64_t seed, uint64_t j, int ris, char *visited,
                         int32_t *members, int64_t *len_out, int32_t *src_out, uint32_t *retries_out,
                         uint64_t *coins_out)
{
    int64_t v = ris ? draw_source_uniform(g, seed, j) : draw_source(g, seed, j);
    *src_out = (int32_t)v;
    *retries_out = 0;
    int64_t len = 0;
    visited[v] = 1;
    members[len++] = (int32_t)v;
    uint64_t coins = 0;
    int64_t x = v;
    for (uint64_t t = 0;; t++) {
        int64_t b = g->off[x], e_end = g->off[x + 1];
        coins += (uint64_t)(e_end - b);
        if (e_end == b) break;
        uint32_t blk[4];
        philox_block(seed, t, 0, DOM_LT, j, blk);
        uint64_t S = g->w[x];
        uint64_t y;
        if (t == 0 && !ris) {  /* Pr[u] = w(u, v) / gamma_v */
            uint64_t U = (uint64_t)blk[0] | ((uint64_t)blk[1] << 32);
            y = (uint64_t)(((u128)U * (u128)S) >> 64);
        } else {
            y = blk[0];
            if (y >= S) break;  /* no in-edge kept: the walk ends */
        }
        int64_t e = lt_pick(g, b, e_end, y);
        int32_t u = g->src[e];
        if (visited[u]) break;  /* the walk closes on R_j */
        visited[u] = 1;
        members[len++] = u;
        x = u;
    }
    for (int64_t i = 0; i < len; i++) visited[members[i]] = 0;
    *len_out = len;
    *coins_out = coins;
    return ORC_OK;
}

/* Samples for an explicit list of sample ids. Per sample: src, retries, len,
 * coins, status; members are concatenated (insertion order) into members_out,
 * whose capacity is members_cap; *members_used receives the total. Returns
 * ORC_OK, or ORC_ENOMEM if members_cap is too small (outputs then partial). */
int orc_sample_ids(const orc_graph *g, uint64_t seed, const uint64_t *ids, int64_t count,
                   uint32_t retry_cap, int flags, int32_t *src_out, uint32_t *retries_out,
                   int64_t *len_out, uint64_t *coins_out, int32_t *status_out, int32_t *members_out,
                   int64_t members_cap, int64_t *members_used)
{
    const int ris = flags & ORC_F_RIS;
    if (g->W == 0 && !ris) return ORC_EINVAL;
    char *visited = (char *)calloc((size_t)g->n, 1);
    int32_t *buf = (int32_t *)malloc((size_t)g->n * sizeof(int32_t));
    if (!visited || !buf) { free(visited); free(buf); return ORC_ENOMEM; }
    int64_t used = 0;
    int rc = ORC_OK;
    for (int64_t t = 0; t < count; t++) {
        int64_t len;
        if (g->lt)
            status_out[t] = sample_one_lt(g, seed, ids[t], ris, visited, buf, &len, &src_out[t],
                                          &retries_out[t], &coins_out[t]);
        else
            status_out[t] = sample_one(g, seed, ids[t], retry_cap, flags, visited, buf, &len, &src_out[t],
                                       &retries_out[t], &coins_out[t]);
        len_out[t] = len;
        if (used + len > members_cap) { rc = ORC_ENOMEM; break; }
        memcpy(members_out + used, buf, (size_t)len * sizeof(int32_t));
        used += len;
    }
    *members_used = used;
    free(visited); free(buf);
    return rc;
}

/* ------------------------------------------------------------ sketch -- */

/* The SKIS sketch R = {R_1, ..., R_T} of Alg. 2 (preprocessing): samples
 * with ids 0 .. T-1. */
typedef struct orc_sketch {
    const orc_graph *g;
    int ris;          /* plain RIS samples (n Cov / T estimator) */
    int64_t T;
    int64_t *off;     /* T+1 */
    int32_t *mem;     /* members, sample after sample */
    int32_t *src;
    uint32_t *retries;
    uint64_t *coins;
} orc_sketch;

void orc_sketch_free(orc_sketch *s)
{
    if (!s) return;
    free(s->off); free(s->mem); free(s->src); free(s->retries); free(s->coins);
    free(s);
}

/* Samples j = 0, 1, ... up to T; with stop_entries > 0, the sketch ends at
 * the first sample that brings the total size sum_j |R_j| to stop_entries
 * or more (the stop-at-size rule of the experiments, Sec. VI "Algorithms
 * compared": sample until the total size reaches a target), T bounding it. */
static int sketch_build(const orc_graph *g, uint64_t seed, int64_t T, int64_t stop_entries,
                        uint32_t retry_cap, int flags, orc_sketch **out)
{
    const int ris = flags & ORC_F_RIS;
    *out = NULL;
    if (T < 1 || (g->W == 0 && !ris)) return ORC_EINVAL;
    orc_sketch *s = (orc_sketch *)calloc(1, sizeof(orc_sketch));
    if (!s) return ORC_ENOMEM;
    s->g = g; s->T = T; s->ris = ris;
    s->off = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    s->src = (int32_t *)malloc((size_t)T * sizeof(int32_t));
    s->retries = (uint32_t *)malloc((size_t)T * sizeof(uint32_t));
    s->coins = (uint64_t *)malloc((size_t)T * sizeof(uint64_t));
    int64_t cap = T * 4 + 1024;
    s->mem = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    char *visited = (char *)calloc((size_t)g->n, 1);
    int32_t *buf = (int32_t *)malloc((size_t)g->n * sizeof(int32_t));
    if (!s->off || !s->src || !s->retries || !s->coins || !s->mem || !visited || !buf) {
        free(visited); free(buf); orc_sketch_free(s); return ORC_ENOMEM;
    }
    s->off[0] = 0;
    for (int64_t j = 0; j < T; j++) {
        int64_t len;
        int rc = g->lt ? sample_one_lt(g, seed, (uint64_t)j, ris, visited, buf, &len, &s->src[j],
                                       &s->retries[j], &s->coins[j])
                       : sample_one(g, seed, (uint64_t)j, retry_cap, flags, visited, buf, &len, &s->src[j],
                                    &s->retries[j], &s->coins[j]);
        if (rc != ORC_OK) { free(visited); free(buf); orc_sketch_free(s); return rc; }
        if (s->off[j] + len > cap) {
            while (s->off[j] + len > cap) cap *= 2;
            int32_t *nm = (int32_t *)realloc(s->mem, (size_t)cap * sizeof(int32_t));
            if (!nm) { free(visited); free(buf); orc_sketch_free(s); return ORC_ENOMEM; }
            s->mem = nm;
        }
        memcpy(s->mem + s->off[j], buf, (size_t)len * sizeof(int32_t));
        s->off[j + 1] = s->off[j] + len;
        if (stop_entries > 0 && s->off[j + 1] >= stop_entries) {
            s->T = j + 1;
            break;
        }
    }
    free(visited); free(buf);
    *out = s;
    return ORC_OK;
}

int orc_sketch_build(const orc_graph *g, uint64_t seed, int64_t T, uint32_t retry_cap, int flags,
                     orc_sketch **out)
{
    return sketch_build(g, seed, T, 0, retry_cap, flags, out);
}

/* Stop-at-size sketch: samples until sum_j |R_j| >= target_entries (at most
 * T_max samples); the sample count is orc_sketch_count. */
int orc_sketch_build_to_size(const orc_graph *g, uint64_t seed, int64_t target_entries, int64_t T_max,
                             uint32_t retry_cap, int flags, orc_sketch **out)
{
    if (target_entries < 1) return ORC_EINVAL;
    return sketch_build(g, seed, T_max, target_entries, retry_cap, flags, out);
}

int64_t orc_sketch_count(const orc_sketch *s) { return s->T; }

int64_t orc_sketch_entries(const orc_sketch *s) { return s->off[s->T]; }

void orc_sketch_arrays(const orc_sketch *s, int64_t *off, int32_t *mem, int32_t *src,
                       uint32_t *retries, uint64_t *coins)
{
    if (off) memcpy(off, s->off, (size_t)(s->T + 1) * sizeof(int64_t));
    if (mem) memcpy(mem, s->mem, (size_t)s->off[s->T] * sizeof(int32_t));
    if (src) memcpy(src, s->src, (size_t)s->T * sizeof(int32_t));
    if (retries) memcpy(retries, s->retries, (size_t)s->T * sizeof(uint32_t));
    if (coins) memcpy(coins, s->coins, (size_t)s->T * sizeof(uint64_t));
}

/* Exact estimator numerator and denominator of Eq. 21 in units of 2^-f:
 *   N = Cov * W + T * sum_{v in S} (2^f - w_v),   D = T * 2^f,
 * so that I_R(S) = N / D = Cov/T * Gamma~ + sum (1 - gamma~_v). */
static void estimate_nd(const orc_sketch *s, int64_t cov, u128 sum_c, u128 *N, u128 *D)
{
    if (s->ris) {  /* Lemma 1: I(S) = n Pr[R meets S] */
        *N = (u128)(uint64_t)cov * (u128)(uint64_t)s->g->n;
        *D = (u128)(uint64_t)s->T;
        return;
    }
    *N = (u128)(uint64_t)cov * (u128)s->g->W + (u128)(uint64_t)s->T * sum_c;
    *D = (u128)(uint64_t)s->T << s->g->f;
}

/* Influence queries (Alg. 2's estimate step): for each seed set S_b (CSR seed_off /
 * seeds), Cov_R(S_b) = #{j : R_j meets S_b} and I_R(S_b) by Eq. 21.
 * num/den receive N and D as (low, high) 64-bit halves (may be NULL).
 * Empty, out-of-range or repeated seeds give ORC_EINVAL. */
int orc_coverage(const orc_sketch *s, int32_t q, const int64_t *seed_off, const int32_t *seeds,
                 int64_t *cov_out, double *est_out, uint64_t *num_out, uint64_t *den_out)
{
    const orc_graph *g = s->g;
    char *inS = (char *)calloc((size_t)g->n, 1);
    if (!inS) return ORC_ENOMEM;
    int rc = ORC_OK;
    for (int32_t b = 0; b < q && rc == ORC_OK; b++) {
        int64_t lo = seed_off[b], hi = seed_off[b + 1];
        if (hi <= lo) { rc = ORC_EINVAL; break; }
        u128 sum_c = 0;
        int64_t i;
        for (i = lo; i < hi; i++) {
            int32_t v = seeds[i];
            if (v < 0 || v >= g->n || inS[v]) { rc = ORC_EINVAL; break; }
            inS[v] = 1;
            sum_c += (((uint64_t)1 << g->f) - g->w[v]);
        }
        if (rc == ORC_OK) {
            int64_t cov = 0;
            for (int64_t j = 0; j < s->T; j++) {
                for (int64_t k = s->off[j]; k < s->off[j + 1]; k++)
                    if (inS[s->mem[k]]) { cov++; break; }
            }
            u128 N, D;
            estimate_nd(s, cov, sum_c, &N, &D);
            cov_out[b] = cov;
            est_out[b] = (double)N / (double)D;
            if (num_out) { num_out[2 * b] = (uint64_t)N; num_out[2 * b + 1] = (uint64_t)(N >> 64); }
            if (den_out) { den_out[2 * b] = (uint64_t)D; den_out[2 * b + 1] = (uint64_t)(D >> 64); }
        }
        for (int64_t t = lo; t < i && t < hi; t++) inS[seeds[t]] = 0;
    }
    free(inS);
    return rc;
}

/* Alg. 3: k rounds; each picks v outside S maximising Eq. margin,
 * Delta_R(v, S)/|R| * Gamma + (1 - gamma_v), compared exactly as the integer
 * key Delta * W + T * (2^f - w_v) (Eq. margin times T * 2^f); ties go to the
 * lowest vertex id. Outputs the seeds, the cumulative Cov_R and I_R. */
int orc_greedy(const orc_sketch *s, int32_t k, int32_t *seeds_out, int64_t *cov_out,
               double *est_out)
{
    const orc_graph *g = s->g;
    int64_t n = g->n, T = s->T;
    if (k < 0 || k > n) return ORC_EINVAL;
    int64_t *delta = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *ioff = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t E = s->off[T];
    int64_t *inv = (int64_t *)malloc((size_t)(E > 0 ? E : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    char *covered = (char *)calloc((size_t)T, 1);
    char *inS = (char *)calloc((size_t)n, 1);
    if (!delta || !ioff || !inv || !fill || !covered || !inS) {
        free(delta); free(ioff); free(inv); free(fill); free(covered); free(inS);
        return ORC_ENOMEM;
    }
    /* Delta_R(v, {}) = number of samples containing v; inverted lists */
    for (int64_t x = 0; x < E; x++) delta[s->mem[x]]++;
    for (int64_t v = 0; v < n; v++) ioff[v + 1] = ioff[v] + delta[v];
    for (int64_t j = 0; j < T; j++)
        for (int64_t x = s->off[j]; x < s->off[j + 1]; x++) {
            int32_t v = s->mem[x];
            inv[ioff[v] + fill[v]++] = j;
        }
    int64_t cov = 0;
    u128 sum_c = 0;
    const uint64_t one_f = (uint64_t)1 << g->f;
    for (int32_t i = 0; i < k; i++) {
        int64_t best = -1;
        u128 best_key = 0;
        for (int64_t v = 0; v < n; v++) {
            if (inS[v]) continue;
            u128 key = s->ris ? (u128)(uint64_t)delta[v]
                              : (u128)(uint64_t)delta[v] * (u128)g->W + (u128)(uint64_t)T * (u128)(one_f - g->w[v]);
            if (best < 0 || key > best_key) { best = v; best_key = key; }
        }
        inS[best] = 1;
        cov += delta[best];
        sum_c += one_f - g->w[best];
        for (int64_t x = ioff[best]; x < ioff[best + 1]; x++) {
            int64_t j = inv[x];
            if (covered[j]) continue;
            covered[j] = 1;
            for (int64_t y = s->off[j]; y < s->off[j + 1]; y++) delta[s->mem[y]]--;
        }
        u128 N, D;
        estimate_nd(s, cov, sum_c, &N, &D);
        seeds_out[i] = (int32_t)best;
        cov_out[i] = cov;
        est_out[i] = (double)N / (double)D;
    }
    free(delta); free(ioff); free(inv); free(fill); free(covered); free(inS);
    return ORC_OK;
}
