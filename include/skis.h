/*
 * skis.h — C ABI of the SKIS GB300 library.
 *
 * The library implements the data-parallel hot path of the SKIS method of
 * Nguyen, Dinh, Thai, "Importance Sketching of Influence Dynamics in
 * Billion-scale Networks" (arXiv 1709.03565) on one NVIDIA GB300 (sm_103a):
 * importance sampling of non-singular reverse-reachable sets under the
 * Independent Cascade model (Sec. III, Alg. 1), the SKIS influence estimator
 * (Sec. IV, Eq. 21, Alg. 2) and greedy max-coverage (Sec. V, Alg. 3).
 *
 * Conventions for every entry point:
 *   - Return value: a skis_status code. No exceptions cross the ABI and the
 *     library never aborts. skis_last_error() gives a message for the last
 *     failing call of the calling thread.
 *   - Ownership: the library allocates and owns all device memory behind its
 *     handles (stream-ordered, on the stream of the call). Input arrays
 *     belong to the caller and are copied; output buffers are allocated by
 *     the caller. A graph must outlive every sketch made from it.
 *   - Streams: cuda_stream is a cudaStream_t (NULL = legacy default stream).
 *     Calls on one handle must be ordered: issue them on one stream, or
 *     synchronise between streams. Entry points that return values to the
 *     host (statuses, counts, host outputs) synchronise that stream.
 *     skis_graph_free / skis_sketch_free release memory on the stream of the
 *     handle's last call, which must still exist.
 *   - Member layout: the first sketch scan of skis_estimate after new
 *     samples (sketches of 2^20 samples or more) moves their members into
 *     sample-id order in the sketch's storage. Only the layout changes, never a sample; do not overlap such a
 *     call with other work on the same sketch (a server included).
 *   - Memory spaces: where a call takes SKIS_MEM_HOST or SKIS_MEM_DEVICE,
 *     the pointers it names are host or device pointers accordingly.
 *   - Determinism: sample j of a sketch is a pure function of (graph, seed,
 *     j). The same graph in any input edge order, the same seed and the same
 *     ids give identical samples, coverage counts and greedy seed sets,
 *     whatever the launch configuration.
 *   - Exactness: thresholds, gamma, the source law, coverage counts and the
 *     greedy keys are integers; only the final estimate is a binary64
 *     quotient of two exact integers.
 */
#ifndef SKIS_H
#define SKIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct skis_graph skis_graph;
typedef struct skis_sketch skis_sketch;

typedef enum skis_status {
    SKIS_OK = 0,
    SKIS_EINVAL = 1,           /* bad argument or bad input data */
    SKIS_ENOMEM = 2,           /* device or host allocation failed */
    SKIS_ERR_CUDA = 3,         /* a CUDA call failed (message has the CUDA error) */
    SKIS_ERR_RETRY_LIMIT = 4,  /* a conditioned first step hit the retry cap */
    SKIS_ERR_ARENA_FULL = 5,   /* the sketch arena could not be grown */
    SKIS_ERR_INTERNAL = 6,     /* a library invariant failed on the device (a bug: the message says which) */
    SKIS_ERR_EXCHANGE = 7      /* the caller's all-reduce callback reported a failure */
} skis_status;

/* Edge-probability models (Sec. II-A; Sec. VI "Weight Settings"). Every
 * probability becomes an integer threshold tau = floor(p * 2^32); an edge is
 * live iff its 32-bit Philox coin word x satisfies x < tau.
 * tau = 0xFFFFFFFF is the sentinel "always live" (p >= 1 - 2^-32). */
typedef enum skis_weight_model {
    SKIS_W_EXPLICIT_P = 0,   /* weights = double p[m], each in [0, 1], no NaN */
    SKIS_W_EXPLICIT_TAU = 1, /* weights = uint32 tau[m] */
    SKIS_W_WC = 2,           /* weighted cascade: p = 1 / d_in(v), as
                                tau = floor(2^32 / d_in(v)), sentinel if d_in = 1;
                                weights = NULL */
    SKIS_W_TRI = 3           /* trivalency: p uniform over {0.1, 0.01, 0.001},
                                drawn per canonical edge position from Philox
                                keyed by weight_seed; weights = NULL */
} skis_weight_model;

typedef enum skis_mem_space { SKIS_MEM_HOST = 0, SKIS_MEM_DEVICE = 1 } skis_mem_space;

/* Diffusion model of a loaded graph. */
typedef enum skis_diffusion { SKIS_DIFF_IC = 0, SKIS_DIFF_LT = 1 } skis_diffusion;

typedef struct skis_graph_info {
    int64_t n, m;
    uint64_t W;        /* Gamma in fixed point: Gamma~ = W / 2^f */
    int32_t f;         /* fractional bits: gamma~_v = w_v / 2^f, f = 61 - ceil(log2 n) (IC), 32 (LT) */
    int32_t row_uniform_tau; /* 1 when every in-row has one threshold (WC) */
    double Gamma;      /* W / 2^f as binary64 (informational) */
    int32_t diffusion; /* skis_diffusion */
    int32_t reserved;
} skis_graph_info;

typedef struct skis_stats {
    uint64_t T;              /* samples in the sketch (ids first_id .. first_id + T - 1) */
    uint64_t entries;        /* sum of |R_j| */
    uint64_t coins;          /* sum over samples of in-edges examined (see skis_sample) */
    uint64_t retries;        /* sum of rejected first-step rounds */
    uint64_t arena_capacity; /* entries the arena can hold before it grows */
    uint64_t arena_reserved; /* entries reserved so far (>= entries) */
    uint64_t to_warp;        /* samples of the last skis_sample call handed to the warp tier */
    uint64_t deferred;       /* samples of the last skis_sample call that ran on the CTA tier */
    double last_thread_ms;   /* device time of the last first-tier sampling launch(es) */
    double last_warp_ms;     /* device time of the last warp-tier sampling launch(es) */
    double last_cta_ms;      /* device time of the last CTA-tier sampling launch(es) */
    double last_sample_ms;   /* device time of all sampling launches of the last skis_sample call */
    uint64_t last_passes;    /* sampling passes of the last call (> 1: the arena grew and reran) */
    uint64_t thread_max_deg;   /* the tier split in force (SKIS_OPT_THREAD_MAX_DEG, ...) */
    uint64_t thread_max_steps;
    uint64_t warp_max_coins;
    uint64_t cta_hub_quads;
    uint64_t first_id;       /* sample id of the sketch's first sample (SKIS_OPT_FIRST_ID) */
    double last_query_ms;    /* device time of the coverage launches of the last skis_estimate of at most
                                64 queries (scan or inverted-index walk) */
} skis_stats;

/* Sampling runs in three tiers chained by sample id: one lane per sample
 * (up to 32 members, in-rows up to THREAD_MAX_DEG edges, up to
 * THREAD_MAX_STEPS edge quads, up to THREAD_MAX_RETRIES rejected rounds;
 * the "thread" names below refer to this tier), one warp per sample (up to
 * 256 members, up to WARP_MAX_COINS in-edges), one CTA per sample (any size). Options tune the split; they
 * never change the samples. */
typedef enum skis_option {
    SKIS_OPT_RETRY_CAP = 0,      /* cap on rejected first-step rounds (default 2^24) */
    SKIS_OPT_CTA_SLOTS = 1,      /* CTAs of the CTA tier (default: 1024 threads of them per SM) */
    SKIS_OPT_WARP_BLOCKS = 2,    /* CTAs of the warp tier (default: full occupancy) */
    SKIS_OPT_THREAD_MAX_DEG = 3, /* longest in-row the thread tier expands (default 192; 0 = tier off) */
    SKIS_OPT_THREAD_BLOCKS = 4,  /* CTAs of the thread tier (default: full occupancy) */
    SKIS_OPT_QUERY_INDEX = 5,    /* skis_estimate: 0 = walk the inverted index (vertex -> samples) when
                                    it is built for the current samples, else scan the sketch (default);
                                    1 = build it if needed and walk it; 2 = always scan; 3 = always scan,
                                    with the members in sample-id order whatever the sketch's size (the
                                    scan's layout is otherwise used from 2^20 samples on) */
    SKIS_OPT_THREAD_MAX_STEPS = 6, /* edge quads a sample may take in the thread tier before the warp
                                      tier takes it over (default 256) */
    SKIS_OPT_SAMPLER = 7,         /* 0 = IIS samples (Alg. 1, default); 1 = plain RIS samples (Sec. II-C,
                                     Borgs et al.): uniform source (the column draw alone), one
                                     unconditioned round of the source's in-edges (singular samples
                                     occur), estimator n Cov / T (Lemma 1), greedy key Delta alone.
                                     Set before the first skis_sample. */
    SKIS_OPT_THREAD_MAX_RETRIES = 8, /* rejected first-step rounds a sample may take in the thread tier
                                        before the warp tier (rounds searched in parallel) takes it
                                        over (default 32) */
    SKIS_OPT_FIRST_STEP = 9        /* 0 = conditioned first step by rejection (default); 1 = bucket form
                                      (Eq. probn, no retries): the bucket of the source's row, "in-edges
                                      before i dead, edge i live", is drawn with mass Q_{i-1} - Q_i of the
                                      fixed-point gamma chain (total 2^62 - Q_d) by z = floor(U (2^62 -
                                      Q_d) / 2^64), U the 64-bit word of the Philox block (q 0, retry 0,
                                      domain BUCKET = 6, sample j); the first e with 2^62 - Q_e > z is
                                      live and the in-edges after it get their FIRST coins of round 0.
                                      IC graphs, IIS sampler; set before the first skis_sample; reads
                                      the per-edge chain IC graphs keep from loading. */,
    SKIS_OPT_WARP_MAX_COINS = 10,  /* in-edges a sample's BFS may draw in the warp tier before the CTA
                                      tier (all warps of a block on one sample) takes it over
                                      (default 65536; samples that reach huge in-rows) */
    SKIS_OPT_CTA_HUB_QUADS = 11,   /* CTA tier: in-rows of at least this many edge quads (default 256)
                                      are drawn by the whole block in one strided loop instead of being
                                      dealt with the level's other rows; 0 = never */
    SKIS_OPT_FIRST_ID = 12,        /* sample id of the sketch's first sample (default 0): the sketch
                                      holds ids [first, first + T), so that several sketches with one
                                      seed hold disjoint id ranges of one sketch (Alg. 2's R, sharded
                                      by id). Set before the first skis_sample; at most 2^62. */
    SKIS_OPT_CTA_QUEUE_CAP = 13,   /* member queue entries of a CTA-tier slot (default 2^20, at most n;
                                      in [32, 2^31]): a sample with more members moves to a second
                                      pass over fewer slots with n-entry queues */
    SKIS_OPT_CTA_THREADS = 14      /* threads of a CTA-tier block: 256 (default; four per SM) or 512
                                      (two per SM) */
} skis_option;

/* Load G = (V, E, w) (Sec. II-A) and build the device structures every later
 * step reads:
 *   - the canonical in-CSR: rows by destination, each row sorted by
 *     (source, input index); edge id = CSR position;
 *   - thresholds tau (per edge, or per row for WC);
 *   - gamma_v = 1 - prod over in-edges (1 - w(u,v)) (Eq. gamma_v, Sec. III-A)
 *     in fixed point: Q = 2^62, Q <- floor(Q (2^32 - tau) / 2^32) along the
 *     row (Q = 0 on a sentinel), w_v = (2^62 - Q) >> (ceil(log2 n) + 1);
 *   - W = sum_v w_v (Gamma = sum gamma_v) and the alias table of the source
 *     law Pr[src = v] = w_v / W (Eq. probu);
 *   - the chain of Q values after every in-edge (u64 per edge, computed
 *     with gamma), which the bucket form of the first step reads.
 * src, dst: int32[m] vertex ids in [0, n); weights: see skis_weight_model;
 * all three in mem_space. Rejected with SKIS_EINVAL: n < 1, n > 2^31,
 * m < 0, m >= 2^32 - 8, an id outside [0, n), a self-loop, p outside [0, 1]
 * or NaN. Parallel edges are kept as independent coins. */
int skis_load_graph(skis_graph **out, int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                    const void *weights, int weight_model, uint64_t weight_seed, int mem_space,
                    void *cuda_stream);

/* Load G under the Linear Threshold model (Sec. "Extensions to other
 * diffusion models", LT): the same inputs, CSR and thresholds as
 * skis_load_graph, read as edge weights w = tau / 2^32 (1 for the sentinel),
 * and
 *   - gamma_v = sum over in-edges of w(u,v), exactly: w_v = the row's sum of
 *     tau' (tau' = tau, 2^32 for the sentinel), f = 32;
 *   - the alias table of Pr[src = v] = w_v / W as above.
 * Every in-row must satisfy sum tau' <= 2^32 (the model's sum of in-weights
 * at most 1): otherwise SKIS_EINVAL naming the first such vertex; other
 * errors as skis_load_graph. Sketches of this graph draw LT samples (see
 * skis_sample); queries, greedy and the server are unchanged. */
int skis_load_graph_lt(skis_graph **out, int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                       const void *weights, int weight_model, uint64_t weight_seed, int mem_space,
                       void *cuda_stream);

int skis_graph_get_info(const skis_graph *g, skis_graph_info *info);

/* Copy the graph's device structures to host arrays (any may be NULL):
 * offsets int64[n+1], csr_src int32[m], tau uint32[m] (per-edge thresholds,
 * expanded for WC), perm int64[m] (CSR position -> input index),
 * w uint64[n], prob uint64[n], alias uint32[n]. Synchronises the stream. */
int skis_graph_export(const skis_graph *g, int64_t *offsets, int32_t *csr_src, uint32_t *tau,
                      int64_t *perm, uint64_t *w, uint64_t *prob, uint32_t *alias,
                      void *cuda_stream);

void skis_graph_free(skis_graph *g);

/* Create an empty SKIS sketch R (Alg. 2, preprocessing) over g with the
 * given Philox key. arena_entries is the initial capacity of the member
 * arena (0 = a default); the arena grows on demand. */
int skis_sketch_create(skis_sketch **out, const skis_graph *g, uint64_t seed,
                       uint64_t arena_entries, void *cuda_stream);

int skis_sketch_set_option(skis_sketch *s, int option, uint64_t value);

/* Autotuner of the sampling tiers: times pilot sampling of ids
 * [0, pilot_samples) on a scratch sketch under each candidate split, first
 * the lane/warp split (SKIS_OPT_THREAD_MAX_DEG in {0, 64, 128, 192, 256, 512}
 * x SKIS_OPT_THREAD_MAX_STEPS in {128, 256, 1024}, 16 candidates), then under
 * the fastest of those the warp/CTA split (SKIS_OPT_WARP_MAX_COINS in {4096,
 * 16384, 65536, 262144}); keeps the fastest on s and reports the lane/warp
 * choice (outputs nullable; candidate_ms receives up to candidate_cap pilot
 * times in that order, candidates_out their number; skis_sketch_stats gives
 * the whole split). The pilot samples are discarded; the samples of s never
 * depend on the split. */
int skis_sketch_autotune(skis_sketch *s, uint64_t pilot_samples, uint32_t *chosen_max_deg,
                         uint32_t *chosen_max_steps, double *candidate_ms, int32_t candidate_cap,
                         int32_t *candidates_out, void *cuda_stream);

/* Append IIS samples (Alg. 1) with ids [F + T, F + T + count) to the sketch
 * (F = SKIS_OPT_FIRST_ID, 0 by default). For sample j:
 *   - source: Philox block (key seed, domain SRC, id j) gives col = floor(U1 n)
 *     and y = floor(U2 W); src = col if y < prob[col] else alias[col];
 *   - first step (Alg. 1, Eq. probn) by rejection: round
 *     r = 0, 1, ... flips every in-edge coin of src (domain FIRST, retry r)
 *     until one is live; its live in-neighbours join R_j;
 *   - reverse BFS (Alg. 1): every in-edge e of every other member
 *     gets the coin (domain BFS, sample j, edge e); live edges add their
 *     source. R_j is the reverse-reachable set of src in that live-edge world.
 * Counters per sample: retries r, coins = d_in(src)(r + 1) + sum of d_in
 * over the other members. Returns SKIS_ERR_RETRY_LIMIT (the failing samples
 * are left empty) if a first step reaches the retry cap, SKIS_EINVAL if
 * W = 0 (no non-singular sample exists). Synchronises the stream.
 * next_sample_id_out (nullable) receives the next sample id, F + T. */
int skis_sample(skis_sketch *s, uint64_t count, uint64_t *next_sample_id_out, void *cuda_stream);

/* Stop-at-size sampling (the experiments' rule, Sec. VI "Algorithms
 * compared": samples are generated until their total size reaches h n log n,
 * the target here given in entries). Appends samples T, T+1, ... exactly as
 * skis_sample does and stops at the first one that brings
 * sum_{j < T'} |R_j| (over the whole sketch) to target_entries or more, or
 * after max_count samples. Samples are drawn in batches; those of the last
 * batch after the stopping one are dropped (the next call regenerates the
 * same ids). appended_out / next_sample_id_out (nullable) receive the number
 * appended and the next sample id. Errors as skis_sample; target_entries = 0 is
 * SKIS_EINVAL. Synchronises the stream. */
int skis_sample_to_size(skis_sketch *s, uint64_t target_entries, uint64_t max_count, uint64_t *appended_out,
                        uint64_t *next_sample_id_out, void *cuda_stream);

/* Influence queries (Alg. 2's estimate step, Eq. 21): for each seed set S_b, b <
 * num_queries, given as CSR (seed_offsets int64[q+1], seeds int32[...]):
 *   coverage_out[b] = Cov_R(S_b) = #{j : R_j meets S_b},
 *   estimate_out[b] = N / D with N = Cov W + T sum_{v in S_b} (2^f - w_v) and
 *   D = T 2^f, i.e. Cov/T Gamma~ + sum (1 - gamma~_v).
 * Pointers in mem_space; coverage_out may be NULL. Rejected with
 * SKIS_EINVAL: T = 0, an empty seed set, a seed outside [0, n), a seed
 * repeated within a set. Synchronises the stream. */
int skis_estimate(skis_sketch *s, int32_t num_queries, const int64_t *seed_offsets,
                  const int32_t *seeds, int64_t *coverage_out, double *estimate_out, int mem_space,
                  void *cuda_stream);

/* Greedy max-coverage on the sketch (Alg. 3): k rounds, each adds the vertex
 * v outside S maximising Eq. margin, compared exactly as the integer key
 * Delta_R(v, S) W + T (2^f - w_v); ties go to the lowest vertex id.
 * seeds_out int32[k], coverage_out int64[k] (cumulative Cov_R, nullable) and
 * estimate_out double[k] (I_R of each prefix, nullable) are host arrays.
 * Rejected with SKIS_EINVAL: k < 0, k > n, T = 0. Synchronises the stream. */
int skis_greedy_maxcover(skis_sketch *s, int32_t k, int32_t *seeds_out, int64_t *coverage_out,
                         double *estimate_out, void *cuda_stream);

int skis_sketch_stats(const skis_sketch *s, skis_stats *out);

/* Copy the samples with ids [first_id, first_id + count) (sample ids, as
 * SKIS_OPT_FIRST_ID places them) to host arrays (any may be NULL): src int32[count], retries uint32[count], len uint32[count],
 * coins uint64[count], member_offsets int64[count+1] and members (the
 * members of each sample, in device order, which is unspecified) with
 * capacity members_cap. Returns SKIS_EINVAL if the range is outside the
 * sketch or members_cap is too small. Synchronises the stream. */
int skis_sketch_export(const skis_sketch *s, uint64_t first_id, uint64_t count, int32_t *src,
                       uint32_t *retries, uint32_t *len, uint64_t *coins, int64_t *member_offsets,
                       int32_t *members, uint64_t members_cap, void *cuda_stream);

void skis_sketch_free(skis_sketch *s);

/* skis_estimate without any allocation. The paper has no counterpart: this
 * is a service for callers that cannot allocate device memory when they
 * query — a process whose device memory is already reserved in full by
 * another allocator (a framework's caching allocator or an application pool
 * sized at start-up), where cudaMalloc would fail or fragment that
 * reservation, and latency-critical query loops that must not pay an
 * allocation's unbounded latency and implicit synchronisation.
 * It answers the same queries as skis_estimate (same results) and calls no
 * cudaMalloc, cudaFree or allocating library routine, on the device or the
 * host. Its scratch is one static device array inside the library, held by
 * every GPU that loads the library until the process exits: 8 MiB of
 * per-vertex query masks plus 64 counters and a status word.
 * Limits (SKIS_EINVAL beyond them): the graph has at most 2^20 vertices;
 * num_queries <= 64. All pointers are DEVICE pointers except error_buf
 * (host, nullable, error_len bytes), which receives a message on failure.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current); make
 * that first call before any stream capture. Every call shares the array and
 * clears the part it needs at its start: calls that overlap on the GPU (on
 * two streams at once, or from two threads without ordering) race and give
 * wrong results; serialise them. Synchronises the stream. */
int skis_estimate_noalloc(const skis_sketch *s, int32_t num_queries, const int64_t *seed_offsets,
                          const int32_t *seeds, int64_t *coverage_out, double *estimate_out,
                          char *error_buf, uint64_t error_len, void *cuda_stream);

/* A sketch sharded by sample id over ranks (processes, usually one per GPU).
 * The samples of Alg. 2's sketch R are independent and keyed by id, so rank
 * r of N can hold the ids [F_r, F_r + T_r) of one seed's sketch
 * (SKIS_OPT_FIRST_ID) with disjoint ranges whose union is R. Coverage counts
 * (Eq. 21) and the greedy's marginal counts Delta (Alg. 3, Eq. margin) are
 * sums over the ranks' samples, so the two entry points below write each
 * rank's values into `exchange` and call the caller's all-reduce:
 *
 *   allreduce(ctx, buf, count, cuda_stream) must replace buf[0, count)
 *   (int64, DEVICE memory) on every rank by its sum over all ranks and
 *   return 0 (non-zero: failure, reported as SKIS_ERR_EXCHANGE). The library
 *   has synchronised cuda_stream before the call; when the callback returns,
 *   the sums must be in buf or be ordered before later work on cuda_stream
 *   (an NCCL all-reduce on that stream, or a host-side reduction followed by
 *   a copy back).
 *
 * `exchange` is a caller-owned DEVICE buffer (so that the caller's
 * communication library can own or register it), int64 entries as stated
 * below. Every rank makes the same calls with the same arguments (queries,
 * k); each rank's sketch must be made with the same graph and seed. Results
 * equal those of skis_estimate / skis_greedy_maxcover on one sketch holding
 * the union of the ranks' samples, bit for bit. A rank that fails before an
 * exchange leaves the others waiting in theirs: give the process group a
 * timeout.
 *
 * skis_estimate_sharded: as skis_estimate (outputs on every rank);
 * exchange holds num_queries + 1 entries; every rank's sketch holds at
 * least one sample. Two exchanges per call. */
typedef int (*skis_allreduce_fn)(void *ctx, int64_t *buf, int64_t count, void *cuda_stream);
int skis_estimate_sharded(skis_sketch *s, int32_t num_queries, const int64_t *seed_offsets, const int32_t *seeds,
                          int64_t *coverage_out, double *estimate_out, int mem_space, int64_t *exchange,
                          skis_allreduce_fn allreduce, void *ctx, void *cuda_stream);

/* skis_greedy_maxcover_sharded: as skis_greedy_maxcover (host outputs on
 * every rank); exchange holds n + 1 entries. The ranks sum their sample
 * counts, then their per-vertex list lengths (Delta at S = {}); each round
 * every rank takes the same exact argmax, covers its own samples of the
 * winner and the per-vertex decrements (and the number of newly covered
 * samples, entry n) are summed: k + 2 exchanges, the per-round ones of
 * 8 (n + 1) bytes. */
int skis_greedy_maxcover_sharded(skis_sketch *s, int32_t k, int32_t *seeds_out, int64_t *coverage_out,
                                 double *estimate_out, int64_t *exchange, skis_allreduce_fn allreduce, void *ctx,
                                 void *cuda_stream);

/* Influence maximisation with DSSA-style doubling over SKIS sketches
 * (Sec. V-B; the appendix "Improvements of SSA/DSSA using SKIS sketch"):
 * two independent sketches R (Philox key seed_r) and R^c (seed_rc) start with
 * n0 samples and double in place (capped at n_max) each round t = 1, 2, ...;
 * greedy (Alg. 3) on R gives S_k, which is re-estimated on R^c; the run stops
 * when Cov_R(S_k) >= lambda2 and
 *   (e1 + e2 + e1 e2)(1 - 1/e - eps) + (1 - 1/e) e3 <= eps, with
 *   e1 = I_R / I_Rc - 1, e2 = eps sqrt(n (1 + eps) / (2^(t-1) I_Rc)),
 *   e3 = eps sqrt(n (1 + eps)(1 - 1/e - eps) / ((1 + eps/3) 2^(t-1) I_Rc)),
 * or when R holds n_max samples. The paper gives Lambda_2 only up to a
 * constant: lambda2 = 0 selects ceil((2 Gamma/n + 2 eps/3) ln(2 t_max / delta)
 * / eps^2), t_max = the number of rounds from n0 to n_max. Estimates are
 * formed on the host from exact integers with correctly rounded
 * conversions, so the stopping decisions are reproducible. seeds_out:
 * host int32[k]. Rejected with SKIS_EINVAL: k outside [1, n], eps outside
 * (0, 1 - 1/e), delta outside (0, 1), not 1 <= n0 <= n_max < 2^32, Gamma = 0. */
typedef struct skis_dssa_result {
    int32_t rounds;      /* rounds run (t) */
    int32_t stopped_by;  /* 1: the stop test held; 2: the sample cap was reached */
    uint64_t samples;    /* |R| = |R^c| at the end */
    uint64_t lambda2;    /* coverage threshold used */
    int64_t coverage;    /* Cov_R(S_k) */
    int64_t coverage_c;  /* Cov_{R^c}(S_k) */
    double estimate;     /* I_R(S_k) */
    double estimate_c;   /* I_{R^c}(S_k) */
    double eps1, eps2, eps3;
} skis_dssa_result;
int skis_dssa_maxinf(const skis_graph *g, uint64_t seed_r, uint64_t seed_rc, int32_t k, double eps, double delta,
                     uint64_t lambda2, uint64_t n0, uint64_t n_max, int32_t *seeds_out, skis_dssa_result *res,
                     void *cuda_stream);

/* Continuous-batching influence-oracle server over a device-resident sketch
 * (Alg. 2's estimate step for a stream of requests). skis_server_submit validates a
 * seed set (host array, copied; non-empty, ids in [0, n), no repeats) and
 * queues it, returning a ticket. skis_server_progress retires finished
 * batches and admits queued requests, in arrival order, into every free
 * in-flight slot: up to max_batch requests (<= 64, one query-mask bit each)
 * whose seeds fit the slot's seed_capacity. Each of the `slots` slots has its
 * own stream, pinned staging, device buffers and n-word query-mask scratch
 * (allocated at creation), so batches on different slots overlap on the
 * device. With wait != 0, progress first blocks until one in-flight batch
 * completes. Completed tickets are written to done_tickets (capacity cap).
 * skis_server_poll reports a ticket's state (0 pending, 1 ready, 2 failed)
 * and, when ready, its Cov_R(S) and I_R(S) — the same values skis_estimate
 * gives for that seed set. The sketch must not change while a server uses
 * it; one host thread drives a server. */
typedef struct skis_server skis_server;
int skis_server_create(skis_server **out, skis_sketch *s, int32_t slots, int32_t max_batch,
                       uint64_t seed_capacity);
int skis_server_submit(skis_server *srv, const int32_t *seeds, int32_t nseeds, uint64_t *ticket_out);
int skis_server_progress(skis_server *srv, int32_t wait, uint64_t *done_tickets, int32_t cap,
                         int32_t *ndone_out);
int skis_server_poll(skis_server *srv, uint64_t ticket, int64_t *coverage_out, double *estimate_out,
                     int32_t *state_out);
int skis_server_counts(const skis_server *srv, uint64_t *queued, uint64_t *in_flight, uint64_t *batches,
                       uint64_t *served);
void skis_server_free(skis_server *srv);

/* The integer-ALU ceiling of the coin generator on this GPU (a measurement
 * probe, no counterpart in the paper): `threads` threads each draw the
 * Philox4x32-10 blocks of edge quads [t b, (t + 1) b) of sample id t (BFS
 * domain, key seed; b = blocks_per_thread), four independent blocks a step,
 * and fold every word of every block into one XOR, in one launch with no
 * memory traffic but one atomic per thread: form 0 computes every block as a
 * sampler tier does (20 products), form 1 as the CTA tier's hub loop does
 * (two products hoisted per sample, 18). ms_out receives the launch's device
 * time, fold_out the XOR of all words (it depends on the coins only).
 * threads and blocks_per_thread in [1, 2^31] with fewer than 2^32 blocks in
 * all, form 0 or 1, else SKIS_EINVAL; synchronises the stream. */
int skis_philox_rate(uint64_t seed, uint64_t threads, uint64_t blocks_per_thread, int form, double *ms_out,
                     uint32_t *fold_out, void *cuda_stream);

/* Number of CUDA kernel launches the library has made in this process
 * (diagnostic; counts every launch of every entry point). */
uint64_t skis_kernel_launches(void);

/* Number of device memory allocations the library has made in this
 * process (diagnostic; every entry point's, whatever the allocator). */
uint64_t skis_device_allocations(void);

/* Message of the last failing call on this thread ("" if none). */
const char *skis_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SKIS_H */
