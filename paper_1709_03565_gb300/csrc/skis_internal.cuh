// Internal declarations of the SKIS GB300 library: device data layouts,
// the counter-based Philox coin generator, warp helpers and the launch
// entry points shared between translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/skis.h"

namespace skis {

typedef unsigned __int128 u128;

constexpr uint32_t kSentinel = 0xFFFFFFFFu;  // threshold meaning "always live"
constexpr unsigned kFull = 0xFFFFFFFFu;

// Philox counter domains: one independent stream per use of randomness.
enum : uint32_t { kDomSrc = 1, kDomFirst = 2, kDomBfs = 3, kDomWeight = 4, kDomLt = 5, kDomBucket = 6 };

// Per-vertex in-row record, one 16-byte load on the hot path: CSR offset of
// the row, its length d_in(v) and, for row-uniform models (WC), the row's
// threshold.
struct __align__(16) RowInfo {
    uint64_t off;
    uint32_t deg;
    uint32_t tau;
};

// Alias column (Eq. probu): threshold in [0, W] and the alias vertex.
struct __align__(16) AliasEntry {
    uint64_t prob;
    uint32_t alias;
    uint32_t pad;
};

// Device status word shared by kernels that can fail on the data.
struct DevStatus {
    unsigned int flags;
    unsigned int gave_up;          // a bounded device wait ran out (an invariant failed)
    unsigned long long first_bad;  // smallest failing index / sample id
};
enum : unsigned int {
    kStRetry = 1u,      // a first step hit the retry cap
    kStInval = 2u,      // invalid input data (ids, self-loop, p, query)
    kStArena = 4u,      // an arena reservation did not fit
    kStListFull = 8u,   // a deferral list overflowed (cannot happen by sizing)
};

// ------------------------------------------------------------------ Philox
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): per round,
// the products of words 0 and 2 with the two multipliers are split into
// high/low halves and recombined with words 1, 3 and the round key; the key
// then advances by the two Weyl increments.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        // one 32 x 32 -> 64-bit product per multiplier gives both halves
        const uint64_t pa = (uint64_t)0xD2511F53u * c.x;
        const uint64_t pb = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(pb >> 32) ^ c.y ^ k0, (uint32_t)pb, (uint32_t)(pa >> 32) ^ c.w ^ k1, (uint32_t)pa);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The Philox block holding the coins of edge quad q (edges 4q .. 4q+3) of
// sample j in domain dom and first-step round `retry`. Counter words:
// (q mod 2^32, (q >> 32) & 0xF | retry << 4 | dom << 28, j mod 2^32, j >> 32);
// key = (seed mod 2^32, seed >> 32). Edge e's coin is word e mod 4.
__device__ __forceinline__ uint4 coin_block(uint64_t seed, uint64_t q, uint32_t retry, uint32_t dom,
                                            uint64_t j) {
    uint4 c;
    c.x = (uint32_t)q;
    c.y = ((uint32_t)(q >> 32) & 0xFu) | ((retry & 0xFFFFFFu) << 4) | (dom << 28);
    c.z = (uint32_t)j;
    c.w = (uint32_t)(j >> 32);
    return philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// The ten round keys of a Philox key, (k0 + i W0, k1 + i W1) for round i,
// held in a kernel's parameters so that each round reads its key pair as an
// operand instead of advancing it; the block is the same as philox10's.
struct PhiloxKeys {
    uint32_t k[20];
};

inline PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys r;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        r.k[2 * i] = k0;
        r.k[2 * i + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return r;
}

__device__ __forceinline__ uint4 philox10(uint4 c, const PhiloxKeys& rk) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint64_t pa = (uint64_t)0xD2511F53u * c.x;
        const uint64_t pb = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(pb >> 32) ^ c.y ^ rk.k[2 * i], (uint32_t)pb,
                       (uint32_t)(pa >> 32) ^ c.w ^ rk.k[2 * i + 1], (uint32_t)pa);
    }
    return c;
}

__device__ __forceinline__ uint4 coin_block(const PhiloxKeys& rk, uint64_t q, uint32_t retry, uint32_t dom,
                                            uint64_t j) {
    uint4 c;
    c.x = (uint32_t)q;
    c.y = ((uint32_t)(q >> 32) & 0xFu) | ((retry & 0xFFFFFFu) << 4) | (dom << 28);
    c.z = (uint32_t)j;
    c.w = (uint32_t)(j >> 32);
    return philox10(c, rk);
}

// coin_block(rk, q, 0, dom, j) for one sample j and many edge quads q < 2^32
// (every CSR position is below 2^32, so the counter's second word is dom << 28
// alone). Of the first two rounds' four products, two depend only on (j, dom):
// round 0 multiplies word 2 (the low id word) and round 1 multiplies word 0,
// which round 0 made from the id alone. Those two and the key terms that meet
// them are formed once per sample, leaving 18 products per block instead of
// 20; the block is bit-identical to philox10's.
struct SampleBlock {
    uint32_t a0;   // word 0 after round 0
    uint32_t c1;   // word 1 after round 0, xor round 1's key 0
    uint32_t c2;   // high half of round 1's word-0 product, xor round 1's key 1
    uint32_t c3;   // low half of that product (word 3 after round 1), xor round 2's key 1
    uint32_t k1j;  // round 0's key 1 xor the high id word

    __device__ __forceinline__ SampleBlock(const PhiloxKeys& rk, uint64_t j, uint32_t dom) {
        const uint64_t pb = (uint64_t)0xCD9E8D57u * (uint32_t)j;
        a0 = (uint32_t)(pb >> 32) ^ (dom << 28) ^ rk.k[0];
        c1 = (uint32_t)pb ^ rk.k[2];
        const uint64_t pa = (uint64_t)0xD2511F53u * a0;
        c2 = (uint32_t)(pa >> 32) ^ rk.k[3];
        c3 = (uint32_t)pa ^ rk.k[5];
        k1j = (uint32_t)(j >> 32) ^ rk.k[1];
    }

    __device__ __forceinline__ uint4 operator()(uint32_t q, const PhiloxKeys& rk) const {
        const uint64_t p0 = (uint64_t)0xD2511F53u * q;             // round 0, word 0
        const uint32_t x2 = (uint32_t)(p0 >> 32) ^ k1j, x3 = (uint32_t)p0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;            // round 1, word 2
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ c1, y1 = (uint32_t)p1, y2 = x3 ^ c2;
        const uint64_t p2a = (uint64_t)0xD2511F53u * y0;           // round 2
        const uint64_t p2b = (uint64_t)0xCD9E8D57u * y2;
        uint4 c = make_uint4((uint32_t)(p2b >> 32) ^ y1 ^ rk.k[4], (uint32_t)p2b, (uint32_t)(p2a >> 32) ^ c3,
                             (uint32_t)p2a);
#pragma unroll
        for (int i = 3; i < 10; ++i) {
            const uint64_t pa = (uint64_t)0xD2511F53u * c.x;
            const uint64_t pb = (uint64_t)0xCD9E8D57u * c.z;
            c = make_uint4((uint32_t)(pb >> 32) ^ c.y ^ rk.k[2 * i], (uint32_t)pb,
                           (uint32_t)(pa >> 32) ^ c.w ^ rk.k[2 * i + 1], (uint32_t)pa);
        }
        return c;
    }
};

__device__ __forceinline__ uint32_t word_of(const uint4& x, int k) {
    return k == 0 ? x.x : k == 1 ? x.y : k == 2 ? x.z : x.w;
}

__device__ __forceinline__ bool coin_live(uint32_t x, uint32_t tau) {
    return tau == kSentinel || x < tau;
}

// --------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ u128 shfl_u128(u128 v, int src) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_sync(kFull, lo, src);
    hi = __shfl_sync(kFull, hi, src);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int d) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_down_sync(kFull, lo, d);
    hi = __shfl_down_sync(kFull, hi, d);
    return ((u128)hi << 64) | lo;
}

// binary64 value of an unsigned 128-bit integer (two correctly rounded
// conversions and one rounded addition: relative error below 2^-52).
__host__ __device__ __forceinline__ double u128_to_double(u128 v) {
    const uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// -------------------------------------------------------- device memory
// Stream-ordered allocation helpers (cudaMallocAsync / cudaFreeAsync).
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);
// Synchronous allocation (cudaMalloc), for long-lived buffers.
cudaError_t dev_malloc(void** p, size_t bytes);
// Process-wide count of device allocations made through dev_alloc / dev_malloc.
uint64_t allocations();

template <typename T>
cudaError_t dev_alloc_t(T** p, size_t count, cudaStream_t st) {
    return dev_alloc((void**)p, count * sizeof(T) + (count == 0 ? 16 : 0), st);
}

// ------------------------------------------------------------ primitives
// Exclusive prefix sums with the total appended: out[0] = 0,
// out[i] = in[0] + ... + in[i-1], out[n] = total. Temporary memory is taken
// stream-ordered from the pool.
cudaError_t scan_u32_to_u64(const uint32_t* in, uint64_t* out, int64_t n, cudaStream_t st);
cudaError_t scan_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t st);
cudaError_t scan_u128(const u128* in, u128* out, int64_t n, cudaStream_t st);

// Stable sort of the m edges by key dst << src_bits | src (keys of
// 2 src_bits bits), the input index as value, written out as the CSR arrays:
// csr_src[e], csr_dst[e] and perm[e] (the input index) for every sorted
// position e < m. keys_a / vals_a and keys_b / vals_b (m entries each) are
// scratch. *gave_up (device word) is set nonzero if a look-back wait ran out
// (which only a tile that never ran could cause) or an output position fell
// outside [0, m); the result is then invalid and nothing was written out of
// bounds.
cudaError_t sort_edges(const int32_t* src, const int32_t* dst, int64_t m, int src_bits, int32_t* csr_src,
                       uint32_t* csr_dst, uint32_t* perm, uint64_t* keys_a, uint32_t* vals_a, uint64_t* keys_b,
                       uint32_t* vals_b, unsigned int* gave_up, cudaStream_t st);

// Sum of a uint64 array (integers: order-independent), result in *out (device).
cudaError_t sum_u64(const uint64_t* in, int64_t n, unsigned long long* out, cudaStream_t st);

int sm_count();

// Process-wide count of kernel launches made by the library.
void note_launch();
uint64_t launches();

}  // namespace skis

// Device-resident probabilistic graph G = (V, E, w) (C handle).
struct skis_graph {
    int64_t n = 0, m = 0;
    int64_t m_pad = 0;          // edge arrays padded to a multiple of 4 (+4)
    int32_t s = 0, f = 0;       // gamma~ = w / 2^f, s = 62 - f
    uint64_t W = 0;             // sum of w
    int row_uniform = 0;        // thresholds live in RowInfo.tau (WC)
    int lt = 0;                 // Linear Threshold model: w_v = sum of the row's weights, f = 32
    uint64_t* lt_cum = nullptr; // LT with per-edge thresholds: exclusive running sums of the
                                // weights tau' (2^32 for the sentinel) in CSR order, m + 1
    uint64_t* chain = nullptr;  // bucket first step: the fixed-point chain Q after each in-edge
                                // of its row (m), built on first use
    uint64_t* off = nullptr;    // n+1 CSR offsets
    skis::RowInfo* rows = nullptr;     // n
    int32_t* src = nullptr;     // m_pad, CSR order, padding = 0
    uint32_t* tau = nullptr;    // m_pad per-edge thresholds (nullptr if row_uniform)
    uint32_t* perm = nullptr;   // m: CSR position -> input index
    uint64_t* w = nullptr;      // n fixed-point gamma numerators
    skis::AliasEntry* alias = nullptr;  // n
    cudaStream_t stream = nullptr;      // stream of the last call (for release)
};

namespace skis {
// Device cursors and counters of one skis_sample call.
struct SampleCounters {
    unsigned long long arena;        // arena reservation cursor (persists across calls)
    unsigned long long novf;         // samples whose arena reservation did not fit
    unsigned long long work_thread;  // id cursors of the three tiers
    unsigned long long work_warp;
    unsigned long long work_cta;
    unsigned long long n_to_warp;    // samples handed from the thread tier to the warp tier
    unsigned long long n_to_cta;     // samples handed from the warp tier to the CTA tier
    unsigned long long n_big;        // CTA-tier samples that outgrew a slot's queue
    unsigned long long work_big;     // id cursor of the pass over them
};
}  // namespace skis

// Device-resident SKIS sketch R = {R_0 .. R_{T-1}} (C handle).
struct skis_sketch {
    const skis_graph* g = nullptr;
    uint64_t seed = 0;
    uint64_t T = 0;
    uint64_t hcap = 0;                   // header capacity
    uint64_t* h_off = nullptr;           // arena offset of R_j
    uint32_t* h_len = nullptr;           // |R_j| (0 for a failed sample)
    uint32_t* h_src = nullptr;           // src(R_j)
    uint32_t* h_retries = nullptr;       // rejected first-step rounds
    uint64_t* h_coins = nullptr;         // in-edges examined
    int32_t* arena = nullptr;            // members, sample after sample (with gaps)
    uint64_t arena_cap = 0;
    uint64_t arena_hint = 0;
    skis::SampleCounters* ctr = nullptr;
    skis::DevStatus* status = nullptr;
    uint64_t* to_warp_ids = nullptr;     // thread tier -> warp tier
    uint64_t* to_cta_ids = nullptr;      // warp tier -> CTA tier
    uint64_t* ovf_ids[2] = {nullptr, nullptr};
    uint4* srcrec = nullptr;             // lane tier: prepared source records
    uint2* srcpick = nullptr;            // lane tier, bucket form: prepared first-step picks
    uint64_t list_cap = 0;
    uint32_t* bitmaps = nullptr;         // CTA tier: one n-bit visited bitmap per slot
    int32_t* queues = nullptr;           // CTA tier: one queue_cap-entry queue per slot
    uint32_t queue_cap = 0;              // entries of each slot's queue: min(n, cta_queue_cap)
    uint32_t cta_queue_cap = 1u << 20;   // option: queue entries per CTA-tier slot
    int cta_threads = 256;               // option: threads of a CTA-tier block (256 or 512)
    uint64_t* big_ids = nullptr;         // CTA tier -> the pass with n-entry queues
    int32_t* big_queues = nullptr;       // that pass's queues (n entries each), allocated on first use
    int big_slots = 0;
    uint32_t* lt_hash = nullptr;         // LT medium walks: visited table per lane
    int32_t* lt_list = nullptr;          // LT medium walks: member list per lane
    uint32_t* lt_slot = nullptr;         // LT medium walks: table slot of each listed member
    uint64_t lt_mid_lanes = 0;
    int cta_slots_alloc = 0;
    uint64_t bitmap_words = 0;
    // options
    uint32_t retry_cap = 1u << 24;
    int cta_slots = 0;                   // 0 = automatic
    int warp_blocks = 0;                 // 0 = automatic
    int thread_blocks = 0;               // 0 = automatic
    uint32_t thread_max_deg = 192;       // longest in-row the thread tier expands (0 = tier off)
    uint32_t thread_max_steps = 256;     // edge quads per sample in the thread tier
    uint32_t thread_max_retries = 32;    // rejected rounds in the thread tier before the warp tier
    uint32_t warp_max_coins = 65536;     // in-edges a sample may draw in the warp tier before the CTA tier
    uint32_t cta_hub_quads = 256;        // CTA tier: rows of at least this many edge quads take the hub loop
    uint64_t id_base = 0;                // sample id of header 0: the sketch holds ids [id_base, id_base + T)
    // last-call statistics
    uint64_t last_to_warp = 0, last_deferred = 0, last_passes = 0;
    double last_thread_ms = 0, last_warp_ms = 0, last_cta_ms = 0, last_sample_ms = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // inverted index vertex -> samples (built on demand for the current T)
    uint64_t ordered_T = 0;              // samples [0, ordered_T) hold arena positions [0, ordered_E) in id order
    uint64_t ordered_E = 0;
    uint64_t* inv_off = nullptr;         // n+1
    uint32_t* inv = nullptr;             // sample ids, vertex after vertex
    uint64_t inv_T = 0;                  // T when the index was built (0 = none)
    int query_index = 0;                 // 0 auto (use the index if built), 1 always, 2 never
    int ris = 0;                         // plain RIS samples (uniform source, n Cov / T estimator)
    int bucket = 0;                      // first step in bucket form (Eq. probn) instead of rejection
    uint32_t* vcount = nullptr;          // n: members per vertex over samples [0, vcount_T)
    uint64_t vcount_T = 0;
    bool vcount_ok = true;               // vcount is exact for samples [0, vcount_T)
    // query / greedy scratch (allocated on first use)
    uint64_t* smask = nullptr;           // T per-sample query bits (inverted-index path)
    uint64_t smask_cap = 0;
    uint64_t* qmask = nullptr;           // n per-vertex query bits
    uint32_t* qbits = nullptr;           // n bits: the vertex is a seed of the current batch
    unsigned long long* qcov = nullptr;  // 64 coverage counters
    uint32_t* touched = nullptr;         // ordered scan: samples whose query word was set (for the reset)
    unsigned long long* ntouched = nullptr;  // [0] touched count, [1] task cursor, [2] hit count
    unsigned long long* hits = nullptr;      // ordered scan: (task, position) of members that may be seeds
    uint64_t touched_cap = 0;
    cudaEvent_t qev[2] = {nullptr, nullptr};  // around the coverage launches of a query chunk
    double last_query_ms = 0;            // their device time in the last skis_estimate (<= 64 queries)
    skis::DevStatus* qstatus = nullptr;
    cudaStream_t stream = nullptr;
};

namespace skis {
int sketch_sample(skis_sketch* s, uint64_t count, cudaStream_t st, std::string* err);
int sketch_sample_to_size(skis_sketch* s, uint64_t target, uint64_t max_count, cudaStream_t st, uint64_t* appended,
                          std::string* err);
int sketch_estimate(skis_sketch* s, int32_t q, const int64_t* d_off, const int32_t* d_seeds, const int64_t* h_off,
                    int64_t* d_cov, double* d_est, cudaStream_t st, std::string* err);
int sketch_greedy(skis_sketch* s, int32_t k, int32_t* h_seeds, int64_t* h_cov, double* h_est, cudaStream_t st,
                  std::string* err);
// Eq. 21 and Alg. 3 over a sketch split by sample id across ranks; exch is
// the caller's device buffer that fn sums over the ranks in place.
int sketch_estimate_sharded(skis_sketch* s, int32_t q, const int64_t* d_off, const int32_t* d_seeds,
                            const int64_t* h_off, int64_t* d_cov, double* d_est, int64_t* exch, skis_allreduce_fn fn,
                            void* ctx, cudaStream_t st, std::string* err);
int sketch_greedy_sharded(skis_sketch* s, int32_t k, int32_t* h_seeds, int64_t* h_cov, double* h_est, int64_t* exch,
                          skis_allreduce_fn fn, void* ctx, cudaStream_t st, std::string* err);
// Lays the members of samples [ordered_T, T) out in sample-id order right
// after those of the samples before them (headers rebased, arena cursor
// moved to the end): a warp's consecutive samples then read one contiguous
// run of members. Only the layout changes, never a sample.
int sketch_order_arena(skis_sketch* s, cudaStream_t st, std::string* err);
// Builds (or reuses) the inverted index of the current T samples.
int sketch_inverted(skis_sketch* s, cudaStream_t st, std::string* err);
// Coverage of queries [q0, q0 + qn) of a CSR batch through the inverted
// index: cov[b - q0] = #samples meeting S_b. smask (T words, all zero on
// entry) is restored to zero; chunk_cnt/chunk_off hold nseeds (+1) entries.
cudaError_t coverage_by_index(const skis_sketch* s, const int64_t* off, const int32_t* seeds, int32_t q0,
                              int32_t qn, int64_t seed_base, int64_t nseeds, uint32_t* chunk_cnt,
                              uint64_t* chunk_off, uint64_t* smask, unsigned long long* cov, cudaStream_t st);
void sketch_release(skis_sketch* s);
int sketch_autotune(skis_sketch* s, uint64_t pilot, cudaStream_t st, double* cand_ms, int cand_cap, int* ncand,
                    std::string* err);
// The coin generator's throughput on this GPU (the ALU ceiling probe).
int philox_rate(uint64_t seed, uint64_t threads, uint64_t per, int form, double* ms_out, uint32_t* fold_out,
                cudaStream_t st, std::string* err);

// Records msg as the calling thread's last error (skis_last_error); returns code.
int set_last_error(int code, const std::string& msg);

// Coverage kernels (defined in cover.cu).
__global__ void k_qmask_set(const int64_t* __restrict__ off, const int32_t* __restrict__ seeds, int32_t q0,
                            int32_t qn, int64_t n, uint64_t* __restrict__ qmask, uint32_t* __restrict__ qbits,
                            DevStatus* st);
__global__ void k_qmask_clear(const int64_t* __restrict__ off, const int32_t* __restrict__ seeds, int32_t q0,
                              int32_t qn, int64_t n, uint64_t* __restrict__ qmask, uint32_t* __restrict__ qbits,
                              unsigned long long* __restrict__ reset2);
__global__ void __launch_bounds__(256) k_coverage(const uint64_t* __restrict__ h_off, const uint32_t* __restrict__ h_len, uint64_t T,
                           const int32_t* __restrict__ arena, const uint64_t* __restrict__ qmask,
                           const uint32_t* __restrict__ qbits, int hashed, unsigned long long* __restrict__ cov);
__global__ void k_estimate(const int64_t* __restrict__ off, const int32_t* __restrict__ seeds, int32_t q0,
                           int32_t qn, int64_t n, const uint64_t* __restrict__ w, int f, uint64_t W, uint64_t T,
                           const unsigned long long* __restrict__ cov, int64_t* __restrict__ cov_out,
                           double* __restrict__ est_out, int ris);

// Builds every device structure of g from device edge arrays. Returns a
// skis_status code; *err receives a message on failure.
int graph_build(skis_graph* g, const int32_t* d_src, const int32_t* d_dst, const void* d_weights,
                int model, uint64_t weight_seed, int lt, cudaStream_t st, std::string* err);
void graph_release(skis_graph* g);
int graph_ensure_chain(const skis_graph* g, cudaStream_t st, std::string* err);
}  // namespace skis
