// Graph build on the device (Sec. II-A, Sec. III-A components 1 and 2):
// input validation, the canonical in-CSR, integer thresholds, gamma_v in
// fixed point (Eq. gamma_v) and the alias table of the source law
// Pr[src = v] = gamma_v / Gamma (Eq. probu).
#include <string>

#include "../../include/skis.h"
#include "skis_internal.cuh"

namespace skis {

#define GB_CUDA(call)                                                         \
    do {                                                                      \
        cudaError_t _e = (call);                                              \
        if (_e != cudaSuccess) {                                              \
            *err = std::string("CUDA error in graph build: ") + cudaGetErrorString(_e); \
            rc = _e == cudaErrorMemoryAllocation ? SKIS_ENOMEM : SKIS_ERR_CUDA; \
            goto cleanup;                                                     \
        }                                                                     \
    } while (0)

// tau = floor(p * 2^32) (p * 2^32 is exact in binary64), clamped to the
// always-live sentinel; p >= 1 is always live.
__device__ __forceinline__ uint32_t tau_from_p(double p) {
    if (p >= 1.0) return kSentinel;
    const uint64_t t = (uint64_t)(p * 4294967296.0);
    return t >= kSentinel ? kSentinel : (uint32_t)t;
}

__global__ void k_validate(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                           const double* __restrict__ p, int64_t m, int64_t n, DevStatus* st) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        bool bad = u < 0 || u >= n || v < 0 || v >= n || u == v;
        if (p) {
            const double x = p[e];
            bad = bad || !(x >= 0.0 && x <= 1.0);
        }
        if (bad) {
            atomicOr(&st->flags, kStInval);
            atomicMin(&st->first_bad, (unsigned long long)e);
        }
    }
}

// Row offsets of the canonical CSR from the sorted destinations: off[v] is
// the first position whose destination is >= v. Position e writes off[v]
// for the destinations v in (dst(e - 1), dst(e)], and the last position the
// ones after its destination, so every entry of off[0 .. n] is written once.
__global__ void k_offsets_from_dst(const uint32_t* __restrict__ csr_dst, int64_t m, int64_t n,
                                   uint64_t* __restrict__ off) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = e > 0 ? (int64_t)csr_dst[e - 1] : -1;
        const int64_t cur = e < m ? (int64_t)csr_dst[e] : n;
        for (int64_t v = prev + 1; v <= cur; ++v) off[v] = (uint64_t)e;
    }
}

// Per-edge thresholds of the CSR positions by model (explicit p or tau read
// through the input index; TRI from the WEIGHT coin of the position).
// Padding positions (m .. m_pad) get threshold 0 (never live).
__global__ void k_edge_tau(const uint32_t* __restrict__ perm, int64_t m, int64_t m_pad, int model,
                           const void* __restrict__ weights, uint64_t weight_seed, uint32_t* __restrict__ csr_tau) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m_pad; e += (int64_t)gridDim.x * blockDim.x) {
        if (e >= m) {
            csr_tau[e] = 0;
            continue;
        }
        uint32_t t;
        if (model == SKIS_W_EXPLICIT_P) {
            t = tau_from_p(((const double*)weights)[perm[e]]);
        } else if (model == SKIS_W_EXPLICIT_TAU) {
            t = ((const uint32_t*)weights)[perm[e]];
        } else {  // SKIS_W_TRI: level floor(3 x / 2^32) of the WEIGHT coin of position e
            const uint4 x = coin_block(weight_seed, (uint64_t)e >> 2, 0, kDomWeight, 0);
            const uint32_t level = (uint32_t)(((uint64_t)word_of(x, (int)(e & 3)) * 3u) >> 32);
            t = tau_from_p(level == 0 ? 0.1 : level == 1 ? 0.01 : 0.001);
        }
        csr_tau[e] = t;
    }
}

__global__ void k_rows(const uint64_t* __restrict__ off, int64_t n, int wc, RowInfo* __restrict__ rows) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        RowInfo r;
        r.off = off[v];
        r.deg = (uint32_t)(off[v + 1] - off[v]);
        r.tau = 0;
        if (wc) r.tau = r.deg == 1 ? kSentinel : (r.deg ? (uint32_t)((1ull << 32) / r.deg) : 0u);
        rows[v] = r;
    }
}

// One step of the fixed-point chain, Q <- floor(Q (2^32 - t) / 2^32) for
// Q < 2^62 (0 for the sentinel). With Q = qh 2^32 + ql and c = 2^32 - t,
// the floor is exactly qh c + floor(ql c / 2^32): two independent 32-bit
// products (qh < 2^30, so qh c < 2^62) instead of a 128-bit one, which
// shortens the dependent chain a long row walks edge by edge.
__device__ __forceinline__ uint64_t chain_step(uint64_t Q, uint32_t t) {
    if (t == kSentinel) return 0;
    if (t == 0) return Q;  // c = 2^32
    const uint32_t c = (uint32_t)(0x100000000ull - t);
    return (uint64_t)(uint32_t)(Q >> 32) * c + __umulhi((uint32_t)Q, c);
}

// Eq. gamma_v in fixed point for one row: Q = 2^62; Q <- floor(Q (2^32 -
// tau) / 2^32) for each in-edge in CSR order (0 on a sentinel); the caller
// takes w_v = (2^62 - Q) >> s from the returned last value. With chain !=
// nullptr the running Q after every in-edge is kept as well.
__device__ __forceinline__ uint64_t gamma_row(const RowInfo& r, const uint32_t* __restrict__ csr_tau,
                                              uint64_t* __restrict__ chain) {
    uint64_t Q = 1ull << 62;
    uint32_t k = 0;
    if (!csr_tau) {  // one threshold for the row (weighted cascade)
        const uint32_t t = r.tau;
        if (t == kSentinel || t == 0) {  // every step gives 0, or keeps Q
            const uint64_t q = (t == kSentinel && r.deg) ? 0 : Q;
            if (chain)
                for (; k < r.deg; ++k) chain[r.off + k] = q;
            return q;
        }
        // a pure dependent chain of Q <- qh c + hi32(ql c), four steps an
        // iteration, their values stored two to a 16-byte store when the
        // position is even (the chain array is 16-byte aligned)
        const uint32_t c = (uint32_t)(0x100000000ull - t);
        auto step = [c](uint64_t q) { return (uint64_t)(uint32_t)(q >> 32) * c + __umulhi((uint32_t)q, c); };
        if (chain && ((r.off + k) & 1) && k < r.deg) {
            Q = step(Q);
            chain[r.off + k] = Q;
            ++k;
        }
        for (; k + 4 <= r.deg && (Q != 0 || chain); k += 4) {
            const uint64_t q1 = step(Q), q2 = step(q1), q3 = step(q2), q4 = step(q3);
            if (chain) {
                ulonglong2* p = reinterpret_cast<ulonglong2*>(chain + r.off + k);
                p[0] = make_ulonglong2(q1, q2);
                p[1] = make_ulonglong2(q3, q4);
            }
            Q = q4;
        }
        for (; k < r.deg && (Q != 0 || chain); ++k) {
            Q = step(Q);
            if (chain) chain[r.off + k] = Q;
        }
        return Q;
    }
    for (; k + 8 <= r.deg && (Q != 0 || chain); k += 8) {
        uint32_t t[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = csr_tau[r.off + k + i];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            Q = chain_step(Q, t[i]);
            if (chain) chain[r.off + k + i] = Q;
        }
    }
    for (; k < r.deg && (Q != 0 || chain); ++k) {
        Q = chain_step(Q, csr_tau[r.off + k]);
        if (chain) chain[r.off + k] = Q;
    }
    return Q;
}

// Rows by the bit length of their degree (class b: 2^(b-1) <= d_in < 2^b;
// class 0: no in-edge). A graph with no row of 2^15 in-edges or more walks
// every chain in row order, one a thread, with coalesced row reads and chain
// stores. Otherwise the rows below class kGammaMidClass (under 2^10
// in-edges) still go in row order; the longer ones are ordered by class, so
// that the threads of a warp walk chains of similar length (the order within
// a class is arbitrary: rows are independent), and classes from
// kGammaLongClass up run one row a thread in one-warp blocks: such a chain is
// one dependent sequence of up to ~10^6 steps, and a thread walking it among
// warps busy with short rows would wait for issue slots at every step.
constexpr int kGammaClasses = 33;
constexpr int kGammaMidClass = 11;
constexpr int kGammaLongClass = 16;
constexpr int kGammaOrderItems = 8;

__device__ __forceinline__ int row_class(uint32_t deg) { return deg ? 32 - __clz(deg) : 0; }

__global__ void k_row_class_count(const RowInfo* __restrict__ rows, int64_t n,
                                  unsigned long long* __restrict__ cls) {
    __shared__ unsigned int s_c[kGammaClasses];
    if (threadIdx.x < kGammaClasses) s_c[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int c = row_class(rows[v].deg);
        if (c >= kGammaMidClass) atomicAdd(&s_c[c], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kGammaClasses && s_c[threadIdx.x]) atomicAdd(&cls[threadIdx.x], (unsigned long long)s_c[threadIdx.x]);
}

// class counts -> class starts (exclusive, in place); cls[kGammaClasses] =
// the number of ordered rows
__global__ void k_row_class_starts(unsigned long long* __restrict__ cls) {
    unsigned long long run = 0;
    for (int c = 0; c < kGammaClasses; ++c) {
        const unsigned long long x = cls[c];
        cls[c] = run;
        run += x;
    }
    cls[kGammaClasses] = run;
}

// order[cursor[class]++] = v for the rows of classes kGammaMidClass and up,
// the cursors advanced once per class and chunk of 256 x kGammaOrderItems rows
__global__ void __launch_bounds__(256) k_row_class_order(const RowInfo* __restrict__ rows, int64_t n,
                                                         unsigned long long* __restrict__ cursor,
                                                         uint32_t* __restrict__ order) {
    __shared__ unsigned int s_c[kGammaClasses];
    __shared__ unsigned long long s_base[kGammaClasses];
    constexpr int64_t chunk = 256 * kGammaOrderItems;
    for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < n; c0 += (int64_t)gridDim.x * chunk) {
        if (threadIdx.x < kGammaClasses) s_c[threadIdx.x] = 0;
        __syncthreads();
        int cl[kGammaOrderItems];
        unsigned int at[kGammaOrderItems];
#pragma unroll
        for (int i = 0; i < kGammaOrderItems; ++i) {
            const int64_t v = c0 + i * 256 + threadIdx.x;
            cl[i] = v < n ? row_class(rows[v].deg) : -1;
            if (cl[i] < kGammaMidClass) cl[i] = -1;
            at[i] = cl[i] >= 0 ? atomicAdd(&s_c[cl[i]], 1u) : 0;
        }
        __syncthreads();
        if (threadIdx.x < kGammaClasses)
            s_base[threadIdx.x] = s_c[threadIdx.x] ? atomicAdd(&cursor[threadIdx.x], (unsigned long long)s_c[threadIdx.x]) : 0;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kGammaOrderItems; ++i)
            if (cl[i] >= 0) order[s_base[cl[i]] + at[i]] = (uint32_t)(c0 + i * 256 + threadIdx.x);
        __syncthreads();
    }
}

// w_v = (2^62 - Q_d) >> s for the rows below class c_end, in row order
__global__ void k_gamma(const RowInfo* __restrict__ rows, const uint32_t* __restrict__ csr_tau, int64_t n, int s,
                        uint64_t* __restrict__ w, uint64_t* __restrict__ chain, int c_end) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const RowInfo r = rows[v];
        if (row_class(r.deg) < c_end) w[v] = ((1ull << 62) - gamma_row(r, csr_tau, chain)) >> s;
    }
}

// the same for the ordered rows order[starts[c_lo] .. starts[c_hi]); one-warp
// blocks for the long classes
__global__ void k_gamma_ordered(const RowInfo* __restrict__ rows, const uint32_t* __restrict__ csr_tau, int s,
                                uint64_t* __restrict__ w, uint64_t* __restrict__ chain,
                                const uint32_t* __restrict__ order, const unsigned long long* __restrict__ starts,
                                int c_lo, int c_hi) {
    const int64_t lo = (int64_t)starts[c_lo], hi = (int64_t)starts[c_hi];
    for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = order[i];
        w[v] = ((1ull << 62) - gamma_row(rows[v], csr_tau, chain)) >> s;
    }
}

// Linear Threshold model (Sec. "Extensions to other diffusion models"):
// gamma_v = the sum of the row's weights, exactly, as w_v = sum tau' with
// f = 32 (tau' = tau, or 2^32 for the always-live sentinel). A row above 1
// is not an LT instance and flags the input as invalid.
__device__ __forceinline__ uint64_t lt_weight(uint32_t tau) { return tau == kSentinel ? (1ull << 32) : tau; }

__global__ void k_gamma_lt(const RowInfo* __restrict__ rows, const uint32_t* __restrict__ csr_tau, int64_t n,
                           uint64_t* __restrict__ w, DevStatus* status) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const RowInfo r = rows[v];
        uint64_t S = 0;
        if (csr_tau) {
            for (uint32_t k = 0; k < r.deg; ++k) S += lt_weight(csr_tau[r.off + k]);
        } else {
            S = (uint64_t)r.deg * lt_weight(r.tau);
        }
        if (S > (1ull << 32)) {
            atomicOr(&status->flags, kStInval);
            atomicMin(&status->first_bad, (unsigned long long)v);
            S = 0;
        }
        w[v] = S;
    }
}

__global__ void k_lt_weights(const uint32_t* __restrict__ csr_tau, int64_t m, uint64_t* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = lt_weight(csr_tau[e]);
}

// ------------------------------------------------------------- alias table
// Parallel form of the sweeping alias construction (Huebschle-Schneider and
// Sanders, "Parallel Weighted Random Sampling", ESA 2019) in integers.
// Columns hold W; item v has mass w_v n. Light items (mass < W) and heavy
// items are taken in ascending vertex order; D = exclusive prefix sums of the
// light deficits W - mass, E = inclusive prefix sums of the heavy excesses
// mass - W. Light item i aliases the first heavy j with E_j >= D_i. Heavy j
// closes its own column with r = W + E_j - D_c, c = #{i : D_i <= E_j}; if
// r < W it aliases heavy j+1, else r = W and it aliases itself.
__global__ void k_alias_classify(const uint64_t* __restrict__ w, int64_t n, const unsigned long long* __restrict__ dW,
                                 uint32_t* __restrict__ is_light) {
    const uint64_t W = *dW;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        is_light[v] = (w[v] * (uint64_t)n < W) ? 1u : 0u;
}

__global__ void k_alias_compact(const uint64_t* __restrict__ w, int64_t n, const unsigned long long* __restrict__ dW,
                                const uint64_t* __restrict__ light_idx, uint32_t* __restrict__ light_ids,
                                uint32_t* __restrict__ heavy_ids, u128* __restrict__ deficit,
                                u128* __restrict__ excess) {
    const uint64_t W = *dW;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t mass = w[v] * (uint64_t)n;
        const uint64_t li = light_idx[v];
        if (light_idx[v + 1] != li) {  // light
            light_ids[li] = (uint32_t)v;
            deficit[li] = (u128)(W - mass);
        } else {
            const uint64_t hi = (uint64_t)v - li;
            heavy_ids[hi] = (uint32_t)v;
            excess[hi] = (u128)(mass - W);
        }
    }
}

__global__ void k_alias_light(int64_t nl, const uint32_t* __restrict__ light_ids, const uint64_t* __restrict__ w,
                              int64_t n, const u128* __restrict__ D, const u128* __restrict__ Ex, int64_t nh,
                              const uint32_t* __restrict__ heavy_ids, AliasEntry* __restrict__ table) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += (int64_t)gridDim.x * blockDim.x) {
        const u128 target = D[i];
        // first j in [0, nh) with Ex[j+1] >= target (exists: Ex[nh] = D[nl] > D[i])
        int64_t lo = 0, hi = nh - 1;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (Ex[mid + 1] >= target) hi = mid;
            else lo = mid + 1;
        }
        const uint32_t v = light_ids[i];
        AliasEntry a;
        a.prob = w[v] * (uint64_t)n;
        a.alias = heavy_ids[lo];
        a.pad = 0;
        table[v] = a;
    }
}

__global__ void k_alias_heavy(int64_t nh, const uint32_t* __restrict__ heavy_ids, const u128* __restrict__ D,
                              int64_t nl, const u128* __restrict__ Ex, const unsigned long long* __restrict__ dW,
                              AliasEntry* __restrict__ table) {
    const uint64_t W = *dW;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nh; j += (int64_t)gridDim.x * blockDim.x) {
        const u128 E = Ex[j + 1];
        // c = #{i < nl : D[i] <= E}
        int64_t lo = 0, hi = nl;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (D[mid] <= E) lo = mid + 1;
            else hi = mid;
        }
        const u128 r = (u128)W + E - D[lo];
        const uint32_t v = heavy_ids[j];
        AliasEntry a;
        a.pad = 0;
        if (r < (u128)W && j + 1 < nh) {  // j + 1 < nh always holds when sum(mass) = n W
            a.prob = (uint64_t)r;
            a.alias = heavy_ids[j + 1];
        } else {
            a.prob = W;
            a.alias = v;
        }
        table[v] = a;
    }
}

__global__ void k_alias_empty(int64_t n, AliasEntry* __restrict__ table) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        AliasEntry a;
        a.prob = 0;
        a.alias = (uint32_t)v;
        a.pad = 0;
        table[v] = a;
    }
}

static int bits_for(int64_t n) {  // bits needed to hold values 0 .. n-1
    int b = 0;
    while (b < 63 && ((int64_t)1 << b) < n) ++b;
    return b;
}

void graph_release(skis_graph* g) {
    cudaStream_t st = g->stream;
    dev_free(g->off, st);
    dev_free(g->rows, st);
    dev_free(g->src, st);
    dev_free(g->tau, st);
    dev_free(g->perm, st);
    dev_free(g->w, st);
    dev_free(g->alias, st);
    dev_free(g->lt_cum, st);
    dev_free(g->chain, st);
    g->off = nullptr; g->rows = nullptr; g->src = nullptr; g->tau = nullptr;
    g->perm = nullptr; g->w = nullptr; g->alias = nullptr; g->lt_cum = nullptr; g->chain = nullptr;
}

// IC graphs keep the chain from loading (k_gamma, 8 bytes an edge); LT
// graphs have none, and the bucket form does not apply to them.
int graph_ensure_chain(const skis_graph* g, cudaStream_t, std::string* err) {
    if (g->chain || g->m == 0) return SKIS_OK;
    *err = "the bucket form of the first step needs an IC graph (its gamma chain is kept from loading)";
    return SKIS_EINVAL;
}

int graph_build(skis_graph* g, const int32_t* d_src, const int32_t* d_dst, const void* d_weights, int model,
                uint64_t weight_seed, int lt, cudaStream_t st, std::string* err) {
    int rc = SKIS_OK;
    const int64_t n = g->n, m = g->m;
    const int grid = sm_count() * 8, block = 256;
    const int src_bits = bits_for(n);
    // temporaries
    DevStatus* d_status = nullptr;
    unsigned long long* d_W = nullptr;
    uint64_t *keys_a = nullptr, *keys_b = nullptr;
    uint32_t *vals_a = nullptr, *vals_b = nullptr, *csr_dst = nullptr;
    uint32_t *is_light = nullptr, *light_ids = nullptr, *heavy_ids = nullptr;
    uint64_t* light_idx = nullptr;
    u128 *deficit = nullptr, *excess = nullptr, *D = nullptr, *Ex = nullptr;
    DevStatus h_status;
    uint64_t nl = 0, nh = 0;

    g->lt = lt ? 1 : 0;
    g->s = g->lt ? 0 : bits_for(n) + 1;  // ceil(log2 n) + 1
    g->f = g->lt ? 32 : 62 - g->s;
    g->row_uniform = (model == SKIS_W_WC);
    uint64_t* lt_w = nullptr;
    uint32_t* row_order = nullptr;
    unsigned long long* class_starts = nullptr;
    g->m_pad = ((m + 3) / 4) * 4 + 4;

    GB_CUDA(dev_alloc_t(&d_status, 1, st));
    GB_CUDA(dev_alloc_t(&d_W, 1, st));
    GB_CUDA(cudaMemsetAsync(d_status, 0, sizeof(DevStatus), st));
    GB_CUDA(cudaMemsetAsync(&d_status->first_bad, 0xFF, sizeof(unsigned long long), st));

    // validation first: nothing below may index with an unchecked id
    if (m > 0) {
        k_validate<<<grid, block, 0, st>>>(d_src, d_dst, model == SKIS_W_EXPLICIT_P ? (const double*)d_weights : nullptr,
                                           m, n, d_status); note_launch();
        GB_CUDA(cudaGetLastError());
    }
    GB_CUDA(cudaMemcpyAsync(&h_status, d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (h_status.flags & kStInval) {
        *err = "skis_load_graph: invalid edge at input index " + std::to_string(h_status.first_bad) +
               " (vertex id outside [0, n), self-loop, or p outside [0, 1] / NaN)";
        rc = SKIS_EINVAL;
        goto cleanup;
    }

    // canonical in-CSR
    GB_CUDA(dev_alloc_t(&g->off, (size_t)n + 1, st));
    GB_CUDA(dev_alloc_t(&g->rows, (size_t)n, st));
    GB_CUDA(dev_alloc_t(&g->src, (size_t)g->m_pad, st));
    GB_CUDA(dev_alloc_t(&g->perm, (size_t)(m > 0 ? m : 1), st));
    if (!g->row_uniform) GB_CUDA(dev_alloc_t(&g->tau, (size_t)g->m_pad, st));
    GB_CUDA(dev_alloc_t(&g->w, (size_t)n, st));
    GB_CUDA(dev_alloc_t(&g->alias, (size_t)n, st));
    if (m > 0) {
        GB_CUDA(dev_alloc_t(&keys_a, (size_t)m, st));
        GB_CUDA(dev_alloc_t(&keys_b, (size_t)m, st));
        GB_CUDA(dev_alloc_t(&vals_a, (size_t)m, st));
        GB_CUDA(dev_alloc_t(&vals_b, (size_t)m, st));
        GB_CUDA(dev_alloc_t(&csr_dst, (size_t)m, st));
        GB_CUDA(sort_edges(d_src, d_dst, m, src_bits, g->src, csr_dst, g->perm, keys_a, vals_a, keys_b, vals_b,
                           &d_status->gave_up, st));
    }
    k_offsets_from_dst<<<grid, block, 0, st>>>(csr_dst, m, n, g->off); note_launch();
    GB_CUDA(cudaGetLastError());
    // padding positions (m .. m_pad) get source 0 and, with per-edge models, threshold 0 (never live)
    GB_CUDA(cudaMemsetAsync(g->src + m, 0, (size_t)(g->m_pad - m) * sizeof(int32_t), st));
    if (g->tau) {
        k_edge_tau<<<grid, block, 0, st>>>(g->perm, m, g->m_pad, model, d_weights, weight_seed, g->tau); note_launch();
        GB_CUDA(cudaGetLastError());
    }
    k_rows<<<grid, block, 0, st>>>(g->off, n, g->row_uniform, g->rows); note_launch();
    GB_CUDA(cudaGetLastError());

    // gamma in fixed point and W
    if (g->lt) {
        k_gamma_lt<<<grid, block, 0, st>>>(g->rows, g->tau, n, g->w, d_status); note_launch();
        GB_CUDA(cudaGetLastError());
        GB_CUDA(cudaMemcpyAsync(&h_status, d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        if (h_status.flags & kStInval) {
            *err = "skis_load_graph_lt: the in-edge weights of vertex " + std::to_string(h_status.first_bad) +
                   " sum above 1 (not a Linear Threshold instance)";
            rc = SKIS_EINVAL;
            goto cleanup;
        }
        if (!g->row_uniform && m > 0) {  // running sums for the walk's edge choice
            GB_CUDA(dev_alloc_t(&lt_w, (size_t)m, st));
            GB_CUDA(dev_alloc_t(&g->lt_cum, (size_t)m + 1, st));
            k_lt_weights<<<grid, block, 0, st>>>(g->tau, m, lt_w); note_launch();
            GB_CUDA(cudaGetLastError());
            GB_CUDA(scan_u64(lt_w, g->lt_cum, m, st));
        }
    } else {
        // the chain is kept for the bucket form of the first step (8 bytes an edge)
        if (m > 0) GB_CUDA(dev_alloc_t(&g->chain, (size_t)m, st));
        // the rows' degree classes; with no long row, every chain in row
        // order; else the short chains in row order, then the ordered
        // middle classes, then the long rows
        unsigned long long h_starts[kGammaClasses + 1];
        GB_CUDA(dev_alloc_t(&class_starts, (size_t)2 * (kGammaClasses + 1), st));
        unsigned long long* class_cursor = class_starts + kGammaClasses + 1;
        GB_CUDA(cudaMemsetAsync(class_starts, 0, (kGammaClasses + 1) * sizeof(unsigned long long), st));
        k_row_class_count<<<grid, block, 0, st>>>(g->rows, n, class_starts); note_launch();
        k_row_class_starts<<<1, 1, 0, st>>>(class_starts); note_launch();
        GB_CUDA(cudaMemcpyAsync(h_starts, class_starts, sizeof(h_starts), cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        if (h_starts[kGammaLongClass] == h_starts[kGammaClasses]) {
            k_gamma<<<grid, block, 0, st>>>(g->rows, g->tau, n, g->s, g->w, g->chain, kGammaClasses); note_launch();
        } else {
            GB_CUDA(dev_alloc_t(&row_order, (size_t)h_starts[kGammaClasses], st));
            GB_CUDA(cudaMemcpyAsync(class_cursor, class_starts, (kGammaClasses + 1) * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToDevice, st));
            k_row_class_order<<<grid, 256, 0, st>>>(g->rows, n, class_cursor, row_order); note_launch();
            k_gamma<<<grid, block, 0, st>>>(g->rows, g->tau, n, g->s, g->w, g->chain, kGammaMidClass); note_launch();
            k_gamma_ordered<<<grid, block, 0, st>>>(g->rows, g->tau, g->s, g->w, g->chain, row_order, class_starts,
                                                    kGammaMidClass, kGammaLongClass); note_launch();
            k_gamma_ordered<<<sm_count() * 4, 32, 0, st>>>(g->rows, g->tau, g->s, g->w, g->chain, row_order,
                                                           class_starts, kGammaLongClass, kGammaClasses); note_launch();
        }
        GB_CUDA(cudaGetLastError());
    }
    GB_CUDA(sum_u64(g->w, n, d_W, st));

    // alias table
    GB_CUDA(dev_alloc_t(&is_light, (size_t)n, st));
    GB_CUDA(dev_alloc_t(&light_idx, (size_t)n + 1, st));
    k_alias_classify<<<grid, block, 0, st>>>(g->w, n, d_W, is_light); note_launch();
    GB_CUDA(cudaGetLastError());
    GB_CUDA(scan_u32_to_u64(is_light, light_idx, n, st));
    GB_CUDA(cudaMemcpyAsync(&nl, light_idx + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(&g->W, d_W, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(&h_status, d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (h_status.gave_up) {
        *err = "skis_load_graph: the edge sort failed an internal check (look-back wait or output bounds)";
        rc = SKIS_ERR_INTERNAL;
        goto cleanup;
    }
    nh = (uint64_t)n - nl;
    if (g->W == 0) {
        k_alias_empty<<<grid, block, 0, st>>>(n, g->alias); note_launch();
        GB_CUDA(cudaGetLastError());
    } else {
        GB_CUDA(dev_alloc_t(&light_ids, (size_t)nl + 1, st));
        GB_CUDA(dev_alloc_t(&heavy_ids, (size_t)nh + 1, st));
        GB_CUDA(dev_alloc_t(&deficit, (size_t)nl + 1, st));
        GB_CUDA(dev_alloc_t(&excess, (size_t)nh + 1, st));
        GB_CUDA(dev_alloc_t(&D, (size_t)nl + 1, st));
        GB_CUDA(dev_alloc_t(&Ex, (size_t)nh + 1, st));
        k_alias_compact<<<grid, block, 0, st>>>(g->w, n, d_W, light_idx, light_ids, heavy_ids, deficit, excess); note_launch();
        GB_CUDA(cudaGetLastError());
        GB_CUDA(scan_u128(deficit, D, (int64_t)nl, st));
        GB_CUDA(scan_u128(excess, Ex, (int64_t)nh, st));
        if (nl > 0) {
            k_alias_light<<<grid, block, 0, st>>>((int64_t)nl, light_ids, g->w, n, D, Ex, (int64_t)nh, heavy_ids,
                                                  g->alias); note_launch();
            GB_CUDA(cudaGetLastError());
        }
        k_alias_heavy<<<grid, block, 0, st>>>((int64_t)nh, heavy_ids, D, (int64_t)nl, Ex, d_W, g->alias); note_launch();
        GB_CUDA(cudaGetLastError());
    }
    GB_CUDA(cudaStreamSynchronize(st));

cleanup:
    dev_free(lt_w, st);
    dev_free(row_order, st);
    dev_free(class_starts, st);
    dev_free(d_status, st);
    dev_free(d_W, st);
    dev_free(keys_a, st);
    dev_free(keys_b, st);
    dev_free(vals_a, st);
    dev_free(vals_b, st);
    dev_free(csr_dst, st);
    dev_free(is_light, st);
    dev_free(light_idx, st);
    dev_free(light_ids, st);
    dev_free(heavy_ids, st);
    dev_free(deficit, st);
    dev_free(excess, st);
    dev_free(D, st);
    dev_free(Ex, st);
    if (rc != SKIS_OK) graph_release(g);
    return rc;
}

}  // namespace skis
