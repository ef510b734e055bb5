// C ABI of the SKIS GB300 library (declared in include/skis.h): argument
// checks, host<->device marshalling, handle lifetime and error reporting.
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/skis.h"
#include "skis_internal.cuh"

using namespace skis;

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int skis::set_last_error(int code, const std::string& msg) { return fail(code, msg); }

static int cuda_fail(const char* where, cudaError_t e) {
    return fail(e == cudaErrorMemoryAllocation ? SKIS_ENOMEM : SKIS_ERR_CUDA,
                std::string(where) + ": CUDA error: " + cudaGetErrorString(e));
}

#define API_TRY try {
#define API_CATCH                                                       \
    }                                                                   \
    catch (const std::bad_alloc&) {                                     \
        return fail(SKIS_ENOMEM, "host allocation failed");             \
    }                                                                   \
    catch (...) {                                                       \
        return fail(SKIS_ERR_CUDA, "unexpected exception in library");  \
    }

#define API_CUDA(where, call)                          \
    do {                                               \
        cudaError_t _e = (call);                       \
        if (_e != cudaSuccess) return cuda_fail(where, _e); \
    } while (0)

// ------------------------------------------------------------------ graph
static int load_graph(skis_graph** out, int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                      const void* weights, int weight_model, uint64_t weight_seed, int mem_space, int lt,
                      void* cuda_stream) {
    API_TRY
    if (!out) return fail(SKIS_EINVAL, "skis_load_graph: out is NULL");
    *out = nullptr;
    if (n < 1 || n > (int64_t(1) << 31)) return fail(SKIS_EINVAL, "skis_load_graph: n must be in [1, 2^31]");
    if (m < 0 || m >= (int64_t(1) << 32) - 8) return fail(SKIS_EINVAL, "skis_load_graph: m must be in [0, 2^32 - 8)");
    if (m > 0 && (!src || !dst)) return fail(SKIS_EINVAL, "skis_load_graph: src/dst are NULL");
    if (weight_model < SKIS_W_EXPLICIT_P || weight_model > SKIS_W_TRI)
        return fail(SKIS_EINVAL, "skis_load_graph: unknown weight model");
    const bool need_w = weight_model == SKIS_W_EXPLICIT_P || weight_model == SKIS_W_EXPLICIT_TAU;
    if (need_w && m > 0 && !weights) return fail(SKIS_EINVAL, "skis_load_graph: weights are NULL");
    if (mem_space != SKIS_MEM_HOST && mem_space != SKIS_MEM_DEVICE)
        return fail(SKIS_EINVAL, "skis_load_graph: bad mem_space");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t wbytes = weight_model == SKIS_W_EXPLICIT_P ? sizeof(double) : sizeof(uint32_t);

    const int32_t* d_src = src;
    const int32_t* d_dst = dst;
    const void* d_w = need_w ? weights : nullptr;
    int32_t *t_src = nullptr, *t_dst = nullptr;
    void* t_w = nullptr;
    if (mem_space == SKIS_MEM_HOST && m > 0) {
        API_CUDA("skis_load_graph", dev_alloc_t(&t_src, (size_t)m, st));
        API_CUDA("skis_load_graph", dev_alloc_t(&t_dst, (size_t)m, st));
        API_CUDA("skis_load_graph", cudaMemcpyAsync(t_src, src, (size_t)m * 4, cudaMemcpyHostToDevice, st));
        API_CUDA("skis_load_graph", cudaMemcpyAsync(t_dst, dst, (size_t)m * 4, cudaMemcpyHostToDevice, st));
        if (need_w) {
            API_CUDA("skis_load_graph", dev_alloc(&t_w, (size_t)m * wbytes, st));
            API_CUDA("skis_load_graph", cudaMemcpyAsync(t_w, weights, (size_t)m * wbytes, cudaMemcpyHostToDevice, st));
        }
        d_src = t_src;
        d_dst = t_dst;
        d_w = t_w;
    }
    skis_graph* g = new skis_graph();
    g->n = n;
    g->m = m;
    g->stream = st;
    std::string err;
    const int rc = graph_build(g, d_src, d_dst, d_w, weight_model, weight_seed, lt, st, &err);
    dev_free(t_src, st);
    dev_free(t_dst, st);
    dev_free(t_w, st);
    if (rc != SKIS_OK) {
        delete g;
        return fail(rc, err);
    }
    *out = g;
    return SKIS_OK;
    API_CATCH
}

extern "C" int skis_load_graph(skis_graph** out, int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                               const void* weights, int weight_model, uint64_t weight_seed, int mem_space,
                               void* cuda_stream) {
    return load_graph(out, n, m, src, dst, weights, weight_model, weight_seed, mem_space, 0, cuda_stream);
}

extern "C" int skis_load_graph_lt(skis_graph** out, int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                  const void* weights, int weight_model, uint64_t weight_seed, int mem_space,
                                  void* cuda_stream) {
    return load_graph(out, n, m, src, dst, weights, weight_model, weight_seed, mem_space, 1, cuda_stream);
}

extern "C" int skis_graph_get_info(const skis_graph* g, skis_graph_info* info) {
    if (!g || !info) return fail(SKIS_EINVAL, "skis_graph_get_info: NULL argument");
    info->n = g->n;
    info->m = g->m;
    info->W = g->W;
    info->f = g->f;
    info->row_uniform_tau = g->row_uniform;
    info->Gamma = (double)g->W / (double)(1ull << g->f);
    info->diffusion = g->lt ? SKIS_DIFF_LT : SKIS_DIFF_IC;
    return SKIS_OK;
}

extern "C" int skis_graph_export(const skis_graph* g, int64_t* offsets, int32_t* csr_src, uint32_t* tau,
                                 int64_t* perm, uint64_t* w, uint64_t* prob, uint32_t* alias, void* cuda_stream) {
    API_TRY
    if (!g) return fail(SKIS_EINVAL, "skis_graph_export: NULL graph");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t n = g->n, m = g->m;
    std::vector<uint64_t> off((size_t)n + 1);
    API_CUDA("skis_graph_export", cudaMemcpyAsync(off.data(), g->off, (n + 1) * 8, cudaMemcpyDeviceToHost, st));
    if (csr_src && m)
        API_CUDA("skis_graph_export", cudaMemcpyAsync(csr_src, g->src, m * 4, cudaMemcpyDeviceToHost, st));
    std::vector<uint32_t> p32;
    if (perm && m) {
        p32.resize((size_t)m);
        API_CUDA("skis_graph_export", cudaMemcpyAsync(p32.data(), g->perm, m * 4, cudaMemcpyDeviceToHost, st));
    }
    std::vector<RowInfo> rows;
    if (tau && m) {
        if (g->row_uniform) {
            rows.resize((size_t)n);
            API_CUDA("skis_graph_export",
                     cudaMemcpyAsync(rows.data(), g->rows, n * sizeof(RowInfo), cudaMemcpyDeviceToHost, st));
        } else {
            API_CUDA("skis_graph_export", cudaMemcpyAsync(tau, g->tau, m * 4, cudaMemcpyDeviceToHost, st));
        }
    }
    if (w) API_CUDA("skis_graph_export", cudaMemcpyAsync(w, g->w, n * 8, cudaMemcpyDeviceToHost, st));
    std::vector<AliasEntry> tab;
    if (prob || alias) {
        tab.resize((size_t)n);
        API_CUDA("skis_graph_export",
                 cudaMemcpyAsync(tab.data(), g->alias, n * sizeof(AliasEntry), cudaMemcpyDeviceToHost, st));
    }
    API_CUDA("skis_graph_export", cudaStreamSynchronize(st));
    if (offsets)
        for (int64_t i = 0; i <= n; ++i) offsets[i] = (int64_t)off[i];
    if (perm)
        for (int64_t e = 0; e < m; ++e) perm[e] = (int64_t)p32[e];
    if (tau && m && g->row_uniform)
        for (int64_t v = 0; v < n; ++v)
            for (uint64_t e = off[v]; e < off[v + 1]; ++e) tau[e] = rows[v].tau;
    for (int64_t v = 0; v < n && (prob || alias); ++v) {
        if (prob) prob[v] = tab[v].prob;
        if (alias) alias[v] = tab[v].alias;
    }
    return SKIS_OK;
    API_CATCH
}

extern "C" void skis_graph_free(skis_graph* g) {
    if (!g) return;
    graph_release(g);
    delete g;
}

// ----------------------------------------------------------------- sketch
extern "C" int skis_sketch_create(skis_sketch** out, const skis_graph* g, uint64_t seed, uint64_t arena_entries,
                                  void* cuda_stream) {
    API_TRY
    if (!out || !g) return fail(SKIS_EINVAL, "skis_sketch_create: NULL argument");
    skis_sketch* s = new skis_sketch();
    s->g = g;
    s->seed = seed;
    s->arena_hint = arena_entries;
    s->stream = (cudaStream_t)cuda_stream;
    *out = s;
    return SKIS_OK;
    API_CATCH
}

extern "C" int skis_sketch_set_option(skis_sketch* s, int option, uint64_t value) {
    if (!s) return fail(SKIS_EINVAL, "skis_sketch_set_option: NULL sketch");
    switch (option) {
        case SKIS_OPT_RETRY_CAP:
            if (value < 1 || value > (1u << 24)) return fail(SKIS_EINVAL, "retry cap must be in [1, 2^24]");
            s->retry_cap = (uint32_t)value;
            return SKIS_OK;
        case SKIS_OPT_CTA_SLOTS:
            if (value > 65535) return fail(SKIS_EINVAL, "CTA slots must be at most 65535");
            s->cta_slots = (int)value;
            return SKIS_OK;
        case SKIS_OPT_WARP_BLOCKS:
            if (value > (1u << 20)) return fail(SKIS_EINVAL, "warp blocks must be at most 2^20");
            s->warp_blocks = (int)value;
            return SKIS_OK;
        case SKIS_OPT_THREAD_MAX_DEG:
            if (value > (1u << 30)) return fail(SKIS_EINVAL, "thread-tier degree limit must be at most 2^30");
            s->thread_max_deg = (uint32_t)value;
            return SKIS_OK;
        case SKIS_OPT_THREAD_MAX_STEPS:
            if (value < 1 || value > (1u << 30)) return fail(SKIS_EINVAL, "thread-tier step budget must be in [1, 2^30]");
            s->thread_max_steps = (uint32_t)value;
            return SKIS_OK;
        case SKIS_OPT_FIRST_STEP:
            if (value > 1) return fail(SKIS_EINVAL, "first step must be 0 (rejection) or 1 (bucket)");
            if (s->T != 0) return fail(SKIS_EINVAL, "the first-step form is chosen before the first sample");
            s->bucket = (int)value;
            return SKIS_OK;
        case SKIS_OPT_THREAD_MAX_RETRIES:
            if (value < 1 || value > (1u << 24)) return fail(SKIS_EINVAL, "thread-tier retry limit must be in [1, 2^24]");
            s->thread_max_retries = (uint32_t)value;
            return SKIS_OK;
        case SKIS_OPT_WARP_MAX_COINS:
            if (value < 1 || value > (1u << 31)) return fail(SKIS_EINVAL, "warp-tier coin budget must be in [1, 2^31]");
            s->warp_max_coins = (uint32_t)value;
            return SKIS_OK;
        case SKIS_OPT_CTA_HUB_QUADS:
            if (value > (1u << 30)) return fail(SKIS_EINVAL, "CTA-tier hub threshold must be at most 2^30 quads");
            s->cta_hub_quads = (uint32_t)value;
            return SKIS_OK;
        case SKIS_OPT_CTA_QUEUE_CAP:
            if (value < 32 || value > (1ull << 31)) return fail(SKIS_EINVAL, "CTA-tier queue capacity must be in [32, 2^31]");
            s->cta_queue_cap = (uint32_t)value;
            return SKIS_OK;
        case SKIS_OPT_CTA_THREADS:
            if (value != 256 && value != 512) return fail(SKIS_EINVAL, "CTA-tier block size must be 256 or 512");
            s->cta_threads = (int)value;
            return SKIS_OK;
        case SKIS_OPT_FIRST_ID:
            if (value > (1ull << 62)) return fail(SKIS_EINVAL, "first sample id must be at most 2^62");
            if (s->T != 0) return fail(SKIS_EINVAL, "the first sample id is chosen before the first sample");
            s->id_base = value;
            return SKIS_OK;
        case SKIS_OPT_SAMPLER:
            if (value > 1) return fail(SKIS_EINVAL, "sampler must be 0 (IIS) or 1 (RIS)");
            if (s->T != 0) return fail(SKIS_EINVAL, "the sampler is chosen before the first sample");
            s->ris = (int)value;
            return SKIS_OK;
        case SKIS_OPT_QUERY_INDEX:
            if (value > 3) return fail(SKIS_EINVAL, "query-index mode must be 0, 1, 2 or 3");
            s->query_index = (int)value;
            return SKIS_OK;
        case SKIS_OPT_THREAD_BLOCKS:
            if (value > (1u << 20)) return fail(SKIS_EINVAL, "thread blocks must be at most 2^20");
            s->thread_blocks = (int)value;
            return SKIS_OK;
        default:
            return fail(SKIS_EINVAL, "skis_sketch_set_option: unknown option");
    }
}

extern "C" int skis_sample(skis_sketch* s, uint64_t count, uint64_t* next_sample_id_out, void* cuda_stream) {
    API_TRY
    if (!s) return fail(SKIS_EINVAL, "skis_sample: NULL sketch");
    if (count > (1ull << 40)) return fail(SKIS_EINVAL, "skis_sample: count too large");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->stream = st;
    std::string err;
    const int rc = sketch_sample(s, count, st, &err);
    if (next_sample_id_out) *next_sample_id_out = s->id_base + s->T;
    if (rc != SKIS_OK) return fail(rc, err);
    return SKIS_OK;
    API_CATCH
}

extern "C" int skis_sample_to_size(skis_sketch* s, uint64_t target_entries, uint64_t max_count,
                                   uint64_t* appended_out, uint64_t* next_sample_id_out, void* cuda_stream) {
    API_TRY
    if (!s) return fail(SKIS_EINVAL, "skis_sample_to_size: NULL sketch");
    if (target_entries < 1) return fail(SKIS_EINVAL, "skis_sample_to_size: target_entries must be >= 1");
    if (max_count > (1ull << 40)) return fail(SKIS_EINVAL, "skis_sample_to_size: max_count too large");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->stream = st;
    std::string err;
    uint64_t appended = 0;
    const int rc = sketch_sample_to_size(s, target_entries, max_count, st, &appended, &err);
    if (appended_out) *appended_out = appended;
    if (next_sample_id_out) *next_sample_id_out = s->id_base + s->T;
    if (rc != SKIS_OK) return fail(rc, err);
    return SKIS_OK;
    API_CATCH
}

extern "C" int skis_sketch_autotune(skis_sketch* s, uint64_t pilot_samples, uint32_t* chosen_max_deg,
                                    uint32_t* chosen_max_steps, double* candidate_ms, int32_t candidate_cap,
                                    int32_t* candidates_out, void* cuda_stream) {
    API_TRY
    if (!s) return fail(SKIS_EINVAL, "skis_sketch_autotune: NULL sketch");
    if (pilot_samples < 1 || pilot_samples > (1ull << 32))
        return fail(SKIS_EINVAL, "skis_sketch_autotune: pilot_samples must be in [1, 2^32]");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->stream = st;
    std::string err;
    int nc = 0;
    const int rc = sketch_autotune(s, pilot_samples, st, candidate_ms, candidate_cap, &nc, &err);
    if (candidates_out) *candidates_out = nc;
    if (rc != SKIS_OK) return fail(rc, "skis_sketch_autotune: " + err);
    if (chosen_max_deg) *chosen_max_deg = s->thread_max_deg;
    if (chosen_max_steps) *chosen_max_steps = s->thread_max_steps;
    return SKIS_OK;
    API_CATCH
}

// skis_estimate and skis_estimate_sharded (exch != NULL): argument checks
// and host <-> device marshalling around the device computation.
static int estimate_call(const char* name, skis_sketch* s, int32_t num_queries, const int64_t* seed_offsets,
                         const int32_t* seeds, int64_t* coverage_out, double* estimate_out, int mem_space,
                         int64_t* exch, skis_allreduce_fn fn, void* ctx, void* cuda_stream) {
    const std::string where(name);
    if (!s || !seed_offsets || !estimate_out) return fail(SKIS_EINVAL, where + ": NULL argument");
    if (num_queries < 0) return fail(SKIS_EINVAL, where + ": negative query count");
    if (mem_space != SKIS_MEM_HOST && mem_space != SKIS_MEM_DEVICE) return fail(SKIS_EINVAL, where + ": bad mem_space");
    if (num_queries == 0) return SKIS_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->stream = st;
    // offsets are checked on the host in both memory spaces
    std::vector<int64_t> off((size_t)num_queries + 1);
    if (mem_space == SKIS_MEM_HOST) {
        std::copy(seed_offsets, seed_offsets + num_queries + 1, off.begin());
    } else {
        API_CUDA(name, cudaMemcpyAsync(off.data(), seed_offsets, (num_queries + 1) * 8, cudaMemcpyDeviceToHost, st));
        API_CUDA(name, cudaStreamSynchronize(st));
    }
    if (off[0] < 0) return fail(SKIS_EINVAL, where + ": negative seed offset");
    for (int32_t b = 0; b < num_queries; ++b)
        if (off[b + 1] < off[b]) return fail(SKIS_EINVAL, where + ": seed offsets decrease");
    if (off[num_queries] > 0 && !seeds) return fail(SKIS_EINVAL, where + ": seeds is NULL");
    std::string err;
    auto run = [&](const int64_t* d_off, const int32_t* d_seeds, int64_t* d_cov, double* d_est) {
        return exch ? sketch_estimate_sharded(s, num_queries, d_off, d_seeds, off.data(), d_cov, d_est, exch, fn, ctx,
                                              st, &err)
                    : sketch_estimate(s, num_queries, d_off, d_seeds, off.data(), d_cov, d_est, st, &err);
    };
    int rc;
    if (mem_space == SKIS_MEM_DEVICE) {
        rc = run(seed_offsets, seeds, coverage_out, estimate_out);
    } else {
        const int64_t nseeds = off[num_queries];
        int64_t* d_off = nullptr;
        int32_t* d_seeds = nullptr;
        int64_t* d_cov = nullptr;
        double* d_est = nullptr;
        API_CUDA(name, dev_alloc_t(&d_off, (size_t)num_queries + 1, st));
        API_CUDA(name, dev_alloc_t(&d_seeds, (size_t)std::max<int64_t>(nseeds, 1), st));
        API_CUDA(name, dev_alloc_t(&d_cov, (size_t)num_queries, st));
        API_CUDA(name, dev_alloc_t(&d_est, (size_t)num_queries, st));
        API_CUDA(name, cudaMemcpyAsync(d_off, off.data(), (num_queries + 1) * 8, cudaMemcpyHostToDevice, st));
        if (nseeds) API_CUDA(name, cudaMemcpyAsync(d_seeds, seeds, nseeds * 4, cudaMemcpyHostToDevice, st));
        rc = run(d_off, d_seeds, d_cov, d_est);
        if (rc == SKIS_OK) {
            if (coverage_out)
                API_CUDA(name, cudaMemcpyAsync(coverage_out, d_cov, num_queries * 8, cudaMemcpyDeviceToHost, st));
            API_CUDA(name, cudaMemcpyAsync(estimate_out, d_est, num_queries * 8, cudaMemcpyDeviceToHost, st));
            API_CUDA(name, cudaStreamSynchronize(st));
        }
        dev_free(d_off, st);
        dev_free(d_seeds, st);
        dev_free(d_cov, st);
        dev_free(d_est, st);
    }
    if (rc != SKIS_OK) return fail(rc, err);
    return SKIS_OK;
}

extern "C" int skis_estimate(skis_sketch* s, int32_t num_queries, const int64_t* seed_offsets, const int32_t* seeds,
                             int64_t* coverage_out, double* estimate_out, int mem_space, void* cuda_stream) {
    API_TRY
    return estimate_call("skis_estimate", s, num_queries, seed_offsets, seeds, coverage_out, estimate_out, mem_space,
                         nullptr, nullptr, nullptr, cuda_stream);
    API_CATCH
}

extern "C" int skis_estimate_sharded(skis_sketch* s, int32_t num_queries, const int64_t* seed_offsets,
                                     const int32_t* seeds, int64_t* coverage_out, double* estimate_out, int mem_space,
                                     int64_t* exchange, skis_allreduce_fn allreduce, void* ctx, void* cuda_stream) {
    API_TRY
    if (!exchange || !allreduce) return fail(SKIS_EINVAL, "skis_estimate_sharded: NULL exchange or all-reduce");
    if (s && num_queries > 0 && s->T == 0)
        return fail(SKIS_EINVAL, "skis_estimate_sharded: every rank's sketch must hold a sample");
    return estimate_call("skis_estimate_sharded", s, num_queries, seed_offsets, seeds, coverage_out, estimate_out,
                         mem_space, exchange, allreduce, ctx, cuda_stream);
    API_CATCH
}

extern "C" int skis_greedy_maxcover(skis_sketch* s, int32_t k, int32_t* seeds_out, int64_t* coverage_out,
                                    double* estimate_out, void* cuda_stream) {
    API_TRY
    if (!s || (k > 0 && !seeds_out)) return fail(SKIS_EINVAL, "skis_greedy_maxcover: NULL argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->stream = st;
    std::string err;
    const int rc = sketch_greedy(s, k, seeds_out, coverage_out, estimate_out, st, &err);
    if (rc != SKIS_OK) return fail(rc, err);
    return SKIS_OK;
    API_CATCH
}

extern "C" int skis_greedy_maxcover_sharded(skis_sketch* s, int32_t k, int32_t* seeds_out, int64_t* coverage_out,
                                            double* estimate_out, int64_t* exchange, skis_allreduce_fn allreduce,
                                            void* ctx, void* cuda_stream) {
    API_TRY
    if (!s || (k > 0 && !seeds_out)) return fail(SKIS_EINVAL, "skis_greedy_maxcover_sharded: NULL argument");
    if (!exchange || !allreduce) return fail(SKIS_EINVAL, "skis_greedy_maxcover_sharded: NULL exchange or all-reduce");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->stream = st;
    std::string err;
    const int rc = sketch_greedy_sharded(s, k, seeds_out, coverage_out, estimate_out, exchange, allreduce, ctx, st, &err);
    if (rc != SKIS_OK) return fail(rc, err);
    return SKIS_OK;
    API_CATCH
}

// Per-sample header sums for statistics.
__global__ void k_header_sums(const uint32_t* __restrict__ len, const uint64_t* __restrict__ coins,
                              const uint32_t* __restrict__ retries, uint64_t T, unsigned long long* out) {
    unsigned long long a = 0, b = 0, c = 0;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < T; j += (uint64_t)gridDim.x * blockDim.x) {
        a += len[j];
        b += coins[j];
        c += retries[j];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a += __shfl_down_sync(kFull, a, d);
        b += __shfl_down_sync(kFull, b, d);
        c += __shfl_down_sync(kFull, c, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], a);
        atomicAdd(&out[1], b);
        atomicAdd(&out[2], c);
    }
}

extern "C" int skis_sketch_stats(const skis_sketch* s, skis_stats* out) {
    API_TRY
    if (!s || !out) return fail(SKIS_EINVAL, "skis_sketch_stats: NULL argument");
    std::fill((char*)out, (char*)out + sizeof(skis_stats), 0);
    out->T = s->T;
    out->arena_capacity = s->arena_cap;
    out->to_warp = s->last_to_warp;
    out->deferred = s->last_deferred;
    out->last_thread_ms = s->last_thread_ms;
    out->last_warp_ms = s->last_warp_ms;
    out->last_cta_ms = s->last_cta_ms;
    out->last_sample_ms = s->last_sample_ms;
    out->last_passes = s->last_passes;
    out->thread_max_deg = s->thread_max_deg;
    out->thread_max_steps = s->thread_max_steps;
    out->warp_max_coins = s->warp_max_coins;
    out->cta_hub_quads = s->cta_hub_quads;
    out->first_id = s->id_base;
    out->last_query_ms = s->last_query_ms;
    if (s->T == 0) return SKIS_OK;
    cudaStream_t st = s->stream;
    unsigned long long* d = nullptr;
    unsigned long long h[3] = {0, 0, 0};
    unsigned long long reserved = 0;
    API_CUDA("skis_sketch_stats", dev_alloc_t(&d, 3, st));
    API_CUDA("skis_sketch_stats", cudaMemsetAsync(d, 0, 3 * sizeof(unsigned long long), st));
    const int blocks = (int)std::min<uint64_t>((uint64_t)sm_count() * 4, (s->T + 255) / 256);
    k_header_sums<<<blocks, 256, 0, st>>>(s->h_len, s->h_coins, s->h_retries, s->T, d); note_launch();
    API_CUDA("skis_sketch_stats", cudaGetLastError());
    API_CUDA("skis_sketch_stats", cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    API_CUDA("skis_sketch_stats",
             cudaMemcpyAsync(&reserved, &s->ctr->arena, sizeof(reserved), cudaMemcpyDeviceToHost, st));
    API_CUDA("skis_sketch_stats", cudaStreamSynchronize(st));
    dev_free(d, st);
    out->entries = h[0];
    out->coins = h[1];
    out->retries = h[2];
    out->arena_reserved = reserved;
    return SKIS_OK;
    API_CATCH
}

__global__ void k_gather_members(const uint64_t* __restrict__ h_off, const uint32_t* __restrict__ h_len,
                                 uint64_t first, uint64_t count, const int64_t* __restrict__ out_off,
                                 const int32_t* __restrict__ arena, int32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; t < count; t += nwarps) {
        const uint64_t o = h_off[first + t];
        const uint32_t L = h_len[first + t];
        const int64_t dst = out_off[t];
        for (uint32_t i = lane; i < L; i += 32) out[dst + i] = arena[o + i];
    }
}

extern "C" int skis_sketch_export(const skis_sketch* s, uint64_t first_id, uint64_t count, int32_t* src,
                                  uint32_t* retries, uint32_t* len, uint64_t* coins, int64_t* member_offsets,
                                  int32_t* members, uint64_t members_cap, void* cuda_stream) {
    API_TRY
    if (!s) return fail(SKIS_EINVAL, "skis_sketch_export: NULL sketch");
    if (first_id < s->id_base || first_id - s->id_base > s->T || count > s->T - (first_id - s->id_base))
        return fail(SKIS_EINVAL, "skis_sketch_export: range outside the sketch");
    first_id -= s->id_base;  // header position
    if (count == 0) {
        if (member_offsets) member_offsets[0] = 0;
        return SKIS_OK;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<uint32_t> L((size_t)count);
    API_CUDA("skis_sketch_export", cudaMemcpyAsync(L.data(), s->h_len + first_id, count * 4, cudaMemcpyDeviceToHost, st));
    if (src) API_CUDA("skis_sketch_export", cudaMemcpyAsync(src, s->h_src + first_id, count * 4, cudaMemcpyDeviceToHost, st));
    if (retries)
        API_CUDA("skis_sketch_export",
                 cudaMemcpyAsync(retries, s->h_retries + first_id, count * 4, cudaMemcpyDeviceToHost, st));
    if (coins)
        API_CUDA("skis_sketch_export", cudaMemcpyAsync(coins, s->h_coins + first_id, count * 8, cudaMemcpyDeviceToHost, st));
    API_CUDA("skis_sketch_export", cudaStreamSynchronize(st));
    if (len) std::copy(L.begin(), L.end(), len);
    std::vector<int64_t> mo((size_t)count + 1);
    mo[0] = 0;
    for (uint64_t t = 0; t < count; ++t) mo[t + 1] = mo[t] + L[t];
    if (member_offsets) std::copy(mo.begin(), mo.end(), member_offsets);
    if (!members) return SKIS_OK;
    const uint64_t total = (uint64_t)mo[count];
    if (total > members_cap) return fail(SKIS_EINVAL, "skis_sketch_export: members_cap too small");
    int64_t* d_mo = nullptr;
    int32_t* d_out = nullptr;
    API_CUDA("skis_sketch_export", dev_alloc_t(&d_mo, (size_t)count + 1, st));
    API_CUDA("skis_sketch_export", dev_alloc_t(&d_out, (size_t)std::max<uint64_t>(total, 1), st));
    API_CUDA("skis_sketch_export", cudaMemcpyAsync(d_mo, mo.data(), (count + 1) * 8, cudaMemcpyHostToDevice, st));
    const int blocks = (int)std::min<uint64_t>((uint64_t)sm_count() * 8, (count + 7) / 8);
    k_gather_members<<<blocks, 256, 0, st>>>(s->h_off, s->h_len, first_id, count, d_mo, s->arena, d_out); note_launch();
    API_CUDA("skis_sketch_export", cudaGetLastError());
    if (total)
        API_CUDA("skis_sketch_export", cudaMemcpyAsync(members, d_out, total * 4, cudaMemcpyDeviceToHost, st));
    API_CUDA("skis_sketch_export", cudaStreamSynchronize(st));
    dev_free(d_mo, st);
    dev_free(d_out, st);
    return SKIS_OK;
    API_CATCH
}

void skis::sketch_release(skis_sketch* s) {
    cudaStream_t st = s->stream;
    dev_free(s->h_off, st);
    dev_free(s->h_len, st);
    dev_free(s->h_src, st);
    dev_free(s->h_retries, st);
    dev_free(s->h_coins, st);
    dev_free(s->arena, st);
    dev_free(s->ctr, st);
    dev_free(s->status, st);
    dev_free(s->to_warp_ids, st);
    dev_free(s->to_cta_ids, st);
    dev_free(s->srcrec, st);
    dev_free(s->srcpick, st);
    dev_free(s->ovf_ids[0], st);
    dev_free(s->ovf_ids[1], st);
    dev_free(s->bitmaps, st);
    dev_free(s->queues, st);
    dev_free(s->big_queues, st);
    dev_free(s->big_ids, st);
    dev_free(s->lt_hash, st);
    dev_free(s->lt_list, st);
    dev_free(s->lt_slot, st);
    dev_free(s->qmask, st);
    dev_free(s->qbits, st);
    dev_free(s->inv_off, st);
    dev_free(s->inv, st);
    dev_free(s->smask, st);
    dev_free(s->vcount, st);
    dev_free(s->qcov, st);
    dev_free(s->qstatus, st);
    dev_free(s->touched, st);
    dev_free(s->ntouched, st);
    dev_free(s->hits, st);
    for (int i = 0; i < 2; ++i)
        if (s->qev[i]) cudaEventDestroy(s->qev[i]);
    for (int i = 0; i < 4; ++i)
        if (s->ev[i]) cudaEventDestroy(s->ev[i]);
}

extern "C" void skis_sketch_free(skis_sketch* s) {
    if (!s) return;
    sketch_release(s);
    delete s;
}

extern "C" const char* skis_last_error(void) { return g_err.c_str(); }

extern "C" int skis_philox_rate(uint64_t seed, uint64_t threads, uint64_t blocks_per_thread, int form,
                                double* ms_out, uint32_t* fold_out, void* cuda_stream) {
    API_TRY
    if (!ms_out || !fold_out) return fail(SKIS_EINVAL, "skis_philox_rate: NULL output");
    if (threads < 1 || threads > (1ull << 31) || blocks_per_thread < 1 || blocks_per_thread > (1ull << 31) ||
        form < 0 || form > 1 || threads * blocks_per_thread >= (1ull << 32))
        return fail(SKIS_EINVAL, "skis_philox_rate: threads and blocks per thread in [1, 2^31], fewer than 2^32 "
                                 "blocks, form 0 or 1");
    std::string err;
    const int rc = philox_rate(seed, threads, blocks_per_thread, form, ms_out, fold_out, (cudaStream_t)cuda_stream,
                               &err);
    if (rc != SKIS_OK) return fail(rc, err);
    return SKIS_OK;
    API_CATCH
}

extern "C" uint64_t skis_kernel_launches(void) { return launches(); }

extern "C" uint64_t skis_device_allocations(void) { return allocations(); }
