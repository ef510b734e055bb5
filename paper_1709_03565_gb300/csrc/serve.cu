// Continuous-batching influence-oracle server (Alg. 2's estimate step, Eq. 21, served
// against a device-resident sketch and its inverted index).
//
// Requests (seed sets) are validated and queued on the host at submit time.
// Each progress call retires finished batches (event polling, no host
// threads) and admits queued requests, in arrival order, into every free
// in-flight slot: up to max_batch requests (one query-mask bit each, at most
// 64) whose seeds fit the slot's staging capacity. A slot owns a stream,
// pinned host staging, device buffers and its own per-sample query-mask
// scratch, so batches on different slots overlap on the device. Coverage is
// counted through the sketch's inverted index, so a batch costs the total
// length of its seeds' sample lists, not a scan of the sketch. Results are
// exact integers (coverage) and the same binary64 quotient as skis_estimate,
// whatever batch a request lands in.
#include <algorithm>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include "../../include/skis.h"
#include "skis_internal.cuh"

using namespace skis;

namespace {

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int64_t* h_off = nullptr;  // pinned staging
    int32_t* h_seeds = nullptr;
    int64_t* h_cov = nullptr;
    double* h_est = nullptr;
    DevStatus* h_status = nullptr;
    int64_t* d_off = nullptr;  // device
    int32_t* d_seeds = nullptr;
    int64_t* d_cov = nullptr;
    double* d_est = nullptr;
    uint64_t* d_smask = nullptr;   // T per-sample query bits, zero between batches
    uint32_t* d_chunk_cnt = nullptr;
    uint64_t* d_chunk_off = nullptr;
    unsigned long long* d_qcov = nullptr;
    DevStatus* d_status = nullptr;
    std::vector<uint64_t> tickets;
    bool busy = false;
};

struct Pending {
    uint64_t ticket;
    std::vector<int32_t> seeds;
};

struct Result {
    int64_t cov = 0;
    double est = 0;
    int32_t state = 0;  // 0 queued or in flight, 1 ready, 2 failed on the device
};

}  // namespace

struct skis_server {
    skis_sketch* s = nullptr;
    int32_t max_batch = 64;
    uint64_t seed_cap = 0;
    std::vector<Slot> slots;
    std::deque<Pending> pending;
    std::vector<Result> results;  // indexed by ticket
    uint64_t batches = 0, served = 0;
    std::vector<uint8_t> mark;    // duplicate check at submit (n bytes)
};

static int serve_fail(int code, const std::string& msg) { return set_last_error(code, msg); }

#define SV_CUDA(call)                                                                           \
    do {                                                                                        \
        cudaError_t _e = (call);                                                                \
        if (_e != cudaSuccess)                                                                  \
            return serve_fail(_e == cudaErrorMemoryAllocation ? SKIS_ENOMEM : SKIS_ERR_CUDA,    \
                              std::string("skis_server: CUDA error: ") + cudaGetErrorString(_e)); \
    } while (0)

static void release_slot(Slot& sl) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    cudaFreeHost(sl.h_off);
    cudaFreeHost(sl.h_seeds);
    cudaFreeHost(sl.h_cov);
    cudaFreeHost(sl.h_est);
    cudaFreeHost(sl.h_status);
    cudaFree(sl.d_off);
    cudaFree(sl.d_seeds);
    cudaFree(sl.d_cov);
    cudaFree(sl.d_est);
    cudaFree(sl.d_smask);
    cudaFree(sl.d_chunk_cnt);
    cudaFree(sl.d_chunk_off);
    cudaFree(sl.d_qcov);
    cudaFree(sl.d_status);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    sl = Slot();
}

extern "C" void skis_server_free(skis_server* srv) {
    if (!srv) return;
    for (Slot& sl : srv->slots) release_slot(sl);
    delete srv;
}

extern "C" int skis_server_create(skis_server** out, skis_sketch* s, int32_t slots, int32_t max_batch,
                                  uint64_t seed_capacity) {
    try {
        if (!out || !s) return serve_fail(SKIS_EINVAL, "skis_server_create: NULL argument");
        *out = nullptr;
        if (slots < 1 || slots > 64) return serve_fail(SKIS_EINVAL, "skis_server_create: slots must be in [1, 64]");
        if (max_batch < 1 || max_batch > 64)
            return serve_fail(SKIS_EINVAL, "skis_server_create: max_batch must be in [1, 64]");
        if (seed_capacity < 1 || seed_capacity > (1ull << 31))
            return serve_fail(SKIS_EINVAL, "skis_server_create: seed_capacity must be in [1, 2^31]");
        if (s->T == 0) return serve_fail(SKIS_EINVAL, "skis_server_create: the sketch has no samples");
        {
            // requests are answered through the sketch's inverted index; the
            // members are laid out in id order now, so that no later scan of
            // the (unchanged) sketch moves them while the server reads them
            std::string err;
            int rc = sketch_order_arena(s, s->stream, &err);
            if (rc == SKIS_OK) rc = sketch_inverted(s, s->stream, &err);
            if (rc != SKIS_OK) return serve_fail(rc, err);
            const cudaError_t e = cudaStreamSynchronize(s->stream);
            if (e != cudaSuccess) return serve_fail(SKIS_ERR_CUDA, std::string("skis_server_create: ") + cudaGetErrorString(e));
        }
        skis_server* srv = new skis_server();
        srv->s = s;
        srv->max_batch = max_batch;
        srv->seed_cap = seed_capacity;
        srv->slots.resize((size_t)slots);
        srv->mark.assign((size_t)s->g->n, 0);
        for (Slot& sl : srv->slots) {
            cudaError_t e = cudaSuccess;
            auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
            chk(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
            chk(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
            chk(cudaMallocHost((void**)&sl.h_off, 65 * sizeof(int64_t)));
            chk(cudaMallocHost((void**)&sl.h_seeds, seed_capacity * sizeof(int32_t)));
            chk(cudaMallocHost((void**)&sl.h_cov, 64 * sizeof(int64_t)));
            chk(cudaMallocHost((void**)&sl.h_est, 64 * sizeof(double)));
            chk(cudaMallocHost((void**)&sl.h_status, sizeof(DevStatus)));
            chk(dev_malloc((void**)&sl.d_off, 65 * sizeof(int64_t)));
            chk(dev_malloc((void**)&sl.d_seeds, seed_capacity * sizeof(int32_t)));
            chk(dev_malloc((void**)&sl.d_cov, 64 * sizeof(int64_t)));
            chk(dev_malloc((void**)&sl.d_est, 64 * sizeof(double)));
            chk(dev_malloc((void**)&sl.d_smask, (size_t)s->T * sizeof(uint64_t)));
            chk(dev_malloc((void**)&sl.d_chunk_cnt, seed_capacity * sizeof(uint32_t)));
            chk(dev_malloc((void**)&sl.d_chunk_off, (seed_capacity + 1) * sizeof(uint64_t)));
            chk(dev_malloc((void**)&sl.d_qcov, 64 * sizeof(unsigned long long)));
            chk(dev_malloc((void**)&sl.d_status, sizeof(DevStatus)));
            if (e == cudaSuccess) e = cudaMemsetAsync(sl.d_smask, 0, (size_t)s->T * sizeof(uint64_t), sl.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(sl.stream);
            if (e != cudaSuccess) {
                skis_server_free(srv);
                return serve_fail(e == cudaErrorMemoryAllocation ? SKIS_ENOMEM : SKIS_ERR_CUDA,
                                  std::string("skis_server_create: ") + cudaGetErrorString(e));
            }
        }
        *out = srv;
        return SKIS_OK;
    } catch (const std::bad_alloc&) {
        return serve_fail(SKIS_ENOMEM, "skis_server_create: host allocation failed");
    }
}

extern "C" int skis_server_submit(skis_server* srv, const int32_t* seeds, int32_t nseeds, uint64_t* ticket_out) {
    try {
        if (!srv || !ticket_out || (nseeds > 0 && !seeds)) return serve_fail(SKIS_EINVAL, "skis_server_submit: NULL argument");
        if (nseeds < 1) return serve_fail(SKIS_EINVAL, "skis_server_submit: empty seed set");
        if ((uint64_t)nseeds > srv->seed_cap)
            return serve_fail(SKIS_EINVAL, "skis_server_submit: seed set larger than the slot staging capacity");
        const int64_t n = srv->s->g->n;
        // a seed set is a set of vertices of G (Def. 1)
        int32_t bad = -1;
        for (int32_t i = 0; i < nseeds; ++i) {
            const int32_t v = seeds[i];
            if (v < 0 || v >= n || srv->mark[v]) { bad = i; break; }
            srv->mark[v] = 1;
        }
        for (int32_t i = 0; i < (bad < 0 ? nseeds : bad); ++i) srv->mark[seeds[i]] = 0;
        if (bad >= 0) return serve_fail(SKIS_EINVAL, "skis_server_submit: seed outside [0, n) or repeated");
        Pending p;
        p.ticket = srv->results.size();
        p.seeds.assign(seeds, seeds + nseeds);
        srv->results.emplace_back();
        srv->pending.push_back(std::move(p));
        *ticket_out = srv->pending.back().ticket;
        return SKIS_OK;
    } catch (const std::bad_alloc&) {
        return serve_fail(SKIS_ENOMEM, "skis_server_submit: host allocation failed");
    }
}

static int launch_batch(skis_server* srv, Slot& sl) {
    skis_sketch* s = srv->s;
    const skis_graph* g = s->g;
    int32_t q = 0;
    uint64_t used = 0;
    sl.tickets.clear();
    sl.h_off[0] = 0;
    while (!srv->pending.empty() && q < srv->max_batch) {
        Pending& p = srv->pending.front();
        if (used + p.seeds.size() > srv->seed_cap) break;  // admission by staging memory
        std::copy(p.seeds.begin(), p.seeds.end(), sl.h_seeds + used);
        used += p.seeds.size();
        sl.h_off[q + 1] = (int64_t)used;
        sl.tickets.push_back(p.ticket);
        srv->pending.pop_front();
        ++q;
    }
    if (q == 0) return SKIS_OK;
    cudaStream_t st = sl.stream;
    SV_CUDA(cudaMemcpyAsync(sl.d_off, sl.h_off, (size_t)(q + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    SV_CUDA(cudaMemcpyAsync(sl.d_seeds, sl.h_seeds, used * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    SV_CUDA(cudaMemsetAsync(sl.d_qcov, 0, 64 * sizeof(unsigned long long), st));
    SV_CUDA(cudaMemsetAsync(sl.d_status, 0, sizeof(DevStatus), st));
    const int wb = (q * 32 + 255) / 256;
    SV_CUDA(coverage_by_index(s, sl.d_off, sl.d_seeds, 0, q, 0, (int64_t)used, sl.d_chunk_cnt, sl.d_chunk_off,
                              sl.d_smask, sl.d_qcov, st));
    k_estimate<<<wb, 256, 0, st>>>(sl.d_off, sl.d_seeds, 0, q, g->n, g->w, g->f, g->W, s->T, sl.d_qcov, sl.d_cov,
                                   sl.d_est, s->ris); note_launch();
    SV_CUDA(cudaGetLastError());
    SV_CUDA(cudaMemcpyAsync(sl.h_cov, sl.d_cov, (size_t)q * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SV_CUDA(cudaMemcpyAsync(sl.h_est, sl.d_est, (size_t)q * sizeof(double), cudaMemcpyDeviceToHost, st));
    SV_CUDA(cudaMemcpyAsync(sl.h_status, sl.d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    SV_CUDA(cudaEventRecord(sl.done, st));
    sl.busy = true;
    srv->batches += 1;
    return SKIS_OK;
}

static void retire_batch(skis_server* srv, Slot& sl, uint64_t* done, int32_t cap, int32_t* ndone) {
    const bool bad = (sl.h_status->flags & kStInval) != 0;  // cannot happen: validated at submit
    for (size_t i = 0; i < sl.tickets.size(); ++i) {
        Result& r = srv->results[sl.tickets[i]];
        r.cov = sl.h_cov[i];
        r.est = sl.h_est[i];
        r.state = bad ? 2 : 1;
        if (done && *ndone < cap) done[(*ndone)++] = sl.tickets[i];
    }
    srv->served += sl.tickets.size();
    sl.tickets.clear();
    sl.busy = false;
}

extern "C" int skis_server_progress(skis_server* srv, int32_t wait, uint64_t* done_tickets, int32_t cap,
                                    int32_t* ndone_out) {
    if (!srv) return serve_fail(SKIS_EINVAL, "skis_server_progress: NULL server");
    int32_t ndone = 0;
    bool any_busy = false;
    for (Slot& sl : srv->slots) any_busy = any_busy || sl.busy;
    if (wait && any_busy) {
        // block until the oldest in-flight batch is done
        for (Slot& sl : srv->slots)
            if (sl.busy) {
                SV_CUDA(cudaEventSynchronize(sl.done));
                break;
            }
    }
    for (Slot& sl : srv->slots) {
        if (!sl.busy) continue;
        const cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        SV_CUDA(e);
        retire_batch(srv, sl, done_tickets, cap, &ndone);
    }
    for (Slot& sl : srv->slots) {
        if (srv->pending.empty()) break;
        if (sl.busy) continue;
        const int rc = launch_batch(srv, sl);
        if (rc != SKIS_OK) return rc;
    }
    if (ndone_out) *ndone_out = ndone;
    return SKIS_OK;
}

extern "C" int skis_server_poll(skis_server* srv, uint64_t ticket, int64_t* coverage_out, double* estimate_out,
                                int32_t* state_out) {
    if (!srv || !state_out) return serve_fail(SKIS_EINVAL, "skis_server_poll: NULL argument");
    if (ticket >= srv->results.size()) return serve_fail(SKIS_EINVAL, "skis_server_poll: unknown ticket");
    const Result& r = srv->results[ticket];
    *state_out = r.state;
    if (r.state == 1) {
        if (coverage_out) *coverage_out = r.cov;
        if (estimate_out) *estimate_out = r.est;
    }
    return SKIS_OK;
}

extern "C" int skis_server_counts(const skis_server* srv, uint64_t* queued, uint64_t* in_flight, uint64_t* batches,
                                  uint64_t* served) {
    if (!srv) return serve_fail(SKIS_EINVAL, "skis_server_counts: NULL server");
    uint64_t fl = 0;
    for (const Slot& sl : srv->slots) fl += sl.tickets.size();
    if (queued) *queued = srv->pending.size();
    if (in_flight) *in_flight = fl;
    if (batches) *batches = srv->batches;
    if (served) *served = srv->served;
    return SKIS_OK;
}
