// Influence queries without any allocation: skis_estimate_noalloc.
//
// Some callers cannot allocate device memory at the moment they query: a
// process whose device memory is already reserved in full by another
// allocator (a framework's caching allocator, or an application pool sized
// at start-up), where cudaMalloc would fail or fragment that reservation;
// and latency-critical query loops that must not pay the unbounded latency
// and implicit synchronisation an allocation can bring. This entry point
// answers the same queries as skis_estimate with no cudaMalloc, cudaFree or
// allocating library call: its scratch (per-vertex query masks, coverage
// counters, status word) is the file-scope device array below, which every
// GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/skis.h"
#include "skis_internal.cuh"

namespace skis {

constexpr int64_t kNoallocMaxN = int64_t(1) << 20;  // vertices: 8 MiB of query masks
constexpr int32_t kNoallocMaxQ = 64;                // queries per call (one mask bit each)
constexpr int kNoallocMaxDevices = 64;

// Layout: [0, kNoallocMaxN) per-vertex query masks, then 64 coverage
// counters, then one DevStatus (two words). Zero at module load.
constexpr int64_t kScratchWords = kNoallocMaxN + kNoallocMaxQ + 2;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kScratchWords];

// Device address of g_noalloc_scratch per device. The symbol's name is only a
// host-side stand-in, so host code must never hand it to a kernel; this
// table holds what cudaGetSymbolAddress returned with that device current.
static uint64_t* g_scratch_addr[kNoallocMaxDevices] = {};
static std::once_flag g_scratch_once[kNoallocMaxDevices];
static cudaError_t g_scratch_err[kNoallocMaxDevices] = {};

static cudaError_t scratch_for_current_device(uint64_t** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_scratch_once[dev], [dev] {
        void* p = nullptr;
        g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (g_scratch_err[dev] == cudaSuccess) g_scratch_addr[dev] = static_cast<uint64_t*>(p);
    });
    if (g_scratch_err[dev] != cudaSuccess) return g_scratch_err[dev];
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace skis

using namespace skis;

// Copies msg (+ detail) into the caller's buffer, if one was given: this
// entry point allocates no host memory either, even when it fails.
static int noalloc_fail(char* buf, uint64_t len, int code, const char* msg, const char* detail = nullptr) {
    if (buf && len > 0) {
        uint64_t i = 0;
        for (; msg[i] && i + 1 < len; ++i) buf[i] = msg[i];
        if (detail)
            for (uint64_t k = 0; detail[k] && i + 1 < len; ++k, ++i) buf[i] = detail[k];
        buf[i] = 0;
    }
    return code;
}

extern "C" int skis_estimate_noalloc(const skis_sketch* s, int32_t num_queries, const int64_t* seed_offsets,
                                     const int32_t* seeds, int64_t* coverage_out, double* estimate_out,
                                     char* error_buf, uint64_t error_len, void* cuda_stream) {
    if (error_buf && error_len > 0) error_buf[0] = 0;
    if (!s || !seed_offsets || !estimate_out)
        return noalloc_fail(error_buf, error_len, SKIS_EINVAL, "skis_estimate_noalloc: NULL argument");
    if (num_queries < 0 || num_queries > kNoallocMaxQ)
        return noalloc_fail(error_buf, error_len, SKIS_EINVAL, "skis_estimate_noalloc: num_queries must be in [0, 64]");
    const skis_graph* g = s->g;
    if (g->n > kNoallocMaxN)
        return noalloc_fail(error_buf, error_len, SKIS_EINVAL,
                            "skis_estimate_noalloc: the graph has more than 2^20 vertices, the size of its "
                            "static query-mask scratch; use skis_estimate");
    if (s->T == 0) return noalloc_fail(error_buf, error_len, SKIS_EINVAL, "skis_estimate_noalloc: the sketch has no samples");
    if (num_queries == 0) return SKIS_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint64_t* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return noalloc_fail(error_buf, error_len, SKIS_ERR_CUDA, "skis_estimate_noalloc: scratch set-up: ", cudaGetErrorString(e));
    uint64_t* qmask = scratch;
    unsigned long long* qcov = reinterpret_cast<unsigned long long*>(scratch + kNoallocMaxN);
    DevStatus* status = reinterpret_cast<DevStatus*>(scratch + kNoallocMaxN + kNoallocMaxQ);

    // the seed offsets are checked on the host, in a fixed stack buffer
    int64_t off[kNoallocMaxQ + 1];
    e = cudaMemcpyAsync(off, seed_offsets, (size_t)(num_queries + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(error_buf, error_len, SKIS_ERR_CUDA, "skis_estimate_noalloc: ", cudaGetErrorString(e));
    if (off[0] < 0) return noalloc_fail(error_buf, error_len, SKIS_EINVAL, "skis_estimate_noalloc: negative seed offset");
    for (int32_t b = 0; b < num_queries; ++b)
        if (off[b + 1] < off[b]) return noalloc_fail(error_buf, error_len, SKIS_EINVAL, "skis_estimate_noalloc: seed offsets decrease");
    if (off[num_queries] > 0 && !seeds) return noalloc_fail(error_buf, error_len, SKIS_EINVAL, "skis_estimate_noalloc: seeds is NULL");

    // the array keeps the previous call's contents: clear the masks of this
    // graph's vertices, the counters and the status word
    e = cudaMemsetAsync(qmask, 0, (size_t)g->n * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(qcov, 0, kNoallocMaxQ * sizeof(unsigned long long) + sizeof(DevStatus), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&status->first_bad, 0xFF, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return noalloc_fail(error_buf, error_len, SKIS_ERR_CUDA, "skis_estimate_noalloc: ", cudaGetErrorString(e));

    const int wb = (int)((num_queries * 32 + 255) / 256);
    const uint64_t groups = (s->T + 31) / 32;
    uint64_t cb = (groups + 7) / 8;
    const uint64_t cap = (uint64_t)sm_count() * 8;
    if (cb > cap) cb = cap;
    if (cb < 1) cb = 1;
    k_qmask_set<<<wb, 256, 0, st>>>(seed_offsets, seeds, 0, num_queries, g->n, qmask, nullptr, status); note_launch();
    k_coverage<<<(unsigned)cb, 256, 0, st>>>(s->h_off, s->h_len, s->T, s->arena, qmask, nullptr, 0, qcov); note_launch();
    k_estimate<<<wb, 256, 0, st>>>(seed_offsets, seeds, 0, num_queries, g->n, g->w, g->f, g->W, s->T, qcov,
                                   coverage_out, estimate_out, s->ris); note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(error_buf, error_len, SKIS_ERR_CUDA, "skis_estimate_noalloc: launch: ", cudaGetErrorString(e));
    DevStatus h;
    e = cudaMemcpyAsync(&h, status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(error_buf, error_len, SKIS_ERR_CUDA, "skis_estimate_noalloc: ", cudaGetErrorString(e));
    if (h.flags & kStInval) {
        // the message names the failing query as skis_estimate's does, its
        // index written out in a stack buffer (no allocation)
        char msg[160];
        const char* head = "skis_estimate_noalloc: query ";
        const char* tail = " is empty, has a seed outside [0, n) or repeats a seed";
        char digits[24];
        int nd = 0;
        unsigned long long q = h.first_bad;
        do {
            digits[nd++] = (char)('0' + q % 10);
            q /= 10;
        } while (q && nd < 20);
        int i = 0;
        for (int k = 0; head[k]; ++k) msg[i++] = head[k];
        while (nd) msg[i++] = digits[--nd];
        for (int k = 0; tail[k] && i + 1 < (int)sizeof(msg); ++k) msg[i++] = tail[k];
        msg[i] = 0;
        return noalloc_fail(error_buf, error_len, SKIS_EINVAL, msg);
    }
    return SKIS_OK;
}
