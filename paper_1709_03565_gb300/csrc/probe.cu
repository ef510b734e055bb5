// The coin generator's throughput on this GPU: a launch that draws Philox
// blocks and nothing else, the measured counterpart of the integer-ALU
// ceiling the sampling tiers are held against (under weighted cascade a coin
// moves no byte of memory, so the generator is what binds the CTA tier).
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/skis.h"
#include "skis_internal.cuh"

namespace skis {

// Thread t draws the Philox blocks of edge quads [t per, (t + 1) per) of
// sample id t (BFS domain), four independent blocks a step, and counts the
// coin words below tau: no memory traffic but one count per thread. form 0
// computes each block as coin_block does; form 1 as the CTA tier's hub loop
// does (SampleBlock, two products hoisted per sample). 32-bit loop state:
// the host keeps threads x per below 2^32.
__global__ void __launch_bounds__(256) k_philox_rate(PhiloxKeys rk, uint32_t per, uint32_t threads, uint32_t tau,
                                                     int form, unsigned long long* __restrict__ live) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= threads) return;
    const SampleBlock blk(rk, t, kDomBfs);
    auto block = [&](uint32_t q) { return form ? blk(q, rk) : coin_block(rk, q, 0, kDomBfs, t); };
    auto below = [tau](const uint4& x) {
        return (uint32_t)(x.x < tau) + (uint32_t)(x.y < tau) + (uint32_t)(x.z < tau) + (uint32_t)(x.w < tau);
    };
    uint32_t c = 0;
    const uint32_t q0 = t * per;
    uint32_t k = 0;
    for (; k + 4 <= per; k += 4) {
        const uint4 x0 = block(q0 + k), x1 = block(q0 + k + 1), x2 = block(q0 + k + 2), x3 = block(q0 + k + 3);
        c += below(x0) + below(x1) + below(x2) + below(x3);
    }
    for (; k < per; ++k) c += below(block(q0 + k));
    if (c) atomicAdd(live, (unsigned long long)c);
}

#define PR_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t _e = (call);                                                            \
        if (_e != cudaSuccess) {                                                            \
            *err = std::string("CUDA error in skis_philox_rate: ") + cudaGetErrorString(_e); \
            return _e == cudaErrorMemoryAllocation ? SKIS_ENOMEM : SKIS_ERR_CUDA;           \
        }                                                                                   \
    } while (0)

int philox_rate(uint64_t seed, uint64_t threads, uint64_t per, uint32_t tau, int form, double* ms_out,
                unsigned long long* live_out, cudaStream_t st, std::string* err) {
    unsigned long long* d = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto body = [&]() -> int {
        PR_CUDA(dev_alloc_t(&d, 1, st));
        PR_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st));
        PR_CUDA(cudaEventCreate(&e0));
        PR_CUDA(cudaEventCreate(&e1));
        PR_CUDA(cudaEventRecord(e0, st));
        k_philox_rate<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(philox_keys(seed), (uint32_t)per,
                                                                         (uint32_t)threads, tau, form, d);
        note_launch();
        PR_CUDA(cudaGetLastError());
        PR_CUDA(cudaEventRecord(e1, st));
        PR_CUDA(cudaMemcpyAsync(live_out, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        PR_CUDA(cudaStreamSynchronize(st));
        float ms = 0;
        PR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        *ms_out = ms;
        return SKIS_OK;
    };
    const int rc = body();
    dev_free(d, st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

}  // namespace skis
