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
// sample id t (BFS domain), four independent blocks a step, and folds every
// coin word into one XOR, the least work that keeps each block live: no
// memory traffic but one atomic per thread. kForm 0 computes each block as
// coin_block does; kForm 1 as the CTA tier's hub loop does (SampleBlock, two
// products hoisted per sample). 32-bit loop state: the host keeps threads x
// per below 2^32.
template <int kForm>
__global__ void __launch_bounds__(256) k_philox_rate(PhiloxKeys rk, uint32_t per, uint32_t threads,
                                                     unsigned int* __restrict__ fold) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= threads) return;
    const SampleBlock blk(rk, t, kDomBfs);
    auto block = [&](uint32_t q) { return kForm ? blk(q, rk) : coin_block(rk, q, 0, kDomBfs, t); };
    auto xor4 = [](const uint4& x) { return x.x ^ x.y ^ x.z ^ x.w; };
    uint32_t f = 0;
    const uint32_t q0 = t * per;
    uint32_t k = 0;
    for (; k + 4 <= per; k += 4) {
        const uint4 x0 = block(q0 + k), x1 = block(q0 + k + 1), x2 = block(q0 + k + 2), x3 = block(q0 + k + 3);
        f ^= xor4(x0) ^ xor4(x1) ^ xor4(x2) ^ xor4(x3);
    }
    for (; k < per; ++k) f ^= xor4(block(q0 + k));
    atomicXor(fold, f);
}

#define PR_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t _e = (call);                                                            \
        if (_e != cudaSuccess) {                                                            \
            *err = std::string("CUDA error in skis_philox_rate: ") + cudaGetErrorString(_e); \
            return _e == cudaErrorMemoryAllocation ? SKIS_ENOMEM : SKIS_ERR_CUDA;           \
        }                                                                                   \
    } while (0)

int philox_rate(uint64_t seed, uint64_t threads, uint64_t per, int form, double* ms_out, uint32_t* fold_out,
                cudaStream_t st, std::string* err) {
    unsigned int* d = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto body = [&]() -> int {
        PR_CUDA(dev_alloc_t(&d, 1, st));
        PR_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned int), st));
        PR_CUDA(cudaEventCreate(&e0));
        PR_CUDA(cudaEventCreate(&e1));
        PR_CUDA(cudaEventRecord(e0, st));
        const unsigned grid = (unsigned)((threads + 255) / 256);
        if (form)
            k_philox_rate<1><<<grid, 256, 0, st>>>(philox_keys(seed), (uint32_t)per, (uint32_t)threads, d);
        else
            k_philox_rate<0><<<grid, 256, 0, st>>>(philox_keys(seed), (uint32_t)per, (uint32_t)threads, d);
        note_launch();
        PR_CUDA(cudaGetLastError());
        PR_CUDA(cudaEventRecord(e1, st));
        PR_CUDA(cudaMemcpyAsync(fold_out, d, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
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
