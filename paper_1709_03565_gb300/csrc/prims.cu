// Device primitives used while building the graph and the greedy index:
// stream-ordered allocation, exclusive prefix sums (u32->u64, u64, u128),
// a stable LSD radix sort of (u64 key, u32 value) pairs, and a u64 sum.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "skis_internal.cuh"

namespace skis {

// --------------------------------------------------------------- launches
static std::atomic<uint64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------- allocation
static std::once_flag g_pool_once;
static std::atomic<uint64_t> g_allocs{0};
uint64_t allocations() { return g_allocs.load(std::memory_order_relaxed); }

cudaError_t dev_malloc(void** p, size_t bytes) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(p, bytes);
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st) {
    std::call_once(g_pool_once, [] {
        // Keep freed blocks in this process's default pool so that repeated
        // graph/sketch builds do not return memory to the CUDA driver and map it
        // again. The attribute belongs to this process's pool only.
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocAsync(p, bytes, st);
}

void dev_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

int sm_count() {
    static int cached = 0;
    if (cached == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached = v > 0 ? v : 1;
    }
    return cached;
}

// ------------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t shfl_up_t(uint64_t v, int d) { return __shfl_up_sync(kFull, v, d); }
__device__ __forceinline__ u128 shfl_up_t(u128 v, int d) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_up_sync(kFull, lo, d);
    hi = __shfl_up_sync(kFull, hi, d);
    return ((u128)hi << 64) | lo;
}

// Exclusive scan of one value per thread across the block; returns the
// thread's exclusive prefix, and the block total in *total.
template <typename T>
__device__ T block_exclusive_scan(T val, T* total) {
    __shared__ T s_warp[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T incl = val;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = shfl_up_t(incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T w = lane < kScanThreads / 32 ? s_warp[lane] : T(0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T y = shfl_up_t(w, d);
            if (lane >= d) w += y;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const T warp_excl = wid > 0 ? s_warp[wid - 1] : T(0);
    *total = s_warp[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_excl + incl - val;
}

template <typename TIn, typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const TIn* __restrict__ in, int64_t n,
                                                              T* __restrict__ partial) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += (T)in[base + k];
    T tot;
    block_exclusive_scan<T>(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename TIn, typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const TIn* __restrict__ in, int64_t n,
                                                             const T* __restrict__ offsets,
                                                             T* __restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? (T)in[base + k] : T(0);
        s += v[k];
    }
    T tot;
    T run = block_exclusive_scan<T>(s, &tot) + (offsets ? offsets[blockIdx.x] : T(0));
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = run;
}

template <typename TIn, typename T>
static cudaError_t scan_impl(const TIn* in, T* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(T), st);
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_apply<TIn, T><<<1, kScanThreads, 0, st>>>(in, n, (const T*)nullptr, out); note_launch();
        return cudaGetLastError();
    }
    T* partial = nullptr;
    T* pscan = nullptr;
    cudaError_t e = dev_alloc_t(&partial, (size_t)nb, st);
    if (e != cudaSuccess) return e;
    e = dev_alloc_t(&pscan, (size_t)nb + 1, st);
    if (e != cudaSuccess) { dev_free(partial, st); return e; }
    k_scan_reduce<TIn, T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, partial); note_launch();
    e = scan_impl<T, T>(partial, pscan, nb, st);
    if (e == cudaSuccess) {
        k_scan_apply<TIn, T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, pscan, out); note_launch();
        e = cudaGetLastError();
    }
    dev_free(partial, st);
    dev_free(pscan, st);
    return e;
}

cudaError_t scan_u32_to_u64(const uint32_t* in, uint64_t* out, int64_t n, cudaStream_t st) {
    return scan_impl<uint32_t, uint64_t>(in, out, n, st);
}
cudaError_t scan_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t st) {
    return scan_impl<uint64_t, uint64_t>(in, out, n, st);
}
cudaError_t scan_u128(const u128* in, u128* out, int64_t n, cudaStream_t st) {
    return scan_impl<u128, u128>(in, out, n, st);
}

// ------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;  // 2048 pairs per tile
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                             int shift, uint32_t* __restrict__ hist,
                                                             int nblocks) {
    __shared__ uint32_t s_h[256];
    s_h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int c = 0; c < kSortItems; ++c) {
        const int64_t i = base + (int64_t)c * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&s_h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter of one tile. The tile's items are ranked in order (chunks
// of 256; within a chunk warp w precedes warp w+1 and lanes rank by lane id
// among equal digits) and placed in shared memory in digit order; then the
// tile is written out from shared memory, so that the items of one digit
// leave as one contiguous run (coalesced) at the digit's global base.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint64_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, int64_t n, int shift, const uint32_t* __restrict__ hist,
    const uint64_t* __restrict__ offs, int nblocks) {
    __shared__ uint64_t s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ uint32_t s_wcnt[kSortThreads / 32][256];
    __shared__ uint32_t s_start[256];  // digit start within the tile
    __shared__ uint32_t s_run[256];    // items of the digit placed so far
    __shared__ uint32_t s_wsum[kSortThreads / 32];
    __shared__ uint64_t s_base[256];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    s_base[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    // exclusive scan of this tile's digit counts
    const uint32_t cnt = hist[(int64_t)tid * nblocks + blockIdx.x];
    uint32_t x = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_wsum[wid] = x;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) s_wcnt[w][tid] = 0;
    s_run[tid] = 0;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < wid; ++w) before += s_wsum[w];
    s_start[tid] = before + x - cnt;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int tile_n = (int)min((int64_t)kSortTile, n - base);
    for (int c = 0; c < kSortItems; ++c) {
        const int64_t i = base + (int64_t)c * kSortThreads + tid;
        const bool valid = i < n;
        const uint64_t key = valid ? keys_in[i] : 0;
        const uint32_t val = valid ? vals_in[i] : 0;
        const uint32_t d = valid ? (uint32_t)((key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(kFull, d);
        const int rank = __popc(peers & lanemask_lt());
        if (valid && lane == __ffs(peers) - 1) s_wcnt[wid][d] = (uint32_t)__popc(peers);
        __syncthreads();
        uint32_t run = 0;  // thread tid: digit tid's per-warp offsets within the chunk
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const uint32_t c2 = s_wcnt[w][tid];
            s_wcnt[w][tid] = run;
            run += c2;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_start[d] + s_run[d] + s_wcnt[wid][d] + (uint32_t)rank;
            s_keys[pos] = key;
            s_vals[pos] = val;
        }
        __syncthreads();
        s_run[tid] += run;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) s_wcnt[w][tid] = 0;
        __syncthreads();
    }
    for (int i = tid; i < tile_n; i += kSortThreads) {
        const uint64_t key = s_keys[i];
        const uint32_t d = (uint32_t)((key >> shift) & 255u);
        const uint64_t pos = s_base[d] + (uint64_t)(i - (int)s_start[d]);
        keys_out[pos] = key;
        vals_out[pos] = s_vals[i];
    }
}

cudaError_t radix_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                             uint32_t* vals_out, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                             int bits, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int passes = (bits + 7) / 8;
    if (passes == 0) {
        cudaError_t e = cudaMemcpyAsync(keys_out, keys_in, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(vals_out, vals_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    }
    const int nb = div_up(n, kSortTile);
    uint32_t* hist = nullptr;
    uint64_t* offs = nullptr;
    cudaError_t e = dev_alloc_t(&hist, (size_t)nb * 256, st);
    if (e != cudaSuccess) return e;
    e = dev_alloc_t(&offs, (size_t)nb * 256 + 1, st);
    if (e != cudaSuccess) { dev_free(hist, st); return e; }
    const uint64_t* ksrc = keys_in;
    const uint32_t* vsrc = vals_in;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint64_t* kdst = to_out ? keys_out : keys_alt;
        uint32_t* vdst = to_out ? vals_out : vals_alt;
        k_radix_hist<<<nb, kSortThreads, 0, st>>>(ksrc, n, 8 * p, hist, nb); note_launch();
        e = scan_u32_to_u64(hist, offs, (int64_t)nb * 256, st);
        if (e != cudaSuccess) break;
        k_radix_scatter<<<nb, kSortThreads, 0, st>>>(ksrc, vsrc, kdst, vdst, n, 8 * p, hist, offs, nb); note_launch();
        e = cudaGetLastError();
        ksrc = kdst;
        vsrc = vdst;
    }
    dev_free(hist, st);
    dev_free(offs, st);
    return e;
}

// -------------------------------------------------------------------- sum
__global__ void k_sum_u64(const uint64_t* __restrict__ in, int64_t n, unsigned long long* out) {
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += in[i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(kFull, s, d);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

cudaError_t sum_u64(const uint64_t* in, int64_t n, unsigned long long* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int blocks = (int)std::min<int64_t>((int64_t)sm_count() * 4, std::max<int64_t>(1, (n + 255) / 256));
    k_sum_u64<<<blocks, 256, 0, st>>>(in, n, out); note_launch();
    return cudaGetLastError();
}

}  // namespace skis
