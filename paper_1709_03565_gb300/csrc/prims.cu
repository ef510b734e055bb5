// Device primitives used while building the graph and the greedy index:
// stream-ordered allocation, exclusive prefix sums (u32->u64, u64, u128),
// a stable LSD radix sort of the edges by (destination, source), and a u64
// sum.
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

// ------------------------------------------------------------- edge sort
// Stable LSD radix sort of the edges by key dst << src_bits | src, the input
// index as value (so equal keys keep input order), in 8-bit digits. One
// kernel reads the edges once and counts every digit of every pass; then one
// kernel a pass ("onesweep"): each CTA claims the next tile from a ticket,
// ranks its items per warp (match_any, warp-striped loads: positions in warp
// order, so the ranking is stable), publishes the tile's per-digit counts and
// looks back over the previous tiles' published counts for its global
// offsets (decoupled look-back), then writes the tile out through shared
// memory in digit order, so that each digit's items leave as a contiguous
// run. The first pass builds the keys from the edge arrays in registers.
constexpr int kOsThreads = 256;
constexpr int kOsItems = 16;
constexpr int kOsTile = kOsThreads * kOsItems;  // 4096 items
constexpr int kOsWarps = kOsThreads / 32;
constexpr int kOsMaxPasses = 8;
// status word of (tile, digit): state in bits 62-63 (1: the tile's own
// count, 2: inclusive prefix over tiles 0 .. tile), the pass tag (pass + 1)
// in bits 56-61, the count in bits 0-55. Words of another pass read as not
// yet published, so one zeroing serves every pass.
constexpr unsigned long long kOsAgg = 1ull << 62, kOsIncl = 2ull << 62;
constexpr unsigned long long kOsCount = (1ull << 56) - 1;
constexpr uint32_t kOsSpinLimit = 1u << 22;  // polls of one word before giving up (~0.3 s)
constexpr int kOsWindow = 8;                 // predecessor tiles read at once in the look-back

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t edge_key(const int32_t* src, const int32_t* dst, int64_t e, int src_bits) {
    return ((uint64_t)(uint32_t)dst[e] << src_bits) | (uint64_t)(uint32_t)src[e];
}

// Pass p sorts on the digit (key >> shift[p]) & (2^bits[p] - 1), bits[p] in
// {8, 9}: a 9-bit pass has 512 digits, two a thread in the per-digit steps,
// so that 50- and 52-bit keys take six passes instead of seven.
constexpr int kOsMaxDigits = 512;
struct OsPasses {
    int n;
    int shift[kOsMaxPasses];
    int bits[kOsMaxPasses];
};

// Digit counts of every pass: hist[p * kOsMaxDigits + d] = #{edges whose key
// has digit d in pass p}.
__global__ void __launch_bounds__(256) k_os_hist(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                 int64_t m, int src_bits, OsPasses ps,
                                                 unsigned long long* __restrict__ hist) {
    __shared__ uint32_t s_h[kOsMaxPasses * kOsMaxDigits];
    for (int i = threadIdx.x; i < ps.n * kOsMaxDigits; i += 256) s_h[i] = 0;
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = edge_key(src, dst, e, src_bits);
#pragma unroll
        for (int p = 0; p < kOsMaxPasses; ++p)  // static indices: the pass table stays in the parameters
            if (p < ps.n)
                atomicAdd(&s_h[p * kOsMaxDigits + (uint32_t)((key >> ps.shift[p]) & ((1u << ps.bits[p]) - 1u))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ps.n * kOsMaxDigits; i += 256)
        if (s_h[i]) atomicAdd(&hist[i], (unsigned long long)s_h[i]);
}

// Exclusive prefix of each pass's digit counts, in place: base[p * kOsMaxDigits + d].
__global__ void __launch_bounds__(kOsMaxDigits) k_os_bases(unsigned long long* __restrict__ hist, int passes) {
    __shared__ unsigned long long s_c[kOsMaxDigits];
    for (int p = 0; p < passes; ++p) {
        s_c[threadIdx.x] = hist[p * kOsMaxDigits + threadIdx.x];
        __syncthreads();
        unsigned long long b = 0;
        for (int d = 0; d < (int)threadIdx.x; ++d) b += s_c[d];
        hist[p * kOsMaxDigits + threadIdx.x] = b;
        __syncthreads();
    }
}

// One pass on the kBits-bit digit at `shift`. kFirst: the items are the
// edges (key built from src / dst, value = input index). kLast: the sorted
// items leave as the CSR arrays (source = the key's low src_bits bits,
// destination = the rest, input index) instead of keys and values. Dynamic
// shared memory: kOsTile keys and values.
struct OsOut {
    uint64_t* keys;
    uint32_t* vals;
    int32_t* csr_src;
    uint32_t* csr_dst;
    uint32_t* perm;
};

template <bool kFirst, bool kLast, int kBits>
__global__ void __launch_bounds__(kOsThreads, 3) k_os_pass(
    const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int src_bits,
    const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, OsOut out, int64_t n, int shift,
    unsigned long long tag,
    const unsigned long long* __restrict__ base, unsigned long long* __restrict__ status,
    unsigned int* __restrict__ ticket, unsigned int* __restrict__ gave_up) {
    constexpr int kDigits = 1 << kBits, kPer = kDigits / kOsThreads;  // digits a thread owns
    constexpr uint32_t kMask = kDigits - 1;
    extern __shared__ __align__(16) unsigned char os_smem[];
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(os_smem);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kOsTile);
    __shared__ uint32_t s_wcnt[kOsWarps][kDigits];   // per warp: digit counts, then the warp's start in the digit
    __shared__ uint32_t s_tstart[kDigits];           // digit start within the tile
    __shared__ unsigned long long s_gbase[kDigits];  // output position of the digit's first item of the tile
    __shared__ uint32_t s_wsum[kPer][kOsWarps];
    __shared__ uint32_t s_tile, s_bad;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        s_tile = atomicAdd(ticket, 1u);
        s_bad = 0;
    }
    unsigned long long digit_base[kPer];  // in flight while the tile loads
#pragma unroll
    for (int r = 0; r < kPer; ++r) digit_base[r] = base[tid + r * kOsThreads];
#pragma unroll
    for (int w = 0; w < kOsWarps; ++w)
#pragma unroll
        for (int r = 0; r < kPer; ++r) s_wcnt[w][tid + r * kOsThreads] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t t0 = (int64_t)tile * kOsTile;
    const int64_t wb = t0 + (int64_t)wid * (32 * kOsItems);
    uint64_t key[kOsItems];
    uint32_t val[kOsItems], rnk[kOsItems];
#pragma unroll
    for (int c = 0; c < kOsItems; ++c) {
        const int64_t i = wb + c * 32 + lane;
        if (kFirst) {
            key[c] = i < n ? edge_key(src, dst, i, src_bits) : 0;
            val[c] = (uint32_t)i;
        } else {
            key[c] = i < n ? keys_in[i] : 0;
            val[c] = i < n ? vals_in[i] : 0;
        }
    }
    // rank within the warp: earlier chunks, then lower lanes
#pragma unroll
    for (int c = 0; c < kOsItems; ++c) {
        const bool valid = wb + c * 32 + lane < n;
        const uint32_t d = valid ? (uint32_t)((key[c] >> shift) & kMask) : (uint32_t)kDigits;
        const unsigned peers = __match_any_sync(kFull, d);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (lane == leader && valid) {
            before = s_wcnt[wid][d];
            s_wcnt[wid][d] = before + (uint32_t)__popc(peers);
        }
        __syncwarp();  // this chunk's counts are in before the next chunk's leaders read them
        before = __shfl_sync(kFull, before, leader);
        rnk[c] = before + (uint32_t)__popc(peers & lanemask_lt());
    }
    __syncthreads();
    // thread tid owns digits tid + r kOsThreads: the tile's count and each warp's start
    uint32_t cnt[kPer], x[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int dd = tid + r * kOsThreads;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kOsWarps; ++w) {
            const uint32_t c2 = s_wcnt[w][dd];
            s_wcnt[w][dd] = run;
            run += c2;
        }
        cnt[r] = run;
        st_relaxed_u64(status + (size_t)tile * kDigits + dd, (tile == 0 ? kOsIncl : kOsAgg) | tag | run);
        // tile-local digit starts: exclusive scan of the counts in digit order
        uint32_t y = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t z = __shfl_up_sync(kFull, y, o);
            if (lane >= o) y += z;
        }
        x[r] = y;
        if (lane == 31) s_wsum[r][wid] = y;
    }
    // look back over the earlier tiles for each owned digit's items before
    // the tile, kOsWindow tiles a read: sum their own counts back to the first
    // inclusive prefix, waiting on the first tile not yet published
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int dd = tid + r * kOsThreads;
        unsigned long long excl = 0;
        if (tile > 0) {
            int64_t t = (int64_t)tile - 1;  // the next tile to account for
            uint32_t spins = 0;
            bool done = false;
            while (!done) {
                unsigned long long v[kOsWindow];
#pragma unroll
                for (int k = 0; k < kOsWindow; ++k)
                    v[k] = t - k >= 0 ? ld_relaxed_u64(status + (size_t)(t - k) * kDigits + dd) : 0;
                int k = 0;
#pragma unroll
                for (int q = 0; q < kOsWindow; ++q) {
                    const bool ready = (v[q] & (63ull << 56)) == tag && (v[q] >> 62) != 0;
                    if (!ready) break;
                    excl += v[q] & kOsCount;
                    ++k;
                    if ((v[q] >> 62) == 2) {
                        done = true;
                        break;
                    }
                }
                if (done) break;
                t -= k;  // tile 0 is always inclusive, so t stays >= 0
                if (k < kOsWindow) {  // tile t is not published yet
                    if (++spins > kOsSpinLimit) {  // cannot happen while every claimed tile runs; never hang
                        atomicOr(gave_up, 1u);
                        s_bad = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            st_relaxed_u64(status + (size_t)tile * kDigits + dd, kOsIncl | tag | ((excl + cnt[r]) & kOsCount));
        }
        s_gbase[dd] = digit_base[r] + excl;
    }
    __syncthreads();
    uint32_t lower = 0;  // items of the tile in the digits owned before this pass of r
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        uint32_t before = lower;
        for (int w = 0; w < wid; ++w) before += s_wsum[r][w];
        s_tstart[tid + r * kOsThreads] = before + x[r] - cnt[r];
#pragma unroll
        for (int w = 0; w < kOsWarps; ++w) lower += s_wsum[r][w];
    }
    __syncthreads();
    // the tile in shared memory in digit order
#pragma unroll
    for (int c = 0; c < kOsItems; ++c) {
        if (wb + c * 32 + lane < n) {
            const uint32_t d = (uint32_t)((key[c] >> shift) & kMask);
            const uint32_t pos = s_tstart[d] + s_wcnt[wid][d] + rnk[c];
            s_keys[pos] = key[c];
            s_vals[pos] = val[c];
        }
    }
    __syncthreads();
    if (s_bad) return;  // offsets unknown: write nothing (the host reports the failure)
    const int tile_n = (int)min((int64_t)kOsTile, n - t0);
    for (int i = tid; i < tile_n; i += kOsThreads) {
        const uint64_t k = s_keys[i];
        const uint32_t d = (uint32_t)((k >> shift) & kMask);
        const unsigned long long g = s_gbase[d] + (unsigned long long)(i - (int)s_tstart[d]);
        if (g >= (unsigned long long)n) {  // inconsistent counts (cannot happen): never write out of bounds
            atomicOr(gave_up, 2u);
            continue;
        }
        if (kLast) {
            out.csr_src[g] = (int32_t)(k & ((1ull << src_bits) - 1));
            out.csr_dst[g] = (uint32_t)(k >> src_bits);
            out.perm[g] = s_vals[i];
        } else {
            out.keys[g] = k;
            out.vals[g] = s_vals[i];
        }
    }
}

// The passes for keys of `bits` bits: P = ceil(bits / 9) passes (at least
// one), the last max(0, bits - 8 P) of them 9 bits wide, the others 8 (50
// bits: 8, 8, 8, 8, 9, 9; 40 bits: five of 8).
static OsPasses os_passes(int bits) {
    OsPasses ps{};
    const int P = std::max(1, (bits + 8) / 9);
    const int nine = std::max(0, bits - 8 * P);  // <= P, as 9 P >= bits
    ps.n = P;
    int sh = 0;
    for (int p = 0; p < P; ++p) {
        ps.bits[p] = p >= P - nine ? 9 : 8;
        ps.shift[p] = sh;
        sh += ps.bits[p];
    }
    return ps;
}

template <int kBits>
static cudaError_t os_pass_attr(size_t smem) {
    const void* fns[4] = {(const void*)k_os_pass<true, false, kBits>, (const void*)k_os_pass<false, false, kBits>,
                          (const void*)k_os_pass<true, true, kBits>, (const void*)k_os_pass<false, true, kBits>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int kBits, bool kLast>
static void os_launch(bool first, int64_t ntiles, size_t smem, cudaStream_t st, const int32_t* src, const int32_t* dst,
                      int src_bits, const uint64_t* ksrc, const uint32_t* vsrc, const OsOut& out, int64_t m, int shift,
                      unsigned long long tag, const unsigned long long* base, unsigned long long* status,
                      unsigned int* ticket, unsigned int* gave_up) {
    if (first)
        k_os_pass<true, kLast, kBits><<<(unsigned)ntiles, kOsThreads, smem, st>>>(
            src, dst, src_bits, nullptr, nullptr, out, m, shift, tag, base, status, ticket, gave_up);
    else
        k_os_pass<false, kLast, kBits><<<(unsigned)ntiles, kOsThreads, smem, st>>>(
            nullptr, nullptr, src_bits, ksrc, vsrc, out, m, shift, tag, base, status, ticket, gave_up);
}

cudaError_t sort_edges(const int32_t* src, const int32_t* dst, int64_t m, int src_bits, int32_t* csr_src,
                       uint32_t* csr_dst, uint32_t* perm, uint64_t* keys_a, uint32_t* vals_a, uint64_t* keys_b,
                       uint32_t* vals_b, unsigned int* gave_up, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const OsPasses ps = os_passes(2 * src_bits);
    if (ps.n > kOsMaxPasses) return cudaErrorInvalidValue;
    const int passes = ps.n;
    const int64_t ntiles = (m + kOsTile - 1) / kOsTile;
    const size_t smem = (size_t)kOsTile * (sizeof(uint64_t) + sizeof(uint32_t));
    // set on every call: the attribute belongs to the current device
    cudaError_t attr_err = os_pass_attr<8>(smem);
    if (attr_err == cudaSuccess) attr_err = os_pass_attr<9>(smem);
    if (attr_err != cudaSuccess) return attr_err;
    unsigned long long *hist = nullptr, *status = nullptr;
    unsigned int* tickets = nullptr;
    cudaError_t e = dev_alloc_t(&hist, (size_t)passes * kOsMaxDigits, st);
    if (e == cudaSuccess) e = dev_alloc_t(&status, (size_t)ntiles * kOsMaxDigits, st);
    if (e == cudaSuccess) e = dev_alloc_t(&tickets, (size_t)passes, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(hist, 0, (size_t)passes * kOsMaxDigits * sizeof(unsigned long long), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(status, 0, (size_t)ntiles * kOsMaxDigits * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tickets, 0, (size_t)passes * sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        const int grid = (int)std::min<int64_t>((int64_t)sm_count() * 8, std::max<int64_t>(1, (m + 255) / 256));
        k_os_hist<<<grid, 256, 0, st>>>(src, dst, m, src_bits, ps, hist); note_launch();
        k_os_bases<<<1, kOsMaxDigits, 0, st>>>(hist, passes); note_launch();
        e = cudaGetLastError();
    }
    const uint64_t* ksrc = nullptr;
    const uint32_t* vsrc = nullptr;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        // passes alternate between the a and b buffers; the last one writes the CSR arrays
        const bool last = p == passes - 1;
        const OsOut out{p % 2 == 0 ? keys_a : keys_b, p % 2 == 0 ? vals_a : vals_b, csr_src, csr_dst, perm};
        const unsigned long long tag = (unsigned long long)(p + 1) << 56;
        const unsigned long long* base = hist + p * kOsMaxDigits;
        if (ps.bits[p] == 9) {
            if (last)
                os_launch<9, true>(p == 0, ntiles, smem, st, src, dst, src_bits, ksrc, vsrc, out, m, ps.shift[p], tag,
                                   base, status, tickets + p, gave_up);
            else
                os_launch<9, false>(p == 0, ntiles, smem, st, src, dst, src_bits, ksrc, vsrc, out, m, ps.shift[p], tag,
                                    base, status, tickets + p, gave_up);
        } else {
            if (last)
                os_launch<8, true>(p == 0, ntiles, smem, st, src, dst, src_bits, ksrc, vsrc, out, m, ps.shift[p], tag,
                                   base, status, tickets + p, gave_up);
            else
                os_launch<8, false>(p == 0, ntiles, smem, st, src, dst, src_bits, ksrc, vsrc, out, m, ps.shift[p], tag,
                                    base, status, tickets + p, gave_up);
        }
        note_launch();
        e = cudaGetLastError();
        ksrc = out.keys;
        vsrc = out.vals;
    }
    dev_free(hist, st);
    dev_free(status, st);
    dev_free(tickets, st);
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
