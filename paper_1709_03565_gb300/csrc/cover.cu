// Coverage counting and the SKIS estimator (Sec. IV, Eq. 21, Alg. 2) and
// greedy max-coverage (Sec. V-A, Alg. 3, Eq. margin) on the device sketch.
//
// Coverage: each query of a batch of up to 64 owns one bit of a per-vertex
// mask. A warp takes 32 consecutive samples, spreads their members over its
// lanes, ORs the members' masks per sample in shared memory and counts, per
// query bit, the samples whose OR has it (ballot + popcount). Counts and the
// estimator numerator are exact integers.
//
// Greedy: an inverted index vertex -> samples (counting sort), marginal
// coverage Delta_v, then per round an exact argmax of the integer key
// Delta_v W + T (2^f - w_v) (ties to the lowest id), and the samples of the
// chosen vertex are marked covered and their members' Delta decremented.
#include <cooperative_groups.h>

#include <algorithm>
#include <string>

#include "../../include/skis.h"
#include "skis_internal.cuh"

namespace skis {

constexpr int kCovThreads = 256;

// Calls f(owner_lane, member) for every member of the samples held by the
// lanes (lane i: arena offset off, length len), spread over the warp.
template <int kRuns = 2, class F>
__device__ __forceinline__ void warp_members(uint64_t off, uint32_t len, const int32_t* __restrict__ arena, F&& f) {
    static_assert(kRuns == 1 || kRuns == 2, "one or two runs of 32 members per pass");
    const int lane = threadIdx.x & 31;
    uint64_t incl = len;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    const uint64_t total = __shfl_sync(kFull, incl, 31);
    const uint64_t excl = incl - len;
    if constexpr (kRuns == 1) {
        for (uint64_t base = 0; base < total; base += 32) {
            const uint64_t p = base + lane;
            int owner = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint64_t v = __shfl_sync(kFull, incl, owner + step - 1);
                if (v <= p) owner += step;
            }
            const uint64_t o_off = __shfl_sync(kFull, off, owner);
            const uint64_t o_excl = __shfl_sync(kFull, excl, owner);
            if (p < total) f(owner, arena[o_off + (p - o_excl)]);
        }
    } else {
        // two runs of 32 members per pass: both member loads are in flight
        // before either member is handed to f
        for (uint64_t base = 0; base < total; base += 64) {
            const uint64_t p0 = base + lane, p1 = base + 32 + lane;
            int own0 = 0, own1 = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint64_t v0 = __shfl_sync(kFull, incl, own0 + step - 1);
                const uint64_t v1 = __shfl_sync(kFull, incl, own1 + step - 1);
                if (v0 <= p0) own0 += step;
                if (v1 <= p1) own1 += step;
            }
            const uint64_t off0 = __shfl_sync(kFull, off, own0), ex0 = __shfl_sync(kFull, excl, own0);
            const uint64_t off1 = __shfl_sync(kFull, off, own1), ex1 = __shfl_sync(kFull, excl, own1);
            int32_t u0 = 0, u1 = 0;
            if (p0 < total) u0 = arena[off0 + (p0 - ex0)];
            if (p1 < total) u1 = arena[off1 + (p1 - ex1)];
            if (p0 < total) f(own0, u0);
            if (p1 < total) f(own1, u1);
        }
    }
}

// Lanes adding to the same counter in one step (hub vertices recur across
// samples) are merged: one atomic per distinct address among the calling
// lanes, carrying the number of lanes.
__device__ __forceinline__ void add_aggregated(uint32_t* counter, int32_t u, int sign) {
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, u);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) {
        const uint32_t c = (uint32_t)__popc(peers);
        if (sign > 0) atomicAdd(&counter[u], c);
        else atomicSub(&counter[u], c);
    }
}

// Greedy's cover walk: a block-local table merges the decrements of vertices
// that recur across the samples a seed covers (hubs), so that each such
// vertex takes one global atomic per block and round instead of one per
// warp step. A vertex that finds its slot held by another goes straight to
// the global counter.
constexpr int kHotBits = 10;
constexpr int kHotSlots = 1 << kHotBits;
constexpr uint32_t kHotEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ void sub_merged(uint32_t* counter, int32_t u, uint32_t* hkey, uint32_t* hcnt) {
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, u);
    if ((threadIdx.x & 31) != __ffs(peers) - 1) return;
    const uint32_t c = (uint32_t)__popc(peers);
    const uint32_t slot = ((uint32_t)u * 2654435761u) >> (32 - kHotBits);
    uint32_t old = hkey[slot];
    if (old == kHotEmpty) old = atomicCAS(&hkey[slot], kHotEmpty, (uint32_t)u);
    if (old == kHotEmpty || old == (uint32_t)u) atomicAdd(&hcnt[slot], c);
    else atomicSub(&counter[u], c);
}

// ------------------------------------------------------------- coverage
// qbits (nullable): a filter of the batch's seeds, one bit per vertex for
// graphs of at most 2^20 vertices, else 2^20 bits indexed by a multiplicative
// hash, so that the sketch scan gathers a vertex's 8-byte mask only when the
// vertex may be a seed (false positives have an all-zero mask). At most
// 128 KiB: it fits in one block's shared memory.
constexpr int kFilterLog2 = 20;
constexpr uint32_t kFilterMaxWords = 1u << (kFilterLog2 - 5);

__host__ __device__ __forceinline__ uint32_t filter_words(int64_t n) {  // n in [1, 2^31]
    return n > ((int64_t)1 << kFilterLog2) ? kFilterMaxWords : (uint32_t)((n + 31) / 32);
}

__device__ __forceinline__ uint32_t filter_index(uint32_t v, int hashed) {
    return hashed ? (v * 2654435761u) >> (32 - kFilterLog2) : v;
}
__global__ void k_qmask_set(const int64_t* __restrict__ off, const int32_t* __restrict__ seeds, int32_t q0,
                            int32_t qn, int64_t n, uint64_t* __restrict__ qmask, uint32_t* __restrict__ qbits,
                            DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const int32_t b = q0 + (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (b >= q0 + qn) return;
    const int64_t lo = off[b], hi = off[b + 1];
    const uint64_t bit = 1ull << (b - q0);
    if (hi <= lo && lane == 0) {
        atomicOr(&st->flags, kStInval);
        atomicMin(&st->first_bad, (unsigned long long)b);
    }
    for (int64_t i = lo + lane; i < hi; i += 32) {
        const int32_t v = seeds[i];
        bool bad = v < 0 || v >= n;
        if (!bad) bad = (atomicOr((unsigned long long*)&qmask[v], (unsigned long long)bit) & bit) != 0;
        if (!bad && qbits) {
            const uint32_t f = filter_index((uint32_t)v, n > ((int64_t)1 << kFilterLog2));
            atomicOr(&qbits[f >> 5], 1u << (f & 31));
        }
        if (bad) {
            atomicOr(&st->flags, kStInval);
            atomicMin(&st->first_bad, (unsigned long long)b);
        }
    }
}

__global__ void k_qmask_clear(const int64_t* __restrict__ off, const int32_t* __restrict__ seeds, int32_t q0,
                              int32_t qn, int64_t n, uint64_t* __restrict__ qmask, uint32_t* __restrict__ qbits,
                              unsigned long long* __restrict__ reset2) {
    const int lane = threadIdx.x & 31;
    if (reset2 && blockIdx.x == 0 && threadIdx.x < 3) reset2[threadIdx.x] = 0;  // the ordered scan's counters
    const int32_t b = q0 + (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (b >= q0 + qn) return;
    for (int64_t i = off[b] + lane; i < off[b + 1]; i += 32) {
        const int32_t v = seeds[i];
        if (v >= 0 && v < n) {
            qmask[v] = 0;
            // every bit set in the filter belongs to a seed of this batch
            if (qbits) qbits[filter_index((uint32_t)v, n > ((int64_t)1 << kFilterLog2)) >> 5] = 0;
        }
    }
}

__global__ void __launch_bounds__(kCovThreads) k_coverage(const uint64_t* __restrict__ h_off,
                                                          const uint32_t* __restrict__ h_len, uint64_t T,
                                                          const int32_t* __restrict__ arena,
                                                          const uint64_t* __restrict__ qmask,
                                                          const uint32_t* __restrict__ qbits, int hashed,
                                                          unsigned long long* __restrict__ cov) {
    __shared__ unsigned long long s_acc[kCovThreads / 32][32];
    __shared__ unsigned long long s_cnt[64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (threadIdx.x < 64) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long c_lo = 0, c_hi = 0;  // counts of queries `lane` and `lane + 32`
    const uint64_t nwarps = (uint64_t)gridDim.x * (kCovThreads / 32);
    const uint64_t groups = (T + 31) / 32;
    for (uint64_t gidx = (uint64_t)blockIdx.x * (kCovThreads / 32) + wib; gidx < groups; gidx += nwarps) {
        const uint64_t j = gidx * 32 + lane;
        const bool valid = j < T;
        const uint64_t off = valid ? h_off[j] : 0;
        const uint32_t len = valid ? h_len[j] : 0;
        s_acc[wib][lane] = 0;
        __syncwarp();
        unsigned long long* acc_row = s_acc[wib];
        warp_members(off, len, arena, [&](int owner, int32_t u) {
            if (qbits) {  // not a seed
                const uint32_t f = filter_index((uint32_t)u, hashed);
                if (!((__ldg(qbits + (f >> 5)) >> (f & 31)) & 1u)) return;
            }
            const uint64_t msk = qmask[u];
            if (msk) atomicOr(&acc_row[owner], (unsigned long long)msk);
        });
        __syncwarp();
        const uint64_t acc = s_acc[wib][lane];
        uint64_t present = acc;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) present |= __shfl_xor_sync(kFull, present, d);
        while (present) {
            const int b = __ffsll((long long)present) - 1;
            present &= present - 1;
            const unsigned c = (unsigned)__popc(__ballot_sync(kFull, (acc >> b) & 1ull));
            if (lane == (b & 31)) {
                if (b < 32) c_lo += c;
                else c_hi += c;
            }
        }
    }
    if (c_lo) atomicAdd(&s_cnt[lane], c_lo);
    if (c_hi) atomicAdd(&s_cnt[lane + 32], c_hi);
    __syncthreads();
    if (threadIdx.x < 64 && s_cnt[threadIdx.x]) atomicAdd(&cov[threadIdx.x], s_cnt[threadIdx.x]);
}

// The scan of a sketch whose members are in sample-id order (arena
// positions [h_off[0], ...) contiguous): the seed filter sits in shared
// memory; a warp takes 1024 consecutive samples at a time (from an atomic
// cursor, so that warps meeting large samples or many seeds take fewer), whose
// members are one run, and streams it as 16-byte vectors testing each member
// against the filter. Only a member that is a seed (rare) looks up its
// sample, by a binary search over the task's 1024 offsets, and ORs its query
// mask into the sample's
// word of smask; the first setter of a (sample, query) bit counts it, and the
// first setter of a sample's word lists the sample for the reset.
constexpr int kScanThreads = 1024;

// Asynchronous bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned,
// bytes a multiple of 16): no register waits for it.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
constexpr uint32_t kScanSamples = 1024;
constexpr int kScanUnroll = 4;
constexpr uint64_t kScanAhead = 4;  // warp steps prefetched ahead
constexpr unsigned long long kHitCap = 1ull << 22;  // hits listed per query chunk (32 MiB); more are resolved in the scan

__global__ void __launch_bounds__(kScanThreads, 1) k_scan_ordered(
    const uint64_t* __restrict__ h_off, const uint32_t* __restrict__ h_len, uint64_t T,
    const int32_t* __restrict__ arena, const uint32_t* __restrict__ qbits, uint32_t fwords, int hashed,
    const uint64_t* __restrict__ qmask, unsigned long long* __restrict__ smask, uint32_t* __restrict__ touched,
    unsigned long long* __restrict__ ntouched, unsigned long long* __restrict__ cursor,
    unsigned long long* __restrict__ hits, unsigned long long* __restrict__ nhits, unsigned long long hit_cap,
    unsigned long long* __restrict__ cov) {
    extern __shared__ uint32_t s_f[];
    __shared__ unsigned int s_cnt[64];
    for (uint32_t i = threadIdx.x; i < fwords; i += blockDim.x) s_f[i] = qbits[i];
    if (threadIdx.x < 64) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t ntask = (T + kScanSamples - 1) / kScanSamples;
    unsigned long long claim = 0;
    if (lane == 0) claim = atomicAdd(cursor, 1ull);
    for (;;) {
        const unsigned long long task = __shfl_sync(kFull, claim, 0);
        if (task >= ntask) break;
        if (lane == 0) claim = atomicAdd(cursor, 1ull);  // the next task, claimed while this one streams
        const uint64_t j0 = task * kScanSamples, j1 = min(T, j0 + kScanSamples);
        const uint64_t p0 = h_off[j0], p1 = h_off[j1 - 1] + h_len[j1 - 1];
        auto member = [&](uint64_t pos, int32_t u) {
            const uint32_t f = filter_index((uint32_t)u, hashed);
            if (!((s_f[f >> 5] >> (f & 31)) & 1u)) return;
            // a possible seed: its (task, position) goes to the hit list for
            // k_scan_hits; only when the list is full is it resolved here
            const unsigned long long slot = atomicAdd(nhits, 1ull);
            if (slot < hit_cap) {
                hits[slot] = ((unsigned long long)task << 40) | pos;
                return;
            }
            const uint64_t msk = qmask[u];
            if (!msk) return;  // a filter collision
            uint64_t lo = j0, hi = j1 - 1;  // the last sample whose run starts at or before pos
            while (lo < hi) {
                const uint64_t mid = (lo + hi + 1) >> 1;
                if (h_off[mid] <= pos) lo = mid;
                else hi = mid - 1;
            }
            const unsigned long long old = atomicOr(smask + lo, (unsigned long long)msk);
            if (old == 0) touched[atomicAdd(ntouched, 1ull)] = (uint32_t)lo;
            for (uint64_t nb = msk & ~old; nb; nb &= nb - 1) atomicAdd(&s_cnt[__ffsll((long long)nb) - 1], 1u);
        };
        const uint64_t up = (p0 + 3) & ~(uint64_t)3, down = p1 & ~(uint64_t)3;
        const uint64_t ph = p1 < up ? p1 : up, pt = down > ph ? down : ph;
        if (p0 + lane < ph) member(p0 + lane, arena[p0 + lane]);
        const int4* a4 = reinterpret_cast<const int4*>(arena);
        const uint64_t v_end = pt / 4, v0 = ph / 4;
        // the task's first steps, then each step the one kScanAhead steps on, are
        // prefetched into L2 by one lane, so that the lanes' loads find them there
        constexpr uint64_t kStep = 32 * kScanUnroll;  // 16-byte vectors a warp step loads
        if (lane == 0 && v0 < v_end)
            prefetch_l2(a4 + v0, (uint32_t)(min(v_end - v0, kStep * kScanAhead) * 16));
        uint64_t v = v0 + lane;
        // kScanUnroll 16-byte loads in flight a lane before any member is tested
        // (the last step of a task predicated, not a step per load)
        for (; v < v_end; v += 32 * kScanUnroll) {
            const uint64_t ahead = (v - lane) + kStep * kScanAhead;
            if (lane == 0 && ahead < v_end) prefetch_l2(a4 + ahead, (uint32_t)(min(v_end - ahead, kStep) * 16));
            int4 m[kScanUnroll];
#pragma unroll
            for (int k = 0; k < kScanUnroll; ++k)
                if (v + 32 * k < v_end) m[k] = __ldcs(a4 + v + 32 * k);
#pragma unroll
            for (int k = 0; k < kScanUnroll; ++k) {
                if (v + 32 * k >= v_end) break;
                const uint64_t pos = (v + 32 * k) * 4;
                member(pos, m[k].x);
                member(pos + 1, m[k].y);
                member(pos + 2, m[k].z);
                member(pos + 3, m[k].w);
            }
        }
        if (pt + lane < p1) member(pt + lane, arena[pt + lane]);
    }
    __syncthreads();
    if (threadIdx.x < 64 && s_cnt[threadIdx.x]) atomicAdd(&cov[threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
}

// The hits the scan listed: each (task, position) resolves to its member,
// the member's query mask, and its sample by a binary search over the task's
// offsets; the first setter of a (sample, query) bit counts it.
__global__ void __launch_bounds__(256) k_scan_hits(const unsigned long long* __restrict__ hits,
                                                   const unsigned long long* __restrict__ nhits,
                                                   unsigned long long hit_cap, const uint64_t* __restrict__ h_off,
                                                   uint64_t T, const int32_t* __restrict__ arena,
                                                   const uint64_t* __restrict__ qmask,
                                                   unsigned long long* __restrict__ smask,
                                                   uint32_t* __restrict__ touched,
                                                   unsigned long long* __restrict__ ntouched,
                                                   unsigned long long* __restrict__ cov) {
    __shared__ unsigned int s_cnt[64];
    if (threadIdx.x < 64) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t cnt = min((uint64_t)*nhits, (uint64_t)hit_cap);
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long h = hits[k];
        const uint64_t pos = h & ((1ull << 40) - 1), task = h >> 40;
        const uint64_t msk = qmask[arena[pos]];
        if (!msk) continue;  // a filter collision
        uint64_t lo = task * kScanSamples, hi = min(T, lo + kScanSamples) - 1;
        while (lo < hi) {
            const uint64_t mid = (lo + hi + 1) >> 1;
            if (h_off[mid] <= pos) lo = mid;
            else hi = mid - 1;
        }
        const unsigned long long old = atomicOr(smask + lo, (unsigned long long)msk);
        if (old == 0) touched[atomicAdd(ntouched, 1ull)] = (uint32_t)lo;
        for (uint64_t nb = msk & ~old; nb; nb &= nb - 1) atomicAdd(&s_cnt[__ffsll((long long)nb) - 1], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 64 && s_cnt[threadIdx.x]) atomicAdd(&cov[threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
}

__global__ void k_unmark(const uint32_t* __restrict__ touched, const unsigned long long* __restrict__ ntouched,
                         unsigned long long* __restrict__ smask) {
    const uint64_t cnt = *ntouched;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += (uint64_t)gridDim.x * blockDim.x)
        smask[touched[k]] = 0;
}

// Eq. 21 with exact integers: N = Cov W + T sum_{v in S} (2^f - w_v),
// D = T 2^f, estimate = N / D.
__global__ void k_estimate(const int64_t* __restrict__ off, const int32_t* __restrict__ seeds, int32_t q0,
                           int32_t qn, int64_t n, const uint64_t* __restrict__ w, int f, uint64_t W, uint64_t T,
                           const unsigned long long* __restrict__ cov, int64_t* __restrict__ cov_out,
                           double* __restrict__ est_out, int ris) {
    const int lane = threadIdx.x & 31;
    const int32_t b = q0 + (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (b >= q0 + qn) return;
    const uint64_t one_f = 1ull << f;
    uint64_t s = 0;  // <= |S| 2^f <= 2^61
    for (int64_t i = off[b] + lane; i < off[b + 1]; i += 32) {
        const int32_t v = seeds[i];
        if (v >= 0 && v < n) s += one_f - w[v];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(kFull, s, d);
    if (lane == 0) {
        const uint64_t c = cov[b - q0];
        // RIS (Lemma 1): n Cov / T; SKIS (Eq. 21): (Cov W + T sum) / (T 2^f)
        const u128 N = ris ? (u128)c * (uint64_t)n : (u128)c * W + (u128)T * s;
        const u128 D = ris ? (u128)T : (u128)T << f;
        if (cov_out) cov_out[b] = (int64_t)c;
        est_out[b] = u128_to_double(N) / u128_to_double(D);
    }
}

#define CV_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) {                                                   \
            *err = std::string(where) + ": CUDA error: " + cudaGetErrorString(_e); \
            return _e == cudaErrorMemoryAllocation ? SKIS_ENOMEM : SKIS_ERR_CUDA;  \
        }                                                                          \
    } while (0)

static int coverage_blocks(uint64_t T) {
    const uint64_t groups = (T + 31) / 32;
    const uint64_t want = (groups + (kCovThreads / 32) - 1) / (kCovThreads / 32);
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sm_count() * 8));
}

// ------------------------------------------- coverage by inverted index
// Cov_R(S) for small seed sets: walk the sample list of every seed and set
// the query's bit in a per-sample mask; the first setter of (sample, query)
// counts it. Lists are cut into chunks of kInvChunk entries; one warp takes
// one chunk, found by binary search over the batch's chunk prefix sums.
constexpr uint32_t kInvChunk = 2048;

__global__ void k_seed_chunks(const int32_t* __restrict__ seeds, int64_t seed_base, int64_t nseeds, int64_t n,
                              const uint64_t* __restrict__ inv_off, uint32_t* __restrict__ chunk_cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nseeds; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = seeds[seed_base + i];
        uint32_t c = 0;
        if (v >= 0 && v < n) c = (uint32_t)((inv_off[v + 1] - inv_off[v] + kInvChunk - 1) / kInvChunk);
        chunk_cnt[i] = c;
    }
}

__global__ void __launch_bounds__(kCovThreads) k_cover_inv(const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ seeds, int32_t q0, int32_t qn,
                                                           int64_t seed_base, int64_t nseeds,
                                                           const uint64_t* __restrict__ chunk_off,
                                                           const uint64_t* __restrict__ inv_off,
                                                           const uint32_t* __restrict__ inv,
                                                           uint64_t* __restrict__ smask,
                                                           unsigned long long* __restrict__ cov, int clear) {
    const int lane = threadIdx.x & 31;
    const uint64_t C = chunk_off[nseeds];
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t c = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; c < C; c += nwarps) {
        int64_t lo = 0, hi = nseeds - 1;  // last seed i with chunk_off[i] <= c
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (chunk_off[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        const int64_t i = lo;
        int32_t blo = q0, bhi = q0 + qn - 1;  // last query b with off[b] <= seed_base + i
        while (blo < bhi) {
            const int32_t mid = (blo + bhi + 1) / 2;
            if (off[mid] <= seed_base + i) blo = mid;
            else bhi = mid - 1;
        }
        const uint64_t bit = 1ull << (blo - q0);
        const int32_t v = seeds[seed_base + i];
        const uint64_t start = inv_off[v] + (c - chunk_off[i]) * kInvChunk;
        const uint64_t end = min(start + kInvChunk, inv_off[v + 1]);
        uint32_t fresh = 0;
        for (uint64_t x = start + lane; x < end; x += 32) {
            const uint32_t j = inv[x];
            if (clear) {
                smask[j] = 0;
            } else {
                const unsigned long long old = atomicOr((unsigned long long*)&smask[j], (unsigned long long)bit);
                fresh += (old & bit) ? 0u : 1u;
            }
        }
        if (!clear) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) fresh += __shfl_down_sync(kFull, fresh, d);
            if (lane == 0 && fresh) atomicAdd(&cov[blo - q0], (unsigned long long)fresh);
        }
    }
}

cudaError_t coverage_by_index(const skis_sketch* s, const int64_t* off, const int32_t* seeds, int32_t q0,
                              int32_t qn, int64_t seed_base, int64_t nseeds, uint32_t* chunk_cnt,
                              uint64_t* chunk_off, uint64_t* smask, unsigned long long* cov, cudaStream_t st) {
    if (nseeds <= 0) return cudaSuccess;
    const int b1 = (int)std::max<int64_t>(1, std::min<int64_t>((nseeds + 255) / 256, (int64_t)sm_count() * 4));
    k_seed_chunks<<<b1, 256, 0, st>>>(seeds, seed_base, nseeds, s->g->n, s->inv_off, chunk_cnt); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_u32_to_u64(chunk_cnt, chunk_off, nseeds, st);
    if (e != cudaSuccess) return e;
    const int b2 = sm_count() * 8;
    k_cover_inv<<<b2, kCovThreads, 0, st>>>(off, seeds, q0, qn, seed_base, nseeds, chunk_off, s->inv_off, s->inv,
                                            smask, cov, 0); note_launch();
    k_cover_inv<<<b2, kCovThreads, 0, st>>>(off, seeds, q0, qn, seed_base, nseeds, chunk_off, s->inv_off, s->inv,
                                            smask, cov, 1); note_launch();
    return cudaGetLastError();
}

// Members of samples [0, cnt) (headers off/len) copied to out in sample
// order at their exclusive prefix pre: a warp takes 32 consecutive samples
// and spreads their members over its lanes, so the writes are one
// contiguous run.
__global__ void __launch_bounds__(kCovThreads) k_order_members(const uint64_t* __restrict__ off,
                                                               const uint32_t* __restrict__ len, uint64_t cnt,
                                                               const uint64_t* __restrict__ pre,
                                                               const int32_t* __restrict__ arena,
                                                               int32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (kCovThreads / 32);
    for (uint64_t gi = ((uint64_t)blockIdx.x * kCovThreads + threadIdx.x) / 32; gi * 32 < cnt; gi += nwarps) {
        const uint64_t j = gi * 32 + lane;
        const uint64_t o = j < cnt ? off[j] : 0;
        const uint32_t l = j < cnt ? len[j] : 0u;
        uint32_t incl = l;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31), excl = incl - l;
        const uint64_t dst0 = pre[gi * 32];
        for (uint32_t base = 0; base < total; base += 32) {  // warp-uniform: every lane shuffles
            const uint32_t p = base + lane;
            int owner = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint32_t v = __shfl_sync(kFull, incl, owner + step - 1);
                if (v <= p) owner += step;
            }
            const uint64_t oo = __shfl_sync(kFull, o, owner);
            const uint32_t oe = __shfl_sync(kFull, excl, owner);
            if (p < total) out[dst0 + p] = arena[oo + (p - oe)];
        }
    }
}

__global__ void k_rebase_offsets(uint64_t* __restrict__ off, const uint64_t* __restrict__ pre, uint64_t cnt,
                                 uint64_t base) {
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += (uint64_t)gridDim.x * blockDim.x)
        off[j] = base + pre[j];
}

int sketch_order_arena(skis_sketch* s, cudaStream_t st, std::string* err) {
    const char* where = "member layout";
    if (s->ordered_T == s->T) return SKIS_OK;
    const uint64_t T0 = s->ordered_T, cnt = s->T - T0, E0 = s->ordered_E;
    uint64_t* pre = nullptr;
    int32_t* tmp = nullptr;
    uint64_t E1 = 0;
    auto body = [&]() -> int {
        CV_CUDA(dev_alloc_t(&pre, (size_t)cnt + 1, st));
        CV_CUDA(scan_u32_to_u64(s->h_len + T0, pre, (int64_t)cnt, st));
        CV_CUDA(cudaMemcpyAsync(&E1, pre + cnt, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        CV_CUDA(cudaStreamSynchronize(st));
        CV_CUDA(dev_alloc_t(&tmp, (size_t)std::max<uint64_t>(E1, 1), st));
        const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * 8,
                                                                         (cnt + kCovThreads - 1) / kCovThreads));
        k_order_members<<<blocks, kCovThreads, 0, st>>>(s->h_off + T0, s->h_len + T0, cnt, pre, s->arena, tmp);
        note_launch();
        CV_CUDA(cudaGetLastError());
        if (E1) CV_CUDA(cudaMemcpyAsync(s->arena + E0, tmp, E1 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        k_rebase_offsets<<<blocks, kCovThreads, 0, st>>>(s->h_off + T0, pre, cnt, E0); note_launch();
        CV_CUDA(cudaGetLastError());
        if (s->ctr) {  // later samples are appended right after the ordered ones
            const unsigned long long cur = E0 + E1;
            CV_CUDA(cudaMemcpyAsync(&s->ctr->arena, &cur, sizeof(cur), cudaMemcpyHostToDevice, st));
        }
        CV_CUDA(cudaStreamSynchronize(st));
        return SKIS_OK;
    };
    const int rc = body();
    dev_free(pre, st);
    dev_free(tmp, st);
    if (rc == SKIS_OK) {
        s->ordered_T = s->T;
        s->ordered_E = E0 + E1;
    }
    return rc;
}

int sketch_estimate(skis_sketch* s, int32_t q, const int64_t* d_off, const int32_t* d_seeds, const int64_t* h_off,
                    int64_t* d_cov, double* d_est, cudaStream_t st, std::string* err) {
    const char* where = "skis_estimate";
    const skis_graph* g = s->g;
    if (s->T == 0) {
        *err = "skis_estimate: the sketch has no samples";
        return SKIS_EINVAL;
    }
    if (s->query_index == 1) {
        const int rc = sketch_inverted(s, st, err);
        if (rc != SKIS_OK) return rc;
    }
    const bool by_index = s->query_index < 2 && s->inv && s->inv_T == s->T;
    // a large sketch is scanned with its members in sample-id order (laid out
    // once per new samples); a small one (below 2^20 samples: doubling rounds,
    // tests) directly, where that one-time layout would cost more than it saves
    const bool ordered_scan = !by_index && (s->T >= (1ull << 20) || s->query_index == 3) && s->T < (1ull << 32);
    if (ordered_scan) {
        const int rc = sketch_order_arena(s, st, err);
        if (rc != SKIS_OK) return rc;
    }
    const uint32_t fwords = filter_words(g->n);
    const int hashed = g->n > ((int64_t)1 << kFilterLog2);
    if (!s->qmask) {
        CV_CUDA(dev_alloc_t(&s->qmask, (size_t)g->n, st));
        CV_CUDA(cudaMemsetAsync(s->qmask, 0, (size_t)g->n * sizeof(uint64_t), st));
        CV_CUDA(dev_alloc_t(&s->qbits, (size_t)fwords, st));
        CV_CUDA(cudaMemsetAsync(s->qbits, 0, (size_t)fwords * sizeof(uint32_t), st));
        CV_CUDA(dev_alloc_t(&s->qcov, 64, st));
        CV_CUDA(dev_alloc_t(&s->qstatus, 1, st));
        CV_CUDA(cudaEventCreate(&s->qev[0]));
        CV_CUDA(cudaEventCreate(&s->qev[1]));
    }
    uint32_t* chunk_cnt = nullptr;
    uint64_t* chunk_off = nullptr;
    if (ordered_scan && s->touched_cap < s->T) {
        dev_free(s->touched, st);
        s->touched = nullptr;
        CV_CUDA(dev_alloc_t(&s->touched, (size_t)s->T, st));
        if (!s->ntouched) {  // list count, task cursor and hit count, zero between calls (k_qmask_clear resets them)
            CV_CUDA(dev_alloc_t(&s->ntouched, 3, st));
            CV_CUDA(cudaMemsetAsync(s->ntouched, 0, 3 * sizeof(unsigned long long), st));
            CV_CUDA(dev_alloc_t(&s->hits, (size_t)kHitCap, st));
        }
        s->touched_cap = s->T;
    }
    if (by_index || ordered_scan) {
        if (s->smask_cap < s->T) {
            dev_free(s->smask, st);
            s->smask = nullptr;
            CV_CUDA(dev_alloc_t(&s->smask, (size_t)s->T, st));
            CV_CUDA(cudaMemsetAsync(s->smask, 0, (size_t)s->T * sizeof(uint64_t), st));
            s->smask_cap = s->T;
        }
    }
    if (by_index) {
        int64_t most = 1;
        for (int32_t q0 = 0; q0 < q; q0 += 64)
            most = std::max<int64_t>(most, h_off[std::min<int32_t>(q, q0 + 64)] - h_off[q0]);
        CV_CUDA(dev_alloc_t(&chunk_cnt, (size_t)most, st));
        CV_CUDA(dev_alloc_t(&chunk_off, (size_t)most + 1, st));
    }
    if (ordered_scan)  // the filter takes up to 128 KiB of dynamic shared memory
        CV_CUDA(cudaFuncSetAttribute(k_scan_ordered, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kFilterMaxWords * sizeof(uint32_t))));
    CV_CUDA(cudaMemsetAsync(s->qstatus, 0, sizeof(DevStatus), st));
    CV_CUDA(cudaMemsetAsync(&s->qstatus->first_bad, 0xFF, sizeof(unsigned long long), st));
    const int cblocks = coverage_blocks(s->T);
    float query_ms = 0;
    for (int32_t q0 = 0; q0 < q; q0 += 64) {
        const int32_t qn = std::min<int32_t>(64, q - q0);
        const int wb = div_up((int64_t)qn * 32, 256);
        CV_CUDA(cudaMemsetAsync(s->qcov, 0, 64 * sizeof(unsigned long long), st));
        k_qmask_set<<<wb, 256, 0, st>>>(d_off, d_seeds, q0, qn, g->n, s->qmask, s->qbits, s->qstatus); note_launch();
        CV_CUDA(cudaGetLastError());
        CV_CUDA(cudaEventRecord(s->qev[0], st));
        if (by_index) {
            CV_CUDA(coverage_by_index(s, d_off, d_seeds, q0, qn, h_off[q0], h_off[q0 + qn] - h_off[q0], chunk_cnt,
                                      chunk_off, s->smask, s->qcov, st));
        } else if (ordered_scan) {
            k_scan_ordered<<<sm_count(), kScanThreads, fwords * sizeof(uint32_t), st>>>(
                s->h_off, s->h_len, s->T, s->arena, s->qbits, fwords, hashed, s->qmask,
                reinterpret_cast<unsigned long long*>(s->smask), s->touched, s->ntouched, s->ntouched + 1, s->hits,
                s->ntouched + 2, kHitCap, s->qcov);
            note_launch();
            CV_CUDA(cudaGetLastError());
            k_scan_hits<<<sm_count() * 8, 256, 0, st>>>(s->hits, s->ntouched + 2, kHitCap, s->h_off, s->T, s->arena,
                                                        s->qmask, reinterpret_cast<unsigned long long*>(s->smask),
                                                        s->touched, s->ntouched, s->qcov);
            note_launch();
            CV_CUDA(cudaGetLastError());
            k_unmark<<<sm_count() * 4, 256, 0, st>>>(s->touched, s->ntouched,
                                                     reinterpret_cast<unsigned long long*>(s->smask));
            note_launch();
            CV_CUDA(cudaGetLastError());
        } else {
            k_coverage<<<cblocks, kCovThreads, 0, st>>>(s->h_off, s->h_len, s->T, s->arena, s->qmask, s->qbits, hashed,
                                                        s->qcov);
            note_launch();
            CV_CUDA(cudaGetLastError());
        }
        CV_CUDA(cudaEventRecord(s->qev[1], st));
        k_estimate<<<wb, 256, 0, st>>>(d_off, d_seeds, q0, qn, g->n, g->w, g->f, g->W, s->T, s->qcov, d_cov, d_est,
                                       s->ris); note_launch();
        CV_CUDA(cudaGetLastError());
        k_qmask_clear<<<wb, 256, 0, st>>>(d_off, d_seeds, q0, qn, g->n, s->qmask, s->qbits,
                                          ordered_scan ? s->ntouched : nullptr); note_launch();
        CV_CUDA(cudaGetLastError());
    }
    dev_free(chunk_cnt, st);
    dev_free(chunk_off, st);
    DevStatus h;
    CV_CUDA(cudaMemcpyAsync(&h, s->qstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    if (q > 0 && q <= 64) {  // the device time of the coverage launches (one chunk of queries)
        cudaEventElapsedTime(&query_ms, s->qev[0], s->qev[1]);
        s->last_query_ms = query_ms;
    }
    if (h.flags & kStInval) {
        *err = "skis_estimate: query " + std::to_string(h.first_bad) +
               " is empty, has a seed outside [0, n) or repeats a seed";
        return SKIS_EINVAL;
    }
    return SKIS_OK;
}

// --------------------------------------------------------------- greedy
__global__ void __launch_bounds__(kCovThreads) k_count_members(const uint64_t* __restrict__ h_off,
                                                               const uint32_t* __restrict__ h_len, uint64_t T,
                                                               const int32_t* __restrict__ arena,
                                                               uint32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * (kCovThreads / 32);
    const uint64_t groups = (T + 31) / 32;
    for (uint64_t gidx = (uint64_t)blockIdx.x * (kCovThreads / 32) + wib; gidx < groups; gidx += nwarps) {
        const uint64_t j = gidx * 32 + lane;
        const bool valid = j < T;
        warp_members(valid ? h_off[j] : 0, valid ? h_len[j] : 0u, arena,
                     [&](int, int32_t u) { add_aggregated(cnt, u, +1); });
    }
}

__global__ void __launch_bounds__(kCovThreads) k_fill_inverted(const uint64_t* __restrict__ h_off,
                                                               const uint32_t* __restrict__ h_len, uint64_t T,
                                                               const int32_t* __restrict__ arena,
                                                               const uint64_t* __restrict__ inv_off,
                                                               uint32_t* __restrict__ fill,
                                                               uint32_t* __restrict__ inv) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * (kCovThreads / 32);
    const uint64_t groups = (T + 31) / 32;
    for (uint64_t gidx = (uint64_t)blockIdx.x * (kCovThreads / 32) + wib; gidx < groups; gidx += nwarps) {
        const uint64_t j0 = gidx * 32;
        const uint64_t j = j0 + lane;
        const bool valid = j < T;
        // one slot reservation per entry: lanes rarely share a vertex, and
        // the atomics of those that do are served at L2 in turn
        // one run per pass keeps this latency-bound kernel at 32 registers
        // and every warp slot
        warp_members<1>(valid ? h_off[j] : 0, valid ? h_len[j] : 0u, arena, [&](int owner, int32_t u) {
            const uint32_t pos = atomicAdd(&fill[u], 1u);
            inv[inv_off[u] + pos] = (uint32_t)(j0 + owner);
        });
    }
}

struct KeyId {
    u128 key;
    uint32_t id;
    uint32_t valid;
    uint32_t d;    // Delta of the vertex (carried with the key)
    uint32_t pad;
};

__device__ __forceinline__ bool better(const KeyId& a, const KeyId& b) {
    if (a.valid != b.valid) return a.valid > b.valid;
    if (a.key != b.key) return a.key > b.key;
    return a.id < b.id;
}

__device__ __forceinline__ KeyId shfl_down_keyid(const KeyId& x, int d) {
    KeyId y;
    y.key = shfl_down_u128(x.key, d);
    y.id = __shfl_down_sync(kFull, x.id, d);
    y.valid = __shfl_down_sync(kFull, x.valid, d);
    y.d = __shfl_down_sync(kFull, x.d, d);
    y.pad = 0;
    return y;
}

__device__ __forceinline__ KeyId shfl_keyid(const KeyId& x, int src) {
    KeyId y;
    y.key = ((u128)__shfl_sync(kFull, (unsigned long long)(x.key >> 64), src) << 64) |
            (u128)__shfl_sync(kFull, (unsigned long long)x.key, src);
    y.id = __shfl_sync(kFull, x.id, src);
    y.valid = __shfl_sync(kFull, x.valid, src);
    y.d = __shfl_sync(kFull, x.d, src);
    y.pad = 0;
    return y;
}

__device__ KeyId block_best(KeyId b, KeyId* s_part) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const KeyId o = shfl_down_keyid(b, d);
        if (better(o, b)) b = o;
    }
    if (lane == 0) s_part[wib] = b;
    __syncthreads();
    if (wib == 0) {
        b = lane < (int)(blockDim.x / 32) ? s_part[lane] : KeyId{0, 0xFFFFFFFFu, 0};
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const KeyId o = shfl_down_keyid(b, d);
            if (better(o, b)) b = o;
        }
    }
    return b;  // valid in thread 0
}

struct GreedyArgs {
    const uint64_t* w;
    uint8_t* inS;
    uint32_t* delta;
    int64_t n;
    uint64_t W, T;
    int f;
    int32_t k;
    const uint64_t* inv_off;
    const uint32_t* inv;
    const uint64_t* h_off;
    const uint32_t* h_len;
    const int32_t* arena;
    uint32_t* covered;
    KeyId* partial;
    KeyId* seg_best;  // per segment of kGreedySeg vertices: its best of the last scan
    int64_t nseg;
    int32_t* seeds;
    int64_t* cov_out;
    double* est_out;
    int ris;
};


__device__ __forceinline__ KeyId ldcg_keyid(const KeyId* p) {
    const unsigned long long* q = reinterpret_cast<const unsigned long long*>(p);
    KeyId c;
    c.key = ((u128)__ldcg(q + 1) << 64) | (u128)__ldcg(q);
    const unsigned long long tail = __ldcg(q + 2);
    c.id = (uint32_t)tail;
    c.valid = (uint32_t)(tail >> 32);
    c.d = (uint32_t)__ldcg(q + 3);
    c.pad = 0;
    return c;
}

// All k rounds of Alg. 3 in one cooperative launch, one block per SM. Per
// round: every block scans its share of the vertices for the exact key
// Delta_v W + T (2^f - w_v) (v outside S, ties to the lowest id) and writes
// its best; a grid barrier; every block reduces all the blocks' bests itself
// (the same winner everywhere, no atomic hand-off) and block 0 records it;
// every warp walks the winner's inverted list, marking uncovered samples and
// decrementing their members' Delta (hub decrements merged per block); a grid
// barrier. Every block executes the same sequence of barriers. Data that
// other blocks change during the launch (Delta, the block bests) is read
// through L2 (ld.global.cg), never from a possibly stale L1 line.
constexpr int kGreedyThreads = 1024;
constexpr int kGreedySegLog = 8;  // vertices per segment: 256
constexpr int64_t kGreedySeg = 1ll << kGreedySegLog;
constexpr uint32_t kBigLen = 256;   // covered samples longer than this are walked by the whole block
constexpr int kBigQueue = 64;

__global__ void __launch_bounds__(kGreedyThreads, 1) k_greedy_rounds(GreedyArgs a) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    __shared__ KeyId s_part[kGreedyThreads / 32];
    __shared__ KeyId s_win;
    __shared__ uint32_t s_hkey[kHotSlots], s_hcnt[kHotSlots];
    __shared__ uint64_t s_big_off[kBigQueue];
    __shared__ uint32_t s_big_len[kBigQueue];
    __shared__ uint32_t s_nbig;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t one_f = 1ull << a.f;
    const int nw = kGreedyThreads / 32;
    for (int i = threadIdx.x; i < kHotSlots; i += blockDim.x) {
        s_hkey[i] = kHotEmpty;
        s_hcnt[i] = 0;
    }
    if (threadIdx.x == 0) s_nbig = 0;
    uint64_t cov = 0, sum_c = 0;  // running totals, kept by block 0
    __syncthreads();
    for (int32_t round = 0; round < a.k; ++round) {
        // the best outside S: each lane holds one segment's best at a time.
        // Keys only decrease, so a segment whose best is still outside S
        // with an unchanged Delta keeps it (every other key is at most what
        // it was; ties keep the lowest id), and a segment with no vertex
        // outside S stays so; the others are rescanned, one warp each.
        // warp gw of W takes segments gw + W i, 32 of them at a time (lane l:
        // gw + W (32 i + l)); the block index varies fastest over gw, so a
        // few segments already spread over every SM
        KeyId wbest{0, 0xFFFFFFFFu, 0};
        const int64_t W = (int64_t)gridDim.x * nw, gw = (int64_t)wib * gridDim.x + blockIdx.x;
        for (int64_t g0 = gw; g0 < a.nseg; g0 += 32 * W) {
            const int64_t sg = g0 + lane * W;
            KeyId b{0, 0xFFFFFFFFu, 0};
            bool ok = sg >= a.nseg;
            if (!ok && round > 0) {
                b = ldcg_keyid(a.seg_best + sg);
                ok = !b.valid || (!__ldcg(a.inS + b.id) && __ldcg(a.delta + b.id) == b.d);
            }
            unsigned redo = __ballot_sync(kFull, !ok);
            while (redo) {
                const int src = __ffs(redo) - 1;
                redo &= redo - 1;
                const int64_t v_lo = (g0 + src * W) << kGreedySegLog, v_hi = min(a.n, v_lo + kGreedySeg);
                KeyId r{0, 0xFFFFFFFFu, 0};
                // four of the lane's vertices per pass, their loads issued together
                for (int64_t v0 = v_lo + lane; v0 < v_hi; v0 += 128) {
                    uint8_t in4[4];
                    uint32_t d4[4];
                    uint64_t w4[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int64_t v = v0 + 32 * q;
                        in4[q] = 1;
                        if (v < v_hi) {
                            in4[q] = __ldcg(a.inS + v);
                            d4[q] = __ldcg(a.delta + v);
                            w4[q] = a.w[v];
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (in4[q]) continue;
                        const u128 dv = (u128)d4[q];
                        const KeyId c{a.ris ? dv : dv * a.W + (u128)a.T * (one_f - w4[q]), (uint32_t)(v0 + 32 * q),
                                      1u, d4[q], 0u};
                        if (better(c, r)) r = c;
                    }
                }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) {
                    const KeyId o = shfl_down_keyid(r, d);
                    if (better(o, r)) r = o;
                }
                r = shfl_keyid(r, 0);
                if (lane == src) b = r;
                if (lane == 0) a.seg_best[g0 + src * W] = r;
            }
            if (better(b, wbest)) wbest = b;
        }
        const KeyId best = block_best(wbest, s_part);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = best;
        grid.sync();
        if (wib == 0) {
            KeyId b{0, 0xFFFFFFFFu, 0};
            for (unsigned i = lane; i < gridDim.x; i += 32) {
                const KeyId c = ldcg_keyid(a.partial + i);
                if (better(c, b)) b = c;
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const KeyId o = shfl_down_keyid(b, d);
                if (better(o, b)) b = o;
            }
            if (lane == 0) s_win = b;
        }
        __syncthreads();
        const uint32_t v = s_win.id;
        if (threadIdx.x == 0) {
            if (blockIdx.x == 0) {
                a.inS[v] = 1;  // read (through L2) after the round's last grid barrier
                cov += s_win.d;  // Delta_v as scanned, before any walk of this round
                sum_c += one_f - a.w[v];
                a.seeds[round] = (int32_t)v;
                a.cov_out[round] = (int64_t)cov;
                const u128 N = a.ris ? (u128)cov * (uint64_t)a.n : (u128)cov * a.W + (u128)a.T * sum_c;
                const u128 D = a.ris ? (u128)a.T : (u128)a.T << a.f;
                a.est_out[round] = u128_to_double(N) / u128_to_double(D);
            }
        }
        __syncthreads();
        // cover the uncovered samples of the committed vertex
        // a warp takes spw list entries at a time, spw the power of two that
        // spreads the list over every warp (up to 32), so a short list is
        // not walked by a few warps one member at a time
        const uint64_t lo = a.inv_off[v], cnt = a.inv_off[v + 1] - lo;
        const uint64_t nwarps = (uint64_t)gridDim.x * (kGreedyThreads / 32);
        uint32_t spw = 1;
        while (spw < 32 && (uint64_t)spw * nwarps < cnt) spw <<= 1;
        for (uint64_t base = ((uint64_t)blockIdx.x * (kGreedyThreads / 32) + wib) * spw; base < cnt;
             base += nwarps * spw) {
            const uint64_t x = base + lane;
            uint64_t off = 0;
            uint32_t len = 0;
            if ((uint32_t)lane < spw && x < cnt) {
                const uint32_t j = a.inv[lo + x];
                const uint32_t bit = 1u << (j & 31);
                if ((atomicOr(&a.covered[j >> 5], bit) & bit) == 0) {
                    off = a.h_off[j];
                    len = a.h_len[j];
                    if (len > kBigLen) {  // a large sample: the whole block walks it below
                        const uint32_t q = atomicAdd(&s_nbig, 1u);
                        if (q < (uint32_t)kBigQueue) {
                            s_big_off[q] = off;
                            s_big_len[q] = len;
                            len = 0;
                        }
                    }
                }
            }
            warp_members(off, len, a.arena, [&](int, int32_t u) { sub_merged(a.delta, u, s_hkey, s_hcnt); });
        }
        __syncthreads();
        const uint32_t nbig = min(s_nbig, (uint32_t)kBigQueue);
        for (uint32_t b = 0; b < nbig; ++b) {
            const uint64_t boff = s_big_off[b];
            const uint32_t blen = s_big_len[b];
            for (uint32_t i = threadIdx.x; i < blen; i += blockDim.x) sub_merged(a.delta, a.arena[boff + i], s_hkey, s_hcnt);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nbig = 0;
        for (int i = threadIdx.x; i < kHotSlots; i += blockDim.x) {
            const uint32_t key = s_hkey[i];
            if (key != kHotEmpty) {
                atomicSub(&a.delta[key], s_hcnt[i]);
                s_hkey[i] = kHotEmpty;
                s_hcnt[i] = 0;
            }
        }
        grid.sync();
    }
}

__global__ void k_delta_from_index(const uint64_t* __restrict__ inv_off, int64_t n, uint32_t* __restrict__ delta) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        delta[v] = (uint32_t)(inv_off[v + 1] - inv_off[v]);
}

int sketch_inverted(skis_sketch* s, cudaStream_t st, std::string* err) {
    const char* where = "inverted index";
    if (s->inv && s->inv_T == s->T) return SKIS_OK;
    const int64_t n = s->g->n;
    const uint64_t T = s->T;
    if (T >= (1ull << 32)) {
        *err = "inverted index: the sketch must hold fewer than 2^32 samples";
        return SKIS_EINVAL;
    }
    dev_free(s->inv, st);
    s->inv = nullptr;
    s->inv_T = 0;
    if (!s->inv_off) CV_CUDA(dev_alloc_t(&s->inv_off, (size_t)n + 1, st));
    uint32_t* cnt = nullptr;
    uint64_t E = 0;
    const int cblocks = coverage_blocks(T);
    CV_CUDA(dev_alloc_t(&cnt, (size_t)n, st));
    if (s->vcount && s->vcount_ok && s->vcount_T == T) {  // counted while sampling
        CV_CUDA(cudaMemcpyAsync(cnt, s->vcount, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    } else {
        CV_CUDA(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(uint32_t), st));
        k_count_members<<<cblocks, kCovThreads, 0, st>>>(s->h_off, s->h_len, T, s->arena, cnt); note_launch();
        CV_CUDA(cudaGetLastError());
    }
    CV_CUDA(scan_u32_to_u64(cnt, s->inv_off, n, st));
    CV_CUDA(cudaMemcpyAsync(&E, s->inv_off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    CV_CUDA(dev_alloc_t(&s->inv, (size_t)std::max<uint64_t>(E, 1), st));
    CV_CUDA(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(uint32_t), st));  // reused as fill cursors
    k_fill_inverted<<<cblocks, kCovThreads, 0, st>>>(s->h_off, s->h_len, T, s->arena, s->inv_off, cnt, s->inv); note_launch();
    CV_CUDA(cudaGetLastError());
    dev_free(cnt, st);
    s->inv_T = T;
    return SKIS_OK;
}

int sketch_greedy(skis_sketch* s, int32_t k, int32_t* h_seeds, int64_t* h_cov, double* h_est, cudaStream_t st,
                  std::string* err) {
    const char* where = "skis_greedy_maxcover";
    const skis_graph* g = s->g;
    const int64_t n = g->n;
    const uint64_t T = s->T;
    if (k < 0 || k > n) {
        *err = "skis_greedy_maxcover: k must be in [0, n]";
        return SKIS_EINVAL;
    }
    if (T == 0 || T >= (1ull << 32)) {
        *err = "skis_greedy_maxcover: the sketch must hold between 1 and 2^32 - 1 samples";
        return SKIS_EINVAL;
    }
    if (k == 0) return SKIS_OK;
    int rc = sketch_inverted(s, st, err);
    if (rc != SKIS_OK) return rc;
    uint32_t *delta = nullptr, *covered = nullptr;
    uint8_t* inS = nullptr;
    KeyId* partial = nullptr;
    KeyId* seg_best = nullptr;
    int32_t* d_seeds = nullptr;
    int64_t* d_cov = nullptr;
    double* d_est = nullptr;
    auto body = [&]() -> int {
        int per_sm = 0;
        CV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy_rounds, kGreedyThreads, 0));
        if (per_sm < 1) {
            *err = "skis_greedy_maxcover: the cooperative kernel does not fit on an SM";
            return SKIS_ERR_CUDA;
        }
        const int gblocks = sm_count();  // one block per SM
        CV_CUDA(dev_alloc_t(&delta, (size_t)n, st));
        CV_CUDA(dev_alloc_t(&inS, (size_t)n, st));
        CV_CUDA(dev_alloc_t(&covered, (size_t)((T + 31) / 32), st));
        CV_CUDA(dev_alloc_t(&partial, (size_t)gblocks, st));
        const int64_t nseg = (n + kGreedySeg - 1) / kGreedySeg;
        CV_CUDA(dev_alloc_t(&seg_best, (size_t)nseg, st));
        CV_CUDA(dev_alloc_t(&d_seeds, (size_t)k, st));
        CV_CUDA(dev_alloc_t(&d_cov, (size_t)k, st));
        CV_CUDA(dev_alloc_t(&d_est, (size_t)k, st));
        CV_CUDA(cudaMemsetAsync(inS, 0, (size_t)n, st));
        CV_CUDA(cudaMemsetAsync(covered, 0, (size_t)((T + 31) / 32) * sizeof(uint32_t), st));
        // Delta_R(v, {}) = number of samples containing v = length of v's list
        const int b1 = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8));
        k_delta_from_index<<<b1, 256, 0, st>>>(s->inv_off, n, delta); note_launch();
        CV_CUDA(cudaGetLastError());
        GreedyArgs ga;
        ga.w = g->w;
        ga.inS = inS;
        ga.delta = delta;
        ga.n = n;
        ga.W = g->W;
        ga.T = T;
        ga.f = g->f;
        ga.k = k;
        ga.inv_off = s->inv_off;
        ga.inv = s->inv;
        ga.h_off = s->h_off;
        ga.h_len = s->h_len;
        ga.arena = s->arena;
        ga.covered = covered;
        ga.partial = partial;
        ga.seg_best = seg_best;
        ga.nseg = nseg;
        ga.seeds = d_seeds;
        ga.cov_out = d_cov;
        ga.est_out = d_est;
        ga.ris = s->ris;
        void* kargs[] = {&ga};
        CV_CUDA(cudaLaunchCooperativeKernel((const void*)k_greedy_rounds, gblocks, kGreedyThreads, kargs, 0, st));
        note_launch();
        CV_CUDA(cudaMemcpyAsync(h_seeds, d_seeds, (size_t)k * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        if (h_cov) CV_CUDA(cudaMemcpyAsync(h_cov, d_cov, (size_t)k * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        if (h_est) CV_CUDA(cudaMemcpyAsync(h_est, d_est, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, st));
        CV_CUDA(cudaStreamSynchronize(st));
        return SKIS_OK;
    };
    rc = body();
    dev_free(delta, st);
    dev_free(covered, st);
    dev_free(inS, st);
    dev_free(partial, st);
    dev_free(seg_best, st);
    dev_free(d_seeds, st);
    dev_free(d_cov, st);
    dev_free(d_est, st);
    return rc;
}

}  // namespace skis

// ------------------------------------------------------ sharded sketch
// A sketch split by sample id over ranks (every rank holds the samples of
// one id range of one seed's sketch). Coverage counts and Delta are sums
// over the ranks' samples, so the per-rank values are summed through the
// caller's all-reduce in a caller-owned device buffer, and every rank then
// takes the same decisions as one process holding the union sketch.
namespace skis {

__global__ void k_shard_delta0(const uint64_t* __restrict__ inv_off, int64_t n, int64_t* __restrict__ x) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x)
        x[v] = v < n ? (int64_t)(inv_off[v + 1] - inv_off[v]) : 0;
}

// Block bests of the exact key Delta W + T (2^f - w_v) (RIS: Delta) over v
// outside S, ties to the lowest id.
__global__ void __launch_bounds__(256) k_shard_argmax(const int64_t* __restrict__ delta, const uint64_t* __restrict__ w,
                                                      const uint8_t* __restrict__ inS, int64_t n, uint64_t W,
                                                      uint64_t T, int f, int ris, KeyId* __restrict__ partial) {
    __shared__ KeyId s_part[256 / 32];
    const uint64_t one_f = 1ull << f;
    KeyId best{0, 0xFFFFFFFFu, 0};
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (inS[v]) continue;
        const u128 dv = (u128)(uint64_t)delta[v];
        const KeyId c{ris ? dv : dv * W + (u128)T * (one_f - w[v]), (uint32_t)v, 1u, 0u, 0u};
        if (better(c, best)) best = c;
    }
    best = block_best(best, s_part);
    if (threadIdx.x == 0) partial[blockIdx.x] = best;
}

// The round's winner from the block bests: joins S; recorded as seed r.
__global__ void k_shard_commit(const KeyId* __restrict__ partial, int nparts, uint8_t* __restrict__ inS,
                               int32_t* __restrict__ seeds, int32_t r, uint32_t* __restrict__ win) {
    const int lane = threadIdx.x & 31;
    KeyId b{0, 0xFFFFFFFFu, 0};
    for (int i = lane; i < nparts; i += 32)
        if (better(partial[i], b)) b = partial[i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const KeyId o = shfl_down_keyid(b, d);
        if (better(o, b)) b = o;
    }
    if (lane == 0) {  // a valid winner exists: k <= n and each round adds one vertex
        inS[b.id] = 1;
        seeds[r] = (int32_t)b.id;
        *win = b.id;
    }
}

// Cover this rank's uncovered samples of the winner: x[u] += 1 for every
// member u of each, x[n] += the number of them.
__global__ void __launch_bounds__(256) k_shard_cover(const uint32_t* __restrict__ win,
                                                     const uint64_t* __restrict__ inv_off,
                                                     const uint32_t* __restrict__ inv,
                                                     const uint64_t* __restrict__ h_off,
                                                     const uint32_t* __restrict__ h_len,
                                                     const int32_t* __restrict__ arena, uint32_t* __restrict__ covered,
                                                     int64_t n, int64_t* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    const uint32_t v = *win;
    const uint64_t lo = inv_off[v], cnt = inv_off[v + 1] - lo;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    unsigned long long* xc = reinterpret_cast<unsigned long long*>(x);
    for (uint64_t base = ((uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * 32; base < cnt;
         base += nwarps * 32) {
        uint64_t off = 0;
        uint32_t len = 0;
        if (base + lane < cnt) {
            const uint32_t j = inv[lo + base + lane];
            const uint32_t bit = 1u << (j & 31);
            if ((atomicOr(&covered[j >> 5], bit) & bit) == 0) {
                off = h_off[j];
                len = h_len[j];
                atomicAdd(xc + n, 1ull);
            }
        }
        warp_members(off, len, arena, [&](int, int32_t u) { atomicAdd(xc + u, 1ull); });
    }
}

// Delta -= the summed decrements; the running coverage and Eq. 21 of the
// prefix S (thread 0; acc = {Cov, sum over S of 2^f - w_v}).
__global__ void k_shard_update(int64_t* __restrict__ delta, const int64_t* __restrict__ x, int64_t n,
                               const uint32_t* __restrict__ win, const uint64_t* __restrict__ w, uint64_t W,
                               uint64_t T, int f, int ris, int32_t r, uint64_t* __restrict__ acc,
                               int64_t* __restrict__ cov_out, double* __restrict__ est_out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        delta[v] -= x[v];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint64_t cov = acc[0] + (uint64_t)x[n];
        const uint64_t sum_c = acc[1] + ((1ull << f) - w[*win]);
        acc[0] = cov;
        acc[1] = sum_c;
        cov_out[r] = (int64_t)cov;
        const u128 N = ris ? (u128)cov * (uint64_t)n : (u128)cov * W + (u128)T * sum_c;
        const u128 D = ris ? (u128)T : (u128)T << f;
        est_out[r] = u128_to_double(N) / u128_to_double(D);
    }
}

// The caller's all-reduce of buf[0, count), after the work that wrote it.
static int exchange(skis_allreduce_fn fn, void* ctx, int64_t* buf, int64_t count, cudaStream_t st, const char* where,
                    std::string* err) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *err = std::string(where) + ": CUDA error: " + cudaGetErrorString(e);
        return SKIS_ERR_CUDA;
    }
    if (fn(ctx, buf, count, (void*)st) != 0) {
        *err = std::string(where) + ": the all-reduce callback failed";
        return SKIS_ERR_EXCHANGE;
    }
    return SKIS_OK;
}

int sketch_estimate_sharded(skis_sketch* s, int32_t q, const int64_t* d_off, const int32_t* d_seeds,
                            const int64_t* h_off, int64_t* d_cov, double* d_est, int64_t* exch, skis_allreduce_fn fn,
                            void* ctx, cudaStream_t st, std::string* err) {
    const char* where = "skis_estimate_sharded";
    const skis_graph* g = s->g;
    double* tmp = nullptr;
    CV_CUDA(dev_alloc_t(&tmp, (size_t)q, st));
    // this rank's counts into exch[0, q) (validating the queries), its T into exch[q]
    int rc = sketch_estimate(s, q, d_off, d_seeds, h_off, exch, tmp, st, err);
    dev_free(tmp, st);
    if (rc != SKIS_OK) return rc;
    const int64_t T_rank = (int64_t)s->T;
    CV_CUDA(cudaMemcpyAsync(exch + q, &T_rank, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    rc = exchange(fn, ctx, exch, (int64_t)q + 1, st, where, err);
    if (rc != SKIS_OK) return rc;
    int64_t T = 0;
    CV_CUDA(cudaMemcpyAsync(&T, exch + q, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    for (int32_t q0 = 0; q0 < q; q0 += 64) {
        const int32_t qn = std::min<int32_t>(64, q - q0);
        k_estimate<<<div_up((int64_t)qn * 32, 256), 256, 0, st>>>(
            d_off, d_seeds, q0, qn, g->n, g->w, g->f, g->W, (uint64_t)T,
            reinterpret_cast<const unsigned long long*>(exch + q0), d_cov, d_est, s->ris);
        note_launch();
        CV_CUDA(cudaGetLastError());
    }
    CV_CUDA(cudaStreamSynchronize(st));
    return SKIS_OK;
}

int sketch_greedy_sharded(skis_sketch* s, int32_t k, int32_t* h_seeds, int64_t* h_cov, double* h_est, int64_t* exch,
                          skis_allreduce_fn fn, void* ctx, cudaStream_t st, std::string* err) {
    const char* where = "skis_greedy_maxcover_sharded";
    const skis_graph* g = s->g;
    const int64_t n = g->n;
    if (k < 0 || k > n) {
        *err = "skis_greedy_maxcover_sharded: k must be in [0, n]";
        return SKIS_EINVAL;
    }
    if (s->T >= (1ull << 32)) {
        *err = "skis_greedy_maxcover_sharded: a rank's sketch must hold fewer than 2^32 samples";
        return SKIS_EINVAL;
    }
    if (k == 0) return SKIS_OK;
    // the union sketch's T
    const int64_t T_rank = (int64_t)s->T;
    CV_CUDA(cudaMemcpyAsync(exch, &T_rank, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    int rc = exchange(fn, ctx, exch, 1, st, where, err);
    if (rc != SKIS_OK) return rc;
    int64_t T = 0;
    CV_CUDA(cudaMemcpyAsync(&T, exch, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CV_CUDA(cudaStreamSynchronize(st));
    if (T <= 0) {
        *err = "skis_greedy_maxcover_sharded: the ranks' sketches hold no samples";
        return SKIS_EINVAL;
    }
    rc = sketch_inverted(s, st, err);
    if (rc != SKIS_OK) return rc;
    int64_t* delta = nullptr;
    uint8_t* inS = nullptr;
    uint32_t *covered = nullptr, *win = nullptr;
    KeyId* partial = nullptr;
    int32_t* d_seeds = nullptr;
    int64_t* d_cov = nullptr;
    double* d_est = nullptr;
    uint64_t* acc = nullptr;
    const int nb = sm_count() * 4;
    const uint64_t cwords = std::max<uint64_t>(1, (s->T + 31) / 32);
    auto body = [&]() -> int {
        CV_CUDA(dev_alloc_t(&delta, (size_t)n, st));
        CV_CUDA(dev_alloc_t(&inS, (size_t)n, st));
        CV_CUDA(dev_alloc_t(&covered, (size_t)cwords, st));
        CV_CUDA(dev_alloc_t(&win, 1, st));
        CV_CUDA(dev_alloc_t(&partial, (size_t)nb, st));
        CV_CUDA(dev_alloc_t(&d_seeds, (size_t)k, st));
        CV_CUDA(dev_alloc_t(&d_cov, (size_t)k, st));
        CV_CUDA(dev_alloc_t(&d_est, (size_t)k, st));
        CV_CUDA(dev_alloc_t(&acc, 2, st));
        CV_CUDA(cudaMemsetAsync(inS, 0, (size_t)n, st));
        CV_CUDA(cudaMemsetAsync(covered, 0, cwords * sizeof(uint32_t), st));
        CV_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(uint64_t), st));
        // Delta_R(v, {}) over the union: the ranks' list lengths summed
        const int b1 = (int)std::max<int64_t>(1, std::min<int64_t>((n + 256) / 256, (int64_t)sm_count() * 8));
        k_shard_delta0<<<b1, 256, 0, st>>>(s->inv_off, n, exch); note_launch();
        CV_CUDA(cudaGetLastError());
        int e = exchange(fn, ctx, exch, n + 1, st, where, err);
        if (e != SKIS_OK) return e;
        CV_CUDA(cudaMemcpyAsync(delta, exch, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
        const int cb = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * 8, (s->T + 255) / 256));
        for (int32_t r = 0; r < k; ++r) {
            k_shard_argmax<<<nb, 256, 0, st>>>(delta, g->w, inS, n, g->W, (uint64_t)T, g->f, s->ris, partial);
            note_launch();
            k_shard_commit<<<1, 32, 0, st>>>(partial, nb, inS, d_seeds, r, win); note_launch();
            CV_CUDA(cudaMemsetAsync(exch, 0, (size_t)(n + 1) * sizeof(int64_t), st));
            k_shard_cover<<<cb, 256, 0, st>>>(win, s->inv_off, s->inv, s->h_off, s->h_len, s->arena, covered, n, exch);
            note_launch();
            CV_CUDA(cudaGetLastError());
            e = exchange(fn, ctx, exch, n + 1, st, where, err);
            if (e != SKIS_OK) return e;
            k_shard_update<<<b1, 256, 0, st>>>(delta, exch, n, win, g->w, g->W, (uint64_t)T, g->f, s->ris, r, acc,
                                               d_cov, d_est);
            note_launch();
            CV_CUDA(cudaGetLastError());
        }
        CV_CUDA(cudaMemcpyAsync(h_seeds, d_seeds, (size_t)k * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        if (h_cov) CV_CUDA(cudaMemcpyAsync(h_cov, d_cov, (size_t)k * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        if (h_est) CV_CUDA(cudaMemcpyAsync(h_est, d_est, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, st));
        CV_CUDA(cudaStreamSynchronize(st));
        return SKIS_OK;
    };
    rc = body();
    dev_free(delta, st);
    dev_free(inS, st);
    dev_free(covered, st);
    dev_free(win, st);
    dev_free(partial, st);
    dev_free(d_seeds, st);
    dev_free(d_cov, st);
    dev_free(d_est, st);
    dev_free(acc, st);
    return rc;
}

}  // namespace skis
