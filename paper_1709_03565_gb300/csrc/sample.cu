// Importance Influence Sampling (Sec. III, Alg. 1) on the device, in three
// tiers chained by sample id.
//
// Lane tier (first): one lane per sample; each step draws one edge quad of
// the lane's current row (one Philox block = the 4 coins of a quad). Member
// lists (which are also Alg. 1's FIFO queues Q = members[head .. len)) hold
// up to 32 vertices per sample in shared memory; the row of the next pop is
// loaded ahead; finished samples are written out and lanes refilled in
// batches. A sample whose list outgrows it, that meets an in-row longer than
// the degree threshold, or that uses up its step or retry budget is handed
// by id to the warp tier.
//
// Warp tier: one warp per sample. The member list (256 entries) and an
// open-addressing hash set (the visited set R_j) live in shared memory. Edges
// of up to 32 queued vertices are spread over the lanes one edge quad at a
// time. A sample that outgrows it is handed, by id, to the CTA tier.
//
// CTA tier: one block per sample with a global n-bit visited bitmap and an
// n-entry global queue per block slot.
//
// All tiers compute the same R_j: every coin is a pure function of
// (seed, sample id, domain, round, edge), so R_j is the reverse-reachable set
// of the source in one live-edge world, whatever the order of expansion.
#include <algorithm>
#include <string>

#include "../../include/skis.h"
#include "skis_internal.cuh"

namespace skis {

constexpr int kWarpThreads = 256;  // 8 warps per block
constexpr int kQCap = 256;         // warp-tier member capacity
constexpr int kHCap = 512;         // warp-tier hash slots (load <= 1/2 + one insert round)
constexpr int kHashBits = 9;
constexpr int kIdBatch = 16;       // sample ids taken per work-cursor atomic
constexpr uint32_t kArenaChunk = 2048;        // entries reserved per arena atomic (warp tier)
constexpr uint32_t kLaneArenaChunk = 512;     // entries reserved per arena atomic (lane tiers)
constexpr int kCtaGroupLog2 = 2;
constexpr int kCtaGroup = 1 << kCtaGroupLog2;  // edge quads of a long row a CTA-tier lane draws per step
constexpr int kCtaLongRow = 64;            // quads that make a row long
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

struct SampleArgs {
    const AliasEntry* __restrict__ alias;
    const RowInfo* __restrict__ rows;
    const int32_t* __restrict__ src;
    const uint32_t* __restrict__ tau;  // nullptr: thresholds are per row
    uint64_t n, W, seed;
    PhiloxKeys rk;                     // the round keys of seed
    uint32_t retry_cap;
    uint32_t max_deg;                  // thread tier: longest in-row it expands
    uint32_t max_steps;                // thread tier: edge quads per sample before handing it on
    uint32_t max_retries;              // thread tier: rejected rounds before handing it on
    uint32_t warp_max_coins;           // warp tier: in-edges a BFS may draw before handing it on
    uint32_t cta_hub_quads;            // CTA tier: edge quads that make a row a hub (0 = no hub loop)
    int ris;                           // plain RIS: uniform source, one unconditioned round
    // input ids: first_id + t (ids == nullptr) or ids[t], t < count (or
    // t < *count_dev when the list was filled by the previous tier)
    const uint64_t* ids;
    uint64_t first_id, count;
    const unsigned long long* count_dev;
    uint64_t id_base;                  // sample id of the sketch's first header (headers are indexed j - id_base)
    unsigned long long* work;          // id cursor of this launch
    uint64_t* out_ids;                 // samples handed to the next tier
    unsigned long long* out_count;
    uint64_t* ovf_ids;                 // samples whose arena reservation did not fit
    unsigned long long* novf;
    unsigned long long* arena_cursor;
    uint64_t* h_off;
    uint32_t* h_len;
    uint32_t* h_src;
    uint32_t* h_retries;
    uint64_t* h_coins;
    int32_t* arena;
    uint64_t arena_cap;
    DevStatus* status;
    uint32_t* bitmaps;
    int32_t* queues;
    uint64_t bitmap_words;
    uint32_t queue_cap;      // CTA tier: entries of a slot's queue (also the slots' stride); a sample
                             // with more members is handed to a pass with n-entry queues
    const uint4* srcrec;  // lane tier: source record per input t (k_sources)
    const uint2* srcpick; // lane tier, bucket form: (picked in-edge, its source) per input t
    const uint64_t* lt_cum;  // LT graphs with per-edge thresholds: running weight sums, else nullptr
    const uint64_t* chain;   // bucket first step: the gamma chain per in-edge, else nullptr
    uint32_t* vcount;        // per-vertex member counts kept for the inverted index, or nullptr
    // the lane tier's prepass records for sample ids [up_first, up_first + up_count), which the
    // later tiers reuse for the samples handed on to them (nullptr: draw again)
    const uint4* up_rec;
    const uint2* up_pick;
    uint64_t up_first, up_count;
};


// a member written to the arena counts towards its vertex's list length
__device__ __forceinline__ void count_member(const SampleArgs& a, int32_t u) {
    if (a.vcount) atomicAdd(&a.vcount[u], 1u);
}

__device__ __forceinline__ uint64_t input_count(const SampleArgs& a) {
    return a.count_dev ? (uint64_t)*a.count_dev : a.count;
}

__device__ __forceinline__ uint64_t input_id(const SampleArgs& a, uint64_t t) {
    return a.ids ? a.ids[t] : a.first_id + t;
}

__device__ __forceinline__ void hand_on(const SampleArgs& a, uint64_t j) {
    const unsigned long long k = atomicAdd(a.out_count, 1ull);
    a.out_ids[k] = j;
}

__device__ __forceinline__ void arena_overflow(const SampleArgs& a, uint64_t j) {
    const unsigned long long k = atomicAdd(a.novf, 1ull);
    a.ovf_ids[k] = j;
    atomicOr(&a.status->flags, kStArena);
}

// Eq. probu through the alias table: column floor(U1 n), threshold draw
// floor(U2 W) from the SRC-domain block of sample j.
// (kSeedKey: the Philox keys advanced from the seed in registers, for a
// kernel whose occupancy the preloaded round keys would cut)
template <bool kSeedKey = false>
__device__ __forceinline__ uint32_t draw_source(const SampleArgs& a, uint64_t j) {
    const uint4 x = kSeedKey ? coin_block(a.seed, 0, 0, kDomSrc, j) : coin_block(a.rk, 0, 0, kDomSrc, j);
    const uint64_t u1 = (uint64_t)x.x | ((uint64_t)x.y << 32);
    const uint64_t u2 = (uint64_t)x.z | ((uint64_t)x.w << 32);
    const uint64_t col = __umul64hi(u1, a.n);
    if (a.ris) return (uint32_t)col;  // RIS: the uniform column alone
    const uint64_t y = __umul64hi(u2, a.W);
    const AliasEntry e = a.alias[col];
    return y < e.prob ? (uint32_t)col : e.alias;
}

// The bucket form of Alg. 1's conditioned first step (Eq. probn): bucket i of the source's
// row is "in-edges before i dead, edge i live", of mass Q_{i-1} - Q_i in the
// gamma chain (total 2^62 - Q_d); z = floor(U (2^62 - Q_d) / 2^64) from the
// BUCKET-domain block of sample j picks the first edge e with
// 2^62 - Q_e > z, i.e. Q_e < 2^62 - z (the chain does not increase).
// Returns the edge position; the edges after it get FIRST coins of round 0.
template <bool kSeedKey = false>
__device__ __forceinline__ uint64_t bucket_pick(const SampleArgs& a, uint64_t j, uint64_t off, uint32_t deg) {
    const uint64_t one62 = 1ull << 62;
    const uint64_t G = one62 - a.chain[off + deg - 1];
    const uint4 x = kSeedKey ? coin_block(a.seed, 0, 0, kDomBucket, j) : coin_block(a.rk, 0, 0, kDomBucket, j);
    const uint64_t z = __umul64hi((uint64_t)x.x | ((uint64_t)x.y << 32), G);
    const uint64_t lim = one62 - z;
    uint32_t lo = 0, hi = deg - 1;  // the answer exists: Q_d = 2^62 - G < lim
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.chain[off + mid] < lim) hi = mid;
        else lo = mid + 1;
    }
    return off + lo;
}

// The source record (source, in-row) of sample j, from the prepass when it
// holds j, else drawn; *pe / *pu receive the prepass's bucket pick (or -1).
__device__ __forceinline__ uint32_t source_of(const SampleArgs& a, uint64_t j, RowInfo* rv, int64_t* pe,
                                              int32_t* pu) {
    *pe = -1;
    *pu = -1;
    if (a.up_rec && j - a.up_first < a.up_count) {
        const uint64_t t = j - a.up_first;
        const uint4 r = __ldg(a.up_rec + t);
        rv->deg = r.y;
        rv->off = r.z;
        rv->tau = r.w;
        if (a.up_pick && a.chain && r.y > 0) {
            const uint2 p = __ldg(a.up_pick + t);
            *pe = p.x;
            *pu = (int32_t)p.y;
        }
        return r.x;
    }
    const uint32_t v = draw_source(a, j);
    *rv = a.rows[v];
    return v;
}

// ----------------------------------------------------------- inserters
// Warp tier: shared-memory hash set + shared-memory member queue.
struct WarpInserter {
    uint32_t* hash;
    int32_t* queue;
    uint32_t qlen;
    bool overflow;

    __device__ __forceinline__ void insert(int32_t u) {
        if (overflow) return;  // warp-uniform
        bool fresh = false;
        if (u >= 0) {
            uint32_t h = ((uint32_t)u * 2654435761u) >> (32 - kHashBits);
            for (;;) {
                const uint32_t old = atomicCAS(&hash[h], kEmpty, (uint32_t)u);
                if (old == kEmpty) { fresh = true; break; }
                if (old == (uint32_t)u) break;
                h = (h + 1) & (kHCap - 1);
            }
        }
        const unsigned m = __ballot_sync(kFull, fresh);
        if (m) {
            const uint32_t pos = qlen + __popc(m & lanemask_lt());
            if (fresh && pos < (uint32_t)kQCap) queue[pos] = u;
            qlen += __popc(m);
            if (qlen > (uint32_t)kQCap) overflow = true;
        }
        __syncwarp();
    }
};

// CTA tier, one lane alone (divergent code): test-and-set in the global
// bitmap, append to the global queue through the shared counter. A vertex
// past the queue's capacity gets its bit back, so that the bitmap always
// holds exactly the queued vertices (the counter still counts it: the sample
// is then known to have outgrown the slot).
__device__ __forceinline__ void cta_insert_one(uint32_t* bitmap, int32_t* queue, uint32_t* qlen, uint32_t cap,
                                               int32_t u) {
    const uint32_t bit = 1u << (u & 31);
    if ((atomicOr(&bitmap[u >> 5], bit) & bit) == 0) {
        const uint32_t pos = atomicAdd(qlen, 1u);
        if (pos < cap) queue[pos] = u;
        else atomicAnd(&bitmap[u >> 5], ~bit);
    }
}

// CTA tier: global bitmap (test-and-set) + global queue with a shared counter.
struct CtaInserter {
    uint32_t* bitmap;
    int32_t* queue;
    uint32_t* qlen;  // shared
    uint32_t cap;    // queue capacity (see cta_insert_one)
    bool overflow;   // never set: the CTA tier checks the count between levels

    __device__ __forceinline__ void insert(int32_t u) {
        bool fresh = false;
        if (u >= 0) {
            const uint32_t bit = 1u << (u & 31);
            fresh = (atomicOr(&bitmap[u >> 5], bit) & bit) == 0;
        }
        const unsigned m = __ballot_sync(kFull, fresh);
        if (m) {
            uint32_t base = 0;
            if ((threadIdx.x & 31) == 0) base = atomicAdd(qlen, (uint32_t)__popc(m));
            base = __shfl_sync(kFull, base, 0);
            if (fresh) {
                const uint32_t pos = base + __popc(m & lanemask_lt());
                if (pos < cap) queue[pos] = u;
                else atomicAnd(&bitmap[u >> 5], ~(1u << (u & 31)));
            }
        }
    }
};

// Expand the in-rows held by the lanes (lane i: row off/deg/tau_row, deg = 0
// for none): every in-edge e gets its coin (domain dom, round retry, sample
// j); live edges offer their source to the inserter. Returns, warp-uniform,
// whether any edge was live.
template <class Ins>
__device__ __forceinline__ bool expand_rows(const SampleArgs& a, uint64_t j, uint32_t dom, uint32_t retry,
                                            uint64_t off, uint32_t deg, uint32_t tau_row, Ins& ins) {
    const int lane = threadIdx.x & 31;
    const uint32_t nq = deg ? (uint32_t)(((off + deg - 1) >> 2) - (off >> 2) + 1) : 0u;
    uint32_t incl = nq;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - nq;
    bool any = false;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t g = base + lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t v = __shfl_sync(kFull, incl, owner + step - 1);
            if (v <= g) owner += step;
        }
        const uint64_t o_off = __shfl_sync(kFull, off, owner);
        const uint32_t o_deg = __shfl_sync(kFull, deg, owner);
        const uint32_t o_tau = __shfl_sync(kFull, tau_row, owner);
        const uint32_t o_excl = __shfl_sync(kFull, excl, owner);
        int32_t c0 = -1, c1 = -1, c2 = -1, c3 = -1;
        if (g < total) {
            const uint64_t q = (o_off >> 2) + (g - o_excl);
            const uint4 x = coin_block(a.rk, q, retry, dom, j);
            const uint4 t4 = a.tau ? __ldg(reinterpret_cast<const uint4*>(a.tau) + q)
                                   : make_uint4(o_tau, o_tau, o_tau, o_tau);
            const uint64_t e0 = q << 2, lo = o_off, hi = o_off + o_deg;
            unsigned live = 0;
            live |= (e0 + 0 >= lo && e0 + 0 < hi && coin_live(x.x, t4.x)) ? 1u : 0u;
            live |= (e0 + 1 >= lo && e0 + 1 < hi && coin_live(x.y, t4.y)) ? 2u : 0u;
            live |= (e0 + 2 >= lo && e0 + 2 < hi && coin_live(x.z, t4.z)) ? 4u : 0u;
            live |= (e0 + 3 >= lo && e0 + 3 < hi && coin_live(x.w, t4.w)) ? 8u : 0u;
            if (live) {
                const int4 s4 = __ldg(reinterpret_cast<const int4*>(a.src) + q);
                any = true;
                if (live & 1u) c0 = s4.x;
                if (live & 2u) c1 = s4.y;
                if (live & 4u) c2 = s4.z;
                if (live & 8u) c3 = s4.w;
            }
        }
        if (__any_sync(kFull, (c0 >= 0) | (c1 >= 0) | (c2 >= 0) | (c3 >= 0))) {
            if (__any_sync(kFull, c0 >= 0)) ins.insert(c0);
            if (__any_sync(kFull, c1 >= 0)) ins.insert(c1);
            if (__any_sync(kFull, c2 >= 0)) ins.insert(c2);
            if (__any_sync(kFull, c3 >= 0)) ins.insert(c3);
            if (ins.overflow) break;
        }
    }
    return __any_sync(kFull, any);
}

// Alg. 1's conditioned first step for one warp: the rejection rounds r = 0, 1, ... of the
// source row, until one round has a live coin; the live in-neighbours of that
// round are inserted. Rounds are independent given (j, r), so a short row
// (nq <= 16 edge quads) is searched 32 / nq rounds per pass: lane g takes
// round r0 + g / nq and quad g % nq, and the lowest round with a live coin
// (the first set lane of the ballot, as lanes are ordered by round) is the
// accepted one, exactly as in sequential order. Longer rows take one round
// per pass, spread over the lanes. Returns the accepted round, or the cap
// with *failed set.
template <class Ins>
__device__ __forceinline__ uint32_t first_step_warp(const SampleArgs& a, uint64_t j, const RowInfo& rv, Ins& ins,
                                                    bool* failed, int64_t pick_e = -1, int32_t pick_u = -1) {
    const int lane = threadIdx.x & 31;
    *failed = false;
    if (a.chain) {  // bucket form: the picked in-edge, then round-0 coins after it
        int32_t u = -1;
        uint64_t e = 0;
        if (lane == 0) {
            if (pick_e >= 0) {  // drawn by the prepass
                e = (uint64_t)pick_e;
                u = pick_u;
            } else {
                e = bucket_pick(a, j, rv.off, rv.deg);
                u = a.src[e];
            }
        }
        e = __shfl_sync(kFull, e, 0);
        ins.insert(u);
        const uint64_t rest = rv.off + rv.deg - (e + 1);
        expand_rows(a, j, kDomFirst, 0, e + 1, lane == 0 ? (uint32_t)rest : 0u, rv.tau, ins);
        return 0;
    }
    if (a.ris) {  // RIS: round 0, accepted whatever its coins
        expand_rows(a, j, kDomFirst, 0, rv.off, lane == 0 ? rv.deg : 0u, rv.tau, ins);
        return 0;
    }
    const uint64_t q_first = rv.off >> 2;
    const uint32_t nq = (uint32_t)(((rv.off + rv.deg - 1) >> 2) - q_first + 1);
    if (nq > 16) {
        for (uint32_t r = 0;; ++r) {
            if (r >= a.retry_cap) { *failed = true; return r; }
            if (expand_rows(a, j, kDomFirst, r, rv.off, lane == 0 ? rv.deg : 0u, rv.tau, ins)) return r;
        }
    }
    const uint32_t rounds = 32u / nq;
    const uint32_t ri = (uint32_t)lane / nq, qi = (uint32_t)lane % nq;
    const uint64_t q = q_first + qi;
    const uint64_t e0 = q << 2, lo = rv.off, hi = rv.off + rv.deg;
    const uint4 t4 = a.tau ? __ldg(reinterpret_cast<const uint4*>(a.tau) + q) : make_uint4(rv.tau, rv.tau, rv.tau, rv.tau);
    for (uint32_t r0 = 0; r0 < a.retry_cap; r0 += rounds) {
        const uint32_t r = r0 + ri;
        unsigned live = 0;
        if (ri < rounds && r < a.retry_cap) {
            const uint4 x = coin_block(a.rk, q, r, kDomFirst, j);
            live |= (e0 + 0 >= lo && e0 + 0 < hi && coin_live(x.x, t4.x)) ? 1u : 0u;
            live |= (e0 + 1 >= lo && e0 + 1 < hi && coin_live(x.y, t4.y)) ? 2u : 0u;
            live |= (e0 + 2 >= lo && e0 + 2 < hi && coin_live(x.z, t4.z)) ? 4u : 0u;
            live |= (e0 + 3 >= lo && e0 + 3 < hi && coin_live(x.w, t4.w)) ? 8u : 0u;
        }
        const unsigned bal = __ballot_sync(kFull, live != 0);
        if (bal) {
            const uint32_t acc = (uint32_t)(__ffs(bal) - 1) / nq;  // accepted round = r0 + acc
            int32_t c0 = -1, c1 = -1, c2 = -1, c3 = -1;
            if (ri == acc && live) {
                const int4 s4 = __ldg(reinterpret_cast<const int4*>(a.src) + q);
                if (live & 1u) c0 = s4.x;
                if (live & 2u) c1 = s4.y;
                if (live & 4u) c2 = s4.z;
                if (live & 8u) c3 = s4.w;
            }
            if (__any_sync(kFull, c0 >= 0)) ins.insert(c0);
            if (__any_sync(kFull, c1 >= 0)) ins.insert(c1);
            if (__any_sync(kFull, c2 >= 0)) ins.insert(c2);
            if (__any_sync(kFull, c3 >= 0)) ins.insert(c3);
            return r0 + acc;
        }
    }
    *failed = true;
    return a.retry_cap;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(kFull, v, d);
    return __shfl_sync(kFull, v, 0);
}

__device__ __forceinline__ void record_retry_failure(const SampleArgs& a, uint64_t j, uint32_t v, uint32_t r,
                                                     uint32_t deg) {
    a.h_off[j - a.id_base] = 0;
    a.h_len[j - a.id_base] = 0;
    a.h_src[j - a.id_base] = v;
    a.h_retries[j - a.id_base] = r;
    a.h_coins[j - a.id_base] = (uint64_t)deg * r;
    atomicOr(&a.status->flags, kStRetry);
    atomicMin(&a.status->first_bad, (unsigned long long)j);
}

// Alg. 1's source draw for every input id at once: the source of sample j and its
// in-row, as 16 bytes (source, degree, row offset, row threshold), so that a
// lane-tier lane starting a sample makes one coalesced load; with the bucket
// form, also the first step's picked in-edge and its source (8 bytes), whose
// dependent chain loads are better spread over this many-thread pass than
// paid by a lane at claim time. Row offsets fit 32 bits because graphs hold
// fewer than 2^32 - 8 edges.
__global__ void k_sources(SampleArgs a, uint4* __restrict__ rec, uint2* __restrict__ pick) {
    const uint64_t count = input_count(a);
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = input_id(a, t);
        const uint32_t v = draw_source<true>(a, j);
        const RowInfo rv = a.rows[v];
        rec[t] = make_uint4(v, rv.deg, (uint32_t)rv.off, rv.tau);
        if (a.chain && rv.deg > 0) {  // the bucket form of the first step, drawn here in bulk
            const uint64_t e = bucket_pick<true>(a, j, rv.off, rv.deg);
            pick[t] = make_uint2((uint32_t)e, (uint32_t)a.src[e]);
        }
    }
}

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
    const uint32_t lo = __shfl_sync(kFull, (uint32_t)v, src);
    const uint32_t hi = __shfl_sync(kFull, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}

// ------------------------------------------------------------- lane tier
// One lane per sample with a lean inner step: one edge quad of the lane's
// current row (Philox block, thresholds, four compares); live coins join the
// member list at once (visited check by scanning it); at the end of a row
// the next queued member's row, loaded ahead, takes over. Finished samples
// are written out, and idle lanes refilled, in batches: when at least
// kLaneRefill lanes are idle or nothing else is left.
constexpr int kLaneBlock = 256;
constexpr int kLaneQ = 32;
constexpr int kLaneStride = kLaneQ + 1;  // odd: conflict-free by lane and by member
constexpr int kLaneRefill = 8;

// One of 64 bits for vertex u (the top six bits of a multiplicative hash): a
// lane's sample keeps the OR over its members, so a candidate whose bit is
// clear is new without searching the member list.
__device__ __forceinline__ uint64_t member_bit(uint32_t u) { return 1ull << ((u * 0x9E3779B9u) >> 26); }

__global__ void __launch_bounds__(kLaneBlock, 4) k_iis_lane(SampleArgs a) {
    __shared__ int32_t s_q[kLaneBlock / 32][32 * kLaneStride];
    const int lane = threadIdx.x & 31;
    int32_t* const mq = s_q[threadIdx.x >> 5];
    int32_t* const mine = mq + lane * kLaneStride;
    const uint64_t count = input_count(a);
    const uint4* __restrict__ tau4 = reinterpret_cast<const uint4*>(a.tau);
    const int4* __restrict__ src4 = reinterpret_cast<const int4*>(a.src);

    bool busy = false, done = false, first = false, any = false, pf_ok = false;
    uint64_t j = 0, coins = 0;
    uint32_t v = 0, r = 0, len = 0, head = 0, src_deg = 0, tau_row = 0, steps = 0;
    uint32_t lo = 0, hi = 0, qc = 0, q_last = 0;
    uint32_t pf_off = 0, pf_deg = 0, pf_tau = 0;
    bool exhausted = false;
    uint64_t pool_base = 0;
    uint32_t pool_n = 0, pool_used = 0;
    uint4 rec = make_uint4(0, 0, 0, 0);
    uint2 prec = make_uint2(0, 0);
    uint64_t sig = 0;  // the sample's members, one hashed bit each (member_bit)
    uint64_t chunk_pos = 0, chunk_end = 0;

    for (;;) {
        // ---- batched maintenance: write out finished samples, refill
        const unsigned dn = __ballot_sync(kFull, done);
        const unsigned free_l = __ballot_sync(kFull, !busy || done);
        const bool all_free = free_l == kFull;
        if (__popc(free_l) >= kLaneRefill || all_free) {
            if (dn) {
                const uint32_t mylen = done ? len : 0u;
                uint32_t incl = mylen;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, incl, d);
                    if (lane >= d) incl += y;
                }
                const uint32_t total = __shfl_sync(kFull, incl, 31);
                bool fits = true;
                if (chunk_end - chunk_pos < total) {
                    const uint64_t size = max((uint64_t)kLaneArenaChunk, (uint64_t)total);
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(a.arena_cursor, (unsigned long long)size);
                    base = __shfl_sync(kFull, base, 0);
                    if (base + size > a.arena_cap) {
                        fits = false;
                        chunk_pos = chunk_end = 0;
                    } else {
                        chunk_pos = base;
                        chunk_end = base + size;
                    }
                }
                const uint64_t at = chunk_pos + (incl - mylen);
                if (done) {
                    if (fits) {
                        a.h_off[j - a.id_base] = at;
                        a.h_len[j - a.id_base] = len;
                        a.h_src[j - a.id_base] = v;
                        a.h_retries[j - a.id_base] = r;
                        a.h_coins[j - a.id_base] = coins;
                    } else {
                        arena_overflow(a, j);
                    }
                }
                __syncwarp();
                if (fits && total < 16u * (uint32_t)__popc(dn)) {
                    // short samples: their members end to end over the warp's
                    // lanes, each lane finding the sample that holds its entry
                    // (the first lane whose inclusive end exceeds it)
                    const uint32_t excl = incl - mylen;
                    for (uint32_t b0 = 0; b0 < total; b0 += 32) {
                        const uint32_t idx = b0 + (uint32_t)lane;
                        int owner = 0;
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1)
                            if (__shfl_sync(kFull, incl, owner + step - 1) <= idx) owner += step;
                        const uint32_t start = __shfl_sync(kFull, excl, owner);
                        if (idx < total) {
                            const int32_t u = mq[owner * kLaneStride + (idx - start)];
                            a.arena[chunk_pos + idx] = u;
                            count_member(a, u);
                        }
                    }
                    chunk_pos += total;
                } else if (fits) {
                    unsigned m = dn;
                    while (m) {
                        const int sl = __ffs(m) - 1;
                        m &= m - 1;
                        const uint64_t at_s = shfl_u64(at, sl);
                        const uint32_t len_s = __shfl_sync(kFull, len, sl);
                        if ((uint32_t)lane < len_s) {
                            const int32_t u = mq[sl * kLaneStride + lane];
                            a.arena[at_s + lane] = u;
                            count_member(a, u);
                        }
                    }
                    chunk_pos += total;
                }
                __syncwarp();
                if (done) {
                    done = false;
                    busy = false;
                }
            }
            unsigned idle = __ballot_sync(kFull, !busy);
            while (idle && !exhausted) {
                if (pool_used == pool_n) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(a.work, 32ull);
                    base = __shfl_sync(kFull, base, 0);
                    if (base >= count) {
                        exhausted = true;
                        break;
                    }
                    pool_base = base;
                    pool_n = (uint32_t)min(32ull, count - base);
                    pool_used = 0;
                    if ((uint32_t)lane < pool_n) {
                        rec = __ldg(a.srcrec + base + lane);
                        if (a.srcpick) prec = __ldg(a.srcpick + base + lane);
                    }
                }
                const uint32_t take = min((uint32_t)__popc(idle), pool_n - pool_used);
                const uint32_t rank = __popc(idle & lanemask_lt());
                const int from = (int)min(pool_used + rank, 31u);
                const uint32_t rv_src = __shfl_sync(kFull, rec.x, from);
                const uint32_t rv_deg = __shfl_sync(kFull, rec.y, from);
                const uint32_t rv_off = __shfl_sync(kFull, rec.z, from);
                const uint32_t rv_tau = __shfl_sync(kFull, rec.w, from);
                const uint32_t pk_e = __shfl_sync(kFull, prec.x, from);
                const uint32_t pk_u = __shfl_sync(kFull, prec.y, from);
                if (!busy && rank < take) {
                    j = input_id(a, pool_base + pool_used + rank);
                    v = rv_src;  // Alg. 1's source, drawn by k_sources
                    if (rv_deg > a.max_deg) {
                        hand_on(a, j);
                    } else {
                        busy = true;
                        first = true;
                        any = false;
                        pf_ok = false;
                        r = 0;
                        mine[0] = (int32_t)v;
                        sig = member_bit(v);
                        len = 1;
                        head = 1;
                        src_deg = rv_deg;
                        tau_row = rv_tau;
                        lo = rv_off;
                        hi = rv_off + rv_deg;
                        q_last = hi > lo ? (hi - 1) >> 2 : lo >> 2;
                        if (a.srcpick) {  // bucket form: the picked in-edge, round-0 coins after it
                            mine[1] = (int32_t)pk_u;
                            sig |= member_bit(pk_u);
                            len = 2;
                            lo = pk_e + 1;
                            any = true;
                        }
                        qc = lo >> 2;
                        coins = 0;
                        steps = 0;
                    }
                }
                pool_used += take;
                idle = __ballot_sync(kFull, !busy);
            }
            if (!__any_sync(kFull, busy)) {
                if (exhausted) break;
                continue;
            }
        }
        if (!busy || done) continue;  // the lane waits for the next batch

        // ---- one edge quad: coins of the first step (round r) or of the
        // reverse BFS; a RIS source may have no in-edges
        bool handed = false, failed = false;
        uint32_t qdone = qc;  // the last quad drawn in this step
        if (hi > lo) {
            // up to two quads of the row per step: their thresholds, sources
            // and Philox blocks are independent, so their latencies overlap
            const bool two = qc < q_last;
            qdone = two ? qc + 1 : qc;
            const uint4 t4 = a.tau ? __ldg(tau4 + qc) : make_uint4(tau_row, tau_row, tau_row, tau_row);
            const uint4 t4b = (two && a.tau) ? __ldg(tau4 + qc + 1) : make_uint4(tau_row, tau_row, tau_row, tau_row);
            const uint32_t rr = first ? r : 0u, dom = first ? kDomFirst : kDomBfs;
            const uint4 x = coin_block(a.rk, qc, rr, dom, j);
            uint4 xb = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
            if (two) xb = coin_block(a.rk, qc + 1, rr, dom, j);
            const uint32_t e0 = qc << 2, e1 = e0 + 4;
            unsigned live = 0;
            live |= (e0 + 0 >= lo && e0 + 0 < hi && coin_live(x.x, t4.x)) ? 1u : 0u;
            live |= (e0 + 1 >= lo && e0 + 1 < hi && coin_live(x.y, t4.y)) ? 2u : 0u;
            live |= (e0 + 2 >= lo && e0 + 2 < hi && coin_live(x.z, t4.z)) ? 4u : 0u;
            live |= (e0 + 3 >= lo && e0 + 3 < hi && coin_live(x.w, t4.w)) ? 8u : 0u;
            if (two) {  // e1 > lo: only the row's end bounds the second quad
                live |= (e1 + 0 < hi && coin_live(xb.x, t4b.x)) ? 16u : 0u;
                live |= (e1 + 1 < hi && coin_live(xb.y, t4b.y)) ? 32u : 0u;
                live |= (e1 + 2 < hi && coin_live(xb.z, t4b.z)) ? 64u : 0u;
                live |= (e1 + 3 < hi && coin_live(xb.w, t4b.w)) ? 128u : 0u;
            }
            if (live) {
                any = true;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const unsigned lh = (live >> (4 * h)) & 15u;
                    if (!lh || handed) continue;
                    const int4 s4 = __ldg(src4 + qc + h);
                    const int32_t cand[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (!((lh >> k) & 1u) || handed) continue;
                        const int32_t u = cand[k];
                        bool seen = false;
                        if (sig & member_bit(u))  // else u is certainly new
                            for (uint32_t i = 0; i < len; ++i)
                                if (mine[i] == u) { seen = true; break; }
                        if (seen) continue;
                        if (len == (uint32_t)kLaneQ) handed = true;  // the warp tier takes it
                        else {
                            mine[len++] = u;
                            sig |= member_bit(u);
                        }
                    }
                }
            }
            steps += two ? 2u : 1u;
        }
        if (!handed && (hi <= lo || qdone >= q_last)) {  // the row is used up
            if (first) {
                if (any || a.ris) {
                    first = false;
                    coins = (uint64_t)src_deg * (r + 1);
                } else if (++r >= a.retry_cap) {
                    failed = true;
                } else if (r >= a.max_retries) {
                    handed = true;  // a rare source: the warp tier searches rounds in parallel
                } else {
                    qc = lo >> 2;  // next round over the same row
                }
            }
            if (!first && !failed && !handed) {
                // Alg. 1's reverse BFS: pop the next queued members until one
                // has in-edges (the first one's row was loaded ahead)
                bool row = false;
                while (!row && head < len) {
                    if (!pf_ok) {
                        const RowInfo rw = a.rows[mine[head]];
                        pf_off = (uint32_t)rw.off;
                        pf_deg = rw.deg;
                        pf_tau = rw.tau;
                    }
                    pf_ok = false;
                    ++head;
                    coins += pf_deg;
                    if (pf_deg > a.max_deg) {
                        handed = true;
                        break;
                    }
                    if (pf_deg > 0) {
                        row = true;
                        lo = pf_off;
                        hi = pf_off + pf_deg;
                        tau_row = pf_tau;
                        qc = lo >> 2;
                        q_last = (hi - 1) >> 2;
                    }
                }
                if (!row && !handed) done = true;
            }
        } else if (!handed) {
            qc = qdone + 1;
        }
        if (!done && !handed && steps > a.max_steps) handed = true;
        if (handed) hand_on(a, j);
        if (failed) record_retry_failure(a, j, v, r, src_deg);
        if (handed || failed) busy = false;
        // load the next pop's row ahead while this row's last quads are drawn
        if (busy && !done && !first && !pf_ok && head < len && q_last - qc <= 2u) {
            const RowInfo rw = a.rows[mine[head]];
            pf_off = (uint32_t)rw.off;
            pf_deg = rw.deg;
            pf_tau = rw.tau;
            pf_ok = true;
        }
    }
}

// ------------------------------------------------------------- warp tier
__global__ void __launch_bounds__(kWarpThreads) k_iis_warp(SampleArgs a) {
    __shared__ __align__(16) uint32_t s_hash[kWarpThreads / 32][kHCap];
    __shared__ __align__(16) int32_t s_queue[kWarpThreads / 32][kQCap];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* hash = s_hash[wib];
    int32_t* queue = s_queue[wib];
    uint64_t chunk_pos = 0, chunk_end = 0;  // this warp's arena reservation

    const uint64_t count = input_count(a);
    for (;;) {
        unsigned long long t0 = 0;
        if (lane == 0) t0 = atomicAdd(a.work, (unsigned long long)kIdBatch);
        t0 = __shfl_sync(kFull, t0, 0);
        if (t0 >= count) break;
        const uint64_t t1 = min((uint64_t)t0 + kIdBatch, count);
        for (uint64_t t = t0; t < t1; ++t) {
            const uint64_t j = input_id(a, t);
            // clear the visited set
#pragma unroll
            for (int i = lane; i < kHCap / 4; i += 32)
                reinterpret_cast<uint4*>(hash)[i] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
            __syncwarp();

            // Alg. 1: the source
            RowInfo rv;
            int64_t pe;
            int32_t pu;
            const uint32_t v = source_of(a, j, &rv, &pe, &pu);
            WarpInserter ins{hash, queue, 0u, false};
            ins.insert(lane == 0 ? (int32_t)v : -1);

            // the conditioned first step by rejection: all in-edge coins of v, round r
            bool failed = false;
            const uint32_t r = first_step_warp(a, j, rv, ins, &failed, pe, pu);
            if (failed) {
                if (lane == 0) record_retry_failure(a, j, v, r, rv.deg);
                continue;
            }

            // reverse BFS over the queue, up to 32 vertices at a time
            uint64_t coins = lane == 0 ? (uint64_t)rv.deg * (r + 1) : 0;
            uint64_t drawn = 0;  // in-edges of the rows taken so far (warp-uniform)
            bool heavy = false;
            uint32_t head = 1;
            while (head < ins.qlen && !ins.overflow) {
                const uint32_t cnt = min(ins.qlen - head, 32u);
                RowInfo rw;
                rw.off = 0; rw.deg = 0; rw.tau = 0;
                if ((uint32_t)lane < cnt) rw = a.rows[queue[head + lane]];
                // a sample that reaches huge in-rows goes to the CTA tier,
                // where every warp of a block shares its rows
                drawn += __reduce_add_sync(kFull, min(rw.deg, 1u << 26));
                if (drawn > a.warp_max_coins) {
                    heavy = true;
                    break;
                }
                coins += rw.deg;
                expand_rows(a, j, kDomBfs, 0, rw.off, rw.deg, rw.tau, ins);
                head += cnt;
            }
            if (ins.overflow || heavy) {  // too large for shared memory or too many coins: CTA tier
                if (lane == 0) hand_on(a, j);
                continue;
            }
            coins = warp_sum_u64(coins);

            // arena append from this warp's chunk
            const uint32_t len = ins.qlen;
            if (chunk_end - chunk_pos < len) {
                const uint64_t size = max((uint64_t)kArenaChunk, (uint64_t)len);
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.arena_cursor, (unsigned long long)size);
                base = __shfl_sync(kFull, base, 0);
                if (base + size > a.arena_cap) {
                    chunk_pos = chunk_end = 0;
                    if (lane == 0) arena_overflow(a, j);
                    continue;
                }
                chunk_pos = base;
                chunk_end = base + size;
            }
            for (uint32_t i = lane; i < len; i += 32) {
                a.arena[chunk_pos + i] = queue[i];
                count_member(a, queue[i]);
            }
            if (lane == 0) {
                a.h_off[j - a.id_base] = chunk_pos;
                a.h_len[j - a.id_base] = len;
                a.h_src[j - a.id_base] = v;
                a.h_retries[j - a.id_base] = r;
                a.h_coins[j - a.id_base] = coins;
            }
            chunk_pos += len;
            __syncwarp();
        }
    }
}

// -------------------------------------------------------------- CTA tier
// One block of kCtaThreads threads per sample, 1024 threads of such blocks per
// SM (four of 256 by default, or two of 512: the option SKIS_OPT_CTA_THREADS).
template <int kCtaThreads>
__global__ void __launch_bounds__(kCtaThreads, 1024 / kCtaThreads) k_iis_cta(SampleArgs a) {
    constexpr int kCtaWin = 2 * kCtaThreads;  // queued vertices per load-balanced window
    __shared__ unsigned long long s_j;
    __shared__ uint32_t s_qlen;
    __shared__ unsigned long long s_coins;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_r, s_failed;
    __shared__ uint32_t s_pre[kCtaWin], s_lo[kCtaWin], s_hi[kCtaWin], s_tau[kCtaWin];
    __shared__ uint32_t s_hub[kCtaWin];  // window rows taken by the hub loop
    __shared__ uint32_t s_nhub;
    __shared__ uint32_t s_small[3];      // a small window's quad-group shift, quad groups and hub rows
    __shared__ uint32_t s_wsum[kCtaThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int kWarps = kCtaThreads / 32;
    static_assert(kCtaWin == 2 * kCtaThreads, "two window rows per thread");
    uint32_t* bitmap = a.bitmaps + (uint64_t)blockIdx.x * a.bitmap_words;
    int32_t* queue = a.queues + (uint64_t)blockIdx.x * a.queue_cap;
    const uint64_t count = input_count(a);
    if (threadIdx.x == 0) s_nhub = 0;

    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long t = atomicAdd(a.work, 1ull);
            s_j = t < count ? input_id(a, t) : ~0ull;
        }
        __syncthreads();
        const uint64_t j = s_j;
        if (j == ~0ull) break;

        RowInfo rv;
        int64_t pe;
        int32_t pu;
        const uint32_t v = source_of(a, j, &rv, &pe, &pu);
        if (threadIdx.x == 0) {
            bitmap[v >> 5] |= 1u << (v & 31);
            queue[0] = (int32_t)v;
            s_qlen = 1;
            s_coins = 0;
        }
        __syncthreads();
        CtaInserter ins{bitmap, queue, &s_qlen, a.queue_cap, false};

        // first step: a short source row is searched by warp 0, several
        // rounds per pass; a long one is split over the warps in whole quads
        uint32_t r = 0;
        bool failed = false;
        const uint64_t nq_src = ((rv.off + rv.deg - 1) >> 2) - (rv.off >> 2) + 1;
        if (nq_src <= 16 || a.chain) {
            if (wid == 0) {
                bool f = false;
                const uint32_t rr = first_step_warp(a, j, rv, ins, &f, pe, pu);
                if (lane == 0) {
                    s_r = rr;
                    s_failed = f ? 1u : 0u;
                }
            }
            __syncthreads();
            r = s_r;
            failed = s_failed != 0;
        } else {
            const uint64_t q_lo = rv.off >> 2;
            const uint64_t nq = rv.deg ? ((rv.off + rv.deg - 1) >> 2) - q_lo + 1 : 0;
            const uint64_t per = (nq + kWarps - 1) / kWarps;
            const uint64_t a_lo = max(rv.off, (q_lo + (uint64_t)wid * per) << 2);
            const uint64_t a_hi = min(rv.off + rv.deg, (q_lo + (uint64_t)(wid + 1) * per) << 2);
            const uint32_t sub_deg = a_hi > a_lo ? (uint32_t)(a_hi - a_lo) : 0u;
            for (;;) {
                const bool any_w = expand_rows(a, j, kDomFirst, r, a_lo, lane == 0 ? sub_deg : 0u, rv.tau, ins);
                const int any = __syncthreads_or(any_w ? 1 : 0);
                if (any || a.ris) break;
                if (++r >= a.retry_cap) { failed = true; break; }
            }
        }
        if (failed) {
            if (threadIdx.x == 0) {
                record_retry_failure(a, j, v, r, rv.deg);
                bitmap[v >> 5] = 0;
            }
            __syncthreads();
            continue;
        }

        // reverse BFS, level by level. A level [head, tail) is taken in
        // windows of up to kCtaWin queued vertices; the edge quads of a
        // window's rows are laid end to end and dealt to the warps 32 at a
        // time, so one long in-row (a hub) is shared by every warp.
        uint64_t coins = 0;
        uint32_t head = 1;
        uint32_t tail = s_qlen;  // after the first step's barrier: its inserts are in
        for (;;) {
            if (head >= tail || tail > a.queue_cap) break;  // done, or the sample outgrew the slot
            for (uint32_t w0 = head; w0 < tail; w0 += kCtaWin) {
                const uint32_t nw = min((uint32_t)kCtaWin, tail - w0);
                uint32_t gsh, total, nhub;  // quad-group shift, quad groups and hub rows of the window
                if (nw <= 32) {
                    // a small window (the narrow frontiers of weighted cascade):
                    // warp 0 loads, classifies and prefixes its rows, one barrier
                    if (wid == 0) {
                        uint32_t nq = 0;
                        bool hub = false;
                        if ((uint32_t)lane < nw) {
                            const RowInfo rw = a.rows[queue[w0 + lane]];
                            coins += rw.deg;
                            const uint32_t lo = (uint32_t)rw.off, hi = lo + rw.deg;
                            s_lo[lane] = lo;
                            s_hi[lane] = hi;
                            s_tau[lane] = rw.tau;
                            nq = rw.deg ? ((hi - 1) >> 2) - (lo >> 2) + 1 : 0u;  // edge quads
                            hub = a.cta_hub_quads && nq >= a.cta_hub_quads;
                            if (hub) nq = 0;  // the hub loop takes it
                        }
                        const unsigned hb = __ballot_sync(kFull, hub);
                        if (hub) s_hub[__popc(hb & lanemask_lt())] = (uint32_t)lane;
                        const uint32_t g = __any_sync(kFull, nq >= (uint32_t)kCtaLongRow) ? (uint32_t)kCtaGroupLog2 : 0u;
                        uint32_t x = (nq + (1u << g) - 1) >> g;
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const uint32_t y = __shfl_up_sync(kFull, x, d);
                            if (lane >= d) x += y;
                        }
                        if ((uint32_t)lane < nw) s_pre[lane] = x;
                        if (lane == 31) {
                            s_small[0] = g;
                            s_small[1] = x;
                            s_small[2] = (uint32_t)__popc(hb);
                        }
                    }
                    __syncthreads();
                    gsh = s_small[0];
                    total = s_small[1];
                    nhub = s_small[2];
                } else {
                uint32_t nq2[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t i = 2u * threadIdx.x + h;
                    nq2[h] = 0;
                    if (i < nw) {
                        const RowInfo rw = a.rows[queue[w0 + i]];
                        coins += rw.deg;
                        const uint32_t lo = (uint32_t)rw.off, hi = lo + rw.deg;
                        s_lo[i] = lo;
                        s_hi[i] = hi;
                        s_tau[i] = rw.tau;
                        nq2[h] = rw.deg ? ((hi - 1) >> 2) - (lo >> 2) + 1 : 0u;  // edge quads
                        if (a.cta_hub_quads && nq2[h] >= a.cta_hub_quads) {  // the hub loop takes it
                            s_hub[atomicAdd(&s_nhub, 1u)] = i;
                            nq2[h] = 0;
                        }
                    }
                }
                // a window with a long row (a hub) deals its quads kCtaGroup at
                // a time to amortise the row search; others one at a time, so
                // that short rows keep every lane busy
                gsh = __syncthreads_or(nq2[0] >= (uint32_t)kCtaLongRow || nq2[1] >= (uint32_t)kCtaLongRow)
                          ? (uint32_t)kCtaGroupLog2 : 0u;  // group of 2^gsh quads
                const uint32_t grp0 = 1u << gsh;
#pragma unroll
                for (int h = 0; h < 2; ++h) nq2[h] = (nq2[h] + grp0 - 1) >> gsh;
                // block-wide inclusive prefix of the quad-group counts
                const uint32_t pair = nq2[0] + nq2[1];
                uint32_t x = pair;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, x, d);
                    if (lane >= d) x += y;
                }
                if (lane == 31) s_wsum[wid] = x;
                __syncthreads();
                // every thread reads the hub count between these two barriers,
                // and it is cleared after the second, before any thread can
                // classify the next window's rows
                nhub = s_nhub;
                if (wid == 0) {
                    uint32_t w = lane < kWarps ? s_wsum[lane] : 0u;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const uint32_t y = __shfl_up_sync(kFull, w, d);
                        if (lane >= d) w += y;
                    }
                    if (lane < kWarps) s_wsum[lane] = w;
                }
                __syncthreads();
                if (threadIdx.x == 0) s_nhub = 0;
                const uint32_t before = (wid ? s_wsum[wid - 1] : 0u) + x - pair;
                if (2u * threadIdx.x < nw) s_pre[2u * threadIdx.x] = before + nq2[0];
                if (2u * threadIdx.x + 1 < nw) s_pre[2u * threadIdx.x + 1] = before + pair;
                __syncthreads();
                total = s_pre[nw - 1];
                }
                const uint32_t grp = 1u << gsh;
                // quad group g (nothing when g is past the window): quads q ..
                // q + grp - 1 of one row, independent Philox blocks; a
                // quad inside the row skips the edge bounds. Returns the live
                // edges as a bit mask (bit 4h + k: edge k of quad q + h).
                auto draw = [&](uint32_t g, uint32_t* q_out) -> unsigned {
                    *q_out = 0;
                    if (g >= total) return 0u;
                    uint32_t i = 0;  // the row of group g: entries with prefix <= g
                    // (steps from the window's own size: a lone hub row needs none)
                    for (uint32_t b = nw > 1 ? 1u << (31 - __clz(nw - 1)) : 0u; b; b >>= 1)
                        if (i + b - 1 < nw && s_pre[i + b - 1] <= g) i += b;
                    const uint32_t lo = s_lo[i], hi = s_hi[i], tr = s_tau[i];
                    const uint32_t q = (lo >> 2) + ((g - (i ? s_pre[i - 1] : 0u)) << gsh);
                    const uint32_t q_last = (hi - 1) >> 2;
                    *q_out = q;
                    unsigned live = 0;
#pragma unroll
                    for (int h = 0; h < kCtaGroup; ++h) {
                        const uint32_t qh = q + h;
                        if ((uint32_t)h >= grp || qh > q_last) break;
                        const uint4 x = coin_block(a.rk, qh, 0, kDomBfs, j);
                        const uint4 t4 = a.tau ? __ldg(reinterpret_cast<const uint4*>(a.tau) + qh)
                                               : make_uint4(tr, tr, tr, tr);
                        const uint32_t e0 = qh << 2;
                        unsigned l4 = 0;
                        if (e0 >= lo && e0 + 4 <= hi) {
                            l4 |= coin_live(x.x, t4.x) ? 1u : 0u;
                            l4 |= coin_live(x.y, t4.y) ? 2u : 0u;
                            l4 |= coin_live(x.z, t4.z) ? 4u : 0u;
                            l4 |= coin_live(x.w, t4.w) ? 8u : 0u;
                        } else {
                            l4 |= (e0 + 0 >= lo && e0 + 0 < hi && coin_live(x.x, t4.x)) ? 1u : 0u;
                            l4 |= (e0 + 1 >= lo && e0 + 1 < hi && coin_live(x.y, t4.y)) ? 2u : 0u;
                            l4 |= (e0 + 2 >= lo && e0 + 2 < hi && coin_live(x.z, t4.z)) ? 4u : 0u;
                            l4 |= (e0 + 3 >= lo && e0 + 3 < hi && coin_live(x.w, t4.w)) ? 8u : 0u;
                        }
                        live |= l4 << (4 * h);
                    }
                    return live;
                };
                // one group (32 grp quads) per warp step; the
                // sources of live edges are loaded only when some lane has one
                for (uint32_t c = wid; c * 32u < total; c += kWarps) {
                    uint32_t q;
                    const unsigned live = draw(c * 32u + lane, &q);
                    if (!__any_sync(kFull, live != 0u)) continue;
#pragma unroll
                    for (int h = 0; h < kCtaGroup; ++h) {
                        const unsigned lh = (live >> (4 * h)) & 15u;
                        if (!__any_sync(kFull, lh != 0u)) continue;
                        int4 s4 = make_int4(-1, -1, -1, -1);
                        if (lh) s4 = __ldg(reinterpret_cast<const int4*>(a.src) + q + h);
                        const int32_t cand[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int32_t u = ((lh >> k) & 1u) ? cand[k] : -1;
                            if (__any_sync(kFull, u >= 0)) ins.insert(u);
                        }
                    }
                }
                // hub rows: their quads laid end to end and strided over the
                // block, so a thread runs straight down a row with no search
                // and no per-edge bounds; a live coin is rare there (WC: one
                // expected per row) and is inserted by its lane alone
                if (nhub) {
                    const SampleBlock blk(a.rk, j, kDomBfs);
                    const uint4* __restrict__ tau4 = reinterpret_cast<const uint4*>(a.tau);
                    // the live coins of quad q (Philox block x) within [lo, hi) join the sample
                    auto take = [&](uint32_t q, const uint4& x, const uint4& t4, uint32_t lo, uint32_t hi) {
                        const uint32_t e0 = q << 2;
                        unsigned l4 = 0;
                        l4 |= (e0 + 0 >= lo && e0 + 0 < hi && coin_live(x.x, t4.x)) ? 1u : 0u;
                        l4 |= (e0 + 1 >= lo && e0 + 1 < hi && coin_live(x.y, t4.y)) ? 2u : 0u;
                        l4 |= (e0 + 2 >= lo && e0 + 2 < hi && coin_live(x.z, t4.z)) ? 4u : 0u;
                        l4 |= (e0 + 3 >= lo && e0 + 3 < hi && coin_live(x.w, t4.w)) ? 8u : 0u;
                        if (l4) {
                            const int4 s4 = __ldg(reinterpret_cast<const int4*>(a.src) + q);
                            if (l4 & 1u) cta_insert_one(bitmap, queue, &s_qlen, a.queue_cap, s4.x);
                            if (l4 & 2u) cta_insert_one(bitmap, queue, &s_qlen, a.queue_cap, s4.y);
                            if (l4 & 4u) cta_insert_one(bitmap, queue, &s_qlen, a.queue_cap, s4.z);
                            if (l4 & 8u) cta_insert_one(bitmap, queue, &s_qlen, a.queue_cap, s4.w);
                        }
                    };
                    auto min4 = [](const uint4& x) { return min(min(x.x, x.y), min(x.z, x.w)); };
                    uint32_t g = threadIdx.x;
                    for (uint32_t h = 0; h < nhub; ++h) {
                        const uint32_t i = s_hub[h];
                        const uint32_t lo = s_lo[i], hi = s_hi[i], tr = s_tau[i];
                        const uint32_t qf = lo >> 2, nq = ((hi - 1) >> 2) - qf + 1;
                        if (!tau4) {
                            // one threshold for the row (never the sentinel: a hub row has many
                            // edges): two independent blocks a step, one compare of their minimum
                            const uint4 tr4 = make_uint4(tr, tr, tr, tr);
                            for (; g + kCtaThreads < nq; g += 2 * kCtaThreads) {
                                const uint32_t q0 = qf + g, q1 = q0 + kCtaThreads;
                                const uint4 x0 = blk(q0, a.rk), x1 = blk(q1, a.rk);
                                if (min(min4(x0), min4(x1)) < tr || tr == kSentinel) {
                                    take(q0, x0, tr4, lo, hi);
                                    take(q1, x1, tr4, lo, hi);
                                }
                            }
                            for (; g < nq; g += kCtaThreads) {
                                const uint32_t q = qf + g;
                                const uint4 x = blk(q, a.rk);
                                if (min4(x) < tr || tr == kSentinel) take(q, x, tr4, lo, hi);
                            }
                        } else {
                            for (; g < nq; g += kCtaThreads) {
                                const uint32_t q = qf + g;
                                const uint4 x = blk(q, a.rk);
                                const uint4 t4 = __ldg(tau4 + q);
                                if (coin_live(x.x, t4.x) | coin_live(x.y, t4.y) | coin_live(x.z, t4.z) |
                                    coin_live(x.w, t4.w))
                                    take(q, x, t4, lo, hi);
                            }
                        }
                        g -= nq;
                    }
                }
                __syncthreads();  // the window's shared arrays are reused
            }
            head = tail;
            tail = s_qlen;  // after the level's last barrier: every insert of the level is in
        }
        coins = warp_sum_u64(coins);
        if (lane == 0 && coins) atomicAdd(&s_coins, (unsigned long long)coins);
        __syncthreads();
        const uint32_t len = s_qlen;
        const bool outgrown = len > a.queue_cap;  // the queue kept its first queue_cap members only
        if (threadIdx.x == 0) {
            const unsigned long long base = outgrown ? 0ull : atomicAdd(a.arena_cursor, (unsigned long long)len);
            if (outgrown) {  // to the pass whose slots hold n-entry queues
                if (a.out_ids) hand_on(a, j);
                else atomicOr(&a.status->flags, kStListFull);
                s_base = ~0ull;
            } else if (base + len > a.arena_cap) {
                arena_overflow(a, j);
                s_base = ~0ull;
            } else {
                s_base = base;
                a.h_off[j - a.id_base] = base;
                a.h_len[j - a.id_base] = len;
                a.h_src[j - a.id_base] = v;
                a.h_retries[j - a.id_base] = r;
                a.h_coins[j - a.id_base] = (uint64_t)rv.deg * (r + 1) + s_coins;
            }
        }
        __syncthreads();
        const unsigned long long base = s_base;
        for (uint32_t i = threadIdx.x; i < min(len, a.queue_cap); i += kCtaThreads) {
            const int32_t u = queue[i];
            if (base != ~0ull) {
                a.arena[base + i] = u;
                count_member(a, u);
            }
            bitmap[(uint32_t)u >> 5] = 0;  // restore the all-zero bitmap
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------- LT walks
// Linear Threshold samples (Sec. "Extensions to other diffusion models",
// LT): the source by Eq. probu with gamma_v = the row's weight sum, exactly
// one in-neighbour picked with probability w(u,v) / gamma_v, then the
// reverse walk of RIS for LT: from the last member x, one draw picks at most
// one in-edge of x (edge i when P_{i-1} <= y < P_i for the running weight
// sums P, none when y >= P_d); the walk ends when none is picked or the
// picked vertex is already in R_j. Step t of sample j draws the Philox block
// (q = t, domain LT, sample j): step 0 conditioned (64-bit U, y = floor(U S
// / 2^64)), later steps y = its word 0. Two tiers: one lane per sample with
// up to kLtQ members in shared memory, then one warp per CTA-tier slot with
// the slot's global visited bitmap and queue.
constexpr int kLtBlock = 256;
constexpr int kLtQ = 48;

__device__ __forceinline__ uint64_t lt_weight(uint32_t tau) { return tau == kSentinel ? (1ull << 32) : (uint64_t)tau; }

// one walk step from a vertex with in-row rw: the picked in-neighbour, or -1
// when the walk ends there
__device__ __forceinline__ int32_t lt_step(const SampleArgs& a, uint64_t j, uint32_t t, const RowInfo& rw) {
    if (rw.deg == 0) return -1;
    const uint64_t base = a.lt_cum ? a.lt_cum[rw.off] : 0;
    const uint64_t S = a.lt_cum ? a.lt_cum[rw.off + rw.deg] - base : (uint64_t)rw.deg * lt_weight(rw.tau);
    const uint4 b = coin_block(a.rk, t, 0, kDomLt, j);
    uint64_t y;
    if (t == 0 && !a.ris) {
        y = __umul64hi((uint64_t)b.x | ((uint64_t)b.y << 32), S);  // Pr[u] = w(u, v) / gamma_v
    } else {
        y = b.x;
        if (y >= S) return -1;  // no in-edge kept
    }
    uint32_t i;
    if (!a.lt_cum) {
        i = (uint32_t)(y / lt_weight(rw.tau));
    } else {  // the first position whose running sum exceeds y
        uint32_t lo = 0, hi = rw.deg - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.lt_cum[rw.off + mid + 1] - base > y) hi = mid;
            else lo = mid + 1;
        }
        i = lo;
    }
    return a.src[rw.off + i];
}

__global__ void __launch_bounds__(kLtBlock) k_lt_walk(SampleArgs a) {
    __shared__ int32_t s_q[kLtBlock / 32][kLtQ][32];
    const int lane = threadIdx.x & 31;
    int32_t(*const mq)[32] = s_q[threadIdx.x >> 5];  // mq[k][lane]: member k of this lane's sample
    const uint64_t count = input_count(a);
    bool busy = false, exhausted = false;
    uint64_t j = 0, coins = 0;
    uint32_t v = 0, len = 0, t = 0;
    int32_t x = 0;
    uint64_t chunk_pos = 0, chunk_end = 0;

    for (;;) {
        const unsigned idle = __ballot_sync(kFull, !busy);
        if (idle && !exhausted) {
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(a.work, (unsigned long long)__popc(idle));
            base = __shfl_sync(kFull, base, leader);
            if (base + __popc(idle) >= count) exhausted = true;
            if (!busy) {
                const uint64_t ti = base + __popc(idle & lanemask_lt());
                if (ti < count) {
                    j = input_id(a, ti);
                    v = draw_source(a, j);
                    x = (int32_t)v;
                    mq[0][lane] = x;
                    len = 1;
                    t = 0;
                    coins = 0;
                    busy = true;
                }
            }
        }
        if (!__any_sync(kFull, busy)) {
            if (exhausted) break;
            continue;
        }
        bool done = false;
        if (busy) {
            const RowInfo rw = a.rows[x];
            coins += rw.deg;
            const int32_t u = lt_step(a, j, t, rw);
            ++t;
            if (u < 0) {
                done = true;
            } else {
                bool seen = false;
                for (uint32_t i = 0; i < len; ++i)
                    if (mq[i][lane] == u) { seen = true; break; }
                if (seen) {
                    done = true;  // the walk closes on R_j
                } else if (len == (uint32_t)kLtQ) {
                    hand_on(a, j);  // a long walk: the slot tier redraws it
                    busy = false;
                } else {
                    mq[len++][lane] = u;
                    x = u;
                }
            }
        }
        const unsigned dm = __ballot_sync(kFull, done);
        if (dm) {
            const uint32_t mylen = done ? len : 0u;
            uint32_t incl = mylen;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, d);
                if (lane >= d) incl += y;
            }
            const uint32_t total = __shfl_sync(kFull, incl, 31);
            bool fits = true;
            if (chunk_end - chunk_pos < total) {
                const uint64_t size = max((uint64_t)kLaneArenaChunk, (uint64_t)total);
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.arena_cursor, (unsigned long long)size);
                base = __shfl_sync(kFull, base, 0);
                if (base + size > a.arena_cap) {
                    fits = false;
                    chunk_pos = chunk_end = 0;
                } else {
                    chunk_pos = base;
                    chunk_end = base + size;
                }
            }
            if (done) {
                if (fits) {
                    const uint64_t at = chunk_pos + (incl - mylen);
                    for (uint32_t i = 0; i < len; ++i) {
                        a.arena[at + i] = mq[i][lane];
                        count_member(a, mq[i][lane]);
                    }
                    a.h_off[j - a.id_base] = at;
                    a.h_len[j - a.id_base] = len;
                    a.h_src[j - a.id_base] = v;
                    a.h_retries[j - a.id_base] = 0;
                    a.h_coins[j - a.id_base] = coins;
                } else {
                    arena_overflow(a, j);
                }
                busy = false;
            }
            if (fits) chunk_pos += total;
        }
    }
}

// Medium LT walks: one lane per walk with its own open-addressing visited
// table (kLtMidHash slots, at most half full) and member list in global
// memory; the table is restored to empty slot by slot after each walk. A
// walk longer than kLtMidCap is handed on to the slot tier.
constexpr int kLtMidBlock = 256;
constexpr uint32_t kLtMidHash = 2048;
constexpr uint32_t kLtMidCap = 1024;

__global__ void __launch_bounds__(kLtMidBlock) k_lt_mid(SampleArgs a, uint32_t* __restrict__ hash_all,
                                                        int32_t* __restrict__ list_all,
                                                        uint32_t* __restrict__ slot_all) {
    const uint64_t me = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t* hash = hash_all + me * kLtMidHash;
    int32_t* list = list_all + me * kLtMidCap;
    uint32_t* slot = slot_all + me * kLtMidCap;
    const uint64_t count = input_count(a);
    for (;;) {
        const unsigned long long ti = atomicAdd(a.work, 1ull);
        if (ti >= count) break;
        const uint64_t j = input_id(a, ti);
        const uint32_t v = draw_source(a, j);
        uint32_t len = 0;
        bool over = false;
        uint64_t coins = 0;
        int32_t x = (int32_t)v;
        for (uint32_t t = 0;; ++t) {  // each step adds a new member or ends the walk
            // x joins the visited table and the list
            uint32_t h = ((uint32_t)x * 2654435761u) & (kLtMidHash - 1);
            while (hash[h] != kEmpty) h = (h + 1) & (kLtMidHash - 1);  // x is new: a free slot exists
            hash[h] = (uint32_t)x;
            slot[len] = h;
            list[len++] = x;
            const RowInfo rw = a.rows[x];
            coins += rw.deg;
            const int32_t u = lt_step(a, j, t, rw);
            if (u < 0) break;
            uint32_t g = ((uint32_t)u * 2654435761u) & (kLtMidHash - 1);
            bool seen = false;
            for (;;) {  // the table is at most half full: the probe ends
                const uint32_t key = hash[g];
                if (key == kEmpty) break;
                if (key == (uint32_t)u) { seen = true; break; }
                g = (g + 1) & (kLtMidHash - 1);
            }
            if (seen) break;
            if (len == kLtMidCap) {
                over = true;
                break;
            }
            x = u;
        }
        if (over) {
            hand_on(a, j);
        } else {
            const unsigned long long base = atomicAdd(a.arena_cursor, (unsigned long long)len);
            if (base + len <= a.arena_cap) {
                for (uint32_t i = 0; i < len; ++i) {
                    a.arena[base + i] = list[i];
                    count_member(a, list[i]);
                }
                a.h_off[j - a.id_base] = base;
                a.h_len[j - a.id_base] = len;
                a.h_src[j - a.id_base] = v;
                a.h_retries[j - a.id_base] = 0;
                a.h_coins[j - a.id_base] = coins;
            } else {
                arena_overflow(a, j);
            }
        }
        for (uint32_t i = 0; i < len; ++i) hash[slot[i]] = kEmpty;
    }
}

// Long LT walks: one warp per slot; lane 0 walks with the slot's global
// visited bitmap and queue, the warp copies the members out and clears the
// bitmap.
__global__ void __launch_bounds__(32) k_lt_long(SampleArgs a) {
    const int lane = threadIdx.x & 31;
    uint32_t* bitmap = a.bitmaps + (uint64_t)blockIdx.x * a.bitmap_words;
    int32_t* queue = a.queues + (uint64_t)blockIdx.x * a.queue_cap;
    const uint64_t count = input_count(a);
    for (;;) {
        unsigned long long ti = 0;
        if (lane == 0) ti = atomicAdd(a.work, 1ull);
        ti = __shfl_sync(kFull, ti, 0);
        if (ti >= count) break;
        const uint64_t j = input_id(a, ti);
        uint32_t len = 0, v = 0, outgrown = 0;
        uint64_t coins = 0;
        if (lane == 0) {
            v = draw_source(a, j);
            bitmap[v >> 5] |= 1u << (v & 31);
            queue[0] = (int32_t)v;
            len = 1;
            int32_t x = (int32_t)v;
            for (uint32_t t = 0;; ++t) {  // at most n steps: each adds a new member
                const RowInfo rw = a.rows[x];
                coins += rw.deg;
                const int32_t u = lt_step(a, j, t, rw);
                if (u < 0) break;
                const uint32_t bit = 1u << (u & 31);
                if (bitmap[(uint32_t)u >> 5] & bit) break;
                if (len == a.queue_cap) {  // the walk outgrew the slot's queue
                    outgrown = 1;
                    break;
                }
                bitmap[(uint32_t)u >> 5] |= bit;
                queue[len++] = u;
                x = u;
            }
        }
        __syncwarp();
        len = __shfl_sync(kFull, len, 0);
        v = __shfl_sync(kFull, v, 0);
        coins = __shfl_sync(kFull, coins, 0);
        outgrown = __shfl_sync(kFull, outgrown, 0);
        unsigned long long base = 0;
        if (lane == 0 && !outgrown) base = atomicAdd(a.arena_cursor, (unsigned long long)len);
        base = __shfl_sync(kFull, base, 0);
        const bool fits = !outgrown && base + len <= a.arena_cap;
        for (uint32_t i = lane; i < len; i += 32) {
            const int32_t u = queue[i];
            if (fits) {
                a.arena[base + i] = u;
                count_member(a, u);
            }
            bitmap[(uint32_t)u >> 5] = 0;  // restore the all-zero bitmap
        }
        if (lane == 0) {
            if (fits) {
                a.h_off[j - a.id_base] = base;
                a.h_len[j - a.id_base] = len;
                a.h_src[j - a.id_base] = v;
                a.h_retries[j - a.id_base] = 0;
                a.h_coins[j - a.id_base] = coins;
            } else if (outgrown) {  // to the pass whose slots hold n-entry queues
                if (a.out_ids) hand_on(a, j);
                else atomicOr(&a.status->flags, kStListFull);
            } else {
                arena_overflow(a, j);
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ host
#define SK_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t _e = (call);                                                        \
        if (_e != cudaSuccess) {                                                        \
            *err = std::string("CUDA error in skis_sample: ") + cudaGetErrorString(_e); \
            return _e == cudaErrorMemoryAllocation ? SKIS_ENOMEM : SKIS_ERR_CUDA;       \
        }                                                                               \
    } while (0)

template <typename T>
static cudaError_t grow_copy(T** p, uint64_t old_n, uint64_t new_n, cudaStream_t st) {
    T* q = nullptr;
    cudaError_t e = dev_alloc_t(&q, (size_t)new_n, st);
    if (e != cudaSuccess) return e;
    if (*p && old_n) {
        e = cudaMemcpyAsync(q, *p, old_n * sizeof(T), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { dev_free(q, st); return e; }
    }
    dev_free(*p, st);
    *p = q;
    return cudaSuccess;
}

static int ensure_sample_buffers(skis_sketch* s, uint64_t count, cudaStream_t st, std::string* err) {
    const skis_graph* g = s->g;
    if (!s->ctr) {
        SK_CUDA(dev_alloc_t(&s->ctr, 1, st));
        SK_CUDA(cudaMemsetAsync(s->ctr, 0, sizeof(SampleCounters), st));
        SK_CUDA(dev_alloc_t(&s->status, 1, st));
        for (int i = 0; i < 4; ++i) SK_CUDA(cudaEventCreate(&s->ev[i]));
    }
    const uint64_t need = s->T + count;
    if (need > s->hcap) {
        const uint64_t nc = std::max<uint64_t>(need, s->hcap * 2);
        SK_CUDA(grow_copy(&s->h_off, s->T, nc, st));
        SK_CUDA(grow_copy(&s->h_len, s->T, nc, st));
        SK_CUDA(grow_copy(&s->h_src, s->T, nc, st));
        SK_CUDA(grow_copy(&s->h_retries, s->T, nc, st));
        SK_CUDA(grow_copy(&s->h_coins, s->T, nc, st));
        s->hcap = nc;
    }
    if (count > s->list_cap) {
        dev_free(s->to_warp_ids, st);
        dev_free(s->to_cta_ids, st);
        dev_free(s->big_ids, st);
        dev_free(s->ovf_ids[0], st);
        dev_free(s->ovf_ids[1], st);
        s->to_warp_ids = s->to_cta_ids = s->big_ids = s->ovf_ids[0] = s->ovf_ids[1] = nullptr;
        SK_CUDA(dev_alloc_t(&s->to_warp_ids, (size_t)count, st));
        SK_CUDA(dev_alloc_t(&s->to_cta_ids, (size_t)count, st));
        SK_CUDA(dev_alloc_t(&s->big_ids, (size_t)count, st));
        SK_CUDA(dev_alloc_t(&s->ovf_ids[0], (size_t)count, st));
        SK_CUDA(dev_alloc_t(&s->ovf_ids[1], (size_t)count, st));
        dev_free(s->srcrec, st);
        dev_free(s->srcpick, st);
        s->srcrec = nullptr;
        s->srcpick = nullptr;
        SK_CUDA(dev_alloc_t(&s->srcrec, (size_t)count, st));
        SK_CUDA(dev_alloc_t(&s->srcpick, (size_t)count, st));
        s->list_cap = count;
    }
    if (!s->arena) {
        uint64_t cap = s->arena_hint ? s->arena_hint : std::max<uint64_t>(count * 8, 1u << 20);
        SK_CUDA(dev_alloc_t(&s->arena, (size_t)cap, st));
        s->arena_cap = cap;
    }
    if (g->lt && !s->lt_hash) {  // medium LT walks: one table, list and slot record per lane
        s->lt_mid_lanes = (uint64_t)sm_count() * kLtMidBlock * 2;  // two blocks per SM
        SK_CUDA(dev_alloc_t(&s->lt_hash, (size_t)(s->lt_mid_lanes * kLtMidHash), st));
        SK_CUDA(cudaMemsetAsync(s->lt_hash, 0xFF, s->lt_mid_lanes * kLtMidHash * sizeof(uint32_t), st));
        SK_CUDA(dev_alloc_t(&s->lt_list, (size_t)(s->lt_mid_lanes * kLtMidCap), st));
        SK_CUDA(dev_alloc_t(&s->lt_slot, (size_t)(s->lt_mid_lanes * kLtMidCap), st));
    }
    // CTA-tier slots: an n-bit visited bitmap and a queue of min(n, cta_queue_cap)
    // entries each (a sample with more members moves to a pass over slots with
    // n-entry queues), 1024 threads of blocks per SM within ~8 GB
    const uint32_t qcap = (uint32_t)std::min<uint64_t>((uint64_t)g->n, s->cta_queue_cap);
    int slots = s->cta_slots;
    if (slots <= 0) {
        const uint64_t per_slot = (uint64_t)qcap * 4 + ((uint64_t)g->n + 31) / 32 * 4;
        const uint64_t budget = 8ull << 30;
        const uint64_t per_sm = g->lt ? 2 : 1024 / s->cta_threads;
        slots = (int)std::min<uint64_t>((uint64_t)sm_count() * per_sm, std::max<uint64_t>(1, budget / per_slot));
    }
    if (slots != s->cta_slots_alloc || qcap != s->queue_cap) {
        dev_free(s->bitmaps, st);
        dev_free(s->queues, st);
        s->bitmaps = nullptr;
        s->queues = nullptr;
        s->bitmap_words = ((uint64_t)g->n + 31) / 32;
        SK_CUDA(dev_alloc_t(&s->bitmaps, (size_t)(s->bitmap_words * slots), st));
        SK_CUDA(cudaMemsetAsync(s->bitmaps, 0, s->bitmap_words * slots * sizeof(uint32_t), st));
        SK_CUDA(dev_alloc_t(&s->queues, (size_t)((uint64_t)qcap * slots), st));
        s->cta_slots_alloc = slots;
        s->queue_cap = qcap;
    }
    return SKIS_OK;
}

// The pass over samples that outgrew a CTA-tier slot's queue: slots with
// n-entry queues (their bitmaps are the first slots' of the CTA tier, all
// zero between launches), allocated on first use within ~8 GB.
static int ensure_big_slots(skis_sketch* s, cudaStream_t st, std::string* err) {
    if (s->big_queues) return SKIS_OK;
    const uint64_t n = (uint64_t)s->g->n;
    const uint64_t budget = 8ull << 30;
    const int slots = (int)std::min<uint64_t>((uint64_t)s->cta_slots_alloc, std::max<uint64_t>(1, budget / (n * 4)));
    SK_CUDA(dev_alloc_t(&s->big_queues, (size_t)(n * slots), st));
    s->big_slots = slots;
    return SKIS_OK;
}

static int occupancy_grid(const void* kernel, int threads, int override_blocks, uint64_t max_useful,
                          std::string* err, int* out) {
    int blocks = override_blocks;
    if (blocks <= 0) {
        int per_sm = 0;
        SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0));
        blocks = sm_count() * std::max(per_sm, 1);
    }
    *out = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)blocks, max_useful));
    return SKIS_OK;
}

int sketch_sample(skis_sketch* s, uint64_t count, cudaStream_t st, std::string* err) {
    const skis_graph* g = s->g;
    if (g->W == 0 && !s->ris) {
        *err = "skis_sample: Gamma = 0, the graph has no non-singular sample";
        return SKIS_EINVAL;
    }
    if (count == 0) return SKIS_OK;
    int rc = ensure_sample_buffers(s, count, st, err);
    if (rc != SKIS_OK) return rc;
    const bool thread_tier = s->thread_max_deg > 0;
    int warp_blocks = 0, lane_blocks = 0;
    rc = occupancy_grid((const void*)k_iis_lane, kLaneBlock, s->thread_blocks,
                        (count + kLaneBlock - 1) / kLaneBlock, err, &lane_blocks);
    if (rc != SKIS_OK) return rc;
    rc = occupancy_grid((const void*)k_iis_warp, kWarpThreads, s->warp_blocks,
                        thread_tier ? UINT64_MAX : (count + kIdBatch - 1) / kIdBatch, err, &warp_blocks);
    if (rc != SKIS_OK) return rc;

    SampleArgs base;
    base.alias = g->alias;
    base.rows = g->rows;
    base.src = g->src;
    base.tau = g->row_uniform ? nullptr : g->tau;
    base.n = (uint64_t)g->n;
    base.W = g->W;
    base.seed = s->seed;
    base.rk = philox_keys(s->seed);
    base.retry_cap = s->retry_cap;
    base.max_deg = s->thread_max_deg;
    base.max_steps = s->thread_max_steps;
    base.max_retries = s->thread_max_retries;
    base.warp_max_coins = s->warp_max_coins;
    base.cta_hub_quads = s->cta_hub_quads;
    base.ris = s->ris;
    base.ids = nullptr;
    base.first_id = s->id_base + s->T;
    base.id_base = s->id_base;
    base.count = count;
    base.count_dev = nullptr;
    base.arena_cursor = &s->ctr->arena;
    base.novf = &s->ctr->novf;
    base.h_off = s->h_off;
    base.h_len = s->h_len;
    base.h_src = s->h_src;
    base.h_retries = s->h_retries;
    base.h_coins = s->h_coins;
    base.arena = s->arena;
    base.arena_cap = s->arena_cap;
    base.status = s->status;
    base.bitmaps = s->bitmaps;
    base.queues = s->queues;
    base.bitmap_words = s->bitmap_words;
    base.queue_cap = s->queue_cap;
    base.srcrec = nullptr;
    base.srcpick = nullptr;
    base.up_rec = nullptr;
    base.up_pick = nullptr;
    base.up_first = 0;
    base.up_count = 0;
    base.lt_cum = g->lt_cum;
    // per-vertex member counts, kept while they describe exactly samples
    // [0, T): invalid until this call succeeds
    const bool counting = s->vcount_ok && s->vcount_T == s->T;
    s->vcount_ok = false;
    base.vcount = nullptr;
    if (counting) {
        if (!s->vcount) {
            SK_CUDA(dev_alloc_t(&s->vcount, (size_t)g->n, st));
            SK_CUDA(cudaMemsetAsync(s->vcount, 0, (size_t)g->n * sizeof(uint32_t), st));
        }
        base.vcount = s->vcount;
    }
    base.chain = nullptr;
    if (s->bucket && !s->ris && !g->lt) {
        rc = graph_ensure_chain(g, st, err);
        if (rc != SKIS_OK) return rc;
        base.chain = g->chain;
    }
    int lt_blocks = 0;
    if (g->lt) {
        rc = occupancy_grid((const void*)k_lt_walk, kLtBlock, s->thread_blocks, (count + kLtBlock - 1) / kLtBlock,
                            err, &lt_blocks);
        if (rc != SKIS_OK) return rc;
    }

    DevStatus hst;
    SampleCounters hc;
    int pass = 0;
    s->last_thread_ms = s->last_warp_ms = s->last_cta_ms = s->last_sample_ms = 0;
    s->last_to_warp = s->last_deferred = 0;
    s->last_passes = 0;
    SK_CUDA(cudaMemsetAsync(s->status, 0, sizeof(DevStatus), st));
    SK_CUDA(cudaMemsetAsync(&s->status->first_bad, 0xFF, sizeof(unsigned long long), st));
    for (;;) {
        base.ovf_ids = s->ovf_ids[pass & 1];
        // reset every per-pass cursor and count; the arena cursor persists
        SK_CUDA(cudaMemsetAsync(&s->ctr->novf, 0, sizeof(SampleCounters) - sizeof(unsigned long long), st));
        SampleArgs at = base, aw = base, ac = base;
        // thread tier: the input ids; hands on to the warp tier
        at.work = &s->ctr->work_thread;
        at.out_ids = s->to_warp_ids;
        at.out_count = &s->ctr->n_to_warp;
        // warp tier: the thread tier's hand-ons (or the input ids without it)
        if (thread_tier) {
            aw.ids = s->to_warp_ids;
            aw.count_dev = &s->ctr->n_to_warp;
        }
        aw.work = &s->ctr->work_warp;
        aw.out_ids = s->to_cta_ids;
        aw.out_count = &s->ctr->n_to_cta;
        // CTA tier: the warp tier's hand-ons
        ac.ids = s->to_cta_ids;
        ac.count_dev = &s->ctr->n_to_cta;
        ac.work = &s->ctr->work_cta;
        ac.out_ids = s->big_ids;  // samples that outgrow a slot's queue
        ac.out_count = &s->ctr->n_big;

        SK_CUDA(cudaEventRecord(s->ev[0], st));
        if (g->lt) {  // LT: lane-per-sample walks, lane-per-walk medium walks, long walks on the slots
            aw.ids = s->to_warp_ids;
            aw.count_dev = &s->ctr->n_to_warp;
            k_lt_walk<<<lt_blocks, kLtBlock, 0, st>>>(at); note_launch();
            SK_CUDA(cudaGetLastError());
            SK_CUDA(cudaEventRecord(s->ev[1], st));
            k_lt_mid<<<s->lt_mid_lanes / kLtMidBlock, kLtMidBlock, 0, st>>>(aw, s->lt_hash, s->lt_list, s->lt_slot);
            note_launch();
            SK_CUDA(cudaGetLastError());
            SK_CUDA(cudaEventRecord(s->ev[2], st));
            k_lt_long<<<s->cta_slots_alloc, 32, 0, st>>>(ac); note_launch();
            SK_CUDA(cudaGetLastError());
            SK_CUDA(cudaEventRecord(s->ev[3], st));
        } else {
            if (thread_tier) {
                const uint64_t in_count = base.count;
                k_sources<<<(int)std::max<uint64_t>(1, std::min<uint64_t>((in_count + 255) / 256, (uint64_t)sm_count() * 16)),
                            256, 0, st>>>(at, s->srcrec, s->srcpick); note_launch();
                at.srcrec = s->srcrec;
                at.srcpick = base.chain ? s->srcpick : nullptr;
                if (!base.ids) {  // contiguous ids: later tiers find their samples' records by id
                    aw.up_rec = ac.up_rec = s->srcrec;
                    aw.up_pick = ac.up_pick = at.srcpick;
                    aw.up_first = ac.up_first = base.first_id;
                    aw.up_count = ac.up_count = base.count;
                }
                k_iis_lane<<<lane_blocks, kLaneBlock, 0, st>>>(at); note_launch();
                SK_CUDA(cudaGetLastError());
            }
            SK_CUDA(cudaEventRecord(s->ev[1], st));
            k_iis_warp<<<warp_blocks, kWarpThreads, 0, st>>>(aw); note_launch();
            SK_CUDA(cudaGetLastError());
            SK_CUDA(cudaEventRecord(s->ev[2], st));
            if (s->cta_threads == 512) k_iis_cta<512><<<s->cta_slots_alloc, 512, 0, st>>>(ac);
            else k_iis_cta<256><<<s->cta_slots_alloc, 256, 0, st>>>(ac);
            note_launch();
            SK_CUDA(cudaGetLastError());
            SK_CUDA(cudaEventRecord(s->ev[3], st));
        }
        SK_CUDA(cudaMemcpyAsync(&hc, s->ctr, sizeof(SampleCounters), cudaMemcpyDeviceToHost, st));
        SK_CUDA(cudaMemcpyAsync(&hst, s->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
        SK_CUDA(cudaStreamSynchronize(st));
        float ms_t = 0, ms_w = 0, ms_c = 0, ms_b = 0;
        cudaEventElapsedTime(&ms_t, s->ev[0], s->ev[1]);
        cudaEventElapsedTime(&ms_w, s->ev[1], s->ev[2]);
        cudaEventElapsedTime(&ms_c, s->ev[2], s->ev[3]);
        if (hc.n_big > 0) {  // samples that outgrew a slot's queue, on slots with n-entry queues
            rc = ensure_big_slots(s, st, err);
            if (rc != SKIS_OK) return rc;
            SampleArgs ab = ac;
            ab.ids = s->big_ids;
            ab.count_dev = &s->ctr->n_big;
            ab.work = &s->ctr->work_big;
            ab.queues = s->big_queues;
            ab.queue_cap = (uint32_t)g->n;
            ab.out_ids = nullptr;
            ab.out_count = nullptr;
            SK_CUDA(cudaEventRecord(s->ev[2], st));
            if (g->lt) {
                k_lt_long<<<s->big_slots, 32, 0, st>>>(ab); note_launch();
            } else {
                if (s->cta_threads == 512) k_iis_cta<512><<<s->big_slots, 512, 0, st>>>(ab);
                else k_iis_cta<256><<<s->big_slots, 256, 0, st>>>(ab);
                note_launch();
            }
            SK_CUDA(cudaGetLastError());
            SK_CUDA(cudaEventRecord(s->ev[3], st));
            SK_CUDA(cudaMemcpyAsync(&hc, s->ctr, sizeof(SampleCounters), cudaMemcpyDeviceToHost, st));
            SK_CUDA(cudaMemcpyAsync(&hst, s->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
            SK_CUDA(cudaStreamSynchronize(st));
            cudaEventElapsedTime(&ms_b, s->ev[2], s->ev[3]);
            ms_c += ms_b;
        }
        s->last_thread_ms += ms_t;
        s->last_warp_ms += ms_w;
        s->last_cta_ms += ms_c;
        s->last_sample_ms += ms_t + ms_w + ms_c;
        s->last_to_warp += (thread_tier || g->lt) ? hc.n_to_warp : count;
        s->last_deferred += hc.n_to_cta;
        s->last_passes += 1;
        if (hc.novf == 0) break;
        // some reservations did not fit: grow the arena (keeping every
        // completed sample, all of which lie below the old capacity) and
        // rerun exactly the samples that failed
        const uint64_t old_cap = s->arena_cap;
        const uint64_t new_cap = old_cap * 2 + (uint64_t)kLaneArenaChunk * lane_blocks * (kLaneBlock / 32) +
                                 (uint64_t)kLaneArenaChunk * lt_blocks * (kLtBlock / 32) +
                                 (uint64_t)kArenaChunk * warp_blocks * (kWarpThreads / 32);
        rc = [&]() -> int {
            SK_CUDA(grow_copy(&s->arena, old_cap, new_cap, st));
            return SKIS_OK;
        }();
        if (rc != SKIS_OK) {
            *err = "skis_sample: the member arena could not grow to " + std::to_string(new_cap) + " entries";
            return SKIS_ERR_ARENA_FULL;
        }
        s->arena_cap = new_cap;
        unsigned long long cur = old_cap;
        SK_CUDA(cudaMemcpyAsync(&s->ctr->arena, &cur, sizeof(cur), cudaMemcpyHostToDevice, st));
        base.arena = s->arena;
        base.arena_cap = s->arena_cap;
        base.ids = s->ovf_ids[pass & 1];
        base.first_id = 0;
        base.count = hc.novf;
        ++pass;
    }
    s->T += count;
    if (counting) {
        s->vcount_ok = true;
        s->vcount_T = s->T;
    }
    if (hst.flags & kStListFull) {
        *err = "skis_sample: internal error: a sample outgrew a queue of n entries";
        return SKIS_ERR_INTERNAL;
    }
    if (hst.flags & kStRetry) {
        *err = "skis_sample: a conditioned first step reached the retry cap (" + std::to_string(s->retry_cap) +
               " rounds) at sample id " + std::to_string(hst.first_bad) + "; failed samples are empty";
        return SKIS_ERR_RETRY_LIMIT;
    }
    return SKIS_OK;
}

// The one batch sample whose inclusive prefix of sizes first reaches need:
// pre is the exclusive scan with the total appended, so the index i with
// pre[i] < need <= pre[i + 1] is unique when pre[count] >= need.
__global__ void k_first_reach(const uint64_t* __restrict__ pre, uint64_t count, uint64_t need,
                              unsigned long long* __restrict__ out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        if (pre[i] < need && pre[i + 1] >= need) *out = i;
}

int sketch_sample_to_size(skis_sketch* s, uint64_t target, uint64_t max_count, cudaStream_t st, uint64_t* appended,
                          std::string* err) {
    *appended = 0;
    uint64_t cur = 0;  // sum of |R_j| over the samples already in the sketch
    if (s->T > 0) {
        uint64_t* pre = nullptr;
        SK_CUDA(dev_alloc_t(&pre, (size_t)s->T + 1, st));
        SK_CUDA(scan_u32_to_u64(s->h_len, pre, (int64_t)s->T, st));
        SK_CUDA(cudaMemcpyAsync(&cur, pre + s->T, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        SK_CUDA(cudaStreamSynchronize(st));
        dev_free(pre, st);
    }
    while (cur < target && *appended < max_count) {
        const uint64_t need = target - cur;
        // batch: the expected count to reach the target at the sizes seen
        // so far, plus 5 %, within [2^16, what is left of max_count]
        uint64_t batch = 1u << 16;
        if (s->T > 0 && cur > 0) {
            const double mean = (double)cur / (double)s->T;
            batch = std::max<uint64_t>(batch, (uint64_t)((double)need / mean * 1.05) + 1024);
        }
        batch = std::min<uint64_t>(batch, max_count - *appended);
        const uint64_t T0 = s->T;
        int rc = sketch_sample(s, batch, st, err);
        if (rc != SKIS_OK) return rc;
        uint64_t* pre = nullptr;
        unsigned long long* d_at = nullptr;
        SK_CUDA(dev_alloc_t(&pre, (size_t)batch + 1, st));
        SK_CUDA(dev_alloc_t(&d_at, 1, st));
        SK_CUDA(scan_u32_to_u64(s->h_len + T0, pre, (int64_t)batch, st));
        SK_CUDA(cudaMemsetAsync(d_at, 0xFF, sizeof(unsigned long long), st));
        k_first_reach<<<(int)std::max<uint64_t>(1, std::min<uint64_t>((batch + 255) / 256, (uint64_t)sm_count() * 8)), 256, 0,
                        st>>>(pre, batch, need, d_at); note_launch();
        SK_CUDA(cudaGetLastError());
        uint64_t tot = 0;
        unsigned long long at = 0;
        SK_CUDA(cudaMemcpyAsync(&tot, pre + batch, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        SK_CUDA(cudaMemcpyAsync(&at, d_at, sizeof(at), cudaMemcpyDeviceToHost, st));
        SK_CUDA(cudaStreamSynchronize(st));
        if (tot >= need) {
            uint64_t upto = 0;  // sizes of batch samples 0 .. at
            SK_CUDA(cudaMemcpyAsync(&upto, pre + at + 1, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
            SK_CUDA(cudaStreamSynchronize(st));
            s->T = T0 + at + 1;  // later samples of the batch are dropped
            s->vcount_ok = false;  // the counts include them
            *appended += at + 1;
            cur += upto;
        } else {
            *appended += batch;
            cur += tot;
        }
        dev_free(pre, st);
        dev_free(d_at, st);
    }
    return SKIS_OK;
}

// Autotuner of the tier split: pilot sampling of ids [0, pilot) on a scratch
// sketch under each candidate (thread-tier degree limit, step budget), best of
// two runs each, fastest kept. Samples do not depend on the split, so only
// time is compared.
int sketch_autotune(skis_sketch* s, uint64_t pilot, cudaStream_t st, double* cand_ms, int cand_cap, int* ncand,
                    std::string* err) {
    static const uint32_t kDeg[] = {0, 64, 128, 192, 256, 512};
    static const uint32_t kSteps[] = {128, 256, 1024};
    static const uint32_t kCoins[] = {4096, 16384, 65536, 262144};
    skis_sketch tmp;
    tmp.g = s->g;
    tmp.seed = s->seed;
    tmp.retry_cap = s->retry_cap;
    tmp.ris = s->ris;
    tmp.vcount_ok = false;
    tmp.bucket = s->bucket;
    tmp.thread_max_retries = s->thread_max_retries;
    tmp.warp_max_coins = s->warp_max_coins;
    tmp.cta_hub_quads = s->cta_hub_quads;
    tmp.cta_queue_cap = s->cta_queue_cap;
    tmp.cta_threads = s->cta_threads;
    tmp.cta_slots = s->cta_slots;
    tmp.warp_blocks = s->warp_blocks;
    tmp.thread_blocks = s->thread_blocks;
    tmp.stream = st;
    double best = 1e300;
    uint32_t best_deg = s->thread_max_deg, best_steps = s->thread_max_steps, best_coins = s->warp_max_coins;
    int k = 0, rc = SKIS_OK;
    // the pilot time of the current candidate (best of two runs)
    auto time_pilot = [&]() -> double {
        double ms = 1e300;
        for (int rep = 0; rep < 2 && rc == SKIS_OK; ++rep) {
            tmp.T = 0;
            if (tmp.ctr) {
                const cudaError_t e = cudaMemsetAsync(&tmp.ctr->arena, 0, sizeof(unsigned long long), st);
                if (e != cudaSuccess) { *err = cudaGetErrorString(e); rc = SKIS_ERR_CUDA; }
            }
            if (rc == SKIS_OK) rc = sketch_sample(&tmp, pilot, st, err);
            if (rc == SKIS_OK) ms = std::min(ms, tmp.last_sample_ms);
        }
        if (rc == SKIS_OK && cand_ms && k < cand_cap) cand_ms[k] = ms;
        ++k;
        return ms;
    };
    // first the lane/warp split, then the warp/CTA split under the chosen one
    for (uint32_t d : kDeg) {
        for (uint32_t m : kSteps) {
            if (d == 0 && m != kSteps[0]) continue;  // no thread tier: the budget is moot
            tmp.thread_max_deg = d;
            tmp.thread_max_steps = m;
            const double ms = time_pilot();
            if (rc != SKIS_OK) break;
            if (ms < best) {
                best = ms;
                best_deg = d;
                best_steps = m;
            }
        }
        if (rc != SKIS_OK) break;
    }
    tmp.thread_max_deg = best_deg;
    tmp.thread_max_steps = best_steps;
    for (uint32_t c : kCoins) {
        if (rc != SKIS_OK) break;
        tmp.warp_max_coins = c;
        const double ms = time_pilot();
        if (rc == SKIS_OK && ms < best) {
            best = ms;
            best_coins = c;
        }
    }
    sketch_release(&tmp);
    if (ncand) *ncand = k;
    if (rc != SKIS_OK) return rc;
    s->thread_max_deg = best_deg;
    s->thread_max_steps = best_steps;
    s->warp_max_coins = best_coins;
    return SKIS_OK;
}

}  // namespace skis
