// radix.cuh -- stable on-chip radix ranking and the cluster radix sort.
//
// Used for every "Sort_Seq" of the paper (Fig. 1 step 3 and Fig. 2 step 12):
// the sort of a block of keys for regular sampling, the sort of every bucket
// after routing, and the tile step of the sample sort.  The paper's local sort
// is stable (Sec. 5.1.1); so is this one: an LSD radix sort whose per-digit
// ranking keeps input order among equal digits.
#pragma once

#include "common.cuh"

namespace bsps {

// Items live in registers in a "warp-striped" layout: thread (warp w, lane l)
// holds item i at slot w*32*ITEMS + i*32 + l.  Visiting (w, i, l) in
// lexicographic order visits slots in increasing order, which is what makes
// the warp-synchronous ranking below stable.
template <int THREADS, int ITEMS>
__device__ __forceinline__ int striped_slot(int i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    return warp * 32 * ITEMS + i * 32 + lane;
}

// Lanes of the warp holding the same digit, from one ballot per digit bit
// (cheaper than a match instruction when most digits differ).
template <int BITS>
__device__ __forceinline__ uint32_t warp_peers(uint32_t d) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

// Stable ranking of ITEMS digits per thread (RADIX_BITS-bit digits).
// After rank(): rank[i] = number of items with the same digit and a smaller
// slot; digit_tot[d] = number of items with digit d in this CTA.
template <int THREADS, int ITEMS, int RADIX_BITS>
struct BlockRank {
    static constexpr int WARPS = THREADS / 32;
    static constexpr int RADIX = 1 << RADIX_BITS;
    static_assert(THREADS * ITEMS < 65536, "16-bit warp offsets");
    struct Smem {
        uint16_t warp_hist[WARPS][RADIX];
        uint32_t digit_tot[RADIX];
    };

    __device__ static void rank(Smem &sm, const uint32_t (&digit)[ITEMS], uint32_t (&rk)[ITEMS]) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int d = lane; d < RADIX; d += 32) sm.warp_hist[warp][d] = 0;
        __syncwarp();
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t d = digit[i];
            const uint32_t peers = warp_peers<RADIX_BITS>(d);
            const uint32_t before = __popc(peers & lt);
            const uint32_t cnt = sm.warp_hist[warp][d];
            __syncwarp();
            if (before == 0) sm.warp_hist[warp][d] = (uint16_t)(cnt + __popc(peers));
            __syncwarp();
            rk[i] = cnt + before;
        }
        __syncthreads();
        for (int d = threadIdx.x; d < RADIX; d += THREADS) {
            uint32_t run = 0;
#pragma unroll 4
            for (int w = 0; w < WARPS; ++w) {
                const uint32_t c = sm.warp_hist[w][d];
                sm.warp_hist[w][d] = (uint16_t)run;
                run += c;
            }
            sm.digit_tot[d] = run;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) rk[i] += sm.warp_hist[warp][digit[i]];
    }

    // As rank(), for the first `ia` items of every thread only (ia is the same
    // for the whole CTA; the slot of item i is warp*32*ia + i*32 + lane).
    __device__ static void rank_n(Smem &sm, const uint32_t (&digit)[ITEMS], uint32_t (&rk)[ITEMS], int ia) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int d = lane; d < RADIX; d += 32) sm.warp_hist[warp][d] = 0;
        __syncwarp();
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (i < ia) {
                const uint32_t d = digit[i];
                const uint32_t peers = warp_peers<RADIX_BITS>(d);
                const uint32_t before = __popc(peers & lt);
                const uint32_t cnt = sm.warp_hist[warp][d];
                __syncwarp();
                if (before == 0) sm.warp_hist[warp][d] = (uint16_t)(cnt + __popc(peers));
                __syncwarp();
                rk[i] = cnt + before;
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < RADIX; d += THREADS) {
            uint32_t run = 0;
#pragma unroll 8
            for (int w = 0; w < WARPS; ++w) {
                const uint32_t c = sm.warp_hist[w][d];
                sm.warp_hist[w][d] = (uint16_t)run;
                run += c;
            }
            sm.digit_tot[d] = run;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (i < ia) rk[i] += sm.warp_hist[warp][digit[i]];
    }
};

template <int THREADS>
__device__ __forceinline__ int striped_slot_n(int i, int ia) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    return warp * 32 * ia + i * 32 + lane;
}

// Exclusive scan of RADIX (<= THREADS) values held in `v[]` (in place).
template <int THREADS, int RADIX>
__device__ __forceinline__ void digit_excl_scan(uint32_t *v, uint32_t *tmp) {
    static_assert(RADIX <= THREADS, "one digit per thread");
    constexpr int W = RADIX / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t x = tid < RADIX ? v[tid] : 0, tot;
    const uint32_t e = warp_excl_scan(x, &tot);
    if (tid < RADIX && lane == 31) tmp[warp] = tot;
    __syncthreads();
    if (warp == 0) {
        uint32_t y = lane < W ? tmp[lane] : 0, t;
        const uint32_t ye = warp_excl_scan(y, &t);
        if (lane < W) tmp[lane] = ye;
    }
    __syncthreads();
    if (tid < RADIX) v[tid] = e + tmp[warp];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Cluster radix sort: CL CTAs of one thread-block cluster sort up to
// CL*THREADS*ITEMS keys (with an optional 32-bit companion, e.g. the input
// slot) held in their shared memory.  CTA c holds positions [c*CAP, (c+1)*CAP)
// before and after the sort.  Each pass ranks locally, exchanges the per-digit
// totals through distributed shared memory, and scatters every key into the
// shared memory of the CTA that owns its new position.
// ---------------------------------------------------------------------------
template <typename K, bool HAS_V, int THREADS, int ITEMS, int CL>
struct ClusterSort {
    static constexpr int CAP = THREADS * ITEMS;
    static constexpr int RADIX_BITS = 8, RADIX = 256;
    using Rank = BlockRank<THREADS, ITEMS, RADIX_BITS>;
    struct Smem {
        typename Rank::Smem rank;
        uint32_t base[RADIX];
        uint32_t prefix[RADIX];   // keys of this digit held by lower-ranked CTAs
        uint32_t tmp[40];
        K red_min, red_max;
    };

    // Sort keys[0..CAP) (and vals) of every CTA of the cluster by their low
    // `bits` bits.  Unused slots must hold all-ones keys and sit after the
    // used ones in slot order.
    __device__ static void sort(Smem &sm, K *keys, uint32_t *vals, int bits) {
        auto cluster = cg::this_cluster();
        const unsigned my_rank = CL > 1 ? cluster.block_rank() : 0;
        for (int shift = 0; shift < bits; shift += RADIX_BITS) {
            K k[ITEMS];
            uint32_t v[ITEMS], d[ITEMS], rk[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const int s = striped_slot<THREADS, ITEMS>(i);
                k[i] = keys[s];
                if constexpr (HAS_V) v[i] = vals[s];
                d[i] = (uint32_t)(k[i] >> shift) & (RADIX - 1);
            }
            Rank::rank(sm.rank, d, rk);
            if constexpr (CL > 1) {
                cluster.sync();  // every CTA's totals are final and its items are in registers
                for (int dd = threadIdx.x; dd < RADIX; dd += THREADS) {
                    uint32_t before = 0, total = 0;
#pragma unroll
                    for (int r = 0; r < CL; ++r) {
                        const uint32_t t = *cluster.map_shared_rank(&sm.rank.digit_tot[dd], r);
                        before += (unsigned)r < my_rank ? t : 0;
                        total += t;
                    }
                    sm.base[dd] = total;
                    sm.prefix[dd] = before;
                }
                __syncthreads();
            } else {
                for (int dd = threadIdx.x; dd < RADIX; dd += THREADS) sm.base[dd] = sm.rank.digit_tot[dd];
                __syncthreads();
            }
            digit_excl_scan<THREADS, RADIX>(sm.base, sm.tmp);
            if constexpr (CL > 1) {
                for (int dd = threadIdx.x; dd < RADIX; dd += THREADS) sm.base[dd] += sm.prefix[dd];
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t pos = sm.base[d[i]] + rk[i];
                if constexpr (CL > 1) {
                    const unsigned owner = pos / CAP, slot = pos % CAP;
                    K *dk = cluster.map_shared_rank(keys, owner);
                    dk[slot] = k[i];
                    if constexpr (HAS_V) {
                        uint32_t *dv = cluster.map_shared_rank(vals, owner);
                        dv[slot] = v[i];
                    }
                } else {
                    keys[pos] = k[i];
                    if constexpr (HAS_V) vals[pos] = v[i];
                }
            }
            if constexpr (CL > 1) cluster.sync();
            else __syncthreads();
        }
    }

    // Cluster-wide min and max of per-thread values (all threads call).
    __device__ static void minmax(Smem &sm, K lo, K hi, K &out_lo, K &out_hi) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            K a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
            lo = a < lo ? a : lo;
            hi = b > hi ? b : hi;
        }
        if (threadIdx.x == 0) { sm.red_min = all_ones<K>(); sm.red_max = 0; }
        __syncthreads();
        if (lane == 0) {
            if constexpr (sizeof(K) == 8) {
                atomicMin((unsigned long long *)&sm.red_min, (unsigned long long)lo);
                atomicMax((unsigned long long *)&sm.red_max, (unsigned long long)hi);
            } else {
                atomicMin((unsigned *)&sm.red_min, (unsigned)lo);
                atomicMax((unsigned *)&sm.red_max, (unsigned)hi);
            }
        }
        if constexpr (CL > 1) {
            auto cluster = cg::this_cluster();
            cluster.sync();
            K a = all_ones<K>(), b = 0;
#pragma unroll
            for (int r = 0; r < CL; ++r) {
                const K x = *cluster.map_shared_rank(&sm.red_min, r);
                const K y = *cluster.map_shared_rank(&sm.red_max, r);
                a = x < a ? x : a;
                b = y > b ? y : b;
            }
            out_lo = a;
            out_hi = b;
            cluster.sync();  // nobody rewrites red_min/red_max while others read
        } else {
            __syncthreads();
            out_lo = sm.red_min;
            out_hi = sm.red_max;
            __syncthreads();
        }
    }
};

} // namespace bsps
