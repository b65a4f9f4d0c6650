// radix.cuh -- stable on-chip radix ranking.
//
// The building block of the stable sorts (the paper's local sort is stable,
// Sec. 5.1.1): the stable cluster sort of segsort.cuh (blocks for regular
// sampling, buckets with payloads), the stable partition of the routing with
// payloads, and the scatter of the LSD sample sort.  Ranks keep input order
// among equal digits.
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

} // namespace bsps
