// common.cuh -- types and device helpers shared by the sample-sort kernels.
#pragma once

#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bspsort.h"

namespace bsps {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------
// Key order.  phi maps a key bit pattern to an unsigned integer whose order is
// the key order: identity (uint32), sign flip (int32), IEEE 754 totalOrder
// (float32/float64: negative patterns are complemented, positive ones get the
// sign bit set).  The paper sorts C ints (Sec. 6.1); the float order is this
// library's reading for floating keys.
// ---------------------------------------------------------------------------
template <int DT> struct KeyTraits;
template <> struct KeyTraits<BSPS_U32> {
    using T = uint32_t;
    __host__ __device__ static T phi(T u) { return u; }
    __host__ __device__ static T inv(T v) { return v; }
};
template <> struct KeyTraits<BSPS_I32> {
    using T = uint32_t;
    __host__ __device__ static T phi(T u) { return u ^ 0x80000000u; }
    __host__ __device__ static T inv(T v) { return v ^ 0x80000000u; }
};
template <> struct KeyTraits<BSPS_F32> {
    using T = uint32_t;
    __host__ __device__ static T phi(T u) { return (u & 0x80000000u) ? ~u : (u | 0x80000000u); }
    __host__ __device__ static T inv(T v) { return (v & 0x80000000u) ? (v & 0x7fffffffu) : ~v; }
};
template <> struct KeyTraits<BSPS_F64> {
    using T = uint64_t;
    __host__ __device__ static T phi(T u) {
        return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
    }
    __host__ __device__ static T inv(T v) {
        return (v >> 63) ? (v & 0x7fffffffffffffffull) : ~v;
    }
};

template <typename T> __host__ __device__ constexpr T all_ones() { return ~T(0); }

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// Device status block at the start of every workspace.
// ---------------------------------------------------------------------------
struct DevStatus {
    int32_t error;        // first device-side error code (0 = none)
    int32_t overflow;     // a bucket region overflowed
    int32_t timeouts;     // bounded waits that expired
    int32_t slow_buckets; // sub-buckets handled by the out-of-core path
    unsigned long long max_bucket;
    unsigned long long max_vbucket;
    unsigned long long mispredicted;
    unsigned long long correction_steps;
    uint32_t tile_counter;      // dynamic tile ticket of the routing kernel
    uint32_t run_too_big;       // a block of the regular sample did not fit on chip
    int32_t retry_count;        // sub-buckets for the stable cluster sort (keys only: given back)
    uint32_t pad_[5];
    unsigned long long ext_min_inv;  // ~(smallest phi of bucket 0); 0 = none seen
    unsigned long long ext_max;      // largest phi of the last bucket
};

__device__ __forceinline__ void set_error(DevStatus *st, int code) {
    atomicCAS(&st->error, 0, code);
}

// Upper bound on polls of a flag written by another CTA.  A poll costs a few
// hundred cycles, so the bound is on the order of a second; when it expires
// the kernel records BSPS_ERR_DEVICE_TIMEOUT and carries on without waiting.
constexpr uint32_t kSpinLimit = 1u << 22;

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
// generator of the random sample (Fig. 3 step 4).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
        uint64_t lo0 = m0 * c[0], hi0 = __umul64hi(m0, c[0]);
        uint64_t lo1 = m1 * c[2], hi1 = __umul64hi(m1, c[2]);
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T> __device__ __forceinline__ int bit_length(T v) {
    if constexpr (sizeof(T) == 8) return v ? 64 - __clzll((long long)v) : 0;
    else return v ? 32 - __clz((int)v) : 0;
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t *p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t *>(p) = v;
}

// Warp-wide exclusive prefix sum.
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t *total) {
    const int lane = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Block-wide exclusive scan of `count` values in shared memory (in place).
// Returns the total.  `tmp` needs 32 words.  All threads must call it.
template <int THREADS>
__device__ uint32_t block_excl_scan_smem(uint32_t *data, int count, uint32_t *tmp) {
    constexpr int WARPS = THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (count + THREADS - 1) / THREADS;
    const int lo = tid * per, hi = min(count, lo + per);
    uint32_t local = 0;
    for (int i = lo; i < hi; ++i) local += data[i];
    uint32_t wtot;
    uint32_t wex = warp_excl_scan(local, &wtot);
    if (lane == 31) tmp[warp] = wtot;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < WARPS ? tmp[lane] : 0, t;
        uint32_t e = warp_excl_scan(v, &t);
        if (lane < WARPS) tmp[lane] = e;
        if (lane == 0) tmp[WARPS] = t;
    }
    __syncthreads();
    uint32_t run = tmp[warp] + wex;
    for (int i = lo; i < hi; ++i) {
        uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
    uint32_t total = tmp[WARPS];
    __syncthreads();
    return total;
}

} // namespace bsps
