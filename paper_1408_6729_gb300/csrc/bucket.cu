// bucket.cu -- final sort of every bucket (Fig. 2 step 12 / Fig. 3 step 14):
// the keys a bucket received, in input order, are sorted stably and written
// to the bucket's place in the output.  Each sub-bucket is sorted on chip by
// one thread-block cluster, in up to three tiers:
//   1. keys only: the throughput sort of segsort_keys.cuh (unstable ranks,
//      which equal keys cannot reveal) -- for 8-byte keys in two capacities,
//      two CTAs per SM for the sub-buckets that fit, then one CTA per SM
//      holding twice the keys for the larger ones; with payloads: sub-buckets
//      of one key value are copied as they stand;
//   2. the other sub-buckets with payloads, or what tier 1 gives back: the
//      stable cluster sort of segsort.cuh over a list;
//   3. sub-buckets larger than a cluster's shared memory: an out-of-core
//      radix sort in global memory.
#include "kernels.cuh"
#include "segsort.cuh"
#include "segsort_keys.cuh"
#include "bucket_keys32.cuh"

namespace bsps {

template <typename K> struct BucketArgs {
    const K *reg_keys;        // phi of the routed keys, region v at v*cap
    const uint32_t *reg_vals;
    const uint32_t *vsize;
    const uint64_t *voff;
    int64_t cap;
    K *out_keys;
    uint32_t *out_vals;
    uint32_t *slow_list;
    DevStatus *st;
    const K *vphi;            // sub-bucket splitters (bounds of every sub-bucket)
    int64_t P;
    uint32_t *retry_flag;     // tier 1 gave the sub-bucket back
    uint32_t *retry_list;
    const uint32_t *only;     // tier 2 over a list (nullable: every sub-bucket)
    const int32_t *only_count;
    int64_t defer_above;      // tier 1: sub-buckets above this many keys are left to the larger tier 1
    int64_t take_above;       // larger tier 1: only sub-buckets above this many keys
    int one_value_done;       // sub-buckets of one key value are already in the output
};

template <int DT, bool PAIRS, int CL, int ITEMS>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(1024, 1)
bucket_sort_kernel(const BucketArgs<typename KeyTraits<DT>::T> a) {
    using K = typename KeyTraits<DT>::T;
    using SS = SegSort<K, PAIRS, CL, ITEMS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename SS::Smem &sm = *reinterpret_cast<typename SS::Smem *>(smem_raw);
    K *buf = reinterpret_cast<K *>(smem_raw + ((sizeof(typename SS::Smem) + 15) & ~size_t(15)));
    uint32_t *slots = reinterpret_cast<uint32_t *>(buf + SS::CAP);

    // every sub-bucket (one per cluster), or the listed ones (clusters loop)
    const int64_t nitems = a.only ? *a.only_count : a.P;
    const int64_t clusters = gridDim.x / CL;
    for (int64_t it = blockIdx.x / CL; it < nitems; it += (a.only ? clusters : nitems)) {
        const int64_t v = a.only ? a.only[it] : it;
        const int64_t cnt = imin64(a.vsize[v], a.cap);
        if (cnt == 0) continue;
        const uint64_t off = a.voff[v];
        const K *src = a.reg_keys + v * a.cap;
        const uint32_t *vsrc = a.reg_vals + v * a.cap;
        K *out_k = a.out_keys + off;
        uint32_t *out_v = a.out_vals + off;
        auto emit = [&](uint32_t pos, K key, uint32_t slot) {
            out_k[pos] = KeyTraits<DT>::inv(key);
            if constexpr (PAIRS) out_v[pos] = vsrc[slot];
        };
        const bool done = SS::run(sm, buf, slots, cnt, [&](int64_t e) { return src[e]; }, emit);
        if (!done && blockIdx.x % CL == 0 && threadIdx.x == 0) {
            const int slot = atomicAdd(&a.st->slow_buckets, 1);
            a.slow_list[slot] = (uint32_t)v;
        }
        // the next sub-bucket reuses every CTA's shared memory
        if (a.only) cg::this_cluster().sync();
        else __syncthreads();
    }
}

// With payloads, before the cluster sort: a sub-bucket between two splitters
// of equal phi holds one key value, and routing kept its keys in input order,
// which is their sorted order under the position tie-break (Sec. 5.1.1); it is
// copied out as it stands.  Every other non-empty sub-bucket goes on the list
// the cluster sort then works through.
constexpr int kCopyThreads = 512;
template <int DT, bool PAIRS>
__global__ void __launch_bounds__(kCopyThreads) bucket_copy_kernel(const BucketArgs<typename KeyTraits<DT>::T> a,
                                                                  uint32_t *list, int32_t *list_count) {
    using K = typename KeyTraits<DT>::T;
    for (int64_t v = blockIdx.x; v < a.P; v += gridDim.x) {
        const int64_t cnt = imin64(a.vsize[v], a.cap);
        if (cnt == 0) continue;
        if (v > 0 && v < a.P - 1 && a.vphi[v - 1] == a.vphi[v]) {
            if (a.one_value_done) continue;  // the segment copy wrote it
            const K x = KeyTraits<DT>::inv(a.vphi[v]);
            K *out_k = a.out_keys + a.voff[v];
            uint32_t *out_v = a.out_vals + a.voff[v];
            const uint32_t *vsrc = a.reg_vals + v * a.cap;
#pragma unroll 8
            for (int64_t e = threadIdx.x; e < cnt; e += kCopyThreads) {
                out_k[e] = x;
                if constexpr (PAIRS) out_v[e] = vsrc[e];
            }
        } else if (threadIdx.x == 0) {
            list[atomicAdd(list_count, 1)] = (uint32_t)v;
        }
    }
}

// Tier 1 (keys only): one cluster per sub-bucket; its bounds are the two
// splitters around it (the smallest and largest key for the end buckets).
template <int DT, int CL, int ITEMS>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(512, ITEMS > kKeysItems64 ? 1 : 2)
bucket_keys_kernel(const BucketArgs<typename KeyTraits<DT>::T> a) {
    using K = typename KeyTraits<DT>::T;
    using SS = SegSortKeys<K, CL, ITEMS, false>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t v = blockIdx.x / CL;
    const int64_t cnt = imin64(a.vsize[v], a.cap);
    if (cnt == 0 || cnt > a.defer_above || cnt <= a.take_above) return;
    const K lo = v > 0 ? a.vphi[v - 1] : (K)~a.st->ext_min_inv;
    const K hi = v < a.P - 1 ? a.vphi[v] : (K)a.st->ext_max;
    K *out_k = a.out_keys + a.voff[v];
    if (lo == hi) {  // one key value: nothing to read
        const K x = KeyTraits<DT>::inv(lo);
        const int64_t share = (cnt + CL - 1) / CL, e0 = (int64_t)(blockIdx.x % CL) * share;
        const int64_t e1 = imin64(cnt, e0 + share);
#pragma unroll 4
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) out_k[e] = x;
        return;
    }
    auto emit = [&](uint32_t pos, K key) { out_k[pos] = KeyTraits<DT>::inv(key); };
    if (!SS::run(smem_raw, a.reg_keys + v * a.cap, cnt, lo, hi, emit) && threadIdx.x == 0) {
        if (atomicExch(&a.retry_flag[v], 1u) == 0u) {
            const int slot = atomicAdd(&a.st->retry_count, 1);
            a.retry_list[slot] = (uint32_t)v;
        }
    }
}

// Tier 1 for 32-bit keys: the same cluster per sub-bucket, with the lean
// split / exchange / count sort of bucket_keys32.cuh.
template <int DT, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(512, 2)
bucket_keys32_kernel(const BucketArgs<uint32_t> a) {
    using SS = BucketKeys32<CL>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t v = blockIdx.x / CL;
    const int64_t cnt = imin64(a.vsize[v], a.cap);
    if (cnt == 0) return;
    const uint32_t lo = v > 0 ? a.vphi[v - 1] : (uint32_t)~a.st->ext_min_inv;
    const uint32_t hi = v < a.P - 1 ? a.vphi[v] : (uint32_t)a.st->ext_max;
    uint32_t *out_k = a.out_keys + a.voff[v];
    if (lo == hi) {  // one key value: nothing to read
        const uint32_t x = KeyTraits<DT>::inv(lo);
        const int64_t share = (cnt + CL - 1) / CL, e0 = (int64_t)(blockIdx.x % CL) * share;
        const int64_t e1 = imin64(cnt, e0 + share);
#pragma unroll 4
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) out_k[e] = x;
        return;
    }
    auto emit = [&](uint32_t pos, uint32_t key) { out_k[pos] = KeyTraits<DT>::inv(key); };
    typename SS::Smem &sm = *reinterpret_cast<typename SS::Smem *>(smem_raw);
    if (threadIdx.x == 0) sm.stalled = 0;
    __syncthreads();
    bool done = SS::run(smem_raw, a.reg_keys + v * a.cap, cnt, lo, hi, emit, a.st);
    __syncthreads();
    if (sm.stalled) {  // the staged load's wait ran out: wait for the copy once more, give the sub-bucket back
        SS::wait_staged(sm, kSpinLimit);
        done = false;
    }
    if (!done && threadIdx.x == 0) {
        if (atomicExch(&a.retry_flag[v], 1u) == 0u) {
            const int slot = atomicAdd(&a.st->retry_count, 1);
            a.retry_list[slot] = (uint32_t)v;
        }
    }
}

// ---------------------------------------------------------------------------
// Out-of-core path: one CTA sorts one oversized sub-bucket by LSD passes
// between its region and its output range, chunk by chunk, stably.
// ---------------------------------------------------------------------------
template <int DT, bool PAIRS>
__global__ void __launch_bounds__(kSlowThreads) bucket_slow_kernel(BucketArgs<typename KeyTraits<DT>::T> a,
                                                                  typename KeyTraits<DT>::T *reg_keys_rw,
                                                                  uint32_t *reg_vals_rw) {
    using K = typename KeyTraits<DT>::T;
    using Rank = BlockRank<kSlowThreads, kSlowItems, 8>;
    constexpr int CH = kSlowThreads * kSlowItems;
    __shared__ typename Rank::Smem rsm;
    __shared__ uint32_t hist[256], run[256], tmp[40];
    __shared__ K red[2];
    const int nslow = a.st->slow_buckets;
    for (int idx = blockIdx.x; idx < nslow; idx += gridDim.x) {
        const int64_t v = a.slow_list[idx];
        const int64_t cnt = imin64(a.vsize[v], a.cap);
        const uint64_t off = a.voff[v];
        K *bufk[2] = {reg_keys_rw + v * a.cap, reinterpret_cast<K *>(a.out_keys) + off};
        uint32_t *bufv[2] = {PAIRS ? reg_vals_rw + v * a.cap : nullptr, PAIRS ? a.out_vals + off : nullptr};
        // key range
        K mn = all_ones<K>(), mx = 0;
        for (int64_t e = threadIdx.x; e < cnt; e += kSlowThreads) {
            const K x = bufk[0][e];
            mn = x < mn ? x : mn;
            mx = x > mx ? x : mx;
        }
        if (threadIdx.x == 0) { red[0] = all_ones<K>(); red[1] = 0; }
        __syncthreads();
        if constexpr (sizeof(K) == 8) {
            atomicMin((unsigned long long *)&red[0], (unsigned long long)mn);
            atomicMax((unsigned long long *)&red[1], (unsigned long long)mx);
        } else {
            atomicMin((unsigned *)&red[0], (unsigned)mn);
            atomicMax((unsigned *)&red[1], (unsigned)mx);
        }
        __syncthreads();
        const K base = red[0];
        const int bits = bit_length<K>(red[1] - base);
        __syncthreads();
        int cur = 0;
        for (int shift = 0; shift < bits; shift += 8) {
            const K *sk = bufk[cur];
            K *dk = bufk[1 - cur];
            for (int i = threadIdx.x; i < 256; i += kSlowThreads) { hist[i] = 0; }
            __syncthreads();
            for (int64_t e = threadIdx.x; e < cnt; e += kSlowThreads)
                atomicAdd(&hist[(uint32_t)((sk[e] - base) >> shift) & 255u], 1u);
            __syncthreads();
            digit_excl_scan<kSlowThreads, 256>(hist, tmp);
            for (int i = threadIdx.x; i < 256; i += kSlowThreads) run[i] = hist[i];
            __syncthreads();
            for (int64_t cs = 0; cs < cnt; cs += CH) {
                K kk[kSlowItems];
                uint32_t vv[kSlowItems], d[kSlowItems], rk[kSlowItems];
#pragma unroll
                for (int i = 0; i < kSlowItems; ++i) {
                    const int64_t e = cs + striped_slot<kSlowThreads, kSlowItems>(i);
                    if (e < cnt) {
                        kk[i] = sk[e];
                        if constexpr (PAIRS) vv[i] = bufv[cur][e];
                        d[i] = (uint32_t)((kk[i] - base) >> shift) & 255u;
                    } else {
                        d[i] = 255u;
                    }
                }
                Rank::rank(rsm, d, rk);
#pragma unroll
                for (int i = 0; i < kSlowItems; ++i) {
                    const int64_t e = cs + striped_slot<kSlowThreads, kSlowItems>(i);
                    if (e < cnt) {
                        const uint32_t pos = run[d[i]] + rk[i];
                        dk[pos] = kk[i];
                        if constexpr (PAIRS) bufv[1 - cur][pos] = vv[i];
                    }
                }
                __syncthreads();
                for (int i = threadIdx.x; i < 256; i += kSlowThreads) run[i] += rsm.digit_tot[i];
                __syncthreads();
            }
            cur = 1 - cur;
        }
        // final placement in the output, back to key bits
        for (int64_t e = threadIdx.x; e < cnt; e += kSlowThreads) {
            const K x = bufk[cur][e];
            if constexpr (PAIRS) {
                if (cur == 0) a.out_vals[off + e] = bufv[0][e];
            }
            a.out_keys[off + e] = KeyTraits<DT>::inv(x);
        }
        __syncthreads();
    }
}

template <int DT, bool PAIRS, int CL, int ITEMS>
static cudaError_t launch_cluster(const Ctx &c, const BucketArgs<typename KeyTraits<DT>::T> &a, bool listed) {
    using K = typename KeyTraits<DT>::T;
    using SS = SegSort<K, PAIRS, CL, ITEMS>;
    const size_t smem = SS::smem_bytes();
    auto kern = bucket_sort_kernel<DT, PAIRS, CL, ITEMS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t clusters = c.pl.P;
    if (listed) {  // as many clusters as run at once (one CTA per SM), at least 16
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        clusters = imin64(c.pl.P, imax64(16, sms / CL));
    }
    kern<<<(unsigned)(clusters * CL), 1024, smem, c.stream>>>(a);
    return cudaGetLastError();
}

template <int DT, int CL, int ITEMS>
static cudaError_t launch_keys(const Ctx &c, const BucketArgs<typename KeyTraits<DT>::T> &a) {
    using K = typename KeyTraits<DT>::T;
    if constexpr (sizeof(K) == 4) {
        using SS = BucketKeys32<CL>;
        static_assert(2 * (SS::smem_bytes() + 1024) <= 228 * 1024, "two CTAs per SM");
        const size_t smem = SS::smem_bytes();
        auto kern = bucket_keys32_kernel<DT, CL>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)(c.pl.P * CL), 512, smem, c.stream>>>(a);
        return cudaGetLastError();
    } else {
        using SS = SegSortKeys<K, CL, ITEMS, false>;
        // two CTAs per SM (228 KB of shared memory per SM, 1 KB of it reserved
        // per CTA), or one for the larger tier
        static_assert(2 * (SS::smem_bytes() + 1024) <= 228 * 1024 || ITEMS > kKeysItems64, "two CTAs per SM");
        static_assert(SS::smem_bytes() + 1024 <= 228 * 1024, "one CTA per SM");
        const size_t smem = SS::smem_bytes();
        auto kern = bucket_keys_kernel<DT, CL, ITEMS>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)(c.pl.P * CL), 512, smem, c.stream>>>(a);
        return cudaGetLastError();
    }
}

template <int DT, bool PAIRS> static cudaError_t launch_bucket_t(const Ctx &c) {
    using K = typename KeyTraits<DT>::T;
    BucketArgs<K> a;
    a.reg_keys = (const K *)c.ly.reg_keys;
    a.reg_vals = c.ly.reg_vals;
    a.vsize = c.ly.vsize;
    a.voff = c.ly.voff;
    a.cap = c.pl.cap;
    a.out_keys = (K *)c.keys_out;
    a.out_vals = c.vals_out;
    a.slow_list = c.ly.slow_list;
    a.st = c.ly.status;
    a.vphi = (const K *)c.ly.vphi;
    a.P = c.pl.P;
    a.retry_flag = c.ly.retry_flag;
    a.retry_list = c.ly.retry_list;
    a.only = nullptr;
    a.only_count = nullptr;
    a.defer_above = INT64_MAX;
    a.take_above = 0;
    a.one_value_done = c.pl.seg_route;
    constexpr int IT = PAIRS ? (sizeof(K) == 8 ? kPairItems64 : kPairItems32)
                             : (sizeof(K) == 8 ? kBucketItems64 : kBucketItems32);
    cudaError_t e = cudaSuccess;
    if constexpr (!PAIRS) {
        constexpr int KIT = sizeof(K) == 8 ? kKeysItems64 : kKeysItems32;
        if constexpr (sizeof(K) == 8) {
            // sub-buckets beyond the two-per-SM clusters: clusters of 8 CTAs
            // holding twice the keys each, before anything is given back
            a.defer_above = (int64_t)c.pl.bucket_cl * 512 * KIT;
            if (a.defer_above < (int64_t)8 * 512 * kKeysItems64Large && c.pl.cap > a.defer_above) {
                BucketArgs<K> big = a;
                big.defer_above = INT64_MAX;
                big.take_above = a.defer_above;
                e = launch_keys<DT, 8, kKeysItems64Large>(c, big);
                if (e != cudaSuccess) return e;
            } else {
                a.defer_above = INT64_MAX;
            }
        }
        switch (c.pl.bucket_cl) {
        case 1: e = launch_keys<DT, 1, KIT>(c, a); break;
        case 2: e = launch_keys<DT, 2, KIT>(c, a); break;
        case 4: e = launch_keys<DT, 4, KIT>(c, a); break;
        case 8: e = launch_keys<DT, 8, KIT>(c, a); break;
        default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        // what tier 1 gave back: the stable cluster sort over the list
        a.only = c.ly.retry_list;
        a.only_count = &c.ly.status->retry_count;
        e = launch_cluster<DT, false, 8, IT>(c, a, true);
    } else {
        // one-value sub-buckets are copied; the cluster sort takes the list of the others
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        bucket_copy_kernel<DT, PAIRS><<<(unsigned)imin64(c.pl.P, 4 * (int64_t)sms), kCopyThreads, 0, c.stream>>>(
            a, c.ly.retry_list, &c.ly.status->retry_count);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        a.only = c.ly.retry_list;
        a.only_count = &c.ly.status->retry_count;
        switch (c.pl.bucket_cl) {
        case 1: e = launch_cluster<DT, PAIRS, 1, IT>(c, a, true); break;
        case 2: e = launch_cluster<DT, PAIRS, 2, IT>(c, a, true); break;
        case 4: e = launch_cluster<DT, PAIRS, 4, IT>(c, a, true); break;
        case 8: e = launch_cluster<DT, PAIRS, 8, IT>(c, a, true); break;
        default: return cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return e;
    bucket_slow_kernel<DT, PAIRS><<<64, kSlowThreads, 0, c.stream>>>(a, (K *)c.ly.reg_keys, c.ly.reg_vals);
    return cudaGetLastError();
}

cudaError_t launch_bucket_sort(const Ctx &c) {
    const bool pr = c.pl.pairs != 0;
    switch (c.pl.dtype) {
    case BSPS_U32: return pr ? launch_bucket_t<BSPS_U32, true>(c) : launch_bucket_t<BSPS_U32, false>(c);
    case BSPS_I32: return pr ? launch_bucket_t<BSPS_I32, true>(c) : launch_bucket_t<BSPS_I32, false>(c);
    case BSPS_F32: return pr ? launch_bucket_t<BSPS_F32, true>(c) : launch_bucket_t<BSPS_F32, false>(c);
    default: return pr ? launch_bucket_t<BSPS_F64, true>(c) : launch_bucket_t<BSPS_F64, false>(c);
    }
}

} // namespace bsps
