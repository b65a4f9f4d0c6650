// sample.cu -- oversampling, sample sort, splitter selection (Fig. 1 steps
// 3-7, Fig. 3 steps 3-9) and the optional diagnostics.
#include "classify.cuh"
#include "mlp.cuh"
#include "segsort.cuh"
#include "segsort_keys.cuh"
#include "bucket_keys32.cuh"

namespace bsps {

// ---------------------------------------------------------------------------
// Random oversampling (Fig. 3 step 4): s*p-1 positions drawn i.i.d. from the
// Philox4x64-10 stream; the record of draw j is (phi(key[g_j]), g_j).
// ---------------------------------------------------------------------------
template <int DT>
__global__ void sample_random_kernel(const typename KeyTraits<DT>::T *__restrict__ keys, int64_t n,
                                     int64_t S, uint64_t seed, typename KeyTraits<DT>::T *sphi,
                                     uint32_t *stag) {
    const int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j0 = blk * 4;
    if (j0 >= S) return;
    uint64_t c[4] = {(uint64_t)blk, 0, 0, 0};
    philox4x64_10(c, seed, 0);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int64_t j = j0 + w;
        if (j < S) {
            const uint64_t g = __umul64hi(c[w], (uint64_t)n);
            sphi[j] = KeyTraits<DT>::phi(keys[g]);
            stag[j] = (uint32_t)g;
        }
    }
}

// ---------------------------------------------------------------------------
// Regular oversampling (Fig. 1 steps 3-4): one cluster of CL CTAs sorts the
// block of virtual processor k stably and emits the records at sorted
// positions j*x - 1, j = 1..s.  Positions at or past the block's key count are
// pads (Lemma 5.1's padding), which follow every key in tag order.  For the
// merge final step (Fig. 1 step 12) the sorted block itself is written too
// (`runs`, with its payloads), at the block's place.
// ---------------------------------------------------------------------------
template <int DT, int CL, int ITEMS>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kSortThreads, 1)
run_sample_kernel(const typename KeyTraits<DT>::T *__restrict__ keys, int64_t n, int64_t m,
                  int64_t M, int64_t s, int64_t x, typename KeyTraits<DT>::T *sphi, uint32_t *stag,
                  uint32_t *too_big, const uint32_t *only, typename KeyTraits<DT>::T *runs,
                  const uint32_t *__restrict__ vals, uint32_t *runs_val) {
    using K = typename KeyTraits<DT>::T;
    using SS = SegSort<K, true, CL, ITEMS>;
    if (only && only[blockIdx.x / CL] == 0) return;  // only the blocks the keys-only sort gave back
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename SS::Smem &sm = *reinterpret_cast<typename SS::Smem *>(smem_raw);
    K *buf = reinterpret_cast<K *>(smem_raw + ((sizeof(typename SS::Smem) + 15) & ~size_t(15)));
    uint32_t *slots = reinterpret_cast<uint32_t *>(buf + SS::CAP);

    const int64_t k = blockIdx.x / CL;
    const int64_t lo = k * m;
    const int64_t len = lo < n ? imin64(m, n - lo) : 0;
    if (blockIdx.x % CL == 0) {  // pads: sorted positions len..M-1, in tag order
        for (int64_t j = 1 + threadIdx.x; j <= s; j += kSortThreads) {
            const int64_t pos = j * x - 1;
            if (pos >= len) {
                sphi[k * s + (j - 1)] = all_ones<K>();
                stag[k * s + (j - 1)] = (uint32_t)(n + k * M + pos);
            }
        }
    }
    if (len == 0) return;
    auto load = [&](int64_t e) { return KeyTraits<DT>::phi(keys[lo + e]); };
    auto emit = [&](uint32_t pos, K key, uint32_t slot) {
        if (runs) {  // the sorted block is kept for the merge final step
            runs[lo + pos] = key;
            if (runs_val) runs_val[lo + pos] = vals[lo + slot];
        }
        if ((pos + 1) % x == 0) {
            const int64_t j = (pos + 1) / x;
            sphi[k * s + (j - 1)] = key;
            stag[k * s + (j - 1)] = (uint32_t)(lo + slot);
        }
    };
    if (!SS::run(sm, buf, slots, len, load, emit) && threadIdx.x == 0 && blockIdx.x % CL == 0)
        atomicExch(too_big, 1u);
}

// The same sample from a faster sort: for 32-bit keys, (phi << 32 | position
// in the block) is unique, so the keys-only cluster sort of segsort_keys.cuh
// orders the block exactly as the stable sort does.  A block it gives back
// is flagged and sorted by run_sample_kernel.
constexpr int kRunKeysItems = 20;  // 512 threads x 20 = 10240 keys per CTA (room for uneven owners)
template <int DT, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(512, 1)
run_sample_keys_kernel(const typename KeyTraits<DT>::T *__restrict__ keys, int64_t n, int64_t m, int64_t M,
                       int64_t s, int64_t x, typename KeyTraits<DT>::T *sphi, uint32_t *stag, uint32_t *retry,
                       typename KeyTraits<DT>::T *runs, const uint32_t *__restrict__ vals, uint32_t *runs_val) {
    using K = typename KeyTraits<DT>::T;
    static_assert(sizeof(K) == 4, "32-bit keys and 32-bit positions in one word");
    using SS = SegSortKeys<uint64_t, CL, kRunKeysItems>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t k = blockIdx.x / CL;
    const int64_t lo = k * m;
    const int64_t len = lo < n ? imin64(m, n - lo) : 0;
    if (blockIdx.x % CL == 0) {  // pads: sorted positions len..M-1, in tag order
        for (int64_t j = 1 + threadIdx.x; j <= s; j += blockDim.x) {
            const int64_t pos = j * x - 1;
            if (pos >= len) {
                sphi[k * s + (j - 1)] = all_ones<K>();
                stag[k * s + (j - 1)] = (uint32_t)(n + k * M + pos);
            }
        }
    }
    if (len == 0) return;
    {
        // 64 evenly spaced keys of the block: many repeats mean many equal
        // keys, whose order by position the counting finish cannot resolve;
        // such a block goes to the stable sort at once (every CTA of the
        // cluster reads the same keys and decides alike)
        __shared__ uint32_t probe[64];
        __shared__ int repeats;
        if (threadIdx.x < 64) probe[threadIdx.x] = (uint32_t)KeyTraits<DT>::phi(keys[lo + threadIdx.x * len / 64]);
        if (threadIdx.x == 0) repeats = 0;
        __syncthreads();
        if (threadIdx.x < 64) {
            bool seen = false;
            for (int j = 0; j < (int)threadIdx.x; ++j) seen |= probe[j] == probe[threadIdx.x];
            if (seen) atomicAdd(&repeats, 1);
        }
        __syncthreads();
        if (len >= 64 && repeats > 8) {
            if (threadIdx.x == 0) retry[k] = 1u;
            return;
        }
    }
    auto loadf = [&](uint64_t (&kk)[kRunKeysItems], int64_t e0, int cnt) {
#pragma unroll
        for (int i = 0; i < kRunKeysItems; ++i) {
            const int e = SS::lidx(i);
            if (e < cnt) kk[i] = (uint64_t)KeyTraits<DT>::phi(keys[lo + e0 + e]) << 32 | (uint32_t)(e0 + e);
        }
    };
    const uint32_t xx = (uint32_t)x;
    auto emit = [&](uint32_t pos, uint64_t key) {
        if (runs) {  // the sorted block is kept for the merge final step
            runs[lo + pos] = (K)(key >> 32);
            if (runs_val) runs_val[lo + pos] = vals[lo + (uint32_t)key];
        }
        if ((pos + 1) % xx == 0) {
            const int64_t j = (pos + 1) / xx;
            sphi[k * s + (j - 1)] = (K)(key >> 32);
            stag[k * s + (j - 1)] = (uint32_t)(lo + (uint32_t)key);
        }
    };
    // a split bin of one key value (many equal keys) is ordered by position
    // only, which the counting finish cannot resolve: leave such blocks to the
    // stable sort at once
    auto one_value = [](uint64_t mn, uint64_t mx) { return (mn >> 32) == (mx >> 32); };
    if (!SS::run_load(smem_raw, len, 0ull, ~0ull, loadf, emit, one_value) && threadIdx.x == 0)
        atomicExch(&retry[k], 1u);
}

// ---------------------------------------------------------------------------
// The same sample from the counting sort, when the sorted blocks of keys
// without payloads are kept: a
// block's 32-bit keys (their phi, as they load) are sorted by the keys-only
// counting sort of bucket_keys32.cuh -- the bucket sort's own kernel -- into
// the sorted block; run_sample_tags_kernel then reads the keys at the sampled
// ranks and finds their tags (input positions).  Equal keys leave
// the counting sort in no particular order, which neither the sorted block
// (keys only) nor the tags (recovered in input order) can reveal.  A block
// the counting sort gives back, or with many repeated keys, is flagged for the
// few-values sampler and the stable block sort.
// ---------------------------------------------------------------------------
template <int DT> struct PhiOf {
    __device__ uint32_t operator()(uint32_t u) const { return (uint32_t)KeyTraits<DT>::phi(u); }
};

template <int DT, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(512, 2)
run_sample_count_kernel(const uint32_t *__restrict__ keys, int64_t n, int64_t m, int64_t M, int64_t s, int64_t x,
                        uint32_t *sphi, uint32_t *stag, uint32_t *retry, uint32_t *runs, DevStatus *st) {
    // (sphi, stag: the pads' records only; the keys' records come from run_sample_tags_kernel)
    using SS = BucketKeys32<CL>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t k = blockIdx.x / CL;
    const int64_t lo = k * m;
    const int64_t len = lo < n ? imin64(m, n - lo) : 0;
    if (blockIdx.x % CL == 0) {  // pads: sorted positions len..M-1, in tag order
        for (int64_t j = 1 + threadIdx.x; j <= s; j += blockDim.x) {
            const int64_t pos = j * x - 1;
            if (pos >= len) {
                sphi[k * s + (j - 1)] = 0xffffffffu;
                stag[k * s + (j - 1)] = (uint32_t)(n + k * M + pos);
            }
        }
    }
    if (len == 0) return;
    {
        // many repeats among 64 evenly spaced keys: the few-values sampler
        // (every CTA of the cluster reads the same keys and decides alike)
        __shared__ uint32_t probe[64];
        __shared__ int repeats;
        if (threadIdx.x < 64) probe[threadIdx.x] = keys[lo + threadIdx.x * len / 64];
        if (threadIdx.x == 0) repeats = 0;
        __syncthreads();
        if (threadIdx.x < 64) {
            bool seen = false;
            for (int j = 0; j < (int)threadIdx.x; ++j) seen |= probe[j] == probe[threadIdx.x];
            if (seen) atomicAdd(&repeats, 1);
        }
        __syncthreads();
        if (len >= 64 && repeats > 8) {
            if (threadIdx.x == 0) retry[k] = 1u;
            return;
        }
    }
    auto emit = [&](uint32_t pos, uint32_t key) { runs[lo + pos] = key; };
    typename SS::Smem &sm = *reinterpret_cast<typename SS::Smem *>(smem_raw);
    if (threadIdx.x == 0) sm.stalled = 0;
    __syncthreads();
    bool done = SS::run(smem_raw, keys + lo, len, 0u, 0xffffffffu, emit, st, PhiOf<DT>());
    __syncthreads();
    if (sm.stalled) {  // the staged load's wait ran out: wait for the copy once more, give the block back
        SS::wait_staged(sm, kSpinLimit);
        done = false;
    }
    if (!done && threadIdx.x == 0) retry[k] = 1u;
}

// Tags of the sampled keys of a block sorted by run_sample_count_kernel: the
// sampled rank r = j*x - 1 holds key v, the o-th (o = r - first rank of v) of
// the block's keys equal to v in input order (Sec. 5.1.1), so its tag is the
// o-th smallest input position holding v.  One pass over the block's input
// serves every sampled key: a key that occurs once in the block is found
// through a shared-memory hash of those keys; the positions of a repeated one
// are gathered into a list (a second hash gives each such key its list) and
// the o-th smallest is picked.  A block whose sampled keys overflow the
// hash, or whose repeated keys occur too often (more than kTagRunMax times
// each, or too many positions in all), goes to the stable block sort.
constexpr int kTagThreads = 1024, kTagSlotBitsMax = 14, kTagDupBits = 9, kTagDupSlots = 1 << kTagDupBits,
              kTagListMax = 4096, kTagAhead = 8, kTagRunMax = 32;
// hash slots: a power of two at least four times the sampled keys of a block
static int tag_slot_bits(const Plan &p) {
    const int64_t js = p.m / p.x;
    int b = 10;
    while (b < kTagSlotBitsMax && ((int64_t)1 << b) < 4 * js) ++b;
    return b;
}
static size_t tag_smem(int bits) {
    return sizeof(unsigned long long) * (((size_t)1 << bits) + kTagDupSlots) + sizeof(uint32_t) * (kTagDupSlots * 3 + kTagListMax);
}

template <int DT>
__global__ void __launch_bounds__(kTagThreads, 1)
run_sample_tags_kernel(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ runs, int64_t n, int64_t m,
                       int64_t s, int64_t x, int slot_bits, uint32_t *sphi, uint32_t *stag, uint32_t *retry) {
    extern __shared__ __align__(16) unsigned char tag_raw[];
    const int slots = 1 << slot_bits;
    unsigned long long *H = reinterpret_cast<unsigned long long *>(tag_raw);  // key << 32 | j, 0 = empty
    unsigned long long *D = H + slots;                                       // key << 32 | (d + 1): repeated keys
    uint32_t *dcount = reinterpret_cast<uint32_t *>(D + kTagDupSlots);       // occurrences of repeated key d
    uint32_t *dstart = dcount + kTagDupSlots;                                // its list's start
    uint32_t *dfill = dstart + kTagDupSlots;                                 // positions gathered so far
    uint32_t *list = dfill + kTagDupSlots;                                   // the positions
    __shared__ uint32_t ndist, nlist, bad;
    const int64_t k = blockIdx.x;
    if (retry[k]) return;  // the few-values sampler or the stable sort takes it
    const int64_t lo = k * m;
    const int64_t len = lo < n ? imin64(m, n - lo) : 0;
    if (len == 0) return;
    const int64_t js = len / x;  // sampled ranks j*x - 1 inside the block's keys
    if (js == 0) return;
    if (4 * js > slots) {
        if (threadIdx.x == 0) retry[k] = 1u;
        return;
    }
    const uint32_t *blk = runs + lo;
    auto hash = [](uint32_t v, int bits) { return (v * 0x9e3779b1u) >> (32 - bits); };
    for (int i = threadIdx.x; i < slots; i += kTagThreads) H[i] = 0ull;
    for (int i = threadIdx.x; i < kTagDupSlots; i += kTagThreads) {
        D[i] = 0ull;
        dfill[i] = 0;
    }
    if (threadIdx.x == 0) {
        ndist = 0;
        nlist = 0;
        bad = 0;
    }
    __syncthreads();
    // the sampled keys: once-occurring ones into H; repeated ones into D, with
    // their occurrence counts (the run of equal keys around r)
    for (int64_t j = 1 + threadIdx.x; j <= js; j += kTagThreads) {
        const int64_t r = j * x - 1;
        const uint32_t v = blk[r];
        sphi[k * s + (j - 1)] = v;
        if ((r == 0 || blk[r - 1] != v) && (r + 1 == len || blk[r + 1] != v)) {
            const unsigned long long e = (unsigned long long)v << 32 | (uint32_t)j;
            uint32_t h = hash(v, slot_bits);
            for (int probe = 0; probe < slots; ++probe, h = (h + 1) & (slots - 1))
                if (atomicCAS(&H[h], 0ull, e) == 0ull) break;
            continue;
        }
        uint32_t h = hash(v, kTagDupBits);
        for (int probe = 0; probe < kTagDupSlots; ++probe, h = (h + 1) & (kTagDupSlots - 1)) {
            const unsigned long long cur = D[h];
            if (cur != 0ull && (uint32_t)(cur >> 32) == v) break;  // another sampled rank of the same key
            if (cur == 0ull) {
                const uint32_t d = atomicAdd(&ndist, 1u);
                if (d >= kTagDupSlots / 2) {
                    bad = 1;
                    break;
                }
                const unsigned long long want = (unsigned long long)v << 32 | (d + 1);
                const unsigned long long old = atomicCAS(&D[h], 0ull, want);
                if (old == 0ull) {
                    int64_t a = 0, b = r;  // the run of v: [a, c)
                    while (a < b) {
                        const int64_t mid = (a + b) >> 1;
                        if (blk[mid] < v) a = mid + 1;
                        else b = mid;
                    }
                    int64_t lo2 = r, c = len;
                    while (lo2 < c) {
                        const int64_t mid = (lo2 + c) >> 1;
                        if (blk[mid] <= v) lo2 = mid + 1;
                        else c = mid;
                    }
                    const uint32_t cnt = (uint32_t)(c - a);
                    dcount[d] = cnt;
                    const uint32_t at = atomicAdd(&nlist, cnt);
                    if (cnt > (uint32_t)kTagRunMax || at + cnt > (uint32_t)kTagListMax) bad = 1;
                    dstart[d] = at;
                    break;
                }
                if ((uint32_t)(old >> 32) == v) break;
                // the slot went to another key: probe on (d stays unused)
            }
        }
    }
    __syncthreads();
    if (bad) {  // uniform
        if (threadIdx.x == 0) retry[k] = 1u;
        return;
    }
    const bool any_dup = ndist > 0;
    // one pass over the block's input, kTagAhead keys per thread in flight
    for (int64_t t0 = 0; t0 < len; t0 += (int64_t)kTagThreads * kTagAhead) {
        uint32_t u[kTagAhead];
#pragma unroll
        for (int q = 0; q < kTagAhead; ++q) {
            const int64_t t = t0 + q * kTagThreads + threadIdx.x;
            u[q] = t < len ? (uint32_t)KeyTraits<DT>::phi(keys[lo + t]) : 0u;
        }
#pragma unroll
        for (int q = 0; q < kTagAhead; ++q) {
            const int64_t t = t0 + q * kTagThreads + threadIdx.x;
            if (t >= len) continue;
            uint32_t h = hash(u[q], slot_bits);
            for (int probe = 0; probe < slots; ++probe, h = (h + 1) & (slots - 1)) {
                const unsigned long long e = H[h];
                if (e == 0ull) break;
                if ((uint32_t)(e >> 32) == u[q]) {
                    stag[k * s + ((uint32_t)e - 1)] = (uint32_t)(lo + t);
                    break;
                }
            }
            if (any_dup) {
                uint32_t g = hash(u[q], kTagDupBits);
                for (int probe = 0; probe < kTagDupSlots; ++probe, g = (g + 1) & (kTagDupSlots - 1)) {
                    const unsigned long long e = D[g];
                    if (e == 0ull) break;
                    if ((uint32_t)(e >> 32) == u[q]) {
                        const uint32_t d = (uint32_t)e - 1;
                        const uint32_t at = atomicAdd(&dfill[d], 1u);
                        if (at < dcount[d]) list[dstart[d] + at] = (uint32_t)t;
                        break;
                    }
                }
            }
        }
    }
    if (!any_dup) return;
    __syncthreads();
    // repeated keys: the o-th smallest of the gathered positions
    for (int64_t j = 1 + threadIdx.x; j <= js; j += kTagThreads) {
        const int64_t r = j * x - 1;
        const uint32_t v = blk[r];
        if ((r == 0 || blk[r - 1] != v) && (r + 1 == len || blk[r + 1] != v)) continue;
        uint32_t g = hash(v, kTagDupBits), d = 0;
        for (int probe = 0; probe < kTagDupSlots; ++probe, g = (g + 1) & (kTagDupSlots - 1)) {
            const unsigned long long e = D[g];
            if (e == 0ull) break;
            if ((uint32_t)(e >> 32) == v) {
                d = (uint32_t)e - 1;
                break;
            }
        }
        int64_t a = 0, b = r;  // the first rank of v
        while (a < b) {
            const int64_t mid = (a + b) >> 1;
            if (blk[mid] < v) a = mid + 1;
            else b = mid;
        }
        const uint32_t o = (uint32_t)(r - a), c = dcount[d], *L = list + dstart[d];
        uint32_t tag = 0;
        for (uint32_t i = 0; i < c; ++i) {  // the position with exactly o smaller ones
            uint32_t below = 0;
            for (uint32_t q = 0; q < c; ++q) below += L[q] < L[i];
            if (below == o) tag = L[i];
        }
        stag[k * s + (j - 1)] = (uint32_t)(lo + tag);
    }
}

// ---------------------------------------------------------------------------
// Sample sort (Fig. 1 step 5): LSD radix sort of the records (phi, tag) by the
// bytes of tag, then of phi.  Byte positions on which every record agrees are
// skipped; the pass table is built on the device.
// ---------------------------------------------------------------------------
// Blocks of few distinct keys (regular sampling, 32-bit keys): a block's
// sorted order by (phi, tag) is its distinct values in order, each repeated in
// position order.  One CTA finds the values with a shared-memory hash table;
// warp w of the CTA owns the w-th of 32 contiguous segments of the block and
// counts the values in it.  From the counts come the distinct values' sorted
// starts and, per warp, the keys of each value in earlier segments.  Every
// warp then walks its segment again in position order: the sorted rank of a
// key is the start of its value, plus that value's keys in earlier segments,
// plus its earlier occurrences in this segment (a running count and the lanes
// of the same value below it).  The records at ranks j*x - 1 are emitted
// without sorting.  When the sorted block is kept, its keys are written as
// runs of equal values in position order and every payload at its key's rank
// (a stable counting sort).  Blocks with more than kLowCardMax values keep their flag
// for the stable block sort.
constexpr int kLowCardThreads = 1024, kLowCardMax = 256, kLowCardSlots = 512;
constexpr int kLowCardWarps = kLowCardThreads / 32;
constexpr size_t kLowCardSmem = sizeof(uint32_t) * kLowCardWarps * kLowCardSlots;  // per-warp counts
// blocks of at most kLowCardStashMax keys keep every key's slot from the first
// pass (16 bits each), so the second pass neither reloads nor hashes the keys
constexpr int64_t kLowCardStashMax = 65536;
static size_t lowcard_smem(int64_t m) { return kLowCardSmem + (m <= kLowCardStashMax ? 2 * (size_t)m : 0); }
template <int DT>
__global__ void __launch_bounds__(kLowCardThreads, 1)
run_sample_lowcard_kernel(const typename KeyTraits<DT>::T *__restrict__ keys, int64_t n, int64_t m, int64_t s,
                          int64_t x, typename KeyTraits<DT>::T *sphi, uint32_t *stag, uint32_t *retry,
                          typename KeyTraits<DT>::T *runs, const uint32_t *__restrict__ vals_in,
                          uint32_t *runs_val) {
    using K = typename KeyTraits<DT>::T;
    static_assert(sizeof(K) == 4, "32-bit keys");
    constexpr int T = kLowCardThreads, W = kLowCardWarps, NS = kLowCardSlots;
    extern __shared__ __align__(16) uint32_t wcnt[];       // [W][NS]: keys per slot in warp w's segment
    uint16_t *sid16 = reinterpret_cast<uint16_t *>(wcnt + kLowCardWarps * kLowCardSlots);  // slot of each key
    __shared__ unsigned long long slot[NS];                 // (1 << 32) | phi, 0 = empty
    __shared__ uint32_t start[NS];                          // sorted start of the slot's value
    __shared__ uint32_t vals[kLowCardMax], sid[kLowCardMax], rank_of[kLowCardMax], tot_sorted[kLowCardMax];
    __shared__ uint32_t val_of_rank[kLowCardMax];
    __shared__ uint32_t tmp[W + 1];
    __shared__ int ndistinct, overflow;
    const int64_t k = blockIdx.x;
    if (retry[k] == 0) return;  // sorted by the keys-only block sort
    const bool stash = m <= kLowCardStashMax;
    const uint32_t xx = (uint32_t)x;
    const int64_t lo = k * m;
    const int64_t len = lo < n ? imin64(m, n - lo) : 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < NS; i += T) slot[i] = 0ull;
    for (int i = tid; i < W * NS; i += T) wcnt[i] = 0;
    if (tid == 0) {
        ndistinct = 0;
        overflow = 0;
    }
    __syncthreads();
    auto hash = [](uint32_t f) {  // murmur3's 32-bit finaliser, top 9 bits
        f ^= f >> 16;
        f *= 0x85ebca6bu;
        f ^= f >> 13;
        f *= 0xc2b2ae35u;
        f ^= f >> 16;
        return f >> (32 - 9);
    };
    static_assert(NS == 512, "9-bit hash");
    // slot holding f (inserting it when absent); -1 when the table is full
    auto find = [&](uint32_t f, bool insert) -> int {
        const unsigned long long want = (1ull << 32) | f;
        uint32_t h = hash(f);
        for (int probe = 0; probe < NS; ++probe, h = (h + 1) & (NS - 1)) {
            unsigned long long cur = slot[h];
            if (cur == want) return (int)h;
            if (cur == 0ull) {
                if (!insert) return -1;
                cur = atomicCAS(&slot[h], 0ull, want);
                if (cur == 0ull) {
                    if (atomicAdd(&ndistinct, 1) >= kLowCardMax) overflow = 1;
                    return (int)h;
                }
                if (cur == want) return (int)h;
            }
        }
        return -1;
    };
    // warp w's segment of the block: [seg0, seg1), whole steps of 32 keys
    const int64_t seg = ((len + W - 1) / W + 31) / 32 * 32;
    const int64_t seg0 = imin64(len, warp * seg), seg1 = imin64(len, seg0 + seg);
    uint32_t *mine = wcnt + warp * NS;
    // keys of kAhead steps of 32 are loaded before the first is used
    constexpr int kAhead = 8;
    uint32_t fa[kAhead];
    auto load_ahead = [&](int64_t e0) {
#pragma unroll
        for (int u = 0; u < kAhead; ++u) {
            const int64_t e = e0 + u * 32 + lane;
            fa[u] = e < seg1 ? (uint32_t)KeyTraits<DT>::phi(keys[lo + e]) : 0u;
        }
    };
    // pass 1: distinct values, and their keys per segment
    for (int64_t e0 = seg0; e0 < seg1; e0 += 32 * kAhead) {
        load_ahead(e0);
#pragma unroll
        for (int u = 0; u < kAhead; ++u) {
            const bool ok = e0 + u * 32 + lane < seg1;
            const uint32_t act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const uint32_t f = fa[u];
                const int h = find(f, true);
                const uint32_t peers = __match_any_sync(act, f);
                if (stash) sid16[e0 + u * 32 + lane] = (uint16_t)max(h, 0);
                if (h < 0) overflow = 1;
                else if (lane == __ffs(peers) - 1) mine[h] += (uint32_t)__popc(peers);  // this warp's own counts
            }
        }
    }
    __syncthreads();
    if (overflow || ndistinct > kLowCardMax) return;  // leave the block to the stable sort
    const int nd = ndistinct;
    // the distinct values, compacted in slot order (ballots over the slots)
    if (tid < NS) {
        const uint32_t b = __ballot_sync(0xffffffffu, slot[tid] != 0ull);
        if (lane == 0) tmp[warp] = (uint32_t)__popc(b);
    }
    __syncthreads();
    if (tid < NS) {
        const bool occ = slot[tid] != 0ull;
        uint32_t c = (uint32_t)__popc(__ballot_sync(0xffffffffu, occ) & lanemask_lt());
        for (int w = 0; w < warp; ++w) c += tmp[w];
        if (occ) {
            vals[c] = (uint32_t)slot[tid];
            sid[c] = (uint32_t)tid;
        }
    }
    __syncthreads();
    // value rank = number of smaller values; per value its total and, per
    // warp, its keys in earlier segments (in place of the counts)
    if (tid < nd) {
        uint32_t r = 0;
        const uint32_t v = vals[tid];
        for (int j = 0; j < nd; ++j) r += vals[j] < v;
        rank_of[tid] = r;
        const uint32_t h = sid[tid];
        uint32_t acc = 0;
        for (int w = 0; w < W; ++w) {
            const uint32_t b = wcnt[w * NS + h];
            wcnt[w * NS + h] = acc;
            acc += b;
        }
        tot_sorted[r] = acc;
    }
    __syncthreads();
    // first sorted position of every value: exclusive scan in rank order
    uint32_t ex = 0;
    if (tid < kLowCardMax) {
        uint32_t wt;
        ex = warp_excl_scan(tid < nd ? tot_sorted[tid] : 0u, &wt);
        if (lane == 31) tmp[warp] = wt;
    }
    __syncthreads();
    if (tid < nd) {
        for (int w = 0; w < warp; ++w) ex += tmp[w];
        tot_sorted[tid] = ex;
    }
    __syncthreads();
    if (tid < nd) {
        start[sid[tid]] = tot_sorted[rank_of[tid]];
        val_of_rank[rank_of[tid]] = vals[tid];
    }
    __syncthreads();
    if (runs) {
        // the sorted block's keys: value of rank r over [start_r, start_r+1),
        // written in position order.  Warp w writes positions [w*len/W,
        // (w+1)*len/W), 32 consecutive ones at a time; each lane finds the
        // rank of its first position and then walks forward.
        const int64_t p0 = (int64_t)warp * len / W, p1 = (int64_t)(warp + 1) * len / W;
        int r = 0;
        if (p0 + lane < p1) {
            int l = 0, h = nd - 1;  // the last rank starting at or before the position
            while (l < h) {
                const int mid = (l + h + 1) >> 1;
                if (tot_sorted[mid] <= (uint32_t)(p0 + lane)) l = mid;
                else h = mid - 1;
            }
            r = l;
        }
        for (int64_t t = p0 + lane; t < p1; t += 32) {
            while (r + 1 < nd && tot_sorted[r + 1] <= (uint32_t)t) ++r;
            runs[lo + t] = (K)val_of_rank[r];
        }
    }
    // pass 2: in position order, sorted rank = start + earlier segments + earlier here
    const float inv_x = 1.0f / (float)xx;
    for (int64_t e0 = seg0; e0 < seg1; e0 += 32 * kAhead) {
        if (!stash) load_ahead(e0);
        uint32_t va[kAhead];  // the payloads of the kAhead steps, loaded before the first is stored
        if (runs_val) {
#pragma unroll
            for (int u = 0; u < kAhead; ++u) {
                const int64_t e = e0 + u * 32 + lane;
                va[u] = e < seg1 ? vals_in[lo + e] : 0u;
            }
        }
#pragma unroll
        for (int u = 0; u < kAhead; ++u) {
            const int64_t e = e0 + u * 32 + lane;
            const bool ok = e < seg1;
            const uint32_t act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                int h;
                uint32_t f;
                if (stash) {
                    h = sid16[e];
                    f = (uint32_t)slot[h];
                } else {
                    f = fa[u];
                    h = max(0, find(f, false));  // present: every key was counted
                }
                const uint32_t peers = __match_any_sync(act, (uint32_t)h);
                const uint32_t g1 = start[h] + mine[h] + (uint32_t)__popc(peers & lanemask_lt()) + 1;  // < 2^32
                __syncwarp(act);
                if (lane == __ffs(peers) - 1) mine[h] += (uint32_t)__popc(peers);
                if (runs_val) runs_val[lo + g1 - 1] = va[u];  // payloads at their ranks
                // j = g1 / x when x divides g1 (the quotient from a float
                // estimate, corrected by one either way)
                uint32_t j = (uint32_t)((float)g1 * inv_x);
                int64_t rem = (int64_t)g1 - (int64_t)j * xx;
                if (rem >= (int64_t)xx) { ++j; rem -= xx; }
                if (rem < 0) { --j; rem += xx; }
                if (rem == 0) {
                    sphi[k * s + (j - 1)] = (K)f;
                    stag[k * s + (j - 1)] = (uint32_t)(lo + e);
                }
            }
            __syncwarp();
        }
    }
    if (tid == 0) retry[k] = 0;  // done
}

template <typename K>
__device__ __forceinline__ uint32_t record_digit(K phi, uint32_t tag, int q) {
    return q < 4 ? (tag >> (8 * q)) & 255u : (uint32_t)(phi >> (8 * (q - 4))) & 255u;
}

template <typename K>
__global__ void lsd_hist_kernel(const K *__restrict__ phi, const uint32_t *__restrict__ tag, int64_t S,
                                uint32_t *hist) {
    constexpr int NPOS = 4 + (int)sizeof(K);
    __shared__ uint32_t h[NPOS][256];
    for (int i = threadIdx.x; i < NPOS * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < S;
         r += (int64_t)gridDim.x * blockDim.x) {
        const K f = phi[r];
        const uint32_t t = tag[r];
#pragma unroll
        for (int q = 0; q < NPOS; ++q) atomicAdd(&h[q][record_digit(f, t, q)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NPOS * 256; i += blockDim.x) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
    if constexpr (sizeof(K) == 4) {  // value range of the sample, for the MSD sort
        uint32_t mn_inv = 0, mx = 0;
        for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < S;
             r += (int64_t)gridDim.x * blockDim.x) {
            const uint32_t f = (uint32_t)phi[r];
            mn_inv = max(mn_inv, ~f);
            mx = max(mx, f);
        }
        mn_inv = __reduce_max_sync(0xffffffffu, mn_inv);
        mx = __reduce_max_sync(0xffffffffu, mx);
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&hist[NPOS * 256], mn_inv);
            atomicMax(&hist[NPOS * 256 + 1], mx);
        }
    }
}

// table[0] = passes; then (position, src, dst) per pass; table[1+3*NPOS] = final buffer
template <typename K>
__global__ void lsd_plan_kernel(const uint32_t *hist, int64_t S, int32_t *table, int phi_only) {
    constexpr int NPOS = 4 + (int)sizeof(K);
    __shared__ int trivial[NPOS];
    if (threadIdx.x < NPOS) trivial[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < NPOS * 256; i += blockDim.x)
        if ((int64_t)hist[i] == S) trivial[i / 256] = 1;  // every record has this byte
    __syncthreads();
    if (threadIdx.x != 0) return;
    int np = 0, cur = 0;
    for (int q = phi_only ? 4 : 0; q < NPOS; ++q) {
        if (trivial[q]) continue;
        table[1 + 3 * np] = q;
        table[2 + 3 * np] = cur;
        table[3 + 3 * np] = 1 - cur;
        cur = 1 - cur;
        ++np;
    }
    table[0] = np;
    table[1 + 3 * NPOS] = cur;
}

template <typename K>
__global__ void __launch_bounds__(kLsdThreads)
lsd_upsweep_kernel(const LsdBuffers<K> b, int64_t S, int pass, const int32_t *table, uint32_t *counts,
                   int64_t tiles) {
    if (pass >= table[0]) return;
    const int q = table[1 + 3 * pass], src = table[2 + 3 * pass];
    __shared__ uint32_t h[256];
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
        __syncthreads();
        const int64_t t0 = tile * kLsdTile;
        for (int i = threadIdx.x; i < kLsdTile; i += kLsdThreads) {
            const int64_t r = t0 + i;
            if (r < S) atomicAdd(&h[record_digit(b.phi[src][r], b.tag[src][r], q)], 1u);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += blockDim.x) counts[(int64_t)d * tiles + tile] = h[d];
        __syncthreads();
    }
}

// Exclusive scan of the per-tile counts of one digit (CTA d scans digit d)
// plus the number of records with a smaller digit.
__global__ void __launch_bounds__(256) lsd_scan_kernel(uint32_t *counts, int64_t tiles, int pass,
                                                       const int32_t *table, const uint32_t *hist) {
    if (pass >= table[0]) return;
    __shared__ uint32_t tmp[40];
    __shared__ uint32_t dbase;
    const int q = table[1 + 3 * pass];
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t below = tid < d ? hist[q * 256 + tid] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
    if (lane == 0) tmp[warp] = below;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += tmp[w];
        dbase = t;
    }
    __syncthreads();
    uint32_t *c = counts + (int64_t)d * tiles;
    const int64_t per = (tiles + 255) / 256;
    const int64_t lo = tid * per, hi = imin64(tiles, lo + per);
    uint32_t local = 0;
    for (int64_t i = lo; i < hi; ++i) local += c[i];
    uint32_t wt;
    const uint32_t we = warp_excl_scan(local, &wt);
    __syncthreads();
    if (lane == 31) tmp[warp] = wt;
    __syncthreads();
    if (warp == 0) {
        uint32_t t;
        const uint32_t e = warp_excl_scan(lane < 8 ? tmp[lane] : 0u, &t);
        if (lane < 8) tmp[lane] = e;
    }
    __syncthreads();
    uint32_t run = dbase + tmp[warp] + we;
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t v = c[i];
        c[i] = run;
        run += v;
    }
}

// Scatter of one pass: the tile is ranked stably per digit, grouped by digit
// in shared memory, and each digit's run is written contiguously.
template <typename K> constexpr size_t lsd_downsweep_smem() {
    return sizeof(typename BlockRank<kLsdThreads, kLsdItems, 8>::Smem) + 256 * 4 * 2 + 40 * 4 +
           (size_t)kLsdTile * (sizeof(K) + 4);
}

template <typename K>
__global__ void __launch_bounds__(kLsdThreads)
lsd_downsweep_kernel(LsdBuffers<K> b, int64_t S, int pass, const int32_t *table,
                     const uint32_t *counts, int64_t tiles) {
    if (pass >= table[0]) return;
    const int q = table[1 + 3 * pass], src = table[2 + 3 * pass], dst = table[3 + 3 * pass];
    using Rank = BlockRank<kLsdThreads, kLsdItems, 8>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename Rank::Smem &sm = *reinterpret_cast<typename Rank::Smem *>(smem_raw);
    uint32_t *base = reinterpret_cast<uint32_t *>(smem_raw + sizeof(typename Rank::Smem));
    uint32_t *start = base + 256;
    uint32_t *tmp = start + 256;
    K *st_f = reinterpret_cast<K *>(tmp + 40);
    st_f = reinterpret_cast<K *>((reinterpret_cast<uintptr_t>(st_f) + 15) & ~uintptr_t(15));
    uint32_t *st_t = reinterpret_cast<uint32_t *>(st_f + kLsdTile);
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t t0 = tile * kLsdTile;
        const int n_here = (int)imin64(kLsdTile, S - t0);
        K f[kLsdItems];
        uint32_t t[kLsdItems], d[kLsdItems], rk[kLsdItems];
#pragma unroll
        for (int i = 0; i < kLsdItems; ++i) {
            const int64_t r = t0 + striped_slot<kLsdThreads, kLsdItems>(i);
            if (r < S) {
                f[i] = b.phi[src][r];
                t[i] = b.tag[src][r];
                d[i] = record_digit(f[i], t[i], q);
            } else {
                d[i] = 255;  // after every real record of digit 255 (higher slots)
            }
        }
        Rank::rank(sm, d, rk);
        for (int dd = threadIdx.x; dd < 256; dd += kLsdThreads) {
            base[dd] = counts[(int64_t)dd * tiles + tile];
            start[dd] = sm.digit_tot[dd];
        }
        __syncthreads();
        digit_excl_scan<kLsdThreads, 256>(start, tmp);
#pragma unroll
        for (int i = 0; i < kLsdItems; ++i) {
            const int64_t r = t0 + striped_slot<kLsdThreads, kLsdItems>(i);
            if (r < S) {
                const uint32_t s = start[d[i]] + rk[i];
                st_f[s] = f[i];
                st_t[s] = t[i];
            }
        }
        __syncthreads();
        // staged slot s holds a record of digit dg; its place is base[dg] + s - start[dg]
        for (int s = threadIdx.x; s < n_here; s += kLsdThreads) {
            const uint32_t dg = record_digit(st_f[s], st_t[s], q);
            const uint32_t pos = base[dg] + (uint32_t)s - start[dg];
            b.phi[dst][pos] = st_f[s];
            b.tag[dst][pos] = st_t[s];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// MSD sample sort for 32-bit keys: records are put into 2^BITS bins (4096 up
// to 8M records, 8192 above) by the top BITS bits of phi - min(phi) in one staged pass, and every bin is sorted in
// shared memory by (phi, tag).  Used when no bin holds more than kMsdBinMax
// records; otherwise the LSD passes above run.  Both give the same (unique)
// sorted sample.
//
// Table slots: [kMsdFlag] = 1 when this path is taken, [kMsdShift] = bin
// shift, [kMsdMin] = min(phi).  Scratch in the LSD tile counts: bin counts
// [0, B), bin starts [B, 2B+1), bin cursors [2B+4, 3B+4), B = 2^BITS.
// ---------------------------------------------------------------------------
constexpr int kMsdBinMax = 4096;  // records one CTA sorts in shared memory
constexpr int kMsdFlag = 40, kMsdShift = 41, kMsdMin = 42;
constexpr int64_t kMsdWideSample = 8 << 20;  // samples above this use 8192 bins
template <int BITS> struct Msd {
    static constexpr int kBins = 1 << BITS, kStart = kBins, kCursor = 2 * kBins + 4;
};
constexpr int64_t kMsdMinSample = 1 << 19;  // smaller samples: the LSD passes

__device__ __forceinline__ uint32_t msd_bin(uint32_t f, uint32_t mn, int shift) {
    return (f - mn) >> shift;  // < Msd<BITS>::kBins by the choice of shift
}

template <int BITS>
__global__ void __launch_bounds__(256) msd_hist_kernel(const uint32_t *__restrict__ phi, int64_t S,
                                                       const uint32_t *lsd_hist, int npos, uint32_t *counts) {
    __shared__ uint32_t h[Msd<BITS>::kBins];
    for (int i = threadIdx.x; i < Msd<BITS>::kBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t mn = ~lsd_hist[npos * 256], mx = lsd_hist[npos * 256 + 1];
    const int bl = bit_length<uint32_t>(mx - mn);
    const int shift = bl > BITS ? bl - BITS : 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < S; r += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[msd_bin(phi[r], mn, shift)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < Msd<BITS>::kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], h[i]);
}

// Bin starts; the MSD path is taken when every bin fits one CTA.
template <int BITS>
__global__ void __launch_bounds__(1024) msd_plan_kernel(uint32_t *counts, const uint32_t *lsd_hist, int npos,
                                                        int32_t *table) {
    __shared__ uint32_t tmp[40];
    __shared__ int big;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) big = 0;
    __syncthreads();
    constexpr int PER = Msd<BITS>::kBins / 1024;
    uint32_t v[PER], local = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        v[q] = counts[tid * PER + q];
        local += v[q];
        if (v[q] > (uint32_t)kMsdBinMax) big = 1;
    }
    uint32_t wt;
    const uint32_t we = warp_excl_scan(local, &wt);
    if (lane == 31) tmp[warp] = wt;
    __syncthreads();
    if (warp == 0) {
        uint32_t t;
        const uint32_t e = warp_excl_scan(tmp[lane], &t);
        tmp[lane] = e;
    }
    __syncthreads();
    uint32_t run = tmp[warp] + we;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        counts[Msd<BITS>::kStart + tid * PER + q] = run;
        counts[Msd<BITS>::kCursor + tid * PER + q] = 0;
        run += v[q];
    }
    if (tid == 1023) counts[Msd<BITS>::kStart + Msd<BITS>::kBins] = run;
    if (tid == 0) {
        const uint32_t mn = ~lsd_hist[npos * 256], mx = lsd_hist[npos * 256 + 1];
        const int bl = bit_length<uint32_t>(mx - mn);
        const bool take = !big;
        table[kMsdFlag] = take ? 1 : 0;
        table[kMsdShift] = bl > BITS ? bl - BITS : 0;
        table[kMsdMin] = (int32_t)mn;
        if (take) {
            table[0] = 0;              // no LSD passes
            table[1 + 3 * npos] = 1;   // the sorted sample ends in buffer 1
        }
    }
}

// Records of a tile, grouped by bin in shared memory, each bin's run written
// contiguously at its bin start plus a reserved offset.
constexpr int kMsdThreads = 512, kMsdItems = 16, kMsdTile = kMsdThreads * kMsdItems;
template <int BITS>
__global__ void __launch_bounds__(kMsdThreads) msd_scatter_kernel(LsdBuffers<uint32_t> b, int64_t S,
                                                                  const int32_t *table, uint32_t *counts) {
    if (table[kMsdFlag] == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem_raw);      // Msd<BITS>::kBins + 4
    uint32_t *dlt = cnt + Msd<BITS>::kBins + 4;                           // Msd<BITS>::kBins
    uint32_t *st_f = dlt + Msd<BITS>::kBins;                              // kMsdTile
    uint32_t *st_t = st_f + kMsdTile;                             // kMsdTile
    uint16_t *st_b = reinterpret_cast<uint16_t *>(st_t + kMsdTile);  // kMsdTile
    __shared__ uint32_t tmp[40];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int shift = table[kMsdShift];
    const uint32_t mn = (uint32_t)table[kMsdMin];
    const int64_t t0 = (int64_t)blockIdx.x * kMsdTile;
    const int nh = (int)imin64(kMsdTile, S - t0);
    for (int i = tid; i < Msd<BITS>::kBins; i += kMsdThreads) cnt[i] = 0;
    __syncthreads();
    uint32_t f[kMsdItems], t[kMsdItems], br[kMsdItems];
#pragma unroll
    for (int i = 0; i < kMsdItems; ++i) {
        const int s = i * kMsdThreads + tid;
        if (s < nh) {
            f[i] = b.phi[0][t0 + s];
            t[i] = b.tag[0][t0 + s];
            const uint32_t bin = msd_bin(f[i], mn, shift);
            br[i] = bin << 16 | atomicAdd(&cnt[bin], 1u);
        }
    }
    __syncthreads();
    // starts of the bins inside the tile (8 bins per thread) and reservations
    constexpr int PER = Msd<BITS>::kBins / kMsdThreads;
    uint32_t c[PER], local = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        c[q] = cnt[tid * PER + q];
        local += c[q];
    }
    uint32_t wt;
    const uint32_t we = warp_excl_scan(local, &wt);
    if (lane == 31) tmp[warp] = wt;
    __syncthreads();
    if (warp == 0) {
        uint32_t tt;
        const uint32_t e = warp_excl_scan(lane < kMsdThreads / 32 ? tmp[lane] : 0u, &tt);
        if (lane < kMsdThreads / 32) tmp[lane] = e;
    }
    __syncthreads();
    uint32_t run = tmp[warp] + we;
    uint32_t at[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) at[q] = c[q] ? atomicAdd(&counts[Msd<BITS>::kCursor + tid * PER + q], c[q]) : 0u;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int bin = tid * PER + q;
        cnt[bin] = run;
        dlt[bin] = counts[Msd<BITS>::kStart + bin] + at[q] - run;  // output slot of tile position s: dlt + s
        run += c[q];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kMsdItems; ++i) {
        const int s = i * kMsdThreads + tid;
        if (s < nh) {
            const uint32_t bin = br[i] >> 16, pos = cnt[bin] + (br[i] & 0xffffu);
            st_f[pos] = f[i];
            st_t[pos] = t[i];
            st_b[pos] = (uint16_t)bin;
        }
    }
    __syncthreads();
    for (int s = tid; s < nh; s += kMsdThreads) {
        const uint32_t o = dlt[st_b[s]] + (uint32_t)s;
        b.phi[1][o] = st_f[s];
        b.tag[1][o] = st_t[s];
    }
}
template <int BITS>
constexpr size_t msd_scatter_smem() { return (size_t)(2 * Msd<BITS>::kBins + 4 + 2 * kMsdTile) * 4 + (size_t)kMsdTile * 2; }

// One bin per CTA, (phi, tag) as one 64-bit key: a counting pass on the top
// 11 bits of the bin's range, then each key's place inside its count bin by
// comparison; a bin whose count bins are too long is sorted by a bitonic
// network instead.  (Sampling with replacement can repeat a record: equal
// keys are ordered by their slot.)
constexpr int kMsdLocalThreads = 512, kMsdLocalItems = kMsdBinMax / kMsdLocalThreads;
constexpr int kMsdCountBits = 11, kMsdCountBins = 1 << kMsdCountBits;
template <int BITS>
__global__ void __launch_bounds__(kMsdLocalThreads) msd_local_kernel(LsdBuffers<uint32_t> b, const int32_t *table,
                                                                      const uint32_t *counts) {
    if (table[kMsdFlag] == 0) return;
    __shared__ uint64_t a[kMsdBinMax];
    __shared__ uint32_t ch[kMsdCountBins + 4];
    __shared__ uint32_t tmp[40];
    constexpr int T = kMsdLocalThreads, IT = kMsdLocalItems;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lo = counts[Msd<BITS>::kStart + blockIdx.x], hi = counts[Msd<BITS>::kStart + blockIdx.x + 1];
    const int n = (int)(hi - lo);
    if (n <= 1) return;
    // keys of this bin lie in [klo, khi]
    const int shift = table[kMsdShift];
    const uint32_t mn = (uint32_t)table[kMsdMin];
    const uint64_t flo = (uint64_t)mn + ((uint64_t)blockIdx.x << shift);
    const uint64_t klo = flo << 32, span = (((uint64_t)1 << shift) << 32) - 1;
    const int bits = bit_length<uint64_t>(span);
    const int sh = bits > kMsdCountBits ? bits - kMsdCountBits : 0;
    uint64_t k[IT];
    uint32_t r[IT];
    for (int i = tid; i < kMsdCountBins; i += T) ch[i] = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int e = i * T + tid;
        if (e < n) {
            k[i] = (uint64_t)b.phi[1][lo + e] << 32 | b.tag[1][lo + e];
            const uint64_t d = (k[i] - klo) >> sh;
            r[i] = atomicAdd(&ch[d < kMsdCountBins ? (uint32_t)d : kMsdCountBins - 1], 1u);
        }
    }
    __syncthreads();
    // exclusive scan of the count bins (8 per thread), longest bin
    constexpr int PER = kMsdCountBins / T;
    uint32_t v[PER], loc = 0, mx = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        v[q] = ch[tid * PER + q];
        loc += v[q];
        mx = max(mx, v[q]);
    }
    uint32_t wt;
    const uint32_t we = warp_excl_scan(loc, &wt);
    if (lane == 31) tmp[warp] = wt;
    const bool too_long = __syncthreads_or(mx > 64);
    if (!too_long) {
        if (warp == 0) {
            uint32_t t;
            const uint32_t e = warp_excl_scan(lane < T / 32 ? tmp[lane] : 0u, &t);
            if (lane < T / 32) tmp[lane] = e;
        }
        __syncthreads();
        uint32_t run = tmp[warp] + we;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            ch[tid * PER + q] = run;
            run += v[q];
        }
        if (tid == 0) ch[kMsdCountBins] = (uint32_t)n;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = i * T + tid;
            if (e < n) {
                const uint64_t d = (k[i] - klo) >> sh;
                r[i] += ch[d < kMsdCountBins ? (uint32_t)d : kMsdCountBins - 1];
                a[r[i]] = k[i];
            }
        }
        __syncthreads();
        // keys sharing a count bin: place = bin start + smaller keys in the bin
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = i * T + tid;
            if (e < n) {
                const uint64_t d = (k[i] - klo) >> sh;
                const uint32_t cb = d < kMsdCountBins ? (uint32_t)d : kMsdCountBins - 1;
                const uint32_t b0 = ch[cb], b1 = ch[cb + 1], self = r[i];
                if (b1 - b0 > 1) {
                    uint32_t pos = b0;
                    for (uint32_t y = b0; y < b1; ++y) {
                        const uint64_t x = a[y];
                        pos += (x < k[i]) | ((x == k[i]) & (y < self));
                    }
                    r[i] = pos;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IT; ++i)
            if (i * T + tid < n) a[r[i]] = k[i];
        __syncthreads();
    } else {
        int n2 = 1;
        while (n2 < n) n2 <<= 1;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = i * T + tid;
            if (e < n) a[e] = k[i];
        }
        for (int e = n + tid; e < n2; e += T) a[e] = ~0ull;
        __syncthreads();
        for (int kk = 2; kk <= n2; kk <<= 1)
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int t = tid; t < (n2 >> 1); t += T) {
                    const int i = 2 * t - (t & (j - 1));
                    const int l = i + j;
                    const bool up = (i & kk) == 0;
                    const uint64_t x = a[i], y = a[l];
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
                __syncthreads();
            }
    }
    for (int i = tid; i < n; i += T) {
        b.phi[1][lo + i] = (uint32_t)(a[i] >> 32);
        b.tag[1][lo + i] = (uint32_t)a[i];
    }
}

// ---------------------------------------------------------------------------
// Splitter selection (Fig. 1 step 6): splitter i of the p buckets is the
// sample record of 1-indexed rank i*Q (Q = q regular, s random).  Each bucket
// is refined into B sub-buckets by the records of rank floor(j*Q/B); for
// j = i*B these are the paper's splitters, so the buckets are unchanged.
// "Broadcast" (Fig. 1 step 7) is the copy into every CTA's shared memory.
// ---------------------------------------------------------------------------
template <typename K>
__global__ void splitter_kernel(LsdBuffers<K> b, const int32_t *table, int npos, int64_t P, int64_t Q,
                                int64_t B, K *vphi, uint32_t *vtag, LutParams<K> *lutp) {
    const int fin = table[1 + 3 * npos];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (j < P) {
        const int64_t r = (j * Q) / B;  // 1-indexed rank
        vphi[j - 1] = b.phi[fin][r - 1];
        vtag[j - 1] = b.tag[fin][r - 1];
    }
    if (j == 1 || (P == 1 && blockIdx.x == 0 && threadIdx.x == 0)) {
        LutParams<K> lp;
        if (P > 1) {
            const K lo = b.phi[fin][(1 * Q) / B - 1];
            const K hi = b.phi[fin][((P - 1) * Q) / B - 1];
            lp.base = lo;
            lp.span = hi - lo;
            const int bl = bit_length<K>(lp.span);
            lp.shift = bl > kLutBits ? (uint32_t)(bl - kLutBits) : 0u;
        } else {
            lp.base = 0;
            lp.span = 0;
            lp.shift = 0;
        }
        lp.nsplit = (uint32_t)(P - 1);
        *lutp = lp;
    }
}

template <typename K>
__global__ void lut_kernel(const K *vphi, const LutParams<K> *lutp, uint16_t *lut) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > kLutCells) return;
    const LutParams<K> lp = *lutp;
    uint32_t lo = 0, hi = lp.nsplit;
    if ((K)c > (lp.span >> lp.shift)) {
        lo = lp.nsplit;
    } else {
        const K thr = lp.base + ((K)c << lp.shift);
        while (lo < hi) {  // number of splitters with phi < thr
            const uint32_t mid = (lo + hi) >> 1;
            if (vphi[mid] < thr) lo = mid + 1;
            else hi = mid;
        }
    }
    lut[c] = (uint16_t)lo;
}

// ---------------------------------------------------------------------------
// Diagnostics: records in the paper's tag form, per-key buckets, pad counts.
// ---------------------------------------------------------------------------
template <typename K>
__device__ __forceinline__ bsps_record to_record(K phi, uint32_t tag, int64_t n, int64_t m, int64_t M,
                                                 bool regular) {
    bsps_record r;
    if ((int64_t)tag >= n) {
        r.phi = ~0ull;
        r.tag = (uint64_t)tag - (uint64_t)n;
        r.pad = 1;
    } else {
        r.phi = (uint64_t)phi;
        r.tag = regular ? (uint64_t)(tag / m) * M + tag % m : tag;
        r.pad = 0;
    }
    r.reserved = 0;
    return r;
}

template <typename K>
__global__ void sample_records_kernel(LsdBuffers<K> b, const int32_t *table, int npos, int64_t S,
                                      int64_t n, int64_t m, int64_t M, bool regular, bsps_record *out) {
    const int fin = table[1 + 3 * npos];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S) out[i] = to_record(b.phi[fin][i], b.tag[fin][i], n, m, M, regular);
}

template <typename K>
__global__ void splitter_records_kernel(const K *vphi, const uint32_t *vtag, int64_t p, int64_t B,
                                        int64_t n, int64_t m, int64_t M, bool regular,
                                        bsps_record *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (i < p) out[i - 1] = to_record(vphi[i * B - 1], vtag[i * B - 1], n, m, M, regular);
}

// Per-key buckets of the keys (diagnostics).  With the learned classifier
// every key goes through the same classify_learned (network, index over its
// output, search and check) the routing kernels use, so its result can be
// compared key by key.
template <int DT, bool LEARNED>
__global__ void __launch_bounds__(256) bucket_of_kernel(const typename KeyTraits<DT>::T *keys, int64_t n, int64_t B,
                                 const typename KeyTraits<DT>::T *vphi, const uint32_t *vtag,
                                 const uint16_t *lut,
                                 const LutParams<typename KeyTraits<DT>::T> *lutp, const MlpTables *mlp_tables,
                                 const uint16_t *ylut, int64_t P, uint32_t tag_floor, int32_t *out) {
    __shared__ __align__(16) unsigned char mt_raw[LEARNED ? sizeof(MlpTables) : 16];
    const MlpTables *mt = reinterpret_cast<const MlpTables *>(mt_raw);
    if constexpr (LEARNED) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(mlp_tables);
        uint32_t *dst = reinterpret_cast<uint32_t *>(mt_raw);
        for (int q = threadIdx.x; q < (int)(sizeof(MlpTables) / 4); q += blockDim.x) dst[q] = src[q];
        __syncthreads();
    }
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    uint32_t v;
    if constexpr (LEARNED) {
        uint32_t steps;
        bool mis;
        v = classify_learned<DT>(keys[g], max((uint32_t)g, tag_floor), *mt, ylut, (uint32_t)(P - 1), vphi, vtag,
                                 steps, mis);
    } else {
        const LutParams<typename KeyTraits<DT>::T> lp = *lutp;
        v = classify_key(KeyTraits<DT>::phi(keys[g]), max((uint32_t)g, tag_floor), lp, lut, vphi, vtag);
    }
    out[g] = (int32_t)(v / B);
}

template <typename K>
__global__ void pad_sizes_kernel(int64_t n, int64_t R, int64_t m, int64_t M, int64_t B, const K *vphi,
                                 const uint32_t *vtag, const uint16_t *lut, const LutParams<K> *lutp,
                                 int dup_off, unsigned long long *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * M) return;
    const int64_t k = t / M, j = t % M;
    const int64_t len = k * m < n ? min(m, n - k * m) : 0;
    if (j < len) return;
    const LutParams<K> lp = *lutp;
    // without tags a pad equals the pad splitters and follows them all
    const uint32_t tag = dup_off ? 0xffffffffu : (uint32_t)(n + k * M + j);
    const uint32_t v = classify_key(all_ones<K>(), tag, lp, lut, vphi, vtag);
    atomicAdd(&out[v / B], 1ull);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int DT> static LsdBuffers<typename KeyTraits<DT>::T> lsd_buffers(const Ctx &c) {
    using K = typename KeyTraits<DT>::T;
    LsdBuffers<K> b;
    b.phi[0] = (K *)c.ly.sphi[0];
    b.phi[1] = (K *)c.ly.sphi[1];
    b.tag[0] = c.ly.stag[0];
    b.tag[1] = c.ly.stag[1];
    return b;
}

template <int DT, int CL, int ITEMS> static cudaError_t launch_run_sample(const Ctx &c, const uint32_t *only) {
    using K = typename KeyTraits<DT>::T;
    using SS = SegSort<K, true, CL, ITEMS>;
    const size_t smem = SS::smem_bytes();
    auto kern = run_sample_kernel<DT, CL, ITEMS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const Plan &p = c.pl;
    kern<<<(unsigned)(p.R * CL), kSortThreads, smem, c.stream>>>(
        (const K *)c.keys_in, p.n, p.m, p.M, p.s, p.x, (K *)c.ly.sphi[0], c.ly.stag[0],
        (uint32_t *)&c.ly.status->run_too_big, only, p.keep_runs ? (K *)c.ly.runs : nullptr, c.vals_in,
        p.keep_runs && p.pairs ? c.ly.runs_val : nullptr);
    return cudaGetLastError();
}

template <int DT, int CL> static cudaError_t launch_run_sample_keys(const Ctx &c) {
    using K = typename KeyTraits<DT>::T;
    using SS = SegSortKeys<uint64_t, CL, kRunKeysItems>;
    const size_t smem = SS::smem_bytes();
    auto kern = run_sample_keys_kernel<DT, CL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const Plan &p = c.pl;
    e = cudaMemsetAsync(c.ly.run_retry, 0, (size_t)p.R * 4, c.stream);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)(p.R * CL), 512, smem, c.stream>>>(
        (const K *)c.keys_in, p.n, p.m, p.M, p.s, p.x, (K *)c.ly.sphi[0], c.ly.stag[0], c.ly.run_retry,
        p.keep_runs ? (K *)c.ly.runs : nullptr, c.vals_in, p.keep_runs && p.pairs ? c.ly.runs_val : nullptr);
    return cudaGetLastError();
}

// the kept blocks are sorted by the counting sort: keys without payloads
// (it moves keys only), whole 16-byte groups of keys in every block and in
// the input (its bulk copies read nothing past n)
bool counting_block_sort(const Ctx &c) {
    const Plan &p = c.pl;
    return p.keep_runs && !p.pairs && p.key_bytes == 4 && run_keys_cluster(p) != 0 && p.m % 4 == 0 &&
           p.n % 4 == 0 && ((uintptr_t)c.keys_in & 15) == 0;
}

template <int DT, int CL> static cudaError_t launch_run_sample_count(const Ctx &c) {
    using SS = BucketKeys32<CL>;
    const size_t smem = SS::smem_bytes();
    auto kern = run_sample_count_kernel<DT, CL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const Plan &p = c.pl;
    e = cudaMemsetAsync(c.ly.run_retry, 0, (size_t)p.R * 4, c.stream);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)(p.R * CL), 512, smem, c.stream>>>((const uint32_t *)c.keys_in, p.n, p.m, p.M, p.s, p.x,
                                                        (uint32_t *)c.ly.sphi[0], c.ly.stag[0], c.ly.run_retry,
                                                        (uint32_t *)c.ly.runs, c.ly.status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int bits = tag_slot_bits(p);
    e = cudaFuncSetAttribute(run_sample_tags_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tag_smem(kTagSlotBitsMax));
    if (e != cudaSuccess) return e;
    run_sample_tags_kernel<DT><<<(unsigned)p.R, kTagThreads, tag_smem(bits), c.stream>>>(
        (const uint32_t *)c.keys_in, (const uint32_t *)c.ly.runs, p.n, p.m, p.s, p.x, bits,
        (uint32_t *)c.ly.sphi[0], c.ly.stag[0], c.ly.run_retry);
    return cudaGetLastError();
}

// cluster size of the keys-only block sort (0: not used)
int run_keys_cluster(const Plan &p) {
    if (p.sampling != BSPS_REGULAR || p.key_bytes != 4 || p.m >= ((int64_t)1 << 32)) return 0;
    for (int cl = 1; cl <= 8; cl *= 2)
        if (p.m <= (int64_t)cl * 512 * kRunKeysItems) return cl;
    return 0;
}

template <int DT> static cudaError_t launch_sample_t(const Ctx &c) {
    using K = typename KeyTraits<DT>::T;
    const Plan &p = c.pl;
    if (p.sampling == BSPS_RANDOM) {
        if (p.sample_size == 0) return cudaSuccess;
        const int64_t blocks4 = (p.sample_size + 3) / 4;
        sample_random_kernel<DT><<<(unsigned)((blocks4 + 255) / 256), 256, 0, c.stream>>>(
            (const K *)c.keys_in, p.n, p.sample_size, p.seed, (K *)c.ly.sphi[0], c.ly.stag[0]);
        return cudaGetLastError();
    }
    const uint32_t *only = nullptr;
    if constexpr (sizeof(K) == 4) {
        cudaError_t e = cudaSuccess;
        if (counting_block_sort(c)) {
            switch (run_keys_cluster(p)) {
            case 1: e = launch_run_sample_count<DT, 1>(c); break;
            case 2: e = launch_run_sample_count<DT, 2>(c); break;
            case 4: e = launch_run_sample_count<DT, 4>(c); break;
            default: e = launch_run_sample_count<DT, 8>(c); break;
            }
            only = c.ly.run_retry;
        } else {
            switch (run_keys_cluster(p)) {
            case 0: break;
            case 1: e = launch_run_sample_keys<DT, 1>(c); only = c.ly.run_retry; break;
            case 2: e = launch_run_sample_keys<DT, 2>(c); only = c.ly.run_retry; break;
            case 4: e = launch_run_sample_keys<DT, 4>(c); only = c.ly.run_retry; break;
            default: e = launch_run_sample_keys<DT, 8>(c); only = c.ly.run_retry; break;
            }
        }
        if (e != cudaSuccess) return e;
        if (only) {  // blocks of few distinct keys, before the stable sort
            e = cudaFuncSetAttribute(run_sample_lowcard_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)lowcard_smem(p.m));
            if (e != cudaSuccess) return e;
            run_sample_lowcard_kernel<DT><<<(unsigned)p.R, kLowCardThreads, lowcard_smem(p.m), c.stream>>>(
                (const K *)c.keys_in, p.n, p.m, p.s, p.x, (K *)c.ly.sphi[0], c.ly.stag[0], c.ly.run_retry,
                p.keep_runs ? (K *)c.ly.runs : nullptr, c.vals_in, p.keep_runs && p.pairs ? c.ly.runs_val : nullptr);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    constexpr int IT = sizeof(K) == 8 ? kRunItems64 : kRunItems32;
    switch (p.run_cl) {
    case 1: return launch_run_sample<DT, 1, IT>(c, only);
    case 2: return launch_run_sample<DT, 2, IT>(c, only);
    case 4: return launch_run_sample<DT, 4, IT>(c, only);
    case 8: return launch_run_sample<DT, 8, IT>(c, only);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sample(const Ctx &c) {
    switch (c.pl.dtype) {
    case BSPS_U32: return launch_sample_t<BSPS_U32>(c);
    case BSPS_I32: return launch_sample_t<BSPS_I32>(c);
    case BSPS_F32: return launch_sample_t<BSPS_F32>(c);
    default: return launch_sample_t<BSPS_F64>(c);
    }
}

template <int BITS> static cudaError_t launch_msd(const Ctx &c, LsdBuffers<uint32_t> b, int hist_blocks) {
    const Plan &p = c.pl;
    constexpr int NPOS = 8;
    uint32_t *cnt = c.ly.lsd_counts;
    cudaError_t e = cudaMemsetAsync(cnt, 0, Msd<BITS>::kBins * sizeof(uint32_t), c.stream);
    if (e != cudaSuccess) return e;
    msd_hist_kernel<BITS><<<max(hist_blocks, 1), 256, 0, c.stream>>>(b.phi[0], p.sample_size, c.ly.lsd_hist, NPOS,
                                                                    cnt);
    msd_plan_kernel<BITS><<<1, 1024, 0, c.stream>>>(cnt, c.ly.lsd_hist, NPOS, c.ly.lsd_table);
    e = cudaFuncSetAttribute(msd_scatter_kernel<BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)msd_scatter_smem<BITS>());
    if (e != cudaSuccess) return e;
    const unsigned mt = (unsigned)((p.sample_size + kMsdTile - 1) / kMsdTile);
    msd_scatter_kernel<BITS><<<mt, kMsdThreads, msd_scatter_smem<BITS>(), c.stream>>>(b, p.sample_size,
                                                                                        c.ly.lsd_table, cnt);
    msd_local_kernel<BITS><<<Msd<BITS>::kBins, kMsdLocalThreads, 0, c.stream>>>(b, c.ly.lsd_table, cnt);
    return cudaGetLastError();
}

template <typename K> static cudaError_t launch_sample_sort_t(const Ctx &c, LsdBuffers<K> b) {
    const Plan &p = c.pl;
    constexpr int NPOS = 4 + (int)sizeof(K);
    cudaError_t e = cudaMemsetAsync(c.ly.lsd_hist, 0, (NPOS * 256 + 2) * sizeof(uint32_t), c.stream);
    if (e != cudaSuccess) return e;
    const int hist_blocks = (int)imin64(1024, (p.sample_size + 1023) / 1024);
    lsd_hist_kernel<K><<<max(hist_blocks, 1), 256, 0, c.stream>>>(b.phi[0], b.tag[0], p.sample_size,
                                                                  c.ly.lsd_hist);
    // A regular sample without pads is R runs, each sorted by (phi, tag), in
    // block order; every tag of a block is below every tag of the next, so a
    // stable sort by phi alone leaves equal phi in tag order: the tag bytes
    // need no passes.  (A pad's tag exceeds every key's, so pads break this.)
    const int phi_only = p.sampling == BSPS_REGULAR && p.n == p.R * p.M;
    lsd_plan_kernel<K><<<1, 256, 0, c.stream>>>(c.ly.lsd_hist, p.sample_size, c.ly.lsd_table, phi_only);
    if constexpr (sizeof(K) == 4) {
        if (msd_sample_sort(p)) {
            e = p.sample_size > kMsdWideSample ? launch_msd<13>(c, b, hist_blocks) : launch_msd<12>(c, b, hist_blocks);
            if (e != cudaSuccess) return e;
        }
    }
    const unsigned tiles = (unsigned)p.lsd_tiles;
    const size_t dsm = lsd_downsweep_smem<K>() + 16;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned lsd_grid = (unsigned)std::min<int64_t>(p.lsd_tiles, 2 * (int64_t)std::max(sms, 1));
    e = cudaFuncSetAttribute(lsd_downsweep_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < NPOS && tiles > 0; ++pass) {
        lsd_upsweep_kernel<K><<<lsd_grid, kLsdThreads, 0, c.stream>>>(b, p.sample_size, pass, c.ly.lsd_table,
                                                                     c.ly.lsd_counts, p.lsd_tiles);
        lsd_scan_kernel<<<256, 256, 0, c.stream>>>(c.ly.lsd_counts, p.lsd_tiles, pass, c.ly.lsd_table,
                                                   c.ly.lsd_hist);
        lsd_downsweep_kernel<K><<<lsd_grid, kLsdThreads, dsm, c.stream>>>(b, p.sample_size, pass,
                                                                         c.ly.lsd_table, c.ly.lsd_counts,
                                                                         p.lsd_tiles);
    }
    return cudaGetLastError();
}

bool msd_sample_sort(const Plan &p) {
    // large samples of 32-bit keys; the tile counts double as the MSD scratch
    const int64_t need = p.sample_size > kMsdWideSample ? Msd<13>::kCursor + Msd<13>::kBins
                                                        : Msd<12>::kCursor + Msd<12>::kBins;
    return p.key_bytes == 4 && p.sample_size >= kMsdMinSample && std::max<int64_t>(p.lsd_tiles, 1) * 256 >= need;
}

cudaError_t launch_sample_sort(const Ctx &c) {
    if (c.pl.key_bytes == 8) return launch_sample_sort_t<uint64_t>(c, lsd_buffers<BSPS_F64>(c));
    return launch_sample_sort_t<uint32_t>(c, lsd_buffers<BSPS_U32>(c));
}

template <typename K> static cudaError_t launch_splitters_t(const Ctx &c, LsdBuffers<K> b) {
    const Plan &p = c.pl;
    const int npos = 4 + (int)sizeof(K);
    const int64_t nthreads = imax64(p.P - 1, 1);
    splitter_kernel<K><<<(unsigned)((nthreads + 255) / 256), 256, 0, c.stream>>>(
        b, c.ly.lsd_table, npos, p.P, p.Q, p.B, (K *)c.ly.vphi, c.ly.vtag, (LutParams<K> *)c.ly.lutp);
    lut_kernel<K><<<(kLutCells + 1 + 255) / 256, 256, 0, c.stream>>>((const K *)c.ly.vphi,
                                                                     (const LutParams<K> *)c.ly.lutp,
                                                                     c.ly.lut);
    return cudaGetLastError();
}

cudaError_t launch_splitters(const Ctx &c) {
    if (c.pl.key_bytes == 8) return launch_splitters_t<uint64_t>(c, lsd_buffers<BSPS_F64>(c));
    return launch_splitters_t<uint32_t>(c, lsd_buffers<BSPS_U32>(c));
}

template <int DT> static cudaError_t launch_debug_t(const Ctx &c) {
    using K = typename KeyTraits<DT>::T;
    const Plan &p = c.pl;
    const bool regular = p.sampling == BSPS_REGULAR;
    LsdBuffers<K> b = lsd_buffers<DT>(c);
    const int npos = 4 + (int)sizeof(K);
    if (c.dbg.sample && p.sample_size > 0)
        sample_records_kernel<K><<<(unsigned)((p.sample_size + 255) / 256), 256, 0, c.stream>>>(
            b, c.ly.lsd_table, npos, p.sample_size, p.n, p.m, p.M, regular, c.dbg.sample);
    if (c.dbg.splitters && p.p > 1)
        splitter_records_kernel<K><<<(unsigned)((p.p + 255) / 256), 256, 0, c.stream>>>(
            (const K *)c.ly.vphi, c.ly.vtag, p.p, p.B, p.n, p.m, p.M, regular, c.dbg.splitters);
    if (c.dbg.bucket_of && p.n > 0) {
        auto kern = p.classify == BSPS_LEARNED ? bucket_of_kernel<DT, true> : bucket_of_kernel<DT, false>;
        kern<<<(unsigned)((p.n + 255) / 256), 256, 0, c.stream>>>(
            (const K *)c.keys_in, p.n, p.B, (const K *)c.ly.vphi, c.ly.vtag, c.ly.lut,
            (const LutParams<K> *)c.ly.lutp, c.ly.mlp_tables, c.ly.ylut, p.P,
            p.dup_off ? (uint32_t)(p.n - 1) : 0u, c.dbg.bucket_of);
    }
    if (c.dbg.pad_sizes) {
        cudaError_t e = cudaMemsetAsync(c.dbg.pad_sizes, 0, sizeof(int64_t) * p.p, c.stream);
        if (e != cudaSuccess) return e;
        if (regular && p.R * p.M > p.n)
            pad_sizes_kernel<K><<<(unsigned)((p.R * p.M + 255) / 256), 256, 0, c.stream>>>(
                p.n, p.R, p.m, p.M, p.B, (const K *)c.ly.vphi, c.ly.vtag, c.ly.lut,
                (const LutParams<K> *)c.ly.lutp, p.dup_off, (unsigned long long *)c.dbg.pad_sizes);
    }
    return cudaGetLastError();
}

cudaError_t launch_debug(const Ctx &c) {
    switch (c.pl.dtype) {
    case BSPS_U32: return launch_debug_t<BSPS_U32>(c);
    case BSPS_I32: return launch_debug_t<BSPS_I32>(c);
    case BSPS_F32: return launch_debug_t<BSPS_F32>(c);
    default: return launch_debug_t<BSPS_F64>(c);
    }
}

} // namespace bsps
