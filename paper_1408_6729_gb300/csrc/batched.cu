// batched.cu -- many independent keys-only sorts of uneven sizes in one call
// (no counterpart in the paper; each instance is the paper's sort, Fig. 2 /
// Fig. 3, with its own parameters).
//
// Small instances run the whole method on chip, one CTA of 1024 threads per
// instance, in one persistent launch: the random sample (Fig. 3 step 4, the
// same counter-based draws as the single-instance path), the sample sort
// (Fig. 1 step 5), the splitters of rank i*s (Fig. 2 step 6), classification
// with the tag-free tie-break (Fig. 2 step 9), the bucket histogram and its
// prefix (Fig. 1 step 9), routing into buckets (Fig. 1 step 11) and the final
// sort of the buckets (Fig. 2 step 12), all in shared memory.  The buckets are
// contiguous, ordered value ranges after routing, so one bitonic network over
// the routed array sorts every bucket in place.  Larger instances run the
// single-instance pipeline on several streams; the whole call is recorded
// into one CUDA graph that later calls with the same arguments relaunch.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace bsps {

constexpr int kSmallThreads = 1024;
constexpr int kSmallMax = BSPS_BATCH_SMALL_MAX;    // keys of an on-chip instance
constexpr int kSampleMax = BSPS_BATCH_SAMPLE_MAX;  // sample records of an on-chip instance
constexpr int kSmallBucketsMax = 256;              // buckets of an on-chip instance
constexpr int kLanesMax = 16;

struct SmallJob {
    int64_t off;    // first key of the instance
    int64_t bbase;  // first bucket-size entry
    uint64_t seed;
    int32_t n, p, s, S;  // keys, buckets, samples per bucket, sample records (s*p - 1)
};

// Ascending bitonic network over a[0..n2), n2 a power of two, whole CTA.
template <typename V> __device__ void bitonic_sort(V *a, int n2) {
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < (n2 >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (j - 1));  // bit j of i is clear
                const int l = i + j;
                const bool up = (i & k) == 0;
                const V x = a[i], y = a[l];
                if ((x > y) == up) {
                    a[i] = y;
                    a[l] = x;
                }
            }
            __syncthreads();
        }
}

__host__ __device__ inline int pow2_ceil(int v) {
    int r = 1;
    while (r < v) r <<= 1;
    return r;
}

// Shared memory of the on-chip kernel.
struct SmallSmem {
    uint64_t rec[kSampleMax];        // sample records (phi << 32 | tag)
    uint32_t phi[kSmallMax];         // the instance's keys
    uint32_t stage[kSmallMax];       // the keys routed into buckets
    uint32_t hist[kSmallBucketsMax + 1];
    uint32_t tmp[40];
};

template <int DT>
__global__ void __launch_bounds__(kSmallThreads, 1)
batch_small_kernel(const typename KeyTraits<DT>::T *__restrict__ keys_in, typename KeyTraits<DT>::T *keys_out,
                   const SmallJob *jobs, int32_t njobs, int64_t *bucket_sizes) {
    static_assert(sizeof(typename KeyTraits<DT>::T) == 4, "on-chip instances hold 32-bit keys");
    constexpr int T = kSmallThreads, IT = kSmallMax / kSmallThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem &sm = *reinterpret_cast<SmallSmem *>(smem_raw);
    const int tid = threadIdx.x;

    for (int32_t jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
        const SmallJob J = jobs[jb];
        const int n = J.n, p = J.p;
        if (n == 0) {
            if (bucket_sizes)
                for (int b = tid; b < p; b += T) bucket_sizes[J.bbase + b] = 0;
            continue;
        }
        const typename KeyTraits<DT>::T *src = keys_in + J.off;
        for (int e = tid; e < n; e += T) sm.phi[e] = KeyTraits<DT>::phi(src[e]);
        __syncthreads();
        // ---- random sample of s*p - 1 records (Fig. 3 step 4) and its sort ----
        const int S = J.S;
        if (p > 1 && S > 0) {
            const int S2 = pow2_ceil(S);
            for (int blk = tid; blk * 4 < S2; blk += T) {
                uint64_t c[4] = {(uint64_t)blk, 0, 0, 0};
                if (blk * 4 < S) philox4x64_10(c, J.seed, 0);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int j = blk * 4 + w;
                    if (j < S) {
                        const uint32_t g = (uint32_t)__umul64hi(c[w], (uint64_t)n);
                        sm.rec[j] = (uint64_t)sm.phi[g] << 32 | g;
                    } else if (j < S2) {
                        sm.rec[j] = ~0ull;
                    }
                }
            }
            __syncthreads();
            bitonic_sort(sm.rec, S2);
        }
        // ---- classify (splitter i is the record of rank i*s), histogram ----
        for (int b = tid; b <= p; b += T) sm.hist[b] = 0;
        __syncthreads();
        uint32_t br[IT];  // bucket << 16 | rank inside the bucket
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = i * T + tid;
            if (e < n) {
                const uint64_t key = (uint64_t)sm.phi[e] << 32 | (uint32_t)e;
                uint32_t lo = 0, hi = (uint32_t)p - 1;  // #{splitters <= key} in [lo, hi]
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (sm.rec[(int64_t)mid * J.s - 1] <= key) lo = mid;
                    else hi = mid - 1;
                }
                br[i] = lo << 16 | atomicAdd(&sm.hist[lo], 1u);
            }
        }
        __syncthreads();
        if (tid < 32) {  // bucket sizes and the buckets' starts
            uint32_t carry = 0;
            for (int b0 = 0; b0 < p; b0 += 32) {
                const int b = b0 + tid;
                const uint32_t c = b < p ? sm.hist[b] : 0u;
                if (bucket_sizes && b < p) bucket_sizes[J.bbase + b] = c;
                uint32_t tot;
                const uint32_t ex = warp_excl_scan(c, &tot);
                if (b < p) sm.hist[b] = carry + ex;
                carry += tot;
            }
        }
        __syncthreads();
        // ---- route into the buckets (Fig. 1 step 11) ----
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = i * T + tid;
            if (e < n) sm.stage[sm.hist[br[i] >> 16] + (br[i] & 0xffffu)] = sm.phi[e];
        }
        const int n2 = pow2_ceil(n);
        for (int e = n + tid; e < n2; e += T) sm.stage[e] = 0xffffffffu;
        __syncthreads();
        // ---- final sort of the buckets (Fig. 2 step 12) ----
        bitonic_sort(sm.stage, n2);
        typename KeyTraits<DT>::T *dst = keys_out + J.off;
        for (int e = tid; e < n; e += T) dst[e] = KeyTraits<DT>::inv(sm.stage[e]);
        __syncthreads();
    }
}

// Folds one instance's device status into the batch's.
__global__ void merge_status_kernel(const DevStatus *from, DevStatus *into) {
    if (threadIdx.x != 0) return;
    if (from->error) set_error(into, from->error);
    if (from->overflow) atomicExch(&into->overflow, 1);
    atomicAdd(&into->timeouts, from->timeouts);
    atomicAdd(&into->slow_buckets, from->slow_buckets);
    atomicMax(&into->max_bucket, from->max_bucket);
    atomicMax(&into->max_vbucket, from->max_vbucket);
    atomicAdd(&into->mispredicted, from->mispredicted);
    atomicAdd(&into->correction_steps, from->correction_steps);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int size_class(int64_t n) {
    int c = 0;
    while (((int64_t)1 << c) < n) ++c;
    return c;
}

static bool valid_tune(const bsps_tune *t) {
    if (!t || t->lanes < 1 || t->lanes > kLanesMax || t->small_max_log2 > 14 || t->learned_min_log2 < 0)
        return false;
    for (int c = 0; c < BSPS_BATCH_CLASSES; ++c)
        if (t->p[c] < 1 || t->p[c] > 65535) return false;
    return true;
}

struct Instance {
    int64_t off, n;
    bsps_params prm;
    bool small;
    int S, s;
};

struct BatchPlan {
    std::vector<Instance> inst;
    std::vector<SmallJob> jobs;
    std::vector<int64_t> bbase;
    size_t lane_ws = 0, jobs_bytes = 0, total = 0;
    int lanes = 1;
};

static int make_batch_plan(const int64_t *h_off, int32_t num, int32_t dtype, const bsps_params *prm,
                           const bsps_tune *t, BatchPlan &bp) {
    if (num < 0 || (num > 0 && !h_off) || !prm || !valid_tune(t)) return BSPS_ERR_INVALID_ARG;
    if (dtype < BSPS_U32 || dtype > BSPS_F64) return BSPS_ERR_UNSUPPORTED_DTYPE;
    if (num > 0 && h_off[0] != 0) return BSPS_ERR_INVALID_ARG;
    // the on-chip instances run the bucket-sort path with the tie-break
    if (prm->final_step != BSPS_FINAL_SORT || prm->duplicates != BSPS_DUP_TAGS) return BSPS_ERR_INVALID_ARG;
    bp.inst.resize(num);
    bp.bbase.assign(num + 1, 0);
    bp.jobs.clear();
    bp.lanes = t->lanes;
    size_t lane_ws = 0;
    for (int32_t i = 0; i < num; ++i) {
        const int64_t n = h_off[i + 1] - h_off[i];
        if (n < 0) return BSPS_ERR_INVALID_ARG;
        Instance &I = bp.inst[i];
        I.off = h_off[i];
        I.n = n;
        I.prm = *prm;
        const int c = std::min(size_class(n), BSPS_BATCH_CLASSES - 1);
        I.prm.p = t->p[c];
        I.prm.seed = prm->seed + (uint64_t)i;
        if (t->learned_min_log2 > 0 && c >= t->learned_min_log2) I.prm.classify = BSPS_LEARNED;
        bp.bbase[i + 1] = bp.bbase[i] + I.prm.p;
        bsps_plan pl;
        const int rc = bsps_get_plan(n, dtype, &I.prm, 0, &pl);
        if (rc) return rc;
        I.s = (int)pl.s;
        I.S = (int)pl.sample_size;
        I.small = c <= t->small_max_log2 && n <= kSmallMax && dtype != BSPS_F64 &&
                  I.prm.sampling == BSPS_RANDOM && I.prm.classify == BSPS_TREE && I.prm.p <= kSmallBucketsMax &&
                  pl.sample_size <= kSampleMax;
        if (I.small) {
            SmallJob J;
            J.off = I.off;
            J.bbase = bp.bbase[i];
            J.seed = I.prm.seed;
            J.n = (int32_t)n;
            J.p = I.prm.p;
            J.s = (int32_t)pl.s;
            J.S = (int32_t)pl.sample_size;
            bp.jobs.push_back(J);
        } else {
            size_t w = 0;
            const int rc2 = bsps_workspace_size(n, dtype, &I.prm, 0, &w);
            if (rc2) return rc2;
            lane_ws = std::max(lane_ws, w);
        }
    }
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    bp.lane_ws = up(lane_ws);
    bp.jobs_bytes = up(std::max<size_t>(1, bp.jobs.size()) * sizeof(SmallJob));
    bp.total = up(sizeof(DevStatus)) + bp.jobs_bytes + (bp.lane_ws ? bp.lane_ws * bp.lanes : 0);
    return BSPS_OK;
}

// Streams and events the call forks into (one set per device, made once).
struct LaneSet {
    bool made = false;
    cudaStream_t origin;  // the stream a recorded call is captured from
    cudaStream_t s[kLanesMax];
    cudaEvent_t fork, join[kLanesMax];
};
static LaneSet g_lanes[64];
static std::mutex g_mu;

// The last recorded graph and what it was recorded for.
struct GraphCache {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
};
static GraphCache g_graph[64];

static int lanes_for_device(LaneSet *&L) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BSPS_ERR_CUDA;
    L = &g_lanes[dev];
    if (!L->made) {
        for (int i = 0; i < kLanesMax; ++i) {
            if (cudaStreamCreateWithFlags(&L->s[i], cudaStreamNonBlocking) != cudaSuccess) return BSPS_ERR_CUDA;
            if (cudaEventCreateWithFlags(&L->join[i], cudaEventDisableTiming) != cudaSuccess) return BSPS_ERR_CUDA;
        }
        if (cudaEventCreateWithFlags(&L->fork, cudaEventDisableTiming) != cudaSuccess) return BSPS_ERR_CUDA;
        if (cudaStreamCreateWithFlags(&L->origin, cudaStreamNonBlocking) != cudaSuccess) return BSPS_ERR_CUDA;
        L->made = true;
    }
    return BSPS_OK;
}

template <int DT> static cudaError_t launch_small_t(const void *in, void *out, const SmallJob *jobs, int32_t njobs,
                                                    int64_t *bsz, cudaStream_t st) {
    using K = typename KeyTraits<DT>::T;
    auto kern = batch_small_kernel<DT>;
    const int smem = (int)sizeof(SmallSmem);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min<int>(njobs, sms));
    kern<<<grid, kSmallThreads, smem, st>>>((const K *)in, (K *)out, jobs, njobs, bsz);
    return cudaGetLastError();
}

static cudaError_t launch_small(int32_t dtype, const void *in, void *out, const SmallJob *jobs, int32_t njobs,
                                int64_t *bsz, cudaStream_t st) {
    switch (dtype) {
    case BSPS_U32: return launch_small_t<BSPS_U32>(in, out, jobs, njobs, bsz, st);
    case BSPS_I32: return launch_small_t<BSPS_I32>(in, out, jobs, njobs, bsz, st);
    case BSPS_F32: return launch_small_t<BSPS_F32>(in, out, jobs, njobs, bsz, st);
    default: return cudaErrorInvalidValue;
    }
}

// Everything the call queues, on `stream` and the lanes forked from it.
static int enqueue_batch(const BatchPlan &bp, const void *in, void *out, int32_t dtype, int64_t *bsz,
                         unsigned char *ws, cudaStream_t stream, LaneSet *L) {
#define BSPS_CK(call)                                    \
    do {                                                 \
        if ((call) != cudaSuccess) return BSPS_ERR_CUDA; \
    } while (0)
    DevStatus *bst = (DevStatus *)ws;
    const SmallJob *djobs = (const SmallJob *)(ws + ((sizeof(DevStatus) + 255) & ~size_t(255)));
    unsigned char *lane_ws = ws + ((sizeof(DevStatus) + 255) & ~size_t(255)) + bp.jobs_bytes;
    BSPS_CK(cudaMemsetAsync(bst, 0, sizeof(DevStatus), stream));
    const int nl = bp.lane_ws ? bp.lanes : 0;
    BSPS_CK(cudaEventRecord(L->fork, stream));
    for (int l = 0; l < nl; ++l) BSPS_CK(cudaStreamWaitEvent(L->s[l], L->fork, 0));
    if (!bp.jobs.empty()) BSPS_CK(launch_small(dtype, in, out, djobs, (int32_t)bp.jobs.size(), bsz, stream));
    int l = 0;
    for (size_t i = 0; i < bp.inst.size(); ++i) {
        const Instance &I = bp.inst[i];
        if (I.small) continue;
        unsigned char *w = lane_ws + (size_t)l * bp.lane_ws;
        const size_t kb = dtype == BSPS_F64 ? 8 : 4;
        const int rc = bsps_sort_keys((const unsigned char *)in + I.off * kb, (unsigned char *)out + I.off * kb, I.n,
                                      dtype, &I.prm, bsz ? bsz + bp.bbase[i] : nullptr, w, bp.lane_ws, L->s[l]);
        if (rc) return rc;
        merge_status_kernel<<<1, 32, 0, L->s[l]>>>((const DevStatus *)w, bst);
        BSPS_CK(cudaGetLastError());
        l = (l + 1) % nl;
    }
    for (int q = 0; q < nl; ++q) {
        BSPS_CK(cudaEventRecord(L->join[q], L->s[q]));
        BSPS_CK(cudaStreamWaitEvent(stream, L->join[q], 0));
    }
    return BSPS_OK;
#undef BSPS_CK
}

} // namespace bsps

using namespace bsps;

extern "C" {

int bsps_tune_default(bsps_tune *t) {
    if (!t) return BSPS_ERR_INVALID_ARG;
    std::memset(t, 0, sizeof(*t));
    for (int c = 0; c < BSPS_BATCH_CLASSES; ++c) {
        if (c <= 14) t->p[c] = c <= 9 ? 1 : 4;
        else t->p[c] = (int32_t)std::min<int64_t>(4096, std::max<int64_t>(16, ((int64_t)1 << c) >> 14));
    }
    t->small_max_log2 = 14;
    t->learned_min_log2 = 0;
    t->lanes = 8;
    return BSPS_OK;
}

int bsps_batch_bucket_base(const int64_t *h_offsets, int32_t num, const bsps_tune *t, int64_t *h_base) {
    if (!h_base || num < 0 || (num > 0 && !h_offsets) || !valid_tune(t)) return BSPS_ERR_INVALID_ARG;
    h_base[0] = 0;
    for (int32_t i = 0; i < num; ++i) {
        const int64_t n = h_offsets[i + 1] - h_offsets[i];
        if (n < 0) return BSPS_ERR_INVALID_ARG;
        h_base[i + 1] = h_base[i] + t->p[std::min(size_class(n), BSPS_BATCH_CLASSES - 1)];
    }
    return BSPS_OK;
}

int bsps_batch_workspace_size(const int64_t *h_offsets, int32_t num, int32_t dtype, const bsps_params *prm,
                              const bsps_tune *t, size_t *bytes) {
    if (!bytes) return BSPS_ERR_INVALID_ARG;
    BatchPlan bp;
    const int rc = make_batch_plan(h_offsets, num, dtype, prm, t, bp);
    if (rc) return rc;
    *bytes = bp.total;
    return BSPS_OK;
}

int bsps_sort_batched(const void *d_keys_in, void *d_keys_out, const int64_t *h_offsets, int32_t num,
                      int32_t dtype, const bsps_params *prm, const bsps_tune *t, int64_t *d_bucket_sizes,
                      void *d_ws, size_t ws_bytes, void *stream) {
    BatchPlan bp;
    int rc = make_batch_plan(h_offsets, num, dtype, prm, t, bp);
    if (rc) return rc;
    if (!d_ws || ws_bytes < bp.total) return BSPS_ERR_WORKSPACE_TOO_SMALL;
    if (((uintptr_t)d_ws & 255) != 0) return BSPS_ERR_INVALID_ARG;
    const int64_t nkeys = num > 0 ? h_offsets[num] : 0;
    if (nkeys > 0 && (!d_keys_in || !d_keys_out || d_keys_in == d_keys_out)) return BSPS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *ws = (unsigned char *)d_ws;
    // under a caller's capture the table upload below would become a graph
    // node reading host memory this call does not keep
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return BSPS_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return BSPS_ERR_CAPTURE;
    std::lock_guard<std::mutex> lock(g_mu);
    LaneSet *L = nullptr;
    if ((rc = lanes_for_device(L))) return rc;
    // the on-chip instances' table, uploaded on every call (from pageable
    // memory: the copy has read it when cudaMemcpyAsync returns)
    if (!bp.jobs.empty() &&
        cudaMemcpyAsync(ws + ((sizeof(DevStatus) + 255) & ~size_t(255)), bp.jobs.data(),
                        bp.jobs.size() * sizeof(SmallJob), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return BSPS_ERR_CUDA;

    // graph key: every argument the recorded work depends on
    std::vector<unsigned char> key;
    auto put = [&](const void *p, size_t b) {
        const unsigned char *c = (const unsigned char *)p;
        key.insert(key.end(), c, c + b);
    };
    put(&d_keys_in, sizeof(void *));
    put(&d_keys_out, sizeof(void *));
    put(&d_bucket_sizes, sizeof(void *));
    put(&d_ws, sizeof(void *));
    put(&num, sizeof(num));
    put(&dtype, sizeof(dtype));
    put(prm, sizeof(*prm));
    put(t, sizeof(*t));
    if (num > 0) put(h_offsets, sizeof(int64_t) * (size_t)(num + 1));
    int dev = 0;
    cudaGetDevice(&dev);
    GraphCache &G = g_graph[dev & 63];
    if (!G.exec || G.key != key) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
        G.key.clear();
        // recorded from a private stream, so that any caller stream (the
        // legacy default stream included) can launch the graph
        if (cudaStreamBeginCapture(L->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BSPS_ERR_CUDA;
        rc = enqueue_batch(bp, d_keys_in, d_keys_out, dtype, d_bucket_sizes, ws, L->origin, L);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(L->origin, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess || !g) return BSPS_ERR_CUDA;
        const cudaError_t ei = cudaGraphInstantiate(&G.exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            G.exec = nullptr;
            return BSPS_ERR_CUDA;
        }
        G.key = key;
    }
    return cudaGraphLaunch(G.exec, st) == cudaSuccess ? BSPS_OK : BSPS_ERR_CUDA;
}

// ---- autotuner ----
// Batch used to time size class c: enough instances of 2^c keys to fill the
// GPU, at most 2^24 keys in all.
static int tune_count(int c) { return (int)std::max<int64_t>(4, std::min<int64_t>(256, ((int64_t)1 << 24) >> c)); }

__global__ void tune_keys_kernel(uint32_t *k, int64_t words, uint64_t seed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i * 4 >= words) return;
    uint64_t c[4] = {(uint64_t)i, 0, 0, 0};
    philox4x64_10(c, seed, 7);
    for (int w = 0; w < 4 && i * 4 + w < words; ++w) k[i * 4 + w] = (uint32_t)c[w];
}

int bsps_autotune_workspace_size(int32_t dtype, const bsps_params *prm, int32_t max_log2, size_t *bytes) {
    if (!bytes || !prm || max_log2 < 8 || max_log2 > 24) return BSPS_ERR_INVALID_ARG;
    const size_t kb = dtype == BSPS_F64 ? 8 : 4;
    size_t need = 0;
    std::vector<int64_t> off;
    for (int c = 8; c <= max_log2; ++c) {
        const int cnt = tune_count(c);
        off.assign(cnt + 1, 0);
        for (int i = 0; i < cnt; ++i) off[i + 1] = off[i] + ((int64_t)1 << c);
        bsps_tune t;
        bsps_tune_default(&t);
        t.small_max_log2 = -1;
        for (int32_t pc : {16, 64, 256, 1024, 4096}) {
            if (((int64_t)pc << 4) > ((int64_t)1 << c)) continue;
            t.p[c] = pc;
            size_t w = 0;
            const int rc = bsps_batch_workspace_size(off.data(), cnt, dtype, prm, &t, &w);
            if (rc) return rc;
            need = std::max(need, w);
        }
    }
    size_t keys_max = 0;
    for (int c = 8; c <= max_log2; ++c) keys_max = std::max(keys_max, ((size_t)tune_count(c) << c) * kb);
    *bytes = need + 2 * ((keys_max + 255) & ~size_t(255)) + 4096;
    return BSPS_OK;
}

int bsps_autotune_batched(int32_t dtype, const bsps_params *prm, int32_t max_log2, bsps_tune *t, void *d_ws,
                          size_t ws_bytes, void *stream) {
    if (!t || !prm || max_log2 < 8 || max_log2 > 24 || t->lanes < 1 || t->lanes > kLanesMax) return BSPS_ERR_INVALID_ARG;
    size_t need = 0;
    int rc = bsps_autotune_workspace_size(dtype, prm, max_log2, &need);
    if (rc) return rc;
    if (!d_ws || ws_bytes < need) return BSPS_ERR_WORKSPACE_TOO_SMALL;
    const size_t kb = dtype == BSPS_F64 ? 8 : 4;
    cudaStream_t st = (cudaStream_t)stream;
    size_t keys_max = 0;
    for (int c = 8; c <= max_log2; ++c) keys_max = std::max(keys_max, ((size_t)tune_count(c) << c) * kb);
    keys_max = (keys_max + 255) & ~size_t(255);
    unsigned char *kin = (unsigned char *)d_ws, *kout = kin + keys_max, *bws = kout + keys_max;
    const size_t bws_bytes = ws_bytes - 2 * keys_max;
    const int64_t words = (int64_t)(keys_max / 4);
    tune_keys_kernel<<<(unsigned)((words / 4 + 255) / 256 + 1), 256, 0, st>>>((uint32_t *)kin, words, prm->seed);
    if (cudaGetLastError() != cudaSuccess) return BSPS_ERR_CUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BSPS_ERR_CUDA;
    const bool onchip_ok = dtype != BSPS_F64 && prm->sampling == BSPS_RANDOM;
    int small_max = -1;
    bool small_run = true;
    std::vector<int64_t> off;
    for (int c = 8; c <= max_log2; ++c) {
        const int cnt = tune_count(c);
        off.assign(cnt + 1, 0);
        for (int i = 0; i < cnt; ++i) off[i + 1] = off[i] + ((int64_t)1 << c);
        float best = 1e30f;
        int best_p = t->p[c];
        bool best_chip = false;
        for (int chip = 0; chip <= 1; ++chip) {
            if (chip && !(onchip_ok && c <= 14)) continue;
            std::vector<int32_t> cands = chip ? std::vector<int32_t>{1, 2, 4, 8, 16}
                                              : std::vector<int32_t>{16, 64, 256, 1024, 4096};
            for (int32_t pc : cands) {
                if (!chip && ((int64_t)pc << 4) > ((int64_t)1 << c)) continue;
                bsps_tune tt = *t;
                tt.p[c] = pc;
                tt.small_max_log2 = chip ? 14 : -1;
                tt.learned_min_log2 = 0;
                if (chip) {  // the on-chip form must take every instance of the class
                    bsps_plan pl;
                    bsps_params q = *prm;
                    q.p = pc;
                    if (bsps_get_plan((int64_t)1 << c, dtype, &q, 0, &pl) || pl.sample_size > kSampleMax) continue;
                }
                size_t w = 0;
                if (bsps_batch_workspace_size(off.data(), cnt, dtype, prm, &tt, &w) || w > bws_bytes) continue;
                float ms[3];
                bool ok = true;
                for (int r = -1; r < 3 && ok; ++r) {  // one untimed call records the graph
                    if (r >= 0 && cudaEventRecord(e0, st) != cudaSuccess) ok = false;
                    if (ok && bsps_sort_batched(kin, kout, off.data(), cnt, dtype, prm, &tt, nullptr, bws, bws_bytes, st))
                        ok = false;
                    if (ok && r >= 0) {
                        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms[r], e0, e1) != cudaSuccess)
                            ok = false;
                    }
                }
                if (!ok) continue;
                std::sort(ms, ms + 3);
                if (ms[1] < best) {
                    best = ms[1];
                    best_p = pc;
                    best_chip = chip != 0;
                }
            }
        }
        t->p[c] = best_p;
        if (small_run && best_chip) small_max = c;
        else small_run = false;
    }
    // classes below the first timed one behave like it
    for (int c = 0; c < 8; ++c) t->p[c] = small_max >= 8 ? 1 : t->p[8];
    if (small_max >= 8) small_max = std::max(small_max, 7);
    t->small_max_log2 = small_max;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cudaStreamSynchronize(st) == cudaSuccess ? BSPS_OK : BSPS_ERR_CUDA;
}

} // extern "C"
