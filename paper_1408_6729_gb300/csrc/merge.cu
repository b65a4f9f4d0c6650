// merge.cu -- the end of Sort_Det_BSP on the sorted blocks (Fig. 1 steps 9-12).
//
// The blocks sorted for the regular sample (Fig. 1 step 3) are kept in HBM.
// Step 9: every splitter is located in every sorted block (the partition
// c[k][i] = number of records of block k preceding S_i), which also gives the
// bucket sizes.  Step 11, the route, then moves each bucket's segments
// [c[k][i], c[k][i+1]) in block order, contiguous runs with no per-key
// classification, either into the bucket's region for the bucket sort
// (segment_copy_kernel) or -- the merge final step -- straight into the
// cluster that merges them stably, ties going to the earlier block (step 12,
// Sec. 5.1.1), and writes the bucket to its place in the output.
#include "kernels.cuh"
#include "segsort_keys.cuh"

namespace bsps {

constexpr int kMergeThreads = 512;
constexpr int kMergeItems = 31;                             // outputs per thread per merge round (at most)
constexpr int kMergeCap = kMergeThreads * kMergeItems;     // keys one CTA holds
constexpr int kMergeRunsMax = 8192;                         // blocks R (segment offsets in shared memory)
constexpr int kPartWarps = 16;

__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t key_of_phi32(int dtype, uint32_t v) {
    if (dtype == BSPS_I32) return KeyTraits<BSPS_I32>::inv(v);
    if (dtype == BSPS_F32) return KeyTraits<BSPS_F32>::inv(v);
    return v;
}

// ---------------------------------------------------------------------------
// Step 9, the partition.  Lane l of every warp owns block k = 32*blockIdx.x + l
// and the warp a contiguous range of splitters.  Block k's own sample records
// are its sorted positions j*x - 1 (j = 1..s), so the number j of them that
// precede S_i places c[k][i] in [j*x, (j+1)*x - 1]; j only grows with i, so
// the lane gallops forward through its sample records alongside the splitters.  Inside that
// window of x - 1 keys a binary search decides; a key of block k equal to S_i
// precedes it exactly when k is below S_i's block (Sec. 5.1.1: tags order
// blocks first), and S_i's own block has c = (j+1)*x - 1, the splitter's own
// sorted position.  A pad splitter follows every key.  Without duplicate
// handling the comparisons use the key value alone.  Rows 0 and p hold 0 and
// the block's key count (and the blocks' first and last keys give the
// smallest and largest key, the outer bounds of the first and last bucket).  The bucket sizes come out as differences of row
// sums: size_i = sum_k c[k][i+1] - sum_k c[k][i].  The splitters may be the
// sub-bucket splitters (any sample records): p below is their number plus one.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPartWarps * 32)
merge_partition_kernel(const uint32_t *__restrict__ runs, const uint32_t *__restrict__ rs_phi,
                       const uint32_t *__restrict__ rs_tag, const uint32_t *__restrict__ vphi,
                       const uint32_t *__restrict__ vtag, int64_t n, int64_t p, int64_t R, int64_t m, int64_t s,
                       int64_t x, int dup_off, uint32_t *__restrict__ part, uint32_t *__restrict__ cursor,
                       DevStatus *st) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * 32 + lane;
    const bool live = k < R;
    const int64_t lo = k * m;
    const int64_t len = live && lo < n ? imin64(m, n - lo) : 0;
    auto warp_sum = [](uint32_t v) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    if (blockIdx.y == 0 && warp == 0) {
        if (live) {
            part[k] = 0;
            part[p * R + k] = (uint32_t)len;
        }
        const uint32_t tot = warp_sum((uint32_t)len);
        if (lane == 0) atomicAdd(&cursor[p - 1], tot);
        // the smallest and the largest key (bounds of the first and last
        // bucket for the bucket sort): the blocks' first and last keys
        uint32_t mn = 0xffffffffu, mx = 0u;
        if (len > 0) {
            mn = runs[lo];
            mx = runs[lo + len - 1];
        }
        mn = __reduce_min_sync(0xffffffffu, mn);
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0 && tot) {
            atomicMax(&st->ext_min_inv, ~(unsigned long long)mn);
            atomicMax(&st->ext_max, (unsigned long long)mx);
        }
    }
    const int64_t rows = p - 1;
    const int64_t nw = (int64_t)gridDim.y * kPartWarps;
    const int64_t w = (int64_t)blockIdx.y * kPartWarps + warp;
    const int64_t i0 = 1 + rows * w / nw, i1 = 1 + rows * (w + 1) / nw;
    if (i0 >= i1) return;  // the whole warp (no block-wide synchronisation follows)
    const uint32_t *sp = rs_phi + (live ? k * s : 0), *stg = rs_tag + (live ? k * s : 0);
    const uint32_t un = (uint32_t)n;
    // sample record j (0-indexed) of block k precedes the record (ph, tg)
    auto before = [&](int64_t j, uint32_t ph, uint32_t tg) {
        const uint32_t a = sp[j], b = stg[j];
        if (dup_off) {
            const bool rpad = b >= un, spad = tg >= un;
            return rpad != spad ? spad : a < ph;
        }
        return a < ph || (a == ph && b < tg);
    };
    int64_t j = 0;
    if (live) {
        const uint32_t ph = vphi[i0 - 1], tg = vtag[i0 - 1];
        int64_t hi = s;
        while (j < hi) {
            const int64_t mid = (j + hi) >> 1;
            if (before(mid, ph, tg)) j = mid + 1;
            else hi = mid;
        }
    }
    for (int64_t i = i0; i < i1; ++i) {
        const uint32_t ph = vphi[i - 1], tg = vtag[i - 1];
        uint32_t c = 0;
        if (live) {
            // advance j past this block's records preceding S_i: galloping,
            // since with many equal keys one splitter can pass hundreds (and
            // the lanes of a warp pass them at different splitters)
            if (j < s && before(j, ph, tg)) {
                int64_t step = 1, hi = j + 1;  // records below hi precede S_i
                while (hi < s && before(hi, ph, tg)) {
                    j = hi;
                    step <<= 1;
                    hi = imin64(s, j + step);
                }
                int64_t lo = j + 1;  // the first record not preceding S_i lies in [lo, hi]
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (before(mid, ph, tg)) lo = mid + 1;
                    else hi = mid;
                }
                j = lo;
            }
            if (tg >= un) {
                c = (uint32_t)len;  // a pad splitter follows every key
            } else {
                const int64_t w0 = j * x;
                const int64_t ks = (int64_t)(tg / (uint32_t)m);
                if (!dup_off && ks == k) {
                    c = (uint32_t)(w0 + x - 1);
                } else {
                    const bool eq_before = !dup_off && k < ks;
                    int64_t a = w0, b = imin64(w0 + x - 1, len);
                    while (a < b) {
                        const int64_t mid = (a + b) >> 1;
                        const uint32_t v = runs[lo + mid];
                        if (v < ph || (v == ph && eq_before)) a = mid + 1;
                        else b = mid;
                    }
                    c = (uint32_t)a;
                }
                c = min(c, (uint32_t)len);
            }
            part[i * R + k] = c;
        }
        const uint32_t tot = warp_sum(c);
        if (lane == 0 && tot) {
            atomicAdd(&cursor[i - 1], tot);
            atomicSub(&cursor[i], tot);
        }
    }
}

// ---------------------------------------------------------------------------
// Steps 10-12 on one cluster of CL CTAs per bucket.  The bucket's N keys are
// cut into CL equal position ranges, one per CTA.  Each CTA gathers its range
// from the sorted blocks (segment by segment, in block order) into shared
// memory; the pieces are sorted runs.  Bottom-up rounds then merge adjacent
// pairs of runs, first the CTA's own pieces, then across the cluster (runs of
// 1, 2, 4 CTAs, read through distributed shared memory).  In one round every
// thread produces up to kMergeItems consecutive outputs: it finds its place on
// its pair's merge path by binary search and then merges sequentially, taking
// the earlier run's key on ties -- the stable merge, in which a key of an
// earlier block precedes an equal key of a later one.  The outputs of a round
// are held in registers until every thread has read its inputs, then written
// back in place.  Finally each CTA writes its range of the merged bucket.
// ---------------------------------------------------------------------------
struct MergeArgs {
    const uint32_t *runs;      // sorted blocks, phi; block k at k*m
    const uint32_t *runs_val;  // payloads in the same order (pairs)
    const uint32_t *part;      // (p+1) x R partition
    const uint32_t *vsize;     // bucket sizes
    const uint64_t *voff;      // bucket output offsets
    uint32_t *out_keys;
    uint32_t *out_vals;
    int64_t R, m;
    int dtype, cl;
    DevStatus *st;
};

template <bool PAIRS> constexpr size_t merge_smem_bytes(int64_t R) {
    return (size_t)(PAIRS ? 2 : 1) * kMergeCap * 4 + (size_t)(R + 1) * 4;
}

// One merge round over runs whose boundaries are bnd(0) <= ... <= bnd(nr):
// pair j merges runs [2jw, 2jw + w) with [2jw + w, 2jw + 2w).  This thread
// produces the outputs at positions [o0, o1) into rk / rv.
template <bool PAIRS, typename Bnd, typename LdK, typename LdV>
__device__ __forceinline__ void merge_round(int nr, int w, uint32_t o0, uint32_t o1, Bnd bnd, LdK ldk, LdV ldv,
                                            uint32_t (&rk)[kMergeItems], uint32_t (&rv)[kMergeItems]) {
    if (o0 >= o1) return;
    const int npairs = (nr + 2 * w - 1) / (2 * w);
    int jl = 0, jh = npairs - 1;  // the last pair starting at or before o0 holds o0
    while (jl < jh) {
        const int mid = (jl + jh + 1) >> 1;
        if (bnd(2 * mid * w) <= o0) jl = mid;
        else jh = mid - 1;
    }
    int j = jl;
    uint32_t a0 = bnd(2 * j * w), a1 = bnd(min(2 * j * w + w, nr)), b1 = bnd(min(2 * j * w + 2 * w, nr));
    // place on the merge path: outputs before o0 take lo keys of A
    const uint32_t d = o0 - a0, la = a1 - a0, lb = b1 - a1;
    uint32_t lo = d > lb ? d - lb : 0, hi = min(d, la);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (ldk(a0 + mid) <= ldk(a1 + d - 1 - mid)) lo = mid + 1;
        else hi = mid;
    }
    uint32_t ia = a0 + lo, ib = a1 + d - lo;
    uint32_t ka = ia < a1 ? ldk(ia) : 0u, kb = ib < b1 ? ldk(ib) : 0u;
#pragma unroll
    for (int e = 0; e < kMergeItems; ++e) {
        const uint32_t o = o0 + e;
        if (o < o1) {
            while (o == b1) {  // this pair is done: the next one (empty pairs skipped)
                ++j;
                a0 = bnd(2 * j * w);
                a1 = bnd(min(2 * j * w + w, nr));
                b1 = bnd(min(2 * j * w + 2 * w, nr));
                ia = a0;
                ib = a1;
                ka = ia < a1 ? ldk(ia) : 0u;
                kb = ib < b1 ? ldk(ib) : 0u;
            }
            const bool ta = ib >= b1 || (ia < a1 && ka <= kb);
            rk[e] = ta ? ka : kb;
            if constexpr (PAIRS) rv[e] = ldv(ta ? ia : ib);
            if (ta) {
                ++ia;
                ka = ia < a1 ? ldk(ia) : 0u;
            } else {
                ++ib;
                kb = ib < b1 ? ldk(ib) : 0u;
            }
        }
    }
}

template <bool PAIRS>
__global__ void __launch_bounds__(kMergeThreads, PAIRS ? 1 : 2) merge_bucket_kernel(const MergeArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *vals = keys + kMergeCap;
    uint32_t *soff = keys + (PAIRS ? 2 : 1) * kMergeCap;
    __shared__ uint32_t Pb[9], kbase[8], vbase[8], tmp[40];
    const int tid = threadIdx.x;
    const int CL = a.cl;
    const int c = (int)(blockIdx.x % CL);
    const int64_t bi = blockIdx.x / CL;
    const int64_t R = a.R;
    const uint32_t N = a.vsize[bi];
    if (N == 0) return;  // every CTA of the cluster returns
    if (N > (uint32_t)CL * kMergeCap) {
        if (tid == 0 && c == 0) {
            atomicExch(&a.st->overflow, 1);
            set_error(a.st, BSPS_ERR_BUCKET_OVERFLOW);
        }
        return;
    }
    const uint32_t *rowa = a.part + bi * R, *rowb = a.part + (bi + 1) * R;
    for (int64_t k = tid; k < R; k += kMergeThreads) soff[k] = rowb[k] >= rowa[k] ? rowb[k] - rowa[k] : 0u;
    if (tid <= CL) Pb[tid] = (uint32_t)((uint64_t)N * tid / CL);
    if (tid < CL) {
        kbase[tid] = cluster_addr((uint32_t)__cvta_generic_to_shared(keys), tid);
        vbase[tid] = cluster_addr((uint32_t)__cvta_generic_to_shared(vals), tid);
    }
    __syncthreads();
    const uint32_t total = block_excl_scan_smem<kMergeThreads>(soff, (int)R, tmp);
    if (total != N) {  // the segments do not add up to the bucket (never expected): report, touch nothing
        if (tid == 0 && c == 0) {
            atomicExch(&a.st->overflow, 1);
            set_error(a.st, BSPS_ERR_BUCKET_OVERFLOW);
        }
        return;
    }
    if (tid == 0) soff[R] = N;
    __syncthreads();
    const uint32_t P0 = Pb[c], P1 = Pb[c + 1], cnt = P1 - P0;
    // consecutive outputs per thread, odd: lane t's e-th item sits at t*E + e,
    // so the 32 lanes of a warp touch 32 different shared-memory banks
    const uint32_t E = ((cnt + kMergeThreads - 1) / kMergeThreads) | 1u;
    const uint32_t o0 = min(cnt, tid * E), o1 = min(cnt, o0 + E);
    // the segment holding bucket position q: the last k with soff[k] <= q
    auto seg_of = [&](uint32_t q) {
        int64_t l = 0, h = R - 1;
        while (l < h) {
            const int64_t mid = (l + h + 1) >> 1;
            if (soff[mid] <= q) l = mid;
            else h = mid - 1;
        }
        return l;
    };
    uint32_t rk[kMergeItems], rv[kMergeItems];
    // ---- gather the CTA's range, segment by segment (Fig. 1 step 11) ----
    if (o0 < o1) {
        int64_t kk = seg_of(P0 + o0);
        uint32_t send = soff[kk + 1], sbase = soff[kk], sstart = rowa[kk];
#pragma unroll
        for (int e = 0; e < kMergeItems; ++e) {
            const uint32_t o = o0 + e;
            if (o < o1) {
                const uint32_t q = P0 + o;
                if (q >= send) {
                    do {
                        ++kk;
                        send = soff[kk + 1];
                    } while (q >= send);
                    sbase = soff[kk];
                    sstart = rowa[kk];
                }
                const int64_t idx = kk * a.m + sstart + (q - sbase);
                rk[e] = a.runs[idx];
                if constexpr (PAIRS) rv[e] = a.runs_val[idx];
            }
        }
#pragma unroll
        for (int e = 0; e < kMergeItems; ++e)
            if (o0 + e < o1) {
                keys[o0 + e] = rk[e];
                if constexpr (PAIRS) vals[o0 + e] = rv[e];
            }
    }
    __syncthreads();
    auto write_back = [&]() {
#pragma unroll
        for (int e = 0; e < kMergeItems; ++e)
            if (o0 + e < o1) {
                keys[o0 + e] = rk[e];
                if constexpr (PAIRS) vals[o0 + e] = rv[e];
            }
    };
    // ---- the CTA's own pieces: runs between segment boundaries ----
    if (cnt > 0) {
        const int64_t kl = seg_of(P0), kh = seg_of(P1 - 1);
        const int nr = (int)(kh - kl + 1);
        auto bnd = [&](int r) { return min(max(soff[kl + r], P0), P1) - P0; };
        auto ldk = [&](uint32_t q) { return keys[q]; };
        auto ldv = [&](uint32_t q) { return vals[q]; };
        for (int w = 1; w < nr; w *= 2) {
            merge_round<PAIRS>(nr, w, o0, o1, bnd, ldk, ldv, rk, rv);
            __syncthreads();
            write_back();
            __syncthreads();
        }
    }
    // ---- across the cluster: runs of 1, 2, 4 CTAs ----
    if (CL > 1) {
        auto cluster = cg::this_cluster();
        cluster.sync();  // every CTA's range is merged
        auto owner = [&](uint32_t q) {  // the last CTA whose range starts at or before q
            int l = 0, h = CL - 1;
            while (l < h) {
                const int mid = (l + h + 1) >> 1;
                if (Pb[mid] <= q) l = mid;
                else h = mid - 1;
            }
            return l;
        };
        auto ldk = [&](uint32_t q) {
            if (q >= P0 && q < P1) return keys[q - P0];
            const int r = owner(q);
            return ld_cluster_u32(kbase[r] + 4u * (q - Pb[r]));
        };
        auto ldv = [&](uint32_t q) {
            if (q >= P0 && q < P1) return vals[q - P0];
            const int r = owner(q);
            return ld_cluster_u32(vbase[r] + 4u * (q - Pb[r]));
        };
        auto bnd = [&](int r) { return Pb[r]; };
        for (int w = 1; w < CL; w *= 2) {
            merge_round<PAIRS>(CL, w, P0 + o0, P0 + o1, bnd, ldk, ldv, rk, rv);
            cluster.sync();  // every CTA has read what it needs
            write_back();
            if (2 * w < CL) cluster.sync();  // written before the next round reads
        }
        __syncthreads();
    }
    // ---- write the CTA's range of the bucket ----
    uint32_t *ok = a.out_keys + a.voff[bi] + P0;
    for (uint32_t o = tid; o < cnt; o += kMergeThreads) ok[o] = key_of_phi32(a.dtype, keys[o]);
    if constexpr (PAIRS) {
        uint32_t *ov = a.out_vals + a.voff[bi] + P0;
        for (uint32_t o = tid; o < cnt; o += kMergeThreads) ov[o] = vals[o];
    }
}

// ---------------------------------------------------------------------------
// Step 11 as a copy: sub-bucket v's segments, in block order, into its region
// (the bucket sort then reads the region as the classification route leaves
// it: in input order for equal keys).  The segment offsets inside the bucket
// (a scan over the blocks) and the segments' starts stay in shared memory;
// each warp copies runs of 32 * kSegItems consecutive positions, every lane
// finding its positions' segments by walking forward from the run's first.
// ---------------------------------------------------------------------------
constexpr int kSegThreads = 512, kSegItems = 8;

struct SegCopyArgs {
    const uint32_t *runs, *runs_val, *part, *vsize, *vphi;
    const uint64_t *voff;
    int64_t R, m, cap, P;
    uint32_t *reg_keys, *reg_vals, *out_keys, *out_vals;
    int dtype;
    DevStatus *st;
};

template <bool PAIRS>
__global__ void __launch_bounds__(kSegThreads) segment_copy_kernel(const SegCopyArgs a) {
    extern __shared__ __align__(16) uint32_t ssm[];
    const int64_t R = a.R, m = a.m, cap = a.cap;
    const uint32_t *__restrict__ runs = a.runs;
    const uint32_t *__restrict__ runs_val = a.runs_val;
    const uint32_t *part = a.part;
    DevStatus *st = a.st;
    uint32_t *soff = ssm, *sst = ssm + R + 1;
    __shared__ uint32_t tmp[40];
    const int64_t v = blockIdx.x;
    const uint32_t N = a.vsize[v];
    if (N == 0 || N > cap) return;  // an overflow is already reported
    // a sub-bucket between two equal splitters holds one key value, its
    // segments in block order are its sorted order: keys only, the bucket
    // sort writes it without reading; with payloads they go straight to the
    // output here
    const bool one = v > 0 && v < a.P - 1 && a.vphi[v - 1] == a.vphi[v];
    if (one && !PAIRS) return;
    const uint32_t *rowa = part + v * R, *rowb = part + (v + 1) * R;
    for (int64_t k = threadIdx.x; k < R; k += kSegThreads) {
        const uint32_t x0 = rowa[k], x1 = rowb[k];
        sst[k] = x0;
        soff[k] = x1 >= x0 ? x1 - x0 : 0u;
    }
    __syncthreads();
    const uint32_t total = block_excl_scan_smem<kSegThreads>(soff, (int)R, tmp);
    if (total != N) {  // the segments do not add up to the bucket (never expected): report, touch nothing
        if (threadIdx.x == 0) {
            atomicExch(&st->overflow, 1);
            set_error(st, BSPS_ERR_BUCKET_OVERFLOW);
        }
        return;
    }
    if (threadIdx.x == 0) soff[R] = N;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *dk = one ? a.out_keys + a.voff[v] : a.reg_keys + v * cap;
    uint32_t *dv = PAIRS ? (one ? a.out_vals + a.voff[v] : a.reg_vals + v * cap) : nullptr;
    const uint32_t key1 = one ? key_of_phi32(a.dtype, a.vphi[v]) : 0u;
    constexpr uint32_t RUN = 32 * kSegItems;
    for (uint32_t base = warp * RUN; base < N; base += (kSegThreads / 32) * RUN) {
        int64_t l = 0, h = R - 1;  // the last segment starting at or before base
        while (l < h) {
            const int64_t mid = (l + h + 1) >> 1;
            if (soff[mid] <= base) l = mid;
            else h = mid - 1;
        }
        int64_t seg = l;
        uint32_t kk[kSegItems], vv[kSegItems];
#pragma unroll
        for (int u = 0; u < kSegItems; ++u) {
            const uint32_t q = base + u * 32 + lane;
            if (q < N) {
                while (q >= soff[seg + 1]) ++seg;
                const int64_t src = seg * m + sst[seg] + (q - soff[seg]);
                kk[u] = runs[src];
                if constexpr (PAIRS) vv[u] = runs_val[src];
            }
        }
#pragma unroll
        for (int u = 0; u < kSegItems; ++u) {
            const uint32_t q = base + u * 32 + lane;
            if (q < N) {
                dk[q] = one ? key1 : kk[u];
                if constexpr (PAIRS) dv[q] = vv[u];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int merge_cluster(const Plan &pl) {
    for (int cl = 1; cl <= 8; cl *= 2)
        if (pl.cap <= (int64_t)cl * kMergeCap) return cl;
    return 0;
}

int64_t merge_capacity(int cl) { return (int64_t)cl * kMergeCap; }

int64_t merge_runs_max() { return kMergeRunsMax; }

cudaError_t launch_merge_partition(const Ctx &c) {
    const Plan &p = c.pl;
    const int64_t rows = p.P - 1;
    int64_t gy = (rows + kPartWarps * 16 - 1) / (kPartWarps * 16);
    gy = imax64(1, imin64(gy, 65535));
    dim3 grid((unsigned)((p.R + 31) / 32), (unsigned)gy);
    merge_partition_kernel<<<grid, kPartWarps * 32, 0, c.stream>>>(
        (const uint32_t *)c.ly.runs, c.ly.rs_phi, c.ly.rs_tag, (const uint32_t *)c.ly.vphi, c.ly.vtag, p.n,
        p.P, p.R, p.m, p.s, p.x, p.dup_off, c.ly.part, c.ly.cursor, c.ly.status);
    return cudaGetLastError();
}

cudaError_t launch_segment_copy(const Ctx &c) {
    const Plan &p = c.pl;
    const size_t smem = (size_t)(2 * p.R + 1) * 4;
    auto kern = p.pairs ? segment_copy_kernel<true> : segment_copy_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SegCopyArgs a;
    a.runs = (const uint32_t *)c.ly.runs;
    a.runs_val = c.ly.runs_val;
    a.part = c.ly.part;
    a.vsize = c.ly.vsize;
    a.vphi = (const uint32_t *)c.ly.vphi;
    a.voff = c.ly.voff;
    a.R = p.R;
    a.m = p.m;
    a.cap = p.cap;
    a.P = p.P;
    a.reg_keys = (uint32_t *)c.ly.reg_keys;
    a.reg_vals = c.ly.reg_vals;
    a.out_keys = (uint32_t *)c.keys_out;
    a.out_vals = c.vals_out;
    a.dtype = p.dtype;
    a.st = c.ly.status;
    kern<<<(unsigned)p.P, kSegThreads, smem, c.stream>>>(a);
    return cudaGetLastError();
}

template <bool PAIRS> static cudaError_t launch_merge_buckets_t(const Ctx &c) {
    const Plan &p = c.pl;
    MergeArgs a;
    a.runs = (const uint32_t *)c.ly.runs;
    a.runs_val = c.ly.runs_val;
    a.part = c.ly.part;
    a.vsize = c.ly.vsize;
    a.voff = c.ly.voff;
    a.out_keys = (uint32_t *)c.keys_out;
    a.out_vals = c.vals_out;
    a.R = p.R;
    a.m = p.m;
    a.dtype = p.dtype;
    a.cl = p.bucket_cl;
    a.st = c.ly.status;
    const size_t smem = merge_smem_bytes<PAIRS>(p.R);
    auto kern = merge_bucket_kernel<PAIRS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(p.p * p.bucket_cl));
    cfg.blockDim = dim3(kMergeThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.bucket_cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

cudaError_t launch_merge_buckets(const Ctx &c) {
    return c.pl.pairs ? launch_merge_buckets_t<true>(c) : launch_merge_buckets_t<false>(c);
}

} // namespace bsps
