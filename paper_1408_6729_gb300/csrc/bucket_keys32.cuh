// bucket_keys32.cuh -- keys-only sort of one sub-bucket of 32-bit keys on a
// thread-block cluster (Fig. 2 step 12), laid out for few instructions per
// key.  Equal keys cannot be told apart, so no ranking needs to be stable.
//
// A cluster of CL CTAs (512 threads, two CTAs per SM) sorts one sub-bucket
// whose keys lie in [lo, hi] (bounds from the splitters around it):
//   1. each CTA loads its share of the region into shared memory by one bulk
//      asynchronous copy, reads it into registers (16-byte shared loads) and
//      ranks every key in its split bin (the top 8 bits of key - lo) with
//      one shared-memory atomic; bin and rank stay packed in one register;
//   2. the keys are grouped by split bin in a local stage;
//   3. every CTA reads the cluster's bin counts through distributed shared
//      memory and derives the same layout: where each bin starts in the
//      output, and which CTA owns it (bins go to CTAs in output order, about
//      a CL-th of the keys each);
//   4. each CTA copies its stage, run by run, to the owners' receive buffers
//      (st.shared::cluster at a precomputed address per bin);
//   5. each owner sorts what it received by one counting pass: bins of one
//      value when the owned range is below 2^12 values; up to 3600 bins of 32
//      values, where three occupancy masks per bin (values seen once, twice,
//      three times) place every key whose value occurs at most three times
//      by popcounts alone; for wider ranges up to 8192 bins, where keys
//      sharing a bin (and keys of bins where a value occurs four times) are
//      placed by comparison;
//   6. the sorted keys are written to the output range the owner's bins
//      occupy, which is contiguous.
// Only when some owner would receive more keys than it holds does the
// cluster look for split bins of a single key value; those are written out
// directly by the CTAs holding them and owned by nobody.  If that does not
// help, or a count bin needing comparisons is longer than kBinMax, the
// sub-bucket is given back (run returns false) to the stable cluster sort.
#pragma once

#include "radix.cuh"
#include "segsort_keys.cuh"

namespace bsps {

template <int CL>
struct BucketKeys32 {
    using K = uint32_t;
    static constexpr int T = 512;
    static constexpr int ITEMS = 20;
    static constexpr int CAP = T * ITEMS;            // keys one CTA holds
    static constexpr int R = 256;                    // split bins
    static constexpr int kMaxBins = 8192;            // count bins
    static constexpr int kMaskBins = 3600;           // count bins with occupancy masks (32 values each)
    static constexpr uint32_t kBinMax = 64;          // longest count bin ordered by comparison
    static constexpr uint32_t kListMax = T;          // keys of masked bins placed by comparison
    static constexpr uint32_t kRep = 0x80000000u;    // bin start flag: a value of the bin repeats
    static constexpr uint32_t kLater = 0x40000000u;  // ... and some value occurs four times or more
    static constexpr uint32_t kStart = 0x3fffffffu;
    static_assert(ITEMS % 4 == 0, "whole 16-byte loads per thread");

    struct Smem {
        uint32_t cnt[R];      // my keys per split bin (read by the other CTAs)
        uint32_t lbase[R];    // first stage slot of split bin d
        uint32_t tot[R];      // keys of split bin d in the cluster
        uint32_t pre[R];      // keys of bin d held by lower-ranked CTAs
        uint32_t own[R];      // keys of bin d given to an owner (0 for flat bins)
        uint32_t raddr[R];    // stage slot j of bin d goes to shared::cluster address raddr[d] + 4j,
                              // or (odd) to output position (raddr[d] >> 1) + j
        uint32_t ostart[R];   // output position of bin d's first key within the sub-bucket
        uint32_t rpos[R];     // position of bin d's first key among the owned keys
        uint32_t odelta[R];   // received bin d: output position = odelta[d] + sorted position
        K bmin[R], bmax[R];   // smallest / largest key of my share per split bin (flat-bin pass)
        uint32_t list[kListMax];  // waiting slots of the keys the count sort places by comparison
        unsigned long long mbar;  // completion of the bulk copy of this CTA's share
        uint32_t stalled;         // the wait for that copy ran out (set to 0 by the caller)
        uint32_t orecv[CL], ofirst[CL], olast[CL], obase[CL];
        uint32_t tmp[40];
    };
    // region A: the stage, later the count scratch (histogram and three
    // occupancy masks); region B: the received keys, then the sorted keys
    static constexpr size_t kMaskOff = (size_t)kMaskBins + 4;  // words
    static constexpr size_t kWordsA = (size_t)kMaxBins + 4 > 4 * kMaskOff ? (size_t)kMaxBins + 4 : 4 * kMaskOff;
    static constexpr size_t kBytesA = kWordsA * 4 > (size_t)CAP * 4 ? kWordsA * 4 : (size_t)CAP * 4;
    static constexpr size_t kBytesB = (size_t)CAP * 4;
    static constexpr size_t kSmemHead = (sizeof(Smem) + 15) & ~size_t(15);
    static constexpr size_t smem_bytes() { return kSmemHead + kBytesA + kBytesB; }

    // register i of a thread holds local key (i / 4 * T + tid) * 4 + i % 4
    __device__ static int lidx(int i) { return ((i / 4) * T + (int)threadIdx.x) * 4 + i % 4; }
    // keys taken from shared memory: key i * T + tid
    __device__ static int slot(int i) { return i * T + (int)threadIdx.x; }

    __device__ static void load(K (&k)[ITEMS], const K *__restrict__ src, int n) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
#pragma unroll
        for (int j = 0; j < ITEMS / 4; ++j) {
            const int q = j * T + (int)threadIdx.x;
            if (q * 4 < n) {
                const uint4 w = __ldg(s4 + q);
                k[j * 4 + 0] = w.x; k[j * 4 + 1] = w.y; k[j * 4 + 2] = w.z; k[j * 4 + 3] = w.w;
            }
        }
    }

    // Exclusive scan of v[0..256) into out[0..256) by warp 0 alone (lane l
    // takes eight consecutive entries); returns the total on warp 0.
    __device__ static uint32_t warp_scan256(const uint32_t *v, uint32_t *out) {
        const int lane = threadIdx.x & 31;
        const uint4 a = *reinterpret_cast<const uint4 *>(v + lane * 8);
        const uint4 b = *reinterpret_cast<const uint4 *>(v + lane * 8 + 4);
        const uint32_t s = a.x + a.y + a.z + a.w + b.x + b.y + b.z + b.w;
        uint32_t tot;
        uint32_t run = warp_excl_scan(s, &tot);
        uint4 oa, ob;
        oa.x = run; run += a.x; oa.y = run; run += a.y; oa.z = run; run += a.z; oa.w = run; run += a.w;
        ob.x = run; run += b.x; ob.y = run; run += b.y; ob.z = run; run += b.z; ob.w = run;
        *reinterpret_cast<uint4 *>(out + lane * 8) = oa;
        *reinterpret_cast<uint4 *>(out + lane * 8 + 4) = ob;
        return tot;
    }

    // This CTA's share of the region (n keys at src, 16-byte aligned; reading
    // up to the next 16 bytes stays inside the region) into registers through
    // shared memory: one thread issues a bulk asynchronous copy (the tensor
    // memory accelerator's 1-D form) into `buf` and every thread waits on an
    // mbarrier for its completion, then reads its keys with 16-byte shared
    // loads.  The wait is bounded: when it runs out the status records
    // BSPS_ERR_DEVICE_TIMEOUT and sm.stalled is set; the sort then goes on
    // (on whatever the buffer holds, every index bounded) so that the
    // cluster's barriers stay matched, and the caller waits once more for the
    // copy (wait_staged) and gives the sub-bucket back.
    __device__ static bool wait_staged(Smem &sm, uint32_t limit) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&sm.mbar);
        uint32_t done = 0;
        for (uint32_t polls = 0; !done && polls < limit; ++polls)
            asm volatile(
                "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                : "=r"(done)
                : "r"(bar)
                : "memory");
        return done != 0;
    }
    template <typename Xf>
    __device__ static void load_staged(Smem &sm, K (&k)[ITEMS], const K *__restrict__ src, int n, K *buf,
                                       DevStatus *st, Xf xf) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&sm.mbar);
        const uint32_t bytes = (uint32_t)((n * (int)sizeof(K) + 15) & ~15);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
            if (bytes)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        (uint32_t)__cvta_generic_to_shared(buf)),
                    "l"(src), "r"(bytes), "r"(bar)
                    : "memory");
        }
        if (!__syncthreads_and(wait_staged(sm, kSpinLimit)) && threadIdx.x == 0) {
            sm.stalled = 1;
            atomicAdd(&st->timeouts, 1);
            set_error(st, BSPS_ERR_DEVICE_TIMEOUT);
        }
#pragma unroll
        for (int j = 0; j < ITEMS / 4; ++j) {
            const int q = j * T + (int)threadIdx.x;
            if (q * 4 < n) {
                const uint4 w = *reinterpret_cast<const uint4 *>(buf + q * 4);
                k[j * 4 + 0] = xf(w.x); k[j * 4 + 1] = xf(w.y); k[j * 4 + 2] = xf(w.z); k[j * 4 + 3] = xf(w.w);
            }
        }
    }

    // Bin lengths (with masks: one key per mask bit plus the counted later
    // occurrences), their exclusive scan in place, chist[nb] = total, the
    // repeat flag on every bin where some value occurs twice, and the later
    // flag where some value occurs four times or more.
    template <bool MASKS>
    __device__ static void scan_bins(uint32_t *chist, const uint32_t *m1, const uint32_t *m2, const uint32_t *m3,
                                     int nb, uint32_t *tmp) {
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        constexpr int W = T / 32;
        const int per = (nb + T - 1) / T;  // <= 16
        const int b0 = tid * per, b1 = min(nb, b0 + per);
        // bin length | flags (read twice rather than held in registers)
        auto len_of = [&](int b) {
            const uint32_t later = chist[b];
            uint32_t len = later;
            if constexpr (MASKS) {
                const uint32_t w2 = m2[b];
                len += __popc(m1[b]) + __popc(w2) + __popc(m3[b]);
                len |= (w2 ? kRep : 0u) | (later ? kLater : 0u);
            }
            return len;
        };
        uint32_t s = 0;
        for (int b = b0; b < b1; ++b) s += len_of(b) & kStart;
        uint32_t wtot;
        const uint32_t wex = warp_excl_scan(s, &wtot);
        if (lane == 31) tmp[warp] = wtot;
        __syncthreads();
        if (warp == 0) {
            const uint32_t y = lane < W ? tmp[lane] : 0u;
            uint32_t t;
            const uint32_t ye = warp_excl_scan(y, &t);
            if (lane < W) tmp[lane] = ye;
            if (lane == 0) tmp[W] = t;
        }
        __syncthreads();
        uint32_t run = tmp[warp] + wex;
        for (int b = b0; b < b1; ++b) {
            const uint32_t len = len_of(b);
            chist[b] = run | (len & ~kStart);
            run += len & kStart;
        }
        if (tid == 0) chist[nb] = tmp[W];
        __syncthreads();
    }

    // Count-bin regimes of count_sort.
    enum { kValueBins = 0, kMaskedBins = 1, kSparseBins = 2 };

    // Sorts the keys held in registers (where valid(i)), all in
    // [llo, llo + range], into out[0..n).  scr holds kWordsA words, list
    // kListMax words.  Returns false (uniformly) when the keys that need
    // comparisons are too many or sit in too long a bin.
    template <typename Valid>
    __device__ static bool count_sort(const K (&k)[ITEMS], Valid valid, K llo, K range, K *out, uint32_t *scr,
                                      uint32_t *tmp, uint32_t *list) {
        // bins of one value (range below 2^12); bins of 32 values with three
        // occupancy masks (values seen once, twice, three times) when the
        // range is at most 32 kMaskBins values; else up to kMaxBins bins of
        // about one key, placed by comparison when they hold more
        if (range < (K)4096) return count_sort_mode<kValueBins>(k, valid, llo, range, 0, out, scr, tmp, list);
        if ((range >> 5) < (K)kMaskBins) return count_sort_mode<kMaskedBins>(k, valid, llo, range, 5, out, scr, tmp, list);
        int shift = 0;
        while ((range >> shift) >= (K)kMaxBins) ++shift;
        return count_sort_mode<kSparseBins>(k, valid, llo, range, shift, out, scr, tmp, list);
    }

    template <int MODE, typename Valid>
    __device__ static bool count_sort_mode(const K (&k)[ITEMS], Valid valid, K llo, K range, int shift, K *out,
                                           uint32_t *scr, uint32_t *tmp, uint32_t *list) {
        constexpr bool MASKS = MODE == kMaskedBins;
        const int nb = (int)(range >> shift) + 1;
        uint32_t *chist = scr, *m1 = scr + kMaskOff, *m2 = m1 + kMaskOff, *m3 = m2 + kMaskOff;
        const int tid = threadIdx.x;
        __syncthreads();  // scr and out may still be read by the caller
        {
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
            for (int q = tid * 4; q < nb; q += T * 4) {
                *reinterpret_cast<uint4 *>(chist + q) = z;
                if constexpr (MASKS) {
                    *reinterpret_cast<uint4 *>(m1 + q) = z;
                    *reinterpret_cast<uint4 *>(m2 + q) = z;
                    *reinterpret_cast<uint4 *>(m3 + q) = z;
                }
            }
            if (tid == 0) tmp[38] = 0;  // keys on the comparison list
        }
        __syncthreads();
        // Per key a 16-bit word, two to a register.  Without masks it is the
        // arrival rank inside the bin.  With masks it is the occurrence of the
        // value (bits 14..15: first, second, third, later) and, for later
        // ones, their rank among the bin's later occurrences (bits 0..13),
        // which chist counts.  After placement (sparse bins): the waiting
        // slot, or 0xffff when final.
        uint32_t rp[ITEMS / 2];
        auto get = [&](int i) { return (rp[i >> 1] >> ((i & 1) * 16)) & 0xffffu; };
        auto put = [&](int i, uint32_t x) {
            const int sh = (i & 1) * 16;
            rp[i >> 1] = (rp[i >> 1] & ~(0xffffu << sh)) | (x << sh);
        };
#pragma unroll
        for (int i = 0; i < ITEMS / 2; ++i) rp[i] = 0xffffffffu;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (valid(i)) {
                const uint32_t v = k[i] - llo;
                const uint32_t bb = min(v >> shift, (uint32_t)nb - 1u);
                if constexpr (MASKS) {
                    const uint32_t bit = 1u << (v & 31u);
                    uint32_t o = 0;
                    if (atomicOr(&m1[bb], bit) & bit) {
                        o = 1u << 14;
                        if (atomicOr(&m2[bb], bit) & bit) {
                            o = 2u << 14;
                            if (atomicOr(&m3[bb], bit) & bit) o = 3u << 14 | atomicAdd(&chist[bb], 1u);
                        }
                    }
                    put(i, o);
                } else {
                    put(i, atomicAdd(&chist[bb], 1u));
                }
            }
        __syncthreads();
        scan_bins<MASKS>(chist, m1, m2, m3, nb, tmp);
        bool cmp = false;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (valid(i)) {
                const uint32_t v = k[i] - llo;
                const uint32_t bb = min(v >> shift, (uint32_t)nb - 1u);
                const uint32_t h = chist[bb], b0 = h & kStart, r = get(i);
                if constexpr (MASKS) {
                    // keys of smaller values (their first, second and third
                    // occurrences), then this key's own occurrence
                    const uint32_t below = (1u << (v & 31u)) - 1u;
                    const uint32_t w1 = m1[bb], w2 = m2[bb], w3 = m3[bb], occ = r >> 14;
                    uint32_t pos = b0 + __popc(w1 & below) + __popc(w2 & below) + __popc(w3 & below) + occ;
                    if (h & kLater) {  // some value of the bin occurs four times or more
                        const uint32_t later = r & 0x3fffu, c1 = __popc(w1);
                        if (c1 == 1) {
                            pos = b0 + (occ < 3 ? occ : 3u + later);  // one value: any distinct slot
                        } else {
                            // a distinct waiting slot, listed; the comparisons below place it
                            const uint32_t c12 = c1 + __popc(w2);
                            pos = b0 + __popc(w1 & below);
                            if (occ == 1) pos = b0 + c1 + __popc(w2 & below);
                            else if (occ == 2) pos = b0 + c12 + __popc(w3 & below);
                            else if (occ == 3) pos = b0 + c12 + __popc(w3) + later;
                            const uint32_t at = atomicAdd(&tmp[38], 1u);
                            if (at < kListMax) list[at] = pos;
                            cmp = true;
                        }
                    }
                    out[pos] = k[i];
                } else {
                    const uint32_t pos = b0 + r;
                    const bool fin = MODE == kValueBins || (chist[bb + 1] & kStart) - b0 == 1;
                    out[pos] = k[i];
                    put(i, fin ? 0xffffu : pos);
                    cmp |= !fin;
                }
            }
        if (!__syncthreads_or(cmp)) return true;
        if constexpr (MASKS) {
            // the listed keys: place = bin start + keys of the bin below the
            // key + equal keys stored before it (all of the bin's keys wait in
            // distinct slots of the bin)
            const uint32_t nl = tmp[38];
            if (nl > kListMax) return false;  // uniform
            uint32_t dst = 0xffffffffu;
            K key = 0;
            if (tid < (int)nl) {
                const uint32_t self = list[tid];
                key = out[self];
                const uint32_t bb = min((key - llo) >> shift, (uint32_t)nb - 1u);
                const uint32_t b0 = chist[bb] & kStart, b1 = chist[bb + 1] & kStart;
                dst = b0;
                for (uint32_t y = b0; y < b1; ++y) {
                    const K x = out[y];
                    dst += (x < key) | ((x == key) & (y < self));
                }
            }
            __syncthreads();
            if (dst != 0xffffffffu) out[dst] = key;
            __syncthreads();
            return true;
        } else {
            // place = bin start + keys of the bin below k + equal keys stored before it
            bool too_long = false;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (valid(i) && get(i) != 0xffffu) {
                    const uint32_t bb = min((k[i] - llo) >> shift, (uint32_t)nb - 1u);
                    const uint32_t b0 = chist[bb] & kStart, b1 = chist[bb + 1] & kStart, self = get(i);
                    if (b1 - b0 > kBinMax) {
                        too_long = true;
                    } else {
                        uint32_t pos = b0;
                        for (uint32_t y = b0; y < b1; ++y) {
                            const K x = out[y];
                            pos += (x < k[i]) | ((x == k[i]) & (y < self));
                        }
                        put(i, pos);
                    }
                }
            if (__syncthreads_or(too_long)) return false;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (valid(i) && get(i) != 0xffffu) out[get(i)] = k[i];
            __syncthreads();
            return true;
        }
    }

    // Sorts the cnt keys at src (16-byte aligned; reading up to the next
    // multiple of 4 keys stays inside the caller's region; lo <= key <= hi,
    // lo < hi) and calls emit(position, key) for each.  Returns false when
    // the sub-bucket goes to the stable sort, which rewrites every position.
    // xf maps each loaded word to the key sorted (the order-preserving phi of
    // the caller's key type; by default the words are already keys).
    struct Same {
        __device__ K operator()(K v) const { return v; }
    };
    template <typename Emit, typename Xf = Same>
    __device__ static bool run(unsigned char *smem, const K *__restrict__ src, int64_t cnt, K lo, K hi, Emit emit,
                               DevStatus *st, Xf xf = Xf()) {
        Smem &sm = *reinterpret_cast<Smem *>(smem);
        K *regA = reinterpret_cast<K *>(smem + kSmemHead);
        K *regB = reinterpret_cast<K *>(smem + kSmemHead + kBytesA);
        const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
        const int64_t share = ((cnt + CL - 1) / CL + 3) / 4 * 4;
        if (share > CAP) return false;
        K k[ITEMS];
        if constexpr (CL == 1) {
            const int n = (int)cnt;
            load_staged(sm, k, src, n, regB, st, xf);
            auto mine = [&](int i) { return lidx(i) < n; };
            if (!count_sort(k, mine, lo, hi - lo, regB, reinterpret_cast<uint32_t *>(regA), sm.tmp, sm.list))
                return false;
            for (int j = tid; j < n; j += T) emit((uint32_t)j, regB[j]);
            return true;
        } else {
            auto cluster = cg::this_cluster();
            const int c = (int)cluster.block_rank();
            const int e0 = c * (int)share;
            const int mycnt = (int)imax64(0, imin64(share, cnt - e0));
            load_staged(sm, k, src + e0, mycnt, regB, st, xf);  // (the receive buffer is free until the barrier below)
            auto mine = [&](int i) { return lidx(i) < mycnt; };
            const int bits = bit_length<K>(hi - lo);
            const int shift = bits > 8 ? bits - 8 : 0;
            const uint32_t nbins = 1u << (bits - shift);
            if (tid < R) sm.cnt[tid] = 0;
            __syncthreads();
            // 1. split bin and rank inside it, packed: bin | rank << 8
            uint32_t dr[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (mine(i)) {
                    const uint32_t d = min((k[i] - lo) >> shift, nbins - 1u);
                    dr[i] = d | atomicAdd(&sm.cnt[d], 1u) << 8;
                }
            __syncthreads();
            if (warp == 0) warp_scan256(sm.cnt, sm.lbase);
            __syncthreads();
            // 2. my keys grouped by split bin
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (mine(i)) regA[sm.lbase[dr[i] & 255u] + (dr[i] >> 8)] = k[i];
            cluster.sync();
            // 3. the cluster's counts: bin totals, keys of the bin in lower-ranked CTAs
            if (tid < R) {
                uint32_t tot = 0, pre = 0;
                if (tid < (int)nbins) {
#pragma unroll
                    for (int q = 0; q < CL; ++q) {
                        const uint32_t t = *cluster.map_shared_rank(&sm.cnt[tid], q);
                        pre += q < c ? t : 0u;
                        tot += t;
                    }
                }
                sm.tot[tid] = tot;
                sm.pre[tid] = pre;
                sm.own[tid] = tot;
            }
            __syncthreads();
            for (int attempt = 0;; ++attempt) {
                // warp 0: output starts and owned positions
                if (warp == 0) {
                    warp_scan256(sm.tot, sm.ostart);
                    const uint32_t owned = warp_scan256(sm.own, sm.rpos);
                    if (lane == 0) sm.tmp[39] = max(1u, (owned + CL - 1) / CL);
                    if (lane < CL) {
                        sm.orecv[lane] = 0;
                        sm.ofirst[lane] = 0xffffffffu;
                        sm.olast[lane] = 0;
                        sm.obase[lane] = 0;
                    }
                }
                __syncthreads();
                // owners: bin d goes to CTA rpos[d] / target, so each CTA owns a
                // run of consecutive bins (empty bins included); the first and
                // last bin of every run record its bounds
                const uint32_t target = sm.tmp[39];
                auto owner_of = [&](int d) { return min(CL - 1, (int)(sm.rpos[d] / target)); };
                if (tid < (int)nbins) {
                    const int o = owner_of(tid);
                    if (tid == 0 || owner_of(tid - 1) != o) {
                        sm.ofirst[o] = (uint32_t)tid;
                        sm.obase[o] = sm.rpos[tid];
                    }
                    if (tid == (int)nbins - 1 || owner_of(tid + 1) != o) {
                        sm.olast[o] = (uint32_t)tid;
                        sm.orecv[o] = sm.rpos[tid] + sm.own[tid];  // end; minus obase below
                    }
                }
                __syncthreads();
                if (tid < CL && sm.ofirst[tid] != 0xffffffffu) sm.orecv[tid] -= sm.obase[tid];
                __syncthreads();
                bool over = false;
#pragma unroll
                for (int q = 0; q < CL; ++q) over |= sm.orecv[q] > (uint32_t)CAP;
                if (!over) {
                    if (tid < (int)nbins) {
                        const uint32_t skew = sm.pre[tid] - sm.lbase[tid];  // stage slot j of the bin: j + skew in it
                        const int o = owner_of(tid);
                        // for every bin of the run, flat or empty ones too, so that equal
                        // odelta at both ends means no flat bin lies between them
                        sm.odelta[tid] = sm.ostart[tid] - (sm.rpos[tid] - sm.obase[o]);
                        if (sm.own[tid]) {
                            const uint32_t at = sm.rpos[tid] - sm.obase[o] + skew;
                            sm.raddr[tid] = cluster_addr((uint32_t)__cvta_generic_to_shared(regB), (uint32_t)o) +
                                            at * (uint32_t)sizeof(K);
                        } else {
                            sm.raddr[tid] = (sm.ostart[tid] + skew) << 1 | 1u;  // flat (or empty) bin: straight out
                        }
                    }
                    __syncthreads();
                    break;
                }
                // some owner would overflow: the uniform decision of every CTA
                if (attempt == 1) {
                    cluster.sync();  // nobody reads this CTA's shared memory any more
                    return false;
                }
                // flat-bin pass: smallest and largest key of every split bin;
                // bins of one key value are then written out by their holders
                if (tid < R) {
                    sm.bmin[tid] = 0xffffffffu;
                    sm.bmax[tid] = 0u;
                }
                __syncthreads();
                for (int j = tid; j < mycnt; j += T) {
                    const K x = regA[j];
                    const uint32_t d = min((x - lo) >> shift, nbins - 1u);
                    atomicMin(&sm.bmin[d], x);
                    atomicMax(&sm.bmax[d], x);
                }
                cluster.sync();
                if (tid < (int)nbins && sm.tot[tid]) {
                    K gmin = 0xffffffffu, gmax = 0u;
#pragma unroll
                    for (int q = 0; q < CL; ++q) {
                        gmin = min(gmin, *cluster.map_shared_rank(&sm.bmin[tid], q));
                        gmax = max(gmax, *cluster.map_shared_rank(&sm.bmax[tid], q));
                    }
                    if (gmin == gmax) sm.own[tid] = 0;
                }
                __syncthreads();
            }
            // 4. exchange: stage runs to their owners, flat bins straight out
            // (consecutive lanes take consecutive slots, so a warp's stores
            // cover few 32-byte sectors of the owners' buffers)
#pragma unroll 4
            for (int j = tid; j < mycnt; j += T) {
                const K x = regA[j];
                const uint32_t at = sm.raddr[min((x - lo) >> shift, nbins - 1u)];
                if (at & 1u) emit((at >> 1) + (uint32_t)j, x);
                else st_cluster(at + (uint32_t)j * (uint32_t)sizeof(K), x);
            }
            cluster.sync();
            // 5. count sort of what I received
            const int got = (int)sm.orecv[c];
            if (got == 0) return true;
            const uint32_t first = sm.ofirst[c], last = sm.olast[c];
            const K llo = lo + (first << shift);
            const K lhi = last == nbins - 1u ? hi : lo + ((last + 1u) << shift) - 1u;
            K kr[ITEMS];  // a new array: the loaded keys are dead by now
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) kr[i] = slot(i) < got ? regB[slot(i)] : 0u;
            auto received = [&](int i) { return slot(i) < got; };
            // a CTA that cannot finish gives the sub-bucket back; what the
            // others emit is rewritten, identically, by the stable sort
            if (!count_sort(kr, received, llo, lhi - llo, regB, reinterpret_cast<uint32_t *>(regA), sm.tmp, sm.list))
                return false;
            // 6. out: with no flat bin among mine, one contiguous output range
            if (sm.odelta[first] == sm.odelta[last]) {
                const uint32_t base = sm.odelta[first];
                for (int j = tid; j < got; j += T) emit(base + (uint32_t)j, regB[j]);
            } else {
                for (int j = tid; j < got; j += T) {
                    const K x = regB[j];
                    emit(sm.odelta[min((x - lo) >> shift, nbins - 1u)] + (uint32_t)j, x);
                }
            }
            return true;
        }
    }
};

} // namespace bsps
