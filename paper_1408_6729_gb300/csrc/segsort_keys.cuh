// segsort_keys.cuh -- the keys-only bucket sort (Fig. 2 step 12), tuned for
// throughput: equal keys cannot be told apart, so no ranking needs to be
// stable and every rank comes from shared-memory atomics.
//
// With MINMAX the split also records every bin's smallest and largest key,
// which the caller's give_up predicate reads; without it a bin only keeps one
// of its keys and a flag for any other value, enough to find bins of one
// distinct key.
//
// A cluster of CL CTAs (512 threads, two per SM) sorts one sub-bucket whose
// keys lie in [lo, hi] (bounds from the splitters).  Each CTA loads its share
// into registers with 16-byte loads and ranks its keys per split bin (the top
// bits of key - lo), grouping them by bin in a local stage buffer.  The bin
// counts are read across the cluster through distributed shared memory; bins
// holding one distinct key are written out directly, every other bin is given
// to one CTA, and each CTA copies its stage, bin run by bin run, into the
// owners' receive buffers.  Each CTA then counting-sorts what it received on
// up to kCountBits further bits.  When a count bin spans at most 32 values,
// three occupancy masks per bin record which values occur at least once,
// twice and three times, and later occurrences are only counted; in a bin
// where no value occurs four times a key's place is the bin start plus the
// popcounts of the masks below its value plus its occurrence index.  Keys of
// other bins are placed by comparison.  A bin too large for one CTA,
// or count bins longer than kBinMax that need comparisons, make the cluster
// give the sub-bucket back (returns false) to the stable cluster sort of
// segsort.cuh.
#pragma once

#include "radix.cuh"

namespace bsps {

// address of a shared-memory location of this CTA in CTA `rank` of the
// cluster (shared::cluster window), and a store through such an address
__device__ __forceinline__ uint32_t cluster_addr(uint32_t cta_addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(cta_addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, uint64_t v) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

template <typename K, int CL, int ITEMS, bool MINMAX = true>
struct SegSortKeys {
    static constexpr int T = 512;
    static constexpr int V = 16 / (int)sizeof(K);     // keys per 16-byte load
    static constexpr int CAP = T * ITEMS;             // keys one CTA holds
    static constexpr int SB = 8, R = 1 << SB;         // split bins
    static constexpr int kCountBits = 12, kCountBins = 1 << kCountBits;
    static constexpr int kMaskBits = 5;               // count bins of at most 32 values carry masks
    static constexpr uint32_t kBinMax = 64;           // longest count bin ordered by comparison
    static_assert(ITEMS % V == 0, "whole 16-byte loads per thread");
    static_assert(kCountBins % (4 * T) == 0, "whole 16-byte groups of count bins per thread in the scan");

    struct Smem {
        uint32_t cnt[R];     // my keys per split bin (read by the other CTAs)
        K bmin[R];           // my smallest key per split bin, or (without MINMAX) any of them
        K bmax[MINMAX ? R : 1];  // my largest key per split bin (read by the others)
        uint32_t lbase[R];   // start of the bin in my stage; then where the exchange sends it
        uint32_t start[R];   // first output position of the bin
        uint32_t pre[R];     // keys of the bin held by lower-ranked CTAs
        uint32_t dst[R];     // start of the bin in its owner's receive buffer; then start - dst
        int32_t owner[R];    // -1: bin with one distinct key (or none)
        uint32_t recv[8], own_base[8], ofirst[8], olast[8];
        uint32_t tmp[40];
        uint32_t heavy;      // keys in bins the caller's give_up predicate marks
        uint8_t diff[MINMAX ? 1 : R];  // without MINMAX: my bin holds a key other than bmin
    };
    // the count histogram and the three masks (one word per bin) live in the
    // receive buffer, which is free by then; the buffer is sized for all four
    static constexpr int kM1 = kCountBins + 4, kM2 = kM1 + kCountBins, kM3 = kM2 + kCountBins,
                         kScratchWords = kM3 + kCountBins;
    static constexpr size_t kBufBytes =
        ((size_t)CAP * sizeof(K) > (size_t)kScratchWords * 4 ? (size_t)CAP * sizeof(K) : (size_t)kScratchWords * 4);
    static constexpr size_t smem_bytes() {
        return ((sizeof(Smem) + 15) & ~size_t(15)) + (size_t)CAP * sizeof(K) + kBufBytes;
    }

    // bin of key k: (k - lo) >> shift, clamped to maxb so that a key outside
    // [lo, hi] can never index past a table
    __device__ static uint32_t bin(K k, K lo, int shift, uint32_t maxb) {
        const K d = (K)(k - lo) >> shift;
        return d < (K)maxb ? (uint32_t)d : maxb;
    }
    // register i of a thread holds local key (i / V * T + tid) * V + i % V
    __device__ static int lidx(int i) { return ((i / V) * T + (int)threadIdx.x) * V + i % V; }
    // ... or, for keys taken from shared memory, key i * T + tid
    __device__ static int slot(int i) { return i * T + (int)threadIdx.x; }

    __device__ static void atomic_min_max(K *mn, K *mx, K v) {
        if constexpr (sizeof(K) == 8) {
            atomicMin((unsigned long long *)mn, (unsigned long long)v);
            atomicMax((unsigned long long *)mx, (unsigned long long)v);
        } else {
            atomicMin((unsigned *)mn, (unsigned)v);
            atomicMax((unsigned *)mx, (unsigned)v);
        }
    }

    // n keys from global memory (16-byte aligned; reading up to the next
    // multiple of V keys stays inside the caller's region) into registers
    __device__ static void load(K (&k)[ITEMS], const K *__restrict__ src, int n) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
#pragma unroll
        for (int j = 0; j < ITEMS / V; ++j) {
            const int q = j * T + (int)threadIdx.x;
            if (q * V < n) {
                const uint4 w = __ldg(s4 + q);
                if constexpr (sizeof(K) == 4) {
                    k[j * V + 0] = w.x; k[j * V + 1] = w.y; k[j * V + 2] = w.z; k[j * V + 3] = w.w;
                } else {
                    k[j * V + 0] = ((uint64_t)w.y << 32) | w.x;
                    k[j * V + 1] = ((uint64_t)w.w << 32) | w.z;
                }
            }
        }
    }

    // Exclusive scan of h[0..nb) (nb <= kCountBins) in place, h[nb] = total.
    // With check, returns false (uniformly) if a bin holds more than kBinMax.
    __device__ static bool scan_bins(uint32_t *h, int nb, uint32_t *tmp, bool check) {
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        constexpr int W = T / 32;
        const int per = (nb + T - 1) / T;
        const int b0 = tid * per;
        const bool vec = (per & 3) == 0;
        uint32_t s = 0, mx = 0;
        if (vec) {
            for (int q = 0; q < per; q += 4) {
                const uint4 a = *reinterpret_cast<const uint4 *>(h + b0 + q);
                s += a.x + a.y + a.z + a.w;
                mx = max(max(mx, max(a.x, a.y)), max(a.z, a.w));
            }
        } else {
            for (int q = 0; q < per && b0 + q < nb; ++q) {
                s += h[b0 + q];
                mx = max(mx, h[b0 + q]);
            }
        }
        uint32_t wtot;
        const uint32_t wex = warp_excl_scan(s, &wtot);
        if (lane == 31) tmp[warp] = wtot;
        if (__syncthreads_or(check && mx > kBinMax)) return false;
        if (warp == 0) {
            const uint32_t y = lane < W ? tmp[lane] : 0u;
            uint32_t t;
            const uint32_t ye = warp_excl_scan(y, &t);
            if (lane < W) tmp[lane] = ye;
            if (lane == 0) tmp[W] = t;
        }
        __syncthreads();
        uint32_t run = tmp[warp] + wex;
        if (vec) {
            for (int q = 0; q < per; q += 4) {
                uint4 a = *reinterpret_cast<const uint4 *>(h + b0 + q);
                const uint4 o = make_uint4(run, run + a.x, run + a.x + a.y, run + a.x + a.y + a.z);
                run += a.x + a.y + a.z + a.w;
                *reinterpret_cast<uint4 *>(h + b0 + q) = o;
            }
        } else {
            for (int q = 0; q < per && b0 + q < nb; ++q) {
                const uint32_t x = h[b0 + q];
                h[b0 + q] = run;
                run += x;
            }
        }
        if (tid == 0) h[nb] = tmp[W];
        __syncthreads();
        return true;
    }

    // Sort the keys held in registers (valid where valid(i); all in
    // [lo, lo + 2^bits)) into out[0..n): one counting pass on the top
    // kCountBits bits, then each key's place inside its count bin.  scr is free
    // shared memory of CAP keys.
    template <typename Valid>
    __device__ static bool count_sort(Smem &sm, const K (&k)[ITEMS], Valid valid, K lo, int bits, K *out,
                                      uint32_t *scr) {
        const int nbb = bits < kCountBits ? bits : kCountBits;
        const int shift = bits - nbb;
        const int nb = 1 << nbb;
        const bool masks = shift > 0 && shift <= kMaskBits;
        uint32_t *chist = scr, *m1 = scr + kM1, *m2 = scr + kM2, *m3 = scr + kM3;
        __syncthreads();  // scr may still be read by the caller
        for (int b = threadIdx.x; b < nb; b += T) chist[b] = 0;
        if (masks)
            for (int b = threadIdx.x; b < nb; b += T) m1[b] = m2[b] = m3[b] = 0;
        __syncthreads();
        // without masks r is the rank inside the count bin.  With masks it is
        // the occurrence of the value (bits 28..29: first, second, third,
        // later) and, for later ones, their rank among the bin's later
        // occurrences (bits 0..27), which chist counts.
        uint32_t r[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (valid(i)) {
                const uint32_t bb = bin(k[i], lo, shift, nb - 1);
                if (masks) {
                    const uint32_t bit = 1u << (uint32_t)((k[i] - lo) & (K)31);
                    uint32_t o = 0;
                    if (atomicOr(&m1[bb], bit) & bit) {
                        o = 1u << 28;
                        if (atomicOr(&m2[bb], bit) & bit) {
                            o = 2u << 28;
                            if (atomicOr(&m3[bb], bit) & bit) o = 3u << 28 | atomicAdd(&chist[bb], 1u);
                        }
                    }
                    r[i] = o;
                } else {
                    r[i] = atomicAdd(&chist[bb], 1u);
                }
            }
        __syncthreads();
        if (masks) {  // bin length: one key per mask bit, plus the later occurrences
            for (int b = threadIdx.x; b < nb; b += T) chist[b] += __popc(m1[b]) + __popc(m2[b]) + __popc(m3[b]);
            __syncthreads();
        }
        if (!scan_bins(chist, nb, sm.tmp, !masks && shift > 0)) return false;
        constexpr uint32_t kStart = 0x7fffffffu;  // bin start; bit 31: a value repeats
        bool cmp = false;
        if (masks) {
            for (int b = threadIdx.x; b < nb; b += T)
                if (m2[b]) chist[b] |= ~kStart;
            __syncthreads();
            // In a bin of distinct values a key's place follows from the
            // first mask alone.  In others it is final when no value occurs
            // four times (keys of smaller values + occurrence); otherwise the
            // key waits in a distinct slot of the bin (first occurrences, then
            // second, third and later ones) for the comparisons below.
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (valid(i)) {
                    const uint32_t bb = bin(k[i], lo, shift, nb - 1);
                    const uint32_t h = chist[bb], b0 = h & kStart;
                    const uint32_t below = (1u << (uint32_t)((k[i] - lo) & (K)31)) - 1u;
                    const uint32_t w1 = m1[bb];
                    uint32_t pos = b0 + __popc(w1 & below);
                    bool fin = true;
                    if (h & ~kStart) {
                        const uint32_t len = (chist[bb + 1] & kStart) - b0;
                        const uint32_t w2 = m2[bb], w3 = m3[bb], occ = r[i] >> 28;
                        const uint32_t c1 = __popc(w1), c12 = c1 + __popc(w2), c123 = c12 + __popc(w3);
                        const uint32_t l2 = __popc(w2 & below), l3 = __popc(w3 & below);
                        fin = c123 == len;
                        if (fin) pos += l2 + l3 + occ;
                        else if (occ == 1) pos = b0 + c1 + l2;
                        else if (occ == 2) pos = b0 + c12 + l3;
                        else if (occ == 3) pos = b0 + c123 + (r[i] & 0x0fffffffu);
                    }
                    out[pos] = k[i];
                    r[i] = fin ? 0xffffffffu : pos;
                    cmp |= !fin;
                }
        } else {
            // keys alone in their bin go to their final place, the others
            // wait at bin start + rank
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (valid(i)) {
                    const uint32_t bb = bin(k[i], lo, shift, nb - 1);
                    const uint32_t b0 = chist[bb], pos = b0 + r[i];
                    const bool fin = shift == 0 || chist[bb + 1] - b0 == 1;
                    out[pos] = k[i];
                    r[i] = fin ? 0xffffffffu : pos;
                    cmp |= !fin;
                }
        }
        if (!__syncthreads_or(cmp)) return true;
        // place = bin start + keys of the bin below k + equal keys stored before it
        bool too_long = false;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (valid(i) && r[i] != 0xffffffffu) {
                const uint32_t bb = bin(k[i], lo, shift, nb - 1);
                const uint32_t b0 = chist[bb] & kStart, b1 = chist[bb + 1] & kStart, self = r[i];
                if (b1 - b0 > kBinMax) {
                    too_long = true;
                } else {
                    uint32_t pos = b0;
                    for (uint32_t y = b0; y < b1; ++y) {
                        const K x = out[y];
                        pos += (x < k[i]) | ((x == k[i]) & (y < self));
                    }
                    r[i] = pos;
                }
            }
        if (__syncthreads_or(too_long)) return false;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (valid(i) && r[i] != 0xffffffffu) out[r[i]] = k[i];
        __syncthreads();
        return true;
    }

    // Sorts the cnt keys at gsrc (bounds lo <= key <= hi) and calls
    // emit(position, key) for each.  Returns false when the sub-bucket does not
    // fit this cluster or its bins are too uneven; the caller then hands it to
    // the stable sort, which rewrites every position (keys already emitted are
    // rewritten with the same values).  smem holds Smem, then the stage and the
    // receive buffer (CAP keys each).
    template <typename Emit>
    __device__ static bool run(unsigned char *smem, const K *__restrict__ gsrc, int64_t cnt, K lo, K hi, Emit emit) {
        auto from_global = [&](K (&k)[ITEMS], int64_t e0, int n) { load(k, gsrc + e0, n); };
        auto never = [](K, K) { return false; };
        return run_load(smem, cnt, lo, hi, from_global, emit, never);
    }

    // As run(), with the keys of positions [e0, e0 + n) produced by
    // load(k, e0, n) into register i of each thread for position e0 + lidx(i).
    // give_up(min, max) marks split bins the caller expects to be slow here;
    // when they hold more than a quarter of the keys the sub-bucket is given
    // back right after the split.
    template <typename Load, typename Emit, typename GiveUp>
    __device__ static bool run_load(unsigned char *smem, int64_t cnt, K lo, K hi, Load loadf, Emit emit,
                                    GiveUp give_up) {
        Smem &sm = *reinterpret_cast<Smem *>(smem);
        K *stage = reinterpret_cast<K *>(smem + ((sizeof(Smem) + 15) & ~size_t(15)));
        K *buf = stage + CAP;
        auto cluster = cg::this_cluster();
        const int c = CL > 1 ? (int)cluster.block_rank() : 0;
        const int64_t share = ((cnt + CL - 1) / CL + V - 1) / V * V;
        if (share > CAP) return false;
        const int64_t e0 = (int64_t)c * share;
        const int mycnt = (int)imax64(0, imin64(share, cnt - e0));
        const int bits = bit_length<K>(hi - lo);
        K k[ITEMS];
        loadf(k, e0, mycnt);
        auto mine = [&](int i) { return lidx(i) < mycnt; };
        if (bits == 0) {  // one distinct key
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (mine(i)) emit((uint32_t)(e0 + lidx(i)), k[i]);
            return true;
        }
        if constexpr (CL == 1) {
            if (!count_sort(sm, k, mine, lo, bits, stage, reinterpret_cast<uint32_t *>(buf))) return false;
            for (int j = threadIdx.x; j < mycnt; j += T) emit((uint32_t)j, stage[j]);
            return true;
        } else {
            const int sb = bits < SB ? bits : SB;
            const int shift = bits - sb;
            const int nbins = 1 << sb;
            const int tid = threadIdx.x;
            if (tid < R) {
                sm.cnt[tid] = 0;
                sm.bmin[tid] = all_ones<K>();
                if constexpr (MINMAX) sm.bmax[tid] = 0;
                else sm.diff[tid] = 0;
            }
            if (tid < 8) {
                sm.recv[tid] = 0;
                sm.own_base[tid] = 0xffffffffu;
                sm.ofirst[tid] = 0xffffffffu;
                sm.olast[tid] = 0;
            }
            if (tid == 0) sm.heavy = 0;
            __syncthreads();
            uint32_t r[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (mine(i)) {
                    const uint32_t d = bin(k[i], lo, shift, nbins - 1);
                    r[i] = atomicAdd(&sm.cnt[d], 1u);
                    if constexpr (MINMAX) atomic_min_max(&sm.bmin[d], &sm.bmax[d], k[i]);
                    else sm.bmin[d] = k[i];  // any key of the bin will do

                }
            __syncthreads();
            if (tid < R) sm.lbase[tid] = sm.cnt[tid];
            __syncthreads();
            digit_excl_scan<T, R>(sm.lbase, sm.tmp);
            // group my keys by bin in the stage
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (mine(i)) {
                    const uint32_t d = bin(k[i], lo, shift, nbins - 1);
                    stage[sm.lbase[d] + r[i]] = k[i];
                    if constexpr (!MINMAX)
                        if (k[i] != sm.bmin[d]) sm.diff[d] = 1;
                }
            cluster.sync();
            // every CTA derives the same global bin layout from all counts
            uint32_t tot = 0, pre = 0;
            K gmin = all_ones<K>(), gmax = 0;
            bool one = true;  // without MINMAX: every key of the bin equals gmin
            if (tid < nbins) {
#pragma unroll
                for (int q = 0; q < CL; ++q) {
                    const uint32_t t = *cluster.map_shared_rank(&sm.cnt[tid], q);
                    const K x = *cluster.map_shared_rank(&sm.bmin[tid], q);
                    if constexpr (MINMAX) {
                        const K y = *cluster.map_shared_rank(&sm.bmax[tid], q);
                        gmin = x < gmin ? x : gmin;
                        gmax = y > gmax ? y : gmax;
                    } else {
                        const uint8_t df = *cluster.map_shared_rank(&sm.diff[tid], q);
                        if (t) {
                            one &= df == 0 && (tot == 0 || x == gmin);
                            gmin = x;
                        }
                    }
                    pre += q < c ? t : 0u;
                    tot += t;
                }
            }
            const bool flat = tot == 0 || (MINMAX ? gmin == gmax : one);
            if constexpr (MINMAX)
                if (!flat && give_up(gmin, gmax)) atomicAdd(&sm.heavy, tot);
            if (tid < R) {
                sm.pre[tid] = pre;
                sm.start[tid] = tot;
                sm.dst[tid] = flat ? 0u : tot;
            }
            __syncthreads();
            if (tid == R - 1) sm.tmp[39] = sm.dst[R - 1];
            digit_excl_scan<T, R>(sm.start, sm.tmp);
            const uint32_t last_nf = sm.tmp[39];
            digit_excl_scan<T, R>(sm.dst, sm.tmp);
            const uint32_t total_nf = sm.dst[R - 1] + last_nf;
            const uint32_t target = (total_nf + CL - 1) / CL;
            if (tid < R) {
                int t = -1;
                if (!flat) {
                    t = target ? min(CL - 1, (int)(sm.dst[tid] / target)) : 0;
                    atomicAdd(&sm.recv[t], tot);
                    atomicMin(&sm.own_base[t], sm.dst[tid]);
                    atomicMin(&sm.ofirst[t], (uint32_t)tid);
                    atomicMax(&sm.olast[t], (uint32_t)tid);
                }
                sm.owner[tid] = t;
            }
            __syncthreads();
            if (tid < R) {
                const int t = sm.owner[tid];
                const uint32_t d0 = t >= 0 ? sm.dst[tid] - sm.own_base[t] : 0u;
                // key j of my stage goes to slot x + j of its owner's buffer, or
                // (one-key bins) to output position x + j; received key j of a
                // bin goes to output position dst[d] + j (modular arithmetic).
                // lbase[d] becomes the shared::cluster address of slot x in the
                // owner's buffer (even: K-aligned), or 2x + 1 (x < 2^31 here).
                const uint32_t x = (t >= 0 ? d0 : sm.start[tid]) + sm.pre[tid] - sm.lbase[tid];
                sm.lbase[tid] = t >= 0 ? cluster_addr((uint32_t)__cvta_generic_to_shared(buf), (uint32_t)t) +
                                             x * (uint32_t)sizeof(K)
                                       : x << 1 | 1u;
                sm.dst[tid] = sm.start[tid] - d0;
            }
            bool bail = (int64_t)sm.heavy * 4 > cnt;
#pragma unroll
            for (int q = 0; q < CL; ++q) bail |= sm.recv[q] > (uint32_t)CAP;
            if (bail) {  // uniform: every CTA saw the same counts
                cluster.sync();  // nobody reads this CTA's counts any more
                return false;
            }
            __syncthreads();
            // exchange: stage runs to their owners, one-key bins straight out
            for (int j = tid; j < mycnt; j += T) {
                const K x = stage[j];
                const uint32_t at = sm.lbase[bin(x, lo, shift, nbins - 1)];
                if (at & 1u) emit((at >> 1) + (uint32_t)j, x);
                else st_cluster(at + (uint32_t)j * (uint32_t)sizeof(K), x);
            }
            cluster.sync();
            const int got = (int)sm.recv[c];
            if (got == 0) return true;
            // received keys lie in the owned bins [ofirst, olast]
            const uint32_t first = sm.ofirst[c], last = sm.olast[c];
            const K llo = lo + ((K)first << shift);
            const K lhi = last == (uint32_t)nbins - 1 ? hi : lo + ((K)(last + 1) << shift) - 1;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (slot(i) < got) k[i] = buf[slot(i)];
            auto received = [&](int i) { return slot(i) < got; };
            // a CTA that cannot finish its bins gives the sub-bucket back; what
            // the others emit is rewritten, identically, by the stable sort
            if (!count_sort(sm, k, received, llo, bit_length<K>(lhi - llo), stage, reinterpret_cast<uint32_t *>(buf)))
                return false;
            // with no one-key bin between the owned bins (dst[d] is then the
            // same for all of them) the received keys fill one output range
            if (sm.dst[first] == sm.dst[last]) {
                const uint32_t o = sm.dst[first];
                for (int j = tid; j < got; j += T) emit(o + (uint32_t)j, stage[j]);
            } else {
                for (int j = tid; j < got; j += T) {
                    const K x = stage[j];
                    const uint32_t d = bin(x, lo, shift, nbins - 1);
                    emit(sm.dst[d] + (uint32_t)j, x);
                }
            }
            return true;
        }
    }
};

} // namespace bsps
