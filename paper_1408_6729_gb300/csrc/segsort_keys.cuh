// segsort_keys.cuh -- the keys-only bucket sort (Fig. 2 step 12), tuned for
// throughput: equal keys cannot be told apart, so no ranking needs to be
// stable and every rank comes from one shared-memory atomic.
//
// A cluster of CL CTAs (512 threads, two per SM) sorts one sub-bucket whose
// keys lie in [lo, hi] (bounds from the splitters).  Each CTA copies its share
// into shared memory with 16-byte loads, counts its keys per split bin (the
// top bits of key - lo), the counts are exchanged through distributed shared
// memory, and every key is stored into the shared memory of the CTA that owns
// its bin; bins holding one distinct key are written out directly.  Each CTA
// then counting-sorts what it received on up to kCountBits further bits and
// finishes the (short) count bins by insertion.  A split bin too large for one
// CTA makes the cluster give the sub-bucket back (returns false) to the
// stable cluster sort of segsort.cuh.
#pragma once

#include "radix.cuh"

namespace bsps {

template <typename K, int CL, int ITEMS>
struct SegSortKeys {
    static constexpr int T = 512;
    static constexpr int CAP = T * ITEMS;            // keys one CTA holds
    static constexpr int SB = 8, R = 1 << SB;        // split bins
    static constexpr int kCountBits = 12, kCountBins = 1 << kCountBits;

    struct Smem {
        uint32_t tot[R];     // keys of the bin in the sub-bucket (local counts until the exchange)
        uint32_t pre[R];     // keys of the bin held by lower-ranked CTAs
        uint32_t start[R];   // first sorted position of the bin
        uint32_t nfs[R];     // start among non-flat bins
        uint32_t lstart[R];  // start of the bin in its owner's buffer
        int32_t owner[R];    // -1: flat bin
        K bmin[R], bmax[R];
        uint32_t chist[kCountBins + 1];
        uint32_t recv[8], own_base[8];
        uint32_t tmp[40];
        int32_t bail;
    };
    static constexpr size_t smem_bytes() {
        return ((sizeof(Smem) + 15) & ~size_t(15)) + (size_t)CAP * sizeof(K) + (size_t)CAP * 2 + 64;
    }
    // bin of key k: (k - lo) >> shift, clamped to maxb so that a key outside
    // [lo, hi] can never index past a table
    __device__ static uint32_t bin(K k, K lo, int shift, uint32_t maxb) {
        const K d = (K)(k - lo) >> shift;
        return d < (K)maxb ? (uint32_t)d : maxb;
    }
    // item i of a thread: slot i*T + tid (item-major; layout is free here)
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

    // Copy n keys from global to shared memory (16-byte loads where aligned).
    __device__ static void load(K *dst, const K *__restrict__ src, int n) {
        constexpr int V = 16 / sizeof(K);
        const uintptr_t a = (uintptr_t)src;
        int head = (int)(((16 - (a & 15)) & 15) / sizeof(K));
        if (head > n) head = n;
        if ((a % sizeof(K)) != 0) head = n;  // not even key-aligned: scalar copy
        for (int j = threadIdx.x; j < head; j += T) dst[j] = src[j];
        const int nv = (n - head) / V;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src + head);
        for (int j = threadIdx.x; j < nv; j += T) {
            const uint4 w = __ldg(s4 + j);
            K *d = dst + head + j * V;
            if constexpr (sizeof(K) == 4) {
                d[0] = w.x; d[1] = w.y; d[2] = w.z; d[3] = w.w;
            } else {
                d[0] = ((uint64_t)w.y << 32) | w.x;
                d[1] = ((uint64_t)w.w << 32) | w.z;
            }
        }
        for (int j = head + nv * V + threadIdx.x; j < n; j += T) dst[j] = src[j];
    }

    // Sort buf[0..cnt) (keys in [lo, lo + 2^bits)) in place on this CTA: one
    // counting pass (ranks from atomics, keys held in registers across the
    // scatter), then insertion inside every count bin.
    static constexpr uint32_t kBinMax = 64;  // longest count bin finished by insertion

    __device__ static bool count_sort(Smem &sm, K *buf, int cnt, K lo, int bits) {
        const int nbb = bits < kCountBits ? bits : kCountBits;
        const int shift = bits - nbb;
        const int nb = 1 << nbb;
        for (int b = threadIdx.x; b <= nb; b += T) sm.chist[b] = 0;
        __syncthreads();
        K k[ITEMS];
        uint32_t r[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int j = slot(i);
            if (j < cnt) {
                k[i] = buf[j];
                r[i] = atomicAdd(&sm.chist[bin(k[i], lo, shift, nb - 1)], 1u);
            }
        }
        if (threadIdx.x == 0) sm.bail = 0;
        __syncthreads();
        if (shift > 0) {
            uint32_t longest = 0;
            for (int b = threadIdx.x; b < nb; b += T) longest = max(longest, sm.chist[b]);
            if (longest > kBinMax) sm.bail = 1;
        }
        __syncthreads();
        if (sm.bail) return false;  // uniform in the CTA
        block_excl_scan_smem<T>(sm.chist, nb, sm.tmp);
        if (threadIdx.x == 0) sm.chist[nb] = (uint32_t)cnt;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (slot(i) < cnt) buf[sm.chist[bin(k[i], lo, shift, nb - 1)] + r[i]] = k[i];
        __syncthreads();
        if (shift > 0) {
            for (int b = threadIdx.x; b < nb; b += T) {
                const int b0 = (int)sm.chist[b], b1 = (int)sm.chist[b + 1];
                for (int x = b0 + 1; x < b1; ++x) {
                    const K v = buf[x];
                    int y = x - 1;
                    while (y >= b0 && buf[y] > v) {
                        buf[y + 1] = buf[y];
                        --y;
                    }
                    buf[y + 1] = v;
                }
            }
            __syncthreads();
        }
        return true;
    }

    // Returns false when the sub-bucket does not fit this cluster or a CTA's
    // count bins are too long; the caller then hands it to the stable sort,
    // which rewrites every position (keys already emitted are rewritten with
    // the same values).
    template <typename Emit>
    __device__ static bool run(Smem &sm, K *buf, uint16_t *rk, const K *__restrict__ gsrc, int64_t cnt, K lo, K hi,
                               Emit emit) {
        auto cluster = cg::this_cluster();
        const int c = CL > 1 ? (int)cluster.block_rank() : 0;
        const int64_t share = ((cnt + CL - 1) / CL + 3) & ~int64_t(3);
        if (share > CAP) return false;
        const int64_t e0 = (int64_t)c * share;
        const int mycnt = (int)imax64(0, imin64(share, cnt - e0));
        const int bits = bit_length<K>(hi - lo);
        load(buf, gsrc + e0, mycnt);
        __syncthreads();
        if (bits == 0) {  // one distinct key
            for (int j = threadIdx.x; j < mycnt; j += T) emit((uint32_t)(e0 + j), buf[j]);
            return true;
        }
        if constexpr (CL == 1) {
            if (!count_sort(sm, buf, mycnt, lo, bits)) return false;
            for (int j = threadIdx.x; j < mycnt; j += T) emit((uint32_t)j, buf[j]);
            return true;
        } else {
            const int sb = bits < SB ? bits : SB;
            const int shift = bits - sb;
            const int nbins = 1 << sb;
            for (int b = threadIdx.x; b < R; b += T) {
                sm.tot[b] = 0;
                sm.bmin[b] = all_ones<K>();
                sm.bmax[b] = 0;
            }
            __syncthreads();
            K k[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const int j = slot(i);
                if (j < mycnt) {
                    k[i] = buf[j];
                    const uint32_t d = bin(k[i], lo, shift, nbins - 1);
                    rk[j] = (uint16_t)atomicAdd(&sm.tot[d], 1u);
                    atomic_min_max(&sm.bmin[d], &sm.bmax[d], k[i]);
                }
            }
            cluster.sync();
            // every CTA derives the same global bin layout
            uint32_t tot = 0, pre = 0;
            K gmin = all_ones<K>(), gmax = 0;
            const int b = threadIdx.x;
            if (b < nbins) {
#pragma unroll
                for (int r = 0; r < CL; ++r) {
                    const uint32_t t = *cluster.map_shared_rank(&sm.tot[b], r);
                    const K x = *cluster.map_shared_rank(&sm.bmin[b], r);
                    const K y = *cluster.map_shared_rank(&sm.bmax[b], r);
                    pre += r < c ? t : 0;
                    tot += t;
                    gmin = x < gmin ? x : gmin;
                    gmax = y > gmax ? y : gmax;
                }
            }
            // all remote reads are done and every key sits in registers: from
            // here on a CTA's buffer may be written by the others
            cluster.sync();
            const bool flat = tot == 0 || gmin == gmax;
            if (b < R) {
                sm.tot[b] = tot;
                sm.pre[b] = pre;
                sm.start[b] = tot;
                sm.nfs[b] = flat ? 0 : tot;
            }
            if (threadIdx.x < 8) {
                sm.recv[threadIdx.x] = 0;
                sm.own_base[threadIdx.x] = 0xffffffffu;
            }
            __syncthreads();
            digit_excl_scan<T, R>(sm.start, sm.tmp);
            if (threadIdx.x == R - 1) sm.tmp[39] = sm.nfs[R - 1];
            __syncthreads();
            const uint32_t last_nf = sm.tmp[39];
            digit_excl_scan<T, R>(sm.nfs, sm.tmp);
            const uint32_t total_nf = sm.nfs[R - 1] + last_nf;
            const uint32_t target = (total_nf + CL - 1) / CL;
            if (b < R) {
                if (!flat && tot > 0) {
                    const int t = target ? min(CL - 1, (int)(sm.nfs[b] / target)) : 0;
                    sm.owner[b] = t;
                    atomicAdd(&sm.recv[t], tot);
                    atomicMin(&sm.own_base[t], sm.nfs[b]);
                } else {
                    sm.owner[b] = -1;
                }
            }
            __syncthreads();
            if (b < R) sm.lstart[b] = sm.owner[b] >= 0 ? sm.nfs[b] - sm.own_base[sm.owner[b]] : 0;
            if (threadIdx.x == 0) {
                int bail = 0;
                for (int t = 0; t < CL; ++t) bail |= sm.recv[t] > (uint32_t)CAP;
                sm.bail = bail;
            }
            __syncthreads();
            if (sm.bail) return false;  // uniform; nobody touches another CTA's memory any more
            // exchange: every key to its bin's owner, flat bins straight out
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const int j = slot(i);
                if (j < mycnt) {
                    const uint32_t d = bin(k[i], lo, shift, nbins - 1);
                    const int t = sm.owner[d];
                    if (t < 0) {
                        emit(sm.start[d] + sm.pre[d] + rk[j], k[i]);
                    } else {
                        K *rb = cluster.map_shared_rank(buf, t);
                        rb[sm.lstart[d] + sm.pre[d] + rk[j]] = k[i];
                    }
                }
            }
            cluster.sync();
            const int got = (int)sm.recv[c];
            if (got == 0) return true;
            // received keys lie in the owned bins
            int first = R, last = -1;
            for (int bb = 0; bb < nbins; ++bb)
                if (sm.owner[bb] == c) {
                    first = bb < first ? bb : first;
                    last = bb;
                }
            const K llo = lo + ((K)first << shift);
            const K lhi = last == nbins - 1 ? hi : lo + ((K)(last + 1) << shift) - 1;
            const int lbits = bit_length<K>(lhi - llo);
            // a CTA that cannot finish its bins gives the sub-bucket back; what
            // the others emit is rewritten, identically, by the stable sort
            if (!count_sort(sm, buf, got, llo, lbits)) return false;
            for (int j = threadIdx.x; j < got; j += T) {
                const K x = buf[j];
                const uint32_t d = bin(x, lo, shift, nbins - 1);
                emit(sm.start[d] + (uint32_t)j - sm.lstart[d], x);
            }
            return true;
        }
    }
};

} // namespace bsps
