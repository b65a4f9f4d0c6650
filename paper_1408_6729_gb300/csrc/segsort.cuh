// segsort.cuh -- stable sort of one segment of keys by a thread-block cluster.
//
// This is the "Sort_Seq" of the paper on chip (Fig. 1 step 3 for a block of
// keys, Fig. 2 step 12 for a bucket; stable as Sec. 5.1.1 requires).  The
// segment is split once across the CL CTAs of a cluster by the top bits of
// (key - min): every CTA counts its keys per bin, the counts are exchanged
// through distributed shared memory, and every key is stored into the shared
// memory of the CTA that owns its bin.  Bins whose keys are all equal need no
// sorting and are emitted where they are.  Each CTA then finishes its bins
// with a local LSD radix sort in shared memory.  Input order among equal keys
// is kept throughout (per-warp stable ranking, source CTAs in rank order).
#pragma once

#include "radix.cuh"

namespace bsps {

template <typename K, bool SLOT, int CL, int ITEMS>
struct SegSort {
    static constexpr int T = 1024;                 // threads per CTA
    static constexpr int CAP = T * ITEMS;          // keys one CTA holds
    static constexpr int RB = 8, R = 1 << RB;      // digit bits of every pass
    static constexpr int kCountBits = 12, kCountBins = 1 << kCountBits;
    static constexpr int kBinMax = 48;             // longest bin finished by insertion
    using Rank = BlockRank<T, ITEMS, RB>;

    struct Smem {
        typename Rank::Smem rank;
        uint32_t start[R];   // first sorted position of each bin in the segment
        uint32_t pre[R];     // keys of the bin held by lower-ranked CTAs
        uint32_t tot[R];     // keys of the bin in the segment
        uint32_t nfs[R];     // start among the keys of bins that are not flat
        uint32_t lstart[R];  // start of the bin in its owner's buffer
        int32_t owner[R];    // CTA that sorts the bin, -1 if the bin is flat
        K bmin[R], bmax[R];
        uint32_t base[R];
        uint32_t chist[kCountBins + 1];   // counting sort of the keys-only finish
        uint32_t recv[8], own_base[8];
        uint32_t maxbin;
        uint32_t tmp[40];
        K red_min, red_max;
        int32_t bail;
    };

    static constexpr size_t buffer_bytes() { return (size_t)CAP * (sizeof(K) + (SLOT ? 4 : 0)); }
    static constexpr size_t smem_bytes() { return ((sizeof(Smem) + 15) & ~size_t(15)) + buffer_bytes(); }

    // block min/max (valid items only); cluster-wide when CL > 1
    __device__ static void minmax(Smem &sm, K lo, K hi, K &out_lo, K &out_hi) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const K a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
            lo = a < lo ? a : lo;
            hi = b > hi ? b : hi;
        }
        if (threadIdx.x == 0) { sm.red_min = all_ones<K>(); sm.red_max = 0; }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomic_min_max(&sm.red_min, &sm.red_max, lo, hi);
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
            cluster.sync();
        } else {
            __syncthreads();
            out_lo = sm.red_min;
            out_hi = sm.red_max;
            __syncthreads();
        }
    }

    __device__ static void atomic_min_max(K *mn, K *mx, K lo, K hi) {
        if constexpr (sizeof(K) == 8) {
            atomicMin((unsigned long long *)mn, (unsigned long long)lo);
            atomicMax((unsigned long long *)mx, (unsigned long long)hi);
        } else {
            atomicMin((unsigned *)mn, (unsigned)lo);
            atomicMax((unsigned *)mx, (unsigned)hi);
        }
    }

    // Local LSD sort of buf[0..cnt) (keys in [lo, lo + 2^bits)), stable.
    __device__ static void local_sort(Smem &sm, K *buf, uint32_t *slots, int cnt, K lo, int bits) {
        if (bits <= 0 || cnt <= 1) return;
        const int ia = (cnt + T - 1) / T;
        const int passes = (bits + RB - 1) / RB;
        const int db = (bits + passes - 1) / passes;
        const uint32_t mask = (1u << db) - 1;
        for (int p = 0; p < passes; ++p) {
            const int shift = p * db;
            K k[ITEMS];
            uint32_t v[ITEMS], d[ITEMS], rk[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < ia) {
                    const int s = striped_slot_n<T>(i, ia);
                    const bool ok = s < cnt;
                    k[i] = buf[s];
                    if constexpr (SLOT) v[i] = slots[s];
                    d[i] = ok ? (uint32_t)((k[i] - lo) >> shift) & mask : mask;
                }
            }
            Rank::rank_n(sm.rank, d, rk, ia);
            if (threadIdx.x == 0) sm.rank.digit_tot[mask] -= (uint32_t)(ia * T - cnt);
            __syncthreads();
            for (int dd = threadIdx.x; dd < R; dd += T) sm.base[dd] = dd <= (int)mask ? sm.rank.digit_tot[dd] : 0;
            __syncthreads();
            digit_excl_scan<T, R>(sm.base, sm.tmp);
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < ia) {
                    const uint32_t pos = sm.base[d[i]] + rk[i];
                    buf[pos] = k[i];
                    if constexpr (SLOT) slots[pos] = v[i];
                }
            }
            __syncthreads();
        }
    }

    // Keys only (no companion, order of equal keys free): one counting pass on
    // the top bits of (key - lo) with shared-memory atomics, then every bin is
    // finished by insertion; a bin longer than kBinMax sends the CTA to the
    // LSD sort instead.
    __device__ static void local_count_sort(Smem &sm, K *buf, uint32_t *slots, int cnt, K lo, int bits) {
        if (bits <= 0 || cnt <= 1) return;
        const int nbb = bits < kCountBits ? bits : kCountBits;
        const int shift = bits - nbb;
        const int nb = 1 << nbb;
        for (int b = threadIdx.x; b <= nb; b += T) sm.chist[b] = 0;
        __syncthreads();
        const int ia = (cnt + T - 1) / T;
        K k[ITEMS];
        uint32_t rk[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int j = i * T + (int)threadIdx.x;
            if (i < ia && j < cnt) {
                k[i] = buf[j];
                rk[i] = atomicAdd(&sm.chist[(uint32_t)((k[i] - lo) >> shift)], 1u);
            }
        }
        __syncthreads();
        uint32_t longest = 0;
        for (int b = threadIdx.x; b < nb; b += T) longest = max(longest, sm.chist[b]);
        longest = __reduce_max_sync(0xffffffffu, longest);
        if ((threadIdx.x & 31) == 0) atomicMax(&sm.maxbin, longest);
        block_excl_scan_smem<T>(sm.chist, nb, sm.tmp);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int j = i * T + (int)threadIdx.x;
            if (i < ia && j < cnt) buf[sm.chist[(uint32_t)((k[i] - lo) >> shift)] + rk[i]] = k[i];
        }
        if (threadIdx.x == 0) sm.chist[nb] = (uint32_t)cnt;
        __syncthreads();
        const uint32_t maxbin = sm.maxbin;
        __syncthreads();
        if (shift == 0) return;  // one key value per bin
        if (maxbin > (uint32_t)kBinMax) {
            local_sort(sm, buf, slots, cnt, lo, bits);
            return;
        }
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

    __device__ static void finish(Smem &sm, K *buf, uint32_t *slots, int cnt, K lo, int bits) {
        if constexpr (SLOT) {
            local_sort(sm, buf, slots, cnt, lo, bits);
        } else {
            if (threadIdx.x == 0) sm.maxbin = 0;
            __syncthreads();
            local_count_sort(sm, buf, slots, cnt, lo, bits);
        }
    }

    // Fallback of the split when one bin holding several distinct keys does
    // not fit one CTA: LSD passes over the whole segment; after every pass CTA
    // c holds the sorted positions [c*share, c*share + share), and every key
    // is stored into the shared memory of the CTA that owns its position.
    template <typename Emit>
    __device__ static void cluster_lsd(Smem &sm, K *buf, uint32_t *slots, const K (&k0)[ITEMS], int ia,
                                       int mycnt, int64_t e0, int64_t share, K lo, int bits, Emit emit) {
        auto cluster = cg::this_cluster();
        const int c = CL > 1 ? (int)cluster.block_rank() : 0;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (i < ia) {
                const int s = striped_slot_n<T>(i, ia);
                if (s < mycnt) {
                    buf[s] = k0[i];
                    if constexpr (SLOT) slots[s] = (uint32_t)(e0 + s);
                }
            }
        }
        __syncthreads();
        const int passes = (bits + RB - 1) / RB;
        const int db = (bits + passes - 1) / passes;
        const uint32_t mask = (1u << db) - 1;
        for (int p = 0; p < passes; ++p) {
            const int shift = p * db;
            K kk[ITEMS];
            uint32_t v[ITEMS], d[ITEMS], rk[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < ia) {
                    const int s = striped_slot_n<T>(i, ia);
                    const bool ok = s < mycnt;
                    kk[i] = buf[s];
                    if constexpr (SLOT) v[i] = slots[s];
                    d[i] = ok ? (uint32_t)((kk[i] - lo) >> shift) & mask : mask;
                }
            }
            Rank::rank_n(sm.rank, d, rk, ia);
            if (threadIdx.x == 0) sm.rank.digit_tot[mask] -= (uint32_t)(ia * T - mycnt);
            cluster.sync();
            for (int dd = threadIdx.x; dd < R; dd += T) {
                uint32_t tot = 0, pre = 0;
                if (dd <= (int)mask) {
#pragma unroll
                    for (int r = 0; r < CL; ++r) {
                        const uint32_t t = *cluster.map_shared_rank(&sm.rank.digit_tot[dd], r);
                        pre += r < c ? t : 0;
                        tot += t;
                    }
                }
                sm.base[dd] = tot;
                sm.pre[dd] = pre;
            }
            __syncthreads();
            digit_excl_scan<T, R>(sm.base, sm.tmp);
            for (int dd = threadIdx.x; dd < R; dd += T) sm.base[dd] += sm.pre[dd];
            __syncthreads();
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < ia) {
                    const int s = striped_slot_n<T>(i, ia);
                    if (s < mycnt) {
                        const uint32_t pos = sm.base[d[i]] + rk[i];
                        const int owner = (int)(pos / share);
                        const uint32_t slot = (uint32_t)(pos - (int64_t)owner * share);
                        cluster.map_shared_rank(buf, owner)[slot] = kk[i];
                        if constexpr (SLOT) cluster.map_shared_rank(slots, owner)[slot] = v[i];
                    }
                }
            }
            cluster.sync();
        }
        for (int j = threadIdx.x; j < mycnt; j += T) emit(e0 + j, buf[j], SLOT ? slots[j] : 0u);
    }

    // Sort the `cnt` keys load(0..cnt-1) (phi form).  The companion of key e
    // is e.  emit(pos, key, companion) is called once per key with its
    // position in the sorted segment.  Returns false when the segment does not
    // fit (nothing was emitted); the decision is the same in every CTA.
    template <typename Load, typename Emit>
    __device__ static bool run(Smem &sm, K *buf, uint32_t *slots, int64_t cnt, Load load, Emit emit) {
        auto cluster = cg::this_cluster();
        const int c = CL > 1 ? (int)cluster.block_rank() : 0;
        const int64_t share = (cnt + CL - 1) / CL;
        if (share > CAP) return false;
        const int ia = (int)((share + T - 1) / T);
        const int64_t e0 = (int64_t)c * share;
        const int mycnt = (int)imax64(0, imin64(share, cnt - e0));

        K k[ITEMS];
        uint32_t d[ITEMS], rk[ITEMS];
        K mn = all_ones<K>(), mx = 0;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (i < ia) {
                const int s = striped_slot_n<T>(i, ia);
                k[i] = s < mycnt ? load(e0 + s) : K(0);
                if (s < mycnt) {
                    mn = k[i] < mn ? k[i] : mn;
                    mx = k[i] > mx ? k[i] : mx;
                }
            }
        }
        K lo, hi;
        minmax(sm, mn, mx, lo, hi);
        const int bits = bit_length<K>(hi - lo);
        if (bits == 0) {  // one distinct key: input order is sorted order
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < ia) {
                    const int s = striped_slot_n<T>(i, ia);
                    if (s < mycnt) emit(e0 + s, k[i], (uint32_t)(e0 + s));
                }
            }
            return true;
        }
        if constexpr (CL == 1) {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < ia) {
                    const int s = striped_slot_n<T>(i, ia);
                    buf[s] = k[i];
                    if constexpr (SLOT) slots[s] = (uint32_t)s;
                }
            }
            __syncthreads();
            finish(sm, buf, slots, mycnt, lo, bits);
            for (int j = threadIdx.x; j < mycnt; j += T) emit(j, buf[j], SLOT ? slots[j] : 0u);
            return true;
        } else {
            // ---- split by the top bits across the cluster ----
            const int sb = bits < RB ? bits : RB;
            const int shift = bits - sb;
            const int nbins = 1 << sb;
            for (int b = threadIdx.x; b < R; b += T) {
                sm.bmin[b] = all_ones<K>();
                sm.bmax[b] = 0;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < ia) {
                    const int s = striped_slot_n<T>(i, ia);
                    const bool ok = s < mycnt;
                    d[i] = ok ? (uint32_t)((k[i] - lo) >> shift) : (uint32_t)(nbins - 1);
                    if (ok) atomic_min_max(&sm.bmin[d[i]], &sm.bmax[d[i]], k[i], k[i]);
                }
            }
            if constexpr (SLOT) {
                Rank::rank_n(sm.rank, d, rk, ia);
                if (threadIdx.x == 0) sm.rank.digit_tot[nbins - 1] -= (uint32_t)(ia * T - mycnt);
            } else {
                // keys only: the order of equal keys is free, ranks from atomics
                for (int b = threadIdx.x; b < R; b += T) sm.rank.digit_tot[b] = 0;
                __syncthreads();
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    if (i < ia) {
                        const int s = striped_slot_n<T>(i, ia);
                        if (s < mycnt) rk[i] = atomicAdd(&sm.rank.digit_tot[d[i]], 1u);
                    }
                }
            }
            cluster.sync();
            for (int b = threadIdx.x; b < R; b += T) {
                uint32_t tot = 0, pre = 0;
                K gmin = all_ones<K>(), gmax = 0;
                if (b < nbins) {
#pragma unroll
                    for (int r = 0; r < CL; ++r) {
                        const uint32_t t = *cluster.map_shared_rank(&sm.rank.digit_tot[b], r);
                        const K x = *cluster.map_shared_rank(&sm.bmin[b], r);
                        const K y = *cluster.map_shared_rank(&sm.bmax[b], r);
                        pre += r < c ? t : 0;
                        tot += t;
                        gmin = x < gmin ? x : gmin;
                        gmax = y > gmax ? y : gmax;
                    }
                }
                const bool flat = tot == 0 || gmin == gmax;
                sm.tot[b] = tot;
                sm.pre[b] = pre;
                sm.start[b] = tot;
                sm.nfs[b] = flat ? 0 : tot;
                sm.owner[b] = flat ? -1 : 0;
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
            for (int b = threadIdx.x; b < R; b += T) {
                if (sm.owner[b] >= 0 && sm.tot[b] > 0) {
                    const int t = target ? min(CL - 1, (int)(sm.nfs[b] / target)) : 0;
                    sm.owner[b] = t;
                    atomicAdd(&sm.recv[t], sm.tot[b]);
                    atomicMin(&sm.own_base[t], sm.nfs[b]);
                } else {
                    sm.owner[b] = -1;
                }
            }
            __syncthreads();
            for (int b = threadIdx.x; b < R; b += T)
                sm.lstart[b] = sm.owner[b] >= 0 ? sm.nfs[b] - sm.own_base[sm.owner[b]] : 0;
            if (threadIdx.x == 0) {
                int bail = 0;
                for (int t = 0; t < CL; ++t) bail |= sm.recv[t] > (uint32_t)CAP;
                sm.bail = bail;
            }
            __syncthreads();
            if (sm.bail) {
                cluster.sync();  // everybody is done reading the split counts
                cluster_lsd(sm, buf, slots, k, ia, mycnt, e0, share, lo, bits, emit);
                return true;
            }
            // ---- exchange: every key to its bin's owner, flat bins in place ----
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < ia) {
                    const int s = striped_slot_n<T>(i, ia);
                    if (s < mycnt) {
                        const uint32_t b = d[i];
                        const int t = sm.owner[b];
                        if (t < 0) {
                            emit(sm.start[b] + sm.pre[b] + rk[i], k[i], (uint32_t)(e0 + s));
                        } else {
                            const uint32_t pos = sm.lstart[b] + sm.pre[b] + rk[i];
                            K *rb = cluster.map_shared_rank(buf, t);
                            rb[pos] = k[i];
                            if constexpr (SLOT) {
                                uint32_t *rs = cluster.map_shared_rank(slots, t);
                                rs[pos] = (uint32_t)(e0 + s);
                            }
                        }
                    }
                }
            }
            cluster.sync();
            // ---- finish the bins this CTA owns ----
            const int got = (int)sm.recv[c];
            if (got == 0) return true;
            K lmn = all_ones<K>(), lmx = 0;
            for (int j = threadIdx.x; j < got; j += T) {
                const K x = buf[j];
                lmn = x < lmn ? x : lmn;
                lmx = x > lmx ? x : lmx;
            }
            // block-level reduction (no cluster)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const K a = __shfl_xor_sync(0xffffffffu, lmn, o), b = __shfl_xor_sync(0xffffffffu, lmx, o);
                lmn = a < lmn ? a : lmn;
                lmx = b > lmx ? b : lmx;
            }
            if (threadIdx.x == 0) { sm.red_min = all_ones<K>(); sm.red_max = 0; }
            __syncthreads();
            if ((threadIdx.x & 31) == 0) atomic_min_max(&sm.red_min, &sm.red_max, lmn, lmx);
            __syncthreads();
            const K llo = sm.red_min;
            const int lbits = bit_length<K>(sm.red_max - llo);
            __syncthreads();
            finish(sm, buf, slots, got, llo, lbits);
            for (int j = threadIdx.x; j < got; j += T) {
                const K x = buf[j];
                const uint32_t b = (uint32_t)((x - lo) >> shift);
                emit(sm.start[b] + (uint32_t)j - sm.lstart[b], x, SLOT ? slots[j] : 0u);
            }
            return true;
        }
    }
};

} // namespace bsps
