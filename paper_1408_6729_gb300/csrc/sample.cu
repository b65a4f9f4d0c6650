// sample.cu -- oversampling, sample sort, splitter selection (Fig. 1 steps
// 3-7, Fig. 3 steps 3-9) and the optional diagnostics.
#include "classify.cuh"
#include "segsort.cuh"

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
// pads (Lemma 5.1's padding), which follow every key in tag order.
// ---------------------------------------------------------------------------
template <int DT, int CL, int ITEMS>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kSortThreads, 1)
run_sample_kernel(const typename KeyTraits<DT>::T *__restrict__ keys, int64_t n, int64_t m,
                  int64_t M, int64_t s, int64_t x, typename KeyTraits<DT>::T *sphi, uint32_t *stag,
                  uint32_t *too_big) {
    using K = typename KeyTraits<DT>::T;
    using SS = SegSort<K, true, CL, ITEMS>;
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
        if ((pos + 1) % x == 0) {
            const int64_t j = (pos + 1) / x;
            sphi[k * s + (j - 1)] = key;
            stag[k * s + (j - 1)] = (uint32_t)(lo + slot);
        }
    };
    if (!SS::run(sm, buf, slots, len, load, emit) && threadIdx.x == 0 && blockIdx.x % CL == 0)
        atomicExch(too_big, 1u);
}

// ---------------------------------------------------------------------------
// Sample sort (Fig. 1 step 5): LSD radix sort of the records (phi, tag) by the
// bytes of tag, then of phi.  Byte positions on which every record agrees are
// skipped; the pass table is built on the device.
// ---------------------------------------------------------------------------
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
}

// table[0] = passes; then (position, src, dst) per pass; table[1+3*NPOS] = final buffer
template <typename K>
__global__ void lsd_plan_kernel(const uint32_t *hist, int64_t S, int32_t *table) {
    constexpr int NPOS = 4 + (int)sizeof(K);
    if (threadIdx.x != 0) return;
    int np = 0, cur = 0;
    for (int q = 0; q < NPOS; ++q) {
        bool trivial = false;
        for (int d = 0; d < 256; ++d) trivial |= (int64_t)hist[q * 256 + d] == S;
        if (trivial) continue;
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
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kLsdTile;
    for (int i = threadIdx.x; i < kLsdTile; i += kLsdThreads) {
        const int64_t r = t0 + i;
        if (r < S) atomicAdd(&h[record_digit(b.phi[src][r], b.tag[src][r], q)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) counts[(int64_t)d * tiles + blockIdx.x] = h[d];
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
    const int64_t t0 = (int64_t)blockIdx.x * kLsdTile;
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
        base[dd] = counts[(int64_t)dd * tiles + blockIdx.x];
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

template <int DT>
__global__ void bucket_of_kernel(const typename KeyTraits<DT>::T *keys, int64_t n, int64_t B,
                                 const typename KeyTraits<DT>::T *vphi, const uint32_t *vtag,
                                 const uint16_t *lut,
                                 const LutParams<typename KeyTraits<DT>::T> *lutp, int32_t *out) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const LutParams<typename KeyTraits<DT>::T> lp = *lutp;
    const uint32_t v = classify_key(KeyTraits<DT>::phi(keys[g]), (uint32_t)g, lp, lut, vphi, vtag);
    out[g] = (int32_t)(v / B);
}

template <typename K>
__global__ void pad_sizes_kernel(int64_t n, int64_t R, int64_t m, int64_t M, int64_t B, const K *vphi,
                                 const uint32_t *vtag, const uint16_t *lut, const LutParams<K> *lutp,
                                 unsigned long long *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * M) return;
    const int64_t k = t / M, j = t % M;
    const int64_t len = k * m < n ? min(m, n - k * m) : 0;
    if (j < len) return;
    const LutParams<K> lp = *lutp;
    const uint32_t v = classify_key(all_ones<K>(), (uint32_t)(n + k * M + j), lp, lut, vphi, vtag);
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

template <int DT, int CL, int ITEMS> static cudaError_t launch_run_sample(const Ctx &c) {
    using K = typename KeyTraits<DT>::T;
    using SS = SegSort<K, true, CL, ITEMS>;
    const size_t smem = SS::smem_bytes();
    auto kern = run_sample_kernel<DT, CL, ITEMS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const Plan &p = c.pl;
    kern<<<(unsigned)(p.R * CL), kSortThreads, smem, c.stream>>>(
        (const K *)c.keys_in, p.n, p.m, p.M, p.s, p.x, (K *)c.ly.sphi[0], c.ly.stag[0],
        (uint32_t *)&c.ly.status->run_too_big);
    return cudaGetLastError();
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
    constexpr int IT = sizeof(K) == 8 ? kRunItems64 : kRunItems32;
    switch (p.run_cl) {
    case 1: return launch_run_sample<DT, 1, IT>(c);
    case 2: return launch_run_sample<DT, 2, IT>(c);
    case 4: return launch_run_sample<DT, 4, IT>(c);
    case 8: return launch_run_sample<DT, 8, IT>(c);
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

template <typename K> static cudaError_t launch_sample_sort_t(const Ctx &c, LsdBuffers<K> b) {
    const Plan &p = c.pl;
    constexpr int NPOS = 4 + (int)sizeof(K);
    cudaError_t e = cudaMemsetAsync(c.ly.lsd_hist, 0, NPOS * 256 * sizeof(uint32_t), c.stream);
    if (e != cudaSuccess) return e;
    const int hist_blocks = (int)imin64(1024, (p.sample_size + 1023) / 1024);
    lsd_hist_kernel<K><<<max(hist_blocks, 1), 256, 0, c.stream>>>(b.phi[0], b.tag[0], p.sample_size,
                                                                  c.ly.lsd_hist);
    lsd_plan_kernel<K><<<1, 32, 0, c.stream>>>(c.ly.lsd_hist, p.sample_size, c.ly.lsd_table);
    const unsigned tiles = (unsigned)p.lsd_tiles;
    const size_t dsm = lsd_downsweep_smem<K>() + 16;
    e = cudaFuncSetAttribute(lsd_downsweep_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < NPOS && tiles > 0; ++pass) {
        lsd_upsweep_kernel<K><<<tiles, kLsdThreads, 0, c.stream>>>(b, p.sample_size, pass, c.ly.lsd_table,
                                                                  c.ly.lsd_counts, p.lsd_tiles);
        lsd_scan_kernel<<<256, 256, 0, c.stream>>>(c.ly.lsd_counts, p.lsd_tiles, pass, c.ly.lsd_table,
                                                   c.ly.lsd_hist);
        lsd_downsweep_kernel<K><<<tiles, kLsdThreads, dsm, c.stream>>>(b, p.sample_size, pass, c.ly.lsd_table,
                                                                      c.ly.lsd_counts, p.lsd_tiles);
    }
    return cudaGetLastError();
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
    if (c.dbg.bucket_of && p.n > 0)
        bucket_of_kernel<DT><<<(unsigned)((p.n + 255) / 256), 256, 0, c.stream>>>(
            (const K *)c.keys_in, p.n, p.B, (const K *)c.ly.vphi, c.ly.vtag, c.ly.lut,
            (const LutParams<K> *)c.ly.lutp, c.dbg.bucket_of);
    if (c.dbg.pad_sizes) {
        cudaError_t e = cudaMemsetAsync(c.dbg.pad_sizes, 0, sizeof(int64_t) * p.p, c.stream);
        if (e != cudaSuccess) return e;
        if (regular && p.R * p.M > p.n)
            pad_sizes_kernel<K><<<(unsigned)((p.R * p.M + 255) / 256), 256, 0, c.stream>>>(
                p.n, p.R, p.m, p.M, p.B, (const K *)c.ly.vphi, c.ly.vtag, c.ly.lut,
                (const LutParams<K> *)c.ly.lutp, (unsigned long long *)c.dbg.pad_sizes);
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
