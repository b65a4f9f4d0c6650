// route.cu -- classification, per-bucket prefix and the routing permutation
// (Fig. 1 steps 9-11; Fig. 2 steps 9-11), then the bucket offsets.
//
// One pass over the keys in HBM.  Tiles of kRouteTile keys are taken in
// order from an atomic ticket.  A tile first counts its keys per sub-bucket
// (Fig. 1 step 9), publishes the counts, and finds how many keys of each
// sub-bucket come before it by looking back over earlier tiles' published
// counts (decoupled look-back: the "p independent parallel prefix
// operations" of Fig. 1 step 9, Lemma 4.2).  It then reads its keys again
// (from L2), stably sorts each chunk by sub-bucket in shared memory, and
// writes each sub-bucket's keys as one contiguous run into that sub-bucket's
// region.  Keys keep input order inside every region (Fig. 1 step 11: "the
// initial ordering of the keys is preserved").
#include "classify.cuh"
#include "radix.cuh"

namespace bsps {

constexpr uint32_t kFlagA = 1u << 30;   // aggregate of this tile only
constexpr uint32_t kFlagP = 2u << 30;   // inclusive prefix through this tile
constexpr uint32_t kValMask = (1u << 30) - 1;

template <typename K> struct RouteArgs {
    const K *keys;
    const uint32_t *vals;
    int64_t n;
    const LutParams<K> *lutp;
    const uint32_t *lut;
    const K *vphi;
    const uint32_t *vtag;
    uint32_t P;
    int64_t tiles;
    uint32_t *state;
    K *reg_keys;
    uint32_t *reg_vals;
    int64_t cap;
    DevStatus *st;
};

template <typename K> struct RouteFixed {
    typename BlockRank<kRouteThreads, kRouteItems, 8>::Smem rank;
    uint32_t base[256];
    uint32_t tmp[40];
    uint32_t warp_max[kRouteThreads / 32];
    int64_t tile;
    LutParams<K> lp;
};

template <typename K, bool PAIRS> struct RouteSmemLayout {
    size_t lut, sphi, stag, run, stage_k, stage_v, stage_b, total;
    __host__ __device__ RouteSmemLayout(uint32_t P) {
        size_t o = (sizeof(RouteFixed<K>) + 15) & ~size_t(15);
        lut = o;     o += sizeof(uint32_t) * (kLutCells + 1);
        o = (o + 15) & ~size_t(15);
        sphi = o;    o += sizeof(K) * (P > 1 ? P - 1 : 1);
        o = (o + 15) & ~size_t(15);
        stag = o;    o += sizeof(uint32_t) * (P > 1 ? P - 1 : 1);
        o = (o + 15) & ~size_t(15);
        run = o;     o += sizeof(uint32_t) * P;
        o = (o + 15) & ~size_t(15);
        stage_k = o; o += sizeof(K) * kRouteChunk;
        stage_v = o; o += PAIRS ? sizeof(uint32_t) * kRouteChunk : 0;
        stage_b = o; o += sizeof(uint32_t) * kRouteChunk;
        total = o;
    }
};

template <int DT, bool PAIRS>
__global__ void __launch_bounds__(kRouteThreads, 1) route_kernel(const RouteArgs<typename KeyTraits<DT>::T> a) {
    using K = typename KeyTraits<DT>::T;
    using Rank = BlockRank<kRouteThreads, kRouteItems, 8>;
    constexpr int IT = kRouteItems;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RouteSmemLayout<K, PAIRS> L(a.P);
    RouteFixed<K> &fx = *reinterpret_cast<RouteFixed<K> *>(smem_raw);
    uint32_t *lut = reinterpret_cast<uint32_t *>(smem_raw + L.lut);
    K *sphi = reinterpret_cast<K *>(smem_raw + L.sphi);
    uint32_t *stag = reinterpret_cast<uint32_t *>(smem_raw + L.stag);
    uint32_t *run = reinterpret_cast<uint32_t *>(smem_raw + L.run);
    K *stage_k = reinterpret_cast<K *>(smem_raw + L.stage_k);
    uint32_t *stage_v = reinterpret_cast<uint32_t *>(smem_raw + L.stage_v);
    uint32_t *stage_b = reinterpret_cast<uint32_t *>(smem_raw + L.stage_b);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t P = a.P, nsplit = P - 1;

    // splitters and radix index into shared memory (Fig. 1 step 7, "broadcast")
    for (int i = tid; i <= kLutCells; i += kRouteThreads) lut[i] = a.lut[i];
    for (uint32_t i = tid; i < nsplit; i += kRouteThreads) {
        sphi[i] = a.vphi[i];
        stag[i] = a.vtag[i];
    }
    if (tid == 0) fx.lp = *a.lutp;
    __syncthreads();
    const LutParams<K> lp = fx.lp;
    const int bbits = bit_length<uint32_t>(P);  // sub-bucket ids, with P as "no key"

    for (;;) {
        if (tid == 0) fx.tile = (int64_t)atomicAdd(&a.st->tile_counter, 1u);
        __syncthreads();
        const int64_t tile = fx.tile;
        if (tile >= a.tiles) break;
        const int64_t t0 = tile * kRouteTile;
        const int64_t tlen = imin64(kRouteTile, a.n - t0);

        // ---- counts per sub-bucket of this tile (Fig. 1 step 9) ----
        for (uint32_t b = tid; b < P; b += kRouteThreads) run[b] = 0;
        __syncthreads();
        for (int64_t cs = 0; cs < tlen; cs += kRouteChunk) {
            K kk[IT];
            bool ok[IT];
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int64_t e = cs + striped_slot<kRouteThreads, IT>(i);
                ok[i] = e < tlen;
                kk[i] = ok[i] ? a.keys[t0 + e] : K(0);
            }
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int64_t e = cs + striped_slot<kRouteThreads, IT>(i);
                const uint32_t b = ok[i] ? classify_key(KeyTraits<DT>::phi(kk[i]), (uint32_t)(t0 + e), lp,
                                                        lut, sphi, stag)
                                         : 0xffffffffu;
                const uint32_t peers = __match_any_sync(0xffffffffu, b);
                if (ok[i] && (peers & lanemask_lt()) == 0) atomicAdd(&run[b], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();

        // ---- publish, look back, publish the inclusive prefix (Lemma 4.2) ----
        uint32_t *my = a.state + tile * P;
        if (tile == 0) {
            for (uint32_t b = tid; b < P; b += kRouteThreads) {
                const uint32_t cnt = run[b];
                st_volatile(&my[b], kFlagP | cnt);
                run[b] = 0;
                if (cnt > a.cap) { atomicExch(&a.st->overflow, 1); set_error(a.st, BSPS_ERR_BUCKET_OVERFLOW); }
            }
        } else {
            for (uint32_t b = tid; b < P; b += kRouteThreads) st_volatile(&my[b], kFlagA | run[b]);
            for (uint32_t b = tid; b < P; b += kRouteThreads) {
                uint32_t excl = 0;
                for (int64_t t = tile - 1; t >= 0; --t) {
                    const uint32_t *w = a.state + t * P + b;
                    uint32_t v = ld_volatile(w), polls = 0;
                    while ((v >> 30) == 0 && ++polls < kSpinLimit) {
                        // after any expired wait, nobody waits any more
                        if ((polls & 255) == 0 && ld_volatile((const uint32_t *)&a.st->timeouts) != 0) break;
                        __nanosleep(64);
                        v = ld_volatile(w);
                    }
                    if ((v >> 30) == 0) {
                        atomicAdd(&a.st->timeouts, 1);
                        set_error(a.st, BSPS_ERR_DEVICE_TIMEOUT);
                        break;
                    }
                    excl += v & kValMask;
                    if ((v >> 30) == 2) break;
                }
                const uint32_t cnt = run[b];
                st_volatile(&my[b], kFlagP | ((excl + cnt) & kValMask));
                run[b] = excl;
                if ((uint64_t)excl + cnt > (uint64_t)a.cap) {
                    atomicExch(&a.st->overflow, 1);
                    set_error(a.st, BSPS_ERR_BUCKET_OVERFLOW);
                }
            }
        }
        __syncthreads();

        // ---- route: stable partition of each chunk by sub-bucket, then one
        //      contiguous write per sub-bucket run (Fig. 1 step 11) ----
        for (int64_t cs = 0; cs < tlen; cs += kRouteChunk) {
            const int clen = (int)imin64(kRouteChunk, tlen - cs);
            K kk[IT];
            uint32_t vv[IT], bb[IT], d[IT], rk[IT];
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int s = striped_slot<kRouteThreads, IT>(i);
                if (s < clen) {
                    kk[i] = KeyTraits<DT>::phi(a.keys[t0 + cs + s]);
                    if constexpr (PAIRS) vv[i] = a.vals[t0 + cs + s];
                } else {
                    kk[i] = 0;
                    if constexpr (PAIRS) vv[i] = 0;
                }
            }
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int s = striped_slot<kRouteThreads, IT>(i);
                bb[i] = s < clen ? classify_key(kk[i], (uint32_t)(t0 + cs + s), lp, lut, sphi, stag) : P;
            }
            for (int shift = 0; shift < bbits; shift += 8) {
#pragma unroll
                for (int i = 0; i < IT; ++i) d[i] = (bb[i] >> shift) & 255u;
                Rank::rank(fx.rank, d, rk);
                for (int dd = tid; dd < 256; dd += kRouteThreads) fx.base[dd] = fx.rank.digit_tot[dd];
                __syncthreads();
                digit_excl_scan<kRouteThreads, 256>(fx.base, fx.tmp);
#pragma unroll
                for (int i = 0; i < IT; ++i) {
                    const uint32_t pos = fx.base[d[i]] + rk[i];
                    stage_k[pos] = kk[i];
                    if constexpr (PAIRS) stage_v[pos] = vv[i];
                    stage_b[pos] = bb[i];
                }
                __syncthreads();
                if (shift + 8 < bbits) {
#pragma unroll
                    for (int i = 0; i < IT; ++i) {
                        const int s = striped_slot<kRouteThreads, IT>(i);
                        kk[i] = stage_k[s];
                        if constexpr (PAIRS) vv[i] = stage_v[s];
                        bb[i] = stage_b[s];
                    }
                    __syncthreads();
                }
            }
            // staged keys are ordered by sub-bucket; find each run's first slot
            uint32_t seg[IT];
            uint32_t carry = 0;
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int s = striped_slot<kRouteThreads, IT>(i);
                const uint32_t b = stage_b[s];
                const bool head = s == 0 || stage_b[s - 1] != b;
                uint32_t x = head ? (uint32_t)s : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x = max(x, y);
                }
                x = max(x, carry);
                seg[i] = x;
                carry = __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) fx.warp_max[warp] = carry;
            __syncthreads();
            uint32_t pre = 0;
            for (int w = 0; w < warp; ++w) pre = max(pre, fx.warp_max[w]);
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int s = striped_slot<kRouteThreads, IT>(i);
                const uint32_t b = stage_b[s];
                seg[i] = max(seg[i], pre);
                if (b < P) {
                    const uint32_t idx = run[b] + (uint32_t)s - seg[i];
                    if (idx < a.cap) {
                        a.reg_keys[(int64_t)b * a.cap + idx] = stage_k[s];
                        if constexpr (PAIRS) a.reg_vals[(int64_t)b * a.cap + idx] = stage_v[s];
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int s = striped_slot<kRouteThreads, IT>(i);
                const uint32_t b = stage_b[s];
                const bool tail = s == kRouteChunk - 1 || stage_b[s + 1] != b;
                if (b < P && tail) run[b] += (uint32_t)s - seg[i] + 1;
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Sizes and offsets of the sub-buckets (inclusive prefix of the last tile),
// bucket sizes for the caller and the balance statistics (Lemma 5.1).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
bucket_finish_kernel(const uint32_t *state, int64_t tiles, uint32_t P, int64_t B, int64_t cap,
                     uint32_t *vsize, uint64_t *voff, int64_t *bucket_sizes, DevStatus *st) {
    __shared__ uint32_t tmp[40];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t *last = state + (tiles - 1) * (int64_t)P;
    const int64_t per = ((int64_t)P + 1023) / 1024;
    const int64_t lo = tid * per, hi = imin64(P, lo + per);
    uint64_t local = 0;
    uint32_t vmax = 0;
    for (int64_t v = lo; v < hi; ++v) {
        const uint32_t s = last[v] & kValMask;
        vsize[v] = s;
        local += s;
        vmax = max(vmax, s);
    }
    uint32_t wt;
    const uint32_t we = warp_excl_scan((uint32_t)local, &wt);
    if (lane == 31) tmp[warp] = wt;
    __syncthreads();
    if (warp == 0) {
        uint32_t t;
        const uint32_t e = warp_excl_scan(tmp[lane], &t);
        tmp[lane] = e;
    }
    __syncthreads();
    uint64_t runv = tmp[warp] + we;
    for (int64_t v = lo; v < hi; ++v) {
        voff[v] = runv;
        runv += vsize[v];
    }
    if (hi == P && lo < hi) voff[P] = runv;
    if (vmax > cap) {
        atomicExch(&st->overflow, 1);
        set_error(st, BSPS_ERR_BUCKET_OVERFLOW);
    }
    atomicMax(&st->max_vbucket, (unsigned long long)vmax);
    __syncthreads();
    const int64_t p = P / B;
    for (int64_t i = tid; i < p; i += 1024) {
        uint64_t s = 0;
        for (int64_t j = 0; j < B; ++j) s += vsize[i * B + j];
        if (bucket_sizes) bucket_sizes[i] = (int64_t)s;
        atomicMax(&st->max_bucket, (unsigned long long)s);
    }
}

template <int DT, bool PAIRS> static cudaError_t launch_route_t(const Ctx &c) {
    using K = typename KeyTraits<DT>::T;
    const Plan &p = c.pl;
    RouteArgs<K> a;
    a.keys = (const K *)c.keys_in;
    a.vals = c.vals_in;
    a.n = p.n;
    a.lutp = (const LutParams<K> *)c.ly.lutp;
    a.lut = c.ly.lut;
    a.vphi = (const K *)c.ly.vphi;
    a.vtag = c.ly.vtag;
    a.P = (uint32_t)p.P;
    a.tiles = p.tiles;
    a.state = c.ly.state;
    a.reg_keys = (K *)c.ly.reg_keys;
    a.reg_vals = c.ly.reg_vals;
    a.cap = p.cap;
    a.st = c.ly.status;
    const size_t smem = RouteSmemLayout<K, PAIRS>((uint32_t)p.P).total;
    auto kern = route_kernel<DT, PAIRS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRouteThreads, smem);
    const int64_t grid = imin64(p.tiles, (int64_t)max(occ, 1) * sms);
    kern<<<(unsigned)grid, kRouteThreads, smem, c.stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bucket_finish_kernel<<<1, 1024, 0, c.stream>>>(c.ly.state, p.tiles, (uint32_t)p.P, p.B, p.cap, c.ly.vsize,
                                                   c.ly.voff, c.bucket_sizes, c.ly.status);
    return cudaGetLastError();
}

cudaError_t launch_route(const Ctx &c) {
    const bool pr = c.pl.pairs != 0;
    switch (c.pl.dtype) {
    case BSPS_U32: return pr ? launch_route_t<BSPS_U32, true>(c) : launch_route_t<BSPS_U32, false>(c);
    case BSPS_I32: return pr ? launch_route_t<BSPS_I32, true>(c) : launch_route_t<BSPS_I32, false>(c);
    case BSPS_F32: return pr ? launch_route_t<BSPS_F32, true>(c) : launch_route_t<BSPS_F32, false>(c);
    default: return pr ? launch_route_t<BSPS_F64, true>(c) : launch_route_t<BSPS_F64, false>(c);
    }
}

size_t route_smem_bytes(const Plan &pl) {
    const uint32_t P = (uint32_t)pl.P;
    if (pl.key_bytes == 8)
        return pl.pairs ? RouteSmemLayout<uint64_t, true>(P).total : RouteSmemLayout<uint64_t, false>(P).total;
    return pl.pairs ? RouteSmemLayout<uint32_t, true>(P).total : RouteSmemLayout<uint32_t, false>(P).total;
}

} // namespace bsps
