// route.cu -- classification, per-bucket prefix and the routing permutation
// for keys with payloads (Fig. 1 steps 9-11; Fig. 2 steps 9-11), then the
// bucket offsets for both paths.
//
// One pass over the keys in HBM.  Tiles of kRouteTile keys are taken in
// order from an atomic ticket.  A tile first counts its keys per sub-bucket
// (Fig. 1 step 9), publishes the counts, and finds how many keys of each
// sub-bucket come before it by looking back over earlier tiles' published
// counts (a decoupled look-back computes the per-bucket prefix sums of
// Fig. 1 step 9, Lemma 4.2).  It then reads its keys again (from L2), stably
// sorts each chunk by sub-bucket in shared memory, and writes each
// sub-bucket's keys as one contiguous run into that sub-bucket's region.
// Inside every region keys keep their input order (Fig. 1 step 11), which
// makes the final per-bucket sort stable.
#include "classify.cuh"
#include "mlp.cuh"
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
    const uint16_t *lut;
    const K *vphi;
    const uint32_t *vtag;
    uint32_t P;
    int64_t tiles;
    uint32_t *state;
    uint32_t *cursor;   // keys routed so far per sub-bucket
    uint16_t *ids;      // sub-bucket of every key, written by phase A, read by phase B
    K *reg_keys;
    uint32_t *reg_vals;
    int64_t cap;
    DevStatus *st;
    const MlpTables *mlp_tables;  // learned classifier (nullable): the network's evaluation form
    const uint16_t *ylut;         // ... and the index over its output
    int64_t stall_tile;          // test hook: tile stall_tile - 1 never publishes (0: none)
    uint32_t spin_limit;         // polls of one bounded wait
    uint32_t tag_floor;          // a key's tag is max(position, tag_floor): n - 1 drops the tie-break
};

template <typename K> struct RouteFixed {
    typename BlockRank<kRouteThreads, route_items<K>(), 8>::Smem rank;
    uint32_t base[256];
    uint32_t tmp[40];
    uint32_t warp_max[kRouteThreads / 32];
    int64_t tile;
    LutParams<K> lp;
};

// Shared memory of the routing kernel.  The splitters' phi and tags (tags are
// read on phi ties only, which skewed inputs make common) live in shared
// memory when they fit next to the rest; the tags, then the phi, stay in
// global memory (L1-cached) otherwise.
template <typename K, bool LEARNED = false> struct RouteSmemLayout {
    size_t mlp, lut, sphi, stag, run, stage_k, stage_v, stage_b, total;
    bool sphi_in_smem, stag_in_smem;
    __host__ __device__ RouteSmemLayout(uint32_t P) {
        for (int pass = 0; pass < 3; ++pass) {  // splitters' phi and tags, phi only, neither
            sphi_in_smem = pass < 2;
            stag_in_smem = pass == 0;
            size_t o = (sizeof(RouteFixed<K>) + 15) & ~size_t(15);
            mlp = o;     o += LEARNED ? sizeof(MlpTables) : 0;
            o = (o + 15) & ~size_t(15);
            lut = o;     o += sizeof(uint16_t) * (kLutCells + 1);
            o = (o + 15) & ~size_t(15);
            sphi = o;    o += sphi_in_smem ? sizeof(K) * (P > 1 ? P - 1 : 1) : 0;
            o = (o + 15) & ~size_t(15);
            stag = o;    o += stag_in_smem ? sizeof(uint32_t) * (P > 1 ? P - 1 : 1) : 0;
            o = (o + 15) & ~size_t(15);
            run = o;     o += sizeof(uint32_t) * P;
            o = (o + 15) & ~size_t(15);
            stage_k = o; o += sizeof(K) * route_chunk<K>();
            stage_v = o; o += sizeof(uint32_t) * route_chunk<K>();
            stage_b = o; o += sizeof(uint16_t) * route_chunk<K>();
            total = o;
            if (total <= kRouteSmemBudget) break;
        }
    }
};

__device__ __forceinline__ void discard_l2_line(const void *p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

template <int DT, bool LEARNED>
__global__ void __launch_bounds__(kRouteThreads, 1) route_kernel(const RouteArgs<typename KeyTraits<DT>::T> a) {
    using K = typename KeyTraits<DT>::T;
    constexpr int IT = route_items<K>();
    constexpr int TH = kRouteThreads;
    constexpr int CH = route_chunk<K>();
    using Rank = BlockRank<TH, IT, 8>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RouteSmemLayout<K, LEARNED> L(a.P);
    MlpTables *mt = reinterpret_cast<MlpTables *>(smem_raw + L.mlp);
    uint32_t n_mis = 0, n_steps = 0;
    RouteFixed<K> &fx = *reinterpret_cast<RouteFixed<K> *>(smem_raw);
    uint16_t *lut = reinterpret_cast<uint16_t *>(smem_raw + L.lut);
    K *sphi_s = reinterpret_cast<K *>(smem_raw + L.sphi);
    const K *sphi = L.sphi_in_smem ? sphi_s : a.vphi;
    uint32_t *stag_s = reinterpret_cast<uint32_t *>(smem_raw + L.stag);
    const uint32_t *stag = L.stag_in_smem ? stag_s : a.vtag;
    uint32_t *run = reinterpret_cast<uint32_t *>(smem_raw + L.run);
    K *stage_k = reinterpret_cast<K *>(smem_raw + L.stage_k);
    uint32_t *stage_v = reinterpret_cast<uint32_t *>(smem_raw + L.stage_v);
    uint16_t *stage_b = reinterpret_cast<uint16_t *>(smem_raw + L.stage_b);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t P = a.P, nsplit = P - 1;

    // splitters and radix index into shared memory (Fig. 1 step 7, "broadcast")
    // (with the learned classifier: the index over the network's output)
    static_assert(kYCells == kLutCells, "the learned index takes the radix index's slot");
    const uint16_t *lut_src = LEARNED ? a.ylut : a.lut;
    for (int i = tid; i <= kLutCells; i += TH) lut[i] = lut_src[i];
    if (L.sphi_in_smem)
        for (uint32_t i = tid; i < nsplit; i += TH) sphi_s[i] = a.vphi[i];
    if (L.stag_in_smem)
        for (uint32_t i = tid; i < nsplit; i += TH) stag_s[i] = a.vtag[i];
    if constexpr (LEARNED) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(a.mlp_tables);
        uint32_t *dst = reinterpret_cast<uint32_t *>(mt);
        for (int k = tid; k < (int)(sizeof(MlpTables) / 4); k += TH) dst[k] = src[k];
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
        uint16_t *ids = a.ids + t0;

        // ---- classify and count per sub-bucket (Fig. 1 step 9) ----
        for (uint32_t b = tid; b < P; b += TH) run[b] = 0;
        __syncthreads();
        for (int64_t cs = 0; cs < tlen; cs += CH) {
            K kk[IT];
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int64_t e = cs + i * TH + tid;
                kk[i] = e < tlen ? a.keys[t0 + e] : K(0);
            }
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const int64_t e = cs + i * TH + tid;
                const bool ok = e < tlen;
                uint32_t b = 0xffffffffu;
                if constexpr (LEARNED) {
                    if (ok) {
                        uint32_t steps;
                        bool mis;
                        b = classify_learned<DT>(kk[i], max((uint32_t)(t0 + e), a.tag_floor), *mt, lut, nsplit,
                                                 sphi, stag, steps, mis);
                        n_mis += mis;
                        n_steps += steps;
                    }
                } else {
                    if (ok)
                        b = classify_key(KeyTraits<DT>::phi(kk[i]), max((uint32_t)(t0 + e), a.tag_floor), lp, lut,
                                         sphi, stag);
                }
                // keys of lane 0's bucket are counted with one atomic (runs
                // of equal buckets are common in skewed inputs)
                const uint32_t b0 = __shfl_sync(0xffffffffu, b, 0);
                const uint32_t same = __ballot_sync(0xffffffffu, ok && b == b0);
                if (ok) {
                    if (b != b0) atomicAdd(&run[b], 1u);
                    else if (lane == __ffs(same) - 1) atomicAdd(&run[b], (uint32_t)__popc(same));
                    ids[e] = (uint16_t)b;
                }
            }
        }
        __syncthreads();

        // ---- where this tile's keys go inside every sub-bucket region ----
        {
            // with payloads: input order is kept (Fig. 1 step 11), so every
            // tile needs the keys of each bucket in all earlier tiles -- the
            // p parallel prefix sums of Fig. 1 step 9 (Lemma 4.2), done as a
            // decoupled look-back over earlier tiles' published counts
            uint32_t *my = a.state + tile * P;
            const bool publish = tile + 1 != a.stall_tile;
            for (uint32_t b = tid; b < P; b += TH) {
                if (publish) st_volatile(&my[b], (tile == 0 ? kFlagP : kFlagA) | run[b]);
                if (run[b]) atomicAdd(&a.cursor[b], run[b]);
            }
            if (tile > 0) {
                for (uint32_t b = tid; b < P; b += TH) {
                    uint32_t excl = 0;
                    bool done = false;
                    for (int64_t t = tile - 1; t >= 0 && !done; t -= 8) {
                        uint32_t v[8];
#pragma unroll
                        for (int w = 0; w < 8; ++w) v[w] = t - w >= 0 ? ld_volatile(a.state + (t - w) * P + b) : kFlagP;
#pragma unroll
                        for (int w = 0; w < 8; ++w) {
                            if (done) break;
                            uint32_t x = v[w], polls = 0;
                            while ((x >> 30) == 0 && ++polls < a.spin_limit) {
                                // after any expired wait, nobody waits any more
                                if ((polls & 255) == 0 && ld_volatile((const uint32_t *)&a.st->timeouts) != 0) break;
                                __nanosleep(64);
                                x = ld_volatile(a.state + (t - w) * P + b);
                            }
                            if ((x >> 30) == 0) {
                                atomicAdd(&a.st->timeouts, 1);
                                set_error(a.st, BSPS_ERR_DEVICE_TIMEOUT);
                                done = true;
                                break;
                            }
                            excl += x & kValMask;
                            done = (x >> 30) == 2;
                        }
                    }
                    const uint32_t c = run[b];
                    if (publish) st_volatile(&my[b], kFlagP | ((excl + c) & kValMask));
                    run[b] = excl;
                    if ((uint64_t)excl + c > (uint64_t)a.cap) {
                        atomicExch(&a.st->overflow, 1);
                        set_error(a.st, BSPS_ERR_BUCKET_OVERFLOW);
                    }
                }
            } else {
                for (uint32_t b = tid; b < P; b += TH) {
                    if (run[b] > a.cap) {
                        atomicExch(&a.st->overflow, 1);
                        set_error(a.st, BSPS_ERR_BUCKET_OVERFLOW);
                    }
                    run[b] = 0;
                }
            }
        }
        __syncthreads();

        // ---- route (Fig. 1 step 11): each chunk is grouped by sub-bucket in
        //      shared memory and every sub-bucket run is written contiguously ----
        for (int64_t cs = 0; cs < tlen; cs += CH) {
            const int clen = (int)imin64(CH, tlen - cs);
            {
                // with payloads: stable partition by sub-bucket (LSD over its bits)
                K kk[IT];
                uint32_t vv[IT], bb[IT], d[IT], rk[IT];
#pragma unroll
                for (int i = 0; i < IT; ++i) {
                    const int s = striped_slot<TH, IT>(i);
                    const bool ok = s < clen;
                    kk[i] = ok ? KeyTraits<DT>::phi(a.keys[t0 + cs + s]) : K(0);
                    vv[i] = ok ? a.vals[t0 + cs + s] : 0u;
                    bb[i] = ok ? (uint32_t)ids[cs + s] : P;
                }
                for (int shift = 0; shift < bbits; shift += 8) {
#pragma unroll
                    for (int i = 0; i < IT; ++i) d[i] = (bb[i] >> shift) & 255u;
                    Rank::rank(fx.rank, d, rk);
                    for (int dd = tid; dd < 256; dd += TH) fx.base[dd] = fx.rank.digit_tot[dd];
                    __syncthreads();
                    digit_excl_scan<TH, 256>(fx.base, fx.tmp);
#pragma unroll
                    for (int i = 0; i < IT; ++i) {
                        const uint32_t pos = fx.base[d[i]] + rk[i];
                        stage_k[pos] = kk[i];
                        stage_v[pos] = vv[i];
                        stage_b[pos] = (uint16_t)bb[i];
                    }
                    __syncthreads();
                    if (shift + 8 < bbits) {
#pragma unroll
                        for (int i = 0; i < IT; ++i) {
                            const int s = striped_slot<TH, IT>(i);
                            kk[i] = stage_k[s];
                            vv[i] = stage_v[s];
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
                    const int s = striped_slot<TH, IT>(i);
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
                    const int s = striped_slot<TH, IT>(i);
                    const uint32_t b = stage_b[s];
                    seg[i] = max(seg[i], pre);
                    if (b < P) {
                        const uint32_t idx = run[b] + (uint32_t)s - seg[i];
                        if (idx < a.cap) {
                            a.reg_keys[(int64_t)b * a.cap + idx] = stage_k[s];
                            a.reg_vals[(int64_t)b * a.cap + idx] = stage_v[s];
                        }
                    }
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < IT; ++i) {
                    const int s = striped_slot<TH, IT>(i);
                    const uint32_t b = stage_b[s];
                    const bool tail = s == CH - 1 || stage_b[s + 1] != b;
                    if (b < P && tail) run[b] += (uint32_t)s - seg[i] + 1;
                }
                __syncthreads();
            }
        }
        // the sub-bucket ids of this tile are dead: drop them from L2 unwritten
        for (int64_t line = tid; line * 64 < tlen; line += TH) discard_l2_line(ids + line * 64);
    }
    if constexpr (LEARNED) {  // misprediction statistics of the learned classifier
        const uint32_t m = __reduce_add_sync(0xffffffffu, n_mis), st = __reduce_add_sync(0xffffffffu, n_steps);
        if (lane == 0 && (m | st)) {
            atomicAdd(&a.st->mispredicted, (unsigned long long)m);
            atomicAdd(&a.st->correction_steps, (unsigned long long)st);
        }
    }
}

// ---------------------------------------------------------------------------
// Sizes and offsets of the sub-buckets (inclusive prefix of the last tile),
// bucket sizes for the caller and the balance statistics (Lemma 5.1).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
bucket_finish_kernel(const uint32_t *cursor, uint32_t P, int64_t B, int64_t cap, uint32_t *vsize, uint64_t *voff,
                     int64_t *bucket_sizes, DevStatus *st) {
    __shared__ uint32_t tmp[40];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = ((int64_t)P + 1023) / 1024;
    const int64_t lo = tid * per, hi = imin64(P, lo + per);
    uint64_t local = 0;
    uint32_t vmax = 0;
    for (int64_t v = lo; v < hi; ++v) {
        const uint32_t s = cursor[v];
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

template <int DT, bool LEARNED> static cudaError_t launch_route_t(const Ctx &c) {
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
    a.cursor = c.ly.cursor;
    a.ids = c.ly.ids;
    a.reg_keys = (K *)c.ly.reg_keys;
    a.reg_vals = c.ly.reg_vals;
    a.cap = p.cap;
    a.st = c.ly.status;
    a.mlp_tables = c.ly.mlp_tables;
    a.ylut = c.ly.ylut;
    a.stall_tile = c.dbg.stall_tile;
    a.spin_limit = c.dbg.wait_polls ? c.dbg.wait_polls : kSpinLimit;
    a.tag_floor = c.pl.dup_off ? (uint32_t)(c.pl.n - 1) : 0u;
    const size_t smem = RouteSmemLayout<K, LEARNED>((uint32_t)p.P).total;
    auto kern = route_kernel<DT, LEARNED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRouteThreads, smem);
    const int64_t grid = imin64(p.tiles, (int64_t)max(occ, 1) * sms);
    kern<<<(unsigned)grid, kRouteThreads, smem, c.stream>>>(a);
    return cudaGetLastError();
}

template <int DT> static cudaError_t launch_route_d(const Ctx &c) {
    return c.pl.classify == BSPS_LEARNED ? launch_route_t<DT, true>(c) : launch_route_t<DT, false>(c);
}

static cudaError_t launch_route_pairs(const Ctx &c) {
    switch (c.pl.dtype) {
    case BSPS_U32: return launch_route_d<BSPS_U32>(c);
    case BSPS_I32: return launch_route_d<BSPS_I32>(c);
    case BSPS_F32: return launch_route_d<BSPS_F32>(c);
    default: return launch_route_d<BSPS_F64>(c);
    }
}

cudaError_t launch_route(const Ctx &c) {
    cudaError_t e = c.pl.pairs ? launch_route_pairs(c) : launch_route_keys(c);
    if (e != cudaSuccess) return e;
    return launch_bucket_finish(c);
}

// sub-bucket sizes (in cursor) -> sizes, output offsets, bucket sizes, maxima
cudaError_t launch_bucket_finish(const Ctx &c) {
    const Plan &p = c.pl;
    bucket_finish_kernel<<<1, 1024, 0, c.stream>>>(c.ly.cursor, (uint32_t)p.P, p.B, p.cap, c.ly.vsize, c.ly.voff,
                                                   c.bucket_sizes, c.ly.status);
    return cudaGetLastError();
}

size_t route_smem_bytes(const Plan &pl) {
    if (!pl.pairs) return route_keys_smem_bytes(pl);
    const uint32_t P = (uint32_t)pl.P;
    const bool l = pl.classify == BSPS_LEARNED;
    if (pl.key_bytes == 8) return l ? RouteSmemLayout<uint64_t, true>(P).total : RouteSmemLayout<uint64_t>(P).total;
    return l ? RouteSmemLayout<uint32_t, true>(P).total : RouteSmemLayout<uint32_t>(P).total;
}

} // namespace bsps
