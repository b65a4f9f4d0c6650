// route_keys.cu -- classification and the routing permutation for keys
// without payloads (Fig. 1 steps 9-11; Fig. 2 steps 9-11), in one pass.
//
// Without payloads the order of keys inside a bucket is free (equal keys
// cannot be told apart), so the per-bucket prefix of Fig. 1 step 9 need not
// follow input order: every chunk of kRkChunk keys reserves its run in each
// bucket region with one atomic on that bucket's cursor.  A chunk is loaded
// into registers with 16-byte loads, each key is classified once (Fig. 2
// step 9) and ranked inside the chunk with a shared-memory atomic, the chunk
// is grouped by bucket in shared memory, and every bucket's run is written
// contiguously into its region.  One CTA of 1024 threads per SM; chunks of
// 16K keys keep the reservations to about one per four keys.
#include "classify.cuh"
#include "mlp.cuh"

namespace bsps {

constexpr int kRkThreads = 1024;
constexpr int kEarly = 4;  // buckets per thread reserved before the grouping
constexpr size_t kRkSmemBudget = 227 * 1024;  // splitters in shared memory up to this size
// keys per thread (fewer with the network's registers in use).  8-byte keys
// with the learned classifier take chunks of 10K with the splitters in global
// memory (L1-cached): with thousands of sub-buckets the per-chunk work over
// all of them (scan, reservations) would otherwise weigh as much as the keys,
// and a key reads one or two splitters.  The splitter tree reads more (skewed
// keys crowd a few cells of the radix index) and keeps its splitters on chip
// with chunks of 8K.
template <typename K, bool LEARNED = false> constexpr int rk_items() {
    return sizeof(K) == 8 ? (LEARNED ? 10 : 8) : (LEARNED ? 8 : 16);
}
template <typename K, bool LEARNED = false> constexpr int rk_chunk() { return kRkThreads * rk_items<K, LEARNED>(); }

template <typename K> struct RouteKeysArgs {
    const K *keys;
    int64_t n;
    const LutParams<K> *lutp;
    const uint16_t *lut;
    const K *vphi;
    const uint32_t *vtag;
    uint32_t P;
    int64_t chunks;
    uint32_t *cursor;   // keys routed so far per sub-bucket
    K *reg_keys;
    int64_t cap;
    DevStatus *st;
    const MlpTables *mlp_tables;  // learned classifier (nullable): the network's evaluation form
    const uint16_t *ylut;         // ... and the index over its output
    uint32_t tag_floor;           // a key's tag is max(position, tag_floor): n - 1 drops the tie-break
};

// Shared memory: the radix index (with the learned classifier: the index over
// the network's output, in the same slot, and the network's tables), the
// splitters' phi (global memory, L1-cached, when they do not fit), per-bucket
// counts and write offsets, and the chunk grouped by bucket.
template <typename K, bool LEARNED> struct RouteKeysLayout {
    size_t mlp, lut, sphi, cnt, dlt, stage_k, stage_b, total;
    bool sphi_in_smem;
    __host__ __device__ RouteKeysLayout(uint32_t P) {
        for (int pass = 0; pass < 2; ++pass) {
            sphi_in_smem = pass == 0;
            size_t o = 64;  // LutParams
            mlp = o;     o += LEARNED ? sizeof(MlpTables) : 0;
            o = (o + 15) & ~size_t(15);
            lut = o;     o += sizeof(uint16_t) * (kLutCells + 2);
            o = (o + 15) & ~size_t(15);
            sphi = o;    o += sphi_in_smem ? sizeof(K) * (P > 1 ? P - 1 : 1) : 0;
            o = (o + 15) & ~size_t(15);
            cnt = o;     o += sizeof(uint32_t) * (P + 4);
            o = (o + 15) & ~size_t(15);
            dlt = o;     o += sizeof(uint32_t) * (P + 4);
            o = (o + 15) & ~size_t(15);
            stage_k = o; o += sizeof(K) * rk_chunk<K, LEARNED>();
            stage_b = o; o += sizeof(uint16_t) * rk_chunk<K, LEARNED>();
            o += 128;    // scan scratch
            total = o;
            if (total <= kRkSmemBudget) break;
        }
    }
};
static_assert(sizeof(LutParams<uint64_t>) <= 64, "radix index parameters fit their slot");

template <int DT, bool LEARNED>
__global__ void __launch_bounds__(kRkThreads, 1) route_keys_kernel(const RouteKeysArgs<typename KeyTraits<DT>::T> a) {
    using K = typename KeyTraits<DT>::T;
    constexpr int T = kRkThreads, IT = rk_items<K, LEARNED>(), CH = rk_chunk<K, LEARNED>(), V = 16 / (int)sizeof(K);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RouteKeysLayout<K, LEARNED> L(a.P);
    LutParams<K> &lps = *reinterpret_cast<LutParams<K> *>(smem_raw);
    MlpTables *mt = reinterpret_cast<MlpTables *>(smem_raw + L.mlp);
    uint16_t *lut = reinterpret_cast<uint16_t *>(smem_raw + L.lut);
    K *sphi_s = reinterpret_cast<K *>(smem_raw + L.sphi);
    const K *sphi = L.sphi_in_smem ? sphi_s : a.vphi;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem_raw + L.cnt);
    uint32_t *dlt = reinterpret_cast<uint32_t *>(smem_raw + L.dlt);
    K *stage_k = reinterpret_cast<K *>(smem_raw + L.stage_k);
    uint16_t *stage_b = reinterpret_cast<uint16_t *>(smem_raw + L.stage_b);
    uint32_t *tmp = reinterpret_cast<uint32_t *>(smem_raw + L.total - 128);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t P = a.P;
    static_assert(kYCells == kLutCells, "the learned index takes the radix index's slot");
    const uint16_t *lut_src = LEARNED ? a.ylut : a.lut;
    for (int i = tid; i <= kLutCells; i += T) lut[i] = lut_src[i];
    if (L.sphi_in_smem)
        for (uint32_t i = tid; i + 1 < P; i += T) sphi_s[i] = a.vphi[i];
    for (uint32_t b = tid; b < P; b += T) cnt[b] = 0;
    if constexpr (LEARNED) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(a.mlp_tables);
        uint32_t *dst = reinterpret_cast<uint32_t *>(mt);
        for (int q = tid; q < (int)(sizeof(MlpTables) / 4); q += T) dst[q] = src[q];
    }
    if (tid == 0) lps = *a.lutp;
    __syncthreads();
    const LutParams<K> lp = lps;
    const bool vec = ((uintptr_t)a.keys & 15) == 0;
    // buckets [b_lo, b_hi) are this thread's in the scan and the reservation
    const uint32_t per = (P + T - 1) / T;
    const uint32_t b_lo = min(P, tid * per), b_hi = min(P, b_lo + per);
    K kmin = all_ones<K>(), kmax = K(0);
    uint32_t n_mis = 0, n_steps = 0;

    // chunk keys into registers (key i of a thread is chunk key lidx(i))
    K kk[IT];
    auto load_chunk = [&](int64_t ch) {
        const int64_t e0 = ch * CH;
        const int nh = (int)imin64(CH, a.n - e0);
#pragma unroll
        for (int j = 0; j < IT / V; ++j) {
            const int q = (j * T + tid) * V;
            if (vec && q + V <= nh) {
                const uint4 w = __ldg(reinterpret_cast<const uint4 *>(a.keys + e0 + q));
                if constexpr (sizeof(K) == 4) {
                    kk[j * V + 0] = w.x; kk[j * V + 1] = w.y; kk[j * V + 2] = w.z; kk[j * V + 3] = w.w;
                } else {
                    kk[j * V + 0] = ((uint64_t)w.y << 32) | w.x;
                    kk[j * V + 1] = ((uint64_t)w.w << 32) | w.z;
                }
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) kk[j * V + e] = q + e < nh ? a.keys[e0 + q + e] : K(0);
            }
        }
    };
    if ((int64_t)blockIdx.x < a.chunks) load_chunk(blockIdx.x);

    for (int64_t ch = blockIdx.x; ch < a.chunks; ch += gridDim.x) {
        const int64_t e0 = ch * CH;
        const int nh = (int)imin64(CH, a.n - e0);
        // ---- classify (Fig. 2 step 9) and rank inside the chunk ----
        uint32_t br[IT];  // bucket << 16 | rank inside the chunk (bucket P: no key)
        bool agg = true;  // warp-uniform: merge the atomics of lanes sharing lane 0's bucket
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int q = ((i / V) * T + tid) * V + i % V;
            const bool ok = q < nh;
            const K raw = kk[i], ph = KeyTraits<DT>::phi(raw);
            kk[i] = ph;
            uint32_t b = P;
            if (ok) {
                const uint32_t g = max((uint32_t)(e0 + q), a.tag_floor);  // tag: input position
                if constexpr (LEARNED) {
                    uint32_t steps;
                    bool mis;
                    b = classify_learned<DT>(raw, g, *mt, lut, P - 1, sphi, a.vtag, steps, mis);
                    n_mis += mis;
                    n_steps += steps;
                } else {
                    b = classify_key(ph, g, lp, lut, sphi, a.vtag);
                }
                kmin = ph < kmin ? ph : kmin;
                kmax = ph > kmax ? ph : kmax;
            }
            // keys of lane 0's bucket are ranked with one atomic (runs of equal
            // buckets are common in skewed inputs); the warp keeps doing so in
            // this chunk only if its first two items had such runs
            uint32_t r = 0;
            if (i < 2 || agg) {
                const uint32_t b0 = __shfl_sync(0xffffffffu, b, 0);
                const uint32_t same = __ballot_sync(0xffffffffu, ok && b == b0);
                if (i == 0) agg = __popc(same) > 1;
                if (i == 1) agg |= __popc(same) > 1;
                if (ok) {
                    if (b != b0) {
                        r = atomicAdd(&cnt[b], 1u);
                    } else {
                        const int leader = __ffs(same) - 1;
                        uint32_t r0 = 0;
                        if (lane == leader) r0 = atomicAdd(&cnt[b], (uint32_t)__popc(same));
                        r = __shfl_sync(same, r0, leader) + __popc(same & lanemask_lt());
                    }
                }
            } else if (ok) {
                r = atomicAdd(&cnt[b], 1u);
            }
            br[i] = b << 16 | r;
        }
        __syncthreads();
        // ---- where each bucket starts inside the chunk ----
        uint32_t local = 0;
        for (uint32_t b = b_lo; b < b_hi; ++b) local += cnt[b];
        uint32_t wtot;
        const uint32_t wex = warp_excl_scan(local, &wtot);
        if (lane == 31) tmp[warp] = wtot;
        __syncthreads();
        if (warp == 0) {
            const uint32_t y = lane < T / 32 ? tmp[lane] : 0u;
            uint32_t t;
            const uint32_t ye = warp_excl_scan(y, &t);
            if (lane < T / 32) tmp[lane] = ye;
        }
        __syncthreads();
        uint32_t run = tmp[warp] + wex;
        // the first kEarly of my buckets reserve their runs now, so that the
        // atomics' round trip overlaps the grouping below
        uint32_t at_e[kEarly];
#pragma unroll
        for (int j = 0; j < kEarly; ++j) {
            const uint32_t b = b_lo + j;
            at_e[j] = 0;
            if (b < b_hi) {
                const uint32_t c = cnt[b];
                cnt[b] = run;  // start of the bucket inside the chunk
                dlt[b] = c;
                run += c;
                if (c) at_e[j] = atomicAdd(&a.cursor[b], c);
            }
        }
        for (uint32_t b = b_lo + kEarly; b < b_hi; ++b) {
            const uint32_t c = cnt[b];
            cnt[b] = run;
            dlt[b] = c;
            run += c;
        }
        __syncthreads();
        // ---- group the chunk by bucket ----
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const uint32_t b = br[i] >> 16;
            if (b < P) {
                const uint32_t pos = cnt[b] + (br[i] & 0xffffu);
                stage_k[pos] = kk[i];
                stage_b[pos] = (uint16_t)b;
            }
        }
        // the next chunk's keys load while this one is reserved and written
        if (ch + gridDim.x < a.chunks) load_chunk(ch + gridDim.x);
        // ---- reserve each bucket's run: one atomic per bucket and chunk ----
        auto reserved = [&](uint32_t b, uint32_t c, uint32_t at) {
            if ((uint64_t)at + c > (uint64_t)a.cap) {
                atomicExch(&a.st->overflow, 1);
                set_error(a.st, BSPS_ERR_BUCKET_OVERFLOW);
            }
            dlt[b] = at - cnt[b];  // region slot of chunk position s: dlt[b] + s
        };
#pragma unroll
        for (int j = 0; j < kEarly; ++j)
            if (b_lo + j < b_hi) reserved(b_lo + j, dlt[b_lo + j], at_e[j]);
        for (uint32_t g0 = b_lo + kEarly; g0 < b_hi; g0 += 8) {
            uint32_t c8[8], at[8];  // eight reservations in flight at a time
#pragma unroll
            for (int j = 0; j < 8; ++j) c8[j] = g0 + j < b_hi ? dlt[g0 + j] : 0u;
#pragma unroll
            for (int j = 0; j < 8; ++j) at[j] = c8[j] ? atomicAdd(&a.cursor[g0 + j], c8[j]) : 0u;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (g0 + j < b_hi) reserved(g0 + j, c8[j], at[j]);
        }
        __syncthreads();
        // ---- every bucket's run, contiguously into its region ----
        for (int s = tid; s < nh; s += T) {
            const uint32_t b = stage_b[s];
            const uint32_t idx = dlt[b] + (uint32_t)s;
            if (idx < a.cap) a.reg_keys[(int64_t)b * a.cap + idx] = stage_k[s];
        }
        for (uint32_t b = b_lo; b < b_hi; ++b) cnt[b] = 0;
        __syncthreads();
    }
    // smallest and largest key: outer bounds of the first and last sub-bucket
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const K x = __shfl_xor_sync(0xffffffffu, kmin, o), y = __shfl_xor_sync(0xffffffffu, kmax, o);
        kmin = x < kmin ? x : kmin;
        kmax = y > kmax ? y : kmax;
    }
    if (lane == 0 && kmin <= kmax) {
        atomicMax(&a.st->ext_min_inv, ~(unsigned long long)kmin);
        atomicMax(&a.st->ext_max, (unsigned long long)kmax);
    }
    if constexpr (LEARNED) {
        const uint32_t m = __reduce_add_sync(0xffffffffu, n_mis), stp = __reduce_add_sync(0xffffffffu, n_steps);
        if (lane == 0 && (m | stp)) {
            atomicAdd(&a.st->mispredicted, (unsigned long long)m);
            atomicAdd(&a.st->correction_steps, (unsigned long long)stp);
        }
    }
}

template <int DT, bool LEARNED> static cudaError_t launch_t(const Ctx &c) {
    using K = typename KeyTraits<DT>::T;
    const Plan &p = c.pl;
    RouteKeysArgs<K> a;
    a.keys = (const K *)c.keys_in;
    a.n = p.n;
    a.lutp = (const LutParams<K> *)c.ly.lutp;
    a.lut = c.ly.lut;
    a.vphi = (const K *)c.ly.vphi;
    a.vtag = c.ly.vtag;
    a.P = (uint32_t)p.P;
    a.chunks = (p.n + rk_chunk<K, LEARNED>() - 1) / rk_chunk<K, LEARNED>();
    a.cursor = c.ly.cursor;
    a.reg_keys = (K *)c.ly.reg_keys;
    a.cap = p.cap;
    a.st = c.ly.status;
    a.mlp_tables = c.ly.mlp_tables;
    a.ylut = c.ly.ylut;
    a.tag_floor = c.pl.dup_off ? (uint32_t)(c.pl.n - 1) : 0u;
    if (a.chunks == 0) return cudaSuccess;
    const size_t smem = RouteKeysLayout<K, LEARNED>((uint32_t)p.P).total;
    auto kern = route_keys_kernel<DT, LEARNED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRkThreads, smem);
    const int64_t grid = imin64(a.chunks, (int64_t)max(occ, 1) * sms);
    kern<<<(unsigned)grid, kRkThreads, smem, c.stream>>>(a);
    return cudaGetLastError();
}

template <int DT> static cudaError_t launch_d(const Ctx &c) {
    return c.pl.classify == BSPS_LEARNED ? launch_t<DT, true>(c) : launch_t<DT, false>(c);
}

cudaError_t launch_route_keys(const Ctx &c) {
    switch (c.pl.dtype) {
    case BSPS_U32: return launch_d<BSPS_U32>(c);
    case BSPS_I32: return launch_d<BSPS_I32>(c);
    case BSPS_F32: return launch_d<BSPS_F32>(c);
    default: return launch_d<BSPS_F64>(c);
    }
}

size_t route_keys_smem_bytes(const Plan &pl) {
    const uint32_t P = (uint32_t)pl.P;
    const bool l = pl.classify == BSPS_LEARNED;
    if (pl.key_bytes == 8) return l ? RouteKeysLayout<uint64_t, true>(P).total : RouteKeysLayout<uint64_t, false>(P).total;
    return l ? RouteKeysLayout<uint32_t, true>(P).total : RouteKeysLayout<uint32_t, false>(P).total;
}

bool route_keys_splitters_in_smem(const Plan &pl) {
    const uint32_t P = (uint32_t)pl.P;
    const bool l = pl.classify == BSPS_LEARNED;
    if (pl.key_bytes == 8) return l ? RouteKeysLayout<uint64_t, true>(P).sphi_in_smem : RouteKeysLayout<uint64_t, false>(P).sphi_in_smem;
    return l ? RouteKeysLayout<uint32_t, true>(P).sphi_in_smem : RouteKeysLayout<uint32_t, false>(P).sphi_in_smem;
}

} // namespace bsps
