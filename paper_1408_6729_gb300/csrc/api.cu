// api.cu -- the C ABI: parameter resolution (the paper's defaults), the
// workspace layout, and the order of the steps on the stream.
#include <cmath>
#include <cstring>

#include "kernels.cuh"
#include "mlp.cuh"

namespace bsps {

static int64_t ceil_log2(int64_t n) {
    int64_t r = 0;
    while (((int64_t)1 << r) < n) ++r;
    return r;
}

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

static int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// keys one CTA of the sub-bucket sort holds
static int64_t cta_capacity(int key_bytes, bool slot) {
    if (slot) return (int64_t)kSortThreads * (key_bytes == 8 ? kPairItems64 : kPairItems32);
    return (int64_t)512 * (key_bytes == 8 ? kKeysItems64 : kKeysItems32);
}

// Resolve the parameters and the internal layout.  Defaults follow Sec. 6.1:
// regular oversampling uses s = r*p with r = ceil(lg lg n) (omega_n = lg lg n,
// Fig. 1 step 1); random oversampling uses s = 2 lg^2 n (omega_n^2 = lg n,
// Fig. 3 step 1), with lg n rounded up.
static int make_plan(int64_t n, int dtype, const bsps_params *prm, int pairs, Plan &pl) {
    if (!prm) return BSPS_ERR_INVALID_ARG;
    if (dtype < BSPS_U32 || dtype > BSPS_F64) return BSPS_ERR_UNSUPPORTED_DTYPE;
    if (n < 0 || prm->p < 1 || prm->s < 0 || prm->runs < 0 || prm->refine < 0 || prm->capacity_pct < 0)
        return BSPS_ERR_INVALID_ARG;
    if (prm->sampling != BSPS_REGULAR && prm->sampling != BSPS_RANDOM) return BSPS_ERR_INVALID_ARG;
    if (prm->classify != BSPS_TREE && prm->classify != BSPS_LEARNED) return BSPS_ERR_INVALID_ARG;
    if (prm->refine != 0 && !is_pow2(prm->refine)) return BSPS_ERR_INVALID_ARG;
    if (prm->final_step != BSPS_FINAL_SORT && prm->final_step != BSPS_FINAL_MERGE) return BSPS_ERR_INVALID_ARG;
    if (prm->duplicates != BSPS_DUP_TAGS && prm->duplicates != BSPS_DUP_OFF) return BSPS_ERR_INVALID_ARG;
    if (prm->final_step == BSPS_FINAL_MERGE &&
        (prm->sampling != BSPS_REGULAR || dtype == BSPS_F64 || prm->refine > 1 || prm->classify != BSPS_TREE))
        return BSPS_ERR_INVALID_ARG;
    if (n >= ((int64_t)1 << 30)) return BSPS_ERR_TOO_LARGE;
    std::memset(&pl, 0, sizeof(pl));
    pl.n = n;
    pl.p = prm->p;
    pl.R = prm->runs > 0 ? prm->runs : prm->p;
    pl.sampling = prm->sampling;
    pl.classify = prm->classify;
    pl.dup_off = prm->duplicates == BSPS_DUP_OFF;
    pl.merge = prm->final_step == BSPS_FINAL_MERGE;
    if (pl.merge && pl.R > merge_runs_max()) return BSPS_ERR_INVALID_ARG;
    pl.dtype = dtype;
    pl.pairs = pairs;
    // regular sampling of 4-byte keys routes as the paper does (Fig. 1 steps
    // 9-11): the sorted blocks are kept, partitioned by the splitters and copied
    // segment by segment -- no per-key classification
    pl.seg_route = !pl.merge && prm->sampling == BSPS_REGULAR && dtype != BSPS_F64 && prm->classify == BSPS_TREE &&
                   pl.R <= kSegRouteRunsMax;
    pl.keep_runs = pl.merge || pl.seg_route;
    pl.seed = prm->seed;
    pl.key_bytes = dtype == BSPS_F64 ? 8 : 4;
    if (prm->s > ((int64_t)1 << 31) || prm->runs > ((int64_t)1 << 30)) return BSPS_ERR_TOO_LARGE;
    const int64_t clg = n >= 2 ? ceil_log2(n) : 1;
    pl.m = (n + pl.R - 1) / pl.R;
    if (pl.sampling == BSPS_REGULAR) {
        int64_t r = 1;
        while (((int64_t)1 << r) < clg) ++r;
        pl.s = prm->s > 0 ? prm->s : r * pl.p;
        pl.M = pl.s * ((pl.m + pl.s - 1) / pl.s);
        if (pl.M == 0) pl.M = pl.s;
        pl.x = pl.M / pl.s;
        if ((pl.R * pl.s) % pl.p != 0 || pl.R * pl.s < pl.p) return BSPS_ERR_INVALID_ARG;
        pl.q = pl.R * pl.s / pl.p;
        pl.Q = pl.q;
        pl.sample_size = pl.R * pl.s;
        if (n + pl.R * pl.M >= ((int64_t)1 << 32)) return BSPS_ERR_TOO_LARGE;  // 32-bit pad tags
    } else {
        pl.s = prm->s > 0 ? prm->s : 2 * clg * clg;
        pl.M = pl.m;
        pl.x = 0;
        pl.q = pl.s;
        pl.Q = pl.s;
        pl.sample_size = pl.s * pl.p - 1;
    }
    if (pl.sample_size >= ((int64_t)1 << 31) || pl.p > 65535) return BSPS_ERR_TOO_LARGE;

    // sub-buckets: the smallest refinement whose expected size fits one
    // cluster's shared memory with head room for the sampling imbalance
    const int64_t cap_cta = cta_capacity(pl.key_bytes, pairs);
    auto headroom = [&](int64_t B) {
        return pl.sampling == BSPS_RANDOM ? 1.0 + 5.0 / std::sqrt((double)std::max<int64_t>(1, pl.Q / B))
                                          : 1.25;
    };
    int64_t B = pl.merge ? 1 : prm->refine;
    if (B == 0) {
        B = 1;
        while (B * 2 <= pl.Q && (double)n / (pl.p * B) * headroom(B) > 8.0 * cap_cta) B *= 2;
    }
    if (B > pl.Q) return BSPS_ERR_INVALID_ARG;
    pl.B = B;
    pl.P = pl.p * B;
    // the routing kernel keeps two words per sub-bucket in shared memory:
    // refine less (larger sub-buckets go to the slower sort tiers) if needed,
    // and also while its splitters would have to stay in global memory, as
    // long as the expected sub-bucket stays within 2.5 clusters' capacity
    while (prm->refine == 0 && pl.B > 1 && route_smem_bytes(pl) > 227 * 1024) {
        pl.B /= 2;
        pl.P = pl.p * pl.B;
    }
    while (prm->refine == 0 && pl.B > 1 && !pl.pairs && pl.key_bytes == 4 && !route_keys_splitters_in_smem(pl)) {
        Plan half = pl;
        half.B /= 2;
        half.P = half.p * half.B;
        if ((double)n / half.P * headroom(half.B) > 2.5 * 8.0 * cap_cta) break;
        pl = half;
    }
    B = pl.B;
    if (pl.P > 65535) return BSPS_ERR_TOO_LARGE;  // 16-bit sub-bucket ids
    const double expect = (double)n / pl.P * headroom(B);
    pl.bucket_cl = 8;
    for (int cl = 1; cl <= 8; cl *= 2)
        if (expect <= (double)cl * cap_cta) { pl.bucket_cl = cl; break; }

    if (pl.sampling == BSPS_REGULAR) {
        // Lemma 5.1, refined: a sub-bucket spans at most ceil(Q/B) sample
        // records, hence at most ceil(Q/B)*x + (R-1)*(x-1) + 1 records.
        const int64_t qb = (pl.Q + B - 1) / B;
        pl.cap = std::min<int64_t>(std::max<int64_t>(n, 1), qb * pl.x + (pl.R - 1) * (pl.x > 0 ? pl.x - 1 : 0) + 1);
        const int64_t cap_run = (int64_t)kSortThreads * (pl.key_bytes == 8 ? kRunItems64 : kRunItems32);
        pl.run_cl = 0;
        for (int cl = 1; cl <= 8; cl *= 2)
            if (pl.m <= cl * cap_run) { pl.run_cl = cl; break; }
        if (pl.run_cl == 0) return BSPS_ERR_TOO_LARGE;
    } else {
        const double pct = prm->capacity_pct > 0
                               ? prm->capacity_pct / 100.0
                               : 1.0 + 8.0 / std::sqrt((double)std::max<int64_t>(1, pl.Q / B));
        pl.cap = std::min<int64_t>(std::max<int64_t>(n, 1), (int64_t)std::ceil((double)n / pl.P * pct) + 64);
        pl.run_cl = 1;
    }
    if (pl.merge) {
        // one cluster merges a whole bucket: sized by the bound of Lemma 5.1
        pl.bucket_cl = merge_cluster(pl);
        if (pl.bucket_cl == 0) return BSPS_ERR_TOO_LARGE;
        pl.cap = merge_capacity(pl.bucket_cl);
    }
    pl.cap = (pl.cap + 3) & ~int64_t(3);  // 16-byte aligned regions
    if (!pl.merge && (double)pl.P * pl.cap >= 4.0e9) return BSPS_ERR_TOO_LARGE;
    pl.tiles = (n + kRouteTile - 1) / kRouteTile;
    pl.lsd_tiles = (pl.sample_size + kLsdTile - 1) / kLsdTile;
    pl.lsd_npos = 4 + pl.key_bytes;
    if (route_smem_bytes(pl) > 227 * 1024) return BSPS_ERR_TOO_LARGE;

    // workspace size
    int64_t o = 0;
    auto take = [&](int64_t bytes) { int64_t at = o; o = align_up(o + std::max<int64_t>(bytes, 1), 256); return at; };
    take(sizeof(DevStatus));
    const int64_t S = std::max<int64_t>(pl.sample_size, 1);
    take(S * pl.key_bytes); take(S * pl.key_bytes);
    take(S * 4); take(S * 4);
    take(std::max<int64_t>(pl.lsd_tiles, 1) * 256 * 4);
    take(16 * 256 * 4);
    take(64 * 4);
    take(pl.P * pl.key_bytes);
    take(pl.P * 4);
    take((kLutCells + 2) * 2);
    take(64);
    const bool look_back = pairs && !pl.keep_runs;
    take(look_back ? std::max<int64_t>(pl.tiles, 1) * pl.P * 4 : 0);
    take(look_back ? std::max<int64_t>(pl.tiles, 1) * kRouteTile * 2 : 0);
    take(pl.P * 4);
    take(pl.P * 4); take(pl.P * 4);
    take(pl.sampling == BSPS_REGULAR ? pl.R * 4 : 0);
    const int64_t region_keys = pl.merge ? 0 : pl.P * pl.cap;  // the merge reads the sorted blocks directly
    take(region_keys * pl.key_bytes + 64);
    take(pairs ? region_keys * 4 : 0);
    take(pl.P * 4);
    take((pl.P + 1) * 8);
    take(pl.P * 4);
    if (pl.keep_runs) {
        take(n * pl.key_bytes); take(pairs ? n * 4 : 0);
        take(pl.sample_size * 4); take(pl.sample_size * 4);
        take((pl.P + 1) * pl.R * 4);
    }
    if (pl.classify == BSPS_LEARNED) {
        take(kParams * 4);
        take((int64_t)kMlpGridMax * (kParams + 1) * 4);
        take(kMlpPointsMax * 4); take(kMlpPointsMax * 4);
        take(8);
        take(sizeof(MlpNorm));
        take((int64_t)mlp_opt_bytes());
        take(sizeof(MlpTables));
        take(std::max<int64_t>(pl.P, 1) * 4);
        take((kYCells + 2) * 2);
    }
    pl.ws_bytes = (size_t)o;
    return BSPS_OK;
}

static Layout make_layout(const Plan &pl, void *ws) {
    unsigned char *b = (unsigned char *)ws;
    int64_t o = 0;
    auto take = [&](int64_t bytes) { int64_t at = o; o = align_up(o + std::max<int64_t>(bytes, 1), 256); return (void *)(b + at); };
    Layout l;
    const int64_t S = std::max<int64_t>(pl.sample_size, 1);
    l.status = (DevStatus *)take(sizeof(DevStatus));
    l.sphi[0] = take(S * pl.key_bytes);
    l.sphi[1] = take(S * pl.key_bytes);
    l.stag[0] = (uint32_t *)take(S * 4);
    l.stag[1] = (uint32_t *)take(S * 4);
    l.lsd_counts = (uint32_t *)take(std::max<int64_t>(pl.lsd_tiles, 1) * 256 * 4);
    l.lsd_hist = (uint32_t *)take(16 * 256 * 4);
    l.lsd_table = (int32_t *)take(64 * 4);
    l.vphi = take(pl.P * pl.key_bytes);
    l.vtag = (uint32_t *)take(pl.P * 4);
    l.lut = (uint16_t *)take((kLutCells + 2) * 2);
    l.lutp = take(64);
    const bool look_back = pl.pairs && !pl.keep_runs;
    l.state = (uint32_t *)take(look_back ? std::max<int64_t>(pl.tiles, 1) * pl.P * 4 : 0);
    l.ids = (uint16_t *)take(look_back ? std::max<int64_t>(pl.tiles, 1) * kRouteTile * 2 : 0);
    l.cursor = (uint32_t *)take(pl.P * 4);
    l.retry_flag = (uint32_t *)take(pl.P * 4);
    l.retry_list = (uint32_t *)take(pl.P * 4);
    l.run_retry = (uint32_t *)take(pl.sampling == BSPS_REGULAR ? pl.R * 4 : 0);
    const int64_t region_keys = pl.merge ? 0 : pl.P * pl.cap;
    l.reg_keys = take(region_keys * pl.key_bytes + 64);
    l.reg_vals = (uint32_t *)take(pl.pairs ? region_keys * 4 : 0);
    l.vsize = (uint32_t *)take(pl.P * 4);
    l.voff = (uint64_t *)take((pl.P + 1) * 8);
    l.slow_list = (uint32_t *)take(pl.P * 4);
    if (pl.keep_runs) {
        l.runs = take(pl.n * pl.key_bytes);
        l.runs_val = (uint32_t *)take(pl.pairs ? pl.n * 4 : 0);
        l.rs_phi = (uint32_t *)take(pl.sample_size * 4);
        l.rs_tag = (uint32_t *)take(pl.sample_size * 4);
        l.part = (uint32_t *)take((pl.P + 1) * pl.R * 4);
    } else {
        l.runs = nullptr;
        l.runs_val = l.rs_phi = l.rs_tag = l.part = nullptr;
    }
    if (pl.classify == BSPS_LEARNED) {
        l.mlp_params = (float *)take(kParams * 4);
        l.mlp_part = (float *)take((int64_t)kMlpGridMax * (kParams + 1) * 4);
        l.mlp_x = (float *)take(kMlpPointsMax * 4);
        l.mlp_y = (float *)take(kMlpPointsMax * 4);
        l.mlp_npts = (int64_t *)take(8);
        l.mlp_norm = (MlpNorm *)take(sizeof(MlpNorm));
        l.mlp_opt = take((int64_t)mlp_opt_bytes());
        l.mlp_tables = (MlpTables *)take(sizeof(MlpTables));
        l.mlp_ysplit = (float *)take(std::max<int64_t>(pl.P, 1) * 4);
        l.ylut = (uint16_t *)take((kYCells + 2) * 2);
    } else {
        l.mlp_params = l.mlp_part = l.mlp_x = l.mlp_y = nullptr;
        l.mlp_npts = nullptr;
        l.mlp_norm = nullptr;
        l.mlp_opt = nullptr;
        l.mlp_tables = nullptr;
        l.mlp_ysplit = nullptr;
        l.ylut = nullptr;
    }
    return l;
}

static void to_public(const Plan &p, bsps_plan *out) {
    out->n = p.n; out->p = p.p; out->R = p.R; out->s = p.s; out->m = p.m; out->M = p.M; out->x = p.x;
    out->q = p.q; out->sample_size = p.sample_size; out->sampling = p.sampling; out->dtype = p.dtype;
    out->refine = p.B; out->vbuckets = p.P; out->capacity = p.cap; out->run_cluster = p.run_cl;
    out->bucket_cluster = p.bucket_cl; out->route_tiles = p.tiles; out->workspace_bytes = p.ws_bytes;
}

// Kernels one call launches (the sample sort launches all its pass slots;
// slots whose byte position is constant return at once).
static int kernels_per_call(const Ctx &c) {
    const Plan &pl = c.pl;
    int k = 1;                                   // sample (random draw or block sort)
    if (run_keys_cluster(pl)) k += 2;            // keys-only and few-values block samplers before the stable one
    if (counting_block_sort(c)) k += 1;          // the counting sort's tags
    if (pl.sampling == BSPS_RANDOM && pl.sample_size == 0) k = 0;
    k += 2 + (pl.lsd_tiles > 0 ? 3 * pl.lsd_npos : 0);  // histogram, pass table, passes
    if (msd_sample_sort(pl)) k += 4;                 // MSD histogram, plan, scatter, bin sorts
    k += 2;                                      // splitters, radix index
    if (pl.merge) return k + 3;                  // partition, bucket offsets, merge
    k += 2;                                      // routing (partition and segment copy: one more), bucket offsets
    if (pl.seg_route) k += 1;
    k += 3;                                      // copy or keys-only tier, cluster sort, out-of-core sort
    if (!pl.pairs && pl.key_bytes == 8 && pl.bucket_cl * 512 * kKeysItems64 < 8 * 512 * kKeysItems64Large &&
        pl.cap > (int64_t)pl.bucket_cl * 512 * kKeysItems64)
        k += 1;                                  // the larger keys-only tier
    if (pl.classify == BSPS_LEARNED) k += mlp_train_kernels();  // training set, start, Adam steps, tables, index
    return k;
}

static int debug_kernels(const Ctx &c) {
    const Plan &p = c.pl;
    int k = 0;
    if (c.dbg.sample && p.sample_size > 0) ++k;
    if (c.dbg.splitters && p.p > 1) ++k;
    if (c.dbg.bucket_of && p.n > 0) ++k;
    if (c.dbg.pad_sizes && p.sampling == BSPS_REGULAR && p.R * p.M > p.n) ++k;
    return k;
}

#define BSPS_CUDA(call)                                   \
    do {                                                  \
        if ((call) != cudaSuccess) return BSPS_ERR_CUDA;  \
    } while (0)

static int run(const void *keys_in, const uint32_t *vals_in, void *keys_out, uint32_t *vals_out, int64_t n,
               int32_t dtype, const bsps_params *prm, int64_t *bucket_sizes, const bsps_debug *dbg, void *ws,
               size_t ws_bytes, void *stream) {
    Ctx c;
    std::memset(&c, 0, sizeof(c));
    const int pairs = vals_in != nullptr;
    int rc = make_plan(n, dtype, prm, pairs, c.pl);
    if (rc) return rc;
    if (pairs && !vals_out) return BSPS_ERR_INVALID_ARG;
    if (n > 0 && (!keys_in || !keys_out)) return BSPS_ERR_INVALID_ARG;
    if (n > 0 && keys_in == keys_out) return BSPS_ERR_INVALID_ARG;
    if (pairs && (const void *)vals_in == (const void *)vals_out) return BSPS_ERR_INVALID_ARG;
    if (!ws || ws_bytes < c.pl.ws_bytes) return BSPS_ERR_WORKSPACE_TOO_SMALL;
    if (((uintptr_t)ws & 255) != 0) return BSPS_ERR_INVALID_ARG;
    c.ly = make_layout(c.pl, ws);
    c.keys_in = keys_in;
    c.vals_in = vals_in;
    c.keys_out = keys_out;
    c.vals_out = vals_out;
    c.bucket_sizes = bucket_sizes;
    if (dbg) c.dbg = *dbg;
    c.stream = (cudaStream_t)stream;
    BSPS_CUDA(cudaMemsetAsync(c.ly.status, 0, sizeof(DevStatus), c.stream));
    if (n == 0) {
        if (bucket_sizes) BSPS_CUDA(cudaMemsetAsync(bucket_sizes, 0, sizeof(int64_t) * c.pl.p, c.stream));
        if (dbg && dbg->pad_sizes) BSPS_CUDA(cudaMemsetAsync(dbg->pad_sizes, 0, sizeof(int64_t) * c.pl.p, c.stream));
        return BSPS_OK;
    }
    void *const *ev = dbg ? dbg->phase_events : nullptr;
    auto mark = [&](int i) { return ev ? cudaEventRecord((cudaEvent_t)ev[i], c.stream) : cudaSuccess; };
    if (c.pl.pairs && !c.pl.keep_runs)
        BSPS_CUDA(cudaMemsetAsync(c.ly.state, 0, (size_t)c.pl.tiles * c.pl.P * 4, c.stream));
    BSPS_CUDA(cudaMemsetAsync(c.ly.cursor, 0, (size_t)c.pl.P * 4, c.stream));
    if (!c.pl.pairs) BSPS_CUDA(cudaMemsetAsync(c.ly.retry_flag, 0, (size_t)c.pl.P * 4, c.stream));
    BSPS_CUDA(mark(0));
    BSPS_CUDA(launch_sample(c));
    if (c.pl.keep_runs) {  // every block's own sample records, for the partition (the sample sort reuses the buffer)
        BSPS_CUDA(cudaMemcpyAsync(c.ly.rs_phi, c.ly.sphi[0], (size_t)c.pl.sample_size * 4, cudaMemcpyDeviceToDevice,
                                  c.stream));
        BSPS_CUDA(cudaMemcpyAsync(c.ly.rs_tag, c.ly.stag[0], (size_t)c.pl.sample_size * 4, cudaMemcpyDeviceToDevice,
                                  c.stream));
    }
    BSPS_CUDA(mark(1));
    BSPS_CUDA(launch_sample_sort(c));
    BSPS_CUDA(mark(2));
    BSPS_CUDA(launch_splitters(c));
    if (c.pl.classify == BSPS_LEARNED) BSPS_CUDA(launch_mlp_train(c));
    BSPS_CUDA(mark(3));
    if (c.pl.keep_runs) {
        BSPS_CUDA(launch_merge_partition(c));
        BSPS_CUDA(launch_bucket_finish(c));
        if (c.pl.merge) {
            BSPS_CUDA(mark(4));
            BSPS_CUDA(launch_merge_buckets(c));
        } else {
            BSPS_CUDA(launch_segment_copy(c));
            BSPS_CUDA(mark(4));
            BSPS_CUDA(launch_bucket_sort(c));
        }
        if (dbg && dbg->partition)  // the rows of the p - 1 splitters among the sub-bucket splitters' rows
            BSPS_CUDA(cudaMemcpy2DAsync(dbg->partition, (size_t)c.pl.R * 4, c.ly.part, (size_t)(c.pl.B * c.pl.R * 4),
                                        (size_t)c.pl.R * 4, (size_t)(c.pl.p + 1), cudaMemcpyDeviceToDevice,
                                        c.stream));
    } else {
        BSPS_CUDA(launch_route(c));
        BSPS_CUDA(mark(4));
        BSPS_CUDA(launch_bucket_sort(c));
    }
    BSPS_CUDA(mark(5));
    if (dbg) BSPS_CUDA(launch_debug(c));
    if (dbg && dbg->launches) *dbg->launches = kernels_per_call(c) + debug_kernels(c);
    return BSPS_OK;
}

} // namespace bsps

using namespace bsps;

extern "C" {

int bsps_get_plan(int64_t n, int32_t dtype, const bsps_params *prm, int32_t with_payload, bsps_plan *out) {
    if (!out) return BSPS_ERR_INVALID_ARG;
    Plan pl;
    const int rc = make_plan(n, dtype, prm, with_payload != 0, pl);
    if (rc) return rc;
    to_public(pl, out);
    return BSPS_OK;
}

int bsps_workspace_size(int64_t n, int32_t dtype, const bsps_params *prm, int32_t with_payload, size_t *bytes) {
    if (!bytes) return BSPS_ERR_INVALID_ARG;
    Plan pl;
    const int rc = make_plan(n, dtype, prm, with_payload != 0, pl);
    if (rc) return rc;
    *bytes = pl.ws_bytes;
    return BSPS_OK;
}

int bsps_sort_keys(const void *d_keys_in, void *d_keys_out, int64_t n, int32_t dtype, const bsps_params *prm,
                   int64_t *d_bucket_sizes, void *d_ws, size_t ws_bytes, void *stream) {
    return run(d_keys_in, nullptr, d_keys_out, nullptr, n, dtype, prm, d_bucket_sizes, nullptr, d_ws, ws_bytes,
               stream);
}

int bsps_sort_pairs(const void *d_keys_in, const uint32_t *d_vals_in, void *d_keys_out, uint32_t *d_vals_out,
                    int64_t n, int32_t dtype, const bsps_params *prm, int64_t *d_bucket_sizes, void *d_ws,
                    size_t ws_bytes, void *stream) {
    if (n > 0 && (!d_vals_in || !d_vals_out)) return BSPS_ERR_INVALID_ARG;
    return run(d_keys_in, d_vals_in, d_keys_out, d_vals_out, n, dtype, prm, d_bucket_sizes, nullptr, d_ws,
               ws_bytes, stream);
}

int bsps_sort_debug(const void *d_keys_in, const uint32_t *d_vals_in, void *d_keys_out, uint32_t *d_vals_out,
                    int64_t n, int32_t dtype, const bsps_params *prm, int64_t *d_bucket_sizes,
                    const bsps_debug *dbg, void *d_ws, size_t ws_bytes, void *stream) {
    return run(d_keys_in, d_vals_in, d_keys_out, d_vals_out, n, dtype, prm, d_bucket_sizes, dbg, d_ws, ws_bytes,
               stream);
}

int bsps_read_stats(const void *d_ws, bsps_stats *stats, void *stream) {
    if (!d_ws || !stats) return BSPS_ERR_INVALID_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BSPS_ERR_CUDA;
    DevStatus st;
    if (cudaMemcpy(&st, d_ws, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return BSPS_ERR_CUDA;
    std::memset(stats, 0, sizeof(*stats));
    stats->status = st.error;
    stats->overflow = st.overflow;
    stats->timeouts = st.timeouts;
    stats->slow_buckets = st.slow_buckets;
    stats->max_bucket = (int64_t)st.max_bucket;
    stats->max_vbucket = (int64_t)st.max_vbucket;
    stats->mispredicted = (int64_t)st.mispredicted;
    stats->correction_steps = (int64_t)st.correction_steps;
    return stats->status;
}

const char *bsps_strerror(int status) {
    switch (status) {
    case BSPS_OK: return "ok";
    case BSPS_ERR_INVALID_ARG: return "invalid argument";
    case BSPS_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case BSPS_ERR_UNSUPPORTED_DTYPE: return "unsupported key type";
    case BSPS_ERR_BUCKET_OVERFLOW: return "a bucket exceeded its region";
    case BSPS_ERR_CUDA: return "CUDA error";
    case BSPS_ERR_DEVICE_TIMEOUT: return "a bounded device wait expired";
    case BSPS_ERR_TOO_LARGE: return "problem too large for the library's limits (see bsps_get_plan)";
    case BSPS_ERR_CAPTURE: return "the call cannot be captured into a caller's CUDA graph";
    default: return "unknown status";
    }
}

} // extern "C"
