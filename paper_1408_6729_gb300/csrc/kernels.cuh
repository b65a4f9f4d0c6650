// kernels.cuh -- the plan of one sort call, the workspace layout, and the
// host-side launchers of each step of the path.
#pragma once

#include "common.cuh"

namespace bsps {

struct MlpNorm;

// Number of cells of the radix index placed in front of the splitter tree.
constexpr int kLutBits = 14;
constexpr int kLutCells = 1 << kLutBits;

// Routing geometry (Fig. 1 steps 9-11).
constexpr int kRouteThreads = 1024;
constexpr int kRouteTile = 65536;                           // keys per look-back tile
template <typename K> constexpr int route_items() { return sizeof(K) == 8 ? 4 : 8; }
template <typename K> constexpr int route_chunk() { return kRouteThreads * route_items<K>(); }
constexpr size_t kRouteSmemBudget = 220 * 1024;

// Sample-sort geometry (Fig. 1 step 5).
constexpr int kLsdThreads = 512;
constexpr int kLsdItems = 16;
constexpr int kLsdTile = kLsdThreads * kLsdItems;

// Bucket / block sort geometry (Fig. 1 step 3, Fig. 2 step 12): 1024-thread
// CTAs, keys per thread of the on-chip segment sort.
constexpr int kSortThreads = 1024;
constexpr int kRunItems32 = 10;        // block sort with input-slot companion, 4-byte keys
constexpr int kRunItems64 = 8;         // ... 8-byte keys
constexpr int kBucketItems32 = 14;     // sub-bucket sort, keys only, 4-byte keys
constexpr int kBucketItems64 = 10;     // ... 8-byte keys
constexpr int kPairItems32 = 12;       // sub-bucket sort with payload slots, 4-byte keys
constexpr int kPairItems64 = 8;        // ... 8-byte keys
constexpr int kKeysItems32 = 20;       // throughput keys-only sort: 512 threads x 20 = 10240 keys per CTA
constexpr int kKeysItems64 = 10;       // ... 8-byte keys
constexpr int kKeysItems64Large = 20;  // ... 8-byte keys, one CTA per SM, for the larger sub-buckets
constexpr int kSlowThreads = 512;      // out-of-core sort of an oversized sub-bucket
constexpr int kSlowItems = 8;

// Where the radix index sends a key: cells of width 2^shift above `base`.
template <typename K> struct LutParams {
    K base;        // phi of the smallest splitter
    K span;        // phi(largest splitter) - base
    uint32_t shift;
    uint32_t nsplit; // number of splitters (vbuckets - 1)
};

template <typename K> struct LsdBuffers {
    K *phi[2];
    uint32_t *tag[2];
};

struct Plan {
    int64_t n, p, R, s, m, M, x, q, sample_size;
    int sampling, dtype, pairs, classify;
    int dup_off;       // keys compared by value alone (no tie-break by position)
    int merge;         // final step: merge of the sorted blocks' segments (Fig. 1 step 12)
    int seg_route;     // route by the sorted blocks' partition and segment copies (Fig. 1 steps 9-11)
    int keep_runs;     // the block sorts keep the sorted blocks (merge or seg_route)
    uint64_t seed;
    int64_t B;         // refine: sub-buckets per bucket
    int64_t P;         // vbuckets = p * B
    int64_t Q;         // sample records between consecutive splitters (q or s)
    int64_t cap;       // keys per sub-bucket region
    int run_cl;        // cluster size of the block sort (regular sampling)
    int bucket_cl;     // cluster size of the sub-bucket sort
    int64_t tiles;     // routing tiles
    int64_t lsd_tiles; // sample-sort tiles
    int lsd_npos;      // radix digit positions of a sample record
    int key_bytes;
    size_t ws_bytes;
};

// Device pointers into the caller's workspace (all 256-byte aligned).
struct Layout {
    DevStatus *status;
    void *sphi[2];          // sample record phi (ping-pong), key width
    uint32_t *stag[2];      // sample record tag (ping-pong)
    uint32_t *lsd_counts;   // lsd_tiles * 256
    uint32_t *lsd_hist;     // lsd_npos * 256
    int32_t *lsd_table;     // pass table of the sample sort
    void *vphi;             // P-1 sub-bucket splitters, phi
    uint32_t *vtag;         // P-1 sub-bucket splitters, tag
    uint16_t *lut;          // kLutCells + 1 (sub-bucket counts fit 16 bits)
    void *lutp;             // LutParams<K>
    uint32_t *state;        // tiles * P lookback words
    uint16_t *ids;          // tiles * kRouteTile sub-bucket ids (routing scratch)
    uint32_t *cursor;       // P keys routed per sub-bucket
    uint32_t *retry_flag;   // P: the keys-only sort gave the sub-bucket back
    uint32_t *retry_list;   // P: sub-buckets for the stable cluster sort
    uint32_t *run_retry;    // R: blocks the keys-only block sort gave back
    // learned classifier (classify == BSPS_LEARNED)
    float *mlp_params;                   // 1153
    float *mlp_part;                     // partial gradients of the training CTAs
    float *mlp_x, *mlp_y;                // training points
    int64_t *mlp_npts;
    struct MlpNorm *mlp_norm;
    void *mlp_opt;                       // gradient-descent state
    struct MlpTables *mlp_tables;        // the trained network's evaluation form
    float *mlp_ysplit;                   // the network's output for every splitter
    uint16_t *ylut;                      // index over the network's output (kYCells + 1)
    void *reg_keys;         // P * cap keys (phi), region v at v*cap
    uint32_t *reg_vals;     // P * cap payloads
    uint32_t *vsize;        // P sub-bucket sizes
    uint64_t *voff;         // P + 1 exclusive offsets
    uint32_t *slow_list;    // sub-buckets too large for the on-chip sort
    // the sorted blocks and their partition (keep_runs == 1)
    void *runs;                 // n keys (phi), block k's sorted keys at k*m
    uint32_t *runs_val;         // n payloads in the same order (pairs)
    uint32_t *rs_phi, *rs_tag;  // R * s: every block's own sample records, before the sample sort
    uint32_t *part;             // (P + 1) * R: c[k][v] at v * R + k
};

struct Ctx {
    Plan pl;
    Layout ly;
    const void *keys_in;
    const uint32_t *vals_in;
    void *keys_out;
    uint32_t *vals_out;
    int64_t *bucket_sizes;
    bsps_debug dbg;
    cudaStream_t stream;
};

// Internal record tag: the input position g for a key, n + k*M + j for the
// pad at local index j of virtual processor k; phi of a pad is all ones.
// (pad, phi, k*M+j) order == (phi', tag') order with these encodings.

// launchers (each returns cudaSuccess or the launch error)
cudaError_t launch_sample(const Ctx &c);          // Fig. 1 steps 3-4 / Fig. 3 step 4
cudaError_t launch_sample_sort(const Ctx &c);     // Fig. 1 step 5
cudaError_t launch_splitters(const Ctx &c);       // Fig. 1 steps 6-7
cudaError_t launch_route(const Ctx &c);           // Fig. 1 steps 9-11
cudaError_t launch_bucket_finish(const Ctx &c);   // sizes in cursor -> offsets, bucket sizes, statistics
cudaError_t launch_bucket_sort(const Ctx &c);     // Fig. 2 step 12
cudaError_t launch_debug(const Ctx &c);           // optional diagnostics
cudaError_t launch_mlp_train(const Ctx &c);       // learned classifier: training set, spline start, training,
                                                  // evaluation tables and the index over its output
int mlp_train_kernels();                          // kernels launch_mlp_train queues
size_t mlp_opt_bytes();

// Byte counts of dynamic shared memory (host side).
size_t route_smem_bytes(const Plan &pl);
bool msd_sample_sort(const Plan &p);                // MSD sample sort is launched (32-bit keys, large samples)
int run_keys_cluster(const Plan &p);               // keys-only block sort for regular sampling (0: not used)
bool counting_block_sort(const Ctx &c);            // kept blocks sorted by the counting sort (and tags recovered)
cudaError_t launch_route_keys(const Ctx &c);      // keys without payloads, one pass
// merge final step (Fig. 1 steps 9-12)
cudaError_t launch_merge_partition(const Ctx &c); // c[k][v] and the sub-bucket sizes (into cursor)
cudaError_t launch_segment_copy(const Ctx &c);    // the route as segment copies into the regions
cudaError_t launch_merge_buckets(const Ctx &c);   // gather + stable merge per bucket
int merge_cluster(const Plan &pl);                // CTAs per bucket for a bound pl.cap (0: too large)
int64_t merge_capacity(int cl);                   // keys a cluster of cl CTAs merges
int64_t merge_runs_max();                         // largest R
constexpr int64_t kSegRouteRunsMax = 16384;       // largest R of the segment-copy route (shared memory)
size_t route_keys_smem_bytes(const Plan &pl);
bool route_keys_splitters_in_smem(const Plan &pl);  // keys-only routing holds the splitters on chip

} // namespace bsps
