/*
 * bspsort.h -- C ABI of the GB300 (sm_103a) BSP sample sort.
 *
 * The library implements the data-parallel path of the BSP sample sorts of
 * Gerbessiotis & Siniolakis, "BSP Sorting: An experimental Study":
 *   Sort_Det_BSP  (Fig. 1, Sec. 5.1)  -- regular (deterministic) oversampling
 *   Sort_IRan_BSP (Fig. 3, Sec. 5.2)  -- random oversampling
 * with the duplicate-key handling of Sec. 5.1.1.  On one GPU the p BSP
 * processors become p buckets.  With random oversampling every key is
 * classified against the p-1 splitters (Fig. 2 step 9) and routed once
 * through HBM in input order (Fig. 1 step 11).  With regular oversampling of
 * 4-byte keys the blocks sorted for the sample are kept, every splitter is
 * located in every sorted block (Fig. 1 step 9) and each bucket's segments
 * are copied in block order (steps 10-11).  Each bucket is then sorted in
 * on-chip memory (Fig. 2 step 12), or -- BSPS_FINAL_MERGE -- its sorted
 * segments are merged (Fig. 1 step 12).
 *
 * Conventions shared by every entry point
 *  - Pointers named d_* are DEVICE pointers owned by the caller; the library
 *    never allocates, frees or retains them.  h_* pointers are host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call is asynchronous and stream-ordered; only bsps_read_stats()
 *    synchronises (the stream it is given).
 *  - Key order: a key's bit pattern is mapped to an unsigned integer phi
 *    (uint32: identity; int32: flip the sign bit; float32/float64: IEEE 754
 *    totalOrder, i.e. -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN) and
 *    ties are broken by input position (Sec. 5.1.1: processor id, then local
 *    index).  The output is the stable sort in that order.
 *  - Return value: BSPS_OK (0) or a negative BSPS_ERR_* code.  Argument
 *    errors are detected on the host before anything is launched.  Errors
 *    found on the device (bucket overflow, a bounded wait that expired) are
 *    recorded in the workspace and returned by bsps_read_stats().
 *  - In-place use (input == output) is rejected.  Inputs are never modified.
 */
#ifndef BSPSORT_H
#define BSPSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* key types */
typedef enum { BSPS_U32 = 0, BSPS_I32 = 1, BSPS_F32 = 2, BSPS_F64 = 3 } bsps_dtype;

/* oversampling: Sort_Det_BSP (Fig. 1) or Sort_IRan_BSP (Fig. 3) */
typedef enum { BSPS_REGULAR = 0, BSPS_RANDOM = 1 } bsps_sampling;

/* classification of keys against the splitters (Fig. 2 step 9) */
typedef enum { BSPS_TREE = 0, BSPS_LEARNED = 1 } bsps_classify;

/* the final step: sort every bucket (Fig. 2 step 12), or keep the sorted
 * blocks and merge each bucket's segments (Fig. 1 steps 9-12) */
typedef enum { BSPS_FINAL_SORT = 0, BSPS_FINAL_MERGE = 1 } bsps_final;

/* duplicate keys: ties broken by input position (Sec. 5.1.1), or keys
 * compared by value alone (the paper's version without duplicate handling) */
typedef enum { BSPS_DUP_TAGS = 0, BSPS_DUP_OFF = 1 } bsps_duplicates;

#define BSPS_OK 0
#define BSPS_ERR_INVALID_ARG (-1)
#define BSPS_ERR_WORKSPACE_TOO_SMALL (-2)
#define BSPS_ERR_UNSUPPORTED_DTYPE (-3)
#define BSPS_ERR_BUCKET_OVERFLOW (-4)
#define BSPS_ERR_CUDA (-5)
#define BSPS_ERR_DEVICE_TIMEOUT (-6)
#define BSPS_ERR_TOO_LARGE (-7)
#define BSPS_ERR_CAPTURE (-8)  /* bsps_sort_batched: the stream is being captured */

/*
 * Parameters, as the paper states them.
 *   p         number of buckets (the paper's processors), >= 1.
 *   runs      R, the number of virtual processors holding contiguous blocks of
 *             ceil(n/R) keys (regular mode); 0 -> R = p, as in the paper.
 *   s         oversampling factor.  Regular mode: samples per block (Fig. 1
 *             step 4, s = r*p); 0 -> r = ceil(lg lg n) (Sec. 6.1).  Random
 *             mode: the sample has s*p - 1 keys (Fig. 3 step 4); 0 -> s = 2 *
 *             ceil(lg n)^2 (Sec. 6.1, omega_n^2 = lg n).
 *   sampling  bsps_sampling.
 *   classify  bsps_classify.
 *   seed      random-mode sample stream: draw j is word (j mod 4) of
 *             Philox4x64-10 with key (seed, 0) and counter (floor(j/4),0,0,0);
 *             the sampled position is floor(draw * n / 2^64).
 *   refine    internal sub-bucket factor (power of two; 0 -> automatic).  It
 *             changes neither the splitters nor any result, only how finely
 *             buckets are cut before the on-chip sort.
 *   capacity_pct  random mode: capacity of each bucket region in percent of
 *             the mean sub-bucket size (0 -> automatic).  Regular mode ignores
 *             it and uses the exact bound of Lemma 5.1.
 *   final     bsps_final.  BSPS_FINAL_MERGE ends Sort_Det_BSP as the paper
 *             does: the blocks sorted for the regular sample (Fig. 1 step 3)
 *             are kept, every splitter is located in every sorted block by
 *             binary search (step 9: block k's segment of bucket i is
 *             [c[k][i], c[k][i+1])), and each bucket's segments, taken in
 *             block order (step 11), are merged stably, ties going to the
 *             earlier block (step 12; Sec. 5.1.1).  The results are those of
 *             BSPS_FINAL_SORT.  It requires regular sampling, 4-byte keys,
 *             R <= 8192, refine 0 or 1 and tree classification
 *             (BSPS_ERR_INVALID_ARG otherwise), and a bucket bound of Lemma
 *             5.1 of at most 126,976 keys (BSPS_ERR_TOO_LARGE otherwise).
 *   duplicates  bsps_duplicates.  BSPS_DUP_OFF compares keys by value
 *             alone: a key goes to bucket #{i : phi(S_i) <= phi(key)}, every
 *             key equal to a splitter in the highest such bucket.  It is the
 *             baseline against which the paper measures the cost of its
 *             duplicate handling (Sec. 6.1, Sec. 6.4).  The sorted output is
 *             unchanged; bucket sizes differ when keys repeat, and the bounds
 *             of Lemma 5.1 and Claim 5.1 no longer hold, so many equal keys
 *             overflow a bucket (BSPS_ERR_BUCKET_OVERFLOW from
 *             bsps_read_stats).
 */
typedef struct {
    int32_t p;
    int32_t runs;
    int64_t s;
    int32_t sampling;
    int32_t classify;
    uint64_t seed;
    int32_t refine;
    int32_t capacity_pct;
    int32_t final_step;
    int32_t duplicates;
} bsps_params;

/* A sample or splitter record of the total order: (pad, phi, tag), tag =
 * k*M + j for the key at local index j of virtual processor k (Sec. 5.1.1);
 * pads (Lemma 5.1's padding) have phi = 2^64-1 and pad = 1. */
typedef struct {
    uint64_t phi;
    uint64_t tag;
    uint32_t pad;
    uint32_t reserved;
} bsps_record;

/* Resolved parameters of one call (filled by bsps_get_plan). */
typedef struct {
    int64_t n, p, R, s, m, M, x, q, sample_size;
    int32_t sampling, dtype;
    int64_t refine;          /* sub-buckets per bucket */
    int64_t vbuckets;        /* p * refine */
    int64_t capacity;        /* keys per sub-bucket region */
    int32_t run_cluster;     /* CTAs per block sort (regular mode) */
    int32_t bucket_cluster;  /* CTAs per sub-bucket sort */
    int64_t route_tiles;
    size_t workspace_bytes;
} bsps_plan;

/* Device-side statistics and errors of the last call on a workspace. */
typedef struct {
    int32_t status;          /* BSPS_OK or the first device-side error */
    int32_t overflow;        /* nonzero if a bucket exceeded its region */
    int32_t timeouts;        /* bounded waits that expired */
    int32_t slow_buckets;    /* sub-buckets sorted by the out-of-core path */
    int64_t max_bucket;      /* largest bucket, real keys only */
    int64_t max_vbucket;     /* largest sub-bucket */
    int64_t mispredicted;    /* learned classifier: keys whose prediction was corrected */
    int64_t correction_steps;/* learned classifier: total search steps of the corrections */
} bsps_stats;

/* Optional diagnostics; every field may be NULL / 0.
 *   sample, splitters, bucket_of, pad_sizes: DEVICE buffers the call fills.
 *   phase_events: BSPS_PHASES cudaEvent_t handles (created by the caller) that
 *     the call records on its stream at the phase boundaries: before sampling,
 *     after sampling, after the sample sort, after splitter selection, after
 *     routing, after the bucket sort.
 *   launches: HOST int32 that receives the number of kernels the call launched.
 *   stall_tile, wait_polls: test hooks of the bounded waits (Sec. 5.1: the
 *     prefix step depends on every earlier processor).  With payloads,
 *     routing tile stall_tile - 1 never publishes its per-bucket counts
 *     (0: every tile publishes), so the later tiles' look-back waits on it
 *     expire; wait_polls bounds the polls of one wait (0: the default bound,
 *     about a second).  An expired wait records BSPS_ERR_DEVICE_TIMEOUT,
 *     which bsps_read_stats returns; the call's output is then undefined but
 *     every access stays inside the caller's buffers.
 *   partition: a DEVICE buffer of (p+1)*R uint32 that receives the partition
 *     of Fig. 1 step 9 when the call keeps the sorted blocks (regular
 *     sampling of 4-byte keys with the tree classifier and R <= 16384, or
 *     BSPS_FINAL_MERGE): entry i*R + k is the number of keys of sorted block
 *     k that precede splitter S_i (pads excluded; row 0 is 0, row p the
 *     block's key count); untouched otherwise. */
#define BSPS_PHASES 6
typedef struct {
    bsps_record *sample;     /* plan.sample_size records, sorted */
    bsps_record *splitters;  /* p-1 records */
    int32_t *bucket_of;      /* n bucket ids, by input position */
    int64_t *pad_sizes;      /* p pad counts (regular mode) */
    void *const *phase_events;
    int32_t *launches;
    float *mlp_params;       /* learned classifier: the 1153 trained parameters */
    float *mlp_loss;         /* learned classifier: training loss before and after */
    int32_t stall_tile;      /* test hook (see above); 0: none */
    uint32_t wait_polls;     /* test hook (see above); 0: the default bound */
    uint32_t *partition;     /* (p+1)*R entries (see above) */
} bsps_debug;

/*
 * bsps_get_plan -- resolve the paper's defaults and the internal layout.
 * with_payload: 1 if 32-bit payloads travel with the keys.
 * Returns BSPS_ERR_INVALID_ARG when p < 1, n < 0, s < 0, regular mode has
 * R*s not a multiple of p (the splitter stride q = R*s/p of Fig. 1 step 6
 * must be an integer), or refine is not a power of two; BSPS_ERR_TOO_LARGE
 * when n >= 2^30, s > 2^31 or runs > 2^30, the padded key count n + R*M
 * reaches 2^32 (32-bit tags), the sample reaches 2^31 records, p or the
 * sub-bucket count p*refine exceeds 65535 (16-bit ids), in regular mode a
 * block of ceil(n/R) keys exceeds the block sort's largest cluster (81,920
 * keys of 4 bytes, 65,536 of 8), the bucket regions exceed 4e9 keys, or the
 * routing kernel's shared memory (counters per sub-bucket, the radix index,
 * a staging chunk) exceeds 227 KB for p*refine sub-buckets: with refine = 0
 * the refinement is lowered first, so this limits p itself to about 12,600
 * for 4-byte keys without payloads (about 24,700 with payloads).
 */
int bsps_get_plan(int64_t n, int32_t dtype, const bsps_params *prm, int32_t with_payload,
              bsps_plan *out);

/* bsps_workspace_size -- bytes of device workspace the sort calls need. */
int bsps_workspace_size(int64_t n, int32_t dtype, const bsps_params *prm, int32_t with_payload,
                        size_t *bytes);

/*
 * bsps_sort_keys -- sort n keys (Fig. 1 / Fig. 3 with per-key classification).
 *   d_keys_in      n keys (4 or 8 bytes each, per dtype)
 *   d_keys_out     n keys, sorted; must not alias d_keys_in
 *   d_bucket_sizes p int64 counts of keys per bucket (nullable)
 *   d_ws, ws_bytes workspace of at least bsps_workspace_size() bytes,
 *                  aligned to 256 bytes; reused freely between calls that are
 *                  ordered on the same stream
 */
int bsps_sort_keys(const void *d_keys_in, void *d_keys_out, int64_t n, int32_t dtype,
                   const bsps_params *prm, int64_t *d_bucket_sizes, void *d_ws, size_t ws_bytes,
                   void *stream);

/*
 * bsps_sort_pairs -- as bsps_sort_keys, with a 32-bit payload per key.  The
 * sort is stable: payloads of equal keys keep their input order (Sec. 5.1.1).
 */
int bsps_sort_pairs(const void *d_keys_in, const uint32_t *d_vals_in, void *d_keys_out,
                    uint32_t *d_vals_out, int64_t n, int32_t dtype, const bsps_params *prm,
                    int64_t *d_bucket_sizes, void *d_ws, size_t ws_bytes, void *stream);

/*
 * bsps_sort_debug -- bsps_sort_pairs (d_vals_in may be NULL for keys only)
 * that also writes the optional diagnostics of `dbg`.
 */
int bsps_sort_debug(const void *d_keys_in, const uint32_t *d_vals_in, void *d_keys_out,
                    uint32_t *d_vals_out, int64_t n, int32_t dtype, const bsps_params *prm,
                    int64_t *d_bucket_sizes, const bsps_debug *dbg, void *d_ws, size_t ws_bytes,
                    void *stream);

/*
 * bsps_read_stats -- synchronise `stream` and read the statistics and the
 * device-side status of the last sort that used workspace d_ws.
 * Returns stats->status.
 */
int bsps_read_stats(const void *d_ws, bsps_stats *stats, void *stream);

/*
 * Learned classifier (params.classify = BSPS_LEARNED; not in the paper).  A
 * 1->32->32->1 ReLU network (FP32) fits the empirical CDF of the sorted sample
 * the method draws (Fig. 3 step 4 / Fig. 1 step 4): it starts as the
 * piecewise-linear interpolant of up to 4096 sample points at 33 knots (each
 * unit's three weights rescaled to equal size, the same function) and is then
 * trained on the GPU by full-batch gradient descent with backtracking on all
 * of its parameters (the forward and backward pass behind
 * bsps_mlp_loss_grad), so that its loss never rises.  It is evaluated exactly in its
 * piecewise-affine form: between two consecutive knots of layer 1, layer 2's
 * pre-activations are an affine function of the input.  Its output indexes a
 * table counting, per output cell, the splitters whose own output lies below
 * the cell; a key's bucket is searched among the splitters of its cell and
 * checked against the splitters just outside, so all results equal those of
 * BSPS_TREE whatever the network predicts.  Parameters are packed as W1[32]
 * b1[32] W2[32][32] (row i = unit i of layer 2) b2[32] w3[32] b3.
 *
 * bsps_mlp_loss_grad -- mean squared error of the network `d_params` on the m
 * points (d_x[i], d_y[i]) and its gradient (1153 floats into d_grad; loss into
 * d_loss, nullable).  Workspace: bsps_mlp_workspace_size(m) bytes.
 *
 * bsps_mlp_predict -- the network's output for m inputs d_x (device floats)
 * into d_y, through the piecewise-affine evaluation the classifier uses.
 * Workspace: bsps_mlp_workspace_size(0) bytes, 16-byte aligned.
 */
int bsps_mlp_workspace_size(int64_t m, size_t *bytes);
int bsps_mlp_loss_grad(const float *d_params, const float *d_x, const float *d_y, int64_t m, float *d_grad,
                       float *d_loss, void *d_ws, size_t ws_bytes, void *stream);
int bsps_mlp_predict(const float *d_params, const float *d_x, int64_t m, float *d_y, void *d_ws, size_t ws_bytes,
                     void *stream);

/*
 * bsps_sort_keys_noalloc -- bsps_sort_keys without a caller workspace.
 *
 * No counterpart in the paper.  It is for callers that cannot allocate
 * device memory themselves: code whose device memory belongs to another
 * runtime or framework that exposes no allocator to it, or latency-critical
 * code that must never call cudaMalloc (which may synchronize the device).
 * Instead of d_ws it uses a scratch array of BSPS_NOALLOC_SCRATCH_BYTES that
 * the library declares statically in device memory; every GPU that loads the
 * library holds that array until the process exits.
 *
 * Arguments and results are those of bsps_sort_keys.  The largest accepted
 * problem is the one whose bsps_workspace_size() (keys only) fits the scratch
 * (for int32 keys with p = 256 and random oversampling, about 2^23 keys);
 * anything larger returns BSPS_ERR_TOO_LARGE before any work is queued.  The
 * call allocates nothing (no cudaMalloc, no cudaFree).  The first call on a
 * device looks up the scratch's device address (cudaGetSymbolAddress, once
 * per device, with that device current); make that first call before any
 * stream capture.  All calls in the process share the one scratch array, which
 * keeps the previous call's contents: the call clears what must start at zero
 * itself, and calls whose executions overlap on the GPU (different streams,
 * or different host threads without ordering) race on it and must not be
 * issued.  bsps_noalloc_read_stats reads the device-side status and
 * statistics of the last such call (a bucket overflow or an expired wait
 * happens on the device, after the call has returned BSPS_OK).
 */
#define BSPS_NOALLOC_SCRATCH_BYTES (64ull << 20)
int bsps_sort_keys_noalloc(const void *d_keys_in, void *d_keys_out, int64_t n, int32_t dtype,
                           const bsps_params *prm, int64_t *d_bucket_sizes, void *stream);

/*
 * bsps_noalloc_read_stats -- bsps_read_stats for the no-allocation entry
 * point: synchronises `stream` and reads the status block at the start of the
 * library's static scratch on the current device.  Like the sorts that share
 * that scratch, it must not overlap a bsps_sort_keys_noalloc call running on
 * another stream.  Returns stats->status (BSPS_ERR_CUDA if the scratch's
 * address cannot be looked up).
 */
int bsps_noalloc_read_stats(bsps_stats *stats, void *stream);

/*
 * ---- Batched sorting: many independent keys-only sorts in one call --------
 *
 * No counterpart in the paper: it applies the paper's sort (Fig. 2 / Fig. 3)
 * to many inputs of uneven sizes at once.  Instance i is the key range
 * [h_offsets[i], h_offsets[i+1]) of d_keys_in; it is sorted into the same
 * range of d_keys_out exactly as bsps_sort_keys sorts it with the parameters
 *   p        = t->p[c], c the instance's size class: sizes in (2^(c-1), 2^c]
 *              (class 0: sizes 0 and 1);
 *   s, runs, sampling, refine, capacity_pct  from *prm (s = 0: the paper's
 *              default for that instance's size);
 *   seed     = prm->seed + i;
 *   classify = BSPS_LEARNED for sizes > 2^(t->learned_min_log2 - 1) when
 *              t->learned_min_log2 > 0, else prm->classify.
 * so its sorted keys and its p bucket sizes are those of that single call.
 *
 * Instances of class <= t->small_max_log2 (at most BSPS_BATCH_SMALL_MAX keys)
 * with random oversampling, 32-bit keys, the tree classifier and a sample of
 * at most BSPS_BATCH_SAMPLE_MAX records run the whole method on chip, one CTA
 * per instance, in one persistent launch (sample, sample sort, splitters,
 * classification, bucket histogram, routing into buckets and the final sort
 * all in shared memory).  The others run the single-instance pipeline on
 * t->lanes streams that fork from and join back into `stream`.  The call
 * records all of this into one CUDA graph of its own; the instantiated graph
 * is kept and relaunched by later calls with the same arguments (pointers,
 * offsets, parameters, table).  Because the call keeps and relaunches its own
 * graph and uploads the on-chip instances' table from host memory that it
 * does not keep, it must not itself be captured: on a stream that is being
 * captured it returns BSPS_ERR_CAPTURE and queues nothing.
 *
 * The offsets are a HOST array (not a device one): the size classes, the
 * split into on-chip instances and pipeline lanes, the workspace layout and
 * the graph all depend on them and are planned on the host before anything
 * is queued.  The size-class table t replaces one parameter set per call:
 * every instance takes the p of its size class.
 *
 * h_offsets: host array of num+1 nondecreasing key offsets, h_offsets[0] = 0.
 * d_bucket_sizes: device int64 array (nullable) of the instances' bucket
 *   sizes, instance i's p_i sizes starting at entry h_base[i] from
 *   bsps_batch_bucket_base().
 * Keys are 32- or 64-bit (the on-chip path takes 32-bit keys only).
 * Errors: BSPS_ERR_INVALID_ARG (bad offsets, num < 0, in == out, bad table,
 * prm->final_step or prm->duplicates other than their defaults),
 * BSPS_ERR_WORKSPACE_TOO_SMALL, BSPS_ERR_TOO_LARGE (an instance too large
 * for bsps_sort_keys), BSPS_ERR_CAPTURE, BSPS_ERR_CUDA.  Device-side statuses of all instances
 * (overflow, timeouts) are merged into the batch status that
 * bsps_read_stats(d_ws, ...) reads.
 */
#define BSPS_BATCH_CLASSES 32
#define BSPS_BATCH_SMALL_MAX 16384
#define BSPS_BATCH_SAMPLE_MAX 8192
typedef struct {
    int32_t p[BSPS_BATCH_CLASSES]; /* buckets per size class (>= 1) */
    int32_t small_max_log2;        /* classes up to this one run on chip (<= 14; -1: none) */
    int32_t learned_min_log2;      /* classes from this one up use the learned classifier; 0: never */
    int32_t lanes;                 /* concurrent streams for the other instances, 1..16 */
    int32_t reserved;
} bsps_tune;

/* bsps_tune_default -- a table that needs no measurement. */
int bsps_tune_default(bsps_tune *t);

/* bsps_batch_bucket_base -- h_base[i] (num+1 entries, host) = first entry of
 * instance i in the flat bucket-size array; h_base[num] = its length. */
int bsps_batch_bucket_base(const int64_t *h_offsets, int32_t num, const bsps_tune *t, int64_t *h_base);

/* bsps_batch_workspace_size -- device workspace bytes for bsps_sort_batched. */
int bsps_batch_workspace_size(const int64_t *h_offsets, int32_t num, int32_t dtype, const bsps_params *prm,
                              const bsps_tune *t, size_t *bytes);

int bsps_sort_batched(const void *d_keys_in, void *d_keys_out, const int64_t *h_offsets, int32_t num,
                      int32_t dtype, const bsps_params *prm, const bsps_tune *t, int64_t *d_bucket_sizes,
                      void *d_ws, size_t ws_bytes, void *stream);

/*
 * bsps_autotune_batched -- fills *t by measurement on the current device.
 * For every size class from 8 to max_log2 it sorts seeded uniform keys of
 * that size with each candidate p (on chip: 1, 2, 4, 8, 16; pipeline:
 * 16 ... 4096) and keeps the fastest (CUDA events, median of three runs);
 * small_max_log2 is the largest class for which the on-chip form beat the
 * pipeline.  lanes and learned_min_log2 are taken from *t as given.
 * d_ws: at least bsps_autotune_workspace_size() bytes.  Synchronizes stream.
 */
int bsps_autotune_workspace_size(int32_t dtype, const bsps_params *prm, int32_t max_log2, size_t *bytes);
int bsps_autotune_batched(int32_t dtype, const bsps_params *prm, int32_t max_log2, bsps_tune *t, void *d_ws,
                          size_t ws_bytes, void *stream);

/* bsps_strerror -- static text for a status code. */
const char *bsps_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* BSPSORT_H */
