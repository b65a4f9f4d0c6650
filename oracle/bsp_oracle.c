/*
 * bsp_oracle.c -- plain, slow CPU oracle for the BSP sample sort of
 * Gerbessiotis & Siniolakis, "BSP Sorting: An experimental Study".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * load or call this file: it is used by tests/, by __graft_entry__.smoke()
 * and by the cpu_baseline / reference legs of bench.py, and by nothing else.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes: an explicit BSP simulation with R virtual processors and
 * one superstep per step of the paper's algorithms --
 *   regular oversampling: procedure Sort_Det_BSP (Fig. 1, Sec. 5.1), with the
 *     duplicate handling of Sec. 5.1.1 and the padding of Lemma 5.1's proof;
 *   random oversampling:  procedure Sort_IRan_BSP (Fig. 3, Sec. 5.2), with the
 *     same duplicate handling (Sec. 5.1.1, last paragraph).
 * Supersteps:
 *   SS0 distribute  contiguous blocks of m = ceil(n/R) keys; regular mode pads
 *                   every block to M = s*ceil(m/s) (Lemma 5.1 proof)
 *   SS1 local sort  stable sort of each block (Fig. 1 step 3, Fig. 3 step 3)
 *   SS2 sample      regular: the keys ending the s equal segments of each
 *                   sorted block (Fig. 1 step 4); random: s*p-1 keys drawn
 *                   uniformly at random (Fig. 3 step 4)
 *   SS3 sample sort every sample record gathered and sorted (Fig. 1 step 5)
 *   SS4 splitters   p-1 evenly spaced sample records (Fig. 1 step 6)
 *   SS5 broadcast   every processor receives the splitters (Fig. 1 step 7)
 *   SS6 partition   binary search of each splitter into each sorted block
 *                   (Sec. 5.1, step 9 discussion; Sec. 5.2, IRan discussion)
 *   SS7 prefix      per-bucket counts and receive offsets (Fig. 1 step 9)
 *   SS8 route       order-preserving all-to-all (Fig. 1 steps 10-11)
 *   SS9 merge       stable multi-way merge of each bucket (Fig. 1 step 12)
 * params.variant = OR_RAN runs procedure Sort_Ran_BSP (Fig. 2, Sec. 5.2)
 * instead (random oversampling only): no local sort first; SS6 classifies
 * every key by binary search of the splitters (Fig. 2 step 9) and groups the
 * block by bucket, keeping input order; SS9 sorts each received bucket (Fig. 2
 * step 12).  Its buckets and output are those of Sort_IRan_BSP.
 * params.duplicates = OR_DUP_OFF compares records by (pad, phi) alone in the
 * partition / classification: the paper's version without duplicate handling
 * (Sec. 6.1), whose cost Sec. 6.4 measures.  Sorting stays by the total order.
 * Each superstep is a function of one processor id; all processors run it,
 * one after the other or on several host threads (params.threads), and the
 * next superstep starts only when every processor has finished (the barrier
 * of the BSP model).  Processors of one superstep write disjoint memory, so
 * the result does not depend on the number of threads.
 *
 * The total order (Sec. 5.1.1): records compare by (pad, phi(key), tag).
 * phi maps a key's bit pattern to an unsigned integer whose unsigned order is
 * the key order (IEEE-754 totalOrder for floats).  tag = k*M + j for the key
 * held at local index j of processor k before the local sort -- the two
 * implicit tags (processor id, local array index) of Sec. 5.1.1 in one word.
 * Pads are virtual records that follow every real key.
 *
 * Readings where the paper is silent:
 *  - blocks are contiguous; pads are +infinity records ordered by tag;
 *  - random mode draws positions i.i.d. with replacement:
 *      g_j = floor(h(seed, j) * n / 2^64),  j = 0 .. s*p-2,
 *    h(seed, j) = word (j mod 4) of Philox4x64-10 with key (seed, 0) and
 *    counter (floor(j/4), 0, 0, 0)  [Salmon et al., SC'11];
 *  - splitter i is the sorted-sample record of 1-indexed rank i*q
 *    (q = R*s/p regular, q = s random), and belongs to the upper bucket.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

enum { OR_U32 = 0, OR_I32 = 1, OR_F32 = 2, OR_F64 = 3 };
enum { OR_REGULAR = 0, OR_RANDOM = 1 };
enum { OR_DUP_TAGS = 0, OR_DUP_OFF = 1 };
enum { OR_DET_IRAN = 0, OR_RAN = 1 };

/* one record of the total order, as reported to the caller */
typedef struct {
    uint64_t phi;
    uint64_t tag;
    uint32_t pad;
    uint32_t reserved;
} oracle_record;

typedef struct {
    int32_t p;        /* number of buckets (paper's p) */
    int32_t runs;     /* R virtual processors; 0 -> p */
    int64_t s;        /* oversampling factor; 0 -> paper default */
    int32_t sampling; /* OR_REGULAR or OR_RANDOM */
    int32_t threads;  /* host threads running the processors; 0 -> 1 */
    uint64_t seed;    /* random-mode sample seed */
    int32_t duplicates; /* OR_DUP_TAGS (Sec. 5.1.1) or OR_DUP_OFF */
    int32_t variant;    /* OR_DET_IRAN (Fig. 1 / Fig. 3) or OR_RAN (Fig. 2) */
} oracle_params;

/* the resolved parameters of one call */
typedef struct {
    int64_t n, p, R, s, m, M, x, q, sample_size;
    int32_t sampling;
} oracle_plan;

/* an element held by a virtual processor */
typedef struct {
    uint64_t phi;
    uint64_t tag;
    uint32_t val;
    uint32_t pad;
} elem;

/* ------------------------------------------------------------------ */
/* key <-> phi (IEEE-754 totalOrder on bit patterns for floats)        */

static uint64_t key_bits(int dtype, const void *keys, int64_t i) {
    if (dtype == OR_F64) return ((const uint64_t *)keys)[i];
    return ((const uint32_t *)keys)[i];
}

static uint64_t phi_of(int dtype, uint64_t u) {
    switch (dtype) {
    case OR_U32: return u;
    case OR_I32: return u ^ 0x80000000u;
    case OR_F32: return (u & 0x80000000u) ? (~u & 0xffffffffu) : (u | 0x80000000u);
    default:     return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
    }
}

static uint64_t key_of_phi(int dtype, uint64_t v) {
    switch (dtype) {
    case OR_U32: return v;
    case OR_I32: return v ^ 0x80000000u;
    case OR_F32: return (v & 0x80000000u) ? (v & 0x7fffffffu) : (~v & 0xffffffffu);
    default:     return (v >> 63) ? (v & 0x7fffffffffffffffull) : ~v;
    }
}

static void put_key(int dtype, void *out, int64_t i, uint64_t bits) {
    if (dtype == OR_F64) ((uint64_t *)out)[i] = bits;
    else ((uint32_t *)out)[i] = (uint32_t)bits;
}

/* ------------------------------------------------------------------ */
/* the total order of Sec. 5.1.1: (pad, phi, tag)                      */

static int elem_cmp(const void *a_, const void *b_) {
    const elem *a = (const elem *)a_, *b = (const elem *)b_;
    if (a->pad != b->pad) return a->pad < b->pad ? -1 : 1;
    if (a->phi != b->phi) return a->phi < b->phi ? -1 : 1;
    if (a->tag != b->tag) return a->tag < b->tag ? -1 : 1;
    return 0;
}

static int elem_less(const elem *a, const elem *b) { return elem_cmp(a, b) < 0; }

/* without duplicate handling: (pad, phi) only */
static int elem_less_notag(const elem *a, const elem *b) {
    if (a->pad != b->pad) return a->pad < b->pad;
    return a->phi < b->phi;
}

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)                   */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 prod = (unsigned __int128)a * b;
    *hi = (uint64_t)(prod >> 64);
    *lo = (uint64_t)prod;
}

static void philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ull, c[0], &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ull, c[2], &hi1, &lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* draw j of the sample stream with the given seed */
uint64_t oracle_draw(uint64_t seed, uint64_t j) {
    uint64_t ctr[4] = {j / 4, 0, 0, 0}, key[2] = {seed, 0}, out[4];
    philox4x64_10(ctr, key, out);
    return out[j % 4];
}

/* position of draw j in an input of n keys: floor(h * n / 2^64) */
int64_t oracle_position(uint64_t seed, uint64_t j, int64_t n) {
    unsigned __int128 prod = (unsigned __int128)oracle_draw(seed, j) * (uint64_t)n;
    return (int64_t)(uint64_t)(prod >> 64);
}

/* ------------------------------------------------------------------ */
/* parameter resolution (Sec. 6.1 last item; Fig. 1 step 1; Fig. 2/3 step 1) */

static int64_t ceil_lg(int64_t n) { /* ceil(log2 n), n >= 1 */
    int64_t r = 0;
    while (((int64_t)1 << r) < n) ++r;
    return r;
}

int oracle_plan_of(int64_t n, const oracle_params *prm, oracle_plan *pl) {
    if (!prm || !pl || n < 0 || prm->p < 1) return OR_EINVAL;
    if (prm->sampling != OR_REGULAR && prm->sampling != OR_RANDOM) return OR_EINVAL;
    if (prm->s < 0 || prm->runs < 0) return OR_EINVAL;
    if (prm->duplicates != OR_DUP_TAGS && prm->duplicates != OR_DUP_OFF) return OR_EINVAL;
    if (prm->variant != OR_DET_IRAN && prm->variant != OR_RAN) return OR_EINVAL;
    if (prm->variant == OR_RAN && prm->sampling != OR_RANDOM) return OR_EINVAL;
    memset(pl, 0, sizeof(*pl));
    pl->n = n;
    pl->p = prm->p;
    pl->R = prm->runs > 0 ? prm->runs : prm->p;
    pl->sampling = prm->sampling;
    int64_t clg = n >= 2 ? ceil_lg(n) : 1;
    if (prm->sampling == OR_REGULAR) {
        /* s = r*p with r = ceil(lg lg n) (Sec. 6.1: omega_n = lg lg n) */
        int64_t r = 1;
        while (((int64_t)1 << r) < clg) ++r;
        pl->s = prm->s > 0 ? prm->s : r * pl->p;
        pl->m = (n + pl->R - 1) / pl->R;
        pl->M = pl->s * ((pl->m + pl->s - 1) / pl->s);
        if (pl->M == 0) pl->M = pl->s;
        pl->x = pl->M / pl->s;
        if ((pl->R * pl->s) % pl->p != 0 || pl->R * pl->s < pl->p) return OR_EINVAL;
        pl->q = pl->R * pl->s / pl->p;
        pl->sample_size = pl->R * pl->s;
    } else {
        /* s = 2 omega_n^2 lg n with omega_n^2 = lg n (Sec. 6.1) */
        pl->s = prm->s > 0 ? prm->s : 2 * clg * clg;
        pl->m = (n + pl->R - 1) / pl->R;
        pl->M = pl->m;
        pl->x = 0;
        pl->q = pl->s;
        pl->sample_size = pl->s * pl->p - 1;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* binary min-heap of block heads for the multi-way merge of SS9       */

typedef struct {
    const elem *seg; /* sorted segment */
    int64_t len, pos;
} head;

static void heap_down(head *h, int64_t cnt, int64_t i) {
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < cnt && elem_less(&h[l].seg[h[l].pos], &h[m].seg[h[m].pos])) m = l;
        if (r < cnt && elem_less(&h[r].seg[h[r].pos], &h[m].seg[h[m].pos])) m = r;
        if (m == i) return;
        head t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
}

/* ------------------------------------------------------------------ */

static void to_record(const elem *e, oracle_record *r) {
    r->phi = e->phi; r->tag = e->tag; r->pad = e->pad; r->reserved = 0;
}

/* ------------------------------------------------------------------ */
/* The simulated BSP machine.  A superstep runs the same local computation
 * on every virtual processor, then all processors meet at a barrier before
 * the next superstep reads what the others produced (the BSP model, Sec. 2).
 * The local computations of one superstep touch disjoint data, so they may
 * run on several host threads; the join of those threads is the barrier.
 * With one thread the processors simply run one after the other.         */

typedef struct {
    int dtype;
    const void *keys;
    const uint32_t *vals;
    uint64_t seed;
    oracle_plan pl;
    int regular;
    int dup_off;          /* compare by (pad, phi) alone in SS6 */
    int ran;              /* Sort_Ran_BSP (Fig. 2) */
    elem **local;         /* local[k]: the records held by processor k */
    int64_t *len;         /* records held (keys and pads) */
    int64_t *nreal;       /* real keys held */
    elem *Y;              /* the sample, gathered at processor 0 */
    elem *Spl;            /* the p-1 splitters */
    elem **Sk;            /* Sk[k]: processor k's copy of the splitters */
    int64_t *c;           /* c[k*(p+1)+i]: first position of segment i in block k */
    int64_t *bucket_len;  /* records received by processor i (keys and pads) */
    int64_t *bucket_real; /* real keys received by processor i */
    int64_t *out_off;     /* output position of processor i's first key */
    int64_t *recv_off;    /* recv_off[k*p+i]: where X^k_i lands in Z^i */
    elem **Z;             /* Z[i]: the segments received by processor i */
    void *keys_out;
    uint32_t *vals_out;
    int64_t *pad_sizes;
    int32_t *bucket_of;
    int failed;           /* some processor could not allocate its memory */
} machine;

typedef void (*local_step)(machine *S, int64_t k);

typedef struct {
    machine *S;
    local_step fn;
    int64_t count;
    int threads, t;
} worker;

static void *run_worker(void *arg) {
    worker *w = (worker *)arg;
    for (int64_t k = w->t; k < w->count; k += w->threads) w->fn(w->S, k);
    return NULL;
}

/* run fn(S, k) for k = 0 .. count-1, then the barrier */
static void superstep(machine *S, int threads, int64_t count, local_step fn) {
    if (threads > count) threads = (int)count;
    if (threads <= 1) {
        for (int64_t k = 0; k < count; ++k) fn(S, k);
        return;
    }
    pthread_t th[256];
    worker w[256];
    if (threads > 256) threads = 256;
    int started = 1;
    for (int t = 0; t < threads; ++t) w[t] = (worker){S, fn, count, threads, t};
    for (int t = 1; t < threads; ++t, ++started)
        if (pthread_create(&th[t], NULL, run_worker, &w[t])) break;
    /* a worker that could not be started: the calling thread takes its share */
    for (int t = started; t < threads; ++t) {
        w[t].threads = threads;
        run_worker(&w[t]);
    }
    run_worker(&w[0]);
    for (int t = 1; t < started; ++t) pthread_join(th[t], NULL);
}

static void fail(machine *S) { __atomic_store_n(&S->failed, 1, __ATOMIC_RELAXED); }

/* ---- SS0: processor k receives the contiguous block [k*m, (k+1)*m) and pads
 *      it to M records in regular mode (Lemma 5.1 proof) ---- */
static void ss0_distribute(machine *S, int64_t k) {
    const oracle_plan pl = S->pl;
    const int64_t m = pl.m, M = pl.M, n = pl.n;
    int64_t lo = k * m, hi = lo + m < n ? lo + m : n;
    S->nreal[k] = hi > lo ? hi - lo : 0;
    S->len[k] = S->regular ? M : S->nreal[k];
    elem *blk = malloc(sizeof(elem) * (size_t)(S->len[k] ? S->len[k] : 1));
    S->local[k] = blk;
    if (!blk) { fail(S); return; }
    for (int64_t j = 0; j < S->len[k]; ++j) {
        elem *e = &blk[j];
        e->tag = (uint64_t)(k * M + j);
        if (j < S->nreal[k]) {
            e->phi = phi_of(S->dtype, key_bits(S->dtype, S->keys, lo + j));
            e->val = S->vals ? S->vals[lo + j] : 0;
            e->pad = 0;
        } else {
            e->phi = ~0ull;
            e->val = 0;
            e->pad = 1;
        }
    }
}

/* ---- SS1: local sort on processor k (Fig. 1/3 step 3) ---- */
static void ss1_local_sort(machine *S, int64_t k) {
    if (S->local[k]) qsort(S->local[k], (size_t)S->len[k], sizeof(elem), elem_cmp);
}

/* ---- SS2 (regular): processor k's sample, the last key of each of its s
 *      segments of x keys (Fig. 1 step 4) ---- */
static void ss2_regular_sample(machine *S, int64_t k) {
    elem **local = S->local, *Y = S->Y;
    const oracle_plan pl = S->pl;
    for (int64_t j = 1; j <= pl.s; ++j) Y[k * pl.s + (j - 1)] = local[k][j * pl.x - 1];
}

/* ---- SS5: processor k receives its copy of the splitters (Fig. 1 step 7) ---- */
static void ss5_broadcast(machine *S, int64_t k) {
    const int64_t p = S->pl.p;
    S->Sk[k] = malloc(sizeof(elem) * (size_t)(p > 1 ? p - 1 : 1));
    if (!S->Sk[k]) { fail(S); return; }
    memcpy(S->Sk[k], S->Spl, sizeof(elem) * (size_t)(p - 1));
}

/* ---- SS6: processor k partitions its sorted block by binary search of each
 *      splitter; segment i = [c[i], c[i+1]) (Sec. 5.1 step 9) ---- */
static void ss6_partition(machine *S, int64_t k) {
    elem **local = S->local, **Sk = S->Sk;
    const int64_t p = S->pl.p;
    int64_t *ck = S->c + k * (p + 1);
    ck[0] = 0;
    ck[p] = S->len[k];
    for (int64_t i = 1; i < p; ++i) {
        /* first local position whose record is not smaller than S_i */
        int64_t lo = 0, hi = S->len[k];
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            const int less = S->dup_off ? elem_less_notag(&local[k][mid], &Sk[k][i - 1])
                                        : elem_less(&local[k][mid], &Sk[k][i - 1]);
            if (less) lo = mid + 1;
            else hi = mid;
        }
        ck[i] = lo;
    }
}

/* ---- SS6 of Sort_Ran_BSP: processor k finds the bucket of each of its keys
 *      by binary search of the splitters (Fig. 2 step 9) -- the number of
 *      splitters not above the key -- and groups its block by bucket, each
 *      group in input order; segment i = group i ---- */
static void ss6_classify(machine *S, int64_t k) {
    elem **local = S->local, **Sk = S->Sk;
    const int64_t p = S->pl.p, len = S->len[k];
    int64_t *ck = S->c + k * (p + 1);
    int64_t *b = malloc(sizeof(int64_t) * (size_t)(len ? len : 1));
    elem *grouped = malloc(sizeof(elem) * (size_t)(len ? len : 1));
    if (!b || !grouped) { free(b); free(grouped); fail(S); return; }
    for (int64_t i = 0; i <= p; ++i) ck[i] = 0;
    for (int64_t j = 0; j < len; ++j) {
        /* bucket = #{i : S_i <= e} = first splitter index with e < S_i */
        int64_t lo = 0, hi = p - 1;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            const int less = S->dup_off ? elem_less_notag(&local[k][j], &Sk[k][mid])
                                        : elem_less(&local[k][j], &Sk[k][mid]);
            if (less) hi = mid;
            else lo = mid + 1;
        }
        b[j] = lo;
        ck[lo + 1]++;
    }
    for (int64_t i = 0; i < p; ++i) ck[i + 1] += ck[i];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)p);
    if (!fill) { free(b); free(grouped); fail(S); return; }
    for (int64_t i = 0; i < p; ++i) fill[i] = ck[i];
    for (int64_t j = 0; j < len; ++j) grouped[fill[b[j]]++] = local[k][j];
    free(fill);
    free(b);
    free(local[k]);
    local[k] = grouped;
}

/* ---- SS7: counts of bucket i and the receive offsets of its segments
 *      (Fig. 1 step 9) ---- */
static void ss7_prefix(machine *S, int64_t i) {
    elem **local = S->local;
    const int64_t p = S->pl.p, R = S->pl.R;
    int64_t *pad_sizes = S->pad_sizes;
    int64_t acc = 0, real = 0;
    for (int64_t k = 0; k < R; ++k) {
        const int64_t *ck = S->c + k * (p + 1);
        S->recv_off[k * p + i] = acc;
        acc += ck[i + 1] - ck[i];
        for (int64_t t = ck[i]; t < ck[i + 1]; ++t) {
            if (local[k][t].pad) { if (pad_sizes) pad_sizes[i]++; }
            else real++;
        }
    }
    S->bucket_len[i] = acc;
    S->bucket_real[i] = real;
}

/* ---- SS8: processor i receives X^k_i from every k, in processor order
 *      (Fig. 1 step 11) ---- */
static void ss8_route(machine *S, int64_t i) {
    elem **local = S->local;
    const int64_t p = S->pl.p, R = S->pl.R;
    S->Z[i] = malloc(sizeof(elem) * (size_t)(S->bucket_len[i] ? S->bucket_len[i] : 1));
    if (!S->Z[i]) { fail(S); return; }
    for (int64_t k = 0; k < R; ++k) {
        const int64_t *ck = S->c + k * (p + 1);
        memcpy(S->Z[i] + S->recv_off[k * p + i], local[k] + ck[i],
               sizeof(elem) * (size_t)(ck[i + 1] - ck[i]));
    }
}

/* ---- SS9: processor i merges its received sorted segments stably (Fig. 1
 *      step 12; ties by source processor, Sec. 5.1.1) and emits its keys ---- */
/* ---- SS9 of Sort_Ran_BSP: processor i sorts what it received (Fig. 2
 *      step 12) and emits its keys ---- */
static void ss9_sort(machine *S, int64_t i) {
    const int64_t m = S->pl.m, M = S->pl.M;
    elem *Z = S->Z[i];
    const int64_t len = S->bucket_len[i];
    qsort(Z, (size_t)len, sizeof(elem), elem_cmp);
    int64_t out = S->out_off[i];
    for (int64_t t = 0; t < len; ++t) {
        const elem *e = &Z[t];
        if (e->pad) continue;
        put_key(S->dtype, S->keys_out, out, key_of_phi(S->dtype, e->phi));
        if (S->vals_out) S->vals_out[out] = e->val;
        if (S->bucket_of) {
            int64_t k = (int64_t)(e->tag / (uint64_t)M), j = (int64_t)(e->tag % (uint64_t)M);
            S->bucket_of[k * m + j] = (int32_t)i;
        }
        ++out;
    }
}

static void ss9_merge(machine *S, int64_t i) {
    const int64_t p = S->pl.p, R = S->pl.R, m = S->pl.m, M = S->pl.M;
    const int64_t *c = S->c;
    head *h = malloc(sizeof(head) * (size_t)(R ? R : 1));
    if (!h) { fail(S); return; }
    int64_t out = S->out_off[i];
    int64_t cnt = 0;
    for (int64_t k = 0; k < R; ++k) {
        int64_t seg_len = c[k * (p + 1) + i + 1] - c[k * (p + 1) + i];
        if (seg_len > 0) {
            h[cnt].seg = S->Z[i] + S->recv_off[k * p + i];
            h[cnt].len = seg_len;
            h[cnt].pos = 0;
            ++cnt;
        }
    }
    for (int64_t t = cnt / 2 - 1; t >= 0; --t) heap_down(h, cnt, t);
    while (cnt > 0) {
        const elem *e = &h[0].seg[h[0].pos];
        if (!e->pad) { /* pads are dropped from the output */
            put_key(S->dtype, S->keys_out, out, key_of_phi(S->dtype, e->phi));
            if (S->vals_out) S->vals_out[out] = e->val;
            if (S->bucket_of) {
                int64_t k = (int64_t)(e->tag / (uint64_t)M), j = (int64_t)(e->tag % (uint64_t)M);
                S->bucket_of[k * m + j] = (int32_t)i;
            }
            ++out;
        }
        if (++h[0].pos == h[0].len) h[0] = h[--cnt];
        if (cnt > 0) heap_down(h, cnt, 0);
    }
    free(h);
}

static void free_block(machine *S, int64_t k) {
    free(S->local[k]);
    S->local[k] = NULL;
}

static void release(machine *S) {
    const int64_t R = S->pl.R, p = S->pl.p;
    if (S->local) for (int64_t k = 0; k < R; ++k) free(S->local[k]);
    if (S->Sk) for (int64_t k = 0; k < R; ++k) free(S->Sk[k]);
    if (S->Z) for (int64_t i = 0; i < p; ++i) free(S->Z[i]);
    free(S->local); free(S->len); free(S->nreal); free(S->Y); free(S->Spl); free(S->Sk);
    free(S->c); free(S->bucket_len); free(S->bucket_real); free(S->out_off); free(S->recv_off);
    free(S->Z);
}

/*
 * oracle_sort: sort n keys (and optional 32-bit payloads) by the BSP
 * simulation above.  Outputs (each optional unless noted):
 *   keys_out      n keys in the key dtype (required when n > 0)
 *   vals_out      n payloads, permuted with the keys
 *   bucket_sizes  p counts of real keys per bucket
 *   pad_sizes     p counts of pad records per bucket
 *   sample        plan.sample_size sorted sample records
 *   splitters     p-1 splitter records
 *   bucket_of     n bucket ids, indexed by the input position
 *   partition     R*(p+1) entries c[k][i] at k*(p+1) + i: the first position
 *                 of segment i in sorted block k (SS6; pads included).  With
 *                 OR_RAN: the first position of group i in block k.
 * prm->threads host threads run the processors of each superstep (0 or 1:
 * one after the other); the result does not depend on it.
 */
int oracle_sort(int dtype, const void *keys, const uint32_t *vals, int64_t n,
                const oracle_params *prm, void *keys_out, uint32_t *vals_out,
                int64_t *bucket_sizes, int64_t *pad_sizes, oracle_record *sample,
                oracle_record *splitters, int32_t *bucket_of, int64_t *partition) {
    if (dtype < OR_U32 || dtype > OR_F64) return OR_EINVAL;
    oracle_plan pl;
    int rc = oracle_plan_of(n, prm, &pl);
    if (rc) return rc;
    const int64_t p = pl.p, R = pl.R, m = pl.m, M = pl.M, S_ = pl.sample_size;
    const int T = prm->threads > 1 ? prm->threads : 1;
    if (bucket_sizes) memset(bucket_sizes, 0, sizeof(int64_t) * p);
    if (pad_sizes) memset(pad_sizes, 0, sizeof(int64_t) * p);
    if (n == 0) return OR_OK;

    machine mc;
    memset(&mc, 0, sizeof(mc));
    machine *S = &mc;
    S->dtype = dtype; S->keys = keys; S->vals = vals; S->seed = prm->seed; S->pl = pl;
    S->regular = pl.sampling == OR_REGULAR;
    S->dup_off = prm->duplicates == OR_DUP_OFF;
    S->ran = prm->variant == OR_RAN;
    S->keys_out = keys_out; S->vals_out = vals_out; S->pad_sizes = pad_sizes; S->bucket_of = bucket_of;
    S->local = calloc((size_t)R, sizeof(elem *));
    S->len = calloc((size_t)R, sizeof(int64_t));
    S->nreal = calloc((size_t)R, sizeof(int64_t));
    S->Y = malloc(sizeof(elem) * (size_t)(S_ ? S_ : 1));
    S->Spl = malloc(sizeof(elem) * (size_t)(p > 1 ? p - 1 : 1));
    S->Sk = calloc((size_t)R, sizeof(elem *));
    S->c = malloc(sizeof(int64_t) * (size_t)R * (size_t)(p + 1));
    S->bucket_len = calloc((size_t)p, sizeof(int64_t));
    S->bucket_real = calloc((size_t)p, sizeof(int64_t));
    S->out_off = calloc((size_t)p, sizeof(int64_t));
    S->recv_off = malloc(sizeof(int64_t) * (size_t)R * (size_t)p);
    S->Z = calloc((size_t)p, sizeof(elem *));
    if (!S->local || !S->len || !S->nreal || !S->Y || !S->Spl || !S->Sk || !S->c || !S->bucket_len ||
        !S->bucket_real || !S->out_off || !S->recv_off || !S->Z) {
        release(S);
        return OR_ENOMEM;
    }
    elem *Y = S->Y, *Spl = S->Spl;

    /* ---- SS0: distribute contiguous blocks; pad them (Lemma 5.1 proof) ---- */
    superstep(S, T, R, ss0_distribute);
    if (S->failed) { release(S); return OR_ENOMEM; }

    /* ---- SS1: local sort on every processor (Fig. 1/3 step 3; none in
     *      Sort_Ran_BSP) ---- */
    if (!S->ran) superstep(S, T, R, ss1_local_sort);

    /* ---- SS2: sample (Fig. 1 step 4 / Fig. 3 step 4) ---- */
    if (S->regular) {
        superstep(S, T, R, ss2_regular_sample);
    } else {
        /* s*p-1 keys chosen uniformly at random; the processor owning
         * input position g contributes the record of that key */
        for (int64_t j = 0; j < S_; ++j) {
            int64_t g = oracle_position(prm->seed, (uint64_t)j, n);
            int64_t k = g / m, jj = g - k * m;
            elem e;
            e.phi = phi_of(dtype, key_bits(dtype, keys, g));
            e.tag = (uint64_t)(k * M + jj);
            e.val = 0;
            e.pad = 0;
            Y[j] = e;
        }
    }

    /* ---- SS3: sample sort at one processor (Fig. 1 step 5) ---- */
    qsort(Y, (size_t)S_, sizeof(elem), elem_cmp);
    if (sample)
        for (int64_t t = 0; t < S_; ++t) to_record(&Y[t], &sample[t]);

    /* ---- SS4: p-1 evenly spaced splitters, 1-indexed rank i*q (Fig. 1 step 6) ---- */
    for (int64_t i = 1; i < p; ++i) Spl[i - 1] = Y[i * pl.q - 1];
    if (splitters)
        for (int64_t i = 1; i < p; ++i) to_record(&Spl[i - 1], &splitters[i - 1]);

    /* ---- SS5: broadcast (Fig. 1 step 7): every processor gets a copy ---- */
    superstep(S, T, R, ss5_broadcast);
    if (S->failed) { release(S); return OR_ENOMEM; }

    /* ---- SS6: partition by binary search of each splitter into the sorted
     *      local keys (Sec. 5.1 step 9); Sort_Ran_BSP classifies every key
     *      (Fig. 2 step 9) ---- */
    superstep(S, T, R, S->ran ? ss6_classify : ss6_partition);
    if (S->failed) { release(S); return OR_ENOMEM; }
    if (partition) memcpy(partition, S->c, sizeof(int64_t) * (size_t)R * (size_t)(p + 1));

    /* ---- SS7: per-bucket counts and prefix sums (Fig. 1 step 9) ---- */
    superstep(S, T, p, ss7_prefix);
    int64_t acc = 0;
    for (int64_t i = 0; i < p; ++i) {
        S->out_off[i] = acc;
        acc += S->bucket_real[i];
        if (bucket_sizes) bucket_sizes[i] = S->bucket_real[i];
    }

    /* ---- SS8: route X^k_i to Z^i_k, sources in processor order (Fig. 1 step 11) ---- */
    superstep(S, T, p, ss8_route);
    if (S->failed) { release(S); return OR_ENOMEM; }
    superstep(S, T, R, free_block);  /* the routed records now live in Z */

    /* ---- SS9: stable multi-way merge of the received sorted segments
     *      (Fig. 1 step 12; ties by source processor, Sec. 5.1.1); in
     *      Sort_Ran_BSP a sort of each received bucket (Fig. 2 step 12) ---- */
    superstep(S, T, p, S->ran ? ss9_sort : ss9_merge);
    const int failed = S->failed;
    release(S);
    if (failed) return OR_ENOMEM;
    return acc == n ? OR_OK : OR_EINVAL;
}
