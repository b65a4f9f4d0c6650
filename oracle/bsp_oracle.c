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
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

enum { OR_U32 = 0, OR_I32 = 1, OR_F32 = 2, OR_F64 = 3 };
enum { OR_REGULAR = 0, OR_RANDOM = 1 };

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
    int32_t reserved;
    uint64_t seed;    /* random-mode sample seed */
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
 */
int oracle_sort(int dtype, const void *keys, const uint32_t *vals, int64_t n,
                const oracle_params *prm, void *keys_out, uint32_t *vals_out,
                int64_t *bucket_sizes, int64_t *pad_sizes, oracle_record *sample,
                oracle_record *splitters, int32_t *bucket_of) {
    if (dtype < OR_U32 || dtype > OR_F64) return OR_EINVAL;
    oracle_plan pl;
    int rc = oracle_plan_of(n, prm, &pl);
    if (rc) return rc;
    const int64_t p = pl.p, R = pl.R, m = pl.m, M = pl.M, S = pl.sample_size;
    const int regular = pl.sampling == OR_REGULAR;
    if (bucket_sizes) memset(bucket_sizes, 0, sizeof(int64_t) * p);
    if (pad_sizes) memset(pad_sizes, 0, sizeof(int64_t) * p);
    if (n == 0) return OR_OK;

    /* ---- SS0: distribute contiguous blocks; pad them (Lemma 5.1 proof) ---- */
    elem **local = calloc((size_t)R, sizeof(elem *));
    int64_t *len = calloc((size_t)R, sizeof(int64_t));     /* records held */
    int64_t *nreal = calloc((size_t)R, sizeof(int64_t));   /* real keys held */
    if (!local || !len || !nreal) return OR_ENOMEM;
    for (int64_t k = 0; k < R; ++k) {
        int64_t lo = k * m, hi = lo + m < n ? lo + m : n;
        nreal[k] = hi > lo ? hi - lo : 0;
        len[k] = regular ? M : nreal[k];
        local[k] = malloc(sizeof(elem) * (size_t)(len[k] ? len[k] : 1));
        if (!local[k]) return OR_ENOMEM;
        for (int64_t j = 0; j < len[k]; ++j) {
            elem *e = &local[k][j];
            e->tag = (uint64_t)(k * M + j);
            if (j < nreal[k]) {
                e->phi = phi_of(dtype, key_bits(dtype, keys, lo + j));
                e->val = vals ? vals[lo + j] : 0;
                e->pad = 0;
            } else {
                e->phi = ~0ull;
                e->val = 0;
                e->pad = 1;
            }
        }
    }

    /* ---- SS1: local sort on every processor (Fig. 1/3 step 3) ---- */
    for (int64_t k = 0; k < R; ++k) qsort(local[k], (size_t)len[k], sizeof(elem), elem_cmp);

    /* ---- SS2: sample (Fig. 1 step 4 / Fig. 3 step 4) ---- */
    elem *Y = malloc(sizeof(elem) * (size_t)(S ? S : 1));
    if (!Y) return OR_ENOMEM;
    if (regular) {
        /* processor k: the last key of each of its s segments of x keys */
        for (int64_t k = 0; k < R; ++k)
            for (int64_t j = 1; j <= pl.s; ++j) Y[k * pl.s + (j - 1)] = local[k][j * pl.x - 1];
    } else {
        /* s*p-1 keys chosen uniformly at random; the processor owning
         * input position g contributes the record of that key */
        for (int64_t j = 0; j < S; ++j) {
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
    qsort(Y, (size_t)S, sizeof(elem), elem_cmp);
    if (sample)
        for (int64_t t = 0; t < S; ++t) to_record(&Y[t], &sample[t]);

    /* ---- SS4: p-1 evenly spaced splitters, 1-indexed rank i*q (Fig. 1 step 6) ---- */
    elem *Spl = malloc(sizeof(elem) * (size_t)(p > 1 ? p - 1 : 1));
    if (!Spl) return OR_ENOMEM;
    for (int64_t i = 1; i < p; ++i) Spl[i - 1] = Y[i * pl.q - 1];
    if (splitters)
        for (int64_t i = 1; i < p; ++i) to_record(&Spl[i - 1], &splitters[i - 1]);

    /* ---- SS5: broadcast (Fig. 1 step 7): every processor gets a copy ---- */
    elem **Sk = calloc((size_t)R, sizeof(elem *));
    if (!Sk) return OR_ENOMEM;
    for (int64_t k = 0; k < R; ++k) {
        Sk[k] = malloc(sizeof(elem) * (size_t)(p > 1 ? p - 1 : 1));
        if (!Sk[k]) return OR_ENOMEM;
        memcpy(Sk[k], Spl, sizeof(elem) * (size_t)(p - 1));
    }

    /* ---- SS6: partition by binary search of each splitter into the sorted
     *      local keys; segment i = [c[i], c[i+1]) (Sec. 5.1 step 9) ---- */
    int64_t *c = malloc(sizeof(int64_t) * (size_t)R * (size_t)(p + 1));
    if (!c) return OR_ENOMEM;
    for (int64_t k = 0; k < R; ++k) {
        int64_t *ck = c + k * (p + 1);
        ck[0] = 0;
        ck[p] = len[k];
        for (int64_t i = 1; i < p; ++i) {
            /* first local position whose record is not smaller than S_i */
            int64_t lo = 0, hi = len[k];
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (elem_less(&local[k][mid], &Sk[k][i - 1])) lo = mid + 1;
                else hi = mid;
            }
            ck[i] = lo;
        }
    }

    /* ---- SS7: per-bucket counts and prefix sums (Fig. 1 step 9) ---- */
    int64_t *bucket_len = calloc((size_t)p, sizeof(int64_t));
    int64_t *recv_off = malloc(sizeof(int64_t) * (size_t)R * (size_t)p);
    if (!bucket_len || !recv_off) return OR_ENOMEM;
    for (int64_t i = 0; i < p; ++i) {
        int64_t acc = 0;
        for (int64_t k = 0; k < R; ++k) {
            const int64_t *ck = c + k * (p + 1);
            recv_off[k * p + i] = acc;
            acc += ck[i + 1] - ck[i];
            for (int64_t t = ck[i]; t < ck[i + 1]; ++t) {
                if (local[k][t].pad) { if (pad_sizes) pad_sizes[i]++; }
                else if (bucket_sizes) bucket_sizes[i]++;
            }
        }
        bucket_len[i] = acc;
    }

    /* ---- SS8: route X^k_i to Z^i_k, sources in processor order (Fig. 1 step 11) ---- */
    elem **Z = calloc((size_t)p, sizeof(elem *));
    if (!Z) return OR_ENOMEM;
    for (int64_t i = 0; i < p; ++i) {
        Z[i] = malloc(sizeof(elem) * (size_t)(bucket_len[i] ? bucket_len[i] : 1));
        if (!Z[i]) return OR_ENOMEM;
    }
    for (int64_t k = 0; k < R; ++k) {
        const int64_t *ck = c + k * (p + 1);
        for (int64_t i = 0; i < p; ++i)
            memcpy(Z[i] + recv_off[k * p + i], local[k] + ck[i],
                   sizeof(elem) * (size_t)(ck[i + 1] - ck[i]));
    }

    /* ---- SS9: stable multi-way merge of the received sorted segments
     *      (Fig. 1 step 12; ties by source processor, Sec. 5.1.1) ---- */
    head *h = malloc(sizeof(head) * (size_t)R);
    if (!h) return OR_ENOMEM;
    int64_t out = 0;
    for (int64_t i = 0; i < p; ++i) {
        int64_t cnt = 0;
        for (int64_t k = 0; k < R; ++k) {
            int64_t seg_len = c[k * (p + 1) + i + 1] - c[k * (p + 1) + i];
            if (seg_len > 0) {
                h[cnt].seg = Z[i] + recv_off[k * p + i];
                h[cnt].len = seg_len;
                h[cnt].pos = 0;
                ++cnt;
            }
        }
        for (int64_t t = cnt / 2 - 1; t >= 0; --t) heap_down(h, cnt, t);
        while (cnt > 0) {
            const elem *e = &h[0].seg[h[0].pos];
            if (!e->pad) { /* pads are dropped from the output */
                put_key(dtype, keys_out, out, key_of_phi(dtype, e->phi));
                if (vals_out) vals_out[out] = e->val;
                if (bucket_of) {
                    int64_t k = (int64_t)(e->tag / (uint64_t)M), j = (int64_t)(e->tag % (uint64_t)M);
                    bucket_of[k * m + j] = (int32_t)i;
                }
                ++out;
            }
            if (++h[0].pos == h[0].len) h[0] = h[--cnt];
            if (cnt > 0) heap_down(h, cnt, 0);
        }
    }

    for (int64_t k = 0; k < R; ++k) { free(local[k]); free(Sk[k]); }
    for (int64_t i = 0; i < p; ++i) free(Z[i]);
    free(local); free(len); free(nreal); free(Y); free(Spl); free(Sk); free(c);
    free(bucket_len); free(recv_off); free(Z); free(h);
    return out == n ? OR_OK : OR_EINVAL;
}
