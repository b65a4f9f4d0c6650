"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

Each check below is independent of the oracle's own code path:
  * hand-worked examples of Fig. 1 (tests/golden/*.json);
  * the output against numpy's sort of the typed keys (a library routine);
  * bucket sizes and per-key buckets against the direct count of Lemma 5.1's
    proof (b_i = number of keys smaller than splitter i), done with numpy on
    the typed keys, not on the oracle's order transform;
  * brute force over every input of length <= 5 on the alphabet {0,1,2};
  * the closed form for all-equal keys (Sec. 2: balance "even if all keys are
    the same"), the bound of Lemma 5.1 and the bound of Claim 5.1;
  * the random-sample stream against numpy's Philox4x64 (a library routine);
  * invariance under strictly monotone maps of the keys and, in random mode,
    under the number of virtual processors.
"""
import glob
import itertools
import json
import math
import os

import numpy as np
import pytest

import bsp_inputs as gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NP_DTYPES = {"uint32": np.uint32, "int32": np.int32, "float32": np.float32, "float64": np.float64}


def _as_keys(vals, dtype):
    dt = np.dtype(NP_DTYPES[dtype])
    if dt.kind == "f":
        bits = np.array([int(v, 16) for v in vals], dtype=np.uint32 if dt.itemsize == 4 else np.uint64)
        return bits.view(dt)
    return np.array(vals, dtype=dt)


def _global_index(tag, pl):
    k, j = divmod(int(tag), int(pl.M))
    return k * int(pl.m) + j


def direct_counts(keys, splitters, pl):
    """b_i = #{keys smaller than S_i} in the stable order (key, input position).

    Computed from the typed keys with numpy comparisons (Lemma 5.1 proof)."""
    n = keys.shape[0]
    b = [0]
    for rec in splitters:
        if rec["pad"]:
            b.append(n)
            continue
        g = _global_index(rec["tag"], pl)
        v = keys[g]
        b.append(int(np.count_nonzero(keys < v)) + int(np.count_nonzero(keys[:g] == v)))
    b.append(n)
    return np.array(b, np.int64)


def stable_ranks(keys):
    order = np.argsort(keys, kind="stable")
    r = np.empty(keys.shape[0], np.int64)
    r[order] = np.arange(keys.shape[0])
    return r


def check_against_direct(keys, res):
    pl = res.plan
    b = direct_counts(keys, res.splitters, pl)
    assert np.all(np.diff(b) >= 0)
    assert np.array_equal(res.bucket_sizes, np.diff(b))
    if res.bucket_of is not None:
        want = np.searchsorted(b[1:-1], stable_ranks(keys), side="right")
        assert np.array_equal(res.bucket_of, want)


# ---------------------------------------------------------------- golden files

@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))),
                         ids=lambda p: os.path.basename(p))
def test_golden_hand_worked(path):
    g = json.load(open(path))
    keys = _as_keys(g["keys"], g["dtype"])
    vals = np.array(g["vals"], np.uint32)
    mode = oracle.REGULAR if g["sampling"] == "regular" else oracle.RANDOM
    res = oracle.sort(keys, g["p"], g["s"], g["runs"], mode, g["seed"], vals=vals,
                      want_bucket_of=True)
    for f, v in g["plan"].items():
        assert getattr(res.plan, f) == v, f
    got_sample = [[hex(int(r["phi"])), int(r["tag"]), int(r["pad"])] for r in res.sample]
    assert got_sample == [[hex(int(a, 16)), b, c] for a, b, c in g["sample"]]
    got_spl = [[hex(int(r["phi"])), int(r["tag"]), int(r["pad"])] for r in res.splitters]
    assert got_spl == [[hex(int(a, 16)), b, c] for a, b, c in g["splitters"]]
    assert res.bucket_sizes.tolist() == g["bucket_sizes"]
    assert res.pad_sizes.tolist() == g["pad_sizes"]
    assert res.bucket_of.tolist() == g["bucket_of"]
    want_keys = _as_keys(g["sorted_keys"], g["dtype"])
    assert res.keys.tobytes() == want_keys.tobytes()
    assert res.vals.tolist() == g["sorted_vals"]


# ---------------------------------------------------------------- plan defaults

def test_paper_default_parameters():
    # Sec. 6.1: regular sample p^2 ceil(lg lg n); random sample 2 p lg^2 n
    assert oracle.plan(2**28, 4096).s == 5 * 4096
    assert oracle.plan(2**20, 64).s == 5 * 64
    assert oracle.plan(2**16, 16).s == 4 * 16
    assert oracle.plan(2**26, 1024, sampling=oracle.RANDOM).s == 2 * 26 * 26
    assert oracle.plan(2**28, 4096, sampling=oracle.RANDOM).s == 1568
    assert oracle.plan(2**26, 1024, sampling=oracle.RANDOM).sample_size == 1352 * 1024 - 1
    pl = oracle.plan(2**28, 4096, s=4096, runs=4096)
    assert (pl.m, pl.M, pl.x, pl.q) == (65536, 65536, 16, 4096)
    assert oracle.plan(10, 3, s=2, runs=2) is None          # p does not divide R*s
    assert oracle.plan(10, 0) is None
    assert oracle.plan(-1, 4) is None


# ---------------------------------------------------------------- output vs numpy

CASES = [
    ("uint32", lambda n, p: gen.uniform_u32(n, 3)),
    ("uniform", lambda n, p: gen.uniform(n, p, 1)),
    ("gaussian", lambda n, p: gen.gaussian(n, p, 2)),
    ("bucket_sorted", lambda n, p: gen.bucket_sorted(n, p, 3)),
    ("staggered", lambda n, p: gen.staggered(n, p, 4)),
    ("zero_entropy", lambda n, p: gen.zero_entropy(n)),
    ("zipf", lambda n, p: gen.zipf(n, seed=5)),
    ("gmm_f64", lambda n, p: gen.gmm(n, seed=6)),
    ("f32", lambda n, p: gen.gmm(n, seed=7).astype(np.float32)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("mode", [oracle.REGULAR, oracle.RANDOM], ids=["regular", "random"])
@pytest.mark.parametrize("n,p,runs,s", [(5000, 16, 0, 0), (4099, 8, 12, 6), (777, 32, 32, 1)])
def test_output_and_sizes_match_numpy(name, make, mode, n, p, runs, s):
    keys = make(n, p)
    vals = np.arange(n, dtype=np.uint32)
    if mode == oracle.RANDOM and s == 1:
        s = 3
    res = oracle.sort(keys, p, s, runs, mode, seed=11, vals=vals, want_bucket_of=True)
    order = np.argsort(keys, kind="stable")
    assert res.keys.tobytes() == keys[order].tobytes()
    assert np.array_equal(res.vals, order.astype(np.uint32))
    check_against_direct(keys, res)
    # the sample is sorted in the total order and holds the splitters at ranks i*q
    smp = res.sample
    key3 = list(zip(smp["pad"].tolist(), smp["phi"].tolist(), smp["tag"].tolist()))
    assert key3 == sorted(key3)
    q = res.plan.q
    for i in range(1, p):
        assert smp[i * q - 1].tobytes() == res.splitters[i - 1].tobytes()


# ---------------------------------------------------------------- brute force

def _run_records(keys, pl):
    """(pad, key, tag) triples held by each virtual processor, Python order."""
    n = len(keys)
    runs = []
    for k in range(pl.R):
        lo = k * pl.m
        recs = []
        for j in range(pl.M if pl.sampling == oracle.REGULAR else pl.m):
            if lo + j < n and j < pl.m:
                recs.append((0, keys[lo + j], k * pl.M + j))
            elif pl.sampling == oracle.REGULAR:
                recs.append((1, 0, k * pl.M + j))
        runs.append(recs)
    return runs


@pytest.mark.parametrize("p,runs,s", [(1, 1, 1), (1, 2, 2), (2, 1, 2), (2, 2, 1), (2, 2, 2),
                                      (3, 3, 1), (2, 3, 2), (3, 1, 3), (4, 2, 2), (2, 4, 1)])
def test_brute_force_tiny_regular(p, runs, s):
    for n in range(0, 6):
        for tup in itertools.product((0, 1, 2), repeat=n):
            keys = np.array(tup, np.int32)
            res = oracle.sort(keys, p, s, runs, oracle.REGULAR, vals=np.arange(n, dtype=np.uint32),
                              want_bucket_of=True)
            assert res.keys.tolist() == sorted(tup)
            if n == 0:
                continue
            pl = res.plan
            check_against_direct(keys, res)
            runs_recs = _run_records(list(tup), pl)
            # regular sample: record j of processor k has exactly j*x records of
            # its block at or below it (it ends segment j, Fig. 1 step 4)
            smp = res.sample
            by_run = {}
            for r in smp:
                k = int(r["tag"]) // pl.M
                by_run.setdefault(k, []).append(r)
            for k, recs in by_run.items():
                assert len(recs) == pl.s
                block = runs_recs[k]
                for r in recs:
                    t = int(r["tag"])
                    me = next(b for b in block if b[2] == t)
                    below = sum(1 for b in block if b <= me)
                    assert below % pl.x == 0
                ranks = sorted(sum(1 for b in block if b <= next(bb for bb in block if bb[2] == int(r["tag"])))
                               for r in recs)
                assert ranks == [j * pl.x for j in range(1, pl.s + 1)]
            # splitter i has exactly i*q sample records at or below it (Fig. 1 step 6)
            triples = [(int(r["pad"]), int(r["phi"]), int(r["tag"])) for r in smp]
            for i in range(1, p):
                sp = res.splitters[i - 1]
                me = (int(sp["pad"]), int(sp["phi"]), int(sp["tag"]))
                assert sum(1 for t in triples if t <= me) >= i * pl.q
                assert sum(1 for t in triples if t < me) < i * pl.q
            # Lemma 5.1 (refined): records per bucket, pads included
            bound = max((pl.q + pl.R - 1) * pl.x - pl.R + 1, pl.q * pl.x + 1)
            assert np.all(res.bucket_sizes + res.pad_sizes <= bound)


@pytest.mark.parametrize("p,runs,s", [(1, 1, 1), (2, 1, 1), (2, 3, 2), (3, 2, 1), (4, 1, 2)])
def test_brute_force_tiny_random(p, runs, s):
    for n in range(1, 6):
        for tup in itertools.product((0, 1, 2), repeat=n):
            keys = np.array(tup, np.int32)
            res = oracle.sort(keys, p, s, runs, oracle.RANDOM, seed=n * 7 + 1,
                              vals=np.arange(n, dtype=np.uint32), want_bucket_of=True)
            assert res.keys.tolist() == sorted(tup)
            check_against_direct(keys, res)
            pos = [oracle.position(n * 7 + 1, j, n) for j in range(res.plan.sample_size)]
            want = sorted((int(keys[g]), g) for g in pos)
            assert [(int(np.uint32(r["phi"]) ^ np.uint32(0x80000000)), int(r["tag"]))
                    for r in res.sample] == [(k & 0xFFFFFFFF, g) for k, g in want]


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("R,p,s,n", [(4, 4, 4, 64), (8, 4, 2, 200), (16, 16, 48, 16 * 96),
                                      (6, 3, 5, 61), (64, 64, 8, 2**14)])
def test_all_equal_keys_closed_form(R, p, s, n):
    """All keys equal: the order is the tag order, so sample record j of block k
    has tag k*M + j*x - 1 and splitter i is the sample record of rank i*q."""
    keys = np.full(n, 7, np.int32)
    res = oracle.sort(keys, p, s, R, oracle.REGULAR, want_bucket_of=True)
    pl = res.plan
    m, M, x, q = pl.m, pl.M, pl.x, pl.q
    def nreal(k):
        return max(0, min(m, n - k * m))
    recs = sorted((int(j * x - 1 >= nreal(k)), k * M + j * x - 1)
                  for k in range(R) for j in range(1, s + 1))   # pads follow every key
    tags = [t for _, t in recs]
    assert [int(t) for t in res.sample["tag"]] == tags
    assert [int(v) for v in res.sample["pad"]] == [pd for pd, _ in recs]
    b = [0]
    for i in range(1, p):
        t = tags[i * q - 1]
        k, j = divmod(t, M)
        b.append(n if k * m + j >= n or j >= m else k * m + j)
    b.append(n)
    assert res.bucket_sizes.tolist() == np.diff(b).tolist()
    if n == R * m and M == m:
        # no pads: sizes (M-1, M, ..., M, M+1) when q = s (R = p)
        if R == p:
            assert res.bucket_sizes.tolist() == [M - 1] + [M] * (p - 2) + [M + 1]


def test_all_equal_keys_random_closed_form():
    n, p, s, seed = 5000, 16, 12, 99
    keys = np.full(n, -3, np.int32)
    res = oracle.sort(keys, p, s, 0, oracle.RANDOM, seed=seed)
    bg = np.random.Philox(key=np.array([seed, 0], np.uint64),
                          counter=np.array([2**64 - 1] * 4, np.uint64))
    h = bg.random_raw(s * p - 1).astype(object)
    pos = sorted(int((int(v) * n) >> 64) for v in h)
    assert [int(t) for t in res.sample["tag"]] == pos
    b = [0] + [pos[i * s - 1] for i in range(1, p)] + [n]
    assert res.bucket_sizes.tolist() == np.diff(b).tolist()


def test_two_value_input():
    rng = np.random.default_rng(5)
    keys = np.where(rng.random(3000) < 0.3, 10, 20).astype(np.int32)
    for mode in (oracle.REGULAR, oracle.RANDOM):
        res = oracle.sort(keys, 8, 0, 0, mode, seed=3, want_bucket_of=True)
        check_against_direct(keys, res)


# ---------------------------------------------------------------- random stream

def test_philox_stream_matches_numpy():
    for seed in (0, 1, 12345, 2**63 + 17):
        bg = np.random.Philox(key=np.array([seed, 0], np.uint64),
                              counter=np.array([2**64 - 1] * 4, np.uint64))
        want = bg.random_raw(37)
        got = [oracle.draw(seed, j) for j in range(37)]
        assert got == [int(v) for v in want]
        for k in (1, 20, 31):
            assert [oracle.position(seed, j, 2**k) for j in range(37)] == [int(v) >> (64 - k) for v in want]


# ---------------------------------------------------------------- bounds

def test_lemma_5_1_bound_regular():
    for name, keys in [("U", gen.uniform(2**16, 16, 1)), ("zipf", gen.zipf(2**16, seed=2)),
                       ("B", gen.bucket_sorted(2**16, 16, 3)), ("S", gen.staggered(2**16, 16, 4)),
                       ("equal", gen.zero_entropy(2**16))]:
        for p, runs, s in [(16, 0, 0), (16, 16, 16), (8, 32, 4), (16, 16, 3)]:
            res = oracle.sort(keys, p, s, runs, oracle.REGULAR)
            pl = res.plan
            tot = res.bucket_sizes + res.pad_sizes
            refined = max((pl.q + pl.R - 1) * pl.x - pl.R + 1, pl.q * pl.x + 1)
            assert tot.max() <= refined, name
            assert tot.max() <= (pl.s + pl.p) * pl.x if pl.R == pl.p else True
            if pl.R == pl.p and pl.s % pl.p == 0:
                r = pl.s // pl.p
                n = keys.shape[0]
                assert tot.max() <= (1 + 1 / r) * (n + pl.p * pl.s) / pl.p + 1e-9


def _claim_5_1_eps(n, k, s, rho=1.0):
    base = 2 * rho * math.log(n) + math.log(2 * math.pi * k * k * (k * s - 1)
                                            * math.exp(1.0 / (3 * (k * s - 1))))
    lo, hi = 1e-6, 1.0
    if (1 + hi) / hi**2 * base > s:
        return None
    for _ in range(100):
        mid = (lo + hi) / 2
        if (1 + mid) / mid**2 * base <= s:
            hi = mid
        else:
            lo = mid
    return hi


def test_claim_5_1_bound_random():
    n, p = 2**13, 8
    s = oracle.plan(n, p, sampling=oracle.RANDOM).s
    eps = _claim_5_1_eps(n, p, s)
    assert eps is not None and eps < 1
    bound = math.ceil((1 + eps) * (n - p + 1) / p) + s
    keys = gen.uniform(n, p, 1)
    worst = 0
    for seed in range(300):
        res = oracle.sort(keys, p, 0, 0, oracle.RANDOM, seed=seed, want_sample=False)
        worst = max(worst, int(res.bucket_sizes.max()))
    assert worst <= bound


@pytest.mark.parametrize("mode", [oracle.REGULAR, oracle.RANDOM], ids=["regular", "random"])
def test_paper_observed_imbalance_below_15_percent(mode):
    # Sec. 6.4: max imbalance below 15% with omega_n = lg lg n (det) and
    # omega_n^2 = lg n (ran) at the paper's sizes
    n, p = 2**20, 64
    keys = gen.uniform(n, p, 1)
    res = oracle.sort(keys, p, 0, 0, mode, seed=21, want_sample=False)
    assert res.bucket_sizes.max() / (n / p) - 1 < 0.15


# ---------------------------------------------------------------- metamorphic

def test_monotone_key_maps_keep_the_partition():
    keys = gen.gaussian(20000, 16, 3)          # int32 values in [0, 2^31)
    maps = [lambda k: (k.astype(np.int64) - 2**30).astype(np.int32),
            lambda k: (k.astype(np.int64) + 2**31).astype(np.uint32),
            lambda k: k.astype(np.float64) / 7.0,
            lambda k: -1.0 / (k.astype(np.float64) + 1.0)]
    for mode in (oracle.REGULAR, oracle.RANDOM):
        a = oracle.sort(keys, 16, 0, 0, mode, seed=5, want_bucket_of=True)
        for f in maps:
            b = oracle.sort(f(keys), 16, 0, 0, mode, seed=5, want_bucket_of=True)
            assert np.array_equal(a.bucket_sizes, b.bucket_sizes)
            assert np.array_equal(a.bucket_of, b.bucket_of)
            assert np.array_equal(a.splitters["tag"], b.splitters["tag"])


def test_random_mode_independent_of_virtual_processors():
    keys = gen.zipf(30000, seed=9)
    ref = oracle.sort(keys, 32, 0, 0, oracle.RANDOM, seed=77, want_bucket_of=True)
    for runs in (1, 7, 32, 100):
        r = oracle.sort(keys, 32, 0, runs, oracle.RANDOM, seed=77, want_bucket_of=True)
        assert np.array_equal(r.bucket_sizes, ref.bucket_sizes)
        assert np.array_equal(r.bucket_of, ref.bucket_of)
        assert np.array_equal(r.splitters, ref.splitters)


@pytest.mark.parametrize("mode", [oracle.REGULAR, oracle.RANDOM], ids=["regular", "random"])
@pytest.mark.parametrize("make,p,runs,s", [
    (lambda: gen.uniform(200_003, 64, 3), 64, 0, 0),
    (lambda: gen.zipf(150_000, seed=5), 32, 48, 64),
    (lambda: gen.gmm(100_000, seed=2), 16, 0, 0),
], ids=["uniform", "zipf", "gmm"])
def test_threads_run_the_same_supersteps(mode, make, p, runs, s):
    """The processors of one superstep write disjoint data (BSP model): running
    them on several host threads changes nothing, bit for bit."""
    keys = make()
    vals = np.arange(keys.shape[0], dtype=np.uint32)
    if mode == oracle.RANDOM:
        runs, s = 0, 0
    one = oracle.sort(keys, p, s, runs, mode, 11, vals=vals, want_bucket_of=True, threads=1)
    many = oracle.sort(keys, p, s, runs, mode, 11, vals=vals, want_bucket_of=True, threads=5)
    for f in ("keys", "vals", "bucket_sizes", "pad_sizes", "sample", "splitters", "bucket_of"):
        assert getattr(one, f).tobytes() == getattr(many, f).tobytes(), f
    order = np.argsort(keys, kind="stable")
    assert many.keys.tobytes() == keys[order].tobytes()
    assert np.array_equal(many.vals, order)


def test_std_sort_baseline_sorts():
    """The std::sort / std::stable_sort baseline timed beside the oracle sorts."""
    for keys in (gen.uniform(100_000, 4, 1), gen.uniform_u32(50_000, 2), gen.gmm(30_000, seed=1)):
        for stable in (False, True):
            assert np.array_equal(oracle.std_sort(keys, stable=stable), np.sort(keys))


# ------------------------------------- partition (Fig. 1 step 9), Sort_Ran_BSP (Fig. 2),
#                                        and the version without duplicate handling

def _partition_direct(keys, res):
    """c[k][i] of every block: #{records of block k preceding S_i}, from numpy
    comparisons of the typed keys and input positions; pads follow every key
    and precede a pad splitter of a larger tag (Lemma 5.1's padding)."""
    pl = res.plan
    n, m, M, R, p = keys.shape[0], int(pl.m), int(pl.M), int(pl.R), int(pl.p)
    padded = pl.sampling == oracle.REGULAR
    out = np.zeros((R, p + 1), np.int64)
    for k in range(R):
        lo, hi = min(n, k * m), min(n, (k + 1) * m)
        blk, pos = keys[lo:hi], np.arange(lo, hi)
        held = M if padded else hi - lo
        out[k, p] = held
        for i, rec in enumerate(res.splitters, start=1):
            if rec["pad"]:
                # every key, and the pads of this block whose tag is smaller
                tags = k * M + np.arange(hi - lo, held)
                out[k, i] = (hi - lo) + int(np.count_nonzero(tags < int(rec["tag"])))
                continue
            g = _global_index(rec["tag"], pl)
            v = keys[g]
            out[k, i] = int(np.count_nonzero(blk < v)) + int(np.count_nonzero((blk == v) & (pos < g)))
    return out


PARTITION_CASES = [
    ("uniform_regular", lambda: gen.uniform(5000, 8, 3), oracle.REGULAR, 8, 0, 0),
    ("zipf_regular_pads", lambda: gen.zipf(4999, seed=5), oracle.REGULAR, 8, 16, 32),
    ("equal_regular", lambda: np.full(3000, 7, np.int32), oracle.REGULAR, 4, 8, 8),
    ("zipf_random", lambda: gen.zipf(6001, seed=6), oracle.RANDOM, 16, 0, 0),
    ("gmm_random", lambda: gen.gmm(4000, seed=2), oracle.RANDOM, 8, 4, 3),
]


@pytest.mark.parametrize("name,make,mode,p,runs,s", PARTITION_CASES, ids=[c[0] for c in PARTITION_CASES])
def test_partition_is_the_direct_count(name, make, mode, p, runs, s):
    keys = make()
    res = oracle.sort(keys, p, s, runs, mode, 9, want_partition=True)
    assert np.array_equal(res.partition, _partition_direct(keys, res))


RAN_CASES = [
    ("uniform_i32", lambda: gen.uniform(20000, 16, 1), 16, 0),
    ("zipf_i32", lambda: gen.zipf(20000, seed=3), 32, 0),
    ("equal_i32", lambda: np.full(5000, -3, np.int32), 8, 4),
    ("gmm_f64", lambda: gen.gmm(8000, seed=7), 64, 16),
    ("u32", lambda: gen.uniform_u32(7777, seed=4), 4, 2),
]


@pytest.mark.parametrize("name,make,p,runs", RAN_CASES, ids=[c[0] for c in RAN_CASES])
def test_sort_ran_bsp_equals_sort_iran_bsp(name, make, p, runs):
    """Sort_Ran_BSP (Fig. 2: classify every key, route, sort each bucket) and
    Sort_IRan_BSP (Fig. 3: sort, partition by binary search, route, merge)
    use the same splitters, so they give the same buckets, per-key buckets and
    output; the Fig. 2 grouping of block k puts keys of bucket < i first."""
    keys = make()
    vals = np.arange(keys.shape[0], dtype=np.uint32)
    a = oracle.sort(keys, p, 0, runs, oracle.RANDOM, 11, vals=vals, want_bucket_of=True)
    b = oracle.sort(keys, p, 0, runs, oracle.RANDOM, 11, vals=vals, want_bucket_of=True,
                    variant=oracle.RAN, want_partition=True)
    assert np.array_equal(a.keys, b.keys) and np.array_equal(a.vals, b.vals)
    assert np.array_equal(a.bucket_sizes, b.bucket_sizes)
    assert np.array_equal(a.bucket_of, b.bucket_of)
    assert np.array_equal(a.splitters, b.splitters)
    check_against_direct(keys, b)
    m, n = int(b.plan.m), keys.shape[0]
    for k in range(int(b.plan.R)):
        bof = b.bucket_of[min(n, k * m):min(n, (k + 1) * m)]
        want = np.searchsorted(np.sort(bof), np.arange(p + 1), side="left")
        assert np.array_equal(b.partition[k], want)


def test_sort_ran_bsp_needs_random_sampling():
    with pytest.raises(ValueError):
        oracle.sort(gen.uniform(1000, 4, 1), 4, 0, 0, oracle.REGULAR, variant=oracle.RAN)


DUP_CASES = [
    ("zipf_regular", lambda: gen.zipf(30000, seed=8), oracle.REGULAR, 16, 0, 0),
    ("zipf_random", lambda: gen.zipf(30000, seed=8), oracle.RANDOM, 16, 0, 0),
    ("equal_regular_pads", lambda: np.full(3001, 5, np.int32), oracle.REGULAR, 4, 8, 8),
    ("uniform_random", lambda: gen.uniform(20000, 16, 2), oracle.RANDOM, 32, 0, 0),
    ("f32_regular", lambda: gen.gmm(9000, seed=1).astype(np.float32), oracle.REGULAR, 8, 0, 0),
]


@pytest.mark.parametrize("name,make,mode,p,runs,s", DUP_CASES, ids=[c[0] for c in DUP_CASES])
def test_without_duplicate_handling_buckets_are_value_counts(name, make, mode, p, runs, s):
    """Without the tags (Sec. 6.1's version without duplicate handling) the
    sample and splitters are unchanged, the output is the same stable sort,
    and a key's bucket is the number of splitters whose key is not above it
    (numpy searchsorted on the splitters' typed keys); every pad, equal to
    the pad splitters, lands in the last bucket."""
    keys = make()
    vals = np.arange(keys.shape[0], dtype=np.uint32)
    t = oracle.sort(keys, p, s, runs, mode, 4, vals=vals, want_bucket_of=True)
    d = oracle.sort(keys, p, s, runs, mode, 4, vals=vals, want_bucket_of=True, duplicates=oracle.DUP_OFF)
    assert np.array_equal(t.sample, d.sample) and np.array_equal(t.splitters, d.splitters)
    assert np.array_equal(t.keys, d.keys) and np.array_equal(t.vals, d.vals)
    real = [keys[_global_index(r["tag"], d.plan)] for r in d.splitters if not r["pad"]]
    want = np.searchsorted(np.array(real, keys.dtype), keys, side="right")
    assert np.array_equal(d.bucket_of, want)
    assert np.array_equal(d.bucket_sizes, np.bincount(want, minlength=p))
    assert d.pad_sizes[:-1].sum() == 0
    assert d.pad_sizes[-1] == (int(d.plan.R) * int(d.plan.M) - keys.shape[0] if mode == oracle.REGULAR else 0)
    if name.startswith("zipf") or name.startswith("equal"):
        assert not np.array_equal(t.bucket_sizes, d.bucket_sizes)
