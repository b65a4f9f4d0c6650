"""Pins of the iterative version's oracle (oracle/iterative.py; Sec. 5.1, m
rounds of k-way partitioning): the output is the stable sort; one round is
Sort_Det_BSP exactly (the C oracle's splitters, buckets and per-key buckets);
every key ends on the processor its own classification by each round's
splitters names; every round's buckets keep Lemma 5.1's bound inside their
group; brute force over tiny inputs; planted mistakes each fail a pin."""
import itertools
import sys
import types

import numpy as np
import pytest

import bsp_inputs as gen
import oracle
from oracle import iterative as it


def _le(a, b):
    """a precedes or equals b in (pad, phi, tag) order, written out per record."""
    return (int(a["pad"]), int(a["phi"]), int(a["tag"])) <= (int(b["pad"]), int(b["phi"]), int(b["tag"]))


def _input_records(keys, p, s):
    """Every input key as the record it is in round 1: tag r*M + j."""
    n = keys.shape[0]
    mb = -(-n // p) if n else 0
    M0 = s * max(1, -(-mb // s))
    recs = np.zeros(n, it.REC)
    recs["phi"] = it.phi(keys)
    g = np.arange(n)
    recs["tag"] = (g // mb) * M0 + g % mb if mb else 0
    return recs


def _direct_processor(res, keys, p, k, s):
    """Final processor of every key from the recorded splitters alone: in round
    t the key's group is fixed by its earlier buckets, its bucket there is the
    number of the group's splitters at or below it, and bucket c sends it to the
    c-th subgroup of g/k processors."""
    recs = _input_records(keys, p, s)
    out = np.empty(keys.shape[0], np.int64)
    for e in range(keys.shape[0]):
        first, g = 0, p
        for rnd in res.rounds:
            grp = next(r for r in rnd if r.first == first)
            c = sum(1 for S in grp.splitters if _le(S, recs[e]))
            g //= k
            first += c * g
        out[e] = first
    return out


def _lemma_bound(q, g, x):
    """Lemma 5.1, refined: records of one bucket of a group of g processors."""
    return max((q + g - 1) * x - g + 1, q * x + 1)


def _check_all(mod, keys, p, k, s):
    """Every pin on one input; returns the first failure's name or None."""
    res = mod.sort_iterative(keys, p, k, s)
    n = keys.shape[0]
    if keys.dtype in (np.int32, np.uint32):
        if not np.array_equal(res.positions, np.argsort(keys, kind="stable")):
            return "stable sort"
    else:
        ref = oracle.sort(keys, p, s, p, oracle.REGULAR, 0, vals=np.arange(n, dtype=np.uint32),
                          want_sample=False)
        if not np.array_equal(res.positions, ref.vals.astype(np.int64)):
            return "stable sort"
    if int(res.bucket_sizes.sum()) != n:
        return "key count"
    if not np.array_equal(res.proc_of, _direct_processor(res, keys, p, k, s)):
        return "direct classification"
    g = p
    for t, rnd in enumerate(res.rounds):
        h = g // k
        for grp in rnd:
            q = g * s // k
            if grp.bucket_sizes.max(initial=0) > _lemma_bound(q, g, grp.x):
                return "Lemma 5.1"
            for c in range(k):
                load = res.loads[t + 1][grp.first + c * h: grp.first + (c + 1) * h]
                if load.sum() != grp.bucket_sizes[c] or load.max() - load.min() > 1:
                    return "equal parts"
        g = h
    if k == p and n > 0:
        ref = oracle.sort(keys, p, s, p, oracle.REGULAR, 0, want_bucket_of=True, want_sample=False)
        S = res.rounds[0][0].splitters
        if not (np.array_equal(S["phi"], ref.splitters["phi"])
                and np.array_equal(S["tag"].astype(np.uint64), ref.splitters["tag"])
                and np.array_equal(S["pad"].astype(np.uint32), ref.splitters["pad"])):
            return "Sort_Det_BSP splitters"
        if not np.array_equal(res.bucket_sizes, ref.bucket_sizes) or \
                not np.array_equal(res.proc_of, ref.bucket_of.astype(np.int64)):
            return "Sort_Det_BSP buckets"
    return None


def _few(n, values, seed):
    return np.random.default_rng(seed).integers(0, values, n).astype(np.int32)


INPUTS = [
    ("uniform", lambda: gen.uniform(3000, 16, 1)),
    ("zero_entropy", lambda: gen.zero_entropy(2500)),
    ("staggered", lambda: gen.staggered(4096, 16, 2)),
    ("bucket_sorted", lambda: gen.bucket_sorted(4096, 16, 3)),
    ("det_duplicates", lambda: gen.det_duplicates(4096, 16, 4)),
    ("zipf", lambda: gen.zipf(3333, seed=5)),
    ("few_values", lambda: _few(2049, 3, 6)),
    ("descending", lambda: np.arange(2000, dtype=np.int32)[::-1].copy()),
    ("u32", lambda: gen.uniform_u32(2222, seed=7)),
]
SHAPES = [(16, 4, 8), (16, 2, 4), (16, 16, 8), (64, 4, 4), (8, 2, 40)]


@pytest.mark.parametrize("p,k,s", SHAPES, ids=[f"p{p}_k{k}_s{s}" for p, k, s in SHAPES])
@pytest.mark.parametrize("name,make", INPUTS, ids=[i[0] for i in INPUTS])
def test_iterative_pins(name, make, p, k, s):
    assert _check_all(it, make(), p, k, s) is None


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_float_keys_in_total_order(dt):
    """+-0, +-inf, NaNs of both signs and repeats: the same output as
    Sort_Det_BSP (the result is unique)."""
    rng = np.random.default_rng(11)
    keys = rng.normal(0, 10, 3000).astype(dt)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.5, -1.5], dt)
    keys[rng.integers(0, 3000, 400)] = special[rng.integers(0, special.size, 400)]
    keys[:5] = -keys[:5]  # a negative NaN among them when one was placed there
    keys[7] = -np.float64(np.nan).astype(dt)
    assert _check_all(it, keys, 16, 4, 8) is None


def test_one_round_equals_sort_det_bsp_on_ragged_blocks():
    """n not a multiple of p, s larger than a block (x = 1, pads sampled)."""
    for n, p, s in [(1001, 8, 8), (100, 16, 32), (17, 16, 2), (5, 4, 3)]:
        keys = _few(n, 7, n)
        assert _check_all(it, keys, p, p, s) is None, (n, p, s)


def test_brute_force_tiny_inputs():
    """Every input of 7 keys over {0, 1, 2}, p = 4 processors in two rounds of
    two buckets, s = 1 and 2."""
    for s in (1, 2):
        for t in itertools.product(range(3), repeat=7):
            keys = np.array(t, np.int32)
            assert _check_all(it, keys, 4, 2, s) is None, (t, s)


def test_degenerate_sizes():
    for n in (0, 1, 3):
        keys = np.arange(n, dtype=np.int32)[::-1].copy()
        res = it.sort_iterative(keys, 4, 2, 2)
        assert np.array_equal(res.keys, np.sort(keys)) and int(res.bucket_sizes.sum()) == n
    res = it.sort_iterative(np.array([3, 1, 2], np.int32), 1, 2, 4)  # p = 1: no round
    assert res.keys.tolist() == [1, 2, 3] and res.rounds == []


def test_invalid_parameters():
    with pytest.raises(ValueError):
        it.sort_iterative(np.zeros(10, np.int32), 12, 4, 2)  # p not a power of k
    with pytest.raises(ValueError):
        it.sort_iterative(np.zeros(10, np.int32), 4, 1, 2)
    with pytest.raises(ValueError):
        it.sort_iterative(np.zeros(10, np.int32), 4, 2, 0)


MUTANTS = {
    "splitter_rank": ("S = Y[np.arange(1, k) * q - 1]", "S = Y[np.arange(1, k) * q]"),
    "sample_position": ("padded[np.arange(1, s + 1) * x - 1]", "padded[np.arange(0, s) * x]"),
    "tie_to_lower_bucket": ('(a["tag"] <= b["tag"])', '(a["tag"] < b["tag"])'),
    "subgroup_interleaved": ("new[first + c * h + j]", "new[first + j * k + c]"),
    "int32_sign": ('^ np.uint32(0x80000000)).astype', '^ np.uint32(0)).astype'),
    "pad_with_block_max": ("padded = np.concatenate([a, pads])",
                           "padded = np.concatenate([a, np.repeat(a[-1:], len(pads)) if len(a) else pads])"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_fail_a_pin(name):
    src = open(it.__file__).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType("iterative_mutant")
    sys.modules[mod.__name__] = mod  # dataclasses look their module up
    try:
        exec(compile(src.replace(old, new), "iterative_mutant", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    cases = [(make(), p, k, s) for _, make in INPUTS for p, k, s in SHAPES[:4]]
    cases.append((np.array([-5, 3, -1, 7, 0, -2, 2], np.int32), 4, 2, 1))
    cases.append((gen.uniform(3000, 16, 1) - (1 << 30), 16, 4, 8))  # keys of both signs
    failed = None
    for keys, p, k, s in cases:
        try:
            failed = _check_all(mod, keys, p, k, s)
        except Exception as exc:  # a mutant may also break outright
            failed = repr(exc)
        if failed:
            break
    assert failed, f"mutant {name} passes every pin"
