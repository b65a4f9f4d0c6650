"""GPU path vs the oracle, element by element, through the C ABI.

Compared bit for bit: sorted keys, payloads, bucket sizes, splitters (phi, tag,
pad), the sorted sample, per-key buckets (n <= 2^22) and pad counts.  Sizes span
several routing tiles (65536 keys), chunks (4096 keys) and cluster slots, with
ragged tails; the edge cases are n = 0, 1, p-1, p, p+1, p = 1, all-equal keys,
buckets larger than one cluster's shared memory (out-of-core path) and a bucket
region too small on purpose (overflow is reported, nothing is written past it).
"""
import glob
import json
import os

import numpy as np
import pytest

import bsp_inputs as gen
import oracle
from tests.gpu_util import assert_same, run_gpu
from tests.test_oracle import GOLDEN, _as_keys

pytestmark = pytest.mark.gpu

MODES = [oracle.REGULAR, oracle.RANDOM]
MODE_IDS = ["regular", "random"]


def ref_sort(keys, p, s=0, runs=0, mode=0, seed=0, vals=None):
    return oracle.sort(keys, p, s, runs, mode, seed, vals=vals, want_bucket_of=keys.shape[0] <= (1 << 22),
                       want_partition=mode == oracle.REGULAR)


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))),
                         ids=lambda p: os.path.basename(p))
def test_golden_hand_worked_on_gpu(path):
    g = json.load(open(path))
    keys = _as_keys(g["keys"], g["dtype"])
    vals = np.array(g["vals"], np.uint32)
    r = run_gpu(keys, g["p"], g["s"], g["runs"], oracle.REGULAR, vals=vals)
    assert r.stats.status == 0
    assert r.keys.tobytes() == _as_keys(g["sorted_keys"], g["dtype"]).tobytes()
    assert r.vals.tolist() == g["sorted_vals"]
    assert r.bucket_sizes.tolist() == g["bucket_sizes"]
    assert r.pad_sizes.tolist() == g["pad_sizes"]
    assert r.bucket_of.tolist() == g["bucket_of"]
    assert [[int(x["phi"]), int(x["tag"]), int(x["pad"])] for x in r.splitters] == \
        [[int(a, 16), b, c] for a, b, c in g["splitters"]]
    assert [[int(x["phi"]), int(x["tag"]), int(x["pad"])] for x in r.sample] == \
        [[int(a, 16), b, c] for a, b, c in g["sample"]]


DTYPE_KEYS = {
    "i32": lambda n, p, seed: gen.uniform(n, p, seed),
    "u32": lambda n, p, seed: gen.uniform_u32(n, seed),
    "f32": lambda n, p, seed: gen.gmm(n, seed=seed).astype(np.float32),
    "f64": lambda n, p, seed: gen.gmm(n, seed=seed),
}


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("dt", sorted(DTYPE_KEYS))
@pytest.mark.parametrize("n,p", [(1, 4), (3, 4), (4, 4), (5, 4), (1000, 7), (65537, 16), (300_001, 64)])
@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
def test_edge_sizes_and_dtypes(mode, dt, n, p, pairs):
    keys = DTYPE_KEYS[dt](n, p, 5)
    vals = np.arange(n, dtype=np.uint32)[::-1].copy() if pairs else None
    s = 0
    try:
        ref = ref_sort(keys, p, s, 0, mode, 9, vals)
    except ValueError:
        pytest.skip("parameters invalid for this n")
    gpu = run_gpu(keys, p, s, 0, mode, 9, vals)
    assert_same(gpu, ref)


def test_empty_input():
    keys = np.zeros(0, np.int32)
    r = run_gpu(keys, 8, debug=False)
    assert r.stats.status == 0
    assert r.keys.shape == (0,)
    assert r.bucket_sizes.tolist() == [0] * 8


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_single_bucket(mode):
    keys = gen.gaussian(100_000, 4, 3)
    ref = ref_sort(keys, 1, 0, 4 if mode == oracle.REGULAR else 0, mode, 5)
    gpu = run_gpu(keys, 1, 0, 4 if mode == oracle.REGULAR else 0, mode, 5)
    assert_same(gpu, ref)


ALL_DISTRIBUTIONS = {**gen.DISTRIBUTIONS, **gen.EXTRA_DISTRIBUTIONS}


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("name", sorted(ALL_DISTRIBUTIONS))
def test_distributions_2e20(mode, name):
    n, p = 1 << 20, 256
    keys = ALL_DISTRIBUTIONS[name](n, p, 1)
    vals = np.arange(n, dtype=np.uint32)
    ref = ref_sort(keys, p, 0, 0, mode, 21, vals)
    gpu = run_gpu(keys, p, 0, 0, mode, 21, vals)
    assert_same(gpu, ref)


@pytest.mark.parametrize("s", [8, 512], ids=["s8_literal", "s512"])
def test_config1_regular_u32_2e20(s):
    """n = 2^20 uint32 uniform on [0, 2^32), p = 64, R = 64, regular oversampling."""
    keys = gen.uniform_u32(1 << 20, seed=1)
    ref = ref_sort(keys, 64, s, 64, oracle.REGULAR)
    gpu = run_gpu(keys, 64, s, 64, oracle.REGULAR)
    assert_same(gpu, ref)


@pytest.mark.parametrize("refine", [1, 2, 4])
def test_refinement_changes_nothing(refine):
    keys = gen.uniform(1 << 21, 256, 2)
    ref = ref_sort(keys, 256, 0, 0, oracle.RANDOM, 4)
    gpu = run_gpu(keys, 256, 0, 0, oracle.RANDOM, 4, refine=refine)
    assert_same(gpu, ref)
    assert gpu.plan.vbuckets == 256 * refine


def test_zipf_pairs_regular_duplicates():
    """Duplicate-heavy pairs with the tag-free tie-break (Sec. 5.1.1), regular mode."""
    n, p = 1 << 22, 256
    keys = gen.zipf(n, seed=3)
    vals = np.arange(n, dtype=np.uint32)
    ref = ref_sort(keys, p, p, p, oracle.REGULAR, 0, vals)
    gpu = run_gpu(keys, p, p, p, oracle.REGULAR, 0, vals)
    assert_same(gpu, ref)


def test_gmm_f64_random_small_sample():
    n, p = 1 << 22, 4096
    keys = gen.gmm(n, seed=4)
    ref = ref_sort(keys, p, 16, 0, oracle.RANDOM, 8)
    gpu = run_gpu(keys, p, 16, 0, oracle.RANDOM, 8)
    assert_same(gpu, ref)


@pytest.mark.parametrize("values", [1 << 22, 1 << 17, 1 << 31], ids=["some_repeats", "many_repeats", "distinct"])
@pytest.mark.parametrize("dt", [np.int32, np.uint32, np.float32])
def test_regular_block_counting_sort_and_tags(values, dt):
    """Regular sampling of keys without payloads sorts the blocks by the
    counting sort and recovers the sampled keys' tags: keys that occur once,
    keys repeated a few times in a block (their o-th input occurrence), and
    blocks with so many repeats that they go to the stable block sort."""
    n, p = 1 << 20, 16
    rng = np.random.default_rng(values % 1000 + 7)
    raw = rng.integers(0, values, n)
    keys = (raw.astype(np.float32) - values / 2) if dt == np.float32 else raw.astype(dt)
    ref = ref_sort(keys, p, 1024, 0, oracle.REGULAR, 0)
    gpu = run_gpu(keys, p, 1024, 0, oracle.REGULAR, 0)
    assert_same(gpu, ref)


@pytest.mark.parametrize("name,make,p", [("uniform", lambda: gen.uniform(1 << 21, 256, 3), 256),
                                         ("zipf", lambda: gen.zipf(1 << 21, seed=3), 64),
                                         ("gmm_f64", lambda: gen.gmm(1 << 20, seed=3), 512)],
                         ids=["uniform", "zipf", "gmm_f64"])
def test_random_mode_against_sort_ran_bsp(name, make, p):
    """Random oversampling on the GPU classifies every key and sorts every
    bucket -- the shape of Sort_Ran_BSP (Fig. 2): its per-key buckets, sizes
    and output equal the oracle's Fig. 2 run (as well as its Fig. 3 run)."""
    keys = make()
    ref = oracle.sort(keys, p, 0, 0, oracle.RANDOM, 5, want_bucket_of=True, variant=oracle.RAN)
    gpu = run_gpu(keys, p, 0, 0, oracle.RANDOM, 5)
    assert_same(gpu, ref)


@pytest.mark.parametrize("refine", [1, 2, 4])
def test_f64_sub_buckets_above_the_two_per_sm_clusters(refine):
    """8-byte keys without payloads, few samples per bucket (s = 16): the
    sub-buckets spread from far below to far above the two-CTAs-per-SM
    clusters' 40,960 keys, so the larger keys-only tier (81,920), the stable
    tier and the out-of-core tier all take some."""
    n, p = 1 << 22, 64
    keys = gen.gmm(n, seed=12)
    ref = ref_sort(keys, p, 16, 0, oracle.RANDOM, 5)
    gpu = run_gpu(keys, p, 16, 0, oracle.RANDOM, 5, refine=refine)
    assert_same(gpu, ref)


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
def test_out_of_core_bucket_path(pairs):
    """Buckets far larger than one cluster's shared memory."""
    n, p = 600_000, 2
    keys = gen.gaussian(n, p, 8)
    vals = np.arange(n, dtype=np.uint32) if pairs else None
    ref = ref_sort(keys, p, 0, 0, oracle.RANDOM, 3, vals)
    gpu = run_gpu(keys, p, 0, 0, oracle.RANDOM, 3, vals, refine=1)
    assert gpu.stats.slow_buckets > 0
    assert_same(gpu, ref)


def test_overflow_is_reported_not_written():
    keys = gen.uniform(200_000, 16, 2)
    gpu = run_gpu(keys, 16, 0, 0, oracle.RANDOM, 3, capacity_pct=60, debug=False, expect_status=-4)
    assert gpu.stats.overflow == 1
    assert gpu.stats.status == -4  # BSPS_ERR_BUCKET_OVERFLOW


@pytest.mark.parametrize("name", sorted(gen.DISTRIBUTIONS))
def test_config2_random_2e26(name):
    """n = 2^26 int32, random oversampling, p = 1024, the five seeded inputs."""
    n, p = 1 << 26, 1024
    keys = gen.DISTRIBUTIONS[name](n, p, 1)
    ref = oracle.sort(keys, p, 0, 0, oracle.RANDOM, 1, want_sample=True)
    gpu = run_gpu(keys, p, 0, 0, oracle.RANDOM, 1, bucket_of=False)
    assert_same(gpu, ref)


def _two_close_values_and_outliers(n):
    keys = np.full(n, 1000, np.int32)
    keys[1::2] = 1001
    keys[:: max(1, n // 10)] = 2**30 + np.arange(len(keys[:: max(1, n // 10)]), dtype=np.int32)
    return keys


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_segment_split_fallback(pairs, mode):
    """One split bin holds two distinct keys and more keys than a CTA holds:
    the cluster falls back to full LSD passes through distributed shared memory
    (bucket sort in random mode, block sort of the regular sample in regular mode)."""
    n = 80_000
    keys = _two_close_values_and_outliers(n)
    vals = np.arange(n, dtype=np.uint32) if pairs else None
    if mode == oracle.RANDOM:
        ref = ref_sort(keys, 1, 8, 0, mode, 3, vals)
        gpu = run_gpu(keys, 1, 8, 0, mode, 3, vals, refine=1)
    else:
        ref = ref_sort(keys, 2, 4, 1, mode, 0, vals)
        gpu = run_gpu(keys, 2, 4, 1, mode, 0, vals)
    assert_same(gpu, ref)


def test_zipf_pairs_regular_p4096_2e24():
    """The duplicate-heavy regular configuration at 1/16 of its size:
    p = R = s = 4096 (x = 1 here), Zipf(1.1) on 256 values, payload = index."""
    n, p = 1 << 24, 4096
    keys = gen.zipf(n, seed=3)
    vals = np.arange(n, dtype=np.uint32)
    ref = oracle.sort(keys, p, p, p, oracle.REGULAR, 0, vals=vals, want_sample=True)
    gpu = run_gpu(keys, p, p, p, oracle.REGULAR, 0, vals, bucket_of=False)
    assert_same(gpu, ref)


def test_msd_sample_sort_4096_bins():
    """Random sample of 991,231 records (>= 2^19): the MSD sample sort with 4096
    bins; every sample record and splitter against the oracle."""
    n, p = 1 << 22, 1024
    keys = gen.uniform(n, p, 4)
    ref = oracle.sort(keys, p, 0, 0, oracle.RANDOM, 9, want_sample=True)
    gpu = run_gpu(keys, p, 0, 0, oracle.RANDOM, 9, bucket_of=False)
    assert gpu.plan.sample_size == 2 * 22 * 22 * p - 1
    assert_same(gpu, ref)


def test_msd_sample_sort_8192_bins_regular():
    """Regular sample of 16.8M records (> 8M): 8192 MSD bins, and the keys-only
    block sort of (phi, position) words for the 4096 blocks."""
    n, p = 1 << 24, 4096
    keys = gen.uniform(n, p, 5)
    ref = oracle.sort(keys, p, p, p, oracle.REGULAR, 0, want_sample=True)
    gpu = run_gpu(keys, p, p, p, oracle.REGULAR, 0, bucket_of=False)
    assert gpu.plan.sample_size == p * p
    assert_same(gpu, ref)


@pytest.mark.parametrize("m", [81920, 81919, 40961])
def test_block_sort_at_cluster_capacity(m):
    """Blocks of exactly the keys-only block sort's cluster capacity (8 x 10240),
    one key less (a pad per block), and one key past a 4-CTA cluster."""
    R = p = 4
    keys = gen.uniform(R * m, R, 6)
    ref = ref_sort(keys, p, 32, R, oracle.REGULAR, 0)
    gpu = run_gpu(keys, p, 32, R, oracle.REGULAR, 0)
    assert_same(gpu, ref)


@pytest.mark.parametrize("runs", [8, 2])
def test_block_sort_float_total_order_and_duplicates(runs):
    """float32 blocks with -0/+0, infinities and repeated values through the
    keys-only block sort of (phi, position) words (regular sampling; one CTA
    per block, and clusters of 4)."""
    rng = np.random.default_rng(8)
    n, p = 1 << 16, 8
    keys = rng.normal(0, 1, n).astype(np.float32)
    keys[::97] = -0.0
    keys[1::97] = 0.0
    keys[2::101] = np.inf
    keys[3::101] = -np.inf
    keys[4::7] = keys[5::7][: len(keys[4::7])]
    ref = ref_sort(keys, p, 64, runs, oracle.REGULAR, 0)
    gpu = run_gpu(keys, p, 64, runs, oracle.REGULAR, 0)
    assert_same(gpu, ref)


@pytest.mark.parametrize("dt", ["int32", "float64"])
@pytest.mark.parametrize("span_log2", [19, 20, 21, 23, 25])
def test_bucket_sort_repeat_rates(dt, span_log2):
    """Keys-only bucket sort of 65536-key buckets (clusters of 8) whose values
    repeat at different rates: keys uniform on 2^span consecutive values.  This
    walks a cluster CTA's count sort through its regimes: one value per count
    bin (2^19), occupancy masks with values seen up to three times and bins
    where a value occurs four times or more, placed by comparison (2^20, 2^21),
    the sparse regime of the 2^28 workload (2^23), and comparison only (2^25).
    float64 keys 2^20 + j 2^-32 are consecutive doubles, so their phi values
    repeat at the same rates."""
    n, p = 1 << 20, 16
    rng = np.random.default_rng(span_log2)
    j = rng.integers(0, 1 << span_log2, n)
    keys = j.astype(np.int32) if dt == "int32" else 2.0**20 + j * 2.0**-32
    ref = ref_sort(keys, p, 0, 0, oracle.RANDOM, 5)
    gpu = run_gpu(keys, p, 0, 0, oracle.RANDOM, 5)
    assert gpu.plan.bucket_cluster == 8
    assert_same(gpu, ref)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_pairs_one_value_sub_buckets_are_copied(mode):
    """Payload sort where the two interior buckets lie between equal splitters
    (one key value holds 90% of the keys): they are copied as they stand, each
    larger than a cluster's shared memory, while the end buckets mix values and
    take the cluster or out-of-core sort.  Payloads of equal keys stay in input
    order (Sec. 5.1.1)."""
    n, p = 400_000, 4
    rng = np.random.default_rng(12)
    u = rng.random(n)
    keys = np.full(n, 5, np.int32)
    keys[u < 0.05] = -3
    keys[u > 0.95] = rng.integers(10, 2**31 - 1, int((u > 0.95).sum()), dtype=np.int64).astype(np.int32)
    vals = np.arange(n, dtype=np.uint32)
    if mode == oracle.REGULAR:
        ref = ref_sort(keys, p, 16, 8, mode, 0, vals)  # blocks of 50,000 keys
        gpu = run_gpu(keys, p, 16, 8, mode, 0, vals, refine=1)
    else:
        ref = ref_sort(keys, p, 0, 0, mode, 4, vals)
        gpu = run_gpu(keys, p, 0, 0, mode, 4, vals, refine=1)
    assert_same(gpu, ref)


@pytest.mark.parametrize("pad", [0, 5], ids=["no_pads", "pads"])
def test_regular_keys_with_the_pads_phi(pad):
    """Regular sampling on keys that include INT32_MAX, whose phi (all ones)
    is the pads' phi.  With pads (n below R*M) a pad's tag exceeds every key's,
    so the sample sort must order the tag bytes too; without pads the runs of
    the sample, in block order, are sorted by phi alone.  Few distinct values:
    the blocks also take the few-values sampler."""
    R = p = 16
    s, m = 64, 4096
    n = R * m - pad
    rng = np.random.default_rng(21)
    keys = rng.choice(np.array([2**31 - 1, 7, -100, 0], np.int32), n, p=[0.4, 0.2, 0.2, 0.2])
    ref = ref_sort(keys, p, s, R, oracle.REGULAR, 0)
    gpu = run_gpu(keys, p, s, R, oracle.REGULAR, 0)
    assert gpu.plan.R * gpu.plan.M - n == pad
    assert_same(gpu, ref)


def test_regular_blocks_at_the_few_values_limit():
    """Blocks of 257 distinct values (one more than the few-values sampler's
    table takes) go on to the stable block sort; blocks of 256 stay with the
    few-values sampler.  Half of every block is one value, so the block sort's
    probe sends every block to the few-values sampler first."""
    R = p = 8
    m, s = 32768, 256
    rng = np.random.default_rng(31)
    others = ((np.arange(1, 400, dtype=np.int64) * 16777259) % 2**31 - 2**30).astype(np.int32)
    blocks = []
    for k in range(R):
        d = 257 if k < R // 2 else 256
        b = np.zeros(m, np.int32)
        rest = np.concatenate([others[: d - 1], rng.choice(others[: d - 1], m // 2 - (d - 1))])
        b[m // 2:] = rest
        blocks.append(rng.permutation(b))
    keys = np.concatenate(blocks)
    assert all(len(np.unique(b)) == (257 if k < R // 2 else 256) for k, b in enumerate(blocks))
    ref = ref_sort(keys, p, s, R, oracle.REGULAR, 0)
    gpu = run_gpu(keys, p, s, R, oracle.REGULAR, 0)
    assert_same(gpu, ref)
