"""The merge final step (Fig. 1 steps 9-12, params.final_step = BSPS_FINAL_MERGE)
and the version without duplicate handling (params.duplicates = BSPS_DUP_OFF)
against the oracle, element by element: sorted keys, payloads, bucket sizes,
sample, splitters, per-key buckets, pad counts and -- for the merge -- every
block's partition c[k][i] (the oracle's SS6, restricted to the block's keys)."""
import numpy as np
import pytest

import bsp_inputs as gen
import oracle
from tests.gpu_util import assert_same, lib, run_gpu

pytestmark = pytest.mark.gpu

FINAL_MERGE, DUP_OFF = 1, 1


def _ref(keys, p, s, runs, mode, seed, vals, duplicates=0):
    return oracle.sort(keys, p, s, runs, mode, seed, vals=vals, want_bucket_of=keys.shape[0] <= (1 << 22),
                       want_partition=True, duplicates=duplicates)


def _check_partition(gpu, ref, n):
    pl = ref.plan
    R, m = int(pl.R), int(pl.m)
    real = np.array([max(0, min(m, n - k * m)) for k in range(R)], np.int64)
    want = np.minimum(ref.partition, real[:, None])
    assert np.array_equal(gpu.partition, want), "partition differs"


# (name, keys, p, s, runs): the bound of Lemma 5.1 picks clusters of 1, 2, 4 and 8 CTAs
MERGE_CASES = [
    ("u32_p16_cl1", lambda: gen.uniform_u32(1 << 16, seed=3), 16, 64, 16),
    ("i32_p64_s512_cl2", lambda: gen.uniform(1 << 20, 64, 1), 64, 512, 0),
    ("i32_p64_cl4", lambda: gen.uniform(1 << 21, 64, 2), 64, 128, 0),
    ("i32_p64_cl8", lambda: gen.uniform(1 << 22, 64, 3), 64, 128, 0),
    ("zipf_p256_R512", lambda: gen.zipf(1 << 21, seed=4), 256, 256, 512),
    ("f32_gmm_ragged", lambda: gen.gmm(1_000_003, seed=5).astype(np.float32), 128, 256, 0),
    ("zero_entropy", lambda: gen.zero_entropy(300_007), 32, 64, 0),
    ("staggered_p1024", lambda: gen.staggered(1 << 22, 1024, 6), 1024, 1024, 0),
]


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("name,make,p,s,runs", MERGE_CASES, ids=[c[0] for c in MERGE_CASES])
def test_merge_final_step_matches_oracle(name, make, p, s, runs, pairs):
    keys = make()
    n = keys.shape[0]
    vals = np.arange(n, dtype=np.uint32) if pairs else None
    ref = _ref(keys, p, s, runs, oracle.REGULAR, 0, vals)
    gpu = run_gpu(keys, p, s, runs, oracle.REGULAR, 0, vals, final_step=FINAL_MERGE)
    assert_same(gpu, ref)
    _check_partition(gpu, ref, n)


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 1000, 4097, 65535])
@pytest.mark.parametrize("dt", [np.uint32, np.int32, np.float32])
def test_merge_edge_sizes(n, dt):
    rng = np.random.default_rng(n)
    if dt == np.float32:
        keys = rng.normal(0, 100, n).astype(np.float32)
    else:
        keys = rng.integers(0, 1000, n).astype(dt)  # many repeats
    vals = np.arange(n, dtype=np.uint32)
    p, s = 16, 16
    ref = _ref(keys, p, s, 0, oracle.REGULAR, 0, vals)
    gpu = run_gpu(keys, p, s, 0, oracle.REGULAR, 0, vals, final_step=FINAL_MERGE)
    assert_same(gpu, ref)
    _check_partition(gpu, ref, n)


def test_merge_empty_input():
    bsps = lib()
    import torch
    prm = bsps.make_params(8, s=8, final_step=FINAL_MERGE)
    pl = bsps.bsps_get_plan(0, bsps.BSPS_I32, prm)
    ws = torch.empty(max(pl.workspace_bytes, 1), dtype=torch.uint8, device="cuda:0")
    sizes = torch.full((8,), -1, dtype=torch.int64, device="cuda:0")
    k = torch.empty(0, dtype=torch.int32, device="cuda:0")
    assert bsps.bsps_sort_keys(k, torch.empty_like(k), 0, bsps.BSPS_I32, prm, sizes, ws) == 0
    assert bsps.bsps_read_stats(ws).status == 0
    assert sizes.cpu().tolist() == [0] * 8


def test_merge_m0_regular_shape_2e24():
    """The headline's regular shape (p = R = s, 16 keys per sample segment) at
    2^24 keys: 1024 buckets of 16,384 keys merged from 1024 segments each."""
    keys = gen.uniform(1 << 24, 1024, 1)
    ref = _ref(keys, 1024, 1024, 0, oracle.REGULAR, 0, None)
    gpu = run_gpu(keys, 1024, 1024, 0, oracle.REGULAR, 0, None, final_step=FINAL_MERGE, bucket_of=False)
    assert_same(gpu, ref)
    _check_partition(gpu, ref, keys.shape[0])


# ------------------------------------------------------------ no duplicate handling

def _few_values(n, values, seed):
    return np.random.default_rng(seed).integers(0, values, n).astype(np.int32)


DUP_CASES = [
    ("uniform_random", lambda: gen.uniform(1 << 20, 64, 1), oracle.RANDOM, 64, 0, 0, 0),
    ("uniform_regular", lambda: gen.uniform(1 << 20, 64, 2), oracle.REGULAR, 64, 0, 0, 0),
    ("few_values_random", lambda: _few_values(1 << 20, 3000, 3), oracle.RANDOM, 8, 0, 0, 0),
    ("few_values_regular", lambda: _few_values(1 << 20, 3000, 4), oracle.REGULAR, 16, 64, 64, 0),
    ("zipf_random_p8", lambda: gen.zipf(1 << 20, seed=3), oracle.RANDOM, 8, 0, 0, 800),
    ("f64_random", lambda: gen.gmm(1 << 19, seed=5), oracle.RANDOM, 256, 16, 0, 0),
]


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("name,make,mode,p,s,runs,cap", DUP_CASES, ids=[c[0] for c in DUP_CASES])
def test_without_duplicate_handling_matches_oracle(name, make, mode, p, s, runs, cap, pairs):
    keys = make()
    vals = np.arange(keys.shape[0], dtype=np.uint32) if pairs else None
    ref = _ref(keys, p, s, runs, mode, 7, vals, duplicates=oracle.DUP_OFF)
    gpu = run_gpu(keys, p, s, runs, mode, 7, vals, capacity_pct=cap, duplicates=DUP_OFF)
    assert_same(gpu, ref)


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
def test_merge_without_duplicate_handling_matches_oracle(pairs):
    keys = _few_values(1 << 20, 3000, 9)
    vals = np.arange(keys.shape[0], dtype=np.uint32) if pairs else None
    ref = _ref(keys, 16, 64, 64, oracle.REGULAR, 0, vals, duplicates=oracle.DUP_OFF)
    gpu = run_gpu(keys, 16, 64, 64, oracle.REGULAR, 0, vals, final_step=FINAL_MERGE, duplicates=DUP_OFF)
    assert_same(gpu, ref)
    _check_partition(gpu, ref, keys.shape[0])


def test_without_duplicate_handling_equal_keys_overflow():
    """All keys equal and no tie-break: every key lands in the last bucket,
    past its region (Lemma 5.1's bound needs the tags); the call reports it."""
    keys = gen.zero_entropy(1 << 20)
    gpu = run_gpu(keys, 64, 0, 0, oracle.RANDOM, 1, debug=False, duplicates=DUP_OFF, expect_status=-4)
    assert gpu.stats.overflow == 1
