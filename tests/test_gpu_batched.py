"""Batched sorting (bsps_sort_batched): every instance of a batch must come out
exactly as the single-instance call sorts it with that instance's parameters
(same sorted keys, same bucket sizes), and, for instances the oracle finishes
quickly, as the oracle's BSP simulation with those parameters.

Covers instances on the on-chip path and on the pipeline path in one batch,
empty and one-key instances, repeated calls (the recorded graph is relaunched
with new key values), other key types, and the autotuner's table."""
import numpy as np
import pytest

import bsp_inputs as gen
import oracle
from tests.gpu_util import code_of, lib, to_dev

pytestmark = pytest.mark.gpu


def _batch(sizes, seed, dtype=np.int32):
    parts = []
    for i, n in enumerate(sizes):
        if n == 0:
            parts.append(np.zeros(0, dtype))
        elif i % 2 == 0:
            parts.append(gen.uniform(n, 1, seed + i).astype(dtype))
        else:
            parts.append(gen.zipf(n, seed=seed + i).astype(dtype))
    keys = np.concatenate(parts) if parts else np.zeros(0, dtype)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return keys, off


def _run_batched(keys, off, prm, tune, reuse=None):
    import torch
    bsps = lib()
    code = code_of(keys)
    num = len(off) - 1
    base = bsps.bsps_batch_bucket_base(off, tune)
    if reuse is None:
        ws = torch.empty(max(1, bsps.bsps_batch_workspace_size(off, code, prm, tune)), dtype=torch.uint8,
                         device="cuda:0")
        kin = to_dev(keys)
        kout = torch.empty_like(kin)
        sizes = torch.full((max(1, base[num]),), -1, dtype=torch.int64, device="cuda:0")
    else:
        ws, kin, kout, sizes = reuse
        kin.copy_(to_dev(keys))
    rc = bsps.bsps_sort_batched(kin, kout, off, code, prm, tune, sizes, ws)
    assert rc == 0, bsps.bsps_strerror(rc)
    st = bsps.bsps_read_stats(ws)
    assert st.status == 0 and st.overflow == 0 and st.timeouts == 0
    out = kout.cpu().numpy().view(keys.dtype)
    return out, sizes.cpu().numpy(), base, (ws, kin, kout, sizes)


def _single(keys_i, prm_i):
    import torch
    bsps = lib()
    code = code_of(keys_i)
    n = keys_i.shape[0]
    ws = torch.empty(max(1, bsps.bsps_workspace_size(n, code, prm_i)), dtype=torch.uint8, device="cuda:0")
    kin = to_dev(keys_i) if n else torch.empty(0, dtype=torch.int32, device="cuda:0")
    kout = torch.empty_like(kin)
    sizes = torch.full((prm_i.p,), -1, dtype=torch.int64, device="cuda:0")
    assert bsps.bsps_sort_keys(kin, kout, n, code, prm_i, sizes, ws) == 0
    return kout.cpu().numpy().view(keys_i.dtype), sizes.cpu().numpy()


def _instance_params(prm, tune, i, n):
    bsps = lib()
    c = 0
    while (1 << c) < n:
        c += 1
    c = min(c, 31)
    q = bsps.make_params(tune.p[c], s=prm.s, runs=prm.runs, sampling=prm.sampling, classify=prm.classify,
                         seed=prm.seed + i, refine=prm.refine, capacity_pct=prm.capacity_pct)
    if tune.learned_min_log2 > 0 and c >= tune.learned_min_log2:
        q.classify = bsps.BSPS_LEARNED
    return q


def _check(keys, off, out, sizes, base, prm, tune, oracle_max=20000):
    for i in range(len(off) - 1):
        a, b = int(off[i]), int(off[i + 1])
        ki = keys[a:b]
        q = _instance_params(prm, tune, i, b - a)
        got_k, got_s = out[a:b], sizes[base[i]:base[i + 1]]
        assert np.array_equal(got_k, np.sort(ki)), f"instance {i} (n={b - a}) not sorted"
        ref_k, ref_s = _single(ki, q)
        assert np.array_equal(got_k.view(np.uint8), ref_k.view(np.uint8)), f"instance {i} keys differ"
        assert np.array_equal(got_s, ref_s), f"instance {i} bucket sizes differ from the single call"
        if b - a <= oracle_max:
            o = oracle.sort(ki, q.p, q.s, 0, q.sampling, q.seed, want_sample=False)
            assert np.array_equal(got_s, o.bucket_sizes), f"instance {i} bucket sizes differ from the oracle"


SIZES = [0, 1, 2, 7, 256, 300, 1000, 4096, 5000, 9000, 16384, 16385, 40000, 70000, 200000, 0, 3]


def test_batched_matches_single_and_oracle():
    bsps = lib()
    keys, off = _batch(SIZES, 11)
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM, seed=5)
    tune = bsps.bsps_tune_default()
    tune.p[9] = 4  # several buckets on the on-chip path too
    tune.p[13] = 16
    out, sizes, base, _ = _run_batched(keys, off, prm, tune)
    _check(keys, off, out, sizes, base, prm, tune)


def test_batched_graph_relaunch_sees_new_keys():
    bsps = lib()
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM, seed=9)
    tune = bsps.bsps_tune_default()
    keys, off = _batch(SIZES, 21)
    out, sizes, base, bufs = _run_batched(keys, off, prm, tune)
    _check(keys, off, out, sizes, base, prm, tune, oracle_max=0)
    keys2, off2 = _batch(SIZES, 31)
    assert np.array_equal(off, off2)
    out2, sizes2, base2, _ = _run_batched(keys2, off2, prm, tune, reuse=bufs)
    _check(keys2, off2, out2, sizes2, base2, prm, tune)


@pytest.mark.parametrize("dtype", [np.uint32, np.float32, np.float64])
def test_batched_key_types(dtype):
    bsps = lib()
    rng = np.random.default_rng(3)
    sizes = [500, 12000, 33000, 1]
    if dtype == np.float64:
        parts = [rng.normal(0, 1e3, n) for n in sizes]
    elif dtype == np.float32:
        parts = [rng.normal(0, 1e3, n).astype(np.float32) for n in sizes]
    else:
        parts = [rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32) for n in sizes]
    keys = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM, seed=2)
    tune = bsps.bsps_tune_default()
    out, sz, base, _ = _run_batched(keys, off, prm, tune)
    _check(keys, off, out, sz, base, prm, tune)


def test_batched_regular_sampling_takes_the_pipeline():
    bsps = lib()
    keys, off = _batch([3000, 70000, 20000], 41)
    prm = bsps.make_params(1, sampling=bsps.BSPS_REGULAR)
    tune = bsps.bsps_tune_default()
    for c in range(32):
        tune.p[c] = 4
    out, sizes, base, _ = _run_batched(keys, off, prm, tune)
    _check(keys, off, out, sizes, base, prm, tune)


def test_batched_empty_batch():
    import torch
    bsps = lib()
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM)
    tune = bsps.bsps_tune_default()
    ws = torch.empty(max(1, bsps.bsps_batch_workspace_size([0], bsps.BSPS_I32, prm, tune)), dtype=torch.uint8,
                     device="cuda:0")
    assert bsps.bsps_sort_batched(None, None, [0], bsps.BSPS_I32, prm, tune, None, ws) == 0


def test_autotuned_table_sorts_exactly():
    import torch
    bsps = lib()
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM, seed=4)
    tune = bsps.bsps_tune_default()
    need = bsps.bsps_autotune_workspace_size(bsps.BSPS_I32, prm, 16)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda:0")
    assert bsps.bsps_autotune_batched(bsps.BSPS_I32, prm, 16, tune, ws) == 0
    assert all(1 <= tune.p[c] <= 65535 for c in range(32))
    assert -1 <= tune.small_max_log2 <= 14
    keys, off = _batch([100, 3000, 9000, 16000, 50000], 51)
    out, sizes, base, _ = _run_batched(keys, off, prm, tune)
    _check(keys, off, out, sizes, base, prm, tune)


def test_batched_learned_instances_match_single_calls():
    bsps = lib()
    keys, off = _batch([3000, 300000, 140000], 61)
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM, seed=7)
    tune = bsps.bsps_tune_default()
    tune.learned_min_log2 = 18
    out, sizes, base, _ = _run_batched(keys, off, prm, tune)
    _check(keys, off, out, sizes, base, prm, tune, oracle_max=0)
