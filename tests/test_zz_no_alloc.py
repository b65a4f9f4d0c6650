"""bsps_sort_keys_noalloc: the entry point for callers that cannot allocate
device memory (their memory belongs to another runtime that gives them no
allocator, or they must never call cudaMalloc on a latency-critical path).
It sorts with the library's static device scratch instead of a caller
workspace; its results must equal those of bsps_sort_keys exactly (integer
results: bit-exact, the tolerance of every sort test here), on two calls in a
row, since the second call finds the first call's leftovers in the scratch.

This file is collected last on purpose (test_zz_*), and it passes both alone
in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import bsp_inputs as gen
from tests.gpu_util import lib, to_dev

pytestmark = pytest.mark.gpu


def _both(keys, p, mode, seed):
    import torch
    bsps = lib()
    n = keys.shape[0]
    code = bsps.BSPS_I32 if keys.dtype == np.int32 else bsps.BSPS_F64
    prm = bsps.make_params(p, sampling=mode, seed=seed)
    kin = to_dev(keys)
    out_a, out_b = torch.empty_like(kin), torch.empty_like(kin)
    sizes_a = torch.full((p,), -1, dtype=torch.int64, device="cuda:0")
    sizes_b = torch.full((p,), -1, dtype=torch.int64, device="cuda:0")
    assert bsps.bsps_sort_keys_noalloc(kin, out_a, n, code, prm, sizes_a) == 0
    ws = torch.empty(bsps.bsps_workspace_size(n, code, prm), dtype=torch.uint8, device="cuda:0")
    assert bsps.bsps_sort_keys(kin, out_b, n, code, prm, sizes_b, ws) == 0
    torch.cuda.synchronize()
    return out_a.cpu().numpy(), out_b.cpu().numpy(), sizes_a.cpu().numpy(), sizes_b.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_twice():
    first = gen.uniform(1 << 21, 256, 5)
    second = gen.zipf(3_000_001, seed=6)
    for keys, p, mode, seed in [(first, 256, 1, 11), (second, 256, 0, 0)]:
        a, b, sa, sb = _both(keys, p, mode, seed)
        assert a.tobytes() == b.tobytes()
        assert np.array_equal(sa, sb)
        assert a.tobytes() == np.sort(keys).tobytes()


def test_noalloc_f64_and_rejects_too_large():
    import torch
    bsps = lib()
    keys = gen.gmm(500_000, seed=3)
    a, b, sa, sb = _both(keys, 64, 1, 2)
    assert a.tobytes() == b.tobytes() and np.array_equal(sa, sb)
    n = 1 << 25
    prm = bsps.make_params(4096, sampling=1)
    assert bsps.bsps_workspace_size(n, bsps.BSPS_I32, prm) > bsps.BSPS_NOALLOC_SCRATCH_BYTES
    kin = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    kout = torch.empty_like(kin)
    rc = bsps.bsps_sort_keys_noalloc(kin, kout, n, bsps.BSPS_I32, prm, None)
    assert rc == bsps.BSPS_ERR_TOO_LARGE


def test_noalloc_status_is_readable():
    """A bucket overflow happens on the device after the call has returned
    BSPS_OK; bsps_noalloc_read_stats reads it from the static scratch (a
    capacity of 60% of the mean bucket forces it; every write stays inside
    the regions).  The next call starts from a clear status."""
    import torch
    bsps = lib()
    n, p = 200_000, 16
    keys = gen.uniform(n, p, 2)
    kin = to_dev(keys)
    kout = torch.empty_like(kin)
    small = bsps.make_params(p, sampling=1, seed=3, capacity_pct=60)
    assert bsps.bsps_sort_keys_noalloc(kin, kout, n, bsps.BSPS_I32, small, None) == 0
    st = bsps.bsps_noalloc_read_stats()
    assert st.status == bsps.BSPS_ERR_BUCKET_OVERFLOW and st.overflow == 1
    ok = bsps.make_params(p, sampling=1, seed=3)
    assert bsps.bsps_sort_keys_noalloc(kin, kout, n, bsps.BSPS_I32, ok, None) == 0
    st = bsps.bsps_noalloc_read_stats()
    assert st.status == 0 and st.overflow == 0
    assert kout.cpu().numpy().tobytes() == np.sort(keys).tobytes()
