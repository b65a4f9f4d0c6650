"""Host-side logic of the batched entry points (no GPU needed): the default
table, the flat bucket-size layout, the workspace size, and argument errors
that are rejected before any device work."""
import ctypes

import numpy as np
import pytest


def _lib():
    import paper_1408_6729_gb300 as bsps
    from paper_1408_6729_gb300 import build
    build.build()
    return bsps


def _class(n):
    c = 0
    while (1 << c) < n:
        c += 1
    return min(c, 31)


def test_default_table_is_valid():
    bsps = _lib()
    t = bsps.bsps_tune_default()
    assert all(1 <= t.p[c] <= 65535 for c in range(32))
    assert -1 <= t.small_max_log2 <= 14 and 1 <= t.lanes <= 16 and t.learned_min_log2 >= 0


def test_bucket_base_follows_size_classes():
    bsps = _lib()
    t = bsps.bsps_tune_default()
    for c in range(32):
        t.p[c] = c + 1
    sizes = [0, 1, 2, 3, 255, 256, 257, 16384, 16385, 1 << 20]
    off = np.concatenate([[0], np.cumsum(sizes)])
    base = bsps.bsps_batch_bucket_base(off, t)
    want = np.concatenate([[0], np.cumsum([_class(n) + 1 for n in sizes])])
    assert base == want.tolist()


def test_workspace_grows_with_pipeline_instances():
    bsps = _lib()
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM)
    t = bsps.bsps_tune_default()
    small = bsps.bsps_batch_workspace_size([0, 1000, 5000], bsps.BSPS_I32, prm, t)
    big = bsps.bsps_batch_workspace_size([0, 1000, 5000, 5000 + (1 << 20)], bsps.BSPS_I32, prm, t)
    assert 0 < small < big
    t.lanes = 2
    two = bsps.bsps_batch_workspace_size([0, 1000, 5000, 5000 + (1 << 20)], bsps.BSPS_I32, prm, t)
    assert two < big


@pytest.mark.parametrize("off", [[1, 5], [0, 5, 3], [0, -1]])
def test_bad_offsets_are_rejected(off):
    bsps = _lib()
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM)
    with pytest.raises(ValueError):
        bsps.bsps_batch_workspace_size(off, bsps.BSPS_I32, prm, bsps.bsps_tune_default())


def test_bad_table_is_rejected():
    bsps = _lib()
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM)
    t = bsps.bsps_tune_default()
    t.lanes = 0
    with pytest.raises(ValueError):
        bsps.bsps_batch_workspace_size([0, 10], bsps.BSPS_I32, prm, t)
    t = bsps.bsps_tune_default()
    t.p[3] = 0
    with pytest.raises(ValueError):
        bsps.bsps_batch_workspace_size([0, 10], bsps.BSPS_I32, prm, t)


def test_small_workspace_is_rejected_before_device_work():
    import torch
    bsps = _lib()
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM)
    t = bsps.bsps_tune_default()
    ws = torch.empty(16, dtype=torch.uint8)  # host memory: never touched
    rc = bsps.bsps_sort_batched(None, None, [0, 100], bsps.BSPS_I32, prm, t, None, ws, stream=0)
    assert rc == bsps.BSPS_ERR_WORKSPACE_TOO_SMALL
