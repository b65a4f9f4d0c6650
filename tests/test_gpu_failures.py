"""Failure paths on the GPU that leave the device usable.

* An expired bounded wait.  With payloads, the routing kernel's prefix over
  earlier tiles (the p parallel prefix sums of Fig. 1 step 9, whose result
  depends on every earlier processor, Sec. 5.1) waits on flags that earlier
  tiles publish.  A test hook stops one tile from publishing and bounds a
  wait to a few thousand polls: the later tiles' waits run out, the call
  reports BSPS_ERR_DEVICE_TIMEOUT through bsps_read_stats, nothing hangs or
  traps, and the next call on the same context sorts correctly.
* A batched call issued on a stream that is being captured returns
  BSPS_ERR_CAPTURE and queues nothing; the same call outside the capture
  sorts every instance.
"""
import numpy as np
import pytest

import bsp_inputs as gen
from tests.gpu_util import lib, to_dev

pytestmark = pytest.mark.gpu


def _pairs_call(keys, p, ws, kin, vin, kout, vout, sizes, **hooks):
    bsps = lib()
    prm = bsps.make_params(p, sampling=bsps.BSPS_RANDOM, seed=3, refine=1)
    rc = bsps.bsps_sort_debug(kin, vin, kout, vout, keys.shape[0], bsps.BSPS_I32, prm, sizes, ws, **hooks)
    assert rc == 0, bsps.bsps_strerror(rc)
    return bsps.bsps_read_stats(ws)


def test_expired_lookback_wait_is_reported_and_the_next_call_sorts():
    import torch
    bsps = lib()
    n, p = 300_000, 16  # five routing tiles of 65,536 keys
    keys = gen.uniform(n, p, 4)
    vals = np.arange(n, dtype=np.uint32)
    prm = bsps.make_params(p, sampling=bsps.BSPS_RANDOM, seed=3, refine=1)
    pl = bsps.bsps_get_plan(n, bsps.BSPS_I32, prm, True)
    assert pl.route_tiles >= 3
    ws = torch.empty(pl.workspace_bytes, dtype=torch.uint8, device="cuda:0")
    kin, vin = to_dev(keys), to_dev(vals)
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    sizes = torch.empty(p, dtype=torch.int64, device="cuda:0")
    # tile 1 never publishes: tiles 2.. wait on it for 2000 polls each
    st = _pairs_call(keys, p, ws, kin, vin, kout, vout, sizes, stall_tile=2, wait_polls=2000)
    assert st.status == bsps.BSPS_ERR_DEVICE_TIMEOUT, bsps.bsps_strerror(st.status)
    assert st.timeouts >= 1
    # the context is intact: the same call without the hooks is exact
    st = _pairs_call(keys, p, ws, kin, vin, kout, vout, sizes)
    assert st.status == 0 and st.timeouts == 0
    order = np.argsort(keys, kind="stable")
    assert kout.cpu().numpy().tobytes() == keys[order].tobytes()
    assert np.array_equal(vout.cpu().numpy().view(np.uint32), order.astype(np.uint32))


def test_batched_call_refuses_a_callers_capture():
    import torch
    bsps = lib()
    sizes = [300, 5000, 70_000, 0, 1]
    keys = np.concatenate([gen.uniform(n, 1, 9 + i) for i, n in enumerate(sizes)]).astype(np.int32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    prm = bsps.make_params(1, sampling=bsps.BSPS_RANDOM, seed=5)
    tune = bsps.bsps_tune_default()
    base = bsps.bsps_batch_bucket_base(off, tune)
    ws = torch.empty(bsps.bsps_batch_workspace_size(off, bsps.BSPS_I32, prm, tune), dtype=torch.uint8,
                     device="cuda:0")
    kin = to_dev(keys)
    kout = torch.full_like(kin, 7)
    bsz = torch.full((max(1, base[-1]),), -1, dtype=torch.int64, device="cuda:0")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=side):
        rc = bsps.bsps_sort_batched(kin, kout, off, bsps.BSPS_I32, prm, tune, bsz, ws)
    assert rc == bsps.BSPS_ERR_CAPTURE
    assert bool((kout == 7).all().item())  # nothing was queued
    rc = bsps.bsps_sort_batched(kin, kout, off, bsps.BSPS_I32, prm, tune, bsz, ws)
    assert rc == 0, bsps.bsps_strerror(rc)
    assert bsps.bsps_read_stats(ws).status == 0
    out = kout.cpu().numpy()
    for i in range(len(sizes)):
        a, b = off[i], off[i + 1]
        assert out[a:b].tobytes() == np.sort(keys[a:b]).tobytes()
