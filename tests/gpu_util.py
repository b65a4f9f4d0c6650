"""Helpers of the GPU tests: run the library through its C ABI on cuda:0 and
bring every output back as numpy, next to the oracle's."""
import numpy as np

import oracle

TORCH_OF = {np.dtype(np.int32): "int32", np.dtype(np.uint32): "int32",
            np.dtype(np.float32): "float32", np.dtype(np.float64): "float64"}


def lib():
    import paper_1408_6729_gb300 as bsps
    from paper_1408_6729_gb300 import build
    build.build()
    return bsps


def code_of(keys):
    bsps = lib()
    return {np.dtype(np.uint32): bsps.BSPS_U32, np.dtype(np.int32): bsps.BSPS_I32,
            np.dtype(np.float32): bsps.BSPS_F32, np.dtype(np.float64): bsps.BSPS_F64}[keys.dtype]


def to_dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to("cuda:0")


class GpuResult:
    pass


def run_gpu(keys, p, s=0, runs=0, mode=0, seed=0, vals=None, refine=0, capacity_pct=0,
            debug=True, bucket_of=None, classify=0, final_step=0, duplicates=0, expect_status=0):
    """Sort with the library; returns keys, vals, sizes, sample, splitters, bucket_of, pads, stats
    (and, for the merge final step, the partition as an R x (p+1) array)."""
    import torch
    bsps = lib()
    n = keys.shape[0]
    code = code_of(keys)
    prm = bsps.make_params(p, s=s, runs=runs, sampling=mode, seed=seed, refine=refine,
                           capacity_pct=capacity_pct, classify=classify, final_step=final_step,
                           duplicates=duplicates)
    pl = bsps.bsps_get_plan(n, code, prm, vals is not None)
    ws = torch.empty(max(pl.workspace_bytes, 1), dtype=torch.uint8, device="cuda:0")
    kin = to_dev(keys)
    kout = torch.empty_like(kin)
    vin = to_dev(vals.astype(np.uint32)) if vals is not None else None
    vout = torch.empty_like(vin) if vals is not None else None
    sizes = torch.full((p,), -1, dtype=torch.int64, device="cuda:0")
    rec_bytes = 24
    want_bo = (n <= (1 << 22)) if bucket_of is None else bucket_of
    sample = torch.empty((max(pl.sample_size, 1) * rec_bytes,), dtype=torch.uint8, device="cuda:0") if debug else None
    spl = torch.empty((max(p - 1, 1) * rec_bytes,), dtype=torch.uint8, device="cuda:0") if debug else None
    bo = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda:0") if (debug and want_bo) else None
    pads = torch.full((p,), -1, dtype=torch.int64, device="cuda:0") if debug else None
    mlp_params = torch.zeros(bsps.MLP_PARAMS, dtype=torch.float32, device="cuda:0") if classify else None
    mlp_loss = torch.zeros(2, dtype=torch.float32, device="cuda:0") if classify else None
    # the partition of the sorted blocks (Fig. 1 step 9), when the call keeps them
    keeps = final_step or (mode == oracle.REGULAR and keys.dtype.itemsize == 4 and not classify and pl.R <= 16384)
    part = torch.full(((p + 1) * pl.R,), -1, dtype=torch.int32, device="cuda:0") \
        if (debug and keeps and n > 0) else None
    rc = bsps.bsps_sort_debug(kin, vin, kout, vout, n, code, prm, sizes, ws, sample=sample,
                              splitters=spl, bucket_of=bo, pad_sizes=pads, mlp_params=mlp_params,
                              mlp_loss=mlp_loss, partition=part)
    assert rc == 0, bsps.bsps_strerror(rc)
    st = bsps.bsps_read_stats(ws)
    assert st.status == expect_status, (st.status, bsps.bsps_strerror(st.status))
    r = GpuResult()
    r.plan = pl
    r.stats = st
    r.keys = kout.cpu().numpy().view(keys.dtype)
    r.vals = vout.cpu().numpy().view(np.uint32) if vals is not None else None
    r.bucket_sizes = sizes.cpu().numpy()
    r.sample = sample.cpu().numpy()[: pl.sample_size * rec_bytes].view(oracle.RECORD_DTYPE) if debug else None
    r.splitters = spl.cpu().numpy()[: (p - 1) * rec_bytes].view(oracle.RECORD_DTYPE) if debug else None
    r.bucket_of = bo.cpu().numpy()[:n] if bo is not None else None
    r.pad_sizes = pads.cpu().numpy() if debug else None
    r.mlp_params = mlp_params.cpu().numpy() if classify else None
    r.mlp_loss = mlp_loss.cpu().numpy() if classify else None
    r.partition = part.cpu().numpy().view(np.uint32).reshape(p + 1, pl.R).T.astype(np.int64) \
        if part is not None else None
    return r


def assert_same(gpu, ref, check_sample=True):
    assert gpu.stats.status == 0, gpu.stats.status
    assert gpu.keys.tobytes() == ref.keys.tobytes(), "sorted keys differ"
    if ref.vals is not None:
        assert np.array_equal(gpu.vals, ref.vals), "payloads differ"
    assert np.array_equal(gpu.bucket_sizes, ref.bucket_sizes), "bucket sizes differ"
    if gpu.splitters is not None:
        assert gpu.splitters.tobytes() == ref.splitters.tobytes(), "splitters differ"
    if check_sample and gpu.sample is not None and ref.sample is not None:
        assert gpu.sample.tobytes() == ref.sample.tobytes(), "samples differ"
    if gpu.bucket_of is not None and ref.bucket_of is not None:
        assert np.array_equal(gpu.bucket_of, ref.bucket_of), "per-key buckets differ"
    if gpu.pad_sizes is not None and ref.plan.sampling == oracle.REGULAR:
        assert np.array_equal(gpu.pad_sizes, ref.pad_sizes), "pad counts differ"
    if getattr(gpu, "partition", None) is not None and getattr(ref, "partition", None) is not None:
        # the oracle's c[k][i] counts pads too; the GPU's counts the block's keys
        pl = ref.plan
        n = gpu.keys.shape[0]
        real = np.array([max(0, min(int(pl.m), n - k * int(pl.m))) for k in range(int(pl.R))], np.int64)
        assert np.array_equal(gpu.partition, np.minimum(ref.partition, real[:, None])), "partition differs"
