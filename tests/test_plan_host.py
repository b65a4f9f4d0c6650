"""Host logic of bsps_get_plan (no GPU needed): the paper's default
oversampling it resolves (Sec. 6.1) and the argument and size limits the
header declares, each at the value just inside and just past the limit."""
import ctypes

import pytest


def _lib():
    import paper_1408_6729_gb300 as bsps
    from paper_1408_6729_gb300 import build
    build.build()
    return bsps


def _plan(bsps, n, prm, dtype=None):
    out = bsps.bsps_plan()
    rc = bsps.load().bsps_get_plan(int(n), int(bsps.BSPS_I32 if dtype is None else dtype), ctypes.byref(prm), 0,
                                   ctypes.byref(out))
    return rc, out


def test_default_oversampling():
    """Random: s = 2*ceil(lg n)^2 and s*p - 1 sample keys; regular: s = r*p
    with r = ceil(lg lg n), R = p runs of ceil(n/R) keys padded to M = s*ceil(m/s)."""
    bsps = _lib()
    rc, pl = _plan(bsps, 1 << 28, bsps.make_params(4096, sampling=bsps.BSPS_RANDOM))
    assert rc == 0 and pl.s == 2 * 28 * 28 and pl.sample_size == pl.s * 4096 - 1
    rc, pl = _plan(bsps, 1 << 20, bsps.make_params(64, sampling=bsps.BSPS_REGULAR))
    assert rc == 0 and pl.R == 64 and pl.s == 5 * 64  # lg lg 2^20 = lg 20 = 4.3
    assert pl.m == (1 << 20) // 64 and pl.M == pl.s * -(-pl.m // pl.s) and pl.sample_size == pl.R * pl.s


@pytest.mark.parametrize("kwargs", [dict(p=0), dict(p=8, refine=3), dict(p=3, s=4, runs=4)],
                         ids=["p0", "refine_not_pow2", "Rs_not_multiple_of_p"])
def test_invalid_arguments(kwargs):
    bsps = _lib()
    sampling = bsps.BSPS_REGULAR if "runs" in kwargs or kwargs["p"] == 0 else bsps.BSPS_RANDOM
    rc, _ = _plan(bsps, 1 << 20, bsps.make_params(sampling=sampling, **kwargs))
    assert rc == bsps.BSPS_ERR_INVALID_ARG


def test_key_count_limit():
    bsps = _lib()
    prm = bsps.make_params(64, sampling=bsps.BSPS_RANDOM)
    assert _plan(bsps, (1 << 30) - 1, prm)[0] == 0
    assert _plan(bsps, 1 << 30, prm)[0] == bsps.BSPS_ERR_TOO_LARGE


@pytest.mark.parametrize("dt,block", [("I32", 81920), ("F64", 65536)])
def test_regular_block_limit(dt, block):
    """A regular-mode block must fit the block sort's largest cluster."""
    bsps = _lib()
    code = getattr(bsps, "BSPS_" + dt)
    prm = bsps.make_params(8, s=64, runs=8, sampling=bsps.BSPS_REGULAR)
    rc, pl = _plan(bsps, 8 * block, prm, code)
    assert rc == 0 and pl.m == block
    assert _plan(bsps, 8 * (block + 1), prm, code)[0] == bsps.BSPS_ERR_TOO_LARGE


def test_sub_bucket_limits():
    """p and p*refine stay below 2^16 (16-bit sub-bucket ids) and within what
    the routing kernel's shared memory holds (p = 65535 does not fit); an
    explicit refine whose routing shared memory does not fit is refused,
    while refine = 0 picks one that fits."""
    bsps = _lib()
    assert _plan(bsps, 1 << 24, bsps.make_params(8192, sampling=bsps.BSPS_RANDOM))[0] == 0
    assert _plan(bsps, 1 << 24, bsps.make_params(65535, sampling=bsps.BSPS_RANDOM))[0] == bsps.BSPS_ERR_TOO_LARGE
    assert _plan(bsps, 1 << 24, bsps.make_params(65536, sampling=bsps.BSPS_RANDOM))[0] == bsps.BSPS_ERR_TOO_LARGE
    assert _plan(bsps, 1 << 24, bsps.make_params(4096, sampling=bsps.BSPS_RANDOM, refine=32))[0] == \
        bsps.BSPS_ERR_TOO_LARGE
    assert _plan(bsps, 1 << 28, bsps.make_params(4096, sampling=bsps.BSPS_RANDOM, refine=4))[0] == \
        bsps.BSPS_ERR_TOO_LARGE
    rc, pl = _plan(bsps, 1 << 28, bsps.make_params(4096, sampling=bsps.BSPS_RANDOM))
    assert rc == 0 and pl.vbuckets == 4096 * pl.refine


def _regular_inputs(n, p):
    import numpy as np
    import bsp_inputs as gen
    yield "uniform", gen.uniform(n, p, 1)
    yield "zero_entropy", gen.zero_entropy(n)
    yield "staggered", gen.staggered(n, p, 2)
    yield "bucket_sorted", gen.bucket_sorted(n, p, 3)
    yield "det_duplicates", gen.det_duplicates(n, p, 4)
    yield "2-G", gen.g_group(n, p, 5)
    yield "zipf", gen.zipf(n, seed=6)
    yield "ascending", np.arange(n, dtype=np.int32)
    yield "descending", np.arange(n, dtype=np.int32)[::-1].copy()
    rng = np.random.default_rng(7)
    for t in range(20):  # few values: many keys tie with the splitters
        yield f"values{t}", rng.integers(0, 2 + t % 5, n).astype(np.int32)


@pytest.mark.parametrize("n,p,s,runs", [(4096, 8, 8, 8), (10_007, 16, 32, 16), (65_536, 64, 64, 128),
                                        (30_000, 32, 16, 64), (5_000, 4, 200, 4)])
def test_regular_capacity_holds_every_bucket_the_oracle_forms(n, p, s, runs):
    """Regular oversampling sizes every bucket region by Lemma 5.1's bound, so
    no input may give a bucket more records (keys and pads) than the plan's
    capacity: checked against the buckets the oracle forms on the paper's
    distributions, sorted and reversed input, and inputs of two to six values
    whose keys tie with the splitters (the tie-break's worst case)."""
    import numpy as np
    import oracle
    bsps = _lib()
    rc, pl = _plan(bsps, n, bsps.make_params(p, s=s, runs=runs, sampling=bsps.BSPS_REGULAR, refine=1))
    assert rc == 0 and pl.refine == 1
    worst = 0
    for name, keys in _regular_inputs(n, runs):
        ref = oracle.sort(keys, p, s, runs, oracle.REGULAR, 0, want_sample=False)
        assert int(ref.bucket_sizes.sum()) == n, name
        worst = max(worst, int((ref.bucket_sizes + ref.pad_sizes).max()))
    assert worst <= pl.capacity
    # and the capacity is no looser than the lemma's bound (+1, rounded to 16 bytes)
    x, q, R = pl.x, pl.q, pl.R
    assert pl.capacity <= (((q + R - 1) * x - R + 2) + 3) // 4 * 4
