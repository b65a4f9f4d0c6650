"""The C-ABI library builds, loads and exports every entry point of
include/bspsort.h; host-side argument checks and parameter resolution agree
with the paper's defaults (Sec. 6.1) and with the oracle.  No GPU needed."""
import os
import re

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bspsort.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1408_6729_gb300 import build
    build.build()
    import paper_1408_6729_gb300 as bsps
    return bsps


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bsps_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    import ctypes
    names = declared_functions()
    assert len(names) >= 7
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in names:
        assert hasattr(so, name), name
    assert set(lib.EXPORTS) <= set(names)


def test_plan_defaults_follow_the_paper_and_the_oracle(lib):
    for n, p, mode, s, runs in [(2**20, 64, 0, 8, 64), (2**20, 64, 0, 0, 0), (2**26, 1024, 1, 0, 0),
                                (2**28 - 1, 4096, 1, 0, 0), (1000, 7, 0, 0, 0), (12345, 16, 1, 3, 5),
                                (2**28, 4096, 0, 4096, 4096)]:
        prm = lib.make_params(p, s=s, runs=runs, sampling=mode)
        pl = lib.bsps_get_plan(n, lib.BSPS_I32, prm)
        ref = oracle.plan(n, p, s, runs, mode)
        for f in ("n", "p", "R", "s", "m", "M", "x", "q", "sample_size"):
            assert getattr(pl, f) == getattr(ref, f), (f, n, p, mode)
        assert pl.vbuckets == p * pl.refine
        assert pl.workspace_bytes == lib.bsps_workspace_size(n, lib.BSPS_I32, prm)


def test_host_side_argument_errors(lib):
    bad = [lib.make_params(0), lib.make_params(4, s=-1), lib.make_params(3, s=2, runs=2),
           lib.make_params(4, sampling=7), lib.make_params(4, refine=3)]
    for prm in bad:
        with pytest.raises(ValueError):
            lib.bsps_get_plan(100, lib.BSPS_I32, prm)
    with pytest.raises(ValueError):
        lib.bsps_get_plan(100, 9, lib.make_params(4))
    with pytest.raises(ValueError):
        lib.bsps_get_plan(2**30, lib.BSPS_I32, lib.make_params(4))
    # sort entry points reject before touching the device
    prm = lib.make_params(0)
    rc = lib.load().bsps_sort_keys(None, None, 10, lib.BSPS_I32, prm, None, None, 0, None)
    assert rc == lib.BSPS_ERR_INVALID_ARG
    prm = lib.make_params(4)
    rc = lib.load().bsps_sort_keys(None, None, 10, lib.BSPS_I32, prm, None, None, 0, None)
    assert rc == lib.BSPS_ERR_INVALID_ARG          # null keys
    rc = lib.load().bsps_sort_keys(8, 16, 10, lib.BSPS_I32, prm, None, None, 0, None)
    assert rc == lib.BSPS_ERR_WORKSPACE_TOO_SMALL  # no workspace
    rc = lib.load().bsps_sort_keys(8, 8, 10, lib.BSPS_I32, prm, None, 256, 1 << 40, None)
    assert rc == lib.BSPS_ERR_INVALID_ARG          # in place
    assert lib.bsps_strerror(lib.BSPS_ERR_BUCKET_OVERFLOW)


def test_merge_final_step_and_duplicate_switch_arguments(lib):
    """The merge final step ends Sort_Det_BSP (Fig. 1 step 12): regular
    sampling, 4-byte keys, tree classification, no sub-buckets, at most 8192
    blocks, and a bucket bound of Lemma 5.1 one cluster can merge."""
    M = lib.BSPS_FINAL_MERGE
    for kw in (dict(sampling=lib.BSPS_RANDOM), dict(refine=2), dict(classify=lib.BSPS_LEARNED),
               dict(runs=16384)):
        with pytest.raises(ValueError, match="invalid"):
            lib.bsps_get_plan(1 << 20, lib.BSPS_I32, lib.make_params(64, final_step=M, **kw))
    with pytest.raises(ValueError, match="invalid"):
        lib.bsps_get_plan(1 << 20, lib.BSPS_F64, lib.make_params(64, final_step=M))
    for kw in (dict(final_step=2), dict(duplicates=2)):
        with pytest.raises(ValueError, match="invalid"):
            lib.bsps_get_plan(1 << 20, lib.BSPS_I32, lib.make_params(64, **kw))
    # config 1 with s = 8: the bound (145,347 keys) exceeds a cluster's 126,976
    with pytest.raises(ValueError, match="too large"):
        lib.bsps_get_plan(1 << 20, lib.BSPS_U32, lib.make_params(64, s=8, final_step=M))
    # the regular headline shape: eight CTAs per bucket, no bucket regions
    pl = lib.bsps_get_plan(1 << 28, lib.BSPS_I32, lib.make_params(4096, s=4096, final_step=M))
    assert pl.bucket_cluster == 8 and pl.refine == 1 and pl.capacity == 126976
    plain = lib.bsps_get_plan(1 << 28, lib.BSPS_I32, lib.make_params(4096, s=4096))
    assert pl.workspace_bytes < plain.workspace_bytes
    dup = lib.bsps_get_plan(1 << 20, lib.BSPS_I32, lib.make_params(64, duplicates=lib.BSPS_DUP_OFF))
    assert dup.workspace_bytes == lib.bsps_get_plan(1 << 20, lib.BSPS_I32, lib.make_params(64)).workspace_bytes
