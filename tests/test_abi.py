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
