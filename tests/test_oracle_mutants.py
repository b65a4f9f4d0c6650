"""Plausible mistakes planted in a copy of the oracle must fail its pins.

Each mutant is a one-token change to a private copy of oracle/bsp_oracle.c,
compiled into a temporary directory; the committed oracle is never touched.
The pins used here are the same independent checks as tests/test_oracle.py:
the hand-worked Fig. 1 examples, numpy's sort, the direct count of Lemma 5.1's
proof and numpy's Philox stream.
"""
import ctypes
import glob
import json
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import bsp_inputs as gen
import oracle
from tests.test_oracle import GOLDEN, _as_keys, direct_counts, stable_ranks

SRC = os.path.join(os.path.dirname(oracle.__file__), "bsp_oracle.c")

MUTANTS = {
    "sample_at_segment_start": ("local[k][j * pl.x - 1]", "local[k][(j - 1) * pl.x]"),
    "splitter_rank_off_by_one": ("Y[i * pl.q - 1]", "Y[i * pl.q]"),
    "tag_order_reversed": ("if (a->tag != b->tag) return a->tag < b->tag ? -1 : 1;",
                           "if (a->tag != b->tag) return a->tag < b->tag ? 1 : -1;"),
    "splitter_to_lower_bucket": (": elem_less(&local[k][mid], &Sk[k][i - 1]);",
                                 ": !elem_less(&Sk[k][i - 1], &local[k][mid]);"),
    "classify_splitter_to_lower_bucket": (": elem_less(&local[k][j], &Sk[k][mid]);",
                                          ": !elem_less(&Sk[k][mid], &local[k][j]);"),
    "duplicates_off_keeps_tags": ("S->dup_off = prm->duplicates == OR_DUP_OFF;", "S->dup_off = 0;"),
    "int32_sign_ignored": ("case OR_I32: return u ^ 0x80000000u;", "case OR_I32: return u;"),
    "pads_counted_as_keys": ("if (local[k][t].pad) { if (pad_sizes)", "if (0) { if (pad_sizes)"),
    "random_stream_shifted": ("(unsigned __int128)oracle_draw(seed, j)",
                              "(unsigned __int128)oracle_draw(seed, j + 1)"),
    "float_negatives_unflipped": ("(~u & 0xffffffffu) : (u | 0x80000000u)",
                                  "(u & 0x7fffffffu) : (u | 0x80000000u)"),
    "merge_drops_tie_break": ("if (a->tag != b->tag) return a->tag < b->tag ? -1 : 1;\n    return 0;",
                              "return 0;"),
}


def _build(mutant_src, outdir):
    c = os.path.join(outdir, "m.c")
    so = os.path.join(outdir, "m.so")
    open(c, "w").write(mutant_src)
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", so, c])
    lib = ctypes.CDLL(so)
    P = ctypes.c_void_p
    lib.oracle_sort.argtypes = [ctypes.c_int, P, P, ctypes.c_int64, ctypes.POINTER(oracle.Params),
                                P, P, P, P, P, P, P, P]
    lib.oracle_sort.restype = ctypes.c_int
    lib.oracle_position.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64]
    lib.oracle_position.restype = ctypes.c_int64
    return lib


def _run(lib, keys, p, s, runs, mode, seed, vals, duplicates=oracle.DUP_TAGS, variant=oracle.DET_IRAN):
    n = keys.shape[0]
    pl = oracle.plan(n, p, s, runs, mode, seed)
    out = np.empty_like(keys)
    vout = np.empty(n, np.uint32)
    sizes = np.zeros(pl.p, np.int64)
    pads = np.zeros(pl.p, np.int64)
    smp = np.zeros(pl.sample_size, oracle.RECORD_DTYPE)
    spl = np.zeros(pl.p - 1, oracle.RECORD_DTYPE)
    bof = np.full(n, -1, np.int32)
    prm = oracle.make_params(p, s, runs, mode, seed, duplicates=duplicates, variant=variant)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
    rc = lib.oracle_sort(oracle.DTYPE_CODE[keys.dtype], ptr(keys), ptr(vals), n, ctypes.byref(prm),
                         ptr(out), ptr(vout), ptr(sizes), ptr(pads), ptr(smp), ptr(spl), ptr(bof), None)
    return rc, pl, out, vout, sizes, pads, smp, spl, bof


def _pins_pass(lib):
    """True when every pin below accepts the oracle as it is loaded."""
    # hand-worked Fig. 1 examples
    for path in sorted(glob.glob(os.path.join(GOLDEN, "*.json"))):
        g = json.load(open(path))
        keys = _as_keys(g["keys"], g["dtype"])
        rc, pl, out, vout, sizes, pads, smp, spl, bof = _run(
            lib, keys, g["p"], g["s"], g["runs"], oracle.REGULAR, 0, np.array(g["vals"], np.uint32))
        if rc or sizes.tolist() != g["bucket_sizes"] or pads.tolist() != g["pad_sizes"] \
                or bof.tolist() != g["bucket_of"] or vout.tolist() != g["sorted_vals"] \
                or [int(t) for t in smp["tag"]] != [t for _, t, _ in g["sample"]]:
            return False
    # numpy sort + direct count, both modes, several key types
    for keys in (gen.uniform(3000, 8, 1), gen.zipf(3000, seed=2),
                 gen.gmm(3000, seed=3).astype(np.float32), gen.zero_entropy(3000)):
        for mode in (oracle.REGULAR, oracle.RANDOM):
            rc, pl, out, vout, sizes, pads, smp, spl, bof = _run(
                lib, keys, 8, 0, 0, mode, 5, np.arange(keys.shape[0], dtype=np.uint32))
            if rc:
                return False
            order = np.argsort(keys, kind="stable")
            if out.tobytes() != keys[order].tobytes() or not np.array_equal(vout, order):
                return False
            b = direct_counts(keys, spl, pl)
            if not np.array_equal(sizes, np.diff(b)):
                return False
            if not np.array_equal(bof, np.searchsorted(b[1:-1], stable_ranks(keys), side="right")):
                return False
    # Sort_Ran_BSP (Fig. 2) against the direct count; without duplicate
    # handling, buckets by the splitters' key values alone
    keys = gen.zipf(3000, seed=4)
    vals = np.arange(keys.shape[0], dtype=np.uint32)
    rc, pl, out, vout, sizes, pads, smp, spl, bof = _run(lib, keys, 8, 0, 0, oracle.RANDOM, 5, vals,
                                                         variant=oracle.RAN)
    b = direct_counts(keys, spl, pl)
    if rc or not np.array_equal(bof, np.searchsorted(b[1:-1], stable_ranks(keys), side="right")):
        return False
    for mode in (oracle.REGULAR, oracle.RANDOM):
        rc, pl, out, vout, sizes, pads, smp, spl, bof = _run(lib, keys, 8, 0, 0, mode, 5, vals,
                                                             duplicates=oracle.DUP_OFF)
        real = np.array([keys[k * int(pl.m) + j] for k, j in
                         (divmod(int(r["tag"]), int(pl.M)) for r in spl if not r["pad"])], keys.dtype)
        if rc or not np.array_equal(bof, np.searchsorted(real, keys, side="right")):
            return False
    # numpy's Philox stream
    bg = np.random.Philox(key=np.array([5, 0], np.uint64), counter=np.array([2**64 - 1] * 4, np.uint64))
    want = [int(v) >> 44 for v in bg.random_raw(16)]
    if [lib.oracle_position(5, j, 2**20) for j in range(16)] != want:
        return False
    return True


def test_unmutated_copy_passes():
    with tempfile.TemporaryDirectory() as d:
        assert _pins_pass(_build(open(SRC).read(), d))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as d:
        assert not _pins_pass(_build(src.replace(old, new), d)), name
