"""CPU oracle of the BSP sample sort (Gerbessiotis & Siniolakis, Fig. 1 and Fig. 3).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and
by the cpu_baseline / reference legs of ``bench.py``.  The product path (the
package ``paper_1408_6729_gb300``) never imports it.

The arithmetic lives in ``bsp_oracle.c`` (plain C, compiled here with gcc on
first use); this module only marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsp_oracle.c")
_LIB = os.path.join(_HERE, "libbsp_oracle.so")
_STD_SRC = os.path.join(_HERE, "std_sorts.cpp")
_STD_LIB = os.path.join(_HERE, "libstd_sorts.so")
_lock = threading.Lock()
_lib = None

U32, I32, F32, F64 = 0, 1, 2, 3
REGULAR, RANDOM = 0, 1
DUP_TAGS, DUP_OFF = 0, 1      # duplicate handling of Sec. 5.1.1 on / off
DET_IRAN, RAN = 0, 1          # Sort_Det_BSP / Sort_IRan_BSP (Fig. 1, 3), or Sort_Ran_BSP (Fig. 2)

DTYPE_CODE = {np.dtype(np.uint32): U32, np.dtype(np.int32): I32,
              np.dtype(np.float32): F32, np.dtype(np.float64): F64}


class Params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("runs", ctypes.c_int32), ("s", ctypes.c_int64),
                ("sampling", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("duplicates", ctypes.c_int32), ("variant", ctypes.c_int32)]


class Plan(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in
                ("n", "p", "R", "s", "m", "M", "x", "q", "sample_size")] + \
               [("sampling", ctypes.c_int32)]


RECORD_DTYPE = np.dtype([("phi", np.uint64), ("tag", np.uint64),
                         ("pad", np.uint32), ("reserved", np.uint32)])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + __int128)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                                   "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
        if force or not os.path.exists(_STD_LIB) or os.path.getmtime(_STD_LIB) < os.path.getmtime(_STD_SRC):
            tmp = _STD_LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _STD_SRC])
            os.replace(tmp, _STD_LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_sort.argtypes = [ctypes.c_int, P, P, ctypes.c_int64, ctypes.POINTER(Params),
                                    P, P, P, P, P, P, P, P]
        lib.oracle_sort.restype = ctypes.c_int
        lib.oracle_plan_of.argtypes = [ctypes.c_int64, ctypes.POINTER(Params), ctypes.POINTER(Plan)]
        lib.oracle_plan_of.restype = ctypes.c_int
        lib.oracle_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_draw.restype = ctypes.c_uint64
        lib.oracle_position.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64]
        lib.oracle_position.restype = ctypes.c_int64
        _lib = lib
    return _lib


_std = None


def std_sort(keys: np.ndarray, stable: bool = False) -> np.ndarray:
    """The keys sorted by std::sort (or std::stable_sort), single-threaded: a
    CPU baseline timed beside the oracle, not part of it."""
    global _std
    if _std is None:
        build()
        lib = ctypes.CDLL(_STD_LIB)
        lib.baseline_std_sort.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
        lib.baseline_std_sort.restype = ctypes.c_int
        _std = lib
    out = np.array(keys, copy=True, order="C")
    rc = _std.baseline_std_sort(DTYPE_CODE[out.dtype], out.ctypes.data, out.shape[0], int(stable))
    if rc:
        raise ValueError("std_sort failed")
    return out


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def make_params(p, s=0, runs=0, sampling=REGULAR, seed=0, threads=0, duplicates=DUP_TAGS,
                variant=DET_IRAN) -> Params:
    return Params(p=int(p), runs=int(runs), s=int(s), sampling=int(sampling), threads=int(threads),
                  seed=int(seed) & (2**64 - 1), duplicates=int(duplicates), variant=int(variant))


def plan(n, p, s=0, runs=0, sampling=REGULAR, seed=0) -> Plan | None:
    """Resolved parameters (defaults of Sec. 6.1); None when they are invalid."""
    pl = Plan()
    prm = make_params(p, s, runs, sampling, seed)
    rc = _load().oracle_plan_of(int(n), ctypes.byref(prm), ctypes.byref(pl))
    return None if rc else pl


def draw(seed: int, j: int) -> int:
    """Draw j of the random-sample stream: Philox4x64-10, key (seed,0), counter (j//4,0,0,0)."""
    return int(_load().oracle_draw(seed & (2**64 - 1), j))


def position(seed: int, j: int, n: int) -> int:
    return int(_load().oracle_position(seed & (2**64 - 1), j, n))


@dataclass
class Result:
    keys: np.ndarray
    vals: np.ndarray | None
    bucket_sizes: np.ndarray
    pad_sizes: np.ndarray
    sample: np.ndarray | None
    splitters: np.ndarray
    bucket_of: np.ndarray | None
    plan: Plan
    partition: np.ndarray | None = None


def sort(keys: np.ndarray, p: int, s: int = 0, runs: int = 0, sampling: int = REGULAR,
         seed: int = 0, vals: np.ndarray | None = None, want_sample: bool = True,
         want_bucket_of: bool = False, threads: int = 0, duplicates: int = DUP_TAGS,
         variant: int = DET_IRAN, want_partition: bool = False) -> Result:
    """Run the BSP simulation; raises ValueError on invalid parameters.

    threads > 1 runs the virtual processors of each superstep on that many host
    threads (the result is the same).  duplicates = DUP_OFF drops the tags from
    the partition's comparisons; variant = RAN runs Sort_Ran_BSP (Fig. 2).
    want_partition returns c[k][i] (SS6) as an R x (p+1) array."""
    keys = np.ascontiguousarray(keys)
    code = DTYPE_CODE[keys.dtype]
    n = keys.shape[0]
    pl = plan(n, p, s, runs, sampling, seed)
    if pl is None:
        raise ValueError("invalid parameters")
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        assert vals.shape[0] == n
    keys_out = np.empty_like(keys)
    vals_out = np.empty(n, np.uint32) if vals is not None else None
    sizes = np.zeros(pl.p, np.int64)
    pads = np.zeros(pl.p, np.int64)
    sample = np.zeros(pl.sample_size, RECORD_DTYPE) if (want_sample and n > 0) else None
    spl = np.zeros(max(pl.p - 1, 0), RECORD_DTYPE)
    bof = np.full(n, -1, np.int32) if want_bucket_of else None
    part = np.zeros((pl.R, pl.p + 1), np.int64) if (want_partition and n > 0) else None
    prm = make_params(p, s, runs, sampling, seed, threads, duplicates, variant)
    rc = _load().oracle_sort(code, _ptr(keys), _ptr(vals), n, ctypes.byref(prm), _ptr(keys_out),
                             _ptr(vals_out), _ptr(sizes), _ptr(pads), _ptr(sample), _ptr(spl),
                             _ptr(bof), _ptr(part))
    if rc:
        raise ValueError(f"oracle_sort failed with status {rc}")
    return Result(keys_out, vals_out, sizes, pads, sample, spl, bof, pl, part)
