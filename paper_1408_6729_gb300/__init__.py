"""Python binding of libbspsort.so, the GB300 BSP sample sort (include/bspsort.h).

Every function here has the name of the C entry point it calls and only marshals
arguments: tensors become device pointers, the current torch stream becomes the
cudaStream_t.  Every step of the sort runs in the library's CUDA kernels; there is
no CPU path.  Importing fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbspsort.so")

BSPS_U32, BSPS_I32, BSPS_F32, BSPS_F64 = 0, 1, 2, 3
BSPS_REGULAR, BSPS_RANDOM = 0, 1
BSPS_TREE, BSPS_LEARNED = 0, 1
BSPS_FINAL_SORT, BSPS_FINAL_MERGE = 0, 1
BSPS_DUP_TAGS, BSPS_DUP_OFF = 0, 1
BSPS_OK = 0
BSPS_ERR_INVALID_ARG = -1
BSPS_ERR_WORKSPACE_TOO_SMALL = -2
BSPS_ERR_UNSUPPORTED_DTYPE = -3
BSPS_ERR_BUCKET_OVERFLOW = -4
BSPS_ERR_CUDA = -5
BSPS_ERR_DEVICE_TIMEOUT = -6
BSPS_ERR_TOO_LARGE = -7
BSPS_ERR_CAPTURE = -8

EXPORTS = ["bsps_get_plan", "bsps_workspace_size", "bsps_sort_keys", "bsps_sort_pairs",
           "bsps_sort_debug", "bsps_read_stats", "bsps_mlp_workspace_size", "bsps_mlp_loss_grad", "bsps_mlp_predict",
           "bsps_sort_keys_noalloc", "bsps_noalloc_read_stats", "bsps_tune_default", "bsps_batch_bucket_base",
           "bsps_batch_workspace_size", "bsps_sort_batched", "bsps_autotune_workspace_size",
           "bsps_autotune_batched", "bsps_strerror"]
BSPS_BATCH_CLASSES = 32
BSPS_BATCH_SMALL_MAX = 16384
BSPS_BATCH_SAMPLE_MAX = 8192
BSPS_NOALLOC_SCRATCH_BYTES = 64 << 20
MLP_PARAMS = 1153


class bsps_params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("runs", ctypes.c_int32), ("s", ctypes.c_int64),
                ("sampling", ctypes.c_int32), ("classify", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("refine", ctypes.c_int32), ("capacity_pct", ctypes.c_int32),
                ("final_step", ctypes.c_int32), ("duplicates", ctypes.c_int32)]


class bsps_record(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("pad", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class bsps_plan(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("n", "p", "R", "s", "m", "M", "x", "q", "sample_size")] + \
               [("sampling", ctypes.c_int32), ("dtype", ctypes.c_int32)] + \
               [(f, ctypes.c_int64) for f in ("refine", "vbuckets", "capacity")] + \
               [("run_cluster", ctypes.c_int32), ("bucket_cluster", ctypes.c_int32),
                ("route_tiles", ctypes.c_int64), ("workspace_bytes", ctypes.c_size_t)]


class bsps_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("overflow", ctypes.c_int32), ("timeouts", ctypes.c_int32),
                ("slow_buckets", ctypes.c_int32), ("max_bucket", ctypes.c_int64),
                ("max_vbucket", ctypes.c_int64), ("mispredicted", ctypes.c_int64),
                ("correction_steps", ctypes.c_int64)]


BSPS_PHASES = 6


class bsps_tune(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32 * 32), ("small_max_log2", ctypes.c_int32),
                ("learned_min_log2", ctypes.c_int32), ("lanes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class bsps_debug(ctypes.Structure):
    _fields_ = [("sample", ctypes.c_void_p), ("splitters", ctypes.c_void_p),
                ("bucket_of", ctypes.c_void_p), ("pad_sizes", ctypes.c_void_p),
                ("phase_events", ctypes.POINTER(ctypes.c_void_p)),
                ("launches", ctypes.POINTER(ctypes.c_int32)),
                ("mlp_params", ctypes.c_void_p), ("mlp_loss", ctypes.c_void_p),
                ("stall_tile", ctypes.c_int32), ("wait_polls", ctypes.c_uint32),
                ("partition", ctypes.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library; raises when it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built: run __graft_entry__.build() "
                          "or python -m paper_1408_6729_gb300.build")
    lib = ctypes.CDLL(path)
    P, I64, I32, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
    PP = ctypes.POINTER(bsps_params)
    lib.bsps_get_plan.argtypes = [I64, I32, PP, I32, ctypes.POINTER(bsps_plan)]
    lib.bsps_workspace_size.argtypes = [I64, I32, PP, I32, ctypes.POINTER(SZ)]
    lib.bsps_sort_keys.argtypes = [P, P, I64, I32, PP, P, P, SZ, P]
    lib.bsps_sort_pairs.argtypes = [P, P, P, P, I64, I32, PP, P, P, SZ, P]
    lib.bsps_sort_debug.argtypes = [P, P, P, P, I64, I32, PP, P, ctypes.POINTER(bsps_debug), P, SZ, P]
    lib.bsps_read_stats.argtypes = [P, ctypes.POINTER(bsps_stats), P]
    lib.bsps_mlp_workspace_size.argtypes = [I64, ctypes.POINTER(SZ)]
    lib.bsps_mlp_loss_grad.argtypes = [P, P, P, I64, P, P, P, SZ, P]
    lib.bsps_mlp_predict.argtypes = [P, P, I64, P, P, SZ, P]
    lib.bsps_sort_keys_noalloc.argtypes = [P, P, I64, I32, PP, P, P]
    lib.bsps_noalloc_read_stats.argtypes = [ctypes.POINTER(bsps_stats), P]
    PT, PI64 = ctypes.POINTER(bsps_tune), ctypes.POINTER(ctypes.c_int64)
    lib.bsps_tune_default.argtypes = [PT]
    lib.bsps_batch_bucket_base.argtypes = [PI64, I32, PT, PI64]
    lib.bsps_batch_workspace_size.argtypes = [PI64, I32, I32, PP, PT, ctypes.POINTER(SZ)]
    lib.bsps_sort_batched.argtypes = [P, P, PI64, I32, I32, PP, PT, P, P, SZ, P]
    lib.bsps_autotune_workspace_size.argtypes = [I32, PP, I32, ctypes.POINTER(SZ)]
    lib.bsps_autotune_batched.argtypes = [I32, PP, I32, PT, P, SZ, P]
    lib.bsps_strerror.argtypes = [ctypes.c_int]
    lib.bsps_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "bsps_strerror":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


# ----------------------------------------------------------------- marshalling

def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return ctypes.c_void_p(x.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _nbytes(t):
    return t.numel() * t.element_size()


def dtype_code(t) -> int:
    """BSPS dtype of a torch tensor (int32 -> I32, float32 -> F32, float64 -> F64, uint32 -> U32)."""
    import torch
    table = {torch.int32: BSPS_I32, torch.float32: BSPS_F32, torch.float64: BSPS_F64}
    if hasattr(torch, "uint32"):
        table[torch.uint32] = BSPS_U32
    return table[t.dtype]


def make_params(p, s=0, runs=0, sampling=BSPS_REGULAR, classify=BSPS_TREE, seed=0, refine=0,
                capacity_pct=0, final_step=BSPS_FINAL_SORT, duplicates=BSPS_DUP_TAGS) -> bsps_params:
    return bsps_params(int(p), int(runs), int(s), int(sampling), int(classify), int(seed) & (2**64 - 1),
                       int(refine), int(capacity_pct), int(final_step), int(duplicates))


# ----------------------------------------------------------------- entry points

def bsps_get_plan(n, dtype, params, with_payload=False) -> bsps_plan:
    out = bsps_plan()
    rc = load().bsps_get_plan(int(n), int(dtype), ctypes.byref(params), int(bool(with_payload)),
                              ctypes.byref(out))
    if rc:
        raise ValueError(f"bsps_get_plan: {bsps_strerror(rc)} ({rc})")
    return out


def bsps_workspace_size(n, dtype, params, with_payload=False) -> int:
    out = ctypes.c_size_t()
    rc = load().bsps_workspace_size(int(n), int(dtype), ctypes.byref(params), int(bool(with_payload)),
                                    ctypes.byref(out))
    if rc:
        raise ValueError(f"bsps_workspace_size: {bsps_strerror(rc)} ({rc})")
    return out.value


def bsps_sort_keys(keys_in, keys_out, n, dtype, params, bucket_sizes, workspace, stream=None) -> int:
    return load().bsps_sort_keys(_ptr(keys_in), _ptr(keys_out), int(n), int(dtype), ctypes.byref(params),
                                 _ptr(bucket_sizes), _ptr(workspace), _nbytes(workspace), _stream(stream))


def bsps_sort_keys_noalloc(keys_in, keys_out, n, dtype, params, bucket_sizes, stream=None) -> int:
    """bsps_sort_keys for callers that cannot allocate: the library's static
    device scratch replaces the workspace (see include/bspsort.h)."""
    return load().bsps_sort_keys_noalloc(_ptr(keys_in), _ptr(keys_out), int(n), int(dtype), ctypes.byref(params),
                                         _ptr(bucket_sizes), _stream(stream))


def bsps_noalloc_read_stats(stream=None) -> bsps_stats:
    """Status and statistics of the last bsps_sort_keys_noalloc call (synchronises
    the stream); .status is the device-side status."""
    st = bsps_stats()
    rc = load().bsps_noalloc_read_stats(ctypes.byref(st), _stream(stream))
    if rc == BSPS_ERR_CUDA or rc == BSPS_ERR_INVALID_ARG:
        raise RuntimeError(f"bsps_noalloc_read_stats: {bsps_strerror(rc)} ({rc})")
    return st


def bsps_sort_pairs(keys_in, vals_in, keys_out, vals_out, n, dtype, params, bucket_sizes, workspace,
                    stream=None) -> int:
    return load().bsps_sort_pairs(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), int(n),
                                  int(dtype), ctypes.byref(params), _ptr(bucket_sizes), _ptr(workspace),
                                  _nbytes(workspace), _stream(stream))


def bsps_sort_debug(keys_in, vals_in, keys_out, vals_out, n, dtype, params, bucket_sizes, workspace,
                    sample=None, splitters=None, bucket_of=None, pad_sizes=None, phase_events=None,
                    launches=None, mlp_params=None, mlp_loss=None, stall_tile=0, wait_polls=0,
                    partition=None, stream=None) -> int:
    """phase_events: BSPS_PHASES recorded torch.cuda.Event objects (or raw handles);
    launches: a ctypes.c_int32 that receives the number of kernels launched;
    stall_tile, wait_polls: the test hooks of the bounded waits (include/bspsort.h);
    partition: (p+1)*R uint32 entries of the merge final step's partition."""
    dbg = bsps_debug(_ptr(sample), _ptr(splitters), _ptr(bucket_of), _ptr(pad_sizes), None, None,
                     _ptr(mlp_params), _ptr(mlp_loss), int(stall_tile), int(wait_polls), _ptr(partition))
    if phase_events is not None:
        handles = [e if isinstance(e, int) else e.cuda_event for e in phase_events]
        assert len(handles) == BSPS_PHASES and all(handles), "events must exist (record them once first)"
        dbg.phase_events = (ctypes.c_void_p * BSPS_PHASES)(*handles)
    if launches is not None:
        dbg.launches = ctypes.pointer(launches)
    return load().bsps_sort_debug(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), int(n),
                                  int(dtype), ctypes.byref(params), _ptr(bucket_sizes), ctypes.byref(dbg),
                                  _ptr(workspace), _nbytes(workspace), _stream(stream))


def bsps_mlp_workspace_size(m) -> int:
    out = ctypes.c_size_t()
    rc = load().bsps_mlp_workspace_size(int(m), ctypes.byref(out))
    if rc:
        raise ValueError(f"bsps_mlp_workspace_size: {bsps_strerror(rc)} ({rc})")
    return out.value


def bsps_mlp_loss_grad(params, x, y, m, grad, loss, workspace, stream=None) -> int:
    return load().bsps_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(y), int(m), _ptr(grad), _ptr(loss),
                                     _ptr(workspace), _nbytes(workspace), _stream(stream))


def bsps_mlp_predict(params, x, m, y, workspace, stream=None) -> int:
    return load().bsps_mlp_predict(_ptr(params), _ptr(x), int(m), _ptr(y), _ptr(workspace), _nbytes(workspace),
                                   _stream(stream))


def _offsets(offsets):
    """Host int64 offsets (a sequence or numpy array) as a ctypes array."""
    vals = [int(v) for v in offsets]
    return (ctypes.c_int64 * max(1, len(vals)))(*vals), len(vals) - 1


def bsps_tune_default() -> bsps_tune:
    t = bsps_tune()
    rc = load().bsps_tune_default(ctypes.byref(t))
    if rc:
        raise ValueError(f"bsps_tune_default: {bsps_strerror(rc)} ({rc})")
    return t


def bsps_batch_bucket_base(offsets, tune) -> list:
    arr, num = _offsets(offsets)
    base = (ctypes.c_int64 * (num + 1))()
    rc = load().bsps_batch_bucket_base(arr, num, ctypes.byref(tune), base)
    if rc:
        raise ValueError(f"bsps_batch_bucket_base: {bsps_strerror(rc)} ({rc})")
    return list(base)


def bsps_batch_workspace_size(offsets, dtype, params, tune) -> int:
    arr, num = _offsets(offsets)
    out = ctypes.c_size_t()
    rc = load().bsps_batch_workspace_size(arr, num, int(dtype), ctypes.byref(params), ctypes.byref(tune),
                                          ctypes.byref(out))
    if rc:
        raise ValueError(f"bsps_batch_workspace_size: {bsps_strerror(rc)} ({rc})")
    return out.value


def bsps_sort_batched(keys_in, keys_out, offsets, dtype, params, tune, bucket_sizes, workspace,
                      stream=None) -> int:
    """offsets: host sequence of num+1 key offsets (see include/bspsort.h)."""
    arr, num = _offsets(offsets)
    return load().bsps_sort_batched(_ptr(keys_in), _ptr(keys_out), arr, num, int(dtype), ctypes.byref(params),
                                    ctypes.byref(tune), _ptr(bucket_sizes), _ptr(workspace), _nbytes(workspace),
                                    _stream(stream))


def bsps_autotune_workspace_size(dtype, params, max_log2) -> int:
    out = ctypes.c_size_t()
    rc = load().bsps_autotune_workspace_size(int(dtype), ctypes.byref(params), int(max_log2), ctypes.byref(out))
    if rc:
        raise ValueError(f"bsps_autotune_workspace_size: {bsps_strerror(rc)} ({rc})")
    return out.value


def bsps_autotune_batched(dtype, params, max_log2, tune, workspace, stream=None) -> int:
    return load().bsps_autotune_batched(int(dtype), ctypes.byref(params), int(max_log2), ctypes.byref(tune),
                                        _ptr(workspace), _nbytes(workspace), _stream(stream))


def bsps_read_stats(workspace, stream=None) -> bsps_stats:
    st = bsps_stats()
    load().bsps_read_stats(_ptr(workspace), ctypes.byref(st), _stream(stream))
    return st


def bsps_strerror(status: int) -> str:
    return load().bsps_strerror(int(status)).decode()
