"""ctypes binding over libdpp_gb300.so (the C ABI declared in include/dpp.h).

Argument marshalling only: every step of the sampler runs in the library's
CUDA kernels. torch supplies device memory and the current stream. There is no
fallback: if the library is missing or cannot run, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import struct
from typing import Optional

from . import build as _build

# enums mirrored from include/dpp.h
DPP_OK, DPP_ERR_INVALID_ARG, DPP_ERR_CUDA, DPP_ERR_WORKSPACE, DPP_ERR_UNSUPPORTED = range(5)
DPP_R64, DPP_C128 = 0, 1
DPP_PREC_FP64, DPP_PREC_3XTF32, DPP_PREC_BF16X6, DPP_PREC_FP32 = 0, 1, 2, 3
DPP_OP_SAMPLE_HERMITIAN, DPP_OP_SAMPLE_LU, DPP_OP_LOGPROB_BACKWARD = 0, 1, 2
DPP_OP_GREEDY_HERMITIAN, DPP_OP_GREEDY_LU, DPP_OP_SAMPLE_BATCHED = 3, 4, 5
DPP_STATIC_SCRATCH_BYTES = 4 << 20
DPP_STATIC_MAX_N_R64, DPP_STATIC_MAX_N_C128 = 15418, 7942
DPP_RES_NONFINITE, DPP_RES_TIMEOUT, DPP_RES_INADMISSIBLE, DPP_RES_RECOMPUTE = 1, 2, 4, 8
RESULT_BYTES = 32
RESULT_FMT = "<iiiidd"

PRECISIONS = {"fp64": DPP_PREC_FP64, "3xtf32": DPP_PREC_3XTF32, "bf16x6": DPP_PREC_BF16X6,
              "fp32": DPP_PREC_FP32}

_lib = None


class DPPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dpp status {status}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load the shared library (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    vp, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    L.dpp_abi_version.argtypes = []
    L.dpp_abi_version.restype = i32
    L.dpp_last_error.argtypes = []
    L.dpp_last_error.restype = ctypes.c_char_p
    L.dpp_workspace_size.argtypes = [i32, i64, i32, i32, i32]
    L.dpp_workspace_size.restype = sz
    for name in ("dpp_sample_hermitian", "dpp_sample_lu"):
        f = getattr(L, name)
        f.argtypes = [vp, i64, i64, i32, i32, u64, u64, vp, vp, vp, vp, vp, vp, sz, vp]
        f.restype = i32
    for name in ("dpp_greedy_hermitian", "dpp_greedy_lu"):
        f = getattr(L, name)
        f.argtypes = [vp, i64, i64, i32, i32, vp, vp, vp, vp, vp, sz, vp]
        f.restype = i32
    L.dpp_sample_hermitian_static.argtypes = [vp, i64, i64, i32, u64, u64, vp, vp, vp, vp, vp, vp]
    L.dpp_sample_hermitian_static.restype = i32
    L.dpp_batched_workspace_size.argtypes = [i32, i64, i32]
    L.dpp_batched_workspace_size.restype = sz
    L.dpp_sample_batched.argtypes = [i32, vp, vp, vp, i64, i32, u64, vp, vp, vp, vp, vp, vp, sz, vp]
    L.dpp_sample_batched.restype = i32
    L.dpp_logprob_backward.argtypes = [vp, i64, i64, i32, i32, i32, vp, vp, vp, i64, vp, sz, vp]
    L.dpp_logprob_backward.restype = i32
    L.dpp_logprob_backward_batched.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.dpp_logprob_backward_batched.restype = i32
    L.dpp_logprob_backward_batched_fp32.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.dpp_logprob_backward_batched_fp32.restype = i32
    L.dpp_logprob_backward_batched_workspace.argtypes = [i32, i64]
    L.dpp_logprob_backward_batched_workspace.restype = sz
    L.dpp_uniforms.argtypes = [u64, u64, i64, vp, vp]
    L.dpp_uniforms.restype = i32
    L.dpp_profile_start.argtypes = []
    L.dpp_profile_start.restype = None
    L.dpp_profile_stop.argtypes = [vp, i32]
    L.dpp_profile_stop.restype = i32
    L.dpp_set_tuning.argtypes = [i32, ctypes.c_double]
    L.dpp_set_tuning.restype = i32
    L.dpp_get_tuning.argtypes = [i32]
    L.dpp_get_tuning.restype = ctypes.c_double
    L.dpp_launch_count.argtypes = []
    L.dpp_launch_count.restype = ctypes.c_uint64
    L.dpp_autotune_workspace_size.argtypes = [i32, i64, i32, i32, i32]
    L.dpp_autotune_workspace_size.restype = sz
    L.dpp_autotune.argtypes = [i32, vp, i64, i64, i32, i32, i32, i32, vp, sz, vp, vp]
    L.dpp_autotune_batched.argtypes = [i32, vp, vp, vp, i64, u64, vp, vp, vp, sz, i32, vp, vp]
    L.dpp_autotune_batched.restype = i32
    L.dpp_autotune.restype = i32
    L.dpp_tune_lookup.argtypes = [i32, i64, i32, i32, vp]
    L.dpp_tune_lookup.restype = i32
    L.dpp_tune_save.argtypes = [ctypes.c_char_p]
    L.dpp_tune_save.restype = i32
    L.dpp_tune_load.argtypes = [ctypes.c_char_p]
    L.dpp_tune_load.restype = i32
    L.dpp_lensemble_to_marginal_batched.argtypes = [i32, vp, vp, vp, vp, vp, vp, sz, vp]
    L.dpp_lensemble_to_marginal_batched.restype = i32
    L.dpp_elementary_workspace_size.argtypes = [i64, i64]
    L.dpp_elementary_workspace_size.restype = sz
    L.dpp_sample_elementary.argtypes = [vp, i64, i64, i64, u64, u64, vp, vp, vp, vp, vp, vp, sz, vp]
    L.dpp_sample_elementary.restype = i32
    L.dpp_tune_clear.argtypes = []
    L.dpp_tune_clear.restype = None
    _lib = L
    return L


def last_error() -> str:
    return load().dpp_last_error().decode()


def check(status: int) -> None:
    if status != DPP_OK:
        raise DPPError(status, last_error())


def workspace_size(op: int, n: int, dtype: int, precision: int, hermitian: int = 1) -> int:
    return int(load().dpp_workspace_size(op, n, dtype, precision, hermitian))


def decode_result(raw: bytes) -> dict:
    status, kept, border, oor, logp, ratio = struct.unpack(RESULT_FMT, raw)
    return {"status": status, "n_kept": kept, "n_borderline": border,
            "n_out_of_range": oor, "logp": logp, "max_err_ratio": ratio}


def ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


def profile_start() -> None:
    load().dpp_profile_start()


def profile_stop() -> dict:
    """{category: {launches, total_ms, flops, bytes}} for the profiled window."""
    arr = (KernelStat * 16)()
    k = load().dpp_profile_stop(ctypes.cast(arr, ctypes.c_void_p), 16)
    out = {}
    for i in range(k):
        s = arr[i]
        out[s.name.decode()] = {"launches": int(s.launches), "total_ms": float(s.total_ms),
                                "flops": float(s.flops), "bytes": float(s.bytes)}
    return out


DPP_TUNE_TAU_SAFETY, DPP_TUNE_OUTER_BLOCK, DPP_TUNE_UPDATE_KERNEL, DPP_TUNE_MAX_CTAS = 0, 1, 2, 3
DPP_TUNE_PANEL_PIPELINE = 4
DPP_TUNE_WAIT_NS, DPP_TUNE_FAULT_WITHHOLD, DPP_TUNE_USE_CACHE = 5, 6, 7
DPP_TUNE_UPDATE_VARIANT = 8
DPP_TUNE_PANEL_CTAS = 9
DPP_TUNE_BATCHED_THREADS = 10


class TuneEntry(ctypes.Structure):
    """dpp_tune_entry (include/dpp.h)."""
    _fields_ = [("op", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("n_bucket", ctypes.c_int32),
                ("n", ctypes.c_int64), ("outer_block", ctypes.c_int32),
                ("panel_pipeline", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("samples_per_s", ctypes.c_double),
                ("candidates", ctypes.c_int32), ("update_variant", ctypes.c_int32),
                ("batched_threads", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def tune_lookup(op: int, n: int, dtype: int, precision: int):
    """The tuning table's entry for this key on the current device, or None."""
    e = TuneEntry()
    st = load().dpp_tune_lookup(op, n, dtype, precision, ctypes.byref(e))
    if st == DPP_ERR_UNSUPPORTED:
        return None
    check(st)
    return e.as_dict()


def tune_save(path: str) -> None:
    check(load().dpp_tune_save(os.fsencode(path)))


def tune_load(path: str) -> None:
    check(load().dpp_tune_load(os.fsencode(path)))


def tune_clear() -> None:
    load().dpp_tune_clear()


def set_tuning(key: int, value: float) -> None:
    check(load().dpp_set_tuning(key, float(value)))


def get_tuning(key: int) -> float:
    return float(load().dpp_get_tuning(key))


def launch_count() -> int:
    return int(load().dpp_launch_count())
