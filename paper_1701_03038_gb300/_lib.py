"""ctypes binding of libfstgpu.so (argument marshalling only).

Every entry point of ``include/fstgpu.h`` is declared here with the same
name.  Loading fails loudly when the library has not been built: there is
no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

OK, INVALID_ARG, NO_PATH, OOM, CUDA, TIMEOUT, UNSUPPORTED, STATE = range(8)
WEIGHT_LOG, WEIGHT_COST = 0, 1
FLAG_DEVICE_PTRS = 1
PLAN_SINGLE_WAVE, PLAN_NO_VITERBI, PLAN_NO_FB, PLAN_DENSE_ACC = 1, 2, 4, 8
DRIVER_LAUNCH, DRIVER_PERSISTENT = 0, 1
FAULT_NONE, FAULT_BARRIER_STALL = 0, 1
TUNE_REFRESH = 1
EM_APPLY = 2
SLICE_BY_DESTINATION, SLICE_BY_SOURCE = 0, 1
PLAIN_FRONTIER, PLAIN_SLICE, PLAIN_AUTO, PLAIN_BLOCK = 0, 1, 2, 3
BLOCK_MAX_STATES = 8192

_lock = threading.Lock()
_lib = None

vp = C.c_void_p
i32, i64 = C.c_int32, C.c_int64

# name -> argtypes (all return int, except fst_last_error)
SIGNATURES = {
    "fst_create": [i32, i64, vp, vp, vp, vp, vp, i32, vp, vp, i32, i32, C.POINTER(vp)],
    "fst_destroy": [vp],
    "fst_info": [vp, vp, vp, vp, vp, vp, vp, vp],
    "fst_symbol_stats": [vp, vp, vp, vp],
    "fst_set_weights": [vp, vp, i32, i32],
    "fst_set_state_weights": [vp, vp, vp, i32, i32],
    "fst_viterbi": [vp, vp, i32, vp, vp, vp],
    "fst_viterbi_slice": [vp, vp, i32, vp, vp],
    "fst_set_plain_method": [vp, i32],
    "fst_set_plain_driver": [vp, i32, i32],
    "fst_get_plain_method": [vp, vp, vp, vp],
    "fst_autotune_plain": [vp, vp, vp, i32, vp],
    "fst_forward_backward_slice": [vp, vp, i32, vp, vp],
    "fst_set_slice_order": [vp, i32],
    "fst_forward_backward": [vp, vp, i32, vp, vp],
    "fst_viterbi_batch": [vp, vp, vp, i32, vp, vp, vp, vp, vp],
    "fst_forward_backward_batch": [vp, vp, vp, i32, vp, vp, vp, vp, vp],
    "fst_plan_create": [vp, vp, vp, i32, i64, i32, vp, C.POINTER(vp)],
    "fst_plan_destroy": [vp],
    "fst_plan_info": [vp, vp, vp, vp, vp, vp, vp, vp, vp],
    "fst_plan_viterbi": [vp, vp, vp, vp, vp, vp],
    "fst_plan_forward": [vp, vp, vp, vp],
    "fst_plan_backward": [vp, vp, vp, vp],
    "fst_plan_forward_backward": [vp, vp, vp, vp, vp, vp],
    "fst_plan_backward_ex": [vp, vp, vp, vp, vp, vp],
    "fst_plan_live_work": [vp, vp, vp, vp],
    "fst_plan_forward_backward_ex": [vp, vp, vp, vp, vp, vp, vp, vp],
    "fst_plan_limit_pool": [vp, i64],
    "fst_plan_limit_table": [vp, i64],
    "fst_plan_set_pull": [vp, i64],
    "fst_debug_checks": [vp, vp, vp, vp],
    "fst_plan_table_slots": [vp, vp],
    "fst_set_batch_budget": [vp, i64],
    "fst_set_batch_plan": [vp, i32, i32, i32, i32],
    "fst_plan_set_driver": [vp, i32, i32, i64],
    "fst_plan_get_driver": [vp, vp, vp],
    "fst_plan_fault_inject": [vp, i32, i64],
    "fst_plan_autotune": [vp, vp, i32, vp, vp, vp],
    "fst_profile": [vp, i32],
    "fst_profile_read": [vp, vp, vp],
    "fst_live_work": [vp, vp, vp],
    "fst_plan_profile": [vp, i32],
    "fst_plan_profile_read": [vp, vp, vp],
    "fst_viterbi_noalloc": [vp, vp, i32, vp, vp, vp, vp],
    "fst_log_z_f64": [vp, vp, vp, i32, vp],
    "fst_em_update": [vp, vp, C.c_float, vp, i32],
    "fst_lattice_viterbi": [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp],
    "fst_prefix_log_z": [vp, vp, i32, vp, vp],
    "fst_lattice_forward_backward": [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp],
    "fst_create_clamped": [vp, C.POINTER(vp), vp],
    "fst_clamp_labels": [vp, vp, vp, i64, vp],
}

PROF_KINDS = ["vit_first", "vit_step", "vit_final", "backtrace", "fwd_first", "fwd_sum", "fwd_step", "fb_final",
              "bwd_step", "counts"]


class FstError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with code {code}: {msg}")
        self.code = code


def lib_path() -> str:
    """The in-tree build, unless FSTGPU_LIB names another build of it."""
    return os.environ.get("FSTGPU_LIB") or _build.LIB_PATH


def load(path: str | None = None):
    """Load libfstgpu.so; raises if it is missing (call build() first)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or lib_path()
        if not os.path.exists(p):
            raise RuntimeError(
                f"{p} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = C.CDLL(p)
        for name, args in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        lib.fst_last_error.argtypes = []
        lib.fst_last_error.restype = C.c_char_p
        if path is None:
            _lib = lib
        return lib


def check(rc: int, where: str, allow=(OK,)) -> int:
    if rc not in allow:
        msg = load().fst_last_error().decode(errors="replace")
        raise FstError(rc, where, msg)
    return rc
