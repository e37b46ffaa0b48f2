"""ctypes view of the C ABI declared in include/mpr.h (argument marshalling only).

The shared library is the in-tree build ``_build/libmpr.so``.  Loading fails
loudly when it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmpr.so")

MPR_OK = 0
STATUS = {
    0: "MPR_OK", 1: "MPR_ERR_INVALID_ARG", 2: "MPR_ERR_CUDA", 3: "MPR_ERR_DEGENERATE_RANGE",
    4: "MPR_ERR_NO_SAMPLE_PAIRS", 5: "MPR_ERR_T_OUT_OF_RANGE", 6: "MPR_ERR_WORKSPACE",
    7: "MPR_ERR_STATE", 8: "MPR_ERR_DEVICE",
}
MPR_DEVICE, MPR_HOST = 0, 1
MPR_PATH_TILED, MPR_PATH_PLAIN = 0, 1
MPR_EQUIL, MPR_MEASURE = 0, 1
MPR_MODEL_MPR, MPR_MODEL_GMRF = 0, 1
MPR_RECORD_ENERGY = 1

# every symbol include/mpr.h declares
EXPORTS = (
    "mpr_version", "mpr_last_error", "mpr_status_string", "mpr_default_params",
    "mpr_default_T_opts", "mpr_workspace_size", "mpr_init_grid", "mpr_get_image_info",
    "mpr_estimate_T", "mpr_set_T", "mpr_get_T", "mpr_sweep", "mpr_energy", "mpr_predict",
    "mpr_reset_accumulators", "mpr_get_state", "mpr_set_state", "mpr_get_chain_info",
    "mpr_set_chain_a", "mpr_get_sweep_index", "mpr_set_sweep_index", "mpr_destroy",
    "mpr_lattice_energy", "mpr_lattice_torque", "mpr_lattice_grad", "mpr_philox",
    "mpr_math_probe",
    "mpr_sample_energy_noalloc", "mpr_equilibrate", "mpr_get_energy_history",
    "mpr_get_accumulators", "mpr_set_accumulators",
    "mpr_eT_table_workspace_size", "mpr_eT_table", "mpr_set_T_from_table", "mpr_autotune",
    "mpr_select_q_workspace_size", "mpr_select_q", "mpr_sweep_launches",
)


class MprParams(C.Structure):
    _fields_ = [("q", C.c_double), ("J", C.c_double), ("A_targ", C.c_double), ("k_a", C.c_double),
                ("seed", C.c_uint64), ("freeze_a_in_measure", C.c_int), ("path", C.c_int),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("chain_group", C.c_int),
                ("literal_or", C.c_int), ("use_graphs", C.c_int), ("model", C.c_int)]


class MprTOpts(C.Structure):
    _fields_ = [("L", C.c_int), ("chains", C.c_int), ("n_equil", C.c_int), ("n_meas", C.c_int),
                ("iters", C.c_int), ("T_lo", C.c_double), ("T_hi", C.c_double)]


class MprError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libmpr.so (built by paper_1710_03038_gb300.build) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library {path} is missing: run paper_1710_03038_gb300.build.build() "
                "(there is no CPU fallback)")
        lib = C.CDLL(path)
        vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
        ip = C.POINTER(C.c_int)
        i64p = C.POINTER(C.c_int64)
        dp = C.POINTER(C.c_double)
        fp = C.POINTER(C.c_float)
        u32p = C.POINTER(C.c_uint32)
        pp = C.POINTER(MprParams)
        tp = C.POINTER(MprTOpts)
        sigs = {
            "mpr_version": (C.c_char_p, []),
            "mpr_last_error": (C.c_char_p, []),
            "mpr_status_string": (C.c_char_p, [i]),
            "mpr_default_params": (i, [pp]),
            "mpr_default_T_opts": (i, [tp]),
            "mpr_workspace_size": (i, [i, ip, ip, i64p, i, pp, tp, C.POINTER(sz)]),
            "mpr_init_grid": (i, [C.POINTER(vp), i, ip, ip, i, pp, tp, vp, vp, i, vp, sz, vp]),
            "mpr_get_image_info": (i, [vp, dp, i64p, i64p, fp, fp]),
            "mpr_estimate_T": (i, [vp, dp, vp]),
            "mpr_set_T": (i, [vp, dp, vp]),
            "mpr_get_T": (i, [vp, dp, vp]),
            "mpr_sweep": (i, [vp, i, i, i, vp]),
            "mpr_energy": (i, [vp, vp, i, vp]),
            "mpr_predict": (i, [vp, vp, vp, i, vp]),
            "mpr_reset_accumulators": (i, [vp, vp]),
            "mpr_get_accumulators": (i, [vp, vp, vp, i64p, i, vp]),
            "mpr_set_accumulators": (i, [vp, vp, vp, C.c_int64, i, vp]),
            "mpr_get_state": (i, [vp, vp, i, vp]),
            "mpr_set_state": (i, [vp, vp, i, vp]),
            "mpr_get_chain_info": (i, [vp, fp, u32p, dp, vp]),
            "mpr_set_chain_a": (i, [vp, fp, vp]),
            "mpr_get_sweep_index": (i, [vp, u32p, u32p]),
            "mpr_set_sweep_index": (i, [vp, C.c_uint32, C.c_uint32, vp]),
            "mpr_destroy": (None, [vp]),
            "mpr_lattice_energy": (i, [i, ip, ip, vp, d, d, vp, vp]),
            "mpr_lattice_torque": (i, [i, ip, ip, vp, d, d, vp, vp, vp]),
            "mpr_lattice_grad": (i, [i, ip, ip, vp, d, d, vp, vp, vp, vp]),
            "mpr_philox": (i, [i, vp, u32p, vp, i, vp]),
            "mpr_math_probe": (i, [i, i, vp, vp, vp, vp]),
            "mpr_equilibrate": (i, [vp, i, i, i, ip, vp]),
            "mpr_get_energy_history": (i, [vp, dp, vp]),
            "mpr_eT_table_workspace_size": (i, [i, i, i, C.POINTER(sz)]),
            "mpr_eT_table": (i, [i, i, dp, i, i, i, pp, vp, sz, dp, dp, vp]),
            "mpr_set_T_from_table": (i, [vp, i, dp, dp, dp, vp]),
            "mpr_autotune": (i, [i, ip, ip, i, pp, vp, vp, i, vp, sz, i, dp, vp]),
            "mpr_sample_energy_noalloc": (i, [i, ip, ip, vp, vp, d, d, vp, vp, vp, vp, vp]),
            "mpr_select_q_workspace_size": (i, [i, i, i, pp, tp, C.POINTER(sz)]),
            "mpr_sweep_launches": (i, [vp, ip, ip]),
            "mpr_select_q": (i, [i, i, vp, vp, vp, i, i, dp, i, i, i, pp, tp, vp, sz, dp, dp, dp,
                                 vp]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def check(fn: str, status: int):
    if status != MPR_OK:
        msg = load().mpr_last_error().decode(errors="replace")
        raise MprError(fn, status, msg)


def call(fn: str, *args):
    check(fn, getattr(load(), fn)(*args))


def int_array(vals):
    arr = (C.c_int * len(vals))(*[int(v) for v in vals])
    return arr


def i64_array(vals):
    return (C.c_int64 * len(vals))(*[int(v) for v in vals])
