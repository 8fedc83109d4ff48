"""ctypes declarations of the libtufrg C ABI (include/tufrg.h).

Argument marshalling only.  Loading fails loudly when the library has not been
built: there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

STATUS = {0: "TUFRG_OK", 1: "TUFRG_EINVAL", 2: "TUFRG_ENOMEM", 3: "TUFRG_ECUDA", 4: "TUFRG_ENONFINITE",
          5: "TUFRG_ENOTCONV", 6: "TUFRG_ETIMEOUT", 7: "TUFRG_EFALLBACK", 8: "TUFRG_ENOTSUP", 9: "TUFRG_ETOOBIG"}

FP64, SPLIT32 = 0, 1
PRODUCTS_AUTO, PRODUCTS_TC, PRODUCTS_SIMT = 0, 1, 2
LOOPS_AUTO, LOOPS_TC, LOOPS_SIMT = 0, 1, 2
BASIS_ORBITAL, BASIS_BAND = 0, 1
SYMMETRY_AUTO, SYMMETRY_OFF, SYMMETRY_STATES = 0, 1, 2
SYMMETRIC_STATE = 4   # tufrg_rhs flag: the state has the model's loop symmetries
REG_TEMPERATURE, REG_MOMENTUM_SHELL = 0, 1   # regulators of the loops (Eq. def_lmp)
CH_P, CH_C = 1, 2


class ModelDesc(C.Structure):
    _fields_ = [("n_s", C.c_int), ("n_hop", C.c_int), ("hop_R", C.c_void_p), ("hop_t", C.c_void_p),
                ("mu", C.c_double), ("filling", C.c_double), ("T_mu", C.c_double), ("V0", C.c_void_p),
                ("n_ff", C.c_int), ("ff_R", C.c_void_p), ("Lq", C.c_int), ("nc", C.c_int),
                ("precision", C.c_int), ("products", C.c_int), ("symmetry", C.c_int), ("regulator", C.c_int),
                ("T_reg", C.c_double), ("loops", C.c_int), ("basis", C.c_int)]


class FlowOpts(C.Structure):
    _fields_ = [("T0", C.c_double), ("T_end", C.c_double), ("rtol", C.c_double), ("atol", C.c_double),
                ("h0", C.c_double), ("stop", C.c_double), ("channel_mask", C.c_int), ("max_steps", C.c_int)]


class FlowResult(C.Structure):
    _fields_ = [("Tc", C.c_double), ("crossed", C.c_int), ("n_steps", C.c_int), ("n_reject", C.c_int),
                ("n_rhs", C.c_int), ("amax", C.c_double), ("T_last", C.c_double), ("lead_channel", C.c_int),
                ("lead_q", C.c_int), ("wall_s", C.c_double)]


class FlowStepInfo(C.Structure):
    _fields_ = [("T", C.c_double), ("h", C.c_double), ("err", C.c_double), ("amax", C.c_double),
                ("n_steps", C.c_int), ("n_reject", C.c_int), ("accepted", C.c_int), ("status", C.c_int)]


class TufrgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded library; raises if it has not been built (call build.build() first)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libtufrg is not built ({path} missing); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(path)
            vp, d, i, ip = C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int)
            L.tufrg_init_model.argtypes = [C.POINTER(ModelDesc), vp, C.POINTER(vp)]
            L.tufrg_free.argtypes = [vp]
            L.tufrg_free.restype = None
            L.tufrg_last_error.argtypes = [vp]
            L.tufrg_last_error.restype = C.c_char_p
            L.tufrg_dims.argtypes = [vp, ip, ip, ip, ip, C.POINTER(d)]
            L.tufrg_deltas.argtypes = [vp, vp]
            L.tufrg_model_info.argtypes = [vp, ip, C.POINTER(d), C.POINTER(d)]
            L.tufrg_model_info.restype = C.c_int
            L.tufrg_loop_momenta.argtypes = [vp, ip]
            L.tufrg_loop_momenta.restype = C.c_int
            L.tufrg_form_factors.argtypes = [vp, vp, vp]
            L.tufrg_form_factors.restype = C.c_int
            L.tufrg_irrep_basis.argtypes = [vp, vp, i, vp]
            L.tufrg_irrep_basis.restype = C.c_int
            L.tufrg_shard_classes.argtypes = [vp, ip, vp]
            L.tufrg_shard_classes.restype = C.c_int
            L.tufrg_rhs_shard_transform.argtypes = [vp, vp, i, vp, i, vp]
            L.tufrg_rhs_shard_transform.restype = C.c_int
            L.tufrg_rhs_shard_finish.argtypes = [vp, d, vp, i, vp, vp, i, vp]
            L.tufrg_rhs_shard_finish.restype = C.c_int
            L.tufrg_loops_info.argtypes = [vp, ip]
            L.tufrg_loops_info.restype = C.c_int
            L.tufrg_loop_tiles.argtypes = [vp, ip, ip, vp, i]
            L.tufrg_loop_tiles.restype = C.c_int
            L.tufrg_products_tiles.argtypes = [vp, ip, ip, vp, i]
            L.tufrg_products_tiles.restype = C.c_int
            L.tufrg_symmetry_info.argtypes = [vp, ip, C.POINTER(d), C.POINTER(d)]
            L.tufrg_symmetry_info.restype = C.c_int
            L.tufrg_round_f32.argtypes = [vp, vp, C.c_size_t, vp]
            L.tufrg_widen_f64.argtypes = [vp, vp, C.c_size_t, vp]
            L.tufrg_widen_f64.restype = C.c_int
            L.tufrg_band_basis.argtypes = [vp, vp, vp]
            L.tufrg_band_basis.restype = C.c_int
            L.tufrg_round_f32.restype = C.c_int
            L.tufrg_gather_table.argtypes = [vp, i, vp, i, ip]
            L.tufrg_bands.argtypes = [vp, vp, vp]
            L.tufrg_loops.argtypes = [vp, d, i, vp]
            L.tufrg_project.argtypes = [vp, vp, i, vp, C.POINTER(d)]
            L.tufrg_rhs.argtypes = [vp, d, vp, i, vp]
            L.tufrg_rhs_host.argtypes = [vp, d, vp, i, vp]
            L.tufrg_rhs_host_batch.argtypes = [vp, i, C.POINTER(d), C.POINTER(vp), i, C.POINTER(vp)]
            L.tufrg_rhs_host_batch.restype = C.c_int
            L.tufrg_flow.argtypes = [vp, C.POINTER(FlowOpts), vp, C.POINTER(FlowResult)]
            L.tufrg_loops_noalloc.argtypes = [i, i, vp, vp, d, d, i, vp, i, vp, vp]
            L.tufrg_loops_noalloc.restype = C.c_int
            L.tufrg_flow_batch.argtypes = [vp, i, C.POINTER(FlowOpts), vp]
            L.tufrg_flow_batch.restype = C.c_int
            L.tufrg_flow_start.argtypes = [vp, C.POINTER(FlowOpts)]
            L.tufrg_flow_step.argtypes = [vp, C.POINTER(FlowStepInfo)]
            L.tufrg_flow_amax_channels.argtypes = [vp, vp]
            L.tufrg_flow_end.argtypes = [vp, vp, C.POINTER(FlowResult)]
            L.tufrg_flow_checkpoint_bytes.argtypes = [vp]
            L.tufrg_flow_checkpoint_bytes.restype = C.c_size_t
            L.tufrg_flow_save.argtypes = [vp, vp, C.c_size_t]
            L.tufrg_flow_resume.argtypes = [vp, C.POINTER(FlowOpts), vp, C.c_size_t]
            for fn in ("tufrg_flow_start", "tufrg_flow_step", "tufrg_flow_amax_channels", "tufrg_flow_end",
                       "tufrg_flow_save", "tufrg_flow_resume"):
                getattr(L, fn).restype = C.c_int
            L.tufrg_mlp_create.argtypes = [i, i, i, i, C.c_ulonglong, vp, C.POINTER(vp)]
            L.tufrg_mlp_free.argtypes = [vp]
            L.tufrg_mlp_free.restype = None
            L.tufrg_mlp_last_error.argtypes = [vp]
            L.tufrg_mlp_last_error.restype = C.c_char_p
            L.tufrg_mlp_num_params.argtypes = [vp]
            L.tufrg_mlp_num_params.restype = C.c_longlong
            L.tufrg_mlp_get_params.argtypes = [vp, vp]
            L.tufrg_mlp_set_params.argtypes = [vp, vp]
            L.tufrg_mlp_forward.argtypes = [vp, vp, i, vp]
            L.tufrg_mlp_gradients.argtypes = [vp, vp, vp, i, vp, C.POINTER(C.c_float)]
            L.tufrg_mlp_train_step.argtypes = [vp, vp, vp, i, C.c_float, C.POINTER(C.c_float)]
            for fn in ("tufrg_mlp_create", "tufrg_mlp_get_params", "tufrg_mlp_set_params", "tufrg_mlp_forward",
                       "tufrg_mlp_gradients", "tufrg_mlp_train_step"):
                getattr(L, fn).restype = C.c_int
            L.tufrg_set_surrogate.argtypes = [vp, vp, vp, vp, vp, d, i, vp]
            L.tufrg_set_surrogate.restype = C.c_int
            L.tufrg_surrogate_stats.argtypes = [vp] + [C.POINTER(C.c_longlong)] * 3
            L.tufrg_surrogate_stats.restype = C.c_int
            L.tufrg_set_device_error.argtypes = [vp, i]
            L.tufrg_set_device_error.restype = C.c_int
            L.tufrg_timing_begin.argtypes = [vp]
            L.tufrg_timing_end.argtypes = [vp, vp, i, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
            for fn in ("tufrg_init_model", "tufrg_dims", "tufrg_deltas", "tufrg_gather_table", "tufrg_bands",
                       "tufrg_loops", "tufrg_project", "tufrg_rhs", "tufrg_rhs_host", "tufrg_flow",
                       "tufrg_timing_begin", "tufrg_timing_end"):
                getattr(L, fn).restype = C.c_int
            _lib = L
    return _lib


# names every header in include/ declares; the CPU test checks the exports against the headers
EXPORTS = ("tufrg_init_model", "tufrg_free", "tufrg_last_error", "tufrg_dims", "tufrg_deltas",
           "tufrg_gather_table", "tufrg_bands", "tufrg_loops", "tufrg_project", "tufrg_rhs", "tufrg_rhs_host",
           "tufrg_flow", "tufrg_timing_begin", "tufrg_timing_end", "tufrg_loops_noalloc", "tufrg_model_info", "tufrg_loop_momenta",
           "tufrg_symmetry_info", "tufrg_round_f32", "tufrg_rhs_host_batch",
           "tufrg_band_basis",
           "tufrg_flow_batch", "tufrg_mlp_create", "tufrg_mlp_free", "tufrg_mlp_last_error", "tufrg_mlp_num_params",
           "tufrg_mlp_get_params", "tufrg_mlp_set_params", "tufrg_mlp_forward", "tufrg_mlp_gradients",
           "tufrg_mlp_train_step", "tufrg_set_surrogate", "tufrg_surrogate_stats", "tufrg_set_device_error", "tufrg_loops_info", "tufrg_loop_tiles", "tufrg_products_tiles",
           "tufrg_shard_classes", "tufrg_rhs_shard_transform", "tufrg_rhs_shard_finish", "tufrg_form_factors",
           "tufrg_irrep_basis", "tufrg_flow_start", "tufrg_flow_step", "tufrg_flow_amax_channels", "tufrg_flow_end",
           "tufrg_flow_checkpoint_bytes", "tufrg_flow_save", "tufrg_flow_resume", "tufrg_widen_f64")
