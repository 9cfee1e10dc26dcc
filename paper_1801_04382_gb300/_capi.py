"""ctypes declarations of the C ABI in ``include/krotov_traj.h`` (argument marshalling only).

The shared library is built in-tree by ``paper_1801_04382_gb300.build``.  Loading fails
loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

from .build import lib_path

KT_OK = 0
STATUS_NAMES = {
    0: "KT_OK", -1: "KT_ERR_ARG", -2: "KT_ERR_OOM", -3: "KT_ERR_CUDA", -4: "KT_ERR_TIMEOUT",
    -5: "KT_ERR_NONFINITE", -6: "KT_ERR_RECORD_FULL", -7: "KT_ERR_STATE", -8: "KT_ERR_RANGE",
    -9: "KT_ERR_UNSUPPORTED",
}
KT_FP64, KT_FP32_MIXED = 0, 1

dp = ct.POINTER(ct.c_double)
ip = ct.POINTER(ct.c_int)


class ModelDesc(ct.Structure):
    _fields_ = [
        ("n_nodes", ct.c_int), ("n_loc", ct.c_int), ("h0_local", dp),
        ("n_ctrl", ct.c_int), ("ctrl_node", ip), ("hc_local", dp), ("a_local", dp),
        ("n_pairs", ct.c_int), ("pair_dst", ip), ("pair_src", ip), ("pair_coef", dp),
        ("n_lind", ct.c_int), ("lind_coef", dp),
        ("psi0", dp), ("psi0_batch", dp), ("psi_tgt", dp),
    ]


class Config(ct.Structure):
    _fields_ = [
        ("T", ct.c_double), ("nt", ct.c_int), ("M", ct.c_int), ("prec", ct.c_int),
        ("ckpt_interval", ct.c_int), ("eps_guess", dp), ("shape", dp), ("lambda_a", dp),
        ("uniforms", dp), ("n_passes", ct.c_int), ("draws_per_traj", ct.c_int),
        ("eps_bound", ct.c_double), ("cheb_tol", ct.c_double), ("tile_traj", ct.c_int),
        ("update_rule", ct.c_int), ("jump_scheme", ct.c_int), ("ckpt_prefix", ct.c_int),
        ("traj_offset", ct.c_int), ("M_total", ct.c_int), ("inject_copy_timeout", ct.c_int),
        ("items_per_thread", ct.c_int), ("per_interval_launches", ct.c_int),
    ]


class Info(ct.Structure):
    _fields_ = [
        ("d", ct.c_int), ("max_jumps", ct.c_int), ("cheb_terms", ct.c_int), ("tile_traj", ct.c_int),
        ("n_tiles", ct.c_int), ("threads", ct.c_int), ("e_min", ct.c_double), ("e_max", ct.c_double),
        ("damping", ct.c_double), ("device_bytes", ct.c_longlong), ("passes", ct.c_longlong),
        ("eps_bound", ct.c_double), ("sweeps", ct.c_longlong), ("ckpt_interval", ct.c_int),
        ("ckpt_kept_prefix", ct.c_int), ("costate_slots", ct.c_int), ("items_per_thread", ct.c_int),
        ("whole_sweep", ct.c_int),
    ]


# name -> (restype, argtypes); every symbol declared in include/krotov_traj.h
SIGNATURES = {
    "krotov_init": (ct.c_int, [ct.POINTER(ModelDesc), ct.POINTER(Config), ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "krotov_init_density": (ct.c_int, [ct.POINTER(ModelDesc), ct.POINTER(Config), ct.c_void_p,
                                       ct.POINTER(ct.c_void_p)]),
    "propagate_forward": (ct.c_int, [ct.c_void_p, ct.c_int, dp, ct.c_void_p]),
    "propagate_backward": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "krotov_gradient": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "krotov_set_pulses_device": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "krotov_get_JT": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "krotov_update": (ct.c_int, [ct.c_void_p, ct.c_int, dp, dp, ct.c_void_p]),
    "fidelity": (ct.c_int, [ct.c_void_p, dp, dp]),
    "krotov_get_pulses": (ct.c_int, [ct.c_void_p, dp]),
    "krotov_get_update": (ct.c_int, [ct.c_void_p, dp]),
    "krotov_set_pulses": (ct.c_int, [ct.c_void_p, dp]),
    "krotov_get_records": (ct.c_int, [ct.c_void_p, ip, ip, ip, dp, dp]),
    "krotov_get_states": (ct.c_int, [ct.c_void_p, dp]),
    "krotov_get_costate": (ct.c_int, [ct.c_void_p, ct.c_int, dp]),
    "krotov_get_info": (ct.c_int, [ct.c_void_p, ct.POINTER(Info)]),
    "krotov_set_uniforms": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p]),
    "krotov_pulse_noise": (ct.c_int, [ct.c_void_p, dp, dp, ct.c_void_p]),
    "krotov_set_profiling": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "krotov_get_profile": (ct.c_int, [ct.c_void_p, dp, ct.POINTER(ct.c_longlong)]),
    "krotov_free": (None, [ct.c_void_p]),
    "krotov_last_error": (ct.c_char_p, []),
    "krotov_init_batch": (ct.c_int, [ct.POINTER(ct.POINTER(ModelDesc)), ct.POINTER(ct.POINTER(Config)), ct.c_int,
                                     ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "krotov_batch_update": (ct.c_int, [ct.c_void_p, ct.c_int, dp, ct.c_void_p]),
    "krotov_batch_problem": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_void_p)]),
    "krotov_batch_info": (ct.c_int, [ct.c_void_p, ip, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_longlong)]),
    "krotov_batch_free": (None, [ct.c_void_p]),
    "kt_nccl_unique_id": (ct.c_int, [ct.c_char_p, ct.c_void_p]),
    "krotov_shard_nccl": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_int, ct.c_char_p]),
    "krotov_group_init": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.POINTER(ct.c_void_p)]),
    "krotov_group_update": (ct.c_int, [ct.c_void_p, ct.c_int, dp, ct.c_void_p]),
    "krotov_group_fidelity": (ct.c_int, [ct.c_void_p, dp, ct.c_void_p]),
    "krotov_group_free": (None, [ct.c_void_p]),
    "kt_bessel_j": (ct.c_int, [ct.c_double, ct.c_int, dp]),
    "kt_generator_dense": (ct.c_int, [ct.POINTER(ModelDesc), ct.POINTER(Config), ct.c_int, dp, dp]),
    "kt_update_overlap_noalloc": (ct.c_int, [ct.c_int, ct.c_int, ct.c_int, ip, dp, ct.c_int, ct.c_void_p,
                                             ct.c_void_p, dp, dp, ct.c_void_p, ct.c_void_p]),
}

_LIB = None


def load():
    """Load the in-tree shared library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run paper_1801_04382_gb300.build.build() "
                           "(or __graft_entry__.build()) first; there is no CPU fallback")
    lib = ct.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class KrotovError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int, where: str):
    if status != KT_OK:
        msg = load().krotov_last_error()
        raise KrotovError(status, where, msg.decode() if msg else "")
