"""ctypes binding of include/hyperion.h (argument marshalling only).

Every numerical step runs in the CUDA library ``libhyperion.so``; this module
declares the C signatures and raises if the library is missing.  There is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhyperion.so")

HY_OK, HY_ERR_ARG, HY_ERR_CUDA, HY_ERR_OOM, HY_ERR_TIMEOUT, HY_ERR_UNSUPPORTED = range(6)
HY_F64, HY_F32 = 0, 1
HY_POOL_SPIN_ADAPTED_SD = 0
HY_POOL_QEB = 1

_STATUS = {HY_ERR_ARG: "HY_ERR_ARG", HY_ERR_CUDA: "HY_ERR_CUDA",
           HY_ERR_OOM: "HY_ERR_OOM", HY_ERR_TIMEOUT: "HY_ERR_TIMEOUT",
           HY_ERR_UNSUPPORTED: "HY_ERR_UNSUPPORTED"}


class HyError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


class BatchTile(ctypes.Structure):
    """Mirror of hy_batch_tile."""
    _fields_ = [("gsize", ctypes.c_int), ("groups", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int)]


class AdaptConfig(ctypes.Structure):
    """Mirror of hy_adapt_config."""
    _fields_ = [("bulk", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("eps_grad", ctypes.c_double), ("gtol", ctypes.c_double),
                ("gtol_bulk", ctypes.c_double), ("max_evals", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("refine_every", ctypes.c_int),
                ("screen_top_m", ctypes.c_int),
                ("judge", ctypes.c_int), ("sparse", ctypes.c_int),
                ("sparse_cap", ctypes.c_int64), ("exact_screen_work", ctypes.c_double),
                ("float_from", ctypes.c_int64)]


class AdaptRecord(ctypes.Structure):
    """Mirror of hy_adapt_record."""
    _fields_ = [("iter", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("selected", ctypes.c_int64), ("max_grad", ctypes.c_double),
                ("grad_norm", ctypes.c_double), ("energy", ctypes.c_double),
                ("energy_bulk", ctypes.c_double), ("energy_bulk_err", ctypes.c_double),
                ("n_evals", ctypes.c_int32), ("n_evals_f64", ctypes.c_int32),
                ("true_argmax", ctypes.c_int64), ("true_rank", ctypes.c_int64),
                ("t_screen", ctypes.c_double), ("t_optimise", ctypes.c_double),
                ("t_total", ctypes.c_double), ("t_judge", ctypes.c_double),
                ("support", ctypes.c_int64),
                ("sigma_support", ctypes.c_int64),
                ("screen", ctypes.c_int32), ("pad_", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}

P = ctypes.c_void_p
I32 = ctypes.c_int
I64 = ctypes.c_int64
D = ctypes.c_double
PP = ctypes.POINTER(ctypes.c_void_p)
PI64 = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes)
SIGNATURES = {
    "hy_last_error": (ctypes.c_char_p, []),
    "hy_version": (ctypes.c_char_p, []),
    "hy_launch_count": (I64, []),
    "hy_profile_enable": (I32, [ctypes.c_uint32]),
    "hy_profile_read": (I32, [I32, PI64, ctypes.POINTER(D), ctypes.POINTER(D),
                              ctypes.POINTER(D)]),
    "hy_build_hamiltonian": (I32, [P, P, D, I32, I32, I32, D, PP]),
    "hy_ham_destroy": (I32, [P]),
    "hy_ham_info": (I32, [P, PI64, PI64, PI64, PI64, PI64]),
    "hy_ham_pauli_table": (I32, [P, P, P, P, P]),
    "hy_ham_profile": (I32, [P, I32]),
    "hy_ham_set_coupling": (I32, [P, I32]),
    "hy_ham_set_wait_limit": (I32, [P, I64]),
    "hy_ham_upload_bytes": (I32, [P, P, PI64]),
    "hy_ham_partition": (I32, [P, I32, I32, I32, P]),
    "hy_ham_coupling_ms": (I32, [P, P]),
    "hy_pauli_table_build": (I32, [P, P, D, I32, D, I64, P, P, P, P, PI64, PI64]),
    "hy_rank": (I32, [P, P, P, I64, P]),
    "hy_unrank": (I32, [P, P, P, I64, P]),
    "hy_apply_h": (I32, [P, P, P, I32, P]),
    "hy_apply_h_rows": (I32, [P, P, P, I32, I64, I64, P]),
    "hy_dot_rows": (I32, [P, P, P, I32, I64, I64, P, P]),
    "hy_hmat_bytes": (I32, [P, I32, I64, I64, PI64, PI64]),
    "hy_hmat_build": (I32, [P, I32, I64, I64, P]),
    "hy_hmat_destroy": (I32, [P]),
    "hy_hmat_info": (I32, [P, PI64, PI64, PI64, PI64, PI64]),
    "hy_hmat_apply": (I32, [P, P, P, P]),
    "hy_hmat_row": (I32, [P, I64, P, P, I64, PI64]),
    "hy_support": (I32, [P, P, I32, P, I64, P, P]),
    "hy_apply_h_sparse": (I32, [P, P, P, I32, P, I64, P]),
    "hy_pool_gradients_sparse": (I32, [P, P, P, P, P, I64, P, I64, P, I32, P]),
    "hy_energy": (I32, [P, P, P, I32, P, P]),
    "hy_dot": (I32, [P, P, P, I32, P, P]),
    "hy_normalize": (I32, [P, P, I32, P]),
    "hy_pool_create": (I32, [P, I32, PP]),
    "hy_pool_destroy": (I32, [P]),
    "hy_pool_size": (I32, [P, PI64]),
    "hy_pool_qubit": (I32, [P, ctypes.POINTER(ctypes.c_int)]),
    "hy_pool_describe": (I32, [P, I64, P]),
    "hy_pool_gradients": (I32, [P, P, P, P, P, I64, P, I32, P]),
    "hy_apply_excitation": (I32, [P, P, I64, D, P, I32, I32, P]),
    "hy_apply_excitation_tracked": (I32, [P, P, I64, D, P, I32, P, P]),
    "hy_renormalize": (I32, [P, P, I32, P, P]),
    "hy_pool_gradients_noalloc": (I32, [P, P, P, P, P, I64, P, I32, P]),
    "hy_batch_create": (I32, [P, I32, PP]),
    "hy_batch_destroy": (I32, [P]),
    "hy_batch_info": (I32, [P, PI64, PI64]),
    "hy_batch_offsets": (I32, [P, P]),
    "hy_batch_set_tile": (I32, [P, P]),
    "hy_batch_get_tile": (I32, [P, P]),
    "hy_batch_apply_h": (I32, [P, P, P, I32, P, P]),
    "hy_batch_graph_launch": (I32, [P, P, P, I32, P, P]),
    "hy_batch_tune": (I32, [P, P, P, I32, P, P, P]),
    "hy_batch_set_pools": (I32, [P, P]),
    "hy_batch_pool_offsets": (I32, [P, P]),
    "hy_batch_gradients": (I32, [P, P, P, P, P, I64, P, I32, P]),
    "hy_occupations": (I32, [P, P, I32, P, P]),
    "hy_ranker_features": (I32, [P, P, P, P, I32, P, P, P]),
    "hy_touched_weights": (I32, [P, P, I32, P, P]),
    "hy_touched_weights_sparse": (I32, [P, P, I32, P, I64, P, P]),
    "hy_ranker_create": (I32, [I32, ctypes.c_uint64, PP]),
    "hy_ranker_destroy": (I32, [P]),
    "hy_ranker_info": (I32, [P, PI64, PI64, P, P]),
    "hy_ranker_get_params": (I32, [P, P]),
    "hy_ranker_set_params": (I32, [P, P]),
    "hy_ranker_predict": (I32, [P, P, I64, P, P]),
    "hy_ranker_add_samples": (I32, [P, P, P, I64, P]),
    "hy_ranker_fit": (I32, [P, I32, I32, ctypes.c_float, ctypes.c_uint64, P, P]),
    "hy_ranker_topk": (I32, [P, I64, I64, P, P]),
    "hy_adapt_set_ranker": (I32, [P, P, I32, I32, I32]),
    "hy_adapt_create": (I32, [P, P, P, PP]),
    "hy_adapt_destroy": (I32, [P]),
    "hy_adapt_step": (I32, [P, P, P]),
    "hy_adapt_ansatz": (I32, [P, P, P, I64, PI64]),
    "hy_adapt_refine": (I32, [P, I32, P, P]),
    "hy_adapt_io_bytes": (I32, [P, PI64, PI64]),
    "hy_adapt_set_judge": (I32, [P, I32]),
    "hy_adapt_set_ansatz": (I32, [P, P, P, I64]),
    "hy_adapt_evaluate": (I32, [P, P, I32, P, P, P]),
    "hy_adapt_state": (I32, [P, P, I32, P]),
}


def load():
    """Load libhyperion.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with "
            "paper_2604_01176_gb300.build.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != HY_OK:
        msg = load().hy_last_error()
        raise HyError(status, msg.decode() if msg else "")
