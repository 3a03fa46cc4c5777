"""FP64 CPU oracle for the state-vector ADAPT-VQE hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path
(``paper_2604_01176_gb300``) and never imports it.

The C core (``hy_oracle.c``) computes sigma = H psi by the Slater-Condon rules,
applies operator strings by their second-quantised definition, applies the
exact exponential of pool generators and evaluates pool gradients.  This file
adds the ctypes binding, the dense ground state and the ADAPT-VQE loop.

Parity unpinned: none of the oracle's functions is left without a pin; see
tests/test_oracle_pins.py for each pin and the paper passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hy_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhy_oracle.so")
_lib = None

POOL_DESC_WIDTH = 11


def build(force: bool = False) -> str:
    """Compile the oracle's C core with gcc (OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    D = ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, D]
    lib.orc_destroy.argtypes = [P]
    lib.orc_binom.restype = I64
    lib.orc_binom.argtypes = [ctypes.c_int, ctypes.c_int]
    for f in ("orc_ndet", "orc_nalpha_str", "orc_nbeta_str"):
        getattr(lib, f).restype = I64
        getattr(lib, f).argtypes = [P]
    lib.orc_det.restype = ctypes.c_uint64
    lib.orc_det.argtypes = [P, I64]
    lib.orc_dets.argtypes = [P, P]
    lib.orc_index.restype = I64
    lib.orc_index.argtypes = [P, ctypes.c_uint64]
    lib.orc_apply_ops.restype = ctypes.c_int
    lib.orc_apply_ops.argtypes = [P, ctypes.c_int, ctypes.c_uint64, P, P]
    lib.orc_apply_h_definition.argtypes = [P, P, P]
    lib.orc_matrix_element.restype = D
    lib.orc_matrix_element.argtypes = [P, ctypes.c_uint64, ctypes.c_uint64]
    lib.orc_sigma.argtypes = [P, P, P, ctypes.c_int]
    lib.orc_sigma_rows.argtypes = [P, P, P, I64, P, ctypes.c_int]
    lib.orc_dense_h.argtypes = [P, P]
    lib.orc_pool_build.restype = I64
    lib.orc_pool_build.argtypes = [P, P, I64]
    lib.orc_apply_excitation.argtypes = [P, P, D, P]
    lib.orc_apply_generator.argtypes = [P, P, P, P]
    lib.orc_op_gradient.restype = D
    lib.orc_op_gradient.argtypes = [P, P, P, P]
    lib.orc_pool_gradients.argtypes = [P, P, I64, P, P, P, ctypes.c_int]
    lib.orc_threads_used.restype = ctypes.c_int
    lib.orc_threads_used.argtypes = [ctypes.c_int]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def binom(n: int, k: int) -> int:
    return int(_load().orc_binom(n, k))


def threads_used(nthreads: int = 0) -> int:
    return int(_load().orc_threads_used(nthreads))


class System:
    """One molecule: integrals plus its determinant space Omega_CIk."""

    def __init__(self, h1, h2, e_core, n_orb, n_alpha, n_beta):
        lib = _load()
        self.n, self.na, self.nb = n_orb, n_alpha, n_beta
        self.h1 = np.ascontiguousarray(h1, dtype=np.float64)
        self.h2 = np.ascontiguousarray(h2, dtype=np.float64)
        self.e_core = float(e_core)
        dp = ctypes.POINTER(ctypes.c_double)
        self._h = lib.orc_create(n_orb, n_alpha, n_beta,
                                 self.h1.ctypes.data_as(dp),
                                 self.h2.ctypes.data_as(dp), self.e_core)
        if not self._h:
            raise ValueError("bad system size")
        self.n_det = int(lib.orc_ndet(self._h))
        self.n_astr = int(lib.orc_nalpha_str(self._h))
        self.n_bstr = int(lib.orc_nbeta_str(self._h))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    # determinant space -------------------------------------------------
    def dets(self) -> np.ndarray:
        out = np.empty(self.n_det, dtype=np.uint64)
        _load().orc_dets(self._h, _ptr(out))
        return out

    def index(self, det: int) -> int:
        return int(_load().orc_index(self._h, int(det)))

    def hf_index(self) -> int:
        a = (1 << self.na) - 1
        b = (1 << self.nb) - 1
        return self.index(a | (b << self.n))

    def hf_state(self) -> np.ndarray:
        v = np.zeros(self.n_det)
        v[self.hf_index()] = 1.0
        return v

    # Hamiltonian ---------------------------------------------------------
    def sigma(self, psi: np.ndarray, nthreads: int = 0) -> np.ndarray:
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        out = np.empty(self.n_det)
        _load().orc_sigma(self._h, _ptr(psi), _ptr(out), nthreads)
        return out

    def sigma_rows(self, psi: np.ndarray, rows, nthreads: int = 0) -> np.ndarray:
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty(len(rows))
        _load().orc_sigma_rows(self._h, _ptr(psi), _ptr(rows), len(rows),
                               _ptr(out), nthreads)
        return out

    def sigma_definition(self, psi: np.ndarray) -> np.ndarray:
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        out = np.empty(self.n_det)
        _load().orc_apply_h_definition(self._h, _ptr(psi), _ptr(out))
        return out

    def matrix_element(self, bra: int, ket: int) -> float:
        return float(_load().orc_matrix_element(self._h, int(bra), int(ket)))

    def dense_h(self) -> np.ndarray:
        H = np.empty((self.n_det, self.n_det))
        _load().orc_dense_h(self._h, _ptr(H))
        return H

    def energy(self, psi: np.ndarray) -> float:
        return float(np.dot(psi, self.sigma(psi)))

    def fci_energy(self) -> float:
        """Lowest eigenvalue of the dense H on Omega_CIk (numpy eigh)."""
        return float(np.linalg.eigvalsh(self.dense_h())[0])

    # pool ----------------------------------------------------------------
    def pool(self) -> np.ndarray:
        lib = _load()
        k = int(lib.orc_pool_build(self._h, None, 0))
        desc = np.zeros((k, POOL_DESC_WIDTH), dtype=np.int32)
        lib.orc_pool_build(self._h, _ptr(desc), k)
        return desc

    def apply_excitation(self, op: np.ndarray, theta: float, psi: np.ndarray):
        op = np.ascontiguousarray(op, dtype=np.int32)
        out = np.array(psi, dtype=np.float64, copy=True)
        _load().orc_apply_excitation(self._h, _ptr(op), float(theta), _ptr(out))
        return out

    def apply_generator(self, op: np.ndarray, psi: np.ndarray) -> np.ndarray:
        op = np.ascontiguousarray(op, dtype=np.int32)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        out = np.empty(self.n_det)
        _load().orc_apply_generator(self._h, _ptr(op), _ptr(psi), _ptr(out))
        return out

    def gradients(self, pool: np.ndarray, psi, sigma, nthreads: int = 0):
        pool = np.ascontiguousarray(pool, dtype=np.int32)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        g = np.empty(len(pool))
        _load().orc_pool_gradients(self._h, _ptr(pool), len(pool), _ptr(psi),
                                   _ptr(sigma), _ptr(g), nthreads)
        return g


def apply_operator_string(ops, det: int):
    """Apply sum-free operator string by definition; ops[t] = 2*mode+dagger."""
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    out = ctypes.c_uint64(0)
    sg = ctypes.c_int(0)
    ok = _load().orc_apply_ops(_ptr(ops), len(ops), int(det),
                               ctypes.byref(out), ctypes.byref(sg))
    if not ok:
        return None
    return int(out.value), int(sg.value)
