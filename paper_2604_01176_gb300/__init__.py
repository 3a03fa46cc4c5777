"""GB300-native hot path of exact state-vector ADAPT-VQE emulation.

Thin Python layer over the C ABI in include/hyperion.h (libhyperion.so,
sm_103a CUDA kernels).  PyTorch provides device memory and streams; every
step of H psi, the energy and norm reductions, the pool-gradient screen and
exp(theta A) runs in the library's kernels.  The library fails loudly when it
is not built or no CUDA device is present: there is no CPU fallback.

Paper: arXiv 2604.01176, Sparse State-Vector Emulation section (H applied
to a state on the particle- and S_z-conserving determinant space, inner
products, exponentiated fermionic operators) and the ADAPT-VQE description
of its Numerical performance subsection.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import HY_F32, HY_F64, HyError, check

__all__ = ["Hamiltonian", "Pool", "Adapt", "Ranker", "Batch", "ExplicitH", "HyError", "dtype_code",
           "stream_ptr", "occupations", "ranker_features", "touched_weights", "topk"]

N_FEATURES = 16


def launch_count() -> int:
    """Kernels the library has launched so far in this process."""
    return int(_abi.load().hy_launch_count())


# kernel classes of hy_profile_* (include/hyperion.h, hy_prof_class)
PROFILE_CLASSES = ("hpsi", "hpsi_sparse", "excite", "sparse_excite", "screen", "screen_sparse",
                   "reduce", "features", "hmat")


def profile_enable(classes=()) -> None:
    """Clear the kernel-class counters and record CUDA events around the
    library's launches of the named classes (empty: stop recording)."""
    mask = 0
    for c in classes:
        mask |= 1 << PROFILE_CLASSES.index(c)
    check(_abi.load().hy_profile_enable(mask))


def profile_read(cls: str) -> dict:
    """{launches, ms, bytes, flops} recorded for one class since profile_enable."""
    n, ms, by, fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(_abi.load().hy_profile_read(PROFILE_CLASSES.index(cls), ctypes.byref(n),
                                      ctypes.byref(ms), ctypes.byref(by), ctypes.byref(fl)))
    return {"launches": n.value, "ms": ms.value, "bytes": by.value, "flops": fl.value}


def dtype_code(t: torch.dtype) -> int:
    if t == torch.float64:
        return HY_F64
    if t == torch.float32:
        return HY_F32
    raise TypeError(f"unsupported dtype {t}: use float64 or float32")


def stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _require_cuda(*ts):
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensors must live on a CUDA device")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


class Hamiltonian:
    """H built from integrals (chemists' notation) on Omega_CIk."""

    def __init__(self, h1, h2, e_core, n_orb, n_alpha, n_beta, prune_tol=1e-14, _handle=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        lib = _abi.load()
        self.n_orb, self.n_alpha, self.n_beta = int(n_orb), int(n_alpha), int(n_beta)
        if _handle is not None:
            self.device = torch.device("cuda", torch.cuda.current_device())
            self._h = _handle
            self._info()
            return
        h1 = np.ascontiguousarray(h1, dtype=np.float64)
        h2 = np.ascontiguousarray(h2, dtype=np.float64)
        if h1.shape != (n_orb, n_orb) or h2.shape != (n_orb,) * 4:
            raise ValueError("h1 must be (n, n) and h2 (n, n, n, n)")
        self.device = torch.device("cuda", torch.cuda.current_device())
        handle = ctypes.c_void_p()
        check(lib.hy_build_hamiltonian(
            h1.ctypes.data_as(ctypes.c_void_p), h2.ctypes.data_as(ctypes.c_void_p),
            float(e_core), self.n_orb, self.n_alpha, self.n_beta, float(prune_tol),
            ctypes.byref(handle)))
        self._h = handle
        self._info()

    def _info(self):
        vals = [ctypes.c_int64() for _ in range(5)]
        check(_abi.load().hy_ham_info(self._h, *[ctypes.byref(v) for v in vals]))
        (self.n_det, self.n_alpha_str, self.n_beta_str, self.n_groups,
         self.n_terms) = [v.value for v in vals]
        self._scalar = torch.zeros(4, dtype=torch.float64, device=self.device)

    def partition(self, eta: int, interleaved: bool = False, part: int = 0) -> "Hamiltonian":
        """H_eta (part 0: the Pauli terms inside one of 2^eta qubit blocks) or
        the cross-block rest (part 1) of the SV-MPS split, as a Hamiltonian."""
        h = ctypes.c_void_p()
        check(_abi.load().hy_ham_partition(self._h, int(eta), 1 if interleaved else 0, int(part),
                                           ctypes.byref(h)))
        return Hamiltonian(None, None, 0.0, self.n_orb, self.n_alpha, self.n_beta, _handle=h)

    def close(self):
        if getattr(self, "_h", None):
            _abi.load().hy_ham_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- tables --------------------------------------------------------------
    def pauli_table(self):
        x = np.empty(self.n_terms, dtype=np.uint64)
        z = np.empty(self.n_terms, dtype=np.uint64)
        c = np.empty(self.n_terms, dtype=np.float64)
        off = np.empty(self.n_groups + 1, dtype=np.int64)
        check(_abi.load().hy_ham_pauli_table(
            self._h, x.ctypes.data_as(ctypes.c_void_p), z.ctypes.data_as(ctypes.c_void_p),
            c.ctypes.data_as(ctypes.c_void_p), off.ctypes.data_as(ctypes.c_void_p)))
        return x, z, c, off

    # -- indexing ------------------------------------------------------------
    def rank(self, dets: torch.Tensor, stream=None) -> torch.Tensor:
        _require_cuda(dets)
        if dets.dtype not in (torch.int64, torch.uint64):
            raise TypeError("dets must be 64-bit integers")
        idx = torch.empty(dets.numel(), dtype=torch.int64, device=dets.device)
        check(_abi.load().hy_rank(self._h, _ptr(dets), _ptr(idx), dets.numel(),
                                  stream_ptr(stream)))
        return idx

    def unrank(self, idx: torch.Tensor, stream=None) -> torch.Tensor:
        _require_cuda(idx)
        out = torch.empty(idx.numel(), dtype=torch.int64, device=idx.device)
        check(_abi.load().hy_unrank(self._h, _ptr(idx), _ptr(out), idx.numel(),
                                    stream_ptr(stream)))
        return out

    def set_coupling(self, impl: str) -> None:
        """Float coupling phase A on the tensor cores ("tensor", default) or
        the FP32 SIMT pipes ("simt"); "withheld" runs the tensor-core kernel
        without its MMAs, a test of its bounded waits (wrong results)."""
        check(_abi.load().hy_ham_set_coupling(
            self._h, {"tensor": 0, "simt": 1, "withheld": 2}[impl]))

    def upload_bytes(self, pool=None) -> int:
        """Bytes this Hamiltonian's build (and the pool's) copied host -> device."""
        v = ctypes.c_int64()
        check(_abi.load().hy_ham_upload_bytes(self._h, pool.handle if pool else None,
                                              ctypes.byref(v)))
        return v.value

    def set_wait_limit(self, polls: int) -> None:
        """Polls of a tensor-core stage barrier before the wait gives up."""
        check(_abi.load().hy_ham_set_wait_limit(self._h, int(polls)))

    def profile_coupling(self, on: bool = True):
        """Record CUDA events around the alpha-beta coupling of later apply_h calls."""
        check(_abi.load().hy_ham_profile(self._h, 1 if on else 0))

    def coupling_ms(self) -> float:
        """Device time of the coupling in the last profiled apply_h (waits for it)."""
        ms = ctypes.c_float()
        check(_abi.load().hy_ham_coupling_ms(self._h, ctypes.byref(ms)))
        return ms.value

    def connections_per_det(self) -> float:
        """Nonzero matrix elements of H per determinant row (diagonal, alpha
        and beta singles and doubles, alpha-beta doubles): the number of
        multiply-adds one H psi needs per output amplitude."""
        from math import comb
        n, a, b = self.n_orb, self.n_alpha, self.n_beta
        sa, sb = a * (n - a), b * (n - b)
        da = comb(a, 2) * comb(n - a, 2)
        db = comb(b, 2) * comb(n - b, 2)
        return float(1 + sa + sb + da + db + sa * sb)

    def hf_index(self) -> int:
        # HF = lowest orbitals occupied: rank 0 in both spins
        return 0

    def hf_state(self, dtype=torch.float64) -> torch.Tensor:
        v = torch.zeros(self.n_det, dtype=dtype, device=self.device)
        v[self.hf_index()] = 1.0
        return v

    # -- sweeps --------------------------------------------------------------
    def _check_state(self, *ts):
        _require_cuda(*ts)
        for t in ts:
            if t is not None and t.numel() != self.n_det:
                raise ValueError(f"state must have n_det = {self.n_det} elements")

    def apply_h(self, psi: torch.Tensor, out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        self._check_state(psi, out)
        if out is None:
            out = torch.empty_like(psi)
        check(_abi.load().hy_apply_h(self._h, _ptr(psi), _ptr(out),
                                     dtype_code(psi.dtype), stream_ptr(stream)))
        return out

    def apply_h_rows(self, psi: torch.Tensor, row_begin: int, row_end: int,
                     out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Rows [row_begin, row_end) of H psi (alpha strings): a block of
        (row_end - row_begin) * n_beta_str amplitudes."""
        self._check_state(psi)
        n = (int(row_end) - int(row_begin)) * self.n_beta_str
        if out is None:
            out = torch.empty(max(n, 0), dtype=psi.dtype, device=psi.device)
        _require_cuda(out)
        if out.dtype != psi.dtype or out.numel() != n:
            raise ValueError(f"out must hold {n} amplitudes of the state's dtype")
        check(_abi.load().hy_apply_h_rows(self._h, _ptr(psi), _ptr(out), dtype_code(psi.dtype),
                                          int(row_begin), int(row_end), stream_ptr(stream)))
        return out

    def dot_rows(self, x_rows: torch.Tensor, y_rows: torch.Tensor, row_begin: int,
                 row_end: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """<x|y> over the row block [row_begin, row_end) (FP64 accuracy)."""
        n = (int(row_end) - int(row_begin)) * self.n_beta_str
        _require_cuda(x_rows, y_rows)
        if x_rows.numel() != n or y_rows.numel() != n or x_rows.dtype != y_rows.dtype:
            raise ValueError(f"row blocks must hold {n} amplitudes of one dtype")
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=x_rows.device)
        check(_abi.load().hy_dot_rows(self._h, _ptr(x_rows), _ptr(y_rows),
                                      dtype_code(x_rows.dtype), int(row_begin), int(row_end),
                                      _ptr(out), stream_ptr(stream)))
        return out

    def energy(self, psi: torch.Tensor, sigma: torch.Tensor | None = None,
               out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """<psi|H|psi> (or <psi|sigma>) as a 0-d float64 device tensor."""
        self._check_state(psi, sigma)
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=psi.device)
        check(_abi.load().hy_energy(
            self._h, _ptr(psi), _ptr(sigma) if sigma is not None else None,
            dtype_code(psi.dtype), _ptr(out), stream_ptr(stream)))
        return out

    def dot(self, x: torch.Tensor, y: torch.Tensor, out=None, stream=None):
        self._check_state(x, y)
        if x.dtype != y.dtype:
            raise TypeError("x and y must share a dtype")
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=x.device)
        check(_abi.load().hy_dot(self._h, _ptr(x), _ptr(y), dtype_code(x.dtype),
                                 _ptr(out), stream_ptr(stream)))
        return out

    def normalize(self, psi: torch.Tensor, stream=None) -> torch.Tensor:
        self._check_state(psi)
        check(_abi.load().hy_normalize(self._h, _ptr(psi), dtype_code(psi.dtype),
                                       stream_ptr(stream)))
        return psi

    def renormalize(self, psi: torch.Tensor, norm2: torch.Tensor, stream=None) -> torch.Tensor:
        """psi <- psi / sqrt(norm2) with norm2 a float64 device scalar."""
        self._check_state(psi)
        if norm2.dtype != torch.float64 or norm2.device != psi.device or norm2.numel() != 1:
            raise ValueError("norm2 must be a float64 scalar on the state's device")
        check(_abi.load().hy_renormalize(self._h, _ptr(psi), dtype_code(psi.dtype),
                                         _ptr(norm2), stream_ptr(stream)))
        return psi


class ExplicitH:
    """The Hamiltonian stored explicitly for the determinants whose alpha
    string lies in [row_begin, row_end) (hy_hmat_*): every structural
    nonzero of those rows, sliced by alpha string, in float64 or float32."""

    def __init__(self, ham: Hamiltonian, dtype=torch.float64, row_begin: int = 0,
                 row_end: int | None = None):
        self.ham = ham
        self.dtype = dtype
        self.row_begin = int(row_begin)
        self.row_end = ham.n_alpha_str if row_end is None else int(row_end)
        h = ctypes.c_void_p()
        check(_abi.load().hy_hmat_build(ham.handle, dtype_code(dtype), self.row_begin,
                                        self.row_end, ctypes.byref(h)))
        self._m = h
        vals = [ctypes.c_int64() for _ in range(5)]
        check(_abi.load().hy_hmat_info(self._m, *[ctypes.byref(v) for v in vals]))
        _, _, self.nnz, self.row_len, self.bytes = [v.value for v in vals]

    @staticmethod
    def size(ham: Hamiltonian, dtype=torch.float64, row_begin: int = 0,
             row_end: int | None = None) -> tuple[int, int]:
        """(bytes, stored entries) of the rows [row_begin, row_end)."""
        b, z = ctypes.c_int64(), ctypes.c_int64()
        check(_abi.load().hy_hmat_bytes(ham.handle, dtype_code(dtype), int(row_begin),
                                        ham.n_alpha_str if row_end is None else int(row_end),
                                        ctypes.byref(b), ctypes.byref(z)))
        return b.value, z.value

    def close(self):
        if getattr(self, "_m", None):
            _abi.load().hy_hmat_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._m

    def apply(self, psi: torch.Tensor, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
        """The stored rows of H psi ((row_end - row_begin) * n_beta_str)."""
        self.ham._check_state(psi)
        if psi.dtype != self.dtype:
            raise TypeError("psi must have the matrix's dtype")
        n = (self.row_end - self.row_begin) * self.ham.n_beta_str
        if out is None:
            out = torch.empty(n, dtype=psi.dtype, device=psi.device)
        _require_cuda(out)
        if out.numel() != n or out.dtype != psi.dtype:
            raise ValueError(f"out must hold {n} amplitudes of the matrix's dtype")
        check(_abi.load().hy_hmat_apply(self._m, _ptr(psi), _ptr(out), stream_ptr(stream)))
        return out

    def row(self, det: int):
        """(columns, values) of the stored row of determinant det."""
        n = ctypes.c_int64()
        check(_abi.load().hy_hmat_row(self._m, int(det), None, None, 0, ctypes.byref(n)))
        cols = np.zeros(n.value, dtype=np.int64)
        vals = np.zeros(n.value, dtype=np.float64)
        check(_abi.load().hy_hmat_row(self._m, int(det), cols.ctypes.data_as(ctypes.c_void_p),
                                      vals.ctypes.data_as(ctypes.c_void_p), n.value,
                                      ctypes.byref(n)))
        return cols, vals


class Pool:
    """Operator pool relative to the HF determinant: kind "sd" (spin-adapted
    fermionic singles+doubles) or "qeb" (qubit-excitation-based: one qubit
    excitation per spin-orbital single and double)."""

    def __init__(self, ham: Hamiltonian, kind: str = "sd"):
        lib = _abi.load()
        self.ham = ham
        self.kind = kind
        code = {"sd": _abi.HY_POOL_SPIN_ADAPTED_SD, "qeb": _abi.HY_POOL_QEB}[kind]
        handle = ctypes.c_void_p()
        check(lib.hy_pool_create(ham.handle, code, ctypes.byref(handle)))
        self._p = handle
        k = ctypes.c_int64()
        check(lib.hy_pool_size(self._p, ctypes.byref(k)))
        self.size = k.value

    def close(self):
        if getattr(self, "_p", None):
            _abi.load().hy_pool_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return self.size

    @property
    def handle(self):
        return self._p

    def n_kernels(self, k: int) -> int:
        """Kernel launches of one apply_excitation(k) (one per constituent)."""
        if not hasattr(self, "_nc"):
            self._nc = [int(d[0]) for d in self.descriptors()]
        return self._nc[k]

    def describe(self, k: int) -> np.ndarray:
        d = np.zeros(11, dtype=np.int32)
        check(_abi.load().hy_pool_describe(self._p, int(k),
                                           d.ctypes.data_as(ctypes.c_void_p)))
        return d

    def descriptors(self) -> np.ndarray:
        return np.stack([self.describe(k) for k in range(self.size)]) if self.size \
            else np.zeros((0, 11), dtype=np.int32)

    def gradients(self, psi: torch.Tensor, sigma: torch.Tensor,
                  ops: torch.Tensor | None = None, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
        """g_i = 2 <sigma|A_{ops[i]} psi> (all ops when ops is None)."""
        self.ham._check_state(psi, sigma)
        if psi.dtype != sigma.dtype:
            raise TypeError("psi and sigma must share a dtype")
        n = self.size if ops is None else ops.numel()
        if ops is not None:
            _require_cuda(ops)
            if ops.dtype != torch.int32:
                raise TypeError("ops must be int32")
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=psi.device)
        check(_abi.load().hy_pool_gradients(
            self.ham.handle, self._p, _ptr(psi), _ptr(sigma),
            _ptr(ops) if ops is not None else None, n, _ptr(out),
            dtype_code(psi.dtype), stream_ptr(stream)))
        return out

    def apply_excitation(self, k: int, theta: float, psi: torch.Tensor,
                         renormalize: bool = False, stream=None) -> torch.Tensor:
        self.ham._check_state(psi)
        check(_abi.load().hy_apply_excitation(
            self.ham.handle, self._p, int(k), float(theta), _ptr(psi),
            dtype_code(psi.dtype), 1 if renormalize else 0, stream_ptr(stream)))
        return psi

    def apply_excitation_tracked(self, k: int, theta: float, psi: torch.Tensor,
                                 norm2: torch.Tensor, stream=None) -> torch.Tensor:
        """exp(theta A_k) psi in place, adding the change of ||psi||^2 over
        the rotated pairs to norm2 (a float64 device scalar)."""
        self.ham._check_state(psi)
        if norm2.dtype != torch.float64 or norm2.device != psi.device or norm2.numel() != 1:
            raise ValueError("norm2 must be a float64 scalar on the state's device")
        check(_abi.load().hy_apply_excitation_tracked(
            self.ham.handle, self._p, int(k), float(theta), _ptr(psi),
            dtype_code(psi.dtype), _ptr(norm2), stream_ptr(stream)))
        return psi


class Adapt:
    """ADAPT-VQE driver (hy_adapt_*): screen, select, append, re-optimise.

    precision "f64" is plain double precision; "mixed" keeps the bulk of
    the sweeps in float (state renormalised in double after every
    exp(theta A)) and refines the parameters and the energy in double."""

    def __init__(self, ham: Hamiltonian, pool: Pool, precision="f64", max_iter=64,
                 eps_grad=1e-5, gtol=1e-9, gtol_bulk=1e-5, max_evals=200,
                 refine_steps=4, refine_every=1, screen_top_m=0, judge=False, sparse=False,
                 sparse_cap=0, exact_screen_work=0.0, float_from=0):
        lib = _abi.load()
        self.ham, self.pool = ham, pool
        if precision not in ("f64", "mixed"):
            raise ValueError("precision must be 'f64' or 'mixed'")
        cfg = _abi.AdaptConfig(HY_F64 if precision == "f64" else HY_F32, int(max_iter),
                               float(eps_grad), float(gtol), float(gtol_bulk),
                               int(max_evals), int(refine_steps), int(refine_every),
                               int(screen_top_m), 1 if judge else 0, 1 if sparse else 0,
                               int(sparse_cap), float(exact_screen_work), int(float_from))
        handle = ctypes.c_void_p()
        check(lib.hy_adapt_create(ham.handle, pool.handle, ctypes.byref(cfg),
                                  ctypes.byref(handle)))
        self._a = handle
        self.precision = precision

    def close(self):
        if getattr(self, "_a", None):
            _abi.load().hy_adapt_destroy(self._a)
            self._a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._a

    def step(self, stream=None) -> dict:
        rec = _abi.AdaptRecord()
        check(_abi.load().hy_adapt_step(self._a, ctypes.byref(rec), stream_ptr(stream)))
        return rec.as_dict()

    def run(self, iters: int, stream=None) -> list:
        out = []
        for _ in range(iters):
            r = self.step(stream)
            out.append(r)
            if r["converged"]:
                break
        return out

    def set_judge(self, on: bool):
        """Run the full screen as judge on the following ranked iterations."""
        check(_abi.load().hy_adapt_set_judge(self._a, 1 if on else 0))

    def io_bytes(self):
        """(host->device, device->host) bytes the driver has copied so far."""
        h, d = ctypes.c_int64(), ctypes.c_int64()
        check(_abi.load().hy_adapt_io_bytes(self._a, ctypes.byref(h), ctypes.byref(d)))
        return h.value, d.value

    def refine(self, steps=4, stream=None) -> float:
        """Refine the current ansatz in double precision; the double energy."""
        e = ctypes.c_double()
        check(_abi.load().hy_adapt_refine(self._a, int(steps), ctypes.byref(e),
                                          stream_ptr(stream)))
        return e.value

    def ansatz(self):
        lib = _abi.load()
        n = ctypes.c_int64()
        check(lib.hy_adapt_ansatz(self._a, None, None, 0, ctypes.byref(n)))
        ops = np.zeros(n.value, dtype=np.int64)
        th = np.zeros(n.value)
        if n.value:
            check(lib.hy_adapt_ansatz(self._a, ops.ctypes.data_as(ctypes.c_void_p),
                                      th.ctypes.data_as(ctypes.c_void_p), n.value,
                                      ctypes.byref(n)))
        return ops, th

    def set_ansatz(self, ops, thetas):
        ops = np.ascontiguousarray(ops, dtype=np.int64)
        th = np.ascontiguousarray(thetas, dtype=np.float64)
        check(_abi.load().hy_adapt_set_ansatz(self._a, ops.ctypes.data_as(ctypes.c_void_p),
                                              th.ctypes.data_as(ctypes.c_void_p), len(ops)))

    def evaluate(self, thetas, dtype=torch.float64, stream=None):
        """(E, dE/dtheta) of the current ansatz at `thetas` (adjoint sweep)."""
        th = np.ascontiguousarray(thetas, dtype=np.float64)
        e = ctypes.c_double()
        g = np.zeros(len(th))
        check(_abi.load().hy_adapt_evaluate(self._a, th.ctypes.data_as(ctypes.c_void_p),
                                            dtype_code(dtype), ctypes.byref(e),
                                            g.ctypes.data_as(ctypes.c_void_p),
                                            stream_ptr(stream)))
        return e.value, g

    def set_ranker(self, ranker: "Ranker", warm_iters=3, epochs=30, refresh_every=0):
        check(_abi.load().hy_adapt_set_ranker(self._a, ranker.handle, int(warm_iters),
                                              int(epochs), int(refresh_every)))
        self._ranker = ranker   # keep it alive as long as the driver

    def state(self, dtype=torch.float64, stream=None) -> torch.Tensor:
        out = torch.empty(self.ham.n_det, dtype=dtype, device=self.ham.device)
        check(_abi.load().hy_adapt_state(self._a, _ptr(out), dtype_code(dtype),
                                         stream_ptr(stream)))
        return out


def occupations(ham: Hamiltonian, psi: torch.Tensor, stream=None) -> torch.Tensor:
    """<psi|n_P|psi>/<psi|psi> for the 2n spin orbitals (blocked order)."""
    ham._check_state(psi)
    out = torch.empty(2 * ham.n_orb, dtype=torch.float32, device=psi.device)
    check(_abi.load().hy_occupations(ham.handle, _ptr(psi), dtype_code(psi.dtype),
                                     _ptr(out), stream_ptr(stream)))
    return out


def ranker_features(ham: Hamiltonian, pool: Pool, psi: torch.Tensor,
                    extra: torch.Tensor | None = None, sigma: torch.Tensor | None = None,
                    stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Per-operator ranker features, (K, 16) float32 on the device (into
    `out` when given, e.g. a slice of a packed feature buffer)."""
    ham._check_state(psi, sigma)
    if out is None:
        out = torch.empty((len(pool), N_FEATURES), dtype=torch.float32, device=psi.device)
    elif out.dtype != torch.float32 or out.shape != (len(pool), N_FEATURES) \
            or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 tensor of shape (K, 16)")
    if extra is not None:
        _require_cuda(extra)
        if extra.dtype != torch.float32 or extra.shape != (len(pool), 4):
            raise ValueError("extra must be float32 of shape (K, 4)")
    if sigma is not None and sigma.dtype != psi.dtype:
        raise TypeError("psi and sigma must share a dtype")
    check(_abi.load().hy_ranker_features(
        ham.handle, pool.handle, _ptr(psi), _ptr(sigma) if sigma is not None else None,
        dtype_code(psi.dtype), _ptr(extra) if extra is not None else None, _ptr(out),
        stream_ptr(stream)))
    return out


def touched_weights(ham: Hamiltonian, psi: torch.Tensor, stream=None) -> torch.Tensor:
    """D[(i,a), (j,b)]: weight of |psi|^2 on determinants with i in / a out of
    the alpha string and j in / b out of the beta string (i == a or j == b:
    no condition), shape (n*n, n*n)."""
    ham._check_state(psi)
    n = ham.n_orb
    out = torch.empty(n ** 4, dtype=torch.float32, device=psi.device)
    check(_abi.load().hy_touched_weights(ham.handle, _ptr(psi), dtype_code(psi.dtype),
                                         _ptr(out), stream_ptr(stream)))
    return out.view(n * n, n * n)


def touched_weights_sparse(ham: Hamiltonian, psi: torch.Tensor, support: torch.Tensor,
                           stream=None) -> torch.Tensor:
    """touched_weights from psi's support (int64 device tensor listing every
    nonzero amplitude once, e.g. from hy_support): O(support) work."""
    ham._check_state(psi)
    if support.dtype != torch.int64 or support.device != psi.device:
        raise TypeError("support must be an int64 tensor on the state's device")
    n = ham.n_orb
    out = torch.empty(n ** 4, dtype=torch.float32, device=psi.device)
    check(_abi.load().hy_touched_weights_sparse(ham.handle, _ptr(psi), dtype_code(psi.dtype),
                                                _ptr(support.contiguous()), support.numel(),
                                                _ptr(out), stream_ptr(stream)))
    return out.view(n * n, n * n)


def topk(scores: torch.Tensor, k: int, stream=None) -> torch.Tensor:
    """Indices of the k largest scores (descending, ties to the lower index)."""
    _require_cuda(scores)
    if scores.dtype != torch.float32:
        raise TypeError("scores must be float32")
    out = torch.empty(int(k), dtype=torch.int32, device=scores.device)
    check(_abi.load().hy_ranker_topk(_ptr(scores), scores.numel(), int(k), _ptr(out),
                                     stream_ptr(stream)))
    return out


class Ranker:
    """Learned pool ranker: MLP 16 -> H -> H -> H -> 1 (ReLU, FP32)."""

    def __init__(self, hidden=256, seed=7):
        handle = ctypes.c_void_p()
        check(_abi.load().hy_ranker_create(int(hidden), int(seed), ctypes.byref(handle)))
        self._r = handle
        self.hidden = int(hidden)

    def close(self):
        if getattr(self, "_r", None):
            _abi.load().hy_ranker_destroy(self._r)
            self._r = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._r

    def info(self) -> dict:
        npar, nsam = ctypes.c_int64(), ctypes.c_int64()
        nf, fit = ctypes.c_int(), ctypes.c_int()
        check(_abi.load().hy_ranker_info(self._r, ctypes.byref(npar), ctypes.byref(nsam),
                                         ctypes.byref(nf), ctypes.byref(fit)))
        return {"n_params": npar.value, "n_samples": nsam.value,
                "n_features": nf.value, "fitted": bool(fit.value)}

    def params(self) -> np.ndarray:
        out = np.empty(self.info()["n_params"], dtype=np.float32)
        check(_abi.load().hy_ranker_get_params(self._r, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, w: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float32)
        if w.size != self.info()["n_params"]:
            raise ValueError("parameter count mismatch")
        check(_abi.load().hy_ranker_set_params(self._r, w.ctypes.data_as(ctypes.c_void_p)))

    def predict(self, feat: torch.Tensor, stream=None) -> torch.Tensor:
        _require_cuda(feat)
        out = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
        check(_abi.load().hy_ranker_predict(self._r, _ptr(feat), feat.shape[0], _ptr(out),
                                            stream_ptr(stream)))
        return out

    def add_samples(self, feat: torch.Tensor, g: torch.Tensor, stream=None):
        _require_cuda(feat, g)
        if g.dtype != torch.float64 or feat.dtype != torch.float32:
            raise TypeError("feat must be float32 and g float64")
        check(_abi.load().hy_ranker_add_samples(self._r, _ptr(feat), _ptr(g), g.numel(),
                                                stream_ptr(stream)))

    def fit(self, epochs=30, batch=256, lr=1e-3, seed=1234, stream=None) -> float:
        loss = ctypes.c_float()
        check(_abi.load().hy_ranker_fit(self._r, int(epochs), int(batch), float(lr),
                                        int(seed), ctypes.byref(loss), stream_ptr(stream)))
        return loss.value


class Batch:
    """Many molecules in one persistent launch (hy_batch_*).  States are
    packed into one buffer; `offsets[m]` is molecule m's first amplitude."""

    def __init__(self, hams):
        self.hams = list(hams)
        arr = (ctypes.c_void_p * len(self.hams))(*[h.handle for h in self.hams])
        handle = ctypes.c_void_p()
        check(_abi.load().hy_batch_create(arr, len(self.hams), ctypes.byref(handle)))
        self._b = handle
        tot, nt = ctypes.c_int64(), ctypes.c_int64()
        check(_abi.load().hy_batch_info(self._b, ctypes.byref(tot), ctypes.byref(nt)))
        self.total, self.n_tasks = tot.value, nt.value
        off = np.zeros(len(self.hams) + 1, dtype=np.int64)
        check(_abi.load().hy_batch_offsets(self._b, off.ctypes.data_as(ctypes.c_void_p)))
        self.offsets = off
        self.device = self.hams[0].device

    def close(self):
        if getattr(self, "_b", None):
            _abi.load().hy_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, dtype=torch.float64) -> torch.Tensor:
        return torch.zeros(self.total, dtype=dtype, device=self.device)

    def pack(self, states, dtype=torch.float64) -> torch.Tensor:
        out = self.empty(dtype)
        for m, s in enumerate(states):
            out[self.offsets[m]:self.offsets[m] + self.hams[m].n_det] = s
        return out

    def unpack(self, packed: torch.Tensor):
        return [packed[self.offsets[m]:self.offsets[m] + h.n_det]
                for m, h in enumerate(self.hams)]

    def _check(self, psi, sigma, energies):
        _require_cuda(psi, sigma, energies)
        if psi.numel() != self.total or sigma.numel() != self.total or psi.dtype != sigma.dtype:
            raise ValueError("packed psi / sigma must have `total` elements of one dtype")
        if energies is not None and (energies.dtype != torch.float64
                                     or energies.numel() != len(self.hams)):
            raise ValueError("energies must be float64 with one entry per molecule")

    def apply_h(self, psi, sigma=None, energies=None, graph=False, stream=None):
        if sigma is None:
            sigma = torch.empty_like(psi)
        self._check(psi, sigma, energies)
        fn = _abi.load().hy_batch_graph_launch if graph else _abi.load().hy_batch_apply_h
        check(fn(self._b, _ptr(psi), _ptr(sigma), dtype_code(psi.dtype),
                 _ptr(energies) if energies is not None else None, stream_ptr(stream)))
        return sigma

    def set_pools(self, pools):
        """Attach one pool per molecule (pool m built on Hamiltonian m)."""
        self.pools = list(pools)
        arr = (ctypes.c_void_p * len(self.pools))(*[p.handle for p in self.pools])
        check(_abi.load().hy_batch_set_pools(self._b, arr))
        off = np.zeros(len(self.hams) + 1, dtype=np.int64)
        check(_abi.load().hy_batch_pool_offsets(self._b, off.ctypes.data_as(ctypes.c_void_p)))
        self.pool_offsets = off

    def gradients(self, psi, sigma, ops=None, op_offsets=None, out=None, stream=None):
        """Pool gradients of every molecule in one persistent launch: all
        operators (packed by `pool_offsets`), or per-molecule lists of local
        pool indices `ops` (device int32) with `op_offsets` (device int64,
        molecules + 1 entries; molecule m's entries at [op_offsets[m],
        op_offsets[m + 1]))."""
        self._check(psi, sigma, None)
        if ops is None:
            n = int(self.pool_offsets[-1])
        else:
            _require_cuda(ops, op_offsets)
            if ops.dtype != torch.int32 or op_offsets.dtype != torch.int64 \
                    or op_offsets.numel() != len(self.hams) + 1:
                raise ValueError("ops must be int32, op_offsets int64 with molecules + 1 entries")
            n = ops.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=psi.device)
        if out.dtype != torch.float64 or out.numel() < n:
            raise ValueError("out must be float64 with room for every entry")
        check(_abi.load().hy_batch_gradients(
            self._b, _ptr(psi), _ptr(sigma), _ptr(ops) if ops is not None else None,
            _ptr(op_offsets) if ops is not None else None, n, _ptr(out),
            dtype_code(psi.dtype), stream_ptr(stream)))
        return out

    @property
    def tile(self) -> dict:
        t = _abi.BatchTile()
        check(_abi.load().hy_batch_get_tile(self._b, ctypes.byref(t)))
        return {"gsize": t.gsize, "groups": t.groups, "ctas_per_sm": t.ctas_per_sm}

    def set_tile(self, gsize, groups, ctas_per_sm=0):
        t = _abi.BatchTile(int(gsize), int(groups), int(ctas_per_sm))
        check(_abi.load().hy_batch_set_tile(self._b, ctypes.byref(t)))

    def tune(self, psi, sigma, stream=None):
        """Autotune the tile shape on these buffers; returns (tile, ms)."""
        self._check(psi, sigma, None)
        t = _abi.BatchTile()
        ms = ctypes.c_double()
        check(_abi.load().hy_batch_tune(self._b, _ptr(psi), _ptr(sigma), dtype_code(psi.dtype),
                                        ctypes.byref(t), ctypes.byref(ms), stream_ptr(stream)))
        return {"gsize": t.gsize, "groups": t.groups, "ctas_per_sm": t.ctas_per_sm}, ms.value
