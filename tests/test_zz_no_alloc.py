"""The allocation-free gradient screen (hy_pool_gradients_noalloc) against
the regular one (hy_pool_gradients), called through the C ABI.

It exists for callers that cannot let the library allocate device memory
(a process whose memory another allocator has fully reserved, or a loop
that must never pay cudaFree's device-wide synchronisation).  It keeps its
scratch in a fixed device array shared by all calls, so this test calls it
twice in a row (the second call sees the first call's leftovers) and checks
both against the regular entry point within the FP64 gradient tolerance of
the parity tests (1e-11), and FP32 within 1e-5 relative.  This file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_01176_gb300 as hy
    from paper_2604_01176_gb300 import _abi
    n, na, nb, seed = synth.workload("h8_16q")
    h1, h2, ec = synth.integrals(n, seed)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    pool = hy.Pool(ham)
    return hy, _abi, ham, pool


def call_noalloc(_abi, ham, pool, psi, sigma, ops, out):
    lib = _abi.load()
    n = len(pool) if ops is None else ops.numel()
    st = lib.hy_pool_gradients_noalloc(
        ham.handle, pool.handle, ctypes.c_void_p(psi.data_ptr()),
        ctypes.c_void_p(sigma.data_ptr()),
        None if ops is None else ctypes.c_void_p(ops.data_ptr()), n,
        ctypes.c_void_p(out.data_ptr()), 0 if psi.dtype == torch.float64 else 1,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_regular_screen_twice(setup, dtype):
    hy, _abi, ham, pool = setup
    tol = (lambda ref: 1e-11) if dtype == torch.float64 else \
        (lambda ref: 1e-5 * float(ref.abs().max()))
    for seed in (1, 2):    # two different states, two calls each
        psi = torch.from_numpy(synth.random_state(ham.n_det, seed)).to("cuda", dtype)
        sigma = ham.apply_h(psi)
        ref_all = pool.gradients(psi, sigma)
        sub = torch.tensor([len(pool) - 1, 3, 0, 17], dtype=torch.int32, device="cuda")
        ref_sub = pool.gradients(psi, sigma, ops=sub)
        for _ in range(2):
            g = torch.full((len(pool),), np.nan, dtype=torch.float64, device="cuda")
            assert call_noalloc(_abi, ham, pool, psi, sigma, None, g) == _abi.HY_OK
            gs = torch.full((4,), np.nan, dtype=torch.float64, device="cuda")
            assert call_noalloc(_abi, ham, pool, psi, sigma, sub, gs) == _abi.HY_OK
            torch.cuda.synchronize()
            assert torch.max(torch.abs(g - ref_all)).item() <= tol(ref_all)
            assert torch.max(torch.abs(gs - ref_sub)).item() <= tol(ref_sub)


def test_noalloc_rejects_beyond_capacity(setup):
    hy, _abi, ham, pool = setup
    lib = _abi.load()
    psi = torch.zeros(ham.n_det, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ops = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.hy_pool_gradients_noalloc(
        ham.handle, pool.handle, ctypes.c_void_p(psi.data_ptr()),
        ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(ops.data_ptr()), (1 << 18) + 1,
        ctypes.c_void_p(out.data_ptr()), 0, None)
    assert st == _abi.HY_ERR_ARG
    assert b"no-alloc scratch" in lib.hy_last_error()
