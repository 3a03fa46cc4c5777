"""Host-visible failure paths of the CUDA library, exercised without a GPU
fault: operator lists that hold indices outside the pool, and a bounded
tensor-core wait that runs out.

* The screens (hy_pool_gradients and its sparse and allocation-free
  variants) refuse pool indices outside [0, K): a list in pageable host
  memory is checked before any launch; a device list is checked by the
  kernels, which read nothing out of range, return NaN for that entry and
  leave a report that the next screen call on the pool returns as
  HY_ERR_ARG.
* The float H|psi>'s tensor-core coupling waits on mbarriers with a poll
  limit.  With its MMAs withheld (hy_ham_set_coupling impl 2) no barrier
  ever completes, so every wait runs out, the kernel records a timeout,
  frees its tensor memory and returns; the next hy_apply_h reports
  HY_ERR_TIMEOUT and the handle then works again.  No wait in this test is
  unbounded: each gives up after the short limit set here.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sys12():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_01176_gb300 as hy
    n, na, nb, seed = synth.workload("h6_12q")
    h1, h2, ec = synth.integrals(n, seed)
    ref = oracle.System(h1, h2, ec, n, na, nb)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    return hy, ref, ham, hy.Pool(ham)


def _state(ham, seed=5, dtype=torch.float64):
    psi = torch.from_numpy(synth.random_state(ham.n_det, seed)).to("cuda", dtype)
    return psi, ham.apply_h(psi)


def _screen(lib, fn, ham, pool, psi, sigma, ops_ptr, n, out, extra=()):
    args = [ham.handle, pool.handle, ctypes.c_void_p(psi.data_ptr()),
            ctypes.c_void_p(sigma.data_ptr())]
    if fn == "hy_pool_gradients_sparse":
        args += list(extra)
    args += [ops_ptr, n, ctypes.c_void_p(out.data_ptr()),
             0 if psi.dtype == torch.float64 else 1,
             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)]
    return getattr(lib, fn)(*args)


@pytest.mark.parametrize("fn", ["hy_pool_gradients", "hy_pool_gradients_noalloc",
                                "hy_pool_gradients_sparse"])
def test_device_list_with_bad_index_reported_by_next_screen(sys12, fn):
    hy, ref, ham, pool = sys12
    from paper_2604_01176_gb300 import _abi
    lib = _abi.load()
    K = len(pool)
    psi, sigma = _state(ham)
    full = pool.gradients(psi, sigma)
    extra = ()
    if fn == "hy_pool_gradients_sparse":
        lst = torch.arange(ham.n_det, dtype=torch.int64, device="cuda")   # every entry
        extra = (ctypes.c_void_p(lst.data_ptr()), ham.n_det)
    for bad in (K, K + 1000, -1):
        ops = torch.tensor([3, bad, 0, K - 1], dtype=torch.int32, device="cuda")
        out = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
        assert _screen(lib, fn, ham, pool, psi, sigma, ctypes.c_void_p(ops.data_ptr()), 4,
                       out, extra) == 0
        torch.cuda.synchronize()
        g = out.cpu().numpy()
        assert np.isnan(g[1])
        ok = full[torch.tensor([3, 0, K - 1], device="cuda")].cpu().numpy()
        assert np.abs(g[[0, 2, 3]] - ok).max() < 1e-11
        # the next screen on this pool reports it, then the report is cleared
        out2 = torch.empty(K, dtype=torch.float64, device="cuda")
        st = _screen(lib, fn, ham, pool, psi, sigma, None, K, out2, extra)
        assert st == 1
        msg = lib.hy_last_error().decode()
        assert f"held {bad} at position 1" in msg and f"pool size {K}" in msg
        assert _screen(lib, fn, ham, pool, psi, sigma, None, K, out2, extra) == 0
        torch.cuda.synchronize()
        assert torch.max(torch.abs(out2 - full)).item() < 1e-11


def test_pageable_host_list_checked_before_launch(sys12):
    hy, ref, ham, pool = sys12
    from paper_2604_01176_gb300 import _abi
    lib = _abi.load()
    K = len(pool)
    psi, sigma = _state(ham)
    full = pool.gradients(psi, sigma)
    out = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    l0 = hy.launch_count()
    bad = np.array([1, 2, K + 3], dtype=np.int32)
    st = _screen(lib, "hy_pool_gradients", ham, pool, psi, sigma,
                 bad.ctypes.data_as(ctypes.c_void_p), 3, out)
    assert st == 1
    msg = lib.hy_last_error().decode()
    assert (f"ops_or_null[2] = {K + 3}" in msg) or ("cannot read" in msg)
    assert hy.launch_count() == l0                     # refused before any launch
    assert torch.all(out == 7.0)
    pageable = "cannot read" not in msg
    if pageable:
        good = np.array([1, 2, K - 1], dtype=np.int32)
        st = _screen(lib, "hy_pool_gradients", ham, pool, psi, sigma,
                     good.ctypes.data_as(ctypes.c_void_p), 3, out)
        assert st == 0
        torch.cuda.synchronize()
        ref_g = full[torch.tensor([1, 2, K - 1], device="cuda")]
        assert torch.max(torch.abs(out - ref_g)).item() < 1e-11


@pytest.mark.parametrize("cfg", [(6, 3, 3, 1001), (4, 2, 2, 5)], ids=["n6", "n4"])
def test_tensor_core_wait_runs_out_and_is_reported(cfg):
    """n = 6: the wait that runs out is inside the chunk loop; n = 4 (two
    chunks per tile): it is the drain after the loop."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_01176_gb300 as hy
    n, na, nb, seed = cfg
    h1, h2, ec = synth.integrals(n, seed)
    ref = oracle.System(h1, h2, ec, n, na, nb)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    psi64 = synth.random_state(ham.n_det, 3)
    psi = torch.from_numpy(psi64).to("cuda", torch.float32)
    ham.set_wait_limit(2000)
    ham.set_coupling("withheld")
    ham.apply_h(psi)                      # the kernel gives up and returns
    torch.cuda.synchronize()              # the context is still usable
    with pytest.raises(hy.HyError) as ei:
        ham.apply_h(psi)
    assert ei.value.status == 4 and "timed out" in str(ei.value)
    ham.set_coupling("tensor")
    ham.set_wait_limit(1 << 26)
    sig = ham.apply_h(psi)
    torch.cuda.synchronize()
    s_ref = ref.sigma(psi.double().cpu().numpy())
    assert np.abs(sig.double().cpu().numpy() - s_ref).max() <= 2e-5 * np.abs(s_ref).max()
