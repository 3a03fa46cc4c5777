"""GPU parity of the sparse-state path (hy_support, hy_apply_h_sparse,
hy_pool_gradients_sparse): on states with few nonzero amplitudes (the
paper's early-ADAPT regime) against the oracle and the dense path.

Tolerances: support lists exact (as sets); FP64 sigma 1e-12 max-abs and
gradients 1e-11 (atomic adds change only the summation order); FP32 sigma
2e-5 * max|sigma| and gradients 1e-5 relative, as for the dense sweeps.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


_CACHE = {}


def system(n, na, nb, seed):
    key = (n, na, nb, seed)
    if key not in _CACHE:
        import paper_2604_01176_gb300 as hy
        h1, h2, ec = synth.integrals(n, seed)
        ref = oracle.System(h1, h2, ec, n, na, nb)
        ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
        _CACHE[key] = (ref, ham, hy.Pool(ham))
    return _CACHE[key]


def prepared(ref, seed, nops):
    """HF rotated by a few pool exponentials: a sparse, ADAPT-like state."""
    opd = ref.pool()
    rng = np.random.default_rng(seed)
    psi = ref.hf_state()
    for k in rng.integers(0, len(opd), nops):
        psi = ref.apply_excitation(opd[k], rng.normal(0, 0.4), psi)
    return psi


def support(ham, psi, cap=None):
    from paper_2604_01176_gb300 import _abi, dtype_code, stream_ptr
    cap = ham.n_det if cap is None else cap
    lst = torch.full((max(cap, 1),), -7, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    _abi.check(_abi.load().hy_support(ham.handle, ctypes.c_void_p(psi.data_ptr()),
                                      dtype_code(psi.dtype), ctypes.c_void_p(lst.data_ptr()),
                                      cap, ctypes.c_void_p(cnt.data_ptr()), stream_ptr()))
    return lst, int(cnt.item())


def sparse_h(ham, psi, lst, m):
    from paper_2604_01176_gb300 import _abi, dtype_code, stream_ptr
    sig = torch.full_like(psi, 3.0)   # must be overwritten
    _abi.check(_abi.load().hy_apply_h_sparse(
        ham.handle, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(sig.data_ptr()),
        dtype_code(psi.dtype), ctypes.c_void_p(lst.data_ptr()), m, stream_ptr()))
    return sig


def sparse_g(ham, pool, psi, sig, lst, m, ops=None):
    from paper_2604_01176_gb300 import _abi, dtype_code, stream_ptr
    n = len(pool) if ops is None else ops.numel()
    g = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    _abi.check(_abi.load().hy_pool_gradients_sparse(
        ham.handle, pool.handle, ctypes.c_void_p(psi.data_ptr()),
        ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(lst.data_ptr()), m,
        None if ops is None else ctypes.c_void_p(ops.data_ptr()), n,
        ctypes.c_void_p(g.data_ptr()), dtype_code(psi.dtype), stream_ptr()))
    return g


@pytest.mark.parametrize("cfg", [(6, 3, 3, 1001), (7, 4, 3, 77), (8, 4, 4, 1005),
                                 (10, 5, 5, 1002)])
def test_sparse_path_matches_oracle_and_dense(cfg):
    ref, ham, pool = system(*cfg)
    for seed, nops in [(1, 3), (2, 6)]:
        psi = prepared(ref, seed, nops)
        P = torch.from_numpy(psi).cuda()
        lst, m = support(ham, P)
        assert m == int(np.count_nonzero(psi))
        assert set(lst[:m].cpu().tolist()) == set(np.nonzero(psi)[0].tolist())
        S = sparse_h(ham, P, lst, m)
        s_ref = ref.sigma(psi)
        assert np.abs(S.cpu().numpy() - s_ref).max() < 1e-12
        g = sparse_g(ham, pool, P, S, lst, m).cpu().numpy()
        g_ref = ref.gradients(ref.pool(), psi, s_ref)
        assert np.abs(g - g_ref).max() < 1e-11
        sub = torch.tensor([len(pool) - 1, 2, 0], dtype=torch.int32, device="cuda")
        gs = sparse_g(ham, pool, P, S, lst, m, sub).cpu().numpy()
        assert np.abs(gs - g_ref[[len(pool) - 1, 2, 0]]).max() < 1e-11
        # float: against the dense float path
        P32 = P.float()
        l32, m32 = support(ham, P32)
        S32 = sparse_h(ham, P32, l32, m32)
        D32 = ham.apply_h(P32)
        assert torch.max(torch.abs(S32 - D32)).item() <= 2e-5 * torch.max(torch.abs(D32)).item()
        g32 = sparse_g(ham, pool, P32, D32, l32, m32)
        gd32 = pool.gradients(P32, D32)
        assert torch.max(torch.abs(g32 - gd32)).item() <= 1e-5 * torch.max(torch.abs(gd32)).item()


def test_support_cap_and_empty_state():
    ref, ham, pool = system(6, 3, 3, 1001)
    psi = torch.from_numpy(prepared(ref, 3, 5)).cuda()
    full, m = support(ham, psi)
    part, m2 = support(ham, psi, cap=3)
    assert m2 == m and m > 3
    assert set(part[:3].cpu().tolist()) <= set(full[:m].cpu().tolist())
    z = torch.zeros(ham.n_det, dtype=torch.float64, device="cuda")
    lst, m0 = support(ham, z)
    assert m0 == 0
    S = sparse_h(ham, z, lst, 0)
    assert torch.count_nonzero(S).item() == 0
    assert torch.count_nonzero(sparse_g(ham, pool, z, S, lst, 0)).item() == 0


@pytest.mark.parametrize("n,seed", [(14, 1003), (16, 1004)])
def test_sparse_path_full_size(n, seed):
    """28 / 32 qubits: a state a few excitations from HF; the sparse sigma
    against the dense sweep (all rows) and the oracle (sampled rows), the
    sparse screen against the dense screen."""
    ref, ham, pool = system(n, n // 2, n // 2, seed)
    psi = prepared(ref, 4, 5)
    P = torch.from_numpy(psi).cuda()
    lst, m = support(ham, P)
    assert m == int(np.count_nonzero(psi))
    S = sparse_h(ham, P, lst, m)
    D = ham.apply_h(P)
    assert torch.max(torch.abs(S - D)).item() < 1e-12
    rows = np.concatenate([np.nonzero(psi)[0][:8], [0, ref.n_det - 1]])
    assert np.abs(S[torch.from_numpy(rows).cuda()].cpu().numpy()
                  - ref.sigma_rows(psi, rows)).max() < 1e-12
    g = sparse_g(ham, pool, P, S, lst, m)
    gd = pool.gradients(P, D)
    assert torch.max(torch.abs(g - gd)).item() < 1e-11


@pytest.mark.parametrize("cfg,iters", [((6, 3, 3, 1001), 8), ((8, 4, 4, 1005), 6)])
def test_sparse_driver_follows_dense_driver(cfg, iters):
    """The ADAPT driver with the sparse path enabled selects the same
    operators and reaches the same energies as with the dense sweeps."""
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = system(*cfg)
    dense = hy.Adapt(ham, pool, "f64", max_iter=iters).run(iters)
    sp = hy.Adapt(ham, pool, "f64", max_iter=iters, sparse=True).run(iters)
    assert [r["selected"] for r in sp] == [r["selected"] for r in dense]
    assert max(abs(a["energy"] - b["energy"]) for a, b in zip(sp, dense)) < 1e-10
    mixed = hy.Adapt(ham, pool, "mixed", max_iter=iters, sparse=True).run(iters)
    assert [r["selected"] for r in mixed] == [r["selected"] for r in dense]
    assert abs(mixed[-1]["energy"] - dense[-1]["energy"]) < 1e-6
