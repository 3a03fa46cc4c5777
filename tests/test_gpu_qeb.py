"""The qubit-excitation-based pool (HY_POOL_QEB; paper: Numerical performance
subsection) on the GPU against the oracle's qubit excitations
(oracle/qeb.py): descriptors identical, the full and listed screens (FP64
1e-11, FP32 1e-5 relative), exp(theta A) of every operator (FP64 1e-12), the
sparse-state screen, and the ADAPT driver's trajectory over the QEB pool
(dense sweeps and sparse path) against the oracle's loop (same selections,
energies within 1e-10 Ha)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFGS = [(6, 3, 3, 1001), (7, 4, 3, 77), (5, 1, 4, 12)]
IDS = [f"n{c[0]}a{c[1]}b{c[2]}" for c in CFGS]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


_CACHE = {}


def system(n, na, nb, seed):
    key = (n, na, nb, seed)
    if key not in _CACHE:
        import paper_2604_01176_gb300 as hy
        from oracle.qeb import QubitSystem
        h1, h2, ec = synth.integrals(n, seed)
        ref = QubitSystem(oracle.System(h1, h2, ec, n, na, nb))
        ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
        _CACHE[key] = (ref, ham, hy.Pool(ham, "qeb"))
    return _CACHE[key]


def prepared(ref, pool, seed, nops):
    rng = np.random.default_rng(seed)
    psi = ref.hf_state()
    for k in rng.integers(0, len(pool), nops):
        psi = ref.apply_excitation(pool[k], rng.normal(0, 0.4), psi)
    return psi


@pytest.mark.parametrize("cfg", CFGS, ids=IDS)
def test_qeb_descriptors_match_oracle(cfg):
    ref, ham, pool = system(*cfg)
    assert pool.kind == "qeb"
    assert np.array_equal(pool.descriptors(), ref.pool())


@pytest.mark.parametrize("cfg", CFGS, ids=IDS)
def test_qeb_screen_and_excitations(cfg):
    ref, ham, pool = system(*cfg)
    opd = ref.pool()
    psi = prepared(ref, opd, cfg[3], 5)
    sig = ref.sigma(psi)
    g_ref = ref.gradients(opd, psi, sig)
    P = torch.from_numpy(psi).cuda()
    S = torch.from_numpy(sig).cuda()
    g = pool.gradients(P, S).cpu().numpy()
    assert np.abs(g - g_ref).max() < 1e-11
    sub = torch.tensor([len(opd) - 1, 0, len(opd) // 2], dtype=torch.int32, device="cuda")
    gs = pool.gradients(P, S, ops=sub).cpu().numpy()
    assert np.abs(gs - g_ref[sub.cpu().numpy()]).max() < 1e-11
    g32 = pool.gradients(P.float(), S.float()).cpu().numpy()
    assert np.abs(g32 - g_ref).max() < 1e-5 * max(1.0, np.abs(g_ref).max())
    for k in range(len(opd)):
        x = P.clone()
        pool.apply_excitation(k, 0.37, x)
        assert np.abs(x.cpu().numpy() - ref.apply_excitation(opd[k], 0.37, psi)).max() < 1e-12


def test_qeb_sparse_screen():
    import ctypes
    from paper_2604_01176_gb300 import _abi, dtype_code, stream_ptr
    ref, ham, pool = system(6, 3, 3, 1001)
    opd = ref.pool()
    psi = prepared(ref, opd, 4, 3)
    sig = ref.sigma(psi)
    g_ref = ref.gradients(opd, psi, sig)
    P = torch.from_numpy(psi).cuda()
    S = torch.from_numpy(sig).cuda()
    nz = torch.from_numpy(np.flatnonzero(psi).astype(np.int64)).cuda()
    g = torch.full((len(opd),), np.nan, dtype=torch.float64, device="cuda")
    _abi.check(_abi.load().hy_pool_gradients_sparse(
        ham.handle, pool.handle, ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(S.data_ptr()),
        ctypes.c_void_p(nz.data_ptr()), nz.numel(), None, len(opd),
        ctypes.c_void_p(g.data_ptr()), dtype_code(P.dtype), stream_ptr()))
    assert np.abs(g.cpu().numpy() - g_ref).max() < 1e-11


@pytest.mark.parametrize("sparse", [False, True], ids=["dense", "sparse"])
def test_qeb_adapt_matches_oracle_loop(sparse):
    import oracle.adapt as oadapt
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = system(6, 3, 3, 1001)
    opd = ref.pool()
    rec = oadapt.run(ref, opd, max_iter=6)
    ad = hy.Adapt(ham, pool, "f64", max_iter=6, sparse=sparse)
    got = ad.run(6)
    assert [r["selected"] for r in got] == rec["selected"]
    assert np.abs(np.array([r["energy"] for r in got]) - np.array(rec["energy"])).max() < 1e-10
    ops, th = ad.ansatz()
    e, g = ad.evaluate(th)
    e_ref, g_ref = oadapt.energy_and_gradient(ref, opd, list(ops), np.array(th))
    assert abs(e - e_ref) < 1e-10 and np.abs(g - g_ref).max() < 1e-9
