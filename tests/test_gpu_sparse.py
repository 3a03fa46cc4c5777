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
        # listed zero amplitudes change nothing
        zeros = np.setdiff1d(np.arange(len(psi)), np.nonzero(psi)[0])[:5]
        lz = torch.cat([lst[:m], torch.from_numpy(zeros).cuda()])
        Sz = sparse_h(ham, P, lz, lz.numel())
        assert np.abs(Sz.cpu().numpy() - s_ref).max() < 1e-12
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
    # small supports optimise in double directly ...
    assert all(r["energy_bulk_err"] == 0.0 for r in mixed)
    # ... unless float is asked for at every size: float phase, double
    # refinement, the next screen on the refined double state
    flt = hy.Adapt(ham, pool, "mixed", max_iter=iters, sparse=True, float_from=1).run(iters)
    assert [r["selected"] for r in flt] == [r["selected"] for r in dense]
    assert abs(flt[-1]["energy"] - dense[-1]["energy"]) < 1e-9
    assert all(0.0 < r["energy_bulk_err"] < 1e-4 for r in flt)


def _ansatz(ref, seed, length):
    rng = np.random.default_rng(seed)
    return list(rng.integers(0, len(ref.pool()), length)), rng.normal(0, 0.5, length)


@pytest.mark.parametrize("cfg", [(6, 3, 3, 1001), (7, 4, 3, 77), (8, 4, 4, 1005)])
@pytest.mark.parametrize("cap", ["all", "tiny"])
def test_sparse_state_evaluation_matches_oracle(cfg, cap):
    """hy_adapt_evaluate through the sparse-state path (support list kept
    across the rotations, the adjoint's phi side sparse) and, with a tiny
    capacity, through its overflow fallback: energy, gradient and state
    against the oracle; then a shorter ansatz on the same driver (the lists
    of the longer one must be cleared)."""
    import oracle.adapt as oadapt
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = system(*cfg)
    opd = ref.pool()
    ops, th = _ansatz(ref, 11, 8)
    ad = hy.Adapt(ham, pool, "f64", max_iter=16, sparse=True,
                  sparse_cap=ham.n_det if cap == "all" else 3)
    for length in (8, 8, 3):
        o, t = ops[:length], th[:length] + 0.05 * length
        ad.set_ansatz(o, t)
        e, g = ad.evaluate(t)
        e_ref, g_ref = oadapt.energy_and_gradient(ref, opd, o, t)
        assert abs(e - e_ref) < 1e-10
        assert np.abs(g - g_ref).max() < 1e-9
        psi = ad.state().cpu().numpy()
        assert np.abs(psi - oadapt.prepare(ref, opd, o, t)).max() < 1e-12


@pytest.mark.parametrize("cfg", [(7, 4, 3, 77), (8, 4, 4, 1005)])
def test_support_program_reuse(cfg):
    """One ansatz evaluated at several angles and in both precisions: the
    first double evaluation lists the support and compiles it, the later ones
    (new angles, then float, then double again) run on the compiled pairings;
    every energy and gradient against the oracle."""
    import oracle.adapt as oadapt
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = system(*cfg)
    opd = ref.pool()
    ops, th = _ansatz(ref, 21, 7)
    ad = hy.Adapt(ham, pool, "mixed", max_iter=16, sparse=True, sparse_cap=ham.n_det)
    ad.set_ansatz(ops, th)
    rng = np.random.default_rng(4)
    for dt in (torch.float64, torch.float64, torch.float32, torch.float32, torch.float64):
        t = th + rng.normal(0, 0.3, len(th))
        e, g = ad.evaluate(t, dt)
        e_ref, g_ref = oadapt.energy_and_gradient(ref, opd, ops, t)
        if dt == torch.float64:
            assert abs(e - e_ref) < 1e-10
            assert np.abs(g - g_ref).max() < 1e-9
        else:
            assert abs(e - e_ref) < 2e-6 * max(1.0, abs(e_ref))
            assert np.abs(g - g_ref).max() < 1e-4 * max(1.0, np.abs(g_ref).max())
        psi = ad.state(dt).double().cpu().numpy()
        tol = 1e-12 if dt == torch.float64 else 1e-5
        assert np.abs(psi - oadapt.prepare(ref, opd, ops, t)).max() < tol


@pytest.mark.parametrize("cfg", [(6, 3, 3, 1001), (8, 4, 4, 1005)])
def test_sparse_state_float_evaluation(cfg):
    """Float sparse evaluation (support renormalised in double) against the
    dense float evaluation and the oracle."""
    import oracle.adapt as oadapt
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = system(*cfg)
    opd = ref.pool()
    ops, th = _ansatz(ref, 5, 6)
    sp = hy.Adapt(ham, pool, "mixed", max_iter=16, sparse=True, sparse_cap=ham.n_det)
    de = hy.Adapt(ham, pool, "mixed", max_iter=16)
    sp.set_ansatz(ops, th)
    de.set_ansatz(ops, th)
    e_s, g_s = sp.evaluate(th, torch.float32)
    e_d, g_d = de.evaluate(th, torch.float32)
    e_ref, g_ref = oadapt.energy_and_gradient(ref, opd, ops, th)
    scale = max(1.0, abs(e_ref))
    assert abs(e_s - e_ref) < 2e-6 * scale and abs(e_d - e_ref) < 2e-6 * scale
    assert np.abs(g_s - g_ref).max() < 1e-4 * max(1.0, np.abs(g_ref).max())
    assert np.abs(g_s - g_d).max() < 1e-4 * max(1.0, np.abs(g_ref).max())
    psi = sp.state(torch.float32).double().cpu().numpy()
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-6
    assert np.abs(psi - oadapt.prepare(ref, opd, ops, th)).max() < 1e-5


def test_sparse_state_full_size_against_dense():
    """28 qubits: the sparse-state evaluation of a 6-operator ansatz against
    the dense sweeps (double: 1e-10 energy, 1e-9 gradient) and its support
    against the nonzeros of the dense state."""
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = system(14, 7, 7, 1003)
    ops, th = _ansatz(ref, 9, 6)
    sp = hy.Adapt(ham, pool, "f64", max_iter=8, sparse=True)
    de = hy.Adapt(ham, pool, "f64", max_iter=8)
    sp.set_ansatz(ops, th)
    de.set_ansatz(ops, th)
    e_s, g_s = sp.evaluate(th)
    e_d, g_d = de.evaluate(th)
    assert abs(e_s - e_d) < 1e-10
    assert np.abs(g_s - g_d).max() < 1e-9
    ps, pd = sp.state(), de.state()
    assert torch.max(torch.abs(ps - pd)).item() < 1e-13


@pytest.mark.parametrize("cfg,dt", [((8, 4, 4, 1005), torch.float64), ((10, 5, 5, 1002), torch.float32),
                                    ((16, 8, 8, 1004), torch.float32)])
def test_touched_weights_from_support(cfg, dt):
    """hy_touched_weights_sparse over a sparse state's support equals the
    dense pass (float rounding of the summation order only)."""
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = system(*cfg)
    psi = torch.from_numpy(prepared(ref, 7, 6)).to("cuda", dt)
    lst, m = support(ham, psi)
    dense = hy.touched_weights(ham, psi)
    sparse = hy.touched_weights_sparse(ham, psi, lst[:m])
    assert torch.max(torch.abs(sparse - dense)).item() <= 2e-6 * dense[0, 0].item()
    assert abs(dense[0, 0].item() - float((psi.double() ** 2).sum().item())) < 1e-5


def _ansatz_with_support(ref, lo, hi, seed0):
    """Ten singles and three other operators whose prepared support has
    between lo and hi determinants (searched over seeds, the support
    counted by the oracle; singles spread the state fastest)."""
    import oracle.adapt as oadapt
    opd = ref.pool()
    singles = [k for k, op in enumerate(opd) if op[1] == 1]
    for seed in range(seed0, seed0 + 200):
        rng = np.random.default_rng(seed)
        ops = [int(k) for k in rng.choice(singles, 10)] + \
            [int(k) for k in rng.integers(0, len(opd), 3)]
        th = rng.uniform(0.1, 0.7, len(ops)) * rng.choice([-1.0, 1.0], len(ops))
        m = int(np.count_nonzero(oadapt.prepare(ref, opd, ops, th)))
        if lo < m <= hi:
            return ops, th, m
    raise AssertionError("no ansatz with the requested support size")


@pytest.mark.parametrize("dt", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_support_program_beyond_shared_memory(dt):
    """20 qubits, an ansatz whose support holds 12,289..63,504 determinants:
    the support program then keeps its vectors in global memory (listing
    order, index map).  Energy, forward gradient and state against the
    oracle at several angles (double 1e-10 / 1e-9 / 1e-12; float 2e-6 /
    1e-4 / 1e-5 relative), and the same evaluations on the dense sweeps."""
    import oracle.adapt as oadapt
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = system(10, 5, 5, 1002)
    opd = ref.pool()
    ops, th, m = _ansatz_with_support(ref, 12288, ham.n_det, 100)
    prec = "f64" if dt == torch.float64 else "mixed"
    ad = hy.Adapt(ham, pool, prec, max_iter=16, sparse=True, sparse_cap=ham.n_det)
    de = hy.Adapt(ham, pool, prec, max_iter=16)
    ad.set_ansatz(ops, th)
    de.set_ansatz(ops, th)
    rng = np.random.default_rng(7)
    for rep in range(3):
        t = th + (0 if rep == 0 else rng.normal(0, 0.2, len(th)))
        e, g = ad.evaluate(t, dt)
        e_d, g_d = de.evaluate(t, dt)
        e_ref, g_ref = oadapt.energy_and_gradient(ref, opd, ops, t)
        psi = ad.state(dt).double().cpu().numpy()
        p_ref = oadapt.prepare(ref, opd, ops, t)
        assert int(np.count_nonzero(p_ref)) == m
        if dt == torch.float64:
            assert abs(e - e_ref) < 1e-10 and abs(e_d - e_ref) < 1e-10
            assert np.abs(g - g_ref).max() < 1e-9
            assert np.abs(psi - p_ref).max() < 1e-12
        else:
            scale = max(1.0, abs(e_ref))
            assert abs(e - e_ref) < 2e-6 * scale
            assert np.abs(g - g_ref).max() < 1e-4 * max(1.0, np.abs(g_ref).max())
            assert np.abs(g - g_d).max() < 1e-4 * max(1.0, np.abs(g_ref).max())
            assert np.abs(psi - p_ref).max() < 1e-5


@pytest.mark.parametrize("dt", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_support_sigma_beyond_programs(dt):
    """24 qubits, an ansatz whose support exceeds the support programs'
    65,536 determinants: from the second evaluation on, sigma is formed on
    psi's support only (rows of the support list against the listed
    determinants, no atomics) and the gradient comes from the reverse sweep
    started on that restricted sigma.  Energy, gradient and state against
    the oracle at several angles (double 1e-10 / 1e-9 / 1e-12; float 2e-6 /
    1e-4 / 1e-5 relative), and the screen that follows (which needs all of
    sigma) against the oracle's screen."""
    import oracle.adapt as oadapt
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = system(12, 6, 6, 1006)
    opd = ref.pool()
    ops, th, m = _ansatz_with_support(ref, 65536, ham.n_det // 4, 300)
    prec = "f64" if dt == torch.float64 else "mixed"
    ad = hy.Adapt(ham, pool, prec, max_iter=16, sparse=True, sparse_cap=ham.n_det)
    ad.set_ansatz(ops, th)
    rng = np.random.default_rng(11)
    for rep in range(3):
        t = th + (0 if rep == 0 else rng.normal(0, 0.2, len(th)))
        e, g = ad.evaluate(t, dt)
        if rep == 0:
            e, g = ad.evaluate(t, dt)      # the support is known: restricted sigma
        e_ref, g_ref = oadapt.energy_and_gradient(ref, opd, ops, t)
        psi = ad.state(dt).double().cpu().numpy()
        p_ref = oadapt.prepare(ref, opd, ops, t)
        assert int(np.count_nonzero(p_ref)) == m
        if dt == torch.float64:
            assert abs(e - e_ref) < 1e-10
            assert np.abs(g - g_ref).max() < 1e-9
            assert np.abs(psi - p_ref).max() < 1e-12
        else:
            scale = max(1.0, abs(e_ref))
            assert abs(e - e_ref) < 2e-6 * scale
            assert np.abs(g - g_ref).max() < 1e-4 * max(1.0, np.abs(g_ref).max())
            assert np.abs(psi - p_ref).max() < 1e-5
    if dt == torch.float64:
        # one ADAPT step from this ansatz: its screen reads all of sigma
        ad.set_ansatz(ops, th)
        r = ad.step()
        p_ref = oadapt.prepare(ref, opd, ops, th)
        g_scr = ref.gradients(opd, p_ref, ref.sigma(p_ref))
        best = np.abs(g_scr)
        assert r["selected"] == int(np.argmax(best)) or \
            best[r["selected"]] >= best.max() * (1 - 1e-9)
        assert abs(r["max_grad"] - best.max()) < 1e-9


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_support_rows_match_dense_sweeps_28q(prec):
    """28 qubits (11,778,624 determinants), the ansatz of 11 plain ADAPT
    iterations from Hartree-Fock (support > 65,536): energy and gradient from
    the sparse path (sigma on the support's rows, reverse sweep kept on the
    support) against the dense sweeps at perturbed angles (double 1e-10 /
    1e-9; float 2e-6 / 1e-4 relative)."""
    import paper_2604_01176_gb300 as hy
    n, na, nb, seed = synth.workload("h14_28q")
    h1, h2, ec = synth.integrals(n, seed)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    pool = hy.Pool(ham)
    plain = hy.Adapt(ham, pool, "f64", max_iter=12, sparse=True)
    recs = plain.run(11)
    assert recs[-1]["support"] > 65536
    ops, th = plain.ansatz()
    plain.close()
    dt = torch.float64 if prec == "f64" else torch.float32
    sp = hy.Adapt(ham, pool, prec, max_iter=12, sparse=True)
    de = hy.Adapt(ham, pool, prec, max_iter=12)
    sp.set_ansatz(list(ops), list(th))
    de.set_ansatz(list(ops), list(th))
    rng = np.random.default_rng(5)
    th = np.array(th)
    for rep in range(2):
        t = th + (0 if rep == 0 else rng.normal(0, 0.05, len(th)))
        e_s, g_s = sp.evaluate(t, dt)
        e_s, g_s = sp.evaluate(t, dt)             # the support is known: rows only
        e_d, g_d = de.evaluate(t, dt)
        if prec == "f64":
            assert abs(e_s - e_d) < 1e-10
            assert np.abs(g_s - g_d).max() < 1e-9
        else:
            assert abs(e_s - e_d) < 2e-6 * abs(e_d)
            assert np.abs(g_s - g_d).max() < 1e-4 * max(1.0, np.abs(g_d).max())
    sp.close()
    de.close()
    pool.close()
    ham.close()
