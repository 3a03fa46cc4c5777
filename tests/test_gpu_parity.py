"""GPU parity: every sweep of the CUDA path against the FP64 CPU oracle on the
same seeded inputs, through the C ABI (Python binding = marshalling only).

Tolerances (stated per test):
* FP64: amplitudes max-abs 1e-12, energies 1e-10 Ha, gradients 1e-11;
* indices: bit-exact;
* FP32 (float amplitudes, float accumulation): |err| <= 2e-5 * max|ref|
  elementwise for sigma (at most ~6k terms per element, each rounded at
  2^-24 relative, accumulated in chunks of <= 65); energies and gradients
  are accumulated in double from float products: 1e-5 relative.
"""
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


SMALL = [(6, 3, 3, 1001), (7, 4, 3, 77), (8, 4, 4, 1005), (5, 1, 4, 12),
         (4, 0, 2, 5), (3, 3, 1, 9), (1, 1, 0, 3), (10, 5, 5, 1002)]
IDS = [f"n{c[0]}a{c[1]}b{c[2]}" for c in SMALL]


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


# --------------------------------------------------------------------------
# determinant indexing
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", SMALL, ids=IDS)
def test_rank_unrank_bit_exact(cfg):
    ref, ham, _ = system(*cfg)
    dets = ref.dets()
    d = torch.from_numpy(dets.view(np.int64)).cuda()
    idx = ham.rank(d)
    assert torch.equal(idx.cpu(), torch.arange(ref.n_det, dtype=torch.int64))
    back = ham.unrank(idx)
    assert np.array_equal(back.cpu().numpy().view(np.uint64), dets)


def test_rank_rejects_outside_sector():
    ref, ham, _ = system(6, 3, 3, 1001)
    bad = np.array([0, 0b111, (0b111 << 6) | 0b1111, 1 << 12 | 0b111 | (0b111 << 6),
                    0b1011 | (0b11 << 6)], dtype=np.uint64)
    idx = ham.rank(torch.from_numpy(bad.view(np.int64)).cuda()).cpu().numpy()
    assert np.all(idx == -1)
    out = ham.unrank(torch.tensor([-1, ref.n_det, 10**12], dtype=torch.int64).cuda())
    assert torch.all(out.cpu() == 0)


@pytest.mark.parametrize("n", [14, 16])
def test_rank_large_sampled(n):
    """28 / 32 qubits: sampled indices, oracle determinant -> GPU rank."""
    ref, ham, _ = system(n, n // 2, n // 2, 1003 if n == 14 else 1004)
    rng = np.random.default_rng(n)
    I = np.concatenate([[0, ref.n_det - 1], rng.integers(0, ref.n_det, 4000)])
    dets = np.array([oracle._load().orc_det(ref._h, int(i)) for i in I], dtype=np.uint64)
    idx = ham.rank(torch.from_numpy(dets.view(np.int64)).cuda()).cpu().numpy()
    assert np.array_equal(idx, I)
    back = ham.unrank(torch.from_numpy(I.astype(np.int64)).cuda()).cpu().numpy()
    assert np.array_equal(back.view(np.uint64), dets)


# --------------------------------------------------------------------------
# sigma = H psi, energies, dots
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", SMALL, ids=IDS)
def test_apply_h_f64(cfg):
    ref, ham, _ = system(*cfg)
    for seed in (1, 2):
        psi = synth.random_state(ref.n_det, seed)
        s_ref = ref.sigma(psi)
        s = ham.apply_h(cuda(psi)).cpu().numpy()
        assert np.abs(s - s_ref).max() <= 1e-12


@pytest.mark.parametrize("cfg", SMALL, ids=IDS)
def test_apply_h_f32(cfg):
    ref, ham, _ = system(*cfg)
    psi = synth.random_state(ref.n_det, 3)
    psi32 = psi.astype(np.float32)
    s_ref = ref.sigma(psi32.astype(np.float64))
    s = ham.apply_h(cuda(psi32, torch.float32)).cpu().numpy().astype(np.float64)
    assert np.abs(s - s_ref).max() <= 2e-5 * max(np.abs(s_ref).max(), 1e-30)


def test_apply_h_hf_column_and_sparse_state():
    """H applied to the HF determinant = the HF column of the dense H; a
    state with only a few nonzero amplitudes (the paper's sparse regime)."""
    ref, ham, _ = system(6, 3, 3, 1001)
    Hd = ref.dense_h()
    e = np.zeros(ref.n_det); e[0] = 1.0
    assert np.abs(ham.apply_h(cuda(e)).cpu().numpy() - Hd[:, 0]).max() < 1e-13
    v = np.zeros(ref.n_det); v[[0, 17, 399]] = [0.6, -0.8, 0.1]
    assert np.abs(ham.apply_h(cuda(v)).cpu().numpy() - Hd @ v).max() < 1e-13


@pytest.mark.parametrize("cfg", SMALL[:3], ids=IDS[:3])
def test_energy_dot_normalize(cfg):
    ref, ham, _ = system(*cfg)
    x = synth.random_state(ref.n_det, 4, normalise=False)
    y = synth.random_state(ref.n_det, 5, normalise=False)
    X, Y = cuda(x), cuda(y)
    e_ref = float(x @ ref.sigma(x))
    assert abs(ham.energy(X).item() - e_ref) < 1e-10 * max(1, abs(e_ref))
    assert abs(ham.energy(X, ham.apply_h(X)).item() - e_ref) < 1e-10 * max(1, abs(e_ref))
    assert abs(ham.dot(X, Y).item() - float(x @ y)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)
    ham.normalize(X)
    assert np.abs(X.cpu().numpy() - x / np.linalg.norm(x)).max() < 1e-15
    x32 = x.astype(np.float32)
    e32 = ham.energy(cuda(x32, torch.float32)).item()
    e32_ref = float(x32.astype(np.float64) @ ref.sigma(x32.astype(np.float64)))
    assert abs(e32 - e32_ref) < 1e-5 * abs(e32_ref)


def test_fci_ground_state_energy():
    """The oracle's dense ground state pushed through the GPU H: the energy
    equals E_FCI and sigma = E_FCI psi (eigen-equation residual)."""
    ref, ham, _ = system(6, 3, 3, 1001)
    w, V = np.linalg.eigh(ref.dense_h())
    v = cuda(V[:, 0])
    assert abs(ham.energy(v).item() - w[0]) < 1e-10
    assert np.abs(ham.apply_h(v).cpu().numpy() - w[0] * V[:, 0]).max() < 1e-12


# --------------------------------------------------------------------------
# pool, gradients, exp(theta A)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", SMALL, ids=IDS)
def test_pool_matches_oracle(cfg):
    ref, _, pool = system(*cfg)
    assert np.array_equal(pool.descriptors(), ref.pool())


def correlated_state(ref, seed):
    pool = ref.pool()
    psi = ref.hf_state()
    rng = np.random.default_rng(seed)
    if len(pool) == 0:
        return synth.random_state(ref.n_det, seed)
    for k in rng.integers(0, len(pool), 6):
        psi = ref.apply_excitation(pool[k], rng.normal(0, 0.3), psi)
    return psi


@pytest.mark.parametrize("cfg", SMALL[:7], ids=IDS[:7])
def test_gradients_f64_full_screen_and_subset(cfg):
    ref, ham, pool = system(*cfg)
    if len(pool) == 0:
        pytest.skip("empty pool")
    for psi in (correlated_state(ref, 1), synth.random_state(ref.n_det, 8)):
        sig = ref.sigma(psi)
        g_ref = ref.gradients(ref.pool(), psi, sig)
        P, S = cuda(psi), cuda(sig)
        g = pool.gradients(P, S).cpu().numpy()
        assert np.abs(g - g_ref).max() < 1e-11
        sub = np.array([len(pool) - 1, 0, len(pool) // 2, 0], dtype=np.int32)
        gs = pool.gradients(P, S, ops=torch.from_numpy(sub).cuda()).cpu().numpy()
        assert np.abs(gs - g_ref[sub]).max() < 1e-11


def test_gradients_f32():
    ref, ham, pool = system(8, 4, 4, 1005)
    psi = correlated_state(ref, 2).astype(np.float32).astype(np.float64)
    sig = ref.sigma(psi)
    g_ref = ref.gradients(ref.pool(), psi, sig)
    g = pool.gradients(cuda(psi, torch.float32), cuda(sig, torch.float32)).cpu().numpy()
    assert np.abs(g - g_ref).max() < 1e-5 * np.abs(g_ref).max()


def test_gradient_equals_energy_derivative_on_gpu():
    """g_k from the screen equals the central difference of the GPU energy
    of exp(+-h A_k) psi (property that holds at any size)."""
    ref, ham, pool = system(8, 4, 4, 1005)
    psi = cuda(correlated_state(ref, 3))
    g = pool.gradients(psi, ham.apply_h(psi)).cpu().numpy()
    h = 1e-4
    for k in range(0, len(pool), 29):
        p1, p2 = psi.clone(), psi.clone()
        pool.apply_excitation(k, h, p1)
        pool.apply_excitation(k, -h, p2)
        fd = (ham.energy(p1).item() - ham.energy(p2).item()) / (2 * h)
        assert abs(fd - g[k]) < 1e-7


@pytest.mark.parametrize("cfg", SMALL[:7], ids=IDS[:7])
def test_excitation_f64_every_op(cfg):
    ref, ham, pool = system(*cfg)
    opd = ref.pool()
    psi = synth.random_state(ref.n_det, 6)
    P = cuda(psi)
    step = max(1, len(opd) // 60)
    for k in range(0, len(opd), step):
        theta = 0.1 + 0.37 * k / max(1, len(opd))
        out = P.clone()
        pool.apply_excitation(k, theta, out)
        exp = ref.apply_excitation(opd[k], theta, psi)
        assert np.abs(out.cpu().numpy() - exp).max() < 1e-12


def test_excitation_f32_renormalize():
    ref, ham, pool = system(8, 4, 4, 1005)
    opd = ref.pool()
    psi = synth.random_state(ref.n_det, 7)
    P = cuda(psi, torch.float32)
    exp = psi.copy()
    for k, t in [(3, 0.4), (200, -0.9), (len(opd) - 1, 1.3)]:
        pool.apply_excitation(k, t, P, renormalize=True)
        exp = ref.apply_excitation(opd[k], t, exp)
    got = P.cpu().numpy().astype(np.float64)
    assert abs(np.linalg.norm(got) - 1.0) < 1e-6
    assert np.abs(got - exp).max() < 1e-6


def test_state_preparation_sequence_f64():
    """Ansatz prepared from HF by a sequence of exp(theta A) equals the oracle."""
    ref, ham, pool = system(10, 5, 5, 1002)
    opd = ref.pool()
    rng = np.random.default_rng(5)
    ks = rng.integers(0, len(opd), 8)
    th = rng.normal(0, 0.4, 8)
    psi = ham.hf_state()
    exp = ref.hf_state()
    for k, t in zip(ks, th):
        pool.apply_excitation(int(k), float(t), psi)
        exp = ref.apply_excitation(opd[k], t, exp)
    assert np.abs(psi.cpu().numpy() - exp).max() < 1e-12
    e_ref = float(exp @ ref.sigma(exp))
    assert abs(ham.energy(psi).item() - e_ref) < 1e-10


# --------------------------------------------------------------------------
# full-size workloads (28 and 32 qubits): sampled rows and properties
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,seed", [(14, 1003), (16, 1004)])
def test_apply_h_full_size_sampled(n, seed):
    ref, ham, pool = system(n, n // 2, n // 2, seed)
    psi = synth.random_state(ref.n_det, 11)
    P = cuda(psi)
    S = ham.apply_h(P)
    rng = np.random.default_rng(n)
    rows = np.unique(np.concatenate([[0, ref.n_det - 1],
                                     rng.integers(0, ref.n_det, 48)]))
    s_ref = ref.sigma_rows(psi, rows)
    got = S[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.abs(got - s_ref).max() < 1e-12
    # energy: the fused call (sigma computed inside) against a host dot
    e = ham.energy(P).item()
    assert abs(e - float(np.dot(psi, S.cpu().numpy()))) < 1e-10
    # FP32 sweep on the same rows
    S32 = ham.apply_h(P.float())
    s32_ref = ref.sigma_rows(psi.astype(np.float32).astype(np.float64), rows)
    got32 = S32[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert np.abs(got32 - s32_ref).max() <= 2e-5 * np.abs(s32_ref).max()
    del S32
    # Hermiticity at full size: <phi|H psi> = <H phi|psi>
    phi = cuda(synth.random_state(ref.n_det, 12))
    lhs = ham.dot(phi, S).item()
    rhs = ham.dot(ham.apply_h(phi), P).item()
    assert abs(lhs - rhs) < 1e-10


@pytest.mark.parametrize("n,seed", [(14, 1003), (16, 1004)])
def test_sweeps_full_size_sparse_state(n, seed):
    """Full-size workloads on a state a few excitations away from HF (the
    paper's sparse early-iteration regime): the prepared amplitudes, the
    energy and sampled gradients all against the oracle, which only needs
    sigma on the few determinants the state and A_k psi touch."""
    ref, ham, pool = system(n, n // 2, n // 2, seed)
    opd = ref.pool()
    steps = [(0, 0.3), (len(opd) - 1, -0.2), (len(opd) // 2, 0.25)]
    psi = ref.hf_state()
    P = ham.hf_state()
    for k, t in steps:
        psi = ref.apply_excitation(opd[k], t, psi)
        pool.apply_excitation(k, t, P)
    assert np.abs(P.cpu().numpy() - psi).max() < 1e-12
    S = ham.apply_h(P)
    sup = np.nonzero(psi)[0]
    e_ref = float(psi[sup] @ ref.sigma_rows(psi, sup))
    assert abs(ham.energy(P, S).item() - e_ref) < 1e-10
    g = pool.gradients(P, S).cpu().numpy()
    for k in (1, len(opd) // 3, len(opd) - 2):
        t = ref.apply_generator(opd[k], psi)
        rows = np.nonzero(t)[0]
        g_ref = 2.0 * float(t[rows] @ ref.sigma_rows(psi, rows)) if len(rows) else 0.0
        assert abs(g[k] - g_ref) < 1e-11


def test_tracked_excitations_and_renormalisation():
    """hy_apply_excitation_tracked: the tracked squared norm equals the FP64
    norm of the rotated float state, and one hy_renormalize after the
    product equals the oracle's normalised product."""
    import paper_2604_01176_gb300 as hy
    h1, h2, ec = synth.integrals(8, 1005)
    ref = oracle.System(h1, h2, ec, 8, 4, 4)
    ham = hy.Hamiltonian(h1, h2, ec, 8, 4, 4)
    pool = hy.Pool(ham)
    opd = ref.pool()
    rng = np.random.default_rng(21)
    ops, th = rng.integers(0, len(opd), 9), rng.normal(0, 0.6, 9)
    for dt, tol in ((torch.float32, 2e-6), (torch.float64, 1e-13)):
        psi = torch.zeros(ham.n_det, dtype=dt, device="cuda")
        psi[0] = 1.0
        n2 = torch.ones((), dtype=torch.float64, device="cuda")
        for k, t in zip(ops, th):
            pool.apply_excitation_tracked(int(k), float(t), psi, n2)
        direct = float((psi.double() ** 2).sum().item())
        assert abs(n2.item() - direct) < 1e-13 * direct
        ham.renormalize(psi, n2)
        want = ref.hf_state()
        for k, t in zip(ops, th):
            want = ref.apply_excitation(opd[k], t, want)
        assert np.abs(psi.double().cpu().numpy() - want).max() < tol


def test_float_dot_is_fp64_accurate():
    """Float inner products (Dot2 runs flushed into FP64) against the exact
    FP64 dot of the same float values: aligned and unaligned inputs, a ragged
    tail, and products near the FP32 overflow threshold."""
    import paper_2604_01176_gb300 as hy
    h1, h2, ec = synth.integrals(6, 1001)
    ham = hy.Hamiltonian(h1, h2, ec, 6, 3, 3)
    g = torch.Generator().manual_seed(5)
    N = ham.n_det
    base = torch.randn(2 * N + 3, generator=g, dtype=torch.float32).cuda()
    for off in (0, 1, 3):       # device views 4 * off bytes past a 16-byte boundary
        x = base[off:off + N]
        y = base[N + 3 - off:2 * N + 3 - off]
        xd, yd = x.cpu().double().numpy(), y.cpu().double().numpy()
        want = float(np.dot(xd, yd))
        got = float(ham.dot(x, y).item())
        assert abs(got - want) <= 1e-13 * float(np.abs(xd * yd).sum())
    big = torch.full((N,), 1e19, dtype=torch.float32, device="cuda")
    got = float(ham.dot(big, big).item())
    want = N * float(np.float32(1e19)) ** 2
    assert abs(got - want) <= 1e-12 * want


def test_kernel_class_profiler():
    """hy_profile_*: enabled classes count their launches, device time and
    algorithmic bytes; disabled classes record nothing."""
    import paper_2604_01176_gb300 as hy
    h1, h2, ec = synth.integrals(8, 1005)
    ham = hy.Hamiltonian(h1, h2, ec, 8, 4, 4)
    pool = hy.Pool(ham)
    psi = torch.zeros(ham.n_det, dtype=torch.float32, device="cuda")
    psi[0] = 1.0
    hy.profile_enable(["excite", "reduce"])
    pool.apply_excitation(len(pool) - 1, 0.3, psi)
    ham.dot(psi, psi)
    ham.apply_h(psi)
    torch.cuda.synchronize()
    ex, red, hp = hy.profile_read("excite"), hy.profile_read("reduce"), hy.profile_read("hpsi")
    hy.profile_enable([])
    assert ex["launches"] >= 1 and ex["ms"] > 0 and ex["bytes"] > 0
    assert red["launches"] == 1 and red["bytes"] == 2.0 * ham.n_det * 4
    assert hp["launches"] == 0 and hp["ms"] == 0


@pytest.mark.parametrize("cfg", [(7, 4, 3, 77), (10, 5, 5, 1002), (14, 7, 7, 1003)],
                         ids=["n7a4b3", "n10", "n14"])
def test_f32_coupling_tensor_cores_match_simt(cfg):
    """Float H|psi> with the coupling's dense phase on the tensor cores
    (TF32 MMAs on split hi/lo operands) against the same sweep on the FP32
    SIMT pipes and, on sampled rows, against the oracle: ragged column
    tiles (N_beta = 35, 252, 3432), odd orbital counts, several tiles per
    string."""
    ref, ham, _ = system(*cfg)
    psi = synth.random_state(ref.n_det, 5).astype(np.float32)
    P = cuda(psi, torch.float32)
    ham.set_coupling("simt")
    S_simt = ham.apply_h(P)
    ham.set_coupling("tensor")
    S_tc = ham.apply_h(P)
    scale = torch.max(torch.abs(S_simt)).item()
    assert torch.max(torch.abs(S_tc - S_simt)).item() <= 2e-5 * scale
    rng = np.random.default_rng(cfg[0])
    rows = np.unique(np.concatenate([[0, ref.n_det - 1], rng.integers(0, ref.n_det, 64)]))
    s_ref = ref.sigma_rows(psi.astype(np.float64), rows)
    got = S_tc[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert np.abs(got - s_ref).max() <= 2e-5 * np.abs(s_ref).max()
