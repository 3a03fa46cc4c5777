"""GPU parity of the batched persistent launch (hy_batch_*): every molecule
of an uneven batch against the FP64 oracle, the CUDA-graph replay against
the direct launch, and the autotuner's choice against correctness.

Tolerances: FP64 amplitudes 1e-12 max-abs, energies 1e-10 Ha; FP32 sigma
2e-5 * max|sigma| (the same bound as the single-molecule sweep); graph
replay and direct launch bit-identical.
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


MOLS = [(6, 3, 3, 2000), (8, 4, 4, 2001), (5, 3, 2, 2002), (7, 4, 3, 2003), (10, 5, 5, 2004),
        (4, 2, 2, 2005), (9, 5, 4, 2006), (1, 1, 0, 2007), (3, 0, 2, 2008)]


@pytest.fixture(scope="module")
def batch():
    import paper_2604_01176_gb300 as hy
    refs, hams = [], []
    for n, na, nb, seed in MOLS:
        h1, h2, ec = synth.integrals(n, seed)
        refs.append(oracle.System(h1, h2, ec, n, na, nb))
        hams.append(hy.Hamiltonian(h1, h2, ec, n, na, nb))
    return refs, hams, hy.Batch(hams)


def test_offsets_and_packing(batch):
    refs, hams, b = batch
    assert b.offsets[0] == 0 and np.all(b.offsets % 32 == 0)
    assert np.all(np.diff(b.offsets) >= [r.n_det for r in refs])
    assert b.n_tasks == sum(r.n_astr for r in refs)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_matches_oracle(batch, dtype):
    refs, hams, b = batch
    states = [synth.random_state(r.n_det, 40 + i) for i, r in enumerate(refs)]
    if dtype == torch.float32:
        states = [s.astype(np.float32).astype(np.float64) for s in states]
    psi = b.pack([torch.from_numpy(s) for s in states], dtype)
    e = torch.empty(len(refs), dtype=torch.float64, device="cuda")
    sig = b.unpack(b.apply_h(psi, energies=e))
    e = e.cpu().numpy()
    for i, r in enumerate(refs):
        ref = r.sigma(states[i])
        got = sig[i].double().cpu().numpy()
        if dtype == torch.float64:
            assert np.abs(got - ref).max() < 1e-12
            assert abs(e[i] - float(states[i] @ ref)) < 1e-10
        else:
            assert np.abs(got - ref).max() <= 2e-5 * max(np.abs(ref).max(), 1e-30)
            assert abs(e[i] - float(states[i] @ ref)) < 1e-5 * max(1.0, abs(float(states[i] @ ref)))


def test_graph_replay_and_tuning(batch):
    refs, hams, b = batch
    states = [synth.random_state(r.n_det, 60 + i) for i, r in enumerate(refs)]
    psi = b.pack([torch.from_numpy(s) for s in states])
    s1 = torch.zeros_like(psi)     # padding between molecules is never written
    s2 = torch.zeros_like(psi)
    e1 = torch.empty(len(refs), dtype=torch.float64, device="cuda")
    e2 = torch.empty_like(e1)
    b.apply_h(psi, s1, e1)
    for _ in range(2):           # capture on the first call, replay on the second
        b.apply_h(psi, s2, e2, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2) and torch.equal(e1, e2)
    tile, ms = b.tune(psi, s2)
    assert ms > 0 and tile["gsize"] * tile["groups"] <= 1024
    assert b.tile == tile
    b.apply_h(psi, s2, e2, graph=True)     # re-captured for the new tile
    torch.cuda.synchronize()
    # per-element sums do not depend on the tile: sigma is bit-identical
    assert torch.equal(s1, s2)
    assert torch.allclose(e1, e2, rtol=0, atol=1e-12)
    for gsize, groups in [(32, 1), (32, 15), (128, 8), (1024, 1)]:
        b.set_tile(gsize, groups)
        s3 = b.apply_h(psi, torch.zeros_like(psi))
        torch.cuda.synchronize()
        assert torch.equal(s1, s3)


def test_batch_matches_single_molecule_path(batch):
    refs, hams, b = batch
    states = [synth.random_state(r.n_det, 80 + i) for i, r in enumerate(refs)]
    psi = b.pack([torch.from_numpy(s) for s in states])
    sig = b.unpack(b.apply_h(psi))
    for i, h in enumerate(hams):
        single = h.apply_h(torch.from_numpy(states[i]).cuda())
        assert torch.max(torch.abs(single - sig[i])).item() < 1e-13


def _lists(pools, rng):
    """Per molecule a random subset of its pool in random order, packed."""
    ops, offs = [], [0]
    for p in pools:
        K = len(p)
        sel = rng.permutation(K)[: max(0, K // 3)] if K else np.zeros(0, dtype=np.int64)
        ops.extend(int(k) for k in sel)
        offs.append(len(ops))
    return np.array(ops, dtype=np.int32), np.array(offs, dtype=np.int64)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_gradients_match_oracle_and_lists(batch, dtype):
    """The batched screen (hy_batch_gradients): every molecule's full screen
    against the oracle's gradients of the same state (FP64 1e-11, FP32 1e-4
    relative to max(1, max|g|)), per-molecule operator lists against the
    full screen (1e-13 / 1e-6 relative: only the chunking of the sums
    differs), and
    an out-of-range list entry: NaN in its slot, reported by the next call."""
    import paper_2604_01176_gb300 as hy
    refs, hams, b = batch
    pools = [hy.Pool(h) for h in hams]
    b.set_pools(pools)
    K = [len(p) for p in pools]
    assert np.array_equal(np.diff(b.pool_offsets), K)
    states = [synth.random_state(r.n_det, 60 + i) for i, r in enumerate(refs)]
    if dtype == torch.float32:
        states = [s.astype(np.float32).astype(np.float64) for s in states]
    psi = b.pack([torch.from_numpy(s) for s in states], dtype)
    sig = b.apply_h(psi)
    g = b.gradients(psi, sig).cpu().numpy()
    off = b.pool_offsets
    for i, r in enumerate(refs):
        if K[i] == 0:
            continue
        ref = r.gradients(r.pool(), states[i], r.sigma(states[i]))
        got = g[off[i]:off[i + 1]]
        tol = 1e-11 if dtype == torch.float64 else 1e-4
        assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max()), i
    # lists against the full screen: only the chunking of the sums differs
    # (FP32 sums: float rounding)
    ltol = 1e-13 if dtype == torch.float64 else 1e-6
    rng = np.random.default_rng(3)
    ops, offs = _lists(pools, rng)
    O = torch.from_numpy(ops).cuda()
    OF = torch.from_numpy(offs).cuda()
    gl = b.gradients(psi, sig, ops=O, op_offsets=OF).cpu().numpy()
    for i in range(len(refs)):
        sub = ops[offs[i]:offs[i + 1]]
        if sub.size == 0:
            continue
        want = g[off[i] + sub]
        assert np.abs(gl[offs[i]:offs[i + 1]] - want).max() <= ltol * max(1.0, np.abs(g).max())
    # an index one past molecule m's pool
    m = int(np.argmax(K))
    bad = ops.copy()
    bad[offs[m]] = K[m]
    gb = b.gradients(psi, sig, ops=torch.from_numpy(bad).cuda(), op_offsets=OF).cpu().numpy()
    assert np.isnan(gb[offs[m]])
    with pytest.raises(hy.HyError):
        b.gradients(psi, sig, ops=O, op_offsets=OF)
    gl2 = b.gradients(psi, sig, ops=O, op_offsets=OF).cpu().numpy()   # the report is cleared
    assert np.abs(gl2 - gl).max() <= ltol * max(1.0, np.abs(g).max())
