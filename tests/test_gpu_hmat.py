"""The Hamiltonian stored explicitly (hy_hmat_*) against the FP64 oracle: the
paper assembles H over Omega_CIk as a sparse matrix and distributes its rows
(Sparse State-Vector Emulation section; Table 1 lists its size).

* Structure, bit-exact: the stored columns of a row are exactly the
  determinants within two electron moves of it (the nonzero pattern of a
  two-body H), each once; the row length is 1 + s_a + s_b + d_a + d_b +
  s_a s_b.
* Values: every stored element equals the oracle's Slater-Condon element
  <bra|H|ket> (FP64 1e-12; FP32 the same value rounded once, 2^-24 relative).
* H psi over it: FP64 within 1e-12 of the oracle's sigma (full range and row
  ranges), FP32 within 2e-5 * max|sigma| (float accumulation of <= 6k terms);
  at 24 and 28 qubits against the matrix-free sweep (same tolerances) and
  the oracle on sampled rows.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = [(6, 3, 3, 1001), (7, 4, 3, 77), (8, 4, 4, 1005), (5, 1, 4, 12), (4, 0, 2, 5),
         (3, 3, 1, 9), (10, 5, 5, 1002)]
IDS = [f"n{c[0]}a{c[1]}b{c[2]}" for c in SMALL]


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
        _CACHE[key] = (oracle.System(h1, h2, ec, n, na, nb), hy.Hamiltonian(h1, h2, ec, n, na, nb))
    return _CACHE[key]


def row_length(n, na, nb):
    s = lambda k: k * (n - k)
    d = lambda k: math.comb(k, 2) * math.comb(n - k, 2)
    return 1 + s(na) + s(nb) + d(na) + d(nb) + s(na) * s(nb)


def within_two_moves(ref, det):
    """Brute force: every determinant of Omega_CIk that differs from det by
    at most two electrons (popcount of the XOR <= 4)."""
    dets = ref.dets()
    x = np.bitwise_xor(dets.astype(np.uint64), np.uint64(det))
    pc = np.array([bin(int(v)).count("1") for v in x])
    return set(np.flatnonzero(pc <= 4).tolist())


@pytest.mark.parametrize("cfg", SMALL, ids=IDS)
@pytest.mark.parametrize("dt", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_stored_rows_structure_and_values(cfg, dt):
    import paper_2604_01176_gb300 as hy
    ref, ham = system(*cfg)
    n, na, nb, _ = cfg
    m = hy.ExplicitH(ham, dt)
    w = row_length(n, na, nb)
    assert m.row_len == w and m.nnz == ham.n_det * w
    nbp = (ham.n_beta_str + 7) // 8 * 8
    S = 1 + na * (n - na) + math.comb(na, 2) * math.comb(n - na, 2)
    assert m.bytes == ham.n_alpha_str * (2 * S + w * nbp * (2 + (8 if dt == torch.float64 else 4)))
    dets = ref.dets()
    rng = np.random.default_rng(cfg[0])
    rows = np.unique(np.concatenate([[0, ham.n_det - 1], rng.integers(0, ham.n_det, 12)]))
    for r in rows:
        cols, vals = m.row(int(r))
        assert len(cols) == w and len(set(cols.tolist())) == w            # each column once
        assert set(cols.tolist()) == within_two_moves(ref, int(dets[r]))  # bit-exact pattern
        exact = np.array([ref.matrix_element(int(dets[r]), int(dets[c])) for c in cols])
        if dt == torch.float64:
            assert np.abs(vals - exact).max() < 1e-12
        else:
            assert np.array_equal(vals, exact.astype(np.float32).astype(np.float64)) or \
                np.abs(vals - exact).max() <= 2.0 ** -23 * max(1.0, np.abs(exact).max())


@pytest.mark.parametrize("cfg", SMALL, ids=IDS)
def test_explicit_h_psi_matches_oracle(cfg):
    import paper_2604_01176_gb300 as hy
    ref, ham = system(*cfg)
    psi = synth.random_state(ham.n_det, 21)
    sig_ref = ref.sigma(psi)
    m64 = hy.ExplicitH(ham, torch.float64)
    got = m64.apply(torch.from_numpy(psi).cuda()).cpu().numpy()
    assert np.abs(got - sig_ref).max() < 1e-12
    m32 = hy.ExplicitH(ham, torch.float32)
    got32 = m32.apply(torch.from_numpy(psi).to("cuda", torch.float32)).double().cpu().numpy()
    assert np.abs(got32 - sig_ref).max() <= 2e-5 * np.abs(sig_ref).max()
    # row ranges: uneven blocks, an empty one, the last row alone
    NA, NB = ham.n_alpha_str, ham.n_beta_str
    for b, e in [(0, NA // 2), (NA // 2, NA), (NA // 3, NA // 3), (NA - 1, NA)]:
        mr = hy.ExplicitH(ham, torch.float64, b, e)
        blk = mr.apply(torch.from_numpy(psi).cuda()).cpu().numpy()
        assert np.abs(blk - sig_ref[b * NB: e * NB]).max() < 1e-12 if e > b else blk.size == 0


def test_explicit_h_24q_against_matrix_free_and_oracle():
    import paper_2604_01176_gb300 as hy
    n, na, nb, seed = synth.workload("h12_24q")
    ref, ham = system(n, na, nb, seed)
    psi = torch.from_numpy(synth.random_state(ham.n_det, 8)).cuda()
    mf = ham.apply_h(psi)
    m = hy.ExplicitH(ham, torch.float64)
    assert m.nnz == ham.n_det * row_length(n, na, nb)
    got = m.apply(psi)
    scale = torch.max(torch.abs(mf)).item()
    assert torch.max(torch.abs(got - mf)).item() <= 1e-12 * max(1.0, scale)
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([[0, ham.n_det - 1], rng.integers(0, ham.n_det, 48)]))
    s_ref = ref.sigma_rows(psi.cpu().numpy(), rows)
    assert np.abs(got[torch.from_numpy(rows).cuda()].cpu().numpy() - s_ref).max() < 1e-12
    del m
    m32 = hy.ExplicitH(ham, torch.float32)
    p32 = psi.float()
    g32 = m32.apply(p32)
    mf32 = ham.apply_h(p32)
    assert torch.max(torch.abs(g32 - mf32)).item() <= 2e-5 * scale


def test_explicit_h_28q_row_block():
    """28 qubits: 96 alpha strings (4.5 GB of float matrix) against the
    matrix-free rows and the oracle on sampled determinants."""
    import paper_2604_01176_gb300 as hy
    n, na, nb, seed = synth.workload("h14_28q")
    ref, ham = system(n, na, nb, seed)
    psi64 = synth.random_state(ham.n_det, 8)
    psi = torch.from_numpy(psi64).to("cuda", torch.float32)
    b, e = 1000, 1096
    m = hy.ExplicitH(ham, torch.float32, b, e)
    got = m.apply(psi)
    mf = ham.apply_h_rows(psi, b, e)
    scale = torch.max(torch.abs(mf)).item()
    assert torch.max(torch.abs(got - mf)).item() <= 2e-5 * scale
    NB = ham.n_beta_str
    rng = np.random.default_rng(5)
    rows = np.unique(rng.integers(b * NB, e * NB, 16))
    s_ref = ref.sigma_rows(psi.double().cpu().numpy(), rows)
    g = got[torch.from_numpy(rows - b * NB).cuda()].double().cpu().numpy()
    assert np.abs(g - s_ref).max() <= 2e-5 * scale
    cols, vals = m.row(int(rows[0]))
    assert len(cols) == row_length(n, na, nb) == 3382


def test_explicit_h_size_query_and_bad_ranges():
    import paper_2604_01176_gb300 as hy
    ref, ham = system(6, 3, 3, 1001)
    by, nnz = hy.ExplicitH.size(ham, torch.float32)
    m = hy.ExplicitH(ham, torch.float32)
    assert (by, nnz) == (m.bytes, m.nnz)
    for b, e in [(-1, 2), (3, 2), (0, ham.n_alpha_str + 1)]:
        with pytest.raises(hy.HyError):
            hy.ExplicitH(ham, torch.float64, b, e)
    with pytest.raises(hy.HyError):
        m.row(ham.n_det)
