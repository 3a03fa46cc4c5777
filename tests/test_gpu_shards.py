"""Row-range H|psi> (hy_apply_h_rows, hy_dot_rows): the paper's distribution
of H by rows of Omega_CIk with the state replicated (Sparse State-Vector
Emulation section, parallelisation paragraph), run here as shards one after
another on one GPU.  Every element of a shard is formed by the same
arithmetic in the same order as the unsharded sweep, so the concatenated
blocks must equal hy_apply_h's sigma bit for bit, in FP64, in FP32 with the
tensor-core coupling and in FP32 with the SIMT coupling; the partial inner
products summed over shards give the energy (FP64 accuracy, 1e-12
relative)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFGS = [(6, 3, 3, 1001), (7, 4, 3, 77), (10, 5, 5, 1002), (14, 7, 7, 1003)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _splits(na):
    """Uneven splits, an empty shard, a one-row shard and the whole range."""
    cuts = sorted({0, na, 1 if na > 1 else 0, na // 3, na // 3, (2 * na) // 3, na - 1})
    yield [(0, na)]
    yield list(zip(cuts[:-1], cuts[1:])) + [(na // 3, na // 3)]
    yield [(r * na // 4, (r + 1) * na // 4) for r in range(4)]


@pytest.mark.parametrize("cfg", CFGS, ids=[f"n{c[0]}" for c in CFGS])
@pytest.mark.parametrize("mode", ["f64", "f32-tensor", "f32-simt"])
def test_row_shards_concatenate_bit_for_bit(cfg, mode):
    import paper_2604_01176_gb300 as hy
    n, na, nb, seed = cfg
    h1, h2, ec = synth.integrals(n, seed)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    dt = torch.float64 if mode == "f64" else torch.float32
    if mode == "f32-simt":
        ham.set_coupling("simt")
    psi = torch.from_numpy(synth.random_state(ham.n_det, 11)).to("cuda", dt)
    full = ham.apply_h(psi)
    e_full = ham.energy(psi, full)
    NA, NB = ham.n_alpha_str, ham.n_beta_str
    for split in _splits(NA):
        split = sorted(set(split))
        blocks = {}
        for b, e in split:
            blocks[(b, e)] = ham.apply_h_rows(psi, b, e)
        cover = [s for s in split if s[1] > s[0]]
        cat = torch.cat([blocks[s] for s in cover])
        assert cat.numel() == ham.n_det
        assert torch.equal(cat, full), f"split {split}"
        parts = [ham.dot_rows(psi[b * NB: e * NB], blocks[(b, e)], b, e) for b, e in split]
        e_sum = float(sum(float(p.item()) for p in parts))
        assert abs(e_sum - float(e_full.item())) <= 1e-12 * max(1.0, abs(float(e_full.item())))
    if mode == "f64" and n <= 10:
        ref = oracle.System(h1, h2, ec, n, na, nb)
        b, e = NA // 3, (2 * NA) // 3 + 1
        rows = np.arange(b * NB, e * NB)
        got = ham.apply_h_rows(psi, b, e).cpu().numpy()
        assert np.abs(got - ref.sigma_rows(psi.cpu().numpy(), rows)).max() < 1e-12


def test_row_range_rejects_bad_ranges():
    import paper_2604_01176_gb300 as hy
    h1, h2, ec = synth.integrals(6, 1001)
    ham = hy.Hamiltonian(h1, h2, ec, 6, 3, 3)
    psi = torch.zeros(ham.n_det, dtype=torch.float64, device="cuda")
    for b, e in [(-1, 3), (5, 4), (0, ham.n_alpha_str + 1)]:
        with pytest.raises((hy.HyError, ValueError)):
            ham.apply_h_rows(psi, b, e)
    with pytest.raises(hy.HyError):          # sigma block inside psi
        from paper_2604_01176_gb300 import _abi
        import ctypes
        st = _abi.load().hy_apply_h_rows(ham.handle, ctypes.c_void_p(psi.data_ptr()),
                                         ctypes.c_void_p(psi.data_ptr() + 8 * 20), 0, 0, 1,
                                         None)
        _abi.check(st)
