"""SV-MPS partition on the GPU (hy_ham_partition; paper: Partitioned SV-MPS
Emulation section, H = H_eta + sum B and the split of <psi|H|psi>): the
handles for H_eta and for the cross-block rest against the oracle's own
Jordan-Wigner Pauli expansion filtered by block (oracle/partition.py):
sigma elementwise (FP64 1e-12), <psi|H_eta|psi> (1e-12), E_eta + E_B = E,
both qubit orders and every level eta the chain allows (one block, blocks
of one spin, blocks that split an orbital's two spins)."""
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


@pytest.mark.parametrize("cfg", [(4, 2, 2, 23), (6, 3, 3, 1001), (5, 3, 2, 12)],
                         ids=["n4", "n6", "n5"])
def test_partition_sigma_and_energies_match_oracle(cfg):
    import paper_2604_01176_gb300 as hy
    from oracle import partition as opart
    n, na, nb, seed = cfg
    h1, h2, ec = synth.integrals(n, seed)
    ref = oracle.System(h1, h2, ec, n, na, nb)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    terms = opart.jw_terms(h1, h2, ec, n)
    dets = ref.dets().astype(np.int64)
    psi = synth.random_state(ham.n_det, 17)
    P = torch.from_numpy(psi).cuda()
    e_full = ref.energy(psi)
    etas = [e for e in range(0, 4) if (2 * n) % (1 << e) == 0]
    for eta in etas:
        for inter in (False, True):
            e_parts = []
            for part in (0, 1):
                t = opart.partition_terms(terms, n, eta, inter, part)
                Hd = opart.dense_full(t, 2 * n)[np.ix_(dets, dets)]
                hp = ham.partition(eta, inter, part)
                sig = hp.apply_h(P).cpu().numpy()
                assert np.abs(sig - Hd @ psi).max() < 1e-12, (eta, inter, part)
                e = float(hp.energy(P, hp.apply_h(P)).item())
                assert abs(e - float(psi @ Hd @ psi)) < 1e-12
                e_parts.append(e)
                hp.close()
            assert abs(sum(e_parts) - e_full) < 1e-11


def test_partition_rejects_bad_levels():
    import paper_2604_01176_gb300 as hy
    h1, h2, ec = synth.integrals(5, 12)
    ham = hy.Hamiltonian(h1, h2, ec, 5, 3, 2)
    for eta, part in [(2, 0), (-1, 0), (1, 2)]:        # 2^2 does not divide 10 qubits
        with pytest.raises(hy.HyError):
            ham.partition(eta, False, part)
