"""GPU parity of the ADAPT-VQE driver (hy_adapt_*) against the oracle's
ADAPT loop (oracle/adapt.py), and of the mixed-precision mode against the
plain FP64 mode.

Tolerances: FP64 energies 1e-10 Ha per iteration, identical operator
selections; adjoint gradients 1e-9 (the oracle builds each dE/dtheta_l from
its definition with O(j^2) exponentials); mixed precision: final energy
within 1e-6 Ha of plain FP64 (the stated target of the mixed mode) and the
double-precision refinement at least as low as the float optimum.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import adapt as oadapt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def make(n, na, nb, seed):
    import paper_2604_01176_gb300 as hy
    h1, h2, ec = synth.integrals(n, seed)
    ref = oracle.System(h1, h2, ec, n, na, nb)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    return ref, ham, hy.Pool(ham)


def test_adapt_f64_matches_oracle_loop():
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = make(6, 3, 3, 1001)
    iters = 8
    rec_ref = oadapt.run(ref, ref.pool(), max_iter=iters, gtol=1e-10)
    ad = hy.Adapt(ham, pool, "f64", max_iter=iters, gtol=1e-10)
    recs = ad.run(iters)
    sel = [r["selected"] for r in recs if not r["converged"]]
    assert sel == rec_ref["selected"]
    e = np.array([r["energy"] for r in recs if not r["converged"]])
    assert np.abs(e - np.array(rec_ref["energy"])).max() < 1e-10
    assert np.all(np.diff(e) <= 1e-12)
    assert e[-1] >= ref.fci_energy() - 1e-12
    ops, th = ad.ansatz()
    assert list(ops) == rec_ref["ops"]
    assert np.abs(th - np.array(rec_ref["thetas"])).max() < 1e-5


@pytest.mark.parametrize("n,na,nb,seed", [(6, 3, 3, 1001), (7, 4, 3, 77)])
def test_adjoint_gradient_matches_oracle(n, na, nb, seed):
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = make(n, na, nb, seed)
    opd = ref.pool()
    rng = np.random.default_rng(3)
    ops = rng.integers(0, len(opd), 7)
    th = rng.normal(0, 0.5, 7)
    ad = hy.Adapt(ham, pool, "f64", max_iter=16)
    ad.set_ansatz(ops, th)
    e, g = ad.evaluate(th)
    e_ref, g_ref = oadapt.energy_and_gradient(ref, opd, list(ops), th)
    assert abs(e - e_ref) < 1e-10
    assert np.abs(g - g_ref).max() < 1e-9


def test_checkpoint_resume_reproduces_energy():
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = make(6, 3, 3, 1001)
    ad = hy.Adapt(ham, pool, "f64", max_iter=8)
    recs = ad.run(4)
    ops, th = ad.ansatz()
    ad2 = hy.Adapt(ham, pool, "f64", max_iter=8)
    ad2.set_ansatz(ops, th)
    e, _ = ad2.evaluate(th)
    assert abs(e - recs[-1]["energy"]) < 1e-12
    r1, r2 = ad.step(), ad2.step()
    assert r1["selected"] == r2["selected"]
    assert abs(r1["energy"] - r2["energy"]) < 1e-9


@pytest.mark.parametrize("n,seed,iters", [(6, 1001, 8), (8, 1005, 5)])
def test_mixed_precision_matches_plain(n, seed, iters):
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = make(n, n // 2, n // 2, seed)
    plain = hy.Adapt(ham, pool, "f64", max_iter=iters).run(iters)
    mixed = hy.Adapt(ham, pool, "mixed", max_iter=iters, refine_steps=6, float_from=1).run(iters)
    assert [r["selected"] for r in mixed] == [r["selected"] for r in plain]
    assert abs(mixed[-1]["energy"] - plain[-1]["energy"]) < 1e-6
    for r in mixed:
        # float evaluation error reported per iteration, small
        assert r["energy_bulk_err"] < 1e-4
        assert r["energy"] <= r["energy_bulk"] + 1e-4
        assert r["n_evals_f64"] >= 1


def test_adapt_stops_on_gradient_norm():
    """The driver stops (nothing appended) once ||g||_2 < eps_grad, and
    reports the screen's norm."""
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = make(6, 3, 3, 1001)
    psi = ref.hf_state()
    g = ref.gradients(ref.pool(), psi, ref.sigma(psi))
    gn = float(np.linalg.norm(g))
    ad = hy.Adapt(ham, pool, "f64", max_iter=4, eps_grad=gn * 1.0001)
    r = ad.step()
    assert r["converged"] == 1 and r["selected"] == -1
    assert abs(r["grad_norm"] - gn) < 1e-12
    assert len(ad.ansatz()[0]) == 0
    ad2 = hy.Adapt(ham, pool, "f64", max_iter=4, eps_grad=gn * 0.9999)
    r2 = ad2.step()
    assert r2["converged"] == 0 and r2["selected"] >= 0


@pytest.mark.parametrize("sparse", [False, True], ids=["dense", "sparse"])
def test_refine_after_settled_double_optimisation(sparse):
    """A mixed driver whose iterations all optimise in double (few nonzero
    amplitudes): its refinement returns the last double energy as it stands,
    a fresh double evaluation of the same parameters (steps = 0) agrees with
    it to rounding, and after the parameters move the refinement descends
    again."""
    import paper_2604_01176_gb300 as hy
    ref, ham, pool = make(6, 3, 3, 1001)
    iters = 5
    plain = hy.Adapt(ham, pool, "f64", max_iter=iters, sparse=sparse).run(iters)
    ad = hy.Adapt(ham, pool, "mixed", max_iter=iters, sparse=sparse, float_from=1 << 30)
    recs = ad.run(iters)
    assert [r["selected"] for r in recs] == [r["selected"] for r in plain]
    assert all(r["energy_bulk_err"] == 0.0 for r in recs)
    ops, th = ad.ansatz()
    e_ref = oadapt.energy_and_gradient(ref, ref.pool(), list(ops), np.array(th))[0]
    e_last = recs[-1]["energy"]
    assert abs(e_last - e_ref) < 1e-10
    assert ad.refine(steps=4) == e_last
    assert abs(ad.refine(steps=0) - e_last) < 1e-12
    # moved parameters: the shortcut no longer applies and the refinement
    # descends from the moved point back toward the optimum
    moved = np.array(th) + 1e-2
    e_moved = oadapt.energy_and_gradient(ref, ref.pool(), list(ops), moved)[0]
    ad.set_ansatz(list(ops), list(moved))
    e_ref4 = ad.refine(steps=4)
    assert e_ref4 < e_moved - 1e-9
    assert e_ref4 >= e_last - 1e-9
