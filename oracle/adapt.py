"""ADAPT-VQE loop of the oracle (test infrastructure, FP64, CPU).

Follows the paper's description of ADAPT-VQE (Quantum Algorithms for Chemistry
section and the Numerical performance subsection): start from the Hartree-Fock
determinant; each iteration scores every pool operator by its energy
gradient, appends the operator with the largest |gradient| at theta = 0, then
re-optimises all parameters; stop when the gradient norm is small or after an
iteration cap.

Readings where the paper is silent (same readings as the CUDA path):
* optimiser: BFGS (here scipy's), analytic gradients, started from the
  previous parameters with the new one at 0, tolerance on max |dE/dtheta|;
* argmax tie-break: the lowest pool index among operators whose |g| is within
  1e-12 * max|g| of the maximum;
* dE/dtheta_l is computed from its definition,
  2 <H psi | U_j .. U_{l+1} A_l U_l .. U_1 | HF>, costing O(j^2) applications.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize


def prepare(system, pool, ops, thetas):
    psi = system.hf_state()
    for k, t in zip(ops, thetas):
        psi = system.apply_excitation(pool[k], t, psi)
    return psi


def energy_and_gradient(system, pool, ops, thetas):
    psi = prepare(system, pool, ops, thetas)
    sigma = system.sigma(psi)
    e = float(psi @ sigma)
    grad = np.zeros(len(ops))
    for l in range(len(ops)):
        phi = prepare(system, pool, ops[: l + 1], thetas[: l + 1])
        v = system.apply_generator(pool[ops[l]], phi)
        for m in range(l + 1, len(ops)):
            v = system.apply_excitation(pool[ops[m]], thetas[m], v)
        grad[l] = 2.0 * float(sigma @ v)
    return e, grad


def select(g, rel_tie=1e-12):
    a = np.abs(g)
    m = a.max()
    return int(np.nonzero(a >= m - rel_tie * m)[0][0])


def run(system, pool, max_iter=20, eps_grad=1e-5, gtol=1e-9, pool_subset=None):
    """Returns a dict with the per-iteration record."""
    allowed = (np.arange(len(pool)) if pool_subset is None
               else np.asarray(pool_subset))
    ops: list[int] = []
    thetas = np.zeros(0)
    record = {"energy": [], "grad_norm": [], "selected": [], "max_grad": []}
    for _ in range(max_iter):
        psi = prepare(system, pool, ops, thetas)
        sigma = system.sigma(psi)
        g = system.gradients(pool[allowed], psi, sigma)
        gn = float(np.linalg.norm(g))
        record["grad_norm"].append(gn)
        if gn < eps_grad:
            break
        k = int(allowed[select(g)])
        record["selected"].append(k)
        record["max_grad"].append(float(np.abs(g).max()))
        ops.append(k)
        x0 = np.concatenate([thetas, [0.0]])
        res = minimize(lambda t: energy_and_gradient(system, pool, ops, t), x0,
                       jac=True, method="BFGS", options={"gtol": gtol,
                                                         "maxiter": 500})
        thetas = res.x
        record["energy"].append(float(res.fun))
    record["ops"] = list(ops)
    record["thetas"] = thetas.tolist()
    return record
