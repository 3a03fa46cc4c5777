"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds random-number generation and the recipe for the synthetic
molecular integrals only; none of the emulation arithmetic (Hamiltonian,
determinants, excitations) lives here.

The integrals stand in for the PySCF STO-3G hydrogen-chain integrals of the
paper's Sparse State-Vector Emulation section (H6..H16, Table 1), which are not
available offline.  Recipe (one reading per point, stated here and in the
design notes):

* generator: SplitMix64 (Steele, Lea & Flood 2014) feeding Box-Muller normals;
* h1: symmetric, off-diagonal entries N(0, 0.3^2) (0.3 read as the standard
  deviation), drawn for i < j in row-major order and mirrored; the diagonal is
  overwritten with an even ramp from -1.0 to -0.2;
* h2 (chemists' notation (pq|rs)) = sum_{k=1..8} L_k[p,q] L_k[r,s], each L_k
  symmetric with entries N(0, (0.2/k)^2) drawn for p <= q and mirrored
  (k starts at 1: the literal k = 0 of the recipe would divide by zero);
* the workload of n spatial orbitals uses seed 1000 + c for configuration c,
  molecule i of a batch uses seed 2000 + i; half filling puts ceil(n/2)
  alpha and floor(n/2) beta electrons.
"""
from __future__ import annotations

import math

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 as published by Steele, Lea and Flood (OOPSLA 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in (0, 1]: 53 random bits, shifted off zero."""
        return ((self.next_u64() >> 11) + 1) * (1.0 / 9007199254740992.0)

    def normals(self, count: int) -> np.ndarray:
        """`count` standard normals by the Box-Muller transform (pairs)."""
        out = np.empty(count, dtype=np.float64)
        i = 0
        while i < count:
            u1 = self.uniform()
            u2 = self.uniform()
            r = math.sqrt(-2.0 * math.log(u1))
            out[i] = r * math.cos(2.0 * math.pi * u2)
            if i + 1 < count:
                out[i + 1] = r * math.sin(2.0 * math.pi * u2)
            i += 2
        return out


def half_filling(n_orb: int) -> tuple[int, int]:
    """(n_alpha, n_beta) at half filling: ceil(n/2) alpha, floor(n/2) beta."""
    return (n_orb + 1) // 2, n_orb // 2


def integrals(n_orb: int, seed: int, rank: int = 8):
    """Seeded (h1, h2, e_core) shaped like a minimal-basis hydrogen chain.

    Returns h1 as an (n, n) float64 array, h2 as an (n, n, n, n) float64
    array in chemists' notation (pq|rs), and e_core = 0.
    """
    rng = SplitMix64(seed)
    n = n_orb
    h1 = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    vals = rng.normals(len(iu[0])) * 0.3
    h1[iu] = vals
    h1 = h1 + h1.T
    h1[np.diag_indices(n)] = np.linspace(-1.0, -0.2, n)
    iup = np.triu_indices(n, 0)
    h2 = np.zeros((n, n, n, n))
    for k in range(1, rank + 1):
        L = np.zeros((n, n))
        L[iup] = rng.normals(len(iup[0])) * (0.2 / k)
        L = L + L.T - np.diag(np.diag(L))
        h2 += np.einsum("pq,rs->pqrs", L, L)
    return h1, h2, 0.0


def workload(name: str):
    """Named workloads: (n_orb, n_alpha, n_beta, seed)."""
    table = {
        "h6_12q": (6, 3, 3, 1001),
        "h8_16q": (8, 4, 4, 1005),
        "h10_20q": (10, 5, 5, 1002),
        "h12_24q": (12, 6, 6, 1006),
        "h14_28q": (14, 7, 7, 1003),
        "h16_32q": (16, 8, 8, 1004),
    }
    return table[name]


def batch_molecules(count: int = 64):
    """The uneven batch: molecule i has n = 8 + (i mod 5) orbitals, seed 2000+i."""
    out = []
    for i in range(count):
        n = 8 + (i % 5)
        na, nb = half_filling(n)
        out.append((n, na, nb, 2000 + i))
    return out


def random_state(n_det: int, seed: int, normalise: bool = True) -> np.ndarray:
    """Seeded dense test amplitudes over the determinant space (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(n_det)
    if normalise:
        v /= np.linalg.norm(v)
    return v
