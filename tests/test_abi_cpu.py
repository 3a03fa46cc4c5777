"""CPU-only checks of the C ABI: the library builds and loads, it exports
every entry point include/*.h declares, host-side argument validation, and
the host-built Jordan-Wigner Pauli table (paper, Sparse State-Vector
Emulation section: fermionic operators mapped to qubits and summed) against
Kronecker-product Jordan-Wigner matrices and the oracle's Slater-Condon H.
No call here launches a kernel."""
import ctypes
import glob
import itertools
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from paper_2604_01176_gb300 import _abi, build as hybuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    hybuild.build()
    return _abi.load()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(hy_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_symbols_exported(lib):
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if getattr(lib, n, None) is None]
    assert not missing, missing
    # the ctypes table covers exactly the declared entry points
    assert set(_abi.SIGNATURES) == names


def test_version_and_error_strings(lib):
    assert b"sm_103a" in lib.hy_version()
    out = ctypes.c_void_p()
    h1 = np.zeros((2, 2))
    h2 = np.zeros((2,) * 4)
    st = lib.hy_build_hamiltonian(h1.ctypes.data_as(ctypes.c_void_p),
                                  h2.ctypes.data_as(ctypes.c_void_p), 0.0, 17, 1,
                                  1, 1e-14, ctypes.byref(out))
    assert st == _abi.HY_ERR_ARG and not out.value
    assert b"n_orb" in lib.hy_last_error()


@pytest.mark.parametrize("bad", ["h1", "h2", "nan", "electrons", "null"])
def test_build_rejects_bad_input_before_any_device_call(lib, bad):
    n = 3
    h1, h2, _ = synth.integrals(n, 5)
    na, nb = 2, 1
    if bad == "h1":
        h1 = h1.copy(); h1[0, 1] += 1e-3
    elif bad == "h2":
        h2 = h2.copy(); h2[0, 1, 2, 2] += 1e-3
    elif bad == "nan":
        h1 = h1.copy(); h1[1, 1] = np.nan
    elif bad == "electrons":
        na = 4
    out = ctypes.c_void_p()
    p1 = None if bad == "null" else h1.ctypes.data_as(ctypes.c_void_p)
    st = lib.hy_build_hamiltonian(p1, h2.ctypes.data_as(ctypes.c_void_p), 0.0, n,
                                  na, nb, 1e-14, ctypes.byref(out))
    assert st == _abi.HY_ERR_ARG
    assert not out.value


def test_null_handles_rejected(lib):
    assert lib.hy_apply_h(None, None, None, 0, None) == _abi.HY_ERR_ARG
    assert lib.hy_pool_size(None, None) == _abi.HY_ERR_ARG
    assert lib.hy_ham_destroy(None) == _abi.HY_OK
    assert lib.hy_pool_destroy(None) == _abi.HY_OK


# --------------------------------------------------------------------------
# Pauli table (host-only build) against Jordan-Wigner Kronecker products
# --------------------------------------------------------------------------
def pauli_table(lib, h1, h2, e_core, n, prune=1e-14):
    nt, ng = ctypes.c_int64(), ctypes.c_int64()
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    h2 = np.ascontiguousarray(h2, dtype=np.float64)
    P = ctypes.c_void_p
    _abi.check(lib.hy_pauli_table_build(h1.ctypes.data_as(P), h2.ctypes.data_as(P),
                                        e_core, n, prune, 0, None, None, None,
                                        None, ctypes.byref(nt), ctypes.byref(ng)))
    x = np.empty(nt.value, np.uint64)
    z = np.empty(nt.value, np.uint64)
    c = np.empty(nt.value)
    off = np.empty(nt.value + 1, np.int64)
    _abi.check(lib.hy_pauli_table_build(
        h1.ctypes.data_as(P), h2.ctypes.data_as(P), e_core, n, prune, nt.value,
        x.ctypes.data_as(P), z.ctypes.data_as(P), c.ctypes.data_as(P),
        off.ctypes.data_as(P), ctypes.byref(nt), ctypes.byref(ng)))
    return x, z, c, off[: ng.value + 1]


_PAULI = {
    "I": np.eye(2), "X": np.array([[0, 1], [1, 0]], complex),
    "Y": np.array([[0, -1j], [1j, 0]]), "Z": np.diag([1.0, -1.0]).astype(complex),
}


def pauli_matrix(x, z, M):
    """Hermitian Pauli string on M qubits; qubit 0 is the rightmost factor
    (basis index = sum_j n_j 2^j)."""
    m = sp.identity(1, format="csr", dtype=complex)
    for j in reversed(range(M)):
        xb, zb = (int(x) >> j) & 1, (int(z) >> j) & 1
        lab = "Y" if xb and zb else "X" if xb else "Z" if zb else "I"
        m = sp.kron(m, sp.csr_matrix(_PAULI[lab]), format="csr")
    return m


def jw_hamiltonian(h1, h2, e_core, n):
    M = 2 * n
    sm = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    zz = sp.csr_matrix(np.diag([1.0, -1.0]))
    ii = sp.identity(2, format="csr")
    a = []
    for j in range(M):
        f = [ii] * (M - 1 - j) + [sm] + [zz] * j
        m = f[0]
        for t in f[1:]:
            m = sp.kron(m, t, format="csr")
        a.append(m)
    ad = [t.T.tocsr() for t in a]
    H = sp.identity(1 << M, format="csr") * e_core
    for P, Q in itertools.product(range(M), repeat=2):
        if P // n == Q // n and h1[P % n, Q % n] != 0:
            H = H + h1[P % n, Q % n] * (ad[P] @ a[Q])
    for P, Q, R, S in itertools.product(range(M), repeat=4):
        if P // n != Q // n or R // n != S // n:
            continue
        c = h2[P % n, Q % n, R % n, S % n]
        if c != 0:
            H = H + 0.5 * c * (ad[P] @ ad[R] @ a[S] @ a[Q])
    return H.toarray()


@pytest.mark.parametrize("n", [2, 3, 4])
def test_pauli_table_equals_jordan_wigner_and_slater_condon(lib, n):
    h1, h2, _ = synth.integrals(n, 31 + n)
    e_core = -0.7
    x, z, c, off = pauli_table(lib, h1, h2, e_core, n)
    M = 2 * n
    H = np.zeros((1 << M, 1 << M), complex)
    for xi, zi, ci in zip(x, z, c):
        H += ci * pauli_matrix(xi, zi, M).toarray()
    Hjw = jw_hamiltonian(h1, h2, e_core, n)
    assert np.abs(H.imag).max() < 1e-13
    assert np.abs(H.real - Hjw).max() < 1e-12
    # grouping: sorted by (x, z); each group shares one x
    assert np.all(np.diff(off) > 0) and off[0] == 0 and off[-1] == len(x)
    for g in range(len(off) - 1):
        assert len(set(x[off[g]:off[g + 1]].tolist())) == 1
    keys = list(zip(x.tolist(), z.tolist()))
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # every sector: restriction equals the oracle's Slater-Condon matrix
    for na in range(n + 1):
        for nb in range(n + 1):
            s = oracle.System(h1, h2, e_core, n, na, nb)
            d = s.dets().astype(np.int64)
            assert np.abs(H.real[np.ix_(d, d)] - s.dense_h()).max() < 1e-12


def test_pauli_table_counts_and_pruning(lib):
    """Only X-masks that move an even number of electrons within each spin
    block appear, the identity carries e_core + the trace terms, and a large
    prune threshold removes small terms."""
    n = 6
    h1, h2, _ = synth.integrals(n, 1001)
    x, z, c, off = pauli_table(lib, h1, h2, 0.0, n)
    amask = (1 << n) - 1
    for xi in x[off[:-1]]:
        xi = int(xi)
        assert bin(xi & amask).count("1") % 2 == 0
        assert bin(xi >> n).count("1") % 2 == 0
        assert bin(xi).count("1") <= 4
    # distinct X-masks: identity, alpha / beta single (pq), alpha-alpha /
    # beta-beta double (4 bits in one block) and alpha x beta singles
    c2, c4 = n * (n - 1) // 2, n * (n - 1) * (n - 2) * (n - 3) // 24
    assert len(off) - 1 == 1 + 2 * c2 + 2 * c4 + c2 * c2    # 286 at 12 qubits
    x2, _, cp, _ = pauli_table(lib, h1, h2, 0.0, n, prune=1e-3)
    assert len(x2) < len(x) and np.abs(cp).min() > 1e-3


def test_pauli_table_identical_across_thread_counts():
    """The host Pauli table is built by threads that each own a class of
    X-masks and visit the products in one fixed order, so every coefficient
    is summed in the same order whatever the thread count: the table built
    with 1, 3 and 8 threads (separate processes) is identical bit for bit."""
    import subprocess
    import sys
    code = (
        "import ctypes, hashlib, sys; sys.path.insert(0, {root!r}); import numpy as np, synth;"
        "from tests.test_abi_cpu import pauli_table; from paper_2604_01176_gb300 import _abi;"
        "h1, h2, ec = synth.integrals(10, 1002);"
        "x, z, c, off = pauli_table(_abi.load(), h1, h2, ec, 10);"
        "print(hashlib.sha256(x.tobytes() + z.tobytes() + c.tobytes() + off.tobytes()).hexdigest())"
    ).format(root=ROOT)
    digests = set()
    for threads in ("1", "3", "8"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT,
                             capture_output=True, text=True, timeout=300)
        assert out.returncode == 0, out.stderr
        digests.add(out.stdout.strip().splitlines()[-1])
    assert len(digests) == 1
