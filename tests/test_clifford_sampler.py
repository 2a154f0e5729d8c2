"""Pins of the uniformly random Clifford sampler (``workloads.circuits``),
the paper's own benchmark family (Section "Simulation of Clifford circuits",
Fig. 2a: uniformly random Cliffords, Bravyi-Maslov).

The sampler writes C = P . b1 . w . b2 with b1, b2 uniform in the Borel
subgroup B of Hadamard-free Cliffords and w a signed permutation drawn with
weight 2^len(w).  These checks are exact:

* the insertion code of signed permutations is a bijection onto the
  hyperoctahedral group B_n whose code sum is the Coxeter length (computed
  here from its inversion form, Bjorner & Brenti Sec. 8.1), and the weights
  sum to prod_j (4^j - 1);
* the length-one elements are H on the last qubit and adjacent SWAPs;
* for n = 1, 2 every choice of (b1, w, b2) is enumerated and each resulting
  tableau is computed by the oracle: every element of Sp(2n, 2) receives
  probability exactly 1 / |Sp(2n, 2)| (rational arithmetic), and with the
  Pauli layer every n = 1 Clifford 1/24;
* for n = 3, 4 the sampled C X_0 C^dag is uniform over the 4^n - 1
  non-identity Paulis (chi-square, fixed seeds).
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from workloads import circuits as C


def length_b(w):
    """Coxeter length of a signed permutation: inv + #{i <= j : w_i + w_j < 0}."""
    n = len(w)
    inv = sum(1 for i in range(n) for j in range(i + 1, n) if w[i] > w[j])
    nsp = sum(1 for i in range(n) for j in range(i, n) if w[i] + w[j] < 0)
    return inv + nsp


def all_codes(n):
    return itertools.product(*[range(2 * m) for m in range(1, n + 1)])


def poincare(n):
    return math.prod(4 ** j - 1 for j in range(1, n + 1))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_insertion_code_bijection_and_length(n):
    seen = set()
    total = 0
    for code in all_codes(n):
        w = C.signed_perm_from_code(code)
        assert sorted(abs(v) for v in w) == list(range(1, n + 1))
        assert length_b(w) == sum(code)
        seen.add(tuple(w))
        total += 2 ** sum(code)
    assert len(seen) == 2 ** n * math.factorial(n)
    assert total == poincare(n)


@pytest.mark.parametrize("n", [2, 5])
def test_length_one_elements_are_the_flag_reflections(n):
    op = lambda ws: C.decode(np.concatenate(ws)) if ws else (np.zeros(0),) * 3
    s0 = [-1] + list(range(2, n + 1))
    o, a, _ = op(C._weyl_words(s0))
    assert o.tolist() == [C.TAB_H] and a.tolist() == [n - 1]
    for i in range(1, n):
        w = list(range(1, n + 1))
        w[i - 1], w[i] = w[i], w[i - 1]
        assert length_b(w) == 1
        o, a, b = op(C._weyl_words(w))
        assert o.tolist() == [C.TAB_SWAP] and sorted([a[0], b[0]]) == [n - i - 1, n - i]


def borel_elements(n):
    lower = [(t, c) for t in range(n) for c in range(t)]
    upper = [(i, j) for i in range(n) for j in range(i, n)]
    out = []
    for lb in itertools.product((0, 1), repeat=len(lower)):
        for gb in itertools.product((0, 1), repeat=len(upper)):
            L = np.zeros((n, n), np.uint8)
            G = np.zeros((n, n), np.uint8)
            for (t, c), v in zip(lower, lb):
                L[t, c] = v
            for (i, j), v in zip(upper, gb):
                G[i, j] = v
            out.append(C.borel_words(L, G))
    return out


@pytest.mark.parametrize("n", [2, 5, 9, 16])
def test_cnot_part_is_the_unit_lower_triangular_map(n):
    """The CNOT part of a Borel element maps |x> to |(I + L) x>: destabilizer
    i of the tableau (C X_i C^dag) carries X on column i of I + L."""
    rng = np.random.default_rng(n)
    L = np.tril(rng.integers(0, 2, size=(n, n), dtype=np.uint8), -1)
    words = C.borel_words(L, np.zeros((n, n), np.uint8))
    gates = np.concatenate(words) if words else np.zeros(0, np.uint64)
    _, (x, z, r) = oracle.run_circuit(n, gates)
    M = (np.eye(n, dtype=np.uint8) + L) % 2
    assert np.array_equal(x[:n], M.T)
    assert not z[:n].any() and not r.any()


def tableau(n, gates):
    _, (x, z, r) = oracle.run_circuit(n, gates)
    return x.tobytes() + z.tobytes(), r.tobytes()


@pytest.mark.parametrize("n", [1, 2])
def test_sampler_uniform_on_symplectic_group(n):
    B = borel_elements(n)
    assert len(B) == 2 ** (n * n)
    order = 2 ** (n * n) * poincare(n)  # |Sp(2n, 2)|
    mass = {}
    for code in all_codes(n):
        w = C.signed_perm_from_code(code)
        pw = Fraction(2 ** sum(code), poincare(n)) / (len(B) ** 2)
        for b1 in B:
            for b2 in B:
                key, _ = tableau(n, C.clifford_from_parts(n, b2, w, b1, []))
                mass[key] = mass.get(key, 0) + pw
    assert len(mass) == order
    assert set(mass.values()) == {Fraction(1, order)}


def test_sampler_uniform_on_one_qubit_cliffords_with_signs():
    B = borel_elements(1)
    paulis = [[], [C.encode(C.TAB_X, 0, 0).reshape(1)], [C.encode(C.TAB_Z, 0, 0).reshape(1)],
              [C.encode(C.TAB_Y, 0, 0).reshape(1)]]
    mass = {}
    for code in all_codes(1):
        w = C.signed_perm_from_code(code)
        pw = Fraction(2 ** sum(code), 3) / (len(B) ** 2 * len(paulis))
        for b1 in B:
            for b2 in B:
                for p in paulis:
                    key = tableau(1, C.clifford_from_parts(1, b2, w, b1, p))
                    mass[key] = mass.get(key, 0) + pw
    assert len(mass) == 24
    assert set(mass.values()) == {Fraction(1, 24)}


@pytest.mark.parametrize("n,samples", [(3, 3150), (4, 5100)])
def test_sampled_destabilizer_uniform(n, samples):
    chi2 = pytest.importorskip("scipy.stats").chi2
    cells = 4 ** n - 1
    counts = np.zeros(4 ** n, np.int64)
    for c in range(samples):
        circ = C.random_clifford(n, C.splitmix64(9000 + n * 100003 + c))
        _, (x, z, _) = oracle.run_circuit(n, circ.gates)
        idx = 0
        for j in range(n):
            idx = idx * 4 + 2 * int(x[0, j]) + int(z[0, j])
        counts[idx] += 1
    assert counts[0] == 0  # never the identity
    expect = samples / cells
    stat = float((((counts[1:] - expect) ** 2) / expect).sum())
    assert chi2.sf(stat, cells - 1) > 1e-4, stat


def _symplectic(n, gates):
    """The linear part of a Clifford: row g = (x | z) bits of the image of
    generator g (X_1..X_n, then Z_1..Z_n) -- the tableau the oracle leaves
    after running the circuit on |0^n>."""
    _, (x, z, _) = oracle.run_circuit(n, gates)
    return np.concatenate([x, z], axis=1).astype(np.uint8)


def test_bruhat_double_cosets_n3():
    """At n = 3, for each of the 48 signed permutations w, the set
    {b2 w b1 : b1, b2 in B} (linear parts, as products of the oracle's
    matrices) has exactly |B| 2^len(w) elements, the sets are disjoint, and
    together they are all |Sp(6, 2)| = 1,451,520 elements: the weights
    2^len(w) the sampler draws are the double-coset sizes."""
    n = 3
    gates_of = lambda words: np.concatenate(words) if words else np.zeros(0, np.uint64)
    MB = np.array([_symplectic(n, gates_of(b)) for b in borel_elements(n)])  # (512, 6, 6)
    assert len({m.tobytes() for m in MB}) == 512
    # row j of Q as a 6-bit integer, for every matrix Q
    QB = (MB.astype(np.int64) << np.arange(2 * n)[None, None, :]).sum(axis=2)  # (512, 6)
    seen = set()
    total = 0
    for code in all_codes(n):
        w = C.signed_perm_from_code(code)
        Mw = _symplectic(n, gates_of(C._weyl_words(w)))
        P = (MB.astype(np.int64) @ Mw.astype(np.int64)) % 2  # b2 first, then w: (512, 6, 6)
        # R[a, b] = P[a] . MB[b] over GF(2), rows packed as 6-bit integers
        R = np.zeros((512, 512, 2 * n), np.int64)
        for i in range(2 * n):
            for j in range(2 * n):
                R[:, :, i] ^= np.where(P[:, i, j][:, None] == 1, QB[None, :, j], 0)
        keys = np.unique((R << (6 * np.arange(2 * n))[None, None, :]).sum(axis=2))
        assert keys.size == 512 * 2 ** sum(code), (w, keys.size)
        before = len(seen)
        seen.update(keys.tolist())
        assert len(seen) == before + keys.size  # disjoint from the other cosets
        total += keys.size
    assert total == 2 ** (n * n) * poincare(n) == 1451520


def test_sampled_one_qubit_cliffords_uniform_with_signs():
    """random_clifford itself (with its Pauli layer) at n = 1: the 24
    Cliffords, signs included, are drawn uniformly (chi-square, fixed seeds)."""
    chi2 = pytest.importorskip("scipy.stats").chi2
    counts = {}
    samples = 2400
    for c in range(samples):
        circ = C.random_clifford(1, C.splitmix64(77000 + c))
        key = tableau(1, circ.gates)
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 24
    expect = samples / 24
    stat = sum((v - expect) ** 2 / expect for v in counts.values())
    assert chi2.sf(stat, 23) > 1e-4, stat
