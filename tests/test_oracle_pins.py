"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* gate rules and AG's g: explicit Pauli-matrix conjugation / products;
* whole runs: a brute-force state vector (stabilizer eigen-equations, outcome
  probabilities 0, 1/2, 1, projection onto the oracle's outcomes);
* known stabilizer states (Bell, GHZ, product states, +Y);
* invariants: symplectic form, circuit-times-inverse = identity, repeated
  measurement;
* Philox4x32-10 against the Random123 known-answer vectors (tests/golden).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from tests.statevector import StateVector, gate_matrix, pauli_matrix, pauli_1q
from workloads import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

ONE_Q = {"H": "h", "S": "s", "SDG": "sdg", "X": "x", "Y": "y", "Z": "z"}
TWO_Q = {"CNOT": "cnot", "CZ": "cz", "SWAP": "swap"}
OPNAME = {C.TAB_X: "X", C.TAB_Y: "Y", C.TAB_Z: "Z", C.TAB_H: "H", C.TAB_S: "S",
          C.TAB_SDG: "SDG", C.TAB_CNOT: "CNOT", C.TAB_CZ: "CZ", C.TAB_SWAP: "SWAP"}


def match_pauli(M, n):
    """Find (x, z, r) with M = (-1)^r P(x, z); None if M is not a signed Pauli."""
    for bits in itertools.product((0, 1), repeat=2 * n):
        x, z = bits[:n], bits[n:]
        P = pauli_matrix(x, z)
        if np.allclose(M, P):
            return list(x), list(z), 0
        if np.allclose(M, -P):
            return list(x), list(z), 1
    return None


# ---------------------------------------------------------------- gate rules

@pytest.mark.parametrize("name", sorted(ONE_Q))
def test_one_qubit_rule_vs_conjugation(name):
    U = gate_matrix(name, [0], 1)
    for x, z, r in itertools.product((0, 1), repeat=3):
        t = oracle.Tableau(1)
        X = np.array([[x], [1 - x]], np.uint8)
        Z = np.array([[z], [z]], np.uint8)
        R = np.array([r, 0], np.uint8)
        t.set(X, Z, R)
        getattr(t, ONE_Q[name])(0)
        gx, gz, gr = t.get()
        want = match_pauli(U @ pauli_matrix([x], [z], r) @ U.conj().T, 1)
        assert want is not None
        assert (list(gx[0]), list(gz[0]), int(gr[0])) == (want[0], want[1], want[2]), \
            (name, x, z, r)


@pytest.mark.parametrize("name", sorted(TWO_Q))
@pytest.mark.parametrize("order", [(0, 1), (1, 0)])
def test_two_qubit_rule_vs_conjugation(name, order):
    U = gate_matrix(name, list(order), 2)
    rng = np.random.default_rng(3)
    for bits in itertools.product((0, 1), repeat=5):
        x, z, r = list(bits[0:2]), list(bits[2:4]), bits[4]
        t = oracle.Tableau(2)
        X = rng.integers(0, 2, (4, 2)).astype(np.uint8)
        Z = rng.integers(0, 2, (4, 2)).astype(np.uint8)
        R = rng.integers(0, 2, 4).astype(np.uint8)
        X[1], Z[1], R[1] = x, z, r
        t.set(X, Z, R)
        getattr(t, TWO_Q[name])(*order)
        gx, gz, gr = t.get()
        want = match_pauli(U @ pauli_matrix(x, z, r) @ U.conj().T, 2)
        assert (list(gx[1]), list(gz[1]), int(gr[1])) == want, (name, order, bits)


def test_g_matches_pauli_products():
    for x1, z1, x2, z2 in itertools.product((0, 1), repeat=4):
        prod = pauli_1q(x1, z1) @ pauli_1q(x2, z2)
        base = pauli_1q(x1 ^ x2, z1 ^ z2)
        gv = oracle.g(x1, z1, x2, z2)
        assert gv in (-1, 0, 1)
        assert np.allclose(prod, (1j ** gv) * base), (x1, z1, x2, z2, gv)


def test_rowsum_matches_matrix_product():
    """rowsum(h, i) sets row h to row_i * row_h for commuting rows, else errors."""
    n = 2
    for bi, bh in itertools.product(itertools.product((0, 1), repeat=5), repeat=2):
        xi, zi, ri = list(bi[0:2]), list(bi[2:4]), bi[4]
        xh, zh, rh = list(bh[0:2]), list(bh[2:4]), bh[4]
        t = oracle.Tableau(n)
        X = np.zeros((4, 2), np.uint8)
        Z = np.zeros((4, 2), np.uint8)
        R = np.zeros(4, np.uint8)
        X[0], Z[0], R[0] = xi, zi, ri
        X[1], Z[1], R[1] = xh, zh, rh
        t.set(X, Z, R)
        Pi = pauli_matrix(xi, zi, ri)
        Ph = pauli_matrix(xh, zh, rh)
        commute = np.allclose(Pi @ Ph, Ph @ Pi)
        rc = t.rowsum(1, 0)
        if not commute:
            assert rc == oracle.ORC_EPHASE
            continue
        assert rc == 0
        gx, gz, gr = t.get()
        want = match_pauli(Pi @ Ph, n)
        assert (list(gx[1]), list(gz[1]), int(gr[1])) == want


# ------------------------------------------------------------------- Philox

def load_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            lhs, rhs = line.split("->")
            a = [int(v, 16) for v in lhs.split()]
            rows.append((a[:4], a[4:6], [int(v, 16) for v in rhs.split()]))
    return rows


def test_philox_known_answers():
    rows = load_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(oracle.philox4x32_10(ctr, key)) == want


def test_outcome_bit_counter_layout():
    seed, cid, shot, k = 0x0123456789ABCDEF, 0x1122334455667788, 7, 42
    w = oracle.philox4x32_10([k, shot, cid & 0xFFFFFFFF, cid >> 32],
                             [seed & 0xFFFFFFFF, seed >> 32])
    assert oracle.outcome_bit(seed, cid, shot, k) == (int(w[0]) & 1)
    bits = [oracle.outcome_bit(1, 0, 0, i) for i in range(4000)]
    assert 0.45 < np.mean(bits) < 0.55


# ---------------------------------------------------- brute-force state vector

def stabilizers_hold(t, sv):
    x, z, r = t.get()
    n = t.n
    for i in range(n, 2 * n):
        if not np.allclose(sv.apply_pauli(x[i], z[i], r[i]), sv.psi, atol=1e-9):
            return False
    return True


def run_against_statevector(n, gates, seed, cid=0, shot=0):
    t = oracle.Tableau(n)
    sv = StateVector(n)
    op, q1, q2 = C.decode(gates)
    k = 0
    n_random = 0
    for o, a, b in zip(op, q1, q2):
        o, a, b = int(o), int(a), int(b)
        if o == C.TAB_BARRIER or o == C.TAB_I:
            if o == C.TAB_I:
                t.run(C.encode(o, a, 0).reshape(1))
            continue
        if o in (C.TAB_MZ, C.TAB_MZR):
            p1 = sv.prob_one(a)
            rbit = oracle.outcome_bit(seed, cid, shot, k)
            k += 1
            m, det = t.measure(a, rbit)
            if det:
                assert abs(p1 - m) < 1e-9, (p1, m)
            else:
                assert abs(p1 - 0.5) < 1e-9, p1
                assert m == rbit
                n_random += 1
            sv.project(a, m)
            if o == C.TAB_MZR and m == 1:
                t.x(a)
                sv.apply("X", [a])
        else:
            name = OPNAME[o]
            if name in ONE_Q:
                getattr(t, ONE_Q[name])(a)
                sv.apply(name, [a])
            else:
                getattr(t, TWO_Q[name])(a, b)
                sv.apply(name, [a, b])
        assert stabilizers_hold(t, sv)
    return t, n_random


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_random_circuits_vs_statevector(n):
    for s in range(6 if n < 8 else 3):
        gates = C.random_clifford_ops(n, 60, seed=1000 * n + s, measure_p=0.12,
                                      reset_p=0.06)
        run_against_statevector(n, gates, seed=s + 1, cid=s)


def test_layer_circuit_vs_statevector_n10():
    c = C.config1()
    t, n_random = run_against_statevector(c.n, c.gates, seed=C.PHILOX_SEED)
    assert n_random >= 1


def test_driver_matches_stepwise():
    """orc_run's decoding and measurement counter equal the step-by-step path."""
    n = 6
    gates = C.random_clifford_ops(n, 80, seed=77, measure_p=0.15, reset_p=0.1)
    t1, _ = run_against_statevector(n, gates, seed=9, cid=3, shot=2)
    out, (x, z, r) = oracle.run_circuit(n, gates, seed=9, circuit_id=3, shot=2)
    x1, z1, r1 = t1.get()
    assert np.array_equal(x, x1) and np.array_equal(z, z1) and np.array_equal(r, r1)


# ------------------------------------------------------------ known states

def test_zero_state_measures_zero_deterministically():
    t = oracle.Tableau(5)
    gates = C.encode(np.full(5, C.TAB_MZ), np.arange(5), 0)
    out, det = t.run(gates, with_det=True)
    assert out.tolist() == [0] * 5 and det.all()


def test_x_measures_one():
    t = oracle.Tableau(3)
    g = np.concatenate([C.encode(C.TAB_X, 1, 0).reshape(1),
                        C.encode(np.full(3, C.TAB_MZ), np.arange(3), 0)])
    out, det = t.run(g, with_det=True)
    assert out.tolist() == [0, 1, 0] and det.all()


def test_hadamard_all_random():
    n = 6
    t = oracle.Tableau(n)
    g = np.concatenate([C.encode(np.full(n, C.TAB_H), np.arange(n), 0),
                        C.encode(np.full(n, C.TAB_MZ), np.arange(n), 0)])
    out, det = t.run(g, seed=5, with_det=True)
    assert not det.any()
    assert out.tolist() == [oracle.outcome_bit(5, 0, 0, k) for k in range(n)]


def test_bell_state():
    t = oracle.Tableau(2)
    t.h(0)
    t.cnot(0, 1)
    x, z, r = t.get()
    stabs = {(tuple(x[i]), tuple(z[i]), int(r[i])) for i in (2, 3)}
    # generators of {+XX, +ZZ}: the group must contain both
    group = set()
    for c0, c1 in itertools.product((0, 1), repeat=2):
        M = np.eye(4, dtype=complex)
        for ci, (sx, sz, sr) in zip((c0, c1), sorted(stabs)):
            if ci:
                M = M @ pauli_matrix(sx, sz, sr)
        group.add(tuple(np.round(M, 6).ravel()))
    for P in (pauli_matrix([1, 1], [0, 0]), pauli_matrix([0, 0], [1, 1])):
        assert tuple(np.round(P, 6).ravel()) in group
    for seed in range(1, 6):
        t2 = oracle.Tableau(2)
        g = np.concatenate([C.encode([C.TAB_H, C.TAB_CNOT], [0, 0], [0, 1]),
                            C.encode([C.TAB_MZ, C.TAB_MZ], [0, 1], 0)])
        out, det = t2.run(g, seed=seed, with_det=True)
        assert out[0] == out[1] and not det[0] and det[1]


@pytest.mark.parametrize("n", [3, 7, 12])
def test_ghz(n):
    for seed in range(1, 5):
        t = oracle.Tableau(n)
        g = [C.encode(C.TAB_H, 0, 0).reshape(1)]
        g += [C.encode(C.TAB_CNOT, 0, j).reshape(1) for j in range(1, n)]
        g.append(C.encode(np.full(n, C.TAB_MZ), np.arange(n), 0))
        out, det = t.run(np.concatenate(g), seed=seed, with_det=True)
        assert len(set(out.tolist())) == 1
        assert (not det[0]) and det[1:].all()
        assert out[0] == oracle.outcome_bit(seed, 0, 0, 0)


def test_plus_y_state():
    t = oracle.Tableau(1)
    t.h(0)
    t.s(0)
    x, z, r = t.get()
    assert (x[1, 0], z[1, 0], r[1]) == (1, 1, 0)   # +Y


# ------------------------------------------------------------- invariants

def symplectic_ok(x, z):
    n = x.shape[1]
    M = np.concatenate([x, z], axis=1).astype(np.int64)
    L = np.zeros((2 * n, 2 * n), np.int64)
    L[:n, n:] = np.eye(n, dtype=np.int64)
    L[n:, :n] = np.eye(n, dtype=np.int64)
    return np.array_equal((M @ L @ M.T) % 2, L)


@pytest.mark.parametrize("n", [2, 9, 33, 64])
def test_symplectic_invariant(n):
    gates = C.random_clifford_ops(n, 400, seed=n, measure_p=0.05, reset_p=0.03)
    t = oracle.Tableau(n)
    t.run(gates, seed=3)
    x, z, r = t.get()
    assert symplectic_ok(x, z)


def inverse_gates(gates):
    op, q1, q2 = C.decode(gates)
    inv = {C.TAB_S: C.TAB_SDG, C.TAB_SDG: C.TAB_S}
    op2 = np.array([inv.get(int(o), int(o)) for o in op[::-1]])
    return C.encode(op2, q1[::-1], q2[::-1])


@pytest.mark.parametrize("n", [1, 4, 17, 40])
def test_circuit_then_inverse_is_identity(n):
    gates = C.random_clifford_ops(n, 300, seed=11 * n)
    t = oracle.Tableau(n)
    t.run(gates)
    x, z, r = t.get()
    t.run(inverse_gates(gates))
    x, z, r = t.get()
    ref = oracle.Tableau(n).get()
    assert np.array_equal(x, ref[0]) and np.array_equal(z, ref[1])
    assert np.array_equal(r, ref[2])


def test_repeated_measurement():
    n = 10
    gates = C.random_clifford_ops(n, 200, seed=5)
    for a in range(n):
        t = oracle.Tableau(n)
        t.run(gates)
        m1, _ = t.measure(a, 1)
        m2, d2 = t.measure(a, 0)
        assert d2 and m1 == m2


def test_reset_leaves_zero():
    n = 8
    gates = C.random_clifford_ops(n, 200, seed=8)
    t = oracle.Tableau(n)
    t.run(gates)
    t.run(C.encode(np.full(n, C.TAB_MZR), np.arange(n), 0), seed=4)
    out, det = t.run(C.encode(np.full(n, C.TAB_MZ), np.arange(n), 0), with_det=True)
    assert out.tolist() == [0] * n and det.all()


def test_invalid_inputs_rejected():
    t = oracle.Tableau(4)
    with pytest.raises(RuntimeError):
        t.run(C.encode(C.TAB_H, 4, 0).reshape(1))
    with pytest.raises(RuntimeError):
        t.run(C.encode(C.TAB_CNOT, 1, 1).reshape(1))
    with pytest.raises(RuntimeError):
        t.run(C.encode(18, 0, 0).reshape(1))


# ------------------------------------------- readings the physics leaves open

def test_pivot_is_smallest_stabilizer_row():
    """Reading: the pivot is the smallest stabilizer index with x_pa = 1.

    |++> on two qubits has stabilizers X0 (row 2) and X1 (row 3); after
    CNOT(1,0) row 3 becomes X0 X1, so both rows carry x on qubit 0 and the
    pivot of Z_0 must be row 2, which becomes -Z_0 for outcome 1.
    """
    t = oracle.Tableau(2)
    t.h(0)
    t.h(1)
    t.cnot(1, 0)
    x0, z0, r0 = t.get()
    assert x0[2, 0] == 1 and x0[3, 0] == 1
    m, det = t.measure(0, 1)
    x, z, r = t.get()
    assert not det and m == 1
    assert x[2].tolist() == [0, 0] and z[2].tolist() == [1, 0] and r[2] == 1
    # the old pivot row moved to the paired destabilizer, sign included
    assert x[0].tolist() == x0[2].tolist() and z[0].tolist() == z0[2].tolist()
    assert r[0] == r0[2]


def test_destabilizer_takes_pivot_sign():
    """AG's measurement copies row p, sign included, into row p-n."""
    t = oracle.Tableau(1)
    t.h(0)
    t.z(0)          # stabilizer -X
    x0, z0, r0 = t.get()
    assert r0[1] == 1
    t.measure(0, 0)
    x, z, r = t.get()
    assert (x[0, 0], z[0, 0], r[0]) == (1, 0, 1)
    assert (x[1, 0], z[1, 0], r[1]) == (0, 1, 0)
