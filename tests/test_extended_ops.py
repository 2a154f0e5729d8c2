"""Oracle pins of the extended ops (CPU): X / Y measurement and Pauli noise.

* MX and MY against a state vector that measures with the projectors
  (I +- X)/2 and (I +- Y)/2 directly (not by basis change): deterministic
  outcomes have probability 1, random ones 1/2 and equal the Philox bit, and
  the final stabilizers hold on the projected state.
* Noise: with the probability field 0 nothing happens; op j's Pauli (read
  back from the signs of a one-qubit destabilizer / stabilizer pair) is the
  one the documented Philox rule selects, evaluated here with the oracle's
  Philox (pinned to the Random123 known-answer vectors); the firing rate and
  the X / Y / Z split of DEPOL1 are close to p and 1/3.
"""
import numpy as np
import pytest

import oracle
from tests.statevector import MAT1, StateVector
from tests.test_oracle_pins import stabilizers_hold
from workloads import circuits as C

PAULI = {C.TAB_MX: MAT1["X"], C.TAB_MY: MAT1["Y"]}
NAME1 = {C.TAB_I: "I", C.TAB_X: "X", C.TAB_Y: "Y", C.TAB_Z: "Z", C.TAB_H: "H",
         C.TAB_S: "S", C.TAB_SDG: "SDG"}
NAME2 = {C.TAB_CNOT: "CNOT", C.TAB_CZ: "CZ", C.TAB_SWAP: "SWAP"}


def apply_1q(sv, m, a):
    idx = sv.idx
    b = (idx >> a) & 1
    partner = idx ^ (1 << a)
    psi = sv.psi
    sv.psi = np.where(b == 0, m[0, 0] * psi + m[0, 1] * psi[partner],
                      m[1, 0] * psi[partner] + m[1, 1] * psi)


def prob(sv, m, a, outcome):
    """Probability of eigenvalue (-1)^outcome of the one-qubit Pauli m on a."""
    save = sv.psi.copy()
    proj = 0.5 * (np.eye(2) + (-1) ** outcome * m)
    apply_1q(sv, proj, a)
    p = float(np.vdot(sv.psi, sv.psi).real)
    sv.psi = save
    return p


def project(sv, m, a, outcome):
    apply_1q(sv, 0.5 * (np.eye(2) + (-1) ** outcome * m), a)
    sv.psi /= np.linalg.norm(sv.psi)


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_mx_my_against_projectors(n):
    for s in range(5):
        gates = C.random_extended_ops(n, 70, seed=500 * n + s, p_meas=0.25, p_noise=0.0)
        t = oracle.Tableau(n)
        out, det = t.run(gates, seed=s + 3, circuit_id=s, with_det=True)
        sv = StateVector(n)
        op, q1, q2 = C.decode(gates)
        k = 0
        for o, a, b in zip(op.tolist(), q1.tolist(), q2.tolist()):
            if o in NAME1:
                sv.apply(NAME1[o], [a])
            elif o in NAME2:
                sv.apply(NAME2[o], [a, b])
            elif o in C.MEASURE_ANY:
                m = MAT1["Z"] if o in C.MEASURE else PAULI[o]
                bit = int(out[k])
                p = prob(sv, m, a, bit)
                if det[k]:
                    assert abs(p - 1.0) < 1e-9, (o, p)
                else:
                    assert abs(p - 0.5) < 1e-9, (o, p)
                    assert bit == oracle.outcome_bit(s + 3, s, 0, k)
                project(sv, m, a, bit)
                if o == C.TAB_MZR and bit:
                    sv.apply("X", [a])
                k += 1
        assert k == out.size
        assert stabilizers_hold(t, sv)


def test_mx_my_known_states():
    def run(prep, op):
        n = 1
        g = np.concatenate([C.encode(np.array(prep, dtype=np.int64), 0, 0).reshape(-1),
                            C.encode(op, 0, 0).reshape(1), C.encode(op, 0, 0).reshape(1)])
        out, det = oracle.Tableau(n).run(g, with_det=True)
        return out.tolist(), det.tolist()
    assert run([C.TAB_H], C.TAB_MX) == ([0, 0], [True, True])                  # |+>
    assert run([C.TAB_X, C.TAB_H], C.TAB_MX) == ([1, 1], [True, True])         # |->
    assert run([C.TAB_H, C.TAB_S], C.TAB_MY) == ([0, 0], [True, True])         # |+i>
    assert run([C.TAB_H, C.TAB_SDG], C.TAB_MY) == ([1, 1], [True, True])       # |-i>
    out, det = run([], C.TAB_MX)                                               # |0>: random, then repeatable
    assert det == [False, True] and out[0] == out[1]


def applied_paulis(n, ops, field, seed, cid, shot):
    """Run noise op ops[i] on qubit i of |0^n>; read which Pauli hit each qubit
    from the signs of destabilizer X_i and stabilizer Z_i."""
    g = C.encode(np.array(ops, dtype=np.int64), np.arange(n), field)
    _, (x, z, r) = oracle.run_circuit(n, g, seed=seed, circuit_id=cid, shot=shot)
    return [{(0, 0): "I", (0, 1): "X", (1, 1): "Y", (1, 0): "Z"}[(int(r[i]), int(r[n + i]))]
            for i in range(n)]


def expected_paulis(ops, field, seed, cid, shot):
    out = []
    for j, op in enumerate(ops):
        w = oracle.philox4x32_10([j, shot, cid & 0xFFFFFFFF, cid >> 32],
                                 [seed & 0xFFFFFFFF, (seed >> 32) ^ 0x4E4F4953])
        if (int(w[0]) >> 4) >= field:
            out.append("I")
        elif op == C.TAB_XERR:
            out.append("X")
        elif op == C.TAB_ZERR:
            out.append("Z")
        else:
            out.append("XYZ"[(int(w[1]) * 3) >> 32])
    return out


def test_noise_rule_matches_philox():
    rng = np.random.default_rng(5)
    n = 400
    ops = rng.choice(C.NOISE, size=n).tolist()
    for field, seed, cid, shot in [(C.noise_field(0.4), 7, 3, 2),
                                   (C.noise_field(0.999), (1 << 40) + 5, (1 << 33) + 1, 9)]:
        assert applied_paulis(n, ops, field, seed, cid, shot) == \
            expected_paulis(ops, field, seed, cid, shot)


def test_noise_zero_probability_is_identity():
    n = 50
    base = C.random_clifford_ops(n, 300, seed=3)
    noise = C.encode(np.full(n, C.TAB_DEPOL1), np.arange(n), 0)
    _, want = oracle.run_circuit(n, base)
    _, got = oracle.run_circuit(n, np.concatenate([base[:150], noise, base[150:]]))
    for a, b in zip(want, got):
        assert np.array_equal(a, b)


def test_depolarizing_rates():
    n = 6000
    got = applied_paulis(n, [C.TAB_DEPOL1] * n, C.noise_field(0.6), 11, 0, 0)
    fired = [p for p in got if p != "I"]
    assert abs(len(fired) / n - 0.6) < 0.03
    for p in "XYZ":
        assert abs(fired.count(p) / len(fired) - 1 / 3) < 0.03


# ---------------------------------------------- expectation values (oracle)

def sv_expect(sv, codes):
    x = [c & 1 for c in codes]
    z = [c >> 1 for c in codes]
    return float(np.vdot(sv.psi, sv.apply_pauli(x, z, 0)).real)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_expectation_all_paulis_vs_statevector(n):
    """Every one of the 4^n Pauli strings on random stabilizer states."""
    import itertools
    for s in range(4):
        gates = C.random_clifford_ops(n, 40, seed=700 * n + s)
        t = oracle.Tableau(n)
        t.run(gates)
        sv = StateVector(n)
        op, q1, q2 = C.decode(gates)
        for o, a, b in zip(op.tolist(), q1.tolist(), q2.tolist()):
            sv.apply(NAME1[o], [a]) if o in NAME1 else sv.apply(NAME2[o], [a, b])
        before = t.get()
        for codes in itertools.product(range(4), repeat=n):
            want = sv_expect(sv, codes)
            assert abs(want - t.expect(codes)) < 1e-9, (codes, want)
        for a, b in zip(before, t.get()):
            assert np.array_equal(a, b)


# -------------------------------------------- host lowering (library, CPU)

def test_lowering_equals_op_by_op():
    """tab_lower_ops (what tab_apply runs) gives, in the oracle, the outcomes
    and tableau of the extended ops taken one by one; a run of X / Y
    measurements on distinct qubits becomes one block of Z measurements."""
    tab = pytest.importorskip("paper_2408_00384_gb300.tab")
    rng = np.random.default_rng(4)
    for n, seed in [(7, 3), (40, 5), (130, 8)]:
        base = C.random_extended_ops(n, 400, seed=seed, p_meas=0.15, p_noise=0.1)
        qs = rng.choice(n, size=min(n, 30), replace=False)
        kinds = rng.choice([C.TAB_MX, C.TAB_MY, C.TAB_MZ, C.TAB_MZR], size=qs.size)
        run = C.encode(kinds, qs, 0)
        bar = C.encode(C.TAB_BARRIER, 0, 0).reshape(1)
        g = np.concatenate([base[:200], bar, run, bar, base[200:]])
        low, nk = tab.lower_ops(n, g, seed=9, circuit_id=2, shot=1)
        assert not np.isin(C.decode(low)[0], (13, 14, 15, 16, 17)).any()
        assert nk == int(np.isin(C.decode(g)[0], C.NOISE).sum())
        want_out, want = oracle.run_circuit(n, g, seed=9, circuit_id=2, shot=1)
        got_out, got = oracle.run_circuit(n, low, seed=9, circuit_id=2, shot=1)
        assert np.array_equal(got_out, want_out)
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        # the run's measurements are consecutive in the lowered list
        op = C.decode(low)[0]
        m = np.isin(op, C.MEASURE)
        runs = np.diff(np.concatenate([[0], m.astype(np.int8), [0]]))
        longest = (np.flatnonzero(runs == -1) - np.flatnonzero(runs == 1)).max()
        assert longest >= qs.size


def test_expectation_after_measurements_vs_statevector():
    """orc_expect on post-measurement states (MZ, MZR, MX, MY in the circuit),
    every Pauli string against the projected state vector; a measured Pauli
    has expectation (-1)^outcome right after its measurement."""
    import itertools
    for n in (2, 3, 4):
        for s in range(3):
            gates = C.random_extended_ops(n, 50, seed=900 * n + s, p_meas=0.2, p_noise=0.0)
            t = oracle.Tableau(n)
            out = t.run(gates, seed=s + 1, circuit_id=s)
            sv = StateVector(n)
            op, q1, q2 = C.decode(gates)
            k = 0
            for o, a, b in zip(op.tolist(), q1.tolist(), q2.tolist()):
                if o in NAME1:
                    sv.apply(NAME1[o], [a])
                elif o in NAME2:
                    sv.apply(NAME2[o], [a, b])
                elif o in C.MEASURE_ANY:
                    m = MAT1["Z"] if o in C.MEASURE else PAULI[o]
                    project(sv, m, a, int(out[k]))
                    if o == C.TAB_MZR and out[k]:
                        sv.apply("X", [a])
                    k += 1
            for codes in itertools.product(range(4), repeat=n):
                assert abs(sv_expect(sv, codes) - t.expect(codes)) < 1e-9, (n, s, codes)
    # right after MX / MY on qubit 0, <X_0> / <Y_0> = (-1)^outcome
    for kind, code in ((C.TAB_MX, 1), (C.TAB_MY, 3)):
        g = np.concatenate([C.random_clifford_ops(3, 30, seed=kind),
                            C.encode(kind, 0, 0).reshape(1)])
        t = oracle.Tableau(3)
        o = t.run(g, seed=2)
        assert t.expect([code, 0, 0]) == (-1) ** int(o[-1])


def test_noise_threshold_is_strict():
    """The draw fires when (word 0 >> 4) < field: at field equal to the drawn
    value it does not, one above it does (a boundary no rate test sees)."""
    seed, cid, shot = 12345, 6, 2
    w = oracle.philox4x32_10([0, shot, cid, 0], [seed & 0xFFFFFFFF, (seed >> 32) ^ 0x4E4F4953])
    v = int(w[0]) >> 4
    for field, fires in ((v, False), (v + 1, True)):
        if field >= (1 << 28):
            continue
        g = C.encode(C.TAB_XERR, 0, field).reshape(1)
        _, (x, z, r) = oracle.run_circuit(1, g, seed=seed, circuit_id=cid, shot=shot)
        assert bool(r[1]) == fires, (field, v)


def test_library_noise_threshold_matches():
    """The library's host lowering (what tab_apply runs) takes the same strict
    threshold: field == drawn value -> no Pauli, one above -> X."""
    tab = pytest.importorskip("paper_2408_00384_gb300.tab")
    seed, cid, shot = 12345, 6, 2
    w = oracle.philox4x32_10([0, shot, cid, 0], [seed & 0xFFFFFFFF, (seed >> 32) ^ 0x4E4F4953])
    v = int(w[0]) >> 4
    for field, fires in ((v, False), (v + 1, True)):
        if field >= (1 << 28):
            continue
        low, nk = tab.lower_ops(1, C.encode(C.TAB_XERR, 0, field).reshape(1), seed=seed,
                                circuit_id=cid, shot=shot)
        assert nk == 1
        assert C.decode(low)[0].tolist() == ([C.TAB_X] if fires else [])


def test_host_validation_through_lowering():
    """The host validator every entry point runs first (exercised on the CPU
    through tab_lower_ops): out-of-range qubits, a two-qubit op on one qubit
    and unknown ops are refused with the documented codes; barriers carry no
    qubits to check."""
    tab = pytest.importorskip("paper_2408_00384_gb300.tab")
    n = 5
    ok = np.concatenate([C.encode([C.TAB_H, C.TAB_CNOT, C.TAB_BARRIER, C.TAB_MX],
                                  [0, 1, (1 << 28) - 1, 4], [0, 4, 7, 0])])
    low, _ = tab.lower_ops(n, ok)
    assert low.size >= 3
    cases = [(C.encode(C.TAB_H, n, 0), tab.TAB_ERANGE),
             (C.encode(C.TAB_CZ, 1, n), tab.TAB_ERANGE),
             (C.encode(C.TAB_SWAP, 2, 2), tab.TAB_EINVAL),
             (C.encode(18, 0, 0), tab.TAB_EINVAL),
             (C.encode(C.TAB_MY, n + 3, 0), tab.TAB_ERANGE),
             (C.encode(C.TAB_DEPOL1, n, 5), tab.TAB_ERANGE)]
    for word, code in cases:
        g = np.concatenate([ok, np.asarray(word, np.uint64).reshape(1), ok])
        with pytest.raises(tab.TabError) as ei:
            tab.lower_ops(n, g)
        assert ei.value.code == code, (word, ei.value.code)
