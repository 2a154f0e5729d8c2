"""GPU path vs the CPU oracle, bit for bit, through the C ABI.

Every comparison is element by element: all outcome bytes and every tableau bit
(x, z and sign of all 2n rows).  Both engines (single-CTA and grid) are
checked.  The oracle's inputs come from the seeded generators only.
"""
import numpy as np
import pytest

import oracle
from workloads import circuits as C

pytestmark = pytest.mark.gpu

from paper_2408_00384_gb300 import tab  # noqa: E402  (fails loudly when libtab.so is missing)


def gpu_run(n, gates, seed=1, cid=0, shot=0, engine=None):
    with tab.Tableau(n) as t:
        if engine is not None:
            try:
                t.set_engine(engine)
            except tab.TabError as e:
                if e.code == tab.TAB_ERANGE:
                    pytest.skip(f"engine {engine} does not hold n={n}")
                raise
        t.set_rng(seed, cid, shot)
        t.apply(gates)
        out = t.read_outcomes()
        x, z, r = t.export()
    return out, (x, z, r)


_ORACLE_CACHE = {}


def oracle_result(n, gates, seed, cid, shot):
    """The oracle's run, computed once per distinct case and shared by every
    engine that is compared with it (the large cases take the CPU seconds)."""
    key = (n, seed, cid, shot, gates.size, hash(gates.tobytes()))
    if key not in _ORACLE_CACHE:
        if len(_ORACLE_CACHE) >= 2:
            _ORACLE_CACHE.clear()
        _ORACLE_CACHE[key] = oracle.run_circuit(n, gates, seed=seed, circuit_id=cid, shot=shot)
    return _ORACLE_CACHE[key]


def assert_same(n, gates, seed=1, cid=0, shot=0, engine=None):
    want_out, want = oracle_result(n, gates, seed, cid, shot)
    got_out, got = gpu_run(n, gates, seed, cid, shot, engine)
    assert np.array_equal(got_out, want_out), (n, engine, np.nonzero(got_out != want_out)[0][:10])
    for name, g, w in zip("xzr", got, want):
        bad = np.argwhere(g != w)
        assert bad.size == 0, (n, engine, name, bad[:10].tolist())


ENGINES = [tab.ENGINE_SINGLE_CTA, tab.ENGINE_GRID, tab.ENGINE_STREAM]


@pytest.mark.parametrize("engine", ENGINES)
def test_config1(engine):
    c = C.config1()
    assert_same(c.n, c.gates, seed=C.PHILOX_SEED, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200])
def test_random_ops_all_gates(engine, n):
    gates = C.random_clifford_ops(n, 400, seed=7 * n + 1, measure_p=0.08, reset_p=0.04)
    assert_same(n, gates, seed=3, cid=n, shot=1, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("n,depth", [(257, 12), (480, 6), (511, 5), (640, 4)])
def test_layer_circuits_final_measure(engine, n, depth):
    c = C.random_layer_circuit(n, depth, seed=n, meas_every=3, meas_frac=0.05)
    assert_same(n, c.gates, seed=11, engine=engine)


@pytest.mark.parametrize("engine", [tab.ENGINE_GRID, tab.ENGINE_STREAM])
@pytest.mark.parametrize("n", [700, 1000, 2049, 2400, 4100, 8000])
def test_larger_tableaus(engine, n):
    # the oracle's rowsum costs ~n^2 cache misses per measurement on the CPU:
    # at most ~24 measurements keeps every case within seconds
    c = C.random_layer_circuit(n, 8, seed=n, meas_every=4, meas_frac=min(0.02, 12.0 / n),
                               final_measure=n <= 1000)
    assert_same(n, c.gates, seed=5, engine=engine)


_E = tab
@pytest.mark.parametrize("n,engine,want", [
    (200, _E.ENGINE_AUTO, _E.ENGINE_SINGLE_CTA),
    (1000, _E.ENGINE_AUTO, _E.ENGINE_GRID),
    (1000, _E.ENGINE_GRID, _E.ENGINE_GRID),
    (4100, _E.ENGINE_GRID, _E.ENGINE_GRID),
    (8000, _E.ENGINE_GRID, _E.ENGINE_STREAM),
    (10000, _E.ENGINE_AUTO, _E.ENGINE_STREAM),
    (1000, _E.ENGINE_STREAM, _E.ENGINE_STREAM),
])
def test_engine_resolution(n, engine, want):
    """The engine a measurement run takes: the parity cases of each engine
    above exercise that engine's kernel, not a fallback."""
    with tab.Tableau(n) as t:
        t.set_engine(engine)
        got, ctas = t.engine_resolved()
    assert got == want, (n, engine, got)
    assert ctas >= 1


@pytest.mark.parametrize("engine", [tab.ENGINE_AUTO, tab.ENGINE_GRID, tab.ENGINE_STREAM])
def test_config2_full(engine):
    """n=1000, 1000 random layers, final MZ on all qubits: full compare."""
    c = C.config2()
    assert_same(c.n, c.gates, seed=C.PHILOX_SEED, engine=engine)


def test_config3_prefix_full_size():
    """n=10,000: the first 10 layers and the first 24 MZR of the first round,
    on the full-size tableau, compared with the oracle bit for bit."""
    c = C.config3()
    op, _, _ = C.decode(c.gates)
    first_meas = int(np.argmax(np.isin(op, C.MEASURE)))
    prefix = c.gates[:first_meas + 24]
    assert_same(c.n, prefix, seed=C.PHILOX_SEED)


def commutation_ok(x, z, rows_a, rows_b, n):
    """Tableau rows i, j anticommute iff {i, j} = {k, k+n}."""
    xa, za = x[rows_a].astype(np.int64), z[rows_a].astype(np.int64)
    xb, zb = x[rows_b].astype(np.int64), z[rows_b].astype(np.int64)
    sym = (xa @ zb.T + za @ xb.T) % 2
    want = ((rows_a[:, None] % n == rows_b[None, :] % n) & (rows_a[:, None] != rows_b[None, :]))
    return np.array_equal(sym, want.astype(np.int64))


def test_config3_full_invariants():
    """Whole config 3 on the GPU: the tableau stays symplectic (sampled row
    pairs), and the qubits of the last MZR round measure 0 deterministically."""
    c = C.config3()
    with tab.Tableau(c.n) as t:
        t.set_rng(C.PHILOX_SEED, 0, 0)
        t.apply(c.gates)
        out = t.read_outcomes()
        assert out.size == c.n_meas
        x, z, r = t.export()
        op, q1, _ = C.decode(c.gates)
        last_round = q1[np.isin(op, C.MEASURE)][-(c.n // 10):][:64]
        again = t.measure(last_round.astype(np.int32), seed=99)
    assert not again.any()
    assert 0.4 < out.mean() < 0.6
    rng = np.random.default_rng(0)
    rows = rng.choice(2 * c.n, size=300, replace=False)
    assert commutation_ok(x, z, rows, rows, c.n)
    paired = np.unique(np.concatenate([rows[:100] % c.n, rows[:100] % c.n + c.n]))
    assert commutation_ok(x, z, paired, paired, c.n)


def test_empty_and_measure_first():
    assert_same(5, np.zeros(0, np.uint64))
    g = C.encode(np.full(4, C.TAB_MZ), np.array([0, 1, 1, 3]), 0)
    for e in ENGINES:
        assert_same(4, g, engine=e)


def test_invalid_gate_applies_nothing():
    n = 8
    good = C.random_clifford_ops(n, 50, seed=1)
    bad = np.concatenate([good, C.encode(C.TAB_H, n, 0).reshape(1)])
    with tab.Tableau(n) as t:
        t.apply(good)
        before = t.export()
        with pytest.raises(tab.TabError) as ei:
            t.apply(bad)
        assert ei.value.code == tab.TAB_ERANGE
        with pytest.raises(tab.TabError) as ei:
            t.apply(C.encode(C.TAB_CZ, 2, 2).reshape(1))
        assert ei.value.code == tab.TAB_EINVAL
        after = t.export()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 33, 64, 100, 257, 600])
def test_uniform_random_cliffords(n):
    """The paper's own workload (uniformly random Cliffords, no measurements)
    on the default engines, bit for bit against the oracle."""
    c = C.random_clifford(n, C.splitmix64(4242 + n))
    assert_same(n, c.gates)


@pytest.mark.parametrize("engine", [tab.ENGINE_GRID, tab.ENGINE_STREAM])
def test_uniform_random_clifford_engines(engine):
    c = C.random_clifford(300, C.splitmix64(4343))
    assert_same(300, c.gates, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("n", [1, 2, 5, 33, 130, 300])
def test_extended_ops(engine, n):
    """MX / MY and the three noise ops among every other op, bit for bit
    against the oracle (noise draws under a non-default RNG context)."""
    g = C.random_extended_ops(n, 400, seed=77 + n, p_meas=0.1, p_noise=0.15, noise_p=0.4)
    assert_same(n, g, seed=5, cid=2, shot=1, engine=engine)


def test_extended_ops_long_list():
    """Extended ops in a list long enough for the pipelined apply."""
    c = C.random_layer_circuit(700, 140, seed=23, final_measure=False)
    rng = np.random.default_rng(1)
    pos = np.sort(rng.choice(c.gates.size, 3000, replace=False))
    kind = rng.choice([C.TAB_MX, C.TAB_MY, C.TAB_DEPOL1, C.TAB_XERR, C.TAB_ZERR], size=3000)
    field = np.where(np.isin(kind, C.NOISE), C.noise_field(0.3), 0)
    g = np.insert(c.gates, pos, C.encode(kind, rng.integers(0, 700, size=3000), field))
    assert g.size >= (1 << 17)
    assert_same(700, g, seed=4, cid=1, engine=tab.ENGINE_GRID)


def test_extended_ops_in_programs():
    """Programs take MX / MY (lowered once) but not noise ops (a program
    replays under any RNG setting, and noise is drawn per shot)."""
    n = 40
    g = C.random_extended_ops(n, 300, seed=8, p_noise=0.0)
    with tab.Tableau(n) as t:
        t.set_rng(3, 0, 0)
        p = tab.Program(n, g)
        t.run(p)
        out = t.read_outcomes()
        got = t.export()
        p.close()
    want_out, want = oracle_result(n, g, 3, 0, 0)
    assert np.array_equal(out, want_out)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    noisy = C.random_extended_ops(n, 60, seed=9, p_meas=0.0, p_noise=0.5)
    with pytest.raises(tab.TabError) as ei:
        tab.Program(n, noisy)
    assert ei.value.code == tab.TAB_EINVAL


def _expect_cases(n, x, z, rng):
    """Pauli strings (k x n codes) for a state with tableau rows (x, z): random
    dense and sparse strings, single-qubit X_a / Z_a, and products of random
    stabilizer subsets (which have expectation +-1)."""
    out = [rng.integers(0, 4, size=n) for _ in range(6)]
    for _ in range(6):
        s = np.zeros(n, np.int64)
        sup = rng.choice(n, size=min(n, 3), replace=False)
        s[sup] = rng.integers(1, 4, size=sup.size)
        out.append(s)
    for a in rng.choice(n, size=min(n, 4), replace=False):
        for code in (1, 2):
            s = np.zeros(n, np.int64)
            s[a] = code
            out.append(s)
    for _ in range(12):
        pick = rng.integers(0, 2, size=n).astype(bool)
        px = np.bitwise_xor.reduce(x[n:][pick].astype(np.int64), axis=0) if pick.any() else np.zeros(n, np.int64)
        pz = np.bitwise_xor.reduce(z[n:][pick].astype(np.int64), axis=0) if pick.any() else np.zeros(n, np.int64)
        out.append(px | (pz << 1))
    return np.array(out, dtype=np.uint8)


@pytest.mark.parametrize("engine", [tab.ENGINE_AUTO, tab.ENGINE_GRID])
@pytest.mark.parametrize("n", [1, 3, 31, 32, 33, 100, 257, 1000, 2100])
def test_expectation_values(n, engine):
    """tab_expect against the oracle's product-of-stabilizers expectation, on
    random states; the state is left unchanged."""
    import oracle as orc
    if n <= 300:
        gates = C.random_clifford(n, C.splitmix64(5150 + n)).gates
    else:
        gates = C.random_layer_circuit(n, 8, seed=n, final_measure=False).gates
    t_o = orc.Tableau(n)
    t_o.run(gates)
    x, z, _ = t_o.get()
    cases = _expect_cases(n, x, z, np.random.default_rng(n))
    want = np.array([t_o.expect(s) for s in cases], dtype=np.int8)
    assert (want != 0).sum() >= 12
    with tab.Tableau(n) as t:
        try:
            t.set_engine(engine)
        except tab.TabError as e:
            if e.code == tab.TAB_ERANGE:
                pytest.skip(f"engine {engine} does not hold n={n}")
            raise
        t.apply(gates)
        before = t.export()
        got = t.expect(cases)
        after = t.export()
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


def test_expectation_strings_and_errors():
    with tab.Tableau(2) as t:
        t.apply(np.array([C.encode(C.TAB_H, 0, 0), C.encode(C.TAB_CNOT, 0, 1)], np.uint64))
        assert t.expect(["XX", "ZZ", "YY", "XI", "IZ", "II"]).tolist() == [1, 1, -1, 0, 0, 1]
        with pytest.raises(tab.TabError) as ei:
            t.expect(np.array([[0, 4]], np.uint8))
        assert ei.value.code == tab.TAB_EINVAL


def _sv_name(o):
    return {C.TAB_I: "I", C.TAB_X: "X", C.TAB_Y: "Y", C.TAB_Z: "Z", C.TAB_H: "H",
            C.TAB_S: "S", C.TAB_SDG: "SDG", C.TAB_CNOT: "CNOT", C.TAB_CZ: "CZ",
            C.TAB_SWAP: "SWAP"}[o]


def _phase_fixed(psi):
    k = int(np.flatnonzero(np.abs(psi) > 1e-9)[0])
    return psi * (np.conj(psi[k]) / abs(psi[k]))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_statevector_export(n):
    """tab_statevector against a brute-force state vector of the same circuit
    (gate matrices), up to the documented global phase; the handle's state is
    unchanged."""
    from tests.statevector import StateVector
    gates = C.random_clifford(n, C.splitmix64(6060 + n)).gates
    sv = StateVector(n)
    op, q1, q2 = C.decode(gates)
    for o, a, b in zip(op.tolist(), q1.tolist(), q2.tolist()):
        sv.apply(_sv_name(o), [a] if o in C.ONE_QUBIT else [a, b])
    with tab.Tableau(n) as t:
        t.apply(gates)
        before = t.export()
        v = t.statevector()
        after = t.export()
    assert np.allclose(v, _phase_fixed(sv.psi), atol=1e-5)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


def test_statevector_after_measurement_and_expectations():
    """A post-measurement state (outcomes read back), and at n = 16 the
    exported vector reproduces tab_expect on stabilizer products."""
    from tests.statevector import StateVector
    n = 6
    g = np.concatenate([C.encode(C.TAB_H, 0, 0).reshape(1),
                        C.encode(np.full(n - 1, C.TAB_CNOT), 0, np.arange(1, n)),
                        C.encode(C.TAB_H, 2, 0).reshape(1),
                        C.encode(C.TAB_MZ, 2, 0).reshape(1),
                        C.encode(C.TAB_S, 4, 0).reshape(1)])
    with tab.Tableau(n) as t:
        t.set_rng(7, 0, 0)
        t.apply(g)
        m = int(t.read_outcomes()[0])
        v = t.statevector()
    sv = StateVector(n)
    sv.apply("H", [0])
    for j in range(1, n):
        sv.apply("CNOT", [0, j])
    sv.apply("H", [2])
    sv.project(2, m)
    sv.apply("S", [4])
    assert np.allclose(v, _phase_fixed(sv.psi), atol=1e-5)

    n = 16
    gates = C.random_clifford(n, C.splitmix64(6161)).gates
    with tab.Tableau(n) as t:
        t.apply(gates)
        v = t.statevector().astype(np.complex128)
        x, z, _ = t.export()
        rng = np.random.default_rng(3)
        cases = []
        for _ in range(8):
            pick = rng.integers(0, 2, size=n).astype(bool)
            px = np.bitwise_xor.reduce(x[n:][pick].astype(np.int64), axis=0)
            pz = np.bitwise_xor.reduce(z[n:][pick].astype(np.int64), axis=0)
            cases.append(px | (pz << 1))
        cases += [rng.integers(0, 4, size=n) for _ in range(4)]
        cases = np.array(cases, dtype=np.uint8)
        want = t.expect(cases)
    assert abs(np.vdot(v, v).real - 1.0) < 1e-5
    idx = np.arange(1 << n)
    for codes, w in zip(cases, want):
        xm = int(sum(int(c & 1) << j for j, c in enumerate(codes)))
        zm = int(sum(int(c >> 1) << j for j, c in enumerate(codes)))
        ny = int(sum(1 for c in codes if c == 3))
        par = np.array([bin(int(u)).count("1") & 1 for u in (idx & zm)])
        pv = np.zeros_like(v)
        pv[idx ^ xm] = v * np.where(par == 1, -1, 1)
        e = np.vdot(v, pv * (1j ** ny))
        assert abs(e - w) < 1e-4, (codes, e, w)


@pytest.mark.parametrize("n,shards", [(1, 1), (33, 2), (64, 2), (100, 3), (129, 4), (257, 5),
                                      (300, 1), (700, 7)])
def test_sharded_tableau(n, shards):
    """Rows split over shards driven by host threads (pivot all-reduce, row
    broadcast, partial-product gather): outcomes and the gathered tableau
    bit for bit against the oracle, over two apply calls."""
    g = C.random_clifford_ops(n, 600, seed=90 + n, measure_p=0.08, reset_p=0.04)
    want_out, want = oracle_result(n, g, 6, 1, 0)
    with tab.ShardedTableau(n, shards) as t:
        t.set_rng(6, 1, 0)
        t.apply(g[:300])
        t.apply(g[300:])
        out = t.read_outcomes()
        got = t.export()
    assert np.array_equal(out, want_out)
    for name, a, b in zip("xzr", got, want):
        assert np.array_equal(a, b), name


def test_sharded_ghz_and_layers():
    """Deterministic outcomes across shards (GHZ: one random outcome, then
    equal ones) and a random-layer circuit with a final measurement."""
    n = 200
    g = np.concatenate([C.encode(C.TAB_H, 0, 0).reshape(1),
                        C.encode(np.full(n - 1, C.TAB_CNOT), np.arange(n - 1), np.arange(1, n)),
                        C.encode(np.full(n, C.TAB_MZ), np.arange(n)[::-1].copy(), 0)])
    with tab.ShardedTableau(n, 4) as t:
        t.apply(g)
        out = t.read_outcomes()
    assert len(set(out.tolist())) == 1
    c = C.random_layer_circuit(300, 20, seed=5)
    want_out, want = oracle_result(c.n, c.gates, 2, 0, 0)
    with tab.ShardedTableau(c.n, 3) as t:
        t.set_rng(2, 0, 0)
        t.apply(c.gates)
        assert np.array_equal(t.read_outcomes(), want_out)
        for a, b in zip(t.export(), want):
            assert np.array_equal(a, b)


def test_pipelined_apply_mid_circuit_measurements():
    """A list of more than 2^17 words on the grid engine is compiled in 2^16-
    word chunks while earlier chunks already run; MZR rounds every 5 layers put
    measurement runs across chunk boundaries.  Compared with the oracle bit for
    bit, and with the same list applied in pieces that each run whole."""
    c = C.random_layer_circuit(700, 140, seed=21, meas_every=5, meas_frac=0.05)
    assert c.gates.size >= (1 << 17)
    assert_same(c.n, c.gates, seed=3, engine=tab.ENGINE_GRID)
    with tab.Tableau(c.n) as t:
        t.set_engine(tab.ENGINE_GRID)
        t.set_rng(3, 0, 0)
        for s in range(0, c.gates.size, 40_000):
            t.apply(c.gates[s:s + 40_000])
        out = t.read_outcomes()
        got = t.export()
    want_out, want = oracle_result(c.n, c.gates, 3, 0, 0)
    assert np.array_equal(out, want_out)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_pipelined_apply_invalid_word_applies_nothing():
    """The long-list path validates the whole list before its first launch."""
    c = C.random_layer_circuit(600, 160, seed=22, final_measure=False)
    bad = np.concatenate([c.gates, C.encode(C.TAB_CNOT, 3, 600).reshape(1)])
    assert bad.size >= (1 << 17)
    with tab.Tableau(c.n) as t:
        t.set_engine(tab.ENGINE_GRID)
        t.apply(c.gates[:1000])
        before = t.export()
        with pytest.raises(tab.TabError) as ei:
            t.apply(bad)
        assert ei.value.code == tab.TAB_ERANGE
        after = t.export()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("engine", ENGINES)
def test_checkpoint_resume(engine):
    n = 150
    gates = C.random_clifford_ops(n, 600, seed=42, measure_p=0.05, reset_p=0.05)
    want_out, want = oracle.run_circuit(n, gates, seed=8, circuit_id=2, shot=5)
    half = 300
    op, _, _ = C.decode(gates[:half])
    k = int(np.isin(op, C.MEASURE).sum())
    with tab.Tableau(n) as t:
        t.set_engine(engine)
        t.set_rng(8, 2, 5)
        t.apply(gates[:half])
        out1 = t.read_outcomes()
        snap = t.export()
    with tab.Tableau(n) as t2:
        t2.set_engine(engine)
        t2.set_rng(8, 2, 5)
        t2.import_(*snap, meas_counter=k)
        t2.apply(gates[half:])
        out2 = t2.read_outcomes()
        got = t2.export()
    assert np.array_equal(np.concatenate([out1, out2]), want_out)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_measure_call_seed():
    n = 40
    gates = C.random_clifford_ops(n, 300, seed=3)
    qs = np.array([5, 1, 39, 5, 0], np.int32)
    t_or = oracle.Tableau(n)
    t_or.run(gates)
    want = t_or.run(C.encode(np.full(qs.size, C.TAB_MZ), qs, 0), seed=1234)
    for e in ENGINES:
        with tab.Tableau(n) as t:
            t.set_engine(e)
            t.apply(gates)
            got = t.measure(qs, seed=1234)
        assert np.array_equal(got, want)


def test_create_on_torch_memory_and_stream():
    torch = pytest.importorskip("torch")
    n = 300
    c = C.random_layer_circuit(n, 10, seed=5)
    want_out, want = oracle.run_circuit(n, c.gates, seed=1)
    mem = torch.empty(tab.bytes_required(n), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with tab.Tableau(n, stream=s, memory=mem) as t:
        t.set_engine(tab.ENGINE_GRID)
        t.apply(c.gates)
        out = t.read_outcomes()
        got = t.export()
    assert np.array_equal(out, want_out)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_pipelined_apply_on_user_stream_and_stream_switch():
    """Two pipelined applies, the first on a caller's stream and the second
    after a switch to another stream: the copy stream and the staging areas
    follow the stream order, and the result is the oracle's."""
    torch = pytest.importorskip("torch")
    c = C.random_layer_circuit(600, 300, seed=31)
    half = c.gates.size // 2
    assert half >= (1 << 17)
    want_out, want = oracle_result(c.n, c.gates, 1, 0, 0)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with tab.Tableau(c.n, stream=s1) as t:
        t.set_engine(tab.ENGINE_GRID)
        t.apply(c.gates[:half])
        t.set_stream(s2)
        t.apply(c.gates[half:])
        out = t.read_outcomes()
        got = t.export()
    assert np.array_equal(out, want_out)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_next_step_calls_reject_bad_arguments():
    with tab.Tableau(27) as t:
        with pytest.raises(tab.TabError) as ei:
            t.statevector()
        assert ei.value.code == tab.TAB_ERANGE
        assert t.expect(np.zeros((0, 27), np.uint8)).size == 0
    with pytest.raises(tab.TabError) as ei:
        tab.ShardedTableau(64, 3)  # 64 qubits hold two 32-row words
    assert ei.value.code == tab.TAB_ERANGE
    with tab.ShardedTableau(100, 2) as t:
        with pytest.raises(tab.TabError) as ei:
            t.apply(C.encode(C.TAB_MX, 3, 0).reshape(1))
        assert ei.value.code == tab.TAB_EINVAL


def test_compiled_program_replay():
    c = C.random_layer_circuit(180, 20, seed=9)
    want_out, want = oracle.run_circuit(c.n, c.gates, seed=4)
    prog = tab.Program(c.n, c.gates)
    info = prog.info()
    assert info["n_gates"] == c.n_gates and info["n_meas"] == c.n_meas
    for e in ENGINES:
        with tab.Tableau(c.n) as t:
            t.set_engine(e)
            for _ in range(2):
                t.reset()
                t.set_rng(4, 0, 0)
                t.run(prog)
                out = t.read_outcomes()
                assert np.array_equal(out, want_out)
            got = t.export()
        for g, w in zip(got, want):
            assert np.array_equal(g, w)


def test_batch_small_vs_oracle():
    rng = np.random.default_rng(1)
    circuits = []
    for c in range(24):
        n = int(rng.integers(1, 90))
        depth = int(rng.integers(1, 12))
        circ = C.random_layer_circuit(n, depth, seed=100 + c, meas_every=4 if c % 3 == 0 else 0,
                                      meas_frac=0.2)
        circuits.append((n, circ.gates, int(rng.integers(1, 5)), 1000 + c))
    res = tab.batch_run(circuits, seed=77)
    for (n, g, shots, cid), got in zip(circuits, res):
        for s in range(shots):
            want, _ = oracle.run_circuit(n, g, seed=77, circuit_id=cid, shot=s)
            assert np.array_equal(got[s], want), (n, cid, s)


def test_batch_run_packed_capacity_and_counts():
    """tab_batch_run_packed: the counts it returns are tab_meas_counts', the
    bytes equal tab_batch_run's, and a buffer one byte short is refused with
    TAB_ERANGE without a write past its end (chunks of two circuits, so the
    refusal comes after earlier chunks ran)."""
    rng = np.random.default_rng(5)
    circuits = []
    for c in range(12):
        n = int(rng.integers(2, 70))
        circ = C.random_layer_circuit(n, 6, seed=300 + c, meas_every=3, meas_frac=0.3)
        circuits.append((n, circ.gates, int(rng.integers(1, 4)), 500 + c))
    want = np.concatenate([r.reshape(-1) for r in tab.batch_run(circuits, seed=9)])
    arr, keep = tab._circuit_array(circuits)
    counts = tab._meas_counts(arr, len(circuits))
    total = int(want.size)
    old = tab.get_config()
    try:
        tab.set_config({"batch_chunks": 6})
        out = np.full(total + 8, 0xA5, np.uint8)
        got_counts = np.full(len(circuits), -1, np.int64)
        tab._check(tab._L.tab_batch_run_packed(tab.ctypes.cast(arr, tab._vp), len(circuits), 9,
                                               out.ctypes.data, total, got_counts.ctypes.data))
        assert list(got_counts) == [int(v) for v in counts]
        assert np.array_equal(out[:total], want) and (out[total:] == 0xA5).all()
        short = np.full(total + 8, 0xA5, np.uint8)
        rc = tab._L.tab_batch_run_packed(tab.ctypes.cast(arr, tab._vp), len(circuits), 9,
                                         short.ctypes.data, total - 1, None)
        assert rc == tab.TAB_ERANGE
        assert (short[total - 1:] == 0xA5).all()
        with pytest.raises(ValueError):
            tab.batch_run(circuits, seed=9, out=np.zeros(total - 1, np.uint8))
        assert tab._L.tab_batch_run_packed(tab.ctypes.cast(arr, tab._vp), len(circuits), 9,
                                           out.ctypes.data, -1, None) == tab.TAB_EINVAL
    finally:
        tab.set_config(old)


def test_batch_run_degenerate_lists():
    """Empty circuit lists, circuits without measurements between measured
    ones, and a buffer of exactly the outcome count, in 1 and 3 chunks: the
    bytes of the measured circuits equal the oracle's."""
    assert tab.batch_run([], seed=3) == []
    arr, keep = tab._circuit_array([])
    assert tab._L.tab_batch_run_packed(tab.ctypes.cast(arr, tab._vp), 0, 3, None, 0,
                                       None) == tab.TAB_OK
    circuits = []
    for c in range(6):
        n = 5 + 7 * c
        # odd circuits: gates only, no outcomes
        circ = C.random_layer_circuit(n, 4, seed=900 + c, final_measure=c % 2 == 0)
        circuits.append((n, circ.gates, 2, 700 + c))
    old = tab.get_config()
    try:
        for chunks in (1, 3):
            tab.set_config({"batch_chunks": chunks})
            arr, keep = tab._circuit_array(circuits)
            total = int(sum(2 * m for m in tab._meas_counts(arr, len(circuits))))
            res = tab.batch_run(circuits, seed=3, out=np.zeros(total, np.uint8))
            for (n, g, shots, cid), got in zip(circuits, res):
                for sh in range(shots):
                    want, _ = oracle.run_circuit(n, g, seed=3, circuit_id=cid, shot=sh)
                    assert np.array_equal(got[sh], want), (n, cid, sh, chunks)
    finally:
        tab.set_config(old)


def test_streaming_work_counters():
    """The streaming engine's work counters against their definition on the
    state each measurement meets: a random outcome adds its pivot row's
    support (columns where stabilizer row p, the first with x_pa = 1, is not
    I), a deterministic one the destabilizer rows i with x_ia = 1.  The
    state before each measurement is exported and the measurement then run
    alone; counting off leaves the counters unchanged."""
    n = 40
    # H then two Z measurements of qubit 0: support 1, then one row
    with tab.Tableau(n) as t:
        t.set_engine(tab.ENGINE_STREAM)
        t.count_work(True)
        t.apply(np.array([_gate(C.TAB_H, 0), _gate(C.TAB_MZ, 0), _gate(C.TAB_MZ, 0)], np.uint64))
        assert t.work_counts() == {"support_cols": 1, "det_rows": 1, "random": 1,
                                   "deterministic": 1}
    circ = C.random_layer_circuit(n, 6, seed=4242, final_measure=False)
    rng = np.random.default_rng(7)
    with tab.Tableau(n) as t:
        t.set_engine(tab.ENGINE_STREAM)
        t.set_rng(seed=5, circuit_id=1, shot=0)
        t.apply(circ.gates)
        t.count_work(True)
        want = {"support_cols": 0, "det_rows": 0, "random": 0, "deterministic": 0}
        for a in rng.integers(0, n, 24):
            x, z, _ = t.export()
            piv = np.nonzero(x[n:, a])[0]
            if piv.size:
                p = n + int(piv[0])
                want["support_cols"] += int(np.count_nonzero(x[p] | z[p]))
                want["random"] += 1
            else:
                want["det_rows"] += int(np.count_nonzero(x[:n, a]))
                want["deterministic"] += 1
            t.apply(np.array([_gate(C.TAB_MZ if a % 3 else C.TAB_MZR, int(a))], np.uint64))
        assert want["random"] > 0 and want["deterministic"] > 0
        assert t.work_counts() == want
        t.count_work(False)
        t.apply(np.array([_gate(C.TAB_MZ, 0)], np.uint64))
        assert t.work_counts() == want


def test_batch_work_counters_match_streaming():
    """The batched kernel's work counters equal, per (circuit, shot), the
    streaming engine's counts on the same circuit (pinned to their definition
    above) times the tableau's 32-row words per column: the X|Z evolution,
    and so every pivot row's support, is the same in every shot.  Counting
    off leaves them unchanged."""
    import torch
    rng = np.random.default_rng(3)
    circuits = []
    for c in range(10):
        n = int(rng.integers(3, 70))
        circ = C.random_layer_circuit(n, 5, seed=1300 + c, meas_every=2, meas_frac=0.3)
        circuits.append((n, circ.gates, int(rng.integers(1, 4)), 40 + c))
    want = {"support_words": 0, "det_row_words": 0, "random": 0, "deterministic": 0}
    for n, g, shots, cid in circuits:
        with tab.Tableau(n) as t:
            t.set_engine(tab.ENGINE_STREAM)
            t.set_rng(seed=2, circuit_id=cid, shot=0)
            t.count_work(True)
            t.apply(g)
            w = t.work_counts()
        words = 2 * ((n + 31) // 32)
        want["support_words"] += shots * words * w["support_cols"]
        want["det_row_words"] += shots * words * w["det_rows"]
        want["random"] += shots * w["random"]
        want["deterministic"] += shots * w["deterministic"]
    assert want["random"] > 0 and want["deterministic"] > 0
    b = tab.Batch(circuits)
    out = torch.zeros(max(b.info()["out_bytes"], 1), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    b.count_work(True)
    b.exec(9, out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert b.work_counts() == want
    b.count_work(False)
    b.exec(9, out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert b.work_counts() == want
    b.close()


def test_batch_config4_sample():
    """A slice of the batched family (n up to 512) against the oracle."""
    circs = C.config4(only=list(range(0, 4096, 512)))
    circuits = [(c.n, c.gates, min(c.shots, 2), c.circuit_id) for c in circs]
    res = tab.batch_run(circuits, seed=C.PHILOX_SEED)
    for (n, g, shots, cid), got in zip(circuits, res):
        for s in range(shots):
            want, _ = oracle.run_circuit(n, g, seed=C.PHILOX_SEED, circuit_id=cid, shot=s)
            assert np.array_equal(got[s], want), (n, cid, s)


def test_batch_autotune_keeps_outcomes():
    """Every CTA shape the autotuner tries writes the same outcomes, and the
    shape it keeps replays them bit for bit (first circuit also vs the oracle)."""
    import torch
    circs = C.config4(only=list(range(3, 4096, 128)))
    circuits = [(c.n, c.gates, min(c.shots, 3), c.circuit_id) for c in circs]
    b = tab.Batch(circuits)
    nbytes = max(b.info()["out_bytes"], 1)
    out0 = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    out1 = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    out2 = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    b.exec(C.PHILOX_SEED, out0.data_ptr(), stream)
    threads, ms = b.tune(C.PHILOX_SEED, out1.data_ptr(), stream)
    assert threads in (128, 256, 512, 1024) and ms > 0
    assert b.config()["threads"] == threads
    b.exec(C.PHILOX_SEED, out2.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.equal(out0, out1) and torch.equal(out0, out2)
    n, g, shots, cid = circuits[0]
    want, _ = oracle.run_circuit(n, g, seed=C.PHILOX_SEED, circuit_id=cid, shot=0)
    assert np.array_equal(out2[:want.size].cpu().numpy(), want)
    b.close()


def _gate(op, q1=0, q2=0):
    return int(np.asarray(C.encode(op, q1, q2)).reshape(-1)[0])


def _ghz(n, reverse=False):
    g = [_gate(C.TAB_H, 0)]
    g += [_gate(C.TAB_CNOT, i, i + 1) for i in range(n - 1)]
    qs = range(n - 1, -1, -1) if reverse else range(n)
    g += [_gate(C.TAB_MZ, q) for q in qs]
    return np.array(g, dtype=np.uint64)


def test_batch_sampler_matches_per_shot():
    """Terminal-measurement sampler: the same outcome bits as running every
    shot, on random circuits up to n = 512, GHZ states (deterministic outcomes
    that depend on an earlier random bit), a repeated measurement and a
    circuit with a mid-circuit measurement (not sampled)."""
    import torch
    circs = C.config4(only=list(range(5, 4096, 512)))
    circuits = [(c.n, c.gates, min(c.shots, 6), c.circuit_id) for c in circs]
    circuits.append((24, _ghz(24), 16, 9001))
    circuits.append((17, _ghz(17, reverse=True), 9, 9002))
    rep = np.array([_gate(C.TAB_H, 3), _gate(C.TAB_S, 3), _gate(C.TAB_MZ, 3),
                    _gate(C.TAB_MZ, 3), _gate(C.TAB_MZ, 1)], dtype=np.uint64)
    circuits.append((5, rep, 7, 9003))
    mid = C.random_layer_circuit(40, 8, seed=5, meas_every=3, meas_frac=0.2)
    circuits.append((40, mid.gates, 5, 9004))
    only_meas = np.array([_gate(C.TAB_MZ, q) for q in range(6)], dtype=np.uint64)
    circuits.append((6, only_meas, 3, 9005))
    plain = tab.Batch(circuits)
    samp = tab.Batch(circuits, sample_terminal=True)
    assert samp.sampled == len(circuits) - 1  # all but the mid-circuit one
    assert plain.sampled == 0
    nbytes = plain.info()["out_bytes"]
    assert samp.info()["out_bytes"] == nbytes
    a = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    b = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    plain.exec(C.PHILOX_SEED, a.data_ptr())
    samp.exec(C.PHILOX_SEED, b.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(a, b), int((a != b).sum())
    # GHZ shots against the oracle: outcomes all equal within a shot
    ghz = b.cpu().numpy()
    off = sum(c[2] * int(np.isin(C.decode(c[1])[0], C.MEASURE).sum()) for c in circuits[:-5])
    for s in range(16):
        want, _ = oracle.run_circuit(24, circuits[-5][1], seed=C.PHILOX_SEED, circuit_id=9001, shot=s)
        got = ghz[off + 24 * s: off + 24 * (s + 1)]
        assert np.array_equal(got, want) and len(set(got.tolist())) == 1
    plain.close()
    samp.close()


def test_unknown_engine_rejected():
    with tab.Tableau(8) as t:
        for bad in (3, 5, -1):
            with pytest.raises(tab.TabError) as ei:
                t.set_engine(bad)
            assert ei.value.code == tab.TAB_EINVAL
