"""Whole workload families on the GPU against the oracle's stored results.

The oracle's full runs of these families take minutes on every core, so
``tests/golden/make_oracle_digests.py`` ran them once and stored what they
produce (tests/golden/oracle_cfg*.json): every outcome bit of the n = 10,000
tableau and of each served request, the final tableaus as SHA-256 digests, and
for the 4,096-circuit batch one digest per circuit over all its shots.  Each
test regenerates the same seeded inputs, first checks that they are the gate
words the oracle saw, then compares the library's results bit for bit.  A
mismatch names the first differing measurement (for the batch, the circuit is
rerun on the oracle to find the shot and index).
"""
import numpy as np
import torch
import pytest

import oracle
from tests.golden import digests as D
from workloads import circuits as C

pytestmark = pytest.mark.gpu

from paper_2408_00384_gb300 import tab  # noqa: E402


def check_outcomes(got, entry, what):
    want = D.unpack_outcomes(entry["outcomes_packed"], entry["n_meas"])
    first = D.first_difference(got, want)
    assert first is None, (f"{what}: first differing measurement {first} of {want.size} "
                           f"(got {got.size} outcomes)")
    assert D.outcomes_sha(got) == entry["outcomes_sha256"], what


def check_inputs(gates, entry, what):
    assert D.gates_sha(gates) == entry["gates_sha256"], (
        f"{what}: the seeded generator gave other gate words than the oracle's run")


# ------------------------------------------------------------- config 3 ---

@pytest.fixture(scope="module")
def cfg3():
    return C.config3(), D.load("cfg3")


@pytest.mark.parametrize("path", ["apply", "program"])
def test_config3_full_vs_oracle(cfg3, path):
    """n = 10,000, 100 random layers, ten rounds of 1,000 MZR (10^4
    measurements on the streaming engine): every outcome and the final
    tableau, through the pipelined tab_apply and through a compiled program."""
    c, ref = cfg3
    check_inputs(c.gates, ref, "cfg3")
    with tab.Tableau(c.n) as t:
        assert t.engine_resolved()[0] == tab.ENGINE_STREAM
        t.set_rng(ref["seed"], ref["circuit_id"], ref["shot"])
        if path == "apply":
            t.apply(c.gates)
        else:
            with tab.Program(c.n, c.gates) as p:
                t.run(p)
        got = t.read_outcomes()
        x, z, r = t.export()
    check_outcomes(got, ref, f"cfg3 {path}")
    assert D.tableau_sha(x, z, r) == ref["tableau_sha256"], f"cfg3 {path}: final tableau"


# ------------------------------------------------------------- config 4 ---

@pytest.fixture(scope="module")
def cfg4():
    ref = D.load("cfg4")
    circs = C.config4()
    return circs, ref


def _batch_mismatch(circs, ref, out, offsets):
    """Name the first circuit whose outcomes differ, and its first differing
    (shot, measurement) from an oracle rerun of that circuit."""
    for i, (c, e) in enumerate(zip(circs, ref["circuits"])):
        seg = out[offsets[i]:offsets[i + 1]]
        if D.outcomes_sha(seg)[:32] == e["outcomes_sha256"]:
            continue
        for shot in range(c.shots):
            want = oracle.run_circuit(c.n, c.gates, seed=ref["seed"], circuit_id=c.circuit_id,
                                      shot=shot)[0]
            got = seg[shot * c.n_meas:(shot + 1) * c.n_meas]
            first = D.first_difference(got, want)
            if first is not None:
                return f"circuit {i} (n={c.n}): shot {shot}, measurement {first}"
        return f"circuit {i} (n={c.n}): digest differs"
    return None


@pytest.mark.parametrize("sampler", [False, True])
def test_config4_batch_vs_oracle(cfg4, sampler):
    """All 4,096 circuits with all their shots (3.5e7 outcomes) in one
    persistent launch, per-shot and with the terminal-measurement sampler,
    after the autotuner has picked the launch shape: every circuit's outcome
    bytes against the oracle's digest."""
    torch = pytest.importorskip("torch")
    circs, ref = cfg4
    assert len(ref["circuits"]) == len(circs)
    import hashlib
    gsha = hashlib.sha256("".join(D.gates_sha(c.gates) for c in circs).encode()).hexdigest()
    assert gsha == ref["gates_sha256_of_circuit_shas"], "cfg4: generator gave other gate words"
    b = tab.Batch([(c.n, c.gates, c.shots, c.circuit_id) for c in circs], sample_terminal=sampler)
    try:
        info = b.info()
        dev = torch.empty(info["out_bytes"], dtype=torch.uint8, device="cuda")
        b.tune(ref["seed"], dev.data_ptr())
        dev.fill_(7)
        b.exec(ref["seed"], dev.data_ptr())
        torch.cuda.synchronize()
        out = dev.cpu().numpy()
        if sampler:
            assert b.sampled == len(circs)
    finally:
        b.close()
    sizes = [c.shots * c.n_meas for c in circs]
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    assert offsets[-1] == out.size
    bad = [i for i, e in enumerate(ref["circuits"])
           if D.outcomes_sha(out[offsets[i]:offsets[i + 1]])[:32] != e["outcomes_sha256"]]
    if bad:
        pytest.fail(f"cfg4 ({'sampler' if sampler else 'per shot'}): {len(bad)} circuits differ; "
                    + str(_batch_mismatch(circs, ref, out, offsets)))


def test_config4_batch_run_host_buffers_vs_oracle(cfg4):
    """The same family through tab_batch_run (host gate lists in, host
    outcome buffer out; large enough to run as several chunks whose host
    compile overlaps the previous chunk's launch): every circuit against the
    oracle's digest; then a caller-given layout (circuits in reverse order,
    a gap after each) gets the same bytes in each circuit's span."""
    circs, ref = cfg4
    tc = [(c.n, c.gates, c.shots, c.circuit_id) for c in circs]
    res = tab.batch_run(tc, seed=ref["seed"])
    bad = [i for i, (e, r) in enumerate(zip(ref["circuits"], res))
           if D.outcomes_sha(np.ascontiguousarray(r).reshape(-1))[:32] != e["outcomes_sha256"]]
    assert not bad, f"cfg4 via tab_batch_run: {len(bad)} circuits differ (first {bad[:5]})"
    sizes = [c.shots * c.n_meas for c in circs]
    offs, pos = [0] * len(circs), 0
    for i in reversed(range(len(circs))):
        offs[i] = pos
        pos += sizes[i] + 3
    out = np.full(pos, 7, np.uint8)
    arr, keep = tab._circuit_array(tc)
    offs_arr = (tab._i64 * len(offs))(*offs)
    tab._check(tab._L.tab_batch_run(tab.ctypes.cast(arr, tab._vp), len(tc), ref["seed"],
                                    out.ctypes.data, tab.ctypes.cast(offs_arr, tab._vp)))
    for i in (0, 1, len(circs) // 2, len(circs) - 1):
        got = out[offs[i]:offs[i] + sizes[i]]
        assert np.array_equal(got, np.ascontiguousarray(res[i]).reshape(-1)), i
        assert (out[offs[i] + sizes[i]:offs[i] + sizes[i] + 3] == 7).all(), i
    # the bytes do not depend on the chunking (7 chunks on alternating
    # streams, copied back per chunk into pinned memory; one chunk into
    # pageable memory)
    packed = np.concatenate([np.ascontiguousarray(r).reshape(-1) for r in res])
    old = tab.get_config()
    try:
        tab.set_config({"batch_chunks": 7})
        pinned = torch.full((int(packed.size),), 9, dtype=torch.uint8).pin_memory().numpy()
        tab.batch_run(tc, seed=ref["seed"], out=pinned)
        assert np.array_equal(pinned, packed)
        tab.set_config({"batch_chunks": 1})
        one = np.concatenate([np.ascontiguousarray(r).reshape(-1)
                              for r in tab.batch_run(tc, seed=ref["seed"])])
        assert np.array_equal(one, packed)
    finally:
        tab.set_config(old)


# ------------------------------------------------------------- config 5 ---

@pytest.fixture(scope="module")
def cfg5():
    ref = D.load("cfg5")
    reqs = [C.config5_request(e["c"]) for e in ref["requests"]]
    for r, e in zip(reqs, ref["requests"]):
        check_inputs(r.gates, e, f"cfg5 request {e['c']}")
    return reqs, ref


def test_config5_served_mix_vs_oracle(cfg5):
    """The served family's requests (n up to ~4,800, depth 2n, MZR rounds
    every 20 layers, final MZ) submitted together to the continuous-batching
    server: they overlap on the device, and each request's outcomes equal the
    oracle's run of that request alone."""
    reqs, ref = cfg5
    with tab.Server(mem_budget_bytes=150 << 30, max_inflight=16, n_streams=8, meas_ctas=32,
                    seed=ref["seed"]) as srv:
        tickets = [srv.submit(r.n, r.gates, 1, r.circuit_id) for r in reqs]
        results = [srv.wait(tk, timeout_s=600.0) for tk in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_inflight"] > 1
    for r, e, (rc, out, _) in zip(reqs, ref["requests"], results):
        assert rc == tab.TAB_OK, (e["c"], rc)
        check_outcomes(out, e, f"cfg5 request {e['c']} (n={r.n}) served")


def _engines_for(n):
    engines = [tab.ENGINE_GRID, tab.ENGINE_STREAM]
    if n <= 640:
        engines.append(tab.ENGINE_SINGLE_CTA)
    return engines


def test_config5_requests_each_engine_vs_oracle(cfg5):
    """Each served request alone on every measurement engine that holds it
    (grid-resident, streaming, and single-CTA for n <= 640): every outcome
    and the final tableau.  The largest request runs ~117,000 measurements
    at n = 4,751 on one tableau."""
    reqs, ref = cfg5
    for r, e in zip(reqs, ref["requests"]):
        for eng in _engines_for(r.n):
            with tab.Tableau(r.n) as t:
                try:
                    t.set_engine(eng)
                except tab.TabError as err:
                    if err.code == tab.TAB_ERANGE:
                        continue  # this engine does not hold n qubits
                    raise
                t.set_rng(ref["seed"], r.circuit_id, ref["shot"])
                t.apply(r.gates)
                got = t.read_outcomes()
                x, z, rr = t.export()
            what = f"cfg5 request {e['c']} (n={r.n}) engine {eng}"
            check_outcomes(got, e, what)
            assert D.tableau_sha(x, z, rr) == e["tableau_sha256"], what + ": final tableau"
