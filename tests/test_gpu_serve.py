"""Continuous-batching server: results alone == results in the mix, memory
admission, and host-side failure handling (no GPU fault is ever caused)."""
import numpy as np
import pytest

import oracle
from workloads import circuits as C

pytestmark = pytest.mark.gpu

from paper_2408_00384_gb300 import tab  # noqa: E402


def mixed_requests(count, seed=0, n_hi=900):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(20), np.log(n_hi))))
        depth = int(rng.integers(4, 24))
        c = C.random_layer_circuit(n, depth, seed=5000 + i, meas_every=4, meas_frac=0.05)
        reqs.append((n, c.gates, 1 + (i % 2), 700 + i))
    return reqs


def alone(n, gates, shots, cid, seed):
    outs = []
    with tab.Tableau(n) as t:
        for s in range(shots):
            t.reset()
            t.set_rng(seed, cid, s)
            t.apply(gates)
            outs.append(t.read_outcomes())
    return np.concatenate(outs)


def test_mix_equals_alone_and_overlaps():
    reqs = mixed_requests(28)
    with tab.Server(mem_budget_bytes=4 << 30, max_inflight=8, n_streams=4, meas_ctas=16,
                    seed=31) as srv:
        tickets = [srv.submit(n, g, shots, cid) for (n, g, shots, cid) in reqs]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_inflight"] > 1
    for (n, g, shots, cid), (rc, out, lat) in zip(reqs, results):
        assert rc == tab.TAB_OK and lat > 0
        assert np.array_equal(out, alone(n, g, shots, cid, 31)), (n, cid)
        if n <= 200:
            want = np.concatenate([oracle.run_circuit(n, g, seed=31, circuit_id=cid, shot=s)[0]
                                   for s in range(shots)])
            assert np.array_equal(out, want), (n, cid)


def test_memory_admission():
    reqs = mixed_requests(12, seed=1, n_hi=1200)
    biggest = max(tab.bytes_required(n) for n, *_ in reqs)
    budget = 2 * biggest + (4 << 20)
    with tab.Server(mem_budget_bytes=budget, max_inflight=8, n_streams=4, seed=3) as srv:
        tickets = [srv.submit(n, g, shots, cid) for (n, g, shots, cid) in reqs]
        too_big = srv.submit(8000, C.random_clifford_ops(8000, 10, seed=1), 1, 1)
        results = [srv.wait(t) for t in tickets]
        rc_big, _, _ = srv.wait(too_big)
        st = srv.stats()
    assert rc_big == tab.TAB_ENOMEM
    assert st["peak_mem"] <= budget and st["rejected"] == 1
    for (n, g, shots, cid), (rc, out, _) in zip(reqs, results):
        assert rc == tab.TAB_OK
        assert np.array_equal(out, alone(n, g, shots, cid, 3))


def test_dropped_completion_times_out_and_frees_slot():
    reqs = mixed_requests(6, seed=2, n_hi=300)
    with tab.Server(mem_budget_bytes=1 << 30, max_inflight=1, n_streams=1,
                    request_timeout_s=2.0, seed=9) as srv:
        tickets = [srv.submit(n, g, shots, cid) for (n, g, shots, cid) in reqs]
        srv.inject(tickets[1], tab.FAULT_DROP_COMPLETION)
        results = [srv.wait(t, timeout_s=60.0) for t in tickets]
        st = srv.stats()
    assert results[1][0] == tab.TAB_ETIMEOUT
    assert st["failed"] == 1 and st["completed"] == len(reqs) - 1
    for i, ((n, g, shots, cid), (rc, out, _)) in enumerate(zip(reqs, results)):
        if i == 1:
            continue
        assert rc == tab.TAB_OK
        assert np.array_equal(out, alone(n, g, shots, cid, 9))


def test_invalid_request_refused_at_submit():
    with tab.Server(mem_budget_bytes=1 << 28, max_inflight=2, n_streams=1) as srv:
        with pytest.raises(tab.TabError) as ei:
            srv.submit(5, C.encode(C.TAB_CNOT, 1, 7).reshape(1))
        assert ei.value.code == tab.TAB_ERANGE
        t = srv.submit(5, C.random_clifford_ops(5, 30, seed=2, measure_p=0.2))
        rc, out, _ = srv.wait(t)
        assert rc == tab.TAB_OK
