"""Extended ops (X / Y measurement, Pauli noise) in batches and in the
request server, against the oracle per (circuit, shot).

A batch keeps its noise ops and every shot draws its own noise on the device
(counter from 0 per shot, the Philox block of the documented noise rule); the
gates it runs once for all shots end at the circuit's first measurement or
noise op.  The server lowers X / Y measurements once and draws a noisy
request's noise per shot on the host.  The oracle runs every extended op
itself, one (circuit, shot) at a time.
"""
import numpy as np
import pytest

import oracle
from workloads import circuits as C

pytestmark = pytest.mark.gpu

from paper_2408_00384_gb300 import tab  # noqa: E402

SEED = 13


def mixed_circuits():
    """(n, gates, shots, cid): noise before the first measurement, noise only
    between measurements, X / Y measurements without noise, terminal MX /
    MY layers, noise-free circuits beside them, and a layer circuit."""
    out = []
    for i, (n, count, pm, pn) in enumerate([(8, 120, 0.1, 0.15), (33, 400, 0.08, 0.1),
                                             (64, 500, 0.05, 0.05), (130, 300, 0.1, 0.0),
                                             (5, 60, 0.3, 0.3), (300, 600, 0.02, 0.02)]):
        g = C.random_extended_ops(n, count, seed=100 + i, p_meas=pm, p_noise=pn)
        out.append((n, g, 1 + (i % 3) * 3, 500 + i))
    # gates, then noise only after the first measurement
    n = 50
    gates = C.random_clifford_ops(n, 200, seed=7)
    late = C.random_extended_ops(n, 150, seed=8, p_meas=0.2, p_noise=0.2)
    first_meas = C.encode(C.TAB_MZ, 3, 0).reshape(1)
    out.append((n, np.concatenate([gates, first_meas, late]), 5, 600))
    # a random-layer circuit with terminal X and Y measurements
    c = C.random_layer_circuit(90, 20, seed=5)
    op, q1, _ = C.decode(c.gates)
    g = c.gates.copy()
    mz = np.flatnonzero(op == C.TAB_MZ)
    g[mz[::2]] = C.encode(C.TAB_MX, q1[mz[::2]], 0)
    g[mz[1::2]] = C.encode(C.TAB_MY, q1[mz[1::2]], 0)
    out.append((90, g, 4, 601))
    out.append((40, C.random_clifford_ops(40, 200, seed=3, measure_p=0.1, reset_p=0.05), 3, 602))
    return out


def oracle_shot(n, gates, cid, shot):
    return oracle.run_circuit(n, gates, seed=SEED, circuit_id=cid, shot=shot)[0]


@pytest.mark.parametrize("sample_terminal", [False, True])
def test_batch_extended_ops_match_oracle_per_shot(sample_terminal):
    torch = pytest.importorskip("torch")
    circs = mixed_circuits()
    b = tab.Batch(circs, sample_terminal=sample_terminal)
    try:
        info = b.info()
        dev = torch.full((max(info["out_bytes"], 1),), 7, dtype=torch.uint8, device="cuda")
        b.exec(SEED, dev.data_ptr())
        torch.cuda.synchronize()
        out = dev.cpu().numpy()
    finally:
        b.close()
    off = 0
    for n, g, shots, cid in circs:
        k = tab.n_meas_of(g)
        for s in range(shots):
            want = oracle_shot(n, g, cid, s)
            got = out[off:off + k]
            assert np.array_equal(got, want), (n, cid, s, np.flatnonzero(got != want)[:8])
            off += k
    assert off == info["out_bytes"]


def test_batch_run_extended_ops_host_buffers():
    circs = mixed_circuits()[:4]
    res = tab.batch_run(circs, SEED)
    for (n, g, shots, cid), r in zip(circs, res):
        for s in range(shots):
            assert np.array_equal(r[s], oracle_shot(n, g, cid, s)), (n, cid, s)


def test_server_extended_ops_match_oracle_per_shot():
    circs = mixed_circuits()
    with tab.Server(mem_budget_bytes=1 << 30, max_inflight=4, n_streams=2, seed=SEED) as srv:
        tickets = [srv.submit(n, g, shots, cid) for (n, g, shots, cid) in circs]
        results = [srv.wait(t, timeout_s=120.0) for t in tickets]
    for (n, g, shots, cid), (rc, out, _) in zip(circs, results):
        assert rc == tab.TAB_OK
        k = tab.n_meas_of(g)
        for s in range(shots):
            assert np.array_equal(out[s * k:(s + 1) * k], oracle_shot(n, g, cid, s)), (n, cid, s)
