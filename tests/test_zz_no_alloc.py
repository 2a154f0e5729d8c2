"""tab_measure_noalloc: the measurement entry point for callers that cannot
allocate device memory (their device heap belongs to another allocator, or a
latency-critical loop must not allocate after start-up).  Its outcomes and the
resulting tableau must equal those of tab_measure_async on the same state, on
two calls in a row (the second call reuses the library's fixed scratch array
as the first left it).  At n = 16,384 the measurement launch's CTA count has to
be lowered for its scratch to fit the array, so that case runs a different
launch shape from tab_measure_async.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from workloads import circuits as C

pytestmark = pytest.mark.gpu

from paper_2408_00384_gb300 import tab  # noqa: E402


@pytest.mark.parametrize("n", [40, 300, 1200, 16384])
def test_noalloc_equals_measure_async_two_calls(n):
    torch = pytest.importorskip("torch")
    depth = 12 if n <= 1200 else 2
    gates = C.random_layer_circuit(n, depth, seed=n + 3, final_measure=False).gates
    rng = np.random.default_rng(n)
    calls = [(rng.choice(n, size=min(n, 25), replace=False).astype(np.int32), False),
             (rng.choice(n, size=min(n, 40), replace=False).astype(np.int32), True)]
    # reference: the existing asynchronous measurement entry point
    ref_out = []
    with tab.Tableau(n) as a:
        a.set_rng(21, 4, 2)
        a.apply(gates)
        for qs, reset in calls:
            buf = torch.zeros(qs.size, dtype=torch.uint8, device="cuda")
            if reset:
                a.apply(C.encode(np.full(qs.size, C.TAB_MZR), qs, 0))
                ref_out.append(a.read_outcomes()[-qs.size:])
            else:
                a.measure_async(qs, buf.data_ptr())
                a.sync()
                ref_out.append(buf.cpu().numpy())
        ref_state = a.export()
        engine, ctas = a.engine_resolved()
    if n == 16384:
        # the handle's own launch shape needs more scratch words than the
        # array has, so the no-allocation call must lower its CTA count
        W = 2 * (((n + 31) // 32 + 3) // 4 * 4)
        need = (40 + 63) // 64 * 64 + ctas * 2 * W + 2 * W + 2 * ctas + 64
        assert engine == tab.ENGINE_STREAM and need * 4 > tab.NOALLOC_SCRATCH_BYTES
    # the same through the no-allocation entry point, on caller-owned memory
    mem = torch.empty(tab.bytes_required(n), dtype=torch.uint8, device="cuda")
    got_out = []
    with tab.Tableau(n, memory=mem) as b:
        b.set_rng(21, 4, 2)
        b.apply(gates)
        for qs, reset in calls:
            buf = torch.full((qs.size,), 7, dtype=torch.uint8, device="cuda")
            b.measure_noalloc(qs, buf.data_ptr(), reset=reset)
            b.sync()
            got_out.append(buf.cpu().numpy())
        got_state = b.export()
    for g, w in zip(got_out, ref_out):
        assert np.array_equal(g, w)
    for g, w in zip(got_state, ref_state):
        assert np.array_equal(g, w)
    del got_state, ref_state
    # and both agree with the oracle
    t = oracle.Tableau(n, threads=min(8, oracle.all_cores()))
    t.run(gates)
    t.meas_counter = 0
    want = [t.run(C.encode(np.full(qs.size, C.TAB_MZR if reset else C.TAB_MZ), qs, 0),
                  seed=21, circuit_id=4, shot=2) for qs, reset in calls]
    for g, w in zip(got_out, want):
        assert np.array_equal(g, w)


def test_noalloc_rejects_oversize_and_bad_qubit():
    torch = pytest.importorskip("torch")
    n = 64
    buf = torch.zeros(8, dtype=torch.uint8, device="cuda")
    with tab.Tableau(n) as t:
        too_many = np.zeros(tab.NOALLOC_SCRATCH_BYTES // 4, np.int32)
        with pytest.raises(tab.TabError) as ei:
            t.measure_noalloc(too_many, buf.data_ptr())
        assert ei.value.code == tab.TAB_ERANGE
        with pytest.raises(tab.TabError) as ei:
            t.measure_noalloc(np.array([n], np.int32), buf.data_ptr())
        assert ei.value.code == tab.TAB_ERANGE
        t.sync()
