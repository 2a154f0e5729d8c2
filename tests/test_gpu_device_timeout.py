"""A device-side bounded wait that runs out, and the handle's recovery.

Every spin-wait in the library's kernels has a limit; when it runs out the
kernel latches an error word, every CTA returns, and the next synchronizing
call reports TAB_ETIMEOUT.  This test makes that happen without faulting or
hanging anything: the run-time configuration shortens the grid-barrier limit
to a few milliseconds and turns on the test-only flag under which the last
CTA of a grid-resident measurement launch skips its first grid-barrier
arrival, so the other CTAs' waits run out.  Afterwards, with the flag off,
tab_reset clears the latched error and the same handle runs a circuit bit for
bit like the oracle.
"""
import numpy as np
import pytest

import oracle
from workloads import circuits as C

pytestmark = pytest.mark.gpu

from paper_2408_00384_gb300 import tab  # noqa: E402


def test_grid_barrier_wait_runs_out_and_handle_recovers():
    n = 1000
    c = C.random_layer_circuit(n, 6, seed=11, meas_every=3, meas_frac=0.02)
    old = tab.get_config()
    try:
        with tab.Tableau(n) as t:
            t.set_engine(tab.ENGINE_GRID)
            assert t.engine_resolved()[0] == tab.ENGINE_GRID
            tab.set_config({"wait_limit_ns": 5_000_000,
                            "debug": tab.DEBUG_SKIP_BARRIER_ARRIVAL})
            t.set_rng(5, 0, 0)
            with pytest.raises(tab.TabError) as ei:
                t.apply(c.gates)
                t.sync()
            assert ei.value.code == tab.TAB_ETIMEOUT, tab.last_error()
            # the handle stays unusable until it is reset
            with pytest.raises(tab.TabError):
                t.apply(c.gates[:4])
            tab.set_config(old)
            t.reset()
            t.set_rng(5, 0, 0)
            t.apply(c.gates)
            got = t.read_outcomes()
            x, z, r = t.export()
    finally:
        tab.set_config(old)
    want, (wx, wz, wr) = oracle.run_circuit(n, c.gates, seed=5)
    assert np.array_equal(got, want)
    assert np.array_equal(x, wx) and np.array_equal(z, wz) and np.array_equal(r, wr)
