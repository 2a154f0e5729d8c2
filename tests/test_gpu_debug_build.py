"""The debug build (libtab_debug.so: every kernel checks the qubit indices it
reads; include/tab.h, "debug build").

The test builds the debug library if it is missing (the same sources with
-DTAB_DEBUG), then, in a child process with TAB_DEBUG=1 (the binding picks the
library at import), checks that the device check latches an out-of-range
index as TAB_EDEVICE and passes an in-range one, and that the checks stay
silent on real runs: circuits with random and deterministic measurements on
every engine and a small batch, bit for bit against the oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np
import oracle
from paper_2408_00384_gb300 import tab
from workloads import circuits as C

assert tab.DEBUG and tab.debug_build()
assert tab.debug_check(5, 6) == 5
try:
    tab.debug_check(6, 6)
    raise SystemExit("out-of-range index not reported")
except tab.TabError as e:
    assert e.code == tab.TAB_EDEVICE, e
    assert "out of range" in tab.last_error(), tab.last_error()
for n, engine in ((40, tab.ENGINE_SINGLE_CTA), (300, tab.ENGINE_GRID), (300, tab.ENGINE_STREAM),
                  (1100, tab.ENGINE_GRID)):
    c = C.random_layer_circuit(n, 12, seed=n + engine, meas_every=4, meas_frac=0.1, reset=True)
    want, (wx, wz, wr) = oracle.run_circuit(n, c.gates, seed=9)
    with tab.Tableau(n) as t:
        t.set_engine(engine)
        t.set_rng(9, 0, 0)
        t.apply(c.gates)
        got = t.read_outcomes()
        x, z, r = t.export()
    assert np.array_equal(got, want), (n, engine)
    assert np.array_equal(x, wx) and np.array_equal(z, wz) and np.array_equal(r, wr), (n, engine)
circs = [C.random_layer_circuit(n, n, seed=100 + n, circuit_id=i, shots=3)
         for i, n in enumerate((20, 64, 130))]
res = tab.batch_run([(c.n, c.gates, c.shots, c.circuit_id) for c in circs], seed=4)
for c, out in zip(circs, res):
    for s in range(c.shots):
        want = oracle.run_circuit(c.n, c.gates, seed=4, circuit_id=c.circuit_id, shot=s)[0]
        assert np.array_equal(out[s], want), (c.n, s)
print("debug build ok")
"""


def test_debug_build_checks_and_parity():
    lib = os.path.join(ROOT, "paper_2408_00384_gb300", "libtab_debug.so")
    if not os.path.exists(lib):
        subprocess.run([sys.executable, "-m", "paper_2408_00384_gb300.build", "--debug"],
                       cwd=ROOT, check=True, capture_output=True, timeout=900)
    env = dict(os.environ, TAB_DEBUG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "debug build ok" in r.stdout
