"""The oracle's all-core mode against its one-thread mode.

The threaded mode splits two loops over rows into contiguous shares: each gate
rule's loop (AG Sec. III: a gate updates every row from that row's own bits)
and the target rows of a random-outcome measurement's rowsums (each writes its
own row and reads only the pivot row).  It must give the one-thread result bit
for bit: every outcome, every deterministic flag, the whole tableau and the
measurement counter.  Shares range from more threads than rows (n = 1, 2) to
uneven shares (2n not a multiple of the thread count).
"""
import numpy as np
import pytest

import oracle
from workloads import circuits as C


def run(n, gates, threads, seed=3, cid=5, shot=2):
    t = oracle.Tableau(n, threads=threads)
    assert t.threads == threads
    out, det = t.run(gates, seed=seed, circuit_id=cid, shot=shot, with_det=True)
    return out, det, t.get(), t.meas_counter


@pytest.mark.parametrize("n", [1, 2, 3, 7, 33, 130, 301])
@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threads_equal_one_thread(n, threads):
    gates = C.random_clifford_ops(n, 600, seed=91 * n + threads, measure_p=0.1, reset_p=0.05)
    want = run(n, gates, 1)
    got = run(n, gates, threads)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    for g, w in zip(got[2], want[2]):
        assert np.array_equal(g, w)
    assert got[3] == want[3]


def test_threads_layer_circuit_with_rounds():
    """A random-layer circuit with mid-circuit MZR rounds and a final MZ layer
    (random and deterministic outcomes both occur)."""
    c = C.random_layer_circuit(257, 20, seed=4, meas_every=5, meas_frac=0.2)
    want = run(c.n, c.gates, 1)
    got = run(c.n, c.gates, 5)
    assert want[1].any() and not want[1].all()
    assert np.array_equal(got[0], want[0])
    for g, w in zip(got[2], want[2]):
        assert np.array_equal(g, w)


def test_thread_count_changes_and_errors():
    t = oracle.Tableau(40, threads=4)
    t.set_threads(1)
    assert t.threads == 1
    t.set_threads(6)
    assert t.threads == 6
    with pytest.raises(RuntimeError):
        t.set_threads(0)
    assert oracle.all_cores() >= 1
