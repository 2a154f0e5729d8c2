"""The plain path's autotuner (tab_tune) and its cache file.

Every launch shape the tuner tries must give the same outcomes (the tuner
itself refuses otherwise); the shape it keeps must run the circuit bit for
bit like the oracle; a second call with TAB_AUTOTUNE_CACHE set must take the
stored shape without timing.
"""
import json
import os

import numpy as np
import pytest

import oracle
from workloads import circuits as C

pytestmark = pytest.mark.gpu

from paper_2408_00384_gb300 import tab  # noqa: E402


@pytest.mark.parametrize("n,depth", [(200, 10), (700, 12)])
def test_tuned_shape_matches_oracle_and_is_cached(n, depth, tmp_path, monkeypatch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("TAB_AUTOTUNE_CACHE", str(cache))
    c = C.random_layer_circuit(n, depth, seed=n + 1, meas_every=4, meas_frac=0.05)
    want, (wx, wz, wr) = oracle.run_circuit(n, c.gates, seed=9, circuit_id=3)
    with tab.Program(n, c.gates) as prog, tab.Tableau(n) as t:
        t.set_rng(9, 3, 0)
        got_shape = t.tune(prog, reps=2)
        assert got_shape["from_cache"] == 0 and got_shape["tried"] >= 3
        assert got_shape["engine"] in (tab.ENGINE_SINGLE_CTA, tab.ENGINE_GRID, tab.ENGINE_STREAM)
        assert t.engine_resolved()[0] == got_shape["engine"]
        t.run(prog)
        out = t.read_outcomes()
        x, z, r = t.export()
        lines = [json.loads(l) for l in cache.read_text().splitlines()]
        assert len(lines) == 1 and f"|n{1 << (n - 1).bit_length()}|" in lines[0]["key"]
        # a second handle takes the stored shape without timing
        with tab.Tableau(n) as t2:
            t2.set_rng(9, 3, 0)
            again = t2.tune(prog)
            assert again["from_cache"] == 1
            for k in ("engine", "block_threads", "meas_batch"):
                assert again[k] == got_shape[k]
            t2.run(prog)
            out2 = t2.read_outcomes()
    assert np.array_equal(out, want) and np.array_equal(out2, want)
    assert np.array_equal(x, wx) and np.array_equal(z, wz) and np.array_equal(r, wr)
