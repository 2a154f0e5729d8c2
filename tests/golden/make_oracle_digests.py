"""Write the oracle's full-size results for the workload families whose whole
runs are too long to repeat inside a test: the n = 10,000 tableau with
mid-circuit MZR rounds, the 4,096-circuit batch with all its shots, and the
first requests of the served family (n up to ~4,800).

Every stored value comes from ``oracle/`` run on inputs from
``workloads/circuits.py``; nothing here runs the CUDA library.  The GPU tests
(tests/test_gpu_full_configs.py) compare the library's results with these
files.

Usage: python tests/golden/make_oracle_digests.py [cfg3] [cfg4] [cfg5]
       [--threads T] [--requests R]

Threads: the n = 10,000 and served runs use the oracle's row threads on every
core; the batch runs one circuit per core.  In the batch, a circuit's gates
precede its measurements and do not depend on outcomes, so every shot starts
from the same post-gate tableau: the oracle applies the gates once and copies
that tableau into each shot's run (each shot then draws its own Philox
stream), which is the same tableau as running the gates again from |0^n>.
"""
import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from tests.golden import digests as D  # noqa: E402
from workloads import circuits as C  # noqa: E402

SERVED_REQUESTS = 32


def log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def write(family, obj):
    tmp = D.path(family) + ".tmp"
    with open(tmp, "w") as f:
        json.dump(obj, f, indent=0, sort_keys=True)
        f.write("\n")
    os.replace(tmp, D.path(family))
    log(f"wrote {D.path(family)}")


def whole_run(n, gates, seed, cid, shot, threads):
    t = oracle.Tableau(n, threads=threads)
    out = t.run(gates, seed=seed, circuit_id=cid, shot=shot)
    x, z, r = t.get()
    return out, D.tableau_sha(x, z, r)


def cfg3(threads):
    c = C.config3()
    t0 = time.time()
    out, tsha = whole_run(c.n, c.gates, C.PHILOX_SEED, 0, 0, threads)
    log(f"cfg3: {out.size} outcomes in {time.time() - t0:.0f} s")
    assert out.size == c.n_meas
    write("cfg3", {
        "family": "cfg3", "what": "config 3: n=10000, 100 random layers, MZR on 1000 "
                                  "random qubits after every 10th layer",
        "n": c.n, "seed": C.PHILOX_SEED, "circuit_id": 0, "shot": 0,
        "gates_sha256": D.gates_sha(c.gates), "n_meas": int(out.size),
        "outcomes_sha256": D.outcomes_sha(out), "outcomes_packed": D.pack_outcomes(out),
        "tableau_sha256": tsha, "oracle_threads": threads})


def batch_circuit(c):
    """All shots of one batch circuit: gates once, then every shot's
    measurements from a copy of the post-gate tableau."""
    op, _, _ = C.decode(c.gates)
    meas = np.flatnonzero(np.isin(op, C.MEASURE_ANY + C.NOISE))
    cut = int(meas[0]) if meas.size else c.gates.size
    t = oracle.Tableau(c.n)
    t.run(c.gates[:cut])
    state = t.get()
    outs = []
    for shot in range(c.shots):
        t.set(*state)
        t.meas_counter = 0
        outs.append(t.run(c.gates[cut:], seed=C.PHILOX_SEED, circuit_id=c.circuit_id,
                          shot=shot))
    allout = np.concatenate(outs) if outs else np.zeros(0, np.uint8)
    return {"c": c.circuit_id, "n": c.n, "shots": c.shots, "n_meas": c.n_meas,
            "outcomes_sha256": D.outcomes_sha(allout)[:32]}


def cfg4(threads):
    t0 = time.time()
    circs = C.config4()
    gsha = [D.gates_sha(c.gates) for c in circs]
    log(f"cfg4: generated {len(circs)} circuits in {time.time() - t0:.0f} s")
    # largest first, so the pool ends evenly
    order = sorted(range(len(circs)), key=lambda i: -circs[i].n ** 3 * (1 + circs[i].shots))
    res = [None] * len(circs)
    done = 0
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = {ex.submit(batch_circuit, circs[i]): i for i in order}
        for f in cf.as_completed(futs):
            res[futs[f]] = f.result()
            done += 1
            if done % 256 == 0:
                log(f"cfg4: {done}/{len(circs)} circuits, {time.time() - t0:.0f} s")
    import hashlib
    all_g = hashlib.sha256("".join(gsha).encode()).hexdigest()
    write("cfg4", {
        "family": "cfg4", "what": "config 4: 4096 random-layer circuits, n ~ U{16..512}, "
                                  "depth n, 1-64 shots, final MZ on all qubits",
        "seed": C.PHILOX_SEED, "gates_sha256_of_circuit_shas": all_g,
        "outcomes": "per circuit: sha256 (first 128 bits, hex) of its shots' outcome "
                    "bytes concatenated in shot order",
        "circuits": res, "oracle_threads": threads})


def cfg5(threads, requests):
    reqs = [C.config5_request(c) for c in range(requests)]
    res = [None] * len(reqs)
    t0 = time.time()
    # largest first; the small requests run in parallel, one core each
    big = [i for i in range(len(reqs)) if reqs[i].n >= 1000]
    small = [i for i in range(len(reqs)) if reqs[i].n < 1000]

    def one(i, th):
        r = reqs[i]
        t1 = time.time()
        out, tsha = whole_run(r.n, r.gates, C.PHILOX_SEED, r.circuit_id, 0, th)
        assert out.size == r.n_meas
        log(f"cfg5: request {i} n={r.n} ({r.n_gates} gates, {out.size} meas) "
            f"{time.time() - t1:.0f} s")
        return {"c": r.circuit_id, "n": r.n, "n_gates": r.n_gates, "n_meas": int(out.size),
                "gates_sha256": D.gates_sha(r.gates), "outcomes_sha256": D.outcomes_sha(out),
                "outcomes_packed": D.pack_outcomes(out), "tableau_sha256": tsha}

    for i in sorted(big, key=lambda i: -reqs[i].n):
        res[i] = one(i, threads)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for i, v in zip(small, ex.map(lambda i: one(i, 1), small)):
            res[i] = v
    log(f"cfg5: {len(reqs)} requests in {time.time() - t0:.0f} s")
    write("cfg5", {
        "family": "cfg5", "what": "served family requests 0..R-1: n log-uniform in "
                                  "[50, 5000], depth 2n, MZR on 5% every 20 layers, "
                                  "final MZ on all",
        "seed": C.PHILOX_SEED, "shot": 0, "requests": res, "oracle_threads": threads})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("families", nargs="*", default=["cfg3", "cfg4", "cfg5"])
    ap.add_argument("--threads", type=int, default=oracle.all_cores())
    ap.add_argument("--requests", type=int, default=SERVED_REQUESTS)
    a = ap.parse_args()
    for fam in a.families:
        if fam == "cfg3":
            cfg3(a.threads)
        elif fam == "cfg4":
            cfg4(a.threads)
        elif fam == "cfg5":
            cfg5(a.threads, a.requests)
        else:
            raise SystemExit(f"unknown family {fam}")


if __name__ == "__main__":
    main()
