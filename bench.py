"""Benchmark of the stabilizer-tableau hot path on GB300.

Default workload (the batched family): 4,096 independent random-layer
Clifford circuits, n ~ U{16..512}, depth n (H or S on every qubit, then n/2
random disjoint CNOT/CZ pairs, CNOT:CZ = 3:1), 1-64 shots each, a final Z
measurement of every qubit with Philox outcomes -- 5.5e8 gates (counted once
per circuit) and 3.5e7 measurements (over all shots).  One "step" is one
replay of the whole batch as one persistent launch (a CUDA graph), with the
compiled batch resident in device memory when timing starts; the compiled
batch (2.3 GB) is larger than L2, and L2 is flushed (a 256 MB device write)
before every timed step anyway.

The JSON line carries, beside the batched (per-shot) value:
* the plain path: the same circuits one launch sequence per shot
  (tab_run of a compiled program), timed on every 16th circuit and scaled;
* the terminal-measurement sampler on the same batch (same outcome bytes);
* e2e: tab_batch_run_packed (the batched run through the C ABI) with host
  gate lists and a pinned host output buffer (host compile, upload, run and
  the outcome copy per step);
* the roofline of the batched kernel against the logic-op ceiling measured
  live by tab_measure_peaks;
* the n = 1,000 plain tableau (1,000 layers, 1,000 final measurements) as an
  extra key;
* cpu_baseline: the CPU oracle on (circuit, shot) runs drawn from the same
  batch, on one core and on every core.

`--impl reference` times the CPU oracle (an unpacked one-byte-per-bit
restatement of the same algorithm) on the same workload instead.  Under
torchrun every rank runs an independent replica on its own GPU (weak scaling,
no collective on the data path); rank 0 prints.

Other workloads (`--workload`): `cfg1` (n=10), `cfg2` (the n=1,000 plain
step), `cfg3` (n=10,000 with MZR rounds), `served` (Poisson request stream to
the continuous-batching server), `sweep` (the paper's own benchmark: uniformly
random n-qubit Cliffords, no measurements, n = 2 ... 8192; one JSON line with
a point per n), `extras` (the next-step features timed on their own).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Clifford gates/sec and measurements/sec, batched vs plain path; "
          "p50/p99 latency")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# Algorithmic work per unit (a unit is one 32-row word of a touched column).
# Logic ops of each gate rule per 32-row word: H 1, S 2, S^dag 2, Paulis 1,
# CNOT 4, CZ 4, SWAP 0; a random-outcome measurement's rowsum costs 9 logic
# ops per (column, 32-row word) on the columns where the pivot row is not I,
# about 3/4 of the n columns.  A gate covers 2n/32 words of each column.
GATE_OPS = {1: 1, 2: 1, 3: 1, 4: 1, 5: 2, 6: 2, 7: 4, 8: 4, 9: 0}
MEAS_OPS_PER_UNIT = 9
PIVOT_SUPPORT = 0.75
# Bytes a random-outcome measurement of the streaming engine reads and writes:
# ~3/4 n supported columns, X and Z planes, 2n/8 bytes each, read + written.
# DRAM bytes (read + write) per launch from one ncu capture of the current
# build, by kernel; None until a capture of the current build exists.
# k_batch: the four size-class launches of one step.  Captured on the
# 512-circuit slice (294.9 MB over its four launches for 7.03e7 gates: the
# compiled gate stream, the circuit images and the outcomes, all in
# proportion to the gates), scaled to the full family's 5.52e8 gates.
# k_measure_resident: one launch of the n=1000 step's 1,000 measurements
# (profiles/k_measure_resident_n1000.md, 595.2 KB read, nothing written).
# k_measure: one step of the n=10,000 family, 10 launches (one per MZR
# round) of 173.1 MB each (profiles/k_measure_n10000.md); its roofline's
# algorithmic bytes are per step too.
TRAFFIC_BYTES = {"k_batch": 294.9e6 * 551688025 / 70335522, "k_measure_resident": 595.2e3,
                 "k_measure": 10 * 173.1e6}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="batched",
                   choices=["batched", "cfg1", "cfg2", "cfg3", "served", "sweep", "extras"])
    p.add_argument("--sweep-max", type=int, default=8192, help="sweep: largest n")
    p.add_argument("--requests", type=int, default=500, help="served: number of requests")
    p.add_argument("--circuits", type=int, default=4096, help="batched: number of circuits")
    p.add_argument("--engine", default="auto", choices=["auto", "single", "grid", "stream"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="batched: skip the n=1000 key")
    p.add_argument("--timed-only", action="store_true",
                   help="batched: only the tuned replays (profiler launch lists); no plain-path, "
                        "sampler, e2e, extra or baseline keys")
    return p.parse_args()


# ------------------------------------------------------------ distributed ---

def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- workloads ---

def workload(name, rank):
    from workloads import circuits as C
    if name == "cfg1":
        c = C.config1(seed_index=rank)
        desc = ("plain tableau n=10, 20 random layers (H/S per qubit, 5 CNOT pairs), "
                "final MZ on all qubits, 1 shot")
    elif name == "cfg2":
        c = C.config2(seed_index=rank)
        desc = ("plain tableau n=1000, 1000 random layers (H/S per qubit, n/2 CNOT/CZ "
                "pairs 3:1), final MZ on all qubits, 1 shot")
    else:
        c = C.config3(seed_index=rank)
        desc = ("plain tableau n=10000, 100 random layers, MZR on 1000 random qubits "
                "after every 10th layer, 1 shot")
    return c, desc


def batch_circuits(count, rank):
    """The batched family's circuits (circuit ids offset by rank), generated
    on all cores: each circuit has its own seeded generator, so the result
    does not depend on the thread count."""
    from workloads import circuits as C
    idx = list(range(count))
    chunks = [idx[i::32] for i in range(32)]
    with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
        parts = list(ex.map(lambda ch: C.config4(m=4096, only=ch), chunks))
    circs = [None] * count
    for ch, part in zip(chunks, parts):
        for i, c in zip(ch, part):
            circs[i] = c
    return circs, [(c.n, c.gates, c.shots, c.circuit_id + 4096 * rank) for c in circs]


def split_runs(c):
    """Maximal runs of gates and of measurements of a circuit, in program
    order: [("gates", words), ("measure", words), ...]."""
    from workloads import circuits as C
    op, _, _ = C.decode(c.gates)
    m = np.isin(op, C.MEASURE)
    if m.size == 0:
        return []
    cuts = np.flatnonzero(np.diff(m.astype(np.int8))) + 1
    bounds = [0] + cuts.tolist() + [int(m.size)]
    return [("measure" if m[a] else "gates", c.gates[a:b]) for a, b in zip(bounds[:-1], bounds[1:])]


def gate_ops(c):
    """Logic ops of a circuit's gates (GATE_OPS per 32-row word, 2n/32 words)."""
    from workloads import circuits as C
    op, _, _ = C.decode(c.gates)
    hist = np.bincount(op.astype(np.int64), minlength=16)
    return (2.0 * c.n / 32.0) * float(sum(GATE_OPS.get(i, 0) * int(hist[i]) for i in range(16)))


def meas_ops(n, count):
    """Logic ops of `count` random-outcome measurements on n qubits."""
    return count * MEAS_OPS_PER_UNIT * PIVOT_SUPPORT * n * (2.0 * n / 32.0)


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        # the sampled clock log (TAB_CLOCKS_DIR, else the system temp directory)
        self.path = os.path.join(os.environ.get("TAB_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"tab_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- oracle ---

def all_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_step_seconds(c, budget_s):
    """Oracle seconds (one core) for one full step of circuit c, extrapolated
    from a time-bounded sample: random layers one at a time for about half
    the budget, then the circuit's measurement ops one at a time for the
    other half."""
    import oracle
    from workloads import circuits as C
    op, _, _ = C.decode(c.gates)
    is_meas = np.isin(op, C.MEASURE)
    gate_words = c.gates[~is_meas]
    meas_words = c.gates[is_meas]
    per_layer = c.n + c.n // 2 + 2            # gates + 2 barrier words per layer
    t = oracle.Tableau(c.n)
    layers, t0 = 0, time.perf_counter()
    while layers < c.depth and time.perf_counter() - t0 < budget_s / 2:
        t.run(gate_words[layers * per_layer:(layers + 1) * per_layer])
        layers += 1
    tg = time.perf_counter() - t0
    meas, t1 = 0, time.perf_counter()
    while meas < meas_words.size and time.perf_counter() - t1 < budget_s / 2:
        t.run(meas_words[meas:meas + 1], seed=1)
        meas += 1
    tm = time.perf_counter() - t1
    est = tg * (c.depth / max(layers, 1)) + (tm * (c.n_meas / meas) if meas else 0.0)
    sample = (f"first {layers} of {c.depth} layers ({tg:.2f} s) and {meas} of {c.n_meas} "
              f"measurements ({tm:.2f} s) on one core, scaled to the full step")
    return est, sample


def oracle_batch_rate(shapes, get_circuit, budget_s, threads, seed):
    """The oracle as it stands on the batched family: (circuit, shot) pairs
    drawn uniformly from all of the batch's pairs, each a full run from |0^n>
    (gates, then the shot's measurements), on `threads` threads, new pairs
    started while the elapsed time is under budget_s.  A circuit's gates
    count once per circuit in the metric, so a shot is credited with
    gates / shots (and its n measurements); the ratio of credited work to
    elapsed time estimates the whole batch's rate.  Returns (gates/s,
    meas/s, seconds, pairs done)."""
    import oracle
    from workloads import circuits as C
    ns, shots = shapes
    rng = np.random.default_rng(seed)
    pair_c = np.repeat(np.arange(len(ns)), shots)
    pair_s = np.concatenate([np.arange(s) for s in shots])
    order = rng.permutation(pair_c.size)
    cache = {}

    def run_pair(i):
        c = get_circuit(int(pair_c[i]), cache)
        oracle.run_circuit(c.n, c.gates, seed=C.PHILOX_SEED, circuit_id=c.circuit_id,
                           shot=int(pair_s[i]))
        return c.n_gates / c.shots, c.n_meas

    t0 = time.perf_counter()
    credit_g = credit_m = 0.0
    done = 0
    nxt = 0
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        running = set()
        while True:
            while len(running) < threads and time.perf_counter() - t0 < budget_s \
                    and nxt < order.size:
                running.add(ex.submit(run_pair, order[nxt]))
                nxt += 1
            if not running:
                break
            fin, running = cf.wait(running, return_when=cf.FIRST_COMPLETED)
            for f in fin:
                g, m = f.result()
                credit_g += g
                credit_m += m
                done += 1
    dt = time.perf_counter() - t0
    return credit_g / dt, credit_m / dt, dt, done


def batch_circuit_getter(rank):
    from workloads import circuits as C

    def get(ci, cache):
        if ci not in cache:
            c = C.config4(m=4096, only=[ci])[0]
            c.circuit_id += 4096 * rank
            cache[ci] = c
        return cache[ci]
    return get


# ------------------------------------------------------------- reference ---

def run_reference(args, ws, rank):
    if rank != 0:
        return
    from workloads import circuits as C
    if args.workload in ("cfg1", "cfg2", "cfg3"):
        c, desc = workload(args.workload, 0)
        budget = max(1.0, 150.0 / (args.steps + args.warmup))
        for _ in range(args.warmup):
            oracle_step_seconds(c, min(budget, 2.0))
        times, samples = [], []
        for _ in range(args.steps):
            est, sample = oracle_step_seconds(c, budget)
            times.append(est)
            samples.append(sample)
        ms = 1000.0 * statistics.mean(times)
        value, meas_s = c.n_gates / (ms / 1000.0), c.n_meas / (ms / 1000.0)
        cores, sample = 1, samples[-1]
        config = {"workload": desc, "n": c.n, "gates": c.n_gates, "measurements": c.n_meas}
    else:
        # the batched family: each step is a time-bounded sample of the
        # batch's (circuit, shot) runs on every core; ms_per_step is the
        # sample's own duration
        shapes = C.config4_shapes()
        cores = all_cores()
        budget = min(12.0, max(2.0, 90.0 / (args.steps + args.warmup)))
        get = batch_circuit_getter(0)
        for w in range(args.warmup):
            oracle_batch_rate(shapes, get, min(budget, 2.0), cores, seed=100 + w)
        rates, durs, pairs = [], [], 0
        for s in range(args.steps):
            g, m, dt, done = oracle_batch_rate(shapes, get, budget, cores, seed=200 + s)
            rates.append((g, m))
            durs.append(dt)
            pairs += done
        value = statistics.mean(r[0] for r in rates)
        meas_s = statistics.mean(r[1] for r in rates)
        ms = 1000.0 * statistics.mean(durs)
        sample = (f"{pairs} (circuit, shot) runs drawn uniformly from the batch's "
                  f"{int(shapes[1].sum())}, {args.steps} steps of ~{budget:.0f} s on {cores} "
                  "cores, each shot credited with its circuit's gates / shots")
        config = {"workload": "batched: 4096 random-layer circuits, n ~ U[16,512], depth n, "
                              "1-64 shots, final MZ on all qubits",
                  "step": "a time-bounded sample of (circuit, shot) runs"}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "gates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "meas_per_s": meas_s, "config": config,
        "cpu_baseline": {"value": value, "unit": "gates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "gates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- peaks ---

def measured_hbm():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def live_peaks():
    """Ceilings of this GPU measured now (tab_measure_peaks) plus the
    measured HBM copy bandwidth."""
    from paper_2408_00384_gb300 import tab
    pk = tab.measure_peaks()
    pk["hbm_gbs"], pk["hbm_source"] = measured_hbm()
    return pk


def alu_roofline(kernel, ops, kernel_ms, pk, extra=None):
    achieved = ops / (kernel_ms / 1000.0) / 1e12
    roof = {"kernel": kernel, "bound": "alu", "unit": "Top/s", "achieved": achieved,
            "peak": pk["logic_tops"], "frac": achieved / pk["logic_tops"],
            "peak_source": (f"measured: lop3.b32 on {pk['sms']} SMs at "
                            f"{pk['sm_clock_mhz']:.0f} MHz "
                            f"({pk['logic_ops_per_clk_sm']:.1f} ops/clk/SM), tab_measure_peaks"),
            "traffic": TRAFFIC_BYTES.get(kernel), "kernel_ms": kernel_ms,
            "alg_ops_per_launch": ops}
    if extra:
        roof.update(extra)
    return roof


# ------------------------------------------------------------- plain path ---

def run_plain(args, ws, rank, local, name=None, steps=None, warmup=None, cpu=True, pk=None):
    import torch
    from paper_2408_00384_gb300 import tab
    from workloads import circuits as C

    name = name or args.workload
    steps = steps or args.steps
    warmup = warmup if warmup is not None else args.warmup
    torch.cuda.set_device(local)
    c, desc = workload(name, rank)
    runs = split_runs(c)
    stream = torch.cuda.Stream()
    t = tab.Tableau(c.n, stream=stream)
    eng = {"auto": tab.ENGINE_AUTO, "single": tab.ENGINE_SINGLE_CTA,
           "grid": tab.ENGINE_GRID, "stream": tab.ENGINE_STREAM}
    t.set_engine(eng[args.engine])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # one program per run of gates / of measurements, timed separately (the
    # same launches as one program of all the runs)
    progs = [tab.Program(c.n, words) for _, words in runs]
    kinds = [k for k, _ in runs]

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        t.reset()
        t.set_rng(C.PHILOX_SEED, rank, 0)
        for i, p in enumerate(progs):
            t.run(p)
            if evs:
                evs[i + 1].record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    t.sync()
    if pk is None:
        pk = live_peaks()
    nprog = len(progs)
    all_evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nprog + 1)]
               for _ in range(steps)]
    launches0 = t.launches
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    for s in range(steps):
        with torch.cuda.stream(stream):   # same stream as the timed work
            flush.fill_(s & 0xFF)
        step(all_evs[s])
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    t.sync()
    launches = t.launches - launches0
    per_step = [all_evs[s][0].elapsed_time(all_evs[s][-1]) for s in range(steps)]
    per_kind = {}
    for k in set(kinds):
        per_kind[k] = [sum(all_evs[s][i].elapsed_time(all_evs[s][i + 1])
                           for i, kk in enumerate(kinds) if kk == k) for s in range(steps)]
    ms_local = statistics.mean(per_step)
    ms = allreduce_max(ms_local, ws)
    value = ws * c.n_gates / (ms / 1000.0)
    meas_s = ws * c.n_meas / (ms / 1000.0)

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pinned = torch.from_numpy(c.gates.view(np.int64)).pin_memory()
        host_gates = pinned.numpy().view(np.uint64)
        out = np.zeros(c.n_meas, np.uint8)
        ke = max(3, min(steps, 10))
        for i in range(ke + 2):
            if i == 2:
                torch.cuda.synchronize()
                barrier(ws)
                t0 = time.perf_counter()
                x0 = t.transfer_bytes()
            t.reset()
            t.set_rng(C.PHILOX_SEED, rank, 0)
            t.apply(host_gates)
            got = t.read_outcomes()   # synchronizes: device -> host copy of the outcomes
            out[:got.size] = got
        torch.cuda.synchronize()
        barrier(ws)
        e2e_s = allreduce_max((time.perf_counter() - t0) / ke, ws)
        x1 = t.transfer_bytes()
        # the gate list is read on the host (validated and compiled there);
        # what crosses to the device is the compiled program
        e2e = {"value": ws * c.n_gates / e2e_s, "unit": "gates/s",
               "h2d_bytes_per_step": (x1[0] - x0[0]) // ke,
               "d2h_bytes_per_step": (x1[1] - x0[1]) // ke,
               "host_input_bytes_per_step": int(c.gates.nbytes),
               "ms_per_step": 1000.0 * e2e_s}

    # ---- roofline of the dominant kernel
    kind_ms = {k: statistics.mean(v) for k, v in per_kind.items()}
    dom = max(kind_ms, key=kind_ms.get)
    n = c.n
    eng_res = t.engine_resolved()[0]
    extra = None
    if dom == "measure":
        kname = {tab.ENGINE_SINGLE_CTA: "k_sct_program", tab.ENGINE_GRID: "k_measure_resident",
                 tab.ENGINE_STREAM: "k_measure"}[eng_res]
        alg = meas_ops(n, c.n_meas)
        if kname != "k_measure":
            # exact logic ops: MEAS_OPS_PER_UNIT per (support column, 32-row
            # word) of the random-outcome rowsums, the supports counted by the
            # streaming engine's work counters on one untimed step (every
            # engine meets the same tableaus, bit for bit); the model that
            # takes every measurement as random with a support of 3/4 n is
            # kept beside it
            with tab.Tableau(c.n, stream=stream) as tw:
                tw.set_engine(tab.ENGINE_STREAM)
                tw.count_work(True)
                tw.reset()
                tw.set_rng(C.PHILOX_SEED, rank, 0)
                for prog in progs:
                    tw.run(prog)
                wcnt = tw.work_counts()
            model = alg
            alg = MEAS_OPS_PER_UNIT * wcnt["support_cols"] * 2.0 * ((n + 31) // 32)
            extra = {"work_counts": wcnt,
                     "model": {"ops": model,
                               "frac": model / (kind_ms[dom] / 1000.0) / 1e12 / pk["logic_tops"],
                               "note": "every measurement random, support 3/4 n"}}
    else:
        kname = "k_sct_program" if eng_res == tab.ENGINE_SINGLE_CTA else "k_gates_block"
        alg = gate_ops(c)
    if kname == "k_measure":
        # the streaming engine sweeps the tableau in HBM/L2.  Algorithmic
        # bytes of one step, exactly, from the engine's work counters (one
        # more step, untimed, counted): a random measurement reads the pivot
        # column (n/8 B) and row p (2n/8 B) and reads and writes its pivot
        # row's |supp(p)| columns, 2 planes of 2n/8 B each; a deterministic
        # one reads its k multiplied rows (2n/8 B each).  The model that
        # takes |supp(p)| = 3/4 n (0.75 n^2 bytes per measurement) is kept
        # beside it.  The tableau (n^2/2 bytes) fits GB300's L2 up to
        # n ~ 16,000, so both ceilings are given.
        t.count_work(True)
        step()
        wc = t.work_counts()
        t.count_work(False)
        col = 2.0 * n / 8.0
        alg_bytes = (wc["support_cols"] * 2 * col * 2 + wc["random"] * (n / 8.0 + col)
                     + wc["det_rows"] * col)
        model_bytes = 0.75 * n * n * c.n_meas
        achieved = alg_bytes / (kind_ms[dom] / 1000.0) / 1e9
        roof = {"kernel": kname, "bound": "hbm", "unit": "GB/s", "achieved": achieved,
                "peak": pk["hbm_gbs"], "frac": achieved / pk["hbm_gbs"],
                "peak_source": pk["hbm_source"],
                "l2": {"peak_gbs": pk["l2_rw_gbs"], "frac": achieved / pk["l2_rw_gbs"],
                       "peak_source": "measured: read + write over a 64 MiB set, "
                                      "tab_measure_peaks"},
                "traffic": TRAFFIC_BYTES.get(kname), "kernel_ms": kind_ms,
                "alg_bytes_per_launch": alg_bytes, "work_counts": wc,
                "model": {"bytes": model_bytes,
                          "achieved": model_bytes / (kind_ms[dom] / 1000.0) / 1e9,
                          "note": "0.75 n^2 bytes per measurement (support 3/4 n)"}}
    else:
        roof = alu_roofline(kname, alg, kind_ms[dom], pk, dict({"kernel_ms": kind_ms}, **(extra or {})))

    line = {
        "metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": ws,
        "steps": steps, "warmup": warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "meas_per_s": meas_s,
        "latency_ms": {"p50": float(np.percentile(per_step, 50)),
                       "p99": float(np.percentile(per_step, 99))},
        "config": {"workload": desc, "n": c.n, "gates": c.n_gates,
                   "measurements": c.n_meas, "parallelism": f"replicas x{ws}",
                   "l2": "flushed before every timed step (256 MB device write)",
                   "engine": args.engine,
                   "measure_engine": {tab.ENGINE_SINGLE_CTA: "single-CTA",
                                      tab.ENGINE_GRID: "grid-resident",
                                      tab.ENGINE_STREAM: "streaming"}[t.engine_resolved()[0]]},
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roof,
        "e2e": e2e,
    }
    if cpu and rank == 0 and not args.no_cpu_baseline and ws == 1:
        est, sample = oracle_step_seconds(c, 12.0)
        line["cpu_baseline"] = {"value": c.n_gates / est, "unit": "gates/s", "cores": 1,
                                "kind": "oracle", "sample": sample}
    elif rank == 0 and ws == 1:
        line["cpu_baseline"] = None
    for p in progs:
        p.close()
    t.close()
    return line


# ---------------------------------------------------------- batched path ---

def run_batched(args, ws, rank, local):
    import torch
    from paper_2408_00384_gb300 import tab
    from workloads import circuits as C

    torch.cuda.set_device(local)
    t_gen = time.perf_counter()
    circs, circuits = batch_circuits(args.circuits, rank)
    gen_s = time.perf_counter() - t_gen
    t_c = time.perf_counter()
    b = tab.Batch(circuits)
    compile_s = time.perf_counter() - t_c
    info = b.info()
    out = torch.empty(max(info["out_bytes"], 1), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # autotune the persistent launch's CTA shape on this batch (untimed)
    tuned_threads, tuned_ms = b.tune(C.PHILOX_SEED, out.data_ptr(), stream)
    launch = {"size_classes": [{k: v for k, v in c.items()} for c in b.classes()]}
    for _ in range(args.warmup):
        b.exec(C.PHILOX_SEED, out.data_ptr(), stream)
    torch.cuda.synchronize()
    pk = live_peaks()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
        evs[s][0].record(stream)
        b.exec(C.PHILOX_SEED, out.data_ptr(), stream)
        evs[s][1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    per = [a.elapsed_time(z) for a, z in evs]
    ms = allreduce_max(statistics.mean(per), ws)
    n_gates, n_meas = info["n_gates"], info["n_meas"]

    # ---- the plain one-circuit-per-launch path on every 16th circuit, all
    # its shots (circuits are i.i.d., so 16 x the sample estimates the batch)
    stride = 16
    plain_ms = 0.0
    sample_g = sample_m = 0
    for c, (_, _, _, cid) in zip(circs[::stride], circuits[::stride]):
        if args.timed_only:
            break
        with tab.Program(c.n, c.gates) as prog, tab.Tableau(c.n, stream=stream) as t:
            t.reset()
            t.run(prog)   # warm the engine's first-use set-up outside the timing
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for shot in range(c.shots):
                t.reset()
                t.set_rng(C.PHILOX_SEED, cid, shot)
                t.run(prog)
            e1.record(stream)
            t.sync()
            plain_ms += e0.elapsed_time(e1)
        sample_g += c.n_gates
        sample_m += c.n_meas * c.shots
    plain_gps = sample_g / (plain_ms / 1000.0) if plain_ms else float("nan")
    plain_mps = sample_m / (plain_ms / 1000.0) if plain_ms else float("nan")
    if args.timed_only:
        args.no_e2e = args.no_extras = args.no_cpu_baseline = True

    # ---- the terminal-measurement sampler on the same batch (reported apart
    # from the per-shot numbers): same outcome bytes, checked here
    sampler = None
    sb = None if args.timed_only else tab.Batch(circuits, sample_terminal=True)
    s_out = torch.empty_like(out) if sb is not None else None
    if sb is None:
        s_ms = float("nan")
    else:
        s_threads, _ = sb.tune(C.PHILOX_SEED, s_out.data_ptr(), stream)
        b.exec(C.PHILOX_SEED, out.data_ptr(), stream)
        for _ in range(max(args.warmup, 1)):
            sb.exec(C.PHILOX_SEED, s_out.data_ptr(), stream)
        torch.cuda.synchronize()
        same = bool(torch.equal(out, s_out))
        s_evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
        for s in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(s & 0xFF)
            s_evs[s][0].record(stream)
            sb.exec(C.PHILOX_SEED, s_out.data_ptr(), stream)
            s_evs[s][1].record(stream)
        torch.cuda.synchronize()
        s_ms = allreduce_max(statistics.mean(a.elapsed_time(z) for a, z in s_evs), ws)
        sampler = {"ms_per_step": s_ms, "gates_per_s": ws * n_gates / (s_ms / 1000.0),
                   "meas_per_s": ws * n_meas / (s_ms / 1000.0),
                   "circuits_sampled": sb.sampled, "threads": s_threads,
                   "outcomes_equal_per_shot_run": same,
                   "note": "terminal measurements run once per circuit with affine sign forms, "
                           "every shot evaluated from its Philox bits"}
        sb.close()

    # ---- end to end: tab_batch_run_packed with host gate lists and a pinned
    # host output buffer (host compile, upload, run, outcome copy) per step
    e2e = None
    if not args.no_e2e:
        host_out = torch.empty(max(info["out_bytes"], 1), dtype=torch.uint8).pin_memory().numpy()
        ke = 2
        tab.batch_run(circuits, C.PHILOX_SEED, out=host_out)   # warm-up
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(ke):
            tab.batch_run(circuits, C.PHILOX_SEED, out=host_out)
        e2e_s = allreduce_max((time.perf_counter() - t0) / ke, ws)
        same_e2e = bool(np.array_equal(host_out[:info["out_bytes"]],
                                       out.cpu().numpy()[:info["out_bytes"]]))
        e2e = {"value": ws * n_gates / e2e_s, "unit": "gates/s",
               "h2d_bytes_per_step": int(b.h2d_bytes), "d2h_bytes_per_step": int(info["out_bytes"]),
               "host_input_bytes_per_step": int(sum(c.gates.nbytes for c in circs)),
               "ms_per_step": 1000.0 * e2e_s, "meas_per_s": ws * n_meas / e2e_s,
               "outcomes_equal_device_run": same_e2e,
               "call": "tab.batch_run -> tab_batch_run_packed (chunks compiled on the host "
                       "pool while the device runs the chunk before, uploads, the size-class "
                       "launches of each chunk, per-chunk outcome copies to pinned host "
                       "memory)"}

    # ---- roofline of the batched kernel: every circuit's gates once, and
    # every shot's random-outcome rowsums at MEAS_OPS_PER_UNIT per (support
    # column, 32-row word), the supports counted on the device by one more,
    # untimed replay with the kernel's work counters on.  The model that
    # takes every measurement as random with a support of 3/4 n is kept
    # beside it.
    b.count_work(True)
    b.exec(C.PHILOX_SEED, out.data_ptr(), stream)
    torch.cuda.synchronize()
    work = b.work_counts()
    b.count_work(False)
    ops = sum(gate_ops(c) for c in circs) + MEAS_OPS_PER_UNIT * work["support_words"]
    model_ops = sum(gate_ops(c) + c.shots * meas_ops(c.n, c.n_meas) for c in circs)
    k_ms = statistics.mean(per)
    roof = alu_roofline("k_batch", ops, k_ms, pk,
                        {"smem_gbs_peak": pk["smem_gbs"], "work_counts": work,
                         "model": {"ops": model_ops,
                                   "frac": model_ops / (k_ms / 1000.0) / 1e12 / pk["logic_tops"],
                                   "note": "every measurement random, support 3/4 n"},
                         "note": "per-shot tableaus live in shared memory; the compiled batch "
                                 "streams from HBM once per step"})

    line = {
        "metric": METRIC, "value": ws * n_gates / (ms / 1000.0), "unit": "gates/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "meas_per_s": ws * n_meas / (ms / 1000.0),
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99)),
                       "unit": "per batch replay"},
        "config": {"workload": f"batched: {len(circs)} random-layer circuits, n ~ U[16,512], "
                               "depth n, 1-64 shots, final MZ on all qubits",
                   "gates": n_gates, "measurements": n_meas, "parallelism": f"replicas x{ws}",
                   "l2": "flushed before every timed step (256 MB device write); the compiled "
                         "batch is larger than L2",
                   "launch": launch, "generate_s": gen_s, "compile_s": compile_s,
                   "autotune": {"threads_first_class": tuned_threads,
                                "best_runs_ms_sum": tuned_ms,
                                "tried": "128/256/512/1024 threads per CTA, each size class "
                                         "run alone once per shape"}},
        "gpu_launches": b.launches * args.steps, "clocks": clk, "roofline": roof,
        "e2e": e2e,
        "plain_path": None if args.timed_only else {
            "gates_per_s": ws * plain_gps, "meas_per_s": ws * plain_mps,
            "ms_estimated": n_gates / plain_gps * 1000.0,
            "sample": f"every {stride}th circuit ({len(circs[::stride])}), all its "
                      "shots, one tab_run per shot, CUDA events",
            "batched_speedup": (n_gates / plain_gps * 1000.0) / ms},
        "sampler": sampler,
        "peaks": pk,
    }
    b.close()
    del out, flush
    torch.cuda.empty_cache()
    if not args.no_extras:
        p = run_plain(args, ws, rank, local, name="cfg2", steps=10, warmup=3, cpu=False, pk=pk)
        line["cfg2"] = {k: p[k] for k in ("value", "unit", "ms_per_step", "meas_per_s",
                                          "latency_ms", "roofline", "e2e", "gpu_launches")}
        line["cfg2"]["workload"] = p["config"]["workload"]
        line["gpu_launches"] += p["gpu_launches"]
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        shapes = (np.array([c.n for c in circs]), np.array([c.shots for c in circs]))

        def get(ci, cache):
            return circs[ci]
        g1, m1, d1, n1 = oracle_batch_rate(shapes, get, 8.0, 1, seed=7)
        cores = all_cores()
        ga, ma, da, na = oracle_batch_rate(shapes, get, 8.0, cores, seed=8)
        line["cpu_baseline"] = {
            "value": ga, "unit": "gates/s", "cores": cores, "kind": "oracle",
            "meas_per_s": ma,
            "sample": f"{na} (circuit, shot) runs drawn uniformly from the batch in {da:.1f} s "
                      f"on {cores} threads, each a full oracle run, each shot credited with "
                      "its circuit's gates / shots",
            "single_core": {"value": g1, "meas_per_s": m1, "cores": 1,
                            "sample": f"{n1} runs in {d1:.1f} s on one core"}}
    elif rank == 0 and ws == 1:
        line["cpu_baseline"] = None
    return line


def run_served(args, ws, rank, local):
    """Served family: circuits with n log-uniform in [50, 5000], depth 2n, MZR on
    5 % every 20 layers, final MZ on all qubits.  Pass 1 submits every request
    at once (saturated) to calibrate the service rate mu; pass 2 submits them
    as a Poisson stream at lambda = 0.7 mu and records arrival-to-outcome
    latency.  Tableaus stay resident for their whole circuit; admission is by
    device memory (150 GB cap) and slots."""
    import torch
    from paper_2408_00384_gb300 import tab
    from workloads import circuits as C

    torch.cuda.set_device(local)
    t_gen = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
        reqs = list(ex.map(lambda c: C.config5_request(c + 100000 * rank), range(args.requests)))
    print(f"[served] generated {len(reqs)} requests in {time.perf_counter() - t_gen:.1f} s",
          file=sys.stderr, flush=True)
    gates_total = sum(r.n_gates for r in reqs)
    meas_total = sum(r.n_meas for r in reqs)
    cfg = dict(mem_budget_bytes=150 << 30, max_inflight=16, n_streams=8, meas_ctas=32, seed=C.PHILOX_SEED)

    def serve(arrivals):
        lat = []
        launches = 0
        with tab.Server(**cfg) as srv:
            t0 = time.perf_counter()
            tickets = []
            for i, r in enumerate(reqs):
                if arrivals is not None:
                    delay = t0 + arrivals[i] - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                tickets.append((srv.submit(r.n, r.gates, 1, r.circuit_id), time.perf_counter()))
            for i, ((tk, ts), r) in enumerate(zip(tickets, reqs)):
                rc, out, l = srv.wait(tk, timeout_s=300.0)
                if rc != tab.TAB_OK or out.size != r.n_meas:
                    raise RuntimeError(f"request failed: {rc} {tab.last_error()}")
                lat.append(l)
            wall = time.perf_counter() - t0
            st = srv.stats()
        return wall, lat, st

    # warm-up: a few small requests
    with tab.Server(**cfg) as srv:
        for r in reqs[:2]:
            srv.wait(srv.submit(r.n, r.gates, 1, r.circuit_id))
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    wall_sat, lat_sat, st_sat = serve(None)
    mu = len(reqs) / wall_sat
    lam = 0.7 * mu
    arrivals = C.poisson_arrivals(lam, len(reqs))
    wall, lat, st = serve(arrivals)
    barrier(ws)
    clk = clocks.stop()
    wall = allreduce_max(wall, ws)
    ms = 1000.0 * wall
    line = {
        "metric": METRIC, "value": ws * gates_total / wall, "unit": "gates/s", "n_gpus": ws,
        "steps": 1, "warmup": 1, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "meas_per_s": ws * meas_total / wall,
        "latency_ms": {"p50": 1000.0 * float(np.percentile(lat, 50)),
                       "p99": 1000.0 * float(np.percentile(lat, 99))},
        "throughput_req_per_s": len(reqs) / wall,
        "saturated": {"req_per_s": mu, "gates_per_s": gates_total / wall_sat,
                      "p50_ms": 1000.0 * float(np.percentile(lat_sat, 50)),
                      "p99_ms": 1000.0 * float(np.percentile(lat_sat, 99)),
                      "peak_inflight": st_sat["peak_inflight"]},
        "config": {"workload": f"served: {len(reqs)} requests, n log-uniform [50, 5000], depth 2n, "
                               "MZR on 5% every 20 layers, final MZ on all; Poisson arrivals at "
                               f"0.7 x saturated rate ({lam:.2f} req/s)",
                   "gates": gates_total, "measurements": meas_total,
                   "arrival_rate_per_s": lam, "mem_budget_bytes": 150 << 30,
                   "max_inflight": cfg["max_inflight"], "peak_inflight": st["peak_inflight"],
                   "peak_mem_bytes": st["peak_mem"]},
        "clocks": clk, "roofline": None, "e2e": None,
    }
    return line


# ----------------------------------------------------------------- sweep ---

SWEEP_COUNT = {1024: 10, 2048: 5, 4096: 3, 8192: 2}   # circuits per n (100 below 512)


def run_sweep(args, ws, rank, local):
    """Uniformly random Cliffords (the paper's Fig. 2a workload), no
    measurements: per n, each circuit is applied to |0^n> through the public
    API with its gate list in host memory (host compile, upload and device
    work inside the timed region), after one untimed warm-up circuit.  The
    device column is CUDA-event time of the same circuit compiled and uploaded
    beforehand (tab.Program), on the handle's stream; the CPU column is the
    oracle on one core for n <= 512 (a time-bounded sample of circuits)."""
    import torch
    from paper_2408_00384_gb300 import tab
    from workloads import circuits as C

    torch.cuda.set_device(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = ClockSampler(local)
    clocks.start()
    points = []
    for n in [m for m in C.CLIFFORD_SWEEP_N if m <= args.sweep_max]:
        count = SWEEP_COUNT.get(n, 30 if n == 512 else 100)
        circs = C.clifford_sweep(n, count + 1)
        t = tab.Tableau(n)
        t.apply(circs[0].gates)          # warm-up: kernels, staging, host pool
        t.sync()
        e2e, dev = [], []
        for c in circs[1:]:
            flush.fill_(len(e2e) & 0xFF)
            t.reset()
            torch.cuda.synchronize()
            h0 = time.perf_counter()
            t.apply(c.gates)
            t.sync()
            e2e.append(time.perf_counter() - h0)
            # device time: the same circuit compiled and uploaded beforehand
            prog = tab.Program(n, c.gates)
            flush.fill_(len(e2e) & 0xFF)
            t.reset()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            t.run(prog)
            e1.record()
            torch.cuda.synchronize()
            dev.append(e0.elapsed_time(e1) / 1000.0)
            prog.close()
        t.close()
        gates = statistics.mean(c.n_gates for c in circs[1:])
        pt = {"n": n, "circuits": count, "gates_per_circuit": gates,
              "e2e_ms": 1000.0 * statistics.median(e2e),
              "device_ms": 1000.0 * statistics.median(dev),
              "gates_per_s_e2e": gates / statistics.median(e2e)}
        if n <= 512 and not args.no_cpu_baseline and rank == 0:
            import oracle
            done, t0 = 0, time.perf_counter()
            while done < count and time.perf_counter() - t0 < 2.0:
                oracle.run_circuit(n, circs[1 + done].gates)
                done += 1
            cpu = (time.perf_counter() - t0) / done
            pt["cpu_baseline"] = {"ms": 1000.0 * cpu, "cores": 1, "kind": "oracle",
                                  "sample": f"{done} of {count} circuits"}
        points.append(pt)
    clk = clocks.stop()
    # smallest n from which every compared point has the GPU ahead of the oracle
    cmp_pts = [p for p in points if "cpu_baseline" in p]
    cross = None
    for i, p in enumerate(cmp_pts):
        if all(q["e2e_ms"] < q["cpu_baseline"]["ms"] for q in cmp_pts[i:]):
            cross = p["n"]
            break
    return {"metric": "uniformly random Clifford circuits: time per circuit vs n",
            "unit": "ms per circuit", "n_gpus": ws, "higher_is_better": False,
            "data": "synthetic", "dtype": "u32",
            "config": {"workload": "uniformly random n-qubit Cliffords (Bruhat form "
                                   "b1 w b2 of Sp(2n,2)), no measurements, n = 2 ... "
                                   f"{args.sweep_max}", "l2": "flushed before every circuit"},
            "points": points, "gpu_faster_than_oracle_from_n": cross, "clocks": clk}


# ---------------------------------------------------------------- extras ---

def run_extras(args, ws, rank, local):
    """The next-step features, each timed on its own (CUDA events or host
    wall time around synchronous calls, after one untimed call):
    * expectation values: 1,000 Pauli strings (products of random stabilizer
      subsets and random strings) on the n=1000 random-layer state;
    * the state vector export at n = 20 and 24 (n projector passes over
      2^n amplitudes, then the copy to the host);
    * the row-sharded tableau on the n=1000 random-layer circuit with its
      1,000 final measurements, 1, 2 and 4 shards, against one tableau;
    * the same circuit with 1 % depolarizing noise ops and X / Y measurements
      (host lowering inside tab_apply)."""
    import torch
    from paper_2408_00384_gb300 import tab
    from workloads import circuits as C

    torch.cuda.set_device(local)
    c = C.config2()
    out = {"metric": "next-step features: time per call", "unit": "ms", "n_gpus": ws,
           "higher_is_better": False, "data": "synthetic", "dtype": "u32"}
    # expectation values
    rng = np.random.default_rng(1)
    with tab.Tableau(c.n) as t:
        t.apply(c.gates)
        x, z, _ = t.export()
        strings = []
        for _ in range(900):
            pick = rng.integers(0, 2, size=c.n).astype(bool)
            px = np.bitwise_xor.reduce(x[c.n:][pick].astype(np.int64), axis=0)
            pz = np.bitwise_xor.reduce(z[c.n:][pick].astype(np.int64), axis=0)
            strings.append(px | (pz << 1))
        strings += [rng.integers(0, 4, size=c.n) for _ in range(100)]
        codes = np.array(strings, dtype=np.uint8)
        t.expect(codes[:10])
        reps = []
        for _ in range(5):
            h0 = time.perf_counter()
            v = t.expect(codes)
            reps.append(time.perf_counter() - h0)
        ms = 1000.0 * statistics.median(reps)
        out["expect"] = {"n": c.n, "strings": len(codes), "ms": ms,
                         "strings_per_s": len(codes) / (ms / 1000.0),
                         "nonzero": int((v != 0).sum())}
    # state vector export
    sv = []
    for n in (20, 24):
        g = C.random_clifford(n, C.splitmix64(99 + n)).gates
        with tab.Tableau(n) as t:
            t.apply(g)
            t.statevector()
            reps = []
            for _ in range(3):
                h0 = time.perf_counter()
                t.statevector()
                reps.append(time.perf_counter() - h0)
        ms = 1000.0 * statistics.median(reps)
        sv.append({"n": n, "ms": ms, "amplitudes": 1 << n,
                   "device_bytes_moved": n * 2 * 8 * (1 << n)})
    out["statevector"] = sv
    # row-sharded tableau vs one tableau, the same circuit and outcomes
    sh = []
    with tab.Tableau(c.n) as t:
        t.set_rng(C.PHILOX_SEED, 0, 0)
        t.apply(c.gates)
        want = t.read_outcomes()
        reps = []
        for _ in range(3):
            t.reset()
            t.set_rng(C.PHILOX_SEED, 0, 0)
            h0 = time.perf_counter()
            t.apply(c.gates)
            t.read_outcomes()
            reps.append(time.perf_counter() - h0)
        sh.append({"shards": 0, "ms": 1000.0 * statistics.median(reps)})
    for shards in (1, 2, 4):
        reps, same = [], True
        for _ in range(2):
            with tab.ShardedTableau(c.n, shards) as t:
                t.set_rng(C.PHILOX_SEED, 0, 0)
                h0 = time.perf_counter()
                t.apply(c.gates)
                got = t.read_outcomes()
                reps.append(time.perf_counter() - h0)
                same = same and bool(np.array_equal(got, want))
        sh.append({"shards": shards, "ms": 1000.0 * min(reps), "outcomes_equal": same})
    out["sharded"] = {"workload": "n=1000, 1000 random layers, 1000 final MZ",
                      "points": sh, "note": "shards 0 = one tableau (tab_apply)"}
    # noisy circuit with X / Y measurements
    op, q1, _ = C.decode(c.gates)
    gate_pos = np.flatnonzero(~np.isin(op, C.MEASURE + (C.TAB_BARRIER,)))
    pos = np.sort(rng.choice(gate_pos, size=gate_pos.size // 100, replace=False))
    noise = C.encode(np.full(pos.size, C.TAB_DEPOL1), rng.integers(0, c.n, size=pos.size),
                     C.noise_field(0.01))
    noisy = np.insert(c.gates, pos, noise)
    mz = np.isin(C.decode(noisy)[0], C.MEASURE)
    mx = noisy.copy()
    kinds = np.where(np.arange(mz.sum()) % 2 == 0, C.TAB_MX, C.TAB_MY)
    mx[mz] = C.encode(kinds, C.decode(noisy[mz])[1], 0)
    with tab.Tableau(c.n) as t:
        t.apply(mx)
        t.sync()
        reps = []
        for _ in range(5):
            t.reset()
            h0 = time.perf_counter()
            t.apply(mx)
            t.read_outcomes()
            reps.append(time.perf_counter() - h0)
    out["noisy_xy"] = {"workload": "the n=1000 circuit + 1 % DEPOL1 ops, final MX/MY",
                       "noise_ops": int(pos.size), "ms": 1000.0 * statistics.median(reps)}
    return out


def main():
    args = parse()
    ws, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "extras":
        line = run_extras(args, ws, rank, local)
    elif args.workload == "sweep":
        line = run_sweep(args, ws, rank, local)
    elif args.workload == "batched":
        line = run_batched(args, ws, rank, local)
    elif args.workload == "served":
        line = run_served(args, ws, rank, local)
    else:
        line = run_plain(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
        log = os.environ.get("TAB_BENCH_LOG")  # optional JSONL history of bench lines
        if log:
            with open(log, "a") as f:
                f.write(json.dumps(dict(line, time=time.strftime("%Y-%m-%dT%H:%M:%S"))) + "\n")
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
