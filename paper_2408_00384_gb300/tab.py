"""ctypes binding of libtab (include/tab.h): argument marshalling only.

Every step of the tableau path runs in the library's CUDA kernels; this module
converts numpy arrays and torch streams / tensors to plain pointers and maps
status codes to exceptions.  Importing it raises ImportError when libtab.so is
missing -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TAB_DEBUG=1 selects the debug build (device-side index checks; include/tab.h)
DEBUG = os.environ.get("TAB_DEBUG", "") == "1"
LIB_PATH = os.path.join(_HERE, "libtab_debug.so" if DEBUG else "libtab.so")

TAB_OK, TAB_EINVAL, TAB_ERANGE, TAB_ENOMEM = 0, -1, -2, -3
TAB_ECUDA, TAB_EDEVICE, TAB_ETIMEOUT, TAB_ESTATE = -4, -5, -6, -7
STATUS_NAMES = {0: "TAB_OK", -1: "TAB_EINVAL", -2: "TAB_ERANGE", -3: "TAB_ENOMEM",
                -4: "TAB_ECUDA", -5: "TAB_EDEVICE", -6: "TAB_ETIMEOUT", -7: "TAB_ESTATE"}
MAX_QUBITS = 16384
NOALLOC_SCRATCH_BYTES = 1 << 20
ENGINE_AUTO, ENGINE_SINGLE_CTA, ENGINE_GRID, ENGINE_STREAM = 0, 1, 2, 4
BATCH_MAX_QUBITS = 640

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{os.path.basename(LIB_PATH)} not found at {LIB_PATH}: build it with "
        + ("`python -m paper_2408_00384_gb300.build --debug`" if DEBUG else
           "`python -c 'import __graft_entry__ as g; g.build()'`")
        + " (no CPU fallback exists)")

_L = ctypes.CDLL(LIB_PATH)

_vp, _i32, _i64, _u32, _u64, _sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                    ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t)
_P = ctypes.POINTER


class TabCircuit(ctypes.Structure):
    _fields_ = [("n", _i32), ("gates", _vp), ("n_gates", _i64), ("shots", _i32),
                ("circuit_id", _u64)]


def _sig(name, res, args):
    f = getattr(_L, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("tab_last_error", ctypes.c_char_p, [])
_sig("tab_bytes_required", _sz, [_i32])
_sig("tab_create", ctypes.c_int, [_i32, _P(_vp)])
_sig("tab_create_on", ctypes.c_int, [_i32, _vp, _sz, _vp, _P(_vp)])
_sig("tab_destroy", ctypes.c_int, [_vp])
_sig("tab_num_qubits", ctypes.c_int, [_vp, _P(_i32)])
_sig("tab_set_stream", ctypes.c_int, [_vp, _vp])
_sig("tab_set_rng", ctypes.c_int, [_vp, _u64, _u64, _u32])
_sig("tab_reset", ctypes.c_int, [_vp])
_sig("tab_apply", ctypes.c_int, [_vp, _vp, _i64])
_sig("tab_prog_create", ctypes.c_int, [_i32, _vp, _i64, _P(_vp)])
_sig("tab_prog_destroy", ctypes.c_int, [_vp])
_sig("tab_prog_info", ctypes.c_int, [_vp, _P(_i64), _P(_i64), _P(_i64)])
_sig("tab_run", ctypes.c_int, [_vp, _vp])
_sig("tab_measure", ctypes.c_int, [_vp, _vp, _i32, _u64, _vp])
_sig("tab_measure_async", ctypes.c_int, [_vp, _vp, _i32, _vp])
_sig("tab_read_outcomes", ctypes.c_int, [_vp, _vp, _i64, _P(_i64)])
_sig("tab_expect", ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp])
_sig("tab_statevector", ctypes.c_int, [_vp, _vp, _i64])
_sig("tab_lower_ops", ctypes.c_int, [ctypes.c_int32, _vp, _i64, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_uint32, _P(ctypes.c_uint64), _vp, _i64, _P(_i64)])
_sig("tab_sharded_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P(_vp)])
_sig("tab_sharded_destroy", ctypes.c_int, [_vp])
_sig("tab_sharded_set_rng", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32])
_sig("tab_sharded_apply", ctypes.c_int, [_vp, _vp, _i64])
_sig("tab_sharded_read_outcomes", ctypes.c_int, [_vp, _vp, _i64, _P(_i64)])
_sig("tab_sharded_export", ctypes.c_int, [_vp, _vp, _vp, _vp])
_sig("tab_clear_outcomes", ctypes.c_int, [_vp])
_sig("tab_kernel_launches", ctypes.c_int, [_vp, _P(_i64)])
_sig("tab_count_work", ctypes.c_int, [_vp, _i32])
_sig("tab_work_counts", ctypes.c_int, [_vp, _P(_i64)])
_sig("tab_set_engine", ctypes.c_int, [_vp, ctypes.c_int])
_sig("tab_engine_resolved", ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_int)])
_sig("tab_transfer_bytes", ctypes.c_int, [_vp, _P(_i64), _P(_i64)])
_sig("tab_measure_noalloc", ctypes.c_int, [_vp, _vp, _i32, _i32, _vp])
_sig("tab_export", ctypes.c_int, [_vp, _vp, _vp, _vp])
_sig("tab_import", ctypes.c_int, [_vp, _vp, _vp, _vp, _u64])
_sig("tab_sync", ctypes.c_int, [_vp])
_sig("tab_batch_run", ctypes.c_int, [_vp, _i32, _u64, _vp, _vp])
_sig("tab_batch_run_packed", ctypes.c_int, [_vp, _i32, _u64, _vp, _i64, _vp])
_sig("tab_batch_create", ctypes.c_int, [_vp, _i32, _P(_vp)])
_sig("tab_batch_destroy", ctypes.c_int, [_vp])
_sig("tab_batch_info", ctypes.c_int, [_vp, _P(_i64), _P(_i64), _P(_i64)])
_sig("tab_batch_exec", ctypes.c_int, [_vp, _u64, _vp, _vp])
_sig("tab_batch_launches", ctypes.c_int, [_vp, _P(_i64)])
_sig("tab_batch_count_work", ctypes.c_int, [_vp, _i32])
_sig("tab_batch_work_counts", ctypes.c_int, [_vp, _P(_i64)])
_sig("tab_batch_tune", ctypes.c_int, [_vp, _u64, _vp, _vp, _P(_i32), _P(ctypes.c_float)])
_sig("tab_batch_config", ctypes.c_int, [_vp, _P(_i32), _P(_i32), _P(_i64)])
_sig("tab_batch_create_ex", ctypes.c_int, [_vp, _i32, _u32, _P(_vp)])
_sig("tab_batch_sampled", ctypes.c_int, [_vp, _P(_i32)])
_sig("tab_batch_h2d_bytes", ctypes.c_int, [_vp, _P(_i64)])


class TabServerConfig(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", _u64), ("max_inflight", _i32), ("n_streams", _i32),
                ("meas_ctas", _i32), ("request_timeout_s", ctypes.c_double), ("seed", _u64),
                ("max_grid_inflight", _i32)]


class TabServerStats(ctypes.Structure):
    _fields_ = [("submitted", _i64), ("completed", _i64), ("failed", _i64), ("rejected", _i64),
                ("inflight", _i64), ("queued", _i64), ("peak_inflight", _i64),
                ("mem_used", _u64), ("peak_mem", _u64)]


_sig("tab_server_create", ctypes.c_int, [_P(TabServerConfig), _P(_vp)])
_sig("tab_server_submit", ctypes.c_int, [_vp, _P(TabCircuit), _P(_i64)])
_sig("tab_server_query", ctypes.c_int, [_vp, _i64, _P(ctypes.c_int)])
_sig("tab_server_wait", ctypes.c_int, [_vp, _i64, ctypes.c_double, _vp, _i64, _P(_i64),
                                       _P(ctypes.c_double)])
_sig("tab_server_inject", ctypes.c_int, [_vp, _i64, ctypes.c_int])
_sig("tab_server_stats_get", ctypes.c_int, [_vp, _P(TabServerStats)])
_sig("tab_server_destroy", ctypes.c_int, [_vp])



class TabTuned(ctypes.Structure):
    _fields_ = [("engine", _i32), ("block_threads", _i32), ("meas_batch", _i32),
                ("from_cache", _i32), ("tried", _i32), ("best_ms", ctypes.c_float)]


_sig("tab_tune", ctypes.c_int, [_vp, _vp, _i32, _P(TabTuned)])


class TabConfig(ctypes.Structure):
    _fields_ = [("block_threads", _i32), ("meas_batch", _i32), ("grid_ctas", _i32),
                ("debug", _u32), ("wait_limit_ns", _u64), ("batch_chunks", _i32),
                ("reserved", _i32)]


_sig("tab_get_config", ctypes.c_int, [_P(TabConfig)])
_sig("tab_set_config", ctypes.c_int, [_P(TabConfig)])
DEBUG_SKIP_BARRIER_ARRIVAL = 1


def get_config() -> dict:
    """The process-wide run-time configuration (tab_get_config)."""
    c = TabConfig()
    _check(_L.tab_get_config(ctypes.byref(c)))
    return {k: getattr(c, k) for k, _ in TabConfig._fields_}


def set_config(cfg: dict):
    """Set the run-time configuration (tab_set_config); missing keys keep
    their current values."""
    cur = get_config()
    cur.update(cfg)
    c = TabConfig(*[cur[k] for k, _ in TabConfig._fields_])
    _check(_L.tab_set_config(ctypes.byref(c)))


class TabPeaks(ctypes.Structure):
    _fields_ = [("sms", _i32), ("sm_clock_mhz", ctypes.c_double),
                ("logic_tops", ctypes.c_double), ("logic_ops_per_clk_sm", ctypes.c_double),
                ("logic_ms", ctypes.c_double), ("smem_gbs", ctypes.c_double),
                ("smem_bytes_per_clk_sm", ctypes.c_double), ("l2_read_gbs", ctypes.c_double),
                ("l2_rw_gbs", ctypes.c_double), ("grid_barrier_us", ctypes.c_double)]


_sig("tab_measure_peaks", ctypes.c_int, [_P(TabPeaks)])


def measure_peaks() -> dict:
    """Roofline ceilings of the current device (tab_measure_peaks): logic
    ops/s, shared-memory and L2 bandwidth, grid-barrier latency."""
    p = TabPeaks()
    _check(_L.tab_measure_peaks(ctypes.byref(p)))
    return {k: getattr(p, k) for k, _ in TabPeaks._fields_}


_sig("tab_debug_build", ctypes.c_int, [])
_sig("tab_debug_check", ctypes.c_int, [_u32, _u32, _P(_u32)])


def debug_build() -> bool:
    """True in the debug build (libtab_debug.so, device-side index checks)."""
    return bool(_L.tab_debug_build())


def debug_check(index: int, limit: int) -> int:
    """Run the debug build's device index check once (tab_debug_check):
    returns the index the kernel went on with; raises TabError(TAB_EDEVICE)
    when the debug build finds it out of range."""
    out = _u32(0)
    _check(_L.tab_debug_check(index, limit, ctypes.byref(out)))
    return out.value


REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3
FAULT_DROP_COMPLETION = 1


class TabError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def last_error() -> str:
    m = _L.tab_last_error()
    return m.decode() if m else ""


def _check(rc: int):
    if rc != TAB_OK:
        raise TabError(rc, last_error())


def _u64arr(gates) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(gates, dtype=np.uint64).reshape(-1))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))  # torch.cuda.Stream


def bytes_required(n: int) -> int:
    return int(_L.tab_bytes_required(n))


class Program:
    """A gate list compiled once (validated, layered, uploaded); see tab_prog_create."""

    def __init__(self, n: int, gates):
        g = _u64arr(gates)
        h = _vp()
        _check(_L.tab_prog_create(n, g.ctypes.data if g.size else None, g.size, ctypes.byref(h)))
        self._h = h
        self.n = n

    def info(self):
        a, b, c = _i64(), _i64(), _i64()
        _check(_L.tab_prog_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"n_gates": a.value, "n_meas": b.value, "n_layers": c.value}

    def close(self):
        if getattr(self, "_h", None):
            _L.tab_prog_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Tableau:
    """A device-resident n-qubit tableau (tab_create / tab_create_on)."""

    def __init__(self, n: int, stream=None, memory=None):
        h = _vp()
        self._mem = memory
        if memory is not None:  # a torch CUDA tensor (uint8) the caller keeps alive
            ptr = int(memory.data_ptr())
            nbytes = int(memory.numel() * memory.element_size())
            _check(_L.tab_create_on(n, ptr, nbytes, _stream_handle(stream), ctypes.byref(h)))
        else:
            _check(_L.tab_create(n, ctypes.byref(h)))
            if stream is not None:
                _check(_L.tab_set_stream(h, _stream_handle(stream)))
        self._h = h
        self.n = n

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            _L.tab_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration
    def set_stream(self, stream):
        _check(_L.tab_set_stream(self._h, _stream_handle(stream)))

    def set_rng(self, seed: int = 1, circuit_id: int = 0, shot: int = 0):
        _check(_L.tab_set_rng(self._h, seed, circuit_id, shot))

    def reset(self):
        _check(_L.tab_reset(self._h))

    def set_engine(self, engine: int):
        """One of the ENGINE_* constants (bit-identical results)."""
        _check(_L.tab_set_engine(self._h, engine))

    def transfer_bytes(self):
        """(host->device, device->host) bytes this handle has copied for callers."""
        a, b = _i64(0), _i64(0)
        _check(_L.tab_transfer_bytes(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def engine_resolved(self):
        """(engine, ctas) that a run of measurements takes on this handle."""
        e, c = ctypes.c_int(0), ctypes.c_int(0)
        _check(_L.tab_engine_resolved(self._h, ctypes.byref(e), ctypes.byref(c)))
        return e.value, c.value

    # -- gates / measurements
    def apply(self, gates):
        g = _u64arr(gates)
        _check(_L.tab_apply(self._h, g.ctypes.data if g.size else None, g.size))

    def tune(self, prog: Program, reps: int = 3) -> dict:
        """Autotune this handle's launch shape on a compiled program
        (tab_tune); the tableau is left at |0^n>.  reps < 0 ignores the
        TAB_AUTOTUNE_CACHE file."""
        t = TabTuned()
        _check(_L.tab_tune(self._h, prog._h, int(reps), ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in TabTuned._fields_}

    def run(self, prog: Program):
        _check(_L.tab_run(self._h, prog._h))

    def measure(self, qubits: Sequence[int], seed: int = 1) -> np.ndarray:
        q = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32).reshape(-1))
        out = np.zeros(max(q.size, 1), np.uint8)
        _check(_L.tab_measure(self._h, q.ctypes.data if q.size else None, q.size, seed,
                              out.ctypes.data))
        return out[:q.size]

    def measure_async(self, qubits: Sequence[int], dev_out_ptr: int):
        q = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32).reshape(-1))
        _check(_L.tab_measure_async(self._h, q.ctypes.data if q.size else None, q.size,
                                    dev_out_ptr))

    def measure_noalloc(self, qubits: Sequence[int], dev_out_ptr: int, reset: bool = False):
        """tab_measure_noalloc: like measure_async, but the call allocates no
        device memory (its scratch is the library's fixed 1 MiB device array)."""
        q = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32).reshape(-1))
        _check(_L.tab_measure_noalloc(self._h, q.ctypes.data if q.size else None, q.size,
                                      1 if reset else 0, dev_out_ptr))

    def expect(self, paulis) -> np.ndarray:
        """<P> in {-1, 0, 1} for each row of `paulis` (k x n codes 0=I, 1=X,
        2=Z, 3=Y) or for each string over "IXYZ" in a list."""
        if isinstance(paulis, (list, tuple)) and paulis and isinstance(paulis[0], str):
            lut = {"I": 0, "X": 1, "Z": 2, "Y": 3}
            paulis = np.array([[lut[ch] for ch in s] for s in paulis], dtype=np.uint8)
        codes = np.ascontiguousarray(paulis, dtype=np.uint8).reshape(-1, self.n)
        out = np.zeros(max(codes.shape[0], 1), np.int8)
        _check(_L.tab_expect(self._h, codes.ctypes.data, codes.shape[0], out.ctypes.data))
        return out[:codes.shape[0]]

    def statevector(self) -> np.ndarray:
        """The 2^n amplitudes (complex64; basis index bit q = qubit q; the
        first nonzero amplitude real and positive), n <= 26."""
        out = np.zeros(2 << self.n, np.float32)
        _check(_L.tab_statevector(self._h, out.ctypes.data, out.size))
        return out.view(np.complex64)

    def read_outcomes(self) -> np.ndarray:
        cnt = _i64()
        _check(_L.tab_read_outcomes(self._h, None, 0, ctypes.byref(cnt)))
        out = np.zeros(max(cnt.value, 1), np.uint8)
        _check(_L.tab_read_outcomes(self._h, out.ctypes.data, cnt.value, ctypes.byref(cnt)))
        return out[:cnt.value]

    def clear_outcomes(self):
        _check(_L.tab_clear_outcomes(self._h))

    def sync(self):
        _check(_L.tab_sync(self._h))

    @property
    def launches(self) -> int:
        c = _i64()
        _check(_L.tab_kernel_launches(self._h, ctypes.byref(c)))
        return c.value

    def count_work(self, on: bool = True):
        """Start (zeroing them) or stop the streaming engine's work counters."""
        _check(_L.tab_count_work(self._h, 1 if on else 0))

    def work_counts(self) -> dict:
        """The work counters (tab_work_counts)."""
        c = (_i64 * 4)()
        _check(_L.tab_work_counts(self._h, c))
        return {"support_cols": c[0], "det_rows": c[1], "random": c[2], "deterministic": c[3]}

    # -- state transfer
    def export(self):
        n = self.n
        x = np.zeros((2 * n, n), np.uint8)
        z = np.zeros((2 * n, n), np.uint8)
        r = np.zeros(2 * n, np.uint8)
        _check(_L.tab_export(self._h, x.ctypes.data, z.ctypes.data, r.ctypes.data))
        return x, z, r

    def import_(self, x, z, r, meas_counter: int = 0):
        n = self.n
        x = np.ascontiguousarray(x, dtype=np.uint8).reshape(2 * n, n)
        z = np.ascontiguousarray(z, dtype=np.uint8).reshape(2 * n, n)
        r = np.ascontiguousarray(r, dtype=np.uint8).reshape(2 * n)
        _check(_L.tab_import(self._h, x.ctypes.data, z.ctypes.data, r.ctypes.data,
                             meas_counter))


class ShardedTableau:
    """A tableau split by rows over `shards` shards driven by host threads
    (tab_sharded_*): the same results as a Tableau."""

    def __init__(self, n: int, shards: int):
        self.n = n
        h = _vp()
        _check(_L.tab_sharded_create(n, shards, ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h:
            _L.tab_sharded_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_rng(self, seed: int = 1, circuit_id: int = 0, shot: int = 0):
        _check(_L.tab_sharded_set_rng(self._h, seed, circuit_id, shot))

    def apply(self, gates):
        g = _u64arr(gates)
        _check(_L.tab_sharded_apply(self._h, g.ctypes.data if g.size else None, g.size))

    def read_outcomes(self) -> np.ndarray:
        cnt = _i64()
        _check(_L.tab_sharded_read_outcomes(self._h, None, 0, ctypes.byref(cnt)))
        out = np.zeros(max(cnt.value, 1), np.uint8)
        _check(_L.tab_sharded_read_outcomes(self._h, out.ctypes.data, cnt.value, ctypes.byref(cnt)))
        return out[:cnt.value]

    def export(self):
        n = self.n
        x = np.zeros((2 * n, n), np.uint8)
        z = np.zeros((2 * n, n), np.uint8)
        r = np.zeros(2 * n, np.uint8)
        _check(_L.tab_sharded_export(self._h, x.ctypes.data, z.ctypes.data, r.ctypes.data))
        return x, z, r


def lower_ops(n: int, gates, seed: int = 1, circuit_id: int = 0, shot: int = 0,
              noise_counter: int = 0):
    """The base-op list tab_apply runs for `gates` (host only; no GPU needed)
    and the noise counter after it."""
    g = _u64arr(gates)
    cap = max(4 * g.size + 8, 16)
    out = np.zeros(cap, np.uint64)
    cnt = _i64()
    nk = ctypes.c_uint64(noise_counter)
    _check(_L.tab_lower_ops(n, g.ctypes.data if g.size else None, g.size, seed, circuit_id, shot,
                            ctypes.byref(nk), out.ctypes.data, cap, ctypes.byref(cnt)))
    return out[:cnt.value].copy(), nk.value


def _circuit_array(circuits):
    """circuits: iterable of (n, gates uint64 array, shots, circuit_id)."""
    keep = []
    arr = (TabCircuit * len(circuits))()
    for i, (n, gates, shots, cid) in enumerate(circuits):
        g = _u64arr(gates)
        keep.append(g)
        arr[i] = TabCircuit(n, g.ctypes.data if g.size else None, g.size, shots, cid)
    return arr, keep


def n_meas_of(gates) -> int:
    op = (_u64arr(gates) >> np.uint64(56))
    return int(np.isin(op, (10, 11, 13, 14)).sum())


_sig("tab_meas_counts", ctypes.c_int, [_vp, _i32, _P(_i64)])
_sig("tab_batch_meas_counts", ctypes.c_int, [_vp, _P(_i64)])


def _meas_counts(arr, m) -> list:
    counts = (_i64 * max(m, 1))()
    _check(_L.tab_meas_counts(ctypes.cast(arr, _vp), m, counts))
    return list(counts[:m])


def batch_run(circuits, seed: int = 1, out=None) -> list:
    """Run (n, gates, shots, circuit_id) circuits in one batched call.

    Returns, per circuit, a (shots, n_meas) uint8 array of outcomes (views of
    `out`, a host uint8 array of at least the total outcome count, if given,
    e.g. in pinned memory)."""
    arr, keep = _circuit_array(circuits)
    if out is None:
        nms = _meas_counts(arr, len(circuits))
        total = int(sum(shots * nm for (_, _, shots, _), nm in zip(circuits, nms)))
        out = np.zeros(max(total, 1), np.uint8)
        _check(_L.tab_batch_run(ctypes.cast(arr, _vp), len(circuits), seed, out.ctypes.data,
                                None))
    else:
        # the library bounds the writes by out.size and returns the counts
        if out.dtype != np.uint8 or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous uint8 array")
        nms = np.zeros(max(len(circuits), 1), np.int64)
        code = _L.tab_batch_run_packed(ctypes.cast(arr, _vp), len(circuits), seed,
                                       out.ctypes.data, out.size, nms.ctypes.data)
        if code == TAB_ERANGE:
            raise ValueError("out is smaller than the total outcome count: "
                             + last_error())
        _check(code)
        nms = [int(v) for v in nms[:len(circuits)]]
    sizes = [shots * nm for (_, _, shots, _), nm in zip(circuits, nms)]
    res, off = [], 0
    for (n, g, shots, _), sz in zip(circuits, sizes):
        res.append(out[off:off + sz].reshape(shots, -1) if sz else
                   np.zeros((shots, 0), np.uint8))
        off += sz
    return res


BATCH_SAMPLE_TERMINAL = 1


class TabBatchClass(ctypes.Structure):
    _fields_ = [("lo_n", _i32), ("max_n", _i32), ("threads", _i32), ("ctas", _i32),
                ("smem_bytes", _i64), ("items", _i64)]


_sig("tab_batch_classes", ctypes.c_int, [_vp, _P(_i32)])
_sig("tab_batch_class", ctypes.c_int, [_vp, _i32, _P(TabBatchClass)])


class Batch:
    """A compiled batch (tab_batch_create_ex) replayed with exec().
    sample_terminal: circuits whose measurements all follow their gates run
    the terminal measurements once and sample every shot from the outcome
    forms (same outcome bits)."""

    def __init__(self, circuits, sample_terminal: bool = False):
        arr, keep = _circuit_array(circuits)
        h = _vp()
        flags = BATCH_SAMPLE_TERMINAL if sample_terminal else 0
        _check(_L.tab_batch_create_ex(ctypes.cast(arr, _vp), len(circuits), flags,
                                      ctypes.byref(h)))
        self._h = h
        counts = (_i64 * max(len(circuits), 1))()
        _check(_L.tab_batch_meas_counts(h, counts))
        self.sizes = [shots * counts[i] for i, (_, _, shots, _) in enumerate(circuits)]

    def info(self):
        a, b, c = _i64(), _i64(), _i64()
        _check(_L.tab_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"n_gates": a.value, "n_meas": b.value, "out_bytes": c.value}

    def exec(self, seed: int, dev_out_ptr: int, stream=None):
        _check(_L.tab_batch_exec(self._h, seed, dev_out_ptr, _stream_handle(stream)))

    def tune(self, seed: int, dev_out_ptr: int, stream=None):
        """Autotune the launch's CTA shape on this batch (tab_batch_tune);
        returns (threads per CTA, time of the best run in ms)."""
        t, ms = _i32(), ctypes.c_float()
        _check(_L.tab_batch_tune(self._h, seed, dev_out_ptr, _stream_handle(stream),
                                 ctypes.byref(t), ctypes.byref(ms)))
        return t.value, ms.value

    @property
    def sampled(self) -> int:
        """Circuits that run through the terminal-measurement sampler."""
        c = _i32()
        _check(_L.tab_batch_sampled(self._h, ctypes.byref(c)))
        return c.value

    def classes(self) -> list:
        """Size classes (tab_batch_class): per class its qubit range, launch
        shape and work items, largest qubit counts first."""
        cnt = _i32()
        _check(_L.tab_batch_classes(self._h, ctypes.byref(cnt)))
        out = []
        for k in range(cnt.value):
            ci = TabBatchClass()
            _check(_L.tab_batch_class(self._h, k, ctypes.byref(ci)))
            out.append({f: getattr(ci, f) for f, _ in TabBatchClass._fields_})
        return out

    def config(self):
        """Launch shape of the first (largest-qubit) size class:
        {"threads", "ctas", "smem_bytes"}."""
        t, c, s = _i32(), _i32(), _i64()
        _check(_L.tab_batch_config(self._h, ctypes.byref(t), ctypes.byref(c), ctypes.byref(s)))
        return {"threads": t.value, "ctas": c.value, "smem_bytes": s.value}

    @property
    def launches(self) -> int:
        c = _i64()
        _check(_L.tab_batch_launches(self._h, ctypes.byref(c)))
        return c.value

    def count_work(self, on: bool = True):
        """Start (zeroing them) or stop the batched kernel's work counters."""
        _check(_L.tab_batch_count_work(self._h, 1 if on else 0))

    def work_counts(self) -> dict:
        """The work counters (tab_batch_work_counts), once the counted runs
        have finished."""
        c = (_i64 * 4)()
        _check(_L.tab_batch_work_counts(self._h, c))
        return {"support_words": c[0], "det_row_words": c[1], "random": c[2],
                "deterministic": c[3]}

    @property
    def h2d_bytes(self) -> int:
        """Compiled-table bytes copied to the device at creation."""
        c = _i64()
        _check(_L.tab_batch_h2d_bytes(self._h, ctypes.byref(c)))
        return c.value

    def close(self):
        if getattr(self, "_h", None):
            _L.tab_batch_destroy(self._h)
            self._h = None

    __del__ = close


class Server:
    """Continuous-batching request server (tab_server_*): submit circuits,
    wait for their outcomes and latencies."""

    def __init__(self, mem_budget_bytes: int = 150 << 30, max_inflight: int = 16,
                 n_streams: int = 8, meas_ctas: int = 0, request_timeout_s: float = 0.0,
                 seed: int = 1, max_grid_inflight: int = 1):
        cfg = TabServerConfig(mem_budget_bytes, max_inflight, n_streams, meas_ctas,
                              request_timeout_s, seed, max_grid_inflight)
        h = _vp()
        _check(_L.tab_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}
        self._nmeas = {}

    def submit(self, n: int, gates, shots: int = 1, circuit_id: int = 0) -> int:
        g = _u64arr(gates)
        c = TabCircuit(n, g.ctypes.data if g.size else None, g.size, shots, circuit_id)
        t = _i64()
        _check(_L.tab_server_submit(self._h, ctypes.byref(c), ctypes.byref(t)))
        self._nmeas[t.value] = shots * n_meas_of(g)
        return t.value

    def query(self, ticket: int) -> int:
        st = ctypes.c_int()
        _check(_L.tab_server_query(self._h, ticket, ctypes.byref(st)))
        return st.value

    def wait(self, ticket: int, timeout_s: float = -1.0):
        """Returns (status, outcomes uint8 array, latency seconds)."""
        cap = self._nmeas.get(ticket, 0)
        out = np.zeros(max(cap, 1), np.uint8)
        cnt, lat = _i64(), ctypes.c_double()
        rc = _L.tab_server_wait(self._h, ticket, timeout_s, out.ctypes.data, cap,
                                ctypes.byref(cnt), ctypes.byref(lat))
        if rc == TAB_ESTATE:
            raise TabError(rc, last_error())
        self._nmeas.pop(ticket, None)
        return rc, out[:min(cnt.value, cap)], lat.value

    def inject(self, ticket: int, kind: int = FAULT_DROP_COMPLETION):
        _check(_L.tab_server_inject(self._h, ticket, kind))

    def stats(self) -> dict:
        st = TabServerStats()
        _check(_L.tab_server_stats_get(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in TabServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _L.tab_server_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
