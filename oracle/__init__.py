"""CPU oracle for the stabilizer-tableau path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  It wraps ``chp_oracle.c`` -- an
unpacked, one-byte-per-bit restatement of Aaronson & Gottesman's tableau
algorithm (PRA 70, 052328, 2004, Sec. III), the formalism the paper's Clifford
backend is built on (arXiv:2408.00384, section "Simulation of Clifford
circuits") -- through ctypes.  It shares no code with the CUDA library.

Parity pins (tests/test_oracle_*.py): gate rules and AG's g against explicit
Pauli matrices; whole runs against brute-force state vectors (n <= 10); known
states (Bell, GHZ, product states); the symplectic invariant; circuit-inverse
identity; Philox4x32-10 against the Random123 known-answer vectors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

ORC_OK, ORC_EINVAL, ORC_ERANGE, ORC_ENOMEM, ORC_EPHASE = 0, -1, -2, -3, -8


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i32, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_uint32, ctypes.c_uint64)
        P = ctypes.POINTER
        L.orc_new.restype = vp
        L.orc_new.argtypes = [i32]
        L.orc_free.argtypes = [vp]
        L.orc_reset.argtypes = [vp]
        for name in ("orc_h", "orc_s", "orc_x", "orc_y", "orc_z", "orc_sdg"):
            getattr(L, name).argtypes = [vp, i32]
        for name in ("orc_cnot", "orc_cz", "orc_swap"):
            getattr(L, name).argtypes = [vp, i32, i32]
        L.orc_g.restype = i32
        L.orc_g.argtypes = [i32, i32, i32, i32]
        L.orc_rowsum.restype = i32
        L.orc_rowsum.argtypes = [vp, i64, i64]
        L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        L.orc_outcome_bit.restype = i32
        L.orc_outcome_bit.argtypes = [u64, u64, u32, u64]
        L.orc_measure.restype = i32
        L.orc_measure.argtypes = [vp, i32, i32, P(i32)]
        L.orc_run.restype = i64
        L.orc_run.argtypes = [vp, P(u64), i64, u64, u64, u32, P(u64),
                              P(ctypes.c_uint8), i64, P(ctypes.c_uint8)]
        L.orc_get.argtypes = [vp, vp, vp, vp]
        L.orc_expect.restype = i32
        L.orc_expect.argtypes = [vp, vp]
        L.orc_set.argtypes = [vp, vp, vp, vp]
        L.orc_set_threads.restype = i32
        L.orc_set_threads.argtypes = [vp, i32]
        L.orc_threads.restype = i32
        L.orc_threads.argtypes = [vp]
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def outcome_bit(seed: int, circuit_id: int, shot: int, k: int) -> int:
    return int(lib().orc_outcome_bit(seed, circuit_id, shot, k))


def g(x1, z1, x2, z2) -> int:
    return int(lib().orc_g(x1, z1, x2, z2))


def all_cores() -> int:
    """Cores this process may run on (its affinity mask)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


class Tableau:
    """Unpacked AG tableau: rows 0..n-1 destabilizers, n..2n-1 stabilizers.

    ``threads`` > 1 splits each gate's loop over rows, and the target rows of a
    random-outcome measurement's rowsums, into contiguous shares on that many
    threads (results are identical to one thread)."""

    def __init__(self, n: int, threads: int = 1):
        self.n = int(n)
        self._h = lib().orc_new(self.n)
        if not self._h:
            raise MemoryError("orc_new failed")
        self.meas_counter = 0
        if threads != 1:
            self.set_threads(threads)

    def set_threads(self, threads: int):
        rc = lib().orc_set_threads(self._h, int(threads))
        if rc != ORC_OK:
            raise RuntimeError(f"orc_set_threads error {rc}")

    @property
    def threads(self) -> int:
        return int(lib().orc_threads(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    def reset(self):
        lib().orc_reset(self._h)
        self.meas_counter = 0

    # gates
    def h(self, a): lib().orc_h(self._h, a)
    def s(self, a): lib().orc_s(self._h, a)
    def x(self, a): lib().orc_x(self._h, a)
    def y(self, a): lib().orc_y(self._h, a)
    def z(self, a): lib().orc_z(self._h, a)
    def sdg(self, a): lib().orc_sdg(self._h, a)
    def cnot(self, a, b): lib().orc_cnot(self._h, a, b)
    def cz(self, a, b): lib().orc_cz(self._h, a, b)
    def swap(self, a, b): lib().orc_swap(self._h, a, b)

    def rowsum(self, h, i) -> int:
        return int(lib().orc_rowsum(self._h, h, i))

    def measure(self, a: int, rbit: int):
        """Measure Z_a with pre-drawn bit rbit; returns (outcome, deterministic)."""
        d = ctypes.c_int32(0)
        m = lib().orc_measure(self._h, a, rbit, ctypes.byref(d))
        if m < 0:
            raise RuntimeError(f"orc_measure error {m}")
        return int(m), bool(d.value)

    def run(self, gates, seed: int = 1, circuit_id: int = 0, shot: int = 0,
            with_det: bool = False):
        """Run a gate-word list; returns outcome bytes (and deterministic flags)."""
        gates = np.ascontiguousarray(gates, dtype=np.uint64)
        op = (gates >> np.uint64(56)).astype(np.int64)
        cap = int(np.isin(op, (10, 11, 13, 14)).sum())
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        det = np.zeros(max(cap, 1), dtype=np.uint8)
        ctr = ctypes.c_uint64(self.meas_counter)
        rc = lib().orc_run(self._h, _ptr(gates, ctypes.c_uint64), gates.size, seed,
                           circuit_id, shot, ctypes.byref(ctr),
                           _ptr(out, ctypes.c_uint8), cap, _ptr(det, ctypes.c_uint8))
        if rc < 0:
            raise RuntimeError(f"orc_run error {rc}")
        self.meas_counter = ctr.value
        if with_det:
            return out[:rc].copy(), det[:rc].astype(bool)
        return out[:rc].copy()

    def expect(self, codes) -> int:
        """<P> in {-1, 0, 1} for one Pauli string (n codes: 0 I, 1 X, 2 Z, 3 Y)."""
        c = np.ascontiguousarray(codes, dtype=np.uint8).reshape(self.n)
        v = int(lib().orc_expect(self._h, c.ctypes.data))
        if v < -1:
            raise RuntimeError(f"orc_expect error {v}")
        return v

    def get(self):
        """(x, z, r) as uint8 arrays of shape (2n, n), (2n, n), (2n,)."""
        n = self.n
        x = np.zeros((2 * n, n), np.uint8)
        z = np.zeros((2 * n, n), np.uint8)
        r = np.zeros(2 * n, np.uint8)
        lib().orc_get(self._h, x.ctypes.data, z.ctypes.data, r.ctypes.data)
        return x, z, r

    def set(self, x, z, r):
        n = self.n
        x = np.ascontiguousarray(x, dtype=np.uint8).reshape(2 * n, n)
        z = np.ascontiguousarray(z, dtype=np.uint8).reshape(2 * n, n)
        r = np.ascontiguousarray(r, dtype=np.uint8).reshape(2 * n)
        lib().orc_set(self._h, x.ctypes.data, z.ctypes.data, r.ctypes.data)


def run_circuit(n: int, gates, seed: int = 1, circuit_id: int = 0, shot: int = 0,
                threads: int = 1):
    """Fresh |0^n>, run gates; returns (outcomes, (x, z, r))."""
    t = Tableau(n, threads=threads)
    out = t.run(gates, seed=seed, circuit_id=circuit_id, shot=shot)
    return out, t.get()
