"""Digests of simulation results, for comparing a run with stored oracle
results without storing whole tableaus.

Only hashing and bit packing live here: no tableau arithmetic.  A tableau is
digested in the layout both sides export (x and z as (2n, n) row-major bytes,
r as 2n bytes), bit-packed with numpy's big-endian packbits.
"""
import hashlib
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def path(family: str) -> str:
    return os.path.join(HERE, f"oracle_{family}.json")


def gates_sha(gates) -> str:
    g = np.ascontiguousarray(gates, dtype=np.uint64)
    return hashlib.sha256(g.astype("<u8").tobytes()).hexdigest()


def outcomes_sha(outcomes) -> str:
    o = np.ascontiguousarray(outcomes, dtype=np.uint8)
    return hashlib.sha256(o.tobytes()).hexdigest()


def pack_outcomes(outcomes) -> str:
    return np.packbits(np.asarray(outcomes, dtype=np.uint8)).tobytes().hex()


def unpack_outcomes(hexstr: str, count: int) -> np.ndarray:
    b = np.frombuffer(bytes.fromhex(hexstr), dtype=np.uint8)
    return np.unpackbits(b)[:count]


def tableau_sha(x, z, r) -> str:
    h = hashlib.sha256()
    for a in (x, z, r):
        h.update(np.packbits(np.asarray(a, dtype=np.uint8).reshape(-1)).tobytes())
    return h.hexdigest()


def load(family: str) -> dict:
    with open(path(family)) as f:
        return json.load(f)


def first_difference(got, want):
    """Index of the first differing outcome (or the shorter length), or None."""
    got = np.asarray(got, dtype=np.uint8)
    want = np.asarray(want, dtype=np.uint8)
    m = min(got.size, want.size)
    bad = np.flatnonzero(got[:m] != want[:m])
    if bad.size:
        return int(bad[0])
    return None if got.size == want.size else m
