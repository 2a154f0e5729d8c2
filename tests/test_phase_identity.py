"""The per-column rowsum exponent the GPU kernels accumulate,
    c(p, h) = x_p z_p + x_h z_h - x'_h z'_h + 2 z_p x_h   (x' = x_h ^ x_p, z' = z_h ^ z_p),
equals AG's g(x_p, z_p, x_h, z_h) mod 4 in all 16 cases; and the bit-sliced
mod-4 counter updates used for it (inc/dec planes) add exactly c - 2 z_p x_h.
Pinned against the oracle's g and against 2x2 Pauli matrix products."""
import itertools

import numpy as np

import oracle
from tests.statevector import pauli_1q


def per_column_exponent(xp, zp, xh, zh):
    xn, zn = xh ^ xp, zh ^ zp
    return xp * zp + xh * zh - xn * zn + 2 * zp * xh


def test_exponent_identity_all_cases():
    for xp, zp, xh, zh in itertools.product((0, 1), repeat=4):
        c = per_column_exponent(xp, zp, xh, zh) % 4
        assert c == oracle.g(xp, zp, xh, zh) % 4, (xp, zp, xh, zh)
        # and against the matrices: P(p) P(h) = i^c P(p ^ h)
        prod = pauli_1q(xp, zp) @ pauli_1q(xh, zh)
        assert np.allclose(prod, (1j ** c) * pauli_1q(xp ^ xh, zp ^ zh))


def test_bitsliced_counter_update():
    """Word-parallel form: inc = A & ~B, dec = B & ~A with A = x&z, B = x'&z'
    adds (A - B) to a 2-bit counter per bit lane; hi also toggles on z_p & x_h."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        x = int(rng.integers(0, 2**32))
        z = int(rng.integers(0, 2**32))
        xp, zp = int(rng.integers(0, 2)), int(rng.integers(0, 2))
        XP, ZP = (0xFFFFFFFF if xp else 0), (0xFFFFFFFF if zp else 0)
        lo0 = int(rng.integers(0, 2**32))
        hi0 = int(rng.integers(0, 2**32))
        A = x & z
        B = (x ^ XP) & (z ^ ZP)
        inc, dec = A & ~B & 0xFFFFFFFF, B & ~A & 0xFFFFFFFF
        hi = hi0 ^ (((lo0 & inc) | (~lo0 & dec)) ^ (ZP & x)) & 0xFFFFFFFF
        lo = lo0 ^ (inc | dec)
        for b in range(32):
            xh, zh = (x >> b) & 1, (z >> b) & 1
            before = ((hi0 >> b) & 1) * 2 + ((lo0 >> b) & 1)
            after = ((hi >> b) & 1) * 2 + ((lo >> b) & 1)
            want = (before + per_column_exponent(xp, zp, xh, zh) - xp * zp) % 4
            assert after == want
