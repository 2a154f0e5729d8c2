"""Seeded random Clifford circuits in the library's 64-bit gate-list format.

Gate word (little-endian uint64):  bits 63..56 = op code, 55..28 = first qubit,
27..0 = second qubit (zero for one-qubit ops).  Op codes are the interface
values of the C-ABI (``include/tab.h``) and of the oracle's decoder; they are a
data format, not part of either side's arithmetic.

The workloads stand in for the paper's benchmark data set (uniformly random
Cliffords, Section "Simulation of Clifford circuits", Fig. 2a), which is not
available here.  Each random layer is:

* one single-qubit gate on every qubit, H or S with probability 1/2 each;
* a seeded random permutation pi of the qubits, paired as (pi[2k], pi[2k+1])
  for k < n//2 with the first element as control; each pair is CNOT, or
  (mixed mode) CNOT with probability 3/4 and CZ with probability 1/4.

A ``TAB_BARRIER`` word separates the single-qubit and two-qubit sub-layers.
Barriers are hints only: they never change results.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# ---- op codes (interface values) -------------------------------------------
TAB_I, TAB_X, TAB_Y, TAB_Z, TAB_H, TAB_S, TAB_SDG = 0, 1, 2, 3, 4, 5, 6
TAB_CNOT, TAB_CZ, TAB_SWAP = 7, 8, 9
TAB_MZ, TAB_MZR, TAB_BARRIER = 10, 11, 12
# extended ops: X / Y measurement and single-qubit Pauli noise (the second
# qubit field of a noise op holds its probability as a 28-bit fraction)
TAB_MX, TAB_MY, TAB_DEPOL1, TAB_XERR, TAB_ZERR = 13, 14, 15, 16, 17

ONE_QUBIT = (TAB_I, TAB_X, TAB_Y, TAB_Z, TAB_H, TAB_S, TAB_SDG)
TWO_QUBIT = (TAB_CNOT, TAB_CZ, TAB_SWAP)
MEASURE = (TAB_MZ, TAB_MZR)
MEASURE_ANY = (TAB_MZ, TAB_MZR, TAB_MX, TAB_MY)   # ops that log an outcome
NOISE = (TAB_DEPOL1, TAB_XERR, TAB_ZERR)

OP_NAMES = {TAB_I: "I", TAB_X: "X", TAB_Y: "Y", TAB_Z: "Z", TAB_H: "H",
            TAB_S: "S", TAB_SDG: "SDG", TAB_CNOT: "CNOT", TAB_CZ: "CZ",
            TAB_SWAP: "SWAP", TAB_MZ: "MZ", TAB_MZR: "MZR",
            TAB_BARRIER: "BARRIER", TAB_MX: "MX", TAB_MY: "MY",
            TAB_DEPOL1: "DEPOL1", TAB_XERR: "XERR", TAB_ZERR: "ZERR"}

CONFIG_SEED = 240800384   # fixed generator seed of every workload family
PHILOX_SEED = 1           # fixed outcome seed of every workload family

_MASK28 = (1 << 28) - 1


def encode(op, q1=0, q2=0) -> np.ndarray:
    """Pack op codes and qubit indices (scalars or arrays) into gate words."""
    op = np.asarray(op, dtype=np.uint64)
    q1 = np.asarray(q1, dtype=np.uint64)
    q2 = np.asarray(q2, dtype=np.uint64)
    return (op << np.uint64(56)) | ((q1 & np.uint64(_MASK28)) << np.uint64(28)) \
        | (q2 & np.uint64(_MASK28))


def decode(gates: np.ndarray):
    """Split gate words into (op, q1, q2) int64 arrays."""
    g = np.asarray(gates, dtype=np.uint64)
    op = (g >> np.uint64(56)).astype(np.int64)
    q1 = ((g >> np.uint64(28)) & np.uint64(_MASK28)).astype(np.int64)
    q2 = (g & np.uint64(_MASK28)).astype(np.int64)
    return op, q1, q2


def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014)."""
    m = (1 << 64) - 1
    x = (x + 0x9E3779B97F4A7C15) & m
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & m
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & m
    return x ^ (x >> 31)


def circuit_seed(config_index: int, c: int) -> int:
    """Generator seed of circuit ``c`` of a workload family."""
    return splitmix64((CONFIG_SEED + 7919 * config_index) ^ c)


@dataclasses.dataclass
class Circuit:
    """One synthetic circuit: its gate words and what they contain."""
    n: int
    gates: np.ndarray          # uint64 gate words, program order
    n_gates: int               # Clifford gate ops (barriers and measurements excluded)
    n_meas: int                # measurement ops per shot
    shots: int = 1
    circuit_id: int = 0
    depth: int = 0

    @property
    def n_words(self) -> int:
        return int(self.gates.size)


def random_layer_circuit(n: int, depth: int, seed: int, *, mix_cz: bool = True,
                         meas_every: int = 0, meas_frac: float = 0.0,
                         reset: bool = True, final_measure: bool = True,
                         barriers: bool = True, circuit_id: int = 0,
                         shots: int = 1) -> Circuit:
    """Random-layer Clifford circuit (module docstring gives the layer).

    ``meas_every``/``meas_frac``: after every ``meas_every``-th layer measure
    floor(meas_frac * n) distinct uniformly drawn qubits, in ascending order,
    with reset (``TAB_MZR``) when ``reset`` is true.  ``final_measure`` appends
    ``TAB_MZ`` on every qubit in ascending order.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    one_q = np.where(rng.integers(0, 2, size=(depth, n)) == 0, TAB_H, TAB_S)
    perms = np.argsort(rng.random((depth, n)), axis=1, kind="stable")
    npairs = n // 2
    if mix_cz:
        two_q = np.where(rng.random((depth, npairs)) < 0.75, TAB_CNOT, TAB_CZ)
    else:
        two_q = np.full((depth, npairs), TAB_CNOT)
    n_rounds = depth // meas_every if meas_every else 0
    k_round = int(math.floor(meas_frac * n)) if meas_every else 0
    rounds = []
    for _ in range(n_rounds):
        rounds.append(np.sort(rng.choice(n, size=k_round, replace=False)))

    qubits = np.arange(n, dtype=np.int64)
    # one row of gate words per layer: [1q gates | bar | 2q gates | bar]
    nb = 1 if barriers else 0
    width = n + nb + npairs + (nb if npairs else 0)
    blk = np.empty((depth, width), dtype=np.uint64)
    blk[:, :n] = encode(one_q, qubits[None, :], 0)
    col = n
    if barriers:
        blk[:, col] = encode(TAB_BARRIER)
        col += 1
    if npairs:
        blk[:, col:col + npairs] = encode(two_q, perms[:, 0:2 * npairs:2],
                                          perms[:, 1:2 * npairs:2])
        col += npairs
        if barriers:
            blk[:, col] = encode(TAB_BARRIER)
    parts: List[np.ndarray] = []
    n_meas = 0
    mop = TAB_MZR if reset else TAB_MZ
    if meas_every and k_round:
        start = 0
        for r in range(n_rounds):
            stop = (r + 1) * meas_every
            parts.append(blk[start:stop].reshape(-1))
            qs = rounds[r]
            parts.append(encode(np.full(qs.size, mop), qs, 0))
            n_meas += int(qs.size)
            start = stop
        parts.append(blk[start:].reshape(-1))
    else:
        parts.append(blk.reshape(-1))
    if final_measure:
        parts.append(encode(np.full(n, TAB_MZ), qubits, 0))
        n_meas += n
    gates = np.concatenate(parts) if parts else np.zeros(0, np.uint64)
    return Circuit(n=n, gates=gates, n_gates=depth * (n + npairs),
                   n_meas=n_meas, shots=shots, circuit_id=circuit_id,
                   depth=depth)


# ---- the five workload families ---------------------------------------------

def config1(seed_index: int = 0) -> Circuit:
    """n=10, 20 layers (H/S per qubit, 5 CNOT pairs), final MZ on all 10."""
    return random_layer_circuit(10, 20, circuit_seed(1, seed_index), mix_cz=False)


def config2(seed_index: int = 0, depth: int = 1000, n: int = 1000) -> Circuit:
    """n=1000, 1000 layers (CNOT:CZ = 3:1), final MZ on all qubits."""
    return random_layer_circuit(n, depth, circuit_seed(2, seed_index))


def config3(seed_index: int = 0, n: int = 10000, depth: int = 100) -> Circuit:
    """n=10,000, 100 layers, MZR on floor(n/10) random qubits every 10 layers."""
    return random_layer_circuit(n, depth, circuit_seed(3, seed_index),
                                meas_every=10, meas_frac=0.10, reset=True,
                                final_measure=False)


def config4_shapes(m: int = 4096, n_lo: int = 16, n_hi: int = 512,
                   shots_hi: int = 64):
    """(n, shots) of the batched family: n ~ U{n_lo..n_hi}, shots ~ U{1..shots_hi}."""
    rng = np.random.Generator(np.random.PCG64(circuit_seed(4, 1 << 40)))
    ns = rng.integers(n_lo, n_hi + 1, size=m)
    shots = rng.integers(1, shots_hi + 1, size=m)
    return ns.astype(np.int64), shots.astype(np.int64)


def config4(m: int = 4096, n_lo: int = 16, n_hi: int = 512, shots_hi: int = 64,
            only: Optional[List[int]] = None) -> List[Circuit]:
    """Batched family: m circuits, depth n, final MZ on all qubits, 1..64 shots."""
    ns, shots = config4_shapes(m, n_lo, n_hi, shots_hi)
    idx = range(m) if only is None else only
    return [random_layer_circuit(int(ns[c]), int(ns[c]), circuit_seed(4, c),
                                 circuit_id=c, shots=int(shots[c]))
            for c in idx]


def config5_request(c: int, n_lo: int = 50, n_hi: int = 5000) -> Circuit:
    """Served family request c: n log-uniform in [n_lo, n_hi], depth 2n,
    MZR on floor(n/20) qubits every 20 layers, then final MZ on all qubits."""
    rng = np.random.Generator(np.random.PCG64(circuit_seed(5, 1 << 40 | c)))
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    return random_layer_circuit(n, 2 * n, circuit_seed(5, c), meas_every=20,
                                meas_frac=0.05, reset=True, final_measure=True,
                                circuit_id=c)


def poisson_arrivals(rate_hz: float, count: int, seed: int = CONFIG_SEED):
    """Arrival times (seconds from 0) of a Poisson stream with the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))


def random_clifford_ops(n: int, count: int, seed: int, *, measure_p: float = 0.0,
                        reset_p: float = 0.0, ops=None) -> np.ndarray:
    """Unstructured random gate list over every op (edge-case tests).

    Each entry is a uniformly drawn op from ``ops`` on uniformly drawn distinct
    qubits; with probability ``measure_p`` an MZ and ``reset_p`` an MZR.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if ops is None:
        ops = list(ONE_QUBIT) + (list(TWO_QUBIT) if n >= 2 else [])
    out = np.zeros(count, dtype=np.uint64)
    for i in range(count):
        u = rng.random()
        if u < measure_p:
            out[i] = encode(TAB_MZ, int(rng.integers(0, n)), 0)
            continue
        if u < measure_p + reset_p:
            out[i] = encode(TAB_MZR, int(rng.integers(0, n)), 0)
            continue
        op = int(ops[int(rng.integers(0, len(ops)))])
        if op in TWO_QUBIT:
            a, b = rng.choice(n, size=2, replace=False)
            out[i] = encode(op, int(a), int(b))
        else:
            out[i] = encode(op, int(rng.integers(0, n)), 0)
    return out


def noise_field(p: float) -> int:
    """The 28-bit probability field of a noise op for probability p in [0, 1)."""
    if not 0.0 <= p < 1.0:
        raise ValueError("p must be in [0, 1)")
    return int(p * (1 << 28))


def random_extended_ops(n: int, count: int, seed: int, *, p_meas: float = 0.1,
                        p_noise: float = 0.1, noise_p: float = 0.3) -> np.ndarray:
    """Random gate list over every op, extended ones included: MZ / MZR / MX /
    MY with total probability p_meas, a noise op (DEPOL1, XERR or ZERR with
    probability noise_p) with probability p_noise, else a uniform gate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gates = list(ONE_QUBIT) + (list(TWO_QUBIT) if n >= 2 else [])
    field = noise_field(noise_p)
    out = np.zeros(count, dtype=np.uint64)
    for i in range(count):
        u = rng.random()
        if u < p_meas:
            out[i] = encode(int(rng.choice(MEASURE_ANY)), int(rng.integers(0, n)), 0)
        elif u < p_meas + p_noise:
            out[i] = encode(int(rng.choice(NOISE)), int(rng.integers(0, n)), field)
        else:
            op = int(gates[int(rng.integers(0, len(gates)))])
            if op in TWO_QUBIT:
                a, b = rng.choice(n, size=2, replace=False)
                out[i] = encode(op, int(a), int(b))
            else:
                out[i] = encode(op, int(rng.integers(0, n)), 0)
    return out


def count_ops(gates: np.ndarray):
    """(gate ops, measurement ops) in a gate list; barriers and noise ops are
    not counted."""
    op, _, _ = decode(gates)
    meas = int(np.isin(op, MEASURE_ANY).sum())
    gates_n = int(np.isin(op, ONE_QUBIT + TWO_QUBIT).sum())
    return gates_n, meas


# ---- uniformly random Cliffords (the paper's own benchmark family) ---------
#
# The paper times uniformly random n-qubit Clifford circuits drawn with the
# method of Bravyi and Maslov (Section "Simulation of Clifford circuits",
# Fig. 2a).  Their canonical form writes a Clifford as F1 . (Hadamards,
# permutation) . F2 with Hadamard-free F1, F2; it is the Bruhat decomposition
# of the symplectic group Sp(2n, 2) with respect to the Borel subgroup B of
# Hadamard-free Cliffords that keep the flag <Z_1> < <Z_1, Z_2> < ... .  The
# sampler below draws from that decomposition directly:
#
#   C = P . b1 . w . b2        (b2 applied first)
#
# * b1, b2 uniform in B (mod Paulis).  B is the product of the group of CNOT
#   circuits whose map on computational basis states is unit lower triangular
#   (CNOT c -> t with c < t) and the abelian group of diagonal CZ / S layers
#   (a symmetric GF(2) matrix Gamma: CZ(i, j) where Gamma_ij = 1, S(i) where
#   Gamma_ii = 1); |B| = 2^(n(n-1)/2) 2^(n(n+1)/2) = 2^(n^2).
# * w a Weyl group element (a signed permutation: Hadamards on a subset, then
#   a qubit permutation) drawn with probability 2^len(w) / prod_j (4^j - 1),
#   len the Coxeter length.  The double coset B w B holds |B| 2^len(w)
#   elements and every element of it is b1 w b2 for exactly |B| / 2^len(w)
#   pairs (b1, b2), so C mod Paulis is uniform on Sp(2n, 2).
# * P a uniform Pauli layer, which makes the signs uniform.
#
# The Weyl group is the hyperoctahedral group B_n with generators s_0 (sign
# change of the first letter) and s_i (exchange of letters i, i+1); its
# length is inv(w) + #{i <= j : w(i) + w(j) < 0} (Bjorner & Brenti,
# Combinatorics of Coxeter Groups, Sec. 8.1).  Letter k of a signed
# permutation stands for qubit n - k (0-based), sign + for X and - for Z:
# s_0 is H on qubit n - 1 and s_i is SWAP(n - i, n - i - 1), the Weyl elements
# of length one for the flag above.  A signed permutation is built by
# inserting the letters 1, 2, ..., n: +m inserted with c smaller letters after
# it adds c to the length (c in [0, m)), -m inserted with c - m letters
# before it adds c (c in [m, 2m)); drawing c with probability proportional to
# 2^c at each step gives the 2^len(w) law exactly.


def _trunc_geometric(rng: np.random.Generator, m: int) -> int:
    """K in [0, 2m) with P(K = k) = 2^(2m-1-k) / (4^m - 1): the count of
    leading zeros of a uniform nonzero 2m-bit integer, read from raw 64-bit
    draws (exact, platform independent)."""
    total = 2 * m
    while True:
        k = 0
        while k < total:
            take = min(64, total - k)
            word = int(rng.bit_generator.random_raw()) >> (64 - take)
            if word:
                return k + take - word.bit_length()
            k += take


def signed_perm_from_code(code) -> List[int]:
    """The signed permutation (letters w(1..n)) whose insertion code is
    ``code`` (code[m-1] in [0, 2m) is the length added by letter m)."""
    seq: List[int] = []
    for m, c in enumerate(code, start=1):
        if not 0 <= c < 2 * m:
            raise ValueError(f"code[{m - 1}] = {c} outside [0, {2 * m})")
        if c < m:
            seq.insert(m - 1 - c, m)
        else:
            seq.insert(c - m, -m)
    return seq


def sample_weyl(rng: np.random.Generator, n: int) -> List[int]:
    """A signed permutation of n letters with probability 2^len / prod (4^j - 1)."""
    return signed_perm_from_code([2 * m - 1 - _trunc_geometric(rng, m)
                                  for m in range(1, n + 1)])


def borel_words(L: np.ndarray, G: np.ndarray) -> List[np.ndarray]:
    """Gate words of the element of B (mod Paulis) given by the n x n GF(2)
    matrices L (entries below the diagonal: L[t, c] = 1 puts CNOT c -> t) and
    G (upper triangle and diagonal: G[i, j] = 1 puts CZ(i, j), G[i, i] = 1
    puts S(i)); the CNOT part comes first."""
    n = L.shape[0]
    parts: List[np.ndarray] = []
    # CNOT c -> t (c < t) in rounds of equal c + t, largest sum first.  A
    # round is a set of disjoint pairs, and every gate controlled by q (sum
    # > 2q) precedes every gate targeting q (sum < 2q), so each x_t ^= x_c
    # reads the original x_c: the basis-state map is I + (lower part of L),
    # in 2n - 3 rounds instead of the n^2/4 of a target-by-target order
    for sm in range(2 * n - 3, 0, -1):
        c = np.arange(max(0, sm - n + 1), (sm - 1) // 2 + 1)
        t = sm - c
        on = L[t, c].astype(bool)
        if on.any():
            parts.append(encode(np.full(int(on.sum()), TAB_CNOT), c[on], t[on]))
    # CZ on the pairs of a round-robin schedule (n - 1 rounds of disjoint
    # pairs; the gates commute, so the order only sets the depth), then S
    m = n + (n & 1)
    ring = np.arange(1, m)
    for r in range(m - 1):
        rot = np.roll(ring, r)
        a = np.concatenate(([0], rot[: m // 2 - 1]))
        b = rot[::-1][: m // 2]
        keep = (a < n) & (b < n)
        lo, hi = np.minimum(a, b)[keep], np.maximum(a, b)[keep]
        on = G[lo, hi].astype(bool)
        if on.any():
            parts.append(encode(np.full(int(on.sum()), TAB_CZ), lo[on], hi[on]))
    s = np.nonzero(np.diagonal(G))[0]
    if s.size:
        parts.append(encode(np.full(s.size, TAB_S), s, 0))
    return parts


def _borel_words(rng: np.random.Generator, n: int) -> List[np.ndarray]:
    """A uniform element of B (mod Paulis): every entry of L and G that
    borel_words reads is an independent fair bit."""
    L = rng.integers(0, 2, size=(n, n), dtype=np.uint8)
    G = rng.integers(0, 2, size=(n, n), dtype=np.uint8)
    return borel_words(L, G)


def _weyl_words(w: List[int]) -> List[np.ndarray]:
    """Gate words of the Weyl element ``w``: H on every qubit whose letter is
    negative, then SWAPs that carry qubit n - k to qubit n - |w(k)|."""
    n = len(w)
    parts: List[np.ndarray] = []
    neg = np.array([n - k for k in range(1, n + 1) if w[k - 1] < 0], dtype=np.int64)
    if neg.size:
        parts.append(encode(np.full(neg.size, TAB_H), np.sort(neg), 0))
    dest = [0] * n                      # dest[q]: where the state of qubit q goes
    for k in range(1, n + 1):
        dest[n - k] = n - abs(w[k - 1])
    src = [0] * n
    for q in range(n):
        src[dest[q]] = q
    loc = list(range(n))                # loc[s]: qubit now holding state s
    at = list(range(n))                 # at[p]: state now on qubit p
    sw_a, sw_b = [], []
    for t in range(n):
        s_ = src[t]
        p = loc[s_]
        if p != t:
            sw_a.append(min(p, t))
            sw_b.append(max(p, t))
            u = at[t]
            at[p], at[t] = u, s_
            loc[u], loc[s_] = p, t
    if sw_a:
        parts.append(encode(np.full(len(sw_a), TAB_SWAP), np.array(sw_a), np.array(sw_b)))
    return parts


def _pauli_words(rng: np.random.Generator, n: int) -> List[np.ndarray]:
    xz = rng.integers(0, 4, size=n)
    q = np.nonzero(xz)[0]
    if not q.size:
        return []
    op = np.array([TAB_I, TAB_X, TAB_Z, TAB_Y], dtype=np.int64)[xz[q]]
    return [encode(op, q, 0)]


def clifford_from_parts(n: int, b2: List[np.ndarray], w: List[int], b1: List[np.ndarray],
                        pauli: List[np.ndarray]) -> np.ndarray:
    """Gate list of P . b1 . w . b2 (b2 first) from the parts' gate words."""
    parts = list(b2) + _weyl_words(w) + list(b1) + list(pauli)
    return np.concatenate(parts) if parts else np.zeros(0, np.uint64)


def random_clifford(n: int, seed: int, circuit_id: int = 0) -> Circuit:
    """A uniformly random n-qubit Clifford (mod global phase) as a gate list,
    no measurements: the circuit applied to |0^n> leaves the tableau of that
    Clifford.  About n^2 gates (n^2/4 CNOT and n^2/4 CZ in each of b1, b2)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    b2 = _borel_words(rng, n)
    w = sample_weyl(rng, n)
    b1 = _borel_words(rng, n)
    pauli = _pauli_words(rng, n)
    gates = clifford_from_parts(n, b2, w, b1, pauli)
    return Circuit(n=n, gates=gates, n_gates=int(gates.size), n_meas=0,
                   circuit_id=circuit_id)


CLIFFORD_SWEEP_N = tuple(2 ** k for k in range(1, 14))   # 2 .. 8192, as in Fig. 2a


def clifford_sweep(n: int, count: int):
    """``count`` seeded uniformly random Cliffords on n qubits (the paper
    draws 100 per n)."""
    return [random_clifford(n, splitmix64((CONFIG_SEED + 7919 * 6 + n) ^ c), circuit_id=c)
            for c in range(count)]
