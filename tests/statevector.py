"""Brute-force state-vector simulator used only to pin the oracle (n <= 10).

Dense complex amplitudes, basis index bit q = qubit q.  Gates are applied by
their matrix definitions; measurement probabilities are sums of |amplitude|^2.
"""
import numpy as np

SQ2 = 1.0 / np.sqrt(2.0)
MAT1 = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
    "H": SQ2 * np.array([[1, 1], [1, -1]], dtype=complex),
    "S": np.array([[1, 0], [0, 1j]], dtype=complex),
    "SDG": np.array([[1, 0], [0, -1j]], dtype=complex),
}


def pauli_1q(x, z):
    """P(x,z): (0,0)=I, (1,0)=X, (1,1)=Y, (0,1)=Z."""
    return MAT1[{(0, 0): "I", (1, 0): "X", (1, 1): "Y", (0, 1): "Z"}[(x, z)]]


def kron_qubits(mats):
    """Tensor product with qubit 0 as the least significant basis bit."""
    out = np.array([[1.0 + 0j]])
    for m in reversed(mats):
        out = np.kron(out, m)
    return out


def pauli_matrix(x, z, r=0):
    return ((-1) ** int(r)) * kron_qubits([pauli_1q(int(a), int(b)) for a, b in zip(x, z)])


def gate_matrix(name, qubits, n):
    """Full 2^n x 2^n matrix of a named gate acting on the given qubits."""
    dim = 1 << n
    idx = np.arange(dim)
    if name in MAT1:
        mats = [MAT1["I"]] * n
        mats = list(mats)
        mats[qubits[0]] = MAT1[name]
        return kron_qubits(mats)
    a, b = qubits
    U = np.zeros((dim, dim), dtype=complex)
    ba = (idx >> a) & 1
    bb = (idx >> b) & 1
    if name == "CNOT":
        tgt = idx ^ (ba << b)
        U[tgt, idx] = 1
    elif name == "CZ":
        U[idx, idx] = np.where(ba & bb, -1, 1)
    elif name == "SWAP":
        tgt = idx & ~((1 << a) | (1 << b)) | (bb << a) | (ba << b)
        U[tgt, idx] = 1
    else:
        raise ValueError(name)
    return U


class StateVector:
    def __init__(self, n):
        self.n = n
        self.psi = np.zeros(1 << n, dtype=complex)
        self.psi[0] = 1.0
        self.idx = np.arange(1 << n)

    def apply(self, name, qubits):
        n = self.n
        psi = self.psi
        if name in MAT1:
            a = qubits[0]
            m = MAT1[name]
            b = (self.idx >> a) & 1
            partner = self.idx ^ (1 << a)
            new = np.where(b == 0, m[0, 0] * psi + m[0, 1] * psi[partner],
                           m[1, 0] * psi[partner] + m[1, 1] * psi)
            self.psi = new
        else:
            self.psi = gate_matrix(name, qubits, n) @ psi if n <= 6 else \
                self._apply2(name, qubits)

    def _apply2(self, name, qubits):
        a, b = qubits
        idx = self.idx
        ba = (idx >> a) & 1
        bb = (idx >> b) & 1
        psi = self.psi
        if name == "CNOT":
            src = idx ^ (ba << b)
            return psi[src]
        if name == "CZ":
            return np.where(ba & bb, -psi, psi)
        if name == "SWAP":
            src = idx & ~((1 << a) | (1 << b)) | (bb << a) | (ba << b)
            return psi[src]
        raise ValueError(name)

    def prob_one(self, a):
        return float(np.sum(np.abs(self.psi[((self.idx >> a) & 1) == 1]) ** 2))

    def project(self, a, outcome):
        keep = ((self.idx >> a) & 1) == outcome
        self.psi = np.where(keep, self.psi, 0)
        nrm = np.linalg.norm(self.psi)
        assert nrm > 1e-9
        self.psi /= nrm

    def apply_pauli(self, x, z, r):
        """(-1)^r prod_j P(x_j, z_j) |psi>, with P(1,1) = Y = i X Z."""
        idx = self.idx
        xm = 0
        zm = 0
        for j in range(self.n):
            if x[j]:
                xm |= 1 << j
            if z[j]:
                zm |= 1 << j
        ny = int(np.sum(np.asarray(x) & np.asarray(z)))
        # Z^z first: sign (-1)^{popc(z & b)}; then X^x moves b -> b ^ x.
        par = np.array([bin(int(v)).count("1") & 1 for v in (idx & zm)])
        amp = self.psi * np.where(par == 1, -1, 1)
        out = np.zeros_like(self.psi)
        out[idx ^ xm] = amp
        return out * (1j ** ny) * ((-1) ** int(r))
