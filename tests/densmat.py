"""Density-matrix simulation in numpy -- an independent check of the oracle.

rho -> G rho G^dag for gates and rho -> sum_k K_k rho K_k^dag for channels (the CPTP map
the trajectory method of Sec. 2.2 unravels). Gate and Kraus matrices are written here
from their textbook definitions, separately from the C oracle, so that a wrong
convention in either one makes the comparison fail. Exact rational versions of the
nominal probabilities are provided for brute-force ordering checks.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np

from workloads import GATE, CHANNEL, OP_GATE

_I2 = np.eye(2, dtype=complex)
_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
_Z = np.array([[1, 0], [0, -1]], dtype=complex)
PAULIS = [_I2, _X, _Y, _Z]
_CODE = {v: k for k, v in GATE.items()}
_CH = {v: k for k, v in CHANNEL.items()}


def gate(code: int, params, custom=None) -> np.ndarray:
    name = _CODE[int(code)]
    th, ph, la = (float(x) for x in params)
    if name == "I":
        return _I2.copy()
    if name == "X":
        return _X.copy()
    if name == "Y":
        return _Y.copy()
    if name == "Z":
        return _Z.copy()
    if name == "H":
        return np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2)
    if name == "S":
        return np.diag([1, 1j])
    if name == "SDG":
        return np.diag([1, -1j])
    if name == "T":
        return np.diag([1, np.exp(1j * math.pi / 4)])
    if name == "TDG":
        return np.diag([1, np.exp(-1j * math.pi / 4)])
    if name == "RX":  # exp(-i th X / 2)
        return math.cos(th / 2) * _I2 - 1j * math.sin(th / 2) * _X
    if name == "RY":
        return math.cos(th / 2) * _I2 - 1j * math.sin(th / 2) * _Y
    if name == "RZ":
        return math.cos(th / 2) * _I2 - 1j * math.sin(th / 2) * _Z
    if name == "U3":  # RZ(phi) RY(theta) RZ(lambda) times the global phase e^{i(phi+lambda)/2}
        return (np.exp(0.5j * (ph + la)) * gate(GATE["RZ"], (ph, 0, 0)) @ gate(GATE["RY"], (th, 0, 0))
                @ gate(GATE["RZ"], (la, 0, 0)))
    if name == "CX":  # |c t>, first operand is the high bit of the local index
        return np.kron(np.diag([1, 0]), _I2) + np.kron(np.diag([0, 1]), _X)
    if name == "CZ":
        return np.kron(np.diag([1, 0]), _I2) + np.kron(np.diag([0, 1]), _Z)
    if name == "SWAP":
        return sum(np.kron(P, P) for P in PAULIS) / 2
    if name == "U1":
        return np.asarray(custom, complex)[:2, :2]
    if name == "U2":
        return np.asarray(custom, complex)
    raise ValueError(name)


def kraus(kind: int, p: float, custom=None) -> list[np.ndarray]:
    name = _CH[int(kind)]
    if name == "DEPOL1":
        return [math.sqrt(1 - p) * _I2] + [math.sqrt(p / 3) * P for P in PAULIS[1:]]
    if name == "DEPOL2":
        out = []
        for a in range(4):
            for b in range(4):
                s = math.sqrt(1 - p) if a == b == 0 else math.sqrt(p / 15)
                out.append(s * np.kron(PAULIS[a], PAULIS[b]))
        return out
    if name == "AMPDAMP":
        return [np.array([[1, 0], [0, math.sqrt(1 - p)]], complex),
                np.array([[0, math.sqrt(p)], [0, 0]], complex)]
    if name == "BITFLIP":
        return [math.sqrt(1 - p) * _I2, math.sqrt(p) * _X]
    if name == "PHASEFLIP":
        return [math.sqrt(1 - p) * _I2, math.sqrt(p) * _Z]
    if name == "CUSTOM":
        return [np.asarray(k, complex) for k in custom]
    raise ValueError(name)


def exact_q(kind: int, p: Fraction) -> list[Fraction]:
    """Nominal Kraus probabilities tr(K^dag K)/d as exact rationals (p given as a Fraction)."""
    name = _CH[int(kind)]
    if name == "DEPOL1":
        return [1 - p] + [p / 3] * 3
    if name == "DEPOL2":
        return [1 - p] + [p / 15] * 15
    if name == "AMPDAMP":
        return [1 - p / 2, p / 2]
    if name in ("BITFLIP", "PHASEFLIP"):
        return [1 - p, p]
    raise ValueError(name)


def embed(M: np.ndarray, qubits, n: int) -> np.ndarray:
    """Full 2^n x 2^n operator of M acting on `qubits` (qubit q = bit q of the index; for
    two-qubit M the local index is 2*bit(qubits[0]) + bit(qubits[1]))."""
    N = 1 << n
    k = len(qubits)
    out = np.zeros((N, N), complex)
    for col in range(N):
        lc = 0
        for q in qubits:
            lc = 2 * lc + ((col >> q) & 1)
        base = col
        for q in qubits:
            base &= ~(1 << q)
        for lr in range(1 << k):
            row = base
            for pos, q in enumerate(qubits):
                if (lr >> (k - 1 - pos)) & 1:
                    row |= 1 << q
            out[row, col] += M[lr, lc]
    return out


def channels_of(circ):
    out = []
    for j in range(len(circ.ch_params)):
        kind, arity, nk = (int(x) for x in circ.ch_ints[j])
        custom = None
        if _CH[kind] == "CUSTOM":
            off = int(circ.ch_kraus_off[j])
            d = 1 << arity
            custom = circ.ch_kraus[off: off + nk * d * d].reshape(nk, d, d)
        out.append(kraus(kind, float(circ.ch_params[j]), custom))
    return out


def op_operator(circ, i, chans, k=None):
    kind, gid, nt, t0, t1 = (int(x) for x in circ.op_ints[i])
    qs = [t0] if nt == 1 else [t0, t1]
    if kind == OP_GATE:
        custom = None
        if _CODE[gid] in ("U1", "U2"):
            custom = circ.custom_gates[int(circ.op_params[i][0])]
        return embed(gate(gid, circ.op_params[i], custom), qs, circ.n_qubits)
    return embed(chans[gid][k], qs, circ.n_qubits)


def evolve_rho(circ) -> np.ndarray:
    n = circ.n_qubits
    N = 1 << n
    rho = np.zeros((N, N), complex)
    rho[0, 0] = 1
    chans = channels_of(circ)
    for i in range(circ.n_ops):
        kind, gid = int(circ.op_ints[i][0]), int(circ.op_ints[i][1])
        if kind == OP_GATE:
            G = op_operator(circ, i, chans)
            rho = G @ rho @ G.conj().T
        else:
            new = np.zeros_like(rho)
            for k in range(len(chans[gid])):
                K = op_operator(circ, i, chans, k)
                new += K @ rho @ K.conj().T
            rho = new
    return rho


def all_kraus_sets(circ):
    """Every Kraus combination as a sparse (site, k != 0) list."""
    nks = [int(circ.ch_ints[int(circ.op_ints[i][1])][2]) for i in range(circ.n_ops) if circ.op_ints[i][0] == 1]
    for combo in itertools.product(*[range(n) for n in nks]):
        yield [(s, k) for s, k in enumerate(combo) if k != 0]
