"""Circuit + noise-model descriptions for the five synthetic workloads.

Flat encoding (consumed identically by the C-ABI binding and by the oracle):

* ``op_ints``   int32   [n_ops, 5]  = (kind, id, n_targets, t0, t1)
  kind 0 = coherent gate (id = gate code), kind 1 = noise site (id = channel index).
  For two-qubit operations ``t0`` is the first operand (the control of CX) and the
  local two-qubit basis index is ``2*bit(t0) + bit(t1)``.
* ``op_params`` float64 [n_ops, 3]  gate angles (U3: theta, phi, lambda; RX/RY/RZ: theta);
  for the custom gates U1/U2, ``params[0]`` is the row of ``custom_gates``.
* ``ch_ints``   int32   [n_ch, 3]   = (kind, arity, n_kraus)
* ``ch_params`` float64 [n_ch]      channel strength (p or gamma)
* ``ch_kraus``  complex128 [*]      Kraus matrices of CUSTOM channels, row-major,
  concatenated; ``ch_kraus_off[c]`` is the first entry of channel c (-1 otherwise).
* ``custom_gates`` complex128 [n_custom, 4, 4] (a 1-qubit custom gate uses the top-left 2x2).

Noise sites are numbered 0..S-1 in circuit order. Qubit q is bit q of a basis index.
Random angles come from numpy's PCG64 with a stated seed; nothing here evaluates a
matrix, a probability or a sample.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

OP_GATE, OP_NOISE = 0, 1

GATE = dict(I=0, X=1, Y=2, Z=3, H=4, S=5, SDG=6, T=7, TDG=8, RX=9, RY=10, RZ=11,
            U3=12, CX=13, CZ=14, SWAP=15, U1=16, U2=17)
GATE_ARITY = {g: (2 if g in ("CX", "CZ", "SWAP", "U2") else 1) for g in GATE}

CHANNEL = dict(DEPOL1=0, DEPOL2=1, AMPDAMP=2, BITFLIP=3, PHASEFLIP=4, CUSTOM=5)
CHANNEL_ARITY = dict(DEPOL1=1, DEPOL2=2, AMPDAMP=1, BITFLIP=1, PHASEFLIP=1)
CHANNEL_NKRAUS = dict(DEPOL1=4, DEPOL2=16, AMPDAMP=2, BITFLIP=2, PHASEFLIP=2)


@dataclass
class Circuit:
    n_qubits: int
    op_ints: np.ndarray
    op_params: np.ndarray
    ch_ints: np.ndarray
    ch_params: np.ndarray
    ch_kraus: np.ndarray
    ch_kraus_off: np.ndarray
    custom_gates: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_ops(self) -> int:
        return int(self.op_ints.shape[0])

    @property
    def n_sites(self) -> int:
        return int(np.count_nonzero(self.op_ints[:, 0] == OP_NOISE))

    @property
    def n_gates(self) -> int:
        return int(np.count_nonzero(self.op_ints[:, 0] == OP_GATE))


class CircuitBuilder:
    """Append-only builder; ``build()`` returns the flat :class:`Circuit`."""

    def __init__(self, n_qubits: int, name: str = ""):
        self.n = int(n_qubits)
        self.name = name
        self.ops: list[tuple] = []
        self.params: list[tuple] = []
        self.channels: list[tuple] = []
        self.ch_par: list[float] = []
        self.kraus: list[np.ndarray] = []
        self.kraus_off: list[int] = []
        self._kraus_len = 0
        self.customs: list[np.ndarray] = []

    def channel(self, kind: str, param: float = 0.0, kraus=None) -> int:
        if kind == "CUSTOM":
            ks = np.asarray(kraus, dtype=np.complex128)
            assert ks.ndim == 3 and ks.shape[1] == ks.shape[2] and ks.shape[1] in (2, 4)
            arity = 1 if ks.shape[1] == 2 else 2
            self.channels.append((CHANNEL[kind], arity, ks.shape[0]))
            self.kraus_off.append(self._kraus_len)
            self.kraus.append(ks.reshape(-1))
            self._kraus_len += ks.size
        else:
            self.channels.append((CHANNEL[kind], CHANNEL_ARITY[kind], CHANNEL_NKRAUS[kind]))
            self.kraus_off.append(-1)
        self.ch_par.append(float(param))
        return len(self.channels) - 1

    def gate(self, name: str, qubits, params=(0.0, 0.0, 0.0), matrix=None):
        qubits = [int(q) for q in qubits]
        assert len(qubits) == GATE_ARITY[name], (name, qubits)
        p = [float(x) for x in params] + [0.0] * (3 - len(params))
        if name in ("U1", "U2"):
            m = np.zeros((4, 4), np.complex128)
            mm = np.asarray(matrix, np.complex128)
            m[: mm.shape[0], : mm.shape[1]] = mm
            self.customs.append(m)
            p = [float(len(self.customs) - 1), 0.0, 0.0]
        t1 = qubits[1] if len(qubits) > 1 else 0
        self.ops.append((OP_GATE, GATE[name], len(qubits), qubits[0], t1))
        self.params.append(tuple(p))

    def noise(self, ch: int, qubits):
        qubits = [int(q) for q in qubits]
        assert len(qubits) == self.channels[ch][1]
        t1 = qubits[1] if len(qubits) > 1 else 0
        self.ops.append((OP_NOISE, ch, len(qubits), qubits[0], t1))
        self.params.append((0.0, 0.0, 0.0))

    def build(self, **meta) -> Circuit:
        return Circuit(
            n_qubits=self.n,
            op_ints=np.asarray(self.ops, dtype=np.int32).reshape(-1, 5),
            op_params=np.asarray(self.params, dtype=np.float64).reshape(-1, 3),
            ch_ints=np.asarray(self.channels, dtype=np.int32).reshape(-1, 3),
            ch_params=np.asarray(self.ch_par, dtype=np.float64),
            ch_kraus=(np.concatenate(self.kraus) if self.kraus else np.zeros(0, np.complex128)),
            ch_kraus_off=np.asarray(self.kraus_off, dtype=np.int64),
            custom_gates=(np.stack(self.customs) if self.customs
                          else np.zeros((0, 4, 4), np.complex128)),
            name=self.name, meta=dict(meta),
        )


# ---------------------------------------------------------------------------------------
# Workload families
# ---------------------------------------------------------------------------------------

def brickwork(n: int, layers: int, p1: float, p2: float, seed: int, name: str = "brickwork") -> Circuit:
    """U3 on every qubit (angles ~U[0, 2pi) from PCG64(seed), drawn theta, phi, lambda per
    qubit in layer order), each followed by DEPOL1(p1); then CX on pairs (0,1),(2,3),...
    on even layers and (1,2),(3,4),... on odd layers, each followed by DEPOL2(p2) on
    (control, target). A channel with strength 0 is omitted."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = CircuitBuilder(n, name)
    c1 = b.channel("DEPOL1", p1) if p1 > 0 else None
    c2 = b.channel("DEPOL2", p2) if p2 > 0 else None
    for layer in range(layers):
        for q in range(n):
            th, ph, la = rng.uniform(0.0, 2.0 * math.pi, 3)
            b.gate("U3", [q], (th, ph, la))
            if c1 is not None:
                b.noise(c1, [q])
        start = 0 if layer % 2 == 0 else 1
        for q in range(start, n - 1, 2):
            b.gate("CX", [q, q + 1])
            if c2 is not None:
                b.noise(c2, [q, q + 1])
    return b.build(layers=layers, p1=p1, p2=p2, seed=seed)


# 3x3 data grid (row-major qubits 0..8) and eight checks on ancillas 9..16:
# (ancilla, type, data support). Weight-4 faces alternate X/Z; weight-2 boundary checks
# are X on top/bottom edges and Z on left/right edges, so all checks commute.
SYNDROME17_CHECKS = (
    (9, "X", (0, 1, 3, 4)),
    (10, "X", (4, 5, 7, 8)),
    (11, "Z", (1, 2, 4, 5)),
    (12, "Z", (3, 4, 6, 7)),
    (13, "X", (1, 2)),
    (14, "X", (6, 7)),
    (15, "Z", (0, 3)),
    (16, "Z", (5, 8)),
)


def syndrome17(rounds: int = 3, gamma: float = 5e-4, p: float = 1e-3, seed: int = 1001,
               theta_max: float = 0.2) -> Circuit:
    """Syndrome-extraction-style circuit on 9 data + 8 ancilla qubits. Per round: H on
    the X-type ancillas, CX(ancilla->data) for X checks / CX(data->ancilla) for Z checks
    (ancillas in order 9..16, data ascending), H on the X-type ancillas, then RZ(theta)
    drift with theta ~ U(0, theta_max) on every data qubit. After every gate, on each
    qubit it touches: AMPDAMP(gamma) then DEPOL1(p). No mid-circuit measurement."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = CircuitBuilder(17, "syndrome17")
    ad = b.channel("AMPDAMP", gamma)
    dp = b.channel("DEPOL1", p)

    def noisy(qs):
        for q in qs:
            b.noise(ad, [q])
            b.noise(dp, [q])

    xanc = [a for a, t, _ in SYNDROME17_CHECKS if t == "X"]
    for _ in range(rounds):
        for a in xanc:
            b.gate("H", [a]); noisy([a])
        for a, t, sup in SYNDROME17_CHECKS:
            for d in sup:
                c, tg = (a, d) if t == "X" else (d, a)
                b.gate("CX", [c, tg]); noisy([c, tg])
        for a in xanc:
            b.gate("H", [a]); noisy([a])
        for d in range(9):
            th = rng.uniform(0.0, theta_max)
            b.gate("RZ", [d], (th,)); noisy([d])
    return b.build(rounds=rounds, gamma=gamma, p=p, seed=seed)


def ansatz(n: int = 16, layers: int = 8, gamma: float = 1e-3, p: float = 1e-3,
           seed: int = 1004) -> Circuit:
    """Per layer: RY on every qubit, RZ on every qubit, CZ(i, i+1) for i = 0..n-2; angles
    ~U(0, 2pi) from PCG64(seed) drawn RY-angles then RZ-angles per layer. After every gate,
    on each qubit it touches: AMPDAMP(gamma) then DEPOL1(p). Observable coefficients
    c_i ~ U(-1, 1) (for Z_i Z_{i+1}, i = 0..n-2) come from the same generator afterwards
    and are stored in ``meta['zz_coeffs']``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = CircuitBuilder(n, "ansatz")
    ad = b.channel("AMPDAMP", gamma)
    dp = b.channel("DEPOL1", p)

    def noisy(qs):
        for q in qs:
            b.noise(ad, [q])
            b.noise(dp, [q])

    for _ in range(layers):
        ry = rng.uniform(0.0, 2.0 * math.pi, n)
        rz = rng.uniform(0.0, 2.0 * math.pi, n)
        for q in range(n):
            b.gate("RY", [q], (ry[q],)); noisy([q])
        for q in range(n):
            b.gate("RZ", [q], (rz[q],)); noisy([q])
        for q in range(n - 1):
            b.gate("CZ", [q, q + 1]); noisy([q, q + 1])
    coeffs = rng.uniform(-1.0, 1.0, n - 1)
    return b.build(layers=layers, gamma=gamma, p=p, seed=seed, zz_coeffs=coeffs.tolist())


def uneven_batch(count: int = 512, seed: int = 1002, n_lo: int = 12, n_hi: int = 22,
                 d_lo: int = 10, d_hi: int = 40, p1: float = 1e-3, p2: float = 1e-2):
    """``count`` brickwork circuits with n ~ U{n_lo..n_hi}, depth ~ U{d_lo..d_hi} and shot
    budgets ~ LogUniform(1e3, 1e6); member i uses circuit seed ``seed*1000 + i``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.integers(n_lo, n_hi + 1, count)
    ds = rng.integers(d_lo, d_hi + 1, count)
    shots = np.floor(np.exp(rng.uniform(math.log(1e3), math.log(1e6), count))).astype(np.int64)
    circs = [brickwork(int(ns[i]), int(ds[i]), p1, p2, seed * 1000 + i, name=f"uneven{i}")
             for i in range(count)]
    return circs, shots


CONFIG_NAMES = {
    0: "brickwork10_d20_prop1000_1e5shots",
    1: "syndrome17_3rounds_top1e4_1e8shots",
    2: "uneven512_n12-22_prop64",
    3: "brickwork30_d60_prop2000_1e9shots",
    4: "ansatz16_l8_prop4096",
}


def config(i: int, small: bool = False) -> dict:
    """The five workloads: circuit (or circuits), PTS parameters and seeds (circuit seed
    1000+i, PTS/shot seed 2000+i). ``small=True`` gives a reduced variant of the same
    structure for tests."""
    if i == 0:
        c = brickwork(10, 20, 1e-3, 1e-2, 1000, name="brickwork10")
        return dict(name=CONFIG_NAMES[0], circuit=c, mode="proportional",
                    nsamples=1000, total_shots=100_000, seed=2000)
    if i == 1:
        c = syndrome17(rounds=1 if small else 3)
        return dict(name=CONFIG_NAMES[1], circuit=c, mode="topk",
                    k=(500 if small else 10_000), total_shots=(10**6 if small else 10**8),
                    seed=2001)
    if i == 2:
        circs, shots = uneven_batch(count=(8 if small else 512))
        return dict(name=CONFIG_NAMES[2], circuits=circs, shots=shots, mode="proportional",
                    nsamples=64, seed=2002)
    if i == 3:
        n, layers = (20, 12) if small else (30, 60)
        c = brickwork(n, layers, 5e-4, 5e-4, 1003, name=f"brickwork{n}")
        return dict(name=CONFIG_NAMES[3], circuit=c, mode="proportional",
                    nsamples=(200 if small else 2000), total_shots=(10**6 if small else 10**9),
                    seed=2003)
    if i == 4:
        c = ansatz(n=(8 if small else 16), layers=(4 if small else 8))
        return dict(name=CONFIG_NAMES[4], circuit=c, mode="proportional",
                    nsamples=(256 if small else 4096), total_shots=None, seed=2004)
    raise ValueError(i)
