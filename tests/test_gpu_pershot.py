"""Traditional per-shot trajectories (Algorithm 1) on the GPU against the oracle (-m gpu).

Unitary-mixture channels: the Kraus choice of every site depends only on (seed, site, shot), so
the labels are bit-identical to the oracle and outcomes differ only at CDF boundaries. General
channels (amplitude damping): the branch probabilities come from the complex64 state, so a
choice may flip only where u sits within 1e-6 of a cumulative boundary of the oracle's branch
probabilities (checked shot by shot), and the outcome distribution matches the density matrix."""
import numpy as np
import pytest
from scipy import stats

import densmat
from gpu_common import gpu_ctx, torch_cuda
from workloads import CircuitBuilder, brickwork, syndrome17

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return gpu_ctx()


def _run(P, circ, seed, first, m):
    torch = torch_cuda()
    cid = P.register(circ)
    bits = torch.zeros(m, dtype=torch.int32, device="cuda")
    kraus = torch.zeros((m, max(circ.n_sites, 1)), dtype=torch.uint8, device="cuda")
    P.pershot(cid, seed, first, m, bits, kraus)
    P.synchronize()
    return bits.cpu().numpy().view(np.uint32).astype(np.int64), kraus.cpu().numpy()[:, : circ.n_sites]


def _oracle(oracle_mod, circ, seed, first, m):
    o = oracle_mod.Oracle(circ)
    out, labels = [], []
    for j in range(first, first + m):
        b, k = o.pershot(seed, j, want_kraus=True)
        out.append(b); labels.append(k)
    return np.array(out, np.int64), np.array(labels, np.uint8)


@pytest.mark.parametrize("bits", [9, 12])
def test_tile_size_does_not_change_mixture_shots(P, bits):
    """With unitary mixtures only, the Kraus labels depend on (seed, site, shot) alone and every
    amplitude sees the same operations in the same order whatever the tile: shots and labels are
    bit-identical across the plan's tile sizes."""
    circ = brickwork(16, 4, 0.05, 0.08, seed=77)
    ref = _run(P, circ, 5, 0, 96)
    P.set_pershot_tile_bits(bits)
    try:
        got = _run(P, circ, 5, 0, 96)
    finally:
        P.set_pershot_tile_bits(0)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


@pytest.mark.parametrize("n", [6, 10, 15])
def test_mixture_channels_bit_exact_labels(P, oracle_mod, n):
    circ = brickwork(n, 3, 0.05, 0.08, seed=40 + n)
    m = 300 if n < 15 else 60
    got, gk = _run(P, circ, 17, 5, m)
    want, wk = _oracle(oracle_mod, circ, 17, 5, m)
    assert np.array_equal(gk, wk)
    assert np.count_nonzero(got != want) <= max(1, m // 100)


def _damping_circuit(n, layers, seed):
    rng = np.random.default_rng(seed)
    b = CircuitBuilder(n, f"damp{n}")
    ad = b.channel("AMPDAMP", 0.15)
    dp = b.channel("DEPOL1", 0.05)
    for _ in range(layers):
        for q in range(n):
            b.gate("U3", [q], rng.uniform(0, 6.28, 3)); b.noise(ad, [q]); b.noise(dp, [q])
        for q in range(0, n - 1, 2):
            b.gate("CX", [q, q + 1]); b.noise(ad, [q + 1])
    return b.build()


def _uniform(oracle_mod, seed, c0, c1, c2, c3):
    x = oracle_mod.philox([c0, c1, c2, c3], [seed & 0xFFFFFFFF, seed >> 32])
    return oracle_mod.u53(int(x[0]), int(x[1]))


def _prefix_state(oracle_mod, circ, upto_op, entries):
    """Oracle state (normalised) of the circuit's first `upto_op` operations with the Kraus choices
    `entries` at their sites."""
    from workloads import Circuit
    t = Circuit(circ.n_qubits, circ.op_ints[:upto_op], circ.op_params[:upto_op], circ.ch_ints, circ.ch_params,
                circ.ch_kraus, circ.ch_kraus_off, circ.custom_gates)
    o = oracle_mod.Oracle(t)
    sets = o.pts_targeted([entries], shots=np.zeros(1, np.uint64))
    psi, w, st = o.evolve(sets, 0)
    return psi


def _boundary_ok(C, u, a, b):
    """u lies within BOUNDARY_TOL of every cumulative boundary between outcomes a and b."""
    from gpu_common import BOUNDARY_TOL
    lo, hi = sorted((int(a), int(b)))
    return bool(np.all(np.abs(C[lo:hi] - u) <= BOUNDARY_TOL))


def _damping_kraus(gamma):
    return [np.array([[1, 0], [0, np.sqrt(1 - gamma)]]), np.array([[0, np.sqrt(gamma)], [0, 0]])]


@pytest.mark.parametrize("n,layers,m,tile_bits", [(5, 3, 400, 0), (15, 2, 80, 0), (15, 2, 80, 9), (15, 2, 80, 14)])
def test_general_channels_agree_with_oracle(P, oracle_mod, n, layers, m, tile_bits):
    """Every shot agrees with the oracle except where a uniform sits within 1e-6 of a cumulative
    boundary: at the first site whose Kraus choice differs (branch probabilities <psi|K_k^dag K_k|psi>
    of the oracle's state before that site, Algorithm 1), or, with identical choices, at the
    readout CDF of the final state. The default tile (2^12 amplitudes), 2^9 and 2^14 split the
    15-qubit state over 8, 64 and 2 CTAs whose branch-probability partials every tile sums."""
    circ = _damping_circuit(n, layers, seed=n)
    seed = 23
    P.set_pershot_tile_bits(tile_bits)
    try:
        got, gk = _run(P, circ, seed, 0, m)
    finally:
        P.set_pershot_tile_bits(0)
    want, wk = _oracle(oracle_mod, circ, seed, 0, m)
    op_ints = np.asarray(circ.op_ints)
    noise_ops = [i for i in range(circ.n_ops) if op_ints[i][0] == 1]
    K = _damping_kraus(0.15)
    flips = 0
    for j in range(m):
        diff = np.nonzero(gk[j] != wk[j])[0]
        if len(diff):
            s = int(diff[0])
            op = noise_ops[s]
            ch = int(op_ints[op][1])
            assert int(circ.ch_ints[ch][0]) == 2, f"shot {j}: mixture site {s} chose differently"
            q = int(op_ints[op][3])
            entries = [(t, int(k)) for t, k in enumerate(wk[j][:s]) if k]
            psi = _prefix_state(oracle_mod, circ, op, entries).reshape([2] * n)
            ax = n - 1 - q
            p = []
            for Kk in K:
                v = np.tensordot(Kk, psi, axes=([1], [ax]))
                p.append(float(np.sum(np.abs(v) ** 2)))
            C = np.cumsum(p) / np.sum(p)
            u = _uniform(oracle_mod, seed, s, j & 0xFFFFFFFF, j >> 32, 3)
            assert _boundary_ok(C, u, gk[j][s], wk[j][s]), f"shot {j}: site {s} u={u} C={C}"
            flips += 1
        elif got[j] != want[j]:
            entries = [(t, int(k)) for t, k in enumerate(wk[j]) if k]
            psi = _prefix_state(oracle_mod, circ, circ.n_ops, entries)
            C = np.cumsum(np.abs(psi) ** 2)
            C = C / C[-1]
            u = _uniform(oracle_mod, seed, j & 0xFFFFFFFF, j >> 32, 0, 5)
            assert _boundary_ok(C, u, got[j], want[j]), f"shot {j}: readout u={u}"
            flips += 1
    assert flips <= max(2, m // 50)


def test_damping_histogram_matches_density_matrix(P):
    circ = _damping_circuit(4, 3, seed=9)
    m = 20000
    got, _ = _run(P, circ, 31, 0, m)
    rho = densmat.evolve_rho(circ)
    p = np.real(np.diag(rho))
    counts = np.bincount(got, minlength=len(p)).astype(float)
    exp = p * m
    big = exp >= 5
    o2 = np.append(counts[big], counts[~big].sum()); e2 = np.append(exp[big], exp[~big].sum())
    chi = ((o2 - e2) ** 2 / np.maximum(e2, 1e-300)).sum()
    assert stats.chi2.sf(chi, len(o2) - 1) > 1e-3


def test_shot_windows_are_reproducible(P):
    circ = syndrome17(rounds=1)
    a, ka = _run(P, circ, 3, 0, 48)
    b, kb = _run(P, circ, 3, 16, 32)
    assert np.array_equal(a[16:], b) and np.array_equal(ka[16:], kb)
