"""Traditional per-shot trajectories (Algorithm 1) on the GPU against the oracle (-m gpu).

Unitary-mixture channels: the Kraus choice of every site depends only on (seed, site, shot), so
the labels are bit-identical to the oracle and outcomes differ only at CDF boundaries. General
channels (amplitude damping): the branch probabilities come from the complex64 state, so a
choice may flip where u sits within ~1e-6 of a cumulative boundary; almost all shots agree and
the outcome distribution matches the density matrix."""
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


@pytest.mark.parametrize("n,layers,m", [(5, 3, 400), (15, 2, 80)])
def test_general_channels_agree_with_oracle(P, oracle_mod, n, layers, m):
    circ = _damping_circuit(n, layers, seed=n)
    got, gk = _run(P, circ, 23, 0, m)
    want, wk = _oracle(oracle_mod, circ, 23, 0, m)
    same_labels = np.all(gk == wk, axis=1)
    assert same_labels.mean() >= 0.98
    assert (got[same_labels] == want[same_labels]).mean() >= 0.98


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
