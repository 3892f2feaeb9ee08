"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* Philox4x32-10 against the published known-answer vectors (tests/golden).
* Gate matrices against textbook identities.
* Channels: CPTP condition (Sec. 2.2), unitary-mixture detection (Sec. 2.2 item 2).
* Trajectory evolution + branch weights: summing every Kraus combination reproduces an
  independent numpy density-matrix simulation (Fig. 2: the full distribution of Kraus
  subsets has unit probability), and closed forms for repeated depolarising / damping.
* PTS (Algorithm 2, Sec. 3.1): frequencies vs exact probabilities (chi-square), top-K /
  cutoff / band vs brute force in exact rational arithmetic, apportionment invariants
  and hand-worked cases.
* Sampling (Sec. 3) and Algorithm 1 per-shot trajectories: chi-square against rho's diagonal.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import densmat
from workloads import CircuitBuilder, GATE, config

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------------------------------
# Philox / U53
# ----------------------------------------------------------------------------------------
def test_philox_known_answers(oracle_mod):
    n = 0
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert list(oracle_mod.philox(w[0:4], w[4:6])) == w[6:10]
        n += 1
    assert n == 3


def test_u53_range_and_resolution(oracle_mod):
    assert oracle_mod.u53(0, 0) == 0.0
    assert oracle_mod.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle_mod.u53(0, 1 << 11) == 2.0 ** -53          # lowest bit used from x1
    assert oracle_mod.u53(0, (1 << 11) - 1) == 0.0           # bits below are discarded
    assert oracle_mod.u53(1, 0) == 2.0 ** -32


def test_shot_uniforms_are_uniform(oracle_mod):
    u = np.array([oracle_mod.shot_uniform(7, 3, j) for j in range(20000)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3


# ----------------------------------------------------------------------------------------
# Gates
# ----------------------------------------------------------------------------------------
def G(name, *p):
    from oracle.oracle import gate_matrix
    return gate_matrix(GATE[name], p)


def test_gate_textbook_identities(oracle_mod):
    X = np.array([[0, 1], [1, 0]]); Z = np.diag([1, -1])
    assert np.allclose(G("X"), X) and np.allclose(G("Z"), Z)
    assert np.allclose(G("Y"), 1j * X @ Z)
    assert np.allclose(G("H"), (X + Z) / math.sqrt(2))
    assert np.allclose(G("S") @ G("S"), Z) and np.allclose(G("T") @ G("T"), G("S"))
    assert np.allclose(G("SDG"), G("S").conj().T) and np.allclose(G("TDG"), G("T").conj().T)
    assert np.allclose(G("U3", math.pi, 0, math.pi), X)
    assert np.allclose(G("U3", math.pi / 2, 0, math.pi), G("H"))
    for th in (0.3, 1.7, 4.0):
        assert np.allclose(G("U3", th, 0, 0), G("RY", th))
        assert np.allclose(G("U3", th, -math.pi / 2, math.pi / 2), G("RX", th))
        assert np.allclose(G("U3", 0, 0, th), np.diag([1, np.exp(1j * th)]))
        assert np.allclose(G("RZ", th), np.exp(-0.5j * th) * np.diag([1, np.exp(1j * th)]))
        assert np.allclose(G("RX", th), np.cos(th / 2) * np.eye(2) - 1j * np.sin(th / 2) * X)
    rng = np.random.default_rng(0)
    for _ in range(20):
        th, ph, la = rng.uniform(0, 2 * math.pi, 3)
        U = G("U3", th, ph, la)
        assert np.allclose(U.conj().T @ U, np.eye(2), atol=1e-14)
        assert np.allclose(U, densmat.gate(GATE["U3"], (th, ph, la)), atol=1e-14)
    # two-qubit gates on |c t> basis states (local index 2c + t)
    CX = G("CX")
    for c in range(2):
        for t in range(2):
            v = np.zeros(4); v[2 * c + t] = 1
            w = CX @ v
            assert w[2 * c + (t ^ c)] == 1
    assert np.allclose(G("CZ"), np.diag([1, 1, 1, -1]))
    S = G("SWAP")
    for a in range(2):
        for b in range(2):
            v = np.zeros(4); v[2 * a + b] = 1
            assert (S @ v)[2 * b + a] == 1


# ----------------------------------------------------------------------------------------
# Channels
# ----------------------------------------------------------------------------------------
def random_channel(rng, d, r):
    """Random CPTP channel from an isometry V (d*r x d): K_k = V[k*d:(k+1)*d]."""
    A = rng.normal(size=(d * r, d)) + 1j * rng.normal(size=(d * r, d))
    V, _ = np.linalg.qr(A)
    return V.reshape(r, d, d)


def random_unitary(rng, d):
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    Q, R = np.linalg.qr(A)
    return Q * (np.diag(R) / abs(np.diag(R)))


def small_mixed_circuit(seed=3):
    """3 qubits, every gate and channel kind, 16,384 Kraus combinations."""
    rng = np.random.default_rng(seed)
    b = CircuitBuilder(3, "mixed3")
    d1 = b.channel("DEPOL1", 0.05)
    d2 = b.channel("DEPOL2", 0.08)
    ad = b.channel("AMPDAMP", 0.2)
    bf = b.channel("BITFLIP", 0.1)
    pf = b.channel("PHASEFLIP", 0.15)
    for q in range(3):
        b.gate("U3", [q], rng.uniform(0, 2 * math.pi, 3))
    b.noise(ad, [0]); b.noise(d1, [1])
    b.gate("CX", [0, 2]); b.noise(d2, [0, 2])
    b.gate("RZ", [1], (0.7,)); b.noise(d1, [1])
    b.gate("H", [2]); b.noise(bf, [2])
    b.gate("CZ", [2, 1]); b.noise(pf, [1])
    b.gate("RX", [0], (1.1,)); b.noise(ad, [0])
    b.gate("SWAP", [1, 0]); b.noise(d1, [2])
    return b.build()


def custom_circuit(seed=5):
    """4 qubits with custom gates and custom (non-mixture) channels."""
    rng = np.random.default_rng(seed)
    b = CircuitBuilder(4, "custom4")
    c1 = b.channel("CUSTOM", kraus=random_channel(rng, 2, 3))
    c2 = b.channel("CUSTOM", kraus=random_channel(rng, 4, 2))
    for q in range(4):
        b.gate("U1", [q], matrix=random_unitary(rng, 2))
    b.noise(c1, [1])
    b.gate("U2", [3, 1], matrix=random_unitary(rng, 4))
    b.noise(c2, [3, 1])
    b.gate("T", [0]); b.gate("SDG", [2]); b.gate("Y", [3])
    b.gate("CX", [2, 0]); b.noise(c1, [0])
    b.gate("RY", [2], (0.4,)); b.noise(c1, [2])
    return b.build()


@pytest.mark.parametrize("make", [small_mixed_circuit, custom_circuit])
def test_channels_cptp_and_mixture_flags(oracle_mod, make):
    circ = make()
    o = oracle_mod.Oracle(circ)
    names = {0: True, 1: True, 2: False, 3: True, 4: True}
    for j in range(len(circ.ch_params)):
        info = o.channel(j)
        assert info["cptp_err"] < 1e-14
        assert abs(info["q"].sum() - 1) < 1e-14
        kind = int(circ.ch_ints[j][0])
        want = densmat.kraus(kind, float(circ.ch_params[j]),
                             None if kind != 5 else info["kraus"])
        assert np.allclose(info["kraus"], np.asarray(want), atol=1e-15)
        if kind in names:
            assert info["mixture"] == names[kind]
        else:  # a random Stinespring channel is not a unitary mixture
            assert not info["mixture"]


# ----------------------------------------------------------------------------------------
# Evolution + weights vs the density matrix
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("make", [small_mixed_circuit, custom_circuit])
def test_exhaustive_kraus_sum_equals_density_matrix(oracle_mod, make):
    circ = make()
    o = oracle_mod.Oracle(circ)
    combos = list(densmat.all_kraus_sets(circ))
    sets = o.pts_targeted(combos, shots=np.zeros(len(combos), np.uint64))
    assert sets.count == len(combos)
    N = 1 << circ.n_qubits
    rho = np.zeros((N, N), complex)
    wsum = 0.0
    for i in range(sets.count):
        psi, w, status = o.evolve(sets, i)
        if w > 0:
            assert abs(np.vdot(psi, psi) - 1) < 1e-12
        rho += w * np.outer(psi, psi.conj())
        wsum += w
    ref = densmat.evolve_rho(circ)
    assert abs(wsum - 1) < 1e-12
    assert np.abs(rho - ref).max() < 1e-12


def test_unitary_mixture_weights_equal_nominal(oracle_mod):
    circ = config(0)["circuit"]
    o = oracle_mod.Oracle(circ)
    sets = o.pts_proportional(300, 11, total_shots=3000)
    for i in range(0, sets.count, 17):
        _, w, status = o.evolve(sets, i)
        assert status == 0
        assert abs(w - sets.q[i]) <= 1e-12 * sets.q[i]


def _one_qubit(prep, kind, p, reps):
    b = CircuitBuilder(1)
    ch = b.channel(kind, p)
    b.gate("U3", [0], prep)
    for _ in range(reps):
        b.noise(ch, [0])
    return b.build()


@pytest.mark.parametrize("reps", [1, 3, 6])
def test_depolarising_closed_form(oracle_mod, reps):
    """<Z> after k depolarising channels = (1 - 4p/3)^k <Z>_0."""
    p, th = 0.07, 0.9
    circ = _one_qubit((th, 0.3, 1.2), "DEPOL1", p, reps)
    o = oracle_mod.Oracle(circ)
    combos = list(densmat.all_kraus_sets(circ))
    sets = o.pts_targeted(combos, shots=np.zeros(len(combos), np.uint64))
    ez = 0.0
    for i in range(sets.count):
        psi, w, _ = o.evolve(sets, i)
        ez += w * (abs(psi[0]) ** 2 - abs(psi[1]) ** 2)
    assert abs(ez - (1 - 4 * p / 3) ** reps * math.cos(th)) < 1e-13


@pytest.mark.parametrize("reps", [1, 2, 5])
def test_amplitude_damping_closed_form(oracle_mod, reps):
    """Starting from |1>, P(1) after k damping channels = (1 - gamma)^k."""
    g = 0.13
    circ = _one_qubit((math.pi, 0, math.pi), "AMPDAMP", g, reps)
    o = oracle_mod.Oracle(circ)
    combos = list(densmat.all_kraus_sets(circ))
    sets = o.pts_targeted(combos, shots=np.zeros(len(combos), np.uint64))
    p1 = 0.0
    for i in range(sets.count):
        psi, w, status = o.evolve(sets, i)
        p1 += w * abs(psi[1]) ** 2
        if w == 0:
            assert status == 1   # damping twice in a row from one excitation is impossible
    assert abs(p1 - (1 - g) ** reps) < 1e-13


def test_null_rule_for_impossible_branch(oracle_mod):
    b = CircuitBuilder(2)
    ad = b.channel("AMPDAMP", 0.01)
    b.gate("H", [1])
    b.noise(ad, [0])        # qubit 0 is in |0>: K1 annihilates it
    circ = b.build()
    o = oracle_mod.Oracle(circ)
    sets = o.pts_targeted([[], [(0, 1)]], shots=np.array([5, 5], np.uint64))
    _, w0, s0 = o.evolve(sets, 0)
    _, w1, s1 = o.evolve(sets, 1)
    assert s0 == 0 and abs(w0 - 1) < 1e-15
    assert s1 == 1 and w1 == 0.0


# ----------------------------------------------------------------------------------------
# PTS (Algorithm 2) statistics and bookkeeping
# ----------------------------------------------------------------------------------------
def _few_site_circuit():
    b = CircuitBuilder(2)
    d1 = b.channel("DEPOL1", 0.3)
    ad = b.channel("AMPDAMP", 0.4)
    d2 = b.channel("DEPOL2", 0.2)
    b.gate("H", [0]); b.noise(d1, [0])
    b.gate("CX", [0, 1]); b.noise(d2, [0, 1])
    b.noise(ad, [1])
    return b.build()


def _exact_probabilities(circ):
    """q_alpha of every combination as an exact rational (p given in the circuit as a
    short decimal)."""
    chans = []
    for i in range(circ.n_ops):
        if circ.op_ints[i][0] == 1:
            ch = int(circ.op_ints[i][1])
            kind = int(circ.ch_ints[ch][0])
            chans.append(densmat.exact_q(kind, Fraction(str(float(circ.ch_params[ch])))))
    out = {}
    import itertools
    for combo in itertools.product(*[range(len(c)) for c in chans]):
        pr = Fraction(1)
        for s, k in enumerate(combo):
            pr *= chans[s][k]
        out[tuple((s, k) for s, k in enumerate(combo) if k)] = pr
    return out


def test_proportional_pts_frequencies_match_channel_probabilities(oracle_mod):
    circ = _few_site_circuit()
    o = oracle_mod.Oracle(circ)
    ns = 40000
    sets = o.pts_proportional(ns, 99, total_shots=ns)
    exact = _exact_probabilities(circ)
    assert int(sets.mult.sum()) == ns
    obs, exp = [], []
    seen = set()
    for i in range(sets.count):
        key = tuple(sets.entries(i))
        seen.add(key)
        obs.append(int(sets.mult[i])); exp.append(float(exact[key]) * ns)
        assert abs(sets.q[i] - float(exact[key])) <= 1e-14 * float(exact[key]) + 1e-300
    rest = sum(float(v) for k, v in exact.items() if k not in seen) * ns
    obs.append(0); exp.append(rest)
    obs, exp = np.array(obs, float), np.array(exp, float)
    assert _chi2_p(obs, exp / exp.sum()) > 1e-3
    # shots proportional to multiplicity: exact here (total == nsamples)
    assert np.array_equal(sets.shots, sets.mult)


def test_proportional_pts_is_canonical_and_unique(oracle_mod):
    circ = config(0)["circuit"]
    o = oracle_mod.Oracle(circ)
    sets = o.pts_proportional(1000, 2000, total_shots=100_000)
    lists = [sets.entries(i) for i in range(sets.count)]
    assert lists == sorted(lists)
    assert len(set(map(tuple, lists))) == len(lists)
    assert int(sets.mult.sum()) == 1000 and int(sets.shots.sum()) == 100_000
    assert np.array_equal(sets.shots, sets.mult * 100)       # 1e5 / 1e3 exactly
    assert lists[0] == []                                     # P(no error) ~ 0.33


def test_literal_algorithm2(oracle_mod):
    circ = _few_site_circuit()
    o = oracle_mod.Oracle(circ)
    sets = o.pts_literal(5000, 4, nshots=17)
    assert np.all(sets.shots == 17)
    for i in range(sets.count):
        sites = [s for s, _ in sets.entries(i)]
        assert len(sites) == len(set(sites))   # compatible(): one operator per site


def _literal_law(circ):
    """Exact law of Algorithm 2 as printed (Sec. 3.1): at each site every operator k >= 1 draws its
    own uniform and succeeds with probability q_k, and compatible() keeps the first success in
    listed order, so P(k) = q_k * prod_{1 <= j < k} (1 - q_j) and P(0) = prod_{j >= 1} (1 - q_j);
    sites are independent. Exact rationals."""
    import itertools
    per_site = []
    for i in range(circ.n_ops):
        if circ.op_ints[i][0] != 1:
            continue
        ch = int(circ.op_ints[i][1])
        q = densmat.exact_q(int(circ.ch_ints[ch][0]), Fraction(str(float(circ.ch_params[ch]))))
        law, miss = [], Fraction(1)
        for k in range(1, len(q)):
            law.append(q[k] * miss)
            miss *= 1 - q[k]
        per_site.append([miss] + law)
    out = {}
    for combo in itertools.product(*[range(len(c)) for c in per_site]):
        pr = Fraction(1)
        for s, k in enumerate(combo):
            pr *= per_site[s][k]
        out[tuple((s, k) for s, k in enumerate(combo) if k)] = pr
    return out


def test_literal_algorithm2_outcome_law(oracle_mod):
    """Frequencies of the printed Algorithm 2 against its exact law (chi-square). The law differs
    from the channel's (DEPOL1 p = 0.3: P(1), P(2), P(3) = 0.1, 0.09, 0.081, not 0.1 each), so keeping
    the last success instead of the first, or drawing one categorical per site, fails."""
    from scipy import stats
    circ = _few_site_circuit()
    o = oracle_mod.Oracle(circ)
    ns = 60000
    sets = o.pts_literal(ns, 31, nshots=1)
    law = _literal_law(circ)
    assert sum(law.values()) == 1
    got = {tuple(sets.entries(i)): int(sets.mult[i]) for i in range(sets.count)}
    assert sum(got.values()) == ns and set(got) <= set(law)
    big = [a for a, p in law.items() if p * ns >= 10]
    obs = np.array([got.get(a, 0) for a in big] + [ns - sum(got.get(a, 0) for a in big)], float)
    exp = np.array([float(law[a]) * ns for a in big] + [ns - sum(float(law[a]) * ns for a in big)])
    keep = exp > 0
    chi = float(((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum())
    pval = stats.chi2.sf(chi, int(keep.sum()) - 1)
    assert pval > 1e-3, f"chi-square p = {pval:.2e}"
    # the channel's own law is rejected by the same data (the test has power)
    chan = _exact_probabilities(circ)
    exp2 = np.array([float(chan[a]) * ns for a in big] + [ns - sum(float(chan[a]) * ns for a in big)])
    chi2 = float(((obs - exp2) ** 2 / np.maximum(exp2, 1e-9)).sum())
    assert stats.chi2.sf(chi2, len(big)) < 1e-6


_ORDER_CACHE = {}


def _bruteforce_order(circ):
    key = circ.name
    if key not in _ORDER_CACHE:
        exact = _exact_probabilities(circ)
        _ORDER_CACHE[key] = (exact, sorted(exact.items(), key=lambda kv: (-kv[1], list(kv[0]))))
    return _ORDER_CACHE[key][1]


def _ratio_circuit():
    """Eleven sites with tie classes (same channel on several sites)."""
    b = CircuitBuilder(3, "ratio11")
    d1 = b.channel("DEPOL1", 0.03)
    ad = b.channel("AMPDAMP", 0.05)
    bf = b.channel("BITFLIP", 0.01)
    d2 = b.channel("DEPOL2", 0.02)
    for q in range(3):
        b.gate("H", [q]); b.noise(d1, [q]); b.noise(ad, [q])
    b.gate("CX", [0, 1]); b.noise(d2, [0, 1])
    b.noise(bf, [2]); b.noise(bf, [0]); b.noise(d1, [2]); b.noise(ad, [1])
    return b.build()


@pytest.mark.parametrize("K", [1, 2, 7, 40, 333, 2000])
def test_topk_matches_bruteforce(oracle_mod, K):
    circ = _ratio_circuit()
    o = oracle_mod.Oracle(circ)
    order = _bruteforce_order(circ)
    sets = o.pts_topk(K, total_shots=10**6)
    want = sorted(list(k) for k, _ in order[:K])
    got = [[tuple(e) for e in sets.entries(i)] for i in range(sets.count)]
    assert got == [list(w) for w in want]
    assert int(sets.shots.sum()) == 10**6
    table = dict(order)
    qs = np.array([float(table[tuple(g)]) for g in got])
    assert np.allclose(sets.q, qs, rtol=1e-13, atol=0)


@pytest.mark.parametrize("pmin,pmax", [(1e-3, 1.0), (1e-5, 1.0), (1e-6, 1e-4), (2e-4, 3e-3)])
def test_band_matches_bruteforce(oracle_mod, pmin, pmax):
    circ = _ratio_circuit()
    o = oracle_mod.Oracle(circ)
    _bruteforce_order(circ)
    exact = _ORDER_CACHE[circ.name][0]
    fmin, fmax = Fraction(pmin), Fraction(pmax)
    want = sorted(list(k) for k, v in exact.items() if fmin <= v <= fmax)
    sets = o.pts_band(pmin, pmax, total_shots=1000)
    got = [[tuple(e) for e in sets.entries(i)] for i in range(sets.count)]
    assert got == want


def test_topk_on_syndrome_circuit_has_expected_structure(oracle_mod):
    """Top 10^4 of the 17-qubit syndrome circuit: the empty set, all 780 single errors
    (585 depolarising, 195 damping) and 9,219 depolarising doubles chosen from their tie
    class by canonical order."""
    circ = config(1)["circuit"]
    o = oracle_mod.Oracle(circ)
    sets = o.pts_topk(10_000, total_shots=10**8)
    sizes = np.diff(sets.offsets.astype(np.int64))
    assert sets.count == 10_000
    assert (sizes == 0).sum() == 1 and (sizes == 1).sum() == 780 and (sizes == 2).sum() == 9219
    assert int(sets.shots.sum()) == 10**8
    assert sets.shots[0] > 7 * 10**7


# ----------------------------------------------------------------------------------------
# Apportionment
# ----------------------------------------------------------------------------------------
def test_apportionment_hand_worked(oracle_mod):
    assert oracle_mod.apportion_counts([1, 1, 1], 10).tolist() == [4, 3, 3]
    assert oracle_mod.apportion_counts([5, 3, 2], 7).tolist() == [4, 2, 1]     # 3.5, 2.1, 1.4
    assert oracle_mod.apportion_counts([2, 2, 1], 3).tolist() == [1, 1, 1]     # 1.2, 1.2, 0.6
    assert oracle_mod.apportion_counts([1, 1], 1).tolist() == [1, 0]           # tie -> lower index
    assert oracle_mod.apportion_counts([1, 2, 1], 2).tolist() == [1, 1, 0]     # 0.5, 1, 0.5 -> tie
    assert oracle_mod.apportion_weights([0.5, 0.3, 0.2], 7).tolist() == [4, 2, 1]
    assert oracle_mod.apportion_weights([0.25, 0.25, 0.5], 4).tolist() == [1, 1, 2]
    assert oracle_mod.apportion_counts([7], 12345).tolist() == [12345]
    assert oracle_mod.apportion_counts([3, 0, 1], 0).tolist() == [0, 0, 0]


def test_apportionment_invariants(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(50):
        n = int(rng.integers(1, 60))
        c = rng.integers(0, 1000, n).astype(np.uint64)
        c[0] += 1
        M = int(rng.integers(0, 10**9))
        m = oracle_mod.apportion_counts(c, M).astype(np.float64)
        assert m.sum() == M
        quota = M * c.astype(float) / c.sum()
        assert np.all(np.abs(m - quota) < 1 + 1e-6)
        w = rng.exponential(size=n)
        m = oracle_mod.apportion_weights(w, M).astype(np.float64)
        assert m.sum() == M
        assert np.all(np.abs(m - M * w / w.sum()) < 1 + 1e-6)


# ----------------------------------------------------------------------------------------
# Sampling (Sec. 3) and Algorithm 1
# ----------------------------------------------------------------------------------------
def _chi2_p(counts, probs):
    exp = probs * counts.sum()
    big = exp >= 5
    o2 = np.append(counts[big], counts[~big].sum()); e2 = np.append(exp[big], exp[~big].sum())
    if e2[-1] == 0:
        o2, e2 = o2[:-1], e2[:-1]
    chi = ((o2 - e2) ** 2 / e2).sum()
    return stats.chi2.sf(chi, len(o2) - 1)


def test_sampler_inverse_cdf_and_histogram(oracle_mod):
    rng = np.random.default_rng(4)
    n = 7
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi[5] = 0                       # an impossible outcome
    psi /= np.linalg.norm(psi)
    m = 50000
    out = oracle_mod.sample(n, psi, m, seed=5, alpha=9)
    Cc = oracle_mod.cdf(n, psi)
    assert np.all(np.diff(Cc) >= 0)
    for j in range(0, m, 997):      # every shot lies in its CDF bucket
        t = oracle_mod.shot_uniform(5, 9, j) * Cc[-1]
        i = int(out[j])
        assert t < Cc[i] and (i == 0 or Cc[i - 1] <= t)
    counts = np.bincount(out.astype(np.int64), minlength=1 << n).astype(float)
    assert counts[5] == 0
    assert _chi2_p(counts, np.abs(psi) ** 2) > 1e-3
    # shots are a pure function of (seed, alpha, j): a later window repeats the same values
    assert np.array_equal(oracle_mod.sample(n, psi, 100, 5, 9, first_shot=300), out[300:400])


@pytest.mark.parametrize("make", [_few_site_circuit, small_mixed_circuit])
def test_pershot_algorithm1_matches_density_matrix(oracle_mod, make):
    circ = make()
    o = oracle_mod.Oracle(circ)
    m = 6000
    shots = np.array([o.pershot(31, j) for j in range(m)], np.int64)
    rho = densmat.evolve_rho(circ)
    p = np.real(np.diag(rho))
    counts = np.bincount(shots, minlength=len(p)).astype(float)
    assert _chi2_p(counts, p) > 1e-3


def test_ptsbe_and_pershot_agree_in_distribution(oracle_mod):
    """Pooled PTSBE shots (proportional PTS + BE) and Algorithm 1 shots come from the same
    distribution (Algorithm 2: sets drawn as at state-preparation runtime)."""
    circ = _few_site_circuit()
    o = oracle_mod.Oracle(circ)
    sets = o.pts_proportional(2000, 8, total_shots=20000)
    pooled = []
    for i in range(sets.count):
        psi, w, st = o.evolve(sets, i)
        pooled.append(oracle_mod.sample(circ.n_qubits, psi, int(sets.shots[i]), 9, i))
    pooled = np.concatenate(pooled).astype(np.int64)
    per = np.array([o.pershot(10, j) for j in range(20000)], np.int64)
    a = np.bincount(pooled, minlength=4); b = np.bincount(per, minlength=4)
    _, pv, _, _ = stats.chi2_contingency(np.vstack([a, b]))
    assert pv > 1e-3


def test_loss_is_importance_weighted_expectation(oracle_mod):
    """Summing <psi~_a|O|psi~_a> over every Kraus combination gives Tr(O rho)."""
    circ = small_mixed_circuit()
    o = oracle_mod.Oracle(circ)
    combos = list(densmat.all_kraus_sets(circ))
    sets = o.pts_targeted(combos, shots=np.zeros(len(combos), np.uint64))
    masks = np.array([0b011, 0b110, 0b001], np.uint64)
    coeffs = np.array([0.7, -0.4, 0.25])
    _, per = o.loss(sets, masks, coeffs, per_set=True)
    total = float((per * sets.q).sum())
    rho = densmat.evolve_rho(circ)
    diag = np.real(np.diag(rho))
    x = np.arange(len(diag))
    ov = sum(c * np.where(np.array([bin(v & int(mk)).count("1") % 2 for v in x]) == 1, -1.0, 1.0)
             for mk, c in zip(masks, coeffs))
    assert abs(total - float((diag * ov).sum())) < 1e-12


def test_predicate_sets_against_full_enumeration(oracle_mod):
    """The oracle's rule-based targeted sets equal the sets picked, by the same rule, from the
    independent enumeration of every Kraus combination (tests/densmat.py); with every filter open
    and max_errors = S they are all combinations, whose nominal probabilities sum to 1."""
    circ = small_mixed_circuit()
    o = oracle_mod.Oracle(circ)
    S = o.n_sites
    allc = [sorted(c) for c in densmat.all_kraus_sets(circ)]
    op_ints = np.asarray(circ.op_ints)
    noise_ops = [i for i in range(circ.n_ops) if op_ints[i][0] == 1]

    def site_qubits(s):
        i = noise_ops[s]
        return {int(op_ints[i][3])} | ({int(op_ints[i][4])} if op_ints[i][2] == 2 else set())

    for kw, keep in [
        (dict(max_errors=S, include_empty=True), lambda c: True),
        (dict(max_errors=2), lambda c: 1 <= len(c) <= 2),
        (dict(max_errors=3, qubit_mask=0b101, weight_parity=1),
         lambda c: len(c) in (1, 3) and all(site_qubits(s) <= {0, 2} for s, _ in c)),
        (dict(max_errors=2, kraus_mask=0b0010, site_lo=2, site_hi=8, include_empty=True),
         lambda c: len(c) <= 2 and all(k == 1 and 2 <= s < 8 for s, k in c)),
    ]:
        got = sorted(tuple(x) for x in oracle_mod.predicate_sets(circ, **kw))
        want = sorted(tuple(c) for c in allc if keep(c))
        assert got == want
    sets = o.pts_targeted(oracle_mod.predicate_sets(circ, max_errors=S, include_empty=True), total_shots=10)
    assert abs(float(np.sum(sets.q)) - 1.0) < 1e-12


def test_predicate_sets_gate_filter_against_hand_table(oracle_mod):
    """The gate_mask rule ("the gate a site follows" = the last gate before the site that shares one
    of its qubits) against a table read off small_mixed_circuit by hand: site 7 (DEPOL1 on qubit 2)
    comes right after SWAP(1, 0) but follows CZ(2, 1), the last gate on qubit 2."""
    from workloads import GATE
    circ = small_mixed_circuit()
    follows = {0: "U3", 1: "U3", 2: "CX", 3: "RZ", 4: "H", 5: "CZ", 6: "RX", 7: "CZ"}
    allc = [sorted(c) for c in densmat.all_kraus_sets(circ)]
    for names, max_err in [(("CZ", "U3"), 2), (("SWAP", "H"), 3), (("CX", "RX", "RZ"), 1)]:
        mask = 0
        for g in names:
            mask |= 1 << GATE[g]
        eligible = {s for s, g in follows.items() if g in names}
        got = sorted(tuple(x) for x in oracle_mod.predicate_sets(circ, max_errors=max_err, gate_mask=mask))
        want = sorted(tuple(c) for c in allc if 1 <= len(c) <= max_err and all(s in eligible for s, _ in c))
        assert got == want, names
