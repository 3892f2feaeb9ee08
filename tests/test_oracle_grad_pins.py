"""Pins of the oracle's gradient of the fixed-set estimator (test infrastructure for the adjoint
backward) against facts that do not come from its finite differences:

* parameter shift: every gate angle here enters as exp(-i theta P / 2) of a Pauli P (U3 up to a
  global phase), so d/dtheta of <psi|O|psi> = [f(theta + pi/2) - f(theta - pi/2)] / 2 exactly;
* closed forms for one qubit: RY(theta) then amplitude damping or depolarising, each Kraus branch;
* the estimator identity: with every Kraus combination as a set and q_alpha held fixed,
  sum_alpha q_alpha d(e_alpha/q_alpha) = d Tr(O rho), rho from the independent numpy
  density-matrix simulation (tests/densmat.py), differentiated by its own central differences.
"""
import math

import numpy as np
import pytest

import densmat
from workloads import CircuitBuilder


def zz_masks(n):
    return np.array([(1 << i) | (1 << (i + 1)) for i in range(n - 1)], np.uint64)


def ry_channel_circuit(theta, kind, strength):
    b = CircuitBuilder(1, "one")
    ch = b.channel(kind, strength)
    b.gate("RY", [0], (theta,))
    b.noise(ch, [0])
    return b.build()


def grad_circuit(seed=11):
    """3 qubits: RX, RY, RZ, U3 angles, CZ / CX, damping, depolarising (1 and 2 qubits), bit flip."""
    rng = np.random.default_rng(seed)
    b = CircuitBuilder(3, "grad3")
    ad = b.channel("AMPDAMP", 0.15)
    d1 = b.channel("DEPOL1", 0.06)
    d2 = b.channel("DEPOL2", 0.09)
    bf = b.channel("BITFLIP", 0.12)
    for q in range(3):
        b.gate("U3", [q], rng.uniform(0, 2 * math.pi, 3)); b.noise(ad, [q])
    b.gate("CZ", [0, 1]); b.noise(d1, [0])
    b.gate("RY", [2], (rng.uniform(0, 2 * math.pi),)); b.noise(ad, [2])
    b.gate("CX", [2, 1]); b.noise(d2, [2, 1])
    b.gate("RX", [0], (rng.uniform(0, 2 * math.pi),)); b.noise(bf, [0])
    b.gate("RZ", [1], (rng.uniform(0, 2 * math.pi),)); b.noise(ad, [1])
    b.gate("RY", [1], (rng.uniform(0, 2 * math.pi),))
    return b.build()


def test_fd_matches_parameter_shift(oracle_mod):
    circ = grad_circuit()
    o = oracle_mod.Oracle(circ)
    sets = o.pts_proportional(64, 7, total_shots=6400)
    masks = zz_masks(3)
    coeffs = np.array([0.8, -0.3])
    per, dp, _ = oracle_mod.loss_grad_fd(circ, sets, masks, coeffs, h=1e-4)
    slots = oracle_mod.gate_param_slots(circ)
    assert len(slots) == 3 * 3 + 4
    for (i, j) in slots:
        vals = []
        for s in (+1.0, -1.0):
            P = np.array(circ.op_params, copy=True)
            P[i, j] += s * math.pi / 2
            c2 = oracle_mod._with_params(circ, op_params=P)
            _, ps = oracle_mod.Oracle(c2).loss(sets, masks, coeffs, per_set=True)
            vals.append(ps)
        shift = (vals[0] - vals[1]) / 2
        np.testing.assert_allclose(dp[i, j], shift, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("theta", [0.3, 1.9, 4.0])
def test_closed_form_damping(oracle_mod, theta):
    g = 0.2
    circ = ry_channel_circuit(theta, "AMPDAMP", g)
    o = oracle_mod.Oracle(circ)
    sets = o.pts_targeted([[], [(0, 1)]], shots=np.zeros(2, np.uint64))
    per, dp, dn = oracle_mod.loss_grad_fd(circ, sets, np.array([1], np.uint64), np.array([1.0]), h=1e-5)
    q0, q1 = 1 - g / 2, g / 2
    c2, s2 = math.cos(theta / 2) ** 2, math.sin(theta / 2) ** 2
    # no damping: psi~ = (cos t/2, sqrt(1-g) sin t/2); with damping: psi~ = (sqrt(g) sin t/2, 0)
    np.testing.assert_allclose(per, [(c2 - (1 - g) * s2) / q0, g * s2 / q1], rtol=1e-12)
    np.testing.assert_allclose(dp[0, 0], [-(2 - g) / 2 * math.sin(theta) / q0, math.sin(theta)], rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(dn[0], [s2 / q0, s2 / q1], rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("theta", [0.5, 2.6])
def test_closed_form_depolarising(oracle_mod, theta):
    p = 0.09
    circ = ry_channel_circuit(theta, "DEPOL1", p)
    o = oracle_mod.Oracle(circ)
    sets = o.pts_targeted([[], [(0, 1)], [(0, 3)]], shots=np.zeros(3, np.uint64))
    per, dp, dn = oracle_mod.loss_grad_fd(circ, sets, np.array([1], np.uint64), np.array([1.0]), h=1e-5)
    c = math.cos(theta)
    # K0 = sqrt(1-p) I, K_X = sqrt(p/3) X, K_Z = sqrt(p/3) Z; q fixed at 1-p, p/3, p/3
    np.testing.assert_allclose(per, [c, -c, c], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(dp[0, 0], [-math.sin(theta), math.sin(theta), -math.sin(theta)], rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(dn[0], [-c / (1 - p), -c / p, c / p], rtol=1e-7, atol=1e-9)


def test_estimator_gradient_is_density_matrix_gradient(oracle_mod):
    circ = grad_circuit(seed=4)
    o = oracle_mod.Oracle(circ)
    combos = list(densmat.all_kraus_sets(circ))
    sets = o.pts_targeted(combos, shots=np.zeros(len(combos), np.uint64))
    masks = zz_masks(3)
    coeffs = np.array([0.6, 0.45])
    per, dp, dn = oracle_mod.loss_grad_fd(circ, sets, masks, coeffs, h=1e-4)
    q = np.asarray(sets.q)
    x = np.arange(8)
    ov = sum(c * np.where(np.array([bin(v & int(mk)).count("1") % 2 for v in x]) == 1, -1.0, 1.0)
             for mk, c in zip(masks, coeffs))

    def tr_o_rho(cc):
        return float((np.real(np.diag(densmat.evolve_rho(cc))) * ov).sum())

    h = 1e-5
    for (i, j) in oracle_mod.gate_param_slots(circ):
        P1 = np.array(circ.op_params, copy=True); P1[i, j] += h
        P2 = np.array(circ.op_params, copy=True); P2[i, j] -= h
        ref = (tr_o_rho(oracle_mod._with_params(circ, op_params=P1)) -
               tr_o_rho(oracle_mod._with_params(circ, op_params=P2))) / (2 * h)
        assert abs(float((q * dp[i, j]).sum()) - ref) < 1e-7
    for c in oracle_mod.noise_param_slots(circ):
        P1 = np.array(circ.ch_params, copy=True); P1[c] += h
        P2 = np.array(circ.ch_params, copy=True); P2[c] -= h
        ref = (tr_o_rho(oracle_mod._with_params(circ, ch_params=P1)) -
               tr_o_rho(oracle_mod._with_params(circ, ch_params=P2))) / (2 * h)
        assert abs(float((q * dn[c]).sum()) - ref) < 1e-7


def test_diagonal_observable_outcome_probability(oracle_mod):
    """A dense diagonal that is the indicator of one outcome gives that outcome's probability."""
    circ = grad_circuit(seed=2)
    o = oracle_mod.Oracle(circ)
    combos = list(densmat.all_kraus_sets(circ))
    sets = o.pts_targeted(combos, shots=np.zeros(len(combos), np.uint64))
    diag = np.zeros(8); diag[5] = 1.0
    _, per = o.loss(sets, np.zeros(0, np.uint64), np.zeros(0), per_set=True, diag=diag)
    rho = densmat.evolve_rho(circ)
    assert abs(float((per * np.asarray(sets.q)).sum()) - float(np.real(rho[5, 5]))) < 1e-12
