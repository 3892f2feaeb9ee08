"""Parity of the adjoint backward (ptsbe_backward) with the CPU oracle (-m gpu).

The loss is the fixed-set estimator L = (1/N) sum_a mult_a <psi~_a|O|psi~_a> / q_a over a range of
sets (Sec. 3 with the sets held fixed). The oracle gives per-set values e_a / q_a and their central
finite differences (h = 1e-4, FP64) with respect to gate angles and channel strengths; the GPU's
adjoint gradients must agree to 1e-3 relative (plus 1e-4 of the largest entry for entries near
zero), the loss and per-set values to 1e-5 relative. Cases: every gate and channel kind on 3
qubits, ragged sub-ranges, damping jumps (non-invertible blocks restored from checkpoints),
periodic checkpoints, a dense diagonal observable (an outcome probability), 14-16 qubits
(clusters of 2, 4 and 8 CTAs exchanging qubit positions) and the 16-qubit ansatz at full size.
"""
import math

import numpy as np
import pytest

from gpu_common import gpu_ctx, torch_cuda
from workloads import CircuitBuilder, ansatz

pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-3


@pytest.fixture(scope="module")
def P():
    return gpu_ctx()


def zz(n):
    return np.array([(1 << i) | (1 << (i + 1)) for i in range(n - 1)], np.uint64)


def grad_circuit(seed=11, n=3):
    rng = np.random.default_rng(seed)
    b = CircuitBuilder(n, "grad")
    ad = b.channel("AMPDAMP", 0.15)
    d1 = b.channel("DEPOL1", 0.06)
    d2 = b.channel("DEPOL2", 0.09)
    bf = b.channel("BITFLIP", 0.12)
    pf = b.channel("PHASEFLIP", 0.07)
    for q in range(n):
        b.gate("U3", [q], rng.uniform(0, 2 * math.pi, 3)); b.noise(ad, [q])
    b.gate("CZ", [0, 1]); b.noise(d1, [0])
    b.gate("RY", [2], (rng.uniform(0, 2 * math.pi),)); b.noise(ad, [2])
    b.gate("CX", [2, 1]); b.noise(d2, [2, 1])
    b.gate("H", [0]); b.noise(pf, [0])
    b.gate("RX", [0], (rng.uniform(0, 2 * math.pi),)); b.noise(bf, [0])
    b.gate("SWAP", [0, 2])
    b.gate("RZ", [1], (rng.uniform(0, 2 * math.pi),)); b.noise(ad, [1])
    b.gate("RY", [1], (rng.uniform(0, 2 * math.pi),)); b.noise(ad, [0])
    b.gate("S", [2]); b.gate("RY", [0], (rng.uniform(0, 2 * math.pi),))
    return b.build()


def run_gpu(P, circ, info, first, count, masks, coeffs, diag=None, ckpt=0, cid=None):
    torch = torch_cuda()
    loss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    per = torch.full((max(count, 1),), float("nan"), dtype=torch.float64, device="cuda")
    gp = torch.full((circ.n_ops, 3), float("nan"), dtype=torch.float64, device="cuda")
    gn = torch.full((max(len(circ.ch_params), 1),), float("nan"), dtype=torch.float64, device="cuda")
    d = None if diag is None else torch.as_tensor(diag, dtype=torch.float64, device="cuda")
    P.backward(info.circuit_id if cid is None else cid, info, first, count, masks, coeffs, diag=d,
               checkpoint_every=ckpt, loss=loss, per_set=per, grad_params=gp, grad_noise=gn)
    torch.cuda.synchronize()
    P.synchronize()
    return (float(loss.cpu()[0]), per.cpu().numpy()[:count], gp.cpu().numpy(),
            gn.cpu().numpy()[: len(circ.ch_params)])


def run_ref(oracle_mod, circ, info, first, count, masks, coeffs, diag=None, param_slots=None, noise_slots=None):
    """Oracle loss, per-set values, finite-difference gradients over the range, and per set the
    scale ||psi~_a||^2 / q_a * ||O||_inf that bounds how far complex64 amplitudes can move e_a / q_a."""
    o = oracle_mod.Oracle(circ)
    sets = o.pts_targeted([info.entries(first + i) for i in range(count)], shots=np.zeros(count, np.uint64))
    per, dp, dn = oracle_mod.loss_grad_fd(circ, sets, masks, coeffs, h=1e-4, diag=diag,
                                          param_slots=param_slots, noise_slots=noise_slots)
    _, norm = o.loss(sets, np.zeros(1, np.uint64), np.ones(1), per_set=True)
    onorm = float(np.abs(coeffs).sum()) + (float(np.abs(diag).max()) if diag is not None else 0.0)
    mult = np.asarray(info.mult[first: first + count], np.float64)
    w = mult / mult.sum()
    return float((w * per).sum()), per, (dp * w).sum(axis=-1), (dn * w).sum(axis=-1), norm * onorm, w


def assert_grad(got, want, label):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    scale = max(np.abs(want).max(), 1e-12)
    err = np.abs(got - want)
    bad = err > GRAD_RTOL * np.abs(want) + 1e-4 * scale
    assert not bad.any(), f"{label}: worst {err.max():.3e} at {np.argwhere(bad)[:4].tolist()} (scale {scale:.3e})"


def compare(oracle_mod, P, circ, info, first, count, masks, coeffs, diag=None, ckpt=0, param_slots=None,
            noise_slots=None):
    L, per, gp, gn = run_gpu(P, circ, info, first, count, masks, coeffs, diag, ckpt)
    Lr, perr, gpr, gnr, scale, w = run_ref(oracle_mod, circ, info, first, count, masks, coeffs, diag, param_slots,
                                           noise_slots)
    # complex64 amplitudes: e_a / q_a within 1e-5 of its scale ||psi~_a||^2 / q_a ||O||
    assert np.all(np.abs(per - perr) <= LOSS_RTOL * scale), np.max(np.abs(per - perr) / scale)
    assert abs(L - Lr) <= LOSS_RTOL * float((w * scale).sum()), (L, Lr)
    slots = oracle_mod.gate_param_slots(circ) if param_slots is None else param_slots
    idx = tuple(np.array(slots).T)
    assert_grad(gp[idx], gpr[idx], "gate angles")
    # parameters that are not angles of RX/RY/RZ/U3 have zero gradient
    mask = np.zeros_like(gp, bool)
    mask[tuple(np.array(oracle_mod.gate_param_slots(circ)).T)] = True
    assert np.all(gp[~mask] == 0.0)
    ns = oracle_mod.noise_param_slots(circ) if noise_slots is None else noise_slots
    assert_grad(gn[ns], gnr[ns], "channel strengths")
    return L


def damping_sites(circ):
    noise_ops = np.nonzero(circ.op_ints[:, 0] == 1)[0]
    return [s for s, i in enumerate(noise_ops) if int(circ.ch_ints[int(circ.op_ints[i][1])][0]) == 2]


def test_every_kind_three_qubits(P, oracle_mod):
    circ = grad_circuit()
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=5, nsamples=200, total_shots=20000)
    compare(oracle_mod, P, circ, info, 0, info.count, zz(3), np.array([0.8, -0.3]))


@pytest.mark.parametrize("ckpt", [0, 1, 3])
def test_subrange_and_checkpoints(P, oracle_mod, ckpt):
    circ = grad_circuit(seed=7)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=9, nsamples=300, total_shots=30000)
    first = 2
    count = min(9, info.count - first)
    compare(oracle_mod, P, circ, info, first, count, zz(3), np.array([0.5, 0.9]), ckpt=ckpt)


def test_damping_jumps_and_outcome_probability(P, oracle_mod):
    """Sets that damp a qubit (K_1 cannot be inverted: its block input comes from a checkpoint),
    with the indicator of one outcome as the observable."""
    circ = grad_circuit(seed=3)
    cid = P.register(circ)
    ad = damping_sites(circ)
    sets = [[], [(ad[0], 1)], [(ad[1], 1), (ad[3], 1)], [(ad[2], 1), (ad[-1], 1)], [(ad[0], 1), (ad[-2], 1)]]
    info = P.sample_kraus(cid, "targeted", targeted=[sorted(x) for x in sets])
    diag = np.zeros(8); diag[1] = 1.0
    compare(oracle_mod, P, circ, info, 0, info.count, np.zeros(0, np.uint64), np.zeros(0), diag=diag)
    compare(oracle_mod, P, circ, info, 0, info.count, zz(3), np.array([1.0, -0.5]))
    compare(oracle_mod, P, circ, info, 1, 3, zz(3), np.array([1.0, -0.5]), ckpt=2)


def test_single_trajectory(P, oracle_mod):
    circ = grad_circuit(seed=21)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=2, nsamples=100, total_shots=100)
    for a in [0, info.count // 2, info.count - 1]:
        compare(oracle_mod, P, circ, info, a, 1, zz(3), np.array([1.0, 1.0]))


def test_parameters_of_another_circuit(P, oracle_mod):
    """Sets drawn at one parameter point, loss and gradient at another (same structure)."""
    import dataclasses
    circ = grad_circuit(seed=13)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=4, nsamples=120, total_shots=1200)
    rng = np.random.default_rng(0)
    c2 = dataclasses.replace(circ, op_params=circ.op_params + rng.normal(0, 0.3, circ.op_params.shape),
                             ch_params=np.clip(circ.ch_params * 1.3, 0, 1))
    cid2 = P.register(c2)
    L, per, gp, gn = run_gpu(P, c2, info, 0, info.count, zz(3), np.array([0.7, 0.2]), cid=cid2)
    # the oracle differentiates at c2's parameters, with the q_alpha of the sets drawn at circ
    o = oracle_mod.Oracle(circ)
    sets = o.pts_proportional(120, 4, total_shots=1200)
    per_r, dp, dn = oracle_mod.loss_grad_fd(c2, sets, zz(3), np.array([0.7, 0.2]), h=1e-4)
    _, norm = oracle_mod.Oracle(c2).loss(sets, np.zeros(1, np.uint64), np.ones(1), per_set=True)
    w = np.asarray(info.mult, np.float64) / np.sum(info.mult)
    assert abs(L - float((w * per_r).sum())) <= 1e-5 * 0.9 * float((w * norm).sum())
    slots = oracle_mod.gate_param_slots(circ)
    assert_grad(gp[tuple(np.array(slots).T)], (dp * w).sum(-1)[tuple(np.array(slots).T)], "angles at c2")
    ns = oracle_mod.noise_param_slots(circ)
    assert_grad(gn[ns], (dn * w).sum(-1)[ns], "strengths at c2")
    b = CircuitBuilder(3, "other")
    b.gate("H", [0])
    cid3 = P.register(b.build())
    from paper_2504_16297_gb300.capi import PtsbeError
    with pytest.raises(PtsbeError):
        run_gpu(P, circ, info, 0, info.count, zz(3), np.array([1.0, 1.0]), cid=cid3)


@pytest.mark.parametrize("n", [13, 14, 15, 16])
def test_cluster_sizes(P, oracle_mod, n):
    """13 qubits: one CTA; 14-16: clusters of 2, 4, 8 CTAs with qubit-position swaps."""
    circ = ansatz(n=n, layers=2, gamma=0.02, p=0.02, seed=40 + n)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=n, nsamples=12, total_shots=1200)
    slots = oracle_mod.gate_param_slots(circ)
    # angles on local and high (rank) qubits, early and late in the circuit
    pick = [slots[0], slots[n - 1], slots[n + 2], slots[-1], slots[len(slots) // 2]]
    compare(oracle_mod, P, circ, info, 0, info.count, zz(n), np.asarray(circ.meta["zz_coeffs"]),
            param_slots=pick)


@pytest.mark.parametrize("layers", [8, 16, 32])
def test_gradient_error_with_depth(P, oracle_mod, layers):
    """Deep damped circuits: the 10-qubit ansatz at 8, 16 and 32 layers (up to 928 gates, sets with
    up to 40 Kraus entries, 20+ damping jumps). Two things grow with depth: the amplification of
    rounding when phi is un-computed through damping inverses (the plan stores phi where it would
    pass 2^6: 0, 1 and 2 copies here), and the shrinking of an unnormalised FP32 state by sqrt(gamma)
    per jump (the kernel's general-channel variants are scaled to norm 1 and the scale is divided
    out of the set weight in FP64; unscaled, sets with ~17+ jumps reached FP32 subnormals and an
    angle with zero gradient read 1.7e-4). The first angle (un-computed through every later block),
    the second, a middle one and the last (zero gradient: a diagonal rotation before diagonal
    operators and a ZZ observable) meet the 1e-3 bound against the oracle's FP64 finite
    differences."""
    circ = ansatz(n=10, layers=layers, gamma=0.02, p=0.02, seed=300 + layers)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=layers, nsamples=16, total_shots=1600)
    slots = oracle_mod.gate_param_slots(circ)
    pick = [slots[0], slots[1], slots[len(slots) // 2], slots[-1]]
    L, per, gp, gn = run_gpu(P, circ, info, 0, info.count, zz(10), np.asarray(circ.meta["zz_coeffs"]))
    Lr, perr, gpr, gnr, scale, w = run_ref(oracle_mod, circ, info, 0, info.count, zz(10),
                                           np.asarray(circ.meta["zz_coeffs"]), param_slots=pick, noise_slots=[0, 1])
    idx = tuple(np.array(pick).T)
    bound = GRAD_RTOL * np.abs(gpr[idx]) + 1e-4 * max(np.abs(gpr[idx]).max(), 1e-12)
    used = np.abs(gp[idx] - gpr[idx]) / bound
    print(f"depth {layers}: gates {circ.n_gates}, angle-gradient error at most {used.max():.3f} of the bound")
    assert_grad(gp[idx], gpr[idx], f"angles at depth {layers}")
    assert_grad(gn[[0, 1]], gnr[[0, 1]], f"channel strengths at depth {layers}")


def test_full_size_ansatz(P, oracle_mod):
    """The 16-qubit, 8-layer ansatz with 4,096 proportional samples: the whole range runs, and
    single sets of it match the oracle's finite differences."""
    torch = torch_cuda()
    circ = ansatz()
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=2004, nsamples=4096, total_shots=4096)
    coeffs = np.asarray(circ.meta["zz_coeffs"])
    L, per, gp, gn = run_gpu(P, circ, info, 0, info.count, zz(16), coeffs)
    assert np.isfinite(L) and np.all(np.isfinite(per)) and np.all(np.isfinite(gp)) and np.all(np.isfinite(gn))
    w = np.asarray(info.mult, np.float64) / np.sum(info.mult)
    assert abs(L - float((w * per).sum())) <= 1e-9 * max(1.0, abs(L))
    slots = oracle_mod.gate_param_slots(circ)
    pick = [slots[3], slots[200]]
    lens = [len(info.entries(i)) for i in range(info.count)]
    for a in [0, int(np.argmax(lens))]:
        compare(oracle_mod, P, circ, info, a, 1, zz(16), coeffs, param_slots=pick, noise_slots=[0, 1])


def test_autograd_function(P, oracle_mod):
    torch = torch_cuda()
    from paper_2504_16297_gb300.autograd import fixed_set_loss
    circ = grad_circuit(seed=17)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=8, nsamples=80, total_shots=800)
    op = torch.tensor(circ.op_params, dtype=torch.float64, requires_grad=True)
    ch = torch.tensor(circ.ch_params, dtype=torch.float64, requires_grad=True)
    loss = fixed_set_loss(op, ch, P, circ, info, masks=zz(3), coeffs=np.array([0.4, 0.6]))
    (2.0 * loss).backward()
    L, per, gp, gn = run_gpu(P, circ, info, 0, info.count, zz(3), np.array([0.4, 0.6]))
    assert abs(float(loss.detach()) - L) <= 1e-12 * max(1.0, abs(L))
    np.testing.assert_allclose(op.grad.numpy(), 2.0 * gp, rtol=1e-12, atol=0)
    np.testing.assert_allclose(ch.grad.numpy(), 2.0 * gn, rtol=1e-12, atol=0)


def test_empty_range_and_limits(P):
    torch = torch_cuda()
    circ = grad_circuit()
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=1, nsamples=10, total_shots=10)
    L, per, gp, gn = run_gpu(P, circ, info, 0, 0, zz(3), np.array([1.0, 1.0]))
    assert L == 0.0 and np.all(gp == 0) and np.all(gn == 0)
    from paper_2504_16297_gb300.capi import PtsbeError
    big = ansatz(n=17, layers=1)
    cb = P.register(big)
    ib = P.sample_kraus(cb, "proportional", seed=1, nsamples=4, total_shots=4)
    with pytest.raises(PtsbeError):
        run_gpu(P, big, ib, 0, ib.count, zz(17), np.ones(16))
