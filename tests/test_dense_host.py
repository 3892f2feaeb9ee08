"""The dense tile passes on the CPU: the dense planner and the kernel's per-thread code
(tests/dense_host.cpp runs each CTA's threads one after another, phase by phase), compared with
the oracle. States of 13-18 qubits take several 12-qubit tiles per pass, several passes, qubit
layout changes between passes and trailing passes that restore logical order; Kraus entries go in
as override blocks."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from workloads import CircuitBuilder, brickwork, config

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(ROOT, "paper_2504_16297_gb300", "csrc")


@pytest.fixture(scope="module")
def dh():
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libdense_host.so")
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-I", CSRC,
           "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
           os.path.join(HERE, "dense_host.cpp"), os.path.join(CSRC, "dense_plan.cpp"),
           os.path.join(CSRC, "circuit.cpp"), "-o", lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("dense host harness does not build:\n" + r.stderr[-3000:])
    L = C.CDLL(lib)
    L.dh_evolve.restype = C.c_double
    L.dh_bank_stats.restype = C.c_uint64
    return L


def register(dh, circ):
    from paper_2504_16297_gb300 import capi
    n_ops = circ.n_ops
    ops = (capi.ptsbe_op * max(n_ops, 1))()
    oi, op = np.asarray(circ.op_ints), np.asarray(circ.op_params)
    for i in range(n_ops):
        o = ops[i]
        o.kind, o.id, o.n_targets = int(oi[i, 0]), int(oi[i, 1]), int(oi[i, 2])
        o.targets[0], o.targets[1] = int(oi[i, 3]), int(oi[i, 4])
        o.params[0], o.params[1], o.params[2] = (float(x) for x in op[i])
    n_ch = len(circ.ch_params)
    chans = (capi.ptsbe_channel * max(n_ch, 1))()
    keep = []
    for j in range(n_ch):
        kind, arity, nk = (int(x) for x in circ.ch_ints[j])
        c = chans[j]
        c.kind, c.arity, c.n_kraus, c.param = kind, arity, nk, float(circ.ch_params[j])
        off = int(circ.ch_kraus_off[j])
        if off >= 0:
            d = 1 << arity
            arr = np.ascontiguousarray(circ.ch_kraus[off: off + nk * d * d]).view(np.float64).copy()
            keep.append(arr)
            c.kraus = arr.ctypes.data_as(C.POINTER(C.c_double))
    cg = np.ascontiguousarray(np.asarray(circ.custom_gates, np.complex128)).view(np.float64).reshape(-1)
    passes = dh.dh_register(C.c_uint32(circ.n_qubits), ops, C.c_uint64(n_ops), chans, C.c_uint32(n_ch),
                            C.c_void_p(cg.ctypes.data) if cg.size else None,
                            C.c_uint32(int(circ.custom_gates.shape[0])))
    assert passes > 0, f"dense plan failed with status {-passes}"
    return passes


def stats(dh):
    out = (C.c_uint64 * 11)()
    dh.dh_stats(out)
    keys = ["passes", "fixup", "groups", "blocks", "placed", "misplaced", "blocks2", "gates", "staged", "stage_errors",
            "dr"]
    return dict(zip(keys, [int(x) for x in out]))


def evolve(dh, n, entries):
    sites = np.ascontiguousarray([s for s, _ in entries] + [0], np.uint32)
    ks = np.ascontiguousarray([k for _, k in entries] + [0], np.uint8)
    out = np.zeros(1 << n, np.complex64)
    w = dh.dh_evolve(C.c_void_p(sites.ctypes.data), C.c_void_p(ks.ctypes.data), C.c_uint32(len(entries)),
                     C.c_void_p(out.ctypes.data))
    return out, w


def compare(dh, oracle_mod, circ, sets, idxs):
    n = circ.n_qubits
    o = oracle_mod.Oracle(circ)
    worst = 0.0
    for i in idxs:
        ref, rw, rs = o.evolve(sets, i)
        psi, w = evolve(dh, n, sets.entries(i))
        if rs:
            assert w < 1e-6 * sets.q[i] * 1.0001, f"set {i}: null branch gave weight {w}"
            continue
        nrm = np.linalg.norm(psi.astype(np.complex128))
        err = np.linalg.norm(psi / nrm - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, f"set {i}: rel err {err:.3e}"
        assert abs(w - rw) <= 1e-5 * rw, f"set {i}: weight {w} vs {rw}"
        worst = max(worst, err)
    return worst


@pytest.mark.parametrize("n,layers", [(13, 6), (14, 8), (16, 6)])
def test_brickwork_sets_match_oracle(dh, oracle_mod, n, layers):
    circ = brickwork(n, layers, 0.02, 0.03, seed=300 + n)
    passes = register(dh, circ)
    st = stats(dh)
    assert st["misplaced"] == 0 and st["placed"] == circ.n_ops
    assert st["gates"] == circ.n_gates
    assert passes >= 2
    sets = oracle_mod.Oracle(circ).pts_proportional(30, 11, total_shots=300)
    compare(dh, oracle_mod, circ, sets, range(min(sets.count, 8)))
    st = stats(dh)
    assert st["staged"] > 0 and st["stage_errors"] == 0


@pytest.mark.parametrize("n,layers", [(1, 4), (5, 8), (10, 20), (11, 6)])
def test_small_states_run_zero_padded(dh, oracle_mod, n, layers):
    """A state of fewer than 12 qubits is planned as a 12-qubit one whose added qubits carry no
    operation: its amplitudes are the first 2^n of the plan's state, every other amplitude stays an
    exact zero, and sets match the oracle (the 10-qubit, 20-layer case is the 10-qubit workload's
    shape)."""
    dh.dh_pad_errors.restype = C.c_int
    before = dh.dh_pad_errors()
    if n == 1:
        b = CircuitBuilder(1, "one")
        dp = b.channel("DEPOL1", 0.1)
        for _ in range(layers):
            b.gate("U3", [0], (0.3, 0.7, 1.1)); b.noise(dp, [0])
        circ = b.build()
    else:
        circ = brickwork(n, layers, 0.02, 0.03, seed=700 + n)
    register(dh, circ)
    st = stats(dh)
    assert st["misplaced"] == 0 and st["placed"] == circ.n_ops
    sets = oracle_mod.Oracle(circ).pts_proportional(30, 17, total_shots=300)
    compare(dh, oracle_mod, circ, sets, range(min(sets.count, 6)))
    assert dh.dh_pad_errors() == before


def test_deep_brickwork_many_passes(dh, oracle_mod):
    """16 qubits, 30 layers: many passes, the low bits hand over between passes, and the plan ends
    with passes that restore logical order."""
    circ = brickwork(16, 30, 2e-3, 4e-3, seed=901)
    passes = register(dh, circ)
    st = stats(dh)
    assert st["misplaced"] == 0
    assert passes >= 6
    sets = oracle_mod.Oracle(circ).pts_proportional(20, 3, total_shots=100)
    compare(dh, oracle_mod, circ, sets, range(min(sets.count, 4)))


def test_every_gate_and_channel_kind(dh, oracle_mod):
    """Every gate, named and custom channels (damping renormalised at the end), 14 qubits."""
    from test_gpu_parity import _kitchen_sink
    circ = _kitchen_sink(14, seed=14)
    register(dh, circ)
    sets = oracle_mod.Oracle(circ).pts_proportional(40, 3, total_shots=400)
    compare(dh, oracle_mod, circ, sets, range(min(sets.count, 10)))


def test_errors_inside_fused_blocks(dh, oracle_mod):
    """Targeted sets with one, two and three entries inside the same fused block and in blocks of
    different passes: each override block carries all of the set's operators in it."""
    circ = brickwork(14, 6, 0.05, 0.05, seed=17)
    register(dh, circ)
    S = circ.n_sites
    targeted = [[], [(0, 1)], [(0, 2), (1, 3)], [(14, 5), (15, 1), (16, 3)], [(3, 1), (S // 2, 2), (S - 1, 3)],
                [(S - 2, 1), (S - 1, 15)]]
    o = oracle_mod.Oracle(circ)
    sets = o.pts_targeted(targeted, shots=np.full(len(targeted), 10, np.uint64))
    compare(dh, oracle_mod, circ, sets, range(sets.count))


def test_amplitude_damping_null_branch(dh, oracle_mod):
    """A damping jump on a qubit with no |1> population is impossible: weight 0."""
    b = CircuitBuilder(13)
    ad = b.channel("AMPDAMP", 0.3)
    for q in range(13):
        b.noise(ad, [q])
        b.gate("H", [q])
        b.noise(ad, [q])
    circ = b.build()
    register(dh, circ)
    psi, w = evolve(dh, 13, [(0, 1)])
    assert w == 0.0 and not np.any(psi)
    # the jump after H has probability gamma/2; every later no-jump operator on |+> keeps (2 - gamma)/2
    o = oracle_mod.Oracle(circ)
    sets = o.pts_targeted([[(0, 1)], [(1, 1)], [(1, 1), (25, 1)]], shots=np.full(3, 10, np.uint64))
    compare(dh, oracle_mod, circ, sets, range(3))
    psi, w = evolve(dh, 13, [(1, 1)])
    assert abs(w - 0.15 * 0.85 ** 12) < 1e-6


def test_thirty_qubit_plan(dh):
    """The 30-qubit, 60-layer brickwork: every operation placed once, a pass count near what the
    light cone of a 12-qubit tile allows, and warp lanes that meet distinct shared-memory banks."""
    c = config(3)
    circ = c["circuit"]
    passes = register(dh, circ)
    st = stats(dh)
    assert st["misplaced"] == 0 and st["placed"] == circ.n_ops
    assert st["gates"] == circ.n_gates
    assert passes <= 40
    assert st["staged"] == passes - st["fixup"] and st["stage_errors"] == 0
    # every block but the last on each qubit takes the diagonal-times-real form (U3 = P R_y P)
    assert st["dr"] >= 0.95 * st["blocks"]
    mean = C.c_double()
    bad = dh.dh_bank_stats(C.byref(mean))
    assert mean.value >= 14.0, (bad, mean.value)
