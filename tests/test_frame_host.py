"""The deferred-frame evolution on the CPU: frame-aware plan, program builder and tile steps of the
default evolve kernel, compiled with g++ from the library sources (tests/frame_host.cpp runs each
CTA's threads one after another) and compared with the oracle. Small tiles force multi-stage plans
(permuted layouts between stages, logical-order last stage, prefix reuse across stages)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from workloads import CircuitBuilder, brickwork, syndrome17

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(ROOT, "paper_2504_16297_gb300", "csrc")


@pytest.fixture(scope="module")
def fh():
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libframe_host.so")
    cuda_inc = "/usr/local/cuda/include"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-I", CSRC,
           "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, os.path.join(HERE, "frame_host.cpp"),
           os.path.join(CSRC, "circuit.cpp"), "-o", lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("frame host harness does not build:\n" + r.stderr[-3000:])
    return C.CDLL(lib)


def _register(fh, circ, tile_bits):
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
    stages = fh.fh_register(C.c_uint32(circ.n_qubits), ops, C.c_uint64(n_ops), chans, C.c_uint32(n_ch),
                            C.c_void_p(cg.ctypes.data) if cg.size else None,
                            C.c_uint32(int(circ.custom_gates.shape[0])), C.c_int(tile_bits))
    assert stages > 0, f"frame plan failed with status {-stages}"
    return stages


def _compare(fh, oracle_mod, circ, sets, tile_bits, reuse, check=None):
    stages = _register(fh, circ, tile_bits)
    n, cnt = circ.n_qubits, sets.count
    st = np.zeros((cnt, 1 << n), np.complex64)
    w = np.zeros(cnt)
    s = np.zeros(cnt, np.uint8)
    off = np.ascontiguousarray(sets.offsets, np.uint32)
    site = np.ascontiguousarray(np.append(sets.sites, 0), np.uint32)
    kk = np.ascontiguousarray(np.append(sets.kidx, 0), np.uint8)
    q = np.ascontiguousarray(sets.q)
    P = lambda a: C.c_void_p(a.ctypes.data)
    assert fh.fh_evolve(C.c_uint32(cnt), P(off), P(site), P(kk), P(q), C.c_int(reuse), P(st), P(w), P(s)) == 0
    o = oracle_mod.Oracle(circ)
    for i in (range(cnt) if check is None else check):
        ref, rw, rs = o.evolve(sets, i)
        assert s[i] == rs, f"set {i}: status {s[i]} vs {rs}"
        if rs:
            assert np.all(st[i] == 0)
            continue
        assert np.linalg.norm(st[i] - ref) <= 1e-5 * np.linalg.norm(ref), f"set {i}"
        assert abs(w[i] - rw) <= 1e-5 * rw, f"set {i}: weight {w[i]} vs {rw}"
    return stages


@pytest.mark.parametrize("tile_bits,reuse", [(14, 1), (8, 0), (8, 1), (6, 1)])
def test_brickwork_one_and_several_stages(fh, oracle_mod, tile_bits, reuse):
    circ = brickwork(10, 3, 0.05, 0.08, seed=50)
    sets = oracle_mod.Oracle(circ).pts_proportional(40, 7, total_shots=1000)
    stages = _compare(fh, oracle_mod, circ, sets, tile_bits, reuse)
    assert (stages == 1) == (tile_bits >= 10)


def test_deep_cx_network_restarts_the_frame(fh, oracle_mod):
    """12 qubits, 10 brickwork layers on 7-bit tiles: CX chains spread the physical directions
    of later mixes wider than a tile, so the plan goes back to logical order mid-circuit."""
    circ = brickwork(12, 10, 0.01, 0.02, seed=77)
    sets = oracle_mod.Oracle(circ).pts_proportional(12, 5, total_shots=100)
    stages = _compare(fh, oracle_mod, circ, sets, 7, 1, check=range(min(sets.count, 6)))
    assert stages >= 3


def _order_stats(fh):
    c, v = C.c_int(0), C.c_int(0)
    fh.fh_order_stats(C.byref(c), C.byref(v))
    return c.value, v.value


def test_syndrome_plan_and_states(fh, oracle_mod):
    """One syndrome round on 17 qubits: the CX-heavy circuit fits one frame stage; one CTA per
    state holds every nonzero amplitude and scatters them in logical order (sparse final)."""
    circ = syndrome17(rounds=1)
    sets = oracle_mod.Oracle(circ).pts_topk(24, 1000)
    stages = _compare(fh, oracle_mod, circ, sets, 14, 1, check=range(0, 24, 3))
    assert stages == 1


def test_syndrome_support_in_low_bits(fh, oracle_mod):
    """The 3-round syndrome circuit: the span of its mixing directions has dimension 8, so the
    stage is entered in a layout that puts it on the low 8 tile bits and every nonzero amplitude
    lives below tile address 256 (the small-buffer kernel); the harness fills the rest of the tile
    with a sentinel and fails if any step touches it."""
    circ = syndrome17(rounds=3)
    sets = oracle_mod.Oracle(circ).pts_topk(300, 3000)
    c0, v0 = _order_stats(fh)
    stages = _compare(fh, oracle_mod, circ, sets, 14, 1, check=range(0, 300, 23))
    assert stages == 1
    assert fh.fh_sparse_bits() == 8
    # fused sampling: the order mask ranks every state's 256-entry support increasingly
    c1, v1 = _order_stats(fh)
    assert c1 - c0 >= 300 and v1 == v0


@pytest.mark.parametrize("n,tile_bits", [(10, 8), (12, 9)])
def test_one_stage_multi_tile_sparse_final(fh, oracle_mod, n, tile_bits):
    """A circuit whose mixes fit one tile on a multi-tile state: the one-stage plan with the
    sparse final store (zero-fill, norm and scatter from the tile holding index 0)."""
    b = CircuitBuilder(n)
    ad = b.channel("AMPDAMP", 0.05)
    dp = b.channel("DEPOL1", 0.03)
    for q in range(3):
        b.gate("H", [q]); b.noise(dp, [q])
    for r in range(2):
        for q in range(3, n):
            b.gate("CX", [q % 3, q]); b.noise(ad, [q]); b.noise(dp, [q % 3])
        b.gate("RZ", [1], (0.3 + r,))
        b.gate("H", [2]); b.noise(ad, [2])
    circ = b.build()
    sets = oracle_mod.Oracle(circ).pts_proportional(30, 11, total_shots=300)
    c0, v0 = _order_stats(fh)
    stages = _compare(fh, oracle_mod, circ, sets, tile_bits, 1)
    assert stages == 1
    c1, v1 = _order_stats(fh)
    assert c1 > c0 and v1 == v0


def _sink(n, seed):
    import test_gpu_parity
    return test_gpu_parity._kitchen_sink(n, seed)


@pytest.mark.parametrize("n,tile_bits", [(2, 14), (5, 14), (9, 8), (12, 9)])
def test_every_gate_and_channel_kind(fh, oracle_mod, n, tile_bits):
    """X/Y/Z/H/S/T, U3, RX/RY/RZ, CX/CZ/SWAP, custom 1- and 2-qubit gates, depolarising,
    damping, bit/phase flips and custom channels (general Kraus operators, fused blocks that are
    not monomial)."""
    circ = _sink(n, n)
    sets = oracle_mod.Oracle(circ).pts_proportional(30, 3, total_shots=300)
    _compare(fh, oracle_mod, circ, sets, tile_bits, 1, check=range(min(sets.count, 8)))


def test_null_branch_and_single_qubit(fh, oracle_mod):
    b = CircuitBuilder(1)
    ad = b.channel("AMPDAMP", 0.4)
    b.gate("U3", [0], (1.0, 0.2, 0.3)); b.noise(ad, [0]); b.gate("H", [0]); b.noise(ad, [0])
    circ = b.build()
    sets = oracle_mod.Oracle(circ).pts_targeted([[], [(0, 1)], [(1, 1)], [(0, 1), (1, 1)]],
                                                np.array([1000] * 4, np.uint64))
    _compare(fh, oracle_mod, circ, sets, 14, 1)
    b = CircuitBuilder(12)
    ad = b.channel("AMPDAMP", 0.01)
    for q in range(12):
        if q != 3:
            b.gate("H", [q])
    b.noise(ad, [3]); b.noise(ad, [5])
    circ = b.build()
    sets = oracle_mod.Oracle(circ).pts_targeted([[], [(0, 1)], [(1, 1)]], np.array([50, 60, 70], np.uint64))
    _compare(fh, oracle_mod, circ, sets, 8, 1)


def test_support_order_mask_random(fh):
    """The rank rule of fused sampling on 3,000 random supports: up to 10 coset generators of a
    14-bit tile under random invertible logical maps and offsets, 4 to 20 qubits. Independent
    generators: the bits of each member's logical index at the order mask rank the 2^k members
    0 .. 2^k - 1 in increasing order (brute force: sorted list). Dependent ones: the mask has fewer
    than k bits, which the kernel treats as a fault."""
    fh.fh_order_selftest.restype = C.c_int
    assert fh.fh_order_selftest(C.c_uint64(12345), C.c_int(3000)) == 0
