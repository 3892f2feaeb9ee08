"""Host logic of libptsbe on the CPU (no GPU needed): the C ABI loads and exports every symbol
the header declares, pre-trajectory sampling (Algorithm 2, Sec. 3.1) is bit-identical to the
oracle in every mode, and malformed input is rejected with the documented status."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from workloads import CircuitBuilder, config, GATE

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_2504_16297_gb300 import build, capi
    build()
    return capi


@pytest.fixture(scope="session")
def host(lib):
    from paper_2504_16297_gb300.runtime import Ptsbe
    return Ptsbe(device=-1)


def test_library_exports_every_declared_symbol(lib):
    header = open(os.path.join(ROOT, "include", "ptsbe.h")).read()
    names = re.findall(r"PTSBE_API\s+[\w\s\*]*?\b(ptsbe_\w+)\s*\(", header)
    assert len(names) >= 14
    so = C.CDLL(lib.lib_path())
    for n in names:
        assert hasattr(so, n), n
    assert sorted(names) == sorted(lib.declared_symbols())


def _assert_same_sets(got, want):
    assert got.count == want.count
    assert np.array_equal(got.offsets, want.offsets)
    assert np.array_equal(got.sites, want.sites)
    assert np.array_equal(got.kidx, want.kidx)
    assert np.array_equal(got.mult, want.mult)
    assert np.array_equal(got.q.view(np.uint64), want.q.view(np.uint64))      # bit-exact FP64
    assert np.array_equal(got.shots, want.shots)


@pytest.mark.parametrize("cfg", [0, 3, 4])
def test_proportional_pts_bit_exact_vs_oracle(host, oracle_mod, cfg):
    c = config(cfg, small=(cfg == 3))
    circ = c["circuit"]
    cid = host.register(circ)
    ns = min(c["nsamples"], 2000)
    total = c["total_shots"] or 0
    got = host.sample_kraus(cid, "proportional", seed=c["seed"], nsamples=ns, total_shots=total)
    want = oracle_mod.Oracle(circ).pts_proportional(ns, c["seed"], total_shots=total)
    _assert_same_sets(got, want)
    assert np.array_equal(got.shot_offsets, np.concatenate([[0], np.cumsum(want.shots)]).astype(np.uint64))


def test_topk_syndrome17_bit_exact_vs_oracle(host, oracle_mod):
    c = config(1)
    cid = host.register(c["circuit"])
    got = host.sample_kraus(cid, "topk", k=c["k"], total_shots=c["total_shots"])
    want = oracle_mod.Oracle(c["circuit"]).pts_topk(c["k"], c["total_shots"])
    _assert_same_sets(got, want)


def _ratio_circuit():
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


@pytest.mark.parametrize("K", [1, 5, 64, 777, 5000])
def test_topk_small_bit_exact(host, oracle_mod, K):
    circ = _ratio_circuit()
    cid = host.register(circ)
    got = host.sample_kraus(cid, "topk", k=K, total_shots=123457)
    want = oracle_mod.Oracle(circ).pts_topk(K, 123457)
    _assert_same_sets(got, want)


@pytest.mark.parametrize("pmin,pmax", [(1e-4, 1.0), (1e-6, 1e-3), (3e-5, 2e-4)])
def test_band_bit_exact(host, oracle_mod, pmin, pmax):
    circ = _ratio_circuit()
    cid = host.register(circ)
    got = host.sample_kraus(cid, "band", p_min=pmin, p_max=pmax, total_shots=99991)
    want = oracle_mod.Oracle(circ).pts_band(pmin, pmax, 99991)
    _assert_same_sets(got, want)


def test_literal_bit_exact(host, oracle_mod):
    circ = config(0)["circuit"]
    cid = host.register(circ)
    got = host.sample_kraus(cid, "literal", seed=77, nsamples=700, shots_per_set=33)
    want = oracle_mod.Oracle(circ).pts_literal(700, 77, 33)
    _assert_same_sets(got, want)


def test_targeted_bit_exact(host, oracle_mod):
    circ = config(0)["circuit"]
    cid = host.register(circ)
    sets = [[(3, 1), (10, 2)], [], [(0, 3)], [(3, 1), (10, 2)], [(289, 15)], [(5, 2), (6, 1), (200, 7)]]
    got = host.sample_kraus(cid, "targeted", targeted=sets, total_shots=1001)
    want = oracle_mod.Oracle(circ).pts_targeted(sets, total_shots=1001)
    _assert_same_sets(got, want)
    shots = np.arange(1, 7, dtype=np.uint64) * 10
    got = host.sample_kraus(cid, "targeted", targeted=sets, targeted_shots=shots)
    want = oracle_mod.Oracle(circ).pts_targeted(sets, shots=shots)
    _assert_same_sets(got, want)


def test_rejects_malformed_input(host, lib):
    from paper_2504_16297_gb300.capi import PtsbeError
    # not trace preserving
    b = CircuitBuilder(1)
    bad = b.channel("CUSTOM", kraus=np.array([[[1, 0], [0, 1]], [[0, 0.5], [0, 0]]], complex))
    b.gate("H", [0]); b.noise(bad, [0])
    with pytest.raises(PtsbeError) as e:
        host.register(b.build())
    assert e.value.status == 2
    # qubit out of range
    b = CircuitBuilder(2)
    b.gate("H", [0])
    circ = b.build()
    circ.op_ints[0, 3] = 5
    with pytest.raises(PtsbeError) as e:
        host.register(circ)
    assert e.value.status == 1
    # top-k needs k = 0 to be the most likely branch
    b = CircuitBuilder(1)
    ch = b.channel("BITFLIP", 0.6)
    b.gate("H", [0]); b.noise(ch, [0])
    cid = host.register(b.build())
    with pytest.raises(PtsbeError) as e:
        host.sample_kraus(cid, "topk", k=3, total_shots=10)
    assert e.value.status == 7
    # targeted entries must be valid
    cid = host.register(config(0)["circuit"])
    for badset in ([[(5, 0)]], [[(5, 1), (5, 2)]], [[(4000, 1)]], [[(7, 1), (3, 1)]]):
        with pytest.raises(PtsbeError) as e:
            host.sample_kraus(cid, "targeted", targeted=badset, total_shots=10)
        assert e.value.status == 1
    # device entry points on a host-only context
    info = host.sample_kraus(cid, "proportional", seed=1, nsamples=10, total_shots=10)
    with pytest.raises(PtsbeError) as e:
        lib.ptsbe_evolve_batch(host.ctx, info.set_id, 0, 1, 16, None, None, 0)
    assert e.value.status == 8


def test_circuit_info(host):
    for i in (0, 1, 3, 4):
        circ = config(i)["circuit"]
        cid = host.register(circ)
        nq, ns, ng = host.circuit_info(cid)
        assert (nq, ns, ng) == (circ.n_qubits, circ.n_sites, circ.n_gates)


PREDICATES = [
    dict(max_errors=1),
    dict(max_errors=2, include_empty=True),
    dict(max_errors=2, qubit_mask=0b0000110011, kraus_mask=0b0110),
    dict(max_errors=3, gate_mask=1 << GATE["CX"], site_lo=20, site_hi=90, weight_parity=1),
    dict(max_errors=2, gate_mask=1 << GATE["U3"], kraus_mask=1 << 3, weight_parity=2, include_empty=True),
]


@pytest.mark.parametrize("pred", PREDICATES)
def test_predicate_targeted_bit_exact(host, oracle_mod, pred):
    """Targeted error sets by rule (NEXT-4): the library's enumeration equals the oracle's plain
    enumeration from the definition (sets in canonical order, q_alpha and shots bit-exact)."""
    circ = config(0)["circuit"]
    cid = host.register(circ)
    got = host.sample_kraus(cid, "predicate", total_shots=123457, **pred)
    sets = oracle_mod.predicate_sets(circ, **pred)
    want = oracle_mod.Oracle(circ).pts_targeted(sets, total_shots=123457)
    assert got.count == len(sets) > 0
    _assert_same_sets(got, want)


def test_predicate_refuses_too_many_sets(host):
    from paper_2504_16297_gb300.capi import PtsbeError
    circ = config(0)["circuit"]
    cid = host.register(circ)
    with pytest.raises(PtsbeError) as e:
        host.sample_kraus(cid, "predicate", total_shots=10, max_errors=3, max_sets=1000)
    assert e.value.status == 7


def test_options_validate_values(host):
    """Options are host-side state: accepted values take, others are refused with ERR_INVALID."""
    from paper_2504_16297_gb300 import capi
    for spw in (0, 4, 8, 16):
        host.set_program_sets_per_warp(spw)
    for bad in (1, 2, 5, 32, -4):
        with pytest.raises(capi.PtsbeError) as e:
            host.set_program_sets_per_warp(bad)
        assert e.value.status == 1
    host.set_light_shots(0)
    with pytest.raises(capi.PtsbeError):
        host.set_light_shots(-1)
    with pytest.raises(capi.PtsbeError):
        capi.ptsbe_set_option(host.ctx, 99, 0)
    for pct in (0, 50, 100):
        host.set_split_fill(pct)
    for bad in (101, -1):
        with pytest.raises(capi.PtsbeError):
            capi.ptsbe_set_option(host.ctx, capi.PTSBE_OPT_SPLIT_FILL, bad)
    for bits in (0, 9, 14):
        host.set_pershot_tile_bits(bits)
    for bad in (8, 15, -1):
        with pytest.raises(capi.PtsbeError):
            host.set_pershot_tile_bits(bad)
    host.set_prepass_ahead(False)
    host.set_prepass_ahead(True)
    for bad in (2, -1):
        with pytest.raises(capi.PtsbeError):
            capi.ptsbe_set_option(host.ctx, capi.PTSBE_OPT_PREPASS_AHEAD, bad)


@pytest.mark.parametrize("n", [2, 5, 9])
def test_register_every_op_and_channel_kind(host, oracle_mod, n):
    """Every gate kind, custom gates and custom Kraus channels through the binding's op and channel
    marshalling: the registered circuit has the op and site counts it was given, and proportional
    PTS on it is bit-identical to the oracle's (the channels' probabilities come from the
    marshalled Kraus operators)."""
    import test_gpu_parity
    circ = test_gpu_parity._kitchen_sink(n, n)
    cid = host.register(circ)
    nq, n_sites, n_gates = host.circuit_info(cid)
    assert (nq, n_sites, n_gates) == (n, circ.n_sites, circ.n_ops - circ.n_sites)
    info = host.sample_kraus(cid, "proportional", seed=17, nsamples=400, total_shots=4000)
    ref = oracle_mod.Oracle(circ).pts_proportional(400, 17, total_shots=4000)
    assert info.count == ref.count
    for i in range(info.count):
        assert info.entries(i) == ref.entries(i), i
    np.testing.assert_array_equal(np.asarray(info.shots, np.uint64), np.asarray(ref.shots, np.uint64))
    host.release_set(info)
    host.release_circuit(cid)


def test_backward_conditioning_checkpoints(host):
    """The backward plan stores the state where un-computing through the blocks since the last
    stored copy would multiply rounding by more than 2^6 (the product of the blocks' condition
    numbers): none for unitary circuits or the 16-qubit ansatz with gamma = 1e-3 (product about
    2^0.37), and about one per 2^6 for a deep damped circuit (32 layers, gamma = 0.02: 1,216
    damping sites of 2^0.0146 each, about 2^17.7 in all)."""
    import math
    from workloads import ansatz, brickwork
    uni = host.register(brickwork(10, 8, 0.0, 0.0, seed=3))
    assert host.backward_plan_info(uni)["conditioning_checkpoints"] == 0
    assert host.backward_plan_info(host.register(ansatz()))["conditioning_checkpoints"] == 0
    deep = ansatz(n=10, layers=32, gamma=0.02, p=0.02, seed=332)
    total = 1216 * 0.5 * math.log2(1.0 / 0.98)
    ck = host.backward_plan_info(host.register(deep))["conditioning_checkpoints"]
    assert math.floor(total / 6.0) - 1 <= ck <= math.floor(total / 6.0)

