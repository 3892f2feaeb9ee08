"""Parity of the CUDA path with the CPU oracle (-m gpu).

Batched preparation (Sec. 3) per Kraus set: amplitudes within 1e-5 relative 2-norm (complex64
vs complex128), weights within 1e-5, null flags identical. Shots (Sec. 3): bit-identical to the
oracle fed the GPU's own state, except where the uniform sits within 1e-6 of a CDF boundary.
Sizes span one tile, several tiles / cluster slices, ragged tails and the global-memory path.
"""
import math

import numpy as np
import pytest

from gpu_common import check_shots, compare_state, evolve_gpu, gpu_ctx, torch_cuda
from workloads import CircuitBuilder, brickwork, config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["frame", "sweep", "registers"])
def P(request):
    ctx = gpu_ctx()
    ctx.set_evolve_kernel(request.param)
    return ctx


def _evolve_and_compare(P, oracle_mod, circ, info, idxs, prefix_reuse, first=0, count=None):
    count = info.count - first if count is None else count
    st, w, s = evolve_gpu(P, info, first, count, circ.n_qubits, prefix_reuse)
    o = oracle_mod.Oracle(circ)
    ref_sets = o.pts_targeted([info.entries(i) for i in range(info.count)],
                              shots=np.asarray(info.shots, np.uint64))
    st_h, w_h, s_h = st.cpu().numpy(), w.cpu().numpy(), s.cpu().numpy()
    worst = 0.0
    for i in idxs:
        psi, wr, sr = o.evolve(ref_sets, first + i)
        worst = max(worst, compare_state(st_h[i], psi, w_h[i], wr, s_h[i], sr, f"set {first + i}"))
    return st, s, worst


@pytest.mark.parametrize("reuse", [False, True])
def test_brickwork10_all_sets(P, oracle_mod, reuse):
    """Workload 0 (10 qubits, one tile per state): every one of the ~620 sets."""
    c = config(0)
    circ = c["circuit"]
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=c["seed"], nsamples=c["nsamples"], total_shots=c["total_shots"])
    assert 500 < info.count < 750
    _evolve_and_compare(P, oracle_mod, circ, info, range(info.count), reuse)


@pytest.mark.parametrize("n,layers", [(15, 4), (16, 3), (17, 2)])
@pytest.mark.parametrize("reuse", [False, True])
def test_multi_tile_brickwork(P, oracle_mod, n, layers, reuse):
    """Several tiles per state (2, 4, 8 tiles of 2^14), staged passes through HBM."""
    circ = brickwork(n, layers, 0.02, 0.03, seed=50 + n)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=7, nsamples=60, total_shots=6000)
    idxs = sorted(set([0, 1, info.count // 2, info.count - 1]))
    _evolve_and_compare(P, oracle_mod, circ, info, idxs, reuse)


def test_syndrome_damping_subrange(P, oracle_mod):
    """General (non-mixture) damping channel, 17 qubits, a ragged sub-range of the sets."""
    c = config(1, small=True)
    circ = c["circuit"]
    cid = P.register(circ)
    info = P.sample_kraus(cid, "topk", k=c["k"], total_shots=c["total_shots"])
    first, count = 3, 37
    _evolve_and_compare(P, oracle_mod, circ, info, [0, 1, 17, 36], True, first=first, count=count)


def _kitchen_sink(n, seed):
    rng = np.random.default_rng(seed)
    from test_oracle_pins import random_channel, random_unitary
    b = CircuitBuilder(n, f"sink{n}")
    d1 = b.channel("DEPOL1", 0.05)
    d2 = b.channel("DEPOL2", 0.08)
    ad = b.channel("AMPDAMP", 0.3)
    bf = b.channel("BITFLIP", 0.1)
    pf = b.channel("PHASEFLIP", 0.15)
    cu1 = b.channel("CUSTOM", kraus=random_channel(rng, 2, 3))
    cu2 = b.channel("CUSTOM", kraus=random_channel(rng, 4, 2))
    names1 = ["X", "Y", "Z", "H", "S", "SDG", "T", "TDG"]
    for layer in range(3):
        for q in range(n):
            g = names1[(q + layer) % len(names1)]
            b.gate(g, [q])
            b.gate("U3", [q], rng.uniform(0, 2 * math.pi, 3))
            b.noise([d1, ad, bf, pf, cu1][(q + layer) % 5], [q])
        for q in range(0, n - 1, 2):
            a, t = (q + layer) % n, (q + layer + 1 + layer) % n
            if a == t:
                continue
            b.gate(["CX", "CZ", "SWAP"][(q + layer) % 3], [a, t])
            b.noise(d2 if q % 4 == 0 else cu2, [a, t])
        b.gate("RX", [layer % n], (0.3 + layer,))
        b.gate("RY", [(layer + 1) % n], (1.1,))
        b.gate("RZ", [(layer + 2) % n], (2.2,))
        if n >= 2:
            b.gate("U2", [n - 1, 0], matrix=random_unitary(rng, 4))
        b.gate("U1", [n // 2], matrix=random_unitary(rng, 2))
    return b.build()


@pytest.mark.parametrize("n", [2, 3, 5, 9, 14, 15, 18])
def test_all_gate_and_channel_kinds(P, oracle_mod, n):
    circ = _kitchen_sink(n, seed=n)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=3, nsamples=40, total_shots=400)
    _evolve_and_compare(P, oracle_mod, circ, info, range(min(info.count, 12)), True)


def test_single_qubit_and_empty_range(P, oracle_mod):
    torch = torch_cuda()
    b = CircuitBuilder(1)
    ad = b.channel("AMPDAMP", 0.4)
    b.gate("U3", [0], (1.0, 0.2, 0.3)); b.noise(ad, [0]); b.gate("H", [0]); b.noise(ad, [0])
    circ = b.build()
    cid = P.register(circ)
    info = P.sample_kraus(cid, "targeted", targeted=[[], [(0, 1)], [(1, 1)], [(0, 1), (1, 1)]],
                          targeted_shots=np.array([1000, 1000, 1000, 1000], np.uint64))
    _evolve_and_compare(P, oracle_mod, circ, info, range(4), True)
    st = torch.zeros((1, 2), dtype=torch.complex64, device="cuda")
    P.evolve(info, 2, 0, st)           # empty range is a no-op
    bits = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.sample(info, 0, 0, st, None, 1, bits)
    P.synchronize()


def test_null_branch_zeroed_and_sentinel_shots(P, oracle_mod):
    torch = torch_cuda()
    b = CircuitBuilder(16)
    ad = b.channel("AMPDAMP", 0.01)
    for q in range(16):
        b.gate("H", [q]) if q != 3 else None
    b.noise(ad, [3])                 # qubit 3 stays |0>: damping's K1 annihilates the state
    b.noise(ad, [5])
    circ = b.build()
    cid = P.register(circ)
    info = P.sample_kraus(cid, "targeted", targeted=[[], [(0, 1)], [(1, 1)]],
                          targeted_shots=np.array([50, 60, 70], np.uint64))
    st, s, _ = _evolve_and_compare(P, oracle_mod, circ, info, range(3), False)
    assert s.cpu().tolist() == [0, 1, 0]
    bits = torch.zeros(180, dtype=torch.int32, device="cuda")
    P.sample(info, 0, 3, st, s, 5, bits)
    torch.cuda.synchronize()
    b_h = bits.cpu().numpy().view(np.uint32)
    assert np.all(b_h[50:110] == 0xFFFFFFFF)
    assert np.all(b_h[:50] < (1 << 16)) and np.all(b_h[110:] < (1 << 16))


@pytest.mark.parametrize("n", [4, 10, 14, 15, 16, 17, 18, 19])
def test_sampler_bit_exact(P, oracle_mod, n):
    """Single-CTA (n <= 14), cluster of 2/4/8 CTAs (15-17), global CDF (18+)."""
    torch = torch_cuda()
    circ = brickwork(n, 2, 0.05, 0.05, seed=n)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=11, nsamples=40, total_shots=30000)
    count = min(info.count, 6)
    st, w, s = evolve_gpu(P, info, 0, count, n)
    total = int(info.shot_offsets[count])
    bits = torch.zeros(total, dtype=torch.int32, device="cuda")
    P.sample(info, 0, count, st, s, 1234, bits)
    torch.cuda.synchronize()
    b_h = bits.cpu().numpy().view(np.uint32)
    st_h = st.cpu().numpy()
    for a in range(count):
        o0, o1 = int(info.shot_offsets[a]), int(info.shot_offsets[a + 1])
        check_shots(b_h[o0:o1], st_h[a], 1234, a, 0, oracle_mod, n)


def test_sampler_histogram_chi_square(P, oracle_mod):
    from scipy import stats
    torch = torch_cuda()
    n = 12
    circ = brickwork(n, 3, 0.01, 0.01, seed=9)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "targeted", targeted=[[]], targeted_shots=np.array([400000], np.uint64))
    st, w, s = evolve_gpu(P, info, 0, 1, n)
    bits = torch.zeros(400000, dtype=torch.int32, device="cuda")
    P.sample(info, 0, 1, st, s, 99, bits)
    torch.cuda.synchronize()
    counts = np.bincount(bits.cpu().numpy().astype(np.int64), minlength=1 << n).astype(float)
    psi, _, _ = oracle_mod.Oracle(circ).evolve(oracle_mod.Oracle(circ).pts_targeted([[]], shots=np.array([1], np.uint64)), 0)
    p = np.abs(psi) ** 2
    exp = p * counts.sum()
    big = exp >= 5
    o2 = np.append(counts[big], counts[~big].sum()); e2 = np.append(exp[big], exp[~big].sum())
    chi = ((o2 - e2) ** 2 / e2).sum()
    assert stats.chi2.sf(chi, len(o2) - 1) > 1e-3


def test_sampler_capacity_and_alignment_errors(P):
    torch = torch_cuda()
    from paper_2504_16297_gb300.capi import PtsbeError
    circ = brickwork(6, 2, 0.05, 0.05, seed=1)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=1, nsamples=10, total_shots=100)
    st, w, s = evolve_gpu(P, info, 0, info.count, 6)
    bits = torch.zeros(99, dtype=torch.int32, device="cuda")
    with pytest.raises(PtsbeError) as e:
        P.sample(info, 0, info.count, st, s, 1, bits)
    assert e.value.status == 6
    raw = torch.zeros(2 * 64 + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(PtsbeError) as e:
        from paper_2504_16297_gb300 import capi
        capi.ptsbe_evolve_batch(P.ctx, info.set_id, 0, 1, raw.data_ptr() + 4, None, None, 0)
    assert e.value.status == 1
    with pytest.raises(PtsbeError) as e:
        P.evolve(info, info.count, 1, st)
    assert e.value.status == 1


@pytest.mark.parametrize("n", [15, 17, 20])
def test_sampler_light_states_bit_exact(P, oracle_mod, n):
    """States with few shots (one CTA per state, slices rebuilt only where shots land) next to a
    heavy state (cluster or global path) in the same call."""
    torch = torch_cuda()
    circ = brickwork(n, 2, 0.05, 0.05, seed=70 + n)
    cid = P.register(circ)
    sets = [[], [(0, 1)], [(1, 2)], [(2, 3)], [(3, 1), (5, 2)]]
    shots = np.array([3000, 1, 37, 512, 200], np.uint64)
    info = P.sample_kraus(cid, "targeted", targeted=sets, targeted_shots=shots)
    count = info.count
    st, w, s = evolve_gpu(P, info, 0, count, n)
    total = int(info.shot_offsets[count])
    bits = torch.zeros(total, dtype=torch.int32, device="cuda")
    P.sample(info, 0, count, st, s, 4242, bits)
    torch.cuda.synchronize()
    b_h = bits.cpu().numpy().view(np.uint32)
    st_h = st.cpu().numpy()
    for a in range(count):
        o0, o1 = int(info.shot_offsets[a]), int(info.shot_offsets[a + 1])
        check_shots(b_h[o0:o1], st_h[a], 4242, a, 0, oracle_mod, n)


def test_autotune_keeps_results(oracle_mod):
    """The autotuner times every evolve kernel and sampler shot limit, keeps the fastest, and the
    tuned context still matches the oracle (states) and gives the same shots as before tuning (the
    shot limit changes no shot)."""
    torch = torch_cuda()
    P = gpu_ctx()
    from workloads import syndrome17
    circ = syndrome17(rounds=1)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "topk", k=60, total_shots=200000)
    n = circ.n_qubits
    st = torch.empty((info.count, 1 << n), dtype=torch.complex64, device="cuda")
    w = torch.empty(info.count, dtype=torch.float64, device="cuda")
    s = torch.empty(info.count, dtype=torch.uint8, device="cuda")
    bits = torch.empty(info.total_shots, dtype=torch.int32, device="cuda")
    P.evolve(info, 0, info.count, st, w, s, prefix_reuse=True)
    P.sample(info, 0, info.count, st, s, 77, bits)
    torch.cuda.synchronize()
    before = bits.cpu().numpy().copy()
    res = P.autotune(info, 0, info.count, st, w, s, 77, bits, reps=1)
    assert res["evolve_kernel"] in ("frame", "sweep", "registers", "dense")
    assert res["light_shots"] in res["sample_ms"]
    assert all(v > 0 for v in res["evolve_ms"].values()) and all(v > 0 for v in res["sample_ms"].values())
    st2, w2, s2 = evolve_gpu(P, info, 0, info.count, n, True)
    o = oracle_mod.Oracle(circ)
    ref = o.pts_targeted([info.entries(i) for i in range(info.count)], shots=np.asarray(info.shots, np.uint64))
    for i in range(0, info.count, 7):
        psi, wr, sr = o.evolve(ref, i)
        compare_state(st2.cpu().numpy()[i], psi, float(w2.cpu()[i]), wr, int(s2.cpu()[i]), sr, f"set {i}")
    if res["evolve_kernel"] == "frame":
        P.sample(info, 0, info.count, st2, s2, 77, bits)
        torch.cuda.synchronize()
        assert np.array_equal(bits.cpu().numpy(), before)


@pytest.mark.parametrize("which", ["syndrome", "small"])
def test_unique_shot_statistic(oracle_mod, which):
    """Distinct outcomes per set (the unique-shot statistic of Sec. 4) against numpy's count of
    the same shots; the null-branch sentinel is not an outcome."""
    torch = torch_cuda()
    P = gpu_ctx()
    if which == "syndrome":
        from workloads import syndrome17
        circ = syndrome17(rounds=1)
        info = P.sample_kraus(P.register(circ), "topk", k=40, total_shots=300000)
    else:
        circ = brickwork(4, 3, 0.05, 0.05, 9)
        info = P.sample_kraus(P.register(circ), "proportional", seed=3, nsamples=50, total_shots=5000)
    n = circ.n_qubits
    st, w, s = evolve_gpu(P, info, 0, info.count, n, True)
    bits = torch.empty(max(info.total_shots, 1), dtype=torch.int32, device="cuda")
    P.sample(info, 0, info.count, st, s, 5, bits)
    u = torch.zeros(info.count, dtype=torch.int64, device="cuda")
    P.unique_shots(info, 0, info.count, bits, u)
    torch.cuda.synchronize()
    b = bits.cpu().numpy().view(np.uint32)
    got = u.cpu().numpy()
    for a in range(info.count):
        x = b[int(info.shot_offsets[a]): int(info.shot_offsets[a + 1])]
        x = x[x < (1 << n)]
        assert got[a] == len(np.unique(x)), (a, got[a], len(np.unique(x)))


def test_uneven_batch_matches_single_context(oracle_mod):
    """The uneven-batch runner (several contexts, one stream each, circuits of different sizes)
    gives every circuit the same shots as a direct run of the same calls on one context."""
    torch = torch_cuda()
    from paper_2504_16297_gb300.batch import UnevenBatch
    cfg = config(2, small=True)
    circs, shots = cfg["circuits"], cfg["shots"]
    B = UnevenBatch(streams=3, max_qubits=max(c.n_qubits for c in circs), max_sets=cfg["nsamples"],
                    max_shots=int(np.max(shots)))
    B.autotune(circs, shots, cfg["nsamples"], cfg["seed"])
    secs, total, counts, kept = B.run(circs, shots, cfg["nsamples"], cfg["seed"], keep=set(range(len(circs))))
    assert total == int(np.sum(shots))
    P = gpu_ctx()
    for i, c in enumerate(circs):
        P.set_evolve_kernel(B.kernel_by_n[c.n_qubits])
        info = P.sample_kraus(P.register(c), "proportional", seed=cfg["seed"] + i, nsamples=cfg["nsamples"],
                              total_shots=int(shots[i]))
        st, w, s = evolve_gpu(P, info, 0, info.count, c.n_qubits, True)
        bits = torch.empty(info.total_shots, dtype=torch.int32, device="cuda")
        P.sample(info, 0, info.count, st, s, cfg["seed"] + i, bits)
        torch.cuda.synchronize()
        assert np.array_equal(bits.cpu().numpy(), kept[i][0].numpy()), f"circuit {i}"
        assert info.count == counts[i]
