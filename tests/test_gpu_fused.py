"""Batched execution in one call, ptsbe_evolve_sample (-m gpu).

Its states, weights, status and shots are bit-identical to ptsbe_evolve_batch followed by
ptsbe_sample_shots on the same inputs (Sec. 3: prepare each unique state once, draw all of its
shots at once). That holds whether the last evolve launch draws a state's shots from the support it
holds on chip (a sparse final stage; states with at most the light-shot limit) or leaves them to
the sampler kernels. The fused shots also match the oracle fed the GPU's own state.
"""
import numpy as np
import pytest

from gpu_common import check_shots, gpu_ctx, torch_cuda
from workloads import CircuitBuilder, brickwork, syndrome17

pytestmark = pytest.mark.gpu


def _run(P, info, n, seed, fused, reuse=True, status=True):
    """Outputs of one way of running the range, every buffer pre-filled with garbage so that an
    output not written shows."""
    torch = torch_cuda()
    count = info.count
    total = int(info.shot_offsets[count])
    st = torch.full((count, 1 << n), 7.0 + 3.0j, dtype=torch.complex64, device="cuda")
    w = torch.full((count,), -1.0, dtype=torch.float64, device="cuda")
    s = torch.full((count,), 9, dtype=torch.uint8, device="cuda") if status else None
    bits = torch.full((max(total, 1),), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    if fused:
        P.evolve_sample(info, 0, count, st, w, s, seed, bits, prefix_reuse=reuse)
    else:
        P.evolve(info, 0, count, st, w, s, prefix_reuse=reuse)
        P.sample(info, 0, count, st, s, seed, bits)
    torch.cuda.synchronize()
    P.synchronize()
    return st, w, s, bits[:total]


def _same(a, b):
    torch = torch_cuda()
    for x, y, name in zip(a, b, ("states", "weights", "status", "shots")):
        if x is None:
            assert y is None
            continue
        if x.dtype == torch.complex64:
            x, y = torch.view_as_real(x), torch.view_as_real(y)
        assert torch.equal(x, y), f"{name} differ"


def _light_launches(P, info, n, seed, reuse=True):
    from paper_2504_16297_gb300 import capi
    P.set_timing(True)
    P.timing(capi.PTSBE_TIMER_SAMPLE_LIGHT, reset=True)
    P.timing(capi.PTSBE_TIMER_SAMPLE, reset=True)
    out = _run(P, info, n, seed, True, reuse)
    light = P.timing(capi.PTSBE_TIMER_SAMPLE_LIGHT, reset=True)[1]
    cluster = P.timing(capi.PTSBE_TIMER_SAMPLE, reset=True)[1]
    P.set_timing(False)
    return out, light, cluster


def test_syndrome_fused_matches_two_calls_and_oracle(oracle_mod):
    """17-qubit syndrome circuit, the 2,000 most likely sets, 2x10^7 shots: every light state's
    shots come from the evolve launch (no light-sampler launch), the error-free state's from the
    support sampler over the CDF the evolve launch exported; everything equals the two-call path,
    and sampled sets match the oracle."""
    P = gpu_ctx()
    circ = syndrome17(rounds=3)
    n = circ.n_qubits
    cid = P.register(circ)
    info = P.sample_kraus(cid, "topk", k=2000, total_shots=20_000_000)
    seed = 97
    sep = _run(P, info, n, seed, False)
    fused, light, cluster = _light_launches(P, info, n, seed)
    assert light == 0 and cluster >= 1
    _same(sep, fused)
    st_h = fused[0].cpu().numpy()
    b_h = fused[3].cpu().numpy().view(np.uint32)
    lens = [len(info.entries(i)) for i in range(info.count)]
    shots = np.asarray(info.shots)
    doubles = [i for i in range(info.count) if lens[i] == 2 and shots[i] > 0]
    picks = [1, 2, info.count // 2, info.count - 1] + doubles[:2]
    assert len(doubles) >= 2
    for a in picks:
        o0, o1 = int(info.shot_offsets[a]), int(info.shot_offsets[a + 1])
        if o1 > o0:
            check_shots(b_h[o0:o1], st_h[a], seed, a, 0, oracle_mod, n)


@pytest.mark.parametrize("limit", [1, 300, 1 << 20])
def test_light_limit_splits_fused_and_sampler_states(limit):
    """The light-shot limit decides which states the evolve launch samples; the shots do not
    depend on it."""
    P = gpu_ctx()
    circ = syndrome17(rounds=2)
    n = circ.n_qubits
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=5, nsamples=4000, total_shots=400_000)
    ref = _run(P, info, n, 11, False)
    P.set_light_shots(limit)
    _same(ref, _run(P, info, n, 11, True))
    _same(ref, _run(P, info, n, 11, True, reuse=False))


def _null_circuit():
    """A small support (three mixed qubits spread by CX) on 16 qubits; damping on qubit 15, which
    stays |0>, makes its K1 branch null."""
    b = CircuitBuilder(16)
    ad = b.channel("AMPDAMP", 0.02)
    dp = b.channel("DEPOL1", 0.01)
    for q in range(3):
        b.gate("H", [q]); b.noise(dp, [q])
    for q in range(3, 15):
        b.gate("CX", [q % 3, q]); b.noise(ad, [q])
    b.noise(ad, [15])
    return b.build()


@pytest.mark.parametrize("status,limit", [(True, 65536), (False, 65536), (True, 0), (False, 0)])
def test_null_states_fused(status, limit):
    """Null branches: the all-ones marker with a status buffer, the last index without one (what
    the samplers draw from a zeroed state), in both paths; with limit 0 every state leaves its
    support CDF (or its marker) for the support sampler."""
    torch = torch_cuda()
    P = gpu_ctx()
    P.set_light_shots(limit)
    circ = _null_circuit()
    n = circ.n_qubits
    cid = P.register(circ)
    sites = circ.n_sites
    info = P.sample_kraus(cid, "targeted", targeted=[[], [(sites - 1, 1)], [(3, 1)], [(0, 2)], [(3, 1), (sites - 1, 1)]],
                          targeted_shots=np.array([500, 60, 70, 80, 90], np.uint64))
    sep = _run(P, info, n, 3, False, status=status)
    fused = _run(P, info, n, 3, True, status=status)
    _same(sep, fused)
    if status:
        light, support = _light_launches(P, info, n, 3)[1:]
        assert light == 0 and (support == 0) == (limit > 0)   # limit 0: every state exported
    b_h = fused[3].cpu().numpy().view(np.uint32)
    mark = 0xFFFFFFFF if status else (1 << n) - 1
    null = [i for i in range(info.count) if (sites - 1, 1) in [tuple(e) for e in info.entries(i)]]
    assert len(null) == 2
    w_h = fused[1].cpu().numpy()
    for i in range(info.count):
        o0, o1 = int(info.shot_offsets[i]), int(info.shot_offsets[i + 1])
        if i in null:
            assert np.all(b_h[o0:o1] == mark) and w_h[i] < 1e-6, i
            if status:
                assert int(fused[2][i]) == 1
        else:
            assert np.all(b_h[o0:o1] < (1 << n)) and w_h[i] > 1e-6, i


@pytest.mark.parametrize("kernel", ["frame", "sweep"])
def test_dense_states_fall_back_to_samplers(kernel):
    """A brickwork circuit (dense states: no sparse final stage) and the non-frame kernels: the
    one call is the two calls."""
    P = gpu_ctx()
    P.set_evolve_kernel(kernel)
    circ = brickwork(12, 6, 0.01, 0.02, seed=123)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=8, nsamples=300, total_shots=30_000)
    _same(_run(P, info, 12, 21, False), _run(P, info, 12, 21, True))


@pytest.mark.parametrize("fused,percent", [(True, 100), (True, 37), (False, 100), (False, 50)])
def test_zero_fill_beside_program_prepass(fused, percent):
    """Part (or all) of the states' zero fill of a one-stage sparse final plan runs on the context's
    second stream beside the program prepass, the rest inside the evolve launch: the outputs equal
    those of the fill inside the evolve launch, and the split fill is one launch of its own over
    that share of every state (whole 4 KB chunks)."""
    from paper_2504_16297_gb300 import capi
    P = gpu_ctx()
    circ = syndrome17(rounds=2)
    n = circ.n_qubits
    cid = P.register(circ)
    info = P.sample_kraus(cid, "topk", k=1500, total_shots=3_000_000)
    try:
        P.set_split_fill(0)
        off = _run(P, info, n, 29, fused)
        P.set_split_fill(percent)
        P.set_timing(True)
        P.timing(capi.PTSBE_TIMER_ZERO_FILL, reset=True)
        on = _run(P, info, n, 29, fused)
        _, launches, nbytes = P.timing(capi.PTSBE_TIMER_ZERO_FILL, reset=True)
    finally:
        P.set_timing(False)
        P.set_split_fill(0)
    _same(off, on)
    state = 8 << n
    assert launches == 1 and nbytes == info.count * (state * percent // 100 // 4096 * 4096)


def test_prepass_ahead_back_to_back():
    """Calls issued back to back with no synchronisation between them, each registering its own
    circuit and Kraus set and releasing both right after (the bench's step), one-call and two-call
    paths mixed, two calls writing the same state buffer: with the prepass ahead (uploads and
    program prepass on the second stream, overlapping the previous call) every output equals the
    same sequence run with the prepass on the context stream. Also the prepass ahead of a circuit
    and a set uploaded by an earlier call on the context stream."""
    torch = torch_cuda()
    from paper_2504_16297_gb300.runtime import Ptsbe
    gpu_ctx()
    jobs = [(2, 5e-4, 1e-3, 1200, True), (3, 1e-3, 1e-3, 2000, False), (2, 2e-3, 5e-4, 900, True),
            (3, 5e-4, 2e-3, 2500, True), (1, 1e-3, 1e-3, 400, False)]

    def run(ahead):
        P = Ptsbe(device=0)
        P.set_prepass_ahead(ahead)
        shared = torch.full((2500, 1 << 17), 5.0 + 1.0j, dtype=torch.complex64, device="cuda")
        outs = []
        torch.cuda.synchronize()
        for i, (rounds, gamma, p, k, fused) in enumerate(jobs):
            circ = syndrome17(rounds=rounds, gamma=gamma, p=p, seed=1100 + i)
            cid = P.register(circ)
            info = P.sample_kraus(cid, "topk", k=k, total_shots=400_000 * (i + 1), export=False)
            total = int(info.total_shots)
            st = shared[:info.count] if i in (2, 3) else torch.full((info.count, 1 << 17), 7.0 + 3.0j,
                                                                    dtype=torch.complex64, device="cuda")
            w = torch.full((info.count,), -1.0, dtype=torch.float64, device="cuda")
            s = torch.full((info.count,), 9, dtype=torch.uint8, device="cuda")
            b = torch.full((total,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
            if fused:
                P.evolve_sample(info, 0, info.count, st, w, s, 40 + i, b, prefix_reuse=True)
            else:
                P.evolve(info, 0, info.count, st, w, s, prefix_reuse=True)
                P.sample(info, 0, info.count, st, s, 40 + i, b)
            # the shared buffer is overwritten by the next call: keep a copy made in stream order
            outs.append((st.clone() if i == 2 else st, w, s, b))
            P.release_set(info)
            P.release_circuit(cid)
        # a circuit and set uploaded on the context stream, then prepared with the prepass ahead
        circ = syndrome17(rounds=2, seed=1200)
        cid = P.register(circ)
        info = P.sample_kraus(cid, "topk", k=700, total_shots=100_000, export=False)
        P.set_prepass_ahead(False)
        first = [torch.empty((info.count, 1 << 17), dtype=torch.complex64, device="cuda"),
                 torch.empty(info.count, dtype=torch.float64, device="cuda"),
                 torch.empty(info.count, dtype=torch.uint8, device="cuda"),
                 torch.empty(100_000, dtype=torch.int32, device="cuda")]
        P.evolve_sample(info, 0, info.count, *first[:3], 3, first[3], prefix_reuse=True)
        P.set_prepass_ahead(ahead)
        again = [torch.full_like(x, 0) for x in first]
        P.evolve_sample(info, 0, info.count, *again[:3], 3, again[3], prefix_reuse=True)
        outs.append(tuple(first))
        outs.append(tuple(again))
        P.synchronize()
        torch.cuda.synchronize()
        P.close()
        return outs

    ref = run(False)
    got = run(True)
    assert len(ref) == len(got)
    for i, (a, b) in enumerate(zip(ref, got)):
        for x, y, name in zip(a, b, ("states", "weights", "status", "shots")):
            if x.dtype == torch.complex64:
                x, y = torch.view_as_real(x), torch.view_as_real(y)
            assert torch.equal(x, y), f"call {i}: {name} differ"
    _same(ref[-2], ref[-1])


def test_evolve_sample_errors():
    """Capacity and pointer checks before any launch."""
    torch = torch_cuda()
    from paper_2504_16297_gb300 import capi
    P = gpu_ctx()
    circ = syndrome17(rounds=1)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "topk", k=10, total_shots=1000)
    st = torch.empty((10, 1 << 17), dtype=torch.complex64, device="cuda")
    small = torch.empty(999, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.PtsbeError) as e:
        P.evolve_sample(info, 0, 10, st, None, None, 1, small)
    assert e.value.status == 6   # PTSBE_ERR_BUFFER_TOO_SMALL
    with pytest.raises(capi.PtsbeError) as e:
        P.evolve_sample(info, 0, 11, st, None, None, 1, small)
    assert e.value.status == 1   # PTSBE_ERR_INVALID
