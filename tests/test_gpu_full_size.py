"""The benchmark workload at its full size, in the launch configuration bench.py times (-m gpu):
17-qubit syndrome circuit (3 rounds, 390 sites), the 10^4 most likely Kraus sets, 10^8 shots,
prefix reuse, default kernels.

* PTS: every set, q_alpha and shot count bit-identical to the oracle's independent top-K.
* Preparation: sampled states (the error-free set, single and double errors, the last set)
  within 1e-5 relative 2-norm of the oracle, weights within 1e-5, flags identical.
* Shots: for the same sets, the first shots (all of them for small sets) bit-identical to the
  oracle fed the GPU's own state, except within 1e-6 of a CDF boundary. The error-free set's
  8 x 10^7 shots go through the cluster sampler, the others through the one-CTA sampler.
"""
import numpy as np
import pytest

from gpu_common import check_shots, compare_state, gpu_ctx, torch_cuda
from workloads import config

pytestmark = pytest.mark.gpu


def test_bench_workload_full_size(oracle_mod):
    torch = torch_cuda()
    P = gpu_ctx()
    cfg = config(1)
    circ = cfg["circuit"]
    n = circ.n_qubits
    K, M = cfg["k"], cfg["total_shots"]
    cid = P.register(circ)
    info = P.sample_kraus(cid, "topk", k=K, total_shots=M)
    o = oracle_mod.Oracle(circ)
    ref = o.pts_topk(K, M)
    assert info.count == ref.count == K
    for i in range(K):
        assert info.entries(i) == ref.entries(i), i
    np.testing.assert_array_equal(np.asarray(info.q), np.asarray(ref.q))
    np.testing.assert_array_equal(np.asarray(info.shots, np.uint64), np.asarray(ref.shots, np.uint64))
    assert int(np.sum(info.shots)) == M

    states = torch.empty((K, 1 << n), dtype=torch.complex64, device="cuda")
    w = torch.empty(K, dtype=torch.float64, device="cuda")
    s = torch.empty(K, dtype=torch.uint8, device="cuda")
    bits = torch.empty(M, dtype=torch.int32, device="cuda")
    seed = cfg["seed"]
    P.evolve(info, 0, K, states, w, s, prefix_reuse=True)
    P.sample(info, 0, K, states, s, seed, bits)
    torch.cuda.synchronize()

    lens = [len(info.entries(i)) for i in range(K)]
    picks = [0, 1, lens.index(2), K // 2, K - 1]
    w_h, s_h = w.cpu().numpy(), s.cpu().numpy()
    for i in picks:
        psi_gpu = states[i].cpu().numpy()
        psi, wr, sr = o.evolve(ref, i)
        compare_state(psi_gpu, psi, w_h[i], wr, s_h[i], sr, f"set {i}")
        if sr == 1:
            continue
        off = int(info.shot_offsets[i])
        m = min(int(info.shots[i]), 20000)
        got = bits[off: off + m].cpu().numpy().view(np.uint32)
        check_shots(got, psi_gpu, seed, i, 0, oracle_mod, n)


@pytest.mark.parametrize("limit", [65536, 512])
def test_bench_workload_one_call(oracle_mod, limit):
    """The call bench.py times (ptsbe_evolve_sample) at full size, at the default light-shot limit
    and at 512 (the autotuner's choice on some boxes): states, weights, flags and all 10^8 shots
    bit-identical to ptsbe_evolve_batch + ptsbe_sample_shots; the error-free state's shots (support
    sampler over its exported CDF) and sampled light states' shots against the oracle."""
    torch = torch_cuda()
    P = gpu_ctx()
    P.set_light_shots(limit)
    cfg = config(1)
    circ = cfg["circuit"]
    n = circ.n_qubits
    K, M = cfg["k"], cfg["total_shots"]
    cid = P.register(circ)
    info = P.sample_kraus(cid, "topk", k=K, total_shots=M)
    seed = cfg["seed"]
    outs = []
    for fused in (False, True):
        states = torch.empty((K, 1 << n), dtype=torch.complex64, device="cuda")
        w = torch.empty(K, dtype=torch.float64, device="cuda")
        s = torch.empty(K, dtype=torch.uint8, device="cuda")
        bits = torch.full((M,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        if fused:
            P.evolve_sample(info, 0, K, states, w, s, seed, bits, prefix_reuse=True)
        else:
            P.evolve(info, 0, K, states, w, s, prefix_reuse=True)
            P.sample(info, 0, K, states, s, seed, bits)
        torch.cuda.synchronize()
        P.synchronize()
        outs.append((states, w, s, bits))
    (s0, w0, f0, b0), (s1, w1, f1, b1) = outs
    assert torch.equal(torch.view_as_real(s0), torch.view_as_real(s1))
    assert torch.equal(w0, w1) and torch.equal(f0, f1) and torch.equal(b0, b1)
    del s0, w0, f0, b0
    lens = [len(info.entries(i)) for i in range(K)]
    for i in [0, 1, lens.index(2), K - 1]:
        if int(info.shots[i]) == 0:
            continue
        psi = s1[i].cpu().numpy()
        off = int(info.shot_offsets[i])
        m = min(int(info.shots[i]), 20000)
        check_shots(b1[off: off + m].cpu().numpy().view(np.uint32), psi, seed, i, 0, oracle_mod, n)
