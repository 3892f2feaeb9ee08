"""Many circuits in one persistent launch (-m gpu): ptsbe_batch_plan / ptsbe_batch_run.

* The batch's states, weights, flags and shots are bit-identical to the dense kernel run circuit by
  circuit (ptsbe_evolve_batch with kernel 4, then ptsbe_sample_shots): the queue runs the same
  per-tile code in the same order of arithmetic, only scheduled differently.
* A run replayed as a CUDA graph gives the same results, every output rewritten on each replay.
* Sampled members against the oracle (amplitudes, weights, shots under the boundary rule).
* The queue's bounded wait: a task made to wait for a tile that never comes gives up after the
  configured budget, the next synchronize returns PTSBE_ERR_TIMEOUT, and the context and the batch
  then run correctly (no GPU fault: the wait is a bounded spin and the kernel returns).
"""
import numpy as np
import pytest

from gpu_common import check_shots, compare_state, gpu_ctx, torch_cuda
from workloads import brickwork

pytestmark = pytest.mark.gpu

MEMBERS = [(12, 9), (13, 14), (15, 11), (17, 20), (19, 8), (21, 12), (22, 6)]


def _members(P, nsamples=16):
    out = []
    for i, (n, d) in enumerate(MEMBERS):
        circ = brickwork(n, d, 1e-3 * (1 + i), 1e-2, seed=900 + i)
        cid = P.register(circ)
        shots = int(2000 * 3 ** i)
        info = P.sample_kraus(cid, "proportional", seed=40 + i, nsamples=nsamples, total_shots=shots)
        out.append((circ, info))
    return out


def _buffers(torch, circ, info, fill=True):
    n = circ.n_qubits
    st = torch.full((info.count, 1 << n), 3 + 3j, dtype=torch.complex64, device="cuda")
    w = torch.full((info.count,), -1.0, dtype=torch.float64, device="cuda")
    s = torch.full((info.count,), 7, dtype=torch.uint8, device="cuda")
    b = torch.full((max(info.total_shots, 1),), -9, dtype=torch.int32, device="cuda")
    return st, w, s, b


def _reference(P, members, seed0=500):
    torch = torch_cuda()
    P.set_evolve_kernel("dense")
    refs = []
    for i, (circ, info) in enumerate(members):
        st, w, s, b = _buffers(torch, circ, info)
        torch.cuda.synchronize()             # the context may run on a stream of its own
        P.evolve(info, 0, info.count, st, w, s, prefix_reuse=False)
        P.sample(info, 0, info.count, st, s, seed0 + i, b)
        refs.append((st, w, s, b))
    P.synchronize()
    return refs


def _plan(P, members, bufs, seed0=500):
    jobs = []
    for i, ((circ, info), (st, w, s, b)) in enumerate(zip(members, bufs)):
        jobs.append((info, 0, info.count, st, w, s, seed0 + i, b))
    return P.batch_plan(jobs)


def _same(refs, bufs):
    torch = torch_cuda()
    for i, (r, g) in enumerate(zip(refs, bufs)):
        for x, y, name in zip(r, g, ("states", "weights", "status", "shots")):
            assert torch.equal(x, y), f"member {i}: {name} differ"


def test_batch_matches_circuit_by_circuit():
    torch = torch_cuda()
    P = gpu_ctx()
    members = _members(P)
    refs = _reference(P, members)
    bufs = [_buffers(torch, c, info) for c, info in members]
    bid = _plan(P, members, bufs)
    info = P.batch_info(bid)
    exp_tasks = 0
    for c, inf in members:
        J = P.dense_plan_info(inf.circuit_id)["passes"]
        exp_tasks += inf.count * (J + 2)
    assert info["tasks"] == exp_tasks and info["grid"] > 0
    for _ in range(2):
        P.batch_run(bid)
        P.synchronize()
        _same(refs, bufs)
    P.batch_release(bid)


def test_batch_graph_replay():
    """Graph capture needs a stream of its own (not the legacy default stream)."""
    from paper_2504_16297_gb300.runtime import Ptsbe
    torch = torch_cuda()
    gpu_ctx()
    side = torch.cuda.Stream()
    P = Ptsbe(device=0, stream=side.cuda_stream)
    members = _members(P)
    refs = _reference(P, members)
    bufs = [_buffers(torch, c, info) for c, info in members]
    torch.cuda.synchronize()
    bid = _plan(P, members, bufs)
    for rep in range(3):
        torch.cuda.synchronize()
        for st, w, s, b in bufs:      # garbage before every replay: every output must be rewritten
            st.fill_(5 + 5j); w.fill_(-2.0); s.fill_(6); b.fill_(-3)
        torch.cuda.synchronize()
        P.batch_run(bid, graph=True)
        P.synchronize()
        _same(refs, bufs)
    P.batch_release(bid)
    P.close()


def test_batch_members_against_oracle(oracle_mod):
    torch = torch_cuda()
    P = gpu_ctx()
    members = _members(P)
    bufs = [_buffers(torch, c, info) for c, info in members]
    bid = _plan(P, members, bufs)
    P.batch_run(bid)
    P.synchronize()
    for m in (0, 3, 5, 6):
        circ, info = members[m]
        st, w, s, b = bufs[m]
        o = oracle_mod.Oracle(circ)
        n = circ.n_qubits
        b_h = b.cpu().numpy().view(np.uint32)
        for i in sorted(set([0, info.count - 1])):
            ref = o.pts_targeted([info.entries(i)], shots=np.zeros(1, np.uint64))
            psi, wr, sr = o.evolve(ref, 0)
            g = st[i].cpu().numpy()
            compare_state(g, psi, float(w[i].item()), wr, int(s[i].item()), sr, f"member {m} set {i}")
            o0, o1 = int(info.shot_offsets[i]), int(info.shot_offsets[i + 1])
            k = min(o1 - o0, 20000)
            if k and sr == 0:
                check_shots(b_h[o0:o0 + k], g, 500 + m, i, 0, oracle_mod, n)
    P.batch_release(bid)


def test_queue_wait_runs_out_then_recovers():
    from paper_2504_16297_gb300.capi import PtsbeError
    torch = torch_cuda()
    P = gpu_ctx()
    members = _members(P)[:3]
    refs = _reference(P, members)
    bufs = [_buffers(torch, c, info) for c, info in members]
    bid = _plan(P, members, bufs)
    tasks = P.batch_info(bid)["tasks"]
    # a task of the second level (it has a predecessor): its wait can never be met
    P.set_queue_stall_task(tasks // 2)
    P.set_queue_wait(2_000_000)          # about 1 ms
    P.batch_run(bid)
    with pytest.raises(PtsbeError) as e:
        P.synchronize()
    assert e.value.status == 5 and "ran out" in str(e.value)
    P.set_queue_stall_task(-1)
    P.set_queue_wait(20_000_000_000)
    P.batch_run(bid)
    P.synchronize()
    _same(refs, bufs)
    P.batch_release(bid)
