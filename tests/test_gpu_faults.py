"""Host-side fault injection (-m gpu): every allocation a call makes can fail with PTSBE_ERR_OOM.
The failure is made on the host (PTSBE_OPT_FAIL_ALLOC: the k-th allocation of the context fails
as if memory ran out), never by faulting the GPU. For every k up to the number of allocations of
the call: the call returns PTSBE_ERR_OOM, its outputs keep the values they had (every allocation
precedes the call's first launch), and the same context then runs the call correctly."""
import numpy as np
import pytest

from gpu_common import gpu_ctx, torch_cuda
from workloads import brickwork, config

pytestmark = pytest.mark.gpu


def _fill(torch, n_sets, n, shots, states=True):
    st = torch.full((n_sets, 1 << n), 7 + 7j, dtype=torch.complex64, device="cuda") if states else None
    w = torch.full((n_sets,), -3.0, dtype=torch.float64, device="cuda")
    s = torch.full((n_sets,), 9, dtype=torch.uint8, device="cuda")
    b = torch.full((max(shots, 1),), -5, dtype=torch.int32, device="cuda")
    return st, w, s, b


def _untouched(torch, st, w, s, b):
    if st is not None:
        assert bool((st == (7 + 7j)).all())
    assert bool((w == -3.0).all()) and bool((s == 9).all()) and bool((b == -5).all())


def _injection_sweep(make_call, circ, pts, kernel=None, states=True, max_k=64):
    from paper_2504_16297_gb300 import capi
    from paper_2504_16297_gb300.capi import PtsbeError
    torch = torch_cuda()
    ref = None
    failures = 0
    for k in list(range(max_k)) + [-1]:
        P = gpu_ctx()
        if kernel:
            P.set_evolve_kernel(kernel)
        cid = P.register(circ)
        info = pts(P, cid)
        st, w, s, b = _fill(torch, info.count, circ.n_qubits, info.total_shots, states)
        capi.ptsbe_set_option(P.ctx, capi.PTSBE_OPT_FAIL_ALLOC, k)
        try:
            make_call(P, info, st, w, s, b)
            P.synchronize()
            ok = True
        except PtsbeError as e:
            assert e.status == 3, str(e)            # PTSBE_ERR_OOM, nothing else
            assert "injected" in str(e)
            ok = False
        if not ok:
            failures += 1
            torch.cuda.synchronize()
            _untouched(torch, st, w, s, b)
            # the same context stays usable
            capi.ptsbe_set_option(P.ctx, capi.PTSBE_OPT_FAIL_ALLOC, -1)
            make_call(P, info, st, w, s, b)
            P.synchronize()
        out = (w.cpu().numpy(), s.cpu().numpy(), b.cpu().numpy())
        if ref is None:
            ref = out
        assert all(np.array_equal(x, y) for x, y in zip(out, ref))
        P.close()
        if ok and k >= 0:
            break                                   # the call makes fewer than k + 1 allocations
    assert failures >= 3
    return failures


def test_oom_in_every_allocation_of_the_one_call_path():
    """Syndrome round on 17 qubits (frame kernel, fused sampling, support-CDF export)."""
    circ = config(1, small=True)["circuit"]
    pts = lambda P, cid: P.sample_kraus(cid, "topk", k=200, total_shots=500_000)
    call = lambda P, info, st, w, s, b: P.evolve_sample(info, 0, info.count, st, w, s, 11, b, prefix_reuse=True)
    _injection_sweep(call, circ, pts)


def test_oom_in_every_allocation_of_the_dense_path_without_states():
    """19-qubit brickwork, dense passes, states not returned (branch buffers, global-memory CDF)."""
    circ = brickwork(19, 6, 5e-3, 5e-3, seed=19)
    pts = lambda P, cid: P.sample_kraus(cid, "proportional", seed=3, nsamples=40, total_shots=40_000)
    call = lambda P, info, st, w, s, b: P.evolve_sample(info, 0, info.count, None, w, s, 11, b)
    _injection_sweep(call, circ, pts, states=False)


def test_oom_in_every_allocation_of_dense_batch_and_sampler():
    circ = brickwork(16, 5, 5e-3, 5e-3, seed=16)
    pts = lambda P, cid: P.sample_kraus(cid, "proportional", seed=3, nsamples=40, total_shots=40_000)

    def call(P, info, st, w, s, b):
        P.evolve(info, 0, info.count, st, w, s, prefix_reuse=True)
        P.sample(info, 0, info.count, st, s, 5, b)
    # two calls: a failure in the sampler leaves its shots untouched (the states are written by
    # then), so only the first call is checked for untouched outputs; the sweep still ends with
    # both calls correct on the same context
    from paper_2504_16297_gb300 import capi
    from paper_2504_16297_gb300.capi import PtsbeError
    torch = torch_cuda()
    for k in range(40):
        P = gpu_ctx()
        P.set_evolve_kernel("dense")
        cid = P.register(circ)
        info = pts(P, cid)
        st, w, s, b = _fill(torch, info.count, circ.n_qubits, info.total_shots)
        capi.ptsbe_set_option(P.ctx, capi.PTSBE_OPT_FAIL_ALLOC, k)
        try:
            P.evolve(info, 0, info.count, st, w, s, prefix_reuse=True)
            P.synchronize()
        except PtsbeError as e:
            assert e.status == 3
            _untouched(torch, st, w, s, b)
            capi.ptsbe_set_option(P.ctx, capi.PTSBE_OPT_FAIL_ALLOC, -1)
            call(P, info, st, w, s, b)
            P.synchronize()
            assert int(s.sum()) == 0 and bool((b >= 0).all())
            P.close()
            continue
        P.close()
        assert k >= 3
        break
