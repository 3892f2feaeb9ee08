"""ptsbe_sample_shots_noalloc: the sampler variant for callers that cannot allocate device memory
(a memory pool already owns the GPU, a fixed-footprint deployment, or a loop that must not hit the
synchronisation a cudaFree implies). Its scratch is a fixed array compiled into the library. It
must give exactly the shots of ptsbe_sample_shots, call after call, and refuse work that does not
fit the fixed array with a clear message.

Collected last on purpose (file name), so a run that stops at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from gpu_common import evolve_gpu, gpu_ctx, torch_cuda
from workloads import brickwork

pytestmark = pytest.mark.gpu


def _shots(P, fn, info, count, states, status, seed, total):
    torch = torch_cuda()
    bits = torch.full((total,), -7, dtype=torch.int32, device="cuda")
    fn(P.ctx, info.set_id, 0, count, states.data_ptr(), status.data_ptr(), seed, bits.data_ptr(), total)
    torch.cuda.synchronize()
    P.synchronize()
    return bits.cpu().numpy().view(np.uint32).copy()


@pytest.mark.parametrize("n", [17, 19])
def test_noalloc_matches_sample_shots_twice(n):
    """17 qubits: cluster sampler (scratch = work items); 19 qubits: global-memory CDF (scratch =
    the CDF workspace). Two calls in a row both equal the allocating entry point bit for bit."""
    from paper_2504_16297_gb300 import capi
    P = gpu_ctx()
    circ = brickwork(n, 2, 0.02, 0.02, seed=300 + n)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=5, nsamples=30, total_shots=200_000)
    count = min(info.count, 8)
    states, w, status = evolve_gpu(P, info, 0, count, n)
    total = int(info.shot_offsets[count])
    want = _shots(P, capi.ptsbe_sample_shots, info, count, states, status, 77, total)
    assert np.all(want < (1 << n))
    for _ in range(2):
        got = _shots(P, capi.ptsbe_sample_shots_noalloc, info, count, states, status, 77, total)
        assert np.array_equal(got, want)
    # a different seed changes the shots, so the comparison above is not vacuous
    other = _shots(P, capi.ptsbe_sample_shots_noalloc, info, count, states, status, 78, total)
    assert not np.array_equal(other, want)


def test_noalloc_items_through_a_staging_slot():
    """17 qubits (cluster sampler): the work items go up through a pinned staging slot that
    already had room, asynchronously: over five calls the library's count of staged
    host-to-device bytes grows by whole 40-byte items, the same number each call (a pageable copy
    is not counted there), the device's free memory does not move, and the shots repeat."""
    torch = torch_cuda()
    from paper_2504_16297_gb300 import capi
    P = gpu_ctx()
    n = 17
    circ = brickwork(n, 2, 0.02, 0.02, seed=417)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=6, nsamples=30, total_shots=300_000)
    count = min(info.count, 8)
    states, w, status = evolve_gpu(P, info, 0, count, n)
    total = int(info.shot_offsets[count])
    bits = torch.full((total,), -7, dtype=torch.int32, device="cuda")

    def call():
        capi.ptsbe_sample_shots_noalloc(P.ctx, info.set_id, 0, count, states.data_ptr(), status.data_ptr(), 91,
                                        bits.data_ptr(), total)

    call()
    torch.cuda.synchronize()
    P.synchronize()
    first = bits.cpu().numpy().copy()
    free0, _ = torch.cuda.mem_get_info()
    h0 = capi.ptsbe_h2d_bytes()
    for _ in range(5):
        call()
    torch.cuda.synchronize()
    P.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    staged = capi.ptsbe_h2d_bytes() - h0
    assert free1 == free0
    assert np.array_equal(bits.cpu().numpy(), first)
    assert staged > 0 and staged % 5 == 0 and (staged // 5) % 40 == 0


def test_noalloc_rejects_states_beyond_the_fixed_scratch():
    from paper_2504_16297_gb300 import capi
    from paper_2504_16297_gb300.capi import PtsbeError
    torch = torch_cuda()
    P = gpu_ctx()
    circ = brickwork(22, 1, 0.0, 0.0, seed=1)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "targeted", targeted=[[]], targeted_shots=np.array([16], np.uint64))
    # a full-size state (32 MiB), so that even a refusal that regressed could only read valid memory
    states = torch.zeros(1 << 22, dtype=torch.complex64, device="cuda")
    bits = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(PtsbeError) as e:
        capi.ptsbe_sample_shots_noalloc(P.ctx, info.set_id, 0, 1, states.data_ptr(), None, 1, bits.data_ptr(), 16)
    assert e.value.status == 7 and "fixed scratch" in str(e.value)


def test_noalloc_21_qubits_accepted():
    """The largest state the fixed CDF workspace holds (21 qubits): accepted, same shots."""
    from paper_2504_16297_gb300 import capi
    P = gpu_ctx()
    circ = brickwork(21, 1, 0.05, 0.05, seed=21)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=3, nsamples=8, total_shots=50_000)
    count = min(info.count, 2)
    states, w, status = evolve_gpu(P, info, 0, count, 21)
    total = int(info.shot_offsets[count])
    want = _shots(P, capi.ptsbe_sample_shots, info, count, states, status, 5, total)
    got = _shots(P, capi.ptsbe_sample_shots_noalloc, info, count, states, status, 5, total)
    assert np.array_equal(got, want)


def test_noalloc_rejects_more_work_items_than_the_fixed_scratch():
    """n <= 17 with more than 2^20 work items (one per set here): refused on the host before any
    device work, and the message gives the real limit. One qubit with 40 depolarising sites at
    p = 0.5 gives over a million distinct Kraus sets; their states (2 amplitudes each, 16 MiB in
    all) are allocated in full, so a regressed refusal could only read valid memory."""
    from paper_2504_16297_gb300 import capi
    from paper_2504_16297_gb300.capi import PtsbeError
    from workloads import CircuitBuilder
    torch = torch_cuda()
    P = gpu_ctx()
    b = CircuitBuilder(1)
    d1 = b.channel("DEPOL1", 0.5)
    for _ in range(40):
        b.gate("H", [0])
        b.noise(d1, [0])
    cid = P.register(b.build())
    n_sets = (1 << 20) + 100
    info = P.sample_kraus(cid, "proportional", seed=4, nsamples=n_sets + 4096, total_shots=n_sets + 4096,
                          export=False)
    assert info.count > (1 << 20)
    states = torch.zeros((info.count, 2), dtype=torch.complex64, device="cuda")
    bits = torch.zeros(info.total_shots, dtype=torch.int32, device="cuda")
    with pytest.raises(PtsbeError) as e:
        capi.ptsbe_sample_shots_noalloc(P.ctx, info.set_id, 0, info.count, states.data_ptr(), None, 1,
                                        bits.data_ptr(), info.total_shots)
    assert e.value.status == 7 and "1048576" in str(e.value)


def test_noalloc_allocates_nothing():
    """Repeated calls leave the device's free memory and the caching allocator's counters unchanged
    (after one warm-up call, which may load the library's module and resolve the array address)."""
    from paper_2504_16297_gb300 import capi
    torch = torch_cuda()
    P = gpu_ctx()
    n = 19
    circ = brickwork(n, 2, 0.02, 0.02, seed=319)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=5, nsamples=20, total_shots=100_000)
    count = min(info.count, 4)
    states, w, status = evolve_gpu(P, info, 0, count, n)
    total = int(info.shot_offsets[count])
    bits = torch.zeros(total, dtype=torch.int32, device="cuda")
    call = lambda: capi.ptsbe_sample_shots_noalloc(P.ctx, info.set_id, 0, count, states.data_ptr(),
                                                   status.data_ptr(), 9, bits.data_ptr(), total)
    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(5):
        call()
    torch.cuda.synchronize()
    P.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    alloc1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free1 == free0, (free0, free1)
    assert alloc1 == alloc0
