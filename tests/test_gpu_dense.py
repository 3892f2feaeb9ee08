"""Dense tile passes on the GPU (-m gpu): parity with the CPU oracle and with the library's other
paths (Sec. 3, batched execution: each Kraus set's state prepared once, its shots drawn from it).

* 13-24 qubits: amplitudes within 1e-5 relative 2-norm of the complex128 oracle, per-amplitude
  and per-outcome-probability checks for the large amplitudes, weights within 1e-5, null flags
  identical, shots identical to the oracle fed the GPU's own state (1e-6 boundary rule).
* States not returned (prepared branch by branch in library buffers): weights, flags and every
  shot bit-identical to the dense kernel with caller states followed by ptsbe_sample_shots.
* 30 qubits (8 GiB states): a 60-layer brickwork with the one CX between qubits 14 and 15 left
  out is a product of two 15-qubit states, which the oracle prepares exactly -- the whole
  2^30-amplitude GPU state is compared with their tensor product; and a 60-layer circuit
  followed by its inverse must return to |0...0>.
"""
import math
import os

import numpy as np
import pytest

from gpu_common import (AMP_RTOL, check_shots, compare_state, evolve_gpu, gpu_ctx, oracle_states_parallel,
                        torch_cuda)
from workloads import CircuitBuilder, brickwork, config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    ctx = gpu_ctx()
    ctx.set_evolve_kernel("dense")
    return ctx


def compare_sets(P, oracle_mod, circ, info, idxs, reuse, shots=True, parallel=False):
    torch = torch_cuda()
    n = circ.n_qubits
    st, w, s = evolve_gpu(P, info, 0, info.count, n, reuse)
    entries = [info.entries(i) for i in range(info.count)]
    if parallel:
        refs = oracle_states_parallel(circ, entries, idxs)
    else:
        o = oracle_mod.Oracle(circ)
        refs = {}
        for i in idxs:
            sets = o.pts_targeted([entries[i]], shots=np.zeros(1, np.uint64))
            refs[i] = o.evolve(sets, 0)
    w_h, s_h = w.cpu().numpy(), s.cpu().numpy()
    bits = None
    if shots and info.total_shots:
        bits = torch.empty(info.total_shots, dtype=torch.int32, device="cuda")
        P.sample(info, 0, info.count, st, s, 777, bits)
        torch.cuda.synchronize()
        bits = bits.cpu().numpy().view(np.uint32)
    for i in idxs:
        psi_g = st[i].cpu().numpy()
        psi, wr, sr = refs[i]
        compare_state(psi_g, psi, w_h[i], wr, s_h[i], sr, f"set {i}")
        if bits is not None and sr == 0:
            o0, o1 = int(info.shot_offsets[i]), int(info.shot_offsets[i + 1])
            m = min(o1 - o0, 20000)
            if m:
                check_shots(bits[o0:o0 + m], psi_g, 777, i, 0, oracle_mod, n)
    return st, w, s


@pytest.mark.parametrize("n,layers", [(3, 6), (10, 20), (11, 8), (12, 10), (13, 8), (15, 6), (18, 4)])
@pytest.mark.parametrize("reuse", [False, True])
def test_dense_brickwork_matches_oracle(P, oracle_mod, n, layers, reuse):
    """n < 12 runs zero-padded to 12 qubits in a library buffer and is copied out to the caller's
    buffer of 2^n amplitudes per state."""
    circ = brickwork(n, layers, 0.02, 0.03, seed=70 + n)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=9, nsamples=60, total_shots=6000)
    idxs = sorted(set([0, 1, 2, info.count // 2, info.count - 1]))
    compare_sets(P, oracle_mod, circ, info, idxs, reuse)


def test_dense_padded_writes_only_the_callers_states(P):
    """The copy out of the padded buffer writes exactly count x 2^n amplitudes: a guard region past
    the caller's states keeps its fill, and the states are normalised."""
    torch = torch_cuda()
    circ = brickwork(9, 6, 0.02, 0.03, seed=77)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=3, nsamples=40, total_shots=400)
    n, cnt = 9, info.count
    buf = torch.full(((cnt + 1) << n,), 5.0 + 7.0j, dtype=torch.complex64, device="cuda")
    st = buf[: cnt << n].view(cnt, 1 << n)
    w = torch.empty(cnt, dtype=torch.float64, device="cuda")
    s = torch.empty(cnt, dtype=torch.uint8, device="cuda")
    P.evolve(info, 0, cnt, st, w, s)
    torch.cuda.synchronize()
    P.synchronize()
    guard = buf[cnt << n:].cpu().numpy()
    assert np.all(guard == np.complex64(5.0 + 7.0j))
    norms = (st.abs() ** 2).sum(dim=1).cpu().numpy()
    ok = s.cpu().numpy() == 0
    assert np.allclose(norms[ok], 1.0, atol=1e-5)


@pytest.mark.parametrize("n", [13, 16])
def test_dense_every_gate_and_channel_kind(P, oracle_mod, n):
    from test_gpu_parity import _kitchen_sink
    circ = _kitchen_sink(n, seed=n + 100)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=5, nsamples=40, total_shots=400)
    compare_sets(P, oracle_mod, circ, info, range(min(info.count, 10)), True)


def test_dense_damping_and_null_branches(P, oracle_mod):
    """General (damping) channels renormalised at the end; null branches zeroed with sentinel shots."""
    c = config(1, small=True)
    circ = c["circuit"]
    cid = P.register(circ)
    info = P.sample_kraus(cid, "topk", k=120, total_shots=120_000)
    st, w, s = compare_sets(P, oracle_mod, circ, info, [0, 1, 2, 50, 119], True)
    torch = torch_cuda()
    s_h = s.cpu().numpy()
    bits = torch.empty(info.total_shots, dtype=torch.int32, device="cuda")
    P.sample(info, 0, info.count, st, s, 3, bits)
    b = bits.cpu().numpy().view(np.uint32)
    for i in np.nonzero(s_h)[0]:
        o0, o1 = int(info.shot_offsets[i]), int(info.shot_offsets[i + 1])
        assert np.all(b[o0:o1] == 0xFFFFFFFF)
        assert not torch.any(st[int(i)] != 0)


@pytest.mark.parametrize("n,layers", [(22, 20), (24, 8)])
def test_dense_large_brickwork_full_depth(P, oracle_mod, n, layers):
    """The 30-qubit workload's family at 22 and 24 qubits (p = 5e-4 per gate), full depth, prefix
    reuse on: the error-free set and sets with errors, compared amplitude by amplitude with the
    oracle (run in parallel worker processes), and their shots."""
    circ = brickwork(n, layers, 5e-4, 5e-4, seed=1003)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=2003, nsamples=400, total_shots=400_000)
    lens = np.diff(info.offsets)
    idxs = [0] + [int(i) for i in np.nonzero(lens == 1)[0][:2]] + [int(i) for i in np.nonzero(lens >= 2)[0][:1]]
    idxs = sorted(set(idxs + [info.count - 1]))
    compare_sets(P, oracle_mod, circ, info, idxs, True, parallel=True)


def _stream_vs_batch(P, info, n, reuse=True):
    torch = torch_cuda()
    st, w, s = evolve_gpu(P, info, 0, info.count, n, reuse)
    bits_a = torch.empty(max(info.total_shots, 1), dtype=torch.int32, device="cuda")
    P.sample(info, 0, info.count, st, s, 4321, bits_a)
    del st
    w2 = torch.empty(info.count, dtype=torch.float64, device="cuda")
    s2 = torch.empty(info.count, dtype=torch.uint8, device="cuda")
    bits_b = torch.full((max(info.total_shots, 1),), -7, dtype=torch.int32, device="cuda")
    P.evolve_sample(info, 0, info.count, None, w2, s2, 4321, bits_b)
    P.synchronize()
    assert torch.equal(s, s2)
    assert torch.equal(w, w2), float((w - w2).abs().max())
    assert torch.equal(bits_a, bits_b)
    return w2, s2, bits_b


@pytest.mark.parametrize("n,layers", [(12, 12), (15, 10), (18, 8), (22, 6)])
def test_stream_matches_batch(P, oracle_mod, n, layers):
    circ = brickwork(n, layers, 4e-3, 8e-3, seed=40 + n)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=12, nsamples=150, total_shots=150_000)
    _stream_vs_batch(P, info, n)
    applied, full = P.reuse_stats()
    assert 0 < applied < full


def test_stream_damping_targeted(P, oracle_mod):
    """Branches inside branches: targeted sets sharing first entries, damping (null branches)."""
    c = config(1, small=True)
    circ = c["circuit"]
    cid = P.register(circ)
    base = [(0, 1), (10, 1), (40, 1)]
    targeted = [[], [(0, 1)], [(0, 1), (10, 1)], base, [(0, 1), (41, 1)], [(5, 1)], [(5, 1), (120, 1)], [(1, 1)]]
    info = P.sample_kraus(cid, "targeted", targeted=targeted, targeted_shots=np.full(len(targeted), 5000, np.uint64))
    w, s, _ = _stream_vs_batch(P, info, circ.n_qubits)
    o = oracle_mod.Oracle(circ)
    ref = o.pts_targeted([info.entries(i) for i in range(info.count)], shots=np.asarray(info.shots, np.uint64))
    w_h, s_h = w.cpu().numpy(), s.cpu().numpy()
    for i in range(info.count):
        _, wr, sr = o.evolve(ref, i)
        assert int(s_h[i]) == sr
        if sr == 0:
            assert abs(w_h[i] - wr) <= 1e-5 * wr


def test_config3_family_20_qubits_stream(P, oracle_mod):
    """The 30-qubit workload's reduced variant (20 qubits, 12 layers, 200 samples, 10^6 shots) in
    the mode the benchmark runs: states not returned, prepared branch by branch."""
    c = config(3, small=True)
    circ = c["circuit"]
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=c["seed"], nsamples=c["nsamples"], total_shots=c["total_shots"])
    w, s, bits = _stream_vs_batch(P, info, circ.n_qubits)
    applied, full = P.reuse_stats()
    assert applied < 0.8 * full
    # sampled sets against the oracle (states from the batch path, which is bit-identical)
    lens = np.diff(info.offsets)
    idxs = sorted(set([0, int(np.argmax(lens)), info.count - 1]))
    compare_sets(P, oracle_mod, circ, info, idxs, True, shots=True)


# --- 30 qubits ------------------------------------------------------------------------------

def split_brickwork(n, layers, p1, p2, seed, cut):
    """Brickwork (as workloads.brickwork) without the CX pairs that cross qubit `cut`, and the two
    half circuits (qubits [0, cut) and [cut, n)) with the same angles and noise; returns
    (full, low, high, site_map) with site_map[full site] = (half, site in that half)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bf, bl, bh = CircuitBuilder(n), CircuitBuilder(cut), CircuitBuilder(n - cut)
    ch = [(b.channel("DEPOL1", p1), b.channel("DEPOL2", p2)) for b in (bf, bl, bh)]
    smap, cnt = [], [0, 0]
    for layer in range(layers):
        for q in range(n):
            ang = tuple(rng.uniform(0.0, 2.0 * math.pi, 3))
            half = 0 if q < cut else 1
            hb, off = (bl, 0) if half == 0 else (bh, cut)
            for b, qq, c in ((bf, q, ch[0]), (hb, q - off, ch[1 + half])):
                b.gate("U3", [qq], ang)
                b.noise(c[0], [qq])
            smap.append((half, cnt[half])); cnt[half] += 1
        for q in range(0 if layer % 2 == 0 else 1, n - 1, 2):
            if q + 1 == cut:
                continue
            half = 0 if q < cut else 1
            hb, off = (bl, 0) if half == 0 else (bh, cut)
            for b, qq, c in ((bf, q, ch[0]), (hb, q - off, ch[1 + half])):
                b.gate("CX", [qq, qq + 1])
                b.noise(c[1], [qq, qq + 1])
            smap.append((half, cnt[half])); cnt[half] += 1
    return bf.build(), bl.build(), bh.build(), smap


def _gpu_mem_ok(gb):
    torch = torch_cuda()
    free, _ = torch.cuda.mem_get_info()
    return free >= gb * (1 << 30)


def test_thirty_qubit_product_state(P, oracle_mod):
    """30 qubits, 60 layers (2,640 gates, 5,280 noise sites): the full GPU state against the tensor
    product of the oracle's two 15-qubit halves, for the error-free set and sets with errors in
    both halves; then shots of the states-not-returned path against the same product."""
    torch = torch_cuda()
    if not _gpu_mem_ok(40):
        pytest.skip("needs 40 GiB of free device memory")
    n, cut = 30, 15
    full, low, high, smap = split_brickwork(n, 60, 5e-4, 5e-4, seed=1303, cut=cut)
    S = full.n_sites
    targeted = [[], [(7, 2)], [(100, 1), (S - 3, 3)], [(40, 5), (S // 2, 2), (S - 1, 9)]]
    cid = P.register(full)
    info = P.sample_kraus(cid, "targeted", targeted=targeted, targeted_shots=np.full(4, 50_000, np.uint64))
    ol, oh = oracle_mod.Oracle(low), oracle_mod.Oracle(high)
    st = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    w = torch.empty(1, dtype=torch.float64, device="cuda")
    s = torch.empty(1, dtype=torch.uint8, device="cuda")
    for i in range(info.count):
        ent = info.entries(i)
        el = [(smap[a][1], k) for a, k in ent if smap[a][0] == 0]
        eh = [(smap[a][1], k) for a, k in ent if smap[a][0] == 1]
        pl, wl, sl = ol.evolve(ol.pts_targeted([el], shots=np.zeros(1, np.uint64)), 0)
        ph, wh, sh = oh.evolve(oh.pts_targeted([eh], shots=np.zeros(1, np.uint64)), 0)
        assert sl == 0 and sh == 0
        P.evolve(info, i, 1, st, w, s)
        torch.cuda.synchronize()
        assert int(s.item()) == 0
        assert abs(float(w.item()) - wl * wh) <= 1e-5 * wl * wh
        a = torch.from_numpy(pl).cuda()          # index bits [0, 15)
        b = torch.from_numpy(ph).cuda()          # index bits [15, 30)
        g = st[0].view(1 << (n - cut), 1 << cut)
        err2 = ref2 = 0.0
        for r0 in range(0, 1 << (n - cut), 1024):
            ref = b[r0:r0 + 1024, None] * a[None, :]
            d = g[r0:r0 + 1024].to(torch.complex128) - ref
            err2 += float((d.abs() ** 2).sum())
            ref2 += float((ref.abs() ** 2).sum())
        err = math.sqrt(err2 / ref2)
        assert err <= AMP_RTOL, f"set {i}: rel err {err:.3e}"
        # the largest amplitudes one by one
        top_a = torch.topk(a.abs(), 8).indices
        top_b = torch.topk(b.abs(), 8).indices
        ref_t = (b[top_b][:, None] * a[top_a][None, :]).reshape(-1)
        got = g[top_b][:, top_a].reshape(-1).to(torch.complex128)
        rel = ((got - ref_t).abs() / ref_t.abs()).max().item()
        assert rel <= 1e-4, f"set {i}: top amplitudes rel err {rel:.3e}"
    del st
    torch.cuda.empty_cache()
    # states not returned: every shot a valid outcome; marginal histograms of the two halves
    w2 = torch.empty(info.count, dtype=torch.float64, device="cuda")
    s2 = torch.empty(info.count, dtype=torch.uint8, device="cuda")
    bits = torch.empty(info.total_shots, dtype=torch.int32, device="cuda")
    P.evolve_sample(info, 0, info.count, None, w2, s2, 99, bits)
    P.synchronize()
    assert int(s2.sum()) == 0
    bh = bits.cpu().numpy().view(np.uint32).astype(np.int64)
    from scipy import stats as sst
    for i in range(info.count):
        ent = info.entries(i)
        el = [(smap[a][1], k) for a, k in ent if smap[a][0] == 0]
        pl, _, _ = ol.evolve(ol.pts_targeted([el], shots=np.zeros(1, np.uint64)), 0)
        o0, o1 = int(info.shot_offsets[i]), int(info.shot_offsets[i + 1])
        lo = bh[o0:o1] & ((1 << cut) - 1)
        # marginal of the low half over its 16 most likely outcomes (+ the rest)
        p = np.abs(pl) ** 2
        top = np.argsort(-p)[:16]
        cnt = np.array([np.count_nonzero(lo == t) for t in top] + [0])
        cnt[-1] = len(lo) - cnt[:-1].sum()
        exp = np.append(p[top], 1 - p[top].sum()) * len(lo)
        keep = exp > 5
        chi = ((cnt[keep] - exp[keep]) ** 2 / exp[keep]).sum()
        pval = sst.chi2.sf(chi, keep.sum() - 1)
        assert pval > 1e-3, f"set {i}: low-half marginal chi-square p = {pval:.2e}"


def test_thirty_qubit_mirror_returns_to_zero(P):
    """60 brickwork layers on 30 qubits followed by their inverse (reverse order, U3 -> U3(-t, -l, -p)):
    the state returns to |0...0> up to FP32 rounding over 2 x 2,670 gates."""
    torch = torch_cuda()
    if not _gpu_mem_ok(20):
        pytest.skip("needs 20 GiB of free device memory")
    n, layers = 30, 60
    rng = np.random.Generator(np.random.PCG64(77))
    ops = []
    for layer in range(layers):
        for q in range(n):
            ops.append(("U3", [q], tuple(rng.uniform(0.0, 2.0 * math.pi, 3))))
        for q in range(0 if layer % 2 == 0 else 1, n - 1, 2):
            ops.append(("CX", [q, q + 1], ()))
    b = CircuitBuilder(n)
    for g, qs, ang in ops:
        b.gate(g, qs, ang if ang else (0.0, 0.0, 0.0))
    for g, qs, ang in reversed(ops):
        b.gate(g, qs, (-ang[0], -ang[2], -ang[1]) if ang else (0.0, 0.0, 0.0))
    circ = b.build()
    cid = P.register(circ)
    info = P.sample_kraus(cid, "targeted", targeted=[[]], targeted_shots=np.array([1000], np.uint64))
    st = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    w = torch.empty(1, dtype=torch.float64, device="cuda")
    s = torch.empty(1, dtype=torch.uint8, device="cuda")
    P.evolve(info, 0, 1, st, w, s)
    torch.cuda.synchronize()
    a0 = st[0, 0].item()
    rest = float((st[0, 1:].abs().to(torch.float64) ** 2).sum())
    assert abs(abs(a0) - 1.0) <= 1e-4, a0
    assert rest <= 1e-8, rest
    bits = torch.empty(1000, dtype=torch.int32, device="cuda")
    P.sample(info, 0, 1, st, s, 5, bits)
    assert int((bits != 0).sum()) == 0
