"""Shared helpers of the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np

AMP_RTOL = 1e-5      # per-state relative 2-norm, complex64 path vs complex128 oracle
W_RTOL = 1e-5        # branch weights
BOUNDARY_TOL = 1e-6  # a shot may differ only when u lies this close to every CDF boundary between


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def gpu_ctx():
    from paper_2504_16297_gb300 import build
    from paper_2504_16297_gb300.runtime import Ptsbe
    build()
    torch_cuda()
    return Ptsbe(device=0)


def evolve_gpu(P, info, first, count, n, prefix_reuse=False):
    torch = torch_cuda()
    st = torch.empty((max(count, 1), 1 << n), dtype=torch.complex64, device="cuda")
    w = torch.empty(max(count, 1), dtype=torch.float64, device="cuda")
    s = torch.empty(max(count, 1), dtype=torch.uint8, device="cuda")
    P.evolve(info, first, count, st, w, s, prefix_reuse=prefix_reuse)
    torch.cuda.synchronize()
    P.synchronize()
    return st, w, s


BIG_PROB = 1e-6      # amplitudes with |psi_i|^2 at least this are also checked one by one
# One by one, an amplitude carries the rounding of every complex64 operation applied to it: about
# 2^-24 sqrt(G) of the magnitudes being combined, for G operations (~3e-6 at the ~2,700 operations
# of the deepest test circuits; the largest of thousands of errors sits a few times above that).
# The combined magnitudes are of the order of the state's RMS amplitude ||psi||/sqrt(N), so an
# amplitude below the RMS (a near cancellation) has a larger relative error: the element error is
# taken relative to max(|psi_i|, RMS) and bounded by 5e-5; outcome probabilities P_i = |psi_i|^2 have
# twice the relative error (dP/P = 2 d|psi|/|psi|), relative to max(P_i, ||psi||^2/N): 1e-4. The state
# as a whole (relative 2-norm) and the probability vector as a whole stay at 1e-5.
AMP_ELEM_RTOL = 5e-5
PROB_ELEM_RTOL = 2 * AMP_ELEM_RTOL


def compare_state(psi_gpu, psi_ref, w_gpu, w_ref, st_gpu, st_ref, label=""):
    """Per-state relative 2-norm within 1e-5; every amplitude with |psi_i|^2 >= 1e-6 within 5e-5 of
    max(|psi_i|, RMS amplitude) and its outcome probability within 1e-4 of max(P_i, mean P); the
    probability vector within 1e-5 in relative 2-norm; weight within 1e-5; status identical."""
    assert int(st_gpu) == int(st_ref), f"status {label}: gpu {st_gpu} oracle {st_ref}"
    if st_ref == 1:
        assert np.all(psi_gpu == 0), f"null state not zeroed {label}"
        return 0.0
    g = psi_gpu.astype(np.complex128)
    err = np.linalg.norm(g - psi_ref) / np.linalg.norm(psi_ref)
    assert err <= AMP_RTOL, f"amplitudes {label}: rel err {err:.3e}"
    big = np.abs(psi_ref) ** 2 >= BIG_PROB
    if np.any(big):
        a, r = g[big], psi_ref[big]
        rms = np.linalg.norm(psi_ref) / np.sqrt(psi_ref.size)
        rel = np.abs(a - r) / np.maximum(np.abs(r), rms)
        assert rel.max() <= AMP_ELEM_RTOL, f"amplitude {label}: max rel err {rel.max():.3e} over {big.sum()} amplitudes"
        pr = np.abs(r) ** 2
        prel = np.abs(np.abs(a) ** 2 - pr) / np.maximum(pr, rms ** 2)
        assert prel.max() <= PROB_ELEM_RTOL, f"probability {label}: max rel err {prel.max():.3e}"
    pg, pr = np.abs(g) ** 2, np.abs(psi_ref) ** 2
    perr = np.linalg.norm(pg - pr) / np.linalg.norm(pr)
    assert perr <= AMP_RTOL, f"probability vector {label}: rel err {perr:.3e}"
    assert abs(w_gpu - w_ref) <= W_RTOL * abs(w_ref), f"weight {label}: {w_gpu} vs {w_ref}"
    return err


def check_shots(bits, psi, seed, alpha, first_shot, oracle_mod, n):
    """bits (uint32 numpy) of shots [first_shot, first_shot + len) of set alpha drawn from state psi
    (the GPU's own complex64 state): identical to the oracle fed the same state, except where the
    uniform lies within BOUNDARY_TOL of every CDF boundary between the two indices."""
    m = len(bits)
    want = oracle_mod.sample(n, psi.astype(np.complex128), m, seed, alpha, first_shot).astype(np.int64)
    got = bits.astype(np.int64)
    bad = np.nonzero(got != want)[0]
    if len(bad):
        C = oracle_mod.cdf(n, psi.astype(np.complex128))
        T = C[-1]
        for j in bad:
            lo, hi = sorted((int(got[j]), int(want[j])))
            assert 0 <= lo and hi < (1 << n), (j, got[j], want[j])
            u = oracle_mod.shot_uniform(seed, alpha, first_shot + int(j))
            dist = np.abs(C[lo:hi] / T - u).max()
            assert dist <= BOUNDARY_TOL, f"shot {j}: gpu {got[j]} oracle {want[j]} |C/T-u| {dist:.2e}"
    assert len(bad) <= max(2, m // 1000), f"{len(bad)} boundary mismatches out of {m}"
    return len(bad)


def _oracle_evolve_worker(args):
    """Oracle state of one Kraus set given by its entries (run in a spawned worker process)."""
    circ, entries, i = args
    from oracle import oracle as o
    O = o.Oracle(circ)
    sets = O.pts_targeted([entries], shots=np.zeros(1, np.uint64))
    psi, w, st = O.evolve(sets, 0)
    return i, psi, w, st


def oracle_states_parallel(circ, entries, idxs, workers=None):
    """{i: (psi, w, status)} from the oracle for the sets `entries[i]`, i in idxs, evaluated in
    parallel in processes started with spawn (safe after CUDA is initialised)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    idxs = list(idxs)
    workers = workers or max(1, min(len(idxs), (os.cpu_count() or 2)))
    out = {}
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for i, psi, w, st in ex.map(_oracle_evolve_worker, [(circ, list(entries[i]), i) for i in idxs]):
            out[i] = (psi, w, st)
    return out
