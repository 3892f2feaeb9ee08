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


def compare_state(psi_gpu, psi_ref, w_gpu, w_ref, st_gpu, st_ref, label=""):
    assert int(st_gpu) == int(st_ref), f"status {label}: gpu {st_gpu} oracle {st_ref}"
    if st_ref == 1:
        assert np.all(psi_gpu == 0), f"null state not zeroed {label}"
        return 0.0
    err = np.linalg.norm(psi_gpu.astype(np.complex128) - psi_ref) / np.linalg.norm(psi_ref)
    assert err <= AMP_RTOL, f"amplitudes {label}: rel err {err:.3e}"
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
