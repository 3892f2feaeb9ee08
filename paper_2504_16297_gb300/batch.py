"""Uneven batches: many noisy circuits of different sizes, each with its own Kraus sets and shot
budget, through several libptsbe contexts (one CUDA stream each) so that small circuits share the
GPU while the host runs PTS for the next ones.

Per circuit: register, pre-trajectory sampling (host), ptsbe_evolve_sample (state preparation
and shots in one call) on the circuit's context (asynchronous), release. Circuits go to the
contexts round-robin; each context reuses one state, weight, status and shot buffer, ordered by
its own stream. The evolve kernel for each qubit count is chosen once by the library's autotuner
on the first circuit of that size. Marshalling only: every step runs in libptsbe.
"""
from __future__ import annotations

import time

import numpy as np

from .runtime import Ptsbe


class UnevenBatch:
    def __init__(self, device: int = 0, streams: int = 4, max_qubits: int = 22, max_sets: int = 64,
                 max_shots: int = 1 << 20):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        self.ctxs = [Ptsbe(device, stream=s.cuda_stream) for s in self.streams]
        self.max_qubits, self.max_sets, self.max_shots = max_qubits, max_sets, max_shots
        amps = max_sets << max_qubits
        self.states = [torch.empty(amps, dtype=torch.complex64, device=self.dev) for _ in self.ctxs]
        self.weights = [torch.empty(max_sets, dtype=torch.float64, device=self.dev) for _ in self.ctxs]
        self.status = [torch.empty(max_sets, dtype=torch.uint8, device=self.dev) for _ in self.ctxs]
        self.bits = [torch.empty(max_shots, dtype=torch.int32, device=self.dev) for _ in self.ctxs]
        self.kernel_by_n = {}
        torch.cuda.synchronize(self.dev)

    def _views(self, j, count, n, shots):
        st = self.states[j][: count << n].view(count, 1 << n)
        return st, self.weights[j][:count], self.status[j][:count], self.bits[j][:max(shots, 1)]

    def autotune(self, circuits, shots, nsamples: int, seed: int):
        """Evolve kernel per qubit count, from the library autotuner on the first circuit of each size."""
        P = self.ctxs[0]
        for i, c in enumerate(circuits):
            n = c.n_qubits
            if n in self.kernel_by_n:
                continue
            cid = P.register(c)
            info = P.sample_kraus(cid, "proportional", seed=seed + i, nsamples=nsamples, total_shots=int(shots[i]),
                                  export=False)
            st, w, s, b = self._views(0, info.count, n, info.total_shots)
            res = P.autotune(info, 0, info.count, st, w, s, seed + i, b, prefix_reuse=True, reps=1)
            self.kernel_by_n[n] = res["evolve_kernel"]
            P.release_set(info)
            P.release_circuit(cid)
        self.torch.cuda.synchronize(self.dev)
        return dict(self.kernel_by_n)

    def run(self, circuits, shots, nsamples: int, seed: int, keep=None):
        """Runs every circuit; returns (seconds, total shots, per-circuit set counts). keep: optional
        list of circuit indices whose shots are copied to host (returned as a dict)."""
        torch = self.torch
        if any(c.n_qubits > self.max_qubits for c in circuits) or int(np.max(shots)) > self.max_shots:
            raise ValueError("circuit larger than the batch buffers")
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        counts, total, kept = [], 0, {}
        for i, c in enumerate(circuits):
            j = i % len(self.ctxs)
            P = self.ctxs[j]
            n = c.n_qubits
            if n in self.kernel_by_n:
                P.set_evolve_kernel(self.kernel_by_n[n])
            cid = P.register(c)
            info = P.sample_kraus(cid, "proportional", seed=seed + i, nsamples=nsamples, total_shots=int(shots[i]),
                                  export=keep is not None and i in keep)
            if info.count > self.max_sets:
                raise ValueError("more unique sets than the batch buffers hold")
            st, w, s, b = self._views(j, info.count, n, info.total_shots)
            P.evolve_sample(info, 0, info.count, st, w, s, seed + i, b, prefix_reuse=True)
            if keep is not None and i in keep:
                with torch.cuda.stream(self.streams[j]):
                    kept[i] = (b[: info.total_shots].cpu(), info)
            P.release_set(info)
            P.release_circuit(cid)
            counts.append(info.count)
            total += info.total_shots
        torch.cuda.synchronize(self.dev)
        return time.perf_counter() - t0, total, counts, kept
