"""Marshalling between Python objects and the libptsbe C ABI.

Circuits come in the flat encoding of ``workloads`` (op_ints, op_params, channels); device
buffers are PyTorch tensors whose pointers and the current CUDA stream are handed to the
library. No arithmetic of the method happens here.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import capi


@dataclass
class KrausSetInfo:
    set_id: int
    circuit_id: int
    count: int
    n_entries: int
    total_shots: int
    offsets: np.ndarray
    sites: np.ndarray
    kidx: np.ndarray
    mult: np.ndarray
    q: np.ndarray
    shots: np.ndarray
    shot_offsets: np.ndarray

    def entries(self, i):
        b, e = int(self.offsets[i]), int(self.offsets[i + 1])
        return list(zip(self.sites[b:e].tolist(), self.kidx[b:e].tolist()))


def _ptr(t) -> int | None:
    if t is None:
        return None
    return int(t.data_ptr())


_OP_DTYPE = np.dtype({
    "names": ["kind", "id", "n_targets", "targets", "params"],
    "formats": [np.uint32, np.uint32, np.uint32, (np.uint32, 2), (np.float64, 3)],
    "offsets": [capi.ptsbe_op.kind.offset, capi.ptsbe_op.id.offset, capi.ptsbe_op.n_targets.offset,
                capi.ptsbe_op.targets.offset, capi.ptsbe_op.params.offset],
    "itemsize": C.sizeof(capi.ptsbe_op),
})


class Ptsbe:
    """One libptsbe context. device=-1 gives a host-only context (registration and PTS)."""

    def __init__(self, device: int = 0, stream=None):
        self.device = device
        self._keep = []
        if stream is None and device >= 0:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.ctx = capi.ptsbe_create(device, stream)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            capi.ptsbe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        capi.ptsbe_set_stream(self.ctx, stream)

    def synchronize(self):
        capi.ptsbe_synchronize(self.ctx)

    # -- registration ----------------------------------------------------------------------------
    def register(self, circ) -> int:
        n_ops = circ.n_ops
        # ptsbe_op records filled column by column through a numpy view of the same layout
        op_rec = np.zeros(max(n_ops, 1), dtype=_OP_DTYPE)   # kept alive until the call returns
        if n_ops:
            oi = np.asarray(circ.op_ints)
            op = np.asarray(circ.op_params, np.float64)
            op_rec["kind"][:n_ops], op_rec["id"][:n_ops], op_rec["n_targets"][:n_ops] = oi[:, 0], oi[:, 1], oi[:, 2]
            op_rec["targets"][:n_ops] = oi[:, 3:5]
            op_rec["params"][:n_ops] = op[:, 0:3]
        ops = C.cast(op_rec.ctypes.data, C.POINTER(capi.ptsbe_op))
        n_ch = len(circ.ch_params)
        chans = (capi.ptsbe_channel * max(n_ch, 1))()
        keep = []
        for j in range(n_ch):
            kind, arity, nk = (int(x) for x in circ.ch_ints[j])
            c = chans[j]
            c.kind, c.arity, c.n_kraus, c.param = kind, arity, nk, float(circ.ch_params[j])
            off = int(circ.ch_kraus_off[j])
            if off >= 0:
                d = 1 << arity
                arr = np.ascontiguousarray(circ.ch_kraus[off: off + nk * d * d]).view(np.float64).copy()
                keep.append(arr)
                c.kraus = arr.ctypes.data_as(C.POINTER(C.c_double))
        cg = np.ascontiguousarray(np.asarray(circ.custom_gates, np.complex128)).view(np.float64).reshape(-1)
        cg_ptr = cg.ctypes.data if cg.size else None
        cid = capi.ptsbe_register_circuit(self.ctx, circ.n_qubits, ops, n_ops, chans, n_ch, cg_ptr,
                                          int(circ.custom_gates.shape[0]))
        del op_rec, keep
        return cid

    def release_circuit(self, cid):
        capi.ptsbe_release_circuit(self.ctx, cid)

    def set_evolve_kernel(self, kernel: str):
        """'auto' (= 'frame'), 'frame' (permutations and diagonals deferred; tile passes only for
        operators that mix amplitudes), 'sweep' (one shared-memory pass per operator), 'registers' or
        'dense' (register-blocked fused 1-/2-qubit blocks, one HBM pass per planned pass; a state of
        fewer than 12 qubits runs zero-padded to 12)."""
        capi.ptsbe_set_option(self.ctx, capi.PTSBE_OPT_EVOLVE_KERNEL,
                              {"auto": 0, "sweep": 1, "registers": 2, "frame": 3, "dense": 4}[kernel])

    def autotune(self, info: KrausSetInfo, first: int, count: int, states, weights, status, seed: int, bits,
                 prefix_reuse: bool = True, reps: int = 3):
        """Times every evolve kernel and sampler shot limit on this workload and keeps the fastest
        (host-synchronous). Returns a dict of the choice and the measured milliseconds."""
        flags = capi.PTSBE_EVOLVE_PREFIX_REUSE if prefix_reuse else 0
        t = capi.ptsbe_autotune(self.ctx, info.set_id, first, count, _ptr(states), _ptr(weights), _ptr(status), flags,
                                seed, _ptr(bits), bits.numel(), reps)
        names = {1: "sweep", 2: "registers", 3: "frame", 4: "dense"}
        return {"evolve_kernel": names.get(t.evolve_kernel, t.evolve_kernel), "light_shots": t.light_shots,
                "evolve_ms": {names[k]: t.evolve_ms[k] for k in (1, 2, 3, 4) if t.evolve_ms[k] > 0},
                "sample_ms": {int(t.light_candidates[i]): t.sample_ms[i] for i in range(4)}}

    def set_program_sets_per_warp(self, spw: int):
        """Kraus sets per warp of the frame program prepass (4, 8 or 16; 0 = default, 8)."""
        capi.ptsbe_set_option(self.ctx, capi.PTSBE_OPT_PROGRAM_SETS_PER_WARP, int(spw))

    def set_split_fill(self, percent: int):
        """Percentage of each state of a small sparse final stage zeroed on the context's second
        stream beside the program prepass (default 0: all of it inside the evolve launch)."""
        capi.ptsbe_set_option(self.ctx, capi.PTSBE_OPT_SPLIT_FILL, int(percent))

    def set_prepass_ahead(self, on: bool):
        """One-stage frame plans: uploads and program prepass on the context's second stream,
        overlapping earlier calls (default on)."""
        capi.ptsbe_set_option(self.ctx, capi.PTSBE_OPT_PREPASS_AHEAD, 1 if on else 0)

    def set_pershot_tile_bits(self, bits: int):
        """Tile bits of the per-shot (Algorithm 1) plan (9..14; 0 = default)."""
        capi.ptsbe_set_option(self.ctx, capi.PTSBE_OPT_PERSHOT_TILE_BITS, int(bits))

    def set_light_shots(self, limit: int):
        """Shot count up to which a state is sampled by the one-CTA light sampler."""
        capi.ptsbe_set_option(self.ctx, capi.PTSBE_OPT_LIGHT_SHOTS, int(limit))

    def set_timing(self, enable: bool):
        capi.ptsbe_set_timing(self.ctx, enable)

    def timing(self, kernel_class: int, reset: bool = False):
        """(milliseconds, launches, algorithmic bytes) accumulated for one kernel class."""
        return capi.ptsbe_get_timing(self.ctx, kernel_class, reset)

    def batch_plan(self, jobs):
        """Plans one persistent launch over many jobs: each job is (info, first, count, states, weights,
        status, seed, bits) with device tensors (weights, status, bits may be None). Returns a batch id."""
        recs = []
        for (info, first, count, states, weights, status, seed, bits) in jobs:
            recs.append(capi.ptsbe_job(info.set_id, first, count, _ptr(states), _ptr(weights), _ptr(status), seed,
                                       _ptr(bits), bits.numel() if bits is not None else 0))
        return capi.ptsbe_batch_plan(self.ctx, recs)

    def batch_run(self, batch_id, graph: bool = False):
        capi.ptsbe_batch_run(self.ctx, batch_id, capi.PTSBE_BATCH_GRAPH if graph else 0)

    def batch_info(self, batch_id):
        t, i, g, k = capi.ptsbe_batch_info(self.ctx, batch_id)
        return {"tasks": t, "items": i, "grid": g, "kernels_per_run": k}

    def batch_release(self, batch_id):
        capi.ptsbe_batch_release(self.ctx, batch_id)

    def set_queue_wait(self, cycles: int):
        capi.ptsbe_set_option(self.ctx, capi.PTSBE_OPT_QUEUE_SPIN_CYCLES, int(cycles))

    def set_queue_stall_task(self, task: int):
        capi.ptsbe_set_option(self.ctx, capi.PTSBE_OPT_QUEUE_STALL_TASK, int(task))

    def reuse_stats(self):
        """(gates applied, gates without prefix reuse) of the last evolve call."""
        return capi.ptsbe_reuse_stats(self.ctx)

    def dense_work(self):
        """(pass launches, FP32 multiply-adds) of the last call that ran dense passes."""
        return capi.ptsbe_dense_work(self.ctx)

    def dense_plan_info(self, cid):
        p, fx, b1, b2, f = capi.ptsbe_dense_plan_info(self.ctx, cid)
        return {"passes": p, "fixup_passes": fx, "blocks_1q": b1, "blocks_2q": b2, "fma_per_amplitude": f}

    def plan(self, info: KrausSetInfo, first: int, count: int):
        """Schedule of ptsbe_evolve_sample without states for the range, without running it; returns
        (gates applied, gates without prefix reuse)."""
        capi.ptsbe_evolve_sample(self.ctx, info.set_id, first, count, None, None, None, capi.PTSBE_EVOLVE_PLAN_ONLY,
                                 0, None, 0)
        return capi.ptsbe_reuse_stats(self.ctx)

    def circuit_info(self, cid):
        return capi.ptsbe_circuit_info(self.ctx, cid)

    # -- pre-trajectory sampling -------------------------------------------------------------------
    def sample_kraus(self, cid: int, mode: str, seed: int = 0, *, nsamples=0, k=0, p_min=0.0, p_max=1.0,
                     total_shots=0, shots_per_set=0, shot_alloc=None, targeted=None, targeted_shots=None,
                     export=True, max_errors=1, include_empty=False, qubit_mask=0, kraus_mask=0, gate_mask=0,
                     site_lo=0, site_hi=0, weight_parity=0, max_sets=0):
        p = capi.ptsbe_pts_params()
        modes = dict(proportional=capi.PTSBE_PTS_PROPORTIONAL, topk=capi.PTSBE_PTS_TOPK,
                     band=capi.PTSBE_PTS_BAND, targeted=capi.PTSBE_PTS_TARGETED, literal=capi.PTSBE_PTS_LITERAL,
                     predicate=capi.PTSBE_PTS_PREDICATE)
        p.mode = modes[mode]
        allocs = dict(count=capi.PTSBE_SHOTS_BY_COUNT, uniform=capi.PTSBE_SHOTS_UNIFORM,
                      prob=capi.PTSBE_SHOTS_BY_PROB, given=capi.PTSBE_SHOTS_GIVEN)
        if shot_alloc is None:
            shot_alloc = {"proportional": "count", "topk": "prob", "band": "prob", "literal": "uniform",
                          "targeted": "given" if targeted_shots is not None else "prob", "predicate": "prob"}[mode]
        p.shot_alloc = allocs[shot_alloc]
        p.nsamples, p.k, p.p_min, p.p_max = nsamples, k, p_min, p_max
        p.total_shots, p.shots_per_set = total_shots, shots_per_set
        p.max_errors, p.include_empty, p.qubit_mask = int(max_errors), int(bool(include_empty)), int(qubit_mask)
        p.kraus_mask, p.gate_mask, p.site_lo, p.site_hi = int(kraus_mask), int(gate_mask), int(site_lo), int(site_hi)
        p.weight_parity, p.max_sets = int(weight_parity), int(max_sets)
        keep = []
        if targeted is not None:
            offs, sites, ks = [0], [], []
            for s in targeted:
                for (a, b) in s:
                    sites.append(a); ks.append(b)
                offs.append(len(sites))
            to = np.asarray(offs, np.uint32); ts = np.asarray(sites + [0], np.uint32); tk = np.asarray(ks + [0], np.uint8)
            keep += [to, ts, tk]
            p.t_count = len(targeted)
            p.t_offsets = to.ctypes.data_as(C.POINTER(C.c_uint32))
            p.t_sites = ts.ctypes.data_as(C.POINTER(C.c_uint32))
            p.t_kidx = tk.ctypes.data_as(C.POINTER(C.c_uint8))
            if targeted_shots is not None:
                tsh = np.ascontiguousarray(targeted_shots, np.uint64)
                keep.append(tsh)
                p.t_shots = tsh.ctypes.data_as(C.POINTER(C.c_uint64))
        sid, cnt, ne, tot = capi.ptsbe_sample_kraus(self.ctx, cid, p, seed)
        info = KrausSetInfo(sid, cid, cnt, ne, tot, *(np.zeros(0),) * 7)
        if export:
            self.export(info)
        return info

    def export(self, info: KrausSetInfo):
        n, e = info.count, info.n_entries
        info.offsets = np.zeros(n + 1, np.uint32)
        info.sites = np.zeros(max(e, 1), np.uint32)
        info.kidx = np.zeros(max(e, 1), np.uint8)
        info.mult = np.zeros(max(n, 1), np.uint64)
        info.q = np.zeros(max(n, 1), np.float64)
        info.shots = np.zeros(max(n, 1), np.uint64)
        info.shot_offsets = np.zeros(n + 1, np.uint64)
        v = capi.ptsbe_set_view(info.offsets.ctypes.data, info.sites.ctypes.data, info.kidx.ctypes.data,
                                info.mult.ctypes.data, info.q.ctypes.data, info.shots.ctypes.data,
                                info.shot_offsets.ctypes.data)
        capi.ptsbe_set_export(self.ctx, info.set_id, v)
        info.sites, info.kidx = info.sites[:e], info.kidx[:e]
        info.mult, info.q, info.shots = info.mult[:n], info.q[:n], info.shots[:n]
        return info

    def release_set(self, info: KrausSetInfo):
        capi.ptsbe_release_set(self.ctx, info.set_id)

    # -- batched execution ---------------------------------------------------------------------------
    def evolve(self, info: KrausSetInfo, first: int, count: int, states, weights=None, status=None,
               prefix_reuse: bool = False):
        flags = capi.PTSBE_EVOLVE_PREFIX_REUSE if prefix_reuse else 0
        capi.ptsbe_evolve_batch(self.ctx, info.set_id, first, count, _ptr(states), _ptr(weights), _ptr(status), flags)

    def sample(self, info: KrausSetInfo, first: int, count: int, states, status, seed: int, bits):
        capi.ptsbe_sample_shots(self.ctx, info.set_id, first, count, _ptr(states), _ptr(status), seed, _ptr(bits),
                                bits.numel())

    def evolve_sample(self, info: KrausSetInfo, first: int, count: int, states, weights, status, seed: int, bits,
                      prefix_reuse: bool = False):
        """evolve() then sample() in one call (same outputs); light states' shots are drawn by the last
        evolve launch from the support it holds on chip. states=None (n > 12): the states stay in
        library buffers, prepared one branch at a time with dense passes (see ptsbe_evolve_sample)."""
        flags = capi.PTSBE_EVOLVE_PREFIX_REUSE if prefix_reuse else 0
        capi.ptsbe_evolve_sample(self.ctx, info.set_id, first, count, _ptr(states), _ptr(weights), _ptr(status), flags,
                                 seed, _ptr(bits), bits.numel() if bits is not None else 0)

    def backward(self, cid: int, info: KrausSetInfo, first: int, count: int, masks=(), coeffs=(), diag=None,
                 checkpoint_every: int = 0, loss=None, per_set=None, grad_params=None, grad_noise=None):
        """Adjoint loss and gradients of the fixed-set estimator over sets [first, first + count) at the
        parameters of circuit `cid` (same structure as the set's circuit). Outputs are float64 device
        tensors (loss [1], per_set [count], grad_params [n_ops, 3], grad_noise [n_channels]); any may
        be None. masks / coeffs: Z-string terms; diag: float64 device tensor [2^n] or None."""
        m = np.ascontiguousarray(np.asarray(masks, np.uint64).reshape(-1))
        c = np.ascontiguousarray(np.asarray(coeffs, np.float64).reshape(-1))
        if m.size != c.size:
            raise ValueError("masks and coeffs differ in length")
        obs = capi.ptsbe_observable()
        obs.n_terms = int(m.size)
        obs.masks = m.ctypes.data_as(C.POINTER(C.c_uint64)) if m.size else None
        obs.coeffs = c.ctypes.data_as(C.POINTER(C.c_double)) if c.size else None
        obs.d_diag = _ptr(diag)
        capi.ptsbe_backward(self.ctx, cid, info.set_id, first, count, obs, checkpoint_every, _ptr(loss), _ptr(per_set),
                            _ptr(grad_params), _ptr(grad_noise))

    def unique_shots(self, info: KrausSetInfo, first: int, count: int, bits, out):
        """out[a] (int64 device tensor) = number of distinct outcomes among the shots of set first + a."""
        capi.ptsbe_unique_shots(self.ctx, info.set_id, first, count, _ptr(bits), _ptr(out))

    def backward_plan_info(self, cid: int):
        """One- and two-qubit blocks, qubit-position swaps, differentiable blocks, and blocks before
        which the state is stored by the conditioning rule."""
        b1, b2, sw, nd, ck = capi.ptsbe_backward_plan_info(self.ctx, cid)
        return {"blocks_1q": b1, "blocks_2q": b2, "swaps": sw, "differentiable_blocks": nd,
                "conditioning_checkpoints": ck}

    def pershot(self, cid: int, seed: int, first_shot: int, n_shots: int, bits, kraus=None):
        capi.ptsbe_pershot_run(self.ctx, cid, seed, first_shot, n_shots, _ptr(bits), _ptr(kraus))
