#!/usr/bin/env python3
"""Throughput of the PTSBE hot path on one GB300 (or N, one process each).

Workload: the 17-qubit syndrome-extraction circuit (9 data + 8 ancilla qubits, 3 rounds, amplitude
damping 5e-4 + depolarising 1e-3 after every gate on every touched qubit, 390 noise sites), the
10^4 most likely Kraus sets (top-K pre-trajectory sampling), 10^8 shots recorded with their
Kraus-set labels. One step = register the circuit, run PTS on the host, prepare all 10^4 states
with prefix reuse (10.5 GB of complex64 states, larger than L2), draw the 10^8 shots.

Output: one JSON line (rank 0) with shots/s, the roofline of the dominant kernel (algorithmic
bytes per launch over CUDA-event time, against the measured HBM copy peak), the end-to-end figure
through host buffers, the CPU oracle timed on a bounded sample, and the clocks seen meanwhile.
`--impl reference` times the CPU oracle (the reference arm) on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "syndrome17_3rounds_top1e4_1e8shots"
DENSE30_SETS = 48
METRIC = "shots/s & gate-apply HBM GB/s, PTSBE batched vs per-shot trajectories, 1 GB300"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--k", type=int, default=10_000)
    ap.add_argument("--shots", type=int, default=100_000_000)
    ap.add_argument("--evolve-kernel", default="auto", choices=["auto", "frame", "sweep", "registers"])
    ap.add_argument("--e2e-copy", default="overlap", choices=["overlap", "serial"],
                    help="e2e device-to-host copies on a side stream or on the compute stream")
    ap.add_argument("--split-fill", type=int, default=0, metavar="PERCENT",
                    help="percentage of each state's zero fill run beside the program prepass (0: all in the evolve launch)")
    ap.add_argument("--no-prepass-ahead", action="store_true",
                    help="run the program prepass on the context stream (default: on the second stream, ahead of it)")
    ap.add_argument("--separate", action="store_true",
                    help="time ptsbe_evolve_batch + ptsbe_sample_shots instead of the one-call ptsbe_evolve_sample")
    ap.add_argument("--no-backward", action="store_true",
                    help="skip the adjoint-backward measurement (16-qubit ansatz, 4,096 samples)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (evolve kernel and sampler shot limit timed on the workload)")
    ap.add_argument("--backward-only", action="store_true",
                    help="run only the adjoint-backward measurement and print its JSON object")
    ap.add_argument("--backward-samples", type=int, default=4096)
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the uneven batch (512 brickwork circuits, 12-22 qubits, 64 samples each)")
    ap.add_argument("--uneven-only", action="store_true", help="run only the uneven batch and print its JSON object")
    ap.add_argument("--pershot-tile-bits", type=int, default=0, help="tile bits of the per-shot plan (0: default)")
    ap.add_argument("--pershot-shots", type=int, default=2048,
                    help="shots of the traditional per-shot path timed for comparison (0 = skip)")
    ap.add_argument("--dense30-sets", type=int, default=DENSE30_SETS,
                    help="Kraus sets of the 30-qubit workload timed in the dense leg, a prefix of the trie "
                         "(canonical) order (0 = skip the leg, -1 = the whole job)")
    ap.add_argument("--dense30-only", action="store_true", help="run only the 30-qubit dense leg and print it")
    ap.add_argument("--config0-only", action="store_true",
                    help="run only the 10-qubit PTSBE-against-per-shot comparison (a few MB on the device: the "
                         "profiling case of the per-operator kernels) and print it")
    ap.add_argument("--dense-probe", type=int, default=0, metavar="QUBITS",
                    help="prepare and sample one error-free brickwork set (16 layers) of QUBITS qubits with the "
                         "dense passes, states not returned, and print its timing (the profiling case)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # the sampler is running (its first line written) before the timed region starts
            t0 = time.perf_counter()
            while os.path.getsize(self.path) == 0 and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": num(rows[0][2]),
                "samples": len(rows), "reasons": sorted(reasons)}


def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, bytes_per_launch: float = 0.0, units: int = 0):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on the current source.
    A per-state record (a smaller capture of the same launch) is scaled to this launch: reads by the
    state count; writes by the further states' bytes and the difference between this launch's shot
    bytes (its algorithmic bytes beyond the states) and the capture's."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(kernel)
        if not e or e.get("source_sha") != source_sha(e["sources"]):
            return None
        c = e.get("capture")
        if e.get("model") == "per_amplitude" and c and units:
            return float((c["dram_bytes_read"] + c["dram_bytes_write"]) * units / c["amplitudes"])
        if e.get("model") == "per_state" and c and units:
            shot_bytes = bytes_per_launch - units * c["state_bytes"]
            return float(c["dram_bytes_read"] * units / c["states"] + c["dram_bytes_write"]
                         + (units - c["states"]) * c["state_bytes"] + (shot_bytes - c["shot_bytes"]))
        return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def inst_for(kernel: str, sets: int):
    """Warp instructions of one launch over `sets` Kraus sets, from a committed ncu count taken on
    the current source (None otherwise)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            e = json.load(f).get(kernel)
        if e and e.get("source_sha") == source_sha(e["sources"]):
            return float(e["warp_inst_per_set"]) * sets
    except Exception:
        pass
    return None


# ----------------------------------------------------------------------------------------------
# CPU oracle leg
# ----------------------------------------------------------------------------------------------
def oracle_estimate(budget_s: float, k: int, shots: int, seed: int, parts: dict | None = None):
    """Times the oracle on a bounded sample of the workload and extrapolates the whole job:
    top-K PTS once, state preparation of a few sets (each costs a full 17-qubit evolution), CDF
    construction and per-shot inverse-CDF draws. Returns (shots/s, description)."""
    from oracle import oracle as orc
    from workloads import config
    c = config(1)
    circ = c["circuit"]
    n = circ.n_qubits
    t0 = time.perf_counter()
    o = orc.Oracle(circ)
    sets = o.pts_topk(k, shots)
    t_pts = time.perf_counter() - t0
    picks = [0, 1, sets.count // 2, sets.count - 1]
    t_ev, n_ev = 0.0, 0
    psi0 = None
    while n_ev < len(picks) or (t_ev < 0.5 * budget_s and n_ev < 64):
        i = picks[n_ev % len(picks)] if n_ev < len(picks) else (n_ev * 7919) % sets.count
        t0 = time.perf_counter()
        psi, w, st = o.evolve(sets, i)
        t_ev += time.perf_counter() - t0
        if psi0 is None:
            psi0 = psi
        n_ev += 1
    t0 = time.perf_counter()
    orc.cdf(n, psi0)
    t_cdf = time.perf_counter() - t0
    m = 200_000
    t0 = time.perf_counter()
    while True:
        orc.sample(n, psi0, m, seed, 0)
        el = time.perf_counter() - t0
        if el > 0.2 * budget_s or m >= 4_000_000:
            break
        m *= 2
    t_shot = el / m   # includes one CDF build per call, negligible at this m
    total = t_pts + sets.count * (t_ev / n_ev + t_cdf) + shots * t_shot
    desc = (f"complex128 C oracle, 1 thread: top-{k} PTS once ({t_pts:.1f}s), {n_ev} of {sets.count} state "
            f"preparations ({t_ev / n_ev:.3f}s each), CDF build {t_cdf * 1e3:.1f} ms, {m} shots "
            f"({t_shot * 1e9:.0f} ns each); extrapolated to {sets.count} states + {shots} shots = {total:.0f}s")
    if parts is not None:
        parts.update(pts=t_pts, evolve=t_ev / n_ev, cdf=t_cdf, shot=t_shot)
    return shots / total, desc


_ORC = {}


def _orc_init(k, shots):
    """Worker of the all-cores oracle timing: the oracle and its top-K sets, built once per process."""
    from oracle import oracle as orc
    from workloads import config
    circ = config(1)["circuit"]
    o = orc.Oracle(circ)
    _ORC["o"] = o
    _ORC["sets"] = o.pts_topk(k, shots)


def _orc_evolve(i):
    o, sets = _ORC["o"], _ORC["sets"]
    o.evolve(sets, i % sets.count)
    return i


def _oracle_pool(k: int, shots: int):
    """One spawned oracle process per host core, each initialised with the workload and warm."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    cores = os.cpu_count() or 1
    ex = ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"), initializer=_orc_init,
                             initargs=(k, shots))
    list(ex.map(_orc_evolve, range(cores)))
    return ex, cores


def _oracle_pool_sample(ex, cores: int, k: int, shots: int, t_single: dict, n: int, offset: int = 0):
    """n state preparations of the workload spread over the pool: the job's shots/s extrapolated
    from them (PTS once on one core; CDF builds and shot draws divided over the cores)."""
    t0 = time.perf_counter()
    list(ex.map(_orc_evolve, [((offset + j) * 7919) % k for j in range(n)], chunksize=1))
    el = time.perf_counter() - t0
    per_state = el / n
    total = t_single["pts"] + k * (per_state + t_single["cdf"] / cores) + shots * t_single["shot"] / cores
    desc = (f"complex128 C oracle, {cores} processes (one per host core, spawned): {n} state preparations in "
            f"{el:.1f}s ({per_state * 1e3:.1f} ms per state over all cores); PTS once on one core "
            f"({t_single['pts']:.1f}s); CDF and shot draws divided over the cores; extrapolated to {k} states + "
            f"{shots} shots = {total:.0f}s")
    return shots / total, desc


def oracle_all_cores(k: int, shots: int, budget_s: float, t_single: dict):
    """The oracle as it stands, one process per host core (spawned), each preparing its share of
    the Kraus sets of the same workload: measured state preparations per second over all cores,
    extrapolated to the whole job like the one-thread estimate. Returns (shots/s, cores, desc)."""
    ex, cores = _oracle_pool(k, shots)
    try:
        n = max(cores, int(budget_s / max(t_single["evolve"], 1e-3)) * cores // 2)
        n = min(n, 16 * cores)
        v, desc = _oracle_pool_sample(ex, cores, k, shots, t_single, n)
    finally:
        ex.shutdown()
    return v, cores, desc


def result_errors(P, dev, info, states, weights, status, bits, seed, picks):
    """Error of the GPU results against the FP64 oracle for sampled Kraus sets (outside the timed
    region): relative 2-norm of the state, the largest relative error of any amplitude with
    |psi|^2 >= 1e-6 and of its probability, the weight, and the shots that differ from the oracle
    fed the GPU's own state (allowed only within 1e-6 of a CDF boundary)."""
    from oracle import oracle as orc
    from workloads import config
    circ = config(1)["circuit"]
    n = circ.n_qubits
    o = orc.Oracle(circ)
    out = []
    w_h, s_h = weights.cpu().numpy(), status.cpu().numpy()
    b_h = bits.cpu().numpy().view(np.uint32)
    for i in picks:
        ref = o.pts_targeted([info.entries(i)], shots=np.zeros(1, np.uint64))
        psi, wr, sr = o.evolve(ref, 0)
        g = states[i].cpu().numpy().astype(np.complex128)
        e = {"set": int(i), "errors": len(info.entries(i)), "status": int(s_h[i]), "oracle_status": int(sr)}
        if sr == 0:
            e["state_rel_2norm"] = float(np.linalg.norm(g - psi) / np.linalg.norm(psi))
            big = np.abs(psi) ** 2 >= 1e-6
            e["amp_max_rel"] = float((np.abs(g[big] - psi[big]) / np.abs(psi[big])).max())
            pg, pr = np.abs(g[big]) ** 2, np.abs(psi[big]) ** 2
            e["prob_max_rel"] = float((np.abs(pg - pr) / pr).max())
            e["weight_rel"] = float(abs(w_h[i] - wr) / wr)
            o0, o1 = int(info.shot_offsets[i]), int(info.shot_offsets[i + 1])
            m = min(o1 - o0, 200_000)
            want = orc.sample(n, g, m, seed, int(i))
            e["shots_checked"] = m
            e["shots_differing"] = int(np.count_nonzero(want != b_h[o0:o0 + m]))
        out.append(e)
    return out


def oracle_config0(seed: int = 2000):
    """The oracle on workload 0, the whole job on one core: PTS, every set's state, and every set's
    shots (its CDF and inverse-CDF draws). Returns (seconds, description)."""
    from oracle import oracle as orc
    from workloads import config
    c = config(0)
    circ = c["circuit"]
    n = circ.n_qubits
    t0 = time.perf_counter()
    o = orc.Oracle(circ)
    sets = o.pts_proportional(c["nsamples"], c["seed"], total_shots=c["total_shots"])
    for i in range(sets.count):
        psi, w, st = o.evolve(sets, i)
        m = int(sets.shots[i])
        if m and st == 0:
            orc.sample(n, psi, m, seed, i)
    el = time.perf_counter() - t0
    return el, (f"complex128 C oracle, 1 thread, the whole job: PTS, {sets.count} state preparations, "
                f"{int(np.sum(sets.shots))} shots in {el:.2f}s")


def oracle_dense30_estimate(ops30: int, sets: int, shots: int, n_small: int = 24):
    """The oracle on the 30-qubit workload, extrapolated: one error-free trajectory of a one-layer
    brickwork at n_small qubits (a state far larger than the host caches) is timed per operation
    and scaled by 2^(30 - n_small) per operation (each operation streams the whole state) to the
    30-qubit circuit's operations and sets; CDF and shot costs likewise. Returns (shots/s, desc)."""
    from oracle import oracle as orc
    from workloads import brickwork
    small = brickwork(n_small, 1, 5e-4, 5e-4, seed=1003)
    o = orc.Oracle(small)
    ks = o.pts_targeted([[]], shots=np.zeros(1, np.uint64))
    t0 = time.perf_counter()
    psi, w, st = o.evolve(ks, 0)
    t_ev = time.perf_counter() - t0
    t0 = time.perf_counter()
    orc.cdf(n_small, psi)
    t_cdf = time.perf_counter() - t0
    # each sample call builds the CDF once: the per-shot cost is the difference of two sizes
    t0 = time.perf_counter()
    orc.sample(n_small, psi, 100_000, 1, 0)
    t1 = time.perf_counter()
    orc.sample(n_small, psi, 2_100_000, 1, 0)
    t2 = time.perf_counter()
    t_shot = max((t2 - t1) - (t1 - t0), 0.0) / 2_000_000
    scale = float(1 << (30 - n_small))
    per_op = t_ev / small.n_ops
    total = sets * (per_op * scale * ops30 + t_cdf * scale) + shots * t_shot * 30.0 / n_small
    return shots / total, (f"complex128 C oracle, 1 thread: one {n_small}-qubit trajectory ({small.n_ops} operations, "
                           f"{per_op * 1e3:.1f} ms each, CDF {t_cdf:.2f}s, {t_shot * 1e9:.0f} ns per shot) scaled "
                           f"by 2^{30 - n_small} per operation to {ops30} operations x {sets} sets + {shots} shots "
                           f"= {total / 3600:.0f} h")


def config0_ratio(P, dev, seed: int = 2000, cpu: bool = False):
    """Workload 0 (10-qubit brickwork, 20 layers, 1,000 proportional samples, 10^5 shots): PTSBE
    (one call, prefix reuse) against the per-shot path (Algorithm 1) on the same GPU, same shots."""
    import torch
    from workloads import config
    c = config(0)
    circ = c["circuit"]
    n = circ.n_qubits
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=c["seed"], nsamples=c["nsamples"], total_shots=c["total_shots"])
    st = torch.empty((info.count, 1 << n), dtype=torch.complex64, device=dev)
    w = torch.empty(info.count, dtype=torch.float64, device=dev)
    s = torch.empty(info.count, dtype=torch.uint8, device=dev)
    bits = torch.empty(info.total_shots, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the evolve kernel and sampler shot limit tuned on this workload (outside the timing), as for
    # the main workload
    tuning = P.autotune(info, 0, info.count, st, w, s, seed, bits, prefix_reuse=True, reps=2)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    pt_ms = timed(lambda: P.evolve_sample(info, 0, info.count, st, w, s, seed, bits, prefix_reuse=True), 10)
    m = info.total_shots
    ps_bits = torch.empty(m, dtype=torch.int32, device=dev)
    ps_ms = timed(lambda: P.pershot(cid, seed, 0, m, ps_bits), 2)
    P.release_set(info)
    P.release_circuit(cid)
    out = {"workload": c["name"], "sets": info.count, "shots": m, "tuning": tuning, "ptsbe_ms": pt_ms, "pershot_ms": ps_ms,
           "ptsbe_shots_per_s": m / (pt_ms / 1e3), "pershot_shots_per_s": m / (ps_ms / 1e3),
           "ratio": ps_ms / pt_ms}
    if cpu:
        s_cpu, desc = oracle_config0(seed)
        out["cpu_oracle"] = {"value": m / s_cpu, "unit": "shots/s", "cores": 1, "kind": "oracle", "sample": desc}
    return out


def backward_leg(P, dev, reps: int = 3, cpu: bool = True, nsamples: int = 4096):
    """Adjoint gradients of the 16-qubit, 8-layer noisy ansatz (256 angles, damping and
    depolarising strengths) over 4,096 proportional samples: loss L = sum_i c_i <Z_i Z_i+1> of the
    fixed-set estimator and its 258 derivatives, timed with CUDA events on the launch stream."""
    import torch
    from workloads import ansatz
    circ = ansatz()
    n = circ.n_qubits
    cid = P.register(circ)
    info = P.sample_kraus(cid, "proportional", seed=2004, nsamples=nsamples, total_shots=nsamples)
    masks = np.array([(1 << i) | (1 << (i + 1)) for i in range(n - 1)], np.uint64)
    coeffs = np.asarray(circ.meta["zz_coeffs"])
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    gp = torch.empty((circ.n_ops, 3), dtype=torch.float64, device=dev)
    gn = torch.empty(len(circ.ch_params), dtype=torch.float64, device=dev)

    def once():
        P.backward(cid, info, 0, info.count, masks, coeffs, loss=loss, grad_params=gp, grad_noise=gn)
    once()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        once()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # FP32 roofline of the adjoint (state and adjoint stay on chip): useful FLOPs per set, a
    # complex multiply-add counted as 8 flops. Forward: B phi (one-qubit block 4 cmadd per pair,
    # two-qubit 16 per quad); reverse: B^-1 phi, the outer product and B^dag mu (3x that).
    plan = P.backward_plan_info(cid)
    per_amp = 8 * ((2 * plan["blocks_1q"] + 4 * plan["blocks_2q"]) * 4)      # fwd + 3x rev, per amplitude
    flops = float(info.count) * float(1 << n) * per_amp
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12              # FP32 FMA lanes x 2 x max clock
    out = {"workload": f"ansatz16_8layers_{nsamples}samples", "sets": info.count, "ms": ms,
           "plan": plan,
           "roofline": {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": flops / (ms / 1e3) / 1e12 / peak,
                        "peak_kind": "derived: SMs x 128 FP32 FMA lanes x 2 flops x 2.07 GHz (no measured FP32 peak)"},
           "sets_per_s": info.count / (ms / 1e3), "gradient_entries": 256 + 2, "loss": float(loss.cpu()[0]),
           "kernel": "k_backward (cluster of 8 CTAs per set, state and adjoint in DSMEM) + k_backward_finish"}
    if cpu:
        # oracle: one fixed-set loss evaluation of one set; a central-difference gradient needs
        # 2 x 258 + 1 of them per set
        from oracle import oracle as orc
        o = orc.Oracle(circ)
        one = o.pts_targeted([info.entries(info.count // 2)], shots=np.zeros(1, np.uint64))
        t0 = time.perf_counter()
        o.loss(one, masks, coeffs)
        t = time.perf_counter() - t0
        out["cpu_fd_oracle"] = {"s_per_loss_eval": t, "s_per_set_gradient": t * (2 * 258 + 1), "cores": 1,
                                "kind": "oracle central differences, extrapolated from one loss evaluation"}
    P.release_set(info)
    P.release_circuit(cid)
    return out


def uneven_leg(dev, reps: int = 2, margin_gb: float = 24.0):
    """The uneven batch: 512 brickwork circuits (n ~ U{12..22}, depth ~ U{10..40}, DEPOL1 1e-3 after
    every U3, DEPOL2 1e-2 after every CX), 64 proportional samples each, shot budgets
    ~ LogUniform(1e3, 1e6). Registration, PTS and the batch plan run on the host once (timed
    apart); every run is ONE persistent cooperative launch (a device work queue) that prepares all
    28,769 states (181 GB of complex64) with dense passes, then the samplers draw the 7.08x10^7
    shots. The run is captured as a CUDA graph and replayed; the timed region is `reps` replays,
    CUDA events on the launch stream. If the device cannot hold every state at once, the circuits
    are split into chunks, one launch (and graph) each, and the line says so."""
    import torch
    from paper_2504_16297_gb300.runtime import Ptsbe
    from workloads import config
    cfg = config(2)
    circs, shots = cfg["circuits"], cfg["shots"]
    # a stream of its own: the legacy default stream cannot be captured into a graph
    side = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    P = Ptsbe(device=dev.index if dev.index is not None else 0, stream=side.cuda_stream)
    t0 = time.perf_counter()
    infos = []
    for i, circ in enumerate(circs):
        cid = P.register(circ)
        infos.append((circ, cid, P.sample_kraus(cid, "proportional", seed=cfg["seed"] + i, nsamples=cfg["nsamples"],
                                                 total_shots=int(shots[i]))))
    t_pts = time.perf_counter() - t0
    need = sum(info.count * (8 << circ.n_qubits) for circ, _, info in infos)
    free, _ = torch.cuda.mem_get_info(dev)
    budget = max(1.0, free - margin_gb * 2 ** 30)
    chunks, cur, cur_b = [], [], 0
    for k, (circ, cid, info) in enumerate(infos):
        b = info.count * (8 << circ.n_qubits)
        if cur and cur_b + b > budget:
            chunks.append(cur)
            cur, cur_b = [], 0
        cur.append(k)
        cur_b += b
    if cur:
        chunks.append(cur)
    # the states of a chunk are views into one flat buffer; chunks run one after another on the
    # stream, each reusing the same memory (one chunk: every state at once)
    chunk_amps = [sum(infos[k][2].count << infos[k][0].n_qubits for k in ch) for ch in chunks]
    flat = torch.empty(max(chunk_amps), dtype=torch.complex64, device=dev)
    bufs = []
    for circ, cid, info in infos:
        bufs.append([None, torch.empty(info.count, dtype=torch.float64, device=dev),
                     torch.empty(info.count, dtype=torch.uint8, device=dev),
                     torch.empty(max(info.total_shots, 1), dtype=torch.int32, device=dev)])
    for ch in chunks:
        off = 0
        for k in ch:
            circ, _, info = infos[k]
            m = info.count << circ.n_qubits
            bufs[k][0] = flat[off:off + m].view(info.count, 1 << circ.n_qubits)
            off += m
    t0 = time.perf_counter()
    batches = []
    for ch in chunks:
        jobs = [(infos[k][2], 0, infos[k][2].count, bufs[k][0], bufs[k][1], bufs[k][2], 7000 + k, bufs[k][3]) for k in ch]
        batches.append(P.batch_plan(jobs))
    t_plan = time.perf_counter() - t0
    info0 = [P.batch_info(b) for b in batches]
    torch.cuda.synchronize()                 # the buffers were made on the default stream
    stream = side
    for b in batches:
        P.batch_run(b)                  # warm-up (plain launches)
    for b in batches:
        P.batch_run(b, graph=True)      # captures each chunk's graph and launches it
    P.synchronize()
    torch.cuda.synchronize()
    clk = Clocks(dev.index if dev.index is not None else 0)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        for b in batches:
            P.batch_run(b, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    P.synchronize()
    ms = e0.elapsed_time(e1) / reps
    total_shots = int(sum(int(info.total_shots) for _, _, info in infos))
    sets = int(sum(info.count for _, _, info in infos))
    logical_gates = float(sum(info.count * circ.n_gates for circ, _, info in infos))
    null = int(sum(int(b[2].sum().item()) for b in bufs))
    for b in batches:
        P.batch_release(b)
    P.close()
    del flat, bufs
    return {"workload": cfg["name"], "circuits": len(circs), "sets": sets, "shots": total_shots,
            "state_bytes": need, "launch_chunks": len(chunks), "ms_per_run": ms, "shots_per_s": total_shots / (ms / 1e3),
            "trajectory_gates_per_s": logical_gates / (ms / 1e3), "null_sets": null,
            "queue": info0, "host_pts_s": t_pts, "host_plan_s": t_plan, "reps": reps, "clocks": clocks,
            "kind": ("one persistent cooperative launch (device work queue, bounded waits) per run over all circuits, "
                     "then the samplers; replayed as a CUDA graph")}


def dense30_leg(P, dev, max_sets: int, clocks_index: int, seed: int = 2003, cpu: bool = False):
    """The 30-qubit workload: brickwork, 60 layers (1,800 U3 + 870 CX), DEPOL1 after every U3 and
    DEPOL2 after every CX at p = 5e-4, 2,000 proportional samples, 10^9 shots. States (8 GiB each)
    are not returned: ptsbe_evolve_sample prepares the sets branch by branch with dense passes
    (prefix reuse: sets share the state up to the pass of their first entry) and samples each from
    its global-memory CDF. Timed with CUDA events on the launch stream: a prefix of the sets in
    canonical (trie) order -- the error-free set, then the sets by first error site -- or the whole
    job. The full job's schedule is planned (no device work) for its prefix-reuse savings."""
    import torch
    from workloads import config
    from paper_2504_16297_gb300 import capi
    c = config(3)
    circ = c["circuit"]
    n = circ.n_qubits
    cid = P.register(circ)
    t0 = time.perf_counter()
    info = P.sample_kraus(cid, "proportional", seed=c["seed"], nsamples=c["nsamples"], total_shots=c["total_shots"])
    t_pts = time.perf_counter() - t0
    plan = P.dense_plan_info(cid)
    full_applied, full_nominal = P.plan(info, 0, info.count)
    count = info.count if max_sets < 0 else min(max_sets, info.count)
    shots = int(info.shot_offsets[count])
    w = torch.empty(count, dtype=torch.float64, device=dev)
    s = torch.empty(count, dtype=torch.uint8, device=dev)
    bits = torch.empty(max(shots, 1), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # warm-up: uploads, workspace, library buffers (one set)
    P.evolve_sample(info, 0, 1, None, w, s, seed, bits)
    torch.cuda.synchronize()
    P.set_timing(True)
    for k in range(capi.PTSBE_TIMER_CLASSES):
        P.timing(k, reset=True)
    clk = Clocks(clocks_index)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    P.evolve_sample(info, 0, count, None, w, s, seed, bits)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    applied, nominal = P.reuse_stats()
    launches, fma = P.dense_work()
    kern = {}
    for cls, name in [(capi.PTSBE_TIMER_DENSE, "dense_pass"), (capi.PTSBE_TIMER_EVOLVE_FINALIZE, "finalize"),
                      (capi.PTSBE_TIMER_SAMPLE, "sample"), (capi.PTSBE_TIMER_SAMPLE_LIGHT, "sample_light")]:
        kms, kl, kb = P.timing(cls, reset=True)
        if kl:
            kern[name] = {"ms": kms, "launches": kl, "bytes": kb}
    P.set_timing(False)
    null = int(s.sum().item())
    # the traditional per-shot path on this workload: one trajectory prepared from |0...0> for one
    # shot (for these unitary-mixture channels Algorithm 1's Kraus draws do not depend on the state,
    # so a shot costs one full preparation); timed on the error-free trajectory
    one = P.sample_kraus(cid, "targeted", targeted=[[]], targeted_shots=np.array([1], np.uint64))
    b1 = torch.empty(1, dtype=torch.int32, device=dev)
    P.evolve_sample(one, 0, 1, None, w, s, seed, b1)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    P.evolve_sample(one, 0, 1, None, w, s, seed, b1)
    f1.record(stream)
    torch.cuda.synchronize()
    ps_ms = f0.elapsed_time(f1)
    P.release_set(one)
    hbm_peak, hbm_kind = peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    alu_peak = n_sm * 128 * 2 * mhz * 1e6 / 1e12             # FP32 TFLOP/s: SMs x 128 FMA lanes x 2 x clock
    d = kern.get("dense_pass")
    dense = None
    if d:
        gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
        tfl = 2 * fma / (d["ms"] / 1e3) / 1e12
        dense = {"ms": d["ms"], "launches": d["launches"], "algorithmic_bytes": d["bytes"],
                 "gate_apply_gbs": gbs, "hbm_frac": gbs / hbm_peak, "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": hbm_kind,
                 "fma": fma, "fp32_tflops": tfl, "alu_frac": tfl / alu_peak, "alu_peak_tflops": alu_peak,
                 "alu_peak_kind": "derived: SMs x 128 FP32 lanes x 2 flops x median sampled SM clock",
                 "ms_per_pass_launch": d["ms"] / d["launches"]}
    est_s = None
    if applied:
        est_s = (ms / 1e3) * full_applied / applied
    out = {"workload": c["name"], "qubits": n, "layers": 60, "gates": circ.n_gates, "noise_sites": circ.n_sites,
           "sets_total": info.count, "sets_timed": count, "shots_total": info.total_shots, "shots_timed": shots,
           "timed": "whole job" if count == info.count else f"first {count} of {info.count} sets in canonical (trie) order",
           "ms": ms, "shots_per_s": shots / (ms / 1e3), "null_sets": null, "host_pts_s": t_pts,
           "trajectory_gates_per_s": {"applied": applied / (ms / 1e3), "logical": count * circ.n_gates / (ms / 1e3)},
           "prefix_reuse": {"timed_sets": {"gates_applied": applied, "gates_without_reuse": nominal,
                                           "savings": 1 - applied / nominal if nominal else None},
                            "full_job": {"gates_applied": full_applied, "gates_without_reuse": full_nominal,
                                         "savings": 1 - full_applied / full_nominal if full_nominal else None}},
           "plan": plan, "kernels": kern, "dense": dense,
           "roofline": ({"bound": "alu", "kernel": "k_dense_pass", "achieved": dense["fp32_tflops"], "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": dense["alu_frac"],
                         "traffic": traffic_for("dense_pass", units=1 << n)} if dense else None),
           "roofline_hbm": ({"bound": "hbm", "kernel": "k_dense_pass", "achieved": dense["gate_apply_gbs"],
                             "peak": hbm_peak, "unit": "GB/s", "frac": dense["hbm_frac"],
                             "traffic": traffic_for("dense_pass", units=1 << n)} if dense else None),
           "full_job_estimate_s": est_s,
           "pershot": {"value": 1.0 / (ps_ms / 1e3), "unit": "shots/s", "ms_per_shot": ps_ms,
                       "kind": "one full 30-qubit trajectory prepared per shot (dense passes, no reuse)"},
           "speedup_vs_pershot": (shots / (ms / 1e3)) / (1.0 / (ps_ms / 1e3)),
           "clocks": clocks}
    if cpu:
        v, desc = oracle_dense30_estimate(circ.n_ops, info.count, info.total_shots)
        out["cpu_oracle"] = {"value": v, "unit": "shots/s", "cores": 1, "kind": "oracle", "sample": desc}
    P.release_set(info)
    P.release_circuit(cid)
    del bits, w, s
    torch.cuda.empty_cache()
    return out


def two_in_flight(P, circ, dev, K: int, M: int, seed: int, tuning, split_fill: int, ahead: bool, steps: int = 20):
    """The same steps with two independent batches in flight: a second context on a second
    stream, steps alternating between the two (each its own states, weights, flags and shots).
    The latency-bound program prepass of one step overlaps the HBM-bound launches of the other.
    Timed with CUDA events across both streams. (A host thread per context measured the same: the
    device, not the host, sets the pace here.)"""
    import torch
    from paper_2504_16297_gb300.runtime import Ptsbe
    n = circ.n_qubits
    s2 = torch.cuda.Stream(dev)
    s1 = torch.cuda.current_stream(dev)
    Q = Ptsbe(device=dev.index or 0, stream=s2.cuda_stream)
    if tuning:                                   # the first context's autotuned choices
        Q.set_evolve_kernel(tuning["evolve_kernel"])
        Q.set_light_shots(int(tuning["light_shots"]))
    Q.set_split_fill(split_fill)
    Q.set_prepass_ahead(ahead)
    bufs = [(torch.empty((K, 1 << n), dtype=torch.complex64, device=dev), torch.empty(K, dtype=torch.float64, device=dev),
             torch.empty(K, dtype=torch.uint8, device=dev), torch.empty(M, dtype=torch.int32, device=dev)) for _ in range(2)]
    ctxs = [P, Q]

    def step(i):
        C = ctxs[i]
        st, w, s, b = bufs[i]
        cid = C.register(circ)
        info = C.sample_kraus(cid, "topk", k=K, total_shots=M, export=False)
        C.evolve_sample(info, 0, K, st, w, s, seed, b, prefix_reuse=True)
        C.release_set(info)
        C.release_circuit(cid)
    torch.cuda.synchronize()
    for _ in range(3):
        step(0)
        step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s1)
    s2.wait_event(e0)
    for k in range(steps):
        step(k % 2)
    s1.wait_stream(s2)
    e1.record(s1)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    Q.close()
    del bufs
    torch.cuda.empty_cache()
    return {"value": M / (ms / 1e3), "unit": "shots/s", "ms_per_step": ms, "steps": steps,
            "kind": "two contexts on two streams, steps alternating (two batches in flight)"}


def dense_probe(dev, n: int, layers: int = 16, seed: int = 1003):
    """One error-free set of an n-qubit brickwork (U3 layer + CX brickwork, `layers` times) prepared
    by the dense passes and sampled (1,000 shots), states not returned: the small case the dense
    pass kernel is profiled on. Three runs; the last is timed with CUDA events."""
    import torch
    from workloads import brickwork
    from paper_2504_16297_gb300 import capi
    from paper_2504_16297_gb300.runtime import Ptsbe
    P = Ptsbe(device=dev.index or 0, stream=torch.cuda.current_stream(dev).cuda_stream)
    circ = brickwork(n, layers, 5e-4, 5e-4, seed)
    cid = P.register(circ)
    info = P.sample_kraus(cid, "targeted", targeted=[[]], targeted_shots=np.array([1000], np.uint64))
    w = torch.empty(1, dtype=torch.float64, device=dev)
    s = torch.empty(1, dtype=torch.uint8, device=dev)
    bits = torch.empty(1000, dtype=torch.int32, device=dev)
    for _ in range(2):
        P.evolve_sample(info, 0, 1, None, w, s, 7, bits)
    torch.cuda.synchronize()
    P.set_timing(True)
    P.timing(capi.PTSBE_TIMER_DENSE, reset=True)
    P.evolve_sample(info, 0, 1, None, w, s, 7, bits)
    P.synchronize()
    dms, dl, db = P.timing(capi.PTSBE_TIMER_DENSE, reset=True)
    P.set_timing(False)
    out = {"qubits": n, "layers": layers, "passes": dl, "dense_ms": dms, "ms_per_pass": dms / max(dl, 1),
           "gate_apply_gbs": db / (dms / 1e3) / 1e9 if dms else None, "weight": float(w.item()),
           "status": int(s.item())}
    P.release_set(info)
    P.release_circuit(cid)
    P.close()
    return out


def workload_config(args, world: int) -> dict:
    """The measured workload, the same object on both arms of the bench."""
    return {"workload": WORKLOAD, "qubits": 17, "kraus_sets": args.k, "shots": args.shots, "pts": "topk",
            "prefix_reuse": True, "call": "evolve_batch + sample_shots" if args.separate else "evolve_sample",
            "amplitudes": "complex64, FP64 norms, CDF in 2^-62 fixed point (exact integer sums)",
            "l2": "inputs larger than L2 (10.5 GB of states per step)",
            "zero_fill": (f"{args.split_fill}% of each state on a second stream beside the program prepass, the rest in the evolve launch"
                          if args.split_fill else "in the evolve launch"),
            "prepass": ("on the context stream" if (args.no_prepass_ahead or args.split_fill) else
                        "ahead: uploads and program prepass on the context's second stream, overlapping the previous step"),
            "parallelism": f"{world} independent replicas (weak scaling)"}


def run_reference(args):
    """The reference arm: the oracle as it stands on the host's cores. The per-operation costs
    (PTS, one state, CDF, one shot) come from one bounded one-thread sample; then every step is a
    bounded sample of state preparations spread over one process per core (2 per core), and the
    line reports the median step. Falls back to the one-thread estimate without a process pool."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    parts = {}
    v1, desc1 = oracle_estimate(max(5.0, args.cpu_budget / 2), args.k, args.shots, 2001, parts)
    vals = []
    desc, cores = desc1, 1
    try:
        ex, cores = _oracle_pool(args.k, args.shots)
        try:
            for step in range(args.warmup + args.steps):
                v, desc = _oracle_pool_sample(ex, cores, args.k, args.shots, parts, 2 * cores, offset=step * 2 * cores)
                if step >= args.warmup:
                    vals.append(v)
        finally:
            ex.shutdown()
    except Exception as e:          # no process pool on this host: the one-thread figure stands
        vals, cores, desc = [v1], 1, f"all-cores run unavailable ({e}); {desc1}"
    val = float(np.median(vals))
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "shots/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "dtype": "f64", "data": "synthetic", "vs_baseline": None,
           "config": workload_config(args, args.gpus),
           "cpu_baseline": {"value": val, "unit": "shots/s", "cores": cores, "kind": "oracle", "sample": desc,
                            "single_thread": {"value": v1, "unit": "shots/s", "cores": 1, "sample": desc1}},
           "e2e": {"value": val, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------------------------
# Ranks (torchrun, one GPU each): weak scaling. Every rank prepares the same top-K Kraus sets and
# draws its own M shots (shot seed = base + rank), so ranks exchange no data; only the timing uses
# a barrier and a max over ranks, and the job's shots are world * M.
# ----------------------------------------------------------------------------------------------
def rank_seed(base: int, rank: int) -> int:
    return base + rank


def max_over_ranks(ms: float, dist, device) -> float:
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, shots_per_rank: int, ms_per_step: float) -> float:
    return world * shots_per_rank / (ms_per_step / 1e3)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    from paper_2504_16297_gb300 import build, capi
    from paper_2504_16297_gb300.runtime import Ptsbe
    from workloads import config
    build()

    if args.uneven_only:
        if rank == 0:
            print(json.dumps({"uneven": uneven_leg(torch.device("cuda", local))}), flush=True)
        return

    if args.config0_only:
        dev = torch.device("cuda", local)
        if rank == 0:
            P0 = Ptsbe(device=local, stream=torch.cuda.current_stream(dev).cuda_stream)
            print(json.dumps({"config0_vs_pershot": config0_ratio(P0, dev)}), flush=True)
            P0.close()
        return

    if args.dense_probe:
        if rank == 0:
            print(json.dumps({"dense_probe": dense_probe(torch.device("cuda", local), args.dense_probe)}), flush=True)
        return

    if args.dense30_only:
        dev = torch.device("cuda", local)
        P = Ptsbe(device=local, stream=torch.cuda.current_stream(dev).cuda_stream)
        d30 = dense30_leg(P, dev, args.dense30_sets, local)
        if rank == 0:
            print(json.dumps({"dense30": d30}), flush=True)
        return

    if args.backward_only:
        dev = torch.device("cuda", local)
        P = Ptsbe(device=local, stream=torch.cuda.current_stream(dev).cuda_stream)
        bw = backward_leg(P, dev, cpu=not args.no_cpu_baseline, nsamples=args.backward_samples)
        if rank == 0:
            print(json.dumps({"backward": bw}), flush=True)
        return

    cfg = config(1)
    circ = cfg["circuit"]
    n = circ.n_qubits
    K, M = args.k, args.shots
    seed = rank_seed(cfg["seed"], rank)   # weak scaling: every rank collects its own 1e8 shots
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    P = Ptsbe(device=local, stream=stream.cuda_stream)
    P.set_evolve_kernel(args.evolve_kernel)
    P.set_split_fill(args.split_fill)
    P.set_prepass_ahead(not args.no_prepass_ahead)
    states = torch.empty((K, 1 << n), dtype=torch.complex64, device=dev)
    # Results of consecutive steps alternate between two buffers, so the copy of step i's shots,
    # weights and flags to the host (its own stream) overlaps step i+1's kernels.
    weights = [torch.empty(K, dtype=torch.float64, device=dev) for _ in range(2)]
    status = [torch.empty(K, dtype=torch.uint8, device=dev) for _ in range(2)]
    bits = [torch.empty(M, dtype=torch.int32, device=dev) for _ in range(2)]
    host_bits = [torch.empty(M, dtype=torch.int32, pin_memory=True) for _ in range(2)]
    host_w = [torch.empty(K, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    host_s = [torch.empty(K, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    # e2e copies: on their own stream, overlapping the next step's kernels ("overlap"), or on the
    # compute stream after the step's kernels ("serial")
    copy_stream = torch.cuda.Stream(dev) if args.e2e_copy == "overlap" else stream
    done = [torch.cuda.Event(), torch.cuda.Event()]      # buffer b's copy finished
    h2d_bytes = [0]
    count = [0]

    def step(e2e: bool):
        b = count[0] % 2
        count[0] += 1
        cid = P.register(circ)
        info = P.sample_kraus(cid, "topk", k=K, total_shots=M, export=False)
        assert info.count == K and info.total_shots == M
        stream.wait_event(done[b])                        # buffer b is free again
        if args.separate:
            P.evolve(info, 0, K, states, weights[b], status[b], prefix_reuse=True)
            P.sample(info, 0, K, states, status[b], seed, bits[b])
        else:
            P.evolve_sample(info, 0, K, states, weights[b], status[b], seed, bits[b], prefix_reuse=True)
        if e2e:
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                host_bits[b].copy_(bits[b], non_blocking=True)
                host_w[b].copy_(weights[b], non_blocking=True)
                host_s[b].copy_(status[b], non_blocking=True)
            done[b].record(copy_stream)
        P.release_set(info)
        P.release_circuit(cid)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(e2e: bool, steps: int, instrument: bool):
        barrier()
        if instrument:
            P.set_timing(True)
            for cls in range(capi.PTSBE_TIMER_CLASSES):
                P.timing(cls, reset=True)
        l0 = capi.ptsbe_kernel_launches()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            step(e2e)
        stream.wait_stream(copy_stream)                   # the region ends after the last copy
        ev1.record(stream)
        barrier()
        ms = ev0.elapsed_time(ev1)
        launches = capi.ptsbe_kernel_launches() - l0
        kern = {}
        if instrument:
            for cls, name in [(capi.PTSBE_TIMER_EVOLVE_STAGE, "evolve_stage"), (capi.PTSBE_TIMER_EVOLVE_FINALIZE, "evolve_finalize"),
                              (capi.PTSBE_TIMER_SAMPLE, "sample"), (capi.PTSBE_TIMER_PERSHOT, "pershot"),
                              (capi.PTSBE_TIMER_EVOLVE_PROGRAM, "evolve_program"), (capi.PTSBE_TIMER_SAMPLE_LIGHT, "sample_light"),
                              (capi.PTSBE_TIMER_ZERO_FILL, "zero_fill")]:
                kms, kl, kb = P.timing(cls, reset=True)
                if kl:
                    kern[name] = {"ms": kms, "launches": kl, "bytes": kb}
            P.set_timing(False)
        return max_over_ranks(ms, dist, dev), launches, kern

    tuning = None
    if not args.no_autotune:
        # the library times its evolve kernels and sampler shot limits on this workload and keeps
        # the fastest (NEXT-1 autotuner); done before the warm-up, outside the timed region
        cid = P.register(circ)
        info = P.sample_kraus(cid, "topk", k=K, total_shots=M, export=False)
        tuning = P.autotune(info, 0, K, states, weights[0], status[0], seed, bits[0], prefix_reuse=True, reps=2)
        P.release_set(info)
        P.release_circuit(cid)
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(False)
    clocks = Clocks(local)
    clocks.start()
    ms, launches, kern = timed(False, args.steps, True)
    clk = clocks.stop()
    steps_e2e = max(2, args.steps)
    for _ in range(max(2, min(args.warmup, 3))):          # the first copies into the pinned buffers
        step(True)
    hb0 = capi.ptsbe_h2d_bytes()
    ms_e2e, _, _ = timed(True, steps_e2e, False)
    h2d_bytes[0] = (capi.ptsbe_h2d_bytes() - hb0) // steps_e2e

    # The legs below (comparator, oracle checks, the other workloads) run on one GPU only: under
    # torchrun they would hold every rank's GPU while rank 0 measures them.
    single = world == 1

    # Each leg below is measured outside the timed region; one that fails reports its error in its
    # key instead of taking the headline line with it.
    def leg(fn):
        try:
            return fn()
        except Exception as e:                       # noqa: BLE001 (reported, not hidden)
            torch.cuda.empty_cache()
            return {"error": f"{type(e).__name__}: {e}"[:400]}


    # Traditional trajectories (Algorithm 1) on the same GPU and workload: one prepared state per
    # shot, Kraus operators drawn during the evolution. Timed on a bounded number of shots.
    def pershot_leg():
        cid = P.register(circ)
        P.set_pershot_tile_bits(args.pershot_tile_bits)
        ps_bits = torch.empty(args.pershot_shots, dtype=torch.int32, device=dev)
        P.pershot(cid, seed, 0, min(64, args.pershot_shots), ps_bits)      # warm-up
        barrier()
        P.set_timing(True)
        P.timing(capi.PTSBE_TIMER_PERSHOT, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.pershot(cid, seed, 0, args.pershot_shots, ps_bits)
        e1.record(stream)
        barrier()
        ps_ms = e0.elapsed_time(e1)
        k_ms, k_launches, k_bytes = P.timing(capi.PTSBE_TIMER_PERSHOT, reset=True)
        P.set_timing(False)
        P.release_circuit(cid)
        del ps_bits
        # its own roofline: every stage reads and writes each state once (16 B per amplitude); its
        # stage kernels run back to back (the readout is timed with the samplers)
        ps_gbs = k_bytes / (k_ms / 1e3) / 1e9 if k_ms else None
        hbm_peak, hbm_kind = peaks()
        pershot = {"value": args.pershot_shots / (ps_ms / 1e3), "unit": "shots/s", "shots": args.pershot_shots,
                   "ms": ps_ms, "kind": "Algorithm 1 on the same GPU, same tile kernels, one state per shot",
                   "tile_bits": args.pershot_tile_bits or "default", "launches": k_launches, "algorithmic_bytes": k_bytes,
                   "roofline": {"bound": "hbm", "achieved": ps_gbs, "peak": hbm_peak, "unit": "GB/s",
                                "frac": ps_gbs / hbm_peak if ps_gbs else None, "peak_kind": hbm_kind}}
        return pershot

    pershot = leg(pershot_leg) if (args.pershot_shots > 0 and single) else None
    if pershot is not None and "error" in pershot:
        pershot_error, pershot = pershot, None
    else:
        pershot_error = None

    # unique-shot statistic (Sec. 4): distinct outcomes among the shots of the heaviest sets, from
    # one more step outside the timed region
    def unique_leg():
        cid = P.register(circ)
        info = P.sample_kraus(cid, "topk", k=K, total_shots=M)
        P.evolve_sample(info, 0, K, states, weights[0], status[0], seed, bits[0], prefix_reuse=True)
        top = 4
        u = torch.zeros(top, dtype=torch.int64, device=dev)
        P.unique_shots(info, 0, top, bits[0], u)
        torch.cuda.synchronize()
        uc = u.cpu().numpy()
        out = [{"set": a, "errors": len(info.entries(a)), "shots": int(info.shots[a]), "unique": int(uc[a]),
                "fraction": float(uc[a]) / max(1, int(info.shots[a]))} for a in range(top)]
        P.release_set(info)
        P.release_circuit(cid)
        return out

    uniq = leg(unique_leg) if rank == 0 else None

    def sampler_leg(reps: int = 5):
        """The samplers alone on the step's prepared states (ptsbe_sample_shots over the 10^4 sets
        and 10^8 shots, the states already in HBM), timed with CUDA events."""
        cid = P.register(circ)
        info = P.sample_kraus(cid, "topk", k=K, total_shots=M)
        P.evolve(info, 0, K, states, weights[0], status[0], prefix_reuse=True)
        P.sample(info, 0, K, states, status[0], seed, bits[0])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            P.sample(info, 0, K, states, status[0], seed, bits[0])
        e1.record(stream)
        torch.cuda.synchronize()
        ms_s = e0.elapsed_time(e1) / reps
        P.release_set(info)
        P.release_circuit(cid)
        return {"value": M / (ms_s / 1e3), "unit": "shots/s", "ms_per_call": ms_s,
                "kind": "ptsbe_sample_shots alone over the prepared states (support, light and cluster samplers)"}

    sampler = leg(sampler_leg) if (rank == 0 and single) else None

    def context_stream_leg():
        """The headline step with the program prepass on the context stream (no overlap with the
        previous step), for comparison."""
        P.set_prepass_ahead(False)
        try:
            for _ in range(3):
                step(False)
            ms1, _, kern1 = timed(False, args.steps, True)
        finally:
            P.set_prepass_ahead(True)
        return {"value": job_throughput(world, M, ms1 / args.steps), "unit": "shots/s",
                "ms_per_step": ms1 / args.steps, "steps": args.steps,
                "kernel_ms_per_step": {k: v["ms"] / args.steps for k, v in kern1.items()}, "kernels": kern1,
                "kind": "same step, program prepass on the context stream after the previous step"}

    prepass_serial = leg(context_stream_leg) if (single and not args.no_prepass_ahead and not args.split_fill) else None

    def errors_leg():
        cid = P.register(circ)
        info = P.sample_kraus(cid, "topk", k=K, total_shots=M)
        P.evolve_sample(info, 0, K, states, weights[0], status[0], seed, bits[0], prefix_reuse=True)
        torch.cuda.synchronize()
        out = result_errors(P, dev, info, states, weights[0], status[0], bits[0], seed, [0, 1, 2, K // 2, K - 1])
        P.release_set(info)
        P.release_circuit(cid)
        return out

    def config0_leg():
        P0 = Ptsbe(device=local, stream=stream.cuda_stream)
        try:
            return config0_ratio(P0, dev, cpu=(rank == 0 and world == 1 and not args.no_cpu_baseline))
        finally:
            P0.close()

    def dense30_leg_own():
        P30 = Ptsbe(device=local, stream=stream.cuda_stream)
        try:
            return dense30_leg(P30, dev, args.dense30_sets, local, cpu=(world == 1 and not args.no_cpu_baseline))
        finally:
            P30.close()
            torch.cuda.empty_cache()

    errors = c0 = overlap = bw = unev = d30 = None
    if rank == 0 and single:
        errors = leg(errors_leg)
        c0 = leg(config0_leg)
        overlap = leg(lambda: two_in_flight(P, circ, dev, K, M, seed, tuning, args.split_fill, not args.no_prepass_ahead))
    if not args.no_backward and single:
        bw = leg(lambda: backward_leg(P, dev, cpu=(rank == 0 and world == 1 and not args.no_cpu_baseline)))
    if args.dense30_sets != 0 and rank == 0 and single:
        d30 = leg(dense30_leg_own)
    if not args.no_uneven and rank == 0 and single:
        unev = leg(lambda: uneven_leg(dev))
        torch.cuda.empty_cache()

    ms_step = ms / args.steps
    value = job_throughput(world, M, ms_step)
    e2e_value = job_throughput(world, M, ms_e2e / steps_e2e)
    peak, peak_kind = peaks()
    # With the prepass ahead, the program prepass runs on the context's second stream beside the
    # previous step's launches, so its event span is not a time of its own: the dominant kernel
    # is taken among the launches on the context stream.
    ahead = not args.no_prepass_ahead and not args.split_fill
    critical = {k: v for k, v in kern.items() if not (ahead and k == "evolve_program")}
    dom = max(critical.items(), key=lambda kv: kv[1]["ms"])[0] if critical else None

    def hbm_roof(name, kern=kern):
        d = kern[name]
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": traffic_for(name, d["bytes"] / d["launches"], K), "bytes_per_launch": d["bytes"] / d["launches"],
                "ms_per_launch": d["ms"] / d["launches"]}

    roof, roof_hbm, roof_unshared = None, None, None
    if prepass_serial and "kernels" in prepass_serial and "evolve_stage" in prepass_serial["kernels"]:
        # the same kernel in the comparison leg, its launches not sharing the GPU with a prepass
        roof_unshared = hbm_roof("evolve_stage", prepass_serial["kernels"])
    byte_kernels = [k for k, v in kern.items() if v["bytes"] > 0]
    if byte_kernels:
        roof_hbm = hbm_roof(max(byte_kernels, key=lambda k: kern[k]["ms"]))
    if dom and kern[dom]["bytes"] > 0:
        roof = roof_hbm
    elif dom:
        # The program prepass moves almost no data: one serial builder chain per Kraus set, bound
        # by instruction issue and latency. Its roofline is the warp-instruction issue rate (one
        # warp instruction per cycle on each of the 4 schedulers of every SM) at the measured SM
        # clock, against the warp instructions one launch executes (ncu count of this source,
        # scaled by the sets of the launch).
        d = kern[dom]
        inst = inst_for(dom, K)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        peak_issue = 4 * n_sm * mhz * 1e6 / 1e9
        ms_launch = d["ms"] / d["launches"]
        achieved = inst / (ms_launch / 1e3) / 1e9 if inst else None
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_issue, "unit": "Gwarp-inst/s",
                "frac": (achieved / peak_issue) if achieved else None, "peak_kind": "4 schedulers x SMs x measured SM clock",
                "traffic": None, "warp_inst_per_launch": inst, "ms_per_launch": ms_launch}

    def cpu_leg():
        parts = {}
        v1, desc1 = oracle_estimate(args.cpu_budget, K, M, seed, parts)
        try:
            va, cores, desca = oracle_all_cores(K, M, args.cpu_budget, parts)
        except Exception as e:          # no process pool on this host: the one-thread figure stands
            va, cores, desca = v1, 1, f"all-cores run unavailable ({e}); {desc1}"
        return {"value": va, "unit": "shots/s", "cores": cores, "kind": "oracle", "sample": desca,
                "single_thread": {"value": v1, "unit": "shots/s", "cores": 1, "sample": desc1}}

    cpu = leg(cpu_leg) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None

    if rank == 0:
        gate_ms = kern.get("evolve_stage", {}).get("ms")
        prep = prepass_serial["kernels"] if (prepass_serial and "kernels" in prepass_serial) else kern
        out = {
            "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": workload_config(args, world),
            "tuning": tuning,
            "gate_apply_gbs": (kern["evolve_stage"]["bytes"] / (gate_ms / 1e3) / 1e9) if gate_ms else None,
            # logical gates x sets per second of preparation (program prepass + evolve launches,
            # from launches that do not overlap: the comparison leg's when the prepass runs ahead)
            "trajectory_gates_per_s": (circ.n_gates * K / ((prep["evolve_stage"]["ms"] + prep.get("evolve_program", {}).get("ms", 0.0))
                                                           / args.steps / 1e3)) if "evolve_stage" in prep else None,
            "sampler_alone": sampler,
            "pershot": pershot if pershot is not None else pershot_error,
            "speedup_vs_pershot": (value / world / pershot["value"]) if pershot else None,
            "kernels": kern,
            "roofline": roof,
            "roofline_hbm": roof_hbm if roof_hbm is not roof else None,
            "roofline_unshared": roof_unshared,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "shots/s", "h2d_bytes_per_step": h2d_bytes[0],
                    "d2h_bytes_per_step": M * 4 + K * 9, "copies": args.e2e_copy},
            "gpu_launches": launches,
            "clocks": clk,
            "backward": bw,
            "unique_shots": uniq,
            "errors_vs_oracle": errors,
            "config0_vs_pershot": c0,
            "prepass_on_context_stream": prepass_serial,
            "two_in_flight": overlap,
            "uneven": unev,
            "dense30": d30,
            "other_legs": None if single else "measured at N = 1 only (comparator, oracle checks, 30-qubit, uneven, backward)",
        }
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
