"""Address and undefined-behaviour sanitizers on the host code, CPU only (`-m "not gpu"`).

The oracle (oracle/ptsbe_oracle.c) and the library's host-side planning and builder code (circuit
registration, frame plans, per-set frame programs and their tile steps, dense plans and override
blocks, run through the CPU harnesses tests/frame_host.cpp and tests/dense_host.cpp) are built
with -fsanitize=address,undefined (aborting at the first report) and run on circuits covering
every gate and channel kind, custom gates and channels, damping, multi-stage frame plans and
zero-padded dense plans. A clean exit means no out-of-bounds access, use after free, leak (the
oracle), overflow or other undefined behaviour on those paths."""
import os
import subprocess

import numpy as np
import pytest

from workloads import brickwork, syndrome17

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(ROOT, "paper_2504_16297_gb300", "csrc")
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g", "-O1"]


def _build(tmp, exe, cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(f"{exe} does not build:\n" + r.stderr[-3000:])
    return exe


@pytest.fixture(scope="module")
def drivers(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("san"))
    orc = _build(tmp, os.path.join(tmp, "san_oracle"),
                 ["gcc", "-std=gnu11", *SAN, os.path.join(HERE, "sanitize_oracle.c"),
                  os.path.join(ROOT, "oracle", "ptsbe_oracle.c"), "-lm", "-o", os.path.join(tmp, "san_oracle")])
    inc = ["-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include"]
    host = _build(tmp, os.path.join(tmp, "san_host"),
                  ["g++", "-std=c++17", *SAN, "-ffp-contract=off", *inc, os.path.join(HERE, "sanitize_host.cpp"),
                   os.path.join(HERE, "frame_host.cpp"), os.path.join(HERE, "dense_host.cpp"),
                   os.path.join(CSRC, "circuit.cpp"), os.path.join(CSRC, "dense_plan.cpp"),
                   "-o", os.path.join(tmp, "san_host")])
    return tmp, orc, host


def _dump(path, circ, sets=None):
    oi = np.ascontiguousarray(circ.op_ints, np.int32)
    op = np.ascontiguousarray(circ.op_params, np.float64)
    ci = np.ascontiguousarray(circ.ch_ints, np.int32)
    cp = np.ascontiguousarray(circ.ch_params, np.float64)
    kr = np.ascontiguousarray(circ.ch_kraus, np.complex128)
    ko = np.ascontiguousarray(circ.ch_kraus_off, np.int64)
    cg = np.ascontiguousarray(circ.custom_gates, np.complex128)
    with open(path, "wb") as f:
        np.array([circ.n_qubits, circ.n_ops, len(cp), kr.size, cg.shape[0]], np.int64).tofile(f)
        for a in (oi, op, ci, cp, kr.view(np.float64), ko, cg.view(np.float64)):
            a.tofile(f)
        if sets is not None:
            np.array([sets.count], np.int64).tofile(f)
            np.ascontiguousarray(sets.offsets, np.uint32).tofile(f)
            np.ascontiguousarray(sets.sites, np.uint32).tofile(f)
            np.ascontiguousarray(sets.kidx, np.uint8).tofile(f)
            np.ascontiguousarray(sets.q, np.float64).tofile(f)


def _circuits():
    from test_gpu_parity import _kitchen_sink
    return {"kitchen_sink_5": _kitchen_sink(5, seed=5), "brickwork_11": brickwork(11, 4, 0.02, 0.03, seed=11),
            "syndrome17_r1": syndrome17(rounds=1)}


def _run(exe, dump, leaks):
    env = dict(os.environ, ASAN_OPTIONS=f"detect_leaks={1 if leaks else 0}:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe, dump], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, f"{os.path.basename(exe)} on {os.path.basename(dump)}: exit {r.returncode}\n" + \
        (r.stderr[-4000:] or r.stdout[-2000:])
    assert "runtime error" not in r.stderr and "ERROR: AddressSanitizer" not in r.stderr, r.stderr[-4000:]


@pytest.mark.parametrize("name", ["kitchen_sink_5", "brickwork_11", "syndrome17_r1"])
def test_oracle_under_sanitizers(drivers, name):
    tmp, orc, _ = drivers
    dump = os.path.join(tmp, name + ".bin")
    _dump(dump, _circuits()[name])
    _run(orc, dump, leaks=True)


@pytest.mark.parametrize("name", ["kitchen_sink_5", "brickwork_11", "syndrome17_r1"])
def test_host_planning_and_builders_under_sanitizers(drivers, oracle_mod, name):
    tmp, _, host = drivers
    circ = _circuits()[name]
    sets = oracle_mod.Oracle(circ).pts_proportional(24, 5, total_shots=240)
    dump = os.path.join(tmp, name + "_sets.bin")
    _dump(dump, circ, sets)
    _run(host, dump, leaks=False)
