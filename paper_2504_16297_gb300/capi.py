"""ctypes binding of the libptsbe C ABI (include/ptsbe.h): same function names, argument
marshalling only. Loading fails loudly when the library has not been built; there is no
fallback implementation."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

PTSBE_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_INVALID", 2: "ERR_NOT_CPTP", 3: "ERR_OOM", 4: "ERR_CUDA",
                5: "ERR_TIMEOUT", 6: "ERR_BUFFER_TOO_SMALL", 7: "ERR_UNSUPPORTED", 8: "ERR_NO_DEVICE"}

PTSBE_OP_GATE, PTSBE_OP_NOISE = 0, 1
(PTSBE_PTS_PROPORTIONAL, PTSBE_PTS_TOPK, PTSBE_PTS_BAND, PTSBE_PTS_TARGETED, PTSBE_PTS_LITERAL,
 PTSBE_PTS_PREDICATE) = range(6)
PTSBE_SHOTS_BY_COUNT, PTSBE_SHOTS_UNIFORM, PTSBE_SHOTS_BY_PROB, PTSBE_SHOTS_GIVEN = range(4)
PTSBE_EVOLVE_PREFIX_REUSE = 1
PTSBE_EVOLVE_PLAN_ONLY = 2
PTSBE_OPT_EVOLVE_KERNEL = 0
PTSBE_OPT_LIGHT_SHOTS = 1
PTSBE_OPT_PROGRAM_SETS_PER_WARP = 2
PTSBE_OPT_FAIL_ALLOC = 3
PTSBE_OPT_QUEUE_SPIN_CYCLES = 4
PTSBE_OPT_QUEUE_STALL_TASK = 5
PTSBE_OPT_SPLIT_FILL = 6
PTSBE_OPT_PERSHOT_TILE_BITS = 7
PTSBE_OPT_PREPASS_AHEAD = 8
PTSBE_BATCH_GRAPH = 1
(PTSBE_TIMER_EVOLVE_STAGE, PTSBE_TIMER_EVOLVE_FINALIZE, PTSBE_TIMER_SAMPLE, PTSBE_TIMER_PERSHOT,
 PTSBE_TIMER_EVOLVE_PROGRAM, PTSBE_TIMER_SAMPLE_LIGHT, PTSBE_TIMER_BACKWARD, PTSBE_TIMER_DENSE,
 PTSBE_TIMER_ZERO_FILL) = range(9)
PTSBE_TIMER_CLASSES = 9


class ptsbe_op(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("id", C.c_uint32), ("n_targets", C.c_uint32),
                ("targets", C.c_uint32 * 2), ("params", C.c_double * 3)]


class ptsbe_channel(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("arity", C.c_uint32), ("n_kraus", C.c_uint32),
                ("param", C.c_double), ("kraus", C.POINTER(C.c_double))]


class ptsbe_pts_params(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("shot_alloc", C.c_uint32), ("nsamples", C.c_uint64),
                ("k", C.c_uint64), ("p_min", C.c_double), ("p_max", C.c_double),
                ("total_shots", C.c_uint64), ("shots_per_set", C.c_uint64), ("t_count", C.c_uint32),
                ("t_offsets", C.POINTER(C.c_uint32)), ("t_sites", C.POINTER(C.c_uint32)),
                ("t_kidx", C.POINTER(C.c_uint8)), ("t_shots", C.POINTER(C.c_uint64)),
                ("max_errors", C.c_uint32), ("include_empty", C.c_uint32), ("qubit_mask", C.c_uint64),
                ("kraus_mask", C.c_uint32), ("gate_mask", C.c_uint32), ("site_lo", C.c_uint32),
                ("site_hi", C.c_uint32), ("weight_parity", C.c_uint32), ("max_sets", C.c_uint64)]


class ptsbe_set_view(C.Structure):
    _fields_ = [("offsets", C.c_void_p), ("sites", C.c_void_p), ("kidx", C.c_void_p),
                ("mult", C.c_void_p), ("q", C.c_void_p), ("shots", C.c_void_p),
                ("shot_offsets", C.c_void_p)]


class ptsbe_observable(C.Structure):
    _fields_ = [("n_terms", C.c_uint32), ("masks", C.POINTER(C.c_uint64)), ("coeffs", C.POINTER(C.c_double)),
                ("d_diag", C.c_void_p)]


class ptsbe_tuning(C.Structure):
    _fields_ = [("evolve_kernel", C.c_int32), ("light_shots", C.c_uint64), ("evolve_ms", C.c_double * 5),
                ("light_candidates", C.c_uint64 * 4), ("sample_ms", C.c_double * 4)]


class ptsbe_job(C.Structure):
    _fields_ = [("set_id", C.c_uint32), ("first", C.c_uint32), ("count", C.c_uint32), ("d_states", C.c_void_p),
                ("d_weights", C.c_void_p), ("d_status", C.c_void_p), ("seed", C.c_uint64), ("d_bits", C.c_void_p),
                ("d_bits_capacity", C.c_uint64)]


class PtsbeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_PROTOS = {
    "ptsbe_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "ptsbe_destroy": (C.c_int, [C.c_void_p]),
    "ptsbe_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ptsbe_last_error": (C.c_char_p, [C.c_void_p]),
    "ptsbe_synchronize": (C.c_int, [C.c_void_p]),
    "ptsbe_register_circuit": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(ptsbe_op), C.c_uint64,
                                         C.POINTER(ptsbe_channel), C.c_uint32, C.c_void_p, C.c_uint32,
                                         C.POINTER(C.c_uint32)]),
    "ptsbe_circuit_info": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                     C.POINTER(C.c_uint64)]),
    "ptsbe_release_circuit": (C.c_int, [C.c_void_p, C.c_uint32]),
    "ptsbe_sample_kraus": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(ptsbe_pts_params), C.c_uint64,
                                     C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                     C.POINTER(C.c_uint64)]),
    "ptsbe_set_export": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(ptsbe_set_view)]),
    "ptsbe_release_set": (C.c_int, [C.c_void_p, C.c_uint32]),
    "ptsbe_evolve_batch": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_uint32]),
    "ptsbe_sample_shots": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p,
                                     C.c_uint64, C.c_void_p, C.c_uint64]),
    "ptsbe_evolve_sample": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_uint32, C.c_uint64, C.c_void_p, C.c_uint64]),
    "ptsbe_sample_shots_noalloc": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_void_p,
                                             C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint64]),
    "ptsbe_backward": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                 C.POINTER(ptsbe_observable), C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "ptsbe_autotune": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_uint32, C.c_uint64, C.c_void_p, C.c_uint64, C.c_uint32, C.POINTER(ptsbe_tuning)]),
    "ptsbe_unique_shots": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p]),
    "ptsbe_backward_plan_info": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "ptsbe_kernel_launches": (C.c_int, [C.POINTER(C.c_uint64)]),
    "ptsbe_h2d_bytes": (C.c_int, [C.POINTER(C.c_uint64)]),
    "ptsbe_reuse_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "ptsbe_batch_plan": (C.c_int, [C.c_void_p, C.POINTER(ptsbe_job), C.c_uint32, C.POINTER(C.c_uint32)]),
    "ptsbe_batch_run": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32]),
    "ptsbe_batch_info": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                   C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)]),
    "ptsbe_batch_release": (C.c_int, [C.c_void_p, C.c_uint32]),
    "ptsbe_dense_work": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_double)]),
    "ptsbe_dense_plan_info": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                        C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_double)]),
    "ptsbe_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int64]),
    "ptsbe_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "ptsbe_get_timing": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_uint64),
                                   C.POINTER(C.c_double), C.c_int]),
    "ptsbe_pershot_run": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint64, C.c_void_p,
                                    C.c_void_p]),
}


def lib_path() -> str:
    return LIB


def load():
    """Loads libptsbe.so (built by paper_2504_16297_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libptsbe is not built ({LIB} missing): run __graft_entry__.build() "
                               "or python -m paper_2504_16297_gb300.build")
        lib = C.CDLL(LIB)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def declared_symbols():
    return list(_PROTOS)


def check(ctx, status: int):
    if status != PTSBE_OK:
        msg = load().ptsbe_last_error(ctx)
        raise PtsbeError(status, msg.decode() if msg else "")


# Thin wrappers with the C names (they raise PtsbeError on a non-OK status). ---------------------
def ptsbe_create(device: int = 0, stream: int | None = None):
    h = C.c_void_p()
    st = load().ptsbe_create(C.byref(h), device, stream)
    if st != PTSBE_OK:
        raise PtsbeError(st, "ptsbe_create failed")
    return h


def ptsbe_destroy(ctx):
    return load().ptsbe_destroy(ctx)


def ptsbe_set_stream(ctx, stream):
    check(ctx, load().ptsbe_set_stream(ctx, stream))


def ptsbe_synchronize(ctx):
    check(ctx, load().ptsbe_synchronize(ctx))


def ptsbe_last_error(ctx) -> str:
    return load().ptsbe_last_error(ctx).decode()


def ptsbe_register_circuit(ctx, n_qubits, ops, n_ops, channels, n_channels, custom, n_custom) -> int:
    cid = C.c_uint32()
    check(ctx, load().ptsbe_register_circuit(ctx, n_qubits, ops, n_ops, channels, n_channels, custom, n_custom,
                                             C.byref(cid)))
    return cid.value


def ptsbe_circuit_info(ctx, circuit_id):
    nq, ns, ng = C.c_uint32(), C.c_uint64(), C.c_uint64()
    check(ctx, load().ptsbe_circuit_info(ctx, circuit_id, C.byref(nq), C.byref(ns), C.byref(ng)))
    return nq.value, ns.value, ng.value


def ptsbe_release_circuit(ctx, circuit_id):
    check(ctx, load().ptsbe_release_circuit(ctx, circuit_id))


def ptsbe_sample_kraus(ctx, circuit_id, params: ptsbe_pts_params, seed: int):
    sid, cnt, ne, tot = C.c_uint32(), C.c_uint32(), C.c_uint64(), C.c_uint64()
    check(ctx, load().ptsbe_sample_kraus(ctx, circuit_id, C.byref(params), seed, C.byref(sid), C.byref(cnt),
                                         C.byref(ne), C.byref(tot)))
    return sid.value, cnt.value, ne.value, tot.value


def ptsbe_set_export(ctx, set_id, view: ptsbe_set_view):
    check(ctx, load().ptsbe_set_export(ctx, set_id, C.byref(view)))


def ptsbe_release_set(ctx, set_id):
    check(ctx, load().ptsbe_release_set(ctx, set_id))


def ptsbe_evolve_batch(ctx, set_id, first, count, d_states, d_weights, d_status, flags):
    check(ctx, load().ptsbe_evolve_batch(ctx, set_id, first, count, d_states, d_weights, d_status, flags))


def ptsbe_evolve_sample(ctx, set_id, first, count, d_states, d_weights, d_status, flags, seed, d_bits, capacity):
    check(ctx, load().ptsbe_evolve_sample(ctx, set_id, first, count, d_states, d_weights, d_status, flags, seed,
                                          d_bits, capacity))


def ptsbe_sample_shots(ctx, set_id, first, count, d_states, d_status, seed, d_bits, capacity):
    check(ctx, load().ptsbe_sample_shots(ctx, set_id, first, count, d_states, d_status, seed, d_bits, capacity))


def ptsbe_sample_shots_noalloc(ctx, set_id, first, count, d_states, d_status, seed, d_bits, capacity):
    check(ctx, load().ptsbe_sample_shots_noalloc(ctx, set_id, first, count, d_states, d_status, seed, d_bits, capacity))


def ptsbe_backward(ctx, circuit_id, set_id, first, count, obs: ptsbe_observable, checkpoint_every, d_loss,
                   d_per_set, d_grad_params, d_grad_noise):
    check(ctx, load().ptsbe_backward(ctx, circuit_id, set_id, first, count, C.byref(obs), checkpoint_every, d_loss,
                                     d_per_set, d_grad_params, d_grad_noise))


def ptsbe_autotune(ctx, set_id, first, count, d_states, d_weights, d_status, flags, seed, d_bits, capacity, reps):
    t = ptsbe_tuning()
    check(ctx, load().ptsbe_autotune(ctx, set_id, first, count, d_states, d_weights, d_status, flags, seed, d_bits,
                                     capacity, reps, C.byref(t)))
    return t


def ptsbe_unique_shots(ctx, set_id, first, count, d_bits, d_unique):
    check(ctx, load().ptsbe_unique_shots(ctx, set_id, first, count, d_bits, d_unique))


def ptsbe_backward_plan_info(ctx, circuit_id):
    v = [C.c_uint32() for _ in range(5)]
    check(ctx, load().ptsbe_backward_plan_info(ctx, circuit_id, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def ptsbe_kernel_launches() -> int:
    n = C.c_uint64()
    st = load().ptsbe_kernel_launches(C.byref(n))
    if st != PTSBE_OK:
        raise PtsbeError(st, "ptsbe_kernel_launches failed")
    return n.value


def ptsbe_h2d_bytes() -> int:
    n = C.c_uint64()
    st = load().ptsbe_h2d_bytes(C.byref(n))
    if st != PTSBE_OK:
        raise PtsbeError(st, "ptsbe_h2d_bytes failed")
    return n.value


def ptsbe_reuse_stats(ctx):
    a, f = C.c_uint64(), C.c_uint64()
    check(ctx, load().ptsbe_reuse_stats(ctx, C.byref(a), C.byref(f)))
    return a.value, f.value


def ptsbe_dense_work(ctx):
    n, f = C.c_uint64(), C.c_double()
    check(ctx, load().ptsbe_dense_work(ctx, C.byref(n), C.byref(f)))
    return n.value, f.value


def ptsbe_dense_plan_info(ctx, circuit_id):
    p, fx, b1, b2, f = C.c_uint32(), C.c_uint32(), C.c_uint64(), C.c_uint64(), C.c_double()
    check(ctx, load().ptsbe_dense_plan_info(ctx, circuit_id, C.byref(p), C.byref(fx), C.byref(b1), C.byref(b2),
                                            C.byref(f)))
    return p.value, fx.value, b1.value, b2.value, f.value


def ptsbe_batch_plan(ctx, jobs) -> int:
    arr = (ptsbe_job * max(len(jobs), 1))(*jobs)
    bid = C.c_uint32()
    check(ctx, load().ptsbe_batch_plan(ctx, arr, len(jobs), C.byref(bid)))
    return bid.value


def ptsbe_batch_run(ctx, batch_id, flags=0):
    check(ctx, load().ptsbe_batch_run(ctx, batch_id, flags))


def ptsbe_batch_info(ctx, batch_id):
    t, i, g, k = C.c_uint64(), C.c_uint64(), C.c_uint32(), C.c_uint64()
    check(ctx, load().ptsbe_batch_info(ctx, batch_id, C.byref(t), C.byref(i), C.byref(g), C.byref(k)))
    return t.value, i.value, g.value, k.value


def ptsbe_batch_release(ctx, batch_id):
    check(ctx, load().ptsbe_batch_release(ctx, batch_id))


def ptsbe_set_option(ctx, option: int, value: int):
    check(ctx, load().ptsbe_set_option(ctx, option, value))


def ptsbe_set_timing(ctx, enable: bool):
    check(ctx, load().ptsbe_set_timing(ctx, 1 if enable else 0))


def ptsbe_get_timing(ctx, kernel_class: int, reset: bool = False):
    ms, n, b = C.c_double(), C.c_uint64(), C.c_double()
    check(ctx, load().ptsbe_get_timing(ctx, kernel_class, C.byref(ms), C.byref(n), C.byref(b), 1 if reset else 0))
    return ms.value, n.value, b.value


def ptsbe_pershot_run(ctx, circuit_id, seed, first_shot, n_shots, d_bits, d_kraus):
    check(ctx, load().ptsbe_pershot_run(ctx, circuit_id, seed, first_shot, n_shots, d_bits, d_kraus))
