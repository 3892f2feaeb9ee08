"""ctypes wrapper around the complex128 C oracle (``ptsbe_oracle.c``) -- test infrastructure.

Passages: see the header of ``ptsbe_oracle.c`` (Sec. 2.2, Algorithms 1 and 2, Sec. 3, Sec. 3.1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptsbe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")


def oracle_lib_path() -> str:
    return os.path.join(_BUILD, "libptsbe_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no contraction)."""
    out = oracle_lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)
    return out


_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C")


def _load():
    lib = C.CDLL(build_oracle())
    vp = C.c_void_p
    lib.or_philox.argtypes = [_u32p, _u32p, _u32p]
    lib.or_u53.argtypes = [C.c_uint32, C.c_uint32]; lib.or_u53.restype = C.c_double
    lib.or_gate_matrix.argtypes = [C.c_int, _f64p, vp, _f64p]; lib.or_gate_matrix.restype = C.c_int
    lib.or_circuit_new.argtypes = [C.c_int, C.c_int, _i32p, _f64p, C.c_int, _i32p, _f64p, _f64p, _i64p,
                                   _f64p, C.c_int]
    lib.or_circuit_new.restype = vp
    lib.or_circuit_free.argtypes = [vp]
    lib.or_circuit_sites.argtypes = [vp]; lib.or_circuit_sites.restype = C.c_int
    lib.or_circuit_Q0.argtypes = [vp]; lib.or_circuit_Q0.restype = C.c_double
    lib.or_channel_info.argtypes = [vp, C.c_int, vp, vp, vp, vp]; lib.or_channel_info.restype = C.c_int
    lib.or_set_free.argtypes = [vp]
    lib.or_set_count.argtypes = [vp]; lib.or_set_count.restype = C.c_uint32
    lib.or_set_entries.argtypes = [vp]; lib.or_set_entries.restype = C.c_uint64
    lib.or_set_export.argtypes = [vp, _u32p, _u32p, _u8p, _u64p, _f64p, _u64p]
    lib.or_apportion_counts.argtypes = [C.c_uint32, _u64p, C.c_uint64, _u64p]
    lib.or_apportion_weights.argtypes = [C.c_uint32, _f64p, C.c_uint64, _u64p]
    lib.or_pts_proportional.argtypes = [vp, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int, C.c_uint64]
    lib.or_pts_proportional.restype = vp
    lib.or_pts_literal.argtypes = [vp, C.c_uint64, C.c_uint64, C.c_uint64]; lib.or_pts_literal.restype = vp
    lib.or_pts_topk.argtypes = [vp, C.c_uint64, C.c_uint64, C.c_int, C.c_uint64]; lib.or_pts_topk.restype = vp
    lib.or_pts_band.argtypes = [vp, C.c_double, C.c_double, C.c_uint64, C.c_int, C.c_uint64]
    lib.or_pts_band.restype = vp
    lib.or_pts_targeted.argtypes = [vp, C.c_uint32, _u32p, _u32p, _u8p, vp, C.c_uint64]
    lib.or_pts_targeted.restype = vp
    lib.or_evolve.argtypes = [vp, vp, C.c_uint32, _f64p, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.or_evolve.restype = C.c_int
    lib.or_cdf.argtypes = [C.c_int, _f64p, _f64p]
    lib.or_sample.argtypes = [C.c_int, _f64p, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint64, _u64p]
    lib.or_shot_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64]; lib.or_shot_uniform.restype = C.c_double
    lib.or_pershot.argtypes = [vp, C.c_uint64, C.c_uint64, vp]; lib.or_pershot.restype = C.c_uint64
    lib.or_loss.argtypes = [vp, vp, C.c_uint32, _u64p, _f64p, vp]; lib.or_loss.restype = C.c_double
    lib.or_loss_diag.argtypes = [vp, vp, C.c_uint32, _u64p, _f64p, vp, vp]; lib.or_loss_diag.restype = C.c_double
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = _load()
    return _LIB


class KrausSets:
    """Exported PTS result: CSR over sets in canonical order."""

    def __init__(self, handle):
        L = lib()
        n = L.or_set_count(handle)
        e = L.or_set_entries(handle)
        self.offsets = np.zeros(n + 1, np.uint32)
        self.sites = np.zeros(max(e, 1), np.uint32)
        self.kidx = np.zeros(max(e, 1), np.uint8)
        self.mult = np.zeros(max(n, 1), np.uint64)
        self.q = np.zeros(max(n, 1), np.float64)
        self.shots = np.zeros(max(n, 1), np.uint64)
        L.or_set_export(handle, self.offsets, self.sites, self.kidx, self.mult, self.q, self.shots)
        self.sites, self.kidx = self.sites[:e], self.kidx[:e]
        self.mult, self.q, self.shots = self.mult[:n], self.q[:n], self.shots[:n]
        self.count = n
        self.handle = handle

    def entries(self, i):
        b, e = int(self.offsets[i]), int(self.offsets[i + 1])
        return list(zip(self.sites[b:e].tolist(), self.kidx[b:e].tolist()))

    def free(self):
        if self.handle:
            lib().or_set_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Oracle:
    """One registered circuit on the CPU oracle."""

    def __init__(self, circ):
        L = lib()
        self.circ = circ
        self.n = circ.n_qubits
        kraus = np.ascontiguousarray(np.asarray(circ.ch_kraus, np.complex128).view(np.float64))
        if kraus.size == 0:
            kraus = np.zeros(2, np.float64)
        cg = np.ascontiguousarray(np.asarray(circ.custom_gates, np.complex128).view(np.float64).reshape(-1))
        if cg.size == 0:
            cg = np.zeros(32, np.float64)
        self.h = L.or_circuit_new(self.n, circ.n_ops, np.ascontiguousarray(circ.op_ints, np.int32).reshape(-1),
                                  np.ascontiguousarray(circ.op_params, np.float64).reshape(-1),
                                  len(circ.ch_params), np.ascontiguousarray(circ.ch_ints, np.int32).reshape(-1),
                                  np.ascontiguousarray(circ.ch_params, np.float64),
                                  kraus, np.ascontiguousarray(circ.ch_kraus_off, np.int64),
                                  cg, int(circ.custom_gates.shape[0]))
        if not self.h:
            raise ValueError("oracle rejected the circuit")
        self.n_sites = L.or_circuit_sites(self.h)
        self.Q0 = L.or_circuit_Q0(self.h)

    def __del__(self):
        try:
            if self.h:
                lib().or_circuit_free(self.h)
        except Exception:
            pass

    def channel(self, j):
        L = lib()
        c = self.circ.ch_ints[j]
        d = 1 << int(c[1])
        nk = int(c[2])
        kr = np.zeros(nk * d * d * 2, np.float64)
        q = np.zeros(nk, np.float64)
        mix = C.c_int(0)
        err = C.c_double(0)
        L.or_channel_info(self.h, j, kr.ctypes.data, q.ctypes.data, C.byref(mix), C.byref(err))
        return dict(kraus=kr.view(np.complex128).reshape(nk, d, d), q=q, mixture=bool(mix.value),
                    cptp_err=err.value)

    # --- PTS ---------------------------------------------------------------------------
    def pts_proportional(self, nsamples, seed, total_shots=0, alloc=0, nshots=0):
        return KrausSets(lib().or_pts_proportional(self.h, nsamples, seed, total_shots, alloc, nshots))

    def pts_literal(self, nsamples, seed, nshots):
        return KrausSets(lib().or_pts_literal(self.h, nsamples, seed, nshots))

    def pts_topk(self, k, total_shots, alloc=0, nshots=0):
        h = lib().or_pts_topk(self.h, k, total_shots, alloc, nshots)
        if not h:
            raise ValueError("top-k needs q_{s,0} to be the strict maximum at every site")
        return KrausSets(h)

    def pts_band(self, pmin, pmax, total_shots, alloc=0, nshots=0):
        h = lib().or_pts_band(self.h, pmin, pmax, total_shots, alloc, nshots)
        if not h:
            raise ValueError("band selection rejected")
        return KrausSets(h)

    def pts_targeted(self, sets, shots=None, total_shots=0):
        offsets = [0]
        sites, kidx = [], []
        for s in sets:
            for (site, k) in s:
                sites.append(site); kidx.append(k)
            offsets.append(len(sites))
        sh = None if shots is None else np.ascontiguousarray(shots, np.uint64)
        h = lib().or_pts_targeted(self.h, len(sets), np.asarray(offsets, np.uint32),
                                  np.asarray(sites + [0], np.uint32), np.asarray(kidx + [0], np.uint8),
                                  None if sh is None else sh.ctypes.data, total_shots)
        if not h:
            raise ValueError("invalid targeted set")
        return KrausSets(h)

    # --- BE ------------------------------------------------------------------------------
    def evolve(self, sets: KrausSets, i):
        st = np.zeros(2 << self.n, np.float64)
        w = C.c_double(0)
        status = C.c_int(0)
        rc = lib().or_evolve(self.h, sets.handle, i, st, C.byref(w), C.byref(status))
        if rc:
            raise IndexError(i)
        return st.view(np.complex128), w.value, status.value

    def pershot(self, seed, j, want_kraus=False):
        if want_kraus:
            kr = np.zeros(max(self.n_sites, 1), np.uint8)
            out = lib().or_pershot(self.h, seed, j, kr.ctypes.data)
            return out, kr[: self.n_sites]
        return lib().or_pershot(self.h, seed, j, None)

    def loss(self, sets: KrausSets, masks, coeffs, per_set=False, diag=None):
        """L = (1/N) sum_a mult_a <psi~_a|O|psi~_a> / q_a over the whole set (N = sum of mult), O the
        Z-string terms plus an optional dense diagonal; per_set: also e_a / q_a for every set."""
        masks = np.ascontiguousarray(masks, np.uint64).reshape(-1)
        coeffs = np.ascontiguousarray(coeffs, np.float64).reshape(-1)
        if masks.size == 0:
            masks, coeffs = np.zeros(1, np.uint64), np.zeros(1, np.float64)
        ps = np.zeros(max(sets.count, 1), np.float64)
        if diag is None:
            v = lib().or_loss(self.h, sets.handle, len(coeffs), masks, coeffs, ps.ctypes.data)
        else:
            d = np.ascontiguousarray(diag, np.float64)
            if d.size != 1 << self.n:
                raise ValueError("diag needs 2^n values")
            v = lib().or_loss_diag(self.h, sets.handle, len(coeffs), masks, coeffs, d.ctypes.data, ps.ctypes.data)
        return (v, ps[: sets.count]) if per_set else v


# Gate codes whose matrices depend on op params: RX, RY, RZ (theta) and U3 (theta, phi, lambda).
PARAM_GATES = {9: 1, 10: 1, 11: 1, 12: 3}


def gate_param_slots(circ):
    """(op index, param index) of every gate angle the circuit's matrices depend on."""
    out = []
    for i in range(circ.n_ops):
        kind, gid = int(circ.op_ints[i][0]), int(circ.op_ints[i][1])
        if kind == 0 and gid in PARAM_GATES:
            out += [(i, j) for j in range(PARAM_GATES[gid])]
    return out


def noise_param_slots(circ):
    """Channel indices whose Kraus operators are a function of their strength (the named kinds)."""
    return [j for j in range(len(circ.ch_params)) if int(circ.ch_ints[j][0]) != 5]


def _with_params(circ, op_params=None, ch_params=None):
    import dataclasses
    return dataclasses.replace(circ, op_params=circ.op_params if op_params is None else op_params,
                               ch_params=circ.ch_params if ch_params is None else ch_params)


def loss_grad_fd(circ, sets, masks, coeffs, h=1e-4, diag=None, param_slots=None, noise_slots=None):
    """Central finite differences of the fixed-set estimator (Sec. 3 with the Kraus sets and their
    nominal q_alpha held fixed) with respect to every gate angle and every named channel strength.

    Each perturbed circuit is a new oracle circuit (its matrices and Kraus operators rebuilt from
    the perturbed parameters); the sets, their multiplicities and q_alpha stay those of `sets`.
    Returns (per_set e_a/q_a [count], dper_params [n_ops, 3, count], dper_noise [n_ch, count]);
    the gradient of the loss over a range of sets is the mult-weighted mean of these rows.
    param_slots / noise_slots restrict the differences to those (op, j) pairs / channels (others 0)."""
    base = Oracle(circ)
    _, per = base.loss(sets, masks, coeffs, per_set=True, diag=diag)
    dp = np.zeros((circ.n_ops, 3, sets.count))
    dn = np.zeros((len(circ.ch_params), sets.count))
    for (i, j) in (gate_param_slots(circ) if param_slots is None else param_slots):
        vals = []
        for sgn in (+1.0, -1.0):
            P = np.array(circ.op_params, np.float64, copy=True)
            P[i, j] += sgn * h
            _, ps = Oracle(_with_params(circ, op_params=P)).loss(sets, masks, coeffs, per_set=True, diag=diag)
            vals.append(ps)
        dp[i, j] = (vals[0] - vals[1]) / (2 * h)
    for c in (noise_param_slots(circ) if noise_slots is None else noise_slots):
        vals = []
        for sgn in (+1.0, -1.0):
            P = np.array(circ.ch_params, np.float64, copy=True)
            P[c] += sgn * h
            _, ps = Oracle(_with_params(circ, ch_params=P)).loss(sets, masks, coeffs, per_set=True, diag=diag)
            vals.append(ps)
        dn[c] = (vals[0] - vals[1]) / (2 * h)
    return per, dp, dn


def predicate_sets(circ, max_errors, include_empty=False, qubit_mask=0, kraus_mask=0, gate_mask=0,
                   site_lo=0, site_hi=0, weight_parity=0):
    """Targeted error sets by rule (Sec. 3.1, "selection criteria"), written out from their
    definition: an error (s, k) is eligible when s lies in [site_lo, site_hi) (site_hi 0: every
    site), every qubit of the site is in qubit_mask, k >= 1 is in kraus_mask and the gate the site
    follows (the last gate before it sharing one of its qubits) is in gate_mask (a zero mask
    accepts all); the sets are all combinations of 1 .. max_errors eligible errors at distinct
    sites whose number of errors has the requested parity (0 any, 1 odd, 2 even), plus the empty
    set when include_empty. Returns them as (site, k) lists with increasing sites."""
    import itertools
    op_ints = np.asarray(circ.op_ints)
    noise_ops = [i for i in range(circ.n_ops) if op_ints[i][0] == 1]
    S = len(noise_ops)
    hi = S if site_hi == 0 else min(site_hi, S)

    def qubits(i):
        return [int(op_ints[i][3])] + ([int(op_ints[i][4])] if op_ints[i][2] == 2 else [])

    def gate_before(i):
        for j in range(i - 1, -1, -1):
            if op_ints[j][0] == 0 and set(qubits(j)) & set(qubits(i)):
                return int(op_ints[j][1])
        return None

    options = []
    for s in range(site_lo, hi):
        i = noise_ops[s]
        if qubit_mask and not all((qubit_mask >> q) & 1 for q in qubits(i)):
            continue
        if gate_mask:
            g = gate_before(i)
            if g is None or not (gate_mask >> g) & 1:
                continue
        nk = int(circ.ch_ints[int(op_ints[i][1])][2])
        ks = [k for k in range(1, nk) if not kraus_mask or (kraus_mask >> k) & 1]
        if ks:
            options.append((s, ks))
    out = [[]] if include_empty else []
    for w in range(1, max_errors + 1):
        if weight_parity == 1 and w % 2 == 0 or weight_parity == 2 and w % 2 == 1:
            continue
        for combo in itertools.combinations(options, w):
            for kk in itertools.product(*[ks for (_, ks) in combo]):
                out.append([(s, k) for (s, _), k in zip(combo, kk)])
    return out


def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().or_philox(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def u53(x0, x1):
    return lib().or_u53(int(x0), int(x1))


def gate_matrix(code, params=(0.0, 0.0, 0.0), custom=None):
    out = np.zeros(32, np.float64)
    cu = None if custom is None else np.ascontiguousarray(np.asarray(custom, np.complex128).view(np.float64))
    d = lib().or_gate_matrix(code, np.asarray(list(params) + [0.0] * (3 - len(params)), np.float64),
                             None if cu is None else cu.ctypes.data, out)
    return out[: 2 * d * d].view(np.complex128).reshape(d, d)


def cdf(n, state):
    st = np.ascontiguousarray(np.asarray(state, np.complex128).view(np.float64))
    C_ = np.zeros(1 << n, np.float64)
    lib().or_cdf(n, st, C_)
    return C_


def sample(n, state, m, seed, alpha, first_shot=0):
    st = np.ascontiguousarray(np.asarray(state, np.complex128).view(np.float64))
    out = np.zeros(max(m, 1), np.uint64)
    lib().or_sample(n, st, m, seed, alpha, first_shot, out)
    return out[:m]


def shot_uniform(seed, alpha, j):
    return lib().or_shot_uniform(seed, alpha, j)


def apportion_counts(c, M):
    c = np.ascontiguousarray(c, np.uint64)
    out = np.zeros(max(len(c), 1), np.uint64)
    lib().or_apportion_counts(len(c), c, M, out)
    return out[: len(c)]


def apportion_weights(w, M):
    w = np.ascontiguousarray(w, np.float64)
    out = np.zeros(max(len(w), 1), np.uint64)
    lib().or_apportion_weights(len(w), w, M, out)
    return out[: len(w)]
