"""ctypes binding of libqfd.so (the C ABI declared in include/qfd.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of the library.  Arrays may be numpy arrays (host), or torch tensors on the
CUDA device (passed as device pointers) or in (pinned) host memory.
The binding refuses to work without the compiled library: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# QFD_LIBRARY selects another build of the same library (e.g. a tuning variant)
LIB_PATH = os.environ.get("QFD_LIBRARY") or os.path.join(_PKG, "libqfd.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "qfd.h")

OK, ERR_ARG, ERR_OOM, ERR_UNSTABLE_DT, ERR_DIVERGED, ERR_TIMEOUT, ERR_CUDA, ERR_NOT_CONVERGED, ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
STATUS_NAMES = {0: "QFD_OK", -1: "QFD_ERR_ARG", -2: "QFD_ERR_OOM", -3: "QFD_ERR_UNSTABLE_DT",
                -4: "QFD_ERR_DIVERGED", -5: "QFD_ERR_TIMEOUT", -6: "QFD_ERR_CUDA",
                -7: "QFD_ERR_NOT_CONVERGED", -8: "QFD_ERR_STATE"}
PRECISION = {"c128": 0, "c64_refine": 1, "c64": 2, "df64": 3, "c64_refine_df": 4}
CENTRE = {"grid": 0, "offgrid": 1}
POTENTIAL = {"zero": 0, "ho": 1, "cornell": 2, "coulomb": 3, "softcoul": 4}
STOP_RULE = {"paper": 0, "tail": 1}
PASS_KINDS = {"update_x": 0, "fwd_y": 1, "z_kinetic": 2, "inv_y": 3, "fwd_x": 4,
              "gs_dots": 5, "project_x": 6, "reduce": 7, "other": 8}


class QfdError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class QfdParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("a", ctypes.c_double), ("mass", ctypes.c_double),
                ("dtau", ctypes.c_double), ("kinetic", ctypes.c_int32), ("rest_mass", ctypes.c_int32),
                ("nstates", ctypes.c_int32), ("precision", ctypes.c_int32), ("ortho_every", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("centre", ctypes.c_int32), ("stop_rule", ctypes.c_int32),
                ("max_steps", ctypes.c_int64), ("tol", ctypes.c_double), ("tol_bulk", ctypes.c_double),
                ("stream", ctypes.c_void_p)]


class ServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_double), ("max_active", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("ortho_every", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("cohorts", ctypes.c_int32), ("autotune", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("a", ctypes.c_double), ("mass", ctypes.c_double), ("dtau", ctypes.c_double),
                ("kinetic", ctypes.c_int32), ("rest_mass", ctypes.c_int32), ("nstates", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("potential", ctypes.c_int32), ("stop_rule", ctypes.c_int32),
                ("pot_coeffs", ctypes.c_double * 2),
                ("centre", ctypes.c_int32), ("parity", ctypes.c_int32 * 8), ("seed", ctypes.c_uint64),
                ("max_steps", ctypes.c_int64), ("tol", ctypes.c_double), ("tol_bulk", ctypes.c_double),
                ("grf_amplitude", ctypes.c_double), ("grf_corr", ctypes.c_double), ("grf_seed", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("nstates", ctypes.c_int32),
                ("energy", ctypes.c_double * 8), ("steps", ctypes.c_int64 * 8), ("steps_c64", ctypes.c_int64 * 8),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


_lib = None


def header_functions():
    """Names of the functions include/qfd.h declares."""
    text = open(HEADER_PATH).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w*]+\s*\*?\s*(qfd_\w+)\s*\(", text, re.M)))


def load():
    """Loads libqfd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2006_16935_gb300.build.build_library()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "qfd_plan": (I, [ctypes.POINTER(QfdParams), ctypes.POINTER(P)]),
        "qfd_destroy": (None, [P]),
        "qfd_last_error": (ctypes.c_char_p, [P]),
        "qfd_set_potential": (I, [P, P, I]),
        "qfd_fill_potential": (I, [P, I, ctypes.POINTER(D), I]),
        "qfd_get_potential": (I, [P, P, I]),
        "qfd_add_random_field": (I, [P, ctypes.c_uint64, D, D]),
        "qfd_set_psi": (I, [P, I, P, I]),
        "qfd_fill_psi_uniform": (I, [P, I, ctypes.c_uint64]),
        "qfd_get_psi": (I, [P, I, P, I]),
        "qfd_set_parity": (I, [P, I, I]),
        "qfd_observables": (I, [P, I, D, ctypes.POINTER(D), I]),
        "qfd_step": (I, [P, I, I64]),
        "qfd_step_batch": (I, [ctypes.POINTER(P), ctypes.POINTER(I), I, I64]),
        "qfd_energy": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "qfd_solve_states": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "qfd_set_limits": (I, [P, I64, D, D]),
        "qfd_autotune": (I, [P, ctypes.POINTER(D)]),
        "qfd_set_tuning": (I, [P, I, I, I, I]),
        "qfd_has_tma": (I, [P]),
        "qfd_set_tma_test": (I, [P, I]),
        "qfd_snapshot_states": (I, [P, I, I, I64, ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "qfd_get_history": (I, [P, I, ctypes.POINTER(I64), ctypes.POINTER(D), I, ctypes.POINTER(I)]),
        "qfd_get_stats": (I, [P, I, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(D)]),
        "qfd_get_decay": (I, [P, I, ctypes.POINTER(D)]),
        "qfd_timing_enable": (I, [P, I]),
        "qfd_timing_reset": (I, [P]),
        "qfd_timing_query": (I, [P, I, ctypes.POINTER(I64), ctypes.POINTER(D)]),
        "qfd_launch_count": (I64, [P]),
        "qfd_fma_rate": (I, [I, ctypes.POINTER(D)]),
        "qfd_get_stream": (P, [P]),
        "qfd_sync": (I, [P]),
        "qfd_energy_noalloc": (I, [P, P, I64, D, D, I, I, P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "qfd_plan_bytes": (ctypes.c_size_t, [ctypes.POINTER(QfdParams)]),
        "qfd_server_create": (I, [ctypes.POINTER(ServerParams), ctypes.POINTER(P)]),
        "qfd_server_destroy": (None, [P]),
        "qfd_server_last_error": (ctypes.c_char_p, [P]),
        "qfd_server_clock": (D, [P]),
        "qfd_server_submit": (I, [P, ctypes.POINTER(Request), ctypes.POINTER(I64)]),
        "qfd_server_poll": (I, [P, ctypes.POINTER(Result), I, ctypes.POINTER(I)]),
        "qfd_server_set_timeout": (I, [P, D]),
        "qfd_server_kernels": (I, [P, ctypes.POINTER(I64)]),
        "qfd_server_stats": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I64),
                                 ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(arr, dtype):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor of `dtype` layout."""
    mod = type(arr).__module__
    if mod.startswith("torch"):
        import torch
        want = torch.complex128 if dtype == np.complex128 else torch.float64
        if arr.dtype != want or not arr.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return arr.data_ptr(), int(arr.is_cuda), arr
    a = np.ascontiguousarray(arr, dtype=dtype)
    return a.ctypes.data, 0, a


def fma_rate(fp64=True):
    """qfd_fma_rate: measured FMA rate (TFLOP/s) of the FP64 (or FP32) pipe of
    the current device."""
    lib = load()
    t = ctypes.c_double()
    st = lib.qfd_fma_rate(int(bool(fp64)), ctypes.byref(t))
    if st != OK:
        raise QfdError(st, "qfd_fma_rate failed")
    return t.value


def energy_noalloc(psi, V, n, a, mass, kinetic, rest_mass=0, stream=None):
    """qfd_energy_noalloc on device tensors psi (complex128, n^3) and V (float64, n^3):
    the energy and squared norm, evaluated without any device allocation (n <= 128)."""
    lib = load()
    pp, dev_p, keep_p = _ptr(psi, np.complex128)
    pv, dev_v, keep_v = _ptr(V, np.float64)
    if not (dev_p and dev_v):
        raise TypeError("psi and V must be CUDA device tensors")
    e, n2 = ctypes.c_double(), ctypes.c_double()
    st = lib.qfd_energy_noalloc(pp, pv, int(n), float(a), float(mass), int(kinetic), int(rest_mass), stream,
                                ctypes.byref(e), ctypes.byref(n2))
    if st != OK:
        raise QfdError(st, "qfd_energy_noalloc failed")
    del keep_p, keep_v
    return e.value, n2.value


class Plan:
    """One solver plan: a lattice, its kinetic term, potential and state stack."""

    def __init__(self, n, a, mass, dtau, kinetic, *, rest_mass=0, nstates=1, precision="c128",
                 ortho_every=10, check_every=100, centre="grid", max_steps=100000, tol=1e-9,
                 tol_bulk=1e-6, stop_rule="paper", stream=None):
        self.lib = load()
        self.n = int(n)
        p = QfdParams(n=self.n, a=a, mass=mass, dtau=dtau, kinetic=kinetic, rest_mass=rest_mass,
                      nstates=nstates, precision=PRECISION[precision], ortho_every=ortho_every,
                      check_every=check_every, centre=CENTRE[centre], stop_rule=STOP_RULE[stop_rule],
                      max_steps=max_steps,
                      tol=tol, tol_bulk=tol_bulk, stream=stream)
        self.params = p
        h = ctypes.c_void_p()
        st = self.lib.qfd_plan(ctypes.byref(p), ctypes.byref(h))
        if st != OK:
            raise QfdError(st, self.lib.qfd_last_error(None).decode())
        self.h = h

    # -- plumbing
    def _check(self, st, ok=(OK,)):
        if st not in ok:
            raise QfdError(st, self.lib.qfd_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.qfd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self):
        return (self.n, self.n, self.n)

    # -- inputs
    def set_potential(self, V):
        ptr, dev, keep = _ptr(V, np.float64)
        self._check(self.lib.qfd_set_potential(self.h, ptr, dev))
        del keep

    def fill_potential(self, kind, coeffs=()):
        c = (ctypes.c_double * max(1, len(coeffs)))(*coeffs)
        self._check(self.lib.qfd_fill_potential(self.h, POTENTIAL[kind], c, len(coeffs)))

    def add_random_field(self, seed, corr, amplitude):
        """qfd_add_random_field: V += seeded Gaussian random field (corr in lattice units)."""
        self._check(self.lib.qfd_add_random_field(self.h, int(seed), float(corr), float(amplitude)))

    def get_potential(self, out=None):
        if out is None:
            out = np.empty(self.shape, np.float64)
        ptr, dev, keep = _ptr(out, np.float64)
        self._check(self.lib.qfd_get_potential(self.h, ptr, dev))
        return out

    def set_psi(self, state, psi):
        ptr, dev, keep = _ptr(psi, np.complex128)
        self._check(self.lib.qfd_set_psi(self.h, state, ptr, dev))
        del keep

    def fill_psi_uniform(self, state, seed):
        self._check(self.lib.qfd_fill_psi_uniform(self.h, state, seed))

    def set_parity(self, state, parity):
        self._check(self.lib.qfd_set_parity(self.h, state, parity))

    # -- outputs
    def get_psi(self, state, out=None):
        if out is None:
            out = np.empty(self.shape, np.complex128)
        ptr, dev, keep = _ptr(out, np.complex128)
        self._check(self.lib.qfd_get_psi(self.h, state, ptr, dev))
        return out

    def observables(self, state=0, min_sep_edge=0.3):
        """dict of the observables of qfd_observables (lattice units)."""
        out = (ctypes.c_double * 12)()
        self._check(self.lib.qfd_observables(self.h, state, float(min_sep_edge), out, 12))
        keys = ["norm2", "norm2_box", "rho_box", "rho2", "x", "y", "z", "w_plus", "w_minus",
                "w_axis1", "w_axis2", "w_axis3"]
        return dict(zip(keys, list(out)))

    def step(self, state, nsteps):
        self._check(self.lib.qfd_step(self.h, state, nsteps))

    def energy(self, state=0):
        e, n2 = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.qfd_energy(self.h, state, ctypes.byref(e), ctypes.byref(n2)))
        return e.value, n2.value

    def solve_states(self, nstates, parity=None, allow_unconverged=False):
        par = (ctypes.c_int * nstates)(*(parity or [0] * nstates))
        es = (ctypes.c_double * nstates)()
        steps = (ctypes.c_int64 * nstates)()
        ok = (OK, ERR_NOT_CONVERGED) if allow_unconverged else (OK,)
        st = self._check(self.lib.qfd_solve_states(self.h, nstates, par, es, steps), ok)
        return list(es), list(steps), st == OK

    def snapshot_states(self, nout, parity=0, snap_every=None, allow_unconverged=False):
        """Excited states from the snapshots of one evolution of state 0
        (qfd_snapshot_states); returns (energies, steps, converged)."""
        es = (ctypes.c_double * nout)()
        steps = ctypes.c_int64()
        ok = (OK, ERR_NOT_CONVERGED) if allow_unconverged else (OK,)
        se = self.params.check_every if snap_every is None else snap_every
        st = self._check(self.lib.qfd_snapshot_states(self.h, nout, parity, int(se), es, ctypes.byref(steps)), ok)
        return list(es), steps.value, st == OK

    def autotune(self):
        """qfd_autotune; returns {policy: {"y": [default, wide, two-stage radix],
        "z": [1 group, 2 groups, two-stage radix], "x": [default, half width]}} in
        ms (NaN where not timed: the two-stage schedule exists for complex64 at
        n = 128..1024, the TMA pass A ("x"[2]) for complex64 at 256..1024, "x"
        needs a potential)."""
        ms = (ctypes.c_double * 27)()
        self._check(self.lib.qfd_autotune(self.h, ms))
        out = {}
        for pid, name in enumerate(("c128", "c64", "df64")):
            v = list(ms[9 * pid:9 * pid + 9])
            if not all(x != x for x in v):
                out[name] = {"y": v[:3], "z": v[3:6], "x": v[6:9]}
        return out

    def has_tma(self):
        """qfd_has_tma: whether the TMA-staged pass A is available to this plan."""
        return bool(self.lib.qfd_has_tma(self.h))

    def set_tma_test(self, arm_without_copies):
        """qfd_set_tma_test: 1 makes every bounded wait of the TMA pass A run out."""
        self._check(self.lib.qfd_set_tma_test(self.h, int(arm_without_copies)))

    def set_tuning(self, policy, y_variant, z_variant, x_variant=0):
        self._check(self.lib.qfd_set_tuning(self.h, int(policy), int(y_variant), int(z_variant), int(x_variant)))

    def set_limits(self, max_steps, tol, tol_bulk=None):
        tb = self.params.tol_bulk if tol_bulk is None else tol_bulk
        self._check(self.lib.qfd_set_limits(self.h, int(max_steps), float(tol), float(tb)))
        self.params.max_steps, self.params.tol, self.params.tol_bulk = int(max_steps), float(tol), float(tb)

    def history(self, state):
        """[(step, E)] of every check of the last solve of `state`."""
        cnt = ctypes.c_int()
        self._check(self.lib.qfd_get_history(self.h, state, None, None, 0, ctypes.byref(cnt)))
        n = cnt.value
        st = (ctypes.c_int64 * max(1, n))()
        es = (ctypes.c_double * max(1, n))()
        self._check(self.lib.qfd_get_history(self.h, state, st, es, n, ctypes.byref(cnt)))
        return [(st[i], es[i]) for i in range(n)]

    def decay_energy(self, state):
        """(1 - lambda) / dtau at the last check of `state` (qfd_get_decay)."""
        e = ctypes.c_double()
        self._check(self.lib.qfd_get_decay(self.h, state, ctypes.byref(e)))
        return e.value

    def stats(self, state):
        s64, s128, eb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        self._check(self.lib.qfd_get_stats(self.h, state, ctypes.byref(s64), ctypes.byref(s128), ctypes.byref(eb)))
        return {"steps_c64": s64.value, "steps_c128": s128.value, "e_bulk": eb.value}

    # -- instrumentation
    def timing(self, enable=True):
        self._check(self.lib.qfd_timing_enable(self.h, int(enable)))

    def timing_reset(self):
        self._check(self.lib.qfd_timing_reset(self.h))

    def timing_query(self, kind):
        n, ms = ctypes.c_int64(), ctypes.c_double()
        self._check(self.lib.qfd_timing_query(self.h, PASS_KINDS[kind] if isinstance(kind, str) else kind,
                                              ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def launch_count(self):
        return self.lib.qfd_launch_count(self.h)

    @property
    def stream(self):
        return self.lib.qfd_get_stream(self.h)

    def sync(self):
        self._check(self.lib.qfd_sync(self.h))


def make_request(n, a, mass, dtau, kinetic, *, rest_mass=0, nstates=1, precision="c128", potential="ho",
                 pot_coeffs=(1.0, 0.0), centre="grid", parity=None, seed=1, max_steps=100000, tol=1e-9,
                 tol_bulk=1e-10, stop_rule="paper", grf=None):
    """A qfd_request structure from keyword arguments; grf = (seed, corr,
    amplitude) adds a random field to the potential."""
    r = Request(n=n, a=a, mass=mass, dtau=dtau, kinetic=kinetic, rest_mass=rest_mass, nstates=nstates,
                precision=PRECISION[precision], potential=POTENTIAL[potential], stop_rule=STOP_RULE[stop_rule],
                centre=CENTRE[centre], seed=seed,
                max_steps=max_steps, tol=tol, tol_bulk=tol_bulk)
    r.pot_coeffs[0], r.pot_coeffs[1] = (list(pot_coeffs) + [0.0, 0.0])[:2]
    for i, v in enumerate(parity or [0] * nstates):
        r.parity[i] = v
    if grf is not None:
        r.grf_seed, r.grf_corr, r.grf_amplitude = int(grf[0]), float(grf[1]), float(grf[2])
    return r


class Server:
    """Continuous-batching request server of the C ABI (qfd_server_*)."""

    def __init__(self, hbm_budget_bytes, *, max_active=0, check_every=100, ortho_every=10, use_graphs=True,
                 stream=None, cohorts=False, autotune=False):
        self.lib = load()
        prm = ServerParams(hbm_budget_bytes=float(hbm_budget_bytes), max_active=max_active, check_every=check_every,
                           ortho_every=ortho_every, use_graphs=int(use_graphs), stream=stream,
                           cohorts=int(bool(cohorts)), autotune=int(bool(autotune)))
        h = ctypes.c_void_p()
        st = self.lib.qfd_server_create(ctypes.byref(prm), ctypes.byref(h))
        if st != OK:
            raise QfdError(st, "qfd_server_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.qfd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def clock(self):
        return self.lib.qfd_server_clock(self.h)

    def submit(self, request):
        rid = ctypes.c_int64()
        st = self.lib.qfd_server_submit(self.h, ctypes.byref(request), ctypes.byref(rid))
        if st != OK:
            raise QfdError(st, self.lib.qfd_server_last_error(self.h).decode())
        return rid.value

    def poll(self, capacity=256):
        buf = (Result * capacity)()
        cnt = ctypes.c_int()
        st = self.lib.qfd_server_poll(self.h, buf, capacity, ctypes.byref(cnt))
        if st != OK:
            raise QfdError(st, self.lib.qfd_server_last_error(self.h).decode())
        out = []
        for i in range(cnt.value):
            r = buf[i]
            out.append({"id": r.id, "status": r.status, "nstates": r.nstates,
                        "energy": [r.energy[k] for k in range(r.nstates)],
                        "steps": [r.steps[k] for k in range(r.nstates)],
                        "steps_c64": [r.steps_c64[k] for k in range(r.nstates)],
                        "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done})
        return out

    def set_timeout(self, seconds):
        """qfd_server_set_timeout: end a request whose period is still in flight
        `seconds` after it was queued with QFD_ERR_TIMEOUT (0 turns it off)."""
        st = self.lib.qfd_server_set_timeout(self.h, float(seconds))
        if st != OK:
            raise QfdError(st, self.lib.qfd_server_last_error(self.h).decode())

    def stats(self):
        w, a, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        per, rep, cap = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        st = self.lib.qfd_server_stats(self.h, ctypes.byref(w), ctypes.byref(a), ctypes.byref(u), ctypes.byref(per),
                                       ctypes.byref(rep), ctypes.byref(cap))
        if st != OK:
            raise QfdError(st, "qfd_server_stats failed")
        k = ctypes.c_int64()
        if self.lib.qfd_server_kernels(self.h, ctypes.byref(k)) != OK:
            raise QfdError(st, "qfd_server_kernels failed")
        return {"waiting": w.value, "active": a.value, "used_bytes": u.value, "periods": per.value,
                "graph_replays": rep.value, "graph_captures": cap.value, "kernels": k.value}

    def run_until_done(self, n_expected, capacity=256):
        """Polls until n_expected results have come back; returns them by id."""
        res = {}
        while len(res) < n_expected:
            for r in self.poll(capacity):
                res[r["id"]] = r
        return res


MAX_BATCH = 32  # QFD_MAX_BATCH


def step_batch(plans, states, nsteps):
    """qfd_step_batch: advances states[i] of plans[i] by nsteps steps, each pass
    of a step one launch over all the lattices (same n, arithmetic and FFT
    kinetic kind; at most MAX_BATCH plans)."""
    lib = load()
    plans = list(plans)
    if isinstance(states, int):
        states = [states] * len(plans)
    states = list(states)
    if len(states) != len(plans):
        raise ValueError(f"{len(plans)} plans but {len(states)} states")
    hs = (ctypes.c_void_p * max(1, len(plans)))(*[p.h for p in plans])
    ss = (ctypes.c_int * max(1, len(plans)))(*[int(s) for s in states])
    st = lib.qfd_step_batch(hs, ss, len(plans), int(nsteps))
    if st != OK:
        msg = lib.qfd_last_error(plans[0].h if plans and 1 <= len(plans) <= MAX_BATCH else None)
        raise QfdError(st, msg.decode() if msg else "")


def plan_bytes(n, precision="c128", nstates=1):
    """Device bytes of a plan (qfd_plan_bytes)."""
    p = QfdParams(n=n, a=1.0, mass=1.0, dtau=1e-6, kinetic=2, nstates=nstates, precision=PRECISION[precision],
                  ortho_every=1, check_every=1)
    return load().qfd_plan_bytes(ctypes.byref(p))
