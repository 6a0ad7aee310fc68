"""Serving loop over the continuous-batching server (qfd_server_*).

A seeded Poisson stream of solve requests of mixed lattice sizes, kinetic
terms, masses and state counts is offered to the server as the requests
arrive; each request is a ground state plus up to two excited states (Gram-
Schmidt against the lower ones, Sec. 2.3) of a Cornell potential, solved to a
relative energy tolerance (Sec. 5.1, TOLERANCE).  The loop reports per-request
latency (arrival to result), its p50/p99 and the solves/s of the whole run.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import qfd

SIZES = (64, 128, 256, 512)
WEIGHTS = (0.4, 0.3, 0.2, 0.1)


def kinetic_max(kinetic: int, a: float, mass: float, rest_mass: int = 0) -> float:
    """Largest value of T(k) on the lattice (every axis at its Nyquist mode
    k a = pi): Eqs. (HK1)-(HK3)."""
    if kinetic == 1:
        return 3.0 * math.pi ** 2 / (2.0 * a * a * mass)
    if kinetic == 2:
        return 12.0 / (2.0 * a * a * mass)
    return math.sqrt(12.0 / (a * a) + mass * mass) - (0.0 if rest_mass else mass)


def poisson_stream(count: int, *, rate: float = 20.0, seed: int = 5, sizes=SIZES, weights=WEIGHTS, a: float = 0.2,
                   courant: float = 0.5, tol: float = 1e-9, stop_rule: str = "tail", max_steps: int = 400000):
    """`count` requests as (arrival seconds, request keywords): exponential gaps
    of mean 1/rate; n drawn from `sizes` with `weights`; kinetic term uniform
    over H_K(1..3) (H_K(3) without the rest mass); mass U[1,5]; 1-3 states with
    parities +, -, +; Cornell V = -alpha/r + sigma r with alpha U[0.1,0.5],
    sigma U[0.1,0.3]; spacing `a` for every size; dtau = courant * 2 / max T(k)
    (the update's stability limit); seeded uniform starts; every state solved
    to `tol` under `stop_rule` (the tail rule bounds the distance to the limit,
    the paper's rule only the last change)."""
    rng = np.random.default_rng(seed)
    w = np.asarray(weights, dtype=float)
    w = w / w.sum()
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.choice(np.asarray(sizes), p=w))
        kinetic = int(rng.integers(1, 4))
        mass = float(rng.uniform(1.0, 5.0))
        nstates = int(rng.integers(1, 4))
        alpha = float(rng.uniform(0.1, 0.5))
        sigma = float(rng.uniform(0.1, 0.3))
        dtau = courant * 2.0 / kinetic_max(kinetic, a, mass, 0)
        out.append((t, dict(n=n, a=a, mass=mass, dtau=dtau, kinetic=kinetic, rest_mass=0, nstates=nstates,
                            potential="cornell", pot_coeffs=(alpha, sigma), parity=[1, -1, 1][:nstates],
                            seed=1000 + 10 * i, tol=tol, tol_bulk=1e-10, stop_rule=stop_rule,
                            max_steps=max_steps)))
    return out


def batch_stream(count: int, *, seed: int = 4, sizes=(64, 96, 128, 192), a: float = 0.1, courant: float = 0.5,
                 tol: float = 1e-9, grf_corr: float = 4.0, grf_amplitude: float = 0.05, max_steps: int = 400000):
    """`count` independent solves, all present at time 0: n uniform over
    `sizes`; Cornell V = -alpha/r + sigma r with alpha U[0.1,0.5], sigma
    U[0.1,0.3], plus a seeded Gaussian random field (correlation length
    grf_corr lattice units, standard deviation grf_amplitude); kinetic term
    uniform over H_K(1..3); mass U[1,5]; 1-3 states without parity (the random
    field breaks the reflection symmetry); spacing `a`; dtau = courant * 2 /
    max T(k); tol under the tail rule."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(np.asarray(sizes)))
        kinetic = int(rng.integers(1, 4))
        mass = float(rng.uniform(1.0, 5.0))
        nstates = int(rng.integers(1, 4))
        alpha = float(rng.uniform(0.1, 0.5))
        sigma = float(rng.uniform(0.1, 0.3))
        dtau = courant * 2.0 / kinetic_max(kinetic, a, mass, 0)
        out.append((0.0, dict(n=n, a=a, mass=mass, dtau=dtau, kinetic=kinetic, rest_mass=0, nstates=nstates,
                              potential="cornell", pot_coeffs=(alpha, sigma), seed=2000 + 10 * i, tol=tol,
                              tol_bulk=1e-10, stop_rule="tail", max_steps=max_steps,
                              grf=(7000 + i, grf_corr, grf_amplitude))))
    return out


def serve(stream, precision: str, *, budget_bytes: float = 150e9, check_every: int = 100, ortho_every: int = 10,
          use_graphs: bool = True, stream_handle=None, max_active: int = 0, cohorts: bool = False,
          autotune: bool = False):
    """Offers `stream` (from poisson_stream) to a server in real time: each
    request is submitted once the server clock passes its arrival time; the
    loop polls until every result is back.  Returns (records, server stats);
    a record holds the request's arrival, admission and completion times
    (seconds from the start), latency, steps, energies and status."""
    recs = [None] * len(stream)
    ids = {}
    with qfd.Server(budget_bytes, check_every=check_every, ortho_every=ortho_every, use_graphs=use_graphs,
                    stream=stream_handle, max_active=max_active, cohorts=cohorts, autotune=autotune) as sv:
        t0 = sv.clock()
        nxt = 0
        got = 0
        while got < len(stream):
            now = sv.clock() - t0
            while nxt < len(stream) and stream[nxt][0] <= now:
                req = qfd.make_request(precision=precision, **stream[nxt][1])
                ids[sv.submit(req)] = nxt
                nxt += 1
            st = sv.stats()
            if st["active"] == 0 and st["waiting"] == 0:
                if nxt < len(stream):  # idle until the next arrival
                    time.sleep(max(0.0, stream[nxt][0] - (sv.clock() - t0)))
                continue
            for r in sv.poll():
                i = ids[r["id"]]
                arr, kw = stream[i]
                recs[i] = {"n": kw["n"], "kinetic": kw["kinetic"], "nstates": kw["nstates"], "arrival": arr,
                           "admit": r["t_admit"] - t0, "done": r["t_done"] - t0,
                           "latency": r["t_done"] - t0 - arr, "status": r["status"], "energy": r["energy"],
                           "steps": r["steps"], "steps_c64": r["steps_c64"]}
                got += 1
        stats = sv.stats()
    return recs, stats


def summarize(recs, stats=None):
    """p50/p99/mean latency, solves/s (requests / time from the first arrival
    to the last result), site-updates/s of a serving run, the same per lattice
    size, and (given the server stats) kernel launches per imaginary-time
    step of one lattice."""
    lat = np.array([r["latency"] for r in recs])
    first = min(r["arrival"] for r in recs)
    last = max(r["done"] for r in recs)
    span = last - first
    sites = sum(float(r["n"]) ** 3 * sum(r["steps"]) for r in recs)
    out = {"requests": len(recs), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "mean_s": float(lat.mean()), "max_s": float(lat.max()), "makespan_s": span,
           "solves_per_s": len(recs) / span, "site_updates_per_s": sites / span,
           "ok": sum(1 for r in recs if r["status"] == 0),
           "not_converged": sum(1 for r in recs if r["status"] == qfd.ERR_NOT_CONVERGED)}
    per = {}
    for n in sorted({r["n"] for r in recs}):
        rs = [r for r in recs if r["n"] == n]
        per[str(n)] = {"requests": len(rs), "site_updates_per_s": sum(float(n) ** 3 * sum(r["steps"]) for r in rs) / span,
                       "p50_s": float(np.percentile([r["latency"] for r in rs], 50))}
    out["per_size"] = per
    if stats is not None:
        steps = sum(sum(r["steps"]) for r in recs)
        out["kernel_launches"] = stats.get("kernels")
        out["launches_per_lattice_step"] = stats.get("kernels", 0) / max(1, steps)
    return out
