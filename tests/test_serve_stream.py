"""The seeded request stream of the serving loop (host logic, no GPU)."""
import math

import numpy as np

from paper_2006_16935_gb300 import serve


def test_stream_is_seeded_and_shaped():
    a = serve.poisson_stream(400, seed=9)
    b = serve.poisson_stream(400, seed=9)
    assert a == b
    t = np.array([x[0] for x in a])
    assert np.all(np.diff(t) > 0)
    # exponential gaps of mean 1/20 s: the sample mean of 400 gaps is within 5 sigma
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 0.05) < 5 * 0.05 / math.sqrt(400)
    ns = [x[1]["n"] for x in a]
    counts = [ns.count(n) for n in serve.SIZES]
    assert counts == sorted(counts, reverse=True)  # weighted toward small lattices
    for _, r in a:
        assert r["kinetic"] in (1, 2, 3) and 1 <= r["nstates"] <= 3 and 1.0 <= r["mass"] <= 5.0
        assert 0.1 <= r["pot_coeffs"][0] <= 0.5 and 0.1 <= r["pot_coeffs"][1] <= 0.3
        assert r["parity"] == [1, -1, 1][:r["nstates"]]
        # half the update's stability limit dtau * max T = 2
        assert abs(r["dtau"] * serve.kinetic_max(r["kinetic"], r["a"], r["mass"], 0) - 1.0) < 1e-12


def test_kinetic_max_matches_the_mode_sum():
    a, m = 0.2, 1.7
    k = np.pi  # every axis at its Nyquist mode
    assert math.isclose(serve.kinetic_max(1, a, m), 3 * k * k / (2 * a * a * m))
    assert math.isclose(serve.kinetic_max(2, a, m), 3 * 4 * math.sin(k / 2) ** 2 / (2 * a * a * m))
    p2 = 3 * 4 * math.sin(k / 2) ** 2 / (a * a)
    assert math.isclose(serve.kinetic_max(3, a, m, 0), math.sqrt(p2 + m * m) - m)
    assert math.isclose(serve.kinetic_max(3, a, m, 1), math.sqrt(p2 + m * m))


def test_summary_of_records():
    recs = [{"n": 64, "arrival": 0.1 * i, "done": 0.1 * i + 1.0, "latency": 1.0, "status": 0, "steps": [100]}
            for i in range(10)]
    s = serve.summarize(recs)
    assert s["p50_s"] == 1.0 and s["p99_s"] == 1.0 and s["requests"] == 10 and s["ok"] == 10
    assert math.isclose(s["makespan_s"], 1.9) and math.isclose(s["solves_per_s"], 10 / 1.9)
    assert math.isclose(s["site_updates_per_s"], 10 * 64 ** 3 * 100 / 1.9)


def test_batch_stream_is_seeded_and_shaped():
    a = serve.batch_stream(64)
    assert a == serve.batch_stream(64)
    assert all(t == 0.0 for t, _ in a)
    sizes = {r["n"] for _, r in a}
    assert sizes == {64, 96, 128, 192}
    for _, r in a:
        assert r["a"] == 0.1 and r["stop_rule"] == "tail" and "parity" not in r
        seed, corr, amp = r["grf"]
        assert corr == 4.0 and amp == 0.05
        assert abs(r["dtau"] * serve.kinetic_max(r["kinetic"], r["a"], r["mass"], 0) - 1.0) < 1e-12
    assert len({r["grf"][0] for _, r in a}) == 64  # one field per solve
