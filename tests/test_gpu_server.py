"""The request server (continuous batching): results are the same for a request
alone, in a mix with other requests, and through qfd_solve_states; admission
respects the device-memory budget; unchanged periods replay a CUDA graph."""
import pytest

from paper_2006_16935_gb300 import qfd as Q

pytestmark = pytest.mark.gpu

CHECK, ORTHO = 40, 10
REQS = [
    dict(n=16, a=0.4, mass=1.5, dtau=0.02, kinetic=3, nstates=2, precision="c128", potential="cornell",
         pot_coeffs=(0.3, 0.2), parity=[1, -1], seed=11, tol=1e-9, max_steps=20000),
    dict(n=32, a=0.2, mass=1.0, dtau=0.004, kinetic=2, nstates=1, precision="c64_refine_df", potential="ho",
         pot_coeffs=(1.0, 0.0), seed=12, tol=1e-9, max_steps=20000),
    dict(n=16, a=0.3, mass=2.0, dtau=0.01, kinetic=1, nstates=1, precision="df64", potential="softcoul",
         pot_coeffs=(0.01, 0.0), seed=13, tol=1e-9, max_steps=20000),
    dict(n=8, a=0.5, mass=1.0, dtau=0.05, kinetic=2, nstates=3, precision="c64_refine", potential="ho",
         pot_coeffs=(1.0, 0.0), parity=[1, -1, 1], seed=14, tol=1e-9, max_steps=20000),
]


def via_solve_states(req):
    with Q.Plan(req["n"], req["a"], req["mass"], req["dtau"], req["kinetic"], nstates=req["nstates"],
                precision=req["precision"], ortho_every=ORTHO, check_every=CHECK, max_steps=req["max_steps"],
                tol=req["tol"], tol_bulk=1e-10, centre=req.get("centre", "grid")) as p:
        p.fill_potential(req["potential"], req["pot_coeffs"])
        for s in range(req["nstates"]):
            p.fill_psi_uniform(s, req["seed"] + s)
        es, steps, _ = p.solve_states(req["nstates"], req.get("parity"), allow_unconverged=True)
    return es, steps


def run_server(reqs, budget=64e9, use_graphs=True, max_active=0):
    with Q.Server(budget, check_every=CHECK, ortho_every=ORTHO, use_graphs=use_graphs, max_active=max_active) as sv:
        ids = [sv.submit(Q.make_request(**r)) for r in reqs]
        res = sv.run_until_done(len(ids))
        return [res[i] for i in ids], sv.stats()


def test_results_same_alone_in_mix_and_through_solve_states(qfdlib):
    mix, stats = run_server(REQS)
    assert stats["graph_replays"] > 0 and stats["graph_captures"] > 0
    for req, got in zip(REQS, mix):
        assert got["status"] == 0
        alone, _ = run_server([req])
        es, steps = via_solve_states(req)
        assert got["energy"] == alone[0]["energy"] == es
        assert got["steps"] == alone[0]["steps"] == steps


def test_graph_replay_matches_direct_launches(qfdlib):
    a, _ = run_server(REQS[:2], use_graphs=True)
    b, _ = run_server(REQS[:2], use_graphs=False)
    assert [r["energy"] for r in a] == [r["energy"] for r in b]


def test_admission_respects_the_memory_budget(qfdlib):
    budget = 1.5 * max(Q.plan_bytes(r["n"], r["precision"], r["nstates"]) for r in REQS)
    with Q.Server(budget, check_every=CHECK, ortho_every=ORTHO) as sv:
        ids = [sv.submit(Q.make_request(**r)) for r in REQS]
        got = {}
        while len(got) < len(ids):
            st = sv.stats()
            assert st["used_bytes"] <= budget
            for r in sv.poll():
                got[r["id"]] = r
        assert all(got[i]["status"] == 0 for i in ids)
        assert all(got[i]["t_admit"] >= got[i]["t_submit"] for i in ids)


def test_short_requests_overtake_a_long_one(qfdlib):
    """Requests advance independently: short solves queued behind a long one are
    admitted at once (budget permitting) and finish first."""
    long_req = dict(n=64, a=0.1, mass=1.0, dtau=0.001, kinetic=1, nstates=1, precision="c128", potential="ho",
                    pot_coeffs=(1.0, 0.0), seed=21, tol=-1.0, max_steps=4000)
    with Q.Server(64e9, check_every=CHECK, ortho_every=ORTHO) as sv:
        lid = sv.submit(Q.make_request(**long_req))
        sids = [sv.submit(Q.make_request(**r)) for r in REQS[2:]]
        res = sv.run_until_done(1 + len(sids))
    assert res[lid]["status"] == 0 and res[lid]["steps"] == [4000]
    for i in sids:
        assert res[i]["status"] == 0
        assert res[i]["t_admit"] < res[lid]["t_done"]
        assert res[i]["t_done"] < res[lid]["t_done"]


def test_server_serves_fdtd_radix12_and_random_field_requests(qfdlib):
    """Requests with the finite-difference kinetic term, a 96^3 (radix-12)
    lattice and a random-field potential give the numbers of the same solve
    through a plan."""
    reqs = [
        dict(n=16, a=0.35, mass=1.5, dtau=0.0075, kinetic=0, nstates=2, precision="df64", potential="cornell",
             pot_coeffs=(0.3, 0.2), centre="offgrid", parity=[1, -1], seed=31, tol=1e-9, max_steps=20000),
        dict(n=96, a=0.2, mass=2.0, dtau=0.01, kinetic=2, nstates=1, precision="c64_refine_df", potential="ho",
             pot_coeffs=(1.0, 0.0), seed=32, tol=1e-9, max_steps=40000, grf=(5, 4.0, 0.05)),
    ]
    mix, _ = run_server(reqs)
    for req, got in zip(reqs, mix):
        assert got["status"] == 0
        kw = dict(nstates=req["nstates"], precision=req["precision"], ortho_every=ORTHO, check_every=CHECK,
                  max_steps=req["max_steps"], tol=req["tol"], tol_bulk=1e-10, centre=req.get("centre", "grid"))
        with Q.Plan(req["n"], req["a"], req["mass"], req["dtau"], req["kinetic"], **kw) as p:
            p.fill_potential(req["potential"], req["pot_coeffs"])
            if "grf" in req:
                p.add_random_field(*req["grf"])
            for s in range(req["nstates"]):
                p.fill_psi_uniform(s, req["seed"] + s)
            es, steps, _ = p.solve_states(req["nstates"], req.get("parity"))
        assert got["energy"] == es and got["steps"] == steps


def test_request_that_never_fits_ends_with_oom(qfdlib):
    big = dict(REQS[1], n=64)
    budget = 0.5 * Q.plan_bytes(64, big["precision"], big["nstates"])
    res, _ = run_server([big, REQS[3]], budget=max(budget, 1.5 * Q.plan_bytes(8, "c64_refine", 3)))
    assert res[0]["status"] == Q.ERR_OOM
    assert res[1]["status"] == 0


# Cohort mode: requests of one size advance together, each pass one launch over
# the members of one arithmetic.  A mix of several requests per size, with
# different arithmetics, kinetic terms (H_K(0) included), state counts and
# stop points, so that members join and leave cohorts while others run on.
COHORT_REQS = [
    dict(n=16, a=0.3, mass=1.0 + 0.3 * i, dtau=0.01, kinetic=1 + i % 3, nstates=1 + i % 3,
         precision=("c128", "df64", "c64_refine_df", "c64", "c64_refine")[i % 5],
         potential=("ho", "cornell", "softcoul")[i % 3], pot_coeffs=((1.0, 0.0), (0.3, 0.2), (0.01, 0.0))[i % 3],
         parity=[1, -1, 1][:1 + i % 3], seed=50 + i, tol=1e-6 if i % 5 == 3 else 1e-9, max_steps=20000)
    for i in range(7)
] + [
    dict(n=32, a=0.2, mass=1.5, dtau=0.004, kinetic=2, nstates=2, precision="c64_refine_df", potential="cornell",
         pot_coeffs=(0.3, 0.2), parity=[1, -1], seed=60, tol=1e-9, max_steps=20000),
    dict(n=32, a=0.2, mass=2.5, dtau=0.004, kinetic=3, nstates=1, precision="c64_refine_df", potential="ho",
         pot_coeffs=(1.0, 0.0), seed=61, tol=1e-9, max_steps=20000),
    dict(n=16, a=0.35, mass=1.5, dtau=0.0075, kinetic=0, nstates=1, precision="df64", potential="cornell",
         pot_coeffs=(0.3, 0.2), centre="offgrid", seed=62, tol=1e-9, max_steps=20000),
]


def run_cohorts(reqs, use_graphs=True, budget=64e9):
    with Q.Server(budget, check_every=CHECK, ortho_every=ORTHO, use_graphs=use_graphs, cohorts=True) as sv:
        ids = [sv.submit(Q.make_request(**r)) for r in reqs]
        res = sv.run_until_done(len(ids))
        return [res[i] for i in ids], sv.stats()


def test_cohort_results_equal_per_request_results_and_solve_states(qfdlib):
    mix, stats = run_cohorts(COHORT_REQS)
    assert stats["graph_replays"] > 0 and stats["graph_captures"] > 0
    per_req, _ = run_server(COHORT_REQS)
    for req, got, ref in zip(COHORT_REQS, mix, per_req):
        assert got["status"] == 0 and ref["status"] == 0
        assert got["energy"] == ref["energy"]
        assert got["steps"] == ref["steps"] and got["steps_c64"] == ref["steps_c64"]
    for req, got in zip(COHORT_REQS[:3] + COHORT_REQS[-3:], mix[:3] + mix[-3:]):
        es, steps = via_solve_states(req)
        assert got["energy"] == es and got["steps"] == steps


def test_cohort_alone_equals_cohort_in_mix_and_without_graphs(qfdlib):
    mix, _ = run_cohorts(COHORT_REQS[:5])
    direct, st = run_cohorts(COHORT_REQS[:5], use_graphs=False)
    assert st["graph_replays"] == 0
    assert [r["energy"] for r in mix] == [r["energy"] for r in direct]
    for req, got in zip(COHORT_REQS[:2], mix[:2]):
        alone, _ = run_cohorts([req])
        assert alone[0]["energy"] == got["energy"] and alone[0]["steps"] == got["steps"]


def test_cohort_admission_respects_the_budget_and_the_watchdog_works(qfdlib):
    budget = 2.5 * max(Q.plan_bytes(r["n"], r["precision"], r["nstates"]) for r in COHORT_REQS)
    big = dict(COHORT_REQS[7], n=128, a=0.1, dtau=0.001, max_steps=100000)
    budget = max(budget, 1.2 * Q.plan_bytes(128, big["precision"], big["nstates"]))
    with Q.Server(budget, check_every=CHECK, ortho_every=ORTHO, cohorts=True) as sv:
        ids = [sv.submit(Q.make_request(**r)) for r in COHORT_REQS]
        got = {}
        while len(got) < len(ids):
            assert sv.stats()["used_bytes"] <= budget
            for r in sv.poll():
                got[r["id"]] = r
        assert all(got[i]["status"] == 0 for i in ids)
        # a cohort whose period overruns the watchdog ends its members with a timeout
        sv.set_timeout(1e-6)
        rid = sv.submit(Q.make_request(**big))
        assert sv.run_until_done(1)[rid]["status"] == Q.ERR_TIMEOUT
        assert sv.stats()["active"] == 0 and sv.stats()["used_bytes"] == 0


def test_autotuning_server_gives_requests_of_one_kind_the_same_shapes(qfdlib):
    # the first request of each (size, precision) is tuned; later ones take its
    # shapes, so identical requests give identical numbers, alone or together
    reqs = [COHORT_REQS[1], COHORT_REQS[7], COHORT_REQS[1], COHORT_REQS[7]]
    with Q.Server(64e9, check_every=CHECK, ortho_every=ORTHO, cohorts=True, autotune=True) as sv:
        ids = [sv.submit(Q.make_request(**r)) for r in reqs]
        res = sv.run_until_done(len(ids))
    got = [res[i] for i in ids]
    assert all(r["status"] == 0 for r in got)
    assert got[0]["energy"] == got[2]["energy"] and got[1]["energy"] == got[3]["energy"]
    assert got[0]["steps"] == got[2]["steps"] and got[1]["steps"] == got[3]["steps"]
