"""Batched lockstep steps (qfd_step_batch) through the C ABI.

Each pass of a step (y transforms, z pass with T(k), update with the x
transforms; Sec. 2.1 and Eq. (iter_proced) of Sec. 2.2) runs as one launch
over several lattices of one size.  qfd_step runs the same kernels over a
batch of one lattice, so with the same launch shapes the states after
qfd_step_batch equal those after qfd_step bit for bit in every arithmetic.
The cases use plans that differ in mass, kinetic term, spacing,
dtau, potential, cadence, parity sector and stepped state, and that enter the
batch at different points of their cadence (W already transformed or not,
normalisations falling on different steps).  One case is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import qfd_oracle as O
from paper_2006_16935_gb300 import inputs
from paper_2006_16935_gb300 import qfd as Q

pytestmark = pytest.mark.gpu

PRECS = ["c128", "df64", "c64"]


def assert_same(prec, a, b, what):
    assert np.array_equal(a, b), (prec, what)


def assert_same_energy(prec, a, b, what):
    assert a == b, (prec, what)


def stable_dt(n, a, m, kin, frac):
    return frac / O.kinetic_max(n, a, m, kin, 0)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def plan_specs(n, count):
    """Per-plan parameters: kinetic 1..3 in turn, masses, spacings, Courant
    fractions, potentials, cadences, parity sectors and the stepped state."""
    pots = [("cornell", (0.3, 0.2)), ("ho", (1.0,)), ("softcoul", (0.01,)), ("coulomb", (0.5,))]
    out = []
    for i in range(count):
        kin = 1 + i % 3
        mass = 1.0 + 0.37 * i
        a = 0.1 + 0.01 * (i % 4)
        out.append(dict(kin=kin, mass=mass, a=a, dt=stable_dt(n, a, mass, kin, 0.3 + 0.1 * (i % 5)),
                        pot=pots[i % len(pots)], ortho=(3, 5, 10, 4)[i % 4], state=i % 2,
                        parity=(0, 1, -1)[i % 3], pre=(0, 1, 2, 7)[i % 4]))
    return out


def make_plan(n, spec, prec, seed):
    p = Q.Plan(n, spec["a"], spec["mass"], spec["dt"], spec["kin"], nstates=2, ortho_every=spec["ortho"],
               precision=prec)
    p.fill_potential(*spec["pot"])
    p.set_psi(0, O.normalize(inputs.uniform_psi(n, seed)))
    p.set_psi(1, inputs.uniform_psi(n, seed + 1))
    if spec["state"] == 1:
        p.set_parity(1, spec["parity"])
    else:
        p.set_parity(0, spec["parity"])
    if spec["pre"]:  # enter the batch at another point of the cadence
        p.step(spec["state"], spec["pre"])
    return p


def twin_runs(n, prec, count, nsteps, seed0=40):
    specs = plan_specs(n, count)
    single = [make_plan(n, s, prec, seed0 + 10 * i) for i, s in enumerate(specs)]
    batch = [make_plan(n, s, prec, seed0 + 10 * i) for i, s in enumerate(specs)]
    try:
        for p, s in zip(single, specs):
            p.step(s["state"], nsteps)
        Q.step_batch(batch, [s["state"] for s in specs], nsteps)
        got = [(p.get_psi(s["state"]), q.get_psi(s["state"])) for p, q, s in zip(single, batch, specs)]
        ens = [(p.energy(s["state"]), q.energy(s["state"])) for p, q, s in zip(single, batch, specs)]
    finally:
        for p in single + batch:
            p.close()
    return got, ens


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [16, 64, 96])
def test_batch_equals_single_plan_steps(qfdlib, n, prec):
    got, ens = twin_runs(n, prec, 6, 23)
    for i, (a, b) in enumerate(got):
        assert_same(prec, a, b, i)
    for i, (a, b) in enumerate(ens):
        assert_same_energy(prec, a, b, i)


def test_batch_of_32_smallest_lattices(qfdlib):
    # the largest batch, on 8^3 lattices (CTAs of fewer than 32 threads)
    got, _ = twin_runs(8, "df64", Q.MAX_BATCH, 11)
    for i, (a, b) in enumerate(got):
        assert_same("df64", a, b, i)
    got, _ = twin_runs(8, "c128", Q.MAX_BATCH, 11)
    for i, (a, b) in enumerate(got):
        assert_same("c128", a, b, i)


def test_batch_of_256_lattices(qfdlib):
    got, _ = twin_runs(256, "c64", 2, 4)
    for i, (a, b) in enumerate(got):
        assert_same("c64", a, b, i)


@pytest.mark.parametrize("prec", ["c128", "df64"])
def test_batch_matches_oracle(qfdlib, prec):
    n, nsteps = 16, 12
    specs = []
    for kin, mass in ((1, 1.0), (2, 1.7), (3, 2.5)):
        specs.append(dict(kin=kin, mass=mass, dt=stable_dt(n, 0.2, mass, kin, 0.8)))
    V = O.potential(n, 0.2, "cornell", (0.3, 0.2))
    psi0 = [inputs.uniform_psi(n, 70 + i) for i in range(len(specs))]
    plans = [Q.Plan(n, 0.2, s["mass"], s["dt"], s["kin"], ortho_every=5, precision=prec) for s in specs]
    try:
        for p, ps in zip(plans, psi0):
            p.set_potential(V)
            p.set_psi(0, ps)
        Q.step_batch(plans, 0, nsteps)
        got = [p.get_psi(0) for p in plans]
    finally:
        for p in plans:
            p.close()
    for g, s, ps in zip(got, specs, psi0):
        prob = O.Problem(n, 0.2, s["mass"], s["dt"], s["kin"], V, ortho_every=5)
        ref, _ = O.evolve(ps, prob, nsteps)
        assert rel_l2(g, ref) < 1e-10


def test_batch_zero_steps_and_continuation(qfdlib):
    # nsteps = 0 only applies a pending normalisation; a solve afterwards
    # proceeds from the batched states exactly as from single-plan steps
    n = 32
    specs = plan_specs(n, 3)
    single = [make_plan(n, s, "df64", 90 + i) for i, s in enumerate(specs)]
    batch = [make_plan(n, s, "df64", 90 + i) for i, s in enumerate(specs)]
    try:
        Q.step_batch(batch, [s["state"] for s in specs], 0)
        for p, q, s in zip(single, batch, specs):
            p.step(s["state"], 0)
            assert np.array_equal(p.get_psi(s["state"]), q.get_psi(s["state"]))
        Q.step_batch(batch, [s["state"] for s in specs], 9)
        for p, q, s in zip(single, batch, specs):
            p.step(s["state"], 9)
            p.step(s["state"], 6)
            q.step(s["state"], 6)
            assert np.array_equal(p.get_psi(s["state"]), q.get_psi(s["state"]))
    finally:
        for p in single + batch:
            p.close()


def test_batch_rejections_step_nothing(qfdlib):
    n = 16
    dt = stable_dt(n, 0.2, 1.0, 2, 0.5)
    with Q.Plan(n, 0.2, 1.0, dt, 2) as p, Q.Plan(n, 0.2, 1.0, dt, 2) as q, \
            Q.Plan(32, 0.2, 1.0, dt, 2) as r, Q.Plan(n, 0.2, 1.0, dt, 2, precision="df64") as d, \
            Q.Plan(n, 0.2, 1.0, dt, 0) as f, Q.Plan(n, 0.2, 1.0, dt, 2) as nopot:
        for pl in (p, q, r, d, f):
            pl.fill_potential("ho", (1.0,))
            pl.fill_psi_uniform(0, 3)
        before = p.get_psi(0)
        cases = [([p, q, r], 0), ([p, d], 0), ([p, p], 0), ([p, f], 0), ([p, q], [0, 1]), ([p, nopot], 0)]
        for plans, states in cases:
            with pytest.raises(Q.QfdError) as e:
                Q.step_batch(plans, states, 5)
            want = Q.ERR_STATE if nopot in plans else Q.ERR_ARG
            assert e.value.status == want
        with pytest.raises(Q.QfdError) as e:
            Q.step_batch([p, q], 0, -1)
        assert e.value.status == Q.ERR_ARG
        assert np.array_equal(p.get_psi(0), before)


@pytest.mark.parametrize("vx", [0, 1, 2])
def test_batch_of_one_512_lattice_equals_qfd_step(qfdlib, vx):
    # the benchmark's lattice size, through the batch entry point, with either
    # pass-A tile width: the same kernels as qfd_step, so the same bits
    outs = []
    for batched in (False, True):
        with Q.Plan(512, 0.05, 1.0, 5e-4, 2, precision="c64", ortho_every=2) as p:
            p.set_tuning(1, 0, -1, vx)
            p.fill_potential("softcoul", (0.01,))
            p.fill_psi_uniform(0, 3)
            if batched:
                Q.step_batch([p], 0, 3)
            else:
                p.step(0, 3)
            outs.append(p.get_psi(0))
    assert np.array_equal(outs[0], outs[1])
