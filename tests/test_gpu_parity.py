"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (the FP64 target of the method; the complex64 bound follows from FP32 rounding):
  complex128 and double-float ("df64"): relative L2 on psi <= 1e-10,
              relative energy <= 1e-9
  complex64:  relative L2 on psi <= 2e-6 per 10 steps (FP32 FFT rounding,
              eps32 * log2(N) per transform, entering the update times dtau T <= 2)
"""
import math

import numpy as np
import pytest

from oracle import qfd_oracle as O
from paper_2006_16935_gb300 import inputs
from paper_2006_16935_gb300 import qfd as Q

pytestmark = pytest.mark.gpu

TOL_PSI = 1e-10
TOL_E = 1e-9
FP64_CLASS = ["c128", "df64"]


def df_round(x):
    """A complex128 array rounded to the double-float representation hi + lo."""
    def split(r):
        hi = r.astype(np.float32).astype(np.float64)
        lo = (r - hi).astype(np.float32).astype(np.float64)
        return hi + lo
    return split(x.real) + 1j * split(x.imag)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def stable_dt(n, a, m, kin, frac=0.9, rest_mass=0):
    return frac / O.kinetic_max(n, a, m, kin, rest_mass)


def test_uniform_fill_is_bit_exact(qfdlib):
    for prec in ("c128", "c64", "df64"):
        with Q.Plan(16, 0.1, 1.0, 1e-4, 2, precision=prec) as p:
            p.fill_psi_uniform(0, 7)
            got = p.get_psi(0)
        ref = inputs.uniform_psi(16, 7)
        if prec == "c64":
            ref = ref.astype(np.complex64).astype(np.complex128)
        if prec == "df64":
            ref = df_round(ref)
        assert np.array_equal(got, ref)


def test_set_get_roundtrip_and_energy_of_plane_wave(qfdlib):
    n, a, m = 16, 0.2, 1.1
    j = np.arange(n)
    j1, j2, j3 = np.meshgrid(j, j, j, indexing="ij")
    pw = np.exp(2j * np.pi * (3 * j1 + 8 * j2 + 13 * j3) / n)
    with Q.Plan(n, a, m, stable_dt(n, a, m, 3), 3) as p:
        p.fill_potential("zero")
        p.set_psi(0, pw)
        assert np.array_equal(p.get_psi(0), pw)
        e, n2 = p.energy(0)
    T = O.kinetic_symbol(n, a, m, 3)
    assert e == pytest.approx(T[3, 8, 13], rel=1e-13)
    assert n2 == pytest.approx(n ** 3, rel=1e-14)


@pytest.mark.parametrize("centre", ["grid", "offgrid"])
@pytest.mark.parametrize("kind,coeffs", [("ho", (1.0,)), ("cornell", (0.3, 0.2)), ("coulomb", ()),
                                         ("softcoul", (0.01,)), ("zero", ())])
def test_potential_fill_matches_oracle(qfdlib, kind, coeffs, centre):
    n, a = 32, 0.05
    with Q.Plan(n, a, 1.0, 1e-4, 2, centre=centre) as p:
        p.fill_potential(kind, coeffs)
        V = p.get_potential()
    ref = O.potential(n, a, kind, coeffs, centre)
    assert np.max(np.abs(V - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", FP64_CLASS)
@pytest.mark.parametrize("nsteps", [10, 12])
@pytest.mark.parametrize("kin", [1, 2, 3])
@pytest.mark.parametrize("n", [8, 16, 32, 64, 96])
def test_step_parity_fp64_class(qfdlib, n, kin, nsteps, prec):
    a, m = 0.1, 1.3
    dt = stable_dt(n, a, m, kin)
    V = O.potential(n, a, "cornell", (0.3, 0.2))
    psi0 = inputs.uniform_psi(n, 11)
    with Q.Plan(n, a, m, dt, kin, ortho_every=5, precision=prec) as p:
        p.set_potential(V)
        p.set_psi(0, psi0)
        p.step(0, nsteps)
        got = p.get_psi(0)
    ref, _ = O.evolve(psi0, O.Problem(n, a, m, dt, kin, V, ortho_every=5), nsteps)
    assert rel_l2(got, ref) < TOL_PSI


@pytest.mark.parametrize("prec", FP64_CLASS)
@pytest.mark.parametrize("kin", [1, 3])
def test_step_parity_split_calls_and_rest_mass(qfdlib, kin, prec):
    # steps issued in several calls continue the same cadence counter
    n, a, m = 32, 0.12, 2.0
    dt = stable_dt(n, a, m, kin, 0.5, rest_mass=1)
    V = O.potential(n, a, "ho", (0.7,))
    psi0 = inputs.uniform_psi(n, 12)
    with Q.Plan(n, a, m, dt, kin, rest_mass=1, ortho_every=4, precision=prec) as p:
        p.set_potential(V)
        p.set_psi(0, psi0)
        for k in (3, 1, 5, 2):
            p.step(0, k)
        got = p.get_psi(0)
    ref, _ = O.evolve(psi0, O.Problem(n, a, m, dt, kin, V, rest_mass=1, ortho_every=4), 11)
    assert rel_l2(got, ref) < TOL_PSI


@pytest.mark.parametrize("prec", FP64_CLASS)
@pytest.mark.parametrize("centre", ["grid", "offgrid"])
@pytest.mark.parametrize("parity", [1, -1])
def test_step_parity_with_projection_and_gram_schmidt(qfdlib, centre, parity, prec):
    n, a, m, kin = 16, 0.2, 1.5, 3
    dt = stable_dt(n, a, m, kin)
    V = O.potential(n, a, "cornell", (0.3, 0.2), centre)
    phi0 = O.normalize(inputs.uniform_psi(n, 1))
    phi1 = O.normalize(O.gram_schmidt(inputs.uniform_psi(n, 2), [phi0]))
    psi = inputs.uniform_psi(n, 3)
    if prec == "df64":
        phi0, phi1 = df_round(phi0), df_round(phi1)
    with Q.Plan(n, a, m, dt, kin, nstates=3, ortho_every=3, centre=centre, precision=prec) as p:
        p.set_potential(V)
        p.set_psi(0, phi0)
        p.set_psi(1, phi1)
        p.set_psi(2, psi)
        p.set_parity(2, parity)
        p.step(2, 9)
        got = p.get_psi(2)
        # the lower states are untouched
        assert np.array_equal(p.get_psi(0), phi0)
    prob = O.Problem(n, a, m, dt, kin, V, ortho_every=3, centre=centre)
    ref, _ = O.evolve(psi, prob, 9, parity=parity, lower=(phi0, phi1))
    assert rel_l2(got, ref) < TOL_PSI
    # Gram-Schmidt comes last in the cadence: no overlap with the lower states
    # (which are not parity eigenstates here, so the sector is not pure)
    assert abs(O.inner(phi0, got)) < 1e-12 and abs(O.inner(phi1, got)) < 1e-12


@pytest.mark.parametrize("centre", ["grid", "offgrid"])
@pytest.mark.parametrize("parity", [1, -1])
def test_parity_sector_is_kept_by_steps(qfdlib, centre, parity):
    # with an R-symmetric potential and no lower states the state stays in its
    # sector to rounding between projections (Eq. (parity))
    n, a, m, kin = 32, 0.1, 1.0, 2
    dt = stable_dt(n, a, m, kin)
    with Q.Plan(n, a, m, dt, kin, ortho_every=4, centre=centre) as p:
        p.fill_potential("cornell", (0.3, 0.2))
        p.fill_psi_uniform(0, 44)
        p.set_parity(0, parity)
        p.step(0, 7)  # projected at step 4, then 3 free steps
        got = p.get_psi(0)
    assert np.linalg.norm(O.parity_project(got, -parity, centre)) < 1e-13 * np.linalg.norm(got)


@pytest.mark.parametrize("prec", FP64_CLASS)
@pytest.mark.parametrize("kin", [1, 2, 3])
@pytest.mark.parametrize("n", [16, 64, 96])
def test_energy_parity(qfdlib, n, kin, prec):
    a, m = 0.1, 1.0
    V = O.potential(n, a, "softcoul", (0.01,))
    psi = inputs.uniform_psi(n, 21)
    with Q.Plan(n, a, m, stable_dt(n, a, m, kin), kin, precision=prec) as p:
        p.set_potential(V)
        p.set_psi(0, psi)
        e, n2 = p.energy(0)
    T = O.kinetic_symbol(n, a, m, kin)
    assert e == pytest.approx(O.energy(psi, V, T), rel=1e-12)
    assert n2 == pytest.approx(O.norm2(psi), rel=1e-13)


@pytest.mark.parametrize("prec", FP64_CLASS)
@pytest.mark.parametrize("kin,dt", [(1, 0.001), (2, 0.002), (3, 0.002)])
def test_solve_parity_oscillator_32(qfdlib, kin, dt, prec):
    # 32^3, A = 0.1, M = 1, V = r^2/2 from the box centre, uniform start (seed 1),
    # 2000 steps, energy and normalisation every 100 steps
    n, a, m = 32, 0.1, 1.0
    with Q.Plan(n, a, m, dt, kin, ortho_every=100, check_every=100, max_steps=2000, tol=-1, precision=prec) as p:
        p.fill_potential("ho", (1.0,))
        p.fill_psi_uniform(0, 1)
        es, steps, _ = p.solve_states(1)
        psi = p.get_psi(0)
        e_decay = p.decay_energy(0)
    V = O.potential(n, a, "ho", (1.0,))
    prob = O.Problem(n, a, m, dt, kin, V, ortho_every=100, check_every=100)
    res = O.solve_state(inputs.uniform_psi(n, 1), prob, 2000, -1)
    assert steps[0] == res.steps == 2000
    assert abs(es[0] - res.energy) <= TOL_E * abs(res.energy)
    assert rel_l2(psi, res.psi) < TOL_PSI
    assert abs(e_decay - res.e_decay) <= TOL_E * abs(res.e_decay)


@pytest.mark.parametrize("prec", FP64_CLASS)
def test_solve_states_excited_with_parity(qfdlib, prec):
    # Cornell -0.3/r + 0.2 r, relativistic sqrt(p^2+m^2)-m with m = 1.5, states {even, odd, even}
    n, a, m, kin = 16, 0.4, 1.5, 3
    dt = stable_dt(n, a, m, kin, 0.5)
    par = [1, -1, 1]
    with Q.Plan(n, a, m, dt, kin, nstates=3, ortho_every=10, check_every=50, max_steps=20000, tol=1e-10,
                precision=prec) as p:
        p.fill_potential("cornell", (0.3, 0.2))
        for s in range(3):
            p.fill_psi_uniform(s, 100 + s)
        es, steps, conv = p.solve_states(3, par)
        psis = [p.get_psi(s) for s in range(3)]
        decays = [p.decay_energy(s) for s in range(3)]
    assert conv
    V = O.potential(n, a, "cornell", (0.3, 0.2))
    prob = O.Problem(n, a, m, dt, kin, V, ortho_every=10, check_every=50)
    res = O.solve_states([inputs.uniform_psi(n, 100 + s) for s in range(3)], prob, 20000, 1e-10, par)
    for s in range(3):
        assert steps[s] == res[s].steps
        assert abs(es[s] - res[s].energy) <= TOL_E * abs(res[s].energy)
        # decay-rate energy after the projections of the excited states
        assert abs(decays[s] - res[s].e_decay) <= 1e-8 * abs(res[s].e_decay)
        assert rel_l2(psis[s], res[s].psi) < 1e-9
    # the even ground state lies lowest; the second even state may lie below the odd one
    assert es[0] < es[1] and es[0] < es[2]


@pytest.mark.parametrize("prec", FP64_CLASS + ["c64_refine_df"])
def test_tail_stop_rule_matches_oracle_and_reaches_the_limit(qfdlib, prec):
    # the states of the excited-state case under the tail stop rule: same checks as
    # the oracle's rule (FP64 class), and every energy within tol of its limit
    n, a, m, kin = 16, 0.4, 1.5, 3
    dt = stable_dt(n, a, m, kin, 0.5)
    par, tol = [1, -1, 1], 1e-9
    with Q.Plan(n, a, m, dt, kin, nstates=3, ortho_every=10, check_every=50, max_steps=40000, tol=tol,
                tol_bulk=1e-10, stop_rule="tail", precision=prec) as p:
        p.fill_potential("cornell", (0.3, 0.2))
        for s in range(3):
            p.fill_psi_uniform(s, 100 + s)
        es, steps, conv = p.solve_states(3, par)
    assert conv
    V = O.potential(n, a, "cornell", (0.3, 0.2))
    prob = O.Problem(n, a, m, dt, kin, V, ortho_every=10, check_every=50)
    psi0 = [inputs.uniform_psi(n, 100 + s) for s in range(3)]
    limit = O.solve_states(psi0, prob, 60000, 1e-14, par)
    if prec != "c64_refine_df":
        res = O.solve_states(psi0, prob, 40000, tol, par, rule="tail")
        paper = O.solve_states(psi0, prob, 40000, tol, par)
        for s in range(3):
            assert steps[s] == res[s].steps >= paper[s].steps
            assert abs(es[s] - res[s].energy) <= TOL_E * abs(res[s].energy)
    for s in range(3):
        assert abs(es[s] - limit[s].energy) <= 2 * tol * abs(limit[s].energy)


@pytest.mark.parametrize("prec", FP64_CLASS)
def test_snapshot_states_match_oracle(qfdlib, prec):
    # one 600-step evolution of the 16^3 Cornell case (H_K(3), even parity),
    # snapshots every 200 steps: ground = final state, excited = the snapshots
    # at steps 400 and 200 deflated (Sec. 2.2)
    n, a, m, kin = 16, 0.4, 1.5, 3
    dt = stable_dt(n, a, m, kin, 0.5)
    with Q.Plan(n, a, m, dt, kin, nstates=4, ortho_every=10, check_every=50, max_steps=600, tol=-1,
                precision=prec) as p:
        p.fill_potential("cornell", (0.3, 0.2))
        p.fill_psi_uniform(0, 7)
        es, steps, _ = p.snapshot_states(3, parity=1, snap_every=200)
        psis = [p.get_psi(s) for s in range(3)]
    V = O.potential(n, a, "cornell", (0.3, 0.2))
    prob = O.Problem(n, a, m, dt, kin, V, ortho_every=10, check_every=50)
    psi0 = inputs.uniform_psi(n, 7)
    res = O.snapshot_states(df_round(psi0) if prec == "df64" else psi0, prob, 600, -1, 200, parity=1, nout=3)
    assert steps == res[0].steps == 600
    # an excited estimate is a snapshot minus its (dominant) lower-state part:
    # a difference of rounding between the two sides grows by the ratio of the
    # snapshot to what remains (up to ~1e3 for the step-200 snapshot here)
    for s in range(3):
        assert abs(es[s] - res[s].energy) <= TOL_E * abs(res[s].energy)
        assert rel_l2(psis[s], res[s].psi) < (TOL_PSI if s == 0 else 1e3 * TOL_PSI)
    assert es[0] < es[1] < es[2]


@pytest.mark.parametrize("prec,snap,tol", [("c128", 40, 1e-9), ("df64", 40, 1e-9), ("c64", 20, 1e-3)])
def test_snapshot_states_plane_wave_levels(qfdlib, prec, snap, tol):
    # the plane-wave case of the oracle pin, on the GPU: V = 0, three modes.
    # complex64 resolves components down to ~1e-7 only, so its snapshots are
    # closer together (the second excited mode keeps 3e-4 of the weight)
    n, a, m, kin = 8, 1.0, 1.0, 2
    x = np.arange(n)
    X1, X2, X3 = np.meshgrid(x, x, x, indexing="ij")
    modes = [(0, 0, 0), (1, 0, 0), (2, 0, 0)]
    pws = [np.exp(2j * np.pi * (k1 * X1 + k2 * X2 + k3 * X3) / n) for (k1, k2, k3) in modes]
    lev = [0.0, 2 * math.sin(math.pi / 8) ** 2, 1.0]
    with Q.Plan(n, a, m, 0.3, kin, nstates=4, ortho_every=10, check_every=10, max_steps=3 * snap, tol=-1,
                precision=prec) as p:
        p.fill_potential("zero", ())
        p.set_psi(0, pws[0] + 0.7 * pws[1] + 0.4 * pws[2])
        es, steps, _ = p.snapshot_states(3, snap_every=snap)
        psis = [p.get_psi(s) for s in range(3)]
    for i in range(3):
        assert es[i] == pytest.approx(lev[i], abs=tol)
        assert abs(np.vdot(pws[i], psis[i])) / math.sqrt(n ** 3) == pytest.approx(1.0, abs=tol)


def test_snapshot_states_argument_errors(qfdlib):
    with Q.Plan(8, 1.0, 1.0, 0.1, 2, nstates=3, ortho_every=10, check_every=10, max_steps=40, tol=-1) as p:
        p.fill_potential("zero", ())
        p.fill_psi_uniform(0, 1)
        with pytest.raises(Q.QfdError):  # three outputs need four state slots
            p.snapshot_states(3, snap_every=10)
        with pytest.raises(Q.QfdError):  # not a multiple of ortho_every
            p.snapshot_states(2, snap_every=15)
        with pytest.raises(Q.QfdError) as ei:  # one spacing: no snapshot before the end
            p.snapshot_states(2, snap_every=40)
        assert ei.value.status == Q.ERR_STATE
    with Q.Plan(8, 1.0, 1.0, 0.1, 2, nstates=3, precision="c64_refine", ortho_every=10, check_every=10) as p:
        p.fill_potential("zero", ())
        with pytest.raises(Q.QfdError):
            p.snapshot_states(2, snap_every=10)


# ------------------------------------------------------------- complex64 ----

@pytest.mark.parametrize("kin", [1, 2, 3])
@pytest.mark.parametrize("n", [16, 64, 96])
def test_step_parity_c64(qfdlib, n, kin):
    a, m = 0.1, 1.3
    dt = stable_dt(n, a, m, kin)
    V = O.potential(n, a, "cornell", (0.3, 0.2))
    psi0 = inputs.uniform_psi(n, 31).astype(np.complex64).astype(np.complex128)
    with Q.Plan(n, a, m, dt, kin, precision="c64", ortho_every=5) as p:
        p.set_potential(V)
        p.set_psi(0, psi0)
        p.step(0, 10)
        got = p.get_psi(0)
        e, _ = p.energy(0)
    ref, _ = O.evolve(psi0, O.Problem(n, a, m, dt, kin, V, ortho_every=5), 10)
    assert rel_l2(got, ref) < 2e-6
    assert e == pytest.approx(O.energy(ref, V, O.kinetic_symbol(n, a, m, kin)), rel=1e-5)


@pytest.mark.parametrize("prec", ["c64_refine", "c64_refine_df"])
def test_mixed_precision_solve_reaches_fp64_energy(qfdlib, prec):
    n, a, m, kin = 16, 0.25, 1.0, 2
    dt = 0.01
    kw = dict(ortho_every=20, check_every=100, max_steps=40000, tol=1e-10)
    with Q.Plan(n, a, m, dt, kin, precision=prec, tol_bulk=1e-6, **kw) as p:
        p.fill_potential("ho", (1.0,))
        p.fill_psi_uniform(0, 1)
        es, steps, conv = p.solve_states(1)
        st = p.stats(0)
        psi = p.get_psi(0)
    assert conv and st["steps_c64"] > 0 and st["steps_c128"] > 0
    V = O.potential(n, a, "ho", (1.0,))
    prob = O.Problem(n, a, m, dt, kin, V, ortho_every=20, check_every=100)
    res = O.solve_state(inputs.uniform_psi(n, 1), prob, 40000, 1e-10)
    assert abs(es[0] - res.energy) <= TOL_E * abs(res.energy)
    assert abs(abs(O.inner(psi, res.psi)) - 1) < 1e-8


def test_timing_and_launch_counters(qfdlib):
    n = 32
    with Q.Plan(n, 0.1, 1.0, 0.001, 2, ortho_every=10) as p:
        p.fill_potential("ho", (1.0,))
        p.fill_psi_uniform(0, 1)
        p.step(0, 1)
        p.timing(True)
        p.timing_reset()
        p.step(0, 20)
        cnt, ms = p.timing_query("update_x")
        assert cnt == 20 and ms > 0
        assert p.timing_query("z_kinetic")[0] == 20
        assert p.launch_count() >= 80


# ---------------------------------------------------------- observables ----

@pytest.mark.parametrize("prec", ["c128", "df64", "c64"])
@pytest.mark.parametrize("centre", ["grid", "offgrid"])
def test_observables_match_oracle(qfdlib, prec, centre):
    n = 32
    psi = inputs.uniform_psi(n, 61)
    d = O.displacement(n, centre)
    d1, d2, d3 = np.meshgrid(d, d, d, indexing="ij")
    psi = psi * np.exp(-((d1 - 2) ** 2 + d2 ** 2 + (d3 + 1) ** 2) / 60.0)  # localised, off-centre
    if prec == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    if prec == "df64":
        psi = df_round(psi)
    with Q.Plan(n, 0.1, 1.0, 1e-4, 2, precision=prec, centre=centre) as p:
        p.fill_potential("zero")
        p.set_psi(0, psi)
        got = p.observables(0, 0.3)
    ref = O.observables(psi, centre, 0.3)
    for k, v in ref.items():
        assert got[k] == pytest.approx(v, rel=1e-12, abs=1e-12), k


@pytest.mark.parametrize("n,corr", [(32, 4.0), (64, 4.0), (64, 3.0)])
def test_random_field_matches_oracle(qfdlib, n, corr):
    # Cornell plus a seeded Gaussian random field of amplitude 0.05
    with Q.Plan(n, 0.1, 1.0, 1e-4, 2) as p:
        p.fill_potential("cornell", (0.3, 0.2))
        p.add_random_field(17, corr, 0.05)
        V = p.get_potential()
    ref = O.potential(n, 0.1, "cornell", (0.3, 0.2)) + O.random_field(inputs.gaussian_noise(n, 17), corr, 0.05)
    assert np.max(np.abs(V - ref)) < 1e-12


def test_random_field_potential_solve_matches_oracle(qfdlib):
    n, a, m, kin = 16, 0.3, 1.2, 2
    dt = stable_dt(n, a, m, kin, 0.5)
    with Q.Plan(n, a, m, dt, kin, ortho_every=10, check_every=50, max_steps=20000, tol=1e-10) as p:
        p.fill_potential("cornell", (0.3, 0.2))
        p.add_random_field(5, 4.0, 0.05)
        p.fill_psi_uniform(0, 9)
        es, steps, _ = p.solve_states(1)
    V = O.potential(n, a, "cornell", (0.3, 0.2)) + O.random_field(inputs.gaussian_noise(n, 5), 4.0, 0.05)
    res = O.solve_state(inputs.uniform_psi(n, 9), O.Problem(n, a, m, dt, kin, V, ortho_every=10, check_every=50),
                        20000, 1e-10)
    assert steps[0] == res.steps
    assert abs(es[0] - res.energy) <= TOL_E * abs(res.energy)


# ------------------------------------------------- radix-12 lattices (96, 192)

@pytest.mark.parametrize("prec", FP64_CLASS + ["c64"])
def test_radix12_lattice_projection_observables_and_fields(qfdlib, prec):
    # N = 96 (12 elements per thread, radix 12-4-2): parity projection with
    # Gram-Schmidt, the observables and a random field at a lattice that is
    # not a power of two
    n, a, m, kin = 96, 0.1, 1.5, 3
    dt = stable_dt(n, a, m, kin)
    V = O.potential(n, a, "cornell", (0.3, 0.2)) + O.random_field(inputs.gaussian_noise(n, 3), 4.0, 0.05)
    phi0 = O.normalize(inputs.uniform_psi(n, 1))
    psi = inputs.uniform_psi(n, 2)
    if prec == "df64":
        phi0 = df_round(phi0)
    with Q.Plan(n, a, m, dt, kin, nstates=2, ortho_every=3, precision=prec) as p:
        p.fill_potential("cornell", (0.3, 0.2))
        p.add_random_field(3, 4.0, 0.05)
        assert np.max(np.abs(p.get_potential() - V)) < 1e-12
        p.set_psi(0, phi0)
        p.set_psi(1, psi)
        p.set_parity(1, -1)
        p.step(1, 6)
        got = p.get_psi(1)
        lower = p.get_psi(0)
        ob = p.observables(1, 0.3)
    prob = O.Problem(n, a, m, dt, kin, V, ortho_every=3)
    ref, _ = O.evolve(psi, prob, 6, parity=-1, lower=(lower,))
    assert rel_l2(got, ref) < (TOL_PSI if prec != "c64" else 2e-6)
    want = O.observables(got, "grid", 0.3)
    for k, v in want.items():
        assert ob[k] == pytest.approx(v, rel=1e-12, abs=1e-12), k


@pytest.mark.parametrize("prec", FP64_CLASS)
def test_radix12_192_steps_match_library_oracle(qfdlib, prec):
    n, a, m, kin = 192, 0.05, 1.0, 2
    dt = stable_dt(n, a, m, kin)
    V = O.potential(n, a, "softcoul", (0.01,))
    psi0 = inputs.uniform_psi(n, 8)
    with Q.Plan(n, a, m, dt, kin, ortho_every=4, precision=prec) as p:
        p.set_potential(V)
        p.set_psi(0, psi0)
        p.step(0, 6)
        got = p.get_psi(0)
        e, _ = p.energy(0)
    prob = O.Problem(n, a, m, dt, kin, V, ortho_every=4, method="library")
    ref, _ = O.evolve(psi0, prob, 6)
    assert rel_l2(got, ref) < TOL_PSI
    e_ref = O.energy(ref, V, prob.T, "library")
    assert abs(e - e_ref) <= TOL_E * abs(e_ref)


def test_radix12_fdtd_step(qfdlib):
    n, a, m = 96, 0.1, 1.3
    dt = 0.9 / O.kinetic_max(n, a, m, 0)
    V = O.potential(n, a, "ho", (1.0,), "offgrid")
    psi0 = inputs.uniform_psi(n, 5)
    with Q.Plan(n, a, m, dt, 0, ortho_every=5, centre="offgrid") as p:
        p.set_potential(V)
        p.set_psi(0, psi0)
        p.step(0, 10)
        got = p.get_psi(0)
    ref, _ = O.evolve(psi0, O.Problem(n, a, m, dt, 0, V, ortho_every=5, centre="offgrid"), 10)
    assert rel_l2(got, ref) < TOL_PSI


# ------------------------------------------------------------- edge cases

@pytest.mark.parametrize("prec", FP64_CLASS)
def test_eight_states_the_largest_stack(qfdlib, prec):
    # the deepest Gram-Schmidt: state 7 deflated against seven lower states
    n, a, m, kin = 8, 0.5, 1.0, 2
    dt = stable_dt(n, a, m, kin, 0.5)
    V = aniso_potential(n, a)
    with Q.Plan(n, a, m, dt, kin, nstates=8, ortho_every=5, check_every=25, max_steps=40000, tol=1e-10,
                precision=prec) as p:
        p.set_potential(V)
        for s in range(8):
            p.fill_psi_uniform(s, 300 + s)
        es, steps, conv = p.solve_states(8)
        psis = [p.get_psi(s) for s in range(8)]
    prob = O.Problem(n, a, m, dt, kin, V, ortho_every=5, check_every=25)
    res = O.solve_states([inputs.uniform_psi(n, 300 + s) for s in range(8)], prob, 40000, 1e-10)
    for s in range(8):
        assert steps[s] == res[s].steps
        assert abs(es[s] - res[s].energy) <= TOL_E * abs(res[s].energy)
    gram = np.array([[O.inner(psis[i], psis[j]) for j in range(8)] for i in range(8)])
    assert np.max(np.abs(gram - np.eye(8))) < 1e-12


def aniso_potential(n, a):
    # anisotropic oscillator: no degenerate levels among the lowest eight
    d = O.displacement(n)
    d1, d2, d3 = np.meshgrid(d, d, d, indexing="ij")
    return 0.5 * a * a * (1.0 * d1 ** 2 + 2.3 * d2 ** 2 + 5.1 * d3 ** 2)


def test_zero_steps_and_tiny_cases(qfdlib):
    n = 8
    psi = inputs.uniform_psi(n, 3)
    with Q.Plan(n, 0.5, 1.0, 0.01, 2, max_steps=0) as p:
        p.fill_potential("ho", (1.0,))
        p.set_psi(0, psi)
        p.step(0, 0)  # no steps: the state is untouched
        assert np.array_equal(p.get_psi(0), psi)
        with pytest.raises(Q.QfdError) as ei:  # max_steps 0: no check, not converged
            p.solve_states(1)
        assert ei.value.status == Q.ERR_NOT_CONVERGED
