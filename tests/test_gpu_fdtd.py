"""Parity of the finite-difference kinetic term H_K(0) (Sec. 2.1, Eq. HK0 with
Dirichlet boundaries) on the GPU with the FP64 oracle, through the C ABI.

Tolerances as for the FFT terms: complex128 and double-float relative L2 on
psi <= 1e-10 and relative energy <= 1e-9; complex64 relative L2 <= 2e-6 after
10 steps (FP32 rounding of a seven-point sum and the update)."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dt_for(a, m, frac=0.9):
    return frac / O.kinetic_max(8, a, m, 0)


@pytest.mark.parametrize("prec", FP64_CLASS)
@pytest.mark.parametrize("nsteps", [10, 12])
@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_fdtd_step_parity_fp64_class(qfdlib, n, nsteps, prec):
    a, m = 0.1, 1.3
    dt = dt_for(a, m)
    V = O.potential(n, a, "cornell", (0.3, 0.2), "offgrid")
    psi0 = inputs.uniform_psi(n, 11)
    with Q.Plan(n, a, m, dt, 0, ortho_every=5, centre="offgrid", precision=prec) as p:
        p.set_potential(V)
        p.set_psi(0, psi0)
        p.step(0, nsteps)
        got = p.get_psi(0)
        e, n2 = p.energy(0)
    prob = O.Problem(n, a, m, dt, 0, V, ortho_every=5, centre="offgrid")
    ref, _ = O.evolve(psi0, prob, nsteps)
    assert rel_l2(got, ref) < TOL_PSI
    e_ref = O.energy(ref, V, prob.T)
    assert abs(e - e_ref) <= TOL_E * abs(e_ref)
    assert n2 == pytest.approx(O.norm2(ref), rel=1e-12)


@pytest.mark.parametrize("n", [16, 64])
def test_fdtd_step_parity_c64(qfdlib, n):
    a, m = 0.1, 1.3
    dt = dt_for(a, m)
    V = O.potential(n, a, "ho", (1.0,), "offgrid")
    psi0 = inputs.uniform_psi(n, 5)
    with Q.Plan(n, a, m, dt, 0, ortho_every=5, centre="offgrid", precision="c64") as p:
        p.set_potential(V)
        p.set_psi(0, psi0)
        p.step(0, 10)
        got = p.get_psi(0)
    ref, _ = O.evolve(psi0, O.Problem(n, a, m, dt, 0, V, ortho_every=5, centre="offgrid"), 10)
    assert rel_l2(got, ref) < 2e-6


@pytest.mark.parametrize("prec", FP64_CLASS)
@pytest.mark.parametrize("parity", [1, -1])
def test_fdtd_projection_and_gram_schmidt(qfdlib, parity, prec):
    n, a, m = 16, 0.2, 1.5
    dt = dt_for(a, m)
    V = O.potential(n, a, "cornell", (0.3, 0.2), "offgrid")
    phi0 = O.normalize(inputs.uniform_psi(n, 1))
    psi = inputs.uniform_psi(n, 3)
    with Q.Plan(n, a, m, dt, 0, nstates=2, ortho_every=3, centre="offgrid", precision=prec) as p:
        p.set_potential(V)
        p.set_psi(0, phi0)
        p.set_psi(1, psi)
        p.set_parity(1, parity)
        p.step(1, 9)
        got = p.get_psi(1)
        ref_phi0 = p.get_psi(0)
    prob = O.Problem(n, a, m, dt, 0, V, ortho_every=3, centre="offgrid")
    ref, _ = O.evolve(psi, prob, 9, parity=parity, lower=(ref_phi0,))
    assert rel_l2(got, ref) < TOL_PSI
    assert abs(O.inner(ref_phi0, got)) < 1e-12


@pytest.mark.parametrize("prec", FP64_CLASS + ["c64_refine_df"])
def test_fdtd_solve_states_with_parity(qfdlib, prec):
    # Cornell, states {even, odd, odd} about the off-grid centre of the
    # Dirichlet box, solved to 1e-10 with the tail rule: the ground state and
    # two members of the P triplet (same level).  (The next even state is
    # nearly degenerate with its neighbour in this box and converges slowly.)
    n, a, m = 16, 0.35, 1.5
    dt = dt_for(a, m, 0.5)
    par = [1, -1, -1]
    with Q.Plan(n, a, m, dt, 0, nstates=3, ortho_every=10, check_every=50, max_steps=40000, tol=1e-10,
                tol_bulk=1e-10, stop_rule="tail", centre="offgrid", precision=prec) as p:
        p.fill_potential("cornell", (0.3, 0.2))
        for s in range(3):
            p.fill_psi_uniform(s, 100 + s)
        es, steps, conv = p.solve_states(3, par)
    assert conv
    V = O.potential(n, a, "cornell", (0.3, 0.2), "offgrid")
    prob = O.Problem(n, a, m, dt, 0, V, ortho_every=10, check_every=50, centre="offgrid")
    psi0 = [inputs.uniform_psi(n, 100 + s) for s in range(3)]
    limit = O.solve_states(psi0, prob, 60000, 1e-14, par)
    for s in range(3):
        assert abs(es[s] - limit[s].energy) <= 2e-10 * abs(limit[s].energy)
    assert es[1] == pytest.approx(es[2], rel=2e-10)
    if prec != "c64_refine_df":
        res = O.solve_states(psi0, prob, 40000, 1e-10, par, rule="tail")
        assert steps == [r.steps for r in res]


@pytest.mark.parametrize("prec", ["c128", "df64", "c64"])
def test_fdtd_sine_modes_at_512(qfdlib, prec):
    # full size: with V = 0 a product of Dirichlet sine modes is an exact
    # eigenvector of H_K(0) with eigenvalue (1/2M) sum_l (4/A^2) sin^2(k_l/2),
    # k_l = pi j_l / (N + 1); two steps multiply it by (1 - dtau lambda)^2.
    # Checked at 4096 sampled sites.
    n, a, m = 512, 0.05, 1.0
    dt = dt_for(a, m)
    js = [(1, 2, 3), (5, 1, 1)]
    x = np.arange(n)
    rng = np.random.default_rng(2)
    idx = rng.integers(0, n, size=(4096, 3))
    lam = [sum(4 / (a * a) * math.sin(math.pi * jl / (n + 1) / 2) ** 2 for jl in j) / (2 * m) for j in js]
    coeff = [1.0, 0.5j]
    modes = [[np.sin(np.pi * jl * (x + 1) / (n + 1)) for jl in j] for j in js]

    def field(steps):
        out = np.zeros(len(idx), complex)
        for c, md, lm in zip(coeff, modes, lam):
            out += c * (1 - dt * lm) ** steps * md[0][idx[:, 0]] * md[1][idx[:, 1]] * md[2][idx[:, 2]]
        return out

    psi0 = np.zeros((n, n, n), complex)
    for c, md in zip(coeff, modes):
        psi0 += c * np.einsum("i,j,k->ijk", *md)
    with Q.Plan(n, a, m, dt, 0, ortho_every=1000, precision=prec) as p:
        p.fill_potential("zero", ())
        p.set_psi(0, psi0)
        del psi0
        p.step(0, 2)
        got = p.get_psi(0)[idx[:, 0], idx[:, 1], idx[:, 2]]
    want = field(2)
    tol = 1e-12 if prec != "c64" else 2e-6
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
