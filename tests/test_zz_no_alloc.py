"""qfd_energy_noalloc: the energy entry point for callers that cannot allocate
device memory (its scratch is a static device array, lattices up to 128^3).

Collected last on purpose.  Two calls in a row (different lattices, sizes and
kinetic terms), then a repeat of the first, are each compared with the energy
of the same state and potential from the plan-based qfd_energy and from the
oracle (library FFT), within the FP64 tolerance the other parity tests use;
one call runs on a non-default stream and checks that the caller's psi and V
are left as they were.
"""
import numpy as np
import pytest

from oracle import qfd_oracle as O
from paper_2006_16935_gb300 import qfd as Q

pytestmark = pytest.mark.gpu

CASES = [  # n, a, mass, kinetic, rest_mass, potential, seed
    (32, 0.1, 1.0, 2, 0, ("softcoul", (0.01,)), 5),
    (64, 0.05, 1.5, 3, 0, ("cornell", (0.3, 0.2)), 6),
    (128, 0.05, 2.0, 1, 0, ("ho", (1.0,)), 7),
    (96, 0.1, 1.2, 2, 0, ("cornell", (0.3, 0.2)), 8),  # radix-12 transforms
]


def plan_energy(n, a, mass, kin, rest, pot, seed):
    with Q.Plan(n, a, mass, 1e-5, kin, rest_mass=rest) as p:
        p.fill_potential(*pot)
        p.fill_psi_uniform(0, seed)
        e, n2 = p.energy(0)
        return e, n2, p.get_psi(0), p.get_potential()


def oracle_energy(n, a, mass, kin, rest, psi, V):
    T = O.kinetic_symbol(n, a, mass, kin, rest)
    return O.energy(psi, V, T, method="library"), O.norm2(psi)


def test_noalloc_energy_matches_plan_energy_and_oracle(qfdlib):
    import torch

    refs = [plan_energy(*c) for c in CASES]
    order = [0, 1, 3, 2, 0]  # different calls in a row, then a repeat
    for i in order:
        n, a, mass, kin, rest, _, _ = CASES[i]
        e_ref, n2_ref, psi, V = refs[i]
        psi_d = torch.from_numpy(psi.reshape(-1)).cuda()
        V_d = torch.from_numpy(V.reshape(-1)).cuda()
        stream = torch.cuda.current_stream().cuda_stream
        e, n2 = Q.energy_noalloc(psi_d, V_d, n, a, mass, kin, rest, stream)
        assert e == pytest.approx(e_ref, rel=1e-12)
        assert n2 == pytest.approx(n2_ref, rel=1e-13)
        e_o, n2_o = oracle_energy(n, a, mass, kin, rest, psi, V)
        assert e == pytest.approx(e_o, rel=1e-12)
        assert n2 == pytest.approx(n2_o, rel=1e-13)


def test_noalloc_on_a_side_stream_leaves_its_inputs_unchanged(qfdlib):
    import torch

    n, a, mass, kin, rest, pot, seed = CASES[0]
    e_ref, n2_ref, psi, V = plan_energy(n, a, mass, kin, rest, pot, seed)
    psi_d = torch.from_numpy(psi.reshape(-1)).cuda()
    V_d = torch.from_numpy(V.reshape(-1)).cuda()
    psi_before, V_before = psi_d.clone(), V_d.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())  # the copies above are on the current stream
    with torch.cuda.stream(side):
        e, n2 = Q.energy_noalloc(psi_d, V_d, n, a, mass, kin, rest, side.cuda_stream)
    torch.cuda.synchronize()
    assert e == pytest.approx(e_ref, rel=1e-12) and n2 == pytest.approx(n2_ref, rel=1e-13)
    assert torch.equal(psi_d, psi_before) and torch.equal(V_d, V_before)


def test_noalloc_rejects_lattices_beyond_its_static_scratch(qfdlib):
    import torch

    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(Q.QfdError) as ei:
        Q.energy_noalloc(x, v, 256, 0.1, 1.0, 2)
    assert ei.value.status == Q.ERR_ARG


def test_noalloc_rejects_the_finite_difference_term(qfdlib):
    # H_K(0) has no Parseval form: only the FFT kinetic terms 1..3 are accepted
    import torch

    x = torch.zeros(8 ** 3, dtype=torch.complex128, device="cuda")
    v = torch.zeros(8 ** 3, dtype=torch.float64, device="cuda")
    for kin in (0, 4):
        with pytest.raises(Q.QfdError) as ei:
            Q.energy_noalloc(x, v, 8, 0.1, 1.0, kin)
        assert ei.value.status == Q.ERR_ARG
