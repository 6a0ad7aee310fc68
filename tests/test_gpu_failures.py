"""Failure detection without a GPU fault: every failure here is made on the host
(non-finite values copied in through the C ABI, a watchdog shorter than the
work it watches), and the library must report it as a status while the device
context stays usable for the next call."""
import numpy as np
import pytest

from oracle import qfd_oracle as O
from paper_2006_16935_gb300 import inputs
from paper_2006_16935_gb300 import qfd as Q

pytestmark = pytest.mark.gpu


def _plan(prec, n=16, **kw):
    return Q.Plan(n, 0.2, 1.0, 0.01, 2, precision=prec, ortho_every=10, check_every=20, max_steps=200,
                  tol=1e-9, **kw)


@pytest.mark.parametrize("prec", ["c128", "df64", "c64", "c64_refine_df"])
@pytest.mark.parametrize("bad", [np.nan, 1e300])
def test_non_finite_or_huge_state_is_reported_as_diverged(qfdlib, prec, bad):
    # a state whose norm is not finite (NaN, or |psi|^2 overflowing FP64 and
    # FP32) makes the first energy check of a solve return QFD_ERR_DIVERGED
    psi = inputs.uniform_psi(16, 1)
    psi[3, 4, 5] = bad
    with _plan(prec) as p:
        p.fill_potential("ho", (1.0,))
        p.set_psi(0, psi)
        with pytest.raises(Q.QfdError) as ei:
            p.solve_states(1)
        assert ei.value.status == Q.ERR_DIVERGED
        # the plan and the context are still usable: a clean start solves
        p.set_psi(0, inputs.uniform_psi(16, 2))
        es, _, conv = p.solve_states(1, allow_unconverged=True)
        assert np.isfinite(es[0])


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_potential_is_refused(qfdlib, bad):
    V = O.potential(16, 0.2, "ho", (1.0,))
    V[1, 2, 3] = bad
    with _plan("c128") as p:
        with pytest.raises(Q.QfdError) as ei:
            p.set_potential(V)
        assert ei.value.status == Q.ERR_UNSTABLE_DT
        # no potential is held after the refusal: stepping is out of order
        p.fill_psi_uniform(0, 1)
        with pytest.raises(Q.QfdError) as ei:
            p.step(0, 1)
        assert ei.value.status == Q.ERR_STATE
        # a finite potential is accepted afterwards
        V[1, 2, 3] = 0.0
        p.set_potential(V)
        p.step(0, 1)


def test_server_watchdog_ends_an_overrunning_request_with_timeout(qfdlib):
    slow = Q.make_request(128, 0.1, 1.0, 0.002, 2, precision="c128", potential="cornell", pot_coeffs=(0.3, 0.2),
                          seed=3, tol=1e-9, max_steps=100000)
    quick = Q.make_request(16, 0.3, 1.0, 0.01, 2, precision="c128", potential="ho", pot_coeffs=(1.0, 0.0),
                           seed=4, tol=1e-9, max_steps=20000)
    with Q.Server(64e9, check_every=100, ortho_every=10) as sv:
        with pytest.raises(Q.QfdError) as ei:
            sv.set_timeout(-1.0)
        assert ei.value.status == Q.ERR_ARG
        # a 128^3 period (100 steps) takes far longer than a microsecond
        sv.set_timeout(1e-6)
        rid = sv.submit(slow)
        res = sv.run_until_done(1)
        assert res[rid]["status"] == Q.ERR_TIMEOUT
        assert sv.stats()["active"] == 0 and sv.stats()["used_bytes"] == 0
        # the server and the device go on: without the watchdog a request solves
        sv.set_timeout(0.0)
        rid = sv.submit(quick)
        res = sv.run_until_done(1)
        assert res[rid]["status"] == Q.OK and np.isfinite(res[rid]["energy"][0])


def test_tma_pass_a_bounded_wait_reports_timeout_and_recovers(qfdlib):
    # the TMA-staged pass A with its barriers armed but no copy issued: every
    # wait runs out (about a second), the kernel stops with no copy in flight,
    # and the step reports QFD_ERR_TIMEOUT; afterwards the plan steps normally
    n, a, m, dt = 256, 0.05, 1.0, 5e-4
    psi0 = inputs.uniform_psi(n, 3)
    with Q.Plan(n, a, m, dt, 2, precision="c64", ortho_every=2) as p, \
            Q.Plan(n, a, m, dt, 2, precision="c64", ortho_every=2) as ref:
        assert p.has_tma()
        for q in (p, ref):
            q.fill_potential("softcoul", (0.01,))
        p.set_tuning(1, 0, -1, 2)
        p.set_psi(0, psi0)
        p.set_tma_test(1)
        with pytest.raises(Q.QfdError) as ei:
            p.step(0, 1)
        assert ei.value.status == Q.ERR_TIMEOUT
        p.set_tma_test(0)
        p.set_psi(0, psi0)
        p.step(0, 3)
        ref.set_psi(0, psi0)
        ref.step(0, 3)
        got, want = p.get_psi(0), ref.get_psi(0)
        assert np.linalg.norm(got - want) <= 2e-6 * np.linalg.norm(want)
