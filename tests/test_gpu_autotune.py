"""The launch-shape autotuner: every tile width / line grouping it chooses
between computes the same arithmetic per line, so results agree to rounding
(the compiler may contract a multiply-add into an FMA differently in the
different instantiations of the complex128 and complex64 kernels; the
double-float kernels spell every rounding out and are bit-identical), and a
tuned plan solves as an untuned one."""
import numpy as np
import pytest

from paper_2006_16935_gb300 import qfd as Q

pytestmark = pytest.mark.gpu

POLICY = {"c128": 0, "c64": 1, "df64": 2}


@pytest.mark.parametrize("prec", ["c128", "c64", "df64"])
@pytest.mark.parametrize("n", [16, 64, 128, 256, 512])
def test_every_launch_shape_gives_identical_states(qfdlib, n, prec):
    outs = []
    for vy, vz, vx in [(0, -1, 0), (1, -1, 0), (0, 0, 0), (0, 1, 0), (0, -1, 1), (1, 1, 1), (2, 2, 0), (2, 1, 2)]:
        with Q.Plan(n, 0.1, 1.3, 1e-4, 2, ortho_every=5, precision=prec) as p:
            p.set_tuning(POLICY[prec], vy, vz, vx)
            p.fill_potential("cornell", (0.3, 0.2))
            p.fill_psi_uniform(0, 4)
            p.step(0, 12)
            outs.append(p.get_psi(0))
    tol = {"df64": 0.0, "c128": 1e-14, "c64": 2e-6}[prec]
    if prec == "df64":  # no two-stage schedule, no TMA pass A: both run the defaults
        assert np.array_equal(outs[-2], outs[0]) and np.array_equal(outs[-1], outs[0])
    for o in outs[1:]:
        if tol == 0.0:
            assert np.array_equal(o, outs[0])
        else:
            assert np.linalg.norm(o - outs[0]) <= tol * np.linalg.norm(outs[0])


@pytest.mark.parametrize("prec", ["c64_refine_df", "c128"])
def test_autotuned_solve_is_bit_identical(qfdlib, prec):
    kw = dict(nstates=2, ortho_every=10, check_every=50, max_steps=20000, tol=1e-10, precision=prec)
    res = []
    for tune in (False, True):
        with Q.Plan(64, 0.2, 1.0, 2e-3, 2, **kw) as p:
            if tune:
                times = p.autotune()
                used = {"c64_refine_df": {"c64", "df64"}, "c128": {"c128"}}[prec]
                assert set(times) == used
                for t in times.values():
                    assert all(x > 0 for x in t["y"][:2] + t["z"][:2])
            p.fill_potential("ho", (1.0,))
            if tune:
                times = p.autotune()  # with a potential: pass A's tile width too
                for t in times.values():
                    assert all(x > 0 for x in t["x"][:2])
            p.fill_psi_uniform(0, 1)
            p.fill_psi_uniform(1, 2)
            res.append(p.solve_states(2, [1, -1]))
    (e0, s0, c0), (e1, s1, c1) = res
    assert c0 and c1 and s0 == s1
    assert e0 == pytest.approx(e1, rel=1e-12)
