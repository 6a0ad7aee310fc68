"""Host-side checks that need no GPU: the C ABI library, argument validation,
the plan-time stability check and the seeded input generator."""
import ctypes
import math

import numpy as np
import pytest

from oracle import qfd_oracle as O
from paper_2006_16935_gb300 import build, inputs, qfd


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return qfd.load()


def test_library_exports_every_header_function(lib):
    names = qfd.header_functions()
    assert len(names) >= 19
    missing = [f for f in names if not hasattr(lib, f)]
    assert not missing


def _params(**kw):
    base = dict(n=32, a=0.1, mass=1.0, dtau=0.001, kinetic=1, rest_mass=0, nstates=1, precision=0,
                ortho_every=100, check_every=100, centre=0, stop_rule=0, max_steps=2000, tol=-1.0,
                tol_bulk=1e-6, stream=None)
    base.update(kw)
    return qfd.QfdParams(**base)


def _plan_status(lib, **kw):
    h = ctypes.c_void_p()
    st = lib.qfd_plan(ctypes.byref(_params(**kw)), ctypes.byref(h))
    if h.value:
        lib.qfd_destroy(h)
    return st, lib.qfd_last_error(None).decode()


@pytest.mark.parametrize("bad", [dict(n=48), dict(n=2048), dict(a=0.0), dict(mass=-1.0), dict(dtau=0.0),
                                 dict(kinetic=-1), dict(kinetic=4), dict(nstates=0), dict(nstates=9),
                                 dict(precision=5), dict(ortho_every=0), dict(check_every=0), dict(centre=2),
                                 dict(stop_rule=2), dict(rest_mass=2), dict(max_steps=-1)])
def test_plan_rejects_bad_arguments(lib, bad):
    st, msg = _plan_status(lib, **bad)
    assert st == qfd.ERR_ARG and msg


def test_plan_rejects_unstable_time_step(lib):
    # 32^3, A = 0.1, M = 1, H_K(1): max T = 3 pi^2 / (2 A^2 M) = 1480.4; dtau = 0.002 gives 2.96 >= 2
    st, msg = _plan_status(lib, dtau=0.002, kinetic=1)
    assert st == qfd.ERR_UNSTABLE_DT and "2.96" in msg
    tmax = O.kinetic_max(32, 0.1, 1.0, 1)
    assert 0.002 * tmax == pytest.approx(2.9608813, rel=1e-6)
    # just below and just above the bound, for every kinetic term
    for kin in (1, 2, 3):
        tmax = O.kinetic_max(32, 0.1, 1.0, kin)
        st, _ = _plan_status(lib, kinetic=kin, dtau=2.0001 / tmax)
        assert st == qfd.ERR_UNSTABLE_DT
        st, _ = _plan_status(lib, kinetic=kin, dtau=1.9999 / tmax)
        assert st != qfd.ERR_UNSTABLE_DT  # (fails later without a GPU, with QFD_ERR_CUDA)


def test_step_batch_rejects_bad_batches_without_a_plan(lib):
    # rejected before any plan is touched: null arrays, count outside 1..32
    P = ctypes.c_void_p * 33
    I = ctypes.c_int * 33
    for plans, states, count in [(None, None, 1), (P(), I(), 0), (P(), I(), 33), (P(), I(), -2), (P(), I(), 1)]:
        st = lib.qfd_step_batch(plans, states, count, 1)
        assert st == qfd.ERR_ARG
        assert "qfd_step_batch" in lib.qfd_last_error(None).decode()
    # the binding: one state per plan, and the library's rejection of an empty batch
    class Fake:
        h = None
    with pytest.raises(ValueError):
        qfd.step_batch([Fake(), Fake()], [0], 1)
    with pytest.raises(qfd.QfdError) as e:
        qfd.step_batch([], 0, 1)
    assert e.value.status == qfd.ERR_ARG
    import re
    hdr = open(qfd.HEADER_PATH).read()
    assert int(re.search(r"#define QFD_MAX_BATCH (\d+)", hdr).group(1)) == qfd.MAX_BATCH == 32


def test_splitmix64_published_first_output():
    # SplitMix64 from state 0 yields 0xE220A8397B1DCDAF first (Steele, Lea, Flood 2014; Vigna's splitmix64.c)
    assert int(inputs.splitmix64(np.array([0], np.uint64))[0]) == 0xE220A8397B1DCDAF


def test_uniform_psi_is_seeded_and_in_range():
    a = inputs.uniform_psi(8, 3)
    b = inputs.uniform_psi(8, 3)
    c = inputs.uniform_psi(8, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    v = a.view(np.float64)
    assert v.min() >= -1 and v.max() < 1
    assert abs(v.mean()) < 0.1 and math.isclose(v.var(), 1 / 3, rel_tol=0.15)
    # chunked generation is identical to one-shot generation
    d = inputs.uniform_psi(8, 3, chunk=7)
    assert np.array_equal(a, d)


def test_binding_struct_sizes_match_the_header():
    import ctypes

    assert ctypes.sizeof(qfd.QfdParams) == 96
    assert ctypes.sizeof(qfd.Request) == 168 and qfd.Request.pot_coeffs.offset == 56
    assert ctypes.sizeof(qfd.Result) == 232
    assert ctypes.sizeof(qfd.ServerParams) == 40 and qfd.ServerParams.cohorts.offset == 32
    assert qfd.ServerParams.autotune.offset == 36


def test_server_watchdog_and_fma_probe_reject_bad_arguments_without_a_gpu(lib):
    # argument checks that run before any CUDA call
    assert lib.qfd_server_set_timeout(None, 1.0) == qfd.ERR_ARG
    assert lib.qfd_fma_rate(2, None) == qfd.ERR_ARG
    t = ctypes.c_double()
    assert lib.qfd_fma_rate(-1, ctypes.byref(t)) == qfd.ERR_ARG
