"""Host check of the scaled-twiddle table of the complex128 radix-8 stages
(qfd::scaled_twiddle_table in csrc/qfd_launch.h).

The table is compiled into a small host program, which writes it for several
lattice sizes.  Each entry is then put through the butterfly algebra that
scaled_bfly8 applies, restated here with numpy.  The result must equal the
twiddled DFT-8, sum_r x_r w^(e0 r) exp(DIR 2 pi i r k / 8), with the DFT-8
formed as a matrix product, for every e0 and both directions.  A wrong form bit,
factor, ratio, slot or direction block changes that result far beyond rounding.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2006_16935_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"
SIZES = (64, 128, 256, 512, 1024)

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "qfd_launch.h"
int main(int argc, char** argv) {
  const long n = std::atol(argv[1]);
  std::vector<double2> tw(3 * n);
  for (long e = 0; e < n; ++e) {
    const long double a = 2.0L * 3.14159265358979323846264338327950288L * (long double)e / (long double)n;
    tw[e] = double2{(double)cosl(a), (double)-sinl(a)};
  }
  qfd::scaled_twiddle_table(n, tw.data(), tw.data() + n);
  std::fwrite(tw.data(), sizeof(double2), 3 * n, stdout);
  return 0;
}
"""


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx or not os.path.isdir(CUDA_INC):
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    d = tmp_path_factory.mktemp("tw")
    src, exe = d / "harness.cpp", d / "harness"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I" + CUDA_INC, "-I" + CSRC, str(src), "-o", str(exe)], check=True)
    out = {}
    for n in SIZES:
        raw = subprocess.run([str(exe), str(n)], check=True, capture_output=True).stdout
        out[n] = np.frombuffer(raw, dtype=np.float64).reshape(3 * n, 2)
    return out


def mul_i(a, DIR):  # DIR i a
    return 1j * a if DIR > 0 else -1j * a


def butterfly(x, ent, bits, DIR):
    """The scaled-twiddle radix-8 butterfly, step by step as scaled_bfly8."""
    tc = ent[:8]
    s1, s2, s4, r13, r15, r26, r37, kap = ent[8:]
    z = [x[0]]
    for r in range(1, 8):
        a = x[r]
        z.append(a * (tc[r] + 1j) if (bits >> r) & 1 else a * (1 + 1j * tc[r]))
    s0, d0 = z[0] + s4 * z[4], z[0] - s4 * z[4]
    s1p, d1p = z[2] + r26 * z[6], mul_i(z[2] - r26 * z[6], DIR)
    E = [s0 + s2 * s1p, d0 + s2 * d1p, s0 - s2 * s1p, d0 - s2 * d1p]
    t0, u0 = z[1] + r15 * z[5], z[1] - r15 * z[5]
    t1, u1 = z[3] + r37 * z[7], mul_i(z[3] - r37 * z[7], DIR)
    w8 = (lambda a: (1 + DIR * 1j) * a)  # without 1/sqrt 2, carried by kap
    O = [t0 + r13 * t1, w8(u0 + r13 * u1), mul_i(t0 - r13 * t1, DIR), mul_i(w8(u0 - r13 * u1), DIR)]
    sc = [s1, kap, s1, kap]
    X = np.zeros(8, complex)
    for k in range(4):
        X[k], X[k + 4] = E[k] + sc[k] * O[k], E[k] - sc[k] * O[k]
    return X


@pytest.mark.parametrize("n", SIZES)
def test_scaled_butterfly_equals_twiddled_dft8(tables, n):
    raw = tables[n]
    # the plain twiddles are left as they were
    e = np.arange(n)
    assert np.allclose(raw[:n, 0] + 1j * raw[:n, 1], np.exp(-2j * np.pi * e / n), atol=1e-15)
    blk = raw[n:].reshape(2, n // 8, 16)
    rng = np.random.default_rng(n)
    k = np.arange(8)
    worst = 0.0
    for d, DIR in ((0, -1), (1, 1)):
        F = np.exp(DIR * 2j * np.pi * np.outer(k, k) / 8)
        for e0 in range(n // 8):
            ent = blk[d, e0].copy()
            bits = int(np.frombuffer(ent[0].tobytes(), dtype=np.int64)[0])
            assert 0 <= bits < 256 and bits & 1 == 0
            ent[0] = 0.0
            # every form keeps |tan|, |cot| <= 1 and |s| >= 1/sqrt 2
            assert np.all(np.abs(ent[1:8]) <= 1.0 + 1e-15)
            assert min(abs(ent[8]), abs(ent[9]), abs(ent[10])) >= 0.7071
            x = rng.standard_normal(8) + 1j * rng.standard_normal(8)
            want = F @ (x * np.exp(DIR * 2j * np.pi * e0 * k / n))
            got = butterfly(x, ent, bits, DIR)
            worst = max(worst, np.abs(got - want).max() / np.abs(want).max())
    assert worst < 1e-14, worst


def test_cot_form_is_taken_at_quarter_turns(tables):
    # at theta = pi/2 (e0 r / n = 1/4) the tangent form would divide by zero
    n = 64
    blk = tables[n][n:].reshape(2, n // 8, 16)
    bits = int(np.frombuffer(blk[0, 4, 0].tobytes(), dtype=np.int64)[0])  # e0 = 4, r = 4: 16/64
    assert (bits >> 4) & 1
    assert abs(blk[0, 4, 4]) < 1e-15  # cot(pi/2), from a cosine of the harness's rounding
