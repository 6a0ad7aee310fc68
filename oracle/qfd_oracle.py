"""Plain, slow FP64 CPU oracle of the imaginary-time FFT solver of arXiv:2006.16935.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import this module.  The product path (the CUDA
library under paper_2006_16935_gb300/csrc and its Python binding) never calls
it and shares no code, table or constant generator with it.

Everything is complex128 / float64 and follows the paper's notation:
lattice of N points per axis, spacing A, mass M, time step EPS = dtau,
kinetic term KINTERM in {0, 1, 2, 3}.

Sections and equations cited below are those of the paper:
  Sec. 2.1  kinetic terms: Eq. (eigenmodes), Eqs. (HK1)-(HK3), FFT/IFFT definitions;
            the finite-difference term H_K(0) with Dirichlet boundaries (Eq. HK0)
  Sec. 2.2  iterative procedure: Eq. (iter_proced) and the coefficients A, B
  Sec. 2.4  parity projection: Eq. (parity)
  Sec. 5.1  SNAPUPDATE (normalise + symmetrise cadence), TOLERANCE (stop rule)
  Sec. 5.3  hard-coded potentials (harmonic oscillator, Coulomb, Cornell)

Readings of points the paper leaves open:
  * energy estimator: Rayleigh quotient <psi|H_K + V|psi> / <psi|psi>
  * V_b = V, V_s = 0 (Sec. 5.1 recommends this)
  * relativistic term: rest_mass=1 keeps sqrt(p^2+M^2) as printed in Eq. (HK3);
    rest_mass=0 subtracts M (the sqrt(p^2+m^2)-m form)
  * lattice centre: on-grid site N/2 (reflection x -> (N-x) mod N) by default,
    or the paper's off-grid (N-1)/2 (reflection x -> N-1-x)
  * cadence: after every `ortho_every`-th step apply parity, then classical
    Gram-Schmidt against the lower states, then normalise; energy every
    `check_every` steps; stop when |E_t - E_prev| <= tol * |E_t| (or, with the
    optional tail rule, also when the geometric tail of the changes is within
    tol)
  * decay-rate energy: (1 - lambda) / dtau from the norm decay over the steps
    since the last normalisation, after the cadence's projections
  * snapshot-overlap excited states: snapshots after the cadence of every
    snap_every-th step; excited estimate k = the k-th latest snapshot before
    the end, deflated against the lower estimates

Pins (tests/test_oracle_pins.py): DFT against a brute-force textbook 3D DFT,
numpy.fft, deltas, plane waves and Parseval; H_K(2) against the periodic
7-point finite-difference Laplacian; H_K(3)^2 = 2M H_K(2) + M^2; H_K(1) on a
band-limited Gaussian against the continuum Laplacian; the update on plane
waves with constant V; the converged iteration against dense eigen-solvers of
independently assembled matrices (ground state, parity sector, Gram-Schmidt
deflated state); the 3D oscillator levels 3/2 w and 5/2 w; the heavy-mass
limit; parity and orthogonality invariants; the box-normalised hydrogen radii
printed in Sec. 3.3 (observables); the tail stop rule on geometric and turning
sequences; the decay-rate energy against the dense fixed-point eigenvalue; the
snapshot-overlap states on a three-plane-wave evolution with known levels.
No function here is unpinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

try:  # library FFT (multi-threaded) for the large-lattice mode
    import scipy.fft as _libfft

    def _lib_fftn(x):
        return _libfft.fftn(x, workers=-1)

    def _lib_ifftn_unnormalised(x):
        return _libfft.ifftn(x, norm="forward", workers=-1)
except ImportError:  # pragma: no cover
    def _lib_fftn(x):
        return np.fft.fftn(x)

    def _lib_ifftn_unnormalised(x):
        return np.fft.ifftn(x, norm="forward")

# --------------------------------------------------------------------------
# Sec. 2.1: momenta, DFT, kinetic symbols
# --------------------------------------------------------------------------


def k_modes(n: int) -> np.ndarray:
    """Eq. (eigenmodes): k = A p for DFT index j; k = 2 pi j / N for j <= N/2,
    2 pi (j - N) / N otherwise, so k lies in (-pi, pi] with Nyquist at +pi."""
    j = np.arange(n)
    m = np.where(j <= n // 2, j, j - n)
    return 2.0 * np.pi * m / n


def dft_matrix(n: int, sign: int) -> np.ndarray:
    """F[j, k] = exp(sign * 2 pi i * (j k mod N) / N).

    The exponent is reduced modulo N in integers before the angle is formed,
    so every entry is one of the N roots of unity."""
    j = np.arange(n)
    m = np.outer(j, j) % n
    ang = 2.0 * np.pi * m / n
    return np.cos(ang) + 1j * sign * np.sin(ang)


def dft_axis(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """Unnormalised 1D DFT along `axis`: X[k] = sum_j x[j] exp(sign 2 pi i j k / N)
    (Sec. 2.1, FFT/IFFT definitions; sign -1 forward, +1 inverse)."""
    n = x.shape[axis]
    f = dft_matrix(n, sign)
    y = np.tensordot(f, x, axes=([1], [axis]))  # new axis 0 = k
    return np.moveaxis(y, 0, axis)


def fft3(x: np.ndarray, method: str = "naive") -> np.ndarray:
    """FFT[Psi](k) = sum_x Psi(x) exp(-i k.x), unnormalised (Sec. 2.1).

    method 'naive' applies the DFT definition axis by axis; 'library' calls
    scipy.fft.fftn on all cores (a library FFT, used only at lattice sizes
    where the naive transform is too slow)."""
    if method == "library":
        return _lib_fftn(x)
    y = x.astype(np.complex128)
    for ax in range(3):
        y = dft_axis(y, ax, -1)
    return y


def ifft3(x: np.ndarray, method: str = "naive") -> np.ndarray:
    """IFFT[Psi~](x) = sum_k Psi~(k) exp(+i k.x), unnormalised (Sec. 2.1)."""
    if method == "library":
        return _lib_ifftn_unnormalised(x)
    y = x.astype(np.complex128)
    for ax in range(3):
        y = dft_axis(y, ax, +1)
    return y


def kinetic_symbol(n: int, a: float, mass: float, kinterm: int, rest_mass: int = 0) -> np.ndarray:
    """T(k1, k2, k3) on the [N, N, N] grid of DFT indices, without the 1/N^3.

    Eq. (HK1):  T = sum_l k_l^2 / (2 A^2 M)
    Eq. (HK2):  T = 4 sum_l sin^2(k_l / 2) / (2 A^2 M)
    Eq. (HK3):  T = sqrt(4 sum_l sin^2(k_l / 2) + (A M)^2) / A   [- M if rest_mass == 0]
    """
    k = k_modes(n)
    k1, k2, k3 = np.meshgrid(k, k, k, indexing="ij")
    return _symbol(k1, k2, k3, a, mass, kinterm, rest_mass)


def kinetic_symbol_at(n: int, a: float, mass: float, kinterm: int, idx: np.ndarray, rest_mass: int = 0) -> np.ndarray:
    """T(k) at the DFT index triples idx[:, 0..2] (the same formulas as
    kinetic_symbol, without building the whole N^3 table)."""
    k = k_modes(n)
    return _symbol(k[idx[:, 0]], k[idx[:, 1]], k[idx[:, 2]], a, mass, kinterm, rest_mass)


def _symbol(k1, k2, k3, a, mass, kinterm, rest_mass):
    if kinterm == 1:
        return (k1 ** 2 + k2 ** 2 + k3 ** 2) / (2.0 * a * a * mass)
    s = 4.0 * (np.sin(k1 / 2) ** 2 + np.sin(k2 / 2) ** 2 + np.sin(k3 / 2) ** 2)
    if kinterm == 2:
        return s / (2.0 * a * a * mass)
    if kinterm == 3:
        t = np.sqrt(s + (a * mass) ** 2) / a
        return t if rest_mass else t - mass
    raise ValueError(f"kinetic term {kinterm} is not an FFT kinetic term")


class FdtdKinetic:
    """H_K(0), the finite-difference kinetic term with Dirichlet boundaries
    (Sec. 2.1, Eq. HK0), normalised as its momentum-space form (Eq.
    HK0_momentum_space_1, (1/2M) sum_l (4/A^2) sin^2(k_l/2)), i.e.

        H_K(0) Psi = -(1 / (2 M A^2)) sum_l [Psi(r + A e_l) + Psi(r - A e_l) - 2 Psi(r)],

    with Psi = 0 outside the lattice (every lattice site evolves; the missing
    neighbours of an edge site are zero)."""

    def __init__(self, a: float, mass: float):
        self.a, self.mass = a, mass

    def __call__(self, psi: np.ndarray) -> np.ndarray:
        p = np.pad(psi, 1)
        lap = (p[2:, 1:-1, 1:-1] + p[:-2, 1:-1, 1:-1] + p[1:-1, 2:, 1:-1] + p[1:-1, :-2, 1:-1]
               + p[1:-1, 1:-1, 2:] + p[1:-1, 1:-1, :-2] - 6.0 * psi)
        return -lap / (2.0 * self.mass * self.a * self.a)


def kinetic_max(n: int, a: float, mass: float, kinterm: int, rest_mass: int = 0) -> float:
    """Largest eigenvalue of H_K on the lattice (max of T over the modes); for
    H_K(0) the bound 6 / (A^2 M) of its momentum-space form."""
    if kinterm == 0:
        return 6.0 / (a * a * mass)
    return float(np.max(kinetic_symbol(n, a, mass, kinterm, rest_mass)))


def apply_kinetic(psi: np.ndarray, T, method: str = "naive") -> np.ndarray:
    """H_K Psi = (1/N^3) IFFT[T * FFT[Psi]]  (Eqs. HK1-HK3); T may instead be
    the finite-difference operator FdtdKinetic (Eq. HK0)."""
    if callable(T):
        return T(psi)
    n3 = psi.size
    return ifft3(T * fft3(psi, method), method) / n3


# --------------------------------------------------------------------------
# Sec. 2.2: the iterative procedure
# --------------------------------------------------------------------------


def update_coefficients(V: np.ndarray, dtau: float):
    """A = (1 - dtau V/2) / (1 + dtau V/2),  B = 1 / (1 + dtau V/2)  (Sec. 2.2)."""
    h = 0.5 * dtau * V
    return (1.0 - h) / (1.0 + h), 1.0 / (1.0 + h)


def imaginary_time_step(psi, V, T, dtau, method="naive"):
    """Eq. (iter_proced): Psi(tau + dtau) = A Psi(tau) - B dtau H_K Psi(tau)."""
    A, B = update_coefficients(V, dtau)
    return A * psi - B * dtau * apply_kinetic(psi, T, method)


# --------------------------------------------------------------------------
# Sec. 2.4: parity; Sec. 2.2 / 5.1: Gram-Schmidt, normalisation, energy
# --------------------------------------------------------------------------


def reflect(psi: np.ndarray, centre: str = "grid") -> np.ndarray:
    """Psi(-r) on the lattice: r measured from the potential's centre.

    centre 'grid': centre at site N/2, so x -> (N - x) mod N.
    centre 'offgrid': centre at (N-1)/2, so x -> N - 1 - x."""
    n = psi.shape[0]
    if centre == "grid":
        idx = (n - np.arange(n)) % n
    elif centre == "offgrid":
        idx = n - 1 - np.arange(n)
    else:
        raise ValueError(centre)
    return psi[np.ix_(idx, idx, idx)]


def reflect_axes(psi: np.ndarray, axes, centre: str = "grid") -> np.ndarray:
    """Psi with the coordinates of `axes` (a subset of 0, 1, 2) reflected about
    the centre, the others kept."""
    n = psi.shape[0]
    flip = (n - np.arange(n)) % n if centre == "grid" else n - 1 - np.arange(n)
    keep = np.arange(n)
    ix = [flip if k in axes else keep for k in range(3)]
    return psi[np.ix_(*ix)]


def axis_parity_minus(psi: np.ndarray, k: int, centre: str = "grid") -> np.ndarray:
    """P-_{e_k} of Eq. (parity_axis) (read with the missing comma restored),
    normalised as a projector: (1/4) [psi(x) + psi with the two other axes
    reflected - psi with axis k reflected - psi(-x)] (the printed 1/2 makes the
    operator twice a projector)."""
    others = tuple(j for j in range(3) if j != k)
    return 0.25 * (psi + reflect_axes(psi, others, centre) - reflect_axes(psi, (k,), centre) - reflect(psi, centre))


def parity_project(psi, parity: int, centre: str = "grid"):
    """Eq. (parity): P+- Psi(r) = (Psi(r) +- Psi(-r)) / 2; parity 0 leaves Psi alone."""
    if parity == 0:
        return psi
    return 0.5 * (psi + parity * reflect(psi, centre))


def inner(u, v) -> complex:
    """<u|v> = sum_x conj(u(x)) v(x)."""
    return complex(np.vdot(u.ravel(), v.ravel()))


def gram_schmidt(psi, lower):
    """Classical Gram-Schmidt: Psi <- Psi - sum_j <phi_j|Psi> phi_j, all overlaps
    taken from the same input Psi (the lower states phi_j are orthonormal)."""
    coeffs = [inner(phi, psi) for phi in lower]
    out = psi.copy()
    for c, phi in zip(coeffs, lower):
        out = out - c * phi
    return out


def norm2(psi) -> float:
    return float(np.sum(np.abs(psi) ** 2))


def normalize(psi):
    """Sum over the full lattice of |Psi|^2 = 1 (Sec. 2.2)."""
    return psi / math.sqrt(norm2(psi))


def energy(psi, V, T, method="naive") -> float:
    """Rayleigh quotient <Psi|H_K + V|Psi> / <Psi|Psi> (energy estimator reading)."""
    hk = apply_kinetic(psi, T, method)
    num = inner(psi, hk + V * psi)
    return num.real / norm2(psi)


# --------------------------------------------------------------------------
# Sec. 5.3: potentials (the synthetic workloads' forms)
# --------------------------------------------------------------------------


def displacement(n: int, centre: str = "grid") -> np.ndarray:
    """Lattice displacement from the centre, per axis, in lattice units.

    'grid': d = x - N/2 in [-N/2, N/2 - 1]; 'offgrid': d = x - (N-1)/2."""
    x = np.arange(n, dtype=np.float64)
    return x - (n // 2) if centre == "grid" else x - (n - 1) / 2.0


def radius(n: int, a: float, centre: str = "grid") -> np.ndarray:
    d = displacement(n, centre)
    d1, d2, d3 = np.meshgrid(d, d, d, indexing="ij")
    return a * np.sqrt(d1 * d1 + d2 * d2 + d3 * d3)


def potential(n: int, a: float, kind: str, params=(), centre: str = "grid") -> np.ndarray:
    """V(r) on the lattice, r = A |x - centre|.

    'zero':      V = 0                                  (POTENTIAL 0)
    'ho':        V = k r^2 / 2,   params (k,)           (POTENTIAL 4, read as +r^2/2)
    'cornell':   V = -kappa / r + sigma r, r >= A/2     (POTENTIAL 6 without string breaking)
    'coulomb':   V = -1 / r, r >= A/2                   (POTENTIAL 2 clamped at the origin)
    'softcoul':  V = -1 / sqrt(r^2 + eps2), params (eps2,)
    """
    return potential_of_radius(radius(n, a, centre), a, kind, params)


def potential_at(n: int, a: float, kind: str, params, sites: np.ndarray, centre: str = "grid") -> np.ndarray:
    """V at the lattice sites `sites` (integer array [m, 3] of x1, x2, x3),
    without building the whole lattice: the same V(r) as `potential`."""
    d = displacement(n, centre)[np.asarray(sites)]
    r = a * np.sqrt(np.sum(d * d, axis=1))
    return potential_of_radius(r, a, kind, params)


def potential_of_radius(r: np.ndarray, a: float, kind: str, params=()) -> np.ndarray:
    """The potential forms of `potential` as functions of r = A |x - centre|."""
    if kind == "zero":
        return np.zeros_like(r)
    if kind == "ho":
        k = params[0] if params else 1.0
        return 0.5 * k * r * r
    if kind == "cornell":
        kappa, sigma = params
        rc = np.maximum(r, 0.5 * a)
        return -kappa / rc + sigma * rc
    if kind == "coulomb":
        rc = np.maximum(r, 0.5 * a)
        return -1.0 / rc
    if kind == "softcoul":
        eps2 = params[0] if params else 0.01
        return -1.0 / np.sqrt(r * r + eps2)
    raise ValueError(kind)


# --------------------------------------------------------------------------
# Sec. 2.3 / 2.4 / 5.1: observables
# --------------------------------------------------------------------------


def observables(psi, centre: str = "grid", min_sep_edge: float = 0.3) -> dict:
    """Observables of a state, in lattice units, d = x - centre per axis:

    box normalisation (Sec. 2.3): the effective volume keeps the sites with
    |d_l| <= (1 - min_sep_edge) N / 2 on every axis; <rho>_box = sum over the box
    of rho |psi|^2 / sum over the box of |psi|^2 (Eq. (box_normalization));
    parity weights (Sec. 2.4): sum over the box of |P+- psi|^2, box-normalised,
    so that w+ + w- = 1, and of |P-_{e_k} psi|^2 for the three axes;
    UPDATE observables (Sec. 5.1): <x>, <y>, <z>, <rho^2> over the full lattice.
    """
    n = psi.shape[0]
    d = displacement(n, centre)
    d1, d2, d3 = np.meshgrid(d, d, d, indexing="ij")
    rho = np.sqrt(d1 * d1 + d2 * d2 + d3 * d3)
    half = (1.0 - min_sep_edge) * n / 2.0
    box = (np.abs(d1) <= half) & (np.abs(d2) <= half) & (np.abs(d3) <= half)
    p2 = np.abs(psi) ** 2
    n_full = p2.sum()
    n_box = p2[box].sum()
    refl = reflect(psi, centre)
    wp = (np.abs(0.5 * (psi + refl)) ** 2)[box].sum() / n_box
    wm = (np.abs(0.5 * (psi - refl)) ** 2)[box].sum() / n_box
    wax = [(np.abs(axis_parity_minus(psi, k, centre)) ** 2)[box].sum() / n_box for k in range(3)]
    return {"norm2": float(n_full), "norm2_box": float(n_box),
            "rho_box": float((rho * p2)[box].sum() / n_box),
            "rho2": float((rho * rho * p2).sum() / n_full),
            "x": float((d1 * p2).sum() / n_full), "y": float((d2 * p2).sum() / n_full),
            "z": float((d3 * p2).sum() / n_full),
            "w_plus": float(wp), "w_minus": float(wm),
            "w_axis1": float(wax[0]), "w_axis2": float(wax[1]), "w_axis3": float(wax[2])}


def random_field(noise: np.ndarray, corr: float, amplitude: float) -> np.ndarray:
    """Smooth Gaussian random field from white noise (the seeded stand-in for
    the paper's file-based potentials): multiply the noise by
    exp(-k^2 corr^2 / 2) in momentum space (k per axis from Eq. (eigenmodes),
    corr in lattice units), transform back, then shift and scale the result to
    mean 0 and standard deviation `amplitude` over the lattice."""
    n = noise.shape[0]
    k = k_modes(n)
    g = np.exp(-0.5 * corr * corr * k * k)
    f = np.fft.ifftn(np.fft.fftn(noise) * g[:, None, None] * g[None, :, None] * g[None, None, :]).real
    f = f - f.mean()
    return amplitude * f / np.sqrt((f * f).mean())


# --------------------------------------------------------------------------
# The solve loop (Sec. 2.2 evolution; Sec. 5.1 SNAPUPDATE / TOLERANCE cadence)
# --------------------------------------------------------------------------


@dataclass
class Problem:
    n: int
    a: float
    mass: float
    dtau: float
    kinterm: int
    V: np.ndarray
    rest_mass: int = 0
    centre: str = "grid"
    ortho_every: int = 10
    check_every: int = 100
    method: str = "naive"
    T: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        if self.T is None:
            self.T = FdtdKinetic(self.a, self.mass) if self.kinterm == 0 else \
                kinetic_symbol(self.n, self.a, self.mass, self.kinterm, self.rest_mass)


def cadence_n2(psi, prob: Problem, parity: int, lower):
    """Parity projection, then Gram-Schmidt against the lower states, then
    normalisation.  Returns (normalised psi, squared norm before normalising)."""
    psi = parity_project(psi, parity, prob.centre)
    if lower:
        psi = gram_schmidt(psi, lower)
    n2 = norm2(psi)
    return psi / np.sqrt(n2), n2


def cadence(psi, prob: Problem, parity: int, lower):
    """Parity projection, then Gram-Schmidt against the lower states, then normalisation."""
    return cadence_n2(psi, prob, parity, lower)[0]


def decay_energy(n2: float, k: int, dtau: float) -> float:
    """The decay-rate energy estimator (1 - lambda) / dtau, with lambda the
    per-step norm ratio ||psi_(t+1)|| / ||psi_t|| (Sec. 2.2: the state decays
    as exp(-E tau)); n2 is the squared norm after k steps (and the cadence's
    projections) from a normalised state, so lambda = n2^(1/(2k))."""
    return (1.0 - n2 ** (0.5 / k)) / dtau


def evolve_n2(psi, prob: Problem, nsteps: int, t0: int = 0, parity: int = 0, lower=()):
    """evolve, also returning the squared norm before the last cadence's
    normalisation (None when no cadence ran)."""
    t = t0
    n2 = None
    for _ in range(nsteps):
        psi = imaginary_time_step(psi, prob.V, prob.T, prob.dtau, prob.method)
        t += 1
        if t % prob.ortho_every == 0:
            psi, n2 = cadence_n2(psi, prob, parity, lower)
    return psi, t, n2


def evolve(psi, prob: Problem, nsteps: int, t0: int = 0, parity: int = 0, lower=()):
    """Advance nsteps steps of Eq. (iter_proced) from step counter t0; after each
    step t with t % ortho_every == 0 apply the cadence.  Returns (psi, t)."""
    psi, t, _ = evolve_n2(psi, prob, nsteps, t0, parity, lower)
    return psi, t


@dataclass
class StateResult:
    energy: float
    psi: np.ndarray
    steps: int
    converged: bool
    history: list
    e_decay: float = float("nan")  # decay-rate energy at the last check


def stop_check(energies, tol: float, rule: str = "paper") -> bool:
    """Stop rule after the latest energy check (energies: every check so far).

    "paper": TOLERANCE of Sec. 5.1, d_k = |E_k - E_(k-1)| <= tol |E_k|.
    "tail": the same, and besides the change still to come is bounded.  The
    update operator is not symmetric, so its fixed point is not an eigenvector
    of H and the energy error is linear in the slowest remaining modes: it can
    fall below the limit and turn back, and a component of one sign can hide
    behind a faster one of the other.  So stop only when d_k <= 1e-3 tol |E_k|,
    or when the last three differences share one sign, their ratio
    r = D_k / D_(k-1) has not fallen (r >= 0.9 D_(k-1) / D_(k-2), i.e. one mode
    dominates) and the geometric tail d_k r / (1 - r) <= tol |E_k|."""
    if tol < 0 or len(energies) < 2:
        return False
    e = energies[-1]
    dk = e - energies[-2]
    if abs(dk) > tol * abs(e):
        return False
    if rule == "paper" or abs(dk) <= 1e-3 * tol * abs(e):
        return True
    if len(energies) < 4:
        return False
    d1 = energies[-2] - energies[-3]
    d2 = energies[-3] - energies[-4]
    if not (dk * d1 > 0 and d1 * d2 > 0):
        return False
    r, r_prev = dk / d1, d1 / d2
    return r < 1.0 and r >= 0.9 * r_prev and abs(dk) * r / (1.0 - r) <= tol * abs(e)


def solve_state(psi0, prob: Problem, max_steps: int, tol: float, parity: int = 0, lower=(), rule: str = "paper"):
    """One state: cadence at t = 0, then steps; every check_every steps the energy
    is taken and the loop stops once stop_check says so (tol < 0: never)."""
    psi = cadence(psi0.astype(np.complex128), prob, parity, lower)
    t = 0
    energies = []
    hist = []
    converged = False
    e_decay = float("nan")
    while t < max_steps:
        psi, t, n2 = evolve_n2(psi, prob, prob.check_every, t, parity, lower)
        e = energy(psi, prob.V, prob.T, prob.method)
        if n2 is not None and t % prob.ortho_every == 0:
            e_decay = decay_energy(n2, prob.ortho_every, prob.dtau)
        hist.append((t, e))
        energies.append(e)
        if stop_check(energies, tol, rule):
            converged = True
            break
    return StateResult(e, normalize(psi), t, converged, hist, e_decay)


def snapshot_states(psi0, prob: Problem, max_steps: int, tol: float, snap_every: int, parity: int = 0,
                    nout: int = 3, rule: str = "paper"):
    """Excited states from snapshots of one evolution (Sec. 2.2).

    The state is evolved as in solve_state; after the cadence of every step t
    with t % snap_every == 0 the normalised state is kept as a snapshot.  The
    ground-state estimate is the final state; the k-th excited estimate is the
    k-th latest snapshot taken before the end, with the parity projection and
    the components along the lower estimates removed, normalised."""
    psi = cadence(psi0.astype(np.complex128), prob, parity, ())
    t = 0
    snaps = []  # (step, snapshot), newest first
    energies, hist = [], []
    converged = False
    e = float("nan")
    while t < max_steps:
        for _ in range(prob.check_every):
            psi = imaginary_time_step(psi, prob.V, prob.T, prob.dtau, prob.method)
            t += 1
            if t % prob.ortho_every == 0:
                psi = cadence(psi, prob, parity, ())
                if nout > 1 and t % snap_every == 0:
                    snaps.insert(0, (t, psi.copy()))
                    del snaps[nout:]
        e = energy(psi, prob.V, prob.T, prob.method)
        hist.append((t, e))
        energies.append(e)
        if stop_check(energies, tol, rule):
            converged = True
            break
    states = [normalize(psi)]
    sources = [p for (ts, p) in snaps if ts < t][:nout - 1]
    if len(sources) < nout - 1:
        raise ValueError("fewer snapshots than excited states")
    out = [StateResult(e, states[0], t, converged, hist)]
    for src in sources:
        phi = cadence(src, prob, parity, tuple(states))
        states.append(phi)
        out.append(StateResult(energy(phi, prob.V, prob.T, prob.method), phi, t, converged, []))
    return out


def solve_states(psi0s, prob: Problem, max_steps: int, tol: float, parities=None, rule: str = "paper"):
    """Ground and excited states in turn; state i is Gram-Schmidt deflated
    against the converged states 0..i-1 (each normalised)."""
    out = []
    lower = []
    for i, p0 in enumerate(psi0s):
        par = 0 if parities is None else parities[i]
        res = solve_state(p0, prob, max_steps, tol, par, tuple(lower), rule)
        out.append(res)
        lower.append(res.psi)
    return out
