// C ABI and plan runtime of the imaginary-time FFT solver (see include/qfd.h).
//
// The runtime keeps, per plan, a stack of states, one work lattice W and a
// small state machine recording how far the current step's passes have run on
// W, so that an energy check reuses the next step's forward passes instead of
// transforming psi again.  All arithmetic of the method runs in the kernels of
// qfd_kernels.cuh and the small kernels below; the host only sequences
// launches, sets up tables and takes the convergence decision.
#include <cuda.h>  // CUtensorMap and the tensor-map encoder's signature (called through the runtime)
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <deque>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "qfd.h"
#include "qfd_kernels.cuh"
#include "qfd_launch.h"

using namespace qfd;

namespace {

thread_local std::string g_create_error;

enum Stage { ST_NONE = 0, ST_X = 1, ST_XY = 2, ST_C = 3, ST_D = 4 };
// device scalar slots
enum { SC_SUMS = 0, SC_N2 = 40, SC_PV = 41, SC_PT = 42, SC_SCALE = 43, SC_E = 44, SC_COUNT = 64 };
enum { OP_SUMS = 0, OP_NORM = 1, OP_N2PV = 2, OP_ENERGY = 3, OP_OBS = 4 };
constexpr int NOBS = 12;
constexpr int GS_BLOCKS = 4 * 152;
constexpr int FIN_THREADS = 1024;

}  // namespace

// ============================================================ small kernels
namespace qfd {

// Fixed-order sums of per-CTA partials, then the derived scalars of `op`.
__global__ void __launch_bounds__(FIN_THREADS)
k_finalize_op(const double* __restrict__ part, int nq, int count, double* __restrict__ scal, float* __restrict__ scalf,
              int op) {
  __shared__ double red[32];
  __shared__ double sums[2 * MAX_LOWER];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < nq; ++q) {
    double x = 0.0;
    for (int i = threadIdx.x; i < count; i += FIN_THREADS) x += part[(int64_t)q * count + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
      double y = red[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
      if (lane == 0) sums[q] = y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (op == OP_SUMS) {
      for (int q = 0; q < nq; ++q) scal[SC_SUMS + q] = sums[q];
    } else if (op == OP_NORM || op == OP_N2PV) {
      scal[SC_N2] = sums[0];
      scal[SC_PV] = sums[1];
      if (op == OP_NORM) {
        const double f = 1.0 / sqrt(sums[0]);
        scal[SC_SCALE] = f;
        const df d = dsplit(f);
        scalf[0] = (float)f;
        scalf[1] = d.h;
        scalf[2] = d.l;
      }
    } else if (op == OP_ENERGY) {
      scal[SC_PT] = sums[0];
      scal[SC_E] = (sums[0] + scal[SC_PV]) / scal[SC_N2];
    } else if (op == OP_OBS) {
      // sums: n2, n2_box, rho_box, rho^2, x, y, z, |P+ psi|^2_box, |P- psi|^2_box,
      // |P-_e1 psi|^2_box, |P-_e2 psi|^2_box, |P-_e3 psi|^2_box
      const double n2 = sums[0], nb = sums[1];
      scal[SC_SUMS + 0] = n2;
      scal[SC_SUMS + 1] = nb;
      scal[SC_SUMS + 2] = sums[2] / nb;
      scal[SC_SUMS + 3] = sums[3] / n2;
      scal[SC_SUMS + 4] = sums[4] / n2;
      scal[SC_SUMS + 5] = sums[5] / n2;
      scal[SC_SUMS + 6] = sums[6] / n2;
      scal[SC_SUMS + 7] = sums[7] / nb;
      scal[SC_SUMS + 8] = sums[8] / nb;
      scal[SC_SUMS + 9] = sums[9] / nb;
      scal[SC_SUMS + 10] = sums[10] / nb;
      scal[SC_SUMS + 11] = sums[11] / nb;
    }
  }
}

// Analytic potentials (r = A |x - centre|, see QFD_POT_*).
__global__ void k_potential(double* __restrict__ V, int64_t n, double a, int kind, double c0, double c1,
                            int offgrid) {
  const int64_t n3 = n * n * n;
  const double cen = offgrid ? 0.5 * (double)(n - 1) : (double)(n / 2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double dz = (double)(i % n) - cen, dy = (double)((i / n) % n) - cen, dx = (double)(i / (n * n)) - cen;
    const double r = a * sqrt(dx * dx + dy * dy + dz * dz);
    double v = 0.0;
    if (kind == QFD_POT_HO) {
      v = 0.5 * c0 * r * r;
    } else if (kind == QFD_POT_CORNELL) {
      const double rc = fmax(r, 0.5 * a);
      v = -c0 / rc + c1 * rc;
    } else if (kind == QFD_POT_COULOMB) {
      v = -1.0 / fmax(r, 0.5 * a);
    } else if (kind == QFD_POT_SOFTCOUL) {
      v = -1.0 / sqrt(r * r + c0);
    }
    V[i] = v;
  }
}

// Update coefficients of Sec. 2.2 from V, per arithmetic: FP64 {A, B dtau}
// (complex128 pass A reads them precomputed); for H_K(0) plans also FP32 and
// double-float {B dtau, 1 - A} with 1 - A = dtau V B formed in FP64 (the FFT
// passes of those arithmetics derive them from V instead); V split into
// double-float pairs (the energy sums of the FP32-pipe arithmetics and the
// double-float pass A read it) and rounded to FP32 (the complex64 pass A).
// fdtd_c > 0 (H_K(0) plans, c = 1 / (2 M A^2)): the coefficients take the
// stencil's diagonal in, so that the update applied to the neighbour sum S
// gives A psi - B dtau c (6 psi - S) = (A - 6 c B dtau) psi + c B dtau S.
__global__ void k_coef(const double* __restrict__ V, int64_t n3, double dtau, double fdtd_c,
                       double2* __restrict__ c64, dfc* __restrict__ cdf, float2* __restrict__ c32,
                       df* __restrict__ vdf, float* __restrict__ v32, int* __restrict__ bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = V[i];
    const double h = 0.5 * dtau * v;
    const double den = 1.0 + h;
    if (!(den > 0.0) || !isfinite(v)) atomicOr(bad, 1);
    const double A = (1.0 - h) / den, B = 1.0 / den;
    double a64 = A, g1 = B * dtau, g2 = dtau * v * B;
    if (fdtd_c > 0.0) {
      a64 = (1.0 - h - 6.0 * fdtd_c * dtau) / den;  // A - 6 c B dtau
      g2 = dtau * (v + 6.0 * fdtd_c) * B;            // (1 - A) + 6 c B dtau
      g1 = -fdtd_c * g1;                             // -c B dtau
    }
    if (c64) c64[i] = double2{a64, g1};
    if (cdf) cdf[i] = dfc{dsplit(g1), dsplit(g2)};
    if (c32) c32[i] = float2{(float)g1, (float)g2};
    if (vdf) vdf[i] = dsplit(v);
    if (v32) v32[i] = (float)v;
  }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <class A>
__global__ void k_fill_uniform(typename A::C* __restrict__ psi, int64_t n3, uint64_t seed) {
  const uint64_t base = seed * 0x9E3779B97F4A7C15ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z0 = splitmix64(base ^ (uint64_t)(2 * i)), z1 = splitmix64(base ^ (uint64_t)(2 * i + 1));
    const double u0 = (double)(z0 >> 11) * 0x1.0p-53, u1 = (double)(z1 >> 11) * 0x1.0p-53;
    psi[i] = A::from_d2(double2{2.0 * u0 - 1.0, 2.0 * u1 - 1.0});
  }
}

// Site index <-> (x, y, z) of an n^3 lattice ([x][y][z], z fastest): shifts
// and masks when n = 2^lg (lg >= 0), divisions otherwise (n = 96, 192).
struct Lat {
  int64_t n;
  int lg;
};
__device__ __forceinline__ void lat_xyz(Lat L, int64_t i, int64_t& x, int64_t& y, int64_t& z) {
  if (L.lg >= 0) {
    z = i & (L.n - 1);
    y = (i >> L.lg) & (L.n - 1);
    x = i >> (2 * L.lg);
  } else {
    z = i % L.n;
    const int64_t q = i / L.n;
    y = q % L.n;
    x = q / L.n;
  }
}
__device__ __forceinline__ int64_t lat_idx(Lat L, int64_t x, int64_t y, int64_t z) { return (x * L.n + y) * L.n + z; }
__device__ __forceinline__ int64_t lat_wrap(Lat L, int64_t c) {
  return L.lg >= 0 ? (c & (L.n - 1)) : ((c % L.n) + L.n) % L.n;
}

// Observables of Sec. 2.3 / 2.4 / 5.1 in lattice units (d = x - centre per
// axis): partial sums of |psi|^2 (full and effective volume), rho |psi|^2 over
// the effective volume (|d_l| <= half on every axis), rho^2 |psi|^2, d |psi|^2,
// and |P+- psi|^2 and |P-_{e_k} psi|^2 (k = 1, 2, 3) over the effective volume,
// all in FP64.  P-_{e_k} of Eq. (parity_axis), normalised as a projector:
// (1/4) [psi(x) + psi(F_other x) - psi(F_k x) - psi(-x)], F_k the reflection of
// axis k and F_other that of the two other axes.
template <class A>
__global__ void __launch_bounds__(256)
k_observables(const typename A::C* __restrict__ psi, Lat L, int offgrid, double half, double* __restrict__ part) {
  const int64_t n = L.n, n3 = n * n * n;
  const double cen = offgrid ? 0.5 * (double)(n - 1) : (double)(n / 2);
  double acc[NOBS];
#pragma unroll
  for (int q = 0; q < NOBS; ++q) acc[q] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t x, y, z;
    lat_xyz(L, i, x, y, z);
    const int64_t rx = offgrid ? n - 1 - x : lat_wrap(L, n - x), ry = offgrid ? n - 1 - y : lat_wrap(L, n - y),
                  rz = offgrid ? n - 1 - z : lat_wrap(L, n - z);
    const double2 p = A::to_d2(psi[i]), r = A::to_d2(psi[lat_idx(L, rx, ry, rz)]);
    const double dx = (double)x - cen, dy = (double)y - cen, dz = (double)z - cen;
    const double rho2 = dx * dx + dy * dy + dz * dz;
    const double a2 = p.x * p.x + p.y * p.y;
    acc[0] += a2;
    acc[3] += rho2 * a2;
    acc[4] += dx * a2;
    acc[5] += dy * a2;
    acc[6] += dz * a2;
    if (fabs(dx) <= half && fabs(dy) <= half && fabs(dz) <= half) {
      acc[1] += a2;
      acc[2] += sqrt(rho2) * a2;
      const double sx = 0.5 * (p.x + r.x), sy = 0.5 * (p.y + r.y), mx = 0.5 * (p.x - r.x), my = 0.5 * (p.y - r.y);
      acc[7] += sx * sx + sy * sy;
      acc[8] += mx * mx + my * my;
      auto at = [&](int64_t X, int64_t Y, int64_t Z) { return A::to_d2(psi[lat_idx(L, X, Y, Z)]); };
      const double2 f1 = at(rx, y, z), f2 = at(x, ry, z), f3 = at(x, y, rz);        // one axis reflected
      const double2 g1 = at(x, ry, rz), g2 = at(rx, y, rz), g3 = at(rx, ry, z);     // the two others
      const double2 fk[3] = {f1, f2, f3}, gk[3] = {g1, g2, g3};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double ax = 0.25 * (p.x + gk[k].x - fk[k].x - r.x), ay = 0.25 * (p.y + gk[k].y - fk[k].y - r.y);
        acc[9 + k] += ax * ax + ay * ay;
      }
    }
  }
  block_reduce_store<NOBS>(acc, part);
}

template <class AI, class AO>
__global__ void k_convert(const typename AI::C* __restrict__ in, typename AO::C* __restrict__ out, int64_t n3) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = AO::from_d2(AI::to_d2(in[i]));
}

// ------------------------------------------------ finite-difference H_K(0)
// H_K(0) psi at site idx of the n^3 lattice with psi = 0 outside it
// (Eq. HK0 with Dirichlet boundaries, normalised as its momentum-space form,
// Eq. HK0_momentum_space_1): c (6 psi - the sum of the six neighbours) with
// c = 1 / (2 M A^2).  `self` receives psi at idx.
template <class A>
__device__ __forceinline__ typename A::C fdtd_sum(const typename A::C* __restrict__ psi, int64_t idx, Lat L,
                                                  typename A::C& self) {
  using C = typename A::C;
  const int64_t n = L.n, n2 = n * n;
  int64_t x, y, z;
  lat_xyz(L, idx, x, y, z);
  const C zero{};
  self = psi[idx];
  C s = x > 0 ? psi[idx - n2] : zero;
  s = cadd(s, x + 1 < n ? psi[idx + n2] : zero);
  s = cadd(s, y > 0 ? psi[idx - n] : zero);
  s = cadd(s, y + 1 < n ? psi[idx + n] : zero);
  s = cadd(s, z > 0 ? psi[idx - 1] : zero);
  s = cadd(s, z + 1 < n ? psi[idx + 1] : zero);
  return s;
}
template <class A>
__device__ __forceinline__ typename A::C fdtd_hk(const typename A::C* __restrict__ psi, int64_t idx, Lat L,
                                                 typename A::S c, typename A::C& self) {
  const typename A::C s = fdtd_sum<A>(psi, idx, L, self);
  return cscale(csub(cscale(self, A::scalar(6.0)), s), c);
}

// One imaginary-time step of Eq. (iter_proced) with H_K(0): out = A psi -
// B dtau H_K(0) psi (times the pending normalisation factor), partial sums per
// STATS.  The coefficients of H_K(0) plans hold the stencil's diagonal (see
// k_coef), so the update takes the neighbour sum.  psi and out are different
// lattices (the stencil reads neighbours).
template <class A, int STATS>
__global__ void __launch_bounds__(256)
k_fdtd_update(const typename A::C* __restrict__ psi, typename A::C* __restrict__ out,
              const typename A::K* __restrict__ coef, const typename A::VT* __restrict__ V,
              const double* __restrict__ scale, const float* __restrict__ scale_f, Lat L, double* __restrict__ part) {
  using C = typename A::C;
  const int64_t n3 = L.n * L.n * L.n;
  const bool scaled = scale != nullptr;
  typename A::S s{};
  if (scaled) s = A::load_scale(scale, scale_f);
  typename A::Acc nacc;
  typename A::Full facc;
  // sites per thread unrolled in the stencil loop (measured at 512^3: four
  // for the 16-byte arithmetics, one for complex64)
  constexpr int U = A::id == 1 ? 1 : 4;
#pragma unroll U
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += (int64_t)gridDim.x * blockDim.x) {
    C self;
    const C sum = fdtd_sum<A>(psi, idx, L, self);
    C nw = A::update(self, sum, coef[idx]);
    if (scaled) nw = cscale(nw, s);
    out[idx] = nw;
    if constexpr (STATS == STATS_NORM) nacc.add_norm(nw);
    if constexpr (STATS == STATS_FULL) facc.add(nw, V[idx]);
  }
  if constexpr (STATS == STATS_NORM) norm_reduce_store<A>(nacc, part);
  if constexpr (STATS == STATS_FULL) full_store<A>(facc, part);
}

// Per-CTA partials of <psi|H_K(0)|psi> (FP64 accumulation).
template <class A>
__global__ void __launch_bounds__(256)
k_fdtd_energy(const typename A::C* __restrict__ psi, Lat L, typename A::S c, double* __restrict__ part) {
  using C = typename A::C;
  const int64_t n3 = L.n * L.n * L.n;
  double e = 0.0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += (int64_t)gridDim.x * blockDim.x) {
    C self;
    const C hk = fdtd_hk<A>(psi, idx, L, c, self);
    const double2 u = A::to_d2(self), h = A::to_d2(hk);
    e += u.x * h.x + u.y * h.y;
  }
  double q[1] = {e};
  block_reduce_store<1>(q, part);
}

// ------------------------------------------------- Gaussian random fields
// White noise: per site the two counter-mode uniforms of k_fill_uniform
// (u in [0, 1)) through the Box-Muller transform, sqrt(-2 ln(1 - u0)) cos(2 pi u1).
__global__ void k_grf_noise(double* __restrict__ f, int64_t n3, uint64_t seed) {
  const uint64_t base = seed * 0x9E3779B97F4A7C15ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z0 = splitmix64(base ^ (uint64_t)(2 * i)), z1 = splitmix64(base ^ (uint64_t)(2 * i + 1));
    const double u0 = (double)(z0 >> 11) * 0x1.0p-53, u1 = (double)(z1 >> 11) * 0x1.0p-53;
    f[i] = sqrt(-2.0 * log(1.0 - u0)) * cospi(2.0 * u1);
  }
}

// Taps exp(-j^2 / (2 c^2)), j = -r..r, of a real-space Gaussian.
constexpr int GRF_MAX_R = 200;
struct GrfTaps {
  double g[2 * GRF_MAX_R + 1];
  int r;
};

// Periodic convolution along one axis (0: x, 1: y, 2: z): taps wrapping past
// the lattice add up, which is the periodic sum of the Gaussian.
__global__ void k_grf_conv(const double* __restrict__ in, double* __restrict__ out, Lat L, int axis, GrfTaps taps) {
  const int64_t n = L.n, n3 = n * n * n;
  const int64_t stride = axis == 0 ? n * n : axis == 1 ? n : 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t xyz[3];
    lat_xyz(L, i, xyz[0], xyz[1], xyz[2]);
    const int64_t c = xyz[axis], base = i - c * stride;
    double acc = 0.0;
    for (int j = -taps.r; j <= taps.r; ++j) acc += taps.g[j + taps.r] * in[base + lat_wrap(L, c + j) * stride];
    out[i] = acc;
  }
}

// Per-CTA partial sums of f and f^2.
__global__ void __launch_bounds__(256) k_grf_moments(const double* __restrict__ f, int64_t n3, double* __restrict__ part) {
  double q[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    q[0] += f[i];
    q[1] += f[i] * f[i];
  }
  block_reduce_store<2>(q, part);
}

// V += amplitude (f - mean) / std, with the sums of f and f^2 in sums[0..1].
__global__ void k_grf_add(double* __restrict__ V, const double* __restrict__ f, int64_t n3,
                          const double* __restrict__ sums, double amplitude) {
  const double mean = sums[0] / (double)n3;
  const double var = sums[1] / (double)n3 - mean * mean;
  const double s = amplitude / sqrt(var);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    V[i] += s * (f[i] - mean);
}

}  // namespace qfd

// ================================================================== plan
struct qfd_plan_s {
  qfd_params p{};
  int64_t n3 = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  // device memory: nstates + 1 lattices per representation; sp16/sp32 map a
  // state to its lattice and the extra one receives each projected state
  void* psi16 = nullptr;    // state lattices, 16 bytes per site (F64 or DF)
  float2* psi32 = nullptr;  // state lattices, complex64
  std::vector<char*> sp16, sp32;
  char* spare16 = nullptr;
  char* spare32 = nullptr;
  double2* W = nullptr;     // work lattice (16 bytes per site; complex64 uses half)
  void* coef16 = nullptr;   // F64 {A, B dtau}, or (H_K(0) plans) DF {B dtau, 1 - A}
  float2* coef32 = nullptr;  // (H_K(0) plans) complex64 {B dtau, 1 - A}
  float* V32 = nullptr;      // V in FP32 (complex64 pass A of the FFT kinetic terms)
  double* V = nullptr;
  df* Vdf = nullptr;        // V as double-float pairs (plans with an FP32-pipe arithmetic)
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  dfc* twdf = nullptr;
  double* ktab64 = nullptr;
  float* ktab32 = nullptr;
  df* ktabdf = nullptr;
  double* partA = nullptr;
  double* partC = nullptr;
  double* partG = nullptr;
  int nA = 0, nC = 0;
  double* scal = nullptr;
  float* scalf = nullptr;  // the normalisation factor in FP32 and double-float form
  int* flag = nullptr;
  int* errflag = nullptr;   // set by a kernel whose bounded wait ran out (the TMA-staged pass A)
  double* hscal = nullptr;  // pinned host copy of the scalars (+ the error flag)
  // the TMA-staged pass A (complex64, n = 256..1024): device array of tensor
  // maps, [0] W as complex64, [1] V in FP32, [2 + i] complex64 state buffer i;
  // null when the variant is not available for the plan
  CUtensorMap* tmaps = nullptr;
  int tma_test = 0;  // 1: the TMA pass A arms its barriers without issuing copies
  // host-side state
  KinParams kin{};
  int tune_vy[3] = {0, 0, 0};     // launch shapes per policy id (autotuner; see LaunchArgs)
  int tune_vz[3] = {-1, -1, -1};
  int tune_vx[3] = {0, 0, 0};
  UpdParams up{};  // dtau in the representations of the V-derived coefficients
  int lg = -1;          // n = 2^lg, or -1 (n = 96, 192)
  double fdtd_c = 0.0;  // 1 / (2 M A^2) of H_K(0)
  int arith16 = 0;  // policy id of the 16-byte representation: 0 F64, 2 DF
  std::vector<int64_t> t;
  std::vector<int> parity;
  std::vector<int64_t> steps16, steps32;
  std::vector<double> ebulk;
  std::vector<double> edecay;  // decay-rate energy at the last check
  // energy at every check of the last solve, per state: (phase-local step, E)
  std::vector<std::vector<std::pair<int64_t, double>>> hist;
  // snapshot-overlap excited states: while snap_every > 0, state slots
  // 1..nsnap hold the latest snapshots of state 0, newest first, taken at the
  // cadence every snap_every steps; snap_t[i] is the step of slot 1 + i
  int64_t snap_every = 0;
  int nsnap = 0;
  std::vector<int64_t> snap_t;
  int w_state = -1, w_stage = ST_NONE, w_phase = -1;
  bool pending = false;
  int phase = 0;  // policy id of the current arithmetic
  bool has_pot = false;
  // instrumentation
  bool timing = false;
  int64_t launches = 0;
  std::vector<cudaEvent_t> ev[PASS_COUNT];
  size_t evused[PASS_COUNT] = {};
};

namespace {

qfd_status fail(qfd_plan_t pl, qfd_status s, const std::string& msg) {
  if (pl) pl->err = msg;
  return s;
}

#define QFD_CK(call)                                                                             \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(pl, QFD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Launch f() (which returns cudaError_t), bracketed by timing events when enabled.
template <class F>
cudaError_t run(qfd_plan_t pl, int kind, F&& f) {
  ++pl->launches;
  if (!pl->timing) return f();
  size_t& u = pl->evused[kind];
  auto& v = pl->ev[kind];
  if (u + 2 > v.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return cudaErrorMemoryAllocation;
    if (cudaEventCreate(&b) != cudaSuccess) return cudaErrorMemoryAllocation;
    v.push_back(a);
    v.push_back(b);
  }
  cudaEventRecord(v[u], pl->st);
  cudaError_t e = f();
  cudaEventRecord(v[u + 1], pl->st);
  u += 2;
  return e;
}

#define QFD_RUN(kind, expr)                                                                      \
  do {                                                                                           \
    cudaError_t e_ = run(pl, kind, [&]() -> cudaError_t { return (expr); });                     \
    if (e_ != cudaSuccess) return fail(pl, QFD_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
  } while (0)

int grid_for(int64_t n3) {
  int64_t g = (n3 + 255) / 256;
  return (int)(g < 8 * 152 ? (g < 1 ? 1 : g) : 8 * 152);
}

// exp(-2 pi i e / n) with the angle reduced to the first octant in integers,
// so quadrant points are exact and the table is symmetric.
void unit_root(int64_t e, int64_t n, double* c, double* s) {
  e %= n;
  const int64_t q = (4 * e) / n;
  const int64_t rem = 4 * e - q * n;  // angle = pi/2 * (q + rem/n)
  double cp, sp;
  if (2 * rem <= n) {
    const double phi = (M_PI / 2) * (double)rem / (double)n;
    cp = std::cos(phi);
    sp = std::sin(phi);
  } else {
    const double phi = (M_PI / 2) * (double)(n - rem) / (double)n;
    cp = std::sin(phi);
    sp = std::cos(phi);
  }
  double ct, st;
  switch (q) {
    case 0: ct = cp; st = sp; break;
    case 1: ct = -sp; st = cp; break;
    case 2: ct = -cp; st = -sp; break;
    default: ct = sp; st = -cp; break;
  }
  *c = ct;
  *s = -st;
}

df host_split(double x) {
  const float h = (float)x;
  return df{h, (float)(x - (double)h)};
}

// ---------------------------------------------------------- policy access
template <class A> typename A::C* psi_of(qfd_plan_t pl, int s) {
  return reinterpret_cast<typename A::C*>(A::id == 1 ? pl->sp32[s] : pl->sp16[s]);
}
template <class A> typename A::C* spare_of(qfd_plan_t pl) {
  return reinterpret_cast<typename A::C*>(A::id == 1 ? pl->spare32 : pl->spare16);
}
// The projected state now lives in the spare lattice: swap the two roles.
template <class A> void swap_spare(qfd_plan_t pl, int s) {
  if (A::id == 1) std::swap(pl->sp32[s], pl->spare32);
  else std::swap(pl->sp16[s], pl->spare16);
}
template <class A> typename A::S host_scalar(double x) {
  if constexpr (A::id == 0) return x;
  else if constexpr (A::id == 1) return (float)x;
  else return host_split(x);
}
// V as the policy's energy sums read it (FP64, or the double-float copy)
template <class A> const typename A::VT* v_of(qfd_plan_t pl) {
  if constexpr (A::id == 0) return pl->V;
  else return pl->Vdf;
}
// the H_K(0) update's coefficient array
template <class A> const void* coef_of(qfd_plan_t pl) { return A::id == 1 ? (const void*)pl->coef32 : pl->coef16; }
// pass A's per-site input for the FFT kinetic terms: {A, B dtau} (F64), V in
// FP32 (F32) or as double-float pairs (DF)
template <class A> const void* uin_of(qfd_plan_t pl) {
  if constexpr (A::id == 0) return pl->coef16;
  else if constexpr (A::id == 1) return pl->V32;
  else return pl->Vdf;
}
template <class A> const void* tw_of(qfd_plan_t pl) {
  return A::id == 0 ? (const void*)pl->tw64 : A::id == 1 ? (const void*)pl->tw32 : (const void*)pl->twdf;
}
template <class A> const void* ktab_of(qfd_plan_t pl) {
  return A::id == 0 ? (const void*)pl->ktab64 : A::id == 1 ? (const void*)pl->ktab32 : (const void*)pl->ktabdf;
}

// Runs f(policy) for the policy with id `phase`.
template <class F>
qfd_status with_policy(int phase, F&& f) {
  if (phase == 0) return f(F64{});
  if (phase == 1) return f(F32{});
  return f(DF{});
}

template <class A>
LaunchArgs base_args(qfd_plan_t pl) {
  LaunchArgs a;
  a.n = pl->p.n;
  a.W = pl->W;
  a.tw = tw_of<A>(pl);
  a.ktab = ktab_of<A>(pl);
  a.kin = &pl->kin;
  a.coef = uin_of<A>(pl);
  a.up = &pl->up;
  a.V = v_of<A>(pl);
  a.stream = pl->st;
  a.vy = pl->tune_vy[A::id];
  a.vz = pl->tune_vz[A::id];
  a.vx = pl->tune_vx[A::id] == 2 && !(A::id == 1 && pl->tmaps) ? 0 : pl->tune_vx[A::id];
  a.err = pl->errflag;
  a.tma_test = pl->tma_test;
  if (A::id == 1 && pl->tmaps) {
    a.tmap[0] = pl->tmaps;
    a.tmap[2] = pl->tmaps + 1;
  }
  return a;
}

// Waits for the plan's stream; an error of any kernel queued on it surfaces
// here as QFD_ERR_CUDA.
qfd_status sync_checked(qfd_plan_t pl) {
  int e = 0;
  if (pl->tmaps) QFD_CK(cudaMemcpyAsync(&e, pl->errflag, sizeof(int), cudaMemcpyDeviceToHost, pl->st));
  QFD_CK(cudaStreamSynchronize(pl->st));
  if (e) {
    cudaMemsetAsync(pl->errflag, 0, sizeof(int), pl->st);
    return fail(pl, QFD_ERR_TIMEOUT, "the TMA-staged pass A gave up waiting for its tile copies");
  }
  return QFD_OK;
}

// The tensor map (device address) of the complex64 state lattice `p`, for the
// TMA-staged pass A, or null.
const void* psi_tmap(qfd_plan_t pl, const void* p) {
  if (!pl->tmaps || !pl->psi32) return nullptr;
  const size_t bytes = (size_t)pl->n3 * sizeof(float2);
  const size_t off = (size_t)((const char*)p - (const char*)pl->psi32);
  if (off % bytes != 0 || off / bytes > (size_t)pl->p.nstates) return nullptr;
  return pl->tmaps + 2 + off / bytes;
}

qfd_status finalize(qfd_plan_t pl, const double* part, int nq, int count, int op) {
  QFD_RUN(PASS_FINALIZE,
          (k_finalize_op<<<1, FIN_THREADS, 0, pl->st>>>(part, nq, count, pl->scal, pl->scalf, op),
           cudaGetLastError()));
  return QFD_OK;
}

// forward DFT_x of src (times the pending factor if use_scale) into W; psi_out
// optionally receives the scaled input.  Partials per `stats` -> partA.
template <class A>
qfd_status pass_forward_x(qfd_plan_t pl, const void* src, void* psi_out, bool use_scale, int stats) {
  LaunchArgs a = base_args<A>(pl);
  a.src = src;
  a.psi_out = psi_out;
  a.scale = use_scale ? pl->scal + SC_SCALE : nullptr;
  a.scale_f = pl->scalf;
  a.part = pl->partA;
  a.stats = stats;
  int nb = 0;
  QFD_RUN(PASS_FWD_X, launch_forward_x<A>(a, &nb));
  pl->nA = nb;
  return QFD_OK;
}

template <class A>
qfd_status advance_to_d(qfd_plan_t pl, int parseval_at_c) {
  LaunchArgs a = base_args<A>(pl);
  if (pl->w_stage == ST_X) {
    QFD_RUN(PASS_FWD_Y, launch_fft_y<A>(a, -1));
    pl->w_stage = ST_XY;
  }
  if (pl->w_stage == ST_XY) {
    a.part = pl->partC;
    a.stats = parseval_at_c;
    int nb = 0;
    QFD_RUN(PASS_ZKIN, launch_zpass<A>(a, &nb));
    pl->nC = nb;
    pl->w_stage = ST_C;
    if (parseval_at_c) return QFD_OK;  // caller reads the Parseval partials before pass D
  }
  if (pl->w_stage == ST_C) {
    QFD_RUN(PASS_INV_Y, launch_fft_y<A>(a, +1));
    pl->w_stage = ST_D;
  }
  return QFD_OK;
}

template <class A>
void mark_w(qfd_plan_t pl, int s, int stage) {
  pl->w_state = s;
  pl->w_phase = A::id;
  pl->w_stage = stage;
}

template <class A>
qfd_status ensure_w(qfd_plan_t pl, int s) {
  if (pl->w_state != s || pl->w_phase != A::id || pl->w_stage == ST_NONE) {
    pl->pending = false;
    qfd_status r = pass_forward_x<A>(pl, psi_of<A>(pl, s), nullptr, false, STATS_NONE);
    if (r != QFD_OK) return r;
    mark_w<A>(pl, s, ST_X);
  }
  return QFD_OK;
}

bool projects(qfd_plan_t pl, int s) { return s > 0 || pl->parity[s] != 0; }

// Parity projection, Gram-Schmidt against states 0..s-1, normalisation.
// The projection (when there is one) runs fused with the forward x transform
// into the spare lattice; in every case the normalisation factor is only
// computed here and applied by the next pass A (the update is linear).
template <class A>
qfd_status cadence(qfd_plan_t pl, int s, int check) {
  qfd_status r;
  if (projects(pl, s)) {
    if (pl->pending) return fail(pl, QFD_ERR_STATE, "internal: pending scale at projection");
    LaunchArgs a = base_args<A>(pl);
    a.src = psi_of<A>(pl, s);
    a.dst = spare_of<A>(pl);
    a.k = s;
    for (int j = 0; j < s; ++j) a.lower[j] = psi_of<A>(pl, j);
    a.parity = pl->parity[s];
    a.offgrid = pl->p.centre == QFD_CENTRE_OFFGRID;
    a.sums = pl->scal + SC_SUMS;
    if (s > 0) {
      a.part = pl->partG;
      QFD_RUN(PASS_GS_DOTS, launch_gs_dots<A>(a, GS_BLOCKS));
      if ((r = finalize(pl, pl->partG, 2 * s, GS_BLOCKS, OP_SUMS)) != QFD_OK) return r;
    }
    a.part = pl->partA;
    a.stats = check ? STATS_FULL : STATS_NORM;
    int nb = 0;
    QFD_RUN(PASS_GS_APPLY, launch_project_x<A>(a, &nb));
    pl->nA = nb;
    swap_spare<A>(pl, s);
    mark_w<A>(pl, s, ST_X);
  }
  if ((r = finalize(pl, pl->partA, 2, pl->nA, OP_NORM)) != QFD_OK) return r;
  pl->pending = true;
  return QFD_OK;
}

// Rotates the snapshot slots (the oldest buffer becomes the newest slot) and
// copies the normalised state 0 into it.
template <class A>
qfd_status take_snapshot(qfd_plan_t pl) {
  auto& sp = A::id == 1 ? pl->sp32 : pl->sp16;
  char* oldest = sp[pl->nsnap];
  for (int i = pl->nsnap; i > 1; --i) {
    sp[i] = sp[i - 1];
    pl->snap_t[i - 1] = pl->snap_t[i - 2];
  }
  sp[1] = oldest;
  pl->snap_t[0] = pl->t[0];
  QFD_RUN(PASS_OTHER, (k_scale_copy<A><<<grid_for(pl->n3), 256, 0, pl->st>>>(
                           psi_of<A>(pl, 1), psi_of<A>(pl, 0), pl->n3, pl->pending ? pl->scal + SC_SCALE : nullptr),
                       cudaGetLastError()));
  return QFD_OK;
}

// One H_K(0) step: the stencil update from the state into the spare lattice,
// which then becomes the state (W is not used).
template <class A>
qfd_status fdtd_update(qfd_plan_t pl, int s, int stats) {
  const double* scale = pl->pending ? pl->scal + SC_SCALE : nullptr;
  auto go = [&](auto kern) -> cudaError_t {
    kern<<<GS_BLOCKS, 256, 0, pl->st>>>(psi_of<A>(pl, s), spare_of<A>(pl),
                                        static_cast<const typename A::K*>(coef_of<A>(pl)), v_of<A>(pl), scale, pl->scalf,
                                        Lat{pl->p.n, pl->lg}, pl->partA);
    return cudaGetLastError();
  };
  auto launch = [&]() -> cudaError_t {
    if (stats == STATS_FULL) return go(k_fdtd_update<A, STATS_FULL>);
    if (stats == STATS_NORM) return go(k_fdtd_update<A, STATS_NORM>);
    return go(k_fdtd_update<A, STATS_NONE>);
  };
  QFD_RUN(PASS_UPDATE_X, launch());
  swap_spare<A>(pl, s);
  pl->nA = GS_BLOCKS;
  pl->w_stage = ST_NONE;
  return QFD_OK;
}

// <psi|H_K(0)|psi> of state s into the energy partials (the Parseval sum of
// the FFT terms).
template <class A>
qfd_status fdtd_energy_partials(qfd_plan_t pl, int s) {
  const typename A::S c = host_scalar<A>(pl->fdtd_c);
  QFD_RUN(PASS_ZKIN, (k_fdtd_energy<A><<<GS_BLOCKS, 256, 0, pl->st>>>(psi_of<A>(pl, s), Lat{pl->p.n, pl->lg}, c, pl->partC),
                      cudaGetLastError()));
  pl->nC = GS_BLOCKS;
  return QFD_OK;
}

template <class A>
qfd_status step_once(qfd_plan_t pl, int s, int check) {
  qfd_status r;
  const bool fdtd = pl->p.kinetic == 0;
  if (!fdtd) {
    if ((r = ensure_w<A>(pl, s)) != QFD_OK) return r;
    if ((r = advance_to_d<A>(pl, 0)) != QFD_OK) return r;
  }
  const bool ortho_next = (pl->t[s] + 1) % pl->p.ortho_every == 0;
  const bool proj = projects(pl, s);
  int stats = STATS_NONE;
  if (ortho_next) stats = proj ? STATS_NONE : (check ? STATS_FULL : STATS_NORM);
  else if (check) stats = STATS_FULL;
  if (fdtd) {
    if ((r = fdtd_update<A>(pl, s, stats)) != QFD_OK) return r;
  } else {
    LaunchArgs a = base_args<A>(pl);
    a.psi = psi_of<A>(pl, s);
    a.tmap[1] = psi_tmap(pl, a.psi);
    a.scale = pl->pending ? pl->scal + SC_SCALE : nullptr;
    a.scale_f = pl->scalf;
    a.part = pl->partA;
    a.stats = stats;
    int nb = 0;
    QFD_RUN(PASS_UPDATE_X, launch_update_x<A>(a, &nb));
    pl->nA = nb;
    pl->w_stage = ST_X;
  }
  pl->pending = false;
  pl->t[s] += 1;
  if (pl->t[s] % pl->p.ortho_every == 0) {
    if ((r = cadence<A>(pl, s, check)) != QFD_OK) return r;
    if (pl->snap_every > 0 && s == 0 && pl->t[s] % pl->snap_every == 0 && (r = take_snapshot<A>(pl)) != QFD_OK)
      return r;
  } else if (check) {
    if ((r = finalize(pl, pl->partA, 2, pl->nA, OP_N2PV)) != QFD_OK) return r;
  }
  return QFD_OK;
}

// Applies a pending normalisation factor to the stored state (W is dropped).
template <class A>
qfd_status materialize(qfd_plan_t pl, int s) {
  if (pl->pending) {
    QFD_RUN(PASS_OTHER, (k_scale<A><<<grid_for(pl->n3), 256, 0, pl->st>>>(psi_of<A>(pl, s), pl->n3, pl->scal + SC_SCALE, 0),
                         cudaGetLastError()));
    pl->pending = false;
    pl->w_stage = ST_NONE;
  }
  return QFD_OK;
}

// Energy of the state whose partials (N2, PV) were just finalised and whose
// x-transform sits in W: passes B and C (with the Parseval sum), then E.
template <class A>
qfd_status energy_tail(qfd_plan_t pl, double* E, double* n2) {
  qfd_status r;
  if (pl->w_stage != ST_X) return fail(pl, QFD_ERR_STATE, "internal: energy needs W after the x pass");
  if ((r = advance_to_d<A>(pl, 1)) != QFD_OK) return r;
  if ((r = finalize(pl, pl->partC, 1, pl->nC, OP_ENERGY)) != QFD_OK) return r;
  double h[SC_COUNT];
  QFD_CK(cudaMemcpyAsync(h, pl->scal, sizeof(h), cudaMemcpyDeviceToHost, pl->st));
  if ((r = sync_checked(pl)) != QFD_OK) return r;
  if (E) *E = h[SC_E];
  if (n2) *n2 = h[SC_N2];
  return QFD_OK;
}

template <class A>
qfd_status energy_full(qfd_plan_t pl, int s, double* E, double* n2) {
  qfd_status r;
  if ((r = materialize<A>(pl, s)) != QFD_OK) return r;
  if ((r = pass_forward_x<A>(pl, psi_of<A>(pl, s), nullptr, false, STATS_FULL)) != QFD_OK) return r;
  mark_w<A>(pl, s, ST_X);
  if ((r = finalize(pl, pl->partA, 2, pl->nA, OP_N2PV)) != QFD_OK) return r;
  if (pl->p.kinetic != 0) return energy_tail<A>(pl, E, n2);
  // H_K(0): the kinetic expectation by the stencil instead of Parseval
  if ((r = fdtd_energy_partials<A>(pl, s)) != QFD_OK) return r;
  if ((r = finalize(pl, pl->partC, 1, pl->nC, OP_ENERGY)) != QFD_OK) return r;
  double h[SC_COUNT];
  QFD_CK(cudaMemcpyAsync(h, pl->scal, sizeof(h), cudaMemcpyDeviceToHost, pl->st));
  if ((r = sync_checked(pl)) != QFD_OK) return r;
  if (E) *E = h[SC_E];
  if (n2) *n2 = h[SC_N2];
  return QFD_OK;
}

// One state in one arithmetic is a phase: begin_phase (counter reset and the
// cadence at t = 0), then periods of check_every steps each ending with the
// energy, then finish_phase (normalise).  qfd_solve_states and the request
// server share these pieces, so a request gives the same numbers alone, in a
// server mix, or through qfd_solve_states.
template <class A>
qfd_status begin_phase(qfd_plan_t pl, int s) {
  qfd_status r;
  pl->t[s] = 0;
  pl->pending = false;
  pl->w_stage = ST_NONE;
  if (!projects(pl, s)) {
    if ((r = pass_forward_x<A>(pl, psi_of<A>(pl, s), nullptr, false, STATS_NORM)) != QFD_OK) return r;
    mark_w<A>(pl, s, ST_X);
  }
  return cadence<A>(pl, s, 0);
}

// check_every steps and the energy of their last state; the scalars (E at
// SC_E, N2 at SC_N2) are copied asynchronously into `host` (pinned, SC_COUNT
// doubles).  Nothing here synchronises, so a period can be captured into a
// CUDA graph.
template <class A>
qfd_status period_launch(qfd_plan_t pl, int s, double* host) {
  qfd_status r;
  const int ce = pl->p.check_every;
  for (int j = 0; j < ce; ++j)
    if ((r = step_once<A>(pl, s, j == ce - 1)) != QFD_OK) return r;
  if (pl->p.kinetic == 0) {
    if ((r = fdtd_energy_partials<A>(pl, s)) != QFD_OK) return r;
  } else {
    if (pl->w_stage != ST_X) return fail(pl, QFD_ERR_STATE, "internal: energy needs W after the x pass");
    if ((r = advance_to_d<A>(pl, 1)) != QFD_OK) return r;
  }
  if ((r = finalize(pl, pl->partC, 1, pl->nC, OP_ENERGY)) != QFD_OK) return r;
  QFD_CK(cudaMemcpyAsync(host, pl->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, pl->st));
  QFD_CK(cudaMemcpyAsync(host + SC_COUNT, pl->errflag, sizeof(int), cudaMemcpyDeviceToHost, pl->st));
  return QFD_OK;
}

template <class A>
qfd_status finish_phase(qfd_plan_t pl, int s) {
  // leave the state normalised (its last finalised N2 is of the stored values)
  QFD_RUN(PASS_OTHER, (k_scale<A><<<grid_for(pl->n3), 256, 0, pl->st>>>(psi_of<A>(pl, s), pl->n3, pl->scal + SC_N2, 1),
                       cudaGetLastError()));
  pl->pending = false;
  pl->w_stage = ST_NONE;
  return QFD_OK;
}

// The stop rule applied after every period (TOLERANCE of Sec. 5.1): done when
// |E - E_prev| <= tol |E| from the second check on; under QFD_STOP_TAIL a final
// phase also needs a change below 1e-3 tol |E|, or three changes of one sign
// whose ratio r has not fallen and whose geometric tail d r / (1 - r) is within
// tol |E| (the update is not symmetric: the energy can undershoot its limit and
// turn back, so neither a small change nor a single ratio suffices).  A complex64
// bulk phase also stops once its energy rises between checks after the third
// one (FP32 noise floor).  Returns QFD_ERR_DIVERGED for a non-finite energy or
// norm.
struct PhaseTracker {
  double e_prev = NAN;
  double d1 = 0.0, d2 = 0.0;  // the last two signed changes E_k - E_(k-1)
  int checks = 0;
};
qfd_status phase_check(qfd_plan_t pl, int s, const double* host, double tol, bool bulk, PhaseTracker& tr,
                       bool* done, double* e_out) {
  const double e = host[SC_E], n2 = host[SC_N2];
  int kerr = 0;
  std::memcpy(&kerr, host + SC_COUNT, sizeof(int));
  if (kerr) {
    cudaMemsetAsync(pl->errflag, 0, sizeof(int), pl->st);
    return fail(pl, QFD_ERR_TIMEOUT, "the TMA-staged pass A gave up waiting for its tile copies");
  }
  if (!std::isfinite(e) || !std::isfinite(n2) || !(n2 > 0))
    return fail(pl, QFD_ERR_DIVERGED, "energy or norm is not finite (time step or potential too large?)");
  pl->hist[s].push_back({pl->t[s], e});
  {  // decay-rate energy over the steps since the last normalisation
    const int64_t K = pl->p.ortho_every, k = pl->t[s] % K == 0 ? K : pl->t[s] % K;
    pl->edecay[s] = -std::expm1(std::log(n2) * (0.5 / (double)k)) / pl->p.dtau;
  }
  ++tr.checks;
  const double dk = tr.checks > 1 ? e - tr.e_prev : INFINITY;
  const double ae = std::fabs(e);
  bool stop = tol >= 0 && std::fabs(dk) <= tol * ae;
  if (stop && !bulk && pl->p.stop_rule == QFD_STOP_TAIL && std::fabs(dk) > 1e-3 * tol * ae) {
    // one sign over the last three changes, a ratio that has not fallen, and a
    // geometric tail within tolerance
    stop = false;
    if (tr.checks > 3 && dk * tr.d1 > 0 && tr.d1 * tr.d2 > 0) {
      const double r = dk / tr.d1, r_prev = tr.d1 / tr.d2;
      stop = r < 1.0 && r >= 0.9 * r_prev && std::fabs(dk) * r / (1.0 - r) <= tol * ae;
    }
  }
  *done = stop || (bulk && tr.checks > 3 && e > tr.e_prev);
  tr.d2 = tr.d1;
  tr.d1 = dk;
  tr.e_prev = e;
  *e_out = e;
  return QFD_OK;
}

template <class A>
qfd_status solve_phase(qfd_plan_t pl, int s, double tol, int64_t max_steps, double* E_out, int64_t* steps,
                       bool* converged, bool bulk = false) {
  qfd_status r;
  if ((r = begin_phase<A>(pl, s)) != QFD_OK) return r;
  PhaseTracker tr;
  double e = NAN;
  *converged = false;
  while (pl->t[s] < max_steps) {
    if ((r = period_launch<A>(pl, s, pl->hscal)) != QFD_OK) return r;
    QFD_CK(cudaStreamSynchronize(pl->st));
    if ((r = phase_check(pl, s, pl->hscal, tol, bulk, tr, converged, &e)) != QFD_OK) return r;
    if (*converged) break;
  }
  if ((r = finish_phase<A>(pl, s)) != QFD_OK) return r;
  *E_out = e;
  *steps = pl->t[s];
  return QFD_OK;
}

// Snapshot-overlap excited states (Sec. 2.2): one evolution of state 0 to the
// stop rule, snapshots every snap_every steps; the ground state is the final
// state, excited state k the k-th latest snapshot taken before the end, parity
// projected, Gram-Schmidt deflated against states 0..k-1 and normalised.
template <class A>
qfd_status snapshot_states(qfd_plan_t pl, int nout, int parity, int64_t snap_every, double* E_out,
                           int64_t* steps_out, bool* conv) {
  const int K = nout > 1 ? nout : 0;
  pl->nsnap = K;
  pl->snap_t.assign(K, -1);
  pl->snap_every = K ? snap_every : 0;
  pl->parity[0] = parity;
  pl->steps32[0] = pl->steps16[0] = 0;
  pl->ebulk[0] = NAN;
  pl->hist[0].clear();
  double e = NAN;
  int64_t steps = 0;
  qfd_status r = solve_phase<A>(pl, 0, pl->p.tol, pl->p.max_steps, &e, &steps, conv);
  pl->snap_every = 0;
  if (r != QFD_OK) return r;
  if (A::id == 1) pl->steps32[0] = steps;
  else pl->steps16[0] = steps;
  E_out[0] = e;
  if (steps_out) *steps_out = steps;
  // the sources, newest first: snapshots strictly before the end
  auto& sp = A::id == 1 ? pl->sp32 : pl->sp16;
  std::vector<char*> srcs, rest;
  for (int i = 0; i < K; ++i)
    ((pl->snap_t[i] >= 0 && pl->snap_t[i] < pl->t[0] && (int)srcs.size() < nout - 1) ? srcs : rest).push_back(sp[1 + i]);
  if ((int)srcs.size() < nout - 1)
    return fail(pl, QFD_ERR_STATE, "fewer snapshots than excited states: raise max_steps or lower snap_every");
  for (int i = 0; i < K; ++i) sp[1 + i] = i < (int)srcs.size() ? srcs[i] : rest[i - srcs.size()];
  for (int k = 1; k < nout; ++k) {
    pl->parity[k] = parity;
    pl->hist[k].clear();
    pl->steps32[k] = pl->steps16[k] = 0;
    double n2 = 0.0;
    if ((r = cadence<A>(pl, k, 0)) != QFD_OK) return r;
    if ((r = materialize<A>(pl, k)) != QFD_OK) return r;
    if ((r = energy_full<A>(pl, k, &E_out[k], &n2)) != QFD_OK) return r;
  }
  return QFD_OK;
}

// Median time (ms) of `reps` launches of f on the plan's stream after `warm`.
template <class F>
qfd_status time_launch(qfd_plan_t pl, F&& f, int warm, int reps, double* ms) {
  cudaEvent_t e0, e1;
  QFD_CK(cudaEventCreate(&e0));
  QFD_CK(cudaEventCreate(&e1));
  std::vector<double> t;
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < warm + reps && err == cudaSuccess; ++i) {
    cudaEventRecord(e0, pl->st);
    err = f();
    cudaEventRecord(e1, pl->st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float m = 0.f;
    if (err == cudaSuccess && i >= warm && cudaEventElapsedTime(&m, e0, e1) == cudaSuccess) t.push_back(m);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(pl, QFD_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(err));
  std::sort(t.begin(), t.end());
  *ms = t.empty() ? INFINITY : t[t.size() / 2];
  return QFD_OK;
}

// Whether lattice size n has the two-stage radix schedule in policy A.
template <class A> bool has_two_stage(int64_t n) {
  bool out = false;
  dispatch_n(n, [&](auto t) {
    out = Shape<A, decltype(t)::value>::HAS_R1;
    return cudaSuccess;
  });
  return out;
}

// Index of the smallest of the first k timings.
int argmin(const double* ms, int k) {
  int b = 0;
  for (int i = 1; i < k; ++i)
    if (ms[i] < ms[b]) b = i;
  return b;
}

// Times the y-pass shapes (default width, twice it, and - complex64 - the
// two-stage radix schedule), the z-pass shapes (one or two line groups, and
// the two-stage schedule) and both pass-A tile widths of policy A (pass A on
// the work lattice and the spare state lattice, which hold nothing yet to be
// kept) and keeps the fastest of each.  ms[0..2] y, ms[3..5] z, ms[6..8] x.
template <class A>
qfd_status autotune_policy(qfd_plan_t pl, double* ms) {
  qfd_status r;
  QFD_CK(cudaMemsetAsync(pl->W, 0, (size_t)pl->n3 * sizeof(double2), pl->st));
  QFD_CK(cudaMemsetAsync(spare_of<A>(pl), 0, (size_t)pl->n3 * sizeof(typename A::C), pl->st));
  const int nv = has_two_stage<A>(pl->p.n) ? 3 : 2;
  for (int v = 0; v < nv; ++v) {
    LaunchArgs a = base_args<A>(pl);
    a.vy = v;
    if ((r = time_launch(pl, [&]() { return launch_fft_y<A>(a, -1); }, 2, 5, &ms[v])) != QFD_OK) return r;
  }
  for (int v = 0; v < nv; ++v) {
    LaunchArgs a = base_args<A>(pl);
    a.vz = v;
    a.stats = 0;
    a.part = pl->partC;
    if ((r = time_launch(pl, [&]() { return launch_zpass<A>(a, nullptr); }, 2, 5, &ms[3 + v])) != QFD_OK) return r;
  }
  if (pl->p.kinetic != 0 && pl->has_pot) {
    const int nxv = A::id == 1 && pl->tmaps ? 3 : 2;  // 2: the TMA-staged pass A
    for (int v = 0; v < nxv; ++v) {
      LaunchArgs a = base_args<A>(pl);
      a.vx = v;
      a.psi = spare_of<A>(pl);
      a.tmap[1] = psi_tmap(pl, a.psi);
      a.part = pl->partA;
      a.stats = STATS_NONE;
      if ((r = time_launch(pl, [&]() { return launch_update_x<A>(a, nullptr); }, 2, 5, &ms[6 + v])) != QFD_OK)
        return r;
    }
    pl->tune_vx[A::id] = argmin(ms + 6, nxv);
  }
  pl->tune_vy[A::id] = argmin(ms, nv);
  pl->tune_vz[A::id] = argmin(ms + 3, nv);
  return QFD_OK;
}

// Copies state s between the 16-byte representation and complex64.
qfd_status convert_state(qfd_plan_t pl, int s, int to_f32) {
  const int g = grid_for(pl->n3);
  return with_policy(pl->arith16, [&](auto pol) -> qfd_status {
    using A = decltype(pol);
    if (to_f32) {
      QFD_RUN(PASS_OTHER, (k_convert<A, F32><<<g, 256, 0, pl->st>>>(psi_of<A>(pl, s), psi_of<F32>(pl, s), pl->n3),
                           cudaGetLastError()));
    } else {
      QFD_RUN(PASS_OTHER, (k_convert<F32, A><<<g, 256, 0, pl->st>>>(psi_of<F32>(pl, s), psi_of<A>(pl, s), pl->n3),
                           cudaGetLastError()));
    }
    if (pl->w_state == s) pl->w_stage = ST_NONE;
    return QFD_OK;
  });
}

qfd_status check_state(qfd_plan_t pl, int s) {
  if (!pl) return QFD_ERR_ARG;
  if (s < 0 || s >= pl->p.nstates) return fail(pl, QFD_ERR_ARG, "state index out of range");
  return QFD_OK;
}

qfd_status derive_coefficients(qfd_plan_t pl) {
  QFD_CK(cudaMemsetAsync(pl->flag, 0, sizeof(int), pl->st));
  double2* c64 = (pl->coef16 && pl->arith16 == 0) ? (double2*)pl->coef16 : nullptr;
  dfc* cdf = (pl->coef16 && pl->arith16 == 2) ? (dfc*)pl->coef16 : nullptr;
  QFD_RUN(PASS_OTHER, (k_coef<<<grid_for(pl->n3), 256, 0, pl->st>>>(pl->V, pl->n3, pl->p.dtau,
                                                                     pl->p.kinetic == 0 ? pl->fdtd_c : 0.0, c64,
                                                                     cdf, pl->coef32, pl->Vdf, pl->V32, pl->flag),
                       cudaGetLastError()));
  int bad = 0;
  QFD_CK(cudaMemcpyAsync(&bad, pl->flag, sizeof(int), cudaMemcpyDeviceToHost, pl->st));
  QFD_CK(cudaStreamSynchronize(pl->st));
  if (bad) {
    pl->has_pot = false;
    return fail(pl, QFD_ERR_UNSTABLE_DT, "1 + dtau V/2 <= 0 or non-finite V at some site");
  }
  pl->has_pot = true;
  return QFD_OK;
}

bool uses16(int precision) { return precision != QFD_C64; }
bool uses32(int precision);
// any arithmetic on the FP32 pipe (complex64 or double-float)
bool uses_vdf(int precision) { return precision != QFD_C128; }
int arith16_of(int precision) { return (precision == QFD_DF64 || precision == QFD_C64_REFINE_DF) ? 2 : 0; }
// Which per-site update arrays a plan holds: the FP64 coefficients (complex128
// pass A, and every 16-byte H_K(0) update), the complex64 H_K(0) coefficients,
// and V in FP32 (complex64 pass A of the FFT terms).
bool needs_coef16(const qfd_params& p) { return uses16(p.precision) && (arith16_of(p.precision) == 0 || p.kinetic == 0); }
bool needs_coef32(const qfd_params& p) { return uses32(p.precision) && p.kinetic == 0; }
bool needs_v32(const qfd_params& p) { return uses32(p.precision) && p.kinetic != 0; }
// Device bytes a plan with these parameters allocates (lattices, tables, partials).
size_t plan_device_bytes(const qfd_params& p) {
  const size_t n = (size_t)p.n, n3 = n * n * n;
  const size_t npart = (size_t)std::max(
      std::max(std::max(max_partials<F64>(p.n), max_partials<F32>(p.n)), max_partials<DF>(p.n)), GS_BLOCKS);
  size_t b = n3 * 16 + n3 * 8 + n * (48 + 8 + 16 + 8 + 4 + 8) + npart * 8 * (3 + 2 * MAX_LOWER) + 1024;
  if (uses16(p.precision)) b += (size_t)(p.nstates + 1) * n3 * 16;
  if (uses32(p.precision)) b += (size_t)(p.nstates + 1) * n3 * 8;
  if (needs_coef16(p)) b += n3 * 16;
  if (needs_coef32(p)) b += n3 * 8;
  if (needs_v32(p)) b += n3 * sizeof(float);
  if (uses_vdf(p.precision)) b += n3 * sizeof(df);
  return b;
}
bool uses32(int precision) {
  return precision == QFD_C64 || precision == QFD_C64_REFINE || precision == QFD_C64_REFINE_DF;
}
bool refines(int precision) { return precision == QFD_C64_REFINE || precision == QFD_C64_REFINE_DF; }

// One step of Eq. (iter_proced) for `count` lattices of one size in
// arithmetic A, with exactly the operations step_once applies to each lattice
// (check = 1: the energy-check step of a period), but each pass one launch
// over the lattices: the lattices whose W holds the forward x transform take
// passes B, C and D as three batched launches (any other advances alone),
// then pass A runs as one batched launch per partial-sum mode; the cadence
// and the bookkeeping are step_once's, per plan.  Every plan's stream must be
// `st` (the caller arranges it).
template <class A>
qfd_status batch_step_once(qfd_plan_s* const* pls, const int* ss, int count, int check, cudaStream_t st) {
  qfd_plan_t p0 = pls[0];
  const int64_t n = p0->p.n;
  // launch shapes: plans[0]'s (the choice depends only on n and the arithmetic);
  // the TMA pass A needs every plan's tensor maps
  const int vy = p0->tune_vy[A::id], vz = p0->tune_vz[A::id];
  int vx = p0->tune_vx[A::id];
  for (int i = 0; i < count && vx == 2; ++i)
    if (!(A::id == 1 && pls[i]->tmaps)) vx = 0;
  qfd_status r;
  BatchY by{};
  BatchZ bz{};
  int nx = 0;
  for (int i = 0; i < count; ++i) {
    qfd_plan_t pl = pls[i];
    if ((r = ensure_w<A>(pl, ss[i])) != QFD_OK) return r;
    if (pl->w_stage == ST_X) {
      by.W[nx] = bz.W[nx] = pl->W;
      by.tw[nx] = bz.tw[nx] = tw_of<A>(pl);
      bz.ktab[nx] = ktab_of<A>(pl);
      bz.kp[nx] = pl->kin;
      ++nx;
    } else if ((r = advance_to_d<A>(pl, 0)) != QFD_OK) {
      return r;
    }
  }
  if (nx > 0) {
    qfd_plan_t pl = p0;  // the batched launches are counted and timed on plans[0]
    QFD_RUN(PASS_FWD_Y, launch_fft_y_batch<A>(n, by, nx, -1, vy, st));
    QFD_RUN(PASS_ZKIN, launch_zpass_batch<A>(n, bz, nx, 0, vz, st, nullptr));
    QFD_RUN(PASS_INV_Y, launch_fft_y_batch<A>(n, by, nx, +1, vy, st));
  }
  // pass A, grouped by partial-sum mode as step_once chooses it: STATS_NORM
  // where the step ends in a cadence without a projection, STATS_FULL on the
  // check step (unless a projection recomputes the partials), else none
  BatchU bu[3] = {};
  int nu[3] = {0, 0, 0};
  uint32_t scaled[3] = {0u, 0u, 0u};
  for (int i = 0; i < count; ++i) {
    qfd_plan_t pl = pls[i];
    const int s = ss[i];
    const bool ortho_next = (pl->t[s] + 1) % pl->p.ortho_every == 0;
    int g = STATS_NONE;
    if (ortho_next) g = projects(pl, s) ? STATS_NONE : (check ? STATS_FULL : STATS_NORM);
    else if (check) g = STATS_FULL;
    const int j = nu[g]++;
    BatchU& b = bu[g];
    b.W[j] = pl->W;
    b.psi[j] = psi_of<A>(pl, s);
    b.u[j] = uin_of<A>(pl);
    b.up[j] = pl->up;
    b.V[j] = v_of<A>(pl);
    b.scale[j] = pl->scal + SC_SCALE;
    b.scale_f[j] = pl->scalf;
    b.tw[j] = tw_of<A>(pl);
    b.part[j] = pl->partA;
    b.err[j] = pl->errflag;
    if (A::id == 1 && pl->tmaps) {
      b.tmap[j][0] = pl->tmaps;
      b.tmap[j][1] = psi_tmap(pl, b.psi[j]);
      b.tmap[j][2] = pl->tmaps + 1;
    }
    if (pl->pending) scaled[g] |= 1u << j;
  }
  int nb = 0;
  for (int g = 0; g < 3; ++g) {
    if (nu[g] == 0) continue;
    qfd_plan_t pl = p0;
    QFD_RUN(PASS_UPDATE_X, launch_update_x_batch<A>(n, bu[g], nu[g], scaled[g], g, vx, st, &nb, p0->tma_test));
  }
  // every plan's bookkeeping first, so that psi, W and the step counter
  // agree for all of them even if a later cadence fails
  for (int i = 0; i < count; ++i) {
    qfd_plan_t pl = pls[i];
    pl->nA = nb;
    pl->w_stage = ST_X;
    pl->pending = false;
    pl->t[ss[i]] += 1;
  }
  for (int i = 0; i < count; ++i) {
    qfd_plan_t pl = pls[i];
    const int s = ss[i];
    if (pl->t[s] % pl->p.ortho_every == 0) {
      if ((r = cadence<A>(pl, s, check)) != QFD_OK) return r;
      if (pl->snap_every > 0 && s == 0 && pl->t[s] % pl->snap_every == 0 && (r = take_snapshot<A>(pl)) != QFD_OK)
        return r;
    } else if (check) {
      if ((r = finalize(pl, pl->partA, 2, pl->nA, OP_N2PV)) != QFD_OK) return r;
    }
  }
  return QFD_OK;
}

// qfd_step_batch after its checks (every plan's stream pointed at plans[0]'s).
template <class A>
qfd_status step_batch(qfd_plan_s* const* pls, const int* ss, int count, int64_t nsteps) {
  qfd_status r;
  for (int64_t it = 0; it < nsteps; ++it)
    if ((r = batch_step_once<A>(pls, ss, count, 0, pls[0]->st)) != QFD_OK) return r;
  for (int i = 0; i < count; ++i)
    if ((r = materialize<A>(pls[i], ss[i])) != QFD_OK) return r;
  return QFD_OK;
}

// period_launch for `count` lattices of one size in arithmetic A at once (FFT
// kinetic terms): check_every batched steps, the last one with the energy
// check's partials, then passes B and C with the Parseval partial as batched
// launches and each plan's energy, whose scalars are copied asynchronously
// into that plan's pinned host buffer.  Nothing synchronises, so the period
// can be captured into a CUDA graph.  Every plan's stream must be `st`.
template <class A>
qfd_status batch_period_launch(qfd_plan_s* const* pls, const int* ss, int count, cudaStream_t st) {
  qfd_plan_t p0 = pls[0];
  const int64_t n = p0->p.n;
  const int ce = p0->p.check_every;
  qfd_status r;
  for (int j = 0; j < ce; ++j)
    if ((r = batch_step_once<A>(pls, ss, count, j == ce - 1, st)) != QFD_OK) return r;
  BatchY by{};
  BatchZ bz{};
  for (int i = 0; i < count; ++i) {
    qfd_plan_t pl = pls[i];
    if (pl->w_stage != ST_X) return fail(pl, QFD_ERR_STATE, "internal: energy needs W after the x pass");
    by.W[i] = bz.W[i] = pl->W;
    by.tw[i] = bz.tw[i] = tw_of<A>(pl);
    bz.ktab[i] = ktab_of<A>(pl);
    bz.kp[i] = pl->kin;
    bz.part[i] = pl->partC;
  }
  int nc = 0;
  {
    qfd_plan_t pl = p0;
    const int vy = p0->tune_vy[A::id], vz = p0->tune_vz[A::id];
    QFD_RUN(PASS_FWD_Y, launch_fft_y_batch<A>(n, by, count, -1, vy, st));
    QFD_RUN(PASS_ZKIN, launch_zpass_batch<A>(n, bz, count, 1, vz, st, &nc));
  }
  for (int i = 0; i < count; ++i) {
    qfd_plan_t pl = pls[i];
    pl->nC = nc;
    pl->w_stage = ST_C;
    if ((r = finalize(pl, pl->partC, 1, pl->nC, OP_ENERGY)) != QFD_OK) return r;
    QFD_CK(cudaMemcpyAsync(pl->hscal, pl->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
    QFD_CK(cudaMemcpyAsync(pl->hscal + SC_COUNT, pl->errflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  return QFD_OK;
}

}  // namespace

// ------------------------------------------------ tensor maps (TMA pass A)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime.
EncodeTiled tensor_map_encoder() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

// A lattice at `base` viewed as N rows (x) of N^2 sites (y, z) of elem_bytes
// each; boxes of xt sites by min(N, 256) rows, no swizzle, no fill.
bool encode_lattice_map(EncodeTiled enc, CUtensorMap* m, void* base, int64_t n, int elem_bytes, int xt) {
  const cuuint64_t dims[2] = {(cuuint64_t)(n * n), (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)(n * n * elem_bytes)};
  const cuuint32_t box[2] = {(cuuint32_t)xt, (cuuint32_t)(n < 256 ? n : 256)};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return enc(m, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of the complex64 work lattice, V in FP32 and every complex64
// state buffer (the spare included), copied to the device for the TMA pass A.
bool build_tensor_maps(qfd_plan_t pl) {
  const EncodeTiled enc = tensor_map_encoder();
  const int xt = launch_tma_xt<F32>(pl->p.n);
  if (!enc || xt <= 0 || !pl->psi32 || !pl->V32) return false;
  const int64_t n = pl->p.n;
  std::vector<CUtensorMap> maps((size_t)pl->p.nstates + 3);
  bool ok = encode_lattice_map(enc, &maps[0], pl->W, n, 8, xt) && encode_lattice_map(enc, &maps[1], pl->V32, n, 4, xt);
  for (int i = 0; ok && i <= pl->p.nstates; ++i)
    ok = encode_lattice_map(enc, &maps[2 + i], (char*)pl->psi32 + (size_t)i * pl->n3 * sizeof(float2), n, 8, xt);
  if (!ok) return false;
  void* d = nullptr;
  if (cudaMalloc(&d, maps.size() * sizeof(CUtensorMap)) != cudaSuccess) return false;
  if (cudaMemcpy(d, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return false;
  }
  pl->tmaps = static_cast<CUtensorMap*>(d);
  return true;
}

// ================================================================ C ABI
extern "C" {

qfd_status qfd_plan(const qfd_params* params, qfd_plan_t* out) {
  if (out) *out = nullptr;
  if (!params || !out) {
    g_create_error = "null argument";
    return QFD_ERR_ARG;
  }
  const qfd_params& p = *params;
  if (!supported_n(p.n)) {
    g_create_error = "n must be one of 8, 16, 32, 64, 96, 128, 192, 256, 512, 1024";
    return QFD_ERR_ARG;
  }
  if (!(p.a > 0) || !(p.mass > 0) || !(p.dtau > 0) || p.kinetic < 0 || p.kinetic > 3 || p.nstates < 1 ||
      p.nstates > MAX_LOWER || p.precision < 0 || p.precision > QFD_C64_REFINE_DF || p.ortho_every < 1 ||
      p.check_every < 1 || (p.centre != QFD_CENTRE_GRID && p.centre != QFD_CENTRE_OFFGRID) || (p.stop_rule != QFD_STOP_PAPER && p.stop_rule != QFD_STOP_TAIL) ||
      p.max_steps < 0 || (p.rest_mass != 0 && p.rest_mass != 1)) {
    g_create_error = "invalid parameter (a, mass, dtau > 0; kinetic 0..3; nstates 1..8; precision 0..4; cadences >= 1)";
    return QFD_ERR_ARG;
  }
  const int64_t n = p.n;
  // per-axis kinetic table and the largest T(k) (all three k at the table maximum)
  std::vector<double> ktab(n);
  double kmax = 0;
  for (int64_t j = 0; j < n; ++j) {
    const int64_t m = j <= n / 2 ? j : j - n;
    if (p.kinetic == 1) {
      const double k = 2.0 * M_PI * (double)m / (double)n;
      ktab[j] = k * k;
    } else {
      const double sn = std::sin(M_PI * (double)(m < 0 ? -m : m) / (double)n);
      ktab[j] = 4.0 * sn * sn;
    }
    kmax = std::fmax(kmax, ktab[j]);
  }
  const double n3d = (double)n * (double)n * (double)n;
  KinParams kin{};
  kin.kinterm = p.kinetic;
  kin.pref = 1.0 / (2.0 * p.a * p.a * p.mass * n3d);
  kin.am2 = (p.a * p.mass) * (p.a * p.mass);
  kin.inv_a_n3 = 1.0 / (p.a * n3d);
  kin.m0_n3 = p.rest_mass ? 0.0 : p.mass / n3d;
  kin.f_pref = (float)kin.pref;
  kin.f_am2 = (float)kin.am2;
  kin.f_ia = (float)kin.inv_a_n3;
  kin.f_m0 = (float)kin.m0_n3;
  kin.d_pref = host_split(kin.pref);
  kin.d_am2 = host_split(kin.am2);
  kin.d_ia = host_split(kin.inv_a_n3);
  kin.d_m0 = host_split(kin.m0_n3);
  const double smax = 3.0 * kmax;
  const double tmax = p.kinetic == 3 ? std::sqrt(smax + kin.am2) / p.a - (p.rest_mass ? 0.0 : p.mass)
                                     : smax / (2.0 * p.a * p.a * p.mass);
  if (!(p.dtau * tmax < 2.0)) {
    char buf[160];
    snprintf(buf, sizeof(buf), "unstable time step: dtau * max T(k) = %.6g >= 2", p.dtau * tmax);
    g_create_error = buf;
    return QFD_ERR_UNSTABLE_DT;
  }

  qfd_plan_t pl = new qfd_plan_s();
  pl->p = p;
  pl->n3 = n * n * n;
  pl->kin = kin;
  if ((n & (n - 1)) == 0)
    for (pl->lg = 0; ((int64_t)1 << pl->lg) < n; ++pl->lg) {
    }
  pl->fdtd_c = 1.0 / (2.0 * p.mass * p.a * p.a);
  pl->up.f_dtau = (float)p.dtau;
  pl->up.f_hdt = (float)(0.5 * p.dtau);
  pl->up.d_dtau = host_split(p.dtau);
  pl->up.d_hdt = host_split(0.5 * p.dtau);
  pl->t.assign(p.nstates, 0);
  pl->parity.assign(p.nstates, 0);
  pl->steps16.assign(p.nstates, 0);
  pl->steps32.assign(p.nstates, 0);
  pl->ebulk.assign(p.nstates, NAN);
  pl->edecay.assign(p.nstates, NAN);
  pl->hist.assign(p.nstates, {});
  pl->arith16 = arith16_of(p.precision);
  pl->phase = uses32(p.precision) ? 1 : pl->arith16;

  auto cleanup_fail = [&](qfd_status s, const std::string& msg) {
    g_create_error = msg;
    qfd_destroy(pl);
    return s;
  };
  if (p.stream) {
    pl->st = (cudaStream_t)p.stream;
  } else {
    if (cudaStreamCreateWithFlags(&pl->st, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup_fail(QFD_ERR_CUDA, "cudaStreamCreate failed");
    pl->own_stream = true;
  }
  const int64_t n3 = pl->n3;
  const int npart =
      std::max(std::max(std::max(max_partials<F64>(n), max_partials<F32>(n)), max_partials<DF>(n)), GS_BLOCKS);
  struct Alloc {
    void** ptr;
    size_t bytes;
  };
  std::vector<Alloc> allocs = {
      {(void**)&pl->W, (size_t)n3 * 16},
      {(void**)&pl->V, (size_t)n3 * sizeof(double)},
      {(void**)&pl->tw64, (size_t)3 * n * sizeof(double2)},  // plain twiddles + the scaled radix-8 block
      {(void**)&pl->tw32, (size_t)n * sizeof(float2)},
      {(void**)&pl->twdf, (size_t)n * sizeof(dfc)},
      {(void**)&pl->ktab64, (size_t)n * sizeof(double)},
      {(void**)&pl->ktab32, (size_t)n * sizeof(float)},
      {(void**)&pl->ktabdf, (size_t)n * sizeof(df)},
      {(void**)&pl->partA, (size_t)2 * npart * sizeof(double)},
      {(void**)&pl->partC, (size_t)npart * sizeof(double)},
      {(void**)&pl->partG, (size_t)2 * MAX_LOWER * npart * sizeof(double)},
      {(void**)&pl->scal, SC_COUNT * sizeof(double)},
      {(void**)&pl->scalf, 16 * sizeof(float)},
      {(void**)&pl->flag, sizeof(int)},
      {(void**)&pl->errflag, sizeof(int)},
  };
  if (uses16(p.precision)) allocs.push_back({(void**)&pl->psi16, (size_t)(p.nstates + 1) * n3 * 16});
  if (uses32(p.precision)) allocs.push_back({(void**)&pl->psi32, (size_t)(p.nstates + 1) * n3 * sizeof(float2)});
  if (needs_coef16(p)) allocs.push_back({(void**)&pl->coef16, (size_t)n3 * 16});
  if (needs_coef32(p)) allocs.push_back({(void**)&pl->coef32, (size_t)n3 * sizeof(float2)});
  if (needs_v32(p)) allocs.push_back({(void**)&pl->V32, (size_t)n3 * sizeof(float)});
  if (uses_vdf(p.precision)) allocs.push_back({(void**)&pl->Vdf, (size_t)n3 * sizeof(df)});
  for (auto& a : allocs) {
    if (cudaMalloc(a.ptr, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      char buf[128];
      snprintf(buf, sizeof(buf), "cudaMalloc of %zu bytes failed", a.bytes);
      return cleanup_fail(QFD_ERR_OOM, buf);
    }
  }
  for (int j = 0; j < p.nstates; ++j) {
    pl->sp16.push_back(pl->psi16 ? (char*)pl->psi16 + (size_t)j * n3 * 16 : nullptr);
    pl->sp32.push_back(pl->psi32 ? (char*)pl->psi32 + (size_t)j * n3 * sizeof(float2) : nullptr);
  }
  pl->spare16 = pl->psi16 ? (char*)pl->psi16 + (size_t)p.nstates * n3 * 16 : nullptr;
  pl->spare32 = pl->psi32 ? (char*)pl->psi32 + (size_t)p.nstates * n3 * sizeof(float2) : nullptr;
  std::vector<double2> tw(3 * n);
  std::vector<float2> tw32(n);
  std::vector<dfc> twdf(n);
  std::vector<float> kt32(n);
  std::vector<df> ktdf(n);
  for (int64_t e = 0; e < n; ++e) {
    double c, s;
    unit_root(e, n, &c, &s);
    tw[e] = double2{c, s};
    tw32[e] = float2{(float)c, (float)s};
    twdf[e] = dfc{host_split(c), host_split(s)};
    kt32[e] = (float)ktab[e];
    ktdf[e] = host_split(ktab[e]);
  }
  scaled_twiddle_table(n, tw.data(), tw.data() + n);
  bool ok = cudaMemcpy(pl->tw64, tw.data(), 3 * n * sizeof(double2), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->tw32, tw32.data(), n * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->twdf, twdf.data(), n * sizeof(dfc), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->ktab64, ktab.data(), n * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->ktab32, kt32.data(), n * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->ktabdf, ktdf.data(), n * sizeof(df), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(pl->scal, 0, SC_COUNT * sizeof(double)) == cudaSuccess;
  if (!ok) return cleanup_fail(QFD_ERR_CUDA, "table upload failed");
  if (cudaHostAlloc((void**)&pl->hscal, (SC_COUNT + 1) * sizeof(double), cudaHostAllocDefault) != cudaSuccess)
    return cleanup_fail(QFD_ERR_OOM, "pinned host buffer allocation failed");
  std::memset(pl->hscal, 0, (SC_COUNT + 1) * sizeof(double));
  if (cudaMemset(pl->errflag, 0, sizeof(int)) != cudaSuccess) return cleanup_fail(QFD_ERR_CUDA, "memset failed");
  // the TMA-staged pass A is optional: without the encoder or on failure the
  // plan simply runs the direct kernels
  if (needs_v32(p) && launch_tma_xt<F32>(n) > 0 && !build_tensor_maps(pl)) cudaGetLastError();
  *out = pl;
  return QFD_OK;
}

void qfd_destroy(qfd_plan_t pl) {
  if (!pl) return;
  if (pl->st) cudaStreamSynchronize(pl->st);
  void* bufs[] = {pl->psi16, pl->psi32, pl->W,      pl->coef16, pl->coef32, pl->V,     pl->tw64,
                  pl->tw32,  pl->twdf,  pl->ktab64, pl->ktab32, pl->ktabdf, pl->partA, pl->partC,
                  pl->partG, pl->scal,  pl->scalf, pl->flag, pl->Vdf, pl->V32, pl->errflag, pl->tmaps};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (pl->hscal) cudaFreeHost(pl->hscal);
  for (auto& v : pl->ev)
    for (auto e : v) cudaEventDestroy(e);
  if (pl->own_stream && pl->st) cudaStreamDestroy(pl->st);
  delete pl;
}

const char* qfd_last_error(qfd_plan_t pl) { return pl ? pl->err.c_str() : g_create_error.c_str(); }

qfd_status qfd_set_potential(qfd_plan_t pl, const double* V, int on_device) {
  if (!pl || !V) return fail(pl, QFD_ERR_ARG, "null argument");
  QFD_CK(cudaMemcpyAsync(pl->V, V, pl->n3 * sizeof(double),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, pl->st));
  return derive_coefficients(pl);
}

qfd_status qfd_fill_potential(qfd_plan_t pl, int kind, const double* coeffs, int ncoeffs) {
  if (!pl) return QFD_ERR_ARG;
  if (kind < QFD_POT_ZERO || kind > QFD_POT_SOFTCOUL || ncoeffs < 0 || (ncoeffs > 0 && !coeffs))
    return fail(pl, QFD_ERR_ARG, "unknown potential kind or missing coefficients");
  const int need = kind == QFD_POT_CORNELL ? 2 : (kind == QFD_POT_HO || kind == QFD_POT_SOFTCOUL) ? 1 : 0;
  if (ncoeffs < need) return fail(pl, QFD_ERR_ARG, "too few potential coefficients");
  const double c0 = need > 0 ? coeffs[0] : 0.0, c1 = need > 1 ? coeffs[1] : 0.0;
  QFD_RUN(PASS_OTHER, (k_potential<<<grid_for(pl->n3), 256, 0, pl->st>>>(pl->V, pl->p.n, pl->p.a, kind, c0, c1,
                                                                         pl->p.centre == QFD_CENTRE_OFFGRID),
                       cudaGetLastError()));
  return derive_coefficients(pl);
}

qfd_status qfd_add_random_field(qfd_plan_t pl, uint64_t seed, double corr, double amplitude) {
  if (!pl) return QFD_ERR_ARG;
  if (!pl->has_pot) return fail(pl, QFD_ERR_STATE, "set a potential before adding a random field");
  if (!(corr > 0) || !(amplitude >= 0))
    return fail(pl, QFD_ERR_ARG, "corr > 0 and amplitude >= 0 required");
  GrfTaps taps{};
  taps.r = (int)std::ceil(corr * std::sqrt(2.0 * std::log(1e18)));
  if (taps.r > GRF_MAX_R) return fail(pl, QFD_ERR_ARG, "corr too large (at most 21 lattice units)");
  for (int j = -taps.r; j <= taps.r; ++j) taps.g[j + taps.r] = std::exp(-(double)j * j / (2.0 * corr * corr));
  // the work lattice holds the two real scratch fields
  double* f0 = reinterpret_cast<double*>(pl->W);
  double* f1 = f0 + pl->n3;
  pl->w_stage = ST_NONE;
  pl->w_state = -1;
  const int g = grid_for(pl->n3);
  QFD_RUN(PASS_OTHER, (k_grf_noise<<<g, 256, 0, pl->st>>>(f0, pl->n3, seed), cudaGetLastError()));
  QFD_RUN(PASS_OTHER, (k_grf_conv<<<g, 256, 0, pl->st>>>(f0, f1, Lat{pl->p.n, pl->lg}, 0, taps), cudaGetLastError()));
  QFD_RUN(PASS_OTHER, (k_grf_conv<<<g, 256, 0, pl->st>>>(f1, f0, Lat{pl->p.n, pl->lg}, 1, taps), cudaGetLastError()));
  QFD_RUN(PASS_OTHER, (k_grf_conv<<<g, 256, 0, pl->st>>>(f0, f1, Lat{pl->p.n, pl->lg}, 2, taps), cudaGetLastError()));
  QFD_RUN(PASS_OTHER, (k_grf_moments<<<GS_BLOCKS, 256, 0, pl->st>>>(f1, pl->n3, pl->partG), cudaGetLastError()));
  qfd_status r = finalize(pl, pl->partG, 2, GS_BLOCKS, OP_SUMS);
  if (r != QFD_OK) return r;
  QFD_RUN(PASS_OTHER, (k_grf_add<<<g, 256, 0, pl->st>>>(pl->V, f1, pl->n3, pl->scal + SC_SUMS, amplitude),
                       cudaGetLastError()));
  return derive_coefficients(pl);
}

qfd_status qfd_get_potential(qfd_plan_t pl, double* V, int on_device) {
  if (!pl || !V) return fail(pl, QFD_ERR_ARG, "null argument");
  if (!pl->has_pot) return fail(pl, QFD_ERR_STATE, "no potential set");
  QFD_CK(cudaMemcpyAsync(V, pl->V, pl->n3 * sizeof(double),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, pl->st));
  QFD_CK(cudaStreamSynchronize(pl->st));
  return QFD_OK;
}

qfd_status qfd_set_psi(qfd_plan_t pl, int s, const double* psi, int on_device) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  if (!psi) return fail(pl, QFD_ERR_ARG, "null psi");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t bytes = pl->n3 * sizeof(double2);
  const int g = grid_for(pl->n3);
  if (pl->psi16 && pl->arith16 == 0) {
    QFD_CK(cudaMemcpyAsync(psi_of<F64>(pl, s), psi, bytes, kind, pl->st));
  } else {
    // stage the complex128 values in W, then round into the plan's representation
    QFD_CK(cudaMemcpyAsync(pl->W, psi, bytes, kind, pl->st));
    if (pl->psi16)
      QFD_RUN(PASS_OTHER,
              (k_convert<F64, DF><<<g, 256, 0, pl->st>>>(pl->W, psi_of<DF>(pl, s), pl->n3), cudaGetLastError()));
    else
      QFD_RUN(PASS_OTHER,
              (k_convert<F64, F32><<<g, 256, 0, pl->st>>>(pl->W, psi_of<F32>(pl, s), pl->n3), cudaGetLastError()));
    pl->w_stage = ST_NONE;
  }
  if (pl->psi16 && pl->psi32 && (r = convert_state(pl, s, 1)) != QFD_OK) return r;
  pl->t[s] = 0;
  if (pl->w_state == s) pl->w_stage = ST_NONE;
  if (!on_device) QFD_CK(cudaStreamSynchronize(pl->st));  // caller may reuse its host buffer
  return QFD_OK;
}

qfd_status qfd_fill_psi_uniform(qfd_plan_t pl, int s, uint64_t seed) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  const int g = grid_for(pl->n3);
  if (pl->psi16 && pl->arith16 == 0)
    QFD_RUN(PASS_OTHER,
            (k_fill_uniform<F64><<<g, 256, 0, pl->st>>>(psi_of<F64>(pl, s), pl->n3, seed), cudaGetLastError()));
  if (pl->psi16 && pl->arith16 == 2)
    QFD_RUN(PASS_OTHER,
            (k_fill_uniform<DF><<<g, 256, 0, pl->st>>>(psi_of<DF>(pl, s), pl->n3, seed), cudaGetLastError()));
  if (pl->psi32)
    QFD_RUN(PASS_OTHER,
            (k_fill_uniform<F32><<<g, 256, 0, pl->st>>>(psi_of<F32>(pl, s), pl->n3, seed), cudaGetLastError()));
  pl->t[s] = 0;
  if (pl->w_state == s) pl->w_stage = ST_NONE;
  return QFD_OK;
}

qfd_status qfd_get_psi(qfd_plan_t pl, int s, double* out, int on_device) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  if (!out) return fail(pl, QFD_ERR_ARG, "null output");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t bytes = pl->n3 * sizeof(double2);
  r = with_policy(pl->phase, [&](auto pol) -> qfd_status {
    using A = decltype(pol);
    qfd_status q = materialize<A>(pl, s);
    if (q != QFD_OK) return q;
    if (A::id == 0) {
      QFD_CK(cudaMemcpyAsync(out, psi_of<A>(pl, s), bytes, kind, pl->st));
    } else {
      QFD_RUN(PASS_OTHER, (k_convert<A, F64><<<grid_for(pl->n3), 256, 0, pl->st>>>(psi_of<A>(pl, s), pl->W, pl->n3),
                           cudaGetLastError()));
      pl->w_stage = ST_NONE;
      QFD_CK(cudaMemcpyAsync(out, pl->W, bytes, kind, pl->st));
    }
    return QFD_OK;
  });
  if (r != QFD_OK) return r;
  QFD_CK(cudaStreamSynchronize(pl->st));
  return QFD_OK;
}

qfd_status qfd_observables(qfd_plan_t pl, int s, double min_sep_edge, double* out, int nout) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  if (!out || nout < 1 || !(min_sep_edge >= 0.0) || !(min_sep_edge < 1.0))
    return fail(pl, QFD_ERR_ARG, "need an output buffer and 0 <= min_sep_edge < 1");
  const Lat lat{pl->p.n, pl->lg};
  const double half = (1.0 - min_sep_edge) * (double)pl->p.n / 2.0;
  const int offgrid = pl->p.centre == QFD_CENTRE_OFFGRID;
  r = with_policy(pl->phase, [&](auto pol) -> qfd_status {
    using A = decltype(pol);
    qfd_status q = materialize<A>(pl, s);
    if (q != QFD_OK) return q;
    QFD_RUN(PASS_OTHER, (k_observables<A><<<GS_BLOCKS, 256, 0, pl->st>>>(psi_of<A>(pl, s), lat, offgrid, half, pl->partG),
                         cudaGetLastError()));
    return finalize(pl, pl->partG, NOBS, GS_BLOCKS, OP_OBS);
  });
  if (r != QFD_OK) return r;
  double h[NOBS];
  QFD_CK(cudaMemcpyAsync(h, pl->scal + SC_SUMS, sizeof(h), cudaMemcpyDeviceToHost, pl->st));
  QFD_CK(cudaStreamSynchronize(pl->st));
  for (int i = 0; i < nout && i < NOBS; ++i) out[i] = h[i];
  return QFD_OK;
}

qfd_status qfd_set_parity(qfd_plan_t pl, int s, int parity) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  if (parity < -1 || parity > 1) return fail(pl, QFD_ERR_ARG, "parity must be -1, 0 or 1");
  pl->parity[s] = parity;
  return QFD_OK;
}

qfd_status qfd_step(qfd_plan_t pl, int s, int64_t nsteps) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  if (!pl->has_pot) return fail(pl, QFD_ERR_STATE, "set a potential before stepping");
  if (nsteps < 0) return fail(pl, QFD_ERR_ARG, "nsteps < 0");
  return with_policy(pl->phase, [&](auto pol) -> qfd_status {
    using A = decltype(pol);
    for (int64_t i = 0; i < nsteps; ++i) {
      qfd_status q = step_once<A>(pl, s, 0);
      if (q != QFD_OK) return q;
    }
    qfd_status q = materialize<A>(pl, s);
    return q != QFD_OK ? q : sync_checked(pl);
  });
}

qfd_status qfd_step_batch(const qfd_plan_t* plans, const int* states, int count, int64_t nsteps) {
  static_assert(QFD_MAX_BATCH == MAX_BATCH, "batch size of the header and of the kernels");
  if (!plans || !states || count < 1 || count > QFD_MAX_BATCH || !plans[0]) {
    g_create_error = "qfd_step_batch: null array or plan, or count outside 1..QFD_MAX_BATCH";
    return QFD_ERR_ARG;
  }
  qfd_plan_t p0 = plans[0];
  for (int i = 0; i < count; ++i) {
    qfd_plan_t pl = plans[i];
    if (!pl) return fail(p0, QFD_ERR_ARG, "null plan in the batch");
    for (int j = 0; j < i; ++j)
      if (plans[j] == pl) return fail(p0, QFD_ERR_ARG, "a plan appears twice in the batch");
    if (states[i] < 0 || states[i] >= pl->p.nstates) return fail(p0, QFD_ERR_ARG, "state index out of range");
    if (pl->p.n != p0->p.n || pl->phase != p0->phase)
      return fail(p0, QFD_ERR_ARG, "the plans of a batch share n and the current arithmetic");
    if (pl->p.kinetic == 0) return fail(p0, QFD_ERR_ARG, "batched steps take the FFT kinetic terms (kinetic 1..3)");
    if (!pl->has_pot) return fail(p0, QFD_ERR_STATE, "set a potential before stepping");
  }
  if (nsteps < 0) return fail(p0, QFD_ERR_ARG, "nsteps < 0");
  // order every plan's earlier work before the batch, run the batch on
  // plans[0]'s stream, order every plan's later work after it
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
    return fail(p0, QFD_ERR_CUDA, "cudaEventCreate failed");
  std::vector<cudaStream_t> own(count);
  for (int i = 0; i < count; ++i) {
    own[i] = plans[i]->st;
    if (own[i] != p0->st) {
      cudaEventRecord(ev, own[i]);
      cudaStreamWaitEvent(p0->st, ev, 0);
    }
    plans[i]->st = p0->st;
  }
  qfd_status r = with_policy(p0->phase, [&](auto pol) -> qfd_status {
    return step_batch<decltype(pol)>(plans, states, count, nsteps);
  });
  cudaEventRecord(ev, p0->st);
  for (int i = 0; i < count; ++i) {
    plans[i]->st = own[i];
    if (own[i] != p0->st) cudaStreamWaitEvent(own[i], ev, 0);
  }
  cudaEventDestroy(ev);
  if (r != QFD_OK) return r;
  for (int i = 0; i < count; ++i)
    if ((r = sync_checked(plans[i])) != QFD_OK) return r;
  return QFD_OK;
}

qfd_status qfd_energy(qfd_plan_t pl, int s, double* E, double* norm2) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  if (!pl->has_pot) return fail(pl, QFD_ERR_STATE, "set a potential before taking the energy");
  return with_policy(pl->phase, [&](auto pol) -> qfd_status { return energy_full<decltype(pol)>(pl, s, E, norm2); });
}

qfd_status qfd_solve_states(qfd_plan_t pl, int nstates, const int* parity, double* E_out, int64_t* steps_out) {
  if (!pl) return QFD_ERR_ARG;
  if (nstates < 1 || nstates > pl->p.nstates) return fail(pl, QFD_ERR_ARG, "nstates out of range");
  if (!pl->has_pot) return fail(pl, QFD_ERR_STATE, "set a potential before solving");
  for (int s = 0; s < nstates; ++s)
    if (parity && (parity[s] < -1 || parity[s] > 1)) return fail(pl, QFD_ERR_ARG, "parity must be -1, 0 or 1");
  const bool refine = refines(pl->p.precision);
  bool all_conv = true;
  for (int s = 0; s < nstates; ++s) {
    pl->parity[s] = parity ? parity[s] : 0;
    double e = NAN;
    int64_t steps = 0;
    bool conv = false;
    qfd_status r;
    pl->steps32[s] = pl->steps16[s] = 0;
    pl->ebulk[s] = NAN;
    pl->hist[s].clear();
    if (refine) {
      // complex64 bulk to tol_bulk, then the 16-byte arithmetic to tol
      pl->phase = 1;
      if ((r = convert_state(pl, s, 1)) != QFD_OK) return r;
      if ((r = solve_phase<F32>(pl, s, pl->p.tol_bulk, pl->p.max_steps, &e, &steps, &conv, true)) != QFD_OK)
        return r;
      pl->steps32[s] = steps;
      pl->ebulk[s] = e;
      if ((r = convert_state(pl, s, 0)) != QFD_OK) return r;
      pl->phase = pl->arith16;
    } else {
      pl->phase = uses32(pl->p.precision) ? 1 : pl->arith16;
    }
    r = with_policy(pl->phase, [&](auto pol) -> qfd_status {
      return solve_phase<decltype(pol)>(pl, s, pl->p.tol, pl->p.max_steps, &e, &steps, &conv);
    });
    if (r != QFD_OK) return r;
    if (pl->phase == 1) pl->steps32[s] = steps;
    else pl->steps16[s] = steps;
    if (refine && (r = convert_state(pl, s, 1)) != QFD_OK) return r;  // lower state for later bulk phases
    if (E_out) E_out[s] = e;
    if (steps_out) steps_out[s] = pl->steps32[s] + pl->steps16[s];
    if (pl->p.tol >= 0 && !conv) all_conv = false;
  }
  QFD_CK(cudaStreamSynchronize(pl->st));
  if (!all_conv) return fail(pl, QFD_ERR_NOT_CONVERGED, "max_steps reached before the tolerance");
  return QFD_OK;
}

qfd_status qfd_snapshot_states(qfd_plan_t pl, int nout, int parity, int64_t snap_every, double* E_out,
                               int64_t* steps_out) {
  if (!pl) return QFD_ERR_ARG;
  if (!E_out) return fail(pl, QFD_ERR_ARG, "null argument");
  if (nout < 1 || nout > 3 || (nout > 1 && pl->p.nstates < nout + 1))
    return fail(pl, QFD_ERR_ARG, "nout must be 1..3 and the plan must hold nout + 1 states");
  if (snap_every < 1 || snap_every % pl->p.ortho_every != 0)
    return fail(pl, QFD_ERR_ARG, "snap_every must be a positive multiple of ortho_every");
  if (parity < -1 || parity > 1) return fail(pl, QFD_ERR_ARG, "parity must be -1, 0 or 1");
  if (refines(pl->p.precision)) return fail(pl, QFD_ERR_ARG, "snapshot states run in one arithmetic (no refinement)");
  if (!pl->has_pot) return fail(pl, QFD_ERR_STATE, "set a potential before solving");
  pl->phase = uses32(pl->p.precision) ? 1 : pl->arith16;
  bool conv = false;
  qfd_status r = with_policy(pl->phase, [&](auto pol) -> qfd_status {
    return snapshot_states<decltype(pol)>(pl, nout, parity, snap_every, E_out, steps_out, &conv);
  });
  if (r != QFD_OK) return r;
  QFD_CK(cudaStreamSynchronize(pl->st));
  if (pl->p.tol >= 0 && !conv) return fail(pl, QFD_ERR_NOT_CONVERGED, "max_steps reached before the tolerance");
  return QFD_OK;
}

qfd_status qfd_autotune(qfd_plan_t pl, double* ms_out) {
  if (!pl) return QFD_ERR_ARG;
  double ms[27];
  for (double& m : ms) m = NAN;
  QFD_CK(cudaStreamSynchronize(pl->st));
  qfd_status r = QFD_OK;
  if (uses32(pl->p.precision) && (r = autotune_policy<F32>(pl, ms + 9)) != QFD_OK) return r;
  if (pl->psi16 && pl->arith16 == 0 && (r = autotune_policy<F64>(pl, ms + 0)) != QFD_OK) return r;
  if (pl->psi16 && pl->arith16 == 2 && (r = autotune_policy<DF>(pl, ms + 18)) != QFD_OK) return r;
  if ((r = sync_checked(pl)) != QFD_OK) return r;  // a TMA timing launch that gave up
  pl->w_stage = ST_NONE;  // W was used as the timing lattice
  pl->w_state = -1;
  if (ms_out) std::memcpy(ms_out, ms, sizeof(ms));
  return QFD_OK;
}

qfd_status qfd_set_tuning(qfd_plan_t pl, int policy, int y_variant, int z_variant, int x_variant) {
  if (!pl) return QFD_ERR_ARG;
  if (policy < 0 || policy > 2 || y_variant < 0 || y_variant > 2 || z_variant < -1 || z_variant > 2 ||
      x_variant < 0 || x_variant > 2)
    return fail(pl, QFD_ERR_ARG, "policy 0..2, y_variant 0..2, z_variant -1..2, x_variant 0..2");
  pl->tune_vy[policy] = y_variant;
  pl->tune_vz[policy] = z_variant;
  pl->tune_vx[policy] = x_variant;
  return QFD_OK;
}

qfd_status qfd_set_tma_test(qfd_plan_t pl, int arm_without_copies) {
  if (!pl) return QFD_ERR_ARG;
  if (arm_without_copies != 0 && arm_without_copies != 1) return fail(pl, QFD_ERR_ARG, "0 or 1");
  pl->tma_test = arm_without_copies;
  return QFD_OK;
}

int qfd_has_tma(qfd_plan_t pl) { return pl && pl->tmaps ? 1 : 0; }

qfd_status qfd_set_limits(qfd_plan_t pl, int64_t max_steps, double tol, double tol_bulk) {
  if (!pl) return QFD_ERR_ARG;
  if (max_steps < 0) return fail(pl, QFD_ERR_ARG, "max_steps < 0");
  pl->p.max_steps = max_steps;
  pl->p.tol = tol;
  pl->p.tol_bulk = tol_bulk;
  return QFD_OK;
}

qfd_status qfd_get_stats(qfd_plan_t pl, int s, int64_t* steps_c64, int64_t* steps_c128, double* e_bulk) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  if (steps_c64) *steps_c64 = pl->steps32[s];
  if (steps_c128) *steps_c128 = pl->steps16[s];
  if (e_bulk) *e_bulk = pl->ebulk[s];
  return QFD_OK;
}

qfd_status qfd_get_decay(qfd_plan_t pl, int s, double* e_decay) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  if (!e_decay) return fail(pl, QFD_ERR_ARG, "null argument");
  *e_decay = pl->edecay[s];
  return QFD_OK;
}

qfd_status qfd_get_history(qfd_plan_t pl, int s, int64_t* steps, double* E, int capacity, int* count) {
  qfd_status r = check_state(pl, s);
  if (r != QFD_OK) return r;
  if (capacity < 0 || (capacity > 0 && (!steps || !E))) return fail(pl, QFD_ERR_ARG, "bad history buffers");
  const auto& h = pl->hist[s];
  const int n = (int)std::min<size_t>(h.size(), (size_t)capacity);
  for (int i = 0; i < n; ++i) {
    steps[i] = h[i].first;
    E[i] = h[i].second;
  }
  if (count) *count = (int)h.size();
  return QFD_OK;
}

qfd_status qfd_timing_enable(qfd_plan_t pl, int enable) {
  if (!pl) return QFD_ERR_ARG;
  pl->timing = enable != 0;
  return QFD_OK;
}

qfd_status qfd_timing_reset(qfd_plan_t pl) {
  if (!pl) return QFD_ERR_ARG;
  QFD_CK(cudaStreamSynchronize(pl->st));
  for (auto& u : pl->evused) u = 0;
  pl->launches = 0;
  return QFD_OK;
}

qfd_status qfd_timing_query(qfd_plan_t pl, int kind, int64_t* launches, double* total_ms) {
  if (!pl) return QFD_ERR_ARG;
  if (kind < 0 || kind >= PASS_COUNT) return fail(pl, QFD_ERR_ARG, "unknown pass kind");
  QFD_CK(cudaStreamSynchronize(pl->st));
  double tot = 0;
  for (size_t i = 0; i + 1 < pl->evused[kind]; i += 2) {
    float ms = 0;
    QFD_CK(cudaEventElapsedTime(&ms, pl->ev[kind][i], pl->ev[kind][i + 1]));
    tot += ms;
  }
  if (launches) *launches = (int64_t)(pl->evused[kind] / 2);
  if (total_ms) *total_ms = tot;
  return QFD_OK;
}

int64_t qfd_launch_count(qfd_plan_t pl) { return pl ? pl->launches : -1; }

void* qfd_get_stream(qfd_plan_t pl) { return pl ? (void*)pl->st : nullptr; }

qfd_status qfd_sync(qfd_plan_t pl) {
  if (!pl) return QFD_ERR_ARG;
  QFD_CK(cudaStreamSynchronize(pl->st));
  return QFD_OK;
}

}  // extern "C"

// ================================================================ server
static_assert(sizeof(qfd_params) == 96 && sizeof(qfd_request) == 168 && sizeof(qfd_result) == 232 &&
                  sizeof(qfd_server_params) == 40,
              "C ABI struct layouts are fixed (the Python binding mirrors them)");
// Continuous batching of solve requests: requests wait in FIFO order and are
// admitted while their device bytes fit the budget.  Every admitted request
// owns a plan on its own stream, whose priority rises as the lattice shrinks
// (short solves are not held behind the blocks of long ones), and advances by
// periods (check_every steps and an energy check) independently of the
// others: qfd_server_poll issues a period for every request that has none in
// flight, waits until at least one period has ended, and applies the stop rule
// of each ended request, moving it to its next phase, state or completion.
// From its second period in a phase on, a request's period is captured once as
// a CUDA graph on its stream and replayed.
//
// Cohort mode (qfd_server_params.cohorts = 1): requests of one lattice size
// share a stream and advance together, up to QFD_MAX_BATCH of them.  A cohort
// period is one period of every member: each pass of each step is one launch
// over the members of one arithmetic (the batched kernels, which are also the
// single-lattice kernels), the cadence and the stop rule stay per request.
// Once no member is in the first period of a phase, the cohort period is
// captured as a CUDA graph and replayed while the members and their states
// and phases stay the same.
struct Cohort;
struct ReqRun {
  int64_t id = 0;
  qfd_request req{};
  qfd_plan_t plan = nullptr;
  Cohort* cohort = nullptr;         // cohort mode: the cohort the request belongs to
  cudaStream_t st = nullptr;        // the request's stream (owned by the server, or its cohort's)
  cudaEvent_t ev = nullptr;         // end of the period in flight
  cudaGraphExec_t exec = nullptr;   // captured period of (gstate, gphase)
  int64_t exec_kernels = 0;         // kernel launches the captured period holds
  int gstate = -1, gphase = -1;
  size_t bytes = 0;
  int state = 0;
  int phase = 0;          // policy id of the running phase
  bool bulk = false;      // complex64 bulk of a mixed request
  bool fresh = true;      // its first period in this phase is still to run
  bool inflight = false;  // a period is queued on st
  std::chrono::steady_clock::time_point t_issue;  // when the period in flight was queued
  PhaseTracker tr;
  qfd_result res{};
};

struct Cohort {
  int64_t n = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<ReqRun*> members;  // admitted to the cohort
  std::vector<ReqRun*> running;  // the members of the period in flight
  bool inflight = false;
  std::chrono::steady_clock::time_point t_issue;
  cudaGraphExec_t exec = nullptr;  // the captured cohort period
  int64_t exec_kernels = 0;        // kernel launches it holds
  std::vector<int64_t> sig;        // (member id, state, phase) of each member it was captured for
};

struct qfd_server_s {
  qfd_server_params p{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  std::deque<ReqRun*> waiting;
  std::vector<ReqRun*> active;
  std::vector<Cohort*> cohorts;  // cohort mode
  std::vector<qfd_result> done;
  size_t used = 0;
  int64_t next_id = 1;
  cudaEvent_t fork = nullptr;  // admitted requests start after the server stream's work
  int prio_least = 0, prio_greatest = 0;
  double timeout_s = 0.0;  // watchdog on a period in flight (0: none)
  // autotune = 1: launch shapes per (lattice size, precision), taken by the
  // first plan of each and given to every later one (vy, vz, vx per policy)
  std::vector<std::pair<std::pair<int64_t, int>, std::array<int, 9>>> shapes;
  int64_t periods = 0, replays = 0, captures = 0;
  int64_t kernels = 0;  // kernel launches queued, direct or in replayed graphs
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
};

namespace {

double server_clock(qfd_server_t sv) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - sv->t0).count();
}

qfd_status sfail(qfd_server_t sv, qfd_status s, const std::string& msg) {
  sv->err = msg;
  return s;
}

qfd_params request_params(const qfd_server_t sv, const qfd_request& r) {
  qfd_params p{};
  p.n = r.n;
  p.a = r.a;
  p.mass = r.mass;
  p.dtau = r.dtau;
  p.kinetic = r.kinetic;
  p.rest_mass = r.rest_mass;
  p.nstates = r.nstates;
  p.precision = r.precision;
  p.ortho_every = sv->p.ortho_every;
  p.check_every = sv->p.check_every;
  p.centre = r.centre;
  p.stop_rule = r.stop_rule;
  p.max_steps = r.max_steps;
  p.tol = r.tol;
  p.tol_bulk = r.tol_bulk;
  p.stream = nullptr;
  return p;
}

// Stream priority of a request: the highest for n <= 64, one level lower per
// doubling of n, clamped to the device's range.
int request_priority(const qfd_server_t sv, int64_t n) {
  int lvl = 0;
  for (int64_t m = n; m > 64; m >>= 1) ++lvl;
  return std::min(sv->prio_greatest + lvl, sv->prio_least);
}

void release_request(ReqRun* m) {
  if (m->st) cudaStreamSynchronize(m->st);
  if (m->plan) qfd_destroy(m->plan);
  if (m->exec) cudaGraphExecDestroy(m->exec);
  if (m->ev) cudaEventDestroy(m->ev);
  if (m->cohort) {
    auto& mem = m->cohort->members;
    mem.erase(std::remove(mem.begin(), mem.end(), m), mem.end());
  } else if (m->st) {
    cudaStreamDestroy(m->st);
  }
  delete m;
}

void destroy_cohort(Cohort* c) {
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->ev) cudaEventDestroy(c->ev);
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
}

// The cohort a newly admitted request of size n joins: one of that size with
// room, else a new one (its stream's priority as for a request of size n).
Cohort* cohort_for(qfd_server_t sv, int64_t n) {
  for (Cohort* c : sv->cohorts)
    if (c->n == n && (int)c->members.size() < QFD_MAX_BATCH) return c;
  Cohort* c = new Cohort();
  c->n = n;
  if (cudaStreamCreateWithPriority(&c->st, cudaStreamNonBlocking, request_priority(sv, n)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess) {
    destroy_cohort(c);
    return nullptr;
  }
  sv->cohorts.push_back(c);
  return c;
}

// Starts state `s` of a request: the complex64 bulk for mixed requests, else
// the plan's arithmetic.
qfd_status start_state(ReqRun* m, int s) {
  qfd_plan_t pl = m->plan;
  qfd_status r;
  m->state = s;
  m->tr = PhaseTracker{};
  m->fresh = true;
  pl->parity[s] = m->req.parity[s];
  pl->steps32[s] = pl->steps16[s] = 0;
  pl->ebulk[s] = NAN;
  pl->hist[s].clear();
  if (refines(pl->p.precision)) {
    m->bulk = true;
    m->phase = 1;
    if ((r = convert_state(pl, s, 1)) != QFD_OK) return r;
  } else {
    m->bulk = false;
    m->phase = uses32(pl->p.precision) ? 1 : pl->arith16;
  }
  pl->phase = m->phase;
  return with_policy(m->phase, [&](auto pol) -> qfd_status { return begin_phase<decltype(pol)>(pl, s); });
}

void finish_request(qfd_server_t sv, ReqRun* m, qfd_status status) {
  if (status != QFD_OK) m->res.status = status;
  m->res.t_done = server_clock(sv);
  m->res.nstates = m->req.nstates;
  sv->done.push_back(m->res);
}

// Launch shapes of a new request's plan when the server autotunes: those of
// the first plan of the same lattice size and precision, which is tuned once
// (qfd_autotune, before its states are filled).
qfd_status server_shapes(qfd_server_t sv, qfd_plan_t pl) {
  const std::pair<int64_t, int> key{pl->p.n, pl->p.precision};
  for (auto& e : sv->shapes) {
    if (e.first != key) continue;
    for (int q = 0; q < 3; ++q) {
      pl->tune_vy[q] = e.second[3 * q];
      pl->tune_vz[q] = e.second[3 * q + 1];
      pl->tune_vx[q] = e.second[3 * q + 2];
    }
    return QFD_OK;
  }
  qfd_status r = qfd_autotune(pl, nullptr);
  if (r != QFD_OK) return r;
  std::array<int, 9> v{};
  for (int q = 0; q < 3; ++q) {
    v[3 * q] = pl->tune_vy[q];
    v[3 * q + 1] = pl->tune_vz[q];
    v[3 * q + 2] = pl->tune_vx[q];
  }
  sv->shapes.push_back({key, v});
  return QFD_OK;
}

qfd_status admit(qfd_server_t sv) {
  while (!sv->waiting.empty()) {
    if (sv->p.max_active > 0 && (int)sv->active.size() >= sv->p.max_active) break;
    ReqRun* m = sv->waiting.front();
    qfd_params prm = request_params(sv, m->req);
    m->bytes = plan_device_bytes(prm);
    if (sv->used + m->bytes > (size_t)sv->p.hbm_budget_bytes) {
      if (!sv->active.empty()) break;  // wait for memory to free up
      sv->waiting.pop_front();         // can never fit the budget
      finish_request(sv, m, QFD_ERR_OOM);
      delete m;
      continue;
    }
    bool ok;
    cudaStream_t setup = nullptr;  // cohort mode: a new member is set up on a stream of its own
    if (sv->p.cohorts) {
      // the set-up synchronises its stream (derived coefficients are checked on
      // the host); on the cohort's stream it would wait for the period in flight
      m->cohort = cohort_for(sv, m->req.n);
      ok = m->cohort && cudaStreamCreateWithFlags(&setup, cudaStreamNonBlocking) == cudaSuccess &&
           cudaStreamWaitEvent(setup, sv->fork, 0) == cudaSuccess;
      if (ok) {
        m->st = setup;
        m->cohort->members.push_back(m);
      }
    } else {
      ok = cudaStreamCreateWithPriority(&m->st, cudaStreamNonBlocking, request_priority(sv, m->req.n)) == cudaSuccess &&
           cudaEventCreateWithFlags(&m->ev, cudaEventDisableTiming) == cudaSuccess &&
           cudaStreamWaitEvent(m->st, sv->fork, 0) == cudaSuccess;
    }
    // hands a cohort member's plan over from its set-up stream to the cohort's
    auto join_cohort = [&]() -> qfd_status {
      if (!setup) return QFD_OK;
      cudaEvent_t ev = nullptr;
      const bool good = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
                        cudaEventRecord(ev, setup) == cudaSuccess &&
                        cudaStreamWaitEvent(m->cohort->st, ev, 0) == cudaSuccess;
      if (ev) cudaEventDestroy(ev);
      cudaStreamDestroy(setup);  // released once its queued work is done
      setup = nullptr;
      m->st = m->cohort->st;
      if (m->plan) m->plan->st = m->st;
      return good ? QFD_OK : QFD_ERR_CUDA;
    };
    if (!ok) {
      join_cohort();
      sv->waiting.pop_front();
      finish_request(sv, m, QFD_ERR_CUDA);
      release_request(m);
      continue;
    }
    prm.stream = (void*)m->st;
    qfd_status r = qfd_plan(&prm, &m->plan);
    if (r == QFD_ERR_OOM && !sv->active.empty()) {  // retry once memory frees up
      if (m->cohort) {
        auto& mem = m->cohort->members;
        mem.erase(std::remove(mem.begin(), mem.end(), m), mem.end());
        m->cohort = nullptr;
        cudaStreamDestroy(setup);
      } else {
        cudaStreamDestroy(m->st);
        cudaEventDestroy(m->ev);
      }
      m->st = nullptr;
      m->ev = nullptr;
      break;
    }
    sv->waiting.pop_front();
    if (r == QFD_OK) {
      const double c[2] = {m->req.pot_coeffs[0], m->req.pot_coeffs[1]};
      r = qfd_fill_potential(m->plan, m->req.potential, c, 2);
      if (r == QFD_OK && sv->p.autotune) r = server_shapes(sv, m->plan);
      if (r == QFD_OK && m->req.grf_amplitude > 0)
        r = qfd_add_random_field(m->plan, m->req.grf_seed, m->req.grf_corr, m->req.grf_amplitude);
      for (int s = 0; r == QFD_OK && s < m->req.nstates; ++s) r = qfd_fill_psi_uniform(m->plan, s, m->req.seed + s);
      if (r == QFD_OK) r = start_state(m, 0);
    }
    const qfd_status rj = join_cohort();
    if (r == QFD_OK) r = rj;
    if (r != QFD_OK) {
      finish_request(sv, m, r);
      release_request(m);
      continue;
    }
    m->res.t_admit = server_clock(sv);
    sv->used += m->bytes;
    sv->active.push_back(m);
  }
  return QFD_OK;
}

// After a period: stop rule, then the next phase, state or completion.
qfd_status advance_request(ReqRun* m, bool* finished) {
  qfd_plan_t pl = m->plan;
  const int s = m->state;
  *finished = false;
  m->fresh = false;
  bool done = false;
  double e = NAN;
  qfd_status r = phase_check(pl, s, pl->hscal, m->bulk ? pl->p.tol_bulk : pl->p.tol, m->bulk, m->tr, &done, &e);
  if (r != QFD_OK) return r;
  if (!done && pl->t[s] < pl->p.max_steps) return QFD_OK;
  const bool converged = done;
  r = with_policy(m->phase, [&](auto pol) -> qfd_status { return finish_phase<decltype(pol)>(pl, s); });
  if (r != QFD_OK) return r;
  if (m->bulk) {  // hand the state over to the refinement arithmetic
    pl->steps32[s] = pl->t[s];
    pl->ebulk[s] = e;
    if ((r = convert_state(pl, s, 0)) != QFD_OK) return r;
    m->bulk = false;
    m->phase = pl->arith16;
    pl->phase = m->phase;
    m->tr = PhaseTracker{};
    m->fresh = true;
    return with_policy(m->phase, [&](auto pol) -> qfd_status { return begin_phase<decltype(pol)>(pl, s); });
  }
  if (m->phase == 1) pl->steps32[s] = pl->t[s];
  else pl->steps16[s] = pl->t[s];
  m->res.energy[s] = e;
  m->res.steps[s] = pl->steps32[s] + pl->steps16[s];
  m->res.steps_c64[s] = pl->steps32[s];
  if (!converged && pl->p.tol >= 0) m->res.status = QFD_ERR_NOT_CONVERGED;
  if (refines(pl->p.precision) && (r = convert_state(pl, s, 1)) != QFD_OK) return r;
  if (s + 1 < m->req.nstates) return start_state(m, s + 1);
  QFD_CK(cudaStreamSynchronize(pl->st));
  *finished = true;
  return QFD_OK;
}

// Queues one period of request m on its stream: directly for the first period
// of a phase (or without graphs), else by replaying - after capturing once -
// the graph of the period.  The device repeats the captured period; the host
// state advances as it did during the capture (only the step counter of the
// state changes between periods of a phase).
qfd_status issue_period(qfd_server_t sv, ReqRun* m) {
  qfd_plan_t pl = m->plan;
  const int64_t l0 = pl->launches;
  auto launch = [&]() -> qfd_status {
    qfd_status r = with_policy(m->phase, [&](auto pol) -> qfd_status {
      return period_launch<decltype(pol)>(pl, m->state, pl->hscal);
    });
    return r == QFD_OK ? r : sfail(sv, r, pl->err);
  };
  qfd_status r = QFD_OK;
  if (!sv->p.use_graphs || m->fresh) {
    r = launch();
    sv->kernels += pl->launches - l0;
  } else if (m->exec && m->gstate == m->state && m->gphase == m->phase) {
    if (cudaGraphLaunch(m->exec, m->st) != cudaSuccess) return sfail(sv, QFD_ERR_CUDA, "graph launch");
    pl->t[m->state] += pl->p.check_every;
    sv->kernels += m->exec_kernels;
    ++sv->replays;
  } else {
    if (m->exec) {
      cudaGraphExecDestroy(m->exec);
      m->exec = nullptr;
    }
    if (cudaStreamBeginCapture(m->st, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return sfail(sv, QFD_ERR_CUDA, "begin capture");
    r = launch();
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(m->st, &g);
    if (r != QFD_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (ce != cudaSuccess || !g) return sfail(sv, QFD_ERR_CUDA, "end capture");
    const cudaError_t ie = cudaGraphInstantiate(&m->exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      m->exec = nullptr;
      return sfail(sv, QFD_ERR_CUDA, "graph instantiate");
    }
    m->gstate = m->state;
    m->gphase = m->phase;
    m->exec_kernels = pl->launches - l0;
    sv->kernels += m->exec_kernels;
    if (cudaGraphLaunch(m->exec, m->st) != cudaSuccess) return sfail(sv, QFD_ERR_CUDA, "graph launch");
    ++sv->captures;
  }
  if (r != QFD_OK) return r;
  if (cudaEventRecord(m->ev, m->st) != cudaSuccess) return sfail(sv, QFD_ERR_CUDA, "event record");
  m->t_issue = std::chrono::steady_clock::now();
  m->inflight = true;
  ++sv->periods;
  return QFD_OK;
}

// The kernel sequence of one cohort period: per arithmetic, the members with
// an FFT kinetic term take batch_period_launch together (each pass one launch
// over them); H_K(0) members run period_launch one after the other.  All of it
// is on the cohort's stream, which is every member plan's stream.
qfd_status launch_cohort_period(qfd_server_t sv, Cohort* c) {
  for (int ph = 0; ph < 3; ++ph) {
    std::vector<qfd_plan_s*> pls;
    std::vector<int> ss;
    for (ReqRun* m : c->running) {
      if (m->phase != ph) continue;
      qfd_plan_t pl = m->plan;
      if (pl->p.kinetic == 0) {
        const qfd_status r = with_policy(ph, [&](auto pol) -> qfd_status {
          return period_launch<decltype(pol)>(pl, m->state, pl->hscal);
        });
        if (r != QFD_OK) return sfail(sv, r, pl->err);
      } else {
        pls.push_back(pl);
        ss.push_back(m->state);
      }
    }
    if (pls.empty()) continue;
    const qfd_status r = with_policy(ph, [&](auto pol) -> qfd_status {
      return batch_period_launch<decltype(pol)>(pls.data(), ss.data(), (int)pls.size(), c->st);
    });
    if (r != QFD_OK) return sfail(sv, r, pls[0]->err);
  }
  return QFD_OK;
}

// Queues one period of every member of cohort c: directly while a member is
// in the first period of its phase (or without graphs), else by replaying -
// after capturing once - the graph of the cohort period, which stays valid
// while the members and their states and phases are the same (the host state
// of each member then advances by its step counter only, as for a request's
// own graph).
qfd_status issue_cohort_period(qfd_server_t sv, Cohort* c) {
  c->running = c->members;
  auto launched = [&]() {
    int64_t k = 0;
    for (ReqRun* m : c->running) k += m->plan->launches;
    return k;
  };
  const int64_t l0 = launched();
  bool any_fresh = false;
  std::vector<int64_t> sig;
  for (ReqRun* m : c->running) {
    any_fresh = any_fresh || m->fresh;
    sig.push_back(m->id);
    sig.push_back(m->state);
    sig.push_back(m->phase);
  }
  qfd_status r = QFD_OK;
  if (!sv->p.use_graphs || any_fresh) {
    r = launch_cohort_period(sv, c);
    sv->kernels += launched() - l0;
  } else if (c->exec && c->sig == sig) {
    if (cudaGraphLaunch(c->exec, c->st) != cudaSuccess) return sfail(sv, QFD_ERR_CUDA, "graph launch");
    for (ReqRun* m : c->running) m->plan->t[m->state] += m->plan->p.check_every;
    sv->kernels += c->exec_kernels;
    ++sv->replays;
  } else {
    if (c->exec) {
      cudaGraphExecDestroy(c->exec);
      c->exec = nullptr;
    }
    if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return sfail(sv, QFD_ERR_CUDA, "begin capture");
    r = launch_cohort_period(sv, c);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c->st, &g);
    if (r != QFD_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (ce != cudaSuccess || !g) return sfail(sv, QFD_ERR_CUDA, "end capture");
    const cudaError_t ie = cudaGraphInstantiate(&c->exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      c->exec = nullptr;
      return sfail(sv, QFD_ERR_CUDA, "graph instantiate");
    }
    c->sig = sig;
    c->exec_kernels = launched() - l0;
    sv->kernels += c->exec_kernels;
    if (cudaGraphLaunch(c->exec, c->st) != cudaSuccess) return sfail(sv, QFD_ERR_CUDA, "graph launch");
    ++sv->captures;
  }
  if (r != QFD_OK) return r;
  if (cudaEventRecord(c->ev, c->st) != cudaSuccess) return sfail(sv, QFD_ERR_CUDA, "event record");
  c->t_issue = std::chrono::steady_clock::now();
  c->inflight = true;
  sv->periods += (int64_t)c->running.size();
  return QFD_OK;
}

// Ends request m (finished, failed or timed out): result, budget, memory.
void retire_request(qfd_server_t sv, ReqRun* m, qfd_status status) {
  finish_request(sv, m, status);
  sv->used -= m->bytes;
  sv->active.erase(std::remove(sv->active.begin(), sv->active.end(), m), sv->active.end());
  release_request(m);
}

// run_periods in cohort mode: a period for every cohort without one in
// flight, a wait (bounded by the watchdog) until one has ended, then the stop
// rule and the next phase, state or completion of each of its members.
qfd_status run_cohort_periods(qfd_server_t sv) {
  std::vector<std::pair<Cohort*, qfd_status>> ended;  // QFD_OK: the period completed
  for (Cohort* c : sv->cohorts) {
    if (c->inflight || c->members.empty()) continue;
    const qfd_status r = issue_cohort_period(sv, c);
    if (r != QFD_OK) ended.push_back({c, r});
  }
  while (ended.empty()) {
    bool waiting_any = false;
    const auto now = std::chrono::steady_clock::now();
    for (Cohort* c : sv->cohorts) {
      if (!c->inflight) continue;
      waiting_any = true;
      const cudaError_t q = cudaEventQuery(c->ev);
      if (q == cudaSuccess) {
        c->inflight = false;
        ended.push_back({c, QFD_OK});
      } else if (q != cudaErrorNotReady) {
        return sfail(sv, QFD_ERR_CUDA, cudaGetErrorString(q));
      } else if (sv->timeout_s > 0 && std::chrono::duration<double>(now - c->t_issue).count() > sv->timeout_s) {
        c->inflight = false;
        ended.push_back({c, QFD_ERR_TIMEOUT});
      }
    }
    if (!waiting_any || !ended.empty()) break;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  for (auto& e : ended) {
    Cohort* c = e.first;
    const std::vector<ReqRun*> running = c->running;
    c->running.clear();
    for (ReqRun* m : running) {
      if (e.second != QFD_OK) {
        m->res.status = e.second;
        retire_request(sv, m, e.second);
        continue;
      }
      bool finished = false;
      const qfd_status q = advance_request(m, &finished);
      if (q != QFD_OK || finished) retire_request(sv, m, q);
    }
  }
  // cohorts left without members and work in flight are released
  std::vector<Cohort*> keep;
  for (Cohort* c : sv->cohorts) {
    if (c->members.empty() && !c->inflight) destroy_cohort(c);
    else keep.push_back(c);
  }
  sv->cohorts.swap(keep);
  return QFD_OK;
}

// Issues a period for every active request without one in flight, waits until
// at least one period has ended, and retires the requests whose periods ended.
// With a watchdog set, the wait is bounded: a period still in flight that long
// after it was queued ends its request with QFD_ERR_TIMEOUT (release_request
// then waits for the work already queued on the request's stream before its
// memory is freed).
qfd_status run_periods(qfd_server_t sv) {
  if (sv->p.cohorts) return run_cohort_periods(sv);
  std::vector<ReqRun*> keep;
  std::vector<char> ended(sv->active.size(), 0);
  bool any_ended = false;
  for (size_t i = 0; i < sv->active.size(); ++i) {
    ReqRun* m = sv->active[i];
    if (m->inflight) continue;
    const qfd_status r = issue_period(sv, m);
    if (r != QFD_OK) {  // the request ends with the error; the others go on
      m->res.status = r;
      ended[i] = 2;
      any_ended = true;
    }
  }
  while (!any_ended) {
    bool waiting_any = false;
    const auto now = std::chrono::steady_clock::now();
    for (size_t i = 0; i < sv->active.size(); ++i) {
      ReqRun* m = sv->active[i];
      if (!m->inflight) continue;
      waiting_any = true;
      const cudaError_t q = cudaEventQuery(m->ev);
      if (q == cudaSuccess) {
        m->inflight = false;
        ended[i] = 1;
        any_ended = true;
      } else if (q != cudaErrorNotReady) {
        return sfail(sv, QFD_ERR_CUDA, cudaGetErrorString(q));
      } else if (sv->timeout_s > 0 &&
                 std::chrono::duration<double>(now - m->t_issue).count() > sv->timeout_s) {
        m->inflight = false;
        m->res.status = QFD_ERR_TIMEOUT;
        ended[i] = 2;
        any_ended = true;
      }
    }
    if (!waiting_any || any_ended) break;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  for (size_t i = 0; i < sv->active.size(); ++i) {
    ReqRun* m = sv->active[i];
    bool finished = ended[i] == 2;
    qfd_status q = finished ? (qfd_status)m->res.status : QFD_OK;
    if (ended[i] == 1) {
      q = advance_request(m, &finished);
      if (q != QFD_OK) finished = true;
    }
    if (finished) {
      finish_request(sv, m, q);
      sv->used -= m->bytes;
      release_request(m);
    } else {
      keep.push_back(m);
    }
  }
  sv->active.swap(keep);
  return QFD_OK;
}

}  // namespace

extern "C" {

size_t qfd_plan_bytes(const qfd_params* p) { return p ? plan_device_bytes(*p) : 0; }

qfd_status qfd_server_create(const qfd_server_params* params, qfd_server_t* out) {
  if (out) *out = nullptr;
  if (!params || !out || !(params->hbm_budget_bytes > 0) || params->ortho_every < 1 || params->check_every < 1 ||
      params->check_every % params->ortho_every != 0 || params->max_active < 0 ||
      (params->cohorts != 0 && params->cohorts != 1) || (params->autotune != 0 && params->autotune != 1))
    return QFD_ERR_ARG;
  qfd_server_t sv = new qfd_server_s();
  sv->p = *params;
  if (params->stream) {
    sv->st = (cudaStream_t)params->stream;
  } else if (cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete sv;
    return QFD_ERR_CUDA;
  } else {
    sv->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&sv->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaDeviceGetStreamPriorityRange(&sv->prio_least, &sv->prio_greatest) != cudaSuccess) {
    qfd_server_destroy(sv);
    return QFD_ERR_CUDA;
  }
  *out = sv;
  return QFD_OK;
}

void qfd_server_destroy(qfd_server_t sv) {
  if (!sv) return;
  if (sv->st) cudaStreamSynchronize(sv->st);
  for (ReqRun* m : sv->active) release_request(m);
  for (ReqRun* m : sv->waiting) delete m;
  for (Cohort* c : sv->cohorts) destroy_cohort(c);
  if (sv->fork) cudaEventDestroy(sv->fork);
  if (sv->own_stream && sv->st) cudaStreamDestroy(sv->st);
  delete sv;
}

const char* qfd_server_last_error(qfd_server_t sv) { return sv ? sv->err.c_str() : ""; }

double qfd_server_clock(qfd_server_t sv) { return sv ? server_clock(sv) : 0.0; }

qfd_status qfd_server_submit(qfd_server_t sv, const qfd_request* req, int64_t* id) {
  if (!sv || !req) return QFD_ERR_ARG;
  if (req->nstates < 1 || req->nstates > MAX_LOWER || !supported_n(req->n))
    return sfail(sv, QFD_ERR_ARG, "request: nstates 1..8 and a supported n");
  for (int s = 0; s < req->nstates; ++s)
    if (req->parity[s] < -1 || req->parity[s] > 1) return sfail(sv, QFD_ERR_ARG, "request: parity -1, 0 or 1");
  ReqRun* m = new ReqRun();
  m->id = sv->next_id++;
  m->req = *req;
  m->res.id = m->id;
  m->res.status = QFD_OK;
  m->res.nstates = req->nstates;
  m->res.t_submit = server_clock(sv);
  for (int s = 0; s < 8; ++s) m->res.energy[s] = NAN;
  sv->waiting.push_back(m);
  if (id) *id = m->id;
  return QFD_OK;
}

qfd_status qfd_server_poll(qfd_server_t sv, qfd_result* out, int capacity, int* count) {
  if (!sv || capacity < 0 || (capacity > 0 && !out)) return QFD_ERR_ARG;
  if (!sv->waiting.empty() && cudaEventRecord(sv->fork, sv->st) != cudaSuccess)
    return sfail(sv, QFD_ERR_CUDA, "fork event");
  qfd_status r = admit(sv);
  if (r == QFD_OK && !sv->active.empty()) r = run_periods(sv);
  const int n = (int)std::min<size_t>(sv->done.size(), (size_t)capacity);
  for (int i = 0; i < n; ++i) out[i] = sv->done[i];
  sv->done.erase(sv->done.begin(), sv->done.begin() + n);
  if (count) *count = n;
  return r;
}

qfd_status qfd_server_kernels(qfd_server_t sv, int64_t* kernels) {
  if (!sv || !kernels) return QFD_ERR_ARG;
  *kernels = sv->kernels;
  return QFD_OK;
}

qfd_status qfd_server_set_timeout(qfd_server_t sv, double seconds) {
  if (!sv) return QFD_ERR_ARG;
  if (!(seconds >= 0.0) || !std::isfinite(seconds)) return sfail(sv, QFD_ERR_ARG, "timeout must be finite and >= 0");
  sv->timeout_s = seconds;
  return QFD_OK;
}

qfd_status qfd_server_stats(qfd_server_t sv, int* waiting, int* active, double* used_bytes, int64_t* periods,
                            int64_t* graph_replays, int64_t* graph_captures) {
  if (!sv) return QFD_ERR_ARG;
  if (waiting) *waiting = (int)sv->waiting.size();
  if (active) *active = (int)sv->active.size();
  if (used_bytes) *used_bytes = (double)sv->used;
  if (periods) *periods = sv->periods;
  if (graph_replays) *graph_replays = sv->replays;
  if (graph_captures) *graph_captures = sv->captures;
  return QFD_OK;
}

}  // extern "C"

namespace qfd {
bool supported_n(int64_t n) {
  return n == 8 || n == 16 || n == 32 || n == 64 || n == 96 || n == 128 || n == 192 || n == 256 || n == 512 ||
         n == 1024;
}
}  // namespace qfd
