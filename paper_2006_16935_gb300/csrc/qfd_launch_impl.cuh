// Launcher bodies of Launch<A, N>; included by qfd_inst.cu, which the build
// compiles once per (arithmetic policy, lattice size) pair.
#pragma once

#include "qfd_kernels.cuh"
#include "qfd_launch.h"
#include "qfd_tma.cuh"

namespace qfd {

// Opts in to more than the default 48 KB of shared memory per CTA when the
// dynamic part, together with the kernels' static reduction buffers (a few
// KB), could exceed it.
template <class K>
static void ensure_smem(K kern, size_t bytes) {
  if (bytes > 40 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class A, int N>
cudaError_t Launch<A, N>::update_x(const LaunchArgs& a, int* nblocks) {
  BatchU b{};
  b.W[0] = a.W;
  b.psi[0] = a.psi;
  b.u[0] = a.coef;
  b.V[0] = a.V;
  b.scale[0] = a.scale;
  b.scale_f[0] = a.scale_f;
  b.tw[0] = a.tw;
  b.part[0] = a.part;
  if (a.up) b.up[0] = *a.up;
  for (int j = 0; j < 3; ++j) b.tmap[0][j] = a.tmap[j];
  b.err[0] = a.err;
  return update_x_batch(b, 1, a.scale ? 1u : 0u, a.stats, a.vx, a.stream, nblocks, a.tma_test);
}

template <class A, int N>
int Launch<A, N>::tma_xt() {
  return TmaShape<A, N>::OK ? TmaShape<A, N>::XT : 0;
}

template <class A, int N>
cudaError_t Launch<A, N>::forward_x(const LaunchArgs& a, int* nblocks) {
  using C = typename A::C;
  using VT = typename A::VT;
  using SH = Shape<A, N>;
  const size_t smem = (size_t)N * SH::XPITCH * sizeof(C);
  const int grid = (int)((int64_t)N * N / SH::XCOLS);
  auto go = [&](auto kern) {
    ensure_smem(kern, smem);
    kern<<<grid, SH::XTHREADS, smem, a.stream>>>((const C*)a.src, (C*)a.W, (C*)a.psi_out, (const VT*)a.V, a.scale,
                                                  a.scale_f, (const C*)a.tw, a.part);
  };
  if (a.stats == STATS_FULL) go(k_forward_x<A, N, STATS_FULL>);
  else if (a.stats == STATS_NORM) go(k_forward_x<A, N, STATS_NORM>);
  else go(k_forward_x<A, N, STATS_NONE>);
  if (nblocks) *nblocks = grid;
  return cudaGetLastError();
}

template <class A, int N>
cudaError_t Launch<A, N>::fft_y(const LaunchArgs& a, int dir) {
  BatchY b{};
  b.W[0] = a.W;
  b.tw[0] = a.tw;
  return fft_y_batch(b, 1, dir, a.vy, a.stream);
}

template <class A, int N>
cudaError_t Launch<A, N>::zpass(const LaunchArgs& a, int* nblocks) {
  BatchZ b{};
  b.W[0] = a.W;
  b.tw[0] = a.tw;
  b.ktab[0] = a.ktab;
  b.part[0] = a.part;
  b.kp[0] = *a.kin;
  return zpass_batch(b, 1, a.stats, a.vz, a.stream, nblocks);
}

template <class A, int N>
cudaError_t Launch<A, N>::project_x(const LaunchArgs& a, int* nblocks) {
  using C = typename A::C;
  using VT = typename A::VT;
  using SH = Shape<A, N>;
  const size_t smem = (size_t)N * SH::XPITCH * sizeof(C);
  const int grid = (int)((int64_t)N * N / SH::XCOLS);
  LowerPtrs lp;
  for (int j = 0; j < MAX_LOWER; ++j) lp.p[j] = a.lower[j];
  auto go = [&](auto kern) {
    ensure_smem(kern, smem);
    kern<<<grid, SH::XTHREADS, smem, a.stream>>>((const C*)a.src, lp, a.sums, a.k, a.parity, a.offgrid,
                                                      (C*)a.dst, (C*)a.W, (const VT*)a.V, (const C*)a.tw, a.part);
  };
  if (a.k > 0) {
    if (a.stats == STATS_FULL) go(k_project_x<A, N, STATS_FULL, true>);
    else go(k_project_x<A, N, STATS_NORM, true>);
  } else {
    if (a.stats == STATS_FULL) go(k_project_x<A, N, STATS_FULL, false>);
    else go(k_project_x<A, N, STATS_NORM, false>);
  }
  if (nblocks) *nblocks = grid;
  return cudaGetLastError();
}

template <class A, int N>
cudaError_t Launch<A, N>::gs_dots(const LaunchArgs& a, int nblocks) {
  LowerPtrs lp;
  for (int j = 0; j < MAX_LOWER; ++j) lp.p[j] = a.lower[j];
  k_gs_dots<A, N><<<nblocks, 256, 0, a.stream>>>((const typename A::C*)a.src, lp, a.k, a.parity, a.offgrid, a.part);
  return cudaGetLastError();
}

template <class A, int N>
cudaError_t Launch<A, N>::fft_y_batch(const BatchY& b, int count, int dir, int vy, cudaStream_t st) {
  using C = typename A::C;
  using SH = Shape<A, N>;
  auto go = [&](auto kern, int yc, int tpc) {
    const size_t smem = (size_t)N * yc * sizeof(C);
    const int tiles_inner = N / yc;
    ensure_smem(kern, smem);
    kern<<<dim3(N * tiles_inner, count), tpc * yc, smem, st>>>(b, (int64_t)N, tiles_inner,
                                                                          (int64_t)N * N);
  };
  if constexpr (SH::HAS_R1) {
    if (vy == 2) {  // the two-stage radix schedule
      if (dir < 0) go(k_fft_strided<A, N, -1, SH::YCOLS_R1, 1>, SH::YCOLS_R1, SH::T1);
      else go(k_fft_strided<A, N, +1, SH::YCOLS_R1, 1>, SH::YCOLS_R1, SH::T1);
      return cudaGetLastError();
    }
  }
  if (vy == 1) {
    if (dir < 0) go(k_fft_strided<A, N, -1, SH::YCOLS2>, SH::YCOLS2, SH::T);
    else go(k_fft_strided<A, N, +1, SH::YCOLS2>, SH::YCOLS2, SH::T);
  } else {
    if (dir < 0) go(k_fft_strided<A, N, -1, SH::YCOLS>, SH::YCOLS, SH::T);
    else go(k_fft_strided<A, N, +1, SH::YCOLS>, SH::YCOLS, SH::T);
  }
  return cudaGetLastError();
}

template <class A, int N>
cudaError_t Launch<A, N>::zpass_batch(const BatchZ& b, int count, int parseval, int vz, cudaStream_t st,
                                      int* nblocks) {
  using C = typename A::C;
  using SH = Shape<A, N>;
  if constexpr (SH::HAS_R1) {
    if (vz == 2) {  // the two-stage radix schedule, one line group
      const size_t smem = (size_t)SH::LINES_R1 * SH::LPAD_R1 * sizeof(C);
      const int grid = (int)((int64_t)N * N / SH::LINES_R1);
      auto go1 = [&](auto kern) {
        ensure_smem(kern, smem);
        kern<<<dim3(grid, count), SH::T1 * SH::LINES_R1, smem, st>>>(b);
      };
      if (parseval) go1(k_zpass<A, N, true, 1, 1>);
      else go1(k_zpass<A, N, false, 1, 1>);
      if (nblocks) *nblocks = grid;
      return cudaGetLastError();
    }
  }
  const size_t smem = (size_t)SH::LINES * SH::LPAD * sizeof(C);
  // z-pass line groups: the policy's default, or the autotuner's 1 / 2
  const int zg = vz == 0 ? 1 : vz == 1 ? SH::ZG2 : SH::ZG;
  const int grid = (int)((int64_t)N * N / (SH::LINES * zg));
  auto go = [&](auto kern) {
    ensure_smem(kern, smem);
    kern<<<dim3(grid, count), SH::LINE_THREADS, smem, st>>>(b);
  };
  if (zg == 1) {
    if (parseval) go(k_zpass<A, N, true, 1>);
    else go(k_zpass<A, N, false, 1>);
  } else {
    if (parseval) go(k_zpass<A, N, true, SH::ZG2>);
    else go(k_zpass<A, N, false, SH::ZG2>);
  }
  if (nblocks) *nblocks = grid;
  return cudaGetLastError();
}

template <class A, int N>
cudaError_t Launch<A, N>::update_x_batch(const BatchU& b, int count, uint32_t scaled, int stats, int vx,
                                         cudaStream_t st, int* nblocks, int tma_test) {
  using C = typename A::C;
  using SH = Shape<A, N>;
  if constexpr (TmaShape<A, N>::OK) {
    // the TMA variant needs every lattice's tensor maps and error flag: without
    // them the default width runs
    for (int i = 0; i < count && vx == 2; ++i)
      if (!b.tmap[i][0] || !b.tmap[i][1] || !b.tmap[i][2] || !b.err[i]) vx = 0;
    if (vx == 2) {  // the TMA-staged persistent pass A: one CTA per SM and lattice
      using TS = TmaShape<A, N>;
      int dev = 0, sms = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      constexpr int NT = N * N / TS::XT;
      const int grid = sms < NT ? sms : NT;
      auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TS::SMEM);
        kern<<<dim3(grid, count), TS::THREADS, TS::SMEM, st>>>(b, scaled, tma_test);
      };
      if (stats == STATS_FULL) go(k_update_x_tma<A, N, STATS_FULL>);
      else if (stats == STATS_NORM) go(k_update_x_tma<A, N, STATS_NORM>);
      else go(k_update_x_tma<A, N, STATS_NONE>);
      if (nblocks) *nblocks = grid;
      return cudaGetLastError();
    }
  }
  auto go = [&](auto kern, int xc) {
    const size_t smem = (size_t)N * xc * sizeof(C);
    const int grid = (int)((int64_t)N * N / xc);
    ensure_smem(kern, smem);
    kern<<<dim3(grid, count), SH::T * xc, smem, st>>>(b, scaled);
    if (nblocks) *nblocks = grid;
  };
  if (vx == 1) {
    constexpr int XC = SH::XCOLS2;
    if (stats == STATS_FULL) go(k_update_x<A, N, STATS_FULL, XC>, XC);
    else if (stats == STATS_NORM) go(k_update_x<A, N, STATS_NORM, XC>, XC);
    else go(k_update_x<A, N, STATS_NONE, XC>, XC);
  } else {
    constexpr int XC = SH::XCOLS;
    if (stats == STATS_FULL) go(k_update_x<A, N, STATS_FULL, XC>, XC);
    else if (stats == STATS_NORM) go(k_update_x<A, N, STATS_NORM, XC>, XC);
    else go(k_update_x<A, N, STATS_NONE, XC>, XC);
  }
  return cudaGetLastError();
}

template <class A, int N>
int Launch<A, N>::partials() {
  using SH = Shape<A, N>;
  const int x = (int)((int64_t)N * N / SH::XCOLS2);  // pass A's half-width tiles
  const int z1 = (int)((int64_t)N * N / SH::LINES_R1);  // the two-stage z pass
  const int z = (int)((int64_t)N * N / SH::LINES);
  const int m = x > z ? x : z;
  return SH::HAS_R1 && z1 > m ? z1 : m;
}

}  // namespace qfd
