// Launcher bodies of Launch<A, N>; included by qfd_inst.cu, which the build
// compiles once per (arithmetic policy, lattice size) pair.
#pragma once

#include "qfd_kernels.cuh"
#include "qfd_launch.h"

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
  using C = typename A::C;
  using VT = typename A::VT;
  using SH = Shape<A, N>;
  const size_t smem = (size_t)N * SH::XPITCH * sizeof(C);
  const int grid = (int)((int64_t)N * N / SH::XCOLS);
  auto go = [&](auto kern) {
    ensure_smem(kern, smem);
    kern<<<grid, SH::XTHREADS, smem, a.stream>>>((C*)a.W, (C*)a.psi, (const typename A::K*)a.coef, (const VT*)a.V,
                                                  a.scale, a.scale_f, (const C*)a.tw, a.part);
  };
  if (a.stats == STATS_FULL) go(k_update_x<A, N, STATS_FULL>);
  else if (a.stats == STATS_NORM) go(k_update_x<A, N, STATS_NORM>);
  else go(k_update_x<A, N, STATS_NONE>);
  if (nblocks) *nblocks = grid;
  return cudaGetLastError();
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
  using C = typename A::C;
  using SH = Shape<A, N>;
  auto go = [&](auto kern, int yc) {
    const size_t smem = (size_t)N * yc * sizeof(C);
    const int tiles_inner = N / yc;
    ensure_smem(kern, smem);
    kern<<<N * tiles_inner, SH::T * yc, smem, a.stream>>>((C*)a.W, (const C*)a.tw, (int64_t)N, tiles_inner,
                                                          (int64_t)N * N);
  };
  if (a.vy == 1) {
    if (dir < 0) go(k_fft_strided<A, N, -1, SH::YCOLS2>, SH::YCOLS2);
    else go(k_fft_strided<A, N, +1, SH::YCOLS2>, SH::YCOLS2);
  } else {
    if (dir < 0) go(k_fft_strided<A, N, -1>, SH::YCOLS);
    else go(k_fft_strided<A, N, +1>, SH::YCOLS);
  }
  return cudaGetLastError();
}

template <class A, int N>
cudaError_t Launch<A, N>::zpass(const LaunchArgs& a, int* nblocks) {
  using C = typename A::C;
  using SH = Shape<A, N>;
  const size_t smem = (size_t)SH::LINES * SH::LPAD * sizeof(C);
  // z-pass line groups: the policy's default, or the autotuner's 1 / 2
  const int zg = a.vz == 0 ? 1 : a.vz == 1 ? SH::ZG2 : SH::ZG;
  const int grid = (int)((int64_t)N * N / (SH::LINES * zg));
  auto go = [&](auto kern) {
    ensure_smem(kern, smem);
    kern<<<grid, SH::LINE_THREADS, smem, a.stream>>>((C*)a.W, (const C*)a.tw, (const typename A::T*)a.ktab, *a.kin,
                                                      a.part);
  };
  if (zg == 1) {
    if (a.stats) go(k_zpass<A, N, true, 1>);
    else go(k_zpass<A, N, false, 1>);
  } else if (zg == SH::ZG2) {
    if (a.stats) go(k_zpass<A, N, true, SH::ZG2>);
    else go(k_zpass<A, N, false, SH::ZG2>);
  } else {
    if (a.stats) go(k_zpass<A, N, true>);
    else go(k_zpass<A, N, false>);
  }
  if (nblocks) *nblocks = grid;
  return cudaGetLastError();
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
cudaError_t Launch<A, N>::fft_y_batch(const BatchY& b, int count, int dir, cudaStream_t st) {
  if constexpr (N > MAX_BATCH_N) {
    return cudaErrorInvalidValue;
  } else {
    using SH = Shape<A, N>;
    constexpr int yc = SH::YCOLS;
    const size_t smem = (size_t)N * yc * sizeof(typename A::C);
    const int tiles_inner = N / yc;
    auto go = [&](auto kern) {
      ensure_smem(kern, smem);
      kern<<<dim3(N * tiles_inner, count), SH::T * yc, smem, st>>>(b, (int64_t)N, tiles_inner, (int64_t)N * N);
    };
    if (dir < 0) go(k_fft_strided_batch<A, N, -1>);
    else go(k_fft_strided_batch<A, N, +1>);
    return cudaGetLastError();
  }
}

template <class A, int N>
cudaError_t Launch<A, N>::zpass_batch(const BatchZ& b, int count, cudaStream_t st) {
  if constexpr (N > MAX_BATCH_N) {
    return cudaErrorInvalidValue;
  } else {
    using SH = Shape<A, N>;
    const size_t smem = (size_t)SH::LINES * SH::LPAD * sizeof(typename A::C);
    const int grid = (int)((int64_t)N * N / (SH::LINES * SH::ZG));
    auto kern = k_zpass_batch<A, N>;
    ensure_smem(kern, smem);
    kern<<<dim3(grid, count), SH::LINE_THREADS, smem, st>>>(b);
    return cudaGetLastError();
  }
}

template <class A, int N>
cudaError_t Launch<A, N>::update_x_batch(const BatchU& b, int count, uint32_t scaled, int stats, cudaStream_t st,
                                         int* nblocks) {
  if constexpr (N > MAX_BATCH_N) {
    return cudaErrorInvalidValue;
  } else {
    using SH = Shape<A, N>;
    const size_t smem = (size_t)N * SH::XPITCH * sizeof(typename A::C);
    const int grid = (int)((int64_t)N * N / SH::XCOLS);
    auto go = [&](auto kern) {
      ensure_smem(kern, smem);
      kern<<<dim3(grid, count), SH::XTHREADS, smem, st>>>(b, scaled);
    };
    if (stats == STATS_NORM) go(k_update_x_batch<A, N, STATS_NORM>);
    else go(k_update_x_batch<A, N, STATS_NONE>);
    if (nblocks) *nblocks = grid;
    return cudaGetLastError();
  }
}

template <class A, int N>
int Launch<A, N>::partials() {
  using SH = Shape<A, N>;
  const int x = (int)((int64_t)N * N / SH::XCOLS);
  const int z = (int)((int64_t)N * N / SH::LINES);  // bounds the persistent z-pass grid too
  return x > z ? x : z;
}

}  // namespace qfd
