// Launcher bodies, included once per arithmetic type by qfd_k64.cu / qfd_k32.cu.
#pragma once

#include <type_traits>

#include "qfd_kernels.cuh"
#include "qfd_launch.h"

namespace qfd {

template <class F>
static bool dispatch_n(int64_t n, F&& f) {
  switch (n) {
    case 8: f(std::integral_constant<int, 8>()); return true;
    case 16: f(std::integral_constant<int, 16>()); return true;
    case 32: f(std::integral_constant<int, 32>()); return true;
    case 64: f(std::integral_constant<int, 64>()); return true;
    case 128: f(std::integral_constant<int, 128>()); return true;
    case 256: f(std::integral_constant<int, 256>()); return true;
    case 512: f(std::integral_constant<int, 512>()); return true;
    case 1024: f(std::integral_constant<int, 1024>()); return true;
    default: return false;
  }
}

template <class K>
static void ensure_smem(K kern, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R>
cudaError_t launch_update_x(const LaunchArgs& a, int* nblocks) {
  using C = typename CxT<R>::T;
  cudaError_t err = cudaErrorInvalidValue;
  dispatch_n(a.n, [&](auto nc) {
    constexpr int N = decltype(nc)::value;
    using SH = Shape<R, N>;
    const size_t smem = (size_t)N * SH::COLS * sizeof(C);
    auto kern = k_update_x<R, N>;
    ensure_smem(kern, smem);
    const int grid = (int)((int64_t)N * N / SH::COLS);
    kern<<<grid, SH::TILE_THREADS, smem, a.stream>>>(
        (C*)a.W, (C*)a.psi, (const typename Coef<R>::T*)a.coef, a.V, a.scale, (const C*)a.tw, a.part, a.check);
    if (nblocks) *nblocks = grid;
    err = cudaGetLastError();
  });
  return err;
}

template <typename R>
cudaError_t launch_forward_x(const LaunchArgs& a, int* nblocks) {
  using C = typename CxT<R>::T;
  cudaError_t err = cudaErrorInvalidValue;
  dispatch_n(a.n, [&](auto nc) {
    constexpr int N = decltype(nc)::value;
    using SH = Shape<R, N>;
    const size_t smem = (size_t)N * SH::COLS * sizeof(C);
    auto kern = k_forward_x<R, N>;
    ensure_smem(kern, smem);
    const int grid = (int)((int64_t)N * N / SH::COLS);
    kern<<<grid, SH::TILE_THREADS, smem, a.stream>>>((const C*)a.src, (C*)a.W, (C*)a.psi_out, a.V, a.scale,
                                                      (const C*)a.tw, a.part, a.check);
    if (nblocks) *nblocks = grid;
    err = cudaGetLastError();
  });
  return err;
}

template <typename R>
cudaError_t launch_fft_y(const LaunchArgs& a, int dir) {
  using C = typename CxT<R>::T;
  cudaError_t err = cudaErrorInvalidValue;
  dispatch_n(a.n, [&](auto nc) {
    constexpr int N = decltype(nc)::value;
    using SH = Shape<R, N>;
    const size_t smem = (size_t)N * SH::COLS * sizeof(C);
    const int tiles_inner = N / SH::COLS;
    const int grid = N * tiles_inner;
    if (dir < 0) {
      auto kern = k_fft_strided<R, N, -1>;
      ensure_smem(kern, smem);
      kern<<<grid, SH::TILE_THREADS, smem, a.stream>>>((C*)a.W, (const C*)a.tw, (int64_t)N, tiles_inner,
                                                        (int64_t)N * N);
    } else {
      auto kern = k_fft_strided<R, N, +1>;
      ensure_smem(kern, smem);
      kern<<<grid, SH::TILE_THREADS, smem, a.stream>>>((C*)a.W, (const C*)a.tw, (int64_t)N, tiles_inner,
                                                        (int64_t)N * N);
    }
    err = cudaGetLastError();
  });
  return err;
}

template <typename R>
cudaError_t launch_fft_x_plain(const LaunchArgs& a, int dir) {
  using C = typename CxT<R>::T;
  cudaError_t err = cudaErrorInvalidValue;
  dispatch_n(a.n, [&](auto nc) {
    constexpr int N = decltype(nc)::value;
    using SH = Shape<R, N>;
    const size_t smem = (size_t)N * SH::COLS * sizeof(C);
    const int tiles_inner = N * N / SH::COLS;
    if (dir < 0) {
      auto kern = k_fft_strided<R, N, -1>;
      ensure_smem(kern, smem);
      kern<<<tiles_inner, SH::TILE_THREADS, smem, a.stream>>>((C*)a.W, (const C*)a.tw, (int64_t)N * N,
                                                               tiles_inner, 0);
    } else {
      auto kern = k_fft_strided<R, N, +1>;
      ensure_smem(kern, smem);
      kern<<<tiles_inner, SH::TILE_THREADS, smem, a.stream>>>((C*)a.W, (const C*)a.tw, (int64_t)N * N,
                                                               tiles_inner, 0);
    }
    err = cudaGetLastError();
  });
  return err;
}

template <typename R>
cudaError_t launch_zpass(const LaunchArgs& a, int* nblocks) {
  using C = typename CxT<R>::T;
  cudaError_t err = cudaErrorInvalidValue;
  dispatch_n(a.n, [&](auto nc) {
    constexpr int N = decltype(nc)::value;
    using SH = Shape<R, N>;
    constexpr int LINES = SH::LINES;
    const size_t smem = (size_t)LINES * SH::LPAD * sizeof(C);
    auto kern = k_zpass<R, N>;
    ensure_smem(kern, smem);
    const int grid = (int)((int64_t)N * N / LINES);
    kern<<<grid, SH::LINE_THREADS, smem, a.stream>>>((C*)a.W, (const C*)a.tw, (const R*)a.ktab,
                                                      *(const KinParams*)a.kin, a.part, a.check);
    if (nblocks) *nblocks = grid;
    err = cudaGetLastError();
  });
  return err;
}

template <typename R>
cudaError_t launch_gs_dots(const void* psi, const void* lower, int k, int parity, int offgrid, int64_t n, double* part,
                           int nblocks, cudaStream_t st) {
  using C = typename CxT<R>::T;
  k_gs_dots<R><<<nblocks, 256, 0, st>>>((const C*)psi, (const C*)lower, k, parity, offgrid, n, part);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gs_apply(const void* psi, const void* lower, const double* sums, int k, int parity, int offgrid,
                            int64_t n, void* out, const double* V, double* part, int check, int nblocks,
                            cudaStream_t st) {
  using C = typename CxT<R>::T;
  k_gs_apply<R><<<nblocks, 256, 0, st>>>((const C*)psi, (const C*)lower, sums, k, parity, offgrid, n, (C*)out, V,
                                         part, check);
  return cudaGetLastError();
}

template <typename R>
int max_partials(int64_t n) {
  int best = 0;
  dispatch_n(n, [&](auto nc) {
    constexpr int N = decltype(nc)::value;
    using SH = Shape<R, N>;
    const int a = (int)((int64_t)N * N / SH::COLS);
    const int c = (int)((int64_t)N * N / SH::LINES);
    best = a > c ? a : c;
  });
  return best;
}

#define QFD_INSTANTIATE_LAUNCHERS(R)                                                                                \
  template cudaError_t launch_update_x<R>(const LaunchArgs&, int*);                                                 \
  template cudaError_t launch_forward_x<R>(const LaunchArgs&, int*);                                                \
  template cudaError_t launch_fft_y<R>(const LaunchArgs&, int);                                                     \
  template cudaError_t launch_fft_x_plain<R>(const LaunchArgs&, int);                                               \
  template cudaError_t launch_zpass<R>(const LaunchArgs&, int*);                                                    \
  template cudaError_t launch_gs_dots<R>(const void*, const void*, int, int, int, int64_t, double*, int,            \
                                         cudaStream_t);                                                             \
  template cudaError_t launch_gs_apply<R>(const void*, const void*, const double*, int, int, int, int64_t, void*,   \
                                          const double*, double*, int, int, cudaStream_t);                          \
  template int max_partials<R>(int64_t);

}  // namespace qfd
