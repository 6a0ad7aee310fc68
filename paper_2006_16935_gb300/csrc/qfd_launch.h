// Host-side launchers of the device kernels, one explicit instantiation per
// arithmetic type (qfd_k64.cu: complex128, qfd_k32.cu: complex64).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qfd {

struct KinParams;

// Which pass (used for the per-kernel timing instrumentation too).
enum PassKind {
  PASS_UPDATE_X = 0,  // pass A
  PASS_FWD_Y = 1,     // pass B
  PASS_ZKIN = 2,      // pass C
  PASS_INV_Y = 3,     // pass D
  PASS_FWD_X = 4,     // forward x of a fresh / projected psi
  PASS_GS_DOTS = 5,
  PASS_GS_APPLY = 6,
  PASS_FINALIZE = 7,
  PASS_OTHER = 8,
  PASS_COUNT = 9
};

struct LaunchArgs {
  int64_t n = 0;
  void* W = nullptr;          // work lattice (complex)
  void* psi = nullptr;        // state lattice (complex)
  const void* src = nullptr;  // forward-x input (may alias W)
  void* psi_out = nullptr;    // forward-x: where to store the scaled input (or null)
  const void* coef = nullptr; // update coefficients (double2 / float2 per site)
  const double* V = nullptr;  // FP64 potential
  const double* scale = nullptr;
  const void* tw = nullptr;   // twiddles exp(-2 pi i e / N), e < N
  const void* ktab = nullptr; // per-axis kinetic table
  const void* kin = nullptr;  // KinParams*
  double* part = nullptr;     // per-CTA partials
  int check = 0;
  cudaStream_t stream = 0;
};

// Each launcher returns cudaSuccess or the launch error; *nblocks receives the
// number of CTAs (= partials per reduced quantity) when non-null.
template <typename R> cudaError_t launch_update_x(const LaunchArgs& a, int* nblocks);
template <typename R> cudaError_t launch_forward_x(const LaunchArgs& a, int* nblocks);
template <typename R> cudaError_t launch_fft_y(const LaunchArgs& a, int dir);
template <typename R> cudaError_t launch_fft_x_plain(const LaunchArgs& a, int dir);
template <typename R> cudaError_t launch_zpass(const LaunchArgs& a, int* nblocks);
template <typename R> cudaError_t launch_gs_dots(const void* psi, const void* lower, int k, int parity, int offgrid,
                                                 int64_t n, double* part, int nblocks, cudaStream_t st);
template <typename R> cudaError_t launch_gs_apply(const void* psi, const void* lower, const double* sums, int k,
                                                  int parity, int offgrid, int64_t n, void* out, const double* V,
                                                  double* part, int check, int nblocks, cudaStream_t st);
template <typename R> int max_partials(int64_t n);  // largest CTA count of any reducing pass
bool supported_n(int64_t n);

}  // namespace qfd
