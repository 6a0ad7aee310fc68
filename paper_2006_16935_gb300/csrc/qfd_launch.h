// Host-side launchers of the device kernels.
//
// Launch<A, N> holds the launchers of one arithmetic policy A (F64, F32, DF)
// and lattice size N; qfd_inst.cu is compiled once per (A, N) pair so that
// the large unrolled kernels compile in parallel.  The launch_* templates
// below dispatch a runtime N to those instantiations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

namespace qfd {

// The scaled twiddles of the complex128 radix-8 stages (scaled_bfly8 in
// qfd_kernels.cuh), built from the plain table tw[e] = exp(-2 pi i e / n):
// 2 n double2 (forward block, then inverse), each e0 < n / 8 eight double2.
// The complex128 twiddle table of a lattice is tw followed by this block.
// Quotients are formed in long double and rounded once.
inline void scaled_twiddle_table(int64_t n, const double2* tw, double2* out) {
  using LD = long double;
  for (int d = 0; d < 2; ++d)
    for (int64_t e0 = 0; e0 < n / 8; ++e0) {
      double sig[8] = {1.0, 0, 0, 0, 0, 0, 0, 0}, tc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      int64_t bits = 0;
      for (int r = 1; r < 8; ++r) {
        const double2 w = tw[(e0 * r) % n];
        const double c = w.x, sn = d == 0 ? w.y : -w.y;
        if (std::fabs(c) >= std::fabs(sn)) {  // w = c (1 + i sn/c)
          sig[r] = c;
          tc[r] = (double)((LD)sn / (LD)c);
        } else {  // w = sn (c/sn + i)
          sig[r] = sn;
          tc[r] = (double)((LD)c / (LD)sn);
          bits |= (int64_t)1 << r;
        }
      }
      double fl;
      std::memcpy(&fl, &bits, sizeof(fl));
      double2* q = out + d * n + e0 * 8;
      q[0] = double2{fl, tc[1]};
      q[1] = double2{tc[2], tc[3]};
      q[2] = double2{tc[4], tc[5]};
      q[3] = double2{tc[6], tc[7]};
      q[4] = double2{sig[1], sig[2]};
      q[5] = double2{sig[4], (double)((LD)sig[3] / (LD)sig[1])};
      q[6] = double2{(double)((LD)sig[5] / (LD)sig[1]), (double)((LD)sig[6] / (LD)sig[2])};
      q[7] = double2{(double)((LD)sig[7] / (LD)sig[3]), (double)((LD)sig[1] * 0.70710678118654752440084436210485L)};
    }
}

struct KinParams;
struct UpdParams;
struct BatchY;
struct BatchZ;
struct BatchU;
struct F64;
struct F32;
struct DF;

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
  void* W = nullptr;           // work lattice
  void* psi = nullptr;         // state lattice
  const void* src = nullptr;   // forward-x input (may alias W)
  void* psi_out = nullptr;     // forward-x: where to store the scaled input (or null)
  const void* coef = nullptr;  // pass A's per-site update input: {A, B dtau} (F64) or V (F32, DF)
  const UpdParams* up = nullptr;  // time-step parameters of the V-derived coefficients
  const void* V = nullptr;     // potential as the policy's energy sums read it:
                               // FP64 (F64), double-float pairs (F32, DF)
  const double* scale = nullptr;  // normalisation factor (FP64) or null
  const float* scale_f = nullptr;  // its FP32 rounding and double-float split
  const void* tw = nullptr;    // twiddles exp(-2 pi i e / N), e < N
  const void* ktab = nullptr;  // per-axis kinetic table
  const KinParams* kin = nullptr;
  double* part = nullptr;      // per-CTA partials
  int stats = 0;               // STATS_* for passes A / forward x, Parseval flag for pass C
  cudaStream_t stream = 0;
  // projection / Gram-Schmidt
  const void* lower[8] = {};   // lower states (k of them)
  int k = 0;                   // number of lower states
  int parity = 0;              // 0, +1, -1
  int offgrid = 0;             // reflection about the off-grid centre
  const double* sums = nullptr;  // overlaps (2 doubles per lower state)
  void* dst = nullptr;         // projected state output
  // launch shapes (autotuner): y tiles of the default width (0), twice it (1)
  // or the two-stage radix schedule (2); z-pass line groups of the policy
  // default (-1), 1 (0), 2 (1) or the two-stage schedule (2); pass A tiles of
  // the default width (0), half of it with two CTAs per SM (1), or the
  // TMA-staged persistent kernel (2)
  int vy = 0;
  int vz = -1;
  int vx = 0;
  // the TMA-staged pass A: device addresses of the tensor maps of W, psi and
  // the update input, the plan's error flag, and the test switch that arms
  // its barriers without issuing copies
  const void* tmap[3] = {};
  int* err = nullptr;
  int tma_test = 0;
};

// Each launcher returns cudaSuccess or the launch error; *nblocks receives the
// number of CTAs (= partials per reduced quantity) when non-null.
template <class A, int N> struct Launch {
  // one lattice (a batch of one): the step passes
  static cudaError_t update_x(const LaunchArgs& a, int* nblocks);
  static cudaError_t fft_y(const LaunchArgs& a, int dir);
  static cudaError_t zpass(const LaunchArgs& a, int* nblocks);
  // one lattice: the cadence and energy passes
  static cudaError_t forward_x(const LaunchArgs& a, int* nblocks);
  static cudaError_t project_x(const LaunchArgs& a, int* nblocks);
  static cudaError_t gs_dots(const LaunchArgs& a, int nblocks);
  static int partials();  // largest CTA count of a reducing pass
  // the step passes over `count` lattices with the launch shapes vy, vz, vx
  // (as in LaunchArgs); pass A with any STATS mode, pass C with or without
  // the Parseval partial; *nblocks = CTAs per lattice
  static cudaError_t fft_y_batch(const BatchY& b, int count, int dir, int vy, cudaStream_t st);
  static cudaError_t zpass_batch(const BatchZ& b, int count, int parseval, int vz, cudaStream_t st, int* nblocks);
  static cudaError_t update_x_batch(const BatchU& b, int count, uint32_t scaled, int stats, int vx, cudaStream_t st,
                                    int* nblocks, int tma_test = 0);
  static int tma_xt();  // tile width of the TMA-staged pass A (vx = 2), 0 where it does not exist
};

template <int N> struct Tag {
  static constexpr int value = N;
};

template <class F>
inline cudaError_t dispatch_n(int64_t n, F&& f) {
  switch (n) {
    case 8: return f(Tag<8>());
    case 16: return f(Tag<16>());
    case 32: return f(Tag<32>());
    case 64: return f(Tag<64>());
    case 96: return f(Tag<96>());
    case 128: return f(Tag<128>());
    case 192: return f(Tag<192>());
    case 256: return f(Tag<256>());
    case 512: return f(Tag<512>());
    case 1024: return f(Tag<1024>());
    default: return cudaErrorInvalidValue;
  }
}

template <class A> cudaError_t launch_update_x(const LaunchArgs& a, int* nb) {
  return dispatch_n(a.n, [&](auto t) { return Launch<A, decltype(t)::value>::update_x(a, nb); });
}
template <class A> cudaError_t launch_forward_x(const LaunchArgs& a, int* nb) {
  return dispatch_n(a.n, [&](auto t) { return Launch<A, decltype(t)::value>::forward_x(a, nb); });
}
template <class A> cudaError_t launch_fft_y(const LaunchArgs& a, int dir) {
  return dispatch_n(a.n, [&](auto t) { return Launch<A, decltype(t)::value>::fft_y(a, dir); });
}
template <class A> cudaError_t launch_zpass(const LaunchArgs& a, int* nb) {
  return dispatch_n(a.n, [&](auto t) { return Launch<A, decltype(t)::value>::zpass(a, nb); });
}
template <class A> cudaError_t launch_project_x(const LaunchArgs& a, int* nb) {
  return dispatch_n(a.n, [&](auto t) { return Launch<A, decltype(t)::value>::project_x(a, nb); });
}
template <class A> cudaError_t launch_gs_dots(const LaunchArgs& a, int nblocks) {
  return dispatch_n(a.n, [&](auto t) { return Launch<A, decltype(t)::value>::gs_dots(a, nblocks); });
}
template <class A>
cudaError_t launch_fft_y_batch(int64_t n, const BatchY& b, int count, int dir, int vy, cudaStream_t st) {
  return dispatch_n(n, [&](auto t) { return Launch<A, decltype(t)::value>::fft_y_batch(b, count, dir, vy, st); });
}
template <class A>
cudaError_t launch_zpass_batch(int64_t n, const BatchZ& b, int count, int parseval, int vz, cudaStream_t st, int* nb) {
  return dispatch_n(
      n, [&](auto t) { return Launch<A, decltype(t)::value>::zpass_batch(b, count, parseval, vz, st, nb); });
}
template <class A>
cudaError_t launch_update_x_batch(int64_t n, const BatchU& b, int count, uint32_t scaled, int stats, int vx,
                                  cudaStream_t st, int* nb, int tma_test = 0) {
  return dispatch_n(n, [&](auto t) {
    return Launch<A, decltype(t)::value>::update_x_batch(b, count, scaled, stats, vx, st, nb, tma_test);
  });
}
template <class A> int launch_tma_xt(int64_t n) {
  int out = 0;
  dispatch_n(n, [&](auto t) {
    out = Launch<A, decltype(t)::value>::tma_xt();
    return cudaSuccess;
  });
  return out;
}
template <class A> int max_partials(int64_t n) {
  int out = 0;
  dispatch_n(n, [&](auto t) {
    out = Launch<A, decltype(t)::value>::partials();
    return cudaSuccess;
  });
  return out;
}

bool supported_n(int64_t n);

}  // namespace qfd
