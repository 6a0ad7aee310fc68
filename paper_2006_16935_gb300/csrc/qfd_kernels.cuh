// Device kernels of the imaginary-time FFT solver (arXiv:2006.16935, Sec. 2).
//
// One imaginary-time step of Eq. (iter_proced) with an FFT kinetic term
// (Eqs. HK1-HK3) is four passes over the N^3 lattice (layout [x][y][z], z
// contiguous, interleaved complex):
//
//   pass A  x-lines : inverse DFT_x of W  -> H_K psi, the A/B update of Sec. 2.2,
//                     norm / <V> partial sums, forward DFT_x of the new psi -> W
//   pass B  y-lines : forward DFT_y of W (in place)
//   pass C  z-lines : forward DFT_z, multiply by T(k)/N^3, Parseval partial
//                     sum of <H_K>, inverse DFT_z (in place)
//   pass D  y-lines : inverse DFT_y (in place)
//
// Every line transform is a radix-8/4/2 Stockham FFT held in registers:
// thread t of a line owns the 8 elements t + m*N/8 (m = 0..7) before and after
// the transform, stages exchange through shared memory.  Complex data is
// double2 (complex128) or float2 (complex64); every reduction accumulates in
// FP64 and combines per-CTA partials in a fixed order (deterministic).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qfd {

// ------------------------------------------------------------------ complex
template <typename R> struct CxT;
template <> struct CxT<double> { using T = double2; };
template <> struct CxT<float> { using T = float2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C w) {
  return C{fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x)};
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C w) {  // a * conj(w)
  return C{fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y)};
}
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { return C{a.x * s, a.y * s}; }

// multiply by -i (DIR = -1, forward) or +i (DIR = +1, inverse)
template <int DIR, typename C> __device__ __forceinline__ C mul_i(C a) {
  return DIR > 0 ? C{-a.y, a.x} : C{a.y, -a.x};
}
// multiply by exp(DIR * 2 pi i / 8) = (1 + DIR i) / sqrt 2
template <int DIR, typename C> __device__ __forceinline__ C mul_w8(C a) {
  using R = decltype(a.x);
  const R h = R(0.70710678118654752440084436210485);
  return DIR > 0 ? C{(a.x - a.y) * h, (a.x + a.y) * h} : C{(a.x + a.y) * h, (a.y - a.x) * h};
}

template <int DIR, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}
template <int DIR, typename C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C s0 = cadd(x0, x2), d0 = csub(x0, x2);
  C s1 = cadd(x1, x3), d1 = mul_i<DIR>(csub(x1, x3));
  x0 = cadd(s0, s1);
  x2 = csub(s0, s1);
  x1 = cadd(d0, d1);
  x3 = csub(d0, d1);
}
template <int DIR, typename C> __device__ __forceinline__ void dft8(C* x) {
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  o1 = mul_w8<DIR>(o1);
  o2 = mul_i<DIR>(o2);
  o3 = mul_i<DIR>(mul_w8<DIR>(o3));
  x[0] = cadd(e0, o0);
  x[4] = csub(e0, o0);
  x[1] = cadd(e1, o1);
  x[5] = csub(e1, o1);
  x[2] = cadd(e2, o2);
  x[6] = csub(e2, o2);
  x[3] = cadd(e3, o3);
  x[7] = csub(e3, o3);
}

// ------------------------------------------------------------ FFT planning
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// N = 2^p: floor(p/3) radix-8 stages, then one radix-2 or radix-4 stage.
template <int N> struct FftPlan {
  static constexpr int P = ilog2c(N);
  static constexpr int Q = P / 3;
  static constexpr int REM = P % 3;
  static constexpr int S = Q + (REM ? 1 : 0);
  __host__ __device__ static constexpr int radix(int i) { return i < Q ? 8 : (REM == 1 ? 2 : 4); }
  __host__ __device__ static constexpr int ns(int i) { return i == 0 ? 1 : ns(i - 1) * radix(i - 1); }
};

// One Stockham stage on the register-resident canonical set v[m] = x[t + m N/8].
// Butterfly b = t + u N/8 (u < 8/RAD) takes x[b + r N/RAD] = v[u + r (8/RAD)],
// multiplies input r by w_N^{(b mod NS) r N/(NS RAD)}, and applies DFT_RAD.
template <typename C, int N, int RAD, int NS, int DIR>
__device__ __forceinline__ void stage_compute(C (&v)[8], int t, const C* __restrict__ tw) {
  constexpr int NB = 8 / RAD;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    C x[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) x[r] = v[u + r * NB];
    if (NS > 1) {
      const int b = t + u * (N / 8);
      const int e0 = (b % NS) * (N / (NS * RAD));
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        const C w = __ldg(&tw[e0 * r]);
        x[r] = DIR < 0 ? cmul(x[r], w) : cmulc(x[r], w);
      }
    }
    if (RAD == 8) dft8<DIR>(x);
    if (RAD == 4) dft4<DIR>(x[0], x[1], x[2], x[3]);
    if (RAD == 2) dft2<DIR>(x[0], x[1]);
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[u + r * NB] = x[r];
  }
}

// Writes stage outputs to their Stockham positions, then reads the canonical set.
template <typename C, int N, int RAD, int NS, class Acc>
__device__ __forceinline__ void stage_exchange(C (&v)[8], int t, Acc& acc) {
  constexpr int NB = 8 / RAD;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int b = t + u * (N / 8);
    const int base = (b / NS) * NS * RAD + (b % NS);
#pragma unroll
    for (int r = 0; r < RAD; ++r) acc.at(base + r * NS) = v[u + r * NB];
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = acc.at(t + m * (N / 8));
  __syncthreads();
}

template <typename C, int N, int DIR, int I, class Acc>
__device__ __forceinline__ void fft_stages(C (&v)[8], int t, const C* __restrict__ tw, Acc& acc) {
  if constexpr (I < FftPlan<N>::S) {
    constexpr int RAD = FftPlan<N>::radix(I);
    constexpr int NS = FftPlan<N>::ns(I);
    stage_compute<C, N, RAD, NS, DIR>(v, t, tw);
    if constexpr (I + 1 < FftPlan<N>::S) stage_exchange<C, N, RAD, NS>(v, t, acc);
    fft_stages<C, N, DIR, I + 1>(v, t, tw, acc);
  }
}

// Unnormalised length-N DFT, sign DIR, canonical layout in and out.
template <typename C, int N, int DIR, class Acc>
__device__ __forceinline__ void fft_line(C (&v)[8], int t, const C* __restrict__ tw, Acc& acc) {
  fft_stages<C, N, DIR, 0>(v, t, tw, acc);
}

// Shared-memory views. Tile of C_ columns of a strided axis: [pos][col].
template <typename C, int CW> struct AccTile {
  C* sm;
  int col;
  __device__ __forceinline__ C& at(int pos) { return sm[pos * CW + col]; }
};
// One contiguous line, padded by one element every 8 (bank-conflict free).
template <typename C> struct AccLine {
  C* sm;
  __device__ __forceinline__ C& at(int pos) { return sm[pos + (pos >> 3)]; }
};

// ---------------------------------------------------------- launch shapes
template <typename R, int N> struct Shape {
  static constexpr int T = N / 8;                       // threads per line
  static constexpr int CMIN = sizeof(R) == 8 ? 8 : 16;  // 128-byte row segments
  static constexpr int C0 = (256 / T > CMIN) ? 256 / T : CMIN;
  static constexpr int C1 = C0 < 1024 / T ? C0 : 1024 / T;
  static constexpr int COLS = C1 < N ? C1 : N;          // strided-tile columns
  static constexpr int TILE_THREADS = T * COLS;
  static constexpr int LINES0 = (256 / T) > 1 ? 256 / T : 1;
  static constexpr int LINES = LINES0 < N * N ? LINES0 : N * N;  // z-pass lines per CTA
  static constexpr int LINE_THREADS = T * LINES;
  static constexpr int LPAD = N + N / 8;
};

// ------------------------------------------------------------- reductions
// Block sum of NQ doubles; thread 0 writes part[q * nblocks + blockIdx.x].
// Blocks of fewer than 32 threads (the 8^3 lattice) sum serially in thread
// order instead (no warp shuffle over lanes that do not exist).
template <int NQ>
__device__ __forceinline__ void block_reduce_store(double (&val)[NQ], double* __restrict__ part) {
  __shared__ double red[NQ][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  if (blockDim.x < 32) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q][threadIdx.x] = val[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) s += red[q][i];
        part[(int64_t)q * gridDim.x + blockIdx.x] = s;
      }
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double x = val[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[q][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = lane < nwarps ? red[q][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) part[(int64_t)q * gridDim.x + blockIdx.x] = x;
    }
  }
}

// ------------------------------------------------------------ parameters
struct KinParams {
  int kinterm;       // 1, 2, 3 (Eqs. HK1-HK3)
  double pref;       // HK1/HK2: 1 / (2 A^2 M N^3)
  double am2;        // (A M)^2 (HK3)
  double inv_a_n3;   // 1 / (A N^3) (HK3)
  double m0_n3;      // M / N^3 subtracted when the rest mass is removed (HK3)
};

template <typename R>
__device__ __forceinline__ R kin_value(R s, const KinParams& kp) {
  if (kp.kinterm == 3) return sqrt(s + R(kp.am2)) * R(kp.inv_a_n3) - R(kp.m0_n3);
  return s * R(kp.pref);
}

// Update coefficients: complex128 stores {A, B dtau} and forms A psi - (B dtau) H_K psi
// as printed; complex64 stores {B dtau, 1 - A} and forms psi - (1-A) psi - (B dtau) H_K psi
// so that the O(dtau) increment keeps full FP32 relative precision.
template <typename R> struct Coef;
template <> struct Coef<double> { using T = double2; };
template <> struct Coef<float> { using T = float2; };

template <typename C, typename K>
__device__ __forceinline__ C update_site(C ps, C hk, K cf);
template <>
__device__ __forceinline__ double2 update_site<double2, double2>(double2 ps, double2 hk, double2 cf) {
  return double2{cf.x * ps.x - cf.y * hk.x, cf.x * ps.y - cf.y * hk.y};
}
template <>
__device__ __forceinline__ float2 update_site<float2, float2>(float2 ps, float2 hk, float2 cf) {
  return float2{ps.x - (cf.y * ps.x + cf.x * hk.x), ps.y - (cf.y * ps.y + cf.x * hk.y)};
}

// ================================================================ kernels

// Pass B / D (and the x-direction forward transform of a fresh psi when src
// is given): in-place strided line FFT over tiles of COLS contiguous columns.
// Tile id -> base = (id / tiles_inner) * outer_stride + (id % tiles_inner) * COLS.
template <typename R, int N, int DIR>
__global__ void __launch_bounds__(Shape<R, N>::TILE_THREADS)
k_fft_strided(typename CxT<R>::T* W, const typename CxT<R>::T* __restrict__ tw, int64_t stride,
              int tiles_inner, int64_t outer_stride) {
  using C = typename CxT<R>::T;
  using SH = Shape<R, N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int col = threadIdx.x % SH::COLS, t = threadIdx.x / SH::COLS;
  const int64_t base = (int64_t)(blockIdx.x / tiles_inner) * outer_stride +
                       (int64_t)(blockIdx.x % tiles_inner) * SH::COLS + col;
  C v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = W[base + (int64_t)(t + m * SH::T) * stride];
  AccTile<C, SH::COLS> acc{sm, col};
  fft_line<C, N, DIR>(v, t, tw, acc);
#pragma unroll
  for (int m = 0; m < 8; ++m) W[base + (int64_t)(t + m * SH::T) * stride] = v[m];
}

// Pass C: forward DFT_z, times T(k)/N^3 (+ Parseval partial), inverse DFT_z.
// The canonical layout is the same before and after a transform, so the
// multiply sits in registers between the two transforms.
template <typename R, int N>
__global__ void __launch_bounds__(Shape<R, N>::LINE_THREADS)
k_zpass(typename CxT<R>::T* W, const typename CxT<R>::T* __restrict__ tw, const R* __restrict__ ktab,
        KinParams kp, double* __restrict__ part, int parseval) {
  using C = typename CxT<R>::T;
  using SH = Shape<R, N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int l = threadIdx.x / SH::T, t = threadIdx.x % SH::T;
  const int64_t line = (int64_t)blockIdx.x * SH::LINES + l;  // = kx * N + ky
  C* p = W + line * N;
  C v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = p[t + m * SH::T];
  AccLine<C> acc{sm + l * SH::LPAD};
  fft_line<C, N, -1>(v, t, tw, acc);
  const R sxy = ktab[line / N] + ktab[line % N];
  double pt = 0.0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const R tk = kin_value<R>(sxy + ktab[t + m * SH::T], kp);
    if (parseval) pt += (double)tk * ((double)v[m].x * v[m].x + (double)v[m].y * v[m].y);
    v[m] = cscale(v[m], tk);
  }
  fft_line<C, N, +1>(v, t, tw, acc);
#pragma unroll
  for (int m = 0; m < 8; ++m) p[t + m * SH::T] = v[m];
  if (parseval) {
    double q[1] = {pt};
    block_reduce_store<1>(q, part);
  }
}

// Pass A: inverse DFT_x of W gives H_K psi at the tile's sites; the update of
// Eq. (iter_proced) with the coefficients of Sec. 2.2 (times an optional
// normalisation factor *scale carried from the previous step); partials of
// sum |psi|^2 and (check) sum V |psi|^2; forward DFT_x of the new psi into W.
template <typename R, int N>
__global__ void __launch_bounds__(Shape<R, N>::TILE_THREADS)
k_update_x(typename CxT<R>::T* W, typename CxT<R>::T* __restrict__ psi,
           const typename Coef<R>::T* __restrict__ coef, const double* __restrict__ V,
           const double* __restrict__ scale, const typename CxT<R>::T* __restrict__ tw,
           double* __restrict__ part, int check) {
  using C = typename CxT<R>::T;
  using SH = Shape<R, N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int col = threadIdx.x % SH::COLS, t = threadIdx.x / SH::COLS;
  const int64_t base = (int64_t)blockIdx.x * SH::COLS + col;
  constexpr int64_t S = (int64_t)N * N;
  C v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = W[base + (t + m * SH::T) * S];
  AccTile<C, SH::COLS> acc{sm, col};
  fft_line<C, N, +1>(v, t, tw, acc);
  const R s = scale ? R(*scale) : R(1);
  double n2 = 0.0, pv = 0.0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int64_t idx = base + (t + m * SH::T) * S;
    C nw = update_site(psi[idx], v[m], coef[idx]);
    if (scale) nw = cscale(nw, s);
    psi[idx] = nw;
    v[m] = nw;
    const double a2 = (double)nw.x * nw.x + (double)nw.y * nw.y;
    n2 += a2;
    if (check) pv += V[idx] * a2;
  }
  fft_line<C, N, -1>(v, t, tw, acc);
#pragma unroll
  for (int m = 0; m < 8; ++m) W[base + (t + m * SH::T) * S] = v[m];
  double q[2] = {n2, pv};
  block_reduce_store<2>(q, part);
}

// Forward DFT_x of src (optionally times *scale, optionally also written to
// psi_out) into W; partials of sum |.|^2 and sum V |.|^2 of the scaled input.
// src may alias W (each CTA reads its whole tile before writing it).
template <typename R, int N>
__global__ void __launch_bounds__(Shape<R, N>::TILE_THREADS)
k_forward_x(const typename CxT<R>::T* src, typename CxT<R>::T* W, typename CxT<R>::T* psi_out,
            const double* __restrict__ V, const double* __restrict__ scale,
            const typename CxT<R>::T* __restrict__ tw, double* __restrict__ part, int check) {
  using C = typename CxT<R>::T;
  using SH = Shape<R, N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int col = threadIdx.x % SH::COLS, t = threadIdx.x / SH::COLS;
  const int64_t base = (int64_t)blockIdx.x * SH::COLS + col;
  constexpr int64_t S = (int64_t)N * N;
  const R s = scale ? R(*scale) : R(1);
  C v[8];
  double n2 = 0.0, pv = 0.0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int64_t idx = base + (t + m * SH::T) * S;
    C x = src[idx];
    if (scale) x = cscale(x, s);
    v[m] = x;
    const double a2 = (double)x.x * x.x + (double)x.y * x.y;
    n2 += a2;
    if (check) pv += V[idx] * a2;
  }
  if (psi_out) {
#pragma unroll
    for (int m = 0; m < 8; ++m) psi_out[base + (t + m * SH::T) * S] = v[m];
  }
  AccTile<C, SH::COLS> acc{sm, col};
  fft_line<C, N, -1>(v, t, tw, acc);
#pragma unroll
  for (int m = 0; m < 8; ++m) W[base + (t + m * SH::T) * S] = v[m];
  double q[2] = {n2, pv};
  block_reduce_store<2>(q, part);
}

// ------------------------------------------------- elementwise site kernels
__host__ __device__ __forceinline__ int64_t reflect_index(int64_t i, int64_t n, int offgrid) {
  const int64_t z = i % n, y = (i / n) % n, x = i / (n * n);
  const int64_t rx = offgrid ? n - 1 - x : (n - x) % n;
  const int64_t ry = offgrid ? n - 1 - y : (n - y) % n;
  const int64_t rz = offgrid ? n - 1 - z : (n - z) % n;
  return (rx * n + ry) * n + rz;
}

constexpr int MAX_LOWER = 8;

// Overlaps <phi_j | P psi> (FP64) for j < k, P the parity projector (Eq. parity).
template <typename R>
__global__ void k_gs_dots(const typename CxT<R>::T* __restrict__ psi, const typename CxT<R>::T* __restrict__ lower,
                          int k, int parity, int offgrid, int64_t n, double* __restrict__ part) {
  const int64_t n3 = n * n * n;
  double acc[2 * MAX_LOWER];
#pragma unroll
  for (int j = 0; j < 2 * MAX_LOWER; ++j) acc[j] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    auto p = psi[i];
    double px = p.x, py = p.y;
    if (parity) {
      auto q = psi[reflect_index(i, n, offgrid)];
      px = 0.5 * (px + parity * (double)q.x);
      py = 0.5 * (py + parity * (double)q.y);
    }
#pragma unroll
    for (int j = 0; j < MAX_LOWER; ++j) {
      if (j < k) {
        auto f = lower[j * n3 + i];
        acc[2 * j] += (double)f.x * px + (double)f.y * py;
        acc[2 * j + 1] += (double)f.x * py - (double)f.y * px;
      }
    }
  }
  block_reduce_store<2 * MAX_LOWER>(acc, part);
}

// out = P psi - sum_j c_j phi_j  (c_j = sums[2j] + i sums[2j+1]);
// partials of sum |out|^2 and sum V |out|^2.
template <typename R>
__global__ void k_gs_apply(const typename CxT<R>::T* __restrict__ psi, const typename CxT<R>::T* __restrict__ lower,
                           const double* __restrict__ sums, int k, int parity, int offgrid, int64_t n,
                           typename CxT<R>::T* __restrict__ out, const double* __restrict__ V,
                           double* __restrict__ part, int check) {
  using C = typename CxT<R>::T;
  const int64_t n3 = n * n * n;
  double n2 = 0.0, pv = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    C p = psi[i];
    if (parity) {
      const C q = psi[reflect_index(i, n, offgrid)];
      p = C{R(0.5) * (p.x + R(parity) * q.x), R(0.5) * (p.y + R(parity) * q.y)};
    }
    for (int j = 0; j < k; ++j) {
      const C f = lower[j * n3 + i];
      const R cr = R(sums[2 * j]), ci = R(sums[2 * j + 1]);
      p.x -= cr * f.x - ci * f.y;
      p.y -= cr * f.y + ci * f.x;
    }
    out[i] = p;
    const double a2 = (double)p.x * p.x + (double)p.y * p.y;
    n2 += a2;
    if (check) pv += V[i] * a2;
  }
  double q[2] = {n2, pv};
  block_reduce_store<2>(q, part);
}

}  // namespace qfd
