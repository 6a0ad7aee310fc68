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
// the transform, stages exchange through shared memory.
//
// Three arithmetic policies share the code:
//   F64  complex128 (double2), native FP64 arithmetic;
//   F32  complex64 (float2), FP32 arithmetic;
//   DF   complex stored as double-float pairs (hi + lo FP32, 16 bytes like
//        complex128), arithmetic on the FP32 pipe with error-free
//        transformations (two-sum, FMA two-product): about 2^-46 relative
//        rounding per operation.  GB300 issues FP32 ~58x faster than FP64.
// Reductions always end in FP64: per-thread partials of |psi|^2 are exact
// double-float sums (F32/DF) or FP64 (F64), converted to double once per
// thread, then combined per CTA and across CTAs in a fixed order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qfd {

// ============================================================ float/double
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C w) {
  return C{fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x)};
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C w) {  // a * conj(w)
  return C{fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y)};
}
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { return C{a.x * s, a.y * s}; }
// butterfly additions (double-float overloads below defer the renormalisation)
template <typename C> __device__ __forceinline__ C cadd_l(C a, C b) { return cadd(a, b); }
template <typename C> __device__ __forceinline__ C csub_l(C a, C b) { return csub(a, b); }
template <typename C> __device__ __forceinline__ C cnorm(C a) { return a; }
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

// ============================================================ double-float
// Error-free transformations (Knuth two-sum, Dekker fast-two-sum, FMA
// two-product) with round-to-nearest intrinsics so that nothing is contracted
// or reassociated.
struct df {
  float h, l;
};
struct __align__(16) dfc {
  df x, y;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df dneg(df a) { return df{-a.h, -a.l}; }
// a + b with error below ~2^-45 (|a| + |b|)
__device__ __forceinline__ df dadd(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df dsub(df a, df b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ df dmul(df a, df b) {
  const df p = two_prod(a.h, b.h);
  float e = __fmaf_rn(a.h, b.l, p.l);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p.h, e);
}
// a*b - c*d and a*b + c*d with one renormalisation
__device__ __forceinline__ df dmul_sub(df a, df b, df c, df d) {
  const df p = two_prod(a.h, b.h), q = two_prod(c.h, d.h);
  const df s = two_sum(p.h, -q.h);
  float e = __fadd_rn(s.l, __fsub_rn(p.l, q.l));
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  e = __fmaf_rn(-c.h, d.l, e);
  e = __fmaf_rn(-c.l, d.h, e);
  return fast_two_sum(s.h, e);
}
__device__ __forceinline__ df dmul_add(df a, df b, df c, df d) { return dmul_sub(a, b, dneg(c), d); }
__device__ __forceinline__ df dsqrt(df a) {
  if (!(a.h > 0.f)) return df{0.f, 0.f};
  const float s = sqrtf(a.h);
  const df s2 = two_prod(s, s);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, s2.h), s2.l), a.l);
  return fast_two_sum(s, __fmul_rn(r, __fdiv_rn(0.5f, s)));
}
__device__ __forceinline__ df dsplit(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double dval(df a) { return (double)a.h + (double)a.l; }

// Lazy sum inside a butterfly: error-free two-sum of the high parts, the low
// parts added without renormalising; cnorm renormalises the butterfly outputs.
// Within one radix-8 butterfly the low part stays within a few ulp of the high
// part, so the accuracy of the renormalised result is unchanged.
__device__ __forceinline__ df dadd_l(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return df{s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ df dsub_l(df a, df b) { return dadd_l(a, dneg(b)); }
__device__ __forceinline__ dfc cadd_l(dfc a, dfc b) { return dfc{dadd_l(a.x, b.x), dadd_l(a.y, b.y)}; }
__device__ __forceinline__ dfc csub_l(dfc a, dfc b) { return dfc{dsub_l(a.x, b.x), dsub_l(a.y, b.y)}; }
__device__ __forceinline__ dfc cnorm(dfc a) { return dfc{fast_two_sum(a.x.h, a.x.l), fast_two_sum(a.y.h, a.y.l)}; }
__device__ __forceinline__ dfc cadd(dfc a, dfc b) { return dfc{dadd(a.x, b.x), dadd(a.y, b.y)}; }
__device__ __forceinline__ dfc csub(dfc a, dfc b) { return dfc{dsub(a.x, b.x), dsub(a.y, b.y)}; }
__device__ __forceinline__ dfc cmul(dfc a, dfc w) {
  return dfc{dmul_sub(a.x, w.x, a.y, w.y), dmul_add(a.x, w.y, a.y, w.x)};
}
__device__ __forceinline__ dfc cmulc(dfc a, dfc w) {
  return dfc{dmul_add(a.x, w.x, a.y, w.y), dmul_sub(a.y, w.x, a.x, w.y)};
}
__device__ __forceinline__ dfc cscale(dfc a, df s) { return dfc{dmul(a.x, s), dmul(a.y, s)}; }
template <int DIR> __device__ __forceinline__ dfc mul_i(dfc a) {
  return DIR > 0 ? dfc{dneg(a.y), a.x} : dfc{a.y, dneg(a.x)};
}
template <int DIR> __device__ __forceinline__ dfc mul_w8(dfc a) {
  const df h{0.70710677f, 1.2101617486e-08f};  // sqrt(1/2) = h.h + h.l to 2^-51
  return DIR > 0 ? dfc{dmul(dsub_l(a.x, a.y), h), dmul(dadd_l(a.x, a.y), h)}
                 : dfc{dmul(dadd_l(a.x, a.y), h), dmul(dsub_l(a.y, a.x), h)};
}

// ================================================================ policies
struct KinParams {
  int kinterm;      // 1, 2, 3 (Eqs. HK1-HK3)
  double pref;      // HK1/HK2: 1 / (2 A^2 M N^3)
  double am2;       // (A M)^2 (HK3)
  double inv_a_n3;  // 1 / (A N^3) (HK3)
  double m0_n3;     // M / N^3 subtracted when the rest mass is removed (HK3)
  float f_pref, f_am2, f_ia, f_m0;      // the same rounded to FP32
  df d_pref, d_am2, d_ia, d_m0;         // the same as double-float pairs
};

// Time-step parameters of the update in the representations that derive the
// coefficients of Sec. 2.2 from V inside pass A (FP32 and double-float).
struct UpdParams {
  float f_dtau, f_hdt;  // dtau and dtau / 2 in FP32
  df d_dtau, d_hdt;     // the same as double-float pairs
};

struct F64 {
  using C = double2;  // lattice element
  using K = double2;  // update coefficients {A, B dtau}
  using U = double2;  // what pass A reads per site: the precomputed {A, B dtau}
  using T = double;   // per-axis kinetic table entry
  using S = double;   // scalar
  using VT = double;  // potential as read by the energy partials
  static constexpr int id = 0;
  static __device__ __forceinline__ C ldtw(const C* p) { return __ldg(p); }
  static __device__ __forceinline__ T kadd(T a, T b) { return a + b; }
  static __device__ __forceinline__ T kin(T s, const KinParams& kp) {
    return kp.kinterm == 3 ? sqrt(s + kp.am2) * kp.inv_a_n3 - kp.m0_n3 : s * kp.pref;
  }
  static __device__ __forceinline__ S scalar(double s) { return s; }
  // the normalisation factor as written by the reduction kernel: FP64 value,
  // then its FP32 rounding and double-float split in a float array
  static __device__ __forceinline__ S load_scale(const double* d, const float*) { return *d; }
  // complex128 passes are bound by FP64 issue, so the coefficients are read
  // precomputed (16 B) rather than derived per site with an FP64 division
  static __device__ __forceinline__ K coef_from(U u, const UpdParams&) { return u; }
  // Eq. (iter_proced) as printed: A psi - (B dtau) H_K psi
  static __device__ __forceinline__ C update(C ps, C hk, K cf) {
    return C{cf.x * ps.x - cf.y * hk.x, cf.x * ps.y - cf.y * hk.y};
  }
  static __device__ __forceinline__ double2 to_d2(C v) { return v; }
  static __device__ __forceinline__ C from_d2(double2 v) { return v; }
  static __device__ __forceinline__ double norm2_d(C v) { return v.x * v.x + v.y * v.y; }
  static __device__ __forceinline__ double tval(T t) { return t; }
  // (p + par q) / 2
  static __device__ __forceinline__ C half_comb(C p, C q, int par) {
    return par > 0 ? C{0.5 * (p.x + q.x), 0.5 * (p.y + q.y)} : C{0.5 * (p.x - q.x), 0.5 * (p.y - q.y)};
  }
  struct Acc {
    double s = 0.0;
    __device__ __forceinline__ void add_norm(C v) { s += v.x * v.x + v.y * v.y; }
    __device__ __forceinline__ double value() const { return s; }
  };
  struct Dot {  // sum of conj(f) p
    double re = 0.0, im = 0.0;
    __device__ __forceinline__ void add(C f, C p) {
      re += f.x * p.x + f.y * p.y;
      im += f.x * p.y - f.y * p.x;
    }
    __device__ __forceinline__ double2 value() const { return double2{re, im}; }
  };
  struct Full {  // sums of |psi|^2 and V |psi|^2
    double n2 = 0.0, pv = 0.0;
    __device__ __forceinline__ void add(C v, VT vv) {
      const double a2 = v.x * v.x + v.y * v.y;
      n2 += a2;
      pv += vv * a2;
    }
  };
  struct Pars {  // Parseval sum of T |psi~|^2
    double pt = 0.0;
    __device__ __forceinline__ void add(T tk, C v) { pt += tk * (v.x * v.x + v.y * v.y); }
  };
};

struct F32 {
  using C = float2;
  using K = float2;  // {B dtau, 1 - A}
  using U = float;   // pass A reads V in FP32 and derives K
  using T = float;
  using S = float;
  using VT = df;     // the double-float copy of V
  static constexpr int id = 1;
  static __device__ __forceinline__ C ldtw(const C* p) { return __ldg(p); }
  static __device__ __forceinline__ T kadd(T a, T b) { return a + b; }
  static __device__ __forceinline__ T kin(T s, const KinParams& kp) {
    return kp.kinterm == 3 ? sqrtf(s + kp.f_am2) * kp.f_ia - kp.f_m0 : s * kp.f_pref;
  }
  static __device__ __forceinline__ S scalar(double s) { return (float)s; }
  static __device__ __forceinline__ S load_scale(const double*, const float* f) { return f[0]; }
  // Sec. 2.2 with h = dtau V / 2: B dtau = dtau / (1 + h) and 1 - A = 2h / (1 + h)
  // = V (B dtau).  Nothing cancels, so both keep FP32 relative precision.
  static __device__ __forceinline__ K coef_from(U v, const UpdParams& up) {
    const float g1 = up.f_dtau * __frcp_rn(1.0f + v * up.f_hdt);
    return K{g1, v * g1};
  }
  // psi - ((1 - A) psi + (B dtau) H_K psi): the O(dtau) increment keeps FP32 relative precision
  static __device__ __forceinline__ C update(C ps, C hk, K cf) {
    return C{ps.x - (cf.y * ps.x + cf.x * hk.x), ps.y - (cf.y * ps.y + cf.x * hk.y)};
  }
  static __device__ __forceinline__ double2 to_d2(C v) { return double2{(double)v.x, (double)v.y}; }
  static __device__ __forceinline__ C from_d2(double2 v) { return C{(float)v.x, (float)v.y}; }
  static __device__ __forceinline__ double norm2_d(C v) {
    return (double)v.x * v.x + (double)v.y * v.y;
  }
  static __device__ __forceinline__ double tval(T t) { return t; }
  static __device__ __forceinline__ C half_comb(C p, C q, int par) {
    return par > 0 ? C{0.5f * (p.x + q.x), 0.5f * (p.y + q.y)} : C{0.5f * (p.x - q.x), 0.5f * (p.y - q.y)};
  }
  struct Acc {  // exact double-float accumulation of the squares
    df s{0.f, 0.f};
    __device__ __forceinline__ void add_norm(C v) {
      const df a = two_prod(v.x, v.x), b = two_prod(v.y, v.y);
      s = dadd(s, dadd(a, b));
    }
    __device__ __forceinline__ double value() const { return dval(s); }
  };
  struct Dot {  // sum of conj(f) p with error-free products, double-float sums
    df re{0.f, 0.f}, im{0.f, 0.f};
    __device__ __forceinline__ void add(C f, C p) {
      re = dadd(re, dadd(two_prod(f.x, p.x), two_prod(f.y, p.y)));
      im = dadd(im, dsub(two_prod(f.x, p.y), two_prod(f.y, p.x)));
    }
    __device__ __forceinline__ double2 value() const { return double2{dval(re), dval(im)}; }
  };
  // energy partials in double-float on the FP32 pipe (exact squares)
  struct Full {
    df n2{0.f, 0.f}, pv{0.f, 0.f};
    __device__ __forceinline__ void add(C v, VT vv) {
      const df a2 = dadd(two_prod(v.x, v.x), two_prod(v.y, v.y));
      n2 = dadd(n2, a2);
      pv = dadd(pv, dmul(a2, vv));
    }
  };
  struct Pars {
    df pt{0.f, 0.f};
    __device__ __forceinline__ void add(T tk, C v) {
      pt = dadd(pt, dmul(dadd(two_prod(v.x, v.x), two_prod(v.y, v.y)), df{tk, 0.f}));
    }
  };
};

struct DF {
  using C = dfc;
  using K = dfc;  // {B dtau, 1 - A} as double-float pairs
  using U = df;   // pass A reads V as a double-float pair and derives K
  using T = df;
  using S = df;
  using VT = df;  // the double-float copy of V
  static constexpr int id = 2;
  static __device__ __forceinline__ C ldtw(const C* p) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    return dfc{df{q.x, q.y}, df{q.z, q.w}};
  }
  static __device__ __forceinline__ T kadd(T a, T b) { return dadd(a, b); }
  static __device__ __forceinline__ T kin(T s, const KinParams& kp) {
    return kp.kinterm == 3 ? dsub(dmul(dsqrt(dadd(s, kp.d_am2)), kp.d_ia), kp.d_m0) : dmul(s, kp.d_pref);
  }
  static __device__ __forceinline__ S scalar(double s) { return dsplit(s); }
  static __device__ __forceinline__ S load_scale(const double*, const float* f) { return df{f[1], f[2]}; }
  // B dtau = dtau r and 1 - A = V (B dtau) with r = 1 / (1 + h), h = dtau V / 2:
  // r from the FP32 reciprocal r0 and one Newton step r0 + r0 (1 - d r0), the
  // residual 1 - d r0 formed from the exact product of the high parts (its
  // leading difference is exact), so r carries about 2^-46 relative error.
  static __device__ __forceinline__ K coef_from(U v, const UpdParams& up) {
    const df d = dadd(df{1.0f, 0.0f}, dmul(v, up.d_hdt));
    const float r0 = __frcp_rn(d.h);
    const df p = two_prod(d.h, r0);
    const float e = __fmaf_rn(-d.l, r0, __fsub_rn(__fsub_rn(1.0f, p.h), p.l));
    const df r = fast_two_sum(r0, __fmul_rn(r0, e));
    const df g1 = dmul(up.d_dtau, r);
    return K{g1, dmul(v, g1)};
  }
  static __device__ __forceinline__ C update(C ps, C hk, K cf) {
    const df dx = dmul_add(cf.y, ps.x, cf.x, hk.x), dy = dmul_add(cf.y, ps.y, cf.x, hk.y);
    return dfc{dsub(ps.x, dx), dsub(ps.y, dy)};
  }
  static __device__ __forceinline__ double2 to_d2(C v) { return double2{dval(v.x), dval(v.y)}; }
  static __device__ __forceinline__ C from_d2(double2 v) { return dfc{dsplit(v.x), dsplit(v.y)}; }
  static __device__ __forceinline__ double norm2_d(C v) {
    const double2 d = to_d2(v);
    return d.x * d.x + d.y * d.y;
  }
  static __device__ __forceinline__ double tval(T t) { return dval(t); }
  static __device__ __forceinline__ df half(df a) { return df{0.5f * a.h, 0.5f * a.l}; }  // exact
  static __device__ __forceinline__ C half_comb(C p, C q, int par) {
    return par > 0 ? dfc{half(dadd(p.x, q.x)), half(dadd(p.y, q.y))}
                   : dfc{half(dsub(p.x, q.x)), half(dsub(p.y, q.y))};
  }
  struct Dot {
    df re{0.f, 0.f}, im{0.f, 0.f};
    __device__ __forceinline__ void add(C f, C p) {
      re = dadd(re, dmul_add(f.x, p.x, f.y, p.y));
      im = dadd(im, dmul_sub(f.x, p.y, f.y, p.x));
    }
    __device__ __forceinline__ double2 value() const { return double2{dval(re), dval(im)}; }
  };
  struct Acc {
    df s{0.f, 0.f};
    __device__ __forceinline__ void add_norm(C v) {
      // |v|^2 = xh^2 + 2 xh xl + yh^2 + 2 yh yl (+ O(2^-48))
      const df a = two_prod(v.x.h, v.x.h), b = two_prod(v.y.h, v.y.h);
      df t = two_sum(a.h, b.h);
      float e = __fadd_rn(t.l, __fadd_rn(a.l, b.l));
      e = __fmaf_rn(2.f * v.x.h, v.x.l, e);
      e = __fmaf_rn(2.f * v.y.h, v.y.l, e);
      s = dadd(s, fast_two_sum(t.h, e));
    }
    __device__ __forceinline__ double value() const { return dval(s); }
  };
  // energy partials in double-float (|v|^2 as in Acc, products by dmul)
  static __device__ __forceinline__ df norm2_df(C v) { return dadd(dmul(v.x, v.x), dmul(v.y, v.y)); }
  struct Full {
    df n2{0.f, 0.f}, pv{0.f, 0.f};
    __device__ __forceinline__ void add(C v, VT vv) {
      const df a2 = norm2_df(v);
      n2 = dadd(n2, a2);
      pv = dadd(pv, dmul(a2, vv));
    }
  };
  struct Pars {
    df pt{0.f, 0.f};
    __device__ __forceinline__ void add(T tk, C v) { pt = dadd(pt, dmul(norm2_df(v), tk)); }
  };
};

// ============================================================ FFT planning
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// E elements per thread and the radix schedule of a length-N transform.
// Schedule R = 0:
//   N = 2^p: E = 8; floor(p/3) radix-8 stages, then one radix-2 or radix-4 stage.
//   N = 12 * 2^p (96, 192): E = 12; one radix-12 stage, then floor(p/2) radix-4
//   stages and a radix-2 stage when p is odd (every radix divides E).
// Schedule R = 1 (two stages, one exchange; N = 2^p with p >= 7, else as R = 0):
//   E = 2^ceil(p/2); a radix-E stage, then radix N/E (16.8 for 128, 16.16 for
//   256, 32.16 for 512, 32.32 for 1024).  Four times the registers of R = 0
//   for half the shared-memory exchanges: used by the complex64 y and z passes
//   when the autotuner finds it faster.
template <int N, int R = 0> struct FftPlan {
  static constexpr bool R3 = N % 3 == 0;
  static constexpr int P2 = ilog2c(N);
  static constexpr bool TWO = R == 1 && !R3 && P2 >= 7;
  static constexpr int E = TWO ? (1 << ((P2 + 1) / 2)) : (R3 ? 12 : 8);
  static constexpr int T = N / E;  // threads per line
  static constexpr int P = ilog2c(R3 ? N / 12 : N);
  static constexpr int Q = R3 ? P / 2 : P / 3;
  static constexpr int REM = R3 ? P % 2 : P % 3;
  static constexpr int S = TWO ? 2 : (R3 ? 1 + Q + REM : Q + (REM ? 1 : 0));
  __host__ __device__ static constexpr int radix(int i) {
    return TWO ? (i == 0 ? E : N / E) : R3 ? (i == 0 ? 12 : (i <= Q ? 4 : 2)) : (i < Q ? 8 : (REM == 1 ? 2 : 4));
  }
  __host__ __device__ static constexpr int ns(int i) { return i == 0 ? 1 : ns(i - 1) * radix(i - 1); }
};

// Complex constants in the representation of C.
__device__ __forceinline__ double2 cconst(double re, double im, double2) { return double2{re, im}; }
__device__ __forceinline__ float2 cconst(double re, double im, float2) { return float2{(float)re, (float)im}; }
__device__ __forceinline__ dfc cconst(double re, double im, dfc) { return dfc{dsplit(re), dsplit(im)}; }

template <int DIR, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd_l(t, b);
  b = csub_l(t, b);
}
template <int DIR, typename C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C s0 = cadd_l(x0, x2), d0 = csub_l(x0, x2);
  C s1 = cadd_l(x1, x3), d1 = mul_i<DIR>(csub_l(x1, x3));
  x0 = cadd_l(s0, s1);
  x2 = csub_l(s0, s1);
  x1 = cadd_l(d0, d1);
  x3 = csub_l(d0, d1);
}
// DFT-3 with w = exp(DIR 2 pi i / 3): X0 = a + s, X1,2 = a - s/2 -+ DIR i (sqrt3/2) (b - c),
// s = b + c (normalised sums; used by the radix-12 butterfly only).
template <int DIR, typename C> __device__ __forceinline__ void dft3(C& a, C& b, C& c) {
  const C s = cadd(b, c), d = csub(b, c);
  const C m = csub(a, cmul(s, cconst(0.5, 0.0, C{})));
  const C r = mul_i<DIR>(cmul(d, cconst(0.86602540378443864676, 0.0, C{})));
  a = cadd(a, s);
  b = cadd(m, r);
  c = csub(m, r);
}
// DFT-12 as 3 x 4 (Cooley-Tukey): DFT-3 over x[n2 + 4 n1] for each n2, the
// factors w12^(n2 k1), DFT-4 over n2 for each k1; X[k1 + 3 k2].
template <int DIR, typename C> __device__ __forceinline__ void dft12(C* x) {
  C y[4][3];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C a = x[n2], b = x[n2 + 4], c = x[n2 + 8];
    dft3<DIR>(a, b, c);
    y[n2][0] = a;
    y[n2][1] = b;
    y[n2][2] = c;
  }
  const double h = 0.5, r3 = 0.86602540378443864676, sg = DIR > 0 ? 1.0 : -1.0;
  y[1][1] = cmul(y[1][1], cconst(r3, sg * h, C{}));   // w12^1
  y[1][2] = cmul(y[1][2], cconst(h, sg * r3, C{}));   // w12^2
  y[2][1] = cmul(y[2][1], cconst(h, sg * r3, C{}));   // w12^2
  y[2][2] = cmul(y[2][2], cconst(-h, sg * r3, C{}));  // w12^4
  y[3][1] = mul_i<DIR>(y[3][1]);                      // w12^3
  y[3][2] = cmul(y[3][2], cconst(-1.0, 0.0, C{}));    // w12^6
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    C a = y[0][k1], b = y[1][k1], c = y[2][k1], d = y[3][k1];
    dft4<DIR>(a, b, c, d);
    x[k1] = a;
    x[k1 + 3] = b;
    x[k1 + 6] = c;
    x[k1 + 9] = d;
  }
}
// a * exp(DIR 2 pi i m / M) for M = 16 or 32 (0 <= m < M): quarter turns as
// exchanges, odd eighth turns through mul_w8, other angles as a product with
// the constant cos + DIR i sin of m pi (32 / M) / 16.
template <int M, int DIR, typename C> __device__ __forceinline__ C mul_wm(C a, int m) {
  // cos(j pi / 16), j = 0..8
  constexpr double CS[9] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
                            0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173,
                            0.19509032201612826785, 0.0};
  const int m32 = m * (32 / M);
  const int q = m32 / 8, r = m32 % 8;
  if (r == 0) {
    if (q == 0) return a;
    if (q == 1) return mul_i<DIR>(a);
    if (q == 2) return cscale(a, decltype(a.x)(-1));
    return cscale(mul_i<DIR>(a), decltype(a.x)(-1));
  }
  if (r == 4) {
    const C b = mul_w8<DIR>(a);
    if (q == 0) return b;
    if (q == 1) return mul_i<DIR>(b);
    if (q == 2) return cscale(b, decltype(a.x)(-1));
    return cscale(mul_i<DIR>(b), decltype(a.x)(-1));
  }
  const double c0 = CS[r], s0 = CS[8 - r];
  const double c = q == 0 ? c0 : q == 1 ? -s0 : q == 2 ? -c0 : s0;
  const double s = q == 0 ? s0 : q == 1 ? c0 : q == 2 ? -s0 : -c0;
  return cmul(a, cconst(c, DIR > 0 ? s : -s, C{}));
}

template <int RAD, int DIR, typename C> __device__ __forceinline__ void dft_small(C* x);

// DFT of length N1 N2 as N1 x N2 (Cooley-Tukey): with n = N2 n1 + n2 and
// k = k1 + N1 k2, DFT-N1 over n1 for each n2, the factors
// exp(DIR 2 pi i n2 k1 / (N1 N2)), DFT-N2 over n2 for each k1; X[k] in
// natural order.  Used for the radix-16 (4 x 4) and radix-32 (4 x 8) stages.
template <int N1, int N2, int DIR, typename C> __device__ __forceinline__ void dft_ct(C* x) {
  C y[N2][N1];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) {
    C t[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) t[n1] = x[N2 * n1 + n2];
    dft_small<N1, DIR>(t);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) y[n2][k1] = (n2 && k1) ? mul_wm<N1 * N2, DIR>(t[k1], n2 * k1) : t[k1];
  }
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    C t[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) t[n2] = y[n2][k1];
    dft_small<N2, DIR>(t);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) x[k1 + N1 * k2] = t[k2];
  }
}

template <int DIR, typename C> __device__ __forceinline__ void dft8(C* x) {
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  o1 = mul_w8<DIR>(o1);
  o2 = mul_i<DIR>(o2);
  o3 = mul_i<DIR>(mul_w8<DIR>(o3));
  x[0] = cadd_l(e0, o0);
  x[4] = csub_l(e0, o0);
  x[1] = cadd_l(e1, o1);
  x[5] = csub_l(e1, o1);
  x[2] = cadd_l(e2, o2);
  x[6] = csub_l(e2, o2);
  x[3] = cadd_l(e3, o3);
  x[7] = csub_l(e3, o3);
}

template <int RAD, int DIR, typename C> __device__ __forceinline__ void dft_small(C* x) {
  if constexpr (RAD == 2) dft2<DIR>(x[0], x[1]);
  if constexpr (RAD == 4) dft4<DIR>(x[0], x[1], x[2], x[3]);
  if constexpr (RAD == 8) dft8<DIR>(x);
}

// Twiddled radix-8 butterfly of the complex128 stages with scaled twiddles
// (the tangent form of Linzer and Feig).  Each twiddle is w_r = s_r q_r with
// q_r = 1 + i tan(theta_r) where |cos| >= |sin|, else q_r = cot(theta_r) + i,
// so |s_r| >= 1/sqrt 2 and |tan|, |cot| <= 1.  x_r q_r takes two FMAs, and the
// real factors s_r enter, as ratios, the multiply-adds that replace the
// DFT-8's additions: 70 FP64 operations a butterfly against 84 for seven
// complex products and the DFT-8 (the FP64 pipe bounds the complex128 passes).
// The host table after the N plain twiddles holds, per direction (forward,
// then inverse) and e0 < N/8, eight double2: the form bits (bit r set: cot
// form, stored as the low word of a double), tan or cot of w^r for r = 1..7,
// s_1, s_2, s_4, s_3/s_1, s_5/s_1, s_6/s_2, s_7/s_3 and s_1/sqrt 2.
__device__ __forceinline__ double neg_bits(double v) {  // -v by the sign bit (no FP64 operation)
  return __hiloint2double(__double2hiint(v) ^ (int)0x80000000, __double2loint(v));
}
__device__ __forceinline__ double2 rot_q(double2 a, double tc, bool cot) {
  // tan form: (a.x - tc a.y, a.y + tc a.x); cot form: (tc a.x - a.y, tc a.y + a.x)
  const double p = cot ? a.x : a.y, c = cot ? neg_bits(a.y) : a.x, tr = cot ? tc : neg_bits(tc);
  const double m = cot ? a.y : a.x, d = cot ? a.x : a.y;
  return double2{fma(tr, p, c), fma(tc, m, d)};
}
__device__ __forceinline__ double2 axpy2(double2 a, double s, double2 b) {  // a + s b
  return double2{fma(s, b.x, a.x), fma(s, b.y, a.y)};
}
// (1 + DIR i) a: the additions of the multiplication by exp(DIR 2 pi i / 8) without 1/sqrt 2
template <int DIR> __device__ __forceinline__ double2 w8_sum(double2 a) {
  return DIR > 0 ? double2{a.x - a.y, a.x + a.y} : double2{a.x + a.y, a.y - a.x};
}
template <int DIR, int N>
__device__ __forceinline__ void scaled_bfly8(double2 (&x)[8], const double2* __restrict__ tw, int e0) {
  const double2* te = tw + N + (DIR < 0 ? 0 : N) + e0 * 8;
  double2 q[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) q[i] = __ldg(te + i);
  const int fl = __double2loint(q[0].x);
  const double tc[8] = {0.0, q[0].y, q[1].x, q[1].y, q[2].x, q[2].y, q[3].x, q[3].y};
  const double s1 = q[4].x, s2 = q[4].y, s4 = q[5].x, r13 = q[5].y, r15 = q[6].x, r26 = q[6].y, r37 = q[7].x,
               kap = q[7].y;
  double2 z[8];
  z[0] = x[0];
#pragma unroll
  for (int r = 1; r < 8; ++r) z[r] = rot_q(x[r], tc[r], (fl >> r) & 1);
  // even inputs (z0, s2 z2, s4 z4, s2 r26 z6): DFT-4 with s2 folded in
  const double2 s0 = axpy2(z[0], s4, z[4]), d0 = axpy2(z[0], -s4, z[4]);
  const double2 s1p = axpy2(z[2], r26, z[6]), d1p = mul_i<DIR>(axpy2(z[2], -r26, z[6]));
  const double2 E0 = axpy2(s0, s2, s1p), E2 = axpy2(s0, -s2, s1p);
  const double2 E1 = axpy2(d0, s2, d1p), E3 = axpy2(d0, -s2, d1p);
  // odd inputs over s1: (z1, r13 z3, r15 z5, r13 r37 z7)
  const double2 t0 = axpy2(z[1], r15, z[5]), u0 = axpy2(z[1], -r15, z[5]);
  const double2 t1 = axpy2(z[3], r37, z[7]), u1 = mul_i<DIR>(axpy2(z[3], -r37, z[7]));
  const double2 O0 = axpy2(t0, r13, t1), O2 = mul_i<DIR>(axpy2(t0, -r13, t1));
  const double2 O1 = w8_sum<DIR>(axpy2(u0, r13, u1)), O3 = mul_i<DIR>(w8_sum<DIR>(axpy2(u0, -r13, u1)));
  x[0] = axpy2(E0, s1, O0);
  x[4] = axpy2(E0, -s1, O0);
  x[2] = axpy2(E2, s1, O2);
  x[6] = axpy2(E2, -s1, O2);
  x[1] = axpy2(E1, kap, O1);
  x[5] = axpy2(E1, -kap, O1);
  x[3] = axpy2(E3, kap, O3);
  x[7] = axpy2(E3, -kap, O3);
}

// One Stockham stage on the register-resident canonical set v[m] = x[t + m N/E].
// Butterfly b = t + u N/E (u < E/RAD) takes x[b + r N/RAD] = v[u + r (E/RAD)],
// multiplies input r by w_N^{(b mod NS) r N/(NS RAD)}, and applies DFT_RAD.
// TWC: the twiddles of a stage from one sincospif and products of powers
// instead of table loads (complex64 only; used where the table loads compete
// with the shared-memory exchanges for the L1 pipe: the z-pass and the
// inverse y pass).
template <class A, int N, int R, int RAD, int NS, int DIR, bool LAST, bool TWC = false>
__device__ __forceinline__ void stage_compute(typename A::C (&v)[FftPlan<N, R>::E], int t,
                                              const typename A::C* __restrict__ tw) {
  using C = typename A::C;
  constexpr int E = FftPlan<N, R>::E;
  constexpr int NB = E / RAD;
  // complex128 twiddled radix-8 stages: the scaled-twiddle butterfly
  constexpr bool SCALED = A::id == 0 && RAD == 8 && NS > 1 && R == 0;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    C x[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) x[r] = v[u + r * NB];
    if constexpr (SCALED) {
      const int b = t + u * (N / E);
      scaled_bfly8<DIR, N>(x, tw, (b % NS) * (N / (NS * RAD)));
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[u + r * NB] = x[r];
      continue;
    }
    if (NS > 1) {
      const int b = t + u * (N / E);
      const int e0 = (b % NS) * (N / (NS * RAD));
      if constexpr (TWC && A::id == 1) {
        // w = exp(-2 pi i e0 / N) from sincospif, its powers by products
        // (a few ulp of FP32, like the rounding of the transform itself)
        float sn, cs;
        sincospif(-2.0f * (float)e0 / (float)N, &sn, &cs);
        C w[RAD];
        w[1] = C{cs, sn};
#pragma unroll
        for (int r = 2; r < RAD; ++r) w[r] = cmul(w[r / 2], w[r - r / 2]);
#pragma unroll
        for (int r = 1; r < RAD; ++r) x[r] = DIR < 0 ? cmul(x[r], w[r]) : cmulc(x[r], w[r]);
      } else {
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          const C w = A::ldtw(&tw[e0 * r]);
          x[r] = DIR < 0 ? cmul(x[r], w) : cmulc(x[r], w);
        }
      }
    }
    if constexpr (RAD == 32) dft_ct<4, 8, DIR>(x);
    if constexpr (RAD == 16) dft_ct<4, 4, DIR>(x);
    if constexpr (RAD == 12) dft12<DIR>(x);
    if constexpr (RAD == 8) dft8<DIR>(x);
    if constexpr (RAD == 4) dft4<DIR>(x[0], x[1], x[2], x[3]);
    if constexpr (RAD == 2) dft2<DIR>(x[0], x[1]);
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[u + r * NB] = cnorm(x[r]);
  }
}

// Writes stage outputs to their Stockham positions, then reads the canonical set.
template <typename C, int N, int R, int RAD, int NS, class Acc>
__device__ __forceinline__ void stage_exchange(C (&v)[FftPlan<N, R>::E], int t, Acc& acc) {
  constexpr int E = FftPlan<N, R>::E;
  constexpr int NB = E / RAD;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int b = t + u * (N / E);
    const int base = (b / NS) * NS * RAD + (b % NS);
#pragma unroll
    for (int r = 0; r < RAD; ++r) acc.at(base + r * NS) = v[u + r * NB];
  }
  acc.sync();
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = acc.at(t + m * (N / E));
  acc.sync();
}

template <class A, int N, int R, int DIR, int I, bool TWC, class Acc>
__device__ __forceinline__ void fft_stages(typename A::C (&v)[FftPlan<N, R>::E], int t,
                                           const typename A::C* __restrict__ tw, Acc& acc) {
  using PL = FftPlan<N, R>;
  if constexpr (I < PL::S) {
    constexpr int RAD = PL::radix(I);
    constexpr int NS = PL::ns(I);
    stage_compute<A, N, R, RAD, NS, DIR, I + 1 == PL::S, TWC>(v, t, tw);
    if constexpr (I + 1 < PL::S) stage_exchange<typename A::C, N, R, RAD, NS>(v, t, acc);
    fft_stages<A, N, R, DIR, I + 1, TWC>(v, t, tw, acc);
  }
}

// Unnormalised length-N DFT, sign DIR, canonical layout in and out, radix
// schedule R.
template <class A, int N, int DIR, class Acc, bool TWC = false, int R = 0>
__device__ __forceinline__ void fft_line(typename A::C (&v)[FftPlan<N, R>::E], int t,
                                         const typename A::C* __restrict__ tw, Acc& acc) {
  fft_stages<A, N, R, DIR, 0, TWC>(v, t, tw, acc);
}

// Shared-memory views. Tile of CW columns of a strided axis: [pos][col] with a
// row pitch of PITCH >= CW elements.  (Rows of 64 bytes take twice the
// minimum shared-memory wavefronts in the first exchange, where each thread
// writes its E outputs E rows apart; a padding row every E rows removes that
// but was measured slower at 512^3, by the index arithmetic it adds to every
// access, so the tiles are unpadded.)  The columns of a tile interleave across
// all warps of the CTA, so an exchange synchronises the whole CTA.
template <typename C, int CW, int PITCH> struct AccTile {
  C* sm;
  int col;
  __device__ __forceinline__ C& at(int pos) { return sm[pos * PITCH + col]; }
  __device__ __forceinline__ void sync() { __syncthreads(); }
};
// One contiguous line of T threads, padded by one element every 2^PS elements
// (128 bytes for the radix-8 schedule; every E elements for the two-stage one,
// whose first exchange writes each thread's E outputs contiguously).  Lines
// synchronise independently: a warp barrier when lines do not straddle warps
// (T <= 32), else the named barrier 1 + line (T threads).
template <typename C, int PS, int T> struct AccLine {
  C* sm;
  int line;
  __device__ __forceinline__ C& at(int pos) { return sm[pos + (pos >> PS)]; }
  __device__ __forceinline__ void sync() {
    if constexpr (T <= 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + line), "r"(T) : "memory");
    }
  }
};

// ---------------------------------------------------------- launch shapes
// Tile shapes (overridable at compile time for tuning sweeps).  Strided tiles
// hold COLS contiguous columns and aim at QFD_TILE_TARGET threads; the
// x-direction tiles (stride N^2: one CTA touches the whole lattice) take at
// least QFD_XCOLS_MIN16 / QFD_XCOLS_MIN8 columns of 16- / 8-byte elements, the
// y-direction tiles (stride N) QFD_YCOLS_MIN16 / QFD_YCOLS_MIN8.  z-pass CTAs
// aim at QFD_LINE_TARGET16 / QFD_LINE_TARGET8 threads.
#ifndef QFD_XCOLS_MIN16
#define QFD_XCOLS_MIN16 8
#endif
#ifndef QFD_XCOLS_MIN8
#define QFD_XCOLS_MIN8 16
#endif
#ifndef QFD_YCOLS_MIN16
#define QFD_YCOLS_MIN16 4
#endif
#ifndef QFD_ZG8
#define QFD_ZG8 2
#endif
#ifndef QFD_ZG16
#define QFD_ZG16 1
#endif
#ifndef QFD_YCOLS_MIN8
#define QFD_YCOLS_MIN8 8
#endif
#ifndef QFD_TILE_TARGET
#define QFD_TILE_TARGET 256
#endif
#ifndef QFD_LINE_TARGET16
#define QFD_LINE_TARGET16 256
#endif
#ifndef QFD_LINE_TARGET8
#define QFD_LINE_TARGET8 128
#endif
template <int N, int CMIN> struct TileCols {
  static constexpr int T = N / FftPlan<N>::E;
  static constexpr int C0 = (QFD_TILE_TARGET / T > CMIN) ? QFD_TILE_TARGET / T : CMIN;
  static constexpr int C1 = C0 < 1024 / T ? C0 : 1024 / T;
  static constexpr int value = C1 < N ? C1 : N;
};
template <class A, int N> struct Shape {
  static constexpr bool WIDE = sizeof(typename A::C) >= 16;
  static constexpr int E = FftPlan<N>::E;  // elements per thread
  static constexpr int T = N / E;          // threads per line
  static constexpr int XCOLS = TileCols<N, WIDE ? QFD_XCOLS_MIN16 : QFD_XCOLS_MIN8>::value;
  static constexpr int YCOLS = TileCols<N, WIDE ? QFD_YCOLS_MIN16 : QFD_YCOLS_MIN8>::value;
  static constexpr int XTHREADS = T * XCOLS;
  static constexpr int YTHREADS = T * YCOLS;
  static constexpr int XPITCH = XCOLS;  // shared-memory row pitch of the tiles
  static constexpr int YPITCH = YCOLS;
  static constexpr int LTARGET = WIDE ? QFD_LINE_TARGET16 : QFD_LINE_TARGET8;
  static constexpr int LINES0 = (LTARGET / T) > 1 ? LTARGET / T : 1;
  static constexpr int LINES = LINES0 < N * N ? LINES0 : N * N;  // z-pass lines per CTA
  static constexpr int LINE_THREADS = T * LINES;
  // z-pass line groups per CTA (see k_zpass), when they divide the lines
  static constexpr int ZG0 = WIDE ? QFD_ZG16 : QFD_ZG8;
  static constexpr int ZG = (N * N / LINES) % ZG0 == 0 && N * N / LINES >= ZG0 ? ZG0 : 1;
  // the autotuner's alternatives: y tiles twice as wide (within 1024 threads
  // and N columns), z-pass line groups 1 or 2
  static constexpr int YCOLS2 = 2 * YCOLS * T <= 1024 && N % (2 * YCOLS) == 0 ? 2 * YCOLS : YCOLS;
  static_assert(N % YCOLS == 0 && (N * N) % XCOLS == 0, "tiles must divide the lattice");
  static constexpr int ZG2 = (N * N / LINES) % 2 == 0 && N * N / LINES >= 2 ? 2 : 1;
  // pass A's alternative: tiles of half the width, two CTAs per SM (one CTA's
  // loads then overlap the other's transforms)
  static constexpr int XCOLS2 = XCOLS >= 2 ? XCOLS / 2 : XCOLS;
  // the two-stage radix schedule (complex64 y and z passes, about 150
  // registers a thread at n = 512, 1024): y tiles and z-pass CTAs of about 128
  // threads, so that three CTAs fit an SM; one line group
  static constexpr bool HAS_R1 = A::id == 1 && FftPlan<N, 1>::TWO;
  static constexpr int T1 = FftPlan<N, 1>::T;
  static constexpr int YCOLS_R1 = (128 / T1 < N ? 128 / T1 : N) > 1 ? (128 / T1 < N ? 128 / T1 : N) : 1;
  static constexpr int LINES_R1 = LTARGET / T1 > 1 ? LTARGET / T1 : 1;
  static constexpr int PAD_SHIFT_R1 = ilog2c(FftPlan<N, 1>::E);
  static constexpr int LPAD_R1 = N + (N >> PAD_SHIFT_R1);
  // one padding element per 128 bytes of a line
  static constexpr int PAD_SHIFT = WIDE ? 3 : 4;
  static constexpr int LPAD = N + (N >> PAD_SHIFT);
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

// Block sum of NQ double-float values in double-float, stored as FP64
// partials part[q * nblocks + blockIdx.x] (one conversion per CTA).  Same
// shape as block_reduce_store: serial in thread order below 32 threads, else
// a warp shuffle tree and one across the warps.
template <int NQ>
__device__ __forceinline__ void df_reduce_store(df (&val)[NQ], double* __restrict__ part) {
  __shared__ df red[NQ][32];
  if (blockDim.x < 32) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q][threadIdx.x] = val[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        df s = val[q];
        for (int i = 1; i < (int)blockDim.x; ++i) s = dadd(s, red[q][i]);
        part[(int64_t)q * gridDim.x + blockIdx.x] = dval(s);
      }
    }
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    df s = val[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      s = dadd(s, df{__shfl_down_sync(0xffffffffu, s.h, o), __shfl_down_sync(0xffffffffu, s.l, o)});
    if (lane == 0) red[q][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      df s = lane < nw ? red[q][lane] : df{0.f, 0.f};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        s = dadd(s, df{__shfl_down_sync(0xffffffffu, s.h, o), __shfl_down_sync(0xffffffffu, s.l, o)});
      if (lane == 0) part[(int64_t)q * gridDim.x + blockIdx.x] = dval(s);
    }
  }
}

// The STATS_NORM partial of a CTA (part[blockIdx.x], with 0 for the second
// quantity at part[gridDim.x + blockIdx.x]).  For the FP32-pipe policies the
// per-thread exact double-float sums are reduced in double-float and turned
// into FP64 once per CTA: FP64 instructions issue at a small fraction of the
// FP32 rate on this GPU, and a per-thread conversion and FP64 shuffle tree
// cost as much as a thread's share of a transform.
template <class A>
__device__ __forceinline__ void norm_reduce_store(const typename A::Acc& acc, double* __restrict__ part) {
  if constexpr (A::id == 0) {
    double q[2] = {acc.value(), 0.0};
    block_reduce_store<2>(q, part);
  } else {
    df q[1] = {acc.s};
    df_reduce_store<1>(q, part);
    if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = 0.0;
  }
}

// The STATS_FULL partials (sum |psi|^2, sum V |psi|^2) and the Parseval
// partial (sum T |psi~|^2) of a CTA, in the policy's accumulator.
template <class A>
__device__ __forceinline__ void full_store(const typename A::Full& f, double* __restrict__ part) {
  if constexpr (A::id == 0) {
    double q[2] = {f.n2, f.pv};
    block_reduce_store<2>(q, part);
  } else {
    df q[2] = {f.n2, f.pv};
    df_reduce_store<2>(q, part);
  }
}
template <class A>
__device__ __forceinline__ void pars_store(const typename A::Pars& f, double* __restrict__ part) {
  if constexpr (A::id == 0) {
    double q[1] = {f.pt};
    block_reduce_store<1>(q, part);
  } else {
    df q[1] = {f.pt};
    df_reduce_store<1>(q, part);
  }
}

// Partial-sum modes of the passes that write psi (pass A and forward x):
//   STATS_NONE  no reduction (the common step)
//   STATS_NORM  sum |psi|^2 (steps that end in a normalisation)
//   STATS_FULL  sum |psi|^2 and sum V |psi|^2 (energy checks; FP64 sums for
//               complex128, exact double-float sums on the FP32 pipe otherwise)
enum { STATS_NONE = 0, STATS_NORM = 1, STATS_FULL = 2 };

// ------------------------------------------------------------ lattice batches
// Every step kernel runs one pass over a batch of up to MAX_BATCH lattices of
// one size and arithmetic: blockIdx.y selects the lattice, blockIdx.x the tile,
// so each lattice sees exactly the arithmetic of a launch over it alone.  A
// single lattice is a batch of one: the plan's own steps, the lockstep batches
// and the request server all run the same kernels.  The per-lattice pointers
// and parameters travel as __grid_constant__ kernel parameters.
constexpr int MAX_BATCH = 32;
struct BatchY {  // passes B and D
  void* W[MAX_BATCH];
  const void* tw[MAX_BATCH];
};
struct BatchZ {  // pass C
  void* W[MAX_BATCH];
  const void* tw[MAX_BATCH];
  const void* ktab[MAX_BATCH];
  double* part[MAX_BATCH];  // Parseval partials (energy checks)
  KinParams kp[MAX_BATCH];
};
struct BatchU {  // pass A
  void* W[MAX_BATCH];
  void* psi[MAX_BATCH];
  const void* u[MAX_BATCH];   // per-site update input: {A, B dtau} (F64) or V (F32, DF)
  const void* V[MAX_BATCH];   // V as the energy partials read it
  const double* scale[MAX_BATCH];
  const float* scale_f[MAX_BATCH];
  const void* tw[MAX_BATCH];
  double* part[MAX_BATCH];
  UpdParams up[MAX_BATCH];
  // the TMA-staged pass A (qfd_tma.cuh): device addresses of the tensor maps of
  // W, psi and the update input, and the plan's error flag for bounded waits
  const void* tmap[MAX_BATCH][3];
  int* err[MAX_BATCH];
};
static_assert(sizeof(BatchZ) <= 4096 && sizeof(BatchU) <= 4096, "kernel parameter space");

// ================================================================ kernels

// Pass B / D (and the plain x transform): in-place strided line FFT over tiles
// of COLS contiguous columns.  Tile id ->
// base = (id / tiles_inner) * outer_stride + (id % tiles_inner) * COLS.
// YC (the tile width) is a launch-shape choice of the autotuner; the
// arithmetic of every column is the same for all widths.
template <class A, int N, int DIR, int YC, int R>
__device__ __forceinline__ void fft_strided_body(typename A::C* W, const typename A::C* __restrict__ tw,
                                                 int64_t stride, int tiles_inner, int64_t outer_stride) {
  using C = typename A::C;
  using PL = FftPlan<N, R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int col = threadIdx.x % YC, t = threadIdx.x / YC;
  const int64_t base = (int64_t)(blockIdx.x / tiles_inner) * outer_stride +
                       (int64_t)(blockIdx.x % tiles_inner) * YC + col;
  C v[PL::E];
#pragma unroll
  for (int m = 0; m < PL::E; ++m) v[m] = W[base + (int64_t)(t + m * PL::T) * stride];
  AccTile<C, YC, YC> acc{sm, col};
  // complex64 inverse y pass and the two-stage schedule: computed twiddles
  // (measured faster there; the forward y pass of schedule 0 is faster with
  // the table)
  fft_line<A, N, DIR, decltype(acc), (DIR > 0 || R == 1), R>(v, t, tw, acc);
#pragma unroll
  for (int m = 0; m < PL::E; ++m) W[base + (int64_t)(t + m * PL::T) * stride] = v[m];
}
// Resident CTAs per SM asked of the compiler for the y passes: complex64
// keeps about 48 warps per SM (register-light transforms whose exchanges need
// many warps in flight), the 16-byte arithmetics take what their registers allow.
template <class A, int N, int YC> struct YOcc {
  static constexpr int THREADS = N / FftPlan<N>::E * YC;
  static constexpr int B0 = A::id == 1 ? 1536 / THREADS : 1;
  static constexpr int value = B0 < 1 ? 1 : (B0 > 8 ? 8 : B0);
};
template <class A, int N, int DIR, int YC, int R = 0>
__global__ void __launch_bounds__(FftPlan<N, R>::T * YC, R == 0 ? YOcc<A, N, YC>::value : 1)
k_fft_strided(const __grid_constant__ BatchY b, int64_t stride, int tiles_inner, int64_t outer_stride) {
  using C = typename A::C;
  fft_strided_body<A, N, DIR, YC, R>(static_cast<C*>(b.W[blockIdx.y]), static_cast<const C*>(b.tw[blockIdx.y]),
                                     stride, tiles_inner, outer_stride);
}

// Pass C: forward DFT_z, times T(k)/N^3 (+ Parseval partial when PARSEVAL),
// inverse DFT_z.  The canonical layout is the same before and after a
// transform, so the multiply sits in registers between the two transforms.
// A CTA takes ZG groups of LINES consecutive lines in turn; the loads of the
// next group are issued before the current group's transforms, so they are in
// flight while it computes.
// R: the radix schedule (FftPlan); LINES lines of T threads per CTA.
template <class A, int N, bool PARSEVAL, int ZG, int R, int LINES>
__device__ __forceinline__ void zpass_body(typename A::C* W, const typename A::C* __restrict__ tw,
                                           const typename A::T* __restrict__ ktab, const KinParams& kp,
                                           double* __restrict__ part) {
  using C = typename A::C;
  using T = typename A::T;
  using SH = Shape<A, N>;
  using PL = FftPlan<N, R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int l = threadIdx.x / PL::T, t = threadIdx.x % PL::T;
  const int64_t line0 = (int64_t)blockIdx.x * LINES * ZG + l;  // line = kx * N + ky
  C v[PL::E];
#pragma unroll
  for (int m = 0; m < PL::E; ++m) v[m] = W[line0 * N + t + m * PL::T];
  static_assert(PL::T <= 32 || LINES <= 15, "one named barrier per line");
  constexpr int PS = R == 0 ? SH::PAD_SHIFT : SH::PAD_SHIFT_R1;
  constexpr int LP = R == 0 ? SH::LPAD : SH::LPAD_R1;
  AccLine<C, PS, PL::T> acc{sm + l * LP, l};
  typename A::Pars pacc;
#pragma unroll
  for (int g = 0; g < ZG; ++g) {
    const int64_t line = line0 + (int64_t)g * LINES;
    C* p = W + line * N;
    C nx[ZG > 1 ? PL::E : 1];
    if (g + 1 < ZG) {
#pragma unroll
      for (int m = 0; m < PL::E; ++m) nx[m] = p[(int64_t)LINES * N + t + m * PL::T];
    }
    fft_line<A, N, -1, decltype(acc), true, R>(v, t, tw, acc);
    const T sxy = A::kadd(ktab[line / N], ktab[line % N]);
#pragma unroll
    for (int m = 0; m < PL::E; ++m) {
      const T tk = A::kin(A::kadd(sxy, ktab[t + m * PL::T]), kp);
      if constexpr (PARSEVAL) pacc.add(tk, v[m]);
      v[m] = cscale(v[m], tk);
    }
    fft_line<A, N, +1, decltype(acc), true, R>(v, t, tw, acc);
#pragma unroll
    for (int m = 0; m < PL::E; ++m) p[t + m * PL::T] = v[m];
    if (g + 1 < ZG) {
#pragma unroll
      for (int m = 0; m < PL::E; ++m) v[m] = nx[m];
    }
  }
  if constexpr (PARSEVAL) pars_store<A>(pacc, part);
}
template <class A, int N, int R> struct ZLines {
  static constexpr int value = R == 0 ? Shape<A, N>::LINES : Shape<A, N>::LINES_R1;
};
template <class A, int N, bool PARSEVAL, int ZG, int R = 0>
__global__ void __launch_bounds__(FftPlan<N, R>::T * ZLines<A, N, R>::value) k_zpass(const __grid_constant__ BatchZ b) {
  using C = typename A::C;
  const int i = blockIdx.y;
  zpass_body<A, N, PARSEVAL, ZG, R, ZLines<A, N, R>::value>(static_cast<C*>(b.W[i]), static_cast<const C*>(b.tw[i]),
                                                             static_cast<const typename A::T*>(b.ktab[i]), b.kp[i],
                                                             b.part[i]);
}

// Pass A: inverse DFT_x of W gives H_K psi at the tile's sites; the update of
// Eq. (iter_proced) with the coefficients of Sec. 2.2 (read precomputed for
// complex128, derived from V in the FP32-pipe arithmetics), times an optional
// normalisation factor s carried from the previous step; partial sums per
// STATS; forward DFT_x of the new psi into W.  The core takes a thread's
// column of W, psi and the update input already in registers, so that the
// direct kernel (loads from global memory) and the TMA-staged one (loads from
// shared memory) run the same arithmetic code.  XC is the tile width.
template <class A, int N, int STATS, int XC>
__device__ __forceinline__ void update_x_core(typename A::C (&v)[FftPlan<N>::E], const typename A::C (&ps)[FftPlan<N>::E],
                                              const typename A::U (&cf)[FftPlan<N>::E], int t, int col, int64_t base,
                                              typename A::C* W, typename A::C* __restrict__ psi, const UpdParams& upar,
                                              const typename A::VT* __restrict__ V, const double* __restrict__ scale,
                                              const float* __restrict__ scale_f, const typename A::C* __restrict__ tw,
                                              typename A::C* sm, typename A::Acc& nacc, typename A::Full& facc) {
  using C = typename A::C;
  using SH = Shape<A, N>;
  constexpr int64_t S = (int64_t)N * N;
  AccTile<C, XC, XC> acc{sm, col};
  fft_line<A, N, +1>(v, t, tw, acc);
  const bool scaled = scale != nullptr;
  typename A::S s{};
  if (scaled) s = A::load_scale(scale, scale_f);
#pragma unroll
  for (int m = 0; m < SH::E; ++m) {
    const int64_t idx = base + (t + m * SH::T) * S;
    C nw = A::update(ps[m], v[m], A::coef_from(cf[m], upar));
    if (scaled) nw = cscale(nw, s);
    psi[idx] = nw;
    v[m] = nw;
    if constexpr (STATS == STATS_NORM) nacc.add_norm(nw);
    if constexpr (STATS == STATS_FULL) facc.add(nw, V[idx]);
  }
  fft_line<A, N, -1>(v, t, tw, acc);
#pragma unroll
  for (int m = 0; m < SH::E; ++m) W[base + (t + m * SH::T) * S] = v[m];
}

// The direct pass A: psi and the per-site update input are loaded before the
// inverse transform so that their latency overlaps it.
template <class A, int N, int STATS, int XC>
__device__ __forceinline__ void update_x_body(typename A::C* W, typename A::C* __restrict__ psi,
                                              const typename A::U* __restrict__ uin, const UpdParams& upar,
                                              const typename A::VT* __restrict__ V, const double* __restrict__ scale,
                                              const float* __restrict__ scale_f, const typename A::C* __restrict__ tw,
                                              double* __restrict__ part) {
  using C = typename A::C;
  using U = typename A::U;
  using SH = Shape<A, N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int col = threadIdx.x % XC, t = threadIdx.x / XC;
  const int64_t base = (int64_t)blockIdx.x * XC + col;
  constexpr int64_t S = (int64_t)N * N;
  C v[SH::E], ps[SH::E];
  U cf[SH::E];
#pragma unroll
  for (int m = 0; m < SH::E; ++m) v[m] = W[base + (t + m * SH::T) * S];
#pragma unroll
  for (int m = 0; m < SH::E; ++m) ps[m] = psi[base + (t + m * SH::T) * S];
#pragma unroll
  for (int m = 0; m < SH::E; ++m) cf[m] = uin[base + (t + m * SH::T) * S];
  typename A::Acc nacc;
  typename A::Full facc;
  update_x_core<A, N, STATS, XC>(v, ps, cf, t, col, base, W, psi, upar, V, scale, scale_f, tw, sm, nacc, facc);
  if constexpr (STATS == STATS_NORM) norm_reduce_store<A>(nacc, part);
  if constexpr (STATS == STATS_FULL) full_store<A>(facc, part);
}
// Lattice i of the batch applies its pending normalisation factor when bit i
// of `scaled` is set.  The half-width tiles (XC < XCOLS) are compiled for two
// resident CTAs per SM.
template <class A, int N, int STATS, int XC>
__global__ void __launch_bounds__(N / FftPlan<N>::E * XC, XC < Shape<A, N>::XCOLS ? 2 : 1)
k_update_x(const __grid_constant__ BatchU b, uint32_t scaled) {
  using C = typename A::C;
  const int i = blockIdx.y;
  update_x_body<A, N, STATS, XC>(static_cast<C*>(b.W[i]), static_cast<C*>(b.psi[i]),
                                 static_cast<const typename A::U*>(b.u[i]), b.up[i],
                                 static_cast<const typename A::VT*>(b.V[i]), (scaled >> i) & 1u ? b.scale[i] : nullptr,
                                 b.scale_f[i], static_cast<const C*>(b.tw[i]), b.part[i]);
}

// Forward DFT_x of src (optionally times *scale, optionally also written to
// psi_out) into W; partials per STATS of the scaled input.  src may alias W
// (each CTA reads its whole tile before writing it).
template <class A, int N, int STATS>
__global__ void __launch_bounds__(Shape<A, N>::XTHREADS)
k_forward_x(const typename A::C* src, typename A::C* W, typename A::C* psi_out, const typename A::VT* __restrict__ V,
            const double* __restrict__ scale, const float* __restrict__ scale_f, const typename A::C* __restrict__ tw,
            double* __restrict__ part) {
  using C = typename A::C;
  using SH = Shape<A, N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int col = threadIdx.x % SH::XCOLS, t = threadIdx.x / SH::XCOLS;
  const int64_t base = (int64_t)blockIdx.x * SH::XCOLS + col;
  constexpr int64_t S = (int64_t)N * N;
  const bool scaled = scale != nullptr;
  typename A::S s{};
  if (scaled) s = A::load_scale(scale, scale_f);
  C v[SH::E];
  typename A::Acc nacc;
  typename A::Full facc;
#pragma unroll
  for (int m = 0; m < SH::E; ++m) {
    const int64_t idx = base + (t + m * SH::T) * S;
    C x = src[idx];
    if (scaled) x = cscale(x, s);
    v[m] = x;
    if constexpr (STATS == STATS_NORM) nacc.add_norm(x);
    if constexpr (STATS == STATS_FULL) facc.add(x, V[idx]);
  }
  if (psi_out) {
#pragma unroll
    for (int m = 0; m < SH::E; ++m) psi_out[base + (t + m * SH::T) * S] = v[m];
  }
  AccTile<C, SH::XCOLS, SH::XPITCH> acc{sm, col};
  fft_line<A, N, -1>(v, t, tw, acc);
#pragma unroll
  for (int m = 0; m < SH::E; ++m) W[base + (t + m * SH::T) * S] = v[m];
  if constexpr (STATS == STATS_NORM) norm_reduce_store<A>(nacc, part);
  if constexpr (STATS == STATS_FULL) full_store<A>(facc, part);
}

// ------------------------------------------------- projection and overlaps
constexpr int MAX_LOWER = 8;

// Up to MAX_LOWER lower states (each a whole lattice), passed by value.
struct LowerPtrs {
  const void* p[MAX_LOWER];
};

// Lattice reflection r -> -r about the potential's centre (Eq. (parity)):
// grid centre x -> (N - x) mod N, off-grid centre x -> N - 1 - x.
template <int N>
__device__ __forceinline__ int reflect1(int x, int offgrid) {
  return offgrid ? N - 1 - x : (N - x) % N;
}

// Overlaps <phi_j | P psi> for j < k (P the parity projector of Eq. (parity),
// the identity for parity 0), summed per CTA in the policy's exact
// accumulator and stored as FP64 partials (2 per lower state).
template <class A, int N>
__global__ void __launch_bounds__(256)
k_gs_dots(const typename A::C* __restrict__ psi, LowerPtrs lower, int k, int parity, int offgrid,
          double* __restrict__ part) {
  using C = typename A::C;
  constexpr int64_t N3 = (int64_t)N * N * N;
  typename A::Dot acc[MAX_LOWER];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N3; i += (int64_t)gridDim.x * blockDim.x) {
    C p = psi[i];
    if (parity) {
      const int z = (int)(i % N), y = (int)((i / N) % N), x = (int)(i / ((int64_t)N * N));
      const int64_t ri = ((int64_t)reflect1<N>(x, offgrid) * N + reflect1<N>(y, offgrid)) * N +
                         reflect1<N>(z, offgrid);
      p = A::half_comb(p, psi[ri], parity);
    }
#pragma unroll
    for (int j = 0; j < MAX_LOWER; ++j)
      if (j < k) acc[j].add(static_cast<const C*>(lower.p[j])[i], p);
  }
  double q[2 * MAX_LOWER];
#pragma unroll
  for (int j = 0; j < MAX_LOWER; ++j) {
    const double2 d = acc[j].value();
    q[2 * j] = d.x;
    q[2 * j + 1] = d.y;
  }
  block_reduce_store<2 * MAX_LOWER>(q, part);
}

// The cadence's projection fused with the forward x transform: psi' = P psi -
// sum_j c_j phi_j (c_j = sums[2j] + i sums[2j+1], the overlaps of k_gs_dots)
// is written to dst (a different buffer than src: other CTAs still read the
// reflected sites of src) and its forward DFT_x to W; partials per STATS of
// psi'.  The normalisation is applied by the next pass A.
// LOWER: whether there are lower states (k > 0); the parity-only instance
// carries no Gram-Schmidt code at all.
template <class A, int N, int STATS, bool LOWER = true>
__global__ void __launch_bounds__(Shape<A, N>::XTHREADS)
k_project_x(const typename A::C* __restrict__ src, LowerPtrs lower, const double* __restrict__ sums, int k, int parity,
            int offgrid, typename A::C* __restrict__ dst, typename A::C* __restrict__ W,
            const typename A::VT* __restrict__ V,
            const typename A::C* __restrict__ tw, double* __restrict__ part) {
  using C = typename A::C;
  using SH = Shape<A, N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int col = threadIdx.x % SH::XCOLS, t = threadIdx.x / SH::XCOLS;
  const int64_t base = (int64_t)blockIdx.x * SH::XCOLS + col;  // = y * N + z
  constexpr int64_t S = (int64_t)N * N;
  const int y = (int)(base / N), z = (int)(base % N);
  const int64_t rbase = (int64_t)reflect1<N>(y, offgrid) * N + reflect1<N>(z, offgrid);
  // the overlaps in the policy's representation (converted only when there
  // are lower states: conversions from FP64 run on the slow FP64 pipe)
  C cc[MAX_LOWER];
  if (LOWER && k > 0) {
#pragma unroll
    for (int j = 0; j < MAX_LOWER; ++j)
      if (j < k) cc[j] = A::from_d2(double2{sums[2 * j], sums[2 * j + 1]});
  }
  // every load of the state and of its reflection is issued before any use
  C v[SH::E], rv[SH::E];
#pragma unroll
  for (int m = 0; m < SH::E; ++m) v[m] = src[base + (t + m * SH::T) * S];
  if (parity) {
#pragma unroll
    for (int m = 0; m < SH::E; ++m) rv[m] = src[rbase + (int64_t)reflect1<N>(t + m * SH::T, offgrid) * S];
  }
  typename A::Acc nacc;
  typename A::Full facc;
#pragma unroll
  for (int m = 0; m < SH::E; ++m) {
    const int x = t + m * SH::T;
    const int64_t idx = base + x * S;
    C p = v[m];
    if (parity) p = A::half_comb(p, rv[m], parity);
#pragma unroll
    for (int j = 0; j < MAX_LOWER; ++j)
      if (LOWER && j < k) p = csub(p, cmul(static_cast<const C*>(lower.p[j])[idx], cc[j]));
    dst[idx] = p;
    v[m] = p;
    if constexpr (STATS == STATS_NORM) nacc.add_norm(p);
    if constexpr (STATS == STATS_FULL) facc.add(p, V[idx]);
  }
  AccTile<C, SH::XCOLS, SH::XPITCH> acc{sm, col};
  fft_line<A, N, -1>(v, t, tw, acc);
#pragma unroll
  for (int m = 0; m < SH::E; ++m) W[base + (t + m * SH::T) * S] = v[m];
  if constexpr (STATS == STATS_NORM) norm_reduce_store<A>(nacc, part);
  if constexpr (STATS == STATS_FULL) full_store<A>(facc, part);
}

// psi *= f in the policy's arithmetic, f = scal[0] (mode 0) or 1 / sqrt(scal[1]) (mode 1).
template <class A>
__global__ void k_scale(typename A::C* __restrict__ psi, int64_t n3, const double* __restrict__ f_or_n2, int mode) {
  const double f = mode == 0 ? f_or_n2[0] : 1.0 / sqrt(f_or_n2[0]);
  const typename A::S fs = A::scalar(f);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    psi[i] = cscale(psi[i], fs);
}

// dst = src * f, f = *scale (1 when scale is null), in the policy's arithmetic.
template <class A>
__global__ void k_scale_copy(typename A::C* __restrict__ dst, const typename A::C* __restrict__ src, int64_t n3,
                             const double* __restrict__ scale) {
  const typename A::S fs = A::scalar(scale ? scale[0] : 1.0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = cscale(src[i], fs);
}

}  // namespace qfd
