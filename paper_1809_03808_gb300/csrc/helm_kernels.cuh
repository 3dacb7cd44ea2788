// Device helpers shared by the sm_103a kernels of the Helmholtz fast solver.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "helm_internal.h"

namespace helm {

template <typename T>
struct cpx;
template <>
struct cpx<float> {
  using type = float2;
};
template <>
struct cpx<double> {
  using type = double2;
};

template <typename C>
__device__ __forceinline__ C mk(double re, double im) {
  C c;
  c.x = (decltype(c.x))re;
  c.y = (decltype(c.y))im;
  return c;
}
template <typename C, typename S>
__device__ __forceinline__ C cvt(S s) {
  C c;
  c.x = (decltype(c.x))s.x;
  c.y = (decltype(c.y))s.y;
  return c;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// c + a * b and c - a * b as four fused multiply-adds (one rounding per
// component step instead of a product rounded before the sum)
template <typename C>
__device__ __forceinline__ C cfma(C a, C b, C c) {
  c.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
  c.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
  return c;
}
template <typename C>
__device__ __forceinline__ C cfms(C c, C a, C b) {
  c.x = fma(-a.x, b.x, fma(a.y, b.y, c.x));
  c.y = fma(-a.x, b.y, fma(-a.y, b.x, c.y));
  return c;
}
// Principal square root of a complex FP64 value.
__device__ __forceinline__ double2 csqrt_d(double2 z) {
  const double r = hypot(z.x, z.y);
  double re = sqrt(0.5 * (r + fabs(z.x))), im = 0.0;
  if (re > 0.0) im = 0.5 * z.y / re;
  if (z.x < 0.0) {  // sqrt(z) = |im| + i sign(y) re
    const double t = fabs(im);
    im = z.y < 0.0 ? -re : re;
    re = t;
  }
  return make_double2(re, im);
}

// Prefetch the global-memory line holding p into L2 (no data returned).
__device__ __forceinline__ void l2_prefetch(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
// a * conj(b)
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename C, typename T>
__device__ __forceinline__ C cscale(C a, T s) {
  a.x *= s;
  a.y *= s;
  return a;
}
// 1 / a.  FP64: conj(a) / |a|^2 with one division (the operands of these
// solvers stay within 1e-150..1e150, far inside FP64 range).  FP32: Smith's
// scaling, so that |a|^2 neither over- nor under-flows the narrow exponent.
__device__ __forceinline__ double2 crecip(double2 a) {
  const double inv = 1.0 / fma(a.x, a.x, a.y * a.y);
  return make_double2(a.x * inv, -a.y * inv);
}
template <typename C>
__device__ __forceinline__ C crecip(C a) {
  using T = decltype(a.x);
  C r;
  if (fabs(a.x) >= fabs(a.y)) {
    T q = a.y / a.x;
    T d = a.x + a.y * q;
    T inv = T(1) / d;
    r.x = inv;
    r.y = -q * inv;
  } else {
    T q = a.x / a.y;
    T d = a.x * q + a.y;
    T inv = T(1) / d;
    r.x = q * inv;
    r.y = -inv;
  }
  return r;
}

template <typename C>
__device__ __forceinline__ C shfl_down(C v, int off) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, off);
  v.y = __shfl_down_sync(0xffffffffu, v.y, off);
  return v;
}
template <typename C>
__device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = cadd(v, shfl_down(v, off));
  return v;
}

// Float-float arithmetic: a real value held as hi + lo with |lo| <= ulp(hi)/2
// (about 48 significant bits) and computed on the FP32 pipes.  Built from the
// error-free transformations TwoSum (Knuth), FastTwoSum (Dekker, |a| >= |b|)
// and TwoProduct through a fused multiply-add.  The build never reassociates
// floating-point additions, which these rely on.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// (sh, sl) += (ch + cl) (uh + ul), dropping cl ul (below 2^-48 relative)
__device__ __forceinline__ void ff_mac(float& sh, float& sl, float ch, float cl, float uh, float ul) {
  const float p = ch * uh;
  float e = fmaf(ch, uh, -p);
  e = fmaf(ch, ul, fmaf(cl, uh, e));
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl += t + e;
}
// (hi, lo) += v, renormalised
__device__ __forceinline__ void ff_add_f(float& hi, float& lo, float v) {
  float s, e;
  two_sum(hi, v, s, e);
  fast_two_sum(s, lo + e, hi, lo);
}

// Entries of the 1D mass matrix of one axis: h [(den-2)/den on the interior
// diagonal, half of it at the ends, 1/den off the diagonal].  den = 6 is
// eq. matrixM (the paper's elements, exact integrals); den = 12 the modified
// elements with every integral by the 2-point rule at +-sqrt(2/3) (the mean
// of the consistent and the lumped mass; fourth-order dispersion).
struct MassCoef {
  double in, end, off;
};
__host__ __device__ __forceinline__ MassCoef mass_coef(double h, double den) {
  return MassCoef{(den - 2.0) * h / den, ((den - 2.0) / 2.0) * h / den, h / den};
}

// Line matrix T = K + s M along the tridiagonal axis (eqs. matrixK/matrixM;
// K with absorbing corners 1 - i w h).  diag in the interior, diag at both
// ends, constant off-diagonal.
template <typename C>
struct LineCoef {
  C a;   // interior diagonal
  C ac;  // end diagonal (absorbing corner)
  C b;   // off-diagonal
};

template <typename C>
__device__ __forceinline__ LineCoef<C> line_coef(double sre, double sim, double h, double omega, double den) {
  const MassCoef m = mass_coef(h, den);
  LineCoef<C> c;
  c.a = mk<C>(sre * m.in + 2.0 / h, sim * m.in);
  c.ac = mk<C>(sre * m.end + 1.0 / h, sim * m.end - omega);
  c.b = mk<C>(sre * m.off - 1.0 / h, sim * m.off);
  return c;
}

}  // namespace helm
