// FP64 residual r = f - A u of the Kronecker operators of eq. A2D (9-point)
// and eq. A3D (27-point), used by iterative refinement of the complex64
// solves.  A u is the tensor-product stencil: the coefficient of neighbour
// offset (d_1, ..., d_D) is  sum_j prod_k X^{(j)}_k(i_k, i_k + d_k)
// - w^2 prod_k M_k(i_k, i_k + d_k), with X^{(j)}_k = K_k if k == j else M_k
// (1D matrices of eqs. matrixK / matrixM).  Interior points use precomputed
// real coefficients; points on a face use the complex corner entries.
#include <algorithm>

#include "helm_kernels.cuh"
#include "helm_solve.h"

namespace helm {

namespace {

struct Axis1D {
  int64_t n;
  double h;
};

// 1D entries M(i, i+d) and K(i, i+d) (K complex at the absorbing corners).
__device__ __forceinline__ void entries(const Axis1D& ax, int64_t i, int d, double omega, double& m,
                                        double& kre, double& kim) {
  const bool end = (i == 0 || i == ax.n - 1);
  if (d == 0) {
    m = (end ? 2.0 : 4.0) * ax.h / 6.0;
    kre = (end ? 1.0 : 2.0) / ax.h;
    kim = end ? -omega : 0.0;
  } else {
    m = ax.h / 6.0;
    kre = -1.0 / ax.h;
    kim = 0.0;
  }
}

struct ResidArgs {
  Axis1D ax[3];
  int dim;
  double omega;
  double cin[27];  // interior coefficients, index (d0+1)*9 + (d1+1)*3 + (d2+1) (3D) or (d0+1)*3+(d1+1)
};

// Float-float copies of the coefficients (each value as hi + lo floats).
struct FF2 {
  float h, l;
};
struct AxisFF {
  FF2 mdi, mde, mo;   // M: interior diagonal, end diagonal, off-diagonal
  FF2 kdi, kder, ko;  // K: interior diagonal, end diagonal (real part), off-diagonal
  FF2 kdei;           // K end diagonal, imaginary part (-w)
  FF2 cdi, cde, co;   // K - w^2 M: interior diagonal, end diagonal (real), off-diagonal
};
struct ResidFFArgs {
  int64_t n[3];
  double h[3];
  double omega;
  AxisFF ax[3];
  FF2 cin[9];  // 2D interior coefficients, index (d0+1)*3 + (d1+1)
  // 2D perimeter coefficients (complex: [0] re, [1] im) by the end class of
  // each index (0: first, 1: inside, 2: last), index (d0+1)*3 + (d1+1)
  FF2 per[3][3][9][2];
};

__global__ void __launch_bounds__(256) k_residual(ResidArgs a, const double2* __restrict__ f,
                                                  const double2* __restrict__ u, float2* __restrict__ r,
                                                  double* __restrict__ sums, int64_t N,
                                                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double sr[8], sf[8];
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0, f2 = 0.0;
  if (gid < N) {
    int64_t idx[3] = {0, 0, 0};
    int64_t rem = gid;
    for (int k = a.dim - 1; k >= 0; --k) {
      idx[k] = rem % a.ax[k].n;
      rem /= a.ax[k].n;
    }
    int64_t stride[3];
    stride[a.dim - 1] = 1;
    for (int k = a.dim - 2; k >= 0; --k) stride[k] = stride[k + 1] * a.ax[k + 1].n;
    bool interior = true;
    for (int k = 0; k < a.dim; ++k) interior = interior && idx[k] > 0 && idx[k] < a.ax[k].n - 1;
    double ar = 0.0, ai = 0.0;
    if (a.dim == 2) {
      for (int d0 = -1; d0 <= 1; ++d0) {
        const int64_t i0 = idx[0] + d0;
        if (i0 < 0 || i0 >= a.ax[0].n) continue;
        for (int d1 = -1; d1 <= 1; ++d1) {
          const int64_t i1 = idx[1] + d1;
          if (i1 < 0 || i1 >= a.ax[1].n) continue;
          const double2 v = u[i0 * stride[0] + i1];
          double cre, cim;
          if (interior) {
            cre = a.cin[(d0 + 1) * 3 + (d1 + 1)];
            cim = 0.0;
          } else {
            double m0, k0r, k0i, m1, k1r, k1i;
            entries(a.ax[0], idx[0], d0, a.omega, m0, k0r, k0i);
            entries(a.ax[1], idx[1], d1, a.omega, m1, k1r, k1i);
            cre = k0r * m1 + m0 * k1r - a.omega * a.omega * m0 * m1;
            cim = k0i * m1 + m0 * k1i;
          }
          ar += cre * v.x - cim * v.y;
          ai += cre * v.y + cim * v.x;
        }
      }
    } else {
      for (int d0 = -1; d0 <= 1; ++d0) {
        const int64_t i0 = idx[0] + d0;
        if (i0 < 0 || i0 >= a.ax[0].n) continue;
        for (int d1 = -1; d1 <= 1; ++d1) {
          const int64_t i1 = idx[1] + d1;
          if (i1 < 0 || i1 >= a.ax[1].n) continue;
          for (int d2 = -1; d2 <= 1; ++d2) {
            const int64_t i2 = idx[2] + d2;
            if (i2 < 0 || i2 >= a.ax[2].n) continue;
            const double2 v = u[i0 * stride[0] + i1 * stride[1] + i2];
            double cre, cim;
            if (interior) {
              cre = a.cin[(d0 + 1) * 9 + (d1 + 1) * 3 + (d2 + 1)];
              cim = 0.0;
            } else {
              double m0, k0r, k0i, m1, k1r, k1i, m2, k2r, k2i;
              entries(a.ax[0], idx[0], d0, a.omega, m0, k0r, k0i);
              entries(a.ax[1], idx[1], d1, a.omega, m1, k1r, k1i);
              entries(a.ax[2], idx[2], d2, a.omega, m2, k2r, k2i);
              cre = k0r * m1 * m2 + m0 * k1r * m2 + m0 * m1 * k2r - a.omega * a.omega * m0 * m1 * m2;
              cim = k0i * m1 * m2 + m0 * k1i * m2 + m0 * m1 * k2i;
            }
            ar += cre * v.x - cim * v.y;
            ai += cre * v.y + cim * v.x;
          }
        }
      }
    }
    const double2 fv = f[gid];
    const double rr = fv.x - ar, ri = fv.y - ai;
    r[gid] = make_float2((float)rr, (float)ri);
    r2 = rr * rr + ri * ri;
    f2 = fv.x * fv.x + fv.y * fv.y;
  }
  // block reduction (deterministic)
  for (int off = 16; off > 0; off >>= 1) {
    r2 += __shfl_down_sync(0xffffffffu, r2, off);
    f2 += __shfl_down_sync(0xffffffffu, f2, off);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sr[w] = r2;
    sf[w] = f2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a2 = 0, b2 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a2 += sr[i];
      b2 += sf[i];
    }
    sums[2 * blockIdx.x] = a2;
    sums[2 * blockIdx.x + 1] = b2;
  }
}

// 2D residual, one thread per y column segment of RX rows: rolling
// registers over x (rows x-1, x, x+1 of the three y neighbours), interior
// points with the nine precomputed real coefficients.
constexpr int RX2 = 16;

__global__ void __launch_bounds__(256) k_residual2d(ResidArgs a, const double2* __restrict__ f,
                                                    const double2* __restrict__ u, float2* __restrict__ r,
                                                    double* __restrict__ sums, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double sr[8], sf[8];
  const int64_t nx = a.ax[0].n, ny = a.ax[1].n;
  const int64_t iy = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t x0 = (int64_t)blockIdx.y * RX2;
  // |r|^2 and |f|^2 only decide convergence: per-thread sums in FP32 (from the
  // rounded values), FP64 across threads and blocks
  float r2f = 0.f, f2f = 0.f;
  double r2 = 0.0, f2 = 0.0;
  if (iy < ny) {
    const bool ym = iy > 0, yp = iy < ny - 1;
    auto ld = [&](int64_t ix, int64_t jy) -> double2 {
      return (ix >= 0 && ix < nx) ? __ldg(&u[ix * ny + jy]) : make_double2(0.0, 0.0);
    };
    double2 w[3][3];  // [dx+1][dy+1]
    for (int d = 0; d < 2; ++d) {
      const int64_t ix = x0 - 1 + d;
      w[d][0] = ym ? ld(ix, iy - 1) : make_double2(0, 0);
      w[d][1] = ld(ix, iy);
      w[d][2] = yp ? ld(ix, iy + 1) : make_double2(0, 0);
    }
    const int64_t x1 = min(x0 + RX2, nx);
    for (int64_t ix = x0; ix < x1; ++ix) {
      w[2][0] = ym ? ld(ix + 1, iy - 1) : make_double2(0, 0);
      w[2][1] = ld(ix + 1, iy);
      w[2][2] = yp ? ld(ix + 1, iy + 1) : make_double2(0, 0);
      double ar = 0.0, ai = 0.0;
      const bool interior = ix > 0 && ix < nx - 1 && iy > 0 && iy < ny - 1;
      if (interior) {
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            const double c = a.cin[dx * 3 + dy];
            ar = fma(c, w[dx][dy].x, ar);
            ai = fma(c, w[dx][dy].y, ai);
          }
      } else {
        for (int dx = -1; dx <= 1; ++dx) {
          if (ix + dx < 0 || ix + dx >= nx) continue;
          double m0, k0r, k0i;
          entries(a.ax[0], ix, dx, a.omega, m0, k0r, k0i);
          for (int dy = -1; dy <= 1; ++dy) {
            if (iy + dy < 0 || iy + dy >= ny) continue;
            double m1, k1r, k1i;
            entries(a.ax[1], iy, dy, a.omega, m1, k1r, k1i);
            const double cre = k0r * m1 + m0 * k1r - a.omega * a.omega * m0 * m1;
            const double cim = k0i * m1 + m0 * k1i;
            const double2 v = w[dx + 1][dy + 1];
            ar += cre * v.x - cim * v.y;
            ai += cre * v.y + cim * v.x;
          }
        }
      }
      const double2 fv = __ldg(&f[ix * ny + iy]);
      const float2 rf = make_float2((float)(fv.x - ar), (float)(fv.y - ai));
      r[ix * ny + iy] = rf;
      const float2 ff = make_float2((float)fv.x, (float)fv.y);
      r2f = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, r2f));
      f2f = fmaf(ff.x, ff.x, fmaf(ff.y, ff.y, f2f));
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        w[0][dy] = w[1][dy];
        w[1][dy] = w[2][dy];
      }
    }
  }
  r2 = r2f;
  f2 = f2f;
  for (int off = 16; off > 0; off >>= 1) {
    r2 += __shfl_down_sync(0xffffffffu, r2, off);
    f2 += __shfl_down_sync(0xffffffffu, f2, off);
  }
  const int wp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sr[wp] = r2;
    sf[wp] = f2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a2 = 0, b2 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a2 += sr[i];
      b2 += sf[i];
    }
    const int64_t bid = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    sums[2 * bid] = a2;
    sums[2 * bid + 1] = b2;
  }
}

// 3D residual through the tensor structure of eq. A3D:
//   A = (Kx - w^2 Mx) (x) My (x) Mz + Mx (x) (Ky (x) Mz + My (x) Kz).
// A CTA owns a TY x TZ tile of (y, z) columns and a run of RX3 x-planes.  For
// each x-plane (one before and one after the run included) it stages the
// tile plus a one-point halo in shared memory, applies Mz and Kz along z,
// then My, Ky along y, giving P_M = (My Mz) u and P_K = (Ky Mz + My Kz) u of
// that plane; the last three planes' (P_M, P_K) stay in registers and the x
// operators finish A u.  The 1D entries follow eqs. matrixK / matrixM, with
// the absorbing corner 1/h - i w at both ends of every axis.
constexpr int TZ3 = 32, TY3 = 8, RX3 = 32;

struct Coef1D {
  double md, mo;   // M diagonal (2h/6 at an end, 4h/6 inside), off-diagonal h/6
  double kdr, kdi; // K diagonal (1/h - i w at an end, 2/h inside)
  double ko;       // K off-diagonal -1/h
};

__device__ __forceinline__ Coef1D coef1d(const Axis1D& ax, int64_t i, double omega) {
  const bool end = (i == 0 || i == ax.n - 1);
  Coef1D c;
  c.md = (end ? 2.0 : 4.0) * ax.h / 6.0;
  c.mo = ax.h / 6.0;
  c.kdr = (end ? 1.0 : 2.0) / ax.h;
  c.kdi = end ? -omega : 0.0;
  c.ko = -1.0 / ax.h;
  return c;
}

// d * v with d = (dr, di); di is nonzero only at an absorbing end
__device__ __forceinline__ double2 cmul_rd(double dr, double di, double2 v) {
  double2 o;
  o.x = dr * v.x;
  o.y = dr * v.y;
  if (di != 0.0) {
    o.x = fma(-di, v.y, o.x);
    o.y = fma(di, v.x, o.y);
  }
  return o;
}

__global__ void __launch_bounds__(TZ3* TY3) k_residual3d(ResidArgs a, const double2* __restrict__ f,
                                                         const double2* __restrict__ u, float2* __restrict__ r,
                                                         double* __restrict__ sums, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double2 sU[TY3 + 2][TZ3 + 2];
  __shared__ double2 sTM[TY3 + 2][TZ3], sTK[TY3 + 2][TZ3];
  __shared__ double sr[TY3], sf[TY3];
  const int64_t nx = a.ax[0].n, ny = a.ax[1].n, nz = a.ax[2].n;
  const int tz = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TZ3 + tz;
  const int64_t z0 = (int64_t)blockIdx.x * TZ3, y0 = (int64_t)blockIdx.y * TY3;
  const int64_t xs = (int64_t)blockIdx.z * RX3, xe = min(xs + RX3, nx);  // outputs [xs, xe)
  const int64_t gz = z0 + tz, gy = y0 + ty;
  const bool own = gz < nz && gy < ny;
  const double w2 = a.omega * a.omega;
  const Coef1D cy = coef1d(a.ax[1], gy, a.omega);
  float r2f = 0.f, f2f = 0.f;
  const double2 zero = make_double2(0, 0);
  double2 PM[3] = {zero, zero, zero}, PK[3] = {zero, zero, zero};  // planes x-1, x, x+1
  for (int64_t ip = xs - 1; ip <= xe; ++ip) {
    // stage plane ip (zero outside the domain)
    const bool pin = ip >= 0 && ip < nx;
    for (int e = tid; e < (TY3 + 2) * (TZ3 + 2); e += TZ3 * TY3) {
      const int yy = e / (TZ3 + 2), zz = e - yy * (TZ3 + 2);
      const int64_t jy = y0 - 1 + yy, jz = z0 - 1 + zz;
      double2 v = zero;
      if (pin && jy >= 0 && jy < ny && jz >= 0 && jz < nz) v = __ldg(&u[(ip * ny + jy) * nz + jz]);
      sU[yy][zz] = v;
    }
    __syncthreads();
    // Mz and Kz along z for the TY+2 staged rows
    for (int e = tid; e < (TY3 + 2) * TZ3; e += TZ3 * TY3) {
      const int yy = e / TZ3, zc = e - yy * TZ3;
      const Coef1D cz = coef1d(a.ax[2], z0 + zc, a.omega);
      const double2 c0 = sU[yy][zc + 1];
      const double2 sn = make_double2(sU[yy][zc].x + sU[yy][zc + 2].x, sU[yy][zc].y + sU[yy][zc + 2].y);
      sTM[yy][zc] = make_double2(fma(cz.md, c0.x, cz.mo * sn.x), fma(cz.md, c0.y, cz.mo * sn.y));
      const double2 kc = cmul_rd(cz.kdr, cz.kdi, c0);
      sTK[yy][zc] = make_double2(fma(cz.ko, sn.x, kc.x), fma(cz.ko, sn.y, kc.y));
    }
    __syncthreads();
    // My and Ky along y: this plane's P_M, P_K at the thread's column
    {
      const double2 m0 = sTM[ty + 1][tz], mm = sTM[ty][tz], mp = sTM[ty + 2][tz];
      const double2 k0 = sTK[ty + 1][tz], km = sTK[ty][tz], kp = sTK[ty + 2][tz];
      const double2 sm = make_double2(mm.x + mp.x, mm.y + mp.y), sk = make_double2(km.x + kp.x, km.y + kp.y);
      PM[0] = PM[1];
      PK[0] = PK[1];
      PM[1] = PM[2];
      PK[1] = PK[2];
      PM[2] = make_double2(fma(cy.md, m0.x, cy.mo * sm.x), fma(cy.md, m0.y, cy.mo * sm.y));
      const double2 km0 = cmul_rd(cy.kdr, cy.kdi, m0);
      double2 pk;
      pk.x = fma(cy.ko, sm.x, km0.x);
      pk.y = fma(cy.ko, sm.y, km0.y);
      pk.x = fma(cy.md, k0.x, fma(cy.mo, sk.x, pk.x));
      pk.y = fma(cy.md, k0.y, fma(cy.mo, sk.y, pk.y));
      PK[2] = pk;
    }
    // along x: output plane ix = ip - 1 once planes ix-1, ix, ix+1 are in
    const int64_t ix = ip - 1;
    if (own && ix >= xs && ix < xe) {
      const Coef1D cx = coef1d(a.ax[0], ix, a.omega);
      const double2 spm = make_double2(PM[0].x + PM[2].x, PM[0].y + PM[2].y);
      const double2 spk = make_double2(PK[0].x + PK[2].x, PK[0].y + PK[2].y);
      // (Kx - w^2 Mx) P_M + Mx P_K
      double2 au = cmul_rd(cx.kdr - w2 * cx.md, cx.kdi, PM[1]);
      const double od = cx.ko - w2 * cx.mo;
      au.x = fma(od, spm.x, au.x);
      au.y = fma(od, spm.y, au.y);
      au.x = fma(cx.md, PK[1].x, fma(cx.mo, spk.x, au.x));
      au.y = fma(cx.md, PK[1].y, fma(cx.mo, spk.y, au.y));
      const int64_t gi = (ix * ny + gy) * nz + gz;
      const double2 fv = __ldg(&f[gi]);
      const float2 rf = make_float2((float)(fv.x - au.x), (float)(fv.y - au.y));
      r[gi] = rf;
      const float2 ff = make_float2((float)fv.x, (float)fv.y);
      r2f = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, r2f));
      f2f = fmaf(ff.x, ff.x, fmaf(ff.y, ff.y, f2f));
    }
  }
  double r2 = r2f, f2 = f2f;
  for (int off = 16; off > 0; off >>= 1) {
    r2 += __shfl_down_sync(0xffffffffu, r2, off);
    f2 += __shfl_down_sync(0xffffffffu, f2, off);
  }
  if (tz == 0) {
    sr[ty] = r2;
    sf[ty] = f2;
  }
  __syncthreads();
  if (tid == 0) {
    double a2 = 0, b2 = 0;
    for (int i = 0; i < TY3; ++i) {
      a2 += sr[i];
      b2 += sf[i];
    }
    const int64_t bid = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    sums[2 * bid] = a2;
    sums[2 * bid + 1] = b2;
  }
}

// ---------------------------------------------------------------------------
// Float-float residual r = f - A u (f and u as float-float complex vectors,
// float4 per point: re_hi, im_hi, re_lo, im_lo), about 48 significant bits
// per value, on the FP32 pipes; the products and sums of the stencil are
// exact up to the dropped lo x lo terms and the rounding of the lo parts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ffc_add(float4 a, float4 b) {
  float4 o;
  float e;
  two_sum(a.x, b.x, o.x, e);
  o.z = e + (a.z + b.z);
  two_sum(a.y, b.y, o.y, e);
  o.w = e + (a.w + b.w);
  return o;
}
// acc += c v, c a real float-float constant
__device__ __forceinline__ void ffc_mac_r(float4& acc, FF2 c, float4 v) {
  ff_mac(acc.x, acc.z, c.h, c.l, v.x, v.z);
  ff_mac(acc.y, acc.w, c.h, c.l, v.y, v.w);
}
// acc += (cr + i ci) v
__device__ __forceinline__ void ffc_mac_c(float4& acc, FF2 cr, FF2 ci, float4 v) {
  ff_mac(acc.x, acc.z, cr.h, cr.l, v.x, v.z);
  ff_mac(acc.x, acc.z, -ci.h, -ci.l, v.y, v.w);
  ff_mac(acc.y, acc.w, cr.h, cr.l, v.y, v.w);
  ff_mac(acc.y, acc.w, ci.h, ci.l, v.x, v.z);
}
// r = f - a, rounded to complex64; the norms' per-thread FP32 sums
__device__ __forceinline__ float2 ff_resid(float4 fv, float4 au, float& r2f, float& f2f) {
  float dr, er, di, ei;
  two_sum(fv.x, -au.x, dr, er);
  two_sum(fv.y, -au.y, di, ei);
  const float2 rf = make_float2(dr + (er + (fv.z - au.z)), di + (ei + (fv.w - au.w)));
  r2f = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, r2f));
  f2f = fmaf(fv.x, fv.x, fmaf(fv.y, fv.y, f2f));
  return rf;
}

// Block sums of the two norms: warp stage in FP32 (the norms only decide
// convergence; FP64 instructions are the scarce resource), block stage in FP64.
template <int NW>
__device__ __forceinline__ void block_norm_sums(float r2f, float f2f, double* __restrict__ sums, int64_t bid) {
  __shared__ double sr[NW], sf[NW];
  for (int off = 16; off > 0; off >>= 1) {
    r2f += __shfl_down_sync(0xffffffffu, r2f, off);
    f2f += __shfl_down_sync(0xffffffffu, f2f, off);
  }
  const double r2 = r2f, f2 = f2f;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) {
    sr[tid >> 5] = r2;
    sf[tid >> 5] = f2;
  }
  __syncthreads();
  if (tid == 0) {
    double a2 = 0, b2 = 0;
    for (int i = 0; i < NW; ++i) {
      a2 += sr[i];
      b2 += sf[i];
    }
    sums[2 * bid] = a2;
    sums[2 * bid + 1] = b2;
  }
}

// 2D, interior points (the perimeter is k_perimeter2d_ff): thread per y
// column, RX2 rows rolling along x, rows advanced by pointer increments.  The
// nine coefficients of eq. A2D take four values inside (centre, x pair,
// y pair, corners), so the neighbours are first summed in float-float, with
// the y-pair sum of each row reused for the corners of the next rows: three
// float-float sums and four products per component.
__global__ void __launch_bounds__(256) k_residual2d_ff(ResidFFArgs a, const float4* __restrict__ f,
                                                       const float4* __restrict__ u, float2* __restrict__ r,
                                                       double* __restrict__ sums, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t nx = a.n[0], ny = a.n[1];
  const int64_t iy = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t x0 = 1 + (int64_t)blockIdx.y * RX2;
  const int64_t x1 = min(x0 + RX2, nx - 1);
  float r2f = 0.f, f2f = 0.f;
  if (iy < ny - 1) {
    // interior coefficients [dx+1][dy+1]: centre (1,1), x pair (0,1), y pair (1,0), corners (0,0)
    const FF2 cc = a.cin[4], cxp = a.cin[1], cyp = a.cin[3], ccn = a.cin[0];
    const float4* un = u + (x0 + 1) * ny + iy;  // row ix + 1 (exists: ix + 1 <= nx - 1)
    const float4* fp = f + x0 * ny + iy;
    float2* rp = r + x0 * ny + iy;
    const float4* qm = un - 2 * ny;
    const float4* q0 = un - ny;
    float4 cm = __ldg(qm), pm = ffc_add(__ldg(qm - 1), __ldg(qm + 1));
    float4 c0 = __ldg(q0), p0 = ffc_add(__ldg(q0 - 1), __ldg(q0 + 1));
    // software pipeline: row ix + 2 and f of row ix + 1 load while row ix computes
    float4 nl = __ldg(un - 1), nc = __ldg(un), nr = __ldg(un + 1), nf = __ldg(fp);
    for (int64_t ix = x0; ix < x1; ++ix, rp += ny) {
      const float4 cp = nc, pp = ffc_add(nl, nr);
      const float4 fv = nf;
      if (ix + 1 < x1) {
        un += ny;
        fp += ny;
        nl = __ldg(un - 1);
        nc = __ldg(un);
        nr = __ldg(un + 1);
        nf = __ldg(fp);
      }
      float4 au = make_float4(0, 0, 0, 0);
      ffc_mac_r(au, cc, c0);
      ffc_mac_r(au, cxp, ffc_add(cm, cp));
      ffc_mac_r(au, cyp, p0);
      ffc_mac_r(au, ccn, ffc_add(pm, pp));
      *rp = ff_resid(fv, au, r2f, f2f);
      cm = c0;
      c0 = cp;
      pm = p0;
      p0 = pp;
    }
  }
  block_norm_sums<8>(r2f, f2f, sums, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
}

// 2D perimeter (rows 0 and nx-1, columns 0 and ny-1): one thread per point,
// the complex corner entries from the float-float table of its end class.
// Its block sums follow the interior kernel's, from sums + 2 * sum0.
__global__ void __launch_bounds__(256) k_perimeter2d_ff(ResidFFArgs a, const float4* __restrict__ f,
                                                        const float4* __restrict__ u, float2* __restrict__ r,
                                                        double* __restrict__ sums, int64_t sum0,
                                                        const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t nx = a.n[0], ny = a.n[1];
  const int64_t P = 2 * ny + 2 * (nx - 2);
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float r2f = 0.f, f2f = 0.f;
  if (p < P) {
    int64_t ix, iy;
    if (p < ny) {
      ix = 0;
      iy = p;
    } else if (p < 2 * ny) {
      ix = nx - 1;
      iy = p - ny;
    } else if (p < 2 * ny + nx - 2) {
      ix = 1 + (p - 2 * ny);
      iy = 0;
    } else {
      ix = 1 + (p - 2 * ny - (nx - 2));
      iy = ny - 1;
    }
    const int cx = ix == 0 ? 0 : (ix == nx - 1 ? 2 : 1);
    const int cy = iy == 0 ? 0 : (iy == ny - 1 ? 2 : 1);
    float4 au = make_float4(0, 0, 0, 0);
    for (int dx = -1; dx <= 1; ++dx) {
      if (ix + dx < 0 || ix + dx >= nx) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        if (iy + dy < 0 || iy + dy >= ny) continue;
        const int k = (dx + 1) * 3 + (dy + 1);
        ffc_mac_c(au, a.per[cx][cy][k][0], a.per[cx][cy][k][1], __ldg(&u[(ix + dx) * ny + iy + dy]));
      }
    }
    r[ix * ny + iy] = ff_resid(__ldg(&f[ix * ny + iy]), au, r2f, f2f);
  }
  block_norm_sums<8>(r2f, f2f, sums, sum0 + blockIdx.x);
}

// 3D: the separable traversal of k_residual3d in float-float.
__global__ void __launch_bounds__(TZ3* TY3) k_residual3d_ff(ResidFFArgs a, const float4* __restrict__ f,
                                                            const float4* __restrict__ u, float2* __restrict__ r,
                                                            double* __restrict__ sums, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ float4 sU[TY3 + 2][TZ3 + 2];
  __shared__ float4 sTM[TY3 + 2][TZ3], sTK[TY3 + 2][TZ3];
  const int64_t nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int tz = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TZ3 + tz;
  const int64_t z0 = (int64_t)blockIdx.x * TZ3, y0 = (int64_t)blockIdx.y * TY3;
  const int64_t xs = (int64_t)blockIdx.z * RX3, xe = min(xs + RX3, nx);
  const int64_t gz = z0 + tz, gy = y0 + ty;
  const bool own = gz < nz && gy < ny;
  const float4 z4 = make_float4(0, 0, 0, 0);
  const AxisFF& AY = a.ax[1];
  const AxisFF& AZ = a.ax[2];
  const AxisFF& AX = a.ax[0];
  const bool yend = gy == 0 || gy == ny - 1;
  float r2f = 0.f, f2f = 0.f;
  float4 PM[3] = {z4, z4, z4}, PK[3] = {z4, z4, z4};
  // the staged tile of plane ip is loaded into registers one plane ahead
  // (each thread owns at most kStage of its points), so the loads of the next
  // plane are in flight while the current one is computed
  constexpr int kStage = ((TY3 + 2) * (TZ3 + 2) + TZ3 * TY3 - 1) / (TZ3 * TY3);
  float4 nxt[kStage];
  auto fetch = [&](int64_t ip) {
    const bool pin = ip >= 0 && ip < nx;
#pragma unroll
    for (int q = 0; q < kStage; ++q) {
      const int e = tid + q * TZ3 * TY3;
      float4 v = z4;
      if (e < (TY3 + 2) * (TZ3 + 2)) {
        const int yy = e / (TZ3 + 2), zz = e - yy * (TZ3 + 2);
        const int64_t jy = y0 - 1 + yy, jz = z0 - 1 + zz;
        if (pin && jy >= 0 && jy < ny && jz >= 0 && jz < nz) v = __ldg(&u[(ip * ny + jy) * nz + jz]);
      }
      nxt[q] = v;
    }
  };
  fetch(xs - 1);
  for (int64_t ip = xs - 1; ip <= xe; ++ip) {
#pragma unroll
    for (int q = 0; q < kStage; ++q) {
      const int e = tid + q * TZ3 * TY3;
      if (e < (TY3 + 2) * (TZ3 + 2)) sU[e / (TZ3 + 2)][e % (TZ3 + 2)] = nxt[q];
    }
    __syncthreads();
    if (ip < xe) fetch(ip + 1);
    for (int e = tid; e < (TY3 + 2) * TZ3; e += TZ3 * TY3) {
      const int yy = e / TZ3, zc = e - yy * TZ3;
      const int64_t jz = z0 + zc;
      const bool zend = jz == 0 || jz == nz - 1;
      const float4 c0 = sU[yy][zc + 1];
      const float4 sn = ffc_add(sU[yy][zc], sU[yy][zc + 2]);
      float4 tm = z4, tk = z4;
      ffc_mac_r(tm, zend ? AZ.mde : AZ.mdi, c0);
      ffc_mac_r(tm, AZ.mo, sn);
      if (zend) ffc_mac_c(tk, AZ.kder, AZ.kdei, c0);
      else ffc_mac_r(tk, AZ.kdi, c0);
      ffc_mac_r(tk, AZ.ko, sn);
      sTM[yy][zc] = tm;
      sTK[yy][zc] = tk;
    }
    __syncthreads();
    {
      const float4 m0 = sTM[ty + 1][tz], k0 = sTK[ty + 1][tz];
      const float4 sm = ffc_add(sTM[ty][tz], sTM[ty + 2][tz]);
      const float4 sk = ffc_add(sTK[ty][tz], sTK[ty + 2][tz]);
      PM[0] = PM[1];
      PK[0] = PK[1];
      PM[1] = PM[2];
      PK[1] = PK[2];
      float4 pm = z4, pk = z4;
      ffc_mac_r(pm, yend ? AY.mde : AY.mdi, m0);
      ffc_mac_r(pm, AY.mo, sm);
      if (yend) ffc_mac_c(pk, AY.kder, AY.kdei, m0);
      else ffc_mac_r(pk, AY.kdi, m0);
      ffc_mac_r(pk, AY.ko, sm);
      ffc_mac_r(pk, yend ? AY.mde : AY.mdi, k0);
      ffc_mac_r(pk, AY.mo, sk);
      PM[2] = pm;
      PK[2] = pk;
    }
    const int64_t ix = ip - 1;
    if (own && ix >= xs && ix < xe) {
      const bool xend = ix == 0 || ix == nx - 1;
      const float4 spm = ffc_add(PM[0], PM[2]), spk = ffc_add(PK[0], PK[2]);
      float4 au = z4;
      // (Kx - w^2 Mx) P_M + Mx P_K
      if (xend) ffc_mac_c(au, AX.cde, AX.kdei, PM[1]);
      else ffc_mac_r(au, AX.cdi, PM[1]);
      ffc_mac_r(au, AX.co, spm);
      ffc_mac_r(au, xend ? AX.mde : AX.mdi, PK[1]);
      ffc_mac_r(au, AX.mo, spk);
      const int64_t gi = (ix * ny + gy) * nz + gz;
      r[gi] = ff_resid(__ldg(&f[gi]), au, r2f, f2f);
    }
  }
  block_norm_sums<TZ3 * TY3 / 32>(r2f, f2f, sums,
                                 ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
}

// f (complex128) -> float-float; u (float-float) -> complex128.  Both work on
// the bit fields with integer instructions (FP64 instructions are the scarce
// resource here).  hi is x rounded to nearest (ties to even) float, the same
// value as a plain conversion; lo = x - hi is the remaining signed fraction
// (|lo| <= 2^-24 |hi|, 29 bits) rounded to float by one integer-to-float
// conversion, so |x - (hi + lo)| <= 2^-48 |x|.  Values whose hi or lo would
// leave the normal float range, and infinities and NaNs, take the plain
// conversions.
__device__ __forceinline__ void split_d(double x, float& hi, float& lo) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
  if (e - 948 <= 0 || e - 896 >= 254) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
    return;
  }
  const uint64_t m = b & 0xfffffffffffffull;
  const uint32_t top = (uint32_t)(m >> 29), rem = (uint32_t)(m & 0x1fffffffull);
  const bool up = rem > 0x10000000u || (rem == 0x10000000u && (top & 1u));
  // the carry of top + 1 runs into the exponent field when the fraction is all ones
  hi = __uint_as_float((sgn | ((uint32_t)(e - 896) << 23) | top) + (up ? 1u : 0u));
  // x - hi = (rem - up 2^29) 2^(e - 1075), with the sign of x
  const int32_t r = (int32_t)rem - (up ? 0x20000000 : 0);
  const float scale = __uint_as_float((uint32_t)(e - 948) << 23);
  lo = __uint_as_float(__float_as_uint(__int2float_rn(r) * scale) ^ sgn);
}
// float -> double by the bit fields, exact for normal floats and zeros: the
// exponent is rebiased (+896) and the fraction moves 29 bits up.
__device__ __forceinline__ double widen_f(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t mag = u & 0x7fffffffu;
  const uint32_t hi = (u & 0x80000000u) | (mag ? (mag >> 3) + (896u << 20) : 0u);
  return __hiloint2double((int)hi, (int)(u << 29));
}
// subnormal, infinite or NaN (the values widen_f does not cover)
__device__ __forceinline__ bool widen_special(float v) {
  const uint32_t mag = __float_as_uint(v) & 0x7fffffffu;
  return mag != 0 && mag - 0x00800000u >= 0x7f000000u;
}
// the plain conversions, kept out of line so that the common path holds no
// FP64 conversion (a select would evaluate both sides)
__device__ __noinline__ double2 join_plain(float4 v) {
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}
__device__ __forceinline__ double2 join_one(float4 v) {
  if (widen_special(v.x) | widen_special(v.y) | widen_special(v.z) | widen_special(v.w)) return join_plain(v);
  return make_double2(widen_f(v.x) + widen_f(v.z), widen_f(v.y) + widen_f(v.w));
}
// Element-wise kernels: each thread issues kEw independent loads before it
// converts and stores them (enough bytes in flight to cover HBM latency).
constexpr int kEw = 4;
// hi (optional): the hi parts again as a complex64 vector, the first
// transform's input
__global__ void __launch_bounds__(256) k_split_ff(const double2* __restrict__ f, float4* __restrict__ o,
                                                  float2* __restrict__ hi, int64_t N) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kEw - 1) * stride < N; i += kEw * stride) {
    double2 v[kEw];
#pragma unroll
    for (int j = 0; j < kEw; ++j) v[j] = __ldcs(&f[i + j * stride]);
#pragma unroll
    for (int j = 0; j < kEw; ++j) {
      float4 q;
      split_d(v[j].x, q.x, q.z);
      split_d(v[j].y, q.y, q.w);
      o[i + j * stride] = q;
      if (hi) hi[i + j * stride] = make_float2(q.x, q.y);
    }
  }
  for (; i < N; i += stride) {
    const double2 v = f[i];
    float4 q;
    split_d(v.x, q.x, q.z);
    split_d(v.y, q.y, q.w);
    o[i] = q;
    if (hi) hi[i] = make_float2(q.x, q.y);
  }
}
__global__ void __launch_bounds__(256) k_join_ff(const float4* __restrict__ q, double2* __restrict__ o, int64_t N) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kEw - 1) * stride < N; i += kEw * stride) {
    float4 v[kEw];
#pragma unroll
    for (int j = 0; j < kEw; ++j) v[j] = __ldcs(&q[i + j * stride]);
#pragma unroll
    for (int j = 0; j < kEw; ++j)
      o[i + j * stride] = join_one(v[j]);
  }
  for (; i < N; i += stride) {
    const float4 v = q[i];
    o[i] = join_one(v);
  }
}

__global__ void __launch_bounds__(1024) k_residual_finalize(const double* __restrict__ sums, int64_t nblocks, RefineState* st,
                                    cudaGraphConditionalHandle cond) {
  if (st->done) {
    if (cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
    return;
  }
  // fixed order: kFinStreams interleaved partial sums per thread (independent
  // loads in flight), then the warps, then the block
  constexpr int kFinStreams = 4;
  __shared__ double sr[32], sf[32];
  const double2* s2 = reinterpret_cast<const double2*>(sums);
  double2 acc[kFinStreams];
#pragma unroll
  for (int j = 0; j < kFinStreams; ++j) acc[j] = make_double2(0.0, 0.0);
  const int64_t step = (int64_t)blockDim.x * kFinStreams;
  for (int64_t i0 = threadIdx.x; i0 < nblocks; i0 += step) {
    double2 v[kFinStreams];
#pragma unroll
    for (int j = 0; j < kFinStreams; ++j) {
      const int64_t i = i0 + (int64_t)j * blockDim.x;
      v[j] = i < nblocks ? s2[i] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int j = 0; j < kFinStreams; ++j) {
      acc[j].x += v[j].x;
      acc[j].y += v[j].y;
    }
  }
  double a2 = (acc[0].x + acc[1].x) + (acc[2].x + acc[3].x);
  double b2 = (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y);
  for (int off = 16; off > 0; off >>= 1) {
    a2 += __shfl_down_sync(0xffffffffu, a2, off);
    b2 += __shfl_down_sync(0xffffffffu, b2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = a2;
    sf[threadIdx.x >> 5] = b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (int)(blockDim.x >> 5);
    for (int w = 1; w < nw; ++w) {
      sr[0] += sr[w];
      sf[0] += sf[w];
    }
    const double rel = sf[0] > 0 ? sqrt(sr[0] / sf[0]) : sqrt(sr[0]);
    const int it = st->iters;
    if (it < 16) st->resid[it] = rel;
    st->iters = it + 1;
    st->fnorm2 = sf[0];
    if (rel <= st->tol) {
      st->converged = 1;
      st->done = 1;
    } else if (it + 1 >= st->max_iter + 1) {
      st->done = 1;
    }
    if (cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
  }
}

}  // namespace

cudaError_t launch_residual(int dim, const int64_t* n, const double* h, double omega, const double2* f,
                            const double2* u, float2* r, double* sums, int64_t* nblocks, const int* skip,
                            cudaStream_t st) {
  ResidArgs a{};
  a.dim = dim;
  a.omega = omega;
  int64_t N = 1;
  for (int k = 0; k < dim; ++k) {
    a.ax[k].n = n[k];
    a.ax[k].h = h[k];
    N *= n[k];
  }
  // interior coefficients (all entries real away from the corners)
  double m[3][3], kk[3][3];
  for (int k = 0; k < dim; ++k) {
    m[k][0] = m[k][2] = h[k] / 6.0;
    m[k][1] = 4.0 * h[k] / 6.0;
    kk[k][0] = kk[k][2] = -1.0 / h[k];
    kk[k][1] = 2.0 / h[k];
  }
  if (dim == 2) {
    for (int d0 = 0; d0 < 3; ++d0)
      for (int d1 = 0; d1 < 3; ++d1)
        a.cin[d0 * 3 + d1] = kk[0][d0] * m[1][d1] + m[0][d0] * kk[1][d1] - omega * omega * m[0][d0] * m[1][d1];
  } else {
    for (int d0 = 0; d0 < 3; ++d0)
      for (int d1 = 0; d1 < 3; ++d1)
        for (int d2 = 0; d2 < 3; ++d2)
          a.cin[d0 * 9 + d1 * 3 + d2] = kk[0][d0] * m[1][d1] * m[2][d2] + m[0][d0] * kk[1][d1] * m[2][d2] +
                                        m[0][d0] * m[1][d1] * kk[2][d2] -
                                        omega * omega * m[0][d0] * m[1][d1] * m[2][d2];
  }
  const int bs = 256;
  if (dim == 2) {
    const dim3 grid((unsigned)((n[1] + bs - 1) / bs), (unsigned)((n[0] + RX2 - 1) / RX2));
    *nblocks = (int64_t)grid.x * grid.y;
    k_residual2d<<<grid, bs, 0, st>>>(a, f, u, r, sums, skip);
    return cudaGetLastError();
  }
  if (dim == 3) {
    const dim3 grid((unsigned)((n[2] + TZ3 - 1) / TZ3), (unsigned)((n[1] + TY3 - 1) / TY3),
                    (unsigned)((n[0] + RX3 - 1) / RX3));
    *nblocks = (int64_t)grid.x * grid.y * grid.z;
    k_residual3d<<<grid, dim3(TZ3, TY3), 0, st>>>(a, f, u, r, sums, skip);
    return cudaGetLastError();
  }
  const int64_t grid = (N + bs - 1) / bs;
  *nblocks = grid;
  k_residual<<<(unsigned)grid, bs, 0, st>>>(a, f, u, r, sums, N, skip);
  return cudaGetLastError();
}

static FF2 split_host(double x) {
  FF2 c;
  c.h = (float)x;
  c.l = (float)(x - (double)c.h);
  return c;
}

cudaError_t launch_residual_ff(int dim, const int64_t* n, const double* h, double omega, const float4* f,
                               const float4* u, float2* r, double* sums, int64_t* nblocks, const int* skip,
                               cudaStream_t st) {
  ResidFFArgs a{};
  a.omega = omega;
  const double w2 = omega * omega;
  for (int k = 0; k < dim; ++k) {
    a.n[k] = n[k];
    a.h[k] = h[k];
    const double hk = h[k];
    AxisFF& x = a.ax[k];
    x.mdi = split_host(4.0 * hk / 6.0);
    x.mde = split_host(2.0 * hk / 6.0);
    x.mo = split_host(hk / 6.0);
    x.kdi = split_host(2.0 / hk);
    x.kder = split_host(1.0 / hk);
    x.ko = split_host(-1.0 / hk);
    x.kdei = split_host(-omega);
    x.cdi = split_host(2.0 / hk - w2 * (4.0 * hk / 6.0));
    x.cde = split_host(1.0 / hk - w2 * (2.0 * hk / 6.0));
    x.co = split_host(-1.0 / hk - w2 * (hk / 6.0));
  }
  if (dim == 2) {
    double m[2][3], kk[2][3];
    for (int k = 0; k < 2; ++k) {
      m[k][0] = m[k][2] = h[k] / 6.0;
      m[k][1] = 4.0 * h[k] / 6.0;
      kk[k][0] = kk[k][2] = -1.0 / h[k];
      kk[k][1] = 2.0 / h[k];
    }
    for (int d0 = 0; d0 < 3; ++d0)
      for (int d1 = 0; d1 < 3; ++d1)
        a.cin[d0 * 3 + d1] = split_host(kk[0][d0] * m[1][d1] + m[0][d0] * kk[1][d1] - w2 * m[0][d0] * m[1][d1]);
    const int bs = 256;
    // perimeter table: entries of eqs. matrixK / matrixM at the first, an inner
    // and the last index of each axis
    auto ent = [&](int k, int64_t i, int d, double& m, double& kr, double& ki) {
      const bool end = (i == 0 || i == n[k] - 1);
      if (d == 0) {
        m = (end ? 2.0 : 4.0) * h[k] / 6.0;
        kr = (end ? 1.0 : 2.0) / h[k];
        ki = end ? -omega : 0.0;
      } else {
        m = h[k] / 6.0;
        kr = -1.0 / h[k];
        ki = 0.0;
      }
    };
    for (int cx = 0; cx < 3; ++cx)
      for (int cy = 0; cy < 3; ++cy) {
        const int64_t ix = cx == 0 ? 0 : (cx == 1 ? 1 : n[0] - 1), iy = cy == 0 ? 0 : (cy == 1 ? 1 : n[1] - 1);
        for (int dx = -1; dx <= 1; ++dx)
          for (int dy = -1; dy <= 1; ++dy) {
            double m0, k0r, k0i, m1, k1r, k1i;
            ent(0, ix, dx, m0, k0r, k0i);
            ent(1, iy, dy, m1, k1r, k1i);
            const int k = (dx + 1) * 3 + (dy + 1);
            a.per[cx][cy][k][0] = split_host(k0r * m1 + m0 * k1r - w2 * m0 * m1);
            a.per[cx][cy][k][1] = split_host(k0i * m1 + m0 * k1i);
          }
      }
    const dim3 grid((unsigned)((n[1] - 2 + bs - 1) / bs), (unsigned)((n[0] - 2 + RX2 - 1) / RX2));
    const int64_t nmain = (int64_t)grid.x * grid.y;
    const int64_t P = 2 * n[1] + 2 * (n[0] - 2);
    const int64_t gper = (P + bs - 1) / bs;
    *nblocks = nmain + gper;
    k_residual2d_ff<<<grid, bs, 0, st>>>(a, f, u, r, sums, skip);
    k_perimeter2d_ff<<<(unsigned)gper, bs, 0, st>>>(a, f, u, r, sums, nmain, skip);
    return cudaGetLastError();
  }
  const dim3 grid((unsigned)((n[2] + TZ3 - 1) / TZ3), (unsigned)((n[1] + TY3 - 1) / TY3),
                  (unsigned)((n[0] + RX3 - 1) / RX3));
  *nblocks = (int64_t)grid.x * grid.y * grid.z;
  k_residual3d_ff<<<grid, dim3(TZ3, TY3), 0, st>>>(a, f, u, r, sums, skip);
  return cudaGetLastError();
}

// One resident wave of 256-thread blocks (8 per SM), fewer for small N.
static int64_t ew_grid(int64_t N) {
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, (int64_t)nsm * 8));
}

cudaError_t launch_split_ff(const double2* f, float4* out, float2* hi, int64_t N, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  const int64_t grid = ew_grid(N);
  k_split_ff<<<(unsigned)grid, 256, 0, st>>>(f, out, hi, N);
  return cudaGetLastError();
}

cudaError_t launch_join_ff(const float4* u, double2* out, int64_t N, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  const int64_t grid = ew_grid(N);
  k_join_ff<<<(unsigned)grid, 256, 0, st>>>(u, out, N);
  return cudaGetLastError();
}

// Deterministic pseudo-random complex load for plan-time trials: the
// splitmix64 finaliser of (seed, index), mapped to [-1, 1) per component.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void k_trial_rhs(double2* __restrict__ f, int64_t N, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = mix64(seed + 0x9e3779b97f4a7c15ull * (uint64_t)(2 * i + 1));
    const uint64_t b = mix64(seed + 0x9e3779b97f4a7c15ull * (uint64_t)(2 * i + 2));
    f[i] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, (double)(b >> 11) * 0x1.0p-52 - 1.0);
  }
}

cudaError_t launch_trial_rhs(double2* f, int64_t N, uint64_t seed, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>((N + 255) / 256, 152 * 16);
  k_trial_rhs<<<(unsigned)grid, 256, 0, st>>>(f, N, seed);
  return cudaGetLastError();
}

__global__ void k_refine_init(RefineState* st, double tol, int max_iter) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    RefineState s{};
    s.tol = tol;
    s.max_iter = max_iter;
    *st = s;
  }
}

cudaError_t launch_refine_init(RefineState* st, double tol, int max_iter, cudaStream_t stream) {
  k_refine_init<<<1, 32, 0, stream>>>(st, tol, max_iter);
  return cudaGetLastError();
}

int64_t residual_blocks(int dim, const int64_t* n) {
  if (dim == 2) {
    // the larger of the FP64 grid and the float-float interior + perimeter grids
    const int64_t fp64 = ((n[1] + 255) / 256) * ((n[0] + RX2 - 1) / RX2);
    const int64_t ff = ((n[1] - 2 + 255) / 256) * ((n[0] - 2 + RX2 - 1) / RX2) + (2 * n[1] + 2 * (n[0] - 2) + 255) / 256;
    return std::max(fp64, ff);
  }
  return ((n[2] + TZ3 - 1) / TZ3) * ((n[1] + TY3 - 1) / TY3) * ((n[0] + RX3 - 1) / RX3);
}

cudaError_t launch_residual_finalize(const double* sums, int64_t nblocks, RefineState* state,
                                     unsigned long long cond, cudaStream_t st) {
  k_residual_finalize<<<1, 1024, 0, st>>>(sums, nblocks, state, (cudaGraphConditionalHandle)cond);
  return cudaGetLastError();
}

}  // namespace helm
