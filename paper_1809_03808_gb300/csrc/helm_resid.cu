// FP64 residual r = f - A u of the Kronecker operators of eq. A2D (9-point)
// and eq. A3D (27-point), used by iterative refinement of the complex64
// solves.  A u is the tensor-product stencil: the coefficient of neighbour
// offset (d_1, ..., d_D) is  sum_j prod_k X^{(j)}_k(i_k, i_k + d_k)
// - w^2 prod_k M_k(i_k, i_k + d_k), with X^{(j)}_k = K_k if k == j else M_k
// (1D matrices of eqs. matrixK / matrixM).  Interior points use precomputed
// real coefficients; points on a face use the complex corner entries.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <complex>

#include "helm_async.cuh"
#include "helm_kernels.cuh"
#include "helm_solve.h"

namespace helm {

namespace {

// Tile shapes of the float-float residuals: 2D rows per thread; 3D z, y
// tile and x planes per CTA.
constexpr int RX2 = 16;
constexpr int TZ3 = 32, TY3 = 8, RX3 = 32;

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

// ---------------------------------------------------------------------------
// FP64 residual with the fewest FP64 instructions.  On this GPU an FP64
// instruction costs the SM about as much issue time as 64 FP32 ones, so the
// stencil is rearranged to minimise them; everything else (staging, norms,
// conversions) runs on the FP32 and integer pipes.
//
// Per axis k the 1D matrices of eqs. matrixK / matrixM are
//   M_k = m0 I + m1 S_k,  K_k = k0 I + k1 S_k,
// with S_k the sum of the two neighbours along axis k (one at an end node),
// m1 = h/6, k1 = -1/h, and m0 = 4h/6, k0 = 2/h inside, m0 = 2h/6,
// k0 = 1/h - i w at the absorbing ends.  So the operator of eq. A3D is
//   A u = sum_{a,b,c in {0,1}} C_abc Sx^a Sy^b Sz^c u,
//   C_abc = Kx_a My_b Mz_c + Mx_a Ky_b Mz_c + Mx_a My_b Kz_c - w^2 Mx_a My_b Mz_c,
// where X_0 / X_1 are the I / S coefficients of X; C_abc depends on whether
// the node is an end node of each axis (real inside, complex on a face).  The
// S_x part (a = 1) uses only the off-diagonal entries, so it does not depend
// on the x class.  With the plane monomials P_bc = Sy^b Sz^c u of each
// x-plane,
//   Q(x) = sum_bc C_0bc P_bc(x),  R(x) = sum_bc C_1bc P_bc(x),
//   r(x) = f(x) - Q(x) - R(x-1) - R(x+1).
// Per real component inside: 3 neighbour sums, 4 + 4 multiply-adds (Q from
// f), 2 subtractions: 13 FP64 instructions (26 per complex unknown; 2D: 7).
// ---------------------------------------------------------------------------

// The plain conversion, out of line so that the common path of round_d2f
// holds no FP64 instruction (a select would evaluate both sides).
__device__ __noinline__ float round_d2f_plain(double x) { return (float)x; }

// x rounded to the nearest float (ties to even) on the integer pipe; values
// outside the normal float range take the plain conversion.
__device__ __forceinline__ float round_d2f(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e - 896 <= 0 || e - 896 >= 254) return round_d2f_plain(x);
  const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t m = b & 0xfffffffffffffull;
  const uint32_t top = (uint32_t)(m >> 29), rem = (uint32_t)(m & 0x1fffffffull);
  const bool up = rem > 0x10000000u || (rem == 0x10000000u && (top & 1u));
  return __uint_as_float((sgn | ((uint32_t)(e - 896) << 23) | top) + (up ? 1u : 0u));
}

struct ResidQArgs {
  int64_t n[3];
  // 3D: c0[4 cx + 2 cy + cz][2 b + c], c1[2 cy + cz][2 b + c]; 2D: c0[2 cx + cy][b], c1[cy][b]
  double2 c0[8][4];
  double2 c1[4][4];
  // 3D corrections of the end classes against the same class inside y and z:
  // dc0[cls][bc] = c0[cls][bc] - c0[cls & 4][bc], dc1[cyz][bc] = c1[cyz][bc] - c1[0][bc]
  double2 dc0[8][4];
  double2 dc1[4][4];
};

// (acc.x, acc.y) += c v
__device__ __forceinline__ void cadd_mul(double2& acc, double2 c, double2 v) {
  acc.x = fma(c.x, v.x, fma(-c.y, v.y, acc.x));
  acc.y = fma(c.x, v.y, fma(c.y, v.x, acc.y));
}

// (acc.x, acc.y) -= c v for complex c (boundary classes)
__device__ __forceinline__ void csub_mul(double2& acc, double2 c, double2 v) {
  acc.x = fma(-c.x, v.x, fma(c.y, v.y, acc.x));
  acc.y = fma(-c.x, v.y, fma(-c.y, v.x, acc.y));
}

// Block sums of |r|^2 and |f|^2 (per-thread FP32 sums of the rounded
// values; the norms only decide convergence), fixed order.
template <int NT>
__device__ __forceinline__ void block_norms(float r2f, float f2f, double* sums, int64_t bid) {
  __shared__ float sr[NT / 32], sf[NT / 32];
  for (int off = 16; off > 0; off >>= 1) {
    r2f += __shfl_down_sync(0xffffffffu, r2f, off);
    f2f += __shfl_down_sync(0xffffffffu, f2f, off);
  }
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) {
    sr[tid >> 5] = r2f;
    sf[tid >> 5] = f2f;
  }
  __syncthreads();
  if (tid == 0) {
    double a2 = 0, b2 = 0;
    for (int i = 0; i < NT / 32; ++i) {
      a2 += (double)sr[i];
      b2 += (double)sf[i];
    }
    sums[2 * bid] = a2;
    sums[2 * bid + 1] = b2;
  }
}

constexpr int QZ = 32, QY = 16, QX = 64;  // 3D tile: z, y columns, x planes per CTA
constexpr int QE = ((QY + 2) * (QZ + 2) + QZ * QY - 1) / (QZ * QY);  // staged values per thread

__global__ void __launch_bounds__(QZ* QY) k_residual3d_q(ResidQArgs a, const double2* __restrict__ f,
                                                         const double2* __restrict__ u, float2* __restrict__ r,
                                                         double* __restrict__ sums, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double2 sU[QY + 2][QZ + 2];
  __shared__ double2 sSz[QY + 2][QZ];
  const int64_t nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int tz = threadIdx.x, ty = threadIdx.y, tid = ty * QZ + tz;
  const int64_t z0 = (int64_t)blockIdx.x * QZ, y0 = (int64_t)blockIdx.y * QY;
  const int64_t xs = (int64_t)blockIdx.z * QX, xe = min(xs + QX, nx);
  const int64_t gz = z0 + tz, gy = y0 + ty;
  const bool own = gz < nz && gy < ny;
  const int cy = (gy == 0 || gy == ny - 1) ? 1 : 0, cz = (gz == 0 || gz == nz - 1) ? 1 : 0;
  const int cyz = 2 * cy + cz;
  const double2 zero = make_double2(0.0, 0.0);
  float r2f = 0.f, f2f = 0.f;
  // staging prefetch of the next plane
  double2 pf[QE];
  auto fetch = [&](int64_t ip) {
#pragma unroll
    for (int k = 0; k < QE; ++k) {
      const int e = tid + k * QZ * QY;
      pf[k] = zero;
      if (e < (QY + 2) * (QZ + 2) && ip >= 0 && ip < nx) {
        const int yy = e / (QZ + 2), zz = e - yy * (QZ + 2);
        const int64_t jy = y0 - 1 + yy, jz = z0 - 1 + zz;
        if (jy >= 0 && jy < ny && jz >= 0 && jz < nz) pf[k] = __ldg(&u[(ip * ny + jy) * nz + jz]);
      }
    }
  };
  fetch(xs - 1);
  double2 Rm = zero, Rc = zero, Qc = zero;  // R(x-2), R(x-1), f - Q at x-1
  for (int64_t ip = xs - 1; ip <= xe; ++ip) {
    __syncthreads();  // the previous plane's reads of sU, sSz are done
#pragma unroll
    for (int k = 0; k < QE; ++k) {
      const int e = tid + k * QZ * QY;
      if (e < (QY + 2) * (QZ + 2)) (&sU[0][0])[e] = pf[k];
    }
    if (ip + 1 <= xe) fetch(ip + 1);
    const bool outp = own && ip >= xs && ip < xe;
    double2 fv = zero;
    if (outp) fv = __ldg(&f[(ip * ny + gy) * nz + gz]);
    __syncthreads();
    for (int e = tid; e < (QY + 2) * QZ; e += QZ * QY) {
      const int yy = e / QZ, zc = e - yy * QZ;
      const double2 lo = sU[yy][zc], hi = sU[yy][zc + 2];
      sSz[yy][zc] = make_double2(lo.x + hi.x, lo.y + hi.y);
    }
    __syncthreads();
    double2 Rn = zero, Qn = fv;
    if (own && ip >= 0 && ip < nx) {
      const double2 P00 = sU[ty + 1][tz + 1], P01 = sSz[ty + 1][tz];
      const double2 ym = sU[ty][tz + 1], yp = sU[ty + 2][tz + 1];
      const double2 sm = sSz[ty][tz], sp = sSz[ty + 2][tz];
      const double2 P10 = make_double2(ym.x + yp.x, ym.y + yp.y), P11 = make_double2(sm.x + sp.x, sm.y + sp.y);
      const int cx = (ip == 0 || ip == nx - 1) ? 1 : 0;
      // every lane takes the interior coefficients (real: C_1bc for R, C_0bc
      // for Q inside along x; complex C_0bc on the two x-end planes, a
      // plane-uniform branch) ...
      Rn.x = fma(a.c1[0][3].x, P11.x, fma(a.c1[0][2].x, P10.x, fma(a.c1[0][1].x, P01.x, a.c1[0][0].x * P00.x)));
      Rn.y = fma(a.c1[0][3].x, P11.y, fma(a.c1[0][2].x, P10.y, fma(a.c1[0][1].x, P01.y, a.c1[0][0].x * P00.y)));
      if (outp) {
        if (cx == 0) {
          Qn.x = fma(-a.c0[0][3].x, P11.x, fma(-a.c0[0][2].x, P10.x, fma(-a.c0[0][1].x, P01.x, fma(-a.c0[0][0].x, P00.x, Qn.x))));
          Qn.y = fma(-a.c0[0][3].x, P11.y, fma(-a.c0[0][2].x, P10.y, fma(-a.c0[0][1].x, P01.y, fma(-a.c0[0][0].x, P00.y, Qn.y))));
        } else {
          csub_mul(Qn, a.c0[4][0], P00);
          csub_mul(Qn, a.c0[4][1], P01);
          csub_mul(Qn, a.c0[4][2], P10);
          csub_mul(Qn, a.c0[4][3], P11);
        }
      }
      // ... and lanes on a y or z face add the coefficients that differ there:
      // a y end changes the b = 0 monomials, a z end the c = 0 ones
      if (cyz) {
        if (cy | cz) cadd_mul(Rn, a.dc1[cyz][0], P00);
        if (cy) cadd_mul(Rn, a.dc1[cyz][1], P01);
        if (cz) cadd_mul(Rn, a.dc1[cyz][2], P10);
        if (outp) {
          const int cls = 4 * cx + cyz;
          if (cy | cz) csub_mul(Qn, a.dc0[cls][0], P00);
          if (cy) csub_mul(Qn, a.dc0[cls][1], P01);
          if (cz) csub_mul(Qn, a.dc0[cls][2], P10);
        }
      }
    }
    // output plane ip - 1: r = (f - Q)(x) - R(x-1) - R(x+1)
    const int64_t ix = ip - 1;
    if (own && ix >= xs && ix < xe) {
      const float2 rf = make_float2(round_d2f(Qc.x - Rm.x - Rn.x), round_d2f(Qc.y - Rm.y - Rn.y));
      r[(ix * ny + gy) * nz + gz] = rf;
      r2f = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, r2f));
    }
    if (outp) {
      const float fx = round_d2f(fv.x), fy = round_d2f(fv.y);
      f2f = fmaf(fx, fx, fmaf(fy, fy, f2f));
    }
    Rm = Rc;
    Rc = Rn;
    Qc = Qn;
  }
  block_norms<QZ * QY>(r2f, f2f, sums, ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
}

// The same 3D residual with the u planes brought in by the tensor memory
// accelerator: one thread issues a tiled load of the plane's (QY+2) x (QZ+2)
// halo box, whose parts outside the grid arrive as zeros, so the staging
// needs no per-thread index or bounds arithmetic and no registers.  Three
// plane buffers: while plane i is used, planes i+1 and i+2 are in flight; the
// z sums are double-buffered, so one barrier per plane separates every reuse.
// The plane's f tile comes by the same kind of load on the same barrier.
// Every wait is bounded: a copy that does not arrive sets *err, the whole CTA
// stops, and thread 0 lets its copies still in flight land before it exits.
constexpr int QUB = (QY + 2) * (QZ + 2) * (int)sizeof(double2);  // bytes of one staged u plane
constexpr int QUS = (QUB + 127) / 128 * 128;                      // its stride (TMA destinations: 128 B)
constexpr int QFB = QY * QZ * (int)sizeof(double2);               // bytes of one f plane tile
constexpr int QNB = 3;                                            // plane buffers
constexpr int QSZB = 2 * (QY + 2) * QZ * (int)sizeof(double2);    // the two z-sum buffers
constexpr size_t kResidTmaSmem = (size_t)QNB * (QUS + QFB) + QSZB + QNB * sizeof(uint64_t);

__global__ void __launch_bounds__(QZ* QY, 2)
    k_residual3d_tma(const __grid_constant__ CUtensorMap umap, const __grid_constant__ CUtensorMap fmap, ResidQArgs a,
                     float2* __restrict__ r, double* __restrict__ sums, const int* __restrict__ skip, int* err) {
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char rsm[];
  unsigned char* sUb = rsm;                                               // [QNB][QUS] u halo planes
  unsigned char* sFb = sUb + QNB * QUS;                                   // [QNB][QFB] f plane tiles
  double2(*sSz)[QY + 2][QZ] = reinterpret_cast<double2(*)[QY + 2][QZ]>(sFb + QNB * QFB);  // [2]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sFb + QNB * QFB + QSZB);
  const int64_t nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int tz = threadIdx.x, ty = threadIdx.y, tid = ty * QZ + tz;
  const int64_t z0 = (int64_t)blockIdx.x * QZ, y0 = (int64_t)blockIdx.y * QY;
  const int64_t xs = (int64_t)blockIdx.z * QX, xe = min(xs + QX, nx);
  const int np = (int)(xe - xs + 2);  // planes xs-1 .. xe (at least 3)
  const int64_t gz = z0 + tz, gy = y0 + ty;
  const bool own = gz < nz && gy < ny;
  const int cy = (gy == 0 || gy == ny - 1) ? 1 : 0, cz = (gz == 0 || gz == nz - 1) ? 1 : 0;
  const int cyz = 2 * cy + cz;
  const double2 zero = make_double2(0.0, 0.0);
  float r2f = 0.f, f2f = 0.f;
  if (tid == 0) {
    for (int b = 0; b < QNB; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // plane xs - 1 + i of u (halo box) and of f (the tile) into buffer i % QNB
  // (thread 0 only; boxes outside the grid arrive as zeros)
  auto issue = [&](int i) {
    const int b = i % QNB;
    mbar_arrive_expect_tx(&bar[b], (uint32_t)(QUB + QFB));
    tma_load_3d(sUb + b * QUS, &umap, (int)(2 * (z0 - 1)), (int)(y0 - 1), (int)(xs - 1 + i), &bar[b]);
    tma_load_3d(sFb + b * QFB, &fmap, (int)(2 * z0), (int)y0, (int)(xs - 1 + i), &bar[b]);
  };
  int issued = 0;
  if (tid == 0) {
    issue(0);
    issue(1);
    issued = 2;
  }
  double2 Rm = zero, Rc = zero, Qc = zero;  // R(x-2), R(x-1), f - Q at x-1
  int i = 0;
  bool failed = false;
  for (; i < np; ++i) {
    const int64_t ip = xs - 1 + i;
    const double2* U = reinterpret_cast<const double2*>(sUb + (i % QNB) * QUS);  // [QY+2][QZ+2]
    const double2* F = reinterpret_cast<const double2*>(sFb + (i % QNB) * QFB);  // [QY][QZ]
    double2(*Sz)[QZ] = sSz[i & 1];
    const bool outp = own && ip >= xs && ip < xe;
    const bool got = mbar_wait_bounded(&bar[i % QNB], (uint32_t)((i / QNB) & 1), err);
    for (int e = tid; e < (QY + 2) * QZ; e += QZ * QY) {
      const int yy = e / QZ, zc = e - yy * QZ;
      const double2 lo = U[yy * (QZ + 2) + zc], hi = U[yy * (QZ + 2) + zc + 2];
      Sz[yy][zc] = make_double2(lo.x + hi.x, lo.y + hi.y);
    }
    if (__syncthreads_or(!got)) {  // block-uniform
      failed = true;
      break;
    }
    // every thread is past plane i - 1: its buffers take plane i + 2
    if (tid == 0 && i + 2 < np) {
      issue(i + 2);
      issued = i + 3;
    }
    const double2 fv = outp ? F[ty * QZ + tz] : zero;
    double2 Rn = zero, Qn = fv;
    if (own && ip >= 0 && ip < nx) {
      const double2 P00 = U[(ty + 1) * (QZ + 2) + tz + 1], P01 = Sz[ty + 1][tz];
      const double2 ym = U[ty * (QZ + 2) + tz + 1], yp = U[(ty + 2) * (QZ + 2) + tz + 1];
      const double2 sm = Sz[ty][tz], sp = Sz[ty + 2][tz];
      const double2 P10 = make_double2(ym.x + yp.x, ym.y + yp.y), P11 = make_double2(sm.x + sp.x, sm.y + sp.y);
      const int cx = (ip == 0 || ip == nx - 1) ? 1 : 0;
      Rn.x = fma(a.c1[0][3].x, P11.x, fma(a.c1[0][2].x, P10.x, fma(a.c1[0][1].x, P01.x, a.c1[0][0].x * P00.x)));
      Rn.y = fma(a.c1[0][3].x, P11.y, fma(a.c1[0][2].x, P10.y, fma(a.c1[0][1].x, P01.y, a.c1[0][0].x * P00.y)));
      if (outp) {
        if (cx == 0) {
          Qn.x = fma(-a.c0[0][3].x, P11.x, fma(-a.c0[0][2].x, P10.x, fma(-a.c0[0][1].x, P01.x, fma(-a.c0[0][0].x, P00.x, Qn.x))));
          Qn.y = fma(-a.c0[0][3].x, P11.y, fma(-a.c0[0][2].x, P10.y, fma(-a.c0[0][1].x, P01.y, fma(-a.c0[0][0].x, P00.y, Qn.y))));
        } else {
          csub_mul(Qn, a.c0[4][0], P00);
          csub_mul(Qn, a.c0[4][1], P01);
          csub_mul(Qn, a.c0[4][2], P10);
          csub_mul(Qn, a.c0[4][3], P11);
        }
      }
      if (cyz) {
        if (cy | cz) cadd_mul(Rn, a.dc1[cyz][0], P00);
        if (cy) cadd_mul(Rn, a.dc1[cyz][1], P01);
        if (cz) cadd_mul(Rn, a.dc1[cyz][2], P10);
        if (outp) {
          const int cls = 4 * cx + cyz;
          if (cy | cz) csub_mul(Qn, a.dc0[cls][0], P00);
          if (cy) csub_mul(Qn, a.dc0[cls][1], P01);
          if (cz) csub_mul(Qn, a.dc0[cls][2], P10);
        }
      }
    }
    const int64_t ix = ip - 1;
    if (own && ix >= xs && ix < xe) {
      const float2 rf = make_float2(round_d2f(Qc.x - Rm.x - Rn.x), round_d2f(Qc.y - Rm.y - Rn.y));
      r[(ix * ny + gy) * nz + gz] = rf;
      r2f = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, r2f));
    }
    if (outp) {
      const float fx = round_d2f(fv.x), fy = round_d2f(fv.y);
      f2f = fmaf(fx, fx, fmaf(fy, fy, f2f));
    }
    Rm = Rc;
    Rc = Rn;
    Qc = Qn;
  }
  if (failed && tid == 0)
    for (int j = i; j < issued; ++j) mbar_wait_bounded(&bar[j % QNB], (uint32_t)((j / QNB) & 1), nullptr);
  block_norms<QZ * QY>(r2f, f2f, sums, ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
}

// The driver's tensor-map encoder, looked up once through the runtime (no
// link-time dependence on the driver library); null if unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* q = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      q = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(q);
  }();
  return fn;
}

// Tensor map of a [nx][ny][nz] complex128 array viewed as [nx][ny][2 nz]
// FP64, with a box of bz complex values x by rows along y; false if it cannot
// be made (the caller then stages the planes with plain loads).
bool residual_map(CUtensorMap* m, const double2* v, const int64_t* n, int bz, int by) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || ((uintptr_t)v & 15) || 2 * n[2] > (int64_t)UINT32_MAX || n[1] > (int64_t)UINT32_MAX ||
      n[0] > (int64_t)INT32_MAX - 2)
    return false;
  const cuuint64_t gdim[3] = {(cuuint64_t)(2 * n[2]), (cuuint64_t)n[1], (cuuint64_t)n[0]};
  const cuuint64_t gstride[2] = {(cuuint64_t)(2 * n[2] * sizeof(double)), (cuuint64_t)(n[1] * 2 * n[2] * sizeof(double))};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * bz), (cuuint32_t)by, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double2*>(v), gdim, gstride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D: thread per y column, QR2 rows rolling along x; monomials P_0 = u,
// P_1 = Sy u of each row; r(x) = f(x) - Q(x) - R(x-1) - R(x+1).
constexpr int QR2 = 32;
__global__ void __launch_bounds__(256) k_residual2d_q(ResidQArgs a, const double2* __restrict__ f,
                                                      const double2* __restrict__ u, float2* __restrict__ r,
                                                      double* __restrict__ sums, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t nx = a.n[0], ny = a.n[1];
  const int64_t iy = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t xs = (int64_t)blockIdx.y * QR2, xe = min(xs + QR2, nx);
  const bool own = iy < ny;
  const int cy = (iy == 0 || iy == ny - 1) ? 1 : 0;
  const double2 zero = make_double2(0.0, 0.0);
  float r2f = 0.f, f2f = 0.f;
  double2 Rm = zero, Rc = zero, Qc = zero;
  if (own) {
    const bool ym = iy > 0, yp = iy < ny - 1;
    // row loads one row ahead
    double2 c0v = zero, cmv = zero, cpv = zero, fv = zero;
    auto load = [&](int64_t ix, double2& c, double2& m, double2& p) {
      c = m = p = zero;
      if (ix >= 0 && ix < nx) {
        const double2* row = u + ix * ny + iy;
        c = __ldg(row);
        if (ym) m = __ldg(row - 1);
        if (yp) p = __ldg(row + 1);
      }
    };
    load(xs - 1, c0v, cmv, cpv);
    for (int64_t ip = xs - 1; ip <= xe; ++ip) {
      const double2 P0 = c0v;
      const double2 P1 = make_double2(cmv.x + cpv.x, cmv.y + cpv.y);
      const bool outp = ip >= xs && ip < xe;
      if (outp) fv = __ldg(&f[ip * ny + iy]);
      if (ip + 1 <= xe) load(ip + 1, c0v, cmv, cpv);
      double2 Rn = zero, Qn = fv;
      if (ip >= 0 && ip < nx) {
        const int cx = (ip == 0 || ip == nx - 1) ? 1 : 0;
        if (cy == 0 && cx == 0) {
          Rn.x = fma(a.c1[0][1].x, P1.x, a.c1[0][0].x * P0.x);
          Rn.y = fma(a.c1[0][1].x, P1.y, a.c1[0][0].x * P0.y);
          if (outp) {
            Qn.x = fma(-a.c0[0][1].x, P1.x, fma(-a.c0[0][0].x, P0.x, Qn.x));
            Qn.y = fma(-a.c0[0][1].x, P1.y, fma(-a.c0[0][0].x, P0.y, Qn.y));
          }
        } else {
          csub_mul(Rn, a.c1[cy][0], P0);
          csub_mul(Rn, a.c1[cy][1], P1);
          Rn = make_double2(-Rn.x, -Rn.y);
          if (outp) {
            csub_mul(Qn, a.c0[2 * cx + cy][0], P0);
            csub_mul(Qn, a.c0[2 * cx + cy][1], P1);
          }
        }
      }
      const int64_t ix = ip - 1;
      if (ix >= xs && ix < xe) {
        const float2 rf = make_float2(round_d2f(Qc.x - Rm.x - Rn.x), round_d2f(Qc.y - Rm.y - Rn.y));
        r[ix * ny + iy] = rf;
        r2f = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, r2f));
      }
      if (outp) {
        const float fx = round_d2f(fv.x), fy = round_d2f(fv.y);
        f2f = fmaf(fx, fx, fmaf(fy, fy, f2f));
      }
      Rm = Rc;
      Rc = Rn;
      Qc = Qn;
    }
  }
  block_norms<256>(r2f, f2f, sums, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
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

cudaError_t launch_residual(int dim, const int64_t* n, const double* h, double omega, const double* wc,
                            const double2* f,
                            const double2* u, float2* r, double* sums, int64_t* nblocks, const int* skip,
                            cudaStream_t st, int* err, double mden) {
  const int bs = 256;
  if (dim == 2 || dim == 3) {
    // monomial coefficients by end class (see the FP64-instruction-lean kernels)
    ResidQArgs q{};
    for (int k = 0; k < dim; ++k) q.n[k] = n[k];
    using cd = std::complex<double>;
    auto Mk = [&](int k, int end, int bit) -> cd {
      const MassCoef m = mass_coef(h[k], mden);
      return bit ? m.off : (end ? m.end : m.in);
    };
    auto Kk = [&](int k, int end, int bit) -> cd {
      return bit ? cd(-1.0 / h[k], 0.0) : (end ? cd(1.0 / h[k], -wc[k]) : cd(2.0 / h[k], 0.0));
    };
    const double w2 = omega * omega;
    auto put = [](double2& d, cd v) { d = make_double2(v.real(), v.imag()); };
    if (dim == 3) {
      for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy)
          for (int cz = 0; cz < 2; ++cz)
            for (int a1 = 0; a1 < 2; ++a1)
              for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) {
                  const cd v = Kk(0, cx, a1) * Mk(1, cy, b) * Mk(2, cz, c) + Mk(0, cx, a1) * Kk(1, cy, b) * Mk(2, cz, c) +
                               Mk(0, cx, a1) * Mk(1, cy, b) * Kk(2, cz, c) - w2 * Mk(0, cx, a1) * Mk(1, cy, b) * Mk(2, cz, c);
                  if (a1 == 0) put(q.c0[4 * cx + 2 * cy + cz][2 * b + c], v);
                  else if (cx == 0) put(q.c1[2 * cy + cz][2 * b + c], v);
                }
      for (int cls = 0; cls < 8; ++cls)
        for (int bc = 0; bc < 4; ++bc) {
          q.dc0[cls][bc] = make_double2(q.c0[cls][bc].x - q.c0[cls & 4][bc].x, q.c0[cls][bc].y - q.c0[cls & 4][bc].y);
          if (cls < 4)
            q.dc1[cls][bc] = make_double2(q.c1[cls][bc].x - q.c1[0][bc].x, q.c1[cls][bc].y - q.c1[0][bc].y);
        }
      const dim3 grid((unsigned)((n[2] + QZ - 1) / QZ), (unsigned)((n[1] + QY - 1) / QY), (unsigned)((n[0] + QX - 1) / QX));
      *nblocks = (int64_t)grid.x * grid.y * grid.z;
      CUtensorMap um, fm;
      const cudaError_t attr = allow_dynamic_smem((const void*)k_residual3d_tma, kResidTmaSmem);
      if (attr == cudaSuccess && residual_map(&um, u, n, QZ + 2, QY + 2) && residual_map(&fm, f, n, QZ, QY))
        k_residual3d_tma<<<grid, dim3(QZ, QY), kResidTmaSmem, st>>>(um, fm, q, r, sums, skip, err);
      else
        k_residual3d_q<<<grid, dim3(QZ, QY), 0, st>>>(q, f, u, r, sums, skip);
      return cudaGetLastError();
    }
    for (int cx = 0; cx < 2; ++cx)
      for (int cy = 0; cy < 2; ++cy)
        for (int a1 = 0; a1 < 2; ++a1)
          for (int b = 0; b < 2; ++b) {
            const cd v = Kk(0, cx, a1) * Mk(1, cy, b) + Mk(0, cx, a1) * Kk(1, cy, b) - w2 * Mk(0, cx, a1) * Mk(1, cy, b);
            if (a1 == 0) put(q.c0[2 * cx + cy][b], v);
            else if (cx == 0) put(q.c1[cy][b], v);
          }
    const dim3 grid((unsigned)((n[1] + bs - 1) / bs), (unsigned)((n[0] + QR2 - 1) / QR2));
    *nblocks = (int64_t)grid.x * grid.y;
    k_residual2d_q<<<grid, bs, 0, st>>>(q, f, u, r, sums, skip);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

static FF2 split_host(double x) {
  FF2 c;
  c.h = (float)x;
  c.l = (float)(x - (double)c.h);
  return c;
}

cudaError_t launch_residual_ff(int dim, const int64_t* n, const double* h, double omega, const double* wc,
                               const float4* f,
                               const float4* u, float2* r, double* sums, int64_t* nblocks, const int* skip,
                               cudaStream_t st, double mden) {
  ResidFFArgs a{};
  a.omega = omega;
  const double w2 = omega * omega;
  for (int k = 0; k < dim; ++k) {
    a.n[k] = n[k];
    a.h[k] = h[k];
    const double hk = h[k];
    const MassCoef mk_ = mass_coef(hk, mden);
    AxisFF& x = a.ax[k];
    x.mdi = split_host(mk_.in);
    x.mde = split_host(mk_.end);
    x.mo = split_host(mk_.off);
    x.kdi = split_host(2.0 / hk);
    x.kder = split_host(1.0 / hk);
    x.ko = split_host(-1.0 / hk);
    x.kdei = split_host(-wc[k]);
    x.cdi = split_host(2.0 / hk - w2 * mk_.in);
    x.cde = split_host(1.0 / hk - w2 * mk_.end);
    x.co = split_host(-1.0 / hk - w2 * mk_.off);
  }
  if (dim == 2) {
    double m[2][3], kk[2][3];
    for (int k = 0; k < 2; ++k) {
      const MassCoef mk_ = mass_coef(h[k], mden);
      m[k][0] = m[k][2] = mk_.off;
      m[k][1] = mk_.in;
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
      const MassCoef mk_ = mass_coef(h[k], mden);
      if (d == 0) {
        m = end ? mk_.end : mk_.in;
        kr = (end ? 1.0 : 2.0) / h[k];
        ki = end ? -wc[k] : 0.0;
      } else {
        m = mk_.off;
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
    const int64_t fp64 = ((n[1] + 255) / 256) * ((n[0] + QR2 - 1) / QR2);
    const int64_t ff = ((n[1] - 2 + 255) / 256) * ((n[0] - 2 + RX2 - 1) / RX2) + (2 * n[1] + 2 * (n[0] - 2) + 255) / 256;
    return std::max(fp64, ff);
  }
  const int64_t ff = ((n[2] + TZ3 - 1) / TZ3) * ((n[1] + TY3 - 1) / TY3) * ((n[0] + RX3 - 1) / RX3);
  const int64_t q = ((n[2] + QZ - 1) / QZ) * ((n[1] + QY - 1) / QY) * ((n[0] + QX - 1) / QX);
  return std::max(ff, q);
}

cudaError_t launch_residual_finalize(const double* sums, int64_t nblocks, RefineState* state,
                                     unsigned long long cond, cudaStream_t st) {
  k_residual_finalize<<<1, 1024, 0, st>>>(sums, nblocks, state, (cudaGraphConditionalHandle)cond);
  return cudaGetLastError();
}

}  // namespace helm
