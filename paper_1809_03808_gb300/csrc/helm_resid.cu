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

__global__ void k_residual_finalize(const double* __restrict__ sums, int64_t nblocks, RefineState* st,
                                    int last) {
  if (st->done) return;
  __shared__ double sr[256], sf[256];
  double a2 = 0, b2 = 0;
  for (int64_t i = threadIdx.x; i < nblocks; i += blockDim.x) {
    a2 += sums[2 * i];
    b2 += sums[2 * i + 1];
  }
  sr[threadIdx.x] = a2;
  sf[threadIdx.x] = b2;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      sf[threadIdx.x] += sf[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double rel = sf[0] > 0 ? sqrt(sr[0] / sf[0]) : sqrt(sr[0]);
    const int it = st->iters;
    if (it < 16) st->resid[it] = rel;
    st->iters = it + 1;
    st->fnorm2 = sf[0];
    if (rel <= st->tol) {
      st->converged = 1;
      st->done = 1;
    } else if (last) {
      st->done = 1;
    }
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
  const int64_t grid = (N + bs - 1) / bs;
  *nblocks = grid;
  k_residual<<<(unsigned)grid, bs, 0, st>>>(a, f, u, r, sums, N, skip);
  return cudaGetLastError();
}

cudaError_t launch_residual_finalize(const double* sums, int64_t nblocks, RefineState* state, int last,
                                     cudaStream_t st) {
  k_residual_finalize<<<1, 256, 0, st>>>(sums, nblocks, state, last);
  return cudaGetLastError();
}

}  // namespace helm
