// 2D solve kernels (Section 4.2): per-mode tridiagonal solves along x with
// the Step-1/2/3 right-hand sides and boundary-row reductions, the C_bb face
// operator (eq. Cbb), and the FP64 residual of eq. A2D used by refinement.
//
// Layout: arrays [nx][n1], x1 = the last axis (n1 modes after the DFT), the
// tridiagonal axis is x (nx points, spacing hx).  Line l (one x1 mode) is the
// column {ix * n1 + l}; thread l owns it, so consecutive threads touch
// consecutive addresses at every ix.
//
// Per-mode tridiagonal (Section 4.1.2, blocks of eqs. HB2D / HA2D):
//   B modes: mu_l [K_x + (Lam^B_l - w^2) M_x],  Lam^B real (eq. eigvaluesPer)
//   A modes:       K_x + (Lam^A_l - w^2) M_x,    Lam^A complex (eq. EVP1a)
// solved by the Thomas algorithm (LU without pivoting).  The forward sweep
// stores (c'_ix, d'_ix) in scratch; the backward sweep reads them back.
#include <algorithm>

#include "helm_dft.h"
#include "helm_kernels.cuh"
#include "helm_solve.h"

namespace helm {

namespace {

template <typename C>
struct Thomas {
  LineCoef<C> k;
  int n;
  C c_prev, d_prev;
  __device__ __forceinline__ void first(C r, C& c, C& d) {
    C inv = crecip(k.ac);
    c = cmul(k.b, inv);
    d = cmul(r, inv);
    c_prev = c;
    d_prev = d;
  }
  __device__ __forceinline__ void step(int ix, C r, C& c, C& d) {
    C a = (ix == n - 1) ? k.ac : k.a;
    C den = csub(a, cmul(k.b, c_prev));
    C inv = crecip(den);
    c = cmul(k.b, inv);
    d = cmul(csub(r, cmul(k.b, d_prev)), inv);
    c_prev = c;
    d_prev = d;
  }
};

// Step 1 (eqs. 2dLUBs1, 2dBs1): z_l = (1/mu_l) T_l^-1 fhat_l, reduced to the
// x1 faces v_1 = (1/n1) sum_l z_l, v_n = (1/n1) sum_l e^{-2 pi i l/n1} z_l.
// Step 3 (eqs. 2dLUBs3): rhs fhat_l + d_1 + e^{+2 pi i l/n1} d_n (the DFT of
// the rank-2 correction, eq. step3term), z3 written to `out`.
// Step 2 (eqs. step2-1..step2-3): rhs (c_1 + par_l c_n) (= g_l / V[1,l]),
// solve with T^A_l, reduce w_1 = sum sigma_l z, w_n = sum par_l sigma_l z.
template <typename T, int STEP>
__global__ void __launch_bounds__(128) k_tri2d(const typename cpx<T>::type* __restrict__ fhat,
                                               typename cpx<T>::type* __restrict__ cbuf,
                                               typename cpx<T>::type* __restrict__ dbuf,
                                               typename cpx<T>::type* __restrict__ partial,
                                               const typename cpx<T>::type* __restrict__ faces,
                                               Solve2DArgs a, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // a warp lying entirely beyond the last mode has no work and no partial slot
  if ((l & ~(int64_t)31) >= n1) return;
  const bool act = l < n1;
  const int64_t lc = act ? l : 0;
  // line coefficients
  double sre, sim;
  if (STEP == 2) {
    sre = a.lamA[2 * lc] - a.omega * a.omega;
    sim = a.lamA[2 * lc + 1];
  } else {
    sre = a.lamB[lc] - a.omega * a.omega;
    sim = 0.0;
  }
  Thomas<C> th;
  th.k = line_coef<C>(sre, sim, a.hx, a.omega);
  th.n = (int)nx;
  const T scal = (STEP == 2) ? T(1) : (T)(1.0 / a.muB[lc]);
  const C twl = mk<C>(a.tw[2 * lc], a.tw[2 * lc + 1]);  // e^{-2 pi i l / n1}
  const T par = (T)a.parA[lc];
  const C sig = mk<C>(a.sigA[2 * lc], a.sigA[2 * lc + 1]);
  const C* f1 = faces;       // Step 2: c_1 ; Step 3: d_1
  const C* fn = faces + nx;  // Step 2: c_n ; Step 3: d_n
  auto rhs = [&](int64_t ix) -> C {
    if (STEP == 1) return cscale(fhat[ix * n1 + lc], scal);
    if (STEP == 2) return cadd(f1[ix], cscale(fn[ix], par));
    // STEP 3: fhat + d_1 + conj(twl) d_n
    C v = cadd(fhat[ix * n1 + lc], f1[ix]);
    v = cadd(v, cmulc(fn[ix], twl));
    return cscale(v, scal);
  };
  if (act) {
    C c, d;
    th.first(rhs(0), c, d);
    cbuf[lc] = c;
    dbuf[lc] = d;
    for (int64_t ix = 1; ix < nx; ++ix) {
      th.step((int)ix, rhs(ix), c, d);
      cbuf[ix * n1 + lc] = c;
      dbuf[ix * n1 + lc] = d;
    }
  }
  // backward sweep
  const int lane = threadIdx.x & 31;
  const int64_t warp = l >> 5;
  const int64_t nwarps = (n1 + 31) >> 5;
  C x = mk<C>(0, 0);
  for (int64_t ix = nx - 1; ix >= 0; --ix) {
    if (act) {
      C d = dbuf[ix * n1 + lc];
      x = (ix == nx - 1) ? d : csub(d, cmul(cbuf[ix * n1 + lc], x));
    }
    if (STEP == 3) {
      if (act) dbuf[ix * n1 + lc] = x;
    } else {
      C s1, sn;
      if (STEP == 1) {
        s1 = act ? x : mk<C>(0, 0);
        sn = act ? cmul(x, twl) : mk<C>(0, 0);
      } else {
        C t = act ? cmul(x, sig) : mk<C>(0, 0);
        s1 = t;
        sn = cscale(t, par);
      }
      s1 = warp_sum(s1);
      sn = warp_sum(sn);
      if (lane == 0) {
        partial[warp * nx + ix] = s1;
        partial[(nwarps + warp) * nx + ix] = sn;
      }
    }
  }
}

// Sum the per-warp partials: out[face * nx + ix] = scale * sum_w partial.
template <typename T>
__global__ void k_reduce_faces(const typename cpx<T>::type* __restrict__ partial,
                               typename cpx<T>::type* __restrict__ out, int64_t nx, int64_t nwarps,
                               double scale, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * nx) return;
  const int64_t face = i / nx, ix = i - face * nx;
  C acc = mk<C>(0, 0);
  for (int64_t w = 0; w < nwarps; ++w) acc = cadd(acc, partial[(face * nwarps + w) * nx + ix]);
  out[i] = cscale(acc, (decltype(acc.x))scale);
}

// C_bb applied to the x1 faces (eqs. BminA, Cbb):
//   c_1 = D11 M v_1 + E11 K v_1 + D1n M v_n + E1n K v_n,  c_n symmetric,
// with D11 = (1 + i w h1)/h1 - p h1/3, D1n = -1/h1 - p h1/6, E11 = h1/3,
// E1n = h1/6 (p = w^2 for the outer problem), M, K along x (spacing hx,
// absorbing corners).  in = v (+ w if `in2`), out = c.
template <typename T>
__global__ void k_apply_cbb(const typename cpx<T>::type* __restrict__ in,
                            const typename cpx<T>::type* __restrict__ in2,
                            typename cpx<T>::type* __restrict__ out, int64_t nx, double hx, double h1,
                            double omega, double p, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= nx) return;
  auto get = [&](int face, int64_t j) -> C {
    C v = in[face * nx + j];
    if (in2) v = cadd(v, in2[face * nx + j]);
    return v;
  };
  // M and K rows of x at ix
  const bool end = (ix == 0 || ix == nx - 1);
  const double md = end ? 2.0 * hx / 6.0 : 4.0 * hx / 6.0, mo = hx / 6.0;
  const double kd_re = end ? 1.0 / hx : 2.0 / hx, kd_im = end ? -omega : 0.0, ko = -1.0 / hx;
  C Mv[2], Kv[2];
  for (int f = 0; f < 2; ++f) {
    C v0 = get(f, ix);
    C vm = ix > 0 ? get(f, ix - 1) : mk<C>(0, 0);
    C vp = ix < nx - 1 ? get(f, ix + 1) : mk<C>(0, 0);
    C nb = cadd(vm, vp);
    Mv[f] = cadd(cscale(v0, (decltype(v0.x))md), cscale(nb, (decltype(v0.x))mo));
    Kv[f] = cadd(cmul(v0, mk<C>(kd_re, kd_im)), cscale(nb, (decltype(v0.x))ko));
  }
  const C D11 = mk<C>(1.0 / h1 - p * h1 / 3.0, omega);
  const C D1n = mk<C>(-1.0 / h1 - p * h1 / 6.0, 0.0);
  const auto E11 = (decltype(D11.x))(h1 / 3.0), E1n = (decltype(D11.x))(h1 / 6.0);
  C c1 = cadd(cadd(cmul(D11, Mv[0]), cscale(Kv[0], E11)), cadd(cmul(D1n, Mv[1]), cscale(Kv[1], E1n)));
  C cn = cadd(cadd(cmul(D1n, Mv[0]), cscale(Kv[0], E1n)), cadd(cmul(D11, Mv[1]), cscale(Kv[1], E11)));
  out[ix] = c1;
  out[nx + ix] = cn;
}

}  // namespace

cudaError_t launch_tri2d(int prec, int step, const void* fhat, void* cbuf, void* dbuf, void* partial,
                         const void* faces, const Solve2DArgs& a, const int* skip, cudaStream_t st) {
  const int bs = 128;
  const unsigned grid = (unsigned)((a.n1 + bs - 1) / bs);
#define HELM_TRI_LAUNCH(T, S)                                                                          \
  k_tri2d<T, S><<<grid, bs, 0, st>>>(                                                                  \
      (const cpx<T>::type*)fhat, (cpx<T>::type*)cbuf, (cpx<T>::type*)dbuf, (cpx<T>::type*)partial,   \
      (const cpx<T>::type*)faces, a, skip)
  if (prec == kPrecF64) {
    if (step == 1) HELM_TRI_LAUNCH(double, 1);
    else if (step == 2) HELM_TRI_LAUNCH(double, 2);
    else HELM_TRI_LAUNCH(double, 3);
  } else {
    if (step == 1) HELM_TRI_LAUNCH(float, 1);
    else if (step == 2) HELM_TRI_LAUNCH(float, 2);
    else HELM_TRI_LAUNCH(float, 3);
  }
#undef HELM_TRI_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_reduce_faces(int prec, const void* partial, void* out, int64_t nx, int64_t nwarps,
                                double scale, const int* skip, cudaStream_t st) {
  const int bs = 256;
  const unsigned grid = (unsigned)((2 * nx + bs - 1) / bs);
  if (prec == kPrecF64)
    k_reduce_faces<double><<<grid, bs, 0, st>>>((const double2*)partial, (double2*)out, nx, nwarps, scale, skip);
  else
    k_reduce_faces<float><<<grid, bs, 0, st>>>((const float2*)partial, (float2*)out, nx, nwarps, scale, skip);
  return cudaGetLastError();
}

cudaError_t launch_apply_cbb(int prec, const void* in, const void* in2, void* out, int64_t nx, double hx,
                             double h1, double omega, double p, const int* skip, cudaStream_t st) {
  const int bs = 256;
  const unsigned grid = (unsigned)((nx + bs - 1) / bs);
  if (prec == kPrecF64)
    k_apply_cbb<double><<<grid, bs, 0, st>>>((const double2*)in, (const double2*)in2, (double2*)out, nx, hx,
                                             h1, omega, p, skip);
  else
    k_apply_cbb<float><<<grid, bs, 0, st>>>((const float2*)in, (const float2*)in2, (float2*)out, nx, hx, h1,
                                            omega, p, skip);
  return cudaGetLastError();
}

}  // namespace helm
