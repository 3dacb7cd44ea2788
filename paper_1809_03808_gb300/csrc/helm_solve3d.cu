// 3D solve (Section 5): the three steps along the outer periodic axis, each
// per-mode block solve H_A^-1 / H_B^-1 (eqs. HA3D, HB3D) done by the 2D fast
// solver on the remaining plane (Section 5.1.2, eqs. A2D2, B2D2 and their
// auxiliaries A2D2aux, B2D2aux).
//
// Array [nx][ny][nz], z fastest.  Outer periodic axis ("x1") = y, inner
// periodic axis ("x2") = z, tridiagonal axis = x.  After the 2D DFT over
// (y, z) the unknowns are indexed (x, l, m): l outer mode, m inner mode.
//
// k_plane3d: one CTA per outer mode l, one thread per inner mode m.  The CTA
// runs the inner Steps 1-3 for plane l (the 2D algorithm of Section 4.2 with
// mass shift p = w^2 - Lam_{1,l}; the absorbing corners keep the physical w),
// reducing the inner boundary rows over m in shared memory.  Its output is the
// inner-mode-space solution y3(x, l, m), written over the Thomas scratch.
// The outer boundary rows are then reduced over l by k_reduce_outer.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>
#include <type_traits>

#include "helm_async.cuh"
#include "helm_dft.h"
#include "helm_kernels.cuh"
#include "helm_solve3d.h"

namespace helm {

namespace {

struct Plane3DArgs {
  int64_t nx, ny, nz;
  double hx, hy, hz, omega;
  double wx, wy, wz;  // w of the absorbing ends of each axis (0: Neumann axis)
  // outer axis (y) eigen-data (Lam^B and 1/mu complex: gamma-circulant auxiliary)
  const double *lamBo, *invmuo, *lamAo, *sigAo, *parAo, *two;
  // inner axis (z) eigen-data
  const double *lamBi, *invmui, *lamAi, *sigAi, *parAi, *twi;
  double en_o[2], eninv_o[2], g_o[2], ginv_o[2];
  double en_i[2], eninv_i[2], g_i[2], ginv_i[2];
  double mden;  // mass matrix denominator (MassCoef): 6 the paper's elements, 12 the modified ones
};

constexpr int XC = 32;  // rows per reduction chunk

constexpr int kMW = 16;       // inner modes per tile
constexpr int kLineVals = 5;  // per-line table values (see k_plane_tables)
constexpr int kPivRows = 32;  // pivot rows staged in shared memory (rows below a line's settling row)
constexpr int kRoutedFlag = 1 << 30;  // in the settling-row table: the line is solved in FP64
// Routing is off by default: the complex64 solve's error does sit in the
// near-singular lines (92 % of it in 1 % of the lines on a 160^3 grid of the
// 512^3 workload's spacing and wave number), but it is the complex64
// rounding of those modes' inputs, amplified by the line's conditioning, not
// the FP32 arithmetic of its sweeps: FP64 sweeps leave it unchanged (-0.6 %).
constexpr double kDefaultRouteTau = 0.0;

template <typename C>
struct ThomasRow {
  LineCoef<C> k;
  int n;
  C c_prev, d_prev;
  __device__ __forceinline__ void step(int ix, C r, C& c, C& d) {
    if (ix == 0) {
      C inv = crecip(k.ac);
      c = cmul(k.b, inv);
      d = cmul(r, inv);
    } else {
      C a = (ix == n - 1) ? k.ac : k.a;
      C den = csub(a, cmul(k.b, c_prev));
      C inv = crecip(den);
      c = cmul(k.b, inv);
      d = cmul(csub(r, cmul(k.b, d_prev)), inv);
    }
    c_prev = c;
    d_prev = d;
  }
};

// Inner C_bb of the plane problem (eq. Cbb for the auxiliary B2D2aux):
//   c_1 = D11 M v_1 + E11 K v_1 + D1n M v_n + E1n K v_n  (and symmetric c_n),
//   D11 = (1 + i w hz)/hz - p hz/3, D1n = -1/hz - p hz/6, E11 = hz/3, E1n = hz/6,
// M, K along x; p = w^2 - Lam_{1,l} (complex for outer A modes).
template <typename C>
__device__ void plane_cbb(const C* v, const C* w2, C* out, int nx, double hx, double hz, double wx, double wz,
                          double pre, double pim, C g, C ginv, double mden) {
  for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
    auto get = [&](int face, int j) -> C {
      C t = v[face * nx + j];
      if (w2) t = cadd(t, w2[face * nx + j]);
      return t;
    };
    const bool end = (ix == 0 || ix == nx - 1);
    const MassCoef mc = mass_coef(hx, mden), mcz = mass_coef(hz, mden);
    const double md = end ? mc.end : mc.in, mo = mc.off;
    const double kdr = end ? 1.0 / hx : 2.0 / hx, kdi = end ? -wx : 0.0, ko = -1.0 / hx;
    C Mv[2], Kv[2];
    for (int f = 0; f < 2; ++f) {
      C v0 = get(f, ix);
      C vm = ix > 0 ? get(f, ix - 1) : mk<C>(0, 0);
      C vp = ix < nx - 1 ? get(f, ix + 1) : mk<C>(0, 0);
      C nb = cadd(vm, vp);
      Mv[f] = cadd(cscale(v0, (decltype(v0.x))md), cscale(nb, (decltype(v0.x))mo));
      Kv[f] = cadd(cmul(v0, mk<C>(kdr, kdi)), cscale(nb, (decltype(v0.x))ko));
    }
    const C D11 = mk<C>(1.0 / hz - pre * mcz.end, wz - pim * mcz.end);
    const C D1n = mk<C>(-1.0 / hz - pre * mcz.off, -pim * mcz.off);
    const auto E11 = (decltype(D11.x))mcz.end, E1n = (decltype(D11.x))mcz.off;
    out[ix] = cadd(cadd(cmul(D11, Mv[0]), cscale(Kv[0], E11)), cmul(ginv, cadd(cmul(D1n, Mv[1]), cscale(Kv[1], E1n))));
    out[nx + ix] = cadd(cmul(g, cadd(cmul(D1n, Mv[0]), cscale(Kv[0], E1n))), cadd(cmul(D11, Mv[1]), cscale(Kv[1], E11)));
  }
}

// OSTEP 1: G = fhat / mu_l                        (outer Step 1, eq. 3dHBs1)
// OSTEP 2: G = chat_1 + par_l chat_n, outer A mode (outer Step 2, eq. step2-2-3d)
// OSTEP 3: G = (fhat + dhat_1 + e^{+i theta_l} e^{-t(ny-1)} dhat_n) / mu_l  (eq. 3dHBs3)
// TAB: read the reciprocal pivots 1/den_ix of the inner lines from per-plan
// tables (tabB: inner B-type lines, tabA: inner A-type, both for this outer
// mode type) instead of recomputing them; the forward sweep then stores only
// d and the backward sweep rebuilds c = b / den from the table.
template <typename T, int OSTEP, bool TAB>
__global__ void __launch_bounds__(1024) k_plane3d(const typename cpx<T>::type* __restrict__ fhat,
                                                  typename cpx<T>::type* __restrict__ cbuf,
                                                  typename cpx<T>::type* __restrict__ dbuf,
                                                  const typename cpx<T>::type* __restrict__ gfaces,
                                                  const typename cpx<T>::type* __restrict__ tabB,
                                                  const typename cpx<T>::type* __restrict__ tabA,
                                                  Plane3DArgs a, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = (int)a.nx;
  const int64_t ny = a.ny, nz = a.nz;
  const int nw = blockDim.x >> 5;
  C* vin = reinterpret_cast<C*>(smem_raw);  // [2][nx]
  C* win = vin + 2 * nx;                     // [2][nx]
  C* cin = win + 2 * nx;                     // [2][nx]
  C* red = cin + 2 * nx;                     // [nw][2][XC]
  const int64_t l = blockIdx.x;
  const int m = threadIdx.x;
  const bool act = m < nz;
  const int64_t mc = act ? m : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double w2 = a.omega * a.omega;
  // outer-mode quantities
  double lo_re, lo_im;
  if (OSTEP == 2) {
    lo_re = a.lamAo[2 * l];
    lo_im = a.lamAo[2 * l + 1];
  } else {
    lo_re = a.lamBo[2 * l];
    lo_im = a.lamBo[2 * l + 1];
  }
  const C gscale = (OSTEP == 2) ? mk<C>(1, 0) : mk<C>(a.invmuo[2 * l], a.invmuo[2 * l + 1]);
  const T paro = (T)a.parAo[l];
  // e^{+i theta_l} e^{-t(ny-1)}: weight of the last outer face in the Step-3 rhs
  const C wl = cmul(mk<C>(a.two[2 * l], -a.two[2 * l + 1]), mk<C>(a.eninv_o[0], a.eninv_o[1]));
  // inner-mode quantities
  const double lBi_re = a.lamBi[2 * mc], lBi_im = a.lamBi[2 * mc + 1];
  const C twm = mk<C>(a.twi[2 * mc], a.twi[2 * mc + 1]);
  const C wm = cmul(mk<C>(a.twi[2 * mc], -a.twi[2 * mc + 1]), mk<C>(a.eninv_i[0], a.eninv_i[1]));
  const C invmu_i = mk<C>(a.invmui[2 * mc], a.invmui[2 * mc + 1]);
  const C gi = mk<C>(a.g_i[0], a.g_i[1]), giv = mk<C>(a.ginv_i[0], a.ginv_i[1]);
  const T pari = (T)a.parAi[mc];
  const C sigi = mk<C>(a.sigAi[2 * mc], a.sigAi[2 * mc + 1]);
  const int64_t plane = l * nz + mc;                 // offset inside an x slab
  const int64_t xs = ny * nz;                         // x stride
  const C* g1 = gfaces;                               // [2][nx][nz]
  const C* gn = gfaces ? gfaces + (int64_t)nx * nz : nullptr;
  auto G = [&](int ix) -> C {
    if (OSTEP == 1) return cmul(fhat[ix * xs + plane], gscale);
    if (OSTEP == 2) return cadd(g1[(int64_t)ix * nz + mc], cscale(gn[(int64_t)ix * nz + mc], paro));
    C v = cadd(fhat[ix * xs + plane], g1[(int64_t)ix * nz + mc]);
    v = cadd(v, cmul(gn[(int64_t)ix * nz + mc], wl));
    return cmul(v, gscale);
  };
  ThomasRow<C> thB, thA;
  thB.k = line_coef<C>(lo_re + lBi_re - w2, lo_im + lBi_im, a.hx, a.wx, a.mden);
  thB.n = nx;
  thA.k = line_coef<C>(lo_re + a.lamAi[2 * mc] - w2, lo_im + a.lamAi[2 * mc + 1], a.hx, a.wx, a.mden);
  thA.n = nx;
  const double pre = w2 - lo_re, pim = -lo_im;

  // ---- generic sweep: forward with rhs(ix), backward with emit(ix, x) ----
  // rows are processed in batches of PB: the batch's right-hand sides (and,
  // backward, its scratch values) are loaded before the dependent recurrence
  constexpr int PB = 8;
  auto forward = [&](ThomasRow<C>& th, const C* tab, auto rhs) {
    if (!act) return;
    for (int i0 = 0; i0 < nx; i0 += PB) {
      C rr[PB], iv[PB];
#pragma unroll
      for (int t = 0; t < PB; ++t)
        if (i0 + t < nx) {
          rr[t] = rhs(i0 + t);
          if (TAB) iv[t] = tab[(i0 + t) * xs + plane];
        }
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        const int ix = i0 + t;
        if (ix < nx) {
          if (TAB) {
            const C d = cmul(ix == 0 ? rr[t] : csub(rr[t], cmul(th.k.b, th.d_prev)), iv[t]);
            th.d_prev = d;
            dbuf[ix * xs + plane] = d;
          } else {
            C c, d;
            th.step(ix, rr[t], c, d);
            cbuf[ix * xs + plane] = c;
            dbuf[ix * xs + plane] = d;
          }
        }
      }
    }
  };
  // c_ix of the line: from the scratch, or b / den_ix from the table
  auto cval = [&](const ThomasRow<C>& th, const C* tab, int ix) -> C {
    if (TAB) return cmul(th.k.b, tab[ix * xs + plane]);
    return cbuf[ix * xs + plane];
  };
  // backward sweep reducing (s1, sn) contributions over m into out[2][nx]
  auto backward_reduce = [&](const ThomasRow<C>& th, const C* tab, auto contrib, C* out, C scale0, C scale1) {
    C x = mk<C>(0, 0);
    for (int x0 = nx - 1; x0 >= 0; x0 -= XC) {
      const int x1 = max(0, x0 - XC + 1);
      for (int b0 = x0; b0 >= x1; b0 -= PB) {
        C dd[PB], cc[PB];
#pragma unroll
        for (int t = 0; t < PB; ++t) {
          const int ix = b0 - t;
          if (act && ix >= x1) {
            dd[t] = dbuf[ix * xs + plane];
            cc[t] = cval(th, tab, ix);
          }
        }
#pragma unroll
        for (int t = 0; t < PB; ++t) {
          const int ix = b0 - t;
          if (ix < x1) break;
          if (act) x = (ix == nx - 1) ? dd[t] : csub(dd[t], cmul(cc[t], x));
          C s1, sn;
          contrib(act, x, s1, sn);
          s1 = warp_sum(s1);
          sn = warp_sum(sn);
          if (lane == 0) {
            red[(warp * 2 + 0) * XC + (x0 - ix)] = s1;
            red[(warp * 2 + 1) * XC + (x0 - ix)] = sn;
          }
        }
      }
      __syncthreads();
      const int cnt = x0 - x1 + 1;
      for (int t = threadIdx.x; t < 2 * cnt; t += blockDim.x) {
        const int face = t / cnt, j = t - face * cnt;
        C acc = mk<C>(0, 0);
        for (int w = 0; w < nw; ++w) acc = cadd(acc, red[(w * 2 + face) * XC + j]);
        out[face * nx + (x0 - j)] = cmul(acc, face == 0 ? scale0 : scale1);
      }
      __syncthreads();
    }
  };

  // inner Step 1: B-aux solve, reduce to inner faces v_in
  forward(thB, tabB, [&](int ix) { return cmul(G(ix), invmu_i); });
  backward_reduce(
      thB, tabB,
      [&](bool ac, C x, C& s1, C& sn) {
        s1 = ac ? x : mk<C>(0, 0);
        sn = ac ? cmul(x, twm) : mk<C>(0, 0);
      },
      vin, mk<C>(1.0 / (double)nz, 0), mk<C>(a.en_i[0] / (double)nz, a.en_i[1] / (double)nz));
  plane_cbb(vin, (const C*)nullptr, cin, nx, a.hx, a.hz, a.wx, a.wz, pre, pim, gi, giv, a.mden);
  __syncthreads();
  // inner Step 2: A solve on the generated rhs, reduce to w_in
  forward(thA, tabA, [&](int ix) { return cadd(cin[ix], cscale(cin[nx + ix], pari)); });
  backward_reduce(
      thA, tabA,
      [&](bool ac, C x, C& s1, C& sn) {
        C t = ac ? cmul(x, sigi) : mk<C>(0, 0);
        s1 = t;
        sn = cscale(t, pari);
      },
      win, mk<C>(1, 0), mk<C>(1, 0));
  plane_cbb(vin, win, cin, nx, a.hx, a.hz, a.wx, a.wz, pre, pim, gi, giv, a.mden);
  __syncthreads();
  // inner Step 3: corrected B-aux solve, y3 written over the scratch
  forward(thB, tabB, [&](int ix) {
    C v = cadd(G(ix), cin[ix]);
    v = cadd(v, cmul(cin[nx + ix], wm));
    return cmul(v, invmu_i);
  });
  if (act) {
    C x = mk<C>(0, 0);
    for (int b0 = nx - 1; b0 >= 0; b0 -= PB) {
      C dd[PB], cc[PB];
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        const int ix = b0 - t;
        if (ix >= 0) {
          dd[t] = dbuf[ix * xs + plane];
          cc[t] = cval(thB, tabB, ix);
        }
      }
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        const int ix = b0 - t;
        if (ix < 0) break;
        x = (ix == nx - 1) ? dd[t] : csub(dd[t], cmul(cc[t], x));
        dbuf[ix * xs + plane] = x;
      }
    }
  }
}

// Outer boundary rows (eq. 3dBs1 / step2-3-3d) in inner-mode space:
//   out[face][x][m] = sum_l wgt_face(l) * y3(x, l, m)
// step 1: wgt = (1/ny, e^{-2 pi i l/ny}/ny); step 2: wgt = (sigma_l, par_l sigma_l).
// The weights of a run of outer modes are staged in shared memory in the
// compute precision; each thread sums over l in order, loading kOuterBatch
// values ahead of the dependent sums.
constexpr int kOuterChunk = 1024;
constexpr int kOuterBatch = 8;
template <typename T, int OSTEP>
__global__ void __launch_bounds__(256) k_reduce_outer(const typename cpx<T>::type* __restrict__ y3,
                                                      typename cpx<T>::type* __restrict__ out, Plane3DArgs a,
                                                      const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;  // uniform over the grid
  __shared__ C sw[kOuterChunk];
  __shared__ T sp[OSTEP == 2 ? kOuterChunk : 1];
  const int64_t ny = a.ny, nz = a.nz;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i < a.nx * nz;
  const int64_t ix = act ? i / nz : 0, m = act ? i - ix * nz : 0;
  const C* src = y3 + ix * ny * nz + m;
  C s1 = mk<C>(0, 0), sn = mk<C>(0, 0);
  auto add = [&](C v, int j) {
    if (OSTEP == 1) {
      s1 = cadd(s1, v);
      sn = cadd(sn, cmul(v, sw[j]));
    } else {
      const C t = cmul(v, sw[j]);
      s1 = cadd(s1, t);
      sn = cadd(sn, cscale(t, sp[j]));
    }
  };
  for (int64_t l0 = 0; l0 < ny; l0 += kOuterChunk) {
    const int cnt = (int)min((int64_t)kOuterChunk, ny - l0);
    __syncthreads();  // the previous run's weights are consumed
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int64_t l = l0 + j;
      if (OSTEP == 1) {
        sw[j] = mk<C>(a.two[2 * l], a.two[2 * l + 1]);
      } else {
        sw[j] = mk<C>(a.sigAo[2 * l], a.sigAo[2 * l + 1]);
        sp[j] = (T)a.parAo[l];
      }
    }
    __syncthreads();
    if (act) {
      int j = 0;
      for (; j + kOuterBatch <= cnt; j += kOuterBatch) {
        C v[kOuterBatch];
#pragma unroll
        for (int q = 0; q < kOuterBatch; ++q) v[q] = src[(l0 + j + q) * nz];
#pragma unroll
        for (int q = 0; q < kOuterBatch; ++q) add(v[q], j + q);
      }
      for (; j < cnt; ++j) add(src[(l0 + j) * nz], j);
    }
  }
  if (!act) return;
  if (OSTEP == 1) {
    s1 = cscale(s1, (decltype(s1.x))(1.0 / (double)ny));
    sn = cmul(sn, mk<C>(a.en_o[0] / (double)ny, a.en_o[1] / (double)ny));
  }
  out[i] = s1;
  out[a.nx * nz + i] = sn;
}

// Outer C_bb on the y faces (eq. Cbb for eq. B3D - A3D): with P = M_x (x) M_z
// and S = K_x (x) M_z + M_x (x) K_z - w^2 M_x (x) M_z on the (x, z) plane,
//   c_1 = (hy/3) S v_1 + ((1 + i w hy)/hy) P v_1 + g^-1 [(hy/6) S v_n - (1/hy) P v_n],
//   c_n = g [(hy/6) S v_1 - (1/hy) P v_1] + (hy/3) S v_n + ((1 + i w hy)/hy) P v_n,
// g the wrap factor of the gamma-circulant auxiliary (1: periodic).
template <typename T>
__global__ void k_outer_cbb(const typename cpx<T>::type* __restrict__ v, const typename cpx<T>::type* __restrict__ w,
                            typename cpx<T>::type* __restrict__ out, Plane3DArgs a, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int64_t nx = a.nx, nz = a.nz;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx * nz) return;
  const int64_t ix = i / nz, iz = i - ix * nz;
  auto ent = [&](int64_t n, double h, double w, int64_t j, int d, double& m, double& kr, double& ki) {
    const bool end = (j == 0 || j == n - 1);
    const MassCoef mc = mass_coef(h, a.mden);
    if (d == 0) {
      m = end ? mc.end : mc.in;
      kr = (end ? 1.0 : 2.0) / h;
      ki = end ? -w : 0.0;
    } else {
      m = mc.off;
      kr = -1.0 / h;
      ki = 0.0;
    }
  };
  C Sv[2] = {mk<C>(0, 0), mk<C>(0, 0)}, Pv[2] = {mk<C>(0, 0), mk<C>(0, 0)};
  const double w2 = a.omega * a.omega;
  for (int dx = -1; dx <= 1; ++dx) {
    const int64_t jx = ix + dx;
    if (jx < 0 || jx >= nx) continue;
    double mx, kxr, kxi;
    ent(nx, a.hx, a.wx, ix, dx, mx, kxr, kxi);
    for (int dz = -1; dz <= 1; ++dz) {
      const int64_t jz = iz + dz;
      if (jz < 0 || jz >= nz) continue;
      double mz, kzr, kzi;
      ent(nz, a.hz, a.wz, iz, dz, mz, kzr, kzi);
      const C cs = mk<C>(kxr * mz + mx * kzr - w2 * mx * mz, kxi * mz + mx * kzi);
      const auto cp = (decltype(cs.x))(mx * mz);
      for (int f = 0; f < 2; ++f) {
        C t = v[f * nx * nz + jx * nz + jz];
        if (w) t = cadd(t, w[f * nx * nz + jx * nz + jz]);
        Sv[f] = cadd(Sv[f], cmul(cs, t));
        Pv[f] = cadd(Pv[f], cscale(t, cp));
      }
    }
  }
  using T2 = decltype(Sv[0].x);
  const MassCoef mcy = mass_coef(a.hy, a.mden);
  const T2 e11 = (T2)mcy.end, e1n = (T2)mcy.off;
  const C d11 = mk<C>(1.0 / a.hy, a.wy);
  const T2 d1n = (T2)(-1.0 / a.hy);
  const C g = mk<C>(a.g_o[0], a.g_o[1]), gv = mk<C>(a.ginv_o[0], a.ginv_o[1]);
  out[i] = cadd(cadd(cscale(Sv[0], e11), cmul(d11, Pv[0])), cmul(gv, cadd(cscale(Sv[1], e1n), cscale(Pv[1], d1n))));
  out[nx * nz + i] = cadd(cmul(g, cadd(cscale(Sv[0], e1n), cscale(Pv[0], d1n))), cadd(cscale(Sv[1], e11), cmul(d11, Pv[1])));
}

// Reciprocal pivots of the inner tridiagonal lines of one line type (outer
// mode type x inner mode type), for every (x, l, m): the FP64 recurrence of
// ThomasRow, stored in the compute precision at the layout of the scratch.
//
// Per line it also records where the recurrence u_j = a - b^2 / u_{j-1}
// (constant a, b inside the line) has settled at its attracting fixed point
// u_inf, the root of u^2 - a u + b^2 = 0 of larger modulus: rows j >= len
// (below the last row) satisfy |1/u_j - 1/u_inf| <= tol |1/u_inf| (tol 2^-27
// for complex64 tables, a quarter of the FP32 rounding; 2^-50 for
// complex128), so the tiled sweeps read the table only for rows < len and use
// 1/u_inf beyond.  Per line (kLineVals values, line = l * nz + m): 1/u_inf,
// 1/u_{nx-1} (the corner row), the off-diagonal b of the line matrix, and
// the carry coefficients alpha, beta of a chunk of ch settled rows (see
// k_inner3d), all from the FP64 values.  For propagating modes the
// pivots keep oscillating and len covers the whole line.

template <typename T>
__global__ void k_plane_tables(typename cpx<T>::type* __restrict__ tab, typename cpx<T>::type* __restrict__ lend,
                               int* __restrict__ lenL, Plane3DArgs a, int outerA, int innerA, int ch) {
  using C = typename cpx<T>::type;
  const int64_t ny = a.ny, nz = a.nz, nx = a.nx;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // l * nz + m
  if (i >= ny * nz) return;
  const int64_t l = i / nz, m = i - l * nz;
  const double* lo = outerA ? a.lamAo : a.lamBo;
  const double* li = innerA ? a.lamAi : a.lamBi;
  const double w2 = a.omega * a.omega;
  const LineCoef<double2> k = line_coef<double2>(lo[2 * l] + li[2 * m] - w2, lo[2 * l + 1] + li[2 * m + 1], a.hx, a.wx, a.mden);
  // attracting fixed point of the interior recurrence
  const double2 disc = csqrt_d(csub(cmul(k.a, k.a), cscale(cmul(k.b, k.b), 4.0)));
  const double2 r1 = cscale(cadd(k.a, disc), 0.5), r2 = cscale(csub(k.a, disc), 0.5);
  const double2 uinf = (r1.x * r1.x + r1.y * r1.y >= r2.x * r2.x + r2.y * r2.y) ? r1 : r2;
  const double2 iinf = crecip(uinf);
  const double tol = sizeof(T) == 4 ? 7.450580596923828e-09 : 8.881784197001252e-16;  // 2^-27, 2^-50
  const double tol2 = tol * tol * (iinf.x * iinf.x + iinf.y * iinf.y);
  double2 c = make_double2(0, 0);
  int64_t last_bad = -1;
  double2 inv = make_double2(0, 0);
  for (int64_t ix = 0; ix < nx; ++ix) {
    const double2 aj = (ix == 0 || ix == nx - 1) ? k.ac : k.a;
    const double2 den = ix == 0 ? aj : csub(aj, cmul(k.b, c));
    inv = crecip(den);
    c = cmul(k.b, inv);
    tab[ix * ny * nz + i] = cvt<C>(inv);
    if (ix < nx - 1) {
      const double dx = inv.x - iinf.x, dy = inv.y - iinf.y;
      if (!(dx * dx + dy * dy <= tol2)) last_bad = ix;
    }
  }
  if (lend) {
    // chunk constants of a chunk of ch settled rows: q = -b / u_inf,
    // alpha = q^ch, beta = sum_k q^k q^(k+1) (the carries' coefficients)
    const double2 q = cmul(make_double2(-k.b.x, -k.b.y), iinf);
    double2 al = make_double2(1, 0), be = make_double2(0, 0);
    for (int j = 0; j < ch; ++j) {
      const double2 an = cmul(al, q);
      be = cadd(be, cmul(al, an));
      al = an;
    }
    lend[kLineVals * i] = cvt<C>(iinf);
    lend[kLineVals * i + 1] = cvt<C>(inv);
    lend[kLineVals * i + 2] = cvt<C>(k.b);
    lend[kLineVals * i + 3] = cvt<C>(al);
    lend[kLineVals * i + 4] = cvt<C>(be);
    lenL[i] = (int)(last_bad + 1);
  }
}

Plane3DArgs make_args(const Plan3D& p) {
  Plane3DArgs a;
  a.nx = p.n[0];
  a.ny = p.n[1];
  a.nz = p.n[2];
  a.hx = p.h[0];
  a.hy = p.h[1];
  a.hz = p.h[2];
  a.omega = p.omega;
  a.wx = p.wc[0];
  a.wy = p.wc[1];
  a.wz = p.wc[2];
  a.mden = p.mden;
  a.lamBo = p.axo->lamB;
  a.invmuo = p.axo->invmu;
  a.lamAo = p.axo->lamA;
  a.sigAo = p.axo->sigA;
  a.parAo = p.axo->parA;
  a.two = p.axo->tw;
  a.lamBi = p.axi->lamB;
  a.invmui = p.axi->invmu;
  a.lamAi = p.axi->lamA;
  a.sigAi = p.axi->sigA;
  a.parAi = p.axi->parA;
  a.twi = p.axi->tw;
  for (int k = 0; k < 2; ++k) {
    a.en_o[k] = p.axo->en[k];
    a.eninv_o[k] = p.axo->eninv[k];
    a.g_o[k] = p.axo->g[k];
    a.ginv_o[k] = p.axo->ginv[k];
    a.en_i[k] = p.axi->en[k];
    a.eninv_i[k] = p.axi->eninv[k];
    a.g_i[k] = p.axi->g[k];
    a.ginv_i[k] = p.axi->ginv[k];
  }
  return a;
}

// ---------------------------------------------------------------------------
// Tiled inner sweeps (a6).  The inner Steps 1-3 of Section 5.1.2 for outer
// mode l run as three launches (k_inner3d) with a per-plane reduction between
// them (k_inner_reduce), instead of one CTA per plane that streams its Thomas
// scratch through HBM.
//
// A CTA of k_inner3d owns kMW consecutive inner modes m of one outer mode l
// (the lines (x, l, m0..m0+kMW-1), x = 0..nx-1).  It stages their right-hand
// sides in shared memory ([x][kMW], read from HBM once), and solves each line
// by the chunked LU of Section 4.1.2's per-mode solves: thread (m, c) owns rows
// [c*ch, c*ch + ch) of line m.
//   pass 1: with the carries d_{s-1} = 0, x_{e+1} = 0 the chunk's forward
//     substitution d_j = (r_j - b d_{j-1}) / u_j gives d_loc at its last row
//     and, through the running products alpha_j = prod_{i<=j} (-b / u_i), the
//     backward substitution's value x_loc at its first row, plus the
//     rhs-independent alpha_e and beta = sum_j alpha_{j-1} alpha_j, so that
//       d_e = d_loc + alpha_e d_{s-1},
//       x_s = x_loc + beta d_{s-1} + alpha_e x_{e+1};
//   scan: these affine maps composed over the chunks of each line by one warp
//     (Kogge-Stone over lanes), forward for d and backward for x;
//   pass 2: the chunk's substitutions again from the exact carries; d and then
//     x overwrite the staged right-hand sides.
// The pivots 1/u_j come from the per-plan FP64 tables, read only for rows
// before the line's pivots settle (k_plane_tables); later rows use 1/u_inf and
// the corner row 1/u_{nx-1}.  Inner Steps 1 and 2 then form the CTA's share of
// the inner boundary rows (eqs. 2dBs1, step2-3 on the plane) from the solved
// tile, summing its inner modes in a fixed order, and accumulate them over the
// CTA's nmb tiles into one face partial per CTA; inner Step 3 writes the
// plane solution y3(x, l, m).
// ---------------------------------------------------------------------------
struct InnerArgs {
  Plane3DArgs a;
  int ch;      // rows per chunk
  int nc;      // chunks per line
  int nmb;     // tiles per CTA (inner modes kMW * nmb per CTA)
  int nparts;  // face partials per plane = gridDim.x
};

// Shared memory of k_inner3d: solved-row tile, pivot rows, chunk summaries
// (padded), face accumulators, per-line and per-mode constants, powers of the
// settled pivot ratio, the plane's inner C_bb faces (inner Steps 2 and 3),
// settling rows.  istep 0: the largest of the three steps.
inline size_t inner_smem_bytes(int64_t nx, int nc, int ch, size_t cb, int istep = 0) {
  return ((size_t)nx * kMW + (size_t)kPivRows * kMW + 4 * (size_t)kMW * (nc + 1) + 2 * (size_t)nx + 9 * kMW + 3 +
          (size_t)ch * kMW + (istep != 1 ? 2 * (size_t)nx : 0)) *
             cb +
         2 * kMW * sizeof(int);
}

// affine map x -> p x + q, composed as (p2, q2) o (p1, q1) = (p2 p1, p2 q1 + q2)
template <typename C>
__device__ __forceinline__ void affine_compose(C& p, C& q, C p1, C q1) {
  q = cadd(cmul(p, q1), q);
  p = cmul(p, p1);
}

template <typename C>
__device__ __forceinline__ C shfl_up_c(C v, int off) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, off);
  v.y = __shfl_up_sync(0xffffffffu, v.y, off);
  return v;
}

// Launch bound: 1024 threads (64 chunks of kMW lines) in complex64, 512 in
// complex128 (its wider registers).
template <typename T>
constexpr int inner_max_threads() {
  return sizeof(T) == 4 ? 1024 : 512;
}

// Chunks per line the tiled sweeps allow for (precision, rows per chunk); 0
// unless CH is one of the compiled 8, 16, 32.
inline int inner_max_chunks(int prec, int ch) {
  if (ch != 8 && ch != 16 && ch != 32) return 0;
  return (prec == kPrecF64 ? inner_max_threads<double>() : inner_max_threads<float>()) / kMW;
}

// Lanes per line in the chunk scan (a warp scans 32 / kScanLanes lines).
constexpr int kScanLanes = 8;

template <typename C>
__device__ __forceinline__ C shfl_up_w(C v, int off) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, off, kScanLanes);
  v.y = __shfl_up_sync(0xffffffffu, v.y, off, kScanLanes);
  return v;
}

template <typename C>
__device__ __forceinline__ C shfl_down_w(C v, int off) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, off, kScanLanes);
  v.y = __shfl_down_sync(0xffffffffu, v.y, off, kScanLanes);
  return v;
}

template <typename T, int OSTEP, int ISTEP, int CH>
__global__ void __launch_bounds__(inner_max_threads<T>()) k_inner3d(
    InnerArgs ia, const typename cpx<T>::type* __restrict__ fhat, const typename cpx<T>::type* __restrict__ gfaces,
    const typename cpx<T>::type* __restrict__ cin, const typename cpx<T>::type* __restrict__ tab,
    const typename cpx<T>::type* __restrict__ lend, const int* __restrict__ lenL,
    typename cpx<T>::type* __restrict__ part, typename cpx<T>::type* __restrict__ y3, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  constexpr bool kFhatRows = OSTEP != 2 && ISTEP != 2;  // the right-hand side reads f_hat
  if (skip && *skip) return;
  const Plane3DArgs& a = ia.a;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = (int)a.nx;
  const int64_t ny = a.ny, nz = a.nz;
  const int nc = ia.nc;
  const int ncp = nc + 1;  // padded chunk stride of the summaries: conflict-free in both layouts
  C* tile = reinterpret_cast<C*>(smem_raw);  // [nx][kMW]
  C* piv = tile + (size_t)nx * kMW;          // [kPivRows][kMW] first rows of the pivot tables
  C* sums = piv + kPivRows * kMW;            // [4][kMW][ncp]: d_loc, x_loc, alpha, beta; then the carries
  C* facc = sums + 4 * kMW * ncp;            // [2][nx] face accumulators (inner Steps 1, 2)
  C* mw = facc + 2 * nx;                     // [kMW] rhs scale, [kMW] weight of the last face, [2][kMW] face weights
  // [kMW] b, [kMW] 1/u_inf, [kMW] 1/u_{nx-1}; [3] outer-mode constants; [kMW] alpha, [kMW] beta of a settled chunk
  C* lc = mw + 4 * kMW;
  C* apow = lc + 5 * kMW + 3;  // [CH][kMW] q^(k+1), q = -b / u_inf
  C* scin = apow + CH * kMW;   // [2][nx] inner C_bb faces of this plane (inner Steps 2, 3)
  int* sL = reinterpret_cast<int*>(scin + (ISTEP != 1 ? 2 * nx : 0));  // [kMW] settling rows
  int* sR = sL + kMW;                                 // [kMW] 1: routed to FP64
  const int64_t l = blockIdx.y;
  const int tid = threadIdx.x, nthr = blockDim.x;
  // thread (mi, c): the two half-warps of warp w take chunks w and nc-1-w, so
  // that the first and the last chunk of a line (never settled: the first
  // rows and the corner row) share a warp; with nc odd the middle warp's
  // second half idles
  const int mi = tid & (kMW - 1), wk = tid / (2 * kMW), half = (tid / kMW) & 1;
  const int c = half ? nc - 1 - wk : wk;
  const bool cok = half ? (nc - 1 - wk > wk) : (wk < nc);
  const int64_t xs = ny * nz;
  if (tid == 0) {
    // outer-mode constants: 1/mu_l (outer B modes), e^{+i theta_l} e^{-t(ny-1)}, parity (outer A modes)
    lc[3 * kMW] = OSTEP == 2 ? mk<C>(1, 0) : mk<C>(a.invmuo[2 * l], a.invmuo[2 * l + 1]);
    lc[3 * kMW + 1] = cmul(mk<C>(a.two[2 * l], -a.two[2 * l + 1]), mk<C>(a.eninv_o[0], a.eninv_o[1]));
    lc[3 * kMW + 2] = mk<C>(a.parAo[l], 0);
  }
  // the plane's inner C_bb faces into shared memory (they land with the
  // first tile's copies)
  if (ISTEP != 1)
    for (int e = tid; e < 2 * nx; e += nthr) cp_async<sizeof(C)>(scin + e, cin + l * 2 * nx + e);
  const C* cin1 = scin;
  const C* cinn = scin + nx;
  if (ISTEP != 3)
    for (int e = tid; e < 2 * nx; e += nthr) facc[e] = mk<C>(0, 0);
  // the right-hand sides of this CTA's later tiles into L2 while the first
  // is staged and solved: one 128-byte line (16 inner modes) per row,
  // prefetched by lane 0 of each half-warp for its chunk's rows
  if (ISTEP != 2 && mi == 0 && cok)
    for (int mb = 1; mb < ia.nmb; ++mb) {
      const int64_t mq = ((int64_t)blockIdx.x * ia.nmb + mb) * kMW;
      if (mq >= nz) break;
      for (int k = 0; k < CH && c * CH + k < nx; ++k) {
        const int64_t x = c * CH + k;
        if (OSTEP != 2) l2_prefetch(fhat + (x * ny + l) * nz + mq);
        if (OSTEP != 1) {
          l2_prefetch(gfaces + x * nz + mq);
          l2_prefetch(gfaces + ((int64_t)nx + x) * nz + mq);
        }
      }
    }

  for (int mb = 0; mb < ia.nmb; ++mb) {
    const int64_t m0 = ((int64_t)blockIdx.x * ia.nmb + mb) * kMW;
    if (m0 >= nz) break;
    __syncthreads();  // the previous tile's face sums are done
    // ---- asynchronous copies of the tile's f_hat rows (thread (mi, c): its
    // own chunk rows; the 16 lanes of a half-warp read 16 consecutive inner
    // modes of a row) and of the first pivot rows, all in flight while the
    // line constants are formed; no registers hold them ----
    {
      const int64_t m = m0 + mi;
      const int s0 = c * CH, e0 = min(s0 + CH, nx) - 1;
      if (kFhatRows && cok && m < nz) {
        const C* fp = fhat + ((int64_t)s0 * ny + l) * nz + m;
#pragma unroll
        for (int k = 0; k < CH; ++k)
          if (s0 + k <= e0) cp_async<sizeof(C)>(tile + (s0 + k) * kMW + mi, fp + k * xs);
      }
      // rows below the settling row are read from here, the others never
      for (int e = tid; e < kPivRows * kMW; e += nthr) {
        const int j = e / kMW, mm = e - j * kMW;
        if (j < nx && m0 + mm < nz) cp_async<sizeof(C)>(piv + e, tab + (int64_t)j * xs + l * nz + m0 + mm);
      }
    }
    if (tid < kMW) {
      const int64_t m = m0 + tid;
      const bool on = m < nz;
      const int64_t mc = on ? m : 0;
      // right-hand side of inner Step 1 / 3: (G + [C_bb terms]) / mu_m; Step 2: c_1 + par_m c_n
      mw[tid] = on ? (ISTEP == 2 ? mk<C>(1, 0) : mk<C>(a.invmui[2 * mc], a.invmui[2 * mc + 1])) : mk<C>(0, 0);
      mw[kMW + tid] = ISTEP == 2 ? mk<C>(a.parAi[mc], 0)
                                 : cmul(mk<C>(a.twi[2 * mc], -a.twi[2 * mc + 1]), mk<C>(a.eninv_i[0], a.eninv_i[1]));
      // face weights of the inner boundary rows: Step 1 (1, e^{-i theta_m}), Step 2 (sigma_m, par_m sigma_m)
      C w1 = mk<C>(1, 0), wn = mk<C>(a.twi[2 * mc], a.twi[2 * mc + 1]);
      if (ISTEP == 2) {
        w1 = mk<C>(a.sigAi[2 * mc], a.sigAi[2 * mc + 1]);
        wn = cscale(w1, (T)a.parAi[mc]);
      }
      mw[2 * kMW + tid] = on ? w1 : mk<C>(0, 0);
      mw[3 * kMW + tid] = on ? wn : mk<C>(0, 0);
      // line constants from the plan tables
      const int64_t line = l * nz + mc;
      const C b = lend[kLineVals * line + 2], iinf = lend[kLineVals * line];
      lc[tid] = b;
      lc[kMW + tid] = iinf;
      lc[2 * kMW + tid] = lend[kLineVals * line + 1];
      lc[3 * kMW + 3 + tid] = lend[kLineVals * line + 3];
      lc[4 * kMW + 3 + tid] = lend[kLineVals * line + 4];
      // powers of q = -b / u_inf: the forward carry's weight in a settled chunk
      const C q = cmul(mk<C>(-b.x, -b.y), iinf);
      C qk = q;
      for (int k = 0; k < CH; ++k) {
        apow[k * kMW + tid] = qk;
        qk = cmul(qk, q);
      }
      // a line routed to FP64 (flag bit) gets a zero right-hand side here, so
      // it adds nothing to the faces; the FP64 kernel solves it
      const int lr = on ? lenL[line] : 0;
      const bool routed = (lr & kRoutedFlag) != 0;
      sL[tid] = routed ? 0 : lr;
      if (routed) {
        mw[tid] = mk<C>(0, 0);
        mw[kMW + tid] = mk<C>(0, 0);
        mw[2 * kMW + tid] = mk<C>(0, 0);
        mw[3 * kMW + tid] = mk<C>(0, 0);
      }
      sR[tid] = routed ? 1 : 0;
    }
    cp_async_wait_all();
    __syncthreads();  // line constants formed, every thread's copies landed
    // ---- thread (mi, c) forms the right-hand sides of its own chunk rows in
    // place (from the copied f_hat rows, the outer faces, the inner C_bb
    // faces) ----
    const int64_t m = m0 + mi;
    const bool act = m < nz && cok;
    const int s0 = c * CH, e0 = min(s0 + CH, nx) - 1;
    C* trow = tile + s0 * kMW + mi;  // row s0 + k of this line: trow[k * kMW]
    if (cok) {
      const C gscale = lc[3 * kMW], wl = lc[3 * kMW + 1];
      const T paro = lc[3 * kMW + 2].x;
      const C sc = mw[mi], wk2 = mw[kMW + mi];
      const C gs = cmul(gscale, sc);
      const bool zero_rhs = !act || (ISTEP == 2 && sR[mi]);
      const int64_t mcl = act ? m : 0;
      const C* g1p = OSTEP != 1 ? gfaces + (int64_t)s0 * nz + mcl : nullptr;  // outer faces (Steps 2, 3)
      const C* gnp = OSTEP != 1 ? g1p + (int64_t)nx * nz : nullptr;
#pragma unroll(CH <= 16 ? CH : 8)
      for (int k = 0; k < CH; ++k) {
        if (s0 + k <= e0) {
          C v = mk<C>(0, 0);
          if (!zero_rhs) {
            if (ISTEP == 2) {
              v = cadd(cin1[s0 + k], cmul(cinn[s0 + k], wk2));
            } else {
              if (OSTEP == 1) v = cmul(trow[k * kMW], gs);
              else if (OSTEP == 2) v = cmul(cadd(g1p[k * nz], cscale(gnp[k * nz], paro)), sc);
              else v = cmul(cadd(cadd(trow[k * kMW], g1p[k * nz]), cmul(gnp[k * nz], wl)), gs);
              if (ISTEP == 3) v = cadd(v, cmul(cadd(cin1[s0 + k], cmul(cinn[s0 + k], wk2)), sc));
            }
          }
          trow[k * kMW] = v;
        }
      }
    }
    // ---- line constants of thread (mi, c) ----
    const C b = lc[mi], iinf = lc[kMW + mi], ilast = lc[2 * kMW + mi];
    const C nb = mk<C>(-b.x, -b.y);
    const C cinf = cmul(b, iinf);
    const int L = sL[mi];  // 0 for a routed line
    const C* tcol = tab + l * nz + (m < nz ? m : 0);
    // The rows of a chunk that is not settled, in three runs: rows [s0, jt)
    // below the settling row take 1/u_j from the pivot table (four loads in
    // flight at a time), rows [jt, jc) take 1/u_inf, and the corner row nx - 1
    // (if the chunk holds it) 1/u_{nx-1}.  fn(j, 1/u_j, g_j) with
    // g_j = -b / u_j, the weight of the previous row's value in
    // d_j = r_j / u_j + g_j d_{j-1} and of the next row's in x_j = d_j + g_j x_{j+1}.
    const int jt = min(e0 + 1, max(s0, L));
    const int jc = e0 == nx - 1 ? e0 : e0 + 1;
    const C q = cmul(nb, iinf), glast = cmul(nb, ilast);
    auto tpiv = [&](int j) -> C { return j < kPivRows ? piv[j * kMW + mi] : tcol[(int64_t)j * xs]; };
    auto rows_up = [&](auto&& fn) {
#pragma unroll 1
      for (int j0 = s0; j0 < jt; j0 += 4) {
        C pv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) pv[k] = j0 + k < jt ? tpiv(j0 + k) : iinf;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (j0 + k < jt) fn(j0 + k, pv[k], cmul(nb, pv[k]));
      }
#pragma unroll 4
      for (int j = jt; j < jc; ++j) fn(j, iinf, q);
      if (jc == e0) fn(e0, ilast, glast);
    };
    auto rows_down = [&](auto&& fn) {
      if (jc == e0) fn(e0, ilast, glast);
#pragma unroll 4
      for (int j = jc - 1; j >= jt; --j) fn(j, iinf, q);
#pragma unroll 1
      for (int j0 = jt - 1; j0 >= s0; j0 -= 4) {
        C pv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) pv[k] = j0 - k >= s0 ? tpiv(j0 - k) : iinf;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (j0 - k >= s0) fn(j0 - k, pv[k], cmul(nb, pv[k]));
      }
    };
    // ---- pass 1 ----
    // Forward with d_{s-1} = 0 (d_loc written over the rhs), then the
    // backward substitution with x_{e+1} = 0 over it by Horner's rule gives
    // x_loc.  alpha_e = prod (-b/u_j) and beta = sum alpha_{j-1} alpha_j do
    // not depend on the data: a settled chunk takes them from the plan, the
    // others form them.  Warp-uniform: a warp takes the settled path only if
    // all its chunks are settled (the general path is exact for them too).
    const bool settled = __all_sync(0xffffffffu, !act || (s0 >= L && e0 < nx - 1 && e0 - s0 + 1 == CH));
    if (act) {
      C d = mk<C>(0, 0), al = mk<C>(1, 0), be = mk<C>(0, 0), x = mk<C>(0, 0);
      if (settled) {
        // d_j = r_j / u_inf + q d_{j-1}, q = -b / u_inf
#pragma unroll 16
        for (int k = 0; k < CH; ++k) {
          d = cfma(q, d, cmul(trow[k * kMW], iinf));
          trow[k * kMW] = d;
        }
#pragma unroll 16
        for (int k = CH - 1; k >= 0; --k) x = cfms(trow[k * kMW], cinf, x);
        al = lc[3 * kMW + 3 + mi];
        be = lc[4 * kMW + 3 + mi];
      } else {
        rows_up([&](int j, C inv, C g) {
          d = cfma(g, d, cmul(tile[j * kMW + mi], inv));
          tile[j * kMW + mi] = d;
          const C an = cmul(al, g);
          be = cfma(al, an, be);
          al = an;
        });
        rows_down([&](int j, C, C g) { x = cfma(g, x, tile[j * kMW + mi]); });
      }
      sums[(0 * kMW + mi) * ncp + c] = d;
      sums[(1 * kMW + mi) * ncp + c] = x;
      sums[(2 * kMW + mi) * ncp + c] = al;
      sums[(3 * kMW + mi) * ncp + c] = be;
    }
    __syncthreads();
    // ---- scan over the chunks of each line: kScanLanes lanes per line, each
    // lane a group of consecutive chunks, the groups composed by shuffles ----
    {
      const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
      const int sl = lane & (kScanLanes - 1), seg = lane / kScanLanes;
      constexpr int lpw = 32 / kScanLanes;             // lines per warp
      const int g = (nc + kScanLanes - 1) / kScanLanes;  // chunks per lane
      for (int mm0 = warp * lpw; mm0 < kMW; mm0 += nw * lpw) {
        const int mm = mm0 + seg;
        C* sd = sums + (0 * kMW + mm) * ncp;  // d_loc, then the carry-in d_{s-1}
        C* sx = sums + (1 * kMW + mm) * ncp;  // x_loc, then the carry-in x_{e+1}
        const C* sa = sums + (2 * kMW + mm) * ncp;
        const C* sb = sums + (3 * kMW + mm) * ncp;
        const int c0 = sl * g, c1 = min(c0 + g, nc);
        // forward: D_c = dloc_c + alpha_c D_{c-1}; the lane's group as one map
        C P = mk<C>(1, 0), Q = mk<C>(0, 0);
        for (int cc = c0; cc < c1; ++cc) {
          Q = cadd(cmul(sa[cc], Q), sd[cc]);
          P = cmul(sa[cc], P);
        }
        for (int off = 1; off < kScanLanes; off <<= 1) {
          const C Pu = shfl_up_w(P, off), Qu = shfl_up_w(Q, off);
          if (sl >= off) affine_compose(P, Q, Pu, Qu);
        }
        C Din = shfl_up_w(Q, 1);  // D before the lane's group (inclusive scan shifted)
        if (sl == 0) Din = mk<C>(0, 0);
        // carry-in d_{s-1} of each chunk; keep E_c = xloc_c + beta_c D_{c-1}
        for (int cc = c0; cc < c1; ++cc) {
          const C dl = sd[cc];
          sx[cc] = cadd(sx[cc], cmul(sb[cc], Din));
          sd[cc] = Din;
          Din = cadd(dl, cmul(sa[cc], Din));
        }
        // backward: X_c = E_c + alpha_c X_{c+1}; the lane's group as one map of X after the group
        P = mk<C>(1, 0);
        Q = mk<C>(0, 0);
        for (int cc = c1 - 1; cc >= c0; --cc) {
          Q = cadd(cmul(sa[cc], Q), sx[cc]);
          P = cmul(sa[cc], P);
        }
        for (int off = 1; off < kScanLanes; off <<= 1) {
          const C Pd = shfl_down_w(P, off), Qd = shfl_down_w(Q, off);
          if (sl + off < kScanLanes) affine_compose(P, Q, Pd, Qd);
        }
        C Xin = shfl_down_w(Q, 1);  // X just after the lane's group
        if (sl == kScanLanes - 1) Xin = mk<C>(0, 0);
        for (int cc = c1 - 1; cc >= c0; --cc) {
          const C E = sx[cc];
          sx[cc] = Xin;  // carry-in x_{e+1} of chunk cc
          Xin = cadd(E, cmul(sa[cc], Xin));
        }
      }
    }
    __syncthreads();
    // ---- pass 2 ----
    // d_j = d_loc_j + alpha_j d_{s-1} over the chunk, then the backward
    // substitution from the exact carry x_{e+1}; in a settled chunk
    // alpha_j = q^(j-s+1) and both run in one backward sweep.
    if (act) {
      const C Din = sums[(0 * kMW + mi) * ncp + c];
      C x = sums[(1 * kMW + mi) * ncp + c];
      C* yrow = y3 + ((int64_t)s0 * ny + l) * nz + m;  // y3 rows of this line (Step 3)
      if (settled) {
#pragma unroll 16
        for (int k = CH - 1; k >= 0; --k) {
          x = cfms(cfma(apow[k * kMW + mi], Din, trow[k * kMW]), cinf, x);
          if (ISTEP == 3) yrow[k * xs] = x;
          else trow[k * kMW] = x;
        }
      } else {
        C al = mk<C>(1, 0);
        rows_up([&](int j, C, C g) {
          al = cmul(al, g);
          tile[j * kMW + mi] = cfma(al, Din, tile[j * kMW + mi]);
        });
        rows_down([&](int j, C, C g) {
          x = cfma(g, x, tile[j * kMW + mi]);
          if (ISTEP == 3) yrow[(int64_t)(j - s0) * xs] = x;
          else tile[j * kMW + mi] = x;
        });
      }
    }
    if (ISTEP != 3) {
      __syncthreads();
      // this tile's share of the inner boundary rows, inner modes summed in a
      // fixed (row-rotated, bank-conflict-free) order
      for (int x = tid; x < nx; x += nthr) {
        C s1 = mk<C>(0, 0), sn = mk<C>(0, 0);
#pragma unroll
        for (int k = 0; k < kMW; ++k) {
          const int mm = (k + x) & (kMW - 1);
          const C v = tile[x * kMW + mm];
          // Step 1's first-row weight is 1 (modes off the grid or routed
          // hold zeros in the tile)
          s1 = ISTEP == 1 ? cadd(s1, v) : cfma(v, mw[2 * kMW + mm], s1);
          sn = cfma(v, mw[3 * kMW + mm], sn);
        }
        facc[x] = cadd(facc[x], s1);
        facc[nx + x] = cadd(facc[nx + x], sn);
      }
    }
  }
  if (ISTEP != 3) {
    __syncthreads();
    C* out = part + ((int64_t)l * ia.nparts + blockIdx.x) * 2 * nx;
    for (int e = tid; e < 2 * nx; e += nthr) out[e] = facc[e];
  }
}

// Precision routing (a9): the inner lines whose line matrix is close to
// singular, solved with FP64 arithmetic from the same (complex64) inputs.  One
// warp per routed line: lane c owns rows [c*chr, (c+1)*chr) and the chunked LU
// of k_inner3d runs in FP64 (pass 1, warp scan of the affine carries, pass 2
// through a per-line FP64 scratch), with FP64 reciprocal pivots from the
// plan.  Inner Steps 1, 2 write the line's weighted boundary-row
// contributions to rpart[route] (added per plane by k_inner_reduce); inner
// Step 3 writes y3 over the zero the tile kernel left for the line.
template <typename T, int OSTEP, int ISTEP>
__global__ void __launch_bounds__(128) k_inner3d_r(InnerArgs ia, const typename cpx<T>::type* __restrict__ fhat,
                                                   const typename cpx<T>::type* __restrict__ gfaces,
                                                   const typename cpx<T>::type* __restrict__ cin,
                                                   const int* __restrict__ rlist, const double2* __restrict__ rtab,
                                                   int nroute, typename cpx<T>::type* __restrict__ rpart,
                                                   double2* __restrict__ rtmp, typename cpx<T>::type* __restrict__ y3,
                                                   const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const Plane3DArgs& a = ia.a;
  const int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (q >= nroute) return;  // warp-uniform
  const int lane = threadIdx.x & 31;
  const int nx = (int)a.nx;
  const int64_t ny = a.ny, nz = a.nz;
  const int64_t line = rlist[q], l = line / nz, m = line - l * nz;
  const double w2 = a.omega * a.omega;
  const double* lo = OSTEP == 2 ? a.lamAo : a.lamBo;
  const double* li = ISTEP == 2 ? a.lamAi : a.lamBi;
  const double sre = lo[2 * l] + li[2 * m] - w2, sim = lo[2 * l + 1] + li[2 * m + 1];
  const double mo = mass_coef(a.hx, a.mden).off;
  const double2 b = make_double2(sre * mo - 1.0 / a.hx, sim * mo);
  const double2 nb = make_double2(-b.x, -b.y);
  // rhs factors of the line, as in k_inner3d, in FP64
  const double2 gscale = OSTEP == 2 ? make_double2(1, 0) : make_double2(a.invmuo[2 * l], a.invmuo[2 * l + 1]);
  const double paro = a.parAo[l];
  const double2 wl = cmul(make_double2(a.two[2 * l], -a.two[2 * l + 1]), make_double2(a.eninv_o[0], a.eninv_o[1]));
  const double2 imu = make_double2(a.invmui[2 * m], a.invmui[2 * m + 1]);
  const double2 wm = cmul(make_double2(a.twi[2 * m], -a.twi[2 * m + 1]), make_double2(a.eninv_i[0], a.eninv_i[1]));
  const double pari = a.parAi[m];
  const C* cin1 = cin ? cin + l * 2 * nx : nullptr;
  const C* cinn = cin ? cin1 + nx : nullptr;
  const C* g1 = gfaces;
  const C* gn = gfaces ? gfaces + (int64_t)nx * nz : nullptr;
  auto rhs = [&](int j) -> double2 {
    if (ISTEP == 2) return cadd(cvt<double2>(cin1[j]), cscale(cvt<double2>(cinn[j]), pari));
    double2 g;
    if (OSTEP == 1) g = cmul(cvt<double2>(fhat[((int64_t)j * ny + l) * nz + m]), gscale);
    else if (OSTEP == 2) g = cadd(cvt<double2>(g1[(int64_t)j * nz + m]), cscale(cvt<double2>(gn[(int64_t)j * nz + m]), paro));
    else
      g = cmul(cadd(cadd(cvt<double2>(fhat[((int64_t)j * ny + l) * nz + m]), cvt<double2>(g1[(int64_t)j * nz + m])),
                    cmul(cvt<double2>(gn[(int64_t)j * nz + m]), wl)),
               gscale);
    if (ISTEP == 3) g = cadd(g, cadd(cvt<double2>(cin1[j]), cmul(cvt<double2>(cinn[j]), wm)));
    return cmul(g, imu);
  };
  const double2* piv = rtab + (int64_t)q * nx;
  double2* dtmp = rtmp + (int64_t)q * nx;
  const int chr = (nx + 31) / 32;
  const int s0 = lane * chr, e0 = min(s0 + chr, nx) - 1;
  // pass 1
  double2 d = make_double2(0, 0), al = make_double2(1, 0), xl = make_double2(0, 0), be = make_double2(0, 0);
  for (int j = s0; j <= e0; ++j) {
    const double2 inv = piv[j];
    d = cmul(csub(rhs(j), cmul(b, d)), inv);
    xl = cadd(xl, cmul(al, d));
    const double2 an = cmul(al, cmul(nb, inv));
    be = cadd(be, cmul(al, an));
    al = an;
  }
  if (s0 > e0) {  // a lane without rows: identity maps
    d = make_double2(0, 0);
    al = make_double2(1, 0);
  }
  // forward carries D (inclusive scan of x -> al x + d), then E = xl + be D_in
  double2 P = al, Q = d;
  for (int off = 1; off < 32; off <<= 1) {
    const double2 Pu = shfl_up_c(P, off), Qu = shfl_up_c(Q, off);
    if (lane >= off) affine_compose(P, Q, Pu, Qu);
  }
  double2 Din = shfl_up_c(Q, 1);
  if (lane == 0) Din = make_double2(0, 0);
  const double2 E = cadd(xl, cmul(be, Din));
  // backward carries: X_c = E_c + al_c X_{c+1}
  P = al;
  Q = s0 > e0 ? make_double2(0, 0) : E;
  for (int off = 1; off < 32; off <<= 1) {
    const double2 Pd = shfl_down(P, off), Qd = shfl_down(Q, off);
    if (lane + off < 32) affine_compose(P, Q, Pd, Qd);
  }
  double2 Xin = shfl_down(Q, 1);
  if (lane == 31) Xin = make_double2(0, 0);
  // pass 2
  d = Din;
  for (int j = s0; j <= e0; ++j) {
    d = cmul(csub(rhs(j), cmul(b, d)), piv[j]);
    dtmp[j] = d;
  }
  double2 x = Xin;
  double2 w1 = make_double2(1, 0), wn = make_double2(a.twi[2 * m], a.twi[2 * m + 1]);
  if (ISTEP == 2) {
    w1 = make_double2(a.sigAi[2 * m], a.sigAi[2 * m + 1]);
    wn = cscale(w1, pari);
  }
  C* rp = ISTEP == 3 ? nullptr : rpart + (int64_t)q * 2 * nx;
  for (int j = e0; j >= s0; --j) {
    x = csub(dtmp[j], cmul(cmul(b, piv[j]), x));
    if (ISTEP == 3) {
      y3[((int64_t)j * ny + l) * nz + m] = cvt<C>(x);
    } else {
      rp[j] = cvt<C>(cmul(x, w1));
      rp[nx + j] = cvt<C>(cmul(x, wn));
    }
  }
}

// FP64 reciprocal pivots of the routed lines (the recurrence of
// k_plane_tables), and the routed flag in the settling-row table.
__global__ void k_route_tables(double2* __restrict__ rtab, int* __restrict__ lenL, const int* __restrict__ rlist,
                               int nroute, Plane3DArgs a, int outerA, int innerA) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nroute) return;
  const int64_t nx = a.nx, nz = a.nz;
  const int64_t line = rlist[q], l = line / nz, m = line - l * nz;
  const double* lo = outerA ? a.lamAo : a.lamBo;
  const double* li = innerA ? a.lamAi : a.lamBi;
  const double w2 = a.omega * a.omega;
  const LineCoef<double2> k = line_coef<double2>(lo[2 * l] + li[2 * m] - w2, lo[2 * l + 1] + li[2 * m + 1], a.hx, a.wx, a.mden);
  double2 c = make_double2(0, 0);
  for (int64_t ix = 0; ix < nx; ++ix) {
    const double2 aj = (ix == 0 || ix == nx - 1) ? k.ac : k.a;
    const double2 den = ix == 0 ? aj : csub(aj, cmul(k.b, c));
    const double2 inv = crecip(den);
    c = cmul(k.b, inv);
    rtab[(int64_t)q * nx + ix] = inv;
  }
  lenL[line] |= kRoutedFlag;
}

// Per outer mode l: the inner boundary rows from the CTAs' partials (fixed
// order), scaled as in eq. 2dBs1 (Step 1: 1/nz and e^{t(nz-1)}/nz) or eq.
// step2-3 (Step 2: 1), kept in vw[l] (v_in after Step 1, w_in after Step 2),
// and the inner C_bb of eq. Cbb applied (Step 1: to v_in; Step 2: to
// v_in + w_in) for the next inner Step's right-hand side.
template <typename T, int OSTEP, int ISTEP>
__global__ void __launch_bounds__(256) k_inner_reduce(InnerArgs ia, const typename cpx<T>::type* __restrict__ part,
                                                      typename cpx<T>::type* __restrict__ vw,
                                                      typename cpx<T>::type* __restrict__ cin,
                                                      const int* __restrict__ roff,
                                                      const typename cpx<T>::type* __restrict__ rpart,
                                                      const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  constexpr bool kFhatRows = OSTEP != 2 && ISTEP != 2;  // the right-hand side reads f_hat
  if (skip && *skip) return;
  const Plane3DArgs& a = ia.a;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = (int)a.nx;
  const int64_t l = blockIdx.x;
  C* sv = reinterpret_cast<C*>(smem_raw);  // [2][nx] v_in
  C* sw = sv + 2 * nx;                     // [2][nx] w_in
  C* vwl = vw + l * 4 * nx;                // [v_in 2 nx][w_in 2 nx]
  const C* pp = part + l * (int64_t)ia.nparts * 2 * nx;
  const C sc1 = ISTEP == 1 ? mk<C>(1.0 / (double)a.nz, 0) : mk<C>(1, 0);
  const C scn = ISTEP == 1 ? mk<C>(a.en_i[0] / (double)a.nz, a.en_i[1] / (double)a.nz) : mk<C>(1, 0);
  for (int e = threadIdx.x; e < 2 * nx; e += blockDim.x) {
    C acc = mk<C>(0, 0);
    for (int q = 0; q < ia.nparts; ++q) acc = cadd(acc, pp[(int64_t)q * 2 * nx + e]);
    if (roff)  // lines of this plane solved in FP64, in route order
      for (int q = roff[l]; q < roff[l + 1]; ++q) acc = cadd(acc, rpart[(int64_t)q * 2 * nx + e]);
    acc = cmul(acc, e < nx ? sc1 : scn);
    if (ISTEP == 1) {
      sv[e] = acc;
      vwl[e] = acc;
    } else {
      sv[e] = vwl[e];
      sw[e] = acc;
      vwl[2 * nx + e] = acc;
    }
  }
  __syncthreads();
  const double lo_re = OSTEP == 2 ? a.lamAo[2 * l] : a.lamBo[2 * l];
  const double lo_im = OSTEP == 2 ? a.lamAo[2 * l + 1] : a.lamBo[2 * l + 1];
  const double pre = a.omega * a.omega - lo_re, pim = -lo_im;
  plane_cbb(sv, ISTEP == 2 ? (const C*)sw : (const C*)nullptr, cin + l * 2 * nx, nx, a.hx, a.hz, a.wx, a.wz, pre, pim,
            mk<C>(a.g_i[0], a.g_i[1]), mk<C>(a.ginv_i[0], a.ginv_i[1]), a.mden);
}

template <typename T>
cudaError_t launch_plane(int ostep, const Plan3D& p, const void* gfaces, const int* skip, cudaStream_t st) {
  using C = typename cpx<T>::type;
  const int bs = (int)((p.n[2] + 31) / 32 * 32);
  const int nw = bs / 32;
  const size_t smem = (size_t)(6 * p.n[0] + nw * 2 * XC) * sizeof(C);
  Plane3DArgs a = make_args(p);
  // tables of this outer mode type: [outer A][inner A]
  const int oA = ostep == 2 ? 1 : 0;
  const C* tB = (const C*)p.tab[2 * oA + 0];
  const C* tA = (const C*)p.tab[2 * oA + 1];
  auto run = [&](auto kern) {
    allow_dynamic_smem((const void*)kern, smem);
    kern<<<(unsigned)p.n[1], bs, smem, st>>>((const C*)p.fhat, (C*)p.cbuf, (C*)p.dbuf, (const C*)gfaces, tB, tA, a,
                                             skip);
  };
  const bool tab = tB && tA;
  if (ostep == 1) tab ? run(k_plane3d<T, 1, true>) : run(k_plane3d<T, 1, false>);
  else if (ostep == 2) tab ? run(k_plane3d<T, 2, true>) : run(k_plane3d<T, 2, false>);
  else tab ? run(k_plane3d<T, 3, true>) : run(k_plane3d<T, 3, false>);
  return cudaGetLastError();
}

// Inner Steps 1-3 of every outer mode by the tiled sweeps: three k_inner3d
// launches with the per-plane reductions between them; y3 goes to p.dbuf.
template <typename T, int OSTEP>
cudaError_t launch_inner_t(const Plan3D& p, const void* gfaces, const int* skip, cudaStream_t st, Profiler* prof) {
  using C = typename cpx<T>::type;
  InnerArgs ia{make_args(p), p.inner_ch, p.inner_nc, p.inner_nmb, p.inner_nparts};
  const int nx = (int)p.n[0];
  const int nthr = kMW * ((p.inner_nc + 1) & ~1);
  const dim3 grid((unsigned)p.inner_nparts, (unsigned)p.n[1]);
  const int oA = OSTEP == 2 ? 1 : 0;
  const C* fh = (const C*)p.fhat;
  const C* gf = (const C*)gfaces;
  C* part = (C*)p.ipart;
  C* vw = (C*)p.ivw;
  C* cin = (C*)p.icin;
  const size_t rsm = 4 * (size_t)nx * sizeof(C);
  static const char* const names[3][3] = {{"inner_o1_i1", "inner_o1_i2", "inner_o1_i3"},
                                          {"inner_o2_i1", "inner_o2_i2", "inner_o2_i3"},
                                          {"inner_o3_i1", "inner_o3_i2", "inner_o3_i3"}};
  cudaError_t e;
  auto sweep = [&](auto kern, int istep, int innerA) -> cudaError_t {
    const int t = 2 * oA + innerA;
    ProfScope ps(prof, names[OSTEP - 1][istep - 1], st);
    const size_t smem = inner_smem_bytes(nx, p.inner_nc, p.inner_ch, sizeof(C), istep);
    allow_dynamic_smem((const void*)kern, smem);
    kern<<<grid, nthr, smem, st>>>(ia, fh, gf, cin, (const C*)p.tab[t], (const C*)p.lend[t], p.lenL[t], part,
                                   (C*)p.dbuf, skip);
    return cudaGetLastError();
  };
  auto routed = [&](auto kern, int innerA) -> cudaError_t {
    const int t = 2 * oA + innerA;
    if (!p.nroute[t]) return cudaSuccess;
    ProfScope ps(prof, "inner_fp64_lines", st);
    kern<<<(unsigned)((p.nroute[t] + 3) / 4), 128, 0, st>>>(ia, fh, gf, cin, p.rlist[t], (const double2*)p.rtab[t],
                                                          p.nroute[t], (C*)p.rpart, (double2*)p.rtmp, (C*)p.dbuf,
                                                          skip);
    return cudaGetLastError();
  };
  auto reduce = [&](auto kern, int innerA) -> cudaError_t {
    const int t = 2 * oA + innerA;
    ProfScope ps(prof, "inner_reduce", st);
    allow_dynamic_smem((const void*)kern, rsm);
    kern<<<(unsigned)p.n[1], 256, rsm, st>>>(ia, part, vw, cin, p.nroute[t] ? p.roff[t] : nullptr, (const C*)p.rpart,
                                             skip);
    return cudaGetLastError();
  };
  // the sweep kernel of inner step ISTEP for the plan's rows per chunk
  auto sweep_ch = [&](auto istep, int innerA) -> cudaError_t {
    constexpr int IS = decltype(istep)::value;
    switch (p.inner_ch) {
      case 8: return sweep(k_inner3d<T, OSTEP, IS, 8>, IS, innerA);
      case 16: return sweep(k_inner3d<T, OSTEP, IS, 16>, IS, innerA);
      case 32: return sweep(k_inner3d<T, OSTEP, IS, 32>, IS, innerA);
      default: return cudaErrorInvalidValue;
    }
  };
  if ((e = sweep_ch(std::integral_constant<int, 1>{}, 0)) != cudaSuccess) return e;
  if ((e = routed(k_inner3d_r<T, OSTEP, 1>, 0)) != cudaSuccess) return e;
  if ((e = reduce(k_inner_reduce<T, OSTEP, 1>, 0)) != cudaSuccess) return e;
  if ((e = sweep_ch(std::integral_constant<int, 2>{}, 1)) != cudaSuccess) return e;
  if ((e = routed(k_inner3d_r<T, OSTEP, 2>, 1)) != cudaSuccess) return e;
  if ((e = reduce(k_inner_reduce<T, OSTEP, 2>, 1)) != cudaSuccess) return e;
  if ((e = sweep_ch(std::integral_constant<int, 3>{}, 0)) != cudaSuccess) return e;
  return routed(k_inner3d_r<T, OSTEP, 3>, 0);
}

template <typename T>
cudaError_t launch_inner(int ostep, const Plan3D& p, const void* gfaces, const int* skip, cudaStream_t st,
                         Profiler* prof) {
  if (ostep == 1) return launch_inner_t<T, 1>(p, gfaces, skip, st, prof);
  if (ostep == 2) return launch_inner_t<T, 2>(p, gfaces, skip, st, prof);
  return launch_inner_t<T, 3>(p, gfaces, skip, st, prof);
}

template <typename T>
cudaError_t launch_reduce_outer(int ostep, const Plan3D& p, void* out, const int* skip, cudaStream_t st) {
  using C = typename cpx<T>::type;
  const int bs = 256;
  const unsigned grid = (unsigned)((p.n[0] * p.n[2] + bs - 1) / bs);
  Plane3DArgs a = make_args(p);
  if (ostep == 1) k_reduce_outer<T, 1><<<grid, bs, 0, st>>>((const C*)p.dbuf, (C*)out, a, skip);
  else k_reduce_outer<T, 2><<<grid, bs, 0, st>>>((const C*)p.dbuf, (C*)out, a, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_outer_cbb(const Plan3D& p, const void* v, const void* w, void* out, const int* skip, cudaStream_t st) {
  using C = typename cpx<T>::type;
  const int bs = 256;
  const unsigned grid = (unsigned)((p.n[0] * p.n[2] + bs - 1) / bs);
  k_outer_cbb<T><<<grid, bs, 0, st>>>((const C*)v, (const C*)w, (C*)out, make_args(p), skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t solve3d_t(Plan3D& p, const void* in, int in_is_double, void* out, int out_mode, double accum_scale,
                      const int* skip, void* dbg_fhat, void* dbg_v, void* dbg_w, cudaStream_t st, Profiler* prof) {
  using C = typename cpx<T>::type;
  const int prec = std::is_same<T, double>::value ? kPrecF64 : kPrecF32;
  const int64_t nx = p.n[0], ny = p.n[1], nz = p.n[2];
  const int64_t F = nx * nz;  // values per outer face
  const void* two = prec == kPrecF64 ? (const void*)p.axo->tw : (const void*)p.axo->tw32;
  const void* twi = prec == kPrecF64 ? (const void*)p.axi->tw : (const void*)p.axi->tw32;
  const int cmode = prec == kPrecF64 ? kOutC128 : kOutC64;
  const bool f64 = prec == kPrecF64;
  const void* sci_i = f64 ? (const void*)p.axi->sc_in : (const void*)p.axi->sc_in32;
  const void* sco_i = f64 ? (const void*)p.axi->sc_out : (const void*)p.axi->sc_out32;
  const void* sci_o = f64 ? (const void*)p.axo->sc_in : (const void*)p.axo->sc_in32;
  const void* sco_o = f64 ? (const void*)p.axo->sc_out : (const void*)p.axo->sc_out32;
  C* faces = (C*)p.faces;
  C* Vh = faces;           // reduced outer rows, inner-mode space   [2][nx][nz]
  C* v = faces + 2 * F;    // outer rows of v, physical
  C* w = faces + 4 * F;    // outer rows of w, physical
  C* c = faces + 6 * F;    // C_bb applied, physical
  C* ch = faces + 8 * F;   // its inner DFT
  cudaError_t e;
#define CK(x)                               \
  do {                                      \
    if ((e = (x)) != cudaSuccess) return e; \
  } while (0)
#define PK(name, x)                         \
  do {                                      \
    ProfScope ps_(prof, name, st);          \
    CK(x);                                  \
  } while (0)
  // a1: 2D DFT over (y, z): rows along z, then columns along y (in place)
  PK("dft_z_fwd", launch_dft_rows(prec, in, in_is_double, p.fhat, cmode, nx * ny, p.axi->dft, twi, -1, 1.0, 0.0, sci_i,
                                  nullptr, skip, st));
  PK("dft_y_fwd", launch_dft_cols(prec, p.fhat, f64, p.fhat, cmode, nx, nz, p.axo->dft, two, -1, 1.0, 0.0, sci_o, nullptr,
                                  skip, st));
  if (dbg_fhat) CK(cudaMemcpyAsync(dbg_fhat, p.fhat, nx * ny * nz * sizeof(C), cudaMemcpyDeviceToDevice, st));
  // outer Step 1
  if (p.inner_nmb) CK(launch_inner<T>(1, p, nullptr, skip, st, prof));
  else PK("plane3d_step1", launch_plane<T>(1, p, nullptr, skip, st));
  PK("reduce_outer", launch_reduce_outer<T>(1, p, Vh, skip, st));
  CK(launch_dft_rows(prec, Vh, f64, v, cmode, 2 * nx, p.axi->dft, twi, +1, 1.0 / (double)nz, 0.0, nullptr, sco_i, skip, st));
  if (dbg_v) CK(cudaMemcpyAsync(dbg_v, v, 2 * F * sizeof(C), cudaMemcpyDeviceToDevice, st));
  CK(launch_outer_cbb<T>(p, v, nullptr, c, skip, st));
  CK(launch_dft_rows(prec, c, f64, ch, cmode, 2 * nx, p.axi->dft, twi, -1, 1.0, 0.0, sci_i, nullptr, skip, st));
  // outer Step 2
  if (p.inner_nmb) CK(launch_inner<T>(2, p, ch, skip, st, prof));
  else PK("plane3d_step2", launch_plane<T>(2, p, ch, skip, st));
  PK("reduce_outer", launch_reduce_outer<T>(2, p, Vh, skip, st));
  CK(launch_dft_rows(prec, Vh, f64, w, cmode, 2 * nx, p.axi->dft, twi, +1, 1.0 / (double)nz, 0.0, nullptr, sco_i, skip, st));
  if (dbg_w) CK(cudaMemcpyAsync(dbg_w, w, 2 * F * sizeof(C), cudaMemcpyDeviceToDevice, st));
  CK(launch_outer_cbb<T>(p, v, w, c, skip, st));
  CK(launch_dft_rows(prec, c, f64, ch, cmode, 2 * nx, p.axi->dft, twi, -1, 1.0, 0.0, sci_i, nullptr, skip, st));
  // outer Step 3, then the inverse 2D DFT
  if (p.inner_nmb) CK(launch_inner<T>(3, p, ch, skip, st, prof));
  else PK("plane3d_step3", launch_plane<T>(3, p, ch, skip, st));
  PK("dft_y_inv", launch_dft_cols(prec, p.dbuf, f64, p.dbuf, cmode, nx, nz, p.axo->dft, two, +1, 1.0 / (double)ny, 0.0,
                                  nullptr, sco_o, skip, st));
  PK("dft_z_inv", launch_dft_rows(prec, p.dbuf, f64, out, out_mode, nx * ny, p.axi->dft, twi, +1, 1.0 / (double)nz,
                                  accum_scale, nullptr, sco_i, skip, st));
#undef PK
#undef CK
  return cudaSuccess;
}

}  // namespace

cudaError_t plan3d_init(Plan3D& p, int prec, const int64_t* n, const double* h, double omega, const double* wc, double mden,
                        const AxisData& axo, const AxisData& axi, size_t* bytes) {
  p.prec = prec;
  for (int k = 0; k < 3; ++k) {
    p.n[k] = n[k];
    p.h[k] = h[k];
    p.wc[k] = wc[k];
  }
  p.omega = omega;
  p.mden = mden;
  p.axo = &axo;
  p.axi = &axi;
  const size_t cb = prec == kPrecF64 ? sizeof(double2) : sizeof(float2);
  const int64_t N = n[0] * n[1] * n[2];
  const int64_t F = n[0] * n[2];
  cudaError_t e;
  void** bufs[4] = {&p.fhat, &p.cbuf, &p.dbuf, &p.faces};
  size_t sizes[4] = {N * cb, N * cb, N * cb, 10 * F * cb};
  for (int i = 0; i < 4; ++i) {
    if ((e = dmalloc((void**)bufs[i], sizes[i])) != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    *bytes += sizes[i];
  }
  // per-plan pivot tables of the four inner line types (with the per-line
  // settling data of the tiled sweeps); without room for them the kernels
  // recompute the pivots
  const int64_t lines = n[1] * n[2];
  const size_t per_type = N * cb + lines * (kLineVals * cb + sizeof(int));
  for (int t = 0; t < 4; ++t) {
    if (dmalloc((void**)&p.tab[t], N * cb) != cudaSuccess || dmalloc((void**)&p.lend[t], lines * kLineVals * cb) != cudaSuccess ||
        dmalloc((void**)&p.lenL[t], lines * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      for (int u = 0; u < 4; ++u) {
        dfree(p.tab[u]);
        dfree(p.lend[u]);
        dfree(p.lenL[u]);
        p.tab[u] = p.lend[u] = nullptr;
        p.lenL[u] = nullptr;
      }
      *bytes -= (size_t)t * per_type;
      break;
    }
    *bytes += per_type;
  }
  // tiled inner sweeps: when the tables exist and a tile of kMW lines fits
  // the shared memory of one CTA
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // 16 rows per chunk, 32 for lines too long for 16 (the kernels hold a
  // chunk in registers, so CH is one of 8, 16, 32)
  int ch = 16, nc = (int)((n[0] + 15) / 16);
  if (nc > inner_max_chunks(prec, ch)) {
    ch = 32;
    nc = (int)((n[0] + 31) / 32);
  }
  const size_t ismem = inner_smem_bytes(n[0], nc, ch, cb);
  if (p.tab[0] && nc <= inner_max_chunks(prec, ch) && ismem <= (size_t)smem_max) {
    const int64_t tiles = (n[2] + kMW - 1) / kMW;
    const int64_t total = tiles * n[1];
    int nmb = (int)std::max<int64_t>(1, std::min<int64_t>(4, total / (152 * 8)));
    nmb = (int)std::min<int64_t>(nmb, tiles);
    const int nparts = (int)((tiles + nmb - 1) / nmb);
    const size_t sz[3] = {(size_t)n[1] * nparts * 2 * n[0] * cb, (size_t)n[1] * 4 * n[0] * cb,
                          (size_t)n[1] * 2 * n[0] * cb};
    void** dst[3] = {&p.ipart, &p.ivw, &p.icin};
    bool ok = true;
    for (int i = 0; i < 3 && ok; ++i) {
      ok = dmalloc((void**)dst[i], sz[i]) == cudaSuccess;
      if (ok) *bytes += sz[i];
    }
    if (ok) {
      p.inner_ch = ch;
      p.inner_nc = nc;
      p.inner_nmb = nmb;
      p.inner_nparts = nparts;
    } else {
      cudaGetLastError();
    }
  }
  p.route_tau = prec == kPrecF32 ? kDefaultRouteTau : 0.0;
  p.ready = true;
  return plan3d_tables(p);
}

cudaError_t plan3d_tables_no_routing(Plan3D& p);

namespace {

void free_routing(Plan3D& p) {
  for (int t = 0; t < 4; ++t) {
    dfree(p.rlist[t]);
    dfree(p.roff[t]);
    dfree(p.rtab[t]);
    p.rlist[t] = p.roff[t] = nullptr;
    p.rtab[t] = nullptr;
    p.nroute[t] = 0;
  }
  dfree(p.rpart);
  dfree(p.rtmp);
  p.rpart = p.rtmp = nullptr;
  p.route_bytes = 0;
}

// The routed lines of every line type: the inner lines (l, m) whose line
// matrix K_x + s M_x, s = Lam_outer,l + Lam_inner,m - w^2, has an eigenvalue
// Lam^A_x,k + s within tau w^2 of zero (Lam^A_x: the pencil of the
// tridiagonal axis, absorbing or Neumann).  Those matrices amplify the
// rounding of the complex64 sweeps by their condition number; they are few
// (the modes next to the resonance surface).  The nearest Lam^A_x,k to -s is
// found by bisection on the real parts (the pencil's eigenvalues lie close to
// the real axis) and a window of neighbours.
cudaError_t build_routing(Plan3D& p) {
  free_routing(p);
  if (p.route_tau <= 0 || p.prec != kPrecF32 || !p.inner_nmb) return cudaSuccess;
  const int64_t nx = p.n[0], ny = p.n[1], nz = p.n[2];
  std::vector<double> lamx(2 * nx), sigx(2 * nx);
  std::vector<int8_t> parx(nx);
  if (abc_eigen(nx, p.h[0], p.wc[0], lamx.data(), sigx.data(), parx.data(), p.mden) != 0) return cudaSuccess;
  std::vector<std::pair<double, double>> ex(nx);
  for (int64_t k = 0; k < nx; ++k) ex[k] = {lamx[2 * k], lamx[2 * k + 1]};
  std::sort(ex.begin(), ex.end());
  std::vector<double> lbo(2 * ny), lao(2 * ny), lbi(2 * nz), lai(2 * nz);
  cudaError_t e;
  if ((e = cudaMemcpy(lbo.data(), p.axo->lamB, 2 * ny * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(lao.data(), p.axo->lamA, 2 * ny * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(lbi.data(), p.axi->lamB, 2 * nz * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(lai.data(), p.axi->lamA, 2 * nz * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return e;
  const double w2 = p.omega * p.omega, lim2 = (p.route_tau * w2) * (p.route_tau * w2);
  const Plane3DArgs a = make_args(p);
  int maxr = 0;
  for (int t = 0; t < 4; ++t) {
    const std::vector<double>& lo = (t >> 1) ? lao : lbo;
    const std::vector<double>& li = (t & 1) ? lai : lbi;
    std::vector<int> list, off(ny + 1, 0);
    for (int64_t l = 0; l < ny; ++l) {
      off[l] = (int)list.size();
      for (int64_t m = 0; m < nz; ++m) {
        const double sr = lo[2 * l] + li[2 * m] - w2, si = lo[2 * l + 1] + li[2 * m + 1];
        const auto it = std::lower_bound(ex.begin(), ex.end(), std::make_pair(-sr, -1e300));
        const int64_t c0 = it - ex.begin();
        double best = HUGE_VAL;
        for (int64_t k = std::max<int64_t>(0, c0 - 8); k < std::min<int64_t>(nx, c0 + 8); ++k) {
          const double dr = ex[k].first + sr, di = ex[k].second + si;
          best = std::min(best, dr * dr + di * di);
        }
        if (best < lim2) list.push_back((int)(l * nz + m));
      }
    }
    off[ny] = (int)list.size();
    p.nroute[t] = (int)list.size();
    if (list.empty()) continue;
    maxr = std::max(maxr, p.nroute[t]);
    const size_t sz[3] = {list.size() * sizeof(int), (size_t)(ny + 1) * sizeof(int),
                          list.size() * (size_t)nx * sizeof(double2)};
    if ((e = dmalloc((void**)&p.rlist[t], sz[0])) != cudaSuccess || (e = dmalloc((void**)&p.roff[t], sz[1])) != cudaSuccess ||
        (e = dmalloc(&p.rtab[t], sz[2])) != cudaSuccess) {
      free_routing(p);
      return cudaSuccess;  // no room: every line stays in complex64
    }
    p.route_bytes += sz[0] + sz[1] + sz[2];
    if ((e = cudaMemcpy(p.rlist[t], list.data(), sz[0], cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p.roff[t], off.data(), sz[1], cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
    k_route_tables<<<(unsigned)((list.size() + 127) / 128), 128>>>((double2*)p.rtab[t], p.lenL[t], p.rlist[t],
                                                                   p.nroute[t], a, t >> 1, t & 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (maxr) {
    const size_t cb = sizeof(float2);
    if (dmalloc(&p.rpart, (size_t)maxr * 2 * nx * cb) != cudaSuccess ||
        dmalloc(&p.rtmp, (size_t)maxr * nx * sizeof(double2)) != cudaSuccess) {
      free_routing(p);
      return plan3d_tables_no_routing(p);
    }
    p.route_bytes += (size_t)maxr * nx * (2 * cb + sizeof(double2));
  }
  return cudaStreamSynchronize(nullptr);  // plan-time kernels run on the legacy stream
}

}  // namespace

cudaError_t plan3d_tables(Plan3D& p) {
  if (!p.tab[0]) return cudaSuccess;
  cudaError_t e = plan3d_tables_no_routing(p);
  if (e != cudaSuccess) return e;
  return build_routing(p);
}

cudaError_t plan3d_set_routing(Plan3D& p, double tau) {
  p.route_tau = tau > 0 ? tau : 0;
  if (!p.tab[0]) return cudaSuccess;
  // the routed flags live in the settling-row tables: rebuild them first
  cudaError_t e = plan3d_tables_no_routing(p);
  if (e != cudaSuccess) return e;
  return build_routing(p);
}

int plan3d_routed_lines(const Plan3D& p) { return p.nroute[0] + p.nroute[1] + p.nroute[2] + p.nroute[3]; }

cudaError_t plan3d_set_inner(Plan3D& p, int ch, int nmb) {
  if (!p.inner_nmb || nmb < 1 || nmb > 8) return cudaErrorInvalidValue;
  const size_t cb = p.prec == kPrecF64 ? sizeof(double2) : sizeof(float2);
  const int max_nc = inner_max_chunks(p.prec, ch);  // 0 unless ch is 8, 16 or 32
  const int nc = (int)((p.n[0] + ch - 1) / ch);
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (nc > max_nc || inner_smem_bytes(p.n[0], nc, ch, cb) > (size_t)smem_max) return cudaErrorInvalidValue;
  const int64_t tiles = (p.n[2] + kMW - 1) / kMW;
  nmb = (int)std::min<int64_t>(nmb, tiles);
  const int nparts = (int)((tiles + nmb - 1) / nmb);
  if (nparts > p.inner_nparts) {  // more face partials: a larger buffer
    void* q = nullptr;
    cudaError_t e = dmalloc(&q, (size_t)p.n[1] * nparts * 2 * p.n[0] * cb);
    if (e != cudaSuccess) return e;
    dfree(p.ipart);
    p.ipart = q;
  }
  p.inner_ch = ch;
  p.inner_nc = nc;
  p.inner_nmb = nmb;
  p.inner_nparts = nparts;
  return plan3d_tables(p);  // the settled-chunk constants depend on ch
}

cudaError_t plan3d_tables_no_routing(Plan3D& p) {
  if (!p.tab[0]) return cudaSuccess;
  const Plane3DArgs a = make_args(p);
  const int bs = 128;
  const unsigned grid = (unsigned)((p.n[1] * p.n[2] + bs - 1) / bs);
  for (int t = 0; t < 4; ++t) {
    if (p.prec == kPrecF64)
      k_plane_tables<double><<<grid, bs>>>((double2*)p.tab[t], (double2*)p.lend[t], p.lenL[t], a, t >> 1, t & 1,
                                           p.inner_ch > 0 ? p.inner_ch : 16);
    else
      k_plane_tables<float><<<grid, bs>>>((float2*)p.tab[t], (float2*)p.lend[t], p.lenL[t], a, t >> 1, t & 1,
                                          p.inner_ch > 0 ? p.inner_ch : 16);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(nullptr);  // plan-time kernels run on the legacy stream
}

void free_plan3d(Plan3D& p) {
  free_routing(p);
  for (int t = 0; t < 4; ++t) {
    dfree(p.tab[t]);
    dfree(p.lend[t]);
    dfree(p.lenL[t]);
  }
  dfree(p.ipart);
  dfree(p.ivw);
  dfree(p.icin);
  dfree(p.fhat);
  dfree(p.cbuf);
  dfree(p.dbuf);
  dfree(p.ybuf);
  dfree(p.faces);
  dfree(p.partial);
  p = Plan3D{};
}

cudaError_t solve3d_core(Plan3D& p, int prec, const void* in, int in_is_double, void* out, int out_mode,
                         double accum_scale, const int* skip, void* dbg_fhat, void* dbg_v, void* dbg_w,
                         cudaStream_t st, Profiler* prof) {
  if (!p.ready) return cudaErrorNotReady;
  if (prec == kPrecF64)
    return solve3d_t<double>(p, in, in_is_double, out, out_mode, accum_scale, skip, dbg_fhat, dbg_v, dbg_w, st, prof);
  return solve3d_t<float>(p, in, in_is_double, out, out_mode, accum_scale, skip, dbg_fhat, dbg_v, dbg_w, st, prof);
}

}  // namespace helm
