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
#include <type_traits>

#include "helm_dft.h"
#include "helm_kernels.cuh"
#include "helm_solve3d.h"

namespace helm {

namespace {

struct Plane3DArgs {
  int64_t nx, ny, nz;
  double hx, hy, hz, omega;
  // outer axis (y) eigen-data (Lam^B and 1/mu complex: gamma-circulant auxiliary)
  const double *lamBo, *invmuo, *lamAo, *sigAo, *parAo, *two;
  // inner axis (z) eigen-data
  const double *lamBi, *invmui, *lamAi, *sigAi, *parAi, *twi;
  double en_o[2], eninv_o[2], g_o[2], ginv_o[2];
  double en_i[2], eninv_i[2], g_i[2], ginv_i[2];
};

constexpr int XC = 32;  // rows per reduction chunk

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
__device__ void plane_cbb(const C* v, const C* w2, C* out, int nx, double hx, double hz, double omega,
                          double pre, double pim, C g, C ginv) {
  for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
    auto get = [&](int face, int j) -> C {
      C t = v[face * nx + j];
      if (w2) t = cadd(t, w2[face * nx + j]);
      return t;
    };
    const bool end = (ix == 0 || ix == nx - 1);
    const double md = end ? 2.0 * hx / 6.0 : 4.0 * hx / 6.0, mo = hx / 6.0;
    const double kdr = end ? 1.0 / hx : 2.0 / hx, kdi = end ? -omega : 0.0, ko = -1.0 / hx;
    C Mv[2], Kv[2];
    for (int f = 0; f < 2; ++f) {
      C v0 = get(f, ix);
      C vm = ix > 0 ? get(f, ix - 1) : mk<C>(0, 0);
      C vp = ix < nx - 1 ? get(f, ix + 1) : mk<C>(0, 0);
      C nb = cadd(vm, vp);
      Mv[f] = cadd(cscale(v0, (decltype(v0.x))md), cscale(nb, (decltype(v0.x))mo));
      Kv[f] = cadd(cmul(v0, mk<C>(kdr, kdi)), cscale(nb, (decltype(v0.x))ko));
    }
    const C D11 = mk<C>(1.0 / hz - pre * hz / 3.0, omega - pim * hz / 3.0);
    const C D1n = mk<C>(-1.0 / hz - pre * hz / 6.0, -pim * hz / 6.0);
    const auto E11 = (decltype(D11.x))(hz / 3.0), E1n = (decltype(D11.x))(hz / 6.0);
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
  thB.k = line_coef<C>(lo_re + lBi_re - w2, lo_im + lBi_im, a.hx, a.omega);
  thB.n = nx;
  thA.k = line_coef<C>(lo_re + a.lamAi[2 * mc] - w2, lo_im + a.lamAi[2 * mc + 1], a.hx, a.omega);
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
  plane_cbb(vin, (const C*)nullptr, cin, nx, a.hx, a.hz, a.omega, pre, pim, gi, giv);
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
  plane_cbb(vin, win, cin, nx, a.hx, a.hz, a.omega, pre, pim, gi, giv);
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
  auto ent = [&](int64_t n, double h, int64_t j, int d, double& m, double& kr, double& ki) {
    const bool end = (j == 0 || j == n - 1);
    if (d == 0) {
      m = (end ? 2.0 : 4.0) * h / 6.0;
      kr = (end ? 1.0 : 2.0) / h;
      ki = end ? -a.omega : 0.0;
    } else {
      m = h / 6.0;
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
    ent(nx, a.hx, ix, dx, mx, kxr, kxi);
    for (int dz = -1; dz <= 1; ++dz) {
      const int64_t jz = iz + dz;
      if (jz < 0 || jz >= nz) continue;
      double mz, kzr, kzi;
      ent(nz, a.hz, iz, dz, mz, kzr, kzi);
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
  const T2 e11 = (T2)(a.hy / 3.0), e1n = (T2)(a.hy / 6.0);
  const C d11 = mk<C>(1.0 / a.hy, a.omega);
  const T2 d1n = (T2)(-1.0 / a.hy);
  const C g = mk<C>(a.g_o[0], a.g_o[1]), gv = mk<C>(a.ginv_o[0], a.ginv_o[1]);
  out[i] = cadd(cadd(cscale(Sv[0], e11), cmul(d11, Pv[0])), cmul(gv, cadd(cscale(Sv[1], e1n), cscale(Pv[1], d1n))));
  out[nx * nz + i] = cadd(cmul(g, cadd(cscale(Sv[0], e1n), cscale(Pv[0], d1n))), cadd(cscale(Sv[1], e11), cmul(d11, Pv[1])));
}

// Reciprocal pivots of the inner tridiagonal lines of one line type (outer
// mode type x inner mode type), for every (x, l, m): the FP64 recurrence of
// ThomasRow, stored in the compute precision at the layout of the scratch.
template <typename T>
__global__ void k_plane_tables(typename cpx<T>::type* __restrict__ tab, Plane3DArgs a, int outerA, int innerA) {
  using C = typename cpx<T>::type;
  const int64_t ny = a.ny, nz = a.nz, nx = a.nx;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // l * nz + m
  if (i >= ny * nz) return;
  const int64_t l = i / nz, m = i - l * nz;
  const double* lo = outerA ? a.lamAo : a.lamBo;
  const double* li = innerA ? a.lamAi : a.lamBi;
  const double w2 = a.omega * a.omega;
  const LineCoef<double2> k = line_coef<double2>(lo[2 * l] + li[2 * m] - w2, lo[2 * l + 1] + li[2 * m + 1], a.hx, a.omega);
  double2 c = make_double2(0, 0);
  for (int64_t ix = 0; ix < nx; ++ix) {
    const double2 aj = (ix == 0 || ix == nx - 1) ? k.ac : k.a;
    const double2 den = ix == 0 ? aj : csub(aj, cmul(k.b, c));
    const double2 inv = crecip(den);
    c = cmul(k.b, inv);
    tab[ix * ny * nz + i] = cvt<C>(inv);
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
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<(unsigned)p.n[1], bs, smem, st>>>((const C*)p.fhat, (C*)p.cbuf, (C*)p.dbuf, (const C*)gfaces, tB, tA, a,
                                             skip);
  };
  const bool tab = tB && tA;
  if (ostep == 1) tab ? run(k_plane3d<T, 1, true>) : run(k_plane3d<T, 1, false>);
  else if (ostep == 2) tab ? run(k_plane3d<T, 2, true>) : run(k_plane3d<T, 2, false>);
  else tab ? run(k_plane3d<T, 3, true>) : run(k_plane3d<T, 3, false>);
  return cudaGetLastError();
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
  PK("plane3d_step1", launch_plane<T>(1, p, nullptr, skip, st));
  PK("reduce_outer", launch_reduce_outer<T>(1, p, Vh, skip, st));
  CK(launch_dft_rows(prec, Vh, f64, v, cmode, 2 * nx, p.axi->dft, twi, +1, 1.0 / (double)nz, 0.0, nullptr, sco_i, skip, st));
  if (dbg_v) CK(cudaMemcpyAsync(dbg_v, v, 2 * F * sizeof(C), cudaMemcpyDeviceToDevice, st));
  CK(launch_outer_cbb<T>(p, v, nullptr, c, skip, st));
  CK(launch_dft_rows(prec, c, f64, ch, cmode, 2 * nx, p.axi->dft, twi, -1, 1.0, 0.0, sci_i, nullptr, skip, st));
  // outer Step 2
  PK("plane3d_step2", launch_plane<T>(2, p, ch, skip, st));
  PK("reduce_outer", launch_reduce_outer<T>(2, p, Vh, skip, st));
  CK(launch_dft_rows(prec, Vh, f64, w, cmode, 2 * nx, p.axi->dft, twi, +1, 1.0 / (double)nz, 0.0, nullptr, sco_i, skip, st));
  if (dbg_w) CK(cudaMemcpyAsync(dbg_w, w, 2 * F * sizeof(C), cudaMemcpyDeviceToDevice, st));
  CK(launch_outer_cbb<T>(p, v, w, c, skip, st));
  CK(launch_dft_rows(prec, c, f64, ch, cmode, 2 * nx, p.axi->dft, twi, -1, 1.0, 0.0, sci_i, nullptr, skip, st));
  // outer Step 3, then the inverse 2D DFT
  PK("plane3d_step3", launch_plane<T>(3, p, ch, skip, st));
  PK("dft_y_inv", launch_dft_cols(prec, p.dbuf, f64, p.dbuf, cmode, nx, nz, p.axo->dft, two, +1, 1.0 / (double)ny, 0.0,
                                  nullptr, sco_o, skip, st));
  PK("dft_z_inv", launch_dft_rows(prec, p.dbuf, f64, out, out_mode, nx * ny, p.axi->dft, twi, +1, 1.0 / (double)nz,
                                  accum_scale, nullptr, sco_i, skip, st));
#undef PK
#undef CK
  return cudaSuccess;
}

}  // namespace

cudaError_t plan3d_init(Plan3D& p, int prec, const int64_t* n, const double* h, double omega, const AxisData& axo,
                        const AxisData& axi, size_t* bytes) {
  p.prec = prec;
  for (int k = 0; k < 3; ++k) {
    p.n[k] = n[k];
    p.h[k] = h[k];
  }
  p.omega = omega;
  p.axo = &axo;
  p.axi = &axi;
  const size_t cb = prec == kPrecF64 ? sizeof(double2) : sizeof(float2);
  const int64_t N = n[0] * n[1] * n[2];
  const int64_t F = n[0] * n[2];
  cudaError_t e;
  void** bufs[4] = {&p.fhat, &p.cbuf, &p.dbuf, &p.faces};
  size_t sizes[4] = {N * cb, N * cb, N * cb, 10 * F * cb};
  for (int i = 0; i < 4; ++i) {
    if ((e = cudaMalloc(bufs[i], sizes[i])) != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    *bytes += sizes[i];
  }
  // per-plan pivot tables of the four inner line types; without room for
  // them the kernels recompute the pivots
  for (int t = 0; t < 4; ++t) {
    if (cudaMalloc(&p.tab[t], N * cb) != cudaSuccess) {
      cudaGetLastError();
      for (int u = 0; u < 4; ++u) {
        cudaFree(p.tab[u]);
        p.tab[u] = nullptr;
      }
      *bytes -= (size_t)t * N * cb;
      break;
    }
    *bytes += N * cb;
  }
  p.ready = true;
  return plan3d_tables(p);
}

cudaError_t plan3d_tables(Plan3D& p) {
  if (!p.tab[0]) return cudaSuccess;
  const Plane3DArgs a = make_args(p);
  const int bs = 128;
  const unsigned grid = (unsigned)((p.n[1] * p.n[2] + bs - 1) / bs);
  for (int t = 0; t < 4; ++t) {
    if (p.prec == kPrecF64)
      k_plane_tables<double><<<grid, bs>>>((double2*)p.tab[t], a, t >> 1, t & 1);
    else
      k_plane_tables<float><<<grid, bs>>>((float2*)p.tab[t], a, t >> 1, t & 1);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaDeviceSynchronize();
}

void free_plan3d(Plan3D& p) {
  for (int t = 0; t < 4; ++t) cudaFree(p.tab[t]);
  cudaFree(p.fhat);
  cudaFree(p.cbuf);
  cudaFree(p.dbuf);
  cudaFree(p.ybuf);
  cudaFree(p.faces);
  cudaFree(p.partial);
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
