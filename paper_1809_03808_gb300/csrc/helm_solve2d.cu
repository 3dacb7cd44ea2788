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
// solved by the Thomas algorithm (LU without pivoting), evaluated in chunks of
// rows so that every (line, chunk) pair is a thread: no N-sized scratch, and
// enough parallelism for long lines.
#include <algorithm>

#include "helm_dft.h"
#include "helm_kernels.cuh"
#include "helm_solve.h"

namespace helm {

namespace {

// Chunked Thomas.  T = L U with pivots u_j (u_0 = a_0, u_j = a_j - b^2/u_{j-1}),
// multipliers m_j = b/u_{j-1}; forward y_j = r_j - m_j y_{j-1}; backward
// x_j = (y_j - b x_{j+1}) / u_j.  The line is cut into chunks of CH rows.
// Inside chunk k (rows s..e), with Y = y_{s-1} and X = x_{e+1} the carries,
//   y_j = ylo_j + P_j Y,          P_j = prod_{i=s..j} (-m_i),
//   x_s = sum_j w_j y_j - b w_e X, w_j = (U_kk^-1)_{s,j} = w_{j-1} (-b)/u_j,
// so the carries obey  Y(k) = a_k + Pe_k Y(k-1)  and
//   X(k) = bsum_k + cc_k Y(k-1) - b we_k X(k+1)
// with a_k = ylo_e, bsum_k = sum_j w_j ylo_j, cc_k = sum_j w_j P_j.  Pass 1
// computes the chunk summaries, k_tri_carry runs the two short scans per line,
// pass 2 redoes Thomas inside each chunk from the exact carries.  The pivots
// are the same sequence as plain Thomas: each chunk restarts it from u_{s-1},
// computed once per plan (k_pivots).

// Per-chunk summary record (one per line and chunk).
template <typename C>
struct ChunkRec {
  C a, bsum, pe, cc, we;
};

// Right-hand side of line lc at row ix.  Step 1: fhat / mu_l.  Step 2:
// c_1 + par_l c_n.  Step 3: (fhat + d_1 + e^{+i theta_l} e^{-t(n1-1)} d_n) / mu_l
// (wl = e^{+i theta_l} e^{-t(n1-1)}).
template <typename C>
__device__ __forceinline__ C line_rhs(int step, int64_t ix, int64_t lc, int64_t n1, const C* __restrict__ fhat,
                                      const C* __restrict__ f1, const C* __restrict__ fn, C scal,
                                      decltype(C().x) par, C wl) {
  if (step == 1) return cmul(fhat[ix * n1 + lc], scal);
  if (step == 2) return cadd(f1[ix], cscale(fn[ix], par));
  C v = cadd(fhat[ix * n1 + lc], f1[ix]);
  v = cadd(v, cmul(fn[ix], wl));
  return cmul(v, scal);
}

template <typename C>
__device__ __forceinline__ C step3_weight(const Solve2DArgs& a, int64_t l) {
  // conj(tw_l) * e^{-t(n1-1)}
  const C twc = mk<C>(a.tw[2 * l], -a.tw[2 * l + 1]);
  return cmul(twc, mk<C>(a.eninv[0], a.eninv[1]));
}

struct LineParams {
  double sre, sim;
};

__device__ __forceinline__ LineParams line_params(int step, const Solve2DArgs& a, int64_t lc) {
  LineParams p;
  if (step == 2) {
    p.sre = a.lamA[2 * lc] - a.omega * a.omega;
    p.sim = a.lamA[2 * lc + 1];
  } else {
    p.sre = a.lamB[2 * lc] - a.omega * a.omega;
    p.sim = a.lamB[2 * lc + 1];
  }
  return p;
}

template <typename T, int STEP, int CH>
__global__ void __launch_bounds__(128) k_tri_pass1(const typename cpx<T>::type* __restrict__ fhat,
                                                   const typename cpx<T>::type* __restrict__ faces,
                                                   const typename cpx<T>::type* __restrict__ ustart,
                                                   ChunkRec<typename cpx<T>::type>* __restrict__ rec,
                                                   Solve2DArgs a, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n1) return;
  const int64_t k = blockIdx.y;
  const int64_t s = k * CH, e = min(s + (int64_t)CH, nx) - 1;
  const int cnt = (int)(e - s + 1);
  const LineParams lp = line_params(STEP, a, l);
  const LineCoef<C> co = line_coef<C>(lp.sre, lp.sim, a.hx, a.omega);
  const C scal = (STEP == 2) ? mk<C>(1, 0) : mk<C>(a.invmu[2 * l], a.invmu[2 * l + 1]);
  const C wl = step3_weight<C>(a, l);
  const T par = (T)a.parA[l];
  const C* f1 = faces;
  const C* fn = faces + nx;
  const C zero = mk<C>(0, 0);
  // 1/u of the row before the chunk (the pivot entering it); carried so that
  // each row needs one complex reciprocal
  C inv = (k > 0) ? crecip(ustart[k * n1 + l]) : zero;
  C ylo = zero, P = zero, w = zero, bsum = zero, cc = zero;
  const C mb = mk<C>(-(double)co.b.x, -(double)co.b.y);  // -b
  // all right-hand sides of the chunk first: independent loads in flight
  C rr[CH];
#pragma unroll
  for (int t = 0; t < CH; ++t)
    if (t < cnt) rr[t] = line_rhs<C>(STEP, s + t, l, n1, fhat, f1, fn, scal, par, wl);
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    if (t >= cnt) break;
    const int64_t j = s + t;
    const C aj = (j == 0 || j == nx - 1) ? co.ac : co.a;
    const C r = rr[t];
    C m = zero, u;
    if (j > 0) {
      m = cmul(co.b, inv);
      u = csub(aj, cmul(m, co.b));
    } else {
      u = aj;
    }
    inv = crecip(u);
    ylo = (j == s) ? r : csub(r, cmul(m, ylo));
    const C mm = mk<C>(-(double)m.x, -(double)m.y);
    P = (j == s) ? mm : cmul(P, mm);
    w = (j == s) ? inv : cmul(cmul(w, mb), inv);
    bsum = cadd(bsum, cmul(w, ylo));
    cc = cadd(cc, cmul(w, P));
  }
  ChunkRec<C> R;
  R.a = ylo;
  R.bsum = bsum;
  R.pe = (k > 0) ? P : zero;
  R.cc = (k > 0) ? cc : zero;
  R.we = w;
  rec[k * n1 + l] = R;
}

// Two scans per line over its chunks: forward carry Y, backward carry X.
// Overwrites rec[k].a with Y(k-1) and rec[k].bsum with X(k+1).  The records of
// a batch of CB chunks are loaded before the dependent recurrence runs over
// them, and the next batch is requested while the current one is processed,
// so the sequential chain waits on arithmetic rather than on memory.
template <typename T, int STEP>
__global__ void k_tri_carry(ChunkRec<typename cpx<T>::type>* __restrict__ rec, Solve2DArgs a,
                            const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  constexpr int CB = 8;
  if (skip && *skip) return;
  const int64_t n1 = a.n1;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n1) return;
  const int64_t K = a.nchunks;
  const LineParams lp = line_params(STEP, a, l);
  const LineCoef<C> co = line_coef<C>(lp.sre, lp.sim, a.hx, a.omega);
  // forward: Y(k) = a_k + pe_k Y(k-1)
  C Y = mk<C>(0, 0);
  C ra[CB], rp[CB], na[CB], np[CB];
  auto loadf = [&](int64_t k0, C* A, C* Pp) {
#pragma unroll
    for (int t = 0; t < CB; ++t) {
      const int64_t k = k0 + t;
      if (k < K) {
        A[t] = rec[k * n1 + l].a;
        Pp[t] = rec[k * n1 + l].pe;
      }
    }
  };
  loadf(0, ra, rp);
  for (int64_t k0 = 0; k0 < K; k0 += CB) {
    if (k0 + CB < K) loadf(k0 + CB, na, np);
#pragma unroll
    for (int t = 0; t < CB; ++t) {
      const int64_t k = k0 + t;
      if (k < K) {
        rec[k * n1 + l].a = Y;  // Y(k-1)
        Y = cadd(ra[t], cmul(rp[t], Y));
      }
    }
#pragma unroll
    for (int t = 0; t < CB; ++t) {
      ra[t] = na[t];
      rp[t] = np[t];
    }
  }
  // backward: X(k) = bsum_k + cc_k Y(k-1) - b we_k X(k+1)
  C X = mk<C>(0, 0);
  C rb[CB], rc[CB], rw[CB], ry[CB], nb[CB], nc[CB], nw[CB], ny[CB];
  auto loadb = [&](int64_t k1, C* B, C* Cc, C* W, C* Yp) {  // chunks k1, k1-1, ...
#pragma unroll
    for (int t = 0; t < CB; ++t) {
      const int64_t k = k1 - t;
      if (k >= 0) {
        const ChunkRec<C>& R = rec[k * n1 + l];
        B[t] = R.bsum;
        Cc[t] = R.cc;
        W[t] = R.we;
        Yp[t] = R.a;
      }
    }
  };
  loadb(K - 1, rb, rc, rw, ry);
  for (int64_t k1 = K - 1; k1 >= 0; k1 -= CB) {
    if (k1 - CB >= 0) loadb(k1 - CB, nb, nc, nw, ny);
#pragma unroll
    for (int t = 0; t < CB; ++t) {
      const int64_t k = k1 - t;
      if (k >= 0) {
        rec[k * n1 + l].bsum = X;  // X(k+1)
        X = csub(cadd(rb[t], cmul(rc[t], ry[t])), cmul(cmul(co.b, rw[t]), X));
      }
    }
#pragma unroll
    for (int t = 0; t < CB; ++t) {
      rb[t] = nb[t];
      rc[t] = nc[t];
      rw[t] = nw[t];
      ry[t] = ny[t];
    }
  }
}

// Pass 2: Thomas inside each chunk from the exact carries; emit x.
template <typename T, int STEP, int CH>
__global__ void __launch_bounds__(128) k_tri_pass2(const typename cpx<T>::type* __restrict__ fhat,
                                                   const typename cpx<T>::type* __restrict__ faces,
                                                   const typename cpx<T>::type* __restrict__ ustart,
                                                   const ChunkRec<typename cpx<T>::type>* __restrict__ rec,
                                                   typename cpx<T>::type* __restrict__ out,
                                                   typename cpx<T>::type* __restrict__ partial, Solve2DArgs a,
                                                   const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((l & ~(int64_t)31) >= n1) return;  // whole warp beyond the last line
  const bool act = l < n1;
  const int64_t lc = act ? l : 0;
  const int64_t k = blockIdx.y;
  const int64_t s = k * CH, e = min(s + CH, nx) - 1;
  const int cnt = (int)(e - s + 1);
  const LineParams lp = line_params(STEP, a, lc);
  const LineCoef<C> co = line_coef<C>(lp.sre, lp.sim, a.hx, a.omega);
  const C scal = (STEP == 2) ? mk<C>(1, 0) : mk<C>(a.invmu[2 * lc], a.invmu[2 * lc + 1]);
  const C twl = mk<C>(a.tw[2 * lc], a.tw[2 * lc + 1]);
  const C wl = step3_weight<C>(a, lc);
  const T par = (T)a.parA[lc];
  const C sig = mk<C>(a.sigA[2 * lc], a.sigA[2 * lc + 1]);
  const C* f1 = faces;
  const C* fn = faces + nx;
  const C zero = mk<C>(0, 0);
  C y[CH], iu[CH];
  const ChunkRec<C> R = rec[k * n1 + lc];
  C inv = (k > 0) ? crecip(ustart[k * n1 + lc]) : zero;
  C yp = R.a;  // Y(k-1)
  // right-hand sides into registers first (y[] holds them until overwritten)
#pragma unroll
  for (int t = 0; t < CH; ++t)
    if (t < cnt) y[t] = line_rhs<C>(STEP, s + t, lc, n1, fhat, f1, fn, scal, par, wl);
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    if (t < cnt) {
      const int64_t j = s + t;
      const C aj = (j == 0 || j == nx - 1) ? co.ac : co.a;
      const C r = y[t];
      C m = zero, u;
      if (j > 0) {
        m = cmul(co.b, inv);
        u = csub(aj, cmul(m, co.b));
      } else {
        u = aj;
      }
      inv = crecip(u);
      iu[t] = inv;
      yp = csub(r, cmul(m, yp));
      y[t] = yp;
    }
  }
  const int lane = threadIdx.x & 31;
  const int64_t warp = l >> 5;
  const int64_t nwarps = (n1 + 31) >> 5;
  C xn = R.bsum;  // X(k+1)
#pragma unroll
  for (int t = CH - 1; t >= 0; --t) {
    if (t < cnt) {
      const int64_t j = s + t;
      const C x = cmul(csub(y[t], cmul(co.b, xn)), iu[t]);
      xn = x;
      if (STEP == 3) {
        if (act) out[j * n1 + lc] = x;
      } else {
        C s1, sn;
        if (STEP == 1) {
          s1 = act ? x : zero;
          sn = act ? cmul(x, twl) : zero;
        } else {
          const C tt = act ? cmul(x, sig) : zero;
          s1 = tt;
          sn = cscale(tt, par);
        }
        s1 = warp_sum(s1);
        sn = warp_sum(sn);
        if (lane == 0) {
          partial[warp * nx + j] = s1;
          partial[(nwarps + warp) * nx + j] = sn;
        }
      }
    }
  }
}

// Pivot entering each chunk, u_{kCH-1}, for every line: FP64 sequential
// recurrence once per plan (same sequence as plain Thomas).
template <typename T>
__global__ void k_pivots(typename cpx<T>::type* __restrict__ ustart, Solve2DArgs a, int step) {
  using C = typename cpx<T>::type;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n1) return;
  const LineParams lp = line_params(step, a, l);
  const LineCoef<double2> co = line_coef<double2>(lp.sre, lp.sim, a.hx, a.omega);
  double2 u = co.ac;
  const double2 b2 = cmul(co.b, co.b);
  if ((a.ch - 1) == 0 && a.nchunks > 1) ustart[1 * n1 + l] = cvt<C>(u);
  for (int64_t j = 1; j < nx; ++j) {
    const double2 aj = (j == nx - 1) ? co.ac : co.a;
    u = csub(aj, cmul(b2, crecip(u)));
    if ((j + 1) % a.ch == 0 && (j + 1) / a.ch < a.nchunks) ustart[((j + 1) / a.ch) * n1 + l] = cvt<C>(u);
  }
}

// Sum the per-warp partials: out[face * nx + ix] = scale * sum_w partial.
template <typename T>
__global__ void k_reduce_faces(const typename cpx<T>::type* __restrict__ partial,
                               typename cpx<T>::type* __restrict__ out, int64_t nx, int64_t nwarps, double s0r,
                               double s0i, double s1r, double s1i, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * nx) return;
  const int64_t face = i / nx, ix = i - face * nx;
  C acc = mk<C>(0, 0);
  for (int64_t w = 0; w < nwarps; ++w) acc = cadd(acc, partial[(face * nwarps + w) * nx + ix]);
  out[i] = cmul(acc, face == 0 ? mk<C>(s0r, s0i) : mk<C>(s1r, s1i));
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
                            double omega, double p, double gr, double gi, double gir, double gii,
                            const int* __restrict__ skip) {
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
  // wrap entries of the gamma-circulant: first row x 1/g, last row x g
  C c1 = cadd(cadd(cmul(D11, Mv[0]), cscale(Kv[0], E11)),
              cmul(mk<C>(gir, gii), cadd(cmul(D1n, Mv[1]), cscale(Kv[1], E1n))));
  C cn = cadd(cmul(mk<C>(gr, gi), cadd(cmul(D1n, Mv[0]), cscale(Kv[0], E1n))),
              cadd(cmul(D11, Mv[1]), cscale(Kv[1], E11)));
  out[ix] = c1;
  out[nx + ix] = cn;
}

}  // namespace

cudaError_t launch_tri2d(int prec, int step, const void* fhat, const void* faces, const void* ustart, void* rec,
                         void* out, void* partial, const Solve2DArgs& a, const int* skip, cudaStream_t st,
                         Profiler* prof) {
  static const char* n1s[3] = {"tri_step1_pass1", "tri_step2_pass1", "tri_step3_pass1"};
  static const char* ncs[3] = {"tri_step1_carry", "tri_step2_carry", "tri_step3_carry"};
  static const char* n2s[3] = {"tri_step1_pass2", "tri_step2_pass2", "tri_step3_pass2"};
  const int bs = 128;
  const dim3 grid((unsigned)((a.n1 + bs - 1) / bs), (unsigned)a.nchunks);
  const unsigned gl = (unsigned)((a.n1 + bs - 1) / bs);
#define HELM_TRI(T, S, CH)                                                                                        \
  do {                                                                                                         \
    using C = cpx<T>::type;                                                                                    \
    {                                                                                                          \
      ProfScope ps(prof, n1s[S - 1], st);                                                                      \
      k_tri_pass1<T, S, CH><<<grid, bs, 0, st>>>((const C*)fhat, (const C*)faces, (const C*)ustart,            \
                                            (ChunkRec<C>*)rec, a, skip);                                      \
    }                                                                                                          \
    {                                                                                                          \
      ProfScope ps(prof, ncs[S - 1], st);                                                                      \
      k_tri_carry<T, S><<<gl, bs, 0, st>>>((ChunkRec<C>*)rec, a, skip);                                        \
    }                                                                                                          \
    {                                                                                                          \
      ProfScope ps(prof, n2s[S - 1], st);                                                                      \
      k_tri_pass2<T, S, CH><<<grid, bs, 0, st>>>((const C*)fhat, (const C*)faces, (const C*)ustart,            \
                                                (const ChunkRec<C>*)rec, (C*)out, (C*)partial, a, skip);      \
    }                                                                                                          \
  } while (0)
  if (prec == kPrecF64) {
    if (a.ch != kChunkF64) return cudaErrorInvalidValue;
    if (step == 1) HELM_TRI(double, 1, kChunkF64);
    else if (step == 2) HELM_TRI(double, 2, kChunkF64);
    else HELM_TRI(double, 3, kChunkF64);
  } else {
    if (a.ch != kChunkF32) return cudaErrorInvalidValue;
    if (step == 1) HELM_TRI(float, 1, kChunkF32);
    else if (step == 2) HELM_TRI(float, 2, kChunkF32);
    else HELM_TRI(float, 3, kChunkF32);
  }
#undef HELM_TRI
  return cudaGetLastError();
}

cudaError_t launch_pivots(int prec, void* ustart, const Solve2DArgs& a, int step, cudaStream_t st) {
  const int bs = 128;
  const unsigned grid = (unsigned)((a.n1 + bs - 1) / bs);
  if (prec == kPrecF64)
    k_pivots<double><<<grid, bs, 0, st>>>((double2*)ustart, a, step);
  else
    k_pivots<float><<<grid, bs, 0, st>>>((float2*)ustart, a, step);
  return cudaGetLastError();
}

size_t chunk_record_bytes(int prec) { return prec == kPrecF64 ? sizeof(ChunkRec<double2>) : sizeof(ChunkRec<float2>); }

cudaError_t launch_reduce_faces(int prec, const void* partial, void* out, int64_t nx, int64_t nwarps,
                                const double* s0, const double* s1, const int* skip, cudaStream_t st) {
  const int bs = 256;
  const unsigned grid = (unsigned)((2 * nx + bs - 1) / bs);
  if (prec == kPrecF64)
    k_reduce_faces<double><<<grid, bs, 0, st>>>((const double2*)partial, (double2*)out, nx, nwarps, s0[0], s0[1],
                                                s1[0], s1[1], skip);
  else
    k_reduce_faces<float><<<grid, bs, 0, st>>>((const float2*)partial, (float2*)out, nx, nwarps, s0[0], s0[1], s1[0],
                                               s1[1], skip);
  return cudaGetLastError();
}

cudaError_t launch_apply_cbb(int prec, const void* in, const void* in2, void* out, int64_t nx, double hx,
                             double h1, double omega, double p, const double* g, const double* ginv,
                             const int* skip, cudaStream_t st) {
  const int bs = 256;
  const unsigned grid = (unsigned)((nx + bs - 1) / bs);
  if (prec == kPrecF64)
    k_apply_cbb<double><<<grid, bs, 0, st>>>((const double2*)in, (const double2*)in2, (double2*)out, nx, hx,
                                             h1, omega, p, g[0], g[1], ginv[0], ginv[1], skip);
  else
    k_apply_cbb<float><<<grid, bs, 0, st>>>((const float2*)in, (const float2*)in2, (float2*)out, nx, hx, h1,
                                            omega, p, g[0], g[1], ginv[0], ginv[1], skip);
  return cudaGetLastError();
}

}  // namespace helm
