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
#include "helm_async.cuh"
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

// Per-chunk summary records (one per line and chunk), stored as five
// separate arrays indexed [chunk][line] so that a warp's accesses to one field
// are contiguous.
template <typename C>
struct ChunkRec {
  C a, bsum, pe, cc, we;
};
template <typename C>
struct RecSoA {
  C* a;
  C* bsum;
  C* pe;
  C* cc;
  C* we;
};
template <typename C>
__host__ __device__ inline RecSoA<C> rec_soa(void* base, size_t nrec) {
  C* b = reinterpret_cast<C*>(base);
  return RecSoA<C>{b, b + nrec, b + 2 * nrec, b + 3 * nrec, b + 4 * nrec};
}

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

// Per-line constants of one line type (B: Steps 1, 3; A: Step 2) in the
// compute precision, built once per plan: the three matrix entries, the rhs
// scale 1/mu_l, the Step-3 face weight, the Step-1 face weight e^{-i theta_l},
// sigma_l and the parity.  Eight arrays of n1 values.
template <typename C>
struct LineConst {
  const C* a;
  const C* ac;
  const C* b;
  const C* scal;
  const C* wl;
  const C* twl;
  const C* sig;
  const C* par;  // (+-1, 0)
};
template <typename C>
__host__ __device__ inline LineConst<C> line_const(const void* base, int64_t n1) {
  const C* p = reinterpret_cast<const C*>(base);
  return LineConst<C>{p, p + n1, p + 2 * n1, p + 3 * n1, p + 4 * n1, p + 5 * n1, p + 6 * n1, p + 7 * n1};
}

// The same values the tridiagonal kernels would compute per thread.
template <typename T, typename Cc>
struct LineValues {
  LineCoef<Cc> co;
  Cc scal, wl, twl, sig;
  T par;
};

template <typename T>
__device__ __forceinline__ LineValues<T, typename cpx<T>::type> line_values(int step, const Solve2DArgs& a,
                                                                            int64_t lc, const void* consts) {
  using C = typename cpx<T>::type;
  LineValues<T, C> v;
  if (consts) {
    const LineConst<C> t = line_const<C>(consts, a.n1);
    v.co.a = t.a[lc];
    v.co.ac = t.ac[lc];
    v.co.b = t.b[lc];
    v.scal = t.scal[lc];
    v.wl = t.wl[lc];
    v.twl = t.twl[lc];
    v.sig = t.sig[lc];
    v.par = t.par[lc].x;
    return v;
  }
  const LineParams lp = line_params(step, a, lc);
  v.co = line_coef<C>(lp.sre, lp.sim, a.hx, a.wx, a.mden);
  v.scal = (step == 2) ? mk<C>(1, 0) : mk<C>(a.invmu[2 * lc], a.invmu[2 * lc + 1]);
  v.wl = step3_weight<C>(a, lc);
  v.twl = mk<C>(a.tw[2 * lc], a.tw[2 * lc + 1]);
  v.sig = mk<C>(a.sigA[2 * lc], a.sigA[2 * lc + 1]);
  v.par = (T)a.parA[lc];
  return v;
}

template <typename T>
__global__ void k_line_consts(typename cpx<T>::type* __restrict__ out, Solve2DArgs a, int step) {
  using C = typename cpx<T>::type;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= a.n1) return;
  const LineValues<T, C> v = line_values<T>(step, a, l, nullptr);
  const int64_t n1 = a.n1;
  out[l] = v.co.a;
  out[n1 + l] = v.co.ac;
  out[2 * n1 + l] = v.co.b;
  out[3 * n1 + l] = v.scal;
  out[4 * n1 + l] = v.wl;
  out[5 * n1 + l] = v.twl;
  out[6 * n1 + l] = v.sig;
  out[7 * n1 + l] = mk<C>((double)v.par, 0);
}

template <typename T, int STEP, int CH>
__global__ void __launch_bounds__(128) k_tri_pass1(const typename cpx<T>::type* __restrict__ fhat,
                                                   const typename cpx<T>::type* __restrict__ faces,
                                                   const typename cpx<T>::type* __restrict__ ustart,
                                                   RecSoA<typename cpx<T>::type> rec, Solve2DArgs a,
                                                   const void* __restrict__ consts, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n1) return;
  const int64_t k = blockIdx.y;
  const int64_t s = k * CH, e = min(s + (int64_t)CH, nx) - 1;
  const int cnt = (int)(e - s + 1);
  const LineValues<T, C> lv = line_values<T>(STEP, a, l, consts);
  const LineCoef<C> co = lv.co;
  const C scal = lv.scal;
  const C wl = lv.wl;
  const T par = lv.par;
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
  const int64_t i = k * n1 + l;
  rec.a[i] = ylo;
  rec.bsum[i] = bsum;
  rec.pe[i] = (k > 0) ? P : zero;
  rec.cc[i] = (k > 0) ? cc : zero;
  rec.we[i] = cmul(mb, w);  // q = -b we
}

// Two scans per line over its chunks: forward carry Y, backward carry X.
// Overwrites rec.a[k] with Y(k-1) and rec.bsum[k] with X(k+1).
//
// Each chunk's carry step is an affine map: Y(k) = a_k + pe_k Y(k-1) forward,
// X(k) = c_k + q_k X(k+1) backward with c_k = bsum_k + cc_k Y(k-1) and
// q_k = -b we_k (stored in rec.we).  A block takes kCarryLines lines (one per
// x thread, so every load of a field is a contiguous run of lines) and splits
// their chunks into kCarrySeg contiguous segments (one per y thread).  Each
// thread composes the maps of its segment, the segment maps are folded in
// shared memory to give each segment its incoming carry, and each thread then
// runs its segment's recurrence from that carry.  Same recurrences as the
// sequential scan, regrouped once, in the precision of the records.
constexpr int kCarryLines = 16;
constexpr int kCarrySeg = 32;
// chunk records loaded ahead of each recurrence; complex64 takes half as many
// so that two blocks fit on an SM (every block of a 4096-line solve resident)
template <typename T>
__host__ __device__ constexpr int carry_batch() {
  return sizeof(T) == 4 ? 4 : 8;
}

template <typename T>
__global__ void __launch_bounds__(kCarryLines* kCarrySeg, sizeof(T) == 4 ? 2 : 1)
    k_tri_carry(RecSoA<typename cpx<T>::type> rec, int64_t n1, int64_t K, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  constexpr int B = carry_batch<T>();
  if (skip && *skip) return;  // uniform over the grid
  __shared__ C shC[kCarrySeg][kCarryLines], shP[kCarrySeg][kCarryLines];
  const int lx = threadIdx.x, sg = threadIdx.y;
  const int64_t l = (int64_t)blockIdx.x * kCarryLines + lx;
  const bool act = l < n1;
  const int64_t S = (K + kCarrySeg - 1) / kCarrySeg;
  const int64_t k0 = min(K, sg * S), k1 = min(K, k0 + S);
  const C one = mk<C>(1, 0), zero = mk<C>(0, 0);
  // forward: compose the segment's maps
  C A = zero, P = one;
  if (act)
    for (int64_t kb = k0; kb < k1; kb += B) {
      C av[B], pv[B];
#pragma unroll
      for (int t = 0; t < B; ++t)
        if (kb + t < k1) {
          av[t] = rec.a[(kb + t) * n1 + l];
          pv[t] = rec.pe[(kb + t) * n1 + l];
        }
#pragma unroll
      for (int t = 0; t < B; ++t)
        if (kb + t < k1) {
          const C pk = pv[t];
          A = cadd(av[t], cmul(pk, A));
          P = cmul(pk, P);
        }
    }
  shC[sg][lx] = A;
  shP[sg][lx] = P;
  __syncthreads();
  C Y = zero;
  for (int g = 0; g < sg; ++g) Y = cadd(shC[g][lx], cmul(shP[g][lx], Y));
  // forward recurrence; c_k replaces bsum_k
  if (act)
    for (int64_t kb = k0; kb < k1; kb += B) {
      C av[B], pv[B], bv[B], cv[B];
#pragma unroll
      for (int t = 0; t < B; ++t)
        if (kb + t < k1) {
          const int64_t i = (kb + t) * n1 + l;
          av[t] = rec.a[i];
          pv[t] = rec.pe[i];
          bv[t] = rec.bsum[i];
          cv[t] = rec.cc[i];
        }
#pragma unroll
      for (int t = 0; t < B; ++t)
        if (kb + t < k1) {
          const int64_t i = (kb + t) * n1 + l;
          rec.a[i] = Y;  // Y(k-1)
          rec.bsum[i] = cadd(bv[t], cmul(cv[t], Y));
          Y = cadd(av[t], cmul(pv[t], Y));
        }
    }
  __syncthreads();
  // backward: compose the segment's maps, last chunk first
  C Cs = zero, Q = one;
  if (act)
    for (int64_t kb = k1 - 1; kb >= k0; kb -= B) {
      C cv[B], qv[B];
#pragma unroll
      for (int t = 0; t < B; ++t)
        if (kb - t >= k0) {
          cv[t] = rec.bsum[(kb - t) * n1 + l];
          qv[t] = rec.we[(kb - t) * n1 + l];
        }
#pragma unroll
      for (int t = 0; t < B; ++t)
        if (kb - t >= k0) {
          const C qk = qv[t];
          Cs = cadd(cv[t], cmul(qk, Cs));
          Q = cmul(qk, Q);
        }
    }
  shC[sg][lx] = Cs;
  shP[sg][lx] = Q;
  __syncthreads();
  C X = zero;
  for (int g = kCarrySeg - 1; g > sg; --g) X = cadd(shC[g][lx], cmul(shP[g][lx], X));
  if (act)
    for (int64_t kb = k1 - 1; kb >= k0; kb -= B) {
      C cv[B], qv[B];
#pragma unroll
      for (int t = 0; t < B; ++t)
        if (kb - t >= k0) {
          cv[t] = rec.bsum[(kb - t) * n1 + l];
          qv[t] = rec.we[(kb - t) * n1 + l];
        }
#pragma unroll
      for (int t = 0; t < B; ++t)
        if (kb - t >= k0) {
          rec.bsum[(kb - t) * n1 + l] = X;  // X(k+1)
          X = cadd(cv[t], cmul(qv[t], X));
        }
    }
}

// Sum the face contributions of a block's 128 lines for each of its `cnt`
// rows (red[face][row][thread]) and write one partial per block and row:
// partial[(face * nparts + blk) * nx + row0 + t].  Fixed summation order.
template <typename C, int CH>
__device__ __forceinline__ void block_face_sums(C* red, int cnt, C* __restrict__ partial, int64_t blk,
                                                int64_t nparts, int64_t nx, int64_t row0) {
  constexpr int NQ = 2 * CH;    // sums: face * CH + row
  constexpr int SP = NQ + 1;    // padded stride of the segment sums
  __shared__ C seg[16 * SP];
  __syncthreads();
  // stage 1: thread -> (sum q, segment g of 8 consecutive lines, lines g, g+16,
  // ..., g+112); a half-warp reads 16 consecutive values (no bank conflicts)
  for (int w = threadIdx.x; w < NQ * 16; w += blockDim.x) {
    const int q = w >> 4, g = w & 15;
    const C* src = red + q * 128 + g;
    C acc = src[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) acc = cadd(acc, src[16 * i]);
    seg[g * SP + q] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
    const int face = q / CH, t = q - face * CH;
    if (t >= cnt) continue;
    C acc = seg[q];
#pragma unroll
    for (int g = 1; g < 16; ++g) acc = cadd(acc, seg[g * SP + q]);
    partial[(face * nparts + blk) * nx + row0 + t] = acc;
  }
}

// Pass 2: Thomas inside each chunk from the exact carries; emit x.
template <typename T, int STEP, int CH>
__global__ void __launch_bounds__(128) k_tri_pass2(const typename cpx<T>::type* __restrict__ fhat,
                                                   const typename cpx<T>::type* __restrict__ faces,
                                                   const typename cpx<T>::type* __restrict__ ustart,
                                                   RecSoA<typename cpx<T>::type> rec,
                                                   typename cpx<T>::type* __restrict__ out,
                                                   typename cpx<T>::type* __restrict__ partial, Solve2DArgs a,
                                                   const void* __restrict__ consts, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (STEP == 3 && (l & ~(int64_t)31) >= n1) return;  // no block sync in Step 3
  const bool act = l < n1;
  const int64_t lc = act ? l : 0;
  const int64_t k = blockIdx.y;
  const int64_t s = k * CH, e = min(s + CH, nx) - 1;
  const int cnt = (int)(e - s + 1);
  const LineValues<T, C> lv = line_values<T>(STEP, a, lc, consts);
  const LineCoef<C> co = lv.co;
  const C scal = lv.scal;
  const C twl = lv.twl;
  const C wl = lv.wl;
  const T par = lv.par;
  const C sig = lv.sig;
  const C* f1 = faces;
  const C* fn = faces + nx;
  const C zero = mk<C>(0, 0);
  C y[CH], iu[CH];
  const C Yin = rec.a[k * n1 + lc];     // Y(k-1)
  const C Xin = rec.bsum[k * n1 + lc];  // X(k+1)
  C inv = (k > 0) ? crecip(ustart[k * n1 + lc]) : zero;
  C yp = Yin;
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
  // face contributions of the block's 128 lines, reduced per row in shared memory
  __shared__ C red[2 * CH * 128];
  const int64_t nparts = (n1 + 127) / 128;
  C xn = Xin;
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
        red[(0 * CH + t) * 128 + threadIdx.x] = s1;
        red[(1 * CH + t) * 128 + threadIdx.x] = sn;
      }
    }
  }
  if (STEP != 3) block_face_sums<C, CH>(red, cnt, partial, (int64_t)blockIdx.x, nparts, nx, s);
}

// ---------------------------------------------------------------------------
// FP64 path with per-plan tables.  Everything in the chunked Thomas that does
// not depend on the right-hand side is computed once per plan: for every line
// and row the multiplier m_j = b/u_{j-1}, the reciprocal pivot 1/u_j and the
// weight w_j = (U_kk^-1)_{s,j}; for every chunk pe, cc, we.  Each solve then
// does only the two recurrences that involve the data.
// ---------------------------------------------------------------------------
struct LineTables {
  double2* m;
  double2* iu;
  double2* w;
  double2* pe;
  double2* cc;
  double2* we;
};

inline LineTables line_tables(void* base, size_t N, size_t nrec) {
  double2* b = reinterpret_cast<double2*>(base);
  return LineTables{b, b + N, b + 2 * N, b + 3 * N, b + 3 * N + nrec, b + 3 * N + 2 * nrec};
}

__global__ void k_line_tables(LineTables t, Solve2DArgs a, int step) {
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n1) return;
  const LineParams lp = line_params(step, a, l);
  const LineCoef<double2> co = line_coef<double2>(lp.sre, lp.sim, a.hx, a.wx, a.mden);
  const double2 zero = make_double2(0, 0);
  const double2 mb = make_double2(-co.b.x, -co.b.y);
  // limit of the pivots and the settling row of this line
  const double2 disc = csqrt_d(csub(cmul(co.a, co.a), cscale(cmul(co.b, co.b), 4.0)));
  const double2 r1 = cscale(cadd(co.a, disc), 0.5), r2 = cscale(csub(co.a, disc), 0.5);
  const double2 iinf = crecip((r1.x * r1.x + r1.y * r1.y >= r2.x * r2.x + r2.y * r2.y) ? r1 : r2);
  const double tol = 7.450580596923828e-09;  // 2^-27
  const double tol2 = tol * tol * (iinf.x * iinf.x + iinf.y * iinf.y);
  int64_t last_bad = -1;
  double2 iu = zero, P = zero, w = zero, cc = zero;
  for (int64_t j = 0; j < nx; ++j) {
    const int64_t k = j / a.ch, s = k * a.ch;
    const double2 aj = (j == 0 || j == nx - 1) ? co.ac : co.a;
    double2 m = zero, u;
    if (j > 0) {
      m = cmul(co.b, iu);
      u = csub(aj, cmul(m, co.b));
    } else {
      u = aj;
    }
    iu = crecip(u);
    const double2 mm = make_double2(-m.x, -m.y);
    P = (j == s) ? mm : cmul(P, mm);
    w = (j == s) ? iu : cmul(cmul(w, mb), iu);
    cc = (j == s) ? cmul(w, P) : cadd(cc, cmul(w, P));
    t.m[j * n1 + l] = m;
    t.iu[j * n1 + l] = iu;
    t.w[j * n1 + l] = w;
    if (j == min(s + a.ch, nx) - 1) {
      t.pe[k * n1 + l] = (k > 0) ? P : zero;
      t.cc[k * n1 + l] = (k > 0) ? cc : zero;
      t.we[k * n1 + l] = cmul(mb, w);  // q = -b we
    }
  }
}

template <int STEP, int CH>
__global__ void __launch_bounds__(128) k_tri_pass1_tab(const double2* __restrict__ fhat,
                                                       const double2* __restrict__ faces, LineTables tb,
                                                       RecSoA<double2> rec, Solve2DArgs a,
                                                       const int* __restrict__ skip) {
  using C = double2;
  if (skip && *skip) return;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n1) return;
  const int64_t k = blockIdx.y;
  const int64_t s = k * CH, e = min(s + (int64_t)CH, nx) - 1;
  const int cnt = (int)(e - s + 1);
  const C scal = (STEP == 2) ? mk<C>(1, 0) : mk<C>(a.invmu[2 * l], a.invmu[2 * l + 1]);
  const C wl = step3_weight<C>(a, l);
  const double par = a.parA[l];
  const C* f1 = faces;
  const C* fn = faces + nx;
  C rr[CH], mj[CH], wj[CH];
#pragma unroll
  for (int t = 0; t < CH; ++t)
    if (t < cnt) {
      const int64_t i = (s + t) * n1 + l;
      rr[t] = line_rhs<C>(STEP, s + t, l, n1, fhat, f1, fn, scal, par, wl);
      mj[t] = tb.m[i];
      wj[t] = tb.w[i];
    }
  C ylo = make_double2(0, 0), bsum = make_double2(0, 0);
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    if (t >= cnt) break;
    ylo = (t == 0) ? rr[t] : csub(rr[t], cmul(mj[t], ylo));
    bsum = cadd(bsum, cmul(wj[t], ylo));
  }
  rec.a[k * n1 + l] = ylo;
  rec.bsum[k * n1 + l] = bsum;
}

template <int STEP, int CH>
__global__ void __launch_bounds__(128) k_tri_pass2_tab(const double2* __restrict__ fhat,
                                                       const double2* __restrict__ faces, LineTables tb,
                                                       RecSoA<double2> rec, double2* __restrict__ out,
                                                       double2* __restrict__ partial, Solve2DArgs a,
                                                       const int* __restrict__ skip) {
  using C = double2;
  if (skip && *skip) return;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (STEP == 3 && (l & ~(int64_t)31) >= n1) return;  // no block sync in Step 3
  const bool act = l < n1;
  const int64_t lc = act ? l : 0;
  const int64_t k = blockIdx.y;
  const int64_t s = k * CH, e = min(s + (int64_t)CH, nx) - 1;
  const int cnt = (int)(e - s + 1);
  const LineParams lp = line_params(STEP, a, lc);
  const LineCoef<C> co = line_coef<C>(lp.sre, lp.sim, a.hx, a.wx, a.mden);
  const C scal = (STEP == 2) ? mk<C>(1, 0) : mk<C>(a.invmu[2 * lc], a.invmu[2 * lc + 1]);
  const C twl = mk<C>(a.tw[2 * lc], a.tw[2 * lc + 1]);
  const C wl = step3_weight<C>(a, lc);
  const double par = a.parA[lc];
  const C sig = mk<C>(a.sigA[2 * lc], a.sigA[2 * lc + 1]);
  const C* f1 = faces;
  const C* fn = faces + nx;
  const C zero = mk<C>(0, 0);
  C y[CH], mj[CH], iu[CH];
#pragma unroll
  for (int t = 0; t < CH; ++t)
    if (t < cnt) {
      const int64_t i = (s + t) * n1 + lc;
      y[t] = line_rhs<C>(STEP, s + t, lc, n1, fhat, f1, fn, scal, par, wl);
      mj[t] = tb.m[i];
      iu[t] = tb.iu[i];
    }
  C yp = rec.a[k * n1 + lc];  // Y(k-1)
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    if (t < cnt) {
      yp = csub(y[t], cmul(mj[t], yp));
      y[t] = yp;
    }
  }
  // face contributions of the block's 128 lines, reduced per row in shared memory
  __shared__ C red[2 * CH * 128];
  const int64_t nparts = (n1 + 127) / 128;
  C xn = rec.bsum[k * n1 + lc];  // X(k+1)
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
        red[(0 * CH + t) * 128 + threadIdx.x] = s1;
        red[(1 * CH + t) * 128 + threadIdx.x] = sn;
      }
    }
  }
  if (STEP != 3) block_face_sums<C, CH>(red, cnt, partial, (int64_t)blockIdx.x, nparts, nx, s);
}

// ---------------------------------------------------------------------------
// complex64 path with a per-plan pivot table.  The reciprocal pivots 1/u_j of
// every line are computed once per plan in FP64 and stored rounded to FP32
// (8 bytes per unknown and line type), with the chunk constants pe, cc and
// q = -b we.  The solves rebuild the multipliers m_j = b / u_{j-1} and the
// chunk weights w_j from the table with one complex multiply each, so no
// division is left in the recurrences.
// ---------------------------------------------------------------------------
// Lines per CTA and chunks per CTA of the bulk-copy fed tridiagonal kernels.
constexpr int kBulkLines = 128;
constexpr int kBulkChunks = 8;

// iinf: per line 1/u_inf, the limit of the pivots (u_inf the root of
// u^2 - a u + b^2 = 0 of larger modulus); lcta: per block of kBulkLines
// lines, the first row from which every line's 1/u_j (below the last row)
// is within 2^-27 |1/u_inf| of it, so the bulk kernels read no table rows
// for chunks past it (propagating modes never settle: their blocks read the
// whole table).
struct LineTables32 {
  float2* iu;
  float2* pe;
  float2* cc;
  float2* we;
  float2* iinf;
  int* lcta;
};

inline LineTables32 line_tables32(void* base, size_t N, size_t nrec, size_t n1) {
  float2* b = reinterpret_cast<float2*>(base);
  float2* ii = b + N + 3 * nrec;
  return LineTables32{b, b + N, b + N + nrec, b + N + 2 * nrec, ii, reinterpret_cast<int*>(ii + n1)};
}

__global__ void k_line_tables32(LineTables32 t, Solve2DArgs a, int step) {
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n1) return;
  const LineParams lp = line_params(step, a, l);
  const LineCoef<double2> co = line_coef<double2>(lp.sre, lp.sim, a.hx, a.wx, a.mden);
  const double2 zero = make_double2(0, 0);
  const double2 mb = make_double2(-co.b.x, -co.b.y);
  // limit of the pivots and the settling row of this line
  const double2 disc = csqrt_d(csub(cmul(co.a, co.a), cscale(cmul(co.b, co.b), 4.0)));
  const double2 r1 = cscale(cadd(co.a, disc), 0.5), r2 = cscale(csub(co.a, disc), 0.5);
  const double2 iinf = crecip((r1.x * r1.x + r1.y * r1.y >= r2.x * r2.x + r2.y * r2.y) ? r1 : r2);
  const double tol = 7.450580596923828e-09;  // 2^-27
  const double tol2 = tol * tol * (iinf.x * iinf.x + iinf.y * iinf.y);
  int64_t last_bad = -1;
  double2 iu = zero, P = zero, w = zero, cc = zero;
  for (int64_t j = 0; j < nx; ++j) {
    const int64_t k = j / a.ch, s = k * a.ch;
    const double2 aj = (j == 0 || j == nx - 1) ? co.ac : co.a;
    double2 m = zero, u;
    if (j > 0) {
      m = cmul(co.b, iu);
      u = csub(aj, cmul(m, co.b));
    } else {
      u = aj;
    }
    iu = crecip(u);
    const double2 mm = make_double2(-m.x, -m.y);
    P = (j == s) ? mm : cmul(P, mm);
    w = (j == s) ? iu : cmul(cmul(w, mb), iu);
    cc = (j == s) ? cmul(w, P) : cadd(cc, cmul(w, P));
    t.iu[j * n1 + l] = cvt<float2>(iu);
    if (j < nx - 1) {
      const double dx = iu.x - iinf.x, dy = iu.y - iinf.y;
      if (!(dx * dx + dy * dy <= tol2)) last_bad = j;
    }
    if (j == min(s + a.ch, nx) - 1) {
      t.pe[k * n1 + l] = cvt<float2>((k > 0) ? P : zero);
      t.cc[k * n1 + l] = cvt<float2>((k > 0) ? cc : zero);
      t.we[k * n1 + l] = cvt<float2>(cmul(mb, w));  // q = -b we
    }
  }
  t.iinf[l] = cvt<float2>(iinf);
  atomicMax(&t.lcta[l / kBulkLines], (int)(last_bad + 1));
}

template <int STEP, int CH>
__global__ void __launch_bounds__(128) k_tri_pass1_t32(const float2* __restrict__ fhat, const float2* __restrict__ faces,
                                                       LineTables32 tb, RecSoA<float2> rec, Solve2DArgs a,
                                                       const void* __restrict__ consts, const int* __restrict__ skip) {
  using C = float2;
  if (skip && *skip) return;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n1) return;
  const int64_t k = blockIdx.y;
  const int64_t s = k * CH, e = min(s + (int64_t)CH, nx) - 1;
  const int cnt = (int)(e - s + 1);
  const LineValues<float, C> lv = line_values<float>(STEP, a, l, consts);
  const C b = lv.co.b, mb = mk<C>(-b.x, -b.y);
  const C* f1 = faces;
  const C* fn = faces + nx;
  C rr[CH], iu[CH];
#pragma unroll
  for (int t = 0; t < CH; ++t)
    if (t < cnt) {
      rr[t] = line_rhs<C>(STEP, s + t, l, n1, fhat, f1, fn, lv.scal, lv.par, lv.wl);
      iu[t] = tb.iu[(s + t) * n1 + l];
    }
  C ylo = rr[0], w = iu[0];
  C bsum = cmul(w, ylo);
#pragma unroll
  for (int t = 1; t < CH; ++t) {
    if (t >= cnt) break;
    const C m = cmul(b, iu[t - 1]);
    ylo = csub(rr[t], cmul(m, ylo));
    w = cmul(cmul(w, mb), iu[t]);
    bsum = cadd(bsum, cmul(w, ylo));
  }
  rec.a[k * n1 + l] = ylo;
  rec.bsum[k * n1 + l] = bsum;
}

template <int STEP, int CH>
__global__ void __launch_bounds__(128) k_tri_pass2_t32(const float2* __restrict__ fhat, const float2* __restrict__ faces,
                                                       LineTables32 tb, RecSoA<float2> rec, float2* __restrict__ out,
                                                       float2* __restrict__ partial, Solve2DArgs a,
                                                       const void* __restrict__ consts, const int* __restrict__ skip) {
  using C = float2;
  if (skip && *skip) return;
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (STEP == 3 && (l & ~(int64_t)31) >= n1) return;  // no block sync in Step 3
  const bool act = l < n1;
  const int64_t lc = act ? l : 0;
  const int64_t k = blockIdx.y;
  const int64_t s = k * CH, e = min(s + (int64_t)CH, nx) - 1;
  const int cnt = (int)(e - s + 1);
  const LineValues<float, C> lv = line_values<float>(STEP, a, lc, consts);
  const C b = lv.co.b;
  const C* f1 = faces;
  const C* fn = faces + nx;
  const C zero = mk<C>(0, 0);
  C y[CH], iu[CH];
#pragma unroll
  for (int t = 0; t < CH; ++t)
    if (t < cnt) {
      y[t] = line_rhs<C>(STEP, s + t, lc, n1, fhat, f1, fn, lv.scal, lv.par, lv.wl);
      iu[t] = tb.iu[(s + t) * n1 + lc];
    }
  C iprev = (s > 0) ? tb.iu[(s - 1) * n1 + lc] : zero;  // 1/u_{s-1}
  C yp = rec.a[k * n1 + lc];                               // Y(k-1)
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    if (t < cnt) {
      yp = csub(y[t], cmul(cmul(b, iprev), yp));
      y[t] = yp;
      iprev = iu[t];
    }
  }
  __shared__ C red[2 * CH * 128];
  const int64_t nparts = (n1 + 127) / 128;
  C xn = rec.bsum[k * n1 + lc];  // X(k+1)
#pragma unroll
  for (int t = CH - 1; t >= 0; --t) {
    if (t < cnt) {
      const int64_t j = s + t;
      const C x = cmul(csub(y[t], cmul(b, xn)), iu[t]);
      xn = x;
      if (STEP == 3) {
        if (act) out[j * n1 + lc] = x;
      } else {
        C s1, sn;
        if (STEP == 1) {
          s1 = act ? x : zero;
          sn = act ? cmul(x, lv.twl) : zero;
        } else {
          const C tt = act ? cmul(x, lv.sig) : zero;
          s1 = tt;
          sn = cscale(tt, lv.par);
        }
        red[(0 * CH + t) * 128 + threadIdx.x] = s1;
        red[(1 * CH + t) * 128 + threadIdx.x] = sn;
      }
    }
  }
  if (STEP != 3) block_face_sums<C, CH>(red, cnt, partial, (int64_t)blockIdx.x, nparts, nx, s);
}

// ---------------------------------------------------------------------------
// complex64 chunk passes fed by bulk copies.  A CTA owns 128 consecutive lines
// and a run of kBulkChunks consecutive chunks.  Its tiles (the chunk's rows of
// f_hat and of the pivot table, 1 KB per row and array) arrive in shared
// memory by cp.async.bulk into two buffers: while the CTA computes chunk k,
// the copies of chunk k+1 are in flight, so the memory system is kept busy
// without holding the tiles in registers.  Same arithmetic as
// k_tri_pass1_t32 / k_tri_pass2_t32.  Needs 16-byte aligned rows (even n1).
// ---------------------------------------------------------------------------

// Tile of one buffer, per kernel instance: [f_hat rows (Steps 1, 3)][1/u
// rows][face values f1 (CH) and fn (CH + 2, from the even index at or before
// nx + s: 16-byte aligned sources)][carries Y(k-1), X(k+1) of the block's
// lines (pass 2)].  Offsets and the buffer size are whole 128-byte rows: a
// warp's 32 consecutive values then take the minimum two shared-memory
// wavefronts.
__host__ __device__ constexpr int bulk_round16(int v) { return (v + 15) & ~15; }
template <int STEP, int CH>
__host__ __device__ constexpr int bulk_iu_offset() {
  return STEP != 2 ? CH * kBulkLines : 0;
}
template <int STEP, int CH>
__host__ __device__ constexpr int bulk_face_offset() {
  return bulk_iu_offset<STEP, CH>() + CH * kBulkLines;
}
template <int STEP, int CH>
__host__ __device__ constexpr int bulk_carry_offset() {
  return bulk_round16(bulk_face_offset<STEP, CH>() + 2 * CH + 2);
}
template <int PASS, int STEP, int CH>
__host__ __device__ constexpr int bulk_tile_values() {
  return bulk_round16(bulk_carry_offset<STEP, CH>() + (PASS == 2 ? 2 * kBulkLines : 0));
}
template <int PASS, int STEP, int CH>
constexpr size_t bulk_tile_bytes() {
  return (size_t)2 * bulk_tile_values<PASS, STEP, CH>() * sizeof(float2);  // two buffers
}

// Sum over the 32 lanes of a warp of NQ = 32 complex values per lane by
// recursive halving: at each level a lane keeps the half of its values chosen
// by one bit of its lane index and adds the partner's copy of that half;
// afterwards lane q holds the warp's sum of v[q].  Fixed summation order.
template <int NQ>
__device__ __forceinline__ float2 warp_transpose_sum(float2 (&v)[NQ], int lane) {
  static_assert(NQ == 32, "one sum per lane");
#pragma unroll
  for (int n = NQ, off = 16; off >= 1; n >>= 1, off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const float2 keep = upper ? v[i + n / 2] : v[i];
      const float2 send = upper ? v[i] : v[i + n / 2];
      v[i].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, off);
      v[i].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, off);
    }
  }
  return v[0];
}

template <int PASS, int STEP, int CH>
__global__ void __launch_bounds__(kBulkLines) k_tri_bulk_t32(const float2* __restrict__ fhat,
                                                             const float2* __restrict__ faces, LineTables32 tb,
                                                             RecSoA<float2> rec, float2* __restrict__ out,
                                                             float2* __restrict__ partial, Solve2DArgs a,
                                                             const void* __restrict__ consts,
                                                             const int* __restrict__ skip, int* __restrict__ err) {
  using C = float2;
  constexpr int TILE = bulk_tile_values<PASS, STEP, CH>();  // values per buffer
  constexpr int IU = bulk_iu_offset<STEP, CH>();
  constexpr int FO = bulk_face_offset<STEP, CH>();
  constexpr int CO = bulk_carry_offset<STEP, CH>();
  constexpr bool SUMS = PASS == 2 && STEP != 3;  // face contributions reduced per block
  static_assert(!SUMS || 2 * CH == 32, "one face sum per lane");
  constexpr bool RHS = STEP != 2;               // Step 2 takes its rhs from the face vectors
  constexpr bool FACES = STEP != 1;             // Steps 2, 3 read the face vectors f1, fn
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* const tile = reinterpret_cast<C*>(smem_raw);
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ C wpart[SUMS ? kBulkLines : 1];  // [warp][quantity] warp sums of the face contributions
  const int64_t n1 = a.n1, nx = a.nx;
  const int64_t l0 = (int64_t)blockIdx.x * kBulkLines;
  const int nl = (int)min((int64_t)kBulkLines, n1 - l0);
  const int64_t kb = (int64_t)blockIdx.y * kBulkChunks, ke = min(kb + (int64_t)kBulkChunks, a.nchunks);
  const int tid = threadIdx.x;
  const bool act = tid < nl;
  const int64_t l = l0 + (act ? tid : 0);
  // chunks from row lset on (except the one holding the last row) use each
  // line's 1/u_inf: their table rows are not copied
  const int64_t lset = tb.lcta[blockIdx.x];
  auto settled = [&](int64_t k) { return k * CH >= lset && min((k + 1) * CH, nx) < nx; };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // thread 0: the copies of chunk k into buffer bsel
  auto issue = [&](int64_t k, int bsel) {
    const int64_t s = k * CH;
    const int cnt = (int)min((int64_t)CH, nx - s);
    const uint32_t row_bytes = (uint32_t)nl * (uint32_t)sizeof(C);
    // face values f1[s, s+cnt) and fn[s, s+cnt) = faces[nx+s, nx+s+cnt),
    // each widened to whole 16-byte pairs: f1 from s (even), fn from the even
    // index at or before nx + s; the widened ends stay inside [0, 2 nx)
    const int64_t fa = (nx + s) & ~(int64_t)1;
    const uint32_t n_f1 = (uint32_t)((cnt + 1) & ~1);
    const uint32_t n_fn = (uint32_t)((((nx + s + cnt + 1) & ~(int64_t)1)) - fa);
    const uint32_t face_bytes = FACES ? (n_f1 + n_fn) * (uint32_t)sizeof(C) : 0u;
    const uint32_t carry_bytes = PASS == 2 ? 2u * row_bytes : 0u;
    const bool tab = !settled(k);
    mbar_arrive_expect_tx(&bar[bsel],
                          (uint32_t)cnt * row_bytes * ((RHS ? 1u : 0u) + (tab ? 1u : 0u)) + face_bytes + carry_bytes);
    C* buf = tile + bsel * TILE;
    for (int t = 0; t < cnt; ++t) {
      if (RHS) bulk_g2s(buf + t * kBulkLines, fhat + (s + t) * n1 + l0, row_bytes, &bar[bsel]);
      if (tab) bulk_g2s(buf + IU + t * kBulkLines, tb.iu + (s + t) * n1 + l0, row_bytes, &bar[bsel]);
    }
    if (FACES) {
      C* fb = buf + FO;
      bulk_g2s(fb, faces + s, n_f1 * (uint32_t)sizeof(C), &bar[bsel]);
      bulk_g2s(fb + CH, faces + fa, n_fn * (uint32_t)sizeof(C), &bar[bsel]);
    }
    if (PASS == 2) {
      C* cb = buf + CO;
      bulk_g2s(cb, rec.a + k * n1 + l0, row_bytes, &bar[bsel]);
      bulk_g2s(cb + kBulkLines, rec.bsum + k * n1 + l0, row_bytes, &bar[bsel]);
    }
  };
  // thread 0's book of copies in flight: bit b of `pending` (buffer b busy),
  // bit b of `want` (parity of its phase)
  uint32_t pending = 0, want = 0;
  if (tid == 0) {
    issue(kb, 0);
    pending |= 1u;
    if (kb + 1 < ke) {
      issue(kb + 1, 1);
      pending |= 2u;
    }
  }
  const LineValues<float, C> lv = line_values<float>(STEP, a, l, consts);
  const C b = lv.co.b, mb = mk<C>(-b.x, -b.y);
  const C iinf = tb.iinf[l];
  const C zero = mk<C>(0, 0);
  const int64_t nparts = (n1 + kBulkLines - 1) / kBulkLines;
  C iprev = (PASS == 2 && kb > 0) ? tb.iu[(kb * CH - 1) * n1 + l] : zero;  // 1/u of the row before the run
  bool failed = false;
  for (int64_t k = kb; k < ke; ++k) {
    const int bsel = (int)((k - kb) & 1);
    const uint32_t parity = (uint32_t)(((k - kb) >> 1) & 1);
    const int64_t s = k * CH;
    const int cnt = (int)min((int64_t)CH, nx - s);
    const bool got = mbar_wait_bounded(&bar[bsel], parity, err);
    if (__syncthreads_or(!got)) {  // block-uniform decision
      failed = true;
      break;
    }
    if (tid == 0) pending &= ~(1u << bsel);
    const C* const frow = tile + bsel * TILE;  // [CH][128] f_hat rows (Steps 1, 3)
    const C* const irow = frow + IU;           // [CH][128] 1/u rows (not copied for a settled chunk)
    const bool set = settled(k);                 // block-uniform
    auto piv = [&](int t) -> C { return set ? iinf : irow[t * kBulkLines + tid]; };
    const C* const sf1 = frow + FO;            // f1[s + t]
    const C* const sfn = sf1 + CH + (int)((nx + s) & 1);  // fn[s + t]
    C yp = zero, xn = zero;
    if (PASS == 2) {
      yp = frow[CO + tid];               // Y(k-1)
      xn = frow[CO + kBulkLines + tid];  // X(k+1)
    }
    auto rhs = [&](int t) -> C {
      if (STEP == 1) return cmul(frow[t * kBulkLines + tid], lv.scal);
      if (STEP == 2) return cadd(sf1[t], cscale(sfn[t], lv.par));
      C v = cadd(frow[t * kBulkLines + tid], sf1[t]);
      v = cadd(v, cmul(sfn[t], lv.wl));
      return cmul(v, lv.scal);
    };
    if (PASS == 1) {
      C ylo = rhs(0), w = piv(0);
      C bsum = cmul(w, ylo);
#pragma unroll
      for (int t = 1; t < CH; ++t) {
        if (t >= cnt) break;
        const C m = cmul(b, piv(t - 1));
        ylo = csub(rhs(t), cmul(m, ylo));
        w = cmul(cmul(w, mb), piv(t));
        bsum = cadd(bsum, cmul(w, ylo));
      }
      if (act) {
        rec.a[k * n1 + l] = ylo;
        rec.bsum[k * n1 + l] = bsum;
      }
    } else {
      C y[CH];
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        if (t < cnt) {
          yp = csub(rhs(t), cmul(cmul(b, iprev), yp));
          y[t] = yp;
          iprev = piv(t);
        }
      }
      // backward sweep; Steps 1, 2 keep their face contributions in
      // registers (sv[face * CH + row]) for the warp sums
      C sv[SUMS ? 2 * CH : 1];
#pragma unroll
      for (int t = CH - 1; t >= 0; --t) {
        if (t < cnt) {
          const C x = cmul(csub(y[t], cmul(b, xn)), piv(t));
          xn = x;
          if constexpr (!SUMS) {
            if (act) out[(s + t) * n1 + l] = x;
          } else {
            C s1, sn;
            if (STEP == 1) {
              s1 = act ? x : zero;
              sn = act ? cmul(x, lv.twl) : zero;
            } else {
              const C tt = act ? cmul(x, lv.sig) : zero;
              s1 = tt;
              sn = cscale(tt, lv.par);
            }
            sv[t] = s1;
            sv[CH + t] = sn;
          }
        } else if constexpr (SUMS) {
          sv[t] = zero;
          sv[CH + t] = zero;
        }
      }
      if constexpr (SUMS) {
        // lane q of each warp: the warp's sum of quantity q = face * CH + row;
        // then thread q adds the four warps' sums in order
        const int lane = tid & 31, warp = tid >> 5;
        wpart[warp * 32 + lane] = warp_transpose_sum<2 * CH>(sv, lane);
        __syncthreads();  // also: every thread has finished with the tile
        if (tid < 2 * CH) {
          const int face = tid / CH, t = tid - face * CH;
          if (t < cnt) {
            C acc = wpart[tid];
#pragma unroll
            for (int w = 1; w < kBulkLines / 32; ++w) acc = cadd(acc, wpart[w * 32 + tid]);
            partial[(face * nparts + (int64_t)blockIdx.x) * nx + s + t] = acc;
          }
        }
      }
    }
    // the buffer is consumed: it may be refilled (in pass 2 of Steps 1, 2 the
    // barrier of the warp sums already follows the last read of the tile)
    if (!SUMS) __syncthreads();
    if (tid == 0 && k + 2 < ke) {
      issue(k + 2, bsel);
      pending |= 1u << bsel;
      want = (want & ~(1u << bsel)) | ((parity ^ 1u) << bsel);
    }
  }
  if (failed && tid == 0) {
    // let the copies still in flight land (bounded) before the CTA's shared
    // memory is released
    for (int bsel = 0; bsel < 2; ++bsel)
      if (pending & (1u << bsel)) mbar_wait_bounded(&bar[bsel], (want >> bsel) & 1u, nullptr);
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
  const LineCoef<double2> co = line_coef<double2>(lp.sre, lp.sim, a.hx, a.wx, a.mden);
  double2 u = co.ac;
  const double2 b2 = cmul(co.b, co.b);
  if ((a.ch - 1) == 0 && a.nchunks > 1) ustart[1 * n1 + l] = cvt<C>(u);
  for (int64_t j = 1; j < nx; ++j) {
    const double2 aj = (j == nx - 1) ? co.ac : co.a;
    u = csub(aj, cmul(b2, crecip(u)));
    if ((j + 1) % a.ch == 0 && (j + 1) / a.ch < a.nchunks) ustart[((j + 1) / a.ch) * n1 + l] = cvt<C>(u);
  }
}

// Sum the per-block partials: out[face * nx + ix] = scale * sum_w partial.
// Four lanes per output (lanes j, j+8, j+16, j+24 of a warp), each summing
// the partials w = q, q+4, ... (independent loads), combined by two fixed
// shuffles: a fixed summation order.
constexpr int kFaceLanes = 4;
template <typename T>
__global__ void __launch_bounds__(256) k_reduce_faces(const typename cpx<T>::type* __restrict__ partial,
                                                      typename cpx<T>::type* __restrict__ out, int64_t nx,
                                                      int64_t nwarps, double s0r, double s0i, double s1r,
                                                      double s1i, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31, q = lane >> 3;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / kFaceLanes + (lane & 7);
  const bool act = i < 2 * nx;
  const int64_t face = act ? i / nx : 0, ix = act ? i - face * nx : 0;
  C acc = mk<C>(0, 0);
  if (act) {
    const C* src = partial + (face * nwarps) * nx + ix;
#pragma unroll 8
    for (int64_t w = q; w < nwarps; w += kFaceLanes) acc = cadd(acc, src[w * nx]);
  }
  for (int off = 8; off < 32; off <<= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  if (act && q == 0) out[i] = cmul(acc, face == 0 ? mk<C>(s0r, s0i) : mk<C>(s1r, s1i));
}

// C_bb applied to the x1 faces (eqs. BminA, Cbb):
//   c_1 = D11 M v_1 + E11 K v_1 + D1n M v_n + E1n K v_n,  c_n symmetric,
// with D11 = (1 + i w h1)/h1 - p h1/3, D1n = -1/h1 - p h1/6, E11 = h1/3,
// E1n = h1/6 (p = w^2 for the outer problem), M, K along x (spacing hx,
// absorbing corners).  in = v (+ w if `in2`), out = c.
struct CbbConsts {
  double md_end, md_in, mo;        // M rows: diagonal (end, inner), off-diagonal
  double kd_end_re, kd_end_im;     // K diagonal at the absorbing ends
  double kd_in, ko;                // K diagonal inside, off-diagonal
  double d11_re, d11_im, d1n_re;   // D11, D1n (real)
  double e11, e1n;                 // E11, E1n
  double gr, gi, gir, gii;         // g and 1/g: wrap entries of the gamma-circulant
};

template <typename T>
__global__ void k_apply_cbb(const typename cpx<T>::type* __restrict__ in,
                            const typename cpx<T>::type* __restrict__ in2,
                            typename cpx<T>::type* __restrict__ out, int64_t nx, CbbConsts k,
                            const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  using R = decltype(C().x);
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
  const R md = (R)(end ? k.md_end : k.md_in), mo = (R)k.mo, ko = (R)k.ko;
  const C kd = end ? mk<C>(k.kd_end_re, k.kd_end_im) : mk<C>(k.kd_in, 0.0);
  C Mv[2], Kv[2];
  for (int f = 0; f < 2; ++f) {
    C v0 = get(f, ix);
    C vm = ix > 0 ? get(f, ix - 1) : mk<C>(0, 0);
    C vp = ix < nx - 1 ? get(f, ix + 1) : mk<C>(0, 0);
    C nb = cadd(vm, vp);
    Mv[f] = cadd(cscale(v0, md), cscale(nb, mo));
    Kv[f] = cadd(cmul(v0, kd), cscale(nb, ko));
  }
  const C D11 = mk<C>(k.d11_re, k.d11_im);
  const C D1n = mk<C>(k.d1n_re, 0.0);
  const R E11 = (R)k.e11, E1n = (R)k.e1n;
  // wrap entries of the gamma-circulant: first row x 1/g, last row x g
  C c1 = cadd(cadd(cmul(D11, Mv[0]), cscale(Kv[0], E11)),
              cmul(mk<C>(k.gir, k.gii), cadd(cmul(D1n, Mv[1]), cscale(Kv[1], E1n))));
  C cn = cadd(cmul(mk<C>(k.gr, k.gi), cadd(cmul(D1n, Mv[0]), cscale(Kv[0], E1n))),
              cadd(cmul(D11, Mv[1]), cscale(Kv[1], E11)));
  out[ix] = c1;
  out[nx + ix] = cn;
}

}  // namespace

cudaError_t launch_tri2d(int prec, int step, const void* fhat, const void* faces, const void* ustart, void* rec,
                         void* out, void* partial, const Solve2DArgs& a, const int* skip, cudaStream_t st,
                         Profiler* prof, const void* consts) {
  static const char* n1s[3] = {"tri_step1_pass1", "tri_step2_pass1", "tri_step3_pass1"};
  static const char* ncs[3] = {"tri_step1_carry", "tri_step2_carry", "tri_step3_carry"};
  static const char* n2s[3] = {"tri_step1_pass2", "tri_step2_pass2", "tri_step3_pass2"};
  const int bs = 128;
  const dim3 grid((unsigned)((a.n1 + bs - 1) / bs), (unsigned)a.nchunks);
  const unsigned gcar = (unsigned)((a.n1 + kCarryLines - 1) / kCarryLines);
  const dim3 bcar(kCarryLines, kCarrySeg);
  const size_t nrec = (size_t)a.nchunks * a.n1;
#define HELM_TRI(T, S, CH)                                                                                        \
  do {                                                                                                         \
    using C = cpx<T>::type;                                                                                    \
    {                                                                                                          \
      ProfScope ps(prof, n1s[S - 1], st);                                                                      \
      k_tri_pass1<T, S, CH><<<grid, bs, 0, st>>>((const C*)fhat, (const C*)faces, (const C*)ustart,            \
                                            rec_soa<C>(rec, nrec), a, consts, skip);                          \
    }                                                                                                          \
    {                                                                                                          \
      ProfScope ps(prof, ncs[S - 1], st);                                                                      \
      k_tri_carry<T><<<gcar, bcar, 0, st>>>(rec_soa<C>(rec, nrec), a.n1, a.nchunks, skip);                         \
    }                                                                                                          \
    {                                                                                                          \
      ProfScope ps(prof, n2s[S - 1], st);                                                                      \
      k_tri_pass2<T, S, CH><<<grid, bs, 0, st>>>((const C*)fhat, (const C*)faces, (const C*)ustart,            \
                                                rec_soa<C>(rec, nrec), (C*)out, (C*)partial, a, consts, skip);\
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

cudaError_t launch_tri2d_tab(int step, const void* fhat, const void* faces, const void* tables, void* rec,
                             void* out, void* partial, const Solve2DArgs& a, const int* skip, cudaStream_t st,
                             Profiler* prof) {
  static const char* n1s[3] = {"tri_step1_pass1", "tri_step2_pass1", "tri_step3_pass1"};
  static const char* ncs[3] = {"tri_step1_carry", "tri_step2_carry", "tri_step3_carry"};
  static const char* n2s[3] = {"tri_step1_pass2", "tri_step2_pass2", "tri_step3_pass2"};
  if (a.ch != kChunkF64) return cudaErrorInvalidValue;
  const int bs = 128;
  const dim3 grid((unsigned)((a.n1 + bs - 1) / bs), (unsigned)a.nchunks);
  const unsigned gcar = (unsigned)((a.n1 + kCarryLines - 1) / kCarryLines);
  const dim3 bcar(kCarryLines, kCarrySeg);
  const size_t nrec = (size_t)a.nchunks * a.n1;
  const LineTables tb = line_tables(const_cast<void*>(tables), (size_t)a.nx * a.n1, nrec);
  RecSoA<double2> r = rec_soa<double2>(rec, nrec);
  r.pe = tb.pe;  // rhs-independent chunk constants live in the tables
  r.cc = tb.cc;
  r.we = tb.we;
#define HELM_TRI_TAB(S)                                                                                     \
  do {                                                                                                   \
    {                                                                                                    \
      ProfScope ps(prof, n1s[S - 1], st);                                                                \
      k_tri_pass1_tab<S, kChunkF64><<<grid, bs, 0, st>>>((const double2*)fhat, (const double2*)faces, tb, r, \
                                                         a, skip);                                     \
    }                                                                                                    \
    {                                                                                                    \
      ProfScope ps(prof, ncs[S - 1], st);                                                                \
      k_tri_carry<double><<<gcar, bcar, 0, st>>>(r, a.n1, a.nchunks, skip);                                 \
    }                                                                                                    \
    {                                                                                                    \
      ProfScope ps(prof, n2s[S - 1], st);                                                                \
      k_tri_pass2_tab<S, kChunkF64><<<grid, bs, 0, st>>>((const double2*)fhat, (const double2*)faces, tb, r, \
                                                         (double2*)out, (double2*)partial, a, skip);   \
    }                                                                                                    \
  } while (0)
  if (step == 1) HELM_TRI_TAB(1);
  else if (step == 2) HELM_TRI_TAB(2);
  else HELM_TRI_TAB(3);
#undef HELM_TRI_TAB
  return cudaGetLastError();
}

cudaError_t launch_tri2d_t32(int step, const void* fhat, const void* faces, const void* tables, void* rec, void* out,
                             void* partial, const Solve2DArgs& a, const int* skip, cudaStream_t st, Profiler* prof,
                             const void* consts, int* err) {
  static const char* n1s[3] = {"tri_step1_pass1", "tri_step2_pass1", "tri_step3_pass1"};
  static const char* ncs[3] = {"tri_step1_carry", "tri_step2_carry", "tri_step3_carry"};
  static const char* n2s[3] = {"tri_step1_pass2", "tri_step2_pass2", "tri_step3_pass2"};
  if (a.ch != kChunkF32) return cudaErrorInvalidValue;
  const int bs = 128;
  const dim3 grid((unsigned)((a.n1 + bs - 1) / bs), (unsigned)a.nchunks);
  const unsigned gcar = (unsigned)((a.n1 + kCarryLines - 1) / kCarryLines);
  const dim3 bcar(kCarryLines, kCarrySeg);
  const size_t nrec = (size_t)a.nchunks * a.n1;
  const LineTables32 tb = line_tables32(const_cast<void*>(tables), (size_t)a.nx * a.n1, nrec, (size_t)a.n1);
  RecSoA<float2> r = rec_soa<float2>(rec, nrec);
  r.pe = tb.pe;  // rhs-independent chunk constants live in the tables
  r.cc = tb.cc;
  r.we = tb.we;
  // even n1: 16-byte aligned rows, the bulk-copy fed kernels
  const bool bulk = (a.n1 % 2) == 0 && !a.tri_regs;
  const dim3 gbulk((unsigned)((a.n1 + kBulkLines - 1) / kBulkLines),
                   (unsigned)((a.nchunks + kBulkChunks - 1) / kBulkChunks));

#define HELM_TRI_T32(S)                                                                                        \
  do {                                                                                                        \
    if (bulk) {                                                                                               \
      auto k1 = k_tri_bulk_t32<1, S, kChunkF32>;                                                              \
      auto k2 = k_tri_bulk_t32<2, S, kChunkF32>;                                                              \
      const size_t sb1 = bulk_tile_bytes<1, S, kChunkF32>(), sb2 = bulk_tile_bytes<2, S, kChunkF32>();        \
      allow_dynamic_smem((const void*)k1, sb1);                                                               \
      allow_dynamic_smem((const void*)k2, sb2);                                                               \
      {                                                                                                       \
        ProfScope ps(prof, n1s[S - 1], st);                                                                   \
        k1<<<gbulk, kBulkLines, sb1, st>>>((const float2*)fhat, (const float2*)faces, tb, r, nullptr, nullptr, \
                                             a, consts, skip, err);                                           \
      }                                                                                                       \
      {                                                                                                       \
        ProfScope ps(prof, ncs[S - 1], st);                                                                   \
        k_tri_carry<float><<<gcar, bcar, 0, st>>>(r, a.n1, a.nchunks, skip);                                  \
      }                                                                                                       \
      {                                                                                                       \
        ProfScope ps(prof, n2s[S - 1], st);                                                                   \
        k2<<<gbulk, kBulkLines, sb2, st>>>((const float2*)fhat, (const float2*)faces, tb, r, (float2*)out,  \
                                             (float2*)partial, a, consts, skip, err);                         \
      }                                                                                                       \
      break;                                                                                                  \
    }                                                                                                         \
    {                                                                                                         \
      ProfScope ps(prof, n1s[S - 1], st);                                                                     \
      k_tri_pass1_t32<S, kChunkF32><<<grid, bs, 0, st>>>((const float2*)fhat, (const float2*)faces, tb, r, a, \
                                                         consts, skip);                                       \
    }                                                                                                         \
    {                                                                                                         \
      ProfScope ps(prof, ncs[S - 1], st);                                                                     \
      k_tri_carry<float><<<gcar, bcar, 0, st>>>(r, a.n1, a.nchunks, skip);                                    \
    }                                                                                                         \
    {                                                                                                         \
      ProfScope ps(prof, n2s[S - 1], st);                                                                     \
      k_tri_pass2_t32<S, kChunkF32><<<grid, bs, 0, st>>>((const float2*)fhat, (const float2*)faces, tb, r,    \
                                                         (float2*)out, (float2*)partial, a, consts, skip);    \
    }                                                                                                         \
  } while (0)
  if (step == 1) HELM_TRI_T32(1);
  else if (step == 2) HELM_TRI_T32(2);
  else HELM_TRI_T32(3);
#undef HELM_TRI_T32
  return cudaGetLastError();
}

size_t line_tables32_bytes(int64_t nx, int64_t n1, int64_t nchunks) {
  return (size_t)(nx * n1 + 3 * nchunks * n1 + n1) * sizeof(float2) +
         (size_t)((n1 + kBulkLines - 1) / kBulkLines) * sizeof(int);
}

cudaError_t launch_line_tables32(void* tables, const Solve2DArgs& a, int step, cudaStream_t st) {
  const int bs = 128;
  const unsigned grid = (unsigned)((a.n1 + bs - 1) / bs);
  const LineTables32 tb = line_tables32(tables, (size_t)a.nx * a.n1, (size_t)a.nchunks * a.n1, (size_t)a.n1);
  cudaError_t e = cudaMemsetAsync(tb.lcta, 0, (size_t)((a.n1 + kBulkLines - 1) / kBulkLines) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_line_tables32<<<grid, bs, 0, st>>>(tb, a, step);
  return cudaGetLastError();
}

size_t line_tables_bytes(int64_t nx, int64_t n1, int64_t nchunks) {
  return (size_t)(3 * nx * n1 + 3 * nchunks * n1) * sizeof(double2);
}

cudaError_t launch_line_tables(void* tables, const Solve2DArgs& a, int step, cudaStream_t st) {
  const int bs = 128;
  const unsigned grid = (unsigned)((a.n1 + bs - 1) / bs);
  const LineTables tb = line_tables(tables, (size_t)a.nx * a.n1, (size_t)a.nchunks * a.n1);
  k_line_tables<<<grid, bs, 0, st>>>(tb, a, step);
  return cudaGetLastError();
}

size_t line_consts_bytes(int prec, int64_t n1) { return (size_t)8 * n1 * (prec == kPrecF64 ? sizeof(double2) : sizeof(float2)); }

cudaError_t launch_line_consts(int prec, void* out, const Solve2DArgs& a, int step, cudaStream_t st) {
  const int bs = 128;
  const unsigned grid = (unsigned)((a.n1 + bs - 1) / bs);
  if (prec == kPrecF64)
    k_line_consts<double><<<grid, bs, 0, st>>>((double2*)out, a, step);
  else
    k_line_consts<float><<<grid, bs, 0, st>>>((float2*)out, a, step);
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
  const unsigned grid = (unsigned)((2 * nx * kFaceLanes + bs - 1) / bs);
  if (prec == kPrecF64)
    k_reduce_faces<double><<<grid, bs, 0, st>>>((const double2*)partial, (double2*)out, nx, nwarps, s0[0], s0[1],
                                                s1[0], s1[1], skip);
  else
    k_reduce_faces<float><<<grid, bs, 0, st>>>((const float2*)partial, (float2*)out, nx, nwarps, s0[0], s0[1], s1[0],
                                               s1[1], skip);
  return cudaGetLastError();
}

cudaError_t launch_apply_cbb(int prec, const void* in, const void* in2, void* out, int64_t nx, double hx,
                             double h1, double wx, double wy, double p, const double* g, const double* ginv,
                             const int* skip, cudaStream_t st, double mden) {
  // the entries of eqs. BminA, Cbb once, in double, on the host
  const MassCoef mx = mass_coef(hx, mden), m1 = mass_coef(h1, mden);
  CbbConsts k;
  k.md_end = mx.end;
  k.md_in = mx.in;
  k.mo = mx.off;
  k.kd_end_re = 1.0 / hx;
  k.kd_end_im = -wx;
  k.kd_in = 2.0 / hx;
  k.ko = -1.0 / hx;
  k.d11_re = 1.0 / h1 - p * m1.end;
  k.d11_im = wy;
  k.d1n_re = -1.0 / h1 - p * m1.off;
  k.e11 = m1.end;
  k.e1n = m1.off;
  k.gr = g[0];
  k.gi = g[1];
  k.gir = ginv[0];
  k.gii = ginv[1];
  const int bs = 256;
  const unsigned grid = (unsigned)((nx + bs - 1) / bs);
  if (prec == kPrecF64)
    k_apply_cbb<double><<<grid, bs, 0, st>>>((const double2*)in, (const double2*)in2, (double2*)out, nx, k, skip);
  else
    k_apply_cbb<float><<<grid, bs, 0, st>>>((const float2*)in, (const float2*)in2, (float2*)out, nx, k, skip);
  return cudaGetLastError();
}

}  // namespace helm
