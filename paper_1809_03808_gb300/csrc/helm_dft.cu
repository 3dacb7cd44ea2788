// Batched DFT kernels (sm_103a): f_hat_l = sum_k e^{-2 pi i (k-1)(l-1)/n} f_k
// (eq. step1FFTfcoeff) and its inverse with 1/n (eq. step3IFFTz3coeff),
// applied to every line of a batch.  Stockham auto-sort, mixed radix
// (8, 4, 2 butterflies; any other prime by a direct R-point DFT), the whole
// line resident in shared memory, ping-pong between two buffers per stage.
//
// Two access patterns:
//   rows    : lines are contiguous (the last array axis), L lines per CTA;
//   columns : lines are strided by `inner` (a middle array axis); a CTA loads
//             a [n][TC] tile (TC consecutive inner indices) and transforms
//             its TC columns.
#include <algorithm>

#include "helm_dft.h"
#include "helm_kernels.cuh"

namespace helm {

namespace {

// Twiddle e^{sign 2 pi i e / n} from the forward table (sign = -1 forward).
template <typename C>
__device__ __forceinline__ C tw_get(const C* __restrict__ tw, int e, int sign) {
  C w = tw[e];
  if (sign > 0) w.y = -w.y;
  return w;
}

// One Stockham stage for butterfly j of a line: src/dst point to the line,
// element i of the line is at src[i * ps] (ps = point stride in smem).
template <typename C>
__device__ __forceinline__ void butterfly(const C* __restrict__ src, C* __restrict__ dst, int ps, int n,
                                          int R, int Ns, int j, const C* __restrict__ tw, int sign,
                                          C* __restrict__ scratch_line) {
  using T = decltype(src[0].x);
  const int nb = n / R;
  const int k = j % Ns;
  const int base = (j / Ns) * Ns * R + k;
  const int st = n / (Ns * R);  // twiddle stride
  if (R == 2) {
    C a0 = src[j * ps], a1 = src[(j + nb) * ps];
    if (k) a1 = cmul(a1, tw_get(tw, k * st, sign));
    dst[base * ps] = cadd(a0, a1);
    dst[(base + Ns) * ps] = csub(a0, a1);
  } else if (R == 4) {
    C a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = src[(j + r * nb) * ps];
    if (k) {
#pragma unroll
      for (int r = 1; r < 4; ++r) a[r] = cmul(a[r], tw_get(tw, r * k * st, sign));
    }
    C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    C t2 = cadd(a[1], a[3]), t3 = csub(a[1], a[3]);
    // multiply t3 by (sign * i)
    C t3r;
    t3r.x = -(T)sign * t3.y;
    t3r.y = (T)sign * t3.x;
    dst[base * ps] = cadd(t0, t2);
    dst[(base + Ns) * ps] = cadd(t1, t3r);
    dst[(base + 2 * Ns) * ps] = csub(t0, t2);
    dst[(base + 3 * Ns) * ps] = csub(t1, t3r);
  } else if (R == 8) {
    C a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = src[(j + r * nb) * ps];
    if (k) {
#pragma unroll
      for (int r = 1; r < 8; ++r) a[r] = cmul(a[r], tw_get(tw, r * k * st, sign));
    }
    const T s = (T)sign;
    const T h = (T)0.70710678118654752440;
    // even part: DFT4 of a0 a2 a4 a6; odd part: DFT4 of a1 a3 a5 a7
    C e0 = cadd(a[0], a[4]), e1 = csub(a[0], a[4]), e2 = cadd(a[2], a[6]), e3 = csub(a[2], a[6]);
    C o0 = cadd(a[1], a[5]), o1 = csub(a[1], a[5]), o2 = cadd(a[3], a[7]), o3 = csub(a[3], a[7]);
    C e3r, o3r;
    e3r.x = -s * e3.y;
    e3r.y = s * e3.x;
    o3r.x = -s * o3.y;
    o3r.y = s * o3.x;
    C E0 = cadd(e0, e2), E2 = csub(e0, e2), E1 = cadd(e1, e3r), E3 = csub(e1, e3r);
    C O0 = cadd(o0, o2), O2 = csub(o0, o2), O1 = cadd(o1, o3r), O3 = csub(o1, o3r);
    // W8^1 = (h, s h), W8^2 = (0, s), W8^3 = (-h, s h)
    C W1O1, W2O2, W3O3;
    W1O1.x = h * (O1.x - s * O1.y);
    W1O1.y = h * (O1.y + s * O1.x);
    W2O2.x = -s * O2.y;
    W2O2.y = s * O2.x;
    W3O3.x = h * (-O3.x - s * O3.y);
    W3O3.y = h * (-O3.y + s * O3.x);
    dst[base * ps] = cadd(E0, O0);
    dst[(base + Ns) * ps] = cadd(E1, W1O1);
    dst[(base + 2 * Ns) * ps] = cadd(E2, W2O2);
    dst[(base + 3 * Ns) * ps] = cadd(E3, W3O3);
    dst[(base + 4 * Ns) * ps] = csub(E0, O0);
    dst[(base + 5 * Ns) * ps] = csub(E1, W1O1);
    dst[(base + 6 * Ns) * ps] = csub(E2, W2O2);
    dst[(base + 7 * Ns) * ps] = csub(E3, W3O3);
  } else {
    // direct R-point DFT; inputs twiddled into the thread's private scratch
    for (int r = 0; r < R; ++r) {
      C v = src[(j + r * nb) * ps];
      if (k && r) v = cmul(v, tw_get(tw, r * k * st, sign));
      scratch_line[r] = v;
    }
    for (int q = 0; q < R; ++q) {
      C acc = scratch_line[0];
      int e = 0;
      for (int r = 1; r < R; ++r) {
        e += q;
        if (e >= R) e -= R;
        acc = cadd(acc, cmul(scratch_line[r], tw_get(tw, e * nb, sign)));
      }
      dst[(base + q * Ns) * ps] = acc;
    }
  }
}

template <typename T>
__device__ __forceinline__ typename cpx<T>::type load_in(const void* p, int in_is_double, int64_t i) {
  using C = typename cpx<T>::type;
  if (in_is_double == kInC128) return cvt<C>(reinterpret_cast<const double2*>(p)[i]);
  if (in_is_double == kInFF) {
    const float4 q = reinterpret_cast<const float4*>(p)[i];
    return mk<C>(q.x, q.y);
  }
  return cvt<C>(reinterpret_cast<const float2*>(p)[i]);
}

template <typename C>
__device__ __forceinline__ void store_out(void* p, int mode, int64_t i, C v, double accum_scale) {
  if (mode == kOutC128) {
    reinterpret_cast<double2*>(p)[i] = make_double2((double)v.x, (double)v.y);
  } else if (mode == kOutC64) {
    reinterpret_cast<float2*>(p)[i] = make_float2((float)v.x, (float)v.y);
  } else if (mode == kOutAccumC128) {  // u += accum_scale * v
    double2 u = reinterpret_cast<double2*>(p)[i];
    u.x += accum_scale * (double)v.x;
    u.y += accum_scale * (double)v.y;
    reinterpret_cast<double2*>(p)[i] = u;
  } else if (mode == kOutFF) {
    reinterpret_cast<float4*>(p)[i] = make_float4((float)v.x, (float)v.y, 0.f, 0.f);
  } else {  // kOutAccumFF: float-float u += accum_scale * v
    float4 u = reinterpret_cast<float4*>(p)[i];
    ff_add_f(u.x, u.z, (float)accum_scale * (float)v.x);
    ff_add_f(u.y, u.w, (float)accum_scale * (float)v.y);
    reinterpret_cast<float4*>(p)[i] = u;
  }
}

// Generic-radix scratch: one line of up to kMaxGenericRadix values per thread.
constexpr int kMaxGenericRadix = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_dft_rows(const void* __restrict__ in, int in_is_double,
                                                  void* __restrict__ out, int out_mode, int64_t nrows,
                                                  int L, DftPlan p,
                                                  const typename cpx<T>::type* __restrict__ tw, int sign,
                                                  T scale, double accum_scale,
                                                  const typename cpx<T>::type* __restrict__ sc_in,
                                                  const typename cpx<T>::type* __restrict__ sc_out,
                                                  const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = p.n;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + (size_t)L * n;
  const int64_t row0 = (int64_t)blockIdx.x * L;
  const int Lh = (int)min((int64_t)L, nrows - row0);
  const int tot = Lh * n;
  const int64_t g0 = row0 * n;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    C v = load_in<T>(in, in_is_double, g0 + e);
    if (sc_in) v = cmul(v, sc_in[e % n]);
    buf0[e] = v;
  }
  __syncthreads();
  C* cur = buf0;
  C* nxt = buf1;
  int Ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    const int R = p.radix[s];
    const int nb = n / R;
    const int work = Lh * nb;
    for (int b = threadIdx.x; b < work; b += blockDim.x) {
      const int line = b / nb, j = b - line * nb;
      if (R == 2 || R == 4 || R == 8) {
        butterfly<C>(cur + line * n, nxt + line * n, 1, n, R, Ns, j, tw, sign, nullptr);
      } else {
        C loc[kMaxGenericRadix];
        butterfly<C>(cur + line * n, nxt + line * n, 1, n, R, Ns, j, tw, sign, loc);
      }
    }
    __syncthreads();
    C* t = cur;
    cur = nxt;
    nxt = t;
    Ns *= R;
  }
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    C v = cscale(cur[e], scale);
    if (sc_out) v = cmul(v, sc_out[e % n]);
    store_out<C>(out, out_mode, g0 + e, v, accum_scale);
  }
}

// Column transform along a middle axis: array viewed as [outer][n][inner];
// CTA handles TC consecutive inner indices of one outer slab.  smem layout:
// point k of column c at buf[k * TC + c].
template <typename T>
__global__ void __launch_bounds__(256) k_dft_cols(const void* __restrict__ in, int in_is_double,
                                                  void* __restrict__ out, int out_mode, int64_t outer,
                                                  int64_t inner, int TC, DftPlan p,
                                                  const typename cpx<T>::type* __restrict__ tw, int sign,
                                                  T scale, double accum_scale,
                                                  const typename cpx<T>::type* __restrict__ sc_in,
                                                  const typename cpx<T>::type* __restrict__ sc_out,
                                                  const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = p.n;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + (size_t)TC * n;
  const int64_t tiles_per_slab = (inner + TC - 1) / TC;
  const int64_t slab = blockIdx.x / tiles_per_slab;
  const int64_t c0 = (blockIdx.x - slab * tiles_per_slab) * TC;
  const int TCh = (int)min((int64_t)TC, inner - c0);
  const int64_t g0 = slab * (int64_t)n * inner + c0;
  for (int e = threadIdx.x; e < n * TC; e += blockDim.x) {
    const int k = e / TC, c = e - k * TC;
    if (c < TCh) {
      C v = load_in<T>(in, in_is_double, g0 + (int64_t)k * inner + c);
      if (sc_in) v = cmul(v, sc_in[k]);
      buf0[e] = v;
    }
  }
  __syncthreads();
  C* cur = buf0;
  C* nxt = buf1;
  int Ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    const int R = p.radix[s];
    const int nb = n / R;
    const int work = TCh * nb;
    for (int b = threadIdx.x; b < work; b += blockDim.x) {
      const int j = b / TCh, c = b - j * TCh;
      if (R == 2 || R == 4 || R == 8) {
        butterfly<C>(cur + c, nxt + c, TC, n, R, Ns, j, tw, sign, nullptr);
      } else {
        C loc[kMaxGenericRadix];
        butterfly<C>(cur + c, nxt + c, TC, n, R, Ns, j, tw, sign, loc);
      }
    }
    __syncthreads();
    C* t = cur;
    cur = nxt;
    nxt = t;
    Ns *= R;
  }
  for (int e = threadIdx.x; e < n * TC; e += blockDim.x) {
    const int k = e / TC, c = e - k * TC;
    if (c < TCh) {
      C v = cscale(cur[e], scale);
      if (sc_out) v = cmul(v, sc_out[k]);
      store_out<C>(out, out_mode, g0 + (int64_t)k * inner + c, v, accum_scale);
    }
  }
}

// Bluestein's chirp-z transform for lengths with a prime factor above 64.
// With w_j = e^{i pi j^2 / n} and jk = (j^2 + k^2 - (k - j)^2) / 2,
//   sum_j x_j e^{-2 pi i jk/n} = conj(w_k) sum_j (x_j conj(w_j)) w_{k-j},
//   sum_j x_j e^{+2 pi i jk/n} = w_k sum_j (x_j w_j) conj(w_{k-j}),
// a convolution computed as a cyclic one of length m >= 2n - 1 (a power of
// two): the zero-padded sequence is transformed, multiplied by the plan's
// transform of the chirp sequence (already divided by m), and transformed
// back.  Each line stays in shared memory; HBM sees one read and one write.
template <typename C>
__device__ __forceinline__ C chirp(const C* __restrict__ w, int j, int sign) {
  C v = w[j];
  if (sign < 0) v.y = -v.y;  // forward: conj(w_j)
  return v;
}

// In-smem length-m transform of one or several lines (point stride ps, line
// offset lo between lines handled by the caller's index map): radices of m.
template <typename C>
__device__ __forceinline__ C* bs_fft(C* cur, C* nxt, int ps, int nlines, int lstride, const DftPlan& p,
                                     const C* __restrict__ tw, int sign) {
  const int m = p.bm;
  int Ns = 1;
  for (int s = 0; s < p.bstages; ++s) {
    const int R = p.bradix[s];
    const int nb = m / R;
    const int work = nlines * nb;
    for (int b = threadIdx.x; b < work; b += blockDim.x) {
      const int line = b / nb, j = b - line * nb;
      butterfly<C>(cur + line * lstride, nxt + line * lstride, ps, m, R, Ns, j, tw, sign, nullptr);
    }
    __syncthreads();
    C* t = cur;
    cur = nxt;
    nxt = t;
    Ns *= R;
  }
  return cur;
}

// Rows: one line per CTA.
template <typename T>
__global__ void __launch_bounds__(256) k_dft_rows_bs(const void* __restrict__ in, int in_is_double,
                                                     void* __restrict__ out, int out_mode, int64_t nrows, DftPlan p,
                                                     int sign, T scale, double accum_scale,
                                                     const typename cpx<T>::type* __restrict__ sc_in,
                                                     const typename cpx<T>::type* __restrict__ sc_out,
                                                     const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = p.n, m = p.bm;
  const C* w = reinterpret_cast<const C*>(p.bw);
  const C* bf = reinterpret_cast<const C*>(p.bf[sign > 0 ? 1 : 0]);
  const C* tw = reinterpret_cast<const C*>(p.btw);
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + m;
  const int64_t g0 = (int64_t)blockIdx.x * n;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    C v = mk<C>(0, 0);
    if (j < n) {
      v = load_in<T>(in, in_is_double, g0 + j);
      if (sc_in) v = cmul(v, sc_in[j]);
      v = cmul(v, chirp(w, j, sign));
    }
    buf0[j] = v;
  }
  __syncthreads();
  C* cur = bs_fft<C>(buf0, buf1, 1, 1, 0, p, tw, -1);
  for (int k = threadIdx.x; k < m; k += blockDim.x) cur[k] = cmul(cur[k], bf[k]);
  __syncthreads();
  C* oth = cur == buf0 ? buf1 : buf0;
  cur = bs_fft<C>(cur, oth, 1, 1, 0, p, tw, +1);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    C v = cscale(cmul(cur[k], chirp(w, k, sign)), scale);
    if (sc_out) v = cmul(v, sc_out[k]);
    store_out<C>(out, out_mode, g0 + k, v, accum_scale);
  }
}

// Columns along a middle axis ([outer][n][inner]): TC columns per CTA, point
// k of column c at buf[k * TC + c].
template <typename T>
__global__ void __launch_bounds__(256) k_dft_cols_bs(const void* __restrict__ in, int in_is_double,
                                                     void* __restrict__ out, int out_mode, int64_t outer,
                                                     int64_t inner, int TC, DftPlan p, int sign, T scale,
                                                     double accum_scale,
                                                     const typename cpx<T>::type* __restrict__ sc_in,
                                                     const typename cpx<T>::type* __restrict__ sc_out,
                                                     const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = p.n, m = p.bm;
  const C* w = reinterpret_cast<const C*>(p.bw);
  const C* bf = reinterpret_cast<const C*>(p.bf[sign > 0 ? 1 : 0]);
  const C* tw = reinterpret_cast<const C*>(p.btw);
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + (size_t)TC * m;
  const int64_t tiles_per_slab = (inner + TC - 1) / TC;
  const int64_t slab = blockIdx.x / tiles_per_slab;
  const int64_t c0 = (blockIdx.x - slab * tiles_per_slab) * TC;
  const int TCh = (int)min((int64_t)TC, inner - c0);
  const int64_t g0 = slab * (int64_t)n * inner + c0;
  for (int e = threadIdx.x; e < m * TC; e += blockDim.x) {
    const int k = e / TC, c = e - k * TC;
    C v = mk<C>(0, 0);
    if (k < n && c < TCh) {
      v = load_in<T>(in, in_is_double, g0 + (int64_t)k * inner + c);
      if (sc_in) v = cmul(v, sc_in[k]);
      v = cmul(v, chirp(w, k, sign));
    }
    buf0[e] = v;
  }
  __syncthreads();
  // TC lines of stride 1 between lines, point stride TC
  C* cur = bs_fft<C>(buf0, buf1, TC, TC, 1, p, tw, -1);
  for (int e = threadIdx.x; e < m * TC; e += blockDim.x) cur[e] = cmul(cur[e], bf[e / TC]);
  __syncthreads();
  C* oth = cur == buf0 ? buf1 : buf0;
  cur = bs_fft<C>(cur, oth, TC, TC, 1, p, tw, +1);
  for (int e = threadIdx.x; e < n * TC; e += blockDim.x) {
    const int k = e / TC, c = e - k * TC;
    if (c < TCh) {
      C v = cscale(cmul(cur[e], chirp(w, k, sign)), scale);
      if (sc_out) v = cmul(v, sc_out[k]);
      store_out<C>(out, out_mode, g0 + (int64_t)k * inner + c, v, accum_scale);
    }
  }
}

}  // namespace

bool dft_needs_bluestein(const DftPlan& p) {
  for (int s = 0; s < p.nstages; ++s)
    if (p.radix[s] > kMaxGenericRadix) return true;
  return false;
}

int64_t bluestein_length(int64_t n) {
  int64_t m = 1;
  while (m < 2 * n - 1) m <<= 1;
  return m;
}

bool dft_supported(const DftPlan& p, size_t elem_bytes, int max_smem) {
  if (dft_needs_bluestein(p)) {
    const int64_t m = bluestein_length(p.n);
    return m <= 8192 && (size_t)2 * m * elem_bytes <= (size_t)max_smem;
  }
  return (size_t)2 * p.n * elem_bytes <= (size_t)max_smem;
}

cudaError_t launch_dft_rows(int prec, const void* in, int in_is_double, void* out, int out_mode,
                            int64_t nrows, const DftPlan& p, const void* tw, int sign, double scale,
                            double accum_scale, const void* sc_in, const void* sc_out, const int* skip,
                            cudaStream_t st, int* err) {
  // the tensor-core variant, for calls whose scalings are those its tables hold
  if (prec == kPrecF32 && p.gw[sign < 0 ? 0 : 1] && (in_is_double == kInC64 || in_is_double == kInC128) &&
      (out_mode == kOutC64 || out_mode == kOutC128 || out_mode == kOutAccumC128)) {
    const bool fwd = sign < 0;
    const bool same = fwd ? (sc_in == p.gsc[0] && !sc_out && scale == 1.0)
                          : (sc_out == p.gsc[1] && !sc_in && scale == p.gscale);
    if (same)
      return launch_dft_rows_tc(p.gw[fwd ? 0 : 1], p.n, in, in_is_double, out, out_mode, nrows, accum_scale, skip, st,
                                err);
  }
  if (p.bm) {
    if (nrows == 0) return cudaSuccess;
    const size_t es = prec == kPrecF64 ? sizeof(double2) : sizeof(float2);
    const size_t smem = (size_t)2 * p.bm * es;
    if (prec == kPrecF64) {
      auto k = k_dft_rows_bs<double>;
      allow_dynamic_smem((const void*)k, smem);
      k<<<(unsigned)nrows, 256, smem, st>>>(in, in_is_double, out, out_mode, nrows, p, sign, scale, accum_scale,
                                            (const double2*)sc_in, (const double2*)sc_out, skip);
    } else {
      auto k = k_dft_rows_bs<float>;
      allow_dynamic_smem((const void*)k, smem);
      k<<<(unsigned)nrows, 256, smem, st>>>(in, in_is_double, out, out_mode, nrows, p, sign, (float)scale,
                                            accum_scale, (const float2*)sc_in, (const float2*)sc_out, skip);
    }
    return cudaGetLastError();
  }
  if (dft_needs_bluestein(p)) return cudaErrorInvalidValue;  // large prime without its chirp tables
  if (dft_rows_pow2_supported(p.n))
    return launch_dft_rows_pow2(prec, in, in_is_double, out, out_mode, nrows, p.n, tw, sign, scale, accum_scale,
                                sc_in, sc_out, skip, st, err);
  const size_t es = prec == kPrecF64 ? sizeof(double2) : sizeof(float2);
  // lines per CTA: enough points to keep 256 threads busy, bounded by smem
  int L = (int)std::max<int64_t>(1, std::min<int64_t>(nrows, 2048 / std::max(1, p.n)));
  while (L > 1 && (size_t)2 * L * p.n * es > 96 * 1024) --L;
  const size_t smem = (size_t)2 * L * p.n * es;
  const int64_t grid = (nrows + L - 1) / L;
  if (grid == 0) return cudaSuccess;
  if (prec == kPrecF64) {
    auto k = k_dft_rows<double>;
    allow_dynamic_smem((const void*)k, smem);
    k<<<(unsigned)grid, 256, smem, st>>>(in, in_is_double, out, out_mode, nrows, L, p,
                                         reinterpret_cast<const double2*>(tw), sign, scale, accum_scale,
                                         (const double2*)sc_in, (const double2*)sc_out, skip);
  } else {
    auto k = k_dft_rows<float>;
    allow_dynamic_smem((const void*)k, smem);
    k<<<(unsigned)grid, 256, smem, st>>>(in, in_is_double, out, out_mode, nrows, L, p,
                                         reinterpret_cast<const float2*>(tw), sign, (float)scale, accum_scale,
                                         (const float2*)sc_in, (const float2*)sc_out, skip);
  }
  return cudaGetLastError();
}

cudaError_t launch_dft_cols(int prec, const void* in, int in_is_double, void* out, int out_mode,
                            int64_t outer, int64_t inner, const DftPlan& p, const void* tw, int sign,
                            double scale, double accum_scale, const void* sc_in, const void* sc_out,
                            const int* skip, cudaStream_t st) {
  if (p.bm) {
    const size_t es = prec == kPrecF64 ? sizeof(double2) : sizeof(float2);
    int TC = 16;
    while (TC > 1 && (size_t)2 * TC * p.bm * es > 200 * 1024) TC /= 2;
    if (TC > inner) TC = (int)inner;
    const size_t smem = (size_t)2 * TC * p.bm * es;
    const int64_t grid = outer * ((inner + TC - 1) / TC);
    if (grid == 0) return cudaSuccess;
    if (prec == kPrecF64) {
      auto k = k_dft_cols_bs<double>;
      allow_dynamic_smem((const void*)k, smem);
      k<<<(unsigned)grid, 256, smem, st>>>(in, in_is_double, out, out_mode, outer, inner, TC, p, sign, scale,
                                           accum_scale, (const double2*)sc_in, (const double2*)sc_out, skip);
    } else {
      auto k = k_dft_cols_bs<float>;
      allow_dynamic_smem((const void*)k, smem);
      k<<<(unsigned)grid, 256, smem, st>>>(in, in_is_double, out, out_mode, outer, inner, TC, p, sign,
                                           (float)scale, accum_scale, (const float2*)sc_in, (const float2*)sc_out,
                                           skip);
    }
    return cudaGetLastError();
  }
  if (dft_needs_bluestein(p)) return cudaErrorInvalidValue;
  if (dft_cols_pow2_supported(p.n))
    return launch_dft_cols_pow2(prec, in, in_is_double, out, out_mode, outer, inner, p.n, tw, sign, scale,
                                accum_scale, sc_in, sc_out, skip, st);
  const size_t es = prec == kPrecF64 ? sizeof(double2) : sizeof(float2);
  int TC = 16;
  while (TC > 1 && (size_t)2 * TC * p.n * es > 200 * 1024) TC /= 2;
  if (TC > inner) TC = (int)inner;
  const size_t smem = (size_t)2 * TC * p.n * es;
  const int64_t grid = outer * ((inner + TC - 1) / TC);
  if (grid == 0) return cudaSuccess;
  if (prec == kPrecF64) {
    auto k = k_dft_cols<double>;
    allow_dynamic_smem((const void*)k, smem);
    k<<<(unsigned)grid, 256, smem, st>>>(in, in_is_double, out, out_mode, outer, inner, TC, p,
                                         reinterpret_cast<const double2*>(tw), sign, scale, accum_scale,
                                         (const double2*)sc_in, (const double2*)sc_out, skip);
  } else {
    auto k = k_dft_cols<float>;
    allow_dynamic_smem((const void*)k, smem);
    k<<<(unsigned)grid, 256, smem, st>>>(in, in_is_double, out, out_mode, outer, inner, TC, p,
                                         reinterpret_cast<const float2*>(tw), sign, (float)scale, accum_scale,
                                         (const float2*)sc_in, (const float2*)sc_out, skip);
  }
  return cudaGetLastError();
}

}  // namespace helm
