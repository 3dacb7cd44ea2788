// Batched DFT of power-of-two lines along the contiguous axis (the transform
// of eqs. step1FFTfcoeff / step3IFFTz3coeff for n = 2^m, 16 <= n <= 8192).
//
// Stockham auto-sort with the radices fixed at compile time: one leading pass
// of radix 2^(m mod 4) when m is not a multiple of 4, then radix-16 passes.
// Every thread owns 16 points of a line in registers through every pass
// (n / 16 threads per line): it reads its butterflies' inputs, multiplies by
// the twiddles, runs the 16 / R R-point DFTs in registers and writes the
// outputs to their Stockham positions.  The first pass reads global memory
// directly (coalesced across the threads of a line), the last pass writes it
// directly; the passes in between exchange through shared memory padded by
// one point per 16 so that both the strided writes and the unit-stride reads
// are free of bank conflicts.
#include <algorithm>

#include "helm_async.cuh"
#include "helm_dft.h"
#include "helm_kernels.cuh"

namespace helm {

namespace {

template <typename C, int SIGN>
__device__ __forceinline__ C twid(const C* __restrict__ tw, int e) {
  C w = __ldg(&tw[e]);  // forward table e^{-2 pi i e / n}
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// (SIGN i) a
template <typename C, int SIGN>
__device__ __forceinline__ C mul_si(C a) {
  C o;
  if (SIGN > 0) {
    o.x = -a.y;
    o.y = a.x;
  } else {
    o.x = a.y;
    o.y = -a.x;
  }
  return o;
}

// (cr + i ci) a for compile-time constants
template <typename C>
__device__ __forceinline__ C mul_c(C a, double cr, double ci) {
  using T = decltype(a.x);
  C o;
  o.x = a.x * (T)cr - a.y * (T)ci;
  o.y = a.x * (T)ci + a.y * (T)cr;
  return o;
}

// In-register R-point DFTs, natural order in and out:
// y_q = sum_r v_r e^{SIGN 2 pi i r q / R}.
template <typename C, int SIGN>
__device__ __forceinline__ void dft2(C* v) {
  const C a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}

template <typename C, int SIGN>
__device__ __forceinline__ void dft4s(C& v0, C& v1, C& v2, C& v3) {
  const C t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = mul_si<C, SIGN>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v1 = cadd(t1, t3);
  v2 = csub(t0, t2);
  v3 = csub(t1, t3);
}

template <typename C, int SIGN>
__device__ __forceinline__ void dft4(C* v) {
  dft4s<C, SIGN>(v[0], v[1], v[2], v[3]);
}

constexpr double kH = 0.70710678118654752440;   // cos(pi/4)
constexpr double kC8 = 0.92387953251128675613;  // cos(pi/8)
constexpr double kS8 = 0.38268343236508977173;  // sin(pi/8)

template <typename C, int SIGN>
__device__ __forceinline__ void dft8(C* v) {
  // even and odd halves: E_q in v[2q], O_q in v[2q+1]
  dft4s<C, SIGN>(v[0], v[2], v[4], v[6]);
  dft4s<C, SIGN>(v[1], v[3], v[5], v[7]);
  const double s = SIGN;
  const C o1 = mul_c(v[3], kH, s * kH);     // W8^1 O_1
  const C o2 = mul_si<C, SIGN>(v[5]);       // W8^2 O_2
  const C o3 = mul_c(v[7], -kH, s * kH);    // W8^3 O_3
  const C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

template <typename C, int SIGN>
__device__ __forceinline__ void dft16(C* v) {
  // r = b + 4a: DFT4 over a for each b (results Z_b[q1] at v[b + 4 q1])
#pragma unroll
  for (int b = 0; b < 4; ++b) dft4s<C, SIGN>(v[b], v[b + 4], v[b + 8], v[b + 12]);
  // twiddles W16^{b q1}
  const double s = SIGN;
  v[5] = mul_c(v[5], kC8, s * kS8);     // b1 q1 = 1
  v[9] = mul_c(v[9], kH, s * kH);       // b1 q2 = 2
  v[13] = mul_c(v[13], kS8, s * kC8);   // b1 q3 = 3
  v[6] = mul_c(v[6], kH, s * kH);       // b2 q1 = 2
  v[10] = mul_si<C, SIGN>(v[10]);       // b2 q2 = 4
  v[14] = mul_c(v[14], -kH, s * kH);    // b2 q3 = 6
  v[7] = mul_c(v[7], kS8, s * kC8);     // b3 q1 = 3
  v[11] = mul_c(v[11], -kH, s * kH);    // b3 q2 = 6
  v[15] = mul_c(v[15], -kC8, -s * kS8); // b3 q3 = 9
  // DFT4 over b for each q1: y[q1 + 4 q2] lands at v[4 q1 + q2]
#pragma unroll
  for (int q1 = 0; q1 < 4; ++q1) dft4s<C, SIGN>(v[4 * q1], v[4 * q1 + 1], v[4 * q1 + 2], v[4 * q1 + 3]);
  C y[16];
#pragma unroll
  for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) y[q1 + 4 * q2] = v[4 * q1 + q2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = y[i];
}

template <typename C, int R, int SIGN>
__device__ __forceinline__ void dft_r(C* v) {
  if constexpr (R == 2) dft2<C, SIGN>(v);
  else if constexpr (R == 4) dft4<C, SIGN>(v);
  else if constexpr (R == 8) dft8<C, SIGN>(v);
  else dft16<C, SIGN>(v);
}

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// Butterfly q of thread t in a pass of radix R: j = t + q n/16; its input r
// is point j + r n/R; its output r' goes to (j - k) R + k + r' NS, k = j mod NS.
template <int N, int R>
__device__ __forceinline__ int in_index(int t, int q, int r) {
  return t + q * (N / 16) + r * (N / R);
}
template <int N, int R, int NS>
__device__ __forceinline__ int out_index(int t, int q, int rp) {
  const int j = t + q * (N / 16);
  const int k = j & (NS - 1);
  return (j - k) * R + k + rp * NS;
}

// Twiddles and R-point DFTs of one pass on the thread's 16 registers.  The
// input r of a butterfly is multiplied by w^r, w = e^{SIGN 2 pi i k / (NS R)}.
// FP64 reads every w^r from the table (FP64 multiplies are the scarce
// resource); FP32 reads w once and forms w^2 .. w^(R-1) by binary powering
// (at most four dependent products, a few ulps).
template <typename C, int N, int R, int NS, int SIGN>
__device__ __forceinline__ void pass_compute(C* v, int t, const C* __restrict__ tw) {
  using T = decltype(C().x);
#pragma unroll
  for (int q = 0; q < 16 / R; ++q) {
    if constexpr (NS > 1) {
      const int k = (t + q * (N / 16)) & (NS - 1);
      constexpr int S = N / (NS * R);
      if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], twid<C, SIGN>(tw, r * k * S));
      } else {
        C w[R];
        w[1] = twid<C, SIGN>(tw, k * S);
#pragma unroll
        for (int r = 2; r < R; ++r) {
          // r = hb + rest with hb the highest power of two <= r
          const int hb = (r >= 8) ? 8 : (r >= 4) ? 4 : 2;
          w[r] = (r == hb) ? cmul(w[hb / 2], w[hb / 2]) : cmul(w[hb], w[r - hb]);
        }
#pragma unroll
        for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], w[r]);
      }
    }
    dft_r<C, R, SIGN>(v + q * R);
  }
}

template <typename T>
__device__ __forceinline__ typename cpx<T>::type load_pt(const void* p, int in_is_double, int64_t i) {
  using C = typename cpx<T>::type;
  if (in_is_double == kInC128) return cvt<C>(__ldg(reinterpret_cast<const double2*>(p) + i));
  if (in_is_double == kInFF) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p) + i);
    return mk<C>(q.x, q.y);
  }
  return cvt<C>(__ldg(reinterpret_cast<const float2*>(p) + i));
}

// The 16 input points of thread t in the first pass (point e = q R0 + r at
// base + in_index(t, q, r) * stride), scaled by sc_in: the input kind is
// resolved once and every load of a batch is issued before any is used, so
// the loads of a thread are in flight together (8 at a time for 16-byte
// points, all 16 for 8-byte ones).
template <typename T, int N, int R0>
__device__ __forceinline__ void load16(typename cpx<T>::type (&v)[16], const void* in, int kind, int64_t base,
                                       int64_t stride, bool act, int t, const typename cpx<T>::type* sc_in) {
  using C = typename cpx<T>::type;
  auto idx = [&](int e) -> int64_t { return (int64_t)in_index<N, R0>(t, e / R0, e % R0) * stride; };
  if (!act) {
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = mk<C>(0, 0);
    return;
  }
  if (kind == kInC128) {
    const double2* p = reinterpret_cast<const double2*>(in) + base;
#pragma unroll
    for (int hb = 0; hb < 2; ++hb) {
      double2 tmp[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) tmp[k] = __ldg(p + idx(8 * hb + k));
#pragma unroll
      for (int k = 0; k < 8; ++k) v[8 * hb + k] = cvt<C>(tmp[k]);
    }
  } else if (kind == kInFF) {
    const float4* p = reinterpret_cast<const float4*>(in) + base;
#pragma unroll
    for (int hb = 0; hb < 2; ++hb) {
      float4 tmp[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) tmp[k] = __ldg(p + idx(8 * hb + k));
#pragma unroll
      for (int k = 0; k < 8; ++k) v[8 * hb + k] = mk<C>(tmp[k].x, tmp[k].y);
    }
  } else {
    const float2* p = reinterpret_cast<const float2*>(in) + base;
    float2 tmp[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) tmp[e] = __ldg(p + idx(e));
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = cvt<C>(tmp[e]);
  }
  if (sc_in) {
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = cmul(v[e], __ldg(&sc_in[in_index<N, R0>(t, e / R0, e % R0)]));
  }
}

template <typename C>
__device__ __forceinline__ void store_pt(void* p, int mode, int64_t i, C v, double accum_scale) {
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

// Passes 1 .. NP-1 (radix 16, span NS): shared memory in, shared memory or
// (last pass) global memory out.
template <typename T, int N, int SIGN, int NS, int LEFT>
__device__ __forceinline__ void later_passes(typename cpx<T>::type* v, typename cpx<T>::type* buf, int t,
                                             bool act, int64_t g0, void* __restrict__ out, int out_mode,
                                             const typename cpx<T>::type* __restrict__ tw, T scale,
                                             double accum_scale, const typename cpx<T>::type* __restrict__ sc_out) {
  using C = typename cpx<T>::type;
  __syncthreads();  // the previous pass's outputs are in buf
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = buf[pad16(in_index<N, 16>(t, 0, r))];
  pass_compute<C, N, 16, NS, SIGN>(v, t, tw);
  if constexpr (LEFT == 1) {
    if (act) {
#pragma unroll
      for (int rp = 0; rp < 16; ++rp) {
        const int o = out_index<N, 16, NS>(t, 0, rp);
        C x = cscale(v[rp], scale);
        if (sc_out) x = cmul(x, __ldg(&sc_out[o]));
        store_pt<C>(out, out_mode, g0 + o, x, accum_scale);
      }
    }
  } else {
    __syncthreads();  // every thread has read its inputs
#pragma unroll
    for (int rp = 0; rp < 16; ++rp) buf[pad16(out_index<N, 16, NS>(t, 0, rp))] = v[rp];
    later_passes<T, N, SIGN, NS * 16, LEFT - 1>(v, buf, t, act, g0, out, out_mode, tw, scale, accum_scale, sc_out);
  }
}

template <int LOG2N>
__host__ __device__ constexpr int pow2_threads() {
  return LOG2N >= 13 ? (1 << LOG2N) / 16 : 256;
}

template <typename T, int LOG2N, int SIGN>
__global__ void __launch_bounds__(pow2_threads<LOG2N>())
    k_dft_rows_pow2(const void* __restrict__ in, int in_is_double, void* __restrict__ out, int out_mode,
                    int64_t nrows, const typename cpx<T>::type* __restrict__ tw, T scale, double accum_scale,
                    const typename cpx<T>::type* __restrict__ sc_in,
                    const typename cpx<T>::type* __restrict__ sc_out, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  constexpr int N = 1 << LOG2N;
  constexpr int TPL = N / 16;                      // threads per line
  constexpr int L = pow2_threads<LOG2N>() / TPL;  // lines per CTA
  constexpr int NPAD = N + N / 16;
  constexpr int E = LOG2N % 4;
  constexpr int R0 = E ? (1 << E) : 16;
  constexpr int NP = (LOG2N + 3) / 4;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x % TPL;
  const int line = threadIdx.x / TPL;
  const int64_t row = (int64_t)blockIdx.x * L + line;
  const bool act = row < nrows;
  const int64_t g0 = row * N;
  C* buf = reinterpret_cast<C*>(smem_raw) + line * NPAD;
  C v[16];
  // pass 0 (radix R0, no twiddles): global memory in
  load16<T, N, R0>(v, in, in_is_double, g0, 1, act, t, sc_in);
  pass_compute<C, N, R0, 1, SIGN>(v, t, tw);
  if constexpr (NP == 1) {
    if (act) {
#pragma unroll
      for (int q = 0; q < 16 / R0; ++q)
#pragma unroll
        for (int rp = 0; rp < R0; ++rp) {
          const int o = out_index<N, R0, 1>(t, q, rp);
          C x = cscale(v[q * R0 + rp], scale);
          if (sc_out) x = cmul(x, __ldg(&sc_out[o]));
          store_pt<C>(out, out_mode, g0 + o, x, accum_scale);
        }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16 / R0; ++q)
#pragma unroll
      for (int rp = 0; rp < R0; ++rp) buf[pad16(out_index<N, R0, 1>(t, q, rp))] = v[q * R0 + rp];
    later_passes<T, N, SIGN, R0, NP - 1>(v, buf, t, act, g0, out, out_mode, tw, scale, accum_scale, sc_out);
  }
}

// Column variant: lines along a middle axis of an array viewed as
// [outer][N][inner].  A CTA takes TC consecutive inner indices (columns) of
// one outer slab; thread (t, c) = (threadIdx.x / TC, threadIdx.x % TC) owns
// 16 points of column c, so the lanes of a warp touch TC consecutive columns
// of the same line point (contiguous in global and in shared memory, where
// point i of column c sits at i * TC + c).
// Columns per CTA: TC * N / 16 threads, at most 512 (complex64) or 256
// (complex128, whose CTAs also need twice the shared memory per column).
template <typename T, int LOG2N>
__host__ __device__ constexpr int cols_tc() {
  return sizeof(T) == 4 ? ((8192 >> LOG2N) > 64 ? 64 : (8192 >> LOG2N))
                        : ((4096 >> LOG2N) > 32 ? 32 : ((4096 >> LOG2N) < 1 ? 1 : (4096 >> LOG2N)));
}

template <typename T, int N, int SIGN, int NS, int LEFT, int TC>
__device__ __forceinline__ void later_passes_cols(typename cpx<T>::type* v, typename cpx<T>::type* buf, int t, int c,
                                                  bool act, int64_t g0, int64_t inner, void* __restrict__ out,
                                                  int out_mode, const typename cpx<T>::type* __restrict__ tw, T scale,
                                                  double accum_scale,
                                                  const typename cpx<T>::type* __restrict__ sc_out) {
  using C = typename cpx<T>::type;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = buf[in_index<N, 16>(t, 0, r) * TC + c];
  pass_compute<C, N, 16, NS, SIGN>(v, t, tw);
  if constexpr (LEFT == 1) {
    if (act) {
#pragma unroll
      for (int rp = 0; rp < 16; ++rp) {
        const int o = out_index<N, 16, NS>(t, 0, rp);
        C x = cscale(v[rp], scale);
        if (sc_out) x = cmul(x, __ldg(&sc_out[o]));
        store_pt<C>(out, out_mode, g0 + (int64_t)o * inner, x, accum_scale);
      }
    }
  } else {
    __syncthreads();
#pragma unroll
    for (int rp = 0; rp < 16; ++rp) buf[out_index<N, 16, NS>(t, 0, rp) * TC + c] = v[rp];
    later_passes_cols<T, N, SIGN, NS * 16, LEFT - 1, TC>(v, buf, t, c, act, g0, inner, out, out_mode, tw, scale,
                                                         accum_scale, sc_out);
  }
}

template <typename T, int LOG2N, int SIGN>
__global__ void __launch_bounds__(cols_tc<T, LOG2N>() * (1 << LOG2N) / 16)
    k_dft_cols_pow2(const void* __restrict__ in, int in_is_double, void* __restrict__ out, int out_mode,
                    int64_t outer, int64_t inner, const typename cpx<T>::type* __restrict__ tw, T scale,
                    double accum_scale, const typename cpx<T>::type* __restrict__ sc_in,
                    const typename cpx<T>::type* __restrict__ sc_out, const int* __restrict__ skip) {
  using C = typename cpx<T>::type;
  constexpr int N = 1 << LOG2N;
  constexpr int TC = cols_tc<T, LOG2N>();
  constexpr int E = LOG2N % 4;
  constexpr int R0 = E ? (1 << E) : 16;
  constexpr int NP = (LOG2N + 3) / 4;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int c = threadIdx.x % TC;
  const int t = threadIdx.x / TC;
  const int64_t tiles = (inner + TC - 1) / TC;
  const int64_t slab = blockIdx.x / tiles;
  const int64_t col = (blockIdx.x - slab * tiles) * TC + c;
  const bool act = col < inner;
  const int64_t g0 = slab * (int64_t)N * inner + col;  // point i at g0 + i * inner
  C v[16];
  load16<T, N, R0>(v, in, in_is_double, g0, inner, act, t, sc_in);
  pass_compute<C, N, R0, 1, SIGN>(v, t, tw);
  if constexpr (NP == 1) {
    if (act) {
#pragma unroll
      for (int q = 0; q < 16 / R0; ++q)
#pragma unroll
        for (int rp = 0; rp < R0; ++rp) {
          const int o = out_index<N, R0, 1>(t, q, rp);
          C x = cscale(v[q * R0 + rp], scale);
          if (sc_out) x = cmul(x, __ldg(&sc_out[o]));
          store_pt<C>(out, out_mode, g0 + (int64_t)o * inner, x, accum_scale);
        }
    }
  } else {
    // in place (out == in) is safe: every input of the CTA is read before
    // the first output is written
#pragma unroll
    for (int q = 0; q < 16 / R0; ++q)
#pragma unroll
      for (int rp = 0; rp < R0; ++rp) buf[out_index<N, R0, 1>(t, q, rp) * TC + c] = v[q * R0 + rp];
    later_passes_cols<T, N, SIGN, R0, NP - 1, TC>(v, buf, t, c, act, g0, inner, out, out_mode, tw, scale,
                                                  accum_scale, sc_out);
  }
}

template <typename T, int LOG2N, int SIGN>
cudaError_t launch_cols_pow2_t(const void* in, int in_is_double, void* out, int out_mode, int64_t outer,
                               int64_t inner, const void* tw, double scale, double accum_scale, const void* sc_in,
                               const void* sc_out, const int* skip, cudaStream_t st) {
  using C = typename cpx<T>::type;
  constexpr int N = 1 << LOG2N;
  constexpr int TC = cols_tc<T, LOG2N>();
  constexpr int threads = TC * N / 16;
  constexpr int NP = (LOG2N + 3) / 4;
  const size_t smem = NP > 1 ? (size_t)TC * N * sizeof(C) : 0;
  const int64_t grid = outer * ((inner + TC - 1) / TC);
  if (grid == 0) return cudaSuccess;
  auto k = k_dft_cols_pow2<T, LOG2N, SIGN>;
  if (smem > 48 * 1024) {
    const cudaError_t e = allow_dynamic_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
  }
  k<<<(unsigned)grid, threads, smem, st>>>(in, in_is_double, out, out_mode, outer, inner, (const C*)tw, (T)scale,
                                           accum_scale, (const C*)sc_in, (const C*)sc_out, skip);
  return cudaGetLastError();
}

template <typename T, int SIGN>
cudaError_t launch_cols_pow2_s(int log2n, const void* in, int in_is_double, void* out, int out_mode, int64_t outer,
                               int64_t inner, const void* tw, double scale, double accum_scale, const void* sc_in,
                               const void* sc_out, const int* skip, cudaStream_t st) {
#define HELM_COLS2(LG)                                                                                          \
  case LG:                                                                                                      \
    return launch_cols_pow2_t<T, LG, SIGN>(in, in_is_double, out, out_mode, outer, inner, tw, scale, accum_scale, \
                                           sc_in, sc_out, skip, st);
  switch (log2n) {
    HELM_COLS2(4)
    HELM_COLS2(5)
    HELM_COLS2(6)
    HELM_COLS2(7)
    HELM_COLS2(8)
    HELM_COLS2(9)
    HELM_COLS2(10)
    default:
      return cudaErrorInvalidValue;
  }
#undef HELM_COLS2
}

// Persistent variant for complex64 lines of 4096 or 8192 points: each CTA
// loops over lines (row = blockIdx.x + i gridDim.x) and the next line
// arrives in shared memory by one cp.async.bulk while the current one is
// transformed (two input buffers, mbarrier completion, bounded waits).  The
// passes, the twiddles and the epilogue are those of k_dft_rows_pow2.
template <int LOG2N, int SIGN>
__global__ void __launch_bounds__(pow2_threads<LOG2N>())
    k_dft_rows_pow2_bulk(const float2* __restrict__ in, void* __restrict__ out, int out_mode, int64_t nrows,
                         const float2* __restrict__ tw, float scale, double accum_scale,
                         const float2* __restrict__ sc_in, const float2* __restrict__ sc_out,
                         const int* __restrict__ skip, int* __restrict__ err) {
  using C = float2;
  constexpr int N = 1 << LOG2N;
  constexpr int E = LOG2N % 4;
  constexpr int R0 = E ? (1 << E) : 16;
  constexpr int NP = (LOG2N + 3) / 4;
  static_assert(pow2_threads<LOG2N>() == N / 16, "one line per CTA");
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* const inbuf = reinterpret_cast<C*>(smem_raw);  // [2][N]
  C* const buf = inbuf + 2 * N;                      // exchange, [NPAD]
  __shared__ __align__(8) uint64_t bar[2];
  const int t = threadIdx.x;
  const int64_t stride = gridDim.x;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int64_t row, int b) {
    mbar_arrive_expect_tx(&bar[b], (uint32_t)(N * sizeof(C)));
    bulk_g2s(inbuf + b * N, in + row * N, (uint32_t)(N * sizeof(C)), &bar[b]);
  };
  // thread 0's book of copies in flight: bit b of `pending` (buffer b busy),
  // bit b of `want` (parity of its phase)
  uint32_t pending = 0, want = 0;
  const int64_t r0 = blockIdx.x;
  if (t == 0) {
    if (r0 < nrows) {
      issue(r0, 0);
      pending |= 1u;
    }
    if (r0 + stride < nrows) {
      issue(r0 + stride, 1);
      pending |= 2u;
    }
  }
  bool failed = false;
  int64_t i = 0;
  for (int64_t row = r0; row < nrows; row += stride, ++i) {
    const int b = (int)(i & 1);
    const uint32_t parity = (uint32_t)((i >> 1) & 1);
    const bool got = mbar_wait_bounded(&bar[b], parity, err);
    if (__syncthreads_or(!got)) {
      failed = true;
      break;
    }
    if (t == 0) pending &= ~(1u << b);
    const C* src = inbuf + b * N;
    C v[16];
#pragma unroll
    for (int q = 0; q < 16 / R0; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int k = in_index<N, R0>(t, q, r);
        C x = src[k];
        if (sc_in) x = cmul(x, __ldg(&sc_in[k]));
        v[q * R0 + r] = x;
      }
    // every thread has read this buffer (and the previous line's exchange
    // reads are over): refill the buffer with the line after next
    __syncthreads();
    if (t == 0 && row + 2 * stride < nrows) {
      issue(row + 2 * stride, b);
      pending |= 1u << b;
      want = (want & ~(1u << b)) | ((parity ^ 1u) << b);
    }
    pass_compute<C, N, R0, 1, SIGN>(v, t, tw);
#pragma unroll
    for (int q = 0; q < 16 / R0; ++q)
#pragma unroll
      for (int rp = 0; rp < R0; ++rp) buf[pad16(out_index<N, R0, 1>(t, q, rp))] = v[q * R0 + rp];
    later_passes<float, N, SIGN, R0, NP - 1>(v, buf, t, true, row * N, out, out_mode, tw, scale, accum_scale, sc_out);
  }
  if (failed && t == 0) {
    for (int b = 0; b < 2; ++b)
      if (pending & (1u << b)) mbar_wait_bounded(&bar[b], (want >> b) & 1u, nullptr);
  }
}

template <int LOG2N, int SIGN>
cudaError_t launch_pow2_bulk(const void* in, void* out, int out_mode, int64_t nrows, const void* tw, double scale,
                             double accum_scale, const void* sc_in, const void* sc_out, const int* skip, int* err,
                             cudaStream_t st) {
  constexpr int N = 1 << LOG2N;
  const size_t smem = (size_t)(2 * N + N + N / 16) * sizeof(float2);
  auto k = k_dft_rows_pow2_bulk<LOG2N, SIGN>;
  const cudaError_t e = allow_dynamic_smem((const void*)k, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, pow2_threads<LOG2N>(), smem);
  const int64_t grid = std::min<int64_t>(nrows, (int64_t)std::max(1, nsm) * std::max(1, per_sm));
  if (grid <= 0) return cudaSuccess;
  k<<<(unsigned)grid, pow2_threads<LOG2N>(), smem, st>>>((const float2*)in, out, out_mode, nrows, (const float2*)tw,
                                                         (float)scale, accum_scale, (const float2*)sc_in,
                                                         (const float2*)sc_out, skip, err);
  return cudaGetLastError();
}

template <typename T, int LOG2N, int SIGN>
cudaError_t launch_pow2_t(const void* in, int in_is_double, void* out, int out_mode, int64_t nrows,
                          const void* tw, double scale, double accum_scale, const void* sc_in, const void* sc_out,
                          const int* skip, cudaStream_t st) {
  using C = typename cpx<T>::type;
  constexpr int N = 1 << LOG2N;
  constexpr int threads = pow2_threads<LOG2N>();
  constexpr int L = threads / (N / 16);
  constexpr int NP = (LOG2N + 3) / 4;
  const size_t smem = NP > 1 ? (size_t)L * (N + N / 16) * sizeof(C) : 0;
  const int64_t grid = (nrows + L - 1) / L;
  if (grid == 0) return cudaSuccess;
  auto k = k_dft_rows_pow2<T, LOG2N, SIGN>;
  if (smem > 48 * 1024) {
    const cudaError_t e = allow_dynamic_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
  }
  k<<<(unsigned)grid, threads, smem, st>>>(in, in_is_double, out, out_mode, nrows, (const C*)tw, (T)scale,
                                           accum_scale, (const C*)sc_in, (const C*)sc_out, skip);
  return cudaGetLastError();
}

template <typename T, int SIGN>
cudaError_t launch_pow2_s(int log2n, const void* in, int in_is_double, void* out, int out_mode, int64_t nrows,
                          const void* tw, double scale, double accum_scale, const void* sc_in, const void* sc_out,
                          const int* skip, cudaStream_t st) {
#define HELM_POW2(LG)                                                                                       \
  case LG:                                                                                                  \
    return launch_pow2_t<T, LG, SIGN>(in, in_is_double, out, out_mode, nrows, tw, scale, accum_scale, sc_in, \
                                      sc_out, skip, st);
  switch (log2n) {
    HELM_POW2(4)
    HELM_POW2(5)
    HELM_POW2(6)
    HELM_POW2(7)
    HELM_POW2(8)
    HELM_POW2(9)
    HELM_POW2(10)
    HELM_POW2(11)
    HELM_POW2(12)
    HELM_POW2(13)
    default:
      return cudaErrorInvalidValue;
  }
#undef HELM_POW2
}

}  // namespace

bool dft_rows_pow2_supported(int64_t n) { return n >= 16 && n <= 8192 && (n & (n - 1)) == 0; }
bool dft_cols_pow2_supported(int64_t n) { return n >= 16 && n <= 1024 && (n & (n - 1)) == 0; }

cudaError_t launch_dft_cols_pow2(int prec, const void* in, int in_is_double, void* out, int out_mode, int64_t outer,
                                 int64_t inner, int64_t n, const void* tw, int sign, double scale, double accum_scale,
                                 const void* sc_in, const void* sc_out, const int* skip, cudaStream_t st) {
  if (!dft_cols_pow2_supported(n)) return cudaErrorInvalidValue;
  int log2n = 0;
  while ((int64_t(1) << log2n) < n) ++log2n;
  if (prec == kPrecF64) {
    return sign < 0 ? launch_cols_pow2_s<double, -1>(log2n, in, in_is_double, out, out_mode, outer, inner, tw, scale,
                                                      accum_scale, sc_in, sc_out, skip, st)
                    : launch_cols_pow2_s<double, 1>(log2n, in, in_is_double, out, out_mode, outer, inner, tw, scale,
                                                     accum_scale, sc_in, sc_out, skip, st);
  }
  return sign < 0 ? launch_cols_pow2_s<float, -1>(log2n, in, in_is_double, out, out_mode, outer, inner, tw, scale,
                                                 accum_scale, sc_in, sc_out, skip, st)
                  : launch_cols_pow2_s<float, 1>(log2n, in, in_is_double, out, out_mode, outer, inner, tw, scale,
                                                accum_scale, sc_in, sc_out, skip, st);
}

cudaError_t launch_dft_rows_pow2(int prec, const void* in, int in_is_double, void* out, int out_mode, int64_t nrows,
                                 int64_t n, const void* tw, int sign, double scale, double accum_scale,
                                 const void* sc_in, const void* sc_out, const int* skip, cudaStream_t st, int* err) {
  if (!dft_rows_pow2_supported(n)) return cudaErrorInvalidValue;
  int log2n = 0;
  while ((int64_t(1) << log2n) < n) ++log2n;
  // long complex64 lines: the persistent kernel with bulk prefetch
  if (prec == kPrecF32 && in_is_double == kInC64 && err && (log2n == 12 || log2n == 13)) {
    if (log2n == 12)
      return sign < 0 ? launch_pow2_bulk<12, -1>(in, out, out_mode, nrows, tw, scale, accum_scale, sc_in, sc_out, skip,
                                                 err, st)
                      : launch_pow2_bulk<12, 1>(in, out, out_mode, nrows, tw, scale, accum_scale, sc_in, sc_out, skip,
                                                err, st);
    return sign < 0 ? launch_pow2_bulk<13, -1>(in, out, out_mode, nrows, tw, scale, accum_scale, sc_in, sc_out, skip,
                                               err, st)
                    : launch_pow2_bulk<13, 1>(in, out, out_mode, nrows, tw, scale, accum_scale, sc_in, sc_out, skip,
                                              err, st);
  }
  if (prec == kPrecF64) {
    return sign < 0 ? launch_pow2_s<double, -1>(log2n, in, in_is_double, out, out_mode, nrows, tw, scale,
                                                 accum_scale, sc_in, sc_out, skip, st)
                    : launch_pow2_s<double, 1>(log2n, in, in_is_double, out, out_mode, nrows, tw, scale,
                                                accum_scale, sc_in, sc_out, skip, st);
  }
  return sign < 0 ? launch_pow2_s<float, -1>(log2n, in, in_is_double, out, out_mode, nrows, tw, scale, accum_scale,
                                            sc_in, sc_out, skip, st)
                  : launch_pow2_s<float, 1>(log2n, in, in_is_double, out, out_mode, nrows, tw, scale, accum_scale,
                                           sc_in, sc_out, skip, st);
}

}  // namespace helm
