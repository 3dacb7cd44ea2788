// Short DFTs along the contiguous axis as dense matrix products on the 5th-
// generation tensor cores (tcgen05, kind::tf32), a variant of the transforms
// of eqs. step1FFTfcoeff / step3IFFTz3coeff for lines of at most 128 points.
//
// A line of n complex values is a row of 2n reals [re_0, im_0, re_1, ...];
// its transform is that row times the real 2n x 2n matrix of the complex
// DFT matrix W (with the auxiliary's diagonal scalings and the inverse's 1/n
// folded in), so 128 lines at a time are one (128 x 2n) x (2n x 2n) product.
// TF32 keeps 11 significant bits, so each operand is split into a TF32 high
// part and a TF32 low part (the remainder) and the product is accumulated
// from the three terms hi*hi + hi*lo + lo*hi in FP32 (22-bit operands; the
// rounding of a dense DFT grows like sqrt(n), an FFT's like log n).
//
// Per CTA (128 threads, thread t owns line 128 b + t and TMEM lane t):
//   * one warp allocates the FP32 accumulator in tensor memory (128 lanes x
//     N columns);
//   * for each 32-wide K chunk: thread 0 brings the chunk of W (high and low
//     parts, already in the shared-memory layout the tensor cores read) by one
//     bulk copy; every thread splits its line's chunk into high and low parts
//     and stores them in that layout; thread 0 issues the 3 x 4 MMAs
//     (K = 8 each) and commits them to an mbarrier;
//   * each warp reads its 32 accumulator lanes (tcgen05.ld) and writes its
//     lines in the requested output mode.
// Shared-memory operands use the K-major layout without swizzling: 8-row x
// 16-byte core matrices, 128 bytes apart along K and 1024 bytes apart along
// the rows.  Every wait is bounded; on a timeout the CTA stops, lets its copy
// and products in flight finish (bounded), frees its tensor memory and sets
// the error word.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "helm_async.cuh"
#include "helm_dft.h"
#include "helm_kernels.cuh"

namespace helm {

namespace {

constexpr int kTcM = 128;                // lines per CTA = MMA M = threads
constexpr int kTcKc = 32;                // K chunk in FP32 elements (128 bytes of a row)
constexpr int kTcRowChunkBytes = kTcKc * 4;
constexpr int kTcGroupBytes = 8 * kTcRowChunkBytes;  // 8 rows of a chunk: 8 core matrices along K

// Byte offset of element (row, k), k < 32, in a [rows][32] FP32 chunk laid
// out as core matrices (K-major, no swizzle).
__host__ __device__ __forceinline__ uint32_t tc_off(int row, int k) {
  return (uint32_t)((row >> 3) * kTcGroupBytes + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices along K: 128), stride-dimension byte offset
// (between 8-row groups: 1024), the fixed version bits, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(kTcGroupBytes >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D in FP32, A and B TF32, both
// K-major, N and M.
__host__ __device__ constexpr uint32_t tc_idesc(int n, int m) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (tensor memory) (+)= A * B^T, A and B described in shared memory.
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The mbarrier completes once every MMA issued so far by this thread is done.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// w: per K chunk, the high then the low part of the B operand ([np][32]
// core-matrix layout each); np = N (a multiple of 16), nchunks = K / 32.
__global__ void __launch_bounds__(kTcM) k_dft_rows_tc(const float* __restrict__ w, int n, int np, int nchunks,
                                                      uint32_t tcols, const void* __restrict__ in, int in_is_double,
                                                      void* __restrict__ out, int out_mode, int64_t nrows,
                                                      double accum_scale, const int* __restrict__ skip, int* err) {
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char tsm[];
  unsigned char* sA = tsm;                                 // [2][128][32] high, low
  unsigned char* sB = sA + 2 * kTcM * kTcRowChunkBytes;    // [2][np][32] high, low
  const uint32_t bbytes = (uint32_t)np * kTcRowChunkBytes;  // one part of a B chunk
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + 2 * bbytes);  // [0] B chunk landed, [1] products done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int t = threadIdx.x, warp = t >> 5;
  const int64_t row = (int64_t)blockIdx.x * kTcM + t;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tc_idesc(np, kTcM);
  bool failed = false;
  int copies = 0, commits = 0;  // thread 0: chunks copied / product groups committed
  int c = 0;
  for (; c < nchunks; ++c) {
    bool ok = true;
    if (c > 0) ok = mbar_wait_bounded(&bar[1], (uint32_t)((c - 1) & 1), err);  // sA, sB free again
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (t == 0) {
      mbar_arrive_expect_tx(&bar[0], 2 * bbytes);
      bulk_g2s(sB, w + (size_t)c * 2 * bbytes / sizeof(float), 2 * bbytes, &bar[0]);
      copies = c + 1;
    }
    // this line's values [16 c, 16 c + 16) as reals [32 c, 32 c + 32)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float x[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 16 * c + 2 * q + h;
        if (row < nrows && j < n) {
          if (in_is_double == kInC128) {
            const double2 v = reinterpret_cast<const double2*>(in)[row * n + j];
            x[2 * h] = (float)v.x;
            x[2 * h + 1] = (float)v.y;
          } else {
            const float2 v = reinterpret_cast<const float2*>(in)[row * n + j];
            x[2 * h] = v.x;
            x[2 * h + 1] = v.y;
          }
        }
      }
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        hi[e] = tf32_rna(x[e]);
        lo[e] = tf32_rna(x[e] - __uint_as_float(hi[e]));
      }
      const uint32_t o = tc_off(t, 4 * q);
      *reinterpret_cast<uint4*>(sA + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(sA + kTcM * kTcRowChunkBytes + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    fence_proxy_async_smem();  // the stores above, then the tensor cores' reads
    __syncthreads();
    if (t == 0) {
      if (mbar_wait_bounded(&bar[0], (uint32_t)(c & 1), err)) {
        tc_fence_after();
        const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
#pragma unroll
        for (int ks = 0; ks < kTcKc / 8; ++ks) {  // K = 8 per MMA: two core matrices, 256 bytes
          const uint64_t ah = tc_desc(a0 + ks * 256), al = tc_desc(a0 + kTcM * kTcRowChunkBytes + ks * 256);
          const uint64_t bh = tc_desc(b0 + ks * 256), bl = tc_desc(b0 + bbytes + ks * 256);
          tc_mma(tmem, ah, bh, idesc, (c | ks) ? 1u : 0u);
          tc_mma(tmem, ah, bl, idesc, 1u);
          tc_mma(tmem, al, bh, idesc, 1u);
        }
        tc_commit(&bar[1]);
        commits = c + 1;
      }
      // a copy that did not land: no commit, so the next wait (or the one
      // after the loop) runs out for every thread
    }
  }
  bool ok = !failed && mbar_wait_bounded(&bar[1], (uint32_t)((nchunks - 1) & 1), err);
  if (__syncthreads_or(!ok)) failed = true;
  if (failed) {
    if (t == 0) {
      // let the last copy and the committed products finish before the
      // shared and tensor memory are released
      if (copies > 0) mbar_wait_bounded(&bar[0], (uint32_t)((copies - 1) & 1), nullptr);
      if (commits > 0) mbar_wait_bounded(&bar[1], (uint32_t)((commits - 1) & 1), nullptr);
    }
  } else {
    tc_fence_after();
    // lane t of warp w holds line 32 w + t: columns 2k, 2k + 1 are output k
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    for (int c0 = 0; c0 < np; c0 += 16) {
      float v[16];
      tmem_ld16(lane_base + (uint32_t)c0, v);
      if (row < nrows) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = c0 / 2 + i;
          if (k < n) {
            const int64_t e = row * n + k;
            if (out_mode == kOutC64) {
              reinterpret_cast<float2*>(out)[e] = make_float2(v[2 * i], v[2 * i + 1]);
            } else if (out_mode == kOutC128) {
              reinterpret_cast<double2*>(out)[e] = make_double2(v[2 * i], v[2 * i + 1]);
            } else {  // kOutAccumC128
              double2 u = reinterpret_cast<double2*>(out)[e];
              u.x += accum_scale * (double)v[2 * i];
              u.y += accum_scale * (double)v[2 * i + 1];
              reinterpret_cast<double2*>(out)[e] = u;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tmem, tcols);
}

// TF32 rounding of x, to nearest with ties away from zero (the rounding the
// kernel's cvt.rna applies to the line values).
float tf32_round_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace

bool dft_gemm_supported(int64_t n) { return n >= 2 && n <= kDftGemmMaxN; }

size_t dft_gemm_table_floats(int64_t n) {
  const int64_t np = (2 * n + 15) / 16 * 16, kp = (2 * n + kTcKc - 1) / kTcKc * kTcKc;
  return (size_t)(kp / kTcKc) * 2 * (size_t)np * kTcKc;
}

// W[j][k] (input j, output k) given in FP64 as w(j, k); the B operand is the
// transpose of the real 2n x 2n matrix of W, split into TF32 high and low
// parts, chunked along K and laid out as the kernel's shared memory.
void dft_gemm_table(int64_t n, const std::complex<double>* W, float* out) {
  const int np = (int)((2 * n + 15) / 16 * 16), kp = (int)((2 * n + kTcKc - 1) / kTcKc * kTcKc);
  const int nchunks = kp / kTcKc;
  const size_t part = (size_t)np * kTcKc;  // floats of one part of a chunk
  std::memset(out, 0, sizeof(float) * nchunks * 2 * part);
  for (int kk = 0; kk < 2 * (int)n; ++kk)     // input real index (K)
    for (int nn = 0; nn < 2 * (int)n; ++nn) {  // output real index (N)
      const std::complex<double> v = W[(size_t)(kk >> 1) * n + (nn >> 1)];
      // real block of the complex product: [re -im; im re] acting on [x_re, x_im]
      const double r = (kk & 1) == 0 ? ((nn & 1) == 0 ? v.real() : v.imag()) : ((nn & 1) == 0 ? -v.imag() : v.real());
      const float f = (float)r;
      const float hi = tf32_round_host(f);
      const float lo = tf32_round_host((float)(r - (double)hi));
      const int c = kk / kTcKc, kl = kk % kTcKc;
      const size_t base = (size_t)c * 2 * part;
      out[base + tc_off(nn, kl) / 4] = hi;
      out[base + part + tc_off(nn, kl) / 4] = lo;
    }
}

cudaError_t launch_dft_rows_tc(const float* table, int64_t n, const void* in, int in_is_double, void* out,
                               int out_mode, int64_t nrows, double accum_scale, const int* skip, cudaStream_t st,
                               int* err) {
  if (!dft_gemm_supported(n) || nrows < 0) return cudaErrorInvalidValue;
  if (nrows == 0) return cudaSuccess;
  const int np = (int)((2 * n + 15) / 16 * 16), kp = (int)((2 * n + kTcKc - 1) / kTcKc * kTcKc);
  uint32_t tcols = 32;
  while ((int)tcols < np) tcols <<= 1;
  // shared memory: operands, two barriers, the tensor-memory address; padded
  // so that no more CTAs share an SM than its 512 tensor-memory columns hold
  size_t smem = (size_t)2 * kTcM * kTcRowChunkBytes + (size_t)2 * np * kTcRowChunkBytes + 32;
  int dev = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const size_t per_sm = 512 / tcols;  // CTAs whose accumulators fit at once
  smem = std::max(smem, (size_t)smem_sm / (per_sm + 1) + 1024);
  cudaError_t e = allow_dynamic_smem((const void*)k_dft_rows_tc, smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = (nrows + kTcM - 1) / kTcM;
  k_dft_rows_tc<<<(unsigned)grid, kTcM, smem, st>>>(table, (int)n, np, kp / kTcKc, tcols, in, in_is_double, out,
                                                     out_mode, nrows, accum_scale, skip, err);
  return cudaGetLastError();
}

}  // namespace helm
