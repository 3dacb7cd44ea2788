// Host launchers for the batched DFT kernels and the 2D/3D solve kernels.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>

#include "helm_internal.h"

namespace helm {

enum { kPrecF64 = 0, kPrecF32 = 1 };
enum { kOutC128 = 0, kOutC64 = 1, kOutAccumC128 = 2, kOutFF = 3, kOutAccumFF = 4 };
// Input kinds (the in_is_double argument): complex64, complex128, or a
// float-float complex vector (float4 per point: re_hi, im_hi, re_lo, im_lo),
// of which the transform reads the leading (hi) part.
enum { kInC64 = 0, kInC128 = 1, kInFF = 2 };

bool dft_supported(const DftPlan& p, size_t elem_bytes, int max_smem);
// A length whose factorisation has a prime above 64 is transformed by
// Bluestein's chirp-z method; its power-of-two convolution length (>= 2n - 1).
bool dft_needs_bluestein(const DftPlan& p);

// Tensor-core (tcgen05, kind::tf32 with high/low operand splitting) dense
// DFT of complex64 lines of n <= kDftGemmMaxN points; see helm_dft_tc.cu.
constexpr int kDftGemmMaxN = 128;
bool dft_gemm_supported(int64_t n);
// Floats of one table (one direction) for length n.
size_t dft_gemm_table_floats(int64_t n);
// The table of the matrix W (n x n, input index major, FP64) in the kernel's
// operand layout.
void dft_gemm_table(int64_t n, const std::complex<double>* W, float* out);
// nrows lines: in (kInC64 / kInC128) times the table's matrix to out
// (kOutC64, kOutC128 or kOutAccumC128 with accum_scale).
cudaError_t launch_dft_rows_tc(const float* table, int64_t n, const void* in, int in_is_double, void* out,
                               int out_mode, int64_t nrows, double accum_scale, const int* skip, cudaStream_t st,
                               int* err);
int64_t bluestein_length(int64_t n);

// Lines along the contiguous (last) axis: nrows lines of length p.n.
// in: of kind in_is_double (kIn*); computed in `prec`; out per out_mode
// (kOutAccumC128: out += accum_scale * result; kOutFF: float-float vector
// (result, 0); kOutAccumFF: float-float out += accum_scale * result).  sign -1 forward,
// +1 inverse; `scale` multiplies the transform.  skip: optional device flag,
// the kernel returns at once when *skip != 0.
// sc_in / sc_out: optional per-point complex factors (length p.n, compute
// precision) applied to the input before and to the output after the
// transform: the diagonal scalings of the gamma-circulant auxiliary.
// err: optional device error word; when given, complex64 input lines of 4096
// or 8192 points use a persistent kernel fed by bulk copies with bounded
// waits, which report there.
cudaError_t launch_dft_rows(int prec, const void* in, int in_is_double, void* out, int out_mode,
                            int64_t nrows, const DftPlan& p, const void* tw, int sign, double scale,
                            double accum_scale, const void* sc_in, const void* sc_out, const int* skip,
                            cudaStream_t st, int* err = nullptr);

// Power-of-two lines (16 <= n <= 8192) along the contiguous axis: the same
// contract as launch_dft_rows with the radices fixed at compile time.
bool dft_rows_pow2_supported(int64_t n);
cudaError_t launch_dft_rows_pow2(int prec, const void* in, int in_is_double, void* out, int out_mode, int64_t nrows,
                                 int64_t n, const void* tw, int sign, double scale, double accum_scale,
                                 const void* sc_in, const void* sc_out, const int* skip, cudaStream_t st,
                                 int* err = nullptr);

// Power-of-two lines (16 <= n <= 1024) along a middle axis: the contract of
// launch_dft_cols with compile-time radices; in place (out == in) allowed.
bool dft_cols_pow2_supported(int64_t n);
cudaError_t launch_dft_cols_pow2(int prec, const void* in, int in_is_double, void* out, int out_mode, int64_t outer,
                                 int64_t inner, int64_t n, const void* tw, int sign, double scale, double accum_scale,
                                 const void* sc_in, const void* sc_out, const int* skip, cudaStream_t st);

// Lines along a middle axis: the array viewed as [outer][p.n][inner].
cudaError_t launch_dft_cols(int prec, const void* in, int in_is_double, void* out, int out_mode,
                            int64_t outer, int64_t inner, const DftPlan& p, const void* tw, int sign,
                            double scale, double accum_scale, const void* sc_in, const void* sc_out,
                            const int* skip, cudaStream_t st);

}  // namespace helm
