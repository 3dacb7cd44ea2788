// Host launchers for the batched DFT kernels and the 2D/3D solve kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "helm_internal.h"

namespace helm {

enum { kPrecF64 = 0, kPrecF32 = 1 };
enum { kOutC128 = 0, kOutC64 = 1, kOutAccumC128 = 2 };

bool dft_supported(const DftPlan& p, size_t elem_bytes, int max_smem);

// Lines along the contiguous (last) axis: nrows lines of length p.n.
// in: complex128 if in_is_double else complex64; computed in `prec`; out per
// out_mode (kOutAccumC128: out += accum_scale * result).  sign -1 forward,
// +1 inverse; `scale` multiplies the transform.  skip: optional device flag,
// the kernel returns at once when *skip != 0.
// sc_in / sc_out: optional per-point complex factors (length p.n, compute
// precision) applied to the input before and to the output after the
// transform: the diagonal scalings of the gamma-circulant auxiliary.
cudaError_t launch_dft_rows(int prec, const void* in, int in_is_double, void* out, int out_mode,
                            int64_t nrows, const DftPlan& p, const void* tw, int sign, double scale,
                            double accum_scale, const void* sc_in, const void* sc_out, const int* skip,
                            cudaStream_t st);

// Lines along a middle axis: the array viewed as [outer][p.n][inner].
cudaError_t launch_dft_cols(int prec, const void* in, int in_is_double, void* out, int out_mode,
                            int64_t outer, int64_t inner, const DftPlan& p, const void* tw, int sign,
                            double scale, double accum_scale, const void* sc_in, const void* sc_out,
                            const int* skip, cudaStream_t st);

}  // namespace helm
