// Internal declarations shared by the host plan code and the CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "helm.h"

namespace helm {

constexpr int kMaxStages = 24;

// Counted device allocations of plan memory (helm_alloc.cpp): the library
// allocates and frees device memory only through these.
cudaError_t dmalloc(void** ptr, size_t bytes);
void dfree(void* ptr);
// Lets `func` launch with up to `bytes` of dynamic shared memory on the
// current device.  The attribute is process-wide, so it is only ever raised
// (under a lock): threads that launch the same kernel with different sizes
// (a plan build beside a served solve) cannot lower it under one another.
cudaError_t allow_dynamic_smem(const void* func, size_t bytes);

// Mixed-radix factorisation of a DFT length: 8, 4, 2 first, then odd primes.
struct DftPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
  // Lengths with a prime factor above 64 (Bluestein's chirp-z transform):
  // bm = the power-of-two convolution length (0: not used), its radices, and
  // device tables in the plan's compute precision: bw the chirp
  // e^{i pi j^2 / n} (n values), bf[0] / bf[1] the length-bm DFT of the chirp
  // sequence for the forward / inverse transform, scaled by 1/bm, btw the
  // twiddles e^{-2 pi i k / bm}.
  int bm;
  int bstages;
  int bradix[kMaxStages];
  const void* bw;
  const void* bf[2];
  const void* btw;
  // Tensor-core variant (complex64 lines of at most 128 points): gw[0] /
  // gw[1] the forward / inverse matrix tables of launch_dft_rows_tc (null:
  // not built), made with the FP32 scalings gsc[0] (input, forward) and
  // gsc[1] (output, inverse) and the inverse's scale gscale folded in; used
  // only by calls that pass exactly those.
  const float* gw[2];
  const void* gsc[2];
  double gscale;
};

int dft_factor(int64_t n, DftPlan* p);

// Eigen-data of the absorbing 1D pencil (see helm_eigen.cpp).
// mden: the mass matrix denominator (6: the paper's elements, 12: the
// modified ones; see MassCoef).
int abc_eigen(int64_t n, double h, double omega, double* lam, double* sigma, int8_t* parity, double mden = 6.0);

// abc_eigen in a caller workspace of >= 2n + 9 ceil(n/2) + 16 doubles,
// single-threaded, no heap use.
int abc_eigen_static(int64_t n, double h, double omega, double* lam, double* sigma, int8_t* parity, double* work,
                     int64_t work_len);

// e^{-2 pi i k / n}, k = 0..n-1.
void unit_roots(int64_t n, double* re, double* im);

// Per-axis eigen-data of an axis that carries a periodic auxiliary
// (the paper's x1 in 2D; x1 and x2 in 3D), stored on the device as doubles.
//
// The auxiliary is the gamma-circulant pencil (K^B_g, M^B_g): the circulant
// matrices of eqs. matrixKper / matrixMper with the wrap-around entries
// multiplied by g (last row) and 1/g (first row), g = e^{n t},
// t = (rho + i q pi/2)/n.  g = 1 (rho = q = 0) is the paper's periodic
// auxiliary.  It is diagonalised by F D^-1 with D = diag(e^{t j}):
//   K^B_g = D F^-1 diag(kappa_l) F D^-1,  kappa_l = (2 - 2 cosh(t + i theta_l))/h,
//   M^B_g = D F^-1 diag(mu_l) F D^-1,     mu_l = h (4 + 2 cosh(t + i theta_l))/6.
struct AxisData {
  int64_t n = 0;
  double h = 0;
  double wc = 0;   // w of this axis's absorbing end rows (0: Neumann axis, Gamma_N)
  double rho = 0;  // damping of the auxiliary (0: periodic)
  int q = 0;       // phase of the auxiliary in quarter turns
  // device arrays (double)
  double* lamB = nullptr;   // Lam^B_l = kappa_l / mu_l, complex (re, im)
  double* invmu = nullptr;  // 1 / mu_l, complex
  double* sc_in = nullptr;  // e^{-t j}, j = 0..n-1, complex (nullptr when g = 1)
  double* sc_out = nullptr; // e^{+t j}
  float* sc_in32 = nullptr;
  float* sc_out32 = nullptr;
  double en[2] = {1, 0};     // e^{t (n-1)}
  double eninv[2] = {1, 0};  // e^{-t (n-1)}
  double g[2] = {1, 0};      // e^{n t}
  double ginv[2] = {1, 0};   // e^{-n t}
  double* lamA = nullptr;   // absorbing eigenvalues (re, im) interleaved (eq. EVP1a)
  double* sigA = nullptr;   // V[1,l]^2 (re, im) interleaved (eq. EVPcondA)
  double* parA = nullptr;   // +-1 : V[n,l] = par * V[1,l]
  double* tw = nullptr;     // e^{-2 pi i k/n} (re, im) interleaved, FP64
  float* tw32 = nullptr;    // same, FP32
  void* bs[4] = {nullptr, nullptr, nullptr, nullptr};  // Bluestein tables of dft (chirp, 2 spectra, twiddles)
  float* gemm[2] = {nullptr, nullptr};                  // tensor-core DFT tables of dft (forward, inverse)
  DftPlan dft{};
};

}  // namespace helm
