// Internal declarations shared by the host plan code and the CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include "helm.h"

namespace helm {

constexpr int kMaxStages = 24;

// Mixed-radix factorisation of a DFT length: 8, 4, 2 first, then odd primes.
struct DftPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
};

int dft_factor(int64_t n, DftPlan* p);

// Eigen-data of the absorbing 1D pencil (see helm_eigen.cpp).
int abc_eigen(int64_t n, double h, double omega, double* lam, double* sigma, int8_t* parity);

// e^{-2 pi i k / n}, k = 0..n-1.
void unit_roots(int64_t n, double* re, double* im);

// Per-axis eigen-data of an axis that carries a periodic auxiliary
// (the paper's x1 in 2D; x1 and x2 in 3D), stored on the device as doubles.
struct AxisData {
  int64_t n = 0;
  double h = 0;
  // device arrays (double)
  double* lamB = nullptr;   // periodic eigenvalues Lam^B_l = kappa_l / mu_l (eq. eigvaluesPer)
  double* muB = nullptr;    // mu_l = h (4 + 2 cos theta_l) / 6, eigenvalues of M^B
  double* lamA = nullptr;   // absorbing eigenvalues (re, im) interleaved (eq. EVP1a)
  double* sigA = nullptr;   // V[1,l]^2 (re, im) interleaved (eq. EVPcondA)
  double* parA = nullptr;   // +-1 : V[n,l] = par * V[1,l]
  double* tw = nullptr;     // e^{-2 pi i k/n} (re, im) interleaved, FP64
  float* tw32 = nullptr;    // same, FP32
  DftPlan dft{};
};

}  // namespace helm
