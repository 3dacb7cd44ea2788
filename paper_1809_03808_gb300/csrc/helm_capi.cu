// C ABI of the fast Helmholtz solver: plan construction (the paper's
// initialisation), solve orchestration (Steps 1-3 of Sections 4.2 / 5.2),
// mixed-precision refinement, host-buffer and step-by-step variants.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "helm.h"
#include "helm_dft.h"
#include "helm_internal.h"
#include "helm_solve.h"
#include "helm_prof.h"
#include "helm_solve3d.h"
#include "helm_async.cuh"

using namespace helm;

struct helm_plan {
  int dim = 2;
  int64_t n[3] = {1, 1, 1};
  double h[3] = {0, 0, 0};
  double omega = 0;
  int32_t bc[3] = {HELM_BC_ABC, HELM_BC_ABC, HELM_BC_ABC};  // boundary kind of each axis (both faces)
  double wc[3] = {0, 0, 0};  // w of each axis's absorbing ends: omega, or 0 on a Neumann axis
  int dtype = HELM_C128;
  int prec = kPrecF64;  // compute precision of the solves
  cudaStream_t stream = nullptr;
  // 2D: x1 = axis 1 (ax[0] below); 3D: outer x1 = axis 1 (y), inner x2 = axis 2 (z)
  AxisData axo;  // outer periodic axis
  AxisData axi;  // inner periodic axis (3D only)
  // device buffers
  void* fhat = nullptr;
  void* cbuf = nullptr;
  void* dbuf = nullptr;
  void* partial = nullptr;
  void* faces = nullptr;  // v (2 faces), w (2 faces), c (2 faces), scratch
  void* ustartB = nullptr;  // 2D: pivot entering each chunk, B-type lines
  void* ustartA = nullptr;  // 2D: same for A-type lines
  void* rec = nullptr;      // 2D: chunk records
  void* tabB = nullptr;     // 2D: per-plan line tables, B-type lines (Steps 1, 3)
  void* tabA = nullptr;     // 2D: same, A-type lines (Step 2)
  void* constB = nullptr;   // 2D: per-line constants, B-type lines
  void* constA = nullptr;   // 2D: per-line constants, A-type lines
  int64_t face_len = 0;   // values per face
  int64_t nwarps = 0;
  float2* rbuf = nullptr;
  double* sums = nullptr;
  RefineState* state = nullptr;
  double2* host_f = nullptr;  // staging for helm_solve_host (allocated on first use)
  double2* host_u = nullptr;
  cudaStream_t out_stream = nullptr;  // helm_solve_host: the early copy of u to the host
  cudaEvent_t out_ready = nullptr, out_done = nullptr;
  size_t bytes = 0;
  double plan_seconds = 0;
  double tol = 1e-14;
  int max_iter = 10;
  double aux_trial_resid = -1.0;  // plan-time trial residual of the chosen auxiliary
  int* dev_err = nullptr;         // device error word of the kernels' bounded waits
  int resid_kind = HELM_RESID_FP64;
  float4* ffb = nullptr;  // float-float refinement: f (hi, lo) ...
  float4* ufb = nullptr;  // ... and the accumulated u
  // refinement loop as a CUDA graph (see build_refine_graph)
  bool use_graphs = true;
  cudaStream_t cap[2] = {nullptr, nullptr};  // private capture streams
  cudaGraph_t rg_graph = nullptr;
  cudaGraphExec_t rg_exec = nullptr;
  const void* rg_f = nullptr;  // f, u baked into the graph (FP64 residual)
  void* rg_u = nullptr;
  uint64_t version = 0;  // bumped by every setting a captured solve depends on
  Plan3D p3;
  Profiler prof;
  std::string err;
  // helm_solve_many: extra workspaces (plans sharing this plan's operator
  // data: eigen-data, pivot tables, routing), one stream each, and the
  // events that fork them from and join them to the plan's stream.  A
  // workspace has `parent` set and owns only the allocations in `owned`.
  helm_plan* parent = nullptr;
  std::vector<void*> owned;
  std::vector<helm_plan*> ws;
  std::vector<cudaStream_t> ws_stream;
  std::vector<cudaEvent_t> ws_done;
  cudaEvent_t fork = nullptr;
  int rhs_concurrency = 4;
  int dft_gemm = 0;  // HELM_VARIANT_DFT: row transforms on the tensor cores
  int element = HELM_ELEMENT_Q1;  // helm_element of the plan
  double mden = 6.0;              // its mass matrix denominator (MassCoef)
  int tri_regs = 0;  // 2D complex64: register-tile passes (variant HELM_VARIANT_TRI2D = 1)
  int last_many = 0;  // workspaces used by the last helm_solve_many (0: none)
};

// A group of plans solved as one CUDA graph (helm_batch_*).
struct helm_batch {
  std::vector<helm_plan*> plans;
  cudaStream_t stream = nullptr;            // launch stream
  cudaStream_t cap[2] = {nullptr, nullptr};  // private capture streams
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> kf;  // pointers and plan settings baked into the graph
  std::vector<void*> ku;
  std::vector<uint64_t> kv;
  std::string err;
};

namespace {

int cuda_fail(helm_plan* p, cudaError_t e, const char* what) {
  if (p) {
    p->err = std::string(what) + ": " + cudaGetErrorString(e);
  }
  return HELM_ECUDA;
}

#define HELM_CK(call)                                             \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return cuda_fail(p, e_, #call);        \
  } while (0)
// HELM_CK with per-kernel event timing when profiling is enabled
#define HELM_PK(name, call)                                       \
  do {                                                            \
    ProfScope ps_(&p->prof, name, p->stream);                     \
    HELM_CK(call);                                                \
  } while (0)

int dev_alloc(helm_plan* p, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = dmalloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    p->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    *ptr = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HELM_ENOMEM : HELM_ECUDA;
  }
  p->bytes += bytes;
  return HELM_OK;
}

void free_axis(AxisData& a) {
  dfree(a.lamB);
  dfree(a.invmu);
  dfree(a.sc_in);
  dfree(a.sc_out);
  dfree(a.sc_in32);
  dfree(a.sc_out32);
  dfree(a.lamA);
  dfree(a.sigA);
  dfree(a.parA);
  dfree(a.tw);
  dfree(a.tw32);
  for (void* q : a.bs) dfree(q);
  for (float* q : a.gemm) dfree(q);
  a = AxisData{};
}

void free_dft_gemm(helm_plan* p, AxisData& a) {
  for (float*& q : a.gemm) {
    if (q) p->bytes -= dft_gemm_table_floats(a.n) * sizeof(float);
    dfree(q);
    q = nullptr;
  }
  a.dft.gw[0] = a.dft.gw[1] = nullptr;
  a.dft.gsc[0] = a.dft.gsc[1] = nullptr;
}

// Tables of the tensor-core transform of axis a (complex64 plans, lines of
// at most 128 points): forward W[j][k] = s_j e^{-2 pi i jk/n} with the input
// scaling s = e^{-t j}, inverse W[k][j] = (1/n) e^{+2 pi i jk/n} d_j with the
// output scaling d = e^{+t j} (eqs. step1FFTfcoeff, step3IFFTz3coeff with
// the auxiliary's D^-1, D folded in), in FP64 on the host.
int build_dft_gemm(helm_plan* p, AxisData& a) {
  free_dft_gemm(p, a);
  const int64_t n = a.n;
  if (!dft_gemm_supported(n)) return HELM_EUNSUPPORTED;
  using cd = std::complex<double>;
  std::vector<cd> si(n, cd(1, 0)), so(n, cd(1, 0));
  if (a.sc_in) {
    HELM_CK(cudaMemcpy(si.data(), a.sc_in, n * sizeof(cd), cudaMemcpyDeviceToHost));
    HELM_CK(cudaMemcpy(so.data(), a.sc_out, n * sizeof(cd), cudaMemcpyDeviceToHost));
  }
  const double tp = 2.0 * M_PI / (double)n;
  std::vector<cd> W((size_t)n * n);
  std::vector<float> tab(dft_gemm_table_floats(n));
  for (int dir = 0; dir < 2; ++dir) {
    for (int64_t j = 0; j < n; ++j)
      for (int64_t k = 0; k < n; ++k) {
        const double ang = tp * (double)((j * k) % n);
        if (dir == 0) W[(size_t)j * n + k] = si[j] * cd(std::cos(ang), -std::sin(ang));
        else W[(size_t)k * n + j] = so[j] * cd(std::cos(ang), std::sin(ang)) / (double)n;
      }
    dft_gemm_table(n, W.data(), tab.data());
    void* d = nullptr;
    if (int rc = dev_alloc(p, &d, tab.size() * sizeof(float))) return rc;
    a.gemm[dir] = static_cast<float*>(d);
    HELM_CK(cudaMemcpy(d, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  a.dft.gw[0] = a.gemm[0];
  a.dft.gw[1] = a.gemm[1];
  a.dft.gsc[0] = a.sc_in32;
  a.dft.gsc[1] = a.sc_out32;
  a.dft.gscale = 1.0 / (double)n;
  return HELM_OK;
}

// Default auxiliary: damped periodic wrap g = e^{rho + i q pi/2} (see helm.h):
// rho = 1, q = 1 in 2D and rho = 1, q = 0 in 3D (the choices that gave the
// smallest FP64 error and the fastest refinement on the benchmark grids).
constexpr double kDefaultAuxRho = 1.0;
constexpr int kDefaultAuxQ = 1;
constexpr int kDefaultAuxQ3D = 0;

int upload(helm_plan* p, double** d, const std::vector<double>& v) {
  if (!*d) {
    int r = dev_alloc(p, (void**)d, v.size() * sizeof(double));
    if (r) return r;
  }
  cudaError_t e = cudaMemcpy(*d, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? HELM_OK : cuda_fail(p, e, "cudaMemcpy plan tables");
}

int upload32(helm_plan* p, float** d, const std::vector<float>& v) {
  if (!*d) {
    int r = dev_alloc(p, (void**)d, v.size() * sizeof(float));
    if (r) return r;
  }
  cudaError_t e = cudaMemcpy(*d, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? HELM_OK : cuda_fail(p, e, "cudaMemcpy plan tables");
}

// Auxiliary (B) tables of one periodic axis for t = (rho + i q pi/2)/n:
// Lam^B_l = kappa_l/mu_l and 1/mu_l with kappa_l = -4 s^2/h,
// mu_l = h (1 + 2 s^2/3), s = sinh((t + i theta_l)/2) -- eq. eigvaluesPer for
// t = 0, written without cancellation at small theta -- and the scalings
// e^{-+t j} that turn the DFT into the transform of the gamma-circulant.
int build_axis_aux(helm_plan* p, AxisData& a, double rho, int q) {
  const int64_t n = a.n;
  const double h = a.h;
  a.rho = rho;
  a.q = ((q % 4) + 4) % 4;
  const double pi = 3.14159265358979323846;
  std::vector<double> r4re(4 * n), r4im(4 * n);  // e^{-2 pi i k/(4n)} = e^{-i pi k/(2n)}
  unit_roots(4 * n, r4re.data(), r4im.data());
  std::vector<double> lamB(2 * n), invmu(2 * n);
  const double ar = 0.5 * rho / (double)n;  // Re(t)/2
  for (int64_t l = 0; l < n; ++l) {
    // b = Im(t + i theta_l)/2 = (q pi/2 + 2 pi l)/(2n)
    const double b = (0.5 * pi * a.q + 2.0 * pi * (double)l) / (2.0 * (double)n);
    const std::complex<double> sh(std::sinh(ar) * std::cos(b), std::cosh(ar) * std::sin(b));
    const std::complex<double> s2 = sh * sh;
    const std::complex<double> kappa = -4.0 * s2 / h;
    // mu = h ((den - 2) + 2 cosh z)/den = h (1 + (4/den) sinh^2(z/2)),
    // den = 6 for the paper's elements
    const std::complex<double> mu = h * (1.0 + (4.0 / p->mden) * s2);
    const std::complex<double> lb = kappa / mu, im = 1.0 / mu;
    lamB[2 * l] = lb.real();
    lamB[2 * l + 1] = lb.imag();
    invmu[2 * l] = im.real();
    invmu[2 * l + 1] = im.imag();
  }
  int rc;
  if ((rc = upload(p, &a.lamB, lamB)) || (rc = upload(p, &a.invmu, invmu))) return rc;
  // e^{t j} = e^{rho j/n} e^{+i q pi j/(2n)}
  auto et = [&](int64_t j, double sign) -> std::complex<double> {
    const int64_t k = (a.q * j) % (4 * n);
    const std::complex<double> ph(r4re[k], -sign * r4im[k]);  // sign +1: conj(root) = e^{+i ..}
    return std::exp(sign * rho * (double)j / (double)n) * ph;
  };
  const std::complex<double> en = et(n - 1, +1.0), eninv = et(n - 1, -1.0);
  a.en[0] = en.real();
  a.en[1] = en.imag();
  a.eninv[0] = eninv.real();
  a.eninv[1] = eninv.imag();
  const double gr[4] = {1, 0, -1, 0}, gi[4] = {0, 1, 0, -1};  // e^{i q pi/2}
  a.g[0] = std::exp(rho) * gr[a.q];
  a.g[1] = std::exp(rho) * gi[a.q];
  a.ginv[0] = std::exp(-rho) * gr[a.q];
  a.ginv[1] = -std::exp(-rho) * gi[a.q];
  if (rho == 0.0 && a.q == 0) {
    dfree(a.sc_in);
    dfree(a.sc_out);
    dfree(a.sc_in32);
    dfree(a.sc_out32);
    a.sc_in = a.sc_out = nullptr;
    a.sc_in32 = a.sc_out32 = nullptr;
    return HELM_OK;
  }
  std::vector<double> si(2 * n), so(2 * n);
  std::vector<float> si32(2 * n), so32(2 * n);
  for (int64_t j = 0; j < n; ++j) {
    const std::complex<double> ei = et(j, -1.0), eo = et(j, +1.0);
    si[2 * j] = ei.real();
    si[2 * j + 1] = ei.imag();
    so[2 * j] = eo.real();
    so[2 * j + 1] = eo.imag();
    si32[2 * j] = (float)ei.real();
    si32[2 * j + 1] = (float)ei.imag();
    so32[2 * j] = (float)eo.real();
    so32[2 * j + 1] = (float)eo.imag();
  }
  if ((rc = upload(p, &a.sc_in, si)) || (rc = upload(p, &a.sc_out, so)) || (rc = upload32(p, &a.sc_in32, si32)) ||
      (rc = upload32(p, &a.sc_out32, so32)))
    return rc;
  return HELM_OK;
}

// Bluestein tables of an axis whose length has a prime factor above 64, in
// the compute precision `prec`: the chirp w_j = e^{i pi j^2/n} (j^2 reduced
// mod 2n in integers), the length-m DFTs of the chirp sequence b (b_j = w_j
// for |j| < n, cyclic) for the forward transform and of conj(b) for the
// inverse one, both divided by m, and the length-m twiddles.  FP64 on the
// host (the spectra by a direct O(m^2) sum).
int build_bluestein(helm_plan* p, AxisData& a, int prec) {
  const int64_t n = a.n, m = bluestein_length(n);
  const double pi = 3.14159265358979323846;
  std::vector<std::complex<double>> w(n), b(m, 0.0), f0(m), f1(m);
  for (int64_t j = 0; j < n; ++j) {
    const int64_t r = (j * j) % (2 * n);
    w[j] = std::polar(1.0, pi * (double)r / (double)n);
    b[j] = w[j];
    if (j) b[m - j] = w[j];
  }
  std::vector<double> rre(m), rim(m);
  unit_roots(m, rre.data(), rim.data());  // e^{-2 pi i k/m}
  for (int64_t k = 0; k < m; ++k) {
    std::complex<double> s0 = 0.0, s1 = 0.0;
    for (int64_t j = 0; j < m; ++j) {
      const int64_t e = (j * k) % m;
      const std::complex<double> t(rre[e], rim[e]);
      s0 += b[j] * t;
      s1 += std::conj(b[j]) * t;
    }
    f0[k] = s0 / (double)m;
    f1[k] = s1 / (double)m;
  }
  const size_t es = prec == kPrecF64 ? sizeof(double2) : sizeof(float2);
  auto put = [&](void** dst, const std::vector<std::complex<double>>& v) -> int {
    std::vector<char> host(v.size() * es);
    for (size_t i = 0; i < v.size(); ++i) {
      if (prec == kPrecF64) reinterpret_cast<double2*>(host.data())[i] = make_double2(v[i].real(), v[i].imag());
      else reinterpret_cast<float2*>(host.data())[i] = make_float2((float)v[i].real(), (float)v[i].imag());
    }
    if (int rc = dev_alloc(p, dst, host.size())) return rc;
    return cudaMemcpy(*dst, host.data(), host.size(), cudaMemcpyHostToDevice) == cudaSuccess ? HELM_OK : HELM_ECUDA;
  };
  std::vector<std::complex<double>> twm(m);
  for (int64_t k = 0; k < m; ++k) twm[k] = {rre[k], rim[k]};
  int rc;
  if ((rc = put(&a.bs[0], w)) || (rc = put(&a.bs[1], f0)) || (rc = put(&a.bs[2], f1)) || (rc = put(&a.bs[3], twm)))
    return rc;
  DftPlan mp;
  dft_factor(m, &mp);
  a.dft.bm = (int)m;
  a.dft.bstages = mp.nstages;
  for (int s = 0; s < mp.nstages; ++s) a.dft.bradix[s] = mp.radix[s];
  a.dft.bw = a.bs[0];
  a.dft.bf[0] = a.bs[1];
  a.dft.bf[1] = a.bs[2];
  a.dft.btw = a.bs[3];
  return HELM_OK;
}

// Eigen-data of one periodic axis (Section 3.2): absorbing-pencil eigen-data
// (eqs. EVP1a, EVPcondA; wc = 0: the Neumann pencil of a Gamma_N axis), DFT
// twiddles, and the auxiliary tables.
int build_axis(helm_plan* p, AxisData& a, int64_t n, double h, double wc, double rho, int q) {
  a.n = n;
  a.h = h;
  a.wc = wc;
  dft_factor(n, &a.dft);
  if (dft_needs_bluestein(a.dft))
    if (int rc = build_bluestein(p, a, p->prec)) return rc;
  std::vector<double> twre(n), twim(n);
  unit_roots(n, twre.data(), twim.data());
  std::vector<double> tw(2 * n), lamA(2 * n), sigA(2 * n), parA(n);
  std::vector<float> tw32(2 * n);
  std::vector<int8_t> par8(n);
  for (int64_t l = 0; l < n; ++l) {
    tw[2 * l] = twre[l];
    tw[2 * l + 1] = twim[l];
    tw32[2 * l] = (float)twre[l];
    tw32[2 * l + 1] = (float)twim[l];
  }
  int rc = abc_eigen(n, h, wc, lamA.data(), sigA.data(), par8.data(), p->mden);
  if (rc != HELM_OK) {
    p->err = "absorbing-pencil eigenvalue iteration failed";
    return rc;
  }
  for (int64_t l = 0; l < n; ++l) parA[l] = par8[l];
  if ((rc = upload(p, &a.lamA, lamA)) || (rc = upload(p, &a.sigA, sigA)) || (rc = upload(p, &a.parA, parA)) ||
      (rc = upload(p, &a.tw, tw)) || (rc = upload32(p, &a.tw32, tw32)))
    return rc;
  return build_axis_aux(p, a, rho, q);
}

int validate_common(double omega, int dtype) {
  if (!(omega > 0) || !std::isfinite(omega)) return HELM_EINVAL;
  if (dtype != HELM_C128 && dtype != HELM_C64_REFINED && dtype != HELM_C64_RAW) return HELM_EINVAL;
  return HELM_OK;
}

size_t cbytes(int prec) { return prec == kPrecF64 ? sizeof(double2) : sizeof(float2); }

Solve2DArgs args2d(const helm_plan* p) {
  const AxisData& ax = p->axo;
  Solve2DArgs a{p->n[0], p->n[1], p->h[0], p->h[1], p->omega, ax.lamB, ax.invmu, ax.lamA, ax.sigA, ax.parA, ax.tw,
                0, 0, {ax.eninv[0], ax.eninv[1]}};
  a.ch = p->prec == kPrecF64 ? kChunkF64 : kChunkF32;
  a.nchunks = (p->n[0] + a.ch - 1) / a.ch;
  a.wx = p->wc[0];
  a.wy = p->wc[1];
  a.tri_regs = p->tri_regs;
  a.mden = p->mden;
  return a;
}

// ---------------------------------------------------------------------------
// 2D solve: in (complex128 if in_is_double) -> out per out_mode.
// ---------------------------------------------------------------------------
int solve2d_core(helm_plan* p, const void* in, int in_is_double, void* out, int out_mode,
                 double accum_scale, const int* skip, void* dbg_fhat, void* dbg_v, void* dbg_w) {
  const int prec = p->prec;
  const int64_t nx = p->n[0], n1 = p->n[1];
  const size_t cb = cbytes(prec);
  const AxisData& ax = p->axo;
  const void* tw = prec == kPrecF64 ? (const void*)ax.tw : (const void*)ax.tw32;
  cudaStream_t st = p->stream;
  char* faces = (char*)p->faces;
  void* fv = faces;                 // v_1, v_n
  void* fw = faces + 2 * nx * cb;   // w_1, w_n
  void* fc = faces + 4 * nx * cb;   // c (or d)
  Solve2DArgs a = args2d(p);
  const int fhat_mode = prec == kPrecF64 ? kOutC128 : kOutC64;
  // a1: forward DFT along x1 (eq. step1FFTfcoeff), f_hat kept for Step 3
  const bool f64 = prec == kPrecF64;
  const void* sci = f64 ? (const void*)ax.sc_in : (const void*)ax.sc_in32;
  const void* sco = f64 ? (const void*)ax.sc_out : (const void*)ax.sc_out32;
  const double one[2] = {1.0, 0.0}, inv_n1[2] = {1.0 / (double)n1, 0.0};
  const double en_n1[2] = {ax.en[0] / (double)n1, ax.en[1] / (double)n1};
  const int64_t nparts = (n1 + 127) / 128;  // face partials: one per block of 128 lines
  HELM_PK("dft_fwd", launch_dft_rows(prec, in, in_is_double, p->fhat, fhat_mode, nx, ax.dft, tw, -1, 1.0, 0.0, sci,
                                     nullptr, skip, st, p->dev_err));
  if (dbg_fhat) HELM_CK(cudaMemcpyAsync(dbg_fhat, p->fhat, nx * n1 * cb, cudaMemcpyDeviceToDevice, st));
  // a2: Step 1
  if (p->tabB && prec == kPrecF64)
    HELM_CK(launch_tri2d_tab(1, p->fhat, nullptr, p->tabB, p->rec, nullptr, p->partial, a, skip, st, p->prof.on ? &p->prof : nullptr));
  else if (p->tabB)
    HELM_CK(launch_tri2d_t32(1, p->fhat, nullptr, p->tabB, p->rec, nullptr, p->partial, a, skip, st, p->prof.on ? &p->prof : nullptr,
                             p->constB, p->dev_err));
  else
    HELM_CK(launch_tri2d(prec, 1, p->fhat, nullptr, p->ustartB, p->rec, nullptr, p->partial, a, skip, st, p->prof.on ? &p->prof : nullptr, p->constB));
  HELM_PK("reduce_faces", launch_reduce_faces(prec, p->partial, fv, nx, nparts, inv_n1, en_n1, skip, st));
  if (dbg_v) HELM_CK(cudaMemcpyAsync(dbg_v, fv, 2 * nx * cb, cudaMemcpyDeviceToDevice, st));
  // a3: Step 2
  HELM_PK("apply_cbb", launch_apply_cbb(prec, fv, nullptr, fc, nx, p->h[0], p->h[1], p->wc[0], p->wc[1], p->omega * p->omega, ax.g,
                                        ax.ginv, skip, st, p->mden));
  if (p->tabA && prec == kPrecF64)
    HELM_CK(launch_tri2d_tab(2, nullptr, fc, p->tabA, p->rec, nullptr, p->partial, a, skip, st, p->prof.on ? &p->prof : nullptr));
  else if (p->tabA)
    HELM_CK(launch_tri2d_t32(2, nullptr, fc, p->tabA, p->rec, nullptr, p->partial, a, skip, st, p->prof.on ? &p->prof : nullptr,
                             p->constA, p->dev_err));
  else
    HELM_CK(launch_tri2d(prec, 2, nullptr, fc, p->ustartA, p->rec, nullptr, p->partial, a, skip, st, p->prof.on ? &p->prof : nullptr, p->constA));
  HELM_PK("reduce_faces", launch_reduce_faces(prec, p->partial, fw, nx, nparts, one, one, skip, st));
  if (dbg_w) HELM_CK(cudaMemcpyAsync(dbg_w, fw, 2 * nx * cb, cudaMemcpyDeviceToDevice, st));
  // a4: Step 3
  HELM_PK("apply_cbb", launch_apply_cbb(prec, fv, fw, fc, nx, p->h[0], p->h[1], p->wc[0], p->wc[1], p->omega * p->omega, ax.g,
                                        ax.ginv, skip, st, p->mden));
  if (p->tabB && prec == kPrecF64)
    HELM_CK(launch_tri2d_tab(3, p->fhat, fc, p->tabB, p->rec, p->dbuf, nullptr, a, skip, st, p->prof.on ? &p->prof : nullptr));
  else if (p->tabB)
    HELM_CK(launch_tri2d_t32(3, p->fhat, fc, p->tabB, p->rec, p->dbuf, nullptr, a, skip, st, p->prof.on ? &p->prof : nullptr,
                             p->constB, p->dev_err));
  else
    HELM_CK(launch_tri2d(prec, 3, p->fhat, fc, p->ustartB, p->rec, p->dbuf, nullptr, a, skip, st, p->prof.on ? &p->prof : nullptr, p->constB));
  // a5: inverse DFT along x1 (eq. step3IFFTz3coeff)
  HELM_PK("dft_inv", launch_dft_rows(prec, p->dbuf, prec == kPrecF64, out, out_mode, nx, ax.dft, tw, +1, 1.0 / (double)n1,
                                     accum_scale, nullptr, sco, skip, st));
  return HELM_OK;
}

int solve_core(helm_plan* p, const void* in, int in_is_double, void* out, int out_mode, double accum_scale,
               const int* skip, void* dbg_fhat, void* dbg_v, void* dbg_w) {
  if (p->dim == 2) return solve2d_core(p, in, in_is_double, out, out_mode, accum_scale, skip, dbg_fhat, dbg_v, dbg_w);
  cudaError_t e = solve3d_core(p->p3, p->prec, in, in_is_double, out, out_mode, accum_scale, skip, dbg_fhat,
                               dbg_v, dbg_w, p->stream, p->prof.on ? &p->prof : nullptr);
  return e == cudaSuccess ? HELM_OK : cuda_fail(p, e, "solve3d");
}

// --- iterative refinement (HELM_C64_REFINED) -------------------------------
// u0 = S(f); then r = f - A u, u += S(r) until ||r||/||f|| <= tol or max_iter
// corrections.  S is the complex64 solve.  HELM_RESID_FP64 keeps u in the
// caller's complex128 buffer and forms r in FP64; HELM_RESID_FF splits f once
// into a float-float vector, accumulates u as float-float in the inverse
// transform's epilogue, forms r in float-float and writes u at the end.

bool refine_ff(const helm_plan* p) { return p->resid_kind == HELM_RESID_FF; }

// u0 = S(f)
int refine_first(helm_plan* p, const void* f, void* u, void* dbg_fhat, void* dbg_v, void* dbg_w) {
  // the split left the hi parts of f in the residual buffer (complex64): the
  // first transform reads 8 B per unknown
  if (refine_ff(p)) return solve_core(p, p->rbuf, kInC64, p->ufb, kOutFF, 0.0, nullptr, dbg_fhat, dbg_v, dbg_w);
  return solve_core(p, f, kInC128, u, kOutC128, 0.0, nullptr, dbg_fhat, dbg_v, dbg_w);
}

// residual + convergence test (cond: graph while-node handle, 0 outside a graph)
int refine_check(helm_plan* p, const void* f, const void* u, unsigned long long cond) {
  const int* skip = &p->state->done;
  int64_t nblocks = 0;
  if (refine_ff(p))
    HELM_PK("residual_ff", launch_residual_ff(p->dim, p->n, p->h, p->omega, p->wc, p->ffb, p->ufb, p->rbuf, p->sums,
                                              &nblocks, skip, p->stream, p->mden));
  else
    HELM_PK("residual_fp64", launch_residual(p->dim, p->n, p->h, p->omega, p->wc, (const double2*)f, (const double2*)u,
                                             p->rbuf, p->sums, &nblocks, skip, p->stream, p->dev_err, p->mden));
  HELM_PK("residual_finalize", launch_residual_finalize(p->sums, nblocks, p->state, cond, p->stream));
  return HELM_OK;
}

// u += S(r), skipped on the device once the state is done
int refine_correct(helm_plan* p, void* u) {
  const int* skip = &p->state->done;
  if (refine_ff(p)) return solve_core(p, p->rbuf, kInC64, p->ufb, kOutAccumFF, 1.0, skip, nullptr, nullptr, nullptr);
  return solve_core(p, p->rbuf, kInC64, u, kOutAccumC128, 1.0, skip, nullptr, nullptr, nullptr);
}

void drop_refine_graph(helm_plan* p) {
  if (p->rg_exec) cudaGraphExecDestroy(p->rg_exec);
  if (p->rg_graph) cudaGraphDestroy(p->rg_graph);
  p->rg_exec = nullptr;
  p->rg_graph = nullptr;
  p->rg_f = nullptr;
  p->rg_u = nullptr;
}

// Capture u0 = S(f) and the refinement loop as one CUDA graph: the loop is a
// conditional while node whose body (residual, test, correction) runs again
// while the test kernel leaves the condition at 1.  The test sets it to 0 once
// the state is done, which happens after at most max_iter + 1 residuals, so
// the loop always ends.  Kernel arguments are baked in: the graph is rebuilt
// when f or u (FP64 residual) or the auxiliary change.
// With a stream capture in progress on `cap` and p->stream == cap: append the
// refinement loop after the captured work, as a conditional while node whose
// body (residual, test, correction) is captured on `body`.  The test kernel
// sets the node's condition; it ends the loop after at most max_iter + 1
// residuals, so the loop always ends.
int append_refine_loop(helm_plan* p, const void* f, void* u, cudaStream_t cap, cudaStream_t body) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cap, &status, nullptr, &g, &deps, nullptr, &ndeps);
  if (e != cudaSuccess || status != cudaStreamCaptureStatusActive) return cuda_fail(p, e, "capture info");
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    return cuda_fail(p, e, "cudaGraphConditionalHandleCreate");
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t cn;
  if ((e = cudaGraphAddNode(&cn, g, deps, nullptr, ndeps, &np)) != cudaSuccess)
    return cuda_fail(p, e, "cudaGraphAddNode(while)");
  if ((e = cudaStreamUpdateCaptureDependencies(cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
    return cuda_fail(p, e, "cudaStreamUpdateCaptureDependencies");
  if ((e = cudaStreamBeginCaptureToGraph(body, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_fail(p, e, "cudaStreamBeginCaptureToGraph");
  p->stream = body;
  int rc = refine_check(p, f, u, (unsigned long long)h);
  if (!rc) rc = refine_correct(p, u);
  cudaGraph_t bg = nullptr;
  e = cudaStreamEndCapture(body, &bg);
  p->stream = cap;
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(p, e, "end body capture");
  return HELM_OK;
}

// Capture u0 = S(f) and the refinement loop of one plan as a CUDA graph.
// Kernel arguments are baked in: the graph is rebuilt when f or u (FP64
// residual), the residual kind or the auxiliary change.
int build_refine_graph(helm_plan* p, const void* f, void* u) {
  drop_refine_graph(p);
  for (int k = 0; k < 2; ++k)
    if (!p->cap[k]) HELM_CK(cudaStreamCreateWithFlags(&p->cap[k], cudaStreamNonBlocking));
  cudaStream_t saved = p->stream;
  p->stream = p->cap[0];
  HELM_CK(cudaStreamBeginCapture(p->cap[0], cudaStreamCaptureModeThreadLocal));
  int rc = refine_first(p, f, u, nullptr, nullptr, nullptr);
  if (!rc) rc = append_refine_loop(p, f, u, p->cap[0], p->cap[1]);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(p->cap[0], &g);
  p->stream = saved;
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc ? rc : cuda_fail(p, e, "end capture");
  }
  p->rg_graph = g;
  cudaError_t ei;
  if ((ei = cudaGraphInstantiate(&p->rg_exec, g, 0)) != cudaSuccess) {
    drop_refine_graph(p);
    return cuda_fail(p, ei, "cudaGraphInstantiate");
  }
  p->rg_f = f;
  p->rg_u = u;
  return HELM_OK;
}

int run_refined(helm_plan* p, const void* f, void* u, void* dbg_fhat, void* dbg_v, void* dbg_w) {
  const int64_t N = p->n[0] * p->n[1] * p->n[2];
  int rc;
  RefineState init{};
  init.tol = p->tol;
  init.max_iter = p->max_iter;
  HELM_CK(cudaMemcpyAsync(p->state, &init, sizeof(init), cudaMemcpyHostToDevice, p->stream));
  if (refine_ff(p)) {
    if (!p->ffb) {  // allocated by helm_set_residual; the solve never allocates
      p->err = "float-float vectors missing";
      return HELM_EINVAL;
    }
    HELM_PK("split_ff", launch_split_ff((const double2*)f, p->ffb, p->rbuf, N, p->stream));
  }
  const bool graph = p->use_graphs && !p->prof.on && !dbg_fhat && !dbg_v && !dbg_w;
  if (graph) {
    // the float-float graph touches plan buffers only; the FP64 one reads f, u
    const void* kf = refine_ff(p) ? nullptr : f;
    void* ku = refine_ff(p) ? nullptr : u;
    if (!p->rg_exec || p->rg_f != kf || p->rg_u != ku) {
      if ((rc = build_refine_graph(p, f, u))) return rc;
      p->rg_f = kf;
      p->rg_u = ku;
    }
    HELM_CK(cudaGraphLaunch(p->rg_exec, p->stream));
  } else {
    if ((rc = refine_first(p, f, u, dbg_fhat, dbg_v, dbg_w))) return rc;
    for (int it = 0; it <= p->max_iter; ++it) {
      if ((rc = refine_check(p, f, u, 0))) return rc;
      if (it == p->max_iter) break;
      if ((rc = refine_correct(p, u))) return rc;
    }
  }
  if (refine_ff(p)) HELM_PK("join_ff", launch_join_ff(p->ufb, (double2*)u, N, p->stream));
  return HELM_OK;
}

int run_solve(helm_plan* p, const void* f, void* u, void* dbg_fhat, void* dbg_v, void* dbg_w) {
  if (p->dtype == HELM_C128) return solve_core(p, f, kInC128, u, kOutC128, 0.0, nullptr, dbg_fhat, dbg_v, dbg_w);
  if (p->dtype == HELM_C64_RAW) return solve_core(p, f, kInC64, u, kOutC64, 0.0, nullptr, dbg_fhat, dbg_v, dbg_w);
  return run_refined(p, f, u, dbg_fhat, dbg_v, dbg_w);
}

int alloc_buffers_2d(helm_plan* p) {
  const int64_t nx = p->n[0], n1 = p->n[1], N = nx * n1;
  const size_t cb = cbytes(p->prec);
  int rc;
  p->nwarps = (n1 + 31) / 32;
  p->face_len = nx;
  const Solve2DArgs a = args2d(p);
  const size_t nrec = (size_t)a.nchunks * n1;
  if ((rc = dev_alloc(p, &p->fhat, N * cb)) || (rc = dev_alloc(p, &p->dbuf, N * cb)) ||
      (rc = dev_alloc(p, &p->partial, 2 * p->nwarps * nx * cb)) || (rc = dev_alloc(p, &p->faces, 8 * nx * cb)) ||
      (rc = dev_alloc(p, &p->ustartB, nrec * cb)) || (rc = dev_alloc(p, &p->ustartA, nrec * cb)) ||
      (rc = dev_alloc(p, &p->rec, nrec * chunk_record_bytes(p->prec))))
    return rc;
  // per-line constants and pivots entering each chunk (rhs independent)
  if ((rc = dev_alloc(p, &p->constB, line_consts_bytes(p->prec, n1))) ||
      (rc = dev_alloc(p, &p->constA, line_consts_bytes(p->prec, n1))))
    return rc;
  HELM_CK(launch_line_consts(p->prec, p->constB, a, 1, nullptr));
  HELM_CK(launch_line_consts(p->prec, p->constA, a, 2, nullptr));
  HELM_CK(launch_pivots(p->prec, p->ustartB, a, 1, nullptr));
  HELM_CK(launch_pivots(p->prec, p->ustartA, a, 2, nullptr));
  // The rhs-independent parts of every line's LU, once per plan: FP64 keeps
  // multipliers, reciprocal pivots and chunk weights (3 complex128 values per
  // unknown and line type), complex64 the rounded reciprocal pivots alone (1
  // complex64 value).  If the device cannot hold them the solve recomputes
  // them on the fly instead.
  {
    const bool f64 = p->prec == kPrecF64;
    const size_t tb = f64 ? line_tables_bytes(nx, n1, a.nchunks) : line_tables32_bytes(nx, n1, a.nchunks);
    if (dev_alloc(p, &p->tabB, tb) == HELM_OK && dev_alloc(p, &p->tabA, tb) == HELM_OK) {
      HELM_CK(f64 ? launch_line_tables(p->tabB, a, 1, nullptr) : launch_line_tables32(p->tabB, a, 1, nullptr));
      HELM_CK(f64 ? launch_line_tables(p->tabA, a, 2, nullptr) : launch_line_tables32(p->tabA, a, 2, nullptr));
    } else {
      dfree(p->tabB);
      dfree(p->tabA);
      p->tabB = p->tabA = nullptr;
      p->err.clear();
    }
  }
  HELM_CK(cudaStreamSynchronize(nullptr));  // plan-time kernels run on the legacy stream
  return HELM_OK;
}

int alloc_refine(helm_plan* p) {
  int64_t N = p->n[0] * p->n[1] * p->n[2];
  int rc;
  if ((rc = dev_alloc(p, (void**)&p->dev_err, sizeof(int)))) return rc;
  HELM_CK(cudaMemset(p->dev_err, 0, sizeof(int)));
  if (p->dtype != HELM_C64_REFINED) {
    rc = dev_alloc(p, (void**)&p->state, sizeof(RefineState));
    return rc;
  }
  if ((rc = dev_alloc(p, (void**)&p->rbuf, N * sizeof(float2))) ||
      (rc = dev_alloc(p, (void**)&p->sums, residual_blocks(p->dim, p->n) * 2 * sizeof(double))) ||
      (rc = dev_alloc(p, (void**)&p->state, sizeof(RefineState))))
    return rc;
  return HELM_OK;
}

// Bytes of one f or u vector of plan p (complex64 for HELM_C64_RAW, else complex128).
size_t plan_vec_bytes(const helm_plan* p) {
  const int64_t N = p->n[0] * p->n[1] * p->n[2];
  return (size_t)N * (p->dtype == HELM_C64_RAW ? sizeof(float2) : sizeof(double2));
}

// Do [a, a + bytes) and [b, b + bytes) share a byte?
bool overlaps(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bytes && y < x + bytes;
}

// f and u of a solve: overlapping ranges, or an address that is not a
// multiple of the element size (16 B complex128, 8 B complex64), which the
// kernels' vector loads and stores need.
bool bad_pair(const void* f, const void* u, size_t bytes, size_t elem) {
  const uintptr_t m = (uintptr_t)(elem - 1);
  return overlaps(f, u, bytes) || ((uintptr_t)f & m) || ((uintptr_t)u & m);
}

size_t plan_elem_bytes(const helm_plan* p) { return p->dtype == HELM_C64_RAW ? sizeof(float2) : sizeof(double2); }

// The plan's stream and its workspace streams have finished their work (the
// tables they read may be rebuilt or freed after this).
cudaError_t sync_plan_streams(helm_plan* p) {
  cudaError_t e = cudaStreamSynchronize(p->stream);
  for (cudaStream_t st : p->ws_stream)
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

void destroy_workspace(helm_plan* w) {
  for (void* q : w->owned) dfree(q);
  drop_refine_graph(w);
  for (int k = 0; k < 2; ++k)
    if (w->cap[k]) cudaStreamDestroy(w->cap[k]);
  w->prof.destroy();
  delete w;
}

void destroy_plan(helm_plan* p) {
  if (!p) return;
  if (p->parent) {
    destroy_workspace(p);
    return;
  }
  for (helm_plan* w : p->ws) destroy_workspace(w);
  for (cudaStream_t st : p->ws_stream) cudaStreamDestroy(st);
  for (cudaEvent_t ev : p->ws_done) cudaEventDestroy(ev);
  if (p->fork) cudaEventDestroy(p->fork);
  free_axis(p->axo);
  free_axis(p->axi);
  dfree(p->fhat);
  dfree(p->cbuf);
  dfree(p->dbuf);
  dfree(p->partial);
  dfree(p->faces);
  dfree(p->ustartB);
  dfree(p->ustartA);
  dfree(p->rec);
  dfree(p->tabB);
  dfree(p->tabA);
  dfree(p->constB);
  dfree(p->constA);
  dfree(p->rbuf);
  dfree(p->sums);
  dfree(p->ffb);
  dfree(p->ufb);
  dfree(p->dev_err);
  dfree(p->state);
  dfree(p->host_f);
  dfree(p->host_u);
  if (p->out_stream) cudaStreamDestroy(p->out_stream);
  if (p->out_ready) cudaEventDestroy(p->out_ready);
  if (p->out_done) cudaEventDestroy(p->out_done);
  free_plan3d(p->p3);
  drop_refine_graph(p);
  for (int k = 0; k < 2; ++k)
    if (p->cap[k]) cudaStreamDestroy(p->cap[k]);
  p->prof.destroy();
  delete p;
}

// A workspace for helm_solve_many: a plan that borrows p's operator data
// (axis eigen-data, pivot and line tables, 3D settling and routing tables)
// and owns fresh scratch of the same sizes.  Its solves run the same kernels
// on the same operator data as p's, so each result is p's own result.
helm_plan* make_workspace(helm_plan* p) {
  helm_plan* w = new (std::nothrow) helm_plan();
  if (!w) return nullptr;
  w->parent = p;
  w->dim = p->dim;
  for (int k = 0; k < 3; ++k) {
    w->n[k] = p->n[k];
    w->h[k] = p->h[k];
    w->bc[k] = p->bc[k];
    w->wc[k] = p->wc[k];
  }
  w->omega = p->omega;
  w->dtype = p->dtype;
  w->prec = p->prec;
  w->axo = p->axo;
  w->axi = p->axi;
  w->tol = p->tol;
  w->max_iter = p->max_iter;
  w->resid_kind = p->resid_kind;
  w->use_graphs = p->use_graphs;
  w->tri_regs = p->tri_regs;
  w->element = p->element;
  w->mden = p->mden;
  w->version = p->version;
  const int64_t N = p->n[0] * p->n[1] * p->n[2];
  const size_t cb = cbytes(p->prec);
  bool ok = true;
  auto own = [&](void** q, size_t bytes) {
    if (!ok) return;
    if (dmalloc(q, bytes ? bytes : 16) != cudaSuccess) {
      ok = false;
      *q = nullptr;
      return;
    }
    w->owned.push_back(*q);
    w->bytes += bytes;
  };
  if (p->dim == 2) {
    w->ustartB = p->ustartB;
    w->ustartA = p->ustartA;
    w->tabB = p->tabB;
    w->tabA = p->tabA;
    w->constB = p->constB;
    w->constA = p->constA;
    w->nwarps = p->nwarps;
    w->face_len = p->face_len;
    const Solve2DArgs a = args2d(p);
    const size_t nrec = (size_t)a.nchunks * p->n[1];
    own(&w->fhat, N * cb);
    own(&w->dbuf, N * cb);
    own(&w->partial, 2 * p->nwarps * p->n[0] * cb);
    own(&w->faces, 8 * p->n[0] * cb);
    own(&w->rec, nrec * chunk_record_bytes(p->prec));
  } else {
    w->p3 = p->p3;  // tables and routing borrowed; scratch replaced below
    const int64_t F = p->n[0] * p->n[2];
    own(&w->p3.fhat, N * cb);
    own(&w->p3.dbuf, N * cb);
    own(&w->p3.faces, 10 * F * cb);
    w->p3.cbuf = nullptr;
    if (!p->p3.tab[0]) own(&w->p3.cbuf, N * cb);  // the untabled sweeps keep their multipliers there
    if (p->p3.inner_nmb) {
      own(&w->p3.ipart, (size_t)p->n[1] * p->p3.inner_nparts * 2 * p->n[0] * cb);
      own(&w->p3.ivw, (size_t)p->n[1] * 4 * p->n[0] * cb);
      own(&w->p3.icin, (size_t)p->n[1] * 2 * p->n[0] * cb);
    }
    int maxr = 0;
    for (int t = 0; t < 4; ++t) maxr = std::max(maxr, p->p3.nroute[t]);
    if (maxr) {
      own(&w->p3.rpart, (size_t)maxr * 2 * p->n[0] * sizeof(float2));
      own(&w->p3.rtmp, (size_t)maxr * p->n[0] * sizeof(double2));
    }
    w->p3.partial = w->p3.ybuf = nullptr;
  }
  own((void**)&w->dev_err, sizeof(int));
  own((void**)&w->state, sizeof(RefineState));
  if (ok && cudaMemset(w->dev_err, 0, sizeof(int)) != cudaSuccess) ok = false;
  if (p->dtype == HELM_C64_REFINED) {
    own((void**)&w->rbuf, N * sizeof(float2));
    own((void**)&w->sums, residual_blocks(p->dim, p->n) * 2 * sizeof(double));
    if (p->ffb) {
      own((void**)&w->ffb, N * sizeof(float4));
      own((void**)&w->ufb, N * sizeof(float4));
    }
  }
  if (!ok) {
    destroy_workspace(w);
    return nullptr;
  }
  return w;
}

// ---------------------------------------------------------------------------
// Allocation-free small 2D solve (helm_solve_2d_static).
//
// For callers that cannot allocate device memory at solve time -- code that
// runs where cudaMalloc is not allowed or not wanted (inside a host callback,
// under an allocator lock held by a larger framework, in a process whose
// device memory is reserved up front) -- the whole complex128 2D solve runs
// out of one fixed device array that the library reserves when it is loaded.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int64_t kStaticMaxN1 = 1024;                     // longest x1 axis
constexpr int kStaticMaxDevices = 64;

// Device scratch of the allocation-free solve: every GPU that loads the library
// holds these 16 MiB until the process exits.  Host code must not use the
// symbol as a pointer; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_helm_static_scratch[kStaticScratchBytes];

// Device address of g_helm_static_scratch per device, looked up once.
static void* g_static_addr[kStaticMaxDevices];

// Host workspace for the per-call eigen-data (static: no heap use).
static double g_st_work[2 * kStaticMaxN1 + 9 * ((kStaticMaxN1 + 1) / 2) + 64];
static double g_st_lamA[2 * kStaticMaxN1], g_st_sigA[2 * kStaticMaxN1], g_st_parA[kStaticMaxN1];
static double g_st_lamB[2 * kStaticMaxN1], g_st_invmu[2 * kStaticMaxN1], g_st_tw[2 * kStaticMaxN1];
static double g_st_sci[2 * kStaticMaxN1], g_st_sco[2 * kStaticMaxN1];
static double g_st_twre[kStaticMaxN1], g_st_twim[kStaticMaxN1];
static double g_st_r4re[4 * kStaticMaxN1], g_st_r4im[4 * kStaticMaxN1];
static int8_t g_st_par8[kStaticMaxN1];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Auxiliary tables of build_axis_aux computed into the static host arrays.
void static_aux_tables(AxisData& a, double rho, int q) {
  const int64_t n = a.n;
  const double h = a.h;
  a.rho = rho;
  a.q = ((q % 4) + 4) % 4;
  const double pi = 3.14159265358979323846;
  unit_roots(4 * n, g_st_r4re, g_st_r4im);
  const double ar = 0.5 * rho / (double)n;
  for (int64_t l = 0; l < n; ++l) {
    const double b = (0.5 * pi * a.q + 2.0 * pi * (double)l) / (2.0 * (double)n);
    const std::complex<double> sh(std::sinh(ar) * std::cos(b), std::cosh(ar) * std::sin(b));
    const std::complex<double> s2 = sh * sh;
    const std::complex<double> mu = h * (1.0 + (2.0 / 3.0) * s2);
    const std::complex<double> lb = (-4.0 * s2 / h) / mu, im = 1.0 / mu;
    g_st_lamB[2 * l] = lb.real();
    g_st_lamB[2 * l + 1] = lb.imag();
    g_st_invmu[2 * l] = im.real();
    g_st_invmu[2 * l + 1] = im.imag();
  }
  auto et = [&](int64_t j, double sign) -> std::complex<double> {
    const int64_t k = (a.q * j) % (4 * n);
    return std::exp(sign * rho * (double)j / (double)n) * std::complex<double>(g_st_r4re[k], -sign * g_st_r4im[k]);
  };
  for (int64_t j = 0; j < n; ++j) {
    const std::complex<double> ei = et(j, -1.0), eo = et(j, +1.0);
    g_st_sci[2 * j] = ei.real();
    g_st_sci[2 * j + 1] = ei.imag();
    g_st_sco[2 * j] = eo.real();
    g_st_sco[2 * j + 1] = eo.imag();
  }
  const std::complex<double> en = et(n - 1, +1.0), eninv = et(n - 1, -1.0);
  a.en[0] = en.real();
  a.en[1] = en.imag();
  a.eninv[0] = eninv.real();
  a.eninv[1] = eninv.imag();
  const double gr[4] = {1, 0, -1, 0}, gi[4] = {0, 1, 0, -1};
  a.g[0] = std::exp(rho) * gr[a.q];
  a.g[1] = std::exp(rho) * gi[a.q];
  a.ginv[0] = std::exp(-rho) * gr[a.q];
  a.ginv[1] = -std::exp(-rho) * gi[a.q];
}

// Rebuild every table that depends on the auxiliary of the periodic axes.
int apply_aux(helm_plan* p, double rho, int phase_quarters) {
  drop_refine_graph(p);  // its kernels hold the old eigen-data
  ++p->version;
  int rc = build_axis_aux(p, p->axo, rho, phase_quarters);
  if (!rc && p->dim == 3) rc = build_axis_aux(p, p->axi, rho, phase_quarters);
  // the tensor-core transform tables hold the scalings of the auxiliary
  if (!rc && p->dft_gemm) rc = build_dft_gemm(p, p->dim == 3 ? p->axi : p->axo);
  if (rc) return rc;
  if (p->dim == 2) {
    const Solve2DArgs a = args2d(p);
    HELM_CK(launch_pivots(p->prec, p->ustartB, a, 1, nullptr));
    if (p->constB) HELM_CK(launch_line_consts(p->prec, p->constB, a, 1, nullptr));
    if (p->tabB)
      HELM_CK(p->prec == kPrecF64 ? launch_line_tables(p->tabB, a, 1, nullptr)
                                  : launch_line_tables32(p->tabB, a, 1, nullptr));
    HELM_CK(cudaStreamSynchronize(nullptr));  // plan-time kernels run on the legacy stream
  } else {
    HELM_CK(plan3d_tables(p->p3));
  }
  return HELM_OK;
}

// The auxiliary B (damping rho and phase q of the gamma-circulant, reading
// R13) is chosen per plan.  Steps 1-3 are exact for every B, but the rounding
// errors of a solve grow with the conditioning of B's own problems, which
// depends on where the grid's modes fall relative to w^2: no fixed (rho, q)
// suits every grid.  Each candidate gets one solve, in the plan's precision,
// of a fixed pseudo-random load f (refined plans: and one correction sweep);
// the candidate with the smallest relative residual ||f - A u|| / ||f||
// (FP64, eq. A2D / A3D) is kept.  For refined plans that residual is the
// product of the first two contraction factors of the refinement.
struct AuxCand {
  double rho;
  int q;
};
constexpr AuxCand kAuxCandidates[] = {{1.0, 1}, {0.5, 0}, {1.0, 0}, {0.5, 1}, {0.0, 0}};

int tune_auxiliary(helm_plan* p) {
  const int64_t N = p->n[0] * p->n[1] * p->n[2];
  double2 *tf = nullptr, *tu = nullptr;
  float2* tr = p->rbuf;
  double* ts = p->sums;
  bool own_r = false;
  auto cleanup = [&]() {
    dfree(tf);
    dfree(tu);
    if (own_r) {
      dfree(tr);
      dfree(ts);
    }
    cudaGetLastError();
  };
  const int64_t nb_max = residual_blocks(p->dim, p->n);
  if (dmalloc((void**)&tf, N * sizeof(double2)) != cudaSuccess || dmalloc((void**)&tu, N * sizeof(double2)) != cudaSuccess) {
    cleanup();
    return HELM_OK;  // no room for the trials: keep the default auxiliary
  }
  if (!tr) {
    own_r = true;
    if (dmalloc((void**)&tr, N * sizeof(float2)) != cudaSuccess ||
        dmalloc((void**)&ts, nb_max * 2 * sizeof(double)) != cudaSuccess) {
      cleanup();
      return HELM_OK;
    }
  }
  cudaStream_t saved = p->stream;
  p->stream = nullptr;
  std::vector<double> hs(2 * nb_max);
  double best = HUGE_VAL;
  AuxCand pick = kAuxCandidates[0];
  int rc = HELM_OK;
  if (launch_trial_rhs(tf, N, 0x5eedull, nullptr) != cudaSuccess) rc = cuda_fail(p, cudaGetLastError(), "trial rhs");
  for (const AuxCand& c : kAuxCandidates) {
    if (rc) break;
    if ((rc = apply_aux(p, c.rho, c.q))) break;
    if ((rc = solve_core(p, tf, kInC128, tu, kOutC128, 0.0, nullptr, nullptr, nullptr, nullptr))) break;
    int64_t nb = 0;
    cudaError_t e = launch_residual(p->dim, p->n, p->h, p->omega, p->wc, tf, tu, tr, ts, &nb, nullptr, nullptr, p->dev_err, p->mden);
    if (e == cudaSuccess && p->dtype == HELM_C64_REFINED) {
      // refined plans: one correction sweep as well, so that the residual
      // measures the contraction of the sweeps, not only the first solve
      if ((rc = solve_core(p, tr, kInC64, tu, kOutAccumC128, 1.0, nullptr, nullptr, nullptr, nullptr))) break;
      e = launch_residual(p->dim, p->n, p->h, p->omega, p->wc, tf, tu, tr, ts, &nb, nullptr, nullptr, p->dev_err, p->mden);
    }
    if (e == cudaSuccess) e = cudaMemcpy(hs.data(), ts, nb * 2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      rc = cuda_fail(p, e, "auxiliary trial");
      break;
    }
    double r2 = 0, f2 = 0;
    for (int64_t i = 0; i < nb; ++i) {
      r2 += hs[2 * i];
      f2 += hs[2 * i + 1];
    }
    const double rel = f2 > 0 ? std::sqrt(r2 / f2) : HUGE_VAL;
    if (rel < best) {
      best = rel;
      pick = c;
    }
  }
  if (!rc) rc = apply_aux(p, pick.rho, pick.q);
  p->stream = saved;
  p->aux_trial_resid = best;
  cleanup();
  return rc;
}

// Append plan p's whole solve (f -> u) to the capture in progress on `cap`:
// the plain solve, or for refined plans the state reset, the float-float
// split, u0 = S(f), the refinement loop (while node, body on `body`) and the
// final join.
int append_solve(helm_plan* p, const void* f, void* u, cudaStream_t cap, cudaStream_t body) {
  const int64_t N = p->n[0] * p->n[1] * p->n[2];
  cudaStream_t saved = p->stream;
  p->stream = cap;
  int rc = HELM_OK;
  if (p->dtype == HELM_C128) {
    rc = solve_core(p, f, kInC128, u, kOutC128, 0.0, nullptr, nullptr, nullptr, nullptr);
  } else if (p->dtype == HELM_C64_RAW) {
    rc = solve_core(p, f, kInC64, u, kOutC64, 0.0, nullptr, nullptr, nullptr, nullptr);
  } else {
    cudaError_t e = launch_refine_init(p->state, p->tol, p->max_iter, cap);
    if (e != cudaSuccess) rc = cuda_fail(p, e, "refine init");
    if (!rc && refine_ff(p) && (e = launch_split_ff((const double2*)f, p->ffb, p->rbuf, N, cap)) != cudaSuccess)
      rc = cuda_fail(p, e, "split");
    if (!rc) rc = refine_first(p, f, u, nullptr, nullptr, nullptr);
    if (!rc) rc = append_refine_loop(p, f, u, cap, body);
    if (!rc && refine_ff(p) && (e = launch_join_ff(p->ufb, (double2*)u, N, cap)) != cudaSuccess)
      rc = cuda_fail(p, e, "join");
  }
  p->stream = saved;
  return rc;
}

void drop_batch_graph(helm_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->kf.clear();
  b->ku.clear();
  b->kv.clear();
}

// One graph for the whole batch: every plan's solve hangs from an empty root
// node, so the plans are independent branches that the GPU runs side by side.
int build_batch_graph(helm_batch* b, const void* const* f, void* const* u) {
  drop_batch_graph(b);
  for (int k = 0; k < 2; ++k)
    if (!b->cap[k] && cudaStreamCreateWithFlags(&b->cap[k], cudaStreamNonBlocking) != cudaSuccess) {
      b->err = "cudaStreamCreate";
      return HELM_ECUDA;
    }
  cudaStream_t cs = b->cap[0];
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    b->err = "cudaStreamBeginCapture";
    return HELM_ECUDA;
  }
  int rc = HELM_OK;
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  cudaGraphNode_t root = nullptr;
  if (cudaStreamGetCaptureInfo(cs, &status, nullptr, &g) != cudaSuccess || cudaGraphAddEmptyNode(&root, g, nullptr, 0) != cudaSuccess) {
    b->err = "batch graph root";
    rc = HELM_ECUDA;
  }
  for (size_t i = 0; i < b->plans.size() && !rc; ++i) {
    if (cudaStreamUpdateCaptureDependencies(cs, &root, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess) {
      b->err = "cudaStreamUpdateCaptureDependencies";
      rc = HELM_ECUDA;
      break;
    }
    rc = append_solve(b->plans[i], f[i], u[i], cs, b->cap[1]);
    if (rc) b->err = std::string("plan ") + std::to_string(i) + ": " + b->plans[i]->err;
  }
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &out);
  if (rc || e != cudaSuccess) {
    if (out) cudaGraphDestroy(out);
    cudaGetLastError();
    if (!rc) b->err = "cudaStreamEndCapture";
    return rc ? rc : HELM_ECUDA;
  }
  b->graph = out;
  if (cudaGraphInstantiate(&b->exec, out, 0) != cudaSuccess) {
    drop_batch_graph(b);
    b->err = "cudaGraphInstantiate";
    return HELM_ECUDA;
  }
  b->kf.assign(f, f + b->plans.size());
  b->ku.assign(u, u + b->plans.size());
  for (helm_plan* p : b->plans) b->kv.push_back(p->version);
  return HELM_OK;
}

// Failure-detection check: an mbarrier that expects 16 bytes of copies that
// are never issued, waited on by the same bounded wait the bulk-copy kernels
// use, with a short limit.  The wait gives up, sets the plan's error word and
// the kernel returns; nothing is in flight.
__global__ void k_debug_wait_timeout(int* err, uint32_t tries) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  mbar_arrive_expect_tx(&bar, 16);
  mbar_wait_bounded(&bar, 0, err, tries);
}

// Boundary kinds per axis: each HELM_BC_ABC or HELM_BC_NEUMANN, at least one
// absorbing axis (it keeps A non-singular for every real w).
int validate_bc(int dim, const int32_t* bc) {
  if (!bc) return HELM_OK;
  int nabc = 0;
  for (int k = 0; k < dim; ++k) {
    if (bc[k] != HELM_BC_ABC && bc[k] != HELM_BC_NEUMANN) return HELM_EINVAL;
    nabc += bc[k] == HELM_BC_ABC;
  }
  return nabc ? HELM_OK : HELM_EINVAL;
}

void set_element(helm_plan* p, int element) {
  p->element = element;
  p->mden = element == HELM_ELEMENT_Q1_MODIFIED ? 12.0 : 6.0;
}

void set_bc(helm_plan* p, const int32_t* bc) {
  for (int k = 0; k < p->dim; ++k) {
    p->bc[k] = bc ? bc[k] : HELM_BC_ABC;
    p->wc[k] = p->bc[k] == HELM_BC_ABC ? p->omega : 0.0;
  }
}

int plan_2d(helm_plan_t* out, int64_t nx, int64_t ny, double hx, double hy, double omega, int dtype,
            const int32_t* bc, int element) {
  if (!out) return HELM_EINVAL;
  *out = nullptr;
  if (nx < 3 || ny < 3 || !(hx > 0) || !(hy > 0) || !std::isfinite(hx) || !std::isfinite(hy)) return HELM_EINVAL;
  if (int rc = validate_common(omega, dtype)) return rc;
  if (int rc = validate_bc(2, bc)) return rc;
  if (element != HELM_ELEMENT_Q1 && element != HELM_ELEMENT_Q1_MODIFIED) return HELM_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  helm_plan* p = new (std::nothrow) helm_plan();
  if (!p) return HELM_ENOMEM;
  p->dim = 2;
  p->n[0] = nx;
  p->n[1] = ny;
  p->n[2] = 1;
  p->h[0] = hx;
  p->h[1] = hy;
  p->omega = omega;
  p->dtype = dtype;
  p->prec = dtype == HELM_C128 ? kPrecF64 : kPrecF32;
  set_bc(p, bc);
  set_element(p, element);
  DftPlan dp;
  dft_factor(ny, &dp);
  int dev = 0, smem = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return HELM_ECUDA;
  }
  if (!dft_supported(dp, cbytes(p->prec), smem)) {
    delete p;
    return HELM_EUNSUPPORTED;
  }
  int rc = build_axis(p, p->axo, ny, hy, p->wc[1], kDefaultAuxRho, kDefaultAuxQ);
  if (!rc) rc = alloc_buffers_2d(p);
  if (!rc) rc = alloc_refine(p);
  if (!rc) rc = tune_auxiliary(p);
  if (rc) {
    destroy_plan(p);
    return rc;
  }
  p->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = p;
  return HELM_OK;
}

int plan_3d(helm_plan_t* out, int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz, double omega,
            int dtype, const int32_t* bc, int element) {
  if (!out) return HELM_EINVAL;
  if (element != HELM_ELEMENT_Q1 && element != HELM_ELEMENT_Q1_MODIFIED) return HELM_EINVAL;
  *out = nullptr;
  if (nx < 3 || ny < 3 || nz < 3 || !(hx > 0) || !(hy > 0) || !(hz > 0) || !std::isfinite(hx) ||
      !std::isfinite(hy) || !std::isfinite(hz))
    return HELM_EINVAL;
  if (int rc = validate_common(omega, dtype)) return rc;
  if (int rc = validate_bc(3, bc)) return rc;
  auto t0 = std::chrono::steady_clock::now();
  helm_plan* p = new (std::nothrow) helm_plan();
  if (!p) return HELM_ENOMEM;
  p->dim = 3;
  p->n[0] = nx;
  p->n[1] = ny;
  p->n[2] = nz;
  p->h[0] = hx;
  p->h[1] = hy;
  p->h[2] = hz;
  p->omega = omega;
  p->dtype = dtype;
  p->prec = dtype == HELM_C128 ? kPrecF64 : kPrecF32;
  set_bc(p, bc);
  set_element(p, element);
  int smem = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return HELM_ECUDA;
  }
  if (nz > 1024 || ny > 1024 ||
      (size_t)(6 * nx + 2 * 32 * 32) * cbytes(p->prec) > (size_t)smem) {
    delete p;
    return HELM_EUNSUPPORTED;
  }
  int rc = build_axis(p, p->axo, ny, hy, p->wc[1], kDefaultAuxRho, kDefaultAuxQ3D);
  if (!rc) rc = build_axis(p, p->axi, nz, hz, p->wc[2], kDefaultAuxRho, kDefaultAuxQ3D);
  if (!rc) {
    DftPlan a = p->axo.dft, b = p->axi.dft;
    if (!dft_supported(a, cbytes(p->prec), smem) || !dft_supported(b, cbytes(p->prec), smem)) rc = HELM_EUNSUPPORTED;
  }
  if (!rc) {
    cudaError_t ce = plan3d_init(p->p3, p->prec, p->n, p->h, omega, p->wc, p->mden, p->axo, p->axi, &p->bytes);
    if (ce == cudaErrorMemoryAllocation) rc = HELM_ENOMEM;
    else if (ce != cudaSuccess) rc = cuda_fail(p, ce, "plan3d_init");
  }
  if (!rc) rc = alloc_refine(p);
  if (!rc) rc = tune_auxiliary(p);
  if (rc) {
    destroy_plan(p);
    return rc;
  }
  p->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = p;
  return HELM_OK;
}

}  // namespace

extern "C" {

int helm_debug_wait_timeout(helm_plan_t p, int64_t tries) {
  if (!p || tries < 1 || tries > (int64_t)kMbarWaitLimit) return HELM_EINVAL;
  k_debug_wait_timeout<<<1, 32, 0, p->stream>>>(p->dev_err, (uint32_t)tries);
  HELM_CK(cudaGetLastError());
  return HELM_OK;
}

int helm_plan_2d(helm_plan_t* out, int64_t nx, int64_t ny, double hx, double hy, double omega, int dtype) {
  return plan_2d(out, nx, ny, hx, hy, omega, dtype, nullptr, HELM_ELEMENT_Q1);
}

int helm_plan_2d_bc(helm_plan_t* out, int64_t nx, int64_t ny, double hx, double hy, double omega, int dtype,
                    const int32_t* axis_bc) {
  if (!axis_bc) return HELM_EINVAL;
  return plan_2d(out, nx, ny, hx, hy, omega, dtype, axis_bc, HELM_ELEMENT_Q1);
}

int helm_plan_2d_ex(helm_plan_t* out, int64_t nx, int64_t ny, double hx, double hy, double omega, int dtype,
                    const struct helm_plan_opts* opts) {
  if (!opts) return plan_2d(out, nx, ny, hx, hy, omega, dtype, nullptr, HELM_ELEMENT_Q1);
  return plan_2d(out, nx, ny, hx, hy, omega, dtype, opts->axis_bc, opts->element);
}

int helm_plan_3d(helm_plan_t* out, int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz,
                 double omega, int dtype) {
  return plan_3d(out, nx, ny, nz, hx, hy, hz, omega, dtype, nullptr, HELM_ELEMENT_Q1);
}

int helm_plan_3d_bc(helm_plan_t* out, int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz,
                    double omega, int dtype, const int32_t* axis_bc) {
  if (!axis_bc) return HELM_EINVAL;
  return plan_3d(out, nx, ny, nz, hx, hy, hz, omega, dtype, axis_bc, HELM_ELEMENT_Q1);
}

int helm_plan_3d_ex(helm_plan_t* out, int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz,
                    double omega, int dtype, const struct helm_plan_opts* opts) {
  if (!opts) return plan_3d(out, nx, ny, nz, hx, hy, hz, omega, dtype, nullptr, HELM_ELEMENT_Q1);
  return plan_3d(out, nx, ny, nz, hx, hy, hz, omega, dtype, opts->axis_bc, opts->element);
}

int helm_set_auxiliary(helm_plan_t p, double rho, int phase_quarters) {
  if (!p || !std::isfinite(rho) || rho < 0.0 || rho > 8.0) return HELM_EINVAL;
  HELM_CK(sync_plan_streams(p));
  p->aux_trial_resid = -1.0;  // chosen by the caller, not by the plan's trials
  return apply_aux(p, rho, phase_quarters);
}

int helm_set_precision_routing(helm_plan_t p, double tau) {
  if (!p || !std::isfinite(tau) || tau < 0 || tau > 1) return HELM_EINVAL;
  if (p->dim != 3 || p->prec != kPrecF32) return HELM_EUNSUPPORTED;
  HELM_CK(sync_plan_streams(p));
  drop_refine_graph(p);  // its kernels hold the old routing
  ++p->version;
  HELM_CK(plan3d_set_routing(p->p3, tau));
  return HELM_OK;
}

int helm_set_variant(helm_plan_t p, int knob, int value) {
  if (!p || p->parent) return HELM_EINVAL;
  HELM_CK(sync_plan_streams(p));
  if (knob == HELM_VARIANT_TRI2D) {
    if (p->dim != 2 || p->prec != kPrecF32) return HELM_EUNSUPPORTED;
    if (value != 0 && value != 1) return HELM_EINVAL;
    p->tri_regs = value;
  } else if (knob == HELM_VARIANT_DFT) {
    if (value != 0 && value != 1) return HELM_EINVAL;
    AxisData& ax = p->dim == 3 ? p->axi : p->axo;  // the axis transformed along rows
    if (value && (p->prec != kPrecF32 || !dft_gemm_supported(ax.n))) return HELM_EUNSUPPORTED;
    if (value) {
      if (int rc = build_dft_gemm(p, ax)) return rc;
    } else {
      free_dft_gemm(p, ax);
    }
    p->dft_gemm = value;
  } else if (knob == HELM_VARIANT_INNER_CHUNK || knob == HELM_VARIANT_INNER_TILES) {
    if (p->dim != 3 || !p->p3.inner_nmb) return HELM_EUNSUPPORTED;
    const int ch = knob == HELM_VARIANT_INNER_CHUNK ? value : p->p3.inner_ch;
    const int nmb = knob == HELM_VARIANT_INNER_TILES ? value : p->p3.inner_nmb;
    const cudaError_t e = plan3d_set_inner(p->p3, ch, nmb);
    if (e == cudaErrorInvalidValue) {
      cudaGetLastError();
      return HELM_EINVAL;
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "plan3d_set_inner");
  } else {
    return HELM_EINVAL;
  }
  drop_refine_graph(p);  // its kernels were captured with the old variant
  ++p->version;
  return HELM_OK;
}

int helm_get_variant(helm_plan_t p, int knob, int* value) {
  if (!p || !value) return HELM_EINVAL;
  if (knob == HELM_VARIANT_TRI2D) *value = p->tri_regs;
  else if (knob == HELM_VARIANT_INNER_CHUNK) *value = p->dim == 3 ? p->p3.inner_ch : 0;
  else if (knob == HELM_VARIANT_INNER_TILES) *value = p->dim == 3 ? p->p3.inner_nmb : 0;
  else if (knob == HELM_VARIANT_DFT) *value = p->dft_gemm;
  else return HELM_EINVAL;
  return HELM_OK;
}

int helm_time_solve(helm_plan_t p, int reps, double* ms) {
  if (!p || p->parent || reps < 1 || !ms) return HELM_EINVAL;
  const int64_t N = p->n[0] * p->n[1] * p->n[2];
  double2 *tf = nullptr, *tu = nullptr;
  if (dmalloc((void**)&tf, N * sizeof(double2)) != cudaSuccess ||
      dmalloc((void**)&tu, N * sizeof(double2)) != cudaSuccess) {
    dfree(tf);
    return HELM_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HELM_OK;
  auto once = [&]() { return solve_core(p, tf, kInC128, tu, kOutC128, 0.0, nullptr, nullptr, nullptr, nullptr); };
  if (launch_trial_rhs(tf, N, 0x7eedull, p->stream) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = cuda_fail(p, cudaGetLastError(), "timing set-up");
  }
  if (!rc) rc = once();  // warm-up
  if (!rc && cudaEventRecord(e0, p->stream) != cudaSuccess) rc = HELM_ECUDA;
  for (int r = 0; r < reps && !rc; ++r) rc = once();
  if (!rc && cudaEventRecord(e1, p->stream) != cudaSuccess) rc = HELM_ECUDA;
  float t = 0.f;
  if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
    rc = HELM_ECUDA;
  if (!rc) *ms = (double)t / reps;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(p->stream);
  dfree(tf);
  dfree(tu);
  cudaGetLastError();
  return rc;
}

int helm_set_stream(helm_plan_t p, void* s) {
  if (!p) return HELM_EINVAL;
  p->stream = (cudaStream_t)s;
  return HELM_OK;
}

int helm_set_refinement(helm_plan_t p, double tol, int max_iter) {
  if (!p || !(tol >= 0) || max_iter < 1 || max_iter > 15) return HELM_EINVAL;
  ++p->version;
  p->tol = tol;
  p->max_iter = max_iter;
  return HELM_OK;
}

int helm_set_residual(helm_plan_t p, int kind) {
  if (!p || p->dtype != HELM_C64_REFINED || (kind != HELM_RESID_FP64 && kind != HELM_RESID_FF)) return HELM_EINVAL;
  if (kind == HELM_RESID_FF && !p->ffb) {
    // the float-float f and u live as long as the plan: allocated here, never in a solve
    const int64_t N = p->n[0] * p->n[1] * p->n[2];
    int rc;
    if ((rc = dev_alloc(p, (void**)&p->ffb, N * sizeof(float4))) ||
        (rc = dev_alloc(p, (void**)&p->ufb, N * sizeof(float4)))) {
      dfree(p->ffb);
      p->ffb = nullptr;
      p->ufb = nullptr;
      p->bytes -= std::min(p->bytes, (size_t)N * sizeof(float4));
      return rc;
    }
  }
  ++p->version;
  if (p->resid_kind != kind) drop_refine_graph(p);
  p->resid_kind = kind;
  return HELM_OK;
}

int helm_set_graphs(helm_plan_t p, int enable) {
  if (!p) return HELM_EINVAL;
  p->use_graphs = enable != 0;
  return HELM_OK;
}

int helm_solve(helm_plan_t p, const void* f, void* u) {
  if (!p || !f || !u || bad_pair(f, u, plan_vec_bytes(p), plan_elem_bytes(p))) return HELM_EINVAL;
  p->last_many = 0;
  return run_solve(p, f, u, nullptr, nullptr, nullptr);
}

int helm_set_rhs_concurrency(helm_plan_t p, int k) {
  if (!p || p->parent || k < 1 || k > 16) return HELM_EINVAL;
  p->rhs_concurrency = k;
  return HELM_OK;
}

int helm_solve_many(helm_plan_t p, int64_t nrhs, const void* f, void* u) {
  if (!p || p->parent || nrhs < 1 || !f || !u) return HELM_EINVAL;
  const size_t vb = plan_vec_bytes(p);
  if (bad_pair(f, u, vb * (size_t)nrhs, plan_elem_bytes(p))) return HELM_EINVAL;
  p->last_many = 0;
  if (nrhs == 1) return run_solve(p, f, u, nullptr, nullptr, nullptr);
  int k = (int)std::min<int64_t>(nrhs, p->rhs_concurrency);
  // workspaces follow the plan's settings: rebuilt when any has changed
  for (helm_plan* w : p->ws)
    if (w->version != p->version || (p->ffb && !w->ffb)) {
      HELM_CK(cudaStreamSynchronize(p->stream));
      for (size_t i = 0; i < p->ws_stream.size(); ++i) HELM_CK(cudaStreamSynchronize(p->ws_stream[i]));
      for (helm_plan* q : p->ws) destroy_workspace(q);
      p->ws.clear();
      break;
    }
  while ((int)p->ws.size() < k - 1) {
    helm_plan* w = make_workspace(p);
    if (!w) break;  // no room: fewer right-hand sides at once
    p->ws.push_back(w);
  }
  k = std::min<int>(k, 1 + (int)p->ws.size());
  while ((int)p->ws_stream.size() < k) {
    cudaStream_t st;
    cudaEvent_t ev;
    HELM_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(st);
      return cuda_fail(p, cudaGetLastError(), "cudaEventCreate");
    }
    p->ws_stream.push_back(st);
    p->ws_done.push_back(ev);
  }
  if (!p->fork) HELM_CK(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
  // fork: every workspace stream starts after the work already on the plan's stream
  HELM_CK(cudaEventRecord(p->fork, p->stream));
  for (int w = 0; w < k; ++w) HELM_CK(cudaStreamWaitEvent(p->ws_stream[w], p->fork, 0));
  const cudaStream_t caller = p->stream;
  int rc = HELM_OK;
  for (int64_t i = 0; i < nrhs && !rc; ++i) {
    const int w = (int)(i % k);
    helm_plan* q = w == 0 ? p : p->ws[w - 1];
    q->stream = p->ws_stream[w];
    // the FP64-residual graph is tied to f and u: workspaces solve kernel by kernel
    const bool graphs = q->use_graphs;
    if (p->dtype == HELM_C64_REFINED && !refine_ff(p)) q->use_graphs = false;
    rc = run_solve(q, static_cast<const char*>(f) + i * vb, static_cast<char*>(u) + i * vb, nullptr, nullptr, nullptr);
    q->use_graphs = graphs;
    if (rc && q != p) p->err = q->err;
  }
  p->stream = caller;
  // join: the plan's stream continues after every workspace stream
  for (int w = 0; w < k; ++w) {
    HELM_CK(cudaEventRecord(p->ws_done[w], p->ws_stream[w]));
    HELM_CK(cudaStreamWaitEvent(p->stream, p->ws_done[w], 0));
  }
  if (!rc) p->last_many = k;
  return rc;
}

int helm_solve_debug(helm_plan_t p, const void* f, void* u, void* fhat, void* v_b, void* w_b) {
  if (!p || !f || !u || bad_pair(f, u, plan_vec_bytes(p), plan_elem_bytes(p))) return HELM_EINVAL;
  return run_solve(p, f, u, fhat, v_b, w_b);
}

namespace {

// Device address of page-locked host memory mapped into the device's address
// space, or nullptr (pageable memory, or not mapped).
void* mapped_host(const void* h) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

namespace {

// helm_solve_host with the FP64 residual, f already in p->host_f: the
// refinement runs sweep by sweep, the host reading each test's state (a few
// bytes) before it enqueues the next correction.  When the last two
// residuals predict that the next test converges, the copy of u to the host
// starts beside that test (both only read u) on a second stream; if the test
// does not converge after all, the next correction waits for the copy, and u
// is copied again at the end.  The kernels and their order are those of the
// kernel-by-kernel refinement loop, so u is the same bit for bit.
int solve_host_refined(helm_plan* p, void* u_host, size_t bytes) {
  if (!p->out_stream) {
    HELM_CK(cudaStreamCreateWithFlags(&p->out_stream, cudaStreamNonBlocking));
    HELM_CK(cudaEventCreateWithFlags(&p->out_ready, cudaEventDisableTiming));
    HELM_CK(cudaEventCreateWithFlags(&p->out_done, cudaEventDisableTiming));
  }
  bool copying = false;  // a copy of the current u to u_host is on out_stream
  // every return waits for that copy: the caller may reuse u_host at once
  auto fail = [&](int rc) {
    if (copying) cudaStreamSynchronize(p->out_stream);
    return rc;
  };
  auto ck = [&](cudaError_t e, const char* what) { return e == cudaSuccess ? HELM_OK : fail(cuda_fail(p, e, what)); };
  int rc;
  RefineState init{};
  init.tol = p->tol;
  init.max_iter = p->max_iter;
  if ((rc = ck(cudaMemcpyAsync(p->state, &init, sizeof(init), cudaMemcpyHostToDevice, p->stream), "refinement state")))
    return rc;
  if ((rc = refine_first(p, p->host_f, p->host_u, nullptr, nullptr, nullptr))) return rc;
  for (int it = 0; it <= p->max_iter; ++it) {
    if ((rc = refine_check(p, p->host_f, p->host_u, 0))) return fail(rc);
    RefineState st{};
    if ((rc = ck(cudaMemcpyAsync(&st, p->state, sizeof(st), cudaMemcpyDeviceToHost, p->stream), "refinement state")) ||
        (rc = ck(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize")))
      return rc;
    if (st.done || it == p->max_iter) break;
    if (copying) {  // the prediction missed: no correction changes u under the copy
      if ((rc = ck(cudaStreamWaitEvent(p->stream, p->out_done, 0), "cudaStreamWaitEvent"))) return rc;
      copying = false;
    }
    if ((rc = refine_correct(p, p->host_u))) return fail(rc);
    const int k = std::min(st.iters, 16) - 1;  // resid[k]: the last test's ||r|| / ||f||
    if (k >= 1 && st.resid[k - 1] > 0 && st.resid[k] * (st.resid[k] / st.resid[k - 1]) <= st.tol) {
      if ((rc = ck(cudaEventRecord(p->out_ready, p->stream), "cudaEventRecord")) ||
          (rc = ck(cudaStreamWaitEvent(p->out_stream, p->out_ready, 0), "cudaStreamWaitEvent")))
        return rc;
      copying = true;
      if ((rc = ck(cudaMemcpyAsync(u_host, p->host_u, bytes, cudaMemcpyDeviceToHost, p->out_stream), "copy of u")) ||
          (rc = ck(cudaEventRecord(p->out_done, p->out_stream), "cudaEventRecord")))
        return rc;
    }
  }
  if (!copying && (rc = ck(cudaMemcpyAsync(u_host, p->host_u, bytes, cudaMemcpyDeviceToHost, p->stream), "copy of u")))
    return rc;
  if ((rc = ck(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize"))) return rc;
  copying = false;
  return ck(cudaStreamSynchronize(p->out_stream), "copy of u");
}

}  // namespace

int helm_solve_host(helm_plan_t p, const void* f_host, void* u_host) {
  if (!p || !f_host || !u_host || bad_pair(f_host, u_host, plan_vec_bytes(p), plan_elem_bytes(p))) return HELM_EINVAL;
  p->last_many = 0;
  const int64_t N = p->n[0] * p->n[1] * p->n[2];
  const size_t eb = p->dtype == HELM_C64_RAW ? sizeof(float2) : sizeof(double2);
  int rc;
  // The float-float refinement reads f only in its split and writes u only in
  // its join: with mapped page-locked buffers those two kernels work on host
  // memory directly (the transfers overlap the conversions; no staging).
  if (p->dtype == HELM_C64_REFINED && refine_ff(p)) {
    void* fd = mapped_host(f_host);
    void* ud = mapped_host(u_host);
    if (fd && ud) {
      if ((rc = run_solve(p, fd, ud, nullptr, nullptr, nullptr))) return rc;
      HELM_CK(cudaStreamSynchronize(p->stream));
      return HELM_OK;
    }
  }
  if (!p->host_f) {
    if ((rc = dev_alloc(p, (void**)&p->host_f, N * eb)) || (rc = dev_alloc(p, (void**)&p->host_u, N * eb))) return rc;
  }
  HELM_CK(cudaMemcpyAsync(p->host_f, f_host, N * eb, cudaMemcpyHostToDevice, p->stream));
  if (p->dtype == HELM_C64_REFINED && !refine_ff(p)) return solve_host_refined(p, u_host, N * eb);
  rc = run_solve(p, p->host_f, p->host_u, nullptr, nullptr, nullptr);
  if (rc) return rc;
  HELM_CK(cudaMemcpyAsync(u_host, p->host_u, N * eb, cudaMemcpyDeviceToHost, p->stream));
  HELM_CK(cudaStreamSynchronize(p->stream));
  return HELM_OK;
}

int helm_get_info(helm_plan_t p, helm_info* info) {
  if (!p || !info) return HELM_EINVAL;
  std::memset(info, 0, sizeof(*info));
  // The state is read on the plan's own stream (the workspaces' streams join
  // it at the end of helm_solve_many), not the legacy stream: with another
  // thread building plans on the legacy stream, reading a finished plan's
  // state does not wait for that work.
  const cudaStream_t st = p->stream;
  RefineState s{};
  HELM_CK(cudaMemcpyAsync(&s, p->state, sizeof(s), cudaMemcpyDeviceToHost, st));
  HELM_CK(cudaStreamSynchronize(st));
  int derr_ws = 0;
  for (int w = 1; w < p->last_many; ++w) {
    // after helm_solve_many: report the right-hand side whose refinement ended
    // worst (not converged, else the largest final residual)
    RefineState t{};
    int e = 0;
    HELM_CK(cudaMemcpyAsync(&t, p->ws[w - 1]->state, sizeof(t), cudaMemcpyDeviceToHost, st));
    HELM_CK(cudaMemcpyAsync(&e, p->ws[w - 1]->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    HELM_CK(cudaStreamSynchronize(st));
    derr_ws |= e;
    const double rt = t.iters > 0 ? t.resid[std::min(t.iters, 16) - 1] : 0.0;
    const double rs = s.iters > 0 ? s.resid[std::min(s.iters, 16) - 1] : 0.0;
    if (p->dtype == HELM_C64_REFINED && (t.converged < s.converged || (t.converged == s.converged && rt > rs))) s = t;
  }
  info->dim = p->dim;
  info->dtype = p->dtype;
  for (int k = 0; k < 3; ++k) info->n[k] = p->n[k];
  info->iterations = p->dtype == HELM_C64_REFINED ? std::max(0, s.iters - 1) : 0;
  info->converged = p->dtype == HELM_C64_REFINED ? s.converged : 1;
  for (int k = 0; k < 16 && k < s.iters; ++k) info->residual[k] = s.resid[k];
  info->plan_seconds = p->plan_seconds;
  info->tol = p->tol;
  info->max_iter = p->max_iter;
  info->n_dft_stages = p->axo.dft.nstages;
  info->device_bytes = p->bytes + (p->dim == 3 ? p->p3.route_bytes : 0);
  for (const helm_plan* w : p->ws) info->device_bytes += w->bytes;
  info->fp64_lines = p->dim == 3 ? plan3d_routed_lines(p->p3) : 0;
  info->element = p->element;
  info->residual_kind = p->resid_kind;
  info->aux_q = p->axo.q;
  info->aux_rho = p->axo.rho;
  info->aux_trial_residual = p->aux_trial_resid;
  for (int k = 0; k < 3; ++k) info->axis_bc[k] = k < p->dim ? p->bc[k] : HELM_BC_ABC;
  int derr = derr_ws;
  if (p->dev_err) {
    int e0 = 0;
    HELM_CK(cudaMemcpyAsync(&e0, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    HELM_CK(cudaStreamSynchronize(st));
    derr |= e0;
  }
  if (derr) {
    p->err = "a bounded device wait gave up (copies did not arrive)";
    return HELM_ETIMEOUT;
  }
  if (p->dtype == HELM_C64_REFINED && !s.converged) return HELM_ENOTCONV;
  return HELM_OK;
}

int helm_batch_create(helm_batch_t* out, int32_t count, const helm_plan_t* plans) {
  if (!out) return HELM_EINVAL;
  *out = nullptr;
  if (count < 1 || !plans) return HELM_EINVAL;
  for (int32_t i = 0; i < count; ++i)
    if (!plans[i]) return HELM_EINVAL;
  helm_batch* b = new (std::nothrow) helm_batch();
  if (!b) return HELM_ENOMEM;
  b->plans.assign(plans, plans + count);
  // float-float buffers must exist before a capture (no allocation inside it)
  for (helm_plan* p : b->plans)
    if (p->dtype == HELM_C64_REFINED && refine_ff(p) && !p->ffb) {
      const int64_t N = p->n[0] * p->n[1] * p->n[2];
      int rc;
      if ((rc = dev_alloc(p, (void**)&p->ffb, N * sizeof(float4))) ||
          (rc = dev_alloc(p, (void**)&p->ufb, N * sizeof(float4)))) {
        delete b;
        return rc;
      }
    }
  *out = b;
  return HELM_OK;
}

int helm_batch_set_stream(helm_batch_t b, void* s) {
  if (!b) return HELM_EINVAL;
  b->stream = (cudaStream_t)s;
  return HELM_OK;
}

int helm_batch_solve(helm_batch_t b, const void* const* f, void* const* u) {
  if (!b || !f || !u) return HELM_EINVAL;
  const size_t n = b->plans.size();
  for (size_t i = 0; i < n; ++i) {
    helm_plan* p = b->plans[i];
    if (!f[i] || !u[i] || bad_pair(f[i], u[i], plan_vec_bytes(p), plan_elem_bytes(p))) return HELM_EINVAL;
    if (p->prof.on) return HELM_EINVAL;  // event timing cannot live inside the graph
    if (p->dtype == HELM_C64_REFINED && refine_ff(p) && !p->ffb) return HELM_EINVAL;  // kind changed after create
  }
  bool same = b->exec && b->kf.size() == n;
  for (size_t i = 0; same && i < n; ++i)
    same = b->kf[i] == f[i] && b->ku[i] == u[i] && b->kv[i] == b->plans[i]->version;
  if (!same) {
    // the capture reads plan state built by earlier work on other streams
    if (cudaDeviceSynchronize() != cudaSuccess) {
      b->err = "cudaDeviceSynchronize";
      return HELM_ECUDA;
    }
    if (int rc = build_batch_graph(b, f, u)) return rc;
  }
  if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) {
    cudaGetLastError();
    b->err = "cudaGraphLaunch";
    return HELM_ECUDA;
  }
  return HELM_OK;
}

const char* helm_batch_last_error(helm_batch_t b) { return b ? b->err.c_str() : "null batch"; }

int helm_batch_destroy(helm_batch_t b) {
  if (!b) return HELM_OK;
  drop_batch_graph(b);
  for (int k = 0; k < 2; ++k)
    if (b->cap[k]) cudaStreamDestroy(b->cap[k]);
  delete b;
  return HELM_OK;
}

int helm_destroy(helm_plan_t p) {
  if (!p) return HELM_OK;
  // every stream of the plan is done with its memory before it is freed
  cudaStreamSynchronize(p->stream);
  for (cudaStream_t st : p->ws_stream) cudaStreamSynchronize(st);
  destroy_plan(p);
  return HELM_OK;
}

const char* helm_status_string(int s) {
  switch (s) {
    case HELM_OK: return "HELM_OK";
    case HELM_EINVAL: return "HELM_EINVAL: invalid argument";
    case HELM_ENOMEM: return "HELM_ENOMEM: allocation failed";
    case HELM_ECUDA: return "HELM_ECUDA: CUDA runtime error";
    case HELM_ENOTCONV: return "HELM_ENOTCONV: refinement did not reach the tolerance";
    case HELM_ETIMEOUT: return "HELM_ETIMEOUT: bounded device wait gave up";
    case HELM_EUNSUPPORTED: return "HELM_EUNSUPPORTED: size not supported by the kernels";
    case HELM_ENUMERIC: return "HELM_ENUMERIC: plan eigen-data failed";
    default: return "unknown helm status";
  }
}

const char* helm_last_error(helm_plan_t p) { return p ? p->err.c_str() : ""; }

int helm_set_profiling(helm_plan_t p, int enable) {
  if (!p) return HELM_EINVAL;
  p->prof.on = enable != 0;
  p->prof.reset();
  return HELM_OK;
}

int helm_get_profile(helm_plan_t p, helm_profile_entry* out, int max_entries) {
  if (!p || (max_entries > 0 && !out)) return HELM_EINVAL;
  HELM_CK(cudaStreamSynchronize(p->stream));
  std::vector<double> ms(p->prof.names.size(), 0.0);
  std::vector<int> cnt(p->prof.names.size(), 0);
  for (auto& m : p->prof.marks) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) {
      ms[m.name] += t;
      cnt[m.name] += 1;
    }
  }
  cudaGetLastError();
  int k = 0;
  for (size_t i = 0; i < ms.size() && k < max_entries; ++i) {
    if (!cnt[i]) continue;
    std::memset(&out[k], 0, sizeof(out[k]));
    std::strncpy(out[k].name, p->prof.names[i].c_str(), sizeof(out[k].name) - 1);
    out[k].launches = cnt[i];
    out[k].total_ms = ms[i];
    ++k;
  }
  p->prof.reset();
  return k;
}

int helm_solve_2d_static(int64_t nx, int64_t ny, double hx, double hy, double omega, const void* f, void* u,
                         void* cuda_stream) {
  if (!f || !u) return HELM_EINVAL;
  if (nx < 3 || ny < 3 || !(hx > 0) || !(hy > 0) || !std::isfinite(hx) || !std::isfinite(hy)) return HELM_EINVAL;
  if (validate_common(omega, HELM_C128)) return HELM_EINVAL;
  if (ny > kStaticMaxN1) return HELM_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // stack plan: same kernels and argument blocks as helm_solve (complex128)
  helm_plan sp;
  sp.dim = 2;
  sp.n[0] = nx;
  sp.n[1] = ny;
  sp.h[0] = hx;
  sp.h[1] = hy;
  sp.omega = omega;
  sp.wc[0] = sp.wc[1] = omega;
  sp.dtype = HELM_C128;
  sp.prec = kPrecF64;
  sp.stream = st;
  AxisData& ax = sp.axo;
  ax.n = ny;
  ax.h = hy;
  ax.wc = omega;
  dft_factor(ny, &ax.dft);
  int dev = 0, smem = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices ||
      cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return HELM_ECUDA;
  }
  if (!dft_supported(ax.dft, sizeof(double2), smem) || dft_needs_bluestein(ax.dft)) return HELM_EUNSUPPORTED;
  // scratch layout
  const int64_t N = nx * ny;
  const Solve2DArgs a0 = args2d(&sp);
  const size_t nrec = (size_t)a0.nchunks * ny;
  const int64_t nwarps = (ny + 31) / 32;
  const size_t tab = align256(2 * ny * sizeof(double));
  size_t off[16], cur = 0;
  const size_t sizes[14] = {tab, tab, tab, tab, align256(ny * sizeof(double)), tab, tab, tab,
                            align256(N * sizeof(double2)), align256(N * sizeof(double2)),
                            align256(2 * nwarps * nx * sizeof(double2)), align256(8 * nx * sizeof(double2)),
                            align256(2 * nrec * sizeof(double2)), align256(nrec * chunk_record_bytes(kPrecF64))};
  for (int i = 0; i < 14; ++i) {
    off[i] = cur;
    cur += sizes[i];
  }
  if (cur > kStaticScratchBytes) return HELM_EUNSUPPORTED;
  if (bad_pair(f, u, (size_t)N * sizeof(double2), sizeof(double2))) return HELM_EINVAL;
  // set-up once per device, with that device current: the device address of
  // the static array (the host-side symbol is not a device pointer)
  if (!g_static_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_helm_static_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return HELM_ECUDA;
    }
    g_static_addr[dev] = ptr;
  }
  char* base = (char*)g_static_addr[dev];
  // plan-time data on the host, into static arrays
  if (abc_eigen_static(ny, hy, omega, g_st_lamA, g_st_sigA, g_st_par8, g_st_work,
                       (int64_t)(sizeof(g_st_work) / sizeof(double))) != HELM_OK)
    return HELM_ENUMERIC;
  for (int64_t l = 0; l < ny; ++l) g_st_parA[l] = g_st_par8[l];
  unit_roots(ny, g_st_twre, g_st_twim);
  for (int64_t l = 0; l < ny; ++l) {
    g_st_tw[2 * l] = g_st_twre[l];
    g_st_tw[2 * l + 1] = g_st_twim[l];
  }
  static_aux_tables(ax, kDefaultAuxRho, kDefaultAuxQ);
  ax.lamB = (double*)(base + off[0]);
  ax.invmu = (double*)(base + off[1]);
  ax.lamA = (double*)(base + off[2]);
  ax.sigA = (double*)(base + off[3]);
  ax.parA = (double*)(base + off[4]);
  ax.tw = (double*)(base + off[5]);
  ax.sc_in = (double*)(base + off[6]);
  ax.sc_out = (double*)(base + off[7]);
  sp.fhat = base + off[8];
  sp.dbuf = base + off[9];
  sp.partial = base + off[10];
  sp.faces = base + off[11];
  sp.ustartB = base + off[12];
  sp.ustartA = base + off[12] + nrec * sizeof(double2);
  sp.rec = base + off[13];
  sp.nwarps = nwarps;
  sp.face_len = nx;
  const size_t tb = 2 * ny * sizeof(double);
  const struct {
    void* dst;
    const void* src;
    size_t bytes;
  } up[8] = {{ax.lamB, g_st_lamB, tb},  {ax.invmu, g_st_invmu, tb}, {ax.lamA, g_st_lamA, tb},
             {ax.sigA, g_st_sigA, tb},  {ax.parA, g_st_parA, ny * sizeof(double)},
             {ax.tw, g_st_tw, tb},      {ax.sc_in, g_st_sci, tb},     {ax.sc_out, g_st_sco, tb}};
  for (int i = 0; i < 8; ++i)
    if (cudaMemcpyAsync(up[i].dst, up[i].src, up[i].bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      cudaGetLastError();
      return HELM_ECUDA;
    }
  // the array keeps the previous call's contents: clear the face sums
  if (cudaMemsetAsync(sp.partial, 0, sizes[10] + sizes[11], st) != cudaSuccess) {
    cudaGetLastError();
    return HELM_ECUDA;
  }
  const Solve2DArgs a = args2d(&sp);
  if (launch_pivots(kPrecF64, sp.ustartB, a, 1, st) != cudaSuccess ||
      launch_pivots(kPrecF64, sp.ustartA, a, 2, st) != cudaSuccess) {
    cudaGetLastError();
    return HELM_ECUDA;
  }
  return solve2d_core(&sp, f, 1, u, kOutC128, 0.0, nullptr, nullptr, nullptr, nullptr);
}

int helm_abc_eigen(int64_t n, double h, double omega, double* lam, double* sigma, int8_t* parity) {
  if (!lam || !sigma || !parity) return HELM_EINVAL;
  return abc_eigen(n, h, omega, lam, sigma, parity);
}

int helm_dft_factor(int64_t n, int32_t* radices, int32_t max_stages) {
  DftPlan p;
  int ns = dft_factor(n, &p);
  if (radices)
    for (int i = 0; i < ns && i < max_stages; ++i) radices[i] = p.radix[i];
  return ns;
}

}  // extern "C"
