// Host launchers and argument blocks for the solve kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "helm_internal.h"
#include "helm_prof.h"

namespace helm {

// Arguments of the 2D per-mode tridiagonal kernels (device pointers to the
// x1-axis eigen-data, FP64).
struct Solve2DArgs {
  int64_t nx;     // points along the tridiagonal axis
  int64_t n1;     // x1 length (modes)
  double hx;      // tridiagonal-axis spacing
  double h1;      // x1 spacing
  double omega;
  const double* lamB;   // complex Lam^B_l of the auxiliary
  const double* invmu;  // complex 1/mu_l
  const double* lamA;
  const double* sigA;
  const double* parA;
  const double* tw;
  int64_t ch;       // rows per chunk of the tridiagonal sweeps
  int64_t nchunks;  // ceil(nx / ch)
  double eninv[2];  // e^{-t (n1-1)}: weight of the last x1 face in the Step-3 rhs
  double wx = 0;    // w of the absorbing corners along x (0: Neumann x faces)
  double wy = 0;    // w of the absorbing x1 faces (0: Neumann), in C_bb
  int tri_regs = 0;  // complex64 passes: 1 = register-tile kernels even where the bulk-copy ones apply
  double mden = 6.0;  // mass matrix denominator: 6 the paper's elements, 12 the modified ones (MassCoef)
};

constexpr int kChunkF32 = 16;
constexpr int kChunkF64 = 8;

// One per-mode tridiagonal step (1, 2 or 3): pass 1, carry scan, pass 2.
// ustart: pivot entering each chunk (launch_pivots, per step type: B for 1 and
// 3, A for 2); rec: nchunks*n1 chunk records; out: x (step 3); partial: face
// sums (steps 1, 2).
// consts: optional per-line constants (launch_line_consts, same line type as
// the step); nullptr makes the kernels compute them per thread.
cudaError_t launch_tri2d(int prec, int step, const void* fhat, const void* faces, const void* ustart, void* rec,
                         void* out, void* partial, const Solve2DArgs& a, const int* skip, cudaStream_t st,
                         Profiler* prof, const void* consts = nullptr);
size_t line_consts_bytes(int prec, int64_t n1);
cudaError_t launch_line_consts(int prec, void* out, const Solve2DArgs& a, int step, cudaStream_t st);
cudaError_t launch_pivots(int prec, void* ustart, const Solve2DArgs& a, int step, cudaStream_t st);
// FP64 path with per-plan line tables (multipliers, reciprocal pivots, chunk
// weights): table memory per line type, building them, and the step launch.
size_t line_tables_bytes(int64_t nx, int64_t n1, int64_t nchunks);
cudaError_t launch_line_tables(void* tables, const Solve2DArgs& a, int step, cudaStream_t st);
cudaError_t launch_tri2d_tab(int step, const void* fhat, const void* faces, const void* tables, void* rec,
                             void* out, void* partial, const Solve2DArgs& a, const int* skip, cudaStream_t st,
                             Profiler* prof);
// complex64 path with a per-plan pivot table (1/u_j rounded from FP64, chunk
// constants): table memory per line type, building it, and the step launch.
size_t line_tables32_bytes(int64_t nx, int64_t n1, int64_t nchunks);
cudaError_t launch_line_tables32(void* tables, const Solve2DArgs& a, int step, cudaStream_t st);
// err: device error word (bounded waits of the bulk-copy fed kernels).
cudaError_t launch_tri2d_t32(int step, const void* fhat, const void* faces, const void* tables, void* rec, void* out,
                             void* partial, const Solve2DArgs& a, const int* skip, cudaStream_t st, Profiler* prof,
                             const void* consts, int* err);
size_t chunk_record_bytes(int prec);
// out[face][ix] = scale_face * sum_w partial (complex scales, face 0 then 1).
cudaError_t launch_reduce_faces(int prec, const void* partial, void* out, int64_t nx, int64_t nwarps,
                                const double* scale0, const double* scale1, const int* skip, cudaStream_t st);
// C_bb of the auxiliary with wrap factor g (eq. Cbb; g = 1: periodic).
// wx, wy: w of the absorbing x ends and x1 faces (0 on a Neumann axis).
cudaError_t launch_apply_cbb(int prec, const void* in, const void* in2, void* out, int64_t nx, double hx,
                             double h1, double wx, double wy, double p, const double* g, const double* ginv,
                             const int* skip, cudaStream_t st, double mden);

// Refinement state kept on the device (one per plan).
struct RefineState {
  int done;         // set when ||r||/||f|| <= tol; later sweeps skip their kernels
  int iters;        // residual evaluations performed
  int converged;
  int max_iter;     // correction sweeps allowed: done after max_iter + 1 residuals
  double tol;
  double fnorm2;
  double resid[16];
};

// r = f - A u in FP64 (eq. A2D / A3D), r stored as complex64, per-block sums
// of |r|^2 and |f|^2 into `sums` (2 doubles per block).  Returns the number of
// blocks used through *nblocks.
// wc[k]: w of the absorbing ends of axis k (0 on a Neumann axis).  err: the
// device error word set if a bounded wait of the 3D kernel runs out.  mden:
// the mass matrix denominator of the elements (MassCoef).
cudaError_t launch_residual(int dim, const int64_t* n, const double* h, double omega, const double* wc,
                            const double2* f,
                            const double2* u, float2* r, double* sums, int64_t* nblocks, const int* skip,
                            cudaStream_t st, int* err, double mden);
// The same residual with f and u as float-float complex vectors (float4 per
// point: re_hi, im_hi, re_lo, im_lo), about 48 significant bits, computed on
// the FP32 pipes.  Same grid and sums layout as launch_residual.
cudaError_t launch_residual_ff(int dim, const int64_t* n, const double* h, double omega, const double* wc,
                               const float4* f,
                               const float4* u, float2* r, double* sums, int64_t* nblocks, const int* skip,
                               cudaStream_t st, double mden);
// complex128 -> float-float (hi = round(x), lo = round(x - hi)) and back.
// f (complex128) -> float-float out; hi (may be null) also receives the hi
// parts as complex64.
cudaError_t launch_split_ff(const double2* f, float4* out, float2* hi, int64_t N, cudaStream_t st);
cudaError_t launch_join_ff(const float4* u, double2* out, int64_t N, cudaStream_t st);
// Reset *st to the start of a refinement (a kernel, so that it can be captured).
cudaError_t launch_refine_init(RefineState* st, double tol, int max_iter, cudaStream_t stream);
// Deterministic pseudo-random complex128 vector (plan-time trials).
cudaError_t launch_trial_rhs(double2* f, int64_t N, uint64_t seed, cudaStream_t st);
// Number of per-block sums launch_residual writes for this grid.
int64_t residual_blocks(int dim, const int64_t* n);
// Reduce the block sums, record ||r||/||f|| as the next residual of *state,
// set state->done when it is <= tol or after max_iter + 1 residuals.  With
// `cond` != 0 also set that graph conditional to !done (the while node of a
// captured refinement loop); cond = 0 outside a graph.
cudaError_t launch_residual_finalize(const double* sums, int64_t nblocks, RefineState* state,
                                     unsigned long long cond, cudaStream_t st);

}  // namespace helm
