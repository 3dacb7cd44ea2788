// 3D solve (Section 5): the 2D fast solver applied per outer mode.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "helm_internal.h"
#include "helm_prof.h"

namespace helm {

struct Plan3D {
  int prec = 0;
  int64_t n[3] = {0, 0, 0};
  double h[3] = {0, 0, 0};
  double omega = 0;
  double wc[3] = {0, 0, 0};  // w of the absorbing ends of each axis (0: Neumann axis)
  double mden = 6.0;         // mass matrix denominator of the elements (MassCoef)
  const AxisData* axo = nullptr;  // outer periodic axis (array axis 1)
  const AxisData* axi = nullptr;  // inner periodic axis (array axis 2)
  void* fhat = nullptr;
  void* cbuf = nullptr;
  void* dbuf = nullptr;
  void* ybuf = nullptr;
  void* faces = nullptr;
  void* partial = nullptr;
  // reciprocal pivots of the inner lines, [outer A][inner A] (nullptr: none)
  void* tab[4] = {nullptr, nullptr, nullptr, nullptr};
  // per inner line of each type: 1/u_inf and 1/u_{nx-1} (2 complex values),
  // and the row from which the pivots have settled at 1/u_inf
  void* lend[4] = {nullptr, nullptr, nullptr, nullptr};
  int* lenL[4] = {nullptr, nullptr, nullptr, nullptr};
  // tiled inner sweeps: face partials [ny][nparts][2][nx], inner faces
  // v_in, w_in [ny][2][2][nx], inner C_bb output [ny][2][nx]
  void* ipart = nullptr;
  void* ivw = nullptr;
  void* icin = nullptr;
  int inner_ch = 0;      // rows per chunk of the tiled sweeps
  int inner_nc = 0;      // chunks per line
  int inner_nmb = 0;     // inner-mode blocks per CTA (0: tiled sweeps off)
  int inner_nparts = 0;  // face partials per plane
  // precision routing (complex64 plans): inner lines of each type whose line
  // matrix is close to singular are solved in FP64 by a separate kernel.
  // rlist: their line indices l * nz + m, ascending; roff: per outer mode l
  // the range [roff[l], roff[l+1]) of rlist; rtab: their FP64 reciprocal
  // pivots [route][nx]; rpart: their face contributions [route][2][nx];
  // rtmp: FP64 Thomas scratch [route][nx].
  double route_tau = 0;  // routing threshold (0: off)
  int nroute[4] = {0, 0, 0, 0};
  int* rlist[4] = {nullptr, nullptr, nullptr, nullptr};
  int* roff[4] = {nullptr, nullptr, nullptr, nullptr};
  void* rtab[4] = {nullptr, nullptr, nullptr, nullptr};
  void* rpart = nullptr;
  void* rtmp = nullptr;
  size_t route_bytes = 0;  // device memory of the routing tables
  bool ready = false;
};

cudaError_t plan3d_init(Plan3D& p, int prec, const int64_t* n, const double* h, double omega, const double* wc, double mden,
                        const AxisData& axo, const AxisData& axi, size_t* bytes);
// (Re)build the pivot tables from the current eigen-data (after a change of
// the auxiliary), and the precision routing of complex64 plans.
cudaError_t plan3d_tables(Plan3D& p);
// Set the routing threshold tau (complex64 plans; 0 turns routing off) and
// rebuild the routing tables.  A line is routed to FP64 when the smallest
// |Lam^A_x,k + Lam_outer + Lam_inner - w^2| over the eigenvalues Lam^A_x,k of
// its own axis is below tau w^2.
cudaError_t plan3d_set_routing(Plan3D& p, double tau);
// Routed lines of all four line types.
int plan3d_routed_lines(const Plan3D& p);
// Shape of the tiled inner sweeps: ch rows per chunk, nmb tiles per CTA
// (cudaErrorInvalidValue if the tile does not fit); rebuilds the tables.
cudaError_t plan3d_set_inner(Plan3D& p, int ch, int nmb);
// The pivot tables alone (the routed flags cleared).
cudaError_t plan3d_tables_no_routing(Plan3D& p);
void free_plan3d(Plan3D& p);
cudaError_t solve3d_core(Plan3D& p, int prec, const void* in, int in_is_double, void* out, int out_mode,
                         double accum_scale, const int* skip, void* dbg_fhat, void* dbg_v, void* dbg_w,
                         cudaStream_t st, Profiler* prof);

}  // namespace helm
