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
  bool ready = false;
};

cudaError_t plan3d_init(Plan3D& p, int prec, const int64_t* n, const double* h, double omega, const double* wc,
                        const AxisData& axo, const AxisData& axi, size_t* bytes);
// (Re)build the pivot tables from the current eigen-data (after a change of
// the auxiliary).
cudaError_t plan3d_tables(Plan3D& p);
void free_plan3d(Plan3D& p);
cudaError_t solve3d_core(Plan3D& p, int prec, const void* in, int in_is_double, void* out, int out_mode,
                         double accum_scale, const int* skip, void* dbg_fhat, void* dbg_v, void* dbg_w,
                         cudaStream_t st, Profiler* prof);

}  // namespace helm
