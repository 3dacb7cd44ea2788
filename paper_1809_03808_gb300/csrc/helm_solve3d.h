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
  bool ready = false;
};

cudaError_t plan3d_init(Plan3D& p, int prec, const int64_t* n, const double* h, double omega, const AxisData& axo,
                        const AxisData& axi, size_t* bytes);
// (Re)build the pivot tables from the current eigen-data (after a change of
// the auxiliary).
cudaError_t plan3d_tables(Plan3D& p);
void free_plan3d(Plan3D& p);
cudaError_t solve3d_core(Plan3D& p, int prec, const void* in, int in_is_double, void* out, int out_mode,
                         double accum_scale, const int* skip, void* dbg_fhat, void* dbg_v, void* dbg_w,
                         cudaStream_t st, Profiler* prof);

}  // namespace helm
