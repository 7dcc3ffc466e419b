// rd_df64.h -- launchers of the RD_DF64 triangle kernels on explicit arrays
// (used by the plain state and by the partitioned state).
#pragma once

#include "rd_device.h"
#include "rd_kernels.cuh"

namespace rd {

// FP64 layout; rec holds 16 double-float values per triangle.  Stage 1 reads
// Z, spd; stage 2 reads Z (= Z*), Wn, Ws.
struct TriArraysDF {
  int nt = 0;
  const int* tri = nullptr;
  DevGeo<double> g{};
  const double *Z = nullptr, *spd = nullptr, *Wn = nullptr, *Ws = nullptr;
  double* share = nullptr;
  void* rec = nullptr;
  double* cfl = nullptr;
  DevCtl* ctl = nullptr;
  int occ = 1;  // kernel variant: 1 (255 registers), 2 (128), 3 (128, block barriers between phases)
};
int launch_tri_stage1_df(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
                         cudaStream_t st);
int launch_tri_stage2_df(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
                         cudaStream_t st);

}  // namespace rd
