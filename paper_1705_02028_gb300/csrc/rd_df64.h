// rd_df64.h -- launchers of the RD_DF64 triangle kernels on explicit arrays
// (used by the plain state and by the partitioned state).
#pragma once

#include "rd_device.h"
#include "rd_kernels.cuh"

#include <vector>

namespace rd {

// Geometry of the double-float kernels: nx, ny, hl [3][nt] and area [nt] as
// double-float pairs (float2 hi, lo), l_max [nt] in double.
struct DevGeoDF {
  const float2 *nx = nullptr, *ny = nullptr, *hl = nullptr, *area = nullptr;
  const double* lmax = nullptr;
};

// FP64 state layout; rec holds 16 double-float values per triangle.  Stage 1
// reads Z, spd; stage 2 reads Z (= Z*) and dw = W* - W^n split into
// double-float pairs ([nv][4] float2, written by the stage-1 update).
struct TriArraysDF {
  int nt = 0;
  const int* tri = nullptr;
  DevGeoDF g{};
  const double *Z = nullptr, *spd = nullptr;
  const float2* dw = nullptr;
  double* share = nullptr;
  void* rec = nullptr;
  double* cfl = nullptr;
  DevCtl* ctl = nullptr;
  // kernel variant: 2 (128 registers), 3 (128, block barriers between phases),
  // 4 (96 registers, barriers), 5 (80 registers, barriers)
  int variant = 2;
  const double* dtm = nullptr;      // batched form: per-mesh dt, indexed by tmesh[t]
  const uint16_t* tmesh = nullptr;
};
int launch_tri_stage1_df(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
                         cudaStream_t st);
// The kernels of one variant: REGS registers per thread (128, 96 or 80), SYNC a
// block barrier between the phases of the per-triangle algebra.  Defined in
// rd_df64_kernels.cuh, instantiated in rd_df64_s{1,2}_r128.cu and
// rd_df64_s{1,2}_r96_80.cu.
template <int REGS, bool SYNC>
int df_stage1(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
              cudaStream_t st);
template <int REGS, bool SYNC>
int df_stage2(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
              cudaStream_t st);
int launch_tri_stage2_df(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
                         cudaStream_t st);

// Upload the mesh's double-float geometry once (rd_mesh::geo_df).
int mesh_geometry_df(rd_mesh* m);
void split_df_host(const std::vector<double>& x, std::vector<float2>& out);

}  // namespace rd
