// rd_df64.cu -- the RD_DF64 precision's host side: dispatch of its triangle
// kernels (rd_df64_kernels.cuh, instantiated in rd_df64_s*_r*.cu) by variant,
// the state's arrays for them, and the mesh's double-float geometry.

#include <cuda_runtime.h>

#include <vector>

#include "rd_device.h"
#include "rd_df64.h"
#include "rd_internal.h"
#include "rd_tiled.h"

namespace rd {

int launch_tri_stage1_df(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
                         cudaStream_t st) {
  switch (a.variant) {
    case 3: return df_stage1<128, true>(p, a, ba, grid, block, st);
    case 4: return df_stage1<96, true>(p, a, ba, grid, block, st);
    case 5: return df_stage1<80, true>(p, a, ba, grid, block, st);
    default: return df_stage1<128, false>(p, a, ba, grid, block, st);
  }
}

int launch_tri_stage2_df(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
                         cudaStream_t st) {
  switch (a.variant) {
    case 3: return df_stage2<128, true>(p, a, ba, grid, block, st);
    case 4: return df_stage2<96, true>(p, a, ba, grid, block, st);
    case 5: return df_stage2<80, true>(p, a, ba, grid, block, st);
    default: return df_stage2<128, false>(p, a, ba, grid, block, st);
  }
}

// The state's arrays for the launchers above.
static TriArraysDF state_arrays(const rd_state* s) {
  const rd_mesh* m = s->m;
  TriArraysDF a;
  a.nt = m->h.nt;
  a.tri = (const int*)m->tri.p;
  a.g.nx = (const float2*)m->geo_df[0].p;
  a.g.ny = (const float2*)m->geo_df[1].p;
  a.g.hl = (const float2*)m->geo_df[2].p;
  a.g.area = (const float2*)m->geo_df[3].p;
  a.g.lmax = (const double*)m->geo[0][4].p;
  a.share = (double*)s->share.p;
  a.rec = s->rec.p;
  a.cfl = (double*)s->cfl.p;
  a.ctl = (DevCtl*)s->ctl.p;
  a.variant = s->df_variant;  // stage 1's; stage 2 sets its own
  return a;
}

int launch_tri_stage1_df(const rd_state* s, int a, unsigned grid, int block, cudaStream_t st) {
  TriArraysDF x = state_arrays(s);
  x.Z = (const double*)s->Z[a].p;
  x.spd = (const double*)s->spd[a].p;
  BlendArgs<double> ba = tile_blend_args<double>(s);
  ba.vr = (unsigned long long*)s->vr.p;
  return launch_tri_stage1_df(s->p, x, ba, grid, block, st);
}

int launch_tri_stage2_df(const rd_state* s, int a, unsigned grid, int block, cudaStream_t st) {
  TriArraysDF x = state_arrays(s);
  x.Z = (const double*)s->Zs.p;
  x.dw = (const float2*)s->dWdf.p;
  x.variant = s->df_variant2;
  BlendArgs<double> ba = tile_blend_args<double>(s);
  unsigned long long* vr0 = (unsigned long long*)s->vr.p;
  ba.vr = vr0 ? vr0 + 2 : nullptr;
  return launch_tri_stage2_df(s->p, x, ba, grid, block, st);
}

// Per-triangle geometry split into double-float pairs (the same split as
// to_df on the device): nx, ny, hl [3][nt] and area [nt] as float2.
int mesh_geometry_df(rd_mesh* m) {
  if (m->geo_df_ready) return RD_OK;
  const std::vector<double>* src[4] = {&m->h.nx, &m->h.ny, &m->h.hl, &m->h.area};
  std::vector<float2> tmp;
  for (int k = 0; k < 4; ++k) {
    split_df_host(*src[k], tmp);
    CK(dev_alloc(m->geo_df[k], tmp.size() * sizeof(float2), m->stream));
    CU(cudaMemcpyAsync(m->geo_df[k].p, tmp.data(), tmp.size() * sizeof(float2), cudaMemcpyHostToDevice, m->stream));
    CU(cudaStreamSynchronize(m->stream));
  }
  m->geo_df_ready = true;
  return RD_OK;
}

void split_df_host(const std::vector<double>& x, std::vector<float2>& out) {
  out.resize(x.size());
  for (size_t i = 0; i < x.size(); ++i) {
    const float h = (float)x[i];
    out[i] = make_float2(h, (float)(x[i] - (double)h));
  }
}

}  // namespace rd
