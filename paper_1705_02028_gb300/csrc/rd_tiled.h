// rd_tiled.h -- the tiled step (rd_tiled.cu) as seen by the C ABI (rd_api.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "rd_device.h"
#include "rd_internal.h"
#include "rd_kernels.cuh"

namespace rd {

// Device copy of a plan for state s with bt threads per block.
int tile_plan_upload(rd_state* s, const TilePlanHost& hp, int bt, bool gs, TilePlan** out);
// Dynamic shared memory of the stage-1 / stage-2 tile kernels (gs: with the
// tile's geometry staged in shared memory).
size_t tile_smem_bytes(int precision, int stage, int tt, int slots, bool gs);
// Stage 1 + the boundary gather and dt (every scheme); ev[1] (nullable array)
// is recorded between the two kernels.
template <class T>
int tiled_stage1(rd_state* s, int a, cudaEvent_t* ev);
// Stage 2 + the final update W[a] -> W[1-a]; ev[4] recorded between the two.
template <class T>
int tiled_stage2(rd_state* s, int a, cudaEvent_t* ev);
// Stage 2 runs tiled for two-stage schemes other than Bx on meshes without
// walls or ghost vertices.
bool tiled_stage2_applies(const rd_state* s);

// Blend configuration of a state's two-stage triangle kernels (Sec. 3.3.3, Sec. 3.4).
template <class T>
BlendArgs<T> tile_blend_args(const rd_state* s) {
  BlendArgs<T> ba;
  ba.mode = s->p.scheme == RD_BMAX2 ? BLEND_MAX : s->p.scheme == RD_BMIN2 ? BLEND_MIN
            : s->p.scheme == RD_BX2 ? BLEND_X : BLEND_B;
  ba.sl = s->p.lumping == RD_LUMP_SELECTIVE;
  double L = s->m->h.Lx > s->m->h.Ly ? s->m->h.Lx : s->m->h.Ly;
  ba.L = (T)(L > 0.0 ? L : 1.0);
  return ba;
}

}  // namespace rd
