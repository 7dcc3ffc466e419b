// rd_device.h -- device-memory helpers and the mesh handle shared by the C ABI
// translation units (rd_api.cu, rd_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include "rd_internal.h"

namespace rd {

// A device buffer and the allocator that owns it.
struct DevBuf {
  void* p = nullptr;
  rd_free_fn fr = nullptr;  // allocator that owns p (nullptr: cudaFree)
  void* ctx = nullptr;
};

// Allocate through the installed allocator hook (default cudaMalloc).
int dev_alloc(DevBuf& b, size_t bytes, cudaStream_t s);
void dev_free(DevBuf& b);

#define CU(x)                 \
  do {                        \
    cudaError_t e_ = (x);     \
    if (e_ != cudaSuccess) {  \
      cudaGetLastError();     \
      return RD_ECUDA;        \
    }                         \
  } while (0)

#define CK(x)                   \
  do {                          \
    int s_ = (x);               \
    if (s_ != RD_OK) return s_; \
  } while (0)

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// Default block sizes (the autotuner may pick others): triangle kernels allow
// up to 256 threads per block, vertex kernels up to 512.
constexpr int TRI_BLOCK = 128;
constexpr int VTX_BLOCK = 256;
constexpr int VTX_BLOCK_MIN = 128;

// Launch the dt gather with a runtime block size of 128, 256 or 512.
template <class T>
void launch_gather_cfl(int vblock, cudaStream_t st, int nv, const int* ptr, const int* ent, const T* share,
                       const T* cfl, const T* V, T* R1, T* partial, T cflnum, DevCtl* ctl);

// Tiled step (rd_state_set_tiling).  Triangles, sorted by their smallest
// vertex id, are cut into tiles of tt consecutive triangles; tile p owns the
// vertex range [vs[p], vs[p+1]) (vs[p] = smallest vertex of triangle p tt).
// A vertex all of whose triangles lie in its own tile is interior and is
// gathered on chip; the others (boundary vertices) through global memory.
struct TilePlan {
  int tt = 0, bt = 0;     // triangles per tile, threads per block
  bool gs = false;        // stage each tile's geometry in shared memory (RD_TILE_STAGE_GEOMETRY)
  int n_tiles = 0, n_bvert = 0;
  int slots = 0;          // max over tiles of owned + halo vertices
  DevBuf vs;              // [n_tiles + 1] int32 vertex range of each tile
  DevBuf hptr, hlist;     // [n_tiles + 1], halo vertex ids (ascending per tile)
  DevBuf lslot;           // [3][nt] uint16: slot of each corner in its tile
  DevBuf bmask;           // [nt] uint8: bit c = corner c is a boundary vertex
  DevBuf bvert;           // [n_bvert] int32 boundary vertices, ascending
  DevBuf partial;         // dt block minima: tiles, then boundary blocks (8 B each)
};
void tile_plan_free(TilePlan* tp);

}  // namespace rd

struct rd_adjoint_store;
struct rd_state;
namespace rd {
void adjoint_free(rd_adjoint_store* a);
// One committed step of a state reading buffer a (fixed_dt > 0 replaces the CFL dt).
int state_step(rd_state* s, int a, double fixed_dt);
// Boundary data of a mesh (rd_boundary.cu).
template <class T>
int mesh_wall_geometry(rd_mesh* m);
void mesh_boundary_free(rd_mesh* m);
int state_read_ctl(const rd_state* s, DevCtl& c);
}

// The mesh handle: host mesh store plus its device arrays.
struct rd_mesh {
  rd::HostMesh h;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  rd::DevBuf tri, ptr, ent, vperm, vinv;  // vperm: internal -> caller vertex, vinv: caller -> internal
  // geometry per precision (0: double, 1: float): nx, ny, hl, area, lmax, V
  rd::DevBuf geo[2][6];
  bool geo_ready[2] = {false, false};
  // RD_DF64: nx, ny, hl [3][nt] and area [nt] as double-float pairs (float2)
  rd::DevBuf geo_df[4];
  bool geo_df_ready = false;
  // boundary conditions (Sec. 3.5), set by rd_mesh_set_boundary
  int bc_version = 0;
  int32_t n_ghost = 0, n_wall = 0;
  double wall_alpha = 0.75;
  rd::DevBuf ghost_of;   // [nv] int32: ghost slot of each internal vertex, -1 if none
  rd::DevBuf ghost_ids;  // [n_ghost] internal vertex ids
  rd::DevBuf wptr;       // [nv + 1] wall CSR: internal vertex -> wall-edge ends
  rd::DevBuf wother;     // [2 n_wall] the other vertex of each end's edge
  rd::DevBuf wgeo[2];    // per precision: [2 n_wall][3] outward unit normal x, y, half length
  std::vector<double> wgeo_host;
  bool wgeo_ready[2] = {false, false};
};

namespace rd {
// Triangle kernels of an RD_DF64 state (rd_df64.cu): stage 1 reads buffer a,
// stage 2 reads W^n from buffer a and W*, Z* from the stage scratch.
int launch_tri_stage1_df(const rd_state* s, int a, unsigned grid, int block, cudaStream_t st);
int launch_tri_stage2_df(const rd_state* s, int a, unsigned grid, int block, cudaStream_t st);
}

// The state handle: double-buffered vertex state, step scratch and the device
// control block (dt, time, step count, status).
struct rd_state {
  rd_mesh* m = nullptr;
  rd_params p{};
  int pi = 0;     // 0: double, 1: float
  size_t ts = 8;  // sizeof(T)
  rd::DevBuf W[2], Z[2], spd[2];
  rd::DevBuf Ws, Zs, R1, share, rec, cfl, partial, ctl, cons_partial, cons_out;
  rd::DevBuf dWdf;         // RD_DF64 two-stage: W* - W^n as double-float pairs, [nv][4] float2
  rd::DevBuf stage;        // [4][nv] double, caller vertex order (host I/O)
  rd::DevBuf vr;           // RD_BX2: |v| max / min bits, slot 0 (W^n) and slot 1 (W*)
  rd::DevBuf ghostW;       // [n_ghost][4] T: initial state of the ghost vertices
  int bc_version = 0;      // mesh boundary version the state was set up for
  bool bc_init = false;
  long long launched = 0;  // host view of the committed step count (parity of the buffers)
  int tri_block = rd::TRI_BLOCK, vtx_block = rd::VTX_BLOCK;  // launch shapes (autotuned); tri_block: stage 1
  int tri_block2 = rd::TRI_BLOCK;                             // stage-2 triangle kernel
  // RD_DF64 triangle-kernel variant of stage 1 and stage 2 (2: 128 registers;
  // 3: 128 with phase barriers; 4: 96 with phase barriers; 5: 80 with phase
  // barriers; autotuned per stage)
  int df_variant = 2, df_variant2 = 2;
  rd::TilePlan* tiles = nullptr;  // tiled step (nullptr: per-triangle share arrays)
  cudaGraphExec_t g2 = nullptr;  // two steps (even -> odd -> even)
  bool graph_failed = false;
  rd_adjoint_store* adj = nullptr;  // checkpoints and buffers of the adjoint rollout
};
