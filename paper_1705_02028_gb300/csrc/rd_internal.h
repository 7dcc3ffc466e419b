// rd_internal.h -- internal types shared by the mesh store (host) and the CUDA kernels.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/rd.h"

namespace rd {

// Host-side mesh store: everything the device buffers are built from.
// Internal order: vertices and triangles renumbered by the chosen reordering.
struct HostMesh {
  int32_t nv = 0, nt = 0;
  double Lx = 0, Ly = 0;
  std::vector<int32_t> vperm;    // [nv]  internal vertex -> caller vertex
  std::vector<int32_t> vinv;     // [nv]  caller vertex -> internal vertex
  std::vector<int32_t> tperm;    // [nt]  internal triangle -> caller triangle
  std::vector<int32_t> tri;      // [3][nt] corners (internal vertex ids), component-major
  std::vector<double> nx, ny;    // [3][nt] unit inward normal of the edge opposite each corner
  std::vector<double> hl;        // [3][nt] half length of that edge
  std::vector<double> area;      // [nt]   |T|
  std::vector<double> lmax;      // [nt]   longest edge l_max^T
  std::vector<double> V;         // [nv]   V_i = sum_{T containing i} |T| / 3
  std::vector<int32_t> csr_ptr;  // [nv+1] vertex -> incident (triangle, corner) entries
  std::vector<int32_t> csr_ent;  // [3 nt] entry = 3 * triangle + corner, ascending per vertex
};

// Validates and builds the host mesh store.  Returns an RD_* status.
int build_host_mesh(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
                    const int8_t* shift, double Lx, double Ly, int32_t reorder, HostMesh& out);

// Plan of part r of a P-way vertex partition (rd_partition.cpp): owned
// internal vertex range [v0, v1); local vertices lv (owned first, then the
// ghost vertices ascending); local triangles lt (ascending internal ids: every
// triangle with an owned corner) with their corners ltri [3][nlt] in local
// vertex ids; the CSR of the owned local vertices over local triangle
// entries 3 k + c; per peer q the ghosts it owns, local slots
// [n_own + recv_ptr[q], n_own + recv_ptr[q+1]), and the owned local vertices
// it needs, send_idx[send_ptr[q] .. send_ptr[q+1]) in q's ghost order.
struct PartPlanHost {
  int P = 1, r = 0;
  int32_t v0 = 0, v1 = 0;
  std::vector<int32_t> lv, lt, ltri, csr_ptr, csr_ent, recv_ptr, send_ptr, send_idx;
};
int build_part_plan(const HostMesh& h, int P, int r, PartPlanHost& out);

// Tile plan of the tiled step (host form; the device copy is rd::TilePlan).
// Triangles, sorted by their smallest vertex id, form tiles of tt consecutive
// triangles; tile p owns the vertices [vs[p], vs[p+1]); its halo vertices are
// hlist[hptr[p] .. hptr[p+1]); lslot[c][t] is corner c's slot in its tile
// (owned vertex v -> v - vs[p], halo vertex -> owned count + halo index);
// a vertex is a boundary vertex when one of its triangles precedes its tile,
// and bmask[t] bit c flags corner c of t at such a vertex.
constexpr int MAX_TILE_TRIANGLES = 4096;
struct TilePlanHost {
  int tt = 0, n_tiles = 0, n_bvert = 0, slots = 0;
  std::vector<int32_t> vs, hptr, hlist, bvert;
  std::vector<uint16_t> lslot;
  std::vector<uint8_t> bmask;
};

// Plan for tiles of tt triangles (a multiple of 32, at most
// MAX_TILE_TRIANGLES).  RD_ENOTSUP if the triangles are not sorted by their
// smallest vertex id (a mesh created without reordering) or a tile would
// touch more than 65535 vertices.
int build_tile_plan(const HostMesh& h, int tt, TilePlanHost& out);

// Device control block of one state (one per mesh in batched mode).
struct DevCtl {
  double dt;              // dt of the current step
  double t;               // simulation time after the last committed step
  double t_end;           // > 0: stop when t reaches t_end
  long long steps;        // committed steps
  int status;             // sticky error bits (RD_ST_*)
  int stop;               // nonzero: remaining kernels of this run are no-ops
  unsigned int ticket;    // last-block-done counter of the dt reduction
  int pad;
};

// Control word of the standalone CFL reduction (must start at zero).
struct DtScratchCtl {
  unsigned int ticket;
  int status;
};

// Standalone CFL time step on caller-owned device arrays (rd_cfl_dt): argument
// check, then launch on `stream` with the given scratch (block minima of
// ceil(nv / 256) doubles and the control word) and wait for the result.
int cfl_dt_check(int32_t nv, int32_t nt, int32_t precision, const void* W, const int32_t* tri, const void* lmax,
                 const void* V, const int32_t* ptr, const int32_t* ent, double gamma, double cfl, double* dt_out);
int cfl_dt_launch(int32_t nv, int32_t nt, int32_t precision, const void* W, const int32_t* tri, const void* lmax,
                  const void* V, const int32_t* ptr, const int32_t* ent, double gamma, double cfl, double* dt_out,
                  void* stream, double* partial, DtScratchCtl* ctl);
constexpr int CFL_DT_BLOCK = 256;

enum : int {
  ST_NONPHYS_VERTEX = 1,  // rho <= 0, p <= 0 or NaN at a vertex
  ST_ROE = 2,             // c^2 <= 0 at a Roe state
  ST_SINGULAR = 4,        // zero pivot in (sum_j K_j^-)
};

}  // namespace rd
