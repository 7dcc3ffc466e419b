/*
 * rd.h -- C ABI of the GB300 residual-distribution Euler solver.
 *
 * The library advances the two-dimensional Euler equations of an ideal gas
 * (Paardekooper 2017, Sec. 3) on a triangular mesh with the multidimensional
 * upwind residual-distribution schemes of Sec. 3.3 (N, LDA and the blended B
 * scheme) and either the forward-Euler update of Eq. (eqUpdate) or the
 * explicit two-stage scheme of Sec. 3.4 (Eqs. eqRK1, eqRK2).
 *
 * Conventions (every function):
 *   - Return value: RD_OK (0) or one of the RD_E* codes below; rd_strerror()
 *     gives a message.  No C++ exception crosses this boundary.
 *   - Host arrays passed in are owned by the caller and only read (or, for
 *     *_out arguments, written) during the call.
 *   - The library owns every device buffer and every opaque handle; device
 *     memory comes from the allocator installed with rd_set_allocator()
 *     (default: cudaMalloc/cudaFree) and is released by the *_destroy calls.
 *   - All device work of a mesh and of the states / batches built on it is
 *     ordered on the CUDA stream given to rd_mesh_create().
 *   - Conserved state arrays are component-major ("SoA"): W[k * n_vertex + i]
 *     for component k in (rho, rho u, rho v, e) and vertex i, in the caller's
 *     vertex order.  e = rho |v|^2 / 2 + p / (gamma - 1)  (Sec. 3).
 */
#ifndef RD_H
#define RD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RD_OK 0
#define RD_EINVAL 1        /* bad argument, index, orientation or zero area   */
#define RD_ENOMEM 2        /* device or host allocation failed                */
#define RD_ECUDA 3         /* a CUDA runtime call failed                      */
#define RD_ENONPHYSICAL 4  /* rho<=0, p<=0, Roe c^2<=0, singular N^ or NaN;
                              the state stays at the last good step           */
#define RD_ETIMEOUT 5      /* a bounded device-side wait expired              */
#define RD_ENOTSUP 6       /* combination of options the library does not offer */

/* ---- schemes (Sec. 3.3, Sec. 3.4; labels as in the paper's figures) ------ */
#define RD_N1 0   /* N scheme, forward Euler (first order in space and time)    */
#define RD_B2 1   /* blended B scheme, two-stage update, m^LDA, global lumping */
#define RD_LDA2 2 /* LDA scheme, two-stage update                               */
/* Blended variants of Sec. 3.3.3, two-stage update:
 *   RD_BMAX2 every diagonal entry of Theta set to max_k Theta_kk (favours N),
 *   RD_BMIN2 every diagonal entry set to min_k Theta_kk (favours LDA),
 *   RD_BX2   scalar theta of the shock sensor: theta = min(1, s^2 h_T / L),
 *            s = max(0, -L div v / (|v|_max - |v|_min)), div v of the linear
 *            vertex velocities, h_T = sqrt(2 |T|), L = max(Lx, Ly), |v|
 *            extremes over all vertices of the state being distributed
 *            (0 when they coincide); on the unit box theta = s^2 h.
 * In stage 2 Bmax / Bmin reduce the total-residual Theta_kk; Bx evaluates the
 * sensor at W*.  RD_BX2 is not available in batched mode (RD_ENOTSUP). */
#define RD_BMAX2 3
#define RD_BMIN2 4
#define RD_BX2 5

/* ---- lumping of the stage-2 time derivative (Sec. 3.4) ----------------- */
#define RD_LUMP_GLOBAL 0    /* mass matrices m^N, m^LDA, global lumping       */
#define RD_LUMP_SELECTIVE 1 /* + sum_j (|T| delta_ij / 3 - m^G_ij)(W*_j - W^n_j)/dt,
                               m^G_ij = |T| (delta_ij + 1) / 12 (Galerkin);
                               two-stage schemes only                        */

/* ---- arithmetic precision of the device path --------------------------- */
#define RD_FP64 0
#define RD_FP32 1
/* RD_DF64: FP64 state and FP64 vertex kernels (gathers, updates, dt), with
 * the per-triangle algebra run in double-float arithmetic (pairs of FP32
 * numbers, about 48 significant bits) on the FP32 pipe.  Per triangle the
 * nodal mean Zbar, the differences Z_i - Zbar and (stage 2) W*_i - W^n_i are
 * formed in FP64 first, so the double-float arithmetic acts on the
 * differences that carry the residual.  Same arrays, arguments and results
 * as RD_FP64 to within round-off.  The untiled per-triangle step only: no
 * tiling (RD_ENOTSUP) and no adjoint (RD_ENOTSUP); the batched form and the
 * partitioned step take it. */
#define RD_DF64 2

/* ---- vertex / triangle reordering applied inside the mesh store -------- */
#define RD_ORDER_NONE 0
#define RD_ORDER_MORTON 1 /* Morton (Z-order) of vertex coordinates (Sec. 4.1.4) */
#define RD_ORDER_RCM 2    /* reverse Cuthill-McKee of the vertex graph           */

typedef struct rd_mesh rd_mesh;
typedef struct rd_state rd_state;
typedef struct rd_batch rd_batch;

/* Scheme parameters.
 *   scheme    RD_N1 | RD_B2 | RD_LDA2 | RD_BMAX2 | RD_BMIN2 | RD_BX2
 *   precision RD_FP64 | RD_FP32
 *   cfl       Courant number multiplying the stability bound of Sec. 3.2:
 *             dt = cfl * min_i 2 V_i / sum_{T containing i} l_max^T lambda_max^T
 *   gamma     ratio of specific heats (Sec. 3)
 *   eps_fix   |lambda| is replaced below delta = eps_fix * c * |n_i| / 2 by
 *             (lambda^2 + delta^2) / (2 delta) so that N^ = (sum_j K_j^-)^-1
 *             (Sec. 3.3.1) exists at stagnation; 0 disables it.
 *   lumping   RD_LUMP_GLOBAL (0, the paper's choice for all its tests) |
 *             RD_LUMP_SELECTIVE (two-stage schemes; RD_EINVAL with RD_N1)
 *   reserved  must be 0                                                       */
typedef struct {
  int32_t scheme;
  int32_t precision;
  double cfl;
  double gamma;
  double eps_fix;
  int32_t lumping;
  int32_t reserved;
} rd_params;

/* Device allocator hook: alloc(bytes, cuda_stream, ctx) returns a device
 * pointer (NULL on failure); free(ptr, ctx) releases it.  Installed
 * process-wide; affects buffers allocated after the call.  Passing NULL for
 * both restores cudaMalloc/cudaFree. */
typedef void *(*rd_alloc_fn)(size_t bytes, void *cuda_stream, void *ctx);
typedef void (*rd_free_fn)(void *ptr, void *ctx);
int rd_set_allocator(rd_alloc_fn alloc, rd_free_fn free_fn, void *ctx);

const char *rd_strerror(int status);
int rd_version(void);

/* ---- mesh store -----------------------------------------------------------
 * rd_mesh_create: validate a triangulation, compute its geometry, reorder it
 * and upload it.
 *   n_vertex, xy      vertex coordinates, xy[2*i], xy[2*i+1] (host)
 *   n_tri, tri        corners of each triangle, tri[3*t + c], counter-clockwise
 *                     (Sec. 4.1.2 "triangleVertices")
 *   image_shift       NULL, or per corner the periodic image (dx, dy) in
 *                     {-1,0,1} periods: the corner sits at
 *                     xy[v] + (dx*Lx, dy*Ly).  Periodic boundaries are
 *                     "handled by the mesh" (Sec. 3.5).
 *   Lx, Ly            periods used with image_shift
 *   reorder           RD_ORDER_NONE | RD_ORDER_MORTON | RD_ORDER_RCM
 *   cuda_stream       cudaStream_t for all device work of this mesh (NULL:
 *                     the library creates a non-blocking stream)
 * Geometry per triangle: inward normals n_i of the edge opposite corner i
 * with |n_i| = edge length, area |T|, longest edge l_max; nodal volume
 * V_i = sum |T|/3 (Sec. 3.2).  A vertex -> (triangle, corner) CSR replaces the
 * atomic accumulation of Sec. 4.2.1 by a deterministic gather.
 * Errors: RD_EINVAL for an index out of range, a shift outside {-1,0,1}, a
 * clockwise or zero-area triangle, or a vertex in no triangle.             */
int rd_mesh_create(int32_t n_vertex, const double *xy, int32_t n_tri, const int32_t *tri,
                   const int8_t *image_shift, double Lx, double Ly, int32_t reorder,
                   void *cuda_stream, rd_mesh **out);
void rd_mesh_destroy(rd_mesh *m);
/* Internal order chosen by the reorder: vertex_perm[new] = caller vertex,
 * tri_perm[new] = caller triangle (either pointer may be NULL). */
int rd_mesh_permutation(const rd_mesh *m, int32_t *vertex_perm, int32_t *tri_perm);
int rd_mesh_sizes(const rd_mesh *m, int32_t *n_vertex, int32_t *n_tri);

/* Boundary conditions of a mesh that is not periodic everywhere (Sec. 3.5).
 *   ghost   NULL, or [n_vertex] (caller order): 1 marks a ghost vertex whose
 *           state is held at its initial value -- the state given to
 *           rd_state_init / rd_state_set -- at the start of every step
 *           (non-reflecting or inflow boundaries); in a two-stage step its
 *           W* is the ordinary stage-1 update.
 *   wall    [n_wall][2] (caller triangle, corner): the edge opposite that
 *           corner is a reflecting wall, imposed weakly: with the wall's
 *           outward unit normal n and f = -(rho v_n, rho u v_n, rho v v_n,
 *           rho h v_n) at its two vertices a, b (v_n = v . n), the correction
 *           residuals Phi^c_a = |e|/2 (alpha f_a + (1 - alpha) f_b) and
 *           Phi^c_b = |e|/2 ((1 - alpha) f_a + alpha f_b) are added to the
 *           vertices' residuals: at W^n in the first stage (and in RD_N1),
 *           as (Phi^c(W^n) + Phi^c(W*)) / 2 in the second.
 *   alpha   the split, 0.75 in the paper.
 * Replaces any earlier boundary.  States created before the call return
 * RD_EINVAL from rd_step / rd_run until rd_state_set gives them a new
 * initial state.  Batched mode and the adjoint take periodic meshes only
 * (RD_ENOTSUP).  Errors: RD_EINVAL for a triangle or corner out of range, an
 * edge that another triangle shares (not on the boundary), an edge listed
 * twice, or alpha outside [0, 1].  The caller owns both arrays. */
int rd_mesh_set_boundary(rd_mesh *m, const uint8_t *ghost, int32_t n_wall, const int32_t *wall, double alpha);

/* ---- periodic Delaunay refinement mesh generator (Sec. 2.3, 2.4, 4.1) -----
 * rd_meshgen_run builds, on the device, a Delaunay triangulation of the
 * periodic rectangle [0, Lx) x [0, Ly) in which every triangle has
 * circumradius <= max_circumradius (size bound R) and circumradius over
 * shortest edge <= quality (bound B >= 1; sqrt 2 in Ruppert's algorithm).
 * It starts from an nx0 x ny0 grid (>= 3 each) with seeded jitter, restores
 * the Delaunay property by edge flips, and then repeats: test every triangle
 * (Sec. 2.4.1), locate the circumcentres of the bad ones by walking (Sec.
 * 2.4.2), select insertions with disjoint cavities by random-priority locks
 * (Sec. 4.1.1), split the containing triangles, and flip non-Delaunay edges
 * in parallel independent sets until none is left (Sec. 2.4.6, 4.1.4).
 * Predicates are exact: coordinates are integers on 2^30 units per period of
 * x (Ly is rounded to that unit; rd_meshgen_domain returns the periods used),
 * and Orient2D / InCircle2D are evaluated in 64/128-bit integers (exact while
 * coordinate differences stay below half a period, which holds with >= 3
 * initial cells per period).  Runs are deterministic for a given seed.
 * Bounds: max_vertices (capacity), max_rounds insertion rounds and
 * max_flip_rounds flip rounds per restoration; reaching a round bound returns
 * RD_ETIMEOUT, a full capacity RD_ENOMEM (the handle is still returned with
 * the mesh as far as it got).  Output (rd_meshgen_get, host arrays): xy
 * [nv][2], tri [nt][3] counter-clockwise, shift [nt][3][2] in {0, 1} periods --
 * the input format of rd_mesh_create -- and optionally the integer
 * coordinates xy_units [nv][2].  times: ms in quality test + location,
 * cavities, insertion, flips, and the whole run (CUDA events). */
typedef struct rd_meshgen rd_meshgen;
typedef struct {
  double Lx, Ly;
  double max_circumradius;
  double quality;
  int32_t nx0, ny0;
  int32_t max_vertices;
  int32_t max_rounds;
  int32_t max_flip_rounds;
  int32_t reserved;
  uint64_t seed;
} rd_meshgen_params;
int rd_meshgen_run(const rd_meshgen_params *p, void *cuda_stream, rd_meshgen **out);
int rd_meshgen_sizes(const rd_meshgen *g, int32_t *n_vertex, int32_t *n_tri, int32_t *rounds, int32_t *flips);
int rd_meshgen_times(const rd_meshgen *g, double ms[5]);
int rd_meshgen_get(const rd_meshgen *g, double *xy, int32_t *tri, int8_t *shift, int64_t *xy_units);
int rd_meshgen_domain(const rd_meshgen *g, double *Lx, double *Ly, int64_t *Px, int64_t *Py);
void rd_meshgen_destroy(rd_meshgen *g);

/* ---- solver state ---------------------------------------------------------
 * rd_state_init: allocate the device state of one mesh and upload W (host,
 * component-major, caller order).  Errors: RD_EINVAL (bad params),
 * RD_ENONPHYSICAL (rho<=0 or p<=0 or non-finite in W), RD_ENOMEM, RD_ECUDA. */
int rd_state_init(rd_mesh *m, const double *W, const rd_params *p, rd_state **out);
/* Replace the state by W (host, component-major, caller order); time and step
 * counters are kept.  A page-locked W (cudaHostAlloc / cudaHostRegister, e.g.
 * a pinned PyTorch tensor) is read in place by a kernel over the host link; a
 * pageable W is copied to a device staging buffer first.  Both give the same
 * state.  The call synchronises.  Errors: RD_ENONPHYSICAL (rho<=0, p<=0 or
 * non-finite in W), RD_EINVAL, RD_ECUDA. */
int rd_state_set(rd_state *s, const double *W);
/* One full time step (both stages for RD_B2 / RD_LDA2).  dt_out (nullable):
 * if non-NULL the call synchronises and returns the step's dt. */
int rd_step(rd_state *s, double *dt_out);
/* n_steps steps, replayed from a captured CUDA graph, dt and the stop test
 * kept on the device.  t_end > 0 clips the last dt so that t reaches t_end
 * exactly and stops there.  steps_done (nullable) receives the number of
 * steps completed; the call synchronises once at the end. */
int rd_run(rd_state *s, int32_t n_steps, double t_end, int32_t *steps_done);
/* Device -> host copy of the current state (component-major, caller order);
 * a page-locked W_out is written in place by a kernel, a pageable one through
 * a device staging buffer.  The call synchronises. */
int rd_get_state(const rd_state *s, double *W_out);
/* sum_i V_i W_i per component, accumulated in double in a fixed order. */
int rd_conserved_totals(const rd_state *s, double out[4]);
int rd_get_time(const rd_state *s, double *t, int64_t *steps);
/* dt of the last completed step. */
int rd_get_dt(const rd_state *s, double *dt);
void rd_state_destroy(rd_state *s);

/* ---- per-triangle residuals (inspection / parity) ---------------------------
 * Stage-1 shares of every triangle at the current state (Sec. 3.3):
 * out[(t*3 + c)*4 + k] for caller triangle t, corner c, component k.
 * which = 0: phi^N_i, 1: phi^LDA_i, 2: phi^B_i.  Also returns, if non-NULL,
 * cfl_term[t] = l_max^T lambda_max^T (Sec. 3.2). */
int rd_state_triangle_shares(rd_state *s, int32_t which, double *out, double *cfl_term);

/* ---- CFL time step of a caller-owned device state (Sec. 3.2) ---------------
 * dt = cfl * min_i 2 V_i / sum_{T containing i} l_max^T lambda_max^T with
 * lambda_max^T = max_{j in T} (|v_j| + c_j) evaluated at the vertex states.
 * Every array argument is a DEVICE pointer owned by the caller; element type
 * double (RD_FP64) or float (RD_FP32) for W, lmax, V:
 *   W        [4][n_vertex] conserved state, component-major
 *   tri      [3][n_tri] int32 corners, component-major: tri[c * n_tri + t]
 *   lmax     [n_tri] longest edge of each triangle
 *   V        [n_vertex] nodal volumes
 *   csr_ptr  [n_vertex + 1], csr_ent [3 n_tri]: the corners (3 t + c) of the
 *            triangles containing each vertex
 *   dt_out   one double, written on the stream
 * Scratch (one double per 256 vertices and a counter) comes from the installed
 * allocator and is released before return; the call waits for the stream.
 * Errors: RD_EINVAL, RD_ENOMEM, RD_ECUDA, RD_ENONPHYSICAL (rho <= 0 or p <= 0
 * at a vertex; dt_out is then not meaningful). */
int rd_cfl_dt(int32_t n_vertex, int32_t n_tri, int32_t precision, const void *W, const int32_t *tri,
              const void *lmax, const void *V, const int32_t *csr_ptr, const int32_t *csr_ent, double gamma,
              double cfl, double *dt_out, void *cuda_stream);

/* Allocation-free variant of rd_cfl_dt.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at the
 * moment they need a time step -- code whose device heap is owned by another
 * allocator (for example a caching allocator that has reserved the memory),
 * code that must not trigger cudaMalloc's implicit device synchronisation, or
 * latency-critical loops that may not allocate at all.  Same arguments, same
 * kernel and same result as rd_cfl_dt; it calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   - Scratch is a fixed array built into the library (512 KiB of block minima
 *     plus an 8-byte control word), held by every device that loads the
 *     library until the process exits.
 *   - Limit: n_vertex <= 16,777,216 (65536 blocks of 256 vertices); larger
 *     meshes are rejected with RD_EINVAL before any device work.
 *   - The first call on a device, with that device current, looks up the
 *     device address of the array (cudaGetSymbolAddress) and caches it.  With
 *     CUDA's lazy module loading (the default since CUDA 12.2) that lookup is
 *     also what loads the library's device code on that device, which
 *     allocates the array and may synchronise the device; it can fail with
 *     RD_ECUDA when another allocator has already reserved the free memory.
 *     So make one warm-up call per device at set-up, before any stream
 *     capture and before a caching allocator fills the device; "allocates
 *     nothing" and "no implicit synchronisation" hold from then on.  Call it
 *     with the device that holds the arrays current.
 *   - The cached address belongs to the device's primary context.  After a
 *     cudaDeviceReset in the calling process the address is stale: do not
 *     call this entry point on that device again in that process.
 *   - Every call shares the array, which keeps the last call's contents; the
 *     control word is cleared at the start of each call.  Calls whose device
 *     work overlaps (other streams, other host threads) race on the array and
 *     must be serialised by the caller.
 *   - Waits for the stream before returning, like rd_cfl_dt. */
int rd_cfl_dt_noalloc(int32_t n_vertex, int32_t n_tri, int32_t precision, const void *W, const int32_t *tri,
                      const void *lmax, const void *V, const int32_t *csr_ptr, const int32_t *csr_ent,
                      double gamma, double cfl, double *dt_out, void *cuda_stream);

/* ---- vertex-partitioned step (one part per GPU) ------------------------------
 * The step of Sec. 3.4 (Fig. of the paper's GPU data flow, Sec. 4.2) reads per
 * triangle the states of its three corners and gathers the shares per vertex.
 * Part r of P owns the contiguous internal vertex range
 * [r nv / P, (r + 1) nv / P) of the mesh store's Morton (or RCM) order and
 * computes every triangle with an owned corner (triangles on a part boundary
 * are computed by each part that touches them, from identical inputs); the
 * other corners of those triangles are its ghost vertices.  Per step the
 * caller moves the ghosts' W^n (before stage 1) and W* (before stage 2) from
 * their owners and replaces each part's CFL dt by the minimum over the parts;
 * the owned vertices then equal the single-part step bitwise.
 *
 * rd_partition_plan: the plan of part `part` of `n_parts` on the host only (no
 *   GPU needed), for the mesh given as to rd_mesh_create.  sizes[4] =
 *   {owned, ghosts, local triangles, send entries}; call once with the array
 *   pointers NULL to get the sizes, then with arrays of those sizes:
 *   local_vertices [owned + ghosts] caller vertex ids (owned first, ghosts in
 *   ascending internal order); local_triangles [local triangles] caller ids;
 *   local_corners [3][local triangles] local vertex ids; csr_ptr [owned + 1],
 *   csr_ent [..]: owned vertex -> local (triangle, corner) entries 3 k + c in
 *   the global CSR order; send_ptr [n_parts + 1], send_idx [send entries]:
 *   owned local vertices to send to each part, in that part's ghost order;
 *   recv_ptr [n_parts + 1]: the ghost slots [recv_ptr[q], recv_ptr[q+1])
 *   (counted from the first ghost) that part q owns.
 * rd_part_create: part `part` of `n_parts` of a state on mesh m (periodic
 *   meshes; RD_BX2, whose blend needs the global |v| range, and meshes with
 *   boundary conditions return RD_ENOTSUP), initialised from the full state W
 *   (host, caller order, component-major).  The plan is rd_partition_plan's.
 * rd_part_phase: one phase of a step on the mesh's stream, in this order:
 *   RD_PART_PACK_W (buf: device [send entries][4] of the state's word type,
 *   written), exchange, RD_PART_UNPACK_W (buf: device [ghosts][4], read),
 *   RD_PART_STAGE1, dt <- min over parts (rd_part_dt_device / rd_part_set_dt),
 *   RD_PART_UPDATE1 (N1: the step is complete), RD_PART_PACK_WS, exchange,
 *   RD_PART_UNPACK_WS, RD_PART_STAGE2.  buf is ignored by the other phases.
 * rd_part_dt_device: device address of this part's dt (one double), for an
 *   in-place all-reduce (min) between RD_PART_STAGE1 and RD_PART_UPDATE1.
 * rd_part_get_dt / rd_part_set_dt: the same through the host (synchronising).
 * rd_part_get_owned: W of the owned vertices, [4][owned] host, in the order
 *   of local_vertices.  rd_part_status: time, step count and status.       */
typedef struct rd_part rd_part;
#define RD_PART_PACK_W 0
#define RD_PART_UNPACK_W 1
#define RD_PART_STAGE1 2
#define RD_PART_UPDATE1 3
#define RD_PART_PACK_WS 4
#define RD_PART_UNPACK_WS 5
#define RD_PART_STAGE2 6
int rd_partition_plan(int32_t n_vertex, const double *xy, int32_t n_tri, const int32_t *tri,
                      const int8_t *image_shift, double Lx, double Ly, int32_t reorder, int32_t n_parts,
                      int32_t part, int32_t sizes[4], int32_t *local_vertices, int32_t *local_triangles,
                      int32_t *local_corners, int32_t *csr_ptr, int32_t *csr_ent, int32_t *send_ptr,
                      int32_t *send_idx, int32_t *recv_ptr);
int rd_part_create(rd_mesh *m, int32_t n_parts, int32_t part, const double *W, const rd_params *p, rd_part **out);
int rd_part_sizes(const rd_part *q, int32_t sizes[4]);
int rd_part_lists(const rd_part *q, int32_t *local_vertices, int32_t *send_ptr, int32_t *recv_ptr);
int rd_part_phase(rd_part *q, int32_t phase, void *buf);
int rd_part_dt_device(rd_part *q, void **dt);
int rd_part_get_dt(const rd_part *q, double *dt);
int rd_part_set_dt(rd_part *q, double dt);
int rd_part_get_owned(const rd_part *q, double *W_out);
int rd_part_status(const rd_part *q, double *t, int64_t *steps);
void rd_part_destroy(rd_part *q);

/* ---- discrete adjoint of a rollout ------------------------------------------
 * rd_adjoint_forward: advance s by n_steps ordinary steps (CFL dt), recording
 * every step's dt (dts_out, nullable, [n_steps] host) and keeping the state
 * on the device every ckpt_every steps (ceil(n_steps / ckpt_every) copies).
 * rd_adjoint_backward: given dL/dW at the end of that rollout (host,
 * component-major, caller order), return dL/dW at its start for the same
 * discrete map with the recorded dt sequence held fixed (dt's own dependence
 * on W is not differentiated).  Each checkpoint segment is re-run keeping W^n
 * of every step and, per triangle and stage, a mask of the branches the N / B
 * schemes took (regularised |lambda| of each node and eigenvalue, signs and
 * guards inside Theta); the segment is then reversed step by step with the
 * hand-written adjoint kernels (stage-2 triangle reverse, gather, stage-1
 * triangle reverse, gather -- the transposes of Sec. 3.4's updates), which
 * branch on those masks.  Device memory: ckpt_every + 1 state copies, two
 * masks per triangle and step of a segment, and per-corner adjoint records.
 * The state itself is left where rd_adjoint_forward put it.  The adjoint
 * covers RD_N1, RD_B2 and RD_LDA2 with global lumping; other parameter sets
 * return RD_ENOTSUP.
 * rd_run_fixed_dt: n_steps steps with the prescribed dt sequence (host,
 * [n_steps]) instead of the CFL dt, e.g. the recorded one, for finite
 * differences of the same map. */
int rd_adjoint_forward(rd_state *s, int32_t n_steps, int32_t ckpt_every, double *dts_out);
int rd_adjoint_backward(rd_state *s, const double *dL_dW_final, double *dL_dW0);
int rd_run_fixed_dt(rd_state *s, int32_t n_steps, const double *dts);
/* Branch masks of the next step of s (stage 1 at the current state, stage 2
 * at that step's W* with the CFL dt), one 64-bit word per caller triangle
 * (nullable outputs; mask2 is zero for RD_N1).  Bits: 0-8 regularised
 * |lambda| branch of node i, eigenvalue k at bit 3i+k; 9-17 lambda < 0;
 * 18-21 total residual < 0; 22-25 total residual == 0; 26-29 Theta's
 * denominator is sum_i |N_ik|; 30-33 denominator > 0; 34-45 N_ik < 0 at bit
 * 34+4i+k; 46-57 N_ik == 0.  The state does not advance. */
int rd_state_branch_masks(rd_state *s, uint64_t *mask1, uint64_t *mask2);

/* ---- measurement ------------------------------------------------------------
 * rd_state_profile: n_steps steps with CUDA events recorded on the mesh stream
 * around every kernel; ms_per_launch[6] receives the mean duration of
 * (stage-1 triangle, dt gather, stage-1 update, stage-2 triangle, final
 * update, commit) per step (zeros for kernels a scheme does not launch);
 * launches_per_step (nullable) the number of kernels one step launches.
 * The steps are real steps: the state advances. */
int rd_state_profile(rd_state *s, int32_t n_steps, double *ms_per_launch, int32_t *launches_per_step);
/* Floating-point operations of one triangle in the stage-1 (stage=1) or
 * stage-2 (stage=2) triangle kernel of a scheme, counted by running the
 * kernels' own per-triangle code on a counting scalar type (host only):
 * out = {add/sub, mul, div, sqrt}.  An FMA counts as one add and one mul. */
int rd_count_flops(int32_t scheme, int32_t stage, double out[4]);
/* FMA throughput of the current device (flop/s, 2 per FMA) measured with a
 * dependent-chain-free FMA kernel; precision RD_FP64 or RD_FP32. */
int rd_probe_fma_peak(int32_t precision, double *flops_per_s);

/* Element-wise evaluation of an arithmetic helper of the triangle kernels on
 * device arrays, for tests that hold it against CUDA's IEEE operations:
 *   RD_MATH_RCP  the double reciprocal the FP64 triangle kernels divide with
 *                (hardware approximation refined by two Newton-Raphson steps
 *                for |x| in [2^-1000, 2^1000); IEEE 1/x elsewhere).
 * x, out: n doubles in device memory (caller-owned); synchronises the stream.
 * Errors: RD_EINVAL (unknown fn, n < 0, NULL arrays), RD_ECUDA. */
#define RD_MATH_RCP 0
int rd_math_eval(int32_t fn, int64_t n, const double *x, double *out, void *cuda_stream);

/* Launch-shape autotuner of one state: times one uncommitted step (the
 * committed state is not changed) for triangle-kernel blocks of 64, 128, 192,
 * 256 threads and vertex-kernel blocks of 128, 256, 512 and keeps the
 * fastest; then, on meshes of at least 4096 triangles created with a
 * reordering, times the tiled step (rd_state_set_tiling) for a few tile sizes
 * and keeps the fastest if it beats the untiled step by 2 % (otherwise the
 * state is left untiled).  Returns the block choice (either pointer may
 * be NULL; the tiling is read with rd_state_get_tiling).  Results do not
 * depend on the launch shape (every sum has a fixed order). */
int rd_state_autotune(rd_state *s, int32_t *tri_block, int32_t *vtx_block);
/* Launch shapes a state uses (after rd_state_autotune): the stage-1 triangle
 * block size, the vertex block size and, for RD_DF64, the variant of the
 * stage-1 triangle kernel (rd_state_stage_shapes gives each stage's).  The
 * RD_DF64 variants: 2: 128 registers per thread; 3: 128 registers with a block
 * barrier between the phases of the per-triangle algebra, so that a block's
 * warps fetch the long straight-line code together; 4: 96 registers with the
 * barriers; 5: 80 registers with the barriers (fewer registers: more resident
 * warps, more spills).  The autotuner times every variant and triangle block
 * size and keeps the fastest for each stage.  Any pointer may be NULL. */
int rd_state_launch_shapes(const rd_state *s, int32_t *tri_block, int32_t *vtx_block, int32_t *df_variant);
/* Set the launch shapes by hand, the same for both stages: tri_block in {64,
 * 128, 192, 256}, vtx_block in {128, 256, 512}, df_variant in {2, 3, 4, 5}
 * (ignored unless RD_DF64); RD_EINVAL otherwise.  Results do not depend on them. */
int rd_state_set_launch_shapes(rd_state *s, int32_t tri_block, int32_t vtx_block, int32_t df_variant);
/* Triangle block size and RD_DF64 kernel variant of one stage (1 or 2) of the
 * two-stage step: read (pointers may be NULL) and set (same ranges as above;
 * RD_EINVAL otherwise).  Results do not depend on them. */
int rd_state_stage_shapes(const rd_state *s, int32_t stage, int32_t *tri_block, int32_t *df_variant);
int rd_state_set_stage_shapes(rd_state *s, int32_t stage, int32_t tri_block, int32_t df_variant);

/* Tiled step (Sec. 3.3-3.4 and Eqs. eqRK1/eqRK2 computed as in rd_step; the
 * distribution of Sec. 4.2.1 done on chip).  The triangles, in the mesh
 * store's order (sorted by smallest internal vertex id), are cut into tiles of
 * tile_triangles consecutive triangles, each processed by one thread block of
 * `threads` threads.  The block keeps its triangles' corner shares in shared
 * memory and sums them for every vertex whose triangles all lie in the tile;
 * only the shares of the other (boundary) vertices go through device memory.
 * Stage 2 and the final update are fused the same way for the two-stage
 * schemes except RD_BX2 and on meshes without walls or ghost vertices (those
 * keep the per-triangle stage 2).  Every sum keeps the CSR order, so states
 * are bitwise identical to the untiled step's.
 *   tile_triangles: 0 (untiled, the default) or a multiple of 32 in
 *                   [32, 4096]; threads: a multiple of 32 in [32, 256].
 * Errors: RD_EINVAL for values out of range; RD_ENOTSUP when the mesh was
 * created with RD_ORDER_NONE (its triangles are not sorted), a tile would
 * touch more than 65535 vertices, or its shared memory exceeds the device's
 * per-block limit.  The host builds the tile plan (O(n_tri log) work) and
 * uploads it; the state's captured graph is rebuilt on the next rd_run. */
int rd_state_set_tiling(rd_state *s, int32_t tile_triangles, int32_t threads);
/* rd_state_set_tiling with flags: RD_TILE_STAGE_GEOMETRY copies each tile's
 * geometry (normals, half edge lengths, areas, l_max, corner slots, boundary
 * masks) into shared memory with the vertex states, before the triangle loop,
 * so that the loop reads no device memory.  Results are bitwise the same. */
#define RD_TILE_STAGE_GEOMETRY 1
int rd_state_set_tiling_ex(rd_state *s, int32_t tile_triangles, int32_t threads, int32_t flags);
/* Current tiling (0, 0, 0 when untiled) and the number of boundary vertices;
 * any pointer may be NULL. */
int rd_state_get_tiling(const rd_state *s, int32_t *tile_triangles, int32_t *threads,
                        int32_t *n_boundary_vertices);
/* Flags of the current tiling (0 when untiled). */
int rd_state_get_tiling_flags(const rd_state *s, int32_t *flags);

/* ---- batched form: many independent meshes, one graph launch -------------
 * rd_batch_create: n_mesh (1..65535) meshes created on the same stream, with
 * their own initial states W0[m] (host, component-major, caller order of mesh
 * m).  The meshes are concatenated into one vertex and one triangle range;
 * every kernel of a step runs once over the whole batch, and each mesh keeps
 * its own CFL dt (Sec. 3.2), time and step count.  The meshes must outlive
 * the batch.  Errors as rd_state_init. */
int rd_batch_create(int32_t n_mesh, rd_mesh *const *meshes, const double *const *W0,
                    const rd_params *p, rd_batch **out);
/* n_steps steps of every mesh replayed as ONE CUDA-graph launch (the graph is
 * captured on the first call for a given n_steps and reused). */
int rd_batch_run(rd_batch *b, int32_t n_steps);
/* State of mesh `mesh` (host, component-major, caller order of that mesh). */
int rd_batch_get_state(const rd_batch *b, int32_t mesh, double *W_out);
/* dt of each mesh in the most recently computed step ([n_mesh]). */
int rd_batch_get_dt(const rd_batch *b, double *dt_out);
/* Simulation time and step count of each mesh ([n_mesh] each, nullable). */
int rd_batch_get_time(const rd_batch *b, double *t_out, int64_t *steps_out);
int rd_batch_sizes(const rd_batch *b, int64_t *n_vertex, int64_t *n_tri);
/* Launch-shape autotuner of a batch (as rd_state_autotune: triangle block and
 * RD_DF64 kernel variant per stage, then the vertex block; tri_block returns
 * stage 1's). */
int rd_batch_autotune(rd_batch *b, int32_t *tri_block, int32_t *vtx_block);
/* As rd_state_profile, for a batch (the steps advance the batch). */
int rd_batch_profile(rd_batch *b, int32_t n_steps, double *ms_per_launch);
void rd_batch_destroy(rd_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* RD_H */
