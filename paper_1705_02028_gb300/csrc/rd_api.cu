// rd_api.cu -- C ABI of the GB300 residual-distribution solver (see include/rd.h).
//
// Device memory comes from the installed allocator hook (default cudaMalloc);
// all work of a mesh and its states is ordered on the mesh's stream.  A step
// never synchronises with the host: dt, the simulation time, the step counter
// and a sticky status word live in a device control block (DevCtl).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "rd_df64.h"
#include "rd_device.h"
#include "rd_internal.h"
#include "rd_kernels.cuh"
#include "rd_tiled.h"

using namespace rd;

// ---------------------------------------------------------------------------
// allocator hook
// ---------------------------------------------------------------------------
static rd_alloc_fn g_alloc = nullptr;
static rd_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

extern "C" int rd_set_allocator(rd_alloc_fn alloc, rd_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return RD_EINVAL;
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return RD_OK;
}

namespace rd {

int dev_alloc(DevBuf& b, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (g_alloc) {
    b.p = g_alloc(bytes, (void*)s, g_alloc_ctx);
    if (!b.p) return RD_ENOMEM;
    b.fr = g_free;
    b.ctx = g_alloc_ctx;
    return RD_OK;
  }
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return RD_ENOMEM;
  }
  b.fr = nullptr;
  return RD_OK;
}

void dev_free(DevBuf& b) {
  if (!b.p) return;
  if (b.fr) b.fr(b.p, b.ctx);
  else cudaFree(b.p);
  b.p = nullptr;
}

}  // namespace rd

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
namespace rd {

template <class T>
int upload_vec(DevBuf& b, const std::vector<double>& src, cudaStream_t s) {
  std::vector<T> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = (T)src[i];
  CK(dev_alloc(b, tmp.size() * sizeof(T), s));
  CU(cudaMemcpyAsync(b.p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  CU(cudaStreamSynchronize(s));
  return RD_OK;
}

template <class T>
int mesh_geometry(rd_mesh* m) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  if (m->geo_ready[pi]) return RD_OK;
  const std::vector<double>* src[6] = {&m->h.nx, &m->h.ny, &m->h.hl, &m->h.area, &m->h.lmax, &m->h.V};
  for (int k = 0; k < 6; ++k) CK(upload_vec<T>(m->geo[pi][k], *src[k], m->stream));
  m->geo_ready[pi] = true;
  return RD_OK;
}

template <class T>
DevGeo<T> geo_of(const rd_mesh* m) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  DevGeo<T> g;
  g.nx = (const T*)m->geo[pi][0].p;
  g.ny = (const T*)m->geo[pi][1].p;
  g.hl = (const T*)m->geo[pi][2].p;
  g.area = (const T*)m->geo[pi][3].p;
  g.lmax = (const T*)m->geo[pi][4].p;
  return g;
}

}  // namespace rd

extern "C" int rd_mesh_create(int32_t n_vertex, const double* xy, int32_t n_tri, const int32_t* tri,
                              const int8_t* image_shift, double Lx, double Ly, int32_t reorder,
                              void* cuda_stream, rd_mesh** out) {
  if (!out) return RD_EINVAL;
  *out = nullptr;
  rd_mesh* m = new (std::nothrow) rd_mesh();
  if (!m) return RD_ENOMEM;
  int st = build_host_mesh(n_vertex, xy, n_tri, tri, image_shift, Lx, Ly, reorder, m->h);
  if (st != RD_OK) {
    delete m;
    return st;
  }
  if (cuda_stream) {
    m->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete m;
      return RD_ECUDA;
    }
    m->own_stream = true;
  }
  auto up_int = [&](DevBuf& b, const std::vector<int32_t>& v) -> int {
    CK(dev_alloc(b, v.size() * sizeof(int32_t), m->stream));
    CU(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, m->stream));
    return RD_OK;
  };
  st = up_int(m->tri, m->h.tri);
  if (st == RD_OK) st = up_int(m->ptr, m->h.csr_ptr);
  if (st == RD_OK) st = up_int(m->ent, m->h.csr_ent);
  if (st == RD_OK) st = up_int(m->vperm, m->h.vperm);
  if (st == RD_OK) st = up_int(m->vinv, m->h.vinv);
  if (st == RD_OK && cudaStreamSynchronize(m->stream) != cudaSuccess) {
    cudaGetLastError();
    st = RD_ECUDA;
  }
  if (st != RD_OK) {
    rd_mesh_destroy(m);
    return st;
  }
  *out = m;
  return RD_OK;
}

extern "C" void rd_mesh_destroy(rd_mesh* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  dev_free(m->tri);
  dev_free(m->ptr);
  dev_free(m->ent);
  dev_free(m->vperm);
  dev_free(m->vinv);
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < 6; ++k) dev_free(m->geo[p][k]);
  for (int k = 0; k < 4; ++k) dev_free(m->geo_df[k]);
  mesh_boundary_free(m);
  if (m->own_stream) cudaStreamDestroy(m->stream);
  delete m;
}

extern "C" int rd_mesh_permutation(const rd_mesh* m, int32_t* vertex_perm, int32_t* tri_perm) {
  if (!m) return RD_EINVAL;
  if (vertex_perm) std::memcpy(vertex_perm, m->h.vperm.data(), sizeof(int32_t) * m->h.nv);
  if (tri_perm) std::memcpy(tri_perm, m->h.tperm.data(), sizeof(int32_t) * m->h.nt);
  return RD_OK;
}

extern "C" int rd_mesh_sizes(const rd_mesh* m, int32_t* n_vertex, int32_t* n_tri) {
  if (!m) return RD_EINVAL;
  if (n_vertex) *n_vertex = m->h.nv;
  if (n_tri) *n_tri = m->h.nt;
  return RD_OK;
}

// ---------------------------------------------------------------------------
// state (struct rd_state is defined in rd_device.h)
// ---------------------------------------------------------------------------

namespace {

bool valid_params(const rd_params* p) {
  if (!p) return false;
  if (p->scheme < RD_N1 || p->scheme > RD_BX2) return false;
  if (p->lumping != RD_LUMP_GLOBAL && p->lumping != RD_LUMP_SELECTIVE) return false;
  if (p->lumping == RD_LUMP_SELECTIVE && p->scheme == RD_N1) return false;
  if (p->reserved != 0) return false;
  if (p->precision != RD_FP64 && p->precision != RD_FP32 && p->precision != RD_DF64) return false;
  if (!(p->cfl > 0.0) || !(p->gamma > 1.0) || !(p->eps_fix >= 0.0)) return false;
  if (!std::isfinite(p->cfl) || !std::isfinite(p->gamma) || !std::isfinite(p->eps_fix)) return false;
  return true;
}

__global__ void k_begin(DevCtl* ctl, double t_end) {
  if (ctl->status == 0) ctl->stop = 0;
  ctl->t_end = t_end;
}

}  // namespace

template <class T>
void rd::launch_gather_cfl(int vblock, cudaStream_t st, int nv, const int* ptr, const int* ent, const T* share,
                           const T* cfl, const T* V, T* R1, T* partial, T cflnum, DevCtl* ctl) {
  switch (vblock) {
    case 128:
      k_gather_cfl<T, 128><<<nblk(nv, 128), 128, 0, st>>>(nv, ptr, ent, share, cfl, V, R1, partial, cflnum, ctl);
      break;
    case 512:
      k_gather_cfl<T, 512><<<nblk(nv, 512), 512, 0, st>>>(nv, ptr, ent, share, cfl, V, R1, partial, cflnum, ctl);
      break;
    default:
      k_gather_cfl<T, 256><<<nblk(nv, 256), 256, 0, st>>>(nv, ptr, ent, share, cfl, V, R1, partial, cflnum, ctl);
      break;
  }
}
template void rd::launch_gather_cfl<double>(int, cudaStream_t, int, const int*, const int*, const double*,
                                            const double*, const double*, double*, double*, double, DevCtl*);
template void rd::launch_gather_cfl<float>(int, cudaStream_t, int, const int*, const int*, const float*,
                                           const float*, const float*, float*, float*, float, DevCtl*);

namespace {

// Launches one step reading buffer a and writing buffer 1-a.  ev (nullable):
// seven events recorded before each kernel and after the last one.
__global__ void k_fix_dt(DevCtl* ctl, double dt) {
  if (!ctl->stop) ctl->dt = dt;
}

template <class T>
BlendArgs<T> blend_args(const rd_state* s) {
  return tile_blend_args<T>(s);
}

template <class T>
int launch_step(rd_state* s, int a, cudaEvent_t* ev = nullptr, bool commit = true, double fixed_dt = 0.0) {
  rd_mesh* m = s->m;
  const int nt = m->h.nt, nv = m->h.nv, b = 1 - a;
  cudaStream_t st = m->stream;
  DevGeo<T> g = geo_of<T>(m);
  const T* V = (const T*)m->geo[s->pi][5].p;
  const int* tri = (const int*)m->tri.p;
  const int* ptr = (const int*)m->ptr.p;
  const int* ent = (const int*)m->ent.p;
  DevCtl* ctl = (DevCtl*)s->ctl.p;
  T gamma = (T)s->p.gamma, eps = (T)s->p.eps_fix, cfl = (T)s->p.cfl;
  T* share = (T*)s->share.p;
  T* rec = (T*)s->rec.p;
  T* cf = (T*)s->cfl.p;
  const int TB = s->tri_block, TB2 = s->tri_block2, VB = s->vtx_block;
  unsigned gt = nblk(nt, TB), gt2 = nblk(nt, TB2), gv = nblk(nv, VB);
  const T* Za = (const T*)s->Z[a].p;
  const T* Sa = (const T*)s->spd[a].p;
  auto mark = [&](int k) {
    if (ev) cudaEventRecord(ev[k], st);
  };
  BlendArgs<T> ba1 = blend_args<T>(s), ba2 = ba1;
  WallArgs<T> wa1, wa2;  // stage 1 / N1 at the pass's state; stage 2 half at W*, half at W^n
  GhostArgs<T> ga;       // the final update of the step resets ghost vertices
  if (m->n_wall > 0) {
    wa1.ptr = (const int*)m->wptr.p;
    wa1.other = (const int*)m->wother.p;
    wa1.geo = (const T*)m->wgeo[s->pi].p;
    wa1.alpha = (T)m->wall_alpha;
    wa2 = wa1;
    wa2.Wn = (const T*)s->W[a].p;
  }
  if (m->n_ghost > 0) {
    ga.of = (const int*)m->ghost_of.p;
    ga.W = (const T*)s->ghostW.p;
  }
  unsigned long long* vr0 = (unsigned long long*)s->vr.p;          // |v| range of W^n
  unsigned long long* vr1 = vr0 ? vr0 + 2 : nullptr;              // |v| range of W*
  ba1.vr = vr0;
  ba2.vr = vr1;
  mark(0);
  const bool tiled = s->tiles != nullptr;
  const bool df = sizeof(T) == 8 && s->p.precision == RD_DF64;
  if (tiled) {
    CK(tiled_stage1<T>(s, a, ev));
  } else {
  if (df) {
    CK(launch_tri_stage1_df(s, a, gt, TB, st));
  } else
  switch (s->p.scheme) {
    case RD_N1:
      k_tri_stage1<T, RD_N1><<<gt, TB, 0, st>>>(nt, nv, tri, g, Za, Sa, Gas<T>::of(gamma), eps, share, nullptr, cf, ctl);
      break;
    case RD_LDA2:
      k_tri_stage1<T, RD_LDA2><<<gt, TB, 0, st>>>(nt, nv, tri, g, Za, Sa, Gas<T>::of(gamma), eps, share, rec, cf, ctl);
      break;
    default:  // RD_B2, RD_BMAX2, RD_BMIN2, RD_BX2
      if (s->p.scheme == RD_B2 && s->p.lumping == RD_LUMP_GLOBAL)
        k_tri_stage1<T, RD_B2><<<gt, TB, 0, st>>>(nt, nv, tri, g, Za, Sa, Gas<T>::of(gamma), eps, share, rec, cf,
                                                  ctl);
      else  // generic blend instantiation: Bmax, Bmin, Bx, B with selective lumping
        k_tri_stage1<T, RD_BMAX2><<<gt, TB, 0, st>>>(nt, nv, tri, g, Za, Sa, Gas<T>::of(gamma), eps, share, rec, cf,
                                                     ctl, ba1);
      break;
  }
  mark(1);
  launch_gather_cfl<T>(VB, st, nv, ptr, ent, share, cf, V, (T*)s->R1.p, (T*)s->partial.p, cfl, ctl);
  }
  if (fixed_dt > 0.0) k_fix_dt<<<1, 1, 0, st>>>(ctl, fixed_dt);
  mark(2);
  if (s->p.scheme == RD_N1) {
    k_update<T><<<gv, VB, 0, st>>>(nv, (const T*)s->W[a].p, (const T*)s->R1.p, ptr, ent, nullptr, V, gamma,
                                          (T*)s->W[b].p, (T*)s->Z[b].p, (T*)s->spd[b].p, ctl, nullptr, nullptr,
                                          nullptr, wa1, ga);
    mark(3);
    mark(4);
    mark(5);
  } else if (tiled && tiled_stage2_applies(s)) {
    mark(3);
    CK(tiled_stage2<T>(s, a, ev));
    mark(5);
  } else {
    if (vr1) k_vr_reset<<<1, 1, 0, st>>>(vr1, ctl, 0);
    k_update<T><<<gv, VB, 0, st>>>(nv, (const T*)s->W[a].p, (const T*)s->R1.p, ptr, ent, nullptr, V, gamma,
                                          (T*)s->Ws.p, (T*)s->Zs.p, nullptr, ctl, nullptr, nullptr, vr1, wa1,
                                          GhostArgs<T>(), df ? (float2*)s->dWdf.p : nullptr);
    mark(3);
    if (df)
      CK(launch_tri_stage2_df(s, a, gt2, TB2, st));
    else if (s->p.scheme == RD_LDA2)
      k_tri_stage2<T, RD_LDA2><<<gt2, TB2, 0, st>>>(nt, nv, tri, g, (const T*)s->Zs.p, (const T*)s->W[a].p,
                                                  (const T*)s->Ws.p, rec, Gas<T>::of(gamma), eps, share, ctl,
                                                  nullptr, nullptr, ba2);
    else if (s->p.scheme == RD_B2 && s->p.lumping == RD_LUMP_GLOBAL)
      k_tri_stage2<T, RD_B2><<<gt2, TB2, 0, st>>>(nt, nv, tri, g, (const T*)s->Zs.p, (const T*)s->W[a].p,
                                                (const T*)s->Ws.p, rec, Gas<T>::of(gamma), eps, share, ctl);
    else
      k_tri_stage2<T, RD_BMAX2><<<gt2, TB2, 0, st>>>(nt, nv, tri, g, (const T*)s->Zs.p, (const T*)s->W[a].p,
                                                   (const T*)s->Ws.p, rec, Gas<T>::of(gamma), eps, share, ctl,
                                                   nullptr, nullptr, ba2);
    mark(4);
    if (vr0) k_vr_reset<<<1, 1, 0, st>>>(vr0, ctl, 0);
    k_update<T><<<gv, VB, 0, st>>>(nv, (const T*)s->Ws.p, nullptr, ptr, ent, share, V, gamma,
                                          (T*)s->W[b].p, (T*)s->Z[b].p, (T*)s->spd[b].p, ctl, nullptr, nullptr, vr0,
                                          wa2, ga);
    mark(5);
  }
  if (commit) k_commit<<<1, 1, 0, st>>>(ctl);
  mark(6);
  CU(cudaGetLastError());
  return RD_OK;
}

// Kernel launches of one committed step as launch_step issues them.
int step_launches(const rd_state* s) {
  const bool bx = s->p.scheme == RD_BX2;
  int n = 2 + 1;  // stage 1 + gather (tiled: tile kernel + boundary gather), commit
  if (s->p.scheme == RD_N1) return n + 1;
  if (s->tiles && tiled_stage2_applies(s)) return n + 1 + (s->tiles->n_bvert > 0 ? 1 : 0);
  return n + 3 + (bx ? 2 : 0);  // update1, stage 2, update2 (+ the two |v| range resets of Bx)
}

int launch_step_any(rd_state* s, int a, cudaEvent_t* ev = nullptr, bool commit = true, double fixed_dt = 0.0) {
  if (s->bc_version != s->m->bc_version) return RD_EINVAL;  // boundary changed: rd_state_set first
  return s->pi == 0 ? launch_step<double>(s, a, ev, commit, fixed_dt) : launch_step<float>(s, a, ev, commit, fixed_dt);
}

int read_ctl(const rd_state* s, DevCtl& c) {
  CU(cudaMemcpyAsync(&c, s->ctl.p, sizeof(DevCtl), cudaMemcpyDeviceToHost, s->m->stream));
  CU(cudaStreamSynchronize(s->m->stream));
  return RD_OK;
}

int status_to_rd(int st) { return st ? RD_ENONPHYSICAL : RD_OK; }

// Host (caller order, double) -> device staging -> internal order in T, then Z and |v|+c.
// Device address of a caller's host array when it is page-locked and mapped
// into the device's address space (cudaHostAlloc / cudaHostRegister memory, as
// PyTorch's pinned tensors are), so that the state kernels can read or write it
// in place over the host link instead of through a staging copy; NULL for
// pageable memory, which takes the staging copy.
static const double* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return (const double*)a.devicePointer;
}

template <class T>
int upload_state(rd_state* s, const double* W, int buf) {
  rd_mesh* m = s->m;
  const int nv = m->h.nv;
  cudaStream_t st = m->stream;
  DevCtl* ctl = (DevCtl*)s->ctl.p;
  if (const double* Wd = mapped_host(W)) {  // page-locked caller array: read it in place
    k_host_in<T><<<nblk(nv, VTX_BLOCK), VTX_BLOCK, 0, st>>>(nv, (const int*)m->vinv.p, Wd, (T*)s->W[buf].p, ctl);
  } else {
    CU(cudaMemcpyAsync(s->stage.p, W, 4 * (size_t)nv * sizeof(double), cudaMemcpyHostToDevice, st));
    k_permute_in<T><<<nblk(nv, VTX_BLOCK), VTX_BLOCK, 0, st>>>(nv, (const int*)m->vperm.p,
                                                               (const double*)s->stage.p, (T*)s->W[buf].p, ctl);
  }
  // boundary data for this state: wall geometry in T and the ghosts' initial state
  if (!s->bc_init || s->bc_version != m->bc_version) {
    CK(mesh_wall_geometry<T>(m));
    dev_free(s->ghostW);
    if (m->n_ghost > 0) CK(dev_alloc(s->ghostW, 4 * (size_t)m->n_ghost * sizeof(T), st));
    if (s->g2) {  // the captured steps hold the old boundary arrays
      cudaGraphExecDestroy(s->g2);
      s->g2 = nullptr;
    }
    s->bc_version = m->bc_version;
    s->bc_init = true;
  }
  if (m->n_ghost > 0)
    k_ghost_capture<T><<<nblk(m->n_ghost, VTX_BLOCK), VTX_BLOCK, 0, st>>>(m->n_ghost, (const int*)m->ghost_ids.p,
                                                                         (const T*)s->W[buf].p, (T*)s->ghostW.p);
  unsigned long long* vr0 = (unsigned long long*)s->vr.p;
  if (vr0) k_vr_reset<<<1, 1, 0, st>>>(vr0, ctl, 1);
  k_prepare<T><<<nblk(nv, VTX_BLOCK), VTX_BLOCK, 0, st>>>(nv, (const T*)s->W[buf].p, (T)s->p.gamma,
                                                          (T*)s->Z[buf].p, (T*)s->spd[buf].p, ctl, vr0);
  CU(cudaGetLastError());
  DevCtl c;
  CK(read_ctl(s, c));
  return status_to_rd(c.status);
}

// Device internal order in T -> staging (caller order, double) -> host.
template <class T>
int download_state(const rd_state* s, int buf, double* W_out) {
  rd_mesh* m = s->m;
  const int nv = m->h.nv;
  cudaStream_t st = m->stream;
  if (double* Wd = const_cast<double*>(mapped_host(W_out))) {  // page-locked caller array: write it in place
    k_host_out<T><<<nblk(nv, VTX_BLOCK), VTX_BLOCK, 0, st>>>(nv, (const int*)m->vinv.p, (const T*)s->W[buf].p, Wd);
    CU(cudaGetLastError());
  } else {
    k_permute_out<T><<<nblk(nv, VTX_BLOCK), VTX_BLOCK, 0, st>>>(nv, (const int*)m->vperm.p, (const T*)s->W[buf].p,
                                                                (double*)s->stage.p);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(W_out, s->stage.p, 4 * (size_t)nv * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CU(cudaStreamSynchronize(st));
  return RD_OK;
}

int alloc_state(rd_state* s) {
  rd_mesh* m = s->m;
  const size_t nv = m->h.nv, nt = m->h.nt, ts = s->ts;
  cudaStream_t st = m->stream;
  for (int b = 0; b < 2; ++b) {
    CK(dev_alloc(s->W[b], 4 * nv * ts, st));
    CK(dev_alloc(s->Z[b], 4 * nv * ts, st));
    CK(dev_alloc(s->spd[b], nv * ts, st));
  }
  CK(dev_alloc(s->R1, 4 * nv * ts, st));
  CK(dev_alloc(s->share, 12 * nt * ts, st));
  CK(dev_alloc(s->cfl, nt * ts, st));
  CK(dev_alloc(s->partial, (size_t)nblk(nv, VTX_BLOCK_MIN) * ts, st));
  CK(dev_alloc(s->ctl, sizeof(DevCtl), st));
  CK(dev_alloc(s->cons_partial, (size_t)nblk(nv, VTX_BLOCK) * 4 * sizeof(double), st));
  CK(dev_alloc(s->cons_out, 4 * sizeof(double), st));
  CK(dev_alloc(s->stage, 4 * nv * sizeof(double), st));
  if (s->p.scheme == RD_BX2) CK(dev_alloc(s->vr, 4 * sizeof(unsigned long long), st));
  if (s->p.scheme != RD_N1) {
    CK(dev_alloc(s->Ws, 4 * nv * ts, st));
    CK(dev_alloc(s->Zs, 4 * nv * ts, st));
    CK(dev_alloc(s->rec, 16 * nt * ts, st));
    if (s->p.precision == RD_DF64) CK(dev_alloc(s->dWdf, 4 * nv * 2 * sizeof(float), st));
  }
  DevCtl c{};
  CU(cudaMemcpyAsync(s->ctl.p, &c, sizeof(DevCtl), cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));
  return RD_OK;
}

int build_graph(rd_state* s) {
  if (s->g2 || s->graph_failed) return RD_OK;
  cudaStream_t st = s->m->stream;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    s->graph_failed = true;
    return RD_OK;
  }
  int r0 = launch_step_any(s, 0);
  int r1 = r0 == RD_OK ? launch_step_any(s, 1) : r0;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (r1 != RD_OK || e != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    s->graph_failed = true;
    return RD_OK;
  }
  if (cudaGraphInstantiate(&s->g2, g, 0) != cudaSuccess) {
    cudaGetLastError();
    s->g2 = nullptr;
    s->graph_failed = true;
  }
  cudaGraphDestroy(g);
  return RD_OK;
}

}  // namespace

// Helpers shared with the adjoint translation unit.
int rd::state_step(rd_state* s, int a, double fixed_dt) {
  k_begin<<<1, 1, 0, s->m->stream>>>((DevCtl*)s->ctl.p, 0.0);
  return launch_step_any(s, a, nullptr, true, fixed_dt);
}
int rd::state_read_ctl(const rd_state* s, DevCtl& c) { return read_ctl(s, c); }

extern "C" int rd_run_fixed_dt(rd_state* s, int32_t n_steps, const double* dts) {
  if (!s || n_steps < 0 || (n_steps > 0 && !dts)) return RD_EINVAL;
  for (int32_t k = 0; k < n_steps; ++k)
    if (!(dts[k] > 0.0) || !std::isfinite(dts[k])) return RD_EINVAL;
  DevCtl c0;
  CK(read_ctl(s, c0));
  s->launched = c0.steps;
  if (c0.status) return RD_ENONPHYSICAL;
  k_begin<<<1, 1, 0, s->m->stream>>>((DevCtl*)s->ctl.p, 0.0);
  for (int32_t k = 0; k < n_steps; ++k) {
    CK(launch_step_any(s, (int)(s->launched & 1), nullptr, true, dts[k]));
    s->launched++;
  }
  DevCtl c;
  CK(read_ctl(s, c));
  s->launched = c.steps;
  return status_to_rd(c.status);
}

extern "C" int rd_state_init(rd_mesh* m, const double* W, const rd_params* p, rd_state** out) {
  if (!m || !W || !out || !valid_params(p)) return RD_EINVAL;
  *out = nullptr;
  rd_state* s = new (std::nothrow) rd_state();
  if (!s) return RD_ENOMEM;
  s->m = m;
  s->p = *p;
  s->pi = p->precision == RD_FP32 ? 1 : 0;  // RD_DF64 keeps the FP64 state
  s->ts = s->pi == 0 ? sizeof(double) : sizeof(float);
  int st = s->pi == 0 ? mesh_geometry<double>(m) : mesh_geometry<float>(m);
  if (st == RD_OK && p->precision == RD_DF64) st = mesh_geometry_df(m);
  if (st == RD_OK) st = alloc_state(s);
  if (st == RD_OK) st = s->pi == 0 ? upload_state<double>(s, W, 0) : upload_state<float>(s, W, 0);
  if (st != RD_OK) {
    rd_state_destroy(s);
    return st;
  }
  *out = s;
  return RD_OK;
}

extern "C" int rd_state_set(rd_state* s, const double* W) {
  if (!s || !W) return RD_EINVAL;
  DevCtl c;
  CK(read_ctl(s, c));
  if (c.status) return RD_ENONPHYSICAL;
  int buf = (int)(c.steps & 1);
  s->launched = c.steps;
  return s->pi == 0 ? upload_state<double>(s, W, buf) : upload_state<float>(s, W, buf);
}

extern "C" int rd_step(rd_state* s, double* dt_out) {
  if (!s) return RD_EINVAL;
  cudaStream_t st = s->m->stream;
  k_begin<<<1, 1, 0, st>>>((DevCtl*)s->ctl.p, 0.0);
  CK(launch_step_any(s, (int)(s->launched & 1)));
  s->launched++;
  if (dt_out) {
    DevCtl c;
    CK(read_ctl(s, c));
    s->launched = c.steps;
    *dt_out = c.dt;
    if (c.status) return RD_ENONPHYSICAL;
  }
  return RD_OK;
}

extern "C" int rd_run(rd_state* s, int32_t n_steps, double t_end, int32_t* steps_done) {
  if (!s || n_steps < 0) return RD_EINVAL;
  if (s->bc_version != s->m->bc_version) return RD_EINVAL;
  cudaStream_t st = s->m->stream;
  DevCtl c0;
  CK(read_ctl(s, c0));
  s->launched = c0.steps;
  if (c0.status) {
    if (steps_done) *steps_done = 0;
    return RD_ENONPHYSICAL;
  }
  k_begin<<<1, 1, 0, st>>>((DevCtl*)s->ctl.p, t_end > 0.0 ? t_end : 0.0);
  CU(cudaGetLastError());
  int32_t left = n_steps;
  if (left > 0 && (s->launched & 1)) {
    CK(launch_step_any(s, 1));
    s->launched++;
    left--;
  }
  if (left >= 2) CK(build_graph(s));
  while (left >= 2 && s->g2) {
    CU(cudaGraphLaunch(s->g2, st));
    s->launched += 2;
    left -= 2;
  }
  while (left > 0) {
    CK(launch_step_any(s, (int)(s->launched & 1)));
    s->launched++;
    left--;
  }
  DevCtl c;
  CK(read_ctl(s, c));
  s->launched = c.steps;
  if (steps_done) *steps_done = (int32_t)(c.steps - c0.steps);
  return status_to_rd(c.status);
}

extern "C" int rd_state_profile(rd_state* s, int32_t n_steps, double* ms_per_launch, int32_t* launches_per_step) {
  if (!s || n_steps <= 0 || !ms_per_launch) return RD_EINVAL;
  cudaStream_t st = s->m->stream;
  DevCtl c0;
  CK(read_ctl(s, c0));
  s->launched = c0.steps;
  if (c0.status) return RD_ENONPHYSICAL;
  k_begin<<<1, 1, 0, st>>>((DevCtl*)s->ctl.p, 0.0);
  std::vector<cudaEvent_t> ev(7 * (size_t)n_steps, nullptr);
  int rc = RD_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = RD_ECUDA;
  for (int32_t k = 0; k < n_steps && rc == RD_OK; ++k) {
    rc = launch_step_any(s, (int)(s->launched & 1), ev.data() + 7 * (size_t)k);
    s->launched++;
  }
  if (rc == RD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = RD_ECUDA;
  for (int j = 0; j < 6; ++j) ms_per_launch[j] = 0.0;
  for (int32_t k = 0; k < n_steps && rc == RD_OK; ++k)
    for (int j = 0; j < 6; ++j) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[7 * (size_t)k + j], ev[7 * (size_t)k + j + 1]) != cudaSuccess) rc = RD_ECUDA;
      ms_per_launch[j] += ms / n_steps;
    }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  if (launches_per_step) *launches_per_step = step_launches(s);
  if (rc != RD_OK) return rc;
  DevCtl c;
  CK(read_ctl(s, c));
  s->launched = c.steps;
  return status_to_rd(c.status);
}

extern "C" int rd_state_autotune(rd_state* s, int32_t* tri_block, int32_t* vtx_block) {
  if (!s) return RD_EINVAL;
  DevCtl c0;
  CK(read_ctl(s, c0));
  if (c0.status) return RD_ENONPHYSICAL;
  const int a = (int)(c0.steps & 1);
  cudaStream_t st = s->m->stream;
  const int tri_c[] = {64, 128, 192, 256};
  const int vtx_c[] = {128, 256, 512};
  cudaEvent_t ev[7];
  for (auto& e : ev) cudaEventCreate(&e);
  // One untimed and one timed step with the shapes set on the state: ms the whole
  // step, ms1 / ms2 the stage-1 / stage-2 triangle kernels (events 0-1 and 3-4).
  auto time_step = [&](float& ms, float& ms1, float& ms2) -> int {
    k_begin<<<1, 1, 0, st>>>((DevCtl*)s->ctl.p, 0.0);
    CK(launch_step_any(s, a, nullptr, false));  // warm
    CK(launch_step_any(s, a, ev, false));
    CU(cudaStreamSynchronize(st));
    CU(cudaEventElapsedTime(&ms, ev[0], ev[6]));
    CU(cudaEventElapsedTime(&ms1, ev[0], ev[1]));
    CU(cudaEventElapsedTime(&ms2, ev[3], ev[4]));
    return RD_OK;
  };
  int best_t = TRI_BLOCK, best_t2 = TRI_BLOCK, best_v = VTX_BLOCK, rc = RD_OK;
  int best_o = s->df_variant, best_o2 = s->df_variant2;
  float best = 1e30f, best1 = 1e30f, best2 = 1e30f, ms = 0.f, ms1 = 0.f, ms2 = 0.f;
  // Triangle block size (and for RD_DF64 the kernel variant: 128 registers
  // without and with phase barriers, 96 and 80 with barriers) chosen per stage
  // from each stage's own kernel time; the two stages are independent kernels.
  const bool df = s->p.precision == RD_DF64;
  const int o0 = df ? 2 : s->df_variant, o1 = df ? 5 : s->df_variant;
  s->vtx_block = VTX_BLOCK;
  for (int o = o0; o <= o1 && rc == RD_OK; ++o) {
    s->df_variant = s->df_variant2 = o;
    for (int tb : tri_c) {
      s->tri_block = s->tri_block2 = tb;
      if ((rc = time_step(ms, ms1, ms2)) != RD_OK) break;
      if (ms1 < best1) { best1 = ms1; best_t = tb; best_o = o; }
      if (ms2 < best2) { best2 = ms2; best_t2 = tb; best_o2 = o; }
    }
  }
  s->df_variant = best_o;
  s->df_variant2 = best_o2;
  s->tri_block = best_t;
  s->tri_block2 = best_t2;
  for (int vb : vtx_c) {
    s->vtx_block = vb;
    if (rc != RD_OK || (rc = time_step(ms, ms1, ms2)) != RD_OK) break;
    if (ms < best) { best = ms; best_v = vb; }
  }
  s->vtx_block = best_v;
  // tiled step: a few tile sizes against the untiled step with the shapes above
  if (rc == RD_OK && s->m->h.nt >= 4096 && s->p.precision != RD_DF64) {
    float untiled = 1e30f;
    rc = rd_state_set_tiling(s, 0, 0);
    if (rc == RD_OK) rc = time_step(untiled, ms1, ms2);
    // (tile triangles, threads, flags)
    // (Staging the tile geometry in shared memory, RD_TILE_STAGE_GEOMETRY, measured
    // no faster at 4096^2 -- the tile kernels are issue-bound, not waiting on the
    // geometry loads -- and is not among the candidates.)
    const int c32[][3] = {{256, 128, 0}, {512, 128, 0}, {512, 256, 0}, {1024, 256, 0}};
    const int c64[][3] = {{128, 64, 0}, {256, 64, 0}, {256, 128, 0}};
    const int nc = s->pi == 0 ? 3 : 4;
    int best_tt = 0, best_bt = 0, best_fl = 0;
    float best_tiled = untiled;
    for (int k = 0; k < nc && rc == RD_OK; ++k) {
      const int* c = s->pi == 0 ? c64[k] : c32[k];
      int r = rd_state_set_tiling_ex(s, c[0], c[1], c[2]);
      if (r == RD_ENOTSUP) continue;  // no tile plan for this mesh, or not enough shared memory
      if ((rc = r) != RD_OK || (rc = time_step(ms, ms1, ms2)) != RD_OK) break;
      if (ms < best_tiled) { best_tiled = ms; best_tt = c[0]; best_bt = c[1]; best_fl = c[2]; }
    }
    if (best_tt && !(best_tiled < 0.98f * untiled)) {  // keep the untiled step unless tiling wins clearly
      best_tt = 0;
      best_bt = 0;
      best_fl = 0;
    }
    if (rc == RD_OK) rc = rd_state_set_tiling_ex(s, best_tt, best_bt, best_fl);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (s->g2) {  // the captured graph holds the old launch shapes
    cudaGraphExecDestroy(s->g2);
    s->g2 = nullptr;
  }
  if (tri_block) *tri_block = best_t;
  if (vtx_block) *vtx_block = best_v;
  return rc;
}

extern "C" int rd_state_launch_shapes(const rd_state* s, int32_t* tri_block, int32_t* vtx_block, int32_t* df_variant) {
  if (!s) return RD_EINVAL;
  if (tri_block) *tri_block = s->tri_block;
  if (vtx_block) *vtx_block = s->vtx_block;
  if (df_variant) *df_variant = s->df_variant;
  return RD_OK;
}

extern "C" int rd_state_set_launch_shapes(rd_state* s, int32_t tri_block, int32_t vtx_block, int32_t df_variant) {
  if (!s) return RD_EINVAL;
  if (tri_block != 64 && tri_block != 128 && tri_block != 192 && tri_block != 256) return RD_EINVAL;
  if (vtx_block != 128 && vtx_block != 256 && vtx_block != 512) return RD_EINVAL;
  if (df_variant < 2 || df_variant > 5) return RD_EINVAL;
  s->tri_block = s->tri_block2 = tri_block;
  s->vtx_block = vtx_block;
  s->df_variant = s->df_variant2 = df_variant;
  if (s->g2) {  // the captured graph holds the old launch shapes
    cudaStreamSynchronize(s->m->stream);
    cudaGraphExecDestroy(s->g2);
    s->g2 = nullptr;
  }
  return RD_OK;
}

extern "C" int rd_state_stage_shapes(const rd_state* s, int32_t stage, int32_t* tri_block, int32_t* df_variant) {
  if (!s || (stage != 1 && stage != 2)) return RD_EINVAL;
  if (tri_block) *tri_block = stage == 1 ? s->tri_block : s->tri_block2;
  if (df_variant) *df_variant = stage == 1 ? s->df_variant : s->df_variant2;
  return RD_OK;
}

extern "C" int rd_state_set_stage_shapes(rd_state* s, int32_t stage, int32_t tri_block, int32_t df_variant) {
  if (!s || (stage != 1 && stage != 2)) return RD_EINVAL;
  if (tri_block != 64 && tri_block != 128 && tri_block != 192 && tri_block != 256) return RD_EINVAL;
  if (df_variant < 2 || df_variant > 5) return RD_EINVAL;
  (stage == 1 ? s->tri_block : s->tri_block2) = tri_block;
  (stage == 1 ? s->df_variant : s->df_variant2) = df_variant;
  if (s->g2) {  // the captured graph holds the old launch shapes
    cudaStreamSynchronize(s->m->stream);
    cudaGraphExecDestroy(s->g2);
    s->g2 = nullptr;
  }
  return RD_OK;
}

extern "C" int rd_get_state(const rd_state* s, double* W_out) {
  if (!s || !W_out) return RD_EINVAL;
  DevCtl c;
  CK(read_ctl(s, c));
  int buf = (int)(c.steps & 1);
  return s->pi == 0 ? download_state<double>(s, buf, W_out) : download_state<float>(s, buf, W_out);
}

extern "C" int rd_conserved_totals(const rd_state* s, double out[4]) {
  if (!s || !out) return RD_EINVAL;
  DevCtl c;
  CK(read_ctl(s, c));
  int buf = (int)(c.steps & 1);
  const int nv = s->m->h.nv;
  unsigned nb = nblk(nv, VTX_BLOCK);
  cudaStream_t st = s->m->stream;
  if (s->pi == 0)
    k_conserved_partial<double, VTX_BLOCK><<<nb, VTX_BLOCK, 0, st>>>(
        nv, (const double*)s->W[buf].p, (const double*)s->m->geo[0][5].p, (double*)s->cons_partial.p);
  else
    k_conserved_partial<float, VTX_BLOCK><<<nb, VTX_BLOCK, 0, st>>>(
        nv, (const float*)s->W[buf].p, (const float*)s->m->geo[1][5].p, (double*)s->cons_partial.p);
  k_conserved_final<<<1, 32, 0, st>>>((int)nb, (const double*)s->cons_partial.p, (double*)s->cons_out.p);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(out, s->cons_out.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return RD_OK;
}

extern "C" int rd_get_time(const rd_state* s, double* t, int64_t* steps) {
  if (!s) return RD_EINVAL;
  DevCtl c;
  CK(read_ctl(s, c));
  if (t) *t = c.t;
  if (steps) *steps = c.steps;
  return RD_OK;
}

extern "C" int rd_get_dt(const rd_state* s, double* dt) {
  if (!s || !dt) return RD_EINVAL;
  DevCtl c;
  CK(read_ctl(s, c));
  *dt = c.dt;
  return RD_OK;
}

extern "C" int rd_state_triangle_shares(rd_state* s, int32_t which, double* out, double* cfl_term) {
  if (!s || !out || which < 0 || which > 2) return RD_EINVAL;
  DevCtl c;
  CK(read_ctl(s, c));
  int buf = (int)(c.steps & 1);
  rd_mesh* m = s->m;
  const int nt = m->h.nt, nv = m->h.nv;
  DevBuf tmp;
  CK(dev_alloc(tmp, 36 * (size_t)nt * s->ts, m->stream));
  cudaStream_t st = m->stream;
  int rc = RD_OK;
  std::vector<double> terms(36 * (size_t)nt), cf(nt);
  if (s->pi == 0) {
    k_tri_terms<double><<<nblk(nt, TRI_BLOCK), TRI_BLOCK, 0, st>>>(
        nt, nv, (const int*)m->tri.p, geo_of<double>(m), (const double*)s->Z[buf].p, (const double*)s->spd[buf].p,
        s->p.gamma, s->p.eps_fix, (double*)tmp.p, (double*)s->cfl.p, (DevCtl*)s->ctl.p);
    if (cudaMemcpyAsync(terms.data(), tmp.p, terms.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(cf.data(), s->cfl.p, nt * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = RD_ECUDA;
  } else {
    k_tri_terms<float><<<nblk(nt, TRI_BLOCK), TRI_BLOCK, 0, st>>>(
        nt, nv, (const int*)m->tri.p, geo_of<float>(m), (const float*)s->Z[buf].p, (const float*)s->spd[buf].p,
        (float)s->p.gamma, (float)s->p.eps_fix, (float*)tmp.p, (float*)s->cfl.p, (DevCtl*)s->ctl.p);
    std::vector<float> tf(terms.size()), cff(nt);
    if (cudaMemcpyAsync(tf.data(), tmp.p, tf.size() * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(cff.data(), s->cfl.p, nt * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = RD_ECUDA;
    for (size_t i = 0; i < tf.size(); ++i) terms[i] = tf[i];
    for (int i = 0; i < nt; ++i) cf[i] = cff[i];
  }
  if (rc == RD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = RD_ECUDA;
  cudaGetLastError();
  dev_free(tmp);
  if (rc != RD_OK) return rc;
  const size_t off = (size_t)which * 12 * nt;
  for (int t = 0; t < nt; ++t) {
    int to = m->h.tperm[t];
    std::memcpy(out + 12 * (size_t)to, terms.data() + off + 12 * (size_t)t, 12 * sizeof(double));
    if (cfl_term) cfl_term[to] = cf[t];
  }
  CK(read_ctl(s, c));
  return status_to_rd(c.status);
}

extern "C" void rd_state_destroy(rd_state* s) {
  if (!s) return;
  if (s->m && s->m->stream) cudaStreamSynchronize(s->m->stream);
  if (s->g2) cudaGraphExecDestroy(s->g2);
  for (int b = 0; b < 2; ++b) {
    dev_free(s->W[b]);
    dev_free(s->Z[b]);
    dev_free(s->spd[b]);
  }
  DevBuf* bufs[] = {&s->Ws, &s->Zs, &s->R1, &s->share, &s->rec, &s->cfl, &s->partial, &s->ctl,
                    &s->cons_partial, &s->cons_out, &s->stage, &s->vr, &s->ghostW, &s->dWdf};
  for (DevBuf* b : bufs) dev_free(*b);
  adjoint_free(s->adj);
  tile_plan_free(s->tiles);
  delete s;
}

// ---------------------------------------------------------------------------
// standalone CFL time step on caller-owned device arrays
// ---------------------------------------------------------------------------
namespace rd {
// Shared by rd_cfl_dt and its allocation-free variant: validates, clears the
// control word, launches k_cfl_dt on the stream and waits for it.
int cfl_dt_launch(int32_t nv, int32_t nt, int32_t precision, const void* W, const int32_t* tri, const void* lmax,
                  const void* V, const int32_t* ptr, const int32_t* ent, double gamma, double cfl, double* dt_out,
                  void* stream, double* partial, DtScratchCtl* ctl) {
  static_assert(CFL_DT_BLOCK == VTX_BLOCK, "block size of the CFL reduction");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned nb = nblk(nv, VTX_BLOCK);
  CU(cudaMemsetAsync(ctl, 0, sizeof(DtScratchCtl), st));
  if (precision == RD_FP64)
    k_cfl_dt<double, VTX_BLOCK><<<nb, VTX_BLOCK, 0, st>>>(nv, nt, (const double*)W, tri, (const double*)lmax,
                                                          (const double*)V, ptr, ent, gamma, cfl, partial, ctl, dt_out);
  else
    k_cfl_dt<float, VTX_BLOCK><<<nb, VTX_BLOCK, 0, st>>>(nv, nt, (const float*)W, tri, (const float*)lmax,
                                                         (const float*)V, ptr, ent, (float)gamma, (float)cfl, partial,
                                                         ctl, dt_out);
  CU(cudaGetLastError());
  DtScratchCtl c;
  CU(cudaMemcpyAsync(&c, ctl, sizeof(c), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return c.status ? RD_ENONPHYSICAL : RD_OK;
}

int cfl_dt_check(int32_t nv, int32_t nt, int32_t precision, const void* W, const int32_t* tri, const void* lmax,
                 const void* V, const int32_t* ptr, const int32_t* ent, double gamma, double cfl, double* dt_out) {
  if (nv < 1 || nt < 1 || !W || !tri || !lmax || !V || !ptr || !ent || !dt_out) return RD_EINVAL;
  if (precision != RD_FP64 && precision != RD_FP32) return RD_EINVAL;
  if (!(gamma > 1.0) || !(cfl > 0.0)) return RD_EINVAL;
  return RD_OK;
}
}  // namespace rd

extern "C" int rd_cfl_dt(int32_t n_vertex, int32_t n_tri, int32_t precision, const void* W, const int32_t* tri,
                         const void* lmax, const void* V, const int32_t* csr_ptr, const int32_t* csr_ent,
                         double gamma, double cfl, double* dt_out, void* cuda_stream) {
  CK(cfl_dt_check(n_vertex, n_tri, precision, W, tri, lmax, V, csr_ptr, csr_ent, gamma, cfl, dt_out));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf scratch;
  size_t nb = nblk(n_vertex, VTX_BLOCK);
  size_t off = (nb * sizeof(double) + 255) / 256 * 256;
  CK(dev_alloc(scratch, off + sizeof(DtScratchCtl), st));
  int rc = cfl_dt_launch(n_vertex, n_tri, precision, W, tri, lmax, V, csr_ptr, csr_ent, gamma, cfl, dt_out,
                         (void*)st, (double*)scratch.p, (DtScratchCtl*)((char*)scratch.p + off));
  cudaStreamSynchronize(st);
  dev_free(scratch);
  return rc;
}

// ---------------------------------------------------------------------------
// misc
// ---------------------------------------------------------------------------
extern "C" const char* rd_strerror(int status) {
  switch (status) {
    case RD_OK: return "ok";
    case RD_EINVAL: return "invalid argument";
    case RD_ENOMEM: return "out of memory";
    case RD_ECUDA: return "CUDA runtime error";
    case RD_ENONPHYSICAL: return "non-physical state (rho<=0, p<=0, c^2<=0, singular N^ or NaN)";
    case RD_ETIMEOUT: return "bounded device wait expired";
    case RD_ENOTSUP: return "not supported";
    default: return "unknown status";
  }
}

extern "C" int rd_version(void) { return 1; }
