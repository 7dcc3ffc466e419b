// rd_batch.cu -- batched form: many independent periodic meshes advanced together.
//
// The meshes of a batch are concatenated into one vertex range and one
// triangle range (each mesh keeps its own internal order), so every kernel of
// the plain step runs once per step over the whole batch; each mesh keeps its
// own dt (a per-mesh CFL min, Sec. 3.2) and its own time and step count.
// rd_batch_run replays n steps as ONE CUDA-graph launch.  Launch shapes come
// from rd_batch_autotune, which times the candidates on the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "rd_df64.h"
#include "rd_device.h"
#include "rd_internal.h"
#include "rd_kernels.cuh"

using namespace rd;

struct rd_batch {
  int32_t n_mesh = 0;
  rd_params p{};
  int pi = 0;
  size_t ts = 8;
  cudaStream_t stream = nullptr;
  int64_t nv = 0, nt = 0;
  std::vector<rd_mesh*> meshes;
  std::vector<int64_t> voff, toff;  // [n_mesh + 1]
  DevBuf tri, ptr, ent, vmesh, tmesh, geo[6];
  DevBuf W[2], Z[2], spd[2], Ws, Zs, R1, share, rec, cfl, ctl, mmin, dtm, tm, stepsm, stage;
  DevBuf geo_df[4], dWdf;  // RD_DF64: double-float geometry, W* - W^n of every vertex
  int df_variant = 2, df_variant2 = 2;  // RD_DF64 triangle-kernel variant of stage 1 / 2 (autotuned)
  long long launched = 0;
  int tri_block = TRI_BLOCK, tri_block2 = TRI_BLOCK, vtx_block = VTX_BLOCK;  // tri_block: stage 1
  cudaGraphExec_t graph = nullptr;
  int32_t graph_steps = -1;
  int graph_parity = -1;
};

namespace {

__global__ void k_batch_begin(DevCtl* ctl, int n_mesh, unsigned long long* mmin) {
  if (ctl->status == 0) ctl->stop = 0;
  for (int m = threadIdx.x; m < n_mesh; m += blockDim.x)
    mmin[m] = (unsigned long long)__double_as_longlong((double)INFINITY);
}

template <class T>
int batch_step(rd_batch* b, int a, cudaEvent_t* ev, bool commit) {
  const int nt = (int)b->nt, nv = (int)b->nv, c = 1 - a;
  cudaStream_t st = b->stream;
  const int TB = b->tri_block, TB2 = b->tri_block2, VB = b->vtx_block;
  unsigned gt = nblk(nt, TB), gt2 = nblk(nt, TB2), gv = nblk(nv, VB);
  DevGeo<T> g{(const T*)b->geo[0].p, (const T*)b->geo[1].p, (const T*)b->geo[2].p, (const T*)b->geo[3].p,
              (const T*)b->geo[4].p};
  const T* V = (const T*)b->geo[5].p;
  const int* tri = (const int*)b->tri.p;
  const int* ptr = (const int*)b->ptr.p;
  const int* ent = (const int*)b->ent.p;
  const uint16_t* vm = (const uint16_t*)b->vmesh.p;
  const uint16_t* tm = (const uint16_t*)b->tmesh.p;
  DevCtl* ctl = (DevCtl*)b->ctl.p;
  const double* dtm = (const double*)b->dtm.p;
  T gamma = (T)b->p.gamma, eps = (T)b->p.eps_fix;
  T* share = (T*)b->share.p;
  T* rec = (T*)b->rec.p;
  T* cf = (T*)b->cfl.p;
  auto mark = [&](int k) {
    if (ev) cudaEventRecord(ev[k], st);
  };
  mark(0);
  const T* Za = (const T*)b->Z[a].p;
  const T* Sa = (const T*)b->spd[a].p;
  BlendArgs<T> ba;  // Bmax / Bmin and selective lumping; Bx is not offered in batched mode
  ba.mode = b->p.scheme == RD_BMAX2 ? BLEND_MAX : b->p.scheme == RD_BMIN2 ? BLEND_MIN : BLEND_B;
  ba.sl = b->p.lumping == RD_LUMP_SELECTIVE;
  const bool df = sizeof(T) == 8 && b->p.precision == RD_DF64;
  TriArraysDF x;
  if (df) {
    x.nt = nt;
    x.tri = tri;
    x.g.nx = (const float2*)b->geo_df[0].p;
    x.g.ny = (const float2*)b->geo_df[1].p;
    x.g.hl = (const float2*)b->geo_df[2].p;
    x.g.area = (const float2*)b->geo_df[3].p;
    x.g.lmax = (const double*)b->geo[4].p;
    x.share = (double*)share;
    x.rec = rec;
    x.cfl = (double*)cf;
    x.ctl = ctl;
    x.variant = b->df_variant;
    x.dtm = dtm;
    x.tmesh = tm;
  }
  if (df) {
    x.Z = (const double*)Za;
    x.spd = (const double*)Sa;
    CK(launch_tri_stage1_df(b->p, x, *reinterpret_cast<const BlendArgs<double>*>(&ba), gt, TB, st));
  } else
  switch (b->p.scheme) {
    case RD_N1:
      k_tri_stage1<T, RD_N1><<<gt, TB, 0, st>>>(nt, nv, tri, g, Za, Sa, Gas<T>::of(gamma), eps, share, nullptr, cf, ctl);
      break;
    case RD_LDA2:
      k_tri_stage1<T, RD_LDA2><<<gt, TB, 0, st>>>(nt, nv, tri, g, Za, Sa, Gas<T>::of(gamma), eps, share, rec, cf, ctl);
      break;
    default:
      if (b->p.scheme == RD_B2 && b->p.lumping == RD_LUMP_GLOBAL)
        k_tri_stage1<T, RD_B2><<<gt, TB, 0, st>>>(nt, nv, tri, g, Za, Sa, Gas<T>::of(gamma), eps, share, rec, cf,
                                                  ctl);
      else  // generic blend instantiation: Bmax, Bmin, Bx, B with selective lumping
        k_tri_stage1<T, RD_BMAX2><<<gt, TB, 0, st>>>(nt, nv, tri, g, Za, Sa, Gas<T>::of(gamma), eps, share, rec, cf,
                                                     ctl, ba);
      break;
  }
  mark(1);
  k_gather_cfl_batch<T><<<gv, VB, 0, st>>>(nv, ptr, ent, share, cf, V, vm, (T*)b->R1.p,
                                           (unsigned long long*)b->mmin.p, ctl);
  k_batch_dt<<<1, 256, 0, st>>>(b->n_mesh, b->p.cfl, (unsigned long long*)b->mmin.p, (double*)b->dtm.p, ctl);
  mark(2);
  if (b->p.scheme == RD_N1) {
    k_update<T><<<gv, VB, 0, st>>>(nv, (const T*)b->W[a].p, (const T*)b->R1.p, ptr, ent, nullptr, V, gamma,
                                   (T*)b->W[c].p, (T*)b->Z[c].p, (T*)b->spd[c].p, ctl, dtm, vm);
    mark(3);
    mark(4);
    mark(5);
  } else {
    k_update<T><<<gv, VB, 0, st>>>(nv, (const T*)b->W[a].p, (const T*)b->R1.p, ptr, ent, nullptr, V, gamma,
                                   (T*)b->Ws.p, (T*)b->Zs.p, nullptr, ctl, dtm, vm, nullptr, WallArgs<T>(),
                                   GhostArgs<T>(), df ? (float2*)b->dWdf.p : nullptr);
    mark(3);
    if (df) {
      x.Z = (const double*)b->Zs.p;
      x.dw = (const float2*)b->dWdf.p;
      x.variant = b->df_variant2;
      CK(launch_tri_stage2_df(b->p, x, *reinterpret_cast<const BlendArgs<double>*>(&ba), gt2, TB2, st));
    } else if (b->p.scheme == RD_LDA2)
      k_tri_stage2<T, RD_LDA2><<<gt2, TB2, 0, st>>>(nt, nv, tri, g, (const T*)b->Zs.p, (const T*)b->W[a].p,
                                                  (const T*)b->Ws.p, rec, Gas<T>::of(gamma), eps, share, ctl, dtm, tm,
                                                  ba);
    else if (b->p.scheme == RD_B2 && b->p.lumping == RD_LUMP_GLOBAL)
      k_tri_stage2<T, RD_B2><<<gt2, TB2, 0, st>>>(nt, nv, tri, g, (const T*)b->Zs.p, (const T*)b->W[a].p,
                                                (const T*)b->Ws.p, rec, Gas<T>::of(gamma), eps, share, ctl, dtm, tm);
    else
      k_tri_stage2<T, RD_BMAX2><<<gt2, TB2, 0, st>>>(nt, nv, tri, g, (const T*)b->Zs.p, (const T*)b->W[a].p,
                                                   (const T*)b->Ws.p, rec, Gas<T>::of(gamma), eps, share, ctl, dtm,
                                                   tm, ba);
    mark(4);
    k_update<T><<<gv, VB, 0, st>>>(nv, (const T*)b->Ws.p, nullptr, ptr, ent, share, V, gamma, (T*)b->W[c].p,
                                   (T*)b->Z[c].p, (T*)b->spd[c].p, ctl, dtm, vm);
    mark(5);
  }
  if (commit)
    k_commit_batch<<<1, 256, 0, st>>>(b->n_mesh, dtm, (double*)b->tm.p, (long long*)b->stepsm.p, ctl);
  mark(6);
  CU(cudaGetLastError());
  return RD_OK;
}

int batch_step_any(rd_batch* b, int a, cudaEvent_t* ev = nullptr, bool commit = true) {
  return b->pi == 0 ? batch_step<double>(b, a, ev, commit) : batch_step<float>(b, a, ev, commit);
}

int read_ctl(rd_batch* b, DevCtl& c) {
  CU(cudaMemcpyAsync(&c, b->ctl.p, sizeof(DevCtl), cudaMemcpyDeviceToHost, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  return RD_OK;
}

template <class T>
int concat_geometry(rd_batch* b) {
  const int64_t nt = b->nt, nv = b->nv;
  std::vector<T> buf;
  for (int k = 0; k < 6; ++k) {
    const bool per_vertex = (k == 5);
    const int comps = k < 3 ? 3 : 1;
    const int64_t n = per_vertex ? nv : nt;
    buf.assign((size_t)(comps * n), T(0));
    for (int32_t m = 0; m < b->n_mesh; ++m) {
      const HostMesh& h = b->meshes[m]->h;
      const std::vector<double>* src[6] = {&h.nx, &h.ny, &h.hl, &h.area, &h.lmax, &h.V};
      const int64_t off = per_vertex ? b->voff[m] : b->toff[m];
      const int64_t len = per_vertex ? h.nv : h.nt;
      for (int c = 0; c < comps; ++c)
        for (int64_t i = 0; i < len; ++i) buf[(size_t)(c * n + off + i)] = (T)(*src[k])[(size_t)(c * len + i)];
    }
    CK(dev_alloc(b->geo[k], buf.size() * sizeof(T), b->stream));
    CU(cudaMemcpyAsync(b->geo[k].p, buf.data(), buf.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream));
    CU(cudaStreamSynchronize(b->stream));
  }
  return RD_OK;
}

// RD_DF64: nx, ny, hl [3][nt] and area [nt] of the concatenated meshes as
// double-float pairs (the same split as the single-mesh store).
int concat_geometry_df(rd_batch* b) {
  const int64_t nt = b->nt;
  std::vector<double> buf;
  std::vector<float2> sp;
  for (int k = 0; k < 4; ++k) {
    const int comps = k < 3 ? 3 : 1;
    buf.assign((size_t)(comps * nt), 0.0);
    for (int32_t m = 0; m < b->n_mesh; ++m) {
      const HostMesh& h = b->meshes[m]->h;
      const std::vector<double>* src[4] = {&h.nx, &h.ny, &h.hl, &h.area};
      for (int c = 0; c < comps; ++c)
        for (int64_t i = 0; i < h.nt; ++i) buf[(size_t)(c * nt + b->toff[m] + i)] = (*src[k])[(size_t)(c * h.nt + i)];
    }
    split_df_host(buf, sp);
    CK(dev_alloc(b->geo_df[k], sp.size() * sizeof(float2), b->stream));
    CU(cudaMemcpyAsync(b->geo_df[k].p, sp.data(), sp.size() * sizeof(float2), cudaMemcpyHostToDevice, b->stream));
    CU(cudaStreamSynchronize(b->stream));
  }
  return RD_OK;
}

template <class T>
int upload_states(rd_batch* b, const double* const* W0) {
  std::vector<T> buf(4 * (size_t)b->nv);
  for (int32_t m = 0; m < b->n_mesh; ++m) {
    const HostMesh& h = b->meshes[m]->h;
    const double* W = W0[m];
    if (!W) return RD_EINVAL;
    for (int32_t i = 0; i < h.nv; ++i)
      for (int k = 0; k < 4; ++k) {
        double x = W[(size_t)k * h.nv + h.vperm[i]];
        if (!std::isfinite(x)) return RD_ENONPHYSICAL;
        buf[4 * (size_t)(b->voff[m] + i) + k] = (T)x;
      }
  }
  CU(cudaMemcpyAsync(b->W[0].p, buf.data(), buf.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream));
  k_prepare<T><<<nblk(b->nv, 256), 256, 0, b->stream>>>((int)b->nv, (const T*)b->W[0].p, (T)b->p.gamma,
                                                          (T*)b->Z[0].p, (T*)b->spd[0].p, (DevCtl*)b->ctl.p);
  CU(cudaGetLastError());
  DevCtl c;
  CK(read_ctl(b, c));
  return c.status ? RD_ENONPHYSICAL : RD_OK;
}

int build(rd_batch* b, const double* const* W0) {
  const int32_t M = b->n_mesh;
  cudaStream_t st = b->stream;
  b->voff.assign(M + 1, 0);
  b->toff.assign(M + 1, 0);
  for (int32_t m = 0; m < M; ++m) {
    b->voff[m + 1] = b->voff[m] + b->meshes[m]->h.nv;
    b->toff[m + 1] = b->toff[m] + b->meshes[m]->h.nt;
  }
  b->nv = b->voff[M];
  b->nt = b->toff[M];
  if (b->nv >= INT32_MAX / 4 || 3 * b->nt >= INT32_MAX) return RD_EINVAL;
  const int64_t nv = b->nv, nt = b->nt;
  // connectivity with offsets
  std::vector<int32_t> tri(3 * (size_t)nt), ptr((size_t)nv + 1), ent(3 * (size_t)nt);
  std::vector<uint16_t> vm((size_t)nv), tm((size_t)nt);
  for (int32_t m = 0; m < M; ++m) {
    const HostMesh& h = b->meshes[m]->h;
    const int64_t vo = b->voff[m], to = b->toff[m];
    for (int c = 0; c < 3; ++c)
      for (int32_t t = 0; t < h.nt; ++t) tri[(size_t)(c * nt + to + t)] = (int32_t)(h.tri[(size_t)c * h.nt + t] + vo);
    for (int32_t i = 0; i < h.nv; ++i) {
      ptr[(size_t)(vo + i)] = (int32_t)(h.csr_ptr[i] + 3 * to);
      vm[(size_t)(vo + i)] = (uint16_t)m;
    }
    for (int64_t e = 0; e < 3 * (int64_t)h.nt; ++e) ent[(size_t)(3 * to + e)] = (int32_t)(h.csr_ent[e] + 3 * to);
    for (int32_t t = 0; t < h.nt; ++t) tm[(size_t)(to + t)] = (uint16_t)m;
  }
  ptr[(size_t)nv] = (int32_t)(3 * nt);
  auto up = [&](DevBuf& d, const void* src, size_t bytes) -> int {
    CK(dev_alloc(d, bytes, st));
    CU(cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
    return RD_OK;
  };
  CK(up(b->tri, tri.data(), tri.size() * 4));
  CK(up(b->ptr, ptr.data(), ptr.size() * 4));
  CK(up(b->ent, ent.data(), ent.size() * 4));
  CK(up(b->vmesh, vm.data(), vm.size() * 2));
  CK(up(b->tmesh, tm.data(), tm.size() * 2));
  CK(b->pi == 0 ? concat_geometry<double>(b) : concat_geometry<float>(b));
  if (b->p.precision == RD_DF64) CK(concat_geometry_df(b));
  const size_t ts = b->ts;
  for (int k = 0; k < 2; ++k) {
    CK(dev_alloc(b->W[k], 4 * nv * ts, st));
    CK(dev_alloc(b->Z[k], 4 * nv * ts, st));
    CK(dev_alloc(b->spd[k], nv * ts, st));
  }
  CK(dev_alloc(b->R1, 4 * nv * ts, st));
  CK(dev_alloc(b->share, 12 * nt * ts, st));
  CK(dev_alloc(b->cfl, nt * ts, st));
  if (b->p.scheme != RD_N1) {
    CK(dev_alloc(b->Ws, 4 * nv * ts, st));
    CK(dev_alloc(b->Zs, 4 * nv * ts, st));
    CK(dev_alloc(b->rec, 16 * nt * ts, st));
    if (b->p.precision == RD_DF64) CK(dev_alloc(b->dWdf, 4 * nv * sizeof(float2), st));
  }
  CK(dev_alloc(b->ctl, sizeof(DevCtl), st));
  CK(dev_alloc(b->mmin, M * sizeof(unsigned long long), st));
  CK(dev_alloc(b->dtm, M * sizeof(double), st));
  CK(dev_alloc(b->tm, M * sizeof(double), st));
  CK(dev_alloc(b->stepsm, M * sizeof(long long), st));
  CU(cudaMemsetAsync(b->ctl.p, 0, sizeof(DevCtl), st));
  CU(cudaMemsetAsync(b->dtm.p, 0, M * sizeof(double), st));
  CU(cudaMemsetAsync(b->tm.p, 0, M * sizeof(double), st));
  CU(cudaMemsetAsync(b->stepsm.p, 0, M * sizeof(long long), st));
  return b->pi == 0 ? upload_states<double>(b, W0) : upload_states<float>(b, W0);
}

template <class T>
int download(const rd_batch* b, int buf, int32_t m, double* W_out) {
  const HostMesh& h = b->meshes[m]->h;
  std::vector<T> tmp(4 * (size_t)h.nv);
  const T* src = (const T*)b->W[buf].p + 4 * (size_t)b->voff[m];
  CU(cudaMemcpyAsync(tmp.data(), src, tmp.size() * sizeof(T), cudaMemcpyDeviceToHost, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  for (int32_t i = 0; i < h.nv; ++i)
    for (int k = 0; k < 4; ++k) W_out[(size_t)k * h.nv + h.vperm[i]] = (double)tmp[4 * (size_t)i + k];
  return RD_OK;
}

void destroy_graph(rd_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_steps = -1;
  b->graph_parity = -1;
}

// Capture n_steps steps starting from buffer parity `a` into one executable graph.
int capture(rd_batch* b, int32_t n_steps, int a) {
  destroy_graph(b);
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int rc = RD_OK;
  for (int32_t k = 0; k < n_steps && rc == RD_OK; ++k) rc = batch_step_any(b, (a + k) & 1);
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (rc != RD_OK || e != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return rc != RD_OK ? rc : RD_ECUDA;
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->graph = nullptr;
    return RD_ECUDA;
  }
  b->graph_steps = n_steps;
  b->graph_parity = a;
  return RD_OK;
}

}  // namespace

extern "C" int rd_batch_create(int32_t n_mesh, rd_mesh* const* meshes, const double* const* W0, const rd_params* p,
                               rd_batch** out) {
  if (!out) return RD_EINVAL;
  *out = nullptr;
  if (n_mesh < 1 || n_mesh > 65535 || !meshes || !W0 || !p) return RD_EINVAL;
  if (p->scheme < RD_N1 || p->scheme > RD_BX2) return RD_EINVAL;
  if (p->lumping != RD_LUMP_GLOBAL && p->lumping != RD_LUMP_SELECTIVE) return RD_EINVAL;
  if ((p->lumping == RD_LUMP_SELECTIVE && p->scheme == RD_N1) || p->reserved != 0) return RD_EINVAL;
  if (p->scheme == RD_BX2) return RD_ENOTSUP;  // its |v| range is global per mesh
  if (p->precision != RD_FP64 && p->precision != RD_FP32 && p->precision != RD_DF64) return RD_EINVAL;
  if (!(p->cfl > 0.0) || !(p->gamma > 1.0) || !(p->eps_fix >= 0.0)) return RD_EINVAL;
  for (int32_t m = 0; m < n_mesh; ++m)
    if (!meshes[m] || meshes[m]->stream != meshes[0]->stream) return RD_EINVAL;
  for (int32_t m = 0; m < n_mesh; ++m)
    if (meshes[m]->n_ghost || meshes[m]->n_wall) return RD_ENOTSUP;  // periodic meshes only
  rd_batch* b = new (std::nothrow) rd_batch();
  if (!b) return RD_ENOMEM;
  b->n_mesh = n_mesh;
  b->p = *p;
  b->pi = p->precision == RD_FP32 ? 1 : 0;  // RD_DF64 keeps the FP64 state
  b->ts = b->pi == 0 ? 8 : 4;
  b->stream = meshes[0]->stream;
  b->meshes.assign(meshes, meshes + n_mesh);
  int rc = build(b, W0);
  if (rc != RD_OK) {
    rd_batch_destroy(b);
    return rc;
  }
  *out = b;
  return RD_OK;
}

extern "C" int rd_batch_run(rd_batch* b, int32_t n_steps) {
  if (!b || n_steps < 0) return RD_EINVAL;
  DevCtl c0;
  CK(read_ctl(b, c0));
  if (c0.status) return RD_ENONPHYSICAL;
  b->launched = c0.steps;
  if (n_steps == 0) return RD_OK;
  const int a = (int)(b->launched & 1);
  k_batch_begin<<<1, 256, 0, b->stream>>>((DevCtl*)b->ctl.p, b->n_mesh, (unsigned long long*)b->mmin.p);
  CU(cudaGetLastError());
  if (!b->graph || b->graph_steps != n_steps || b->graph_parity != a) CK(capture(b, n_steps, a));
  CU(cudaGraphLaunch(b->graph, b->stream));
  DevCtl c;
  CK(read_ctl(b, c));
  b->launched = c.steps;
  return c.status ? RD_ENONPHYSICAL : RD_OK;
}

extern "C" int rd_batch_get_state(const rd_batch* b, int32_t mesh, double* W_out) {
  if (!b || !W_out || mesh < 0 || mesh >= b->n_mesh) return RD_EINVAL;
  DevCtl c;
  CK(read_ctl(const_cast<rd_batch*>(b), c));
  int buf = (int)(c.steps & 1);
  return b->pi == 0 ? download<double>(b, buf, mesh, W_out) : download<float>(b, buf, mesh, W_out);
}

extern "C" int rd_batch_get_dt(const rd_batch* b, double* dt_out) {
  if (!b || !dt_out) return RD_EINVAL;
  CU(cudaMemcpyAsync(dt_out, b->dtm.p, b->n_mesh * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  return RD_OK;
}

extern "C" int rd_batch_get_time(const rd_batch* b, double* t_out, int64_t* steps_out) {
  if (!b) return RD_EINVAL;
  if (t_out) CU(cudaMemcpyAsync(t_out, b->tm.p, b->n_mesh * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  if (steps_out)
    CU(cudaMemcpyAsync(steps_out, b->stepsm.p, b->n_mesh * sizeof(int64_t), cudaMemcpyDeviceToHost, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  return RD_OK;
}

extern "C" int rd_batch_sizes(const rd_batch* b, int64_t* n_vertex, int64_t* n_tri) {
  if (!b) return RD_EINVAL;
  if (n_vertex) *n_vertex = b->nv;
  if (n_tri) *n_tri = b->nt;
  return RD_OK;
}

// Times one uncommitted step per candidate launch shape and keeps the fastest.
extern "C" int rd_batch_autotune(rd_batch* b, int32_t* tri_block, int32_t* vtx_block) {
  if (!b) return RD_EINVAL;
  DevCtl c0;
  CK(read_ctl(b, c0));
  if (c0.status) return RD_ENONPHYSICAL;
  const int a = (int)(c0.steps & 1);
  const int tri_c[] = {64, 128, 192, 256};
  const int vtx_c[] = {128, 256, 512};
  cudaEvent_t ev[7];
  for (auto& e : ev) cudaEventCreate(&e);
  // one untimed and one timed step: ms the whole step, ms1 / ms2 the stage-1 /
  // stage-2 triangle kernels (events 0-1 and 3-4)
  auto time_step = [&](float& ms, float& ms1, float& ms2) -> int {
    k_batch_begin<<<1, 256, 0, b->stream>>>((DevCtl*)b->ctl.p, b->n_mesh, (unsigned long long*)b->mmin.p);
    CK(batch_step_any(b, a, nullptr, false));  // warm
    k_batch_begin<<<1, 256, 0, b->stream>>>((DevCtl*)b->ctl.p, b->n_mesh, (unsigned long long*)b->mmin.p);
    CK(batch_step_any(b, a, ev, false));
    CU(cudaStreamSynchronize(b->stream));
    CU(cudaEventElapsedTime(&ms, ev[0], ev[6]));
    CU(cudaEventElapsedTime(&ms1, ev[0], ev[1]));
    CU(cudaEventElapsedTime(&ms2, ev[3], ev[4]));
    return RD_OK;
  };
  int best_t = TRI_BLOCK, best_t2 = TRI_BLOCK, best_v = VTX_BLOCK, rc = RD_OK;
  int best_o = b->df_variant, best_o2 = b->df_variant2;
  float best = 1e30f, best1 = 1e30f, best2 = 1e30f, ms = 0.f, ms1 = 0.f, ms2 = 0.f;
  // triangle block size (and for RD_DF64 the kernel variant) per stage, from each
  // stage's own kernel time
  const int o0 = b->p.precision == RD_DF64 ? 2 : b->df_variant, o1 = b->p.precision == RD_DF64 ? 5 : b->df_variant;
  b->vtx_block = VTX_BLOCK;
  for (int o = o0; o <= o1 && rc == RD_OK; ++o) {
    b->df_variant = b->df_variant2 = o;
    for (int tb : tri_c) {
      b->tri_block = b->tri_block2 = tb;
      if ((rc = time_step(ms, ms1, ms2)) != RD_OK) break;
      if (ms1 < best1) { best1 = ms1; best_t = tb; best_o = o; }
      if (ms2 < best2) { best2 = ms2; best_t2 = tb; best_o2 = o; }
    }
  }
  b->df_variant = best_o;
  b->df_variant2 = best_o2;
  b->tri_block = best_t;
  b->tri_block2 = best_t2;
  for (int vb : vtx_c) {
    b->vtx_block = vb;
    if (rc != RD_OK || (rc = time_step(ms, ms1, ms2)) != RD_OK) break;
    if (ms < best) { best = ms; best_v = vb; }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  b->vtx_block = best_v;
  destroy_graph(b);
  if (tri_block) *tri_block = best_t;
  if (vtx_block) *vtx_block = best_v;
  return rc;
}

extern "C" int rd_batch_profile(rd_batch* b, int32_t n_steps, double* ms_per_launch) {
  if (!b || n_steps <= 0 || !ms_per_launch) return RD_EINVAL;
  DevCtl c0;
  CK(read_ctl(b, c0));
  if (c0.status) return RD_ENONPHYSICAL;
  b->launched = c0.steps;
  k_batch_begin<<<1, 256, 0, b->stream>>>((DevCtl*)b->ctl.p, b->n_mesh, (unsigned long long*)b->mmin.p);
  std::vector<cudaEvent_t> ev(7 * (size_t)n_steps, nullptr);
  int rc = RD_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = RD_ECUDA;
  for (int32_t k = 0; k < n_steps && rc == RD_OK; ++k) {
    rc = batch_step_any(b, (int)(b->launched & 1), ev.data() + 7 * (size_t)k);
    b->launched++;
  }
  if (rc == RD_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = RD_ECUDA;
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
  if (rc != RD_OK) return rc;
  DevCtl c;
  CK(read_ctl(b, c));
  b->launched = c.steps;
  return c.status ? RD_ENONPHYSICAL : RD_OK;
}

extern "C" void rd_batch_destroy(rd_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  destroy_graph(b);
  DevBuf* bufs[] = {&b->tri, &b->ptr, &b->ent, &b->vmesh, &b->tmesh, &b->Ws, &b->Zs, &b->R1, &b->share,
                    &b->rec, &b->cfl, &b->ctl, &b->mmin, &b->dtm, &b->tm, &b->stepsm, &b->stage, &b->dWdf};
  for (DevBuf* d : bufs) dev_free(*d);
  for (int k = 0; k < 6; ++k) dev_free(b->geo[k]);
  for (int k = 0; k < 4; ++k) dev_free(b->geo_df[k]);
  for (int k = 0; k < 2; ++k) {
    dev_free(b->W[k]);
    dev_free(b->Z[k]);
    dev_free(b->spd[k]);
  }
  delete b;
}
