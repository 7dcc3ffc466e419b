// rd_part.cu -- one part of a vertex-partitioned step (rd_partition.cpp has
// the plan).  A part holds its owned and ghost vertices and every triangle
// with an owned corner, and runs the kernels of the plain step on them; the
// caller moves the ghost states between parts (NCCL point-to-point, peer
// copies, or plain copies when all parts share one device) and takes the
// minimum of the parts' dt:
//
//   PACK_W   -> exchange -> UNPACK_W    ghosts' W^n (then their Z and |v|+c)
//   STAGE1                              triangles at W^n, gather of the owned
//                                       vertices, this part's CFL dt
//   (dt <- min over parts)
//   UPDATE1                             owned W* (N1: W^{n+1}, step committed)
//   PACK_WS  -> exchange -> UNPACK_WS   ghosts' W* (then their Z*)
//   STAGE2                              stage-2 triangles, owned W^{n+1},
//                                       step committed
//
// Ghost states are exact copies and a triangle computed by several parts
// sees identical inputs, so every part's owned vertices match the
// single-part step bitwise.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "rd_df64.h"
#include "rd_device.h"
#include "rd_internal.h"
#include "rd_kernels.cuh"

using namespace rd;

struct rd_part {
  rd_mesh* m = nullptr;
  rd_params p{};
  PartPlanHost plan;
  int pi = 0;
  size_t ts = 8;
  int32_t n_own = 0, n_gh = 0, nlt = 0, n_send = 0;
  DevBuf tri, ptr, ent, sidx, geo[6];  // geo: nx, ny, hl [3][nlt], area, lmax [nlt], V [n_local]
  DevBuf W[2], Z[2], spd[2], Ws, Zs, spds, R1, share, rec, cfl, partial, ctl, stage;
  DevBuf geo_df[4], dWdf;  // RD_DF64: double-float geometry of the local triangles, W* - W^n of the local vertices
  int a = 0;
  int tri_block = TRI_BLOCK, vtx_block = VTX_BLOCK;
};

namespace {

__global__ void k_part_begin(DevCtl* ctl) {
  if (ctl->status == 0) ctl->stop = 0;
  ctl->t_end = 0.0;
}

__global__ void k_part_commit(DevCtl* ctl) {
  if (ctl->stop) return;
  ctl->t += ctl->dt;
  ctl->steps += 1;
}

template <class T>
__global__ void k_pack(int n, const int* __restrict__ idx, const T* __restrict__ W, T* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  T w[4];
  load_vec4(W, __ldg(idx + k), w);
  st4(out + 4 * (size_t)k, w);
}

// caller order (double, component-major) -> local order in T
template <class T>
__global__ void k_part_in(int n, const int* __restrict__ cid, const double* __restrict__ Wc, int nv_all,
                          T* __restrict__ W, DevCtl* ctl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = __ldg(cid + i);
  T w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = (T)Wc[(size_t)k * nv_all + j];
  st4(W + 4 * (size_t)i, w);
}

template <class T>
__global__ void k_part_out(int n, const T* __restrict__ W, double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int k = 0; k < 4; ++k) out[(size_t)k * n + i] = (double)W[4 * (size_t)i + k];
}

// RD_DF64: W* - W^n of the ghost vertices as double-float pairs (the owned
// ones come from the stage-1 update).
__global__ void k_dw_split(int n, const double* __restrict__ Wn, const double* __restrict__ Ws,
                           float2* __restrict__ dw) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[4], b[4];
  load_vec4(Wn, i, a);
  load_vec4(Ws, i, b);
  dfloat d[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k] = dw::to_df(__dsub_rn(b[k], a[k]));
  float4* o = reinterpret_cast<float4*>(dw + 4 * (size_t)i);
  o[0] = make_float4(d[0].hi, d[0].lo, d[1].hi, d[1].lo);
  o[1] = make_float4(d[2].hi, d[2].lo, d[3].hi, d[3].lo);
}

template <class T>
int upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
  CK(dev_alloc(b, std::max<size_t>(v.size(), 1) * sizeof(T), st));
  if (!v.empty()) CU(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return RD_OK;
}

template <class T>
int part_alloc(rd_part* q, const double* Wc) {
  rd_mesh* m = q->m;
  const HostMesh& h = m->h;
  const PartPlanHost& pl = q->plan;
  cudaStream_t st = m->stream;
  const size_t nl = (size_t)q->n_own + q->n_gh, nlt = q->nlt;
  // connectivity, CSR and send list
  CK(upload(q->tri, pl.ltri, st));
  CK(upload(q->ptr, pl.csr_ptr, st));
  CK(upload(q->ent, pl.csr_ent, st));
  CK(upload(q->sidx, pl.send_idx, st));
  // geometry of the local triangles and volumes of the local vertices, copied
  // (not recomputed) from the mesh store so that they are bitwise the same
  std::vector<T> g3(3 * nlt), g1(nlt), gv(nl);
  const std::vector<double>* per3[3] = {&h.nx, &h.ny, &h.hl};
  for (int k = 0; k < 3; ++k) {
    for (int c = 0; c < 3; ++c)
      for (size_t j = 0; j < nlt; ++j) g3[c * nlt + j] = (T)(*per3[k])[(size_t)c * h.nt + pl.lt[j]];
    CK(upload(q->geo[k], g3, st));
  }
  for (size_t j = 0; j < nlt; ++j) g1[j] = (T)h.area[pl.lt[j]];
  CK(upload(q->geo[3], g1, st));
  for (size_t j = 0; j < nlt; ++j) g1[j] = (T)h.lmax[pl.lt[j]];
  CK(upload(q->geo[4], g1, st));
  for (size_t i = 0; i < nl; ++i) gv[i] = (T)h.V[pl.lv[i]];
  CK(upload(q->geo[5], gv, st));
  if (q->p.precision == RD_DF64) {
    const std::vector<double>* per[4] = {&h.nx, &h.ny, &h.hl, &h.area};
    for (int k = 0; k < 4; ++k) {
      const int ncomp = k < 3 ? 3 : 1;
      std::vector<double> loc((size_t)ncomp * nlt);
      for (int c = 0; c < ncomp; ++c)
        for (size_t j = 0; j < nlt; ++j) loc[c * nlt + j] = (*per[k])[(size_t)c * h.nt + pl.lt[j]];
      std::vector<float2> sp;
      split_df_host(loc, sp);
      CK(upload(q->geo_df[k], sp, st));
    }
    CK(dev_alloc(q->dWdf, 4 * nl * sizeof(float2), st));
  }
  const size_t ts = sizeof(T);
  for (int b = 0; b < 2; ++b) {
    CK(dev_alloc(q->W[b], 4 * nl * ts, st));
    CK(dev_alloc(q->Z[b], 4 * nl * ts, st));
    CK(dev_alloc(q->spd[b], nl * ts, st));
  }
  CK(dev_alloc(q->Ws, 4 * nl * ts, st));
  CK(dev_alloc(q->Zs, 4 * nl * ts, st));
  CK(dev_alloc(q->spds, std::max<size_t>(nl, 1) * ts, st));
  CK(dev_alloc(q->R1, 4 * std::max<size_t>(q->n_own, 1) * ts, st));
  CK(dev_alloc(q->share, 12 * nlt * ts, st));
  CK(dev_alloc(q->rec, 16 * nlt * ts, st));
  CK(dev_alloc(q->cfl, nlt * ts, st));
  CK(dev_alloc(q->partial, (size_t)nblk(std::max(q->n_own, 1), VTX_BLOCK_MIN) * ts, st));
  CK(dev_alloc(q->ctl, sizeof(DevCtl), st));
  CK(dev_alloc(q->stage, 4 * nl * sizeof(double), st));
  DevCtl c{};
  CU(cudaMemcpyAsync(q->ctl.p, &c, sizeof(DevCtl), cudaMemcpyHostToDevice, st));
  // initial state of the owned and ghost vertices from the caller's full state
  std::vector<int32_t> cid(nl);
  for (size_t i = 0; i < nl; ++i) cid[i] = h.vperm[pl.lv[i]];
  DevBuf dcid, dw;
  CK(upload(dcid, cid, st));
  CK(dev_alloc(dw, 4 * (size_t)h.nv * sizeof(double), st));
  CU(cudaMemcpyAsync(dw.p, Wc, 4 * (size_t)h.nv * sizeof(double), cudaMemcpyHostToDevice, st));
  DevCtl* ctl = (DevCtl*)q->ctl.p;
  k_part_in<T><<<nblk(nl, VTX_BLOCK), VTX_BLOCK, 0, st>>>((int)nl, (const int*)dcid.p, (const double*)dw.p, h.nv,
                                                          (T*)q->W[0].p, ctl);
  k_prepare<T><<<nblk(nl, VTX_BLOCK), VTX_BLOCK, 0, st>>>((int)nl, (const T*)q->W[0].p, (T)q->p.gamma,
                                                          (T*)q->Z[0].p, (T*)q->spd[0].p, ctl);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  dev_free(dcid);
  dev_free(dw);
  DevCtl c2;
  CU(cudaMemcpy(&c2, q->ctl.p, sizeof(DevCtl), cudaMemcpyDeviceToHost));
  return c2.status ? RD_ENONPHYSICAL : RD_OK;
}

template <class T>
BlendArgs<T> part_blend(const rd_part* q) {
  BlendArgs<T> ba;
  ba.mode = q->p.scheme == RD_BMAX2 ? BLEND_MAX : q->p.scheme == RD_BMIN2 ? BLEND_MIN : BLEND_B;
  ba.sl = q->p.lumping == RD_LUMP_SELECTIVE;
  return ba;
}

template <class T>
DevGeo<T> part_geo(const rd_part* q) {
  DevGeo<T> g;
  g.nx = (const T*)q->geo[0].p;
  g.ny = (const T*)q->geo[1].p;
  g.hl = (const T*)q->geo[2].p;
  g.area = (const T*)q->geo[3].p;
  g.lmax = (const T*)q->geo[4].p;
  return g;
}

DevGeoDF part_geo_df(const rd_part* q) {
  DevGeoDF g;
  g.nx = (const float2*)q->geo_df[0].p;
  g.ny = (const float2*)q->geo_df[1].p;
  g.hl = (const float2*)q->geo_df[2].p;
  g.area = (const float2*)q->geo_df[3].p;
  g.lmax = (const double*)q->geo[4].p;
  return g;
}

template <class T>
int part_phase(rd_part* q, int phase, void* buf) {
  cudaStream_t st = q->m->stream;
  const int a = q->a, b = 1 - a;
  const size_t off = 4 * (size_t)q->n_own;
  DevCtl* ctl = (DevCtl*)q->ctl.p;
  const T gamma = (T)q->p.gamma, eps = (T)q->p.eps_fix;
  const T* V = (const T*)q->geo[5].p;
  const int* tri = (const int*)q->tri.p;
  const int* ptr = (const int*)q->ptr.p;
  const int* ent = (const int*)q->ent.p;
  const int TB = q->tri_block, VB = q->vtx_block;
  const unsigned gt = nblk(std::max(q->nlt, 1), TB), gv = nblk(std::max(q->n_own, 1), VB);
  const bool df = sizeof(T) == 8 && q->p.precision == RD_DF64;
  DevGeo<T> g = part_geo<T>(q);
  BlendArgs<T> ba = part_blend<T>(q);
  const Gas<T> gas = Gas<T>::of(gamma);
  switch (phase) {
    case RD_PART_PACK_W:
    case RD_PART_PACK_WS: {
      if (q->n_send == 0) break;
      if (!buf) return RD_EINVAL;
      const T* src = (const T*)(phase == RD_PART_PACK_W ? q->W[a].p : q->Ws.p);
      k_pack<T><<<nblk(q->n_send, VTX_BLOCK), VTX_BLOCK, 0, st>>>(q->n_send, (const int*)q->sidx.p, src, (T*)buf);
      break;
    }
    case RD_PART_UNPACK_W:
    case RD_PART_UNPACK_WS: {
      if (q->n_gh == 0) break;
      if (!buf) return RD_EINVAL;
      const bool w = phase == RD_PART_UNPACK_W;
      T* dst = (T*)(w ? q->W[a].p : q->Ws.p) + off;
      CU(cudaMemcpyAsync(dst, buf, 4 * (size_t)q->n_gh * sizeof(T), cudaMemcpyDeviceToDevice, st));
      T* Zd = (T*)(w ? q->Z[a].p : q->Zs.p) + off;
      T* Sd = (T*)(w ? q->spd[a].p : q->spds.p) + q->n_own;
      k_prepare<T><<<nblk(q->n_gh, VTX_BLOCK), VTX_BLOCK, 0, st>>>(q->n_gh, dst, gamma, Zd, Sd, ctl);
      if constexpr (sizeof(T) == 8) {
        if (!w && df)
          k_dw_split<<<nblk(q->n_gh, VTX_BLOCK), VTX_BLOCK, 0, st>>>(q->n_gh, (const double*)q->W[a].p + off,
                                                                     (const double*)q->Ws.p + off,
                                                                     (float2*)q->dWdf.p + off);
      }
      break;
    }
    case RD_PART_STAGE1: {
      k_part_begin<<<1, 1, 0, st>>>(ctl);
      const T* Za = (const T*)q->Z[a].p;
      const T* Sa = (const T*)q->spd[a].p;
      T* share = (T*)q->share.p;
      T* rec = (T*)q->rec.p;
      T* cf = (T*)q->cfl.p;
      if (q->nlt > 0) {
        if (df) {
          if constexpr (sizeof(T) == 8) {
            TriArraysDF x;
            x.nt = q->nlt;
            x.tri = tri;
            x.g = part_geo_df(q);
            x.Z = Za;
            x.spd = Sa;
            x.share = share;
            x.rec = rec;
            x.cfl = cf;
            x.ctl = ctl;
            CK(launch_tri_stage1_df(q->p, x, ba, gt, TB, st));
          }
        } else if (q->p.scheme == RD_N1) {
          k_tri_stage1<T, RD_N1><<<gt, TB, 0, st>>>(q->nlt, 0, tri, g, Za, Sa, gas, eps, share, nullptr, cf, ctl);
        } else if (q->p.scheme == RD_LDA2) {
          k_tri_stage1<T, RD_LDA2><<<gt, TB, 0, st>>>(q->nlt, 0, tri, g, Za, Sa, gas, eps, share, rec, cf, ctl);
        } else if (q->p.scheme == RD_B2 && q->p.lumping == RD_LUMP_GLOBAL) {
          k_tri_stage1<T, RD_B2><<<gt, TB, 0, st>>>(q->nlt, 0, tri, g, Za, Sa, gas, eps, share, rec, cf, ctl);
        } else {
          k_tri_stage1<T, RD_BMAX2><<<gt, TB, 0, st>>>(q->nlt, 0, tri, g, Za, Sa, gas, eps, share, rec, cf, ctl,
                                                       ba);
        }
      }
      launch_gather_cfl<T>(VB, st, q->n_own, ptr, ent, share, cf, V, (T*)q->R1.p, (T*)q->partial.p,
                           (T)q->p.cfl, ctl);
      break;
    }
    case RD_PART_UPDATE1: {
      if (q->p.scheme == RD_N1) {
        k_update<T><<<gv, VB, 0, st>>>(q->n_own, (const T*)q->W[a].p, (const T*)q->R1.p, ptr, ent, nullptr, V, gamma,
                                       (T*)q->W[b].p, (T*)q->Z[b].p, (T*)q->spd[b].p, ctl);
        k_part_commit<<<1, 1, 0, st>>>(ctl);
        q->a = b;
      } else {
        k_update<T><<<gv, VB, 0, st>>>(q->n_own, (const T*)q->W[a].p, (const T*)q->R1.p, ptr, ent, nullptr, V, gamma,
                                       (T*)q->Ws.p, (T*)q->Zs.p, nullptr, ctl, nullptr, nullptr, nullptr,
                                       WallArgs<T>(), GhostArgs<T>(), df ? (float2*)q->dWdf.p : nullptr);
      }
      break;
    }
    case RD_PART_STAGE2: {
      if (q->p.scheme == RD_N1) return RD_EINVAL;
      T* share = (T*)q->share.p;
      if (q->nlt > 0) {
        if (df) {
          if constexpr (sizeof(T) == 8) {
            TriArraysDF x;
            x.nt = q->nlt;
            x.tri = tri;
            x.g = part_geo_df(q);
            x.Z = (const T*)q->Zs.p;
            x.dw = (const float2*)q->dWdf.p;
            x.share = share;
            x.rec = q->rec.p;
            x.ctl = ctl;
            CK(launch_tri_stage2_df(q->p, x, ba, gt, TB, st));
          }
        } else if (q->p.scheme == RD_LDA2) {
          k_tri_stage2<T, RD_LDA2><<<gt, TB, 0, st>>>(q->nlt, 0, tri, g, (const T*)q->Zs.p, (const T*)q->W[a].p,
                                                      (const T*)q->Ws.p, (const T*)q->rec.p, gas, eps, share, ctl,
                                                      nullptr, nullptr, ba);
        } else if (q->p.scheme == RD_B2 && q->p.lumping == RD_LUMP_GLOBAL) {
          k_tri_stage2<T, RD_B2><<<gt, TB, 0, st>>>(q->nlt, 0, tri, g, (const T*)q->Zs.p, (const T*)q->W[a].p,
                                                    (const T*)q->Ws.p, (const T*)q->rec.p, gas, eps, share, ctl);
        } else {
          k_tri_stage2<T, RD_BMAX2><<<gt, TB, 0, st>>>(q->nlt, 0, tri, g, (const T*)q->Zs.p, (const T*)q->W[a].p,
                                                       (const T*)q->Ws.p, (const T*)q->rec.p, gas, eps, share, ctl,
                                                       nullptr, nullptr, ba);
        }
      }
      k_update<T><<<gv, VB, 0, st>>>(q->n_own, (const T*)q->Ws.p, nullptr, ptr, ent, share, V, gamma, (T*)q->W[b].p,
                                     (T*)q->Z[b].p, (T*)q->spd[b].p, ctl);
      k_part_commit<<<1, 1, 0, st>>>(ctl);
      q->a = b;
      break;
    }
    default:
      return RD_EINVAL;
  }
  CU(cudaGetLastError());
  return RD_OK;
}

int read_ctl(const rd_part* q, DevCtl& c) {
  CU(cudaMemcpyAsync(&c, q->ctl.p, sizeof(DevCtl), cudaMemcpyDeviceToHost, q->m->stream));
  CU(cudaStreamSynchronize(q->m->stream));
  return RD_OK;
}

}  // namespace

extern "C" int rd_part_create(rd_mesh* m, int32_t n_parts, int32_t part, const double* W, const rd_params* p,
                              rd_part** out) {
  if (!m || !W || !p || !out) return RD_EINVAL;
  *out = nullptr;
  if (p->scheme < RD_N1 || p->scheme > RD_BX2 || p->reserved != 0) return RD_EINVAL;
  if (p->precision != RD_FP64 && p->precision != RD_FP32 && p->precision != RD_DF64) return RD_EINVAL;
  if (p->lumping != RD_LUMP_GLOBAL && p->lumping != RD_LUMP_SELECTIVE) return RD_EINVAL;
  if (p->lumping == RD_LUMP_SELECTIVE && p->scheme == RD_N1) return RD_EINVAL;
  if (!(p->cfl > 0.0) || !(p->gamma > 1.0) || !(p->eps_fix >= 0.0)) return RD_EINVAL;
  if (p->scheme == RD_BX2 || m->n_ghost || m->n_wall) return RD_ENOTSUP;
  rd_part* q = new (std::nothrow) rd_part();
  if (!q) return RD_ENOMEM;
  q->m = m;
  q->p = *p;
  q->pi = p->precision == RD_FP32 ? 1 : 0;
  q->ts = q->pi ? 4 : 8;
  int st = build_part_plan(m->h, n_parts, part, q->plan);
  if (st == RD_OK) {
    q->n_own = q->plan.v1 - q->plan.v0;
    q->n_gh = (int32_t)q->plan.lv.size() - q->n_own;
    q->nlt = (int32_t)q->plan.lt.size();
    q->n_send = (int32_t)q->plan.send_idx.size();
    st = q->pi ? part_alloc<float>(q, W) : part_alloc<double>(q, W);
  }
  if (st != RD_OK) {
    rd_part_destroy(q);
    return st;
  }
  *out = q;
  return RD_OK;
}

extern "C" void rd_part_destroy(rd_part* q) {
  if (!q) return;
  if (q->m && q->m->stream) cudaStreamSynchronize(q->m->stream);
  DevBuf* bufs[] = {&q->tri, &q->ptr, &q->ent, &q->sidx, &q->W[0], &q->W[1], &q->Z[0], &q->Z[1], &q->spd[0],
                    &q->spd[1], &q->Ws, &q->Zs, &q->spds, &q->R1, &q->share, &q->rec, &q->cfl, &q->partial,
                    &q->ctl, &q->stage};
  for (DevBuf* b : bufs) dev_free(*b);
  for (auto& g : q->geo) dev_free(g);
  for (auto& g : q->geo_df) dev_free(g);
  dev_free(q->dWdf);
  delete q;
}

extern "C" int rd_part_sizes(const rd_part* q, int32_t sizes[4]) {
  if (!q || !sizes) return RD_EINVAL;
  sizes[0] = q->n_own;
  sizes[1] = q->n_gh;
  sizes[2] = q->nlt;
  sizes[3] = q->n_send;
  return RD_OK;
}

extern "C" int rd_part_lists(const rd_part* q, int32_t* local_vertices, int32_t* send_ptr, int32_t* recv_ptr) {
  if (!q) return RD_EINVAL;
  const PartPlanHost& pl = q->plan;
  if (local_vertices)
    for (size_t i = 0; i < pl.lv.size(); ++i) local_vertices[i] = q->m->h.vperm[pl.lv[i]];
  if (send_ptr) std::copy(pl.send_ptr.begin(), pl.send_ptr.end(), send_ptr);
  if (recv_ptr) std::copy(pl.recv_ptr.begin(), pl.recv_ptr.end(), recv_ptr);
  return RD_OK;
}

extern "C" int rd_part_phase(rd_part* q, int32_t phase, void* buf) {
  if (!q) return RD_EINVAL;
  return q->pi ? part_phase<float>(q, phase, buf) : part_phase<double>(q, phase, buf);
}

extern "C" int rd_part_dt_device(rd_part* q, void** dt) {
  if (!q || !dt) return RD_EINVAL;
  *dt = (void*)&((DevCtl*)q->ctl.p)->dt;
  return RD_OK;
}

extern "C" int rd_part_get_dt(const rd_part* q, double* dt) {
  if (!q || !dt) return RD_EINVAL;
  DevCtl c;
  CK(read_ctl(q, c));
  *dt = c.dt;
  return RD_OK;
}

extern "C" int rd_part_set_dt(rd_part* q, double dt) {
  if (!q || !(dt > 0.0)) return RD_EINVAL;
  DevCtl* ctl = (DevCtl*)q->ctl.p;
  CU(cudaMemcpyAsync(&ctl->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, q->m->stream));
  CU(cudaStreamSynchronize(q->m->stream));
  return RD_OK;
}

extern "C" int rd_part_get_owned(const rd_part* q, double* W_out) {
  if (!q || !W_out) return RD_EINVAL;
  cudaStream_t st = q->m->stream;
  if (q->n_own > 0) {
    if (q->pi)
      k_part_out<float><<<nblk(q->n_own, VTX_BLOCK), VTX_BLOCK, 0, st>>>(q->n_own, (const float*)q->W[q->a].p,
                                                                        (double*)q->stage.p);
    else
      k_part_out<double><<<nblk(q->n_own, VTX_BLOCK), VTX_BLOCK, 0, st>>>(q->n_own, (const double*)q->W[q->a].p,
                                                                         (double*)q->stage.p);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(W_out, q->stage.p, 4 * (size_t)q->n_own * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CU(cudaStreamSynchronize(st));
  return RD_OK;
}

extern "C" int rd_part_status(const rd_part* q, double* t, int64_t* steps) {
  if (!q) return RD_EINVAL;
  DevCtl c;
  CK(read_ctl(q, c));
  if (t) *t = c.t;
  if (steps) *steps = c.steps;
  return c.status ? RD_ENONPHYSICAL : RD_OK;
}
