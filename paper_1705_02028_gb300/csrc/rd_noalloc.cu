// rd_noalloc.cu -- allocation-free variant of the CFL time step.
//
// rd_cfl_dt obtains its reduction scratch from the installed device allocator.
// rd_cfl_dt_noalloc computes the same time step with the same kernel but takes
// its scratch from the fixed array below, which is part of the library image:
// every device that loads the library holds it (512 KiB + 8 B) until the
// process exits, and the call allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "rd_internal.h"

namespace {

// One block minimum per 256 vertices: 65536 blocks cover 16,777,216 vertices
// (the 4096 x 4096 mesh).
constexpr int kMaxBlocks = 65536;
constexpr int64_t kMaxVertices = (int64_t)kMaxBlocks * rd::CFL_DT_BLOCK;

struct NoAllocScratch {
  double partial[kMaxBlocks];
  rd::DtScratchCtl ctl;
};

static __device__ __align__(256) NoAllocScratch g_scratch;

// Device address of g_scratch per device, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not an address).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoAllocScratch* g_addr[kMaxDevices] = {};

int scratch_on_current_device(NoAllocScratch** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return RD_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return RD_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return RD_ECUDA;
    }
    g_addr[dev] = (NoAllocScratch*)p;
  }
  *out = g_addr[dev];
  return RD_OK;
}

}  // namespace

extern "C" int rd_cfl_dt_noalloc(int32_t n_vertex, int32_t n_tri, int32_t precision, const void* W,
                                 const int32_t* tri, const void* lmax, const void* V, const int32_t* csr_ptr,
                                 const int32_t* csr_ent, double gamma, double cfl, double* dt_out,
                                 void* cuda_stream) {
  if ((int64_t)n_vertex > kMaxVertices) return RD_EINVAL;
  int rc = rd::cfl_dt_check(n_vertex, n_tri, precision, W, tri, lmax, V, csr_ptr, csr_ent, gamma, cfl, dt_out);
  if (rc != RD_OK) return rc;
  NoAllocScratch* s = nullptr;
  rc = scratch_on_current_device(&s);
  if (rc != RD_OK) return rc;
  // cfl_dt_launch clears the control word before the kernel; the block minima
  // are overwritten by every call.
  return rd::cfl_dt_launch(n_vertex, n_tri, precision, W, tri, lmax, V, csr_ptr, csr_ent, gamma, cfl, dt_out,
                           cuda_stream, s->partial, &s->ctl);
}
