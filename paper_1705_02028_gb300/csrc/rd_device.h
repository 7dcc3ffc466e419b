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

}  // namespace rd

// The mesh handle: host mesh store plus its device arrays.
struct rd_mesh {
  rd::HostMesh h;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  rd::DevBuf tri, ptr, ent, vperm;
  // geometry per precision (0: double, 1: float): nx, ny, hl, area, lmax, V
  rd::DevBuf geo[2][6];
  bool geo_ready[2] = {false, false};
};
