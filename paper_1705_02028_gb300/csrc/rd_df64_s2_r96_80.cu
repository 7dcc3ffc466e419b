// RD_DF64 stage-2 triangle kernels at 96 and 80 registers per thread, with
// phase barriers (more resident warps than at 128, more spills).
#include "rd_df64_kernels.cuh"

RD_DF64_INSTANTIATE(2, 96, true)
RD_DF64_INSTANTIATE(2, 80, true)
