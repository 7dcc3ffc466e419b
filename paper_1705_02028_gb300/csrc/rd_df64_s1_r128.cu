// RD_DF64 stage-1 triangle kernels at 128 registers per thread, without and
// with phase barriers (one translation unit per stage and budget).
#include "rd_df64_kernels.cuh"

RD_DF64_INSTANTIATE(1, 128, false)
RD_DF64_INSTANTIATE(1, 128, true)
