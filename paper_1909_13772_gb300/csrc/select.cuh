// select.cuh -- compile-time (stencil, storage) selection for the per-variant objects.
// Build with -DLBM_Q=19|27 and -DLBM_ST=0 (fp64) | 1 (fp32) | 2 (bf16 deviation) | 3 (fp16 deviation).
#pragma once

#include "launch.hpp"

#ifndef LBM_Q
#define LBM_Q 19
#endif
#ifndef LBM_ST
#define LBM_ST 1
#endif
// -DLBM_MRT_SWEEP=1: the sweep object of the MRT collision (launch_sweep_mrt_<Q>_<ST>)
#ifndef LBM_MRT_SWEEP
#define LBM_MRT_SWEEP 0
#endif
// -DLBM_CUMULANT_SWEEP=1: the sweep object of the cumulant collision (D3Q27,
// launch_sweep_cum_27_<ST>)
#ifndef LBM_CUMULANT_SWEEP
#define LBM_CUMULANT_SWEEP 0
#endif

namespace lbm {
#if LBM_ST == 0
using StoreT = double;
#elif LBM_ST == 1
using StoreT = float;
#elif LBM_ST == 2
using StoreT = __nv_bfloat16;
#else
using StoreT = __half;
#endif
}  // namespace lbm

#define LBM_CAT2(a, b, c) a##b##_##c
#define LBM_CAT(a, b, c) LBM_CAT2(a, b, c)
