// closure.hpp -- host interface of the closure sweep (closure.cu): the network's device form
// and the launch arguments.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "launch.hpp"

namespace lbm {

// The network in the form the tensor-core inference reads (staged in shared memory once per
// CTA): weights in BF16, W1 padded to 16 inputs, w3 as row 0 of an 8-row block (the other
// rows zero) so the output layer is one more MMA; biases and scales in FP32.  W1, b1, W2, b2
// are stored halved (the SiLU is evaluated from z/2).
struct MlpDev {
    __nv_bfloat16 w1[32][16];
    __nv_bfloat16 w2[32][32];
    __nv_bfloat16 w3[8][32];
    float b1[32], b2[32];
    float b3, s_rho, s_pi, s_tau;
};
static_assert(sizeof(MlpDev) % 4 == 0, "MlpDev is copied in 4-byte words");

// Closure kinds (include/lbm.h: LBM_CLOSURE_*).
enum ClosureKind { CLOSURE_NONE = 0, CLOSURE_SMAGORINSKY = 1, CLOSURE_MLP = 2 };

struct ClosureLaunch {
    SweepArgs sw;       // as for the plain sweep (D3Q19, FP32 storage, no body force)
    int closure;        // ClosureKind (1 or 2)
    int trt;            // 1: omega- from Lambda; 0: SRT (omega- = omega+)
    float tau0, cs, lambda;
    const MlpDev *mlp;  // device copy (CLOSURE_MLP)
    int *err;           // device flag: a bounded wait of the tensor-core network gave up
};

// Packed FP32 parameters (1348 values) -> device form.
MlpDev mlp_device_form(const float *packed);

// Sweep with per-cell omega+ from the closure.  cudaErrorNotSupported for launches the
// closure sweep does not cover (body force, general neighbour tables, > 256 threads).
cudaError_t launch_closure_sweep(const ClosureLaunch &s);

}  // namespace lbm
