// Rows a2 + a3 (+ a6), mixed-precision form: the CN mover with cell-crossing
// sub-steps and the charge-conserving deposit of Eqs. 3-4 on the FP32 particle
// store (28 bytes read per push).  The deposit is summed in FP32 over runs of
// at most 32 lanes, converted exactly to FP64 with integer operations and
// added with FP64 atomics (executed in L2), so the kernel issues no FP64
// arithmetic and the Picard residual can still reach 1e-8.  Compiled with
// fast FP32 reciprocals (push_kernels.cuh holds the kernels).
#include "push_kernels.cuh"

namespace pic {
template cudaError_t launch_push<float>(const PushLaunchT<float> &L, cudaStream_t s);
int push_wave_fp32(int general) {
  return (int)(general ? general_grid<float>() : fast_grid<float>());
}
}  // namespace pic
