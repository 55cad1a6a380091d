// Rows a2 + a3 (+ a6), mixed-precision form: the CN mover with cell-crossing
// sub-steps and the charge-conserving deposit of Eqs. 3-4 on the FP32 particle
// store (28 bytes read per push), as one streaming kernel per species and pass
// (push_tile.cuh).  The deposit is summed in FP32 over runs of at most 32
// lanes, converted exactly to FP64 with integer operations and added with
// FP64 atomics (executed in L2), so the kernel issues no FP64 arithmetic and
// the Picard residual can still reach 1e-8.  Compiled with fast FP32
// reciprocals.  With an external B_z every particle takes the general path.
#include "push_tile.cuh"

namespace pic {
template <>
cudaError_t launch_push<float>(const PushLaunchT<float> &L, cudaStream_t s) {
  if (L.wbt == 0.f) return launch_push_tile32(L, s);
  return launch_push_all<float>(L, s);
}
cudaError_t launch_push_fp32_axis(const PushLaunchT<float> &L, cudaStream_t s) {
  if (L.wbt != 0.f) return cudaSuccess;
  return launch_push_promoted32(L, s);
}
int push_wave_fp32(int general) {
  (void)general;
  return tile_grid32();
}
}  // namespace pic
