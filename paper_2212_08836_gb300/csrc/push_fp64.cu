// Rows a2 + a3 (+ a6), plain FP64 form: the Crank-Nicolson mover of Eq. 4 with
// cell-crossing sub-steps fused with the charge-conserving deposit of Eq. 3,
// on the FP64 particle store (52 bytes read per push).  GB300 runs FP64 on a
// narrow pipe, so this form is bound by FP64 issue rather than by HBM; the
// kernels (push_kernels.cuh) keep the FP64 operations per push low.
#include "push_kernels.cuh"

namespace pic {
template cudaError_t launch_push<double>(const PushLaunchT<double> &L, cudaStream_t s);
template void push_shape<double>(PushLaunchT<double> &L, int *nfast, int *ngen);
template cudaError_t launch_push_multi<double>(const PushLaunchT<double> *Ls, const int *first, int nl,
                                               cudaStream_t s);
int push_wave_fp64(int general) {
  return (int)(general ? general_grid<double>() : fast_grid<double>());
}
}  // namespace pic
