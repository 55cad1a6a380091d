// Rows a2 + a3 (+ a6), mixed-precision form: the CN mover with cell-crossing
// sub-steps and the charge-conserving deposit of Eqs. 3-4 on the FP32 particle
// store (28 bytes read per push).  The fast kernel streams the store and
// finishes the particles that stay in their cell; it queues the rest with
// their start state, z-face crossers apart from the others; the general
// kernel takes them in warps of one kind; crossers next to the axis go on to
// FP64 arithmetic (below).  The deposit is summed in FP32 over runs of at most
// 32 lanes, converted exactly to FP64 with integer operations and added with
// FP64 atomics (executed in L2), so the kernels issue no FP64 arithmetic and
// the Picard residual can still reach 1e-8.  Compiled with fast FP32
// reciprocals (push_kernels.cuh holds the first two kernels).
#include "push_kernels.cuh"

namespace pic {
namespace {

// the listed near-axis crossers of one FP32 pass in FP64 arithmetic: state
// and accelerations read from the FP32 store, every sub-step solved in
// double, the end state rounded to FP32 once
__global__ void __launch_bounds__(32) k_push_promoted32(PushLaunchT<float> L) {
  const int lane = threadIdx.x & 31;
  const long long cnt = *L.pcnt;
  GenArgs<double, float> G;
  G.nr = L.g.nr; G.nz = L.g.nz; G.ar = L.ar; G.az = L.az;
  G.wt = 0.0; G.icr = L.icr64; G.icz = L.icz64; G.cz = L.cz64; G.rm = L.rm64;
  G.q = L.q; G.m = L.m; G.qf = L.q; G.ir = L.ir; G.iz = L.iz; G.write = L.write; G.p = L.p;
  G.oop = L.oop; G.dst = L.dst; G.hist = L.hist;
  G.wall_z0 = L.wall_z0; G.wall_zl = L.wall_zl; G.wall_r = L.wall_r; G.ke_lost = L.ke_lost;
  Tally tl = {0, 0, 0, 0, 0, 0, 0};
  // consecutive entries go to different blocks (the list is short: this
  // spreads it over the SMs)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = blockIdx.x + (long long)threadIdx.x * gridDim.x; k < cnt; k += stride) {
    const long long p = L.plist[k];
    push_general<double, false, float>(G, p, L.p.cell[p], (double)L.p.a[p], (double)L.p.b[p],
                                       (double)L.p.vr[p], (double)L.p.vt[p], (double)L.p.vz[p],
                                       (double)L.p.w[p], (double)NAN, (double)NAN, tl);
  }
  flush_tally(L.counters, tl, lane, 0, 0);
}

}  // namespace

template cudaError_t launch_push<float>(const PushLaunchT<float> &L, cudaStream_t s);
template void push_shape<float>(PushLaunchT<float> &L, int *nfast, int *ngen);
template cudaError_t launch_push_multi<float>(const PushLaunchT<float> *Ls, const int *first, int nl,
                                               cudaStream_t s);

cudaError_t launch_push_fp32_axis(const PushLaunchT<float> &L, cudaStream_t s) {
  const long long nsz = L.n_dev ? L.cap : L.n;
  if (nsz <= 0 || !L.pcnt || L.wbt != 0.f) return cudaSuccess;
  k_push_promoted32<<<152, 32, 0, s>>>(L);
  return cudaGetLastError();
}

int push_wave_fp32(int general) {
  return (int)(general ? general_grid<float>() : fast_grid<float>());
}
}  // namespace pic
