// Picard start of a step (Sec. 2.1 leaves it open): inputs of the learned
// guess, the quadratic extrapolation G = 3E^n - 3E^{n-1} + E^{n-2}, the start
// E^{n+1,0} = G + s_d * y (y = network output, or none), and the training
// target (E^{n+1} - G) / s_d.  The padded grid is (nr+1) x (nz+1): E_r on
// rows < nr, E_z on columns < nz, H_theta on both; NCHW FP32 tensors.
#include "pic_internal.cuh"

namespace pic {
namespace {

__device__ __forceinline__ void block_add4(double a, double b, double c, double d, double *out) {
  __shared__ double s[4][32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s[0][w] = a;
    s[1][w] = b;
    s[2][w] = c;
    s[3][w] = d;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += s[threadIdx.x][k];
    if (v != 0.0) atomicAdd(&out[threadIdx.x], v);
  }
}

// sums[0..3] += sum (E^n - E^{n-1})^2, sum (E^n)^2, sum H^2, sum J^2
__global__ void __launch_bounds__(256) k_guess_sums(GuessArgs A) {
  const long long ner = (long long)A.nr * (A.nz + 1), nez = (long long)(A.nr + 1) * A.nz;
  const long long nh = (long long)A.nr * A.nz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (t < ner) {
    double d = A.e[0].r[t] - A.e[1].r[t];
    s0 += d * d;
    s1 += A.e[0].r[t] * A.e[0].r[t];
    s3 += A.jr[t] * A.jr[t];
  }
  if (t < nez) {
    double d = A.e[0].z[t] - A.e[1].z[t];
    s0 += d * d;
    s1 += A.e[0].z[t] * A.e[0].z[t];
    s3 += A.jz[t] * A.jz[t];
  }
  if (t < nh) s2 += A.h[t] * A.h[t];
  block_add4(s0, s1, s2, s3, A.sums);
}

// the 14 input channels at padded point (i, j), G, and s_d
__global__ void __launch_bounds__(256) k_guess_features(GuessArgs A) {
  const int nr = A.nr, nz = A.nz, W = nz + 1;
  const long long P = (long long)(nr + 1) * W;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double ne = (double)nr * (nz + 1) + (double)(nr + 1) * nz;
  const double sd = sqrt(A.sums[0] / ne) + 1e-30, se = sqrt(A.sums[1] / ne) + 1e-30;
  const double sh = sqrt(A.sums[2] / ((double)nr * nz)) + 1e-30, sj = sqrt(A.sums[3] / ne) + 1e-30;
  if (t == 0) *A.sd = sd;
  if (t >= P) return;
  const int i = (int)(t / W), j = (int)(t - (long long)(t / W) * W);
  const bool vr = i < nr, vz = j < nz;
  const long long kr = (long long)i * (nz + 1) + j, kz = (long long)i * nz + j;
  float *x = A.x;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    x[(2 * k) * P + t] = vr ? (float)((A.e[k].r[kr] - A.e[k + 1].r[kr]) / sd) : 0.f;
    x[(2 * k + 1) * P + t] = vz ? (float)((A.e[k].z[kz] - A.e[k + 1].z[kz]) / sd) : 0.f;
  }
  x[6 * P + t] = vr ? (float)(A.e[0].r[kr] / se) : 0.f;
  x[7 * P + t] = vz ? (float)(A.e[0].z[kz] / se) : 0.f;
  x[8 * P + t] = (vr && vz) ? (float)(A.h[kz] / sh) : 0.f;
  x[9 * P + t] = vr ? (float)(A.jr[kr] / sj) : 0.f;
  x[10 * P + t] = vz ? (float)(A.jz[kz] / sj) : 0.f;
  x[11 * P + t] = vr ? 1.f : 0.f;
  x[12 * P + t] = vz ? 1.f : 0.f;
  x[13 * P + t] = (float)((double)i / nr);
  if (vr) A.ger[kr] = 3.0 * A.e[0].r[kr] - 3.0 * A.e[1].r[kr] + A.e[2].r[kr];
  if (vz) A.gez[kz] = 3.0 * A.e[0].z[kz] - 3.0 * A.e[1].z[kz] + A.e[2].z[kz];
}

// start = G + s_d * y (y position-major [P][cp], channel 0 = E_r, 1 = E_z; or
// none), PEC values on z = 0, L, the drive value on r = R; *bad = 1 if not finite
__global__ void __launch_bounds__(256) k_guess_apply(GuessArgs A, const float *y, int cp,
                                                     double ez_edge, double *er1, double *ez1,
                                                     int *bad) {
  const int nr = A.nr, nz = A.nz, W = nz + 1;
  const long long P = (long long)(nr + 1) * W;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const int i = (int)(t / W), j = (int)(t - (long long)(t / W) * W);
  const double sd = *A.sd;
  if (i < nr) {
    const long long k = (long long)i * (nz + 1) + j;
    double v = (j == 0 || j == nz) ? 0.0 : A.ger[k] + (y ? sd * (double)y[t * cp] : 0.0);
    if (!isfinite(v)) *bad = 1;
    er1[k] = v;
  }
  if (j < nz) {
    const long long k = (long long)i * nz + j;
    double v = i == nr ? ez_edge : A.gez[k] + (y ? sd * (double)y[t * cp + 1] : 0.0);
    if (!isfinite(v)) *bad = 1;
    ez1[k] = v;
  }
}

// training target (E^{n+1} - G) / s_d, zero at the padding points
__global__ void __launch_bounds__(256) k_guess_target(GuessArgs A, const double *er_next,
                                                      const double *ez_next, float *tg) {
  const int nr = A.nr, nz = A.nz, W = nz + 1;
  const long long P = (long long)(nr + 1) * W;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const int i = (int)(t / W), j = (int)(t - (long long)(t / W) * W);
  const double sd = *A.sd;
  const long long kr = (long long)i * (nz + 1) + j, kz = (long long)i * nz + j;
  tg[t] = i < nr ? (float)((er_next[kr] - A.ger[kr]) / sd) : 0.f;
  tg[P + t] = j < nz ? (float)((ez_next[kz] - A.gez[kz]) / sd) : 0.f;
}

}  // namespace

cudaError_t launch_guess_inputs(const GuessArgs &A, cudaStream_t s) {
  const long long ner = (long long)A.nr * (A.nz + 1), nez = (long long)(A.nr + 1) * A.nz;
  long long n = ner > nez ? ner : nez;
  cudaError_t e = cudaMemsetAsync(A.sums, 0, 4 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_guess_sums<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A);
  const long long P = (long long)(A.nr + 1) * (A.nz + 1);
  k_guess_features<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_guess_apply(const GuessArgs &A, const float *y, int cp, double ez_edge,
                               double *er1, double *ez1, int *bad, cudaStream_t s) {
  const long long P = (long long)(A.nr + 1) * (A.nz + 1);
  k_guess_apply<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(A, y, cp, ez_edge, er1, ez1, bad);
  return cudaGetLastError();
}

cudaError_t launch_guess_target(const GuessArgs &A, const double *er_next, const double *ez_next,
                                float *tg, cudaStream_t s) {
  const long long P = (long long)(A.nr + 1) * (A.nz + 1);
  k_guess_target<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(A, er_next, ez_next, tg);
  return cudaGetLastError();
}

}  // namespace pic
