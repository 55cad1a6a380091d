// Row a1: pair loading (uniform in the logical coordinates, weight
// proportional to r*J_r as in Sec. 2.1, Maxwellian velocities) and row a9:
// FP64 conservation diagnostics (kinetic and field energy, node charge).
#include "pic_internal.cuh"

namespace pic {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_load(Grid g, long long n, double n0, double vthe,
                                              double vthi, uint64_t seed, PartsT<T> e,
                                              PartsT<T> i) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double u[4];
  draw4(seed, kStreamLoadPos, (uint64_t)p, kLoadStep, 0, u);
  double xi = (double)g.nr * u[0];
  double eta = (double)g.nz * u[1];
  int ic = (int)floor(xi), jc = (int)floor(eta);
  if (ic > g.nr - 1) ic = g.nr - 1;
  if (jc > g.nz - 1) jc = g.nz - 1;
  int32_t cell = ic * g.nz + jc;
  double a = xi - (double)ic, b = eta - (double)jc;
  double w;
  if (g.xa == 0 && g.nd == 0) {
    w = n0 * (kTwoPi * (xi * g.dr)) * g.R * g.L / (double)n;
  } else {  // mapped mesh: w proportional to r J_r, J_r the cell width
    const double jr = g_width(g, ic);
    const double r = (g_rho0(g, ic) + a) * jr;
    w = n0 * (kTwoPi * r) * (jr * (double)g.nr) * g.L / (double)n;
  }
  e.cell[p] = cell; e.a[p] = (T)a; e.b[p] = (T)b; e.w[p] = (T)w; e.id[p] = (uint32_t)p;
  i.cell[p] = cell; i.a[p] = (T)a; i.b[p] = (T)b; i.w[p] = (T)w; i.id[p] = (uint32_t)p;
  double g1, g2, g3, g4;
  draw4(seed, kStreamLoadVe, (uint64_t)p, kLoadStep, 0, u);
  gauss2(u[0], u[1], g1, g2);
  gauss2(u[2], u[3], g3, g4);
  e.vr[p] = (T)(vthe * g1); e.vt[p] = (T)(vthe * g2); e.vz[p] = (T)(vthe * g3);
  draw4(seed, kStreamLoadVi, (uint64_t)p, kLoadStep, 0, u);
  gauss2(u[0], u[1], g1, g2);
  gauss2(u[2], u[3], g3, g4);
  i.vr[p] = (T)(vthi * g1); i.vt[p] = (T)(vthi * g2); i.vz[p] = (T)(vthi * g3);
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block reduction of two doubles into out[0], out[1] (atomics)
__device__ void block_add2(double x, double y, double *out) {
  __shared__ double s[2][32];
  x = wsum(x);
  y = wsum(y);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { s[0][w] = x; s[1][w] = y; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += s[0][k]; b += s[1][k]; }
    atomicAdd(&out[0], a);
    atomicAdd(&out[1], b);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_kinetic(PartsT<T> p, long long n, double m, double q,
                                                 double *out2) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double k = 0.0, c = 0.0;
  if (t < n && p.cell[t] >= 0) {
    double vr = (double)p.vr[t], vt = (double)p.vt[t], vz = (double)p.vz[t], w = (double)p.w[t];
    k = 0.5 * m * w * (vr * vr + vt * vt + vz * vz);
    c = q * w;
  }
  block_add2(k, c, out2);
}

__global__ void __launch_bounds__(256) k_field_energy(Grid g, double eps, double mu,
                                                      const double *er, const double *ez,
                                                      const double *h, double *out) {
  int nr = g.nr, nz = g.nz, nz1 = nz + 1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long ner = (long long)nr * nz1, nez = (long long)(nr + 1) * nz, nh = (long long)nr * nz;
  double W = 0.0;
  double dz = g.dz;
  if (t < ner) {
    int i = (int)(t / nz1), j = (int)(t - (t / nz1) * nz1);
    if (j != 0 && j != nz) {
      double e = er[t];
      W += 0.5 * eps * e * e * g_aeff_r(g, i) * g_width(g, i);
    }
  }
  if (t < nez) {
    int i = (int)(t / nz);
    if (i < nr) {
      double e = ez[t];
      W += 0.5 * eps * e * e * g_aeff_z(g, i) * dz;
    }
  }
  if (t < nh) {
    int i = (int)(t / nz);
    double hh = h[t];
    W += 0.5 * mu * hh * hh * (kTwoPi * g_rcentre(g, i) * g_width(g, i) * dz);
  }
  block_add2(W, 0.0, out);
}

template <typename T>
__global__ void __launch_bounds__(256) k_node_charge(Grid g, PartsT<T> p, long long n, double q,
                                                     double *Q) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int c = p.cell[t];
  if (c < 0) return;
  int nz = g.nz, nz1 = nz + 1;
  int ic = c / nz, jc = c - (c / nz) * nz;
  double a = (double)p.a[t], b = (double)p.b[t], qw = q * (double)p.w[t];
  atomicAdd(&Q[ic * nz1 + jc], qw * (1.0 - a) * (1.0 - b));
  atomicAdd(&Q[(ic + 1) * nz1 + jc], qw * a * (1.0 - b));
  atomicAdd(&Q[ic * nz1 + jc + 1], qw * (1.0 - a) * b);
  atomicAdd(&Q[(ic + 1) * nz1 + jc + 1], qw * a * b);
}

// Gauss residual eps div_h E - Q on the interior nodes (i < nr, 0 < j < nz),
// in the flux form of the integral mesh; zero elsewhere.  Q holds the node
// charge on entry and the residual on exit.
__global__ void __launch_bounds__(256) k_gauss_residual(Grid g, double eps, const double *er,
                                                        const double *ez, const double *wall,
                                                        const double *qc, double *Q) {
  const int nz = g.nz, nz1 = nz + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)(g.nr + 1) * nz1) return;
  const int i = (int)(t / nz1), j = (int)(t - (t / nz1) * nz1);
  if (i >= g.nr || j == 0 || j == nz) {
    Q[t] = 0.0;
    return;
  }
  if (g.nd > 0 && i == g.nr - g.nd && wall) {
    // the charge stuck on the dielectric ring's face (the r-wall tallies)
    const int blk = 2 * (g.nr + 1) + nz1;
    Q[t] += wall[2 * (g.nr + 1) + j] + wall[blk + 2 * (g.nr + 1) + j];
  }
  if (qc) Q[t] += qc[t];
  double flux = g_aeff_r(g, i) * er[i * nz1 + j];
  if (i >= 1) flux -= g_aeff_r(g, i - 1) * er[(i - 1) * nz1 + j];
  flux += g_aeff_z(g, i) * (ez[i * nz + j] - ez[i * nz + j - 1]);
  Q[t] = eps * flux - Q[t];
}

// Fourier-Bessel coefficients (App. A, Eq. A2): block m sums basis row m
// against the field samples f[k * stride], k < n, in a fixed order
__global__ void __launch_bounds__(128) k_fourier_bessel(const double *__restrict__ basis,
                                                        const double *__restrict__ f,
                                                        int stride, int n,
                                                        double *__restrict__ coef) {
  const int m = blockIdx.x;
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    v += basis[(size_t)m * n + k] * f[(size_t)k * stride];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double red[4];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) coef[m] = (red[0] + red[1]) + (red[2] + red[3]);
}

}  // namespace

cudaError_t launch_gauss_residual(const Grid &g, double eps, const double *er, const double *ez,
                                  const double *wall, const double *qc, double *Q, cudaStream_t s) {
  const long long n = (long long)(g.nr + 1) * (g.nz + 1);
  k_gauss_residual<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, eps, er, ez, wall, qc, Q);
  return cudaGetLastError();
}

// Conduction tally of a conducting ring: node (i, j) loses dt S E^{n+1/2} through
// each unknown edge that starts at it and gains it through each that ends at it
__global__ void __launch_bounds__(256) k_conduction(Grid g, double dt, const double *er0,
                                                    const double *ez0, const double *er1,
                                                    const double *ez1, double *qc) {
  const int nr = g.nr, nz = g.nz, nz1 = nz + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)(nr + 1) * nz1) return;
  const int i = (int)(t / nz1), j = (int)(t - (t / nz1) * nz1);
  const double h = 0.5 * dt;
  double d = 0.0;
  if (j >= 1 && j <= nz - 1) {
    if (i < nr) d -= h * g_asig_r(g, i) * (er0[i * nz1 + j] + er1[i * nz1 + j]);
    if (i >= 1) d += h * g_asig_r(g, i - 1) * (er0[(i - 1) * nz1 + j] + er1[(i - 1) * nz1 + j]);
  }
  if (i < nr) {
    const double sz = h * g_asig_z(g, i);
    if (j < nz) d -= sz * (ez0[i * nz + j] + ez1[i * nz + j]);
    if (j >= 1) d += sz * (ez0[i * nz + j - 1] + ez1[i * nz + j - 1]);
  }
  qc[t] += d;
}

cudaError_t launch_conduction(const Grid &g, double dt, const double *er0, const double *ez0,
                              const double *er1, const double *ez1, double *qc, cudaStream_t s) {
  const long long n = (long long)(g.nr + 1) * (g.nz + 1);
  k_conduction<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, dt, er0, ez0, er1, ez1, qc);
  return cudaGetLastError();
}

cudaError_t launch_fourier_bessel(const double *basis, const double *f, int stride, int n,
                                  int nmodes, double *coef, cudaStream_t s) {
  k_fourier_bessel<<<nmodes, 128, 0, s>>>(basis, f, stride, n, coef);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_load(const Grid &g, long long n, double n0, double te_ev, double ti_ev,
                        uint64_t seed, PartsT<T> e, PartsT<T> i, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  double vthe = sqrt(te_ev * kQE / kME), vthi = sqrt(ti_ev * kQE / kMAr);
  k_load<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, n, n0, vthe, vthi, seed, e, i);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kinetic(const PartsT<T> &p, long long n, double m, double q, double *out2,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_kinetic<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, m, q, out2);
  return cudaGetLastError();
}

cudaError_t launch_field_energy(const Grid &g, double eps, double mu, const double *er,
                                const double *ez, const double *h, double *out, cudaStream_t s) {
  long long n = (long long)(g.nr + 1) * (g.nz + 1);
  k_field_energy<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, eps, mu, er, ez, h, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_node_charge(const Grid &g, const PartsT<T> &p, long long n, double q,
                               double *Q, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_node_charge<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, p, n, q, Q);
  return cudaGetLastError();
}

#define PIC_INST(T)                                                                            \
  template cudaError_t launch_load<T>(const Grid &, long long, double, double, double,          \
                                      uint64_t, PartsT<T>, PartsT<T>, cudaStream_t);            \
  template cudaError_t launch_kinetic<T>(const PartsT<T> &, long long, double, double,          \
                                         double *, cudaStream_t);                                \
  template cudaError_t launch_node_charge<T>(const Grid &, const PartsT<T> &, long long,        \
                                             double, double *, cudaStream_t);
PIC_INST(double)
PIC_INST(float)
#undef PIC_INST

}  // namespace pic

// ---------------------------------------------------------------------------
// self-check of the integer-pipe binary64 multiply (pic_check_dmul)
#include "swfp.cuh"
namespace pic {
namespace {
__global__ void __launch_bounds__(256) k_check_dmul(const double *x, const double *y, double *o,
                                                    long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    o[i] = sw_dmul(x[i], y[i]);
}
}  // namespace
}  // namespace pic

extern "C" int pic_check_dmul(const double *x, const double *y, double *out, long long n,
                              void *stream) {
  if (n < 0 || (n > 0 && (!x || !y || !out))) return PIC_E_CONFIG;
  if (n == 0) return PIC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const long long nb = (n + 255) / 256;
  pic::k_check_dmul<<<(unsigned)(nb < 152 * 16 ? nb : 152 * 16), 256, 0, s>>>(x, y, out, n);
  if (cudaGetLastError() != cudaSuccess) return PIC_E_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : PIC_E_CUDA;
}

// ---------------------------------------------------------------------------
// throughput probe of the FP64 FMA pipe (pic_probe_dfma): every thread runs
// eight independent chains of fused multiply-adds, so the pipe, not their
// latency, sets the rate
namespace pic {
namespace {
__device__ double g_dfma_sink;
__global__ void __launch_bounds__(256) k_dfma_probe(int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const double s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == 1.2345678e300) g_dfma_sink = s;  // keeps the chains live, never taken
}
}  // namespace
}  // namespace pic

extern "C" int pic_probe_dfma(int blocks_per_sm, int iters, double *seconds, double *tflops) {
  if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || !seconds || !tflops)
    return PIC_E_CONFIG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PIC_E_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PIC_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PIC_E_CUDA;
  }
  const unsigned nb = (unsigned)(nsm * blocks_per_sm);
  // a near-one multiplier keeps the values finite over any number of steps
  pic::k_dfma_probe<<<nb, 256>>>(iters, 0.9999999, 1e-7);  // warm-up
  cudaEventRecord(e0);
  pic::k_dfma_probe<<<nb, 256>>>(iters, 0.9999999, 1e-7);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return PIC_E_CUDA;
  *seconds = ms * 1e-3;
  *tflops = 2.0 * 8.0 * (double)iters * 256.0 * (double)nb / (*seconds) / 1e12;
  return PIC_OK;
}
