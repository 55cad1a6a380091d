// Row a4: implicit Crank-Nicolson Maxwell solve (Eqs. 1-2, TM: Er, Ez, H_theta;
// H_theta is the primary unknown, Sec. 2.1), integral Yee form:
//   Faraday: mu*Vh*(H1 - H0) = -dt * C^T L E_half
//   Ampere:  eps*A*(E1 - E0) = dt * C H_half - dQ          (unknown edges)
// Eliminating E gives (2 mu Vh + dt^2/2 C^T W C) H_half = rhs.  On the uniform
// mesh with PEC plates (Er = 0 at z = 0, L) and the gap source on r = R, this
// operator is exactly  diag_r(.) (x) T_z + R_r (x) I_z  with T_z the Neumann
// Laplacian along z, so a DCT-II along z diagonalises it into nz independent
// SPD tridiagonal systems along r.  Solve = DCT (FP64 GEMM), Thomas per mode,
// inverse DCT; then H1 = 2 H_half - H0 and E1 explicitly from Ampere.
#include <string.h>

#include "pic_internal.cuh"

namespace pic {
namespace {

__global__ void k_half(long long n1, long long n2, const double *er0, const double *ez0,
                       const double *er1, const double *ez1, double *erh, double *ezh) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n1) erh[t] = 0.5 * (er0[t] + er1[t]);
  else if (t < n1 + n2) {
    long long u = t - n1;
    ezh[u] = 0.5 * (ez0[u] + ez1[u]);
  }
}

// half-step field plus the mixed form's normalised accelerations per species
__global__ void k_half_alpha(long long n1, long long n2, const double *er0, const double *ez0,
                             const double *er1, const double *ez1, double *erh, double *ezh,
                             AlphaOut A) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n1) {
    double e = 0.5 * (er0[t] + er1[t]);
    erh[t] = e;
    const long long i = t / A.nz1;
    if (i < A.xa) {  // mapped mesh: the row's own width
      A.ar[0][t] = (float)(A.srx[0][i] * e);
      A.ar[1][t] = (float)(A.srx[1][i] * e);
    } else {
      A.ar[0][t] = (float)(A.sr[0] * e);
      A.ar[1][t] = (float)(A.sr[1] * e);
    }
  } else if (t < n1 + n2) {
    long long u = t - n1;
    double e = 0.5 * (ez0[u] + ez1[u]);
    ezh[u] = e;
    A.az[0][u] = (float)(A.sz[0] * e);
    A.az[1][u] = (float)(A.sz[1] * e);
  }
}

__global__ void k_half_alpha64(long long n1, long long n2, const double *er0, const double *ez0,
                               const double *er1, const double *ez1, double *erh, double *ezh,
                               AlphaOut64 A) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n1) {
    double e = 0.5 * (er0[t] + er1[t]);
    erh[t] = e;
    const long long i = t / A.nz1;
    if (i < A.xa) {
      A.ar[0][t] = A.srx[0][i] * e;
      A.ar[1][t] = A.srx[1][i] * e;
    } else {
      A.ar[0][t] = A.sr[0] * e;
      A.ar[1][t] = A.sr[1] * e;
    }
  } else if (t < n1 + n2) {
    long long u = t - n1;
    double e = 0.5 * (ez0[u] + ez1[u]);
    ezh[u] = e;
    A.az[0][u] = A.sz[0] * e;
    A.az[1][u] = A.sz[1] * e;
  }
}

// rhs(i,j) = 2 mu Vh H0 - dt * C^T L Et   (Et = (eps A E0 - dQ/2)/D, or the prescribed half value)
// per-row tables: 1/(2D), 1/D of the E_r and E_z edges with D = eps A + dt S/2
// (S: conducting part of the face, zero outside a conducting ring), 2 pi r_{i+1/2},
// the H cell volume, the cell width, and eps A/D of the E_r and E_z edges (1
// outside a conducting ring)
enum { kT2ear = 0, kT2eaz = 1, kTear = 2, kTeaz = 3, kTs = 4, kTvh = 5, kTw = 6, kTgr = 7,
       kTgz = 8, kTabs = 9 };
__device__ __forceinline__ double tab(const FieldOp &F, int k, int i) {
  return F.rtab[k * (F.nr + 1) + i];
}
// axial port: D of the interface edge (i + 1/2, 0), half in the port and half in
// the reactor; of the port's E_r edge between rows q - 1 and q (dual length
// the mean of their heights) and of its E_z edges; 2 E^+ on the end edge
__device__ __forceinline__ double port_dint(const FieldOp &F, int i) {
  return F.eps * tab(F, kTs, i) * 0.5 * (F.port.erq * F.port.htop + F.dz);
}
__device__ __forceinline__ double port_dr(const FieldOp &F, int i, int q) {
  return F.eps * F.port.erq * tab(F, kTs, i) * (0.5 * (F.port.hq[q - 1] + F.port.hq[q]));
}
__device__ __forceinline__ double port_dz(const FieldOp &F, int i) {
  return F.port.erq / tab(F, kTeaz, i);  // erq eps A_z
}
__device__ __forceinline__ double port_ein2(const FieldOp &F, int i, double phi_half) {
  return phi_half * kTwoPi / (tab(F, kTs, i) * F.port.lnr);
}
__device__ __forceinline__ double rhs_at(const FieldOp &F, const double *er0, const double *ez0,
                                        const double *h0, const double *ir, const double *iz,
                                        double v0, double v1, int i, int j) {
  int nr = F.nr, nz = F.nz, nz1 = nz + 1;
  int c = i * nz + j;
  if (F.unit_c >= 0) return c == F.unit_c ? 1.0 : 0.0;
  double dr = tab(F, kTw, i), dz = F.dz;  // E_r edge length: the cell width
  double s = tab(F, kTs, i);
  double r2 = tab(F, kT2ear, i);
  double etb = 0.0, ett = 0.0;
  double gr = tab(F, kTgr, i);
  if (j != 0) etb = er0[i * nz1 + j] * gr - ir[i * nz1 + j] * r2;
  else if (F.port.on && i >= F.port.ip)
    etb = er0[i * nz1] - ir[i * nz1] / (2.0 * port_dint(F, i));  // interface edge
  if (j + 1 != nz) ett = er0[i * nz1 + j + 1] * gr - ir[i * nz1 + j + 1] * r2;
  double etl = ez0[i * nz + j] * tab(F, kTgz, i) - iz[i * nz + j] * tab(F, kT2eaz, i);
  double etr;
  if (i + 1 == nr) etr = F.port.on ? 0.0 : 0.5 * (v0 + v1) / F.L;  // axial port: a conducting wall
  else etr = ez0[(i + 1) * nz + j] * tab(F, kTgz, i + 1) - iz[(i + 1) * nz + j] * tab(F, kT2eaz, i + 1);
  double curl = (-s) * dr * etb + s * dr * ett + s * dz * etl + (-s) * dz * etr;
  return 2.0 * F.mu * tab(F, kTvh, i) * h0[c] - F.dt * curl;
}

__global__ void k_rhs(FieldOp F, const double *er0, const double *ez0, const double *h0,
                      const double *ir, const double *iz, double v0, double v1) {
  if (F.vd) {
    v0 = F.vd[0];
    v1 = F.vd[1];
  }
  if (F.cc.st) v0 = F.cc.st[2];  // the electrode potential phi^n
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int nz = F.nz;
  if (F.half) {
    // mirrored pairs (j, nz-1-j): S = sum into rhs[i*h + j], D = difference into hat-side buffer
    int h = F.half;
    if (c >= F.nr * h) return;
    int i = c / h, j = c - (c / h) * h;
    double x0 = rhs_at(F, er0, ez0, h0, ir, iz, v0, v1, i, j);
    double x1 = rhs_at(F, er0, ez0, h0, ir, iz, v0, v1, i, nz - 1 - j);
    F.rhs[i * h + j] = x0 + x1;
    F.rhs[F.nr * h + i * h + j] = x0 - x1;
    return;
  }
  if (c >= F.nr * nz) return;
  int i = c / nz, j = c - (c / nz) * nz;
  F.rhs[c] = rhs_at(F, er0, ez0, h0, ir, iz, v0, v1, i, j);
}

// Batched C_z[M x N] = A_z[M x K] * B_z[K x N] (z = blockIdx.z), row-major FP64 with
// leading dimensions; 16x16 output tile per 64-thread block, 2x2 per thread, so that
// the small transforms still spread over all SMs (the FP64 pipe is the limit).
struct Gemm {
  int M, N, K, lda, ldb, ldc;
  const double *A[2], *B[2];
  double *C[2];
};
constexpr int GT = 16, GK = 16;
__global__ void __launch_bounds__(64) k_gemm16(Gemm G) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const double *__restrict__ A = G.A[blockIdx.z];
  const double *__restrict__ B = G.B[blockIdx.z];
  double *__restrict__ Cm = G.C[blockIdx.z];
  int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
  double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;
  for (int k0 = 0; k0 < G.K; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 64) {
      int r = e / GK, kk = e - (e / GK) * GK;
      int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < G.M && gk < G.K) ? A[(long long)gr * G.lda + gk] : 0.0;
      int kb = e / GT, cc = e - (e / GT) * GT;
      int gkb = k0 + kb, gc = col0 + cc;
      Bs[kb][cc] = (gkb < G.K && gc < G.N) ? B[(long long)gkb * G.ldb + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
      double b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      acc00 += a0 * b0;
      acc01 += a0 * b1;
      acc10 += a1 * b0;
      acc11 += a1 * b1;
    }
    __syncthreads();
  }
  int gr = row0 + ty * 2, gc = col0 + tx * 2;
  if (gr < G.M && gc < G.N) Cm[(long long)gr * G.ldc + gc] = acc00;
  if (gr < G.M && gc + 1 < G.N) Cm[(long long)gr * G.ldc + gc + 1] = acc01;
  if (gr + 1 < G.M && gc < G.N) Cm[(long long)(gr + 1) * G.ldc + gc] = acc10;
  if (gr + 1 < G.M && gc + 1 < G.N) Cm[(long long)(gr + 1) * G.ldc + gc + 1] = acc11;
}

// C[M x N] = A[M x K] * B[K x N], row-major FP64, 32x32 tile per block, 2x2 per thread
constexpr int TM = 32, TK = 16;
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const double *__restrict__ A,
                                              const double *__restrict__ B,
                                              double *__restrict__ Cm) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TM + 1];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int row0 = blockIdx.y * TM, col0 = blockIdx.x * TM;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = 0; k0 < K; k0 += TK) {
    // load A tile (TM rows x TK cols) and B tile (TK rows x TM cols): 512 elements each
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      int r = e / TK, kk = e - (e / TK) * TK;
      int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? A[(long long)gr * K + gk] : 0.0;
      int kb = e / TM, cc = e - (e / TM) * TM;
      int gkb = k0 + kb, gc = col0 + cc;
      Bs[kb][cc] = (gkb < K && gc < N) ? B[(long long)gkb * N + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
      double b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      int gr = row0 + ty * 2 + u, gc = col0 + tx * 2 + v;
      if (gr < M && gc < N) Cm[(long long)gr * N + gc] = acc[u][v];
    }
}

// ---------------------------------------------------------------------------
// DCTs along z by FFT (Makhoul, IEEE Trans. ASSP 28, 1980): with the even
// samples in order followed by the odd ones reversed, v = (x0, x2, ..., x3,
// x1), the DCT-II is X[m] = Re(exp(-i pi m / 2N) V[m]) with V = DFT(v); two
// real rows are transformed at once as the real and imaginary parts of one
// complex sequence.  The N-point DFT is a mixed-radix (4, 2, 3) Stockham
// autosort FFT in shared memory (Stockham 1966; index form of Govindaraju et
// al., SC 2008).

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// forward DFT (exp(-2 pi i jk / N)) of x; y is scratch; returns the buffer holding the result
__device__ double2 *fft_fwd(const FieldOp &F, double2 *x, double2 *y) {
  const int N = F.fft;
  int Ns = 1;
  for (int p = 0; p < F.nrad; ++p) {
    const int R = F.rad[p], nb = N / R;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      const int k = j % Ns;
      const int ts = (N / (Ns * R)) * k;
      double2 v0 = x[j], v1 = cmul(x[j + nb], F.tw[ts]);
      const int d = (j / Ns) * Ns * R + k;
      if (R == 2) {
        y[d] = cadd(v0, v1);
        y[d + Ns] = csub(v0, v1);
      } else if (R == 4) {
        double2 v2 = cmul(x[j + 2 * nb], F.tw[2 * ts]), v3 = cmul(x[j + 3 * nb], F.tw[3 * ts]);
        double2 s02 = cadd(v0, v2), d02 = csub(v0, v2), s13 = cadd(v1, v3), d13 = csub(v1, v3);
        y[d] = cadd(s02, s13);
        y[d + Ns] = make_double2(d02.x + d13.y, d02.y - d13.x);      // d02 - i d13
        y[d + 2 * Ns] = csub(s02, s13);
        y[d + 3 * Ns] = make_double2(d02.x - d13.y, d02.y + d13.x);  // d02 + i d13
      } else {  // R == 3
        const double s3 = 0.86602540378443864676;  // sqrt(3)/2
        double2 v2 = cmul(x[j + 2 * nb], F.tw[2 * ts]);
        double2 t1 = cadd(v1, v2), dd = csub(v1, v2);
        double2 t2 = make_double2(v0.x - 0.5 * t1.x, v0.y - 0.5 * t1.y);
        double2 t3 = make_double2(s3 * dd.y, -s3 * dd.x);
        y[d] = cadd(v0, t1);
        y[d + Ns] = cadd(t2, t3);
        y[d + 2 * Ns] = csub(t2, t3);
      }
    }
    __syncthreads();
    double2 *t = x;
    x = y;
    y = t;
    Ns *= R;
  }
  return x;
}

__device__ __forceinline__ int dct_perm(int j, int N) { return (j & 1) ? N - 1 - (j >> 1) : (j >> 1); }

// orthonormal DCT-II along z of rows 2b, 2b+1 of src into dst (nr x nz, natural modes)
__global__ void __launch_bounds__(128) k_dct2(FieldOp F, const double *__restrict__ src,
                                              double *__restrict__ dst) {
  extern __shared__ double2 smc[];
  const int N = F.fft;
  double2 *a = smc, *b = smc + N;
  const int r0 = 2 * blockIdx.x, r1 = r0 + 1;
  const bool two = r1 < F.nr;
  for (int j = threadIdx.x; j < N; j += blockDim.x)
    a[dct_perm(j, N)] = make_double2(src[r0 * N + j], two ? src[r1 * N + j] : 0.0);
  __syncthreads();
  const double2 *Z = fft_fwd(F, a, b);
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    const double2 z = Z[m], zr = Z[m == 0 ? 0 : N - m];
    const double2 w = F.pw[m];
    const double c = m == 0 ? F.c0 : F.c1;
    // V_A = (Z + conj Zr)/2, V_B = (Z - conj Zr)/(2i); X = Re(exp(-i pi m/2N) V)
    const double xa = 0.5 * (w.x * (z.x + zr.x) + w.y * (z.y - zr.y));
    const double xb = 0.5 * (w.x * (z.y + zr.y) - w.y * (z.x - zr.x));
    dst[r0 * N + m] = c * xa;
    if (two) dst[r1 * N + m] = c * xb;
  }
}

// orthonormal DCT-III (inverse of k_dct2) of rows 2b, 2b+1
__global__ void __launch_bounds__(128) k_dct3(FieldOp F, const double *__restrict__ src,
                                              double *__restrict__ dst) {
  extern __shared__ double2 smc[];
  const int N = F.fft;
  double2 *a = smc, *b = smc + N;
  const int r0 = 2 * blockIdx.x, r1 = r0 + 1;
  const bool two = r1 < F.nr;
  const double i0 = 1.0 / F.c0, i1 = 1.0 / F.c1;
  // Z = V_A + i V_B with V[m] = exp(i pi m/2N) (X[m] - i X[N-m]), X[N] = 0; the
  // inverse DFT is taken as conj(DFT(conj Z)) / N, so conj Z is stored
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    const double sm = m == 0 ? i0 : i1;
    const double pa = src[r0 * N + m] * sm, pb = two ? src[r1 * N + m] * sm : 0.0;
    const double qa = m == 0 ? 0.0 : -src[r0 * N + N - m] * i1;
    const double qb = (m == 0 || !two) ? 0.0 : -src[r1 * N + N - m] * i1;
    const double2 w = F.pw[m];
    const double2 va = make_double2(pa * w.x - qa * w.y, pa * w.y + qa * w.x);
    const double2 vb = make_double2(pb * w.x - qb * w.y, pb * w.y + qb * w.x);
    a[m] = make_double2(va.x - vb.y, -(va.y + vb.x));
  }
  __syncthreads();
  const double2 *z = fft_fwd(F, a, b);
  const double inv = 1.0 / (double)N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double2 v = z[dct_perm(j, N)];
    dst[r0 * N + j] = v.x * inv;
    if (two) dst[r1 * N + j] = -v.y * inv;
  }
}

// Tridiagonal solve along r per DCT mode by cyclic reduction (Hockney, J. ACM
// 12, 1965): the forward levels s = 1, 2, 4, ... fold rows i = 2sk + 2s - 1
// into d_i += alpha d_{i-s} + gamma d_{i+s}; the back levels solve rows
// j = 2sk + s - 1 as x_j = d_j/b_j - (a_j/b_j) x_{j-s} - (c_j/b_j) x_{j+s}.  The
// operator does not change between solves, so every coefficient is
// precomputed; per solve the dependency chain is 2 log2(n2) levels instead of
// the 2 nr steps of the Thomas algorithm.  One warp per mode, mb modes per
// block staged in shared memory (coalesced along the modes).
__global__ void k_cr(FieldOp F) {
  extern __shared__ double sd[];
  const int n2 = F.n2, nr = F.nr, nz = F.nz;
  const int mb = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * mb;
  for (int e = threadIdx.x; e < n2 * mb; e += blockDim.x) {
    const int i = e / mb, k = e - i * mb, m = m0 + k;
    sd[k * n2 + i] = (i < nr && m < nz) ? F.hat[i * nz + m] : 0.0;
  }
  __syncthreads();
  const int m = m0 + w;
  if (m < nz) {
    double *d = sd + w * n2;
    const double *co = F.crc + (size_t)m * 5 * n2;
    const double *fa = co, *fg = co + n2, *bp = co + 2 * n2, *bq = co + 3 * n2, *br = co + 4 * n2;
    int off = 0;
    for (int s = 1; s < n2; s <<= 1) {
      const int cnt = n2 / (2 * s);
      for (int k = lane; k < cnt; k += 32) {
        const int i = 2 * s * k + 2 * s - 1;
        double v = d[i] + fa[off + k] * d[i - s];
        if (i + s < n2) v += fg[off + k] * d[i + s];
        d[i] = v;
      }
      off += cnt;
      __syncwarp();
    }
    off = 0;
    for (int s = n2; s >= 1; s >>= 1) {
      const int cnt = n2 >= 2 * s ? n2 / (2 * s) : 1;
      for (int k = lane; k < cnt; k += 32) {
        const int j = 2 * s * k + s - 1;
        const double xl = j - s >= 0 ? d[j - s] : 0.0;
        const double xr = j + s < n2 ? d[j + s] : 0.0;
        d[j] = br[off + k] * d[j] - bp[off + k] * xl - bq[off + k] * xr;
      }
      off += cnt;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * mb; e += blockDim.x) {
    const int i = e / mb, k = e - i * mb, mm = m0 + k;
    if (mm < nz) F.hat[i * nz + mm] = sd[k * n2 + i];
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// H_half(i, j): direct, or recombined from the two half-size inverse transforms
__device__ __forceinline__ double hhalf_at(const FieldOp &F, int i, int j) {
  if (!F.half) return F.hhalf[i * F.nz + j];
  int h = F.half;
  const double *P = F.hhalf, *R = F.hhalf + F.nr * h;
  if (j < h) return P[i * h + j] + R[i * h + j];
  int jj = F.nz - 1 - j;
  return P[i * h + jj] - R[i * h + jj];
}

// H^{n+1/2} with the circuit's correction: the solve ran with the electrode
// at V^{n+1}; the actual potential differs by dl, whose response is hu / 2
__device__ __forceinline__ double hh_at(const FieldOp &F, double dl, int i, int j) {
  double v = hhalf_at(F, i, j);
  if (F.cc.st) v += dl * (0.5 * F.cc.hu[i * F.nz + j]);
  return v;
}

// the same for the port's cells (p < np)
__device__ __forceinline__ double hhp_at(const FieldOp &F, double dl, int p) {
  double v = F.port.hhp[p];
  if (F.cc.st) v += dl * (0.5 * F.port.hup[p]);
  return v;
}

// ---- axial port (PortOp) ------------------------------------------------------
// right-hand side of the port cells: 2 mu V_H H^n - dt C^T L Et over their
// edges (the interface edges' Et with the crossed charge; 2 E^+ on the end
// edges, whose -eta H part sits in the port block)
__global__ void k_rhs_port(FieldOp F, const double *er0, const double *ir, double v0, double v1) {
  if (F.vd) {
    v0 = F.vd[0];
    v1 = F.vd[1];
  }
  if (F.cc.st) v0 = F.cc.st[2];  // the electrode potential phi^n
  const PortOp &P = F.port;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  const int k = p / P.nzp, q = p - k * P.nzp, i = P.ip + k, nz1 = F.nz + 1;
  const double s = tab(F, kTs, i), L = tab(F, kTw, i), dzp = P.hq[q];
  const double etb = q == 0 ? port_ein2(F, i, 0.5 * (v0 + v1)) : P.erp0[p];
  const double ett = q + 1 == P.nzp ? er0[i * nz1] - ir[i * nz1] / (2.0 * port_dint(F, i))
                                     : P.erp0[p + 1];
  const double etl = i == P.ip ? 0.0 : P.ezp0[k * P.nzp + q];
  const double etr = i + 1 == F.nr ? 0.0 : P.ezp0[(k + 1) * P.nzp + q];
  const double curl = (-s) * L * etb + s * L * ett + s * dzp * etl + (-s) * dzp * etr;
  const double vh = tab(F, kTvh, i) * dzp / F.dz;
  P.rhsp[p] = 2.0 * F.mu * vh * P.hp0[p] - F.dt * curl;
}

// y_P = Binv rhs_P: one warp per row
__global__ void k_port_solve(FieldOp F) {
  const PortOp &P = F.port;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= P.np) return;
  const double *a = P.Binv + (long long)row * P.np;
  double v = 0.0;
  for (int c = lane; c < P.np; c += 32) v += a[c] * P.rhsp[c];
  v = warp_sum(v);
  if (lane == 0) P.hhp[row] = v;
}

// t = U^T y (interface differences), ws = Cinv t: one block
__global__ void k_port_wood(FieldOp F) {
  const PortOp &P = F.port;
  extern __shared__ double t[];
  for (int e = threadIdx.x; e < P.m; e += blockDim.x)
    t[e] = hhalf_at(F, P.ip + e, 0) - P.hhp[e * P.nzp + P.nzp - 1];
  __syncthreads();
  for (int e = threadIdx.x; e < P.m; e += blockDim.x) {
    const double *c = P.Cinv + (long long)e * P.m;
    double v = 0.0;
    for (int f = 0; f < P.m; ++f) v += c[f] * t[f];
    P.ws[e] = v;
  }
}

// x = y - Z ws: the reactor's hhalf (in its own layout) and the port's H
__global__ void k_port_fix(FieldOp F, long long nh) {
  const PortOp &P = F.port;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nh) {
    double v = 0.0;
    for (int e = 0; e < P.m; ++e) v += P.ZR[(long long)e * nh + t] * P.ws[e];
    F.hhalf[t] -= v;
  } else if (t < nh + P.np) {
    const int p = (int)(t - nh);
    double v = 0.0;
    for (int e = 0; e < P.m; ++e) v += P.ZP[(long long)e * P.np + p] * P.ws[e];
    P.hhp[p] -= v;
  }
}

// the port's H^{n+1}, E^{n+1} (end edges by Mur's relation) and the energy its
// end delivers; with the blocking capacitor the electrode's correction dl
// (written by k_update, launched before) moves phi^{n+1} and the port's H
__global__ void __launch_bounds__(256) k_update_port(FieldOp F, double v0, double v1,
                                                     DevCounters *cnt) {
  if (F.vd) {
    v0 = F.vd[0];
    v1 = F.vd[1];
  }
  double dl = 0.0;
  if (F.cc.st) {
    v0 = F.cc.st[2];
    dl = F.cc.st[1];
    v1 += dl;
  }
  const PortOp &P = F.port;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nzp = P.nzp;
  double src = 0.0;
  if (t < P.np) {
    const int k = t / nzp, q = t - k * nzp, i = P.ip + k;
    const double s = tab(F, kTs, i), L = tab(F, kTw, i);
    const double hh = hhp_at(F, dl, t);
    P.hp1[t] = 2.0 * hh - P.hp0[t];
    if (q == 0) {
      const double eh = port_ein2(F, i, 0.5 * (v0 + v1)) - P.eta * hh;
      P.erp1[t] = 2.0 * eh - P.erp0[t];
      src = eh * L * F.dt * s * hh;
    } else {
      const double ch = -s * hh + s * hhp_at(F, dl, t - 1);
      P.erp1[t] = P.erp0[t] + F.dt * ch / port_dr(F, i, q);
    }
  }
  const int nez = (P.m + 1) * nzp;
  if (t < nez) {
    const int k = t / nzp, q = t - k * nzp, i = P.ip + k;
    if (i == P.ip || i == F.nr) {
      P.ezp1[t] = 0.0;
    } else {
      const double ch = tab(F, kTs, i) * hhp_at(F, dl, k * nzp + q) -
                        tab(F, kTs, i - 1) * hhp_at(F, dl, (k - 1) * nzp + q);
      P.ezp1[t] = P.ezp0[t] + F.dt * ch / port_dz(F, i);
    }
  }
  src = warp_sum(src);
  if ((threadIdx.x & 31) == 0 && src != 0.0) atomicAdd(&cnt->src, src);
}

// H1 = 2 H_half - H0; E1 from Ampere; Picard norms and drive-gap energy.
// With the blocking capacitor, Eq. 6 fixes the electrode potential first:
// Ampere's law summed over the first row of E_z edges over the electrode
// (i < nr; with the axial port i < ip, the electrode's radius) telescopes, so
// dt x the reactor-side current is dt 2 pi r_{e-1/2} H^{n+1/2}(e-1/2, 1/2)
// (e = nr or ip), affine in the potential; every thread evaluates the same
// expression.
__global__ void __launch_bounds__(256) k_update(FieldOp F, const double *er0, const double *ez0,
                                                const double *h0, const double *ir,
                                                const double *iz, double v0, double v1,
                                                double *er1, double *ez1, double *h1,
                                                const double *er_it, const double *ez_it,
                                                DevCounters *cnt) {
  if (F.vd) {
    v0 = F.vd[0];
    v1 = F.vd[1];
  }
  int nr = F.nr, nz = F.nz, nz1 = nz + 1;
  long long ner = (long long)nr * nz1, nez = (long long)(nr + 1) * nz, nh = (long long)nr * nz;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double dn = 0.0, nn = 0.0, src = 0.0;
  double dz = F.dz, dt = F.dt;
  double dl = 0.0;
  if (F.cc.st) {
    v0 = F.cc.st[2];
    const int rim = (F.port.on ? F.port.ip : nr) - 1;
    const double s = dt * tab(F, kTs, rim);
    const double q0 = s * hhalf_at(F, rim, 0);              // electrode at V^{n+1}
    const double gu = s * (0.5 * F.cc.hu[rim * nz]);        // per unit potential
    dl = -(F.cc.st[0] + q0) / (F.cc.C + gu);
    if (t == 0) {
      F.cc.st[1] = dl;
      F.cc.st[3] = q0 + gu * dl;
    }
    v1 += dl;
  }
  if (t < nh) {
    int i = (int)(t / nz), j = (int)(t - (t / nz) * nz);
    h1[t] = 2.0 * hh_at(F, dl, i, j) - h0[t];
  }
  if (t < ner) {
    int i = (int)(t / nz1), j = (int)(t - (t / nz1) * nz1);
    if (j == 0 && F.port.on && i >= F.port.ip) {
      // interface edge: the port's top cell below, the reactor's first cell above
      const double s = tab(F, kTs, i);
      const double ch = -s * hh_at(F, dl, i, 0) +
                        s * hhp_at(F, dl, (i - F.port.ip) * F.port.nzp + F.port.nzp - 1);
      er1[t] = er0[t] + (dt * ch - ir[t]) / port_dint(F, i);
    } else if (j == 0 || j == nz) {
      er1[t] = 0.0;
    } else {
      double s = tab(F, kTs, i);
      double ch = -s * hh_at(F, dl, i, j) + s * hh_at(F, dl, i, j - 1);
      // (eps A + dt S/2) E1 = (eps A - dt S/2) E0 + dt C H - dQ
      double e1 = er0[t] * (2.0 * tab(F, kTgr, i) - 1.0) + (dt * ch - ir[t]) * tab(F, kTear, i);
      er1[t] = e1;
      if (er_it) {
        double d = e1 - er_it[t];
        dn += d * d;
        nn += e1 * e1;
      }
    }
  }
  if (t < nez) {
    int i = (int)(t / nz), j = (int)(t - (t / nz) * nz);
    double ch = 0.0;
    if (i <= nr - 1) ch += tab(F, kTs, i) * hh_at(F, dl, i, j);
    if (i >= 1) ch += -tab(F, kTs, i - 1) * hh_at(F, dl, i - 1, j);
    if (i == nr && F.port.on) {
      ez1[t] = 0.0;  // the reactor's side wall: a conductor
    } else if (i == nr) {
      double eh;
      if (F.wave) {  // wave port: the boundary field follows H at the outermost node
        eh = 0.5 * (v0 + v1) / F.L - F.eta * hh_at(F, dl, nr - 1, j);
        ez1[t] = 2.0 * eh - ez0[t];
      } else {
        eh = 0.5 * (v0 + v1) / F.L;
        ez1[t] = v1 / F.L;
      }
      src += eh * dz * (iz[t] - dt * ch);
    } else {
      double e1 = ez0[t] * (2.0 * tab(F, kTgz, i) - 1.0) + (dt * ch - iz[t]) * tab(F, kTeaz, i);
      ez1[t] = e1;
      if (ez_it) {
        double d = e1 - ez_it[t];
        dn += d * d;
        nn += e1 * e1;
      }
    }
  }
  __shared__ double red[3][8];
  dn = warp_sum(dn);
  nn = warp_sum(nn);
  src = warp_sum(src);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][w] = dn;
    red[1][w] = nn;
    red[2][w] = src;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      b += red[1][k];
      c += red[2][k];
    }
    if (a != 0.0) atomicAdd(&cnt->norm[0], a);
    if (b != 0.0) atomicAdd(&cnt->norm[1], b);
    if (c != 0.0) atomicAdd(&cnt->src, c);
  }
}

// orthonormal DST-I of rows 2b, 2b+1 of src (nr x M, M = N - 1) into dst, by the
// 2N-point FFT of the odd extensions y_j = x_j, y_{2N-j} = -x_j, y_0 = y_N = 0:
// DFT(y)_m = -2i X_m, so with z = y_A + i y_B, X_A = -Im Z / 2, X_B = Re Z / 2
__global__ void __launch_bounds__(128) k_dst1(FieldOp V, int nrows, int M,
                                              const double *__restrict__ src,
                                              double *__restrict__ dst) {
  extern __shared__ double2 smd[];
  const int N2 = V.fft, N = N2 / 2;
  double2 *a = smd, *b = smd + N2;
  const int r0 = 2 * blockIdx.x, r1 = r0 + 1;
  const bool two = r1 < nrows;
  for (int j = threadIdx.x; j < N2; j += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (j >= 1 && j <= M) {
      v = make_double2(src[r0 * M + j - 1], two ? src[r1 * M + j - 1] : 0.0);
    } else if (j > N) {
      const int k = N2 - j;
      v = make_double2(-src[r0 * M + k - 1], two ? -src[r1 * M + k - 1] : 0.0);
    }
    a[j] = v;
  }
  __syncthreads();
  const double2 *Z = fft_fwd(V, a, b);
  const double sc = 0.5 * sqrt(2.0 / N);
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    const double2 z = Z[m + 1];
    dst[r0 * M + m] = -z.y * sc;
    if (two) dst[r1 * M + m] = z.x * sc;
  }
}

// ---------------------------------------------------------------------------
// electrostatic model (Eq. 8)

__device__ __forceinline__ double es_phi0(const EsOp &E, double phi0) {
  return E.vd ? E.vd[1] : phi0;
}

// node potential with the Dirichlet values on the plates and across the gap
// (axial port: the disc and the port's opening on z = 0, a grounded side
// wall); dl: the circuit's correction of the electrode potential (phi0
// includes it), whose response is the vacuum solution dl (1 - z/L) (with the
// port: dl uphi)
__device__ __forceinline__ double es_node(const EsOp &E, double phi0, double dl, int i, int j) {
  if (j == 0) return E.pip ? phi0 * E.g0[i] : phi0;
  if (j == E.nz) return 0.0;
  if (i == E.nr) return E.pip ? 0.0 : phi0 * (1.0 - (double)j / E.nz);
  const int c = i * E.M + j - 1;
  return E.phi[c] + dl * (E.pip ? E.uphi[c] : 1.0 - (double)j / E.nz);
}

// Eq. 6 with the blocking capacitor: dt x the reactor-side current through the
// dual faces of the first row of E_z edges (i < nr; with the axial port the
// electrode disc, i < pip), displacement plus crossed charge, for the solve at
// V^{n+1}; the response per unit potential is the vacuum value cr (closed
// form, or from the unit solve with the port).  One block, fixed summation order.
__global__ void __launch_bounds__(256) k_es_circuit(EsOp E, const double *iz, double phi0) {
  phi0 = es_phi0(E, phi0);
  const int nr = E.nr, nz = E.nz, ne = E.pip ? E.pip : nr;
  double v = 0.0;
  for (int i = threadIdx.x; i < ne; i += blockDim.x) {
    const double ea = E.tab[2 * nr + i];  // eps A_z(i) / dz
    const double ez1 = (phi0 - E.phi[i * E.M]) / E.dz;
    v += ea * E.dz * (ez1 - E.ez0[i * nz]) + iz[i * nz];
  }
  __shared__ double red[8];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double q0 = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) q0 += red[k];
    const double dl = -(E.cc.st[0] + q0) / (E.cc.C + E.cc.cr);
    E.cc.st[1] = dl;
    E.cc.st[3] = q0 + E.cc.cr * dl;
  }
}

__global__ void k_circuit_commit(Circuit c, const double *vd) {
  const double phi1 = vd[1] + c.st[1];
  c.st[0] = c.C * (vd[1] - phi1);
  c.st[2] = phi1;
}

// rhs of the interior nodes: Q^{n+1} (= Qn - div I) plus the boundary values
__global__ void __launch_bounds__(256) k_es_rhs(EsOp E, const double *Q, const double *ir,
                                                const double *iz, double phi0) {
  phi0 = es_phi0(E, phi0);
  const int nr = E.nr, nz = E.nz, M = E.M;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nr * M) return;
  const int i = t / M, j = t - (t / M) * M + 1;
  double q = Q[i * (nz + 1) + j];
  if (ir) {
    // continuity on the node: Q^{n+1} = Q^n - (outward crossed charge)
    double out = ir[i * (nz + 1) + j] + iz[i * nz + j] - iz[i * nz + j - 1];
    if (i >= 1) out -= ir[(i - 1) * (nz + 1) + j];
    q -= out;
  }
  const double cR = E.tab[i], cZ = E.tab[2 * nr + i];
  if (i == nr - 1 && !E.pip) q += cR * phi0 * (1.0 - (double)j / nz);
  if (j == 1) q += cZ * phi0 * (E.pip ? E.g0[i] : 1.0);
  E.rhs[t] = q;
}

__global__ void __launch_bounds__(256) k_es_advance(EsOp E, double *Q, const double *ir,
                                                    const double *iz) {
  const int nr = E.nr, nz = E.nz, M = E.M;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nr * M) return;
  const int i = t / M, j = t - (t / M) * M + 1;
  double out = ir[i * (nz + 1) + j] + iz[i * nz + j] - iz[i * nz + j - 1];
  if (i >= 1) out -= ir[(i - 1) * (nz + 1) + j];
  Q[i * (nz + 1) + j] -= out;
}

__global__ void __launch_bounds__(256) k_es_field(EsOp E, double phi0, double *er1, double *ez1,
                                                  const double *er_it, const double *ez_it,
                                                  DevCounters *cnt) {
  phi0 = es_phi0(E, phi0);
  double dl = 0.0;
  if (E.cc.st) {
    dl = E.cc.st[1];
    phi0 += dl;
  }
  const int nr = E.nr, nz = E.nz, nz1 = nz + 1;
  const long long ner = (long long)nr * nz1, nez = (long long)(nr + 1) * nz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double dn = 0.0, nn = 0.0;
  if (t < ner) {
    const int i = (int)(t / nz1), j = (int)(t - (t / nz1) * nz1);
    double e = -(es_node(E, phi0, dl, i + 1, j) - es_node(E, phi0, dl, i, j)) / E.tab[3 * nr + i];
    er1[t] = e;
    if (er_it && j != 0 && j != nz) {
      double d = e - er_it[t];
      dn += d * d;
      nn += e * e;
    }
  }
  if (t < nez) {
    const int i = (int)(t / nz), j = (int)(t - (t / nz) * nz);
    double e = -(es_node(E, phi0, dl, i, j + 1) - es_node(E, phi0, dl, i, j)) / E.dz;
    ez1[t] = e;
    if (ez_it && i < nr) {
      double d = e - ez_it[t];
      dn += d * d;
      nn += e * e;
    }
  }
  if (!cnt) return;
  __shared__ double red[2][8];
  dn = warp_sum(dn);
  nn = warp_sum(nn);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][w] = dn;
    red[1][w] = nn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    if (a != 0.0) atomicAdd(&cnt->norm[0], a);
    if (b != 0.0) atomicAdd(&cnt->norm[1], b);
  }
}

}  // namespace

cudaError_t launch_half_field(const Grid &g, const double *er0, const double *ez0,
                              const double *er1, const double *ez1, double *erh, double *ezh,
                              cudaStream_t s) {
  long long n1 = (long long)g.nr * (g.nz + 1), n2 = (long long)(g.nr + 1) * g.nz;
  long long n = n1 + n2;
  k_half<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n1, n2, er0, ez0, er1, ez1, erh, ezh);
  return cudaGetLastError();
}

cudaError_t launch_half_field_alpha(const Grid &g, const double *er0, const double *ez0,
                                    const double *er1, const double *ez1, double *erh,
                                    double *ezh, const AlphaOut &A, cudaStream_t s) {
  long long n1 = (long long)g.nr * (g.nz + 1), n2 = (long long)(g.nr + 1) * g.nz;
  long long n = n1 + n2;
  k_half_alpha<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n1, n2, er0, ez0, er1, ez1, erh, ezh,
                                                           A);
  return cudaGetLastError();
}

cudaError_t launch_half_field_alpha64(const Grid &g, const double *er0, const double *ez0,
                                      const double *er1, const double *ez1, double *erh,
                                      double *ezh, const AlphaOut64 &A, cudaStream_t s) {
  long long n1 = (long long)g.nr * (g.nz + 1), n2 = (long long)(g.nr + 1) * g.nz;
  long long n = n1 + n2;
  k_half_alpha64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n1, n2, er0, ez0, er1, ez1, erh,
                                                             ezh, A);
  return cudaGetLastError();
}

// the reactor's separable solve of F.rhs into F.hhalf (DCT along z, cyclic
// reduction per mode, inverse DCT)
void solve_core(const FieldOp &F, cudaStream_t s) {
  dim3 grid((F.nz + TM - 1) / TM, (F.nr + TM - 1) / TM);
  int h = F.half;
  Gemm G;
  dim3 g16((h + GT - 1) / GT, (F.nr + GT - 1) / GT, 2);
  const unsigned npair = (unsigned)((F.nr + 1) / 2);
  const size_t fsm = (size_t)2 * F.fft * sizeof(double2);
  static bool fattr = false;
  if (F.fft && !fattr) {
    cudaFuncSetAttribute(k_dct2, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
    cudaFuncSetAttribute(k_dct3, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
    fattr = true;
  }
  if (F.fft) {
    k_dct2<<<npair, 128, fsm, s>>>(F, F.rhs, F.hat);
  } else if (h) {
    // hat[:, 0:h] = S * Qe, hat[:, h:nz] = D * Qo   (even / odd DCT modes)
    G.M = F.nr; G.N = h; G.K = h; G.lda = h; G.ldb = h; G.ldc = F.nz;
    G.A[0] = F.rhs; G.A[1] = F.rhs + F.nr * h;
    G.B[0] = F.Q; G.B[1] = F.Q + h * h;
    G.C[0] = F.hat; G.C[1] = F.hat + h;
    k_gemm16<<<g16, 64, 0, s>>>(G);
  } else {
    k_gemm<<<grid, 256, 0, s>>>(F.nr, F.nz, F.nz, F.rhs, F.Q, F.hat);
  }
  // modes per block: up to 8 (one warp each) within the shared-memory budget
  int mb = 8;
  while (mb > 1 && (size_t)F.n2 * mb * sizeof(double) > 160 * 1024) mb >>= 1;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_cr, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  k_cr<<<(F.nz + mb - 1) / mb, 32 * mb, (size_t)F.n2 * mb * sizeof(double), s>>>(F);
  if (F.fft) {
    k_dct3<<<npair, 128, fsm, s>>>(F, F.hat, F.hhalf);
  } else if (h) {
    // P = hat_e * Qe^T, R = hat_o * Qo^T; H_half(j) = P + R, H_half(nz-1-j) = P - R
    G.M = F.nr; G.N = h; G.K = h; G.lda = F.nz; G.ldb = h; G.ldc = h;
    G.A[0] = F.hat; G.A[1] = F.hat + h;
    G.B[0] = F.QT; G.B[1] = F.QT + h * h;
    G.C[0] = F.hhalf; G.C[1] = F.hhalf + F.nr * h;
    k_gemm16<<<g16, 64, 0, s>>>(G);
  } else {
    k_gemm<<<grid, 256, 0, s>>>(F.nr, F.nz, F.nz, F.hat, F.QT, F.hhalf);
  }
}

cudaError_t launch_field_solve(const FieldOp &F, const double *er0, const double *ez0,
                               const double *h0, const double *ir, const double *iz, double v0,
                               double v1, double *er1, double *ez1, double *h1, const double *er_it,
                               const double *ez_it, DevCounters *cnt, cudaStream_t s) {
  cudaError_t e;
  int nc = F.nr * F.nz;
  if ((e = cudaMemsetAsync(&cnt->norm[0], 0, 3 * sizeof(double), s)) != cudaSuccess) return e;
  k_rhs<<<(nc + 255) / 256, 256, 0, s>>>(F, er0, ez0, h0, ir, iz, v0, v1);
  const PortOp &P = F.port;
  if (P.on) k_rhs_port<<<(P.np + 255) / 256, 256, 0, s>>>(F, er0, ir, v0, v1);
  solve_core(F, s);
  if (P.on) {
    // the port block, then the interface coupling (Woodbury)
    k_port_solve<<<(unsigned)(((long long)P.np * 32 + 255) / 256), 256, 0, s>>>(F);
    k_port_wood<<<1, 256, (size_t)P.m * sizeof(double), s>>>(F);
    const long long nh = (long long)F.nr * F.nz;
    k_port_fix<<<(unsigned)((nh + P.np + 255) / 256), 256, 0, s>>>(F, nh);
  }
  long long ner = (long long)F.nr * (F.nz + 1), nez = (long long)(F.nr + 1) * F.nz;
  long long n = ner > nez ? ner : nez;
  k_update<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(F, er0, ez0, h0, ir, iz, v0, v1, er1, ez1,
                                                       h1, er_it, ez_it, cnt);
  if (P.on) {
    const int np2 = P.np > (P.m + 1) * P.nzp ? P.np : (P.m + 1) * P.nzp;
    k_update_port<<<(np2 + 255) / 256, 256, 0, s>>>(F, v0, v1, cnt);
  }
  return cudaGetLastError();
}

// the reactor's separable solve of the unit right-hand side of H cell c into
// F.hhalf (the axial port's set-up: columns of B_R^{-1} U)
cudaError_t launch_unit_solve(const FieldOp &Fin, int c, cudaStream_t s) {
  FieldOp F = Fin;
  F.unit_c = c;
  F.port.on = 0;
  const int nc = F.nr * F.nz;
  k_rhs<<<(nc + 255) / 256, 256, 0, s>>>(F, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0);
  solve_core(F, s);
  return cudaGetLastError();
}

cudaError_t launch_circuit_commit(const Circuit &c, const double *vd, cudaStream_t s) {
  k_circuit_commit<<<1, 1, 0, s>>>(c, vd);
  return cudaGetLastError();
}

cudaError_t launch_es_advance(const EsOp &E, double *Q, const double *ir, const double *iz,
                              cudaStream_t s) {
  const int nc = E.nr * E.M;
  k_es_advance<<<(nc + 255) / 256, 256, 0, s>>>(E, Q, ir, iz);
  return cudaGetLastError();
}

cudaError_t launch_es_solve(const EsOp &E, const double *Q, const double *ir, const double *iz,
                            double phi0, double *er1, double *ez1, const double *er_it,
                            const double *ez_it, DevCounters *cnt, cudaStream_t s) {
  cudaError_t e;
  if (cnt && (e = cudaMemsetAsync(&cnt->norm[0], 0, 3 * sizeof(double), s)) != cudaSuccess)
    return e;
  const int nc = E.nr * E.M;
  k_es_rhs<<<(nc + 255) / 256, 256, 0, s>>>(E, Q, ir, iz, phi0);
  dim3 grid((E.M + TM - 1) / TM, (E.nr + TM - 1) / TM);
  FieldOp D;  // FFT plan of the DST
  memset(&D, 0, sizeof(D));
  D.fft = E.fft2;
  D.nrad = E.nrad;
  for (int k = 0; k < 16; ++k) D.rad[k] = E.rad[k];
  D.tw = E.tw2;
  const unsigned npair = (unsigned)((E.nr + 1) / 2);
  const size_t dsm = (size_t)2 * E.fft2 * sizeof(double2);
  static bool dattr = false;
  if (E.fft2 && !dattr) {
    cudaFuncSetAttribute(k_dst1, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    dattr = true;
  }
  if (E.fft2)
    k_dst1<<<npair, 128, dsm, s>>>(D, E.nr, E.M, E.rhs, E.hat);
  else
    k_gemm<<<grid, 256, 0, s>>>(E.nr, E.M, E.M, E.rhs, E.S, E.hat);
  // the tridiagonal solves of the modes: the cyclic-reduction kernel on an
  // operator view with M columns
  FieldOp V;
  memset(&V, 0, sizeof(V));
  V.nr = E.nr;
  V.nz = E.M;
  V.n2 = E.n2;
  V.crc = E.crc;
  V.hat = E.hat;
  int mb = 8;
  while (mb > 1 && (size_t)E.n2 * mb * sizeof(double) > 160 * 1024) mb >>= 1;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_cr, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_cr<<<(E.M + mb - 1) / mb, 32 * mb, (size_t)E.n2 * mb * sizeof(double), s>>>(V);
  if (E.fft2)
    k_dst1<<<npair, 128, dsm, s>>>(D, E.nr, E.M, E.hat, E.phi);
  else
    k_gemm<<<grid, 256, 0, s>>>(E.nr, E.M, E.M, E.hat, E.S, E.phi);
  if (E.cc.st) k_es_circuit<<<1, 256, 0, s>>>(E, iz, phi0);
  long long ner = (long long)E.nr * (E.nz + 1), nez = (long long)(E.nr + 1) * E.nz;
  long long n = ner > nez ? ner : nez;
  k_es_field<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(E, phi0, er1, ez1, er_it, ez_it, cnt);
  return cudaGetLastError();
}

}  // namespace pic
