// Rows a2 + a3 (+ a6), plain FP64 form: the Crank-Nicolson mover of Eq. 4 with
// cell-crossing sub-steps fused with the charge-conserving deposit of Eq. 3.
//
// Two phases, both in normalised units (see push_general.cuh):
//   1. k_push_fp64_fast: one CN solve over the whole step for particles that
//      stay inside their cell; the deposit of the home cell is reduced over
//      runs of lanes with the same home cell before one FP64 atomic per edge;
//   2. k_push_fp64_general: the queued rest (crossings, faces, near axis, no
//      convergence) through the general sub-step path.
// GB300 runs FP64 on a narrow pipe, so the kernels are FP64-pipe bound; the
// two phases keep the warps of the fast path convergent.
#include "push_general.cuh"

namespace pic {
namespace {

// Fast path (no B_z): one CN solve over the whole step in normalised units
// (cells, fractions of dt) for particles that stay inside their cell, with
// three reciprocals per Newton iteration and an acceleration predictor;
// anything else (crossing, face, near axis, no convergence) is queued for
// the general path above.  Velocities from the CN relations dx = (u+u')/2.
constexpr unsigned kFlopFastNewton = 38, kFlopFastAccept = 27;

__device__ __forceinline__ double tol_r64(double rho1, double da) {
  return fmax(1e-13 * fmin(1.0, fmax(rho1, 0.0)), 1e-15 * fabs(da));
}

__global__ void __launch_bounds__(128) k_push_fp64_fast(PushLaunch L) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int nz = L.g.nz, nz1 = nz + 1, ncell = L.g.nr * nz;
  int home = -1;
  double hr0 = 0.0, hr1 = 0.0, hz0 = 0.0, hz1 = 0.0;
  unsigned n_newton = 0, n_acc = 0;
  bool queued = false;
  int c0 = -1;
  double a = 0.0, b = 0.0, vr = 0.0, vt = 0.0, vz = 0.0, w = 0.0;
  if (p < L.n) {
    c0 = L.p.cell[p];
    a = L.p.a[p];
    b = L.p.b[p];
    vr = L.p.vr[p];
    vt = L.p.vt[p];
    vz = L.p.vz[p];
    w = L.p.w[p];
    if (c0 >= 0 && c0 < ncell) {
      int ic = c0 / nz, jc = c0 - (c0 / nz) * nz;
      double ur = vr * L.cr, ut = vt * L.cr, uz = vz * L.cz;
      double rho = (double)ic + a;
      bool acc = false;
      if (a > 0.0 && a < 1.0 && b > 0.0 && b < 1.0 && fabs(ut) < 0.25 * rho) {
        double ar0 = L.ar[ic * nz1 + jc];
        double gar = L.ar[ic * nz1 + jc + 1] - ar0;
        double az0 = L.az[ic * nz + jc];
        double gaz = L.az[(ic + 1) * nz + jc] - az0;
        double P = rho * ut;
        double da = ur + 0.5 * (ar0 + gar * b + ut * ut / rho);
        double db = uz + 0.5 * (az0 + gaz * a);
        const double f1a = -0.25 * gaz, f2b = -0.25 * gar;
        bool conv = false;
        for (int it = 0; it < 5; ++it) {
          double rho1 = rho + da, rhom = rho + 0.5 * da;
          if (!(rho1 > 0.0) || !(rhom > 0.0)) break;
          double inv1 = 1.0 / rho1, invm = 1.0 / rhom;
          double ut1 = P * inv1;
          double utm = 0.5 * (ut + ut1), dutm = -0.5 * ut1 * inv1;
          double C = utm * utm * invm;
          double dC = utm * invm * (2.0 * dutm - 0.5 * utm * invm);
          double az = az0 + gaz * (a + 0.5 * da);
          double A = ar0 + gar * (b + 0.5 * db) + C;
          double f1 = db - uz - 0.5 * az;
          double f2 = da - ur - 0.5 * A;
          double f2a = 1.0 - 0.5 * dC;
          double idet = 1.0 / (f1a * f2b - f2a);
          double xa = (f2 - f1 * f2b) * idet;
          double xb = (f2a * f1 - f1a * f2) * idet;
          da += xa;
          db += xb;
          n_newton++;
          if (fabs(xa) <= tol_r64(rho + da, da) && fabs(xb) <= fmax(1e-13, 1e-15 * fabs(db))) {
            conv = true;
            break;
          }
        }
        double a1 = a + da, b1 = b + db;
        acc = conv && rho + da > 0.0 && a1 > 0.0 && a1 < 1.0 && b1 > 0.0 && b1 < 1.0;
        if (acc) {
          n_acc++;
          home = c0;
          double fr = L.q * w * da, fz = L.q * w * db;
          double am = a + 0.5 * da, bm = b + 0.5 * db;
          hr0 = fr * (1.0 - bm);
          hr1 = fr * bm;
          hz0 = fz * (1.0 - am);
          hz1 = fz * am;
          if (L.write) {
            L.p.a[p] = a1;
            L.p.b[p] = b1;
            L.p.vr[p] = (2.0 * da - ur) * L.icr;
            L.p.vz[p] = (2.0 * db - uz) * L.icz;
            L.p.vt[p] = P / (rho + da) * L.icr;
          }
        }
      }
      queued = !acc;
    }
  }
  const unsigned full = 0xffffffffu;
  int prev = __shfl_up_sync(full, home, 1);
  bool head = (lane == 0) || (prev != home);
  unsigned heads = __ballot_sync(full, head);
  unsigned below = heads & ((2u << lane) - 1u);
  int seg_start = 31 - __clz(below);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double t0 = __shfl_up_sync(full, hr0, o);
    double t1 = __shfl_up_sync(full, hr1, o);
    double t2 = __shfl_up_sync(full, hz0, o);
    double t3 = __shfl_up_sync(full, hz1, o);
    if (lane - o >= seg_start) {
      hr0 += t0; hr1 += t1; hz0 += t2; hz1 += t3;
    }
  }
  int next = __shfl_down_sync(full, home, 1);
  bool tail = (lane == 31) || (next != home);
  if (tail && home >= 0 && L.ir) {
    int ic = home / nz, jc = home - (home / nz) * nz;
    atomicAdd(&L.ir[ic * nz1 + jc], hr0);
    atomicAdd(&L.ir[ic * nz1 + jc + 1], hr1);
    atomicAdd(&L.iz[ic * nz + jc], hz0);
    atomicAdd(&L.iz[(ic + 1) * nz + jc], hz1);
  }
  unsigned qm = __ballot_sync(full, queued);
  if (qm) {
    int leader = __ffs(qm) - 1;
    int qbase = 0;
    if (lane == leader) qbase = atomicAdd(L.qcount, __popc(qm));
    qbase = __shfl_sync(full, qbase, leader);
    if (queued) {
      int k = qbase + __popc(qm & ((1u << lane) - 1u));
      L.queue[k] = (int)p;
      L.q_cell[k] = c0;
      L.q_a[k] = a; L.q_b[k] = b;
      L.q_vr[k] = vr; L.q_vt[k] = vt; L.q_vz[k] = vz; L.q_w[k] = w;
    }
  }
  Tally T0 = {0, 0, 0, 0, 0};
  flush_tally(L.counters, T0, lane, n_newton, n_acc, kFlopFastNewton, kFlopFastAccept);
}

// Phase 2: queued particles (or all of them when queue == nullptr)
__global__ void __launch_bounds__(128) k_push_fp64_general(PushLaunch L) {
  const int lane = threadIdx.x & 31;
  GenArgs<double> G;
  G.nr = L.g.nr; G.nz = L.g.nz; G.ar = L.ar; G.az = L.az;
  G.wt = L.wb * L.dt; G.icr = L.icr; G.icz = L.icz;
  G.q = L.q; G.m = L.m; G.qf = L.q; G.ir = L.ir; G.iz = L.iz; G.write = L.write; G.p = L.p;
  G.wall_z0 = L.wall_z0; G.wall_zl = L.wall_zl; G.wall_r = L.wall_r; G.ke_lost = L.ke_lost;
  long long count = L.queue ? (long long)*L.qcount : L.n;
  Tally T = {0, 0, 0, 0, 0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x) {
    if (L.queue) {
      push_general<double>(G, L.queue[q], L.q_cell[q], L.q_a[q], L.q_b[q], L.q_vr[q] * L.cr,
                           L.q_vt[q] * L.cr, L.q_vz[q] * L.cz, L.q_w[q], T);
    } else {
      push_general<double>(G, q, L.p.cell[q], L.p.a[q], L.p.b[q], L.p.vr[q] * L.cr,
                           L.p.vt[q] * L.cr, L.p.vz[q] * L.cz, L.p.w[q], T);
    }
  }
  flush_tally(L.counters, T, lane, 0, 0, 0, 0);
}

}  // namespace

cudaError_t launch_push_fp64(const PushLaunch &L, cudaStream_t s) {
  if (L.n <= 0) return cudaSuccess;
  const int bs = 128;
  long long nb = (L.n + bs - 1) / bs;
  if (L.wb == 0.0 && L.queue) {
    cudaError_t e = cudaMemsetAsync(L.qcount, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_push_fp64_fast<<<(unsigned)nb, bs, 0, s>>>(L);
    long long ng = nb < 152 * 16 ? nb : 152 * 16;
    k_push_fp64_general<<<(unsigned)ng, bs, 0, s>>>(L);
  } else {
    PushLaunch A = L;
    A.queue = nullptr;
    k_push_fp64_general<<<(unsigned)nb, bs, 0, s>>>(A);
  }
  return cudaGetLastError();
}

}  // namespace pic
