// Rows a2 + a3 (+ a6), mixed-precision form: the CN mover with cell-crossing
// sub-steps and the charge-conserving deposit of Eqs. 3-4 in FP32.
//
// Normalised units as in push_general.cuh (cells, fractions of dt, velocities
// in cells per step, alpha = (q/m)*E*dt^2/dx prepared per species from the
// FP64 E^{n+1/2} once per pass).  The particle state is FP32 in physical units
// (28 bytes read per push).  Two phases:
//   1. k_push_fp32_fast: one CN solve over the whole step for particles that
//      stay inside their cell (the common case), lean no-B_z Jacobian; the
//      deposit is split: FP32 sums over runs of lanes with the same home cell
//      (at most 32 terms), converted exactly to FP64 with integer operations
//      and added with FP64 atomics (executed in L2), so the kernel issues no
//      FP64 arithmetic and the Picard residual can still reach 1e-8;
//   2. k_push_fp32_general: the queued rest (crossings, faces, near axis,
//      no convergence) through the general sub-step path, from compact queue
//      records written by phase 1.
#include "push_general.cuh"

namespace pic {
namespace {

constexpr float kTol32 = Num<float>::tol;
// algorithmic FP32 operations of the fast path: per Newton iteration, per accept
constexpr unsigned kOpFastNewton = 38, kOpFastAccept = 27;

// Phase 1: one CN solve over the whole step for particles that stay in their
// cell (the common case), lean Jacobian without the optional B_z terms;
// everything else is queued for the general path.
__global__ void __launch_bounds__(256) k_push_fp32_fast(PushLaunch32 L) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int nz = L.g.nz, nz1 = nz + 1, ncell = L.g.nr * nz;
  int home = -1;
  float hr0 = 0.f, hr1 = 0.f, hz0 = 0.f, hz1 = 0.f;
  unsigned fast_newton = 0, fast_acc = 0;
  bool queued = false;
  int c0 = -1;
  float a = 0.f, b = 0.f, ur = 0.f, ut = 0.f, uz = 0.f, w = 0.f;
  if (p < L.n) {
    c0 = L.p.cell[p];
    a = L.p.a[p];
    b = L.p.b[p];
    ur = L.p.vr[p] * L.cr;
    ut = L.p.vt[p] * L.cr;
    uz = L.p.vz[p] * L.cz;
    w = L.p.w[p];
    if (c0 >= 0 && c0 < ncell) {
      // cell -> (ic, jc) without an integer division (c0 < 2^24 is exact in FP32)
      int ic = __float2int_rz(__int2float_rn(c0) * L.inz);
      int jc = c0 - ic * nz;
      if (jc < 0) { ic -= 1; jc += nz; }
      else if (jc >= nz) { ic += 1; jc -= nz; }
      float rho = (float)ic + a;
      bool acc = false;
      float da = 0.f, db = 0.f;
      if (a > 0.f && a < 1.f && b > 0.f && b < 1.f && fabsf(ut) < 0.25f * rho) {
        float ar0 = L.ar[ic * nz1 + jc];
        float gar = L.ar[ic * nz1 + jc + 1] - ar0;
        float az0 = L.az[ic * nz + jc];
        float gaz = L.az[(ic + 1) * nz + jc] - az0;
        float P = rho * ut;
        float A0 = ar0 + gar * b + ut * ut * __fdividef(1.f, rho);
        da = ur + 0.5f * A0;
        db = uz + 0.5f * (az0 + gaz * a);
        const float f1a = -0.25f * gaz, f2b = -0.25f * gar;
        bool conv = false;
#pragma unroll 1
        for (int it = 0; it < 4; ++it) {
          float rho1 = rho + da, rhom = rho + 0.5f * da;
          if (!(rho1 > 0.f) || !(rhom > 0.f)) break;
          float inv1 = __fdividef(1.f, rho1), invm = __fdividef(1.f, rhom);
          float ut1 = P * inv1;
          float utm = 0.5f * (ut + ut1), dutm = -0.5f * ut1 * inv1;
          float C = utm * utm * invm;
          float dC = utm * invm * (2.f * dutm - 0.5f * utm * invm);
          float az = az0 + gaz * (a + 0.5f * da);
          float A = ar0 + gar * (b + 0.5f * db) + C;
          float f1 = db - uz - 0.5f * az;
          float f2 = da - ur - 0.5f * A;
          float f2a = 1.f - 0.5f * dC;
          float idet = __fdividef(1.f, f1a * f2b - f2a);
          float xa = (f2 - f1 * f2b) * idet;
          float xb = (f2a * f1 - f1a * f2) * idet;
          da += xa;
          db += xb;
          fast_newton++;
          if (fabsf(xa) <= tol_r<float>(rho + da, da) && fabsf(xb) <= tol_x<float>(db)) {
            conv = true;
            break;
          }
        }
        float a1 = a + da, b1 = b + db;
        acc = conv && rho + da > 0.f && a1 > 0.f && a1 < 1.f && b1 > 0.f && b1 < 1.f;
        if (acc) {
          fast_acc++;
          home = c0;
          float fr = L.qf * w * da, fz = L.qf * w * db;
          float am = a + 0.5f * da, bm = b + 0.5f * db;
          hr0 = fr * (1.f - bm);
          hr1 = fr * bm;
          hz0 = fz * (1.f - am);
          hz1 = fz * am;
          if (L.write) {
            // CN velocity relations: dx = (u + u')/2 over one step
            L.p.a[p] = a1;
            L.p.b[p] = b1;
            L.p.vr[p] = (2.f * da - ur) * L.icr;
            L.p.vz[p] = (2.f * db - uz) * L.icz;
            L.p.vt[p] = P * __fdividef(1.f, rho + da) * L.icr;
          }
        }
      }
      queued = !acc;
    }
  }
  // warp: segmented FP32 sums of the accepted deposits, FP64 atomics
  const unsigned full = 0xffffffffu;
  int prev = __shfl_up_sync(full, home, 1);
  bool head = (lane == 0) || (prev != home);
  unsigned heads = __ballot_sync(full, head);
  if (heads == 1u) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      hr0 += __shfl_xor_sync(full, hr0, o);
      hr1 += __shfl_xor_sync(full, hr1, o);
      hz0 += __shfl_xor_sync(full, hz0, o);
      hz1 += __shfl_xor_sync(full, hz1, o);
    }
  } else {
    unsigned below = heads & ((2u << lane) - 1u);
    int seg_start = 31 - __clz(below);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      float t0 = __shfl_up_sync(full, hr0, o);
      float t1 = __shfl_up_sync(full, hr1, o);
      float t2 = __shfl_up_sync(full, hz0, o);
      float t3 = __shfl_up_sync(full, hz1, o);
      if (lane - o >= seg_start) {
        hr0 += t0; hr1 += t1; hz0 += t2; hz1 += t3;
      }
    }
  }
  int next = __shfl_down_sync(full, home, 1);
  bool tail = (lane == 31) || (next != home);
  if (tail && home >= 0 && L.ir) {
    int ic = home / nz, jc = home - (home / nz) * nz;
    atomicAdd(&L.ir[ic * nz1 + jc], Num<float>::to_double(hr0));
    atomicAdd(&L.ir[ic * nz1 + jc + 1], Num<float>::to_double(hr1));
    atomicAdd(&L.iz[ic * nz + jc], Num<float>::to_double(hz0));
    atomicAdd(&L.iz[(ic + 1) * nz + jc], Num<float>::to_double(hz1));
  }
  // queue the rest for the general path (warp-aggregated append)
  unsigned qm = __ballot_sync(full, queued);
  if (qm) {
    int leader = __ffs(qm) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(L.qcount, __popc(qm));
    base = __shfl_sync(full, base, leader);
    if (queued) {
      int k = base + __popc(qm & ((1u << lane) - 1u));
      L.queue[k] = (int)p;
      L.q_cell[k] = c0;
      L.q_a[k] = a;
      L.q_b[k] = b;
      L.q_ur[k] = ur;
      L.q_ut[k] = ut;
      L.q_uz[k] = uz;
      L.q_w[k] = w;
    }
  }
  Tally T = {0, 0, 0, 0, 0};
  flush_tally(L.counters, T, lane, fast_newton, fast_acc, kOpFastNewton, kOpFastAccept);
}

// Phase 2: queued particles (or all of them when queue == nullptr)
__global__ void __launch_bounds__(256) k_push_fp32_general(PushLaunch32 L) {
  const int lane = threadIdx.x & 31;
  GenArgs<float> G;
  G.nr = L.g.nr; G.nz = L.g.nz; G.ar = L.ar; G.az = L.az;
  G.wt = L.wbt; G.icr = L.icr; G.icz = L.icz;
  G.q = L.q; G.m = L.m; G.qf = L.qf; G.ir = L.ir; G.iz = L.iz; G.write = L.write; G.p = L.p;
  G.wall_z0 = L.wall_z0; G.wall_zl = L.wall_zl; G.wall_r = L.wall_r; G.ke_lost = L.ke_lost;
  long long count = L.queue ? (long long)*L.qcount : L.n;
  Tally T = {0, 0, 0, 0, 0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x) {
    if (L.queue) {
      push_general<float>(G, L.queue[q], L.q_cell[q], L.q_a[q], L.q_b[q], L.q_ur[q], L.q_ut[q],
                          L.q_uz[q], L.q_w[q], T);
    } else {
      push_general<float>(G, q, L.p.cell[q], L.p.a[q], L.p.b[q], L.p.vr[q] * L.cr,
                          L.p.vt[q] * L.cr, L.p.vz[q] * L.cz, L.p.w[q], T);
    }
  }
  flush_tally(L.counters, T, lane, 0, 0, 0, 0);
}

}  // namespace

cudaError_t launch_push_fp32(const PushLaunch32 &L, cudaStream_t s) {
  if (L.n <= 0) return cudaSuccess;
  const int bs = 256;
  long long nb = (L.n + bs - 1) / bs;
  if (L.wbt == 0.f && L.queue) {
    cudaError_t e = cudaMemsetAsync(L.qcount, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_push_fp32_fast<<<(unsigned)nb, bs, 0, s>>>(L);
    // the queue holds the crossing / near-axis particles (a fraction of n)
    long long ng = nb < 152 * 16 ? nb : 152 * 16;
    k_push_fp32_general<<<(unsigned)ng, bs, 0, s>>>(L);
  } else {
    PushLaunch32 A = L;
    A.queue = nullptr;
    k_push_fp32_general<<<(unsigned)nb, bs, 0, s>>>(A);
  }
  return cudaGetLastError();
}

}  // namespace pic
