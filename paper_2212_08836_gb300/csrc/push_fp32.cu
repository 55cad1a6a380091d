// Rows a2 + a3 (+ a6), mixed-precision form: the CN mover with cell-crossing
// sub-steps and the charge-conserving deposit of Eqs. 3-4 in FP32.
//
// Same method as the FP64 kernel, written in normalised units so that every
// quantity is O(1) in single precision: lengths in cells (r in units of dr,
// z in units of dz), time in units of dt (tau in [0, 1]), velocities in cells
// per step (u = v*dt/dx), accelerations alpha = (q/m)*E*dt^2/dx precomputed per
// species from E^{n+1/2} (FP64) once per pass.  Per sub-step, with
// am = a + da/2, bm = b + db/2 and rho = ic + a:
//   da = tau*ur + tau^2/2*(alpha_r(bm) + C),  db = tau*uz + tau^2/2*alpha_z(am),
//   C = ut_m^2/rho_m + wt*ut_m, ut' from rho*ut + wt*rho^2/2 = const (exact CN).
// The particle state is FP32 in physical units (28 bytes read per push); the
// deposit is split: FP32 sums over runs of lanes with the same home cell
// (at most 32 terms), converted exactly to FP64 with integer operations and
// added with FP64 atomics (executed in L2) into the global flux arrays, so the
// kernel issues no FP64 arithmetic and the Picard residual can still reach
// FP64-level tolerances.
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kNewtonMax32 = 30;
constexpr float kTol32 = 1e-6f;

// FP32 stopping tests: the change of the offset along r is measured relative
// to r' when the particle ends close to the axis (where r' itself is small),
// but never below a few ulp of the unknown, which is all FP32 can resolve
__device__ __forceinline__ float tol_r(float rho1, float da) {
  return fmaxf(kTol32 * fminf(1.f, fmaxf(rho1, 0.f)), 4.8e-7f * fabsf(da));
}
__device__ __forceinline__ float tol_x(float x) { return fmaxf(kTol32, 4.8e-7f * fabsf(x)); }

struct Sub32 {
  float ar0, gar, az0, gaz;
  float a, b, rho, ur, ut, uz, P;
};

struct Res32 {
  float f1, f2, f1a, f1t, f2a, f2b, f2t, A, az, ut1;
};

__device__ __forceinline__ void eval32(const Sub32 &s, float wt, float da, float db, float tau,
                                       Res32 &o) {
  float rho1 = s.rho + da;
  float rhom = s.rho + 0.5f * da;
  float ut1, dut1;
  if (rho1 > 0.f) {
    float inv1 = __fdividef(1.f, rho1);
    ut1 = (s.P - 0.5f * wt * rho1 * rho1) * inv1;
    dut1 = -s.P * inv1 * inv1 - 0.5f * wt;
  } else {
    ut1 = s.ut;
    dut1 = 0.f;
  }
  float utm = 0.5f * (s.ut + ut1);
  float dutm = 0.5f * dut1;
  float C, dC;
  if (rhom > 0.f) {
    float invm = __fdividef(1.f, rhom);
    C = utm * utm * invm + wt * utm;
    dC = 2.f * utm * dutm * invm - 0.5f * utm * utm * invm * invm + wt * dutm;
  } else {
    C = wt * utm;
    dC = wt * dutm;
  }
  float am = s.a + 0.5f * da;
  float bm = s.b + 0.5f * db;
  float az = s.az0 + s.gaz * am;
  float A = s.ar0 + s.gar * bm + C;
  float t2 = tau * tau;
  o.f1 = db - tau * s.uz - 0.5f * t2 * az;
  o.f2 = da - tau * s.ur - 0.5f * t2 * A;
  o.f1a = -0.25f * t2 * s.gaz;
  o.f1t = -s.uz - tau * az;
  o.f2a = 1.f - 0.5f * t2 * dC;
  o.f2b = -0.25f * t2 * s.gar;
  o.f2t = -s.ur - tau * A;
  o.A = A;
  o.az = az;
  o.ut1 = ut1;
}

__device__ __forceinline__ bool interior32(const Sub32 &s, float wt, float tau, float &pda,
                                           float &pdb, unsigned &it_count) {
  // predictor with the acceleration at the start point; the centrifugal term
  // is left out when the angular step is not small (close to the axis)
  float A0 = s.ar0 + s.gar * s.b + wt * s.ut;
  if (s.rho > 0.f && tau * fabsf(s.ut) < 0.25f * s.rho) A0 += s.ut * s.ut / s.rho;
  float da = tau * (s.ur + 0.5f * tau * A0);
  float db = tau * (s.uz + 0.5f * tau * (s.az0 + s.gaz * s.a));
  if (s.P != 0.f && s.rho + da <= 0.f) da = -0.5f * s.rho;
  for (int it = 0; it < kNewtonMax32; ++it) {
    Res32 o;
    eval32(s, wt, da, db, tau, o);
    it_count++;
    // [f1a 1; f2a f2b] [xa; xb] = -[f1; f2]
    float det = o.f1a * o.f2b - o.f2a;
    if (!(det != 0.f) || !isfinite(det)) return false;
    float idet = __fdividef(1.f, det);
    float xa = (-o.f1 * o.f2b + o.f2) * idet;
    float xb = (-o.f1a * o.f2 + o.f2a * o.f1) * idet;
    float nda = da + xa, ndb = db + xb;
    if (s.P != 0.f && s.rho + nda <= 0.f) nda = 0.5f * (da - s.rho);
    float ca = fabsf(nda - da), cb = fabsf(ndb - db);
    da = nda;
    db = ndb;
    if (!isfinite(da) || !isfinite(db)) return false;
    if (ca <= tol_r(s.rho + da, da) && cb <= tol_x(db)) {
      pda = da;
      pdb = db;
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ bool landing32(const Sub32 &s, float wt, int dir, float X, float t0,
                                          float oth0, float &ptau, float &poth,
                                          unsigned &it_count) {
  float tau = t0, oth = oth0;
  for (int it = 0; it < kNewtonMax32; ++it) {
    float da = dir == 0 ? X : oth;
    float db = dir == 0 ? oth : X;
    Res32 o;
    eval32(s, wt, da, db, tau, o);
    it_count++;
    float gF, gFo, gFt, gO, gOo, gOt;
    if (dir == 0) {
      gO = o.f1; gOo = 1.f; gOt = o.f1t;
      if (X != 0.f) {
        gF = o.f2; gFo = o.f2b; gFt = o.f2t;
      } else {
        gF = -s.ur - 0.5f * tau * o.A;
        gFo = -0.25f * tau * s.gar;
        gFt = -0.5f * o.A;
      }
    } else {
      gO = o.f2; gOo = o.f2a; gOt = o.f2t;
      if (X != 0.f) {
        gF = o.f1; gFo = o.f1a; gFt = o.f1t;
      } else {
        gF = -s.uz - 0.5f * tau * o.az;
        gFo = -0.25f * tau * s.gaz;
        gFt = -0.5f * o.az;
      }
    }
    float det = gFo * gOt - gFt * gOo;
    if (!(det != 0.f) || !isfinite(det)) return false;
    float idet = __fdividef(1.f, det);
    float xo = (-gF * gOt + gO * gFt) * idet;
    float xt = (-gFo * gO + gOo * gF) * idet;
    float noth = oth + xo, ntau = tau + xt;
    if (dir == 1 && s.P != 0.f && s.rho + noth <= 0.f) noth = 0.5f * (oth - s.rho);
    float co = fabsf(noth - oth), ct = fabsf(ntau - tau);
    oth = noth;
    tau = ntau;
    if (!isfinite(oth) || !isfinite(tau)) return false;
    float to = dir == 1 ? tol_r(s.rho + oth, oth) : tol_x(oth);
    if (co <= to && ct <= tol_x(tau)) {
      ptau = tau;
      poth = oth;
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ int transition32(int nr, int nz, int &ic, int &jc, float &a, float &b,
                                            float &ur, float &uz) {
  if (a == 1.f && ur > 0.f) {
    if (ic + 1 == nr) return 1;
    ic += 1;
    a = 0.f;
  } else if (a == 0.f && ur < 0.f) {
    if (ic == 0) ur = -ur;
    else { ic -= 1; a = 1.f; }
  }
  if (b == 1.f && uz > 0.f) {
    if (jc + 1 == nz) return 2;
    jc += 1;
    b = 0.f;
  } else if (b == 0.f && uz < 0.f) {
    if (jc == 0) return 3;
    jc -= 1;
    b = 1.f;
  }
  return 0;
}

// exact float -> double by exponent re-biasing in integer registers (no FP64
// instruction; denormals are flushed in this unit anyway)
__device__ __forceinline__ double f2d_exact(float f) {
  unsigned u = __float_as_uint(f);
  unsigned e = (u >> 23) & 0xffu;
  unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                            ((unsigned long long)(e + 896u) << 52) |
                            ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double(e == 0u ? 0ull : bits);
}

__device__ __forceinline__ unsigned long long wsum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Tally {
  unsigned err, abs, sub, fb, newton;
};

// General sub-step loop for one particle (cell crossings, faces, axis, walls,
// fallbacks); every deposit goes straight to the FP64 flux arrays.
__device__ void push_general(const PushLaunch32 &L, long long p, int c0, float a, float b,
                             float ur, float ut, float uz, const float w, Tally &T) {
  const int nr = L.g.nr, nz = L.g.nz, nz1 = nz + 1;
  const float wt = L.wbt;
  if (c0 < 0 || c0 >= nr * nz) return;
  int ic = c0 / nz, jc = c0 - (c0 / nz) * nz;
  float tau = 1.f;
  float tT = tau;
  int nsub = 0;
  int absorbed = transition32(nr, nz, ic, jc, a, b, ur, uz);
  while (tau > 0.f && !absorbed) {
    if (++nsub > kNsubMax) {
      T.err++;
      break;
    }
    Sub32 s;
    s.ar0 = L.ar[ic * nz1 + jc];
    s.gar = L.ar[ic * nz1 + jc + 1] - s.ar0;
    s.az0 = L.az[ic * nz + jc];
    s.gaz = L.az[(ic + 1) * nz + jc] - s.az0;
    s.a = a; s.b = b;
    s.rho = (float)ic + a;
    s.ur = ur; s.ut = ut; s.uz = uz;
    s.P = s.rho * ut + 0.5f * wt * s.rho * s.rho;
    float da, db;
    if (!interior32(s, wt, tT, da, db, T.newton)) {
      tT *= 0.5f;
      T.fb++;
      continue;
    }
    float a1 = a + da, b1 = b + db;
    float step_t;
    int land_dir = -1;
    float land_face = 0.f;
    if (a1 >= 0.f && a1 <= 1.f && b1 >= 0.f && b1 <= 1.f) {
      step_t = tT;
    } else {
      float best_t = 0.f, best_oth = 0.f, best_face = 0.f;
      int best_dir = -1;
#pragma unroll 1
      for (int dir = 0; dir < 2; ++dir) {
        float x0 = dir == 0 ? a : b;
        float x1 = dir == 0 ? a1 : b1;
        float dx = dir == 0 ? da : db;
        float doth = dir == 0 ? db : da;
        float face;
        if (x1 > 1.f) face = 1.f;
        else if (x1 < 0.f) face = 0.f;
        else continue;
        float X = face - x0;
        float v0 = dir == 0 ? ur : uz;
        float g0;
        if (X != 0.f) {
          g0 = tT * (X / dx);
        } else {
          float alpha = 2.f * (dx - v0 * tT) / (tT * tT);
          g0 = -2.f * v0 / alpha;
        }
        float oth0 = doth * (g0 / tT);
        float tt = 0.f, toth = 0.f;
        if (!(g0 > 0.f) || !landing32(s, wt, dir, X, g0, oth0, tt, toth, T.newton)) continue;
        if (!(tt > 0.f) || tt > tT) continue;
        float xo = (dir == 0 ? b : a) + toth;
        if (xo < 0.f || xo > 1.f) continue;
        if (best_dir < 0 || tt < best_t) {
          best_dir = dir;
          best_t = tt;
          best_oth = toth;
          best_face = face;
        }
      }
      if (best_dir < 0) {
        tT *= 0.5f;
        T.fb++;
        continue;
      }
      step_t = best_t;
      land_dir = best_dir;
      land_face = best_face;
      if (best_dir == 0) {
        da = best_face - a;
        db = best_oth;
      } else {
        db = best_face - b;
        da = best_oth;
      }
    }
    Res32 o;
    eval32(s, wt, da, db, step_t, o);
    float am = a + 0.5f * da, bm = b + 0.5f * db;
    float nur = ur + step_t * o.A;
    float nuz = uz + step_t * o.az;
    float nut = o.ut1;
    if (L.ir) {
      float fr = L.qf * w * da, fz = L.qf * w * db;
      atomicAdd(&L.ir[ic * nz1 + jc], f2d_exact(fr * (1.f - bm)));
      atomicAdd(&L.ir[ic * nz1 + jc + 1], f2d_exact(fr * bm));
      atomicAdd(&L.iz[ic * nz + jc], f2d_exact(fz * (1.f - am)));
      atomicAdd(&L.iz[(ic + 1) * nz + jc], f2d_exact(fz * am));
    }
    if (land_dir == 0) {
      a = land_face;
      b = b + db;
    } else if (land_dir == 1) {
      b = land_face;
      a = a + da;
    } else {
      a = a + da;
      b = b + db;
    }
    a = fminf(fmaxf(a, 0.f), 1.f);
    b = fminf(fmaxf(b, 0.f), 1.f);
    ur = nur; ut = nut; uz = nuz;
    tau = tau - step_t;
    T.sub++;
    absorbed = transition32(nr, nz, ic, jc, a, b, ur, uz);
    if (absorbed) break;
    tT = tau;
  }
  float vr = ur * L.icr, vt = ut * L.icr, vz = uz * L.icz;
  if (absorbed) {
    T.abs++;
    if (L.write) {
      double qw = L.q * (double)w;
      if (absorbed == 1 && L.wall_r) {
        atomicAdd(&L.wall_r[jc], qw * (1.0 - (double)b));
        atomicAdd(&L.wall_r[jc + 1], qw * (double)b);
      } else if (absorbed == 2 && L.wall_zl) {
        atomicAdd(&L.wall_zl[ic], qw * (1.0 - (double)a));
        atomicAdd(&L.wall_zl[ic + 1], qw * (double)a);
      } else if (absorbed == 3 && L.wall_z0) {
        atomicAdd(&L.wall_z0[ic], qw * (1.0 - (double)a));
        atomicAdd(&L.wall_z0[ic + 1], qw * (double)a);
      }
    }
    if (L.ke_lost) {
      double v2 = (double)vr * vr + (double)vt * vt + (double)vz * vz;
      atomicAdd(L.ke_lost, 0.5 * L.m * (double)w * v2);
    }
  }
  if (L.write) {
    L.p.cell[p] = absorbed ? -1 : ic * nz + jc;
    L.p.a[p] = a; L.p.b[p] = b;
    L.p.vr[p] = vr; L.p.vt[p] = vt; L.p.vz[p] = vz;
  }
}

__device__ __forceinline__ void flush_counters(const PushLaunch32 &L, const Tally &T, int lane,
                                               unsigned fast_newton, unsigned fast_acc) {
  if (!L.counters) return;
  unsigned long long e0 = wsum64(T.err), e1 = wsum64(T.abs), e2 = wsum64(T.sub),
                     e3 = wsum64(T.fb), e4 = wsum64(T.newton), e5 = wsum64(fast_newton),
                     e6 = wsum64(fast_acc);
  if (lane == 0) {
    if (e0) atomicAdd(&L.counters[0], e0);
    if (e1) atomicAdd(&L.counters[1], e1);
    if (e2 + e6) atomicAdd(&L.counters[2], e2 + e6);
    if (e3) atomicAdd(&L.counters[3], e3);
    // algorithmic FP32 operations: general path 75 per Newton iteration and 93
    // per accepted sub-step; fast path 38 per Newton iteration and 27 per accept
    unsigned long long fl = 75ull * e4 + 93ull * e2 + 38ull * e5 + 27ull * e6;
    if (fl) atomicAdd(&L.counters[4], fl);
  }
}

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
          if (fabsf(xa) <= tol_r(rho + da, da) && fabsf(xb) <= tol_x(db)) {
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
    atomicAdd(&L.ir[ic * nz1 + jc], f2d_exact(hr0));
    atomicAdd(&L.ir[ic * nz1 + jc + 1], f2d_exact(hr1));
    atomicAdd(&L.iz[ic * nz + jc], f2d_exact(hz0));
    atomicAdd(&L.iz[(ic + 1) * nz + jc], f2d_exact(hz1));
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
  flush_counters(L, T, lane, fast_newton, fast_acc);
}

// Phase 2: queued particles (or all of them when queue == nullptr)
__global__ void __launch_bounds__(256) k_push_fp32_general(PushLaunch32 L) {
  const int lane = threadIdx.x & 31;
  long long count = L.queue ? (long long)*L.qcount : L.n;
  Tally T = {0, 0, 0, 0, 0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x) {
    if (L.queue) {
      push_general(L, L.queue[q], L.q_cell[q], L.q_a[q], L.q_b[q], L.q_ur[q], L.q_ut[q],
                   L.q_uz[q], L.q_w[q], T);
    } else {
      push_general(L, q, L.p.cell[q], L.p.a[q], L.p.b[q], L.p.vr[q] * L.cr, L.p.vt[q] * L.cr,
                   L.p.vz[q] * L.cz, L.p.w[q], T);
    }
  }
  flush_counters(L, T, lane, 0, 0);
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
