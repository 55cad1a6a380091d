// Rows a2 + a3 (+ a6): Crank-Nicolson particle mover with cell-crossing
// sub-steps fused with the charge-conserving deposit, FP64 form.
//
// Eq. 4 (Sec. 2.1) is integrated by the CN rule: inside one cell the
// sub-step midpoint equations are
//   dr*da = dtau*vr + dtau^2/2*(qm*Er(bm) + C(da)),  dz*db = dtau*vz + dtau^2/2*qm*Ez(am)
// (Er linear in bm, Ez linear in am: the S0xS1 / S1xS0 gather of the cell's
// edge fields at the segment midpoint), C = vt_m^2/r_m + wb*vt_m with vt' from
// the exactly conserved canonical angular momentum.  A trial sub-step over
// the remaining time is solved by Newton on (da, db); if it leaves the cell,
// the sub-step is shortened to end exactly on a face (Newton on (dtau,
// other offset)).  Each segment deposits q*w*da*S1(bm) on the two Er edges and
// q*w*db*S1(am) on the two Ez edges of the cell (Eq. 3, m = 1, flux form),
// which satisfies the discrete continuity equation node by node.
//
// Parallel layout: one thread per particle of a cell-sorted SoA; a thread
// keeps the deposit of its home cell in registers and a warp reduces runs of
// lanes with the same home cell before one atomic per edge; sub-steps in
// other cells (after a crossing) use direct FP64 atomics.
//
// Compiled with --fmad=false: the arithmetic is performed in the same order
// as the FP64 oracle so that both take the same branches.
#include "pic_internal.cuh"

namespace pic {
namespace {

struct Sub {
  double er0, ger, ez0, gez;
  double a, b, r, vr, vt, vz, pth;
};

struct Res {
  double f1, f2, f1a, f1b, f1t, f2a, f2b, f2t, C, vt1;
};

struct Consts {
  double dr, dz, qm, wb;
};

__device__ __forceinline__ void eval(const Consts &K, const Sub &s, double da, double db,
                                     double dt, Res &o) {
  double r1 = s.r + da * K.dr;
  double rm = 0.5 * (s.r + r1);
  double vt1, dvt1;
  if (r1 > 0.0) {
    vt1 = (s.pth - 0.5 * K.wb * r1 * r1) / r1;
    dvt1 = K.dr * (-s.pth / (r1 * r1) - 0.5 * K.wb);
  } else {
    vt1 = s.vt;
    dvt1 = 0.0;
  }
  double vtm = 0.5 * (s.vt + vt1);
  double dvtm = 0.5 * dvt1;
  double C, dC;
  if (rm > 0.0) {
    C = vtm * vtm / rm + K.wb * vtm;
    dC = 2.0 * vtm * dvtm / rm - vtm * vtm * (0.5 * K.dr) / (rm * rm) + K.wb * dvtm;
  } else {
    C = K.wb * vtm;
    dC = K.wb * dvtm;
  }
  double am = s.a + 0.5 * da;
  double bm = s.b + 0.5 * db;
  double ez = s.ez0 + s.gez * am;
  double er = s.er0 + s.ger * bm;
  double ar = K.qm * er + C;
  double dt2 = dt * dt;
  o.f1 = K.dz * db - dt * s.vz - 0.5 * dt2 * (K.qm * ez);
  o.f2 = K.dr * da - dt * s.vr - 0.5 * dt2 * ar;
  o.f1a = -0.25 * dt2 * K.qm * s.gez;
  o.f1b = K.dz;
  o.f1t = -s.vz - dt * (K.qm * ez);
  o.f2a = K.dr - 0.5 * dt2 * dC;
  o.f2b = -0.25 * dt2 * K.qm * s.ger;
  o.f2t = -s.vr - dt * ar;
  o.C = C;
  o.vt1 = vt1;
}

// Algorithmic FP64 operation counts of the source (add, sub, mul, div each
// count 1): one residual/Jacobian evaluation, one Newton update, the rest of
// an accepted sub-step, and the per-sub-step set-up.
constexpr unsigned kFlopEval = 68, kFlopNewton = 17, kFlopAccept = 30, kFlopSetup = 9;

__device__ bool solve_interior(const Consts &K, const Sub &s, double dt, double &pda,
                               double &pdb, unsigned long long &flops) {
  double da = dt * s.vr / K.dr;
  double db = dt * s.vz / K.dz;
  if (s.pth != 0.0 && s.r + da * K.dr <= 0.0) da = -0.5 * s.r / K.dr;
  for (int it = 0; it < kNewtonMax; ++it) {
    Res o;
    eval(K, s, da, db, dt, o);
    flops += kFlopEval + kFlopNewton;
    double det = o.f1a * o.f2b - o.f1b * o.f2a;
    if (!(det != 0.0) || !isfinite(det)) return false;
    double xa = (-o.f1 * o.f2b + o.f2 * o.f1b) / det;
    double xb = (-o.f1a * o.f2 + o.f2a * o.f1) / det;
    double nda = da + xa;
    double ndb = db + xb;
    if (s.pth != 0.0 && s.r + nda * K.dr <= 0.0) nda = 0.5 * (da - s.r / K.dr);
    double ca = fabs(nda - da), cb = fabs(ndb - db);
    da = nda;
    db = ndb;
    if (!isfinite(da) || !isfinite(db)) return false;
    if (ca <= kTolX && cb <= kTolX) {
      pda = da;
      pdb = db;
      return true;
    }
  }
  return false;
}

// landing on a face normal to direction dir (0: xi, 1: eta) with fixed offset change X
__device__ bool solve_landing(const Consts &K, const Sub &s, int dir, double X, double dt0,
                              double oth0, double tscale, double &pdt, double &poth,
                              unsigned long long &flops) {
  double dt = dt0, oth = oth0;
  for (int it = 0; it < kNewtonMax; ++it) {
    double da = dir == 0 ? X : oth;
    double db = dir == 0 ? oth : X;
    Res o;
    eval(K, s, da, db, dt, o);
    flops += kFlopEval + kFlopNewton;
    double gF, gFo, gFt, gO, gOo, gOt;
    if (dir == 0) {
      gO = o.f1; gOo = o.f1b; gOt = o.f1t;
      if (X != 0.0) {
        gF = o.f2; gFo = o.f2b; gFt = o.f2t;
      } else {
        double bm = s.b + 0.5 * db;
        double ar = K.qm * (s.er0 + s.ger * bm) + o.C;
        gF = -s.vr - 0.5 * dt * ar;
        gFo = -0.25 * dt * K.qm * s.ger;
        gFt = -0.5 * ar;
      }
    } else {
      gO = o.f2; gOo = o.f2a; gOt = o.f2t;
      if (X != 0.0) {
        gF = o.f1; gFo = o.f1a; gFt = o.f1t;
      } else {
        double am = s.a + 0.5 * da;
        double ez = K.qm * (s.ez0 + s.gez * am);
        gF = -s.vz - 0.5 * dt * ez;
        gFo = -0.25 * dt * K.qm * s.gez;
        gFt = -0.5 * ez;
      }
    }
    double det = gFo * gOt - gFt * gOo;
    if (!(det != 0.0) || !isfinite(det)) return false;
    double xo = (-gF * gOt + gO * gFt) / det;
    double xt = (-gFo * gO + gOo * gF) / det;
    double noth = oth + xo;
    double ndt = dt + xt;
    if (dir == 1 && s.pth != 0.0 && s.r + noth * K.dr <= 0.0) noth = 0.5 * (oth - s.r / K.dr);
    double co = fabs(noth - oth), ct = fabs(ndt - dt);
    oth = noth;
    dt = ndt;
    if (!isfinite(oth) || !isfinite(dt)) return false;
    if (co <= kTolX && ct <= kTolT * tscale) {
      pdt = dt;
      poth = oth;
      return true;
    }
  }
  return false;
}

// face transition: 0 stay, 1 absorbed at r = R, 2 at z = L, 3 at z = 0
__device__ __forceinline__ int transition(int nr, int nz, int &ic, int &jc, double &a, double &b,
                                          double &vr, double &vz) {
  if (a == 1.0 && vr > 0.0) {
    if (ic + 1 == nr) return 1;
    ic += 1;
    a = 0.0;
  } else if (a == 0.0 && vr < 0.0) {
    if (ic == 0) vr = -vr;
    else { ic -= 1; a = 1.0; }
  }
  if (b == 1.0 && vz > 0.0) {
    if (jc + 1 == nz) return 2;
    jc += 1;
    b = 0.0;
  } else if (b == 0.0 && vz < 0.0) {
    if (jc == 0) return 3;
    jc -= 1;
    b = 1.0;
  }
  return 0;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// General path: every particle (queue == nullptr) or the queued records of
// the fast kernel; grid-stride, warp-uniform iterations.
__global__ void __launch_bounds__(128) k_push_fp64(PushLaunch L) {
  const int lane = threadIdx.x & 31;
  const int nr = L.g.nr, nz = L.g.nz;
  const int nz1 = nz + 1;
  Consts K;
  K.dr = L.g.dr; K.dz = L.g.dz; K.qm = L.qm; K.wb = L.wb;
  const long long count = L.queue ? (long long)*L.qcount : L.n;
  unsigned long long c_err = 0, c_abs = 0, c_sub = 0, c_fb = 0, c_flop = 0;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < count;
       base += (long long)gridDim.x * blockDim.x) {
  const long long t = base + threadIdx.x;
  int home = -1;
  double hr0 = 0.0, hr1 = 0.0, hz0 = 0.0, hz1 = 0.0;  // home-cell deposit
  double kel = 0.0;

  if (t < count) {
    long long p;
    int c0;
    double a, b, vr, vt, vz, w_;
    if (L.queue) {
      p = L.queue[t];
      c0 = L.q_cell[t];
      a = L.q_a[t]; b = L.q_b[t]; vr = L.q_vr[t]; vt = L.q_vt[t]; vz = L.q_vz[t]; w_ = L.q_w[t];
    } else {
      p = t;
      c0 = L.p.cell[p];
      a = L.p.a[p]; b = L.p.b[p]; vr = L.p.vr[p]; vt = L.p.vt[p]; vz = L.p.vz[p]; w_ = L.p.w[p];
    }
    if (c0 >= 0 && c0 < nr * nz) {
      int ic = c0 / nz, jc = c0 - (c0 / nz) * nz;
      const double w = w_;
      const double qw = L.q * w;
      double tau = L.dt;
      double dtT = tau;
      int nsub = 0;
      int absorbed = transition(nr, nz, ic, jc, a, b, vr, vz);
      home = ic * nz + jc;
      const int hic = ic, hjc = jc;
      while (tau > 0.0 && !absorbed) {
        if (++nsub > kNsubMax) {
          c_err++;
          break;
        }
        Sub s;
        s.er0 = L.er[ic * nz1 + jc];
        s.ger = L.er[ic * nz1 + jc + 1] - s.er0;
        s.ez0 = L.ez[ic * nz + jc];
        s.gez = L.ez[(ic + 1) * nz + jc] - s.ez0;
        s.a = a; s.b = b;
        s.r = ((double)ic + a) * K.dr;
        s.vr = vr; s.vt = vt; s.vz = vz;
        s.pth = s.r * vt + 0.5 * K.wb * s.r * s.r;
        c_flop += kFlopSetup;

        double da, db;
        if (!solve_interior(K, s, dtT, da, db, c_flop)) {
          dtT *= 0.5;
          c_fb++;
          continue;
        }
        double a1 = a + da, b1 = b + db;
        double step_dt;
        int land_dir = -1;
        double land_face = 0.0;
        if (a1 >= 0.0 && a1 <= 1.0 && b1 >= 0.0 && b1 <= 1.0) {
          step_dt = dtT;
        } else {
          double best_dt = 0.0, best_oth = 0.0, best_face = 0.0;
          int best_dir = -1;
          for (int dir = 0; dir < 2; ++dir) {
            double x0 = dir == 0 ? a : b;
            double x1 = dir == 0 ? a1 : b1;
            double dx = dir == 0 ? da : db;
            double doth = dir == 0 ? db : da;
            double face;
            if (x1 > 1.0) face = 1.0;
            else if (x1 < 0.0) face = 0.0;
            else continue;
            double X = face - x0;
            double v0 = dir == 0 ? vr : vz;
            double h = dir == 0 ? K.dr : K.dz;
            double g0;
            if (X != 0.0) {
              g0 = dtT * (X / dx);
            } else {
              double alpha = 2.0 * (dx * h - v0 * dtT) / (dtT * dtT);
              g0 = -2.0 * v0 / alpha;
            }
            double oth0 = doth * (g0 / dtT);
            double tdt = 0.0, toth = 0.0;
            if (!(g0 > 0.0) || !solve_landing(K, s, dir, X, g0, oth0, dtT, tdt, toth, c_flop))
              continue;
            if (!(tdt > 0.0) || tdt > dtT) continue;
            double xo = (dir == 0 ? b : a) + toth;
            if (xo < 0.0 || xo > 1.0) continue;
            if (best_dir < 0 || tdt < best_dt) {
              best_dir = dir;
              best_dt = tdt;
              best_oth = toth;
              best_face = face;
            }
          }
          if (best_dir < 0) {
            dtT *= 0.5;
            c_fb++;
            continue;
          }
          step_dt = best_dt;
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
        Res o;
        eval(K, s, da, db, step_dt, o);
        c_flop += kFlopEval + kFlopAccept;
        double am = a + 0.5 * da, bm = b + 0.5 * db;
        double nvr = vr + step_dt * (K.qm * (s.er0 + s.ger * bm) + o.C);
        double nvz = vz + step_dt * (K.qm * (s.ez0 + s.gez * am));
        double nvt = o.vt1;
        // deposit of this segment (Eq. 3, flux form)
        double fr = qw * da;
        double fz = qw * db;
        double d_r0 = fr * (1.0 - bm), d_r1 = fr * bm;
        double d_z0 = fz * (1.0 - am), d_z1 = fz * am;
        if (ic == hic && jc == hjc) {
          hr0 += d_r0; hr1 += d_r1; hz0 += d_z0; hz1 += d_z1;
        } else if (L.ir) {
          atomicAdd(&L.ir[ic * nz1 + jc], d_r0);
          atomicAdd(&L.ir[ic * nz1 + jc + 1], d_r1);
          atomicAdd(&L.iz[ic * nz + jc], d_z0);
          atomicAdd(&L.iz[(ic + 1) * nz + jc], d_z1);
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
        vr = nvr; vt = nvt; vz = nvz;
        tau = tau - step_dt;
        c_sub++;
        absorbed = transition(nr, nz, ic, jc, a, b, vr, vz);
        if (absorbed) break;
        dtT = tau;
      }
      if (absorbed) {
        c_abs++;
        if (L.write) {
          if (absorbed == 1 && L.wall_r) {
            atomicAdd(&L.wall_r[jc], qw * (1.0 - b));
            atomicAdd(&L.wall_r[jc + 1], qw * b);
          } else if (absorbed == 2 && L.wall_zl) {
            atomicAdd(&L.wall_zl[ic], qw * (1.0 - a));
            atomicAdd(&L.wall_zl[ic + 1], qw * a);
          } else if (absorbed == 3 && L.wall_z0) {
            atomicAdd(&L.wall_z0[ic], qw * (1.0 - a));
            atomicAdd(&L.wall_z0[ic + 1], qw * a);
          }
        }
        kel = 0.5 * L.m * w * (vr * vr + vt * vt + vz * vz);
      }
      if (L.write) {
        L.p.cell[p] = absorbed ? -1 : ic * nz + jc;
        L.p.a[p] = a; L.p.b[p] = b;
        L.p.vr[p] = vr; L.p.vt[p] = vt; L.p.vz[p] = vz;
      }
    }
  }

  // warp: segmented reduction of home-cell deposits over runs of equal home cells
  const unsigned full = 0xffffffffu;
  int prev = __shfl_up_sync(full, home, 1);
  bool head = (lane == 0) || (prev != home);
  unsigned heads = __ballot_sync(full, head);
  // segment start lane for this lane
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
  if (L.ke_lost && kel != 0.0) atomicAdd(L.ke_lost, kel);
  }  // grid-stride
  if (L.counters) {
    c_err = warp_sum_u64(c_err);
    c_abs = warp_sum_u64(c_abs);
    c_sub = warp_sum_u64(c_sub);
    c_fb = warp_sum_u64(c_fb);
    c_flop = warp_sum_u64(c_flop);
    if (lane == 0) {
      if (c_err) atomicAdd(&L.counters[0], c_err);
      if (c_abs) atomicAdd(&L.counters[1], c_abs);
      if (c_sub) atomicAdd(&L.counters[2], c_sub);
      if (c_fb) atomicAdd(&L.counters[3], c_fb);
      if (c_flop) atomicAdd(&L.counters[4], c_flop);
    }
  }
}


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
  if (L.counters) {
    unsigned long long e2 = warp_sum_u64(n_acc), e4 = warp_sum_u64(n_newton);
    if (lane == 0) {
      if (e2) atomicAdd(&L.counters[2], e2);
      unsigned long long fl = (unsigned long long)kFlopFastNewton * e4 +
                              (unsigned long long)kFlopFastAccept * e2;
      if (fl) atomicAdd(&L.counters[4], fl);
    }
  }
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
    k_push_fp64<<<(unsigned)ng, bs, 0, s>>>(L);
  } else {
    PushLaunch A = L;
    A.queue = nullptr;
    k_push_fp64<<<(unsigned)nb, bs, 0, s>>>(A);
  }
  return cudaGetLastError();
}

}  // namespace pic
