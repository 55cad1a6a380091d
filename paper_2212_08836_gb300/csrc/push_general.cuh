// General sub-step path of the CN mover + charge-conserving deposit (rows a2,
// a3, a6; Sec. 2.1, Eqs. 3-4), shared by the FP64 and FP32 forms through the
// scalar type T.  It serves the particles the fast kernels do not finish
// (cell crossings, particles on faces, near the axis, optional external B_z).
//
// Normalised units: lengths in cells (r in units of dr, z in units of dz),
// time in units of dt (tau in [0, 1]), velocities in cells per step
// (u = v*dt/dx), accelerations alpha = (q/m)*E*dt^2/dx per species.  With
// am = a + da/2, bm = b + db/2, rho = ic + a, one sub-step of length tau solves
//   f1 = db - tau*uz - tau^2/2*alpha_z(am)                     = 0
//   f2 = da - tau*ur - tau^2/2*(alpha_r(bm) + C(da))           = 0
//   C  = ut_m^2/rho_m + wt*ut_m,  ut' = (P - wt*rho'^2/2)/rho'
// (P = rho*ut + wt*rho^2/2, the exactly conserved CN canonical angular
// momentum, wt = qm*Bz*dt) by Newton for (da, db) at given tau, or for
// (tau, other offset) when the sub-step must end exactly on a face.
#pragma once

#include "pic_internal.cuh"
#include "swfp.cuh"

namespace pic {

template <typename T>
struct Num;

template <>
struct Num<float> {
  static constexpr float tol = 1e-6f;    // offsets [cells] and tau [steps]
  static constexpr float ulpf = 4.8e-7f;  // a few ulp, relative
  // fast in-cell solve: estimated error below half an ulp of the displacement
  static constexpr float fast_rel = 6e-8f, fast_abs = 1e-12f;
  __device__ static __forceinline__ float rcp(float x) { return __fdividef(1.f, x); }
  // a product that feeds no addition (the FP64 form moves these off its FP64 pipe)
  __device__ static __forceinline__ float mul(float x, float y) { return x * y; }
  // 2x for finite x >= 0
  __device__ static __forceinline__ float twice(float x) { return x + x; }
  // 0 < x < 1 on the bits (positive floats order like their bit patterns)
  __device__ static __forceinline__ bool in01(float x) {
    const int b = __float_as_int(x);
    return b > 0 && b < 0x3F800000;
  }
  // NaN test on the bits (independent of fast-math compilation)
  __device__ static __forceinline__ bool nan_bits(float x) {
    return (__float_as_uint(x) & 0x7fffffffu) > 0x7f800000u;
  }
  // order tests on the bits (see Num<double>)
  __device__ static __forceinline__ float absb(float x) {
    return __uint_as_float(__float_as_uint(x) & 0x7fffffffu);
  }
  __device__ static __forceinline__ bool lt_abs(float x, float y) {
    return (__float_as_uint(x) & 0x7fffffffu) < __float_as_uint(y);
  }
  __device__ static __forceinline__ bool gt(float x, float c) {
    return __float_as_int(x) > __float_as_int(c);
  }
  __device__ static __forceinline__ bool le(float x, float y) {
    return __float_as_uint(x) <= __float_as_uint(y);
  }
  __device__ static __forceinline__ bool lt(float x, float y) {
    return __float_as_uint(x) < __float_as_uint(y);
  }
  __device__ static __forceinline__ float minb(float x, float y) {
    return __uint_as_float(min(__float_as_uint(x), __float_as_uint(y)));
  }
  __device__ static __forceinline__ float maxb(float x, float y) {
    return __uint_as_float(max(__float_as_uint(x), __float_as_uint(y)));
  }
  __device__ static __forceinline__ bool finite(float x) {
    return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
  }
  // exact float -> double by exponent re-biasing in integer registers (no FP64
  // instruction; denormals are flushed in the FP32 unit anyway)
  __device__ static __forceinline__ double to_double(float f) {
    unsigned u = __float_as_uint(f);
    unsigned e = (u >> 23) & 0xffu;
    unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                              ((unsigned long long)(e + 896u) << 52) |
                              ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double(e == 0u ? 0ull : bits);
  }
};

template <>
struct Num<double> {
  static constexpr double tol = 1e-13;
  static constexpr double ulpf = 1e-15;
  static constexpr double fast_rel = 1e-16, fast_abs = 1e-20;
  // reciprocal: the hardware approximation y (about 20 correct bits) refined
  // by one third-order step y <- y (1 + e + e^2), e = 1 - x y, the truncated
  // series of y / (1 - e) = 1/x (the cubic member of the iterations in
  // Markstein, IBM J. Res. Dev. 34, 1990): relative error e^3 < 2^-60 before
  // rounding, three FMAs; within 1 ulp of the correctly rounded 1/x (measured
  // on 2^30 arguments over 2^-300..2^300: 3e-4 of them off by one); x > 0, finite
  __device__ static __forceinline__ double rcp(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
  }
  // 0 < x < 1 with integer compares (no FP64 instruction); exact, NaN excluded
  __device__ static __forceinline__ bool in01(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x3FF0000000000000LL;
  }
  __device__ static __forceinline__ bool nan_bits(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) >
           0x7ff0000000000000ull;
  }
  // Order tests on the bits, so that the decisions take no FP64 instruction
  // (non-negative IEEE numbers order like their bit patterns):
  // |x|; |x| < y for y >= 0 (false for NaN x); x > c for c > 0 (true for a
  // positive NaN, which the callers reject later by finite()); x <= y for
  // x, y >= 0 (false for NaN x); max of x, y >= 0; finiteness
  __device__ static __forceinline__ double absb(double x) {
    return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
  }
  __device__ static __forceinline__ bool lt_abs(double x, double y) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) <
           (unsigned long long)__double_as_longlong(y);
  }
  __device__ static __forceinline__ bool gt(double x, double c) {
    return __double_as_longlong(x) > __double_as_longlong(c);
  }
  __device__ static __forceinline__ bool le(double x, double y) {
    return (unsigned long long)__double_as_longlong(x) <=
           (unsigned long long)__double_as_longlong(y);
  }
  __device__ static __forceinline__ bool lt(double x, double y) {
    return (unsigned long long)__double_as_longlong(x) <
           (unsigned long long)__double_as_longlong(y);
  }
  __device__ static __forceinline__ double minb(double x, double y) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(x),
                             b = (unsigned long long)__double_as_longlong(y);
    return __longlong_as_double((long long)(a < b ? a : b));
  }
  __device__ static __forceinline__ double maxb(double x, double y) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(x),
                             b = (unsigned long long)__double_as_longlong(y);
    return __longlong_as_double((long long)(a > b ? a : b));
  }
  __device__ static __forceinline__ bool finite(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
  }
  __device__ static __forceinline__ double to_double(double f) { return f; }
  // a product that feeds no addition: the correctly rounded integer-pipe
  // multiply (bit-identical to the FP64 pipe's, which stays free for the rest)
  __device__ static __forceinline__ double mul(double x, double y) { return sw_dmul(x, y); }
  // 2x for finite x >= 0, exactly, on the bits: a zero or subnormal doubles its
  // significand field (which carries into the exponent field when it becomes
  // normal), a normal number takes one more in its exponent field
  __device__ static __forceinline__ double twice(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return __longlong_as_double((long long)((b >> 52) == 0 ? b << 1 : b + (1ull << 52)));
  }
};

constexpr int kNewtonMaxGen = 30;

// stopping tests: the change of the r-offset is measured relative to r' close
// to the axis (where r' is small), never below a few ulp of the unknown
// (the min / max of non-negative values on their bits)
template <typename T>
__device__ __forceinline__ T tol_r(T rho1, T da) {
  const T r = Num<T>::gt(rho1, (T)0) ? Num<T>::minb(rho1, (T)1) : (T)0;
  return Num<T>::maxb(Num<T>::tol * r, Num<T>::ulpf * Num<T>::absb(da));
}
template <typename T>
__device__ __forceinline__ T tol_x(T x) {
  return Num<T>::maxb((T)Num<T>::tol, Num<T>::ulpf * Num<T>::absb(x));
}

template <typename T>
struct SubT {
  T ar0, gar, az0, gaz;
  T a, b, rho, ur, ut, uz, P;
};

template <typename T>
struct ResT {
  T f1, f2, f1a, f1t, f2a, f2b, f2t, A, az, ut1;
};

// kB = false: no external B_z (wt = 0, P = rho*ut).  Then, for rho' > 0,
// C = ut_m^2/rho_m = ut^2 (2 rho + da) / (2 rho'^2), which needs one
// reciprocal instead of two.
template <typename T, bool kB>
__device__ __forceinline__ void eval_gen(const SubT<T> &s, T wt, T da, T db, T tau, ResT<T> &o) {
  const T h = (T)0.5, q = (T)0.25, zero = (T)0, one = (T)1, two = (T)2;
  T rho1 = s.rho + da;
  T rhom = s.rho + h * da;
  T ut1, dut1;
  T C, dC;
  if (!kB && rho1 > zero) {
    T inv1 = Num<T>::rcp(rho1);
    T i2 = inv1 * inv1;
    T ut2h = h * s.ut * s.ut * i2;
    ut1 = s.P * inv1;
    C = ut2h * (s.rho + s.rho + da);
    dC = -ut2h * (s.rho + s.rho + s.rho + da) * inv1;
  } else {
    if (rho1 > zero) {
      T inv1 = Num<T>::rcp(rho1);
      ut1 = (s.P - h * wt * rho1 * rho1) * inv1;
      dut1 = -s.P * inv1 * inv1 - h * wt;
    } else {
      ut1 = s.ut;
      dut1 = zero;
    }
    T utm = h * (s.ut + ut1);
    T dutm = h * dut1;
    if (rhom > zero) {
      T invm = Num<T>::rcp(rhom);
      C = utm * utm * invm + wt * utm;
      dC = two * utm * dutm * invm - h * utm * utm * invm * invm + wt * dutm;
    } else {
      C = wt * utm;
      dC = wt * dutm;
    }
  }
  T am = s.a + h * da;
  T bm = s.b + h * db;
  T az = s.az0 + s.gaz * am;
  T A = s.ar0 + s.gar * bm + C;
  T t2 = tau * tau;
  o.f1 = db - tau * s.uz - h * t2 * az;
  o.f2 = da - tau * s.ur - h * t2 * A;
  o.f1a = -q * t2 * s.gaz;
  o.f1t = -s.uz - tau * az;
  o.f2a = one - h * t2 * dC;
  o.f2b = -q * t2 * s.gar;
  o.f2t = -s.ur - tau * A;
  o.A = A;
  o.az = az;
  o.ut1 = ut1;
}

// Early stop of the 2x2 Newton iterations, per unknown: with c the last
// correction, cp the one before and t the tolerance, the contraction rate is
// theta = c/cp; while theta < 1/2 the remaining error is below
// theta/(1-theta) c <= 2 c^2/cp (a contraction-rate bound, as in the stopping
// rule of simplified Newton iterations, Hairer & Wanner, Solving ODEs II,
// IV.8).  Accepting when that bound is below 1 % of the tolerance saves the
// confirming iteration without loosening the accuracy (no division needed).
// (c, cp, t >= 0: compared on their bits)
template <typename T>
__device__ __forceinline__ bool contracted(T c, T cp, T t) {
  return Num<T>::le(c, (T)0) || (Num<T>::lt((T)2 * c, cp) && Num<T>::le((T)200 * c * c, cp * t));
}

template <typename T, bool kB>
__device__ __forceinline__ bool interior_gen(const SubT<T> &s, T wt, T tau, T &pda, T &pdb,
                                             unsigned &it_count) {
  const T h = (T)0.5, zero = (T)0;
  // predictor with the acceleration at the start point; the centrifugal term
  // is left out when the angular step is not small (close to the axis)
  T A0 = s.ar0 + s.gar * s.b + wt * s.ut;
  if (s.rho > zero && tau * fabs(s.ut) < (T)0.25 * s.rho) A0 += s.ut * s.ut * Num<T>::rcp(s.rho);
  T da = tau * (s.ur + h * tau * A0);
  T db = tau * (s.uz + h * tau * (s.az0 + s.gaz * s.a));
  if (s.P != zero && s.rho + da <= zero) da = -h * s.rho;
  T pca = zero, pcb = zero;
  for (int it = 0; it < kNewtonMaxGen; ++it) {
    ResT<T> o;
    eval_gen<T, kB>(s, wt, da, db, tau, o);
    it_count++;
    // [f1a 1; f2a f2b] [xa; xb] = -[f1; f2]
    T det = o.f1a * o.f2b - o.f2a;
    if (!(det != zero) || !isfinite(det)) return false;
    T idet = Num<T>::rcp(det);
    T xa = (-o.f1 * o.f2b + o.f2) * idet;
    T xb = (-o.f1a * o.f2 + o.f2a * o.f1) * idet;
    T nda = da + xa, ndb = db + xb;
    if (s.P != zero && s.rho + nda <= zero) nda = h * (da - s.rho);
    T ca = Num<T>::absb(nda - da), cb = Num<T>::absb(ndb - db);
    da = nda;
    db = ndb;
    if (!isfinite(da) || !isfinite(db)) return false;
    const T ta = tol_r<T>(s.rho + da, da), tb = tol_x<T>(db);
    if ((Num<T>::le(ca, ta) && Num<T>::le(cb, tb)) ||
        (contracted(ca, pca, ta) && contracted(cb, pcb, tb))) {
      pda = da;
      pdb = db;
      return true;
    }
    pca = ca;
    pcb = cb;
  }
  return false;
}

template <typename T, bool kB>
__device__ __forceinline__ bool landing_gen(const SubT<T> &s, T wt, int dir, T X, T t0, T oth0,
                                            T &ptau, T &poth, unsigned &it_count) {
  const T h = (T)0.5, q = (T)0.25, zero = (T)0, one = (T)1;
  T tau = t0, oth = oth0;
  T pco = zero, pct = zero;
  for (int it = 0; it < kNewtonMaxGen; ++it) {
    T da = dir == 0 ? X : oth;
    T db = dir == 0 ? oth : X;
    ResT<T> o;
    eval_gen<T, kB>(s, wt, da, db, tau, o);
    it_count++;
    T gF, gFo, gFt, gO, gOo, gOt;
    if (dir == 0) {
      gO = o.f1; gOo = one; gOt = o.f1t;
      if (X != zero) {
        gF = o.f2; gFo = o.f2b; gFt = o.f2t;
      } else {  // return to the face the particle sits on: residual / tau
        gF = -s.ur - h * tau * o.A;
        gFo = -q * tau * s.gar;
        gFt = -h * o.A;
      }
    } else {
      gO = o.f2; gOo = o.f2a; gOt = o.f2t;
      if (X != zero) {
        gF = o.f1; gFo = o.f1a; gFt = o.f1t;
      } else {
        gF = -s.uz - h * tau * o.az;
        gFo = -q * tau * s.gaz;
        gFt = -h * o.az;
      }
    }
    T det = gFo * gOt - gFt * gOo;
    if (!(det != zero) || !isfinite(det)) return false;
    T idet = Num<T>::rcp(det);
    T xo = (-gF * gOt + gO * gFt) * idet;
    T xt = (-gFo * gO + gOo * gF) * idet;
    T noth = oth + xo, ntau = tau + xt;
    if (dir == 1 && s.P != zero && s.rho + noth <= zero) noth = h * (oth - s.rho);
    T co = Num<T>::absb(noth - oth), ct = Num<T>::absb(ntau - tau);
    oth = noth;
    tau = ntau;
    if (!isfinite(oth) || !isfinite(tau)) return false;
    const T to = dir == 1 ? tol_r<T>(s.rho + oth, oth) : tol_x<T>(oth), tt = tol_x<T>(tau);
    if ((Num<T>::le(co, to) && Num<T>::le(ct, tt)) ||
        (contracted(co, pco, to) && contracted(ct, pct, tt))) {
      ptau = tau;
      poth = oth;
      return true;
    }
    pco = co;
    pct = ct;
  }
  return false;
}

// Start of a face landing: on the quadratic path x(s) = v0 s + alpha s^2/2
// through the trial's end point x(tT) = dx (offsets in cells, s in steps),
// the time of the first crossing of the face at offset X from the start.  A
// face with X != 0 lies between the start and dx, so the path reaches it in
// (0, tT]: the smaller positive root, which is exact for a constant
// acceleration and keeps the solve on the first crossing of a grazing path.
// X = 0 (the face the particle sits on): the nonzero root.
template <typename T>
__device__ __forceinline__ T first_crossing(T X, T dx, T v0, T tT) {
  const T zero = (T)0, one = (T)1, two = (T)2, h = (T)0.5;
  const T it = tT == one ? one : Num<T>::rcp(tT);
  const T alpha = two * (dx - v0 * tT) * (it * it);
  if (X == zero) return -two * v0 * Num<T>::rcp(alpha);
  if (alpha == zero) return X * Num<T>::rcp(v0);
  const T disc = v0 * v0 + two * alpha * X;
  if (!(disc >= zero)) return tT * X * Num<T>::rcp(dx);
  // roots of alpha/2 s^2 + v0 s - X = 0 without cancellation: qq/(alpha/2), -X/qq
  const T sq = sqrt(disc);
  const T qq = -h * (v0 + (v0 >= zero ? sq : -sq));
  const T s1 = two * qq * Num<T>::rcp(alpha);
  const T s2 = qq != zero ? -X * Num<T>::rcp(qq) : s1;
  T sr = -one;
  if (s1 > zero) sr = s1;
  if (s2 > zero && (sr < zero || s2 < sr)) sr = s2;
  return sr > zero ? sr : tT * X * Num<T>::rcp(dx);
}

// particle on a face of its cell with its normal velocity pointing out moves to
// the neighbour cell; r = 0 reflects; walls absorb (1: r = R, 2: z = L, 3: z = 0)
template <typename T>
__device__ __forceinline__ int transition_gen(int nr, int nz, int &ic, int &jc, T &a, T &b, T &ur,
                                              T &uz) {
  const T zero = (T)0, one = (T)1;
  if (a == one && ur > zero) {
    if (ic + 1 == nr) return 1;
    ic += 1;
    a = zero;
  } else if (a == zero && ur < zero) {
    if (ic == 0) ur = -ur;
    else { ic -= 1; a = one; }
  }
  if (b == one && uz > zero) {
    if (jc + 1 == nz) return 2;
    jc += 1;
    b = zero;
  } else if (b == zero && uz < zero) {
    if (jc == 0) return 3;
    jc -= 1;
    b = one;
  }
  return 0;
}

constexpr int kFastNewtonMax = 4;
// algorithmic operations of the fast path: per Newton iteration, and per
// accepted particle (set-up, deposit terms, velocity update)
constexpr unsigned kOpFastNewton = 25, kOpFastAccept = 58;

// ---------------------------------------------------------------------------
// In-cell CN step without B_z.  With rho = ic + a, the unknowns (d, e) =
// (delta a, delta b) over tau = 1 satisfy
//   e = zb + gaz/4 * d,                  zb = uz + (az0 + gaz*a)/2
//   g(d) = k1*d - K - C(d)/2 = 0,         k1 = 1 - gar*gaz/16,
//   K = ur + (ar0 + gar*b)/2 + gar/4 * zb,
//   C(d)/2 = ut^2 (2 rho + d) / (4 (rho + d)^2)
// (C = ut_m^2 / rho_m with the CN-exact ut' = rho*ut/(rho + d)).  g' > 0 on
// d > -rho, so the root is unique.  Newton runs on the cleared forms, with
// r1 = rho + d:
//   G  = g r1^2  = (k1 d - K) r1^2 - ut^2 (2 rho + d) / 4,
//   G' = g' r1^3 = k1 r1^3 + ut^2 (3 rho + d) / 4,
// so that a step s = -g/g' = -G r1 / G' takes one reciprocal.  Newton's error
// after the step is about |g''|/(2 g') s^2 with |g''| = ut^2 (4 rho + d) /
// (2 r1^4), i.e. ut^2 (4 rho + d) s^2 / (4 r1 G'); the iterate is accepted when
// twice that estimate is below half an ulp of d (the CN velocity u' = 2d - u
// must not amplify an unconverged d), tested without a division.
template <typename T>
__device__ __forceinline__ bool fast_solve(T rho, T ut, T K, T k1, T &pd, unsigned &nit) {
  typedef Num<T> N;
  const T zero = (T)0;
  // rho >= 0 and the squares are non-negative: the doublings are exact bit edits
  const T qut2 = N::mul(N::mul(ut, ut), (T)0.25), hut2 = N::twice(qut2);
  const T r2 = N::twice(rho), r3 = r2 + rho, r4 = N::twice(r2);
  T d = K;
#pragma unroll 1
  for (int it = 0; it < kFastNewtonMax; ++it) {
    const T r1 = rho + d;
    if (!N::gt(r1, zero)) return false;
    const T R2 = N::mul(r1, r1);
    const T G = N::mul(k1 * d - K, R2) - qut2 * (r2 + d);
    const T Gp = k1 * N::mul(R2, r1) + N::mul(qut2, r3 + d);
    const T st = -N::mul(N::mul(G, r1), N::rcp(Gp));
    const T lhs = N::mul(N::mul(hut2, r4 + d), N::mul(st, st));
    d += st;
    nit++;
    const T tol = N::maxb(N::mul(N::fast_rel, N::absb(d)), (T)N::fast_abs);
    if (N::le(lhs, N::mul(N::mul(tol, r1), Gp))) {
      pd = d;
      return N::finite(d);
    }
  }
  return false;
}

// Interior sub-step of length tau without B_z through the same scalar
// reduction (tau-scaled coefficients; ut enters as tau*ut); false when the
// reduction does not apply (close to the axis) or does not converge
template <typename T>
__device__ __forceinline__ bool scalar_interior(const SubT<T> &s, T tau, T &pda, T &pdb,
                                                unsigned &nit) {
  const T h = (T)0.5, q = (T)0.25, one = (T)1, zero = (T)0;
  const T t2 = tau * tau, tut = tau * s.ut;
  if (!(s.rho > zero) || !(fabs(tut) < q * s.rho)) return false;
  const T zb = tau * s.uz + h * t2 * (s.az0 + s.gaz * s.a);
  const T K = tau * s.ur + h * t2 * (s.ar0 + s.gar * s.b) + q * t2 * s.gar * zb;
  const T k1 = one - (T)0.0625 * t2 * t2 * s.gar * s.gaz;
  T d;
  if (!(k1 > h) || !fast_solve<T>(s.rho, tut, K, k1, d, nit)) return false;
  pda = d;
  pdb = zb + q * t2 * s.gaz * d;
  return true;
}

// Landing on a z-face without B_z through the scalar reduction of the
// in-cell system (Eq. 4 in the normalised units above).  With the landing
// offset db = X fixed, the r-equation of a sub-step of length tau is the
// in-cell scalar equation in d = da with k1 = 1, K(tau) = tau ur + tau^2/2 Ar,
// Ar = ar0 + gar (b + X/2), and ut -> tau ut (solved by fast_solve); the
// z-equation F(tau) = tau uz + tau^2/2 (az0 + gaz (a + d/2)) - X = 0 is then one
// equation in tau, solved by Newton with dF/dtau = uz + tau Az + tau^2/4 gaz
// dd/dtau, dd/dtau ~ ur + tau (Ar + C(d)).  The root is that of the 2x2
// landing system (landing_gen); false when the reduction does not apply
// (close to the axis) or does not converge.
template <typename T>
__device__ __forceinline__ bool landing_z_scalar(const SubT<T> &s, T X, T t0, T &ptau, T &pda,
                                                 unsigned &nit) {
  typedef Num<T> N;
  const T h = (T)0.5, q = (T)0.25, zero = (T)0, one = (T)1;
  if (!(s.rho > zero)) return false;
  const T Ar = s.ar0 + s.gar * (s.b + h * X);
  const T aza = s.az0 + s.gaz * s.a;
  const T ut2 = s.ut * s.ut;
  T tau = t0, pct = zero;
  for (int it = 0; it < kNewtonMaxGen; ++it) {
    const T tut = tau * s.ut;
    if (!(tau > zero) || !(fabs(tut) < q * s.rho)) return false;
    T d;
    if (!fast_solve<T>(s.rho, tut, tau * s.ur + h * tau * tau * Ar, one, d, nit)) return false;
    const T Az = aza + h * s.gaz * d;
    const T F = tau * s.uz + h * tau * tau * Az - X;
    const T i1 = N::rcp(s.rho + d);
    const T C = h * ut2 * (s.rho + s.rho + d) * (i1 * i1);
    const T dF = s.uz + tau * Az + q * tau * tau * s.gaz * (s.ur + tau * (Ar + C));
    if (!(dF != zero)) return false;
    const T st = -F * N::rcp(dF);
    tau += st;
    if (!N::finite(tau)) return false;
    const T ct = N::absb(st), tt = tol_x<T>(tau);
    if (N::le(ct, tt) || contracted(ct, pct, tt)) {
      // the radial offset at the converged tau (the last d belongs to the tau
      // before the update)
      const T tut1 = tau * s.ut;
      if (!(tau > zero) || !(fabs(tut1) < q * s.rho) ||
          !fast_solve<T>(s.rho, tut1, tau * s.ur + h * tau * tau * Ar, one, d, nit))
        return false;
      ptau = tau;
      pda = d;
      return true;
    }
    pct = ct;
  }
  return false;
}

// The same landing as one Newton iteration on the pair (tau, d): the cleared
// in-cell radial equation of a sub-step of length tau with db = X,
//   G(tau, d) = (d - K) r1^2 - (tau ut)^2 (2 rho + d) / 4 = 0,
//   K = tau ur + tau^2/2 Ar,  r1 = rho + d,
// (fast_solve's form with k1 = 1) and the z-equation
//   F(tau, d) = tau uz + tau^2/2 (az0 + gaz (a + d/2)) - X = 0,
// with their exact partial derivatives: one 2x2 step per iteration instead of
// a scalar solve inside each step in tau, in plain arithmetic (the FP64 form's
// integer-pipe products stay in the in-cell kernel).  Start: (t0, d0).  The
// root is that of landing_z_scalar and of the 2x2 landing system
// (landing_gen); false when the reduction does not apply (close to the axis)
// or does not converge.
template <typename T>
__device__ __forceinline__ bool landing_z_joint(const SubT<T> &s, T X, T t0, T d0, T &ptau,
                                                T &pda, unsigned &nit) {
  typedef Num<T> N;
  const T h = (T)0.5, q = (T)0.25, zero = (T)0;
  if (!(s.rho > zero)) return false;
  const T Ar = s.ar0 + s.gar * (s.b + h * X);
  const T aza = s.az0 + s.gaz * s.a;
  const T ut2 = s.ut * s.ut, r2 = s.rho + s.rho;
  T tau = t0, d = d0, pct = zero, pcd = zero;
  if (!(s.rho + d > zero)) d = zero;
  for (int it = 0; it < kNewtonMaxGen; ++it) {
    if (!(tau > zero) || !(fabs(tau * s.ut) < q * s.rho)) return false;
    const T r1 = s.rho + d;
    const T R2 = r1 * r1, t2 = tau * tau;
    const T qut2 = q * t2 * ut2;
    const T e = d - (tau * s.ur + h * t2 * Ar);
    const T G = e * R2 - qut2 * (r2 + d);
    const T Gd = R2 + (e + e) * r1 - qut2;
    const T Gt = -(s.ur + tau * Ar) * R2 - h * tau * ut2 * (r2 + d);
    const T Az = aza + h * s.gaz * d;
    const T F = tau * s.uz + h * t2 * Az - X;
    const T Ft = s.uz + tau * Az;
    const T Fd = q * t2 * s.gaz;
    const T det = Gd * Ft - Gt * Fd;
    nit++;
    if (!(det != zero) || !N::finite(det)) return false;
    const T idet = N::rcp(det);
    T nd = d + (Gt * F - G * Ft) * idet;
    const T ntau = tau + (Fd * G - Gd * F) * idet;
    if (s.rho + nd <= zero) nd = h * (d - s.rho);
    const T cd = N::absb(nd - d), ct = N::absb(ntau - tau);
    d = nd;
    tau = ntau;
    if (!N::finite(d) || !N::finite(tau)) return false;
    const T td = tol_r<T>(s.rho + d, d), tt = tol_x<T>(tau);
    if ((N::le(cd, td) && N::le(ct, tt)) || (contracted(cd, pcd, td) && contracted(ct, pct, tt))) {
      if (!(tau > zero) || !(fabs(tau * s.ut) < q * s.rho)) return false;
      ptau = tau;
      pda = d;
      return true;
    }
    pcd = cd;
    pct = ct;
  }
  return false;
}

struct Tally {
  unsigned err, abs, sub, fb, newton, snewton;  // snewton: scalar Newton iterations
  unsigned jnewton;                              // joint (tau, d) landing iterations
};

// T: the arithmetic type of the path; S: the scalar type of the particle store
// and of the accelerations (S = float, T = double: FP32 particles pushed in
// FP64 arithmetic, results rounded to FP32 once at the end)
template <typename T, typename S = T>
struct GenArgs {
  int nr, nz;
  const S *ar, *az;      // normalised accelerations of the species
  T wt, icr, icz, cz;    // qm*Bz*dt; dr/dt, dz/dt; dt/dz
  RadialMapT<T> rm;      // per-cell radial scales (mapped mesh)
  double q, m;
  T qf;                  // q in T
  double *ir, *iz;       // crossed charge [C]
  int write, oop;        // write the new state; out of place into dst
  PartsT<S> p, dst;
  double *wall_z0, *wall_zl, *wall_r;
  double *ke_lost;
  unsigned long long *hist;  // accepted sub-steps per particle, 16 bins (nullptr: off)
};

// radial face crossing on a mapped mesh: the normalised radial and azimuthal
// velocities follow the new cell's width
template <typename T>
__device__ __forceinline__ void rescale_radial(const RadialMapT<T> &rm, int ic_old, int ic_new,
                                               T &ur, T &ut) {
  if (ic_new != ic_old && (ic_old < rm.xa || ic_new < rm.xa)) {
    const T f = rm.icrr(ic_old) * rm.crr(ic_new);
    ur *= f;
    ut *= f;
  }
}

// The sub-step loop of one particle from a point of its step: cell (ic, jc),
// offsets (a, b), normalised velocities, the time tau left of the step, nsub
// sub-steps tried and nacc accepted so far; (tr_da, tr_db): the converged
// interior solution of the next sub-step over tau from a start strictly inside
// the cell (NaN: none).  Finishes the step: tallies and (write) the new state.
template <typename T, bool kB, typename S = T>
__device__ void push_sub(const GenArgs<T, S> &L, long long p, int ic, int jc, T a, T b, T ur,
                         T ut, T uz, const T w, T tr_da, T tr_db, T tau, int nsub, int nacc,
                         Tally &Tl) {
  const T zero = (T)0, one = (T)1, h = (T)0.5, two = (T)2;
  const int nr = L.nr, nz = L.nz, nz1 = nz + 1;
  const T wt = L.wt;
  T tT = tau;
  const int nsub0 = nsub;
  int ic_prev = ic;
  int absorbed = transition_gen<T>(nr, nz, ic, jc, a, b, ur, uz);
  rescale_radial<T>(L.rm, ic_prev, ic, ur, ut);
  while (tau > zero && !absorbed) {
    if (++nsub > kNsubMax) {
      Tl.err++;
      break;
    }
    SubT<T> s;
    s.ar0 = (T)L.ar[ic * nz1 + jc];
    s.gar = (T)L.ar[ic * nz1 + jc + 1] - s.ar0;
    s.az0 = (T)L.az[ic * nz + jc];
    s.gaz = (T)L.az[(ic + 1) * nz + jc] - s.az0;
    s.a = a; s.b = b;
    s.rho = L.rm.rho0(ic) + a;
    s.ur = ur; s.ut = ut; s.uz = uz;
    s.P = s.rho * ut + h * wt * s.rho * s.rho;
    T da, db;
    // tight: converged to half an ulp (scalar solves), so the CN velocity
    // relation u' = 2 dx / tau - u may replace an evaluation
    bool tight = true;
    if (nsub == nsub0 + 1 && !Num<T>::nan_bits(tr_da)) {
      da = tr_da;
      db = tr_db;
    } else if (!kB && scalar_interior<T>(s, tT, da, db, Tl.snewton)) {
    } else if (interior_gen<T, kB>(s, wt, tT, da, db, Tl.newton)) {
      tight = false;
    } else {
      tT *= h;
      Tl.fb++;
      continue;
    }
    T a1 = a + da, b1 = b + db;
    T step_t;
    int land_dir = -1;
    T land_face = zero;
    if (a1 >= zero && a1 <= one && b1 >= zero && b1 <= one) {
      step_t = tT;
    } else {
      T best_t = zero, best_oth = zero, best_face = zero;
      int best_dir = -1;
#pragma unroll 1
      for (int dir = 0; dir < 2; ++dir) {
        T x0 = dir == 0 ? a : b;
        T x1 = dir == 0 ? a1 : b1;
        T dx = dir == 0 ? da : db;
        T doth = dir == 0 ? db : da;
        T face;
        if (x1 > one) face = one;
        else if (x1 < zero) face = zero;
        else continue;
        T X = face - x0;
        T v0 = dir == 0 ? ur : uz;
        // the start only seeds Newton: FP32 arithmetic is enough, and keeps the
        // square root and reciprocals off the FP64 form's narrow FP64 pipe
        const T g0 = (T)first_crossing<float>((float)X, (float)dx, (float)v0, (float)tT);
        T oth0 = doth * (g0 * (tT == one ? one : Num<T>::rcp(tT)));
        T tt = zero, toth = zero;
        if (!(g0 > zero)) continue;
        // FP32: a z-face (most crossings: cells are flat in z) through the
        // scalar reduction, else (or if it does not apply) the 2x2 landing
        // system (the FP64 form keeps the 2x2 solve: its scalar solves run on
        // the integer pipes and measured slower in this divergent kernel)
        if (!(!kB && sizeof(T) == 4 && dir == 1 && X != zero &&
              landing_z_scalar<T>(s, X, g0, tt, toth, Tl.snewton)) &&
            !landing_gen<T, kB>(s, wt, dir, X, g0, oth0, tt, toth, Tl.newton))
          continue;
        if (!(tt > zero) || tt > tT) continue;
        T xo = (dir == 0 ? b : a) + toth;
        if (xo < zero || xo > one) continue;
        if (best_dir < 0 || tt < best_t) {
          best_dir = dir;
          best_t = tt;
          best_oth = toth;
          best_face = face;
        }
      }
      if (best_dir < 0) {
        tT *= h;
        Tl.fb++;
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
    ResT<T> o;
    T am = a + h * da, bm = b + h * db;
    T nur, nuz, nut;
    if (!kB && tight && land_dir < 0 && s.rho + da > zero) {
      const T it = step_t == one ? one : Num<T>::rcp(step_t);
      nur = two * da * it - ur;
      nuz = two * db * it - uz;
      nut = s.P * Num<T>::rcp(s.rho + da);
    } else {
      eval_gen<T, kB>(s, wt, da, db, step_t, o);
      nur = ur + step_t * o.A;
      nuz = uz + step_t * o.az;
      nut = o.ut1;
    }
    if (L.ir) {
      T fr = L.qf * w * da, fz = L.qf * w * db;
      atomicAdd(&L.ir[ic * nz1 + jc], Num<T>::to_double(fr * (one - bm)));
      atomicAdd(&L.ir[ic * nz1 + jc + 1], Num<T>::to_double(fr * bm));
      atomicAdd(&L.iz[ic * nz + jc], Num<T>::to_double(fz * (one - am)));
      atomicAdd(&L.iz[(ic + 1) * nz + jc], Num<T>::to_double(fz * am));
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
    a = fmin(fmax(a, zero), one);
    b = fmin(fmax(b, zero), one);
    ur = nur; ut = nut; uz = nuz;
    tau = tau - step_t;
    Tl.sub++;
    nacc++;
    ic_prev = ic;
    absorbed = transition_gen<T>(nr, nz, ic, jc, a, b, ur, uz);
    if (absorbed) break;
    rescale_radial<T>(L.rm, ic_prev, ic, ur, ut);
    tT = tau;
  }
  if (L.hist) atomicAdd(&L.hist[nacc <= 1 ? 0 : (nacc < 16 ? nacc - 1 : 15)], 1ull);
  const T icr = L.rm.icrr(ic);
  T vr = ur * icr, vt = ut * icr, vz = uz * L.icz;
  if (absorbed) {
    Tl.abs++;
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
    L.dst.cell[p] = absorbed ? -1 : ic * nz + jc;
    L.dst.a[p] = (S)a; L.dst.b[p] = (S)b;
    L.dst.vr[p] = (S)vr; L.dst.vt[p] = (S)vt; L.dst.vz[p] = (S)vz;
    if (L.oop) {
      L.dst.w[p] = (S)w;
      L.dst.id[p] = L.p.id[p];
    }
  }
}

// one particle from its start state (offsets a, b; physical velocities);
// (tr_da, tr_db): the converged interior solution of the whole step from a
// start strictly inside the cell (NaN: none), which replaces the first
// interior solve
template <typename T, bool kB, typename S = T>
__device__ void push_general(const GenArgs<T, S> &L, long long p, int c0, T a, T b, T vr0, T vt0,
                             T vz0, const T w, T tr_da, T tr_db, Tally &Tl) {
  const int nr = L.nr, nz = L.nz;
  if (c0 < 0 || c0 >= nr * nz) {
    if (L.write && L.oop) L.dst.cell[p] = c0;  // absorbed earlier: stays out of the store
    return;
  }
  const int ic = c0 / nz, jc = c0 - (c0 / nz) * nz;
  const T cr0 = L.rm.crr(ic);
  push_sub<T, kB, S>(L, p, ic, jc, a, b, vr0 * cr0, vt0 * cr0, vz0 * L.cz, w, tr_da, tr_db, (T)1,
                     0, 0, Tl);
}

// the four face charges of one accepted sub-step (da, db) from (a, b) in cell
// (ic, jc): Eq. 3 with m = 1 in flux form (reading of the deposit)
template <typename T, typename S>
__device__ __forceinline__ void deposit_sub(const GenArgs<T, S> &L, int ic, int jc, T w, T a, T b,
                                            T da, T db) {
  if (!L.ir) return;
  const T h = (T)0.5, one = (T)1;
  const int nz = L.nz, nz1 = nz + 1;
  const T am = a + h * da, bm = b + h * db;
  const T fr = L.qf * w * da, fz = L.qf * w * db;
  atomicAdd(&L.ir[ic * nz1 + jc], Num<T>::to_double(fr * (one - bm)));
  atomicAdd(&L.ir[ic * nz1 + jc + 1], Num<T>::to_double(fr * bm));
  atomicAdd(&L.iz[ic * nz + jc], Num<T>::to_double(fz * (one - am)));
  atomicAdd(&L.iz[(ic + 1) * nz + jc], Num<T>::to_double(fz * am));
}

// A crosser without B_z whose converged whole-step trial (tr_da, tr_db) keeps
// its radial offset inside the cell and leaves it through one z-face (cells
// are flat in z: most crossings), as straight-line code: the landing on that
// face (landing_z_joint), the transition to the next cell and the rest of the
// step there through the in-cell scalar solve, so that a warp of such crossers
// runs converged.  The steps and their arithmetic are those of the sub-step
// loop for it; at any other turn (a landing that fails or leaves the cell, a
// wall, a solve that fails, a second crossing, an end on a face) the particle
// goes on through push_sub from where it stands.
template <typename T, typename S = T>
__device__ void push_zcross(const GenArgs<T, S> &L, long long p, int c0, T a, T b, T vr0, T vt0,
                            T vz0, const T w, T tr_da, T tr_db, Tally &Tl) {
  typedef Num<T> N;
  const T zero = (T)0, one = (T)1, two = (T)2;
  const int nr = L.nr, nz = L.nz, nz1 = nz + 1;
  if (c0 < 0 || c0 >= nr * nz) {
    if (L.write && L.oop) L.dst.cell[p] = c0;  // absorbed earlier: stays out of the store
    return;
  }
  int ic = c0 / nz, jc = c0 - (c0 / nz) * nz;
  const T cr0 = L.rm.crr(ic);
  T ur = vr0 * cr0, ut = vt0 * cr0, uz = vz0 * L.cz;
  if (N::nan_bits(tr_da) || !(b + tr_db < zero || b + tr_db > one)) {
    push_sub<T, false, S>(L, p, ic, jc, a, b, ur, ut, uz, w, tr_da, tr_db, one, 0, 0, Tl);
    return;
  }
  // ---- sub-step 1: the landing on the z-face the trial leaves through
  SubT<T> s;
  s.ar0 = (T)L.ar[ic * nz1 + jc];
  s.gar = (T)L.ar[ic * nz1 + jc + 1] - s.ar0;
  s.az0 = (T)L.az[ic * nz + jc];
  s.gaz = (T)L.az[(ic + 1) * nz + jc] - s.az0;
  s.a = a; s.b = b;
  s.rho = L.rm.rho0(ic) + a;
  s.ur = ur; s.ut = ut; s.uz = uz;
  s.P = s.rho * ut;
  const T face = b + tr_db > one ? one : zero;
  const T X = face - b;
  const T g0 = (T)first_crossing<float>((float)X, (float)tr_db, (float)uz, 1.f);
  // the radial offset at g0 on the quadratic path through the trial's end
  const T d0 = g0 * (ur + g0 * (tr_da - ur));
  T tt = zero, da = zero;
  if (!N::in01(a) || !N::in01(b) || !(g0 > zero) ||
      !landing_z_joint<T>(s, X, g0, d0, tt, da, Tl.jnewton) || !(tt > zero) || tt > one ||
      !(a + da >= zero && a + da <= one)) {
    push_sub<T, false, S>(L, p, ic, jc, a, b, ur, ut, uz, w, tr_da, tr_db, one, 0, 0, Tl);
    return;
  }
  {
    ResT<T> o;
    eval_gen<T, false>(s, zero, da, X, tt, o);
    deposit_sub<T, S>(L, ic, jc, w, a, b, da, X);
    a = fmin(fmax(a + da, zero), one);
    b = face;
    ur = ur + tt * o.A;
    uz = uz + tt * o.az;
    ut = o.ut1;
    Tl.sub++;
  }
  const T tau = one - tt;
  // ---- through the landed face into the next cell (a wall: the loop)
  const bool up = face == one;
  if (!N::in01(a) || (up ? !(uz > zero) || jc + 1 == nz : !(uz < zero) || jc == 0) ||
      !(tau > zero)) {
    push_sub<T, false, S>(L, p, ic, jc, a, b, ur, ut, uz, w, (T)NAN, (T)NAN, tau, 1, 1, Tl);
    return;
  }
  jc += up ? 1 : -1;
  b = up ? zero : one;
  // ---- sub-step 2: the rest of the step inside the next cell
  SubT<T> s2;
  s2.ar0 = (T)L.ar[ic * nz1 + jc];
  s2.gar = (T)L.ar[ic * nz1 + jc + 1] - s2.ar0;
  s2.az0 = (T)L.az[ic * nz + jc];
  s2.gaz = (T)L.az[(ic + 1) * nz + jc] - s2.az0;
  s2.a = a; s2.b = b;
  s2.rho = L.rm.rho0(ic) + a;
  s2.ur = ur; s2.ut = ut; s2.uz = uz;
  s2.P = s2.rho * ut;
  T da2 = zero, db2 = zero;
  const bool in2 = scalar_interior<T>(s2, tau, da2, db2, Tl.snewton);
  const T a2 = a + da2, b2 = b + db2;
  if (!in2 || !(a2 >= zero && a2 <= one && b2 >= zero && b2 <= one) || !(s2.rho + da2 > zero)) {
    push_sub<T, false, S>(L, p, ic, jc, a, b, ur, ut, uz, w, (T)NAN, (T)NAN, tau, 1, 1, Tl);
    return;
  }
  {
    const T it = tau == one ? one : N::rcp(tau);
    const T nur = two * da2 * it - ur, nuz = two * db2 * it - uz;
    const T nut = s2.P * N::rcp(s2.rho + da2);
    deposit_sub<T, S>(L, ic, jc, w, a, b, da2, db2);
    a = fmin(fmax(a2, zero), one);
    b = fmin(fmax(b2, zero), one);
    ur = nur; uz = nuz; ut = nut;
    Tl.sub++;
  }
  if (!N::in01(a) || !N::in01(b)) {
    // ended on a face: the loop moves it (or absorbs it) and finishes
    push_sub<T, false, S>(L, p, ic, jc, a, b, ur, ut, uz, w, (T)NAN, (T)NAN, zero, 2, 2, Tl);
    return;
  }
  if (L.hist) atomicAdd(&L.hist[1], 1ull);  // two accepted sub-steps
  if (L.write) {
    const T icr = L.rm.icrr(ic);
    L.dst.cell[p] = ic * nz + jc;
    L.dst.a[p] = (S)a; L.dst.b[p] = (S)b;
    L.dst.vr[p] = (S)(ur * icr); L.dst.vt[p] = (S)(ut * icr); L.dst.vz[p] = (S)(uz * L.icz);
    if (L.oop) {
      L.dst.w[p] = (S)w;
      L.dst.id[p] = L.p.id[p];
    }
  }
}

// algorithmic operation counts of the general path: 75 per Newton iteration
// (one residual/Jacobian evaluation and update), 93 per accepted sub-step, 60
// per joint landing iteration (landing_z_joint)
constexpr unsigned kOpGenNewton = 75, kOpGenAccept = 93, kOpJointNewton = 60;

// counters[0..4] += errors, absorbed, accepted sub-steps, fallbacks, operations;
// per-thread counts are small, so the warp sums use the 32-bit redux unit
__device__ __forceinline__ void flush_tally(unsigned long long *counters, const Tally &T, int lane,
                                            unsigned fast_newton, unsigned fast_acc) {
  if (!counters) return;
  const unsigned full = 0xffffffffu;
  unsigned e0 = __reduce_add_sync(full, T.err), e1 = __reduce_add_sync(full, T.abs),
           e2 = __reduce_add_sync(full, T.sub), e3 = __reduce_add_sync(full, T.fb),
           e4 = __reduce_add_sync(full, T.newton),
           e5 = __reduce_add_sync(full, fast_newton + T.snewton),
           e6 = __reduce_add_sync(full, fast_acc), e7 = __reduce_add_sync(full, T.jnewton);
  if (lane == 0) {
    if (e0) atomicAdd(&counters[0], (unsigned long long)e0);
    if (e1) atomicAdd(&counters[1], (unsigned long long)e1);
    if (e2 + e6) atomicAdd(&counters[2], (unsigned long long)e2 + e6);
    if (e3) atomicAdd(&counters[3], (unsigned long long)e3);
    unsigned long long fl = (unsigned long long)kOpGenNewton * e4 +
                            (unsigned long long)kOpGenAccept * e2 +
                            (unsigned long long)kOpFastNewton * e5 +
                            (unsigned long long)kOpFastAccept * e6 +
                            (unsigned long long)kOpJointNewton * e7;
    if (fl) atomicAdd(&counters[4], fl);
  }
}

}  // namespace pic
