/*
 * FP64 CPU oracle for the implicit energy- and charge-conserving EM PIC/MCC
 * method of Eremin et al., "Modeling of VHF large-electrode CCPs with a fully
 * electromagnetic PIC code" (arXiv:2212.08836).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code,
 * header or constant table with the CUDA path; both are written from the
 * paper's equations and the same readings of its discretisation (uniform
 * r-z mesh, integral Yee form, linear shapes, lumped gap drive).
 *
 * Plain, serial, slow on purpose.  Compile with -ffp-contract=off so that no
 * multiply-add is fused (the GPU FP64 parity build uses --fmad=false).
 *
 * Conventions (mesh uniform in the logical coordinates, Sec. 2.1: z = eta*dz,
 * r = xi*dr, or the mapped r(xi) of o_rnode with xa > 0):
 *   nodes (i,j), i=0..nr, j=0..nz;  cells (i,j) i<nr, j<nz
 *   Er edge (i+1/2, j): Er[i*(nz+1)+j], i<nr, j<=nz      (Yee, Eq. 2)
 *   Ez edge (i, j+1/2): Ez[i*nz+j],     i<=nr, j<nz
 *   H_theta (i+1/2, j+1/2): H[i*nz+j]
 *   Ir / Iz: charge [C] that crossed the dual face of each edge during the
 *   step (the logical flux form of the current in Eq. 3 with m = 1)
 *   particle: cell = ic*nz+jc (-1 = absorbed), offsets a,b in [0,1]
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_PI 3.14159265358979323846
#define O_TWO_PI 6.283185307179586

/* CODATA 2018 */
#define O_QE 1.602176634e-19
#define O_ME 9.1093837015e-31
#define O_AMU 1.66053906660e-27
#define O_KB 1.380649e-23
#define O_EPS0 8.8541878128e-12
#define O_MU0 1.25663706212e-6

/* ---------------------------------------------------------------- Philox */
/* Philox4x64-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11: 10 rounds of two 64x64->128 multiplies with the
 * round constants and Weyl key increments given in that paper. */
static void o_mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void oracle_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t hi0, lo0, hi1, lo1;
    o_mul128(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
    o_mul128(0xCA5A826395121157ULL, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B97F4A7C15ULL;
    k1 += 0xBB67AE8584CAA73BULL;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in [0,1) */
static double o_u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

static void o_draw4(uint64_t seed, uint64_t stream, uint64_t id, uint64_t step, uint64_t block,
                    double u[4]) {
  uint64_t c[4] = {id, step, block, 0};
  uint64_t k[2] = {seed, stream};
  uint64_t o[4];
  oracle_philox4x64(c, k, o);
  for (int q = 0; q < 4; ++q) u[q] = o_u01(o[q]);
}

/* Box-Muller pair from two uniforms */
static void o_gauss2(double ua, double ub, double *g1, double *g2) {
  double rho = sqrt(-2.0 * log(1.0 - ua));
  double ang = O_TWO_PI * ub;
  *g1 = rho * cos(ang);
  *g2 = rho * sin(ang);
}

/* stream identifiers (key word 1) */
#define O_STREAM_LOAD_POS 0x20ULL
#define O_STREAM_LOAD_VE 0x21ULL
#define O_STREAM_LOAD_VI 0x22ULL
#define O_STREAM_MCC_E 0x10ULL
#define O_STREAM_MCC_I 0x11ULL
#define O_LOAD_STEP 0xFFFFFFFFFFFFFFFFULL

/* ------------------------------------------------------------- geometry */
typedef struct {
  int nr, nz;
  double dr, dz; /* dr: radial spacing of the uniformly spaced part of the mesh */
  int xa;        /* mapped mesh: the first xa cells have r proportional to sqrt(xi) */
  int nd;        /* dielectric ring: the outer nd cells (relative permittivity erd) */
  double erd;
  double sgd;    /* conductivity of the ring's cells [S/m] (0: a pure dielectric) */
} og_grid;

/* Radial mapping (Sec. 2.1, the mapped mesh): r(xi) = 2 dr sqrt(xa xi) for
 * xi <= xa and dr (xi + xa) beyond, continuous with its slope at xi = xa, so
 * that r J_r = 2 dr^2 xa near the axis; xa = 0 is the uniform mesh r = xi dr.
 * Within a cell r is linear in xi (J_r constant per cell). */
static double o_rnode(const og_grid *g, int i) {
  if (i < g->xa) return 2.0 * g->dr * sqrt((double)g->xa * (double)i);
  return ((double)i + (double)g->xa) * g->dr;
}
/* cell width J_r and r at the cell centre */
static double o_drc(const og_grid *g, int i) {
  return i < g->xa ? o_rnode(g, i + 1) - o_rnode(g, i) : g->dr;
}
static double o_rhalf(const og_grid *g, int i) {
  if (i < g->xa) return 0.5 * (o_rnode(g, i) + o_rnode(g, i + 1));
  return ((double)i + 0.5 + (double)g->xa) * g->dr;
}
/* r at the inner face of cell i in units of its width */
static double o_rho0(const og_grid *g, int i) {
  return i < g->xa ? o_rnode(g, i) / o_drc(g, i) : (double)(i + g->xa);
}
/* dual-face areas of Yee edges (integral form of Ampere, Eq. 2): E_r edge
 * (i+1/2, j): the cylinder 2 pi r_{i+1/2} dz; E_z edge (i, j+1/2): the ring
 * between the neighbouring cell centres */
static double o_area_r(const og_grid *g, int i) { return O_TWO_PI * o_rhalf(g, i) * g->dz; }
static double o_area_z(const og_grid *g, int i) {
  if (i == 0) return O_PI * o_rhalf(g, 0) * o_rhalf(g, 0);
  if (i <= g->xa) {
    double ro = o_rhalf(g, i), ri = o_rhalf(g, i - 1);
    return O_PI * (ro * ro - ri * ri);
  }
  return O_TWO_PI * o_rnode(g, i) * g->dr;
}
/* Dielectric ring (the feed region at the periphery, Sec. 2.1's dielectric
 * port read for the side feed): the outer nd cells have relative
 * permittivity erd.  The integral form weights each dual face by the
 * permittivity of the cells it crosses: eps A for the E_r faces of ring rows,
 * the two halves of the ring's inner boundary node separately. */
static double o_aeff_r(const og_grid *g, int i) {
  return (g->nd > 0 && i >= g->nr - g->nd) ? g->erd * o_area_r(g, i) : o_area_r(g, i);
}
static double o_aeff_z(const og_grid *g, int i) {
  const int i0 = g->nr - g->nd;
  if (g->nd == 0 || i < i0) return o_area_z(g, i);
  if (i > i0) return g->erd * o_area_z(g, i);
  const double ri = o_rnode(g, i), rm = o_rhalf(g, i - 1), rp = o_rhalf(g, i);
  return O_PI * (ri * ri - rm * rm) + g->erd * O_PI * (rp * rp - ri * ri);
}
/* Conducting ring (Eq. 2's sigma E term; Sec. 2.1 models metals in EM runs
 * by a large conductivity): the ring's cells carry conductivity sgd, and each
 * dual face conducts sgd times the part of its area inside the ring. */
static double o_asig_r(const og_grid *g, int i) {
  return (g->nd > 0 && i >= g->nr - g->nd) ? g->sgd * o_area_r(g, i) : 0.0;
}
static double o_asig_z(const og_grid *g, int i) {
  const int i0 = g->nr - g->nd;
  if (g->nd == 0 || g->sgd == 0.0 || i < i0) return 0.0;
  if (i > i0) return g->sgd * o_area_z(g, i);
  const double ri = o_rnode(g, i), rp = o_rhalf(g, i);
  return g->sgd * O_PI * (rp * rp - ri * ri);
}
/* primal-cell volume carrying H_theta */
static double o_vol_h(const og_grid *g, int i) {
  return O_TWO_PI * o_rhalf(g, i) * o_drc(g, i) * g->dz;
}

/* ------------------------------------------------------------ particles */
/* Particle loading (a1): pair loading at identical positions, uniform in the
 * logical coordinates, weight proportional to r*J_r (Sec. 2.1), Maxwellian
 * velocities.  Electron p and ion p share position and weight, so the initial
 * node charge vanishes and E = 0, H = 0 is a Gauss-consistent start. */
void oracle_load(int nr, int nz, double dr, double dz, int xa, int nd, double erd, double R,
                 double L, double n0,
                 int64_t n, double te_ev, double ti_ev, double me, double mi, uint64_t seed,
                 int32_t *cell, double *a, double *b, double *vre, double *vte, double *vze,
                 double *vri, double *vti, double *vzi, double *w, uint32_t *id) {
  og_grid g = {nr, nz, dr, dz, xa, nd, erd, 0.0};  /* conductivity: not used here */
  const int np_r = nr - nd; /* particles live inside the ring */
  double vthe = sqrt(te_ev * O_QE / me);
  double vthi = sqrt(ti_ev * O_QE / mi);
  for (int64_t p = 0; p < n; ++p) {
    double u[4];
    o_draw4(seed, O_STREAM_LOAD_POS, (uint64_t)p, O_LOAD_STEP, 0, u);
    double xi = (double)np_r * u[0];
    double eta = (double)nz * u[1];
    int ic = (int)floor(xi);
    int jc = (int)floor(eta);
    if (ic > np_r - 1) ic = np_r - 1;
    if (jc > nz - 1) jc = nz - 1;
    cell[p] = ic * nz + jc;
    a[p] = xi - (double)ic;
    b[p] = eta - (double)jc;
    if (xa == 0 && nd == 0) {
      w[p] = n0 * (O_TWO_PI * (xi * dr)) * R * L / (double)n;
    } else {  /* w proportional to r J_r */
      double Jr = o_drc(&g, ic);
      double r = (o_rho0(&g, ic) + a[p]) * Jr;
      w[p] = n0 * (O_TWO_PI * r) * (Jr * (double)np_r) * L / (double)n;
    }
    id[p] = (uint32_t)p;
    double g1, g2, g3, g4;
    o_draw4(seed, O_STREAM_LOAD_VE, (uint64_t)p, O_LOAD_STEP, 0, u);
    o_gauss2(u[0], u[1], &g1, &g2);
    o_gauss2(u[2], u[3], &g3, &g4);
    vre[p] = vthe * g1; vte[p] = vthe * g2; vze[p] = vthe * g3;
    o_draw4(seed, O_STREAM_LOAD_VI, (uint64_t)p, O_LOAD_STEP, 0, u);
    o_gauss2(u[0], u[1], &g1, &g2);
    o_gauss2(u[2], u[3], &g3, &g4);
    vri[p] = vthi * g1; vti[p] = vthi * g2; vzi[p] = vthi * g3;
  }
  (void)R;
}

/* ---------------------------------------------------------------- mover */
/* Crank-Nicolson integration of Eq. 4 with cell-crossing sub-steps (Sec. 2.1,
 * after Chen et al. 2011).  Within one cell the sub-step midpoint equations
 *   dr*da = dtau*vr + dtau^2/2 * (qm*Er(bm) + C(da))
 *   dz*db = dtau*vz + dtau^2/2 * qm*Ez(am)
 * with am = a + da/2, bm = b + db/2, Er linear in bm, Ez linear in am (the
 * S0 x S1 / S1 x S0 gather of the edge fields of the cell), and
 *   C = vt_m^2/r_m + wb*vt_m  (centrifugal + optional external-Bz Lorentz term)
 * where vt' follows from the exactly conserved CN canonical angular momentum
 * r*vt + wb*r^2/2.  They are solved by Newton for (da,db) at given dtau, or
 * for (dtau, other) when the sub-step must end exactly on a cell face. */

#define O_NSUB_MAX 64
#define O_NEWTON_MAX 30
#define O_TOLX 1e-14
#define O_TOLT 1e-14

typedef struct {
  /* cell constants */
  double er0, ger, ez0, gez;
  double dr, dz;
  double qm, wb;
  /* particle start of sub-step */
  double a, b, r, vr, vt, vz, pth;
} o_sub;

typedef struct {
  double f1, f2;
  double f1a, f1b, f1t, f2a, f2b, f2t;
  double C, vt1;
} o_res;

/* residuals and Jacobian of the sub-step equations at (da, db, dt) */
static void o_eval(const o_sub *s, double da, double db, double dt, o_res *o) {
  double r1 = s->r + da * s->dr;
  double rm = 0.5 * (s->r + r1);
  double vt1, dvt1;
  if (r1 > 0.0) {
    vt1 = (s->pth - 0.5 * s->wb * r1 * r1) / r1;
    dvt1 = s->dr * (-s->pth / (r1 * r1) - 0.5 * s->wb);
  } else {
    vt1 = s->vt;
    dvt1 = 0.0;
  }
  double vtm = 0.5 * (s->vt + vt1);
  double dvtm = 0.5 * dvt1;
  double C, dC;
  if (rm > 0.0) {
    C = vtm * vtm / rm + s->wb * vtm;
    dC = 2.0 * vtm * dvtm / rm - vtm * vtm * (0.5 * s->dr) / (rm * rm) + s->wb * dvtm;
  } else {
    C = s->wb * vtm;
    dC = s->wb * dvtm;
  }
  double am = s->a + 0.5 * da;
  double bm = s->b + 0.5 * db;
  double ez = s->ez0 + s->gez * am;
  double er = s->er0 + s->ger * bm;
  double ar = s->qm * er + C;
  double dt2 = dt * dt;
  o->f1 = s->dz * db - dt * s->vz - 0.5 * dt2 * (s->qm * ez);
  o->f2 = s->dr * da - dt * s->vr - 0.5 * dt2 * ar;
  o->f1a = -0.25 * dt2 * s->qm * s->gez;
  o->f1b = s->dz;
  o->f1t = -s->vz - dt * (s->qm * ez);
  o->f2a = s->dr - 0.5 * dt2 * dC;
  o->f2b = -0.25 * dt2 * s->qm * s->ger;
  o->f2t = -s->vr - dt * ar;
  o->C = C;
  o->vt1 = vt1;
}

/* interior sub-step of length dt: Newton on (da, db).  Returns 1 on success. */
static int o_solve_interior(const o_sub *s, double dt, double *pda, double *pdb) {
  double da = dt * s->vr / s->dr;
  double db = dt * s->vz / s->dz;
  if (s->pth != 0.0 && s->r + da * s->dr <= 0.0) da = -0.5 * s->r / s->dr;
  for (int it = 0; it < O_NEWTON_MAX; ++it) {
    o_res o;
    o_eval(s, da, db, dt, &o);
    double det = o.f1a * o.f2b - o.f1b * o.f2a;
    if (!(det != 0.0) || !isfinite(det)) return 0;
    double xa = (-o.f1 * o.f2b + o.f2 * o.f1b) / det;
    double xb = (-o.f1a * o.f2 + o.f2a * o.f1) / det;
    double nda = da + xa;
    double ndb = db + xb;
    if (s->pth != 0.0 && s->r + nda * s->dr <= 0.0) nda = 0.5 * (da - s->r / s->dr);
    double ca = fabs(nda - da), cb = fabs(ndb - db);
    da = nda;
    db = ndb;
    if (!isfinite(da) || !isfinite(db)) return 0;
    if (ca <= O_TOLX && cb <= O_TOLX) {
      *pda = da;
      *pdb = db;
      return 1;
    }
  }
  return 0;
}

/* landing sub-step on a face normal to xi (dir 0) or eta (dir 1):
 * fixed displacement X in that direction, unknowns (other, dt).  X == 0 is
 * the return to the face the particle sits on: the residual is divided by dt
 * to remove the trivial root. */
static int o_solve_landing(const o_sub *s, int dir, double X, double dt0, double oth0,
                           double tscale, double *pdt, double *poth) {
  double dt = dt0, oth = oth0;
  for (int it = 0; it < O_NEWTON_MAX; ++it) {
    double da = dir == 0 ? X : oth;
    double db = dir == 0 ? oth : X;
    o_res o;
    o_eval(s, da, db, dt, &o);
    /* equations: g_fix (fixed direction), g_oth (other direction) */
    double gF, gFo, gFt, gO, gOo, gOt;
    if (dir == 0) {
      gO = o.f1; gOo = o.f1b; gOt = o.f1t;
      if (X != 0.0) {
        gF = o.f2; gFo = o.f2b; gFt = o.f2t;
      } else {
        double bm = s->b + 0.5 * db;
        double ar = s->qm * (s->er0 + s->ger * bm) + o.C;
        gF = -s->vr - 0.5 * dt * ar;
        gFo = -0.25 * dt * s->qm * s->ger;
        gFt = -0.5 * ar;
      }
    } else {
      gO = o.f2; gOo = o.f2a; gOt = o.f2t;
      if (X != 0.0) {
        gF = o.f1; gFo = o.f1a; gFt = o.f1t;
      } else {
        double am = s->a + 0.5 * da;
        double ez = s->qm * (s->ez0 + s->gez * am);
        gF = -s->vz - 0.5 * dt * ez;
        gFo = -0.25 * dt * s->qm * s->gez;
        gFt = -0.5 * ez;
      }
    }
    /* [gFo gFt; gOo gOt] [x_o; x_t] = -[gF; gO] */
    double det = gFo * gOt - gFt * gOo;
    if (!(det != 0.0) || !isfinite(det)) return 0;
    double xo = (-gF * gOt + gO * gFt) / det;
    double xt = (-gFo * gO + gOo * gF) / det;
    double noth = oth + xo;
    double ndt = dt + xt;
    if (dir == 1 && s->pth != 0.0 && s->r + noth * s->dr <= 0.0) noth = 0.5 * (oth - s->r / s->dr);
    double co = fabs(noth - oth), ct = fabs(ndt - dt);
    oth = noth;
    dt = ndt;
    if (!isfinite(oth) || !isfinite(dt)) return 0;
    if (co <= O_TOLX && ct <= O_TOLT * tscale) {
      *pdt = dt;
      *poth = oth;
      return 1;
    }
  }
  return 0;
}

typedef struct {
  int nr, nz;
  double dr, dz;
  og_grid g;             /* the mesh (radial mapping) */
  const double *er, *ez;
  double *ir, *iz;       /* may be NULL */
  double q, qm, wb;
  /* wall tallies (may be NULL): charge absorbed per wall node */
  double *wall_z0, *wall_zl, *wall_r;
  double m;
  double ke_lost;
  int64_t n_substep_err, n_absorbed, n_substeps, n_fallback;
} o_push;

static void o_deposit(o_push *P, int ic, int jc, double a, double b, double da, double db,
                      double w) {
  if (!P->ir) return;
  double am = a + 0.5 * da;
  double bm = b + 0.5 * db;
  double fr = P->q * w * da;
  double fz = P->q * w * db;
  P->ir[ic * (P->nz + 1) + jc] += fr * (1.0 - bm);
  P->ir[ic * (P->nz + 1) + jc + 1] += fr * bm;
  P->iz[ic * P->nz + jc] += fz * (1.0 - am);
  P->iz[(ic + 1) * P->nz + jc] += fz * am;
}

/* Cell transition for a particle sitting on a face of its cell with its
 * normal velocity pointing out of the cell: it moves to the neighbour cell
 * (offset 1 -> 0 or 0 -> 1).  Axis r = 0: reflection.  Walls r = R, z = 0,
 * z = L: absorption (returns 1, 2, 3 respectively). */
static int o_transition(const o_push *P, int *ic, int *jc, double *a, double *b, double *vr,
                        double *vz) {
  if (*a == 1.0 && *vr > 0.0) {
    if (*ic + 1 == P->nr) return 1;
    *ic += 1;
    *a = 0.0;
  } else if (*a == 0.0 && *vr < 0.0) {
    if (*ic == 0) *vr = -*vr;
    else { *ic -= 1; *a = 1.0; }
  }
  if (*b == 1.0 && *vz > 0.0) {
    if (*jc + 1 == P->nz) return 2;
    *jc += 1;
    *b = 0.0;
  } else if (*b == 0.0 && *vz < 0.0) {
    if (*jc == 0) return 3;
    *jc -= 1;
    *b = 1.0;
  }
  return 0;
}

/* Start of the landing solve: the time at which the quadratic path
 * x(s) = v0 s + alpha s^2 / 2 through the trial's end point, x(dtT) = dxh,
 * first reaches the face at displacement Xh.  For Xh != 0 the face lies
 * between the start and the trial's end point, so the parabola reaches it in
 * (0, dtT]; the smaller positive root is the first crossing (the sub-step ends
 * on the first face crossed).  Xh = 0 is the face the particle sits on: the
 * nonzero root.  With constant acceleration this is the exact crossing time;
 * a start on the far side of a grazing crossing could converge to a later
 * root instead. */
static double o_first_crossing(double Xh, double dxh, double v0, double dtT) {
  double alpha = 2.0 * (dxh - v0 * dtT) / (dtT * dtT);
  if (Xh == 0.0) return -2.0 * v0 / alpha;
  if (alpha == 0.0) return Xh / v0;
  double disc = v0 * v0 + 2.0 * alpha * Xh;
  if (!(disc >= 0.0)) return dtT * (Xh / dxh);
  /* roots of alpha/2 s^2 + v0 s - Xh = 0 without cancellation:
   * s1 = qq / (alpha/2), s2 = -Xh / qq with qq = -(v0 + sgn(v0) sqrt(disc)) / 2 */
  double qq = -0.5 * (v0 + (v0 >= 0.0 ? sqrt(disc) : -sqrt(disc)));
  double s1 = qq / (0.5 * alpha);
  double s2 = qq != 0.0 ? -Xh / qq : s1;
  double s = -1.0;
  if (s1 > 0.0) s = s1;
  if (s2 > 0.0 && (s < 0.0 || s2 < s)) s = s2;
  return s > 0.0 ? s : dtT * (Xh / dxh);
}

/* Advance one particle over dt.  Returns 1 if absorbed at a wall. */
static int o_push_one(o_push *P, int *pic, int *pjc, double *pa, double *pb, double *pvr,
                      double *pvt, double *pvz, double w, double dt_full) {
  int ic = *pic, jc = *pjc;
  double a = *pa, b = *pb, vr = *pvr, vt = *pvt, vz = *pvz;
  double tau = dt_full;
  double dtT = tau;
  int nsub = 0;
  int absorbed = o_transition(P, &ic, &jc, &a, &b, &vr, &vz);
  while (tau > 0.0 && !absorbed) {
    if (++nsub > O_NSUB_MAX) {
      P->n_substep_err++;
      break;
    }
    o_sub s;
    s.er0 = P->er[ic * (P->nz + 1) + jc];
    s.ger = P->er[ic * (P->nz + 1) + jc + 1] - s.er0;
    s.ez0 = P->ez[ic * P->nz + jc];
    s.gez = P->ez[(ic + 1) * P->nz + jc] - s.ez0;
    s.dr = o_drc(&P->g, ic);
    s.dz = P->dz;
    s.qm = P->qm;
    s.wb = P->wb;
    s.a = a; s.b = b;
    s.r = (o_rho0(&P->g, ic) + a) * s.dr;
    s.vr = vr; s.vt = vt; s.vz = vz;
    s.pth = s.r * vt + 0.5 * P->wb * s.r * s.r;

    double da, db;
    if (!o_solve_interior(&s, dtT, &da, &db)) {
      dtT *= 0.5;
      P->n_fallback++;
      continue;
    }
    double a1 = a + da, b1 = b + db;
    double step_dt;
    int land_dir = -1;
    double land_face = 0.0;
    if (a1 >= 0.0 && a1 <= 1.0 && b1 >= 0.0 && b1 <= 1.0) {
      step_dt = dtT;
    } else {
      /* candidate faces: one per direction whose end point is outside */
      double best_dt = 0.0, best_oth = 0.0;
      int best_dir = -1;
      double best_face = 0.0;
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
        double h = dir == 0 ? s.dr : P->dz;
        double g0 = o_first_crossing(X * h, dx * h, v0, dtT);
        double oth0 = doth * (g0 / dtT);
        double tdt = 0.0, toth = 0.0;
        if (!(g0 > 0.0) || !o_solve_landing(&s, dir, X, g0, oth0, dtT, &tdt, &toth)) continue;
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
        P->n_fallback++;
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
    /* accept the sub-step (da, db, step_dt) */
    o_res o;
    o_eval(&s, da, db, step_dt, &o);
    double am = a + 0.5 * da, bm = b + 0.5 * db;
    double nvr = vr + step_dt * (P->qm * (s.er0 + s.ger * bm) + o.C);
    double nvz = vz + step_dt * (P->qm * (s.ez0 + s.gez * am));
    double nvt = o.vt1;
    o_deposit(P, ic, jc, a, b, da, db, w);
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
    P->n_substeps++;
    absorbed = o_transition(P, &ic, &jc, &a, &b, &vr, &vz);
    if (absorbed) break;
    dtT = tau;
  }
  if (absorbed) {
    P->n_absorbed++;
    double qw = P->q * w;
    if (absorbed == 1 && P->wall_r) {
      P->wall_r[jc] += qw * (1.0 - b);
      P->wall_r[jc + 1] += qw * b;
    } else if (absorbed == 2 && P->wall_zl) {
      P->wall_zl[ic] += qw * (1.0 - a);
      P->wall_zl[ic + 1] += qw * a;
    } else if (absorbed == 3 && P->wall_z0) {
      P->wall_z0[ic] += qw * (1.0 - a);
      P->wall_z0[ic + 1] += qw * a;
    }
    P->ke_lost += 0.5 * P->m * w * (vr * vr + vt * vt + vz * vz);
  }
  *pic = ic; *pjc = jc; *pa = a; *pb = b; *pvr = vr; *pvt = vt; *pvz = vz;
  return absorbed != 0;
}

/* Push + deposit of one species (rows a2/a3, and a6 when write != 0).
 * er/ez hold E^{n+1/2}; ir/iz accumulate (caller zeroes).  counters[6]:
 * substep errors, absorbed, substeps, fallbacks (and ke_lost in kelost). */
/* threads of the push (1: the serial form every test uses) */
static int o_threads = 1;

void oracle_set_threads(int n) { o_threads = n < 1 ? 1 : n; }

static void o_push_range(o_push *P, int nz, int64_t p0, int64_t p1, int32_t *cell, double *a,
                         double *b, double *vr, double *vt, double *vz, const double *w,
                         int write, double dt) {
  for (int64_t p = p0; p < p1; ++p) {
    if (cell[p] < 0) continue;
    int ic = cell[p] / nz, jc = cell[p] % nz;
    double pa = a[p], pb = b[p], pvr = vr[p], pvt = vt[p], pvz = vz[p];
    int gone = o_push_one(P, &ic, &jc, &pa, &pb, &pvr, &pvt, &pvz, w[p], dt);
    if (write) {
      cell[p] = gone ? -1 : ic * nz + jc;
      a[p] = pa; b[p] = pb; vr[p] = pvr; vt[p] = pvt; vz[p] = pvz;
    }
  }
}

static void o_add(double *dst, const double *src, size_t n) {
  if (!dst) return;
  for (size_t k = 0; k < n; ++k) dst[k] += src[k];
}

void oracle_push(int nr, int nz, double dr, double dz, int xa, int nd, double erd, double dt,
                 double q, double m, double bz,
                 int64_t n, int32_t *cell, double *a, double *b, double *vr, double *vt,
                 double *vz, const double *w, const double *er, const double *ez, double *ir,
                 double *iz, int write, double *wall_z0, double *wall_zl, double *wall_r,
                 int64_t *counters, double *kelost) {
  o_push P;
  memset(&P, 0, sizeof(P));
  /* particles move inside the dielectric ring: its inner face r_{nr-nd} is
   * their outer wall, where they stop and their charge stays (sticking) */
  P.nr = nr - nd; P.nz = nz; P.dr = dr; P.dz = dz;
  P.g.nr = nr; P.g.nz = nz; P.g.dr = dr; P.g.dz = dz; P.g.xa = xa; P.g.nd = nd; P.g.erd = erd;
  P.er = er; P.ez = ez; P.ir = ir; P.iz = iz;
  P.q = q; P.qm = q / m; P.wb = (q / m) * bz; P.m = m;
  P.wall_z0 = wall_z0; P.wall_zl = wall_zl; P.wall_r = wall_r;
  int nt = o_threads;
  if (nt > 1 && n < 64 * (int64_t)nt) nt = 1;
  if (nt <= 1) {
    o_push_range(&P, nz, 0, n, cell, a, b, vr, vt, vz, w, write, dt);
  } else {
    /* timing form: the particles split into nt contiguous ranges, each pushed
     * with its own crossed-charge and wall arrays, which are summed at the end
     * (another summation order than the serial form: equal to rounding) */
    const size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz;
    const size_t per = ner + nez + 2 * (size_t)(nr + 1) + (size_t)(nz + 1);
    double *buf = (double *)calloc((size_t)nt * per, sizeof(double));
    o_push *Pt = (o_push *)calloc((size_t)nt, sizeof(o_push));
    if (!buf || !Pt) {
      free(buf);
      free(Pt);
      o_push_range(&P, nz, 0, n, cell, a, b, vr, vt, vz, w, write, dt);
    } else {
#pragma omp parallel for num_threads(nt) schedule(static, 1)
      for (int t = 0; t < nt; ++t) {
        double *bt = buf + (size_t)t * per;
        Pt[t] = P;
        Pt[t].ir = ir ? bt : NULL;
        Pt[t].iz = iz ? bt + ner : NULL;
        Pt[t].wall_z0 = wall_z0 ? bt + ner + nez : NULL;
        Pt[t].wall_zl = wall_zl ? bt + ner + nez + (nr + 1) : NULL;
        Pt[t].wall_r = wall_r ? bt + ner + nez + 2 * (nr + 1) : NULL;
        o_push_range(&Pt[t], nz, n * t / nt, n * (t + 1) / nt, cell, a, b, vr, vt, vz, w,
                     write, dt);
      }
      for (int t = 0; t < nt; ++t) {
        double *bt = buf + (size_t)t * per;
        o_add(ir, bt, ner);
        o_add(iz, bt + ner, nez);
        o_add(wall_z0, bt + ner + nez, (size_t)(nr + 1));
        o_add(wall_zl, bt + ner + nez + (nr + 1), (size_t)(nr + 1));
        o_add(wall_r, bt + ner + nez + 2 * (nr + 1), (size_t)(nz + 1));
        P.n_substep_err += Pt[t].n_substep_err;
        P.n_absorbed += Pt[t].n_absorbed;
        P.n_substeps += Pt[t].n_substeps;
        P.n_fallback += Pt[t].n_fallback;
        P.ke_lost += Pt[t].ke_lost;
      }
      free(buf);
      free(Pt);
    }
  }
  if (counters) {
    counters[0] += P.n_substep_err;
    counters[1] += P.n_absorbed;
    counters[2] += P.n_substeps;
    counters[3] += P.n_fallback;
  }
  if (kelost) *kelost += P.ke_lost;
}

/* node charge by S1 x S1 weighting; Q has (nr+1)*(nz+1) entries (i*(nz+1)+j) */
void oracle_node_charge(int nr, int nz, double q, int64_t n, const int32_t *cell,
                        const double *a, const double *b, const double *w, double *Q) {
  for (int64_t p = 0; p < n; ++p) {
    if (cell[p] < 0) continue;
    int ic = cell[p] / nz, jc = cell[p] % nz;
    double qw = q * w[p];
    Q[ic * (nz + 1) + jc] += qw * (1.0 - a[p]) * (1.0 - b[p]);
    Q[(ic + 1) * (nz + 1) + jc] += qw * a[p] * (1.0 - b[p]);
    Q[ic * (nz + 1) + jc + 1] += qw * (1.0 - a[p]) * b[p];
    Q[(ic + 1) * (nz + 1) + jc + 1] += qw * a[p] * b[p];
  }
  (void)nr;
}

/* --------------------------------------------------------- field solve */
/* Implicit CN Maxwell solve of Eq. 2 (TM: Er, Ez, H_theta; H_theta is the
 * primary unknown).  Integral (finite-volume) Yee form on the (mapped) mesh:
 *   Faraday: mu*Vh*(H1-H0) = -dt * C^T L E_half
 *   Ampere:  eps*A*(E1-E0) + dt*S*E_half = dt * C H_half - dQ   (unknown edges)
 * with S the conducting part of the face (sigma A, zero outside a conducting
 * ring).  Per edge, with D = eps A + dt S/2:
 *   E_half = (eps A E0 - dQ/2)/D + dt C H_half / (2D),
 * so eliminating E gives (2 mu Vh + dt^2/2 C^T W C) H_half = rhs, W = L/D,
 * solved here by banded Cholesky.  Prescribed edges: Er = 0 on the plates
 * z=0, z=L; Ez(R, z) = V(t)/L on the r = R gap. */
typedef struct {
  int nr, nz, n, bw, xa, nd;
  double erd, sgd;
  int wave;   /* 1: the r = R boundary is the matched port of o_wave_port */
  double dr, dz, dt, eps, mu;
  double *Lb; /* lower band of the Cholesky factor, n*(bw+1) */
} o_field;

/* Wave port on r = R (Eq. 5 read for our side feed): instead of a prescribed
 * gap field, the boundary edges obey the first-order absorbing condition of
 * an outgoing TEM-like wave with an incoming one,
 *   E_z(R) + eta H_theta(R) = 2 E_in(t),   eta = sqrt(mu/eps),
 * CN-centred, with H_theta(R) taken at the outermost H node r_{nr-1/2} and
 * E_in = V(t) / (2L), so that a slow drive gives the gap voltage V(t) (the
 * open-circuit doubling of the incident wave).  Outgoing waves leave through
 * it.  In the H system this adds dt 2 pi r_{nr-1/2} dz eta to the diagonal of
 * the outermost row. */

/* D = eps A_eff + dt S / 2 of the E_r edges of row i and the E_z edges of node i */
static double o_dnr(const og_grid *g, double eps, double dt, int i) {
  return eps * o_aeff_r(g, i) + 0.5 * dt * o_asig_r(g, i);
}
static double o_dnz(const og_grid *g, double eps, double dt, int i) {
  return eps * o_aeff_z(g, i) + 0.5 * dt * o_asig_z(g, i);
}

static double *o_band(o_field *F, int i, int j) { return &F->Lb[(size_t)i * (F->bw + 1) + (j - i + F->bw)]; }

void *oracle_field_create(int nr, int nz, double dr, double dz, int xa, int nd, double erd,
                          double sgd, double dt, double eps, double mu, int wave) {
  o_field *F = (o_field *)calloc(1, sizeof(o_field));
  og_grid g = {nr, nz, dr, dz, xa, nd, erd, sgd};
  F->nr = nr; F->nz = nz; F->dr = dr; F->dz = dz; F->dt = dt; F->eps = eps; F->mu = mu;
  F->xa = xa;
  F->nd = nd;
  F->erd = erd;
  F->sgd = sgd;
  F->wave = wave;
  F->n = nr * nz;
  F->bw = nz;
  F->Lb = (double *)calloc((size_t)F->n * (F->bw + 1), sizeof(double));
  if (!F->Lb) { free(F); return NULL; }
  double hdt2 = 0.5 * dt * dt;
  /* assemble A (lower band) */
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nz; ++j) {
      int c = i * nz + j;
      *o_band(F, c, c) += 2.0 * mu * o_vol_h(&g, i);
    }
  /* unknown Er edges (i+1/2, j), j = 1..nz-1, between cells (i,j-1) [C=+2pi r] and (i,j) [C=-2pi r] */
  for (int i = 0; i < nr; ++i)
    for (int j = 1; j < nz; ++j) {
      double W = o_drc(&g, i) / o_dnr(&g, eps, dt, i);
      double s_lo = O_TWO_PI * o_rhalf(&g, i);
      double s_hi = -O_TWO_PI * o_rhalf(&g, i);
      int clo = i * nz + (j - 1), chi = i * nz + j;
      *o_band(F, clo, clo) += hdt2 * W * s_lo * s_lo;
      *o_band(F, chi, chi) += hdt2 * W * s_hi * s_hi;
      *o_band(F, chi, clo) += hdt2 * W * s_hi * s_lo;
    }
  /* unknown Ez edges (i, j+1/2), i = 0..nr-1, cells (i-1,j) [C=-2pi r_{i-1/2}] and (i,j) [C=+2pi r_{i+1/2}] */
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nz; ++j) {
      double W = dz / o_dnz(&g, eps, dt, i);
      double s_r = O_TWO_PI * o_rhalf(&g, i);
      int cr = i * nz + j;
      *o_band(F, cr, cr) += hdt2 * W * s_r * s_r;
      if (i >= 1) {
        double s_l = -O_TWO_PI * o_rhalf(&g, i - 1);
        int cl = (i - 1) * nz + j;
        *o_band(F, cl, cl) += hdt2 * W * s_l * s_l;
        *o_band(F, cr, cl) += hdt2 * W * s_l * s_r;
      }
    }
  if (wave) {
    double eta = sqrt(mu / eps);
    for (int j = 0; j < nz; ++j) {
      int c = (nr - 1) * nz + j;
      *o_band(F, c, c) += dt * O_TWO_PI * o_rhalf(&g, nr - 1) * dz * eta;
    }
  }
  /* in-place banded Cholesky A = L L^T */
  int n = F->n, bw = F->bw;
  for (int i = 0; i < n; ++i) {
    int j0 = i - bw < 0 ? 0 : i - bw;
    for (int j = j0; j <= i; ++j) {
      double s = *o_band(F, i, j);
      int k0 = j0 > j - bw ? j0 : j - bw;
      for (int k = k0; k < j; ++k) s -= *o_band(F, i, k) * *o_band(F, j, k);
      if (i == j) {
        if (!(s > 0.0)) { free(F->Lb); free(F); return NULL; }
        *o_band(F, i, i) = sqrt(s);
      } else {
        *o_band(F, i, j) = s / *o_band(F, j, j);
      }
    }
  }
  return F;
}

void oracle_field_destroy(void *p) {
  o_field *F = (o_field *)p;
  if (!F) return;
  free(F->Lb);
  free(F);
}

static void o_chol_solve(o_field *F, double *x) {
  int n = F->n, bw = F->bw;
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    int k0 = i - bw < 0 ? 0 : i - bw;
    for (int k = k0; k < i; ++k) s -= *o_band(F, i, k) * x[k];
    x[i] = s / *o_band(F, i, i);
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    int k1 = i + bw > n - 1 ? n - 1 : i + bw;
    for (int k = i + 1; k <= k1; ++k) s -= *o_band(F, k, i) * x[k];
    x[i] = s / *o_band(F, i, i);
  }
}

/* One implicit field solve.  Inputs: E^n (er0, ez0), H^n (h0), dQ (ir, iz),
 * drive voltages V^n (v0) and V^{n+1} (v1).  Outputs: E^{n+1} (er1, ez1),
 * H^{n+1} (h1); *src = energy delivered through prescribed edges over dt. */
void oracle_field_solve(void *p, const double *er0, const double *ez0, const double *h0,
                        const double *ir, const double *iz, double v0, double v1, double L,
                        double *er1, double *ez1, double *h1, double *src) {
  o_field *F = (o_field *)p;
  int nr = F->nr, nz = F->nz;
  og_grid g = {nr, nz, F->dr, F->dz, F->xa, F->nd, F->erd, F->sgd};
  double dt = F->dt, eps = F->eps, mu = F->mu;
  double *x = (double *)malloc(sizeof(double) * (size_t)F->n);
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nz; ++j) x[i * nz + j] = 2.0 * mu * o_vol_h(&g, i) * h0[i * nz + j];
  /* - dt * C^T L Et over all edges; Et = (eps A E^n - dQ/2)/D (unknown) or E^{n+1/2} (prescribed) */
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j <= nz; ++j) {
      double et;
      if (j == 0 || j == nz) et = 0.0;
      else et = (eps * o_aeff_r(&g, i) * er0[i * (nz + 1) + j] - 0.5 * ir[i * (nz + 1) + j]) /
                o_dnr(&g, eps, dt, i);
      double s = O_TWO_PI * o_rhalf(&g, i);
      if (j <= nz - 1) x[i * nz + j] -= dt * (-s) * o_drc(&g, i) * et;
      if (j >= 1) x[i * nz + (j - 1)] -= dt * (s) * o_drc(&g, i) * et;
    }
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j < nz; ++j) {
      double et;
      /* gap: E_z^{n+1/2}; wave port: its source part 2 E_in^{n+1/2}, the same
       * value (the -eta H part sits in the matrix) */
      if (i == nr) et = 0.5 * (v0 + v1) / L;
      else et = (eps * o_aeff_z(&g, i) * ez0[i * nz + j] - 0.5 * iz[i * nz + j]) /
                o_dnz(&g, eps, dt, i);
      if (i <= nr - 1) x[i * nz + j] -= dt * (O_TWO_PI * o_rhalf(&g, i)) * F->dz * et;
      if (i >= 1) x[(i - 1) * nz + j] -= dt * (-O_TWO_PI * o_rhalf(&g, i - 1)) * F->dz * et;
    }
  o_chol_solve(F, x); /* x = H^{n+1/2} */
  for (int c = 0; c < F->n; ++c) h1[c] = 2.0 * x[c] - h0[c];
  double srcE = 0.0;
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j <= nz; ++j) {
      int e = i * (nz + 1) + j;
      if (j == 0 || j == nz) { er1[e] = 0.0; continue; }
      double s = O_TWO_PI * o_rhalf(&g, i);
      double ch = -s * x[i * nz + j] + s * x[i * nz + j - 1];
      /* Ampere with E_half: (eps A + dt S/2) E1 = (eps A - dt S/2) E0 + dt C H - dQ */
      er1[e] = ((eps * o_aeff_r(&g, i) - 0.5 * dt * o_asig_r(&g, i)) * er0[e] + dt * ch - ir[e]) /
               o_dnr(&g, eps, dt, i);
    }
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j < nz; ++j) {
      int e = i * nz + j;
      double ch = 0.0;
      if (i <= nr - 1) ch += O_TWO_PI * o_rhalf(&g, i) * x[i * nz + j];
      if (i >= 1) ch += -O_TWO_PI * o_rhalf(&g, i - 1) * x[(i - 1) * nz + j];
      if (i == nr) {
        double eh;
        if (F->wave) {  /* E_z^{n+1/2}(R) = 2 E_in^{n+1/2} - eta H^{n+1/2} */
          eh = 0.5 * (v0 + v1) / L - sqrt(F->mu / eps) * x[(nr - 1) * nz + j];
          ez1[e] = 2.0 * eh - ez0[e];
        } else {
          eh = 0.5 * (v0 + v1) / L;
          ez1[e] = v1 / L;
        }
        srcE += eh * F->dz * (iz[e] - dt * ch);
      } else {
        ez1[e] = ((eps * o_aeff_z(&g, i) - 0.5 * dt * o_asig_z(&g, i)) * ez0[e] + dt * ch - iz[e]) /
                 o_dnz(&g, eps, dt, i);
      }
    }
  if (src) *src = srcE;
  free(x);
}

/* Charge carried by the conduction current of a conducting ring over one step
 * (Eq. 2's sigma E at the half step): each unknown edge moves dt S E_half from
 * the node at its lower end to the node at its upper end.  Subtracted from qc
 * (nodes, (nr+1) x (nz+1)), so that Gauss's law holds with qc added to the
 * particle and wall charge.  Returns the Ohmic energy dt sum S L E_half^2. */
double oracle_conduction_charge(void *p, const double *er0, const double *ez0, const double *er1,
                                const double *ez1, double *qc) {
  o_field *F = (o_field *)p;
  int nr = F->nr, nz = F->nz;
  og_grid g = {nr, nz, F->dr, F->dz, F->xa, F->nd, F->erd, F->sgd};
  double dt = F->dt, heat = 0.0;
  for (int i = 0; i < nr; ++i)
    for (int j = 1; j < nz; ++j) {
      int e = i * (nz + 1) + j;
      double q = dt * o_asig_r(&g, i) * 0.5 * (er0[e] + er1[e]);
      qc[i * (nz + 1) + j] -= q;
      qc[(i + 1) * (nz + 1) + j] += q;
      heat += q * 0.5 * (er0[e] + er1[e]) * o_drc(&g, i);
    }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nz; ++j) {
      int e = i * nz + j;
      double q = dt * o_asig_z(&g, i) * 0.5 * (ez0[e] + ez1[e]);
      qc[i * (nz + 1) + j] -= q;
      qc[i * (nz + 1) + j + 1] += q;
      heat += q * 0.5 * (ez0[e] + ez1[e]) * F->dz;
    }
  return heat;
}

/* field energy over unknown edges and H cells */
double oracle_field_energy(int nr, int nz, double dr, double dz, int xa, int nd, double erd,
                           double eps, double mu,
                           const double *er, const double *ez, const double *h) {
  og_grid g = {nr, nz, dr, dz, xa, nd, erd, 0.0};  /* conductivity: not used here */
  double W = 0.0;
  for (int i = 0; i < nr; ++i)
    for (int j = 1; j < nz; ++j) {
      double e = er[i * (nz + 1) + j];
      W += 0.5 * eps * e * e * o_aeff_r(&g, i) * o_drc(&g, i);
    }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nz; ++j) {
      double e = ez[i * nz + j];
      W += 0.5 * eps * e * e * o_aeff_z(&g, i) * dz;
    }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nz; ++j) {
      double hh = h[i * nz + j];
      W += 0.5 * mu * hh * hh * o_vol_h(&g, i);
    }
  return W;
}

/* Gauss residual eps*div E - Q at interior nodes i=0..nr-1, j=1..nz-1 (others 0) */
void oracle_gauss_residual(int nr, int nz, double dr, double dz, int xa, int nd, double erd,
                           double eps,
                           const double *er,
                           const double *ez, const double *Q, double *G) {
  og_grid g = {nr, nz, dr, dz, xa, nd, erd, 0.0};  /* conductivity: not used here */
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j <= nz; ++j) G[i * (nz + 1) + j] = 0.0;
  for (int i = 0; i < nr; ++i)
    for (int j = 1; j < nz; ++j) {
      double flux = o_aeff_r(&g, i) * er[i * (nz + 1) + j];
      if (i >= 1) flux -= o_aeff_r(&g, i - 1) * er[(i - 1) * (nz + 1) + j];
      flux += o_aeff_z(&g, i) * (ez[i * nz + j] - ez[i * nz + j - 1]);
      G[i * (nz + 1) + j] = eps * flux - Q[i * (nz + 1) + j];
    }
}

double oracle_kinetic_energy(double m, int64_t n, const int32_t *cell, const double *vr,
                             const double *vt, const double *vz, const double *w) {
  double K = 0.0;
  for (int64_t p = 0; p < n; ++p) {
    if (cell[p] < 0) continue;
    K += 0.5 * m * w[p] * (vr[p] * vr[p] + vt[p] * vt[p] + vz[p] * vz[p]);
  }
  return K;
}

/* ------------------------------------------------------------------ MCC */
/* Analytic argon-like cross sections [m^2], energies in eV (project forms;
 * the paper uses Phelps data, Sec. 2.1). */
double oracle_sigma_el(double eps) {
  double x = eps / 12.0;
  return 1.5e-19 * x / (1.0 + x * x) + 1e-20;
}
double oracle_sigma_ex(double eps) {
  if (!(eps > 11.5)) return 0.0;
  double u = eps / 11.5;
  return 4e-20 * log(u) / u;
}
double oracle_sigma_iz(double eps) {
  if (!(eps > 15.76)) return 0.0;
  double u = eps / 15.76;
  return 8e-20 * log(u) / u;
}

/* max over eps in (0, 1 keV] of sigma_tot(eps)*v(eps), sampled on a uniform grid, times 1.01 */
double oracle_numax_e(double ng, double me) {
  double best = 0.0;
  for (int k = 1; k <= 200000; ++k) {
    double eps = 1000.0 * (double)k / 200000.0;
    double v = sqrt(2.0 * eps * O_QE / me);
    double s = oracle_sigma_el(eps) + oracle_sigma_ex(eps) + oracle_sigma_iz(eps);
    double nu = ng * s * v;
    if (nu > best) best = nu;
  }
  return 1.01 * best;
}

static void o_iso_dir(double u2, double u3, double *nr_, double *nt_, double *nz_) {
  double ct = 1.0 - 2.0 * u2;
  double st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double ph = O_TWO_PI * u3;
  *nr_ = st * cos(ph);
  *nt_ = st * sin(ph);
  *nz_ = ct;
}

typedef struct {
  int64_t p;
  uint32_t id;
  double v1;
} o_iz;

static int o_iz_cmp(const void *x, const void *y) {
  uint32_t a = ((const o_iz *)x)->id, b = ((const o_iz *)y)->id;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* Null-collision MCC (row a7), after Mertmann et al. 2011 / Vahedi & Surendra.
 * Electrons: elastic, excitation (11.5 eV), ionization (15.76 eV, equal split,
 * new e + Ar+ at the parent's position with its weight).  Ions: charge
 * exchange with constant cross section against a 300 K neutral Maxwellian.
 * pnull_* = 1 - exp(-numax_* dt), supplied by the caller.  New pairs are
 * appended in order of the parent's id (so ids do not depend on how the
 * store happens to be ordered); their ids continue from *next_id_*.  If the
 * capacity cannot take all pairs of this pass, none is appended (rc -5).
 * counts[8]: cand_e, el, ex, iz, cand_i, cx, gmax overflow, capacity overflow */
int oracle_mcc(uint64_t seed, uint64_t step, double ng, double tg, double me, double mi,
               double numax_e, double pnull_e, double pnull_i, double gmax,
               int64_t *ne, int64_t cap_e, int32_t *ce, double *ae, double *be, double *vre,
               double *vte, double *vze, double *we, uint32_t *ide, uint32_t *next_id_e,
               int64_t *ni, int64_t cap_i, int32_t *ci, double *ai, double *bi, double *vri,
               double *vti, double *vzi, double *wi, uint32_t *idi, uint32_t *next_id_i,
               int64_t *counts, double *de_coll) {
  double vthg = sqrt(O_KB * tg / mi);
  int64_t n_e0 = *ne, n_i0 = *ni;
  int rc = 0;
  double dE = 0.0;
  o_iz *izl = (o_iz *)malloc(sizeof(o_iz) * (size_t)(n_e0 > 0 ? n_e0 : 1));
  int64_t niz = 0;
  for (int64_t p = 0; p < n_e0; ++p) {
    if (ce[p] < 0) continue;
    double u[4];
    o_draw4(seed, O_STREAM_MCC_E, ide[p], step, 0, u);
    if (!(u[0] < pnull_e)) continue;
    counts[0]++;
    double v2 = vre[p] * vre[p] + vte[p] * vte[p] + vze[p] * vze[p];
    double v = sqrt(v2);
    double eps = 0.5 * me * v2 / O_QE;
    double nu_el = ng * oracle_sigma_el(eps) * v;
    double nu_ex = ng * oracle_sigma_ex(eps) * v;
    double nu_iz = ng * oracle_sigma_iz(eps) * v;
    double x = u[1] * numax_e;
    double ke0 = 0.5 * me * we[p] * v2;
    if (x < nu_el) {
      double nr_, nt_, nz_;
      o_iso_dir(u[2], u[3], &nr_, &nt_, &nz_);
      double cchi = v > 0.0 ? (nr_ * vre[p] + nt_ * vte[p] + nz_ * vze[p]) / v : 1.0;
      double eps1 = eps * (1.0 - 2.0 * (me / mi) * (1.0 - cchi));
      double v1 = sqrt(2.0 * eps1 * O_QE / me);
      vre[p] = v1 * nr_; vte[p] = v1 * nt_; vze[p] = v1 * nz_;
      counts[1]++;
    } else if (x < nu_el + nu_ex) {
      double nr_, nt_, nz_;
      o_iso_dir(u[2], u[3], &nr_, &nt_, &nz_);
      double eps1 = eps - 11.5;
      double v1 = sqrt(2.0 * eps1 * O_QE / me);
      vre[p] = v1 * nr_; vte[p] = v1 * nt_; vze[p] = v1 * nz_;
      counts[2]++;
    } else if (x < nu_el + nu_ex + nu_iz) {
      counts[3]++;
      double nr_, nt_, nz_;
      o_iso_dir(u[2], u[3], &nr_, &nt_, &nz_);
      double eps1 = 0.5 * (eps - 15.76);
      double v1 = sqrt(2.0 * eps1 * O_QE / me);
      vre[p] = v1 * nr_; vte[p] = v1 * nt_; vze[p] = v1 * nz_;
      izl[niz].p = p;
      izl[niz].id = ide[p];
      izl[niz].v1 = v1;
      niz++;
    } else {
      continue;
    }
    dE += 0.5 * me * we[p] * (vre[p] * vre[p] + vte[p] * vte[p] + vze[p] * vze[p]) - ke0;
  }
  /* new pairs in order of the parent's id (independent of the storage order) */
  qsort(izl, (size_t)niz, sizeof(o_iz), o_iz_cmp);
  if (*ne + niz > cap_e || *ni + niz > cap_i) {
    counts[7] += niz;
    if (niz) rc = -5;
  } else {
    for (int64_t k = 0; k < niz; ++k) {
      int64_t p = izl[k].p;
      double v1 = izl[k].v1;
      double u1[4], u2[4];
      o_draw4(seed, O_STREAM_MCC_E, ide[p], step, 1, u1);
      o_draw4(seed, O_STREAM_MCC_E, ide[p], step, 2, u2);
      int64_t q = *ne;
      double mr, mt, mz;
      o_iso_dir(u1[0], u1[1], &mr, &mt, &mz);
      ce[q] = ce[p]; ae[q] = ae[p]; be[q] = be[p]; we[q] = we[p];
      vre[q] = v1 * mr; vte[q] = v1 * mt; vze[q] = v1 * mz;
      ide[q] = (*next_id_e)++;
      *ne = q + 1;
      double g1, g2, g3, g4;
      o_gauss2(u1[2], u1[3], &g1, &g2);
      o_gauss2(u2[0], u2[1], &g3, &g4);
      int64_t s = *ni;
      ci[s] = ce[p]; ai[s] = ae[p]; bi[s] = be[p]; wi[s] = we[p];
      vri[s] = vthg * g1; vti[s] = vthg * g2; vzi[s] = vthg * g3;
      idi[s] = (*next_id_i)++;
      *ni = s + 1;
      dE += 0.5 * me * we[p] * (v1 * v1) + 0.5 * mi * wi[s] * (vri[s] * vri[s] + vti[s] * vti[s] + vzi[s] * vzi[s]);
    }
  }
  free(izl);
  for (int64_t p = 0; p < n_i0; ++p) {
    if (ci[p] < 0) continue;
    double u[4];
    o_draw4(seed, O_STREAM_MCC_I, idi[p], step, 0, u);
    if (!(u[0] < pnull_i)) continue;
    counts[4]++;
    double u1[4];
    o_draw4(seed, O_STREAM_MCC_I, idi[p], step, 1, u1);
    double g1, g2, g3, g4;
    o_gauss2(u[2], u[3], &g1, &g2);
    o_gauss2(u1[0], u1[1], &g3, &g4);
    double wr = vthg * g1, wt = vthg * g2, wz = vthg * g3;
    double dr_ = vri[p] - wr, dt_ = vti[p] - wt, dz_ = vzi[p] - wz;
    double g = sqrt(dr_ * dr_ + dt_ * dt_ + dz_ * dz_);
    if (g > gmax) counts[6]++;
    if (u[1] * gmax < g) {
      double ke0 = 0.5 * mi * wi[p] * (vri[p] * vri[p] + vti[p] * vti[p] + vzi[p] * vzi[p]);
      vri[p] = wr; vti[p] = wt; vzi[p] = wz;
      dE += 0.5 * mi * wi[p] * (wr * wr + wt * wt + wz * wz) - ke0;
      counts[5]++;
    }
  }
  if (de_coll) *de_coll += dE;
  return rc;
}

/* ----------------------------------------------------------------- sort */
/* Stable counting sort by cell (row a8); absorbed particles (cell < 0) are
 * dropped.  Sorts the SoA in place via a scratch copy; returns new count. */
int64_t oracle_sort(int ncell, int64_t n, int32_t *cell, double *a, double *b, double *vr,
                    double *vt, double *vz, double *w, uint32_t *id) {
  int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  for (int64_t p = 0; p < n; ++p)
    if (cell[p] >= 0) cnt[cell[p] + 1]++;
  for (int c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
  int64_t m = cnt[ncell];
  int32_t *c2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
  double *buf = (double *)malloc(sizeof(double) * 6 * (size_t)(m ? m : 1));
  uint32_t *i2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
  for (int64_t p = 0; p < n; ++p) {
    if (cell[p] < 0) continue;
    int64_t d = cnt[cell[p]]++;
    c2[d] = cell[p];
    buf[0 * m + d] = a[p]; buf[1 * m + d] = b[p]; buf[2 * m + d] = vr[p];
    buf[3 * m + d] = vt[p]; buf[4 * m + d] = vz[p]; buf[5 * m + d] = w[p];
    i2[d] = id[p];
  }
  for (int64_t d = 0; d < m; ++d) {
    cell[d] = c2[d];
    a[d] = buf[0 * m + d]; b[d] = buf[1 * m + d]; vr[d] = buf[2 * m + d];
    vt[d] = buf[3 * m + d]; vz[d] = buf[4 * m + d]; w[d] = buf[5 * m + d];
    id[d] = i2[d];
  }
  free(cnt); free(c2); free(buf); free(i2);
  return m;
}

/* ------------------------------------------------ axial dielectric port */
/* The paper's feed (Sec. 2.2, Fig. 1): below the powered electrode, a coaxial
 * port filled with a dielectric (relative permittivity erq) runs from the
 * electrode radius r_p = r(ip) to r = R, nzp rows of cells deep, of heights
 * hq[q] (q = 0 at the port's end, q = nzp - 1 at the junction; uniform, or
 * graded to lengthen the waveguide in few cells, Sec. 2.1's nonuniform mesh); the
 * electrode's stem (r < r_p) and the outer wall (r = R) are conductors (E_z = 0
 * on them), the powered electrode face (z = 0, r < r_p) stays a plate (E_r = 0)
 * and the reactor's side wall r = R a conductor (E_z = 0).  The port cells
 * carry H_theta like the reactor's; the E_r edges on z = 0 for r > r_p join the
 * two (interface edges: their dual face is half in the port, half in the
 * reactor, D = eps 2 pi r (erq hq[nzp-1] / 2 + dz / 2); the E_r edges between
 * port rows q - 1 and q have the dual length (hq[q-1] + hq[q]) / 2).  At the
 * port's end Eq. 5, Mur's condition for the outgoing TEM wave with an incoming one,
 * is taken in its characteristic form E_r + eta H_theta = 2 E_r^+ (eta =
 * sqrt(mu / (erq eps))), CN-centred, with the incoming wave of Eq. 7's
 * reading: the coaxial TEM field E_r^+(r) = phi^+ / (r ln(R / r_p)) of half
 * the electrode potential, phi^+ = phi / 2 (the paper's phi^+ ~ phi / 2).  So
 * 2 E_r^+ at the half step is phi^{n+1/2} / (r ln(R / r_p)); eliminating E as in
 * the reactor adds dt 2 pi r_{i+1/2} dr_i eta to the diagonal of the bottom
 * port cells.  H unknowns are numbered column by column, the nzp port cells
 * (bottom to top) before the column's reactor cells (dummy identity rows where
 * r < r_p), so the system is banded with bandwidth nzp + nz; banded Cholesky. */
typedef struct {
  int nr, nz, ip, nzp, cs, n, bw, xa;
  double dr, dz, erq, dt, eps, mu, lnr;
  double *hq;   /* nzp row heights */
  double *Lb;
} o_pfield;

static double *o_pband(o_pfield *F, int i, int j) {
  return &F->Lb[(size_t)i * (F->bw + 1) + (j - i + F->bw)];
}
static int o_pidx(const o_pfield *F, int i, int jj) { return i * F->cs + F->nzp + jj; }
static double o_dint(const og_grid *g, const o_pfield *F, int i) {
  return F->eps * O_TWO_PI * o_rhalf(g, i) * (0.5 * F->erq * F->hq[F->nzp - 1] + 0.5 * F->dz);
}
/* the E_r edge between port rows q - 1 and q (q >= 1) */
static double o_dpr(const og_grid *g, const o_pfield *F, int i, int q) {
  return F->eps * F->erq * O_TWO_PI * o_rhalf(g, i) * (0.5 * (F->hq[q - 1] + F->hq[q]));
}
static double o_dpz(const og_grid *g, const o_pfield *F, int i) {
  return F->eps * F->erq * o_area_z(g, i);
}
static double o_vol_hp(const og_grid *g, const o_pfield *F, int i, int q) {
  return O_TWO_PI * o_rhalf(g, i) * o_drc(g, i) * F->hq[q];
}
/* 2 E_r^+ at the half step on the port's end edge (i + 1/2) */
static double o_port_ein2(const og_grid *g, const o_pfield *F, int i, double phi_half) {
  return phi_half / (o_rhalf(g, i) * F->lnr);
}

/* hq: the nzp row heights (copied) */
void *oracle_port_create_graded(int nr, int nz, double dr, double dz, int xa, int ip, int nzp,
                                const double *hq, double erq, double dt, double eps,
                                double mu) {
  if (ip < 1 || ip >= nr || nzp < 1 || !hq) return NULL;
  for (int q = 0; q < nzp; ++q)
    if (!(hq[q] > 0.0)) return NULL;
  o_pfield *F = (o_pfield *)calloc(1, sizeof(o_pfield));
  og_grid g = {nr, nz, dr, dz, xa, 0, 1.0, 0.0};
  F->nr = nr; F->nz = nz; F->ip = ip; F->nzp = nzp; F->xa = xa;
  F->dr = dr; F->dz = dz; F->erq = erq; F->dt = dt; F->eps = eps; F->mu = mu;
  F->hq = (double *)malloc(sizeof(double) * nzp);
  if (!F->hq) { free(F); return NULL; }
  memcpy(F->hq, hq, sizeof(double) * nzp);
  F->lnr = log(o_rnode(&g, nr) / o_rnode(&g, ip));
  F->cs = nzp + nz;
  F->n = nr * F->cs;
  F->bw = F->cs;
  F->Lb = (double *)calloc((size_t)F->n * (F->bw + 1), sizeof(double));
  if (!F->Lb) { free(F->hq); free(F); return NULL; }
  const double hdt2 = 0.5 * dt * dt, eta = sqrt(mu / (erq * eps));
  for (int i = 0; i < nr; ++i) {
    const double s = O_TWO_PI * o_rhalf(&g, i), L = o_drc(&g, i);
    for (int j = 0; j < nz; ++j) *o_pband(F, o_pidx(F, i, j), o_pidx(F, i, j)) += 2.0 * mu * o_vol_h(&g, i);
    for (int q = 0; q < nzp; ++q) {
      const int c = o_pidx(F, i, q - nzp);
      *o_pband(F, c, c) += i >= ip ? 2.0 * mu * o_vol_hp(&g, F, i, q) : 1.0;
    }
    /* reactor E_r edges j = 1..nz-1 */
    for (int j = 1; j < nz; ++j) {
      const double W = L / (eps * o_area_r(&g, i));
      const int lo = o_pidx(F, i, j - 1), hi = o_pidx(F, i, j);
      *o_pband(F, lo, lo) += hdt2 * W * s * s;
      *o_pband(F, hi, hi) += hdt2 * W * s * s;
      *o_pband(F, hi, lo) -= hdt2 * W * s * s;
    }
    if (i < ip) continue;
    /* interface edge (z = 0) and the port's E_r edges between its rows */
    {
      const double W = L / o_dint(&g, F, i);
      const int lo = o_pidx(F, i, -1), hi = o_pidx(F, i, 0);
      *o_pband(F, lo, lo) += hdt2 * W * s * s;
      *o_pband(F, hi, hi) += hdt2 * W * s * s;
      *o_pband(F, hi, lo) -= hdt2 * W * s * s;
    }
    for (int q = 1; q < nzp; ++q) {
      const double W = L / o_dpr(&g, F, i, q);
      const int lo = o_pidx(F, i, q - 1 - nzp), hi = o_pidx(F, i, q - nzp);
      *o_pband(F, lo, lo) += hdt2 * W * s * s;
      *o_pband(F, hi, hi) += hdt2 * W * s * s;
      *o_pband(F, hi, lo) -= hdt2 * W * s * s;
    }
    /* the port's end: E_r = 2 E^+ - eta H */
    { const int c = o_pidx(F, i, -nzp); *o_pband(F, c, c) += dt * s * L * eta; }
  }
  /* E_z edges: reactor (i, j + 1/2) for i < nr (i = nr: wall, E_z = 0); the
   * port's (i, q + 1/2) for ip < i < nr (r_p and R: conductors) */
  for (int i = 0; i < nr; ++i) {
    const double sr = O_TWO_PI * o_rhalf(&g, i);
    const double sl = i >= 1 ? O_TWO_PI * o_rhalf(&g, i - 1) : 0.0;
    for (int j = 0; j < nz; ++j) {
      const double W = dz / (eps * o_area_z(&g, i));
      const int cr = o_pidx(F, i, j);
      *o_pband(F, cr, cr) += hdt2 * W * sr * sr;
      if (i >= 1) {
        const int cl = o_pidx(F, i - 1, j);
        *o_pband(F, cl, cl) += hdt2 * W * sl * sl;
        *o_pband(F, cr, cl) -= hdt2 * W * sl * sr;
      }
    }
    if (i <= ip) continue;
    for (int q = 0; q < nzp; ++q) {
      const double W = F->hq[q] / o_dpz(&g, F, i);
      const int cr = o_pidx(F, i, q - nzp), cl = o_pidx(F, i - 1, q - nzp);
      *o_pband(F, cr, cr) += hdt2 * W * sr * sr;
      *o_pband(F, cl, cl) += hdt2 * W * sl * sl;
      *o_pband(F, cr, cl) -= hdt2 * W * sl * sr;
    }
  }
  int n = F->n, bw = F->bw;
  for (int i = 0; i < n; ++i) {
    int j0 = i - bw < 0 ? 0 : i - bw;
    for (int j = j0; j <= i; ++j) {
      double sum = *o_pband(F, i, j);
      int k0 = j0 > j - bw ? j0 : j - bw;
      for (int k = k0; k < j; ++k) sum -= *o_pband(F, i, k) * *o_pband(F, j, k);
      if (i == j) {
        if (!(sum > 0.0)) { free(F->Lb); free(F->hq); free(F); return NULL; }
        *o_pband(F, i, i) = sqrt(sum);
      } else {
        *o_pband(F, i, j) = sum / *o_pband(F, j, j);
      }
    }
  }
  return F;
}

void *oracle_port_create(int nr, int nz, double dr, double dz, int xa, int ip, int nzp,
                         double dzp, double erq, double dt, double eps, double mu) {
  if (nzp < 1) return NULL;
  double *hq = (double *)malloc(sizeof(double) * nzp);
  if (!hq) return NULL;
  for (int q = 0; q < nzp; ++q) hq[q] = dzp;
  void *F = oracle_port_create_graded(nr, nz, dr, dz, xa, ip, nzp, hq, erq, dt, eps, mu);
  free(hq);
  return F;
}

void oracle_port_destroy(void *p) {
  o_pfield *F = (o_pfield *)p;
  if (!F) return;
  free(F->Lb);
  free(F->hq);
  free(F);
}

/* One implicit field solve with the port.  Reactor arrays as in
 * oracle_field_solve (E_r of j = 0 holds the interface edges for i >= ip, E_z of
 * i = nr stays zero); port arrays: hp[(i-ip)*nzp + q], erp[(i-ip)*nzp + q] (E_r on
 * the port's lower face of cell (i, q): q = 0 the end edge), ezp[(i-ip)*nzp + q]
 * for nodes i = ip..nr (zero on the conductors).  phi0, phi1: electrode
 * potential at n and n+1.  *src: energy delivered through the port's end. */
void oracle_port_solve(void *p, const double *er0, const double *ez0, const double *h0,
                       const double *erp0, const double *ezp0, const double *hp0,
                       const double *ir, const double *iz, double phi0, double phi1,
                       double *er1, double *ez1, double *h1, double *erp1, double *ezp1,
                       double *hp1, double *src) {
  o_pfield *F = (o_pfield *)p;
  const int nr = F->nr, nz = F->nz, ip = F->ip, nzp = F->nzp;
  og_grid g = {nr, nz, F->dr, F->dz, F->xa, 0, 1.0, 0.0};
  const double dt = F->dt, eps = F->eps, mu = F->mu, eta = sqrt(mu / (F->erq * eps));
  const double phih = 0.5 * (phi0 + phi1);
  double *x = (double *)calloc((size_t)F->n, sizeof(double));
  for (int i = 0; i < nr; ++i) {
    for (int j = 0; j < nz; ++j) x[o_pidx(F, i, j)] = 2.0 * mu * o_vol_h(&g, i) * h0[i * nz + j];
    if (i >= ip)
      for (int q = 0; q < nzp; ++q)
        x[o_pidx(F, i, q - nzp)] = 2.0 * mu * o_vol_hp(&g, F, i, q) * hp0[(i - ip) * nzp + q];
  }
  /* - dt C^T L Et over the unknown edges (and the end edges' 2 E^+) */
  for (int i = 0; i < nr; ++i) {
    const double s = O_TWO_PI * o_rhalf(&g, i), L = o_drc(&g, i);
    for (int j = 1; j < nz; ++j) {
      const double D = eps * o_area_r(&g, i);
      const double et = (D * er0[i * (nz + 1) + j] - 0.5 * ir[i * (nz + 1) + j]) / D;
      x[o_pidx(F, i, j)] -= dt * (-s) * L * et;
      x[o_pidx(F, i, j - 1)] -= dt * (s) * L * et;
    }
    if (i < ip) continue;
    {
      const double D = o_dint(&g, F, i);
      const double et = (D * er0[i * (nz + 1)] - 0.5 * ir[i * (nz + 1)]) / D;
      x[o_pidx(F, i, 0)] -= dt * (-s) * L * et;
      x[o_pidx(F, i, -1)] -= dt * (s) * L * et;
    }
    for (int q = 1; q < nzp; ++q) {
      const double et = erp0[(i - ip) * nzp + q];
      x[o_pidx(F, i, q - nzp)] -= dt * (-s) * L * et;
      x[o_pidx(F, i, q - 1 - nzp)] -= dt * (s) * L * et;
    }
    x[o_pidx(F, i, -nzp)] -= dt * (-s) * L * o_port_ein2(&g, F, i, phih);
  }
  for (int i = 0; i < nr; ++i) {
    const double sr = O_TWO_PI * o_rhalf(&g, i);
    const double sl = i >= 1 ? O_TWO_PI * o_rhalf(&g, i - 1) : 0.0;
    for (int j = 0; j < nz; ++j) {
      const double D = eps * o_area_z(&g, i);
      const double et = (D * ez0[i * nz + j] - 0.5 * iz[i * nz + j]) / D;
      x[o_pidx(F, i, j)] -= dt * sr * F->dz * et;
      if (i >= 1) x[o_pidx(F, i - 1, j)] -= dt * (-sl) * F->dz * et;
    }
    if (i <= ip) continue;
    for (int q = 0; q < nzp; ++q) {
      const double et = ezp0[(i - ip) * nzp + q];
      x[o_pidx(F, i, q - nzp)] -= dt * sr * F->hq[q] * et;
      x[o_pidx(F, i - 1, q - nzp)] -= dt * (-sl) * F->hq[q] * et;
    }
  }
  /* banded Cholesky solve: x = H^{n+1/2} */
  {
    const int n = F->n, bw = F->bw;
    for (int i = 0; i < n; ++i) {
      double sum = x[i];
      const int k0 = i - bw < 0 ? 0 : i - bw;
      for (int k = k0; k < i; ++k) sum -= *o_pband(F, i, k) * x[k];
      x[i] = sum / *o_pband(F, i, i);
    }
    for (int i = n - 1; i >= 0; --i) {
      double sum = x[i];
      const int k1 = i + bw > n - 1 ? n - 1 : i + bw;
      for (int k = i + 1; k <= k1; ++k) sum -= *o_pband(F, k, i) * x[k];
      x[i] = sum / *o_pband(F, i, i);
    }
  }
  for (int i = 0; i < nr; ++i) {
    for (int j = 0; j < nz; ++j) h1[i * nz + j] = 2.0 * x[o_pidx(F, i, j)] - h0[i * nz + j];
    if (i >= ip)
      for (int q = 0; q < nzp; ++q)
        hp1[(i - ip) * nzp + q] = 2.0 * x[o_pidx(F, i, q - nzp)] - hp0[(i - ip) * nzp + q];
  }
  double srcE = 0.0;
  for (int i = 0; i < nr; ++i) {
    const double s = O_TWO_PI * o_rhalf(&g, i), L = o_drc(&g, i);
    for (int j = 0; j <= nz; ++j) {
      const int e = i * (nz + 1) + j;
      if (j == nz || (j == 0 && i < ip)) { er1[e] = 0.0; continue; }
      const double ch = -s * x[o_pidx(F, i, j)] + s * x[o_pidx(F, i, j - 1)];
      const double D = j == 0 ? o_dint(&g, F, i) : eps * o_area_r(&g, i);
      er1[e] = (D * er0[e] + dt * ch - ir[e]) / D;
    }
    if (i < ip) continue;
    for (int q = 0; q < nzp; ++q) {
      const int e = (i - ip) * nzp + q;
      if (q == 0) {
        const double xb = x[o_pidx(F, i, -nzp)];
        const double eh = o_port_ein2(&g, F, i, phih) - eta * xb;
        erp1[e] = 2.0 * eh - erp0[e];
        srcE += eh * L * dt * s * xb;
      } else {
        const double ch = -s * x[o_pidx(F, i, q - nzp)] + s * x[o_pidx(F, i, q - 1 - nzp)];
        erp1[e] = erp0[e] + dt * ch / o_dpr(&g, F, i, q);
      }
    }
  }
  for (int i = 0; i <= nr; ++i) {
    const double sr = i < nr ? O_TWO_PI * o_rhalf(&g, i) : 0.0;
    const double sl = i >= 1 ? O_TWO_PI * o_rhalf(&g, i - 1) : 0.0;
    for (int j = 0; j < nz; ++j) {
      const int e = i * nz + j;
      if (i == nr) { ez1[e] = 0.0; continue; }
      double ch = sr * x[o_pidx(F, i, j)];
      if (i >= 1) ch -= sl * x[o_pidx(F, i - 1, j)];
      const double D = eps * o_area_z(&g, i);
      ez1[e] = (D * ez0[e] + dt * ch - iz[e]) / D;
    }
    if (i < ip) continue;
    for (int q = 0; q < nzp; ++q) {
      const int e = (i - ip) * nzp + q;
      if (i == ip || i == nr) { ezp1[e] = 0.0; continue; }
      const double ch = sr * x[o_pidx(F, i, q - nzp)] - sl * x[o_pidx(F, i - 1, q - nzp)];
      ezp1[e] = ezp0[e] + dt * ch / o_dpz(&g, F, i);
    }
  }
  if (src) *src = srcE;
  free(x);
}

/* Field energy of the reactor and the port: sum over edges of D L E^2 / 2 and
 * over H cells of mu V_h H^2 / 2 (the interface edges with their D). */
double oracle_port_energy(void *p, const double *er, const double *ez, const double *h,
                          const double *erp, const double *ezp, const double *hp) {
  o_pfield *F = (o_pfield *)p;
  const int nr = F->nr, nz = F->nz, ip = F->ip, nzp = F->nzp;
  og_grid g = {nr, nz, F->dr, F->dz, F->xa, 0, 1.0, 0.0};
  double W = 0.0;
  for (int i = 0; i < nr; ++i) {
    const double L = o_drc(&g, i);
    for (int j = 0; j < nz; ++j) W += 0.5 * F->mu * o_vol_h(&g, i) * h[i * nz + j] * h[i * nz + j];
    for (int j = 1; j < nz; ++j) {
      const double e = er[i * (nz + 1) + j];
      W += 0.5 * F->eps * o_area_r(&g, i) * L * e * e;
    }
    if (i >= ip) {
      const double e = er[i * (nz + 1)];
      W += 0.5 * o_dint(&g, F, i) * L * e * e;
      for (int q = 0; q < nzp; ++q) {
        const double hv = hp[(i - ip) * nzp + q];
        W += 0.5 * F->mu * o_vol_hp(&g, F, i, q) * hv * hv;
        if (q >= 1) {
          const double ev = erp[(i - ip) * nzp + q];
          W += 0.5 * o_dpr(&g, F, i, q) * L * ev * ev;
        }
      }
    }
  }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nz; ++j) {
      const double e = ez[i * nz + j];
      W += 0.5 * F->eps * o_area_z(&g, i) * F->dz * e * e;
    }
  for (int i = ip + 1; i < nr; ++i)
    for (int q = 0; q < nzp; ++q) {
      const double e = ezp[(i - ip) * nzp + q];
      W += 0.5 * o_dpz(&g, F, i) * F->hq[q] * e * e;
    }
  return W;
}

/* ----------------------------------------------------------- full step */
/* One time step of the implicit method (rows a2-a8): Picard iteration of
 * push+deposit and field solve (Sec. 2.1, after Taitano 2013 / Eremin 2022),
 * commit push with the field iterate whose deposit fed the last solve, MCC,
 * sort.  Species arrays are passed as parallel pointer tables. */
typedef struct {
  int32_t *cell; double *a, *b, *vr, *vt, *vz, *w; uint32_t *id;
  int64_t n, cap;
  uint32_t next_id;
  double q, m;
} orc_species;

typedef struct {
  int nr, nz;
  double dr, dz, R, L, dt;
  double freq, volt, eps, mu, bz;
  double tol; int kmax;
  int mcc_on;
  double ng, tg, numax_e, pnull_e, pnull_i, gmax;
  uint64_t seed;
  double cblock;       /* blocking capacitor [F] between generator and electrode (Eq. 6); 0 = none */
  int xa;              /* mapped mesh: cells near the axis with r proportional to sqrt(xi) */
  int wave;            /* 1: wave port on r = R (the field object must be created with it) */
  int nd;              /* dielectric ring: outer cells, relative permittivity erd */
  double erd;
} orc_cfg;

typedef struct {
  int picard_iters;
  int converged;
  double last_res;
  double src_energy;   /* energy in through the drive gap */
  double ke_lost;      /* kinetic energy of absorbed particles */
  double de_coll;      /* kinetic-energy change from collisions */
  int64_t counters[4]; /* substep err, absorbed, substeps, fallbacks (commit push) */
  int64_t mcc[8];
} orc_stats;

/* Eq. 6 solved for the electrode potential phi^{n+1} of one Picard iteration.
 * The reactor-side current is the displacement current plus the crossed
 * charge (and, in a conducting ring, the conduction current at the half step)
 * through the dual faces of the first row of E_z edges above the
 * powered plate (i < nr, j = 1/2): the integral over the electrode in Eq. 6
 * on the integral-form mesh.  It must equal the capacitor current
 * (C (V^{n+1} - phi^{n+1}) - q^n) / dt.  The field solve is affine in the
 * electrode potential at n+1, so a solve at phi = V^{n+1} and the response to
 * a unit potential (no charge, no fields at n) give phi^{n+1} directly. */
static double o_circuit(const orc_cfg *cfg, void *field, const double *er, const double *ez,
                        const double *h, const double *ir, const double *iz, double phi_n,
                        double v1, double qn) {
  int nr = cfg->nr, nz = cfg->nz;
  size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz, nh = (size_t)nr * nz;
  og_grid g = {nr, nz, cfg->dr, cfg->dz, cfg->xa, cfg->nd, cfg->erd, ((o_field *)field)->sgd};
  double *era = (double *)malloc(sizeof(double) * ner), *eza = (double *)malloc(sizeof(double) * nez);
  double *ha = (double *)malloc(sizeof(double) * nh);
  double *zr = (double *)calloc(ner, sizeof(double)), *zz = (double *)calloc(nez, sizeof(double));
  double *zh = (double *)calloc(nh, sizeof(double));
  double *eru = (double *)malloc(sizeof(double) * ner), *ezu = (double *)malloc(sizeof(double) * nez);
  double *hu = (double *)malloc(sizeof(double) * nh);
  double src;
  oracle_field_solve(field, er, ez, h, ir, iz, phi_n, v1, cfg->L, era, eza, ha, &src);
  oracle_field_solve(field, zr, zz, zh, zr, zz, 0.0, 1.0, cfg->L, eru, ezu, hu, &src);
  double dq = 0.0, gu = 0.0;
  for (int i = 0; i < nr; ++i) {
    double ea = cfg->eps * o_aeff_z(&g, i), hs = 0.5 * cfg->dt * o_asig_z(&g, i);
    dq += ea * (eza[i * nz] - ez[i * nz]) + iz[i * nz] + hs * (eza[i * nz] + ez[i * nz]);
    gu += (ea + hs) * ezu[i * nz];
  }
  free(era); free(eza); free(ha); free(zr); free(zz); free(zh); free(eru); free(ezu); free(hu);
  /* C (V - phi) - q^n = dq + (phi - V) gu */
  return v1 - (qn + dq) / (cfg->cblock + gu);
}

/* the axial port's solver and its fields at n (oracle_step_port) */
typedef struct {
  void *pf;
  double *hp, *erp, *ezp;
} o_port_state;

/* Eq. 6 with the axial port: the reactor-side current is that through the
 * dual faces of the first row of E_z edges over the powered electrode
 * (i < ip, j = 1/2); the solve is affine in phi^{n+1} through Eq. 7's incoming
 * wave, so a solve at phi = V^{n+1} and the response to a unit potential give
 * phi^{n+1} as in o_circuit. */
static double o_circuit_port(const orc_cfg *cfg, o_port_state *ps, const double *er,
                             const double *ez, const double *h, const double *ir,
                             const double *iz, double phi_n, double v1, double qn) {
  const o_pfield *P = (const o_pfield *)ps->pf;
  const int nr = cfg->nr, nz = cfg->nz;
  const size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz, nh = (size_t)nr * nz;
  const size_t np = (size_t)(P->nr - P->ip) * P->nzp, nzz = (size_t)(P->nr - P->ip + 1) * P->nzp;
  og_grid g = {nr, nz, cfg->dr, cfg->dz, cfg->xa, 0, 1.0, 0.0};
  double *a[6], *u[6], *z[8];
  const size_t sz[6] = {ner, nez, nh, np, nzz, np};
  for (int k = 0; k < 6; ++k) {
    a[k] = (double *)malloc(sizeof(double) * sz[k]);
    u[k] = (double *)malloc(sizeof(double) * sz[k]);
    z[k] = (double *)calloc(sz[k], sizeof(double));
  }
  z[6] = (double *)calloc(ner, sizeof(double));
  z[7] = (double *)calloc(nez, sizeof(double));
  double src;
  /* outputs in oracle_port_solve order: er, ez, h, erp, ezp, hp */
  oracle_port_solve(ps->pf, er, ez, h, ps->erp, ps->ezp, ps->hp, ir, iz, phi_n, v1, a[0], a[1],
                    a[2], a[3], a[4], a[5], &src);
  oracle_port_solve(ps->pf, z[0], z[1], z[2], z[3], z[4], z[5], z[6], z[7], 0.0, 1.0, u[0], u[1],
                    u[2], u[3], u[4], u[5], &src);
  double dq = 0.0, gu = 0.0;
  for (int i = 0; i < P->ip; ++i) {
    const double ea = cfg->eps * o_area_z(&g, i);
    dq += ea * (a[1][i * nz] - ez[i * nz]) + iz[i * nz];
    gu += ea * u[1][i * nz];
  }
  for (int k = 0; k < 6; ++k) { free(a[k]); free(u[k]); free(z[k]); }
  free(z[6]); free(z[7]);
  return v1 - (qn + dq) / (cfg->cblock + gu);
}

static int o_step(const orc_cfg *cfg, void *field, o_port_state *ps, uint64_t step,
                  orc_species *sp, int nspec, double *er, double *ez, double *h, double *wall_z0,
                  double *wall_zl, double *wall_r, orc_stats *st, double *circ);

/* circ (nullable; used when cfg->cblock > 0): {capacitor charge q^n,
 * electrode potential phi^n} in, the values at n+1 out after a converged step. */
int oracle_step(const orc_cfg *cfg, void *field, uint64_t step, orc_species *sp, int nspec,
                double *er, double *ez, double *h, double *wall_z0, double *wall_zl,
                double *wall_r, orc_stats *st, double *circ) {
  return o_step(cfg, field, NULL, step, sp, nspec, er, ez, h, wall_z0, wall_zl, wall_r, st, circ);
}

/* The same step with the axial port (its solver from oracle_port_create; its
 * fields hp, erp, ezp at n in, at n+1 out); the electrode follows V(t), or
 * with cfg->cblock > 0 and circ given, Eq. 6's circuit (circ as in oracle_step). */
int oracle_step_port(const orc_cfg *cfg, void *port, uint64_t step, orc_species *sp, int nspec,
                     double *er, double *ez, double *h, double *hp, double *erp, double *ezp,
                     double *wall_z0, double *wall_zl, double *wall_r, orc_stats *st,
                     double *circ) {
  o_port_state ps = {port, hp, erp, ezp};
  return o_step(cfg, NULL, &ps, step, sp, nspec, er, ez, h, wall_z0, wall_zl, wall_r, st, circ);
}

static int o_step(const orc_cfg *cfg, void *field, o_port_state *ps, uint64_t step,
                  orc_species *sp, int nspec, double *er, double *ez, double *h, double *wall_z0,
                  double *wall_zl, double *wall_r, orc_stats *st, double *circ) {
  int nr = cfg->nr, nz = cfg->nz;
  size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz, nh = (size_t)nr * nz;
  double *er1 = (double *)malloc(sizeof(double) * ner), *ez1 = (double *)malloc(sizeof(double) * nez);
  double *ern = (double *)malloc(sizeof(double) * ner), *ezn = (double *)malloc(sizeof(double) * nez);
  double *erh = (double *)malloc(sizeof(double) * ner), *ezh = (double *)malloc(sizeof(double) * nez);
  double *ir = (double *)malloc(sizeof(double) * ner), *iz = (double *)malloc(sizeof(double) * nez);
  double *h1 = (double *)malloc(sizeof(double) * nh);
  double t0 = (double)step * cfg->dt, t1 = (double)(step + 1) * cfg->dt;
  double v0 = cfg->volt * sin(O_TWO_PI * cfg->freq * t0);
  double v1 = cfg->volt * sin(O_TWO_PI * cfg->freq * t1);
  memset(st, 0, sizeof(*st));
  const int circ_on = cfg->cblock > 0.0 && circ != NULL;
  /* the port's fields of the current iterate */
  size_t np = 0, nzz = 0;
  double *hp1 = NULL, *erp1 = NULL, *ezp1 = NULL;
  if (ps) {
    const o_pfield *P = (const o_pfield *)ps->pf;
    np = (size_t)(P->nr - P->ip) * P->nzp;
    nzz = (size_t)(P->nr - P->ip + 1) * P->nzp;
    hp1 = (double *)calloc(np, sizeof(double));
    erp1 = (double *)calloc(np, sizeof(double));
    ezp1 = (double *)calloc(nzz, sizeof(double));
  }
  double phi0 = v0, phi1 = v1; /* electrode potential at n and n+1 */
  if (circ_on) phi0 = circ[1];
  /* initial iterate E^{n+1,0} = E^n (unknown edges); without a capacitor or
   * wave port the prescribed gap edges take V^{n+1}, else they keep E^n's */
  memcpy(er1, er, sizeof(double) * ner);
  memcpy(ez1, ez, sizeof(double) * nez);
  if (!circ_on && !cfg->wave && !ps)
    for (int j = 0; j < nz; ++j) ez1[nr * nz + j] = v1 / cfg->L;
  int conv = 0;
  double src = 0.0, res = 0.0;
  int k;
  for (k = 0; k < cfg->kmax; ++k) {
    for (size_t e = 0; e < ner; ++e) erh[e] = 0.5 * (er[e] + er1[e]);
    for (size_t e = 0; e < nez; ++e) ezh[e] = 0.5 * (ez[e] + ez1[e]);
    memset(ir, 0, sizeof(double) * ner);
    memset(iz, 0, sizeof(double) * nez);
    for (int s = 0; s < nspec; ++s)
      oracle_push(nr, nz, cfg->dr, cfg->dz, cfg->xa, cfg->nd, cfg->erd, cfg->dt, sp[s].q, sp[s].m, cfg->bz, sp[s].n, sp[s].cell,
                  sp[s].a, sp[s].b, sp[s].vr, sp[s].vt, sp[s].vz, sp[s].w, erh, ezh, ir, iz, 0,
                  NULL, NULL, NULL, NULL, NULL);
    if (circ_on && ps) phi1 = o_circuit_port(cfg, ps, er, ez, h, ir, iz, phi0, v1, circ[0]);
    else if (circ_on) phi1 = o_circuit(cfg, field, er, ez, h, ir, iz, phi0, v1, circ[0]);
    if (ps)
      oracle_port_solve(ps->pf, er, ez, h, ps->erp, ps->ezp, ps->hp, ir, iz, phi0, phi1, ern, ezn,
                        h1, erp1, ezp1, hp1, &src);
    else
      oracle_field_solve(field, er, ez, h, ir, iz, phi0, phi1, cfg->L, ern, ezn, h1, &src);
    double dn = 0.0, nn = 0.0;
    for (int i = 0; i < nr; ++i)
      for (int j = 1; j < nz; ++j) {
        size_t e = (size_t)i * (nz + 1) + j;
        double d = ern[e] - er1[e];
        dn += d * d;
        nn += ern[e] * ern[e];
      }
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nz; ++j) {
        size_t e = (size_t)i * nz + j;
        double d = ezn[e] - ez1[e];
        dn += d * d;
        nn += ezn[e] * ezn[e];
      }
    res = sqrt(dn) / fmax(sqrt(nn), 1e-30);
    memcpy(er1, ern, sizeof(double) * ner);
    memcpy(ez1, ezn, sizeof(double) * nez);
    if (res < cfg->tol) { conv = 1; break; }
  }
  st->picard_iters = conv ? k + 1 : k;
  st->last_res = res;
  st->converged = conv;
  int rc = 0;
  if (!conv) {
    rc = -3;
  } else {
    /* commit: erh/ezh still hold the half-step field that produced the deposit of the last solve */
    memset(ir, 0, sizeof(double) * ner);
    memset(iz, 0, sizeof(double) * nez);
    for (int s = 0; s < nspec; ++s)
      oracle_push(nr, nz, cfg->dr, cfg->dz, cfg->xa, cfg->nd, cfg->erd, cfg->dt, sp[s].q, sp[s].m, cfg->bz, sp[s].n, sp[s].cell,
                  sp[s].a, sp[s].b, sp[s].vr, sp[s].vt, sp[s].vz, sp[s].w, erh, ezh, ir, iz, 1,
                  wall_z0 ? wall_z0 + (size_t)s * (nr + 1) : NULL,
                  wall_zl ? wall_zl + (size_t)s * (nr + 1) : NULL,
                  wall_r ? wall_r + (size_t)s * (nz + 1) : NULL, st->counters, &st->ke_lost);
    memcpy(er, er1, sizeof(double) * ner);
    memcpy(ez, ez1, sizeof(double) * nez);
    memcpy(h, h1, sizeof(double) * nh);
    if (ps) {
      memcpy(ps->hp, hp1, sizeof(double) * np);
      memcpy(ps->erp, erp1, sizeof(double) * np);
      memcpy(ps->ezp, ezp1, sizeof(double) * nzz);
    }
    st->src_energy = src;
    if (circ_on) {
      circ[0] = cfg->cblock * (v1 - phi1);
      circ[1] = phi1;
    }
    if (cfg->mcc_on && nspec == 2) {
      int mr = oracle_mcc(cfg->seed, step, cfg->ng, cfg->tg, sp[0].m, sp[1].m, cfg->numax_e,
                          cfg->pnull_e, cfg->pnull_i, cfg->gmax, &sp[0].n, sp[0].cap, sp[0].cell,
                          sp[0].a, sp[0].b, sp[0].vr, sp[0].vt, sp[0].vz, sp[0].w, sp[0].id,
                          &sp[0].next_id, &sp[1].n, sp[1].cap, sp[1].cell, sp[1].a, sp[1].b,
                          sp[1].vr, sp[1].vt, sp[1].vz, sp[1].w, sp[1].id, &sp[1].next_id,
                          st->mcc, &st->de_coll);
      if (mr) rc = mr;
    }
    for (int s = 0; s < nspec; ++s)
      sp[s].n = oracle_sort(nr * nz, sp[s].n, sp[s].cell, sp[s].a, sp[s].b, sp[s].vr, sp[s].vt,
                            sp[s].vz, sp[s].w, sp[s].id);
    if (st->counters[0] && !rc) rc = -4;
  }
  free(er1); free(ez1); free(ern); free(ezn); free(erh); free(ezh); free(ir); free(iz); free(h1);
  free(hp1); free(erp1); free(ezp1);
  return rc;
}
