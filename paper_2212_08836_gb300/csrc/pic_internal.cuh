// Internal declarations of the GB300 hot path (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pic.h"

namespace pic {

// CODATA 2018
constexpr double kQE = 1.602176634e-19;
constexpr double kME = 9.1093837015e-31;
constexpr double kAMU = 1.66053906660e-27;
constexpr double kMAr = 39.948 * kAMU;
constexpr double kKB = 1.380649e-23;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.283185307179586;

// Philox streams (key word 1) and the step word used while loading
constexpr uint64_t kStreamLoadPos = 0x20, kStreamLoadVe = 0x21, kStreamLoadVi = 0x22;
constexpr uint64_t kStreamMccE = 0x10, kStreamMccI = 0x11;
constexpr uint64_t kLoadStep = 0xFFFFFFFFFFFFFFFFull;

// at most this many sub-steps per particle and pass (PIC_E_SUBSTEP beyond)
constexpr int kNsubMax = 64;

// Philox4x64-10 (Salmon et al., SC'11): 64x64 -> 128-bit products via umul64hi.
__device__ __forceinline__ void philox4x64(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    uint64_t hi0 = __umul64hi(m0, c[0]), lo0 = m0 * c[0];
    uint64_t hi1 = __umul64hi(m1, c[2]), lo1 = m1 * c[2];
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
}

// u01(x) < p  <=>  (x >> 11) < thr  with thr = ceil(p * 2^53) (integer test, no FP64)
__device__ __forceinline__ double u01(uint64_t x) {
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ void draw4(uint64_t seed, uint64_t stream, uint64_t id, uint64_t step,
                                      uint64_t block, double u[4]) {
  uint64_t c[4] = {id, step, block, 0};
  philox4x64(c, seed, stream);
  u[0] = u01(c[0]); u[1] = u01(c[1]); u[2] = u01(c[2]); u[3] = u01(c[3]);
}

__device__ __forceinline__ void gauss2(double ua, double ub, double &g1, double &g2) {
  double rho = sqrt(-2.0 * log(1.0 - ua));
  double ang = kTwoPi * ub;
  g1 = rho * cos(ang);
  g2 = rho * sin(ang);
}

// Mesh: uniform in the logical coordinates (xi, eta).  Radial mapping of the
// mapped mesh (Sec. 2.1): r(xi) = 2 dr sqrt(xa xi) in the first xa cells and
// dr (xi + xa) beyond (continuous with its slope; r J_r finite at the axis),
// linear in xi within each cell; xa = 0 is the uniform mesh r = xi dr.
constexpr int kMaxAxisCells = 16;
struct Grid {
  int nr, nz;
  double dr, dz, R, L;  // dr: spacing of the uniformly spaced part
  int xa;               // cells with r proportional to sqrt(xi)
  int nd;               // dielectric ring: the outer nd cells, relative permittivity erd
  double erd;
  double sgd;           // conductivity of the ring's cells [S/m] (0: a pure dielectric)
};

// node radius r_i, cell width J_r, cell-centre radius, and the inner-face
// radius of a cell in units of its width
__host__ __device__ inline double g_rnode(const Grid &g, int i) {
  if (i < g.xa) return 2.0 * g.dr * sqrt((double)g.xa * (double)i);
  return ((double)i + (double)g.xa) * g.dr;
}
__host__ __device__ inline double g_width(const Grid &g, int i) {
  return i < g.xa ? g_rnode(g, i + 1) - g_rnode(g, i) : g.dr;
}
__host__ __device__ inline double g_rcentre(const Grid &g, int i) {
  if (i < g.xa) return 0.5 * (g_rnode(g, i) + g_rnode(g, i + 1));
  return ((double)i + 0.5 + (double)g.xa) * g.dr;
}
__host__ __device__ inline double g_rho0(const Grid &g, int i) {
  return i < g.xa ? g_rnode(g, i) / g_width(g, i) : (double)(i + g.xa);
}
// dual-face area of the E_z edge at node i: the ring between the
// neighbouring cell centres (the disc of radius r_{1/2} on the axis)
__host__ __device__ inline double g_area_z(const Grid &g, int i) {
  if (i == 0) return kPi * g_rcentre(g, 0) * g_rcentre(g, 0);
  if (i <= g.xa) {
    const double ro = g_rcentre(g, i), ri = g_rcentre(g, i - 1);
    return kPi * (ro * ro - ri * ri);
  }
  return kTwoPi * g_rnode(g, i) * g.dr;
}
// dual-face areas weighted by the relative permittivity of the cells they
// cross (the dielectric ring; the ring's inner boundary node by halves)
__host__ __device__ inline double g_aeff_r(const Grid &g, int i) {
  const double a = kTwoPi * g_rcentre(g, i) * g.dz;
  return (g.nd > 0 && i >= g.nr - g.nd) ? g.erd * a : a;
}
__host__ __device__ inline double g_aeff_z(const Grid &g, int i) {
  const int i0 = g.nr - g.nd;
  if (g.nd == 0 || i < i0) return g_area_z(g, i);
  if (i > i0) return g.erd * g_area_z(g, i);
  const double ri = g_rnode(g, i), rm = g_rcentre(g, i - 1), rp = g_rcentre(g, i);
  return kPi * (ri * ri - rm * rm) + g.erd * kPi * (rp * rp - ri * ri);
}
// conducting part of the same dual faces (Eq. 2's sigma E in the ring): the
// ring's conductivity times the face area inside the ring
__host__ __device__ inline double g_asig_r(const Grid &g, int i) {
  return (g.nd > 0 && i >= g.nr - g.nd) ? g.sgd * (kTwoPi * g_rcentre(g, i) * g.dz) : 0.0;
}
__host__ __device__ inline double g_asig_z(const Grid &g, int i) {
  const int i0 = g.nr - g.nd;
  if (g.nd == 0 || g.sgd == 0.0 || i < i0) return 0.0;
  if (i > i0) return g.sgd * g_area_z(g, i);
  const double ri = g_rnode(g, i), rp = g_rcentre(g, i);
  return g.sgd * kPi * (rp * rp - ri * ri);
}

// Particle structure of arrays of one species; T = double (plain FP64 form)
// or float (mixed form: FP32 state in physical units)
template <typename T>
struct PartsT {
  int32_t *cell;
  T *a, *b, *vr, *vt, *vz, *w;
  uint32_t *id;
};
using Parts = PartsT<double>;
using Parts32 = PartsT<float>;

// Device counters written by the push / MCC kernels
struct DevCounters {
  unsigned long long push[5];  // substep errors, absorbed, substeps, fallbacks, FP64 flops
  unsigned long long mcc[8];
  double ke_lost;
  double de_coll;
  double norm[2];              // Picard: sum (E_new - E_it)^2, sum E_new^2
  double src;                  // drive-gap energy of the last solve
  unsigned long long iz_slots; // MCC: ionization keys written
  double pad[1];
};

// Field operator (separable direct solve of the H_theta system)
// Blocking capacitor between the generator and the powered electrode (Eq. 6),
// state on the device so that captured passes stay valid:
//   st[0] = capacitor charge q^n, st[1] = phi^{n+1} - V^{n+1} found by the latest
//   field solve, st[2] = electrode potential phi^n, st[3] = dt x the electrode
//   current of the latest solve.  st == nullptr: the electrode follows V(t).
struct Circuit {
  double *st;
  const double *hu;  // EM: H^{n+1} response to a unit electrode potential at n+1 (nr x nz)
  double C;          // capacitance [F]
  double cr;         // ES: eps sum_{i<nr} A_z(i) / L, the vacuum response of the plate flow
};

// Axial dielectric port below the powered electrode (PIC_FEED_AXIAL): m = nr -
// ip columns of nzp rows of cells, of heights hq[q] (q = 0 at the port's end;
// uniform, or graded from the junction down), relative permittivity erq, Mur's
// condition at the end with the incoming wave of half the electrode potential.
// The H system of reactor and port is B + U W U^T: B = the reactor's separable
// operator and the port block (its dense inverse Binv), U W U^T the m interface
// edges on z = 0 joining reactor cell (ip + e, 0) and port cell (e, nzp - 1).
// Solved exactly (Woodbury): x = y - Z Cinv U^T y, y = B^{-1} b, Z = B^{-1} U
// (ZR: its reactor part in the layout of FieldOp::hhalf, ZP: its port part),
// Cinv = (W^{-1} + U^T Z)^{-1}.
struct PortOp {
  int on, ip, nzp, m, np;
  double htop, erq, eta, lnr;  // htop = hq[nzp - 1], the row at the junction
  const double *hq;            // nzp row heights [m]
  const double *Binv;  // np x np, row-major
  const double *ZR;    // m blocks of the reactor hhalf layout
  const double *ZP;    // m x np
  const double *Cinv;  // m x m
  double *rhsp, *hhp;  // port right-hand side and H^{n+1/2} (np each)
  double *ws;          // m: Cinv U^T y
  const double *hp0, *erp0, *ezp0;  // port fields at n: H, E_r (end edge first), E_z
  double *hp1, *erp1, *ezp1;        // at n+1
  const double *hup;  // with the blocking capacitor: the port's H^{n+1} response to a
                      // unit electrode potential at n+1 (np; Circuit.hu's counterpart)
};

struct FieldOp {
  int nr, nz;
  int half;            // nz/2 when nz is even: even/odd split of the DCT (else 0)
  double dr, dz, dt, eps, mu, L;
  const double *Q;     // split: Qe[j*h+k] = Q(j, 2k), then Qo[j*h+k] = Q(j, 2k+1), j,k < h
                       // else the nz x nz DCT-II basis Q[j*nz+m]
  const double *QT;    // split: Qe^T, Qo^T (h x h each); else the transpose of Q
  // cyclic reduction of the tridiagonal system of column c (split: c = m/2 for
  // even m, h + m/2 for odd m; else c = m), padded to n2 = 2^k >= nr rows:
  // crc[c*5*n2 + ...] = forward multipliers (alpha, gamma), then the
  // back-substitution factors (a/b, c/b, 1/b) level by level
  int n2;
  const double *crc;
  double *rhs;         // nr x nz scratch
  double *hat;         // nr x nz scratch
  double *hhalf;       // nr x nz: H^{n+1/2}
  // FFT path (fft = nz = 2^a 3^b, nz even): the DCTs along z by an nz-point
  // complex FFT per pair of rows (natural mode order, half = 0)
  int fft;
  int nrad, rad[16];   // radices (4, 2, 3) of the mixed-radix Stockham passes
  const double2 *tw;   // tw[k] = exp(-2 pi i k / nz)
  const double2 *pw;   // pw[m] = (cos, sin)(pi m / (2 nz))
  double c0, c1;       // DCT-II normalisation sqrt(1/nz), sqrt(2/nz)
  // per-row tables (nr + 1 entries each): 1/(2 eps A_r), 1/(2 eps A_z),
  // 1/(eps A_r), 1/(eps A_z), 2 pi r_{i+1/2}, V_H, cell width w_i
  const double *rtab;
  // drive voltages V(t^n), V(t^{n+1}) read on the device (vd != nullptr) so
  // that a captured solve stays valid from step to step; else the arguments
  const double *vd;
  Circuit cc;
  // wave port on r = R: E_z^{n+1/2}(R) = 2 E_in^{n+1/2} - eta H^{n+1/2}(nr-1/2)
  int wave;
  double eta;
  // unit right-hand side (>= 0: the solve's rhs is the unit vector of this H
  // cell, for the set-up of the axial port's coupling; else -1)
  int unit_c;
  PortOp port;
};

// Radial scales of a cell in the push's normalised units: lengths in units of
// the cell's width w.  Cells ic < xa of the mapped mesh have their own width
// (tables in device memory: inner-face radius / w, dt / w, w / dt); beyond,
// w = dr, the inner-face radius is (ic + xa) dr and the scalars apply.
template <typename T>
struct RadialMapT {
  int xa;
  T cr, icr;
  const T *rho0x, *crx, *icrx;
  __device__ __forceinline__ T rho0(int ic) const { return ic < xa ? rho0x[ic] : (T)(ic + xa); }
  __device__ __forceinline__ T crr(int ic) const { return ic < xa ? crx[ic] : cr; }
  __device__ __forceinline__ T icrr(int ic) const { return ic < xa ? icrx[ic] : icr; }
};

// One mover + deposit pass over one species (rows a2, a3, a6) in the scalar
// type T of the particle store: double (plain form) or float (mixed form).
template <typename T>
struct PushLaunchT {
  Grid g;
  double q, m;             // species charge [C] and mass [kg]
  T qf;                    // q in T
  T cr, cz, icr, icz;      // dt/dr, dt/dz (velocity -> cells per step) and inverses
  RadialMapT<T> rm;        // per-cell radial scales (mapped mesh)
  T wbt;                   // qm*Bz*dt (0: no external B_z)
  float inz;               // 1/nz (cell -> (i, j) split without an integer division)
  long long n;
  const long long *n_dev;  // particle count on the device (graph-stable launches), or nullptr
  long long cap;           // store capacity (bounds the queue segments when n_dev is used)
  PartsT<T> p;
  const T *ar, *az;        // normalised accelerations qm*E*dt^2/dx of this species
  double *ir, *iz;         // crossed charge [C] (FP64, atomics)
  int write;               // write the new state (commit or speculative pass)
  int oop;                 // out of place: write every field into dst (in place: p)
  PartsT<T> dst;
  double *wall_z0, *wall_zl, *wall_r;
  unsigned long long *counters;
  double *ke_lost;
  unsigned long long *hist;  // accepted sub-steps per particle, 16 bins (nullptr: off)
  // work queue of the general path (queue == nullptr: all particles).  Block b
  // of the fast kernel appends the particles whose whole-step trial leaves the
  // cell through one z-face only to entries [b*qseg, b*qseg + qblock[b]) and the
  // rest from the back of its segment, qblock[qgrid + b] of them, so that the
  // general kernel's warps take those two kinds one after the other.
  int *queue, *qblock;
  long long qseg;
  int qgrid;               // blocks of the fast kernel
  int fgrid, ggrid;        // tuned grids of the fast / general kernels (0: one wave)
  T *q_da, *q_db;          // queued particle's converged whole-step trial (NaN: none);
                           // its start state is re-read from the store, which the
                           // fast kernel leaves untouched for queued particles
  // FP32 store: the queue entries carry the start state (nullptr: re-read
  // from the store, the FP64 form)
  int *q_cell;
  T *q_a, *q_b, *q_vr, *q_vt, *q_vz, *q_w;
  // FP32 store: crossers next to the axis are listed (plist[0 .. *pcnt)) by
  // the general kernel and pushed by a third kernel in FP64 arithmetic
  // (double scales, radial tables rm64); pcnt == nullptr: none
  int *plist;
  unsigned *pcnt;
  double dt;
  double icr64, icz64, cz64;  // dr/dt, dz/dt, dt/dz in double
  RadialMapT<double> rm64;
};
// radial cells next to the axis whose FP32 crossers may take FP64 arithmetic
// (the centrifugal term of Eq. 4 grows like 1/r and amplifies FP32 rounding)
constexpr int kPromoteRows = 2;
// Electrostatic field model (Eq. 8) on the same mesh: potential on the
// nodes, Gauss's law on the interior nodes (i < nr, 0 < j < nz), separable:
// orthonormal DST-I along z (GEMM), cyclic reduction along r (field.cu)
struct EsOp {
  int nr, nz, M, n2;       // M = nz - 1 interior nodes along z; n2 = 2^k >= nr
  double dr, dz;
  const double *S;         // M x M: sqrt(2/nz) sin(pi j m / nz), j, m = 1..M
  const double *crc;       // cyclic-reduction coefficients of mode m in column m - 1
  const double *tab;       // 4 x nr: eps A_r(i)/w_i, eps A_r(i-1)/w_{i-1}, eps A_z(i)/dz,
                           // w_i (cell widths)
  double *rhs, *hat, *phi; // nr x M scratch
  const double *vd;        // phi0 = vd[1] (V(t^{n+1})) if vd, else the argument
  // FFT path (fft2 = 2 nz = 2^a 3^b): the DST-I of two rows as one 2nz-point
  // complex FFT of their odd extensions; else the GEMM with S
  int fft2, nrad, rad[16];
  const double2 *tw2;      // exp(-2 pi i k / (2 nz))
  Circuit cc;
  const double *ez0;       // E_z^n (the plate flow of Eq. 6 with the circuit)
  // axial port (PIC_FEED_AXIAL; pip = 0: none): the powered electrode is the
  // disc of nodes i <= pip on z = 0, the port's opening carries phi0 g0[i]
  // (g0 = ln(r_i / R) / ln(r_pip / R), 1 on the disc), the side wall is grounded
  int pip;
  const double *g0;        // nr + 1
  const double *uphi;      // nr x M: the interior potential of a unit phi0 (no charge)
};
// E (Yee layouts) of the node charges Q (Q = Qn - div I if ir is given);
// Picard norms against er_it / ez_it into cnt when cnt is given
// Q -= div I on the interior nodes (the charge carried to the next step)
// Q <- eps div_h E - Q on the interior nodes (zero elsewhere); with the
// dielectric ring the charge stuck on its face (wall: the wall tallies) joins Q,
// and with a conducting ring the charge its conduction current moved (qc)
cudaError_t launch_gauss_residual(const Grid &g, double eps, const double *er, const double *ez,
                                  const double *wall, const double *qc, double *Q, cudaStream_t s);
// qc -= the charge the conducting ring's current moves over one step, dt S E^{n+1/2}
// per edge from its lower to its upper node (E^n in er0/ez0, E^{n+1} in er1/ez1)
cudaError_t launch_conduction(const Grid &g, double dt, const double *er0, const double *ez0,
                              const double *er1, const double *ez1, double *qc, cudaStream_t s);
// c[m] = sum_k basis[m n + k] f[k stride], m < nmodes (one block per mode)
cudaError_t launch_fourier_bessel(const double *basis, const double *f, int stride, int n,
                                  int nmodes, double *coef, cudaStream_t s);
// end of a converged step with the circuit: q^{n+1} = C (V^{n+1} - phi^{n+1}),
// phi^n <- phi^{n+1}
cudaError_t launch_circuit_commit(const Circuit &c, const double *vd, cudaStream_t s);
cudaError_t launch_es_advance(const EsOp &E, double *Q, const double *ir, const double *iz,
                              cudaStream_t s);
cudaError_t launch_es_solve(const EsOp &E, const double *Q, const double *ir, const double *iz,
                            double phi0, double *er1, double *ez1, const double *er_it,
                            const double *ez_it, DevCounters *cnt, cudaStream_t s);

// Picard start of a step (guess.cu)
struct FieldPair {
  const double *r, *z;  // E_r (nr x (nz+1)), E_z ((nr+1) x nz)
};
struct GuessArgs {
  int nr, nz;
  FieldPair e[4];       // E^n, E^{n-1}, E^{n-2}, E^{n-3}
  const double *h;      // H^n
  const double *jr, *jz;  // charge crossed in the last step
  double *sums;         // scratch: 4 sums of squares
  double *sd;           // s_d (device scalar)
  double *ger, *gez;    // G = 3E^n - 3E^{n-1} + E^{n-2}
  float *x;             // inputs [14][nr+1][nz+1]
};
cudaError_t launch_guess_inputs(const GuessArgs &A, cudaStream_t s);
cudaError_t launch_guess_apply(const GuessArgs &A, const float *y, int cp, double ez_edge,
                               double *er1, double *ez1, int *bad, cudaStream_t s);
cudaError_t launch_guess_target(const GuessArgs &A, const double *er_next, const double *ez_next,
                                float *tg, cudaStream_t s);

// most blocks of 256 threads resident on a GB300 (152 SMs x 8); the queue
// holds up to capacity + kMaxFastBlocks*256 entries
constexpr int kMaxFastBlocks = 152 * 8;
template <typename T>
cudaError_t launch_push(const PushLaunchT<T> &L, cudaStream_t s);
// the virtual grids launch_push would use for L (sets L.qgrid, L.qseg)
template <typename T>
void push_shape(PushLaunchT<T> &L, int *nfast, int *ngen);
// fast and general phases of nl discharges, one launch each (Ls, first in
// device memory: first[0..nl] fast item offsets, first[nl+1..2nl+1] general)
template <typename T>
cudaError_t launch_push_multi(const PushLaunchT<T> *Ls, const int *first, int nl, cudaStream_t s);
// FP32 store: the near-axis crossers launch_push listed, pushed in FP64
// arithmetic (a second launch after it; nothing with an external B_z)
cudaError_t launch_push_fp32_axis(const PushLaunchT<float> &L, cudaStream_t s);
// one resident wave of the persistent push kernels (blocks of 256 threads)
int push_wave_fp64(int general);
int push_wave_fp32(int general);

// launchers (return cudaError_t of the launch)
// the reactor's separable solve of the unit right-hand side of H cell c into
// F.hhalf (set-up of the axial port's coupling)
cudaError_t launch_unit_solve(const FieldOp &F, int c, cudaStream_t s);
cudaError_t launch_field_solve(const FieldOp &F, const double *er0, const double *ez0,
                               const double *h0, const double *ir, const double *iz, double v0,
                               double v1, double *er1, double *ez1, double *h1, const double *er_it,
                               const double *ez_it, DevCounters *cnt, cudaStream_t s);
cudaError_t launch_half_field(const Grid &g, const double *er0, const double *ez0,
                              const double *er1, const double *ez1, double *erh, double *ezh,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_load(const Grid &g, long long n, double n0, double te_ev, double ti_ev,
                        uint64_t seed, PartsT<T> e, PartsT<T> i, cudaStream_t s);

template <typename T>
struct MccLaunchT {
  uint64_t seed, step;
  double ng, tg, numax_e, pnull_e, pnull_i, gmax;
  uint64_t thr_e, thr_i;  // null-collision thresholds on the 53-bit integer draw
  long long ne, ni;
  PartsT<T> e, i;
  // null-collision candidates (slot, top bit set for ions) in per-block
  // segments [b*cseg, b*cseg + cblock[b]) of the select kernel's cgrid blocks
  uint32_t *cand;
  int *cblock;
  long long cseg;
  int cgrid;
  DevCounters *cnt;
  uint64_t *keys, *keys2; // scratch: (parent id << 32 | slot) of ionizing electrons
};
using MccLaunch = MccLaunchT<double>;
// selects the candidates, then collides them; the ionizing parents' keys go to
// keys[0 .. cnt->iz_slots)
template <typename T>
cudaError_t launch_mcc_collide(const MccLaunchT<T> &M, cudaStream_t s);
// orders the tot ionizing parents by id (keys), then appends the pairs in that order
template <typename T>
cudaError_t launch_mcc_append(const MccLaunchT<T> &M, long long tot, long long ne_new0,
                              long long ni_new0, uint32_t id_e0, uint32_t id_i0, cudaStream_t s);

// exclusive scan of n int32 values; total written to *total_dev (int64).
// The scan works in tiles of kScanTile elements and keeps one int64 sum per
// tile (plus one) in its scratch: scan_scratch_bytes(n) bytes
constexpr long long kScanTile = 4096;
size_t scan_scratch_bytes(long long n);
cudaError_t scan_exclusive(const int32_t *in, int32_t *out, long long n, long long *total_dev,
                           void *scratch, cudaStream_t s);

template <typename T>
struct SortLaunchT {
  int ncell;
  long long n;
  PartsT<T> src, dst;
  int32_t *counts;   // ncell + 1
  int32_t *offs;     // ncell + 1
  int32_t *cursor;   // ncell
  long long *total;
  void *scan_scratch;
};
using SortLaunch = SortLaunchT<double>;
template <typename T>
cudaError_t launch_sort(const SortLaunchT<T> &S, cudaStream_t s);

template <typename T>
cudaError_t launch_kinetic(const PartsT<T> &p, long long n, double m, double q, double *out2,
                           cudaStream_t s);
cudaError_t launch_field_energy(const Grid &g, double eps, double mu, const double *er,
                                const double *ez, const double *h, double *out, cudaStream_t s);
template <typename T>
cudaError_t launch_node_charge(const Grid &g, const PartsT<T> &p, long long n, double q,
                               double *Q, cudaStream_t s);

// FP64 form: the same normalised accelerations in FP64 (fast push path)
struct AlphaOut64 {
  double *ar[2], *az[2];
  double sr[2], sz[2];
  int xa, nz1;                        // mapped mesh: rows i < xa scale by their width
  double srx[2][kMaxAxisCells];       // qm*dt^2/w_i, i < xa
};
cudaError_t launch_half_field_alpha64(const Grid &g, const double *er0, const double *ez0,
                                      const double *er1, const double *ez1, double *erh,
                                      double *ezh, const AlphaOut64 &A, cudaStream_t s);

// Mixed form: normalised per-species accelerations alpha = qm*E*dt^2/dx (float)
struct AlphaOut {
  float *ar[2], *az[2];   // per species: Er-edge and Ez-edge layouts
  double sr[2], sz[2];    // scale factors qm*dt^2/dr, qm*dt^2/dz
  int xa, nz1;
  double srx[2][kMaxAxisCells];
};
cudaError_t launch_half_field_alpha(const Grid &g, const double *er0, const double *ez0,
                                    const double *er1, const double *ez1, double *erh,
                                    double *ezh, const AlphaOut &A, cudaStream_t s);




}  // namespace pic
