// C ABI of include/pic.h: context over a caller-owned device workspace, the
// field-operator set-up and the per-step driver (Picard loop of Sec. 2.1:
// push+deposit with E^{n+1/2,k}, implicit field solve, relative-change test;
// then commit push, MCC, sort).  No device allocation anywhere.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <cstdio>
#include <cmath>
#include <vector>

#include "../../include/pic_ensemble.h"
#include "../../include/pic_guess.h"
#include "pic_internal.cuh"

using namespace pic;

namespace pic {
int cnn_forward_async(pic_cnn *x, const float *xin, const float **y_posmajor, int *cp);
int cnn_grid(const pic_cnn *x, int *nr, int *nz);
cudaStream_t cnn_stream(const pic_cnn *x);
int cnn_layers(const pic_cnn *x);
const int *cnn_err_flag(const pic_cnn *x);
}  // namespace pic

struct pic_ctx {
  pic_config cfg;
  Grid g;
  cudaStream_t s;
  double eps, mu, ng;
  char *ws;
  size_t ws_bytes;
  long long cap[2], n[2];
  uint32_t next_id[2];
  long long step;
  Parts P[2][2];             // in the mixed form the real arrays hold float
  int cur[2];
  int mixed;                 // 1: FP32 particle store and push (PIC_MIXED)
  AlphaOut alpha;            // mixed form: normalised accelerations per species
  int *queue, *qblock;       // work queue of the general push path
  int *q_cell;               // mixed form: start state of the queued particles
  float *q_st[6];
  // mixed form: per species the list of near-axis crossers pushed in FP64
  // arithmetic, its count, and the side stream that runs the electrons' list
  // while the ions are pushed
  int *plist[2];
  unsigned *pcnt;
  cudaStream_t pstream;
  cudaEvent_t pev[2];
  int pstream_made;
  // the ions' push of a pass on a second stream beside the electrons' (the
  // persistent kernels fill the SMs the other species' tails leave idle),
  // with its own queue buffers
  cudaStream_t sstream;
  cudaEvent_t sev[2];
  int sstream_made;
  int *queue2, *qblock2;
  float *q_real2[2];
  double *q_real64_2[2];
  int *q_cell2;
  float *q_st2[6];
  // axial port (PIC_FEED_AXIAL): its fields at n and n+1 (the solve's output,
  // copied in when a step commits)
  double *hp, *erp, *ezp, *hp2, *erp2, *ezp2, *hup;
  // pic_step_host: copy streams (device -> host, host -> device) and their events
  cudaStream_t hs_dn, hs_up;
  cudaEvent_t hs_ev[130];
  int hs_made;
  float *q_real[2];          // mixed form queue records (trial displacements)
  double *q_real64[2];       // FP64 form queue records
  AlphaOut64 alpha64;        // FP64 form: normalised accelerations per species
  double *er, *ez, *h;      // E^n, H^n
  double *er1, *ez1;        // Picard iterate E^{n+1,k}
  double *er2, *ez2, *h2;   // solver output
  double *erh, *ezh;        // E^{n+1/2,k}
  double *ir, *iz;          // crossed charge of the pass
  double *wall;             // 2 species x (2(nr+1) + nz+1)
  double *wall_spec;        // wall tallies of a speculative final pass
  double rho_prev;          // last Picard contraction r_k / r_{k-1} observed
  FieldOp F;
  EsOp es;                  // electrostatic model (field_model == PIC_FIELD_ES)
  double *qn;               // node charge at the start of the step (ES model)
  int qn_valid;             // qn carried from the last step (else rebuilt from particles)
  DevCounters *cnt;
  uint32_t *cand;           // MCC: null-collision candidates (per-block segments)
  int *cblock;
  int32_t *counts, *coffs, *cursor;
  uint64_t *keys, *keys2;   // MCC: ionizing parents ordered by id
  long long *total;
  void *scan_scratch;
  double *diag;             // 8 doubles
  // per-step diagnostics (pic_diag_average): node counts of the step, their
  // sums, node charge after the previous step, continuity residual of the
  // last step, wall tallies at the window's start and after the previous step
  int diag_on, cres_valid;
  long long diag_steps;
  double *dcnt, *dacc, *qprev, *cres, *wall0, *wallp;
  double numax_e, gmax, pnull_e, pnull_i;
  long long launches;       // kernels enqueued by this context (host count)
  // optional timing of the push launches (CUDA events on the context stream)
  int prof;
  int nev;
  cudaEvent_t ev[2 * 128];
  double push_ms;
  long long push_launches, pending_launches;
  // Picard start (pic_guess.h): field history E^{n-1..n-3} (rotated pointers),
  // last crossed charge, extrapolation G, inputs / target of the learned guess
  int guess_mode;
  pic_cnn *cnn;
  int hist_n;               // field levels known, E^n included (at most 4)
  double *hr[3], *hz[3];
  double *jr, *jz;
  double *ger, *gez;
  double *gsums, *gsd;      // 4 sums, s_d
  int *gbad;
  float *gx, *gt;           // inputs of the current / last step and its target
  int sample_valid, feat_now;
  // graph-stable launches: particle counts and drive voltages on the device,
  // Picard passes captured once per buffer configuration and replayed
  long long *n_dev;
  double *vdev;             // [0..1] V^n, V^{n+1}; [4..7] blocking-capacitor state (Circuit)
  double *hu;               // EM unit response of the circuit (nr x nz)
  double *qc;               // charge moved by the conducting ring's current (nodes)
  unsigned long long *hist; // sub-step histogram (16 bins) of the state-writing passes
  unsigned long long *hist_spec;  // the same for a speculative final pass
  int hist_on;
  double *rmap64;           // mapped mesh: radial scales of the first cells (RadialMapT)
  float *rmap32;
  int circ_on;
  // generator waveform: sum of harmonics when nharm > 0 (else volt sin(2 pi f t))
  int nharm;
  double hamp[64], hfreq[64], hph[64];
  // Fourier-Bessel basis (App. A) for (fb_alpha, fb_m), 64 x (nr + 1) doubles
  double *fbb;
  int fb_alpha, fb_m;
  double *hn;               // pinned host read-back slots (kHn* below): Picard norms,
                            // sort totals, step counters
  int graphs;               // 1: passes replayed from captured graphs
  int capturing;            // a pass is being captured (no timing events)
  long long passes;         // passes enqueued (the first one is never captured)
  int fgrid[2], ggrid[2];   // tuned push grids (fast / general, per form: index 0)
  struct GraphEntry {
    const void *key[13];
    cudaGraphExec_t exec;
    long long nlaunch;      // kernels in the graph
    // push timing (pic_profile on at capture): events recorded around the
    // pushes by every replay, and the push launches between them
    cudaEvent_t pe[2];
    int ptimed, npush;
  } gcache[64];
  // the push events of the last replayed pass, read after it completed
  cudaEvent_t *rep_pe;
  int rep_npush;
  // the events a pass being captured records around its pushes (else null)
  cudaEvent_t *cap_pe;
  int cap_npush;
  int ngraph;
  cudaStream_t gstream;     // stream of the network
  cudaEvent_t gev[2];
  int gev_made, cnn_layers;
  // Picard iteration on the device (graphs on, timing off): one graph per
  // buffer configuration holding a conditional while-node whose body runs
  // the speculative or the plain pass (an if/else node), the convergence
  // test and the iterate copy; the host waits once, after the loop
  int dloop;                // 1: use it where it applies (the default)
  int dl_capture;           // a loop body is being captured (no host read-back)
  struct LoopEntry {
    const void *key[12];
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    long long nl_plain, nl_spec;  // kernels in one plain / speculative pass
  } lcache[32];
  int nloop;
};

namespace {

const double kSigmaCx = 5e-19;

// 8-byte slots of the pinned read-back buffer pic_ctx::hn: device values are
// copied there asynchronously and read after one wait per phase
enum {
  kHnNorm = 0,    // 3: Picard norms and drive energy of the last pass
  kHnTotal = 4,   // 2: particles kept by the sort, per species
  kHnPush = 8,    // 5: push counters of the commit pass
  kHnKel = 13,    // absorbed kinetic energy
  kHnCirc = 14,   // 4: circuit state
  kHnMcc = 18,    // 8: collision counts
  kHnDe = 26,     // collision energy change
  kHnIz = 27,     // ionization pairs of the MCC pass
  kHnLoop = 32,   // 13: the device Picard loop's state (kPd* below)
  kHnSlots = 48
};

// cyclic-reduction coefficients (the layout k_cr reads) of the tridiagonal
// matrix with sub-diagonal A[i] (coupling i-1), diagonal B, super-diagonal C,
// padded to n2 rows with identity; A, B, C are overwritten
void cr_coeffs(int n2, std::vector<double> &A, std::vector<double> &B, std::vector<double> &Cc,
               double *co) {
  int off = 0;
  for (int s = 1; s < n2; s *= 2) {
    const int cnt = n2 / (2 * s);
    for (int k = 0; k < cnt; ++k) {
      const int i = 2 * s * k + 2 * s - 1;
      const bool up = i + s < n2;
      const double al = -A[i] / B[i - s];
      const double ga = up ? -Cc[i] / B[i + s] : 0.0;
      co[off + k] = al;
      co[n2 + off + k] = ga;
      const double nb = B[i] + al * Cc[i - s] + (up ? ga * A[i + s] : 0.0);
      A[i] = al * A[i - s];
      Cc[i] = up ? ga * Cc[i + s] : 0.0;
      B[i] = nb;
    }
    off += cnt;
  }
  off = 0;
  for (int s = n2; s >= 1; s /= 2) {
    const int cnt = n2 >= 2 * s ? n2 / (2 * s) : 1;
    for (int k = 0; k < cnt; ++k) {
      const int j = 2 * s * k + s - 1;
      co[2 * n2 + off + k] = A[j] / B[j];
      co[3 * n2 + off + k] = Cc[j] / B[j];
      co[4 * n2 + off + k] = 1.0 / B[j];
    }
    off += cnt;
  }
}

double h_sig_el(double eps) {
  double x = eps / 12.0;
  return 1.5e-19 * x / (1.0 + x * x) + 1e-20;
}
double h_sig_ex(double eps) {
  if (!(eps > 11.5)) return 0.0;
  double u = eps / 11.5;
  return 4e-20 * log(u) / u;
}
double h_sig_iz(double eps) {
  if (!(eps > 15.76)) return 0.0;
  double u = eps / 15.76;
  return 8e-20 * log(u) / u;
}

struct Carver {
  char *base;
  size_t off, cap;
  bool ok;
  void *take(size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    void *p = base ? base + off : nullptr;
    off += bytes;
    if (off > cap) ok = false;
    return p;
  }
};

bool valid(const pic_config *c) {
  if (!c) return false;
  if (c->nr < 2 || c->nz < 2 || c->nr > 8192 || c->nz > 8192) return false;
  if (!(c->R > 0) || !(c->L > 0) || !(c->dt > 0)) return false;
  if (c->np_init < 0 || !(c->capacity_factor >= 1.0)) return false;
  if (!(c->picard_tol > 0) || c->picard_max < 1) return false;
  if (c->precision != PIC_FP64 && c->precision != PIC_MIXED) return false;
  if (c->field_model != PIC_FIELD_EM && c->field_model != PIC_FIELD_ES) return false;
  if (c->mcc_on && (!(c->gas_pressure > 0) || !(c->gas_temp > 0))) return false;
  if (!(c->cblock >= 0.0) || !isfinite(c->cblock)) return false;
  if (c->ions_fixed != 0 && c->ions_fixed != 1) return false;
  if (c->axis_cells < 0 || c->axis_cells > kMaxAxisCells || c->axis_cells >= c->nr) return false;
  if (c->feed != PIC_FEED_GAP && c->feed != PIC_FEED_WAVE && c->feed != PIC_FEED_AXIAL) return false;
  if (c->feed == PIC_FEED_AXIAL &&
      (c->ring_cells != 0 ||
       c->sigma_ring != 0.0 || c->port_cells < 1 || !(c->port_len > 0.0) ||
       !isfinite(c->port_len) || c->port_rin < 1 || c->port_rin >= c->nr ||
       !(c->eps_port >= 1.0) || !isfinite(c->eps_port) ||
       !(c->port_grade == 0.0 || (c->port_grade >= 0.25 && c->port_grade <= 4.0)) ||
       c->nr - c->port_rin > 4096 || (long long)(c->nr - c->port_rin) * c->port_cells > 8192))
    return false;
  if (c->ring_cells < 0 || (c->ring_cells > 0 && (!(c->eps_ring >= 1.0) || !isfinite(c->eps_ring) ||
                                                  c->ring_cells + c->axis_cells > c->nr - 2)))
    return false;
  if (c->feed == PIC_FEED_WAVE && (c->field_model != PIC_FIELD_EM || c->cblock > 0.0))
    return false;
  if (!(c->sigma_ring >= 0.0) || !isfinite(c->sigma_ring)) return false;
  if (c->sigma_ring > 0.0 && (c->ring_cells == 0 || c->field_model != PIC_FIELD_EM)) return false;
  if (c->ions_fixed && c->mcc_on) return false;
  return true;
}

long long capacity(const pic_config *c) {
  double v = ceil(c->capacity_factor * (double)c->np_init);
  long long k = (long long)v;
  return k < 1 ? 1 : k;
}

// lays out (or measures, when base == nullptr) the workspace
bool layout(pic_ctx *x, const pic_config *c, char *base, size_t cap, size_t *used) {
  Carver K{base, 0, cap, true};
  int nr = c->nr, nz = c->nz;
  long long pc = capacity(c);
  size_t rs = c->precision == PIC_MIXED ? 4 : 8;
  size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz, nh = (size_t)nr * nz;
  for (int s = 0; s < 2; ++s)
    for (int b = 0; b < 2; ++b) {
      Parts &P = x->P[s][b];
      P.cell = (int32_t *)K.take(pc * 4);
      P.a = (double *)K.take(pc * rs);
      P.b = (double *)K.take(pc * rs);
      P.vr = (double *)K.take(pc * rs);
      P.vt = (double *)K.take(pc * rs);
      P.vz = (double *)K.take(pc * rs);
      P.w = (double *)K.take(pc * rs);
      P.id = (uint32_t *)K.take(pc * 4);
    }
  const size_t qc = pc + (size_t)kMaxFastBlocks * 256;  // queue entries
  x->queue = (int *)K.take(qc * 4);
  x->qblock = (int *)K.take((size_t)2 * kMaxFastBlocks * 4);  // front and back counts
  x->queue2 = (int *)K.take(qc * 4);                           // the ions' (second stream)
  x->qblock2 = (int *)K.take((size_t)2 * kMaxFastBlocks * 4);
  if (c->precision == PIC_MIXED) {
    for (int s = 0; s < 2; ++s) {
      x->alpha.ar[s] = (float *)K.take(ner * 4);
      x->alpha.az[s] = (float *)K.take(nez * 4);
    }
    for (int k = 0; k < 2; ++k) x->q_real[k] = (float *)K.take(qc * 4);
    // queue entries carry the start state: cell, then a, b, vr, vt, vz, w
    x->q_cell = (int *)K.take(qc * 4);
    for (int k = 0; k < 6; ++k) x->q_st[k] = (float *)K.take(qc * 4);
    for (int k = 0; k < 2; ++k) x->q_real2[k] = (float *)K.take(qc * 4);
    x->q_cell2 = (int *)K.take(qc * 4);
    for (int k = 0; k < 6; ++k) x->q_st2[k] = (float *)K.take(qc * 4);
    // per species: near-axis crossers for FP64 arithmetic, and their counts
    x->plist[0] = (int *)K.take((size_t)pc * 4);
    x->plist[1] = (int *)K.take((size_t)pc * 4);
    x->pcnt = (unsigned *)K.take(256);
  } else {
    for (int s = 0; s < 2; ++s) {
      x->alpha64.ar[s] = (double *)K.take(ner * 8);
      x->alpha64.az[s] = (double *)K.take(nez * 8);
    }
    for (int k = 0; k < 2; ++k) x->q_real64[k] = (double *)K.take(qc * 8);
    for (int k = 0; k < 2; ++k) x->q_real64_2[k] = (double *)K.take(qc * 8);
  }
  x->er = (double *)K.take(ner * 8);
  x->ez = (double *)K.take(nez * 8);
  x->h = (double *)K.take(nh * 8);
  x->er1 = (double *)K.take(ner * 8);
  x->ez1 = (double *)K.take(nez * 8);
  x->er2 = (double *)K.take(ner * 8);
  x->ez2 = (double *)K.take(nez * 8);
  x->h2 = (double *)K.take(nh * 8);
  x->erh = (double *)K.take(ner * 8);
  x->ezh = (double *)K.take(nez * 8);
  x->ir = (double *)K.take(ner * 8);
  x->iz = (double *)K.take(nez * 8);
  x->wall = (double *)K.take((size_t)2 * (2 * (nr + 1) + nz + 1) * 8);
  x->wall_spec = (double *)K.take((size_t)2 * (2 * (nr + 1) + nz + 1) * 8);
  x->qc = (double *)K.take((size_t)(nr + 1) * (nz + 1) * 8);
  x->hist = (unsigned long long *)K.take(16 * 8);
  x->hist_spec = (unsigned long long *)K.take(16 * 8);
  x->F.Q = (double *)K.take((size_t)nz * nz * 8);
  x->F.QT = (double *)K.take((size_t)nz * nz * 8);
  int n2 = 1;
  while (n2 < nr) n2 *= 2;
  x->F.n2 = n2;
  x->F.crc = (const double *)K.take((size_t)5 * n2 * nz * 8);
  x->F.rhs = (double *)K.take(nh * 8);
  x->F.hat = (double *)K.take(nh * 8);
  x->F.hhalf = (double *)K.take(nh * 8);
  if (c->feed == PIC_FEED_AXIAL && c->field_model == PIC_FIELD_EM) {
    PortOp &P = x->F.port;
    const int m = nr - c->port_rin, nzp = c->port_cells, np = m * nzp, nzz = (m + 1) * nzp;
    P.Binv = (const double *)K.take((size_t)np * np * 8);
    P.ZR = (const double *)K.take((size_t)m * nh * 8);
    P.ZP = (const double *)K.take((size_t)m * np * 8);
    P.Cinv = (const double *)K.take((size_t)m * m * 8);
    P.rhsp = (double *)K.take((size_t)np * 8);
    P.hhp = (double *)K.take((size_t)np * 8);
    P.ws = (double *)K.take((size_t)m * 8);
    P.hq = (const double *)K.take((size_t)nzp * 8);
    x->hp = (double *)K.take((size_t)np * 8);
    x->erp = (double *)K.take((size_t)np * 8);
    x->ezp = (double *)K.take((size_t)nzz * 8);
    x->hp2 = (double *)K.take((size_t)np * 8);
    x->erp2 = (double *)K.take((size_t)np * 8);
    x->ezp2 = (double *)K.take((size_t)nzz * 8);
    x->hup = (double *)K.take((size_t)np * 8);
  }
  {
    const int M = nz - 1, n2e = x->F.n2;
    x->es.nr = nr;
    x->es.nz = nz;
    x->es.M = M;
    x->es.n2 = n2e;
    x->es.dr = c->R / (nr + c->axis_cells);
    x->es.dz = c->L / nz;
    x->es.S = (const double *)K.take((size_t)M * M * 8);
    x->es.crc = (const double *)K.take((size_t)5 * n2e * M * 8);
    x->es.tab = (const double *)K.take((size_t)4 * nr * 8);
    x->es.rhs = (double *)K.take((size_t)nr * M * 8);
    x->es.hat = (double *)K.take((size_t)nr * M * 8);
    x->es.phi = (double *)K.take((size_t)nr * M * 8);
    x->qn = (double *)K.take((size_t)(nr + 1) * (nz + 1) * 8);
    x->es.tw2 = (const double2 *)K.take((size_t)2 * nz * 16);
    if (c->feed == PIC_FEED_AXIAL && c->field_model == PIC_FIELD_ES) {
      x->es.g0 = (const double *)K.take((size_t)(nr + 1) * 8);
      x->es.uphi = (const double *)K.take((size_t)nr * M * 8);
    }
  }
  x->F.tw = (const double2 *)K.take((size_t)nz * 16);
  x->F.pw = (const double2 *)K.take((size_t)nz * 16);
  x->F.rtab = (const double *)K.take((size_t)9 * (nr + 1) * 8);
  x->cnt = (DevCounters *)K.take(sizeof(DevCounters));
  for (int k = 0; k < 3; ++k) {
    x->hr[k] = (double *)K.take(ner * 8);
    x->hz[k] = (double *)K.take(nez * 8);
  }
  x->jr = (double *)K.take(ner * 8);
  x->jz = (double *)K.take(nez * 8);
  x->ger = (double *)K.take(ner * 8);
  x->gez = (double *)K.take(nez * 8);
  x->gsums = (double *)K.take(8 * 8);
  x->gsd = x->gsums + 4;
  x->gbad = (int *)K.take(256);
  x->n_dev = (long long *)K.take(256);
  x->vdev = (double *)K.take(256);
  x->hu = (double *)K.take((size_t)nr * nz * 8);
  x->rmap64 = (double *)K.take((size_t)3 * kMaxAxisCells * 8);
  x->rmap32 = (float *)K.take((size_t)3 * kMaxAxisCells * 4);
  x->fbb = (double *)K.take((size_t)64 * (nr + 1) * 8);
  {
    size_t P = (size_t)(nr + 1) * (nz + 1);
    x->gx = (float *)K.take(P * PIC_CNN_IN * 4);
    x->gt = (float *)K.take(P * PIC_CNN_OUT * 4);
  }
  x->cand = (uint32_t *)K.take((2 * (size_t)pc + 2 * (size_t)kMaxFastBlocks * 256) * 4);
  x->cblock = (int *)K.take((size_t)kMaxFastBlocks * 4);
  x->keys = (uint64_t *)K.take(pc * 8);
  x->keys2 = (uint64_t *)K.take(pc * 8);
  int ncell = nr * nz;
  x->counts = (int32_t *)K.take((size_t)(ncell + 1) * 4);
  x->coffs = (int32_t *)K.take((size_t)(ncell + 1) * 4);
  x->cursor = (int32_t *)K.take((size_t)ncell * 4);
  x->total = (long long *)K.take(16);  // one slot per species
  long long sn = pc > ncell + 1 ? pc : ncell + 1;
  x->scan_scratch = K.take(scan_scratch_bytes(sn));
  x->diag = (double *)K.take(8 * 8);
  {
    const size_t nn = (size_t)(nr + 1) * (nz + 1), nwall = (size_t)2 * (2 * (nr + 1) + nz + 1);
    x->dcnt = (double *)K.take(2 * nn * 8);
    x->dacc = (double *)K.take(2 * nn * 8);
    x->qprev = (double *)K.take(nn * 8);
    x->cres = (double *)K.take(nn * 8);
    x->wall0 = (double *)K.take(nwall * 8);
    x->wallp = (double *)K.take(nwall * 8);
  }
  K.take(0);
  *used = K.off;
  return K.ok;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? PIC_OK : PIC_E_CUDA; }

Parts &cur(pic_ctx *x, int s) { return x->P[s][x->cur[s]]; }

// the same arrays seen with the element type of the mixed form
Parts32 as32(const Parts &p) {
  return Parts32{p.cell, (float *)p.a, (float *)p.b, (float *)p.vr, (float *)p.vt,
                 (float *)p.vz, (float *)p.w, p.id};
}

double volt_at(const pic_ctx *x, long long step) {
  double t = (double)step * x->cfg.dt;
  if (x->nharm > 0) {
    double v = 0.0;
    for (int k = 0; k < x->nharm; ++k) v += x->hamp[k] * sin(kTwoPi * x->hfreq[k] * t + x->hph[k]);
    return v;
  }
  return x->cfg.volt * sin(kTwoPi * x->cfg.freq * t);
}

// circuit state {q, 0, phi, 0} with q = 0 and the electrode at V(t^n)
cudaError_t circuit_reset(pic_ctx *x) {
  // pageable source: the call returns once it is staged
  const double st[4] = {0.0, 0.0, volt_at(x, x->step), 0.0};
  return cudaMemcpyAsync(x->vdev + 4, st, sizeof(st), cudaMemcpyHostToDevice, x->s);
}

__global__ void k_fill(double *p, int n, double v) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) p[t] = v;
}

// fold finished event pairs into the push timing totals (stream must be idle)
void prof_collect(pic_ctx *x) {
  for (int k = 0; k < x->nev; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, x->ev[2 * k], x->ev[2 * k + 1]) == cudaSuccess) x->push_ms += ms;
    else cudaGetLastError();  // a failed query must not surface as a later launch's error
  }
  x->nev = 0;
  x->push_launches += x->pending_launches;
  x->pending_launches = 0;
  if (x->rep_pe) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, x->rep_pe[0], x->rep_pe[1]) == cudaSuccess) {
      x->push_ms += ms;
      x->push_launches += x->rep_npush;
    } else {
      cudaGetLastError();
    }
    x->rep_pe = nullptr;
  }
}

template <typename T>
void fill_push(pic_ctx *x, int s, double q, double m, const double *erh, const double *ezh,
               double *ir, double *iz, int write, unsigned long long *counters, double *kel,
               double *const ws[3], PushLaunchT<T> &L) {
  (void)erh;
  (void)ezh;
  const double dt = x->cfg.dt;
  L.g = x->g;
  L.g.nr = x->g.nr - x->g.nd;  // particles move inside the dielectric ring
  L.q = q;
  L.m = m;
  L.qf = (T)q;
  L.cr = (T)(dt / x->g.dr);
  L.cz = (T)(dt / x->g.dz);
  L.icr = (T)(x->g.dr / dt);
  L.icz = (T)(x->g.dz / dt);
  L.rm.xa = x->g.xa;
  L.rm.cr = L.cr;
  L.rm.icr = L.icr;
  const T *tb = (const T *)(sizeof(T) == 8 ? (const void *)x->rmap64 : (const void *)x->rmap32);
  L.rm.rho0x = tb;
  L.rm.crx = tb + kMaxAxisCells;
  L.rm.icrx = tb + 2 * kMaxAxisCells;
  L.wbt = (T)(q / m * x->cfg.bz * dt);
  L.inz = 1.0f / (float)x->g.nz;
  L.n = x->n[s];
  L.n_dev = x->n_dev + s;
  L.cap = x->cap[s];
  L.fgrid = x->fgrid[0];
  L.ggrid = x->ggrid[0];
  L.ir = ir;
  L.iz = iz;
  L.write = write;
  L.wall_z0 = ws[0];
  L.wall_zl = ws[1];
  L.wall_r = ws[2];
  L.counters = counters;
  L.ke_lost = kel;
  L.hist = (write && x->hist_on) ? x->hist : nullptr;
  L.dt = dt;
  L.icr64 = x->g.dr / dt;
  L.icz64 = x->g.dz / dt;
  L.cz64 = dt / x->g.dz;
  L.rm64.xa = x->g.xa;
  L.rm64.cr = dt / x->g.dr;
  L.rm64.icr = x->g.dr / dt;
  L.rm64.rho0x = x->rmap64;
  L.rm64.crx = x->rmap64 + kMaxAxisCells;
  L.rm64.icrx = x->rmap64 + 2 * kMaxAxisCells;
  L.pcnt = nullptr;
  L.plist = nullptr;
  L.q_cell = nullptr;
  L.q_a = L.q_b = L.q_vr = L.q_vt = L.q_vz = L.q_w = nullptr;
}

template <typename T>
void set_queue(pic_ctx *x, T *const rec[2], PushLaunchT<T> &L) {
  L.queue = x->queue;
  L.qblock = x->qblock;
  L.q_da = rec[0];
  L.q_db = rec[1];
}

// oop: write the new state into the second buffer of the store (speculative
// final pass), every field; else (write) in place
int push_all(pic_ctx *x, const double *erh, const double *ezh, double *ir, double *iz, int write,
             unsigned long long *counters, double *kel, double *wall, int oop = 0) {
  bool timed = x->prof && x->nev < 128 && !x->capturing;
  if (timed) cudaEventRecord(x->ev[2 * x->nev], x->s);
  // a pass being captured with timing on records its own event pair, which
  // every replay records again
  const bool ctimed = x->capturing && x->cap_pe;
  // external records become event-record nodes that every replay executes
  if (ctimed) cudaEventRecordWithFlags(x->cap_pe[0], x->s, cudaEventRecordExternal);
  const int nsp = x->cfg.ions_fixed ? 1 : 2;
  bool forked = false;
  // the ions on the second stream, forked after the pass's set-up and joined
  // before the field solve
  const bool split = nsp == 2 && x->sstream_made;
  if (split) {
    if (cudaEventRecord(x->sev[0], x->s) != cudaSuccess ||
        cudaStreamWaitEvent(x->sstream, x->sev[0], 0) != cudaSuccess)
      return PIC_E_CUDA;
  }
  for (int s = 0; s < nsp; ++s) {
    const double q = s == 0 ? -kQE : kQE, m = s == 0 ? kME : kMAr;
    const bool two = split && s == 1;
    cudaStream_t ss = two ? x->sstream : x->s;
    double *ws[3] = {nullptr, nullptr, nullptr};
    if (wall) {
      int nr = x->g.nr, nz = x->g.nz;
      double *w0 = wall + (size_t)s * (2 * (nr + 1) + nz + 1);
      ws[0] = w0;
      ws[1] = w0 + (nr + 1);
      ws[2] = w0 + 2 * (nr + 1);
    }
    cudaError_t e;
    long long n = x->n[s];
    bool fast;
    if (x->mixed) {
      PushLaunchT<float> L;
      fill_push(x, s, q, m, erh, ezh, ir, iz, write, counters, kel, ws, L);
      L.p = as32(cur(x, s));
      L.dst = oop ? as32(x->P[s][x->cur[s] ^ 1]) : L.p;
      L.oop = oop;
      if (L.hist && oop) L.hist = x->hist_spec;  // counted once the pass is adopted
      L.ar = x->alpha.ar[s];
      L.az = x->alpha.az[s];
      set_queue(x, two ? x->q_real2 : x->q_real, L);
      if (two) {
        L.queue = x->queue2;
        L.qblock = x->qblock2;
      }
      float *const *qs = two ? x->q_st2 : x->q_st;
      L.q_cell = two ? x->q_cell2 : x->q_cell;
      L.q_a = qs[0];
      L.q_b = qs[1];
      L.q_vr = qs[2];
      L.q_vt = qs[3];
      L.q_vz = qs[4];
      L.q_w = qs[5];
      L.plist = x->plist[s];
      L.pcnt = x->pcnt + s;
      fast = L.wbt == 0.f;
      e = launch_push(L, ss);
      if (e == cudaSuccess && two) {
        e = launch_push_fp32_axis(L, ss);  // the ions' near-axis list after their push
      } else if (e == cudaSuccess) {
        if (x->pstream_made) {
          // the near-axis lists on the side stream, beside the next launches
          // (the electrons' beside the ions' pass), joined at the end
          e = cudaEventRecord(x->pev[0], x->s);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(x->pstream, x->pev[0], 0);
          if (e == cudaSuccess) e = launch_push_fp32_axis(L, x->pstream);
          if (e == cudaSuccess) e = cudaEventRecord(x->pev[1], x->pstream);
          forked = forked || e == cudaSuccess;
        } else {
          e = launch_push_fp32_axis(L, x->s);
        }
      }
    } else {
      PushLaunchT<double> L;
      fill_push(x, s, q, m, erh, ezh, ir, iz, write, counters, kel, ws, L);
      L.p = cur(x, s);
      L.dst = oop ? x->P[s][x->cur[s] ^ 1] : L.p;
      L.oop = oop;
      if (L.hist && oop) L.hist = x->hist_spec;  // counted once the pass is adopted
      L.ar = x->alpha64.ar[s];
      L.az = x->alpha64.az[s];
      set_queue(x, two ? x->q_real64_2 : x->q_real64, L);
      if (two) {
        L.queue = x->queue2;
        L.qblock = x->qblock2;
      }
      fast = L.wbt == 0.0;
      e = launch_push(L, ss);
    }
    if (e != cudaSuccess) return PIC_E_CUDA;
    if (n > 0) {
      x->launches += fast ? 2 : 1;  // fast + general kernels
      if (timed) x->pending_launches += 1;
      if (ctimed) x->cap_npush += 1;
    }
  }
  if (forked && cudaStreamWaitEvent(x->s, x->pev[1], 0) != cudaSuccess) return PIC_E_CUDA;
  if (split && (cudaEventRecord(x->sev[1], x->sstream) != cudaSuccess ||
                cudaStreamWaitEvent(x->s, x->sev[1], 0) != cudaSuccess))
    return PIC_E_CUDA;
  if (ctimed) cudaEventRecordWithFlags(x->cap_pe[1], x->s, cudaEventRecordExternal);
  if (timed) {
    cudaEventRecord(x->ev[2 * x->nev + 1], x->s);
    x->nev += 1;
  }
  return PIC_OK;
}

// One species' push parameters of a pass, as push_all sets them, for a
// launch over several discharges (an ensemble round).  spec: the speculative
// (writing, out of place) pass.
void round_launch(pic_ctx *x, int s, bool spec, PushLaunchT<float> &L) {
  const double q = s == 0 ? -kQE : kQE, m = s == 0 ? kME : kMAr;
  double *ws[3] = {nullptr, nullptr, nullptr};
  if (spec) {
    const int nr = x->g.nr, nz = x->g.nz;
    double *w0 = x->wall_spec + (size_t)s * (2 * (nr + 1) + nz + 1);
    ws[0] = w0;
    ws[1] = w0 + (nr + 1);
    ws[2] = w0 + 2 * (nr + 1);
  }
  fill_push(x, s, q, m, x->erh, x->ezh, x->ir, x->iz, spec ? 1 : 0,
            spec ? x->cnt->push : nullptr, spec ? &x->cnt->ke_lost : nullptr, ws, L);
  L.p = as32(cur(x, s));
  L.dst = spec ? as32(x->P[s][x->cur[s] ^ 1]) : L.p;
  L.oop = spec ? 1 : 0;
  if (L.hist && spec) L.hist = x->hist_spec;
  L.ar = x->alpha.ar[s];
  L.az = x->alpha.az[s];
  set_queue(x, x->q_real, L);
  L.q_cell = x->q_cell;
  L.q_a = x->q_st[0];
  L.q_b = x->q_st[1];
  L.q_vr = x->q_st[2];
  L.q_vt = x->q_st[3];
  L.q_vz = x->q_st[4];
  L.q_w = x->q_st[5];
  L.plist = x->plist[s];
  L.pcnt = x->pcnt + s;
}

void round_launch(pic_ctx *x, int s, bool spec, PushLaunchT<double> &L) {
  const double q = s == 0 ? -kQE : kQE, m = s == 0 ? kME : kMAr;
  double *ws[3] = {nullptr, nullptr, nullptr};
  if (spec) {
    const int nr = x->g.nr, nz = x->g.nz;
    double *w0 = x->wall_spec + (size_t)s * (2 * (nr + 1) + nz + 1);
    ws[0] = w0;
    ws[1] = w0 + (nr + 1);
    ws[2] = w0 + 2 * (nr + 1);
  }
  fill_push(x, s, q, m, x->erh, x->ezh, x->ir, x->iz, spec ? 1 : 0,
            spec ? x->cnt->push : nullptr, spec ? &x->cnt->ke_lost : nullptr, ws, L);
  L.p = cur(x, s);
  L.dst = spec ? x->P[s][x->cur[s] ^ 1] : L.p;
  L.oop = spec ? 1 : 0;
  if (L.hist && spec) L.hist = x->hist_spec;
  L.ar = x->alpha64.ar[s];
  L.az = x->alpha64.az[s];
  set_queue(x, x->q_real64, L);
}

// Per-step diagnostics of one node t (pic_diag_average): adds the node counts
// of the step (cnt: electrons, then ions; sums of w S1 x S1) to the averages,
// and forms the node's charge balance over the step: the change of the
// particles' node charge and of the wall tallies on the node, plus the net
// crossed charge leaving its dual cell (Eq. 3).  init: only the node charge.
__global__ void k_diag_step(int nr, int nz, int i0, const double *cnt, double *acc,
                            const double *ir, const double *iz, const double *wall,
                            const double *wallp, double *qprev, double *cres, int init) {
  const int nz1 = nz + 1;
  const long long nn = (long long)(nr + 1) * nz1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nn) return;
  const int i = (int)(t / nz1), j = (int)(t - (t / nz1) * nz1);
  const double ce = cnt[t], ci = cnt[nn + t];
  const double Q = kQE * ci - kQE * ce;
  if (!init) {
    acc[t] += ce;
    acc[nn + t] += ci;
    const long long blk = 2LL * (nr + 1) + nz1;
    double dW = 0.0;
    for (int sp = 0; sp < 2; ++sp) {
      const long long b = sp * blk;
      if (j == 0) dW += wall[b + i] - wallp[b + i];
      if (j == nz) dW += wall[b + nr + 1 + i] - wallp[b + nr + 1 + i];
      if (i == i0) dW += wall[b + 2 * (nr + 1) + j] - wallp[b + 2 * (nr + 1) + j];
    }
    double div = 0.0;
    if (i < nr) div += ir[(long long)i * nz1 + j];
    if (i > 0) div -= ir[(long long)(i - 1) * nz1 + j];
    if (j < nz) div += iz[(long long)i * nz + j];
    if (j > 0) div -= iz[(long long)i * nz + j - 1];
    cres[t] = (Q - qprev[t]) + dW + div;
  }
  qprev[t] = Q;
}

// node counts (sums of w S1 x S1) of both species into dcnt, then the step's
// diagnostics (init: only the node charge, at the start of a window)
int diag_step(pic_ctx *x, int init) {
  const int nr = x->g.nr, nz = x->g.nz;
  const size_t nn = (size_t)(nr + 1) * (nz + 1), nwall = (size_t)2 * (2 * (nr + 1) + nz + 1);
  cudaStream_t s = x->s;
  if (cudaMemsetAsync(x->dcnt, 0, 2 * nn * 8, s) != cudaSuccess) return PIC_E_CUDA;
  for (int sp = 0; sp < 2; ++sp) {
    cudaError_t e = x->mixed ? launch_node_charge(x->g, as32(cur(x, sp)), x->n[sp], 1.0,
                                                  x->dcnt + sp * nn, s)
                             : launch_node_charge(x->g, cur(x, sp), x->n[sp], 1.0,
                                                  x->dcnt + sp * nn, s);
    if (e != cudaSuccess) return PIC_E_CUDA;
  }
  k_diag_step<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(nr, nz, nr - x->g.nd, x->dcnt, x->dacc,
                                                           x->ir, x->iz, x->wall, x->wallp,
                                                           x->qprev, x->cres, init);
  if (cudaGetLastError() != cudaSuccess) return PIC_E_CUDA;
  if (cudaMemcpyAsync(x->wallp, x->wall, nwall * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PIC_E_CUDA;
  x->launches += 4;
  if (!init) {
    x->diag_steps += 1;
    x->cres_valid = 1;
  }
  return PIC_OK;
}

}  // namespace

extern "C" {

const char *pic_strerror(int code) {
  switch (code) {
    case PIC_OK: return "ok";
    case PIC_E_CONFIG: return "invalid configuration or argument";
    case PIC_E_CUDA: return "CUDA error";
    case PIC_E_NOCONV: return "Picard iteration did not converge";
    case PIC_E_SUBSTEP: return "particle exceeded the sub-step limit";
    case PIC_E_CAPACITY: return "particle capacity exceeded";
    case PIC_E_NAN: return "non-finite field or residual";
    case PIC_E_STATE: return "inconsistent state";
    case PIC_E_WORKSPACE: return "workspace missing, too small or misaligned";
    case PIC_E_IO: return "checkpoint file could not be written or read";
    default: return "unknown status";
  }
}

const char *pic_version(void) { return "pic-gb300 fp64 sm_103a 1"; }

int pic_workspace_size(const pic_config *cfg, size_t *bytes) {
  if (!valid(cfg) || !bytes) return PIC_E_CONFIG;
  pic_ctx tmp;
  memset(&tmp, 0, sizeof(tmp));
  size_t used = 0;
  layout(&tmp, cfg, nullptr, (size_t)-1, &used);
  *bytes = used + 256;
  return PIC_OK;
}

namespace {
// Axial port set-up (PIC_FEED_AXIAL; FieldOp's PortOp): the port block's
// inverse (banded Cholesky, one solve per column), the reactor part of
// B^{-1} U (one separable solve per interface edge), the port part, and the
// interface (capacitance) matrix W^{-1} + U^T Z, inverted.  Synchronises.
int port_setup(pic_ctx *x, const pic_config *cfg) {
  FieldOp &F = x->F;
  PortOp &P = F.port;
  const Grid &G = x->g;
  const int nr = G.nr, nz = G.nz, ip = cfg->port_rin, nzp = cfg->port_cells, m = nr - ip;
  const int np = m * nzp;
  const size_t nh = (size_t)nr * nz;
  P.on = 1;
  P.ip = ip;
  P.nzp = nzp;
  P.m = m;
  P.np = np;
  // row heights: a geometric progression of ratio port_grade from the
  // junction down (0 or 1: uniform), summing to port_len
  std::vector<double> hq(nzp);
  {
    const double gr = cfg->port_grade == 0.0 ? 1.0 : cfg->port_grade;
    if (gr == 1.0) {
      for (int q = 0; q < nzp; ++q) hq[q] = cfg->port_len / nzp;
    } else {
      const double top = cfg->port_len * (gr - 1.0) / (pow(gr, (double)nzp) - 1.0);
      for (int q = 0; q < nzp; ++q) hq[q] = top * pow(gr, (double)(nzp - 1 - q));
    }
  }
  P.htop = hq[nzp - 1];
  P.erq = cfg->eps_port;
  P.eta = sqrt(x->mu / (cfg->eps_port * x->eps));
  P.lnr = log(g_rnode(G, nr) / g_rnode(G, ip));
  P.hp0 = x->hp;
  P.erp0 = x->erp;
  P.ezp0 = x->ezp;
  P.hp1 = x->hp2;
  P.erp1 = x->erp2;
  P.ezp1 = x->ezp2;
  const double dt = cfg->dt, hdt2 = 0.5 * dt * dt, eps = x->eps, mu = x->mu;
  const double erq = P.erq;
  // the port block (mass, the E_r edges between its rows, its interior E_z
  // edges, Mur's term at the end), lower band of width nzp
  const int bw = nzp;
  std::vector<double> Lb((size_t)np * (bw + 1), 0.0);
  auto band = [&](int a, int b) -> double & { return Lb[(size_t)a * (bw + 1) + (b - a + bw)]; };
  for (int k = 0; k < m; ++k) {
    const int i = ip + k;
    const double sv = kTwoPi * g_rcentre(G, i), L = g_width(G, i);
    for (int q = 0; q < nzp; ++q) band(k * nzp + q, k * nzp + q) += 2.0 * mu * sv * L * hq[q];
    for (int q = 1; q < nzp; ++q) {
      const double w = hdt2 * (L / (eps * erq * sv * (0.5 * (hq[q - 1] + hq[q])))) * sv * sv;
      const int lo = k * nzp + q - 1, hi = k * nzp + q;
      band(lo, lo) += w;
      band(hi, hi) += w;
      band(hi, lo) -= w;
    }
    band(k * nzp, k * nzp) += dt * sv * L * P.eta;
  }
  for (int k = 1; k < m; ++k) {
    const int i = ip + k;
    const double sr = kTwoPi * g_rcentre(G, i), sl = kTwoPi * g_rcentre(G, i - 1);
    for (int q = 0; q < nzp; ++q) {
      const double W = hq[q] / (eps * erq * g_area_z(G, i));
      const int cr = k * nzp + q, cl = (k - 1) * nzp + q;
      band(cr, cr) += hdt2 * W * sr * sr;
      band(cl, cl) += hdt2 * W * sl * sl;
      band(cr, cl) -= hdt2 * W * sl * sr;
    }
  }
  for (int a = 0; a < np; ++a) {
    const int j0 = a - bw < 0 ? 0 : a - bw;
    for (int b = j0; b <= a; ++b) {
      double sum = band(a, b);
      const int k0 = j0 > b - bw ? j0 : b - bw;
      for (int k = k0; k < b; ++k) sum -= band(a, k) * band(b, k);
      if (a == b) {
        if (!(sum > 0.0)) return PIC_E_CONFIG;
        band(a, a) = sqrt(sum);
      } else {
        band(a, b) = sum / band(b, b);
      }
    }
  }
  std::vector<double> Binv((size_t)np * np), col(np);
  for (int c = 0; c < np; ++c) {
    std::fill(col.begin(), col.end(), 0.0);
    col[c] = 1.0;
    for (int a = 0; a < np; ++a) {
      double sum = col[a];
      for (int k = a - bw < 0 ? 0 : a - bw; k < a; ++k) sum -= band(a, k) * col[k];
      col[a] = sum / band(a, a);
    }
    for (int a = np - 1; a >= 0; --a) {
      double sum = col[a];
      const int k1 = a + bw > np - 1 ? np - 1 : a + bw;
      for (int k = a + 1; k <= k1; ++k) sum -= band(k, a) * col[k];
      col[a] = sum / band(a, a);
    }
    for (int a = 0; a < np; ++a) Binv[(size_t)a * np + c] = col[a];
  }
  // reactor part of Z: B_R^{-1} e(ip + e, 0), one separable solve each
  cudaError_t ce = cudaSuccess;
  for (int e = 0; e < m && ce == cudaSuccess; ++e) {
    ce = launch_unit_solve(F, (ip + e) * nz, x->s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync((void *)(P.ZR + (size_t)e * nh), F.hhalf, nh * 8,
                           cudaMemcpyDeviceToDevice, x->s);
  }
  std::vector<double> zr((size_t)m * nh);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(zr.data(), P.ZR, zr.size() * 8, cudaMemcpyDeviceToHost, x->s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(x->s);
  if (ce != cudaSuccess) return PIC_E_CUDA;
  // H(i, 0) of a solve in the layout of FieldOp::hhalf
  auto h0of = [&](const double *a, int i) {
    if (!F.half) return a[(size_t)i * nz];
    const int h = F.half;
    return a[(size_t)i * h] + a[(size_t)nr * h + (size_t)i * h];
  };
  std::vector<double> zp((size_t)m * np), cap((size_t)m * m);
  for (int f = 0; f < m; ++f)
    for (int p = 0; p < np; ++p) zp[(size_t)f * np + p] = -Binv[(size_t)p * np + f * nzp + nzp - 1];
  for (int e = 0; e < m; ++e) {
    const int i = ip + e;
    const double sv = kTwoPi * g_rcentre(G, i), L = g_width(G, i);
    const double dint = eps * sv * 0.5 * (erq * P.htop + G.dz);
    const double w = hdt2 * (L / dint) * sv * sv;
    for (int f = 0; f < m; ++f)
      cap[(size_t)e * m + f] = (e == f ? 1.0 / w : 0.0) + h0of(zr.data() + (size_t)f * nh, i) +
                               Binv[(size_t)(e * nzp + nzp - 1) * np + f * nzp + nzp - 1];
  }
  // symmetric positive definite: Cholesky, then the inverse column by column
  for (int a = 0; a < m; ++a)
    for (int b = 0; b <= a; ++b) {
      double sum = cap[(size_t)a * m + b];
      for (int k = 0; k < b; ++k) sum -= cap[(size_t)a * m + k] * cap[(size_t)b * m + k];
      if (a == b) {
        if (!(sum > 0.0)) return PIC_E_CONFIG;
        cap[(size_t)a * m + a] = sqrt(sum);
      } else {
        cap[(size_t)a * m + b] = sum / cap[(size_t)b * m + b];
      }
    }
  std::vector<double> cinv((size_t)m * m), v(m);
  for (int c = 0; c < m; ++c) {
    std::fill(v.begin(), v.end(), 0.0);
    v[c] = 1.0;
    for (int a = 0; a < m; ++a) {
      double sum = v[a];
      for (int k = 0; k < a; ++k) sum -= cap[(size_t)a * m + k] * v[k];
      v[a] = sum / cap[(size_t)a * m + a];
    }
    for (int a = m - 1; a >= 0; --a) {
      double sum = v[a];
      for (int k = a + 1; k < m; ++k) sum -= cap[(size_t)k * m + a] * v[k];
      v[a] = sum / cap[(size_t)a * m + a];
    }
    for (int a = 0; a < m; ++a) cinv[(size_t)a * m + c] = v[a];
  }
  const size_t nzz = (size_t)(m + 1) * nzp;
  ce = cudaMemcpyAsync((void *)P.Binv, Binv.data(), Binv.size() * 8, cudaMemcpyHostToDevice, x->s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void *)P.hq, hq.data(), (size_t)nzp * 8, cudaMemcpyHostToDevice, x->s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void *)P.ZP, zp.data(), zp.size() * 8, cudaMemcpyHostToDevice, x->s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void *)P.Cinv, cinv.data(), cinv.size() * 8, cudaMemcpyHostToDevice, x->s);
  for (double *a : {x->hp, x->erp, x->hp2, x->erp2})
    if (ce == cudaSuccess) ce = cudaMemsetAsync(a, 0, (size_t)np * 8, x->s);
  for (double *a : {x->ezp, x->ezp2})
    if (ce == cudaSuccess) ce = cudaMemsetAsync(a, 0, nzz * 8, x->s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(x->s);
  return ce == cudaSuccess ? PIC_OK : PIC_E_CUDA;
}
}  // namespace

int pic_init(const pic_config *cfg, void *workspace_dev, size_t workspace_bytes, void *stream,
             pic_ctx **out) {
  if (!out) return PIC_E_CONFIG;
  *out = nullptr;
  if (!valid(cfg)) return PIC_E_CONFIG;
  if (!workspace_dev || ((uintptr_t)workspace_dev & 255)) return PIC_E_WORKSPACE;
  pic_ctx *x = (pic_ctx *)calloc(1, sizeof(pic_ctx));
  if (!x) return PIC_E_CONFIG;
  x->cfg = *cfg;
  x->s = (cudaStream_t)stream;
  size_t used = 0;
  if (!layout(x, cfg, (char *)workspace_dev, workspace_bytes, &used)) {
    free(x);
    return PIC_E_WORKSPACE;
  }
  x->ws = (char *)workspace_dev;
  x->ws_bytes = workspace_bytes;
  int nr = cfg->nr, nz = cfg->nz;
  x->g.nr = nr;
  x->g.nz = nz;
  x->g.R = cfg->R;
  x->g.L = cfg->L;
  x->g.xa = cfg->axis_cells;
  x->g.nd = cfg->ring_cells;
  x->g.erd = cfg->ring_cells > 0 ? cfg->eps_ring : 1.0;
  x->g.sgd = cfg->ring_cells > 0 ? cfg->sigma_ring : 0.0;
  x->g.dr = cfg->R / (nr + cfg->axis_cells);
  x->g.dz = cfg->L / nz;
  x->eps = cfg->eps > 0 ? cfg->eps : kEps0;
  x->mu = cfg->mu > 0 ? cfg->mu : kMu0;
  x->cap[0] = x->cap[1] = capacity(cfg);
  x->mixed = cfg->precision == PIC_MIXED ? 1 : 0;
  for (int sp = 0; sp < 2; ++sp) {
    double qm = sp == 0 ? -kQE / kME : kQE / kMAr;
    x->alpha.sr[sp] = x->alpha64.sr[sp] = qm * cfg->dt * cfg->dt / x->g.dr;
    x->alpha.sz[sp] = x->alpha64.sz[sp] = qm * cfg->dt * cfg->dt / x->g.dz;
    for (int i = 0; i < x->g.xa; ++i)
      x->alpha.srx[sp][i] = x->alpha64.srx[sp][i] = qm * cfg->dt * cfg->dt / g_width(x->g, i);
  }
  x->alpha.xa = x->alpha64.xa = x->g.xa;
  x->alpha.nz1 = x->alpha64.nz1 = nz + 1;
  x->ng = cfg->mcc_on ? cfg->gas_pressure / (kKB * cfg->gas_temp) : 0.0;

  // MCC constants (host): nu_max over eps <= 1 keV (x 1.01), ion g_max
  if (cfg->mcc_on) {
    double best = 0.0;
    for (int k = 1; k <= 200000; ++k) {
      double e = 1000.0 * (double)k / 200000.0;
      double v = sqrt(2.0 * e * kQE / kME);
      double nu = x->ng * (h_sig_el(e) + h_sig_ex(e) + h_sig_iz(e)) * v;
      if (nu > best) best = nu;
    }
    x->numax_e = 1.01 * best;
    double vthg = sqrt(kKB * cfg->gas_temp / kMAr);
    x->gmax = sqrt(2.0 * kQE * 1000.0 / kMAr) + 5.0 * vthg;
    double nu_i = x->ng * kSigmaCx * x->gmax;
    x->pnull_e = -expm1(-x->numax_e * cfg->dt);
    x->pnull_i = -expm1(-nu_i * cfg->dt);
  }

  // field operator: DCT-II along z diagonalises the Neumann Laplacian T_z;
  // per mode m an SPD tridiagonal system along r, factorised once (Thomas)
  FieldOp &F = x->F;
  F.nr = nr;
  F.nz = nz;
  F.dr = x->g.dr;
  F.dz = x->g.dz;
  F.dt = cfg->dt;
  F.eps = x->eps;
  F.mu = x->mu;
  F.L = cfg->L;
  F.unit_c = -1;
  double dz = F.dz, hdt2 = 0.5 * cfg->dt * cfg->dt;
  std::vector<double> Q((size_t)nz * nz), QT((size_t)nz * nz), lam(nz);
  // FFT path when nz = 4^a 2^b 3^c is even (at most 4096); else the GEMM path
  F.fft = 0;
  F.nrad = 0;
  if (nz % 2 == 0 && nz <= 4096) {
    int n = nz, k = 0;
    int rad[16];
    while (n % 4 == 0 && k < 16) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < 16) { rad[k++] = 2; n /= 2; }
    while (n % 3 == 0 && k < 16) { rad[k++] = 3; n /= 3; }
    if (n == 1) {
      F.fft = nz;
      F.nrad = k;
      for (int q = 0; q < k; ++q) F.rad[q] = rad[q];
    }
  }
  F.half = (!F.fft && nz % 2 == 0) ? nz / 2 : 0;
  F.c0 = sqrt(1.0 / nz);
  F.c1 = sqrt(2.0 / nz);
  const int hz = F.half;
  auto qbasis = [&](int j, int m) {
    double cm = m == 0 ? sqrt(1.0 / nz) : sqrt(2.0 / nz);
    return cm * cos(kPi * m * (j + 0.5) / nz);
  };
  // column of mode m in the transformed arrays
  std::vector<int> col(nz);
  for (int m = 0; m < nz; ++m) {
    lam[m] = 2.0 - 2.0 * cos(kPi * m / nz);
    col[m] = hz ? ((m % 2 == 0) ? m / 2 : hz + m / 2) : m;
  }
  if (hz) {
    for (int j = 0; j < hz; ++j)
      for (int k = 0; k < hz; ++k) {
        double ve = qbasis(j, 2 * k), vo = qbasis(j, 2 * k + 1);
        Q[(size_t)j * hz + k] = ve;                       // Qe
        Q[(size_t)hz * hz + (size_t)j * hz + k] = vo;     // Qo
        QT[(size_t)k * hz + j] = ve;                      // Qe^T
        QT[(size_t)hz * hz + (size_t)k * hz + j] = vo;    // Qo^T
      }
  } else {
    for (int m = 0; m < nz; ++m)
      for (int j = 0; j < nz; ++j) {
        double v = qbasis(j, m);
        Q[(size_t)j * nz + m] = v;
        QT[(size_t)m * nz + j] = v;
      }
  }
  std::vector<double> mass(nr), kz(nr), kdiag(nr), eoff(nr, 0.0);
  // radial geometry of the (mapped) mesh: cell-centre radius, cell width and
  // E_z dual-face area per row
  const Grid &G = x->g;
  auto rh = [&](int i) { return g_rcentre(G, i); };
  auto wr = [&](int i) { return g_width(G, i); };
  auto az = [&](int i) { return g_aeff_z(G, i); };     // permittivity-weighted
  auto are = [&](int i) { return g_aeff_r(G, i); };
  // D = eps A + dt S / 2 per edge (S: the conducting part, Eq. 2's sigma E at the half step)
  auto dnr = [&](int i) { return x->eps * are(i) + 0.5 * cfg->dt * g_asig_r(G, i); };
  auto dnz = [&](int i) { return x->eps * az(i) + 0.5 * cfg->dt * g_asig_z(G, i); };
  for (int i = 0; i < nr; ++i) {
    mass[i] = 2.0 * x->mu * (kTwoPi * rh(i) * wr(i) * dz);
    double s = kTwoPi * rh(i);
    kz[i] = hdt2 * (wr(i) / dnr(i)) * s * s;
    double wz_i = dz / dnz(i);
    double d = wz_i * s * s;
    if (i + 1 <= nr - 1) d += (dz / dnz(i + 1)) * s * s;
    kdiag[i] = hdt2 * d;
    if (i >= 1) eoff[i] = hdt2 * wz_i * (-kTwoPi * rh(i - 1)) * s;
  }
  // wave port: the boundary field -eta H of the outermost H row enters its
  // Faraday equation (dt 2 pi r_{nr-1/2} dz eta on the diagonal)
  F.wave = cfg->feed == PIC_FEED_WAVE ? 1 : 0;
  F.eta = sqrt(x->mu / x->eps);
  if (F.wave) kdiag[nr - 1] += cfg->dt * kTwoPi * rh(nr - 1) * dz * F.eta;
  // cyclic-reduction coefficients of each column (rows padded to n2 with identity)
  const int n2 = F.n2;
  std::vector<double> cr((size_t)5 * n2 * nz, 0.0);
  std::vector<double> A(n2), B(n2), Cc(n2);
  for (int m = 0; m < nz; ++m) {
    double *co = cr.data() + (size_t)col[m] * 5 * n2;
    for (int i = 0; i < n2; ++i) {
      bool in = i < nr;
      A[i] = in && i >= 1 ? eoff[i] : 0.0;
      Cc[i] = in && i + 1 < nr ? eoff[i + 1] : 0.0;
      B[i] = in ? mass[i] + kz[i] * lam[m] + kdiag[i] : 1.0;
    }
    cr_coeffs(n2, A, B, Cc, co);
  }
  // electrostatic model: DST-I basis, per-row coefficients, mode coefficients
  const int M = nz - 1;
  std::vector<double> Sd((size_t)M * M), et((size_t)4 * nr), ecr((size_t)5 * n2 * M, 0.0);
  for (int j = 1; j <= M; ++j)
    for (int m = 1; m <= M; ++m) Sd[(size_t)(j - 1) * M + (m - 1)] = sqrt(2.0 / nz) * sin(kPi * j * m / nz);
  for (int i = 0; i < nr; ++i) {
    et[i] = x->eps * are(i) / wr(i);                                           // cR: face i+1/2
    et[nr + i] = i >= 1 ? x->eps * are(i - 1) / wr(i - 1) : 0.0;                 // cL: face i-1/2
    et[2 * nr + i] = x->eps * az(i) / dz;                                      // cZ
    et[3 * nr + i] = wr(i);                                                    // E_r edge length
  }
  // FFT plan of the DST-I (2 nz points) when 2 nz = 4^a 2^b 3^c <= 8192
  x->es.fft2 = 0;
  x->es.nrad = 0;
  std::vector<double> tw2((size_t)4 * nz);
  {
    int n = 2 * nz, k = 0;
    int rad[16];
    while (n % 4 == 0 && k < 16) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < 16) { rad[k++] = 2; n /= 2; }
    while (n % 3 == 0 && k < 16) { rad[k++] = 3; n /= 3; }
    if (n == 1 && 2 * nz <= 8192) {
      x->es.fft2 = 2 * nz;
      x->es.nrad = k;
      for (int q = 0; q < k; ++q) x->es.rad[q] = rad[q];
    }
    for (int q = 0; q < 2 * nz; ++q) {
      double t = -kTwoPi * (double)q / (2.0 * nz);
      tw2[2 * q] = cos(t);
      tw2[2 * q + 1] = sin(t);
    }
  }
  for (int m = 1; m <= M; ++m) {
    const double lm = 2.0 - 2.0 * cos(kPi * m / nz);
    for (int i = 0; i < n2; ++i) {
      bool in = i < nr;
      A[i] = in && i >= 1 ? -et[nr + i] : 0.0;
      Cc[i] = in && i + 1 < nr ? -et[i] : 0.0;
      B[i] = in ? et[i] + et[nr + i] + et[2 * nr + i] * lm : 1.0;
    }
    cr_coeffs(n2, A, B, Cc, ecr.data() + (size_t)(m - 1) * 5 * n2);
  }
  // twiddles, DCT phases and per-row reciprocal tables
  std::vector<double> tw((size_t)2 * nz), pw((size_t)2 * nz), rt((size_t)9 * (nr + 1), 0.0);
  for (int k = 0; k < nz; ++k) {
    double t = -kTwoPi * (double)k / nz;
    tw[2 * k] = cos(t);
    tw[2 * k + 1] = sin(t);
    double u = kPi * (double)k / (2.0 * nz);
    pw[2 * k] = cos(u);
    pw[2 * k + 1] = sin(u);
  }
  for (int i = 0; i <= nr; ++i) {
    // the E_r row nr and the E_z node nr are prescribed: only their finite
    // placeholders matter
    double ear = x->eps * (i < nr ? are(i) : kTwoPi * rh(i) * dz);
    double eaz = x->eps * az(i);
    double dr_ = i < nr ? dnr(i) : ear, dz_ = i < nr ? dnz(i) : eaz;
    rt[0 * (nr + 1) + i] = 1.0 / (2.0 * dr_);
    rt[1 * (nr + 1) + i] = 1.0 / (2.0 * dz_);
    rt[2 * (nr + 1) + i] = 1.0 / dr_;
    rt[3 * (nr + 1) + i] = 1.0 / dz_;
    rt[4 * (nr + 1) + i] = kTwoPi * rh(i);
    rt[5 * (nr + 1) + i] = kTwoPi * rh(i) * wr(i) * dz;
    rt[6 * (nr + 1) + i] = wr(i);
    rt[7 * (nr + 1) + i] = dr_ == ear ? 1.0 : ear / dr_;
    rt[8 * (nr + 1) + i] = dz_ == eaz ? 1.0 : eaz / dz_;
  }
  cudaError_t e = cudaSuccess;
  auto up = [&](const void *dst, const void *src, size_t b) {
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)dst, src, b, cudaMemcpyHostToDevice, x->s);
  };
  up(F.tw, tw.data(), tw.size() * 8);
  up(F.pw, pw.data(), pw.size() * 8);
  up(F.rtab, rt.data(), rt.size() * 8);
  up(F.Q, Q.data(), Q.size() * 8);
  up(F.QT, QT.data(), QT.size() * 8);
  up(F.crc, cr.data(), cr.size() * 8);
  up(x->es.S, Sd.data(), Sd.size() * 8);
  up(x->es.tab, et.data(), et.size() * 8);
  up(x->es.crc, ecr.data(), ecr.size() * 8);
  up(x->es.tw2, tw2.data(), tw2.size() * 8);
  // radial scales of the mapped cells: inner-face radius / w, dt / w, w / dt
  std::vector<double> rm64((size_t)3 * kMaxAxisCells, 0.0);
  std::vector<float> rm32((size_t)3 * kMaxAxisCells, 0.f);
  for (int i = 0; i < x->g.xa; ++i) {
    const double w = g_width(x->g, i);
    rm64[i] = g_rho0(x->g, i);
    rm64[kMaxAxisCells + i] = cfg->dt / w;
    rm64[2 * kMaxAxisCells + i] = w / cfg->dt;
    for (int k = 0; k < 3; ++k)
      rm32[k * kMaxAxisCells + i] = (float)rm64[k * kMaxAxisCells + i];
  }
  up(x->rmap64, rm64.data(), rm64.size() * 8);
  up(x->rmap32, rm32.data(), rm32.size() * 4);
  size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz, nh = (size_t)nr * nz;
  if (e == cudaSuccess) e = cudaMemsetAsync(x->er, 0, ner * 8, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->ez, 0, nez * 8, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->h, 0, nh * 8, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->h2, 0, nh * 8, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->wall, 0, (size_t)2 * (2 * (nr + 1) + nz + 1) * 8, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->qc, 0, (size_t)(nr + 1) * (nz + 1) * 8, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->hist, 0, 16 * 8, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->cnt, 0, sizeof(DevCounters), x->s);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&x->hn, 8 * kHnSlots, cudaHostAllocDefault);
  if (e == cudaSuccess && x->mixed) {
    // side stream of the electrons' near-axis FP64 list (runs beside the ions)
    // the highest priority: its few blocks are placed before the next
    // persistent push kernel fills the SMs
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&x->pstream, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->pev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->pev[1], cudaEventDisableTiming);
    if (e == cudaSuccess) x->pstream_made = 1;
  }
  if (e == cudaSuccess) {
    e = cudaStreamCreateWithFlags(&x->sstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->sev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->sev[1], cudaEventDisableTiming);
    if (e == cudaSuccess) x->sstream_made = 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  if (e != cudaSuccess) {
    if (x->hn) cudaFreeHost(x->hn);
    if (x->pstream_made) {
      cudaEventDestroy(x->pev[0]);
      cudaEventDestroy(x->pev[1]);
      cudaStreamDestroy(x->pstream);
    }
    free(x);
    return PIC_E_CUDA;
  }
  x->F.vd = x->vdev;
  x->es.vd = x->vdev;
  x->hist_n = 1;
  x->fb_alpha = -1;
  x->dloop = 1;
  if (cfg->feed == PIC_FEED_AXIAL && cfg->field_model == PIC_FIELD_EM) {
    const int pr = port_setup(x, cfg);
    if (pr) {
      pic_destroy(x);
      return pr;
    }
  }
  if (cfg->feed == PIC_FEED_AXIAL && cfg->field_model == PIC_FIELD_ES) {
    // the electrostatic port: the coaxial line's potential on the opening
    const int ip = cfg->port_rin;
    std::vector<double> g0(nr + 1);
    const double lr = log(g_rnode(x->g, ip) / g_rnode(x->g, nr));
    for (int i = 0; i <= nr; ++i)
      g0[i] = i <= ip ? 1.0 : log(g_rnode(x->g, i) / g_rnode(x->g, nr)) / lr;
    x->es.pip = ip;
    if (e == cudaSuccess)
      e = cudaMemcpy((void *)x->es.g0, g0.data(), (nr + 1) * 8, cudaMemcpyHostToDevice);
    // the interior potential of a unit electrode potential (no charge)
    EsOp U = x->es;
    U.vd = nullptr;
    U.cc = Circuit{};
    const size_t nn = (size_t)(nr + 1) * (nz + 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(x->qn, 0, nn * 8, x->s);
    if (e == cudaSuccess)
      e = launch_es_solve(U, x->qn, nullptr, nullptr, 1.0, x->er2, x->ez2, nullptr, nullptr,
                          nullptr, x->s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void *)x->es.uphi, x->es.phi, (size_t)nr * (nz - 1) * 8,
                          cudaMemcpyDeviceToDevice, x->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
    if (e != cudaSuccess) {
      pic_destroy(x);
      return PIC_E_CUDA;
    }
  }
  if (cfg->cblock > 0.0) {
    // unit response: H^{n+1} of a unit electrode potential at n+1 with no
    // fields at n and no charge (fields, H and the crossed charge are zero here)
    FieldOp U = x->F;
    U.vd = nullptr;
    if (e == cudaSuccess) e = cudaMemsetAsync(x->ir, 0, ner * 8, x->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(x->iz, 0, nez * 8, x->s);
    if (e == cudaSuccess)
      e = launch_field_solve(U, x->er, x->ez, x->h, x->ir, x->iz, 0.0, 1.0, x->er2, x->ez2, x->hu,
                             nullptr, nullptr, x->cnt, x->s);
    // with the axial port the unit potential enters as Eq. 7's incoming wave
    // (the port's fields at n are zero here); keep the port's H^{n+1} as well
    if (e == cudaSuccess && x->F.port.on) {
      e = cudaMemcpyAsync(x->hup, x->hp2, (size_t)x->F.port.np * 8, cudaMemcpyDeviceToDevice, x->s);
      x->F.port.hup = x->hup;
    }
    double cr = 0.0;
    for (int i = 0; i < nr; ++i) cr += x->eps * az(i);
    cr /= cfg->L;
    if (x->es.pip && e == cudaSuccess) {
      // the flow of the unit solve through the faces over the electrode disc
      const int M = nz - 1, ip = x->es.pip;
      std::vector<double> up((size_t)nr * M), tb((size_t)4 * nr);
      e = cudaMemcpy(up.data(), x->es.uphi, up.size() * 8, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(tb.data(), x->es.tab, tb.size() * 8, cudaMemcpyDeviceToHost);
      cr = 0.0;
      for (int i = 0; i < ip; ++i) cr += tb[2 * nr + i] * (1.0 - up[(size_t)i * M]);
    }
    x->circ_on = 1;
    x->F.cc = Circuit{x->vdev + 4, x->hu, cfg->cblock, 0.0};
    x->es.cc = Circuit{x->vdev + 4, nullptr, cfg->cblock, cr};
    x->es.ez0 = nullptr;
    if (e == cudaSuccess) e = circuit_reset(x);
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
    if (e != cudaSuccess) {
      pic_destroy(x);
      return PIC_E_CUDA;
    }
  }
  *out = x;
  return PIC_OK;
}

void pic_destroy(pic_ctx *ctx) {
  if (!ctx) return;
  if (ctx->ngraph || ctx->hn) cudaStreamSynchronize(ctx->s);
  for (int k = 0; k < ctx->ngraph; ++k) {
    cudaGraphExecDestroy(ctx->gcache[k].exec);
    if (ctx->gcache[k].ptimed) {
      cudaEventDestroy(ctx->gcache[k].pe[0]);
      cudaEventDestroy(ctx->gcache[k].pe[1]);
    }
  }
  if (ctx->hn) cudaFreeHost(ctx->hn);
  if (ctx->gev_made) {
    cudaStreamSynchronize(ctx->s);
    cudaEventDestroy(ctx->gev[0]);
    cudaEventDestroy(ctx->gev[1]);
  }
  if (ctx->prof) {
    cudaStreamSynchronize(ctx->s);
    for (int k = 0; k < 2 * 128; ++k) cudaEventDestroy(ctx->ev[k]);
  }
  if (ctx->pstream_made) {
    cudaStreamSynchronize(ctx->pstream);
    cudaEventDestroy(ctx->pev[0]);
    cudaEventDestroy(ctx->pev[1]);
    cudaStreamDestroy(ctx->pstream);
  }
  if (ctx->sstream_made) {
    cudaStreamSynchronize(ctx->sstream);
    cudaEventDestroy(ctx->sev[0]);
    cudaEventDestroy(ctx->sev[1]);
    cudaStreamDestroy(ctx->sstream);
  }
  if (ctx->nloop) cudaStreamSynchronize(ctx->s);
  for (int k = 0; k < ctx->nloop; ++k) {
    cudaGraphExecDestroy(ctx->lcache[k].exec);
    cudaGraphDestroy(ctx->lcache[k].graph);
  }
  if (ctx->hs_made) {
    cudaStreamSynchronize(ctx->hs_dn);
    cudaStreamSynchronize(ctx->hs_up);
    for (int k = 0; k < 130; ++k) cudaEventDestroy(ctx->hs_ev[k]);
    cudaStreamDestroy(ctx->hs_dn);
    cudaStreamDestroy(ctx->hs_up);
  }
  free(ctx);
}

int pic_profile(pic_ctx *x, int enable) {
  if (!x) return PIC_E_CONFIG;
  if (cudaStreamSynchronize(x->s) != cudaSuccess) return PIC_E_CUDA;
  if (enable && !x->prof) {
    for (int k = 0; k < 2 * 128; ++k)
      if (cudaEventCreate(&x->ev[k]) != cudaSuccess) return PIC_E_CUDA;
    x->prof = 1;
  }
  x->nev = 0;
  x->push_ms = 0.0;
  x->push_launches = x->pending_launches = 0;
  x->rep_pe = nullptr;
  if (!enable && x->prof) {
    for (int k = 0; k < 2 * 128; ++k) cudaEventDestroy(x->ev[k]);
    x->prof = 0;
  }
  return PIC_OK;
}

int pic_profile_read(pic_ctx *x, double *push_ms, long long *push_launches) {
  if (!x) return PIC_E_CONFIG;
  if (cudaStreamSynchronize(x->s) != cudaSuccess) return PIC_E_CUDA;
  if (x->prof) prof_collect(x);
  if (push_ms) *push_ms = x->push_ms;
  if (push_launches) *push_launches = x->push_launches;
  return PIC_OK;
}

namespace {

// enqueue the sort of both species (each one's kept count into its pinned
// slot); sort_finish reads the counts after the caller's wait
int sort_enqueue(pic_ctx *x) {
  for (int s = 0; s < (x->cfg.ions_fixed ? 1 : 2); ++s) {
    SortLaunch S;
    S.ncell = x->g.nr * x->g.nz;
    S.n = x->n[s];
    S.src = cur(x, s);
    S.dst = x->P[s][x->cur[s] ^ 1];
    S.counts = x->counts;
    S.offs = x->coffs;
    S.cursor = x->cursor;
    S.total = x->total + s;
    S.scan_scratch = x->scan_scratch;
    cudaError_t se;
    if (x->mixed) {
      SortLaunchT<float> S32{S.ncell, S.n, as32(S.src), as32(S.dst), S.counts, S.offs,
                             S.cursor, S.total, S.scan_scratch};
      se = launch_sort(S32, x->s);
    } else {
      se = launch_sort(S, x->s);
    }
    if (se != cudaSuccess) return PIC_E_CUDA;
    x->launches += S.n > 0 ? 5 : 3;
    if (cudaMemcpyAsync(x->hn + kHnTotal + s, x->total + s, 8, cudaMemcpyDeviceToHost, x->s) !=
        cudaSuccess)
      return PIC_E_CUDA;
    x->cur[s] ^= 1;
  }
  return PIC_OK;
}

void sort_finish(pic_ctx *x) {
  for (int s = 0; s < (x->cfg.ions_fixed ? 1 : 2); ++s)
    memcpy(&x->n[s], x->hn + kHnTotal + s, 8);
}

}  // namespace

int pic_sort(pic_ctx *x) {
  if (!x) return PIC_E_CONFIG;
  int r = sort_enqueue(x);
  if (r) return r;
  if (cudaStreamSynchronize(x->s) != cudaSuccess) return PIC_E_CUDA;
  sort_finish(x);
  return PIC_OK;
}

int pic_load_particles(pic_ctx *x) {
  if (!x) return PIC_E_CONFIG;
  long long n = x->cfg.np_init;
  if (n > x->cap[0] || n > x->cap[1] || n > 0xFFFFFFFFll) return PIC_E_CAPACITY;
  Grid gp = x->g;
  gp.nr = x->g.nr - x->g.nd;  // the plasma region inside the dielectric ring
  cudaError_t le =
      x->mixed ? launch_load(gp, n, x->cfg.n0, x->cfg.te_ev, x->cfg.ti_ev, x->cfg.seed,
                             as32(cur(x, 0)), as32(cur(x, 1)), x->s)
               : launch_load(gp, n, x->cfg.n0, x->cfg.te_ev, x->cfg.ti_ev, x->cfg.seed,
                             cur(x, 0), cur(x, 1), x->s);
  if (le != cudaSuccess) return PIC_E_CUDA;
  if (n > 0) x->launches += 1;
  x->n[0] = x->n[1] = n;
  x->next_id[0] = x->next_id[1] = (uint32_t)n;
  x->hist_n = 1;
  x->sample_valid = 0;
  x->qn_valid = 0;
  if (x->circ_on && circuit_reset(x) != cudaSuccess) return PIC_E_CUDA;
  return pic_sort(x);
}

int pic_set_picard(pic_ctx *x, double tol, int kmax) {
  if (!x || !(tol > 0.0) || !isfinite(tol) || kmax < 1) return PIC_E_CONFIG;
  x->cfg.picard_tol = tol;
  x->cfg.picard_max = kmax;
  return PIC_OK;
}

int pic_set_drive(pic_ctx *x, int n, const double *amp, const double *freq, const double *phase) {
  if (!x || n < 0 || n > 64 || (n > 0 && (!amp || !freq || !phase))) return PIC_E_CONFIG;
  for (int k = 0; k < n; ++k)
    if (!isfinite(amp[k]) || !isfinite(freq[k]) || !isfinite(phase[k])) return PIC_E_CONFIG;
  for (int k = 0; k < n; ++k) {
    x->hamp[k] = amp[k];
    x->hfreq[k] = freq[k];
    x->hph[k] = phase[k];
  }
  x->nharm = n;
  return PIC_OK;
}

// m-th positive zero of J_alpha (alpha = 0, 1): McMahon's asymptotic start,
// then Newton with J_0' = -J_1, J_1' = J_0 - J_1 / x
double bessel_zero(int alpha, int m) {
  const double b = (m + 0.5 * alpha - 0.25) * kPi;
  const double mu = 4.0 * alpha * alpha;
  double x = b - (mu - 1.0) / (8.0 * b);
  for (int it = 0; it < 50; ++it) {
    const double j = std::cyl_bessel_j((double)alpha, x);
    const double d = alpha == 0 ? -std::cyl_bessel_j(1.0, x)
                                : std::cyl_bessel_j(0.0, x) - j / x;
    const double step = j / d;
    x -= step;
    if (fabs(step) < 1e-15 * x) break;
  }
  return x;
}

int pic_fourier_bessel(pic_ctx *x, int alpha, int row, int nmodes, double *coef) {
  if (!x || !coef || (alpha != 0 && alpha != 1) || nmodes < 1 || nmodes > 64) return PIC_E_CONFIG;
  const int nr = x->g.nr, nz = x->g.nz;
  if (alpha == 0 ? (row < 0 || row >= nz) : (row < 0 || row > nz)) return PIC_E_CONFIG;
  const int n = alpha == 0 ? nr + 1 : nr;
  if (x->fb_alpha != alpha || x->fb_m != nmodes) {
    // basis[m][k] = w_k r_k F_m(r_k) / sum_k w_k r_k F_m(r_k)^2 (Eq. A2 by the
    // trapezoid rule on nodes, alpha = 0, or the midpoint rule, alpha = 1)
    const double R = x->cfg.R;
    const Grid &G = x->g;
    std::vector<double> B((size_t)nmodes * n);
    for (int m = 0; m < nmodes; ++m) {
      const double chi = bessel_zero(alpha, m + 1);
      double den = 0.0;
      for (int k = 0; k < n; ++k) {
        // nodes with trapezoid weights, or cell centres with the cell widths
        double r, w;
        if (alpha == 0) {
          r = g_rnode(G, k);
          w = 0.5 * ((k > 0 ? g_width(G, k - 1) : 0.0) + (k < nr ? g_width(G, k) : 0.0));
        } else {
          r = 0.5 * (g_rnode(G, k) + g_rnode(G, k + 1));
          w = g_width(G, k);
        }
        const double F = std::cyl_bessel_j((double)alpha, chi * r / R);
        B[(size_t)m * n + k] = w * r * F;
        den += w * r * F * F;
      }
      for (int k = 0; k < n; ++k) B[(size_t)m * n + k] /= den;
    }
    if (cudaMemcpyAsync(x->fbb, B.data(), B.size() * 8, cudaMemcpyHostToDevice, x->s) !=
            cudaSuccess ||
        cudaStreamSynchronize(x->s) != cudaSuccess)
      return PIC_E_CUDA;
    x->fb_alpha = alpha;
    x->fb_m = nmodes;
  }
  const double *f = alpha == 0 ? x->ez + row : x->er + row;
  const int stride = alpha == 0 ? nz : nz + 1;
  cudaError_t e = launch_fourier_bessel(x->fbb, f, stride, n, nmodes, coef, x->s);
  x->launches += 1;
  return cuda_rc(e);
}

int pic_circuit_get(pic_ctx *x, double *q, double *phi) {
  if (!x) return PIC_E_CONFIG;
  double st[4] = {0.0, 0.0, volt_at(x, x->step), 0.0};
  if (x->circ_on) {
    if (cudaMemcpyAsync(st, x->vdev + 4, sizeof(st), cudaMemcpyDeviceToHost, x->s) != cudaSuccess)
      return PIC_E_CUDA;
    if (cudaStreamSynchronize(x->s) != cudaSuccess) return PIC_E_CUDA;
  }
  if (q) *q = st[0];
  if (phi) *phi = st[2];
  return PIC_OK;
}

int pic_circuit_set(pic_ctx *x, double q, double phi) {
  if (!x || !x->circ_on || !isfinite(q) || !isfinite(phi)) return PIC_E_CONFIG;
  const double st[4] = {q, 0.0, phi, 0.0};
  if (cudaMemcpyAsync(x->vdev + 4, st, sizeof(st), cudaMemcpyHostToDevice, x->s) != cudaSuccess)
    return PIC_E_CUDA;
  return cudaStreamSynchronize(x->s) == cudaSuccess ? PIC_OK : PIC_E_CUDA;
}

int pic_push_deposit(pic_ctx *x, const double *erh, const double *ezh, double *ir, double *iz,
                     int write, unsigned long long *counters, double *kel) {
  if (!x || !erh || !ezh) return PIC_E_CONFIG;
  // normalised accelerations of both species from the caller's E^{n+1/2}
  cudaError_t ae = x->mixed ? launch_half_field_alpha(x->g, erh, ezh, erh, ezh, x->erh, x->ezh,
                                                      x->alpha, x->s)
                            : launch_half_field_alpha64(x->g, erh, ezh, erh, ezh, x->erh,
                                                        x->ezh, x->alpha64, x->s);
  if (ae != cudaSuccess) return PIC_E_CUDA;
  x->launches += 1;
  if (cudaMemcpyAsync(x->n_dev, x->n, 16, cudaMemcpyHostToDevice, x->s) != cudaSuccess)
    return PIC_E_CUDA;
  return push_all(x, erh, ezh, ir, iz, write, counters, kel, write ? x->wall : nullptr);
}

int pic_field_solve(pic_ctx *x, const double *er0, const double *ez0, const double *h0,
                    const double *ir, const double *iz, double v0, double v1, double *er1,
                    double *ez1, double *h1, double *src) {
  if (!x || !er0 || !ez0 || !h0 || !ir || !iz || !er1 || !ez1 || !h1) return PIC_E_CONFIG;
  FieldOp F = x->F;
  F.vd = nullptr;  // the caller's voltages
  F.cc = Circuit{};
  cudaError_t e = launch_field_solve(F, er0, ez0, h0, ir, iz, v0, v1, er1, ez1, h1, nullptr,
                                     nullptr, x->cnt, x->s);
  x->launches += F.port.on ? 10 : 5;
  if (e == cudaSuccess && src)
    e = cudaMemcpyAsync(src, &x->cnt->src, 8, cudaMemcpyDeviceToDevice, x->s);
  return cuda_rc(e);
}

int pic_port_field_solve(pic_ctx *x, const double *er0, const double *ez0, const double *h0,
                         const double *hp0, const double *erp0, const double *ezp0,
                         const double *ir, const double *iz, double phi0, double phi1,
                         double *er1, double *ez1, double *h1, double *hp1, double *erp1,
                         double *ezp1, double *src) {
  if (!x || !x->F.port.on) return PIC_E_CONFIG;
  if (!er0 || !ez0 || !h0 || !hp0 || !erp0 || !ezp0 || !ir || !iz || !er1 || !ez1 || !h1 ||
      !hp1 || !erp1 || !ezp1)
    return PIC_E_CONFIG;
  FieldOp F = x->F;
  F.vd = nullptr;  // the caller's potentials
  F.cc = Circuit{};
  F.port.hp0 = hp0;
  F.port.erp0 = erp0;
  F.port.ezp0 = ezp0;
  F.port.hp1 = hp1;
  F.port.erp1 = erp1;
  F.port.ezp1 = ezp1;
  cudaError_t e = launch_field_solve(F, er0, ez0, h0, ir, iz, phi0, phi1, er1, ez1, h1, nullptr,
                                     nullptr, x->cnt, x->s);
  x->launches += 10;
  if (e == cudaSuccess && src)
    e = cudaMemcpyAsync(src, &x->cnt->src, 8, cudaMemcpyDeviceToDevice, x->s);
  return cuda_rc(e);
}

int pic_es_solve(pic_ctx *x, const double *Q, double phi0, double *er, double *ez) {
  if (!x || !Q || !er || !ez) return PIC_E_CONFIG;
  EsOp E = x->es;
  E.vd = nullptr;  // the caller's potential
  E.cc = Circuit{};
  cudaError_t e = launch_es_solve(E, Q, nullptr, nullptr, phi0, er, ez, nullptr, nullptr, nullptr,
                                  x->s);
  x->launches += 5;
  return cuda_rc(e);
}

namespace {
int mcc_run(pic_ctx *x, unsigned long long step, long long *counts, double *de_coll);
}  // namespace

int pic_mcc(pic_ctx *x, unsigned long long step, long long *counts, double *de_coll) {
  if (!x) return PIC_E_CONFIG;
  return mcc_run(x, step, counts, de_coll);
}

namespace {
// one MCC pass; de_coll (nullable) is read after the appended pairs are
// counted in, which costs a wait: the step instead copies the pinned slot
// kHnDe with its other counters (de_coll = nullptr here)
int mcc_run(pic_ctx *x, unsigned long long step, long long *counts, double *de_coll) {
  cudaError_t e = cudaMemsetAsync(x->cnt->mcc, 0, sizeof(x->cnt->mcc), x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&x->cnt->de_coll, 0, 8, x->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&x->cnt->iz_slots, 0, 8, x->s);
  MccLaunch M;
  M.seed = x->cfg.seed;
  M.step = step;
  M.ng = x->ng;
  M.tg = x->cfg.gas_temp;
  M.numax_e = x->numax_e;
  M.pnull_e = x->pnull_e;
  M.pnull_i = x->pnull_i;
  M.gmax = x->gmax;
  M.thr_e = (uint64_t)ceil(x->pnull_e * 9007199254740992.0);
  M.thr_i = (uint64_t)ceil(x->pnull_i * 9007199254740992.0);
  M.ne = x->n[0];
  M.ni = x->n[1];
  M.e = cur(x, 0);
  M.i = cur(x, 1);
  M.cand = x->cand;
  M.cblock = x->cblock;
  M.cseg = 0;
  M.cgrid = 0;
  M.cnt = x->cnt;
  M.keys = x->keys;
  M.keys2 = x->keys2;
  MccLaunchT<float> M32{M.seed, M.step, M.ng, M.tg, M.numax_e, M.pnull_e, M.pnull_i, M.gmax,
                        M.thr_e, M.thr_i, M.ne, M.ni, as32(M.e), as32(M.i), M.cand, M.cblock,
                        M.cseg, M.cgrid, M.cnt, M.keys, M.keys2};
  if (e == cudaSuccess) e = x->mixed ? launch_mcc_collide(M32, x->s) : launch_mcc_collide(M, x->s);
  x->launches += (M.ne > 0 || M.ni > 0 ? 2 : 0);
  // the process counts are final after the collisions: read them with the
  // number of ionizations in one wait (pinned slots)
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(x->hn + kHnIz, &x->cnt->iz_slots, 8, cudaMemcpyDeviceToHost, x->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(x->hn + kHnMcc, x->cnt->mcc, 64, cudaMemcpyDeviceToHost, x->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  if (e != cudaSuccess) return PIC_E_CUDA;
  long long tot = 0;
  unsigned long long hc[8];
  memcpy(&tot, x->hn + kHnIz, 8);
  memcpy(hc, x->hn + kHnMcc, 64);
  int rc = PIC_OK;
  unsigned long long capov = 0;
  if (tot > 0) {
    if (x->n[0] + tot > x->cap[0] || x->n[1] + tot > x->cap[1] ||
        (long long)x->next_id[0] + tot > 0xFFFFFFFFll || (long long)x->next_id[1] + tot > 0xFFFFFFFFll) {
      rc = PIC_E_CAPACITY;
      capov = (unsigned long long)tot;
    } else {
      e = x->mixed ? launch_mcc_append(M32, tot, x->n[0], x->n[1], x->next_id[0], x->next_id[1], x->s)
                   : launch_mcc_append(M, tot, x->n[0], x->n[1], x->next_id[0], x->next_id[1], x->s);
      if (e != cudaSuccess) return PIC_E_CUDA;
      x->launches += 2;
      x->n[0] += tot;
      x->n[1] += tot;
      x->next_id[0] += (uint32_t)tot;
      x->next_id[1] += (uint32_t)tot;
    }
  }
  hc[7] = capov;
  if (counts)
    for (int k = 0; k < 8; ++k) counts[k] = (long long)hc[k];
  if (de_coll) {
    // the appended pairs' energy is in de_coll after the append
    if (cudaMemcpyAsync(x->hn + kHnDe, &x->cnt->de_coll, 8, cudaMemcpyDeviceToHost, x->s) !=
            cudaSuccess ||
        cudaStreamSynchronize(x->s) != cudaSuccess)
      return PIC_E_CUDA;
    memcpy(de_coll, x->hn + kHnDe, 8);
  }
  return rc;
}
}  // namespace

namespace {

GuessArgs guess_args(pic_ctx *x) {
  GuessArgs A;
  A.nr = x->g.nr;
  A.nz = x->g.nz;
  A.e[0] = FieldPair{x->er, x->ez};
  for (int k = 0; k < 3; ++k) A.e[k + 1] = FieldPair{x->hr[k], x->hz[k]};
  A.h = x->h;
  A.jr = x->jr;
  A.jz = x->jz;
  A.sums = x->gsums;
  A.sd = x->gsd;
  A.ger = x->ger;
  A.gez = x->gez;
  A.x = x->gx;
  return A;
}

// counts and drive voltages of the coming step on the device
int upload_step(pic_ctx *x, double v0, double v1) {
  // pageable sources: the call returns once they are staged, so the stack is safe
  const double st[2] = {v0, v1};
  if (cudaMemcpyAsync(x->vdev, st, 16, cudaMemcpyHostToDevice, x->s) != cudaSuccess) return 1;
  if (cudaMemcpyAsync(x->n_dev, x->n, 16, cudaMemcpyHostToDevice, x->s) != cudaSuccess) return 1;
  return 0;
}

// plain start E^{n+1,0} = E^n with the drive value on r = R
int plain_start(pic_ctx *x, double v1) {
  const int nr = x->g.nr, nz = x->g.nz;
  const size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz;
  cudaError_t e = cudaMemcpyAsync(x->er1, x->er, ner * 8, cudaMemcpyDeviceToDevice, x->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x->ez1, x->ez, nez * 8, cudaMemcpyDeviceToDevice, x->s);
  // with the blocking capacitor, the wave port or the axial port the gap edges
  // keep E^n's
  if (e == cudaSuccess && !x->circ_on && !x->F.wave && !x->F.port.on && !x->es.pip) {
    k_fill<<<(nz + 127) / 128, 128, 0, x->s>>>(x->ez1 + (size_t)nr * nz, nz, v1 / x->cfg.L);
    e = cudaGetLastError();
    x->launches += 1;
  }
  return e == cudaSuccess ? PIC_OK : PIC_E_CUDA;
}

// extrapolated or learned start; *used = the start placed in er1/ez1
// (PIC_GUESS_PLAIN: nothing was placed, the caller falls back)
int guess_start(pic_ctx *x, double v1, int *used) {
  *used = PIC_GUESS_PLAIN;
  GuessArgs A = guess_args(x);
  if (launch_guess_inputs(A, x->s) != cudaSuccess) return PIC_E_CUDA;
  x->launches += 2;
  x->feat_now = 1;
  const float *y = nullptr;
  int cp = 0;
  if (x->guess_mode == PIC_GUESS_CNN) {
    // the network runs on its own stream, ordered after the inputs and before the start
    if (cudaEventRecord(x->gev[0], x->s) != cudaSuccess) return PIC_E_CUDA;
    if (cudaStreamWaitEvent(x->gstream, x->gev[0], 0) != cudaSuccess) return PIC_E_CUDA;
    if (cnn_forward_async(x->cnn, x->gx, &y, &cp)) return PIC_E_CUDA;
    if (cudaEventRecord(x->gev[1], x->gstream) != cudaSuccess) return PIC_E_CUDA;
    if (cudaStreamWaitEvent(x->s, x->gev[1], 0) != cudaSuccess) return PIC_E_CUDA;
    x->launches += 2 + 2 * x->cnn_layers;
  }
  int bad = 0;
  if (cudaMemsetAsync(x->gbad, 0, sizeof(int), x->s) != cudaSuccess) return PIC_E_CUDA;
  if (launch_guess_apply(A, y, cp, v1 / x->cfg.L, x->er1, x->ez1, x->gbad, x->s) != cudaSuccess)
    return PIC_E_CUDA;
  x->launches += 1;
  if (x->circ_on || x->F.wave || x->F.port.on || x->es.pip) {
    // the gap edges keep E^n's, as in the plain start
    const size_t g0 = (size_t)x->g.nr * x->g.nz;
    if (cudaMemcpyAsync(x->ez1 + g0, x->ez + g0, (size_t)x->g.nz * 8, cudaMemcpyDeviceToDevice,
                        x->s) != cudaSuccess)
      return PIC_E_CUDA;
  }
  if (cudaMemcpyAsync(&bad, x->gbad, sizeof(int), cudaMemcpyDeviceToHost, x->s) != cudaSuccess)
    return PIC_E_CUDA;
  int cnn_err = 0;
  if (x->guess_mode == PIC_GUESS_CNN &&
      cudaMemcpyAsync(&cnn_err, cnn_err_flag(x->cnn), sizeof(int), cudaMemcpyDeviceToHost, x->s) !=
          cudaSuccess)
    return PIC_E_CUDA;
  if (cudaStreamSynchronize(x->s) != cudaSuccess) return PIC_E_CUDA;
  if (cnn_err) return PIC_E_CUDA;  // a tensor-core kernel of the network gave up a wait
  if (!bad) *used = x->guess_mode;
  return PIC_OK;
}

// the nonlinear iteration of Sec. 2.1 from the start in er1/ez1: push + deposit
// with E^{n+1/2,k}, implicit field solve, relative-change test
//
// Speculative final pass: the commit push of a converged step repeats the last
// pass with the same E^{n+1/2}, so when the contraction of the last two
// residuals predicts that the next pass converges, that pass already writes
// the new particle state into the second buffer of the store (every field;
// wall tallies into scratch).  If it converges the buffers are swapped and
// the commit push is skipped (*spec = 1); if not, the iteration goes on.
// one Picard pass: E^{n+1/2,k}, push + deposit (speculative: writing the new
// state out of place), field solve, norms copied to pinned host memory
// the pass up to the push: E^{n+1/2,k} and alpha, cleared crossed charge
// (and, speculative, the counters and tallies the writing pass fills)
int enqueue_pre(pic_ctx *x, bool spec) {
  const int nr = x->g.nr, nz = x->g.nz;
  const size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz;
  const size_t nwall = (size_t)2 * (2 * (nr + 1) + nz + 1);
  cudaStream_t s = x->s;
  cudaError_t he =
      x->mixed ? launch_half_field_alpha(x->g, x->er, x->ez, x->er1, x->ez1, x->erh, x->ezh,
                                         x->alpha, s)
               : launch_half_field_alpha64(x->g, x->er, x->ez, x->er1, x->ez1, x->erh, x->ezh,
                                           x->alpha64, s);
  if (he != cudaSuccess) return PIC_E_CUDA;
  x->launches += 1;
  if (cudaMemsetAsync(x->ir, 0, ner * 8, s) != cudaSuccess) return PIC_E_CUDA;
  if (cudaMemsetAsync(x->iz, 0, nez * 8, s) != cudaSuccess) return PIC_E_CUDA;
  if (spec) {
    if (cudaMemsetAsync(x->cnt->push, 0, sizeof(x->cnt->push), s) != cudaSuccess ||
        cudaMemsetAsync(&x->cnt->ke_lost, 0, 8, s) != cudaSuccess ||
        cudaMemsetAsync(x->wall_spec, 0, nwall * 8, s) != cudaSuccess ||
        (x->hist_on && cudaMemsetAsync(x->hist_spec, 0, 16 * 8, s) != cudaSuccess))
      return PIC_E_CUDA;
  }
  return PIC_OK;
}

// the pass after the push: implicit field solve, norms to pinned host memory
int enqueue_post(pic_ctx *x) {
  cudaStream_t s = x->s;
  if (x->cfg.field_model == PIC_FIELD_ES) {
    // Q^{n+1} = Q^n - div I, E^{n+1} = -grad phi^{n+1}; H stays zero
    EsOp E = x->es;
    E.ez0 = x->ez;
    if (launch_es_solve(E, x->qn, x->ir, x->iz, 0.0, x->er2, x->ez2, x->er1, x->ez1, x->cnt,
                        s) != cudaSuccess)
      return PIC_E_CUDA;
    x->launches += x->circ_on ? 6 : 5;
  } else {
    if (launch_field_solve(x->F, x->er, x->ez, x->h, x->ir, x->iz, 0.0, 0.0, x->er2, x->ez2,
                           x->h2, x->er1, x->ez1, x->cnt, s) != cudaSuccess)
      return PIC_E_CUDA;
    x->launches += x->F.port.on ? 10 : 5;  // the axial port adds five kernels
  }
  // (a pass inside the device loop leaves the norms to its convergence test)
  if (!x->dl_capture &&
      cudaMemcpyAsync(x->hn, x->cnt->norm, 3 * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PIC_E_CUDA;
  return PIC_OK;
}

int enqueue_pass(pic_ctx *x, bool spec) {
  int r = enqueue_pre(x, spec);
  if (r) return r;
  if (spec)
    r = push_all(x, x->erh, x->ezh, x->ir, x->iz, 1, x->cnt->push, &x->cnt->ke_lost, x->wall_spec,
                 1);
  else
    r = push_all(x, x->erh, x->ezh, x->ir, x->iz, 0, nullptr, nullptr, nullptr);
  if (r) return r;
  return enqueue_post(x);
}

// the pass for the current buffers, replayed from a graph captured the first
// time this buffer configuration occurs (counts and voltages are read on the
// device, grids depend only on capacities)
int launch_pass(pic_ctx *x, bool spec) {
  // the first pass runs uncaptured (one-time set-up of launch shapes); the
  // legacy default stream cannot be captured, so its passes are never replayed
  if (!x->graphs || x->s == nullptr || x->passes++ == 0) return enqueue_pass(x, spec);
  // a speculative pass captures the sub-step histogram's memset and pointer
  // only while counting is on, so the switch is part of the key
  const void *key[13] = {x->er, x->ez, x->h, x->er1, x->ez1, x->er2, x->ez2, x->h2,
                         (const void *)(uintptr_t)x->cur[0], (const void *)(uintptr_t)x->cur[1],
                         (const void *)(uintptr_t)(spec ? 1 : 0), x->erh,
                         (const void *)(uintptr_t)(x->hist_on ? 1 : 0)};
  for (int k = 0; k < x->ngraph; ++k)
    if (!memcmp(x->gcache[k].key, key, sizeof(key)) && (!x->prof || x->gcache[k].ptimed)) {
      x->launches += x->gcache[k].nlaunch;
      if (x->prof) {
        x->rep_pe = x->gcache[k].pe;
        x->rep_npush = x->gcache[k].npush;
      }
      return cudaGraphLaunch(x->gcache[k].exec, x->s) == cudaSuccess ? PIC_OK : PIC_E_CUDA;
    }
  if (x->ngraph == 64) return enqueue_pass(x, spec);
  pic_ctx::GraphEntry &N = x->gcache[x->ngraph];
  N.ptimed = 0;
  N.npush = 0;
  if (x->prof) {
    if (cudaEventCreate(&N.pe[0]) != cudaSuccess) return PIC_E_CUDA;
    if (cudaEventCreate(&N.pe[1]) != cudaSuccess) {
      cudaEventDestroy(N.pe[0]);
      return PIC_E_CUDA;
    }
    N.ptimed = 1;
    x->cap_pe = N.pe;
    x->cap_npush = 0;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(x->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return PIC_E_CUDA;
  long long l0 = x->launches;
  x->capturing = 1;
  int r = enqueue_pass(x, spec);
  x->capturing = 0;
  x->cap_pe = nullptr;
  N.npush = x->cap_npush;
  cudaError_t e = cudaStreamEndCapture(x->s, &g);
  auto drop_events = [&]() {
    if (N.ptimed) {
      cudaEventDestroy(N.pe[0]);
      cudaEventDestroy(N.pe[1]);
      N.ptimed = 0;
    }
  };
  if (r) {
    if (g) cudaGraphDestroy(g);
    drop_events();
    return r;
  }
  if (e != cudaSuccess) {
    drop_events();
    return PIC_E_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    drop_events();
    return PIC_E_CUDA;
  }
  pic_ctx::GraphEntry &E = x->gcache[x->ngraph++];
  memcpy(E.key, key, sizeof(key));
  E.exec = ex;
  E.nlaunch = x->launches - l0;
  if (E.ptimed) {
    x->rep_pe = E.pe;
    x->rep_npush = E.npush;
  }
  return cudaGraphLaunch(ex, x->s) == cudaSuccess ? PIC_OK : PIC_E_CUDA;
}

// after the pass has completed: residual, buffer swap, convergence and the
// speculation decision for the next pass
void finish_pass(pic_ctx *x, int k, double &rprev, double &res, double &src, double &first,
                 bool &conv, bool &spec, int &spec_ok) {
  const double *hn = x->hn;
  res = sqrt(hn[0]) / fmax(sqrt(hn[1]), 1e-30);
  if (k == 0) first = res;
  src = hn[2];
  double *t;
  t = x->er1; x->er1 = x->er2; x->er2 = t;
  t = x->ez1; x->ez1 = x->ez2; x->ez2 = t;
  if (k > 0 && rprev > 0.0) x->rho_prev = res / rprev;
  if (res < x->cfg.picard_tol) {
    conv = true;
    spec_ok = spec ? 1 : 0;
    return;
  }
  const double rho = k > 0 ? res / rprev : x->rho_prev;
  spec = rho > 0.0 && rho < 1.0 && res * rho < x->cfg.picard_tol;
  rprev = res;
}

// ---- the Picard iteration on the device ---------------------------------------
// State of the loop in vdev[16..28] (doubles; read back once, after the loop):
enum {
  kPdK = 0,       // passes run
  kPdConv,        // 1: converged
  kPdSpec,        // 1: the next pass (after the test: the pass just run) is speculative
  kPdSpecOk,      // 1: the converged pass was the speculative one
  kPdNan,         // 1: the residual was not finite
  kPdRes,         // residual of the last pass
  kPdRprev,       // residual of the pass before (the contraction estimate)
  kPdFirst,       // residual of the first pass
  kPdSrc,         // drive energy of the last solve
  kPdRho,         // contraction rate carried between steps (pic_ctx::rho_prev)
  kPdTol,         // the Picard tolerance
  kPdKmax,        // the iteration limit
  kPdNspec,       // speculative passes run
  kPdSlots = 13
};
constexpr int kPdBase = 16;  // offset of the loop state in vdev

// The convergence test of one pass (the host loop's finish_pass, on the
// device): residual from the solve's norms, the speculation decision for the
// next pass, and the conditions of the while-node (go on) and of the if-node
// (the next pass speculative).  One thread.
__global__ void k_picard_ctl(cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hs,
                             const double *norm, double *pd) {
  const double res = sqrt(norm[0]) / fmax(sqrt(norm[1]), 1e-30);
  const int k = (int)pd[kPdK];
  const double rprev = pd[kPdRprev];
  const bool spec = pd[kPdSpec] != 0.0;
  if (k == 0) pd[kPdFirst] = res;
  pd[kPdRes] = res;
  pd[kPdSrc] = norm[2];
  if (spec) pd[kPdNspec] += 1.0;
  if (k > 0 && rprev > 0.0) pd[kPdRho] = res / rprev;
  unsigned go = 1, next_spec = 0;
  if (!isfinite(res)) {
    pd[kPdNan] = 1.0;
    go = 0;
  } else if (res < pd[kPdTol]) {
    pd[kPdConv] = 1.0;
    pd[kPdSpecOk] = spec ? 1.0 : 0.0;
    go = 0;
  } else {
    const double rho = k > 0 ? res / rprev : pd[kPdRho];
    next_spec = rho > 0.0 && rho < 1.0 && res * rho < pd[kPdTol];
    pd[kPdRprev] = res;
  }
  pd[kPdK] = (double)(k + 1);
  if (k + 1 >= (int)pd[kPdKmax]) go = 0;
  pd[kPdSpec] = next_spec ? 1.0 : 0.0;
  cudaGraphSetConditional(hw, go);
  cudaGraphSetConditional(hs, next_spec);
}

// capture one pass into a body graph of the loop (no dependencies: the first
// node of its branch); *nl = kernels in it
int capture_pass_into(pic_ctx *x, cudaGraph_t body, bool spec, long long *nl) {
  if (cudaStreamBeginCaptureToGraph(x->s, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return PIC_E_CUDA;
  const long long l0 = x->launches;
  x->capturing = 1;
  x->dl_capture = 1;
  const int r = enqueue_pass(x, spec);
  x->capturing = 0;
  x->dl_capture = 0;
  *nl = x->launches - l0;
  x->launches = l0;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(x->s, &g);
  if (r) return r;
  return e == cudaSuccess ? PIC_OK : PIC_E_CUDA;
}

// the loop graph of the current buffer configuration: while (go) { if (spec)
// speculative pass else plain pass; convergence test; er1/ez1 <- er2/ez2 }
// (the copy takes the place of the host loop's pointer swap, so that the
// captured passes keep their buffers)
int build_loop(pic_ctx *x, pic_ctx::LoopEntry &L) {
  const int nr = x->g.nr, nz = x->g.nz;
  const size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz;
  cudaGraph_t G = nullptr;
  if (cudaGraphCreate(&G, 0) != cudaSuccess) return PIC_E_CUDA;
  auto fail = [&](int r) {
    cudaGraphDestroy(G);
    return r;
  };
  cudaGraphConditionalHandle hw, hs;
  if (cudaGraphConditionalHandleCreate(&hw, G, 1, cudaGraphCondAssignDefault) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&hs, G, 0, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(PIC_E_CUDA);
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wn;
  if (cudaGraphAddNode(&wn, G, nullptr, nullptr, 0, &wp) != cudaSuccess) return fail(PIC_E_CUDA);
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hs;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 2;
  cudaGraphNode_t in;
  if (cudaGraphAddNode(&in, body, nullptr, nullptr, 0, &ip) != cudaSuccess)
    return fail(PIC_E_CUDA);
  int r = capture_pass_into(x, ip.conditional.phGraph_out[0], true, &L.nl_spec);
  if (!r) r = capture_pass_into(x, ip.conditional.phGraph_out[1], false, &L.nl_plain);
  if (r) return fail(r);
  if (cudaStreamBeginCaptureToGraph(x->s, body, &in, nullptr, 1,
                                    cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(PIC_E_CUDA);
  k_picard_ctl<<<1, 1, 0, x->s>>>(hw, hs, x->cnt->norm, x->vdev + kPdBase);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(x->er1, x->er2, ner * 8, cudaMemcpyDeviceToDevice, x->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x->ez1, x->ez2, nez * 8, cudaMemcpyDeviceToDevice, x->s);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(x->s, &g);
  if (e != cudaSuccess || ee != cudaSuccess) return fail(PIC_E_CUDA);
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, G, 0) != cudaSuccess) return fail(PIC_E_CUDA);
  L.graph = G;
  L.exec = ex;
  return PIC_OK;
}

// The iteration as one graph launch and one wait.  *handled = false when it
// does not apply (no graphs, timing on, the uncaptured first pass, a full
// cache, a failed build): the host loop runs instead.
int picard_device(pic_ctx *x, pic_step_stats &S, bool &conv, int &k, double &res, double &src,
                  double &first, int &spec_ok, bool &handled) {
  handled = false;
  if (!x->dloop || !x->graphs || x->s == nullptr || x->prof || x->passes == 0) return PIC_OK;
  const void *key[12] = {x->er, x->ez, x->h, x->er1, x->ez1, x->er2, x->ez2, x->h2,
                         (const void *)(uintptr_t)x->cur[0], (const void *)(uintptr_t)x->cur[1],
                         x->erh, (const void *)(uintptr_t)(x->hist_on ? 1 : 0)};
  pic_ctx::LoopEntry *L = nullptr;
  for (int i = 0; i < x->nloop; ++i)
    if (!memcmp(x->lcache[i].key, key, sizeof(key))) L = &x->lcache[i];
  if (!L) {
    if (x->nloop == 32) return PIC_OK;
    pic_ctx::LoopEntry &N = x->lcache[x->nloop];
    if (build_loop(x, N)) {
      // not available here (e.g. a driver without conditional nodes): the
      // host loop from now on; a capture left open would poison the stream
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(x->s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(x->s, &g);
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();
      x->dloop = 0;
      return PIC_OK;
    }
    memcpy(N.key, key, sizeof(key));
    L = &N;
    x->nloop += 1;
  }
  handled = true;
  // pageable source: staged before the call returns
  double pd[kPdSlots] = {};
  pd[kPdRho] = x->rho_prev;
  pd[kPdTol] = x->cfg.picard_tol;
  pd[kPdKmax] = (double)x->cfg.picard_max;
  double *dpd = x->vdev + kPdBase;
  if (cudaMemcpyAsync(dpd, pd, sizeof(pd), cudaMemcpyHostToDevice, x->s) != cudaSuccess)
    return PIC_E_CUDA;
  if (cudaGraphLaunch(L->exec, x->s) != cudaSuccess) return PIC_E_CUDA;
  if (cudaMemcpyAsync(x->hn + kHnLoop, dpd, sizeof(pd), cudaMemcpyDeviceToHost, x->s) !=
      cudaSuccess)
    return PIC_E_CUDA;
  if (cudaStreamSynchronize(x->s) != cudaSuccess) return PIC_E_CUDA;
  memcpy(pd, x->hn + kHnLoop, sizeof(pd));
  const int passes = (int)pd[kPdK], nspec = (int)pd[kPdNspec];
  x->passes += passes;
  x->launches += (long long)(passes - nspec) * L->nl_plain + (long long)nspec * L->nl_spec + passes;
  S.pushes += (long long)passes * (x->n[0] + x->n[1]);
  x->rho_prev = pd[kPdRho];
  res = pd[kPdRes];
  src = pd[kPdSrc];
  first = pd[kPdFirst];
  conv = pd[kPdConv] != 0.0;
  spec_ok = conv && pd[kPdSpecOk] != 0.0 ? 1 : 0;
  k = conv ? passes - 1 : passes;
  if (pd[kPdNan] != 0.0) {
    S.picard_iters = passes;
    return PIC_E_NAN;
  }
  return PIC_OK;
}

// the nonlinear iteration of Sec. 2.1 from the start in er1/ez1: push + deposit
// with E^{n+1/2,k}, implicit field solve, relative-change test
//
// Speculative final pass: the commit push of a converged step repeats the last
// pass with the same E^{n+1/2}, so when the contraction of the last two
// residuals predicts that the next pass converges, that pass already writes
// the new particle state into the second buffer of the store (every field;
// wall tallies into scratch).  If it converges the buffers are swapped and
// the commit push is skipped (*spec = 1); if not, the iteration goes on.
int picard(pic_ctx *x, double v0, double v1, pic_step_stats &S, bool &conv, int &k, double &res,
           double &src, double &first, int &spec_ok) {
  (void)v0;
  (void)v1;
  conv = false;
  res = 0.0;
  src = 0.0;
  first = 0.0;
  spec_ok = 0;
  bool handled = false;
  const int dr = picard_device(x, S, conv, k, res, src, first, spec_ok, handled);
  if (handled) return dr;
  bool spec = false;
  double rprev = 0.0;
  for (k = 0; k < x->cfg.picard_max; ++k) {
    int r = launch_pass(x, spec);
    if (r) return r;
    S.pushes += x->n[0] + x->n[1];
    if (cudaStreamSynchronize(x->s) != cudaSuccess) return PIC_E_CUDA;
    if (x->prof) prof_collect(x);
    finish_pass(x, k, rprev, res, src, first, conv, spec, spec_ok);
    if (!isfinite(res)) {
      S.picard_iters = k + 1;
      return PIC_E_NAN;
    }
    if (conv) break;
  }
  return PIC_OK;
}

__global__ void k_addto(double *dst, const double *src, int n) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] += src[t];
}
__global__ void k_addto_u64(unsigned long long *dst, const unsigned long long *src, int n) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] += src[t];
}

}  // namespace

namespace {

// state of one step between its phases (shared by pic_step and the ensemble)
struct StepState {
  pic_step_stats S;
  long long l0;
  double v0, v1;
  int used;          // Picard start
  bool conv, spec;   // converged; the next pass is speculative
  int k, spec_ok;
  double res, src, first, rprev;
};

// upload counts and voltages, choose and place the Picard start
int step_begin(pic_ctx *x, StepState &T) {
  memset(&T, 0, sizeof(T));
  T.l0 = x->launches;
  T.v0 = volt_at(x, x->step);
  T.v1 = volt_at(x, x->step + 1);
  if (upload_step(x, T.v0, T.v1)) return PIC_E_CUDA;
  if (x->cfg.field_model == PIC_FIELD_ES && !x->qn_valid) {
    // node charge of the particles, once; the steps then carry it by continuity
    const size_t nn = (size_t)(x->g.nr + 1) * (x->g.nz + 1);
    if (cudaMemsetAsync(x->qn, 0, nn * 8, x->s) != cudaSuccess) return PIC_E_CUDA;
    for (int sp = 0; sp < 2; ++sp) {
      const double q = sp == 0 ? -kQE : kQE;
      cudaError_t e = x->mixed ? launch_node_charge(x->g, as32(cur(x, sp)), x->n[sp], q, x->qn, x->s)
                               : launch_node_charge(x->g, cur(x, sp), x->n[sp], q, x->qn, x->s);
      if (e != cudaSuccess) return PIC_E_CUDA;
    }
    x->launches += 2;
    x->qn_valid = 1;
  }
  T.used = PIC_GUESS_PLAIN;
  x->feat_now = 0;
  if (x->guess_mode != PIC_GUESS_PLAIN && x->hist_n >= 4) {
    int gr = guess_start(x, T.v1, &T.used);
    if (gr) return gr;
  }
  if (T.used == PIC_GUESS_PLAIN) return plain_start(x, T.v1);
  return PIC_OK;
}

// commit (or adopt the speculative pass), field rotation, guess history, MCC,
// sort and statistics; *rc collects non-fatal codes
int step_end(pic_ctx *x, StepState &T, int *rc) {
  pic_step_stats &S = T.S;
  const int nr = x->g.nr, nz = x->g.nz;
  const size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz;
  cudaStream_t s = x->s;
  S.guess = T.used;
  S.first_res = T.first;
  S.spec_final = T.spec_ok;
  S.picard_iters = T.conv ? T.k + 1 : T.k;
  S.last_res = T.res;
  S.converged = T.conv ? 1 : 0;
  if (!T.conv) {
    S.n[0] = x->n[0];
    S.n[1] = x->n[1];
    return PIC_E_NOCONV;
  }
  if (T.spec_ok) {
    // the converged pass already wrote the new state into the second buffer
    x->cur[0] ^= 1;
    if (!x->cfg.ions_fixed) x->cur[1] ^= 1;
    const int nwall = 2 * (2 * (nr + 1) + nz + 1);
    k_addto<<<(nwall + 255) / 256, 256, 0, s>>>(x->wall, x->wall_spec, nwall);
    if (cudaGetLastError() != cudaSuccess) return PIC_E_CUDA;
    x->launches += 1;
    if (x->hist_on) {
      k_addto_u64<<<1, 16, 0, s>>>(x->hist, x->hist_spec, 16);
      if (cudaGetLastError() != cudaSuccess) return PIC_E_CUDA;
      x->launches += 1;
    }
  } else {
    // commit: the half field of the last iteration fed the last solve
    if (cudaMemsetAsync(x->ir, 0, ner * 8, s) != cudaSuccess) return PIC_E_CUDA;
    if (cudaMemsetAsync(x->iz, 0, nez * 8, s) != cudaSuccess) return PIC_E_CUDA;
    if (cudaMemsetAsync(x->cnt->push, 0, sizeof(x->cnt->push), s) != cudaSuccess)
      return PIC_E_CUDA;
    if (cudaMemsetAsync(&x->cnt->ke_lost, 0, 8, s) != cudaSuccess) return PIC_E_CUDA;
    int r = push_all(x, x->erh, x->ezh, x->ir, x->iz, 1, x->cnt->push, &x->cnt->ke_lost, x->wall);
    if (r) return r;
    S.pushes += x->n[0] + x->n[1];
  }
  if (x->circ_on) {
    if (launch_circuit_commit(x->F.cc, x->vdev, s) != cudaSuccess) return PIC_E_CUDA;
    x->launches += 1;
  }
  if (x->g.sgd > 0.0) {
    // charge moved by the conducting ring's current over the committed step
    if (launch_conduction(x->g, x->cfg.dt, x->er, x->ez, x->er1, x->ez1, x->qc, s) != cudaSuccess)
      return PIC_E_CUDA;
    x->launches += 1;
  }
  if (x->cfg.field_model == PIC_FIELD_ES) {
    // Q^{n+1} = Q^n - div I of the committed step (ionization pairs are neutral)
    if (launch_es_advance(x->es, x->qn, x->ir, x->iz, s) != cudaSuccess) return PIC_E_CUDA;
    x->launches += 1;
  }
  double *t;
  t = x->er; x->er = x->er1; x->er1 = t;
  t = x->ez; x->ez = x->ez1; x->ez1 = t;
  t = x->h; x->h = x->h2; x->h2 = t;
  if (x->F.port.on) {
    // the port's fields of the last solve (fixed buffers: the captured passes stay valid)
    const PortOp &P = x->F.port;
    const size_t nzz = (size_t)(P.m + 1) * P.nzp;
    if (cudaMemcpyAsync(x->hp, x->hp2, (size_t)P.np * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(x->erp, x->erp2, (size_t)P.np * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(x->ezp, x->ezp2, nzz * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return PIC_E_CUDA;
  }
  if (x->guess_mode != PIC_GUESS_PLAIN) {
    // training target of this step, then E^n joins the history (its buffer
    // is now er1/ez1) and the committed crossed charge is kept
    if (x->feat_now) {
      GuessArgs A = guess_args(x);
      if (launch_guess_target(A, x->er, x->ez, x->gt, s) != cudaSuccess) return PIC_E_CUDA;
      x->launches += 1;
      x->sample_valid = 1;
    }
    t = x->hr[2]; x->hr[2] = x->hr[1]; x->hr[1] = x->hr[0]; x->hr[0] = x->er1; x->er1 = t;
    t = x->hz[2]; x->hz[2] = x->hz[1]; x->hz[1] = x->hz[0]; x->hz[0] = x->ez1; x->ez1 = t;
    if (cudaMemcpyAsync(x->jr, x->ir, ner * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(x->jz, x->iz, nez * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return PIC_E_CUDA;
    if (x->hist_n < 4) x->hist_n += 1;
  }
  S.src_energy = T.src;
  if (x->cfg.mcc_on) {
    int mr = mcc_run(x, (unsigned long long)x->step, S.mcc, nullptr);
    if (mr && mr != PIC_E_CAPACITY) return mr;
    if (mr) *rc = mr;
  }
  // step counters and the sort's counts: one wait
  if (x->circ_on &&
      cudaMemcpyAsync(x->hn + kHnCirc, x->vdev + 4, 32, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PIC_E_CUDA;
  if (cudaMemcpyAsync(x->hn + kHnPush, x->cnt->push, 40, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PIC_E_CUDA;
  if (cudaMemcpyAsync(x->hn + kHnKel, &x->cnt->ke_lost, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PIC_E_CUDA;
  if (x->cfg.mcc_on &&
      cudaMemcpyAsync(x->hn + kHnDe, &x->cnt->de_coll, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PIC_E_CUDA;
  int sr = sort_enqueue(x);
  if (sr) return sr;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_E_CUDA;
  sort_finish(x);
  unsigned long long pc[5];
  double kel = 0.0;
  double cst[4] = {0.0, 0.0, T.v1, 0.0};
  memcpy(pc, x->hn + kHnPush, 40);
  memcpy(&kel, x->hn + kHnKel, 8);
  if (x->circ_on) memcpy(cst, x->hn + kHnCirc, 32);
  if (x->cfg.mcc_on) memcpy(&S.de_coll, x->hn + kHnDe, 8);
  if (x->prof) prof_collect(x);
  S.substep_err = (long long)pc[0];
  S.absorbed = (long long)pc[1];
  S.substeps = (long long)pc[2];
  S.fallbacks = (long long)pc[3];
  S.push_flops = (long long)pc[4];
  S.ke_lost = kel;
  S.q_cap = cst[0];
  S.v_electrode = cst[2];
  S.n[0] = x->n[0];
  S.n[1] = x->n[1];
  if (x->diag_on) {
    // the committed step's crossed charge is still in ir / iz
    int dr = diag_step(x, 0);
    if (dr) return dr;
  }
  S.launches = x->launches - T.l0;
  x->step += 1;
  if (S.substep_err && !*rc) *rc = PIC_E_SUBSTEP;
  return PIC_OK;
}

}  // namespace

int pic_step(pic_ctx *x, int nsteps, pic_step_stats *st) {
  if (!x || nsteps < 0) return PIC_E_CONFIG;
  int rc = PIC_OK;
  for (int it = 0; it < nsteps; ++it) {
    StepState T;
    int r = step_begin(x, T);
    if (r) return r;
    int pr = picard(x, T.v0, T.v1, T.S, T.conv, T.k, T.res, T.src, T.first, T.spec_ok);
    if (!T.conv && T.used != PIC_GUESS_PLAIN && (pr == PIC_OK || pr == PIC_E_NAN)) {
      // the plain start remains the fallback: redo the iteration from E^n
      T.used = PIC_GUESS_PLAIN;
      pr = plain_start(x, T.v1);
      if (!pr) pr = picard(x, T.v0, T.v1, T.S, T.conv, T.k, T.res, T.src, T.first, T.spec_ok);
    }
    if (pr) {
      T.S.guess = T.used;
      T.S.first_res = T.first;
      if (st) *st = T.S;
      return pr;
    }
    r = step_end(x, T, &rc);
    if (st) *st = T.S;
    if (r) return r;
  }
  return rc;
}

int pic_diag(pic_ctx *x, pic_diag_out *out) {
  if (!x || !out) return PIC_E_CONFIG;
  cudaError_t e = cudaMemsetAsync(x->diag, 0, 8 * 8, x->s);
  if (e == cudaSuccess)
    e = x->mixed ? launch_kinetic(as32(cur(x, 0)), x->n[0], kME, -kQE, x->diag, x->s)
                 : launch_kinetic(cur(x, 0), x->n[0], kME, -kQE, x->diag, x->s);
  x->launches += 3;
  if (e == cudaSuccess)
    e = x->mixed ? launch_kinetic(as32(cur(x, 1)), x->n[1], kMAr, kQE, x->diag + 2, x->s)
                 : launch_kinetic(cur(x, 1), x->n[1], kMAr, kQE, x->diag + 2, x->s);
  if (e == cudaSuccess)
    e = launch_field_energy(x->g, x->eps, x->mu, x->er, x->ez, x->h, x->diag + 4, x->s);
  double h[8];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, x->diag, 64, cudaMemcpyDeviceToHost, x->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  if (e != cudaSuccess) return PIC_E_CUDA;
  out->kinetic[0] = h[0];
  out->charge[0] = h[1];
  out->kinetic[1] = h[2];
  out->charge[1] = h[3];
  out->field = h[4];
  out->n[0] = x->n[0];
  out->n[1] = x->n[1];
  return PIC_OK;
}

int pic_diag_average(pic_ctx *x, int enable) {
  if (!x || enable < 0 || enable > 1) return PIC_E_CONFIG;
  if (!enable) {
    x->diag_on = 0;
    return PIC_OK;
  }
  const size_t nn = (size_t)(x->g.nr + 1) * (x->g.nz + 1);
  const size_t nwall = (size_t)2 * (2 * (x->g.nr + 1) + x->g.nz + 1);
  if (cudaMemsetAsync(x->dacc, 0, 2 * nn * 8, x->s) != cudaSuccess ||
      cudaMemcpyAsync(x->wall0, x->wall, nwall * 8, cudaMemcpyDeviceToDevice, x->s) != cudaSuccess)
    return PIC_E_CUDA;
  x->diag_steps = 0;
  x->cres_valid = 0;
  int r = diag_step(x, 1);
  if (r) return r;
  x->diag_on = 1;
  return PIC_OK;
}

int pic_diag_get(pic_ctx *x, int kind, void *dst, size_t bytes, int dst_is_device) {
  if (!x || !dst) return PIC_E_CONFIG;
  const int nr = x->g.nr, nz = x->g.nz;
  const size_t nn = (size_t)(nr + 1) * (nz + 1);
  const size_t ner = (size_t)nr * (nz + 1), nez = (size_t)(nr + 1) * nz, nh = (size_t)nr * nz;
  const size_t nwall = (size_t)2 * (2 * (nr + 1) + nz + 1);
  cudaStream_t s = x->s;
  const cudaMemcpyKind to = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  auto finish = [&]() { return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : PIC_E_CUDA; };
  // host-computed results go out through this buffer
  std::vector<double> hv;
  auto put_host = [&](const void *src, size_t nb) -> int {
    if (dst_is_device) {
      if (cudaMemcpyAsync(dst, src, nb, cudaMemcpyHostToDevice, s) != cudaSuccess) return PIC_E_CUDA;
      return finish();
    }
    memcpy(dst, src, nb);
    return PIC_OK;
  };
  // dual volume / electrode area of a node: the ring between the neighbouring
  // cell centres (the axis disc, the half ring at r = R), times the z extent
  auto ring = [&](int i) {
    const double lo = i == 0 ? 0.0 : g_rcentre(x->g, i - 1);
    const double hi = i == nr ? g_rnode(x->g, nr) : g_rcentre(x->g, i);
    return kPi * (hi * hi - lo * lo);
  };
  switch (kind) {
    case PIC_DIAG_ENERGY: {
      if (dst_is_device || bytes < sizeof(pic_diag_out)) return PIC_E_CONFIG;
      return pic_diag(x, (pic_diag_out *)dst);
    }
    case PIC_DIAG_GAUSS: {
      if (bytes < nn * 8) return PIC_E_CONFIG;
      int r = pic_gauss_residual(x, x->dcnt);
      if (r) return r;
      if (cudaMemcpyAsync(dst, x->dcnt, nn * 8, to, s) != cudaSuccess) return PIC_E_CUDA;
      return finish();
    }
    case PIC_DIAG_CONTINUITY: {
      if (bytes < nn * 8) return PIC_E_CONFIG;
      if (!x->cres_valid) return PIC_E_STATE;
      if (cudaMemcpyAsync(dst, x->cres, nn * 8, to, s) != cudaSuccess) return PIC_E_CUDA;
      return finish();
    }
    case PIC_DIAG_DENSITY_AVG: {
      if (bytes < 2 * nn * 8) return PIC_E_CONFIG;
      if (x->diag_steps < 1) return PIC_E_STATE;
      hv.resize(2 * nn);
      if (cudaMemcpyAsync(hv.data(), x->dacc, 2 * nn * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PIC_E_CUDA;
      int r = finish();
      if (r) return r;
      for (int i = 0; i <= nr; ++i) {
        const double a = ring(i);
        for (int j = 0; j <= nz; ++j) {
          const double v = a * ((j == 0 || j == nz) ? 0.5 : 1.0) * x->g.dz;
          for (int sp = 0; sp < 2; ++sp) {
            double &d = hv[sp * nn + (size_t)i * (nz + 1) + j];
            d = d / ((double)x->diag_steps * v);
          }
        }
      }
      return put_host(hv.data(), 2 * nn * 8);
    }
    case PIC_DIAG_ION_FLUX_AVG: {
      if (bytes < 2 * (size_t)(nr + 1) * 8) return PIC_E_CONFIG;
      if (x->diag_steps < 1) return PIC_E_STATE;
      std::vector<double> w1(nwall), w0(nwall);
      if (cudaMemcpyAsync(w1.data(), x->wall, nwall * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemcpyAsync(w0.data(), x->wall0, nwall * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PIC_E_CUDA;
      int r = finish();
      if (r) return r;
      const size_t blk = 2 * (size_t)(nr + 1) + nz + 1;  // ions: the second species block
      const double tw = (double)x->diag_steps * x->cfg.dt;
      hv.resize(2 * (size_t)(nr + 1));
      for (int e = 0; e < 2; ++e)
        for (int i = 0; i <= nr; ++i) {
          const size_t k = blk + (size_t)e * (nr + 1) + i;
          hv[(size_t)e * (nr + 1) + i] = (w1[k] - w0[k]) / (kQE * tw * ring(i));
        }
      return put_host(hv.data(), hv.size() * 8);
    }
    case PIC_DIAG_FIELDS: {
      const size_t nb = (ner + nez + nh) * 8;
      if (bytes < nb) return PIC_E_CONFIG;
      char *d = (char *)dst;
      if (cudaMemcpyAsync(d, x->er, ner * 8, to, s) != cudaSuccess ||
          cudaMemcpyAsync(d + ner * 8, x->ez, nez * 8, to, s) != cudaSuccess ||
          cudaMemcpyAsync(d + (ner + nez) * 8, x->h, nh * 8, to, s) != cudaSuccess)
        return PIC_E_CUDA;
      return finish();
    }
    case PIC_DIAG_COUNTS: {
      if (bytes < 4 * sizeof(long long)) return PIC_E_CONFIG;
      const long long c[4] = {x->n[0], x->n[1], x->step, x->diag_steps};
      if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_E_CUDA;
      return put_host(c, sizeof(c));
    }
    default:
      return PIC_E_CONFIG;
  }
}

int pic_node_charge(pic_ctx *x, double *q) {
  if (!x || !q) return PIC_E_CONFIG;
  cudaError_t e;
  if (x->mixed) {
    e = launch_node_charge(x->g, as32(cur(x, 0)), x->n[0], -kQE, q, x->s);
    if (e == cudaSuccess) e = launch_node_charge(x->g, as32(cur(x, 1)), x->n[1], kQE, q, x->s);
  } else {
    e = launch_node_charge(x->g, cur(x, 0), x->n[0], -kQE, q, x->s);
    if (e == cudaSuccess) e = launch_node_charge(x->g, cur(x, 1), x->n[1], kQE, q, x->s);
  }
  return cuda_rc(e);
}

int pic_gauss_residual(pic_ctx *x, double *res) {
  if (!x || !res) return PIC_E_CONFIG;
  const size_t nn = (size_t)(x->g.nr + 1) * (x->g.nz + 1);
  if (cudaMemsetAsync(res, 0, nn * 8, x->s) != cudaSuccess) return PIC_E_CUDA;
  int r = pic_node_charge(x, res);
  if (r) return r;
  x->launches += 3;
  return cuda_rc(launch_gauss_residual(x->g, x->eps, x->er, x->ez, x->wall,
                                       x->g.sgd > 0.0 ? x->qc : nullptr, res, x->s));
}

int pic_get_view(pic_ctx *x, pic_view *v) {
  if (!x || !v) return PIC_E_CONFIG;
  for (int s = 0; s < 2; ++s) {
    Parts &P = cur(x, s);
    v->cell[s] = P.cell;
    v->a[s] = (void *)P.a;
    v->b[s] = (void *)P.b;
    v->vr[s] = (void *)P.vr;
    v->vt[s] = (void *)P.vt;
    v->vz[s] = (void *)P.vz;
    v->w[s] = (void *)P.w;
    v->id[s] = P.id;
    v->n[s] = x->n[s];
    v->cap[s] = x->cap[s];
    v->next_id[s] = x->next_id[s];
  }
  v->er = x->er;
  v->ez = x->ez;
  v->h = x->h;
  v->step = x->step;
  v->real_size = x->mixed ? 4 : 8;
  v->wall = x->wall;
  v->qcond = x->qc;
  if (x->F.port.on) {
    v->port_h = x->hp;
    v->port_er = x->erp;
    v->port_ez = x->ezp;
    v->port_m = x->F.port.m;
    v->port_cells = x->F.port.nzp;
  } else {
    v->port_h = v->port_er = v->port_ez = nullptr;
    v->port_m = v->port_cells = 0;
  }
  return PIC_OK;
}

namespace {

// checkpoint header (little-endian host layout, version 1)
struct CkptHeader {
  char magic[8];
  int32_t version, nr, nz, precision, field_model, real_size, circ_on, qn_valid, nharm, xa;
  long long n[2], step;
  uint32_t next_id[2];
  double circ[4], rho_prev;
  double hamp[64], hfreq[64], hph[64];
  int32_t ring_cells, conducting;  // the ring's extent and whether it carries a conduction tally
  int32_t port_m, port_cells;      // the axial port's extent (0, 0: none)
};
const char kCkptMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '1'};

// the device arrays of a checkpoint, in file order
extern "C++" template <typename F>
int ckpt_arrays(pic_ctx *x, const long long n[2], F &&f) {
  const int nr = x->g.nr, nz = x->g.nz;
  const size_t rs = x->mixed ? 4 : 8;
  for (int s = 0; s < 2; ++s) {
    Parts &P = cur(x, s);
    void *arr[8] = {P.cell, P.a, P.b, P.vr, P.vt, P.vz, P.w, P.id};
    for (int k = 0; k < 8; ++k) {
      const size_t es = (k == 0 || k == 7) ? 4 : rs;
      if (int r = f(arr[k], (size_t)n[s] * es)) return r;
    }
  }
  if (int r = f(x->er, (size_t)nr * (nz + 1) * 8)) return r;
  if (int r = f(x->ez, (size_t)(nr + 1) * nz * 8)) return r;
  if (int r = f(x->h, (size_t)nr * nz * 8)) return r;
  if (int r = f(x->wall, (size_t)2 * (2 * (nr + 1) + nz + 1) * 8)) return r;
  if (x->cfg.field_model == PIC_FIELD_ES)
    if (int r = f(x->qn, (size_t)(nr + 1) * (nz + 1) * 8)) return r;
  if (x->g.sgd > 0.0)
    if (int r = f(x->qc, (size_t)(nr + 1) * (nz + 1) * 8)) return r;
  if (x->F.port.on) {
    const PortOp &P = x->F.port;
    if (int r = f(x->hp, (size_t)P.np * 8)) return r;
    if (int r = f(x->erp, (size_t)P.np * 8)) return r;
    if (int r = f(x->ezp, (size_t)(P.m + 1) * P.nzp * 8)) return r;
  }
  return PIC_OK;
}

}  // namespace

int pic_save(pic_ctx *x, const char *path) {
  if (!x || !path) return PIC_E_CONFIG;
  CkptHeader H;
  memset(&H, 0, sizeof(H));
  memcpy(H.magic, kCkptMagic, 8);
  H.version = 3;
  H.port_m = x->F.port.on ? x->F.port.m : 0;
  H.port_cells = x->F.port.on ? x->F.port.nzp : 0;
  H.nr = x->g.nr;
  H.nz = x->g.nz;
  H.precision = x->cfg.precision;
  H.field_model = x->cfg.field_model;
  H.real_size = x->mixed ? 4 : 8;
  H.circ_on = x->circ_on;
  H.qn_valid = x->qn_valid;
  H.nharm = x->nharm;
  H.xa = x->g.xa;
  H.ring_cells = x->g.nd;
  H.conducting = x->g.sgd > 0.0 ? 1 : 0;
  H.n[0] = x->n[0];
  H.n[1] = x->n[1];
  H.step = x->step;
  H.next_id[0] = x->next_id[0];
  H.next_id[1] = x->next_id[1];
  H.rho_prev = x->rho_prev;
  for (int k = 0; k < 64; ++k) {
    H.hamp[k] = x->hamp[k];
    H.hfreq[k] = x->hfreq[k];
    H.hph[k] = x->hph[k];
  }
  if (cudaStreamSynchronize(x->s) != cudaSuccess) return PIC_E_CUDA;
  if (x->circ_on && cudaMemcpy(H.circ, x->vdev + 4, 32, cudaMemcpyDeviceToHost) != cudaSuccess)
    return PIC_E_CUDA;
  FILE *fp = fopen(path, "wb");
  if (!fp) return PIC_E_IO;
  int rc = fwrite(&H, sizeof(H), 1, fp) == 1 ? PIC_OK : PIC_E_IO;
  std::vector<char> buf;
  if (!rc)
    rc = ckpt_arrays(x, H.n, [&](void *dev, size_t bytes) {
      if (!bytes) return PIC_OK;
      buf.resize(bytes);
      if (cudaMemcpy(buf.data(), dev, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return PIC_E_CUDA;
      return fwrite(buf.data(), 1, bytes, fp) == bytes ? PIC_OK : PIC_E_IO;
    });
  if (fclose(fp) != 0 && !rc) rc = PIC_E_IO;
  return rc;
}

int pic_load(pic_ctx *x, const char *path) {
  if (!x || !path) return PIC_E_CONFIG;
  FILE *fp = fopen(path, "rb");
  if (!fp) return PIC_E_IO;
  CkptHeader H;
  int rc = fread(&H, sizeof(H), 1, fp) == 1 ? PIC_OK : PIC_E_IO;
  if (!rc && (memcmp(H.magic, kCkptMagic, 8) != 0 || H.version != 3 || H.nharm < 0 ||
              H.nharm > 64))
    rc = PIC_E_IO;
  if (!rc && (H.nr != x->g.nr || H.nz != x->g.nz || H.precision != x->cfg.precision ||
              H.field_model != x->cfg.field_model || H.xa != x->g.xa ||
              H.ring_cells != x->g.nd || H.conducting != (x->g.sgd > 0.0 ? 1 : 0) ||
              H.port_m != (x->F.port.on ? x->F.port.m : 0) ||
              H.port_cells != (x->F.port.on ? x->F.port.nzp : 0) ||
              H.real_size != (x->mixed ? 4 : 8) || H.n[0] < 0 || H.n[1] < 0 ||
              H.n[0] > x->cap[0] || H.n[1] > x->cap[1] || H.step < 0 ||
              (H.circ_on != 0) != (x->circ_on != 0)))
    rc = PIC_E_STATE;
  std::vector<char> buf;
  if (!rc && cudaStreamSynchronize(x->s) != cudaSuccess) rc = PIC_E_CUDA;
  if (!rc)
    rc = ckpt_arrays(x, H.n, [&](void *dev, size_t bytes) {
      if (!bytes) return PIC_OK;
      buf.resize(bytes);
      if (fread(buf.data(), 1, bytes, fp) != bytes) return PIC_E_IO;
      return cudaMemcpy(dev, buf.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess
                 ? PIC_OK
                 : PIC_E_CUDA;
    });
  fclose(fp);
  if (rc) return rc;
  if (x->circ_on && cudaMemcpy(x->vdev + 4, H.circ, 32, cudaMemcpyHostToDevice) != cudaSuccess)
    return PIC_E_CUDA;
  x->n[0] = H.n[0];
  x->n[1] = H.n[1];
  x->next_id[0] = H.next_id[0];
  x->next_id[1] = H.next_id[1];
  x->step = H.step;
  x->rho_prev = H.rho_prev;
  x->qn_valid = H.qn_valid;
  x->nharm = H.nharm;
  for (int k = 0; k < 64; ++k) {
    x->hamp[k] = H.hamp[k];
    x->hfreq[k] = H.hfreq[k];
    x->hph[k] = H.hph[k];
  }
  x->hist_n = 1;
  x->sample_valid = 0;
  return PIC_OK;
}

int pic_substep_histogram(pic_ctx *x, int enable, unsigned long long *counts) {
  if (!x || enable < -1 || enable > 1) return PIC_E_CONFIG;
  if (counts) {
    if (cudaMemcpyAsync(counts, x->hist, 16 * 8, cudaMemcpyDeviceToHost, x->s) != cudaSuccess ||
        cudaStreamSynchronize(x->s) != cudaSuccess)
      return PIC_E_CUDA;
  }
  if (enable == 1 && cudaMemsetAsync(x->hist, 0, 16 * 8, x->s) != cudaSuccess) return PIC_E_CUDA;
  if (enable >= 0) x->hist_on = enable;
  return PIC_OK;
}

int pic_state_upload(pic_ctx *x, const pic_host_state *in) {
  if (!x || !in) return PIC_E_CONFIG;
  for (int s = 0; s < 2; ++s) {
    if (in->n[s] < 0 || in->n[s] > x->cap[s]) return PIC_E_STATE;
    if (in->n[s] > 0 && (!in->cell[s] || !in->a[s] || !in->b[s] || !in->vr[s] || !in->vt[s] ||
                         !in->vz[s] || !in->w[s] || !in->id[s]))
      return PIC_E_CONFIG;
  }
  if (in->step < 0) return PIC_E_STATE;
  const size_t rs = x->mixed ? 4 : 8;
  const int nr = x->g.nr, nz = x->g.nz;
  cudaStream_t st = x->s;
  cudaError_t e = cudaSuccess;
  auto up = [&](void *dst, const void *src, size_t b) {
    if (e == cudaSuccess && b) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, st);
  };
  for (int s = 0; s < 2; ++s) {
    Parts &P = cur(x, s);
    const size_t n = (size_t)in->n[s];
    up(P.cell, in->cell[s], n * 4);
    up(P.a, in->a[s], n * rs);
    up(P.b, in->b[s], n * rs);
    up(P.vr, in->vr[s], n * rs);
    up(P.vt, in->vt[s], n * rs);
    up(P.vz, in->vz[s], n * rs);
    up(P.w, in->w[s], n * rs);
    up(P.id, in->id[s], n * 4);
  }
  if (in->er) up(x->er, in->er, (size_t)nr * (nz + 1) * 8);
  if (in->ez) up(x->ez, in->ez, (size_t)(nr + 1) * nz * 8);
  if (in->h) up(x->h, in->h, (size_t)nr * nz * 8);
  if (e != cudaSuccess) return PIC_E_CUDA;
  return pic_set_counts(x, in->n[0], in->n[1], in->next_id[0], in->next_id[1], in->step);
}

int pic_state_download(pic_ctx *x, pic_host_state *out) {
  if (!x || !out) return PIC_E_CONFIG;
  for (int s = 0; s < 2; ++s) {
    if (out->n[s] < x->n[s]) return PIC_E_STATE;
    if (x->n[s] > 0 && (!out->cell[s] || !out->a[s] || !out->b[s] || !out->vr[s] ||
                        !out->vt[s] || !out->vz[s] || !out->w[s] || !out->id[s]))
      return PIC_E_CONFIG;
  }
  const size_t rs = x->mixed ? 4 : 8;
  const int nr = x->g.nr, nz = x->g.nz;
  cudaStream_t st = x->s;
  cudaError_t e = cudaSuccess;
  auto dn = [&](void *dst, const void *src, size_t b) {
    if (e == cudaSuccess && b) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, st);
  };
  for (int s = 0; s < 2; ++s) {
    Parts &P = cur(x, s);
    const size_t n = (size_t)x->n[s];
    dn(out->cell[s], P.cell, n * 4);
    dn(out->a[s], P.a, n * rs);
    dn(out->b[s], P.b, n * rs);
    dn(out->vr[s], P.vr, n * rs);
    dn(out->vt[s], P.vt, n * rs);
    dn(out->vz[s], P.vz, n * rs);
    dn(out->w[s], P.w, n * rs);
    dn(out->id[s], P.id, n * 4);
  }
  if (out->er) dn(out->er, x->er, (size_t)nr * (nz + 1) * 8);
  if (out->ez) dn(out->ez, x->ez, (size_t)(nr + 1) * nz * 8);
  if (out->h) dn(out->h, x->h, (size_t)nr * nz * 8);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return PIC_E_CUDA;
  for (int s = 0; s < 2; ++s) {
    out->n[s] = x->n[s];
    out->next_id[s] = x->next_id[s];
  }
  out->step = x->step;
  return PIC_OK;
}

// pic_step_host: the state's arrays as (device, host, bytes) pieces of at
// most kHostPiece bytes, species 0 then 1 (cell, a, b, vr, vt, vz, w, id),
// then the fields
namespace {
constexpr size_t kHostPiece = 64u << 20;
constexpr int kHostPieces = 128;
struct HostPiece {
  char *dev, *host;
  size_t bytes;
};
int host_pieces(pic_ctx *x, pic_host_state *hs, HostPiece *out) {
  const size_t rs = x->mixed ? 4 : 8;
  const int nr = x->g.nr, nz = x->g.nz;
  int k = 0;
  auto add = [&](void *dev, void *host, size_t b) {
    for (size_t o = 0; o < b && k < kHostPieces; o += kHostPiece)
      out[k++] = {(char *)dev + o, (char *)host + o, b - o < kHostPiece ? b - o : kHostPiece};
  };
  for (int s = 0; s < 2; ++s) {
    Parts &P = cur(x, s);
    const size_t n = (size_t)x->n[s];
    add(P.cell, hs->cell[s], n * 4);
    add(P.a, hs->a[s], n * rs);
    add(P.b, hs->b[s], n * rs);
    add(P.vr, hs->vr[s], n * rs);
    add(P.vt, hs->vt[s], n * rs);
    add(P.vz, hs->vz[s], n * rs);
    add(P.w, hs->w[s], n * rs);
    add(P.id, hs->id[s], n * 4);
  }
  if (hs->er) add(x->er, hs->er, (size_t)nr * (nz + 1) * 8);
  if (hs->ez) add(x->ez, hs->ez, (size_t)(nr + 1) * nz * 8);
  if (hs->h) add(x->h, hs->h, (size_t)nr * nz * 8);
  return k;
}
}  // namespace

int pic_step_host(pic_ctx *x, pic_host_state *hs, int nsteps, pic_step_stats *st) {
  if (!x || !hs || nsteps < 0) return PIC_E_CONFIG;
  if (!x->hs_made) {
    bool ok = cudaStreamCreateWithFlags(&x->hs_dn, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&x->hs_up, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; ok && k < 130; ++k)
      ok = cudaEventCreateWithFlags(&x->hs_ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return PIC_E_CUDA;
    x->hs_made = 1;
  }
  int r = pic_state_upload(x, hs);
  if (r) return r;
  int rc = PIC_OK;
  HostPiece pc[kHostPieces];
  long long pushes = 0;
  for (int it = 0; it < nsteps; ++it) {
    r = pic_step(x, 1, st);
    if (st) {
      pushes += st->pushes;
      st->pushes = pushes;
    }
    if (r && r != PIC_E_SUBSTEP && r != PIC_E_CAPACITY) return r;
    if (r) rc = r;
    const int np = host_pieces(x, hs, pc);
    const bool more = it + 1 < nsteps;
    // the result back to the host, piece by piece; the next step's upload of
    // each piece starts as soon as that piece has landed (the link is full duplex)
    cudaError_t e = cudaEventRecord(x->hs_ev[128], x->s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(x->hs_dn, x->hs_ev[128], 0);
    for (int k = 0; k < np && e == cudaSuccess; ++k) {
      e = cudaMemcpyAsync(pc[k].host, pc[k].dev, pc[k].bytes, cudaMemcpyDeviceToHost, x->hs_dn);
      if (e == cudaSuccess && more) e = cudaEventRecord(x->hs_ev[k], x->hs_dn);
      if (e == cudaSuccess && more) e = cudaStreamWaitEvent(x->hs_up, x->hs_ev[k], 0);
      if (e == cudaSuccess && more)
        e = cudaMemcpyAsync(pc[k].dev, pc[k].host, pc[k].bytes, cudaMemcpyHostToDevice, x->hs_up);
    }
    if (e == cudaSuccess && more) e = cudaEventRecord(x->hs_ev[129], x->hs_up);
    if (e == cudaSuccess && more) e = cudaStreamWaitEvent(x->s, x->hs_ev[129], 0);
    if (e == cudaSuccess && !more) e = cudaStreamSynchronize(x->hs_dn);
    if (e != cudaSuccess) return PIC_E_CUDA;
    for (int s = 0; s < 2; ++s) {
      hs->n[s] = x->n[s];
      hs->next_id[s] = x->next_id[s];
    }
    hs->step = x->step;
  }
  return rc;
}

int pic_set_counts(pic_ctx *x, long long ne, long long ni, uint32_t nide, uint32_t nidi,
                   long long step) {
  if (!x) return PIC_E_CONFIG;
  if (ne < 0 || ni < 0 || ne > x->cap[0] || ni > x->cap[1] || step < 0) return PIC_E_STATE;
  x->n[0] = ne;
  x->n[1] = ni;
  x->next_id[0] = nide;
  x->next_id[1] = nidi;
  x->step = step;
  x->qn_valid = 0;
  return PIC_OK;
}

int pic_mcc_constants(pic_ctx *x, double *numax_e, double *gmax, double *pnull_e,
                      double *pnull_i) {
  if (!x) return PIC_E_CONFIG;
  if (numax_e) *numax_e = x->numax_e;
  if (gmax) *gmax = x->gmax;
  if (pnull_e) *pnull_e = x->pnull_e;
  if (pnull_i) *pnull_i = x->pnull_i;
  return PIC_OK;
}

}  // extern "C"

int pic_set_guess(pic_ctx *x, int mode, pic_cnn *cnn) {
  if (!x || mode < PIC_GUESS_PLAIN || mode > PIC_GUESS_CNN) return PIC_E_CONFIG;
  if (mode == PIC_GUESS_CNN) {
    int nr = 0, nz = 0;
    if (!cnn || cnn_grid(cnn, &nr, &nz) || nr != x->g.nr || nz != x->g.nz) return PIC_E_CONFIG;
    if (!x->gev_made) {
      if (cudaEventCreateWithFlags(&x->gev[0], cudaEventDisableTiming) != cudaSuccess)
        return PIC_E_CUDA;
      if (cudaEventCreateWithFlags(&x->gev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaEventDestroy(x->gev[0]);
        return PIC_E_CUDA;
      }
      x->gev_made = 1;
    }
    x->gstream = cnn_stream(cnn);
    x->cnn_layers = cnn_layers(cnn);
  }
  if (x->guess_mode == PIC_GUESS_PLAIN && mode != PIC_GUESS_PLAIN) {
    // the history restarts from the current field
    x->hist_n = 1;
    x->sample_valid = 0;
  }
  x->guess_mode = mode;
  x->cnn = mode == PIC_GUESS_CNN ? cnn : nullptr;
  return PIC_OK;
}

int pic_guess_sample(pic_ctx *x, float *x_dev, float *t_dev, int *valid) {
  if (!x || !valid) return PIC_E_CONFIG;
  *valid = x->sample_valid;
  if (!x->sample_valid) return PIC_OK;
  const size_t P = (size_t)(x->g.nr + 1) * (x->g.nz + 1);
  cudaError_t e = cudaSuccess;
  if (x_dev) e = cudaMemcpyAsync(x_dev, x->gx, P * PIC_CNN_IN * 4, cudaMemcpyDeviceToDevice, x->s);
  if (e == cudaSuccess && t_dev)
    e = cudaMemcpyAsync(t_dev, x->gt, P * PIC_CNN_OUT * 4, cudaMemcpyDeviceToDevice, x->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->s);
  return e == cudaSuccess ? PIC_OK : PIC_E_CUDA;
}

// ---------------------------------------------------------------------------
// ensembles (include/pic_ensemble.h)

struct pic_ensemble {
  int n;
  pic_ctx *m[PIC_ENSEMBLE_MAX];
  // persistent rounds: each species' push of every active member in one
  // launch of the fast and one of the general kernel, on the lead stream
  int persistent;
  cudaStream_t lead;
  cudaEvent_t ev_pre[PIC_ENSEMBLE_MAX], ev_sp[2];
  char *stage;  // pinned: per species, the members' launch parameters, then the item offsets
  char *dbuf;   // device copy
  int ready;
};

namespace {

void drop_graphs(pic_ctx *x) {
  if (x->ngraph) cudaStreamSynchronize(x->s);
  for (int k = 0; k < x->ngraph; ++k) {
    cudaGraphExecDestroy(x->gcache[k].exec);
    if (x->gcache[k].ptimed) {
      cudaEventDestroy(x->gcache[k].pe[0]);
      cudaEventDestroy(x->gcache[k].pe[1]);
    }
  }
  x->rep_pe = nullptr;
  x->ngraph = 0;
}

}  // namespace

// staging of one species' launch parameters (persistent rounds)
constexpr size_t kMaxLaunchBytes = sizeof(PushLaunchT<double>) > sizeof(PushLaunchT<float>)
                                       ? sizeof(PushLaunchT<double>)
                                       : sizeof(PushLaunchT<float>);
constexpr size_t kSlotLaunch = (PIC_ENSEMBLE_MAX * kMaxLaunchBytes + 255) / 256 * 256;
constexpr size_t kSlot = (kSlotLaunch + 2 * (PIC_ENSEMBLE_MAX + 1) * sizeof(int) + 255) / 256 * 256;

// one Picard pass of the members A[0..nl) (all of precision T): each member's
// pre-push part on its stream; on the lead stream, per species, the members'
// launch parameters uploaded and their fast and general phases in one launch
// each (the mixed form's near-axis lists then on each member's stream); then
// each member's field solve on its stream
template <typename T>
int round_persistent(pic_ensemble *E, const int *A, int nl, std::vector<StepState> &St) {
  for (int a = 0; a < nl; ++a) {
    pic_ctx *x = E->m[A[a]];
    int r = enqueue_pre(x, St[A[a]].spec);
    if (r) return r;
    if (cudaEventRecord(E->ev_pre[a], x->s) != cudaSuccess ||
        cudaStreamWaitEvent(E->lead, E->ev_pre[a], 0) != cudaSuccess)
      return PIC_E_CUDA;
  }
  for (int s = 0; s < 2; ++s) {
    char *h = E->stage + s * kSlot;
    char *d = E->dbuf + s * kSlot;
    PushLaunchT<T> *Ls = reinterpret_cast<PushLaunchT<T> *>(h);
    int *first = reinterpret_cast<int *>(h + kSlotLaunch);
    first[0] = 0;
    first[nl + 1] = 0;
    for (int a = 0; a < nl; ++a) {
      round_launch(E->m[A[a]], s, St[A[a]].spec, Ls[a]);
      int nf = 0, ng = 0;
      push_shape(Ls[a], &nf, &ng);
      first[a + 1] = first[a] + nf;
      first[nl + 2 + a] = first[nl + 1 + a] + ng;
    }
    if (cudaMemcpyAsync(d, h, nl * sizeof(PushLaunchT<T>), cudaMemcpyHostToDevice, E->lead) !=
            cudaSuccess ||
        cudaMemcpyAsync(d + kSlotLaunch, h + kSlotLaunch, (size_t)(2 * nl + 2) * sizeof(int),
                        cudaMemcpyHostToDevice, E->lead) != cudaSuccess)
      return PIC_E_CUDA;
    if (launch_push_multi<T>(reinterpret_cast<const PushLaunchT<T> *>(d),
                             reinterpret_cast<const int *>(d + kSlotLaunch), nl,
                             E->lead) != cudaSuccess)
      return PIC_E_CUDA;
    E->m[A[0]]->launches += 2;
    if (cudaEventRecord(E->ev_sp[s], E->lead) != cudaSuccess) return PIC_E_CUDA;
    if constexpr (sizeof(T) == 4) {
      // the near-axis lists of this species on each member's stream, beside
      // the next launches on the lead stream
      for (int a = 0; a < nl; ++a) {
        pic_ctx *x = E->m[A[a]];
        if (cudaStreamWaitEvent(x->s, E->ev_sp[s], 0) != cudaSuccess ||
            launch_push_fp32_axis(Ls[a], x->s) != cudaSuccess)
          return PIC_E_CUDA;
        x->launches += 1;
      }
    }
  }
  for (int a = 0; a < nl; ++a) {
    pic_ctx *x = E->m[A[a]];
    if (sizeof(T) == 8 && cudaStreamWaitEvent(x->s, E->ev_sp[1], 0) != cudaSuccess)
      return PIC_E_CUDA;
    int r = enqueue_post(x);
    if (r) return r;
  }
  return PIC_OK;
}

// members that a persistent round can take together: one precision, both
// species moving, the fast path (no magnetic field) and the queue
bool persistent_ok(const pic_ensemble *E) {
  for (int i = 0; i < E->n; ++i) {
    const pic_ctx *x = E->m[i];
    if (x->mixed != E->m[0]->mixed || x->cfg.ions_fixed || x->cfg.bz != 0.0 || !x->queue)
      return false;
  }
  return true;
}

int pic_set_graphs(pic_ctx *x, int on) {
  if (!x) return PIC_E_CONFIG;
  x->graphs = on ? 1 : 0;
  return PIC_OK;
}

int pic_set_device_picard(pic_ctx *x, int on) {
  if (!x || (on != 0 && on != 1)) return PIC_E_CONFIG;
  x->dloop = on;
  return PIC_OK;
}

int pic_ensemble_create(pic_ctx *const *members, int n, pic_ensemble **out) {
  if (!out) return PIC_E_CONFIG;
  *out = nullptr;
  if (!members || n < 1 || n > PIC_ENSEMBLE_MAX) return PIC_E_CONFIG;
  for (int i = 0; i < n; ++i) {
    if (!members[i]) return PIC_E_CONFIG;
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) return PIC_E_CONFIG;
  }
  pic_ensemble *E = (pic_ensemble *)calloc(1, sizeof(pic_ensemble));
  if (!E) return PIC_E_CONFIG;
  E->n = n;
  for (int i = 0; i < n; ++i) {
    E->m[i] = members[i];
    members[i]->graphs = 1;
  }
  // the lead stream, its events and the launch-parameter staging of
  // persistent rounds
  bool ok = cudaStreamCreateWithFlags(&E->lead, cudaStreamNonBlocking) == cudaSuccess;
  int nev = 0;
  for (; ok && nev < n; ++nev)
    ok = cudaEventCreateWithFlags(&E->ev_pre[nev], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&E->ev_sp[0], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&E->ev_sp[1], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaHostAlloc((void **)&E->stage, 2 * kSlot, cudaHostAllocDefault) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&E->dbuf, 2 * kSlot) == cudaSuccess;
  if (!ok) {
    E->ready = 0;
    pic_ensemble_destroy(E);
    return PIC_E_CUDA;
  }
  E->ready = 1;
  E->persistent = persistent_ok(E) ? 1 : 0;
  *out = E;
  return PIC_OK;
}

void pic_ensemble_destroy(pic_ensemble *E) {
  if (!E) return;
  if (E->lead) {
    cudaStreamSynchronize(E->lead);
    cudaStreamDestroy(E->lead);
  }
  for (int i = 0; i < E->n; ++i)
    if (E->ev_pre[i]) cudaEventDestroy(E->ev_pre[i]);
  for (int k = 0; k < 2; ++k)
    if (E->ev_sp[k]) cudaEventDestroy(E->ev_sp[k]);
  if (E->stage) cudaFreeHost(E->stage);
  if (E->dbuf) cudaFree(E->dbuf);
  free(E);
}

int pic_ensemble_set_persistent(pic_ensemble *E, int on) {
  if (!E) return PIC_E_CONFIG;
  if (on && !persistent_ok(E)) return PIC_E_CONFIG;
  E->persistent = on ? 1 : 0;
  return PIC_OK;
}

int pic_ensemble_step(pic_ensemble *E, int nsteps, pic_step_stats *st) {
  if (!E || nsteps < 0) return PIC_E_CONFIG;
  const int n = E->n;
  int rc = PIC_OK;
  std::vector<StepState> T(n);
  std::vector<char> active(n);
  for (int it = 0; it < nsteps; ++it) {
    for (int i = 0; i < n; ++i) {
      int r = step_begin(E->m[i], T[i]);
      if (r) return r;
      active[i] = 1;
    }
    // rounds: one Picard pass of every unconverged member, then one wait
    int nact = n;
    while (nact) {
      if (E->persistent) {
        int A[PIC_ENSEMBLE_MAX], nl = 0;
        for (int i = 0; i < n; ++i)
          if (active[i]) A[nl++] = i;
        int r = E->m[0]->mixed ? round_persistent<float>(E, A, nl, T)
                               : round_persistent<double>(E, A, nl, T);
        if (r) return r;
        for (int a = 0; a < nl; ++a) T[A[a]].S.pushes += E->m[A[a]]->n[0] + E->m[A[a]]->n[1];
      } else {
        for (int i = 0; i < n; ++i) {
          if (!active[i]) continue;
          pic_ctx *x = E->m[i];
          int r = launch_pass(x, T[i].spec);
          if (r) return r;
          T[i].S.pushes += x->n[0] + x->n[1];
        }
      }
      for (int i = 0; i < n; ++i) {
        if (!active[i]) continue;
        pic_ctx *x = E->m[i];
        if (cudaStreamSynchronize(x->s) != cudaSuccess) return PIC_E_CUDA;
        StepState &S = T[i];
        finish_pass(x, S.k, S.rprev, S.res, S.src, S.first, S.conv, S.spec, S.spec_ok);
        if (!isfinite(S.res)) return PIC_E_NAN;
        if (S.conv) {
          active[i] = 0;
          --nact;
          continue;
        }
        if (++S.k < x->cfg.picard_max) continue;
        if (S.used != PIC_GUESS_PLAIN) {
          // the plain start remains the fallback
          S.used = PIC_GUESS_PLAIN;
          S.k = 0;
          S.spec = false;
          S.rprev = 0.0;
          int r = plain_start(x, S.v1);
          if (r) return r;
        } else {
          active[i] = 0;  // not converged: step_end reports PIC_E_NOCONV
          --nact;
        }
      }
    }
    for (int i = 0; i < n; ++i) {
      int r = step_end(E->m[i], T[i], &rc);
      if (st) st[i] = T[i].S;
      if (r) return r;
    }
  }
  return rc;
}

int pic_ensemble_tune(pic_ensemble *E, int rounds, float *frac_out, int *persistent_out,
                      double *ms_out) {
  if (!E || rounds < 1) return PIC_E_CONFIG;
  const float fr[3] = {1.0f, 0.5f, 0.25f};
  const bool pok = persistent_ok(E);
  double best = 1e300;
  int bi = 0;
  std::vector<StepState> T(E->n);
  int A[PIC_ENSEMBLE_MAX];
  for (int i = 0; i < E->n; ++i) A[i] = i;
  for (int c = 0; c < 6; ++c) {
    const int f = c % 3, pers = c / 3;
    if (ms_out) ms_out[c] = -1.0;
    if (pers && !pok) continue;
    for (int i = 0; i < E->n; ++i) {
      pic_ctx *x = E->m[i];
      drop_graphs(x);
      int wf = x->mixed ? push_wave_fp32(0) : push_wave_fp64(0);
      int wg = x->mixed ? push_wave_fp32(1) : push_wave_fp64(1);
      x->fgrid[0] = fr[f] < 1.0f ? (int)(wf * fr[f]) > 0 ? (int)(wf * fr[f]) : 1 : 0;
      x->ggrid[0] = fr[f] < 1.0f ? (int)(wg * fr[f]) > 0 ? (int)(wg * fr[f]) : 1 : 0;
      if (upload_step(x, volt_at(x, x->step), volt_at(x, x->step + 1))) return PIC_E_CUDA;
      int r = plain_start(x, volt_at(x, x->step + 1));
      if (r) return r;
      memset(&T[i], 0, sizeof(StepState));
    }
    double tbest = 1e300;
    for (int rep = 0; rep < rounds + 1; ++rep) {
      for (int i = 0; i < E->n; ++i)
        if (cudaStreamSynchronize(E->m[i]->s) != cudaSuccess) return PIC_E_CUDA;
      auto t0 = std::chrono::steady_clock::now();
      if (pers) {
        int r = E->m[0]->mixed ? round_persistent<float>(E, A, E->n, T)
                               : round_persistent<double>(E, A, E->n, T);
        if (r) return r;
      } else {
        for (int i = 0; i < E->n; ++i) {
          int r = enqueue_pass(E->m[i], false);
          if (r) return r;
        }
      }
      for (int i = 0; i < E->n; ++i)
        if (cudaStreamSynchronize(E->m[i]->s) != cudaSuccess) return PIC_E_CUDA;
      double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                      .count();
      if (rep > 0 && ms < tbest) tbest = ms;  // the first round warms up
    }
    if (ms_out) ms_out[c] = tbest;
    if (tbest < best) {
      best = tbest;
      bi = c;
    }
  }
  const int f = bi % 3;
  for (int i = 0; i < E->n; ++i) {
    pic_ctx *x = E->m[i];
    drop_graphs(x);
    int wf = x->mixed ? push_wave_fp32(0) : push_wave_fp64(0);
    int wg = x->mixed ? push_wave_fp32(1) : push_wave_fp64(1);
    x->fgrid[0] = f ? (int)(wf * fr[f]) : 0;
    x->ggrid[0] = f ? (int)(wg * fr[f]) : 0;
  }
  E->persistent = bi / 3;
  if (frac_out) *frac_out = fr[f];
  if (persistent_out) *persistent_out = E->persistent;
  return PIC_OK;
}
