/*
 * pic.h — C ABI of the GB300 (sm_103a) hot path of the implicit, energy- and
 * charge-conserving electromagnetic PIC/MCC method of Eremin et al.,
 * arXiv:2212.08836 ("Modeling of VHF large-electrode CCPs with a fully
 * electromagnetic PIC code").
 *
 * One time step = Picard iteration of [CN particle push with cell-crossing
 * sub-steps + charge-conserving deposit (Sec. 2.1, Eqs. 3-4)] and [implicit
 * CN Maxwell solve for H_theta (Eqs. 1-2)], a commit push, null-collision MCC
 * (Sec. 2.1) and a per-step sort of the particle store by cell.
 *
 * Conventions shared by every entry point
 *   - Grid: nr x nz uniform cells on r in [0,R], z in [0,L]; z fastest.
 *       Er edge (i+1/2, j)  -> er[i*(nz+1)+j], i < nr, j <= nz
 *       Ez edge (i, j+1/2)  -> ez[i*nz+j],     i <= nr, j < nz
 *       H_theta (i+1/2,j+1/2)-> h[i*nz+j]
 *       node (i, j)         -> q[i*(nz+1)+j]
 *     "Current" arrays ir/iz hold the charge [C] that crossed the dual face
 *     of each edge during one step (flux form of Eq. 3).
 *   - Particles: species 0 = electrons, 1 = Ar+; structure of arrays
 *     cell (int32, ic*nz+jc, -1 = absorbed), a, b (offsets in [0,1] inside
 *     the cell), vr, vt, vz [m/s], w (physical particles per macro-particle),
 *     id (uint32, RNG counter word).  Stored sorted by cell.
 *   - Memory: the library never allocates device memory.  The caller passes
 *     one device workspace (size from pic_workspace_size) that it owns and
 *     frees after pic_destroy.  Pointers named *_dev are device pointers,
 *     everything else is host memory.
 *   - Streams: all work is enqueued on the cudaStream_t given to pic_init
 *     (passed as void*).  Calls that return host values synchronise it.
 *   - Errors: every int-returning call returns PIC_OK (0) or a negative
 *     PIC_E_* code; it never aborts and never prints.  After an error other
 *     than PIC_E_CUDA the context stays usable.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_E_CONFIG -1    /* invalid configuration or argument */
#define PIC_E_CUDA -2      /* a CUDA call failed (context may be unusable) */
#define PIC_E_NOCONV -3    /* Picard iteration did not reach picard_tol in picard_max */
#define PIC_E_SUBSTEP -4   /* a particle needed more than 64 sub-steps in one pass */
#define PIC_E_CAPACITY -5  /* ionization would exceed the particle capacity */
#define PIC_E_NAN -6       /* non-finite field or residual */
#define PIC_E_STATE -7     /* state arrays inconsistent (counts beyond capacity) */
#define PIC_E_WORKSPACE -8 /* workspace missing, too small or misaligned */
#define PIC_E_IO -9        /* checkpoint file could not be written or read, or is malformed */

#define PIC_FP64 0         /* plain method: FP64 particles, push and deposit */
#define PIC_MIXED 1        /* FP32 particle state, push and deposit; FP64 field solve,
                              Picard norms, current accumulation and diagnostics */

#define PIC_FIELD_EM 0     /* electromagnetic field model (Eqs. 1-2, CN; the default) */
#define PIC_FIELD_ES 1     /* electrostatic model (Eq. 8): E = -grad phi, Gauss's law on
                              the nodes with the charge advanced by continuity (Eq. 3);
                              H = 0 */

#define PIC_FEED_GAP 0      /* r = R carries the prescribed gap field V(t)/L (the default) */
#define PIC_FEED_WAVE 1     /* r = R is a wave port (Eq. 5 read for the side feed): the first-order
                               absorbing condition E_z + eta H_theta = 2 E_in with the incoming
                               wave E_in = V(t)/(2L), eta = sqrt(mu/eps); outgoing waves leave,
                               a slow drive gives the gap voltage V(t).  EM model only. */
#define PIC_FEED_AXIAL 2    /* the paper's feed (Sec. 2.2, Fig. 1): a coaxial port filled with a
                               dielectric (eps_port) below the powered electrode, from its radius
                               r_p = r(port_rin) out to R, port_cells cells of port_len / port_cells
                               deep; the electrode's stem and the outer wall are conductors, as is
                               the reactor's side wall r = R.  At the port's end Eq. 5 (Mur's
                               condition) in the form E_r + eta H = 2 E_r^+ with the incoming TEM
                               wave of Eq. 7's reading, E_r^+ = (V(t) / 2) / (r ln(R / r_p)): half
                               the electrode potential (with cblock > 0, Eq. 6's phi(t) instead
                               of V(t)); the port's fields through pic_get_view.  Electrostatic
                               model (Sec. 2.2's counterpart): the port's opening r_p < r < R of
                               z = 0 carries the coaxial line's potential phi ln(r/R)/ln(r_p/R)
                               as a Dirichlet value, the disc r <= r_p is at phi, the side wall
                               grounded.  No rings or wave port. */

typedef struct pic_ctx pic_ctx; /* opaque; host memory owned by the library */

/* Problem definition, copied at pic_init.  Zero eps/mu select vacuum values. */
typedef struct pic_config {
  int nr, nz;                 /* cells in r and z (nr, nz >= 2) */
  double R, L;                /* electrode radius and gap [m] */
  double dt;                  /* time step [s] */
  double freq, volt;          /* V(t) = volt*sin(2*pi*freq*t) on the powered electrode z = 0 */
  double gas_pressure;        /* argon pressure [Pa] (neutral density p/(k T)) */
  double gas_temp;            /* neutral temperature [K] */
  double n0;                  /* initial plasma density [m^-3] */
  double te_ev, ti_ev;        /* initial electron / ion temperatures [eV] */
  long long np_init;          /* macro-particles per species loaded by pic_load_particles */
  double capacity_factor;     /* capacity per species = ceil(capacity_factor * np_init) (>= 1) */
  double picard_tol;          /* relative Picard tolerance on E (e.g. 1e-8) */
  int picard_max;             /* maximum Picard iterations per step (e.g. 50) */
  int mcc_on;                 /* 1: null-collision MCC after every step */
  double bz;                  /* external uniform B_z [T]; 0 in production (Sec. 2.1) */
  double eps, mu;             /* permittivity / permeability; 0 -> eps0 / mu0 */
  unsigned long long seed;    /* RNG key word (Philox4x64-10) */
  int precision;              /* PIC_FP64 or PIC_MIXED */
  int field_model;            /* PIC_FIELD_EM or PIC_FIELD_ES */
  double cblock;              /* blocking capacitor [F] between the generator V(t) and the
                                 powered electrode (Eq. 6); 0 = none (the electrode is at V(t)) */
  int ions_fixed;             /* 1: ions stay at their positions (no push, deposit or sort), as in
                                 the dispersion test of Sec. 3.1; requires mcc_on = 0 */
  int feed;                   /* PIC_FEED_GAP, PIC_FEED_WAVE (EM model, no capacitor) or
                                 PIC_FEED_AXIAL */
  int ring_cells;             /* dielectric ring: the outer ring_cells cells (r > R_d) are filled
                                 with a dielectric of relative permittivity eps_ring; particles
                                 move in r < R_d and stick at the ring face (0 = none) */
  double eps_ring;            /* relative permittivity of the ring (>= 1; e.g. 3.8 for quartz) */
  int axis_cells;             /* mapped radial mesh (Sec. 2.1), 0..16 (< nr): the first
                                 axis_cells cells have r = 2 dr sqrt(xa xi), the rest
                                 r = dr (xi + xa), dr = R / (nr + xa), r linear in xi inside
                                 each cell; 0 = uniform mesh r = xi R / nr */
  double sigma_ring;          /* conductivity of the ring's cells [S/m] (Eq. 2's sigma E, taken
                                 at the half step); a large value models a metal (Sec. 2.1).
                                 Needs ring_cells > 0 and the EM model (an electrostatic run
                                 models a metal by a large eps_ring); 0 = none */
  int port_cells;             /* PIC_FEED_AXIAL: cells along z of the port (>= 1; EM only,
                                 checked for both models) */
  double port_len;            /* PIC_FEED_AXIAL: the port's length [m] (EM only) */
  int port_rin;               /* PIC_FEED_AXIAL: the port's inner radius is the node r(port_rin),
                                 1 <= port_rin < nr (the powered electrode's radius) */
  double eps_port;            /* PIC_FEED_AXIAL: relative permittivity of the port (>= 1; EM
                                 only) */
  double port_grade;          /* PIC_FEED_AXIAL, EM: the port's rows grow by this ratio from the
                                 junction down to its end (a geometric progression summing to
                                 port_len; the nonuniform axial mesh of Sec. 2.1, lengthening
                                 the waveguide in few cells); 0 or 1: uniform; 0.25..4 */
} pic_config;

/* Per-step statistics (host struct). */
typedef struct pic_step_stats {
  int picard_iters;           /* iterations of the last step */
  int converged;              /* 1 if the last step converged */
  double last_res;            /* last Picard residual */
  double src_energy;          /* energy delivered through the drive gap in the last step [J] */
  double ke_lost;             /* kinetic energy of particles absorbed at walls [J] */
  double de_coll;             /* kinetic-energy change from collisions [J] */
  long long substep_err;      /* particles that hit the sub-step cap (commit pass) */
  long long absorbed;         /* particles absorbed at walls (commit pass) */
  long long substeps;         /* accepted sub-steps (commit pass) */
  long long fallbacks;        /* trial halvings (commit pass) */
  long long mcc[8];           /* cand_e, elastic, excitation, ionization, cand_i, cx, gmax overflow, capacity */
  long long n[2];             /* macro-particles per species after the step */
  long long pushes;           /* particle pushes performed by the step (all passes) */
  long long launches;         /* kernels launched by the step */
  long long push_flops;       /* algorithmic FP64 operations of the commit pass */
  int guess;                  /* Picard start used by the last step (PIC_GUESS_* of pic_guess.h) */
  int spec_final;             /* 1: the converged pass wrote the new state (no separate commit push) */
  double first_res;           /* Picard residual after the first iteration of the last step */
  double v_electrode;         /* powered-electrode potential phi^{n+1} after the last step [V] */
  double q_cap;               /* blocking-capacitor charge q^{n+1} after the last step [C] */
} pic_step_stats;

/* Device pointers and sizes of the context's arrays (for parity tests,
 * checkpoints and callers that fill state directly). */
typedef struct pic_view {
  int32_t *cell[2];
  void *a[2], *b[2], *vr[2], *vt[2], *vz[2], *w[2]; /* double (PIC_FP64) or float (PIC_MIXED) */
  uint32_t *id[2];
  long long n[2], cap[2];
  uint32_t next_id[2];
  double *er, *ez, *h;        /* E^n, H^n */
  long long step;             /* index n of the next step */
  int real_size;              /* bytes per element of a..w: 8 or 4 */
  double *wall;               /* charge [C] absorbed at the walls since pic_init, per species s
                                 at wall + s*(2(nr+1) + nz+1): nodes of z = 0 (nr+1), of z = L
                                 (nr+1), of r = R (nz+1) */
  double *qcond;              /* charge [C] the conducting ring's current moved since pic_init,
                                 per node (nr+1) x (nz+1); Gauss's law holds with it added to
                                 the particle and wall charge (zero without sigma_ring) */
  /* PIC_FEED_AXIAL (else null / 0): the port's fields at n, m = nr - port_rin columns of
   * port_cells cells (q = 0 at the port's end): H at port_h[k * port_cells + q] (cell
   * (port_rin + k, q)), E_r at port_er[k * port_cells + q] (the lower face of that cell: q = 0
   * the end edge; the top faces are the interface edges, E_r of j = 0 in er), E_z at
   * port_ez[k * port_cells + q] for nodes k = 0..m (zero on the conductors k = 0 and m) */
  double *port_h, *port_er, *port_ez;
  int port_m, port_cells;
} pic_view;

/* Conservation diagnostics (row a9), host struct filled by pic_diag. */
typedef struct pic_diag_out {
  double kinetic[2];          /* sum 1/2 m w |v|^2 per species [J] */
  double field;               /* discrete field energy over unknown edges and H cells [J] */
  double charge[2];           /* sum q w per species [C] */
  long long n[2];
} pic_diag_out;

/* Human-readable name of a status code (static string). */
const char *pic_strerror(int code);

/* Library build identifier (static string). */
const char *pic_version(void);

/* Bytes of device workspace pic_init needs for cfg (256-byte aligned base).
 * Errors: PIC_E_CONFIG. */
int pic_workspace_size(const pic_config *cfg, size_t *bytes);

/* Create a context on the current CUDA device over a caller-owned device
 * workspace (workspace_dev, workspace_bytes >= pic_workspace_size).  Builds
 * the mesh metrics and the factorised field operator of Eq. 2 (host set-up,
 * then copied into the workspace on `stream`).  Fields start at zero and no
 * particles are loaded.  Errors: PIC_E_CONFIG, PIC_E_WORKSPACE, PIC_E_CUDA. */
int pic_init(const pic_config *cfg, void *workspace_dev, size_t workspace_bytes, void *stream,
             pic_ctx **out);

/* Release the host context.  The workspace stays the caller's. */
void pic_destroy(pic_ctx *ctx);

/* Row a1 (Sec. 2.1: weights proportional to r*J_r): load np_init electron /
 * Ar+ pairs at identical positions, uniform in the logical coordinates,
 * Maxwellian velocities, on the GPU; then sort by cell.  E = H = 0 is then
 * Gauss-consistent.  Errors: PIC_E_CAPACITY, PIC_E_CUDA. */
int pic_load_particles(pic_ctx *ctx);

/* Advance nsteps full time steps (rows a2-a8; a9 counters in stats).
 * stats may be NULL.  On PIC_E_NOCONV the context holds step n unchanged.
 * Synchronises the stream (Picard convergence test).
 * Errors: PIC_E_NOCONV, PIC_E_SUBSTEP, PIC_E_CAPACITY, PIC_E_NAN, PIC_E_CUDA. */
int pic_step(pic_ctx *ctx, int nsteps, pic_step_stats *stats);

/* Rows a2+a3 (a6 when write != 0), Eq. 4 with cell-crossing sub-steps and
 * the deposit of Eq. 3: one pass over both species with the half-step field
 * er_half_dev / ez_half_dev (layout above).  Adds the crossed charges into
 * ir_dev / iz_dev (caller zeroes them).  write = 0 leaves the particles
 * untouched; write = 1 stores state n+1 (cell -1 for absorbed particles).
 * counters_dev (nullable, 5 x uint64): substep errors, absorbed, substeps,
 * fallbacks, algorithmic FP64 operations (add/sub/mul/div of the source);
 * ke_lost_dev (nullable, double): absorbed kinetic energy.
 * Asynchronous.  Errors: PIC_E_CONFIG, PIC_E_CUDA. */
int pic_push_deposit(pic_ctx *ctx, const double *er_half_dev, const double *ez_half_dev,
                     double *ir_dev, double *iz_dev, int write,
                     unsigned long long *counters_dev, double *ke_lost_dev);

/* Electrostatic model, Eq. 8 on the same mesh: the potential on the nodes
 * with phi = phi0 on the powered plate z = 0, 0 on z = L and phi0 (1 - z/L)
 * across the drive gap at r = R, Gauss's law eps div E = Q on the interior
 * nodes (i < nr, 0 < j < nz) in the flux form of the electromagnetic scheme.
 * Q_dev: node charges [(nr+1) x (nz+1)] (device, only interior nodes used);
 * outputs E_r, E_z in the Yee layouts (device, not aliasing Q).  Solved
 * directly (DST-I along z, cyclic reduction along r).  Asynchronous.
 * Errors: PIC_E_CONFIG, PIC_E_CUDA. */
int pic_es_solve(pic_ctx *ctx, const double *Q_dev, double phi0, double *er_dev, double *ez_dev);

/* Blocking capacitor (Eq. 6, cfg.cblock > 0).  Each Picard iteration solves
 * for the electrode potential phi^{n+1} that makes the reactor-side current
 * (displacement current plus crossed charge through the dual faces of the
 * first row of E_z edges above the powered plate, i < nr; with the axial port
 * i < port_rin, the electrode's radius) equal to the capacitor current
 * (C (V^{n+1} - phi^{n+1}) - q^n) / dt.  The field solve is affine in
 * phi^{n+1}, so the equation is solved exactly from the solve at V^{n+1} and a
 * unit response computed at pic_init (EM, through the port when there is one)
 * or known in closed form (ES: the vacuum potential 1 - z/L).  The potential
 * then drives the gap (EM), the axial port's incoming wave (half of it), or
 * the plate and gap Dirichlet values (ES).  The state starts at
 * q = 0, phi = V(t) at pic_init and pic_load_particles.
 * pic_circuit_get: q^n [C] and phi^n [V] (host, nullable); without a
 * capacitor q = 0 and phi = V(t^n).  Synchronises.
 * pic_circuit_set: sets them (e.g. to resume a run).  Synchronises.
 * Errors: PIC_E_CONFIG (set without a capacitor), PIC_E_CUDA. */
int pic_circuit_get(pic_ctx *ctx, double *q, double *phi);
int pic_circuit_set(pic_ctx *ctx, double q, double phi);

/* Picard tolerance and iteration limit of the following steps (the values
 * of pic_config at pic_init).  A caller may relax them for a step that ends
 * in PIC_E_NOCONV (the state is then still at step n) and retry it.
 * Errors: PIC_E_CONFIG (tol <= 0 or not finite, kmax < 1). */
int pic_set_picard(pic_ctx *ctx, double tol, int kmax);

/* Generator waveform V(t) = sum_k amp[k] sin(2 pi freq[k] t + phase[k]),
 * t = step * dt, k < n (n <= 64), replacing volt * sin(2 pi freq t) from the
 * next step on (the sawtooth excitation of Sec. 3.1 is n harmonics with
 * amp = A/k); n = 0 restores the configured sine.  Errors: PIC_E_CONFIG. */
int pic_set_drive(pic_ctx *ctx, int n, const double *amp, const double *freq,
                  const double *phase);

/* Fourier-Bessel coefficients (App. A, Eq. A2) of the context's field E^n
 * along r at one axial row: c_m = int r f F_m dr / int r F_m^2 dr with
 * F_m = J_alpha(chi_{alpha,m} r / R), chi_{alpha,m} the m-th zero of J_alpha,
 * m = 1..nmodes (nmodes <= 64).  alpha = 0: f = E_z on the edges
 * (i, row + 1/2), i = 0..nr (0 <= row < nz), integrals by the trapezoid rule
 * on the nodes; alpha = 1: f = E_r on the edges (i + 1/2, row), i < nr
 * (0 <= row <= nz), midpoint rule.  coef_dev: nmodes doubles (device).
 * Asynchronous, one kernel; a call with a new (alpha, nmodes) first builds
 * the basis on the host and synchronises.  Errors: PIC_E_CONFIG, PIC_E_CUDA. */
int pic_fourier_bessel(pic_ctx *ctx, int alpha, int row, int nmodes, double *coef_dev);

/* Row a4, Eqs. 1-2 in CN form: one implicit field solve.  Inputs E^n, H^n,
 * crossed charges, drive voltages V^n (v0) and V^{n+1} (v1); outputs E^{n+1},
 * H^{n+1} and, if src_dev != NULL, the energy delivered through the drive
 * gap (double).  All arrays are device arrays in the layout above; outputs
 * must not alias inputs.  Asynchronous.  Errors: PIC_E_CONFIG, PIC_E_CUDA. */
int pic_field_solve(pic_ctx *ctx, const double *er0_dev, const double *ez0_dev,
                    const double *h0_dev, const double *ir_dev, const double *iz_dev, double v0,
                    double v1, double *er1_dev, double *ez1_dev, double *h1_dev, double *src_dev);

/* pic_field_solve with the axial port (PIC_FEED_AXIAL): the port's fields at n
 * (hp0, erp0, ezp0) and n+1 (hp1, erp1, ezp1) in the layout of pic_view's
 * port arrays; phi0, phi1: the electrode potential at n and n+1 (the incoming
 * wave carries half of it).  src_dev (nullable): the energy delivered through
 * the port's end.  Errors: PIC_E_CONFIG (not an axial-port context), PIC_E_CUDA. */
int pic_port_field_solve(pic_ctx *ctx, const double *er0_dev, const double *ez0_dev,
                         const double *h0_dev, const double *hp0_dev, const double *erp0_dev,
                         const double *ezp0_dev, const double *ir_dev, const double *iz_dev,
                         double phi0, double phi1, double *er1_dev, double *ez1_dev,
                         double *h1_dev, double *hp1_dev, double *erp1_dev, double *ezp1_dev,
                         double *src_dev);

/* Row a7 (Sec. 2.1, null collision after Mertmann et al. 2011): one MCC pass
 * over the context's particles for step index `step`, appending ionization
 * pairs in parent order.  counts (host, nullable, 8 entries as in
 * pic_step_stats.mcc); de_coll (host, nullable).  Synchronises.
 * Errors: PIC_E_CAPACITY, PIC_E_CUDA. */
int pic_mcc(pic_ctx *ctx, unsigned long long step, long long *counts, double *de_coll);

/* Row a8: counting sort of both species by cell, dropping absorbed
 * particles (cell < 0).  Synchronises (new counts).  Errors: PIC_E_CUDA. */
int pic_sort(pic_ctx *ctx);

/* Row a9: FP64 kinetic and field energies and charges.  Synchronises. */
int pic_diag(pic_ctx *ctx, pic_diag_out *out);

/* Diagnostic kinds of pic_diag_get (row a9; the time-averaged profiles are
 * the long-run statistics the paper compares, e.g. the ion flux onto the
 * electrodes of Sec. 4.1).  Node (i, j), i = 0..nr, j = 0..nz, z fastest. */
enum {
  PIC_DIAG_ENERGY = 0,       /* pic_diag_out (host destination only) */
  PIC_DIAG_GAUSS = 1,        /* (nr+1)(nz+1) doubles: pic_gauss_residual */
  PIC_DIAG_CONTINUITY = 2,   /* (nr+1)(nz+1) doubles: charge balance of the last committed
                              * step per node, (Q^{n+1} - Q^n) + (W^{n+1} - W^n) + div dQ, with
                              * Q the S1 x S1 node charge of both species, W the wall (and
                              * ring-face) tallies on their nodes, dQ the crossed charge of
                              * the step (Eq. 3); zero up to rounding.  Needs averaging on. */
  PIC_DIAG_DENSITY_AVG = 3,  /* 2 (nr+1)(nz+1) doubles: electrons then ions, node density
                              * [m^-3] averaged over the steps since pic_diag_average(ctx, 1):
                              * sum of w S1 x S1 / (steps x dual volume of the node) */
  PIC_DIAG_ION_FLUX_AVG = 4, /* 2 (nr+1) doubles: mean Ar+ flux [m^-2 s^-1] absorbed by the
                              * electrode z = 0, then z = L, per radial node (its dual ring
                              * on the electrode), over the same window */
  PIC_DIAG_FIELDS = 5,       /* E_r (nr (nz+1)), E_z ((nr+1) nz), H_theta (nr nz) doubles */
  PIC_DIAG_COUNTS = 6        /* 4 long long: n_e, n_i, step index, steps averaged */
};

/* Starts (enable = 1: clears the averages and the window) or stops
 * (enable = 0) the per-step diagnostics: after every committed step the node
 * densities of both species are added to the averages and the step's
 * continuity residual is formed (one extra pass over the particles per
 * step).  Asynchronous.  Errors: PIC_E_CONFIG, PIC_E_CUDA. */
int pic_diag_average(pic_ctx *ctx, int enable);

/* One diagnostic of the kinds above into dst (bytes >= its size; on the
 * device when dst_is_device, else host memory).  Synchronises the stream.
 * Errors: PIC_E_CONFIG (unknown kind, bytes too small, ENERGY to a device
 * destination), PIC_E_STATE (CONTINUITY before a step with averaging on,
 * averages with no step averaged), PIC_E_CUDA. */
int pic_diag_get(pic_ctx *ctx, int kind, void *dst, size_t bytes, int dst_is_device);

/* Node charge by S1 x S1 weighting of both species, added into q_dev
 * ((nr+1)*(nz+1) doubles, caller zeroes).  Asynchronous. */
int pic_node_charge(pic_ctx *ctx, double *q_dev);

/* Row a9: Gauss residual of the state, eps div_h E^n - Q^n on the interior
 * nodes (i < nr, 0 < j < nz) in the flux form of the integral mesh, Q^n the
 * S1 x S1 node charge of both species plus, with the dielectric ring, the
 * charge stuck on the ring's face; zero on the other nodes.  The
 * charge-conserving scheme keeps it at its initial value (zero for the pair
 * loading) to rounding.  res_dev: (nr+1)*(nz+1) doubles (device).
 * Asynchronous.  Errors: PIC_E_CONFIG, PIC_E_CUDA. */
int pic_gauss_residual(pic_ctx *ctx, double *res_dev);

/* Device pointers, counts and capacities of the context's state. */
int pic_get_view(pic_ctx *ctx, pic_view *out);

/* Checkpoint and resume.  pic_save writes the complete state of the method
 * at step n to a file: both species (counts, next ids, every particle field
 * in the context's precision), E^n, H^n, the wall tallies, the step index,
 * the blocking-capacitor state, the generator waveform set by pic_set_drive,
 * the carried node charge of the electrostatic model, the conducting ring's
 * conduction tally and the last Picard contraction (the speculation hint),
 * behind a header with the mesh and model.  pic_load restores them into a
 * context created with the same nr, nz, axis_cells, ring_cells, precision and
 * field model, with or without sigma_ring as the saving one, and with the
 * blocking capacitor on or off as there; the learned-start history restarts (the
 * first steps use the plain start).  A run resumed from a checkpoint takes
 * the same steps as the uninterrupted one (the collision random numbers
 * depend only on particle ids and the step index).  Both synchronise.
 * Errors: PIC_E_IO (file, or a checkpoint of another format version),
 * PIC_E_STATE (mesh, ring, model or precision differ, or counts beyond the
 * capacity), PIC_E_CUDA. */
int pic_save(pic_ctx *ctx, const char *path);
int pic_load(pic_ctx *ctx, const char *path);

/* Histogram of accepted sub-steps per particle over the state-writing push
 * passes (the commit or speculative final pass of each step): bin k (k < 15)
 * counts the particles that took k+1 sub-steps (an in-cell push is one; a
 * particle absorbed before its first sub-step counts in bin 0), bin 15 those
 * that took 16 or more.  A speculative final pass counts only when the step
 * adopts it.  enable = 1: clear the bins and count from the next
 * step on; 0: stop counting; -1: leave as is.  counts (nullable, host, 16
 * values): the bins as they stand before the call acts on enable (synchronises
 * the stream).  Off after pic_init.  Errors: PIC_E_CONFIG, PIC_E_CUDA. */
int pic_substep_histogram(pic_ctx *ctx, int enable, unsigned long long *counts);

/* The state of the method in caller-owned HOST memory: per species a
 * structure of arrays in the layout of pic_view (a..w in the context's
 * precision, pic_view.real_size bytes each; cell int32; id uint32), the
 * counts, next ids and step index, and optionally E^n, H^n in the Yee layouts
 * of pic_view.  Pinned host memory (cudaHostAlloc / cudaHostRegister) moves at
 * the host link's speed; pageable memory works, slower. */
typedef struct pic_host_state {
  long long n[2];             /* macro-particles per species (download: capacity of the arrays in,
                                 count out) */
  uint32_t next_id[2];
  long long step;             /* index n of the next step */
  int32_t *cell[2];
  void *a[2], *b[2], *vr[2], *vt[2], *vz[2], *w[2];
  uint32_t *id[2];
  double *er, *ez, *h;        /* nullable: fields not copied */
} pic_host_state;

/* Host -> device: copies the species arrays (and the fields given) into the
 * context and sets counts, next ids and step index as pic_set_counts does.
 * One cudaMemcpyAsync per array on the context's stream, so it returns before
 * the copies finish: the host memory must stay valid until the stream reaches
 * them (any later synchronising call, e.g. pic_state_download).
 * Errors: PIC_E_CONFIG (null ctx or state, a null array with n > 0),
 * PIC_E_STATE (n beyond capacity, negative counts or step), PIC_E_CUDA. */
int pic_state_upload(pic_ctx *ctx, const pic_host_state *in);

/* Device -> host: writes the counts, next ids and step index into *out and
 * copies the species arrays (and the fields where out->er/ez/h are given).
 * On entry out->n[s] is the capacity of the host arrays of species s.
 * Synchronises the stream.  Errors: PIC_E_CONFIG, PIC_E_STATE (host arrays
 * smaller than the counts; nothing is copied), PIC_E_CUDA. */
int pic_state_download(pic_ctx *ctx, pic_host_state *out);

/* Advances a state kept in caller-owned host memory (pinned, for the copies to
 * run asynchronously) by nsteps steps: per step the state is copied host ->
 * device, stepped (pic_step) and copied device -> host into the same arrays,
 * counts, next ids and step index updated; stats (nullable) receives the last
 * step's statistics with `pushes` summed over the nsteps steps.  The copies are pieces of at most 64 MB on two copy
 * streams of the context: the upload of a piece for step k+1 starts as soon
 * as the same piece of step k's result has landed on the host, so the
 * device -> host and host -> device copies overlap (the host link is full
 * duplex).  The same result as nsteps x (pic_state_upload, pic_step,
 * pic_state_download).  On entry hs->n[s] is the number of particles of
 * species s in the host state; the host arrays must hold the context's
 * capacity of each species (pic_get_view's cap), up to which the counts can
 * grow.  Returns after the last copy has finished.
 * Errors: those of pic_state_upload and pic_step (non-fatal PIC_E_SUBSTEP /
 * PIC_E_CAPACITY after all steps). */
int pic_step_host(pic_ctx *ctx, pic_host_state *hs, int nsteps, pic_step_stats *stats);

/* Set particle counts / next ids / step index after the caller wrote state
 * through pic_get_view.  Errors: PIC_E_STATE (count beyond capacity). */
int pic_set_counts(pic_ctx *ctx, long long ne, long long ni, uint32_t next_id_e,
                   uint32_t next_id_i, long long step);

/* Maximum collision frequencies used by the MCC (host values): electron
 * nu_max [1/s], ion g_max [m/s], null-collision probabilities. */
int pic_mcc_constants(pic_ctx *ctx, double *numax_e, double *gmax, double *pnull_e,
                      double *pnull_i);

/* Opt-in timing of the push+deposit launches (rows a2/a3/a6): enable != 0
 * creates CUDA events and records a pair around every push pass on the
 * context stream; totals are reset by every call.  Synchronises.
 * Errors: PIC_E_CUDA. */
int pic_profile(pic_ctx *ctx, int enable);

/* Accumulated device time [ms] of the timed push passes and the number of
 * push kernel launches they contained.  Synchronises.  Errors: PIC_E_CUDA. */
int pic_profile_read(pic_ctx *ctx, double *push_ms, long long *push_launches);

/* Allocation-free counting sort by cell.  The paper has no counterpart: this
 * entry point exists for callers that cannot give the library any device
 * memory of its own — a host code that reserves all device memory at
 * start-up and allows no allocation afterwards, or a plugin that only sees
 * the particle arrays.  It sorts n particles (SoA inputs cell..id, layout as
 * above, cell < 0 dropped) into the caller's output arrays (capacity >= n)
 * on `stream`, ascending by cell with the order inside a cell unspecified,
 * and returns the number kept in *n_out (host).  All scratch lives in one
 * static device array of about 3 MB per GPU, kept until the process exits;
 * it limits the grid to nr * nz <= 262144 cells (larger grids return
 * PIC_E_CONFIG).  Nothing is allocated: no cudaMalloc, no cudaFree.  The
 * first call on each device looks up the array's device address with
 * cudaGetSymbolAddress and keeps it for the process; do not call it again
 * after cudaDeviceReset on that device.  Every call reuses the same array, so
 * calls that overlap on the GPU (other streams, other threads) race:
 * serialise them.  Each call reads the kept count back to the host and
 * synchronises the stream, so it cannot be recorded into a stream capture.
 * Errors: PIC_E_CONFIG, PIC_E_CUDA. */
int pic_sort_cells_noalloc(int nr, int nz, long long n, const int32_t *cell_dev,
                           const double *a_dev, const double *b_dev, const double *vr_dev,
                           const double *vt_dev, const double *vz_dev, const double *w_dev,
                           const uint32_t *id_dev, int32_t *cell_out_dev, double *a_out_dev,
                           double *b_out_dev, double *vr_out_dev, double *vt_out_dev,
                           double *vz_out_dev, double *w_out_dev, uint32_t *id_out_dev,
                           void *stream, long long *n_out);

/* Self-check of the binary64 multiply the FP64 mover computes on the integer
 * pipes for products that feed no addition (IEEE 754 round to nearest, ties to
 * even, in 64-bit integer arithmetic; operands or results outside the normal
 * range take the hardware multiply).  The paper has no counterpart: it lets a
 * test compare out[i] = x[i] * y[i] bit for bit with any IEEE binary64
 * multiply.  x_dev, y_dev, out_dev: device arrays of n doubles (caller-owned);
 * runs on `stream` (NULL: the legacy default stream) and synchronises it.
 * Errors: PIC_E_CONFIG (n < 0, a null array with n > 0), PIC_E_CUDA. */
int pic_check_dmul(const double *x_dev, const double *y_dev, double *out_dev, long long n,
                   void *stream);

/* Throughput probe of the GPU's FP64 FMA pipe, the bound of the plain form's
 * mover.  The paper has no counterpart: it gives the measured peak that the
 * FP64 roofline fraction is quoted against.  blocks_per_sm x SMs blocks of
 * 256 threads each run 8 independent chains of `iters` fused multiply-adds on
 * the legacy default stream (one warm-up launch, one timed with CUDA events);
 * *seconds: the timed launch, *tflops: 2 flops per FMA over it.  Synchronises.
 * Errors: PIC_E_CONFIG (blocks_per_sm outside 1..8, iters < 1, null
 * outputs), PIC_E_CUDA. */
int pic_probe_dfma(int blocks_per_sm, int iters, double *seconds, double *tflops);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
