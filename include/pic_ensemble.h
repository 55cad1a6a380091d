/* Batched ensembles of independent discharges (C ABI).
 *
 * The method (Sec. 2.1) advances one discharge at a time; an ensemble runs
 * several independent discharges of any sizes side by side on one GPU.  Each
 * member is an ordinary pic_ctx (its own workspace and CUDA stream, created
 * with pic_init and loaded by the caller).  pic_ensemble_step advances all
 * members by whole steps in rounds: one Picard pass of every unconverged
 * member per round, then one host wait; members leave the round loop as they
 * converge.  A round is issued in one of two ways:
 *   persistent (the default when every member has the same precision, both
 *     species moving, no magnetic field): each member's pre-push part (E^{n+1/2}
 *     and cleared currents) on its own stream, then on the ensemble's lead
 *     stream, per species, one launch of the fast and one of the general push
 *     kernel over every active member (work items = (member, virtual block);
 *     each member's launch parameters are uploaded per round), then each
 *     member's field solve on its own stream;
 *   per member: each member's whole pass replayed from a CUDA graph captured
 *     once per buffer configuration, the members' kernels overlapping on the GPU.
 * Both give the same particles, fields and counts as stepping each member alone
 * with pic_step (up to the summation order of the crossed charge).
 *
 * pic_ensemble_tune times whole rounds on the ensemble's own state for the
 * candidates (per member | persistent) x (virtual grid of the push kernels:
 * 1, 1/2, 1/4 of one resident wave, i.e. 1, 2, 4 particle tiles of 256 per
 * block visit) and keeps the fastest.  The sort has no bin size to tune (it
 * sorts by cell).
 *
 * Errors: PIC_OK or a negative PIC_E_* code of pic.h.  The ensemble owns a
 * CUDA stream, events, 2 x ~90 KB of pinned host and device memory for the
 * launch parameters, and none of its members (destroy them after it).
 */
#ifndef PIC_ENSEMBLE_H
#define PIC_ENSEMBLE_H

#include "pic.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ENSEMBLE_MAX 64

typedef struct pic_ensemble pic_ensemble;

/* Replays the Picard passes of ctx from captured CUDA graphs (on = 1) or
 * launches them kernel by kernel (on = 0, the default).  Capture needs a
 * created stream: a context on the legacy default stream (stream 0) always
 * launches kernel by kernel. */
int pic_set_graphs(pic_ctx *ctx, int on);

/* The Picard iteration of Sec. 2.1 run on the device (on = 1, the default):
 * with graph replay on and pic_profile off, each step launches one graph per
 * buffer configuration whose conditional while-node repeats the pass (the
 * speculative or the plain one, chosen by an if/else node), the convergence
 * test on the device (the same residual, tolerance, iteration limit and
 * speculation rule as the host loop) and the copy of the new iterate, until
 * the residual is below the tolerance, not finite, or the limit is reached;
 * the host waits once for the loop instead of once per pass.  The results
 * are those of the host loop (the same kernels in the same order).  on = 0,
 * graphs off, timing on, the context's first pass, or a driver without
 * conditional graph nodes: the host loop.  PIC_E_CONFIG for on not 0 or 1. */
int pic_set_device_picard(pic_ctx *ctx, int on);

/* n members (1..PIC_ENSEMBLE_MAX), distinct, each ready to step; turns graph
 * replay on for every member and chooses persistent rounds where the members
 * allow them.  PIC_E_CONFIG on invalid arguments, PIC_E_CUDA when the stream,
 * events or staging cannot be created. */
int pic_ensemble_create(pic_ctx *const *members, int n, pic_ensemble **out);
void pic_ensemble_destroy(pic_ensemble *ens);

/* Persistent rounds on (1) or per-member rounds (0).  PIC_E_CONFIG when on = 1
 * and the members do not allow persistent rounds (precisions differ, fixed
 * ions, a magnetic field). */
int pic_ensemble_set_persistent(pic_ensemble *ens, int on);

/* Advances every member by nsteps; stats (nullable) receives the last step's
 * statistics of each member (n entries).  The first member error stops the
 * call and is returned; non-fatal codes (PIC_E_CAPACITY, PIC_E_SUBSTEP) are
 * returned after the step. */
int pic_ensemble_step(pic_ensemble *ens, int nsteps, pic_step_stats *stats);

/* Times `rounds` Picard rounds of the whole ensemble for each candidate:
 * c = 0..2 per-member rounds and c = 3..5 persistent rounds, with the push
 * kernels' grid fraction 1, 1/2, 1/4 of one resident wave (c % 3); applies the
 * fastest and returns its fraction in *frac_out and 1 if persistent in
 * *persistent_out (both nullable), with the best time per round of each
 * candidate in ms_out[6] (nullable; -1 for a candidate the members do not
 * allow).  Changes no particle or field state. */
int pic_ensemble_tune(pic_ensemble *ens, int rounds, float *frac_out, int *persistent_out,
                      double *ms_out);

#ifdef __cplusplus
}
#endif

#endif /* PIC_ENSEMBLE_H */
