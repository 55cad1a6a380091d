/* Batched ensembles of independent discharges (C ABI).
 *
 * The method (Sec. 2.1) advances one discharge at a time; an ensemble runs
 * several independent discharges of any sizes side by side on one GPU.  Each
 * member is an ordinary pic_ctx (its own workspace and CUDA stream, created
 * with pic_init and loaded by the caller).  pic_ensemble_step advances all
 * members by whole steps: the Picard passes of the members are issued
 * together (one per member and round, each replayed from a CUDA graph
 * captured once per buffer configuration), so that kernels of different
 * members overlap on the GPU, with one host wait per round; members leave the
 * round loop as they converge.  Results are identical to stepping each
 * member alone with pic_step.
 *
 * pic_ensemble_tune times candidate grid sizes of the persistent push kernels
 * (the particle tile each block strides over) on the ensemble's own state and
 * keeps the fastest.
 *
 * Errors: PIC_OK or a negative PIC_E_* code of pic.h; the ensemble owns no
 * device memory and does not own its members (destroy them after it).
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

/* n members (1..PIC_ENSEMBLE_MAX), distinct, each ready to step; turns graph
 * replay on for every member.  PIC_E_CONFIG on invalid arguments. */
int pic_ensemble_create(pic_ctx *const *members, int n, pic_ensemble **out);
void pic_ensemble_destroy(pic_ensemble *ens);

/* Advances every member by nsteps; stats (nullable) receives the last step's
 * statistics of each member (n entries).  The first member error stops the
 * call and is returned; non-fatal codes (PIC_E_CAPACITY, PIC_E_SUBSTEP) are
 * returned after the step. */
int pic_ensemble_step(pic_ensemble *ens, int nsteps, pic_step_stats *stats);

/* Times `rounds` Picard rounds of the whole ensemble for each candidate grid
 * fraction (1, 1/2, 1/4 of one resident wave of the push kernels), applies the
 * fastest and returns it in *frac_out (nullable) with the times per round in
 * ms_out[3] (nullable).  Changes no particle or field state. */
int pic_ensemble_tune(pic_ensemble *ens, int rounds, float *frac_out, double *ms_out);

#ifdef __cplusplus
}
#endif

#endif /* PIC_ENSEMBLE_H */
