// Batched conjugate gradient on the even-odd normal equations and the
// mixed-precision defect-correction driver (declarations shared by the
// translation units that run global solves).
#pragma once

#include "dd_internal.h"

// Solve D x = b for nrhs systems whose right-hand sides are already packed
// into h->vecs[0].be / .bo (FP64 eo chunks, system r at offset r*12*Vh).
// System r uses the gauge field of slot field0 + r*field_step (field_step 0:
// one shared field, 1: consecutive slots), formatted in eo64 and in the
// inner precision.  On return vecs[0].xe / .xo hold the solution.
// relres (host, nrhs, may be null) receives ||b - D x|| / ||b||, iters (may
// be null) the total inner iterations.  prec: DD_PREC_F64 (plain FP64 CG) or
// DD_PREC_F32 / DD_PREC_F16 (inner solver in that precision, FP64 defect
// correction).  Returns DD_ERR_NOT_CONVERGED if maxit was reached.
// mask = 0: the whole operator D; mask = 1: the Dirichlet block operators
// D_bb + D_ww (every hop that leaves a block dropped), i.e. all block solves
// of the right-hand side's blocks at once, even-odd preconditioned (hops
// inside a block still connect opposite site parities).  colour = 0 / 1
// (mask 1 only): the right-hand sides vanish outside the blocks of that
// colour, so only that colour's sites are visited (the other colour of the
// solution is left as it was).
int solve_packed(dd_handle* h, int nrhs, int field0, int field_step, int prec, double tol, int maxit, int* iters,
                 double* relres, int mask = 0, int colour = -1);
