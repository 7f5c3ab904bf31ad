// Deterministic two-stage grid reduction with a finisher run by the last
// thread block (ticket counter), so that Krylov scalars are formed on the
// device without a host round trip.  Partial sums are FP64; the final sum is
// taken in a fixed order, so results do not depend on block scheduling.
#pragma once

#include "dd_internal.h"

DD_DEV void finish(const Reduce& R, int rhs, double s) {
    switch (R.op) {
        case FIN_STORE:
            R.out[rhs] = s;
            break;
        case FIN_ALPHA: {  // alpha = zz / |A p|^2
            CGState& c = R.st[rhs];
            c.qq = s;
            double a = c.zz / s;
            if (!(s > 0.0) || !isfinite(a)) {
                c.alpha = 0.0;
                c.active = 0;
                c.flags |= 2;
                raise_status(R.status, DD_ERR_NUMERIC);
            } else {
                c.alpha = a;
            }
            break;
        }
        case FIN_RR: {  // convergence test on the recursive residual
            CGState& c = R.st[rhs];
            c.rr = s;
            c.iters += 1;
            if (!isfinite(s)) {
                c.active = 0;
                c.flags |= 2;
                raise_status(R.status, DD_ERR_NUMERIC);
            } else if (s <= c.tol2) {
                c.active = 0;
            } else if (c.iters >= c.maxit) {
                c.active = 0;
                c.flags |= 1;
            }
            break;
        }
        case FIN_BETA: {  // beta = |z_new|^2 / |z_old|^2
            CGState& c = R.st[rhs];
            c.beta = (c.zz > 0.0) ? s / c.zz : 0.0;
            c.zz = s;
            break;
        }
        case FIN_ZZ_INIT: {  // first z: p = z, beta = 0
            CGState& c = R.st[rhs];
            c.zz = s;
            c.beta = 0.0;
            if (!(s > 0.0)) c.active = 0;  // zero right-hand side: nothing to do
            break;
        }
        default:
            break;
    }
}

// Every thread of the block calls this with its contribution.  `sh` needs 34 doubles.
DD_DEV void grid_reduce(const Reduce& R, int rhs, double v, double* sh) {
    double bsum = block_sum(v, sh);
    int* last = reinterpret_cast<int*>(&sh[33]);
    if (threadIdx.x == 0) {
        R.partials[(long long)rhs * gridDim.x + blockIdx.x] = bsum;
        __threadfence();
        unsigned t = atomicAdd(&R.counters[rhs], 1u);
        *last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (*last) {
        __threadfence();
        double s = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
            s += __ldcg(&R.partials[(long long)rhs * gridDim.x + i]);
        s = block_sum(s, sh);
        if (threadIdx.x == 0) {
            finish(R, rhs, s);
            R.counters[rhs] = 0;
        }
    }
}
