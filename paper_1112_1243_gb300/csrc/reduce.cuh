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

// BiCGStab finishers on three sums (v0, v1, v2); complex scalars z = (re, im)
DD_DEV void cdiv(double ar, double ai, double br, double bi, double& cr, double& ci) {
    double d = br * br + bi * bi;
    cr = (ar * br + ai * bi) / d;
    ci = (ai * br - ar * bi) / d;
}
// A zero denominator (Lanczos breakdown) ends the inner solve quietly: the
// outer FP64 loop restarts from the true residual.  Non-finite values are
// reported in the status word.
DD_DEV void bicg_fail(const Reduce& R, CGState& c, bool numeric = false) {
    c.active = 0;
    c.flags |= 4;
    if (numeric) {
        c.flags |= 2;
        raise_status(R.status, DD_ERR_NUMERIC);
    }
}
DD_DEV void finish3(const Reduce& R, int rhs, const double* s) {
    CGState& c = R.st[rhs];
    switch (R.op) {
        case FIN_BI_RHO: {  // s = (Re<rh,r>, Im<rh,r>, |r|^2): convergence, then beta
            c.rr = s[2];
            c.iters += 1;
            if (!isfinite(s[2]) || !isfinite(s[0]) || !isfinite(s[1])) {
                bicg_fail(R, c, true);
                break;
            }
            if (s[2] <= c.tol2) {
                c.active = 0;
                break;
            }
            if (c.iters >= c.maxit) {
                c.active = 0;
                c.flags |= 1;
                break;
            }
            // beta = (rho_new / rho) (alpha / omega)
            double qr, qi, wr, wi;
            cdiv(s[0], s[1], c.rho_re, c.rho_im, qr, qi);
            cdiv(c.al_re, c.al_im, c.om_re, c.om_im, wr, wi);
            c.be_re = qr * wr - qi * wi;
            c.be_im = qr * wi + qi * wr;
            c.rho_re = s[0];
            c.rho_im = s[1];
            if (!(s[0] * s[0] + s[1] * s[1] > 0.0) || !isfinite(c.be_re) || !isfinite(c.be_im)) bicg_fail(R, c);
            break;
        }
        case FIN_BI_ALPHA: {  // s = (Re<rh,v>, Im<rh,v>): alpha = rho / <rh,v>
            double ar, ai;
            if (!isfinite(s[0]) || !isfinite(s[1])) {
                bicg_fail(R, c, true);
                break;
            }
            if (!(s[0] * s[0] + s[1] * s[1] > 0.0)) {
                bicg_fail(R, c);
                break;
            }
            cdiv(c.rho_re, c.rho_im, s[0], s[1], ar, ai);
            c.al_re = ar;
            c.al_im = ai;
            if (!isfinite(ar) || !isfinite(ai)) bicg_fail(R, c);
            break;
        }
        case FIN_BI_OMEGA: {  // s = (Re<t,s>, Im<t,s>, |t|^2): omega = <t,s> / |t|^2
            if (!isfinite(s[0]) || !isfinite(s[1]) || !isfinite(s[2])) {
                bicg_fail(R, c, true);
                break;
            }
            if (!(s[2] > 0.0)) {
                bicg_fail(R, c);
                break;
            }
            c.om_re = s[0] / s[2];
            c.om_im = s[1] / s[2];
            if (!isfinite(c.om_re) || !isfinite(c.om_im)) bicg_fail(R, c);
            break;
        }
        default:
            break;
    }
}

// Three-value variant: partials [rhs][gridDim.x][3].  `sh` needs 34 doubles.
DD_DEV void grid_reduce3(const Reduce& R, int rhs, const double* v, double* sh) {
    double b[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] = block_sum(v[k], sh);
    int* last = reinterpret_cast<int*>(&sh[33]);
    if (threadIdx.x == 0) {
        double* p = R.partials + ((long long)rhs * gridDim.x + blockIdx.x) * 3;
        p[0] = b[0];
        p[1] = b[1];
        p[2] = b[2];
        __threadfence();
        unsigned t = atomicAdd(&R.counters[rhs], 1u);
        *last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (*last) {
        __threadfence();
        double s[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double a = 0.0;
            for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
                a += __ldcg(&R.partials[((long long)rhs * gridDim.x + i) * 3 + k]);
            s[k] = block_sum(a, sh);
        }
        if (threadIdx.x == 0) {
            finish3(R, rhs, s);
            R.counters[rhs] = 0;
        }
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
