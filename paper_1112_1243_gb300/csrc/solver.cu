// Global Krylov solves (Sec. 4: every factor of the stochastic estimate
// needs one solve; these are the inversions behind the acceptance steps).
//
// D x = b is solved through the even-site Schur complement
//   Dtilde = 1 - kappa^2 H_eo H_oe,  b~ = b_e + kappa H_eo b_o,
//   x_e = Dtilde^{-1} b~,  x_o = b_o + kappa H_oe x_e.
// The plain FP64 path runs CG on the normal equations Dtilde^dag Dtilde
// (CGNR, Dtilde^dag = gamma5 Dtilde gamma5) in FP64.  The mixed path runs
// CGNR or BiCGStab on Dtilde with FP32 arithmetic on FP32 or FP16 storage
// as the inner solver of an FP64 defect-correction loop:
//   r = b~ - Dtilde x (FP64), solve Dtilde e = r roughly, x += e,
// until ||r|| <= tol ||b|| (that is the true residual of D x = b, because
// x_o is formed exactly from x_e).  With outer_prec = DD_PREC_DF64 the
// residual, x and b~ are held in double-float arithmetic instead (see
// dfhop.cuh).  All Krylov scalars are FP64 grid reductions finished on the
// device; the host only checks convergence flags every few iterations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dfhop.cuh"
#include "dslash.cuh"
#include "solver.h"

namespace {

// ------------------------------------------------------------- BLAS kernels
template <class R, class SM, class SH>
__global__ void __launch_bounds__(128) cg_xr_kernel(SiteSet S, SM x, SM r, SM p, SM q, SH rh, int copy,
                                                    const CGState* st, Reduce red) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const R alpha = (R)st[rhs].alpha;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double nrm = 0.0;
    if (ti < S.n) {
        const long long i = S.at(ti);
        SM xr = at_rhs(x, rhs), rr = at_rhs(r, rhs), pr = at_rhs(p, rhs), qr = at_rhs(q, rhs);
        Spinor<R> a, b;
        xr.load(i, a);
        pr.load(i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] + alpha * b.c[k];
        xr.store(i, a);
        rr.load(i, a);
        qr.load(i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] - alpha * b.c[k];
        rr.store(i, a);
        if (copy) at_rhs(rh, rhs).store(i, a);
        nrm = (double)snorm2(a);
    }
    grid_reduce(red, rhs, nrm, sh);
}

template <class R, class SM, class SH>
__global__ void __launch_bounds__(128) cg_p_kernel(SiteSet S, SM p, SM z, SH ph, int copy, const CGState* st) {
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const double beta = st[rhs].beta;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    SM pr = at_rhs(p, rhs), zr = at_rhs(z, rhs);
    Spinor<R> a, b;
    zr.load(i, a);
    if (beta != 0.0) {
        pr.load(i, b);
        const R bt = (R)beta;
#pragma unroll
        for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] + bt * b.c[k];
    }
    pr.store(i, a);
    if (copy) at_rhs(ph, rhs).store(i, a);
}

// start an inner solve: x = 0, r = r0 (copied into the hop copy), states armed
template <class R, class SM, class SH>
__global__ void cg_start_kernel(SiteSet S, SM x, SM r, SH rh, int copy, CGState* st, const CGState* outer) {
    const int rhs = blockIdx.y;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (outer && !outer[rhs].active) return;
    if (ti < S.n) {
        const long long i = S.at(ti);
        Spinor<R> z;
        zero(z);
        at_rhs(x, rhs).store(i, z);
        if (copy) {
            Spinor<R> a;
            at_rhs(r, rhs).load(i, a);
            at_rhs(rh, rhs).store(i, a);
        }
    }
}

__global__ void cg_arm_kernel(int nrhs, CGState* st, const CGState* outer, const double* rr0, double tol,
                              double abs_fac, int maxit) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    CGState c;
    c.zz = c.qq = c.alpha = c.beta = 0.0;
    c.rr = rr0[r];
    // relative target tol^2 |r0|^2, or a fraction of the outer absolute target.
    // A mixed inner solve is asked for no more than the outer loop still
    // needs: when ||r_outer|| is within 1/tol_inner of the outer target, the
    // relative target rises to 0.3 target / ||r_outer|| (capped at 0.1), so the
    // last defect cycle does not over-solve.
    double rel2 = tol * tol;
    if (abs_fac < 0.0 && outer && outer[r].rr > 0.0)
        rel2 = fmin(fmax(rel2, 0.09 * outer[r].tol2 / outer[r].rr), 0.01);
    c.tol2 = (abs_fac > 0.0 && outer) ? abs_fac * outer[r].tol2 : rel2 * rr0[r];
    c.active = (outer ? outer[r].active : 1) && rr0[r] > 0.0;
    c.iters = 0;
    c.maxit = maxit;
    c.flags = 0;
    st[r] = c;
}

// outer (defect-correction) bookkeeping: active while rr > tol2; a
// non-finite true residual ends the system and is reported as NUMERIC
__global__ void outer_update_kernel(int nrhs, CGState* outer, const double* rr, int* status) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    outer[r].rr = rr[r];
    if (!isfinite(rr[r])) {
        outer[r].active = 0;
        outer[r].flags |= 2;
        raise_status(status, DD_ERR_NUMERIC);
        return;
    }
    outer[r].active = outer[r].active && (rr[r] > outer[r].tol2);
}
__global__ void outer_arm_kernel(int nrhs, CGState* outer, const double* bb, double tol) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    CGState c;
    c.zz = c.qq = c.alpha = c.beta = 0.0;
    c.rr = bb[r];
    c.tol2 = tol * tol * bb[r];
    c.active = bb[r] > 0.0;
    c.iters = 0;
    c.maxit = 0;
    c.flags = 0;
    outer[r] = c;
}

// x64 += scale * e (any storage; scale = |r_outer| when the inner system was
// normalised, rr = null: 1), r64 = b - t (with |r|^2), v = 0, copies
template <class SE>
__global__ void add_correction_kernel(SiteSet S, SpinorF64 x, SE e, const double* rr, const CGState* outer) {
    const int rhs = blockIdx.y;
    if (outer && !outer[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    const double sc = rr ? sqrt(rr[rhs]) : 1.0;
    Spinor<double> a, b;
    at_rhs(x, rhs).load(i, a);
    at_rhs(e, rhs).load(i, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] + sc * b.c[k];
    at_rhs(x, rhs).store(i, a);
}
// out = in / |in| (|in|^2 given per rhs): the inner solver always sees a
// unit-norm right-hand side, so FP32 squares neither underflow nor overflow
template <class SOut>
__global__ void normalised_copy_kernel(SiteSet S, SpinorF64 in, SOut out, const double* rr, const CGState* outer) {
    const int rhs = blockIdx.y;
    if (outer && !outer[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    const double inv = rr[rhs] > 0.0 ? 1.0 / sqrt(rr[rhs]) : 0.0;
    Spinor<double> a;
    at_rhs(in, rhs).load(i, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) a.c[k] = inv * a.c[k];
    at_rhs(out, rhs).store(i, a);
}
__global__ void fill_kernel(int n, double* p, double v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void __launch_bounds__(128) residual_kernel(SiteSet S, SpinorF64 b, SpinorF64 t, SpinorF64 r,
                                                       const CGState* outer, Reduce red) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    if (outer && !outer[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double nrm = 0.0;
    if (ti < S.n) {
        const long long i = S.at(ti);
        Spinor<double> a, c;
        at_rhs(b, rhs).load(i, a);
        at_rhs(t, rhs).load(i, c);
#pragma unroll
        for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] - c.c[k];
        at_rhs(r, rhs).store(i, a);
        nrm = snorm2(a);
    }
    grid_reduce(red, rhs, nrm, sh);
}
template <class SV>
__global__ void __launch_bounds__(128) norm2_kernel(SiteSet S, SV v, Reduce red) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double nrm = 0.0;
    if (ti < S.n) {
        const long long i = S.at(ti);
        Spinor<double> a;
        at_rhs(v, rhs).load(i, a);
        nrm = snorm2(a);
    }
    grid_reduce(red, rhs, nrm, sh);
}
template <class SIn, class SOut>
__global__ void copy_kernel(SiteSet S, SIn in, SOut out, const CGState* outer) {
    const int rhs = blockIdx.y;
    if (outer && !outer[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    Spinor<double> a;
    at_rhs(in, rhs).load(i, a);
    at_rhs(out, rhs).store(i, a);
}
__global__ void zero64_kernel(SiteSet S, SpinorF64 v) {
    const int rhs = blockIdx.y;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    Spinor<double> z;
    zero(z);
    at_rhs(v, rhs).store(i, z);
}

// ------------------------------------------------------------ CGNR runner
template <class R, class SM, class SH, class LK, int MASK = 0>
struct NormalCG {
    dd_handle* h;
    int nrhs;
    SM x, r, p, q, z;
    SH ph, rh, th;
    int copies;
    LK lk;
    long long lk_rs;
    CGState* st;
    const CGState* outer;
    SiteSet S;  // the sites of the solve (all even sites, or one block colour's)

    Reduce red(int op) const {
        Reduce R_;
        R_.partials = h->d_partials;
        R_.counters = h->d_counters;
        R_.st = st;
        R_.out = nullptr;
        R_.op = op;
        R_.status = h->d_status;
        return R_;
    }
    template <class SIn, class SX, class SOut>
    HopArgs<SIn, SX, SOut, LK> args(int par, SIn in, SX xin, SOut out, double a, double b, int hasx, int g5in,
                                    int g5out, int op) const {
        HopArgs<SIn, SX, SOut, LK> A;
        A.g = h->g;
        A.p = par;
        A.in = in;
        A.xin = xin;
        A.out = out;
        A.lk = lk;
        A.lk_rhs_stride = lk_rs;
        A.a = a;
        A.b = b;
        A.has_x = hasx;
        A.g5in = g5in;
        A.g5out = g5out;
        A.colour_mask = 3;
        A.st = st;
        A.red = red(op);
        A.S = S;
        return A;
    }
    // z = Dtilde^dag r  (two hops), |z|^2 -> op
    void apply_dag_r(int op) {
        const double k2 = h->prm.kappa * h->prm.kappa;
        launch_hop<R, SH, SM, SH, LK, MASK>(args(1, rh, r, th, 0.0, 1.0, 0, 1, 0, FIN_NONE), nrhs, h);
        launch_hop<R, SH, SM, SM, LK, MASK>(args(0, th, r, z, 1.0, -k2, 1, 0, 1, op), nrhs, h);
    }
    // q = Dtilde p, |q|^2 -> alpha
    void apply_p() {
        const double k2 = h->prm.kappa * h->prm.kappa;
        launch_hop<R, SH, SM, SH, LK, MASK>(args(1, ph, p, th, 0.0, 1.0, 0, 0, 0, FIN_NONE), nrhs, h);
        launch_hop<R, SH, SM, SM, LK, MASK>(args(0, th, p, q, 1.0, -k2, 1, 0, 0, FIN_ALPHA), nrhs, h);
    }
    // solve Dtilde x = r (r holds the right-hand side; x starts at 0)
    int run(const double* rr0, double tol, double abs_fac, int maxit, int chunk, int* iters_out) {
        dim3 grid(grid_for(S.n, 128), nrhs);
        if (maxit < 1) maxit = 1;
        DD_KLAUNCH(h, cg_arm_kernel<<<1, 64, 0, h->stream>>>(nrhs, st, outer, rr0, tol, abs_fac, maxit));
        DD_KLAUNCH(h, cg_start_kernel<R, SM, SH><<<grid, 128, 0, h->stream>>>(S, x, r, rh, copies, st, outer));
        apply_dag_r(FIN_ZZ_INIT);
        DD_KLAUNCH(h, cg_p_kernel<R, SM, SH><<<grid, 128, 0, h->stream>>>(S, p, z, ph, copies, st));
        std::vector<CGState> hs(nrhs);
        int done_iters = 0;
        bool polled = false;
        auto body = [&]() -> int {
            for (int it = 0; it < chunk; ++it) {
                apply_p();
                DD_KLAUNCH(h, cg_xr_kernel<R, SM, SH><<<grid, 128, 0, h->stream>>>(S, x, r, p, q, rh, copies, st, red(FIN_RR)));
                apply_dag_r(FIN_BETA);
                DD_KLAUNCH(h, cg_p_kernel<R, SM, SH><<<grid, 128, 0, h->stream>>>(S, p, z, ph, copies, st));
            }
            return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
        };
        // eager: poll the states every chunk iterations
        auto more = [&](bool& m) -> int {
            done_iters += chunk;
            if (cudaMemcpyAsync(hs.data(), st, sizeof(CGState) * nrhs, cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess)
                return DD_ERR_CUDA;
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DD_ERR_CUDA;
            polled = true;
            bool any = false;
            for (int k = 0; k < nrhs; ++k) any = any || hs[k].active;
            m = any && done_iters < maxit + chunk;
            return DD_OK;
        };
        const LoopCond lc{st, nrhs, (maxit + 2 * chunk - 1) / chunk, nullptr, 0, 1};
        int rc = dd_loop(h, body, more, lc);
        if (rc || !polled) return rc;  // captured: breakdowns are raised on the device
        int tot = 0, flags = 0;
        for (int k = 0; k < nrhs; ++k) {
            tot += hs[k].iters;
            flags |= hs[k].flags;
        }
        if (iters_out) *iters_out += tot;
        if (flags & 2) return DD_ERR_NUMERIC;
        return DD_OK;
    }
};

// ------------------------------------------------------------ BiCGStab
// van der Vorst's BiCGStab on Dtilde itself (no normal equations), complex
// scalars formed on the device:
//   rho = <rh, r>, beta = (rho / rho_old)(alpha / omega), p = r + beta (p - omega v),
//   v = A p, alpha = rho / <rh, v>, s = r - alpha v, t = A s,
//   omega = <t, s> / <t, t>, x += alpha p + omega s, r = s - omega t.
template <class R>
DD_DEV cpx<R> cscal(double re, double im) {
    return mk<R>((R)re, (R)im);
}

// p and rhat live only in the hop storage SH: the rounded p is the one that
// both v = Dtilde p and x += alpha p use, and rhat (any fixed vector) is the
// rounded r0.
template <class R, class SM, class SH>
__global__ void bicg_start_kernel(SiteSet S, SM x, SM r, SH rhat, SH p, SM v, const CGState* outer) {
    const int rhs = blockIdx.y;
    if (outer && !outer[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    Spinor<R> z, a;
    zero(z);
    at_rhs(x, rhs).store(i, z);
    at_rhs(p, rhs).store(i, z);
    at_rhs(v, rhs).store(i, z);
    at_rhs(r, rhs).load(i, a);
    at_rhs(rhat, rhs).store(i, a);
}

__global__ void bicg_arm_kernel(int nrhs, CGState* st) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    CGState& c = st[r];
    c.rho_re = c.al_re = c.om_re = 1.0;
    c.rho_im = c.al_im = c.om_im = 0.0;
    c.be_re = c.be_im = 0.0;
}

template <class R, class SM, class SH>
__global__ void __launch_bounds__(128) bicg_rho_kernel(SiteSet S, SH rhat, SM r, const CGState* st, Reduce red) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (ti < S.n) {
        const long long i = S.at(ti);
        Spinor<R> a, b;
        at_rhs(rhat, rhs).load(i, a);
        at_rhs(r, rhs).load(i, b);
        R d0 = 0, d1 = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            d0 += a.c[k].x * b.c[k].x + a.c[k].y * b.c[k].y;
            d1 += a.c[k].x * b.c[k].y - a.c[k].y * b.c[k].x;
        }
        v[0] = (double)d0;
        v[1] = (double)d1;
        v[2] = (double)snorm2(b);
    }
    grid_reduce3(red, rhs, v, sh);
}

// p = r + beta (p - omega v)
template <class R, class SM, class SH>
__global__ void __launch_bounds__(128) bicg_p_kernel(SiteSet S, SH p, SM r, SM v, const CGState* st) {
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    const CGState& c = st[rhs];
    const cpx<R> be = cscal<R>(c.be_re, c.be_im), om = cscal<R>(c.om_re, c.om_im);
    Spinor<R> pp, rr, vv;
    at_rhs(p, rhs).load(i, pp);
    at_rhs(r, rhs).load(i, rr);
    at_rhs(v, rhs).load(i, vv);
#pragma unroll
    for (int k = 0; k < 12; ++k) pp.c[k] = rr.c[k] + cmul(be, pp.c[k] - cmul(om, vv.c[k]));
    at_rhs(p, rhs).store(i, pp);
}

// s = r - alpha v, hop copy of s
template <class R, class SM, class SH>
__global__ void __launch_bounds__(128) bicg_s_kernel(SiteSet S, SM s, SM r, SM v, SH shop, int copy,
                                                     const CGState* st) {
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    const CGState& c = st[rhs];
    const cpx<R> al = cscal<R>(c.al_re, c.al_im);
    Spinor<R> rr, vv;
    at_rhs(r, rhs).load(i, rr);
    at_rhs(v, rhs).load(i, vv);
#pragma unroll
    for (int k = 0; k < 12; ++k) rr.c[k] = rr.c[k] - cmul(al, vv.c[k]);
    at_rhs(s, rhs).store(i, rr);
    if (copy) at_rhs(shop, rhs).store(i, rr);
}

// x += alpha p + omega s, r = s - omega t; <rh, r>, |r|^2 -> FIN_BI_RHO
template <class R, class SM, class SH>
__global__ void __launch_bounds__(128) bicg_xr_kernel(SiteSet S, SM x, SM r, SH p, SM s, SM t, SH rhat,
                                                      const CGState* st, Reduce red) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (ti < S.n) {
        const long long i = S.at(ti);
        const CGState& c = st[rhs];
        const cpx<R> al = cscal<R>(c.al_re, c.al_im), om = cscal<R>(c.om_re, c.om_im);
        Spinor<R> xx, pp, ss, tt, rh;
        at_rhs(x, rhs).load(i, xx);
        at_rhs(p, rhs).load(i, pp);
        at_rhs(s, rhs).load(i, ss);
#pragma unroll
        for (int k = 0; k < 12; ++k) xx.c[k] = xx.c[k] + cmul(al, pp.c[k]) + cmul(om, ss.c[k]);
        at_rhs(x, rhs).store(i, xx);
        at_rhs(t, rhs).load(i, tt);
#pragma unroll
        for (int k = 0; k < 12; ++k) ss.c[k] = ss.c[k] - cmul(om, tt.c[k]);
        at_rhs(r, rhs).store(i, ss);
        at_rhs(rhat, rhs).load(i, rh);
        R d0 = 0, d1 = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            d0 += rh.c[k].x * ss.c[k].x + rh.c[k].y * ss.c[k].y;
            d1 += rh.c[k].x * ss.c[k].y - rh.c[k].y * ss.c[k].x;
        }
        v[0] = (double)d0;
        v[1] = (double)d1;
        v[2] = (double)snorm2(ss);
    }
    grid_reduce3(red, rhs, v, sh);
}

template <class R, class SM, class SH, class LK, int MASK = 0>
struct BiCGStab {
    dd_handle* h;
    int nrhs;
    SM x, r, v, s, t;
    SH p, rhat, shop, th;  // p and rhat only in hop storage; shop: hop copy of s
    int copies;
    LK lk;
    long long lk_rs;
    CGState* st;
    const CGState* outer;
    SiteSet S;  // the sites of the solve (all even sites, or one block colour's)

    Reduce red(int op) const {
        Reduce R_;
        R_.partials = h->d_partials;
        R_.counters = h->d_counters;
        R_.st = st;
        R_.out = nullptr;
        R_.op = op;
        R_.status = h->d_status;
        return R_;
    }
    template <class SIn, class SX, class SOut>
    HopArgs<SIn, SX, SOut, LK> args(int par, SIn in, SX xin, SOut out, double a, double b, int hasx, int op,
                                    int red3) const {
        HopArgs<SIn, SX, SOut, LK> A;
        A.g = h->g;
        A.p = par;
        A.in = in;
        A.xin = xin;
        A.out = out;
        A.lk = lk;
        A.lk_rhs_stride = lk_rs;
        A.a = a;
        A.b = b;
        A.has_x = hasx;
        A.g5in = 0;
        A.g5out = 0;
        A.colour_mask = 3;
        A.st = st;
        A.red = red(op);
        A.red3 = red3;
        if constexpr (std::is_same<SX, SH>::value)
            A.rhat = rhat;  // read by the red3 == 1 form only
        else
            A.rhat = xin;
        A.S = S;
        return A;
    }
    // out = Dtilde in_h (in_m: the same vector in the storage of the xpay term)
    template <class SX>
    void apply(SH in_h, SX in_m, SM out, int op, int red3) {
        const double k2 = h->prm.kappa * h->prm.kappa;
        launch_hop<R, SH, SM, SH, LK, MASK>(args(1, in_h, v, th, 0.0, 1.0, 0, FIN_NONE, 0), nrhs, h);
        launch_hop<R, SH, SX, SM, LK, MASK>(args(0, th, in_m, out, 1.0, -k2, 1, op, red3), nrhs, h);
    }
    // solve Dtilde x = r (r holds the right-hand side; x starts at 0)
    int run(const double* rr0, double tol, double abs_fac, int maxit, int chunk, int* iters_out) {
        dim3 grid(grid_for(S.n, 128), nrhs);
        if (maxit < 1) maxit = 1;
        DD_KLAUNCH(h, cg_arm_kernel<<<1, 64, 0, h->stream>>>(nrhs, st, outer, rr0, tol, abs_fac, maxit));
        DD_KLAUNCH(h, bicg_arm_kernel<<<1, 64, 0, h->stream>>>(nrhs, st));
        DD_KLAUNCH(h, bicg_start_kernel<R, SM, SH><<<grid, 128, 0, h->stream>>>(S, x, r, rhat, p, v, outer));
        DD_KLAUNCH(h, bicg_rho_kernel<R, SM, SH><<<grid, 128, 0, h->stream>>>(S, rhat, r, st, red(FIN_BI_RHO)));
        std::vector<CGState> hs(nrhs);
        int done = 0;
        bool polled = false;
        auto body = [&]() -> int {
            for (int it = 0; it < chunk; ++it) {
                DD_KLAUNCH(h, bicg_p_kernel<R, SM, SH><<<grid, 128, 0, h->stream>>>(S, p, r, v, st));
                apply(p, p, v, FIN_BI_ALPHA, 1);
                DD_KLAUNCH(h, bicg_s_kernel<R, SM, SH><<<grid, 128, 0, h->stream>>>(S, s, r, v, shop, copies, st));
                apply(shop, s, t, FIN_BI_OMEGA, 2);
                DD_KLAUNCH(h, bicg_xr_kernel<R, SM, SH><<<grid, 128, 0, h->stream>>>(S, x, r, p, s, t, rhat, st,
                                                                                     red(FIN_BI_RHO)));
            }
            return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
        };
        auto more = [&](bool& m) -> int {
            done += chunk;
            if (cudaMemcpyAsync(hs.data(), st, sizeof(CGState) * nrhs, cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess)
                return DD_ERR_CUDA;
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DD_ERR_CUDA;
            polled = true;
            bool any = false;
            for (int k = 0; k < nrhs; ++k) any = any || hs[k].active;
            m = any && done < maxit + chunk;
            return DD_OK;
        };
        // a breakdown only ends this inner solve (no NUMERIC stop)
        const LoopCond lc{st, nrhs, (maxit + 2 * chunk - 1) / chunk, nullptr, 0, 0};
        int rc = dd_loop(h, body, more, lc);
        if (rc || !polled) return rc;
        int tot = 0, flags = 0;
        for (int k = 0; k < nrhs; ++k) {
            tot += hs[k].iters;
            flags |= hs[k].flags;
        }
        if (iters_out) *iters_out += tot;
        // a breakdown only ends this inner solve; the outer FP64 loop restarts from the true residual
        (void)flags;
        return DD_OK;
    }
};

template <class LK>
LK field_links(dd_handle* h, int slot);
template <>
LinkF64 field_links<LinkF64>(dd_handle* h, int slot) {
    return LinkF64{h->fields[slot].eo64, h->g.Vh};
}
template <>
LinkF32 field_links<LinkF32>(dd_handle* h, int slot) {
    return LinkF32{h->fields[slot].eo32, h->g.Vh};
}
template <>
LinkF16 field_links<LinkF16>(dd_handle* h, int slot) {
    return LinkF16{h->fields[slot].eo16, h->g.Vh};
}
template <class LK>
long long field_stride(dd_handle* h, int step) {
    if (!step || h->fields.size() < 2) return 0;
    LK a = field_links<LK>(h, 0), b = field_links<LK>(h, 1);
    return (long long)(b.p - a.p);
}

Reduce store_reduce(dd_handle* h, double* out) {
    Reduce R_;
    R_.partials = h->d_partials;
    R_.counters = h->d_counters;
    R_.st = nullptr;
    R_.out = out;
    R_.op = FIN_STORE;
    R_.status = h->d_status;
    return R_;
}

// FP64 hop helper on eo FP64 vectors
template <int MASK>
void hop64(dd_handle* h, SiteSet S, int nrhs, int par, SpinorF64 in, SpinorF64 xin, SpinorF64 out, double a, double b,
           int hasx, LinkF64 lk, long long lk_rs, const CGState* st, Reduce red) {
    HopArgs<SpinorF64, SpinorF64, SpinorF64, LinkF64> A;
    A.g = h->g;
    A.p = par;
    A.in = in;
    A.xin = xin;
    A.out = out;
    A.lk = lk;
    A.lk_rhs_stride = lk_rs;
    A.a = a;
    A.b = b;
    A.has_x = hasx;
    A.g5in = 0;
    A.g5out = 0;
    A.colour_mask = 3;
    A.st = st;
    A.red = red;
    A.S = S;
    launch_hop<double, SpinorF64, SpinorF64, SpinorF64, LinkF64, MASK>(A, nrhs, h);
}

__global__ void not_converged_kernel(int nrhs, const CGState* outer, int* status) {
    for (int k = 0; k < nrhs; ++k)
        if (outer[k].active) {
            raise_status(status, DD_ERR_NOT_CONVERGED);
            return;
        }
}

__global__ void add_scalars_kernel(int n, double* a, const double* b) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) a[r] += b[r];
}

template <int MASK, class Inner>
int defect_correction_df(dd_handle* h, int nrhs, int field0, int step, Inner& cg, double tol, int maxit,
                         int* iters, double* relres);

// One defect-correction solve around an inner solver (NormalCG or BiCGStab;
// its x is the correction, its r starts as the FP64 outer residual).
template <int MASK, class Inner>
int defect_correction(dd_handle* h, int nrhs, int field0, int step, Inner& cg, bool fp64_inner, double tol,
                      int maxit, int* iters, double* relres) {
    if constexpr (std::is_same<decltype(cg.x), SpinorF32>::value) {
        if (!fp64_inner && h->prm.outer_prec == DD_PREC_DF64)
            return defect_correction_df<MASK>(h, nrhs, field0, step, cg, tol, maxit, iters, relres);
    }
    typedef decltype(cg.x) SM;
    SolverVecs& v = h->vecs[0];
    const long long Vh = h->g.Vh;
    const double kappa = h->prm.kappa;
    const SiteSet S = cg.S;
    dim3 grid(grid_for(S.n, 128), nrhs);
    SpinorF64 be{v.be, Vh}, bo{v.bo, Vh}, xe{v.xe, Vh}, xo{v.xo, Vh}, re{v.re, Vh}, t64{v.t64, Vh},
        t64b{v.t64b, Vh};
    LinkF64 lk64 = field_links<LinkF64>(h, field0);
    const long long rs64 = field_stride<LinkF64>(h, step);
    CGState* outer = h->d_cg + h->prm.max_rhs;
    double* bb = h->d_scalars;
    double* tmp = h->d_scalars + nrhs;
    double* rr = h->d_scalars + 2 * nrhs;
    double* ones = h->d_scalars + 3 * nrhs;
    Reduce none;
    none.op = FIN_NONE;
    // |b|^2 over both parities, then b~ = b_e + kappa H_eo b_o (in place)
    DD_KLAUNCH(h, norm2_kernel<SpinorF64><<<grid, 128, 0, h->stream>>>(S, be, store_reduce(h, bb)));
    DD_KLAUNCH(h, norm2_kernel<SpinorF64><<<grid, 128, 0, h->stream>>>(S, bo, store_reduce(h, tmp)));
    DD_KLAUNCH(h, add_scalars_kernel<<<1, 64, 0, h->stream>>>(nrhs, bb, tmp));
    hop64<MASK>(h, S, nrhs, 0, bo, be, be, 1.0, kappa, 1, lk64, rs64, nullptr, none);
    DD_KLAUNCH(h, outer_arm_kernel<<<1, 64, 0, h->stream>>>(nrhs, outer, bb, tol));
    DD_KLAUNCH(h, zero64_kernel<<<grid, 128, 0, h->stream>>>(S, xe));
    DD_KLAUNCH(h, copy_kernel<SpinorF64, SpinorF64><<<grid, 128, 0, h->stream>>>(S, be, re, nullptr));
    DD_KLAUNCH(h, norm2_kernel<SpinorF64><<<grid, 128, 0, h->stream>>>(S, re, store_reduce(h, rr)));
    DD_KLAUNCH(h, outer_update_kernel<<<1, 64, 0, h->stream>>>(nrhs, outer, rr, h->d_status));
    if (cudaGetLastError() != cudaSuccess) return DD_ERR_CUDA;
    const double tol_inner = fp64_inner ? 0.0 : h->prm.tol_inner;
    int total = 0, cycles = 0;
    bool polled = false;
    std::vector<CGState> hs(nrhs);
    auto body = [&]() -> int {
        // inner right-hand side: the current FP64 residual
        // (the mixed inner system is normalised to |r| = 1)
        if (!fp64_inner) {
            DD_KLAUNCH(h, normalised_copy_kernel<SM><<<grid, 128, 0, h->stream>>>(S, re, cg.r, rr, outer));
            DD_KLAUNCH(h, fill_kernel<<<1, 64, 0, h->stream>>>(nrhs, ones, 1.0));
        }
        // inner stopping rule: FP64 inner aims at the outer target directly
        // (with margin), the mixed inner at a relative reduction tol_inner
        int it = 0;
        int rc = cg.run(fp64_inner ? rr : ones, tol_inner, fp64_inner ? 0.25 : -1.0, maxit - total, 16, &it);
        total += it;
        if (rc) return rc;
        DD_KLAUNCH(h, add_correction_kernel<SM><<<grid, 128, 0, h->stream>>>(S, xe, cg.x, fp64_inner ? nullptr : rr,
                                                                          outer));
        // true residual r = b~ - Dtilde x (FP64)
        hop64<MASK>(h, S, nrhs, 1, xe, xe, t64, 0.0, 1.0, 0, lk64, rs64, outer, none);
        hop64<MASK>(h, S, nrhs, 0, t64, xe, t64b, 1.0, -kappa * kappa, 1, lk64, rs64, outer, none);
        DD_KLAUNCH(h, residual_kernel<<<grid, 128, 0, h->stream>>>(S, be, t64b, re, outer, store_reduce(h, rr)));
        DD_KLAUNCH(h, outer_update_kernel<<<1, 64, 0, h->stream>>>(nrhs, outer, rr, h->d_status));
        return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
    };
    auto more = [&](bool& m) -> int {
        ++cycles;
        if (cudaMemcpyAsync(hs.data(), outer, sizeof(CGState) * nrhs, cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess)
            return DD_ERR_CUDA;
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DD_ERR_CUDA;
        polled = true;
        bool any = false;
        for (int k = 0; k < nrhs; ++k) any = any || hs[k].active;
        m = any && total < maxit && cycles < 200;
        return DD_OK;
    };
    // captured: the inner maxit stays the full budget; the outer loop stops
    // once the inner iterations of all cycles reach maxit
    const LoopCond lc{outer, nrhs, 200, cg.st, (long long)maxit, 0};
    int rc = dd_loop(h, body, more, lc);
    if (rc) return rc;
    // x_o = b_o + kappa H_oe x_e
    hop64<MASK>(h, S, nrhs, 1, xe, bo, xo, 1.0, kappa, 1, lk64, rs64, nullptr, none);
    if (cudaGetLastError() != cudaSuccess) return DD_ERR_CUDA;
    if (!polled) {
        // captured: a solve that missed its target is reported in the status word
        DD_KLAUNCH(h, not_converged_kernel<<<1, 1, 0, h->stream>>>(nrhs, outer, h->d_status));
        return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
    }
    std::vector<double> hb(nrhs);
    if (cudaMemcpyAsync(hb.data(), bb, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return DD_ERR_CUDA;
    if (cudaMemcpyAsync(hs.data(), outer, sizeof(CGState) * nrhs, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return DD_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DD_ERR_CUDA;
    bool conv = true, finite = true;
    for (int k = 0; k < nrhs; ++k) {
        double rel = hb[k] > 0 ? std::sqrt(hs[k].rr / hb[k]) : 0.0;
        if (relres) relres[k] = rel;
        if (hs[k].active) conv = false;
        if (!std::isfinite(hs[k].rr) || !std::isfinite(hb[k])) finite = false;
    }
    if (iters) *iters = total;
    {
        long long* st = h->solve_stats[MASK == 0 ? 0 : 1];
        st[0] += 1;
        st[1] += nrhs;
        st[2] += total;
        st[3] += cycles;
        st[4] += (long long)total * S.n;
    }
    if (!finite) return DD_ERR_NUMERIC;
    return conv ? DD_OK : DD_ERR_NOT_CONVERGED;
}


// ------------------------------------------- double-float defect correction
// The outer loop of a mixed-precision solve with the true residual formed in
// double-float arithmetic (dd_params.outer_prec = DD_PREC_DF64, dfhop.cuh).
// Per right-hand side every double-float vector holds sigma times the FP64
// value, sigma = 2^e with |sigma b| in [1, 2); residual norms are reported
// unscaled.

// e_r = -floor(log2 |b_r|) (0 for b_r = 0)
__global__ void df_scale_kernel(int nrhs, const double* bb, double* sig_exp) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    sig_exp[r] = bb[r] > 0.0 ? -(double)ilogb(sqrt(bb[r])) : 0.0;
}
// out = sigma in, split into double-float
__global__ void __launch_bounds__(128) to_df_kernel(SiteSet S, SpinorF64 in, SpinorDF out, const double* sig_exp) {
    const int rhs = blockIdx.y;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    const int e = (int)sig_exp[rhs];
    const SpinorF64 a = at_rhs(in, rhs);
    const SpinorDF o = at_rhs(out, rhs);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 v = a.p[k * a.stride + i];
        o.st(i, k, cdf{df_from_double(ldexp(v.x, e)), df_from_double(ldexp(v.y, e))});
    }
}
// out = (hi + lo) / sigma in FP64
__global__ void __launch_bounds__(128) from_df_kernel(SiteSet S, SpinorDF in, SpinorF64 out, const double* sig_exp) {
    const int rhs = blockIdx.y;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    const int e = -(int)sig_exp[rhs];
    const SpinorDF a = at_rhs(in, rhs);
    const SpinorF64 o = at_rhs(out, rhs);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const cdf c = a.ld(i, k);
        o.p[k * o.stride + i] = make_double2(ldexp(df_to_double(c.re), e), ldexp(df_to_double(c.im), e));
    }
}
// r = in rounded to FP32, |r|^2 / sigma^2 (the residual of x = 0)
__global__ void __launch_bounds__(128) df_round_kernel(SiteSet S, SpinorDF in, SpinorF32 r, const double* sig_exp,
                                                       Reduce red) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double nrm = 0.0;
    if (ti < S.n) {
        const long long i = S.at(ti);
        const SpinorDF a = at_rhs(in, rhs);
        Spinor<float> v;
        float n2 = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const cdf c = a.ld(i, k);
            v.c[k] = mk<float>(__fadd_rn(c.re.hi, c.re.lo), __fadd_rn(c.im.hi, c.im.lo));
            n2 = fmaf(v.c[k].x, v.c[k].x, fmaf(v.c[k].y, v.c[k].y, n2));
        }
        at_rhs(r, rhs).store(i, v);
        nrm = ldexp((double)n2, -2 * (int)sig_exp[rhs]);
    }
    grid_reduce(red, rhs, nrm, sh);
}
// r /= sigma |r| (the inner solver's unit-norm right-hand side)
__global__ void __launch_bounds__(128) df_normalise_kernel(SiteSet S, SpinorF32 r, const double* rr,
                                                           const double* sig_exp, const CGState* outer) {
    const int rhs = blockIdx.y;
    if (outer && !outer[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    const float inv = rr[rhs] > 0.0 ? (float)ldexp(1.0 / sqrt(rr[rhs]), -(int)sig_exp[rhs]) : 0.f;
    const SpinorF32 a = at_rhs(r, rhs);
    Spinor<float> v;
    a.load(i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) v.c[k] = inv * v.c[k];
    a.store(i, v);
}
// x += sigma |r| e (e: the inner solution of the unit-norm system)
template <class SE>
__global__ void __launch_bounds__(128) df_add_correction_kernel(SiteSet S, SpinorDF x, SE e, const double* rr,
                                                                const double* sig_exp, const CGState* outer) {
    const int rhs = blockIdx.y;
    if (outer && !outer[rhs].active) return;
    const long long ti = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= S.n) return;
    const long long i = S.at(ti);
    const dfl sc = df_from_double(ldexp(sqrt(rr[rhs]), (int)sig_exp[rhs]));
    const SpinorDF xr = at_rhs(x, rhs);
    Spinor<float> b;
    at_rhs(e, rhs).load(i, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        cdf c = xr.ld(i, k);
        df_mac(c.re, sc, dfl{b.c[k].x, 0.f});
        df_mac(c.im, sc, dfl{b.c[k].y, 0.f});
        xr.st(i, k, c);
    }
}

template <int MASK, int MODE>
void hopdf(dd_handle* h, int nrhs, DFHopArgs A) {
    const int tpb = std::min(h->tune.hop64_tpb, 128);
    dim3 grid(grid_for(A.S.n, tpb), nrhs);
    bool timed = false;
    if (MASK == 0 && h->timer_on && !h->capturing && !dd_stream_capturing(h))
        timed = (h->timer_seen[3]++ % h->timer_every) == 0;
    A.sites = nullptr;
    if (timed) {
        cudaEvent_t e = dd_timer_event(h, 3);
        if (e) cudaEventRecord(e, h->stream);
        A.sites = h->d_sites + 3;
    }
    DD_KLAUNCH(h, hop_df_kernel<MASK, MODE><<<grid, tpb, 0, h->stream>>>(A));
    if (timed) {
        cudaEvent_t e = dd_timer_event(h, 3);
        if (e) cudaEventRecord(e, h->stream);
    }
}

template <int MASK, class Inner>
int defect_correction_df(dd_handle* h, int nrhs, int field0, int step, Inner& cg, double tol, int maxit,
                         int* iters, double* relres) {
    typedef decltype(cg.x) SM;
    SolverVecs& v = h->vecs[0];
    const long long Vh = h->g.Vh;
    const double kappa = h->prm.kappa;
    const SiteSet S = cg.S;
    dim3 grid(grid_for(S.n, 128), nrhs);
    SpinorF64 be{v.be, Vh}, bo{v.bo, Vh}, xe{v.xe, Vh}, xo{v.xo, Vh};
    // double-float vectors in the FP64 buffers of the plain FP64 solver (same bytes per site)
    SpinorDF xd{reinterpret_cast<float4*>(v.x64), Vh}, td{reinterpret_cast<float4*>(v.p64), Vh},
        btd{reinterpret_cast<float4*>(v.q64), Vh}, bod{reinterpret_cast<float4*>(v.z64), Vh};
    const SpinorF32 r32 = cg.r;
    FieldSlot& f0 = h->fields[field0];
    if (!f0.eodf) return DD_ERR_INVALID_ARG;
    LinkDF lk{f0.eodf, Vh};
    const long long rs = (step && h->fields.size() > 1) ? (long long)(h->fields[1].eodf - h->fields[0].eodf) : 0;
    CGState* outer = h->d_cg + h->prm.max_rhs;
    double* bb = h->d_scalars;
    double* tmp = h->d_scalars + nrhs;
    double* rr = h->d_scalars + 2 * nrhs;
    double* ones = h->d_scalars + 3 * nrhs;
    double* sig = h->d_scalars + 4 * nrhs;
    DFHopArgs A;
    A.g = h->g;
    A.lk = lk;
    A.lk_rhs_stride = rs;
    A.st = nullptr;
    A.sig_exp = sig;
    A.red.op = FIN_NONE;
    A.S = S;
    // |b|^2 over both parities, the scales, b~ = b_e + kappa H_eo b_o
    DD_KLAUNCH(h, norm2_kernel<SpinorF64><<<grid, 128, 0, h->stream>>>(S, be, store_reduce(h, bb)));
    DD_KLAUNCH(h, norm2_kernel<SpinorF64><<<grid, 128, 0, h->stream>>>(S, bo, store_reduce(h, tmp)));
    DD_KLAUNCH(h, add_scalars_kernel<<<1, 64, 0, h->stream>>>(nrhs, bb, tmp));
    DD_KLAUNCH(h, df_scale_kernel<<<1, 64, 0, h->stream>>>(nrhs, bb, sig));
    DD_KLAUNCH(h, to_df_kernel<<<grid, 128, 0, h->stream>>>(S, be, btd, sig));
    DD_KLAUNCH(h, to_df_kernel<<<grid, 128, 0, h->stream>>>(S, bo, bod, sig));
    A.p = 0;
    A.in = bod;
    A.xin = btd;
    A.out = btd;
    A.c = df_from_double(kappa);
    hopdf<MASK, 1>(h, nrhs, A);
    DD_KLAUNCH(h, outer_arm_kernel<<<1, 64, 0, h->stream>>>(nrhs, outer, bb, tol));
    DD_KLAUNCH(h, zero64_kernel<<<grid, 128, 0, h->stream>>>(S, SpinorF64{v.x64, Vh}));
    DD_KLAUNCH(h, df_round_kernel<<<grid, 128, 0, h->stream>>>(S, btd, r32, sig, store_reduce(h, rr)));
    DD_KLAUNCH(h, outer_update_kernel<<<1, 64, 0, h->stream>>>(nrhs, outer, rr, h->d_status));
    if (cudaGetLastError() != cudaSuccess) return DD_ERR_CUDA;
    int total = 0, cycles = 0;
    bool polled = false;
    std::vector<CGState> hs(nrhs);
    auto body = [&]() -> int {
        DD_KLAUNCH(h, df_normalise_kernel<<<grid, 128, 0, h->stream>>>(S, r32, rr, sig, outer));
        DD_KLAUNCH(h, fill_kernel<<<1, 64, 0, h->stream>>>(nrhs, ones, 1.0));
        int it = 0;
        int rc = cg.run(ones, h->prm.tol_inner, -1.0, maxit - total, 16, &it);
        total += it;
        if (rc) return rc;
        DD_KLAUNCH(h, df_add_correction_kernel<SM><<<grid, 128, 0, h->stream>>>(S, xd, cg.x, rr, sig, outer));
        // true residual r = b~ - x + kappa^2 H_eo H_oe x (double-float), rounded into the inner r
        DFHopArgs B = A;
        B.st = outer;
        B.p = 1;
        B.in = xd;
        B.out = td;
        hopdf<MASK, 0>(h, nrhs, B);
        B.p = 0;
        B.in = td;
        B.xin = xd;
        B.bin = btd;
        B.rout = r32;
        B.c = df_from_double(kappa * kappa);
        B.red = store_reduce(h, rr);
        hopdf<MASK, 2>(h, nrhs, B);
        DD_KLAUNCH(h, outer_update_kernel<<<1, 64, 0, h->stream>>>(nrhs, outer, rr, h->d_status));
        return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
    };
    auto more = [&](bool& m) -> int {
        ++cycles;
        if (cudaMemcpyAsync(hs.data(), outer, sizeof(CGState) * nrhs, cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess)
            return DD_ERR_CUDA;
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DD_ERR_CUDA;
        polled = true;
        bool any = false;
        for (int k = 0; k < nrhs; ++k) any = any || hs[k].active;
        m = any && total < maxit && cycles < 200;
        return DD_OK;
    };
    const LoopCond lc{outer, nrhs, 200, cg.st, (long long)maxit, 0};
    int rc = dd_loop(h, body, more, lc);
    if (rc) return rc;
    // x_o = b_o + kappa H_oe x_e, both parities back to FP64
    A.p = 1;
    A.in = xd;
    A.xin = bod;
    A.out = td;
    A.c = df_from_double(kappa);
    hopdf<MASK, 1>(h, nrhs, A);
    DD_KLAUNCH(h, from_df_kernel<<<grid, 128, 0, h->stream>>>(S, xd, xe, sig));
    DD_KLAUNCH(h, from_df_kernel<<<grid, 128, 0, h->stream>>>(S, td, xo, sig));
    if (cudaGetLastError() != cudaSuccess) return DD_ERR_CUDA;
    if (!polled) {
        DD_KLAUNCH(h, not_converged_kernel<<<1, 1, 0, h->stream>>>(nrhs, outer, h->d_status));
        return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
    }
    std::vector<double> hb(nrhs);
    if (cudaMemcpyAsync(hb.data(), bb, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return DD_ERR_CUDA;
    if (cudaMemcpyAsync(hs.data(), outer, sizeof(CGState) * nrhs, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return DD_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DD_ERR_CUDA;
    bool conv = true, finite = true;
    for (int k = 0; k < nrhs; ++k) {
        double rel = hb[k] > 0 ? std::sqrt(hs[k].rr / hb[k]) : 0.0;
        if (relres) relres[k] = rel;
        if (hs[k].active) conv = false;
        if (!std::isfinite(hs[k].rr) || !std::isfinite(hb[k])) finite = false;
    }
    if (iters) *iters = total;
    {
        long long* st = h->solve_stats[MASK == 0 ? 0 : 1];
        st[0] += 1;
        st[1] += nrhs;
        st[2] += total;
        st[3] += cycles;
        st[4] += (long long)total * S.n;
    }
    if (!finite) return DD_ERR_NUMERIC;
    return conv ? DD_OK : DD_ERR_NOT_CONVERGED;
}

#include "sapgcr.cuh"

}  // namespace

template <class B>
static void fill_bicg(dd_handle* h, B& bi, long long Vh, CGState* inner, CGState* outer, int nrhs) {
    bi.nrhs = nrhs;
    SolverVecs& v = h->vecs[0];
    bi.h = h;
    bi.x = SpinorF32{v.x32, Vh};
    bi.r = SpinorF32{v.r32, Vh};
    bi.v = SpinorF32{v.q32, Vh};
    bi.s = SpinorF32{v.z32, Vh};
    bi.t = SpinorF32{v.w32, Vh};
    bi.st = inner;
    bi.outer = outer;
}

template <int MASK>
static int solve_packed_mask(dd_handle* h, SiteSet S, int nrhs, int field0, int step, int prec, double tol,
                             int maxit, int* iters, double* relres) {
    SolverVecs& v = h->vecs[0];
    const long long Vh = h->g.Vh;
    CGState* inner = h->d_cg;
    CGState* outer = h->d_cg + h->prm.max_rhs;
    if (prec == DD_PREC_F64) {
        NormalCG<double, SpinorF64, SpinorF64, LinkF64, MASK> cg;
        cg.h = h;
        cg.nrhs = nrhs;
        // the inner x must not alias the residual temporaries: x64
        cg.x = SpinorF64{v.x64, Vh};
        cg.r = SpinorF64{v.re, Vh};
        cg.p = SpinorF64{v.p64, Vh};
        cg.q = SpinorF64{v.q64, Vh};
        cg.z = SpinorF64{v.z64, Vh};
        cg.ph = cg.p;
        cg.rh = cg.r;
        cg.th = SpinorF64{v.t64, Vh};
        cg.copies = 0;
        cg.lk = field_links<LinkF64>(h, field0);
        cg.lk_rs = field_stride<LinkF64>(h, step);
        cg.st = inner;
        cg.outer = outer;
        cg.S = S;
        return defect_correction<MASK>(h, nrhs, field0, step, cg, true, tol, maxit, iters, relres);
    } else if (MASK == 0 && h->prm.krylov == DD_KRYLOV_SAP_GCR) {
        // SAP-preconditioned flexible GCR on D (global solves only)
        auto fill = [&](auto& sg) {
            sg.h = h;
            sg.nrhs = nrhs;
            sg.x = SpinorF32{v.x32, Vh};
            sg.r = SpinorF32{v.r32, Vh};
            sg.st = inner;
            sg.outer = outer;
            sg.S = S;
            sg.bst = h->d_cg + 2 * h->prm.max_rhs;
            sg.ncy = h->prm.sap_ncy;
            sg.nmr = h->prm.sap_nmr;
            sg.nkv = h->sap.nkv;
        };
        if (prec == DD_PREC_F32) {
            SapGcr<SpinorF32, LinkF32> sg;
            fill(sg);
            sg.lk = field_links<LinkF32>(h, field0);
            sg.lk_rs = field_stride<LinkF32>(h, step);
            return defect_correction<MASK>(h, nrhs, field0, step, sg, false, tol, maxit, iters, relres);
        }
        SapGcr<SpinorF16, LinkF16> sg;
        fill(sg);
        sg.lk = field_links<LinkF16>(h, field0);
        sg.lk_rs = field_stride<LinkF16>(h, step);
        return defect_correction<MASK>(h, nrhs, field0, step, sg, false, tol, maxit, iters, relres);
    } else if (h->prm.krylov != DD_KRYLOV_CGNR) {
        if (prec == DD_PREC_F32) {
            BiCGStab<float, SpinorF32, SpinorF32, LinkF32, MASK> bi;
            fill_bicg(h, bi, Vh, inner, outer, nrhs);
            bi.p = SpinorF32{v.p32, Vh};
            bi.rhat = SpinorF32{v.h32, Vh};
            bi.shop = bi.s;
            bi.th = SpinorF32{v.t32, Vh};
            bi.copies = 0;
            bi.lk = field_links<LinkF32>(h, field0);
            bi.lk_rs = field_stride<LinkF32>(h, step);
            bi.S = S;
            return defect_correction<MASK>(h, nrhs, field0, step, bi, false, tol, maxit, iters, relres);
        }
        BiCGStab<float, SpinorF32, SpinorF16, LinkF16, MASK> bi;
        fill_bicg(h, bi, Vh, inner, outer, nrhs);
        bi.p = SpinorF16{v.p16, v.p16n, Vh};
        bi.rhat = SpinorF16{v.q16, v.q16n, Vh};
        bi.shop = SpinorF16{v.r16, v.r16n, Vh};
        bi.th = SpinorF16{v.t16, v.t16n, Vh};
        bi.copies = 1;
        bi.lk = field_links<LinkF16>(h, field0);
        bi.lk_rs = field_stride<LinkF16>(h, step);
        bi.S = S;
        return defect_correction<MASK>(h, nrhs, field0, step, bi, false, tol, maxit, iters, relres);
    } else if (prec == DD_PREC_F32) {
        NormalCG<float, SpinorF32, SpinorF32, LinkF32, MASK> cg;
        cg.h = h;
        cg.nrhs = nrhs;
        cg.x = SpinorF32{v.x32, Vh};
        cg.r = SpinorF32{v.r32, Vh};
        cg.p = SpinorF32{v.p32, Vh};
        cg.q = SpinorF32{v.q32, Vh};
        cg.z = SpinorF32{v.z32, Vh};
        cg.ph = cg.p;
        cg.rh = cg.r;
        cg.th = SpinorF32{v.t32, Vh};
        cg.copies = 0;
        cg.lk = field_links<LinkF32>(h, field0);
        cg.lk_rs = field_stride<LinkF32>(h, step);
        cg.st = inner;
        cg.outer = outer;
        cg.S = S;
        return defect_correction<MASK>(h, nrhs, field0, step, cg, false, tol, maxit, iters, relres);
    } else {
        NormalCG<float, SpinorF32, SpinorF16, LinkF16, MASK> cg;
        cg.h = h;
        cg.nrhs = nrhs;
        cg.x = SpinorF32{v.x32, Vh};
        cg.r = SpinorF32{v.r32, Vh};
        cg.p = SpinorF32{v.p32, Vh};
        cg.q = SpinorF32{v.q32, Vh};
        cg.z = SpinorF32{v.z32, Vh};
        cg.ph = SpinorF16{v.p16, v.p16n, Vh};
        cg.rh = SpinorF16{v.r16, v.r16n, Vh};
        cg.th = SpinorF16{v.t16, v.t16n, Vh};
        cg.copies = 1;
        cg.lk = field_links<LinkF16>(h, field0);
        cg.lk_rs = field_stride<LinkF16>(h, step);
        cg.st = inner;
        cg.outer = outer;
        cg.S = S;
        return defect_correction<MASK>(h, nrhs, field0, step, cg, false, tol, maxit, iters, relres);
    }
}

int solve_packed(dd_handle* h, int nrhs, int field0, int step, int prec, double tol, int maxit, int* iters,
                 double* relres, int mask, int colour) {
    SiteSet S{nullptr, (long long)h->g.Vh};
    // Dirichlet solves whose right-hand sides live on the blocks of one
    // colour: the other colour's sites stay zero and are not visited
    if (mask == 1 && colour >= 0 && colour <= 1 && h->d_colour_sites[colour])
        S = SiteSet{h->d_colour_sites[colour], (long long)h->g.Vh / 2, colour};
    if (mask == 1) return solve_packed_mask<1>(h, S, nrhs, field0, step, prec, tol, maxit, iters, relres);
    return solve_packed_mask<0>(h, S, nrhs, field0, step, prec, tol, maxit, iters, relres);
}

extern "C" int dd_solve(dd_t h, void* x, const void* b, const void* U, int nrhs, int prec, int* iters,
                        double* relres) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_solve, "dd_solve");
    if (rc) return rc;
    if (!x || !b || !U || nrhs < 1 || nrhs > h->prm.max_rhs) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_solve: bad arguments");
    if (prec < DD_PREC_F64 || prec > DD_PREC_F16) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_solve: unknown precision");
    const long long V = h->g.V;
    rc = format_field(h, (const double*)U, h->fields[0], true, prec == DD_PREC_F32, prec == DD_PREC_F16, false, false);
    if (rc) return rc;
    SolverVecs& v = h->vecs[0];
    launch_pack_spinor_eo(h, (const double*)b, v.be, 0, nrhs, 24 * V);
    launch_pack_spinor_eo(h, (const double*)b, v.bo, 1, nrhs, 24 * V);
    DD_LAUNCH_CHECK(h, "dd_solve pack");
    int it = 0;
    rc = solve_packed(h, nrhs, 0, 0, prec, h->prm.tol_global, h->prm.maxit, &it, relres);
    if (iters) *iters = it;
    if (rc && rc != DD_ERR_NOT_CONVERGED) return dd_fail(h, rc, "dd_solve: solver failed");
    launch_unpack_spinor_eo(h, v.xe, (double*)x, 0, nrhs, 24 * V);
    launch_unpack_spinor_eo(h, v.xo, (double*)x, 1, nrhs, 24 * V);
    DD_LAUNCH_CHECK(h, "dd_solve unpack");
    if (rc == DD_ERR_NOT_CONVERGED) return dd_fail(h, rc, "dd_solve: iteration cap reached");
    return DD_OK;
}

// ncy Schwarz cycles applied to nrhs canonical spinors (see include/dd.h)
extern "C" int dd_sap_apply(dd_t h, void* out, const void* in, const void* U, int nrhs, int prec) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_solve, "dd_sap_apply");
    if (rc) return rc;
    if (!out || !in || !U || nrhs < 1 || nrhs > h->prm.max_rhs || (prec != DD_PREC_F32 && prec != DD_PREC_F16))
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_sap_apply: bad arguments");
    if (h->prm.krylov != DD_KRYLOV_SAP_GCR || !h->sap.halves)
        return dd_fail(h, DD_ERR_UNSUPPORTED, "dd_sap_apply: handle not created with krylov DD_KRYLOV_SAP_GCR");
    if (!h->d_colour_sites[0] || !h->d_colour_sites[1])
        return dd_fail(h, DD_ERR_UNSUPPORTED, "dd_sap_apply: needs an even block extent along axis 0");
    const long long V = h->g.V, Vh = h->g.Vh;
    rc = format_field(h, (const double*)U, h->fields[0], true, prec == DD_PREC_F32, prec == DD_PREC_F16, false, false);
    if (rc) return rc;
    SolverVecs& v = h->vecs[0];
    launch_pack_spinor_eo(h, (const double*)in, v.be, 0, nrhs, 24 * V);
    launch_pack_spinor_eo(h, (const double*)in, v.bo, 1, nrhs, 24 * V);
    const SiteSet S{nullptr, Vh};
    dim3 grid(grid_for(Vh, 128), nrhs);
    CGState* st = h->d_cg;
    double* ones = h->d_scalars + 3 * h->prm.max_rhs;
    DD_KLAUNCH(h, fill_kernel<<<1, 64, 0, h->stream>>>(nrhs, ones, 1.0));
    DD_KLAUNCH(h, cg_arm_kernel<<<1, 64, 0, h->stream>>>(nrhs, st, nullptr, ones, 0.0, 0.0, 1));
    auto go = [&](auto& sg) -> int {
        sg.h = h;
        sg.nrhs = nrhs;
        sg.x = SpinorF32{v.x32, Vh};
        sg.r = SpinorF32{v.r32, Vh};
        sg.st = st;
        sg.outer = nullptr;
        sg.S = S;
        sg.bst = h->d_cg + 2 * h->prm.max_rhs;
        sg.ncy = h->prm.sap_ncy;
        sg.nmr = h->prm.sap_nmr;
        sg.nkv = h->sap.nkv;
        const FullF32 rho = sg.R(), z = sg.Zk(0);
        DD_KLAUNCH(h, copy_kernel<SpinorF64, SpinorF32><<<grid, 128, 0, h->stream>>>(S, SpinorF64{v.be, Vh}, rho.e, nullptr));
        DD_KLAUNCH(h, copy_kernel<SpinorF64, SpinorF32><<<grid, 128, 0, h->stream>>>(S, SpinorF64{v.bo, Vh}, rho.o, nullptr));
        int r2 = sg.precondition(rho, z);
        if (r2) return r2;
        DD_KLAUNCH(h, copy_kernel<SpinorF32, SpinorF64><<<grid, 128, 0, h->stream>>>(S, z.e, SpinorF64{v.xe, Vh}, nullptr));
        DD_KLAUNCH(h, copy_kernel<SpinorF32, SpinorF64><<<grid, 128, 0, h->stream>>>(S, z.o, SpinorF64{v.xo, Vh}, nullptr));
        return DD_OK;
    };
    if (prec == DD_PREC_F32) {
        SapGcr<SpinorF32, LinkF32> sg;
        sg.lk = field_links<LinkF32>(h, 0);
        sg.lk_rs = 0;
        rc = go(sg);
    } else {
        SapGcr<SpinorF16, LinkF16> sg;
        sg.lk = field_links<LinkF16>(h, 0);
        sg.lk_rs = 0;
        rc = go(sg);
    }
    if (rc) return dd_fail(h, rc, "dd_sap_apply failed");
    launch_unpack_spinor_eo(h, v.xe, (double*)out, 0, nrhs, 24 * V);
    launch_unpack_spinor_eo(h, v.xo, (double*)out, 1, nrhs, 24 * V);
    DD_LAUNCH_CHECK(h, "dd_sap_apply");
    return DD_OK;
}
