// Double-float ("df") arithmetic and the even-odd hopping kernel of the
// defect-correction residual in that arithmetic.
//
// A df number is the unevaluated sum hi + lo of two FP32 numbers (Dekker,
// "A floating-point technique for extending the available precision",
// Numer. Math. 18, 1971).  Sums use Knuth's TwoSum, products the exact FMA
// form a*b = p + fma(a, b, -p); the lo parts of sums are accumulated in
// FP32 and the pair is renormalised once per stored value.  Every rounding
// error of a stencil output is then bounded by about 2^-47 times the sum of
// the magnitudes of its terms (48 significant bits against FP64's 53), far
// below the 1e-10 and 1e-12 relative residuals that the outer loop checks,
// while every operation runs on the FP32 pipe (GB300's FP64 rate is about
// 1/64 of its FP32 rate).
//
// The residual r = b~ - Dtilde x of Sec. 5's even-odd system is formed from
// three hops: t = H_oe x, r = b~ - x + kappa^2 H_eo t (the source
// b~ = b_e + kappa H_eo b_o and the odd solution x_o = b_o + kappa H_oe x_e
// use the same kernel).  Vectors are scaled per right-hand side by a power
// of two sigma that brings |sigma b| into [1, 2), so FP32's exponent range
// holds any right-hand side.
#pragma once

#include "dslash.cuh"

struct dfl {
    float hi, lo;
};

// s + e = a + b exactly (Knuth's TwoSum); __fadd_rn keeps the compiler from
// contracting or reassociating
DD_DEV dfl df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    return dfl{s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv))};
}
// renormalised pair (TwoSum, valid for any magnitudes of hi and lo)
DD_DEV dfl df_norm(dfl a) { return df_two_sum(a.hi, a.lo); }
// a + b, lo parts summed unnormalised
DD_DEV dfl df_add(dfl a, dfl b) {
    dfl s = df_two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return s;
}
DD_DEV dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }
DD_DEV dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
// a * b (first term of a sum)
DD_DEV dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.hi, -p);  // exact error of p
    return dfl{p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e))};
}
// acc += a * b
DD_DEV void df_mac(dfl& acc, dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.hi, -p);
    dfl s = df_two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e))));
}
// split of an FP64 value (host constants and the conversion kernels)
DD_HD dfl df_from_double(double d) {
    const float h = (float)d;
    return dfl{h, (float)(d - (double)h)};
}
DD_DEV double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

struct cdf {  // complex df
    dfl re, im;
};
DD_DEV cdf cdf_add(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }
DD_DEV cdf cdf_sub(cdf a, cdf b) { return cdf{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
DD_DEV cdf cdf_neg(cdf a) { return cdf{df_neg(a.re), df_neg(a.im)}; }
DD_DEV cdf cdf_i(cdf a) { return cdf{df_neg(a.im), a.re}; }  // i a
DD_DEV cdf cdf_zero() { return cdf{dfl{0.f, 0.f}, dfl{0.f, 0.f}}; }

// df spinor: 12 chunks of float4 (hi.re, hi.im, lo.re, lo.im), chunk k of
// site i at p[k * stride + i]; per-rhs blocks of 12 * stride chunks (the
// byte layout of an FP64 spinor).
struct SpinorDF {
    float4* p;
    long long stride;
    DD_DEV cdf ld(long long i, int k) const {
        const float4 v = p[k * stride + i];
        return cdf{dfl{v.x, v.z}, dfl{v.y, v.w}};
    }
    DD_DEV void st(long long i, int k, cdf c) const {
        const dfl a = df_norm(c.re), b = df_norm(c.im);
        p[k * stride + i] = make_float4(a.hi, b.hi, a.lo, b.lo);
    }
};
DD_DEV SpinorDF at_rhs(SpinorDF s, int r) {
    s.p += (long long)r * 12 * s.stride;
    return s;
}

// df link, all 9 entries: chunk k (row k / 3, column k % 3) of direction a
// at p[(a * 9 + k) * stride + i]; both parities [parity][dir][chunk][Vh]
struct LinkDF {
    const float4* p;
    long long stride;
    static constexpr int chunks = 9;
    DD_DEV cdf ld(long long i, int a, int k) const {
        const float4 v = p[((long long)a * 9 + k) * stride + i];
        return cdf{dfl{v.x, v.z}, dfl{v.y, v.w}};
    }
};

// acc += u * h (complex)
DD_DEV void cdf_mac(cdf& acc, cdf u, cdf h) {
    df_mac(acc.re, u.re, h.re);
    df_mac(acc.re, df_neg(u.im), h.im);
    df_mac(acc.im, u.re, h.im);
    df_mac(acc.im, u.im, h.re);
}
// acc += conj(u) * h
DD_DEV void cdf_macc(cdf& acc, cdf u, cdf h) {
    df_mac(acc.re, u.re, h.re);
    df_mac(acc.re, u.im, h.im);
    df_mac(acc.im, u.re, h.im);
    df_mac(acc.im, df_neg(u.im), h.re);
}

struct DFHopArgs {
    Geo g;
    int p;             // output parity
    SpinorDF in;       // hop input (parity 1 - p)
    SpinorDF xin;      // MODE 1: out = xin + c H in; MODE 2: r = bin - xin + c H in
    SpinorDF bin;      // MODE 2
    SpinorDF out;      // MODE 0 / 1 output
    SpinorF32 rout;    // MODE 2 output (rounded to FP32)
    LinkDF lk;
    long long lk_rhs_stride;
    dfl c;             // coefficient of H (MODE 1 / 2)
    const CGState* st;      // per-rhs activity (may be null)
    const double* sig_exp;  // MODE 2: per-rhs exponent e of the scale sigma = 2^e
    Reduce red;             // MODE 2: |r|^2 / sigma^2
    SiteSet S;
    unsigned long long* sites;  // timed launches: output sites processed (may be null)
};

// (i sigma_a) applied to a spin pair (v0, v1) -> (o0, o1), a = 0, 1, 2 (runtime,
// the same in every thread of a warp): the spin structure of Sec. 5's
// projectors in the chiral basis, as in the FP64/FP32 stencil
DD_DEV void df_isigma_rt(int a, const cdf* v0, const cdf* v1, cdf* o0, cdf* o1) {
    if (a == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o0[c] = cdf_i(v1[c]);
            o1[c] = cdf_i(v0[c]);
        }
    } else if (a == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o0[c] = v1[c];
            o1[c] = cdf_neg(v0[c]);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o0[c] = cdf_i(v0[c]);
            o1[c] = cdf_neg(cdf_i(v1[c]));
        }
    }
}
// exact multiplication by +-1
DD_DEV cdf cdf_sign(cdf a, float sg) {
    return cdf{dfl{a.re.hi * sg, a.re.lo * sg}, dfl{a.im.hi * sg, a.im.lo * sg}};
}

// One hop: acc += (1 -+ gamma_a) U psi(y) for the forward hop (sg = +1,
// U = U_a(x)) or (1 + gamma_a) U_a(y)^dag psi(y) for the backward hop
// (sg = -1, y = x - a); ph = -1 flips the sign of a time-wrapping hop.  The
// direction is a runtime value (uniform across the warp): one copy of the
// body keeps the kernel inside the instruction cache.
DD_DEV void df_hop(int a, float sg, float ph, int yh, const float4* lk_site, const SpinorDF& in, cdf* acc) {
    // projected half spinor: upper + sg * (lower pair mapped back)
    cdf hf[6];
    {
        cdf up[6], lo[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            up[k] = in.ld(yh, k);
            lo[k] = in.ld(yh, 6 + k);
        }
        if (a == 3) {
#pragma unroll
            for (int k = 0; k < 6; ++k) hf[k] = cdf_add(up[k], cdf_sign(lo[k], sg));
        } else {
            cdf t[6];
            df_isigma_rt(a, &lo[0], &lo[3], &t[0], &t[3]);
#pragma unroll
            for (int k = 0; k < 6; ++k) hf[k] = cdf_add(up[k], cdf_sign(t[k], sg));
        }
    }
    // U h (forward) or U^dag h (backward): entry (i, j) of the applied matrix
    // is chunk 3i+j, or the conjugate of chunk 3j+i
    const long long cs = in.stride;  // links share the per-parity stride Vh
    cdf uh[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        cdf u[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int k = sg > 0.f ? 3 * i + j : 3 * j + i;
            const float4 v = lk_site[k * cs];
            u[j] = cdf{dfl{v.x, v.z}, dfl{v.y * sg, v.w * sg}};
        }
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
            const cdf* v = &hf[3 * sp];
            cdf r;
            r.re = df_mul(u[0].re, v[0].re);
            r.im = df_mul(u[0].re, v[0].im);
            df_mac(r.re, df_neg(u[0].im), v[0].im);
            df_mac(r.im, u[0].im, v[0].re);
#pragma unroll
            for (int j = 1; j < 3; ++j) cdf_mac(r, u[j], v[j]);
            uh[3 * sp + i] = cdf_sign(r, ph);
        }
    }
    // rebuild the lower spin pair and accumulate
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = cdf_add(acc[k], uh[k]);
    if (a == 3) {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[6 + k] = cdf_add(acc[6 + k], cdf_sign(uh[k], sg));
    } else {
        cdf t[6];
        df_isigma_rt(a, &uh[0], &uh[3], &t[0], &t[3]);
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[6 + k] = cdf_add(acc[6 + k], cdf_sign(t[k], -sg));
    }
}

// MODE 0: out = H in; MODE 1: out = xin + c H in; MODE 2: rout = bin - xin + c H in with |rout|^2 / sigma^2
template <int MASK, int MODE>
__global__ void __launch_bounds__(128) hop_df_kernel(DFHopArgs A) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    if (A.st && !A.st[rhs].active) return;
    if (A.sites && threadIdx.x == 0)
        atomicAdd(A.sites, (unsigned long long)min((long long)blockDim.x, A.S.n - (long long)blockIdx.x * blockDim.x));
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double nrm = 0.0;
    if (t < A.S.n) {
        const Geo& g = A.g;
        const long long Vh = g.Vh;
        const int h = (int)A.S.at(t);
        const SpinorDF in = at_rhs(A.in, rhs);
        const LinkDF lk{A.lk.p + (long long)rhs * A.lk_rhs_stride, A.lk.stride};
        const LinkDF lk_p{lk.p + (long long)A.p * 4 * 9 * Vh, Vh};
        const LinkDF lk_q{lk.p + (long long)(1 - A.p) * 4 * 9 * Vh, Vh};
        int x[4];
        eo_coords(g, A.p, h, x);
        const int s = canon_index(g, x);
        cdf acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = cdf_zero();
        // the 8 hops in a runtime loop (see df_hop)
#pragma unroll 1
        for (int d = 0; d < 8; ++d) {
            const int a = d >> 1;
            const bool fwd = (d & 1) == 0;
            const int xa = a == 0 ? x[0] : a == 1 ? x[1] : a == 2 ? x[2] : x[3];
            const int La = g.L[a], ba = g.b[a];
            if (MASK == 1) {
                const int loc = xa % ba;
                if (fwd ? loc == ba - 1 : loc == 0) continue;
            }
            const int yh = (fwd ? (xa == La - 1 ? s - (La - 1) * g.st[a] : s + g.st[a])
                                : (xa == 0 ? s + (La - 1) * g.st[a] : s - g.st[a])) >> 1;
            const float ph = (a == 3 && g.bc < 0 && xa == (fwd ? La - 1 : 0)) ? -1.f : 1.f;
            const float4* lk_site = fwd ? lk_p.p + (long long)a * 9 * Vh + h : lk_q.p + (long long)a * 9 * Vh + yh;
            df_hop(a, fwd ? 1.f : -1.f, ph, yh, lk_site, in, acc);
        }
        if (MODE == 0) {
            const SpinorDF out = at_rhs(A.out, rhs);
#pragma unroll
            for (int k = 0; k < 12; ++k) out.st(h, k, acc[k]);
        } else {
            const SpinorDF xin = at_rhs(A.xin, rhs);
            cdf res[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                cdf base = MODE == 1 ? xin.ld(h, k) : cdf_sub(at_rhs(A.bin, rhs).ld(h, k), xin.ld(h, k));
                const cdf hv{df_norm(acc[k].re), df_norm(acc[k].im)};
                df_mac(base.re, A.c, hv.re);
                df_mac(base.im, A.c, hv.im);
                res[k] = base;
            }
            if (MODE == 1) {
                const SpinorDF out = at_rhs(A.out, rhs);
#pragma unroll
                for (int k = 0; k < 12; ++k) out.st(h, k, res[k]);
            } else {
                Spinor<float> r;
                float n2 = 0.f;
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    r.c[k] = mk<float>(__fadd_rn(res[k].re.hi, res[k].re.lo), __fadd_rn(res[k].im.hi, res[k].im.lo));
                    n2 = fmaf(r.c[k].x, r.c[k].x, fmaf(r.c[k].y, r.c[k].y, n2));
                }
                at_rhs(A.rout, rhs).store(h, r);
                nrm = ldexp((double)n2, -2 * (int)A.sig_exp[rhs]);
            }
        }
    }
    if (MODE == 2) grid_reduce(A.red, rhs, nrm, sh);
}
