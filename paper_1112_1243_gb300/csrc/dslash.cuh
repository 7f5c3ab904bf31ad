// Even-odd Wilson hopping kernel (Sec. 5, the unimproved Wilson-Dirac
// operator; Eq. domdec for the intra-/inter-block restrictions).
//
// One thread per output site of parity p:
//   out(x) = a * xin(x) + b * G5out( sum_hops (1 -+ gamma_a) U psi(x +- a) ),
// psi read from the opposite parity, optionally gamma5-multiplied on load.
// MASK = 0: all hops; 1: hops inside a block only (Dirichlet D_b); 2: only
// hops that cross a block face (D_bw, D_wb).  Links are stored per parity:
// the forward hop of x uses U_a(x) (parity p), the backward hop the link
// U_a(x - a) stored at the neighbour (parity 1 - p).
#pragma once

#include <algorithm>
#include <type_traits>

#include "dd_internal.h"
#include "reduce.cuh"

// per-rhs shifted copies of storage descriptors (contiguous per-rhs blocks)
DD_DEV SpinorF64 at_rhs(SpinorF64 s, int r) {
    s.p += (long long)r * 12 * s.stride;
    return s;
}
DD_DEV SpinorF32 at_rhs(SpinorF32 s, int r) {
    s.p += (long long)r * 6 * s.stride;
    return s;
}
DD_DEV SpinorF16 at_rhs(SpinorF16 s, int r) {
    s.p += (long long)r * 3 * s.stride;
    s.nrm += (long long)r * s.stride;
    return s;
}

template <class SIn, class SX, class SOut, class LK>
struct HopArgs {
    Geo g;
    int p;                    // output parity
    SIn in;                   // input field (parity 1 - p)
    SX xin;                   // a * xin term (parity p), used when has_x
    SOut out;                 // output (parity p)
    LK lk;                    // gauge field, both parities: [parity][dir][chunk][Vh]
    long long lk_rhs_stride;  // elements between the fields of consecutive rhs (0: shared)
    double a, b;
    int has_x;
    int g5in, g5out;
    int colour_mask;          // 3 = every site; else zero the output outside these block colours
    const CGState* st;        // per-rhs activity (may be null)
    Reduce red;               // |out|^2 reduction (red.op == FIN_NONE: off)
    unsigned long long* sites;  // timed launches: output sites processed (may be null)
    // three-value reductions (BiCGStab): 0 off; 1: <rhat, out>; 2: <out, xin> and |out|^2
    int red3 = 0;
    SX rhat;
    SiteSet S = {nullptr, -1};  // output sites (n < 0: all Vh sites of parity p)
};

template <class LK>
DD_DEV LK link_parity(LK lk, int par, long long Vh) {
    lk.p += (long long)par * 4 * LK::chunks * Vh;
    return lk;
}

template <class R, class SIn, class LK, int MASK>
DD_DEV void hop_site(const Geo& g, int p, int h, const int x[4], const SIn& in, const LK& lk_p, const LK& lk_q,
                     int g5in, Spinor<R>& acc) {
    zero(acc);
    const int s = canon_index(g, x);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        // local coordinate in the block (multiply-high division: b_a is not a compile-time constant)
        const int loc = x[a] - fast_div(x[a], g.b[a], g.mb[a]) * g.b[a];
        // forward: (1 - gamma_a) U_a(x) psi(x + a)
        bool okf = true, okb = true;
        if (MASK == 1) {
            okf = loc != g.b[a] - 1;
            okb = loc != 0;
        } else if (MASK == 2) {
            okf = loc == g.b[a] - 1;
            okb = loc == 0;
        }
        if (okf) {
            int yh = neighbour_index(g, s, x, a, +1) >> 1;
            Spinor<R> s;
            R w = in.load_unscaled(yh, s);
            if (g5in) gamma5(s);
            Half<R> hf, uh;
            project<R>(a, +1, s, hf);
            Link<R> u;
            lk_p.load(h, a, u);
            mul_link(u, hf, uh);
            R sc = (a == 3 && x[3] == g.L[3] - 1) ? (R)g.bc * w : w;
            accumulate<R>(a, +1, uh, sc, acc);
        }
        if (okb) {
            int yh = neighbour_index(g, s, x, a, -1) >> 1;
            Spinor<R> s;
            R w = in.load_unscaled(yh, s);
            if (g5in) gamma5(s);
            Half<R> hf, uh;
            project<R>(a, -1, s, hf);
            Link<R> u;
            lk_q.load(yh, a, u);
            mul_link_dag(u, hf, uh);
            R sc = (a == 3 && x[3] == 0) ? (R)g.bc * w : w;
            accumulate<R>(a, -1, uh, sc, acc);
        }
    }
}

// Each thread block covers SPT * blockDim.x consecutive entries of the site
// set (SPT passes of blockDim.x threads; thread block size and SPT are
// chosen by the autotuner, see dd_autotune).
template <class R, class SIn, class SX, class SOut, class LK, int MASK, int RED3, int SPT>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 7 : 0)
    hop_eo_kernel(HopArgs<SIn, SX, SOut, LK> A) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    if (A.st && !A.st[rhs].active) return;
    const long long Vh = A.g.Vh;
    const long long tile = (long long)blockDim.x * SPT;
    if (A.sites && threadIdx.x == 0)
        atomicAdd(A.sites, (unsigned long long)min(tile, A.S.n - (long long)blockIdx.x * tile));
    double v3[3] = {0.0, 0.0, 0.0};
    double nrm = 0.0;
#pragma unroll
    for (int pass = 0; pass < SPT; ++pass) {
        const long long t = (long long)blockIdx.x * tile + (long long)pass * blockDim.x + threadIdx.x;
        if (t >= A.S.n) break;
        int x[4];
        int h;
        if (A.S.colour >= 0) {
            h = colour_site(A.g, A.S.colour, (int)t, A.p, x);
        } else {
            h = (int)A.S.at(t);
            eo_coords(A.g, A.p, h, x);
        }
        const SIn in = at_rhs(A.in, rhs);
        LK lk = A.lk;
        lk.p += (long long)rhs * A.lk_rhs_stride;
        const LK lk_p = link_parity(lk, A.p, Vh);
        const LK lk_q = link_parity(lk, 1 - A.p, Vh);
        Spinor<R> acc;
        hop_site<R, SIn, LK, MASK>(A.g, A.p, h, x, in, lk_p, lk_q, A.g5in, acc);
        if (A.g5out) gamma5(acc);
        Spinor<R> res, xv;
        const R bb = (R)A.b;
        if (A.has_x) {
            at_rhs(A.xin, rhs).load(h, xv);
            const R aa = (R)A.a;
#pragma unroll
            for (int k = 0; k < 12; ++k) res.c[k] = aa * xv.c[k] + bb * acc.c[k];
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) res.c[k] = bb * acc.c[k];
        }
        if (A.colour_mask != 3 && !((A.colour_mask >> block_colour_of(A.g, x)) & 1)) zero(res);
        at_rhs(A.out, rhs).store(h, res);
        // per-site sums in the arithmetic precision, accumulated across sites
        // in FP64 by the grid reduction (FP64 adds per component would cost
        // more than the stencil on GB300's FP64 pipe)
        if (RED3 == 1) {
            Spinor<R> rv;
            at_rhs(A.rhat, rhs).load(h, rv);
            R d0 = 0, d1 = 0;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                d0 += rv.c[k].x * res.c[k].x + rv.c[k].y * res.c[k].y;
                d1 += rv.c[k].x * res.c[k].y - rv.c[k].y * res.c[k].x;
            }
            v3[0] += (double)d0;
            v3[1] += (double)d1;
        } else if (RED3 == 2) {
            R d0 = 0, d1 = 0;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                d0 += res.c[k].x * xv.c[k].x + res.c[k].y * xv.c[k].y;
                d1 += res.c[k].x * xv.c[k].y - res.c[k].y * xv.c[k].x;
            }
            v3[0] += (double)d0;
            v3[1] += (double)d1;
            v3[2] += (double)snorm2(res);
        } else {
            nrm += (double)snorm2(res);
        }
    }
    if (RED3) {
        grid_reduce3(A.red, rhs, v3, sh);
    } else if (A.red.op != FIN_NONE) {
        grid_reduce(A.red, rhs, nrm, sh);
    }
}

// timing class of a hop kernel instance (see dd_handle::timer_*), -1: not timed
template <class SIn, class SOut>
constexpr int hop_kind() {
    return std::is_same<SIn, SpinorF16>::value && std::is_same<SOut, SpinorF16>::value   ? 0
           : std::is_same<SIn, SpinorF16>::value && std::is_same<SOut, SpinorF32>::value ? 1
           : std::is_same<SIn, SpinorF64>::value                                          ? 2
                                                                                          : -1;
}

template <class R, class SIn, class SX, class SOut, class LK, int MASK>
inline void launch_hop(const HopArgs<SIn, SX, SOut, LK>& A, int nrhs, dd_handle* h) {
    HopArgs<SIn, SX, SOut, LK> B = A;
    if (B.S.n < 0) B.S = SiteSet{nullptr, (long long)A.g.Vh};
    // tile shape from the handle's tuning (threads x sites per thread >= 64,
    // which keeps the grid within the reduction partials)
    const bool f64 = std::is_same<R, double>::value;
    const int tpb = std::min(f64 ? h->tune.hop64_tpb : h->tune.hop_tpb, 128);  // the kernels' launch bound
    // two sites per thread only for the FP32-arithmetic kernels (the FP64
    // kernel needs 130-150 registers for one site)
    constexpr int SPT2 = std::is_same<R, double>::value ? 1 : 2;
    const int spt = (!f64 && h->tune.hop_spt == 2) ? 2 : 1;
    dim3 grid(grid_for(B.S.n, (long long)tpb * spt), nrhs);
    constexpr int kind0 = hop_kind<SIn, SOut>();
    // whole-lattice hops keep kinds 0-2; Dirichlet hops are timed as 4 (FP64),
    // 5, 6 (one block colour's sites) or 8, 9 (every site)
    constexpr int kindm = MASK == 0 ? kind0 : (MASK == 1 && kind0 >= 0 ? (kind0 == 2 ? 4 : 5 + kind0) : -1);
    const int kind = (MASK == 1 && kind0 >= 0 && kind0 < 2 && B.S.colour < 0) ? 8 + kind0 : kindm;
    bool timed = false;
    if (kind >= 0 && h->timer_on && !h->capturing && !dd_stream_capturing(h)) timed = (h->timer_seen[kind]++ % h->timer_every) == 0;
    B.sites = nullptr;
    if (timed) {
        cudaEvent_t e = dd_timer_event(h, kind);
        if (e) cudaEventRecord(e, h->stream);
        B.sites = h->d_sites + kind;
    }
    if (A.red3 == 1)
        DD_KLAUNCH(h, (spt == 2 ? hop_eo_kernel<R, SIn, SX, SOut, LK, MASK, 1, SPT2> : hop_eo_kernel<R, SIn, SX, SOut, LK, MASK, 1, 1>)<<<grid, tpb, 0, h->stream>>>(B));
    else if (A.red3 == 2)
        DD_KLAUNCH(h, (spt == 2 ? hop_eo_kernel<R, SIn, SX, SOut, LK, MASK, 2, SPT2> : hop_eo_kernel<R, SIn, SX, SOut, LK, MASK, 2, 1>)<<<grid, tpb, 0, h->stream>>>(B));
    else
        DD_KLAUNCH(h, (spt == 2 ? hop_eo_kernel<R, SIn, SX, SOut, LK, MASK, 0, SPT2> : hop_eo_kernel<R, SIn, SX, SOut, LK, MASK, 0, 1>)<<<grid, tpb, 0, h->stream>>>(B));
    if (timed) {
        cudaEvent_t e = dd_timer_event(h, kind);
        if (e) cudaEventRecord(e, h->stream);
    }
}
