// Proposal step (Eq. 4step step 0): heat-bath / over-relaxation of the
// Wilson plaquette action S_G = beta sum_P (1 - Re tr U_P / 3) on the active
// links of the selected block colours.
//
// Cabibbo-Marinari: for each link the SU(2) subgroups (0,1), (1,2), (0,2) in
// turn; with the staple sum A and W = U A, the subgroup block w of W has the
// SU(2)-proportional part k V; the new element is R = X V^dag, X drawn from
// exp(alpha x0) dX (alpha = 2 beta k / 3) by the Kennedy-Pendleton sampler
// (at most 64 tries), direction of (x1, x2, x3) uniform; U <- R U.
// Over-relaxation: R = (V^dag)^2.  One launch per (colour, direction, site
// parity) group: links of one direction and one site parity share no
// plaquette, so a group is updated in parallel.
#include <algorithm>
#include <cmath>

#include "dd_internal.h"
#include "reduce.cuh"
#include "su3.cuh"

namespace {

struct Q4 {
    double a0, a1, a2, a3;
};
// 2x2 SU(2) matrix in the parametrisation [[a0 + i a3, a2 + i a1], [-a2 + i a1, a0 - i a3]]
struct M2 {
    cpx<double> m[2][2];
};
DD_DEV M2 su2(double a0, double a1, double a2, double a3) {
    M2 r;
    r.m[0][0] = mk<double>(a0, a3);
    r.m[0][1] = mk<double>(a2, a1);
    r.m[1][0] = mk<double>(-a2, a1);
    r.m[1][1] = mk<double>(a0, -a3);
    return r;
}
DD_DEV M2 mul2(const M2& a, const M2& b) {
    M2 c;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) c.m[i][j] = cmul(a.m[i][0], b.m[0][j]) + cmul(a.m[i][1], b.m[1][j]);
    return c;
}
DD_DEV M2 dag2(const M2& a) {
    M2 c;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) c.m[i][j] = conj(a.m[j][i]);
    return c;
}

DD_DEV M3 link_at(const double* U, long long s, int a) { return load_m3(U + (s * 4 + a) * 18); }

__global__ void heatbath_kernel(Geo g, double* U, const int* links, int n, double beta, int overrelax, int sweep,
                                uint64_t seed, uint64_t ctr0, const unsigned long long* ctr_off,
                                unsigned long long* fails) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint64_t ctr = stream_ctr(ctr0, ctr_off);
    const int l = links[k];
    const int s = l >> 2, a = l & 3;
    int x[4];
    canon_coords(g, s, x);
    const int sa = shift_index(g, x, a, +1);
    int xa[4];
    canon_coords(g, sa, xa);
    // staple sum
    M3 A;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A.m[i][j] = mk<double>(0, 0);
    for (int b = 0; b < 4; ++b) {
        if (b == a) continue;
        const int sb = shift_index(g, x, b, +1);
        const int smb = shift_index(g, x, b, -1);
        const int samb = shift_index(g, xa, b, -1);
        // U_b(s+a) U_a(s+b)^dag U_b(s)^dag
        A = add(A, mul_dag_right(mul_dag_right(link_at(U, sa, b), link_at(U, sb, a)), link_at(U, s, b)));
        // U_b(s+a-b)^dag U_a(s-b)^dag U_b(s-b)
        A = add(A, mul(dagger(mul(link_at(U, smb, a), link_at(U, samb, b))), link_at(U, smb, b)));
    }
    M3 u = link_at(U, s, a);
    const int SG[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    unsigned long long nf = 0;
    for (int sg = 0; sg < 3; ++sg) {
        const int i = SG[sg][0], j = SG[sg][1];
        M3 W = mul(u, A);
        double a0 = 0.5 * (W.m[i][i].x + W.m[j][j].x);
        double a3 = 0.5 * (W.m[i][i].y - W.m[j][j].y);
        double a2 = 0.5 * (W.m[i][j].x - W.m[j][i].x);
        double a1 = 0.5 * (W.m[i][j].y + W.m[j][i].y);
        double kk = sqrt(a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3);
        if (!(kk > 1e-300)) continue;
        M2 Vm = su2(a0 / kk, a1 / kk, a2 / kk, a3 / kk);
        M2 R;
        if (overrelax) {
            R = mul2(dag2(Vm), dag2(Vm));
        } else {
            const uint32_t sub_base = ((uint32_t)sweep << 16) | ((uint32_t)sg << 12);
            const double alpha = 2.0 * beta * kk / 3.0;
            double x0 = 1.0;
            bool ok = false;
            for (int t = 0; t < 64 && !ok; ++t) {
                double u1, u2, u3, u4;
                uniform_pair((uint32_t)l, DD_PURPOSE_HEATBATH, sub_base + 2 * t, seed, ctr, u1, u2);
                uniform_pair((uint32_t)l, DD_PURPOSE_HEATBATH, sub_base + 2 * t + 1, seed, ctr, u3, u4);
                double c = cos(6.283185307179586477 * u2);
                double lam2 = -(log(u1) + c * c * log(u3)) / (2.0 * alpha);
                if (u4 * u4 <= 1.0 - lam2) {
                    x0 = 1.0 - 2.0 * lam2;
                    ok = true;
                }
            }
            if (!ok) {
                ++nf;
                continue;
            }
            double u5, u6;
            uniform_pair((uint32_t)l, DD_PURPOSE_HEATBATH, sub_base + 200, seed, ctr, u5, u6);
            double r = sqrt(fmax(0.0, 1.0 - x0 * x0));
            double cth = 2.0 * u5 - 1.0;
            double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
            double phi = 6.283185307179586477 * u6;
            M2 X = su2(x0, r * sth * cos(phi), r * sth * sin(phi), r * cth);
            R = mul2(X, dag2(Vm));
        }
        for (int c = 0; c < 3; ++c) {
            cpx<double> ui = u.m[i][c], uj = u.m[j][c];
            u.m[i][c] = cmul(R.m[0][0], ui) + cmul(R.m[0][1], uj);
            u.m[j][c] = cmul(R.m[1][0], ui) + cmul(R.m[1][1], uj);
        }
    }
    store_m3(U + ((long long)s * 4 + a) * 18, u);
    if (nf) atomicAdd(fails, nf);
}

// ------------------------------------------------ relative gauge fixing
// Sec. 4 (relative gauge fixing of the proposal to the current field; the
// method is not stated there): maximise F[g] = sum Re tr(U_a(x)^dag g(x)
// U'_a(x) g(x+a)^dag) by sweeps over the sites of one parity at a time; at
// site x, F = Re tr(g(x) W(x)) + const with
//   W(x) = sum_a [U'_a(x) g(x+a)^dag U_a(x)^dag + (U_a(x-a)^dag g(x-a) U'_a(x-a))^dag],
// raised by one Cabibbo-Marinari pass: for subgroup (i,j) the 2x2 block of
// g W is k V (V in SU(2)) plus a part that does not contribute, and
// g <- V^dag_emb g.  G: one SU(3) matrix per site (18 doubles).
__global__ void gauge_identity_kernel(long long V, double* G) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < V) store_m3(G + s * 18, identity3());
}

__global__ void __launch_bounds__(128) gauge_fix_kernel(Geo g, const double* __restrict__ U,
                                                        const double* __restrict__ Up, double* G, int par) {
    const int hh = blockIdx.x * blockDim.x + threadIdx.x;
    if (hh >= g.Vh) return;
    int x[4];
    eo_coords(g, par, hh, x);
    const int s = canon_index(g, x);
    M3 W;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) W.m[i][j] = mk<double>(0, 0);
    for (int a = 0; a < 4; ++a) {
        const int y = shift_index(g, x, a, +1);
        const int z = shift_index(g, x, a, -1);
        // U'_a(x) g(x+a)^dag U_a(x)^dag
        W = add(W, mul_dag_right(mul_dag_right(link_at(Up, s, a), load_m3(G + (long long)y * 18)), link_at(U, s, a)));
        // (U_a(z)^dag g(z) U'_a(z))^dag = U'_a(z)^dag g(z)^dag U_a(z)
        W = add(W, mul(mul_dag_left(link_at(Up, z, a), dagger(load_m3(G + (long long)z * 18))), link_at(U, z, a)));
    }
    M3 gx = load_m3(G + (long long)s * 18);
    const int SG[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    for (int sg = 0; sg < 3; ++sg) {
        const int i = SG[sg][0], j = SG[sg][1];
        M3 M = mul(gx, W);
        double a0 = 0.5 * (M.m[i][i].x + M.m[j][j].x);
        double a3 = 0.5 * (M.m[i][i].y - M.m[j][j].y);
        double a2 = 0.5 * (M.m[i][j].x - M.m[j][i].x);
        double a1 = 0.5 * (M.m[i][j].y + M.m[j][i].y);
        double k = sqrt(a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3);
        if (!(k > 1e-300)) continue;
        M2 R = dag2(su2(a0 / k, a1 / k, a2 / k, a3 / k));
        for (int c = 0; c < 3; ++c) {
            cpx<double> gi = gx.m[i][c], gj = gx.m[j][c];
            gx.m[i][c] = cmul(R.m[0][0], gi) + cmul(R.m[0][1], gj);
            gx.m[j][c] = cmul(R.m[1][0], gi) + cmul(R.m[1][1], gj);
        }
    }
    store_m3(G + (long long)s * 18, gx);
}

// U'_a(x) <- g(x) U'_a(x) g(x+a)^dag (every link), and the functional
// sum Re tr(U^dag U'^g) accumulated into *F (may be null)
__global__ void __launch_bounds__(128) gauge_apply_kernel(Geo g, const double* __restrict__ U, const double* G,
                                                          double* Up, Reduce red) {
    __shared__ double sh[34];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double f = 0.0;
    if (s < g.V) {
        int x[4];
        canon_coords(g, s, x);
        const M3 gs = load_m3(G + (long long)s * 18);
        for (int a = 0; a < 4; ++a) {
            const int y = shift_index(g, x, a, +1);
            M3 v = mul_dag_right(mul(gs, link_at(Up, s, a)), load_m3(G + (long long)y * 18));
            store_m3(Up + ((long long)s * 4 + a) * 18, v);
            M3 t = mul_dag_left(link_at(U, s, a), v);
            f += t.m[0][0].x + t.m[1][1].x + t.m[2][2].x;
        }
    }
    if (red.op != FIN_NONE) grid_reduce(red, 0, f, sh);
}

}  // namespace

extern "C" int dd_relative_gauge_fix(dd_t h, const void* U, void* U_new, int sweeps, double* functional) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_estimate, "dd_relative_gauge_fix");
    if (rc) return rc;
    if (!U || !U_new || sweeps < 0 || sweeps > 10000) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_relative_gauge_fix: bad arguments");
    const Geo& g = h->g;
    double* G = h->d_gauge_g;
    DD_KLAUNCH(h, gauge_identity_kernel<<<grid_for(g.V, 128), 128, 0, h->stream>>>(g.V, G));
    for (int k = 0; k < sweeps; ++k)
        for (int par = 0; par < 2; ++par)
            DD_KLAUNCH(h, gauge_fix_kernel<<<grid_for(g.Vh, 128), 128, 0, h->stream>>>(g, (const double*)U,
                                                                                   (const double*)U_new, G, par));
    Reduce red;
    red.partials = h->d_partials;
    red.counters = h->d_counters;
    red.st = nullptr;
    red.out = functional;
    red.op = functional ? FIN_STORE : FIN_NONE;
    red.status = h->d_status;
    DD_KLAUNCH(h, gauge_apply_kernel<<<grid_for(g.V, 128), 128, 0, h->stream>>>(g, (const double*)U, G,
                                                                              (double*)U_new, red));
    DD_LAUNCH_CHECK(h, "dd_relative_gauge_fix");
    return DD_OK;
}

extern "C" int dd_gauge_update(dd_t h, void* U, int colour_mask, double beta, int n_hb, int n_or, uint64_t seed,
                               uint64_t ctr) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    if (!U || colour_mask < 1 || colour_mask > 3 || !(beta > 0) || n_hb < 0 || n_or < 0 || n_hb > 255)
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_gauge_update: bad arguments");
    for (int sweep = 0; sweep < n_hb; ++sweep)
        for (int kind = 0; kind <= n_or; ++kind)
            for (int a = 0; a < 4; ++a)
                for (int par = 0; par < 2; ++par)
                    for (int col = 0; col < 2; ++col) {
                        if (!((colour_mask >> col) & 1)) continue;
                        int gi = (col * 4 + a) * 2 + par;
                        int off = h->h_group_off[gi], cnt = h->h_group_off[gi + 1] - off;
                        if (cnt <= 0) continue;
                        DD_KLAUNCH(h, heatbath_kernel<<<grid_for(cnt, 64), 64, 0, h->stream>>>(
                            h->g, (double*)U, h->d_active_links + off, cnt, beta, kind > 0, sweep, seed, ctr,
                            h->d_ctr_off, h->d_hb_fails));
                    }
    DD_LAUNCH_CHECK(h, "heatbath_kernel");
    return DD_OK;
}
