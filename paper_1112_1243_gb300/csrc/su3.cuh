// FP64 3x3 complex matrix helpers for the gauge-field kernels: products,
// a cyclic Jacobi eigen-solver and the SU(3) power W^t used by the geodesic
// interpolation of Eq. param.
#pragma once

#include "dd_common.cuh"

struct M3 {
    cpx<double> m[3][3];
};

DD_DEV M3 load_m3(const double* p) {
    M3 a;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) a.m[i][j] = mk<double>(p[2 * (3 * i + j)], p[2 * (3 * i + j) + 1]);
    return a;
}
DD_DEV void store_m3(double* p, const M3& a) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            p[2 * (3 * i + j)] = a.m[i][j].x;
            p[2 * (3 * i + j) + 1] = a.m[i][j].y;
        }
}
DD_DEV M3 mul(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cpx<double> s = mk<double>(0, 0);
#pragma unroll
            for (int k = 0; k < 3; ++k) s = cmac(s, a.m[i][k], b.m[k][j]);
            c.m[i][j] = s;
        }
    return c;
}
DD_DEV M3 dagger(const M3& a) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c.m[i][j] = conj(a.m[j][i]);
    return c;
}
// a^dag b
DD_DEV M3 mul_dag_left(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cpx<double> s = mk<double>(0, 0);
#pragma unroll
            for (int k = 0; k < 3; ++k) s = cmacc(s, a.m[k][i], b.m[k][j]);
            c.m[i][j] = s;
        }
    return c;
}
// a b^dag
DD_DEV M3 mul_dag_right(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cpx<double> s = mk<double>(0, 0);
#pragma unroll
            for (int k = 0; k < 3; ++k) s = cmac(s, a.m[i][k], conj(b.m[j][k]));
            c.m[i][j] = s;
        }
    return c;
}
DD_DEV M3 add(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c.m[i][j] = a.m[i][j] + b.m[i][j];
    return c;
}
DD_DEV M3 identity3() {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c.m[i][j] = mk<double>(i == j ? 1.0 : 0.0, 0.0);
    return c;
}

// Unitary rotation J in the (p, q) plane that diagonalises the Hermitian 2x2
// matrix [[a, b], [conj(b), d]] (a, d real): J = diag(1, e^{-i phi}) R with the
// real Jacobi rotation R = [[c, s], [-s, c]] (Numerical Recipes form).
struct Rot2 {
    cpx<double> j00, j01, j10, j11;
};
DD_DEV Rot2 jacobi2(double a, cpx<double> b, double d) {
    Rot2 r;
    double bb = sqrt(norm2(b));
    if (bb < 1e-300) {
        r.j00 = r.j11 = mk<double>(1, 0);
        r.j01 = r.j10 = mk<double>(0, 0);
        return r;
    }
    cpx<double> e = mk<double>(b.x / bb, -b.y / bb);  // e^{-i phi}
    double th = (d - a) / (2.0 * bb);
    double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
    double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
    r.j00 = mk<double>(c, 0);
    r.j01 = mk<double>(s, 0);
    r.j10 = -s * e;
    r.j11 = c * e;
    return r;
}
// V <- V J (columns p, q), and K <- J^dag K J when K is given
DD_DEV void rotate_cols(M3& V, int p, int q, const Rot2& J) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        cpx<double> vp = V.m[i][p], vq = V.m[i][q];
        V.m[i][p] = cmul(vp, J.j00) + cmul(vq, J.j10);
        V.m[i][q] = cmul(vp, J.j01) + cmul(vq, J.j11);
    }
}
DD_DEV void rotate_rows_dag(M3& K, int p, int q, const Rot2& J) {
    // K <- J^dag K (rows p, q)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        cpx<double> kp = K.m[p][j], kq = K.m[q][j];
        K.m[p][j] = cmulc(J.j00, kp) + cmulc(J.j10, kq);
        K.m[q][j] = cmulc(J.j01, kp) + cmulc(J.j11, kq);
    }
}

// Eigenvectors V (columns) of the Hermitian K by cyclic Jacobi sweeps.
DD_DEV M3 jacobi_eigvecs(M3 K) {
    M3 V = identity3();
    for (int sweep = 0; sweep < 12; ++sweep) {
        double off = norm2(K.m[0][1]) + norm2(K.m[0][2]) + norm2(K.m[1][2]);
        double dia = K.m[0][0].x * K.m[0][0].x + K.m[1][1].x * K.m[1][1].x + K.m[2][2].x * K.m[2][2].x;
        if (off <= 1e-34 * (dia + 1e-300)) break;
        const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
        for (int k = 0; k < 3; ++k) {
            int p = P[k], q = Q[k];
            Rot2 J = jacobi2(K.m[p][p].x, K.m[p][q], K.m[q][q].x);
            rotate_cols(K, p, q, J);
            rotate_rows_dag(K, p, q, J);
            rotate_cols(V, p, q, J);
        }
    }
    return V;
}

// W^t for W in SU(3): eigen-decomposition W = V diag(e^{i theta}) V^dag with
// theta in (-pi, pi]; when the phases sum to +-2 pi the largest (smallest)
// phase is moved by -+2 pi so that det W^t = 1 along the path.
// Stage 1 diagonalises the Hermitian K = Re(W) + c Im(W) (generic c); stage 2
// resolves pairs left coupled by (near-)degenerate eigenvalues of K with the
// orthogonal combination S = Im(e^{-i phi0} W), phi0 = atan(c).
// The decomposition (V, theta) is computed once per link by su3_eig and
// W^t = V diag(e^{i t theta}) V^dag evaluated per t by su3_power_eig.
DD_DEV void su3_eig(const M3& W, M3& V, double th[3]) {
    const double c = 0.6180339887498949;
    M3 K;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cpx<double> w = W.m[i][j], wd = conj(W.m[j][i]);
            cpx<double> re = 0.5 * (w + wd);                  // (W + W^dag)/2
            cpx<double> im = mk<double>(0.5 * (w.y - wd.y) * 1.0, -0.5 * (w.x - wd.x));  // (W - W^dag)/(2i)
            K.m[i][j] = re + c * im;
        }
    V = jacobi_eigvecs(K);
    const double n0 = 1.0 / sqrt(1.0 + c * c);
    const double ca = n0, sa = c * n0;  // e^{i phi0} = ca + i sa
    for (int sweep = 0; sweep < 3; ++sweep) {
        M3 G = mul_dag_left(V, mul(W, V));
        const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
        bool any = false;
        for (int k = 0; k < 3; ++k) {
            int p = P[k], q = Q[k];
            if (norm2(G.m[p][q]) + norm2(G.m[q][p]) < 1e-30) continue;
            any = true;
            // S = (e^{-i phi0} B - e^{i phi0} B^dag) / (2i) on the 2x2 block B
            cpx<double> em = mk<double>(ca, -sa);
            cpx<double> Bpp = G.m[p][p], Bpq = G.m[p][q], Bqp = G.m[q][p], Bqq = G.m[q][q];
            auto Sij = [&](cpx<double> bij, cpx<double> bji) {
                cpx<double> x = cmul(em, bij) - conj(cmul(em, bji));
                return mk<double>(0.5 * x.y, -0.5 * x.x);
            };
            cpx<double> spp = Sij(Bpp, Bpp), spq = Sij(Bpq, Bqp), sqq = Sij(Bqq, Bqq);
            Rot2 J = jacobi2(spp.x, spq, sqq.x);
            rotate_cols(V, p, q, J);
            G = mul_dag_left(V, mul(W, V));
        }
        if (!any) break;
    }
    M3 G = mul_dag_left(V, mul(W, V));
#pragma unroll
    for (int j = 0; j < 3; ++j) th[j] = atan2(G.m[j][j].y, G.m[j][j].x);
    double sum = th[0] + th[1] + th[2];
    if (sum > 3.141592653589793) {
        int j = (th[0] >= th[1] && th[0] >= th[2]) ? 0 : (th[1] >= th[2] ? 1 : 2);
        th[j] -= 6.283185307179586;
    } else if (sum < -3.141592653589793) {
        int j = (th[0] <= th[1] && th[0] <= th[2]) ? 0 : (th[1] <= th[2] ? 1 : 2);
        th[j] += 6.283185307179586;
    }
}
DD_DEV M3 su3_power_eig(const M3& V, const double th[3], double t) {
    M3 out;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cpx<double> s = mk<double>(0, 0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double sn, cs;
                sincos(t * th[k], &sn, &cs);
                s = s + cmul(cmul(V.m[i][k], mk<double>(cs, sn)), conj(V.m[j][k]));
            }
            out.m[i][j] = s;
        }
    return out;
}
DD_DEV M3 su3_power(const M3& W, double t) {
    M3 V;
    double th[3];
    su3_eig(W, V, th);
    return su3_power_eig(V, th, t);
}
