// Schwarz-preconditioned flexible GCR: an inner solver of the global
// defect-correction loop (krylov DD_KRYLOV_SAP_GCR).
//
// The inner system Dtilde e = r (even sites) is solved as the full system
//   D (e, e_o) = (r, 0),  D = [[1, -kappa H_eo], [-kappa H_oe, 1]],
// whose even part is e (the odd row gives e_o = kappa H_oe e, the even row
// then reads Dtilde e = r).  Flexible GCR on D, FP32 vectors on both
// parities, preconditioned by ncy cycles of the Schwarz alternating
// procedure over the black/white blocks of the decomposition (Sec. 3):
//   z = 0, y = rho;  per cycle, for colour c = black, white:
//     q = rho - D z on the sites of colour c   (computed as y + kappa H z_other,
//                                                with y = rho - z kept up to date)
//     delta = D_c^{-1} q on every block of colour c, approximately: nmr
//             BiCGStab iterations of the blocks' even-odd Dirichlet system
//             Dtilde_c delta_e = q_e + kappa H_eo q_o, then
//             delta_o = q_o + kappa H_oe delta_e (hops inside the blocks)
//     z += delta, y -= delta
// GCR: z_k = SAP(r), w_k = D z_k, w_k and z_k orthogonalised against the
// kept w_j by classical Gram-Schmidt done twice (the same coefficients on
// z), scaled to |w_k| = 1, alpha = <w_k, r>, x += alpha z_k, r -= alpha w_k;
// after nkv directions the directions are dropped and x, r kept.
// All scalars are FP64 sums formed on the device in a fixed order; the host
// polls the residuals once per GCR iteration.
#pragma once

struct FullF32 {
    SpinorF32 e, o;
};
struct FullSet {
    FullF32 v[DD_SAP_MAX_NKV];
};

DD_DEV FullF32 f_at_rhs(FullF32 f, int r) {
    f.e = at_rhs(f.e, r);
    f.o = at_rhs(f.o, r);
    return f;
}

// complex <a, b> and |b|^2 accumulation in FP32 per site, FP64 across sites
DD_DEV void cdot_acc(const Spinor<float>& a, const Spinor<float>& b, double& re, double& im) {
    float d0 = 0.f, d1 = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        d0 += a.c[k].x * b.c[k].x + a.c[k].y * b.c[k].y;
        d1 += a.c[k].x * b.c[k].y - a.c[k].y * b.c[k].x;
    }
    re += (double)d0;
    im += (double)d1;
}

// per-block partial sums of <A_i, B> for i < na (both parities of the sites
// of S): value v = 2 i (real part) or 2 i + 1 (imaginary part) of system rhs
// at part[(rhs * 2 (MAX + 1) + v) * nblk + block]
__global__ void __launch_bounds__(128) sap_mdot_kernel(SiteSet S, FullSet A, int na, FullF32 B, const CGState* st,
                                                       double* part, int nblk) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    if (st && !st[rhs].active) return;
    double acc[2 * (DD_SAP_MAX_NKV + 1)];
#pragma unroll
    for (int i = 0; i < 2 * (DD_SAP_MAX_NKV + 1); ++i) acc[i] = 0.0;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < S.n) {
        const long long h = S.at(t);
        const FullF32 b = f_at_rhs(B, rhs);
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            Spinor<float> bv;
            (par ? b.o : b.e).load(h, bv);
            for (int i = 0; i < na; ++i) {
                const FullF32 a = f_at_rhs(A.v[i], rhs);
                Spinor<float> av;
                (par ? a.o : a.e).load(h, av);
                cdot_acc(av, bv, acc[2 * i], acc[2 * i + 1]);
            }
        }
    }
    for (int i = 0; i < 2 * na; ++i) {
        const double s = block_sum(acc[i], sh);
        if (threadIdx.x == 0) part[((long long)rhs * 2 * (DD_SAP_MAX_NKV + 1) + i) * nblk + blockIdx.x] = s;
    }
}

// out[rhs * 2 (MAX + 1) + i] = sum over the partials of value i (fixed order)
__global__ void __launch_bounds__(256) sap_sum_kernel(const double* part, int nblk, int nvals, const CGState* st,
                                                      double* out) {
    __shared__ double sh[34];
    const int i = blockIdx.x, rhs = blockIdx.y;
    if (i >= nvals || (st && !st[rhs].active)) return;
    const double* p = part + ((long long)rhs * 2 * (DD_SAP_MAX_NKV + 1) + i) * nblk;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += p[b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[rhs * 2 * (DD_SAP_MAX_NKV + 1) + i] = s;
}

// w_j -= sum_i c_i w_i, z_j -= sum_i c_i z_i (c from the sums of <w_i, w_j>)
__global__ void __launch_bounds__(128) sap_gs_kernel(SiteSet S, FullSet W, FullSet Z, int j, const double* dots,
                                                     const CGState* st) {
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.n) return;
    const long long h = S.at(t);
    const double* c = dots + rhs * 2 * (DD_SAP_MAX_NKV + 1);
#pragma unroll
    for (int par = 0; par < 2; ++par) {
        Spinor<float> w, z;
        const FullF32 wj = f_at_rhs(W.v[j], rhs), zj = f_at_rhs(Z.v[j], rhs);
        (par ? wj.o : wj.e).load(h, w);
        (par ? zj.o : zj.e).load(h, z);
        for (int i = 0; i < j; ++i) {
            const cpx<float> ci = mk<float>((float)c[2 * i], (float)c[2 * i + 1]);
            Spinor<float> wi, zi;
            const FullF32 wa = f_at_rhs(W.v[i], rhs), za = f_at_rhs(Z.v[i], rhs);
            (par ? wa.o : wa.e).load(h, wi);
            (par ? za.o : za.e).load(h, zi);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                w.c[k] = w.c[k] - cmul(ci, wi.c[k]);
                z.c[k] = z.c[k] - cmul(ci, zi.c[k]);
            }
        }
        (par ? wj.o : wj.e).store(h, w);
        (par ? zj.o : zj.e).store(h, z);
    }
}

// scalars of one GCR step (one thread per system):
//   op 0: s = 1 / |w_j| from sums[0] = |w_j|^2 (breakdown: system ends)
//   op 1: alpha = <w_j, r> from sums[0..1]
//   op 2: |r|^2 from sums[0]: convergence, iteration count
__global__ void sap_scalar_kernel(int nrhs, int op, const double* sums, double* sc, CGState* st, int* status) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs || !st[r].active) return;
    const double* s = sums + r * 2 * (DD_SAP_MAX_NKV + 1);
    double* o = sc + r * 4;
    CGState& c = st[r];
    if (op == 0) {
        if (!(s[0] > 0.0) || !isfinite(s[0])) {
            c.active = 0;
            c.flags |= 4;
            if (!isfinite(s[0])) {
                c.flags |= 2;
                raise_status(status, DD_ERR_NUMERIC);
            }
            return;
        }
        o[0] = 1.0 / sqrt(s[0]);
    } else if (op == 1) {
        o[1] = s[0];
        o[2] = s[1];
    } else {
        c.rr = s[0];
        c.iters += 1;
        if (!isfinite(s[0])) {
            c.active = 0;
            c.flags |= 2;
            raise_status(status, DD_ERR_NUMERIC);
        } else if (s[0] <= c.tol2) {
            c.active = 0;
        } else if (c.iters >= c.maxit) {
            c.active = 0;
            c.flags |= 1;
        }
    }
}

// w_j *= s, z_j *= s
__global__ void __launch_bounds__(128) sap_scale_kernel(SiteSet S, FullF32 W, FullF32 Z, const double* sc,
                                                        const CGState* st) {
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.n) return;
    const long long h = S.at(t);
    const float s = (float)sc[rhs * 4];
    const FullF32 w = f_at_rhs(W, rhs), z = f_at_rhs(Z, rhs);
#pragma unroll
    for (int par = 0; par < 2; ++par) {
        Spinor<float> a, b;
        (par ? w.o : w.e).load(h, a);
        (par ? z.o : z.e).load(h, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            a.c[k] = s * a.c[k];
            b.c[k] = s * b.c[k];
        }
        (par ? w.o : w.e).store(h, a);
        (par ? z.o : z.e).store(h, b);
    }
}

// x += alpha z_j, r -= alpha w_j; partial sums of |r|^2
__global__ void __launch_bounds__(128) sap_xr_kernel(SiteSet S, FullF32 X, FullF32 R, FullF32 Z, FullF32 W,
                                                     const double* sc, const CGState* st, double* part, int nblk) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double nrm = 0.0;
    if (t < S.n) {
        const long long h = S.at(t);
        const cpx<float> al = mk<float>((float)sc[rhs * 4 + 1], (float)sc[rhs * 4 + 2]);
        const FullF32 x = f_at_rhs(X, rhs), r = f_at_rhs(R, rhs), z = f_at_rhs(Z, rhs), w = f_at_rhs(W, rhs);
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            Spinor<float> a, b;
            (par ? x.o : x.e).load(h, a);
            (par ? z.o : z.e).load(h, b);
#pragma unroll
            for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] + cmul(al, b.c[k]);
            (par ? x.o : x.e).store(h, a);
            (par ? r.o : r.e).load(h, a);
            (par ? w.o : w.e).load(h, b);
#pragma unroll
            for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] - cmul(al, b.c[k]);
            (par ? r.o : r.e).store(h, a);
            nrm += (double)snorm2(a);
        }
    }
    const double s = block_sum(nrm, sh);
    if (threadIdx.x == 0) part[((long long)rhs * 2 * (DD_SAP_MAX_NKV + 1)) * nblk + blockIdx.x] = s;
}

// start of a GCR solve: x = 0 (both parities), r_o = 0 (r_e holds the right-hand side)
__global__ void __launch_bounds__(128) sap_start_kernel(SiteSet S, FullF32 X, SpinorF32 Ro, const CGState* st) {
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.n) return;
    const long long h = S.at(t);
    Spinor<float> z;
    zero(z);
    const FullF32 x = f_at_rhs(X, rhs);
    x.e.store(h, z);
    x.o.store(h, z);
    at_rhs(Ro, rhs).store(h, z);
}

// start of a preconditioner application: z = 0, y = rho (both parities)
__global__ void __launch_bounds__(128) sap_pre_start_kernel(SiteSet S, FullF32 Z, FullF32 Y, FullF32 Rho,
                                                            const CGState* st) {
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.n) return;
    const long long h = S.at(t);
    const FullF32 z = f_at_rhs(Z, rhs), y = f_at_rhs(Y, rhs), rho = f_at_rhs(Rho, rhs);
    Spinor<float> a, zz;
    zero(zz);
#pragma unroll
    for (int par = 0; par < 2; ++par) {
        (par ? z.o : z.e).store(h, zz);
        (par ? rho.o : rho.e).load(h, a);
        (par ? y.o : y.e).store(h, a);
    }
}

// on the sites of one colour: z += delta, y -= delta
__global__ void __launch_bounds__(128) sap_update_kernel(SiteSet Sc, FullF32 Z, FullF32 Y, SpinorF32 de, SpinorF32 dod,
                                                         const CGState* st) {
    const int rhs = blockIdx.y;
    if (!st[rhs].active) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Sc.n) return;
    const long long h = Sc.at(t);
    const FullF32 z = f_at_rhs(Z, rhs), y = f_at_rhs(Y, rhs);
#pragma unroll
    for (int par = 0; par < 2; ++par) {
        Spinor<float> d, a;
        at_rhs(par ? dod : de, rhs).load(h, d);
        (par ? z.o : z.e).load(h, a);
#pragma unroll
        for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] + d.c[k];
        (par ? z.o : z.e).store(h, a);
        (par ? y.o : y.e).load(h, a);
#pragma unroll
        for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] - d.c[k];
        (par ? y.o : y.e).store(h, a);
    }
}

// |v|^2 of an even-sized FP32 vector on the sites of S (per system), to `out`
__global__ void __launch_bounds__(128) sap_norm_kernel(SiteSet S, SpinorF32 v, const CGState* st, Reduce red) {
    __shared__ double sh[34];
    const int rhs = blockIdx.y;
    if (st && !st[rhs].active) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double nrm = 0.0;
    if (t < S.n) {
        Spinor<float> a;
        at_rhs(v, rhs).load(S.at(t), a);
        nrm = (double)snorm2(a);
    }
    grid_reduce(red, rhs, nrm, sh);
}

// hop-storage view of a SAP half vector (FP16: chunks, then the per-site scales)
template <class SH>
SH sap_hop_storage(dd_handle* h, int k);
template <>
SpinorF32 sap_hop_storage<SpinorF32>(dd_handle* h, int k) {
    return SpinorF32{h->sap.at(k), h->g.Vh};
}
template <>
SpinorF16 sap_hop_storage<SpinorF16>(dd_handle* h, int k) {
    uint4* p = reinterpret_cast<uint4*>(h->sap.at(k));
    const long long Vh = h->g.Vh;
    return SpinorF16{p, reinterpret_cast<float*>(p + (size_t)h->prm.max_rhs * 3 * Vh), Vh};
}

// per-system scalar areas of h->sap.sc (R = max_rhs): sums of the
// reductions [0, 34 R), step scalars [34 R, 38 R), block |rhs|^2 [38 R, 39 R)
inline double* sap_sums(dd_handle* h) { return h->sap.sc; }
inline double* sap_scal(dd_handle* h) { return h->sap.sc + 2 * (DD_SAP_MAX_NKV + 1) * h->prm.max_rhs; }
inline double* sap_rr(dd_handle* h) { return h->sap.sc + (2 * (DD_SAP_MAX_NKV + 1) + 4) * h->prm.max_rhs; }

template <class SH, class LK>
struct SapGcr {
    dd_handle* h;
    int nrhs;
    SpinorF32 x, r;     // even parts: the correction (out) and the right-hand side (in, overwritten)
    CGState* st;        // GCR states
    const CGState* outer;
    SiteSet S;          // all even (and odd) site indices 0 .. Vh - 1
    LK lk;
    long long lk_rs;
    CGState* bst;       // block-solver states
    int ncy, nmr, nkv;

    FullF32 full(int k) const {
        const long long Vh = h->g.Vh;
        return FullF32{SpinorF32{h->sap.at(k), Vh}, SpinorF32{h->sap.at(k + 1), Vh}};
    }
    FullF32 X() const { return FullF32{x, SpinorF32{h->sap.at(0), h->g.Vh}}; }
    FullF32 R() const { return FullF32{r, SpinorF32{h->sap.at(1), h->g.Vh}}; }
    FullF32 Y() const { return full(2); }
    FullF32 Q() const { return full(4); }
    SpinorF32 dod() const { return SpinorF32{h->sap.at(6), h->g.Vh}; }
    FullF32 Zk(int k) const { return full(SapVecs::kFixedHalves + 2 * k); }
    FullF32 Wk(int k) const { return full(SapVecs::kFixedHalves + 2 * nkv + 2 * k); }

    template <class SIn, class SX, int MASK>
    void hop(SiteSet Ss, int par, SIn in, SX xin, SpinorF32 out, double a, double b) {
        HopArgs<SIn, SX, SpinorF32, LK> A;
        A.g = h->g;
        A.p = par;
        A.in = in;
        A.xin = xin;
        A.out = out;
        A.lk = lk;
        A.lk_rhs_stride = lk_rs;
        A.a = a;
        A.b = b;
        A.has_x = 1;
        A.g5in = 0;
        A.g5out = 0;
        A.colour_mask = 3;
        A.st = st;
        Reduce none;
        none.partials = nullptr;
        none.counters = nullptr;
        none.st = nullptr;
        none.out = nullptr;
        none.op = FIN_NONE;
        none.status = nullptr;
        A.red = none;
        A.red3 = 0;
        A.rhat = xin;
        A.S = Ss;
        launch_hop<float, SIn, SX, SpinorF32, LK, MASK>(A, nrhs, h);
    }
    // out = D in on both parities (sites of Ss)
    void apply_D(SiteSet Ss, FullF32 in, FullF32 out) {
        const double k = h->prm.kappa;
        hop<SpinorF32, SpinorF32, 0>(Ss, 0, in.o, in.e, out.e, 1.0, -k);
        hop<SpinorF32, SpinorF32, 0>(Ss, 1, in.e, in.o, out.o, 1.0, -k);
    }
    Reduce store_red(double* out) const {
        Reduce R_;
        R_.partials = h->d_partials;
        R_.counters = h->d_counters;
        R_.st = nullptr;
        R_.out = out;
        R_.op = FIN_STORE;
        R_.status = h->d_status;
        return R_;
    }

    // z = SAP(rho), ncy cycles
    int precondition(FullF32 rho, FullF32 z) {
        const long long Vh = h->g.Vh;
        const double k = h->prm.kappa;
        dim3 grid(grid_for(S.n, 128), nrhs);
        const FullF32 y = Y(), q = Q();
        DD_KLAUNCH(h, sap_pre_start_kernel<<<grid, 128, 0, h->stream>>>(S, z, y, rho, st));
        BiCGStab<float, SpinorF32, SH, LK, 1> b;
        b.h = h;
        b.nrhs = nrhs;
        b.x = SpinorF32{h->sap.at(7), Vh};
        b.r = SpinorF32{h->sap.at(8), Vh};
        b.v = SpinorF32{h->sap.at(9), Vh};
        b.s = SpinorF32{h->sap.at(10), Vh};
        b.t = SpinorF32{h->sap.at(11), Vh};
        b.p = sap_hop_storage<SH>(h, 12);
        b.rhat = sap_hop_storage<SH>(h, 13);
        b.shop = sap_hop_storage<SH>(h, 14);
        b.th = sap_hop_storage<SH>(h, 15);
        b.copies = std::is_same<SH, SpinorF16>::value ? 1 : 0;
        if (!b.copies) b.shop = sap_hop_storage<SH>(h, 10);  // FP32 storage: s is its own hop copy
        b.lk = lk;
        b.lk_rs = lk_rs;
        b.st = bst;
        b.outer = st;
        double* rr = sap_rr(h);  // per-system |rhs|^2 of a block solve
        for (int cy = 0; cy < ncy; ++cy)
            for (int c = 0; c < 2; ++c) {
                if (!h->d_colour_sites[c]) return DD_ERR_UNSUPPORTED;
                const SiteSet Sc{h->d_colour_sites[c], Vh / 2, c};
                b.S = Sc;
                // q = rho - D z on colour c: y + kappa H z (y = rho - z)
                hop<SpinorF32, SpinorF32, 0>(Sc, 0, z.o, y.e, q.e, 1.0, k);
                hop<SpinorF32, SpinorF32, 0>(Sc, 1, z.e, y.o, q.o, 1.0, k);
                // block solves: Dtilde_c d_e = q_e + kappa H_eo q_o (hops inside the blocks)
                hop<SpinorF32, SpinorF32, 1>(Sc, 0, q.o, q.e, b.r, 1.0, k);
                dim3 gc(grid_for(Sc.n, 128), nrhs);
                DD_KLAUNCH(h, sap_norm_kernel<<<gc, 128, 0, h->stream>>>(Sc, b.r, st, store_red(rr)));
                int its = 0;
                int rc = b.run(rr, 0.0, 0.0, nmr, nmr, &its);
                if (rc) return rc;
                // d_o = q_o + kappa H_oe d_e
                hop<SpinorF32, SpinorF32, 1>(Sc, 1, b.x, q.o, dod(), 1.0, k);
                DD_KLAUNCH(h, sap_update_kernel<<<gc, 128, 0, h->stream>>>(Sc, z, y, b.x, dod(), st));
            }
        return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
    }

    // sums of <A_i, B> (i < na) per system into h->sap.sc's sum area
    double* sums() const { return sap_sums(h); }
    void mdot(const FullSet& A, int na, FullF32 B) {
        dim3 grid(h->sap.nblk, nrhs);
        DD_KLAUNCH(h, sap_mdot_kernel<<<grid, 128, 0, h->stream>>>(S, A, na, B, st, h->sap.partials, h->sap.nblk));
        DD_KLAUNCH(h, sap_sum_kernel<<<dim3(2 * na, nrhs), 256, 0, h->stream>>>(h->sap.partials, h->sap.nblk, 2 * na, st,
                                                                                sums()));
    }

    int run(const double* rr0, double tol, double abs_fac, int maxit, int chunk, int* iters_out) {
        (void)chunk;
        if (h->capturing || dd_stream_capturing(h)) return DD_ERR_UNSUPPORTED;  // host-polled loop
        if (maxit < 1) maxit = 1;
        dim3 grid(grid_for(S.n, 128), nrhs);
        double* scal = sap_scal(h);
        DD_KLAUNCH(h, cg_arm_kernel<<<1, 64, 0, h->stream>>>(nrhs, st, outer, rr0, tol, abs_fac, maxit));
        const FullF32 X_ = X(), R_ = R();
        DD_KLAUNCH(h, sap_start_kernel<<<grid, 128, 0, h->stream>>>(S, X_, R_.o, st));
        FullSet W, Z;
        for (int k = 0; k < nkv; ++k) {
            W.v[k] = Wk(k);
            Z.v[k] = Zk(k);
        }
        std::vector<CGState> hs(nrhs);
        int done = 0;
        for (;;) {
            const int j = done % nkv;
            int rc = precondition(R_, Z.v[j]);
            if (rc) return rc;
            apply_D(S, Z.v[j], W.v[j]);
            for (int pass = 0; pass < 2 && j > 0; ++pass) {  // classical Gram-Schmidt, twice
                mdot(W, j, W.v[j]);
                DD_KLAUNCH(h, sap_gs_kernel<<<grid, 128, 0, h->stream>>>(S, W, Z, j, sums(), st));
            }
            FullSet one;
            one.v[0] = W.v[j];
            mdot(one, 1, W.v[j]);  // |w_j|^2 (real part)
            DD_KLAUNCH(h, sap_scalar_kernel<<<grid_for(nrhs, 64), 64, 0, h->stream>>>(nrhs, 0, sums(), scal, st,
                                                                                      h->d_status));
            DD_KLAUNCH(h, sap_scale_kernel<<<grid, 128, 0, h->stream>>>(S, W.v[j], Z.v[j], scal, st));
            mdot(one, 1, R_);  // alpha = <w_j, r>
            DD_KLAUNCH(h, sap_scalar_kernel<<<grid_for(nrhs, 64), 64, 0, h->stream>>>(nrhs, 1, sums(), scal, st,
                                                                                      h->d_status));
            DD_KLAUNCH(h, sap_xr_kernel<<<dim3(h->sap.nblk, nrhs), 128, 0, h->stream>>>(S, X_, R_, Z.v[j], W.v[j], scal,
                                                                                     st, h->sap.partials,
                                                                                     h->sap.nblk));
            DD_KLAUNCH(h, sap_sum_kernel<<<dim3(1, nrhs), 256, 0, h->stream>>>(h->sap.partials, h->sap.nblk, 1, st,
                                                                              sums()));
            DD_KLAUNCH(h, sap_scalar_kernel<<<grid_for(nrhs, 64), 64, 0, h->stream>>>(nrhs, 2, sums(), scal, st,
                                                                                      h->d_status));
            if (cudaGetLastError() != cudaSuccess) return DD_ERR_CUDA;
            ++done;
            if (cudaMemcpyAsync(hs.data(), st, sizeof(CGState) * nrhs, cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess)
                return DD_ERR_CUDA;
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DD_ERR_CUDA;
            bool any = false;
            for (int k = 0; k < nrhs; ++k) any = any || hs[k].active;
            if (!any || done >= maxit) break;
        }
        int tot = 0;
        for (int k = 0; k < nrhs; ++k) tot += hs[k].iters;
        if (iters_out) *iters_out += tot;
        return DD_OK;
    }
};
