// Batched Dirichlet block solves in one persistent launch (Eq. 4step step 1
// and the block inverses A^{-1}, E^{-1} of the Schur complement, Eq. ddfactor).
//
// Every thread block of the grid takes work items (block, factor) from an
// atomic queue and runs a complete solve of D_b x = src for that item with
// the whole thread block: FP64 defect correction around an inner CG on the
// block's normal equations (FP32 arithmetic on FP32 storage, or FP64), all
// vectors in a per-thread-block scratch slot laid out block-local and
// chunk-major (coalesced, L2-resident for blocks up to 8^4 sites).
//
// D_b = 1 - kappa * H restricted to hops with both ends in block b (Dirichlet
// boundary: hops leaving the block are dropped).  Blocks never straddle the
// time edge (at least two blocks per direction), so no boundary phase occurs
// inside a block.  Block data (links, vectors) are stored in block order:
// position q = block_pos * bsites + local index, local index lexicographic.
#pragma once

#include <type_traits>

#include "dd_internal.h"
#include "reduce.cuh"

struct BlockCtx {
    int bd[4];    // block extents
    int st[4];    // local strides
    int nb;       // sites per block
    double kappa;
};

DD_DEV void local_coords(const BlockCtx& c, int j, int l[4]) {
    l[0] = j % c.bd[0];
    int r = j / c.bd[0];
    l[1] = r % c.bd[1];
    r /= c.bd[1];
    l[2] = r % c.bd[2];
    l[3] = r / c.bd[2];
}

// acc = H_b in at local site j (hops inside the block only)
template <class R, class SIn, class LK>
DD_DEV void dirichlet_hop(const BlockCtx& c, int j, const SIn& in, const LK& lk, int g5in, Spinor<R>& acc) {
    int l[4];
    local_coords(c, j, l);
    zero(acc);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        if (l[a] < c.bd[a] - 1) {
            int jn = j + c.st[a];
            Spinor<R> s;
            in.load(jn, s);
            if (g5in) gamma5(s);
            Half<R> hf, uh;
            project<R>(a, +1, s, hf);
            Link<R> u;
            lk.load(j, a, u);
            mul_link(u, hf, uh);
            accumulate<R>(a, +1, uh, (R)1, acc);
        }
        if (l[a] > 0) {
            int jn = j - c.st[a];
            Spinor<R> s;
            in.load(jn, s);
            if (g5in) gamma5(s);
            Half<R> hf, uh;
            project<R>(a, -1, s, hf);
            Link<R> u;
            lk.load(jn, a, u);
            mul_link_dag(u, hf, uh);
            accumulate<R>(a, -1, uh, (R)1, acc);
        }
    }
}

// acc = (H_b[lk1] - H_b[lk2]) in at local site j: only hops whose two links
// differ contribute (the proposal changes the active links only)
template <class SIn, class LK>
DD_DEV void dirichlet_hop_diff(const BlockCtx& c, int j, const SIn& in, const LK& lk1, const LK& lk2,
                               Spinor<double>& acc) {
    int l[4];
    local_coords(c, j, l);
    zero(acc);
    for (int a = 0; a < 4; ++a) {
        for (int dir = +1; dir >= -1; dir -= 2) {
            if (dir > 0 ? (l[a] >= c.bd[a] - 1) : (l[a] <= 0)) continue;
            const int jn = j + dir * c.st[a];
            const int jl = dir > 0 ? j : jn;  // the link sits at the lower end
            Link<double> u1, u2;
            lk1.load(jl, a, u1);
            lk2.load(jl, a, u2);
            bool same = true;
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    u1.m[r][s] = u1.m[r][s] - u2.m[r][s];
                    same = same && u1.m[r][s].x == 0.0 && u1.m[r][s].y == 0.0;
                }
            if (same) continue;
            Spinor<double> sp;
            in.load(jn, sp);
            Half<double> hf, uh;
            project<double>(a, dir, sp, hf);
            if (dir > 0)
                mul_link(u1, hf, uh);
            else
                mul_link_dag(u1, hf, uh);
            accumulate<double>(a, dir, uh, 1.0, acc);
        }
    }
}

// out = D_b in (dag: gamma5 D_b gamma5); returns this thread's |out|^2 (block-reduce it)
template <class R, class SIn, class SOut, class LK>
DD_DEV double dirichlet_apply(const BlockCtx& c, const SIn& in, const SOut& out, const LK& lk, int dag) {
    double n2 = 0.0;
    for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
        Spinor<R> acc, v;
        dirichlet_hop<R>(c, j, in, lk, dag, acc);
        in.load(j, v);
        if (dag) gamma5(v);
        const R mk_ = (R)(-c.kappa);
#pragma unroll
        for (int k = 0; k < 12; ++k) v.c[k] = v.c[k] + mk_ * acc.c[k];
        if (dag) gamma5(v);
        out.store(j, v);
        n2 += (double)snorm2(v);
    }
    return n2;
}

// Inner CG on the normal equations D_b^dag D_b x = D_b^dag r0 (x starts at 0,
// r holds r0 on entry).  Stops when |r|^2 <= tol2rel |r0|^2 or after maxit.
template <class R, class S, class LK>
DD_DEV int block_cgnr(const BlockCtx& c, const S& x, const S& r, const S& p, const S& q, const S& z, const LK& lk,
                      double tol2rel, int maxit, double* sh) {
    double rr0 = 0.0;
    for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
        Spinor<R> zz;
        zero(zz);
        x.store(j, zz);
        Spinor<R> v;
        r.load(j, v);
        rr0 += (double)snorm2(v);
    }
    rr0 = block_sum(rr0, sh);  // includes a barrier: r and x complete
    if (!(rr0 > 0.0)) return 0;
    double zz = block_sum(dirichlet_apply<R>(c, r, z, lk, 1), sh);
    for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
        Spinor<R> v;
        z.load(j, v);
        p.store(j, v);
    }
    __syncthreads();
    const double target = tol2rel * rr0;
    int it = 0;
    while (it < maxit) {
        double qq = block_sum(dirichlet_apply<R>(c, p, q, lk, 0), sh);
        if (!(qq > 0.0)) break;
        const R alpha = (R)(zz / qq);
        double rr = 0.0;
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<R> a, b;
            x.load(j, a);
            p.load(j, b);
#pragma unroll
            for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] + alpha * b.c[k];
            x.store(j, a);
            r.load(j, a);
            q.load(j, b);
#pragma unroll
            for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] - alpha * b.c[k];
            r.store(j, a);
            rr += (double)snorm2(a);
        }
        rr = block_sum(rr, sh);
        ++it;
        if (rr <= target) break;
        double zn = block_sum(dirichlet_apply<R>(c, r, z, lk, 1), sh);
        const R beta = (R)(zn / zz);
        zz = zn;
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<R> a, b;
            z.load(j, a);
            p.load(j, b);
#pragma unroll
            for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] + beta * b.c[k];
            p.store(j, a);
        }
        __syncthreads();
    }
    return it;
}

// N block-wide sums at once (two barriers for all of them); every thread
// gets the sums.  shn: at least 32 * N doubles of shared memory.
template <int N>
DD_DEV void block_sum_n(double* v, double* shn) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();  // earlier readers of shn are done
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) shn[wid * N + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += shn[w * N + k];
        v[k] = t;
    }
}

// Inner BiCGStab (van der Vorst) on D_b itself: x = 0, r holds r0 on entry;
// rhat = r0 is the shadow residual; block-local complex scalars.  Stops when
// |r|^2 <= tol2rel |r0|^2, after maxit iterations or at a breakdown (the
// FP64 refinement around it restarts from the true residual).
template <class R, class S, class LK>
DD_DEV int block_bicgstab(const BlockCtx& c, const S& x, const S& r, const S& rhat, const S& p, const S& v,
                          const S& s, const S& t, const LK& lk, double tol2rel, int maxit, double* sh) {
    double rr0 = 0.0;
    for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
        Spinor<R> z, a;
        zero(z);
        x.store(j, z);
        p.store(j, z);
        v.store(j, z);
        r.load(j, a);
        rhat.store(j, a);
        rr0 += (double)snorm2(a);
    }
    rr0 = block_sum(rr0, sh);  // barrier: x, p, v, rhat complete
    if (!(rr0 > 0.0)) return 0;
    __shared__ double shn[32 * 3];
    const double target = tol2rel * rr0;
    cpx<double> rho_old = mk<double>(1.0, 0.0), alpha = mk<double>(1.0, 0.0), omega = mk<double>(1.0, 0.0);
    int it = 0;
    while (it < maxit) {
        // rho = <rhat, r>
        double d0 = 0.0, d1 = 0.0;
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<R> a, b;
            rhat.load(j, a);
            r.load(j, b);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                d0 += (double)(a.c[k].x * b.c[k].x + a.c[k].y * b.c[k].y);
                d1 += (double)(a.c[k].x * b.c[k].y - a.c[k].y * b.c[k].x);
            }
        }
        double red[3] = {d0, d1, 0.0};
        block_sum_n<2>(red, shn);
        const cpx<double> rho = mk<double>(red[0], red[1]);
        if (!(norm2(rho) > 0.0)) break;
        const double den = norm2(rho_old) * norm2(omega);
        if (!(den > 0.0)) break;
        // beta = (rho / rho_old) (alpha / omega)
        const cpx<double> beta = (1.0 / den) * cmul(cmul(rho, conj(rho_old)), cmul(alpha, conj(omega)));
        const cpx<R> bR = mk<R>((R)beta.x, (R)beta.y), oR = mk<R>((R)omega.x, (R)omega.y);
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<R> pp, rr, vv;
            p.load(j, pp);
            r.load(j, rr);
            v.load(j, vv);
#pragma unroll
            for (int k = 0; k < 12; ++k) pp.c[k] = rr.c[k] + cmul(bR, pp.c[k] - cmul(oR, vv.c[k]));
            p.store(j, pp);
        }
        __syncthreads();
        dirichlet_apply<R>(c, p, v, lk, 0);
        __syncthreads();
        d0 = d1 = 0.0;
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<R> a, b;
            rhat.load(j, a);
            v.load(j, b);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                d0 += (double)(a.c[k].x * b.c[k].x + a.c[k].y * b.c[k].y);
                d1 += (double)(a.c[k].x * b.c[k].y - a.c[k].y * b.c[k].x);
            }
        }
        red[0] = d0;
        red[1] = d1;
        block_sum_n<2>(red, shn);
        const cpx<double> rv = mk<double>(red[0], red[1]);
        if (!(norm2(rv) > 0.0)) break;
        alpha = (1.0 / norm2(rv)) * cmul(rho, conj(rv));
        const cpx<R> aR = mk<R>((R)alpha.x, (R)alpha.y);
        double ss = 0.0;
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<R> rr, vv;
            r.load(j, rr);
            v.load(j, vv);
#pragma unroll
            for (int k = 0; k < 12; ++k) rr.c[k] = rr.c[k] - cmul(aR, vv.c[k]);
            s.store(j, rr);
            ss += (double)snorm2(rr);
        }
        ss = block_sum(ss, sh);  // barrier: s complete
        ++it;
        if (ss <= target) {
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<R> xx, pp;
                x.load(j, xx);
                p.load(j, pp);
#pragma unroll
                for (int k = 0; k < 12; ++k) xx.c[k] = xx.c[k] + cmul(aR, pp.c[k]);
                x.store(j, xx);
            }
            __syncthreads();
            break;
        }
        dirichlet_apply<R>(c, s, t, lk, 0);
        __syncthreads();
        double ts0 = 0.0, ts1 = 0.0, tt = 0.0;
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<R> a, b;
            t.load(j, a);
            s.load(j, b);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                ts0 += (double)(a.c[k].x * b.c[k].x + a.c[k].y * b.c[k].y);
                ts1 += (double)(a.c[k].x * b.c[k].y - a.c[k].y * b.c[k].x);
            }
            tt += (double)snorm2(a);
        }
        red[0] = ts0;
        red[1] = ts1;
        red[2] = tt;
        block_sum_n<3>(red, shn);
        const cpx<double> ts = mk<double>(red[0], red[1]);
        tt = red[2];
        if (!(tt > 0.0)) break;
        omega = (1.0 / tt) * ts;
        const cpx<R> wR = mk<R>((R)omega.x, (R)omega.y);
        double rr = 0.0;
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<R> xx, pp, sv, tv;
            x.load(j, xx);
            p.load(j, pp);
            s.load(j, sv);
            t.load(j, tv);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                xx.c[k] = xx.c[k] + cmul(aR, pp.c[k]) + cmul(wR, sv.c[k]);
                sv.c[k] = sv.c[k] - cmul(wR, tv.c[k]);
            }
            x.store(j, xx);
            r.store(j, sv);
            rr += (double)snorm2(sv);
        }
        rr = block_sum(rr, sh);  // barrier: x and r complete
        rho_old = rho;
        if (rr <= target || !(norm2(omega) > 0.0)) break;
    }
    return it;
}

// ----------------------------------------------------------- the launch
enum BlockMode { BLOCK_FILTER = 0, BLOCK_SOLVE = 1 };

struct BlockItem {
    int block_pos;  // position of the block in block order
    int f_src;      // field slot of the source operator (filter) / unused
    int f_sol;      // field slot of the solve
    int vec;        // factor index (noise sub) / vector index in the banks
    int lat;        // lattice of the item in a multi-lattice launch (0 otherwise)
};

// one lattice of a multi-lattice launch (blocks of different shapes)
struct LatDesc {
    Geo g;
    BlockCtx c;
    const double2* dd64;
    long long dd64_fs;
    const float4* dd32;
    long long dd32_fs;
    double* item_out;
};

struct BlockArgs {
    const LatDesc* lats;  // multi-lattice launch: per-item lattice (null: the fields below)
    Geo g;
    BlockCtx c;
    int mode;
    const BlockItem* items;  // null: block-filter items k -> (block position item_pos0 + k / item_n, vector k % item_n)
    int nitems;
    int item_pos0, item_n;
    int* queue;
    const double2* dd64;  // field slot 0, FP64 links in block order
    long long dd64_fs;    // elements between consecutive field slots
    const float4* dd32;
    long long dd32_fs;
    const double2* in_bank;  // BLOCK_SOLVE right-hand sides (block order, FP64)
    double2* out_bank;       // BLOCK_SOLVE solutions
    long long bank_vs;       // elements between consecutive vectors of a bank
    double* item_out;        // BLOCK_FILTER: -(2 Re<eta, d> + |d|^2) per item
    char* scratch;
    long long slot_bytes;
    uint64_t seed, ctr;
    const unsigned long long* ctr_off;  // added to ctr (graph replays; may be null)
    int purpose;
    double tol2;       // relative target of the FP64 residual (squared)
    double tol2_inner; // relative target of one inner solve (squared)
    int maxit_inner;
    int max_outer;
    int inner_f64;
    int* status;
    unsigned long long* stats;  // items, inner iterations, outer cycles, site-iterations (may be null)
};

// block id of the block at position pos of the block order
DD_DEV int block_id_at(const Geo& g, int pos, int* colour) {
    int half = g.nblocks / 2;
    int col = pos >= half ? 1 : 0;
    int rank = pos - col * half;
    int id = 2 * rank;
    int B1 = (id / g.nbk[0]) % g.nbk[1], B2 = (id / (g.nbk[0] * g.nbk[1])) % g.nbk[2],
        B3 = id / (g.nbk[0] * g.nbk[1] * g.nbk[2]);
    if (((B1 + B2 + B3) & 1) != col) id += 1;
    *colour = col;
    return id;
}
DD_DEV void block_origin(const Geo& g, int id, int o[4]) {
    o[0] = (id % g.nbk[0]) * g.b[0];
    int r = id / g.nbk[0];
    o[1] = (r % g.nbk[1]) * g.b[1];
    r /= g.nbk[1];
    o[2] = (r % g.nbk[2]) * g.b[2];
    o[3] = (r / g.nbk[2]) * g.b[3];
}

template <class LK>
DD_DEV LK make_inner_links(const LatDesc& L, int f, int pos);
template <>
DD_DEV LinkF32 make_inner_links<LinkF32>(const LatDesc& L, int f, int pos) {
    return LinkF32{L.dd32 + (long long)f * L.dd32_fs + (long long)pos * 4 * 3 * L.c.nb, L.c.nb};
}
template <>
DD_DEV LinkF64 make_inner_links<LinkF64>(const LatDesc& L, int f, int pos) {
    return LinkF64{L.dd64 + (long long)f * L.dd64_fs + (long long)pos * 4 * 9 * L.c.nb, L.c.nb};
}
template <class S>
DD_DEV S scratch_spinor(char* base, int index, long long nb);
template <>
DD_DEV SpinorF32 scratch_spinor<SpinorF32>(char* base, int index, long long nb) {
    return SpinorF32{(float4*)base + (long long)index * 6 * nb, nb};
}
template <>
DD_DEV SpinorF64 scratch_spinor<SpinorF64>(char* base, int index, long long nb) {
    return SpinorF64{(double2*)base + (long long)index * 12 * nb, nb};
}

template <class RI, class SI, class LKI>
__global__ void __launch_bounds__(256, 2) block_solve_kernel(BlockArgs A) {
    __shared__ double sh[34];
    __shared__ int s_item;
    // scratch slot of this thread block: FP64 vectors eta, b, x, r; inner vectors x, r, p, q, z
    char* base = A.scratch + (long long)blockIdx.x * A.slot_bytes;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(A.queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= A.nitems) break;
        const BlockItem it = A.items ? A.items[item]
                                     : BlockItem{A.item_pos0 + item / A.item_n, item % A.item_n,
                                                 item % A.item_n + 1, item % A.item_n, 0};
        LatDesc L;
        if (A.lats) {
            L = A.lats[it.lat];
        } else {
            L.g = A.g;
            L.c = A.c;
            L.dd64 = A.dd64;
            L.dd64_fs = A.dd64_fs;
            L.dd32 = A.dd32;
            L.dd32_fs = A.dd32_fs;
            L.item_out = A.item_out;
        }
        const BlockCtx& c = L.c;
        const long long nb = c.nb;
        SpinorF64 eta{(double2*)base, nb};
        SpinorF64 bv{(double2*)base + 12 * nb, nb};
        SpinorF64 xv{(double2*)base + 24 * nb, nb};
        SpinorF64 rv{(double2*)base + 36 * nb, nb};
        char* ib = base + 48 * nb * sizeof(double2);
        SI xi = scratch_spinor<SI>(ib, 0, nb), ri = scratch_spinor<SI>(ib, 1, nb),
           pi = scratch_spinor<SI>(ib, 2, nb), qi = scratch_spinor<SI>(ib, 3, nb), zi = scratch_spinor<SI>(ib, 4, nb);
        LinkF64 lsol{L.dd64 + (long long)it.f_sol * L.dd64_fs + (long long)it.block_pos * 4 * 9 * nb, nb};
        LKI lsoli = make_inner_links<LKI>(L, it.f_sol, it.block_pos);
        int colour;
        int id = block_id_at(L.g, it.block_pos, &colour);
        int org[4];
        block_origin(L.g, id, org);
        // ---- right-hand side
        if (A.mode == BLOCK_FILTER) {
            LinkF64 lsrc{L.dd64 + (long long)it.f_src * L.dd64_fs + (long long)it.block_pos * 4 * 9 * nb, nb};
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                int l[4];
                local_coords(c, j, l);
                int x[4] = {org[0] + l[0], org[1] + l[1], org[2] + l[2], org[3] + l[3]};
                uint32_t s = (uint32_t)canon_index(L.g, x);
                Spinor<double> e;
#pragma unroll
                for (int k = 0; k < 12; ++k)
                    e.c[k] = gaussian(s * 12u + k, (uint32_t)A.purpose, (uint32_t)it.vec, A.seed, stream_ctr(A.ctr, A.ctr_off));
                eta.store(j, e);
            }
            __syncthreads();
            // b = (D_b[src] - D_b[sol]) eta = -kappa (H[src] - H[sol]) eta
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<double> h1;
                dirichlet_hop_diff(c, j, eta, lsrc, lsol, h1);
#pragma unroll
                for (int k = 0; k < 12; ++k) h1.c[k] = (-c.kappa) * h1.c[k];
                bv.store(j, h1);
            }
        } else {
            SpinorF64 src{(double2*)A.in_bank + (long long)it.vec * A.bank_vs + (long long)it.block_pos * 12 * nb, nb};
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<double> v;
                src.load(j, v);
                bv.store(j, v);
            }
        }
        // ---- x = 0, r = b
        double bb = 0.0;
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<double> v, z;
            bv.load(j, v);
            rv.store(j, v);
            zero(z);
            xv.store(j, z);
            bb += snorm2(v);
        }
        bb = block_sum(bb, sh);
        double rr = bb;
        int outer = 0;
        long long inner_its = 0;
        while (rr > A.tol2 * bb && outer < A.max_outer) {
            // inner right-hand side: the FP64 residual, normalised to unit norm
            const double rn = sqrt(rr), rinv = 1.0 / rn;
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<double> v;
                rv.load(j, v);
#pragma unroll
                for (int k = 0; k < 12; ++k) v.c[k] = rinv * v.c[k];
                ri.store(j, v);
            }
            __syncthreads();
            if constexpr (std::is_same<RI, float>::value) {
                // FP32 inner vectors are half the size of the slot's FP64 ones:
                // room for the seven BiCGStab vectors
                SI hi = scratch_spinor<SI>(ib, 5, nb), si = scratch_spinor<SI>(ib, 6, nb),
                   ti = scratch_spinor<SI>(ib, 7, nb);
                inner_its += block_bicgstab<RI>(c, xi, ri, hi, pi, qi, si, ti, lsoli, A.tol2_inner, A.maxit_inner, sh);
            } else {
                inner_its += block_cgnr<RI>(c, xi, ri, pi, qi, zi, lsoli, A.tol2_inner, A.maxit_inner, sh);
            }
            // x += |r| e; r = b - D_b x (FP64)
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<double> a;
                Spinor<RI> e;
                xv.load(j, a);
                xi.load(j, e);
#pragma unroll
                for (int k = 0; k < 12; ++k)
                    a.c[k] = a.c[k] + rn * mk<double>((double)e.c[k].x, (double)e.c[k].y);
                xv.store(j, a);
            }
            __syncthreads();
            rr = 0.0;
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<double> acc, v, b;
                dirichlet_hop<double>(c, j, xv, lsol, 0, acc);
                xv.load(j, v);
                bv.load(j, b);
#pragma unroll
                for (int k = 0; k < 12; ++k) b.c[k] = b.c[k] - (v.c[k] + (-c.kappa) * acc.c[k]);
                rv.store(j, b);
                rr += snorm2(b);
            }
            rr = block_sum(rr, sh);
            ++outer;
        }
        if (rr > A.tol2 * bb && threadIdx.x == 0) raise_status(A.status, DD_ERR_NOT_CONVERGED);
        if (A.stats && threadIdx.x == 0) {
            atomicAdd(A.stats, 1ull);
            atomicAdd(A.stats + 1, (unsigned long long)inner_its);
            atomicAdd(A.stats + 2, (unsigned long long)outer);
            atomicAdd(A.stats + 3, (unsigned long long)inner_its * (unsigned long long)nb);
        }
        if (!isfinite(rr) && threadIdx.x == 0) raise_status(A.status, DD_ERR_NUMERIC);
        // ---- results
        if (A.mode == BLOCK_FILTER) {
            double s = 0.0;
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<double> e, d;
                eta.load(j, e);
                xv.load(j, d);
#pragma unroll
                for (int k = 0; k < 12; ++k) s += 2.0 * (e.c[k].x * d.c[k].x + e.c[k].y * d.c[k].y) + norm2(d.c[k]);
            }
            s = block_sum(s, sh);
            if (threadIdx.x == 0) L.item_out[item] = -s;
        } else {
            SpinorF64 dst{A.out_bank + (long long)it.vec * A.bank_vs + (long long)it.block_pos * 12 * nb, nb};
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<double> v;
                xv.load(j, v);
                dst.store(j, v);
            }
        }
        __syncthreads();
    }
}
