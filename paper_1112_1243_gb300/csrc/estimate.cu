// Stochastic determinant-ratio estimates and acceptance steps.
//
// Global step (Eq. 4step step 3, Sec. 4): with M_i = Dhat[U_{i+1}]^{-1}
// Dhat[U_i] and a fresh complex Gaussian eta_i on the black sites per factor
// (Eq. param), ln r_i = -eta^dag (M^dag M - 1) eta = -(2 Re<eta, d> + |d|^2),
// d = (M - 1) eta.  Using Dhat'^{-1} = (D'^{-1})_bb A' (block inverse of
// Eq. domdec) and A'(Dhat - Dhat') = B'E'^{-1}C' - A'A^{-1}BE^{-1}C:
//   w = C eta, w' = C' eta            (inter-block hops, black -> white)
//   z = E^{-1} w, z' = E'^{-1} w'     (white Dirichlet block solves)
//   v = B z, v' = B' z'               (inter-block hops, white -> black)
//   a = A^{-1} v                      (black Dirichlet block solves)
//   s = v' - A' a                     (black Dirichlet apply)
//   y = D'^{-1} (s, 0),  d = y_black  (global solve)
// All factors are processed as one batch: one launch per stage.
//
// Block filter (Eq. 4step step 1; Sec. 5): per block and factor
//   d = D_b[U_{i+1}]^{-1} (D_b[U_i] - D_b[U_{i+1}]) eta_{b,i},
//   ln r_b = sum_i -(2 Re<eta, d> + |d|^2), accept iff ln u_b < ln r_b.
#include <algorithm>
#include <cmath>
#include <vector>

#include "blocksolve.cuh"
#include "dslash.cuh"
#include "solver.h"

int launch_interpolate(dd_handle* h, const double* U, const double* Up, double* out, int num, int den,
                       bool all_links);
int launch_interpolate_slots(dd_handle* h, const double* U, const double* Up, double* out, long long slot_stride,
                             int nslots, int den, bool all_links);

namespace {

// canonical coordinates of block-order position q
DD_DEV void dd_coords(const Geo& g, const BlockCtx& c, long long q, int x[4], int* colour) {
    int pos = (int)(q / c.nb), j = (int)(q % c.nb);
    int id = block_id_at(g, pos, colour);
    int o[4], l[4];
    block_origin(g, id, o);
    local_coords(c, j, l);
    for (int a = 0; a < 4; ++a) x[a] = o[a] + l[a];
}

// extents of the enclosing blocks of a two-level decomposition (x = 0: none)
DD_DEV bool same_outer_block(int4 ob, const int x[4], const int y[4]) {
    return ob.x == 0 || (x[0] / ob.x == y[0] / ob.x && x[1] / ob.y == y[1] / ob.y && x[2] / ob.z == y[2] / ob.z &&
                         x[3] / ob.w == y[3] / ob.w);
}
DD_DEV int outer_colour(int4 ob, const int x[4]) { return (x[0] / ob.x + x[1] / ob.y + x[2] / ob.z + x[3] / ob.w) & 1; }

// eta on the black sites (purpose / sub), 0 on white; block order.  With
// enclosing blocks (ob.x > 0) only inside the enclosing blocks whose colour
// is in outer_mask.
__global__ void noise_black_kernel(Geo g, BlockCtx c, double2* bank, long long vs, int purpose, uint64_t seed,
                                   uint64_t ctr0, const unsigned long long* ctr_off, int4 ob, int outer_mask) {
    const uint64_t ctr = stream_ctr(ctr0, ctr_off);
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (q >= g.V) return;
    int x[4], col;
    dd_coords(g, c, q, x, &col);
    long long pos = q / c.nb, j = q % c.nb;
    SpinorF64 out{bank + (long long)i * vs + pos * 12 * c.nb, c.nb};
    Spinor<double> e;
    uint32_t s = (uint32_t)canon_index(g, x);
    if (col == 0 && (ob.x == 0 || ((outer_mask >> outer_colour(ob, x)) & 1))) {
        for (int k = 0; k < 12; ++k) e.c[k] = gaussian(s * 12u + k, (uint32_t)purpose, (uint32_t)i, seed, ctr);
    } else {
        zero(e);
    }
    out.store(j, e);
}

// out = -kappa * (hops that cross block faces) in, on the sites of colour
// `target` (0 elsewhere).  Links from the canonical FP64 copy of the field
// of slot f0 + i * fstep for right-hand side i.  With enclosing blocks
// (ob.x > 0), hops that leave the enclosing block are dropped as well.
__global__ void inter_hop_kernel(Geo g, BlockCtx c, const double2* in_bank, double2* out_bank, long long vs,
                                 const double* canon0, long long canon_fs, int f0, int fstep, int target,
                                 int4 ob) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (q >= g.V) return;
    const double* U = canon0 + (long long)(f0 + i * fstep) * canon_fs;
    int x[4], col;
    dd_coords(g, c, q, x, &col);
    long long pos = q / c.nb, j = q % c.nb;
    Spinor<double> acc;
    zero(acc);
    if (col == target) {
        const int s = canon_index(g, x);
        for (int a = 0; a < 4; ++a) {
            // a hop crosses a block face iff x sits on that face (two or more blocks per direction)
            const int loc = x[a] % g.b[a];
            for (int dir = +1; dir >= -1; dir -= 2) {
                if (dir > 0 ? loc != g.b[a] - 1 : loc != 0) continue;
                int y[4] = {x[0], x[1], x[2], x[3]};
                y[a] += dir;
                if (y[a] == g.L[a]) y[a] = 0;
                if (y[a] < 0) y[a] = g.L[a] - 1;
                if (!same_outer_block(ob, x, y)) continue;
                long long qy = dd_position(g, y);
                SpinorF64 src{(double2*)in_bank + (long long)i * vs + (qy / c.nb) * 12 * c.nb, c.nb};
                Spinor<double> sp;
                src.load(qy % c.nb, sp);
                Half<double> hf, uh;
                project<double>(a, dir, sp, hf);
                Link<double> u;
                const int ys = canon_index(g, y);
                const double* lp = U + ((long long)(dir > 0 ? s : ys) * 4 + a) * 18;
                for (int k = 0; k < 9; ++k) u.m[k / 3][k % 3] = mk<double>(lp[2 * k], lp[2 * k + 1]);
                if (dir > 0)
                    mul_link(u, hf, uh);
                else
                    mul_link_dag(u, hf, uh);
                double sc = 1.0;
                if (a == 3 && ((dir > 0 && x[3] == g.L[3] - 1) || (dir < 0 && x[3] == 0))) sc = g.bc;
                accumulate<double>(a, dir, uh, sc, acc);
            }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) acc.c[k] = (-c.kappa) * acc.c[k];
    }
    SpinorF64 dst{out_bank + (long long)i * vs + pos * 12 * c.nb, c.nb};
    dst.store(j, acc);
}

// out = v - D_b[field] a on black sites, 0 on white (block order)
__global__ void schur_source_kernel(Geo g, BlockCtx c, const double2* v_bank, const double2* a_bank,
                                    double2* out_bank, long long vs, const double2* dd64, long long fs, int f0,
                                    int fstep) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (q >= g.V) return;
    long long pos = q / c.nb;
    int j = (int)(q % c.nb);
    SpinorF64 dst{out_bank + (long long)i * vs + pos * 12 * c.nb, c.nb};
    Spinor<double> r;
    if (pos < g.nblocks / 2) {
        SpinorF64 av{(double2*)a_bank + (long long)i * vs + pos * 12 * c.nb, c.nb};
        SpinorF64 vv{(double2*)v_bank + (long long)i * vs + pos * 12 * c.nb, c.nb};
        LinkF64 lk{dd64 + (long long)(f0 + i * fstep) * fs + pos * 4 * 9 * c.nb, c.nb};
        Spinor<double> acc, a;
        dirichlet_hop<double>(c, j, av, lk, 0, acc);
        av.load(j, a);
        vv.load(j, r);
#pragma unroll
        for (int k = 0; k < 12; ++k) r.c[k] = r.c[k] - (a.c[k] + (-c.kappa) * acc.c[k]);
    } else {
        zero(r);
    }
    dst.store(j, r);
}

// block order (FP64) -> eo FP64 chunks of the global solver
__global__ void dd_to_eo_kernel(Geo g, BlockCtx c, const double2* bank, long long vs, double2* be, double2* bo) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (s >= g.V) return;
    int x[4];
    canon_coords(g, s, x);
    long long q = dd_position(g, x);
    SpinorF64 src{(double2*)bank + (long long)i * vs + (q / c.nb) * 12 * c.nb, c.nb};
    Spinor<double> v;
    src.load(q % c.nb, v);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    SpinorF64 dst{(par ? bo : be) + (long long)i * 12 * g.Vh, g.Vh};
    dst.store(s >> 1, v);
}

// ln_i = -sum_black (2 Re<eta, d> + |d|^2), d from the eo solution
__global__ void __launch_bounds__(128) estimate_kernel(Geo g, BlockCtx c, const double2* eta_bank, long long vs,
                                                       const double2* xe, const double2* xo, Reduce red) {
    __shared__ double sh[34];
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    double acc = 0.0;
    if (q < g.V / 2) {  // black sites come first in block order
        int x[4], col;
        dd_coords(g, c, q, x, &col);
        SpinorF64 es{(double2*)eta_bank + (long long)i * vs + (q / c.nb) * 12 * c.nb, c.nb};
        Spinor<double> e, d;
        es.load(q % c.nb, e);
        const int s = canon_index(g, x);
        const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
        SpinorF64 ds{(double2*)(par ? xo : xe) + (long long)i * 12 * g.Vh, g.Vh};
        ds.load(s >> 1, d);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc += 2.0 * (e.c[k].x * d.c[k].x + e.c[k].y * d.c[k].y) + norm2(d.c[k]);
        acc = -acc;
    }
    grid_reduce(red, i, acc, sh);
}

// ln_b[b] = sum of the n item results of block b (0 for blocks without
// items).  item_base: the first item of every block, or null for the
// block-filter order (the blocks of colour_mask in block order from
// position pos0, n consecutive items each)
__global__ void sum_items_kernel(Geo g, const int* item_base, int colour_mask, int pos0, int n,
                                 const double* item_out, double* ln_b) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= g.nblocks) return;
    int base;
    if (item_base) {
        base = item_base[b];
    } else {
        int B[4] = {b % g.nbk[0], (b / g.nbk[0]) % g.nbk[1], (b / (g.nbk[0] * g.nbk[1])) % g.nbk[2],
                    b / (g.nbk[0] * g.nbk[1] * g.nbk[2])};
        int col = (B[0] + B[1] + B[2] + B[3]) & 1;
        base = ((colour_mask >> col) & 1) ? (block_pos_of(g, b, col) - pos0) * n : -1;
    }
    double s = 0.0;
    if (base >= 0)
        for (int i = 0; i < n; ++i) s += item_out[base + i];
    ln_b[b] = s;
}

__global__ void block_accept_kernel(Geo g, int colour_mask, const double* ln_b, uint8_t* accept, uint64_t seed,
                                    uint64_t ctr, const unsigned long long* ctr_off,
                                    int purpose = DD_PURPOSE_BLOCK_ACCEPT) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= g.nblocks) return;
    int B[4] = {b % g.nbk[0], (b / g.nbk[0]) % g.nbk[1], (b / (g.nbk[0] * g.nbk[1])) % g.nbk[2],
                b / (g.nbk[0] * g.nbk[1] * g.nbk[2])};
    int col = (B[0] + B[1] + B[2] + B[3]) & 1;
    if (!((colour_mask >> col) & 1)) {
        accept[b] = 1;
        return;
    }
    double u1, u2;
    uniform_pair((uint32_t)b, (uint32_t)purpose, 0u, seed, stream_ctr(ctr, ctr_off), u1, u2);
    accept[b] = log(u1) < ln_b[b] ? 1 : 0;
}

__global__ void restore_kernel(Geo g, int n, const int* links, const uint8_t* accept, const double* U_old,
                               double* U_new) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int l = links[k];
    int s = l >> 2;
    int x[4];
    canon_coords(g, s, x);
    if (accept[block_id_of(g, x)]) return;
    for (int e = 0; e < 18; ++e) U_new[(long long)l * 18 + e] = U_old[(long long)l * 18 + e];
}

__global__ void global_accept_kernel(const double* ln_r, int n, uint64_t seed, uint64_t ctr,
                                     const unsigned long long* ctr_off, uint8_t* accept, double* margin) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += ln_r[i];
    double u1, u2;
    uniform_pair(0u, DD_PURPOSE_GLOBAL_ACCEPT, 0u, seed, stream_ctr(ctr, ctr_off), u1, u2);
    double lu = log(u1);
    accept[0] = lu < s ? 1 : 0;
    if (margin) margin[0] = s - lu;
}

__global__ void conditional_copy_kernel(long long n, const uint8_t* accept, const double* src, double* dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || accept[0]) return;
    dst[i] = src[i];
}

}  // namespace

// ----------------------------------------------------------------- helpers
static BlockCtx block_ctx(dd_handle* h) {
    BlockCtx c;
    for (int a = 0; a < 4; ++a) c.bd[a] = h->g.b[a];
    c.st[0] = 1;
    c.st[1] = c.bd[0];
    c.st[2] = c.bd[0] * c.bd[1];
    c.st[3] = c.bd[0] * c.bd[1] * c.bd[2];
    c.nb = h->g.bsites;
    c.kappa = h->prm.kappa;
    return c;
}

// format slots 0..nslots-1 from interpolated (or copied) fields
static int prepare_fields(dd_handle* h, const double* U_old, const double* U_new, int n, bool factors, bool eo,
                          bool all_links = false) {
    const int nslots = factors ? n + 1 : 2;
    const int ip = h->prm.inner_prec;
    // all slots of the chain in one launch (slots are equally spaced in the workspace)
    const long long slot_stride = (long long)(h->fields[1].canon - h->fields[0].canon) * 2;
    int rc = launch_interpolate_slots(h, U_old, U_new, (double*)h->fields[0].canon, slot_stride, nslots,
                                      factors ? n : 1, all_links);
    if (rc) return rc;
    for (int k = 0; k < nslots; ++k) {
        FieldSlot& f = h->fields[k];
        bool need_eo = eo;  // old and new fields both enter even-odd solves
        rc = format_field(h, (const double*)f.canon, f, need_eo, need_eo && ip == DD_PREC_F32,
                          need_eo && ip == DD_PREC_F16, true, true);
        if (rc) return rc;
    }
    return DD_OK;
}

// CUDA-event timing of a persistent block-solver launch (timer kind 7; the
// item count is added to the kind's site counter)
__global__ void add_count_kernel(unsigned long long* p, unsigned long long v) { *p += v; }
static bool block_timer_begin(dd_handle* h) {
    const int kind = 7;
    if (!h->timer_on || h->capturing || dd_stream_capturing(h)) return false;
    if ((h->timer_seen[kind]++ % h->timer_every) != 0) return false;
    cudaEvent_t e = dd_timer_event(h, kind);
    if (e) cudaEventRecord(e, h->stream);
    return true;
}
static void block_timer_end(dd_handle* h, int nitems) {
    static_assert(DD_TIMER_KINDS > 7, "timer kind 7 is the persistent block solver");
    cudaEvent_t e = dd_timer_event(h, 7);
    if (e) cudaEventRecord(e, h->stream);
    add_count_kernel<<<1, 1, 0, h->stream>>>(h->d_sites + 7, (unsigned long long)nitems);
}

// block-filter items of the blocks at positions pos0 .. pos0 + nitems / n - 1,
// n noise vectors each, in one persistent launch
static int launch_blocks(dd_handle* h, int mode, int pos0, int n, int nitems, const double2* in_bank,
                         double2* out_bank, uint64_t seed, uint64_t ctr) {
    if (nitems <= 0) return DD_OK;
    DD_CUDA(h, cudaMemsetAsync(h->d_queue, 0, sizeof(int), h->stream));
    BlockArgs A;
    A.lats = nullptr;
    A.g = h->g;
    A.c = block_ctx(h);
    A.mode = mode;
    A.items = nullptr;
    A.nitems = nitems;
    A.item_pos0 = pos0;
    A.item_n = n;
    A.queue = h->d_queue;
    A.dd64 = h->fields[0].dd64;
    A.dd64_fs = (long long)(h->fields[1].dd64 - h->fields[0].dd64);
    A.dd32 = h->fields[0].dd32;
    A.dd32_fs = (long long)(h->fields[1].dd32 - h->fields[0].dd32);
    A.in_bank = in_bank;
    A.out_bank = out_bank;
    A.bank_vs = 12LL * h->g.V;
    A.item_out = h->d_item_out;
    A.scratch = h->block_scratch;
    A.slot_bytes = (long long)h->block_slot_bytes;
    A.seed = seed;
    A.ctr = ctr;
    A.ctr_off = h->d_ctr_off;
    A.purpose = DD_PURPOSE_BLOCK_NOISE;
    A.tol2 = h->prm.tol_block * h->prm.tol_block;
    A.inner_f64 = h->prm.block_prec == DD_PREC_F64;
    A.tol2_inner = A.inner_f64 ? 0.25 * A.tol2 : 1e-10;
    A.maxit_inner = std::min(h->prm.maxit, 2000);
    A.max_outer = A.inner_f64 ? 3 : 12;
    A.status = h->d_status;
    A.stats = h->d_sites + DD_TIMER_KINDS;
    const int grid = std::min(nitems, std::min(h->block_slots, std::max(1, h->num_sms) * h->tune.block_ctas_per_sm));
    const int tpb = h->tune.block_tpb;
    const bool timed = block_timer_begin(h);
    ++h->block_launches;
    if (A.inner_f64)
        DD_KLAUNCH(h, block_solve_kernel<double, SpinorF64, LinkF64><<<grid, tpb, 0, h->stream>>>(A));
    else
        DD_KLAUNCH(h, block_solve_kernel<float, SpinorF32, LinkF32><<<grid, tpb, 0, h->stream>>>(A));
    if (timed) block_timer_end(h, nitems);
    DD_LAUNCH_CHECK(h, "block_solve_kernel");
    return DD_OK;
}

// autotuner probe: one block-filter pass (one noise vector per block, every
// block) on the fields of (U_old, U_new) with the handle's current launch
// shape; *ms = average duration of the persistent launch over reps
int tune_block_filter(dd_handle* h, const double* U_old, const double* U_new, int reps, float* ms) {
    int rc = prepare_fields(h, U_old, U_new, 1, true, false);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    DD_CUDA(h, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return dd_fail(h, DD_ERR_CUDA, "cudaEventCreate");
    }
    rc = launch_blocks(h, BLOCK_FILTER, 0, 1, h->g.nblocks, nullptr, nullptr, 1, 0);
    cudaEventRecord(e0, h->stream);
    for (int r = 0; r < reps && !rc; ++r) rc = launch_blocks(h, BLOCK_FILTER, 0, 1, h->g.nblocks, nullptr, nullptr, 1, 0);
    cudaEventRecord(e1, h->stream);
    float t = -1.f;
    if (!rc && cudaEventSynchronize(e1) == cudaSuccess) {
        cudaEventElapsedTime(&t, e0, e1);
        t /= (float)reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (t < 0) return dd_fail(h, DD_ERR_CUDA, "block-filter timing failed");
    *ms = t;
    return DD_OK;
}

__global__ void set_status_kernel(int* status, int code) { raise_status(status, code); }
static void raise_status_host(dd_handle* h, int code) {
    DD_KLAUNCH(h, set_status_kernel<<<1, 1, 0, h->stream>>>(h->d_status, code));
}

// eo FP64 chunks of the global solver -> block order (FP64); sites of
// blocks whose colour is not in colour_mask are written as zero
__global__ void eo_to_dd_kernel(Geo g, BlockCtx c, const double2* xe, const double2* xo, double2* bank,
                                long long vs, int colour_mask) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (s >= g.V) return;
    int x[4];
    canon_coords(g, s, x);
    long long q = dd_position(g, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    SpinorF64 src{(double2*)(par ? xo : xe) + (long long)i * 12 * g.Vh, g.Vh};
    Spinor<double> v;
    if ((colour_mask >> block_colour_of(g, x)) & 1)
        src.load(s >> 1, v);
    else
        zero(v);
    SpinorF64 dst{bank + (long long)i * vs + (q / c.nb) * 12 * c.nb, c.nb};
    dst.store(q % c.nb, v);
}

// out_bank[i] = (D_bb + D_ww)^{-1} in_bank[i] for i < n, with the gauge field
// of slot field0 + i * step: every Dirichlet block solve of every factor in
// one batched even-odd Krylov solve (inner precision of the handle, FP64
// defect correction to tol_block relative to the whole right-hand side).
// The right-hand sides live on the blocks of one colour (0 black, 1 white);
// only that colour's sites are visited, the other colour of out_bank is 0.
static int dirichlet_solve_bank(dd_handle* h, const double2* in_bank, double2* out_bank, int n, int field0,
                                int step, int colour) {
    const Geo& g = h->g;
    const BlockCtx c = block_ctx(h);
    const long long vs = 12LL * g.V;
    SolverVecs& v = h->vecs[0];
    dim3 gv(grid_for(g.V, 128), n);
    DD_KLAUNCH(h, dd_to_eo_kernel<<<gv, 128, 0, h->stream>>>(g, c, in_bank, vs, v.be, v.bo));
    DD_LAUNCH_CHECK(h, "dd_to_eo_kernel");
    int it = 0;
    int rc = solve_packed(h, n, field0, step, h->prm.inner_prec, h->prm.tol_block, h->prm.maxit, &it, nullptr, 1,
                          colour);
    if (rc && rc != DD_ERR_NOT_CONVERGED) return dd_fail(h, rc, "Dirichlet block solves failed");
    if (rc == DD_ERR_NOT_CONVERGED) raise_status_host(h, DD_ERR_NOT_CONVERGED);
    DD_KLAUNCH(h, eo_to_dd_kernel<<<gv, 128, 0, h->stream>>>(g, c, v.xe, v.xo, out_bank, vs, 1 << colour));
    DD_LAUNCH_CHECK(h, "eo_to_dd_kernel");
    return DD_OK;
}

// ------------------------------------ block filter as whole-lattice solves
// The stochastic block filter computed with the batched Dirichlet solver
// instead of the persistent per-block kernel: every block's noise, source
// and solution live in whole-lattice even-odd vectors (the Dirichlet
// operator is block-diagonal, so the blocks do not mix), one right-hand side
// per factor.  eta_i(x) = block noise (purpose DD_PURPOSE_BLOCK_NOISE,
// element 12 s + k, sub i) on the blocks of colour_mask;
// b_i = (D_b[U_i] - D_b[U_{i+1}]) eta_i = -kappa (H_b[U_i] - H_b[U_{i+1}]) eta_i,
// where only the active links differ.

// Block-filter noise: eta on the sites of the blocks in colour_mask (0
// elsewhere), one Gaussian stream per factor i, stored in even-odd order.
__global__ void filter_noise_kernel(Geo g, int colour_mask, uint64_t seed, uint64_t ctr0,
                                    const unsigned long long* ctr_off, double2* eta_e, double2* eta_o) {
    const uint64_t ctr = stream_ctr(ctr0, ctr_off);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (s >= g.V) return;
    int x[4];
    canon_coords(g, s, x);
    Spinor<double> e;
    zero(e);
    if ((colour_mask >> block_colour_of(g, x)) & 1) {
#pragma unroll
        for (int k = 0; k < 12; ++k)
            e.c[k] = gaussian((uint32_t)s * 12u + k, DD_PURPOSE_BLOCK_NOISE, (uint32_t)i, seed, ctr);
    }
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    SpinorF64 eo{(par ? eta_o : eta_e) + (long long)i * 12 * g.Vh, g.Vh};
    eo.store(s >> 1, e);
}

// Block-filter source b = -kappa (D_b[U_i] - D_b[U_{i+1}]) eta restricted to
// the hops inside a block whose link differs (active links), from the noise
// stored by filter_noise_kernel (a neighbour inside the block has the same
// colour, so its noise is stored).
__global__ void filter_source_kernel(Geo g, int colour_mask, const double* canon0, long long canon_fs,
                                     const uint8_t* active, const double2* eta_e, const double2* eta_o, double2* be,
                                     double2* bo, double kappa) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (s >= g.V) return;
    int x[4];
    canon_coords(g, s, x);
    const bool in = (colour_mask >> block_colour_of(g, x)) & 1;
    Spinor<double> acc;
    zero(acc);
    if (in) {
        const double* U1 = canon0 + (long long)i * canon_fs;
        const double* U2 = canon0 + (long long)(i + 1) * canon_fs;
        const int bid = block_id_of(g, x);
        for (int a = 0; a < 4; ++a) {
            for (int dir = +1; dir >= -1; dir -= 2) {
                const int y = shift_index(g, x, a, dir);
                const int l = (dir > 0 ? s : y) * 4 + a;
                if (!active[l]) continue;
                int xy[4];
                canon_coords(g, y, xy);
                if (block_id_of(g, xy) != bid) continue;  // Dirichlet: hops stay in the block
                Link<double> u;
                bool same = true;
                for (int k = 0; k < 9; ++k) {
                    const double* p1 = U1 + (long long)l * 18 + 2 * k;
                    const double* p2 = U2 + (long long)l * 18 + 2 * k;
                    u.m[k / 3][k % 3] = mk<double>(p1[0] - p2[0], p1[1] - p2[1]);
                    same = same && p1[0] == p2[0] && p1[1] == p2[1];
                }
                if (same) continue;
                const int py = (xy[0] + xy[1] + xy[2] + xy[3]) & 1;
                const SpinorF64 ein{const_cast<double2*>(py ? eta_o : eta_e) + (long long)i * 12 * g.Vh, g.Vh};
                Spinor<double> ey;
                ein.load(y >> 1, ey);
                Half<double> hf, uh;
                project<double>(a, dir, ey, hf);
                if (dir > 0)
                    mul_link(u, hf, uh);
                else
                    mul_link_dag(u, hf, uh);
                accumulate<double>(a, dir, uh, 1.0, acc);
            }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) acc.c[k] = (-kappa) * acc.c[k];
    }
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    SpinorF64 bo_{(par ? bo : be) + (long long)i * 12 * g.Vh, g.Vh};
    bo_.store(s >> 1, acc);
}

__global__ void __launch_bounds__(256) filter_estimate_kernel(Geo g, int colour_mask, const double2* eta_e,
                                                              const double2* eta_o, const double2* xe,
                                                              const double2* xo, int n, double* ln_b) {
    __shared__ double sh[34];
    const int b = blockIdx.x;
    int o[4];
    block_origin(g, b, o);
    const int col = (o[0] / g.b[0] + o[1] / g.b[1] + o[2] / g.b[2] + o[3] / g.b[3]) & 1;
    if (!((colour_mask >> col) & 1)) {
        if (threadIdx.x == 0) ln_b[b] = 0.0;
        return;
    }
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int j = threadIdx.x; j < g.bsites; j += blockDim.x) {
            int x[4] = {o[0] + j % g.b[0], o[1] + (j / g.b[0]) % g.b[1], o[2] + (j / (g.b[0] * g.b[1])) % g.b[2],
                        o[3] + j / (g.b[0] * g.b[1] * g.b[2])};
            const int s = canon_index(g, x);
            const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
            SpinorF64 es{(double2*)(par ? eta_o : eta_e) + (long long)i * 12 * g.Vh, g.Vh};
            SpinorF64 ds{(double2*)(par ? xo : xe) + (long long)i * 12 * g.Vh, g.Vh};
            Spinor<double> e, d;
            es.load(s >> 1, e);
            ds.load(s >> 1, d);
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < 12; ++k) t += 2.0 * (e.c[k].x * d.c[k].x + e.c[k].y * d.c[k].y) + norm2(d.c[k]);
            acc -= t;
        }
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) ln_b[b] = acc;
}

// fields of slots 0..n are prepared (canonical and even-odd formats)
static int block_filter_masked(dd_handle* h, int colour_mask, int n, uint64_t seed, uint64_t ctr, double* ln_b) {
    const Geo& g = h->g;
    SolverVecs& v = h->vecs[0];
    const long long Vh = g.Vh;
    double2* eta_e = h->dd_vec;
    double2* eta_o = h->dd_vec + (long long)h->prm.max_rhs * 12 * Vh;
    const long long canon_fs = (long long)(h->fields[1].canon - h->fields[0].canon) * 2;
    dim3 gv(grid_for(g.V, 128), n);
    DD_KLAUNCH(h, filter_noise_kernel<<<gv, 128, 0, h->stream>>>(g, colour_mask, seed, ctr, h->d_ctr_off, eta_e, eta_o));
    DD_KLAUNCH(h, filter_source_kernel<<<gv, 128, 0, h->stream>>>(g, colour_mask, (const double*)h->fields[0].canon,
                                                                 canon_fs, h->d_active_mask, eta_e, eta_o, v.be,
                                                                 v.bo, h->prm.kappa));
    DD_LAUNCH_CHECK(h, "filter_source_kernel");
    const int colour = colour_mask == 1 ? 0 : colour_mask == 2 ? 1 : -1;
    int it = 0;
    int rc = solve_packed(h, n, 1, 1, h->prm.inner_prec, h->prm.tol_block, h->prm.maxit, &it, nullptr, 1, colour);
    if (rc && rc != DD_ERR_NOT_CONVERGED) return dd_fail(h, rc, "block filter: Dirichlet solves failed");
    if (rc == DD_ERR_NOT_CONVERGED) raise_status_host(h, DD_ERR_NOT_CONVERGED);
    DD_KLAUNCH(h, filter_estimate_kernel<<<g.nblocks, 256, 0, h->stream>>>(g, colour_mask, eta_e, eta_o, v.xe, v.xo, n,
                                                                         ln_b));
    DD_LAUNCH_CHECK(h, "filter_estimate_kernel");
    return DD_OK;
}

// autotuner probe: one masked block-filter pass (n = 1, every block)
int tune_block_filter_masked(dd_handle* h, const double* U_old, const double* U_new, int reps, float* ms) {
    int rc = prepare_fields(h, U_old, U_new, 1, true, true);
    if (rc) return rc;
    double* ln = h->d_item_out;  // only timed; the values are discarded (nblocks <= items_cap)
    cudaEvent_t e0, e1;
    DD_CUDA(h, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return dd_fail(h, DD_ERR_CUDA, "cudaEventCreate");
    }
    rc = block_filter_masked(h, 3, 1, 1, 0, ln);
    cudaEventRecord(e0, h->stream);
    for (int r = 0; r < reps && !rc; ++r) rc = block_filter_masked(h, 3, 1, 1, 0, ln);
    cudaEventRecord(e1, h->stream);
    float t = -1.f;
    if (!rc && cudaEventSynchronize(e1) == cudaSuccess) {
        cudaEventElapsedTime(&t, e0, e1);
        t /= (float)reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (t < 0) return dd_fail(h, DD_ERR_CUDA, "masked block-filter timing failed");
    *ms = t;
    return DD_OK;
}

// ------------------------------------------------------------- entry points
extern "C" int dd_block_filter(dd_t h, const void* U_old, void* U_new, int colour_mask, int mode, int n,
                               uint64_t seed, uint64_t ctr, double* ln_b, uint8_t* accept) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_estimate, "dd_block_filter");
    if (rc) return rc;
    if (!U_old || !U_new || !ln_b || !accept || n < 1 || n > h->prm.max_rhs || colour_mask < 1 || colour_mask > 3)
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_block_filter: bad arguments");
    // with one level of recursion this filter is step 1 of Eq. 4step: the
    // smallest blocks (sub-blocks)
    LevelScope level(h, true);
    if (mode == DD_FILTER_EXACT) {
        rc = block_filter_exact(h, (const double*)U_old, (const double*)U_new, colour_mask, ln_b);
        if (rc) return rc;
    } else if (mode == DD_FILTER_STOCHASTIC && h->tune.filter_masked) {
        rc = prepare_fields(h, (const double*)U_old, (const double*)U_new, n, true, true);
        if (rc) return rc;
        rc = block_filter_masked(h, colour_mask, n, seed, ctr, ln_b);
        if (rc) return rc;
    } else if (mode == DD_FILTER_STOCHASTIC) {
        rc = prepare_fields(h, (const double*)U_old, (const double*)U_new, n, true, false);
        if (rc) return rc;
        const Geo& g = h->g;
        // the blocks of the selected colours are contiguous in block order
        // (black first); n consecutive items per block
        const int half = g.nblocks / 2;
        const int pos0 = colour_mask == 2 ? half : 0;
        const int nb = colour_mask == 3 ? g.nblocks : half;
        rc = launch_blocks(h, BLOCK_FILTER, pos0, n, nb * n, nullptr, nullptr, seed, ctr);
        if (rc) return rc;
        DD_KLAUNCH(h, sum_items_kernel<<<grid_for(g.nblocks, 128), 128, 0, h->stream>>>(g, nullptr, colour_mask, pos0, n,
                                                                                       h->d_item_out, ln_b));
        DD_LAUNCH_CHECK(h, "sum_items_kernel");
    } else {
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_block_filter: unknown mode");
    }
    DD_KLAUNCH(h, block_accept_kernel<<<grid_for(h->g.nblocks, 128), 128, 0, h->stream>>>(h->g, colour_mask, ln_b, accept, seed,
                                                                                         ctr, h->d_ctr_off));
    if (h->n_active > 0)
        DD_KLAUNCH(h, restore_kernel<<<grid_for(h->n_active, 128), 128, 0, h->stream>>>(h->g, h->n_active, h->d_active_links, accept,
                                                                        (const double*)U_old, (double*)U_new));
    DD_LAUNCH_CHECK(h, "block accept");
    return DD_OK;
}

// --------------------------------------------- block filter by block ranges
// ln_b of the blocks at block-order positions [pos0, pos0 + npos), 0 elsewhere
__global__ void sum_range_kernel(Geo g, int pos0, int npos, int n, const double* item_out, double* ln_b) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= g.nblocks) return;
    int B[4] = {b % g.nbk[0], (b / g.nbk[0]) % g.nbk[1], (b / (g.nbk[0] * g.nbk[1])) % g.nbk[2],
                b / (g.nbk[0] * g.nbk[1] * g.nbk[2])};
    const int pos = block_pos_of(g, b, (B[0] + B[1] + B[2] + B[3]) & 1);
    double s = 0.0;
    if (pos >= pos0 && pos < pos0 + npos)
        for (int i = 0; i < n; ++i) s += item_out[(pos - pos0) * n + i];
    ln_b[b] = s;
}

extern "C" int dd_block_ratios_range(dd_t h, const void* U_old, const void* U_new, int pos0, int npos, int n,
                                     uint64_t seed, uint64_t ctr, double* ln_b) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_estimate, "dd_block_ratios_range");
    if (rc) return rc;
    LevelScope level(h, true);
    const Geo& g = h->g;
    if (!U_old || !U_new || !ln_b || n < 1 || n > h->prm.max_rhs || pos0 < 0 || npos < 0 || pos0 + npos > g.nblocks)
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_block_ratios_range: bad arguments");
    rc = prepare_fields(h, (const double*)U_old, (const double*)U_new, n, true, false);
    if (rc) return rc;
    rc = launch_blocks(h, BLOCK_FILTER, pos0, n, npos * n, nullptr, nullptr, seed, ctr);
    if (rc) return rc;
    DD_KLAUNCH(h, sum_range_kernel<<<grid_for(g.nblocks, 128), 128, 0, h->stream>>>(g, pos0, npos, n, h->d_item_out,
                                                                                   ln_b));
    DD_LAUNCH_CHECK(h, "sum_range_kernel");
    return DD_OK;
}

extern "C" int dd_block_accept(dd_t h, const void* U_old, void* U_new, int colour_mask, const double* ln_b,
                               uint64_t seed, uint64_t ctr, uint8_t* accept) {
    if (!h) return DD_ERR_INVALID_ARG;
    if (!U_old || !U_new || !ln_b || !accept || colour_mask < 1 || colour_mask > 3)
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_block_accept: bad arguments");
    LevelScope level(h, true);
    DD_KLAUNCH(h, block_accept_kernel<<<grid_for(h->g.nblocks, 128), 128, 0, h->stream>>>(h->g, colour_mask, ln_b,
                                                                                         accept, seed, ctr,
                                                                                         h->d_ctr_off));
    if (h->n_active > 0)
        DD_KLAUNCH(h, restore_kernel<<<grid_for(h->n_active, 128), 128, 0, h->stream>>>(
                          h->g, h->n_active, h->d_active_links, accept, (const double*)U_old, (double*)U_new));
    DD_LAUNCH_CHECK(h, "dd_block_accept");
    return DD_OK;
}

// ------------------------------------------------ multi-lattice block filter
namespace {
struct BatchPlan {
    size_t lats, items, item_out, queue, bases, scratch, total;
    long long slot_bytes;
    int slots, nitems;
};
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
BatchPlan batch_plan(int nh, dd_handle* const* hs, int n) {
    BatchPlan p;
    int nitems = 0, nbmax = 0, nblk = 0;
    for (int k = 0; k < nh; ++k) {
        nitems += hs[k]->g.nblocks * n;
        nbmax = std::max(nbmax, hs[k]->g.bsites);
        nblk += hs[k]->g.nblocks;
    }
    p.nitems = nitems;
    p.slot_bytes = (long long)((((size_t)nbmax * (4 * 192 + 5 * 192)) + 4096 + 255) & ~(size_t)255);
    p.slots = std::max(1, hs[0]->num_sms) * hs[0]->tune.block_ctas_per_sm;
    size_t off = 0;
    p.lats = off;
    off = align256(off + sizeof(LatDesc) * nh);
    p.items = off;
    off = align256(off + sizeof(BlockItem) * nitems);
    p.item_out = off;
    off = align256(off + sizeof(double) * nitems);
    p.queue = off;
    off = align256(off + 64 * sizeof(int));
    p.bases = off;
    off = align256(off + sizeof(int) * nblk);
    p.scratch = off;
    off = align256(off + (size_t)p.slot_bytes * p.slots);
    p.total = off;
    return p;
}
// the stream a handle was created with (while it records a graph, its work
// goes to the capture stream instead)
cudaStream_t caller_stream(const dd_handle* h) { return h->capturing ? h->user_stream : h->stream; }

int batch_check(int nh, dd_handle* const* hs, int n) {
    if (nh < 1 || !hs) return DD_ERR_INVALID_ARG;
    for (int k = 0; k < nh; ++k) {
        if (!hs[k] || !hs[k]->ws || !hs[k]->feat_estimate || hs[k]->has_sub) return DD_ERR_INVALID_ARG;
        if (n < 1 || n > hs[k]->prm.max_rhs) return DD_ERR_INVALID_ARG;
        if (caller_stream(hs[k]) != caller_stream(hs[0]) || hs[k]->prm.block_prec != hs[0]->prm.block_prec)
            return DD_ERR_INVALID_ARG;
        if (k > 0 && hs[k]->capturing) return DD_ERR_INVALID_ARG;  // only the first handle may record
    }
    return DD_OK;
}
}  // namespace

extern "C" int dd_block_filter_batch_workspace(int nh, const dd_t* hs, int n, size_t* bytes) {
    int rc = batch_check(nh, (dd_handle* const*)hs, n);
    if (rc) return rc;
    if (!bytes) return DD_ERR_INVALID_ARG;
    *bytes = batch_plan(nh, (dd_handle* const*)hs, n).total;
    return DD_OK;
}

extern "C" int dd_block_filter_batch(int nh, const dd_t* hs_, const void* const* U_old, void* const* U_new,
                                     int colour_mask, int n, uint64_t seed, uint64_t ctr, double* const* ln_b,
                                     uint8_t* const* accept, void* ws, size_t ws_bytes) {
    dd_handle* const* hs = (dd_handle* const*)hs_;
    int rc = batch_check(nh, hs, n);
    if (rc) return rc;
    dd_handle* h0 = hs[0];
    if (!U_old || !U_new || !ln_b || !accept || !ws || colour_mask < 1 || colour_mask > 3 || ((uintptr_t)ws & 255))
        return dd_fail(h0, DD_ERR_INVALID_ARG, "dd_block_filter_batch: bad arguments");
    const BatchPlan P = batch_plan(nh, hs, n);
    if (ws_bytes < P.total) return dd_fail(h0, DD_ERR_INVALID_ARG, "dd_block_filter_batch: workspace too small");
    for (int k = 0; k < nh; ++k)
        if (!U_old[k] || !U_new[k] || !ln_b[k] || !accept[k])
            return dd_fail(h0, DD_ERR_INVALID_ARG, "dd_block_filter_batch: null field or output");
    // every launch of the batch runs on the first handle's stream (also while
    // that handle records a CUDA graph): the other handles follow it for the call
    struct FollowFirst {
        dd_handle* const* hs;
        int nh;
        std::vector<cudaStream_t> streams;
        std::vector<bool> capturing;
        FollowFirst(dd_handle* const* hs_, int nh_) : hs(hs_), nh(nh_), streams(nh_), capturing(nh_) {
            for (int k = 0; k < nh; ++k) {
                streams[k] = hs[k]->stream;
                capturing[k] = hs[k]->capturing;
                hs[k]->stream = hs[0]->stream;
                hs[k]->capturing = hs[0]->capturing;
            }
        }
        ~FollowFirst() {
            for (int k = 1; k < nh; ++k) {
                hs[k]->stream = streams[k];
                hs[k]->capturing = capturing[k];
            }
        }
    } follow(hs, nh);
    char* w = (char*)ws;
    LatDesc* d_lats = (LatDesc*)(w + P.lats);
    BlockItem* d_items = (BlockItem*)(w + P.items);
    double* d_out = (double*)(w + P.item_out);
    int* d_queue = (int*)(w + P.queue);
    int* d_bases = (int*)(w + P.bases);
    // interpolated fields of every lattice (each handle's own slots)
    for (int k = 0; k < nh; ++k) {
        rc = prepare_fields(hs[k], (const double*)U_old[k], (const double*)U_new[k], n, true, false);
        if (rc) return rc;
    }
    // lattices with the largest blocks first: their items start first (LPT)
    std::vector<int> order(nh);
    for (int k = 0; k < nh; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return hs[a]->g.bsites > hs[b]->g.bsites; });
    std::vector<LatDesc> lats(nh);
    std::vector<BlockItem> items;
    std::vector<int> bases;
    std::vector<int> base_off(nh);
    items.reserve(P.nitems);
    for (int k = 0; k < nh; ++k) {
        dd_handle* h = hs[k];
        LatDesc& L = lats[k];
        L.g = h->g;
        L.c = block_ctx(h);
        L.dd64 = h->fields[0].dd64;
        L.dd64_fs = (long long)(h->fields[1].dd64 - h->fields[0].dd64);
        L.dd32 = h->fields[0].dd32;
        L.dd32_fs = (long long)(h->fields[1].dd32 - h->fields[0].dd32);
        L.item_out = d_out;
    }
    std::vector<std::vector<int>> per_base(nh);
    for (int oi = 0; oi < nh; ++oi) {
        const int k = order[oi];
        const Geo& g = hs[k]->g;
        per_base[k].assign(g.nblocks, -1);
        const int half = g.nblocks / 2;
        for (int pos = 0; pos < g.nblocks; ++pos) {
            const int col = pos >= half ? 1 : 0;
            if (!((colour_mask >> col) & 1)) continue;
            // block id of this position (host mirror of block_id_at)
            int rank = pos - col * half, id = 2 * rank;
            int B1 = (id / g.nbk[0]) % g.nbk[1], B2 = (id / (g.nbk[0] * g.nbk[1])) % g.nbk[2],
                B3 = id / (g.nbk[0] * g.nbk[1] * g.nbk[2]);
            if (((B1 + B2 + B3) & 1) != col) id += 1;
            per_base[k][id] = (int)items.size();
            for (int i = 0; i < n; ++i) items.push_back(BlockItem{pos, i, i + 1, i, k});
        }
    }
    int off = 0;
    for (int k = 0; k < nh; ++k) {
        base_off[k] = off;
        bases.insert(bases.end(), per_base[k].begin(), per_base[k].end());
        off += hs[k]->g.nblocks;
    }
    cudaStream_t s = h0->stream;
    // descriptor tables (skipped when the workspace already holds them, as
    // it must inside a graph capture)
    rc = upload_cached(h0, 0, d_lats, lats.data(), sizeof(LatDesc) * nh);
    if (!rc && !items.empty()) rc = upload_cached(h0, 1, d_items, items.data(), sizeof(BlockItem) * items.size());
    if (!rc) rc = upload_cached(h0, 2, d_bases, bases.data(), sizeof(int) * bases.size());
    if (rc) return rc;
    DD_CUDA(h0, cudaMemsetAsync(d_queue, 0, sizeof(int), s));
    if (!items.empty()) {
        BlockArgs A;
        A.lats = d_lats;
        A.g = h0->g;
        A.c = block_ctx(h0);
        A.mode = BLOCK_FILTER;
        A.items = d_items;
        A.nitems = (int)items.size();
        A.item_pos0 = 0;
        A.item_n = n;
        A.queue = d_queue;
        A.dd64 = h0->fields[0].dd64;
        A.dd64_fs = 0;
        A.dd32 = h0->fields[0].dd32;
        A.dd32_fs = 0;
        A.in_bank = nullptr;
        A.out_bank = nullptr;
        A.bank_vs = 0;
        A.item_out = d_out;
        A.scratch = w + P.scratch;
        A.slot_bytes = P.slot_bytes;
        A.seed = seed;
        A.ctr = ctr;
        A.ctr_off = h0->d_ctr_off;
        A.purpose = DD_PURPOSE_BLOCK_NOISE;
        A.tol2 = h0->prm.tol_block * h0->prm.tol_block;
        A.inner_f64 = h0->prm.block_prec == DD_PREC_F64;
        A.tol2_inner = A.inner_f64 ? 0.25 * A.tol2 : 1e-10;
        A.maxit_inner = std::min(h0->prm.maxit, 2000);
        A.max_outer = A.inner_f64 ? 3 : 12;
        A.status = h0->d_status;
        A.stats = h0->d_sites + DD_TIMER_KINDS;
        const int grid = std::min((int)items.size(), P.slots);
        const int tpb = h0->tune.block_tpb;
        const bool timed = block_timer_begin(h0);
        ++h0->block_launches;
        if (A.inner_f64)
            DD_KLAUNCH(h0, block_solve_kernel<double, SpinorF64, LinkF64><<<grid, tpb, 0, s>>>(A));
        else
            DD_KLAUNCH(h0, block_solve_kernel<float, SpinorF32, LinkF32><<<grid, tpb, 0, s>>>(A));
        if (timed) block_timer_end(h0, (int)items.size());
        DD_LAUNCH_CHECK(h0, "block_solve_kernel (batch)");
    }
    for (int k = 0; k < nh; ++k) {
        dd_handle* h = hs[k];
        DD_KLAUNCH(h, sum_items_kernel<<<grid_for(h->g.nblocks, 128), 128, 0, s>>>(h->g, d_bases + base_off[k],
                                                                                 colour_mask, 0, n, d_out, ln_b[k]));
        DD_KLAUNCH(h, block_accept_kernel<<<grid_for(h->g.nblocks, 128), 128, 0, s>>>(h->g, colour_mask, ln_b[k],
                                                                                    accept[k], seed, ctr,
                                                                                    h0->d_ctr_off));
        if (h->n_active > 0)
            DD_KLAUNCH(h, restore_kernel<<<grid_for(h->n_active, 128), 128, 0, s>>>(
                              h->g, h->n_active, h->d_active_links, accept[k], (const double*)U_old[k],
                              (double*)U_new[k]));
        DD_LAUNCH_CHECK(h, "dd_block_filter_batch accept");
    }
    return DD_OK;
}

extern "C" int dd_det_ratio_estimate(dd_t h, const void* U_old, const void* U_new, int n, uint64_t seed,
                                     uint64_t ctr, int mode, double* ln_out) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_estimate, "dd_det_ratio_estimate");
    if (rc) return rc;
    const bool all_links = (mode & DD_EST_INTERP_ALL) != 0;
    mode &= ~DD_EST_INTERP_ALL;
    if (!U_old || !U_new || !ln_out || n < 1 || n > h->prm.max_rhs || (mode != DD_EST_FACTORS && mode != DD_EST_REPLICAS))
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_det_ratio_estimate: bad arguments");
    const bool factors = mode == DD_EST_FACTORS;
    rc = prepare_fields(h, (const double*)U_old, (const double*)U_new, n, factors, true, all_links);
    if (rc) return rc;
    const Geo& g = h->g;
    const BlockCtx c = block_ctx(h);
    const int R = h->prm.max_rhs;
    const long long vs = 12LL * g.V;
    double2* bank[6];
    for (int k = 0; k < 6; ++k) bank[k] = h->dd_vec + (long long)k * R * vs;
    // field slot of the old / new operator of factor i: fs * i + {0, 1}
    const int fs = factors ? 1 : 0;
    const long long canon_fs = (long long)(h->fields[1].canon - h->fields[0].canon) * 2;  // doubles
    const long long dd64_fs = (long long)(h->fields[1].dd64 - h->fields[0].dd64);
    dim3 gv(grid_for(g.V, 128), n);
    // 1. eta on black sites
    const int4 no_outer = make_int4(0, 0, 0, 0);
    DD_KLAUNCH(h, noise_black_kernel<<<gv, 128, 0, h->stream>>>(g, c, bank[0], vs, DD_PURPOSE_GLOBAL_NOISE, seed, ctr,
                                                               h->d_ctr_off, no_outer, 3));
    // 2. w = C eta, w' = C' eta (onto white sites)
    DD_KLAUNCH(h, inter_hop_kernel<<<gv, 128, 0, h->stream>>>(g, c, bank[0], bank[1], vs, (const double*)h->fields[0].canon, canon_fs, 0, fs, 1, no_outer));
    DD_KLAUNCH(h, inter_hop_kernel<<<gv, 128, 0, h->stream>>>(g, c, bank[0], bank[2], vs, (const double*)h->fields[0].canon, canon_fs, 1, fs, 1, no_outer));
    DD_LAUNCH_CHECK(h, "schur stage 1-2");
    // 3. z = E^{-1} w, z' = E'^{-1} w': all white-block solves of all factors
    //    as one batched even-odd CG on the Dirichlet operator
    rc = dirichlet_solve_bank(h, bank[1], bank[3], n, 0, fs, 1);
    if (rc) return rc;
    rc = dirichlet_solve_bank(h, bank[2], bank[4], n, 1, fs, 1);
    if (rc) return rc;
    // 4. v = B z, v' = B' z' (onto black sites)
    DD_KLAUNCH(h, inter_hop_kernel<<<gv, 128, 0, h->stream>>>(g, c, bank[3], bank[1], vs, (const double*)h->fields[0].canon, canon_fs, 0, fs, 0, no_outer));
    DD_KLAUNCH(h, inter_hop_kernel<<<gv, 128, 0, h->stream>>>(g, c, bank[4], bank[2], vs, (const double*)h->fields[0].canon, canon_fs, 1, fs, 0, no_outer));
    DD_LAUNCH_CHECK(h, "schur stage 4");
    // 5. a = A^{-1} v (black-block solves)
    rc = dirichlet_solve_bank(h, bank[1], bank[5], n, 0, fs, 0);
    if (rc) return rc;
    // 6. s = v' - A' a  -> bank 3
    DD_KLAUNCH(h, schur_source_kernel<<<gv, 128, 0, h->stream>>>(g, c, bank[2], bank[5], bank[3], vs, h->fields[0].dd64, dd64_fs, 1, fs));
    // 7. global solve D' y = (s, 0)
    SolverVecs& v = h->vecs[0];
    DD_KLAUNCH(h, dd_to_eo_kernel<<<gv, 128, 0, h->stream>>>(g, c, bank[3], vs, v.be, v.bo));
    DD_LAUNCH_CHECK(h, "schur stage 6-7");
    int iters = 0;
    rc = solve_packed(h, n, 1, fs, h->prm.inner_prec, h->prm.tol_global, h->prm.maxit, &iters,
                      nullptr);
    if (rc && rc != DD_ERR_NOT_CONVERGED) return dd_fail(h, rc, "dd_det_ratio_estimate: global solve failed");
    // 8. ln r_i
    Reduce red;
    red.partials = h->d_partials;
    red.counters = h->d_counters;
    red.st = nullptr;
    red.out = ln_out;
    red.op = FIN_STORE;
    red.status = h->d_status;
    dim3 gb(grid_for(g.V / 2, 128), n);
    DD_KLAUNCH(h, estimate_kernel<<<gb, 128, 0, h->stream>>>(g, c, bank[0], vs, v.xe, v.xo, red));
    DD_LAUNCH_CHECK(h, "estimate_kernel");
    if (rc == DD_ERR_NOT_CONVERGED) return dd_fail(h, rc, "dd_det_ratio_estimate: global solve hit maxit");
    return DD_OK;
}

// ------------------------------------------- block Schur filter (step 2)
// ln_b[b] = -sum_i sum_{x in b, black sub-block} (2 Re<eta_i, d_i>_x + |d_i|_x^2)
// for every block b of g1 with colour in colour_mask (0 for the others): one
// thread block per block b, a fixed summation order (deterministic).  eta in
// the block order of the sub-blocks (g2, c2), d in even-odd FP64 chunks.
__global__ void __launch_bounds__(256) estimate_blocks_kernel(Geo g1, Geo g2, BlockCtx c2, const double2* eta_bank,
                                                              long long vs, const double2* xe, const double2* xo,
                                                              int n, int colour_mask, double* ln_b) {
    __shared__ double sh[34];
    const int b = blockIdx.x;
    int o[4];
    block_origin(g1, b, o);
    const int col = (o[0] / g1.b[0] + o[1] / g1.b[1] + o[2] / g1.b[2] + o[3] / g1.b[3]) & 1;
    if (!((colour_mask >> col) & 1)) {
        if (threadIdx.x == 0) ln_b[b] = 0.0;
        return;
    }
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int j = threadIdx.x; j < g1.bsites; j += blockDim.x) {
            int l[4] = {j % g1.b[0], (j / g1.b[0]) % g1.b[1], (j / (g1.b[0] * g1.b[1])) % g1.b[2],
                        j / (g1.b[0] * g1.b[1] * g1.b[2])};
            int x[4] = {o[0] + l[0], o[1] + l[1], o[2] + l[2], o[3] + l[3]};
            if (block_colour_of(g2, x)) continue;  // white sub-block: eta = 0
            const long long q = dd_position(g2, x);
            SpinorF64 es{(double2*)eta_bank + (long long)i * vs + (q / c2.nb) * 12 * c2.nb, c2.nb};
            Spinor<double> e, d;
            es.load(q % c2.nb, e);
            const int s = canon_index(g1, x);
            const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
            SpinorF64 ds{(double2*)(par ? xo : xe) + (long long)i * 12 * g1.Vh, g1.Vh};
            ds.load(s >> 1, d);
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < 12; ++k) t += 2.0 * (e.c[k].x * d.c[k].x + e.c[k].y * d.c[k].y) + norm2(d.c[k]);
            acc -= t;
        }
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) ln_b[b] = acc;
}

extern "C" int dd_block_schur_filter(dd_t h, const void* U_old, void* U_new, int colour_mask, int n, uint64_t seed,
                                     uint64_t ctr, double* ln_b, uint8_t* accept) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_estimate, "dd_block_schur_filter");
    if (rc) return rc;
    if (!h->has_sub) return dd_fail(h, DD_ERR_UNSUPPORTED, "dd_block_schur_filter: the handle has no sub-blocks");
    if (!U_old || !U_new || !ln_b || !accept || n < 1 || n > h->prm.max_rhs || colour_mask < 1 || colour_mask > 3)
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_block_schur_filter: bad arguments");
    const Geo g1 = h->g;
    const int R = h->prm.max_rhs;
    const long long vs = 12LL * g1.V;
    double2* bank[6];
    for (int k = 0; k < 6; ++k) bank[k] = h->dd_vec + (long long)k * R * vs;
    const int4 ob = make_int4(g1.b[0], g1.b[1], g1.b[2], g1.b[3]);
    SolverVecs& v = h->vecs[0];
    Geo g2;
    BlockCtx c2;
    {
        // Schur pieces of the sub-block decomposition inside every block:
        // block order, Dirichlet solves and colour tables of the sub-blocks
        LevelScope level(h, true);
        g2 = h->g;
        c2 = block_ctx(h);
        rc = prepare_fields(h, (const double*)U_old, (const double*)U_new, n, true, true);
        if (rc) return rc;
        const long long canon_fs = (long long)(h->fields[1].canon - h->fields[0].canon) * 2;
        const long long dd64_fs = (long long)(h->fields[1].dd64 - h->fields[0].dd64);
        dim3 gv(grid_for(g2.V, 128), n);
        // 1. eta on the black sub-blocks of the selected blocks
        DD_KLAUNCH(h, noise_black_kernel<<<gv, 128, 0, h->stream>>>(g2, c2, bank[0], vs, DD_PURPOSE_BLOCK_SCHUR_NOISE, seed,
                                                                   ctr, h->d_ctr_off, ob, colour_mask));
        // 2. w = C eta, w' = C' eta (hops across sub-block faces inside a block)
        DD_KLAUNCH(h, inter_hop_kernel<<<gv, 128, 0, h->stream>>>(g2, c2, bank[0], bank[1], vs, (const double*)h->fields[0].canon, canon_fs, 0, 1, 1, ob));
        DD_KLAUNCH(h, inter_hop_kernel<<<gv, 128, 0, h->stream>>>(g2, c2, bank[0], bank[2], vs, (const double*)h->fields[0].canon, canon_fs, 1, 1, 1, ob));
        DD_LAUNCH_CHECK(h, "block schur stage 1-2");
        // 3. z = E^{-1} w, z' = E'^{-1} w' (white sub-blocks)
        rc = dirichlet_solve_bank(h, bank[1], bank[3], n, 0, 1, 1);
        if (rc) return rc;
        rc = dirichlet_solve_bank(h, bank[2], bank[4], n, 1, 1, 1);
        if (rc) return rc;
        // 4. v = B z, v' = B' z'
        DD_KLAUNCH(h, inter_hop_kernel<<<gv, 128, 0, h->stream>>>(g2, c2, bank[3], bank[1], vs, (const double*)h->fields[0].canon, canon_fs, 0, 1, 0, ob));
        DD_KLAUNCH(h, inter_hop_kernel<<<gv, 128, 0, h->stream>>>(g2, c2, bank[4], bank[2], vs, (const double*)h->fields[0].canon, canon_fs, 1, 1, 0, ob));
        DD_LAUNCH_CHECK(h, "block schur stage 4");
        // 5. a = A^{-1} v (black sub-blocks)
        rc = dirichlet_solve_bank(h, bank[1], bank[5], n, 0, 1, 0);
        if (rc) return rc;
        // 6. s = v' - A' a
        DD_KLAUNCH(h, schur_source_kernel<<<gv, 128, 0, h->stream>>>(g2, c2, bank[2], bank[5], bank[3], vs, h->fields[0].dd64, dd64_fs, 1, 1));
        DD_KLAUNCH(h, dd_to_eo_kernel<<<gv, 128, 0, h->stream>>>(g2, c2, bank[3], vs, v.be, v.bo));
        DD_LAUNCH_CHECK(h, "block schur stage 5-6");
    }
    // 7. D1' y = (s, 0): the Dirichlet operator of the blocks plays the part
    //    of D in the global step (even-odd formats do not depend on blocks)
    int iters = 0;
    rc = solve_packed(h, n, 1, 1, h->prm.inner_prec, h->prm.tol_global, h->prm.maxit, &iters, nullptr, 1);
    if (rc && rc != DD_ERR_NOT_CONVERGED) return dd_fail(h, rc, "dd_block_schur_filter: block solve failed");
    if (rc == DD_ERR_NOT_CONVERGED) raise_status_host(h, DD_ERR_NOT_CONVERGED);
    // 8. per-block log-ratios, decisions, restore
    DD_KLAUNCH(h, estimate_blocks_kernel<<<g1.nblocks, 256, 0, h->stream>>>(g1, g2, c2, bank[0], vs, v.xe, v.xo, n,
                                                                          colour_mask, ln_b));
    DD_KLAUNCH(h, block_accept_kernel<<<grid_for(g1.nblocks, 128), 128, 0, h->stream>>>(
                      g1, colour_mask, ln_b, accept, seed, ctr, h->d_ctr_off, DD_PURPOSE_BLOCK_SCHUR_ACCEPT));
    if (h->n_active > 0)
        DD_KLAUNCH(h, restore_kernel<<<grid_for(h->n_active, 128), 128, 0, h->stream>>>(g1, h->n_active, h->d_active_links,
                                                                                      accept, (const double*)U_old,
                                                                                      (double*)U_new));
    DD_LAUNCH_CHECK(h, "block schur accept");
    return DD_OK;
}

extern "C" int dd_global_accept(dd_t h, void* U, const void* U_old, const double* ln_r, int n, uint64_t seed,
                                uint64_t ctr, uint8_t* accept, double* ln_margin) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    if (!U || !U_old || !ln_r || !accept || n < 1) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_global_accept: bad arguments");
    DD_KLAUNCH(h, global_accept_kernel<<<1, 1, 0, h->stream>>>(ln_r, n, seed, ctr, h->d_ctr_off, accept, ln_margin));
    const long long m = (long long)h->g.V * 72;
    DD_KLAUNCH(h, conditional_copy_kernel<<<grid_for(m, 256), 256, 0, h->stream>>>(m, accept, (const double*)U_old, (double*)U));
    DD_LAUNCH_CHECK(h, "global accept");
    return DD_OK;
}
