// Handle life cycle, geometry tables, workspace plan, field formatting and
// the operator-application entry points (dd_apply_D, dd_apply_D_block).
//
// Geometry follows Sec. 3 of the paper: non-overlapping blocks, checkerboard
// colouring of the blocks, block ordering with the black blocks first, and the
// active-link rule (links with at most one endpoint on a block boundary).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "dd_internal.h"
#include "dslash.cuh"

// ------------------------------------------------------------------ errors
int dd_fail(dd_handle* h, int code, const std::string& msg) {
    if (h) h->last_error = msg;
    return code;
}
int dd_cuda_check(dd_handle* h, cudaError_t e, const char* where) {
    return dd_fail(h, DD_ERR_CUDA, std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e));
}
int dd_require_ws(dd_handle* h) {
    if (!h) return DD_ERR_INVALID_ARG;
    if (!h->ws) return dd_fail(h, DD_ERR_NO_WORKSPACE, "no workspace: call dd_set_workspace first");
    return DD_OK;
}

static const char* g_no_handle = "invalid handle";

// ---------------------------------------------------------- host geometry
namespace {

struct HostGeo {
    int L[4], b[4], nbk[4];
    int V;
    int canon(const int x[4]) const { return x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3])); }
    void coords(int s, int x[4]) const {
        x[0] = s % L[0];
        s /= L[0];
        x[1] = s % L[1];
        s /= L[1];
        x[2] = s % L[2];
        x[3] = s / L[2];
    }
    int shift(int s, int a, int d) const {
        int x[4];
        coords(s, x);
        x[a] = (x[a] + d + L[a]) % L[a];
        return canon(x);
    }
    int block_id(int s) const {
        int x[4];
        coords(s, x);
        return x[0] / b[0] + nbk[0] * (x[1] / b[1] + nbk[1] * (x[2] / b[2] + nbk[2] * (x[3] / b[3])));
    }
    int colour(int s) const {
        int x[4];
        coords(s, x);
        return (x[0] / b[0] + x[1] / b[1] + x[2] / b[2] + x[3] / b[3]) & 1;
    }
    int local_index(int s) const {
        int x[4];
        coords(s, x);
        return x[0] % b[0] + b[0] * (x[1] % b[1] + b[1] * (x[2] % b[2] + b[2] * (x[3] % b[3])));
    }
    int nblocks() const { return nbk[0] * nbk[1] * nbk[2] * nbk[3]; }
    int bsites() const { return b[0] * b[1] * b[2] * b[3]; }
    long long dd_pos(int s) const {
        int id = block_id(s), c = colour(s);
        return (long long)(c * (nblocks() / 2) + id / 2) * bsites() + local_index(s);
    }
};

int resolve_mode(const dd_params& p) {
    if (p.active_mode != DD_ACTIVE_AUTO) return p.active_mode;
    int mn = std::min(std::min(p.block[0], p.block[1]), std::min(p.block[2], p.block[3]));
    if (mn <= 2) return DD_ACTIVE_INTRA;
    if (mn >= 8) return DD_ACTIVE_INNER6;
    return DD_ACTIVE_PAPER;
}

// active-link mask [V*4] following the rule of Sec. 3
std::vector<uint8_t> active_links(const HostGeo& G, int mode) {
    std::vector<uint8_t> act((size_t)G.V * 4, 0);
    if (mode == DD_ACTIVE_ALL) {
        std::fill(act.begin(), act.end(), (uint8_t)1);
        return act;
    }
    if (mode == DD_ACTIVE_INTRA) {
        for (int s = 0; s < G.V; ++s)
            for (int a = 0; a < 4; ++a) act[4 * s + a] = G.block_id(G.shift(s, a, +1)) == G.block_id(s);
        return act;
    }
    int lo = (mode == DD_ACTIVE_INNER6) ? 1 : 0;
    // region id: block id for sites inside the (shrunk) block, -1 outside
    std::vector<int> region(G.V);
    for (int s = 0; s < G.V; ++s) {
        int x[4];
        G.coords(s, x);
        bool in = true;
        for (int a = 0; a < 4; ++a) {
            int l = x[a] % G.b[a];
            if (l < lo || l > G.b[a] - 1 - lo) in = false;
        }
        region[s] = in ? G.block_id(s) : -1;
    }
    std::vector<uint8_t> bnd(G.V, 0);
    for (int s = 0; s < G.V; ++s) {
        if (region[s] < 0) continue;
        for (int a = 0; a < 4; ++a)
            if (region[G.shift(s, a, +1)] != region[s] || region[G.shift(s, a, -1)] != region[s]) bnd[s] = 1;
    }
    for (int s = 0; s < G.V; ++s) {
        if (region[s] < 0) continue;
        for (int a = 0; a < 4; ++a) {
            int y = G.shift(s, a, +1);
            act[4 * s + a] = (region[y] == region[s]) && !(bnd[s] && bnd[y]);
        }
    }
    return act;
}

}  // namespace

// --------------------------------------------------------- field formatting
__global__ void format_gauge_kernel(Geo g, const double* __restrict__ U, FieldSlot f) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x[4];
    canon_coords(g, s, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const long long h = s >> 1;
    const long long Vh = g.Vh;
    const long long q = dd_position(g, x);
    const long long bpos = q / g.bsites, j = q % g.bsites;
    const long long nb = g.bsites;
    for (int a = 0; a < 4; ++a) {
        const double* u = U + ((long long)s * 4 + a) * 18;
        if (f.eo64) {
            double2* o = f.eo64 + ((long long)par * 4 + a) * 9 * Vh + h;
            for (int k = 0; k < 9; ++k) o[k * Vh] = make_double2(u[2 * k], u[2 * k + 1]);
        }
        if (f.eo64 && f.eodf) {
            float4* o = f.eodf + ((long long)par * 4 + a) * 9 * Vh + h;
            for (int k = 0; k < 9; ++k) {
                const float rh = (float)u[2 * k], ih = (float)u[2 * k + 1];
                o[k * Vh] = make_float4(rh, ih, (float)(u[2 * k] - (double)rh), (float)(u[2 * k + 1] - (double)ih));
            }
        }
        if (f.eo32) {
            float4* o = f.eo32 + ((long long)par * 4 + a) * 3 * Vh + h;
            for (int k = 0; k < 3; ++k)
                o[k * Vh] = make_float4((float)u[4 * k], (float)u[4 * k + 1], (float)u[4 * k + 2], (float)u[4 * k + 3]);
        }
        if (f.eo16) {
            uint2* o = f.eo16 + ((long long)par * 4 + a) * 3 * Vh + h;
            for (int k = 0; k < 3; ++k) {
                uint2 v;
                __half2* hh = reinterpret_cast<__half2*>(&v);
                hh[0] = __floats2half2_rn((float)u[4 * k], (float)u[4 * k + 1]);
                hh[1] = __floats2half2_rn((float)u[4 * k + 2], (float)u[4 * k + 3]);
                o[k * Vh] = v;
            }
        }
        if (f.dd64) {
            double2* o = f.dd64 + (bpos * 4 + a) * 9 * nb + j;
            for (int k = 0; k < 9; ++k) o[k * nb] = make_double2(u[2 * k], u[2 * k + 1]);
        }
        if (f.dd32) {
            float4* o = f.dd32 + (bpos * 4 + a) * 3 * nb + j;
            for (int k = 0; k < 3; ++k)
                o[k * nb] = make_float4((float)u[4 * k], (float)u[4 * k + 1], (float)u[4 * k + 2], (float)u[4 * k + 3]);
        }
    }
}

int format_field(dd_handle* h, const double* U, FieldSlot& f, bool eo64, bool eo32, bool eo16, bool dd64, bool dd32) {
    FieldSlot t = f;
    if (!eo64) t.eo64 = nullptr;
    if (!eo32) t.eo32 = nullptr;
    if (!eo16) t.eo16 = nullptr;
    if (!dd64) t.dd64 = nullptr;
    if (!dd32) t.dd32 = nullptr;
    DD_KLAUNCH(h, format_gauge_kernel<<<grid_for(h->g.V, 128), 128, 0, h->stream>>>(h->g, U, t));
    DD_LAUNCH_CHECK(h, "format_gauge_kernel");
    return DD_OK;
}

// canonical [V][24 doubles] <-> eo FP64 chunks for one parity
__global__ void pack_spinor_eo_kernel(Geo g, const double* __restrict__ in, double2* out, int parity,
                                      long long in_rs) {
    int hh = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (hh >= g.Vh) return;
    int x[4];
    eo_coords(g, parity, hh, x);
    long long s = canon_index(g, x);
    const double* src = in + r * in_rs + s * 24;
    double2* dst = out + (long long)r * 12 * g.Vh + hh;
    for (int k = 0; k < 12; ++k) dst[(long long)k * g.Vh] = make_double2(src[2 * k], src[2 * k + 1]);
}
__global__ void unpack_spinor_eo_kernel(Geo g, const double2* __restrict__ in, double* out, int parity,
                                        long long out_rs) {
    int hh = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (hh >= g.Vh) return;
    int x[4];
    eo_coords(g, parity, hh, x);
    long long s = canon_index(g, x);
    double* dst = out + r * out_rs + s * 24;
    const double2* src = in + (long long)r * 12 * g.Vh + hh;
    for (int k = 0; k < 12; ++k) {
        double2 v = src[(long long)k * g.Vh];
        dst[2 * k] = v.x;
        dst[2 * k + 1] = v.y;
    }
}
// parity sub-vector [Vh][24 doubles] (sites of one parity in canonical order,
// i.e. by eo index) <-> eo FP64 chunks
__global__ void pack_spinor_sub_kernel(long long Vh, const double* __restrict__ in, double2* out) {
    long long hh = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (hh >= Vh) return;
    const double* src = in + ((long long)r * Vh + hh) * 24;
    double2* dst = out + (long long)r * 12 * Vh + hh;
    for (int k = 0; k < 12; ++k) dst[(long long)k * Vh] = make_double2(src[2 * k], src[2 * k + 1]);
}
__global__ void unpack_spinor_sub_kernel(long long Vh, const double2* __restrict__ in, double* out) {
    long long hh = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (hh >= Vh) return;
    double* dst = out + ((long long)r * Vh + hh) * 24;
    const double2* src = in + (long long)r * 12 * Vh + hh;
    for (int k = 0; k < 12; ++k) {
        double2 v = src[(long long)k * Vh];
        dst[2 * k] = v.x;
        dst[2 * k + 1] = v.y;
    }
}
void launch_pack_spinor_sub(dd_handle* h, const double* in, double2* out, int nrhs) {
    dim3 grid(grid_for(h->g.Vh, 128), nrhs);
    DD_KLAUNCH(h, pack_spinor_sub_kernel<<<grid, 128, 0, h->stream>>>(h->g.Vh, in, out));
}
void launch_unpack_spinor_sub(dd_handle* h, const double2* in, double* out, int nrhs) {
    dim3 grid(grid_for(h->g.Vh, 128), nrhs);
    DD_KLAUNCH(h, unpack_spinor_sub_kernel<<<grid, 128, 0, h->stream>>>(h->g.Vh, in, out));
}
void launch_pack_spinor_eo(dd_handle* h, const double* in, double2* out, int parity, int nrhs, long long in_rs) {
    dim3 grid(grid_for(h->g.Vh, 128), nrhs);
    DD_KLAUNCH(h, pack_spinor_eo_kernel<<<grid, 128, 0, h->stream>>>(h->g, in, out, parity, in_rs));
}
void launch_unpack_spinor_eo(dd_handle* h, const double2* in, double* out, int parity, int nrhs, long long out_rs) {
    dim3 grid(grid_for(h->g.Vh, 128), nrhs);
    DD_KLAUNCH(h, unpack_spinor_eo_kernel<<<grid, 128, 0, h->stream>>>(h->g, in, out, parity, out_rs));
}

// canonical <-> block-ordered FP64 chunks ([blockpos][chunk][bsites])
__global__ void pack_spinor_dd_kernel(Geo g, const double* __restrict__ in, double2* out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (s >= g.V) return;
    int x[4];
    canon_coords(g, s, x);
    long long q = dd_position(g, x);
    long long bpos = q / g.bsites, j = q % g.bsites;
    const double* src = in + ((long long)r * g.V + s) * 24;
    double2* dst = out + (long long)r * 12 * g.V + bpos * 12 * g.bsites + j;
    for (int k = 0; k < 12; ++k) dst[(long long)k * g.bsites] = make_double2(src[2 * k], src[2 * k + 1]);
}
__global__ void unpack_spinor_dd_kernel(Geo g, const double2* __restrict__ in, double* out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (s >= g.V) return;
    int x[4];
    canon_coords(g, s, x);
    long long q = dd_position(g, x);
    long long bpos = q / g.bsites, j = q % g.bsites;
    double* dst = out + ((long long)r * g.V + s) * 24;
    const double2* src = in + (long long)r * 12 * g.V + bpos * 12 * g.bsites + j;
    for (int k = 0; k < 12; ++k) {
        double2 v = src[(long long)k * g.bsites];
        dst[2 * k] = v.x;
        dst[2 * k + 1] = v.y;
    }
}
void launch_pack_spinor_dd(dd_handle* h, const double* in, double2* out, int nrhs) {
    dim3 grid(grid_for(h->g.V, 128), nrhs);
    DD_KLAUNCH(h, pack_spinor_dd_kernel<<<grid, 128, 0, h->stream>>>(h->g, in, out));
}
void launch_unpack_spinor_dd(dd_handle* h, const double2* in, double* out, int nrhs) {
    dim3 grid(grid_for(h->g.V, 128), nrhs);
    DD_KLAUNCH(h, unpack_spinor_dd_kernel<<<grid, 128, 0, h->stream>>>(h->g, in, out));
}

// eo FP64 chunks -> FP32 / FP16 storage and back
template <class SOut>
__global__ void convert_from64_kernel(long long n, SpinorF64 in, SOut out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (i >= n) return;
    Spinor<double> s;
    at_rhs(in, r).load(i, s);
    at_rhs(out, r).store(i, s);
}
template <class SIn>
__global__ void convert_to64_kernel(long long n, SIn in, SpinorF64 out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (i >= n) return;
    Spinor<float> s;
    at_rhs(in, r).load(i, s);
    Spinor<double> d;
    for (int k = 0; k < 12; ++k) d.c[k] = mk<double>(s.c[k].x, s.c[k].y);
    at_rhs(out, r).store(i, d);
}

// ----------------------------------------------------------- workspace plan
namespace {
struct Carver {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

void plan(dd_handle* h, char* base) {
    Carver c{base};
    const long long V = h->g.V, Vh = h->g.Vh;
    const int R = h->prm.max_rhs;
    const int feat = h->prm.features ? h->prm.features : (DD_FEAT_SOLVE | DD_FEAT_ESTIMATE | DD_FEAT_EXACT);
    const bool est = feat & DD_FEAT_ESTIMATE;
    const bool solve = est || (feat & DD_FEAT_SOLVE);
    // gauge-field slots: slot 0 always (eo formats; block-order copies with
    // the estimator), slots 1..R (interpolated fields) with the estimator
    h->fields.assign(R + 1, FieldSlot{});
    for (int k = 0; k <= (est ? R : 0); ++k) {
        FieldSlot& f = h->fields[k];
        f.eo64 = c.take<double2>((size_t)2 * 4 * 9 * Vh);
        f.eo32 = c.take<float4>((size_t)2 * 4 * 3 * Vh);
        f.eo16 = c.take<uint2>((size_t)2 * 4 * 3 * Vh);
        f.eodf = h->prm.outer_prec == DD_PREC_DF64 ? c.take<float4>((size_t)2 * 4 * 9 * Vh) : nullptr;
        if (est) {
            f.dd64 = c.take<double2>((size_t)4 * 9 * V);
            f.dd32 = c.take<float4>((size_t)4 * 3 * V);
            f.canon = c.take<double2>((size_t)4 * 9 * V);
        }
    }
    h->feat_solve = solve;
    h->feat_estimate = est;
    h->feat_exact = feat & DD_FEAT_EXACT;
    // global-solver vectors: each array holds R consecutive systems
    h->vecs.assign(1, SolverVecs{});
    SolverVecs& v = h->vecs[0];
    const int Rv = solve ? R : 0;  // no solver vectors without the solver
    {
    const int R = Rv;
    v.be = c.take<double2>((size_t)R * 12 * Vh);
    v.bo = c.take<double2>((size_t)R * 12 * Vh);
    v.xe = c.take<double2>((size_t)R * 12 * Vh);
    v.xo = c.take<double2>((size_t)R * 12 * Vh);
    v.re = c.take<double2>((size_t)R * 12 * Vh);
    v.t64 = c.take<double2>((size_t)R * 12 * Vh);
    v.t64b = c.take<double2>((size_t)R * 12 * Vh);
    v.x64 = c.take<double2>((size_t)R * 12 * Vh);
    v.p64 = c.take<double2>((size_t)R * 12 * Vh);
    v.q64 = c.take<double2>((size_t)R * 12 * Vh);
    v.z64 = c.take<double2>((size_t)R * 12 * Vh);
    v.x32 = c.take<float4>((size_t)R * 6 * Vh);
    v.r32 = c.take<float4>((size_t)R * 6 * Vh);
    v.p32 = c.take<float4>((size_t)R * 6 * Vh);
    v.q32 = c.take<float4>((size_t)R * 6 * Vh);
    v.z32 = c.take<float4>((size_t)R * 6 * Vh);
    v.t32 = c.take<float4>((size_t)R * 6 * Vh);
    v.w32 = c.take<float4>((size_t)R * 6 * Vh);
    v.h32 = c.take<float4>((size_t)R * 6 * Vh);
    v.p16 = c.take<uint4>((size_t)R * 3 * Vh);
    v.p16n = c.take<float>((size_t)R * Vh);
    v.r16 = c.take<uint4>((size_t)R * 3 * Vh);
    v.r16n = c.take<float>((size_t)R * Vh);
    v.t16 = c.take<uint4>((size_t)R * 3 * Vh);
    v.t16n = c.take<float>((size_t)R * Vh);
    v.q16 = c.take<uint4>((size_t)R * 3 * Vh);
    v.q16n = c.take<float>((size_t)R * Vh);
    }
    // block-ordered FP64 vectors: 6 banks of R vectors (estimator)
    h->dd_vec = c.take<double2>(est ? (size_t)6 * R * 12 * V : 0);
    h->d_cg = c.take<CGState>((size_t)3 * R + 2);
    // SAP-preconditioned GCR (global solves): full FP32 vectors (even, odd
    // halves of R systems each) and the block solver's vectors
    {
        SapVecs& s = h->sap;
        const bool on = solve && h->prm.krylov == DD_KRYLOV_SAP_GCR;
        const int nkv = on ? h->prm.sap_nkv : 0;
        const size_t half = on ? (size_t)R * 6 * Vh : 0;
        s.halves = c.take<float4>(half * (size_t)(SapVecs::kFixedHalves + 4 * nkv));
        s.half = half;
        s.nkv = nkv;
        const long long nblk = grid_for(Vh, 128);
        s.partials = c.take<double>(on ? (size_t)nblk * R * 2 * (DD_SAP_MAX_NKV + 1) : 0);
        s.nblk = (int)nblk;
        s.sc = c.take<double>(on ? (size_t)R * 4 * (DD_SAP_MAX_NKV + 4) : 0);
    }
    // partials of grid reductions with tiles of 64 sites or more (3 values per tile)
    h->partials_cap = (size_t)(grid_for(std::max(Vh, V), 64) + 64) * (R + 1) * 2;
    h->d_partials = c.take<double>(h->partials_cap);
    h->d_counters = c.take<unsigned>((size_t)4 * (R + 1) + 64);
    h->d_scalars = c.take<double>((size_t)64 * (R + 2));
    // persistent block-solver slots
    const long long nb = h->g.bsites;
    // 4 FP64 vectors + 5 inner vectors (FP64 at most) of one block
    h->block_slot_bytes = ((size_t)nb * (4 * 192 + 5 * 192) + 4096 + 255) & ~(size_t)255;
    h->block_slots = std::max(1, h->num_sms) * DD_BLOCK_CTAS_MAX;
    h->block_scratch = c.take<char>(est ? h->block_slot_bytes * h->block_slots : 0);
    h->items_cap = std::max(h->g.nblocks, h->has_sub ? h->g2.nblocks : 0) * 2 * R + 64;
    h->d_items = c.take<int>((size_t)5 * h->items_cap);  // five ints per item
    h->d_item_out = c.take<double>((size_t)h->items_cap);
    h->d_queue = c.take<int>(64);
    h->d_imap = c.take<int>((size_t)h->g.nblocks + 4 * R + 64);
    h->d_gauge_g = c.take<double>(est ? (size_t)V * 18 : 0);
    // dense LU matrices of the exact check path: D, the augmented block
    // systems and Dhat of lattices up to 512 sites (at most 3 (12V)^2
    // complex), or the batch of block operators of small blocks
    if (!(feat & DD_FEAT_EXACT)) {
        h->lu_bytes = 0;
        h->d_lu = nullptr;
    } else if (V <= 512) {
        h->lu_bytes = (size_t)(12 * V) * (12 * V) * 16 * 3 + (size_t)(12 * V) * 64;
        h->d_lu = c.take<double>(h->lu_bytes / 8);
    } else if (nb <= 16 && h->g.nblocks <= 1024) {
        h->lu_bytes = (size_t)h->g.nblocks * (12 * nb) * (12 * nb) * 16 + (size_t)h->g.nblocks * 12 * nb * 8;
        h->d_lu = c.take<double>(h->lu_bytes / 8);
    } else {
        h->lu_bytes = 0;
        h->d_lu = nullptr;
    }
    h->ws_needed = c.off + 256;
}
}  // namespace

// -------------------------------------------------------------- entry points
extern "C" int dd_default_params(dd_params* p) {
    if (!p) return DD_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->kappa = 0.125;
    p->bc_time = -1;
    p->active_mode = DD_ACTIVE_AUTO;
    p->max_rhs = 1;
    p->inner_prec = DD_PREC_F16;
    p->block_prec = DD_PREC_F32;
    p->tol_global = 1e-10;
    p->tol_block = 1e-12;
    p->tol_inner = 1e-3;
    p->maxit = 20000;
    p->sap_ncy = 4;
    p->sap_nmr = 4;
    p->sap_nkv = 6;
    return DD_OK;
}

extern "C" int dd_init(dd_t* out, const dd_params* p, void* stream) {
    if (!out || !p) return DD_ERR_INVALID_ARG;
    *out = nullptr;
    dd_handle* h = new dd_handle();
    h->prm = *p;
    h->stream = (cudaStream_t)stream;
    Geo& g = h->g;
    long long V = 1;
    for (int a = 0; a < 4; ++a) {
        int L = p->dims[a], b = p->block[a];
        if (L < 2 || (L & 1) || b < 1 || L % b) {
            delete h;
            return DD_ERR_INVALID_ARG;
        }
        int nbk = L / b;
        if (nbk < 2 || (nbk & 1)) {
            delete h;
            return DD_ERR_INVALID_ARG;
        }
        g.L[a] = L;
        g.b[a] = b;
        g.nbk[a] = nbk;
        V *= L;
    }
    if (!(p->kappa > 0) || p->max_rhs < 1 || (p->bc_time != 1 && p->bc_time != -1) || V > (1LL << 30)) {
        delete h;
        return DD_ERR_INVALID_ARG;
    }
    // the random streams number the spinor components of a site 12 s + k in
    // one 32-bit counter word: a larger lattice would repeat its noise
    if (12 * V > 0xFFFFFFFFLL) {
        delete h;
        return DD_ERR_UNSUPPORTED;
    }
    if (p->inner_prec < DD_PREC_F64 || p->inner_prec > DD_PREC_F16 || p->block_prec < DD_PREC_F64 ||
        p->block_prec > DD_PREC_F32 || p->active_mode < DD_ACTIVE_AUTO || p->active_mode > DD_ACTIVE_ALL ||
        (p->outer_prec != DD_PREC_F64 && p->outer_prec != DD_PREC_DF64) || p->krylov < DD_KRYLOV_CGNR ||
        p->krylov > DD_KRYLOV_SAP_GCR) {
        delete h;
        return DD_ERR_INVALID_ARG;
    }
    if (p->krylov == DD_KRYLOV_SAP_GCR &&
        (p->outer_prec != DD_PREC_F64 || p->sap_ncy < 1 || p->sap_ncy > 16 || p->sap_nmr < 1 || p->sap_nmr > 64 ||
         p->sap_nkv < 1 || p->sap_nkv > DD_SAP_MAX_NKV)) {
        delete h;
        return DD_ERR_INVALID_ARG;
    }
    g.bc = p->bc_time;
    geo_finish(g);
    // one level of recursion: sub-blocks tile every block with an even
    // number of sub-blocks per direction (the sub-block checkerboard inside a
    // block is then the global one)
    const bool any_sub = p->sub_block[0] || p->sub_block[1] || p->sub_block[2] || p->sub_block[3];
    if (any_sub) {
        Geo& g2 = h->g2;
        g2 = g;
        for (int a = 0; a < 4; ++a) {
            int b2 = p->sub_block[a];
            if (b2 < 1 || g.b[a] % b2 || ((g.b[a] / b2) & 1)) {
                delete h;
                return DD_ERR_INVALID_ARG;
            }
            g2.b[a] = b2;
            g2.nbk[a] = g.L[a] / b2;
        }
        geo_finish(g2);
        h->has_sub = true;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete h;
        return DD_ERR_CUDA;
    }
    // active links of the smallest blocks, grouped by (colour, direction,
    // site parity) for the heat-bath
    const Geo& gf = h->has_sub ? h->g2 : g;
    HostGeo G;
    for (int a = 0; a < 4; ++a) {
        G.L[a] = gf.L[a];
        G.b[a] = gf.b[a];
        G.nbk[a] = gf.nbk[a];
    }
    G.V = gf.V;
    dd_params pf = *p;
    for (int a = 0; a < 4; ++a) pf.block[a] = gf.b[a];
    const int mode = resolve_mode(pf);
    if (mode == DD_ACTIVE_INNER6 && std::min(std::min(gf.b[0], gf.b[1]), std::min(gf.b[2], gf.b[3])) < 4) {
        delete h;
        return DD_ERR_INVALID_ARG;
    }
    h->active_mode = mode;
    std::vector<uint8_t> act = active_links(G, mode);
    std::vector<int> links;
    h->h_group_off.assign(17, 0);
    for (int col = 0; col < 2; ++col)
        for (int a = 0; a < 4; ++a)
            for (int par = 0; par < 2; ++par) {
                h->h_group_off[(col * 4 + a) * 2 + par] = (int)links.size();
                for (int s = 0; s < g.V; ++s) {
                    int x[4];
                    G.coords(s, x);
                    if (act[4 * s + a] && G.colour(s) == col && ((x[0] + x[1] + x[2] + x[3]) & 1) == par)
                        links.push_back(4 * s + a);
                }
            }
    h->h_group_off[16] = (int)links.size();
    h->n_active = (int)links.size();
    e = cudaMalloc(&h->d_active_links, sizeof(int) * std::max<size_t>(1, links.size()));
    if (e == cudaSuccess && !links.empty())
        e = cudaMemcpy(h->d_active_links, links.data(), sizeof(int) * links.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_active_mask, act.size());
    if (e == cudaSuccess) e = cudaMemcpy(h->d_active_mask, act.data(), act.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_hb_fails, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_hb_fails, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_sites, (DD_TIMER_KINDS + DD_BLOCK_STATS) * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_sites, 0, (DD_TIMER_KINDS + DD_BLOCK_STATS) * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_ctr_off, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_ctr_off, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_loop, sizeof(int) * DD_LOOP_SLOTS);
    if (e == cudaSuccess) e = cudaMemset(h->d_loop, 0, sizeof(int) * DD_LOOP_SLOTS);
    // sites of each block colour by even-odd index: with an even block
    // extent along axis 0, x0 = 2 hx and 2 hx + 1 lie in one block, so the
    // list is the same for both site parities (blocks, then sub-blocks)
    for (int lev = 0; lev < (h->has_sub ? 2 : 1); ++lev) {
        const Geo& gl = lev ? h->g2 : g;
        int** dst = lev ? h->d_colour_sites2 : h->d_colour_sites;
        if (e != cudaSuccess || (gl.b[0] & 1)) continue;
        std::vector<int> cs[2];
        for (int hh = 0; hh < gl.Vh; ++hh) {
            int hx = hh % gl.Lh0, r = hh / gl.Lh0;
            int x1 = r % gl.L[1], x2 = (r / gl.L[1]) % gl.L[2], x3 = r / (gl.L[1] * gl.L[2]);
            int x0 = 2 * hx + ((x1 + x2 + x3) & 1);
            int col = (x0 / gl.b[0] + x1 / gl.b[1] + x2 / gl.b[2] + x3 / gl.b[3]) & 1;
            cs[col].push_back(hh);
        }
        for (int col = 0; col < 2 && e == cudaSuccess; ++col) {
            e = cudaMalloc(&dst[col], sizeof(int) * std::max<size_t>(1, cs[col].size()));
            if (e == cudaSuccess)
                e = cudaMemcpy(dst[col], cs[col].data(), sizeof(int) * cs[col].size(), cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        cudaFree(h->d_active_links);
        cudaFree(h->d_active_mask);
        cudaFree(h->d_status);
        cudaFree(h->d_hb_fails);
        cudaFree(h->d_sites);
        cudaFree(h->d_ctr_off);
        cudaFree(h->d_loop);
        cudaFree(h->d_colour_sites[0]);
        cudaFree(h->d_colour_sites[1]);
        cudaFree(h->d_colour_sites2[0]);
        cudaFree(h->d_colour_sites2[1]);
        delete h;
        return DD_ERR_CUDA;
    }
    plan(h, nullptr);
    *out = h;
    return DD_OK;
}

extern "C" int dd_workspace_size(dd_t h, size_t* bytes) {
    if (!h || !bytes) return DD_ERR_INVALID_ARG;
    *bytes = h->ws_needed;
    return DD_OK;
}

extern "C" int dd_set_workspace(dd_t h, void* dev_ptr, size_t bytes) {
    if (!h || !dev_ptr) return dd_fail(h, DD_ERR_INVALID_ARG, "null workspace");
    if (bytes < h->ws_needed) return dd_fail(h, DD_ERR_INVALID_ARG, "workspace too small");
    if (((uintptr_t)dev_ptr) & 255) return dd_fail(h, DD_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    h->ws = (char*)dev_ptr;
    h->ws_size = bytes;
    plan(h, h->ws);
    // reduction tickets and solver states start from zero
    DD_CUDA(h, cudaMemsetAsync(h->d_counters, 0, sizeof(unsigned) * (4 * (h->prm.max_rhs + 1) + 64), h->stream));
    DD_CUDA(h, cudaMemsetAsync(h->d_cg, 0, sizeof(CGState) * (3 * h->prm.max_rhs + 2), h->stream));
    return DD_OK;
}

extern "C" int dd_get_maps(dd_t h, int32_t* nbr, int32_t* sign, int32_t* dd_order, int32_t* block_of,
                           uint8_t* active) {
    if (!h) return DD_ERR_INVALID_ARG;
    HostGeo G;
    for (int a = 0; a < 4; ++a) {
        G.L[a] = h->g.L[a];
        G.b[a] = h->g.b[a];
        G.nbk[a] = h->g.nbk[a];
    }
    G.V = h->g.V;
    for (int s = 0; s < G.V; ++s) {
        int x[4];
        G.coords(s, x);
        for (int a = 0; a < 4; ++a) {
            if (nbr) {
                nbr[8 * s + 2 * a] = G.shift(s, a, +1);
                nbr[8 * s + 2 * a + 1] = G.shift(s, a, -1);
            }
            if (sign) {
                sign[8 * s + 2 * a] = (a == 3 && x[3] == G.L[3] - 1) ? h->g.bc : 1;
                sign[8 * s + 2 * a + 1] = (a == 3 && x[3] == 0) ? h->g.bc : 1;
            }
        }
        if (dd_order) dd_order[G.dd_pos(s)] = s;
        if (block_of) block_of[s] = G.block_id(s);
    }
    if (active) {
        cudaError_t e = cudaMemcpy(active, h->d_active_mask, (size_t)G.V * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return dd_cuda_check(h, e, "dd_get_maps");
    }
    return DD_OK;
}

extern "C" int dd_sync(dd_t h) {
    if (!h) return DD_ERR_INVALID_ARG;
    DD_CUDA(h, cudaStreamSynchronize(h->stream));
    return DD_OK;
}

extern "C" int dd_status(dd_t h, int* device_status, long long* heatbath_fails) {
    if (!h) return DD_ERR_INVALID_ARG;
    int st = 0;
    unsigned long long hb = 0;
    DD_CUDA(h, cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DD_CUDA(h, cudaMemcpyAsync(&hb, h->d_hb_fails, sizeof(hb), cudaMemcpyDeviceToHost, h->stream));
    DD_CUDA(h, cudaStreamSynchronize(h->stream));
    DD_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    if (device_status) *device_status = st;
    if (heatbath_fails) *heatbath_fails = (long long)hb;
    return DD_OK;
}

extern "C" const char* dd_last_error(dd_t h) {
    if (!h) return g_no_handle;
    return h->last_error.c_str();
}

extern "C" int dd_launch_count(dd_t h, long long* launches) {
    if (!h || !launches) return DD_ERR_INVALID_ARG;
    *launches = (long long)h->launches;
    return DD_OK;
}

extern "C" int dd_kernel_timer(dd_t h, int op, int kind, int every, double* total_ms, long long* timed,
                               long long* sites) {
    if (!h || kind < 0 || kind >= DD_TIMER_KINDS) return DD_ERR_INVALID_ARG;
    if (op == 1) {
        h->timer_on = 1;
        h->timer_every = every > 0 ? every : 1;
        for (int k = 0; k < DD_TIMER_KINDS; ++k) {
            h->timer_used[k] = 0;
            h->timer_seen[k] = 0;
        }
        DD_CUDA(h, cudaMemsetAsync(h->d_sites, 0, (DD_TIMER_KINDS + DD_BLOCK_STATS) * sizeof(unsigned long long),
                                   h->stream));
        for (auto& k : h->solve_stats)
            for (long long& v : k) v = 0;
        h->block_launches = 0;
        return DD_OK;
    }
    if (op == 0) {
        h->timer_on = 0;
        return DD_OK;
    }
    if (op != 2) return DD_ERR_INVALID_ARG;
    DD_CUDA(h, cudaStreamSynchronize(h->stream));
    double tot = 0.0;
    long long cnt = 0;
    for (size_t i = 0; i + 1 < h->timer_used[kind]; i += 2) {
        float ms = 0.f;
        DD_CUDA(h, cudaEventElapsedTime(&ms, h->timer_ev[kind][i], h->timer_ev[kind][i + 1]));
        tot += ms;
        ++cnt;
    }
    unsigned long long ns[DD_TIMER_KINDS] = {};
    DD_CUDA(h, cudaMemcpy(ns, h->d_sites, sizeof(ns), cudaMemcpyDeviceToHost));
    if (total_ms) *total_ms = tot;
    if (timed) *timed = cnt;
    if (sites) *sites = (long long)ns[kind];
    return DD_OK;
}

extern "C" int dd_solver_stats(dd_t h, int kind, long long* out) {
    if (!h || !out || kind < 0 || kind > 2) return DD_ERR_INVALID_ARG;
    if (kind < 2) {
        for (int k = 0; k < 5; ++k) out[k] = h->solve_stats[kind][k];
        return DD_OK;
    }
    unsigned long long v[DD_BLOCK_STATS] = {};
    DD_CUDA(h, cudaStreamSynchronize(h->stream));
    DD_CUDA(h, cudaMemcpy(v, h->d_sites + DD_TIMER_KINDS, sizeof(v), cudaMemcpyDeviceToHost));
    out[0] = h->block_launches;
    for (int k = 0; k < 4; ++k) out[1 + k] = (long long)v[k];
    return DD_OK;
}

extern "C" int dd_finalize(dd_t h) {
    if (!h) return DD_ERR_INVALID_ARG;
    for (int k = 0; k < DD_TIMER_KINDS; ++k)
        for (cudaEvent_t e : h->timer_ev[k]) cudaEventDestroy(e);
    cudaFree(h->d_active_links);
    cudaFree(h->d_active_mask);
    cudaFree(h->d_status);
    cudaFree(h->d_hb_fails);
    cudaFree(h->d_sites);
    cudaFree(h->d_ctr_off);
    cudaFree(h->d_loop);
    cudaFree(h->d_colour_sites[0]);
    cudaFree(h->d_colour_sites[1]);
    cudaFree(h->d_colour_sites2[0]);
    cudaFree(h->d_colour_sites2[1]);
    for (cudaStream_t st : h->body_streams) cudaStreamDestroy(st);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
    return DD_OK;
}

// ------------------------------------------------------ operator application
namespace {

template <class SS, class LK>
int apply_eo_ops(dd_handle* h, int op, SS in_e, SS in_o, SS out_e, SS out_o, LK lk, int nrhs, int colour_mask,
                 int mask_mode) {
    const Geo& g = h->g;
    const double k = h->prm.kappa;
    typedef typename SS::real R;
    auto mk_args = [&](int p, SS in, SS x, SS out, double a, double b, int hasx, int g5) {
        HopArgs<SS, SS, SS, LK> A;
        A.g = g;
        A.p = p;
        A.in = in;
        A.xin = x;
        A.out = out;
        A.lk = lk;
        A.lk_rhs_stride = 0;
        A.a = a;
        A.b = b;
        A.has_x = hasx;
        A.g5in = g5;
        A.g5out = g5;
        A.colour_mask = colour_mask;
        A.st = nullptr;
        A.red.op = FIN_NONE;
        return A;
    };
    cudaStream_t s = h->stream;
    if (op == DD_OP_D || op == DD_OP_DDAG) {
        int g5 = (op == DD_OP_DDAG);
        auto A0 = mk_args(0, in_o, in_e, out_e, 1.0, -k, 1, g5);
        auto A1 = mk_args(1, in_e, in_o, out_o, 1.0, -k, 1, g5);
        if (mask_mode == 1) {
            launch_hop<R, SS, SS, SS, LK, 1>(A0, nrhs, h);
            launch_hop<R, SS, SS, SS, LK, 1>(A1, nrhs, h);
        } else {
            launch_hop<R, SS, SS, SS, LK, 0>(A0, nrhs, h);
            launch_hop<R, SS, SS, SS, LK, 0>(A1, nrhs, h);
        }
    } else if (op == DD_OP_INTER) {
        auto A0 = mk_args(0, in_o, in_e, out_e, 0.0, -k, 0, 0);
        auto A1 = mk_args(1, in_e, in_o, out_o, 0.0, -k, 0, 0);
        launch_hop<R, SS, SS, SS, LK, 2>(A0, nrhs, h);
        launch_hop<R, SS, SS, SS, LK, 2>(A1, nrhs, h);
    } else if (op == DD_OP_DTILDE || op == DD_OP_DTILDE_DAG) {
        // out_o used as the odd temporary: t = H_oe psi_e; out_e = psi_e - k^2 H_eo t
        int g5 = (op == DD_OP_DTILDE_DAG);
        auto A1 = mk_args(1, in_e, in_e, out_o, 0.0, 1.0, 0, 0);
        A1.g5in = g5;
        A1.g5out = 0;
        auto A0 = mk_args(0, out_o, in_e, out_e, 1.0, -k * k, 1, 0);
        A0.g5in = 0;
        A0.g5out = g5;
        launch_hop<R, SS, SS, SS, LK, 0>(A1, nrhs, h);
        launch_hop<R, SS, SS, SS, LK, 0>(A0, nrhs, h);
    } else if (op == DD_OP_HEO) {
        auto A0 = mk_args(0, in_o, in_e, out_e, 0.0, 1.0, 0, 0);
        launch_hop<R, SS, SS, SS, LK, 0>(A0, nrhs, h);
    } else {
        return DD_ERR_INVALID_ARG;
    }
    return DD_OK;
}

}  // namespace

static int apply_common(dd_handle* h, void* out, const void* in, const void* U, int op, int prec, int nrhs,
                        int colour_mask, int mask_mode) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_solve, "dd_apply_D");
    if (rc) return rc;
    if (!out || !in || !U || nrhs < 1 || nrhs > h->prm.max_rhs) return dd_fail(h, DD_ERR_INVALID_ARG, "apply: bad arguments");
    if (op < DD_OP_D || op > DD_OP_INTER) return dd_fail(h, DD_ERR_INVALID_ARG, "apply: unknown operator");
    if (prec < DD_PREC_F64 || prec > DD_PREC_F16) return dd_fail(h, DD_ERR_INVALID_ARG, "apply: unknown precision");
    const Geo& g = h->g;
    const long long Vh = g.Vh;
    FieldSlot& f = h->fields[0];
    rc = format_field(h, (const double*)U, f, prec == DD_PREC_F64, prec == DD_PREC_F32, prec == DD_PREC_F16, false, false);
    if (rc) return rc;
    SolverVecs& v = h->vecs[0];
    const bool even_in = (op == DD_OP_DTILDE || op == DD_OP_DTILDE_DAG);
    const bool odd_in = (op == DD_OP_HEO);
    const bool sub_out = even_in || odd_in;
    // input parities in FP64 eo chunks
    if (even_in) {
        launch_pack_spinor_sub(h, (const double*)in, v.be, nrhs);
    } else if (odd_in) {
        launch_pack_spinor_sub(h, (const double*)in, v.bo, nrhs);
    } else {
        launch_pack_spinor_eo(h, (const double*)in, v.be, 0, nrhs, 24LL * g.V);
        launch_pack_spinor_eo(h, (const double*)in, v.bo, 1, nrhs, 24LL * g.V);
    }
    DD_LAUNCH_CHECK(h, "pack");
    dim3 cg(grid_for(Vh, 128), nrhs);
    SpinorF64 be{v.be, Vh}, bo{v.bo, Vh}, xe{v.xe, Vh}, xo{v.xo, Vh};
    if (prec == DD_PREC_F64) {
        LinkF64 lk{f.eo64, Vh};
        rc = apply_eo_ops(h, op, be, bo, xe, xo, lk, nrhs, colour_mask, mask_mode);
    } else if (prec == DD_PREC_F32) {
        SpinorF32 ie{v.r32, Vh}, io{v.t32, Vh}, oe{v.p32, Vh}, oo{v.q32, Vh};
        DD_KLAUNCH(h, convert_from64_kernel<<<cg, 128, 0, h->stream>>>(Vh, be, ie));
        DD_KLAUNCH(h, convert_from64_kernel<<<cg, 128, 0, h->stream>>>(Vh, bo, io));
        LinkF32 lk{f.eo32, Vh};
        rc = apply_eo_ops(h, op, ie, io, oe, oo, lk, nrhs, colour_mask, mask_mode);
        DD_KLAUNCH(h, convert_to64_kernel<<<cg, 128, 0, h->stream>>>(Vh, oe, xe));
        DD_KLAUNCH(h, convert_to64_kernel<<<cg, 128, 0, h->stream>>>(Vh, oo, xo));
    } else {
        SpinorF16 ie{v.r16, v.r16n, Vh}, io{v.t16, v.t16n, Vh}, oe{v.p16, v.p16n, Vh}, oo{v.q16, v.q16n, Vh};
        DD_KLAUNCH(h, convert_from64_kernel<<<cg, 128, 0, h->stream>>>(Vh, be, ie));
        DD_KLAUNCH(h, convert_from64_kernel<<<cg, 128, 0, h->stream>>>(Vh, bo, io));
        LinkF16 lk{f.eo16, Vh};
        rc = apply_eo_ops(h, op, ie, io, oe, oo, lk, nrhs, colour_mask, mask_mode);
        DD_KLAUNCH(h, convert_to64_kernel<<<cg, 128, 0, h->stream>>>(Vh, oe, xe));
        DD_KLAUNCH(h, convert_to64_kernel<<<cg, 128, 0, h->stream>>>(Vh, oo, xo));
    }
    if (rc) return dd_fail(h, rc, "apply: unsupported operator");
    DD_LAUNCH_CHECK(h, "apply");
    if (sub_out) {
        launch_unpack_spinor_sub(h, v.xe, (double*)out, nrhs);
    } else {
        launch_unpack_spinor_eo(h, v.xe, (double*)out, 0, nrhs, 24LL * g.V);
        launch_unpack_spinor_eo(h, v.xo, (double*)out, 1, nrhs, 24LL * g.V);
    }
    DD_LAUNCH_CHECK(h, "unpack");
    return DD_OK;
}

extern "C" int dd_apply_D(dd_t h, void* out, const void* in, const void* U, int op, int prec, int nrhs) {
    if (!h) return DD_ERR_INVALID_ARG;
    return apply_common(h, out, in, U, op, prec, nrhs, 3, 0);
}

extern "C" int dd_apply_D_block(dd_t h, void* out, const void* in, const void* U, int colour_mask, int prec, int nrhs) {
    if (!h) return DD_ERR_INVALID_ARG;
    if (colour_mask < 1 || colour_mask > 3) return dd_fail(h, DD_ERR_INVALID_ARG, "apply_D_block: colour_mask must be 1, 2 or 3");
    return apply_common(h, out, in, U, DD_OP_D, prec, nrhs, colour_mask, 1);
}
