// Allocation-free variant of the stochastic block log-ratios (one factor).
//
// For callers that cannot allocate device memory, e.g. code that runs while a
// CUDA graph is being captured in global mode (where cudaMalloc is illegal),
// plug-ins whose host application owns all device memory, or latency-critical
// loops that cannot pay the implicit device synchronisation of
// cudaMalloc/cudaFree.  Such a caller passes only its inputs and outputs;
// every temporary of the block solves lives in one file-scope device array.
//
// The arithmetic: FP64 defect correction around an FP32 conjugate-gradient
// solve of each block's normal equations (the persistent block solver of
// dd_block_filter runs BiCGStab inside the same refinement), with the links
// read straight from the caller's canonical FP64 fields instead of from
// formatted copies in a workspace.  A block that misses tol_block reports NaN.
#include <mutex>

#include "blocksolve.cuh"

namespace {

// Scratch of the allocation-free entry point: 64 MiB, held by every GPU that
// loads the library until the process exits.  Bytes [0, 256) hold the work
// queue head and a status word; per-thread-block slots follow.
constexpr size_t kNoallocScratchBytes = 64ull << 20;
constexpr size_t kNoallocHeader = 256;
// fixed solver caps of this entry point (stated in include/dd.h)
constexpr int kNoallocMaxCycles = 12;        // FP64 defect-correction cycles
constexpr double kNoallocInnerTol = 1e-10;   // relative target of one FP32 CG solve
constexpr int kNoallocInnerMaxit = 2000;     // iterations of one FP32 CG solve
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// links of one block, read from a canonical FP64 field (V x 4 x 3 x 3 complex)
struct LinkCanonF64 {
    const double* U;
    Geo g;
    BlockCtx c;
    int org[4];
    template <class R>
    DD_DEV void load(long long j, int a, Link<R>& u) const {
        int l[4];
        local_coords(c, (int)j, l);
        int x[4] = {org[0] + l[0], org[1] + l[1], org[2] + l[2], org[3] + l[3]};
        const double* p = U + ((long long)canon_index(g, x) * 4 + a) * 18;
#pragma unroll
        for (int k = 0; k < 9; ++k) u.m[k / 3][k % 3] = mk<R>((R)p[2 * k], (R)p[2 * k + 1]);
    }
};
// the same links rounded to FP32, rows 0-1 stored, row 2 rebuilt (as LinkF32)
struct LinkCanonF32 {
    const double* U;
    Geo g;
    BlockCtx c;
    int org[4];
    template <class R>
    DD_DEV void load(long long j, int a, Link<R>& u) const {
        int l[4];
        local_coords(c, (int)j, l);
        int x[4] = {org[0] + l[0], org[1] + l[1], org[2] + l[2], org[3] + l[3]};
        const double* p = U + ((long long)canon_index(g, x) * 4 + a) * 18;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float re = (float)p[2 * k], im = (float)p[2 * k + 1];
            u.m[k / 3][k % 3] = mk<R>((R)re, (R)im);
        }
        reconstruct_row2(u);
    }
};

struct NoallocArgs {
    Geo g;
    BlockCtx c;
    const double* U_old;
    const double* U_new;
    double* ln_b;          // by block id
    int colour_mask;
    int nitems;            // blocks of the selected colours
    long long slot_bytes;
    uint64_t seed, ctr;
    double tol2;
};

// block id of the k-th block (in block order) among the selected colours
DD_DEV int selected_block(const NoallocArgs& A, int k, int* pos_out) {
    const int half = A.g.nblocks / 2;
    int pos;
    if (A.colour_mask == 3) pos = k;
    else if (A.colour_mask == 1) pos = k;
    else pos = half + k;
    *pos_out = pos;
    int colour;
    return block_id_at(A.g, pos, &colour);
}

__global__ void __launch_bounds__(256) noalloc_block_kernel(NoallocArgs A) {
    __shared__ double sh[34];
    __shared__ int s_item;
    int* queue = reinterpret_cast<int*>(g_noalloc_scratch);
    int* status = queue + 1;
    const BlockCtx& c = A.c;
    const long long nb = c.nb;
    char* base = reinterpret_cast<char*>(g_noalloc_scratch) + kNoallocHeader + (long long)blockIdx.x * A.slot_bytes;
    SpinorF64 eta{(double2*)base, nb};
    SpinorF64 bv{(double2*)base + 12 * nb, nb};
    SpinorF64 xv{(double2*)base + 24 * nb, nb};
    SpinorF64 rv{(double2*)base + 36 * nb, nb};
    char* ib = base + 48 * nb * sizeof(double2);
    SpinorF32 xi{(float4*)ib, nb}, ri{(float4*)ib + 6 * nb, nb}, pi{(float4*)ib + 12 * nb, nb},
        qi{(float4*)ib + 18 * nb, nb}, zi{(float4*)ib + 24 * nb, nb};
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= A.nitems) break;
        int pos;
        const int id = selected_block(A, item, &pos);
        int org[4];
        block_origin(A.g, id, org);
        LinkCanonF64 lsrc{A.U_old, A.g, c, {org[0], org[1], org[2], org[3]}};
        LinkCanonF64 lsol{A.U_new, A.g, c, {org[0], org[1], org[2], org[3]}};
        LinkCanonF32 lsoli{A.U_new, A.g, c, {org[0], org[1], org[2], org[3]}};
        // eta_b (block noise, factor 0) and b = (D_b[U_old] - D_b[U_new]) eta
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            int l[4];
            local_coords(c, j, l);
            int x[4] = {org[0] + l[0], org[1] + l[1], org[2] + l[2], org[3] + l[3]};
            uint32_t s = (uint32_t)canon_index(A.g, x);
            Spinor<double> e;
#pragma unroll
            for (int k = 0; k < 12; ++k) e.c[k] = gaussian(s * 12u + k, DD_PURPOSE_BLOCK_NOISE, 0u, A.seed, A.ctr);
            eta.store(j, e);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<double> h1, h2;
            dirichlet_hop<double>(c, j, eta, lsrc, 0, h1);
            dirichlet_hop<double>(c, j, eta, lsol, 0, h2);
#pragma unroll
            for (int k = 0; k < 12; ++k) h1.c[k] = (-c.kappa) * (h1.c[k] - h2.c[k]);
            bv.store(j, h1);
        }
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
        while (rr > A.tol2 * bb && outer < kNoallocMaxCycles) {
            const double rn = sqrt(rr), rinv = 1.0 / rn;
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<double> v;
                rv.load(j, v);
#pragma unroll
                for (int k = 0; k < 12; ++k) v.c[k] = rinv * v.c[k];
                ri.store(j, v);
            }
            __syncthreads();
            block_cgnr<float>(c, xi, ri, pi, qi, zi, lsoli, kNoallocInnerTol, kNoallocInnerMaxit, sh);
            for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
                Spinor<double> a;
                Spinor<float> e;
                xv.load(j, a);
                xi.load(j, e);
#pragma unroll
                for (int k = 0; k < 12; ++k) a.c[k] = a.c[k] + rn * mk<double>((double)e.c[k].x, (double)e.c[k].y);
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
        // a block that missed tol_block, or went non-finite, reports NaN in
        // the caller's ln_b (the status word below is internal to the call)
        const bool failed = !isfinite(rr) || rr > A.tol2 * bb;
        if (threadIdx.x == 0) {
            if (!isfinite(rr)) raise_status(status, DD_ERR_NUMERIC);
            else if (rr > A.tol2 * bb) raise_status(status, DD_ERR_NOT_CONVERGED);
        }
        double s = 0.0;
        for (int j = threadIdx.x; j < c.nb; j += blockDim.x) {
            Spinor<double> e, d;
            eta.load(j, e);
            xv.load(j, d);
#pragma unroll
            for (int k = 0; k < 12; ++k) s += 2.0 * (e.c[k].x * d.c[k].x + e.c[k].y * d.c[k].y) + norm2(d.c[k]);
        }
        s = block_sum(s, sh);
        if (threadIdx.x == 0) A.ln_b[id] = (failed || !isfinite(s)) ? __longlong_as_double(0x7FF8000000000000LL) : -s;
        __syncthreads();
    }
}

// device address of the scratch array, looked up once per device
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[64] = {};
int g_noalloc_sms[64] = {};

}  // namespace

extern "C" int dd_block_ratios_noalloc(const int dims[4], const int block[4], double kappa, int bc_time,
                                       int colour_mask, const void* U_old, const void* U_new, uint64_t seed,
                                       uint64_t ctr, double tol_block, double* ln_b, void* stream) {
    if (!dims || !block || !U_old || !U_new || !ln_b || !(kappa > 0) || colour_mask < 1 || colour_mask > 3 ||
        (bc_time != 1 && bc_time != -1) || !(tol_block > 0))
        return DD_ERR_INVALID_ARG;
    Geo g;
    long long V = 1;
    for (int a = 0; a < 4; ++a) {
        if (dims[a] < 2 || (dims[a] & 1) || block[a] < 1 || dims[a] % block[a]) return DD_ERR_INVALID_ARG;
        int nbk = dims[a] / block[a];
        if (nbk < 2 || (nbk & 1)) return DD_ERR_INVALID_ARG;
        g.L[a] = dims[a];
        g.b[a] = block[a];
        g.nbk[a] = nbk;
        V *= dims[a];
    }
    if (V > (1LL << 30)) return DD_ERR_INVALID_ARG;
    if (12 * V > 0xFFFFFFFFLL) return DD_ERR_UNSUPPORTED;  // 32-bit noise element word (see dd_init)
    g.bc = bc_time;
    geo_finish(g);
    // one slot (FP64 eta, b, x, r and five FP32 inner vectors of one block) must fit
    const long long slot = (((long long)g.bsites * (4 * 192 + 5 * 96)) + 255) & ~255LL;
    const long long max_slots = (long long)(kNoallocScratchBytes - kNoallocHeader) / slot;
    if (max_slots < 1) return DD_ERR_UNSUPPORTED;  // block larger than the scratch array allows
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DD_ERR_CUDA;
    void* base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DD_ERR_CUDA;
            int n = 0;
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DD_ERR_CUDA;
            g_noalloc_addr[dev] = p;
            g_noalloc_sms[dev] = n;
        }
        base = g_noalloc_addr[dev];
        sms = g_noalloc_sms[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int half = g.nblocks / 2;
    const int nitems = colour_mask == 3 ? g.nblocks : half;
    NoallocArgs A;
    A.g = g;
    for (int a = 0; a < 4; ++a) A.c.bd[a] = g.b[a];
    A.c.st[0] = 1;
    A.c.st[1] = g.b[0];
    A.c.st[2] = g.b[0] * g.b[1];
    A.c.st[3] = g.b[0] * g.b[1] * g.b[2];
    A.c.nb = g.bsites;
    A.c.kappa = kappa;
    A.U_old = (const double*)U_old;
    A.U_new = (const double*)U_new;
    A.ln_b = ln_b;
    A.colour_mask = colour_mask;
    A.nitems = nitems;
    A.slot_bytes = slot;
    A.seed = seed;
    A.ctr = ctr;
    A.tol2 = tol_block * tol_block;
    // the queue head and status word must start at zero; blocks outside the
    // selected colours report 0
    if (cudaMemsetAsync(base, 0, kNoallocHeader, s) != cudaSuccess) return DD_ERR_CUDA;
    if (cudaMemsetAsync(ln_b, 0, sizeof(double) * g.nblocks, s) != cudaSuccess) return DD_ERR_CUDA;
    const int grid = (int)std::min<long long>(std::min<long long>(nitems, max_slots), 2LL * std::max(1, sms));
    noalloc_block_kernel<<<grid, 256, 0, s>>>(A);
    if (cudaGetLastError() != cudaSuccess) return DD_ERR_CUDA;
    return DD_OK;
}
