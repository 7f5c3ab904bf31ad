// Host-side handle and workspace plan of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/dd.h"
#include "dd_common.cuh"

// Per-system state of a batched Krylov solve, kept in device memory so that
// iterations run without host round trips.
struct CGState {
    double zz;     // |z|^2 = |A^dag r|^2
    double qq;     // |A p|^2
    double rr;     // |r|^2
    double alpha;  // step length
    double beta;   // direction update
    double tol2;   // stop when rr <= tol2
    int active;    // 1 while iterating
    int iters;     // iterations done
    int maxit;     // cap
    int flags;     // bit 0: hit maxit, bit 1: non-finite
    // complex scalars of BiCGStab
    double rho_re, rho_im, al_re, al_im, om_re, om_im, be_re, be_im;
};

// reduction finishers run by the last thread block of a reduction
enum FinOp {
    FIN_NONE = 0,
    FIN_STORE = 1,
    FIN_ALPHA = 2,
    FIN_RR = 3,
    FIN_BETA = 4,
    FIN_ZZ_INIT = 5,
    FIN_BI_RHO = 6,    // three values
    FIN_BI_ALPHA = 7,  // three values (third unused)
    FIN_BI_OMEGA = 8   // three values
};

struct Reduce {
    double* partials;     // [rhs][gridDim.x]
    unsigned* counters;   // [rhs]
    CGState* st;          // [rhs] (FIN_ALPHA / RR / BETA / ZZ_INIT)
    double* out;          // [rhs] (FIN_STORE)
    int op;
    int* status;
};

// One formatted copy of a gauge field.
struct FieldSlot {
    double2* eo64;   // eo layout, FP64, 9 chunks, [parity][dir][chunk][Vh]
    float4* eo32;    // eo layout, FP32 rows 0-1, 3 chunks
    uint2* eo16;     // eo layout, FP16 rows 0-1, 3 chunks
    double2* dd64;   // block order, FP64 [blockpos][dir][chunk][bsites]
    float4* dd32;    // block order, FP32 rows 0-1
    double2* canon;  // canonical FP64 copy (interpolated fields)
    float4* eodf;    // eo layout, double-float (hi, lo) pairs, 9 chunks (outer_prec DD_PREC_DF64 only)
};

// Vectors of one right-hand side of the global solver (eo layout, Vh sites).
struct SolverVecs {
    double2* be;   // FP64 even part of b (and b-tilde)
    double2* bo;   // FP64 odd part of b
    double2* xe;   // FP64 even solution
    double2* xo;   // FP64 odd solution
    double2* re;   // FP64 residual
    double2* t64;  // FP64 temporary (odd)
    double2* t64b; // FP64 temporary (even)
    double2* x64;  // FP64 inner vectors of the plain FP64 solver
    double2* p64;
    double2* q64;
    double2* z64;
    float4* x32;   // inner solution (correction)
    float4* r32;
    float4* p32;
    float4* q32;
    float4* z32;
    float4* t32;   // odd temporary (hop output)
    float4* w32;   // BiCGStab t
    float4* h32;   // BiCGStab shadow residual
    uint4* p16;    // FP16 hop copies + scales
    float* p16n;
    uint4* r16;
    float* r16n;
    uint4* t16;
    float* t16n;
    uint4* q16;
    float* q16n;
};

// Work vectors of the SAP-preconditioned GCR: `halves` holds FP32 half
// vectors (one parity of R systems, 6 chunks x Vh float4 each): 0 X_o,
// 1 R_o, 2-3 Y, 4-5 Q, 6 the odd part of a block correction, 7-11 the block
// solver's x, r, v, s, t, 12-15 its hop copies p, rhat, s, t (FP16 or FP32
// storage), then Z_0..Z_{nkv-1} and W_0..W_{nkv-1} (two halves each).
constexpr int DD_SAP_MAX_NKV = 16;
struct SapVecs {
    static constexpr int kFixedHalves = 16;
    float4* halves = nullptr;
    size_t half = 0;        // float4 per half vector
    int nkv = 0;
    double* partials = nullptr;
    int nblk = 0;           // thread blocks of a reduction over Vh sites
    double* sc = nullptr;   // per-system scalars
    float4* at(int k) const { return halves + (size_t)k * half; }
};

constexpr int DD_BLOCK_CTAS_MAX = 4;
// timed kernel kinds: whole-lattice hops 0 FP16 -> FP16, 1 FP16 -> FP32 (xpay),
// 2 FP64, 3 double-float residual; Dirichlet (block-restricted) hops 4 FP64,
// 5 FP16 -> FP16, 6 FP16 -> FP32 on the sites of one block colour; 7 the
// persistent block solver; 8 FP16 -> FP16, 9 FP16 -> FP32 Dirichlet hops over
// every site (both colours)
constexpr int DD_TIMER_KINDS = 10;
// device counters after the timer sites: items, inner iterations, outer
// cycles and site-iterations of the persistent block solver
constexpr int DD_BLOCK_STATS = 4;

// Launch shapes chosen by the autotuner (dd_autotune); defaults are the
// shapes the kernels were written for.
struct TuneConfig {
    int hop_tpb = 128, hop_spt = 1;      // FP16/FP32-storage hop kernels: threads, sites per thread
    int hop64_tpb = 128, hop64_spt = 1;  // FP64 hop kernels
    int block_tpb = 256, block_ctas_per_sm = 2;  // persistent block solver (at most DD_BLOCK_CTAS_MAX per SM)
    int filter_masked = 0;  // stochastic block filter: 0 persistent per-block kernel, 1 whole-lattice Dirichlet solves
    int tuned = 0;                       // bit 0: hops, bit 1: block solver
};

struct dd_handle {
    dd_params prm;
    Geo g;
    cudaStream_t stream;
    int n_active;                    // number of active links
    // device tables owned by the handle
    int* d_active_links = nullptr;   // canonical link indices 4*s + a of the active set, grouped
    std::vector<int> h_group_off;    // offsets of (colour, dir, parity) groups in d_active_links (17 entries)
    uint8_t* d_active_mask = nullptr;  // [V*4]
    int* d_status = nullptr;           // device status word
    unsigned long long* d_hb_fails = nullptr;
    // workspace
    char* ws = nullptr;
    size_t ws_size = 0;
    size_t ws_needed = 0;
    std::vector<FieldSlot> fields;   // max_rhs + 1 slots
    std::vector<SolverVecs> vecs;    // max_rhs systems
    double2* dd_vec = nullptr;       // block-ordered FP64 vectors: [6][max_rhs][12][V]
    CGState* d_cg = nullptr;         // [3 * max_rhs + 2]: inner, outer, SAP block-solver states
    SapVecs sap;                     // SAP-preconditioned GCR (krylov DD_KRYLOV_SAP_GCR)
    double* d_partials = nullptr;    // reduction partials
    unsigned* d_counters = nullptr;  // reduction tickets
    size_t partials_cap = 0;
    double* d_scalars = nullptr;     // scratch doubles [64 * max_rhs]
    char* block_scratch = nullptr;   // persistent block-solver slots
    size_t block_slot_bytes = 0;
    int block_slots = 0;
    double* d_item_out = nullptr;    // per-item results of the block kernel
    int* d_items = nullptr;          // item descriptors
    int* d_queue = nullptr;          // work-queue head
    int* d_imap = nullptr;           // small index maps: [nblocks] item bases, [2*max_rhs] field slots
    int items_cap = 0;
    double* d_lu = nullptr;          // dense matrices for the exact path
    bool lu_tensor = true;           // dense LU: trailing update on the tensor cores (Ozaki slices)
    double* d_gauge_g = nullptr;     // relative gauge fixing: one SU(3) matrix per site [V][18]
    size_t lu_bytes = 0;
    std::string last_error;
    int num_sms = 0;
    bool feat_solve = true, feat_estimate = true, feat_exact = true;  // planned workspace parts
    // instrumentation: kernels launched by this handle, and CUDA-event timing
    // of the even-odd hop kernels (kinds: 0 FP16 -> FP16, 1 FP16 -> FP32 with
    // xpay, 2 FP64), recorded on the handle's stream around every
    // timer_every-th launch of a kind
    unsigned long long launches = 0;
    int timer_on = 0;
    int timer_every = 1;
    unsigned long long timer_seen[DD_TIMER_KINDS] = {};
    std::vector<cudaEvent_t> timer_ev[DD_TIMER_KINDS];
    size_t timer_used[DD_TIMER_KINDS] = {};
    unsigned long long* d_sites = nullptr;  // [DD_TIMER_KINDS + DD_BLOCK_STATS] output sites of the timed launches,
                                            // then the block-solver counters
    // host counters of the polled (eager) defect-correction solves:
    // [0] whole-lattice solves, [1] Dirichlet solves; {solves, systems,
    // inner iterations, outer cycles, site-iterations}; launches of the
    // persistent block solver; reset with the timer
    long long solve_stats[2][5] = {};
    long long block_launches = 0;
    // even-odd indices of the sites of each block colour (null when the
    // block extent along axis 0 is odd); Dirichlet solves of one colour
    // visit only these
    int* d_colour_sites[2] = {nullptr, nullptr};
    // one level of recursion (dd_params.sub_block): geometry and colour
    // tables of the sub-blocks; LevelScope swaps them in for sub-block work
    bool has_sub = false;
    int active_mode = 0;  // resolved DD_ACTIVE_* of the smallest blocks
    Geo g2;
    int* d_colour_sites2[2] = {nullptr, nullptr};
    // graph capture (graph.cu): counter offset added by every kernel that
    // draws random numbers (0 outside graph replays), device loop counters
    // of captured solver loops, capture streams of loop bodies by depth
    unsigned long long* d_ctr_off = nullptr;
    int* d_loop = nullptr;  // [DD_LOOP_SLOTS]
    bool capturing = false;  // dd_graph_begin .. dd_graph_end
    cudaStream_t cap_stream = nullptr;   // private stream the capture runs on
    cudaStream_t user_stream = nullptr;  // the handle's stream, restored by dd_graph_end
    int loop_depth = 0;
    std::vector<cudaStream_t> body_streams;
    // last bytes uploaded per cached upload slot (upload_cached)
    std::vector<char> upload_cache[4];
    TuneConfig tune;
};

constexpr int DD_LOOP_SLOTS = 32;

// Makes the sub-block level the handle's block decomposition for the
// lifetime of the scope (kernels and solvers read h->g and the colour
// tables); a no-op when `sub` is false.
struct LevelScope {
    dd_handle* h;
    bool on;
    Geo saved;
    int* saved_cs[2];
    LevelScope(dd_handle* h_, bool sub) : h(h_), on(sub && h_->has_sub) {
        if (!on) return;
        saved = h->g;
        saved_cs[0] = h->d_colour_sites[0];
        saved_cs[1] = h->d_colour_sites[1];
        h->g = h->g2;
        h->d_colour_sites[0] = h->d_colour_sites2[0];
        h->d_colour_sites[1] = h->d_colour_sites2[1];
    }
    ~LevelScope() {
        if (!on) return;
        h->g = saved;
        h->d_colour_sites[0] = saved_cs[0];
        h->d_colour_sites[1] = saved_cs[1];
    }
    LevelScope(const LevelScope&) = delete;
    LevelScope& operator=(const LevelScope&) = delete;
};

// ----------------------------------------------------------- graph capture
// true while the handle's stream is being captured into a CUDA graph
bool dd_stream_capturing(dd_handle* h);
// Host -> device copy of a small descriptor table through cache slot
// `slot`: skipped when the same bytes were the last upload to dst; inside a
// capture a changed table is an error (DD_ERR_UNSUPPORTED).
int upload_cached(dd_handle* h, int slot, void* dst, const void* src, size_t bytes);
// Stopping rule of a device-side solver loop: continue while any st[k]
// (k < nrhs) is active, the body ran fewer than max_trips times and, when
// it_src is set, the running sum of it_src[k].iters stays below max_total;
// numeric = 1: a state with flag 2 raises DD_ERR_NUMERIC and stops.
struct LoopCond {
    const CGState* st;
    int nrhs;
    int max_trips;
    const CGState* it_src;
    long long max_total;
    int numeric;
};
// Runs body() repeatedly.  Eager: host_more() decides after every pass (it
// may synchronise and read device state).  Inside a capture: one conditional
// WHILE node whose body graph is body() followed by a kernel evaluating cond.
int dd_loop(dd_handle* h, const std::function<int()>& body, const std::function<int(bool&)>& host_more,
            const LoopCond& cond);

// Launch a kernel and count it: DD_KLAUNCH(h, kern<<<grid, block, 0, h->stream>>>(args));
#define DD_KLAUNCH(h, ...) ((__VA_ARGS__), ++(h)->launches)

// next timing event of a kind (pool grows on demand)
inline cudaEvent_t dd_timer_event(dd_handle* h, int kind) {
    auto& v = h->timer_ev[kind];
    if (h->timer_used[kind] == v.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        v.push_back(e);
    }
    return v[h->timer_used[kind]++];
}

// error plumbing
int dd_fail(dd_handle* h, int code, const std::string& msg);
int dd_cuda_check(dd_handle* h, cudaError_t e, const char* where);
#define DD_CUDA(h, call)                                        \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return dd_cuda_check(h, _e, #call); \
    } while (0)
#define DD_LAUNCH_CHECK(h, what)                                    \
    do {                                                            \
        cudaError_t _e = cudaGetLastError();                        \
        if (_e != cudaSuccess) return dd_cuda_check(h, _e, what);   \
    } while (0)

int dd_require_ws(dd_handle* h);
// DD_ERR_UNSUPPORTED unless the workspace was planned with the feature
inline int dd_require_feature(dd_handle* h, bool planned, const char* what) {
    return planned ? DD_OK : dd_fail(h, DD_ERR_UNSUPPORTED, std::string(what) + ": workspace planned without this feature");
}

// exact block log-determinant ratios of the block filter (lu.cu)
int block_filter_exact(dd_handle* h, const double* U_old, const double* U_new, int colour_mask, double* ln_b);

// shared launch helpers (defined in lattice.cu / solver.cu)
inline int grid_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

// field formatting (lattice.cu)
int format_field(dd_handle* h, const double* U, FieldSlot& f, bool eo64, bool eo32, bool eo16, bool dd64, bool dd32);
// spinor packing between canonical FP64 and eo FP64 (lattice.cu)
void launch_pack_spinor_eo(dd_handle* h, const double* in, double2* out, int parity, int nrhs, long long in_rhs_stride);
void launch_unpack_spinor_eo(dd_handle* h, const double2* in, double* out, int parity, int nrhs, long long out_rhs_stride);
void launch_pack_spinor_dd(dd_handle* h, const double* in, double2* out, int nrhs);
void launch_pack_spinor_sub(dd_handle* h, const double* in, double2* out, int nrhs);
void launch_unpack_spinor_sub(dd_handle* h, const double2* in, double* out, int nrhs);
void launch_unpack_spinor_dd(dd_handle* h, const double2* in, double* out, int nrhs);
