// Autotuner of the launch shapes: thread-block size and sites per thread of
// the even-odd hop kernels (FP16/FP32 storage and FP64), thread-block size
// and thread blocks per SM of the persistent block solver.  Each candidate
// is timed with CUDA events on the handle's stream on the handle's own
// lattice; the fastest is kept in the handle.  Results are cached per
// process and, when the environment variable DD_TUNE_CACHE names a file,
// in that file (one line per device and problem shape).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "dslash.cuh"

int tune_block_filter(dd_handle* h, const double* U_old, const double* U_new, int reps, float* ms);
int tune_block_filter_masked(dd_handle* h, const double* U_old, const double* U_new, int reps, float* ms);

namespace {

std::mutex g_tune_mu;
std::map<std::string, TuneConfig> g_tune_cache;

std::string tune_key(dd_handle* h) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, dev);
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s|%d|%dx%dx%dx%d|%dx%dx%dx%d|p%d|r%d", prop.name, prop.multiProcessorCount,
                  h->g.L[0], h->g.L[1], h->g.L[2], h->g.L[3], h->g.b[0], h->g.b[1], h->g.b[2], h->g.b[3],
                  h->prm.inner_prec, h->prm.max_rhs);
    std::string k(buf);
    for (char& c : k)
        if (c == ' ') c = '_';
    return k;
}

bool file_lookup(const std::string& key, TuneConfig& t) {
    const char* path = std::getenv("DD_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        char k[512];
        TuneConfig c;
        if (std::sscanf(line, "%511s %d %d %d %d %d %d %d", k, &c.hop_tpb, &c.hop_spt, &c.hop64_tpb, &c.hop64_spt,
                        &c.block_tpb, &c.block_ctas_per_sm, &c.filter_masked) == 8 &&
            key == k) {
            c.tuned = 3;
            t = c;
            found = true;  // the last line of a key wins
        }
    }
    std::fclose(f);
    return found;
}

void file_store(const std::string& key, const TuneConfig& t) {
    const char* path = std::getenv("DD_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %d %d %d\n", key.c_str(), t.hop_tpb, t.hop_spt, t.hop64_tpb, t.hop64_spt,
                 t.block_tpb, t.block_ctas_per_sm, t.filter_masked);
    std::fclose(f);
}

// average time of one launch of fn over reps launches (two untimed first)
template <class F>
float time_launches(dd_handle* h, int reps, F fn) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.f;
    }
    fn();
    fn();
    cudaEventRecord(e0, h->stream);
    for (int r = 0; r < reps; ++r) fn();
    cudaEventRecord(e1, h->stream);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess) {
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

struct Shape {
    int tpb, spt;
};
// thread-block size x sites per thread >= 64 keeps every grid within the
// reduction partials planned for 64-site tiles
const Shape kHopShapes[] = {{128, 1}, {64, 1}, {128, 2}, {64, 2}};
const Shape kHop64Shapes[] = {{128, 1}, {64, 1}};
const Shape kBlockShapes[] = {{256, 2}, {256, 1}, {128, 2}, {128, 4}, {64, 4}};

}  // namespace

extern "C" int dd_autotune(dd_t h, int what, const void* U_old, const void* U_new, int reps, dd_tune_report* rep) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    if (h->capturing || dd_stream_capturing(h)) return dd_fail(h, DD_ERR_UNSUPPORTED, "dd_autotune inside a capture");
    if (what & ~(DD_TUNE_HOP | DD_TUNE_BLOCK | DD_TUNE_NO_CACHE)) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_autotune: bad flags");
    if ((what & DD_TUNE_BLOCK) && (!U_old || !U_new || !h->feat_estimate))
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_autotune: block tuning needs U_old, U_new and the estimator workspace");
    if ((what & DD_TUNE_HOP) && !h->feat_solve) return dd_fail(h, DD_ERR_UNSUPPORTED, "dd_autotune: no solver workspace");
    if (reps < 1) reps = 20;
    dd_tune_report r;
    std::memset(&r, 0, sizeof(r));
    const std::string key = tune_key(h);
    TuneConfig cached;
    bool hit = false;
    if (!(what & DD_TUNE_NO_CACHE)) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            cached = it->second;
            hit = true;
        } else if (file_lookup(key, cached)) {
            g_tune_cache[key] = cached;
            hit = true;
        }
    }
    if (hit) {
        h->tune = cached;
        r.from_cache = 1;
    } else {
        const long long Vh = h->g.Vh;
        const int R = h->prm.max_rhs;
        SolverVecs& v = h->vecs[0];
        if (what & DD_TUNE_HOP) {
            // inputs: zero vectors (the timing does not depend on the values)
            DD_CUDA(h, cudaMemsetAsync(v.p16, 0, sizeof(uint4) * 3 * Vh * R, h->stream));
            DD_CUDA(h, cudaMemsetAsync(v.p16n, 0, sizeof(float) * Vh * R, h->stream));
            DD_CUDA(h, cudaMemsetAsync(v.x32, 0, sizeof(float4) * 6 * Vh * R, h->stream));
            DD_CUDA(h, cudaMemsetAsync(v.be, 0, sizeof(double2) * 12 * Vh * R, h->stream));
            DD_CUDA(h, cudaMemsetAsync(v.bo, 0, sizeof(double2) * 12 * Vh * R, h->stream));
            const double k2 = h->prm.kappa * h->prm.kappa;
            // the hop of the mixed inner solver: FP16 in, FP32 out with xpay
            HopArgs<SpinorF16, SpinorF32, SpinorF32, LinkF16> A;
            A.g = h->g;
            A.p = 0;
            A.in = SpinorF16{v.p16, v.p16n, Vh};
            A.xin = SpinorF32{v.x32, Vh};
            A.out = SpinorF32{v.p32, Vh};
            A.lk = LinkF16{h->fields[0].eo16, Vh};
            A.lk_rhs_stride = 0;
            A.a = 1.0;
            A.b = -k2;
            A.has_x = 1;
            A.g5in = A.g5out = 0;
            A.colour_mask = 3;
            A.st = nullptr;
            A.red.op = FIN_NONE;
            A.sites = nullptr;
            float best = 1e30f;
            TuneConfig keep = h->tune;
            for (const Shape& s : kHopShapes) {
                h->tune.hop_tpb = s.tpb;
                h->tune.hop_spt = s.spt;
                float ms = time_launches(h, reps, [&] { launch_hop<float, SpinorF16, SpinorF32, SpinorF32, LinkF16, 0>(A, R, h); });
                if (ms < 0) return dd_fail(h, DD_ERR_CUDA, "dd_autotune: hop timing failed");
                if (s.tpb == 128 && s.spt == 1) r.hop_default_ms = ms;
                if (ms < best) {
                    best = ms;
                    keep.hop_tpb = s.tpb;
                    keep.hop_spt = s.spt;
                }
            }
            r.hop_ms = best;
            // FP64 hop of the defect-correction residual
            HopArgs<SpinorF64, SpinorF64, SpinorF64, LinkF64> B;
            B.g = h->g;
            B.p = 0;
            B.in = SpinorF64{v.bo, Vh};
            B.xin = SpinorF64{v.be, Vh};
            B.out = SpinorF64{v.xe, Vh};
            B.lk = LinkF64{h->fields[0].eo64, Vh};
            B.lk_rhs_stride = 0;
            B.a = 1.0;
            B.b = -k2;
            B.has_x = 1;
            B.g5in = B.g5out = 0;
            B.colour_mask = 3;
            B.st = nullptr;
            B.red.op = FIN_NONE;
            B.sites = nullptr;
            best = 1e30f;
            for (const Shape& s : kHop64Shapes) {
                h->tune.hop64_tpb = s.tpb;
                h->tune.hop64_spt = s.spt;
                float ms = time_launches(h, std::max(2, reps / 4), [&] {
                    launch_hop<double, SpinorF64, SpinorF64, SpinorF64, LinkF64, 0>(B, R, h);
                });
                if (ms < 0) return dd_fail(h, DD_ERR_CUDA, "dd_autotune: FP64 hop timing failed");
                if (s.tpb == 128 && s.spt == 1) r.hop64_default_ms = ms;
                if (ms < best) {
                    best = ms;
                    keep.hop64_tpb = s.tpb;
                    keep.hop64_spt = s.spt;
                }
            }
            r.hop64_ms = best;
            keep.tuned |= 1;
            h->tune = keep;
        }
        if (what & DD_TUNE_BLOCK) {
            float best = 1e30f;
            TuneConfig keep = h->tune;
            for (const Shape& s : kBlockShapes) {
                h->tune.block_tpb = s.tpb;
                h->tune.block_ctas_per_sm = s.spt;
                float ms = -1.f;
                rc = tune_block_filter(h, (const double*)U_old, (const double*)U_new, std::max(1, reps / 10), &ms);
                if (rc) {
                    h->tune = keep;
                    return rc;
                }
                if (s.tpb == 256 && s.spt == 2) r.block_default_ms = ms;
                if (ms < best) {
                    best = ms;
                    keep.block_tpb = s.tpb;
                    keep.block_ctas_per_sm = s.spt;
                }
            }
            // the same filter as batched whole-lattice Dirichlet solves
            float msm = -1.f;
            rc = tune_block_filter_masked(h, (const double*)U_old, (const double*)U_new, std::max(1, reps / 10), &msm);
            if (rc) {
                h->tune = keep;
                return rc;
            }
            r.filter_masked_ms = msm;
            keep.filter_masked = msm < best ? 1 : 0;
            r.block_ms = best;
            keep.tuned |= 2;
            h->tune = keep;
        }
        if (!(what & DD_TUNE_NO_CACHE) && (h->tune.tuned & 3) == 3) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[key] = h->tune;
            file_store(key, h->tune);
        }
    }
    r.hop_tpb = h->tune.hop_tpb;
    r.hop_spt = h->tune.hop_spt;
    r.hop64_tpb = h->tune.hop64_tpb;
    r.hop64_spt = h->tune.hop64_spt;
    r.block_tpb = h->tune.block_tpb;
    r.block_ctas_per_sm = h->tune.block_ctas_per_sm;
    r.filter_masked = h->tune.filter_masked;
    if (rep) *rep = r;
    return DD_OK;
}

extern "C" int dd_set_tuning(dd_t h, int hop_tpb, int hop_spt, int hop64_tpb, int hop64_spt, int block_tpb,
                             int block_ctas_per_sm, int filter_masked) {
    if (!h) return DD_ERR_INVALID_ARG;
    auto ok_shape = [](int tpb, int spt, int max_tpb) {
        return (tpb == 64 || tpb == 128 || tpb == 256) && tpb <= max_tpb && (spt == 1 || spt == 2);
    };
    if (!ok_shape(hop_tpb, hop_spt, 128) || !ok_shape(hop64_tpb, hop64_spt, 128) || hop64_spt != 1 ||
        !(block_tpb == 64 || block_tpb == 128 || block_tpb == 256) || block_ctas_per_sm < 1 ||
        block_ctas_per_sm > DD_BLOCK_CTAS_MAX || (filter_masked != 0 && filter_masked != 1))
        return dd_fail(h, DD_ERR_INVALID_ARG, "dd_set_tuning: shape out of range");
    h->tune.hop_tpb = hop_tpb;
    h->tune.hop_spt = hop_spt;
    h->tune.hop64_tpb = hop64_tpb;
    h->tune.hop64_spt = hop64_spt;
    h->tune.block_tpb = block_tpb;
    h->tune.block_ctas_per_sm = block_ctas_per_sm;
    h->tune.filter_masked = filter_masked;
    return DD_OK;
}
