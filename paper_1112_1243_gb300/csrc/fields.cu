// Field-level kernels: Gaussian noise (Sec. 4), the geodesic interpolation
// of active links (Eq. param) and the mean plaquette.
#include <cmath>

#include "dd_internal.h"
#include "reduce.cuh"
#include "su3.cuh"

// ------------------------------------------------------------------- noise
__global__ void noise_kernel(long long V, double* out, int purpose, uint64_t seed, uint64_t ctr0,
                             const unsigned long long* ctr_off) {
    const uint64_t ctr = stream_ctr(ctr0, ctr_off);
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // element = s*12 + k
    int r = blockIdx.y;
    if (e >= V * 12) return;
    cpx<double> z = gaussian((uint32_t)e, (uint32_t)purpose, (uint32_t)r, seed, ctr);
    double* o = out + ((long long)r * V * 12 + e) * 2;
    o[0] = z.x;
    o[1] = z.y;
}

extern "C" int dd_noise(dd_t h, void* eta, int nrhs, int purpose, uint64_t seed, uint64_t ctr) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    if (!eta || nrhs < 1 || purpose < 0 || purpose > 255) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_noise: bad arguments");
    const long long n = (long long)h->g.V * 12;
    dim3 grid(grid_for(n, 256), nrhs);
    DD_KLAUNCH(h, noise_kernel<<<grid, 256, 0, h->stream>>>(h->g.V, (double*)eta, purpose, seed, ctr, h->d_ctr_off));
    DD_LAUNCH_CHECK(h, "noise_kernel");
    return DD_OK;
}

// ---------------------------------------------------------- interpolation
// U_t = U (U^dag U')^t on active links, t = num/den; other links copied.
__global__ void interpolate_kernel(long long nlinks, const double* __restrict__ U, const double* __restrict__ Up,
                                   const uint8_t* __restrict__ active, double* out, int num, int den) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlinks) return;
    const double* a = U + l * 18;
    const double* b = Up + l * 18;
    double* o = out + l * 18;
    if ((active && !active[l]) || num == 0) {
        for (int k = 0; k < 18; ++k) o[k] = a[k];
        return;
    }
    if (num == den) {
        for (int k = 0; k < 18; ++k) o[k] = b[k];
        return;
    }
    // an unchanged link (e.g. in a rejected block) stays on the path: W = 1, W^t = 1
    bool same = true;
    for (int k = 0; k < 18; ++k) same = same && (a[k] == b[k]);
    if (same) {
        for (int k = 0; k < 18; ++k) o[k] = a[k];
        return;
    }
    M3 u = load_m3(a), up = load_m3(b);
    M3 w = mul_dag_left(u, up);  // U^dag U'
    M3 wt = su3_power(w, (double)num / (double)den);
    store_m3(o, mul(u, wt));
}

// Every slot k = 0 .. nslots - 1 of one chain U_{k/den} (slot k at out +
// k * slot_stride doubles): the eigen-decomposition of U^dag U' is computed
// once per link for all slots.
__global__ void interpolate_slots_kernel(long long nlinks, const double* __restrict__ U, const double* __restrict__ Up,
                                         const uint8_t* __restrict__ active, double* out, long long slot_stride,
                                         int nslots, int den) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlinks) return;
    const double* a = U + l * 18;
    const double* b = Up + l * 18;
    bool same = true;
    for (int k = 0; k < 18; ++k) same = same && (a[k] == b[k]);
    if ((active && !active[l]) || same) {
        for (int s = 0; s < nslots; ++s) {
            const double* src = (s == den && !(active && !active[l])) ? b : a;
            double* o = out + s * slot_stride + l * 18;
            for (int k = 0; k < 18; ++k) o[k] = src[k];
        }
        return;
    }
    M3 u = load_m3(a), up = load_m3(b);
    M3 V;
    double th[3];
    su3_eig(mul_dag_left(u, up), V, th);
    for (int s = 0; s < nslots; ++s) {
        double* o = out + s * slot_stride + l * 18;
        if (s == 0) {
            for (int k = 0; k < 18; ++k) o[k] = a[k];
        } else if (s == den) {
            for (int k = 0; k < 18; ++k) o[k] = b[k];
        } else {
            store_m3(o, mul(u, su3_power_eig(V, th, (double)s / (double)den)));
        }
    }
}

int launch_interpolate_slots(dd_handle* h, const double* U, const double* Up, double* out, long long slot_stride,
                             int nslots, int den, bool all_links) {
    const long long n = (long long)h->g.V * 4;
    DD_KLAUNCH(h, interpolate_slots_kernel<<<grid_for(n, 128), 128, 0, h->stream>>>(
                      n, U, Up, all_links ? nullptr : h->d_active_mask, out, slot_stride, nslots, den));
    DD_LAUNCH_CHECK(h, "interpolate_slots_kernel");
    return DD_OK;
}

// all_links: interpolate every link that differs (after a relative gauge
// fixing), else the active links only (the rest is taken from U)
int launch_interpolate(dd_handle* h, const double* U, const double* Up, double* out, int num, int den,
                       bool all_links) {
    const long long n = (long long)h->g.V * 4;
    DD_KLAUNCH(h, interpolate_kernel<<<grid_for(n, 128), 128, 0, h->stream>>>(n, U, Up, all_links ? nullptr : h->d_active_mask,
                                                                              out, num, den));
    DD_LAUNCH_CHECK(h, "interpolate_kernel");
    return DD_OK;
}

extern "C" int dd_interpolate(dd_t h, void* U_t, const void* U, const void* U_new, int i, int n) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    if (!U_t || !U || !U_new || n < 1 || i < 0 || i > n) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_interpolate: bad arguments");
    return launch_interpolate(h, (const double*)U, (const double*)U_new, (double*)U_t, i, n, false);
}

// ---------------------------------------------------------------- plaquette
__global__ void __launch_bounds__(128) plaquette_kernel(Geo g, const double* __restrict__ U, Reduce red) {
    __shared__ double sh[34];
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (s < g.V) {
        int x[4];
        canon_coords(g, s, x);
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) {
                int sa = shift_index(g, x, a, +1), sb = shift_index(g, x, b, +1);
                M3 u1 = load_m3(U + ((long long)s * 4 + a) * 18);
                M3 u2 = load_m3(U + ((long long)sa * 4 + b) * 18);
                M3 u3 = load_m3(U + ((long long)sb * 4 + a) * 18);
                M3 u4 = load_m3(U + ((long long)s * 4 + b) * 18);
                M3 p = mul_dag_right(mul(u1, u2), mul(u4, u3));  // u1 u2 (u4 u3)^dag = u1 u2 u3^dag u4^dag
                acc += p.m[0][0].x + p.m[1][1].x + p.m[2][2].x;
            }
    }
    grid_reduce(red, 0, acc, sh);
}
__global__ void plaquette_scale_kernel(double* out, double inv) { out[0] *= inv; }

extern "C" int dd_plaquette(dd_t h, const void* U, double* out) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    if (!U || !out) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_plaquette: bad arguments");
    Reduce R_;
    R_.partials = h->d_partials;
    R_.counters = h->d_counters;
    R_.st = nullptr;
    R_.out = out;
    R_.op = FIN_STORE;
    R_.status = h->d_status;
    DD_KLAUNCH(h, plaquette_kernel<<<grid_for(h->g.V, 128), 128, 0, h->stream>>>(h->g, (const double*)U, R_));
    DD_KLAUNCH(h, plaquette_scale_kernel<<<1, 1, 0, h->stream>>>(out, 1.0 / (18.0 * h->g.V)));
    DD_LAUNCH_CHECK(h, "plaquette_kernel");
    return DD_OK;
}
