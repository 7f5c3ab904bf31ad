// Exact check path (Sec. 3: the block determinants are obtained exactly from
// an LU factorisation; Eq. ddfactor for the Schur complement): dense FP64
// complex LU with partial pivoting on the GPU, giving ln|det| of
//   D      the whole Wilson-Dirac operator (12V x 12V),
//   D_b    every Dirichlet block operator (batched),
//   Dhat   the domain Schur complement 1 - A^{-1} B E^{-1} C, assembled
//          explicitly with block-diagonal solves and a dense product.
// Right-looking elimination, one pivot launch and one trailing-update launch
// per column (batched over matrices); matrices are column-major.  FP64
// arithmetic on the FP64 FMA pipe: on GB300 the FP64 tensor-core instruction
// (mma.sync m8n8k4) measures 1.10 TFLOP/s against 1.25 for FP64 FMA
// (dd_alu_peaks), so the trailing update gains nothing from it.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dd_internal.h"
#include "su3.cuh"

namespace {

// ------------------------------------------------------------ dense fills
// 4x4 spin matrix (1 - sgn*gamma_a) entry (s, t), built from the spin projector
DD_DEV cpx<double> spin_proj(int a, int sgn, int s, int t) {
    Spinor<double> in, out;
    zero(in);
    zero(out);
    in.c[t * 3] = mk<double>(1.0, 0.0);
    Half<double> hf;
    project<double>(a, sgn, in, hf);
    accumulate<double>(a, sgn, hf, 1.0, out);
    return out.c[s * 3];
}

// D (or the intra-block part of D) as a dense column-major matrix.
// Row / column of site s, spin, colour = 12 * pos(s) + 3 * spin + colour with
// pos = canonical index (order 0), block-order position (order 1), or the
// local index inside the block, matrix = block id (order 2, blocks only).
__global__ void fill_dense_kernel(Geo g, const double* __restrict__ U, double kappa, double2* M, int order, int n,
                                  long long mstride) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x[4];
    canon_coords(g, s, x);
    const int bid = block_id_of(g, x);
    auto pos_of = [&](const int* y, int* mat) -> long long {
        *mat = 0;
        if (order == 0) return canon_index(g, y);
        if (order == 1) return dd_position(g, y);
        *mat = block_id_of(g, y);
        return local_index_of(g, y);
    };
    int mat;
    const long long ps = pos_of(x, &mat);
    double2* A = M + (long long)mat * mstride;
    for (int k = 0; k < 12; ++k) A[(12 * ps + k) + (12 * ps + k) * (long long)n] = make_double2(1.0, 0.0);
    for (int a = 0; a < 4; ++a) {
        for (int dir = +1; dir >= -1; dir -= 2) {
            int y[4] = {x[0], x[1], x[2], x[3]};
            y[a] += dir;
            if (y[a] == g.L[a]) y[a] = 0;
            if (y[a] < 0) y[a] = g.L[a] - 1;
            if (order == 2 && block_id_of(g, y) != bid) continue;
            int m2;
            const long long py = pos_of(y, &m2);
            double sc = -kappa;
            if (a == 3 && ((dir > 0 && x[3] == g.L[3] - 1) || (dir < 0 && x[3] == 0))) sc *= g.bc;
            const int ys = canon_index(g, y);
            const double* lp = U + ((long long)(dir > 0 ? s : ys) * 4 + a) * 18;
            for (int sp = 0; sp < 4; ++sp)
                for (int tp = 0; tp < 4; ++tp) {
                    cpx<double> gm = spin_proj(a, dir, sp, tp);
                    if (gm.x == 0.0 && gm.y == 0.0) continue;
                    for (int c = 0; c < 3; ++c)
                        for (int d = 0; d < 3; ++d) {
                            cpx<double> u = dir > 0 ? mk<double>(lp[2 * (3 * c + d)], lp[2 * (3 * c + d) + 1])
                                                    : mk<double>(lp[2 * (3 * d + c)], -lp[2 * (3 * d + c) + 1]);
                            cpx<double> v = sc * cmul(gm, u);
                            long long r = 12 * ps + 3 * sp + c, col = 12 * py + 3 * tp + d;
                            double2& e = A[r + col * (long long)n];
                            e.x += v.x;
                            e.y += v.y;
                        }
                }
        }
    }
}

__global__ void zero_kernel(long long n, double2* p) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = make_double2(0.0, 0.0);
}

// ------------------------------------------------------- LU elimination
// Step k on a batch of n x ncols matrices (column-major, leading dim n):
// pivot search in column k (rows k..n-1), row swap over all columns,
// ln|pivot| accumulated, multipliers stored below the diagonal.
__global__ void lu_pivot_kernel(double2* M, long long mstride, int n, int ncols, int k, double* logdet,
                                int* status) {
    __shared__ double sv[256];
    __shared__ int si[256];
    double2* A = M + (long long)blockIdx.x * mstride;
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        double2 v = A[i + (long long)k * n];
        double m = v.x * v.x + v.y * v.y;
        if (m > best) {
            best = m;
            bi = i;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double o = sv[threadIdx.x + s];
            int oi = si[threadIdx.x + s];
            if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = o;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int p = si[0];
    if (p != k)
        for (int j = threadIdx.x; j < ncols; j += blockDim.x) {
            double2 t = A[k + (long long)j * n];
            A[k + (long long)j * n] = A[p + (long long)j * n];
            A[p + (long long)j * n] = t;
        }
    __syncthreads();
    const double2 piv = A[k + (long long)k * n];
    const double pm = piv.x * piv.x + piv.y * piv.y;
    if (threadIdx.x == 0) {
        if (!(pm > 0.0)) raise_status(status, DD_ERR_NUMERIC);
        logdet[blockIdx.x] += 0.5 * log(pm);
    }
    if (pm > 0.0) {
        const cpx<double> inv = mk<double>(piv.x / pm, -piv.y / pm);
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double2 v = A[i + (long long)k * n];
            cpx<double> w = cmul(mk<double>(v.x, v.y), inv);
            A[i + (long long)k * n] = make_double2(w.x, w.y);
        }
    }
}

// trailing update a_ij -= l_ik u_kj for i > k, k < j < ncols
__global__ void lu_update_kernel(double2* M, long long mstride, int n, int ncols, int k) {
    __shared__ double2 lcol[16];
    __shared__ double2 urow[16];
    double2* A = M + (long long)blockIdx.z * mstride;
    const int i = k + 1 + blockIdx.y * 16 + threadIdx.y;
    const int j = k + 1 + blockIdx.x * 16 + threadIdx.x;
    if (threadIdx.x == 0) lcol[threadIdx.y] = (i < n) ? A[i + (long long)k * n] : make_double2(0, 0);
    if (threadIdx.y == 0) urow[threadIdx.x] = (j < ncols) ? A[k + (long long)j * n] : make_double2(0, 0);
    __syncthreads();
    if (i < n && j < ncols) {
        double2 l = lcol[threadIdx.y], u = urow[threadIdx.x];
        double2& a = A[i + (long long)j * n];
        a.x -= l.x * u.x - l.y * u.y;
        a.y -= l.x * u.y + l.y * u.x;
    }
}

// back substitution on the right-hand-side columns nelim..ncols-1 of an
// eliminated augmented matrix [U | Y]: step k (descending) scales row k and
// eliminates it from the rows above
__global__ void back_scale_kernel(double2* M, long long mstride, int n, int ncols, int k) {
    double2* A = M + (long long)blockIdx.y * mstride;
    int j = n + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    double2 piv = A[k + (long long)k * n];
    double pm = piv.x * piv.x + piv.y * piv.y;
    cpx<double> inv = mk<double>(piv.x / pm, -piv.y / pm);
    double2 v = A[k + (long long)j * n];
    cpx<double> w = cmul(mk<double>(v.x, v.y), inv);
    A[k + (long long)j * n] = make_double2(w.x, w.y);
}
__global__ void back_update_kernel(double2* M, long long mstride, int n, int ncols, int k) {
    double2* A = M + (long long)blockIdx.z * mstride;
    int i = blockIdx.y * blockDim.y + threadIdx.y;
    int j = n + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k || j >= ncols) return;
    double2 u = A[i + (long long)k * n], x = A[k + (long long)j * n];
    double2& a = A[i + (long long)j * n];
    a.x -= u.x * x.x - u.y * x.y;
    a.y -= u.x * x.y + u.y * x.x;
}

// C (m x n, ld ldc) = alpha * A (m x kk, lda) * B (kk x n, ldb) + beta * C, complex FP64
__global__ void zgemm_kernel(int m, int nn, int kk, const double2* A, int lda, const double2* B, int ldb, double2* C,
                             int ldc, double alpha, double beta) {
    __shared__ double2 As[16][17];
    __shared__ double2 Bs[16][17];
    int r = blockIdx.y * 16 + threadIdx.y, c = blockIdx.x * 16 + threadIdx.x;
    double sr = 0, si = 0;
    for (int t = 0; t < kk; t += 16) {
        As[threadIdx.y][threadIdx.x] = (r < m && t + threadIdx.x < kk) ? A[r + (long long)(t + threadIdx.x) * lda]
                                                                        : make_double2(0, 0);
        Bs[threadIdx.y][threadIdx.x] = (c < nn && t + threadIdx.y < kk) ? B[(t + threadIdx.y) + (long long)c * ldb]
                                                                         : make_double2(0, 0);
        __syncthreads();
        for (int q = 0; q < 16; ++q) {
            double2 a = As[threadIdx.y][q], b = Bs[q][threadIdx.x];
            sr += a.x * b.x - a.y * b.y;
            si += a.x * b.y + a.y * b.x;
        }
        __syncthreads();
    }
    if (r < m && c < nn) {
        double2& o = C[r + (long long)c * ldc];
        o = make_double2(alpha * sr + beta * o.x, alpha * si + beta * o.y);
    }
}

// copy a sub-matrix (rows r0.., cols c0.., size rm x cm) of S (ld lds) into D (ld ldd) at (0, dc)
__global__ void copy_sub_kernel(const double2* S, int lds, int r0, int c0, int rm, int cm, double2* Dm, int ldd,
                                int dc, double scale, int add_identity) {
    int i = blockIdx.y * blockDim.y + threadIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rm || j >= cm) return;
    double2 v = S[(r0 + i) + (long long)(c0 + j) * lds];
    v.x *= scale;
    v.y *= scale;
    if (add_identity && i == j) v.x += 1.0;
    Dm[i + (long long)(dc + j) * ldd] = v;
}

__global__ void zero_doubles_kernel(int n, double* p) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.0;
}

}  // namespace

// LU of `batch` n x ncols matrices, eliminating the first n columns; logdet
// receives sum_k ln|u_kk| per matrix; with back = true the right-hand-side
// columns are overwritten by the solutions.
static int lu_batched(dd_handle* h, double2* M, long long mstride, int batch, int n, int ncols, double* logdet,
                      bool back) {
    DD_KLAUNCH(h, zero_doubles_kernel<<<grid_for(batch, 64), 64, 0, h->stream>>>(batch, logdet));
    for (int k = 0; k < n; ++k) {
        DD_KLAUNCH(h, lu_pivot_kernel<<<batch, 256, 0, h->stream>>>(M, mstride, n, ncols, k, logdet, h->d_status));
        int rows = n - k - 1, cols = ncols - k - 1;
        if (rows > 0 && cols > 0) {
            dim3 grid((cols + 15) / 16, (rows + 15) / 16, batch);
            DD_KLAUNCH(h, lu_update_kernel<<<grid, dim3(16, 16), 0, h->stream>>>(M, mstride, n, ncols, k));
        }
    }
    if (back && ncols > n) {
        for (int k = n - 1; k >= 0; --k) {
            dim3 g1(grid_for(ncols - n, 128), batch);
            DD_KLAUNCH(h, back_scale_kernel<<<g1, 128, 0, h->stream>>>(M, mstride, n, ncols, k));
            if (k > 0) {
                dim3 g2(grid_for(ncols - n, 16), grid_for(k, 16), batch);
                DD_KLAUNCH(h, back_update_kernel<<<g2, dim3(16, 16), 0, h->stream>>>(M, mstride, n, ncols, k));
            }
        }
    }
    DD_LAUNCH_CHECK(h, "lu_batched");
    return DD_OK;
}

static int fill(dd_handle* h, const double* U, double2* M, int order, int n, long long mstride, int nmat) {
    long long tot = (long long)nmat * mstride;
    DD_KLAUNCH(h, zero_kernel<<<grid_for(tot, 256), 256, 0, h->stream>>>(tot, M));
    DD_KLAUNCH(h, fill_dense_kernel<<<grid_for(h->g.V, 64), 64, 0, h->stream>>>(h->g, U, h->prm.kappa, M, order, n, mstride));
    DD_LAUNCH_CHECK(h, "fill_dense_kernel");
    return DD_OK;
}

// ln|det D_b| for every block (by block id) into out
static int logdet_blocks(dd_handle* h, const double* U, double* out) {
    const int nb12 = 12 * h->g.bsites;
    const long long ms = (long long)nb12 * nb12;
    if (h->g.bsites > 256 || !h->d_lu) return dd_fail(h, DD_ERR_UNSUPPORTED, "exact block determinants need blocks of <= 256 sites");
    double2* M = (double2*)h->d_lu;
    int rc = fill(h, U, M, 2, nb12, ms, h->g.nblocks);
    if (rc) return rc;
    return lu_batched(h, M, ms, h->g.nblocks, nb12, nb12, out, false);
}

static int logdet_full(dd_handle* h, const double* U, double* out) {
    const int n = 12 * h->g.V;
    if (h->g.V > 512 || !h->d_lu) return dd_fail(h, DD_ERR_UNSUPPORTED, "exact determinant of D needs V <= 512");
    double2* M = (double2*)h->d_lu;
    int rc = fill(h, U, M, 0, n, (long long)n * n, 1);
    if (rc) return rc;
    return lu_batched(h, M, 0, 1, n, n, out, false);
}

// Dhat = 1 - A^{-1} B E^{-1} C from D in block order, then its LU
static int logdet_schur(dd_handle* h, const double* U, double* out) {
    const int n = 12 * h->g.V, nh = n / 2, nb12 = 12 * h->g.bsites, nbk = h->g.nblocks / 2;
    if (h->g.V > 512 || !h->d_lu) return dd_fail(h, DD_ERR_UNSUPPORTED, "exact determinant of Dhat needs V <= 512");
    double2* D = (double2*)h->d_lu;                  // n x n, block order
    double2* aug = D + (long long)n * n;             // nbk matrices nb12 x (nb12 + nh)
    const long long as = (long long)nb12 * (nb12 + nh);
    double2* Y = aug + (long long)nbk * as;          // nh x nh
    double2* Dh = Y + (long long)nh * nh;            // nh x nh
    double* ld = h->d_scalars;                       // scratch logdets
    int rc = fill(h, U, D, 1, n, (long long)n * n, 1);
    if (rc) return rc;
    dim3 b16(16, 16);
    // X = E^{-1} C: per white block [E_b | C_b]
    for (int b = 0; b < nbk; ++b) {
        int r0 = nh + b * nb12;
        dim3 gE(grid_for(nb12, 16), grid_for(nb12, 16)), gC(grid_for(nh, 16), grid_for(nb12, 16));
        DD_KLAUNCH(h, copy_sub_kernel<<<gE, b16, 0, h->stream>>>(D, n, r0, r0, nb12, nb12, aug + b * as, nb12, 0, 1.0, 0));
        DD_KLAUNCH(h, copy_sub_kernel<<<gC, b16, 0, h->stream>>>(D, n, r0, 0, nb12, nh, aug + b * as, nb12, nb12, 1.0, 0));
    }
    rc = lu_batched(h, aug, as, nbk, nb12, nb12 + nh, ld, true);
    if (rc) return rc;
    // Y = B X: B = D[0:nh, nh:n]; X rows of white block b live in aug b, columns nb12..
    for (int b = 0; b < nbk; ++b) {
        dim3 g(grid_for(nh, 16), grid_for(nh, 16));
        DD_KLAUNCH(h, zgemm_kernel<<<g, b16, 0, h->stream>>>(nh, nh, nb12, D + (long long)(nh + b * nb12) * n, n,
                                                           aug + b * as + (long long)nb12 * nb12, nb12, Y, nh, 1.0,
                                                           b == 0 ? 0.0 : 1.0));
    }
    // Z = A^{-1} Y: per black block [A_b | Y_b]
    for (int b = 0; b < nbk; ++b) {
        int r0 = b * nb12;
        dim3 gA(grid_for(nb12, 16), grid_for(nb12, 16)), gY(grid_for(nh, 16), grid_for(nb12, 16));
        DD_KLAUNCH(h, copy_sub_kernel<<<gA, b16, 0, h->stream>>>(D, n, r0, r0, nb12, nb12, aug + b * as, nb12, 0, 1.0, 0));
        DD_KLAUNCH(h, copy_sub_kernel<<<gY, b16, 0, h->stream>>>(Y, nh, r0, 0, nb12, nh, aug + b * as, nb12, nb12, 1.0, 0));
    }
    rc = lu_batched(h, aug, as, nbk, nb12, nb12 + nh, ld, true);
    if (rc) return rc;
    // Dhat = 1 - Z
    for (int b = 0; b < nbk; ++b) {
        dim3 g(grid_for(nh, 16), grid_for(nb12, 16));
        DD_KLAUNCH(h, copy_sub_kernel<<<g, b16, 0, h->stream>>>(aug + b * as + (long long)nb12 * nb12, nb12, 0, 0, nb12,
                                                              nh, Dh + b * nb12, nh, 0, -1.0, 0));
    }
    // identity: add 1 on the diagonal (rows b*nb12.. of column block b)
    {
        dim3 g(grid_for(nh, 16), grid_for(nh, 16));
        DD_KLAUNCH(h, copy_sub_kernel<<<g, b16, 0, h->stream>>>(Dh, nh, 0, 0, nh, nh, Dh, nh, 0, 1.0, 1));
    }
    return lu_batched(h, Dh, 0, 1, nh, nh, out, false);
}

__global__ void block_ratio_kernel(Geo g, int colour_mask, const double* ld_old, const double* ld_new, double* ln_b) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= g.nblocks) return;
    int B[4] = {b % g.nbk[0], (b / g.nbk[0]) % g.nbk[1], (b / (g.nbk[0] * g.nbk[1])) % g.nbk[2],
                b / (g.nbk[0] * g.nbk[1] * g.nbk[2])};
    int col = (B[0] + B[1] + B[2] + B[3]) & 1;
    ln_b[b] = ((colour_mask >> col) & 1) ? 2.0 * (ld_new[b] - ld_old[b]) : 0.0;
}

int block_filter_exact(dd_handle* h, const double* U_old, const double* U_new, int colour_mask, double* ln_b) {
    double* ld_old = h->d_item_out;
    double* ld_new = h->d_item_out + h->g.nblocks;
    int rc = logdet_blocks(h, U_old, ld_old);
    if (rc) return rc;
    rc = logdet_blocks(h, U_new, ld_new);
    if (rc) return rc;
    DD_KLAUNCH(h, block_ratio_kernel<<<grid_for(h->g.nblocks, 64), 64, 0, h->stream>>>(h->g, colour_mask, ld_old, ld_new, ln_b));
    DD_LAUNCH_CHECK(h, "block_ratio_kernel");
    return DD_OK;
}

extern "C" int dd_logdet_exact(dd_t h, const void* U, int which, double* out) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_exact, "dd_logdet_exact");
    if (rc) return rc;
    if (!U || !out) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_logdet_exact: bad arguments");
    if (which == 0) return logdet_full(h, (const double*)U, out);
    if (which == 1) return logdet_blocks(h, (const double*)U, out);
    if (which == 2) return logdet_schur(h, (const double*)U, out);
    return dd_fail(h, DD_ERR_INVALID_ARG, "dd_logdet_exact: which must be 0, 1 or 2");
}
