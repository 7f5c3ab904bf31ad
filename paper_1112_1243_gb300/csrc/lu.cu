// Exact check path (Sec. 3: the block determinants are obtained exactly from
// an LU factorisation; Eq. ddfactor for the Schur complement): dense FP64
// complex LU with partial pivoting on the GPU, giving ln|det| of
//   D      the whole Wilson-Dirac operator (12V x 12V),
//   D_b    every Dirichlet block operator (batched),
//   Dhat   the domain Schur complement 1 - A^{-1} B E^{-1} C, assembled
//          explicitly with block-diagonal solves and a dense product.
// Blocked right-looking elimination with panels of 32 columns (batched over
// matrices; matrices are column-major): per panel one panel launch, one
// swap-and-triangular-solve launch and one GEMM launch for the trailing
// matrix.  FP64 arithmetic on the FP64 FMA pipe: on GB300 the FP64
// tensor-core instruction (mma.sync m8n8k4) measures 1.10 TFLOP/s against
// 1.25 for FP64 FMA (dd_alu_peaks), so the trailing GEMM stays on FMA.
#include <algorithm>
#include <climits>
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
// Blocked right-looking LU with partial pivoting, batched over matrices
// (column-major, leading dimension n, n x ncols with ncols >= n: columns
// beyond n are right-hand sides that receive the same row operations).  For
// every panel of LU_NB columns k0..k0+nbe-1:
//   1. the panel (rows k0..n-1) is factorised column by column: pivot search
//      (largest |a|, lowest row on ties), row swap inside the panel,
//      multipliers, rank-1 update of the panel's remaining columns;
//   2. the columns right of the panel take the panel's row swaps, and their
//      panel rows become U12 = L11^{-1} A12 (unit lower triangular solve);
//   3. A22 -= L21 U12, a complex FP64 GEMM (zgemm_tile_kernel).
// Panels of matrices up to LU_SINGLE_MAX rows live in the shared memory of
// one thread block.  Larger panels are split into slices of LU_PR rows over
// the thread blocks of one cooperative launch, which meet once per column at
// a grid barrier: every block publishes its best pivot candidate (value,
// row, and the row's panel entries) and the owner of row k publishes that
// row; after the barrier every block picks the same winner and swaps inside
// its own slice.  The published buffers alternate between two copies by
// column parity, so a block never overwrites a copy that a slower block may
// still read.
constexpr int LU_NB = 32;
constexpr int LU_PR = 32;
constexpr int LU_SINGLE_MAX = 384;
constexpr int LU_THREADS = 256;
constexpr int LU_LD = LU_NB + 1;  // padded row of a panel slice in shared memory
constexpr long long LU_SPIN_LIMIT = 1ll << 22;

DD_DEV void argmax_merge(double& v, int& i, double ov, int oi) {
    if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
    }
}

struct LuAux {
    int* ipiv;      // [batch][n]: row swapped with row k at step k
    double* part;   // [2][chunk][ctas][2]: (|a|^2, row) of each block's candidate
    double2* prow;  // [2][chunk][ctas][LU_NB]: that candidate's panel row
    double2* rowk;  // [2][chunk][LU_NB]: panel row k before the swap
    unsigned* bar;  // arrivals at the grid barrier (zeroed before each launch)
    int* perm;      // [batch][4 LU_NB + 1]: the panel's row swaps as one permutation
                    // (destination rows, source rows, count)
};
static_assert(LU_PR >= LU_NB, "the first thread block of a panel must own all its pivot rows");

// (value, row) pair of the largest value, lowest row on ties, over the
// thread block; the result is in sv[0], si[0] for every thread
DD_DEV void block_argmax(double best, int bi, double* sv, int* si) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        argmax_merge(best, bi, ov, oi);
    }
    if ((threadIdx.x & 31) == 0) {
        sv[threadIdx.x >> 5] = best;
        si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) argmax_merge(best, bi, sv[w], si[w]);
        sv[0] = best;
        si[0] = bi;
    }
    __syncthreads();
}

// grid barrier of a cooperative launch; false (and DD_ERR_TIMEOUT in the
// status word) when the other blocks did not arrive within LU_SPIN_LIMIT polls
DD_DEV bool lu_grid_barrier(unsigned* bar, unsigned target, int* status, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        // the arrival releases the block's writes before the barrier (ordered
        // after them by __syncthreads); the acquiring load of the count
        // orders the block's later reads after the other blocks' writes
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        int ok = 1;
        for (long long spin = 0;; ++spin) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if (spin >= LU_SPIN_LIMIT) {
                ok = 0;
                raise_status(status, DD_ERR_TIMEOUT);
                break;
            }
            __nanosleep(16);
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// the panel's swaps as one permutation of the rows they touch (the first
// thread block owns rows k0.. and wrote their pivots): position i of the
// list receives the value that row src[i] held before the panel
DD_DEV void lu_panel_permutation(const LuAux& aux, int m, int n, int k0, int nbe) {
    int rows[2 * LU_NB], src[2 * LU_NB];
    int nrow = nbe;
    for (int t = 0; t < nbe; ++t) rows[t] = src[t] = k0 + t;
    for (int t = 0; t < nbe; ++t) {
        const int p = aux.ipiv[(long long)m * n + k0 + t];
        int q = -1;
        for (int i = 0; i < nrow; ++i)
            if (rows[i] == p) {
                q = i;
                break;
            }
        if (q < 0) {
            q = nrow++;
            rows[q] = src[q] = p;
        }
        const int tmp = src[t];
        src[t] = src[q];
        src[q] = tmp;
    }
    int* pm = aux.perm + (long long)m * (4 * LU_NB + 1);
    for (int i = 0; i < nrow; ++i) {
        pm[i] = rows[i];
        pm[2 * LU_NB + i] = src[i];
    }
    pm[4 * LU_NB] = nrow;
}

// panel factorisation, step 1, of matrices up to LU_SINGLE_MAX rows: one
// thread block per matrix holds all rows k0..n-1 of the panel
__global__ void __launch_bounds__(LU_THREADS) lu_panel_kernel(double2* M, long long mstride, int n, int k0, int nbe,
                                                              int rows_per, LuAux aux, double* logdet, int* status) {
    extern __shared__ double2 pan[];  // [rows_per][LU_LD]
    __shared__ double2 urow[LU_NB];
    __shared__ double sv[LU_THREADS / 32];
    __shared__ int si[LU_THREADS / 32];
    __shared__ int s_p;
    const int m = blockIdx.y, c = blockIdx.x, tid = threadIdx.x;
    double2* A = M + (long long)m * mstride;
    const int r0 = k0 + c * rows_per;
    const int nr = min(rows_per, n - r0);
    for (int e = tid; e < nr * nbe; e += blockDim.x) {
        const int r = e % nr, j = e / nr;
        pan[r * LU_LD + j] = A[(r0 + r) + (long long)(k0 + j) * n];
    }
    __syncthreads();
    for (int j = 0; j < nbe; ++j) {
        const int k = k0 + j;
        double best = -1.0;
        int bi = INT_MAX;
        for (int r = max(0, k - r0) + tid; r < nr; r += blockDim.x) {
            const double2 v = pan[r * LU_LD + j];
            argmax_merge(best, bi, v.x * v.x + v.y * v.y, r0 + r);
        }
        block_argmax(best, bi, sv, si);
        const bool own_k = k >= r0 && k < r0 + nr;
        if (tid == 0) s_p = si[0];
        __syncthreads();
        const int p = s_p;
        if (tid < nbe) {
            const double2 u = pan[(p - r0) * LU_LD + tid], old = pan[(k - r0) * LU_LD + tid];
            urow[tid] = u;
            pan[(k - r0) * LU_LD + tid] = u;
            pan[(p - r0) * LU_LD + tid] = old;
        }
        __syncthreads();
        const double2 piv = urow[j];
        const double pm = piv.x * piv.x + piv.y * piv.y;
        if (tid == 0 && own_k) {
            aux.ipiv[(long long)m * n + k] = s_p;
            if (!(pm > 0.0)) raise_status(status, DD_ERR_NUMERIC);
            logdet[m] += 0.5 * log(pm);
        }
        if (pm > 0.0) {
            const cpx<double> inv = mk<double>(piv.x / pm, -piv.y / pm);
            for (int r = max(0, k + 1 - r0) + tid; r < nr; r += blockDim.x) {
                const double2 a = pan[r * LU_LD + j];
                const cpx<double> l = cmul(mk<double>(a.x, a.y), inv);
                pan[r * LU_LD + j] = make_double2(l.x, l.y);
                for (int jj = j + 1; jj < nbe; ++jj) {
                    const double2 u = urow[jj];
                    double2& t = pan[r * LU_LD + jj];
                    t.x -= l.x * u.x - l.y * u.y;
                    t.y -= l.x * u.y + l.y * u.x;
                }
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < nr * nbe; e += blockDim.x) {
        const int r = e % nr, j = e / nr;
        A[(r0 + r) + (long long)(k0 + j) * n] = pan[r * LU_LD + j];
    }
    if (c == 0 && tid == 0) lu_panel_permutation(aux, m, n, k0, nbe);
}

// Panel factorisation of matrices above LU_SINGLE_MAX rows: thread block b of
// the cooperative launch holds rows k0 + 32 b .. (one row per lane).  Warp 0
// does the pivot search and the exchange of candidates with warp shuffles;
// all warps do the rank-1 update (lane = row, warp = group of columns).  The
// multipliers go to Lm, not into the column being read, so the update needs
// no extra barrier; a row that moves carries its multipliers (Lm, columns
// left of j) and its remaining entries (pan, columns from j on).
static_assert(LU_PR == 32, "one panel row per lane");
__global__ void __launch_bounds__(LU_THREADS) lu_panel_multi_kernel(double2* M, long long mstride, int n, int k0,
                                                                    int nbe, LuAux aux, double* logdet, int* status) {
    __shared__ double2 pan[LU_PR][LU_LD];
    __shared__ double2 Lm[LU_PR][LU_LD];
    __shared__ double2 urow[LU_NB];
    __shared__ double2 s_inv;     // 1 / pivot of the current column
    __shared__ double s_pm[LU_NB];  // |pivot|^2 per column (their logs are summed at the end)
    __shared__ int s_p, s_ok;
    const int m = blockIdx.y, c = blockIdx.x, ctas = gridDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    double2* A = M + (long long)m * mstride;
    const int r0 = k0 + c * LU_PR;
    const int nr = min(LU_PR, n - r0);
    for (int e = tid; e < nr * nbe; e += blockDim.x) {
        const int r = e % nr, j = e / nr;
        pan[r][j] = A[(r0 + r) + (long long)(k0 + j) * n];
    }
    __syncthreads();
    for (int j = 0; j < nbe; ++j) {
        const int k = k0 + j;
        const bool own_k = k >= r0 && k < r0 + nr;
        const long long mc = (long long)(j & 1) * gridDim.y + m;
        if (warp == 0) {
            double best = -1.0;
            int bi = INT_MAX;
            if (lane < nr && r0 + lane >= k) {
                const double2 v = pan[lane][j];
                best = v.x * v.x + v.y * v.y;
                bi = r0 + lane;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                argmax_merge(best, bi, __shfl_xor_sync(0xffffffffu, best, o), __shfl_xor_sync(0xffffffffu, bi, o));
            if (lane == 0) {
                aux.part[(mc * ctas + c) * 2] = best;
                aux.part[(mc * ctas + c) * 2 + 1] = (double)bi;
            }
            if (lane < nbe) {
                if (best >= 0.0) {
                    const int rb = bi - r0;
                    aux.prow[(mc * ctas + c) * LU_NB + lane] = lane < j ? Lm[rb][lane] : pan[rb][lane];
                }
                if (own_k) aux.rowk[mc * LU_NB + lane] = lane < j ? Lm[k - r0][lane] : pan[k - r0][lane];
            }
        }
        if (!lu_grid_barrier(aux.bar, (unsigned)(j + 1) * ctas * gridDim.y, status, &s_ok)) return;
        if (warp == 0) {
            double bv = -1.0;
            int bidx = INT_MAX;
            for (int q = lane; q < ctas; q += 32)
                argmax_merge(bv, bidx, __ldcg(aux.part + (mc * ctas + q) * 2),
                             (int)__ldcg(aux.part + (mc * ctas + q) * 2 + 1));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                argmax_merge(bv, bidx, __shfl_xor_sync(0xffffffffu, bv, o), __shfl_xor_sync(0xffffffffu, bidx, o));
            const int bc = (bidx - k0) / LU_PR;
            if (lane < nbe) {
                const double2 u = __ldcg(aux.prow + (mc * ctas + bc) * LU_NB + lane);
                const double2 old = __ldcg(aux.rowk + mc * LU_NB + lane);
                urow[lane] = u;
                if (lane == j) {  // the pivot: its reciprocal once for the block
                    const double pm = u.x * u.x + u.y * u.y;
                    s_pm[j] = pm;
                    s_inv = pm > 0.0 ? make_double2(u.x / pm, -u.y / pm) : make_double2(0.0, 0.0);
                }
                if (own_k) (lane < j ? Lm[k - r0][lane] : pan[k - r0][lane]) = u;
                if (bidx != k && bidx >= r0 && bidx < r0 + nr) (lane < j ? Lm[bidx - r0][lane] : pan[bidx - r0][lane]) = old;
            }
            if (lane == 0) s_p = bidx;
        }
        __syncthreads();
        const double pm = s_pm[j];
        if (tid == 0 && own_k) {
            aux.ipiv[(long long)m * n + k] = s_p;
            if (!(pm > 0.0)) raise_status(status, DD_ERR_NUMERIC);
        }
        const int r = lane;
        if (r < nr && r0 + r > k) {
            const double2 a = pan[r][j];
            if (pm > 0.0) {
                const cpx<double> l = cmul(mk<double>(a.x, a.y), mk<double>(s_inv.x, s_inv.y));
                if (warp == 0) Lm[r][j] = make_double2(l.x, l.y);
                for (int jj = j + 1 + warp; jj < nbe; jj += nwarps) {
                    const double2 u = urow[jj];
                    double2& t = pan[r][jj];
                    t.x -= l.x * u.x - l.y * u.y;
                    t.y -= l.x * u.y + l.y * u.x;
                }
            } else if (warp == 0) {
                Lm[r][j] = a;  // zero pivot: column left as it is (DD_ERR_NUMERIC raised)
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < nr * nbe; e += blockDim.x) {
        const int rr = e % nr, j = e / nr;
        A[(r0 + rr) + (long long)(k0 + j) * n] = (r0 + rr > k0 + j) ? Lm[rr][j] : pan[rr][j];
    }
    // ln|det| of the panel's pivots (the first thread block owns them)
    if (c == 0 && warp == 0) {
        double l = lane < nbe ? 0.5 * log(s_pm[lane]) : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (lane == 0) logdet[m] += l;
    }
    if (c == 0 && tid == 0) lu_panel_permutation(aux, m, n, k0, nbe);
}

// step 2: one warp per column right of the panel: the panel's row
// permutation (all touched rows gathered, then scattered), then forward
// substitution with the unit lower triangle L11, lane r holding row k0 + r
constexpr int LU_TRSM_WARPS = 4;
__global__ void __launch_bounds__(32 * LU_TRSM_WARPS) lu_swap_trsm_kernel(double2* M, long long mstride, int n,
                                                                         int ncols, int k0, int nbe, const int* perm) {
    __shared__ double2 L[LU_NB][LU_LD];
    __shared__ int s_dst[2 * LU_NB], s_src[2 * LU_NB];
    __shared__ int s_np;
    const int m = blockIdx.y, tid = threadIdx.x, lane = tid & 31;
    double2* A = M + (long long)m * mstride;
    for (int e = tid; e < nbe * nbe; e += blockDim.x) {
        const int r = e % nbe, cc = e / nbe;
        L[r][cc] = A[(k0 + r) + (long long)(k0 + cc) * n];
    }
    const int* pm = perm + (long long)m * (4 * LU_NB + 1);
    if (tid < 2 * LU_NB) {
        s_dst[tid] = pm[tid];
        s_src[tid] = pm[2 * LU_NB + tid];
    }
    if (tid == 0) s_np = pm[4 * LU_NB];
    __syncthreads();
    const int j = k0 + nbe + blockIdx.x * LU_TRSM_WARPS + (tid >> 5);
    if (j >= ncols) return;  // uniform per warp
    double2* col = A + (long long)j * n;
    const int np = s_np;
    const double2 zero = make_double2(0.0, 0.0);
    const double2 v0 = lane < np ? col[s_src[lane]] : zero;
    const double2 v1 = lane + 32 < np ? col[s_src[lane + 32]] : zero;
    __syncwarp();
    if (lane >= nbe && lane < np) col[s_dst[lane]] = v0;
    if (lane + 32 < np) col[s_dst[lane + 32]] = v1;
    double2 x = v0;
    for (int cc = 0; cc + 1 < nbe; ++cc) {
        const double xr = __shfl_sync(0xffffffffu, x.x, cc), xi = __shfl_sync(0xffffffffu, x.y, cc);
        if (lane > cc && lane < nbe) {
            const double2 l = L[lane][cc];
            x.x -= l.x * xr - l.y * xi;
            x.y -= l.x * xi + l.y * xr;
        }
    }
    if (lane < nbe) col[k0 + lane] = x;
}

// ------------------------------------------------ trailing update on tensor cores
// The trailing update A22 -= L21 U12 on the FP16 tensor cores with FP64
// accuracy (Ozaki scheme).  Each row i of [Re L21, Im L21] (64 reals) is
// scaled by 2^-e_i so that its entries are below 1 in magnitude and cut into
// OZ_S slices of OZ_BETA bits: x 2^-e_i = sum_s q_s 2^(-OZ_BETA (s + 1)),
// q_s integers (|q_0| <= 2^OZ_BETA, |q_s| <= 2^(OZ_BETA - 1)), exact in FP16.
// The columns of [Re U12; Im U12] likewise (exponents f_j).  A product of two
// slices is an integer below 2^(2 OZ_BETA); the slice pairs (s, t) of one
// diagonal d = s + t share the weight 2^(-OZ_BETA (d + 2)), and their sum
// over the 64 terms stays below 2^22, so the tensor cores' FP32 accumulation
// of a diagonal is exact.  The diagonals d < OZ_S are combined in groups of
// four in int64 (exact), the groups summed in FP64 and scaled by
// 2^(e_i + f_j).  What is left out (the pairs with s + t >= OZ_S
// and the remainders after OZ_S slices) adds up to less than 2^-48 of the
// product of the row and column maxima, below the rounding bound of an FP64
// dot product of the same 64 terms (64 x 2^-53).  Complex products:
// C_re = [Re L, Im L] [Re U; -Im U], C_im = [Re L, Im L] [Im U; Re U].
constexpr int OZ_BETA = 7;
constexpr int OZ_S = 8;
constexpr int OZ_K = 2 * LU_NB;  // real k of the complex panel width
constexpr int OZ_TM = 64;        // rows of C per thread block (4 groups of 16 rows)
constexpr int OZ_TN = 32;        // columns of C per thread block (two thread blocks per SM)
constexpr int OZ_LD = OZ_K + 8;  // padded smem row of 64 halves (conflict-free fragment loads)

// slices of L21 rows (transposed = false) or U12 columns (transposed = true):
// one warp per row / column; out[s][r][0..63] (FP16), ex[r] the exponent
__global__ void __launch_bounds__(256) ozaki_split_kernel(const double2* X, int ld, int nrows, int nbe, bool transposed,
                                                          __half* out, long long slice_stride, int* ex) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= nrows) return;
    double a0 = 0.0, a1 = 0.0;
    if (lane < nbe) {
        const double2 v = transposed ? X[lane + (long long)r * ld] : X[r + (long long)lane * ld];
        a0 = v.x;
        a1 = v.y;
    }
    double mx = fmax(fabs(a0), fabs(a1));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx < 2^e
    double t0 = ldexp(a0, -e), t1 = ldexp(a1, -e);
    __half* o = out + (long long)r * OZ_K;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
        t0 *= (double)(1 << OZ_BETA);
        t1 *= (double)(1 << OZ_BETA);
        const double q0 = rint(t0), q1 = rint(t1);
        t0 -= q0;
        t1 -= q1;
        o[s * slice_stride + lane] = __double2half(q0);
        o[s * slice_stride + lane + 32] = __double2half(q1);
    }
    if (lane == 0) ex[r] = e;
}

// four 8 x 8 FP16 matrices from shared memory (row addresses from lanes 0-7,
// 8-15, 16-23, 24-31), each thread receiving its fragment pair of each
DD_DEV void ldsm_x4(uint32_t* r, const __half* row_addr) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(row_addr);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

DD_DEV void mma_f16_f32(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C (m x nn complex, column-major, ld ldc) -= L21 U12 from the slices: a
// 64 x 32 tile of C per thread block of 8 warps, 16 x 16 per warp (one m16
// row of two n8 tiles), every slice of the tile's rows and columns staged
// in shared memory once (110 KB: two thread blocks per SM, so that one
// stages while the other computes)
constexpr int OZ_NT = 2;  // n8 tiles per warp
__global__ void __launch_bounds__(256, 2) ozaki_update_kernel(int m, int nn, const __half* As, const int* ea,
                                                              long long sa, const __half* Bs, const int* eb,
                                                              long long sb, double2* C, int ldc) {
    extern __shared__ __align__(16) unsigned char oz_smem[];
    __half* sA = reinterpret_cast<__half*>(oz_smem);
    __half* sB = sA + OZ_S * OZ_TM * OZ_LD;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = blockIdx.y * OZ_TM, c0 = blockIdx.x * OZ_TN;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < OZ_S * OZ_TM * (OZ_K / 8); e += blockDim.x) {
        const int s = e / (OZ_TM * (OZ_K / 8)), rem = e % (OZ_TM * (OZ_K / 8)), row = rem / (OZ_K / 8), q = rem % (OZ_K / 8);
        const uint4 va = r0 + row < m ? reinterpret_cast<const uint4*>(As + s * sa + (long long)(r0 + row) * OZ_K)[q] : z;
        *reinterpret_cast<uint4*>(sA + (s * OZ_TM + row) * OZ_LD + q * 8) = va;
    }
    for (int e = tid; e < OZ_S * OZ_TN * (OZ_K / 8); e += blockDim.x) {
        const int s = e / (OZ_TN * (OZ_K / 8)), rem = e % (OZ_TN * (OZ_K / 8)), col = rem / (OZ_K / 8), q = rem % (OZ_K / 8);
        const uint4 vb = c0 + col < nn ? reinterpret_cast<const uint4*>(Bs + s * sb + (long long)(c0 + col) * OZ_K)[q] : z;
        *reinterpret_cast<uint4*>(sB + (s * OZ_TN + col) * OZ_LD + q * 8) = vb;
    }
    __syncthreads();
    const int wm = warp & 3, wn = warp >> 2, g = lane >> 2, tig = lane & 3;
    double accR[OZ_NT][4], accI[OZ_NT][4];
    long long gR[OZ_NT][4], gI[OZ_NT][4];
#pragma unroll
    for (int nt = 0; nt < OZ_NT; ++nt)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            accR[nt][c] = accI[nt][c] = 0.0;
            gR[nt][c] = gI[nt][c] = 0;
        }
    static_assert(OZ_S % 4 == 0, "diagonals are summed in groups of four");
#pragma unroll 1
    for (int d = 0; d < OZ_S; ++d) {
        float fR[OZ_NT][4], fI[OZ_NT][4];
#pragma unroll
        for (int nt = 0; nt < OZ_NT; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) fR[nt][c] = fI[nt][c] = 0.0f;
#pragma unroll 1
        for (int s = 0; s <= d; ++s) {
            const __half* ab = sA + (s * OZ_TM + 16 * wm) * OZ_LD;
            const __half* bb = sB + ((d - s) * OZ_TN + 8 * OZ_NT * wn) * OZ_LD;
#pragma unroll
            for (int ks = 0; ks < OZ_K / 16; ++ks) {
                // A fragment: rows lane % 16, k half lane / 16 of the 16 x 16 tile
                uint32_t a[4];
                ldsm_x4(a, ab + (lane & 15) * OZ_LD + 16 * ks + (lane >> 4) * 8);
                // first half of k: Re U (real part), Im U (imaginary part);
                // second half: -Im U (real part), Re U (imaginary part)
                const bool hi = 16 * ks >= LU_NB;
                const int ko = hi ? -LU_NB : LU_NB;
                const uint32_t sg = hi ? 0x80008000u : 0u;
                // B fragments of one n8 tile: k and k + 8 for the real part,
                // the same at offset ko for the imaginary part
                const int kl = 16 * ks + ((lane >> 3) & 1) * 8 + ((lane >> 4) ? ko : 0);
#pragma unroll
                for (int nt = 0; nt < OZ_NT; ++nt) {
                    uint32_t b[4];
                    ldsm_x4(b, bb + (8 * nt + (lane & 7)) * OZ_LD + kl);
                    mma_f16_f32(fR[nt], a, b[0] ^ sg, b[1] ^ sg);
                    mma_f16_f32(fI[nt], a, b[2], b[3]);
                }
            }
        }
        // four neighbouring diagonals combine exactly in int64 (Horner in
        // 2^7: below 2^43), so the FP64 pipe sees one conversion and one FMA
        // per element for every four diagonals
#pragma unroll
        for (int nt = 0; nt < OZ_NT; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                gR[nt][c] = gR[nt][c] * (1 << OZ_BETA) + __float2int_rn(fR[nt][c]);
                gI[nt][c] = gI[nt][c] * (1 << OZ_BETA) + __float2int_rn(fI[nt][c]);
            }
        if ((d & 3) == 3) {
            const double w = ldexp(1.0, -OZ_BETA * (d + 2));
#pragma unroll
            for (int nt = 0; nt < OZ_NT; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    accR[nt][c] = fma(w, (double)gR[nt][c], accR[nt][c]);
                    accI[nt][c] = fma(w, (double)gI[nt][c], accI[nt][c]);
                    gR[nt][c] = gI[nt][c] = 0;
                }
        }
    }
#pragma unroll
    for (int nt = 0; nt < OZ_NT; ++nt)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int row = r0 + 16 * wm + g + (c >= 2 ? 8 : 0);
            const int col = c0 + 8 * OZ_NT * wn + 8 * nt + 2 * tig + (c & 1);
            if (row < m && col < nn) {
                const double sc = ldexp(1.0, ea[row] + eb[col]);
                double2& o = C[row + (long long)col * ldc];
                o.x -= sc * accR[nt][c];
                o.y -= sc * accI[nt][c];
            }
        }
}
constexpr size_t OZ_SMEM = (size_t)OZ_S * (OZ_TM + OZ_TN) * OZ_LD * sizeof(__half);

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

// C = beta C + alpha A B for complex FP64 column-major matrices (m x kk times
// kk x nn), batched over blockIdx.z with the strides sA, sB, sC: a 64 x 64
// tile of C per thread block of 256 threads, 4 x 4 elements per thread (rows
// tr + 16 i, columns tc + 16 j), A and B staged through shared memory in
// slices of 16 along k.  Every complex product is four FP64 FMAs; with beta
// == 0 C is not read.
constexpr int ZG_T = 64, ZG_K = 16;
__global__ void __launch_bounds__(256) zgemm_tile_kernel(int m, int nn, int kk, const double2* A, int lda, long long sA,
                                                         const double2* B, int ldb, long long sB, double2* C, int ldc,
                                                         long long sC, double alpha, double beta) {
    __shared__ double2 As[ZG_K][ZG_T + 1];
    __shared__ double2 Bs[ZG_K][ZG_T + 1];
    const long long z = blockIdx.z;
    A += z * sA;
    B += z * sB;
    C += z * sC;
    const int r0 = blockIdx.y * ZG_T, c0 = blockIdx.x * ZG_T;
    const int t = threadIdx.x, tr = t & 15, tc = t >> 4;
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < kk; k0 += ZG_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = t + 256 * q, row = e & 63, kx = e >> 6;
            const int gr = r0 + row, gk = k0 + kx;
            As[kx][row] = (gr < m && gk < kk) ? A[gr + (long long)gk * lda] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = t + 256 * q, kx = e & 15, col = e >> 4;
            const int gc = c0 + col, gk = k0 + kx;
            Bs[kx][col] = (gc < nn && gk < kk) ? B[gk + (long long)gc * ldb] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kx = 0; kx < ZG_K; ++kx) {
            double2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kx][tr + 16 * i];
                b[i] = Bs[kx][tc + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
                    acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
                    acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
                    acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + tr + 16 * i, cc = c0 + tc + 16 * j;
            if (r < m && cc < nn) {
                double2& o = C[r + (long long)cc * ldc];
                const double2 old = beta != 0.0 ? o : make_double2(0.0, 0.0);
                o = make_double2(alpha * acc[i][j].x + beta * old.x, alpha * acc[i][j].y + beta * old.y);
            }
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

// scratch of the blocked LU, behind the matrices of the exact path
static char* lu_scratch(dd_handle* h, size_t* cap) {
    const size_t n = (size_t)12 * h->g.V, nb12 = (size_t)12 * h->g.bsites;
    const size_t off = h->g.V <= 512 ? 2 * n * n * sizeof(double2) : (size_t)h->g.nblocks * nb12 * nb12 * sizeof(double2);
    *cap = h->lu_bytes > off ? h->lu_bytes - off : 0;
    return (char*)h->d_lu + off;
}

// LU of `batch` n x ncols matrices, eliminating the first n columns; logdet
// receives sum_k ln|u_kk| per matrix; with back = true the right-hand-side
// columns are overwritten by the solutions.
static int lu_batched(dd_handle* h, double2* M, long long mstride, int batch, int n, int ncols, double* logdet,
                      bool back) {
    size_t cap = 0;
    char* scr = lu_scratch(h, &cap);
    const bool single = n <= LU_SINGLE_MAX;
    const int ctas0 = single ? 1 : grid_for(n, LU_PR);
    int chunk = batch;
    if (single) {
        const size_t smem = (size_t)n * LU_LD * sizeof(double2);
        cudaError_t e = cudaFuncSetAttribute(lu_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return dd_cuda_check(h, e, "lu_panel_kernel shared memory");
    } else {
        // one cooperative launch holds every thread block of its matrices
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_panel_multi_kernel, LU_THREADS, 0);
        if (e != cudaSuccess) return dd_cuda_check(h, e, "lu_panel_kernel occupancy");
        const long long resident = (long long)per_sm * std::max(1, h->num_sms);
        if (resident < ctas0) return dd_fail(h, DD_ERR_UNSUPPORTED, "dense LU: a panel needs more thread blocks than fit on the GPU");
        chunk = (int)std::min<long long>(batch, resident / ctas0);
    }
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o = 0;
    LuAux aux{};
    aux.ipiv = (int*)(scr + o);
    o += up((size_t)batch * n * sizeof(int));
    aux.perm = (int*)(scr + o);
    o += up((size_t)batch * (4 * LU_NB + 1) * sizeof(int));
    if (!single) {
        aux.part = (double*)(scr + o);
        o += up((size_t)2 * chunk * ctas0 * 2 * sizeof(double));
        aux.prow = (double2*)(scr + o);
        o += up((size_t)2 * chunk * ctas0 * LU_NB * sizeof(double2));
        aux.rowk = (double2*)(scr + o);
        o += up((size_t)2 * chunk * LU_NB * sizeof(double2));
        aux.bar = (unsigned*)(scr + o);
        o += 256;
    }
    if (o > cap) return dd_fail(h, DD_ERR_UNSUPPORTED, "dense LU: no room for the pivot scratch");
    // slices of the tensor-core trailing update (matrices above LU_SINGLE_MAX rows)
    __half *oa = nullptr, *ob = nullptr;
    int *oea = nullptr, *oeb = nullptr;
    const long long osa = (long long)n * OZ_K, osb = (long long)ncols * OZ_K;
    bool tensor = !single && h->lu_tensor;
    if (tensor) {
        size_t need = o + up((size_t)OZ_S * osa * sizeof(__half)) + up((size_t)OZ_S * osb * sizeof(__half)) +
                      up((size_t)n * sizeof(int)) + up((size_t)ncols * sizeof(int));
        if (need > cap) {
            tensor = false;  // no room: the FP64 FMA update
        } else {
            oa = (__half*)(scr + o);
            o += up((size_t)OZ_S * osa * sizeof(__half));
            ob = (__half*)(scr + o);
            o += up((size_t)OZ_S * osb * sizeof(__half));
            oea = (int*)(scr + o);
            o += up((size_t)n * sizeof(int));
            oeb = (int*)(scr + o);
            o += up((size_t)ncols * sizeof(int));
            cudaError_t e = cudaFuncSetAttribute(ozaki_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)OZ_SMEM);
            if (e != cudaSuccess) return dd_cuda_check(h, e, "ozaki_update_kernel shared memory");
        }
    }
    DD_KLAUNCH(h, zero_doubles_kernel<<<grid_for(batch, 64), 64, 0, h->stream>>>(batch, logdet));
    for (int k0 = 0; k0 < n; k0 += LU_NB) {
        const int nbe = std::min(LU_NB, n - k0);
        if (single) {
            const int rows = n - k0;
            const size_t smem = (size_t)rows * LU_LD * sizeof(double2);
            DD_KLAUNCH(h, lu_panel_kernel<<<dim3(1, batch), LU_THREADS, smem, h->stream>>>(
                              M, mstride, n, k0, nbe, rows, aux, logdet, h->d_status));
        } else {
            const int ctas = grid_for(n - k0, LU_PR);
            for (int m0 = 0; m0 < batch; m0 += chunk) {
                const int mb = std::min(chunk, batch - m0);
                cudaError_t e = cudaMemsetAsync(aux.bar, 0, sizeof(unsigned), h->stream);
                if (e != cudaSuccess) return dd_cuda_check(h, e, "lu barrier reset");
                double2* Mc = M + (long long)m0 * mstride;
                double* ldc = logdet + m0;
                LuAux ac = aux;
                ac.ipiv = aux.ipiv + (long long)m0 * n;
                ac.perm = aux.perm + (long long)m0 * (4 * LU_NB + 1);
                int nn = n, kk0 = k0, nb_ = nbe;
                long long ms = mstride;
                int* st = h->d_status;
                void* args[] = {&Mc, &ms, &nn, &kk0, &nb_, &ac, &ldc, &st};
                e = cudaLaunchCooperativeKernel((const void*)lu_panel_multi_kernel, dim3(ctas, mb), dim3(LU_THREADS), args,
                                                0, h->stream);
                ++h->launches;
                if (e != cudaSuccess) return dd_cuda_check(h, e, "lu_panel_kernel (cooperative launch)");
            }
        }
        const int right = ncols - k0 - nbe;
        if (right > 0) {
            DD_KLAUNCH(h, lu_swap_trsm_kernel<<<dim3(grid_for(right, LU_TRSM_WARPS), batch), 32 * LU_TRSM_WARPS, 0,
                                                h->stream>>>(M, mstride, n, ncols, k0, nbe, aux.perm));
            const int below = n - k0 - nbe;
            if (below > 0 && tensor) {
                for (int mi = 0; mi < batch; ++mi) {
                    double2* Mm = M + (long long)mi * mstride;
                    DD_KLAUNCH(h, ozaki_split_kernel<<<grid_for(below, 8), 256, 0, h->stream>>>(
                                      Mm + (k0 + nbe) + (long long)k0 * n, n, below, nbe, false, oa, osa, oea));
                    DD_KLAUNCH(h, ozaki_split_kernel<<<grid_for(right, 8), 256, 0, h->stream>>>(
                                      Mm + k0 + (long long)(k0 + nbe) * n, n, right, nbe, true, ob, osb, oeb));
                    dim3 g(grid_for(right, OZ_TN), grid_for(below, OZ_TM));
                    DD_KLAUNCH(h, ozaki_update_kernel<<<g, 256, OZ_SMEM, h->stream>>>(
                                      below, right, oa, oea, osa, ob, oeb, osb, Mm + (k0 + nbe) + (long long)(k0 + nbe) * n,
                                      n));
                }
            } else if (below > 0) {
                dim3 g(grid_for(right, ZG_T), grid_for(below, ZG_T), batch);
                DD_KLAUNCH(h, zgemm_tile_kernel<<<g, 256, 0, h->stream>>>(
                                  below, right, nbe, M + (k0 + nbe) + (long long)k0 * n, n, mstride,
                                  M + k0 + (long long)(k0 + nbe) * n, n, mstride,
                                  M + (k0 + nbe) + (long long)(k0 + nbe) * n, n, mstride, -1.0, 1.0));
            }
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
    // On the tensor cores (the slices of the LU's trailing update, 32 columns
    // of B and rows of X at a time) Y accumulates -B X.
    size_t cap = 0;
    char* scr = lu_scratch(h, &cap);
    const long long osz = (long long)nh * OZ_K;
    const bool tensor = h->lu_tensor && nb12 % LU_NB == 0 &&
                        2 * (size_t)OZ_S * osz * sizeof(__half) + 2 * (size_t)nh * sizeof(int) <= cap;
    if (tensor) {
        __half* oa = (__half*)scr;
        __half* ob = oa + OZ_S * osz;
        int* oea = (int*)(ob + OZ_S * osz);
        int* oeb = oea + nh;
        cudaError_t e = cudaFuncSetAttribute(ozaki_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)OZ_SMEM);
        if (e != cudaSuccess) return dd_cuda_check(h, e, "ozaki_update_kernel shared memory");
        const long long yn = (long long)nh * nh;
        DD_KLAUNCH(h, zero_kernel<<<grid_for(yn, 256), 256, 0, h->stream>>>(yn, Y));
        for (int b = 0; b < nbk; ++b)
            for (int kc = 0; kc < nb12 / LU_NB; ++kc) {
                DD_KLAUNCH(h, ozaki_split_kernel<<<grid_for(nh, 8), 256, 0, h->stream>>>(
                                  D + (long long)(nh + b * nb12 + kc * LU_NB) * n, n, nh, LU_NB, false, oa, osz, oea));
                DD_KLAUNCH(h, ozaki_split_kernel<<<grid_for(nh, 8), 256, 0, h->stream>>>(
                                  aug + b * as + (long long)nb12 * nb12 + kc * LU_NB, nb12, nh, LU_NB, true, ob, osz, oeb));
                DD_KLAUNCH(h, ozaki_update_kernel<<<dim3(grid_for(nh, OZ_TN), grid_for(nh, OZ_TM)), 256, OZ_SMEM,
                                                    h->stream>>>(nh, nh, oa, oea, osz, ob, oeb, osz, Y, nh));
            }
    } else {
        for (int b = 0; b < nbk; ++b) {
            dim3 g(grid_for(nh, ZG_T), grid_for(nh, ZG_T), 1);
            DD_KLAUNCH(h, zgemm_tile_kernel<<<g, 256, 0, h->stream>>>(nh, nh, nb12, D + (long long)(nh + b * nb12) * n, n,
                                                                    0, aug + b * as + (long long)nb12 * nb12, nb12, 0,
                                                                    Y, nh, 0, 1.0, b == 0 ? 0.0 : 1.0));
        }
    }
    const double ysign = tensor ? -1.0 : 1.0;
    // Z = A^{-1} Y: per black block [A_b | Y_b]
    for (int b = 0; b < nbk; ++b) {
        int r0 = b * nb12;
        dim3 gA(grid_for(nb12, 16), grid_for(nb12, 16)), gY(grid_for(nh, 16), grid_for(nb12, 16));
        DD_KLAUNCH(h, copy_sub_kernel<<<gA, b16, 0, h->stream>>>(D, n, r0, r0, nb12, nb12, aug + b * as, nb12, 0, 1.0, 0));
        DD_KLAUNCH(h, copy_sub_kernel<<<gY, b16, 0, h->stream>>>(Y, nh, r0, 0, nb12, nh, aug + b * as, nb12, nb12, ysign, 0));
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

// check of the bounded wait of the grid barrier: `rounds` barriers of all
// thread blocks; the last one waits for `missing` arrivals that never come
__global__ void barrier_check_kernel(unsigned* bar, int rounds, int missing, int* status, int* passed) {
    __shared__ int s_ok;
    for (int r = 1; r <= rounds; ++r) {
        const unsigned target = (unsigned)r * gridDim.x + (r == rounds ? (unsigned)missing : 0u);
        if (!lu_grid_barrier(bar, target, status, &s_ok)) return;
    }
    if (threadIdx.x == 0) atomicAdd(passed, 1);
}

extern "C" int dd_barrier_check(dd_t h, int missing, int* passed) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    rc = dd_require_feature(h, h->feat_exact, "dd_barrier_check");
    if (rc) return rc;
    if (!passed || missing < 0 || missing > 64) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_barrier_check: bad arguments");
    size_t cap = 0;
    char* scr = lu_scratch(h, &cap);
    if (cap < 256) return dd_fail(h, DD_ERR_UNSUPPORTED, "dd_barrier_check: no scratch");
    unsigned* bar = (unsigned*)scr;
    int* dpassed = (int*)(scr + 128);
    DD_CUDA(h, cudaMemsetAsync(scr, 0, 256, h->stream));
    const int ctas = std::max(1, std::min(8, h->num_sms));
    int rounds = 3;
    void* args[] = {&bar, &rounds, &missing, &h->d_status, &dpassed};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)barrier_check_kernel, dim3(ctas), dim3(LU_THREADS), args,
                                                0, h->stream);
    ++h->launches;
    if (e != cudaSuccess) return dd_cuda_check(h, e, "barrier_check_kernel (cooperative launch)");
    int np = 0;
    DD_CUDA(h, cudaMemcpyAsync(&np, dpassed, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DD_CUDA(h, cudaStreamSynchronize(h->stream));
    *passed = np == ctas ? 1 : 0;
    return DD_OK;
}

extern "C" int dd_lu_tensor_cores(dd_t h, int on) {
    if (!h || on < 0 || on > 1) return DD_ERR_INVALID_ARG;
    h->lu_tensor = on != 0;
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
