// Device-side building blocks shared by the kernels of the library:
// complex arithmetic, field storage formats, lattice index arithmetic,
// the Wilson spin projectors, Philox4x32-10 and block reductions.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define DD_DEV __device__ __forceinline__
#define DD_HD __host__ __device__ __forceinline__

// ------------------------------------------------------------------ complex
template <class R>
struct cpx {
    R x, y;
};
template <class R>
DD_HD cpx<R> mk(R a, R b) {
    cpx<R> c;
    c.x = a;
    c.y = b;
    return c;
}
template <class R>
DD_HD cpx<R> operator+(cpx<R> a, cpx<R> b) { return mk(a.x + b.x, a.y + b.y); }
template <class R>
DD_HD cpx<R> operator-(cpx<R> a, cpx<R> b) { return mk(a.x - b.x, a.y - b.y); }
template <class R>
DD_HD cpx<R> operator-(cpx<R> a) { return mk(-a.x, -a.y); }
template <class R>
DD_HD cpx<R> operator*(R s, cpx<R> a) { return mk(s * a.x, s * a.y); }
template <class R>
DD_HD cpx<R> cmul(cpx<R> a, cpx<R> b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
template <class R>
DD_HD cpx<R> cmulc(cpx<R> a, cpx<R> b) { return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
template <class R>
DD_HD cpx<R> conj(cpx<R> a) { return mk(a.x, -a.y); }
template <class R>
DD_HD cpx<R> itimes(cpx<R> a) { return mk(-a.y, a.x); }
template <class R>
DD_HD R norm2(cpx<R> a) { return a.x * a.x + a.y * a.y; }
template <class R>
DD_HD cpx<R> cmac(cpx<R> acc, cpx<R> a, cpx<R> b) {  // acc + a*b
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}
template <class R>
DD_HD cpx<R> cmacc(cpx<R> acc, cpx<R> a, cpx<R> b) {  // acc + conj(a)*b
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
    return acc;
}

template <class R>
struct Spinor {
    cpx<R> c[12];  // index spin*3 + colour
};
template <class R>
struct Half {
    cpx<R> c[6];  // index spin*3 + colour, spins 0..1
};
template <class R>
struct Link {
    cpx<R> m[3][3];
};

// ----------------------------------------------------------- storage formats
// All fields are stored as 16-byte (or 8-byte) chunks, chunk-major:
// chunk k of site i lives at base[k * stride + i], so consecutive threads
// (consecutive sites) read consecutive addresses.

// FP64 spinor: 12 chunks of double2 (one complex each)
struct SpinorF64 {
    double2* p;
    long long stride;
    typedef double real;
    static constexpr int chunks = 12;
    template <class R>
    DD_DEV void load(long long i, Spinor<R>& s) const {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = p[k * stride + i];
            s.c[k] = mk<R>((R)v.x, (R)v.y);
        }
    }
    // value = returned scale * s (the scale is 1 for this format)
    template <class R>
    DD_DEV R load_unscaled(long long i, Spinor<R>& s) const {
        load(i, s);
        return (R)1;
    }
    template <class R>
    DD_DEV void store(long long i, const Spinor<R>& s) const {
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k * stride + i] = make_double2((double)s.c[k].x, (double)s.c[k].y);
    }
};

// FP32 spinor: 6 chunks of float4 (two complex each)
struct SpinorF32 {
    float4* p;
    long long stride;
    typedef float real;
    static constexpr int chunks = 6;
    template <class R>
    DD_DEV void load(long long i, Spinor<R>& s) const {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 v = p[k * stride + i];
            s.c[2 * k] = mk<R>((R)v.x, (R)v.y);
            s.c[2 * k + 1] = mk<R>((R)v.z, (R)v.w);
        }
    }
    template <class R>
    DD_DEV R load_unscaled(long long i, Spinor<R>& s) const {
        load(i, s);
        return (R)1;
    }
    template <class R>
    DD_DEV void store(long long i, const Spinor<R>& s) const {
#pragma unroll
        for (int k = 0; k < 6; ++k)
            p[k * stride + i] = make_float4((float)s.c[2 * k].x, (float)s.c[2 * k].y, (float)s.c[2 * k + 1].x,
                                            (float)s.c[2 * k + 1].y);
    }
};

// FP16 spinor: 3 chunks of 8 halves (four complex each) + one FP32 scale per
// site; value = half * scale, scale = largest |real or imaginary part|.
struct SpinorF16 {
    uint4* p;
    float* nrm;
    long long stride;
    typedef float real;
    static constexpr int chunks = 3;
    template <class R>
    DD_DEV void load(long long i, Spinor<R>& s) const {
        float sc = nrm[i];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = p[k * stride + i];
            const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 f = __half22float2(h[j]);
                s.c[4 * k + j] = mk<R>((R)(f.x * sc), (R)(f.y * sc));
            }
        }
    }
    // the stored halves without the site scale; returns the scale (the
    // stencil applies it once per hop, after the linear spin/colour algebra)
    template <class R>
    DD_DEV R load_unscaled(long long i, Spinor<R>& s) const {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = p[k * stride + i];
            const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 f = __half22float2(h[j]);
                s.c[4 * k + j] = mk<R>((R)f.x, (R)f.y);
            }
        }
        return (R)nrm[i];
    }
    template <class R>
    DD_DEV void store(long long i, const Spinor<R>& s) const {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf((float)s.c[k].x), fabsf((float)s.c[k].y)));
        // a site whose largest entry is below 1e-30 is stored as zero (1/m would overflow)
        float inv = m > 1e-30f ? 1.0f / m : 0.f;
        if (!(m > 1e-30f)) m = 0.f;
        nrm[i] = m;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v;
            __half2* h = reinterpret_cast<__half2*>(&v);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                h[j] = __floats2half2_rn((float)s.c[4 * k + j].x * inv, (float)s.c[4 * k + j].y * inv);
            p[k * stride + i] = v;
        }
    }
};

// Third row of an SU(3) matrix from the first two: row2 = conj(row0 x row1).
template <class R>
DD_DEV void reconstruct_row2(Link<R>& u) {
    u.m[2][0] = conj(cmul(u.m[0][1], u.m[1][2]) - cmul(u.m[0][2], u.m[1][1]));
    u.m[2][1] = conj(cmul(u.m[0][2], u.m[1][0]) - cmul(u.m[0][0], u.m[1][2]));
    u.m[2][2] = conj(cmul(u.m[0][0], u.m[1][1]) - cmul(u.m[0][1], u.m[1][0]));
}

// FP64 link, all 9 entries: 9 chunks of double2 per direction.
// Link (site i, direction a) chunk k at p[(a*9 + k) * stride + i].
struct LinkF64 {
    const double2* p;
    long long stride;
    static constexpr int chunks = 9;
    template <class R>
    DD_DEV void load(long long i, int a, Link<R>& u) const {
        const double2* q = p + (long long)a * 9 * stride + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 v = q[k * stride];
            u.m[k / 3][k % 3] = mk<R>((R)v.x, (R)v.y);
        }
    }
};

// FP32 link, rows 0-1 stored (3 chunks of float4), row 2 rebuilt.
struct LinkF32 {
    const float4* p;
    long long stride;
    static constexpr int chunks = 3;
    template <class R>
    DD_DEV void load(long long i, int a, Link<R>& u) const {
        const float4* q = p + (long long)a * 3 * stride + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 v = q[k * stride];
            int e0 = 2 * k, e1 = 2 * k + 1;
            u.m[e0 / 3][e0 % 3] = mk<R>((R)v.x, (R)v.y);
            u.m[e1 / 3][e1 % 3] = mk<R>((R)v.z, (R)v.w);
        }
        reconstruct_row2(u);
    }
};

// FP16 link, rows 0-1 stored (3 chunks of 4 halves = 8 bytes), row 2 rebuilt.
struct LinkF16 {
    const uint2* p;
    long long stride;
    static constexpr int chunks = 3;
    template <class R>
    DD_DEV void load(long long i, int a, Link<R>& u) const {
        const uint2* q = p + (long long)a * 3 * stride + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint2 v = q[k * stride];
            const __half2* h = reinterpret_cast<const __half2*>(&v);
            float2 f0 = __half22float2(h[0]);
            float2 f1 = __half22float2(h[1]);
            int e0 = 2 * k, e1 = 2 * k + 1;
            u.m[e0 / 3][e0 % 3] = mk<R>((R)f0.x, (R)f0.y);
            u.m[e1 / 3][e1 % 3] = mk<R>((R)f1.x, (R)f1.y);
        }
        reconstruct_row2(u);
    }
};

// ------------------------------------------------------------------ site sets
// The sites a kernel visits: thread t < n works on site map[t] (map null:
// on site t).  Solves restricted to the blocks of one colour visit only
// that colour's half of the lattice.
struct SiteSet {
    const int* map;
    long long n;
    // >= 0: the set is the sites of the blocks of this colour (even block
    // extent along axis 0), map holds them in increasing even-odd index, and
    // the hop kernel may compute them instead of loading them (colour_site)
    int colour = -1;
    DD_DEV long long at(long long t) const { return map ? (long long)__ldg(map + t) : t; }
};

// ------------------------------------------------------------------ geometry
struct Geo {
    int L[4];     // extents, axis 3 = time
    int Lh0;      // L0 / 2
    int V, Vh;    // sites, sites per parity
    int b[4];     // block extents
    int nbk[4];   // blocks per direction
    int nblocks;  // number of blocks
    int bsites;   // sites per block
    int bc;       // fermion phase on time-wrapping hops (+1 / -1)
    int st[4];    // canonical strides 1, L0, L0 L1, L0 L1 L2
    // multipliers for division by Lh0, L1, L2 with __umulhi (exact for n * d < 2^32; 0: use '/')
    unsigned mLh0, mL1, mL2;
    // the same for Lh0 / 2, b0 / 2 (colour site sets) and the block extents b0..b3
    unsigned mQ, mB, mb[4];
};

// derived members of a Geo whose L, b, nbk and bc are set (host side)
inline void geo_finish(Geo& g) {
    long long V = (long long)g.L[0] * g.L[1] * g.L[2] * g.L[3];
    g.V = (int)V;
    g.Vh = (int)(V / 2);
    g.Lh0 = g.L[0] / 2;
    g.nblocks = g.nbk[0] * g.nbk[1] * g.nbk[2] * g.nbk[3];
    g.bsites = g.b[0] * g.b[1] * g.b[2] * g.b[3];
    g.st[0] = 1;
    g.st[1] = g.L[0];
    g.st[2] = g.L[0] * g.L[1];
    g.st[3] = g.L[0] * g.L[1] * g.L[2];
    auto magic = [&](int d) -> unsigned {
        // ceil(2^32 / d), valid while every dividend n < Vh satisfies n * d < 2^32
        if (d <= 1 || (unsigned long long)g.Vh * (unsigned long long)d >= (1ull << 32)) return 0u;
        return (unsigned)(((1ull << 32) + d - 1) / d);
    };
    g.mLh0 = magic(g.Lh0);
    g.mL1 = magic(g.L[1]);
    g.mL2 = magic(g.L[2]);
    g.mQ = magic(g.Lh0 / 2);
    g.mB = magic(g.b[0] / 2);
    for (int a = 0; a < 4; ++a) {
        // dividends are coordinates (< L_a); the check on Vh above is stricter
        g.mb[a] = magic(g.b[a]);
    }
}

// n / d with a precomputed multiplier (m = 0: plain division)
DD_DEV int fast_div(int n, int d, unsigned m) { return m ? (int)__umulhi((unsigned)n, m) : n / d; }

// coordinates of the site with parity p and even-odd index h (= canonical / 2)
DD_DEV void eo_coords(const Geo& g, int p, int h, int x[4]) {
    int r = fast_div(h, g.Lh0, g.mLh0);
    int hx = h - r * g.Lh0;
    int q = fast_div(r, g.L[1], g.mL1);
    x[1] = r - q * g.L[1];
    int t = fast_div(q, g.L[2], g.mL2);
    x[2] = q - t * g.L[2];
    x[3] = t;
    x[0] = 2 * hx + ((p + x[1] + x[2] + x[3]) & 1);
}

// The t-th site (increasing even-odd index h) of the blocks of colour c,
// for an even block extent along axis 0: every row (x1, x2, x3) holds Lh0/2
// such sites, in runs of b0/2 consecutive h (one run per block of that
// colour along axis 0, every second block).  Returns h; x = coordinates of
// the parity-p site h.  The same list the host stores in the colour maps.
DD_DEV int colour_site(const Geo& g, int c, int t, int p, int x[4]) {
    const int q = g.Lh0 >> 1;
    const int r = fast_div(t, q, g.mQ);
    const int u = t - r * q;
    const int B = g.b[0] >> 1;
    const int m = fast_div(u, B, g.mB);
    const int k = u - m * B;
    const int s1 = fast_div(r, g.L[1], g.mL1);
    x[1] = r - s1 * g.L[1];
    x[3] = fast_div(s1, g.L[2], g.mL2);
    x[2] = s1 - x[3] * g.L[2];
    const int cr = (fast_div(x[1], g.b[1], g.mb[1]) + fast_div(x[2], g.b[2], g.mb[2]) + fast_div(x[3], g.b[3], g.mb[3])) & 1;
    const int hx = (2 * m + ((c + cr) & 1)) * B + k;
    x[0] = 2 * hx + ((p + x[1] + x[2] + x[3]) & 1);
    return hx + g.Lh0 * r;
}

// canonical index of s +- a-hat from the coordinates x of s (periodic)
DD_DEV int neighbour_index(const Geo& g, int s, const int x[4], int a, int dir) {
    if (dir > 0) return (x[a] == g.L[a] - 1) ? s - (g.L[a] - 1) * g.st[a] : s + g.st[a];
    return (x[a] == 0) ? s + (g.L[a] - 1) * g.st[a] : s - g.st[a];
}
DD_HD int canon_index(const Geo& g, const int x[4]) { return x[0] + g.L[0] * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3])); }
DD_DEV void canon_coords(const Geo& g, int s, int x[4]) {
    x[0] = s % g.L[0];
    s /= g.L[0];
    x[1] = s % g.L[1];
    s /= g.L[1];
    x[2] = s % g.L[2];
    x[3] = s / g.L[2];
}
// canonical index of x +- a-hat (periodic)
DD_DEV int shift_index(const Geo& g, const int x[4], int a, int dir) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[a] += dir;
    if (y[a] == g.L[a]) y[a] = 0;
    if (y[a] < 0) y[a] = g.L[a] - 1;
    return canon_index(g, y);
}
// block id and block-ordered position of a site (black blocks first)
DD_DEV int block_id_of(const Geo& g, const int x[4]) {
    return x[0] / g.b[0] + g.nbk[0] * (x[1] / g.b[1] + g.nbk[1] * (x[2] / g.b[2] + g.nbk[2] * (x[3] / g.b[3])));
}
DD_DEV int block_colour_of(const Geo& g, const int x[4]) {
    return (x[0] / g.b[0] + x[1] / g.b[1] + x[2] / g.b[2] + x[3] / g.b[3]) & 1;
}
DD_DEV int local_index_of(const Geo& g, const int x[4]) {
    return x[0] % g.b[0] + g.b[0] * (x[1] % g.b[1] + g.b[1] * (x[2] % g.b[2] + g.b[2] * (x[3] % g.b[3])));
}
// position of block `id` in block order: colour * nblocks/2 + id/2 (needs an even number of blocks along axis 0)
DD_DEV int block_pos_of(const Geo& g, int id, int colour) { return colour * (g.nblocks / 2) + id / 2; }
DD_DEV long long dd_position(const Geo& g, const int x[4]) {
    int id = block_id_of(g, x);
    return (long long)block_pos_of(g, id, block_colour_of(g, x)) * g.bsites + local_index_of(g, x);
}

// --------------------------------------------------- Wilson spin projection
// Chiral basis: gamma_0 (time, lattice axis 3) = [[0,-1],[-1,0]],
// gamma_k (lattice axis k-1) = [[0,-i sigma_k],[i sigma_k,0]].
// Forward hop uses (1 - gamma_a), backward hop (1 + gamma_a).  With
// h = the upper-spin half of the projection, the lower half is
//   time:  (1 -+ gamma_0): lower = +-h
//   space: (1 -+ gamma_k): lower = -+ i sigma_k h.
// i sigma_1 v = (i v1, i v0), i sigma_2 v = (v1, -v0), i sigma_3 v = (i v0, -i v1).
template <class R>
DD_DEV void isigma(int a, const cpx<R>* v0, const cpx<R>* v1, cpx<R>* o0, cpx<R>* o1) {
    // v0, v1: the two spin components (3 colours each); result into o0, o1
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cpx<R> a0 = v0[c], a1 = v1[c];
        if (a == 0) {
            o0[c] = itimes(a1);
            o1[c] = itimes(a0);
        } else if (a == 1) {
            o0[c] = a1;
            o1[c] = -a0;
        } else {
            o0[c] = itimes(a0);
            o1[c] = -itimes(a1);
        }
    }
}

// sgn = +1: (1 - gamma_a) (forward); sgn = -1: (1 + gamma_a) (backward)
template <class R>
DD_DEV void project(int a, int sgn, const Spinor<R>& s, Half<R>& h) {
    if (a == 3) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h.c[k] = (sgn > 0) ? s.c[k] + s.c[k + 6] : s.c[k] - s.c[k + 6];
    } else {
        cpx<R> t0[3], t1[3];
        isigma<R>(a, &s.c[6], &s.c[9], t0, t1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            h.c[c] = (sgn > 0) ? s.c[c] + t0[c] : s.c[c] - t0[c];
            h.c[3 + c] = (sgn > 0) ? s.c[3 + c] + t1[c] : s.c[3 + c] - t1[c];
        }
    }
}

// acc += scale * (full spinor rebuilt from the projected half h)
template <class R>
DD_DEV void accumulate(int a, int sgn, const Half<R>& h, R scale, Spinor<R>& acc) {
#pragma unroll
    for (int k = 0; k < 6; ++k) acc.c[k] = acc.c[k] + scale * h.c[k];
    if (a == 3) {
        R s2 = (sgn > 0) ? scale : -scale;
#pragma unroll
        for (int k = 0; k < 6; ++k) acc.c[6 + k] = acc.c[6 + k] + s2 * h.c[k];
    } else {
        cpx<R> t0[3], t1[3];
        isigma<R>(a, &h.c[0], &h.c[3], t0, t1);
        R s2 = (sgn > 0) ? -scale : scale;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc.c[6 + c] = acc.c[6 + c] + s2 * t0[c];
            acc.c[9 + c] = acc.c[9 + c] + s2 * t1[c];
        }
    }
}

// colour matrix times half spinor: U h, or U^dag h
template <class R>
DD_DEV void mul_link(const Link<R>& u, const Half<R>& h, Half<R>& o) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cpx<R> acc = mk<R>(0, 0);
#pragma unroll
            for (int j = 0; j < 3; ++j) acc = cmac(acc, u.m[i][j], h.c[sp * 3 + j]);
            o.c[sp * 3 + i] = acc;
        }
}
template <class R>
DD_DEV void mul_link_dag(const Link<R>& u, const Half<R>& h, Half<R>& o) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cpx<R> acc = mk<R>(0, 0);
#pragma unroll
            for (int j = 0; j < 3; ++j) acc = cmacc(acc, u.m[j][i], h.c[sp * 3 + j]);
            o.c[sp * 3 + i] = acc;
        }
}

template <class R>
DD_DEV void gamma5(Spinor<R>& s) {
#pragma unroll
    for (int k = 6; k < 12; ++k) s.c[k] = -s.c[k];
}

template <class R>
DD_DEV void zero(Spinor<R>& s) {
#pragma unroll
    for (int k = 0; k < 12; ++k) s.c[k] = mk<R>(0, 0);
}

template <class R>
DD_DEV R snorm2(const Spinor<R>& s) {
    R r = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) r += norm2(s.c[k]);
    return r;
}

// counter of a random stream: the call's counter plus the device offset of
// a graph replay (off may be null)
DD_DEV uint64_t stream_ctr(uint64_t ctr, const unsigned long long* off) { return off ? ctr + *off : ctr; }

// ------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
struct U4 {
    uint32_t x, y, z, w;
};
DD_HD U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * c.x;
        uint64_t p1 = (uint64_t)M1 * c.z;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
    }
    return c;
}
// stream words for (element, purpose, sub, seed, ctr)
DD_HD U4 rng_words(uint32_t element, uint32_t purpose, uint32_t sub, uint64_t seed, uint64_t ctr) {
    U4 c;
    c.x = element;
    c.y = (purpose << 24) | (sub & 0xFFFFFFu);
    c.z = (uint32_t)ctr;
    c.w = (uint32_t)(ctr >> 32);
    return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}
// 53-bit uniform strictly inside (0, 1) from two words
DD_HD double words_to_uniform(uint32_t a, uint32_t b) {
    uint64_t k = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
    return ((double)k + 0.5) * 1.1102230246251565404e-16;  // 2^-53
}
DD_DEV void uniform_pair(uint32_t element, uint32_t purpose, uint32_t sub, uint64_t seed, uint64_t ctr, double& u1,
                         double& u2) {
    U4 w = rng_words(element, purpose, sub, seed, ctr);
    u1 = words_to_uniform(w.x, w.y);
    u2 = words_to_uniform(w.z, w.w);
}
// complex Gaussian with density ~ exp(-|z|^2) (Box-Muller)
DD_DEV cpx<double> gaussian(uint32_t element, uint32_t purpose, uint32_t sub, uint64_t seed, uint64_t ctr) {
    double u1, u2;
    uniform_pair(element, purpose, sub, seed, ctr, u1, u2);
    double r = sqrt(-log(u1));
    double ang = 6.283185307179586477 * u2;
    return mk<double>(r * cos(ang), r * sin(ang));
}

// ---------------------------------------------------------------- reductions
DD_DEV double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Sum over the thread block (deterministic for a fixed block size); the
// result is valid in every thread.  `sh` needs 33 doubles.
DD_DEV double block_sum(double v, double* sh) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[32] = t;
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

// device status word (first error wins)
DD_DEV void raise_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}
