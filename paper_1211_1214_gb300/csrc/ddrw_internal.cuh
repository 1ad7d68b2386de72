// ddrw_internal.cuh -- layouts, geometry and per-site arithmetic shared by the CUDA kernels.
//
// Operator (the Wilson-clover Dirac operator the paper uses, Sec. 1 and Sec. 2; normalisation in
// the mass-additive form that M = 1 + dm D^-1(m2) of Eq. 6 needs):
//
//   (D(m) psi)(x) = A(m)(x) psi(x) - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
//   A(m)(x)       = (4 + m) + C(x),   C = csw (i/4) sum_{mu nu} sigma_{mu nu} Fhat_{mu nu}
//
// Chiral basis: g_mu = [[0, e_mu], [e_mu^dag, 0]] in 2x2 spin blocks with e_0 = -1 and
// e_k = -i sigma_k, so g5 = diag(1, 1, -1, -1) and C is two Hermitian 6x6 blocks (spins 0,1 and
// spins 2,3), each indexed by 3*(spin within the pair) + colour.
//
// Internal site order ("block-major, even-odd split"): with hypercubic blocks of length BL,
//
//   s = p * V/2 + blk * BL^4/2 + h,
//
// p the site parity (t+x+y+z) mod 2, blk the block number with all black blocks first (colour
// of a block = sum of its block coordinates mod 2, block 0 black), h = (in-block lexicographic
// index) / 2.  Every block origin has even coordinates, so the in-block parity is the global
// parity; the sites of one block and one parity are contiguous, and so are the sites of one
// colour and one parity.
//
// Fields are structure-of-arrays over sites: plane k of site s at base[k * stride + s], each
// element 16 bytes (double2 / float4), one field per right-hand side.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ddrw {

constexpr int MAXM = 8;  // mass slots per launch (right-hand sides grouped by mass)

// ----------------------------------------------------------------------------- geometry

struct GeomDev {
    int L[4];          // T, X, Y, Z
    int NB[4];         // blocks per direction (all even, >= 2)
    int nblk;          // number of blocks
    int nblk_c;        // blocks of one colour
    long vh;           // V / 2
    long V;
    const int *blk_nb;  // [nblk][8]: neighbour block in direction 2*mu (+mu) and 2*mu+1 (-mu)
    const int *blk_org; // [nblk][4]: coordinates of the block origin
    const int *blk_index; // [nblk]: block number of the block with lexicographic block index B
    int tsign;          // -1: antiperiodic in time, +1: periodic
    const int4 *nbr;    // [2][V] neighbour table (see NBR_IDX), nullptr while not built
};

// Neighbour table: for site s, nbr[s] = (+0, -0, +1, -1) and nbr[V + s] = (+2, -2, +3, -3), each
// entry the internal index of the neighbour in that direction (bits 0-29), bit 30 set when the hop
// leaves the block, bit 31 (the sign bit) set when the hop crosses the time boundary of the lattice
// (where antiperiodic fields change sign).  Built once per geometry by the same neighbour()
// arithmetic the other kernels use.
constexpr int NBR_IDX = 0x3fffffff;
constexpr int NBR_CROSS = 0x40000000;

template <int BL> struct BlockShape {
    static constexpr int VB = BL * BL * BL * BL;
    static constexpr int VBH = VB / 2;
    static constexpr int ROWH = BL / 2;  // half-sites per z-row
};

template <int BL> struct Site {
    int p, blk, h;
    int c[4];  // in-block coordinates
};

template <int BL>
__device__ __forceinline__ void decode_site(long s, const GeomDev &g, Site<BL> &st)
{
    st.p = (s >= g.vh) ? 1 : 0;
    long r = s - (long)st.p * g.vh;
    st.blk = (int)(r / BlockShape<BL>::VBH);
    st.h = (int)(r - (long)st.blk * BlockShape<BL>::VBH);
    int row = st.h / BlockShape<BL>::ROWH;
    int izh = st.h - row * BlockShape<BL>::ROWH;
    st.c[2] = row % BL;
    row /= BL;
    st.c[1] = row % BL;
    st.c[0] = row / BL;
    st.c[3] = 2 * izh + ((st.c[0] + st.c[1] + st.c[2] + st.p) & 1);
}

// Neighbour of st one step in direction mu (dir = +1/-1).  *cross is set when the hop leaves the
// block; *phase is the boundary sign of the hop.
template <int BL>
__device__ __forceinline__ int neighbour(const Site<BL> &st, int mu, int dir, const GeomDev &g, bool *cross,
                                         int *phase)
{
    int c0 = st.c[0], c1 = st.c[1], c2 = st.c[2], c3 = st.c[3];
    int cm = st.c[mu] + dir;
    int blk = st.blk;
    *cross = false;
    *phase = 1;
    if (cm < 0 || cm >= BL) {
        *cross = true;
        blk = g.blk_nb[st.blk * 8 + 2 * mu + (dir < 0 ? 1 : 0)];
        if (mu == 0 && g.tsign < 0) {
            int t = g.blk_org[st.blk * 4] + st.c[0];
            if ((dir > 0 && t == g.L[0] - 1) || (dir < 0 && t == 0)) *phase = -1;
        }
        cm = (cm < 0) ? BL - 1 : 0;
    }
    if (mu == 0) c0 = cm;
    else if (mu == 1) c1 = cm;
    else if (mu == 2) c2 = cm;
    else c3 = cm;
    int lb = ((c0 * BL + c1) * BL + c2) * BL + c3;
    return (1 - st.p) * (int)g.vh + blk * BlockShape<BL>::VBH + (lb >> 1);
}

// lexicographic site index of an internal site (boundary layout)
template <int BL>
__device__ __forceinline__ long lex_index(const Site<BL> &st, const GeomDev &g)
{
    const int *o = g.blk_org + st.blk * 4;
    int t = o[0] + st.c[0], x = o[1] + st.c[1], y = o[2] + st.c[2], z = o[3] + st.c[3];
    return (((long)t * g.L[1] + x) * g.L[2] + y) * g.L[3] + z;
}

// internal index of the site with global coordinates (t, x, y, z), all in range
template <int BL>
__device__ __forceinline__ long internal_index(const GeomDev &g, int t, int x, int y, int z)
{
    int bt = t / BL, bx = x / BL, by = y / BL, bz = z / BL;
    int B = ((bt * g.NB[1] + bx) * g.NB[2] + by) * g.NB[3] + bz;
    int blk = g.blk_index[B];
    int lb = (((t - bt * BL) * BL + (x - bx * BL)) * BL + (y - by * BL)) * BL + (z - bz * BL);
    int p = (t + x + y + z) & 1;
    return (long)p * g.vh + (long)blk * BlockShape<BL>::VBH + (lb >> 1);
}

// ----------------------------------------------------------------------------- complex arithmetic

template <typename R> struct cpx {
    R re, im;
};

template <typename R> __device__ __forceinline__ cpx<R> mk(R a, R b) { return cpx<R>{a, b}; }
template <typename R> __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ cpx<R> operator-(cpx<R> a) { return {-a.re, -a.im}; }
template <typename R> __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> __device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __device__ __forceinline__ cpx<R> cmulc(cpx<R> a, cpx<R> b)  // conj(a) * b
{
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// Complex multiply-accumulate as explicit fused multiply-adds: acc + a b written as
// (acc + a.re b) + (i-rotated a.im b) takes 4 FMAs, while acc + cmul(a, b) leaves the compiler
// 2 multiplies, 2 FMAs and 2 adds (it does not reassociate the sum).
__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }
template <typename R> __device__ __forceinline__ void cmac(cpx<R> &acc, cpx<R> a, cpx<R> b)  // acc += a b
{
    acc.re = fmad(a.re, b.re, fmad(-a.im, b.im, acc.re));
    acc.im = fmad(a.re, b.im, fmad(a.im, b.re, acc.im));
}
template <typename R> __device__ __forceinline__ void cmacc(cpx<R> &acc, cpx<R> a, cpx<R> b)  // acc += conj(a) b
{
    acc.re = fmad(a.re, b.re, fmad(a.im, b.im, acc.re));
    acc.im = fmad(a.re, b.im, fmad(-a.im, b.re, acc.im));
}
template <typename R> __device__ __forceinline__ void cmsub(cpx<R> &acc, cpx<R> a, cpx<R> b)  // acc -= a b
{
    acc.re = fmad(-a.re, b.re, fmad(a.im, b.im, acc.re));
    acc.im = fmad(-a.re, b.im, fmad(-a.im, b.re, acc.im));
}
template <typename R> __device__ __forceinline__ cpx<R> timesI(cpx<R> a) { return {-a.im, a.re}; }
template <typename R> __device__ __forceinline__ cpx<R> timesMinusI(cpx<R> a) { return {a.im, -a.re}; }

template <typename R> struct Spinor {
    cpx<R> v[4][3];
};
template <typename R> struct Half {
    cpx<R> v[2][3];
};
template <typename R> struct Link {
    cpx<R> m[3][3];
};

template <typename R> __device__ __forceinline__ void zero(Spinor<R> &s)
{
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) s.v[a][c] = {R(0), R(0)};
}

// ----------------------------------------------------------------------------- spin projection
// (1 - g_mu) psi = (h, -e_mu^dag h) with h = psi_u - e_mu psi_d;
// (1 + g_mu) psi = (h,  e_mu^dag h) with h = psi_u + e_mu psi_d.
// sign = -1 selects (1 - g_mu), sign = +1 selects (1 + g_mu).

template <int MU, int SIGN, typename R>
__device__ __forceinline__ void project(const Spinor<R> &p, Half<R> &h)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cpx<R> d0 = p.v[2][c], d1 = p.v[3][c];
        cpx<R> e0, e1;  // e_mu psi_d
        if (MU == 0) { e0 = -d0; e1 = -d1; }
        else if (MU == 1) { e0 = timesMinusI(d1); e1 = timesMinusI(d0); }
        else if (MU == 2) { e0 = -d1; e1 = d0; }
        else { e0 = timesMinusI(d0); e1 = timesI(d1); }
        if (SIGN > 0) { h.v[0][c] = p.v[0][c] + e0; h.v[1][c] = p.v[1][c] + e1; }
        else { h.v[0][c] = p.v[0][c] - e0; h.v[1][c] = p.v[1][c] - e1; }
    }
}

// Storage policies whose spinors carry a per-site norm (16-bit storage) declare NORMED = true.
template <class P, class = void> struct Normed {
    static constexpr bool value = false;
};
template <class P> struct Normed<P, decltype((void)P::NORMED)> {
    static constexpr bool value = P::NORMED;
};

// acc += n (1 +- g_mu)-reconstruction of the half spinor w, the scale n folded into the FMAs that
// add the hop (a 16-bit neighbour's norm and the boundary sign cost no separate multiplies)
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void reconstruct_add_scaled(Spinor<R> &acc, const Half<R> &w, R n)
{
    const R ns = SIGN > 0 ? n : -n;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cpx<R> w0 = w.v[0][c], w1 = w.v[1][c];
        cpx<R> f0, f1;  // e_mu^dag w
        if (MU == 0) { f0 = -w0; f1 = -w1; }
        else if (MU == 1) { f0 = timesI(w1); f1 = timesI(w0); }
        else if (MU == 2) { f0 = w1; f1 = -w0; }
        else { f0 = timesI(w0); f1 = timesMinusI(w1); }
        acc.v[0][c].re = fmad(n, w0.re, acc.v[0][c].re);
        acc.v[0][c].im = fmad(n, w0.im, acc.v[0][c].im);
        acc.v[1][c].re = fmad(n, w1.re, acc.v[1][c].re);
        acc.v[1][c].im = fmad(n, w1.im, acc.v[1][c].im);
        acc.v[2][c].re = fmad(ns, f0.re, acc.v[2][c].re);
        acc.v[2][c].im = fmad(ns, f0.im, acc.v[2][c].im);
        acc.v[3][c].re = fmad(ns, f1.re, acc.v[3][c].re);
        acc.v[3][c].im = fmad(ns, f1.im, acc.v[3][c].im);
    }
}

// acc += coef * (1 +- g_mu)-reconstruction of the half spinor w
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void reconstruct_add(Spinor<R> &acc, const Half<R> &w)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cpx<R> w0 = w.v[0][c], w1 = w.v[1][c];
        cpx<R> f0, f1;  // e_mu^dag w
        if (MU == 0) { f0 = -w0; f1 = -w1; }
        else if (MU == 1) { f0 = timesI(w1); f1 = timesI(w0); }
        else if (MU == 2) { f0 = w1; f1 = -w0; }
        else { f0 = timesI(w0); f1 = timesMinusI(w1); }
        acc.v[0][c] = acc.v[0][c] + w0;
        acc.v[1][c] = acc.v[1][c] + w1;
        if (SIGN > 0) { acc.v[2][c] = acc.v[2][c] + f0; acc.v[3][c] = acc.v[3][c] + f1; }
        else { acc.v[2][c] = acc.v[2][c] - f0; acc.v[3][c] = acc.v[3][c] - f1; }
    }
}

template <typename R>
__device__ __forceinline__ void link_mul(const Link<R> &U, const Half<R> &h, Half<R> &w)
{
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cpx<R> t = cmul(U.m[a][0], h.v[s][0]);
            cmac(t, U.m[a][1], h.v[s][1]);
            cmac(t, U.m[a][2], h.v[s][2]);
            w.v[s][a] = t;
        }
}

template <typename R>
__device__ __forceinline__ void link_dag_mul(const Link<R> &U, const Half<R> &h, Half<R> &w)
{
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cpx<R> t = cmulc(U.m[0][a], h.v[s][0]);
            cmacc(t, U.m[1][a], h.v[s][1]);
            cmacc(t, U.m[2][a], h.v[s][2]);
            w.v[s][a] = t;
        }
}

// ----------------------------------------------------------------------------- storage policies
//
// A policy P gives the arithmetic type P::R and how spinors, links and clover blocks are stored.
//   PrecD: FP64 everything, full 3x3 links (9 double2 planes per direction), clover 36 double2.
//   PrecS: FP32 spinors (6 float4 planes), two-row links (3 float4 planes), clover 18 float4.
//   PrecH / PrecB (lowprec.cuh): FP16 / BF16 storage with per-site norms, FP32 arithmetic.
// BLAS kernels reach a field through ld_chunk / st_chunk: NCHUNK chunks of CW complex numbers per
// site (a 16-bit site is one chunk, because its norm covers all 12 components).

struct PrecD {
    using R = double;
    using SElem = double2;
    static constexpr int ID = 64;
    static constexpr int SPLANES = 12;
    static constexpr int UPLANES = 9;   // per direction
    static constexpr int CPLANES = 36;  // per site, both chiralities
    static constexpr double SBYTES = 192, UBYTES = 144, CBYTES = 576;  // spinor, link, clover
    static constexpr int NCHUNK = 12, CW = 1;  // BLAS granularity: one element of one complex
    using UElem = double2;
    using CElem = double2;
    __host__ __device__ static long field_elems(long V) { return SPLANES * V; }
    __device__ static __forceinline__ void ld_chunk(const SElem *f, long V, long s, int k, cpx<R> *c)
    {
        double2 v = f[k * V + s];
        c[0] = {v.x, v.y};
    }
    __device__ static __forceinline__ void st_chunk(SElem *f, long V, long s, int k, const cpx<R> *c)
    {
        f[k * V + s] = make_double2(c[0].re, c[0].im);
    }

    // in-field offsets are 32-bit (k * stride + s < 2^31: at most 2^27 sites)
    __device__ static __forceinline__ void load_spinor(const SElem *__restrict__ f, int stride, int s, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 12; k++) {
            double2 v = __ldg(f + (k * stride + s));
            p.v[k / 3][k % 3] = {v.x, v.y};
        }
    }
    __device__ static __forceinline__ void load_spinor_rw(const SElem *f, int stride, int s, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 12; k++) {
            double2 v = f[k * stride + s];
            p.v[k / 3][k % 3] = {v.x, v.y};
        }
    }
    __device__ static __forceinline__ void store_spinor(SElem *__restrict__ f, int stride, int s, const Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 12; k++) f[k * stride + s] = make_double2(p.v[k / 3][k % 3].re, p.v[k / 3][k % 3].im);
    }
    // the 6 components of chirality ch (spins 2ch, 2ch+1): planes 6ch .. 6ch+5
    __device__ static __forceinline__ void load_chiral(const SElem *__restrict__ f, int stride, int s, int ch, cpx<R> *v)
    {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            double2 e = __ldg(f + ((6 * ch + k) * stride + s));
            v[k] = {e.x, e.y};
        }
    }
    __device__ static __forceinline__ void load_link(const UElem *__restrict__ U, int V, int mu, int s, Link<R> &L)
    {
        const UElem *b = U + (long)mu * 9 * V;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            double2 v = __ldg(b + (k * V + s));
            L.m[k / 3][k % 3] = {v.x, v.y};
        }
    }
    // raw loads (all issued before any decode) for the batched hop form
    struct SRaw {
        double2 e[12];
    };
    struct URaw {
        double2 e[9];
    };
    __device__ static __forceinline__ void load_raw(const SElem *__restrict__ f, int stride, int s, SRaw &r)
    {
#pragma unroll
        for (int k = 0; k < 12; k++) r.e[k] = __ldg(f + (k * stride + s));
    }
    __device__ static __forceinline__ void decode(const SRaw &r, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 12; k++) p.v[k / 3][k % 3] = {r.e[k].x, r.e[k].y};
    }
    __device__ static __forceinline__ void load_link_raw(const UElem *__restrict__ U, int V, int mu, int s, URaw &r)
    {
        const UElem *b = U + (long)mu * 9 * V;
#pragma unroll
        for (int k = 0; k < 9; k++) r.e[k] = __ldg(b + (k * V + s));
    }
    __device__ static __forceinline__ void decode_link(const URaw &r, Link<R> &L)
    {
#pragma unroll
        for (int k = 0; k < 9; k++) L.m[k / 3][k % 3] = {r.e[k].x, r.e[k].y};
    }
    // reals 0..35 of chirality block ch
    __device__ static __forceinline__ void load_clover(const CElem *__restrict__ Cl, int V, int s, int ch, R *c)
    {
        const CElem *b = Cl + (long)ch * 18 * V;
#pragma unroll
        for (int k = 0; k < 18; k++) {
            double2 v = __ldg(b + (k * V + s));
            c[2 * k] = v.x;
            c[2 * k + 1] = v.y;
        }
    }
};

struct PrecS {
    using R = float;
    using SElem = float4;
    static constexpr int ID = 32;
    static constexpr int SPLANES = 6;
    static constexpr int UPLANES = 3;
    static constexpr int CPLANES = 18;
    static constexpr double SBYTES = 96, UBYTES = 48, CBYTES = 288;
    static constexpr int NCHUNK = 6, CW = 2;
    using UElem = float4;
    using CElem = float4;
    __host__ __device__ static long field_elems(long V) { return SPLANES * V; }
    __device__ static __forceinline__ void ld_chunk(const SElem *f, long V, long s, int k, cpx<R> *c)
    {
        float4 v = f[k * V + s];
        c[0] = {v.x, v.y};
        c[1] = {v.z, v.w};
    }
    __device__ static __forceinline__ void st_chunk(SElem *f, long V, long s, int k, const cpx<R> *c)
    {
        f[k * V + s] = make_float4(c[0].re, c[0].im, c[1].re, c[1].im);
    }

    __device__ static __forceinline__ void load_spinor(const SElem *__restrict__ f, int stride, int s, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float4 v = __ldg(f + (k * stride + s));
            p.v[(2 * k) / 3][(2 * k) % 3] = {v.x, v.y};
            p.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = {v.z, v.w};
        }
    }
    __device__ static __forceinline__ void load_spinor_rw(const SElem *f, int stride, int s, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float4 v = f[k * stride + s];
            p.v[(2 * k) / 3][(2 * k) % 3] = {v.x, v.y};
            p.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = {v.z, v.w};
        }
    }
    __device__ static __forceinline__ void store_spinor(SElem *__restrict__ f, int stride, int s, const Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            cpx<R> a = p.v[(2 * k) / 3][(2 * k) % 3], b = p.v[(2 * k + 1) / 3][(2 * k + 1) % 3];
            f[k * stride + s] = make_float4(a.re, a.im, b.re, b.im);
        }
    }
    // the 6 components of chirality ch (spins 2ch, 2ch+1): planes 3ch .. 3ch+2
    __device__ static __forceinline__ void load_chiral(const SElem *__restrict__ f, int stride, int s, int ch, cpx<R> *v)
    {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float4 e = __ldg(f + ((3 * ch + k) * stride + s));
            v[2 * k] = {e.x, e.y};
            v[2 * k + 1] = {e.z, e.w};
        }
    }
    // two stored rows; row 2 = conj(row0 x row1) (U in SU(3))
    __device__ static __forceinline__ void load_link(const UElem *__restrict__ U, int V, int mu, int s, Link<R> &L)
    {
        const UElem *b = U + (long)mu * 3 * V;
        float4 a0 = __ldg(b + s), a1 = __ldg(b + (V + s)), a2 = __ldg(b + (2 * V + s));
        L.m[0][0] = {a0.x, a0.y};
        L.m[0][1] = {a0.z, a0.w};
        L.m[0][2] = {a1.x, a1.y};
        L.m[1][0] = {a1.z, a1.w};
        L.m[1][1] = {a2.x, a2.y};
        L.m[1][2] = {a2.z, a2.w};
        reconstruct_row2(L);
    }
    struct SRaw {
        float4 e[6];
    };
    struct URaw {
        float4 e[3];
    };
    __device__ static __forceinline__ void load_raw(const SElem *__restrict__ f, int stride, int s, SRaw &r)
    {
#pragma unroll
        for (int k = 0; k < 6; k++) r.e[k] = __ldg(f + (k * stride + s));
    }
    __device__ static __forceinline__ void decode(const SRaw &r, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            p.v[(2 * k) / 3][(2 * k) % 3] = {r.e[k].x, r.e[k].y};
            p.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = {r.e[k].z, r.e[k].w};
        }
    }
    __device__ static __forceinline__ void load_link_raw(const UElem *__restrict__ U, int V, int mu, int s, URaw &r)
    {
        const UElem *b = U + (long)mu * 3 * V;
        r.e[0] = __ldg(b + s);
        r.e[1] = __ldg(b + (V + s));
        r.e[2] = __ldg(b + (2 * V + s));
    }
    __device__ static __forceinline__ void decode_link(const URaw &r, Link<R> &L)
    {
        L.m[0][0] = {r.e[0].x, r.e[0].y};
        L.m[0][1] = {r.e[0].z, r.e[0].w};
        L.m[0][2] = {r.e[1].x, r.e[1].y};
        L.m[1][0] = {r.e[1].z, r.e[1].w};
        L.m[1][1] = {r.e[2].x, r.e[2].y};
        L.m[1][2] = {r.e[2].z, r.e[2].w};
        reconstruct_row2(L);
    }
    __device__ static __forceinline__ void reconstruct_row2(Link<R> &L)
    {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            int i = (c + 1) % 3, j = (c + 2) % 3;
            cpx<R> t = cmul(L.m[0][i], L.m[1][j]);
            cmsub(t, L.m[0][j], L.m[1][i]);
            L.m[2][c] = {t.re, -t.im};
        }
    }
    __device__ static __forceinline__ void load_clover(const CElem *__restrict__ Cl, int V, int s, int ch, R *c)
    {
        const CElem *b = Cl + (long)ch * 9 * V;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            float4 v = __ldg(b + (k * V + s));
            c[4 * k] = v.x;
            c[4 * k + 1] = v.y;
            c[4 * k + 2] = v.z;
            c[4 * k + 3] = v.w;
        }
    }
};

// Hermitian 6x6 block stored as 36 reals: d[0..5] the real diagonal, then the 15 entries above
// the diagonal, row by row, as (re, im).  Index of (i, j), i < j, in that list:
__host__ __device__ constexpr int herm_off(int i, int j) { return i * 5 - (i * (i - 1)) / 2 + (j - i - 1); }

// out = (diag + H) v for a Hermitian 6x6 H in packed form
template <typename R>
__device__ __forceinline__ void herm6_mul(const R *c, R diag, const cpx<R> *v, cpx<R> *out)
{
#pragma unroll
    for (int i = 0; i < 6; i++) out[i] = (diag + c[i]) * v[i];
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            int o = 6 + 2 * herm_off(i, j);
            cpx<R> hij = {c[o], c[o + 1]};
            cmac(out[i], hij, v[j]);
            cmacc(out[j], hij, v[i]);
        }
}

// ----------------------------------------------------------------------------- host helpers

#define DDRW_CUDA_CHECK(call)                                                                         \
    do {                                                                                              \
        cudaError_t err__ = (call);                                                                   \
        if (err__ != cudaSuccess) return ::ddrw::set_cuda_error(ctx, err__, #call, __FILE__, __LINE__); \
    } while (0)

}  // namespace ddrw
