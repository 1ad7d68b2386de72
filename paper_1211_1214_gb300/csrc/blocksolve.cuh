// blocksolve.cuh -- the persistent block-solver kernel (K6); instantiated per storage policy and
// block length in blocksolve_<policy><l>.cu so that the instantiations compile in parallel.
#pragma once

#include "blas.cuh"
#include "ctx.h"
#include "lowprec.cuh"
#include "stencil.cuh"

namespace ddrw {

template <class P> struct BlkArgs {
    using E = typename P::SElem;
    const E *b;
    E *x;
    E *r, *rh, *p, *v, *t, *tmp;
    long rstride;
    const typename P::UElem *U;
    const typename P::CElem *Cl;
    int rpm;
    typename P::R mass4[MAXM];
    const typename P::CElem *Ainv[MAXM];
    int blk0;
    double tol2;
    const double *tol2_dev = nullptr;  // if set, the tolerance is read from device memory (captured graphs)
    int maxiter;
    int *stat;  // [0] max iterations, [1] blocks that missed the tolerance
};

template <int K, int NT>
__device__ __forceinline__ void cta_sum(double (&v)[K], double (*sm)[K])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) {
        double a = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        v[k] = a;
    }
    __syncthreads();  // earlier readers of sm are done
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sm[w][k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) {
        double s = 0;
#pragma unroll
        for (int i = 0; i < NT / 32; i++) s += sm[i][k];
        v[k] = s;
    }
}

template <typename R>
__device__ __forceinline__ void sp_norm_dot(const Spinor<R> &a, const Spinor<R> &b, R &re, R &im)
{  // += conj(a) b
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            cpx<R> z = cmulc(a.v[sp][c], b.v[sp][c]);
            re += z.re;
            im += z.im;
        }
}

template <typename R>
__device__ __forceinline__ R sp_norm2(const Spinor<R> &a)
{
    R s = 0;
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
        for (int c = 0; c < 3; c++) s += a.v[sp][c].re * a.v[sp][c].re + a.v[sp][c].im * a.v[sp][c].im;
    return s;
}

// Per-site pieces of the block operator, kept out of line so that every phase of the kernel
// reuses one register allocation (the fully unrolled stencil is large).

// odd site s:  out(s) = A_oo^-1 ( y(s) + coef * H_intra in (s) )    (y may be null, coef 0 skips the hop)
template <class P, int BL>
__device__ __noinline__ void site_odd(const GeomDev &g, long s, const typename P::SElem *in,
                                      const typename P::SElem *y, typename P::R coef,
                                      const typename P::UElem *__restrict__ U,
                                      const typename P::CElem *__restrict__ Ainv, typename P::SElem *out)
{
    using R = typename P::R;
    Spinor<R> acc;
    zero(acc);
    if (coef != R(0)) {
        Site<BL> st;
        decode_site<BL>(s, g, st);
        hop_sum<P, BL, 1, false>(g, st, s, in, U, acc);
        scale(acc, coef);
    }
    if (y) {
        Spinor<R> q;
        P::load_spinor_rw(y, g.V, s, q);
        axpy(acc, R(1), q);
    }
    clover_apply<P>(Ainv, g.V, s, R(0), acc);
    P::store_spinor(out, g.V, s, acc);
}

template <typename R> struct Dot3 {
    R a, b, c;
};

// even site s:  out(s) = D(x)(s) + coef * H_intra tmp (s), D = A(m) (diag) or 1, and the partial
// inner products of the phase: mode 1 -> conj(w) out; mode 2 -> conj(out) x and |out|^2.
template <class P, int BL>
__device__ __noinline__ Dot3<typename P::R> site_even(const GeomDev &g, long s, const typename P::SElem *tmp,
                                                      const typename P::SElem *x, typename P::R coef, bool diag,
                                                      typename P::R mass4, const typename P::UElem *__restrict__ U,
                                                      const typename P::CElem *__restrict__ Cl,
                                                      const typename P::SElem *w, int mode, typename P::SElem *out)
{
    using R = typename P::R;
    Spinor<R> acc, q;
    zero(acc);
    Site<BL> st;
    decode_site<BL>(s, g, st);
    hop_sum<P, BL, 1, false>(g, st, s, tmp, U, acc);
    scale(acc, coef);
    P::load_spinor_rw(x, g.V, s, q);
    Dot3<R> d{R(0), R(0), R(0)};
    if (diag) {
        Spinor<R> dq = q;
        clover_apply<P>(Cl, g.V, s, mass4, dq);
        axpy(acc, R(1), dq);
    } else {
        axpy(acc, R(1), q);
    }
    P::store_spinor(out, g.V, s, acc);
    if (mode == 1) {
        P::load_spinor_rw(w, g.V, s, q);
        sp_norm_dot(q, acc, d.a, d.b);
    } else if (mode == 2) {
        sp_norm_dot(acc, q, d.a, d.b);
        d.c = sp_norm2(acc);
    }
    return d;
}

template <class P, int BL, int NT>
// 32-bit arithmetic: at most 128 registers (170 for 128 threads) -- two 256-thread CTAs or one
// 512-thread CTA per SM -- so the register allocation keeps the occupancy of the out-of-line site
// functions
__global__ void __launch_bounds__(NT, sizeof(typename P::R) == 4 ? (NT >= 512 ? 1 : NT >= 256 ? 2 : NT >= 128 ? 3 : 1) : 1)
    k_block_solve(GeomDev g, BlkArgs<P> a)
{
    using R = typename P::R;
    using E = typename P::SElem;
    constexpr int VBH = BlockShape<BL>::VBH;
    constexpr int NP = P::NCHUNK, CW = P::CW;
    __shared__ double sm[NT / 32][3];
    // right-hand side fastest: the CTAs of one block run together and share its links in L2
    const int rhs = blockIdx.x;
    const int blk = a.blk0 + blockIdx.y;
    const long ro = (long)rhs * a.rstride;
    const int slot = rhs / a.rpm;
    const R mass4 = a.mass4[slot];
    const typename P::CElem *Ainv = a.Ainv[slot];
    const long e0 = (long)blk * VBH, o0 = g.vh + (long)blk * VBH;
    const long V = g.V;
    const E *b = a.b + ro;
    E *x = a.x + ro, *r = a.r + ro, *rh = a.rh + ro, *p = a.p + ro, *v = a.v + ro, *t = a.t + ro, *tmp = a.tmp + ro;

    // ||b||^2 over the block; tmp_o = A_oo^-1 b_o
    R bbl = 0;
    for (int h = threadIdx.x; h < VBH; h += NT)
        for (int k = 0; k < NP; k++) {
            cpx<R> c[CW], d[CW];
            P::ld_chunk(b, V, e0 + h, k, c);
            P::ld_chunk(b, V, o0 + h, k, d);
#pragma unroll
            for (int q = 0; q < CW; q++)
                bbl += c[q].re * c[q].re + c[q].im * c[q].im + d[q].re * d[q].re + d[q].im * d[q].im;
        }
    for (int h = threadIdx.x; h < VBH; h += NT) site_odd<P, BL>(g, o0 + h, nullptr, b, R(0), a.U, Ainv, tmp);
    double red[3] = {(double)bbl, 0, 0};
    cta_sum<3, NT>(red, sm);
    const double bb = red[0];
    // r = b_e + 1/2 H_eo tmp_o ; rh = p = r ; x_e = 0
    for (int h = threadIdx.x; h < VBH; h += NT)
        site_even<P, BL>(g, e0 + h, tmp, b, R(0.5), false, mass4, a.U, a.Cl, nullptr, 0, r);
    R rl = 0;
    for (int h = threadIdx.x; h < VBH; h += NT)
        for (int k = 0; k < NP; k++) {
            cpx<R> c[CW], z[CW];
            P::ld_chunk(r, V, e0 + h, k, c);
#pragma unroll
            for (int q = 0; q < CW; q++) {
                rl += c[q].re * c[q].re + c[q].im * c[q].im;
                z[q] = {R(0), R(0)};
            }
            P::st_chunk(rh, V, e0 + h, k, c);
            P::st_chunk(p, V, e0 + h, k, c);
            P::st_chunk(x, V, e0 + h, k, z);
        }
    red[0] = (double)rl;
    cta_sum<3, NT>(red, sm);
    double rr = red[0];
    double2 rho = make_double2(rr, 0.0);
    const double thresh = (a.tol2_dev ? *a.tol2_dev : a.tol2) * bb;
    int it = 0;
    bool ok = rr <= thresh;
    while (!ok && it < a.maxiter) {
        // v = S p  and  (rh, v)
        for (int h = threadIdx.x; h < VBH; h += NT) site_odd<P, BL>(g, o0 + h, p, nullptr, R(1), a.U, Ainv, tmp);
        __syncthreads();
        R are = 0, aim = 0;
        for (int h = threadIdx.x; h < VBH; h += NT) {
            Dot3<R> d = site_even<P, BL>(g, e0 + h, tmp, p, R(-0.25), true, mass4, a.U, a.Cl, rh, 1, v);
            are += d.a;
            aim += d.b;
        }
        red[0] = (double)are;
        red[1] = (double)aim;
        cta_sum<3, NT>(red, sm);
        double den = red[0] * red[0] + red[1] * red[1];
        if (den == 0.0 || !(den == den)) break;
        double2 alpha = make_double2((rho.x * red[0] + rho.y * red[1]) / den, (rho.y * red[0] - rho.x * red[1]) / den);
        const cpx<R> al = {R(alpha.x), R(alpha.y)};
        // s = r - alpha v (in r)
        for (int h = threadIdx.x; h < VBH; h += NT)
            for (int k = 0; k < NP; k++) {
                    cpx<R> c[CW], d[CW];
                P::ld_chunk(r, V, e0 + h, k, c);
                P::ld_chunk(v, V, e0 + h, k, d);
#pragma unroll
                for (int q = 0; q < CW; q++) c[q] = c[q] - cmul(al, d[q]);
                P::st_chunk(r, V, e0 + h, k, c);
            }
        __syncthreads();
        // t = S s  and  (t, s), (t, t)
        for (int h = threadIdx.x; h < VBH; h += NT) site_odd<P, BL>(g, o0 + h, r, nullptr, R(1), a.U, Ainv, tmp);
        __syncthreads();
        R tsr = 0, tsi = 0, tt = 0;
        for (int h = threadIdx.x; h < VBH; h += NT) {
            Dot3<R> d = site_even<P, BL>(g, e0 + h, tmp, r, R(-0.25), true, mass4, a.U, a.Cl, nullptr, 2, t);
            tsr += d.a;
            tsi += d.b;
            tt += d.c;
        }
        red[0] = (double)tsr;
        red[1] = (double)tsi;
        red[2] = (double)tt;
        cta_sum<3, NT>(red, sm);
        if (red[2] == 0.0 || !(red[2] == red[2])) break;
        double2 omega = make_double2(red[0] / red[2], red[1] / red[2]);
        const cpx<R> om = {R(omega.x), R(omega.y)};
        // x += alpha p + omega s ; r = s - omega t ; rho' = (rh, r) ; rr = (r, r)
        R hre = 0, him = 0, rrl = 0;
        for (int h = threadIdx.x; h < VBH; h += NT)
            for (int k = 0; k < NP; k++) {
                    cpx<R> xv[CW], pv[CW], sv[CW], tv[CW], hv[CW];
                P::ld_chunk(x, V, e0 + h, k, xv);
                P::ld_chunk(p, V, e0 + h, k, pv);
                P::ld_chunk(r, V, e0 + h, k, sv);
                P::ld_chunk(t, V, e0 + h, k, tv);
                P::ld_chunk(rh, V, e0 + h, k, hv);
#pragma unroll
                for (int q = 0; q < CW; q++) {
                    xv[q] = xv[q] + cmul(al, pv[q]) + cmul(om, sv[q]);
                    sv[q] = sv[q] - cmul(om, tv[q]);
                    cpx<R> z = cmulc(hv[q], sv[q]);
                    hre += z.re;
                    him += z.im;
                    rrl += sv[q].re * sv[q].re + sv[q].im * sv[q].im;
                }
                P::st_chunk(x, V, e0 + h, k, xv);
                P::st_chunk(r, V, e0 + h, k, sv);
            }
        red[0] = (double)hre;
        red[1] = (double)him;
        red[2] = (double)rrl;
        cta_sum<3, NT>(red, sm);
        it++;
        rr = red[2];
        if (!(rr == rr)) break;
        if (rr <= thresh) {
            ok = true;
            break;
        }
        double2 rn = make_double2(red[0], red[1]);
        double d1 = rho.x * rho.x + rho.y * rho.y, d2 = omega.x * omega.x + omega.y * omega.y;
        if (d1 == 0.0 || d2 == 0.0) break;
        double2 q1 = make_double2((rn.x * rho.x + rn.y * rho.y) / d1, (rn.y * rho.x - rn.x * rho.y) / d1);
        double2 q2 = make_double2((alpha.x * omega.x + alpha.y * omega.y) / d2, (alpha.y * omega.x - alpha.x * omega.y) / d2);
        const cpx<R> be = {R(q1.x * q2.x - q1.y * q2.y), R(q1.x * q2.y + q1.y * q2.x)};
        rho = rn;
        // p = r + beta (p - omega v)
        for (int h = threadIdx.x; h < VBH; h += NT)
            for (int k = 0; k < NP; k++) {
                    cpx<R> pv[CW], rv[CW], vv[CW];
                P::ld_chunk(p, V, e0 + h, k, pv);
                P::ld_chunk(r, V, e0 + h, k, rv);
                P::ld_chunk(v, V, e0 + h, k, vv);
#pragma unroll
                for (int q = 0; q < CW; q++) pv[q] = rv[q] + cmul(be, pv[q] - cmul(om, vv[q]));
                P::st_chunk(p, V, e0 + h, k, pv);
            }
        __syncthreads();
    }
    __syncthreads();
    // x_o = A_oo^-1 (b_o + 1/2 H_oe x_e)
    for (int h = threadIdx.x; h < VBH; h += NT) site_odd<P, BL>(g, o0 + h, x, b, R(0.5), a.U, Ainv, x);
    if (threadIdx.x == 0) {
        atomicMax(a.stat, it);
        if (!ok) atomicAdd(a.stat + 1, 1);
    }
}


// ---- NR right-hand sides of one block per CTA (rstride apart, same mass slot): each link and
// clover term is loaded once for all NR, and every thread carries NR independent chains between
// the CTA's barriers.  A right-hand side that has converged (or broken down) is frozen -- its
// scalars become zero, so x and r stay as they are -- while the others iterate on.

template <int NR, typename R> struct DotN {
    R a[NR], b[NR], c[NR];
};

template <class P, int BL, int NR>
__device__ __noinline__ void site_odd_n(const GeomDev &g, long s, const typename P::SElem *in,
                                        const typename P::SElem *y, long rs, typename P::R coef,
                                        const typename P::UElem *__restrict__ U,
                                        const typename P::CElem *__restrict__ Ainv, typename P::SElem *out)
{
    using R = typename P::R;
    Spinor<R> acc[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) zero(acc[r]);
    if (coef != R(0)) {
        Site<BL> st;
        decode_site<BL>(s, g, st);
        hop_dir_multi<P, BL, 1, 0, NR, false>(g, st, s, in, rs, U, acc);
        hop_dir_multi<P, BL, 1, 1, NR, false>(g, st, s, in, rs, U, acc);
        hop_dir_multi<P, BL, 1, 2, NR, false>(g, st, s, in, rs, U, acc);
        hop_dir_multi<P, BL, 1, 3, NR, false>(g, st, s, in, rs, U, acc);
#pragma unroll
        for (int r = 0; r < NR; r++) scale(acc[r], coef);
    }
    if (y) {
#pragma unroll
        for (int r = 0; r < NR; r++) {
            Spinor<R> q;
            P::load_spinor_rw(y + r * rs, g.V, s, q);
            axpy(acc[r], R(1), q);
        }
    }
#pragma unroll
    for (int ch = 0; ch < 2; ch++) {
        R c[36];
        P::load_clover(Ainv, g.V, s, ch, c);
#pragma unroll
        for (int r = 0; r < NR; r++) {
            cpx<R> v6[6], o6[6];
#pragma unroll
            for (int k = 0; k < 6; k++) v6[k] = acc[r].v[2 * ch + k / 3][k % 3];
            herm6_mul<R>(c, R(0), v6, o6);
#pragma unroll
            for (int k = 0; k < 6; k++) acc[r].v[2 * ch + k / 3][k % 3] = o6[k];
        }
    }
#pragma unroll
    for (int r = 0; r < NR; r++) P::store_spinor(out + r * rs, g.V, s, acc[r]);
}

// even site s: out = D x + coef H_intra tmp for NR right-hand sides, D = A(m) (diag) or 1, and
// the partial inner products of the phase: mode 1 -> conj(w) out; mode 2 -> conj(out) x and |out|^2.
template <class P, int BL, int NR>
__device__ __noinline__ DotN<NR, typename P::R> site_even_n(const GeomDev &g, long s, const typename P::SElem *tmp,
                                                            const typename P::SElem *x, long rs, typename P::R coef,
                                                            bool diag, typename P::R mass4,
                                                            const typename P::UElem *__restrict__ U,
                                                            const typename P::CElem *__restrict__ Cl,
                                                            const typename P::SElem *w, int mode, typename P::SElem *out)
{
    using R = typename P::R;
    Spinor<R> acc[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) zero(acc[r]);
    Site<BL> st;
    decode_site<BL>(s, g, st);
    hop_dir_multi<P, BL, 1, 0, NR, false>(g, st, s, tmp, rs, U, acc);
    hop_dir_multi<P, BL, 1, 1, NR, false>(g, st, s, tmp, rs, U, acc);
    hop_dir_multi<P, BL, 1, 2, NR, false>(g, st, s, tmp, rs, U, acc);
    hop_dir_multi<P, BL, 1, 3, NR, false>(g, st, s, tmp, rs, U, acc);
#pragma unroll
    for (int r = 0; r < NR; r++) scale(acc[r], coef);
    // (the clover term of the site is read once per right-hand side; the repeat hits L1)
#pragma unroll
    for (int r = 0; r < NR; r++) {
        Spinor<R> q;
        P::load_spinor_rw(x + r * rs, g.V, s, q);
        if (diag) clover_apply<P>(Cl, g.V, s, mass4, q);
        axpy(acc[r], R(1), q);
    }
    DotN<NR, R> d;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        d.a[r] = R(0);
        d.b[r] = R(0);
        d.c[r] = R(0);
        P::store_spinor(out + r * rs, g.V, s, acc[r]);
        Spinor<R> q;
        if (mode == 1) {
            P::load_spinor_rw(w + r * rs, g.V, s, q);
            sp_norm_dot(q, acc[r], d.a[r], d.b[r]);
        } else if (mode == 2) {
            P::load_spinor_rw(x + r * rs, g.V, s, q);
            sp_norm_dot(acc[r], q, d.a[r], d.b[r]);
            d.c[r] = sp_norm2(acc[r]);
        }
    }
    return d;
}

template <class P, int BL, int NT, int NR>
__global__ void __launch_bounds__(NT, sizeof(typename P::R) == 4 ? (NT >= 512 ? 1 : NT >= 256 ? 2 : 3) : 1)
    k_block_solve_n(GeomDev g, BlkArgs<P> a)
{
    using R = typename P::R;
    using E = typename P::SElem;
    constexpr int VBH = BlockShape<BL>::VBH;
    constexpr int NP = P::NCHUNK, CW = P::CW;
    constexpr int K = 3 * NR;
    __shared__ double sm[NT / 32][K];
    const int rhs0 = blockIdx.x * NR;  // a group of NR right-hand sides of one mass slot
    const int blk = a.blk0 + blockIdx.y;
    const long rs = a.rstride, ro = (long)rhs0 * rs;
    const int slot = rhs0 / a.rpm;
    const R mass4 = a.mass4[slot];
    const typename P::CElem *Ainv = a.Ainv[slot];
    const long e0 = (long)blk * VBH, o0 = g.vh + (long)blk * VBH;
    const long V = g.V;
    const E *b = a.b + ro;
    E *x = a.x + ro, *r = a.r + ro, *rh = a.rh + ro, *p = a.p + ro, *v = a.v + ro, *t = a.t + ro, *tmp = a.tmp + ro;

    // ||b||^2 per right-hand side; tmp_o = A_oo^-1 b_o
    double red[K];
#pragma unroll
    for (int k = 0; k < K; k++) red[k] = 0.0;
#pragma unroll
    for (int q = 0; q < NR; q++) {
        R bbl = 0;
        for (int h = threadIdx.x; h < VBH; h += NT)
            for (int k = 0; k < NP; k++) {
                cpx<R> c[CW], d[CW];
                P::ld_chunk(b + q * rs, V, e0 + h, k, c);
                P::ld_chunk(b + q * rs, V, o0 + h, k, d);
#pragma unroll
                for (int i = 0; i < CW; i++)
                    bbl += c[i].re * c[i].re + c[i].im * c[i].im + d[i].re * d[i].re + d[i].im * d[i].im;
            }
        red[q] = (double)bbl;
    }
    for (int h = threadIdx.x; h < VBH; h += NT) site_odd_n<P, BL, NR>(g, o0 + h, nullptr, b, rs, R(0), a.U, Ainv, tmp);
    cta_sum<K, NT>(red, sm);
    double bb[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) bb[q] = red[q];
    __syncthreads();
    // r = b_e + 1/2 H_eo tmp_o ; rh = p = r ; x_e = 0
    for (int h = threadIdx.x; h < VBH; h += NT)
        site_even_n<P, BL, NR>(g, e0 + h, tmp, b, rs, R(0.5), false, mass4, a.U, a.Cl, nullptr, 0, r);
#pragma unroll
    for (int k = 0; k < K; k++) red[k] = 0.0;
    for (int h = threadIdx.x; h < VBH; h += NT)
#pragma unroll
        for (int q = 0; q < NR; q++)
            for (int k = 0; k < NP; k++) {
                cpx<R> c[CW], z[CW];
                P::ld_chunk(r + q * rs, V, e0 + h, k, c);
                R rl = 0;
#pragma unroll
                for (int i = 0; i < CW; i++) {
                    rl += c[i].re * c[i].re + c[i].im * c[i].im;
                    z[i] = {R(0), R(0)};
                }
                red[q] += (double)rl;
                P::st_chunk(rh + q * rs, V, e0 + h, k, c);
                P::st_chunk(p + q * rs, V, e0 + h, k, c);
                P::st_chunk(x + q * rs, V, e0 + h, k, z);
            }
    cta_sum<K, NT>(red, sm);
    const double t2 = a.tol2_dev ? *a.tol2_dev : a.tol2;
    double rr[NR], thresh[NR];
    double2 rho[NR], alpha[NR], omega[NR];
    bool act[NR], ok[NR];
    int nact = 0;
#pragma unroll
    for (int q = 0; q < NR; q++) {
        rr[q] = red[q];
        rho[q] = make_double2(rr[q], 0.0);
        thresh[q] = t2 * bb[q];
        ok[q] = rr[q] <= thresh[q];
        act[q] = !ok[q];
        nact += act[q] ? 1 : 0;
        alpha[q] = omega[q] = make_double2(0.0, 0.0);
    }
    int it = 0;
    while (nact > 0 && it < a.maxiter) {
        // v = S p  and  (rh, v)
        __syncthreads();
        for (int h = threadIdx.x; h < VBH; h += NT) site_odd_n<P, BL, NR>(g, o0 + h, p, nullptr, rs, R(1), a.U, Ainv, tmp);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; k++) red[k] = 0.0;
        for (int h = threadIdx.x; h < VBH; h += NT) {
            DotN<NR, R> d = site_even_n<P, BL, NR>(g, e0 + h, tmp, p, rs, R(-0.25), true, mass4, a.U, a.Cl, rh, 1, v);
#pragma unroll
            for (int q = 0; q < NR; q++) {
                red[2 * q] += (double)d.a[q];
                red[2 * q + 1] += (double)d.b[q];
            }
        }
        cta_sum<K, NT>(red, sm);
        cpx<R> al[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) {
            const double dr = red[2 * q], di = red[2 * q + 1];
            const double den = dr * dr + di * di;
            if (act[q] && (den == 0.0 || !(den == den))) act[q] = false;  // breakdown: frozen, not converged
            alpha[q] = act[q] ? make_double2((rho[q].x * dr + rho[q].y * di) / den, (rho[q].y * dr - rho[q].x * di) / den)
                              : make_double2(0.0, 0.0);
            al[q] = {R(alpha[q].x), R(alpha[q].y)};
        }
        // s = r - alpha v (in r)
        for (int h = threadIdx.x; h < VBH; h += NT)
#pragma unroll
            for (int q = 0; q < NR; q++)
                for (int k = 0; k < NP; k++) {
                    cpx<R> c[CW], d[CW];
                    P::ld_chunk(r + q * rs, V, e0 + h, k, c);
                    P::ld_chunk(v + q * rs, V, e0 + h, k, d);
#pragma unroll
                    for (int i = 0; i < CW; i++) c[i] = c[i] - cmul(al[q], d[i]);
                    P::st_chunk(r + q * rs, V, e0 + h, k, c);
                }
        __syncthreads();
        // t = S s  and  (t, s), (t, t)
        for (int h = threadIdx.x; h < VBH; h += NT) site_odd_n<P, BL, NR>(g, o0 + h, r, nullptr, rs, R(1), a.U, Ainv, tmp);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; k++) red[k] = 0.0;
        for (int h = threadIdx.x; h < VBH; h += NT) {
            DotN<NR, R> d = site_even_n<P, BL, NR>(g, e0 + h, tmp, r, rs, R(-0.25), true, mass4, a.U, a.Cl, nullptr, 2, t);
#pragma unroll
            for (int q = 0; q < NR; q++) {
                red[3 * q] += (double)d.a[q];
                red[3 * q + 1] += (double)d.b[q];
                red[3 * q + 2] += (double)d.c[q];
            }
        }
        cta_sum<K, NT>(red, sm);
        cpx<R> om[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) {
            const double tt = red[3 * q + 2];
            // breakdown: frozen; the x update below still adds alpha p, which matches the s-step
            // that already moved r
            if (act[q] && (tt == 0.0 || !(tt == tt))) act[q] = false;
            omega[q] = act[q] ? make_double2(red[3 * q] / tt, red[3 * q + 1] / tt) : make_double2(0.0, 0.0);
            om[q] = {R(omega[q].x), R(omega[q].y)};
            al[q] = {R(alpha[q].x), R(alpha[q].y)};
        }
        // x += alpha p + omega s ; r = s - omega t ; rho' = (rh, r) ; rr = (r, r)
#pragma unroll
        for (int k = 0; k < K; k++) red[k] = 0.0;
        for (int h = threadIdx.x; h < VBH; h += NT)
#pragma unroll
            for (int q = 0; q < NR; q++) {
                R hre = 0, him = 0, rrl = 0;
                for (int k = 0; k < NP; k++) {
                    cpx<R> xv[CW], pv[CW], sv[CW], tv[CW], hv[CW];
                    P::ld_chunk(x + q * rs, V, e0 + h, k, xv);
                    P::ld_chunk(p + q * rs, V, e0 + h, k, pv);
                    P::ld_chunk(r + q * rs, V, e0 + h, k, sv);
                    P::ld_chunk(t + q * rs, V, e0 + h, k, tv);
                    P::ld_chunk(rh + q * rs, V, e0 + h, k, hv);
#pragma unroll
                    for (int i = 0; i < CW; i++) {
                        xv[i] = xv[i] + cmul(al[q], pv[i]) + cmul(om[q], sv[i]);
                        sv[i] = sv[i] - cmul(om[q], tv[i]);
                        cpx<R> z = cmulc(hv[i], sv[i]);
                        hre += z.re;
                        him += z.im;
                        rrl += sv[i].re * sv[i].re + sv[i].im * sv[i].im;
                    }
                    P::st_chunk(x + q * rs, V, e0 + h, k, xv);
                    P::st_chunk(r + q * rs, V, e0 + h, k, sv);
                }
                red[3 * q] += (double)hre;
                red[3 * q + 1] += (double)him;
                red[3 * q + 2] += (double)rrl;
            }
        cta_sum<K, NT>(red, sm);
        it++;
        cpx<R> be[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) {
            be[q] = {R(0), R(0)};
            if (!act[q]) continue;
            rr[q] = red[3 * q + 2];
            if (!(rr[q] == rr[q])) {
                act[q] = false;
                continue;
            }
            if (rr[q] <= thresh[q]) {
                ok[q] = true;
                act[q] = false;
                continue;
            }
            const double2 rn = make_double2(red[3 * q], red[3 * q + 1]);
            const double d1 = rho[q].x * rho[q].x + rho[q].y * rho[q].y;
            const double d2 = omega[q].x * omega[q].x + omega[q].y * omega[q].y;
            if (d1 == 0.0 || d2 == 0.0) {
                act[q] = false;
                continue;
            }
            const double2 q1 = make_double2((rn.x * rho[q].x + rn.y * rho[q].y) / d1, (rn.y * rho[q].x - rn.x * rho[q].y) / d1);
            const double2 q2 = make_double2((alpha[q].x * omega[q].x + alpha[q].y * omega[q].y) / d2,
                                            (alpha[q].y * omega[q].x - alpha[q].x * omega[q].y) / d2);
            be[q] = {R(q1.x * q2.x - q1.y * q2.y), R(q1.x * q2.y + q1.y * q2.x)};
            rho[q] = rn;
        }
        nact = 0;
#pragma unroll
        for (int q = 0; q < NR; q++) {
            nact += act[q] ? 1 : 0;
            if (!act[q]) om[q] = {R(0), R(0)};
        }
        if (nact == 0) break;
        // p = r + beta (p - omega v) for the right-hand sides still iterating
        for (int h = threadIdx.x; h < VBH; h += NT)
#pragma unroll
            for (int q = 0; q < NR; q++) {
                if (!act[q]) continue;
                for (int k = 0; k < NP; k++) {
                    cpx<R> pv[CW], rv[CW], vv[CW];
                    P::ld_chunk(p + q * rs, V, e0 + h, k, pv);
                    P::ld_chunk(r + q * rs, V, e0 + h, k, rv);
                    P::ld_chunk(v + q * rs, V, e0 + h, k, vv);
#pragma unroll
                    for (int i = 0; i < CW; i++) pv[i] = rv[i] + cmul(be[q], pv[i] - cmul(om[q], vv[i]));
                    P::st_chunk(p + q * rs, V, e0 + h, k, pv);
                }
            }
    }
    __syncthreads();
    // x_o = A_oo^-1 (b_o + 1/2 H_oe x_e)
    for (int h = threadIdx.x; h < VBH; h += NT) site_odd_n<P, BL, NR>(g, o0 + h, x, b, rs, R(0.5), a.U, Ainv, x);
    if (threadIdx.x == 0) {
        atomicMax(a.stat, it);
        int miss = 0;
#pragma unroll
        for (int q = 0; q < NR; q++) miss += ok[q] ? 0 : 1;
        if (miss) atomicAdd(a.stat + 1, miss);
    }
}

// Launch shape of the block solver: NT threads per (block, right-hand side), or for blocks of at
// least 512 sites per parity on 32- and 16-bit storage also 2 NT threads (one CTA per SM instead of
// two, half the Krylov vectors of the resident CTAs competing for L2).  The first launch of each
// (storage, block length, right-hand sides) shape times both on the real arguments -- the kernel
// reads b and overwrites all of x, so a repeat gives the same result -- and keeps the faster.
template <class P, int BL>
void launch_block_kernel(ddrw_ctx *ctx, const BlkArgs<P> &a, int nrhs)
{
    GeomDev g = geom_dev(ctx);
    dim3 grid((unsigned)nrhs, (unsigned)ctx->nblk_c);
    constexpr int VBH = BlockShape<BL>::VBH;
    constexpr int NT = VBH <= 32 ? 32 : (VBH <= 128 ? 128 : 256);
    constexpr bool WIDE = VBH >= 512 && P::ID != 64;
    constexpr int NT2 = WIDE ? 2 * NT : NT;
    const int kind = P::ID == 64 ? PROF_BLOCK64 : P::ID == 32 ? PROF_BLOCK32 : PROF_BLOCK16;
    // form 2: two right-hand sides per CTA (FP32 storage; pairs inside one mass slot)
    const bool pairs = P::ID == 32 && WIDE && nrhs % 2 == 0 && a.rpm % 2 == 0;
    auto run = [&](int form) {
        ++ctx->launches;
        if constexpr (P::ID == 32 && WIDE) {
            if (form == 2) {
                k_block_solve_n<P, BL, NT2, 2><<<dim3((unsigned)nrhs / 2, (unsigned)ctx->nblk_c), NT2, 0, ctx->stream>>>(g, a);
                return;
            }
        }
        if (form) k_block_solve<P, BL, NT2><<<grid, NT2, 0, ctx->stream>>>(g, a);
        else k_block_solve<P, BL, NT><<<grid, NT, 0, ctx->stream>>>(g, a);
    };
    int form = 0;
    if (WIDE) {
        const std::array<int, 3> key = {P::ID, BL, nrhs * 2 + (pairs ? 1 : 0)};
        auto it = ctx->blk_tune.find(key);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(ctx->stream, &cs);
        if (ctx->blk_form >= 0) {
            form = (ctx->blk_form == 2 && !pairs) ? 1 : ctx->blk_form;  // pinned (ddrw_block_config)
        } else if (it != ctx->blk_tune.end()) {
            form = it->second;
        } else if (ctx->autotune && cs == cudaStreamCaptureStatusNone && a.b != a.x) {
            const int nf = pairs ? 3 : 2;
            cudaEvent_t e[4];
            for (auto &ev : e) cudaEventCreate(&ev);
            cudaEventRecord(e[0], ctx->stream);
            for (int f = 0; f < nf; f++) {
                run(f);
                cudaEventRecord(e[f + 1], ctx->stream);
            }
            cudaEventSynchronize(e[nf]);
            float best = 0;
            form = 0;
            for (int f = 0; f < nf; f++) {
                float ms = 0;
                cudaEventElapsedTime(&ms, e[f], e[f + 1]);
                if (f == 0 || ms < best) best = ms, form = f;
            }
            for (auto &ev : e) cudaEventDestroy(ev);
            if (cudaGetLastError() != cudaSuccess) form = 0;
            ctx->blk_tune[key] = form;
            cudaMemsetAsync(a.stat, 0, 2 * sizeof(int), ctx->stream);  // the timing runs counted too
        }
    }
    ProfScope ps(ctx, kind, 0.0);
    run(form);
}

}  // namespace ddrw
