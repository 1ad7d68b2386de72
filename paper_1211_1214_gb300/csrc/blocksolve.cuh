// blocksolve.cuh -- the persistent block-solver kernel (K6); instantiated per storage policy and
// block length in blocksolve_<policy><l>.cu so that the instantiations compile in parallel.
#pragma once

#include "blas.cuh"
#include "ctx.h"
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

template <class P, int BL, int NT>
__global__ void __launch_bounds__(NT) k_block_solve(GeomDev g, BlkArgs<P> a)
{
    using R = typename P::R;
    constexpr int VBH = BlockShape<BL>::VBH;
    __shared__ double sm[NT / 32][3];
    const int blk = a.blk0 + blockIdx.x;
    const long ro = (long)blockIdx.y * a.rstride;
    const int slot = blockIdx.y / a.rpm;
    const R mass4 = a.mass4[slot];
    const typename P::CElem *Ainv = a.Ainv[slot];
    const long e0 = (long)blk * VBH, o0 = g.vh + (long)blk * VBH;
    const typename P::SElem *b = a.b + ro;
    typename P::SElem *x = a.x + ro, *r = a.r + ro, *rh = a.rh + ro, *p = a.p + ro, *v = a.v + ro, *t = a.t + ro,
                      *tmp = a.tmp + ro;

    // ||b||^2 over the block, tmp_o = A_oo^-1 b_o
    R bbl = 0;
    for (int h = threadIdx.x; h < VBH; h += NT) {
        Spinor<R> q;
        P::load_spinor_rw(b, g.V, e0 + h, q);
        bbl += sp_norm2(q);
        P::load_spinor_rw(b, g.V, o0 + h, q);
        bbl += sp_norm2(q);
        clover_apply<P>(Ainv, g.V, o0 + h, R(0), q);
        P::store_spinor(tmp, g.V, o0 + h, q);
    }
    double red[3] = {(double)bbl, 0, 0};
    cta_sum<3, NT>(red, sm);
    const double bb = red[0];
    // r = b_e + 1/2 H_eo tmp_o ; rh = p = r ; x_e = 0
    R rl = 0;
    for (int h = threadIdx.x; h < VBH; h += NT) {
        long s = e0 + h;
        Site<BL> st;
        decode_site<BL>(s, g, st);
        Spinor<R> acc, q, z;
        zero(acc);
        zero(z);
        hop_sum<P, BL, 1, false>(g, st, s, tmp, a.U, acc);
        P::load_spinor_rw(b, g.V, s, q);
        scale(acc, R(0.5));
        axpy(acc, R(1), q);
        P::store_spinor(r, g.V, s, acc);
        P::store_spinor(rh, g.V, s, acc);
        P::store_spinor(p, g.V, s, acc);
        P::store_spinor(x, g.V, s, z);
        rl += sp_norm2(acc);
    }
    red[0] = (double)rl;
    cta_sum<3, NT>(red, sm);
    double rr = red[0];
    double2 rho = make_double2(rr, 0.0);
    const double thresh = a.tol2 * bb;
    int it = 0;
    bool ok = rr <= thresh;
    while (!ok && it < a.maxiter) {
        // v = S p
        for (int h = threadIdx.x; h < VBH; h += NT) {
            long s = o0 + h;
            Site<BL> st;
            decode_site<BL>(s, g, st);
            Spinor<R> acc;
            zero(acc);
            hop_sum<P, BL, 1, false>(g, st, s, p, a.U, acc);
            clover_apply<P>(Ainv, g.V, s, R(0), acc);
            P::store_spinor(tmp, g.V, s, acc);
        }
        __syncthreads();
        R are = 0, aim = 0;
        for (int h = threadIdx.x; h < VBH; h += NT) {
            long s = e0 + h;
            Site<BL> st;
            decode_site<BL>(s, g, st);
            Spinor<R> acc, q;
            zero(acc);
            hop_sum<P, BL, 1, false>(g, st, s, tmp, a.U, acc);
            scale(acc, R(-0.25));
            P::load_spinor_rw(p, g.V, s, q);
            clover_apply<P>(a.Cl, g.V, s, mass4, q);
            axpy(acc, R(1), q);
            P::store_spinor(v, g.V, s, acc);
            P::load_spinor_rw(rh, g.V, s, q);
            sp_norm_dot(q, acc, are, aim);
        }
        red[0] = (double)are;
        red[1] = (double)aim;
        cta_sum<3, NT>(red, sm);
        double den = red[0] * red[0] + red[1] * red[1];
        if (den == 0.0 || !(den == den)) break;
        double2 alpha = make_double2((rho.x * red[0] + rho.y * red[1]) / den, (rho.y * red[0] - rho.x * red[1]) / den);
        const cpx<R> al = {R(alpha.x), R(alpha.y)};
        // s = r - alpha v (in r)
        for (int h = threadIdx.x; h < VBH; h += NT) {
            long s = e0 + h;
            Spinor<R> q, w;
            P::load_spinor_rw(r, g.V, s, q);
            P::load_spinor_rw(v, g.V, s, w);
#pragma unroll
            for (int sp = 0; sp < 4; sp++)
#pragma unroll
                for (int c = 0; c < 3; c++) q.v[sp][c] = q.v[sp][c] - cmul(al, w.v[sp][c]);
            P::store_spinor(r, g.V, s, q);
        }
        __syncthreads();
        // t = S s
        for (int h = threadIdx.x; h < VBH; h += NT) {
            long s = o0 + h;
            Site<BL> st;
            decode_site<BL>(s, g, st);
            Spinor<R> acc;
            zero(acc);
            hop_sum<P, BL, 1, false>(g, st, s, r, a.U, acc);
            clover_apply<P>(Ainv, g.V, s, R(0), acc);
            P::store_spinor(tmp, g.V, s, acc);
        }
        __syncthreads();
        R tsr = 0, tsi = 0, tt = 0;
        for (int h = threadIdx.x; h < VBH; h += NT) {
            long s = e0 + h;
            Site<BL> st;
            decode_site<BL>(s, g, st);
            Spinor<R> acc, q;
            zero(acc);
            hop_sum<P, BL, 1, false>(g, st, s, tmp, a.U, acc);
            scale(acc, R(-0.25));
            P::load_spinor_rw(r, g.V, s, q);
            Spinor<R> d = q;
            clover_apply<P>(a.Cl, g.V, s, mass4, d);
            axpy(acc, R(1), d);
            P::store_spinor(t, g.V, s, acc);
            sp_norm_dot(acc, q, tsr, tsi);
            tt += sp_norm2(acc);
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
        for (int h = threadIdx.x; h < VBH; h += NT) {
            long s = e0 + h;
            Spinor<R> xv, pv, sv, tv, hv;
            P::load_spinor_rw(x, g.V, s, xv);
            P::load_spinor_rw(p, g.V, s, pv);
            P::load_spinor_rw(r, g.V, s, sv);
            P::load_spinor_rw(t, g.V, s, tv);
            P::load_spinor_rw(rh, g.V, s, hv);
#pragma unroll
            for (int sp = 0; sp < 4; sp++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    xv.v[sp][c] = xv.v[sp][c] + cmul(al, pv.v[sp][c]) + cmul(om, sv.v[sp][c]);
                    sv.v[sp][c] = sv.v[sp][c] - cmul(om, tv.v[sp][c]);
                }
            P::store_spinor(x, g.V, s, xv);
            P::store_spinor(r, g.V, s, sv);
            sp_norm_dot(hv, sv, hre, him);
            rrl += sp_norm2(sv);
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
        for (int h = threadIdx.x; h < VBH; h += NT) {
            long s = e0 + h;
            Spinor<R> pv, rv, vv;
            P::load_spinor_rw(p, g.V, s, pv);
            P::load_spinor_rw(r, g.V, s, rv);
            P::load_spinor_rw(v, g.V, s, vv);
#pragma unroll
            for (int sp = 0; sp < 4; sp++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    pv.v[sp][c] = rv.v[sp][c] + cmul(be, pv.v[sp][c] - cmul(om, vv.v[sp][c]));
            P::store_spinor(p, g.V, s, pv);
        }
        __syncthreads();
    }
    __syncthreads();
    // x_o = A_oo^-1 (b_o + 1/2 H_oe x_e)
    for (int h = threadIdx.x; h < VBH; h += NT) {
        long s = o0 + h;
        Site<BL> st;
        decode_site<BL>(s, g, st);
        Spinor<R> acc, q;
        zero(acc);
        hop_sum<P, BL, 1, false>(g, st, s, x, a.U, acc);
        scale(acc, R(0.5));
        P::load_spinor_rw(b, g.V, s, q);
        axpy(acc, R(1), q);
        clover_apply<P>(Ainv, g.V, s, R(0), acc);
        P::store_spinor(x, g.V, s, acc);
    }
    if (threadIdx.x == 0) {
        atomicMax(a.stat, it);
        if (!ok) atomicAdd(a.stat + 1, 1);
    }
}

template <class P, int BL>
void launch_block_kernel(ddrw_ctx *ctx, const BlkArgs<P> &a, int nrhs)
{
    GeomDev g = geom_dev(ctx);
    dim3 grid((unsigned)ctx->nblk_c, (unsigned)nrhs);
    constexpr int VBH = BlockShape<BL>::VBH;
    constexpr int NT = VBH <= 32 ? 32 : (VBH <= 128 ? 128 : 256);
    ProfScope ps(ctx, sizeof(typename P::R) == 8 ? PROF_BLOCK64 : PROF_BLOCK32, 0.0);
    ++ctx->launches;
    k_block_solve<P, BL, NT><<<grid, NT, 0, ctx->stream>>>(g, a);
}

}  // namespace ddrw
