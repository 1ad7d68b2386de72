// dslash.cu -- the fused hopping + clover stencil of the Wilson-clover operator (K4) and its
// block-restricted forms (K5): D_bb / D_ww keep the hops inside a block, D_bw / D_wb the hops
// between blocks (Eq. 1).  One kernel template serves every form:
//
//   out(x) = POST( alpha * DIAG(x) + beta * sum_mu [ (1 - g_mu) U_mu(x) in(x+mu) + (1 + g_mu) U_mu(x-mu)^dag in(x-mu) ] )
//
// DIAG is A(m) x = (4 + m) x + C x (or x itself), POST an optional A(m)^-1.  Right-hand sides are
// interleaved with the site tiles along gridDim.x (right-hand side fastest) and grouped into mass
// slots (rhs / rpm), so one launch can carry several masses.  The SU(3) x spin stencil is not a dense contraction, so it runs on the FP32/FP64
// ALUs, not on tensor cores.  Each hop projects the neighbour to a 2-spin half spinor before the
// colour multiply (half the complex multiplies of a 4-spin product).
#include "ctx.h"
#include "stencil.cuh"

namespace ddrw {

template <class P> struct DsArgs {
    typename P::SElem *out;
    const typename P::SElem *in;
    const typename P::SElem *x;
    long rstride;
    const typename P::UElem *U;
    const typename P::CElem *Cl;
    typename P::R alpha, beta;
    int diag, post;
    int par0, npar, blk0, nblk;
    int nrhs, rpm;
    typename P::R mass4[MAXM];           // 4 + m per slot
    const typename P::CElem *Ainv[MAXM];  // A(m)^-1 per slot
};

template <class P, int BL, int HOPSEL>
__global__ void __launch_bounds__(128) k_dslash(GeomDev g, DsArgs<P> a)
{
    using R = typename P::R;
    // right-hand side fastest across CTAs: the nrhs CTAs of one site tile run together and share
    // its links and clover term through L2
    const int rhs = blockIdx.x % a.nrhs;
    const long tile = blockIdx.x / a.nrhs;
    const long nper = (long)a.nblk * BlockShape<BL>::VBH;
    const long i = tile * blockDim.x + threadIdx.x;
    if (i >= nper * a.npar) return;
    const long roff = (long)rhs * a.rstride;
    const int slot = rhs / a.rpm;
    const int pp = (int)(i / nper);
    const long s = (long)(a.par0 + pp) * g.vh + (long)a.blk0 * BlockShape<BL>::VBH + (i - pp * nper);
    Site<BL> st;
    decode_site<BL>(s, g, st);

    Spinor<R> acc;
    zero(acc);
    if (a.beta != R(0)) {
        hop_sum<P, BL, HOPSEL>(g, st, s, a.in + roff, a.U, acc);
        scale(acc, a.beta);
    }
    if (a.diag) {
        Spinor<R> d;
        P::load_spinor(a.x + roff, g.V, s, d);
        if (a.diag == 1) clover_apply<P>(a.Cl, g.V, s, a.mass4[slot], d);
        axpy(acc, a.alpha, d);
    }
    if (a.post) clover_apply<P>(a.Ainv[slot], g.V, s, R(0), acc);
    P::store_spinor(a.out + roff, g.V, s, acc);
}

template <class P, int BL>
static void launch_bl(ddrw_ctx *ctx, const DslashCall &c)
{
    using R = typename P::R;
    DsArgs<P> a;
    a.out = (typename P::SElem *)c.out;
    a.in = (const typename P::SElem *)c.in;
    a.x = (const typename P::SElem *)c.x;
    a.rstride = c.rstride;
    a.alpha = R(c.alpha);
    a.beta = R(c.beta);
    a.diag = c.diag;
    a.post = c.post;
    a.par0 = c.par0;
    a.npar = c.npar;
    a.blk0 = c.blk0;
    a.nblk = c.nblk;
    int nm = c.nmass < 1 ? 1 : c.nmass;
    a.nrhs = c.nrhs;
    a.rpm = (c.nrhs + nm - 1) / nm;
    for (int k = 0; k < MAXM; k++) {
        int kk = k < nm ? k : nm - 1;
        a.mass4[k] = R(4.0 + c.masses[kk]);
        a.Ainv[k] = (const typename P::CElem *)c.Ainv[kk];
    }
    if constexpr (sizeof(R) == 8) {
        a.U = (const typename P::UElem *)ctx->U64;
        a.Cl = (const typename P::CElem *)ctx->C64;
    } else {
        a.U = (const typename P::UElem *)ctx->U32;
        a.Cl = (const typename P::CElem *)ctx->C32;
    }
    GeomDev g = geom_dev(ctx);
    long n = (long)c.npar * c.nblk * BlockShape<BL>::VBH;
    if (n == 0 || c.nrhs == 0) return;
    dim3 grid((unsigned)(((n + 127) / 128) * c.nrhs));
    // compulsory bytes of this launch: per output site the R input, output and diagonal-input
    // spinors, the links of its hops (8 per site when the output is one parity, since the backward
    // links are stored at the other parity; 4 per site for both parities), clover terms once
    const double S = sizeof(typename P::SElem) * P::SPLANES, Lk = sizeof(typename P::UElem) * P::UPLANES,
                 Cb = sizeof(typename P::CElem) * P::CPLANES;
    double per = S * c.nrhs * ((c.beta != 0.0) + 1 + (c.diag != 0));
    if (c.beta != 0.0) per += (c.npar == 1 ? 8.0 : 4.0) * Lk;
    if (c.diag == 1) per += Cb;
    if (c.post) per += Cb;
    int kind = (sizeof(R) == 8 ? PROF_DSLASH64 : PROF_DSLASH32) + (c.hopsel != 0 ? 2 : 0);
    ProfScope ps(ctx, kind, per * (double)n);
    ++ctx->launches;
    switch (c.hopsel) {
    case 0: k_dslash<P, BL, 0><<<grid, 128, 0, ctx->stream>>>(g, a); break;
    case 1: k_dslash<P, BL, 1><<<grid, 128, 0, ctx->stream>>>(g, a); break;
    default: k_dslash<P, BL, 2><<<grid, 128, 0, ctx->stream>>>(g, a); break;
    }
}

template <class P>
static void launch(ddrw_ctx *ctx, const DslashCall &c)
{
    switch (ctx->l) {
    case 2: launch_bl<P, 2>(ctx, c); break;
    case 4: launch_bl<P, 4>(ctx, c); break;
    case 6: launch_bl<P, 6>(ctx, c); break;
    default: launch_bl<P, 8>(ctx, c); break;
    }
}

void dslash64(ddrw_ctx *ctx, const DslashCall &c) { launch<PrecD>(ctx, c); }
void dslash32(ddrw_ctx *ctx, const DslashCall &c) { launch<PrecS>(ctx, c); }

}  // namespace ddrw
