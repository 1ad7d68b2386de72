// dslash.cu -- the fused hopping + clover stencil of the Wilson-clover operator (K4) and its
// block-restricted forms (K5): D_bb / D_ww keep the hops inside a block, D_bw / D_wb the hops
// between blocks (Eq. 1).  One kernel template serves every form:
//
//   out(x) = POST( alpha * DIAG(x) + beta * sum_mu [ (1 - g_mu) U_mu(x) in(x+mu) + (1 + g_mu) U_mu(x-mu)^dag in(x-mu) ] )
//
// The SU(3) x spin stencil is not a dense contraction, so it runs on the FP32/FP64 ALUs, not on
// tensor cores.  Each hop projects the neighbour spinor to a 2-spin half spinor before the
// colour multiply (half the complex multiplies of a full 4-spin product).
#include "ctx.h"

namespace ddrw {

template <class P> struct DsArgs {
    typename P::SElem *out;
    const typename P::SElem *in;
    const typename P::SElem *x;
    long rstride;
    const typename P::UElem *U;
    const typename P::CElem *Cl;
    const typename P::CElem *Ainv;
    typename P::R mass4;  // 4 + m
    typename P::R alpha, beta;
    int diag, post;
    int par0, npar, blk0, nblk;
};

template <class P, int BL, int HOPSEL, int MU>
__device__ __forceinline__ void hop_dir(const GeomDev &g, const Site<BL> &st, long s,
                                        const typename P::SElem *__restrict__ in,
                                        const typename P::UElem *__restrict__ U, Spinor<typename P::R> &acc)
{
    using R = typename P::R;
    bool cross;
    int ph;
    {
        long sf = neighbour<BL>(st, MU, +1, g, &cross, &ph);
        if (HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross)) {
            Spinor<R> p;
            P::load_spinor(in, g.V, sf, p);
            Half<R> h, w;
            project<MU, -1>(p, h);
            Link<R> L;
            P::load_link(U, g.V, MU, s, L);
            link_mul(L, h, w);
            if (ph < 0)
#pragma unroll
                for (int a = 0; a < 2; a++)
#pragma unroll
                    for (int c = 0; c < 3; c++) w.v[a][c] = -w.v[a][c];
            reconstruct_add<MU, -1>(acc, w);
        }
    }
    {
        long sb = neighbour<BL>(st, MU, -1, g, &cross, &ph);
        if (HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross)) {
            Spinor<R> p;
            P::load_spinor(in, g.V, sb, p);
            Half<R> h, w;
            project<MU, +1>(p, h);
            Link<R> L;
            P::load_link(U, g.V, MU, sb, L);
            link_dag_mul(L, h, w);
            if (ph < 0)
#pragma unroll
                for (int a = 0; a < 2; a++)
#pragma unroll
                    for (int c = 0; c < 3; c++) w.v[a][c] = -w.v[a][c];
            reconstruct_add<MU, +1>(acc, w);
        }
    }
}

// v <- (diag + H_ch) v on both chirality blocks, H from a packed clover-format array
template <class P>
__device__ __forceinline__ void clover_apply(const typename P::CElem *__restrict__ Cl, long V, long s,
                                             typename P::R diag, Spinor<typename P::R> &v)
{
    using R = typename P::R;
#pragma unroll
    for (int ch = 0; ch < 2; ch++) {
        R c[36];
        P::load_clover(Cl, V, s, ch, c);
        cpx<R> in6[6], out6[6];
#pragma unroll
        for (int i = 0; i < 6; i++) in6[i] = v.v[2 * ch + i / 3][i % 3];
        herm6_mul<R>(c, diag, in6, out6);
#pragma unroll
        for (int i = 0; i < 6; i++) v.v[2 * ch + i / 3][i % 3] = out6[i];
    }
}

template <class P, int BL, int HOPSEL>
__global__ void __launch_bounds__(128) k_dslash(GeomDev g, DsArgs<P> a)
{
    using R = typename P::R;
    const long nper = (long)a.nblk * BlockShape<BL>::VBH;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nper * a.npar) return;
    const long roff = (long)blockIdx.y * a.rstride;
    const int pp = (int)(i / nper);
    const long s = (long)(a.par0 + pp) * g.vh + (long)a.blk0 * BlockShape<BL>::VBH + (i - pp * nper);
    Site<BL> st;
    decode_site<BL>(s, g, st);

    Spinor<R> acc;
    zero(acc);
    if (a.beta != R(0)) {
        const typename P::SElem *in = a.in + roff;
        hop_dir<P, BL, HOPSEL, 0>(g, st, s, in, a.U, acc);
        hop_dir<P, BL, HOPSEL, 1>(g, st, s, in, a.U, acc);
        hop_dir<P, BL, HOPSEL, 2>(g, st, s, in, a.U, acc);
        hop_dir<P, BL, HOPSEL, 3>(g, st, s, in, a.U, acc);
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.v[sp][c] = a.beta * acc.v[sp][c];
    }
    if (a.diag) {
        Spinor<R> d;
        P::load_spinor(a.x + roff, g.V, s, d);
        if (a.diag == 1) clover_apply<P>(a.Cl, g.V, s, a.mass4, d);
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.v[sp][c] = acc.v[sp][c] + a.alpha * d.v[sp][c];
    }
    if (a.post) clover_apply<P>(a.Ainv, g.V, s, R(0), acc);
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
    a.mass4 = R(4.0 + c.mass);
    a.alpha = R(c.alpha);
    a.beta = R(c.beta);
    a.diag = c.diag;
    a.post = c.post;
    a.par0 = c.par0;
    a.npar = c.npar;
    a.blk0 = c.blk0;
    a.nblk = c.nblk;
    a.Ainv = (const typename P::CElem *)c.Ainv;
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
    dim3 grid((unsigned)((n + 127) / 128), (unsigned)c.nrhs);
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
