// stencil.cuh -- per-site hopping and clover arithmetic of the Wilson-clover operator, shared by
// the stencil kernels (dslash.cu) and the persistent block solver (blocksolve.cu).
//
//   hop sum at x:   sum_mu [ (1 - g_mu) U_mu(x) in(x+mu) + (1 + g_mu) U_mu(x-mu)^dag in(x-mu) ]
//   clover apply:   v <- (d + H_ch) v on both chirality blocks (H = C, or an inverse of A(m))
//
// HOPSEL selects the hops: 0 all, 1 only hops inside the block of x (D_bb, D_ww), 2 only hops
// leaving the block (D_bw, D_wb).
#pragma once

#include "ddrw_internal.cuh"

namespace ddrw {

// RO: the input is read-only for the whole kernel (read through the non-coherent path); kernels
// that write their own hop input (the persistent block solver) pass RO = false.
template <class P, int BL, int HOPSEL, int MU, bool RO>
__device__ __forceinline__ void hop_dir(const GeomDev &g, const Site<BL> &st, long s,
                                        const typename P::SElem *in,
                                        const typename P::UElem *__restrict__ U, Spinor<typename P::R> &acc)
{
    using R = typename P::R;
    bool cross;
    int ph;
    {
        int sf = neighbour<BL>(st, MU, +1, g, &cross, &ph);
        if (HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross)) {
            Spinor<R> p;
            if (RO) P::load_spinor(in, g.V, sf, p);
            else P::load_spinor_rw(in, g.V, sf, p);
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
        int sb = neighbour<BL>(st, MU, -1, g, &cross, &ph);
        if (HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross)) {
            Spinor<R> p;
            if (RO) P::load_spinor(in, g.V, sb, p);
            else P::load_spinor_rw(in, g.V, sb, p);
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

template <class P, int BL, int HOPSEL, bool RO = true>
__device__ __forceinline__ void hop_sum(const GeomDev &g, const Site<BL> &st, long s,
                                        const typename P::SElem *in,
                                        const typename P::UElem *__restrict__ U, Spinor<typename P::R> &acc)
{
    hop_dir<P, BL, HOPSEL, 0, RO>(g, st, s, in, U, acc);
    hop_dir<P, BL, HOPSEL, 1, RO>(g, st, s, in, U, acc);
    hop_dir<P, BL, HOPSEL, 2, RO>(g, st, s, in, U, acc);
    hop_dir<P, BL, HOPSEL, 3, RO>(g, st, s, in, U, acc);
}

// Hops of NR right-hand sides at once (fields rstride elements apart): the link of each hop is
// loaded, and for two-row storage reconstructed, once for all NR.
template <class P, int BL, int HOPSEL, int MU, int NR>
__device__ __forceinline__ void hop_dir_multi(const GeomDev &g, const Site<BL> &st, long s,
                                              const typename P::SElem *in, long rstride,
                                              const typename P::UElem *__restrict__ U,
                                              Spinor<typename P::R> (&acc)[NR])
{
    using R = typename P::R;
    bool cross;
    int ph;
    {
        int sf = neighbour<BL>(st, MU, +1, g, &cross, &ph);
        if (HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross)) {
            Link<R> L;
            P::load_link(U, g.V, MU, s, L);
#pragma unroll
            for (int r = 0; r < NR; r++) {
                Spinor<R> p;
                P::load_spinor(in + r * rstride, (int)g.V, sf, p);
                Half<R> h, w;
                project<MU, -1>(p, h);
                link_mul(L, h, w);
                if (ph < 0)
#pragma unroll
                    for (int a = 0; a < 2; a++)
#pragma unroll
                        for (int c = 0; c < 3; c++) w.v[a][c] = -w.v[a][c];
                reconstruct_add<MU, -1>(acc[r], w);
            }
        }
    }
    {
        int sb = neighbour<BL>(st, MU, -1, g, &cross, &ph);
        if (HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross)) {
            Link<R> L;
            P::load_link(U, g.V, MU, sb, L);
#pragma unroll
            for (int r = 0; r < NR; r++) {
                Spinor<R> p;
                P::load_spinor(in + r * rstride, (int)g.V, sb, p);
                Half<R> h, w;
                project<MU, +1>(p, h);
                link_dag_mul(L, h, w);
                if (ph < 0)
#pragma unroll
                    for (int a = 0; a < 2; a++)
#pragma unroll
                        for (int c = 0; c < 3; c++) w.v[a][c] = -w.v[a][c];
                reconstruct_add<MU, +1>(acc[r], w);
            }
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

template <typename R>
__device__ __forceinline__ void scale(Spinor<R> &v, R a)
{
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
        for (int c = 0; c < 3; c++) v.v[sp][c] = a * v.v[sp][c];
}

template <typename R>
__device__ __forceinline__ void axpy(Spinor<R> &y, R a, const Spinor<R> &x)  // y += a x
{
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
        for (int c = 0; c < 3; c++) y.v[sp][c] = y.v[sp][c] + a * x.v[sp][c];
}

}  // namespace ddrw
