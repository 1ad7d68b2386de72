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
// loaded, and for two-row storage reconstructed, once for all NR.  RO = false reads the input
// through the coherent path (kernels that write their own hop input, the persistent block solver).
template <class P, int BL, int HOPSEL, int MU, int NR, bool RO = true>
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
                Half<R> h, w;
                if constexpr (Normed<P>::value && RO) {
                    R n;
                    P::load_spinor_unscaled(in + r * rstride, (int)g.V, sf, p, n);
                    project<MU, -1>(p, h);
                    link_mul(L, h, w);
                    reconstruct_add_scaled<MU, -1>(acc[r], w, ph < 0 ? -n : n);
                } else {
                    if (RO) P::load_spinor(in + r * rstride, (int)g.V, sf, p);
                    else P::load_spinor_rw(in + r * rstride, (int)g.V, sf, p);
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
    }
    {
        int sb = neighbour<BL>(st, MU, -1, g, &cross, &ph);
        if (HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross)) {
            Link<R> L;
            P::load_link(U, g.V, MU, sb, L);
#pragma unroll
            for (int r = 0; r < NR; r++) {
                Spinor<R> p;
                Half<R> h, w;
                if constexpr (Normed<P>::value && RO) {
                    R n;
                    P::load_spinor_unscaled(in + r * rstride, (int)g.V, sb, p, n);
                    project<MU, +1>(p, h);
                    link_dag_mul(L, h, w);
                    reconstruct_add_scaled<MU, +1>(acc[r], w, ph < 0 ? -n : n);
                } else {
                    if (RO) P::load_spinor(in + r * rstride, (int)g.V, sb, p);
                    else P::load_spinor_rw(in + r * rstride, (int)g.V, sb, p);
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
}

// Hops of direction MU with the neighbours read from the neighbour table: nf / nb are the table
// entries of the forward / backward hop (index, block-crossing bit, time-boundary sign bit).
template <class P, int HOPSEL, int MU, int NR>
__device__ __forceinline__ void hop_tab(const GeomDev &g, int nf, int nb, int s, const typename P::SElem *in,
                                        long rstride, const typename P::UElem *__restrict__ U,
                                        Spinor<typename P::R> (&acc)[NR])
{
    using R = typename P::R;
    const int V = (int)g.V;
#pragma unroll
    for (int d = 0; d < 2; d++) {
        const int e = d == 0 ? nf : nb;
        const bool cross = (e & NBR_CROSS) != 0;
        if (!(HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross))) continue;
        const int n = e & NBR_IDX;
        const bool flip = e < 0 && g.tsign < 0;
        Link<R> L;
        P::load_link(U, V, MU, d == 0 ? s : n, L);  // backward links are stored at the neighbour
#pragma unroll
        for (int r = 0; r < NR; r++) {
            Spinor<R> p;
            Half<R> h, w;
            if constexpr (Normed<P>::value) {
                R nrm;
                P::load_spinor_unscaled(in + r * rstride, V, n, p, nrm);
                if (flip) nrm = -nrm;
                if (d == 0) {
                    project<MU, -1>(p, h);
                    link_mul(L, h, w);
                    reconstruct_add_scaled<MU, -1>(acc[r], w, nrm);
                } else {
                    project<MU, +1>(p, h);
                    link_dag_mul(L, h, w);
                    reconstruct_add_scaled<MU, +1>(acc[r], w, nrm);
                }
                continue;
            }
            P::load_spinor(in + r * rstride, V, n, p);
            if (d == 0) {
                project<MU, -1>(p, h);
                link_mul(L, h, w);
            } else {
                project<MU, +1>(p, h);
                link_dag_mul(L, h, w);
            }
            if (flip)
#pragma unroll
                for (int a = 0; a < 2; a++)
#pragma unroll
                    for (int c = 0; c < 3; c++) w.v[a][c] = -w.v[a][c];
            if (d == 0) reconstruct_add<MU, -1>(acc[r], w);
            else reconstruct_add<MU, +1>(acc[r], w);
        }
    }
}

// ---- rolled form: the forward and backward hops of a direction share one body
//
// The projector sign sg (-1 forward, +1 backward) and the boundary phase enter as FMA
// coefficients, and the backward hop's U^dag is formed in registers, so the four direction
// bodies serve both signs: half the code of the unrolled form at nearly the same instruction
// count (the stencil is large enough that instruction fetch limits it otherwise).

// h = psi_u + sg e_mu psi_d
template <int MU, typename R>
__device__ __forceinline__ void project_sg(const Spinor<R> &p, R sg, Half<R> &h)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cpx<R> d0 = p.v[2][c], d1 = p.v[3][c];
        cpx<R> e0, e1;  // e_mu psi_d
        if (MU == 0) { e0 = -d0; e1 = -d1; }
        else if (MU == 1) { e0 = timesMinusI(d1); e1 = timesMinusI(d0); }
        else if (MU == 2) { e0 = -d1; e1 = d0; }
        else { e0 = timesMinusI(d0); e1 = timesI(d1); }
        h.v[0][c] = {p.v[0][c].re + sg * e0.re, p.v[0][c].im + sg * e0.im};
        h.v[1][c] = {p.v[1][c].re + sg * e1.re, p.v[1][c].im + sg * e1.im};
    }
}

// acc += ph (w, sg e_mu^dag w)
template <int MU, typename R>
__device__ __forceinline__ void reconstruct_sg(Spinor<R> &acc, const Half<R> &w, R ph, R sgph)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cpx<R> w0 = w.v[0][c], w1 = w.v[1][c];
        cpx<R> f0, f1;  // e_mu^dag w
        if (MU == 0) { f0 = -w0; f1 = -w1; }
        else if (MU == 1) { f0 = timesI(w1); f1 = timesI(w0); }
        else if (MU == 2) { f0 = w1; f1 = -w0; }
        else { f0 = timesI(w0); f1 = timesMinusI(w1); }
        acc.v[0][c] = {acc.v[0][c].re + ph * w0.re, acc.v[0][c].im + ph * w0.im};
        acc.v[1][c] = {acc.v[1][c].re + ph * w1.re, acc.v[1][c].im + ph * w1.im};
        acc.v[2][c] = {acc.v[2][c].re + sgph * f0.re, acc.v[2][c].im + sgph * f0.im};
        acc.v[3][c] = {acc.v[3][c].re + sgph * f1.re, acc.v[3][c].im + sgph * f1.im};
    }
}

template <typename R> __device__ __forceinline__ void dagger(Link<R> &L)
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        L.m[a][a].im = -L.m[a][a].im;
#pragma unroll
        for (int b = a + 1; b < 3; b++) {
            cpx<R> t = L.m[a][b];
            L.m[a][b] = {L.m[b][a].re, -L.m[b][a].im};
            L.m[b][a] = {t.re, -t.im};
        }
    }
}

// one direction, sign given at run time (dir +1: forward, -1: backward), NR right-hand sides
template <class P, int BL, int HOPSEL, int MU, int NR>
__device__ __forceinline__ void hop_dir_sg(const GeomDev &g, const Site<BL> &st, int s, int dir,
                                           const typename P::SElem *in, long rstride,
                                           const typename P::UElem *__restrict__ U,
                                           Spinor<typename P::R> (&acc)[NR])
{
    using R = typename P::R;
    bool cross;
    int phi;
    const int sn = neighbour<BL>(st, MU, dir, g, &cross, &phi);
    if (!(HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross))) return;
    Link<R> L;
    P::load_link(U, g.V, MU, dir > 0 ? s : sn, L);
    if (dir < 0) dagger(L);
    const R sg = dir > 0 ? R(-1) : R(1);  // (1 - g_mu) forward, (1 + g_mu) backward
    const R ph = phi < 0 ? R(-1) : R(1);
    const R sgph = sg * ph;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        Spinor<R> p;
        Half<R> h, w;
        if constexpr (Normed<P>::value) {
            R n;
            P::load_spinor_unscaled(in + r * rstride, (int)g.V, sn, p, n);
            project_sg<MU>(p, sg, h);
            link_mul(L, h, w);
            reconstruct_sg<MU>(acc[r], w, ph * n, sgph * n);
        } else {
            P::load_spinor(in + r * rstride, (int)g.V, sn, p);
            project_sg<MU>(p, sg, h);
            link_mul(L, h, w);
            reconstruct_sg<MU>(acc[r], w, ph, sgph);
        }
    }
}

template <class P, int BL, int HOPSEL, int NR>
__device__ __forceinline__ void hop_multi_rolled(const GeomDev &g, const Site<BL> &st, int s,
                                                 const typename P::SElem *in, long rstride,
                                                 const typename P::UElem *__restrict__ U,
                                                 Spinor<typename P::R> (&acc)[NR])
{
#pragma unroll 1
    for (int k = 0; k < 2; k++) {
        const int dir = 1 - 2 * k;
        hop_dir_sg<P, BL, HOPSEL, 0, NR>(g, st, s, dir, in, rstride, U, acc);
        hop_dir_sg<P, BL, HOPSEL, 1, NR>(g, st, s, dir, in, rstride, U, acc);
        hop_dir_sg<P, BL, HOPSEL, 2, NR>(g, st, s, dir, in, rstride, U, acc);
        hop_dir_sg<P, BL, HOPSEL, 3, NR>(g, st, s, dir, in, rstride, U, acc);
    }
}

// ---- fully rolled form (one right-hand side): the eight hops share one body -- one link
// multiply, the direction entering the spin projection and reconstruction through a switch of
// four short cases and the signs through negations, never through multiplications (with
// double-single numbers a multiplication by -1 would cost a two-product).  About a quarter of the
// rolled form's code for instruction-fetch-bound storage (the double-single residual).

template <typename R> __device__ __forceinline__ cpx<R> neg_if(cpx<R> a, bool n) { return n ? -a : a; }

// h = psi_u + sg e_mu psi_d, sg = -1 (fwd, the (1 - g_mu) projector) or +1
template <typename R>
__device__ __forceinline__ void project_rt(const Spinor<R> &p, int mu, bool fwd, Half<R> &h)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cpx<R> d0 = p.v[2][c], d1 = p.v[3][c];
        cpx<R> e0, e1;  // e_mu psi_d
        switch (mu) {
        case 0: e0 = -d0; e1 = -d1; break;
        case 1: e0 = timesMinusI(d1); e1 = timesMinusI(d0); break;
        case 2: e0 = -d1; e1 = d0; break;
        default: e0 = timesMinusI(d0); e1 = timesI(d1); break;
        }
        h.v[0][c] = p.v[0][c] + neg_if(e0, fwd);
        h.v[1][c] = p.v[1][c] + neg_if(e1, fwd);
    }
}

// acc += ph (w, sg e_mu^dag w), ph = -1 when flip, sg as in project_rt
template <typename R>
__device__ __forceinline__ void reconstruct_rt(Spinor<R> &acc, const Half<R> &w, int mu, bool fwd, bool flip)
{
    const bool nd = fwd != flip;  // sg ph < 0
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cpx<R> w0 = w.v[0][c], w1 = w.v[1][c];
        cpx<R> f0, f1;  // e_mu^dag w
        switch (mu) {
        case 0: f0 = -w0; f1 = -w1; break;
        case 1: f0 = timesI(w1); f1 = timesI(w0); break;
        case 2: f0 = w1; f1 = -w0; break;
        default: f0 = timesI(w0); f1 = timesMinusI(w1); break;
        }
        acc.v[0][c] = acc.v[0][c] + neg_if(w0, flip);
        acc.v[1][c] = acc.v[1][c] + neg_if(w1, flip);
        acc.v[2][c] = acc.v[2][c] + neg_if(f0, nd);
        acc.v[3][c] = acc.v[3][c] + neg_if(f1, nd);
    }
}

template <class P, int BL, int HOPSEL>
__device__ __forceinline__ void hop_fully_rolled(const GeomDev &g, const Site<BL> &st, int s,
                                                 const typename P::SElem *in,
                                                 const typename P::UElem *__restrict__ U,
                                                 Spinor<typename P::R> &acc)
{
    using R = typename P::R;
#pragma unroll 1
    for (int k = 0; k < 8; k++) {
        const int mu = k >> 1;
        const bool fwd = (k & 1) == 0;
        bool cross;
        int phi;
        const int sn = neighbour<BL>(st, mu, fwd ? 1 : -1, g, &cross, &phi);
        if (!(HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross))) continue;
        Link<R> L;
        P::load_link(U, (int)g.V, mu, fwd ? s : sn, L);
        if (!fwd) dagger(L);
        Spinor<R> p;
        P::load_spinor(in, (int)g.V, sn, p);
        Half<R> h, w;
        project_rt(p, mu, fwd, h);
        link_mul(L, h, w);
        reconstruct_rt(acc, w, mu, fwd, phi < 0);
    }
}

// ---- batched form (one right-hand side): the loads of G hops are all issued before any of them
// is used, so a site waits for memory 8 / G times instead of 8.  Hop k = 0..7 is direction
// mu = k / 2, forward for even k, backward for odd k.

template <class P, int BL, int HOPSEL, int K> struct HopK {
    using R = typename P::R;
    static constexpr int MU = K / 2;
    static constexpr int DIR = (K & 1) ? -1 : 1;
    __device__ static __forceinline__ bool issue(const GeomDev &g, const Site<BL> &st, int s,
                                                 const typename P::SElem *in,
                                                 const typename P::UElem *__restrict__ U,
                                                 typename P::SRaw &sr, typename P::URaw &ur, int &ph)
    {
        bool cross;
        const int sn = neighbour<BL>(st, MU, DIR, g, &cross, &ph);
        if (!(HOPSEL == 0 || (HOPSEL == 1 && !cross) || (HOPSEL == 2 && cross))) return false;
        P::load_raw(in, (int)g.V, sn, sr);
        P::load_link_raw(U, (int)g.V, MU, DIR > 0 ? s : sn, ur);
        return true;
    }
    __device__ static __forceinline__ void compute(const typename P::SRaw &sr, const typename P::URaw &ur, int ph,
                                                   Spinor<R> &acc)
    {
        Spinor<R> p;
        Link<R> L;
        P::decode_link(ur, L);
        Half<R> h, w;
        if constexpr (Normed<P>::value) {
            P::decode_unscaled(sr, p);
            project<MU, -DIR>(p, h);
            if (DIR > 0) link_mul(L, h, w);
            else link_dag_mul(L, h, w);
            reconstruct_add_scaled<MU, -DIR>(acc, w, ph < 0 ? -sr.n : sr.n);
            return;
        }
        P::decode(sr, p);
        project<MU, -DIR>(p, h);
        if (DIR > 0) link_mul(L, h, w);
        else link_dag_mul(L, h, w);
        if (ph < 0)
#pragma unroll
            for (int a = 0; a < 2; a++)
#pragma unroll
                for (int c = 0; c < 3; c++) w.v[a][c] = -w.v[a][c];
        reconstruct_add<MU, -DIR>(acc, w);
    }
};

template <class P, int BL, int HOPSEL, int K0, int G> struct HopBatch {
    using R = typename P::R;
    __device__ static __forceinline__ void run(const GeomDev &g, const Site<BL> &st, int s,
                                               const typename P::SElem *in,
                                               const typename P::UElem *__restrict__ U, Spinor<R> &acc)
    {
        typename P::SRaw sr[G];
        typename P::URaw ur[G];
        int ph[G];
        bool act[G];
        issue_all<0>(g, st, s, in, U, sr, ur, ph, act);
        compute_all<0>(sr, ur, ph, act, acc);
    }
    template <int J>
    __device__ static __forceinline__ void issue_all(const GeomDev &g, const Site<BL> &st, int s,
                                                     const typename P::SElem *in,
                                                     const typename P::UElem *__restrict__ U, typename P::SRaw *sr,
                                                     typename P::URaw *ur, int *ph, bool *act)
    {
        if constexpr (J < G) {
            act[J] = HopK<P, BL, HOPSEL, K0 + J>::issue(g, st, s, in, U, sr[J], ur[J], ph[J]);
            issue_all<J + 1>(g, st, s, in, U, sr, ur, ph, act);
        }
    }
    template <int J>
    __device__ static __forceinline__ void compute_all(const typename P::SRaw *sr, const typename P::URaw *ur,
                                                       const int *ph, const bool *act, Spinor<R> &acc)
    {
        if constexpr (J < G) {
            if (act[J]) HopK<P, BL, HOPSEL, K0 + J>::compute(sr[J], ur[J], ph[J], acc);
            compute_all<J + 1>(sr, ur, ph, act, acc);
        }
    }
};

template <class P, int BL, int HOPSEL, int G>
__device__ __forceinline__ void hop_batched(const GeomDev &g, const Site<BL> &st, int s, const typename P::SElem *in,
                                            const typename P::UElem *__restrict__ U, Spinor<typename P::R> &acc)
{
    HopBatch<P, BL, HOPSEL, 0, G>::run(g, st, s, in, U, acc);
    if constexpr (G < 8) HopBatch<P, BL, HOPSEL, G, G>::run(g, st, s, in, U, acc);
    if constexpr (G < 4) {
        HopBatch<P, BL, HOPSEL, 2 * G, G>::run(g, st, s, in, U, acc);
        HopBatch<P, BL, HOPSEL, 3 * G, G>::run(g, st, s, in, U, acc);
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
