// dslash.cuh -- the fused hopping + clover stencil of the Wilson-clover operator (K4) and its
// block-restricted forms (K5): D_bb / D_ww keep the hops inside a block, D_bw / D_wb the hops
// between blocks (Eq. 1).  One kernel template serves every form:
//
//   out(x) = POST( alpha * DIAG(x) + beta * sum_mu [ (1 - g_mu) U_mu(x) in(x+mu) + (1 + g_mu) U_mu(x-mu)^dag in(x-mu) ] )
//
// DIAG is A(m) x = (4 + m) x + C x (or x itself), POST an optional A(m)^-1.  A thread owns one
// site and NR right-hand sides: each link and clover block is loaded (and two-row links
// reconstructed) once for the NR.  Groups of NR right-hand sides are interleaved with the site
// tiles along gridDim.x (group fastest), so the groups of one tile run together and share the
// tile's links and clover terms through L2.  Right-hand sides carry mass slots (rhs / rpm), so one
// launch can hold several masses.  The SU(3) x spin stencil is not a dense contraction, so it
// runs on the FP32/FP64 ALUs, not on tensor cores.  Each hop projects the neighbour to a 2-spin
// half spinor before the colour multiply (half the complex multiplies of a 4-spin product).
//
// The launcher autotunes NR and the CTA size per launch shape on first use (dslash_tune.cu);
// every launch of this kernel is idempotent (its output sites are never among its inputs), so the
// tuning runs are harmless.
#pragma once

#include <type_traits>

#include "ctx.h"
#include "ddprec.cuh"
#include "lowprec.cuh"
#include "stencil.cuh"
#include "tma.cuh"

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
    const typename P::UElem *Ubw;         // backward links U_mu(x - mu) stored at x (staged form)
    int *err;                             // device error flags (bit 0: a staging wait ran out)
    int stall_tx;                         // test switch: bytes announced on top of the staged copies
    const typename P::SElem *w;           // fused inner products: the other vector of red 1
    double *part;                         // per-warp partial sums [rhs][n / 32][3]
    long nwt;                             // warps of 32 output sites per right-hand side (n / 32)
};

// ---- staged form (FP32 two-row links): one CTA covers a tile of consecutive output sites for all
// right-hand sides of one mass slot.  One warp stages the tile's links (forward ones at the site,
// backward ones from the copy stored at the site), the A^-1 and clover blocks the launch needs and
// the neighbour-table entries into shared memory with bulk asynchronous copies, completed on an
// mbarrier; then every thread runs its site for right-hand sides threadIdx.y, +blockDim.y, ...,
// reading those terms from shared memory and only the spinors from global memory.  Shared memory
// holds [plane][site of the tile] 16-byte elements:
//   0-11 forward links (mu, row-pair), 12-23 backward links, then 18 planes of A^-1 (post),
//   18 of the clover term (diag == 1), 2 of neighbour entries.
constexpr int STAGE_WAIT_TRIES = 1 << 16;

template <int BL>
__global__ void __launch_bounds__(256, 2) k_dslash_staged(GeomDev g, DsArgs<PrecS> a)
{
    using R = float;
    extern __shared__ __align__(128) float4 stg[];
    __shared__ __align__(8) uint64_t bar;
    const int NS = blockDim.x, W = blockDim.y;
    const int tid = threadIdx.y * NS + threadIdx.x;
    const int nslot = (a.nrhs + a.rpm - 1) / a.rpm;
    const long nper = (long)a.nblk * BlockShape<BL>::VBH;
    const long tile = blockIdx.x / nslot;
    const int slot = (int)(blockIdx.x - tile * nslot);
    const long i0 = tile * NS;
    const int nvalid = (int)min((long)NS, nper * a.npar - i0);
    const int pp = (int)(i0 / nper);  // the tile lies in one parity (launcher's rule)
    const long s0 = (long)(a.par0 + pp) * g.vh + (long)a.blk0 * BlockShape<BL>::VBH + (i0 - pp * nper);
    const long V = g.V;
    const int pA = 24, pC = pA + (a.post ? 18 : 0), pN = pC + (a.diag == 1 ? 18 : 0), np = pN + 2;

    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid < 32) {  // warp 0 issues the copies, lane k the planes k, k + 32
        const uint32_t seg = (uint32_t)nvalid * 16u;
        if (tid == 0) mbar_arrive_expect_tx(&bar, seg * (uint32_t)np + (uint32_t)a.stall_tx);
        __syncwarp();
        for (int q = tid; q < np; q += 32) {
            const void *src;
            if (q < 12) src = a.U + (long)q * V + s0;
            else if (q < 24) src = a.Ubw + (long)(q - 12) * V + s0;
            else if (q < pC) src = a.Ainv[slot] + (long)(q - pA) * V + s0;
            else if (q < pN) src = a.Cl + (long)(q - pC) * V + s0;
            else src = g.nbr + (long)(q - pN) * V + s0;
            bulk_copy_g2s(stg + (long)q * NS, src, seg, &bar);
        }
    }
    if (!mbar_wait_bounded(&bar, 0, STAGE_WAIT_TRIES)) {
        if (threadIdx.x == 0) atomicOr(a.err, 1);
        return;
    }
    const int j = threadIdx.x;
    if (j >= nvalid) return;
    const int s = (int)(s0 + j);
    // neighbour entry q = 2 mu + d of this site: component q % 4 of plane pN + q / 4
    const int *nb = reinterpret_cast<const int *>(stg + (long)pN * NS + j);
    const int rb = slot * a.rpm, re = min(rb + a.rpm, a.nrhs);
    for (int r = rb + threadIdx.y; r < re; r += W) {
        const long roff = (long)r * a.rstride;
        Spinor<R> acc;
        zero(acc);
        if (a.beta != R(0)) {
            const float4 *in = a.in + roff;
#pragma unroll
            for (int mu = 0; mu < 4; mu++)
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    const int q = 2 * mu + d;
                    const int e = nb[(q / 4) * 4 * NS + q % 4];
                    const int n = e & NBR_IDX;
                    const bool flip = e < 0 && g.tsign < 0;
                    const float4 *lk = stg + (long)(d * 12 + mu * 3) * NS + j;
                    const float4 a0 = lk[0], a1 = lk[NS], a2 = lk[2 * NS];
                    Link<R> L;
                    L.m[0][0] = {a0.x, a0.y};
                    L.m[0][1] = {a0.z, a0.w};
                    L.m[0][2] = {a1.x, a1.y};
                    L.m[1][0] = {a1.z, a1.w};
                    L.m[1][1] = {a2.x, a2.y};
                    L.m[1][2] = {a2.z, a2.w};
                    PrecS::reconstruct_row2(L);
                    Spinor<R> p;
                    PrecS::load_spinor(in, (int)V, n, p);
                    Half<R> h, w;
                    if (d == 0) {
                        if (mu == 0) project<0, -1>(p, h);
                        else if (mu == 1) project<1, -1>(p, h);
                        else if (mu == 2) project<2, -1>(p, h);
                        else project<3, -1>(p, h);
                        link_mul(L, h, w);
                    } else {
                        if (mu == 0) project<0, +1>(p, h);
                        else if (mu == 1) project<1, +1>(p, h);
                        else if (mu == 2) project<2, +1>(p, h);
                        else project<3, +1>(p, h);
                        link_dag_mul(L, h, w);
                    }
                    if (flip)
#pragma unroll
                        for (int b = 0; b < 2; b++)
#pragma unroll
                            for (int c = 0; c < 3; c++) w.v[b][c] = -w.v[b][c];
                    if (d == 0) {
                        if (mu == 0) reconstruct_add<0, -1>(acc, w);
                        else if (mu == 1) reconstruct_add<1, -1>(acc, w);
                        else if (mu == 2) reconstruct_add<2, -1>(acc, w);
                        else reconstruct_add<3, -1>(acc, w);
                    } else {
                        if (mu == 0) reconstruct_add<0, +1>(acc, w);
                        else if (mu == 1) reconstruct_add<1, +1>(acc, w);
                        else if (mu == 2) reconstruct_add<2, +1>(acc, w);
                        else reconstruct_add<3, +1>(acc, w);
                    }
                }
            scale(acc, a.beta);
        }
        if (a.diag) {
            const float4 *x = a.x + roff;
#pragma unroll
            for (int ch = 0; ch < 2; ch++) {
                cpx<R> v6[6], o6[6];
                PrecS::load_chiral(x, (int)V, s, ch, v6);
                if (a.diag == 1) {
                    R c[36];
#pragma unroll
                    for (int k = 0; k < 9; k++) {
                        const float4 q = stg[(long)(pC + ch * 9 + k) * NS + j];
                        c[4 * k] = q.x;
                        c[4 * k + 1] = q.y;
                        c[4 * k + 2] = q.z;
                        c[4 * k + 3] = q.w;
                    }
                    herm6_mul<R>(c, a.mass4[slot], v6, o6);
                } else {
#pragma unroll
                    for (int k = 0; k < 6; k++) o6[k] = v6[k];
                }
#pragma unroll
                for (int k = 0; k < 6; k++)
                    acc.v[2 * ch + k / 3][k % 3] = acc.v[2 * ch + k / 3][k % 3] + a.alpha * o6[k];
            }
        }
        if (a.post) {
#pragma unroll
            for (int ch = 0; ch < 2; ch++) {
                R c[36];
#pragma unroll
                for (int k = 0; k < 9; k++) {
                    const float4 q = stg[(long)(pA + ch * 9 + k) * NS + j];
                    c[4 * k] = q.x;
                    c[4 * k + 1] = q.y;
                    c[4 * k + 2] = q.z;
                    c[4 * k + 3] = q.w;
                }
                cpx<R> v6[6], o6[6];
#pragma unroll
                for (int k = 0; k < 6; k++) v6[k] = acc.v[2 * ch + k / 3][k % 3];
                herm6_mul<R>(c, R(0), v6, o6);
#pragma unroll
                for (int k = 0; k < 6; k++) acc.v[2 * ch + k / 3][k % 3] = o6[k];
            }
        }
        PrecS::store_spinor(a.out + roff, (int)V, s, acc);
    }
}

// shared memory of a staged launch, and the largest any staged launch asks for
inline size_t staged_smem(int nt, int diag, int post) { return (size_t)(26 + 18 * (post != 0) + 18 * (diag == 1)) * nt * 16; }
constexpr size_t STAGED_SMEM_MAX = (size_t)62 * 128 * 16;

// ROLL selects the hop code form: 0 unrolled, 1 rolled, 2 / 3 batched loads of 4 / 8 hops,
// 4 / 5 unrolled compiled for at least 3 / 2 CTAs of 256 threads per SM (<= 85 / 128 registers),
// 6 / 7 as 5 / 4 with the neighbours read from the neighbour table instead of computed,
// 11 fully rolled (one body for the eight hops; double-single storage only)
// RED != 0 adds the inner products of the output to the epilogue (red 1: conj(w) out; red 2:
// conj(out) x and |out|^2), one partial per warp of 32 sites, summed in FP64 by k_bicg_fin; the
// launcher only fuses launches whose output sites fill whole CTAs (no thread leaves early)
template <class P, int BL, int HOPSEL, int NR, int ROLL = 0, int RED = 0>
__global__ void __launch_bounds__(256, (ROLL == 4 || ROLL == 7) ? 3 : (ROLL == 5 || ROLL == 6) ? 2 : 1)
    k_dslash(GeomDev g, DsArgs<P> a)
{
    using R = typename P::R;
    // groups of NR right-hand sides; a CTA holds blockDim.y groups (one per row of threads) of
    // the same site tile, so its rows share the tile's links and clover terms in L1
    const int ncg = a.nrhs / (NR * (int)blockDim.y);
    const int grp = (blockIdx.x % ncg) * blockDim.y + threadIdx.y;
    const long tile = blockIdx.x / ncg;
    const long nper = (long)a.nblk * BlockShape<BL>::VBH;
    const long i = tile * blockDim.x + threadIdx.x;
    if (i >= nper * a.npar) return;
    const int r0 = grp * NR;
    const long roff = (long)r0 * a.rstride;
    const int pp = (int)(i / nper);
    const long s = (long)(a.par0 + pp) * g.vh + (long)a.blk0 * BlockShape<BL>::VBH + (i - pp * nper);
    Site<BL> st;
    int4 n0;
    if constexpr (ROLL == 6 || ROLL == 7) {
        n0 = g.nbr[s];
    } else {
        decode_site<BL>(s, g, st);
    }

    Spinor<R> acc[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) zero(acc[r]);
    if (a.beta != R(0)) {
        const typename P::SElem *in = a.in + roff;
        if constexpr (ROLL == 2 || ROLL == 3) {  // batched loads, one right-hand side: 2 -> 4 hops, 3 -> 8 hops per batch
            static_assert(NR == 1, "batched hops take one right-hand side per thread");
            hop_batched<P, BL, HOPSEL, ROLL == 2 ? 4 : 8>(g, st, (int)s, in, a.U, acc[0]);
        } else if constexpr (ROLL == 11) {  // fully rolled, one right-hand side
            static_assert(NR == 1, "the fully rolled form takes one right-hand side per thread");
            hop_fully_rolled<P, BL, HOPSEL>(g, st, (int)s, in, a.U, acc[0]);
        } else if constexpr (ROLL == 6 || ROLL == 7) {
            hop_tab<P, HOPSEL, 0, NR>(g, n0.x, n0.y, (int)s, in, a.rstride, a.U, acc);
            hop_tab<P, HOPSEL, 1, NR>(g, n0.z, n0.w, (int)s, in, a.rstride, a.U, acc);
            const int4 n1 = g.nbr[g.V + s];  // loaded here: fewer registers live over the first hops
            hop_tab<P, HOPSEL, 2, NR>(g, n1.x, n1.y, (int)s, in, a.rstride, a.U, acc);
            hop_tab<P, HOPSEL, 3, NR>(g, n1.z, n1.w, (int)s, in, a.rstride, a.U, acc);
        } else if constexpr (ROLL == 1) {
            hop_multi_rolled<P, BL, HOPSEL, NR>(g, st, (int)s, in, a.rstride, a.U, acc);
        } else {
            hop_dir_multi<P, BL, HOPSEL, 0, NR>(g, st, s, in, a.rstride, a.U, acc);
            hop_dir_multi<P, BL, HOPSEL, 1, NR>(g, st, s, in, a.rstride, a.U, acc);
            hop_dir_multi<P, BL, HOPSEL, 2, NR>(g, st, s, in, a.rstride, a.U, acc);
            hop_dir_multi<P, BL, HOPSEL, 3, NR>(g, st, s, in, a.rstride, a.U, acc);
        }
#pragma unroll
        for (int r = 0; r < NR; r++) scale(acc[r], a.beta);
    }
    if constexpr (std::is_same<P, PrecDD>::value) {
        // double-single: one chirality body run twice (the clover multiply in FP32 pairs is large,
        // and this kernel is limited by instruction fetch)
        if (a.diag) {
            const typename P::SElem *x = a.x + roff;
#pragma unroll 1
            for (int ch = 0; ch < 2; ch++) {
                R c[36];
                cpx<R> v6[6], o6[6];
                P::load_chiral(x, g.V, s, ch, v6);
                if (a.diag == 1) {
                    P::load_clover(a.Cl, g.V, s, ch, c);
                    herm6_mul<R>(c, a.mass4[r0 / a.rpm], v6, o6);
                } else {
#pragma unroll
                    for (int k = 0; k < 6; k++) o6[k] = v6[k];
                }
                if (ch == 0) {
#pragma unroll
                    for (int k = 0; k < 6; k++) acc[0].v[k / 3][k % 3] = acc[0].v[k / 3][k % 3] + a.alpha * o6[k];
                } else {
#pragma unroll
                    for (int k = 0; k < 6; k++)
                        acc[0].v[2 + k / 3][k % 3] = acc[0].v[2 + k / 3][k % 3] + a.alpha * o6[k];
                }
            }
        }
    } else if (a.diag) {
        const typename P::SElem *x = a.x + roff;
#pragma unroll
        for (int ch = 0; ch < 2; ch++) {
            R c[36];
            if (a.diag == 1) P::load_clover(a.Cl, g.V, s, ch, c);
#pragma unroll
            for (int r = 0; r < NR; r++) {
                cpx<R> v6[6], o6[6];
                P::load_chiral(x + r * a.rstride, g.V, s, ch, v6);
                if (a.diag == 1) herm6_mul<R>(c, a.mass4[(r0 + r) / a.rpm], v6, o6);
                else
#pragma unroll
                    for (int k = 0; k < 6; k++) o6[k] = v6[k];
#pragma unroll
                for (int k = 0; k < 6; k++)
                    acc[r].v[2 * ch + k / 3][k % 3] = acc[r].v[2 * ch + k / 3][k % 3] + a.alpha * o6[k];
            }
        }
    }
    if (a.post) {
        // a group of NR right-hand sides never straddles two mass slots (launcher's rule)
        const typename P::CElem *Ai = a.Ainv[r0 / a.rpm];
#pragma unroll
        for (int ch = 0; ch < 2; ch++) {
            R c[36];
            P::load_clover(Ai, g.V, s, ch, c);
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
    }
    if constexpr (RED != 0) {
        static_assert(NR == 1, "fused inner products take one right-hand side per thread");
        Spinor<R> q;
        P::load_spinor(RED == 1 ? a.w + roff : a.x + roff, g.V, s, q);
        R d0 = 0, d1 = 0, d2 = 0;
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const cpx<R> z = RED == 1 ? cmulc(q.v[sp][c], acc[0].v[sp][c]) : cmulc(acc[0].v[sp][c], q.v[sp][c]);
                d0 += z.re;
                d1 += z.im;
                d2 += acc[0].v[sp][c].re * acc[0].v[sp][c].re + acc[0].v[sp][c].im * acc[0].v[sp][c].im;
            }
        double e0 = d0, e1 = d1, e2 = d2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e0 += __shfl_xor_sync(0xffffffffu, e0, o);
            e1 += __shfl_xor_sync(0xffffffffu, e1, o);
            e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        }
        if ((threadIdx.x & 31) == 0) {
            double *pp = a.part + ((long)r0 * a.nwt + tile * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 3;
            pp[0] = e0;
            pp[1] = e1;
            pp[2] = e2;
        }
    }
#pragma unroll
    for (int r = 0; r < NR; r++) P::store_spinor(a.out + roff + r * a.rstride, g.V, s, acc[r]);
}

// ---- pipelined form (FP32 storage, all hops, one right-hand side per thread): the neighbour
// spinor and the link of every hop are brought into a two-slot ring in shared memory with 16-byte
// asynchronous copies (cp.async), two hops ahead of the arithmetic, so that the loads in flight
// hold no registers and each thread keeps two hops' worth of memory requests outstanding.  The
// neighbours come from the neighbour table, the backward links from their copy stored at the site
// (coalesced).  Ring layout: [slot][plane 0-5 spinor, 6-8 link][thread], 16-byte elements.

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

inline size_t pipe_smem(int nthreads) { return (size_t)2 * 9 * nthreads * 16; }

// issue the copies of hop q (2 mu + backward) of site s into ring slot q % 2
__device__ __forceinline__ void pipe_issue(float4 *ring, int nth, int tid, int q, int e, int s, long V, const float4 *in,
                                           const float4 *U, const float4 *Ubw)
{
    float4 *dst = ring + (long)((q & 1) * 9) * nth + tid;
    const int n = e & NBR_IDX, mu = q >> 1;
#pragma unroll
    for (int k = 0; k < 6; k++) cp_async16(dst + k * nth, in + k * V + n);
    const float4 *L = ((q & 1) ? Ubw : U) + (long)mu * 3 * V + s;
#pragma unroll
    for (int k = 0; k < 3; k++) cp_async16(dst + (6 + k) * nth, L + k * V);
    cp_async_commit();
}

// hop Q from its ring slot: acc += (1 -+ g_mu) U^(dag) in(x +- mu), then refill the slot with hop Q + 2
template <int Q>
__device__ __forceinline__ void pipe_hop(float4 *ring, int nth, int tid, const int (&nb)[8], int s, long V,
                                         const float4 *in, const float4 *U, const float4 *Ubw, int tsign,
                                         Spinor<float> &acc)
{
    constexpr int MU = Q >> 1;
    if (Q < 7) cp_async_wait<1>();
    else cp_async_wait<0>();
    const float4 *src = ring + (long)((Q & 1) * 9) * nth + tid;
    Spinor<float> p;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const float4 v = src[k * nth];
        p.v[(2 * k) / 3][(2 * k) % 3] = {v.x, v.y};
        p.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = {v.z, v.w};
    }
    PrecS::URaw ur;
#pragma unroll
    for (int k = 0; k < 3; k++) ur.e[k] = src[(6 + k) * nth];
    Link<float> L;
    PrecS::decode_link(ur, L);
    Half<float> h, w;
    if ((Q & 1) == 0) {
        project<MU, -1>(p, h);
        link_mul(L, h, w);
    } else {
        project<MU, +1>(p, h);
        link_dag_mul(L, h, w);
    }
    if (nb[Q] < 0 && tsign < 0)
#pragma unroll
        for (int x = 0; x < 2; x++)
#pragma unroll
            for (int c = 0; c < 3; c++) w.v[x][c] = -w.v[x][c];
    if ((Q & 1) == 0) reconstruct_add<MU, -1>(acc, w);
    else reconstruct_add<MU, +1>(acc, w);
    if (Q + 2 < 8) pipe_issue(ring, nth, tid, Q + 2, nb[(Q + 2) & 7], s, V, in, U, Ubw);
}

template <int BL, int MINB>
__global__ void __launch_bounds__(256, MINB) k_dslash_pipe(GeomDev g, DsArgs<PrecS> a)
{
    using R = float;
    extern __shared__ __align__(16) float4 ring[];
    const int nth = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int ncg = a.nrhs / (int)blockDim.y;
    const int grp = (blockIdx.x % ncg) * blockDim.y + threadIdx.y;
    const long tile = blockIdx.x / ncg;
    const long nper = (long)a.nblk * BlockShape<BL>::VBH;
    const long i = tile * blockDim.x + threadIdx.x;
    if (i >= nper * a.npar) return;  // no barrier below: threads past the end may leave
    const long roff = (long)grp * a.rstride;
    const int pp = (int)(i / nper);
    const int s = (int)((long)(a.par0 + pp) * g.vh + (long)a.blk0 * BlockShape<BL>::VBH + (i - pp * nper));
    const long V = g.V;
    Spinor<R> acc;
    zero(acc);
    if (a.beta != R(0)) {
        const float4 *in = a.in + roff;
        const int4 n0 = g.nbr[s], n1 = g.nbr[V + s];
        const int nb[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
        pipe_issue(ring, nth, tid, 0, nb[0], s, V, in, a.U, a.Ubw);
        pipe_issue(ring, nth, tid, 1, nb[1], s, V, in, a.U, a.Ubw);
        pipe_hop<0>(ring, nth, tid, nb, s, V, in, a.U, a.Ubw, g.tsign, acc);
        pipe_hop<1>(ring, nth, tid, nb, s, V, in, a.U, a.Ubw, g.tsign, acc);
        pipe_hop<2>(ring, nth, tid, nb, s, V, in, a.U, a.Ubw, g.tsign, acc);
        pipe_hop<3>(ring, nth, tid, nb, s, V, in, a.U, a.Ubw, g.tsign, acc);
        pipe_hop<4>(ring, nth, tid, nb, s, V, in, a.U, a.Ubw, g.tsign, acc);
        pipe_hop<5>(ring, nth, tid, nb, s, V, in, a.U, a.Ubw, g.tsign, acc);
        pipe_hop<6>(ring, nth, tid, nb, s, V, in, a.U, a.Ubw, g.tsign, acc);
        pipe_hop<7>(ring, nth, tid, nb, s, V, in, a.U, a.Ubw, g.tsign, acc);
        scale(acc, a.beta);
    }
    if (a.diag) {
        const float4 *x = a.x + roff;
#pragma unroll
        for (int ch = 0; ch < 2; ch++) {
            R c[36];
            if (a.diag == 1) PrecS::load_clover(a.Cl, V, s, ch, c);
            cpx<R> v6[6], o6[6];
            PrecS::load_chiral(x, (int)V, s, ch, v6);
            if (a.diag == 1) herm6_mul<R>(c, a.mass4[grp / a.rpm], v6, o6);
            else
#pragma unroll
                for (int k = 0; k < 6; k++) o6[k] = v6[k];
#pragma unroll
            for (int k = 0; k < 6; k++) acc.v[2 * ch + k / 3][k % 3] = acc.v[2 * ch + k / 3][k % 3] + a.alpha * o6[k];
        }
    }
    if (a.post) {
        const float4 *Ai = a.Ainv[grp / a.rpm];
#pragma unroll
        for (int ch = 0; ch < 2; ch++) {
            R c[36];
            PrecS::load_clover(Ai, V, s, ch, c);
            cpx<R> v6[6], o6[6];
#pragma unroll
            for (int k = 0; k < 6; k++) v6[k] = acc.v[2 * ch + k / 3][k % 3];
            herm6_mul<R>(c, R(0), v6, o6);
#pragma unroll
            for (int k = 0; k < 6; k++) acc.v[2 * ch + k / 3][k % 3] = o6[k];
        }
    }
    PrecS::store_spinor(a.out + roff, (int)V, s, acc);
}

// launch configuration of one stencil launch
struct DsConfig {
    int nr = 1;    // right-hand sides per thread
    int nt = 128;  // sites per CTA (threads per CTA row)
    int nw = 1;    // CTA rows: groups of nr right-hand sides per CTA (nt * nw <= 256)
    int roll = 0;  // 8: staged (FP32 storage; nt sites by nw rows of right-hand sides, links and
                   // clover terms in shared memory, every right-hand side of a mass slot per CTA);
                   // 1: forward and backward hops share the direction bodies (smaller code);
                   // 2 / 3: batched loads of 4 / 8 hops before their arithmetic (nr = 1); 4 / 5:
                   // unrolled with at most 85 / 128 registers, more warps per SM (nr = 1 / nr <= 2);
                   // 6 / 7: 5 / 4 with the neighbours from the neighbour table (nr <= 2 / nr = 1);
                   // 9 / 10: pipelined (FP32 storage, nr = 1): neighbour spinors and links two
                   // hops ahead through a shared-memory ring, at least 2 / 3 CTAs per SM
};

template <class P, int BL>
DsArgs<P> make_args(ddrw_ctx *ctx, const DslashCall &c)
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
    a.U = (const typename P::UElem *)links_for(ctx, P::ID);
    a.Cl = (const typename P::CElem *)clover_for(ctx, P::ID);
    a.Ubw = std::is_same<P, PrecS>::value ? (const typename P::UElem *)ctx->Ubw32 : nullptr;
    a.err = ctx->d_err;
    a.stall_tx = ctx->stall_tx;
    a.w = (const typename P::SElem *)c.w;
    a.part = c.red_part;
    a.nwt = (long)c.npar * c.nblk * BlockShape<BL>::VBH / 32;
    return a;
}

template <class P, int BL>
void launch_cfg(ddrw_ctx *ctx, const DslashCall &c, const DsArgs<P> &a, DsConfig cfg)
{
    GeomDev g = geom_dev(ctx);
    long n = (long)c.npar * c.nblk * BlockShape<BL>::VBH;
    // double-single launches and hops between blocks take one row; hops inside blocks take the
    // unrolled, register-capped or table form with one right-hand side per thread
    if (c.hopsel == 2) cfg.nr = 1, cfg.nw = 1, cfg.roll = 0;
    // double-single: one right-hand side per thread, unrolled or rolled hop code (the rolled form
    // has half the code of the unrolled one, which is instruction-fetch bound)
    if (std::is_same<P, PrecDD>::value)
        cfg.nr = 1, cfg.nw = 1, cfg.roll = ((cfg.roll == 1 || cfg.roll == 11) && c.hopsel != 2) ? cfg.roll : 0;
    if (!std::is_same<P, PrecDD>::value && c.hopsel == 1 && (cfg.nr != 1 || (cfg.roll != 0 && cfg.roll != 5 && cfg.roll != 6)))
        cfg.nr = 1, cfg.nw = 1, cfg.roll = 0;
    if (c.hopsel == 1 && cfg.roll == 6 && !g.nbr) cfg.roll = 5;
    if constexpr (std::is_same<P, PrecS>::value) {
        if (c.red != 0) {
            // the fused epilogue: one right-hand side per thread, unrolled or register-capped form,
            // whole CTAs (the caller checks that 256 divides the output sites)
            if (cfg.nr != 1 || (cfg.roll != 0 && cfg.roll != 5) || n % cfg.nt) cfg = DsConfig{1, 64, 1, 5};
            const unsigned gr = (unsigned)((n / cfg.nt) * (c.nrhs / cfg.nw));
            const dim3 bk((unsigned)cfg.nt, (unsigned)cfg.nw);
            ++ctx->launches;
            if (c.red == 1) {
                if (cfg.roll == 5) k_dslash<P, BL, 0, 1, 5, 1><<<gr, bk, 0, ctx->stream>>>(g, a);
                else k_dslash<P, BL, 0, 1, 0, 1><<<gr, bk, 0, ctx->stream>>>(g, a);
            } else {
                if (cfg.roll == 5) k_dslash<P, BL, 0, 1, 5, 2><<<gr, bk, 0, ctx->stream>>>(g, a);
                else k_dslash<P, BL, 0, 1, 0, 2><<<gr, bk, 0, ctx->stream>>>(g, a);
            }
            return;
        }
    }
    if (cfg.roll >= 6 && cfg.roll <= 7 && !g.nbr) cfg.roll = 11 - cfg.roll;  // no table: the computed-neighbour twin
    if (cfg.roll == 8) {
        // the staged form: FP32 storage, all hops, a tile never straddles the two parities
        const long nper = n / std::max(c.npar, 1);
        const bool ok = std::is_same<P, PrecS>::value && c.hopsel == 0 && g.nbr && a.Ubw && a.err &&
                        (c.npar == 1 || nper % cfg.nt == 0) && cfg.nt <= 128;
        if (!ok) cfg.nr = 1, cfg.nw = 1, cfg.roll = 5;
    }
    if (cfg.roll == 9 || cfg.roll == 10) {
        const bool ok = std::is_same<P, PrecS>::value && c.hopsel == 0 && g.nbr && a.Ubw && cfg.nr == 1;
        if (!ok) cfg.nr = 1, cfg.nw = 1, cfg.roll = 5;
    }
    if constexpr (std::is_same<P, PrecS>::value) {
        if (cfg.roll == 9 || cfg.roll == 10) {
            const int nth = cfg.nt * cfg.nw;
            const size_t smem = pipe_smem(nth);
            unsigned grid = (unsigned)(((n + cfg.nt - 1) / cfg.nt) * (c.nrhs / cfg.nw));
            ++ctx->launches;
            if (cfg.roll == 9) {
                cudaFuncSetAttribute(k_dslash_pipe<BL, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pipe_smem(256));
                k_dslash_pipe<BL, 2><<<grid, dim3((unsigned)cfg.nt, (unsigned)cfg.nw), smem, ctx->stream>>>(g, a);
            } else {
                cudaFuncSetAttribute(k_dslash_pipe<BL, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pipe_smem(256));
                k_dslash_pipe<BL, 3><<<grid, dim3((unsigned)cfg.nt, (unsigned)cfg.nw), smem, ctx->stream>>>(g, a);
            }
            return;
        }
        if (cfg.roll == 8) {
            const int nslot = (c.nrhs + a.rpm - 1) / a.rpm;
            static bool attr = false;  // per block length: the kernel may take up to STAGED_SMEM_MAX
            if (!attr) {
                cudaFuncSetAttribute(k_dslash_staged<BL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)STAGED_SMEM_MAX);
                attr = true;
            }
            ++ctx->launches;
            k_dslash_staged<BL><<<(unsigned)(((n + cfg.nt - 1) / cfg.nt) * nslot), dim3((unsigned)cfg.nt, (unsigned)cfg.nw),
                                  staged_smem(cfg.nt, c.diag, c.post), ctx->stream>>>(g, a);
            return;
        }
    }
    unsigned grid = (unsigned)(((n + cfg.nt - 1) / cfg.nt) * (c.nrhs / (cfg.nr * cfg.nw)));
    dim3 blk((unsigned)cfg.nt, (unsigned)cfg.nw);
    ++ctx->launches;
    if constexpr (std::is_same<P, PrecDD>::value) {  // one right-hand side per thread
        if (c.hopsel == 0 && cfg.roll == 1) k_dslash<P, BL, 0, 1, 1><<<grid, blk, 0, ctx->stream>>>(g, a);
        else if (c.hopsel == 1 && cfg.roll == 1) k_dslash<P, BL, 1, 1, 1><<<grid, blk, 0, ctx->stream>>>(g, a);
        else if (c.hopsel == 0 && cfg.roll == 11) k_dslash<P, BL, 0, 1, 11><<<grid, blk, 0, ctx->stream>>>(g, a);
        else if (c.hopsel == 1 && cfg.roll == 11) k_dslash<P, BL, 1, 1, 11><<<grid, blk, 0, ctx->stream>>>(g, a);
        else if (c.hopsel == 0) k_dslash<P, BL, 0, 1><<<grid, blk, 0, ctx->stream>>>(g, a);
        else if (c.hopsel == 1) k_dslash<P, BL, 1, 1><<<grid, blk, 0, ctx->stream>>>(g, a);
        else k_dslash<P, BL, 2, 1><<<grid, blk, 0, ctx->stream>>>(g, a);
    } else {
        if (c.hopsel == 0) {
            switch (cfg.roll * 8 + cfg.nr) {
            case 4: k_dslash<P, BL, 0, 4><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 2: k_dslash<P, BL, 0, 2><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 12: k_dslash<P, BL, 0, 4, 1><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 10: k_dslash<P, BL, 0, 2, 1><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 9: k_dslash<P, BL, 0, 1, 1><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 17: k_dslash<P, BL, 0, 1, 2><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 25: k_dslash<P, BL, 0, 1, 3><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 33: k_dslash<P, BL, 0, 1, 4><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 41: k_dslash<P, BL, 0, 1, 5><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 42: k_dslash<P, BL, 0, 2, 5><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 49: k_dslash<P, BL, 0, 1, 6><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 50: k_dslash<P, BL, 0, 2, 6><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            case 57: k_dslash<P, BL, 0, 1, 7><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            default: k_dslash<P, BL, 0, 1><<<grid, blk, 0, ctx->stream>>>(g, a); break;
            }
        } else if (c.hopsel == 1) {
            if (cfg.roll == 5) k_dslash<P, BL, 1, 1, 5><<<grid, blk, 0, ctx->stream>>>(g, a);
            else if (cfg.roll == 6) k_dslash<P, BL, 1, 1, 6><<<grid, blk, 0, ctx->stream>>>(g, a);
            else k_dslash<P, BL, 1, 1><<<grid, blk, 0, ctx->stream>>>(g, a);
        } else {
            k_dslash<P, BL, 2, 1><<<grid, blk, 0, ctx->stream>>>(g, a);
        }
    }
}

// compulsory bytes of a launch: per output site the R input, output and diagonal-input spinors,
// the links of its hops (8 per site when the output is one parity, since the backward links are
// stored at the other parity; 4 per site for both parities), clover terms once
template <class P>
double compulsory_bytes(const DslashCall &c, long n)
{
    const double S = P::SBYTES, Lk = P::UBYTES, Cb = P::CBYTES;
    double per = S * c.nrhs * ((c.beta != 0.0) + 1 + (c.diag != 0));
    if (c.beta != 0.0) per += (c.npar == 1 ? 8.0 : 4.0) * Lk;
    if (c.diag == 1) per += Cb;
    if (c.post) per += Cb;
    if (c.red == 1) per += S * c.nrhs;  // the fused inner product's second vector
    return per * (double)n;
}

DsConfig tuned_config(ddrw_ctx *ctx, const DslashCall &c, int prec, int bl,
                      void (*run)(ddrw_ctx *, const DslashCall &, DsConfig));

template <class P, int BL>
void run_cfg(ddrw_ctx *ctx, const DslashCall &c, DsConfig cfg)
{
    launch_cfg<P, BL>(ctx, c, make_args<P, BL>(ctx, c), cfg);
}

template <class P, int BL>
void launch_bl(ddrw_ctx *ctx, const DslashCall &c)
{
    using R = typename P::R;
    long n = (long)c.npar * c.nblk * BlockShape<BL>::VBH;
    if (n == 0 || c.nrhs == 0) return;
    DsConfig cfg;
    constexpr bool split = std::is_same<P, PrecDD>::value;
    if (c.hopsel != 2) cfg = tuned_config(ctx, c, P::ID, BL, &run_cfg<P, BL>);
    int kind = split ? PROF_DSLASH_DS
                     : P::ID < 32 ? PROF_DSLASH16 + (c.hopsel != 0)
                                  : (sizeof(R) == 8 ? PROF_DSLASH64 : PROF_DSLASH32) + (c.hopsel != 0 ? 2 : 0);
    ProfScope ps(ctx, kind, compulsory_bytes<P>(c, n), (double)n * c.nrhs);
    launch_cfg<P, BL>(ctx, c, make_args<P, BL>(ctx, c), cfg);
}

template <class P>
void launch(ddrw_ctx *ctx, const DslashCall &c)
{
    switch (ctx->l) {
    case 2: launch_bl<P, 2>(ctx, c); break;
    case 4: launch_bl<P, 4>(ctx, c); break;
    case 6: launch_bl<P, 6>(ctx, c); break;
    default: launch_bl<P, 8>(ctx, c); break;
    }
}

}  // namespace ddrw
