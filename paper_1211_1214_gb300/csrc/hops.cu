// hops.cu -- the hopping terms between blocks of Eq. 1 (D_wb, D_bw, K5b) in FP64.
//
// Only the sites on a block face have a hop that leaves their block (one per site on average for
// 8^4 blocks).  A launch over all sites of a colour idles most lanes of a warp on most of the
// eight hop bodies; here each direction is one launch over exactly the face sites of that
// direction, so every thread does one hop and no lane idles.  The eight launches run in order, so
// a site on an edge or corner (faces of several directions) is updated by one launch at a time.
#include "ctx.h"
#include "stencil.cuh"

namespace ddrw {

namespace {

// out(s) += beta * [hop of direction k across the face], s on the face of direction k of a block
// of [blk0, blk0 + nblk); k = 2 mu (forward, (1 - g_mu) U_mu(s) in(s + mu)) or 2 mu + 1 (backward,
// (1 + g_mu) U_mu(s - mu)^dag in(s - mu)); right-hand side blockIdx.y
template <int BL>
__global__ void __launch_bounds__(128) k_hop_face(GeomDev g, const double2 *__restrict__ in, double2 *out, long rs,
                                                  int blk0, int nblk, int k, double beta,
                                                  const double2 *__restrict__ U)
{
    constexpr int F = BL * BL * BL;  // face sites of one block and direction (both parities)
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)nblk * F) return;
    const long ro = (long)blockIdx.y * rs;
    const int b = blk0 + (int)(i / F);
    int rem = (int)(i % F);
    const int mu = k >> 1;
    const bool fwd = (k & 1) == 0;
    int c[4];
#pragma unroll
    for (int nu = 3; nu >= 0; nu--) {  // the three free in-block coordinates, z fastest
        if (nu == mu) continue;
        c[nu] = rem % BL;
        rem /= BL;
    }
    c[mu] = fwd ? BL - 1 : 0;
    const int lb = ((c[0] * BL + c[1]) * BL + c[2]) * BL + c[3];
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;  // block origins are even
    const int s = (int)((long)par * g.vh + (long)b * BlockShape<BL>::VBH + (lb >> 1));
    Site<BL> st;
    decode_site<BL>(s, g, st);
    bool cross;
    int phi;
    const int sn = neighbour<BL>(st, mu, fwd ? 1 : -1, g, &cross, &phi);
    Link<double> L;
    PrecD::load_link(U, (int)g.V, mu, fwd ? s : sn, L);
    if (!fwd) dagger(L);
    Spinor<double> p;
    PrecD::load_spinor(in + ro, (int)g.V, sn, p);
    Half<double> h, w;
    project_rt(p, mu, fwd, h);
    link_mul(L, h, w);
    Spinor<double> acc;
    zero(acc);
    reconstruct_rt(acc, w, mu, fwd, phi < 0);
    Spinor<double> o;
    PrecD::load_spinor_rw(out + ro, (int)g.V, s, o);
    axpy(o, beta, acc);
    PrecD::store_spinor(out + ro, (int)g.V, s, o);
}

template <int BL>
void hop_faces(ddrw_ctx *ctx, int blk0, int nblk, const double2 *in, double2 *out, int nrhs, double beta)
{
    GeomDev g = geom_dev(ctx);
    const long n = (long)nblk * BL * BL * BL;
    const dim3 grid((unsigned)((n + 127) / 128), (unsigned)nrhs);
    for (int k = 0; k < 8; k++) {
        ++ctx->launches;
        k_hop_face<BL><<<grid, 128, 0, ctx->stream>>>(g, in, out, 12 * ctx->V, blk0, nblk, k, beta, ctx->U64);
    }
}

}  // namespace

void hop_between64(ddrw_ctx *ctx, int rows, const double2 *in, double2 *out, int nrhs, double beta)
{
    const int blk0 = rows == DDRW_BLACK ? 0 : ctx->nblk_c, nblk = ctx->nblk_c;
    const int l = ctx->l;
    // compulsory bytes: the face sites' links, their neighbours' spinors, out read and written
    const double faces = 8.0 * nblk * l * l * l;
    ProfScope ps(ctx, PROF_DSLASH64_BLK, faces * (PrecD::UBYTES + 3.0 * PrecD::SBYTES * nrhs), faces * nrhs);
    switch (l) {
    case 2: hop_faces<2>(ctx, blk0, nblk, in, out, nrhs, beta); break;
    case 4: hop_faces<4>(ctx, blk0, nblk, in, out, nrhs, beta); break;
    case 6: hop_faces<6>(ctx, blk0, nblk, in, out, nrhs, beta); break;
    default: hop_faces<8>(ctx, blk0, nblk, in, out, nrhs, beta); break;
    }
}

}  // namespace ddrw
