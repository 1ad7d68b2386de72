// clover.cuh -- the clover-term kernel (K2), instantiated per block length in clover_<l>.cu.
//   C = csw (i/4) sum sigma_{mu nu} Fhat_{mu nu},  Fhat = (Q_{mu nu} - Q_{nu mu}) / 8  from the four
//   plaquette leaves at each site, stored as two packed Hermitian 6x6 chirality blocks.
#pragma once

#include "ctx.h"

namespace ddrw {

struct M3 {
    cpx<double> m[3][3];
};

__device__ __forceinline__ M3 load_u(const double2 *U64, long V, int mu, long s)
{
    M3 r;
    for (int k = 0; k < 9; k++) {
        double2 v = U64[((long)mu * 9 + k) * V + s];
        r.m[k / 3][k % 3] = {v.x, v.y};
    }
    return r;
}
__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b)
{
    M3 c;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cpx<double> t = {0, 0};
            for (int k = 0; k < 3; k++) t = t + cmul(a.m[i][k], b.m[k][j]);
            c.m[i][j] = t;
        }
    return c;
}
__device__ __forceinline__ M3 dag(const M3 &a)
{
    M3 c;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c.m[i][j] = {a.m[j][i].re, -a.m[j][i].im};
    return c;
}

template <int BL>
__device__ long site_at(const GeomDev &g, const int *x, int mu, int dmu, int nu, int dnu)
{
    int c[4] = {x[0], x[1], x[2], x[3]};
    c[mu] = (c[mu] + dmu + g.L[mu]) % g.L[mu];
    c[nu] = (c[nu] + dnu + g.L[nu]) % g.L[nu];
    return internal_index<BL>(g, c[0], c[1], c[2], c[3]);
}

// Fhat_{mu nu}(x) = (Q - Q^dag) / 8, Q the sum of the four counter-clockwise leaves at x
template <int BL>
__device__ M3 fhat(const GeomDev &g, const double2 *U64, const int *x, int mu, int nu)
{
    long s = site_at<BL>(g, x, mu, 0, nu, 0);
    long pm = site_at<BL>(g, x, mu, 1, nu, 0), pn = site_at<BL>(g, x, mu, 0, nu, 1);
    long mm = site_at<BL>(g, x, mu, -1, nu, 0), mn = site_at<BL>(g, x, mu, 0, nu, -1);
    long mm_pn = site_at<BL>(g, x, mu, -1, nu, 1), mm_mn = site_at<BL>(g, x, mu, -1, nu, -1);
    long mn_pm = site_at<BL>(g, x, mu, 1, nu, -1);
    long V = g.V;
    M3 Q = mul(mul(load_u(U64, V, mu, s), load_u(U64, V, nu, pm)), mul(dag(load_u(U64, V, mu, pn)), dag(load_u(U64, V, nu, s))));
    M3 t = mul(mul(load_u(U64, V, nu, s), dag(load_u(U64, V, mu, mm_pn))), mul(dag(load_u(U64, V, nu, mm)), load_u(U64, V, mu, mm)));
    for (int i = 0; i < 9; i++) Q.m[i / 3][i % 3] = Q.m[i / 3][i % 3] + t.m[i / 3][i % 3];
    t = mul(mul(dag(load_u(U64, V, mu, mm)), dag(load_u(U64, V, nu, mm_mn))), mul(load_u(U64, V, mu, mm_mn), load_u(U64, V, nu, mn)));
    for (int i = 0; i < 9; i++) Q.m[i / 3][i % 3] = Q.m[i / 3][i % 3] + t.m[i / 3][i % 3];
    t = mul(mul(dag(load_u(U64, V, nu, mn)), load_u(U64, V, mu, mn)), mul(load_u(U64, V, nu, mn_pm), dag(load_u(U64, V, mu, s))));
    for (int i = 0; i < 9; i++) Q.m[i / 3][i % 3] = Q.m[i / 3][i % 3] + t.m[i / 3][i % 3];
    M3 F;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            F.m[i][j] = {(Q.m[i][j].re - Q.m[j][i].re) * 0.125, (Q.m[i][j].im + Q.m[j][i].im) * 0.125};
    return F;
}

// In the chiral basis sigma_{0k} = diag(s_k, -s_k) and sigma_{jk} = -eps_{jkl} diag(s_l, s_l), so
//   C_+ = csw (i/2) sum_l s_l (x) Y+_l,  Y+ = (F01 - F23, F02 + F13, F03 - F12)
//   C_- = csw (i/2) sum_l s_l (x) Y-_l,  Y- = (-F01 - F23, -F02 + F13, -F03 - F12)
// and with G_l = (i/2) csw Y_l (Hermitian):  C_ch = [[G3, G1 - i G2], [G1 + i G2, -G3]].
template <int BL>
__global__ void k_clover(GeomDev g, const double2 *__restrict__ U64, double csw, double2 *C64, float4 *C32)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    const int *o = g.blk_org + st.blk * 4;
    int x[4] = {o[0] + st.c[0], o[1] + st.c[1], o[2] + st.c[2], o[3] + st.c[3]};
    M3 F01 = fhat<BL>(g, U64, x, 0, 1), F02 = fhat<BL>(g, U64, x, 0, 2), F03 = fhat<BL>(g, U64, x, 0, 3);
    M3 F12 = fhat<BL>(g, U64, x, 1, 2), F13 = fhat<BL>(g, U64, x, 1, 3), F23 = fhat<BL>(g, U64, x, 2, 3);
    for (int ch = 0; ch < 2; ch++) {
        double sg = ch == 0 ? 1.0 : -1.0;
        M3 G[3];
        for (int i = 0; i < 9; i++) {
            int a = i / 3, b = i % 3;
            cpx<double> y1 = sg * F01.m[a][b] - F23.m[a][b];
            cpx<double> y2 = sg * F02.m[a][b] + F13.m[a][b];
            cpx<double> y3 = sg * F03.m[a][b] - F12.m[a][b];
            // G = (i/2) csw Y
            G[0].m[a][b] = timesI(0.5 * csw * y1);
            G[1].m[a][b] = timesI(0.5 * csw * y2);
            G[2].m[a][b] = timesI(0.5 * csw * y3);
        }
        cpx<double> H[6][6];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                H[a][b] = G[2].m[a][b];
                H[3 + a][3 + b] = -G[2].m[a][b];
                H[a][3 + b] = G[0].m[a][b] - timesI(G[1].m[a][b]);
                H[3 + a][b] = G[0].m[a][b] + timesI(G[1].m[a][b]);
            }
        double r[36];
        for (int i = 0; i < 6; i++) r[i] = H[i][i].re;
        for (int i = 0; i < 6; i++)
            for (int j = i + 1; j < 6; j++) {
                int k = 6 + 2 * herm_off(i, j);
                r[k] = H[i][j].re;
                r[k + 1] = H[i][j].im;
            }
        for (int k = 0; k < 18; k++) C64[((long)ch * 18 + k) * g.V + s] = make_double2(r[2 * k], r[2 * k + 1]);
        for (int k = 0; k < 9; k++)
            C32[((long)ch * 9 + k) * g.V + s] =
                make_float4((float)r[4 * k], (float)r[4 * k + 1], (float)r[4 * k + 2], (float)r[4 * k + 3]);
    }
}

template <int BL>
void clover_launch(ddrw_ctx *ctx)
{
    GeomDev g = geom_dev(ctx);
    dim3 grid((unsigned)((ctx->V + 63) / 64));
    ++ctx->launches;
    k_clover<BL><<<grid, 64, 0, ctx->stream>>>(g, ctx->U64, ctx->csw, ctx->C64, ctx->C32);
}

}  // namespace ddrw
