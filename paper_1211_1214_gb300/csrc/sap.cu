// sap.cu -- the Schwarz-preconditioned flexible GCR solver of the full-lattice system D(m) x = b.
//
// The outer solve of the estimate (delta = A(m2)^-1 r, one Dirac inversion per noise vector, Sec. 2)
// reuses the domain decomposition the paper builds on (Sec. 1): the lattice is cut into small
// hypercubic Schwarz blocks of side 4, coloured black/white like a checkerboard, and the
// preconditioner is the multiplicative Schwarz alternating procedure (SAP):
//
//   psi = 0, rho = eta;  ncy cycles of { for colour c = black, white:
//        chi = approximate D_blk^-1 rho on every block of colour c (Dirichlet boundary),
//        psi += chi,  rho -= D chi }
//
// which approximates D^-1 eta.  Each block solve is nmr minimal-residual steps on the block's
// even-odd reduced operator Ahat = A_ee - 1/4 H_eo A_oo^-1 H_oe (hops inside the block only),
// started from zero.  One CTA owns one Schwarz block for NR right-hand sides and keeps everything
// the steps touch in shared memory: the block's links and clover terms (staged once), the
// residual on the even sites, the odd-site intermediate and A_oo^-1 rho_o.  After the steps
// rho is the block's minimal residual on the even sites and zero on the odd sites (exactly, by
// construction of the odd-site solution), and the change rho -= D chi on the neighbouring blocks
// of the other colour is applied by the next sweep when it loads its residual (the hops that
// cross the Schwarz-block faces, read from the chi of the previous sweep).
//
// SAP with MR steps is not a fixed linear operator, so the Krylov method is flexible GCR:
//   z_k = SAP(r),  w_k = D z_k,  w_k and z_k orthogonalised against w_0..w_{k-1} (classical
//   Gram-Schmidt, FP64 sums), alpha_k = <w_k, r>/|w_k|^2,  r -= alpha_k w_k;  x += sum alpha_k z_k
//   at every restart (after nkv directions), where r is recomputed as b - D x.
// All right-hand sides run in lockstep with their own scalars (device resident); one that has
// converged stops updating.  Fields are FP32 (the inner solve of the FP64 defect correction).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "blas.cuh"
#include "ctx.h"
#include "stencil.cuh"

namespace ddrw {

namespace {

constexpr int SB = 4;          // side of a Schwarz block
constexpr int SBV = 256;       // sites per Schwarz block
constexpr int SBH = 128;       // sites of one parity per Schwarz block
constexpr int NKV_MAX = 16;    // search directions kept between restarts
constexpr int GNT = 256;       // threads per CTA of the GCR vector kernels

// in-block coordinates of half index h (parity p) of a Schwarz block (side 4, origin even)
__device__ __forceinline__ void sb_coords(int h, int p, int (&a)[4])
{
    int row = h >> 1;
    const int izh = h & 1;
    a[2] = row & 3;
    row >>= 2;
    a[1] = row & 3;
    a[0] = row >> 2;
    a[3] = 2 * izh + ((a[0] + a[1] + a[2] + p) & 1);
}

// half index of the in-block neighbour of a in direction mu (dir +1 / -1), or -1 outside the block
__device__ __forceinline__ int sb_nb(const int (&a)[4], int mu, int dir)
{
    int b[4] = {a[0], a[1], a[2], a[3]};
    b[mu] += dir;
    if (b[mu] < 0 || b[mu] >= SB) return -1;
    return (((b[0] * SB + b[1]) * SB + b[2]) * SB + b[3]) >> 1;
}

// shared-memory spinor of 6 float4 planes, plane k of half site h at base[k * SBH + h]
__device__ __forceinline__ void ld_sp(const float4 *base, int h, Spinor<float> &p)
{
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 v = base[k * SBH + h];
        p.v[(2 * k) / 3][(2 * k) % 3] = {v.x, v.y};
        p.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = {v.z, v.w};
    }
}
__device__ __forceinline__ void st_sp(float4 *base, int h, const Spinor<float> &p)
{
#pragma unroll
    for (int k = 0; k < 6; k++) {
        cpx<float> a = p.v[(2 * k) / 3][(2 * k) % 3], b = p.v[(2 * k + 1) / 3][(2 * k + 1) % 3];
        base[k * SBH + h] = make_float4(a.re, a.im, b.re, b.im);
    }
}

// two-row FP32 link of direction mu at block site q from shared memory (planes [mu][3][SBV])
__device__ __forceinline__ void ld_link(const float4 *sU, int mu, int q, Link<float> &L)
{
    const float4 a0 = sU[(mu * 3 + 0) * SBV + q], a1 = sU[(mu * 3 + 1) * SBV + q], a2 = sU[(mu * 3 + 2) * SBV + q];
    L.m[0][0] = {a0.x, a0.y};
    L.m[0][1] = {a0.z, a0.w};
    L.m[0][2] = {a1.x, a1.y};
    L.m[1][0] = {a1.z, a1.w};
    L.m[1][1] = {a2.x, a2.y};
    L.m[1][2] = {a2.z, a2.w};
    PrecS::reconstruct_row2(L);
}

// v <- (diag + H) v with the two Hermitian 6x6 blocks of block site q (planes [18][SBV])
__device__ __forceinline__ void clover_sm(const float4 *sC, int q, float diag, Spinor<float> &v)
{
#pragma unroll
    for (int ch = 0; ch < 2; ch++) {
        float c[36];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            float4 e = sC[(ch * 9 + k) * SBV + q];
            c[4 * k] = e.x;
            c[4 * k + 1] = e.y;
            c[4 * k + 2] = e.z;
            c[4 * k + 3] = e.w;
        }
        cpx<float> in6[6], out6[6];
#pragma unroll
        for (int i = 0; i < 6; i++) in6[i] = v.v[2 * ch + i / 3][i % 3];
        herm6_mul<float>(c, diag, in6, out6);
#pragma unroll
        for (int i = 0; i < 6; i++) v.v[2 * ch + i / 3][i % 3] = out6[i];
    }
}

// acc += sum over the in-block hops of site (h, p): (1 - g_mu) U_mu(x) in(x + mu) + (1 + g_mu)
// U_mu(x - mu)^dag in(x - mu), in = the other parity's vector in shared memory
template <int MU>
__device__ __forceinline__ void hop_in_dir(const float4 *sU, const float4 *in, const int (&a)[4], int h, int p,
                                           Spinor<float> &acc)
{
    const int nf = sb_nb(a, MU, +1);
    if (nf >= 0) {
        Spinor<float> s;
        ld_sp(in, nf, s);
        Half<float> hh, w;
        project<MU, -1>(s, hh);
        Link<float> L;
        ld_link(sU, MU, p * SBH + h, L);
        link_mul(L, hh, w);
        reconstruct_add<MU, -1>(acc, w);
    }
    const int nb = sb_nb(a, MU, -1);
    if (nb >= 0) {
        Spinor<float> s;
        ld_sp(in, nb, s);
        Half<float> hh, w;
        project<MU, +1>(s, hh);
        Link<float> L;
        ld_link(sU, MU, (1 - p) * SBH + nb, L);
        link_dag_mul(L, hh, w);
        reconstruct_add<MU, +1>(acc, w);
    }
}

__device__ __forceinline__ void hop_in(const float4 *sU, const float4 *in, int h, int p, Spinor<float> &acc)
{
    int a[4];
    sb_coords(h, p, a);
    hop_in_dir<0>(sU, in, a, h, p, acc);
    hop_in_dir<1>(sU, in, a, h, p, acc);
    hop_in_dir<2>(sU, in, a, h, p, acc);
    hop_in_dir<3>(sU, in, a, h, p, acc);
}

// acc += the hops of global site s that leave its Schwarz block (a: in-block coordinates), read
// from the field f (global, the other colour's sites)
template <int BL, int MU>
__device__ __forceinline__ void hop_out_dir(const GeomDev &g, const Site<BL> &st, int s, const int (&a)[4],
                                            const float4 *f, const float4 *__restrict__ U, Spinor<float> &acc)
{
    bool cross;
    int ph;
    if (a[MU] == SB - 1) {
        const int sf = neighbour<BL>(st, MU, +1, g, &cross, &ph);
        Spinor<float> p;
        PrecS::load_spinor_rw(f, (int)g.V, sf, p);
        Half<float> h, w;
        project<MU, -1>(p, h);
        Link<float> L;
        PrecS::load_link(U, (int)g.V, MU, s, L);
        link_mul(L, h, w);
        if (ph < 0)
#pragma unroll
            for (int x = 0; x < 2; x++)
#pragma unroll
                for (int c = 0; c < 3; c++) w.v[x][c] = -w.v[x][c];
        reconstruct_add<MU, -1>(acc, w);
    }
    if (a[MU] == 0) {
        const int sb = neighbour<BL>(st, MU, -1, g, &cross, &ph);
        Spinor<float> p;
        PrecS::load_spinor_rw(f, (int)g.V, sb, p);
        Half<float> h, w;
        project<MU, +1>(p, h);
        Link<float> L;
        PrecS::load_link(U, (int)g.V, MU, sb, L);
        link_dag_mul(L, h, w);
        if (ph < 0)
#pragma unroll
            for (int x = 0; x < 2; x++)
#pragma unroll
                for (int c = 0; c < 3; c++) w.v[x][c] = -w.v[x][c];
        reconstruct_add<MU, +1>(acc, w);
    }
}

template <int BL>
__device__ __forceinline__ void hop_out(const GeomDev &g, int s, const int (&a)[4], const float4 *f,
                                     const float4 *__restrict__ U, Spinor<float> &acc)
{
    Site<BL> st;
    decode_site<BL>(s, g, st);
    hop_out_dir<BL, 0>(g, st, s, a, f, U, acc);
    hop_out_dir<BL, 1>(g, st, s, a, f, U, acc);
    hop_out_dir<BL, 2>(g, st, s, a, f, U, acc);
    hop_out_dir<BL, 3>(g, st, s, a, f, U, acc);
}

}  // namespace

struct SapArgs {
    GeomDev g;
    int colour;
    int nsb[4];            // Schwarz blocks per direction (each even, >= 2)
    const float4 *rho_in;  // residual read on this colour's sites
    float4 *rho_out;       // residual written on this colour's sites (may equal rho_in)
    const float4 *chi_prev;  // the other colour's last increment (null: none yet)
    float4 *chi;           // this sweep's increment (written on this colour's sites)
    float4 *psi;           // the preconditioned vector
    int psi_init;          // 1: psi = chi on this colour's sites, 0: psi += chi
    long rs;               // elements between right-hand sides of a field
    int rpm;               // right-hand sides per mass slot
    float mass4[MAXM];
    const float4 *Ainv[MAXM];
    const float4 *U;   // FP32 two-row links [4][3][V]
    const float4 *Cl;  // FP32 clover [2][9][V]
    int nmr;
};

namespace {

// dynamic shared memory of one CTA (float4 elements)
__host__ __device__ constexpr int sap_smem_f4(int nr) { return 12 * SBV + 18 * SBV + nr * 3 * 6 * SBH + 2 * nr * 4; }

// One sweep of SAP over the Schwarz blocks of one colour: CTA (block j of the colour, group of
// NR right-hand sides), 128 NR threads; thread (r, h) owns even site h and odd site h of
// right-hand side r of the group.
template <int BL, int NR>
__global__ void __launch_bounds__(128 * NR, 1) k_sap_sweep(SapArgs a)
{
    extern __shared__ float4 smem[];
    float4 *sU = smem;                   // [4][3][SBV] links U_mu(x) at the block's sites
    float4 *sC = sU + 12 * SBV;          // [18][SBV]: C on even sites, A_oo^-1 on odd sites
    float4 *sR = sC + 18 * SBV;          // [NR][6][SBH] even: residual, then the solution
    float4 *sT = sR + NR * 6 * SBH;      // [NR][6][SBH] odd: A_oo^-1 H_oe r
    float4 *sY = sT + NR * 6 * SBH;      // [NR][6][SBH] odd: A_oo^-1 rho_o
    float *sRed = (float *)(sY + NR * 6 * SBH);  // [NR][4 warps][2]

    const GeomDev &g = a.g;
    const int V = (int)g.V;
    // Schwarz block coordinates: the blocks of one colour alternate along z within each z-row
    const int nrow = a.nsb[3] / 2;
    int row = blockIdx.x / nrow;
    const int iz = blockIdx.x - row * nrow;
    const int by = row % a.nsb[2];
    row /= a.nsb[2];
    const int bx = row % a.nsb[1];
    const int bt = row / a.nsb[1];
    const int bz = 2 * iz + ((bt + bx + by + a.colour) & 1);
    const int org[4] = {bt * SB, bx * SB, by * SB, bz * SB};

    const int tid = threadIdx.x;
    const int r = tid >> 7, h = tid & 127;
    const int rhs = blockIdx.y * NR + r;
    const int slot = (blockIdx.y * NR) / a.rpm;
    const long ro = (long)rhs * a.rs;

    // stage links and the diagonal terms of the block (every thread helps)
    const float4 *Ainv = a.Ainv[slot];
    for (int q = tid; q < SBV; q += 128 * NR) {
        int c[4];
        sb_coords(q & 127, q >> 7, c);
        const int s = (int)internal_index<BL>(g, org[0] + c[0], org[1] + c[1], org[2] + c[2], org[3] + c[3]);
#pragma unroll
        for (int k = 0; k < 12; k++) sU[k * SBV + q] = __ldg(a.U + (long)k * V + s);
        const float4 *cl = (q < SBH) ? a.Cl : Ainv;
#pragma unroll
        for (int k = 0; k < 18; k++) sC[k * SBV + q] = __ldg(cl + (long)k * V + s);
    }

    // own sites
    int ae[4], ao[4];
    sb_coords(h, 0, ae);
    sb_coords(h, 1, ao);
    const int se = (int)internal_index<BL>(g, org[0] + ae[0], org[1] + ae[1], org[2] + ae[2], org[3] + ae[3]);
    const int so = (int)internal_index<BL>(g, org[0] + ao[0], org[1] + ao[1], org[2] + ao[2], org[3] + ao[3]);
    const float4 *rin = a.rho_in + ro;
    Spinor<float> rho_e, rho_o;
    PrecS::load_spinor_rw(rin, V, se, rho_e);
    PrecS::load_spinor_rw(rin, V, so, rho_o);
    if (a.chi_prev) {
        // rho -= D chi_prev: only the hops into the other colour's blocks contribute (-1/2 H)
        Spinor<float> acc;
        zero(acc);
        hop_out<BL>(g, se, ae, a.chi_prev + ro, a.U, acc);
        axpy(rho_e, 0.5f, acc);
        zero(acc);
        hop_out<BL>(g, so, ao, a.chi_prev + ro, a.U, acc);
        axpy(rho_o, 0.5f, acc);
    }
    float4 *myR = sR + r * 6 * SBH, *myT = sT + r * 6 * SBH, *myY = sY + r * 6 * SBH;
    __syncthreads();  // staged terms visible
    // y_o = A_oo^-1 rho_o
    clover_sm(sC, SBH + h, 0.0f, rho_o);
    st_sp(myY, h, rho_o);
    __syncthreads();
    // rhat_e = rho_e + 1/2 H_eo y_o  (the even-odd reduced right-hand side)
    {
        Spinor<float> acc;
        zero(acc);
        hop_in(sU, myY, h, 0, acc);
        axpy(rho_e, 0.5f, acc);
    }
    st_sp(myR, h, rho_e);
    const float mass4 = a.mass4[slot];
    Spinor<float> xe;
    zero(xe);
    const int lane = tid & 31, wq = (tid >> 5) & 3;
    for (int it = 0; it < a.nmr; it++) {
        __syncthreads();  // r_e complete
        // t_o = A_oo^-1 H_oe r_e
        {
            Spinor<float> acc;
            zero(acc);
            hop_in(sU, myR, h, 1, acc);
            clover_sm(sC, SBH + h, 0.0f, acc);
            st_sp(myT, h, acc);
        }
        __syncthreads();
        // q_e = A_ee r_e - 1/4 H_eo t_o
        Spinor<float> re, q;
        ld_sp(myR, h, re);
        q = re;
        clover_sm(sC, h, mass4, q);
        {
            Spinor<float> acc;
            zero(acc);
            hop_in(sU, myT, h, 0, acc);
            axpy(q, -0.25f, acc);
        }
        // alpha = <q, r> / <q, q> over the block (per right-hand side)
        float qr_re = 0.f, qr_im = 0.f, qq = 0.f;
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const cpx<float> z = cmulc(q.v[sp][c], re.v[sp][c]);
                qr_re += z.re;
                qr_im += z.im;
                qq += q.v[sp][c].re * q.v[sp][c].re + q.v[sp][c].im * q.v[sp][c].im;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            qr_re += __shfl_xor_sync(0xffffffffu, qr_re, o);
            qr_im += __shfl_xor_sync(0xffffffffu, qr_im, o);
            qq += __shfl_xor_sync(0xffffffffu, qq, o);
        }
        if (lane == 0) {
            sRed[(r * 4 + wq) * 3 + 0] = qr_re;
            sRed[(r * 4 + wq) * 3 + 1] = qr_im;
            sRed[(r * 4 + wq) * 3 + 2] = qq;
        }
        __syncthreads();
        float tre = 0.f, tim = 0.f, tqq = 0.f;
#pragma unroll
        for (int w = 0; w < 4; w++) {
            tre += sRed[(r * 4 + w) * 3 + 0];
            tim += sRed[(r * 4 + w) * 3 + 1];
            tqq += sRed[(r * 4 + w) * 3 + 2];
        }
        const cpx<float> al = tqq > 0.f ? cpx<float>{tre / tqq, tim / tqq} : cpx<float>{0.f, 0.f};
        // x_e += alpha r_e ; r_e -= alpha q_e
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                cmac(xe.v[sp][c], al, re.v[sp][c]);
                cmsub(re.v[sp][c], al, q.v[sp][c]);
            }
        __syncthreads();  // every thread has read sRed and its neighbours' r_e
        st_sp(myR, h, re);
    }
    // the block's new residual: the minimal residual on the even sites, zero on the odd sites
    {
        Spinor<float> re;
        ld_sp(myR, h, re);
        PrecS::store_spinor(a.rho_out + ro, V, se, re);
        Spinor<float> z;
        zero(z);
        PrecS::store_spinor(a.rho_out + ro, V, so, z);
    }
    __syncthreads();  // every thread has read its r_e
    st_sp(myR, h, xe);
    __syncthreads();
    // chi_o = y_o + 1/2 A_oo^-1 H_oe chi_e
    Spinor<float> xo;
    {
        Spinor<float> acc;
        zero(acc);
        hop_in(sU, myR, h, 1, acc);
        clover_sm(sC, SBH + h, 0.0f, acc);
        ld_sp(myY, h, xo);
        axpy(xo, 0.5f, acc);
    }
    PrecS::store_spinor(a.chi + ro, V, se, xe);
    PrecS::store_spinor(a.chi + ro, V, so, xo);
    float4 *ps = a.psi + ro;
    if (!a.psi_init) {
        Spinor<float> pv;
        PrecS::load_spinor_rw(ps, V, se, pv);
        axpy(xe, 1.0f, pv);
        PrecS::load_spinor_rw(ps, V, so, pv);
        axpy(xo, 1.0f, pv);
    }
    PrecS::store_spinor(ps, V, se, xe);
    PrecS::store_spinor(ps, V, so, xo);
}

// ---- GCR vector kernels (FP32 fields of 6 float4 planes, FP64 sums)

struct GcrScal {
    double2 c[NKV_MAX];  // projections of the new direction on the kept ones
    double nn[NKV_MAX];  // |w_j|^2
    double2 a[NKV_MAX];  // step lengths alpha_j
    double rr, thresh;
    int active, iters, maxiter, pad;
};

struct GArgs {
    long V, rs, fs;  // sites, elements between right-hand sides, elements between basis fields
};

__device__ __forceinline__ float4 f4_cmac(float4 acc, float2 c, float4 v)  // acc + c v (two complexes)
{
    acc.x = fmaf(c.x, v.x, fmaf(-c.y, v.y, acc.x));
    acc.y = fmaf(c.x, v.y, fmaf(c.y, v.x, acc.y));
    acc.z = fmaf(c.x, v.z, fmaf(-c.y, v.w, acc.z));
    acc.w = fmaf(c.x, v.w, fmaf(c.y, v.z, acc.w));
    return acc;
}

// r = b, rr = |b|^2, active when rr > thresh
__global__ void __launch_bounds__(GNT) k_gcr_init(GArgs ga, const float4 *b, float4 *r, GcrScal *sc, double *part,
                                                  unsigned *ticket)
{
    const long rb = (long)blockIdx.y * ga.rs;
    float acc = 0.f;
    for (long i = (long)blockIdx.x * GNT + threadIdx.x; i < 6 * ga.V; i += (long)gridDim.x * GNT) {
        const float4 v = b[rb + i];
        r[rb + i] = v;
        acc += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
    }
    double t[1] = {(double)acc};
    if (grid_sum<1, GNT>(t, part, ticket)) {
        GcrScal &s = sc[blockIdx.y];
        s.rr = t[0];
        s.iters = 0;
        s.active = (t[0] > s.thresh && s.maxiter > 0) ? 1 : 0;
    }
}

// c_j = <w_j, w_k> / |w_j|^2 for j < k
template <int K>
__global__ void __launch_bounds__(GNT) k_gcr_dots(GArgs ga, const float4 *W, int k, GcrScal *sc, double *part,
                                                  unsigned *ticket)
{
    if (!sc[blockIdx.y].active) return;
    const long rb = (long)blockIdx.y * ga.rs;
    const float4 *wk = W + (long)k * ga.fs + rb;
    float acc[2 * K];
#pragma unroll
    for (int j = 0; j < 2 * K; j++) acc[j] = 0.f;
    for (long i = (long)blockIdx.x * GNT + threadIdx.x; i < 6 * ga.V; i += (long)gridDim.x * GNT) {
        const float4 v = wk[i];
#pragma unroll
        for (int j = 0; j < K; j++) {
            if (j < k) {
                const float4 u = W[(long)j * ga.fs + rb + i];
                acc[2 * j] += u.x * v.x + u.y * v.y + u.z * v.z + u.w * v.w;
                acc[2 * j + 1] += u.x * v.y - u.y * v.x + u.z * v.w - u.w * v.z;
            }
        }
    }
    double t[2 * K];
#pragma unroll
    for (int j = 0; j < 2 * K; j++) t[j] = acc[j];
    if (grid_sum<2 * K, GNT>(t, part, ticket)) {
        GcrScal &s = sc[blockIdx.y];
        for (int j = 0; j < k; j++) {
            const double n = s.nn[j];
            s.c[j] = n > 0 ? make_double2(t[2 * j] / n, t[2 * j + 1] / n) : make_double2(0.0, 0.0);
        }
    }
}

// w_k -= sum_j c_j w_j, z_k -= sum_j c_j z_j; nn_k = |w_k|^2, alpha_k = <w_k, r> / nn_k
template <int K>
__global__ void __launch_bounds__(GNT) k_gcr_ortho(GArgs ga, float4 *W, float4 *Z, const float4 *r, int k,
                                                   GcrScal *sc, double *part, unsigned *ticket)
{
    GcrScal &s0 = sc[blockIdx.y];
    if (!s0.active) {
        if (blockIdx.x == 0 && threadIdx.x == 0) s0.a[k] = make_double2(0.0, 0.0);
        return;
    }
    const long rb = (long)blockIdx.y * ga.rs;
    float2 cj[K];
#pragma unroll
    for (int j = 0; j < K; j++) cj[j] = j < k ? make_float2(-(float)s0.c[j].x, -(float)s0.c[j].y) : make_float2(0.f, 0.f);
    float4 *wk = W + (long)k * ga.fs + rb, *zk = Z + (long)k * ga.fs + rb;
    float nn = 0.f, dre = 0.f, dim = 0.f;
    for (long i = (long)blockIdx.x * GNT + threadIdx.x; i < 6 * ga.V; i += (long)gridDim.x * GNT) {
        float4 w = wk[i], z = zk[i];
#pragma unroll
        for (int j = 0; j < K; j++) {
            if (j < k) {
                w = f4_cmac(w, cj[j], W[(long)j * ga.fs + rb + i]);
                z = f4_cmac(z, cj[j], Z[(long)j * ga.fs + rb + i]);
            }
        }
        wk[i] = w;
        zk[i] = z;
        const float4 rv = r[rb + i];
        nn += w.x * w.x + w.y * w.y + w.z * w.z + w.w * w.w;
        dre += w.x * rv.x + w.y * rv.y + w.z * rv.z + w.w * rv.w;
        dim += w.x * rv.y - w.y * rv.x + w.z * rv.w - w.w * rv.z;
    }
    double t[3] = {(double)nn, (double)dre, (double)dim};
    if (grid_sum<3, GNT>(t, part, ticket)) {
        GcrScal &s = sc[blockIdx.y];
        s.nn[k] = t[0];
        s.a[k] = t[0] > 0 ? make_double2(t[1] / t[0], t[2] / t[0]) : make_double2(0.0, 0.0);
    }
}

// r -= alpha_k w_k ; rr = |r|^2 ; iteration count and the continue decision
__global__ void __launch_bounds__(GNT) k_gcr_r(GArgs ga, const float4 *W, float4 *r, int k, GcrScal *sc,
                                               double *part, unsigned *ticket)
{
    const GcrScal &s0 = sc[blockIdx.y];
    if (!s0.active) return;
    const long rb = (long)blockIdx.y * ga.rs;
    const float2 al = make_float2(-(float)s0.a[k].x, -(float)s0.a[k].y);
    const float4 *wk = W + (long)k * ga.fs + rb;
    float acc = 0.f;
    for (long i = (long)blockIdx.x * GNT + threadIdx.x; i < 6 * ga.V; i += (long)gridDim.x * GNT) {
        float4 v = f4_cmac(r[rb + i], al, wk[i]);
        r[rb + i] = v;
        acc += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
    }
    double t[1] = {(double)acc};
    if (grid_sum<1, GNT>(t, part, ticket)) {
        GcrScal &s = sc[blockIdx.y];
        s.rr = t[0];
        s.iters += 1;
        if (!(t[0] == t[0]) || t[0] <= s.thresh || s.iters >= s.maxiter) s.active = 0;
    }
}

// x += sum_{j < nk} alpha_j z_j (the steps of one restart cycle)
template <int K>
__global__ void __launch_bounds__(GNT) k_gcr_x(GArgs ga, const float4 *Z, float4 *x, int nk, const GcrScal *sc)
{
    const GcrScal &s = sc[blockIdx.y];
    const long rb = (long)blockIdx.y * ga.rs;
    float2 aj[K];
#pragma unroll
    for (int j = 0; j < K; j++) aj[j] = j < nk ? make_float2((float)s.a[j].x, (float)s.a[j].y) : make_float2(0.f, 0.f);
    for (long i = (long)blockIdx.x * GNT + threadIdx.x; i < 6 * ga.V; i += (long)gridDim.x * GNT) {
        float4 v = x[rb + i];
#pragma unroll
        for (int j = 0; j < K; j++)
            if (j < nk) v = f4_cmac(v, aj[j], Z[(long)j * ga.fs + rb + i]);
        x[rb + i] = v;
    }
}

// after a restart: r = b + res (res = -D x), rr = |r|^2, active when above the threshold
__global__ void __launch_bounds__(GNT) k_gcr_restart(GArgs ga, const float4 *b, const float4 *res, float4 *r,
                                                     GcrScal *sc, double *part, unsigned *ticket)
{
    if (!sc[blockIdx.y].active) return;
    const long rb = (long)blockIdx.y * ga.rs;
    float acc = 0.f;
    for (long i = (long)blockIdx.x * GNT + threadIdx.x; i < 6 * ga.V; i += (long)gridDim.x * GNT) {
        const float4 u = b[rb + i], d = res[rb + i];
        const float4 v = make_float4(u.x + d.x, u.y + d.y, u.z + d.z, u.w + d.w);
        r[rb + i] = v;
        acc += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
    }
    double t[1] = {(double)acc};
    if (grid_sum<1, GNT>(t, part, ticket)) {
        GcrScal &s = sc[blockIdx.y];
        s.rr = t[0];
        if (!(t[0] == t[0]) || t[0] <= s.thresh || s.iters >= s.maxiter) s.active = 0;
    }
}

unsigned ggrid(long n)
{
    long g = (n + GNT - 1) / GNT;
    return (unsigned)(g < 1 ? 1 : (g > 608 ? 608 : g));
}

template <int BL, int NR> void launch_sweep(ddrw_ctx *ctx, const SapArgs &a, int nblk_colour, int nrhs)
{
    const int smem = sap_smem_f4(NR) * 16;
    cudaFuncSetAttribute(k_sap_sweep<BL, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    ++ctx->launches;
    k_sap_sweep<BL, NR><<<dim3((unsigned)nblk_colour, (unsigned)(nrhs / NR)), 128 * NR, smem, ctx->stream>>>(a);
}

template <int BL> void launch_sweep_bl(ddrw_ctx *ctx, const SapArgs &a, int nb, int nrhs, int nr)
{
    if (nr == 2) launch_sweep<BL, 2>(ctx, a, nb, nrhs);
    else launch_sweep<BL, 1>(ctx, a, nb, nrhs);
}

}  // namespace

bool sap_supported(const ddrw_ctx *ctx)
{
    for (int mu = 0; mu < 4; mu++)
        if (ctx->dims[mu] % (2 * SB)) return false;
    return ctx->l == 2 || ctx->l == 4 || ctx->l == 6 || ctx->l == 8;
}

size_t sap_bytes_per_site_rhs(const ddrw_ctx *ctx)
{
    // FP32 fields: z and w per kept direction, r, x, b copy, rho, chi, residual
    return (size_t)96 * (2 * ctx->sap_nkv + 6);
}

// psi = SAP(eta) for nrhs FP32 fields (rho, chi: work fields)
static void sap_apply(ddrw_ctx *ctx, const MassSet &ms, const float4 *eta, float4 *psi, float4 *rho, float4 *chi,
                      int nrhs, int nr)
{
    SapArgs a;
    a.g = geom_dev(ctx);
    for (int mu = 0; mu < 4; mu++) a.nsb[mu] = ctx->dims[mu] / SB;
    a.rs = 6 * ctx->V;
    a.rpm = (nrhs + std::max(ms.n, 1) - 1) / std::max(ms.n, 1);
    for (int k = 0; k < MAXM; k++) {
        const int kk = k < ms.n ? k : 0;
        a.mass4[k] = (float)(4.0 + ms.m[kk]);
        a.Ainv[k] = ms.inv[kk]->A32;
    }
    a.U = ctx->U32;
    a.Cl = ctx->C32;
    a.nmr = ctx->sap_nmr;
    const int nb = (int)(ctx->V / SBV / 2);
    ProfScope ps(ctx, PROF_SAP, 0.0, (double)ctx->V * nrhs * ctx->sap_ncy * (ctx->sap_nmr + 1));
    for (int cy = 0; cy < ctx->sap_ncy; cy++)
        for (int c = 0; c < 2; c++) {
            a.colour = c;
            a.rho_in = cy == 0 ? eta : rho;
            a.rho_out = rho;
            a.chi_prev = (cy == 0 && c == 0) ? nullptr : chi;
            a.chi = chi;
            a.psi = psi;
            a.psi_init = cy == 0 ? 1 : 0;
            switch (ctx->l) {
            case 2: launch_sweep_bl<2>(ctx, a, nb, nrhs, nr); break;
            case 4: launch_sweep_bl<4>(ctx, a, nb, nrhs, nr); break;
            case 6: launch_sweep_bl<6>(ctx, a, nb, nrhs, nr); break;
            default: launch_sweep_bl<8>(ctx, a, nb, nrhs, nr); break;
            }
        }
}

// out = D(ms) in on the whole lattice (FP32; alpha = 1: D, alpha = -1: -D)
static void apply_full32(ddrw_ctx *ctx, const MassSet &ms, const float4 *in, float4 *out, int nrhs, double sign)
{
    DslashCall c;
    c.in = in;
    c.x = in;
    c.out = out;
    c.rstride = 6 * ctx->V;
    c.nrhs = nrhs;
    c.nmass = ms.n;
    for (int k = 0; k < ms.n; k++) {
        c.masses[k] = ms.m[k];
        c.Ainv[k] = ms.inv[k]->A32;
    }
    c.alpha = sign;
    c.beta = -0.5 * sign;
    c.diag = 1;
    c.par0 = 0;
    c.npar = 2;
    c.blk0 = 0;
    c.nblk = ctx->nblk;
    dslash32(ctx, c);
}

template <int K>
static void gcr_dots_k(ddrw_ctx *ctx, const GArgs &ga, const float4 *W, int k, GcrScal *sc, double *part,
                       unsigned *tk, int nrhs)
{
    ++ctx->launches;
    k_gcr_dots<K><<<dim3(ggrid(6 * ga.V), nrhs), GNT, 0, ctx->stream>>>(ga, W, k, sc, part, tk);
}

ddrw_status sap_gcr(ddrw_ctx *ctx, const MassSet &ms, const float4 *b, float4 *x, int nrhs,
                    const std::vector<double> &thresh, int maxiter, int *iters)
{
    const long V = ctx->V, rs = 6 * V, fs = rs * nrhs;
    const size_t fb = sizeof(float4) * (size_t)fs;
    const int nkv = std::max(1, std::min(ctx->sap_nkv, NKV_MAX));
    const int rpm = (nrhs + std::max(ms.n, 1) - 1) / std::max(ms.n, 1);
    const int nr = (rpm % 2 == 0 && nrhs % 2 == 0) ? 2 : 1;
    ddrw_status st;
    float4 *W, *Z, *r, *rho, *chi, *res;
    if ((st = workspace(ctx, "gcr_W", fb * nkv, (void **)&W))) return st;
    if ((st = workspace(ctx, "gcr_Z", fb * nkv, (void **)&Z))) return st;
    if ((st = workspace(ctx, "gcr_r", fb, (void **)&r))) return st;
    if ((st = workspace(ctx, "gcr_rho", fb, (void **)&rho))) return st;
    if ((st = workspace(ctx, "gcr_chi", fb, (void **)&chi))) return st;
    if ((st = workspace(ctx, "gcr_res", fb, (void **)&res))) return st;
    GcrScal *sc;
    double *part;
    unsigned *tk;
    if ((st = workspace(ctx, "gcr_scal", sizeof(GcrScal) * nrhs, (void **)&sc))) return st;
    if ((st = workspace(ctx, "gcr_part", sizeof(double) * 2 * NKV_MAX * 608 * (size_t)nrhs, (void **)&part))) return st;
    {
        double *p4;
        if ((st = reduce_ws(ctx, nrhs, &p4, &tk))) return st;
    }
    std::vector<GcrScal> h(nrhs);
    for (int k = 0; k < nrhs; k++) {
        h[k] = GcrScal{};
        h[k].thresh = thresh[k];
        h[k].maxiter = maxiter;
    }
    DDRW_CUDA_CHECK(cudaMemcpyAsync(sc, h.data(), sizeof(GcrScal) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
    DDRW_CUDA_CHECK(cudaMemsetAsync(x, 0, fb, ctx->stream));
    const GArgs ga{V, rs, fs};
    const dim3 gg(ggrid(6 * V), nrhs);
    ++ctx->launches;
    k_gcr_init<<<gg, GNT, 0, ctx->stream>>>(ga, b, r, sc, part, tk);

    // host copy of the scalars, read once per iteration for the continue decision
    GcrScal *hs = (GcrScal *)ctx->h_pinned;
    if ((size_t)nrhs * sizeof(GcrScal) > ctx->h_pinned_bytes) return set_error(ctx, DDRW_EINVAL, "too many right-hand sides");
    auto any_active = [&](bool *out) -> ddrw_status {
        DDRW_CUDA_CHECK(cudaMemcpyAsync(hs, sc, sizeof(GcrScal) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
        DDRW_SYNC(ctx);
        bool a = false;
        for (int k = 0; k < nrhs; k++) a |= hs[k].active != 0;
        *out = a;
        return DDRW_OK;
    };
    bool act;
    if ((st = any_active(&act))) return st;
    int it = 0;
    while (act && it < maxiter) {
        int k = 0;
        for (; k < nkv && act && it < maxiter; k++, it++) {
            float4 *zk = Z + (long)k * fs, *wk = W + (long)k * fs;
            sap_apply(ctx, ms, r, zk, rho, chi, nrhs, nr);
            apply_full32(ctx, ms, zk, wk, nrhs, 1.0);
            {
                ProfScope ps(ctx, PROF_BLAS, 0.0);
                if (k > 0) {
                    if (k <= 4) gcr_dots_k<4>(ctx, ga, W, k, sc, part, tk, nrhs);
                    else if (k <= 8) gcr_dots_k<8>(ctx, ga, W, k, sc, part, tk, nrhs);
                    else gcr_dots_k<NKV_MAX>(ctx, ga, W, k, sc, part, tk, nrhs);
                }
                ++ctx->launches;
                if (k <= 4) k_gcr_ortho<4><<<gg, GNT, 0, ctx->stream>>>(ga, W, Z, r, k, sc, part, tk);
                else if (k <= 8) k_gcr_ortho<8><<<gg, GNT, 0, ctx->stream>>>(ga, W, Z, r, k, sc, part, tk);
                else k_gcr_ortho<NKV_MAX><<<gg, GNT, 0, ctx->stream>>>(ga, W, Z, r, k, sc, part, tk);
                ++ctx->launches;
                k_gcr_r<<<gg, GNT, 0, ctx->stream>>>(ga, W, r, k, sc, part, tk);
            }
            if ((st = any_active(&act))) return st;
        }
        {
            ProfScope ps(ctx, PROF_BLAS, 0.0);
            ++ctx->launches;
            if (k <= 4) k_gcr_x<4><<<gg, GNT, 0, ctx->stream>>>(ga, Z, x, k, sc);
            else if (k <= 8) k_gcr_x<8><<<gg, GNT, 0, ctx->stream>>>(ga, Z, x, k, sc);
            else k_gcr_x<NKV_MAX><<<gg, GNT, 0, ctx->stream>>>(ga, Z, x, k, sc);
        }
        if (!act || it >= maxiter) break;
        // restart from the recomputed residual r = b - D x
        apply_full32(ctx, ms, x, res, nrhs, -1.0);
        {
            ProfScope ps(ctx, PROF_BLAS, 0.0);
            ++ctx->launches;
            k_gcr_restart<<<gg, GNT, 0, ctx->stream>>>(ga, b, res, r, sc, part, tk);
        }
        if ((st = any_active(&act))) return st;
    }
    *iters += it;
    ctx->sap_last_iters = it;
    return DDRW_OK;
}

}  // namespace ddrw

using namespace ddrw;

extern "C" ddrw_status ddrw_apply_sap(ddrw_ctx *ctx, double m, const double *in, double *out, int nrhs)
{
    if (!ctx || !in || !out || nrhs <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    if (!sap_supported(ctx)) return set_error(ctx, DDRW_EINVAL, "Schwarz blocks of side 4 need every dimension a multiple of 8");
    cudaSetDevice(ctx->device);
    MassSet ms;
    ddrw_status st;
    if ((st = make_massset(ctx, 1, &m, &ms))) return st;
    const long V = ctx->V;
    const size_t ub = sizeof(double) * 24 * (size_t)V * nrhs, f64 = sizeof(double2) * 12 * (size_t)V * nrhs,
                 f32 = sizeof(float4) * 6 * (size_t)V * nrhs;
    const void *din;
    void *dout;
    bool host;
    double2 *F;
    float4 *e32, *p32, *rho, *chi;
    if ((st = stage_in(ctx, in, ub, "stage_in", &din))) return st;
    if ((st = stage_out(ctx, out, ub, "stage_out", &dout, &host))) return st;
    if ((st = workspace(ctx, "api_f0", f64, (void **)&F))) return st;
    if ((st = workspace(ctx, "sapi_e", f32, (void **)&e32))) return st;
    if ((st = workspace(ctx, "sapi_p", f32, (void **)&p32))) return st;
    if ((st = workspace(ctx, "gcr_rho", f32, (void **)&rho))) return st;
    if ((st = workspace(ctx, "gcr_chi", f32, (void **)&chi))) return st;
    pack_spinor64(ctx, (const double *)din, F, nrhs);
    const VecRange all{V, 0, V, 12 * V, nrhs};
    to_low<PrecS>(ctx, all, 6 * V, F, e32, nullptr);
    sap_apply(ctx, ms, e32, p32, rho, chi, nrhs, nrhs % 2 == 0 ? 2 : 1);
    DDRW_CUDA_CHECK(cudaMemsetAsync(F, 0, f64, ctx->stream));
    add_low<PrecS>(ctx, all, 6 * V, p32, F, nullptr);
    unpack_spinor64(ctx, F, (double *)dout, nrhs);
    if ((st = finish_out(ctx, out, dout, ub, host))) return st;
    return sync(ctx);
}
