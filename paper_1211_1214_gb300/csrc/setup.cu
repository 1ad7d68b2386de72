// setup.cu -- once-per-configuration work (K1, K2) and layout conversion at the boundary:
//   * gauge field: boundary layout U[lex][mu][3][3] -> FP64 SoA planes, FP32 two-row planes;
//   * clover term: see clover.cuh;
//   * per-mass inverses of A(m) = (4 + m) + C (Gauss-Jordan in FP64 per site and chirality);
//   * spinor fields boundary layout <-> internal planes, packed supp-P vectors <-> fields.
#include "ctx.h"

namespace ddrw {

// ----------------------------------------------------------------------------- gauge

template <int BL>
__global__ void k_pack_gauge(GeomDev g, const double *__restrict__ Ulex, double2 *U64, float4 *U32)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    long x = lex_index<BL>(st, g);
    for (int mu = 0; mu < 4; mu++) {
        const double *u = Ulex + (x * 4 + mu) * 18;
        for (int k = 0; k < 9; k++) U64[((long)mu * 9 + k) * g.V + s] = make_double2(u[2 * k], u[2 * k + 1]);
        // two-row FP32: (u00 u01) (u02 u10) (u11 u12)
        for (int k = 0; k < 3; k++)
            U32[((long)mu * 3 + k) * g.V + s] =
                make_float4((float)u[4 * k], (float)u[4 * k + 1], (float)u[4 * k + 2], (float)u[4 * k + 3]);
    }
}

// ----------------------------------------------------------------------------- neighbour table

// one entry per site and hop, from decode_site / neighbour (the geometry copy has tsign = -1, so
// that neighbour() reports every hop across the time boundary, whatever the boundary condition)
template <int BL>
__global__ void k_nbr_table(GeomDev g, int4 *t)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    int e[8];
#pragma unroll
    for (int mu = 0; mu < 4; mu++)
#pragma unroll
        for (int d = 0; d < 2; d++) {
            bool cross;
            int ph;
            unsigned n = (unsigned)neighbour<BL>(st, mu, d == 0 ? +1 : -1, g, &cross, &ph);
            if (cross) n |= (unsigned)NBR_CROSS;
            if (ph < 0) n |= 0x80000000u;
            e[2 * mu + d] = (int)n;
        }
    t[s] = make_int4(e[0], e[1], e[2], e[3]);
    t[g.V + s] = make_int4(e[4], e[5], e[6], e[7]);
}

// FP32 two-row U_mu(x - mu) copied to x, so that a tile of output sites finds all 8 of its links
// in contiguous planes
__global__ void k_bw_links(long V, const int4 *__restrict__ nbr, const float4 *__restrict__ U32, float4 *Ubw)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const int4 n0 = nbr[s], n1 = nbr[V + s];
    const int b[4] = {n0.y & NBR_IDX, n0.w & NBR_IDX, n1.y & NBR_IDX, n1.w & NBR_IDX};
#pragma unroll
    for (int mu = 0; mu < 4; mu++)
#pragma unroll
        for (int k = 0; k < 3; k++) Ubw[(long)(mu * 3 + k) * V + s] = U32[(long)(mu * 3 + k) * V + b[mu]];
}

// ----------------------------------------------------------------------------- clover

template <int BL> void clover_launch(ddrw_ctx *ctx);

// The inverse of the Hermitian 6x6 block A = (4 + m) + H (H packed: 6 real diagonal entries, then
// the 15 upper entries at 6 + 2 herm_off(i, j)) by the factorisation A = L D L^dag (L unit lower
// triangular, D real diagonal) without pivoting, then A^-1 = X^dag D^-1 X with X = L^-1; all in
// registers with the loops unrolled.  Returns false if a pivot is not clearly nonzero (then the
// caller falls back to Gauss-Jordan with partial pivoting).
__device__ __forceinline__ bool herm6_inverse_ldl(const double *r, double mass, double *o)
{
    cpx<double> L[6][6];
    double d[6], dinv[6];
    double scale = 0.0;
#pragma unroll
    for (int i = 0; i < 6; i++) scale = fmax(scale, fabs(4.0 + mass + r[i]));
#pragma unroll
    for (int j = 0; j < 6; j++) {
        double dj = 4.0 + mass + r[j];
#pragma unroll
        for (int k = 0; k < j; k++) dj -= (L[j][k].re * L[j][k].re + L[j][k].im * L[j][k].im) * d[k];
        if (!(fabs(dj) > 1e-10 * scale)) return false;
        d[j] = dj;
        dinv[j] = 1.0 / dj;
#pragma unroll
        for (int i = j + 1; i < 6; i++) {
            const int q = 6 + 2 * herm_off(j, i);
            cpx<double> a = {r[q], -r[q + 1]};  // A[i][j] = conj(A[j][i])
#pragma unroll
            for (int k = 0; k < j; k++) {
                const cpx<double> t = cmulc(L[j][k], L[i][k]);  // conj(L[j][k]) L[i][k]
                a = {a.re - d[k] * t.re, a.im - d[k] * t.im};
            }
            L[i][j] = {a.re * dinv[j], a.im * dinv[j]};
        }
    }
    // X = L^-1 (unit lower triangular)
    cpx<double> X[6][6];
#pragma unroll
    for (int j = 0; j < 6; j++) {
#pragma unroll
        for (int i = j + 1; i < 6; i++) {
            cpx<double> a = {-L[i][j].re, -L[i][j].im};
#pragma unroll
            for (int k = j + 1; k < i; k++) a = a - cmul(L[i][k], X[k][j]);
            X[i][j] = a;
        }
    }
    // A^-1_ij = sum_{k >= max(i, j)} conj(X_ki) X_kj / d_k  (X_kk = 1)
#pragma unroll
    for (int i = 0; i < 6; i++) {
        double s = dinv[i];
#pragma unroll
        for (int k = i + 1; k < 6; k++) s += (X[k][i].re * X[k][i].re + X[k][i].im * X[k][i].im) * dinv[k];
        o[i] = s;
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            cpx<double> s2 = {X[j][i].re * dinv[j], -X[j][i].im * dinv[j]};  // k = j: conj(X_ji) X_jj
#pragma unroll
            for (int k = j + 1; k < 6; k++) {
                const cpx<double> t = cmulc(X[k][i], X[k][j]);
                s2 = {s2.re + t.re * dinv[k], s2.im + t.im * dinv[k]};
            }
            const int q = 6 + 2 * herm_off(i, j);
            o[q] = s2.re;
            o[q + 1] = s2.im;
        }
    }
    return true;
}

// the same by Gauss-Jordan with partial pivoting (any nonsingular block)
__device__ __noinline__ void herm6_inverse_gj(const double *r, double mass, double *o)
{
    {
        cpx<double> A[6][12];
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 12; j++) A[i][j] = {0.0, 0.0};
        for (int i = 0; i < 6; i++) {
            A[i][i] = {4.0 + mass + r[i], 0.0};
            A[i][6 + i] = {1.0, 0.0};
            for (int j = i + 1; j < 6; j++) {
                int k = 6 + 2 * herm_off(i, j);
                A[i][j] = {r[k], r[k + 1]};
                A[j][i] = {r[k], -r[k + 1]};
            }
        }
        for (int c = 0; c < 6; c++) {
            int piv = c;
            double best = A[c][c].re * A[c][c].re + A[c][c].im * A[c][c].im;
            for (int i = c + 1; i < 6; i++) {
                double v = A[i][c].re * A[i][c].re + A[i][c].im * A[i][c].im;
                if (v > best) { best = v; piv = i; }
            }
            if (piv != c)
                for (int j = 0; j < 12; j++) { cpx<double> t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
            cpx<double> d = A[c][c];
            double dn = d.re * d.re + d.im * d.im;
            cpx<double> inv = {d.re / dn, -d.im / dn};
            for (int j = 0; j < 12; j++) A[c][j] = cmul(inv, A[c][j]);
            for (int i = 0; i < 6; i++) {
                if (i == c) continue;
                cpx<double> f = A[i][c];
                for (int j = 0; j < 12; j++) A[i][j] = A[i][j] - cmul(f, A[c][j]);
            }
        }
        for (int i = 0; i < 6; i++) o[i] = A[i][6 + i].re;
        for (int i = 0; i < 6; i++)
            for (int j = i + 1; j < 6; j++) {
                int k = 6 + 2 * herm_off(i, j);
                // average the (i,j) entry and the conjugate of (j,i): exact Hermitian result
                o[k] = 0.5 * (A[i][6 + j].re + A[j][6 + i].re);
                o[k + 1] = 0.5 * (A[i][6 + j].im - A[j][6 + i].im);
            }
    }
}

// A(m)^-1 = ((4 + m) + C_ch)^-1 per chirality in FP64 (LDL^dag, Gauss-Jordan if a pivot vanishes)
__global__ void k_inverse(long V, const double2 *__restrict__ C64, double mass, double2 *A64, float4 *A32)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
#pragma unroll 1
    for (int ch = 0; ch < 2; ch++) {
        double r[36];
#pragma unroll
        for (int k = 0; k < 18; k++) {
            double2 v = C64[((long)ch * 18 + k) * V + s];
            r[2 * k] = v.x;
            r[2 * k + 1] = v.y;
        }
        double o[36];
        if (!herm6_inverse_ldl(r, mass, o)) {
            // rare: copies in local memory for the pivoting fallback, so that r and o stay in
            // registers on the common path
            double rr[36], oo[36];
#pragma unroll
            for (int k = 0; k < 36; k++) rr[k] = r[k];
            herm6_inverse_gj(rr, mass, oo);
#pragma unroll
            for (int k = 0; k < 36; k++) o[k] = oo[k];
        }
#pragma unroll
        for (int k = 0; k < 18; k++) A64[((long)ch * 18 + k) * V + s] = make_double2(o[2 * k], o[2 * k + 1]);
#pragma unroll
        for (int k = 0; k < 9; k++)
            A32[((long)ch * 9 + k) * V + s] =
                make_float4((float)o[4 * k], (float)o[4 * k + 1], (float)o[4 * k + 2], (float)o[4 * k + 3]);
    }
}

// ----------------------------------------------------------------------------- spinor layout

template <int BL>
__global__ void k_pack_spinor(GeomDev g, const double *__restrict__ user, double2 *f)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int r = blockIdx.y;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    long x = lex_index<BL>(st, g);
    const double *u = user + ((long)r * g.V + x) * 24;
    double2 *o = f + (long)r * 12 * g.V + s;
    for (int k = 0; k < 12; k++) o[(long)k * g.V] = make_double2(u[2 * k], u[2 * k + 1]);
}

template <int BL>
__global__ void k_unpack_spinor(GeomDev g, const double2 *__restrict__ f, double *user)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int r = blockIdx.y;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    long x = lex_index<BL>(st, g);
    double *u = user + ((long)r * g.V + x) * 24;
    const double2 *in = f + (long)r * 12 * g.V + s;
    for (int k = 0; k < 12; k++) {
        double2 v = in[(long)k * g.V];
        u[2 * k] = v.x;
        u[2 * k + 1] = v.y;
    }
}

__global__ void k_pack_P(long V, long nP, const int *__restrict__ idx, const double2 *__restrict__ f, double *out)
{
    long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nP) return;
    int r = blockIdx.y;
    long s = idx[j];
    const double2 *in = f + (long)r * 12 * V + s;
    double *o = out + ((long)r * nP + j) * 24;
    for (int k = 0; k < 12; k++) {
        double2 v = in[(long)k * V];
        o[2 * k] = v.x;
        o[2 * k + 1] = v.y;
    }
}

__global__ void k_unpack_P(long V, long nP, const int *__restrict__ idx, const double *__restrict__ in, double2 *f)
{
    long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nP) return;
    int r = blockIdx.y;
    long s = idx[j];
    double2 *o = f + (long)r * 12 * V + s;
    const double *u = in + ((long)r * nP + j) * 24;
    for (int k = 0; k < 12; k++) o[(long)k * V] = make_double2(u[2 * k], u[2 * k + 1]);
}

// ----------------------------------------------------------------------------- launchers

#define DISPATCH_BL(ctx, KERNEL, GRID, BLOCK, ...)                                                        \
    ++(ctx)->launches;                                                                                    \
    switch ((ctx)->l) {                                                                                   \
    case 2: KERNEL<2><<<GRID, BLOCK, 0, (ctx)->stream>>>(__VA_ARGS__); break;                             \
    case 4: KERNEL<4><<<GRID, BLOCK, 0, (ctx)->stream>>>(__VA_ARGS__); break;                             \
    case 6: KERNEL<6><<<GRID, BLOCK, 0, (ctx)->stream>>>(__VA_ARGS__); break;                             \
    default: KERNEL<8><<<GRID, BLOCK, 0, (ctx)->stream>>>(__VA_ARGS__); break;                            \
    }

void pack_gauge(ddrw_ctx *ctx, const double *Ulex)
{
    GeomDev g = geom_dev(ctx);
    dim3 grid((unsigned)((ctx->V + 127) / 128));
    DISPATCH_BL(ctx, k_pack_gauge, grid, 128, g, Ulex, ctx->U64, ctx->U32);
}

void build_nbr_table(ddrw_ctx *ctx)
{
    GeomDev g = geom_dev(ctx);
    g.tsign = -1;
    dim3 grid((unsigned)((ctx->V + 127) / 128));
    DISPATCH_BL(ctx, k_nbr_table, grid, 128, g, ctx->d_nbr);
}

void build_bw_links(ddrw_ctx *ctx)
{
    ++ctx->launches;
    k_bw_links<<<(unsigned)((ctx->V + 127) / 128), 128, 0, ctx->stream>>>(ctx->V, ctx->d_nbr, ctx->U32, ctx->Ubw32);
}

void build_clover(ddrw_ctx *ctx)
{
    switch (ctx->l) {
    case 2: clover_launch<2>(ctx); break;
    case 4: clover_launch<4>(ctx); break;
    case 6: clover_launch<6>(ctx); break;
    default: clover_launch<8>(ctx); break;
    }
}

void build_inverse(ddrw_ctx *ctx, double m, MassInv &mi)
{
    dim3 grid((unsigned)((ctx->V + 63) / 64));
    ++ctx->launches;
    k_inverse<<<grid, 64, 0, ctx->stream>>>(ctx->V, ctx->C64, m, mi.A64, mi.A32);
}

void pack_spinor64(ddrw_ctx *ctx, const double *user, double2 *f, int nrhs)
{
    GeomDev g = geom_dev(ctx);
    dim3 grid((unsigned)((ctx->V + 127) / 128), (unsigned)nrhs);
    DISPATCH_BL(ctx, k_pack_spinor, grid, 128, g, user, f);
}

void unpack_spinor64(ddrw_ctx *ctx, const double2 *f, double *user, int nrhs)
{
    GeomDev g = geom_dev(ctx);
    dim3 grid((unsigned)((ctx->V + 127) / 128), (unsigned)nrhs);
    DISPATCH_BL(ctx, k_unpack_spinor, grid, 128, g, f, user);
}

void pack_P64(ddrw_ctx *ctx, const double2 *f, double *packed, int nrhs)
{
    if (ctx->nP == 0) return;
    dim3 grid((unsigned)((ctx->nP + 127) / 128), (unsigned)nrhs);
    ++ctx->launches;
    k_pack_P<<<grid, 128, 0, ctx->stream>>>(ctx->V, ctx->nP, ctx->d_suppP, f, packed);
}

void unpack_P64(ddrw_ctx *ctx, const double *packed, double2 *f, int nrhs)
{
    cudaMemsetAsync(f, 0, sizeof(double2) * 12 * (size_t)ctx->V * nrhs, ctx->stream);
    if (ctx->nP == 0) return;
    dim3 grid((unsigned)((ctx->nP + 127) / 128), (unsigned)nrhs);
    ++ctx->launches;
    k_unpack_P<<<grid, 128, 0, ctx->stream>>>(ctx->V, ctx->nP, ctx->d_suppP, packed, f);
}

}  // namespace ddrw
