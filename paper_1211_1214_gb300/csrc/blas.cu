// blas.cu -- vector kernels and reductions of the Krylov solvers (K7).
//
// A vector is a site range [off, off + n) of a field (all planes), for nrhs right-hand sides along
// gridDim.y.  Reductions: each thread accumulates in the storage precision's arithmetic type,
// warps and CTAs sum in FP64 (warp shuffles, shared memory), and the last CTA of a right-hand side
// to finish (atomic ticket after a fence) sums the per-CTA partials in a fixed order, so the
// result does not depend on scheduling.  The solver scalars stay on the device; the last CTA
// also performs the scalar update of the Krylov recurrence.
#include "blas.cuh"
#include "ctx.h"
#include "lowprec.cuh"

namespace ddrw {

// ----------------------------------------------------------------------------- element access

template <class P> struct VecArgs {
    long V, off, n, rs;  // plane stride, first site, sites, rhs stride (elements)
};

constexpr int NT = 256;

// ----------------------------------------------------------------------------- BiCGStab steps
// Scalars per right-hand side in KScal (blas.cuh).  r holds s = r - alpha v after the s-step.

template <class P>
__global__ void __launch_bounds__(NT) k_bicg_init(VecArgs<P> va, typename P::SElem *r, typename P::SElem *rh,
                                                  typename P::SElem *p, typename P::SElem *x, KScal *sc,
                                                  double *part, unsigned *ticket)
{
    using R = typename P::R;
    const long rb = (long)blockIdx.y * va.rs;
    R acc = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> c[P::CW], z[P::CW];
            P::ld_chunk(r + rb, va.V, va.off + j, k, c);
#pragma unroll
            for (int q = 0; q < P::CW; q++) {
                acc += c[q].re * c[q].re + c[q].im * c[q].im;
                z[q] = {R(0), R(0)};
            }
            P::st_chunk(rh + rb, va.V, va.off + j, k, c);
            P::st_chunk(p + rb, va.V, va.off + j, k, c);
            P::st_chunk(x + rb, va.V, va.off + j, k, z);
        }
    double v[1] = {(double)acc};
    if (grid_sum<1, NT>(v, part, ticket)) {
        KScal &s = sc[blockIdx.y];
        s.rho = make_double2(v[0], 0.0);
        s.rr = v[0];
        s.iters = 0;
        s.breakdown = 0;
        s.active = (v[0] > s.thresh) ? 1 : 0;
    }
}

template <class P>
__global__ void __launch_bounds__(NT) k_bicg_alpha(VecArgs<P> va, const typename P::SElem *rh,
                                                   const typename P::SElem *v, KScal *sc, double *part,
                                                   unsigned *ticket)
{
    using R = typename P::R;
    if (!sc[blockIdx.y].active) return;
    const long rb = (long)blockIdx.y * va.rs;
    R are = 0, aim = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> c[P::CW], d[P::CW];
            P::ld_chunk(rh + rb, va.V, va.off + j, k, c);
            P::ld_chunk(v + rb, va.V, va.off + j, k, d);
#pragma unroll
            for (int q = 0; q < P::CW; q++) {
                cpx<R> t = cmulc(c[q], d[q]);
                are += t.re;
                aim += t.im;
            }
        }
    double val[2] = {(double)are, (double)aim};
    if (grid_sum<2, NT>(val, part, ticket)) {
        KScal &s = sc[blockIdx.y];
        double den = val[0] * val[0] + val[1] * val[1];
        if (den == 0.0 || !(den == den)) {
            s.breakdown = 1;
            s.active = 0;
            s.alpha = make_double2(0.0, 0.0);
            return;
        }
        // alpha = rho / (rh, v)
        s.alpha = make_double2((s.rho.x * val[0] + s.rho.y * val[1]) / den, (s.rho.y * val[0] - s.rho.x * val[1]) / den);
    }
}

template <class P>
__global__ void __launch_bounds__(NT) k_bicg_s(VecArgs<P> va, typename P::SElem *r, const typename P::SElem *v,
                                               const KScal *sc)
{
    using R = typename P::R;
    const KScal &s = sc[blockIdx.y];
    if (!s.active) return;
    const cpx<R> al = {R(s.alpha.x), R(s.alpha.y)};
    const long rb = (long)blockIdx.y * va.rs;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> c[P::CW], d[P::CW];
            P::ld_chunk(r + rb, va.V, va.off + j, k, c);
            P::ld_chunk(v + rb, va.V, va.off + j, k, d);
#pragma unroll
            for (int q = 0; q < P::CW; q++) c[q] = c[q] - cmul(al, d[q]);
            P::st_chunk(r + rb, va.V, va.off + j, k, c);
        }
}

template <class P>
__global__ void __launch_bounds__(NT) k_bicg_omega(VecArgs<P> va, const typename P::SElem *t,
                                                   const typename P::SElem *r, KScal *sc, double *part,
                                                   unsigned *ticket)
{
    using R = typename P::R;
    if (!sc[blockIdx.y].active) return;
    const long rb = (long)blockIdx.y * va.rs;
    R tsr = 0, tsi = 0, tt = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> c[P::CW], d[P::CW];
            P::ld_chunk(t + rb, va.V, va.off + j, k, c);
            P::ld_chunk(r + rb, va.V, va.off + j, k, d);
#pragma unroll
            for (int q = 0; q < P::CW; q++) {
                cpx<R> z = cmulc(c[q], d[q]);
                tsr += z.re;
                tsi += z.im;
                tt += c[q].re * c[q].re + c[q].im * c[q].im;
            }
        }
    double val[3] = {(double)tsr, (double)tsi, (double)tt};
    if (grid_sum<3, NT>(val, part, ticket)) {
        KScal &s = sc[blockIdx.y];
        if (val[2] == 0.0 || !(val[2] == val[2])) {
            s.breakdown = 2;
            s.active = 0;
            s.omega = make_double2(0.0, 0.0);
            return;
        }
        s.omega = make_double2(val[0] / val[2], val[1] / val[2]);
    }
}

// x += alpha p + omega s;  r = s - omega t;  rho' = (rh, r), rr = (r, r);  beta = (rho'/rho)(alpha/omega)
template <class P>
__global__ void __launch_bounds__(NT) k_bicg_xr(VecArgs<P> va, typename P::SElem *x, const typename P::SElem *p,
                                                typename P::SElem *r, const typename P::SElem *t,
                                                const typename P::SElem *rh, KScal *sc, double *part,
                                                unsigned *ticket)
{
    using R = typename P::R;
    const KScal &s0 = sc[blockIdx.y];
    if (!s0.active) return;
    const cpx<R> al = {R(s0.alpha.x), R(s0.alpha.y)}, om = {R(s0.omega.x), R(s0.omega.y)};
    const long rb = (long)blockIdx.y * va.rs;
    R rhre = 0, rhim = 0, rr = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> xv[P::CW], pv[P::CW], sv[P::CW], tv[P::CW], hv[P::CW];
            P::ld_chunk(x + rb, va.V, va.off + j, k, xv);
            P::ld_chunk(p + rb, va.V, va.off + j, k, pv);
            P::ld_chunk(r + rb, va.V, va.off + j, k, sv);
            P::ld_chunk(t + rb, va.V, va.off + j, k, tv);
            P::ld_chunk(rh + rb, va.V, va.off + j, k, hv);
#pragma unroll
            for (int q = 0; q < P::CW; q++) {
                xv[q] = xv[q] + cmul(al, pv[q]) + cmul(om, sv[q]);
                sv[q] = sv[q] - cmul(om, tv[q]);
                cpx<R> z = cmulc(hv[q], sv[q]);
                rhre += z.re;
                rhim += z.im;
                rr += sv[q].re * sv[q].re + sv[q].im * sv[q].im;
            }
            P::st_chunk(x + rb, va.V, va.off + j, k, xv);
            P::st_chunk(r + rb, va.V, va.off + j, k, sv);
        }
    double val[3] = {(double)rhre, (double)rhim, (double)rr};
    if (grid_sum<3, NT>(val, part, ticket)) {
        KScal &s = sc[blockIdx.y];
        s.rr = val[2];
        s.iters += 1;
        double2 rn = make_double2(val[0], val[1]);
        // beta = (rn / rho) * (alpha / omega)
        double d1 = s.rho.x * s.rho.x + s.rho.y * s.rho.y;
        double d2 = s.omega.x * s.omega.x + s.omega.y * s.omega.y;
        double2 q1 = make_double2((rn.x * s.rho.x + rn.y * s.rho.y) / d1, (rn.y * s.rho.x - rn.x * s.rho.y) / d1);
        double2 q2 = make_double2((s.alpha.x * s.omega.x + s.alpha.y * s.omega.y) / d2,
                                  (s.alpha.y * s.omega.x - s.alpha.x * s.omega.y) / d2);
        s.beta = make_double2(q1.x * q2.x - q1.y * q2.y, q1.x * q2.y + q1.y * q2.x);
        s.rho = rn;
        if (!(val[2] == val[2])) {
            s.breakdown = 3;
            s.active = 0;
        } else if (val[2] <= s.thresh || s.iters >= s.maxiter) {
            s.active = 0;
        } else if (rn.x * rn.x + rn.y * rn.y == 0.0 || d1 == 0.0) {
            s.breakdown = 4;
            s.active = 0;
        }
    }
}

template <class P>
__global__ void __launch_bounds__(NT) k_bicg_p(VecArgs<P> va, typename P::SElem *p, const typename P::SElem *r,
                                               const typename P::SElem *v, const KScal *sc)
{
    using R = typename P::R;
    const KScal &s = sc[blockIdx.y];
    if (!s.active) return;
    const cpx<R> be = {R(s.beta.x), R(s.beta.y)}, om = {R(s.omega.x), R(s.omega.y)};
    const long rb = (long)blockIdx.y * va.rs;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> pv[P::CW], rv[P::CW], vv[P::CW];
            P::ld_chunk(p + rb, va.V, va.off + j, k, pv);
            P::ld_chunk(r + rb, va.V, va.off + j, k, rv);
            P::ld_chunk(v + rb, va.V, va.off + j, k, vv);
#pragma unroll
            for (int q = 0; q < P::CW; q++) pv[q] = rv[q] + cmul(be, pv[q] - cmul(om, vv[q]));
            P::st_chunk(p + rb, va.V, va.off + j, k, pv);
        }
}

// alpha (MODE 1) or omega (MODE 2) from the per-warp partial sums a fused stencil epilogue wrote:
// part[(r * nwt + j) * 3 + k], summed in FP64 in a fixed order (one CTA per right-hand side)
template <int MODE>
__global__ void __launch_bounds__(NT) k_bicg_fin(const double *part, long nwt, KScal *sc)
{
    __shared__ double sm[NT / 32][3];
    const int r = blockIdx.x;
    if (!sc[r].active) return;
    double v[3] = {0.0, 0.0, 0.0};
    for (long j = threadIdx.x; j < nwt; j += NT) {
        const double *pp = part + ((long)r * nwt + j) * 3;
        v[0] += pp[0];
        v[1] += pp[1];
        v[2] += pp[2];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; k++) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 3; k++) sm[w][k] = v[k];
    __syncthreads();
    if (threadIdx.x != 0) return;
    double val[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NT / 32; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) val[k] += sm[i][k];
    KScal &s = sc[r];
    if (MODE == 1) {  // alpha = rho / (rh, v)
        const double den = val[0] * val[0] + val[1] * val[1];
        if (den == 0.0 || !(den == den)) {
            s.breakdown = 1;
            s.active = 0;
            s.alpha = make_double2(0.0, 0.0);
            return;
        }
        s.alpha = make_double2((s.rho.x * val[0] + s.rho.y * val[1]) / den, (s.rho.y * val[0] - s.rho.x * val[1]) / den);
    } else {  // omega = (t, s) / (t, t)
        if (val[2] == 0.0 || !(val[2] == val[2])) {
            s.breakdown = 2;
            s.active = 0;
            s.omega = make_double2(0.0, 0.0);
            return;
        }
        s.omega = make_double2(val[0] / val[2], val[1] / val[2]);
    }
}

void bicg_fin(ddrw_ctx *ctx, int mode, int nrhs, const double *part, long nwt, KScal *sc)
{
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    if (mode == 1) k_bicg_fin<1><<<nrhs, NT, 0, ctx->stream>>>(part, nwt, sc);
    else k_bicg_fin<2><<<nrhs, NT, 0, ctx->stream>>>(part, nwt, sc);
}

// ----------------------------------------------------------------------------- generic kernels

// out[r] = sum |f|^2 over the range (FP64 result per right-hand side)
template <class P>
__global__ void __launch_bounds__(NT) k_norm2(VecArgs<P> va, const typename P::SElem *f, double *out,
                                              double *part, unsigned *ticket)
{
    using R = typename P::R;
    const long rb = (long)blockIdx.y * va.rs;
    R acc = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> c[P::CW];
            P::ld_chunk(f + rb, va.V, va.off + j, k, c);
#pragma unroll
            for (int q = 0; q < P::CW; q++) acc += c[q].re * c[q].re + c[q].im * c[q].im;
        }
    double v[1] = {(double)acc};
    if (grid_sum<1, NT>(v, part, ticket)) out[blockIdx.y] = v[0];
}

// out[3r .. 3r+2] = (sum |d|^2, Re sum conj(d) e, Im sum conj(d) e) -- the exponents
// ||delta||^2 + 2 Re <eta, delta> and <eta, delta>
template <class P>
__global__ void __launch_bounds__(NT) k_norm_dot(VecArgs<P> va, const typename P::SElem *d,
                                                 const typename P::SElem *e, double *out, double *part,
                                                 unsigned *ticket)
{
    using R = typename P::R;
    const long rb = (long)blockIdx.y * va.rs;
    R nn = 0, dr = 0, di = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> c[P::CW], f[P::CW];
            P::ld_chunk(d + rb, va.V, va.off + j, k, c);
            P::ld_chunk(e + rb, va.V, va.off + j, k, f);
#pragma unroll
            for (int q = 0; q < P::CW; q++) {
                nn += c[q].re * c[q].re + c[q].im * c[q].im;
                dr += c[q].re * f[q].re + c[q].im * f[q].im;
                di += c[q].re * f[q].im - c[q].im * f[q].re;
            }
        }
    double v[3] = {(double)nn, (double)dr, (double)di};
    if (grid_sum<3, NT>(v, part, ticket)) {
        out[3 * blockIdx.y] = v[0];
        out[3 * blockIdx.y + 1] = v[1];
        out[3 * blockIdx.y + 2] = v[2];
    }
}

// y = a x + b y with real per-launch scalars
template <class P>
__global__ void __launch_bounds__(NT) k_axpby(VecArgs<P> va, double a, const typename P::SElem *x, double b,
                                              typename P::SElem *y)
{
    using R = typename P::R;
    const long rb = (long)blockIdx.y * va.rs;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> c[P::CW], d[P::CW];
            P::ld_chunk(x + rb, va.V, va.off + j, k, c);
            P::ld_chunk(y + rb, va.V, va.off + j, k, d);
#pragma unroll
            for (int q = 0; q < P::CW; q++) d[q] = R(a) * c[q] + R(b) * d[q];
            P::st_chunk(y + rb, va.V, va.off + j, k, d);
        }
}

// FP64 -> storage precision P with a per-right-hand-side scale: out = in * scale[r]
template <class P>
__global__ void __launch_bounds__(NT) k_to_low(long V, long off, long n, long rs64, long rsl, const double2 *in,
                                               typename P::SElem *out, const double *scale)
{
    using R = typename P::R;
    const double sc = scale ? scale[blockIdx.y] : 1.0;
    const double2 *ib = in + (long)blockIdx.y * rs64;
    typename P::SElem *ob = out + (long)blockIdx.y * rsl;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> c[P::CW];
#pragma unroll
            for (int q = 0; q < P::CW; q++) {
                double2 a = ib[(long)(k * P::CW + q) * V + off + j];
                c[q] = {R(a.x * sc), R(a.y * sc)};
            }
            P::st_chunk(ob, V, off + j, k, c);
        }
}

// x64 += scale[r] * e (e in storage precision P)
template <class P>
__global__ void __launch_bounds__(NT) k_add_low(long V, long off, long n, long rs64, long rsl,
                                                const typename P::SElem *e, double2 *x, const double *scale)
{
    using R = typename P::R;
    const double sc = scale ? scale[blockIdx.y] : 1.0;
    const typename P::SElem *eb = e + (long)blockIdx.y * rsl;
    double2 *xb = x + (long)blockIdx.y * rs64;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::NCHUNK; k++) {
            cpx<R> c[P::CW];
            P::ld_chunk(eb, V, off + j, k, c);
#pragma unroll
            for (int q = 0; q < P::CW; q++) {
                double2 *a = xb + (long)(k * P::CW + q) * V + off + j;
                double2 av = *a;
                *a = make_double2(av.x + sc * (double)c[q].re, av.y + sc * (double)c[q].im);
            }
        }
}

// FP32 link / clover planes -> 16-bit planes of the same order
template <bool BF> __global__ void k_f32_to_low(long n, const float4 *__restrict__ in, uint2 *out)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 v = in[i];
    out[i] = make_uint2(Pack16<BF>::pack(v.x, v.y), Pack16<BF>::pack(v.z, v.w));
}

// ----------------------------------------------------------------------------- host side

static unsigned grid_for(long n)
{
    long g = (n + NT - 1) / NT;
    return (unsigned)(g < 1 ? 1 : (g > 608 ? 608 : g));
}

ddrw_status reduce_ws(ddrw_ctx *ctx, int nrhs, double **part, unsigned **ticket)
{
    void *p;
    ddrw_status st = workspace(ctx, "red_part", sizeof(double) * 4 * 608 * (size_t)nrhs, &p);
    if (st) return st;
    *part = (double *)p;
    DevBuf &t = ctx->ws["red_ticket"];
    if (t.bytes < sizeof(unsigned) * (size_t)nrhs) {
        clear_graphs(ctx);
        if (t.p) cudaFree(t.p);
        t.p = nullptr;
        t.bytes = 0;
        size_t bytes = sizeof(unsigned) * (size_t)(nrhs < 64 ? 64 : nrhs);
        if (cudaMalloc(&t.p, bytes) != cudaSuccess) return set_error(ctx, DDRW_ENOMEM, "ticket buffer");
        cudaMemsetAsync(t.p, 0, bytes, ctx->stream);
        t.bytes = bytes;
    }
    *ticket = (unsigned *)t.p;
    return DDRW_OK;
}

template <class P>
ddrw_status Blas<P>::bicg_init(ddrw_ctx *ctx, const VecRange &vr, E *r, E *rh, E *p, E *x, KScal *sc)
{
    double *part;
    unsigned *tk;
    ddrw_status st = reduce_ws(ctx, vr.nrhs, &part, &tk);
    if (st) return st;
    VecArgs<P> va{vr.V, vr.off, vr.n, vr.rs};
    dim3 g(grid_for(vr.n), vr.nrhs);
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_bicg_init<P><<<g, NT, 0, ctx->stream>>>(va, r, rh, p, x, sc, part, tk);
    return DDRW_OK;
}

template <class P>
ddrw_status Blas<P>::bicg_alpha(ddrw_ctx *ctx, const VecRange &vr, const E *rh, const E *v, KScal *sc)
{
    double *part;
    unsigned *tk;
    ddrw_status st = reduce_ws(ctx, vr.nrhs, &part, &tk);
    if (st) return st;
    VecArgs<P> va{vr.V, vr.off, vr.n, vr.rs};
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_bicg_alpha<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(va, rh, v, sc, part, tk);
    return DDRW_OK;
}

template <class P>
void Blas<P>::bicg_s(ddrw_ctx *ctx, const VecRange &vr, E *r, const E *v, const KScal *sc)
{
    VecArgs<P> va{vr.V, vr.off, vr.n, vr.rs};
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_bicg_s<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(va, r, v, sc);
}

template <class P>
ddrw_status Blas<P>::bicg_omega(ddrw_ctx *ctx, const VecRange &vr, const E *t, const E *r, KScal *sc)
{
    double *part;
    unsigned *tk;
    ddrw_status st = reduce_ws(ctx, vr.nrhs, &part, &tk);
    if (st) return st;
    VecArgs<P> va{vr.V, vr.off, vr.n, vr.rs};
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_bicg_omega<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(va, t, r, sc, part, tk);
    return DDRW_OK;
}

template <class P>
ddrw_status Blas<P>::bicg_xr(ddrw_ctx *ctx, const VecRange &vr, E *x, const E *p, E *r, const E *t, const E *rh,
                             KScal *sc)
{
    double *part;
    unsigned *tk;
    ddrw_status st = reduce_ws(ctx, vr.nrhs, &part, &tk);
    if (st) return st;
    VecArgs<P> va{vr.V, vr.off, vr.n, vr.rs};
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_bicg_xr<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(va, x, p, r, t, rh, sc, part, tk);
    return DDRW_OK;
}

template <class P>
void Blas<P>::bicg_p(ddrw_ctx *ctx, const VecRange &vr, E *p, const E *r, const E *v, const KScal *sc)
{
    VecArgs<P> va{vr.V, vr.off, vr.n, vr.rs};
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_bicg_p<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(va, p, r, v, sc);
}

template <class P>
ddrw_status Blas<P>::norm2(ddrw_ctx *ctx, const VecRange &vr, const E *f, double *out)
{
    double *part;
    unsigned *tk;
    ddrw_status st = reduce_ws(ctx, vr.nrhs, &part, &tk);
    if (st) return st;
    VecArgs<P> va{vr.V, vr.off, vr.n, vr.rs};
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_norm2<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(va, f, out, part, tk);
    return DDRW_OK;
}

template <class P>
ddrw_status Blas<P>::norm_dot(ddrw_ctx *ctx, const VecRange &vr, const E *d, const E *e, double *out)
{
    double *part;
    unsigned *tk;
    ddrw_status st = reduce_ws(ctx, vr.nrhs, &part, &tk);
    if (st) return st;
    VecArgs<P> va{vr.V, vr.off, vr.n, vr.rs};
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_norm_dot<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(va, d, e, out, part, tk);
    return DDRW_OK;
}

template <class P>
void Blas<P>::axpby(ddrw_ctx *ctx, const VecRange &vr, double a, const E *x, double b, E *y)
{
    VecArgs<P> va{vr.V, vr.off, vr.n, vr.rs};
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_axpby<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(va, a, x, b, y);
}

template <class P>
void to_low(ddrw_ctx *ctx, const VecRange &vr, long rsl, const double2 *in, typename P::SElem *out,
            const double *scale)
{
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_to_low<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(vr.V, vr.off, vr.n, vr.rs, rsl, in, out, scale);
}

template <class P>
void add_low(ddrw_ctx *ctx, const VecRange &vr, long rsl, const typename P::SElem *e, double2 *x, const double *scale)
{
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_add_low<P><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(vr.V, vr.off, vr.n, vr.rs, rsl, e, x, scale);
}

void f32_to_low(ddrw_ctx *ctx, const float4 *in, uint2 *out, long n, bool bf)
{
    ++ctx->launches;
    unsigned g = (unsigned)((n + 255) / 256);
    if (bf) k_f32_to_low<true><<<g, 256, 0, ctx->stream>>>(n, in, out);
    else k_f32_to_low<false><<<g, 256, 0, ctx->stream>>>(n, in, out);
}

// FP32 field -> 16-bit field over a site range (the 16-bit spinor takes its per-site norm anew)
template <class P16>
__global__ void __launch_bounds__(NT) k_f32_to_16(long V, long off, long n, long rs32, long rs16, const float4 *in,
                                                  typename P16::SElem *out)
{
    const float4 *ib = in + (long)blockIdx.y * rs32;
    typename P16::SElem *ob = out + (long)blockIdx.y * rs16;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < n; j += (long)gridDim.x * NT) {
        Spinor<float> p;
        PrecS::load_spinor_rw(ib, (int)V, (int)(off + j), p);
        P16::store_spinor(ob, (int)V, (int)(off + j), p);
    }
}

// x32 += x16 over a site range, then x16 = 0 (the reliable update of a 16-bit Krylov solve)
template <class P16>
__global__ void __launch_bounds__(NT) k_fold_16_into_32(long V, long off, long n, long rs16, long rs32,
                                                        typename P16::SElem *x16, float4 *x32)
{
    typename P16::SElem *hb = x16 + (long)blockIdx.y * rs16;
    float4 *fb = x32 + (long)blockIdx.y * rs32;
    Spinor<float> z;
    zero(z);
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < n; j += (long)gridDim.x * NT) {
        const int sj = (int)(off + j);
        Spinor<float> a, b;
        P16::load_spinor_rw(hb, (int)V, sj, a);
        PrecS::load_spinor_rw(fb, (int)V, sj, b);
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) b.v[sp][c] = b.v[sp][c] + a.v[sp][c];
        PrecS::store_spinor(fb, (int)V, sj, b);
        P16::store_spinor(hb, (int)V, sj, z);
    }
}

template <class P16>
void f32_to_16(ddrw_ctx *ctx, const VecRange &vr, long rs16, const float4 *in, typename P16::SElem *out)
{
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_f32_to_16<P16><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(vr.V, vr.off, vr.n, vr.rs, rs16, in, out);
}

template <class P16>
void fold_16_into_32(ddrw_ctx *ctx, const VecRange &vr, long rs16, typename P16::SElem *x16, float4 *x32)
{
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_fold_16_into_32<P16><<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(vr.V, vr.off, vr.n, rs16, vr.rs, x16,
                                                                                   x32);
}
template void f32_to_16<PrecH>(ddrw_ctx *, const VecRange &, long, const float4 *, PrecH::SElem *);
template void f32_to_16<PrecB>(ddrw_ctx *, const VecRange &, long, const float4 *, PrecB::SElem *);
template void fold_16_into_32<PrecH>(ddrw_ctx *, const VecRange &, long, PrecH::SElem *, float4 *);
template void fold_16_into_32<PrecB>(ddrw_ctx *, const VecRange &, long, PrecB::SElem *, float4 *);

#define DDRW_LOW_INST(P)                                                                                      \
    template void to_low<P>(ddrw_ctx *, const VecRange &, long, const double2 *, P::SElem *, const double *); \
    template void add_low<P>(ddrw_ctx *, const VecRange &, long, const P::SElem *, double2 *, const double *);
DDRW_LOW_INST(PrecS)
DDRW_LOW_INST(PrecH)
DDRW_LOW_INST(PrecB)

template struct Blas<PrecD>;
template struct Blas<PrecS>;
template struct Blas<PrecH>;
template struct Blas<PrecB>;

}  // namespace ddrw
