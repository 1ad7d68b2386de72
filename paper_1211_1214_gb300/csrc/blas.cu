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

namespace ddrw {

// ----------------------------------------------------------------------------- element access

template <class P> struct VecArgs {
    long V, off, n, rs;  // plane stride, first site, sites, rhs stride (elements)
};

// ----------------------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum v[0..K) over the grid's CTAs for right-hand side blockIdx.y.  Returns true in thread 0 of the
// last CTA, with the totals in v.  part: [nrhs][gridDim.x][K] doubles, ticket: [nrhs] zeroed.
template <int K, int NT>
__device__ bool grid_sum(double (&v)[K], double *part, unsigned *ticket)
{
    __shared__ double sm[NT / 32][K];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sm[w][k] = v[k];
    __syncthreads();
    const int r = blockIdx.y, G = gridDim.x;
    if (threadIdx.x == 0) {
        double *pp = part + ((long)r * G + blockIdx.x) * K;
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = 0;
            for (int i = 0; i < NT / 32; i++) s += sm[i][k];
            pp[k] = s;
        }
        __threadfence();
        unsigned t = atomicAdd(ticket + r, 1u);
        last = (t == (unsigned)(G - 1));
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = 0;
    for (int i = threadIdx.x; i < G; i += NT) {
        const double *pp = part + ((long)r * G + i) * K;
#pragma unroll
        for (int k = 0; k < K; k++) acc[k] += __ldcg(pp + k);
    }
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = warp_sum(acc[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sm[w][k] = acc[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = 0;
            for (int i = 0; i < NT / 32; i++) s += sm[i][k];
            v[k] = s;
        }
        ticket[r] = 0;
        return true;
    }
    return false;
}

constexpr int NT = 256;

// ----------------------------------------------------------------------------- BiCGStab steps
// Scalars per right-hand side in KScal (blas.cuh).  r holds s = r - alpha v after the s-step.

template <class P>
__global__ void __launch_bounds__(NT) k_bicg_init(VecArgs<P> va, typename P::SElem *r, typename P::SElem *rh,
                                                  typename P::SElem *p, typename P::SElem *x, KScal *sc,
                                                  double *part, unsigned *ticket)
{
    using E = typename P::SElem;
    using L = El<E>;
    using R = typename L::R;
    const long ro = (long)blockIdx.y * va.rs + va.off;
    R acc = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::SPLANES; k++) {
            long a = ro + k * va.V + j;
            cpx<R> c[L::NC], z[L::NC];
            L::ld(r + a, c);
#pragma unroll
            for (int q = 0; q < L::NC; q++) {
                acc += c[q].re * c[q].re + c[q].im * c[q].im;
                z[q] = {R(0), R(0)};
            }
            L::st(rh + a, c);
            L::st(p + a, c);
            L::st(x + a, z);
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
    using E = typename P::SElem;
    using L = El<E>;
    using R = typename L::R;
    if (!sc[blockIdx.y].active) return;
    const long ro = (long)blockIdx.y * va.rs + va.off;
    R are = 0, aim = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::SPLANES; k++) {
            long a = ro + k * va.V + j;
            cpx<R> c[L::NC], d[L::NC];
            L::ld(rh + a, c);
            L::ld(v + a, d);
#pragma unroll
            for (int q = 0; q < L::NC; q++) {
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
    using E = typename P::SElem;
    using L = El<E>;
    using R = typename L::R;
    const KScal &s = sc[blockIdx.y];
    if (!s.active) return;
    const cpx<R> al = {R(s.alpha.x), R(s.alpha.y)};
    const long ro = (long)blockIdx.y * va.rs + va.off;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::SPLANES; k++) {
            long a = ro + k * va.V + j;
            cpx<R> c[L::NC], d[L::NC];
            L::ld(r + a, c);
            L::ld(v + a, d);
#pragma unroll
            for (int q = 0; q < L::NC; q++) c[q] = c[q] - cmul(al, d[q]);
            L::st(r + a, c);
        }
}

template <class P>
__global__ void __launch_bounds__(NT) k_bicg_omega(VecArgs<P> va, const typename P::SElem *t,
                                                   const typename P::SElem *r, KScal *sc, double *part,
                                                   unsigned *ticket)
{
    using E = typename P::SElem;
    using L = El<E>;
    using R = typename L::R;
    if (!sc[blockIdx.y].active) return;
    const long ro = (long)blockIdx.y * va.rs + va.off;
    R tsr = 0, tsi = 0, tt = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::SPLANES; k++) {
            long a = ro + k * va.V + j;
            cpx<R> c[L::NC], d[L::NC];
            L::ld(t + a, c);
            L::ld(r + a, d);
#pragma unroll
            for (int q = 0; q < L::NC; q++) {
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
    using E = typename P::SElem;
    using L = El<E>;
    using R = typename L::R;
    const KScal &s0 = sc[blockIdx.y];
    if (!s0.active) return;
    const cpx<R> al = {R(s0.alpha.x), R(s0.alpha.y)}, om = {R(s0.omega.x), R(s0.omega.y)};
    const long ro = (long)blockIdx.y * va.rs + va.off;
    R rhre = 0, rhim = 0, rr = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::SPLANES; k++) {
            long a = ro + k * va.V + j;
            cpx<R> xv[L::NC], pv[L::NC], sv[L::NC], tv[L::NC], hv[L::NC];
            L::ld(x + a, xv);
            L::ld(p + a, pv);
            L::ld(r + a, sv);
            L::ld(t + a, tv);
            L::ld(rh + a, hv);
#pragma unroll
            for (int q = 0; q < L::NC; q++) {
                xv[q] = xv[q] + cmul(al, pv[q]) + cmul(om, sv[q]);
                sv[q] = sv[q] - cmul(om, tv[q]);
                cpx<R> z = cmulc(hv[q], sv[q]);
                rhre += z.re;
                rhim += z.im;
                rr += sv[q].re * sv[q].re + sv[q].im * sv[q].im;
            }
            L::st(x + a, xv);
            L::st(r + a, sv);
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
    using E = typename P::SElem;
    using L = El<E>;
    using R = typename L::R;
    const KScal &s = sc[blockIdx.y];
    if (!s.active) return;
    const cpx<R> be = {R(s.beta.x), R(s.beta.y)}, om = {R(s.omega.x), R(s.omega.y)};
    const long ro = (long)blockIdx.y * va.rs + va.off;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::SPLANES; k++) {
            long a = ro + k * va.V + j;
            cpx<R> pv[L::NC], rv[L::NC], vv[L::NC];
            L::ld(p + a, pv);
            L::ld(r + a, rv);
            L::ld(v + a, vv);
#pragma unroll
            for (int q = 0; q < L::NC; q++) pv[q] = rv[q] + cmul(be, pv[q] - cmul(om, vv[q]));
            L::st(p + a, pv);
        }
}

// ----------------------------------------------------------------------------- generic kernels

// out[r] = sum |f|^2 over the range (FP64 result per right-hand side)
template <class P>
__global__ void __launch_bounds__(NT) k_norm2(VecArgs<P> va, const typename P::SElem *f, double *out,
                                              double *part, unsigned *ticket)
{
    using E = typename P::SElem;
    using L = El<E>;
    using R = typename L::R;
    const long ro = (long)blockIdx.y * va.rs + va.off;
    R acc = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::SPLANES; k++) {
            cpx<R> c[L::NC];
            L::ld(f + ro + k * va.V + j, c);
#pragma unroll
            for (int q = 0; q < L::NC; q++) acc += c[q].re * c[q].re + c[q].im * c[q].im;
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
    using E = typename P::SElem;
    using L = El<E>;
    using R = typename L::R;
    const long ro = (long)blockIdx.y * va.rs + va.off;
    R nn = 0, dr = 0, di = 0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::SPLANES; k++) {
            cpx<R> c[L::NC], f[L::NC];
            L::ld(d + ro + k * va.V + j, c);
            L::ld(e + ro + k * va.V + j, f);
#pragma unroll
            for (int q = 0; q < L::NC; q++) {
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
    using E = typename P::SElem;
    using L = El<E>;
    using R = typename L::R;
    const long ro = (long)blockIdx.y * va.rs + va.off;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < va.n; j += (long)gridDim.x * NT)
        for (int k = 0; k < P::SPLANES; k++) {
            long ad = ro + k * va.V + j;
            cpx<R> c[L::NC], d[L::NC];
            L::ld(x + ad, c);
            L::ld(y + ad, d);
#pragma unroll
            for (int q = 0; q < L::NC; q++) d[q] = R(a) * c[q] + R(b) * d[q];
            L::st(y + ad, d);
        }
}

// FP64 -> FP32 with a per-right-hand-side scale: out = in * scale[r]
__global__ void __launch_bounds__(NT) k_to32(long V, long off, long n, long rs64, long rs32, const double2 *in,
                                             float4 *out, const double *scale)
{
    const double sc = scale ? scale[blockIdx.y] : 1.0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < n; j += (long)gridDim.x * NT)
        for (int k = 0; k < 6; k++) {
            double2 a = in[(long)blockIdx.y * rs64 + (2 * k) * V + off + j];
            double2 b = in[(long)blockIdx.y * rs64 + (2 * k + 1) * V + off + j];
            out[(long)blockIdx.y * rs32 + k * V + off + j] =
                make_float4((float)(a.x * sc), (float)(a.y * sc), (float)(b.x * sc), (float)(b.y * sc));
        }
}

// x64 += scale[r] * e32
__global__ void __launch_bounds__(NT) k_add32(long V, long off, long n, long rs64, long rs32, const float4 *e,
                                              double2 *x, const double *scale)
{
    const double sc = scale ? scale[blockIdx.y] : 1.0;
    for (long j = (long)blockIdx.x * NT + threadIdx.x; j < n; j += (long)gridDim.x * NT)
        for (int k = 0; k < 6; k++) {
            float4 v = e[(long)blockIdx.y * rs32 + k * V + off + j];
            double2 *a = x + (long)blockIdx.y * rs64 + (2 * k) * V + off + j;
            double2 *b = x + (long)blockIdx.y * rs64 + (2 * k + 1) * V + off + j;
            double2 av = *a, bv = *b;
            *a = make_double2(av.x + sc * v.x, av.y + sc * v.y);
            *b = make_double2(bv.x + sc * v.z, bv.y + sc * v.w);
        }
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

void to32(ddrw_ctx *ctx, const VecRange &vr, long rs32, const double2 *in, float4 *out, const double *scale)
{
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_to32<<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(vr.V, vr.off, vr.n, vr.rs, rs32, in, out, scale);
}

void add32(ddrw_ctx *ctx, const VecRange &vr, long rs32, const float4 *e, double2 *x, const double *scale)
{
    ProfScope ps(ctx, PROF_BLAS, 0.0);
    ++ctx->launches;
    k_add32<<<dim3(grid_for(vr.n), vr.nrhs), NT, 0, ctx->stream>>>(vr.V, vr.off, vr.n, vr.rs, rs32, e, x, scale);
}

template struct Blas<PrecD>;
template struct Blas<PrecS>;

}  // namespace ddrw
