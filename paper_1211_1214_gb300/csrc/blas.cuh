// blas.cuh -- declarations of the vector kernels and reductions (blas.cu).
#pragma once

#include "../../include/ddrw.h"
#include "ddrw_internal.cuh"

namespace ddrw {

// One 16-byte field element as complex numbers in its arithmetic type (double2: 1, float4: 2).
template <class E> struct El;
template <> struct El<double2> {
    using R = double;
    static constexpr int NC = 1;
    __device__ static __forceinline__ void ld(const double2 *p, cpx<R> *c)
    {
        double2 v = *p;
        c[0] = {v.x, v.y};
    }
    __device__ static __forceinline__ void st(double2 *p, const cpx<R> *c) { *p = make_double2(c[0].re, c[0].im); }
};
template <> struct El<float4> {
    using R = float;
    static constexpr int NC = 2;
    __device__ static __forceinline__ void ld(const float4 *p, cpx<R> *c)
    {
        float4 v = *p;
        c[0] = {v.x, v.y};
        c[1] = {v.z, v.w};
    }
    __device__ static __forceinline__ void st(float4 *p, const cpx<R> *c)
    {
        *p = make_float4(c[0].re, c[0].im, c[1].re, c[1].im);
    }
};

// Krylov scalars of one right-hand side, resident on the device.
struct KScal {
    double2 rho, alpha, omega, beta;
    double rr;      // ||r||^2 of the current iterate
    double thresh;  // stop when rr <= thresh (tol^2 ||b||^2)
    int active;     // 0 once converged, stalled or broken down
    int iters;
    int maxiter;
    int breakdown;  // 0 none, else the step that found a zero denominator or NaN
};

// sites [off, off + n) of every plane (plane stride V), nrhs right-hand sides rs elements apart
struct VecRange {
    long V, off, n, rs;
    int nrhs;
};

template <class P> struct Blas {
    using E = typename P::SElem;
    static ddrw_status bicg_init(ddrw_ctx *ctx, const VecRange &vr, E *r, E *rh, E *p, E *x, KScal *sc);
    static ddrw_status bicg_alpha(ddrw_ctx *ctx, const VecRange &vr, const E *rh, const E *v, KScal *sc);
    static void bicg_s(ddrw_ctx *ctx, const VecRange &vr, E *r, const E *v, const KScal *sc);
    static ddrw_status bicg_omega(ddrw_ctx *ctx, const VecRange &vr, const E *t, const E *r, KScal *sc);
    static ddrw_status bicg_xr(ddrw_ctx *ctx, const VecRange &vr, E *x, const E *p, E *r, const E *t, const E *rh,
                               KScal *sc);
    static void bicg_p(ddrw_ctx *ctx, const VecRange &vr, E *p, const E *r, const E *v, const KScal *sc);
    static ddrw_status norm2(ddrw_ctx *ctx, const VecRange &vr, const E *f, double *out);
    static ddrw_status norm_dot(ddrw_ctx *ctx, const VecRange &vr, const E *d, const E *e, double *out);
    static void axpby(ddrw_ctx *ctx, const VecRange &vr, double a, const E *x, double b, E *y);
};

// FP64 <-> FP32 fields over a range, with a per-right-hand-side scale (may be null)
void to32(ddrw_ctx *ctx, const VecRange &vr, long rs32, const double2 *in, float4 *out, const double *scale);
void add32(ddrw_ctx *ctx, const VecRange &vr, long rs32, const float4 *e, double2 *x, const double *scale);

}  // namespace ddrw
