// blas.cuh -- declarations of the vector kernels and reductions (blas.cu).
#pragma once

#include "../../include/ddrw.h"
#include "ddrw_internal.cuh"

namespace ddrw {

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

// FP64 fields <-> storage precision P (FP32, FP16, BF16) over a range, with a per-right-hand-side
// scale (may be null); rsl is the field stride of the P fields
template <class P>
void to_low(ddrw_ctx *ctx, const VecRange &vr, long rsl, const double2 *in, typename P::SElem *out,
            const double *scale);
template <class P>
void add_low(ddrw_ctx *ctx, const VecRange &vr, long rsl, const typename P::SElem *e, double2 *x, const double *scale);
// FP32 link / clover planes -> 16-bit planes of the same order (n float4 elements; bf: BF16, else FP16)
void f32_to_low(ddrw_ctx *ctx, const float4 *in, uint2 *out, long n, bool bf);

}  // namespace ddrw
