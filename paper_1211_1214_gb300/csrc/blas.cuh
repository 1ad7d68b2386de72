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

// ----------------------------------------------------------------------------- reductions
// (deterministic grid-wide sums shared by the vector kernels of blas.cu and sap.cu)

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

// alpha (mode 1) or omega (mode 2) of the BiCGStab recurrence from the per-warp partial sums of a
// fused stencil epilogue (DslashCall::red), nwt partials of 3 doubles per right-hand side
void bicg_fin(ddrw_ctx *ctx, int mode, int nrhs, const double *part, long nwt, KScal *sc);

// partial-sum and ticket buffers of grid_sum for nrhs right-hand sides (at most 608 CTAs per
// right-hand side and 4 doubles per CTA)
ddrw_status reduce_ws(ddrw_ctx *ctx, int nrhs, double **part, unsigned **ticket);

// FP64 fields <-> storage precision P (FP32, FP16, BF16) over a range, with a per-right-hand-side
// scale (may be null); rsl is the field stride of the P fields
template <class P>
void to_low(ddrw_ctx *ctx, const VecRange &vr, long rsl, const double2 *in, typename P::SElem *out,
            const double *scale);
template <class P>
void add_low(ddrw_ctx *ctx, const VecRange &vr, long rsl, const typename P::SElem *e, double2 *x, const double *scale);
// FP32 field (stride vr.rs) -> 16-bit field (stride rs16) over the range; and x32 += x16, x16 = 0
template <class P16>
void f32_to_16(ddrw_ctx *ctx, const VecRange &vr, long rs16, const float4 *in, typename P16::SElem *out);
template <class P16>
void fold_16_into_32(ddrw_ctx *ctx, const VecRange &vr, long rs16, typename P16::SElem *x16, float4 *x32);
// FP32 link / clover planes -> 16-bit planes of the same order (n float4 elements; bf: BF16, else FP16)
void f32_to_low(ddrw_ctx *ctx, const float4 *in, uint2 *out, long n, bool bf);

}  // namespace ddrw
