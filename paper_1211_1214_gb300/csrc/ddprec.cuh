// ddprec.cuh -- double-single ("double-float") arithmetic for the defect-correction residuals of
// the mixed path.
//
// GB300 runs FP64 at about 1/58 of its FP32 rate, so the FP64 stencil of the residual
// r = b - D x costs several FP32 stencils.  Here each real number is an unevaluated sum hi + lo of
// two FP32 numbers (|lo| <= ulp(hi)/2), about 44 significant bits, and the arithmetic uses the
// error-free transformations of Knuth's two-sum and the FMA-based two-product (Dekker's
// double-length arithmetic with a fused multiply-add).  Every operation is written with the
// round-to-nearest intrinsics, which the compiler never contracts or reassociates.
//
// Storage: a "split" field holds one complex number per 16-byte element (re.hi, re.lo, im.hi,
// im.lo), the same bytes as an FP64 field; links (9 complex per direction) and the clover term
// (72 reals per site) are split once per configuration, the stencil input once per residual, and
// the result is written back as FP64 (hi + lo).
#pragma once

#include "ddrw_internal.cuh"

namespace ddrw {

struct dd {
    float hi, lo;
    __host__ __device__ dd() {}
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ dd(double x)
    {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
    __host__ __device__ dd(int x) : dd((double)x) {}
};

// a + b with a two-sum of the leading parts (relative error ~2^-44 of |a| + |b|)
__device__ __forceinline__ dd operator+(dd a, dd b)
{
    float s = __fadd_rn(a.hi, b.hi);
    float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    float h = __fadd_rn(s, e);
    return dd(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
// a * b with an FMA two-product of the leading parts
__device__ __forceinline__ dd operator*(dd a, dd b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float h = __fadd_rn(p, e);
    return dd(h, __fsub_rn(e, __fsub_rn(h, p)));
}
__device__ __forceinline__ bool operator!=(dd a, dd b) { return a.hi != b.hi || a.lo != b.lo; }

// Storage policy of the double-single stencil: split spinors, links and clover in, FP64 out.
struct PrecDD {
    using R = dd;
    using SElem = float4;  // one complex number (re.hi, re.lo, im.hi, im.lo)
    static constexpr int ID = 128;
    static constexpr double SBYTES = 192, UBYTES = 144, CBYTES = 576;
    static constexpr int SPLANES = 12;
    static constexpr int UPLANES = 9;
    static constexpr int CPLANES = 36;
    using UElem = float4;
    using CElem = float4;

    __device__ static __forceinline__ cpx<dd> unpack(float4 v) { return cpx<dd>{dd(v.x, v.y), dd(v.z, v.w)}; }

    __device__ static __forceinline__ void load_spinor(const SElem *__restrict__ f, int stride, int s, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 12; k++) p.v[k / 3][k % 3] = unpack(__ldg(f + (k * stride + s)));
    }
    __device__ static __forceinline__ void load_spinor_rw(const SElem *f, int stride, int s, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 12; k++) p.v[k / 3][k % 3] = unpack(f[k * stride + s]);
    }
    // the output field is FP64 (16-byte double2 elements at the same offsets)
    __device__ static __forceinline__ void store_spinor(SElem *__restrict__ f, int stride, int s, const Spinor<R> &p)
    {
        double2 *o = reinterpret_cast<double2 *>(f);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const cpx<dd> &c = p.v[k / 3][k % 3];
            o[k * stride + s] = make_double2((double)c.re.hi + (double)c.re.lo, (double)c.im.hi + (double)c.im.lo);
        }
    }
    __device__ static __forceinline__ void load_chiral(const SElem *__restrict__ f, int stride, int s, int ch, cpx<R> *v)
    {
#pragma unroll
        for (int k = 0; k < 6; k++) v[k] = unpack(__ldg(f + ((6 * ch + k) * stride + s)));
    }
    __device__ static __forceinline__ void load_link(const UElem *__restrict__ U, int V, int mu, int s, Link<R> &L)
    {
        const UElem *b = U + (long)mu * 9 * V;
#pragma unroll
        for (int k = 0; k < 9; k++) L.m[k / 3][k % 3] = unpack(__ldg(b + (k * V + s)));
    }
    // 36 reals of chirality block ch, stored as 18 elements of two (hi, lo) reals each
    __device__ static __forceinline__ void load_clover(const CElem *__restrict__ Cl, int V, int s, int ch, R *c)
    {
        const CElem *b = Cl + (long)ch * 18 * V;
#pragma unroll
        for (int k = 0; k < 18; k++) {
            float4 v = __ldg(b + (k * V + s));
            c[2 * k] = dd(v.x, v.y);
            c[2 * k + 1] = dd(v.z, v.w);
        }
    }
};

}  // namespace ddrw
