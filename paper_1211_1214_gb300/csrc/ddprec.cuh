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
// Sums of products (link and clover multiplies) use accumulated pairs normalised once per result
// (dd_acc below).
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

// ---- accumulated products.  A sum of products sum_k x_k y_k is kept as an unnormalised pair:
// each product's leading part enters the leading word through a two-sum, its rounding error and
// the two-sum's error collect in the trailing word, and the pair is normalised once at the end
// (12 FP32 operations per product instead of 18 for a normalised product plus a normalised sum).
struct dd_acc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void mac(dd x, dd y)  // += x y
    {
        float p = __fmul_rn(x.hi, y.hi);
        float e = __fmaf_rn(x.hi, y.hi, -p);
        e = __fmaf_rn(x.hi, y.lo, e);
        e = __fmaf_rn(x.lo, y.hi, e);
        float s = __fadd_rn(hi, p);
        float v = __fsub_rn(s, hi);
        float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(t, e));
    }
    __device__ __forceinline__ void msub(dd x, dd y) { mac(x, dd(-y.hi, -y.lo)); }  // -= x y
    __device__ __forceinline__ dd get() const
    {
        float h = __fadd_rn(hi, lo);
        return dd(h, __fsub_rn(lo, __fsub_rn(h, hi)));
    }
};

// w = U h and w = U^dag h on the two spin components of a half spinor, in accumulated form
template <> __device__ __forceinline__ void link_mul<dd>(const Link<dd> &U, const Half<dd> &h, Half<dd> &w)
{
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            dd_acc re, im;
#pragma unroll
            for (int b = 0; b < 3; b++) {
                re.mac(U.m[a][b].re, h.v[s][b].re);
                re.msub(U.m[a][b].im, h.v[s][b].im);
                im.mac(U.m[a][b].re, h.v[s][b].im);
                im.mac(U.m[a][b].im, h.v[s][b].re);
            }
            w.v[s][a] = cpx<dd>{re.get(), im.get()};
        }
}
template <> __device__ __forceinline__ void link_dag_mul<dd>(const Link<dd> &U, const Half<dd> &h, Half<dd> &w)
{
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            dd_acc re, im;
#pragma unroll
            for (int b = 0; b < 3; b++) {  // conj(U[b][a]) h[b]
                re.mac(U.m[b][a].re, h.v[s][b].re);
                re.mac(U.m[b][a].im, h.v[s][b].im);
                im.mac(U.m[b][a].re, h.v[s][b].im);
                im.msub(U.m[b][a].im, h.v[s][b].re);
            }
            w.v[s][a] = cpx<dd>{re.get(), im.get()};
        }
}

// out = (diag + H) v for a packed Hermitian 6x6 H (layout of herm6_mul), in accumulated form
template <> __device__ __forceinline__ void herm6_mul<dd>(const dd *c, dd diag, const cpx<dd> *v, cpx<dd> *out)
{
    dd_acc re[6], im[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const dd d = diag + c[i];
        re[i].mac(d, v[i].re);
        im[i].mac(d, v[i].im);
    }
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            const int o = 6 + 2 * herm_off(i, j);
            const dd hr = c[o], hi = c[o + 1];
            // out_i += h_ij v_j ; out_j += conj(h_ij) v_i
            re[i].mac(hr, v[j].re);
            re[i].msub(hi, v[j].im);
            im[i].mac(hr, v[j].im);
            im[i].mac(hi, v[j].re);
            re[j].mac(hr, v[i].re);
            re[j].mac(hi, v[i].im);
            im[j].mac(hr, v[i].im);
            im[j].msub(hi, v[i].re);
        }
#pragma unroll
    for (int i = 0; i < 6; i++) out[i] = cpx<dd>{re[i].get(), im[i].get()};
}

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
