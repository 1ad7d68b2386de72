// lowprec.cuh -- 16-bit storage policies (FP16 and BF16) with FP32 arithmetic, for the inner solves
// of the mixed precisions DDRW_MIXED_FP16 / DDRW_MIXED_BF16.
//
// Spinor field: three planes of 16-byte elements (8 sixteen-bit numbers = 4 complex components,
// plane k holding spin-colour components 4k .. 4k+3) followed by one plane of per-site FP32 norms:
// a site's 24 reals are stored divided by their largest magnitude, which is the norm.  FP16's
// range (6e-5 .. 6.5e4 normal) would otherwise lose the small components of unit-norm Krylov
// vectors on large lattices; BF16 shares FP32's range but keeps the same layout.  A field occupies
// 3 V + V/4 elements (V is a multiple of 16).
//
// Links: the two stored rows of U_mu(x) as three 8-byte elements per direction (2 complex each),
// plane layout [mu][3][V]; row 2 is rebuilt as conj(row0 x row1).  Clover terms and in-block
// inverses: two packed Hermitian 6x6 blocks, 9 eight-byte elements (4 reals each) per chirality,
// layout [ch][9][V].  Link entries are bounded by 1 and clover entries by a few units, so they need
// no norm.  The 16-bit link and clover planes are converted from the FP32 ones (same plane
// order, each float4 becoming four 16-bit numbers).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "ddrw_internal.cuh"

namespace ddrw {

// two floats <-> one 32-bit word holding two 16-bit numbers (round to nearest even)
template <bool BF> struct Pack16;
template <> struct Pack16<false> {
    __device__ static __forceinline__ float2 unpack(uint32_t w)
    {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    __device__ static __forceinline__ uint32_t pack(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};
template <> struct Pack16<true> {
    __device__ static __forceinline__ float2 unpack(uint32_t w)
    {
        __nv_bfloat162 h;
        memcpy(&h, &w, 4);
        return __bfloat1622float2(h);
    }
    __device__ static __forceinline__ uint32_t pack(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};

template <bool BF> struct PrecLow {
    using R = float;
    using SElem = uint4;
    using UElem = uint2;
    using CElem = uint2;
    using K = Pack16<BF>;
    static constexpr int ID = BF ? 17 : 16;
    static constexpr int SPLANES = 3;  // + the norm plane
    static constexpr int UPLANES = 3;
    static constexpr int CPLANES = 18;
    static constexpr double SBYTES = 52, UBYTES = 24, CBYTES = 144;
    static constexpr int NCHUNK = 1, CW = 12;  // BLAS granularity: the whole site (one norm)
    // the hop code keeps a neighbour's norm apart and applies it in the FMAs that add the hop
    static constexpr bool NORMED = true;
    __host__ __device__ static long field_elems(long V) { return 3 * V + V / 4; }

    __device__ static __forceinline__ cpx<R> cx(uint32_t w, float n)
    {
        float2 f = K::unpack(w);
        return {f.x * n, f.y * n};
    }
    template <bool RO, typename I>
    __device__ static __forceinline__ void load_all(const SElem *f, I stride, I s, cpx<R> *c)
    {
        const float *nrm = reinterpret_cast<const float *>(f + 3 * stride);
        const float n = RO ? __ldg(nrm + s) : nrm[s];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint4 e = RO ? __ldg(f + (k * stride + s)) : f[k * stride + s];
            c[4 * k] = cx(e.x, n);
            c[4 * k + 1] = cx(e.y, n);
            c[4 * k + 2] = cx(e.z, n);
            c[4 * k + 3] = cx(e.w, n);
        }
    }
    template <typename I> __device__ static __forceinline__ void store_all(SElem *f, I stride, I s, const cpx<R> *c)
    {
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < 12; i++) m = fmaxf(m, fmaxf(fabsf(c[i].re), fabsf(c[i].im)));
        const float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint4 e;
            e.x = K::pack(c[4 * k].re * inv, c[4 * k].im * inv);
            e.y = K::pack(c[4 * k + 1].re * inv, c[4 * k + 1].im * inv);
            e.z = K::pack(c[4 * k + 2].re * inv, c[4 * k + 2].im * inv);
            e.w = K::pack(c[4 * k + 3].re * inv, c[4 * k + 3].im * inv);
            f[k * stride + s] = e;
        }
        reinterpret_cast<float *>(f + 3 * stride)[s] = m;
    }

    __device__ static __forceinline__ void load_spinor(const SElem *__restrict__ f, int stride, int s, Spinor<R> &p)
    {
        cpx<R> c[12];
        load_all<true>(f, stride, s, c);
#pragma unroll
        for (int i = 0; i < 12; i++) p.v[i / 3][i % 3] = c[i];
    }
    // the stored (normalised) components and the site's norm n: the spinor is n p
    __device__ static __forceinline__ void load_spinor_unscaled(const SElem *__restrict__ f, int stride, int s,
                                                                Spinor<R> &p, R &n)
    {
        n = __ldg(reinterpret_cast<const float *>(f + 3 * stride) + s);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint4 e = __ldg(f + (k * stride + s));
            const uint32_t w[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float2 u = K::unpack(w[q]);
                p.v[(4 * k + q) / 3][(4 * k + q) % 3] = {u.x, u.y};
            }
        }
    }
    __device__ static __forceinline__ void load_spinor_rw(const SElem *f, int stride, int s, Spinor<R> &p)
    {
        cpx<R> c[12];
        load_all<false>(f, stride, s, c);
#pragma unroll
        for (int i = 0; i < 12; i++) p.v[i / 3][i % 3] = c[i];
    }
    __device__ static __forceinline__ void store_spinor(SElem *__restrict__ f, int stride, int s, const Spinor<R> &p)
    {
        cpx<R> c[12];
#pragma unroll
        for (int i = 0; i < 12; i++) c[i] = p.v[i / 3][i % 3];
        store_all(f, stride, s, c);
    }
    // components 6ch .. 6ch+5 (spins 2ch, 2ch+1) sit in elements ch and ch+1, words 2ch .. 2ch+5
    __device__ static __forceinline__ void load_chiral(const SElem *__restrict__ f, int stride, int s, int ch, cpx<R> *v)
    {
        const float n = __ldg(reinterpret_cast<const float *>(f + 3 * stride) + s);
        uint4 e0 = __ldg(f + (ch * stride + s)), e1 = __ldg(f + ((ch + 1) * stride + s));
        const uint32_t w[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
        for (int i = 0; i < 6; i++) v[i] = cx(w[2 * ch + i], n);
    }
    __device__ static __forceinline__ void load_link(const UElem *__restrict__ U, int V, int mu, int s, Link<R> &L)
    {
        const UElem *b = U + (long)mu * 3 * V;
        uint2 a0 = __ldg(b + s), a1 = __ldg(b + (V + s)), a2 = __ldg(b + (2 * V + s));
        L.m[0][0] = cx(a0.x, 1.f);
        L.m[0][1] = cx(a0.y, 1.f);
        L.m[0][2] = cx(a1.x, 1.f);
        L.m[1][0] = cx(a1.y, 1.f);
        L.m[1][1] = cx(a2.x, 1.f);
        L.m[1][2] = cx(a2.y, 1.f);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            int i = (c + 1) % 3, j = (c + 2) % 3;
            cpx<R> t = cmul(L.m[0][i], L.m[1][j]);
            cmsub(t, L.m[0][j], L.m[1][i]);
            L.m[2][c] = {t.re, -t.im};
        }
    }
    __device__ static __forceinline__ void load_clover(const CElem *__restrict__ Cl, int V, int s, int ch, R *c)
    {
        const CElem *b = Cl + (long)ch * 9 * V;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            uint2 v = __ldg(b + (k * V + s));
            float2 lo = K::unpack(v.x), hi = K::unpack(v.y);
            c[4 * k] = lo.x;
            c[4 * k + 1] = lo.y;
            c[4 * k + 2] = hi.x;
            c[4 * k + 3] = hi.y;
        }
    }
    struct SRaw {
        uint4 e[3];
        float n;
    };
    struct URaw {
        uint2 e[3];
    };
    __device__ static __forceinline__ void load_raw(const SElem *__restrict__ f, int stride, int s, SRaw &r)
    {
        r.n = __ldg(reinterpret_cast<const float *>(f + 3 * stride) + s);
#pragma unroll
        for (int k = 0; k < 3; k++) r.e[k] = __ldg(f + (k * stride + s));
    }
    __device__ static __forceinline__ void decode_unscaled(const SRaw &r, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint32_t w[4] = {r.e[k].x, r.e[k].y, r.e[k].z, r.e[k].w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float2 u = K::unpack(w[q]);
                p.v[(4 * k + q) / 3][(4 * k + q) % 3] = {u.x, u.y};
            }
        }
    }
    __device__ static __forceinline__ void decode(const SRaw &r, Spinor<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            p.v[(4 * k) / 3][(4 * k) % 3] = cx(r.e[k].x, r.n);
            p.v[(4 * k + 1) / 3][(4 * k + 1) % 3] = cx(r.e[k].y, r.n);
            p.v[(4 * k + 2) / 3][(4 * k + 2) % 3] = cx(r.e[k].z, r.n);
            p.v[(4 * k + 3) / 3][(4 * k + 3) % 3] = cx(r.e[k].w, r.n);
        }
    }
    __device__ static __forceinline__ void load_link_raw(const UElem *__restrict__ U, int V, int mu, int s, URaw &r)
    {
        const UElem *b = U + (long)mu * 3 * V;
        r.e[0] = __ldg(b + s);
        r.e[1] = __ldg(b + (V + s));
        r.e[2] = __ldg(b + (2 * V + s));
    }
    __device__ static __forceinline__ void decode_link(const URaw &r, Link<R> &L)
    {
        L.m[0][0] = cx(r.e[0].x, 1.f);
        L.m[0][1] = cx(r.e[0].y, 1.f);
        L.m[0][2] = cx(r.e[1].x, 1.f);
        L.m[1][0] = cx(r.e[1].y, 1.f);
        L.m[1][1] = cx(r.e[2].x, 1.f);
        L.m[1][2] = cx(r.e[2].y, 1.f);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            int i = (c + 1) % 3, j = (c + 2) % 3;
            cpx<R> t = cmul(L.m[0][i], L.m[1][j]);
            cmsub(t, L.m[0][j], L.m[1][i]);
            L.m[2][c] = {t.re, -t.im};
        }
    }
    // BLAS access: the whole site as one chunk
    __device__ static __forceinline__ void ld_chunk(const SElem *f, long V, long s, int, cpx<R> *c)
    {
        load_all<false>(f, V, s, c);
    }
    __device__ static __forceinline__ void st_chunk(SElem *f, long V, long s, int, const cpx<R> *c)
    {
        store_all(f, V, s, c);
    }
};

using PrecH = PrecLow<false>;
using PrecB = PrecLow<true>;

}  // namespace ddrw
