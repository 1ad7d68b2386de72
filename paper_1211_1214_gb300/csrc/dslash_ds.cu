// double-single instantiations of the stencil (see dslash.cuh and ddprec.cuh): the residual
// stencil of the mixed path's defect correction
#include "dslash.cuh"

namespace ddrw {

// the block lengths are instantiated in dslash_ds<l>.cu, so that they compile in parallel
extern template void launch_bl<PrecDD, 2>(ddrw_ctx *, const DslashCall &);
extern template void launch_bl<PrecDD, 4>(ddrw_ctx *, const DslashCall &);
extern template void launch_bl<PrecDD, 6>(ddrw_ctx *, const DslashCall &);
extern template void launch_bl<PrecDD, 8>(ddrw_ctx *, const DslashCall &);

void dslash_ds(ddrw_ctx *ctx, const DslashCall &c) { launch<PrecDD>(ctx, c); }

// one complex FP64 number (x, y) per element -> (hi(x), lo(x), hi(y), lo(y)).  The elements are
// those of the sites [off, off + len) of parities par0 .. par0 + npar - 1 in the 12 planes of nrhs
// fields (planes V apart, parities vh apart, fields rs apart).
// grid: x over the sites, y over (plane, parity), z over the fields -- no per-element division
__global__ void k_split(long V, long vh, long off, long len, int par0, int npar, long rs,
                        const double2 *__restrict__ in, float4 *out)
{
    const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    const int k = blockIdx.y / npar, p = blockIdx.y - k * npar;
    const long idx = (long)blockIdx.z * rs + (long)k * V + (long)(par0 + p) * vh + off + j;
    double2 v = in[idx];
    float xh = (float)v.x, yh = (float)v.y;
    out[idx] = make_float4(xh, (float)(v.x - (double)xh), yh, (float)(v.y - (double)yh));
}

void split64(ddrw_ctx *ctx, const double2 *in, float4 *out, long V, long vh, long off, long len, int par0, int npar,
             int nrhs, long rs)
{
    if (len <= 0 || npar <= 0 || nrhs <= 0) return;
    ++ctx->launches;
    const dim3 grid((unsigned)((len + 255) / 256), (unsigned)(12 * npar), (unsigned)nrhs);
    k_split<<<grid, 256, 0, ctx->stream>>>(V, vh, off, len, par0, npar, rs, in, out);
}

}  // namespace ddrw
