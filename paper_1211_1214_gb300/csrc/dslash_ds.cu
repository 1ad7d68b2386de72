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
__global__ void k_split(long V, long vh, long off, long len, int par0, int npar, int nrhs, long rs,
                        const double2 *__restrict__ in, float4 *out)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = 12 * npar * len;
    if (i >= per * nrhs) return;
    long r = i / per, e = i - r * per;
    long j = e % len, kp = e / len;
    long idx = r * rs + (kp / npar) * V + (par0 + kp % npar) * vh + off + j;
    double2 v = in[idx];
    float xh = (float)v.x, yh = (float)v.y;
    out[idx] = make_float4(xh, (float)(v.x - (double)xh), yh, (float)(v.y - (double)yh));
}

void split64(ddrw_ctx *ctx, const double2 *in, float4 *out, long V, long vh, long off, long len, int par0, int npar,
             int nrhs, long rs)
{
    long n = 12L * npar * len * nrhs;
    if (n == 0) return;
    ++ctx->launches;
    k_split<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(V, vh, off, len, par0, npar, nrhs, rs, in, out);
}

}  // namespace ddrw
