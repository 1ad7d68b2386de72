// noalloc.cu -- a block solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool is frozen or inside a
// host callback, or a host framework that owns every device allocation and forbids libraries from
// making their own.  ddrw_solve_block_noalloc gives them the block solve x = D_cc(m)^-1 b with all
// of its scratch (the internal copies of b and x, the six Krylov vectors of the persistent block
// solver, the defect-correction residual and correction, the reduction slots) in one file-scope
// device array of fixed size.  The caller still passes b and x.
//
// The array is a host-side stand-in in host code; its device address is looked up on every call,
// with the context's device current, by cudaGetSymbolAddress (cheap, and never stale after a
// device reset).  Every GPU that loads this code holds the array until the process exits.  Every
// call shares the array and leaves its contents from the last call behind; two calls that overlap
// on the GPU (different streams or contexts on one device) race on it.  The call synchronises its
// stream and reads scalars back to the host, so it refuses to run inside a stream capture.
#include <cmath>
#include <vector>

#include "blocksolve.cuh"

namespace ddrw {

// the persistent block-solver kernels are instantiated in bs_d<l>.cu
extern template void launch_block_kernel<PrecD, 2>(ddrw_ctx *, const BlkArgs<PrecD> &, int);
extern template void launch_block_kernel<PrecD, 4>(ddrw_ctx *, const BlkArgs<PrecD> &, int);
extern template void launch_block_kernel<PrecD, 6>(ddrw_ctx *, const BlkArgs<PrecD> &, int);
extern template void launch_block_kernel<PrecD, 8>(ddrw_ctx *, const BlkArgs<PrecD> &, int);

// largest lattice (sites) the scratch array serves: 12^4
constexpr long NOALLOC_MAX_SITES = 20736;
// FP64 spinor fields in the scratch array: b, x, r, rh, p, v, t, tmp, residual, correction
constexpr int NOALLOC_FIELDS = 10;
constexpr long NOALLOC_FIELD_ELEMS = 12 * NOALLOC_MAX_SITES;  // double2 per field
constexpr long NOALLOC_RED_ELEMS = 64;                       // reduction slots (double2)

static __device__ __align__(256) double2 noalloc_scratch[NOALLOC_FIELDS * NOALLOC_FIELD_ELEMS + NOALLOC_RED_ELEMS];

namespace {

// device address of the scratch array on the current device (the context's device is current)
ddrw_status scratch_address(ddrw_ctx *ctx, double2 **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
    if (e != cudaSuccess || !p) return set_cuda_error(ctx, e, "cudaGetSymbolAddress(noalloc_scratch)", __FILE__, __LINE__);
    *out = (double2 *)p;
    return DDRW_OK;
}

// out[0] = sum of |f|^2 over the sites of one colour (both parities), one CTA, fixed order
__global__ void __launch_bounds__(1024) k_colour_norm(const double2 *f, long V, long vh, long lo, long nc, double *out)
{
    __shared__ double sm[32];
    double acc = 0.0;
    for (long j = threadIdx.x; j < 2 * nc; j += 1024) {
        long s = (j < nc) ? lo + j : vh + lo + (j - nc);
        for (int k = 0; k < 12; k++) {
            double2 v = f[(long)k * V + s];
            acc += v.x * v.x + v.y * v.y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 32; i++) s += sm[i];
        out[0] = s;
    }
}

ddrw_status colour_norm(ddrw_ctx *ctx, int colour, const double2 *f, double *dslot, double *host)
{
    long vbh = (long)ctx->l * ctx->l * ctx->l * ctx->l / 2, nc = (long)ctx->nblk_c * vbh;
    ++ctx->launches;
    k_colour_norm<<<1, 1024, 0, ctx->stream>>>(f, ctx->V, ctx->vh, colour * nc, nc, dslot);
    DDRW_CUDA_CHECK(cudaMemcpyAsync(host, dslot, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    DDRW_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    return DDRW_OK;
}

VecRange colour_range_na(const ddrw_ctx *ctx, int colour, int parity)
{
    long vbh = (long)ctx->l * ctx->l * ctx->l * ctx->l / 2, nc = (long)ctx->nblk_c * vbh;
    return VecRange{ctx->V, parity * ctx->vh + colour * nc, nc, 12 * ctx->V, 1};
}

void launch_block_na(ddrw_ctx *ctx, const BlkArgs<PrecD> &a)
{
    switch (ctx->l) {
    case 2: launch_block_kernel<PrecD, 2>(ctx, a, 1); break;
    case 4: launch_block_kernel<PrecD, 4>(ctx, a, 1); break;
    case 6: launch_block_kernel<PrecD, 6>(ctx, a, 1); break;
    default: launch_block_kernel<PrecD, 8>(ctx, a, 1); break;
    }
}

}  // namespace
}  // namespace ddrw

using namespace ddrw;

extern "C" ddrw_status ddrw_solve_block_noalloc(ddrw_ctx *ctx, int colour, double m, const double *b, double *x,
                                                ddrw_solve_info *info)
{
    if (!ctx) return DDRW_EINVAL;
    if (!b || !x || (colour != DDRW_BLACK && colour != DDRW_WHITE)) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    if (ctx->V > NOALLOC_MAX_SITES)
        return set_error(ctx, DDRW_EINVAL, "ddrw_solve_block_noalloc serves lattices of at most 20736 sites (12^4)");
    if (!is_device_ptr(b) || !is_device_ptr(x))
        return set_error(ctx, DDRW_EINVAL, "ddrw_solve_block_noalloc takes device pointers only (no staging buffer)");
    if (m != ctx->m1 && m != ctx->m2)
        return set_error(ctx, DDRW_EINVAL, "ddrw_solve_block_noalloc needs m = m1 or m2 of ddrw_set_params");
    MassInv *mi = nullptr;
    for (auto &e : ctx->inv)
        if (e.m == m) mi = &e;
    if (!mi) return set_error(ctx, DDRW_ESTATE, "the in-block inverse of m1 / m2 is missing (call ddrw_set_params)");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, DDRW_ECUDA, "cudaSetDevice");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return set_error(ctx, DDRW_ESTATE, "ddrw_solve_block_noalloc cannot run inside a stream capture");

    double2 *base;
    ddrw_status st = scratch_address(ctx, &base);
    if (st) return st;
    const long V = ctx->V, fe = 12 * V;
    double2 *F[NOALLOC_FIELDS];
    for (int k = 0; k < NOALLOC_FIELDS; k++) F[k] = base + k * fe;
    double2 *fb = F[0], *fx = F[1], *fres = F[8], *fe64 = F[9];
    double *red = (double *)(base + NOALLOC_FIELDS * NOALLOC_FIELD_ELEMS);
    int *stat = (int *)(red + 8);
    double *h = ctx->h_pinned;

    pack_spinor64(ctx, b, fb, 1);
    DDRW_CUDA_CHECK(cudaMemsetAsync(fx, 0, sizeof(double2) * fe, ctx->stream));
    if ((st = colour_norm(ctx, colour, fb, red, h))) return st;
    const double bb = h[0];
    if (!std::isfinite(bb)) return set_error(ctx, DDRW_ENUMERIC, "non-finite right-hand side");

    BlkArgs<PrecD> a;
    a.r = F[2];
    a.rh = F[3];
    a.p = F[4];
    a.v = F[5];
    a.t = F[6];
    a.tmp = F[7];
    a.rstride = fe;
    a.rpm = 1;
    for (int k = 0; k < MAXM; k++) {
        a.mass4[k] = 4.0 + m;
        a.Ainv[k] = mi->A64;
    }
    a.U = ctx->U64;
    a.Cl = ctx->C64;
    a.blk0 = colour == DDRW_BLACK ? 0 : ctx->nblk_c;
    a.tol2 = 0.25 * ctx->tol_block * ctx->tol_block;
    a.maxiter = ctx->maxiter;
    a.stat = stat;

    double rel = bb > 0 ? 1.0 : 0.0;
    int itmax = 0, itsum = 0, cycles = 0;
    const double2 *rhs = fb;
    while (bb > 0 && cycles < 10) {
        DDRW_CUDA_CHECK(cudaMemsetAsync(stat, 0, sizeof(int) * 2, ctx->stream));
        a.b = rhs;
        a.x = cycles == 0 ? fx : fe64;
        launch_block_na(ctx, a);
        if (cycles > 0)
            for (int p = 0; p < 2; p++) Blas<PrecD>::axpby(ctx, colour_range_na(ctx, colour, p), 1.0, fe64, 1.0, fx);
        // residual b - D_cc x in FP64
        DslashCall c;
        c.in = fx;
        c.x = fx;
        c.out = fres;
        c.rstride = fe;
        c.nrhs = 1;
        c.masses[0] = m;
        c.Ainv[0] = mi->A64;
        c.alpha = -1.0;
        c.beta = 0.5;
        c.diag = 1;
        c.hopsel = 1;
        c.par0 = 0;
        c.npar = 2;
        c.blk0 = a.blk0;
        c.nblk = ctx->nblk_c;
        dslash64(ctx, c);
        for (int p = 0; p < 2; p++) Blas<PrecD>::axpby(ctx, colour_range_na(ctx, colour, p), 1.0, fb, 1.0, fres);
        int hs[2];
        DDRW_CUDA_CHECK(cudaMemcpyAsync(hs, stat, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
        if ((st = colour_norm(ctx, colour, fres, red + 1, h))) return st;
        itmax = std::max(itmax, hs[0]);
        itsum += hs[0];
        cycles++;
        rel = std::sqrt(h[0] / bb);
        if (!(rel == rel)) return set_error(ctx, DDRW_ENUMERIC, "NaN in a block solve");
        if (rel <= ctx->tol_block) break;
        rhs = fres;
    }
    unpack_spinor64(ctx, fx, x, 1);
    if ((st = sync(ctx))) return st;
    if (info) {
        *info = ddrw_solve_info{};
        info->block_iters_max = itmax;
        info->iters_inner_total = itsum;
        info->cycles = cycles;
        info->true_rel_residual = rel;
    }
    return rel <= ctx->tol_block ? DDRW_OK : set_error(ctx, DDRW_ENOCONV, "block solve did not reach its tolerance");
}
