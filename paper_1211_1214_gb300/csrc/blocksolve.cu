// blocksolve.cu -- the persistent block solver (K6): x = D_cc(m)^-1 b for every block of one colour
// c in one launch (D_bb and D_ww are block-diagonal, Eq. 1, so the blocks are independent).
//
// One CTA owns one (block, right-hand side) pair and runs the whole Krylov solve inside the kernel:
// in-block even-odd preconditioning S = A_ee - 1/4 H_eo A_oo^-1 H_oe (hops inside the block only),
// BiCGStab on S with CTA-wide reductions (warp shuffles + shared memory, FP64 above the thread),
// then x_o = A_oo^-1 (b_o + 1/2 H_oe x_e).  The block's sites of one parity are contiguous in the
// block-major layout, so every pass is a coalesced sweep over the block.
//
// The host driver wraps the kernel in FP64 defect correction: r = b - D_cc x in FP64, the kernel
// (FP64 or FP32) solves D_cc e = r to a relative tolerance per block, x += e, until
// ||b - D_cc x|| <= tol ||b|| for every right-hand side (norms over the colour).
#include <algorithm>
#include <cmath>
#include <vector>

#include "blocksolve.cuh"
#include "lowprec.cuh"

namespace ddrw {

template <class P, int BL> void launch_block_kernel(ddrw_ctx *ctx, const BlkArgs<P> &a, int nrhs);

// ----------------------------------------------------------------------------- host side

template <class P>
static void launch_block(ddrw_ctx *ctx, const BlkArgs<P> &a, int nrhs)
{
    switch (ctx->l) {
    case 2: launch_block_kernel<P, 2>(ctx, a, nrhs); break;
    case 4: launch_block_kernel<P, 4>(ctx, a, nrhs); break;
    case 6: launch_block_kernel<P, 6>(ctx, a, nrhs); break;
    default: launch_block_kernel<P, 8>(ctx, a, nrhs); break;
    }
}

// colour ranges: sites of colour c and parity p are [p vh + c n_c, p vh + (c + 1) n_c)
static VecRange colour_range(const ddrw_ctx *ctx, int colour, int parity, int nrhs, long rs)
{
    long vbh = (long)ctx->l * ctx->l * ctx->l * ctx->l / 2;
    long nc = (long)ctx->nblk_c * vbh;
    return VecRange{ctx->V, parity * ctx->vh + colour * nc, nc, rs, nrhs};
}

template <class P>
static void fill_args(ddrw_ctx *ctx, BlkArgs<P> &a, const MassSet &ms, int colour)
{
    using R = typename P::R;
    int nm = ms.n < 1 ? 1 : ms.n;
    for (int k = 0; k < MAXM; k++) {
        int kk = k < nm ? k : nm - 1;
        a.mass4[k] = R(4.0 + ms.m[kk]);
        a.Ainv[k] = (const typename P::CElem *)ainv_for(ms.inv[kk], P::ID);
    }
    a.U = (const typename P::UElem *)links_for(ctx, P::ID);
    a.Cl = (const typename P::CElem *)clover_for(ctx, P::ID);
    a.blk0 = colour == DDRW_BLACK ? 0 : ctx->nblk_c;
}

// norms over a colour (both parities) of nrhs FP64 fields -> host
static ddrw_status colour_norms(ddrw_ctx *ctx, int colour, const double2 *f, int nrhs, std::vector<double> &out)
{
    double *d;
    ddrw_status st = workspace(ctx, "blk_norms", sizeof(double) * 2 * nrhs, (void **)&d);
    if (st) return st;
    long rs = 12 * ctx->V;
    for (int p = 0; p < 2; p++) {
        st = Blas<PrecD>::norm2(ctx, colour_range(ctx, colour, p, nrhs, rs), f, d + p * nrhs);
        if (st) return st;
    }
    std::vector<double> h(2 * nrhs);
    DDRW_CUDA_CHECK(cudaMemcpyAsync(h.data(), d, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    DDRW_SYNC(ctx);
    out.resize(nrhs);
    for (int r = 0; r < nrhs; r++) out[r] = h[r] + h[nrhs + r];
    return DDRW_OK;
}

// One inner cycle of the mixed block solve in storage policy P: the colour's sites of rhs, scaled
// by scale_d[r], go to P's storage, the persistent kernel solves them to tol_inner, and the
// solution, scaled back by scale_d[nrhs + r], is added to x (zeroed first on the first cycle).
template <class P>
static ddrw_status low_cycle(ddrw_ctx *ctx, int colour, const MassSet &ms, const double2 *rhs, double2 *x, bool first,
                             int nrhs, void *const *w, const double *scale_d, double tol_inner, int maxiter, int *stat,
                             const double *tol2_dev = nullptr)
{
    using E = typename P::SElem;
    const long rs64 = 12 * ctx->V, rsl = P::field_elems(ctx->V);
    const size_t fl = sizeof(E) * rsl * nrhs;
    void *bl, *el;
    ddrw_status st;
    if (P::ID != 32 && P::ID != 64 && ctx->block_method == 1 && !tol2_dev && ctx->reliable_updates()) {
        // 16-bit Krylov vectors on all blocks of the colour with reliable updates into FP32 fields
        float4 *b32, *x32;
        const size_t f32 = sizeof(float4) * 6 * ctx->V * nrhs;
        if ((st = workspace(ctx, "blkl_b32", f32, (void **)&b32))) return st;
        if ((st = workspace(ctx, "blkl_e32", f32, (void **)&x32))) return st;
        for (int p = 0; p < 2; p++) to_low<PrecS>(ctx, colour_range(ctx, colour, p, nrhs, rs64), 6 * ctx->V, rhs, b32, scale_d);
        int it = 0;
        std::vector<double> th(nrhs, tol_inner * tol_inner);
        if ((st = colour_bicgstab_reliable(ctx, P::ID, ms, b32, x32, nrhs, th, maxiter, &it, colour))) return st;
        int hs[2] = {it, 0};
        DDRW_CUDA_CHECK(cudaMemcpyAsync(stat, hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
        DDRW_SYNC(ctx);  // hs is stack memory
        if (first) zero_colour64(ctx, x, colour, nrhs);
        for (int p = 0; p < 2; p++)
            add_low<PrecS>(ctx, colour_range(ctx, colour, p, nrhs, rs64), 6 * ctx->V, x32, x, scale_d + nrhs);
        return DDRW_OK;
    }
    if ((st = workspace(ctx, "blkl_b", fl, &bl))) return st;
    if ((st = workspace(ctx, "blkl_e", fl, &el))) return st;
    for (int p = 0; p < 2; p++) to_low<P>(ctx, colour_range(ctx, colour, p, nrhs, rs64), rsl, rhs, (E *)bl, scale_d);
    BlkArgs<P> a;
    a.b = (const E *)bl;
    a.x = (E *)el;
    a.r = (E *)w[0]; a.rh = (E *)w[1]; a.p = (E *)w[2];
    a.v = (E *)w[3]; a.t = (E *)w[4]; a.tmp = (E *)w[5];
    a.rstride = rsl;
    a.rpm = (nrhs + std::max(ms.n, 1) - 1) / std::max(ms.n, 1);
    fill_args(ctx, a, ms, colour);
    a.tol2 = tol_inner * tol_inner;
    a.tol2_dev = tol2_dev;
    a.maxiter = maxiter;
    a.stat = stat;
    if (ctx->block_method == 1 && !tol2_dev) {
        // all blocks of the colour as one block-diagonal system in the Krylov-loop BiCGStab
        // (tuned stencil launches, graph-captured loop); per right-hand side the colour's residual
        int it = 0;
        std::vector<double> th(nrhs, tol_inner * tol_inner);
        if ((st = colour_bicgstab(ctx, P::ID, ms, bl, el, nrhs, th, maxiter, &it, colour))) return st;
        int hs[2] = {it, 0};
        DDRW_CUDA_CHECK(cudaMemcpyAsync(stat, hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
        DDRW_SYNC(ctx);  // hs is stack memory
    } else {
        launch_block(ctx, a, nrhs);
    }
    if (first) zero_colour64(ctx, x, colour, nrhs);
    for (int p = 0; p < 2; p++) add_low<P>(ctx, colour_range(ctx, colour, p, nrhs, rs64), rsl, (const E *)el, x, scale_d + nrhs);
    return DDRW_OK;
}

// out = -D_cc(ms) x on the sites of colour c (the stencil part of the residual b - D_cc x)
static DslashCall residual_call(const ddrw_ctx *ctx, const MassSet &ms, int colour, const double2 *x, double2 *out,
                                int nrhs)
{
    DslashCall c;
    c.in = x;
    c.x = x;
    c.out = out;
    c.rstride = 12 * ctx->V;
    c.nrhs = nrhs;
    c.nmass = ms.n;
    for (int k = 0; k < ms.n; k++) {
        c.masses[k] = ms.m[k];
        c.Ainv[k] = ms.inv[k]->A64;
    }
    c.alpha = -1.0;
    c.beta = 0.5;
    c.diag = 1;
    c.hopsel = 1;
    c.par0 = 0;
    c.npar = 2;
    c.blk0 = colour == DDRW_BLACK ? 0 : ctx->nblk_c;
    c.nblk = ctx->nblk_c;
    return c;
}

// ---- device-controlled form (the estimate captured as one graph): the same cycles, with the
// host's decisions taken by a one-thread control kernel on device norms

// mode 0, before the first cycle: inner settings from nr = bb.  mode 1, after a cycle: statistics,
// the continue decision (handle), then the next inner settings from nr = rr.  Norms come per
// parity (2 nrhs values: parity 0 then parity 1).  ctl[0] counts the cycles.
__global__ void k_blk_ctl(int mode, int nrhs, const double *bb2, const double *rr2, double tol, double floor, int mixed,
                          const int *stat, double *scale, double *tol2, int *ctl, DcStats *dc, int slot,
                          cudaGraphConditionalHandle h)
{
    const double *nr2 = mode == 0 ? bb2 : rr2;
    if (mode == 1) {
        const int cyc = ++ctl[0];
        dc->loop_iters[slot] += 1;
        dc->block_cycles += 1;
        dc->fp64_dslash_half += 1;
        dc->block_iters_max = max(dc->block_iters_max, stat[0]);
        dc->block_iters_total += stat[0];
        double worst = 0.0;
        bool nan = false;
        for (int r = 0; r < nrhs; r++) {
            const double b = bb2[r] + bb2[nrhs + r], q = rr2[r] + rr2[nrhs + r];
            if (!isfinite(q)) nan = true;
            else if (b > 0) worst = fmax(worst, sqrt(q / b));
        }
        dc->block_rel_residual = fmax(dc->block_rel_residual, worst);
        unsigned cont = 1;
        if (nan) {
            dc->nan = 1;
            cont = 0;
        } else if (worst <= tol) {
            cont = 0;
        } else if (cyc >= 50 || (!mixed && stat[1] > 0 && cyc >= 4)) {
            dc->noconv = 1;
            cont = 0;
        }
        cudaGraphSetConditional(h, cont);
    } else {
        ctl[0] = 0;
    }
    double need = 1.0;
    for (int r = 0; r < nrhs; r++) {
        const double b = bb2[r] + bb2[nrhs + r], q = nr2[r] + nr2[nrhs + r];
        if (q > 0) need = fmin(need, 0.5 * tol * sqrt(b / q));
        scale[r] = q > 0 ? 1.0 / sqrt(q) : 0.0;
        scale[nrhs + r] = sqrt(q);
    }
    const double ti = mixed ? fmax(floor, fmin(need, 0.5)) : 0.5 * tol;
    *tol2 = ti * ti;
}

__global__ void k_zero_ints(int *p, int n)  // (a kernel node: loop bodies hold kernels only)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

static ddrw_status colour_norms_dev(ddrw_ctx *ctx, int colour, const double2 *f, int nrhs, double *out2)
{
    ddrw_status st;
    for (int p = 0; p < 2; p++)
        if ((st = Blas<PrecD>::norm2(ctx, colour_range(ctx, colour, p, nrhs, 12 * ctx->V), f, out2 + p * nrhs))) return st;
    return DDRW_OK;
}

// device buffers of the controlled form (allocated before a capture)
ddrw_status block_solve_dc_prepare(ddrw_ctx *ctx, int nrhs)
{
    void *p;
    ddrw_status st;
    if ((st = workspace(ctx, "dcb_norms", sizeof(double) * 4 * nrhs, &p))) return st;
    if ((st = workspace(ctx, "dcb_scale", sizeof(double) * 2 * nrhs, &p))) return st;
    if ((st = workspace(ctx, "dcb_ctl", sizeof(double) * 2, &p))) return st;
    if ((st = workspace(ctx, "blk_e64", sizeof(double2) * 12 * ctx->V * nrhs, &p))) return st;
    return DDRW_OK;
}

static ddrw_status block_solve_dc(ddrw_ctx *ctx, int colour, const MassSet &ms, const double2 *b, double2 *x, int nrhs,
                                  double tol, int maxiter, ddrw_prec prec)
{
    const bool mixed = prec != DDRW_FP64;
    const long V = ctx->V, rs64 = 12 * V;
    const size_t f64 = sizeof(double2) * rs64 * nrhs, f32 = sizeof(float4) * 6 * V * nrhs;
    const double floor = prec == DDRW_MIXED_FP32 ? 1e-6 : prec == DDRW_MIXED_FP16 ? 1e-3 : 5e-3;
    ddrw_status st;
    int *stat;
    double2 *res64, *e64;
    double *norms, *scale, *ctlbuf;
    if ((st = workspace(ctx, "blk_stat", sizeof(int) * 2, (void **)&stat))) return st;
    if ((st = workspace(ctx, "blk_res64", f64, (void **)&res64))) return st;
    if ((st = workspace(ctx, "blk_e64", f64, (void **)&e64))) return st;
    if ((st = workspace(ctx, "dcb_norms", sizeof(double) * 4 * nrhs, (void **)&norms))) return st;
    if ((st = workspace(ctx, "dcb_scale", sizeof(double) * 2 * nrhs, (void **)&scale))) return st;
    if ((st = workspace(ctx, "dcb_ctl", sizeof(double) * 2, (void **)&ctlbuf))) return st;
    double *bb2 = norms, *rr2 = norms + 2 * nrhs, *tol2 = ctlbuf;
    int *cyc = (int *)(ctlbuf + 1);
    void *w[6];
    const char *names64[6] = {"blk_r", "blk_rh", "blk_p", "blk_v", "blk_t", "blk_tmp"};
    const char *names32[6] = {"blk32_r", "blk32_rh", "blk32_p", "blk32_v", "blk32_t", "blk32_tmp"};
    for (int k = 0; k < 6; k++)
        if ((st = workspace(ctx, mixed ? names32[k] : names64[k], mixed ? f32 : f64, &w[k]))) return st;

    if ((st = colour_norms_dev(ctx, colour, b, nrhs, bb2))) return st;
    DDRW_CUDA_CHECK(cudaMemcpyAsync(res64, b, f64, cudaMemcpyDeviceToDevice, ctx->stream));
    zero_colour64(ctx, x, colour, nrhs);
    ++ctx->launches;
    k_blk_ctl<<<1, 1, 0, ctx->stream>>>(0, nrhs, bb2, rr2, tol, floor, mixed, stat, scale, tol2, cyc, ctx->dc, 0, 0);
    return capture_while(ctx, (const void *)k_blk_ctl, [&](cudaGraphConditionalHandle h, int slot) -> ddrw_status {
        ddrw_status s2;
        ++ctx->launches;
        k_zero_ints<<<1, 32, 0, ctx->stream>>>(stat, 2);
        if (mixed) {  // the solution is added to x (zeroed above)
            if (prec == DDRW_MIXED_FP32)
                s2 = low_cycle<PrecS>(ctx, colour, ms, res64, x, false, nrhs, w, scale, 1.0, maxiter, stat, tol2);
            else if (prec == DDRW_MIXED_FP16)
                s2 = low_cycle<PrecH>(ctx, colour, ms, res64, x, false, nrhs, w, scale, 1.0, maxiter, stat, tol2);
            else
                s2 = low_cycle<PrecB>(ctx, colour, ms, res64, x, false, nrhs, w, scale, 1.0, maxiter, stat, tol2);
            if (s2) return s2;
        } else {
            BlkArgs<PrecD> a;
            a.b = res64;
            a.x = e64;
            a.r = (double2 *)w[0]; a.rh = (double2 *)w[1]; a.p = (double2 *)w[2];
            a.v = (double2 *)w[3]; a.t = (double2 *)w[4]; a.tmp = (double2 *)w[5];
            a.rstride = rs64;
            a.rpm = (nrhs + std::max(ms.n, 1) - 1) / std::max(ms.n, 1);
            fill_args(ctx, a, ms, colour);
            a.tol2 = 0.0;
            a.tol2_dev = tol2;
            a.maxiter = maxiter;
            a.stat = stat;
            launch_block(ctx, a, nrhs);
            for (int p = 0; p < 2; p++)
                Blas<PrecD>::axpby(ctx, colour_range(ctx, colour, p, nrhs, rs64), 1.0, e64, 1.0, x);
        }
        DslashCall c = residual_call(ctx, ms, colour, x, res64, nrhs);
        if ((s2 = residual_stencil(ctx, c, mixed))) return s2;
        for (int p = 0; p < 2; p++) Blas<PrecD>::axpby(ctx, colour_range(ctx, colour, p, nrhs, rs64), 1.0, b, 1.0, res64);
        if ((s2 = colour_norms_dev(ctx, colour, res64, nrhs, rr2))) return s2;
        ++ctx->launches;
        k_blk_ctl<<<1, 1, 0, ctx->stream>>>(1, nrhs, bb2, rr2, tol, floor, mixed, stat, scale, tol2, cyc, ctx->dc, slot, h);
        return DDRW_OK;
    });
}

// x = D_cc(ms)^-1 b on the sites of colour c (FP64 fields, full-field layout, nrhs rhs).
// Sites of the other colour in x are left untouched.
ddrw_status block_solve64(ddrw_ctx *ctx, int colour, const MassSet &ms, const double2 *b, double2 *x, int nrhs,
                          double tol, int maxiter, ddrw_prec prec, SolveStats *stats)
{
    // under the 16-bit precisions the block solves may run in FP32 instead (ddrw_set_low_precision)
    if ((prec == DDRW_MIXED_FP16 || prec == DDRW_MIXED_BF16) && !ctx->block16) prec = DDRW_MIXED_FP32;
    if (ctx->devctl) return block_solve_dc(ctx, colour, ms, b, x, nrhs, tol, maxiter, prec);
    const bool mixed = prec != DDRW_FP64;
    const long V = ctx->V, rs64 = 12 * V;
    // the inner Krylov vectors: FP64 fields, or the largest low-precision field (FP32)
    const size_t f64 = sizeof(double2) * rs64 * nrhs, f32 = sizeof(float4) * 6 * V * nrhs;
    // deepest relative residual an inner solve is asked for: what its storage reliably reaches
    // (16-bit Krylov-loop block solves with reliable updates reach what FP32 reaches)
    const bool rel16 = prec != DDRW_MIXED_FP32 && ctx->block_method == 1 && ctx->reliable_updates();
    const double floor = (prec == DDRW_MIXED_FP32 || rel16) ? 1e-6 : prec == DDRW_MIXED_FP16 ? 1e-3 : 5e-3;
    ddrw_status st;
    std::vector<double> bb, rr;
    if ((st = colour_norms(ctx, colour, b, nrhs, bb))) return st;
    for (int r = 0; r < nrhs; r++)
        if (!std::isfinite(bb[r])) return set_error(ctx, DDRW_ENUMERIC, "non-finite right-hand side");
    int *stat;
    if ((st = workspace(ctx, "blk_stat", sizeof(int) * 2, (void **)&stat))) return st;
    double2 *res64, *e64 = nullptr;
    if ((st = workspace(ctx, "blk_res64", f64, (void **)&res64))) return st;

    // inner workspaces
    void *w[6];
    const char *names64[6] = {"blk_r", "blk_rh", "blk_p", "blk_v", "blk_t", "blk_tmp"};
    const char *names32[6] = {"blk32_r", "blk32_rh", "blk32_p", "blk32_v", "blk32_t", "blk32_tmp"};
    for (int k = 0; k < 6; k++)
        if ((st = workspace(ctx, mixed ? names32[k] : names64[k], mixed ? f32 : f64, &w[k]))) return st;
    double *scale_d = nullptr;
    if (mixed) {
        if ((st = workspace(ctx, "blk_scale", sizeof(double) * 2 * nrhs, (void **)&scale_d))) return st;
    } else {
        if ((st = workspace(ctx, "blk_e64", f64, (void **)&e64))) return st;
    }
    // tolerance of one inner solve: the target itself in FP64; in low precision what is still
    // missing to reach tol (margin 2, worst right-hand side), but no deeper than the floor
    double tol_inner = mixed ? std::max(tol, floor) : tol * 0.5;
    const double2 *rhs = b;  // first cycle: r = b, x = 0
    bool first = true;
    int cycles = 0;
    std::vector<double> scale(nrhs), unscale(nrhs);
    for (; cycles < 50; cycles++) {
        DDRW_CUDA_CHECK(cudaMemsetAsync(stat, 0, sizeof(int) * 2, ctx->stream));
        if (mixed) {
            const std::vector<double> &nr = first ? bb : rr;
            double need = 1.0;
            for (int r = 0; r < nrhs; r++)
                if (nr[r] > 0) need = std::min(need, 0.5 * tol * std::sqrt(bb[r] / nr[r]));
            tol_inner = std::max(floor, std::min(need, 0.5));
            for (int r = 0; r < nrhs; r++) {
                double n = std::sqrt(nr[r]);
                scale[r] = n > 0 ? 1.0 / n : 0.0;
                unscale[r] = n;
            }
            DDRW_CUDA_CHECK(cudaMemcpyAsync(scale_d, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
            DDRW_CUDA_CHECK(cudaMemcpyAsync(scale_d + nrhs, unscale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice,
                                            ctx->stream));
            if (prec == DDRW_MIXED_FP32)
                st = low_cycle<PrecS>(ctx, colour, ms, rhs, x, first, nrhs, w, scale_d, tol_inner, maxiter, stat);
            else if (prec == DDRW_MIXED_FP16)
                st = low_cycle<PrecH>(ctx, colour, ms, rhs, x, first, nrhs, w, scale_d, tol_inner, maxiter, stat);
            else
                st = low_cycle<PrecB>(ctx, colour, ms, rhs, x, first, nrhs, w, scale_d, tol_inner, maxiter, stat);
            if (st) return st;
        } else {
            BlkArgs<PrecD> a;
            a.b = rhs;
            a.x = first ? x : e64;
            a.r = (double2 *)w[0]; a.rh = (double2 *)w[1]; a.p = (double2 *)w[2];
            a.v = (double2 *)w[3]; a.t = (double2 *)w[4]; a.tmp = (double2 *)w[5];
            a.rstride = rs64;
            a.rpm = (nrhs + std::max(ms.n, 1) - 1) / std::max(ms.n, 1);
            fill_args(ctx, a, ms, colour);
            a.tol2 = tol_inner * tol_inner;
            a.maxiter = maxiter;
            a.stat = stat;
            launch_block(ctx, a, nrhs);
            if (!first)
                for (int p = 0; p < 2; p++)
                    Blas<PrecD>::axpby(ctx, colour_range(ctx, colour, p, nrhs, rs64), 1.0, e64, 1.0, x);
        }
        int hstat[2];
        DDRW_CUDA_CHECK(cudaMemcpyAsync(hstat, stat, sizeof(hstat), cudaMemcpyDeviceToHost, ctx->stream));
        // true residual res = b - D_cc x in FP64
        DslashCall c = residual_call(ctx, ms, colour, x, res64, nrhs);
        if ((st = residual_stencil(ctx, c, mixed))) return st;
        if (stats) stats->fp64_dslash_half += 1;
        for (int p = 0; p < 2; p++) Blas<PrecD>::axpby(ctx, colour_range(ctx, colour, p, nrhs, rs64), 1.0, b, 1.0, res64);
        if ((st = colour_norms(ctx, colour, res64, nrhs, rr))) return st;
        if (stats) {
            stats->block_iters_max = std::max(stats->block_iters_max, hstat[0]);
            stats->block_iters_total += hstat[0];
            stats->block_cycles += 1;
        }
        double worst = 0;
        for (int r = 0; r < nrhs; r++)
            if (!std::isfinite(rr[r])) worst = NAN;
            else if (bb[r] > 0 && !(worst != worst)) worst = std::max(worst, std::sqrt(rr[r] / bb[r]));
        if (stats) stats->block_rel_residual = std::max(stats->block_rel_residual, worst);
        if (!(worst == worst)) return set_error(ctx, DDRW_ENUMERIC, "NaN in a block solve");
        if (worst <= tol) return DDRW_OK;
        rhs = res64;
        first = false;
        if (!mixed && hstat[1] > 0 && cycles >= 3) break;
    }
    return set_error(ctx, DDRW_ENOCONV, "block solve did not reach its tolerance");
}

}  // namespace ddrw
