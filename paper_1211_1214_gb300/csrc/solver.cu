// solver.cu -- the full-lattice Krylov solver (K8): x = D(m)^-1 b, used for the inverse of the
// Schur complement through Dhat^-1 = 1 - P Dcal_bw D_wb (Sec. 1: one Dirac inversion per estimate).
//
//   even-odd reduction:  Mhat = A_ee - 1/4 H_eo A_oo^-1 H_oe,  btil_e = b_e + 1/2 H_eo A_oo^-1 b_o,
//                        x_o = A_oo^-1 (b_o + 1/2 H_oe x_e)
//   Krylov method:       BiCGStab on Mhat x_e = btil_e, all right-hand sides in lockstep with their
//                        own scalars (device resident); a right-hand side that has converged stops
//                        updating while the others continue.
//   graphs:              after the first iterations (which tune the launches) the rest of the loop
//                        is one CUDA graph: a conditional while-node whose condition kernel stops on
//                        convergence of every right-hand side or at the iteration cap.
//   precision:           FP64 defect correction around the inner solve:
//                        r = b - D x (FP64 or double-single stencil), inner solve D e = r / ||r|| in
//                        FP64 (FP64 path), FP32, or 16-bit storage with reliable updates into FP32
//                        (mixed paths), x += ||r|| e, until ||b - D x|| <= tol ||b||.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "blas.cuh"
#include "ctx.h"
#include "lowprec.cuh"

namespace ddrw {

ddrw_status make_massset(ddrw_ctx *ctx, int n, const double *m, MassSet *ms)
{
    if (n < 1 || n > MAXM) return set_error(ctx, DDRW_EINVAL, "1 to 8 masses per call");
    ms->n = n;
    for (int k = 0; k < n; k++) {
        ms->m[k] = m[k];
        ddrw_status st = mass_inverse(ctx, m[k], &ms->inv[k]);
        if (st) return st;
    }
    return DDRW_OK;
}

namespace {

// sets the while-condition of the captured Krylov loop: continue while any right-hand side is
// active and the iteration cap is not reached (the cap bounds every device-side loop)
__global__ void k_bicg_cond(cudaGraphConditionalHandle h, const KScal *sc, int nrhs, int *count, int step, int maxiter)
{
    int act = 0;
    for (int r = 0; r < nrhs; r++) act |= sc[r].active;
    int it = (*count += step);
    cudaGraphSetConditional(h, (act && it < maxiter) ? 1u : 0u);
}

// sets the while-condition of a captured 16-bit Krylov loop with reliable updates: continue while no
// right-hand side of the pass (act0) has stopped or fallen below delta2 times its residual at the
// last reliable update, and the iteration cap is not reached
__global__ void k_rel_cond(cudaGraphConditionalHandle h, const KScal *sc, const double *rr_ref, const int *act0,
                           int nrhs, int *count, int step, int maxiter, double delta2)
{
    int any = 0, trig = 0;
    for (int r = 0; r < nrhs; r++) {
        if (!act0[r]) continue;
        any = 1;
        if (!sc[r].active || sc[r].rr < delta2 * rr_ref[r]) trig = 1;
    }
    int it = (*count += step);
    cudaGraphSetConditional(h, (any && !trig && it < maxiter) ? 1u : 0u);
}

using LoopKey = std::array<uintptr_t, 13 + 2 * MAXM>;

// The graph of a device-controlled Krylov loop: a conditional while-node whose body is `check`
// iterations followed by the condition kernel (cond launches it with the node's handle); built on
// first use of the key, then taken from ctx->graphs.
static ddrw_status loop_graph(ddrw_ctx *ctx, const LoopKey &key, int check,
                              const std::function<ddrw_status()> &iteration,
                              const std::function<void(cudaGraphConditionalHandle)> &cond, cudaGraphExec_t *out)
{
    auto git = ctx->graphs.find(key);
    if (git != ctx->graphs.end()) {
        *out = git->second.exec;
        return DDRW_OK;
    }
    cudaGraph_t graph = nullptr;
    DDRW_CUDA_CHECK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    DDRW_CUDA_CHECK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    DDRW_CUDA_CHECK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    DDRW_CUDA_CHECK(cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ddrw_status cap = DDRW_OK;
    for (int k = 0; k < check && !cap; k++) cap = iteration();
    ++ctx->launches;
    cond(handle);
    cudaGraph_t captured = nullptr;
    cudaError_t ec = cudaStreamEndCapture(ctx->stream, &captured);
    if (cap || ec != cudaSuccess) {
        cudaGraphDestroy(graph);
        if (cap) return cap;
        return set_cuda_error(ctx, ec, "cudaStreamEndCapture", __FILE__, __LINE__);
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_cuda_error(ctx, ei, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
    ctx->graphs[key] = GraphEntry{graph, exec};
    *out = exec;
    return DDRW_OK;
}

template <class P> void stencil(ddrw_ctx *ctx, const DslashCall &c)
{
    switch (P::ID) {
    case 64: dslash64(ctx, c); break;
    case 32: dslash32(ctx, c); break;
    case 16: dslash16(ctx, c); break;
    default: dslashb16(ctx, c); break;
    }
}

// colour < 0: the whole lattice (all hops); colour 0 / 1: the blocks of that colour with the hops
// inside the blocks only (the block operator D_bb / D_ww of Eq. 1)
template <class P> DslashCall base_call(const ddrw_ctx *ctx, const MassSet &ms, int nrhs, long rs, int colour = -1)
{
    DslashCall c;
    c.rstride = rs;
    c.nrhs = nrhs;
    c.nmass = ms.n;
    for (int k = 0; k < ms.n; k++) {
        c.masses[k] = ms.m[k];
        c.Ainv[k] = ainv_for(ms.inv[k], P::ID);
    }
    c.blk0 = colour < 0 ? 0 : colour * ctx->nblk_c;
    c.nblk = colour < 0 ? ctx->nblk : ctx->nblk_c;
    c.hopsel = colour < 0 ? 0 : 1;
    c.npar = 1;
    return c;
}

// out_e = Mhat in_e  (tmp on odd sites)
template <class P>
void apply_mhat(ddrw_ctx *ctx, const MassSet &ms, int nrhs, long rs, const typename P::SElem *in,
                typename P::SElem *tmp, typename P::SElem *out, int colour = -1, int red = 0,
                const typename P::SElem *w = nullptr, double *part = nullptr)
{
    DslashCall c = base_call<P>(ctx, ms, nrhs, rs, colour);
    c.in = in;
    c.out = tmp;
    c.beta = 1.0;
    c.post = 1;
    c.par0 = 1;
    stencil<P>(ctx, c);
    DslashCall d = base_call<P>(ctx, ms, nrhs, rs, colour);
    d.in = tmp;
    d.x = in;
    d.out = out;
    d.alpha = 1.0;
    d.beta = -0.25;
    d.diag = 1;
    d.par0 = 0;
    d.red = red;  // fused inner products of the output (1: with w, 2: with the input, and its norm)
    d.w = w;
    d.red_part = part;
    stencil<P>(ctx, d);
}

// One BiCGStab iteration on the even-odd operator for nrhs right-hand sides (scalars on the device)
template <class P>
static ddrw_status bicg_iteration(ddrw_ctx *ctx, const MassSet &ms, int nrhs, long rs, const VecRange &ev,
                                  typename P::SElem *x, typename P::SElem *r, typename P::SElem *rh,
                                  typename P::SElem *p, typename P::SElem *v, typename P::SElem *t,
                                  typename P::SElem *tmp, KScal *sc, int colour = -1)
{
    ddrw_status s2;
    if (P::ID == 32 && colour < 0 && ctx->fuse_dots && ctx->vh % 256 == 0) {
        // the inner products of alpha and omega in the epilogue of the stencil that writes v and t
        const long nwt = ctx->vh / 32;
        double *part;
        if ((s2 = workspace(ctx, "eo_redpart", sizeof(double) * 3 * (size_t)nwt * nrhs, (void **)&part))) return s2;
        apply_mhat<P>(ctx, ms, nrhs, rs, p, tmp, v, colour, 1, rh, part);
        bicg_fin(ctx, 1, nrhs, part, nwt, sc);
        Blas<P>::bicg_s(ctx, ev, r, v, sc);
        apply_mhat<P>(ctx, ms, nrhs, rs, r, tmp, t, colour, 2, nullptr, part);
        bicg_fin(ctx, 2, nrhs, part, nwt, sc);
    } else {
        apply_mhat<P>(ctx, ms, nrhs, rs, p, tmp, v, colour);
        if ((s2 = Blas<P>::bicg_alpha(ctx, ev, rh, v, sc))) return s2;
        Blas<P>::bicg_s(ctx, ev, r, v, sc);
        apply_mhat<P>(ctx, ms, nrhs, rs, r, tmp, t, colour);
        if ((s2 = Blas<P>::bicg_omega(ctx, ev, t, r, sc))) return s2;
    }
    if ((s2 = Blas<P>::bicg_xr(ctx, ev, x, p, r, t, rh, sc))) return s2;
    Blas<P>::bicg_p(ctx, ev, p, r, v, sc);
    return DDRW_OK;
}

// Inner even-odd BiCGStab in policy P: solve D x = b (full fields) until the even-odd residual of
// right-hand side r satisfies ||r||^2 <= thresh[r].  Adds iterations to *iters.  With colour 0 or
// 1 it solves the block operator D_cc of that colour instead (all its blocks as one block-diagonal
// system, hops inside the blocks only): only the sites of that colour are read and written.
template <class P>
ddrw_status eo_bicgstab(ddrw_ctx *ctx, const MassSet &ms, const typename P::SElem *b, typename P::SElem *x, int nrhs,
                        const std::vector<double> &thresh, int maxiter, int *iters, int colour = -1)
{
    using E = typename P::SElem;
    const long rs = P::field_elems(ctx->V);
    const size_t fb = sizeof(E) * rs * nrhs;
    const char *names[6] = {"eo_r", "eo_rh", "eo_p", "eo_v", "eo_t", "eo_tmp"};
    void *w[6];
    ddrw_status st;
    for (int k = 0; k < 6; k++) {
        char nm[32];
        snprintf(nm, sizeof nm, "%s%d", names[k], P::ID);
        if ((st = workspace(ctx, nm, fb, &w[k]))) return st;
    }
    E *r = (E *)w[0], *rh = (E *)w[1], *p = (E *)w[2], *v = (E *)w[3], *t = (E *)w[4], *tmp = (E *)w[5];
    KScal *sc;
    if ((st = workspace(ctx, "eo_kscal", sizeof(KScal) * nrhs, (void **)&sc))) return st;

    // btil_e = b_e + 1/2 H_eo A_oo^-1 b_o  (into r)
    DslashCall c = base_call<P>(ctx, ms, nrhs, rs, colour);
    c.x = b;
    c.out = tmp;
    c.alpha = 1.0;
    c.diag = 2;
    c.post = 1;
    c.par0 = 1;
    stencil<P>(ctx, c);
    DslashCall d = base_call<P>(ctx, ms, nrhs, rs, colour);
    d.in = tmp;
    d.x = b;
    d.out = r;
    d.alpha = 1.0;
    d.beta = 0.5;
    d.diag = 2;
    d.par0 = 0;
    stencil<P>(ctx, d);

    std::vector<KScal> h(nrhs);
    for (int k = 0; k < nrhs; k++) {
        h[k] = KScal{};
        h[k].thresh = thresh[k];
        h[k].maxiter = maxiter;
    }
    DDRW_CUDA_CHECK(cudaMemcpyAsync(sc, h.data(), sizeof(KScal) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
    const long nc = (long)ctx->nblk_c * (ctx->vh / ctx->nblk);  // sites of one colour and parity
    VecRange ev = colour < 0 ? VecRange{ctx->V, 0, ctx->vh, rs, nrhs} : VecRange{ctx->V, colour * nc, nc, rs, nrhs};
    if ((st = Blas<P>::bicg_init(ctx, ev, r, rh, p, x, sc))) return st;

    KScal *hs = (KScal *)ctx->h_pinned;
    const int check = sizeof(typename P::R) == 8 ? 1 : 4;
    auto iteration = [&]() -> ddrw_status { return bicg_iteration<P>(ctx, ms, nrhs, rs, ev, x, r, rh, p, v, t, tmp, sc, colour); };
    int it = 0;
    bool done = false;
    // first iterations eagerly: they tune the stencil launches and create every workspace
    for (int k = 0; k < check; k++, it++)
        if ((st = iteration())) return st;
    DDRW_CUDA_CHECK(cudaMemcpyAsync(hs, sc, sizeof(KScal) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    DDRW_SYNC(ctx);
    {
        int active = 0;
        for (int k = 0; k < nrhs; k++) active += hs[k].active;
        done = !active || it >= maxiter;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    if (!done && ctx->use_graphs && cs == cudaStreamCaptureStatusNone) {
        // the rest of the loop as one CUDA graph: a conditional while-node around `check`
        // iterations and the condition kernel; no host round trip until convergence or the cap
        int *count;
        if ((st = workspace(ctx, "eo_graph_count", sizeof(int), (void **)&count))) return st;
        LoopKey key{};
        key[0] = P::ID + 1000 * (colour + 1);  // the colour selects other launches
        key[1] = (uintptr_t)nrhs;
        key[2] = (uintptr_t)maxiter;
        const void *ptrs[9] = {r, rh, p, v, t, tmp, x, sc, count};
        for (int k = 0; k < 9; k++) key[3 + k] = (uintptr_t)ptrs[k];
        key[12] = (uintptr_t)ms.n;
        // masses and the device arrays of their inverses are baked into the captured launches
        for (int k = 0; k < ms.n; k++) {  // at most MAXM slots (make_massset)
            double mk = ms.m[k];
            memcpy(&key[13 + 2 * k], &mk, sizeof(double));
            key[14 + 2 * k] = (uintptr_t)ainv_for(ms.inv[k], P::ID);
        }
        cudaGraphExec_t exec = nullptr;
        if ((st = loop_graph(ctx, key, check, iteration, [&](cudaGraphConditionalHandle h) {
                 k_bicg_cond<<<1, 1, 0, ctx->stream>>>(h, sc, nrhs, count, check, maxiter);
             }, &exec)))
            return st;
        const int it0 = it;
        DDRW_CUDA_CHECK(cudaMemcpyAsync(count, &it, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        DDRW_CUDA_CHECK(cudaGraphLaunch(exec, ctx->stream));
        ++ctx->graph_launches;
        DDRW_CUDA_CHECK(cudaMemcpyAsync(&it, count, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        DDRW_CUDA_CHECK(cudaMemcpyAsync(hs, sc, sizeof(KScal) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
        DDRW_SYNC(ctx);
        // kernels the graph ran: 9 per iteration (4 stencil sweeps, 5 vector kernels) and one
        // condition kernel per `check` iterations
        ctx->launches += (long)(it - it0) * 9 + (it - it0) / check;
    } else {
        while (!done) {
            for (int k = 0; k < check; k++, it++)
                if ((st = iteration())) return st;
            DDRW_CUDA_CHECK(cudaMemcpyAsync(hs, sc, sizeof(KScal) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
            DDRW_SYNC(ctx);
            int active = 0;
            for (int k = 0; k < nrhs; k++) active += hs[k].active;
            done = !active || it >= maxiter;
        }
    }
    int itmax = 0;
    for (int k = 0; k < nrhs; k++) itmax = std::max(itmax, hs[k].iters);
    *iters += itmax;
    // x_o = A_oo^-1 (b_o + 1/2 H_oe x_e)
    DslashCall e = base_call<P>(ctx, ms, nrhs, rs, colour);
    e.in = x;
    e.x = b;
    e.out = x;
    e.alpha = 1.0;
    e.beta = 0.5;
    e.diag = 2;
    e.post = 1;
    e.par0 = 1;
    stencil<P>(ctx, e);
    return DDRW_OK;
}

}  // namespace

// the block operator D_cc of one colour solved by the Krylov-loop BiCGStab above, on fields in the
// storage of policy id pid (32 FP32, 16 FP16, 17 BF16)
ddrw_status colour_bicgstab(ddrw_ctx *ctx, int pid, const MassSet &ms, const void *b, void *x, int nrhs,
                            const std::vector<double> &thresh, int maxiter, int *iters, int colour)
{
    switch (pid) {
    case 32: return eo_bicgstab<PrecS>(ctx, ms, (const float4 *)b, (float4 *)x, nrhs, thresh, maxiter, iters, colour);
    case 16: return eo_bicgstab<PrecH>(ctx, ms, (const PrecH::SElem *)b, (PrecH::SElem *)x, nrhs, thresh, maxiter, iters, colour);
    default: return eo_bicgstab<PrecB>(ctx, ms, (const PrecB::SElem *)b, (PrecB::SElem *)x, nrhs, thresh, maxiter, iters, colour);
    }
}

namespace {

ddrw_status full_norms(ddrw_ctx *ctx, const double2 *f, int nrhs, std::vector<double> &out)
{
    double *d;
    ddrw_status st = workspace(ctx, "full_norms", sizeof(double) * nrhs, (void **)&d);
    if (st) return st;
    VecRange all{ctx->V, 0, ctx->V, 12 * ctx->V, nrhs};
    if ((st = Blas<PrecD>::norm2(ctx, all, f, d))) return st;
    out.resize(nrhs);
    DDRW_CUDA_CHECK(cudaMemcpyAsync(out.data(), d, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    DDRW_SYNC(ctx);
    return DDRW_OK;
}

}  // namespace

// Even-odd BiCGStab on 16-bit storage with reliable updates: the Krylov vectors (r, rh, p, v, t)
// and the running solution increment x16 live in P16 (FP16 or BF16 with per-site norms); whenever a
// right-hand side's recursive residual has fallen by the factor delta since the last update (or
// has reached its target), the increment is folded into the FP32 solution x32, the true residual
// of the even-odd system b - Mhat x32 is recomputed with the FP32 operator and replaces r, and
// rho = (rh, r) is recomputed; p, v and the scalars carry on (the Krylov space is kept).  The
// solve thus reaches FP32 accuracy with 16-bit storage traffic, instead of stalling near the
// 16-bit rounding and restarting.  b and x are full FP32 fields; stops when ||r32||^2 <= thresh[r].
// With colour 0 / 1 it solves the block operator of that colour (its sites only, hops inside the
// blocks), as eo_bicgstab does.
template <class P16>
static ddrw_status eo_bicgstab_reliable(ddrw_ctx *ctx, const MassSet &ms, const float4 *b, float4 *x, int nrhs,
                                        const std::vector<double> &thresh, int maxiter, int *iters, int colour = -1)
{
    using E = typename P16::SElem;
    const long V = ctx->V, rs16 = P16::field_elems(V), rs32 = 6 * V;
    const size_t fb16 = sizeof(E) * rs16 * nrhs, fb32 = sizeof(float4) * rs32 * nrhs;
    const char *names[7] = {"eo_r", "eo_rh", "eo_p", "eo_v", "eo_t", "eo_tmp", "eo_x"};
    void *w[7];
    ddrw_status st;
    for (int k = 0; k < 7; k++) {
        char nm[32];
        snprintf(nm, sizeof nm, "%s%d", names[k], P16::ID);
        if ((st = workspace(ctx, nm, fb16, &w[k]))) return st;
    }
    E *r = (E *)w[0], *rh = (E *)w[1], *p = (E *)w[2], *v = (E *)w[3], *t = (E *)w[4], *tmp = (E *)w[5], *x16 = (E *)w[6];
    float4 *bh32, *r32, *tmp32;
    if ((st = workspace(ctx, "rel_bh32", fb32, (void **)&bh32))) return st;
    if ((st = workspace(ctx, "rel_r32", fb32, (void **)&r32))) return st;
    if ((st = workspace(ctx, "rel_tmp32", fb32, (void **)&tmp32))) return st;
    KScal *sc;
    double *red;
    if ((st = workspace(ctx, "eo_kscal", sizeof(KScal) * nrhs, (void **)&sc))) return st;
    if ((st = workspace(ctx, "rel_red", sizeof(double) * 4 * nrhs, (void **)&red))) return st;
    // the even sites of the whole lattice, or of the blocks of one colour (block operator)
    const long nc = colour < 0 ? ctx->vh : (long)ctx->nblk_c * (ctx->vh / ctx->nblk), o0 = colour < 0 ? 0 : colour * nc;
    const VecRange ev32{V, o0, nc, rs32, nrhs}, ev16{V, o0, nc, rs16, nrhs};

    // bhat = b_e + 1/2 H_eo A_oo^-1 b_o in FP32; x32 = 0; r32 = bhat
    DslashCall c = base_call<PrecS>(ctx, ms, nrhs, rs32, colour);
    c.x = b;
    c.out = tmp32;
    c.alpha = 1.0;
    c.diag = 2;
    c.post = 1;
    c.par0 = 1;
    dslash32(ctx, c);
    DslashCall d = base_call<PrecS>(ctx, ms, nrhs, rs32, colour);
    d.in = tmp32;
    d.x = b;
    d.out = bh32;
    d.alpha = 1.0;
    d.beta = 0.5;
    d.diag = 2;
    d.par0 = 0;
    dslash32(ctx, d);
    DDRW_CUDA_CHECK(cudaMemsetAsync(x, 0, fb32, ctx->stream));
    f32_to_16<P16>(ctx, ev32, rs16, bh32, r);

    std::vector<KScal> hk(nrhs);
    for (int k = 0; k < nrhs; k++) {
        hk[k] = KScal{};
        hk[k].thresh = thresh[k];
        hk[k].maxiter = maxiter;
    }
    DDRW_CUDA_CHECK(cudaMemcpyAsync(sc, hk.data(), sizeof(KScal) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
    if ((st = Blas<P16>::bicg_init(ctx, ev16, r, rh, p, x16, sc))) return st;
    KScal *hs = (KScal *)ctx->h_pinned;
    DDRW_CUDA_CHECK(cudaMemcpyAsync(hs, sc, sizeof(KScal) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    DDRW_SYNC(ctx);
    std::vector<double> rr_ref(nrhs), hred(4 * nrhs);
    std::vector<char> done(nrhs, 0);
    for (int k = 0; k < nrhs; k++) {
        rr_ref[k] = hs[k].rr;
        done[k] = hs[k].active ? 0 : 1;
    }
    const double delta2 = 1e-2;  // reliable update when the residual fell by 10 since the last one
    const long rs_ = rs16;
    int it = 0;
    bool all_done = true;
    for (int k = 0; k < nrhs; k++) all_done &= done[k] != 0;
    constexpr int check = 4;
    auto iteration = [&]() -> ddrw_status {
        return bicg_iteration<P16>(ctx, ms, nrhs, rs_, ev16, x16, r, rh, p, v, t, tmp, sc, colour);
    };
    // between reliable updates the iterations run as one CUDA graph (after a first eager pass that
    // tunes the launches): a conditional while-node stops when an update is due or at the cap
    int *count = nullptr, *act0_d = nullptr;
    double *rref_d = nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    const bool graphs = ctx->use_graphs && cs == cudaStreamCaptureStatusNone;
    if (graphs) {
        if ((st = workspace(ctx, "rel_count", sizeof(int), (void **)&count))) return st;
        if ((st = workspace(ctx, "rel_rref", sizeof(double) * nrhs, (void **)&rref_d))) return st;
        if ((st = workspace(ctx, "rel_act0", sizeof(int) * nrhs, (void **)&act0_d))) return st;
    }
    std::vector<int> act0(nrhs);
    bool eager_pass = true;
    while (!all_done && it < maxiter) {
        if (graphs && !eager_pass) {
            LoopKey key{};
            key[0] = 100000 + P16::ID + 1000 * (colour + 1);
            key[1] = (uintptr_t)nrhs;
            key[2] = (uintptr_t)maxiter;
            const void *ptrs[9] = {r, rh, p, v, t, tmp, x16, sc, count};
            for (int k = 0; k < 9; k++) key[3 + k] = (uintptr_t)ptrs[k];
            key[12] = (uintptr_t)ms.n;
            for (int k = 0; k < ms.n; k++) {
                double mk = ms.m[k];
                memcpy(&key[13 + 2 * k], &mk, sizeof(double));
                key[14 + 2 * k] = (uintptr_t)ainv_for(ms.inv[k], P16::ID);
            }
            cudaGraphExec_t exec = nullptr;
            if ((st = loop_graph(ctx, key, check, iteration, [&](cudaGraphConditionalHandle h) {
                     k_rel_cond<<<1, 1, 0, ctx->stream>>>(h, sc, rref_d, act0_d, nrhs, count, check, maxiter, delta2);
                 }, &exec)))
                return st;
            for (int k = 0; k < nrhs; k++) act0[k] = done[k] ? 0 : 1;
            DDRW_CUDA_CHECK(cudaMemcpyAsync(rref_d, rr_ref.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
            DDRW_CUDA_CHECK(cudaMemcpyAsync(act0_d, act0.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
            const int it0 = it;
            DDRW_CUDA_CHECK(cudaMemcpyAsync(count, &it, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
            DDRW_CUDA_CHECK(cudaGraphLaunch(exec, ctx->stream));
            ++ctx->graph_launches;
            DDRW_CUDA_CHECK(cudaMemcpyAsync(&it, count, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            DDRW_CUDA_CHECK(cudaMemcpyAsync(hs, sc, sizeof(KScal) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
            DDRW_SYNC(ctx);  // (also keeps the host arrays above alive until the copies have run)
            ctx->launches += (long)(it - it0) * 9 + (it - it0) / check;
        } else {
            for (int k = 0; k < check; k++, it++)
                if ((st = iteration())) return st;
            DDRW_CUDA_CHECK(cudaMemcpyAsync(hs, sc, sizeof(KScal) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
            DDRW_SYNC(ctx);
        }
        eager_pass = false;
        bool trigger = it >= maxiter, any_active = false;
        for (int k = 0; k < nrhs; k++) {
            if (done[k]) continue;
            any_active |= hs[k].active != 0;
            if (!hs[k].active || hs[k].rr < delta2 * rr_ref[k]) trigger = true;
        }
        if (!any_active) trigger = true;
        if (!trigger) continue;
        // reliable update of every right-hand side: x32 += x16, x16 = 0, r = bhat - Mhat x32 in FP32
        fold_16_into_32<P16>(ctx, ev32, rs16, x16, x);
        apply_mhat<PrecS>(ctx, ms, nrhs, rs32, x, tmp32, r32, colour);
        Blas<PrecS>::axpby(ctx, ev32, 1.0, bh32, -1.0, r32);
        if ((st = Blas<PrecS>::norm2(ctx, ev32, r32, red))) return st;
        f32_to_16<P16>(ctx, ev32, rs16, r32, r);
        if ((st = Blas<P16>::norm_dot(ctx, ev16, rh, r, red + nrhs))) return st;
        DDRW_CUDA_CHECK(cudaMemcpyAsync(hred.data(), red, sizeof(double) * 4 * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
        DDRW_SYNC(ctx);
        all_done = true;
        for (int k = 0; k < nrhs; k++) {
            const double rr = hred[k];
            if (!(rr == rr)) return set_error(ctx, DDRW_ENUMERIC, "NaN in a reliable update");
            rr_ref[k] = rr;
            if (rr <= thresh[k] || hs[k].breakdown) done[k] = 1;
            hs[k].rr = rr;
            hs[k].rho = make_double2(hred[nrhs + 3 * k + 1], hred[nrhs + 3 * k + 2]);
            hs[k].active = (!done[k] && it < maxiter) ? 1 : 0;
            all_done &= done[k] != 0;
        }
        DDRW_CUDA_CHECK(cudaMemcpyAsync(sc, hs, sizeof(KScal) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
    }
    *iters += it;
    // x_o = A_oo^-1 (b_o + 1/2 H_oe x_e) in FP32
    DslashCall e = base_call<PrecS>(ctx, ms, nrhs, rs32, colour);
    e.in = x;
    e.x = b;
    e.out = x;
    e.alpha = 1.0;
    e.beta = 0.5;
    e.diag = 2;
    e.post = 1;
    e.par0 = 1;
    dslash32(ctx, e);
    return DDRW_OK;
}

ddrw_status colour_bicgstab_reliable(ddrw_ctx *ctx, int pid, const MassSet &ms, const float4 *b, float4 *x, int nrhs,
                                     const std::vector<double> &thresh, int maxiter, int *iters, int colour)
{
    if (pid == 16) return eo_bicgstab_reliable<PrecH>(ctx, ms, b, x, nrhs, thresh, maxiter, iters, colour);
    return eo_bicgstab_reliable<PrecB>(ctx, ms, b, x, nrhs, thresh, maxiter, iters, colour);
}

// One inner solve of the defect correction in storage policy P: e = D^-1 rhs (rhs scaled by
// scale_d[r] into P's storage, the solution scaled back by scale_d[nrhs + r] and added to x, which
// is zeroed first on the first cycle).
template <class P>
static ddrw_status inner_solve(ddrw_ctx *ctx, const MassSet &ms, const double2 *rhs, double2 *x, bool first, int nrhs,
                               const double *scale_d, const std::vector<double> &th, int maxiter, int *iters)
{
    using E = typename P::SElem;
    const long V = ctx->V, rsl = P::field_elems(V);
    const size_t fl = sizeof(E) * rsl * nrhs;
    char nb[32], ne[32];
    snprintf(nb, sizeof nb, "full_b%d", P::ID);
    snprintf(ne, sizeof ne, "full_e%d", P::ID);
    void *bl, *el;
    ddrw_status st;
    if ((st = workspace(ctx, nb, fl, &bl))) return st;
    if ((st = workspace(ctx, ne, fl, &el))) return st;
    VecRange all{V, 0, V, 12 * V, nrhs};
    if (P::ID != 32 && ctx->reliable_updates()) {
        // 16-bit Krylov vectors with reliable updates into FP32 fields
        float4 *b32, *x32;
        const size_t f32 = sizeof(float4) * 6 * V * nrhs;
        if ((st = workspace(ctx, "full_b32", f32, (void **)&b32))) return st;
        if ((st = workspace(ctx, "full_e32", f32, (void **)&x32))) return st;
        to_low<PrecS>(ctx, all, 6 * V, rhs, b32, scale_d);
        if ((st = eo_bicgstab_reliable<P>(ctx, ms, b32, x32, nrhs, th, maxiter, iters))) return st;
        if (first) DDRW_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double2) * 12 * V * nrhs, ctx->stream));
        add_low<PrecS>(ctx, all, 6 * V, x32, x, scale_d + nrhs);
        return DDRW_OK;
    }
    to_low<P>(ctx, all, rsl, rhs, (E *)bl, scale_d);
    if (P::ID == 32 && ctx->outer_method == 1 && sap_supported(ctx)) {
        // Schwarz-preconditioned flexible GCR on the FP32 fields
        if ((st = sap_gcr(ctx, ms, (const float4 *)bl, (float4 *)el, nrhs, th, maxiter, iters))) return st;
    } else if ((st = eo_bicgstab<P>(ctx, ms, (const E *)bl, (E *)el, nrhs, th, maxiter, iters))) {
        return st;
    }
    if (first) DDRW_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double2) * 12 * V * nrhs, ctx->stream));
    add_low<P>(ctx, all, rsl, (const E *)el, x, scale_d + nrhs);
    return DDRW_OK;
}

// out = -D(ms) x over the whole lattice (the stencil part of the residual b - D x)
static DslashCall outer_residual_call(const ddrw_ctx *ctx, const MassSet &ms, const double2 *x, double2 *out, int nrhs)
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
    c.blk0 = 0;
    c.nblk = ctx->nblk;
    c.par0 = 0;
    c.npar = 2;
    return c;
}

// ---- device-controlled forms (the estimate captured as one graph)

// KScal of every right-hand side from device thresholds (the host form copies them)
__global__ void k_kscal_init(KScal *sc, const double *th, int nrhs, int maxiter)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    KScal k = {};
    k.thresh = th[r];
    k.maxiter = maxiter;
    sc[r] = k;
}

// loop condition of the captured Krylov loop (k_bicg_cond plus the body count of its loop)
__global__ void k_bicg_cond_dc(cudaGraphConditionalHandle h, const KScal *sc, int nrhs, int *count, int step,
                               int maxiter, int *body_count)
{
    int act = 0;
    for (int r = 0; r < nrhs; r++) act |= sc[r].active;
    int it = (*count += step);
    *body_count += 1;
    cudaGraphSetConditional(h, (act && it < maxiter) ? 1u : 0u);
}

__global__ void k_zero_count(int *c) { *c = 0; }

// outer iterations of a finished Krylov loop: the most any right-hand side needed
__global__ void k_iters_acc(const KScal *sc, int nrhs, int *acc)
{
    int m = 0;
    for (int r = 0; r < nrhs; r++) m = max(m, sc[r].iters);
    *acc += m;
}

template <class P>
static ddrw_status eo_bicgstab_dc(ddrw_ctx *ctx, const MassSet &ms, const typename P::SElem *b, typename P::SElem *x,
                                  int nrhs, const double *th, int maxiter)
{
    using E = typename P::SElem;
    const long rs = P::field_elems(ctx->V);
    const size_t fb = sizeof(E) * rs * nrhs;
    const char *names[6] = {"eo_r", "eo_rh", "eo_p", "eo_v", "eo_t", "eo_tmp"};
    void *w[6];
    ddrw_status st;
    for (int k = 0; k < 6; k++) {
        char nm[32];
        snprintf(nm, sizeof nm, "%s%d", names[k], P::ID);
        if ((st = workspace(ctx, nm, fb, &w[k]))) return st;
    }
    E *r = (E *)w[0], *rh = (E *)w[1], *p = (E *)w[2], *v = (E *)w[3], *t = (E *)w[4], *tmp = (E *)w[5];
    KScal *sc;
    int *count;
    if ((st = workspace(ctx, "eo_kscal", sizeof(KScal) * nrhs, (void **)&sc))) return st;
    if ((st = workspace(ctx, "eo_graph_count", sizeof(int), (void **)&count))) return st;
    DslashCall c = base_call<P>(ctx, ms, nrhs, rs);  // btil_e = b_e + 1/2 H_eo A_oo^-1 b_o
    c.x = b;
    c.out = tmp;
    c.alpha = 1.0;
    c.diag = 2;
    c.post = 1;
    c.par0 = 1;
    stencil<P>(ctx, c);
    DslashCall d = base_call<P>(ctx, ms, nrhs, rs);
    d.in = tmp;
    d.x = b;
    d.out = r;
    d.alpha = 1.0;
    d.beta = 0.5;
    d.diag = 2;
    d.par0 = 0;
    stencil<P>(ctx, d);
    ++ctx->launches;
    k_kscal_init<<<(nrhs + 63) / 64, 64, 0, ctx->stream>>>(sc, th, nrhs, maxiter);
    VecRange ev{ctx->V, 0, ctx->vh, rs, nrhs};
    if ((st = Blas<P>::bicg_init(ctx, ev, r, rh, p, x, sc))) return st;
    ++ctx->launches;
    k_zero_count<<<1, 1, 0, ctx->stream>>>(count);  // a kernel node: this may sit in an outer loop body
    const int check = sizeof(typename P::R) == 8 ? 1 : 4;
    st = capture_while(ctx, (const void *)k_bicg_cond_dc, [&](cudaGraphConditionalHandle h, int slot) -> ddrw_status {
        ddrw_status s2;
        for (int k = 0; k < check; k++)
            if ((s2 = bicg_iteration<P>(ctx, ms, nrhs, rs, ev, x, r, rh, p, v, t, tmp, sc))) return s2;
        ++ctx->launches;
        k_bicg_cond_dc<<<1, 1, 0, ctx->stream>>>(h, sc, nrhs, count, check, maxiter, &ctx->dc->loop_iters[slot]);
        return DDRW_OK;
    });
    if (st) return st;
    ++ctx->launches;
    k_iters_acc<<<1, 1, 0, ctx->stream>>>(sc, nrhs, &ctx->dc->outer_iters);
    DslashCall e = base_call<P>(ctx, ms, nrhs, rs);  // x_o = A_oo^-1 (b_o + 1/2 H_oe x_e)
    e.in = x;
    e.x = b;
    e.out = x;
    e.alpha = 1.0;
    e.beta = 0.5;
    e.diag = 2;
    e.post = 1;
    e.par0 = 1;
    stencil<P>(ctx, e);
    return DDRW_OK;
}

// control of the outer defect correction: mode 0 before the first cycle (nr = bb), mode 1 after a
// cycle (statistics, continue decision, then the next inner settings from nr = rr); ctl[0] counts
// the cycles
__global__ void k_full_ctl(int mode, int nrhs, const double *bb, const double *rr, double tol, double floor, int mixed,
                           int maxiter, double *scale, double *th, int *ctl, DcStats *dc, int slot,
                           cudaGraphConditionalHandle h)
{
    const double *nr = mode == 0 ? bb : rr;
    if (mode == 1) {
        const int cyc = ++ctl[0];
        dc->loop_iters[slot] += 1;
        dc->outer_cycles = cyc;
        dc->fp64_dslash_full += 1;
        double worst = 0.0;
        bool nan = false;
        for (int r = 0; r < nrhs; r++) {
            if (!isfinite(rr[r])) nan = true;
            else if (bb[r] > 0) worst = fmax(worst, sqrt(rr[r] / bb[r]));
        }
        dc->outer_rel_residual = worst;
        unsigned cont = 1;
        if (nan) {
            dc->nan = 1;
            cont = 0;
        } else if (worst <= tol) {
            cont = 0;
        } else if (cyc >= 40 || dc->outer_iters >= 4 * maxiter) {
            dc->noconv = 1;
            cont = 0;
        }
        cudaGraphSetConditional(h, cont);
    } else {
        ctl[0] = 0;
    }
    for (int r = 0; r < nrhs; r++) {
        const double q = nr[r];
        scale[r] = q > 0 ? 1.0 / sqrt(q) : 0.0;
        scale[nrhs + r] = sqrt(q);
        if (mixed) {
            const double need = q > 0 ? 0.5 * tol * sqrt(bb[r] / q) : 1.0;
            const double ti = fmax(floor, fmin(need, 0.5));
            th[r] = q > 0 ? ti * ti : 0.0;
        } else {
            th[r] = 0.25 * tol * tol * bb[r];
        }
    }
}

template <class P>
static ddrw_status inner_solve_dc(ddrw_ctx *ctx, const MassSet &ms, const double2 *rhs, double2 *x, int nrhs,
                                  const double *scale, const double *th, int maxiter)
{
    using E = typename P::SElem;
    const long V = ctx->V, rsl = P::field_elems(V);
    const size_t fl = sizeof(E) * rsl * nrhs;
    char nb[32], ne[32];
    snprintf(nb, sizeof nb, "full_b%d", P::ID);
    snprintf(ne, sizeof ne, "full_e%d", P::ID);
    void *bl, *el;
    ddrw_status st;
    if ((st = workspace(ctx, nb, fl, &bl))) return st;
    if ((st = workspace(ctx, ne, fl, &el))) return st;
    VecRange all{V, 0, V, 12 * V, nrhs};
    to_low<P>(ctx, all, rsl, rhs, (E *)bl, scale);
    if ((st = eo_bicgstab_dc<P>(ctx, ms, (const E *)bl, (E *)el, nrhs, th, maxiter))) return st;
    add_low<P>(ctx, all, rsl, (const E *)el, x, scale + nrhs);
    return DDRW_OK;
}

ddrw_status full_solve_dc_prepare(ddrw_ctx *ctx, int nrhs)
{
    void *p;
    ddrw_status st;
    if ((st = workspace(ctx, "dcf_norms", sizeof(double) * 2 * nrhs, &p))) return st;
    if ((st = workspace(ctx, "dcf_scale", sizeof(double) * 3 * nrhs, &p))) return st;
    if ((st = workspace(ctx, "dcf_ctl", sizeof(int), &p))) return st;
    if ((st = workspace(ctx, "full_e64", sizeof(double2) * 12 * ctx->V * nrhs, &p))) return st;
    if ((st = workspace(ctx, "eo_graph_count", sizeof(int), &p))) return st;
    if ((st = workspace(ctx, "eo_redpart", sizeof(double) * 3 * (size_t)(ctx->vh / 32) * nrhs, &p))) return st;
    return DDRW_OK;
}

static ddrw_status full_solve_dc(ddrw_ctx *ctx, const MassSet &ms, const double2 *b, double2 *x, int nrhs, double tol,
                                 int maxiter, ddrw_prec prec)
{
    const long V = ctx->V, rs64 = 12 * V;
    const size_t f64 = sizeof(double2) * rs64 * nrhs;
    const bool mixed = prec != DDRW_FP64;
    const double floor = prec == DDRW_MIXED_FP32 ? 1e-6 : prec == DDRW_MIXED_FP16 ? 1e-3 : 5e-3;
    ddrw_status st;
    double2 *res, *e64;
    double *norms, *scale;
    int *cyc;
    if ((st = workspace(ctx, "full_res", f64, (void **)&res))) return st;
    if ((st = workspace(ctx, "full_e64", f64, (void **)&e64))) return st;
    if ((st = workspace(ctx, "dcf_norms", sizeof(double) * 2 * nrhs, (void **)&norms))) return st;
    if ((st = workspace(ctx, "dcf_scale", sizeof(double) * 3 * nrhs, (void **)&scale))) return st;
    if ((st = workspace(ctx, "dcf_ctl", sizeof(int), (void **)&cyc))) return st;
    double *bb = norms, *rr = norms + nrhs, *th = scale + 2 * nrhs;
    const VecRange all{V, 0, V, rs64, nrhs};
    if ((st = Blas<PrecD>::norm2(ctx, all, b, bb))) return st;
    DDRW_CUDA_CHECK(cudaMemcpyAsync(res, b, f64, cudaMemcpyDeviceToDevice, ctx->stream));
    DDRW_CUDA_CHECK(cudaMemsetAsync(x, 0, f64, ctx->stream));
    ++ctx->launches;
    k_full_ctl<<<1, 1, 0, ctx->stream>>>(0, nrhs, bb, rr, tol, floor, mixed, maxiter, scale, th, cyc, ctx->dc, 0, 0);
    return capture_while(ctx, (const void *)k_full_ctl, [&](cudaGraphConditionalHandle h, int slot) -> ddrw_status {
        ddrw_status s2;
        if (mixed) {
            if (prec == DDRW_MIXED_FP32) s2 = inner_solve_dc<PrecS>(ctx, ms, res, x, nrhs, scale, th, maxiter);
            else if (prec == DDRW_MIXED_FP16) s2 = inner_solve_dc<PrecH>(ctx, ms, res, x, nrhs, scale, th, maxiter);
            else s2 = inner_solve_dc<PrecB>(ctx, ms, res, x, nrhs, scale, th, maxiter);
            if (s2) return s2;
        } else {
            if ((s2 = eo_bicgstab_dc<PrecD>(ctx, ms, res, e64, nrhs, th, maxiter))) return s2;
            Blas<PrecD>::axpby(ctx, all, 1.0, e64, 1.0, x);
        }
        DslashCall c = outer_residual_call(ctx, ms, x, res, nrhs);
        if ((s2 = residual_stencil(ctx, c, mixed))) return s2;
        Blas<PrecD>::axpby(ctx, all, 1.0, b, 1.0, res);
        if ((s2 = Blas<PrecD>::norm2(ctx, all, res, rr))) return s2;
        ++ctx->launches;
        k_full_ctl<<<1, 1, 0, ctx->stream>>>(1, nrhs, bb, rr, tol, floor, mixed, maxiter, scale, th, cyc, ctx->dc, slot, h);
        return DDRW_OK;
    });
}

ddrw_status full_solve64(ddrw_ctx *ctx, const MassSet &ms, const double2 *b, double2 *x, int nrhs, double tol,
                         int maxiter, ddrw_prec prec, SolveStats *stats)
{
    if (ctx->devctl) return full_solve_dc(ctx, ms, b, x, nrhs, tol, maxiter, prec);
    const long V = ctx->V, rs64 = 12 * V;
    const size_t f64 = sizeof(double2) * rs64 * nrhs;
    const bool mixed = prec != DDRW_FP64;
    // deepest relative residual an inner solve is asked for: what its storage reliably reaches (16-bit
    // storage with reliable updates reaches what their FP32 residuals reach)
    const double floor = (prec == DDRW_MIXED_FP32 || ctx->reliable_updates()) ? 1e-6 : prec == DDRW_MIXED_FP16 ? 1e-3 : 5e-3;
    ddrw_status st;
    std::vector<double> bb, rr;
    if ((st = full_norms(ctx, b, nrhs, bb))) return st;
    for (int r = 0; r < nrhs; r++)
        if (!std::isfinite(bb[r])) return set_error(ctx, DDRW_ENUMERIC, "non-finite right-hand side");
    double2 *res, *e64 = nullptr;
    double *scale_d = nullptr;
    if ((st = workspace(ctx, "full_res", f64, (void **)&res))) return st;
    if (mixed) {
        if ((st = workspace(ctx, "full_scale", sizeof(double) * 2 * nrhs, (void **)&scale_d))) return st;
    } else if ((st = workspace(ctx, "full_e64", f64, (void **)&e64))) {
        return st;
    }
    // inner target per right-hand side and cycle: what is still missing to reach tol, with a
    // margin of 2, but no deeper than the inner storage reliably goes (floor)
    const double2 *rhs = b;
    bool first = true;
    std::vector<double> scale(nrhs), unscale(nrhs), ones(nrhs, 1.0);
    int iters = 0, cycles = 0;
    for (; cycles < 40; cycles++) {
        const std::vector<double> &nr = first ? bb : rr;
        if (mixed) {
            for (int r = 0; r < nrhs; r++) {
                double n = std::sqrt(nr[r]);
                scale[r] = n > 0 ? 1.0 / n : 0.0;
                unscale[r] = n;
            }
            DDRW_CUDA_CHECK(cudaMemcpyAsync(scale_d, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
            DDRW_CUDA_CHECK(cudaMemcpyAsync(scale_d + nrhs, unscale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice,
                                            ctx->stream));
            std::vector<double> th(nrhs);
            for (int r = 0; r < nrhs; r++) {
                double need = nr[r] > 0 ? 0.5 * tol * std::sqrt(bb[r] / nr[r]) : 1.0;
                double ti = std::max(floor, std::min(need, 0.5));
                th[r] = nr[r] > 0 ? ti * ti : 0.0;
            }
            if (prec == DDRW_MIXED_FP32) st = inner_solve<PrecS>(ctx, ms, rhs, x, first, nrhs, scale_d, th, maxiter, &iters);
            else if (prec == DDRW_MIXED_FP16) st = inner_solve<PrecH>(ctx, ms, rhs, x, first, nrhs, scale_d, th, maxiter, &iters);
            else st = inner_solve<PrecB>(ctx, ms, rhs, x, first, nrhs, scale_d, th, maxiter, &iters);
            if (st) return st;
        } else {
            double2 *target = first ? x : e64;
            std::vector<double> th(nrhs);
            for (int r = 0; r < nrhs; r++) th[r] = 0.25 * tol * tol * bb[r];
            if ((st = eo_bicgstab<PrecD>(ctx, ms, rhs, target, nrhs, th, maxiter, &iters))) return st;
            if (!first) Blas<PrecD>::axpby(ctx, VecRange{V, 0, V, rs64, nrhs}, 1.0, e64, 1.0, x);
        }
        // res = b - D x in FP64
        DslashCall c = outer_residual_call(ctx, ms, x, res, nrhs);
        if ((st = residual_stencil(ctx, c, mixed))) return st;
        if (stats) stats->fp64_dslash_full += 1;
        Blas<PrecD>::axpby(ctx, VecRange{V, 0, V, rs64, nrhs}, 1.0, b, 1.0, res);
        if ((st = full_norms(ctx, res, nrhs, rr))) return st;
        double worst = 0;
        for (int r = 0; r < nrhs; r++)
            if (!std::isfinite(rr[r])) worst = NAN;
            else if (bb[r] > 0 && !(worst != worst)) worst = std::max(worst, std::sqrt(rr[r] / bb[r]));
        if (stats) {
            stats->outer_cycles = cycles + 1;
            stats->outer_rel_residual = worst;
        }
        if (!(worst == worst)) return set_error(ctx, DDRW_ENUMERIC, "NaN in the outer solve");
        if (worst <= tol) break;
        if (iters >= maxiter * 4) break;
        rhs = res;
        first = false;
    }
    if (stats) stats->outer_iters += iters;
    if (stats && stats->outer_rel_residual > tol) return set_error(ctx, DDRW_ENOCONV, "outer solve did not converge");
    return DDRW_OK;
}

}  // namespace ddrw
