// api.cu -- the C ABI (include/ddrw.h): context, geometry tables, parameters, operator
// applications.  Solvers and the estimate live in solver.cu and estimate.cu.
#include <chrono>
#include <cstdio>
#include <cstring>

#include "blas.cuh"
#include "ctx.h"
#include "lowprec.cuh"

namespace ddrw {

ddrw_status set_error(ddrw_ctx *ctx, ddrw_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

ddrw_status set_cuda_error(ddrw_ctx *ctx, cudaError_t e, const char *what, const char *file, int line)
{
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return set_error(ctx, e == cudaErrorMemoryAllocation ? DDRW_ENOMEM : DDRW_ECUDA, buf);
}

// Captured Krylov-loop graphs hold raw device pointers (workspaces, reduction buffers, inverses):
// every graph is destroyed before any such buffer is freed or moved.
void clear_graphs(ddrw_ctx *ctx)
{
    ctx->est_seen.clear();
    if (ctx->graphs.empty() && ctx->est_graphs.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
    }
    ctx->graphs.clear();
    for (auto &kv : ctx->est_graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
    }
    ctx->est_graphs.clear();
}

// arms a loop: its condition is 1 when the loop node is reached (each time, also inside an outer loop)
static __global__ void k_arm_loop(cudaGraphConditionalHandle h) { cudaGraphSetConditional(h, 1u); }

ddrw_status capture_while(ddrw_ctx *ctx, const void *cond_fn,
                          const std::function<ddrw_status(cudaGraphConditionalHandle, int)> &body)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    DDRW_CUDA_CHECK(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &graph, &deps, &ed, &nd));
    if (cs != cudaStreamCaptureStatusActive) return set_error(ctx, DDRW_ESTATE, "loop capture outside a stream capture");
    if (ctx->cap_depth >= 4 || ctx->dc_loops >= DC_LOOPS)
        return set_error(ctx, DDRW_EINVAL, "too many nested or captured loops");
    cudaGraphConditionalHandle h;
    DDRW_CUDA_CHECK(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
    // a kernel node in front of the loop sets its condition to 1: the default applies only at graph
    // launch, and a loop nested in another loop's body must start afresh on every outer pass
    ++ctx->launches;
    k_arm_loop<<<1, 1, 0, ctx->stream>>>(h);
    DDRW_CUDA_CHECK(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &graph, &deps, &ed, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    DDRW_CUDA_CHECK(cudaGraphAddNode(&node, graph, deps, ed, nd, &cp));
    DDRW_CUDA_CHECK(cudaStreamUpdateCaptureDependencies(ctx->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    cudaStream_t &side = ctx->cap_streams[ctx->cap_depth];
    if (!side) DDRW_CUDA_CHECK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    DDRW_CUDA_CHECK(cudaStreamBeginCaptureToGraph(side, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaStream_t saved = ctx->stream;
    ctx->stream = side;
    const int slot = ctx->dc_loops++;
    const long l0 = ctx->launches;
    ctx->cap_depth++;
    ctx->cap_nested[ctx->cap_depth] = 0;
    ddrw_status st = body(h, slot);
    const long inner = ctx->cap_nested[ctx->cap_depth];
    ctx->cap_depth--;
    ctx->stream = saved;
    cudaGraph_t g2 = nullptr;
    cudaError_t e = cudaStreamEndCapture(side, &g2);
    if (st) return st;
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaStreamEndCapture(loop body)", __FILE__, __LINE__);
    // the launches of this body, without those of loops nested in it (counted per their own runs)
    const long all = ctx->launches - l0;
    ctx->cap_loop_launches.push_back({slot, all - inner});
    ctx->cap_nested[ctx->cap_depth] += all;
    // the body must contain its condition kernel, or the loop would never end
    size_t nn = 0;
    DDRW_CUDA_CHECK(cudaGraphGetNodes(bodyg, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) DDRW_CUDA_CHECK(cudaGraphGetNodes(bodyg, nodes.data(), &nn));
    bool found = false;
    for (auto n : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(n, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(n, &kp) == cudaSuccess && kp.func == cond_fn) found = true;
    }
    if (!found) return set_error(ctx, DDRW_ECUDA, "a captured loop body lacks its condition kernel");
    return DDRW_OK;
}

ddrw_status workspace(ddrw_ctx *ctx, const char *name, size_t bytes, void **out)
{
    DevBuf &b = ctx->ws[name];
    if (b.bytes < bytes) {
        // a graph capture must find every buffer allocated (allocating would end the capture)
        if (ctx->devctl) return set_error(ctx, DDRW_ESTATE, std::string("workspace allocation during capture: ") + name);
        clear_graphs(ctx);
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        cudaError_t e = cudaMalloc(&b.p, bytes);
        if (e != cudaSuccess) {
            b.p = nullptr;
            return set_cuda_error(ctx, e, "cudaMalloc(workspace)", __FILE__, __LINE__);
        }
        b.bytes = bytes;
    }
    *out = b.p;
    return DDRW_OK;
}

void release_workspace(ddrw_ctx *ctx, const char *name)
{
    auto it = ctx->ws.find(name);
    if (it == ctx->ws.end()) return;
    clear_graphs(ctx);
    cudaStreamSynchronize(ctx->stream);
    if (it->second.p) cudaFree(it->second.p);
    ctx->ws.erase(it);
}

GeomDev geom_dev(const ddrw_ctx *ctx)
{
    GeomDev g;
    for (int mu = 0; mu < 4; mu++) {
        g.L[mu] = ctx->dims[mu];
        g.NB[mu] = ctx->NB[mu];
    }
    g.nblk = ctx->nblk;
    g.nblk_c = ctx->nblk_c;
    g.vh = ctx->vh;
    g.V = ctx->V;
    g.blk_nb = ctx->d_blk_nb;
    g.blk_org = ctx->d_blk_org;
    g.blk_index = ctx->d_blk_index;
    g.tsign = ctx->antiperiodic ? -1 : 1;
    g.nbr = ctx->d_nbr;
    return g;
}

ddrw_status mass_inverse(ddrw_ctx *ctx, double m, MassInv **out)
{
    for (auto &mi : ctx->inv)
        if (mi.m == m) {
            *out = &mi;
            return DDRW_OK;
        }
    MassInv mi;
    mi.m = m;
    cudaError_t e = cudaMalloc(&mi.A64, sizeof(double2) * 36 * (size_t)ctx->V);
    if (e == cudaSuccess) e = cudaMalloc(&mi.A32, sizeof(float4) * 18 * (size_t)ctx->V);
    if (e == cudaSuccess) e = cudaMalloc(&mi.A16, sizeof(uint2) * 18 * (size_t)ctx->V);
    if (e == cudaSuccess) e = cudaMalloc(&mi.Ab16, sizeof(uint2) * 18 * (size_t)ctx->V);
    if (e != cudaSuccess) {
        cudaFree(mi.A64);
        cudaFree(mi.A32);
        cudaFree(mi.A16);
        cudaFree(mi.Ab16);
        return set_cuda_error(ctx, e, "cudaMalloc(in-block inverse)", __FILE__, __LINE__);
    }
    build_inverse(ctx, m, mi);
    f32_to_low(ctx, mi.A32, mi.A16, 18L * ctx->V, false);
    f32_to_low(ctx, mi.A32, mi.Ab16, 18L * ctx->V, true);
    DDRW_CUDA_CHECK(cudaGetLastError());
    ctx->inv.push_back(mi);
    *out = &ctx->inv.back();
    return DDRW_OK;
}

static void free_inverses(ddrw_ctx *ctx)
{
    clear_graphs(ctx);
    for (auto &mi : ctx->inv) {
        cudaFree(mi.A64);
        cudaFree(mi.A32);
        cudaFree(mi.A16);
        cudaFree(mi.Ab16);
    }
    ctx->inv.clear();
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

ddrw_status stage_in(ddrw_ctx *ctx, const void *user, size_t bytes, const char *name, const void **dev)
{
    if (is_device_ptr(user)) {
        *dev = user;
        return DDRW_OK;
    }
    void *p;
    ddrw_status st = workspace(ctx, name, bytes, &p);
    if (st) return st;
    DDRW_CUDA_CHECK(cudaMemcpyAsync(p, user, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *dev = p;
    return DDRW_OK;
}

ddrw_status stage_out(ddrw_ctx *ctx, void *user, size_t bytes, const char *name, void **dev, bool *host)
{
    if (is_device_ptr(user)) {
        *dev = user;
        *host = false;
        return DDRW_OK;
    }
    *host = true;
    return workspace(ctx, name, bytes, dev);
}

ddrw_status finish_out(ddrw_ctx *ctx, void *user, const void *dev, size_t bytes, bool host)
{
    if (host) DDRW_CUDA_CHECK(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    return DDRW_OK;
}

ddrw_status sync(ddrw_ctx *ctx)
{
    DDRW_CUDA_CHECK(cudaGetLastError());
    DDRW_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    if (ctx->h_err && *(volatile int *)ctx->h_err) {
        *(volatile int *)ctx->h_err = 0;
        return set_error(ctx, DDRW_ETIMEOUT, "a staged stencil launch gave up waiting for its shared-memory copies");
    }
    return DDRW_OK;
}

// internal index from global coordinates (host mirror of the device function)
long host_internal_index(const ddrw_ctx *ctx, const std::vector<int> &blk_index, const int *x)
{
    int l = ctx->l;
    int b[4], c[4];
    for (int mu = 0; mu < 4; mu++) {
        b[mu] = x[mu] / l;
        c[mu] = x[mu] - b[mu] * l;
    }
    int B = ((b[0] * ctx->NB[1] + b[1]) * ctx->NB[2] + b[2]) * ctx->NB[3] + b[3];
    int lb = ((c[0] * l + c[1]) * l + c[2]) * l + c[3];
    int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    long vbh = (long)l * l * l * l / 2;
    return (long)p * ctx->vh + (long)blk_index[B] * vbh + (lb >> 1);
}

ddrw_status residual_stencil(ddrw_ctx *ctx, DslashCall c, bool ds)
{
    if (!ds) {
        dslash64(ctx, c);
        return DDRW_OK;
    }
    // the stencil reads `in` at the hop neighbours and `x` at the site; both are the same field here
    if (c.x && c.x != c.in) return set_error(ctx, DDRW_EINVAL, "double-single residual needs x == in");
    if (c.hopsel == 2) return set_error(ctx, DDRW_EINVAL, "double-single residual of a hop between blocks");
    float4 *xs;
    ddrw_status st = workspace(ctx, "ds_split", sizeof(float4) * (size_t)c.rstride * c.nrhs, (void **)&xs);
    if (st) return st;
    // only the sites the stencil reads: its own blocks (hops inside blocks) or every site
    long vbh = (long)ctx->l * ctx->l * ctx->l * ctx->l / 2;
    if (c.hopsel == 1)
        split64(ctx, (const double2 *)c.in, xs, ctx->V, ctx->vh, c.blk0 * vbh, c.nblk * vbh, 0, 2, c.nrhs, c.rstride);
    else
        split64(ctx, (const double2 *)c.in, xs, ctx->V, ctx->vh, 0, ctx->vh, 0, 2, c.nrhs, c.rstride);
    c.in = xs;
    c.x = xs;
    dslash_ds(ctx, c);
    return DDRW_OK;
}

// zero the sites of one colour (both parities) in nrhs FP64 fields
__global__ void k_zero_colour(double2 *f, long V, long vh, long lo, long n, int nrhs)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = 2 * n;  // both parities
    if (i >= per * 12 * nrhs) return;
    long r = i / (per * 12);
    long rem = i - r * per * 12;
    long k = rem / per;
    long j = rem - k * per;
    long p = j / n;
    long s = p * vh + lo + (j - p * n);
    f[(r * 12 + k) * V + s] = make_double2(0.0, 0.0);
}

void zero_colour64(ddrw_ctx *ctx, double2 *f, int colour, int nrhs)
{
    long vbh = (long)ctx->l * ctx->l * ctx->l * ctx->l / 2;
    long n = (long)ctx->nblk_c * vbh;
    long lo = colour == DDRW_BLACK ? 0 : n;
    long tot = 2 * n * 12 * nrhs;
    ++ctx->launches;
    k_zero_colour<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(f, ctx->V, ctx->vh, lo, n, nrhs);
}

static cudaEvent_t pool_event(ddrw_ctx *ctx)
{
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(ddrw_ctx *c, int k, double b, double u) : ctx(c), kind(k), bytes(b), units(u)
{
    if (!ctx->prof_on) return;
    // launches captured into a graph are not timed (graph bodies hold no event nodes)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    if (cs != cudaStreamCaptureStatusNone) return;
    a = pool_event(ctx);
    cudaEventRecord(a, ctx->stream);
}

ProfScope::~ProfScope()
{
    if (!a) return;
    cudaEvent_t b = pool_event(ctx);
    cudaEventRecord(b, ctx->stream);
    ctx->prof_pending.push_back({a, b, kind, bytes, units});
}

static void prof_collect(ddrw_ctx *ctx)
{
    if (ctx->prof_pending.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &r : ctx->prof_pending) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        ctx->prof_count[r.kind] += 1;
        ctx->prof_ms[r.kind] += ms;
        ctx->prof_bytes[r.kind] += r.bytes;
        ctx->prof_units[r.kind] += r.units;
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
}

// the storage-precision stencil on full fields: out = D(m) in, or A(m)^-1 D(m) in (post)
template <class P>
static ddrw_status apply_low(ddrw_ctx *ctx, double m, int post, const double2 *fin, double2 *fout, int nrhs)
{
    using E = typename P::SElem;
    const long rsl = P::field_elems(ctx->V);
    E *lin, *lout;
    ddrw_status st;
    if ((st = workspace(ctx, "api_low0", sizeof(E) * rsl * nrhs, (void **)&lin))) return st;
    if ((st = workspace(ctx, "api_low1", sizeof(E) * rsl * nrhs, (void **)&lout))) return st;
    MassInv *mi = nullptr;
    if (post && (st = mass_inverse(ctx, m, &mi))) return st;
    const VecRange all{ctx->V, 0, ctx->V, 12 * ctx->V, nrhs};
    to_low<P>(ctx, all, rsl, fin, lin, nullptr);
    DslashCall c;
    c.in = lin;
    c.x = lin;
    c.out = lout;
    c.rstride = rsl;
    c.nrhs = nrhs;
    c.masses[0] = m;
    if (post) c.Ainv[0] = ainv_for(mi, P::ID);
    c.alpha = 1.0;
    c.beta = -0.5;
    c.diag = 1;
    c.post = post;
    c.par0 = 0;
    c.npar = 2;
    c.blk0 = 0;
    c.nblk = ctx->nblk;
    if constexpr (P::ID == 32) dslash32(ctx, c);
    else if constexpr (P::ID == 16) dslash16(ctx, c);
    else dslashb16(ctx, c);
    DDRW_CUDA_CHECK(cudaMemsetAsync(fout, 0, sizeof(double2) * 12 * ctx->V * nrhs, ctx->stream));
    add_low<P>(ctx, all, rsl, lout, fout, nullptr);
    return DDRW_OK;
}

}  // namespace ddrw

using namespace ddrw;

extern "C" {

ddrw_status ddrw_profile(ddrw_ctx *ctx, int enable)
{
    if (!ctx) return DDRW_EINVAL;
    prof_collect(ctx);
    for (int k = 0; k < 16; k++) {
        ctx->prof_count[k] = 0;
        ctx->prof_ms[k] = 0;
        ctx->prof_bytes[k] = 0;
        ctx->prof_units[k] = 0;
    }
    ctx->prof_on = enable != 0;
    ctx->launches = 0;
    return DDRW_OK;
}

ddrw_status ddrw_use_graphs(ddrw_ctx *ctx, int enable, long *graph_launches)
{
    if (!ctx) return DDRW_EINVAL;
    if (enable > 2) return set_error(ctx, DDRW_EINVAL, "graph mode must be 0, 1 or 2");
    if (enable >= 0) {
        ctx->use_graphs = enable != 0;
        ctx->use_est_graphs = enable == 1;  // captured graphs are kept for when the mode returns
    }
    if (graph_launches) *graph_launches = ctx->graph_launches;
    return DDRW_OK;
}

ddrw_status ddrw_profile_read(ddrw_ctx *ctx, int kind, long *launches, double *ms, double *bytes)
{
    if (!ctx || kind < 0 || kind > PROF_NKIND) return DDRW_EINVAL;
    prof_collect(ctx);
    if (kind == PROF_NKIND) {  // every kernel launch of the library
        if (launches) *launches = ctx->launches;
        if (ms) *ms = 0;
        if (bytes) *bytes = 0;
        return DDRW_OK;
    }
    if (launches) *launches = ctx->prof_count[kind];
    if (ms) *ms = ctx->prof_ms[kind];
    if (bytes) *bytes = ctx->prof_bytes[kind];
    return DDRW_OK;
}

ddrw_status ddrw_profile_units(ddrw_ctx *ctx, int kind, double *site_updates)
{
    if (!ctx || !site_updates || kind < 0 || kind >= PROF_NKIND) return DDRW_EINVAL;
    prof_collect(ctx);
    *site_updates = ctx->prof_units[kind];
    return DDRW_OK;
}

ddrw_status ddrw_create(ddrw_ctx **out, const int dims[4], const int block[4], int device, void *cuda_stream)
{
    if (!out || !dims || !block) return DDRW_EINVAL;
    *out = nullptr;
    int l = block[0];
    for (int mu = 0; mu < 4; mu++) {
        if (block[mu] != l) return DDRW_EINVAL;
        if (dims[mu] <= 0 || dims[mu] % l) return DDRW_EINVAL;
        int nb = dims[mu] / l;
        if (nb < 2 || nb % 2) return DDRW_EINVAL;
    }
    if (l != 2 && l != 4 && l != 6 && l != 8) return DDRW_EINVAL;
    ddrw_ctx *ctx = new ddrw_ctx();
    ctx->l = l;
    ctx->V = 1;
    for (int mu = 0; mu < 4; mu++) {
        ctx->dims[mu] = dims[mu];
        ctx->NB[mu] = dims[mu] / l;
        ctx->V *= dims[mu];
    }
    if (ctx->V > (1L << 27)) {  // in-field offsets of the kernels are 32-bit
        delete ctx;
        return DDRW_EINVAL;
    }
    ctx->vh = ctx->V / 2;
    ctx->nblk = ctx->NB[0] * ctx->NB[1] * ctx->NB[2] * ctx->NB[3];
    ctx->nblk_c = ctx->nblk / 2;
    ctx->device = device;
    auto fail = [&](ddrw_status st) {
        ddrw_destroy(ctx);
        return st;
    };
    if (cudaSetDevice(device) != cudaSuccess) return fail(DDRW_ECUDA);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(DDRW_ECUDA);
        ctx->own_stream = true;
    }

    // block tables: colour-major numbering, black blocks first
    int nb = ctx->nblk;
    std::vector<int> number(nb), org(4 * nb), nbr(8 * nb);
    int nblack = 0, nwhite = 0;
    for (int B = 0; B < nb; B++) {
        int r = B, c[4];
        for (int mu = 3; mu >= 0; mu--) {
            c[mu] = r % ctx->NB[mu];
            r /= ctx->NB[mu];
        }
        int colour = (c[0] + c[1] + c[2] + c[3]) & 1;
        number[B] = colour == 0 ? nblack++ : ctx->nblk_c + nwhite++;
    }
    if (nblack != ctx->nblk_c || nwhite != ctx->nblk_c) return fail(DDRW_EINVAL);
    for (int B = 0; B < nb; B++) {
        int r = B, c[4];
        for (int mu = 3; mu >= 0; mu--) {
            c[mu] = r % ctx->NB[mu];
            r /= ctx->NB[mu];
        }
        int k = number[B];
        for (int mu = 0; mu < 4; mu++) org[4 * k + mu] = c[mu] * l;
        for (int mu = 0; mu < 4; mu++)
            for (int d = 0; d < 2; d++) {
                int cc[4] = {c[0], c[1], c[2], c[3]};
                cc[mu] = (cc[mu] + (d == 0 ? 1 : -1) + ctx->NB[mu]) % ctx->NB[mu];
                int B2 = ((cc[0] * ctx->NB[1] + cc[1]) * ctx->NB[2] + cc[2]) * ctx->NB[3] + cc[3];
                nbr[8 * k + 2 * mu + d] = number[B2];
            }
    }
    // supp P: black sites on a block face (the neighbouring block across any face is white)
    std::vector<int> suppP;
    for (long x = 0; x < ctx->V; x++) {
        long r = x;
        int c[4];
        for (int mu = 3; mu >= 0; mu--) {
            c[mu] = (int)(r % dims[mu]);
            r /= dims[mu];
        }
        int colour = (c[0] / l + c[1] / l + c[2] / l + c[3] / l) & 1;
        if (colour) continue;
        bool face = false;
        for (int mu = 0; mu < 4; mu++) {
            int cm = c[mu] % l;
            if (cm == 0 || cm == l - 1) face = true;
        }
        if (face) suppP.push_back((int)host_internal_index(ctx, number, c));
    }
    ctx->nP = (long)suppP.size();
    if (cudaMalloc(&ctx->d_blk_nb, sizeof(int) * 8 * nb) != cudaSuccess ||
        cudaMalloc(&ctx->d_blk_org, sizeof(int) * 4 * nb) != cudaSuccess ||
        cudaMalloc(&ctx->d_blk_index, sizeof(int) * nb) != cudaSuccess ||
        cudaMalloc(&ctx->d_suppP, sizeof(int) * (suppP.size() + 1)) != cudaSuccess)
        return fail(DDRW_ENOMEM);
    cudaMemcpy(ctx->d_blk_nb, nbr.data(), sizeof(int) * 8 * nb, cudaMemcpyHostToDevice);
    cudaMemcpy(ctx->d_blk_org, org.data(), sizeof(int) * 4 * nb, cudaMemcpyHostToDevice);
    cudaMemcpy(ctx->d_blk_index, number.data(), sizeof(int) * nb, cudaMemcpyHostToDevice);
    if (!suppP.empty()) cudaMemcpy(ctx->d_suppP, suppP.data(), sizeof(int) * suppP.size(), cudaMemcpyHostToDevice);
    if (cudaMalloc(&ctx->d_nbr, sizeof(int4) * 2 * (size_t)ctx->V) != cudaSuccess ||
        cudaMalloc(&ctx->Ubw32, sizeof(float4) * 12 * (size_t)ctx->V) != cudaSuccess)
        return fail(DDRW_ENOMEM);
    if (cudaHostAlloc(&ctx->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess) return fail(DDRW_ENOMEM);
    *ctx->h_err = 0;
    if (cudaHostGetDevicePointer(&ctx->d_err, ctx->h_err, 0) != cudaSuccess) return fail(DDRW_ECUDA);
    build_nbr_table(ctx);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return fail(DDRW_ECUDA);

    size_t V = ctx->V;
    if (cudaMalloc(&ctx->U64, sizeof(double2) * 36 * V) != cudaSuccess ||
        cudaMalloc(&ctx->U32, sizeof(float4) * 12 * V) != cudaSuccess ||
        cudaMalloc(&ctx->C64, sizeof(double2) * 36 * V) != cudaSuccess ||
        cudaMalloc(&ctx->C32, sizeof(float4) * 18 * V) != cudaSuccess ||
        cudaMalloc(&ctx->U16, sizeof(uint2) * 12 * V) != cudaSuccess ||
        cudaMalloc(&ctx->Ub16, sizeof(uint2) * 12 * V) != cudaSuccess ||
        cudaMalloc(&ctx->C16, sizeof(uint2) * 18 * V) != cudaSuccess ||
        cudaMalloc(&ctx->Cb16, sizeof(uint2) * 18 * V) != cudaSuccess ||
        cudaMalloc(&ctx->Udd, sizeof(float4) * 36 * V) != cudaSuccess ||
        cudaMalloc(&ctx->Cdd, sizeof(float4) * 36 * V) != cudaSuccess)
        return fail(DDRW_ENOMEM);
    if (cudaMallocHost(&ctx->h_pinned, 1 << 20) != cudaSuccess) return fail(DDRW_ENOMEM);
    ctx->h_pinned_bytes = 1 << 20;
    if (cudaGetLastError() != cudaSuccess) return fail(DDRW_ECUDA);
    *out = ctx;
    return DDRW_OK;
}

void ddrw_destroy(ddrw_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->d_blk_nb);
    cudaFree(ctx->d_blk_org);
    cudaFree(ctx->d_blk_index);
    cudaFree(ctx->d_suppP);
    cudaFree(ctx->d_nbr);
    cudaFree(ctx->Ubw32);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    cudaFree(ctx->U64);
    cudaFree(ctx->U32);
    cudaFree(ctx->U64f);
    cudaFree(ctx->U32f);
    cudaFree(ctx->C64);
    cudaFree(ctx->C32);
    cudaFree(ctx->U16);
    cudaFree(ctx->Ub16);
    cudaFree(ctx->C16);
    cudaFree(ctx->Cb16);
    cudaFree(ctx->Udd);
    cudaFree(ctx->Cdd);
    free_inverses(ctx);
    for (auto &kv : ctx->ws) cudaFree(kv.second.p);
    for (auto &r : ctx->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    clear_graphs(ctx);
    for (auto e : ctx->prof_pool) cudaEventDestroy(e);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    for (auto &sd : ctx->cap_streams)
        if (sd) cudaStreamDestroy(sd);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *ddrw_last_error(const ddrw_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

ddrw_status ddrw_suppP_size(ddrw_ctx *ctx, long *n)
{
    if (!ctx || !n) return DDRW_EINVAL;
    *n = ctx->nP;
    return DDRW_OK;
}

ddrw_status ddrw_volume(ddrw_ctx *ctx, long *n)
{
    if (!ctx || !n) return DDRW_EINVAL;
    *n = ctx->V;
    return DDRW_OK;
}

static ddrw_status rebuild(ddrw_ctx *ctx)
{
    if (ctx->cut > 0 && ctx->U64f) {  // the clover term comes from the full field's links
        DDRW_CUDA_CHECK(cudaMemcpyAsync(ctx->U64, ctx->U64f, sizeof(double2) * 36 * (size_t)ctx->V,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
        DDRW_CUDA_CHECK(cudaMemcpyAsync(ctx->U32, ctx->U32f, sizeof(float4) * 12 * (size_t)ctx->V,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
    }
    build_clover(ctx);
    if (ctx->cut > 0) cut_links(ctx);
    build_bw_links(ctx);
    DDRW_CUDA_CHECK(cudaGetLastError());
    // 16-bit copies of the two-row links and the clover term for the FP16 / BF16 inner solves
    f32_to_low(ctx, ctx->U32, ctx->U16, 12L * ctx->V, false);
    f32_to_low(ctx, ctx->U32, ctx->Ub16, 12L * ctx->V, true);
    f32_to_low(ctx, ctx->C32, ctx->C16, 18L * ctx->V, false);
    f32_to_low(ctx, ctx->C32, ctx->Cb16, 18L * ctx->V, true);
    // split copies of links and clover for the double-single residual stencil
    // 36 planes of V elements each: three "fields" of 12 planes
    split64(ctx, ctx->U64, ctx->Udd, ctx->V, 0, 0, ctx->V, 0, 1, 3, 12L * ctx->V);
    split64(ctx, ctx->C64, ctx->Cdd, ctx->V, 0, 0, ctx->V, 0, 1, 3, 12L * ctx->V);
    // in-block inverses of the masses already in use: recomputed in place, so that the captured
    // graphs, which hold their addresses, stay valid; a long list of masses is dropped instead
    if (ctx->inv.size() > (size_t)MAXM + 2) free_inverses(ctx);
    for (auto &mi : ctx->inv) {
        build_inverse(ctx, mi.m, mi);
        f32_to_low(ctx, mi.A32, mi.A16, 18L * ctx->V, false);
        f32_to_low(ctx, mi.A32, mi.Ab16, 18L * ctx->V, true);
    }
    MassInv *mi;
    ddrw_status st = mass_inverse(ctx, ctx->m1, &mi);
    if (st) return st;
    if (ctx->m2 != ctx->m1) st = mass_inverse(ctx, ctx->m2, &mi);
    if (st) return st;
    st = sync(ctx);
    ctx->built = st == DDRW_OK;
    return st;
}

ddrw_status ddrw_load_gauge(ddrw_ctx *ctx, const double *U)
{
    if (!ctx || !U) return set_error(ctx, DDRW_EINVAL, "null argument");
    cudaSetDevice(ctx->device);
    const void *dU;
    ddrw_status st = stage_in(ctx, U, sizeof(double) * 72 * (size_t)ctx->V, "stage_gauge", &dU);
    if (st) return st;
    pack_gauge(ctx, (const double *)dU);
    DDRW_CUDA_CHECK(cudaGetLastError());
    if (ctx->cut > 0) {  // keep the full field's links for the clover term
        if (!ctx->U64f && cudaMalloc(&ctx->U64f, sizeof(double2) * 36 * (size_t)ctx->V) != cudaSuccess)
            return set_error(ctx, DDRW_ENOMEM, "links of the full field");
        if (!ctx->U32f && cudaMalloc(&ctx->U32f, sizeof(float4) * 12 * (size_t)ctx->V) != cudaSuccess)
            return set_error(ctx, DDRW_ENOMEM, "links of the full field");
        DDRW_CUDA_CHECK(cudaMemcpyAsync(ctx->U64f, ctx->U64, sizeof(double2) * 36 * (size_t)ctx->V,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
        DDRW_CUDA_CHECK(cudaMemcpyAsync(ctx->U32f, ctx->U32, sizeof(float4) * 12 * (size_t)ctx->V,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
    }
    ctx->have_gauge = true;
    ctx->built = false;
    // the staging buffer stays for the next configuration (allocating it again would drop the
    // captured graphs, like any workspace allocation)
    return rebuild(ctx);
}

ddrw_status ddrw_set_params(ddrw_ctx *ctx, double csw, double m1, double m2, int antiperiodic_t)
{
    if (!ctx) return DDRW_EINVAL;
    if (!(csw == csw) || !(m1 == m1) || !(m2 == m2)) return set_error(ctx, DDRW_EINVAL, "NaN parameter");
    cudaSetDevice(ctx->device);
    const int ap = antiperiodic_t ? 1 : 0;
    // the same parameters on a built configuration: nothing to recompute
    if (ctx->have_gauge && ctx->built && csw == ctx->csw && m1 == ctx->m1 && m2 == ctx->m2 && ap == ctx->antiperiodic)
        return DDRW_OK;
    ctx->csw = csw;
    ctx->m1 = m1;
    ctx->m2 = m2;
    ctx->antiperiodic = ap;
    ctx->built = false;
    if (!ctx->have_gauge) return DDRW_OK;
    return rebuild(ctx);
}

ddrw_status ddrw_set_solver(ddrw_ctx *ctx, ddrw_prec prec, double tol_outer, double tol_block, int maxiter)
{
    if (!ctx) return DDRW_EINVAL;
    if (prec < DDRW_FP64 || prec > DDRW_MIXED_BF16) return set_error(ctx, DDRW_EINVAL, "unknown precision");
    if (!(tol_outer > 0) || !(tol_block > 0) || maxiter <= 0) return set_error(ctx, DDRW_EINVAL, "bad tolerance");
    ctx->prec = prec;
    ctx->tol_outer = tol_outer;
    ctx->tol_block = tol_block;
    ctx->maxiter = maxiter;
    return DDRW_OK;
}

ddrw_status ddrw_set_dirichlet(ddrw_ctx *ctx, int cut)
{
    if (!ctx) return DDRW_EINVAL;
    if (ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "ddrw_set_dirichlet must precede ddrw_load_gauge");
    if (cut < 0 || (cut > 0 && cut % ctx->l != 0)) return set_error(ctx, DDRW_EINVAL, "cut must be a multiple of the block length");
    for (int mu = 0; mu < 4 && cut > 0; mu++)
        if (ctx->dims[mu] % cut) return set_error(ctx, DDRW_EINVAL, "cut must divide every lattice dimension");
    ctx->cut = cut;
    return DDRW_OK;
}

ddrw_status ddrw_set_max_rhs(ddrw_ctx *ctx, int max_rhs)
{
    if (!ctx) return DDRW_EINVAL;
    if (max_rhs < 0) return set_error(ctx, DDRW_EINVAL, "max_rhs must be >= 0");
    ctx->max_rhs = max_rhs;
    return DDRW_OK;
}

ddrw_status ddrw_block_config(ddrw_ctx *ctx, int form)
{
    if (!ctx) return DDRW_EINVAL;
    if (form < -1 || form > 2) return set_error(ctx, DDRW_EINVAL, "block-solver launch shape must be -1, 0, 1 or 2");
    ctx->blk_form = form;
    return DDRW_OK;
}

ddrw_status ddrw_set_low_precision(ddrw_ctx *ctx, int reliable_updates, int block_solves_16bit)
{
    if (!ctx) return DDRW_EINVAL;
    ctx->reliable16 = reliable_updates != 0;
    ctx->block16 = block_solves_16bit != 0;
    clear_graphs(ctx);
    return DDRW_OK;
}

ddrw_status ddrw_fuse_reductions(ddrw_ctx *ctx, int enable)
{
    if (!ctx) return DDRW_EINVAL;
    ctx->fuse_dots = enable != 0;
    clear_graphs(ctx);  // captured iterations keep the kernels they were captured with
    return DDRW_OK;
}

ddrw_status ddrw_set_block_solver(ddrw_ctx *ctx, int method)
{
    if (!ctx) return DDRW_EINVAL;
    if (method < 0 || method > 1) return set_error(ctx, DDRW_EINVAL, "block solver method must be 0 or 1");
    ctx->block_method = method;
    return DDRW_OK;
}

ddrw_status ddrw_set_outer_solver(ddrw_ctx *ctx, int method, int ncy, int nmr, int nkv)
{
    if (!ctx) return DDRW_EINVAL;
    if (method < 0 || method > 1 || ncy < 1 || ncy > 16 || nmr < 1 || nmr > 32 || nkv < 1 || nkv > 16)
        return set_error(ctx, DDRW_EINVAL, "bad outer solver setting");
    ctx->outer_method = method;
    ctx->sap_ncy = ncy;
    ctx->sap_nmr = nmr;
    ctx->sap_nkv = nkv;
    return DDRW_OK;
}

ddrw_status ddrw_apply_block(ddrw_ctx *ctx, int rows, int cols, double m, const double *in, double *out, int nrhs)
{
    if (!ctx || !in || !out || nrhs <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (rows < 0 || rows > 2 || cols < 0 || cols > 2) return set_error(ctx, DDRW_EINVAL, "bad colour");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    size_t ubytes = sizeof(double) * 24 * (size_t)ctx->V * nrhs;
    size_t fbytes = sizeof(double2) * 12 * (size_t)ctx->V * nrhs;
    const void *din;
    void *dout;
    bool host_out;
    double2 *fin, *fout;
    ddrw_status st;
    if ((st = stage_in(ctx, in, ubytes, "stage_in", &din))) return st;
    if ((st = stage_out(ctx, out, ubytes, "stage_out", &dout, &host_out))) return st;
    if ((st = workspace(ctx, "api_f0", fbytes, (void **)&fin))) return st;
    if ((st = workspace(ctx, "api_f1", fbytes, (void **)&fout))) return st;
    pack_spinor64(ctx, (const double *)din, fin, nrhs);

    DslashCall c;
    c.in = fin;
    c.x = fin;
    c.out = fout;
    c.rstride = 12 * ctx->V;
    c.nrhs = nrhs;
    c.masses[0] = m;
    c.alpha = 1.0;
    c.beta = -0.5;
    c.par0 = 0;
    c.npar = 2;
    if (rows != DDRW_ALL && cols != DDRW_ALL) {
        DDRW_CUDA_CHECK(cudaMemsetAsync(fout, 0, fbytes, ctx->stream));
        c.blk0 = rows == DDRW_BLACK ? 0 : ctx->nblk_c;
        c.nblk = ctx->nblk_c;
        if (rows == cols) {
            c.diag = 1;
            c.hopsel = 1;
            dslash64(ctx, c);
        } else {
            hop_between64(ctx, rows, fin, fout, nrhs, -0.5);  // fout is zero on every row (above)
        }
    } else {
        if (cols != DDRW_ALL) zero_colour64(ctx, fin, 1 - cols, nrhs);
        c.diag = 1;
        c.hopsel = 0;
        c.blk0 = 0;
        c.nblk = ctx->nblk;
        dslash64(ctx, c);
        if (rows != DDRW_ALL) zero_colour64(ctx, fout, 1 - rows, nrhs);
    }
    unpack_spinor64(ctx, fout, (double *)dout, nrhs);
    if ((st = finish_out(ctx, out, dout, ubytes, host_out))) return st;
    return sync(ctx);
}

ddrw_status ddrw_apply_D(ddrw_ctx *ctx, double m, const double *in, double *out, int nrhs)
{
    return ddrw_apply_block(ctx, DDRW_ALL, DDRW_ALL, m, in, out, nrhs);
}

ddrw_status ddrw_apply_D_low(ddrw_ctx *ctx, ddrw_prec prec, double m, int post, const double *in, double *out,
                             int nrhs)
{
    if (!ctx || !in || !out || nrhs <= 0 || (prec != DDRW_MIXED_FP32 && prec != DDRW_MIXED_FP16 && prec != DDRW_MIXED_BF16))
        return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    size_t ubytes = sizeof(double) * 24 * (size_t)ctx->V * nrhs;
    size_t fbytes = sizeof(double2) * 12 * (size_t)ctx->V * nrhs;
    const void *din;
    void *dout;
    bool host_out;
    double2 *fin, *fout;
    ddrw_status st;
    if ((st = stage_in(ctx, in, ubytes, "stage_in", &din))) return st;
    if ((st = stage_out(ctx, out, ubytes, "stage_out", &dout, &host_out))) return st;
    if ((st = workspace(ctx, "api_f0", fbytes, (void **)&fin))) return st;
    if ((st = workspace(ctx, "api_f1", fbytes, (void **)&fout))) return st;
    pack_spinor64(ctx, (const double *)din, fin, nrhs);
    if (prec == DDRW_MIXED_FP32) st = apply_low<PrecS>(ctx, m, post != 0, fin, fout, nrhs);
    else if (prec == DDRW_MIXED_FP16) st = apply_low<PrecH>(ctx, m, post != 0, fin, fout, nrhs);
    else st = apply_low<PrecB>(ctx, m, post != 0, fin, fout, nrhs);
    if (st) return st;
    unpack_spinor64(ctx, fout, (double *)dout, nrhs);
    if ((st = finish_out(ctx, out, dout, ubytes, host_out))) return st;
    return sync(ctx);
}

ddrw_status ddrw_apply_D_ds(ddrw_ctx *ctx, double m, const double *in, double *out, int nrhs)
{
    if (!ctx || !in || !out || nrhs <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    size_t ubytes = sizeof(double) * 24 * (size_t)ctx->V * nrhs;
    size_t fbytes = sizeof(double2) * 12 * (size_t)ctx->V * nrhs;
    const void *din;
    void *dout;
    bool host_out;
    double2 *fin, *fout;
    ddrw_status st;
    if ((st = stage_in(ctx, in, ubytes, "stage_in", &din))) return st;
    if ((st = stage_out(ctx, out, ubytes, "stage_out", &dout, &host_out))) return st;
    if ((st = workspace(ctx, "api_f0", fbytes, (void **)&fin))) return st;
    if ((st = workspace(ctx, "api_f1", fbytes, (void **)&fout))) return st;
    pack_spinor64(ctx, (const double *)din, fin, nrhs);
    DslashCall c;
    c.in = fin;
    c.x = fin;
    c.out = fout;
    c.rstride = 12 * ctx->V;
    c.nrhs = nrhs;
    c.masses[0] = m;
    c.alpha = 1.0;
    c.beta = -0.5;
    c.diag = 1;
    c.par0 = 0;
    c.npar = 2;
    c.blk0 = 0;
    c.nblk = ctx->nblk;
    if ((st = residual_stencil(ctx, c, true))) return st;
    unpack_spinor64(ctx, fout, (double *)dout, nrhs);
    if ((st = finish_out(ctx, out, dout, ubytes, host_out))) return st;
    return sync(ctx);
}

}  // extern "C"
