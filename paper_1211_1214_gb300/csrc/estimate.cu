// estimate.cu -- the stochastic estimate of 1/det(Mh^dag Mh) (Eq. 3; Eq. 8 with N = 1) for the
// Schur complement A(m) = P Dhat(m) P (Sec. 1), and the entry points built on it:
//
//   noise (K3)   eta_k = sqrt(-ln u1) exp(2 pi i u2), u from Philox4x32-10 (counter (k, hit, 0, 0))
//   r (K9)       r = (A(m1) - A(m2)) eta = dm P D_bb(m1)^-1 [D_bw a12 + D_bb(m2)^-1 D_bw a2],
//                u = D_wb eta, a2 = D_ww(m2)^-1 u, a12 = D_ww(m1)^-1 a2      (resolvent form)
//   delta        delta = A(m2)^-1 r = r - P x_b,  D(m2) x = (0_b ; D_wb r)     (Dhat^-1 = 1 - P Dcal_bw D_wb)
//   e (K10)      e = ||delta||^2 + 2 Re <eta, delta>  (= ||Mh eta||^2 - ||eta||^2 without cancellation)
//
// Right-hand sides: nmass target masses x nhit noise vectors, slot-major (rhs = k * nhit + j uses
// m2[k] and eta_j).  All fields are FP64; the solves run in the context's precision.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "blas.cuh"
#include "ctx.h"

namespace ddrw {

// ----------------------------------------------------------------------------- Philox4x32-10

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; round++) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// eta for packed component k of hit h -> internal field (and optionally the packed output)
// (dparams, if given: {seed, hit offset} read from device memory, so that a replayed graph draws new noise)
__global__ void k_noise(long V, long nP, const int *__restrict__ idx, uint32_t k0, uint32_t k1, uint64_t hit0,
                        int nhit, int nrep, double2 *field, double *packed, const uint64_t *dparams = nullptr)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 12 * nP) return;
    int h = blockIdx.y;
    if (dparams) {
        k0 = (uint32_t)(dparams[0] & 0xffffffffu);
        k1 = (uint32_t)(dparams[0] >> 32);
        hit0 = dparams[1];
    }
    uint32_t c[4] = {(uint32_t)k, (uint32_t)(hit0 + (uint64_t)h), 0u, 0u};
    philox4x32_10(c, k0, k1);
    double u1 = ((double)c[0] + 1.0) * (1.0 / 4294967296.0);
    double u2 = (double)c[1] * (1.0 / 4294967296.0);
    double rho = sqrt(-log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    double2 z = make_double2(rho * cs, rho * sn);
    long j = k / 12;
    int comp = (int)(k - j * 12);
    long s = idx[j];
    if (field)
        for (int rep = 0; rep < nrep; rep++) field[((long)(rep * nhit + h) * 12 + comp) * V + s] = z;
    if (packed) {
        packed[((long)h * nP * 12 + k) * 2] = z.x;
        packed[((long)h * nP * 12 + k) * 2 + 1] = z.y;
    }
}

// replicate rhs j of a nhit-field into slots: f[k * nhit + j] = f[j], k = 1 .. nrep-1
__global__ void k_replicate(long n, long nhit, int nrep, double2 *f)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nhit) return;
    for (int k = 1; k < nrep; k++) f[(long)k * n * nhit + i] = f[i];
}

// r <- dm[slot] * P r on black sites (zero off supp P); also zero every white site
template <int BL>
__global__ void k_project_P(GeomDev g, double2 *r, int rpm, const double *dm, long rs)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    long s = i;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    double f = 0.0;
    if (st.blk < g.nblk_c) {
        bool face = false;
#pragma unroll
        for (int mu = 0; mu < 4; mu++) face |= (st.c[mu] == 0 || st.c[mu] == BL - 1);
        if (face) f = dm[blockIdx.y / rpm];
    }
    double2 *o = r + (long)blockIdx.y * rs + s;
    for (int k = 0; k < 12; k++) {
        double2 v = o[(long)k * g.V];
        o[(long)k * g.V] = make_double2(f * v.x, f * v.y);
    }
}

// delta = P (r - x) on supp P, zero elsewhere
template <int BL>
__global__ void k_delta(GeomDev g, const double2 *r, const double2 *x, double2 *d, long rs, int g5x = 0)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    bool in = false;
    if (st.blk < g.nblk_c)
#pragma unroll
        for (int mu = 0; mu < 4; mu++) in |= (st.c[mu] == 0 || st.c[mu] == BL - 1);
    long o = (long)blockIdx.y * rs + s;
    for (int k = 0; k < 12; k++) {
        double2 a = r[o + (long)k * g.V], b = x[o + (long)k * g.V];
        if (g5x && k >= 6) b = make_double2(-b.x, -b.y);  // g5 = diag(1, 1, -1, -1) on x
        d[o + (long)k * g.V] = in ? make_double2(a.x - b.x, a.y - b.y) : make_double2(0.0, 0.0);
    }
}

#define DISPATCH_BL(ctx, KERNEL, GRID, BLOCK, ...)                                                        \
    ++(ctx)->launches;                                                                                    \
    switch ((ctx)->l) {                                                                                   \
    case 2: KERNEL<2><<<GRID, BLOCK, 0, (ctx)->stream>>>(__VA_ARGS__); break;                             \
    case 4: KERNEL<4><<<GRID, BLOCK, 0, (ctx)->stream>>>(__VA_ARGS__); break;                             \
    case 6: KERNEL<6><<<GRID, BLOCK, 0, (ctx)->stream>>>(__VA_ARGS__); break;                             \
    default: KERNEL<8><<<GRID, BLOCK, 0, (ctx)->stream>>>(__VA_ARGS__); break;                            \
    }

static void noise_launch(ddrw_ctx *ctx, uint64_t seed, uint64_t hit0, int nhit, int nrep, double2 *field, double *packed,
                         const uint64_t *dparams = nullptr)
{
    dim3 grid((unsigned)((12 * ctx->nP + 255) / 256), (unsigned)nhit);
    ++ctx->launches;
    k_noise<<<grid, 256, 0, ctx->stream>>>(ctx->V, ctx->nP, ctx->d_suppP, (uint32_t)(seed & 0xffffffffu),
                                           (uint32_t)(seed >> 32), hit0, nhit, nrep, field, packed, dparams);
}

// ---- supports of the operator variants of Fig. 1's comparison (ddrw_estimate_variant)

// idx[i] = internal index of the i-th site of the support in lexicographic order: every site
// (even_only = 0) or the even sites (t + x + y + z even; Z even, so every z-row holds Z/2 of them)
template <int BL>
__global__ void k_support(GeomDev g, int even_only, long n, int *idx)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int t, x, y, z;
    if (even_only) {
        const int zh = g.L[3] / 2;
        long row = i / zh;
        int j = (int)(i - row * zh);
        y = (int)(row % g.L[2]);
        row /= g.L[2];
        x = (int)(row % g.L[1]);
        t = (int)(row / g.L[1]);
        z = 2 * j + ((t + x + y) & 1);
    } else {
        long r = i;
        z = (int)(r % g.L[3]);
        r /= g.L[3];
        y = (int)(r % g.L[2]);
        r /= g.L[2];
        x = (int)(r % g.L[1]);
        t = (int)(r / g.L[1]);
    }
    idx[i] = (int)internal_index<BL>(g, t, x, y, z);
}

// caller's packed noise (nhit vectors of 12 n complex components, support order) -> fields
__global__ void k_scatter_packed(const int *__restrict__ idx, long n, const double *__restrict__ packed, long V,
                                 double2 *field)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 12 * n) return;
    const int h = blockIdx.y;
    const long j = k / 12;
    const int comp = (int)(k - j * 12);
    const double *p = packed + ((long)h * 12 * n + k) * 2;
    field[((long)h * 12 + comp) * V + idx[j]] = make_double2(p[0], p[1]);
}

// y = g5 x on every site (spins 2, 3 flipped) for nrhs full FP64 fields
__global__ void k_gamma5_field(long n12V, long V, int nrhs, const double2 *x, double2 *y)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n12V * nrhs) return;
    long e = i % n12V;
    double2 v = x[i];
    y[i] = e / V >= 6 ? make_double2(-v.x, -v.y) : v;
}

// out_e = S(m) in_e with S = A_ee - 1/4 H_eo A_oo^-1 H_oe (FP64, all blocks; tmp holds A_oo^-1 H_oe in)
static ddrw_status apply_schur_eo64(ddrw_ctx *ctx, double m, const double2 *in, double2 *out, double2 *tmp,
                                    int nrhs)
{
    MassInv *mi;
    ddrw_status st = mass_inverse(ctx, m, &mi);
    if (st) return st;
    DslashCall c;
    c.in = in;
    c.out = tmp;
    c.rstride = 12 * ctx->V;
    c.nrhs = nrhs;
    c.masses[0] = m;
    c.Ainv[0] = mi->A64;
    c.beta = 1.0;
    c.post = 1;
    c.par0 = 1;
    c.npar = 1;
    c.blk0 = 0;
    c.nblk = ctx->nblk;
    dslash64(ctx, c);
    DslashCall d = c;
    d.in = tmp;
    d.x = in;
    d.out = out;
    d.alpha = 1.0;
    d.beta = -0.25;
    d.diag = 1;
    d.post = 0;
    d.par0 = 0;
    dslash64(ctx, d);
    return DDRW_OK;
}

// hop between blocks: out (colour rows) += -1/2 H_{rows <- other colour} in (out is zero on those
// rows before: every caller clears it); other rows untouched
static void hop_between(ddrw_ctx *ctx, int rows, const double2 *in, double2 *out, int nrhs)
{
    hop_between64(ctx, rows, in, out, nrhs, -0.5);
}

static double elapsed(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

static void fill_info(ddrw_solve_info *info, const SolveStats &s, double secs)
{
    if (!info) return;
    info->iters_outer = s.outer_iters;
    info->cycles = s.outer_cycles;
    info->fp64_dslash_calls = s.fp64_dslash_full;
    info->block_iters_max = s.block_iters_max;
    info->iters_inner_total = (int)std::min<long>(s.block_iters_total, 2147483647L);
    info->true_rel_residual = s.outer_rel_residual;
    info->seconds = secs;
}

// r = (A(m1) - A(m2[slot])) eta for nrhs = nmass * nhit fields (eta: FP64 full fields, zero off
// supp P).  Work fields f[0..2] (FP64, nrhs each).  Result in r.
static ddrw_status apply_dA_fields(ddrw_ctx *ctx, const MassSet &m2s, const MassSet &m1s, const double2 *eta,
                                   double2 *r, double2 *const *f, int nrhs, SolveStats *stats)
{
    const bool mixed = ctx->prec != DDRW_FP64;
    const size_t fb = sizeof(double2) * 12 * ctx->V * nrhs;
    double2 *u = f[0], *a2 = f[1], *a12 = r, *c2 = f[2];
    ddrw_status st;
    DDRW_CUDA_CHECK(cudaMemsetAsync(u, 0, fb, ctx->stream));
    hop_between(ctx, DDRW_WHITE, eta, u, nrhs);  // u = D_wb eta
    if ((st = block_solve64(ctx, DDRW_WHITE, m2s, u, a2, nrhs, ctx->tol_block, ctx->maxiter, ctx->prec, stats))) return st;
    if ((st = block_solve64(ctx, DDRW_WHITE, m1s, a2, a12, nrhs, ctx->tol_block, ctx->maxiter, ctx->prec, stats))) return st;
    // c = D_bw a12 (into u, black rows), c2 = D_bw a2
    DDRW_CUDA_CHECK(cudaMemsetAsync(u, 0, fb, ctx->stream));
    DDRW_CUDA_CHECK(cudaMemsetAsync(c2, 0, fb, ctx->stream));
    hop_between(ctx, DDRW_BLACK, a12, u, nrhs);
    hop_between(ctx, DDRW_BLACK, a2, c2, nrhs);
    // t = D_bb(m2)^-1 c2 (into a2); w = c + t (into u)
    if ((st = block_solve64(ctx, DDRW_BLACK, m2s, c2, a2, nrhs, ctx->tol_block, ctx->maxiter, ctx->prec, stats))) return st;
    Blas<PrecD>::axpby(ctx, VecRange{ctx->V, 0, ctx->V, 12 * ctx->V, nrhs}, 1.0, a2, 1.0, u);
    // r = dm P D_bb(m1)^-1 w
    DDRW_CUDA_CHECK(cudaMemsetAsync(r, 0, fb, ctx->stream));
    if ((st = block_solve64(ctx, DDRW_BLACK, m1s, u, r, nrhs, ctx->tol_block, ctx->maxiter, ctx->prec, stats))) return st;
    double *dm;
    if ((st = workspace(ctx, "est_dm", sizeof(double) * MAXM, (void **)&dm))) return st;
    if (!ctx->devctl) {  // a captured estimate finds the mass differences written before the capture
        double hdm[MAXM];
        for (int k = 0; k < MAXM; k++) hdm[k] = k < m2s.n ? m1s.m[k < m1s.n ? k : 0] - m2s.m[k] : 0.0;
        DDRW_CUDA_CHECK(cudaMemcpyAsync(dm, hdm, sizeof(hdm), cudaMemcpyHostToDevice, ctx->stream));
    }
    GeomDev g = geom_dev(ctx);
    int rpm = (nrhs + m2s.n - 1) / m2s.n;
    dim3 grid((unsigned)((ctx->V + 127) / 128), (unsigned)nrhs);
    DISPATCH_BL(ctx, k_project_P, grid, 128, g, r, rpm, dm, 12 * ctx->V);
    return DDRW_OK;
}

// delta = A(m)^-1 b for FP64 fields b supported on supp P; work fields f[0], f[1]
static ddrw_status solve_schur_fields(ddrw_ctx *ctx, const MassSet &ms, const double2 *b, double2 *delta,
                                      double2 *const *f, int nrhs, SolveStats *stats)
{
    const size_t fb = sizeof(double2) * 12 * ctx->V * nrhs;
    double2 *src = f[0], *x = f[1];
    DDRW_CUDA_CHECK(cudaMemsetAsync(src, 0, fb, ctx->stream));
    hop_between(ctx, DDRW_WHITE, b, src, nrhs);  // (0_b ; D_wb b)
    ddrw_status st = full_solve64(ctx, ms, src, x, nrhs, ctx->tol_outer, ctx->maxiter, ctx->prec, stats);
    if (st && st != DDRW_ENOCONV) return st;
    GeomDev g = geom_dev(ctx);
    dim3 grid((unsigned)((ctx->V + 127) / 128), (unsigned)nrhs);
    DISPATCH_BL(ctx, k_delta, grid, 128, g, b, x, delta, 12 * ctx->V);
    return st;
}

static ddrw_status fields(ddrw_ctx *ctx, const char *prefix, int n, int nrhs, double2 **out)
{
    for (int k = 0; k < n; k++) {
        char nm[32];
        snprintf(nm, sizeof nm, "%s%d", prefix, k);
        ddrw_status st = workspace(ctx, nm, sizeof(double2) * 12 * ctx->V * nrhs, (void **)&out[k]);
        if (st) return st;
    }
    return DDRW_OK;
}

// ---- the whole estimate chunk as one CUDA graph
//
// With ctx->use_graphs, Philox noise and no delta output, the first call of a chunk shape runs
// eagerly (it tunes the stencil and allocates every buffer), the second captures the chunk with
// the solvers' device-controlled forms (every defect-correction cycle and Krylov loop a
// conditional while-node whose condition a one-thread kernel sets from device norms, each with an
// iteration cap), and later calls replay it: the noise seed and hit offset go in through device
// memory, the exponents and the statistics come back after one synchronisation.

using EstKey = std::array<uintptr_t, 24>;

static EstKey est_key(const ddrw_ctx *ctx, int nmass, const double *ma, const double *m2, int nhit, bool distinct)
{
    EstKey k{};
    k[0] = (uintptr_t)nmass;
    k[1] = (uintptr_t)nhit;
    k[2] = distinct;
    k[3] = (uintptr_t)ctx->prec;
    k[4] = (uintptr_t)ctx->maxiter;
    memcpy(&k[5], &ctx->tol_block, sizeof(double));
    memcpy(&k[6], &ctx->tol_outer, sizeof(double));
    for (int i = 0; i < nmass && i < MAXM; i++) {
        memcpy(&k[7 + 2 * i], &ma[i], sizeof(double));
        memcpy(&k[8 + 2 * i], &m2[i], sizeof(double));
    }
    return k;
}

static ddrw_status apply_dA_fields(ddrw_ctx *ctx, const MassSet &m2s, const MassSet &m1s, const double2 *eta,
                                   double2 *r, double2 *const *f, int nrhs, SolveStats *stats);
static ddrw_status solve_schur_fields(ddrw_ctx *ctx, const MassSet &ms, const double2 *b, double2 *delta,
                                      double2 *const *f, int nrhs, SolveStats *stats);

// the device work of one chunk (the same calls as the eager chunk, noise parameters from device)
static ddrw_status chunk_body(ddrw_ctx *ctx, int nmass, int nhit, bool distinct, const MassSet &m2s,
                              const MassSet &m1s, double2 *const *F, const uint64_t *dparams, double *red)
{
    const int nrhs = nmass * nhit;
    double2 *eta = F[0], *r = F[1], *delta = F[2];
    double2 *work[3] = {F[3], F[4], F[2]};
    double2 *w2[2] = {F[3], F[4]};
    DDRW_CUDA_CHECK(cudaMemsetAsync(eta, 0, sizeof(double2) * 12 * ctx->V * nrhs, ctx->stream));
    if (distinct) noise_launch(ctx, 0, 0, nrhs, 1, eta, nullptr, dparams);
    else noise_launch(ctx, 0, 0, nhit, nmass, eta, nullptr, dparams);
    ddrw_status st;
    if ((st = apply_dA_fields(ctx, m2s, m1s, eta, r, work, nrhs, nullptr))) return st;
    st = solve_schur_fields(ctx, m2s, r, delta, w2, nrhs, nullptr);
    if (st && st != DDRW_ENOCONV) return st;
    long vbh = (long)ctx->l * ctx->l * ctx->l * ctx->l / 2, nc = (long)ctx->nblk_c * vbh;
    for (int p = 0; p < 2; p++)
        if ((st = Blas<PrecD>::norm_dot(ctx, VecRange{ctx->V, p * ctx->vh, nc, 12 * ctx->V, nrhs}, delta, eta,
                                        red + 3 * p * nrhs)))
            return st;
    return DDRW_OK;
}

static ddrw_status chunk_capture(ddrw_ctx *ctx, int nmass, const double *ma, const double *m2, int nhit, bool distinct,
                                 const MassSet &m2s, const MassSet &m1s, double2 *const *F, EstGraph &out)
{
    const int nrhs = nmass * nhit;
    ddrw_status st;
    void *p;
    double *red, *dm;
    uint64_t *dparams;
    // every buffer the capture uses, allocated now
    if ((st = block_solve_dc_prepare(ctx, nrhs))) return st;
    if ((st = full_solve_dc_prepare(ctx, nrhs))) return st;
    if ((st = workspace(ctx, "dc_stats", sizeof(DcStats), &p))) return st;
    ctx->dc = (DcStats *)p;
    if ((st = workspace(ctx, "dc_noise", sizeof(uint64_t) * 2, (void **)&dparams))) return st;
    if ((st = workspace(ctx, "est_red", sizeof(double) * 6 * nrhs, (void **)&red))) return st;
    if ((st = workspace(ctx, "est_dm", sizeof(double) * MAXM, (void **)&dm))) return st;
    double hdm[MAXM];
    for (int k = 0; k < MAXM; k++) hdm[k] = k < m2s.n ? m1s.m[k < m1s.n ? k : 0] - m2s.m[k] : 0.0;
    DDRW_CUDA_CHECK(cudaMemcpyAsync(dm, hdm, sizeof(hdm), cudaMemcpyHostToDevice, ctx->stream));
    DDRW_SYNC(ctx);

    DDRW_CUDA_CHECK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed));
    ctx->devctl = true;
    ctx->dc_loops = 0;
    ctx->cap_depth = 0;
    ctx->cap_nested[0] = 0;
    ctx->cap_loop_launches.clear();
    const long l0 = ctx->launches;
    cudaError_t em = cudaMemsetAsync(ctx->dc, 0, sizeof(DcStats), ctx->stream);
    st = em == cudaSuccess ? chunk_body(ctx, nmass, nhit, distinct, m2s, m1s, F, dparams, red)
                           : set_cuda_error(ctx, em, "cudaMemsetAsync(stats)", __FILE__, __LINE__);
    ctx->devctl = false;
    const long captured = ctx->launches - l0;
    ctx->launches = l0;  // nothing ran yet
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (st || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st ? st : set_cuda_error(ctx, e, "cudaStreamEndCapture(estimate)", __FILE__, __LINE__);
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(g);
        return set_cuda_error(ctx, ei, "cudaGraphInstantiate(estimate)", __FILE__, __LINE__);
    }
    out.graph = g;
    out.exec = exec;
    out.top_launches = captured - ctx->cap_nested[0];
    out.loop_launches = ctx->cap_loop_launches;
    return DDRW_OK;
}

static ddrw_status chunk_replay(ddrw_ctx *ctx, const EstGraph &eg, int nrhs, uint64_t seed, uint64_t hit0,
                                double *exponents, double *e1, SolveStats &stats)
{
    ddrw_status st;
    void *p;
    double *red;
    uint64_t *dparams;
    if ((st = workspace(ctx, "dc_stats", sizeof(DcStats), &p))) return st;
    if ((st = workspace(ctx, "dc_noise", sizeof(uint64_t) * 2, (void **)&dparams))) return st;
    if ((st = workspace(ctx, "est_red", sizeof(double) * 6 * nrhs, (void **)&red))) return st;
    const uint64_t prm[2] = {seed, hit0};
    DDRW_CUDA_CHECK(cudaMemcpyAsync(dparams, prm, sizeof(prm), cudaMemcpyHostToDevice, ctx->stream));
    DDRW_CUDA_CHECK(cudaGraphLaunch(eg.exec, ctx->stream));
    ++ctx->graph_launches;
    std::vector<double> h(6 * nrhs);
    DcStats d;
    DDRW_CUDA_CHECK(cudaMemcpyAsync(h.data(), red, sizeof(double) * 6 * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    DDRW_CUDA_CHECK(cudaMemcpyAsync(&d, p, sizeof(DcStats), cudaMemcpyDeviceToHost, ctx->stream));
    if ((st = sync(ctx))) return st;
    long launches = eg.top_launches;
    for (auto &sl : eg.loop_launches) launches += sl.second * d.loop_iters[sl.first];
    ctx->launches += launches;
    stats.block_iters_max = std::max(stats.block_iters_max, d.block_iters_max);
    stats.block_iters_total += d.block_iters_total;
    stats.block_cycles += d.block_cycles;
    stats.block_rel_residual = std::max(stats.block_rel_residual, d.block_rel_residual);
    stats.fp64_dslash_half += d.fp64_dslash_half;
    stats.outer_iters += d.outer_iters;
    stats.outer_cycles = d.outer_cycles;
    stats.fp64_dslash_full += d.fp64_dslash_full;
    stats.outer_rel_residual = d.outer_rel_residual;
    for (int rr = 0; rr < nrhs; rr++) {
        double nn = h[3 * rr] + h[3 * nrhs + 3 * rr], dr = h[3 * rr + 1] + h[3 * nrhs + 3 * rr + 1];
        double di = h[3 * rr + 2] + h[3 * nrhs + 3 * rr + 2];
        exponents[rr] = nn + 2.0 * dr;
        if (e1) {
            e1[2 * rr] = dr;
            e1[2 * rr + 1] = -di;
        }
    }
    if (d.nan) return set_error(ctx, DDRW_ENUMERIC, "NaN in a solve of the captured estimate");
    if (d.noconv) return set_error(ctx, DDRW_ENOCONV, "a solve of the captured estimate missed its tolerance");
    return DDRW_OK;
}

// One chunk of the estimate: nmass target masses x nhit noise vectors as nrhs = nmass * nhit
// right-hand sides; writes the FP64 exponents e[k * nhit + j].  eta_user (packed, nhit vectors)
// or the Philox noise of hits hit0 .. hit0 + nhit - 1.
//
// Slot k pairs the masses (ma[k], mb[k]): Mh = A(mb)^-1 A(ma) (the sweep uses ma = m1 for every slot,
// the mass interpolation of Eq. 8 ma = m_{i-1}, mb = m_i).  With distinct_noise every slot draws its
// own noise vectors (hits hit0 + k * nhit + j), else all slots share hits hit0 + j.  e1 (optional,
// 2 doubles per rhs) receives the one-flavour exponent eta^dag (Mh - 1) eta = <eta, delta> (Eq. 11).
static ddrw_status estimate_chunk(ddrw_ctx *ctx, int nmass, const double *ma, const double *m2, int nhit,
                                  uint64_t seed, uint64_t hit0, bool distinct_noise, const double *eta_user,
                                  double *exponents, double *e1, double *delta_user, SolveStats &stats)
{
    const int nrhs = nmass * nhit;
    MassSet m2s, m1s;
    ddrw_status st;
    if ((st = make_massset(ctx, nmass, m2, &m2s))) return st;
    if ((st = make_massset(ctx, nmass, ma, &m1s))) return st;
    double2 *F[5];
    if ((st = fields(ctx, "est_f", 5, nrhs, F))) return st;
    // the whole chunk as a graph: captured on the second call of this shape, replayed later
    const bool graphable = ctx->use_graphs && ctx->use_est_graphs && !eta_user && !delta_user && !ctx->devctl;
    EstKey key{};
    if (graphable) {
        key = est_key(ctx, nmass, ma, m2, nhit, distinct_noise);
        auto it = ctx->est_graphs.find(key);
        if (it == ctx->est_graphs.end() && ctx->est_seen.count(key)) {
            EstGraph eg;
            if ((st = chunk_capture(ctx, nmass, ma, m2, nhit, distinct_noise, m2s, m1s, F, eg))) return st;
            it = ctx->est_graphs.emplace(key, eg).first;
        }
        if (it != ctx->est_graphs.end())
            return chunk_replay(ctx, it->second, nrhs, seed, hit0, exponents, e1, stats);
    }
    double2 *eta = F[0], *r = F[1], *delta = F[2];
    double2 *work[3] = {F[3], F[4], F[2]};
    const size_t pbytes = sizeof(double) * 24 * ctx->nP;
    // eta for every slot
    if (eta_user) {
        const void *d;
        if ((st = stage_in(ctx, eta_user, pbytes * nhit, "stage_eta", &d))) return st;
        unpack_P64(ctx, (const double *)d, eta, nhit);
        long n = 12 * ctx->V;
        ++ctx->launches;
        if (nmass > 1) k_replicate<<<(unsigned)((n * nhit + 255) / 256), 256, 0, ctx->stream>>>(n, nhit, nmass, eta);
    } else {
        DDRW_CUDA_CHECK(cudaMemsetAsync(eta, 0, sizeof(double2) * 12 * ctx->V * nrhs, ctx->stream));
        if (distinct_noise) noise_launch(ctx, seed, hit0, nrhs, 1, eta, nullptr);
        else noise_launch(ctx, seed, hit0, nhit, nmass, eta, nullptr);
    }
    ddrw_status conv = DDRW_OK;
    if ((st = apply_dA_fields(ctx, m2s, m1s, eta, r, work, nrhs, &stats))) return st;
    double2 *w2[2] = {F[3], F[4]};
    st = solve_schur_fields(ctx, m2s, r, delta, w2, nrhs, &stats);
    if (st == DDRW_ENOCONV) conv = st;
    else if (st) return st;
    // e = ||delta||^2 + 2 Re <eta, delta> over the black sites
    double *red;
    if ((st = workspace(ctx, "est_red", sizeof(double) * 6 * nrhs, (void **)&red))) return st;
    long vbh = (long)ctx->l * ctx->l * ctx->l * ctx->l / 2, nc = (long)ctx->nblk_c * vbh;
    for (int p = 0; p < 2; p++)
        if ((st = Blas<PrecD>::norm_dot(ctx, VecRange{ctx->V, p * ctx->vh, nc, 12 * ctx->V, nrhs}, delta, eta,
                                        red + 3 * p * nrhs)))
            return st;
    std::vector<double> h(6 * nrhs);
    DDRW_CUDA_CHECK(cudaMemcpyAsync(h.data(), red, sizeof(double) * 6 * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    if (delta_user) {
        void *dd;
        bool host;
        if ((st = stage_out(ctx, delta_user, pbytes * nrhs, "stage_delta", &dd, &host))) return st;
        pack_P64(ctx, delta, (double *)dd, nrhs);
        if ((st = finish_out(ctx, delta_user, dd, pbytes * nrhs, host))) return st;
    }
    if ((st = sync(ctx))) return st;
    if (graphable) ctx->est_seen[key] = 1;  // after the eager run: its allocations clear the table
    for (int rr = 0; rr < nrhs; rr++) {
        // h: |delta|^2, Re sum conj(delta) eta, Im sum conj(delta) eta (two parities)
        double nn = h[3 * rr] + h[3 * nrhs + 3 * rr], dr = h[3 * rr + 1] + h[3 * nrhs + 3 * rr + 1];
        double di = h[3 * rr + 2] + h[3 * nrhs + 3 * rr + 2];
        exponents[rr] = nn + 2.0 * dr;
        if (e1) {  // <eta, delta> = conj(sum conj(delta) eta)
            e1[2 * rr] = dr;
            e1[2 * rr + 1] = -di;
        }
    }
    return conv;
}

// The forward chain of the estimate for the force: the noise field (nhit rhs), delta = A(m2)^-1 r
// and the exponents, for the context's m1 and m2 (copies of the estimate's work fields).
ddrw_status estimate_fields_for_force(ddrw_ctx *ctx, int nhit, uint64_t seed, uint64_t hit0, const double *eta_user,
                                      double2 *eta_out, double2 *delta_out, double *exponents, SolveStats &stats)
{
    ddrw_status st = estimate_chunk(ctx, 1, &ctx->m1, &ctx->m2, nhit, seed, hit0, false, eta_user, exponents, nullptr,
                                    nullptr, stats);
    if (st && st != DDRW_ENOCONV) return st;
    double2 *F[5];
    ddrw_status s2 = fields(ctx, "est_f", 5, nhit, F);
    if (s2) return s2;
    const size_t fb = sizeof(double2) * 12 * ctx->V * nhit;
    DDRW_CUDA_CHECK(cudaMemcpyAsync(eta_out, F[0], fb, cudaMemcpyDeviceToDevice, ctx->stream));
    DDRW_CUDA_CHECK(cudaMemcpyAsync(delta_out, F[2], fb, cudaMemcpyDeviceToDevice, ctx->stream));
    return st;
}

// right-hand sides that fit the free device memory (about 3 KB per site and right-hand side of
// FP64/FP32 fields in the estimate, the block solves and the outer solve), at most 64
static int rhs_budget(ddrw_ctx *ctx)
{
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    size_t have = fr;
    for (auto &kv : ctx->ws) have += kv.second.bytes;  // workspaces are reused
    double per = 4096.0 * (double)ctx->V;
    if (ctx->prec == DDRW_MIXED_FP32 && ctx->outer_method == 1 && sap_supported(ctx))
        per += (double)sap_bytes_per_site_rhs(ctx) * (double)ctx->V;  // the GCR search directions
    int n = (int)((double)have * 0.85 / per);
    return std::max(1, std::min(n, 64));
}

// The estimate for nmass target masses: exponents[k * nhit + j], logW[k], rel_var[k].  The
// masses and hits are processed in chunks of right-hand sides that fit the device memory.
ddrw_status estimate_multi(ddrw_ctx *ctx, int nmass, const double *m2, int nhit, uint64_t seed, uint64_t hit0,
                           const double *eta_user, double *exponents, double *logW, double *rel_var, double *delta_user,
                           ddrw_solve_info *info)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    if (nhit <= 0 || nmass <= 0 || nmass > MAXM) return set_error(ctx, DDRW_EINVAL, "bad nhit or number of masses");
    const int budget = ctx->max_rhs > 0 ? ctx->max_rhs : rhs_budget(ctx);
    std::vector<double> eall((size_t)nmass * nhit);
    SolveStats stats;
    ddrw_status conv = DDRW_OK, st;
    if (eta_user != nullptr || delta_user != nullptr) {
        // the caller's vectors go through in one chunk
        if (nmass * nhit > budget)
            return set_error(ctx, DDRW_ENOMEM, "caller-supplied noise or delta for more right-hand sides than fit");
        std::vector<double> ma(nmass, ctx->m1);
        st = estimate_chunk(ctx, nmass, ma.data(), m2, nhit, seed, hit0, false, eta_user, eall.data(), nullptr,
                            delta_user, stats);
        if (st == DDRW_ENOCONV) conv = st;
        else if (st) return st;
    } else {
        // whole masses per chunk while nhit fits, else one mass and as many hits as fit
        const int mper = std::max(1, std::min(nmass, budget / nhit));
        const int hper = mper == 1 ? std::min(nhit, budget) : nhit;
        for (int k0 = 0; k0 < nmass; k0 += mper) {
            const int km = std::min(mper, nmass - k0);
            for (int j0 = 0; j0 < nhit; j0 += hper) {
                const int jn = std::min(hper, nhit - j0);
                std::vector<double> ec((size_t)km * jn);
                std::vector<double> ma(km, ctx->m1);
                st = estimate_chunk(ctx, km, ma.data(), m2 + k0, jn, seed, hit0 + j0, false, nullptr, ec.data(),
                                    nullptr, nullptr, stats);
                if (st == DDRW_ENOCONV) conv = st;
                else if (st) return st;
                for (int k = 0; k < km; k++)
                    for (int j = 0; j < jn; j++) eall[(size_t)(k0 + k) * nhit + j0 + j] = ec[(size_t)k * jn + j];
            }
        }
    }
    bool bad = false;
    for (int k = 0; k < nmass; k++) {
        std::vector<double> e(nhit);
        for (int j = 0; j < nhit; j++) {
            int rr = k * nhit + j;
            e[j] = eall[rr];
            if (!(e[j] == e[j])) bad = true;
            if (exponents) exponents[rr] = e[j];
        }
        // log W = log((1/N) sum exp(-e_j)) by log-sum-exp; rel_var = var(exp(-e)) / W^2
        double mx = -e[0];
        for (int j = 1; j < nhit; j++) mx = std::max(mx, -e[j]);
        double s = 0, s2 = 0;
        for (int j = 0; j < nhit; j++) {
            double w = std::exp(-e[j] - mx);
            s += w;
            s2 += w * w;
        }
        double mean = s / nhit;
        if (logW) logW[k] = mx + std::log(mean);
        if (rel_var) rel_var[k] = nhit > 1 ? (s2 / nhit - mean * mean) * nhit / (nhit - 1) / (mean * mean) : 0.0;
    }
    fill_info(info, stats, elapsed(t0));
    if (bad) return set_error(ctx, DDRW_ENUMERIC, "NaN exponent");
    return conv;
}

}  // namespace ddrw

using namespace ddrw;

extern "C" {

ddrw_status ddrw_noise(ddrw_ctx *ctx, uint64_t seed, uint64_t hit_offset, int nhit, double *eta)
{
    if (!ctx || !eta || nhit <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    cudaSetDevice(ctx->device);
    size_t bytes = sizeof(double) * 24 * ctx->nP * nhit;
    void *d;
    bool host;
    ddrw_status st;
    if ((st = stage_out(ctx, eta, bytes, "stage_noise", &d, &host))) return st;
    noise_launch(ctx, seed, hit_offset, nhit, 1, nullptr, (double *)d);
    if ((st = finish_out(ctx, eta, d, bytes, host))) return st;
    return sync(ctx);
}

ddrw_status ddrw_estimate(ddrw_ctx *ctx, int nhit, uint64_t seed, uint64_t hit_offset, const double *eta,
                          double *exponents, double *logW, double *rel_var, double *delta, ddrw_solve_info *info)
{
    if (!ctx) return DDRW_EINVAL;
    cudaSetDevice(ctx->device);
    return estimate_multi(ctx, 1, &ctx->m2, nhit, seed, hit_offset, eta, exponents, logW, rel_var, delta, info);
}

// log of the mean of exp(-e_j) (log-sum-exp) and the sample variance of exp(-e_j) over its squared mean
static void two_flavour_factor(const double *e, int n, double *logF, double *relvar)
{
    double mx = -e[0];
    for (int j = 1; j < n; j++) mx = std::max(mx, -e[j]);
    double s = 0, s2 = 0;
    for (int j = 0; j < n; j++) {
        double w = std::exp(-e[j] - mx);
        s += w;
        s2 += w * w;
    }
    double mean = s / n;
    *logF = mx + std::log(mean);
    *relvar = n > 1 ? (s2 / n - mean * mean) * n / (n - 1) / (mean * mean) : 0.0;
}

// Re of the mean of exp(-e1_j) for complex e1 (Eq. 11): (log |Re F|, sign of Re F)
static void one_flavour_factor(const double *e1, int n, double *logabs, double *sign)
{
    double mx = -e1[0];
    for (int j = 1; j < n; j++) mx = std::max(mx, -e1[2 * j]);
    double s = 0;
    for (int j = 0; j < n; j++) s += std::exp(-e1[2 * j] - mx) * std::cos(e1[2 * j + 1]);
    double mean = s / n;
    *logabs = mx + std::log(std::fabs(mean));
    *sign = mean >= 0 ? 1.0 : -1.0;
}

// sample variance of the complex one-flavour estimator exp(-eta^dag (M - 1) eta) over its squared
// modulus mean (Eq. 12 measured on the samples: E|X|^2 - |E X|^2), scale-free via a common shift
static double one_flavour_rel_var(const double *e1, int n)
{
    if (n < 2) return 0.0;
    double mx = -e1[0];
    for (int j = 1; j < n; j++) mx = std::max(mx, -e1[2 * j]);
    double mr = 0, mi = 0;
    for (int j = 0; j < n; j++) {
        const double a = std::exp(-e1[2 * j] - mx);
        mr += a * std::cos(e1[2 * j + 1]);
        mi -= a * std::sin(e1[2 * j + 1]);
    }
    mr /= n;
    mi /= n;
    double v = 0;
    for (int j = 0; j < n; j++) {
        const double a = std::exp(-e1[2 * j] - mx);
        const double dr = a * std::cos(e1[2 * j + 1]) - mr, di = -a * std::sin(e1[2 * j + 1]) - mi;
        v += dr * dr + di * di;
    }
    return v / (n - 1) / (mr * mr + mi * mi);
}

ddrw_status ddrw_estimate_interp(ddrw_ctx *ctx, int N, int nhit, uint64_t seed, uint64_t hit_offset, double *exponents,
                                 double *exponents_1f, double *logW, double *logW_factors, double *rel_var,
                                 double *rel_var_1f, ddrw_solve_info *info)
{
    if (!ctx) return DDRW_EINVAL;
    if (N < 1 || N > MAXM || nhit <= 0) return set_error(ctx, DDRW_EINVAL, "1 <= N <= 8 interpolation steps, nhit > 0");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    // m_i = (i/N) m2 + ((N-i)/N) m1, factor i = 1..N pairs (m_{i-1}, m_i)
    std::vector<double> ma(N), mb(N);
    for (int i = 1; i <= N; i++) {
        ma[i - 1] = ((double)(i - 1) * ctx->m2 + (double)(N - i + 1) * ctx->m1) / N;
        mb[i - 1] = ((double)i * ctx->m2 + (double)(N - i) * ctx->m1) / N;
    }
    const int budget = ctx->max_rhs > 0 ? ctx->max_rhs : rhs_budget(ctx);
    std::vector<double> e((size_t)N * nhit), e1((size_t)2 * N * nhit);
    SolveStats stats;
    ddrw_status conv = DDRW_OK, st;
    if (N * nhit <= budget) {
        // every factor as one mass slot, each with its own noise vectors (hits hit_offset + i nhit + j)
        st = estimate_chunk(ctx, N, ma.data(), mb.data(), nhit, seed, hit_offset, true, nullptr, e.data(), e1.data(),
                            nullptr, stats);
        if (st == DDRW_ENOCONV) conv = st;
        else if (st) return st;
    } else {
        const int hper = std::min(nhit, budget);
        for (int i = 0; i < N; i++)
            for (int j0 = 0; j0 < nhit; j0 += hper) {
                const int jn = std::min(hper, nhit - j0);
                st = estimate_chunk(ctx, 1, &ma[i], &mb[i], jn, seed, hit_offset + (uint64_t)i * nhit + j0, false,
                                    nullptr, e.data() + (size_t)i * nhit + j0, e1.data() + 2 * ((size_t)i * nhit + j0),
                                    nullptr, stats);
                if (st == DDRW_ENOCONV) conv = st;
                else if (st) return st;
            }
    }
    double l2 = 0, l1 = 0, sg = 1;
    for (int i = 0; i < N; i++) {
        double lf, rv, la, sgn;
        two_flavour_factor(e.data() + (size_t)i * nhit, nhit, &lf, &rv);
        one_flavour_factor(e1.data() + 2 * (size_t)i * nhit, nhit, &la, &sgn);
        l2 += lf;
        l1 += la;
        sg *= sgn;
        if (logW_factors) logW_factors[i] = lf;
        if (rel_var) rel_var[i] = rv;
        if (rel_var_1f) rel_var_1f[i] = one_flavour_rel_var(e1.data() + 2 * (size_t)i * nhit, nhit);
    }
    if (exponents) std::copy(e.begin(), e.end(), exponents);
    if (exponents_1f) std::copy(e1.begin(), e1.end(), exponents_1f);
    if (logW) {
        logW[0] = l2;        // two flavours: log W_gl (Eq. 8)
        logW[1] = l1;        // one flavour: log |W_1f| (Eq. 11, real part of each factor)
        logW[2] = sg;        // sign of W_1f
        logW[3] = 0.5 * l2;  // root trick: log sqrt(W_gl)
    }
    fill_info(info, stats, elapsed(t0));
    for (double v : e)
        if (!(v == v)) return set_error(ctx, DDRW_ENUMERIC, "NaN exponent");
    return conv;
}

ddrw_status ddrw_estimate_variant(ddrw_ctx *ctx, int variant, int N, int nhit, uint64_t seed, uint64_t hit_offset,
                                  const double *eta, double *exponents, double *logW, double *rel_var, long *dim,
                                  ddrw_solve_info *info)
{
    if (!ctx) return DDRW_EINVAL;
    if (variant < 0 || variant > 2) return set_error(ctx, DDRW_EINVAL, "variant 0 (total), 1 (even-odd) or 2 (blocks)");
    if (N < 1 || N > MAXM || nhit <= 0) return set_error(ctx, DDRW_EINVAL, "1 <= N <= 8 interpolation steps, nhit > 0");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    if (variant == 2) {
        if (eta) return set_error(ctx, DDRW_EINVAL, "the block variant draws its own noise (ddrw_estimate_interp)");
        double lw[4];
        if (dim) *dim = 12 * ctx->nP;
        ddrw_status st = ddrw_estimate_interp(ctx, N, nhit, seed, hit_offset, exponents, nullptr, lw, nullptr, nullptr,
                                              rel_var, info);
        if (logW) *logW = lw[0];
        return st;
    }
    auto t0 = std::chrono::steady_clock::now();
    const long V = ctx->V, nsites = variant == 0 ? V : ctx->vh;
    if (dim) *dim = 12 * nsites;
    ddrw_status st;
    int *idx;
    if ((st = workspace(ctx, "var_idx", sizeof(int) * nsites, (void **)&idx))) return st;
    DISPATCH_BL(ctx, k_support, (unsigned)((nsites + 255) / 256), 256, geom_dev(ctx), variant == 1 ? 1 : 0, nsites,
                idx);
    ++ctx->launches;
    std::vector<double> ma(N), mb(N);
    for (int i = 1; i <= N; i++) {
        ma[i - 1] = ((double)(i - 1) * ctx->m2 + (double)(N - i + 1) * ctx->m1) / N;
        mb[i - 1] = ((double)i * ctx->m2 + (double)(N - i) * ctx->m1) / N;
    }
    const int budget = std::max(1, (ctx->max_rhs > 0 ? ctx->max_rhs : rhs_budget(ctx)) / 2);
    const int hper = std::min(nhit, budget);
    double2 *F[4];
    if ((st = fields(ctx, "var_f", 4, hper, F))) return st;
    double *nd;
    if ((st = workspace(ctx, "var_nd", sizeof(double) * 3 * hper, (void **)&nd))) return st;
    std::vector<double> e((size_t)N * nhit), h(3 * (size_t)hper);
    SolveStats stats;
    ddrw_status conv = DDRW_OK;
    const size_t fb = sizeof(double2) * 12 * (size_t)V;
    for (int i = 0; i < N; i++) {
        MassSet mbs;
        if ((st = make_massset(ctx, 1, &mb[i], &mbs))) return st;
        const double dm = ma[i] - mb[i];
        for (int j0 = 0; j0 < nhit; j0 += hper) {
            const int jn = std::min(hper, nhit - j0);
            DDRW_CUDA_CHECK(cudaMemsetAsync(F[0], 0, fb * jn, ctx->stream));
            ++ctx->launches;
            dim3 grid((unsigned)((12 * nsites + 255) / 256), (unsigned)jn);
            if (eta)
                k_scatter_packed<<<grid, 256, 0, ctx->stream>>>(idx, nsites, eta + 2 * 12 * nsites * ((size_t)i * nhit + j0),
                                                                V, F[0]);
            else
                k_noise<<<grid, 256, 0, ctx->stream>>>(V, nsites, idx, (uint32_t)(seed & 0xffffffffu),
                                                       (uint32_t)(seed >> 32), hit_offset + (uint64_t)i * nhit + j0, jn,
                                                       1, F[0], nullptr);
            const double2 *rhs = F[0];
            if (variant == 1) {
                // rhs_e = (S(m_{i-1}) - S(m_i)) eta_e, odd sites zero; the solution's even part is
                // S(m_i)^-1 rhs_e = delta (the full solve with b_o = 0)
                if ((st = apply_schur_eo64(ctx, ma[i], F[0], F[2], F[1], jn))) return st;
                DDRW_CUDA_CHECK(cudaMemsetAsync(F[3], 0, fb * jn, ctx->stream));
                if ((st = apply_schur_eo64(ctx, mb[i], F[0], F[3], F[1], jn))) return st;
                Blas<PrecD>::axpby(ctx, VecRange{V, 0, ctx->vh, 12 * V, jn}, 1.0, F[2], -1.0, F[3]);
                rhs = F[3];
            }
            SolveStats s1;
            st = full_solve64(ctx, mbs, rhs, F[1], jn, ctx->tol_outer, ctx->maxiter, ctx->prec, &s1);
            if (st == DDRW_ENOCONV) conv = st;
            else if (st) return st;
            stats.outer_iters += s1.outer_iters;
            stats.outer_cycles = std::max(stats.outer_cycles, s1.outer_cycles);
            stats.fp64_dslash_full += s1.fp64_dslash_full;
            stats.outer_rel_residual = std::max(stats.outer_rel_residual, s1.outer_rel_residual);
            // total: delta = dm x, e = dm^2 |x|^2 + 2 dm Re <eta, x>;  even-odd: delta = x_e
            const long n_range = variant == 0 ? V : ctx->vh;
            if ((st = Blas<PrecD>::norm_dot(ctx, VecRange{V, 0, n_range, 12 * V, jn}, F[1], F[0], nd))) return st;
            DDRW_CUDA_CHECK(cudaMemcpyAsync(h.data(), nd, sizeof(double) * 3 * jn, cudaMemcpyDeviceToHost, ctx->stream));
            DDRW_SYNC(ctx);
            for (int j = 0; j < jn; j++) {
                const double a = h[3 * j], b = h[3 * j + 1];
                e[(size_t)i * nhit + j0 + j] = variant == 0 ? dm * dm * a + 2.0 * dm * b : a + 2.0 * b;
            }
        }
    }
    double l2 = 0;
    for (int i = 0; i < N; i++) {
        double lf, rv;
        two_flavour_factor(e.data() + (size_t)i * nhit, nhit, &lf, &rv);
        l2 += lf;
        if (rel_var) rel_var[i] = rv;
    }
    if (exponents) std::copy(e.begin(), e.end(), exponents);
    if (logW) *logW = l2;
    fill_info(info, stats, elapsed(t0));
    for (double v : e)
        if (!(v == v)) return set_error(ctx, DDRW_ENUMERIC, "NaN exponent");
    return conv;
}

ddrw_status ddrw_estimate_masses(ddrw_ctx *ctx, int nmass, const double *m2, int nhit, uint64_t seed,
                                 uint64_t hit_offset, double *exponents, double *logW, double *rel_var,
                                 ddrw_solve_info *info)
{
    if (!ctx || !m2) return set_error(ctx, DDRW_EINVAL, "bad argument");
    cudaSetDevice(ctx->device);
    return estimate_multi(ctx, nmass, m2, nhit, seed, hit_offset, nullptr, exponents, logW, rel_var, nullptr, info);
}

ddrw_status ddrw_apply_dA(ddrw_ctx *ctx, const double *eta, double *r, int nrhs, ddrw_solve_info *info)
{
    if (!ctx || !eta || !r || nrhs <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    MassSet m2s, m1s;
    ddrw_status st;
    if ((st = make_massset(ctx, 1, &ctx->m2, &m2s))) return st;
    if ((st = make_massset(ctx, 1, &ctx->m1, &m1s))) return st;
    double2 *F[5];
    if ((st = fields(ctx, "est_f", 5, nrhs, F))) return st;
    size_t pbytes = sizeof(double) * 24 * ctx->nP * nrhs;
    const void *din;
    void *dout;
    bool host;
    if ((st = stage_in(ctx, eta, pbytes, "stage_in", &din))) return st;
    if ((st = stage_out(ctx, r, pbytes, "stage_out", &dout, &host))) return st;
    unpack_P64(ctx, (const double *)din, F[0], nrhs);
    SolveStats stats;
    double2 *work[3] = {F[2], F[3], F[4]};
    if ((st = apply_dA_fields(ctx, m2s, m1s, F[0], F[1], work, nrhs, &stats))) return st;
    pack_P64(ctx, F[1], (double *)dout, nrhs);
    if ((st = finish_out(ctx, r, dout, pbytes, host))) return st;
    st = sync(ctx);
    fill_info(info, stats, elapsed(t0));
    return st;
}

ddrw_status ddrw_solve_schur(ddrw_ctx *ctx, double m, const double *b, double *x, int nrhs, ddrw_solve_info *info)
{
    if (!ctx || !b || !x || nrhs <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    MassSet ms;
    ddrw_status st;
    if ((st = make_massset(ctx, 1, &m, &ms))) return st;
    double2 *F[4];
    if ((st = fields(ctx, "sch_f", 4, nrhs, F))) return st;
    size_t pbytes = sizeof(double) * 24 * ctx->nP * nrhs;
    const void *din;
    void *dout;
    bool host;
    if ((st = stage_in(ctx, b, pbytes, "stage_in", &din))) return st;
    if ((st = stage_out(ctx, x, pbytes, "stage_out", &dout, &host))) return st;
    unpack_P64(ctx, (const double *)din, F[0], nrhs);
    SolveStats stats;
    double2 *work[2] = {F[2], F[3]};
    ddrw_status conv = solve_schur_fields(ctx, ms, F[0], F[1], work, nrhs, &stats);
    if (conv && conv != DDRW_ENOCONV) return conv;
    pack_P64(ctx, F[1], (double *)dout, nrhs);
    if ((st = finish_out(ctx, x, dout, pbytes, host))) return st;
    if ((st = sync(ctx))) return st;
    fill_info(info, stats, elapsed(t0));
    return conv;
}

ddrw_status ddrw_apply_schur(ddrw_ctx *ctx, double m, int dagger, const double *in, double *out, int nrhs)
{
    if (!ctx || !in || !out || nrhs <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    MassSet ms;
    ddrw_status st;
    if ((st = make_massset(ctx, 1, &m, &ms))) return st;
    double2 *F[4];
    if ((st = fields(ctx, "sch_f", 4, nrhs, F))) return st;
    size_t pbytes = sizeof(double) * 24 * ctx->nP * nrhs, fb = sizeof(double2) * 12 * ctx->V * nrhs;
    const void *din;
    void *dout;
    bool host;
    if ((st = stage_in(ctx, in, pbytes, "stage_in", &din))) return st;
    if ((st = stage_out(ctx, out, pbytes, "stage_out", &dout, &host))) return st;
    const bool mixed = ctx->prec != DDRW_FP64;
    unpack_P64(ctx, (const double *)din, F[0], nrhs);
    GeomDev g = geom_dev(ctx);
    dim3 grid((unsigned)((ctx->V + 127) / 128), (unsigned)nrhs);
    if (!dagger) {
        // A v = v - P D_bb^-1 D_bw D_ww^-1 D_wb v
        DDRW_CUDA_CHECK(cudaMemsetAsync(F[1], 0, fb, ctx->stream));
        hop_between(ctx, DDRW_WHITE, F[0], F[1], nrhs);
        if ((st = block_solve64(ctx, DDRW_WHITE, ms, F[1], F[2], nrhs, ctx->tol_block, ctx->maxiter, ctx->prec, nullptr))) return st;
        DDRW_CUDA_CHECK(cudaMemsetAsync(F[1], 0, fb, ctx->stream));
        hop_between(ctx, DDRW_BLACK, F[2], F[1], nrhs);
        if ((st = block_solve64(ctx, DDRW_BLACK, ms, F[1], F[3], nrhs, ctx->tol_block, ctx->maxiter, ctx->prec, nullptr))) return st;
        DISPATCH_BL(ctx, k_delta, grid, 128, g, F[0], F[3], F[1], 12 * ctx->V, 0);
    } else {
        // A^dag v = v - P (D_wb)^dag (D_ww^-1)^dag (D_bw)^dag (D_bb^-1)^dag v, and D^dag = g5 D g5 gives
        // (D_XY)^dag = g5 D_YX g5 for the blocks of Eq. 1:  A^dag v = v - P g5 D_bw D_ww^-1 D_wb D_bb^-1 g5 v
        const long n12 = 12 * ctx->V;
        ++ctx->launches;
        k_gamma5_field<<<(unsigned)((n12 * nrhs + 255) / 256), 256, 0, ctx->stream>>>(n12, ctx->V, nrhs, F[0], F[1]);
        if ((st = block_solve64(ctx, DDRW_BLACK, ms, F[1], F[2], nrhs, ctx->tol_block, ctx->maxiter, ctx->prec, nullptr))) return st;
        DDRW_CUDA_CHECK(cudaMemsetAsync(F[1], 0, fb, ctx->stream));
        hop_between(ctx, DDRW_WHITE, F[2], F[1], nrhs);
        if ((st = block_solve64(ctx, DDRW_WHITE, ms, F[1], F[3], nrhs, ctx->tol_block, ctx->maxiter, ctx->prec, nullptr))) return st;
        DDRW_CUDA_CHECK(cudaMemsetAsync(F[1], 0, fb, ctx->stream));
        hop_between(ctx, DDRW_BLACK, F[3], F[1], nrhs);
        DISPATCH_BL(ctx, k_delta, grid, 128, g, F[0], F[1], F[1], 12 * ctx->V, 1);  // element-wise in place
    }
    pack_P64(ctx, F[1], (double *)dout, nrhs);
    if ((st = finish_out(ctx, out, dout, pbytes, host))) return st;
    return sync(ctx);
}

ddrw_status ddrw_solve_block(ddrw_ctx *ctx, int colour, double m, const double *b, double *x, int nrhs,
                             ddrw_solve_info *info)
{
    if (!ctx || !b || !x || nrhs <= 0 || (colour != DDRW_BLACK && colour != DDRW_WHITE))
        return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    MassSet ms;
    ddrw_status st;
    if ((st = make_massset(ctx, 1, &m, &ms))) return st;
    double2 *F[2];
    if ((st = fields(ctx, "api_s", 2, nrhs, F))) return st;
    size_t ub = sizeof(double) * 24 * ctx->V * nrhs;
    const void *din;
    void *dout;
    bool host;
    if ((st = stage_in(ctx, b, ub, "stage_in", &din))) return st;
    if ((st = stage_out(ctx, x, ub, "stage_out", &dout, &host))) return st;
    pack_spinor64(ctx, (const double *)din, F[0], nrhs);
    DDRW_CUDA_CHECK(cudaMemsetAsync(F[1], 0, sizeof(double2) * 12 * ctx->V * nrhs, ctx->stream));
    SolveStats stats;
    st = block_solve64(ctx, colour, ms, F[0], F[1], nrhs, ctx->tol_block, ctx->maxiter, ctx->prec, &stats);
    if (st && st != DDRW_ENOCONV) return st;
    ddrw_status conv = st;
    unpack_spinor64(ctx, F[1], (double *)dout, nrhs);
    if ((st = finish_out(ctx, x, dout, ub, host))) return st;
    if ((st = sync(ctx))) return st;
    if (info) {
        fill_info(info, stats, elapsed(t0));
        info->true_rel_residual = stats.block_rel_residual;
        info->cycles = stats.block_cycles;
    }
    return conv;
}

ddrw_status ddrw_solve_D(ddrw_ctx *ctx, double m, const double *b, double *x, int nrhs, ddrw_solve_info *info)
{
    if (!ctx || !b || !x || nrhs <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    MassSet ms;
    ddrw_status st;
    if ((st = make_massset(ctx, 1, &m, &ms))) return st;
    double2 *F[2];
    if ((st = fields(ctx, "api_s", 2, nrhs, F))) return st;
    size_t ub = sizeof(double) * 24 * ctx->V * nrhs;
    const void *din;
    void *dout;
    bool host;
    if ((st = stage_in(ctx, b, ub, "stage_in", &din))) return st;
    if ((st = stage_out(ctx, x, ub, "stage_out", &dout, &host))) return st;
    pack_spinor64(ctx, (const double *)din, F[0], nrhs);
    SolveStats stats;
    st = full_solve64(ctx, ms, F[0], F[1], nrhs, ctx->tol_outer, ctx->maxiter, ctx->prec, &stats);
    if (st && st != DDRW_ENOCONV) return st;
    ddrw_status conv = st;
    unpack_spinor64(ctx, F[1], (double *)dout, nrhs);
    if ((st = finish_out(ctx, x, dout, ub, host))) return st;
    if ((st = sync(ctx))) return st;
    fill_info(info, stats, elapsed(t0));
    return conv;
}

}  // extern "C"
