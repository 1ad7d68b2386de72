// blockdet.cu -- the exact block determinants of Eq. 7: W = W_gl prod_k det D_k^2(m2) / det D_k^2(m1),
// k over the black and the white blocks, D_k the block Dirac operators on the diagonal of D_bb and
// D_ww (Eq. 1: the hops inside the block).
//
// Per block the determinant is reduced to the block's even sites: with the block operator in
// even/odd form [[A_ee, D_eo], [D_oe, A_oo]] (A the site-diagonal part (4 + m) + C),
//
//     det D_k = det A_oo * det S_k,    S_k = A_ee - D_eo A_oo^-1 D_oe = A_ee - 1/4 H_eo A_oo^-1 H_oe,
//
// so the dense matrix has dimension 6 l^4 instead of 12 l^4 (eight times less LU work).
//   * det A_oo: product over the block's odd sites of the determinants of the two Hermitian 6x6
//     chirality blocks of A(x) (k_site_logdet, a 6x6 LU per site and chirality);
//   * S_k: assembled column by column by the FP64 stencil with hops restricted to the blocks --
//     a unit vector at the same even site and component of every block gives that column of every
//     S_k at once, because the blocks do not couple (k_unit_fields, two stencil launches,
//     k_scatter_cols);
//   * det S_k: a batched LU with partial pivoting in FP64, one CTA per matrix, blocked right-looking
//     (panels of NB columns factorised in place, the trailing matrix updated once per panel with
//     the panel's multipliers held in registers and the panel's U rows staged in shared memory).
// det D_k is real (g5-hermiticity of the block operator); the phase of the LU product is returned
// as a sign after checking that it is real.
#include <cmath>
#include <vector>

#include "blas.cuh"
#include "ctx.h"

namespace ddrw {

namespace {

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 csub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cdiv2(double2 a, double2 b)
{
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ----------------------------------------------------------------------------- assembly of S_k

// X[r] = unit vector at even site h = (j0 + r) / 12, component (j0 + r) % 12 of every block
// (fields already zeroed; nrhs fields 12 V elements apart)
__global__ void k_unit_fields(double2 *X, long V, int vbh, int nblk, int j0, int ncol)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)nblk * ncol) return;
    int r = (int)(i / nblk), k = (int)(i - (long)r * nblk);
    int j = j0 + r, h = j / 12, a = j % 12;
    X[(long)r * 12 * V + (long)a * V + (long)k * vbh + h] = make_double2(1.0, 0.0);
}

// S_k[(j0 + r) n + i] = Y[r] at even site h' = i / 12, component i % 12 of block k0 + kb
__global__ void k_scatter_cols(const double2 *__restrict__ Y, long V, int vbh, int n, int k0, int nb, int j0,
                               int ncol, double2 *S)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = (long)ncol * n;
    if (t >= per * nb) return;
    int kb = (int)(t / per);
    long rem = t - (long)kb * per;
    int r = (int)(rem / n), i = (int)(rem - (long)r * n);
    int h = i / 12, a = i % 12;
    S[(size_t)kb * n * n + (size_t)(j0 + r) * n + i] = Y[(long)r * 12 * V + (long)a * V + (long)(k0 + kb) * vbh + h];
}

// ----------------------------------------------------------------------------- Dirichlet cut

// zero the links U_mu(x) with x_mu = cut - 1 mod cut (FP64 full and FP32 two-row copies)
template <int BL>
__global__ void k_cut_links(GeomDev g, int cut, double2 *U64, float4 *U32)
{
    const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    const int *o = g.blk_org + st.blk * 4;
    for (int mu = 0; mu < 4; mu++) {
        if ((o[mu] + st.c[mu]) % cut != cut - 1) continue;
        for (int k = 0; k < 9; k++) U64[(long)(mu * 9 + k) * g.V + s] = make_double2(0.0, 0.0);
        for (int k = 0; k < 3; k++) U32[(long)(mu * 3 + k) * g.V + s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// the FP64 links in the boundary layout: out[(lex * 4 + mu) * 9 + k] = U64[(mu * 9 + k) V + s]
template <int BL>
__global__ void k_gauge_lex(GeomDev g, const double2 *U64, double2 *out)
{
    const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    const long x = lex_index<BL>(st, g);
    for (int mu = 0; mu < 4; mu++)
        for (int k = 0; k < 9; k++) out[(x * 4 + mu) * 9 + k] = U64[(long)(mu * 9 + k) * g.V + s];
}

#define DISPATCH_L(ctx, KERNEL, ...)                                                                    \
    do {                                                                                                \
        const unsigned gr__ = (unsigned)(((ctx)->V + 255) / 256);                                       \
        ++(ctx)->launches;                                                                              \
        switch ((ctx)->l) {                                                                             \
        case 2: KERNEL<2><<<gr__, 256, 0, (ctx)->stream>>>(__VA_ARGS__); break;                         \
        case 4: KERNEL<4><<<gr__, 256, 0, (ctx)->stream>>>(__VA_ARGS__); break;                         \
        case 6: KERNEL<6><<<gr__, 256, 0, (ctx)->stream>>>(__VA_ARGS__); break;                         \
        default: KERNEL<8><<<gr__, 256, 0, (ctx)->stream>>>(__VA_ARGS__); break;                        \
        }                                                                                               \
    } while (0)

void gauge_to_lex(ddrw_ctx *ctx, double2 *out) { DISPATCH_L(ctx, k_gauge_lex, geom_dev(ctx), ctx->U64, out); }

// ----------------------------------------------------------------------------- det A_oo

// log |det| and sign of a 6x6 complex matrix by LU with partial pivoting (in place)
__device__ void lu6(double2 (&M)[6][6], double &lg, double &ang)
{
    lg = 0.0;
    ang = 0.0;
    for (int k = 0; k < 6; k++) {
        int p = k;
        double best = M[k][k].x * M[k][k].x + M[k][k].y * M[k][k].y;
        for (int i = k + 1; i < 6; i++) {
            double a = M[i][k].x * M[i][k].x + M[i][k].y * M[i][k].y;
            if (a > best) {
                best = a;
                p = i;
            }
        }
        if (p != k) {
            for (int j = 0; j < 6; j++) {
                double2 t = M[k][j];
                M[k][j] = M[p][j];
                M[p][j] = t;
            }
            ang += M_PI;
        }
        double2 piv = M[k][k];
        lg += 0.5 * log(piv.x * piv.x + piv.y * piv.y);
        ang += atan2(piv.y, piv.x);
        for (int i = k + 1; i < 6; i++) {
            double2 l = cdiv2(M[i][k], piv);
            for (int j = k + 1; j < 6; j++) M[i][j] = csub2(M[i][j], cmul2(l, M[k][j]));
        }
    }
}

// per block (one CTA): sum over its odd sites and both chiralities of log |det (4 + m + C_ch(x))|,
// and the phase; thread-ordered partial sums reduced in a fixed order (deterministic)
constexpr int SITE_NT = 128;
__global__ void __launch_bounds__(SITE_NT) k_site_logdet(const double2 *__restrict__ C64, long V, long vh, int vbh,
                                                        double mass4, double *lg_out, double *ang_out)
{
    __shared__ double slg[SITE_NT], sang[SITE_NT];
    const int k = blockIdx.x;
    double lg = 0.0, ang = 0.0;
    for (int t = threadIdx.x; t < 2 * vbh; t += SITE_NT) {
        const int h = t >> 1, ch = t & 1;
        const long s = vh + (long)k * vbh + h;
        double c[36];
        for (int q = 0; q < 18; q++) {
            double2 v = C64[((long)ch * 18 + q) * V + s];
            c[2 * q] = v.x;
            c[2 * q + 1] = v.y;
        }
        double2 M[6][6];
        for (int i = 0; i < 6; i++) M[i][i] = make_double2(mass4 + c[i], 0.0);
        for (int i = 0; i < 6; i++)
            for (int j = i + 1; j < 6; j++) {
                int o = 6 + 2 * herm_off(i, j);
                M[i][j] = make_double2(c[o], c[o + 1]);
                M[j][i] = make_double2(c[o], -c[o + 1]);
            }
        double l, a;
        lu6(M, l, a);
        lg += l;
        ang += a;
    }
    slg[threadIdx.x] = lg;
    sang[threadIdx.x] = ang;
    __syncthreads();
    for (int w = SITE_NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            slg[threadIdx.x] += slg[threadIdx.x + w];
            sang[threadIdx.x] += sang[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        lg_out[k] = slg[0];
        ang_out[k] = sang[0];
    }
}

// ----------------------------------------------------------------------------- batched LU

constexpr int LU_NT = 256;
constexpr int NB = 16;   // panel width
constexpr int TJ = 32;   // columns of U12 staged in shared memory per pass

// warp/CTA argmax of |a|^2 (ties to the lowest index)
__device__ __forceinline__ void argmax_update(double &v, int &i, double v2, int i2)
{
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

// One CTA per n x n column-major complex matrix (element (i, j) at A[j n + i]).  Returns
// log |det| and the phase angle (sum of the pivots' arguments plus pi per row swap).
__global__ void __launch_bounds__(LU_NT) k_lu_logdet(int n, double2 *mats, double *lg_out, double *ang_out)
{
    double2 *A = mats + (size_t)blockIdx.x * n * n;
    __shared__ double sv[LU_NT / 32];
    __shared__ int si[LU_NT / 32];
    __shared__ int piv_row;
    __shared__ double2 L11[NB][NB];
    __shared__ double2 U12[NB][TJ];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double lg = 0.0, ang = 0.0;  // thread 0's accumulators
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int kb = min(NB, n - k0);
        // ---- panel: columns k0 .. k0 + kb - 1, rows k0 .. n - 1
        for (int kk = k0; kk < k0 + kb; kk++) {
            double bv = -1.0;
            int bi = kk;
            for (int i = kk + threadIdx.x; i < n; i += LU_NT) {
                double2 v = A[(size_t)kk * n + i];
                argmax_update(bv, bi, v.x * v.x + v.y * v.y, i);
            }
            for (int o = 16; o > 0; o >>= 1) {
                double v2 = __shfl_down_sync(0xffffffffu, bv, o);
                int i2 = __shfl_down_sync(0xffffffffu, bi, o);
                argmax_update(bv, bi, v2, i2);
            }
            if (lane == 0) {
                sv[w] = bv;
                si[w] = bi;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double v = sv[0];
                int i = si[0];
                for (int q = 1; q < LU_NT / 32; q++) argmax_update(v, i, sv[q], si[q]);
                piv_row = i;
            }
            __syncthreads();
            const int p = piv_row;
            if (p != kk) {  // swap rows kk and p in the active columns k0 .. n - 1
                for (int j = k0 + threadIdx.x; j < n; j += LU_NT) {
                    double2 t = A[(size_t)j * n + kk];
                    A[(size_t)j * n + kk] = A[(size_t)j * n + p];
                    A[(size_t)j * n + p] = t;
                }
                if (threadIdx.x == 0) ang += M_PI;
                __syncthreads();
            }
            const double2 pv = A[(size_t)kk * n + kk];
            if (threadIdx.x == 0) {
                lg += 0.5 * log(pv.x * pv.x + pv.y * pv.y);
                ang += atan2(pv.y, pv.x);
            }
            for (int i = kk + 1 + threadIdx.x; i < n; i += LU_NT) A[(size_t)kk * n + i] = cdiv2(A[(size_t)kk * n + i], pv);
            __syncthreads();
            // update the panel's remaining columns
            const int ncp = k0 + kb - kk - 1, nr = n - kk - 1;
            for (long t = threadIdx.x; t < (long)ncp * nr; t += LU_NT) {
                const int jj = kk + 1 + (int)(t / nr), i = kk + 1 + (int)(t % nr);
                A[(size_t)jj * n + i] = csub2(A[(size_t)jj * n + i], cmul2(A[(size_t)kk * n + i], A[(size_t)jj * n + kk]));
            }
            __syncthreads();
        }
        const int j1 = k0 + kb;
        if (j1 >= n) break;
        // ---- unit lower triangle of the panel into shared memory
        for (int t = threadIdx.x; t < NB * NB; t += LU_NT) {
            const int r = t / NB, q = t % NB;
            L11[r][q] = (r < kb && q < kb) ? A[(size_t)(k0 + q) * n + k0 + r] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        // ---- U12 = L11^-1 A12 (rows k0 .. k0 + kb - 1, columns j1 .. n - 1), one thread per column
        for (int j = j1 + threadIdx.x; j < n; j += LU_NT) {
            double2 u[NB];
#pragma unroll
            for (int r = 0; r < NB; r++) u[r] = r < kb ? A[(size_t)j * n + k0 + r] : make_double2(0.0, 0.0);
#pragma unroll
            for (int r = 1; r < NB; r++)
#pragma unroll
                for (int q = 0; q < r; q++) u[r] = csub2(u[r], cmul2(L11[r][q], u[q]));
#pragma unroll
            for (int r = 0; r < NB; r++)
                if (r < kb) A[(size_t)j * n + k0 + r] = u[r];
        }
        __syncthreads();
        // ---- trailing update A22 -= L21 U12: rows j1 .. n - 1 (threads), columns in passes of TJ
        for (int c0 = j1; c0 < n; c0 += TJ) {
            const int tc = min(TJ, n - c0);
            for (int t = threadIdx.x; t < NB * TJ; t += LU_NT) {
                const int q = t / TJ, c = t % TJ;
                U12[q][c] = (q < kb && c < tc) ? A[(size_t)(c0 + c) * n + k0 + q] : make_double2(0.0, 0.0);
            }
            __syncthreads();
            for (int i = j1 + threadIdx.x; i < n; i += LU_NT) {
                double2 l[NB];
#pragma unroll
                for (int q = 0; q < NB; q++) l[q] = q < kb ? A[(size_t)(k0 + q) * n + i] : make_double2(0.0, 0.0);
                for (int c = 0; c < tc; c++) {
                    double2 a = A[(size_t)(c0 + c) * n + i];
#pragma unroll
                    for (int q = 0; q < NB; q++) a = csub2(a, cmul2(l[q], U12[q][c]));
                    A[(size_t)(c0 + c) * n + i] = a;
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        lg_out[blockIdx.x] = lg;
        ang_out[blockIdx.x] = ang;
    }
}

}  // namespace

void cut_links(ddrw_ctx *ctx) { DISPATCH_L(ctx, k_cut_links, geom_dev(ctx), ctx->cut, ctx->U64, ctx->U32); }

// log |det D_k(m)| and sign for all blocks (host vectors, library block numbering)
static ddrw_status block_logdets(ddrw_ctx *ctx, double m, std::vector<double> &logdet, std::vector<double> &sign)
{
    if (ctx->l > 6) return set_error(ctx, DDRW_EINVAL, "block determinants need blocks of at most 6^4 sites");
    ddrw_status st;
    MassInv *mi;
    if ((st = mass_inverse(ctx, m, &mi))) return st;
    const long V = ctx->V;
    const int vbh = ctx->l * ctx->l * ctx->l * ctx->l / 2, nblk = ctx->nblk;
    const int n = 12 * vbh;
    const size_t mat = (size_t)n * n * sizeof(double2);

    // det A_oo per block
    double *dlg, *dang;
    if ((st = workspace(ctx, "bdet_site", sizeof(double) * 4 * nblk, (void **)&dlg))) return st;
    dang = dlg + nblk;
    double *dslg = dlg + 2 * nblk, *dsang = dlg + 3 * nblk;
    ++ctx->launches;
    k_site_logdet<<<nblk, SITE_NT, 0, ctx->stream>>>(ctx->C64, V, ctx->vh, vbh, 4.0 + m, dlg, dang);
    DDRW_CUDA_CHECK(cudaGetLastError());

    // batches of blocks whose matrices fit in a fraction of the free memory
    size_t fre = 0, tot = 0;
    DDRW_CUDA_CHECK(cudaMemGetInfo(&fre, &tot));
    const int ncol = 32;  // columns per stencil batch
    const size_t fields = sizeof(double2) * 12 * (size_t)V * ncol;
    long fit = (long)((fre > 3 * fields ? fre - 3 * fields : 0) * 0.6 / mat);
    if (fit < 1) return set_error(ctx, DDRW_ENOMEM, "one block matrix does not fit in device memory");
    const int bb = (int)std::min<long>(fit, nblk);
    double2 *S, *X, *T, *Y;
    if ((st = workspace(ctx, "bdet_mats", mat * bb, (void **)&S))) return st;
    if ((st = workspace(ctx, "bdet_x", fields, (void **)&X))) return st;
    if ((st = workspace(ctx, "bdet_t", fields, (void **)&T))) return st;
    if ((st = workspace(ctx, "bdet_y", fields, (void **)&Y))) return st;

    for (int k0 = 0; k0 < nblk; k0 += bb) {
        const int nb = std::min(bb, nblk - k0);
        for (int j0 = 0; j0 < n; j0 += ncol) {
            const int nc = std::min(ncol, n - j0);
            DDRW_CUDA_CHECK(cudaMemsetAsync(X, 0, sizeof(double2) * 12 * (size_t)V * nc, ctx->stream));
            ++ctx->launches;
            k_unit_fields<<<(unsigned)(((long)nblk * nc + 255) / 256), 256, 0, ctx->stream>>>(X, V, vbh, nblk, j0, nc);
            // T_o = A_oo^-1 H_oe X   (hops inside the blocks)
            DslashCall c;
            c.in = X;
            c.out = T;
            c.rstride = 12 * V;
            c.nrhs = nc;
            c.nmass = 1;
            c.masses[0] = m;
            c.Ainv[0] = mi->A64;
            c.beta = 1.0;
            c.post = 1;
            c.hopsel = 1;
            c.par0 = 1;
            c.npar = 1;
            c.blk0 = 0;
            c.nblk = nblk;
            dslash64(ctx, c);
            // Y_e = A_ee X - 1/4 H_eo T_o = S X
            DslashCall d = c;
            d.in = T;
            d.x = X;
            d.out = Y;
            d.alpha = 1.0;
            d.beta = -0.25;
            d.diag = 1;
            d.post = 0;
            d.par0 = 0;
            dslash64(ctx, d);
            ++ctx->launches;
            long tot_el = (long)nb * nc * n;
            k_scatter_cols<<<(unsigned)((tot_el + 255) / 256), 256, 0, ctx->stream>>>(Y, V, vbh, n, k0, nb, j0, nc, S);
        }
        ++ctx->launches;
        k_lu_logdet<<<nb, LU_NT, 0, ctx->stream>>>(n, S, dslg + k0, dsang + k0);
        DDRW_CUDA_CHECK(cudaGetLastError());
    }
    std::vector<double> h(4 * nblk);
    DDRW_CUDA_CHECK(cudaMemcpyAsync(h.data(), dlg, sizeof(double) * 4 * nblk, cudaMemcpyDeviceToHost, ctx->stream));
    DDRW_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    // the dense matrices and column batches are large and needed once per configuration
    for (const char *nm : {"bdet_mats", "bdet_x", "bdet_t", "bdet_y"}) release_workspace(ctx, nm);
    logdet.resize(nblk);
    sign.resize(nblk);
    for (int k = 0; k < nblk; k++) {
        logdet[k] = h[k] + h[2 * nblk + k];
        double a = h[nblk + k] + h[3 * nblk + k];
        double c = std::cos(a), s = std::sin(a);
        if (!(std::fabs(s) < 1e-6)) return set_error(ctx, DDRW_ENUMERIC, "block determinant is not real");
        sign[k] = c > 0 ? 1.0 : -1.0;
    }
    return DDRW_OK;
}

}  // namespace ddrw

using namespace ddrw;

extern "C" {

ddrw_status ddrw_block_logdet(ddrw_ctx *ctx, double m, double *logdet, double *sign)
{
    if (!ctx || !logdet) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    std::vector<double> ld, sg;
    ddrw_status st = block_logdets(ctx, m, ld, sg);
    if (st) return st;
    const size_t bytes = sizeof(double) * ld.size();
    if (is_device_ptr(logdet)) DDRW_CUDA_CHECK(cudaMemcpy(logdet, ld.data(), bytes, cudaMemcpyHostToDevice));
    else memcpy(logdet, ld.data(), bytes);
    if (sign) {
        if (is_device_ptr(sign)) DDRW_CUDA_CHECK(cudaMemcpy(sign, sg.data(), bytes, cudaMemcpyHostToDevice));
        else memcpy(sign, sg.data(), bytes);
    }
    return DDRW_OK;
}

ddrw_status ddrw_block_factor(ddrw_ctx *ctx, double *log_w_blk)
{
    if (!ctx || !log_w_blk) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    std::vector<double> l1, s1, l2, s2;
    ddrw_status st;
    if ((st = block_logdets(ctx, ctx->m1, l1, s1))) return st;
    if ((st = block_logdets(ctx, ctx->m2, l2, s2))) return st;
    double acc = 0.0;  // fixed summation order
    for (size_t k = 0; k < l1.size(); k++) acc += 2.0 * (l2[k] - l1[k]);
    *log_w_blk = acc;
    return DDRW_OK;
}

// The block factor of Eq. 7 for blocks too large for a dense determinant, by the nested
// decomposition of Sec. 2.2 (caption of Fig. 2): each block's Dirichlet operator D_k is cut into
// sub-blocks of length lsub (a black/white checkerboard inside the block), so that
//   det D_k = det Shat_k * prod_{sub in k} det D_sub,
// Shat_k the Schur complement of D_k with respect to its sub-blocks (Sec. 1).  The sub-block
// determinants are exact (ddrw_block_factor on sub-blocks); the product over the blocks of
// det Shat_k^2(m2) / det Shat_k^2(m1) is the global factor of the direct sum of the blocks' Dirichlet
// operators with sub-block domain decomposition, and it is estimated stochastically with Eq. 3
// (nhit noise vectors) -- the same estimator as W_gl, on an auxiliary context: the same lattice
// and field, blocks of length lsub, every hop across a face of the original blocks removed
// (ddrw_set_dirichlet) while the clover term stays the full field's.
ddrw_status ddrw_block_factor_nested(ddrw_ctx *ctx, int lsub, int nhit, uint64_t seed, double *out, double *exponents,
                                     double *rel_var)
{
    if (!ctx || !out || nhit <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    if (ctx->cut) return set_error(ctx, DDRW_EINVAL, "the context is itself cut into Dirichlet boxes");
    if (lsub < 2 || lsub > 6 || lsub % 2 || ctx->l % lsub || (ctx->l / lsub) % 2)
        return set_error(ctx, DDRW_EINVAL, "lsub must be 2, 4 or 6 with an even number of sub-blocks per block side");
    cudaSetDevice(ctx->device);
    // the field in the boundary layout, from the context's FP64 links (device buffer)
    double2 *lex = nullptr;
    if (cudaMalloc(&lex, sizeof(double2) * 36 * (size_t)ctx->V) != cudaSuccess)
        return set_error(ctx, DDRW_ENOMEM, "gauge field copy");
    gauge_to_lex(ctx, lex);
    ddrw_status st = sync(ctx);
    ddrw_ctx *aux = nullptr;
    const int blk[4] = {lsub, lsub, lsub, lsub};
    double fx = 0.0, lw = 0.0;
    if (!st) st = ddrw_create(&aux, ctx->dims, blk, ctx->device, ctx->stream);
    if (!st) st = ddrw_set_dirichlet(aux, ctx->l);
    if (!st) st = ddrw_set_params(aux, ctx->csw, ctx->m1, ctx->m2, ctx->antiperiodic);
    if (!st) st = ddrw_load_gauge(aux, (const double *)lex);
    if (!st) st = ddrw_set_solver(aux, ctx->prec, ctx->tol_outer, ctx->tol_block, ctx->maxiter);
    if (!st) st = ddrw_block_factor(aux, &fx);
    if (!st) {
        st = ddrw_estimate(aux, nhit, seed, 0, nullptr, exponents, &lw, rel_var, nullptr, nullptr);
        if (st == DDRW_ENOCONV) st = DDRW_OK, lw = NAN;
    }
    if (st && aux) ctx->err = std::string("nested block factor: ") + ddrw_last_error(aux);
    if (aux) ddrw_destroy(aux);
    cudaFree(lex);
    if (st) return st;
    out[0] = fx + lw;
    out[1] = fx;
    out[2] = lw;
    return lw == lw ? DDRW_OK : set_error(ctx, DDRW_ENOCONV, "nested block factor: a solve missed its tolerance");
}

}  // extern "C"
