// force.cu -- the adjoint of the estimate (K11): derivatives of e = eta^dag (Mh^dag Mh - 1) eta
// (Eq. 3, Eq. 8 with N = 1) with respect to every link and to the target mass m2.
//
// Reverse mode, with y = Mh eta = eta + delta and Mh = A2^-1 A1 (A_k = A(m_k) = P Dhat(m_k) P):
//
//   de = 2 Re <y, d Mh eta> = 2 Re <z, dA1 eta - dA2 y>,   z = A2^-dag y,
//   z  = y - P g5 D_bw u'_w,   D(m2) u' = g5 y          (A^-1 = P(1 - Dcal_bw D_wb)P and D^dag = g5 D g5)
//
// and, for A = P(1 - B^-1 C W^-1 E)P with B = D_bb, C = D_bw, W = D_ww, E = D_wb at one mass,
//
//   <z, dA v> = <zt, dD rho> + <wt, dD sigma>,
//   a = W^-1 E v,  q = B^-1 C a,  zt = B^-dag z = g5 B^-1 g5 z,  wt = W^-dag C^dag zt = g5 W^-1 E g5 zt,
//   rho = q (black) - a (white),  sigma = a (white) - v (black).
//
// So de = 2 Re sum_k c_k <L_k, dD R_k> over four (L, R) pairs per noise vector (c = +w for the m1
// pair, -w for the m2 pair, w the caller's weight of that e_j).  Per link U_mu(x), with the
// direction dU = i T_a U (T_a = lambda_a / 2, left multiplication):
//
//   hopping:  de_a = Im tr(T_a (U Y - Z U^dag)),  Y = sum c [(1-g_mu) R(x+mu)] L(x)^dag,
//                                                  Z = sum c [(1+g_mu) R(x)] L(x+mu)^dag  (spin summed)
//   clover:   de = -(csw/8) sum_{x, mu<nu} Im tr(dQ_{mu nu}(x) Omega_{mu nu}(x)),
//             Omega = Lambda + Lambda^dag,  Lambda_{mu nu} = sum c sigma_{mu nu} R L^dag (spin summed);
//             for a link W_k = U of a plaquette loop W_0 W_1 W_2 W_3 with Omega_j at the corner
//             before W_j:  E_k = O_{k+1} W_{k+1} W_{k+2} W_{k+3} + W_{k+1} O_{k+2} W_{k+2} W_{k+3}
//                                + W_{k+1} W_{k+2} O_{k+3} W_{k+3} + W_{k+1} W_{k+2} W_{k+3} O_k,
//             K += -(csw/8) i U E_k  (and +(csw/8) i E_k U^dag where the loop holds U^dag),
//   and de_a = Im tr(T_a K) for the total K of the link.
//
//   mass:     de/dm2 = -2 Re [<zt_2, q_2> + <wt_2, a_2>]   (m1 fixed).
//
// Solutions are recomputed (forward chain, one adjoint full solve, eight block solves batched as
// two mass slots), not stored from the forward pass.  The force kernels run in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "blas.cuh"
#include "ctx.h"
#include "stencil.cuh"

namespace ddrw {

ddrw_status estimate_fields_for_force(ddrw_ctx *ctx, int nhit, uint64_t seed, uint64_t hit0, const double *eta_user,
                                      double2 *eta, double2 *delta, double *exponents, SolveStats &stats);

namespace {

struct M3c {
    cpx<double> m[3][3];
};

__device__ __forceinline__ M3c m3_zero()
{
    M3c r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.m[i][j] = {0.0, 0.0};
    return r;
}
__device__ __forceinline__ M3c m3_mul(const M3c &a, const M3c &b)
{
    M3c c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cpx<double> t = cmul(a.m[i][0], b.m[0][j]);
            t = t + cmul(a.m[i][1], b.m[1][j]);
            t = t + cmul(a.m[i][2], b.m[2][j]);
            c.m[i][j] = t;
        }
    return c;
}
__device__ __forceinline__ M3c m3_dag(const M3c &a)
{
    M3c c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.m[i][j] = {a.m[j][i].re, -a.m[j][i].im};
    return c;
}
__device__ __forceinline__ void m3_acc(M3c &a, const M3c &b, double s)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) a.m[i][j] = a.m[i][j] + s * b.m[i][j];
}
__device__ __forceinline__ M3c load_link64(const double2 *U64, long V, int mu, long s)
{
    M3c r;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        double2 v = __ldg(U64 + ((long)mu * 9 + k) * V + s);
        r.m[k / 3][k % 3] = {v.x, v.y};
    }
    return r;
}

// chiral-basis gamma matrices (same convention as the operator): row a has one non-zero entry
__device__ __forceinline__ void gamma_entry(int mu, int a, int *col, cpx<double> *val)
{
    // g0: [[0,-1],[-1,0]];  g_k: [[0, -i s_k], [i s_k, 0]] in 2x2 spin blocks
    const int cols[4][4] = {{2, 3, 0, 1}, {3, 2, 1, 0}, {3, 2, 1, 0}, {2, 3, 0, 1}};
    *col = cols[mu][a];
    double re = 0, im = 0;
    if (mu == 0) re = -1;
    else if (mu == 1) im = (a < 2) ? -1 : 1;
    else if (mu == 2) re = (a == 0 || a == 3) ? -1 : 1;
    else im = (a == 0 || a == 3) ? -1 : 1;
    *val = {re, im};
}

// (1 + s g_mu) psi, full 4-spin result
__device__ __forceinline__ void one_pm_gamma(int mu, double s, const Spinor<double> &p, Spinor<double> &o)
{
#pragma unroll
    for (int a = 0; a < 4; a++) {
        int b;
        cpx<double> g;
        gamma_entry(mu, a, &b, &g);
#pragma unroll
        for (int c = 0; c < 3; c++) o.v[a][c] = p.v[a][c] + s * cmul(g, p.v[b][c]);
    }
}

// sigma_{mu nu} = (i/2)[g_mu, g_nu] as a dense 4x4
__device__ void sigma_matrix(int mu, int nu, cpx<double> S[4][4])
{
    cpx<double> G1[4][4], G2[4][4];
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) G1[a][b] = G2[a][b] = {0.0, 0.0};
    for (int a = 0; a < 4; a++) {
        int b;
        cpx<double> g;
        gamma_entry(mu, a, &b, &g);
        G1[a][b] = g;
        gamma_entry(nu, a, &b, &g);
        G2[a][b] = g;
    }
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            cpx<double> t = {0.0, 0.0};
            for (int k = 0; k < 4; k++) t = t + cmul(G1[a][k], G2[k][b]) - cmul(G2[a][k], G1[k][b]);
            S[a][b] = timesI(0.5 * t);
        }
}

__device__ __forceinline__ void load_sp64(const double2 *f, long V, long s, Spinor<double> &p)
{
#pragma unroll
    for (int k = 0; k < 12; k++) {
        double2 v = f[(long)k * V + s];
        p.v[k / 3][k % 3] = {v.x, v.y};
    }
}

// K += c * (sum_spin a_spin (x) b_spin^dag)
__device__ __forceinline__ void outer_acc(M3c &K, const Spinor<double> &a, const Spinor<double> &b, double c)
{
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) K.m[i][j] = K.m[i][j] + c * cmulc(b.v[sp][j], a.v[sp][i]);
}

struct ForceArgs {
    const double2 *L1, *R1, *L2, *R2;  // nrhs fields each
    const double *c;                   // per rhs coefficient
    int nrhs;
    long rs;
    const double2 *U64;
    double2 *omega;  // [6 planes][9][V]
    double csw;
    double *out;     // [V lexicographic][4][8]
};

// Omega_{mu nu}(x) = Lambda + Lambda^dag, Lambda = sum_rhs c sum_pairs sigma_{mu nu} R L^dag
template <int BL>
__global__ void k_omega(GeomDev g, ForceArgs a)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int pl = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, pl++) {
            cpx<double> S[4][4];
            sigma_matrix(mu, nu, S);
            M3c Lam = m3_zero();
            for (int r = 0; r < a.nrhs; r++) {
                for (int pr = 0; pr < 2; pr++) {
                    const double2 *L = (pr ? a.L2 : a.L1) + r * a.rs, *R = (pr ? a.R2 : a.R1) + r * a.rs;
                    Spinor<double> lv, rv, sr;
                    load_sp64(L, g.V, s, lv);
                    load_sp64(R, g.V, s, rv);
                    for (int al = 0; al < 4; al++)
                        for (int c = 0; c < 3; c++) {
                            cpx<double> t = {0.0, 0.0};
                            for (int be = 0; be < 4; be++) t = t + cmul(S[al][be], rv.v[be][c]);
                            sr.v[al][c] = t;
                        }
                    outer_acc(Lam, sr, lv, a.c[r]);
                }
            }
            M3c Om = Lam;
            m3_acc(Om, m3_dag(Lam), 1.0);
            for (int k = 0; k < 9; k++) a.omega[((long)pl * 9 + k) * g.V + s] = make_double2(Om.m[k / 3][k % 3].re, Om.m[k / 3][k % 3].im);
        }
}

__device__ __forceinline__ M3c load_omega(const double2 *om, long V, int pl, long s)
{
    M3c r;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        double2 v = om[((long)pl * 9 + k) * V + s];
        r.m[k / 3][k % 3] = {v.x, v.y};
    }
    return r;
}

__device__ __forceinline__ int plane_index(int mu, int nu)  // mu < nu
{
    const int idx[4][4] = {{-1, 0, 1, 2}, {-1, -1, 3, 4}, {-1, -1, -1, 5}, {-1, -1, -1, -1}};
    return idx[mu][nu];
}

template <int BL>
__device__ long site_shift(const GeomDev &g, const int *x, int mu, int dmu, int nu, int dnu)
{
    int c[4] = {x[0], x[1], x[2], x[3]};
    c[mu] = (c[mu] + dmu + g.L[mu]) % g.L[mu];
    c[nu] = (c[nu] + dnu + g.L[nu]) % g.L[nu];
    return internal_index<BL>(g, c[0], c[1], c[2], c[3]);
}

// E_k of a plaquette loop W0 W1 W2 W3 with Omega O_j at the corner before W_j (k: position of the link)
__device__ M3c loop_env(const M3c *W, const M3c *O, int k)
{
    const M3c &A = W[(k + 1) & 3], &B = W[(k + 2) & 3], &C = W[(k + 3) & 3];
    M3c AB = m3_mul(A, B), BC = m3_mul(B, C), ABC = m3_mul(AB, C);
    M3c E = m3_mul(O[(k + 1) & 3], ABC);
    m3_acc(E, m3_mul(m3_mul(A, O[(k + 2) & 3]), BC), 1.0);
    m3_acc(E, m3_mul(m3_mul(AB, O[(k + 3) & 3]), C), 1.0);
    m3_acc(E, m3_mul(ABC, O[k & 3]), 1.0);
    return E;
}

// per link: K from the hopping bilinears and the clover insertions, then de_a = Im tr(T_a K)
template <int BL>
__global__ void k_force(GeomDev g, ForceArgs a, const double *lam /* 8 Gell-Mann matrices, [8][3][3][2] */)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int mu = blockIdx.y;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    const int *o = g.blk_org + st.blk * 4;
    int x[4] = {o[0] + st.c[0], o[1] + st.c[1], o[2] + st.c[2], o[3] + st.c[3]};
    bool cross;
    int ph;
    long sf = neighbour<BL>(st, mu, +1, g, &cross, &ph);
    M3c U = load_link64(a.U64, g.V, mu, s);

    // hopping: Y = sum c [(1-g)R(x+mu)] L(x)^dag, Z = sum c [(1+g)R(x)] L(x+mu)^dag
    M3c Y = m3_zero(), Z = m3_zero();
    for (int r = 0; r < a.nrhs; r++)
        for (int pr = 0; pr < 2; pr++) {
            const double2 *L = (pr ? a.L2 : a.L1) + r * a.rs, *R = (pr ? a.R2 : a.R1) + r * a.rs;
            Spinor<double> l0, l1, r0, r1, t;
            load_sp64(L, g.V, s, l0);
            load_sp64(L, g.V, sf, l1);
            load_sp64(R, g.V, s, r0);
            load_sp64(R, g.V, sf, r1);
            one_pm_gamma(mu, -1.0, r1, t);
            outer_acc(Y, t, l0, a.c[r] * ph);
            one_pm_gamma(mu, +1.0, r0, t);
            outer_acc(Z, t, l1, a.c[r] * ph);
        }
    M3c K = m3_mul(U, Y);
    m3_acc(K, m3_mul(Z, m3_dag(U)), -1.0);

    // clover: the six plaquettes that contain U_mu(x)
    if (a.csw != 0.0) {
        const double f = a.csw / 8.0;
        for (int nu = 0; nu < 4; nu++) {
            if (nu == mu) continue;
            int al = mu < nu ? mu : nu, be = mu < nu ? nu : mu;
            int pl = plane_index(al, be);
            for (int side = 0; side < 2; side++) {
                // lower-left corner zc of the plaquette in the (al, be) plane holding the link
                int zc[4] = {x[0], x[1], x[2], x[3]};
                int k;  // position of the link in the loop
                if (mu == al) {  // the link runs along the first direction: W0 (side 0) or W2^dag (side 1)
                    if (side == 1) zc[be] = (zc[be] - 1 + g.L[be]) % g.L[be];
                    k = side == 0 ? 0 : 2;
                } else {          // along the second direction: W1 (side 0, corner x - al) or W3^dag (side 1, corner x)
                    if (side == 0) zc[al] = (zc[al] - 1 + g.L[al]) % g.L[al];
                    k = side == 0 ? 1 : 3;
                }
                long c0 = site_shift<BL>(g, zc, al, 0, be, 0), c1 = site_shift<BL>(g, zc, al, 1, be, 0);
                long c2 = site_shift<BL>(g, zc, al, 1, be, 1), c3 = site_shift<BL>(g, zc, al, 0, be, 1);
                M3c W[4], O[4];
                W[0] = load_link64(a.U64, g.V, al, c0);
                W[1] = load_link64(a.U64, g.V, be, c1);
                W[2] = m3_dag(load_link64(a.U64, g.V, al, c3));
                W[3] = m3_dag(load_link64(a.U64, g.V, be, c0));
                O[0] = load_omega(a.omega, g.V, pl, c0);
                O[1] = load_omega(a.omega, g.V, pl, c1);
                O[2] = load_omega(a.omega, g.V, pl, c2);
                O[3] = load_omega(a.omega, g.V, pl, c3);
                M3c E = loop_env(W, O, k);
                // K += -f i U E (link held as U) or +f i E U^dag (held as U^dag)
                M3c T = (k < 2) ? m3_mul(U, E) : m3_mul(E, m3_dag(U));
                double sg = (k < 2) ? -f : f;
                for (int i = 0; i < 9; i++) K.m[i / 3][i % 3] = K.m[i / 3][i % 3] + sg * timesI(T.m[i / 3][i % 3]);
            }
        }
    }
    // de_a = Im tr(T_a K), T_a = lambda_a / 2
    long lx = (((long)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
    for (int aa = 0; aa < 8; aa++) {
        cpx<double> tr = {0.0, 0.0};
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                cpx<double> l = {0.5 * lam[((aa * 3 + i) * 3 + j) * 2], 0.5 * lam[((aa * 3 + i) * 3 + j) * 2 + 1]};
                tr = tr + cmul(l, K.m[j][i]);
            }
        a.out[(lx * 4 + mu) * 8 + aa] = tr.im;
    }
}

// y = g5 x on every site (flip spins 2, 3)
__global__ void k_gamma5(long n12V, long V, int nrhs, long rs, const double2 *x, double2 *y)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n12V * nrhs) return;
    long r = i / n12V, e = i - r * n12V;
    long k = e / V;
    double2 v = x[r * rs + e];
    y[r * rs + e] = k >= 6 ? make_double2(-v.x, -v.y) : v;
}

// z = P (y - g5 t) on supp P, zero elsewhere
template <int BL>
__global__ void k_zvec(GeomDev g, const double2 *y, const double2 *t, double2 *z, long rs)
{
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    Site<BL> st;
    decode_site<BL>(s, g, st);
    bool in = false;
    if (st.blk < g.nblk_c)
        for (int m = 0; m < 4; m++) in |= (st.c[m] == 0 || st.c[m] == BL - 1);
    long o = (long)blockIdx.y * rs + s;
    for (int k = 0; k < 12; k++) {
        double2 a = y[o + (long)k * g.V], b = t[o + (long)k * g.V];
        if (k >= 6) b = make_double2(-b.x, -b.y);
        z[o + (long)k * g.V] = in ? make_double2(a.x - b.x, a.y - b.y) : make_double2(0.0, 0.0);
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

void gamma5(ddrw_ctx *ctx, const double2 *x, double2 *y, int nrhs)
{
    long n = 12 * ctx->V;
    ++ctx->launches;
    k_gamma5<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, ctx->stream>>>(n, ctx->V, nrhs, n, x, y);
}

void hop_between_rows64(ddrw_ctx *ctx, int rows, const double2 *in, double2 *out, int nrhs)
{
    DslashCall c;
    c.in = in;
    c.out = out;
    c.rstride = 12 * ctx->V;
    c.nrhs = nrhs;
    c.beta = -0.5;
    c.hopsel = 2;
    c.par0 = 0;
    c.npar = 2;
    c.blk0 = rows == DDRW_BLACK ? 0 : ctx->nblk_c;
    c.nblk = ctx->nblk_c;
    dslash64(ctx, c);
}

}  // namespace

static const double GELL_MANN[8][3][3][2] = {
    {{{0, 0}, {1, 0}, {0, 0}}, {{1, 0}, {0, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, -1}, {0, 0}}, {{0, 1}, {0, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}}},
    {{{1, 0}, {0, 0}, {0, 0}}, {{0, 0}, {-1, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {1, 0}}, {{0, 0}, {0, 0}, {0, 0}}, {{1, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, -1}}, {{0, 0}, {0, 0}, {0, 0}}, {{0, 1}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {0, 0}, {1, 0}}, {{0, 0}, {1, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, -1}}, {{0, 0}, {0, 1}, {0, 0}}},
    {{{0.57735026918962576, 0}, {0, 0}, {0, 0}},
     {{0, 0}, {0.57735026918962576, 0}, {0, 0}},
     {{0, 0}, {0, 0}, {-1.1547005383792515, 0}}},
};

}  // namespace ddrw

using namespace ddrw;

extern "C" ddrw_status ddrw_force(ddrw_ctx *ctx, int nhit, uint64_t seed, uint64_t hit_offset, const double *eta_user,
                                  const double *weights, double *exponents, double *dU, double *dm2,
                                  ddrw_solve_info *info)
{
    if (!ctx || nhit <= 0) return set_error(ctx, DDRW_EINVAL, "bad argument");
    if (!ctx->have_gauge) return set_error(ctx, DDRW_ESTATE, "no gauge field loaded");
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    const long V = ctx->V, rs = 12 * V;
    const int R2 = 2 * nhit;
    const size_t f1 = sizeof(double2) * rs * nhit, f2 = sizeof(double2) * rs * R2;
    const bool mixed = ctx->prec != DDRW_FP64;
    ddrw_status st;
    // fields: eta, delta (nhit) from the forward chain
    double2 *eta, *delta;
    if ((st = workspace(ctx, "frc_eta", f1, (void **)&eta))) return st;
    if ((st = workspace(ctx, "frc_delta", f1, (void **)&delta))) return st;
    std::vector<double> e(nhit);
    SolveStats stats;
    st = estimate_fields_for_force(ctx, nhit, seed, hit_offset, eta_user, eta, delta, e.data(), stats);
    ddrw_status conv = DDRW_OK;
    if (st == DDRW_ENOCONV) conv = st;
    else if (st) return st;
    if (exponents) std::copy(e.begin(), e.end(), exponents);

    double2 *F[8];
    const char *names[8] = {"frc_v2", "frc_a", "frc_q", "frc_zt", "frc_wt", "frc_t1", "frc_t2", "frc_z"};
    for (int k = 0; k < 8; k++)
        if ((st = workspace(ctx, names[k], f2, (void **)&F[k]))) return st;
    double2 *V2 = F[0], *A = F[1], *Q = F[2], *ZT = F[3], *WT = F[4], *T1 = F[5], *T2 = F[6], *Zf = F[7];
    // y = eta + delta into slot 1 of V2, eta into slot 0
    DDRW_CUDA_CHECK(cudaMemcpyAsync(V2, eta, f1, cudaMemcpyDeviceToDevice, ctx->stream));
    DDRW_CUDA_CHECK(cudaMemcpyAsync(V2 + rs * nhit, eta, f1, cudaMemcpyDeviceToDevice, ctx->stream));
    Blas<PrecD>::axpby(ctx, VecRange{V, 0, V, rs, nhit}, 1.0, delta, 1.0, V2 + rs * nhit);
    double2 *y = V2 + rs * nhit;

    MassSet m2s, m12;
    double mm[2] = {ctx->m1, ctx->m2};
    if ((st = make_massset(ctx, 1, &ctx->m2, &m2s))) return st;
    if ((st = make_massset(ctx, 2, mm, &m12))) return st;

    // z = y - P g5 D_bw u'_w, D(m2) u' = g5 y
    gamma5(ctx, y, T1, nhit);
    DDRW_CUDA_CHECK(cudaMemsetAsync(T2, 0, f1, ctx->stream));
    st = full_solve64(ctx, m2s, T1, T2, nhit, ctx->tol_outer, ctx->maxiter, ctx->prec, &stats);
    if (st == DDRW_ENOCONV) conv = st;
    else if (st) return st;
    DDRW_CUDA_CHECK(cudaMemsetAsync(T1, 0, f1, ctx->stream));
    hop_between_rows64(ctx, DDRW_BLACK, T2, T1, nhit);
    GeomDev g = geom_dev(ctx);
    {
        dim3 grid((unsigned)((V + 127) / 128), (unsigned)nhit);
        DISPATCH_BL(ctx, k_zvec, grid, 128, g, y, T1, Zf, rs);
    }
    // two mass slots (m1: v = eta, m2: v = y) of the four block solves
    auto bsolve = [&](int colour, const double2 *b, double2 *x) -> ddrw_status {
        DDRW_CUDA_CHECK(cudaMemsetAsync(x, 0, f2, ctx->stream));
        ddrw_status s2 = block_solve64(ctx, colour, m12, b, x, R2, ctx->tol_block, ctx->maxiter, ctx->prec, &stats);
        if (s2 == DDRW_ENOCONV) conv = s2;
        else if (s2) return s2;
        return DDRW_OK;
    };
    DDRW_CUDA_CHECK(cudaMemsetAsync(T1, 0, f2, ctx->stream));
    hop_between_rows64(ctx, DDRW_WHITE, V2, T1, R2);  // E v
    if ((st = bsolve(DDRW_WHITE, T1, A))) return st;  // a = W^-1 E v
    DDRW_CUDA_CHECK(cudaMemsetAsync(T1, 0, f2, ctx->stream));
    hop_between_rows64(ctx, DDRW_BLACK, A, T1, R2);  // C a
    if ((st = bsolve(DDRW_BLACK, T1, Q))) return st;  // q = B^-1 C a
    // g5 z in both slots
    gamma5(ctx, Zf, T1, nhit);
    DDRW_CUDA_CHECK(cudaMemcpyAsync(T1 + rs * nhit, T1, f1, cudaMemcpyDeviceToDevice, ctx->stream));
    if ((st = bsolve(DDRW_BLACK, T1, T2))) return st;  // B^-1 g5 z
    gamma5(ctx, T2, ZT, R2);                            // zt = g5 B^-1 g5 z
    DDRW_CUDA_CHECK(cudaMemsetAsync(T1, 0, f2, ctx->stream));
    hop_between_rows64(ctx, DDRW_WHITE, T2, T1, R2);  // E g5 zt
    if ((st = bsolve(DDRW_WHITE, T1, T2))) return st;
    gamma5(ctx, T2, WT, R2);  // wt = g5 W^-1 E g5 zt
    // rho = q - a (into Q), sigma = a - v (into A)
    Blas<PrecD>::axpby(ctx, VecRange{V, 0, V, rs, R2}, -1.0, A, 1.0, Q);
    Blas<PrecD>::axpby(ctx, VecRange{V, 0, V, rs, R2}, -1.0, V2, 1.0, A);

    // coefficients: +w (m1 slot), -w (m2 slot)
    std::vector<double> c(R2);
    for (int j = 0; j < nhit; j++) {
        double w = weights ? weights[j] : 1.0;
        c[j] = w;
        c[nhit + j] = -w;
    }
    double *cd, *lamd, *red;
    if ((st = workspace(ctx, "frc_c", sizeof(double) * (R2 + 144 + 12 * R2), (void **)&cd))) return st;
    lamd = cd + R2;
    red = lamd + 144;
    DDRW_CUDA_CHECK(cudaMemcpyAsync(cd, c.data(), sizeof(double) * R2, cudaMemcpyHostToDevice, ctx->stream));
    DDRW_CUDA_CHECK(cudaMemcpyAsync(lamd, GELL_MANN, sizeof(GELL_MANN), cudaMemcpyHostToDevice, ctx->stream));

    // de/dm2 = -2 Re[<zt_2, q_2> + <wt_2, a_2>] = -2 Re[<L1, rho> + <L2, sigma>] on the m2 slot
    if (dm2) {
        if ((st = Blas<PrecD>::norm_dot(ctx, VecRange{V, 0, V, rs, nhit}, ZT + rs * nhit, Q + rs * nhit, red))) return st;
        if ((st = Blas<PrecD>::norm_dot(ctx, VecRange{V, 0, V, rs, nhit}, WT + rs * nhit, A + rs * nhit, red + 3 * nhit)))
            return st;
        std::vector<double> h(6 * nhit);
        DDRW_CUDA_CHECK(cudaMemcpyAsync(h.data(), red, sizeof(double) * 6 * nhit, cudaMemcpyDeviceToHost, ctx->stream));
        DDRW_SYNC(ctx);
        for (int j = 0; j < nhit; j++) dm2[j] = -2.0 * (h[3 * j + 1] + h[3 * nhit + 3 * j + 1]);
    }
    if (dU) {
        double2 *omega;
        if ((st = workspace(ctx, "frc_omega", sizeof(double2) * 54 * V, (void **)&omega))) return st;
        double *out;
        void *dout;
        bool host;
        size_t ob = sizeof(double) * 32 * V;
        if ((st = stage_out(ctx, dU, ob, "stage_force", &dout, &host))) return st;
        out = (double *)dout;
        ForceArgs fa{ZT, Q, WT, A, cd, R2, rs, ctx->U64, omega, ctx->csw, out};
        {
            dim3 grid((unsigned)((V + 63) / 64));
            DISPATCH_BL(ctx, k_omega, grid, 64, g, fa);
        }
        {
            dim3 grid((unsigned)((V + 63) / 64), 4u);
            DISPATCH_BL(ctx, k_force, grid, 64, g, fa, lamd);
        }
        if ((st = finish_out(ctx, dU, out, ob, host))) return st;
    }
    if ((st = sync(ctx))) return st;
    if (info) {
        info->iters_outer = stats.outer_iters;
        info->cycles = stats.outer_cycles;
        info->fp64_dslash_calls = stats.fp64_dslash_full;
        info->block_iters_max = stats.block_iters_max;
        info->iters_inner_total = (int)std::min<long>(stats.block_iters_total, 2147483647L);
        info->true_rel_residual = stats.outer_rel_residual;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return conv;
}
