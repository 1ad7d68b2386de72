/*
 * ddrw_oracle.c -- plain, slow FP64 CPU oracle for the domain-decomposed stochastic estimate of
 * 1/det(M^dag M) (Finkenrath, Knechtli, Leder, Lattice 2012).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg load this file's library.  It shares no code, header, table or helper with the CUDA
 * library: it has its own geometry, gamma matrices, clover term, operator, solver, Philox
 * generator and estimator, each written from its definition.
 *
 * Conventions (the paper names the operator, Sec. 1 and Sec. 2, but prints no formula for it;
 * the readings below are the ones the whole project uses):
 *
 *   site index   x = ((t*L1 + x1)*L2 + x2)*L3 + x3, dims L = (T, X, Y, Z);
 *   links        U[x][mu][a][b], U_mu(x) the link from x to x + mu;
 *   spinor       psi[x][alpha][a], component index 3*alpha + a (12 per site, the "12V" of Eq. 5);
 *
 *   (D(m) psi)(x) = (4 + m) psi(x) + C(x) psi(x)
 *                   - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *
 *   C(x) = csw (i/4) sum_{mu,nu} sigma_{mu nu} (x) Fhat_{mu nu}(x),  sigma_{mu nu} = (i/2)[g_mu, g_nu],
 *   Fhat_{mu nu} = (Q_{mu nu} - Q_{nu mu}) / 8,  Q_{mu nu} = sum of the four plaquette leaves at x.
 *
 * The mass enters additively, so D(m1) - D(m2) = (m1 - m2) * 1, the structure behind
 * M = 1 + dm * D^-1(m2) of Eq. 6.  Gamma matrices are in the chiral basis with
 * g5 = g0 g1 g2 g3 = diag(1, 1, -1, -1).
 *
 * Blocks (Eq. 1): block coordinate b_mu = floor(x_mu / B_mu); colour = (sum_mu b_mu) mod 2,
 * colour 0 = black.  D_XY is the restriction of D to rows in X and columns in Y, so D_bb and
 * D_ww are block-diagonal and D_bw, D_wb hold exactly the hops between blocks.  supp P is the set
 * of black sites with a neighbour in a white block (all 12 components), so that D_wb P = D_wb
 * (Sec. 1).
 *
 * Every solve is CG on the normal equations (CGNR) in FP64, stopped on the recomputed true
 * residual ||b - A x|| / ||b||.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define NC 3
#define NS 4
#define NSC 12

enum { SEL_BLACK = 0, SEL_WHITE = 1, SEL_ALL = 2 };

typedef struct {
    int L[4];
    int B[4];
    long V;
    int antiperiodic_t;
    double csw;
    cplx *U;        /* [V][4][3][3] */
    cplx *C;        /* [V][12][12] dense clover term */
    unsigned char *colour; /* [V] 0 black, 1 white */
    unsigned char *suppP;  /* [V] 1 if black site with a white neighbour */
} orc_lat;

/* ------------------------------------------------------------------ geometry */

static void site_coords(const orc_lat *g, long s, int c[4])
{
    c[3] = (int)(s % g->L[3]); s /= g->L[3];
    c[2] = (int)(s % g->L[2]); s /= g->L[2];
    c[1] = (int)(s % g->L[1]); s /= g->L[1];
    c[0] = (int)s;
}

static long site_index(const orc_lat *g, const int c[4])
{
    return (((long)c[0] * g->L[1] + c[1]) * g->L[2] + c[2]) * g->L[3] + c[3];
}

/* neighbour of s one step in direction mu (dir = +1 or -1), periodic wrap */
static long neighbour(const orc_lat *g, long s, int mu, int dir)
{
    int c[4];
    site_coords(g, s, c);
    c[mu] = (c[mu] + dir + g->L[mu]) % g->L[mu];
    return site_index(g, c);
}

/* boundary phase of the hop s -> s + dir*mu: -1 across the time boundary if antiperiodic */
static double hop_phase(const orc_lat *g, long s, int mu, int dir)
{
    if (!g->antiperiodic_t || mu != 0) return 1.0;
    int c[4];
    site_coords(g, s, c);
    if (dir > 0 && c[0] == g->L[0] - 1) return -1.0;
    if (dir < 0 && c[0] == 0) return -1.0;
    return 1.0;
}

/* ------------------------------------------------------------------ gamma matrices */

static cplx GAMMA[4][4][4];
static int gamma_ready = 0;

static void init_gamma(void)
{
    if (gamma_ready) return;
    memset(GAMMA, 0, sizeof(GAMMA));
    /* g0 = [[0, -1], [-1, 0]] in 2x2 spin blocks */
    GAMMA[0][0][2] = -1; GAMMA[0][1][3] = -1; GAMMA[0][2][0] = -1; GAMMA[0][3][1] = -1;
    /* g_k = [[0, -i s_k], [i s_k, 0]], s_k the Pauli matrices */
    GAMMA[1][0][3] = -I; GAMMA[1][1][2] = -I; GAMMA[1][2][1] = I;  GAMMA[1][3][0] = I;
    GAMMA[2][0][3] = -1; GAMMA[2][1][2] = 1;  GAMMA[2][2][1] = 1;  GAMMA[2][3][0] = -1;
    GAMMA[3][0][2] = -I; GAMMA[3][1][3] = I;  GAMMA[3][2][0] = I;  GAMMA[3][3][1] = -I;
    gamma_ready = 1;
}

void orc_gamma(int mu, double *out /* [4][4] complex */)
{
    init_gamma();
    memcpy(out, GAMMA[mu], sizeof(GAMMA[mu]));
}

/* ------------------------------------------------------------------ 3x3 complex helpers */

static void m3_mul(const cplx *a, const cplx *b, cplx *c)      /* c = a b */
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
}

static void m3_dag(const cplx *a, cplx *c)                     /* c = a^dag */
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c[3 * i + j] = conj(a[3 * j + i]);
}

static void m3_prod4(const cplx *a, const cplx *b, const cplx *c, const cplx *d, cplx *out)
{
    cplx t1[9], t2[9];
    m3_mul(a, b, t1);
    m3_mul(t1, c, t2);
    m3_mul(t2, d, out);
}

static const cplx *link(const orc_lat *g, long s, int mu) { return g->U + ((size_t)s * 4 + mu) * 9; }

/* ------------------------------------------------------------------ clover term */

/* Q_{mu nu}(x): the four counter-clockwise plaquette leaves in the (mu, nu) plane at x. */
static void clover_leaves(const orc_lat *g, long x, int mu, int nu, cplx *Q)
{
    cplx Ud[4][9], leaf[9];
    long xpm = neighbour(g, x, mu, +1), xpn = neighbour(g, x, nu, +1);
    long xmm = neighbour(g, x, mu, -1), xmn = neighbour(g, x, nu, -1);
    long xmm_pn = neighbour(g, xmm, nu, +1), xmm_mn = neighbour(g, xmm, nu, -1);
    long xmn_pm = neighbour(g, xmn, mu, +1);
    for (int k = 0; k < 9; k++) Q[k] = 0;

    /* leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
    m3_dag(link(g, xpn, mu), Ud[0]);
    m3_dag(link(g, x, nu), Ud[1]);
    m3_prod4(link(g, x, mu), link(g, xpm, nu), Ud[0], Ud[1], leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];
    /* leaf 2: U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu) */
    m3_dag(link(g, xmm_pn, mu), Ud[0]);
    m3_dag(link(g, xmm, nu), Ud[1]);
    m3_prod4(link(g, x, nu), Ud[0], Ud[1], link(g, xmm, mu), leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];
    /* leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu) */
    m3_dag(link(g, xmm, mu), Ud[0]);
    m3_dag(link(g, xmm_mn, nu), Ud[1]);
    m3_prod4(Ud[0], Ud[1], link(g, xmm_mn, mu), link(g, xmn, nu), leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];
    /* leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag */
    m3_dag(link(g, xmn, nu), Ud[0]);
    m3_dag(link(g, x, mu), Ud[1]);
    m3_prod4(Ud[0], link(g, xmn, mu), link(g, xmn_pm, nu), Ud[1], leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];
}

static void build_clover(orc_lat *g)
{
    init_gamma();
    /* sigma_{mu nu} = (i/2)[g_mu, g_nu] */
    cplx sigma[4][4][4][4];
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++)
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    cplx s = 0;
                    for (int k = 0; k < 4; k++)
                        s += GAMMA[mu][a][k] * GAMMA[nu][k][b] - GAMMA[nu][a][k] * GAMMA[mu][k][b];
                    sigma[mu][nu][a][b] = 0.5 * I * s;
                }
#pragma omp parallel for schedule(static)
    for (long x = 0; x < g->V; x++) {
        cplx *Cx = g->C + (size_t)x * NSC * NSC;
        for (int k = 0; k < NSC * NSC; k++) Cx[k] = 0;
        if (g->csw == 0.0) continue;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = 0; nu < 4; nu++) {
                if (mu == nu) continue;
                cplx Q[9], F[9];
                clover_leaves(g, x, mu, nu, Q);
                /* Fhat = (Q_{mu nu} - Q_{nu mu}) / 8 and Q_{nu mu} = Q_{mu nu}^dag */
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) F[3 * i + j] = (Q[3 * i + j] - conj(Q[3 * j + i])) / 8.0;
                cplx pref = g->csw * 0.25 * I;
                for (int al = 0; al < 4; al++)
                    for (int be = 0; be < 4; be++) {
                        cplx s = pref * sigma[mu][nu][al][be];
                        if (s == 0) continue;
                        for (int a = 0; a < 3; a++)
                            for (int b = 0; b < 3; b++)
                                Cx[(3 * al + a) * NSC + 3 * be + b] += s * F[3 * a + b];
                    }
            }
    }
}

/* ------------------------------------------------------------------ context */

void *orc_create(const int *L, const int *B, const double *U, double csw, int antiperiodic_t)
{
    orc_lat *g = (orc_lat *)calloc(1, sizeof(orc_lat));
    if (!g) return NULL;
    g->V = 1;
    for (int mu = 0; mu < 4; mu++) {
        g->L[mu] = L[mu];
        g->B[mu] = B[mu];
        g->V *= L[mu];
    }
    g->csw = csw;
    g->antiperiodic_t = antiperiodic_t;
    g->U = (cplx *)malloc(sizeof(cplx) * 36 * (size_t)g->V);
    g->C = (cplx *)malloc(sizeof(cplx) * NSC * NSC * (size_t)g->V);
    g->colour = (unsigned char *)malloc((size_t)g->V);
    g->suppP = (unsigned char *)malloc((size_t)g->V);
    if (!g->U || !g->C || !g->colour || !g->suppP) {
        free(g->U); free(g->C); free(g->colour); free(g->suppP); free(g);
        return NULL;
    }
    memcpy(g->U, U, sizeof(cplx) * 36 * (size_t)g->V);
    for (long x = 0; x < g->V; x++) {
        int c[4], sum = 0;
        site_coords(g, x, c);
        for (int mu = 0; mu < 4; mu++) sum += c[mu] / g->B[mu];
        g->colour[x] = (unsigned char)(sum % 2);
    }
    for (long x = 0; x < g->V; x++) {
        int in_p = 0;
        if (g->colour[x] == 0)
            for (int mu = 0; mu < 4; mu++)
                for (int dir = -1; dir <= 1; dir += 2)
                    if (g->colour[neighbour(g, x, mu, dir)] == 1) in_p = 1;
        g->suppP[x] = (unsigned char)in_p;
    }
    build_clover(g);
    return g;
}

/* Replace the links of the hopping term, keeping the clover term built at creation: with links
 * that are zero across the faces of boxes, D becomes the direct sum of the boxes' Dirichlet
 * operators (each D_k of Eq. 7 is such a box operator: hops inside the block, the full clover). */
void orc_set_hopping_links(void *p, const double *U)
{
    orc_lat *g = (orc_lat *)p;
    memcpy(g->U, U, sizeof(cplx) * 36 * (size_t)g->V);
}

void orc_destroy(void *p)
{
    orc_lat *g = (orc_lat *)p;
    if (!g) return;
    free(g->U); free(g->C); free(g->colour); free(g->suppP); free(g);
}

long orc_volume(void *p) { return ((orc_lat *)p)->V; }

void orc_clover_matrix(void *p, long x, double *out /* [12][12] complex */)
{
    orc_lat *g = (orc_lat *)p;
    memcpy(out, g->C + (size_t)x * NSC * NSC, sizeof(cplx) * NSC * NSC);
}

void orc_colour(void *p, unsigned char *out) { orc_lat *g = (orc_lat *)p; memcpy(out, g->colour, (size_t)g->V); }
void orc_suppP(void *p, unsigned char *out) { orc_lat *g = (orc_lat *)p; memcpy(out, g->suppP, (size_t)g->V); }

/* ------------------------------------------------------------------ the operator */

static int selected(const orc_lat *g, long x, int sel)
{
    return sel == SEL_ALL || g->colour[x] == sel;
}

/*
 * out = D_{rows, cols}(m) in   (dagger = 0)   or   out = (D^dag)_{rows, cols}(m) in   (dagger = 1).
 * Rows outside `rowsel` are set to zero; input sites outside `colsel` are ignored.
 * D^dag is written out from the conjugate transpose of the hopping matrix elements:
 * (D^dag)[x, x+mu] = -1/2 (1 + g_mu) U_mu(x), (D^dag)[x, x-mu] = -1/2 (1 - g_mu) U_mu(x-mu)^dag,
 * and C^dag on the diagonal.
 */
static void apply_dirac(const orc_lat *g, double m, int dagger, int rowsel, int colsel,
                        const cplx *in, cplx *out)
{
    init_gamma();
#pragma omp parallel for schedule(static)
    for (long x = 0; x < g->V; x++) {
        cplx acc[NSC];
        for (int i = 0; i < NSC; i++) acc[i] = 0;
        if (!selected(g, x, rowsel)) {
            memcpy(out + (size_t)x * NSC, acc, sizeof(acc));
            continue;
        }
        if (selected(g, x, colsel)) {
            const cplx *Cx = g->C + (size_t)x * NSC * NSC;
            const cplx *px = in + (size_t)x * NSC;
            for (int i = 0; i < NSC; i++) {
                cplx s = (4.0 + m) * px[i];
                for (int j = 0; j < NSC; j++)
                    s += (dagger ? conj(Cx[j * NSC + i]) : Cx[i * NSC + j]) * px[j];
                acc[i] += s;
            }
        }
        for (int mu = 0; mu < 4; mu++) {
            for (int dir = -1; dir <= 1; dir += 2) {
                long y = neighbour(g, x, mu, dir);
                if (!selected(g, y, colsel)) continue;
                double ph = hop_phase(g, x, mu, dir);
                /* colour matrix: U_mu(x) forward, U_mu(x-mu)^dag backward */
                cplx W[9];
                if (dir > 0) memcpy(W, link(g, x, mu), sizeof(W));
                else m3_dag(link(g, y, mu), W);
                /* spin matrix: (1 - s g_mu) with s = +1 forward / -1 backward; flipped for D^dag */
                double s = (dir > 0) ? 1.0 : -1.0;
                if (dagger) s = -s;
                const cplx *py = in + (size_t)y * NSC;
                cplx Wpsi[NSC];
                for (int al = 0; al < 4; al++)
                    for (int a = 0; a < 3; a++) {
                        cplx t = 0;
                        for (int b = 0; b < 3; b++) t += W[3 * a + b] * py[3 * al + b];
                        Wpsi[3 * al + a] = t;
                    }
                for (int al = 0; al < 4; al++)
                    for (int a = 0; a < 3; a++) {
                        cplx t = Wpsi[3 * al + a];
                        for (int be = 0; be < 4; be++) t -= s * GAMMA[mu][al][be] * Wpsi[3 * be + a];
                        acc[3 * al + a] -= 0.5 * ph * t;
                    }
            }
        }
        memcpy(out + (size_t)x * NSC, acc, sizeof(acc));
    }
}

void orc_apply(void *p, double m, int dagger, int rowsel, int colsel, const double *in, double *out)
{
    apply_dirac((const orc_lat *)p, m, dagger, rowsel, colsel, (const cplx *)in, (cplx *)out);
}

/* ------------------------------------------------------------------ vector helpers */

static double vnorm2(long n, const cplx *a)
{
    double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long i = 0; i < n; i++) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

static cplx vdot(long n, const cplx *a, const cplx *b) /* sum conj(a) b */
{
    double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (long i = 0; i < n; i++) {
        cplx t = conj(a[i]) * b[i];
        re += creal(t);
        im += cimag(t);
    }
    return re + I * im;
}

/* ------------------------------------------------------------------ CGNR */

/*
 * Solve D_{sel,sel}(m) x = b by CG on (D^dag D) x = D^dag b, x started from zero.  Returns the
 * number of operator applications of D (not counting D^dag), or -1 if the true relative residual
 * did not reach tol within maxiter iterations; *relres receives the final true relative residual.
 */
static long cgnr_d(const orc_lat *g, double m, int dag, int sel, const cplx *b, cplx *x, double tol, long maxiter,
                   double *relres);

static long cgnr(const orc_lat *g, double m, int sel, const cplx *b, cplx *x, double tol, long maxiter,
                 double *relres)
{
    return cgnr_d(g, m, 0, sel, b, x, tol, maxiter, relres);
}

/* CGNR for A = D_{sel,sel} (dag = 0) or A = (D^dag)_{sel,sel} (dag = 1): CG on A^dag A x = A^dag b. */
static long cgnr_d(const orc_lat *g, double m, int dag, int sel, const cplx *b, cplx *x, double tol, long maxiter,
                   double *relres)
{
    long n = g->V * NSC;
    cplx *r = (cplx *)malloc(sizeof(cplx) * n), *z = (cplx *)malloc(sizeof(cplx) * n);
    cplx *pp = (cplx *)malloc(sizeof(cplx) * n), *w = (cplx *)malloc(sizeof(cplx) * n);
    double bn2 = vnorm2(n, b);
    long it = 0;
    memset(x, 0, sizeof(cplx) * n);
    if (bn2 == 0.0) {
        if (relres) *relres = 0.0;
        free(r); free(z); free(pp); free(w);
        return 0;
    }
    double res = 1.0;
    for (int restart = 0; restart < 50 && it < maxiter; restart++) {
        /* true residual r = b - A x */
        apply_dirac(g, m, dag, sel, sel, x, w);
        for (long i = 0; i < n; i++) r[i] = b[i] - w[i];
        res = sqrt(vnorm2(n, r) / bn2);
        if (res <= tol) break;
        apply_dirac(g, m, !dag, sel, sel, r, z);
        memcpy(pp, z, sizeof(cplx) * n);
        double zz = vnorm2(n, z);
        while (it < maxiter) {
            apply_dirac(g, m, dag, sel, sel, pp, w);
            it++;
            double ww = vnorm2(n, w);
            if (ww == 0.0) break;
            double alpha = zz / ww;
            for (long i = 0; i < n; i++) {
                x[i] += alpha * pp[i];
                r[i] -= alpha * w[i];
            }
            double rr = vnorm2(n, r);
            if (sqrt(rr / bn2) <= 0.5 * tol) break;
            apply_dirac(g, m, !dag, sel, sel, r, z);
            double zz_new = vnorm2(n, z);
            double beta = zz_new / zz;
            zz = zz_new;
            for (long i = 0; i < n; i++) pp[i] = z[i] + beta * pp[i];
        }
    }
    apply_dirac(g, m, dag, sel, sel, x, w);
    for (long i = 0; i < n; i++) r[i] = b[i] - w[i];
    res = sqrt(vnorm2(n, r) / bn2);
    if (relres) *relres = res;
    free(r); free(z); free(pp); free(w);
    return res <= tol ? it : -1;
}

long orc_solve(void *p, double m, int sel, const double *b, double *x, double tol, long maxiter, double *relres)
{
    return cgnr((const orc_lat *)p, m, sel, (const cplx *)b, (cplx *)x, tol, maxiter, relres);
}

/* ------------------------------------------------------------------ the estimator, one noise vector */

static void mask_suppP(const orc_lat *g, cplx *v)
{
    for (long x = 0; x < g->V; x++)
        if (!g->suppP[x])
            for (int i = 0; i < NSC; i++) v[(size_t)x * NSC + i] = 0;
}

/*
 * One term of Eq. 3 / Eq. 8 (N = 1) for the Schur complement:  e = eta^dag (Mh^dag Mh - 1) eta with
 * Mh = A(m2)^-1 A(m1), A(m) = P Dhat(m) P and Dhat(m) = 1 - D_bb^-1 D_bw D_ww^-1 D_wb (Sec. 1).
 *
 *   r     = (A(m1) - A(m2)) eta
 *         = dm P D_bb(m1)^-1 [ D_bw a12 + D_bb(m2)^-1 D_bw a2 ],  dm = m1 - m2,
 *           u = D_wb eta, a2 = D_ww(m2)^-1 u, a12 = D_ww(m1)^-1 a2
 *           (the resolvent identity D(m1)^-1 - D(m2)^-1 = -dm D(m1)^-1 D(m2)^-1 on each block operator);
 *   delta = A(m2)^-1 r = r - P x_b, where D(m2) x = (0_b ; D_wb r)   (Dhat^-1 = 1 - P Dcal_bw D_wb, Sec. 1);
 *   e     = ||eta + delta||^2 - ||eta||^2 = ||delta||^2 + 2 Re <eta, delta>.
 *
 * eta is a full-lattice vector that must vanish outside supp P.  r_out and delta_out (full-lattice,
 * may be NULL) receive r and delta.  iters[0..4] (may be NULL) receive the CGNR counts of the five
 * solves.  Returns 0 on success, -1 if a solve failed to converge.
 */
int orc_exponent(void *p, double m1, double m2, const double *eta_d, double tol_block, double tol_outer,
                 long maxiter, double *e_out, double *r_out, double *delta_out, long *iters)
{
    const orc_lat *g = (const orc_lat *)p;
    const cplx *eta = (const cplx *)eta_d;
    long n = g->V * NSC;
    double dm = m1 - m2, rel;
    cplx *u = (cplx *)calloc(n, sizeof(cplx)), *a2 = (cplx *)calloc(n, sizeof(cplx));
    cplx *a12 = (cplx *)calloc(n, sizeof(cplx)), *c = (cplx *)calloc(n, sizeof(cplx));
    cplx *c2 = (cplx *)calloc(n, sizeof(cplx)), *t = (cplx *)calloc(n, sizeof(cplx));
    cplx *r = (cplx *)calloc(n, sizeof(cplx)), *bfull = (cplx *)calloc(n, sizeof(cplx));
    cplx *x = (cplx *)calloc(n, sizeof(cplx)), *delta = (cplx *)calloc(n, sizeof(cplx));
    long it[5] = {0, 0, 0, 0, 0};
    int status = 0;

    apply_dirac(g, 0.0, 0, SEL_WHITE, SEL_BLACK, eta, u);             /* u = D_wb eta */
    if ((it[0] = cgnr(g, m2, SEL_WHITE, u, a2, tol_block, maxiter, &rel)) < 0) status = -1;
    if ((it[1] = cgnr(g, m1, SEL_WHITE, a2, a12, tol_block, maxiter, &rel)) < 0) status = -1;
    apply_dirac(g, 0.0, 0, SEL_BLACK, SEL_WHITE, a12, c);              /* c = D_bw a12 */
    apply_dirac(g, 0.0, 0, SEL_BLACK, SEL_WHITE, a2, c2);              /* c2 = D_bw a2 */
    if ((it[2] = cgnr(g, m2, SEL_BLACK, c2, t, tol_block, maxiter, &rel)) < 0) status = -1;
    for (long i = 0; i < n; i++) c[i] += t[i];
    if ((it[3] = cgnr(g, m1, SEL_BLACK, c, r, tol_block, maxiter, &rel)) < 0) status = -1;
    for (long i = 0; i < n; i++) r[i] *= dm;
    mask_suppP(g, r);                                                  /* r = dm P D_bb(m1)^-1 [...] */

    apply_dirac(g, 0.0, 0, SEL_WHITE, SEL_BLACK, r, bfull);           /* b = (0_b ; D_wb r) */
    if ((it[4] = cgnr(g, m2, SEL_ALL, bfull, x, tol_outer, maxiter, &rel)) < 0) status = -1;
    for (long i = 0; i < n; i++) delta[i] = (g->suppP[i / NSC]) ? r[i] - x[i] : 0.0;

    double dd = vnorm2(n, delta);
    cplx ed = vdot(n, eta, delta);
    *e_out = dd + 2.0 * creal(ed);
    if (r_out) memcpy(r_out, r, sizeof(cplx) * n);
    if (delta_out) memcpy(delta_out, delta, sizeof(cplx) * n);
    if (iters) memcpy(iters, it, sizeof(it));
    free(u); free(a2); free(a12); free(c); free(c2); free(t); free(r); free(bfull); free(x); free(delta);
    return status;
}

/* ------------------------------------------------------------------ Philox4x32-10 and the noise */

/*
 * Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11): per round, two 32x32 -> 64-bit products of counter words with the
 * multipliers 0xD2511F53 and 0xCD9E8D57 are mixed with the other counter words and the key; the
 * key is bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.
 */
void orc_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Complex Gaussian noise for Eq. 3 with E|eta_k|^2 = 1, as the Gaussian integral requires.
 * Component k of hit h: Philox counter (k, h, 0, 0), key (seed mod 2^32, seed / 2^32);
 * u1 = (w0 + 1) 2^-32 in (0, 1], u2 = w1 2^-32;
 * eta_k = sqrt(-ln u1) (cos 2 pi u2 + i sin 2 pi u2)   (Box-Muller, real and imaginary part N(0, 1/2)).
 * Writes n complex numbers (2n doubles) for hits hit0 .. hit0 + nhit - 1, hit-major.
 */
void orc_noise(uint64_t seed, uint64_t hit0, int nhit, long n, double *eta)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    const double two_pi = 6.283185307179586476925286766559;
    for (int h = 0; h < nhit; h++)
        for (long k = 0; k < n; k++) {
            uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(hit0 + (uint64_t)h), 0u, 0u};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            double u1 = ((double)w[0] + 1.0) * (1.0 / 4294967296.0);
            double u2 = (double)w[1] * (1.0 / 4294967296.0);
            double rho = sqrt(-log(u1));
            eta[2 * ((size_t)h * n + k)] = rho * cos(two_pi * u2);
            eta[2 * ((size_t)h * n + k) + 1] = rho * sin(two_pi * u2);
        }
}

/* ------------------------------------------------------------------ the adjoint (link and mass derivatives) */

/*
 * Derivative of one clover leaf product with respect to the link (lx, lmu) in direction
 * dU = i T_a U (T_a = lambda_a / 2): product rule over the leaf's four factors; a factor that is
 * the link becomes i T_a U, a factor that is its adjoint becomes -i U^dag T_a, the others stay.
 */
typedef struct {
    long site;
    int dir;
    int dag;
} factor;

static const double LAMBDA8 = 0.57735026918962576451;

static void gell_mann_half(int a, cplx *T)
{
    for (int k = 0; k < 9; k++) T[k] = 0;
    switch (a) {
    case 0: T[1] = T[3] = 0.5; break;
    case 1: T[1] = -0.5 * I; T[3] = 0.5 * I; break;
    case 2: T[0] = 0.5; T[4] = -0.5; break;
    case 3: T[2] = T[6] = 0.5; break;
    case 4: T[2] = -0.5 * I; T[6] = 0.5 * I; break;
    case 5: T[5] = T[7] = 0.5; break;
    case 6: T[5] = -0.5 * I; T[7] = 0.5 * I; break;
    default: T[0] = T[4] = 0.5 * LAMBDA8; T[8] = -LAMBDA8; break;
    }
}

static void factor_matrix(const orc_lat *g, factor f, long lx, int lmu, const cplx *T, int deriv, cplx *out)
{
    const cplx *u = link(g, f.site, f.dir);
    if (!deriv) {
        if (f.dag) m3_dag(u, out);
        else memcpy(out, u, sizeof(cplx) * 9);
        return;
    }
    (void)lx; (void)lmu;
    cplx t[9];
    if (!f.dag) { /* i T U */
        m3_mul(T, u, t);
        for (int k = 0; k < 9; k++) out[k] = I * t[k];
    } else { /* -i U^dag T */
        cplx ud[9];
        m3_dag(u, ud);
        m3_mul(ud, T, t);
        for (int k = 0; k < 9; k++) out[k] = -I * t[k];
    }
}

/* dQ_{mu nu}(y): derivative of the four-leaf sum at y with respect to link (lx, lmu), generator a */
static int clover_leaves_deriv(const orc_lat *g, long y, int mu, int nu, long lx, int lmu, const cplx *T, cplx *dQ)
{
    long ypm = neighbour(g, y, mu, +1), ypn = neighbour(g, y, nu, +1);
    long ymm = neighbour(g, y, mu, -1), ymn = neighbour(g, y, nu, -1);
    long ymm_pn = neighbour(g, ymm, nu, +1), ymm_mn = neighbour(g, ymm, nu, -1);
    long ymn_pm = neighbour(g, ymn, mu, +1);
    factor leaves[4][4] = {
        {{y, mu, 0}, {ypm, nu, 0}, {ypn, mu, 1}, {y, nu, 1}},
        {{y, nu, 0}, {ymm_pn, mu, 1}, {ymm, nu, 1}, {ymm, mu, 0}},
        {{ymm, mu, 1}, {ymm_mn, nu, 1}, {ymm_mn, mu, 0}, {ymn, nu, 0}},
        {{ymn, nu, 1}, {ymn, mu, 0}, {ymn_pm, nu, 0}, {y, mu, 1}},
    };
    int any = 0;
    for (int k = 0; k < 9; k++) dQ[k] = 0;
    for (int l = 0; l < 4; l++)
        for (int d = 0; d < 4; d++) {
            if (leaves[l][d].site != lx || leaves[l][d].dir != lmu) continue;
            any = 1;
            cplx m[4][9], t1[9], t2[9], prod[9];
            for (int f = 0; f < 4; f++) factor_matrix(g, leaves[l][f], lx, lmu, T, f == d, m[f]);
            m3_mul(m[0], m[1], t1);
            m3_mul(t1, m[2], t2);
            m3_mul(t2, m[3], prod);
            for (int k = 0; k < 9; k++) dQ[k] += prod[k];
        }
    return any;
}

/* out_k(y) = dC(y) in_k(y) on every site y whose clover term depends on link (lx, lmu), for k < nin;
 * returns the number of those sites, listed in sites[] */
static int apply_dclover(const orc_lat *g, long lx, int lmu, const cplx *T, int nin, cplx *const *in, cplx *const *out,
                         long *sites)
{
    init_gamma();
    cplx sigma[4][4][4][4];
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++)
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    cplx s = 0;
                    for (int k = 0; k < 4; k++)
                        s += GAMMA[mu][a][k] * GAMMA[nu][k][b] - GAMMA[nu][a][k] * GAMMA[mu][k][b];
                    sigma[mu][nu][a][b] = 0.5 * I * s;
                }
    /* candidate sites: lx, lx + lmu, and their shifts by +-nu */
    long cand[64];
    int nc = 0;
    long base[2] = {lx, neighbour(g, lx, lmu, +1)};
    for (int b = 0; b < 2; b++) {
        cand[nc++] = base[b];
        for (int nu = 0; nu < 4; nu++) {
            if (nu == lmu) continue;
            cand[nc++] = neighbour(g, base[b], nu, +1);
            cand[nc++] = neighbour(g, base[b], nu, -1);
        }
    }
    int ns = 0;
    for (int i = 0; i < nc; i++) {
        int dup = 0;
        for (int j = 0; j < ns; j++)
            if (sites[j] == cand[i]) dup = 1;
        if (dup) continue;
        long y = cand[i];
        cplx dC[NSC * NSC];
        for (int k = 0; k < NSC * NSC; k++) dC[k] = 0;
        int any = 0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = 0; nu < 4; nu++) {
                if (mu == nu) continue;
                cplx dQ[9], dF[9];
                if (!clover_leaves_deriv(g, y, mu, nu, lx, lmu, T, dQ)) continue;
                any = 1;
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) dF[3 * a + b] = (dQ[3 * a + b] - conj(dQ[3 * b + a])) / 8.0;
                cplx pref = g->csw * 0.25 * I;
                for (int al = 0; al < 4; al++)
                    for (int be = 0; be < 4; be++) {
                        cplx s = pref * sigma[mu][nu][al][be];
                        if (s == 0) continue;
                        for (int a = 0; a < 3; a++)
                            for (int b = 0; b < 3; b++) dC[(3 * al + a) * NSC + 3 * be + b] += s * dF[3 * a + b];
                    }
            }
        if (!any) continue;
        sites[ns++] = y;
        for (int k = 0; k < nin; k++)
            for (int i2 = 0; i2 < NSC; i2++) {
                cplx acc = 0;
                for (int j = 0; j < NSC; j++) acc += dC[i2 * NSC + j] * in[k][(size_t)y * NSC + j];
                out[k][(size_t)y * NSC + i2] += acc;
            }
    }
    return ns;
}

/* sum_k c_k sum_y L_k(y)^dag (dD R_k)(y) for the derivative of D with respect to link (lx, lmu),
 * generator a; work: a zeroed full-lattice vector per pair (left zeroed on return) */
static cplx dD_bilinear(const orc_lat *g, long lx, int lmu, const cplx *T, int npair, cplx *const *L,
                        cplx *const *R, const double *c, cplx *const *work)
{
    long sites[64];
    long xp = neighbour(g, lx, lmu, +1);
    double ph = hop_phase(g, lx, lmu, +1);
    /* hopping: (x, x+mu) entry -1/2 (1 - g) dU, (x+mu, x) entry -1/2 (1 + g) dU^dag */
    cplx dU[9], dUd[9], t[9], ud[9];
    const cplx *u = link(g, lx, lmu);
    m3_mul(T, u, t);
    for (int k = 0; k < 9; k++) dU[k] = I * t[k];
    m3_dag(u, ud);
    m3_mul(ud, T, t);
    for (int k = 0; k < 9; k++) dUd[k] = -I * t[k];
    cplx acc = 0;
    for (int pr = 0; pr < npair; pr++)
        for (int side = 0; side < 2; side++) {
            long row = side ? xp : lx, col = side ? lx : xp;
            const cplx *W = side ? dUd : dU;
            double sg = side ? 1.0 : -1.0; /* (1 + sg g) */
            const cplx *r = R[pr] + (size_t)col * NSC;
            cplx Wr[NSC], o[NSC];
            for (int al = 0; al < 4; al++)
                for (int a = 0; a < 3; a++) {
                    cplx v = 0;
                    for (int b = 0; b < 3; b++) v += W[3 * a + b] * r[3 * al + b];
                    Wr[3 * al + a] = v;
                }
            for (int al = 0; al < 4; al++)
                for (int a = 0; a < 3; a++) {
                    cplx v = Wr[3 * al + a];
                    for (int be = 0; be < 4; be++) v += sg * GAMMA[lmu][al][be] * Wr[3 * be + a];
                    o[3 * al + a] = -0.5 * ph * v;
                }
            const cplx *l = L[pr] + (size_t)row * NSC;
            for (int i = 0; i < NSC; i++) acc += c[pr] * conj(l[i]) * o[i];
        }
    /* clover: dC built once, applied to every pair */
    if (g->csw != 0.0) {
        int ns = apply_dclover(g, lx, lmu, T, npair, R, work, sites);
        for (int pr = 0; pr < npair; pr++)
            for (int k = 0; k < ns; k++) {
                long y = sites[k];
                for (int i = 0; i < NSC; i++) {
                    acc += c[pr] * conj(L[pr][(size_t)y * NSC + i]) * work[pr][(size_t)y * NSC + i];
                    work[pr][(size_t)y * NSC + i] = 0;
                }
            }
    }
    return acc;
}

/*
 * Link and mass derivatives of e = eta^dag (Mh^dag Mh - 1) eta (one noise vector eta on supp P):
 *   de = 2 Re <y, dMh eta> with y = Mh eta;  dMh = A2^-1 (dA1 - dA2 Mh);  z = A2^-dag y;
 *   A_k^-dag = P(1 - D_wb^dag Dcal_bw^dag)P, Dcal_bw^dag y = [(D^dag)^-1 y]_w;
 *   <z, dA v> = -<z, dX v>, X = B^-1 C W^-1 E, expanded by the product rule into
 *   <zt, dD (q - a)> + <wt, dD (a - v)>, a = W^-1 E v, q = B^-1 C a, zt = B^-dag z,
 *   wt = W^-dag C^dag zt (adjoints from D^dag written out; solves by CGNR).
 * dU[(x*4 + mu)*8 + a] = d e / dt for U_mu(x) -> exp(i t lambda_a/2) U_mu(x); *dm2 = d e / d m2.
 */
int orc_force(void *p, double m1, double m2, const double *eta_d, double tol_block, double tol_outer, long maxiter,
              double *e_out, double *dU, double *dm2)
{
    const orc_lat *g = (const orc_lat *)p;
    const cplx *eta = (const cplx *)eta_d;
    long n = g->V * NSC;
    double rel;
    int status = 0;
    cplx *y = (cplx *)calloc(n, sizeof(cplx)), *u = (cplx *)calloc(n, sizeof(cplx));
    cplx *z = (cplx *)calloc(n, sizeof(cplx)), *t = (cplx *)calloc(n, sizeof(cplx));
    cplx *work = (cplx *)calloc(n, sizeof(cplx));
    cplx *Lk[2][2], *Rk[2][2];
    for (int k = 0; k < 2; k++)
        for (int q = 0; q < 2; q++) {
            Lk[k][q] = (cplx *)calloc(n, sizeof(cplx));
            Rk[k][q] = (cplx *)calloc(n, sizeof(cplx));
        }
    if (orc_exponent(p, m1, m2, eta_d, tol_block, tol_outer, maxiter, e_out, NULL, (double *)y, NULL)) status = -1;
    for (long i = 0; i < n; i++) y[i] += eta[i];

    /* z = y - P D_wb^dag u_w,  D(m2)^dag u = (y_b ; 0) */
    if (cgnr_d(g, m2, 1, SEL_ALL, y, u, tol_outer, maxiter, &rel) < 0) status = -1;
    for (long x = 0; x < g->V; x++)
        if (g->colour[x] == 0)
            for (int i = 0; i < NSC; i++) u[(size_t)x * NSC + i] = 0;
    apply_dirac(g, 0.0, 1, SEL_BLACK, SEL_WHITE, u, t);
    for (long i = 0; i < n; i++) z[i] = y[i] - t[i];
    mask_suppP(g, z);

    double masses[2] = {m1, m2};
    const cplx *vk[2] = {eta, y};
    cplx *a = (cplx *)calloc(n, sizeof(cplx)), *q = (cplx *)calloc(n, sizeof(cplx));
    cplx *zt = (cplx *)calloc(n, sizeof(cplx)), *wt = (cplx *)calloc(n, sizeof(cplx));
    double dm2_acc = 0.0;
    for (int k = 0; k < 2; k++) {
        double m = masses[k];
        apply_dirac(g, 0.0, 0, SEL_WHITE, SEL_BLACK, vk[k], t);          /* E v */
        if (cgnr_d(g, m, 0, SEL_WHITE, t, a, tol_block, maxiter, &rel) < 0) status = -1;
        apply_dirac(g, 0.0, 0, SEL_BLACK, SEL_WHITE, a, t);              /* C a */
        if (cgnr_d(g, m, 0, SEL_BLACK, t, q, tol_block, maxiter, &rel) < 0) status = -1;
        if (cgnr_d(g, m, 1, SEL_BLACK, z, zt, tol_block, maxiter, &rel) < 0) status = -1;
        apply_dirac(g, 0.0, 1, SEL_WHITE, SEL_BLACK, zt, t);             /* C^dag zt */
        if (cgnr_d(g, m, 1, SEL_WHITE, t, wt, tol_block, maxiter, &rel) < 0) status = -1;
        for (long i = 0; i < n; i++) {
            Lk[k][0][i] = zt[i];
            Rk[k][0][i] = q[i] - a[i];
            Lk[k][1][i] = wt[i];
            Rk[k][1][i] = a[i] - vk[k][i];
        }
        if (k == 1) dm2_acc = -2.0 * (creal(vdot(n, zt, q)) + creal(vdot(n, wt, a)));
    }
    if (dm2) *dm2 = dm2_acc;
    if (dU) {
        cplx *Lp[4] = {Lk[0][0], Lk[0][1], Lk[1][0], Lk[1][1]};
        cplx *Rp[4] = {Rk[0][0], Rk[0][1], Rk[1][0], Rk[1][1]};
        const double cp[4] = {1.0, 1.0, -1.0, -1.0};
#pragma omp parallel
        {
            cplx *w[4];
            for (int k = 0; k < 4; k++) w[k] = (cplx *)calloc(n, sizeof(cplx));
#pragma omp for schedule(dynamic, 16)
            for (long x = 0; x < g->V; x++)
                for (int mu = 0; mu < 4; mu++)
                    for (int aa = 0; aa < 8; aa++) {
                        cplx T[9];
                        gell_mann_half(aa, T);
                        cplx s = dD_bilinear(g, x, mu, T, 4, Lp, Rp, cp, w);
                        dU[((size_t)x * 4 + mu) * 8 + aa] = 2.0 * creal(s);
                    }
            for (int k = 0; k < 4; k++) free(w[k]);
        }
    }
    free(y); free(u); free(z); free(t); free(work); free(a); free(q); free(zt); free(wt);
    for (int k = 0; k < 2; k++)
        for (int q2 = 0; q2 < 2; q2++) {
            free(Lk[k][q2]);
            free(Rk[k][q2]);
        }
    return status;
}
