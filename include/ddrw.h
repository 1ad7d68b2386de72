/*
 * ddrw.h -- C ABI of the GB300 library for the domain-decomposed stochastic estimate of fermion
 * determinant ratios (Finkenrath, Knechtli, Leder, "Application of Domain Decomposition to the
 * Evaluation of Fermion Determinant Ratios", Lattice 2012).
 *
 * What the library computes (all references are to that paper):
 *
 *   D(m)     the O(a)-improved Wilson-clover Dirac operator (Sec. 1, Sec. 2), in the form
 *            D(m) = (4 + m) + C - 1/2 sum_mu [(1 - g_mu) U_mu(x) T_+mu + (1 + g_mu) U_mu(x-mu)^dag T_-mu],
 *            C = csw (i/4) sum_{mu nu} sigma_{mu nu} Fhat_{mu nu}; the mass enters additively so that
 *            M = D^-1(m2) D(m1) = 1 + dm D^-1(m2) with dm = m1 - m2 (Eq. 2, Eq. 6);
 *   blocks   the lattice is cut into hypercubic blocks of length l, coloured black/white like a
 *            checkerboard (block 0 black); D = [[D_bb, D_bw], [D_wb, D_ww]] (Eq. 1);
 *   Dhat     the Schur complement 1 - D_bb^-1 D_bw D_ww^-1 D_wb, restricted to the support of the
 *            projector P with D_wb P = D_wb (Sec. 1): A(m) = P Dhat(m) P;
 *   estimate 1/det(Mh^dag Mh) ~ (1/N_hit) sum_j exp(-eta_j^dag (Mh^dag Mh - 1) eta_j) with
 *            Mh = A(m2)^-1 A(m1) and complex Gaussian eta_j (Eq. 3, Eq. 8 with N = 1).
 *
 * Conventions at the boundary
 *   - dims = {T, X, Y, Z}; lexicographic site index ((t*X + x)*Y + y)*Z + z.
 *   - gauge field: double U[V][4][3][3][2] (complex, row-major 3x3, mu = t, x, y, z), SU(3) links.
 *   - spinor field: double psi[nrhs][V][4][3][2]; spins in the chiral basis (g5 = diag(1,1,-1,-1),
 *     g0 = [[0,-1],[-1,0]], g_k = [[0,-i s_k],[i s_k,0]] in 2x2 spin blocks).
 *   - packed supp-P vector: double v[nrhs][n_P][4][3][2], the supp-P sites (black sites with a
 *     neighbour in a white block) in ascending lexicographic order; n_P from ddrw_suppP_size().
 *   - Pointers may be host or device memory: the library asks the CUDA runtime which one each
 *     pointer is.  Host buffers are staged through the context's device workspace.
 *   - The caller owns every buffer it passes; the library never frees or keeps them.  The context
 *     owns its internal copies of the gauge field and clover term and its workspaces.
 *   - Every call is stream-ordered on the context's stream and returns when its results are in
 *     the output buffers (the call synchronises the stream before returning).
 *
 * Errors: every call returns a ddrw_status; no call aborts or exits.  A message for the last
 * error of a context is available from ddrw_last_error().  A call that fails leaves its outputs
 * unspecified unless stated otherwise.
 */
#ifndef DDRW_H
#define DDRW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddrw_ctx ddrw_ctx;

typedef enum {
    DDRW_OK = 0,
    DDRW_EINVAL = 1,    /* bad argument: null pointer, bad size, unsupported geometry */
    DDRW_ENOMEM = 2,    /* device allocation failed */
    DDRW_ECUDA = 3,     /* a CUDA call failed (message names it) */
    DDRW_ENOCONV = 4,   /* a solver hit its iteration cap; outputs hold the last iterate */
    DDRW_ENUMERIC = 5,  /* NaN or Inf in a reduction */
    DDRW_EDOMAIN = 6,   /* the estimate is outside its domain of definition */
    DDRW_ESTATE = 7,    /* call out of order (e.g. no gauge field loaded) */
    DDRW_ETIMEOUT = 8   /* a bounded device-side wait ran out (the staged stencil's copies did not
                           land); the call's outputs are invalid, the context stays usable */
} ddrw_status;

typedef enum {
    DDRW_FP64 = 0,       /* every kernel in FP64 */
    DDRW_MIXED_FP32 = 1, /* inner solves in FP32 storage and arithmetic; defect correction on FP64
                            fields with residuals b - D x in double-single arithmetic (ddrw_apply_D_ds) */
    DDRW_MIXED_FP16 = 2, /* inner solves on FP16 storage (per-site FP32 norm for spinors, two-row
                            links, 16-bit clover and inverses) with FP32 arithmetic and reliable
                            updates into FP32 (ddrw_set_low_precision; block solves in FP32 by
                            default); FP64 defect correction as for DDRW_MIXED_FP32 */
    DDRW_MIXED_BF16 = 3  /* as DDRW_MIXED_FP16 with BF16 storage */
} ddrw_prec;

typedef enum { DDRW_BLACK = 0, DDRW_WHITE = 1, DDRW_ALL = 2 } ddrw_colour;

typedef struct {
    int iters_outer;          /* outer Krylov iterations (summed over defect-correction cycles) */
    int iters_inner_total;    /* inner iterations: the in-block iterations of every block-solver
                                 launch (the largest over the blocks of the launch), summed over
                                 launches and defect-correction cycles */
    int cycles;               /* defect-correction cycles (1 for the FP64 path) */
    int fp64_dslash_calls;    /* full-lattice FP64 operator applications */
    int block_iters_max;      /* largest iteration count of any block solve */
    double true_rel_residual; /* max over right-hand sides of ||b - D x|| / ||b||, recomputed in FP64 */
    double seconds;           /* wall time of the call */
} ddrw_solve_info;

/* Create a context on CUDA device `device` for a T x X x Y x Z lattice cut into hypercubic blocks
 * of length block[0] = block[1] = block[2] = block[3] = l (Eq. 1; Sec. 2 uses 6^4 and 8^4 blocks).
 * l must be 2, 4, 6 or 8, divide every dimension, and leave an even number (>= 2) of blocks in
 * each direction, so that neighbouring blocks always have opposite colours; at most 2^27 sites.  cuda_stream is a
 * cudaStream_t (NULL: the context creates its own).  DDRW_EINVAL on a bad geometry. */
ddrw_status ddrw_create(ddrw_ctx **out, const int dims[4], const int block[4], int device, void *cuda_stream);
void ddrw_destroy(ddrw_ctx *ctx);
const char *ddrw_last_error(const ddrw_ctx *ctx);

/* Sites of supp P (black sites with a neighbour in a white block, Sec. 1), and the volume. */
ddrw_status ddrw_suppP_size(ddrw_ctx *ctx, long *n_sites);
ddrw_status ddrw_volume(ddrw_ctx *ctx, long *n_sites);

/* Load the gauge field U[V][4][3][3][2] (host or device); builds the clover term with the csw of
 * the last ddrw_set_params() (csw = 0 before it) and recomputes, in place, the in-block inverses
 * of every mass in use.  The field is copied; the caller keeps U.  A host field goes through a
 * device staging buffer that the context keeps for the next configuration (72 V doubles). */
ddrw_status ddrw_load_gauge(ddrw_ctx *ctx, const double *U);

/* csw (clover coefficient), m1 (ensemble mass) and m2 (target mass) of W(U, m1, m2) (Eq. 2),
 * and the time boundary condition of the quark fields (0 periodic, 1 antiperiodic).  Rebuilds the
 * clover term and the per-mass inverses of the site-diagonal part; the same values again on a
 * built configuration change nothing and return at once. */
ddrw_status ddrw_set_params(ddrw_ctx *ctx, double csw, double m1, double m2, int antiperiodic_t);

/* Solver settings: precision of the inner solves, relative true-residual target of the outer
 * (full-lattice) solve (default 1e-10), relative residual target of the block solves (default
 * 1e-13), and the iteration cap of every solver (default 20000). */
ddrw_status ddrw_set_solver(ddrw_ctx *ctx, ddrw_prec prec, double tol_outer, double tol_block, int maxiter);

/* Krylov method of the full-lattice solves D(m) x = b whose inner solves run on FP32 fields
 * (DDRW_MIXED_FP32): method 0 (the default) is even-odd BiCGStab; method 1 is flexible GCR
 * preconditioned by the Schwarz alternating procedure on the domain decomposition of Sec. 1 --
 * Schwarz blocks of side 4 coloured black/white, ncy cycles over both colours, each block solved
 * approximately by nmr minimal-residual steps on its even-odd reduced operator with Dirichlet
 * boundary conditions, nkv search directions kept between restarts (defaults 4, 4, 8).  Method 1
 * needs every lattice dimension to be a multiple of 8 (else BiCGStab runs); the FP64 path, the
 * 16-bit storage precisions and whole-estimate graphs (ddrw_use_graphs mode 1) always use
 * BiCGStab.  Both reach the same FP64 true residual through the defect correction.
 * DDRW_EINVAL outside method 0..1, ncy 1..16, nmr 1..32, nkv 1..16. */
ddrw_status ddrw_set_outer_solver(ddrw_ctx *ctx, int method, int ncy, int nmr, int nkv);

/* Right-hand sides per chunk of the batched estimates (ddrw_estimate, ddrw_estimate_masses,
 * ddrw_estimate_interp, ddrw_force): max_rhs = 0 (the default) sizes the chunks from the free
 * device memory (about 4 KB per site and right-hand side); max_rhs >= 1 caps them, which leaves
 * memory to the caller or exercises the chunking.  Whole masses go into one chunk while their hits
 * fit, else one mass and as many hits as fit; the results agree with one chunk to the solver
 * tolerances.  DDRW_EINVAL for max_rhs < 0. */
ddrw_status ddrw_set_max_rhs(ddrw_ctx *ctx, int max_rhs);

/* Launch shape of the persistent block solver (Sec. 1: all blocks of a colour in one launch) for
 * blocks of at least 512 sites per parity: form 0 one CTA of 256 threads per block and right-hand
 * side; 1 the same with 512 threads; 2 (FP32 storage, an even number of right-hand sides per mass
 * slot; else 1) one CTA of 512 threads per block and pair of right-hand sides, each link and clover
 * term loaded once for both.  -1 (the default): the first launch of each shape times the candidates
 * on its real arguments and keeps the fastest.  Same results in every form.  DDRW_EINVAL outside -1..2. */
ddrw_status ddrw_block_config(ddrw_ctx *ctx, int form);

/* The 16-bit storage precisions (DDRW_MIXED_FP16, DDRW_MIXED_BF16).  reliable_updates != 0 (the
 * default): the full-lattice inner solves keep the BiCGStab vectors in 16-bit storage with a per-site
 * norm and make reliable updates -- whenever a right-hand side's recursive residual has fallen ten-fold,
 * the 16-bit solution increment is folded into an FP32 solution and the true residual of the even-odd
 * system, recomputed with the FP32 operator, replaces the recursive one -- so that they reach FP32
 * accuracy (relative residual 1e-6 per defect-correction cycle) with 16-bit vector traffic; 0:
 * plain 16-bit inner solves that stop near the 16-bit rounding (1e-3 / 5e-3) and restart at every
 * cycle.  block_solves_16bit != 0: the block solves run on 16-bit storage too; 0 (the default): in
 * FP32 (on 64x32^3 with 8^4 blocks the 16-bit block solves need a second defect-correction cycle and
 * its double-single residual, and the step is 5 % slower).  Whole-estimate graphs (ddrw_use_graphs
 * mode 1) use the plain form. */
ddrw_status ddrw_set_low_precision(ddrw_ctx *ctx, int reliable_updates, int block_solves_16bit);

/* With enable != 0 the FP32 even-odd BiCGStab of the full-lattice solves computes the inner
 * products of alpha = rho / (rh, v) and omega = (t, s) / (t, t) in the epilogue of the stencil launch
 * that writes v and t (one partial per warp of 32 sites, summed in FP64 in a fixed order by a small
 * kernel) instead of re-reading v, t and s in separate reductions; 0 (the default) uses the
 * separate reduction kernels -- on one GB300 the fused launch is 40 % slower than the plain one,
 * which outweighs the reductions it saves.  Results differ only by the rounding of the sums. */
ddrw_status ddrw_fuse_reductions(ddrw_ctx *ctx, int enable);

/* How the block solves D_cc(m)^-1 of the mixed precisions run (Eq. 1; the four solves of r and the
 * block solves of the Schur operator): method 0, the persistent kernel -- one CTA per (block,
 * right-hand side) running the whole in-block even-odd BiCGStab with CTA-wide reductions; method 1,
 * all blocks of the colour as one block-diagonal system in the graph-captured even-odd BiCGStab
 * of the outer solver (tuned stencil launches restricted to the hops inside the blocks, scalars
 * per right-hand side over the colour).  Both feed the same FP64 defect correction to tol_block;
 * the FP64 path and whole-estimate graphs (ddrw_use_graphs mode 1) use method 0.  DDRW_EINVAL
 * for another method. */
ddrw_status ddrw_set_block_solver(ddrw_ctx *ctx, int method);

/* out = M_SAP(m) in: one application of the Schwarz preconditioner of method 1 above (the
 * context's ncy and nmr) to nrhs full-lattice fields, evaluated on FP32 fields and widened to
 * FP64 (layouts as ddrw_apply_D).  With ncy = 1 and enough steps it is one block Gauss-Seidel
 * sweep over the black, then the white Schwarz blocks; for testing the preconditioner. */
ddrw_status ddrw_apply_sap(ddrw_ctx *ctx, double m, const double *in, double *out, int nrhs);

/* out = D(m) in for nrhs full-lattice spinor fields, in FP64. */
ddrw_status ddrw_apply_D(ddrw_ctx *ctx, double m, const double *in, double *out, int nrhs);

/* out = D(m) in evaluated in the double-single arithmetic (FP32 pairs, ~44 significant bits) that
 * the mixed precisions use for their defect-correction residuals b - D x; for checking that
 * arithmetic against ddrw_apply_D. */
ddrw_status ddrw_apply_D_ds(ddrw_ctx *ctx, double m, const double *in, double *out, int nrhs);

/* The operator of Eq. 1 as the inner solves evaluate it: in is rounded to the storage precision
 * prec (DDRW_MIXED_FP32: FP32 fields; DDRW_MIXED_FP16 / DDRW_MIXED_BF16: 16-bit fields with a
 * per-site scale), one stencil launch in that storage with FP32 arithmetic (the tuned or pinned
 * launch form, see ddrw_stencil_config) computes D(m) in, or A(m)^-1 D(m) in (the site-diagonal
 * inverse applied to the result) when post != 0, and the result is widened to FP64 into out.
 * Layouts as ddrw_apply_D (host or device buffers).  DDRW_EINVAL for another prec. */
ddrw_status ddrw_apply_D_low(ddrw_ctx *ctx, ddrw_prec prec, double m, int post, const double *in, double *out,
                             int nrhs);

/* out = D_{rows,cols}(m) in: the block of Eq. 1 with rows in colour `rows` and columns in colour
 * `cols` (DDRW_BLACK, DDRW_WHITE or DDRW_ALL); rows outside `rows` are set to zero.  D_bb and
 * D_ww are the block-diagonal block operators, D_bw and D_wb the hops between blocks. */
ddrw_status ddrw_apply_block(ddrw_ctx *ctx, int rows, int cols, double m, const double *in, double *out, int nrhs);

/* x = D_cc(m)^-1 b for colour c = DDRW_BLACK or DDRW_WHITE: all blocks of the colour are solved
 * in one persistent kernel, each block to relative residual tol_block.  b and x are full-lattice
 * fields; only the sites of colour c are read and written (x is zero elsewhere). */
ddrw_status ddrw_solve_block(ddrw_ctx *ctx, int colour, double m, const double *b, double *x, int nrhs,
                             ddrw_solve_info *info);

/* x = D(m)^-1 b for full-lattice fields, to the outer tolerance. */
ddrw_status ddrw_solve_D(ddrw_ctx *ctx, double m, const double *b, double *x, int nrhs, ddrw_solve_info *info);

/* out = A(m) in with A(m) = P Dhat(m) P (Sec. 1), on packed supp-P vectors; with dagger != 0
 * out = A(m)^dag in = in - P g5 D_bw D_ww^-1 D_wb D_bb^-1 g5 in, from D^dag = g5 D g5 applied to the
 * blocks of Eq. 1 ((D_XY)^dag = g5 D_YX g5).  Block solves to tol_block in the context's precision. */
ddrw_status ddrw_apply_schur(ddrw_ctx *ctx, double m, int dagger, const double *in, double *out, int nrhs);

/* r = (A(m1) - A(m2)) eta on packed supp-P vectors, in the resolvent form
 * r = dm P D_bb(m1)^-1 [D_bw a12 + D_bb(m2)^-1 D_bw a2], u = D_wb eta, a2 = D_ww(m2)^-1 u,
 * a12 = D_ww(m1)^-1 a2 (no cancellation between the two masses). */
ddrw_status ddrw_apply_dA(ddrw_ctx *ctx, const double *eta, double *r, int nrhs, ddrw_solve_info *info);

/* x = A(m)^-1 b on packed supp-P vectors: one full-lattice solve D(m) y = (0_b ; D_wb b) and
 * x = b - P y_b, from Dhat^-1 = 1 - P Dcal_bw D_wb (Sec. 1). */
ddrw_status ddrw_solve_schur(ddrw_ctx *ctx, double m, const double *b, double *x, int nrhs, ddrw_solve_info *info);

/* nhit packed complex Gaussian noise vectors with E|eta_k|^2 = 1 (Eq. 3): component k of hit h
 * from Philox4x32-10 with counter (k, hit_offset + h, 0, 0) and key (seed mod 2^32, seed >> 32),
 * u1 = (w0 + 1) 2^-32, u2 = w1 2^-32, eta_k = sqrt(-ln u1) exp(2 pi i u2). */
ddrw_status ddrw_noise(ddrw_ctx *ctx, uint64_t seed, uint64_t hit_offset, int nhit, double *eta);

/* The stochastic estimate of Eq. 3 / Eq. 8 (N = 1) for the Schur complement: for each of nhit
 * noise vectors (from ddrw_noise(seed, hit_offset) when eta == NULL, else the caller's packed
 * vectors) exponents[j] = eta_j^dag (Mh^dag Mh - 1) eta_j = ||delta_j||^2 + 2 Re <eta_j, delta_j>
 * with delta_j = A(m2)^-1 (A(m1) - A(m2)) eta_j.  *logW = log((1/nhit) sum_j exp(-e_j)) (FP64
 * log-sum-exp) and *rel_var = sample variance of exp(-e_j) / W^2 (both optional).  delta (optional,
 * packed) receives the delta_j.  DDRW_ENOCONV if a solve missed its tolerance (outputs filled). */
ddrw_status ddrw_estimate(ddrw_ctx *ctx, int nhit, uint64_t seed, uint64_t hit_offset, const double *eta,
                          double *exponents, double *logW, double *rel_var, double *delta, ddrw_solve_info *info);

/* The global factor of Eq. 8 (mass interpolation, N steps, nhit noise vectors per factor) for the
 * operators Fig. 1 compares (Sec. 2): variant 0 the total operator, Mh_i = D(m_i)^-1 D(m_{i-1}) on
 * all 12 V components; variant 1 the even-odd Schur complement S = A_ee - D_eo A_oo^-1 D_oe (the
 * block Schur complement for blocks of one site), Mh_i = S(m_i)^-1 S(m_{i-1}) on the 6 V
 * components of the even sites; variant 2 the block Schur complement of this context (as
 * ddrw_estimate_interp).  m_i = (i/N) m2 + ((N-i)/N) m1.  exponents[N][nhit] (optional) =
 * eta^dag (Mh_i^dag Mh_i - 1) eta, *logW (optional) = sum_i log((1/nhit) sum_j exp(-e_ij)),
 * rel_var[N] (optional) = per-factor sample variance of exp(-e_ij) over its squared mean, *dim
 * (optional) = the dimension of the support (12 V, 6 V or 12 dim P).  Noise: eta (variants 0 and
 * 1 only; packed [N][nhit][dim] complex, sites of the support in lexicographic order, 12
 * components each) or Philox (seed, hit hit_offset + i nhit + j, component index in that packed
 * order).  1 <= N <= 8. */
ddrw_status ddrw_estimate_variant(ddrw_ctx *ctx, int variant, int N, int nhit, uint64_t seed, uint64_t hit_offset,
                                  const double *eta, double *exponents, double *logW, double *rel_var, long *dim,
                                  ddrw_solve_info *info);

/* The estimate for several target masses in one batched call (the mass sweep of a reweighting
 * study): right-hand side k * nhit + j carries m2[k] and noise vector j (the same noise vectors for
 * every mass), all in one multi-right-hand-side pass.  exponents[nmass * nhit], logW[nmass] and
 * rel_var[nmass] as in ddrw_estimate (each optional).  1 <= nmass <= 8; m1 from ddrw_set_params. */
ddrw_status ddrw_estimate_masses(ddrw_ctx *ctx, int nmass, const double *m2, int nhit, uint64_t seed,
                                 uint64_t hit_offset, double *exponents, double *logW, double *rel_var,
                                 ddrw_solve_info *info);

/* Mass interpolation (Eq. 8) with the one-flavour estimator (Eq. 11) and the root trick.
 * m_i = (i/N) m2 + ((N-i)/N) m1 for i = 0..N; factor i uses Mh_i = A(m_i)^-1 A(m_{i-1}) and its own
 * noise vectors eta_{i,j} (Philox hits hit_offset + (i-1) nhit + j).  All N factors run as mass
 * slots of one batched pass when they fit the device memory.  Outputs (each optional):
 *   exponents[N][nhit]       e_ij = eta^dag (Mh_i^dag Mh_i - 1) eta            (two flavours, Eq. 8)
 *   exponents_1f[N][nhit][2] eta^dag (Mh_i - 1) eta = <eta, delta>, complex  (one flavour, Eq. 11)
 *   logW[4]                  log W_gl = sum_i log((1/N_hit) sum_j exp(-e_ij)); log |W_1f| with
 *                            W_1f = prod_i Re((1/N_hit) sum_j exp(-e1_ij)); sign of W_1f; and the
 *                            root trick log sqrt(W_gl) = logW[0] / 2
 *   logW_factors[N], rel_var[N]  per factor: log of its two-flavour estimate, sample variance / mean^2.
 *   rel_var_1f[N]            per factor: the sample variance of the complex one-flavour estimator
 *                            exp(-e1_ij), E|X|^2 - |E X|^2 (what Eq. 12 gives exactly), over |mean|^2.
 * 1 <= N <= 8. */
ddrw_status ddrw_estimate_interp(ddrw_ctx *ctx, int N, int nhit, uint64_t seed, uint64_t hit_offset, double *exponents,
                                 double *exponents_1f, double *logW, double *logW_factors, double *rel_var,
                                 double *rel_var_1f, ddrw_solve_info *info);

/* The adjoint of the estimate: for each of nhit noise vectors (as in ddrw_estimate) the exponent
 * e_j, its derivative with respect to every link and with respect to m2 (m1 fixed), by reverse
 * mode through the Schur complement (recomputing the solutions, not storing Krylov iterates):
 *   dU[x][mu][a] = sum_j w_j d e_j / dt,  U_mu(x) -> exp(i t lambda_a/2) U_mu(x)  (left multiplication,
 *                  Gell-Mann matrices lambda_a, a = 1..8 stored 0..7; x lexicographic),
 *   dm2[j]       = d e_j / d m2.
 * weights w_j (null: all 1); eta packed or null (Philox noise of seed, hit_offset); exponents[nhit],
 * dU[V][4][8] (host or device) and dm2[nhit] are each optional.  Solves run in the context's
 * precision; the force kernels in FP64. */
ddrw_status ddrw_force(ddrw_ctx *ctx, int nhit, uint64_t seed, uint64_t hit_offset, const double *eta,
                       const double *weights, double *exponents, double *dU, double *dm2, ddrw_solve_info *info);

/* ddrw_solve_block for callers that cannot allocate device memory.  The paper has no counterpart:
 * this is an integration aid.  Some callers may not call cudaMalloc -- code running while a
 * framework's memory pool is frozen, or a host application that owns every device allocation and
 * forbids libraries their own -- and ddrw_solve_block grows its workspace with cudaMalloc.  This
 * call allocates nothing: its scratch (about 40 MB: ten FP64 fields of up to 20736 sites plus
 * reduction slots) is one fixed array in device memory that every GPU using the library holds
 * until the process exits.
 *   - One right-hand side, FP64 (whatever ddrw_set_solver chose), tolerance tol_block, same
 *     result as ddrw_solve_block: x = D_cc(m)^-1 b on colour c, x zero on the other colour.
 *   - Lattices of at most 20736 sites (12^4); larger ones return DDRW_EINVAL with a message.
 *   - b and x must be device pointers (boundary layout); host pointers return DDRW_EINVAL.
 *   - m must be m1 or m2 of the last ddrw_set_params (their inverses already exist); other
 *     masses return DDRW_EINVAL.  A non-finite b returns DDRW_ENUMERIC.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress) with the context's
 *     device current.  The call synchronises its stream and reads scalars back to the host, so it
 *     must not be made while the context's stream is being captured: it then returns DDRW_ESTATE.
 *   - All calls share the array and it keeps the last call's contents; calls that overlap on the
 *     GPU (other streams or contexts on the same device) race on it, so serialise them.
 *   - With kernel timing (ddrw_profile) on, the timing events are created on first use. */
ddrw_status ddrw_solve_block_noalloc(ddrw_ctx *ctx, int colour, double m, const double *b, double *x,
                                     ddrw_solve_info *info);

/* CUDA graphs (default mode 2).  Mode 2: the outer Krylov loop, after its first iterations, runs as
 * one graph with a conditional while-node (device-side convergence test, iteration cap); the
 * defect-correction cycles around it are host-driven.  Mode 1: the same, and in addition an
 * estimate chunk with library-drawn noise is, from the second call with the same lattice, solver
 * settings, masses and number of hits, captured whole into one graph and replayed: noise, block
 * solves, outer solves and their defect-correction cycles, whose continue decisions and inner
 * tolerances are taken by condition kernels on the device (nested conditional while-nodes, every
 * loop capped); measured on one GB300 it is as fast as mode 2 on 16^4 and 32x16^3 and 0.6 % slower
 * on 64x32^3.  Mode 0: no graphs.  -1 leaves the setting; *graph_launches (optional) receives the
 * number of graph launches so far.  Results are bitwise the same in every mode.  Block solves are
 * single persistent launches. */
ddrw_status ddrw_use_graphs(ddrw_ctx *ctx, int enable, long *graph_launches);

/* Autotuner of the stencil launches: on the first launch of each shape (precision, block length,
 * parities, right-hand sides, diagonal/post modes) it times right-hand sides per thread {1,2,4},
 * sites per CTA row {64,128,256}, right-hand-side rows per CTA {1,2} and the hop code form
 * (unrolled, rolled, batched loads, register caps, neighbour table) with CUDA events and keeps the fastest.  Tuned choices are
 * also kept for the process, by device and lattice geometry, and reused by later contexts of the
 * same geometry.  enable = 0 uses a fixed choice; either call clears the tuned tables of the context
 * and of the process.  The report lists the tuned shapes, one per line, and the launch shapes the
 * persistent block solver chose (ddrw_block_config). */
ddrw_status ddrw_autotune(ddrw_ctx *ctx, int enable);
ddrw_status ddrw_autotune_report(ddrw_ctx *ctx, char *buf, long len);

/* Pins the configuration of every tunable stencil launch (overrides the autotuner): nr
 * right-hand sides per thread (1, 2 or 4), nt sites per CTA row (32 .. 256, a multiple of 32),
 * nw right-hand-side rows per CTA (nt * nw <= 256), roll 0 / 1 (unrolled / rolled hop code),
 * 2 / 3 (the loads of 4 / 8 hops issued ahead of their arithmetic), 4 / 5 (unrolled with at
 * most 85 / 128 registers per thread), 6 / 7 (as 5 / 4, with the neighbour indices read from a
 * table built at ddrw_create, 32 bytes per site, instead of computed from the block-major site
 * order) or 8 (staged, FP32 storage only: a CTA of nt sites x nw rows covers every right-hand side
 * of one mass slot; the tile's links, A^-1 / clover terms and neighbour entries are brought into
 * shared memory once by bulk asynchronous copies and shared by those right-hand sides; nt <= 128;
 * other storage precisions run form 5 instead), 9 / 10 (pipelined, FP32 storage only: each thread
 * copies the neighbour spinor and link of its hops into a two-slot shared-memory ring with 16-byte
 * asynchronous copies two hops ahead of the arithmetic; at least 2 / 3 CTAs per SM; other
 * precisions run form 5) or 11 (fully rolled: one body for the eight hops, the direction and
 * the signs chosen at run time; used by the double-single residual stencil, which is limited by
 * instruction fetch, and as form 0 elsewhere); roll 2-4 and 7-11 need nr = 1, roll 5 and 6
 * nr <= 2.  The double-single stencil runs forms 0, 1 and 11, with nr = nw = 1.
 * A launch whose right-hand sides per mass slot are not a multiple of nr * nw runs with nr = nw = 1.
 * nr = 0 returns to autotuning.  DDRW_EINVAL for values outside these ranges.  A change drops the
 * captured CUDA graphs (they are captured again with the new form on next use). */
ddrw_status ddrw_stencil_config(ddrw_ctx *ctx, int nr, int nt, int nw, int roll);

/* Test switch of the staged stencil's bounded wait (form 8): with enable != 0 every staged launch
 * announces 16 bytes more than its copies deliver, so its shared-memory barrier never completes;
 * each CTA stops polling after a bounded number of tries, sets the context's device error flag and
 * returns, and the call that launched it returns DDRW_ETIMEOUT at its next synchronisation.
 * enable = 0 restores normal operation; the context remains usable either way. */
ddrw_status ddrw_test_stall_staging(ddrw_ctx *ctx, int enable);

/* The exact block factor of Eq. 7: W = W_gl prod_k det D_k^2(m2) / det D_k^2(m1), k over the black
 * and the white blocks, D_k the block Dirac operators on the diagonal of D_bb and D_ww (Eq. 1).
 * ddrw_block_logdet writes log |det D_k(m)| and the sign of det D_k(m) (real by g5-hermiticity)
 * for every block, in the library's block numbering: black blocks first, then white, each in
 * lexicographic order of the block coordinates (t slowest); logdet and sign hold nblk = V / l^4
 * doubles, host or device (sign may be null).  ddrw_block_factor writes
 * log prod_k det D_k^2(m2) / det D_k^2(m1) for the m1, m2 of ddrw_set_params (two flavours).
 * Method: det D_k = det A_oo det S_k with S_k = A_ee - D_eo A_oo^-1 D_oe the block's even-odd
 * Schur complement (dimension 6 l^4), assembled by the FP64 block stencil and factorised by a
 * batched LU with partial pivoting in FP64 (one CTA per block).  The paper calls the exact block
 * determinants feasible for l^4 <= 6^4; l > 6 returns DDRW_EINVAL, and blocks are processed in
 * batches that fit 60 % of the free device memory (DDRW_ENOMEM if one matrix does not fit).
 * Cost: (6 l^4)^3 / 3 complex FP64 multiply-adds per block and mass, one SM per block: 16^4
 * with l = 4 takes about 9 s for both masses (256 blocks), 12^4 with l = 6 about 4 minutes per
 * mass (16 blocks, 16 SMs busy). */
ddrw_status ddrw_block_logdet(ddrw_ctx *ctx, double m, double *logdet, double *sign);
ddrw_status ddrw_block_factor(ddrw_ctx *ctx, double *log_w_blk);

/* The block factor of Eq. 7 for blocks too large for a dense determinant (8^4), by the nested
 * decomposition of Sec. 2.2 (caption of Fig. 2: the 8^4 blocks are decomposed further into an 8^4
 * Schur complement with Dirichlet boundaries and 4^4 blocks).  Each block operator D_k is cut into
 * sub-blocks of length lsub, coloured black/white inside the block:
 *     det D_k = det Shat_k * prod_{sub in k} det D_sub     (Sec. 1, applied to D_k),
 * so  log prod_k det D_k^2(m2)/det D_k^2(m1) = [sub-block factor, exact, as ddrw_block_factor on
 * blocks of length lsub] + [log prod_k det Shat_k^2(m2)/det Shat_k^2(m1), estimated with Eq. 3 from
 * nhit Philox noise vectors (seed, hits 0 .. nhit-1) on the supp P of the sub-blocks].  out[0] the
 * sum, out[1] the exact part, out[2] the stochastic part; exponents[nhit] and rel_var (each
 * optional) as in ddrw_estimate.  The work runs on an auxiliary context of the same lattice and
 * field with blocks of length lsub and the hops across the faces of this context's blocks removed
 * (the clover term kept): about the memory of a second context.  lsub in {2, 4, 6} with
 * l / lsub even; precision and tolerances of ddrw_set_solver. */
ddrw_status ddrw_block_factor_nested(ddrw_ctx *ctx, int lsub, int nhit, uint64_t seed, double *out, double *exponents,
                                     double *rel_var);

/* Dirichlet boxes: with cut > 0 (a multiple of the block length dividing every dimension) the hops
 * across the faces of the cut^4 boxes (U_mu(x) with x_mu = cut - 1 mod cut) are removed from the
 * operator after the clover term has been built from the full field, so that D is the direct sum of
 * the boxes' Dirichlet operators D_k of Eq. 7.  Must precede ddrw_load_gauge (DDRW_ESTATE after);
 * 0 (the default) keeps every hop.  Used by ddrw_block_factor_nested; the full field's links are
 * kept on the device for rebuilding the clover term. */
ddrw_status ddrw_set_dirichlet(ddrw_ctx *ctx, int cut);

/* Kernel timing for measurement (not part of the method): with profiling enabled, CUDA events
 * bracket every launch of the instrumented kernel classes on the context's stream, and
 * ddrw_profile_read returns, per class, the number of launches, their summed device time (ms) and
 * their summed compulsory bytes (each field counted once per launch: spinors per right-hand
 * side, links and clover terms once).  Classes: 0 FP64 stencil, 1 FP32 stencil (all hops),
 * 2 / 3 FP64 / FP32 stencil restricted to hops inside or between blocks, 4 / 5 FP64 / FP32
 * persistent block solver (bytes not counted), 6 Krylov vector kernels and reductions (bytes not
 * counted), 7 double-single residual stencil, 8 and 9 the stencil on 16-bit storage (all hops /
 * block-restricted), 10 the persistent block solver on 16-bit storage (bytes not counted), 11 the
 * Schwarz-preconditioner sweeps of the GCR outer solver (bytes not counted); class 12 returns in
 * *launches the number of kernel launches of every kind since the last reset.  ddrw_profile(ctx, enable) resets the counters. */
ddrw_status ddrw_profile(ddrw_ctx *ctx, int enable);
ddrw_status ddrw_profile_read(ddrw_ctx *ctx, int kind, long *launches, double *ms, double *bytes);

/* Site updates (output sites x right-hand sides) summed over the timed launches of a stencil
 * class (0-3, 7-9) since the last ddrw_profile call; other classes report 0. */
ddrw_status ddrw_profile_units(ddrw_ctx *ctx, int kind, double *site_updates);

#ifdef __cplusplus
}
#endif
#endif /* DDRW_H */
