// ctx.h -- the library context (host side) and helpers shared by the .cu files.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "../../include/ddrw.h"
#include "ddrw_internal.cuh"

namespace ddrw {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Per-mass inverse of the site-diagonal part A(m) = (4 + m) + C, in every storage precision.
struct MassInv {
    double m;
    double2 *A64 = nullptr;  // [2][18][V]
    float4 *A32 = nullptr;   // [2][9][V]
    uint2 *A16 = nullptr;    // [2][9][V] FP16
    uint2 *Ab16 = nullptr;   // [2][9][V] BF16
};

// the in-block inverse of mass slot m in the storage of policy id (64, 32, 16 = FP16, 17 = BF16)
inline const void *ainv_for(const MassInv *m, int id)
{
    return id == 64 ? (const void *)m->A64 : id == 32 ? (const void *)m->A32 : id == 16 ? (const void *)m->A16
                                                                                     : (const void *)m->Ab16;
}

// an instantiated Krylov-loop graph (solver.cu)
struct GraphEntry {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

// Device-side record of a graph-captured estimate: written by the loops' control kernels, read by
// the host after the replay (estimate.cu, blocksolve.cu, solver.cu).
constexpr int DC_LOOPS = 32;
struct DcStats {
    int block_iters_max, block_cycles, outer_iters, outer_cycles;
    long block_iters_total;
    int fp64_dslash_half, fp64_dslash_full;
    int nan, noconv;
    double block_rel_residual, outer_rel_residual;
    int loop_iters[DC_LOOPS];  // executions of each captured loop body (launch accounting)
};

// a captured whole-estimate graph
struct EstGraph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    long top_launches;                              // kernel launches outside the loops
    std::vector<std::pair<int, long>> loop_launches;  // (loop slot, launches per body execution)
};

// a tuned stencil launch configuration
struct TuneEntry {
    int nr, nt, nw, roll;  // right-hand sides per thread, sites per CTA row, right-hand-side groups
                           // per CTA, rolled hop bodies
    float ms;
};

// A set of masses, one per right-hand-side slot (rhs r uses slot r / ceil(nrhs / n)).
struct MassSet {
    int n = 1;
    double m[MAXM] = {0.0};
    MassInv *inv[MAXM] = {nullptr};
};

// Work counters of a solve, summed over its phases.
struct SolveStats {
    int block_iters_max = 0;     // largest in-kernel iteration count of any block solve
    int block_cycles = 0;        // block defect-correction cycles
    long block_iters_total = 0;  // in-kernel iterations summed over block-solver launches (max over blocks each)
    double block_rel_residual = 0;
    int fp64_dslash_half = 0;    // FP64 stencil sweeps over half the lattice (one colour)
    int outer_iters = 0;         // outer Krylov iterations, summed over cycles
    int outer_cycles = 0;        // outer defect-correction cycles
    int fp64_dslash_full = 0;    // FP64 full-lattice operator applications
    double outer_rel_residual = 0;
};

}  // namespace ddrw

struct ddrw_ctx {
    // geometry
    int dims[4];
    int l;
    int NB[4];
    long V, vh;
    int nblk, nblk_c;
    int *d_blk_nb = nullptr, *d_blk_org = nullptr, *d_blk_index = nullptr;
    int4 *d_nbr = nullptr;  // neighbour table of the stencil's table forms, [2][V]
    float4 *Ubw32 = nullptr;  // [12][V]: FP32 two-row U_mu(x - mu) stored at x (staged stencil)
    int *h_err = nullptr, *d_err = nullptr;  // device error flags, host-mapped (bit 0: staging wait ran out)
    int stall_tx = 0;                        // test switch of the staged stencil (extra announced bytes)
    long nP = 0;
    int *d_suppP = nullptr;  // internal site index of the k-th supp-P site (lexicographic order)

    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    // parameters
    double csw = 0.0, m1 = 0.0, m2 = 0.0;
    int antiperiodic = 0;
    bool have_gauge = false;
    bool built = false;  // clover term and in-block inverses match the gauge field and the parameters
    ddrw_prec prec = DDRW_FP64;
    double tol_outer = 1e-10, tol_block = 1e-13;
    int maxiter = 20000;
    int max_rhs = 0;  // right-hand sides per chunk of a batched estimate (0: from free memory)
    // outer Krylov method of the mixed-precision full-lattice solves: 0 even-odd BiCGStab, 1 flexible
    // GCR preconditioned by the Schwarz alternating procedure (sap.cu); its cycles, minimal-residual
    // steps per block and kept search directions, and the iterations of the last inner solve
    int outer_method = 0;
    int sap_ncy = 4, sap_nmr = 4, sap_nkv = 8;
    int sap_last_iters = 0;
    // block solves of the mixed precisions: 0 the persistent kernel (one CTA per block and right-hand
    // side), 1 the Krylov-loop BiCGStab on the colour's blocks as one block-diagonal system
    int block_method = 0;
    // the BiCGStab inner products of alpha and omega fused into the epilogue of the stencil launch
    // that writes v and t (FP32 storage, full lattice); off (the default, measured faster on
    // GB300): separate reduction kernels
    bool fuse_dots = false;
    // 16-bit storage precisions: the full-lattice inner solves keep their Krylov vectors in 16-bit
    // storage with reliable updates into FP32 (true), or restart at each defect-correction cycle;
    // the block solves run on 16-bit storage (true) or in FP32
    bool reliable16 = true;
    bool block16 = false;

    // Dirichlet cut (ddrw_set_dirichlet): hops across the faces of cut^4 boxes removed from the
    // hopping term after the clover term is built from the full field, whose links stay in U64f / U32f
    int cut = 0;
    double2 *U64f = nullptr;
    float4 *U32f = nullptr;

    // resident fields
    double2 *U64 = nullptr;  // [4][9][V]
    float4 *U32 = nullptr;   // [4][3][V] two-row
    double2 *C64 = nullptr;  // [2][18][V]
    float4 *C32 = nullptr;   // [2][9][V]
    uint2 *U16 = nullptr;    // [4][3][V] two-row FP16
    uint2 *Ub16 = nullptr;   // [4][3][V] two-row BF16
    uint2 *C16 = nullptr;    // [2][9][V] FP16
    uint2 *Cb16 = nullptr;   // [2][9][V] BF16
    float4 *Udd = nullptr;   // [4][9][V] links split into FP32 pairs (double-single stencil)
    float4 *Cdd = nullptr;   // [2][18][V] clover split into FP32 pairs
    std::deque<ddrw::MassInv> inv;  // deque: MassInv addresses stay valid as entries are added

    // workspaces by name (grow-only)
    std::map<std::string, ddrw::DevBuf> ws;
    double *h_pinned = nullptr;  // small pinned host buffer for scalars
    size_t h_pinned_bytes = 0;

    // CUDA graphs of the outer Krylov loop, by launch shape and buffers
    bool use_graphs = true;       // Krylov-loop graphs
    bool use_est_graphs = false;  // whole estimate chunks as one graph (mode 1; needs use_graphs)
    // reliable updates are on and not excluded by the whole-estimate graphs, whose captured solvers
    // (and, for equal results, the eager calls of that mode) use the plain 16-bit form
    bool reliable_updates() const { return reliable16 && !(use_graphs && use_est_graphs); }
    long graph_launches = 0;
    std::map<std::array<uintptr_t, 13 + 2 * ddrw::MAXM>, ddrw::GraphEntry> graphs;
    // whole-estimate graphs (estimate.cu): captured on the second call of a shape, replayed after
    std::map<std::array<uintptr_t, 24>, ddrw::EstGraph> est_graphs;
    std::map<std::array<uintptr_t, 24>, int> est_seen;
    // device-side loop control while an estimate is captured
    bool devctl = false;                  // capturing: solvers use their device-controlled forms
    ddrw::DcStats *dc = nullptr;          // device record of the capture being built / replayed
    cudaStream_t cap_streams[4] = {};     // side streams that capture nested loop bodies
    int cap_depth = 0, dc_loops = 0;
    long cap_nested[5] = {0};             // launches of nested bodies, per capture depth
    std::vector<std::pair<int, long>> cap_loop_launches;

    // stencil autotuner (dslash_tune.cu); pinned_nr > 0 overrides it with the pinned configuration
    bool autotune = true;
    int pinned_nr = 0, pinned_nt = 128, pinned_nw = 1, pinned_roll = 0;
    std::map<std::array<int, 8>, ddrw::TuneEntry> tune;
    std::map<std::array<int, 3>, int> blk_tune;  // block-solver launch shape (blocksolve.cuh)
    int blk_form = -1;                             // pinned block-solver launch shape, -1: tuned

    // kernel timing (ddrw_profile): CUDA events around the instrumented launches
    bool prof_on = false;
    long launches = 0;  // kernel launches since creation or the last ddrw_profile call
    struct ProfRec {
        cudaEvent_t a, b;
        int kind;
        double bytes, units;
    };
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    long prof_count[16] = {0};
    double prof_ms[16] = {0}, prof_bytes[16] = {0}, prof_units[16] = {0};

    std::string err;
};

namespace ddrw {

// kernel classes timed by ddrw_profile (see include/ddrw.h)
enum {
    PROF_DSLASH64 = 0,      // FP64 stencil, all hops
    PROF_DSLASH32 = 1,      // FP32 stencil, all hops
    PROF_DSLASH64_BLK = 2,  // FP64 stencil, hops inside / between blocks
    PROF_DSLASH32_BLK = 3,
    PROF_BLOCK64 = 4,       // persistent block solver, FP64
    PROF_BLOCK32 = 5,       // persistent block solver, FP32
    PROF_BLAS = 6,          // Krylov vector kernels and reductions
    PROF_DSLASH_DS = 7,     // double-single residual stencil (mixed path)
    PROF_DSLASH16 = 8,      // 16-bit storage (FP16 or BF16) stencil, all hops
    PROF_DSLASH16_BLK = 9,  // 16-bit storage stencil, block-restricted hops
    PROF_BLOCK16 = 10,      // persistent block solver on 16-bit storage
    PROF_SAP = 11,          // Schwarz preconditioner sweeps (SAP-GCR outer solver)
    PROF_NKIND = 12
};

// Records CUDA events around the launches in its scope when profiling is on.
struct ProfScope {
    ddrw_ctx *ctx;
    int kind;
    double bytes, units;  // algorithmic bytes and site updates (sites x right-hand sides) of the launch
    cudaEvent_t a = nullptr;
    ProfScope(ddrw_ctx *c, int k, double b, double u = 0.0);
    ~ProfScope();
};

ddrw_status set_error(ddrw_ctx *ctx, ddrw_status st, const std::string &msg);
ddrw_status set_cuda_error(ddrw_ctx *ctx, cudaError_t e, const char *what, const char *file, int line);

// destroy the captured Krylov-loop and estimate graphs (before any buffer they reference is freed
// or moved)
void clear_graphs(ddrw_ctx *ctx);

// While the estimate is being captured on ctx->stream: appends a while-loop node whose body is
// captured from body(handle, slot) with ctx->stream switched to a capturing side stream.  The body
// must end with a kernel that sets the loop's condition handle (cudaGraphSetConditional) and
// counts its executions in dc->loop_iters[slot]; the helper checks, before anything runs, that the
// captured body contains the kernel cond_fn.
ddrw_status capture_while(ddrw_ctx *ctx, const void *cond_fn,
                          const std::function<ddrw_status(cudaGraphConditionalHandle, int)> &body);

// device workspace of at least `bytes`, reused across calls under `name`
ddrw_status workspace(ddrw_ctx *ctx, const char *name, size_t bytes, void **out);
// frees a workspace (after the stream has drained); for large one-off buffers
void release_workspace(ddrw_ctx *ctx, const char *name);

GeomDev geom_dev(const ddrw_ctx *ctx);
void build_nbr_table(ddrw_ctx *ctx);
void build_bw_links(ddrw_ctx *ctx);

// mass-dependent inverse of A(m), built on first use
ddrw_status mass_inverse(ddrw_ctx *ctx, double m, MassInv **out);

// host/device staging of caller buffers (see the pointer rules of include/ddrw.h)
bool is_device_ptr(const void *p);
ddrw_status stage_in(ddrw_ctx *ctx, const void *user, size_t bytes, const char *name, const void **dev);
ddrw_status stage_out(ddrw_ctx *ctx, void *user, size_t bytes, const char *name, void **dev, bool *host);
ddrw_status finish_out(ddrw_ctx *ctx, void *user, const void *dev, size_t bytes, bool host);
ddrw_status sync(ddrw_ctx *ctx);
// synchronises the stream and reports CUDA errors and the device error flags as the caller's status
#define DDRW_SYNC(ctx)                       \
    do {                                     \
        ddrw_status s__ = sync(ctx);         \
        if (s__ != DDRW_OK) return s__;      \
    } while (0)
void zero_colour64(ddrw_ctx *ctx, double2 *f, int colour, int nrhs);

// ---- launchers (all on ctx->stream)
// Full-lattice FP64 fields: element (rhs r, plane k, site s) at f[r * 12 V + k * V + s].
void pack_spinor64(ddrw_ctx *ctx, const double *user, double2 *f, int nrhs);
void unpack_spinor64(ddrw_ctx *ctx, const double2 *f, double *user, int nrhs);
void pack_P64(ddrw_ctx *ctx, const double2 *f, double *packed, int nrhs);
void unpack_P64(ddrw_ctx *ctx, const double *packed, double2 *f, int nrhs);  // zero outside supp P

// links and clover term in the storage of policy id (128 = double-single split, 64, 32, 16 = FP16,
// 17 = BF16)
inline const void *links_for(const ddrw_ctx *ctx, int id)
{
    switch (id) {
    case 128: return ctx->Udd;
    case 64: return ctx->U64;
    case 32: return ctx->U32;
    case 16: return ctx->U16;
    default: return ctx->Ub16;
    }
}
inline const void *clover_for(const ddrw_ctx *ctx, int id)
{
    switch (id) {
    case 128: return ctx->Cdd;
    case 64: return ctx->C64;
    case 32: return ctx->C32;
    case 16: return ctx->C16;
    default: return ctx->Cb16;
    }
}

void pack_gauge(ddrw_ctx *ctx, const double *Ulex);  // fills U64 and U32
void cut_links(ddrw_ctx *ctx);                       // zeroes U64 / U32 links across the cut faces
void build_clover(ddrw_ctx *ctx);                    // fills C64 and C32 from U64
void build_inverse(ddrw_ctx *ctx, double m, MassInv &mi);

// Hopping + clover kernel (K4/K5), policy-generic:
//   out = POST( alpha * DIAG(x) + beta * sum_mu [hops of `in` selected by hopsel] )
//   DIAG: 0 none, 1 A(m) x, 2 x;  POST: 0 none, 1 A(m)^-1 (per-mass inverse)
//   hopsel: 0 all hops, 1 hops inside a block, 2 hops between blocks.
// Output sites: parities par0 .. par0+npar-1, blocks blk0 .. blk0+nblk-1.
struct DslashCall {
    const void *in = nullptr;
    const void *x = nullptr;
    void *out = nullptr;
    long rstride = 0;  // elements between right-hand sides
    int nrhs = 1;
    int nmass = 1;                      // mass slots: rhs r uses slot r / ceil(nrhs / nmass)
    double masses[MAXM] = {0.0};
    const void *Ainv[MAXM] = {nullptr};  // A(m)^-1 of each slot, in the policy's precision
    double alpha = 0.0, beta = 0.0;
    int diag = 0, post = 0, hopsel = 0;
    int par0 = 0, npar = 2, blk0 = 0, nblk = 0;
    // fused inner products of the output (FP32 storage, all hops, one parity, one right-hand side
    // per thread): red 1 -> conj(w) out, red 2 -> conj(out) x and |out|^2, per warp of 32 sites into
    // red_part[(rhs * (n / 32) + warp) * 3 + k]
    int red = 0;
    const void *w = nullptr;
    double *red_part = nullptr;
};
void dslash64(ddrw_ctx *ctx, const DslashCall &c);
// out (rows of colour `rows`) += beta H_{rows <- other colour} in: the hops between blocks in FP64,
// one launch per direction over the face sites (hops.cu); other rows untouched
void hop_between64(ddrw_ctx *ctx, int rows, const double2 *in, double2 *out, int nrhs, double beta);
void dslash32(ddrw_ctx *ctx, const DslashCall &c);
void dslash16(ddrw_ctx *ctx, const DslashCall &c);   // FP16 storage, FP32 arithmetic
void dslashb16(ddrw_ctx *ctx, const DslashCall &c);  // BF16 storage, FP32 arithmetic
// double-single stencil: in / x are split fields (float4 per complex), out an FP64 field
void dslash_ds(ddrw_ctx *ctx, const DslashCall &c);
// FP64 -> split elements at k V + p vh + off + j (k < 12 planes, parities p = par0 .. par0 + npar - 1,
// j < len) of nrhs fields rs elements apart; the same offsets in out
void split64(ddrw_ctx *ctx, const double2 *in, float4 *out, long V, long vh, long off, long len, int par0, int npar,
             int nrhs, long rs);
// out = alpha D x + ... as DslashCall c on FP64 fields, in FP64 (ds = false) or in double-single
// arithmetic through a split copy of the input (ds = true)
ddrw_status residual_stencil(ddrw_ctx *ctx, DslashCall c, bool ds);

// x = D_cc(ms)^-1 b on the sites of colour c (persistent block solver + FP64 defect correction)
// device buffers of the device-controlled block solve (to allocate before a capture)
ddrw_status block_solve_dc_prepare(ddrw_ctx *ctx, int nrhs);
ddrw_status block_solve64(ddrw_ctx *ctx, int colour, const MassSet &ms, const double2 *b, double2 *x, int nrhs,
                          double tol, int maxiter, ddrw_prec prec, SolveStats *stats);
// x = D(ms)^-1 b on the full lattice (even-odd BiCGStab + FP64 defect correction)
// device buffers of the device-controlled outer solve (to allocate before a capture)
ddrw_status full_solve_dc_prepare(ddrw_ctx *ctx, int nrhs);
ddrw_status full_solve64(ddrw_ctx *ctx, const MassSet &ms, const double2 *b, double2 *x, int nrhs, double tol,
                         int maxiter, ddrw_prec prec, SolveStats *stats);
// the block operator of one colour by the Krylov-loop even-odd BiCGStab (solver.cu), fields in the
// storage of policy id pid (32, 16 = FP16, 17 = BF16)
ddrw_status colour_bicgstab(ddrw_ctx *ctx, int pid, const MassSet &ms, const void *b, void *x, int nrhs,
                            const std::vector<double> &thresh, int maxiter, int *iters, int colour);
// the same on 16-bit Krylov vectors (pid 16 FP16, 17 BF16) with reliable updates into the FP32
// fields b and x (full-field layout)
ddrw_status colour_bicgstab_reliable(ddrw_ctx *ctx, int pid, const MassSet &ms, const float4 *b, float4 *x, int nrhs,
                                     const std::vector<double> &thresh, int maxiter, int *iters, int colour);
// Schwarz-preconditioned flexible GCR on FP32 fields (sap.cu): x = D(ms)^-1 b on the full lattice
// until |b - D x|^2 <= thresh[r] per right-hand side; adds its iterations to *iters
bool sap_supported(const ddrw_ctx *ctx);
size_t sap_bytes_per_site_rhs(const ddrw_ctx *ctx);
ddrw_status sap_gcr(ddrw_ctx *ctx, const MassSet &ms, const float4 *b, float4 *x, int nrhs,
                    const std::vector<double> &thresh, int maxiter, int *iters);
// mass set from a list of masses (builds the inverses on first use)
ddrw_status make_massset(ddrw_ctx *ctx, int n, const double *m, MassSet *ms);

}  // namespace ddrw
