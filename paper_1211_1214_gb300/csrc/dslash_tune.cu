// dslash_tune.cu -- autotuner of the stencil launches.
//
// For each launch shape (precision, block length, parities, right-hand sides, diagonal and
// post-multiply modes, right-hand sides per mass slot) the first launch times every candidate
// configuration -- right-hand sides per thread NR in {1, 2, 4} (dividing the right-hand sides per
// mass slot), sites per CTA row in {64, 128, 256}, CTA rows (groups of NR right-hand sides of the
// same sites, sharing links and clover terms in L1) in {1, 2}, at most 256 threads per CTA, and
// the hop code form (unrolled, rolled, with the loads of 4 or 8 hops batched ahead of their
// arithmetic, or unrolled under a register cap of 85 or 128 for more warps per SM, the last two
// also with the neighbours read from the precomputed neighbour table) -- with CUDA
// events on the context's stream, keeps the fastest,
// and reuses it for every later launch of that shape.  The candidates run on the real
// arguments, which is harmless only while a launch does not read its own output sites: the hop
// input of a one-parity launch lies on the other parity, but a launch whose output is its
// diagonal input x, or its hop input with both parities written, would change its own input on
// every repetition.  Such a launch is never timed: it runs the default form and leaves its shape
// untuned for a later launch with separate buffers.  While the stream is being captured into a
// graph nothing is timed and the default is used.
#include <cstdio>
#include <mutex>
#include <string>

#include "dslash.cuh"

namespace ddrw {

// Tuned shapes are also kept for the whole process, by device and lattice geometry, so that a new
// context on the same lattice (the auxiliary context of the nested block factor, a second
// configuration) starts from the measured choices instead of timing them again.
namespace {
std::mutex g_tune_mutex;
std::map<std::array<long, 15>, TuneEntry> g_tune;

std::array<long, 15> process_key(const ddrw_ctx *ctx, const std::array<int, 8> &k)
{
    std::array<long, 15> pk{};
    pk[0] = ctx->device;
    for (int mu = 0; mu < 4; mu++) pk[1 + mu] = ctx->dims[mu];
    pk[5] = ctx->l;
    pk[6] = ctx->cut;
    for (int i = 0; i < 8; i++) pk[7 + i] = k[i];
    return pk;
}
}  // namespace

// right-hand sides per thread each hop code form supports
static bool form_allowed(int nr, int roll)
{
    if (roll < 0 || roll > 11) return false;
    if ((roll >= 2 && roll <= 4) || roll >= 7) return nr == 1;
    if (roll == 5 || roll == 6) return nr <= 2;
    return true;
}

DsConfig tuned_config(ddrw_ctx *ctx, const DslashCall &c, int prec, int bl,
                      void (*run)(ddrw_ctx *, const DslashCall &, DsConfig))
{
    const int nm = c.nmass < 1 ? 1 : c.nmass;
    const int rpm = (c.nrhs + nm - 1) / nm;
    if (ctx->pinned_nr > 0) {
        DsConfig p{ctx->pinned_nr, ctx->pinned_nt, ctx->pinned_nw, ctx->pinned_roll};
        if (p.roll != 8 && (c.nrhs % (p.nr * p.nw) || rpm % (p.nr * p.nw))) p.nr = 1, p.nw = 1;
        return p;
    }
    std::array<int, 8> key = {prec, bl, c.npar, c.nrhs, c.diag, c.post, rpm, (c.beta != 0.0) + 2 * c.hopsel};
    auto it = ctx->tune.find(key);
    if (it != ctx->tune.end()) return DsConfig{it->second.nr, it->second.nt, it->second.nw, it->second.roll};
    if (ctx->autotune) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto g = g_tune.find(process_key(ctx, key));
        if (g != g_tune.end()) {
            ctx->tune[key] = g->second;
            return DsConfig{g->second.nr, g->second.nt, g->second.nw, g->second.roll};
        }
    }

    DsConfig def;
    def.nr = (rpm % 2 == 0 && c.nrhs % 2 == 0) ? 2 : 1;
    def.nt = 128;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    if (!ctx->autotune || cs != cudaStreamCaptureStatusNone) {
        if (cs == cudaStreamCaptureStatusNone) ctx->tune[key] = TuneEntry{def.nr, def.nt, def.nw, def.roll, -1.0f};
        return def;
    }
    // output aliasing an input on the sites it reads: repeated runs would not be idempotent
    if ((c.diag != 0 && c.x != nullptr && c.x == c.out) || (c.in != nullptr && c.in == c.out && c.npar == 2))
        return def;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    DsConfig best = def;
    float best_ms = 1e30f;
    const int nrs[3] = {1, 2, 4}, nts[3] = {64, 128, 256}, nws[2] = {1, 2}, nws8[4] = {1, 2, 4, 8};
    for (int roll = 0; roll < 12; roll++)
    for (int nr : nrs) {
        // the batched and register-capped forms are for 32- and 16-bit storage: with FP64 data
        // they spill; the staged and pipelined forms are for FP32 storage; the fully rolled form
        // for the double-single residual
        if (c.nrhs % nr || rpm % nr || (roll >= 2 && prec == 64) || !form_allowed(nr, roll) ||
            (roll >= 8 && roll <= 10 && prec != 32) || (roll == 11 && prec != 128))
            continue;
        // double-single launches: unrolled, rolled or fully rolled, one right-hand side per thread,
        // one row (also for the hops inside the blocks)
        if (prec == 128 && (nr != 1 || (roll > 1 && roll != 11))) continue;
        // other launches restricted to the hops inside the blocks come in the unrolled,
        // register-capped and table forms with one right-hand side per thread
        if (prec != 128 && c.hopsel != 0 && (nr != 1 || (roll != 0 && roll != 5 && roll != 6))) continue;
        const int *nwl = roll == 8 ? nws8 : nws;
        const int nnw = roll == 8 ? 4 : 2;
        for (int iw = 0; iw < nnw; iw++)
        for (int nt : nts) {
            const int nw = nwl[iw];
            if (prec == 128 && nw != 1) continue;
            if (roll == 8 ? (nt > 128 || nw > rpm) : (c.nrhs / nr) % nw != 0) continue;
            if (nt * nw > 256) continue;
            DsConfig cfg{nr, nt, nw, roll};
            run(ctx, c, cfg);  // warm
            cudaEventRecord(e0, ctx->stream);
            run(ctx, c, cfg);
            run(ctx, c, cfg);
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (cudaGetLastError() == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best = cfg;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune[key] = TuneEntry{best.nr, best.nt, best.nw, best.roll, best_ms / 2};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune[process_key(ctx, key)] = ctx->tune[key];
    }
    return best;
}

}  // namespace ddrw

using namespace ddrw;

extern "C" {

ddrw_status ddrw_autotune(ddrw_ctx *ctx, int enable)
{
    if (!ctx) return DDRW_EINVAL;
    ctx->autotune = enable != 0;
    ctx->tune.clear();
    ctx->blk_tune.clear();
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune.clear();
    }
    clear_graphs(ctx);  // captured launches keep the form they were captured with
    return DDRW_OK;
}

ddrw_status ddrw_stencil_config(ddrw_ctx *ctx, int nr, int nt, int nw, int roll)
{
    if (!ctx) return DDRW_EINVAL;
    if (nr == 0) {
        if (ctx->pinned_nr) clear_graphs(ctx);  // captured launches keep the form they were captured with
        ctx->pinned_nr = 0;
        return DDRW_OK;
    }
    if ((nr != 1 && nr != 2 && nr != 4) || nt < 32 || nt > 256 || nt % 32 || nw < 1 || nt * nw > 256 ||
        !form_allowed(nr, roll) || (roll == 8 && nt > 128))
        return set_error(ctx, DDRW_EINVAL, "bad stencil configuration");
    if (ctx->pinned_nr != nr || ctx->pinned_nt != nt || ctx->pinned_nw != nw || ctx->pinned_roll != roll)
        clear_graphs(ctx);
    ctx->pinned_nr = nr;
    ctx->pinned_nt = nt;
    ctx->pinned_nw = nw;
    ctx->pinned_roll = roll;
    return DDRW_OK;
}

ddrw_status ddrw_test_stall_staging(ddrw_ctx *ctx, int enable)
{
    if (!ctx) return DDRW_EINVAL;
    ctx->stall_tx = enable ? 16 : 0;
    clear_graphs(ctx);  // captured launches hold the switch's value
    return DDRW_OK;
}

ddrw_status ddrw_autotune_report(ddrw_ctx *ctx, char *buf, long len)
{
    if (!ctx || !buf || len <= 0) return DDRW_EINVAL;
    std::string s;
    for (auto &kv : ctx->tune) {
        const auto &k = kv.first;
        char line[200];
        snprintf(line, sizeof line,
                 "fp%d l=%d npar=%d nrhs=%d diag=%d post=%d rpm=%d hop=%d sel=%d -> nr=%d nt=%d nw=%d roll=%d ms=%.4f\n",
                 k[0], k[1], k[2], k[3], k[4], k[5], k[6], k[7] & 1, k[7] >> 1, kv.second.nr, kv.second.nt, kv.second.nw,
                 kv.second.roll, kv.second.ms);
        s += line;
    }
    for (auto &kv : ctx->blk_tune) {  // persistent block solver: key (storage, l, 2 nrhs + pairs allowed)
        char line[120];
        snprintf(line, sizeof line, "block fp%d l=%d nrhs=%d -> form=%d\n", kv.first[0], kv.first[1], kv.first[2] / 2,
                 kv.second);
        s += line;
    }
    if ((long)s.size() + 1 > len) return set_error(ctx, DDRW_EINVAL, "report buffer too small");
    memcpy(buf, s.c_str(), s.size() + 1);
    return DDRW_OK;
}

}  // extern "C"
