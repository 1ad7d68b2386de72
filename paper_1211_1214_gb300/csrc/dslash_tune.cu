// dslash_tune.cu -- autotuner of the stencil launches.
//
// For each launch shape (precision, block length, parities, right-hand sides, diagonal and
// post-multiply modes, right-hand sides per mass slot) the first launch times every candidate
// configuration -- right-hand sides per thread NR in {1, 2, 4} (dividing the right-hand sides per
// mass slot) and CTA sizes {64, 128, 256} -- with CUDA events on the context's stream, keeps the
// fastest, and reuses it for every later launch of that shape.  The candidates run on the real
// arguments: a stencil launch never reads its own output sites, so repeating it is harmless.
// While the stream is being captured into a graph nothing is timed and the default is used.
#include <cstdio>
#include <string>

#include "dslash.cuh"

namespace ddrw {

DsConfig tuned_config(ddrw_ctx *ctx, const DslashCall &c, int prec, int bl,
                      void (*run)(ddrw_ctx *, const DslashCall &, DsConfig))
{
    const int nm = c.nmass < 1 ? 1 : c.nmass;
    const int rpm = (c.nrhs + nm - 1) / nm;
    std::array<int, 8> key = {prec, bl, c.npar, c.nrhs, c.diag, c.post, rpm, c.beta != 0.0};
    auto it = ctx->tune.find(key);
    if (it != ctx->tune.end()) return DsConfig{it->second.nr, it->second.nt};

    DsConfig def;
    def.nr = (rpm % 2 == 0 && c.nrhs % 2 == 0) ? 2 : 1;
    def.nt = 128;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    if (!ctx->autotune || cs != cudaStreamCaptureStatusNone) {
        if (cs == cudaStreamCaptureStatusNone) ctx->tune[key] = TuneEntry{def.nr, def.nt, -1.0f};
        return def;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    DsConfig best = def;
    float best_ms = 1e30f;
    const int nrs[3] = {1, 2, 4}, nts[3] = {64, 128, 256};
    for (int nr : nrs) {
        if (c.nrhs % nr || rpm % nr) continue;
        for (int nt : nts) {
            DsConfig cfg{nr, nt};
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
    ctx->tune[key] = TuneEntry{best.nr, best.nt, best_ms / 2};
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
    return DDRW_OK;
}

ddrw_status ddrw_autotune_report(ddrw_ctx *ctx, char *buf, long len)
{
    if (!ctx || !buf || len <= 0) return DDRW_EINVAL;
    std::string s;
    for (auto &kv : ctx->tune) {
        const auto &k = kv.first;
        char line[200];
        snprintf(line, sizeof line, "fp%d l=%d npar=%d nrhs=%d diag=%d post=%d rpm=%d hop=%d -> nr=%d nt=%d ms=%.4f\n", k[0],
                 k[1], k[2], k[3], k[4], k[5], k[6], k[7], kv.second.nr, kv.second.nt, kv.second.ms);
        s += line;
    }
    if ((long)s.size() + 1 > len) return set_error(ctx, DDRW_EINVAL, "report buffer too small");
    memcpy(buf, s.c_str(), s.size() + 1);
    return DDRW_OK;
}

}  // extern "C"
