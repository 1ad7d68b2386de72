// pending.cu -- entry points whose kernels are not in this build yet; each returns DDRW_ESTATE.
#include "ctx.h"
using namespace ddrw;
extern "C" {
ddrw_status ddrw_solve_block(ddrw_ctx *ctx, int, double, const double *, double *, int, ddrw_solve_info *) { return set_error(ctx, DDRW_ESTATE, "not built"); }
ddrw_status ddrw_solve_D(ddrw_ctx *ctx, double, const double *, double *, int, ddrw_solve_info *) { return set_error(ctx, DDRW_ESTATE, "not built"); }
ddrw_status ddrw_apply_schur(ddrw_ctx *ctx, double, const double *, double *, int) { return set_error(ctx, DDRW_ESTATE, "not built"); }
ddrw_status ddrw_apply_dA(ddrw_ctx *ctx, const double *, double *, int, ddrw_solve_info *) { return set_error(ctx, DDRW_ESTATE, "not built"); }
ddrw_status ddrw_solve_schur(ddrw_ctx *ctx, double, const double *, double *, int, ddrw_solve_info *) { return set_error(ctx, DDRW_ESTATE, "not built"); }
ddrw_status ddrw_noise(ddrw_ctx *ctx, uint64_t, uint64_t, int, double *) { return set_error(ctx, DDRW_ESTATE, "not built"); }
ddrw_status ddrw_estimate(ddrw_ctx *ctx, int, uint64_t, uint64_t, const double *, double *, double *, double *, double *, ddrw_solve_info *) { return set_error(ctx, DDRW_ESTATE, "not built"); }
}
