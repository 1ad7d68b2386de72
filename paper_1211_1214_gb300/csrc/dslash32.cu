// FP32 instantiations of the stencil (see dslash.cuh)
#include "dslash.cuh"

namespace ddrw {
void dslash32(ddrw_ctx *ctx, const DslashCall &c) { launch<PrecS>(ctx, c); }
}
