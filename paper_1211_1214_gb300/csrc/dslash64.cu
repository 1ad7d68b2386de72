// FP64 instantiations of the stencil (see dslash.cuh)
#include "dslash.cuh"

namespace ddrw {
void dslash64(ddrw_ctx *ctx, const DslashCall &c) { launch<PrecD>(ctx, c); }
}
