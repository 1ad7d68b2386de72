// FP16-storage instantiations of the stencil (see dslash.cuh and lowprec.cuh)
#include "dslash.cuh"

namespace ddrw {
void dslash16(ddrw_ctx *ctx, const DslashCall &c) { launch<PrecH>(ctx, c); }
}
