// BF16-storage instantiations of the stencil (see dslash.cuh and lowprec.cuh)
#include "dslash.cuh"

namespace ddrw {
void dslashb16(ddrw_ctx *ctx, const DslashCall &c) { launch<PrecB>(ctx, c); }
}
