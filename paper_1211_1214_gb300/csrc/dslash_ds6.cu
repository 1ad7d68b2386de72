// one block length of the double-single residual stencil (see dslash_ds.cu)
#include "dslash.cuh"

namespace ddrw {
template void launch_bl<PrecDD, 6>(ddrw_ctx *ctx, const DslashCall &c);
}
