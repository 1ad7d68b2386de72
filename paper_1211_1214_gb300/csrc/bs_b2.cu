// one instantiation of the persistent block solver (see blocksolve.cuh)
#include "blocksolve.cuh"

namespace ddrw {
template void launch_block_kernel<PrecB, 2>(ddrw_ctx *ctx, const BlkArgs<PrecB> &a, int nrhs);
}
