// one instantiation of the persistent block solver (see blocksolve.cuh)
#include "blocksolve.cuh"

namespace ddrw {
template void launch_block_kernel<PrecH, 8>(ddrw_ctx *ctx, const BlkArgs<PrecH> &a, int nrhs);
}
