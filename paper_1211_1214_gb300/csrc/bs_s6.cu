// one instantiation of the persistent block solver (see blocksolve.cuh)
#include "blocksolve.cuh"

namespace ddrw {
template void launch_block_kernel<PrecS, 6>(ddrw_ctx *ctx, const BlkArgs<PrecS> &a, int nrhs);
}
