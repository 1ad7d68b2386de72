// one instantiation of the clover-term kernel (see clover.cuh)
#include "clover.cuh"

namespace ddrw {
template void clover_launch<6>(ddrw_ctx *ctx);
}
