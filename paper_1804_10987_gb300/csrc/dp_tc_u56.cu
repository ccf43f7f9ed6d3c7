// dp_tc_u56.cu -- the reduced-precision group kernel for 56 and 64 padded
// users (dp_tc_impl.cuh), compiled as its own translation unit.
#include "dp_tc_impl.cuh"

namespace dp {
template struct TcOps<56>;
template struct TcOps<64>;
}  // namespace dp
