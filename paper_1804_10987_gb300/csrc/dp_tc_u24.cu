// dp_tc_u24.cu -- the reduced-precision group kernel for 24 and 32 padded
// users (dp_tc_impl.cuh), compiled as its own translation unit.
#include "dp_tc_impl.cuh"

namespace dp {
template struct TcOps<24>;
template struct TcOps<32>;
}  // namespace dp
