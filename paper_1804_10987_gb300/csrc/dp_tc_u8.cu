// dp_tc_u8.cu -- the reduced-precision group kernel for 8 and 16 padded
// users (dp_tc_impl.cuh), compiled as its own translation unit.
#include "dp_tc_impl.cuh"

namespace dp {
template struct TcOps<8>;
template struct TcOps<16>;
}  // namespace dp
