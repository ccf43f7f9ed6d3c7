// dp_tc_u40.cu -- the reduced-precision group kernel for 40 and 48 padded
// users (dp_tc_impl.cuh), compiled as its own translation unit.
#include "dp_tc_impl.cuh"

namespace dp {
template struct TcOps<40>;
template struct TcOps<48>;
}  // namespace dp
