// dp_fp32_u56.cu -- the FP32 kernels for 56 and 64 padded users
// (dp_fp32_impl.cuh), compiled as their own translation unit.
#include "dp_fp32_impl.cuh"

namespace dp {
template struct Fp32Ops<56>;
template struct Fp32Ops<64>;
}  // namespace dp
