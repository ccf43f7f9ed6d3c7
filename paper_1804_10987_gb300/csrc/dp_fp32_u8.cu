// dp_fp32_u8.cu -- the FP32 kernels for 8 and 16 padded users
// (dp_fp32_impl.cuh), compiled as their own translation unit.
#include "dp_fp32_impl.cuh"

namespace dp {
template struct Fp32Ops<8>;
template struct Fp32Ops<16>;
}  // namespace dp
