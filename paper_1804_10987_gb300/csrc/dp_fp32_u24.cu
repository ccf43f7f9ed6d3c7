// dp_fp32_u24.cu -- the FP32 kernels for 24 and 32 padded users
// (dp_fp32_impl.cuh), compiled as their own translation unit.
#include "dp_fp32_impl.cuh"

namespace dp {
template struct Fp32Ops<24>;
template struct Fp32Ops<32>;
}  // namespace dp
