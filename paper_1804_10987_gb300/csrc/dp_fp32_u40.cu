// dp_fp32_u40.cu -- the FP32 kernels for 40 and 48 padded users
// (dp_fp32_impl.cuh), compiled as their own translation unit.
#include "dp_fp32_impl.cuh"

namespace dp {
template struct Fp32Ops<40>;
template struct Fp32Ops<48>;
}  // namespace dp
