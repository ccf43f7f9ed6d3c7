// dp_tc.cu -- dispatch of the reduced-precision group kernel's launchers on
// the padded user count (the kernels: dp_tc_impl.cuh, instantiated per user
// count in dp_tc_u*.cu so that they compile in parallel).
#include "dp_internal.h"

namespace dp {

extern template struct TcOps<8>;
extern template struct TcOps<16>;
extern template struct TcOps<24>;
extern template struct TcOps<32>;
extern template struct TcOps<40>;
extern template struct TcOps<48>;
extern template struct TcOps<56>;
extern template struct TcOps<64>;

#define DP_TC_DISPATCH(UPV, CALL, FAIL)             \
  switch (UPV) {                                    \
    case 8: { using O = TcOps<8>; return CALL; }    \
    case 16: { using O = TcOps<16>; return CALL; }  \
    case 24: { using O = TcOps<24>; return CALL; }  \
    case 32: { using O = TcOps<32>; return CALL; }  \
    case 40: { using O = TcOps<40>; return CALL; }  \
    case 48: { using O = TcOps<48>; return CALL; }  \
    case 56: { using O = TcOps<56>; return CALL; }  \
    case 64: { using O = TcOps<64>; return CALL; }  \
    default: return FAIL;                           \
  }

bool tc_supported(int UP) { return UP >= 8 && UP <= 64 && UP % 8 == 0; }

int tc_systems_per_group(int UP) {
  return UP > 0 && UP <= 64 ? (128 / (2 * UP) > 0 ? 128 / (2 * UP) : 1) : 1;
}

cudaError_t launch_batch_tc(int UP, bool bf16, const InstDesc *insts, const WorkItem *items,
                            int n_items, int *queue, int Kmax, int grid, cudaStream_t s,
                            const int *fix_list, const int *fix_count, int phase,
                            const SplitWs &ws) {
  DP_TC_DISPATCH(UP, O::batch(bf16, insts, items, n_items, queue, Kmax, grid, s, fix_list,
                              fix_count, phase, ws),
                 cudaErrorInvalidValue);
}

int tc_max_blocks_per_sm(int UP, bool bf16, int Kmax) {
  DP_TC_DISPATCH(UP, O::blocks(bf16, Kmax), 0);
}

cudaError_t launch_fused_tc(const SysDesc &d, int UP, bool bf16, const float2 *H, const float2 *S,
                            float2 *X, int *status, float *scale_out, cudaStream_t s) {
  DP_TC_DISPATCH(UP, O::fused(d, bf16, H, S, X, status, scale_out, s), cudaErrorInvalidValue);
}

cudaError_t launch_fixup_tc(const SysDesc &d, int UP, bool bf16, const float2 *H, const float2 *S,
                            float2 *X, int *status, const int *fix_list, int *fix_count,
                            int grid, cudaStream_t s) {
  DP_TC_DISPATCH(UP, O::fixup(d, bf16, H, S, X, status, fix_list, fix_count, grid, s),
                 cudaErrorInvalidValue);
}

}  // namespace dp
