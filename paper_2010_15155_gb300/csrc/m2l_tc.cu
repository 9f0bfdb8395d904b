// M->L on tcgen05 tensor cores (split BF16x3, FP32 accumulation in TMEM).
#include "plan.cuh"

namespace kafmm {

bool tc_supported(Plan& P) { return false; }

int m2l_tc_launch(Plan& P, const int4* tiles, int ntiles, const int* boxlist, cudaStream_t st) {
  return fail(P, KAFMM_ERR_STATE, "tensor-core M->L is not available");
}

}  // namespace kafmm
