// RPY sphere velocities: assembly u + a^2/6 lap u (Eq. RPYtrgvel) and the overlap
// post-processing of Sec. II.B.
#include "plan.cuh"

namespace kafmm {

int rpy_velocity(Plan& P, const void* s, const void* a, const void* g, void* ua, int dtype) {
  return fail(P, KAFMM_ERR_STATE, "kafmm_rpy_velocity is not available in this build");
}

}  // namespace kafmm
