// mixed.cu -- mixed-precision frequency solves and field evaluation (filled in below).
#include "bie_common.cuh"

namespace bie {

int solve_mixed(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep) {
  return fail(BIE_ERR_INVALID_ARG, "BIE_MODE_MIXED is not available in this build");
}

int field_mixed(bie_ctx* c, const double* kv, int nk, const cd* surf, const double* xp, int64_t M,
                const int32_t* foot_elem, const double* foot, cd* T, void* scratch, size_t scratch_bytes) {
  return fail(BIE_ERR_INVALID_ARG, "BIE_MODE_MIXED is not available in this build");
}

}  // namespace bie
