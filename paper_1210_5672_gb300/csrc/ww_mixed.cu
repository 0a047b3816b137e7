// ww_mixed.cu -- mixed-precision DtN linear algebra (placeholder until the
// tensor-core path lands; ww_create rejects WW_MIXED meanwhile).
#include "ww_internal.cuh"

namespace ww {

int mixed_create(Ctx *) { return fail(WW_ERR_ARG, "WW_MIXED is not available in this build"); }
void mixed_destroy(Ctx *) {}
int mixed_setup(Ctx *) { return fail(WW_ERR_ARG, "WW_MIXED is not available in this build"); }
int mixed_solve(Ctx *, double *, int) { return fail(WW_ERR_ARG, "WW_MIXED is not available in this build"); }
int mixed_apply_G(Ctx *, int, int) { return fail(WW_ERR_ARG, "WW_MIXED is not available in this build"); }

}  // namespace ww
