// Split-precision (Ozaki-style BF16/FP16 slices on tcgen05) planning: not yet built.
#include "tnx_plan.h"

void tnx_build_split_parts(Plan& p, StepPlan& s) {
  (void)p;
  (void)s;
  fail(TNX_ERR_UNSUPPORTED, "split precision is not available in this build");
}

void tnx_enqueue_split(Plan& p, StepPlan& s, cudaStream_t st) {
  (void)p;
  (void)s;
  (void)st;
  fail(TNX_ERR_UNSUPPORTED, "split precision is not available in this build");
}
