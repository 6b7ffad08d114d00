// Tucker-format driver (placeholder until the Tucker kernels land).
#include <cstdio>

#include "dvm_context.h"

using namespace dvm;

static int unsupported() {
  set_error("Tucker format not available in this build");
  return DVM_ERR_UNSUPPORTED;
}
int tucker_alloc(dvm_ctx *) { return unsupported(); }
void tucker_free(dvm_ctx *) {}
int tucker_init_from_full(dvm_ctx *, const double *) { return unsupported(); }
int tucker_step(dvm_ctx *, int32_t, double *) { return unsupported(); }
int tucker_moments(dvm_ctx *, double *) { return unsupported(); }
int tucker_get_f(dvm_ctx *, int64_t, int64_t, double *) { return unsupported(); }
int tucker_get_ranks(dvm_ctx *, int32_t *) { return unsupported(); }
int tucker_memory(dvm_ctx *, size_t *) { return unsupported(); }
int tucker_save(dvm_ctx *, FILE *) { return unsupported(); }
int tucker_load(dvm_ctx *, FILE *) { return unsupported(); }
