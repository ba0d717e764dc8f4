// Entry points whose kernels are not compiled into this build yet: they validate nothing and
// report STENCIL_ERR_UNSUPPORTED.
#include "../../include/stencil.h"

extern "C" {
int stencil_batch_plan(stencil_batch *out, const stencil_batch_item *, int, int) {
    if (out) *out = nullptr;
    return STENCIL_ERR_UNSUPPORTED;
}
int stencil_batch_launch(stencil_batch, void *) { return STENCIL_ERR_UNSUPPORTED; }
int stencil_batch_status(stencil_batch, void *) { return STENCIL_ERR_UNSUPPORTED; }
int stencil_batch_destroy(stencil_batch) { return STENCIL_OK; }
}
