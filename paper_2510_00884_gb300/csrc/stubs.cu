// Entry points whose kernels are not built into this library yet.
#include "internal.h"

namespace commet {

int launch_const_update_bf16(const commet_model *, int64_t, const void *, void *, void *, void *, int32_t *,
                             cudaStream_t) {
    return COMMET_ERR_UNSUPPORTED;
}
int launch_newton_assemble(const commet_model *, const commet_mesh *, const void *, void *, void *, int32_t *,
                           cudaStream_t) {
    return COMMET_ERR_UNSUPPORTED;
}

}  // namespace commet
