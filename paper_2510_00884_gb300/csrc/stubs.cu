// Entry points whose kernels are not built into this library yet.
#include "internal.h"

namespace commet {


}  // namespace commet
