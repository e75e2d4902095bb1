// count_k7_8.cu -- instantiates the counting kernels for k = 7, 8 (split across translation
// units only so that the build compiles them in parallel).
#include "count_impl.cuh"

namespace citron_host {
CITRON_LAUNCH_K_DEF(7)
CITRON_LAUNCH_K_DEF(8)
}  // namespace citron_host
