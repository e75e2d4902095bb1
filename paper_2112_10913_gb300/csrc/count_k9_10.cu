// count_k9_10.cu -- instantiates the counting kernels for k = 9, 10 (split across translation
// units only so that the build compiles them in parallel).
#include "count_impl.cuh"

namespace citron_host {
CITRON_LAUNCH_K_DEF(9)
CITRON_LAUNCH_K_DEF(10)
}  // namespace citron_host
