// count_k3_6.cu -- instantiates the counting kernels for k = 3, 4, 5, 6 (split across translation
// units only so that the build compiles them in parallel).
#include "count_impl.cuh"

namespace citron_host {
CITRON_LAUNCH_K_DEF(3)
CITRON_LAUNCH_K_DEF(4)
CITRON_LAUNCH_K_DEF(5)
CITRON_LAUNCH_K_DEF(6)
}  // namespace citron_host
