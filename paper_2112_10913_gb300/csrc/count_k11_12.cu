// count_k11_12.cu -- instantiates the counting kernels for k = 11, 12 (split across translation
// units only so that the build compiles them in parallel).
#include "count_impl.cuh"

namespace citron_host {
CITRON_LAUNCH_K_DEF(11)
CITRON_LAUNCH_K_DEF(12)
}  // namespace citron_host
