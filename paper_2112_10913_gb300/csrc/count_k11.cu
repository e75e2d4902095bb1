// count_k11.cu -- instantiates the counting kernels for k = 11 (one translation unit per k
// from 7 up, where the recursion is deep, so that the build compiles them in parallel).
#include "count_impl.cuh"

namespace citron_host {
CITRON_LAUNCH_K_DEF(11)
}  // namespace citron_host
