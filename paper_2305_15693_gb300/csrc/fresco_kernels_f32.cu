// float instantiation of the libfresco kernels.
#include "fresco_kernels.cuh"

namespace fresco {
template struct Launch<float>;
}
