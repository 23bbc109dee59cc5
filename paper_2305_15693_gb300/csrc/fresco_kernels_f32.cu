// float instantiation of the libfresco launchers (the width-specialised ones come from the
// fresco_w_f32_*.cu units).
#include "fresco_kernels.cuh"

namespace fresco {
FRESCO_EXTERN_WIDTH_OPS(float)
template struct Launch<float>;
}
