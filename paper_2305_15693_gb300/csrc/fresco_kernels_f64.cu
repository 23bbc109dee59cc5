// double instantiation of the libfresco launchers (the width-specialised ones come from the
// fresco_w_f64_*.cu units).
#include "fresco_kernels.cuh"

namespace fresco {
FRESCO_EXTERN_WIDTH_OPS(double)
template struct Launch<double>;
}
