// float, 3D, ES kernel widths 9-16: the width-specialised launchers and their kernels.
#include "fresco_kernels.cuh"

namespace fresco {
FRESCO_WIDTHS_HI(FRESCO_INST_WOPS, float, 3)
}
