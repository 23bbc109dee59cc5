// double, 2D, ES kernel widths 2-8: the width-specialised launchers and their kernels.
#include "fresco_kernels.cuh"

namespace fresco {
FRESCO_WIDTHS_LO(FRESCO_INST_WOPS, double, 2)
FRESCO_WIDTHS_LO(FRESCO_INST_WOPSB, double)
}
