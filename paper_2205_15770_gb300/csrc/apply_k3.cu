// Cell-kernel instantiations for velocity degree k = 3 (split per degree for parallel builds).
#include "apply_launch.cuh"
SMF_INSTANTIATE_K(3)
