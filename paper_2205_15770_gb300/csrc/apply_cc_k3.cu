// Cell-component kernel instantiations for velocity degree k = 3 (own translation unit: its
// 1D tables live in this unit's constant memory).
#include "apply_cc.cuh"
#include "host_tables.h"

namespace smf {
template int launch_cell_apply_cc_k<3, float>(const LevelDesc<float> &, int, const float *, const float *, float *,
                                              float *, const float *, const GridBarrier *, cudaStream_t);
template int launch_cell_apply_cc_k<3, double>(const LevelDesc<double> &, int, const double *, const double *,
                                               double *, double *, const double *, const GridBarrier *, cudaStream_t);
template int upload_cc_tables<3>(const Tab1D<double> &, cudaStream_t);
template int launch_cell_apply_cc_fused_k<3, float>(const LevelDesc<float> &, int, const float *, const float *,
                                                     float *, float *, const float *, const Fuse<float> &,
                                                     cudaStream_t);
template int launch_cell_apply_cc_fused_k<3, double>(const LevelDesc<double> &, int, const double *,
                                                      const double *, double *, double *, const double *,
                                                      const Fuse<double> &, cudaStream_t);
}  // namespace smf
