// Cell-component kernel instantiations for velocity degree k = 2 (own translation unit: its
// 1D tables live in this unit's constant memory), and the batched work-queue kernel, whose cell
// items use the same tables.
#include "apply_cc.cuh"
#include "host_tables.h"
#include "queue.cuh"

namespace smf {
template int launch_cell_apply_cc_k<2, float>(const LevelDesc<float> &, int, const float *, const float *, float *,
                                              float *, const float *, const GridBarrier *, cudaStream_t);
template int launch_cell_apply_cc_k<2, double>(const LevelDesc<double> &, int, const double *, const double *,
                                               double *, double *, const double *, const GridBarrier *, cudaStream_t);
template int upload_cc_tables<2>(const Tab1D<double> &, cudaStream_t);
template int launch_cell_apply_cc_fused_k<2, float>(const LevelDesc<float> &, int, const float *, const float *,
                                                     float *, float *, const float *, const Fuse<float> &,
                                                     cudaStream_t);
template int launch_cell_apply_cc_fused_k<2, double>(const LevelDesc<double> &, int, const double *,
                                                      const double *, double *, double *, const double *,
                                                      const Fuse<double> &, cudaStream_t);
}  // namespace smf
