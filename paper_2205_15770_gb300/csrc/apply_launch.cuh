// Launchers of the cell kernels for one polynomial degree K (included by apply_kK.cu).
#pragma once
#include "apply.cuh"
#include "host_tables.h"

namespace smf {

template <int DIM, int K, typename T, bool CART>
static int launch_apply_dim(const LevelDesc<T> &L, const Tab1D<T> *tab, int mode, const T *u, const T *p, T *yu,
                            T *yp, cudaStream_t s) {
  using CS = CellShape<DIM, K>;
  const long long blocks = (L.n_cells + CS::CPB - 1) / CS::CPB;
  const size_t smem = sizeof(Tab1D<T>) + (size_t)CS::CPB * CS::PER_CELL * sizeof(T);
  stokes_cell_apply<DIM, K, T, CART><<<(unsigned)blocks, CS::THREADS, smem, s>>>(L, tab, mode, u, p, yu, yp);
  return 0;
}

template <int K, typename T>
int launch_cell_apply_k(const LevelDesc<T> &L, const Tab1D<T> *tab, int mode, const T *u, const T *p, T *yu, T *yp,
                        cudaStream_t s) {
  if (L.dim == 3)
    return L.cartesian ? launch_apply_dim<3, K, T, true>(L, tab, mode, u, p, yu, yp, s)
                       : launch_apply_dim<3, K, T, false>(L, tab, mode, u, p, yu, yp, s);
  return L.cartesian ? launch_apply_dim<2, K, T, true>(L, tab, mode, u, p, yu, yp, s)
                     : launch_apply_dim<2, K, T, false>(L, tab, mode, u, p, yu, yp, s);
}

template <int DIM, int K, typename T, bool CART>
static int launch_diag_dim(const LevelDesc<T> &L, const Tab1D<T> *tab, T *dAs, T *dSloc, T *dMp, cudaStream_t s) {
  using CS = CellShape<DIM, K>;
  stokes_cell_diagonals<DIM, K, T, CART><<<(unsigned)L.n_cells, CS::NP, 0, s>>>(L, tab, dAs, dSloc, dMp);
  return 0;
}

template <int K, typename T>
int launch_cell_diag_k(const LevelDesc<T> &L, const Tab1D<T> *tab, T *dAs, T *dSloc, T *dMp, cudaStream_t s) {
  if (L.dim == 3)
    return L.cartesian ? launch_diag_dim<3, K, T, true>(L, tab, dAs, dSloc, dMp, s)
                       : launch_diag_dim<3, K, T, false>(L, tab, dAs, dSloc, dMp, s);
  return L.cartesian ? launch_diag_dim<2, K, T, true>(L, tab, dAs, dSloc, dMp, s)
                     : launch_diag_dim<2, K, T, false>(L, tab, dAs, dSloc, dMp, s);
}

}  // namespace smf

#define SMF_INSTANTIATE_K(KK)                                                                                  \
  namespace smf {                                                                                              \
  template int launch_cell_apply_k<KK, float>(const LevelDesc<float> &, const Tab1D<float> *, int,             \
                                               const float *, const float *, float *, float *, cudaStream_t);  \
  template int launch_cell_apply_k<KK, double>(const LevelDesc<double> &, const Tab1D<double> *, int,          \
                                                const double *, const double *, double *, double *,            \
                                                cudaStream_t);                                                  \
  template int launch_cell_diag_k<KK, double>(const LevelDesc<double> &, const Tab1D<double> *, double *,      \
                                               double *, double *, cudaStream_t);                              \
  }
