#pragma once
#include <vector>

#include "common.cuh"

namespace smf {
void gauss_legendre01(int n, double *x, double *w);
void gauss_lobatto01(int deg, double *x);
double lagrange(const double *nodes, int n, int i, double x);
double lagrange_deriv(const double *nodes, int n, int i, double x);
void build_tables(int k, Tab1D<double> &t);
void build_transfer(int k, TransferTab<double> &tt);
double tridiag_max_eig(const std::vector<double> &a, const std::vector<double> &b);

template <typename T>
int launch_cell_apply(const LevelDesc<T> &L, const Tab1D<T> *tab, int mode, const T *u, const T *p, T *yu, T *yp,
                      cudaStream_t s, int shape, const T *geo = nullptr, const T *rho = nullptr,
                      const GridBarrier *det = nullptr);
template <typename T>
int launch_cell_diag(const LevelDesc<T> &L, const Tab1D<T> *tab, T *dAs, T *dSloc, T *dMp, cudaStream_t s,
                     const T *rho, int sym);
template <int K, typename T>
int launch_cell_apply_k(const LevelDesc<T> &L, const Tab1D<T> *tab, int mode, const T *u, const T *p, T *yu, T *yp,
                        cudaStream_t s, int shape, const T *geo, const T *rho);
template <typename T>
int launch_cell_apply_fused(const LevelDesc<T> &L, int mode, const T *u, const T *p, T *yu, T *yp, cudaStream_t s,
                            int shape, const Fuse<T> &F, const T *geo);
template <int K, typename T>
int launch_cell_apply_fused_k(const LevelDesc<T> &L, int mode, const T *u, const T *p, T *yu, T *yp, cudaStream_t s,
                              int shape, const Fuse<T> &F, const T *geo);
template <int K, typename T>
int launch_cell_C_k(const LevelDesc<T> &L, const Tab1D<T> *tab, T cm, T cg, const T *p, T *yp, T sign, T *diag,
                    const T *Ce, cudaStream_t s);
template <int K, typename T>
int launch_cell_C_matrix_k(const LevelDesc<T> &L, const Tab1D<T> *tab, T cm, T cg, T *Ce, cudaStream_t s);
template <int K, typename T>
int launch_col_geometry_k(const LevelDesc<T> &L, T *geo, cudaStream_t s);
template <int K, typename T>
int launch_cell_grad_k(const LevelDesc<T> &L, const Tab1D<T> *tab, const T *u, const T *lam, T *g, cudaStream_t s);
template <int K>
int upload_col_tables(const Tab1D<double> &t, cudaStream_t s);
// Cell-component kernel (launch shape 5, apply_cc.cuh): 3D Cartesian levels with k = 2, 3 (FP32
// and FP64) and trilinear levels with k = 2 (FP32; FP64 where the per-point geometry is stored).
// launch_cell_apply_cc_k returns -1 for a level or mode it does not serve, 0 on a launch, and a
// cudaError_t code when the (deterministic, cooperative) launch fails.
inline bool cc_level_supported(int dim, int k, int cartesian, size_t elt) {
  (void)elt;
  if (dim != 3) return false;
  if (cartesian) return k == 2 || k == 3;
  return k == 2;
}
template <int K, typename T>
int launch_cell_apply_cc_k(const LevelDesc<T> &L, int mode, const T *u, const T *p, T *yu, T *yp, const T *geo,
                           const GridBarrier *det, cudaStream_t s);
template <int K>
int upload_cc_tables(const Tab1D<double> &t, cudaStream_t s);
template <int K, typename T>
int launch_cell_apply_cc_fused_k(const LevelDesc<T> &L, int mode, const T *u, const T *p, T *yu, T *yp,
                                 const T *geo, const Fuse<T> &F, cudaStream_t s);
template <int K, typename T>
int launch_cell_diag_k(const LevelDesc<T> &L, const Tab1D<T> *tab, T *dAs, T *dSloc, T *dMp, cudaStream_t s,
                       const T *rho, int sym);
}  // namespace smf
