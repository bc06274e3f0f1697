// Launchers of the cell kernels for one polynomial degree K (included by apply_kK.cu).
#pragma once
#include <cstdlib>
#include "apply.cuh"
#include "apply_col.cuh"
#include "apply_c.cuh"
#include "vec.cuh"
#include "host_tables.h"

namespace smf {

// STOKES_GENERIC_KERNEL=1 routes 3D applications to the point-per-thread kernel (for A/B runs).
static inline bool getenv_generic() {
  static int v = -1;
  if (v < 0) {
    const char *e = getenv("STOKES_GENERIC_KERNEL");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v == 1;
}

template <int DIM, int K, typename T, bool CART>
static int launch_apply_dim(const LevelDesc<T> &L, const Tab1D<T> *tab, int mode, const T *u, const T *p, T *yu,
                            T *yp, cudaStream_t s, const T *rho) {
  using CS = CellShape<DIM, K>;
  const long long blocks = (L.n_cells + CS::CPB - 1) / CS::CPB;
  const size_t smem = sizeof(Tab1D<T>) + (size_t)CS::CPB * CS::PER_CELL * sizeof(T);
  launch_kernel(stokes_cell_apply<DIM, K, T, CART>, dim3((unsigned)blocks), dim3(CS::THREADS), smem, s, L, tab, mode, u,
                p, yu, yp, rho);
  return 0;
}

template <int K, typename T, int MODE, bool CART, int WARPS, bool FUSED>
static int launch_col_w(const LevelDesc<T> &L, const T *u, const T *p, T *yu, T *yp, cudaStream_t s,
                        const Fuse<T> &F, const T *geo) {
  using CS = ColShape<K>;
  const long long cpb = (long long)CS::CPW * (WARPS == 3 ? 1 : WARPS);  // WARPS 3: one cell group, 3 components
  const long long blocks = (L.n_cells + cpb - 1) / cpb;
  launch_kernel(stokes_cell_apply_col<K, T, MODE, CART, WARPS, FUSED>, dim3((unsigned)blocks), dim3(32 * WARPS), 0, s,
                L, u, p, yu, yp, F, geo);
  return 0;
}

template <int K, typename T, int MODE, bool CART, bool FUSED>
static int launch_col(const LevelDesc<T> &L, const T *u, const T *p, T *yu, T *yp, cudaStream_t s, int shape,
                      const Fuse<T> &F, const T *geo) {
  switch (shape) {
    case 1: return launch_col_w<K, T, MODE, CART, 1, FUSED>(L, u, p, yu, yp, s, F, geo);
    case 3: return launch_col_w<K, T, MODE, CART, 3, FUSED>(L, u, p, yu, yp, s, F, geo);
    default: return launch_col_w<K, T, MODE, CART, 4, FUSED>(L, u, p, yu, yp, s, F, geo);
  }
}

template <int K, typename T, int MODE, bool FUSED>
static int launch_col_mode(const LevelDesc<T> &L, const T *u, const T *p, T *yu, T *yp, cudaStream_t s, int shape,
                           const Fuse<T> &F, const T *geo) {
  return L.cartesian ? launch_col<K, T, MODE, true, FUSED>(L, u, p, yu, yp, s, shape, F, geo)
                     : launch_col<K, T, MODE, false, FUSED>(L, u, p, yu, yp, s, shape, F, geo);
}

// shape: 3D launch shape chosen by the autotuner (1 / 4 warps per CTA column kernel, 3 = column
// kernel with the velocity components split over the 3 warps of a CTA, -1 point kernel,
// 0 default = column kernel with 4 warps).
template <int K, typename T>
int launch_cell_apply_k(const LevelDesc<T> &L, const Tab1D<T> *tab, int mode, const T *u, const T *p, T *yu, T *yp,
                        cudaStream_t s, int shape, const T *geo, const T *rho) {
  // the column kernel serves the Laplacian form with a constant rho; the A block of the
  // symmetric form or with a per-cell rho runs in the generic kernel
  const bool generic_a = (mode & kApplyA) && ((mode & kApplySym) || rho);
  if (L.dim == 3 && !getenv_generic() && shape >= 0 && !generic_a) {
    const Fuse<T> F{};
    switch (mode) {
      case kApplyA: return launch_col_mode<K, T, kApplyA, false>(L, u, p, yu, yp, s, shape, F, geo);
      case kApplyBT: return launch_col_mode<K, T, kApplyBT, false>(L, u, p, yu, yp, s, shape, F, geo);
      case kApplyB: return launch_col_mode<K, T, kApplyB, false>(L, u, p, yu, yp, s, shape, F, geo);
      case kApplyA | kApplyBT: return launch_col_mode<K, T, kApplyA | kApplyBT, false>(L, u, p, yu, yp, s, shape, F, geo);
      case kApplyA | kApplyBT | kApplyB:
        return launch_col_mode<K, T, kApplyA | kApplyBT | kApplyB, false>(L, u, p, yu, yp, s, shape, F, geo);
      default: break;
    }
  }
  if (L.dim == 3)
    return L.cartesian ? launch_apply_dim<3, K, T, true>(L, tab, mode, u, p, yu, yp, s, rho)
                       : launch_apply_dim<3, K, T, false>(L, tab, mode, u, p, yu, yp, s, rho);
  return L.cartesian ? launch_apply_dim<2, K, T, true>(L, tab, mode, u, p, yu, yp, s, rho)
                     : launch_apply_dim<2, K, T, false>(L, tab, mode, u, p, yu, yp, s, rho);
}

template <int DIM, int K, typename T, bool CART>
static void launch_C_dim(const LevelDesc<T> &L, const Tab1D<T> *tab, T cm, T cg, const T *p, T *yp, T sign, T *diag,
                         const T *Ce, cudaStream_t s) {
  const long long nb = (L.n_cells + 127) / 128;
  const dim3 grid((unsigned)(nb < 152 * 16 ? nb : 152 * 16));
  if constexpr (CellShape<DIM, K>::NPP <= kMaxCMatrixNodes) {
    if (Ce && !diag) {
      launch_kernel(stokes_cell_apply_C_mat<DIM, K, T>, grid, dim3(128), 0, s, L, Ce, p, yp, sign);
      return;
    }
  }
  launch_kernel(stokes_cell_apply_C<DIM, K, T, CART>, grid, dim3(128), 0, s, L, tab, cm, cg, p, yp, sign, diag);
}

// Stabilisation block C: yp += sign * C p (diag == null; from the element matrices Ce when not
// null) or diag += diag(C).
template <int K, typename T>
int launch_cell_C_k(const LevelDesc<T> &L, const Tab1D<T> *tab, T cm, T cg, const T *p, T *yp, T sign, T *diag,
                    const T *Ce, cudaStream_t s) {
  if (L.dim == 3) {
    if (L.cartesian)
      launch_C_dim<3, K, T, true>(L, tab, cm, cg, p, yp, sign, diag, Ce, s);
    else
      launch_C_dim<3, K, T, false>(L, tab, cm, cg, p, yp, sign, diag, Ce, s);
  } else {
    if (L.cartesian)
      launch_C_dim<2, K, T, true>(L, tab, cm, cg, p, yp, sign, diag, Ce, s);
    else
      launch_C_dim<2, K, T, false>(L, tab, cm, cg, p, yp, sign, diag, Ce, s);
  }
  return 0;
}

// Packed element matrices of C (stokes_cell_C_matrix): n_cells * NPP (NPP + 1) / 2 entries.
template <int DIM, int K, typename T, bool CART>
static void launch_C_matrix_dim(const LevelDesc<T> &L, const Tab1D<T> *tab, T cm, T cg, T *Ce, cudaStream_t s) {
  if constexpr (CellShape<DIM, K>::NPP <= kMaxCMatrixNodes)
    launch_kernel(stokes_cell_C_matrix<DIM, K, T, CART>,
                  dim3(vec_blocks(L.n_cells * CellShape<DIM, K>::NPP)), dim3(kVecThreads), 0, s, L, tab, cm, cg, Ce);
}
template <int K, typename T>
int launch_cell_C_matrix_k(const LevelDesc<T> &L, const Tab1D<T> *tab, T cm, T cg, T *Ce, cudaStream_t s) {
  if (L.dim == 3) {
    if (L.cartesian)
      launch_C_matrix_dim<3, K, T, true>(L, tab, cm, cg, Ce, s);
    else
      launch_C_matrix_dim<3, K, T, false>(L, tab, cm, cg, Ce, s);
  } else {
    if (L.cartesian)
      launch_C_matrix_dim<2, K, T, true>(L, tab, cm, cg, Ce, s);
    else
      launch_C_matrix_dim<2, K, T, false>(L, tab, cm, cg, Ce, s);
  }
  return 0;
}

template <int K, typename T>
int launch_col_geometry_k(const LevelDesc<T> &L, T *geo, cudaStream_t s) {
  constexpr int NV = K + 1;
  launch_kernel(k_col_geometry<K, T>, dim3(vec_blocks(L.n_cells * NV * NV)), dim3(kVecThreads), 0, s, L, geo);
  return 0;
}

// Fused application (3D column kernel only; shape >= 0): returns -1 for a mode without a fused
// instantiation so that the caller can reject it.
template <int K, typename T>
int launch_cell_apply_fused_k(const LevelDesc<T> &L, int mode, const T *u, const T *p, T *yu, T *yp, cudaStream_t s,
                              int shape, const Fuse<T> &F, const T *geo) {
  if (L.dim != 3 || shape < 0) return -1;
  switch (mode) {
    case kApplyA: return launch_col_mode<K, T, kApplyA, true>(L, u, p, yu, yp, s, shape, F, geo);
    case kApplyBT: return launch_col_mode<K, T, kApplyBT, true>(L, u, p, yu, yp, s, shape, F, geo);
    case kApplyB: return launch_col_mode<K, T, kApplyB, true>(L, u, p, yu, yp, s, shape, F, geo);
    case kApplyA | kApplyBT: return launch_col_mode<K, T, kApplyA | kApplyBT, true>(L, u, p, yu, yp, s, shape, F, geo);
    case kApplyA | kApplyBT | kApplyB:
      return launch_col_mode<K, T, kApplyA | kApplyBT | kApplyB, true>(L, u, p, yu, yp, s, shape, F, geo);
    default: return -1;
  }
}

// 3D: one launch per colour class of cells (fixed summation order at every node).
template <int DIM, int K, typename T, bool CART>
static int launch_diag_dim(const LevelDesc<T> &L, const Tab1D<T> *tab, T *dAs, T *dSloc, T *dMp, cudaStream_t s,
                           const T *rho, int sym) {
  using CS = CellShape<DIM, K>;
  if (DIM != 3) {
    stokes_cell_diagonals<DIM, K, T, CART><<<(unsigned)L.n_cells, CS::NP, 0, s>>>(L, tab, dAs, dSloc, dMp, rho, sym, -1);
    return 0;
  }
  for (int colour = 0; colour < 8; ++colour) {
    const long long cells = (long long)((L.n[0] - (colour & 1) + 1) / 2) * ((L.n[1] - ((colour >> 1) & 1) + 1) / 2) *
                            ((L.n[2] - ((colour >> 2) & 1) + 1) / 2);
    if (cells > 0)
      stokes_cell_diagonals<DIM, K, T, CART><<<(unsigned)cells, CS::NP, 0, s>>>(L, tab, dAs, dSloc, dMp, rho, sym,
                                                                                colour);
  }
  return 0;
}

template <int DIM, int K, typename T, bool CART>
static int launch_grad_dim(const LevelDesc<T> &L, const Tab1D<T> *tab, const T *u, const T *lam, T *g, cudaStream_t s) {
  using CS = CellShape<DIM, K>;
  const long long blocks = (L.n_cells + CS::CPB - 1) / CS::CPB;
  const size_t smem = sizeof(Tab1D<T>) + (size_t)CS::CPB * CS::PER_CELL * sizeof(T);
  launch_kernel(stokes_cell_grad_mu<DIM, K, T, CART>, dim3((unsigned)blocks), dim3(CS::THREADS), smem, s, L, tab, u,
                lam, g);
  return 0;
}

template <int K, typename T>
int launch_cell_grad_k(const LevelDesc<T> &L, const Tab1D<T> *tab, const T *u, const T *lam, T *g, cudaStream_t s) {
  if (L.dim == 3)
    return L.cartesian ? launch_grad_dim<3, K, T, true>(L, tab, u, lam, g, s)
                       : launch_grad_dim<3, K, T, false>(L, tab, u, lam, g, s);
  return L.cartesian ? launch_grad_dim<2, K, T, true>(L, tab, u, lam, g, s)
                     : launch_grad_dim<2, K, T, false>(L, tab, u, lam, g, s);
}

template <int K, typename T>
int launch_cell_diag_k(const LevelDesc<T> &L, const Tab1D<T> *tab, T *dAs, T *dSloc, T *dMp, cudaStream_t s,
                       const T *rho, int sym) {
  if (L.dim == 3)
    return L.cartesian ? launch_diag_dim<3, K, T, true>(L, tab, dAs, dSloc, dMp, s, rho, sym)
                       : launch_diag_dim<3, K, T, false>(L, tab, dAs, dSloc, dMp, s, rho, sym);
  return L.cartesian ? launch_diag_dim<2, K, T, true>(L, tab, dAs, dSloc, dMp, s, rho, sym)
                     : launch_diag_dim<2, K, T, false>(L, tab, dAs, dSloc, dMp, s, rho, sym);
}

}  // namespace smf

#define SMF_INSTANTIATE_K(KK)                                                                                  \
  namespace smf {                                                                                              \
  template int launch_cell_apply_k<KK, float>(const LevelDesc<float> &, const Tab1D<float> *, int,             \
                                               const float *, const float *, float *, float *, cudaStream_t,   \
                                               int, const float *, const float *);                                                           \
  template int launch_cell_apply_k<KK, double>(const LevelDesc<double> &, const Tab1D<double> *, int,          \
                                                const double *, const double *, double *, double *,            \
                                                cudaStream_t, int, const double *, const double *);                                             \
  template int launch_cell_apply_fused_k<KK, float>(const LevelDesc<float> &, int, const float *, const float *, \
                                                     float *, float *, cudaStream_t, int, const Fuse<float> &,       \
                                                     const float *);   \
  template int launch_cell_apply_fused_k<KK, double>(const LevelDesc<double> &, int, const double *,             \
                                                      const double *, double *, double *, cudaStream_t, int,       \
                                                      const Fuse<double> &, const double *);                                      \
  template int launch_cell_C_k<KK, float>(const LevelDesc<float> &, const Tab1D<float> *, float, float,        \
                                           const float *, float *, float, float *, const float *,            \
                                           cudaStream_t);                                                     \
  template int launch_cell_C_k<KK, double>(const LevelDesc<double> &, const Tab1D<double> *, double, double,   \
                                            const double *, double *, double, double *, const double *,      \
                                            cudaStream_t);                                                    \
  template int launch_cell_C_matrix_k<KK, double>(const LevelDesc<double> &, const Tab1D<double> *, double,     \
                                                   double, double *, cudaStream_t);                           \
  template int launch_col_geometry_k<KK, float>(const LevelDesc<float> &, float *, cudaStream_t);             \
  template int launch_col_geometry_k<KK, double>(const LevelDesc<double> &, double *, cudaStream_t);          \
  template int launch_cell_diag_k<KK, double>(const LevelDesc<double> &, const Tab1D<double> *, double *,      \
                                               double *, double *, cudaStream_t, const double *, int);         \
  template int upload_col_tables<KK>(const Tab1D<double> &, cudaStream_t);                                     \
  template int launch_cell_grad_k<KK, double>(const LevelDesc<double> &, const Tab1D<double> *, const double *,  \
                                               const double *, double *, cudaStream_t);                        \
  }
