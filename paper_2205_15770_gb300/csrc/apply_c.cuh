// Stabilisation block C of K = [A B^T; B -C]: per-cell quadrature, stored packed element
// matrices and their application.
#pragma once
#include "apply.cuh"

namespace smf {

// Stabilisation block C (K = [A B^T; B -C]; the paper leaves C open, Sec. 1):
//   c(p, q) = c_mass int p q + c_grad sum_tau h_tau^2 int_tau grad p . grad q,  h_tau = |tau|^(1/d).
// cell_C_local evaluates one cell: the pressure values and reference gradients at the (k+1)^d
// Gauss points by tensor-product evaluation, the metric G = w adj adj^T / det of point_geometry
// and the transposed evaluation, in one pass over the points (the mass and gradient parts are
// accumulated apart; h_tau^2 = (sum_q w det)^(2/d) scales the gradient part at the end).
// diag = false: acc = C_tau pn; diag = true: acc = diag(C_tau) (pn unused).
template <int DIM, int K, typename T, bool CART>
__device__ __forceinline__ void cell_C_local(const LevelDesc<T> &L, const Tab1D<T> *__restrict__ tab, T c_mass,
                                             T c_grad, int cx, int cy, int cz, const T *pn, bool diag, T *acc) {
  using CS = CellShape<DIM, K>;
  constexpr int NQ = CS::NQ, NPR = CS::NPR, NPP = CS::NPP, NPT = CS::NP, NVX = CS::NVERT;
  T verts[NVX * DIM];
  if (!CART) {
    for (int v = 0; v < NVX; ++v) {
      const long long gv = DIM == 3 ? ((long long)(cz + ((v >> 2) & 1)) * (L.n[1] + 1) + (cy + ((v >> 1) & 1))) *
                                              (L.n[0] + 1) + (cx + (v & 1))
                                    : (long long)(cy + ((v >> 1) & 1)) * (L.n[0] + 1) + (cx + (v & 1));
      for (int a = 0; a < DIM; ++a) verts[v * DIM + a] = L.vert[gv * DIM + a];
    }
  }
  T accg[NPP];
#pragma unroll
  for (int n = 0; n < NPP; ++n) acc[n] = accg[n] = T(0);
  T vol = T(0);
#pragma unroll 1
  for (int q = 0; q < NPT; ++q) {
    const int qd[3] = {q % NQ, (q / NQ) % NQ, DIM == 3 ? q / (NQ * NQ) : 0};
    PointGeo<DIM, T> g;
    point_geometry<DIM, K, T, CART>(L, tab->x, tab->w, verts, qd[0], qd[1], qd[2], g);
    vol += g.wdet;
    // basis values and reference gradients of the pressure nodes at this point
    T val[NPP], grd[NPP][DIM];
#pragma unroll
    for (int n = 0; n < NPP; ++n) {
      const int nd[3] = {n % NPR, (n / NPR) % NPR, DIM == 3 ? n / (NPR * NPR) : 0};
      T pv[3], pd[3];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        pv[a] = tab->Pv[qd[a] * NPR + nd[a]];
        pd[a] = tab->Pd[qd[a] * NPR + nd[a]];
      }
      val[n] = pv[0] * pv[1] * (DIM == 3 ? pv[2] : T(1));
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        T f = T(1);
#pragma unroll
        for (int b = 0; b < DIM; ++b) f *= (b == a ? pd[b] : pv[b]);
        grd[n][a] = f;
      }
    }
    const T cm = c_mass * g.wdet;
    if (diag) {
#pragma unroll
      for (int n = 0; n < NPP; ++n) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
          for (int b = 0; b < DIM; ++b) s += grd[n][a] * g.G[a * DIM + b] * grd[n][b];
        acc[n] += cm * val[n] * val[n];
        accg[n] += s;
      }
    } else {
      T pq = T(0), gr[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) gr[a] = T(0);
#pragma unroll
      for (int n = 0; n < NPP; ++n) {
        pq += val[n] * pn[n];
#pragma unroll
        for (int a = 0; a < DIM; ++a) gr[a] += grd[n][a] * pn[n];
      }
      T flux[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < DIM; ++b) s += g.G[a * DIM + b] * gr[b];
        flux[a] = s;
      }
      const T mq = cm * pq;
#pragma unroll
      for (int n = 0; n < NPP; ++n) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) s += grd[n][a] * flux[a];
        acc[n] += val[n] * mq;
        accg[n] += s;
      }
    }
  }
  const T cg = c_grad * (DIM == 3 ? pow(vol, T(2) / T(3)) : vol);
#pragma unroll
  for (int n = 0; n < NPP; ++n) acc[n] += cg * accg[n];
}

template <int DIM, int K, typename T>
__device__ __forceinline__ long long pressure_node(const LevelDesc<T> &L, int cx, int cy, int cz, int n) {
  constexpr int NPR = CellShape<DIM, K>::NPR;
  const int nx = n % NPR, ny = (n / NPR) % NPR, nz = DIM == 3 ? n / (NPR * NPR) : 0;
  return lattice_index<DIM, T>(L.Pn, (K - 1) * cx + nx, (K - 1) * cy + ny, (K - 1) * cz + nz);
}

template <int DIM, typename T>
__device__ __forceinline__ void cell_coords(const LevelDesc<T> &L, long long cell, int &cx, int &cy, int &cz) {
  cx = (int)(cell % L.n[0]);
  const long long r = cell / L.n[0];
  cy = (int)(r % L.n[1]);
  cz = DIM == 3 ? (int)(r / L.n[1]) : 0;
}

// Matrix-free application, one thread per cell.  Apply (diag == null): yp += sign * C p.
// Diagonal (diag != null): diag += diag(C).
template <int DIM, int K, typename T, bool CART>
__global__ void stokes_cell_apply_C(const LevelDesc<T> L, const Tab1D<T> *__restrict__ tab, T c_mass, T c_grad,
                                    const T *__restrict__ p, T *__restrict__ yp, T sign, T *__restrict__ diag) {
  pdl_enter();
  constexpr int NPP = CellShape<DIM, K>::NPP;
  for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < L.n_cells;
       cell += (long long)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    cell_coords<DIM, T>(L, cell, cx, cy, cz);
    T pn[NPP], acc[NPP];
#pragma unroll
    for (int n = 0; n < NPP; ++n) pn[n] = diag ? T(0) : p[pressure_node<DIM, K, T>(L, cx, cy, cz, n)];
    cell_C_local<DIM, K, T, CART>(L, tab, c_mass, c_grad, cx, cy, cz, pn, diag != nullptr, acc);
#pragma unroll
    for (int n = 0; n < NPP; ++n) {
      const long long i = pressure_node<DIM, K, T>(L, cx, cy, cz, n);
      if (diag)
        atomicAdd(&diag[i], acc[n]);
      else
        atomicAdd(&yp[i], sign * acc[n]);
    }
  }
}

// Element matrices of C for the low-order pressure spaces (setup, once per level): entry (n, m)
// with n <= m of cell c at Ce[(m (m + 1) / 2 + n) * n_cells + c] (packed upper triangle, one
// plane per entry so that consecutive cells are consecutive in memory).  Thread per (m, cell):
// column m = C_tau e_m by cell_C_local.
template <int DIM, int K, typename T, bool CART>
__global__ void stokes_cell_C_matrix(const LevelDesc<T> L, const Tab1D<T> *__restrict__ tab, T c_mass, T c_grad,
                                     T *__restrict__ Ce) {
  pdl_enter();
  constexpr int NPP = CellShape<DIM, K>::NPP;
  const long long total = L.n_cells * NPP;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(idx / L.n_cells);
    const long long cell = idx % L.n_cells;
    int cx, cy, cz;
    cell_coords<DIM, T>(L, cell, cx, cy, cz);
    T pn[NPP], acc[NPP];
#pragma unroll
    for (int n = 0; n < NPP; ++n) pn[n] = n == m ? T(1) : T(0);
    cell_C_local<DIM, K, T, CART>(L, tab, c_mass, c_grad, cx, cy, cz, pn, false, acc);
#pragma unroll
    for (int n = 0; n < NPP; ++n)
      if (n <= m) Ce[((long long)m * (m + 1) / 2 + n) * L.n_cells + cell] = acc[n];
  }
}

// yp += sign * C p from the stored element matrices: one thread per cell gathers its NPP
// pressure values, multiplies by the packed symmetric matrix (coalesced entry planes) and
// scatters atomically.
template <int DIM, int K, typename T>
__global__ void stokes_cell_apply_C_mat(const LevelDesc<T> L, const T *__restrict__ Ce, const T *__restrict__ p,
                                        T *__restrict__ yp, T sign) {
  pdl_enter();
  constexpr int NPP = CellShape<DIM, K>::NPP;
  for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < L.n_cells;
       cell += (long long)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    cell_coords<DIM, T>(L, cell, cx, cy, cz);
    T pn[NPP], acc[NPP];
#pragma unroll
    for (int n = 0; n < NPP; ++n) {
      pn[n] = p[pressure_node<DIM, K, T>(L, cx, cy, cz, n)];
      acc[n] = T(0);
    }
#pragma unroll
    for (int m = 0; m < NPP; ++m)
#pragma unroll
      for (int n = 0; n <= m; ++n) {
        const T e = Ce[(long long)(m * (m + 1) / 2 + n) * L.n_cells + cell];
        acc[n] += e * pn[m];
        if (n != m) acc[m] += e * pn[n];
      }
#pragma unroll
    for (int n = 0; n < NPP; ++n) atomicAdd(&yp[pressure_node<DIM, K, T>(L, cx, cy, cz, n)], sign * acc[n]);
  }
}

}  // namespace smf
