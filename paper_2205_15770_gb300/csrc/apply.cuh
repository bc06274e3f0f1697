// Matrix-free cell kernels of the Taylor-Hood Stokes operator by sum factorisation.
//
// Paper Sec. 3.1: K x = sum_tau P_tau K_tau P_tau^T x with the element action evaluated
// on the reference cell through the tensor-product structure of the Q_k / Q_{k-1}
// shape functions (sum factorisation).  Per cell:
//   gather   u_c (k+1)^d nodal values per component, p k^d values   (P_tau^T x)
//   forward  values at the (k+1)^d Gauss points by d 1D interpolation sweeps, then
//            reference gradients by d 1D collocation-derivative sweeps
//   point    fluxes  mu * w adj(J) adj(J)^T / det J * grad_ref u_c - p * w adj(J) e_c
//            mass    gamma*rho * w det J * u_c,  pressure test  -w sum_c adj(J) e_c . grad_ref u_c
//   backward transposed sweeps, scatter-add into y                    (P_tau)
// J is the Jacobian of the bi/trilinear cell map (from the cell's 2^d vertices, or a
// constant diagonal for Cartesian meshes), adj(J) = det(J) J^{-1}, w the Gauss weight.
//
// Launch shape: one thread per point of a cell ((k+1)^d threads), CPB cells per CTA,
// 1D sweeps through shared memory between __syncthreads(); scatter by atomicAdd.
#pragma once
#include "common.cuh"

namespace smf {

template <int DIM, int K>
struct CellShape {
  static constexpr int NQ = K + 1;   // Gauss points per direction
  static constexpr int NV = K + 1;   // velocity nodes per direction
  static constexpr int NPR = K;      // pressure nodes per direction
  static constexpr int NP = ipow(NQ, DIM);
  static constexpr int NPP = ipow(NPR, DIM);
  static constexpr int NVERT = ipow(2, DIM);
  static constexpr int CPB = DIM == 3 ? (K == 2 ? 8 : (K == 3 ? 4 : 2)) : (K == 2 ? 16 : (K == 3 ? 16 : 8));
  static constexpr int THREADS = CPB * NP;
  static constexpr int BUFS = DIM == 3 ? 5 : 4;                // A, B, FX, FY(, FZ)
  static constexpr int PER_CELL = BUFS * NP + NVERT * DIM;     // T values of shared memory per cell
};

// One output of a 1D contraction along DIR for a cell tensor.  Output extents (E0,E1,E2),
// input extent NI along DIR (others as the output).  TR = false: out = sum_m M[id*LD+m] in_m;
// TR = true: out = sum_m M[m*LD+id] in_m.
template <int DIR, int E0, int E1, int E2, int NI, int LD, bool TR, typename T>
__device__ __forceinline__ T contract(int t, const T *in, const T *M) {
  const int i0 = t % E0;
  const int i1 = (t / E0) % E1;
  const int i2 = t / (E0 * E1);
  constexpr int I0 = DIR == 0 ? NI : E0;
  constexpr int I1 = DIR == 1 ? NI : E1;
  int base, id;
  constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? I0 : I0 * I1);
  if (DIR == 0) {
    base = (i2 * I1 + i1) * I0;
    id = i0;
  } else if (DIR == 1) {
    base = i2 * I1 * I0 + i0;
    id = i1;
  } else {
    base = i1 * I0 + i0;
    id = i2;
  }
  T s = T(0);
#pragma unroll
  for (int m = 0; m < NI; ++m) s += (TR ? M[m * LD + id] : M[id * LD + m]) * in[base + m * stride];
  return s;
}

// Geometry of one Gauss point: G = w adj adj^T / det (symmetric, row-major DIMxDIM),
// C = w adj (row-major), wdet = w det J.
template <int DIM, typename T>
struct PointGeo {
  T G[DIM * DIM];
  T C[DIM * DIM];
  T wdet;
};

template <int DIM, int K, typename T, bool CART>
__device__ __forceinline__ void point_geometry(const LevelDesc<T> &L, const T *tab_x, const T *tab_w,
                                               const T *verts, int qx, int qy, int qz, PointGeo<DIM, T> &g) {
  T wq = tab_w[qx] * tab_w[qy];
  if (DIM == 3) wq *= tab_w[qz];
  T J[DIM][DIM];
  if (CART) {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) J[a][b] = a == b ? L.h[a] : T(0);
  } else {
    const T xi[3] = {tab_x[qx], tab_x[qy], DIM == 3 ? tab_x[qz] : T(0)};
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) J[a][b] = T(0);
#pragma unroll
    for (int v = 0; v < (1 << DIM); ++v) {
      const int vb[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
      T nv[3], dv[3];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        nv[d] = vb[d] ? xi[d] : T(1) - xi[d];
        dv[d] = vb[d] ? T(1) : T(-1);
      }
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        T f = T(1);
#pragma unroll
        for (int d = 0; d < DIM; ++d) f *= (d == b ? dv[d] : nv[d]);
#pragma unroll
        for (int a = 0; a < DIM; ++a) J[a][b] += verts[v * DIM + a] * f;
      }
    }
  }
  T adj[DIM][DIM];
  T det;
  if (DIM == 2) {
    adj[0][0] = J[1][1];
    adj[0][1] = -J[0][1];
    adj[1][0] = -J[1][0];
    adj[1][1] = J[0][0];
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  } else {
    adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  }
  const T wdiv = wq / det;
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      T s = T(0);
#pragma unroll
      for (int c = 0; c < DIM; ++c) s += adj[a][c] * adj[b][c];
      g.G[a * DIM + b] = wdiv * s;
      g.C[a * DIM + b] = wq * adj[a][b];
    }
  g.wdet = wq * det;
}

template <int DIM, typename T>
__device__ __forceinline__ long long lattice_index(const int N[3], int gx, int gy, int gz) {
  return DIM == 3 ? ((long long)gz * N[1] + gy) * N[0] + gx : (long long)gy * N[0] + gx;
}

// Load the 1D tables into shared memory (S, D, Pv, x, w).
template <typename T>
__device__ __forceinline__ void load_tables(const Tab1D<T> *tab, T *sm) {
  const T *src = reinterpret_cast<const T *>(tab);
  constexpr int n = sizeof(Tab1D<T>) / sizeof(T);
  for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = src[i];
}

template <int DIM, int K, typename T, bool CART>
__global__ void __launch_bounds__(CellShape<DIM, K>::THREADS)
    stokes_cell_apply(const LevelDesc<T> L, const Tab1D<T> *__restrict__ tab, const int mode,
                      const T *__restrict__ u, const T *__restrict__ p, T *__restrict__ yu,
                      T *__restrict__ yp, const T *__restrict__ rho_cell) {
  pdl_enter();
  using CS = CellShape<DIM, K>;
  constexpr int NQ = CS::NQ, NV = CS::NV, NPR = CS::NPR, NP = CS::NP, NPP = CS::NPP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  Tab1D<T> *st = reinterpret_cast<Tab1D<T> *>(sm);
  T *cellmem = sm + sizeof(Tab1D<T>) / sizeof(T);

  const int lc = threadIdx.x / NP;
  const int t = threadIdx.x - lc * NP;
  const long long cell = (long long)blockIdx.x * CS::CPB + lc;
  const bool valid = cell < L.n_cells;
  T *bufA = cellmem + lc * CS::PER_CELL;
  T *bufB = bufA + NP;
  T *FX = bufB + NP;
  T *FY = FX + NP;
  T *FZ = FY + NP;  // only used in 3D (BUFS = 5)
  T *verts = bufA + CS::BUFS * NP;

  int cx = 0, cy = 0, cz = 0;
  if (valid) {
    cx = (int)(cell % L.n[0]);
    long long r = cell / L.n[0];
    cy = (int)(r % L.n[1]);
    cz = (int)(r / L.n[1]);
  }
  load_tables(tab, sm);
  if (!CART && t < CS::NVERT * DIM) {
    const int v = t / DIM, a = t - (t / DIM) * DIM;
    const int vx = v & 1, vy = (v >> 1) & 1, vz = (v >> 2) & 1;
    long long gv = DIM == 3 ? ((long long)(cz + vz) * (L.n[1] + 1) + (cy + vy)) * (L.n[0] + 1) + (cx + vx)
                            : (long long)(cy + vy) * (L.n[0] + 1) + (cx + vx);
    verts[t] = valid ? L.vert[gv * DIM + a] : T(0);
  }
  __syncthreads();

  const int qx = t % NQ;
  const int qy = (t / NQ) % NQ;
  const int qz = DIM == 3 ? t / (NQ * NQ) : 0;
  PointGeo<DIM, T> g;
  point_geometry<DIM, K, T, CART>(L, st->x, st->w, verts, qx, qy, qz, g);
  const T mu = L.mu_cell ? (valid ? L.mu_cell[cell] : T(0)) : L.mu;
  // gamma rho of the cell (rho per cell when given, else 1)
  const T grho = L.gamma_rho * (rho_cell ? (valid ? rho_cell[cell] : T(0)) : T(1));

  const bool needP = mode & kApplyBT;
  const bool massOp = mode & (kApplyMass | kApplyMassAll);
  const bool needU = (mode & (kApplyA | kApplyB)) || massOp;
  const bool outU = (mode & (kApplyA | kApplyBT)) || massOp;
  const bool outP = mode & kApplyB;

  // ---- pressure at the Gauss points ------------------------------------------------
  T pq = T(0);
  if (needP) {
    if (t < NPP) {
      const int ix = t % NPR, iy = (t / NPR) % NPR, iz = DIM == 3 ? t / (NPR * NPR) : 0;
      const long long gi = lattice_index<DIM, T>(L.Pn, (K - 1) * cx + ix, (K - 1) * cy + iy, (K - 1) * cz + iz);
      bufA[t] = valid ? p[gi] : T(0);
    }
    __syncthreads();
    if (DIM == 3) {
      if (t < NQ * NPR * NPR) bufB[t] = contract<0, NQ, NPR, NPR, NPR, NPR, false>(t, bufA, st->Pv);
      __syncthreads();
      if (t < NQ * NQ * NPR) bufA[t] = contract<1, NQ, NQ, NPR, NPR, NPR, false>(t, bufB, st->Pv);
      __syncthreads();
      pq = contract<2, NQ, NQ, NQ, NPR, NPR, false>(t, bufA, st->Pv);
    } else {
      if (t < NQ * NPR) bufB[t] = contract<0, NQ, NPR, 1, NPR, NPR, false>(t, bufA, st->Pv);
      __syncthreads();
      pq = contract<1, NQ, NQ, 1, NPR, NPR, false>(t, bufB, st->Pv);
    }
    __syncthreads();
  }

  // ---- velocity components -------------------------------------------------------------
  const int ix = t % NV, iy = (t / NV) % NV, iz = DIM == 3 ? t / (NV * NV) : 0;
  const int gx = K * cx + ix, gy = K * cy + iy, gz = K * cz + iz;
  const long long vidx = lattice_index<DIM, T>(L.N, gx, gy, gz);
  const bool vfree = valid && !vel_constrained(L.N, L.faces, DIM, gx, gy, gz);
  // forward sweeps of component c: value and reference gradient at this thread's Gauss point
  auto forward = [&](int c, T &uq, T (&gr)[3]) {
    // b = Z M_v f reads every node of f (boundary values couple into free rows); its transpose
    // M_v Z reads the free nodes only and writes every row
    bufA[t] = ((mode & (kApplyMass | kApplyUnmasked)) ? valid : vfree) ? u[c * L.nv + vidx] : T(0);
    __syncthreads();
    if (DIM == 3) {
      bufB[t] = contract<0, NQ, NV, NV, NV, NV, false>(t, bufA, st->S);
      __syncthreads();
      bufA[t] = contract<1, NQ, NQ, NV, NV, NV, false>(t, bufB, st->S);
      __syncthreads();
      bufB[t] = contract<2, NQ, NQ, NQ, NV, NV, false>(t, bufA, st->S);
      __syncthreads();
      uq = bufB[t];
      gr[0] = contract<0, NQ, NQ, NQ, NQ, NQ, false>(t, bufB, st->D);
      gr[1] = contract<1, NQ, NQ, NQ, NQ, NQ, false>(t, bufB, st->D);
      gr[2] = contract<2, NQ, NQ, NQ, NQ, NQ, false>(t, bufB, st->D);
    } else {
      bufB[t] = contract<0, NQ, NV, 1, NV, NV, false>(t, bufA, st->S);
      __syncthreads();
      bufA[t] = contract<1, NQ, NQ, 1, NV, NV, false>(t, bufB, st->S);
      __syncthreads();
      uq = bufA[t];
      gr[0] = contract<0, NQ, NQ, 1, NQ, NQ, false>(t, bufA, st->D);
      gr[1] = contract<1, NQ, NQ, 1, NQ, NQ, false>(t, bufA, st->D);
    }
  };
  // transposed sweeps of the reference fluxes f and the value term mv, scattered into component c
  auto backward = [&](int c, const T (&f)[3], T mv) {
    FX[t] = f[0];
    FY[t] = f[1];
    if (DIM == 3) FZ[t] = f[2];
    __syncthreads();
    T tq = mv + contract<0, NQ, NQ, (DIM == 3 ? NQ : 1), NQ, NQ, true>(t, FX, st->D) +
           contract<1, NQ, NQ, (DIM == 3 ? NQ : 1), NQ, NQ, true>(t, FY, st->D);
    if (DIM == 3) tq += contract<2, NQ, NQ, NQ, NQ, NQ, true>(t, FZ, st->D);
    bufA[t] = tq;
    __syncthreads();
    T val;
    if (DIM == 3) {
      bufB[t] = contract<2, NQ, NQ, NV, NQ, NV, true>(t, bufA, st->S);
      __syncthreads();
      bufA[t] = contract<1, NQ, NV, NV, NQ, NV, true>(t, bufB, st->S);
      __syncthreads();
      val = contract<0, NV, NV, NV, NQ, NV, true>(t, bufA, st->S);
    } else {
      bufB[t] = contract<1, NQ, NV, 1, NQ, NV, true>(t, bufA, st->S);
      __syncthreads();
      val = contract<0, NV, NV, 1, NQ, NV, true>(t, bufB, st->S);
    }
    if ((mode & kApplyMassAll) ? valid : vfree) atomicAdd(&yu[c * L.nv + vidx], val);
  };
  T qacc = T(0);
  if ((mode & kApplySym) && (mode & kApplyA)) {
    // symmetric-gradient form (Sec. 2): the flux of test component c is mu eps(u)_{c.}, which
    // needs the gradients of every component at the point.  Physical gradients from reference
    // ones: grad_x u_c = adj^T grad u_c / det = (w adj)^T grad u_c / (w det).
    T gq[3][3] = {}, uqa[3] = {};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      forward(c, uqa[c], gq[c]);
      if (outP) {
#pragma unroll
        for (int b = 0; b < DIM; ++b) qacc -= g.C[b * DIM + c] * gq[c][b];
      }
      __syncthreads();
    }
    T gp[3][3];
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) s += g.C[a * DIM + b] * gq[c][a];
        gp[c][b] = s / g.wdet;
      }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      T f[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < DIM; ++b) s += g.C[a * DIM + b] * (T(0.5) * (gp[c][b] + gp[b][c]));
        f[a] = mu * s;
      }
      if (mode & kApplyBT) {
#pragma unroll
        for (int b = 0; b < DIM; ++b) f[b] -= pq * g.C[b * DIM + c];
      }
      backward(c, f, grho * g.wdet * uqa[c]);
      __syncthreads();
    }
  } else {
#pragma unroll 1
    for (int c = 0; c < DIM; ++c) {
      T gr[3] = {T(0), T(0), T(0)};
      T uq = T(0);
      if (needU) forward(c, uq, gr);
      if (outP) {
#pragma unroll
        for (int b = 0; b < DIM; ++b) qacc -= g.C[b * DIM + c] * gr[b];
      }
      if (outU) {
        T f[3] = {T(0), T(0), T(0)};
        T mv = T(0);
        if (mode & kApplyA) {
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < DIM; ++b) s += g.G[a * DIM + b] * gr[b];
            f[a] = mu * s;
          }
          mv = grho * g.wdet * uq;
        }
        if (massOp) mv += g.wdet * uq;
        if (mode & kApplyBT) {
#pragma unroll
          for (int b = 0; b < DIM; ++b) f[b] -= pq * g.C[b * DIM + c];
        }
        backward(c, f, mv);
      }
      __syncthreads();
    }
  }

  // ---- pressure test functions ----------------------------------------------------------
  if (outP) {
    bufA[t] = qacc;
    __syncthreads();
    T val = T(0);
    if (DIM == 3) {
      if (t < NQ * NQ * NPR) bufB[t] = contract<2, NQ, NQ, NPR, NQ, NPR, true>(t, bufA, st->Pv);
      __syncthreads();
      if (t < NQ * NPR * NPR) bufA[t] = contract<1, NQ, NPR, NPR, NQ, NPR, true>(t, bufB, st->Pv);
      __syncthreads();
      if (t < NPP) val = contract<0, NPR, NPR, NPR, NQ, NPR, true>(t, bufA, st->Pv);
    } else {
      if (t < NQ * NPR) bufB[t] = contract<1, NQ, NPR, 1, NQ, NPR, true>(t, bufA, st->Pv);
      __syncthreads();
      if (t < NPP) val = contract<0, NPR, NPR, 1, NQ, NPR, true>(t, bufB, st->Pv);
    }
    if (valid && t < NPP) {
      const int px = t % NPR, py = (t / NPR) % NPR, pz = DIM == 3 ? t / (NPR * NPR) : 0;
      const long long gi = lattice_index<DIM, T>(L.Pn, (K - 1) * cx + px, (K - 1) * cy + py, (K - 1) * cz + pz);
      atomicAdd(&yp[gi], val);
    }
  }
}

// Setup kernel, one cell per CTA, (k+1)^d threads:
//   dAs[node]  += (A_tau)_jj        scalar velocity block diagonal (same for every component);
//                                   symmetric form (sym): dAs[c nv + node] per component c
//   dSloc[i]   += sum_{c, j free} (B_tau)_{i,(c,j)}^2 / (A_tau)_jj   (Eq. diag loc)
//   dMp[i]     += (M_p,tau)_ii      pressure mass diagonal (Eq. diag p)
// colour >= 0 (3D): one launch per class of cells with the same index parities (bit a = parity
// along axis a), the blocks taking that class's cells; no two cells of a class share a node, so a
// node's entries are added in class order and the diagonals are bitwise reproducible (the local
// Schur sum inside a cell is then also added in a fixed order where it fits in shared memory).
template <int DIM, int K, typename T, bool CART>
__global__ void stokes_cell_diagonals(const LevelDesc<T> L, const Tab1D<T> *__restrict__ tab, T *dAs, T *dSloc,
                                      T *dMp, const T *__restrict__ rho_cell, int sym, int colour) {
  using CS = CellShape<DIM, K>;
  constexpr int NQ = CS::NQ, NV = CS::NV, NPR = CS::NPR, NP = CS::NP, NPP = CS::NPP;
  constexpr bool ORDERED = NP * NPP <= 2048;
  __shared__ Tab1D<T> st;
  __shared__ T sG[NP][DIM * DIM];
  __shared__ T sC[NP][DIM * DIM];
  __shared__ T sW[NP];
  __shared__ T sAjj[NP];
  __shared__ T sLoc[NPP];
  __shared__ T sPart[ORDERED ? NP : 1][ORDERED ? NPP : 1];
  __shared__ T verts[CS::NVERT * DIM];
  const int t = threadIdx.x;
  int cx, cy, cz;
  long long cell;
  if (colour < 0) {
    cell = blockIdx.x;
    cx = (int)(cell % L.n[0]);
    cy = (int)((cell / L.n[0]) % L.n[1]);
    cz = (int)(cell / ((long long)L.n[0] * L.n[1]));
  } else {
    const int px = colour & 1, py = (colour >> 1) & 1, pz = (colour >> 2) & 1;
    const long long ex = (L.n[0] - px + 1) / 2, ey = (L.n[1] - py + 1) / 2;
    const long long k = blockIdx.x;
    cx = 2 * (int)(k % ex) + px;
    cy = 2 * (int)((k / ex) % ey) + py;
    cz = 2 * (int)(k / (ex * ey)) + pz;
    cell = ((long long)cz * L.n[1] + cy) * L.n[0] + cx;
  }
  load_tables(tab, reinterpret_cast<T *>(&st));
  if (!CART && t < CS::NVERT * DIM) {
    const int v = t / DIM, a = t % DIM;
    const int vx = v & 1, vy = (v >> 1) & 1, vz = (v >> 2) & 1;
    long long gv = DIM == 3 ? ((long long)(cz + vz) * (L.n[1] + 1) + (cy + vy)) * (L.n[0] + 1) + (cx + vx)
                            : (long long)(cy + vy) * (L.n[0] + 1) + (cx + vx);
    verts[t] = L.vert[gv * DIM + a];
  }
  if (t < NPP) sLoc[t] = T(0);
  __syncthreads();
  const T mu = L.mu_cell ? L.mu_cell[cell] : L.mu;
  {
    const int qx = t % NQ, qy = (t / NQ) % NQ, qz = DIM == 3 ? t / (NQ * NQ) : 0;
    PointGeo<DIM, T> g;
    point_geometry<DIM, K, T, CART>(L, st.x, st.w, verts, qx, qy, qz, g);
#pragma unroll
    for (int i = 0; i < DIM * DIM; ++i) {
      sG[t][i] = mu * g.G[i];
      sC[t][i] = g.C[i];
    }
    sW[t] = g.wdet;
  }
  __syncthreads();
  // velocity node j = t
  const int jx = t % NV, jy = (t / NV) % NV, jz = DIM == 3 ? t / (NV * NV) : 0;
  auto grad_phi = [&](int q, T gr[3], T &val) {
    const int qx = q % NQ, qy = (q / NQ) % NQ, qz = DIM == 3 ? q / (NQ * NQ) : 0;
    const T sx = st.S[qx * NV + jx], sy = st.S[qy * NV + jy], sz = DIM == 3 ? st.S[qz * NV + jz] : T(1);
    const T dx = st.Sd[qx * NV + jx], dy = st.Sd[qy * NV + jy], dz = DIM == 3 ? st.Sd[qz * NV + jz] : T(0);
    gr[0] = dx * sy * sz;
    gr[1] = sx * dy * sz;
    gr[2] = sx * sy * dz;
    val = sx * sy * sz;
  };
  const T grho = L.gamma_rho * (rho_cell ? rho_cell[cell] : T(1));
  // Laplacian form: the same diagonal for every component; symmetric form:
  // mu (1/2 grad phi . grad phi + 1/2 (d_c phi)^2) + gamma rho phi^2 for component c, with
  // d_c phi = (w adj^T grad phi)_c / (w det)
  T ajjc[3] = {T(0), T(0), T(0)};
  for (int q = 0; q < NP; ++q) {
    T gr[3], val;
    grad_phi(q, gr, val);
    T s = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) s += gr[a] * sG[q][a * DIM + b] * gr[b];
    const T m = grho * sW[q] * val * val;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      if (sym) {
        T dc = T(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) dc += sC[q][a * DIM + c] * gr[a];
        ajjc[c] += T(0.5) * s + T(0.5) * mu * dc * dc / sW[q] + m;
      } else {
        ajjc[c] += s + m;
      }
    }
  }
  const T ajj = ajjc[0];
  sAjj[t] = ajj;
  const int gx = K * cx + jx, gy = K * cy + jy, gz = K * cz + jz;
  const bool jfree = !vel_constrained(L.N, L.faces, DIM, gx, gy, gz);
  if (jfree) {
    const long long node = lattice_index<DIM, T>(L.N, gx, gy, gz);
    if (sym) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) atomicAdd(&dAs[c * L.nv + node], ajjc[c]);
    } else {
      atomicAdd(&dAs[node], ajj);
    }
  }
  // local Schur diagonal: columns (c, j = t) of B_tau
  if (ORDERED) {
#pragma unroll
    for (int i = 0; i < NPP; ++i) sPart[ORDERED ? t : 0][ORDERED ? i : 0] = T(0);
  }
  if (jfree) {
    for (int c = 0; c < DIM; ++c) {
      T bcol[NPP];
#pragma unroll
      for (int i = 0; i < NPP; ++i) bcol[i] = T(0);
      for (int q = 0; q < NP; ++q) {
        T gr[3], val;
        grad_phi(q, gr, val);
        T f = T(0);
#pragma unroll
        for (int b = 0; b < DIM; ++b) f += sC[q][b * DIM + c] * gr[b];
        const int qx = q % NQ, qy = (q / NQ) % NQ, qz = DIM == 3 ? q / (NQ * NQ) : 0;
#pragma unroll
        for (int i = 0; i < NPP; ++i) {
          const int px = i % NPR, py = (i / NPR) % NPR, pz = DIM == 3 ? i / (NPR * NPR) : 0;
          T psi = st.Pv[qx * NPR + px] * st.Pv[qy * NPR + py];
          if (DIM == 3) psi *= st.Pv[qz * NPR + pz];
          bcol[i] -= psi * f;
        }
      }
      const T ac = sym ? (c == 0 ? ajjc[0] : (c == 1 ? ajjc[1] : ajjc[2])) : ajj;
      if (ORDERED) {
#pragma unroll
        for (int i = 0; i < NPP; ++i) sPart[ORDERED ? t : 0][ORDERED ? i : 0] += bcol[i] * bcol[i] / ac;
      } else {
#pragma unroll
        for (int i = 0; i < NPP; ++i) atomicAdd(&sLoc[i], bcol[i] * bcol[i] / ac);
      }
    }
  }
  __syncthreads();
  if (ORDERED && t < NPP) {
    T sum = T(0);
    for (int j = 0; j < NP; ++j) sum += sPart[ORDERED ? j : 0][ORDERED ? t : 0];
    sLoc[t] = sum;
  }
  __syncthreads();
  if (t < NPP) {
    const int px = t % NPR, py = (t / NPR) % NPR, pz = DIM == 3 ? t / (NPR * NPR) : 0;
    T mp = T(0);
    for (int q = 0; q < NP; ++q) {
      const int qx = q % NQ, qy = (q / NQ) % NQ, qz = DIM == 3 ? q / (NQ * NQ) : 0;
      T psi = st.Pv[qx * NPR + px] * st.Pv[qy * NPR + py];
      if (DIM == 3) psi *= st.Pv[qz * NPR + pz];
      mp += sW[q] * psi * psi;
    }
    const long long gi = lattice_index<DIM, T>(L.Pn, (K - 1) * cx + px, (K - 1) * cy + py, (K - 1) * cz + pz);
    atomicAdd(&dSloc[gi], sLoc[t]);
    atomicAdd(&dMp[gi], mp);
  }
}

}  // namespace smf

namespace smf {

// Per-cell viscosity gradient of the adjoint method (no counterpart in the paper; the paper
// has constant mu): with K(mu) x = b and K lambda = dJ/dx,
//   dJ/dmu_c = -lambda^T (dK/dmu_c) x = - sum_comp int_c grad lambda_comp . grad u_comp dx,
// evaluated by the same sum-factorised gradients as the operator (w adj adj^T / det at each
// Gauss point).  Constrained velocity DoFs read as 0 (the identity rows of K do not depend on
// mu).  One value per cell, no scatter.
template <int DIM, int K, typename T, bool CART>
__global__ void __launch_bounds__(CellShape<DIM, K>::THREADS)
    stokes_cell_grad_mu(const LevelDesc<T> L, const Tab1D<T> *__restrict__ tab, const T *__restrict__ u,
                        const T *__restrict__ lam, T *__restrict__ g_out) {
  pdl_enter();
  using CS = CellShape<DIM, K>;
  constexpr int NQ = CS::NQ, NV = CS::NV, NP = CS::NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  Tab1D<T> *st = reinterpret_cast<Tab1D<T> *>(sm);
  T *cellmem = sm + sizeof(Tab1D<T>) / sizeof(T);
  const int lc = threadIdx.x / NP;
  const int t = threadIdx.x - lc * NP;
  const long long cell = (long long)blockIdx.x * CS::CPB + lc;
  const bool valid = cell < L.n_cells;
  T *bufA = cellmem + lc * CS::PER_CELL;
  T *bufB = bufA + NP;
  T *verts = bufA + CS::BUFS * NP;
  int cx = 0, cy = 0, cz = 0;
  if (valid) {
    cx = (int)(cell % L.n[0]);
    const long long r = cell / L.n[0];
    cy = (int)(r % L.n[1]);
    cz = (int)(r / L.n[1]);
  }
  load_tables(tab, sm);
  if (!CART && t < CS::NVERT * DIM) {
    const int v = t / DIM, a = t - (t / DIM) * DIM;
    const int vx = v & 1, vy = (v >> 1) & 1, vz = (v >> 2) & 1;
    long long gv = DIM == 3 ? ((long long)(cz + vz) * (L.n[1] + 1) + (cy + vy)) * (L.n[0] + 1) + (cx + vx)
                            : (long long)(cy + vy) * (L.n[0] + 1) + (cx + vx);
    verts[t] = valid ? L.vert[gv * DIM + a] : T(0);
  }
  __syncthreads();
  const int qx = t % NQ, qy = (t / NQ) % NQ, qz = DIM == 3 ? t / (NQ * NQ) : 0;
  PointGeo<DIM, T> geo;
  point_geometry<DIM, K, T, CART>(L, st->x, st->w, verts, qx, qy, qz, geo);
  const int ix = t % NV, iy = (t / NV) % NV, iz = DIM == 3 ? t / (NV * NV) : 0;
  const int gx = K * cx + ix, gy = K * cy + iy, gz = K * cz + iz;
  const long long vidx = lattice_index<DIM, T>(L.N, gx, gy, gz);
  const bool vfree = valid && !vel_constrained(L.N, L.faces, DIM, gx, gy, gz);
  T acc = T(0);
  for (int c = 0; c < DIM; ++c) {
    T gr[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
    for (int f = 0; f < 2; ++f) {
      const T *src = f == 0 ? u : lam;
      bufA[t] = vfree ? src[c * L.nv + vidx] : T(0);
      __syncthreads();
      if (DIM == 3) {
        bufB[t] = contract<0, NQ, NV, NV, NV, NV, false>(t, bufA, st->S);
        __syncthreads();
        bufA[t] = contract<1, NQ, NQ, NV, NV, NV, false>(t, bufB, st->S);
        __syncthreads();
        bufB[t] = contract<2, NQ, NQ, NQ, NV, NV, false>(t, bufA, st->S);
        __syncthreads();
        gr[f][0] = contract<0, NQ, NQ, NQ, NQ, NQ, false>(t, bufB, st->D);
        gr[f][1] = contract<1, NQ, NQ, NQ, NQ, NQ, false>(t, bufB, st->D);
        gr[f][2] = contract<2, NQ, NQ, NQ, NQ, NQ, false>(t, bufB, st->D);
      } else {
        bufB[t] = contract<0, NQ, NV, 1, NV, NV, false>(t, bufA, st->S);
        __syncthreads();
        bufA[t] = contract<1, NQ, NQ, 1, NV, NV, false>(t, bufB, st->S);
        __syncthreads();
        gr[f][0] = contract<0, NQ, NQ, 1, NQ, NQ, false>(t, bufA, st->D);
        gr[f][1] = contract<1, NQ, NQ, 1, NQ, NQ, false>(t, bufA, st->D);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) acc += gr[1][a] * geo.G[a * DIM + b] * gr[0][b];
  }
  bufA[t] = acc;
  __syncthreads();
  if (t == 0 && valid) {
    T s = T(0);
    for (int q = 0; q < NP; ++q) s += bufA[q];
    g_out[cell] = -s;
  }
}

}  // namespace smf
