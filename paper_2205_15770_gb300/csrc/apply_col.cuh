// 3D cell kernel, "column" layout: one thread per (x, y) node column of a cell, the z-line
// of every field held in registers.  Same operator as stokes_cell_apply (paper Sec. 3.1 sum
// factorisation of the Taylor-Hood element action, Sec. 2 bilinear forms), different mapping:
//   * (k+1)^2 threads per cell, 32 / (k+1)^2 cells per warp: a cell never straddles a warp,
//     so the x / y contractions exchange values with __shfl_sync and need no barrier;
//   * z contractions run in registers against the uniform 1D tables in constant memory;
//   * per-thread rows of the x / y tables are kept in registers;
//   * the trilinear Jacobian along a column is linear in zeta for its first two columns and
//     constant for the third, so it is set up once per thread from the 8 vertices and then
//     evaluated at the (k+1) Gauss points of the column with a few FMAs.
// MODE is the block bit set (kApplyA / kApplyBT / kApplyB) fixed at compile time.
// WARPS = 1 or 4: each warp takes its own cells and runs the three velocity components one
// after another.  WARPS = 3 ("component split", for small levels where the kernel's duration is
// the latency of one warp): the three warps of a CTA share the same cells, warp c handles
// velocity component c (geometry and pressure interpolation are evaluated by each warp), and the
// pressure test-function sums of the three warps meet in the atomic scatter.
#pragma once
#include "apply.cuh"
#include "vec.cuh"

namespace smf {

template <int K>
struct ColShape {
  static constexpr int NV = K + 1;            // velocity nodes per direction
  static constexpr int NQ = K + 1;            // Gauss points per direction
  static constexpr int NPR = K;               // pressure nodes per direction
  static constexpr int TPC = NV * NV;         // threads per cell
  static constexpr int CPW = 32 / TPC;        // cells per warp
  static constexpr int MAX_WARPS = 4;         // warps per CTA: 1, 3 (component split) or 4 (autotuned)
  static constexpr int MAX_THREADS = 32 * MAX_WARPS;
};

// Uniform 1D tables of this translation unit's degree (one copy per TU / degree).
// [0] S (NQ x NV), [1] D (NQ x NQ), [2] Pv (NQ x NPR), [3] Gauss weights (NQ) then points (NQ).
static __constant__ float c_colf[4][kMaxN1 * kMaxN1];
static __constant__ double c_cold[4][kMaxN1 * kMaxN1];

template <typename T>
struct CTab;
template <>
struct CTab<float> {
  static __device__ __forceinline__ float S(int i) { return c_colf[0][i]; }
  static __device__ __forceinline__ float D(int i) { return c_colf[1][i]; }
  static __device__ __forceinline__ float P(int i) { return c_colf[2][i]; }
  static __device__ __forceinline__ float W(int i) { return c_colf[3][i]; }
};
template <>
struct CTab<double> {
  static __device__ __forceinline__ double S(int i) { return c_cold[0][i]; }
  static __device__ __forceinline__ double D(int i) { return c_cold[1][i]; }
  static __device__ __forceinline__ double P(int i) { return c_cold[2][i]; }
  static __device__ __forceinline__ double W(int i) { return c_cold[3][i]; }
};

template <int K>
int upload_col_tables(const Tab1D<double> &t, cudaStream_t s) {
  constexpr int NQ = K + 1, NV = K + 1, NPR = K;
  double hd[4][kMaxN1 * kMaxN1] = {};
  for (int q = 0; q < NQ; ++q) {
    for (int m = 0; m < NV; ++m) hd[0][q * NV + m] = t.S[q * NV + m];
    for (int m = 0; m < NQ; ++m) hd[1][q * NQ + m] = t.D[q * NQ + m];
    for (int m = 0; m < NPR; ++m) hd[2][q * NPR + m] = t.Pv[q * NPR + m];
    hd[3][q] = t.w[q];
    hd[3][NQ + q] = t.x[q];
  }
  float hf[4][kMaxN1 * kMaxN1];
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < kMaxN1 * kMaxN1; ++i) hf[a][i] = (float)hd[a][i];
  cudaError_t e = cudaMemcpyToSymbolAsync(c_cold, hd, sizeof(hd), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_colf, hf, sizeof(hf), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? 0 : (int)e;
}

template <typename T>
__device__ __forceinline__ T sel3(int c, T a, T b, T d) {
  return c == 0 ? a : (c == 1 ? b : d);
}

// Geometry of a column's Gauss points (qx = ix, qy = iy, qz = 0..NQ-1) of cell (cx, cy, cz):
// G = mu w adj(J) adj(J)^T / det J (symmetric, 00 01 02 11 12 22), Cm = w adj(J) (when NEED_C),
// Wd = gamma rho w det J, w the tensor Gauss weight: the coefficients of the two terms of the
// viscous block are folded into the per-point factors.  Trilinear cells: the first two Jacobian
// columns are linear in zeta along the column and the third is constant, so they are set up once
// from the 8 vertices and evaluated per point.
template <int K, typename T, bool CART, bool NEED_C>
__device__ __forceinline__ void col_geometry(const LevelDesc<T> &L, int ix, int iy, int cx, int cy, int cz, T mu,
                                             T grho, T (&G)[K + 1][6], T (&Cm)[NEED_C ? K + 1 : 1][9],
                                             T (&Wd)[K + 1]) {
  using CT = CTab<T>;
  constexpr int NQ = K + 1;
  {
    const T wxy = CT::W(ix) * CT::W(iy);
    if (CART) {
      const T h0 = L.h[0], h1 = L.h[1], h2 = L.h[2];
      const T a0 = h1 * h2, a1 = h0 * h2, a2 = h0 * h1, det = h0 * h1 * h2;
#pragma unroll
      for (int qz = 0; qz < NQ; ++qz) {
        const T w = wxy * CT::W(qz), wm = mu * w;
        G[qz][0] = wm * a0 * a0 / det;
        G[qz][1] = T(0);
        G[qz][2] = T(0);
        G[qz][3] = wm * a1 * a1 / det;
        G[qz][4] = T(0);
        G[qz][5] = wm * a2 * a2 / det;
        Wd[qz] = grho * w * det;
        if (NEED_C) {
#pragma unroll
          for (int i = 0; i < 9; ++i) Cm[qz][i] = T(0);
          Cm[qz][0] = w * a0;
          Cm[qz][4] = w * a1;
          Cm[qz][8] = w * a2;
        }
      }
    } else {
      // vertices X[v][a], v = vx + 2 vy + 4 vz
      T X[8][3];
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const long long gv =
            ((long long)(cz + ((v >> 2) & 1)) * (L.n[1] + 1) + (cy + ((v >> 1) & 1))) * (L.n[0] + 1) + (cx + (v & 1));
#pragma unroll
        for (int a = 0; a < 3; ++a) X[v][a] = L.vert[gv * 3 + a];
      }
      const T xi = CT::W(NQ + ix), eta = CT::W(NQ + iy);
      // column 0 (d/dxi) at zeta = 0 and 1: bilinear in eta of the x-edge differences
      // column 1 (d/deta) at zeta = 0 and 1: in xi of the y-edge differences
      // column 2 (d/dzeta): bilinear in (xi, eta) of the z-edge differences (constant in zeta)
      T c0[2][3], c1[2][3], c2[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int z = 0; z < 2; ++z) {
          const T e00 = X[4 * z + 1][a] - X[4 * z + 0][a], e10 = X[4 * z + 3][a] - X[4 * z + 2][a];
          c0[z][a] = e00 + eta * (e10 - e00);
          const T f00 = X[4 * z + 2][a] - X[4 * z + 0][a], f10 = X[4 * z + 3][a] - X[4 * z + 1][a];
          c1[z][a] = f00 + xi * (f10 - f00);
        }
        const T g00 = X[4][a] - X[0][a], g10 = X[5][a] - X[1][a], g01 = X[6][a] - X[2][a], g11 = X[7][a] - X[3][a];
        const T gl = g00 + xi * (g10 - g00), gh = g01 + xi * (g11 - g01);
        c2[a] = gl + eta * (gh - gl);
      }
#pragma unroll
      for (int qz = 0; qz < NQ; ++qz) {
        const T zeta = CT::W(NQ + qz);
        T J[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          J[a][0] = c0[0][a] + zeta * (c0[1][a] - c0[0][a]);
          J[a][1] = c1[0][a] + zeta * (c1[1][a] - c1[0][a]);
          J[a][2] = c2[a];
        }
        T adj[3][3];
        adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const T det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
        const T w = wxy * CT::W(qz);
        const T wd = mu * w / det;
        G[qz][0] = wd * (adj[0][0] * adj[0][0] + adj[0][1] * adj[0][1] + adj[0][2] * adj[0][2]);
        G[qz][1] = wd * (adj[0][0] * adj[1][0] + adj[0][1] * adj[1][1] + adj[0][2] * adj[1][2]);
        G[qz][2] = wd * (adj[0][0] * adj[2][0] + adj[0][1] * adj[2][1] + adj[0][2] * adj[2][2]);
        G[qz][3] = wd * (adj[1][0] * adj[1][0] + adj[1][1] * adj[1][1] + adj[1][2] * adj[1][2]);
        G[qz][4] = wd * (adj[1][0] * adj[2][0] + adj[1][1] * adj[2][1] + adj[1][2] * adj[2][2]);
        G[qz][5] = wd * (adj[2][0] * adj[2][0] + adj[2][1] * adj[2][1] + adj[2][2] * adj[2][2]);
        Wd[qz] = grho * w * det;
        if (NEED_C) {
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) Cm[qz][a * 3 + b] = w * adj[a][b];
        }
      }
    }
  }
}

// FUSED: the inputs are the combinations of a Fuse descriptor, evaluated while gathering, and the
// owners of the gathered nodes perform its side effects (stores, zeroing, p += dp).
template <int K, typename T, int MODE, bool CART, int WARPS, bool FUSED>
__global__ void __launch_bounds__(32 * WARPS)
    stokes_cell_apply_col(const LevelDesc<T> L, const T *__restrict__ u, const T *__restrict__ p,
                          T *__restrict__ yu, T *__restrict__ yp, const Fuse<T> F,
                          const T *__restrict__ geo) {
  pdl_enter();
  using CS = ColShape<K>;
  using CT = CTab<T>;
  constexpr int NV = CS::NV, NQ = CS::NQ, NPR = CS::NPR, TPC = CS::TPC;
  constexpr bool DO_A = MODE & kApplyA, DO_BT = MODE & kApplyBT, DO_B = MODE & kApplyB;
  constexpr bool NEED_U = DO_A || DO_B;
  constexpr bool NEED_C = DO_BT || DO_B;
  constexpr unsigned FULL = 0xffffffffu;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  int sub = lane / TPC;
  const bool pad = sub >= CS::CPW;
  if (pad) sub = 0;
  const int tl = lane - (lane / TPC) * TPC;
  const int ix = pad ? 0 : tl % NV, iy = pad ? 0 : tl / NV;
  const int base = sub * TPC;
  constexpr bool SPLIT = WARPS == 3;
  const long long group = SPLIT ? (long long)blockIdx.x : (long long)blockIdx.x * WARPS + warp;
  const long long cell = group * CS::CPW + sub;
  const int c_begin = SPLIT ? warp : 0, c_end = SPLIT ? warp + 1 : 3;
  const bool valid = !pad && cell < L.n_cells;
  int cx = 0, cy = 0, cz = 0;
  if (valid) {
    cx = (int)(cell % L.n[0]);
    const long long r = cell / L.n[0];
    cy = (int)(r % L.n[1]);
    cz = (int)(r / L.n[1]);
  }
  auto lane_of = [&](int a, int b) { return base + b * NV + a; };
  // ownership of the gathered nodes (each node has exactly one owning cell)
  const bool own_xy = valid && (ix < K || cx == L.n[0] - 1) && (iy < K || cy == L.n[1] - 1);
  const bool pown_xy = valid && (ix < K - 1 || cx == L.n[0] - 1) && (iy < K - 1 || cy == L.n[1] - 1);

  // per-thread rows of the x / y tables
  T Sx[NV], Sy[NV], Dx[NQ], Dy[NQ], StX[NQ], StY[NQ], DtX[NQ], DtY[NQ];
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    Sx[m] = CT::S(ix * NV + m);
    Sy[m] = CT::S(iy * NV + m);
  }
#pragma unroll
  for (int m = 0; m < NQ; ++m) {
    Dx[m] = CT::D(ix * NQ + m);
    Dy[m] = CT::D(iy * NQ + m);
    StX[m] = CT::S(m * NV + ix);
    StY[m] = CT::S(m * NV + iy);
    DtX[m] = CT::D(m * NQ + ix);
    DtY[m] = CT::D(m * NQ + iy);
  }

  // ---- velocity loads, issued one component ahead of their use -----------------------------
  // The gathers of component c+1 are in flight while component c is computed, and those of the
  // first component while the geometry is evaluated, so the warp waits for memory once.
  const int gx = K * cx + ix, gy = K * cy + iy;
  constexpr int NR = FUSED ? kFuseVel + 2 : 1;  // raw values per node: vv[0..2], vd, vb (fused) or u
  T raw[NR][NV];
  bool frs[NV], owns[NV];
#pragma unroll
  for (int iz = 0; iz < NV; ++iz) {
    const int gz = K * cz + iz;
    frs[iz] = valid && !vel_constrained(L.N, L.faces, 3, gx, gy, gz);
    owns[iz] = own_xy && (iz < K || cz == L.n[2] - 1);
  }
  const long long col0 = valid ? lattice_index<3, T>(L.N, gx, gy, K * cz) : 0;
  const long long zstride = (long long)L.N[0] * L.N[1];
  auto load_comp = [&](int c) {
#pragma unroll
    for (int iz = 0; iz < NV; ++iz) {
      const long long gi = c * L.nv + col0 + iz * zstride;
      if (!FUSED) {
        raw[0][iz] = frs[iz] ? u[gi] : T(0);
      } else {
        const bool need = frs[iz] || owns[iz];
        if (F.nv > 0) {
#pragma unroll
          for (int j = 0; j < kFuseVel; ++j) raw[j][iz] = (need && j < F.nv) ? F.vv[j][gi] : T(0);
          raw[kFuseVel][iz] = (need && F.vd) ? F.vd[gi] : T(1);
          raw[kFuseVel + 1][iz] = (need && F.vb) ? F.vb[gi] : T(0);
        } else {
          raw[0][iz] = need ? u[gi] : T(0);
        }
      }
    }
  };
  if (NEED_U) load_comp(c_begin);

  // ---- geometry at the column's Gauss points (qx = ix, qy = iy, qz = 0..NQ-1) --------------
  T G[NQ][6];                 // mu w adj adj^T / det, symmetric: 00 01 02 11 12 22
  T Cm[NEED_C ? NQ : 1][9];   // w adj
  T Wd[NQ];                   // gamma rho w det
  // mu and gamma rho enter the per-point factors (G, Wd) where they are formed
  const T mu = L.mu_cell ? (valid ? L.mu_cell[cell] : T(0)) : L.mu;
  const T grho = L.gamma_rho;
  // geo (trilinear levels): precomputed at setup where the setup stores it (FP64: the geometry is
  // a quarter of the flops of an application; FP32 small levels: it takes the vertex loads and the
  // Jacobian's arithmetic off each launch's dependency chain); otherwise evaluated on the fly.  (A
  // separate kernel argument: a larger level descriptor changes the register allocation of the
  // FP32 kernels.)
  if (!CART && geo) {
    // precomputed by k_col_geometry (col_geometry, same arithmetic): [cell][16][qz][iy][ix]
    const T *gp = geo + (valid ? cell : 0) * (long long)(16 * NQ * NV * NV) + iy * NV + ix;
    constexpr int ST = NQ * NV * NV;  // stride between the 16 fields
#pragma unroll
    for (int qz = 0; qz < NQ; ++qz) {
      const T *q = gp + qz * NV * NV;
      if (DO_A) {
#pragma unroll
        for (int i = 0; i < 6; ++i) G[qz][i] = q[i * ST];
        Wd[qz] = q[15 * ST];
      }
      if (NEED_C) {
#pragma unroll
        for (int i = 0; i < 9; ++i) Cm[qz][i] = q[(6 + i) * ST];
      }
    }
  } else {
    // on the fly (the same arithmetic as col_geometry, kept inline for the kernel's schedule)
    {
      const T wxy = CT::W(ix) * CT::W(iy);
      if (CART) {
        const T h0 = L.h[0], h1 = L.h[1], h2 = L.h[2];
        const T a0 = h1 * h2, a1 = h0 * h2, a2 = h0 * h1, det = h0 * h1 * h2;
  #pragma unroll
        for (int qz = 0; qz < NQ; ++qz) {
          const T w = wxy * CT::W(qz), wm = mu * w;
          G[qz][0] = wm * a0 * a0 / det;
          G[qz][1] = T(0);
          G[qz][2] = T(0);
          G[qz][3] = wm * a1 * a1 / det;
          G[qz][4] = T(0);
          G[qz][5] = wm * a2 * a2 / det;
          Wd[qz] = grho * w * det;
          if (NEED_C) {
  #pragma unroll
            for (int i = 0; i < 9; ++i) Cm[qz][i] = T(0);
            Cm[qz][0] = w * a0;
            Cm[qz][4] = w * a1;
            Cm[qz][8] = w * a2;
          }
        }
      } else {
        // vertices X[v][a], v = vx + 2 vy + 4 vz
        T X[8][3];
  #pragma unroll
        for (int v = 0; v < 8; ++v) {
          const long long gv =
              ((long long)(cz + ((v >> 2) & 1)) * (L.n[1] + 1) + (cy + ((v >> 1) & 1))) * (L.n[0] + 1) + (cx + (v & 1));
  #pragma unroll
          for (int a = 0; a < 3; ++a) X[v][a] = L.vert[gv * 3 + a];
        }
        const T xi = CT::W(NQ + ix), eta = CT::W(NQ + iy);
        // column 0 (d/dxi) at zeta = 0 and 1: bilinear in eta of the x-edge differences
        // column 1 (d/deta) at zeta = 0 and 1: in xi of the y-edge differences
        // column 2 (d/dzeta): bilinear in (xi, eta) of the z-edge differences (constant in zeta)
        T c0[2][3], c1[2][3], c2[3];
  #pragma unroll
        for (int a = 0; a < 3; ++a) {
  #pragma unroll
          for (int z = 0; z < 2; ++z) {
            const T e00 = X[4 * z + 1][a] - X[4 * z + 0][a], e10 = X[4 * z + 3][a] - X[4 * z + 2][a];
            c0[z][a] = e00 + eta * (e10 - e00);
            const T f00 = X[4 * z + 2][a] - X[4 * z + 0][a], f10 = X[4 * z + 3][a] - X[4 * z + 1][a];
            c1[z][a] = f00 + xi * (f10 - f00);
          }
          const T g00 = X[4][a] - X[0][a], g10 = X[5][a] - X[1][a], g01 = X[6][a] - X[2][a], g11 = X[7][a] - X[3][a];
          const T gl = g00 + xi * (g10 - g00), gh = g01 + xi * (g11 - g01);
          c2[a] = gl + eta * (gh - gl);
        }
  #pragma unroll
        for (int qz = 0; qz < NQ; ++qz) {
          const T zeta = CT::W(NQ + qz);
          T J[3][3];
  #pragma unroll
          for (int a = 0; a < 3; ++a) {
            J[a][0] = c0[0][a] + zeta * (c0[1][a] - c0[0][a]);
            J[a][1] = c1[0][a] + zeta * (c1[1][a] - c1[0][a]);
            J[a][2] = c2[a];
          }
          T adj[3][3];
          adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
          adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
          adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
          adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
          adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
          adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
          adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
          adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
          adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
          const T det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
          const T w = wxy * CT::W(qz);
          const T wd = mu * w / det;
          G[qz][0] = wd * (adj[0][0] * adj[0][0] + adj[0][1] * adj[0][1] + adj[0][2] * adj[0][2]);
          G[qz][1] = wd * (adj[0][0] * adj[1][0] + adj[0][1] * adj[1][1] + adj[0][2] * adj[1][2]);
          G[qz][2] = wd * (adj[0][0] * adj[2][0] + adj[0][1] * adj[2][1] + adj[0][2] * adj[2][2]);
          G[qz][3] = wd * (adj[1][0] * adj[1][0] + adj[1][1] * adj[1][1] + adj[1][2] * adj[1][2]);
          G[qz][4] = wd * (adj[1][0] * adj[2][0] + adj[1][1] * adj[2][1] + adj[1][2] * adj[2][2]);
          G[qz][5] = wd * (adj[2][0] * adj[2][0] + adj[2][1] * adj[2][1] + adj[2][2] * adj[2][2]);
          Wd[qz] = grho * w * det;
          if (NEED_C) {
  #pragma unroll
            for (int a = 0; a < 3; ++a)
  #pragma unroll
              for (int b = 0; b < 3; ++b) Cm[qz][a * 3 + b] = w * adj[a][b];
          }
        }
      }
    }
  }

  // ---- pressure at the column's Gauss points ---------------------------------------------------
  T pq[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) pq[q] = T(0);
  if (DO_BT) {
    T pz[NPR];
    const bool pown = valid && ix < NPR && iy < NPR;
    long long pgi[NPR];
#pragma unroll
    for (int iz = 0; iz < NPR; ++iz)
      pgi[iz] = lattice_index<3, T>(L.Pn, (K - 1) * cx + ix, (K - 1) * cy + iy, (K - 1) * cz + iz);
    if (FUSED) {
      // loads first, then the side effects, once per node: its owning cell, and in the split
      // shape only warp 0
#pragma unroll
      for (int iz = 0; iz < NPR; ++iz) {
        T pv = T(0);
        if (pown) {
          if (F.np > 0) {
            T sum = T(0);
#pragma unroll
            for (int j = 0; j < kFusePre; ++j)
              if (j < F.np) sum += F.pc[j] * F.pv[j][pgi[iz]];
            pv = F.pd[pgi[iz]] * sum;
          } else {
            pv = p[pgi[iz]];
          }
        }
        pz[iz] = pv;
      }
#pragma unroll
      for (int iz = 0; iz < NPR; ++iz)
        if (pown && pown_xy && (iz < K - 1 || cz == L.n[2] - 1) && (!SPLIT || warp == 0)) {
          if (F.pacc) F.pacc[pgi[iz]] += pz[iz];
#pragma unroll
          for (int j = 0; j < kFusePre; ++j)
            if (F.pzero[j]) F.pzero[j][pgi[iz]] = T(0);
        }
    } else {
#pragma unroll
      for (int iz = 0; iz < NPR; ++iz) pz[iz] = pown ? p[pgi[iz]] : T(0);
    }
    T a[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T s = T(0);
#pragma unroll
      for (int iz = 0; iz < NPR; ++iz) s += CT::P(q * NPR + iz) * pz[iz];
      a[q] = s;
    }
    // x: role (qx = ix, iy < NPR) from lanes (m, iy)
    T b[NQ];
    const int iyc = iy < NPR ? iy : NPR - 1;
#pragma unroll
    for (int q = 0; q < NQ; ++q) b[q] = T(0);
#pragma unroll
    for (int m = 0; m < NPR; ++m) {
      const T cf = CT::P(ix * NPR + m);
#pragma unroll
      for (int q = 0; q < NQ; ++q) b[q] += cf * __shfl_sync(FULL, a[q], lane_of(m, iyc));
    }
    // y: role (qx, qy = iy) from lanes (ix, m)
#pragma unroll
    for (int m = 0; m < NPR; ++m) {
      const T cf = CT::P(iy * NPR + m);
#pragma unroll
      for (int q = 0; q < NQ; ++q) pq[q] += cf * __shfl_sync(FULL, b[q], lane_of(ix, m));
    }
  }

  // ---- velocity components -----------------------------------------------------------------
  T qacc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) qacc[q] = T(0);
#pragma unroll 1
  for (int c = c_begin; c < c_end; ++c) {
    T v[NQ], gxv[NQ], gyv[NQ], gzv[NQ];
    if (NEED_U) {
      T uz[NV];
      {
        T vals[NV];
#pragma unroll
        for (int iz = 0; iz < NV; ++iz) {
          if (FUSED && F.nv > 0) {
            T sum = F.vc[0] * raw[0][iz];
#pragma unroll
            for (int j = 1; j < kFuseVel; ++j)
              if (j < F.nv) sum += F.vc[j] * raw[j][iz];
            vals[iz] = raw[kFuseVel + 1][iz] + raw[kFuseVel][iz] * sum;
          } else {
            vals[iz] = raw[0][iz];
          }
          uz[iz] = frs[iz] ? vals[iz] : T(0);
        }
        if (FUSED) {
#pragma unroll
          for (int iz = 0; iz < NV; ++iz)
            if (owns[iz]) {
              const long long gi = c * L.nv + col0 + iz * zstride;
              if (F.vstore) F.vstore[gi] = vals[iz];
              if (F.vzero[0]) F.vzero[0][gi] = T(0);
              if (F.vzero[1]) F.vzero[1][gi] = T(0);
            }
        }
        if (c + 1 < c_end) load_comp(c + 1);
      }
      T a[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T s = T(0);
#pragma unroll
        for (int m = 0; m < NV; ++m) s += CT::S(q * NV + m) * uz[m];
        a[q] = s;
      }
      T b[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) b[q] = T(0);
#pragma unroll
      for (int m = 0; m < NV; ++m)
#pragma unroll
        for (int q = 0; q < NQ; ++q) b[q] += Sx[m] * __shfl_sync(FULL, a[q], lane_of(m, iy));
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] = T(0);
#pragma unroll
      for (int m = 0; m < NV; ++m)
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] += Sy[m] * __shfl_sync(FULL, b[q], lane_of(ix, m));
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T s = T(0);
#pragma unroll
        for (int m = 0; m < NQ; ++m) s += CT::D(q * NQ + m) * v[m];
        gzv[q] = s;
        gxv[q] = T(0);
        gyv[q] = T(0);
      }
#pragma unroll
      for (int m = 0; m < NQ; ++m)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          gxv[q] += Dx[m] * __shfl_sync(FULL, v[q], lane_of(m, iy));
          gyv[q] += Dy[m] * __shfl_sync(FULL, v[q], lane_of(ix, m));
        }
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] = gxv[q] = gyv[q] = gzv[q] = T(0);
      if (FUSED && (F.vzero[0] || F.vzero[1])) {
#pragma unroll
        for (int iz = 0; iz < NV; ++iz)
          if (owns[iz]) {
            const long long gi = c * L.nv + col0 + iz * zstride;
            if (F.vzero[0]) F.vzero[0][gi] = T(0);
            if (F.vzero[1]) F.vzero[1][gi] = T(0);
          }
      }
    }
    // column c of C = w adj at each point (selected without dynamic register indexing)
    T cc0[NQ], cc1[NQ], cc2[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int qq = NEED_C ? q : 0;
      cc0[q] = sel3(c, Cm[qq][0], Cm[qq][1], Cm[qq][2]);
      cc1[q] = sel3(c, Cm[qq][3], Cm[qq][4], Cm[qq][5]);
      cc2[q] = sel3(c, Cm[qq][6], Cm[qq][7], Cm[qq][8]);
    }
    if (DO_B) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) qacc[q] -= cc0[q] * gxv[q] + cc1[q] * gyv[q] + cc2[q] * gzv[q];
    }
    if (DO_A || DO_BT) {
      T fx[NQ], fy[NQ], tq[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T f0 = T(0), f1 = T(0), f2 = T(0), mv = T(0);
        if (DO_A) {
          f0 = G[q][0] * gxv[q] + G[q][1] * gyv[q] + G[q][2] * gzv[q];
          f1 = G[q][1] * gxv[q] + G[q][3] * gyv[q] + G[q][4] * gzv[q];
          f2 = G[q][2] * gxv[q] + G[q][4] * gyv[q] + G[q][5] * gzv[q];
          mv = Wd[q] * v[q];
        }
        if (DO_BT) {
          f0 -= pq[q] * cc0[q];
          f1 -= pq[q] * cc1[q];
          f2 -= pq[q] * cc2[q];
        }
        fx[q] = f0;
        fy[q] = f1;
        gzv[q] = f2;  // z flux kept in the gz registers
        tq[q] = mv;
      }
      // transposed derivatives: z in registers, x / y from lanes
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T s = tq[q];
#pragma unroll
        for (int m = 0; m < NQ; ++m) s += CT::D(m * NQ + q) * gzv[m];
        tq[q] = s;
      }
#pragma unroll
      for (int m = 0; m < NQ; ++m)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          tq[q] += DtX[m] * __shfl_sync(FULL, fx[q], lane_of(m, iy));
          tq[q] += DtY[m] * __shfl_sync(FULL, fy[q], lane_of(ix, m));
        }
      // transposed interpolation: y (lanes (ix, m)), x (lanes (m, iy)), z (registers)
      T s1[NQ], s2[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) s1[q] = T(0);
#pragma unroll
      for (int m = 0; m < NQ; ++m)
#pragma unroll
        for (int q = 0; q < NQ; ++q) s1[q] += StY[m] * __shfl_sync(FULL, tq[q], lane_of(ix, m));
#pragma unroll
      for (int q = 0; q < NQ; ++q) s2[q] = T(0);
#pragma unroll
      for (int m = 0; m < NQ; ++m)
#pragma unroll
        for (int q = 0; q < NQ; ++q) s2[q] += StX[m] * __shfl_sync(FULL, s1[q], lane_of(m, iy));
#pragma unroll
      for (int iz = 0; iz < NV; ++iz) {
        T s = T(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) s += CT::S(q * NV + iz) * s2[q];
        if (frs[iz]) atomicAdd(&yu[c * L.nv + col0 + iz * zstride], s);
      }
    }
  }

  // ---- pressure test functions: transposed interpolation y, x (lanes), z (registers) -----------
  if (DO_B) {
    const int iyc = iy < NPR ? iy : NPR - 1;
    const int ixc = ix < NPR ? ix : NPR - 1;
    T s1[NQ], s2[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) s1[q] = T(0);
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const T cf = CT::P(m * NPR + iyc);
#pragma unroll
      for (int q = 0; q < NQ; ++q) s1[q] += cf * __shfl_sync(FULL, qacc[q], lane_of(ix, m));
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) s2[q] = T(0);
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const T cf = CT::P(m * NPR + ixc);
#pragma unroll
      for (int q = 0; q < NQ; ++q) s2[q] += cf * __shfl_sync(FULL, s1[q], lane_of(m, iyc));
    }
    if (valid && ix < NPR && iy < NPR) {
#pragma unroll
      for (int iz = 0; iz < NPR; ++iz) {
        T s = T(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) s += CT::P(q * NPR + iz) * s2[q];
        const long long gi = lattice_index<3, T>(L.Pn, (K - 1) * cx + ix, (K - 1) * cy + iy, (K - 1) * cz + iz);
        atomicAdd(&yp[gi], s);
      }
    }
  }
}

}  // namespace smf

namespace smf {

// Per-point geometry of every cell for the column kernel, written once at setup:
// geo[cell][field][qz][iy][ix], fields G (6), Cm (9), Wd (1) as in col_geometry (mu and gamma rho
// included).
template <int K, typename T>
__global__ void k_col_geometry(const LevelDesc<T> L, T *__restrict__ geo) {
  pdl_enter();
  constexpr int NV = K + 1, NQ = K + 1, ST = NQ * NV * NV;
  SMF_GRID_LOOP(t, L.n_cells * NV * NV) {
    const long long cell = t / (NV * NV);
    const int r = (int)(t - cell * NV * NV), iy = r / NV, ix = r - iy * NV;
    const int cx = (int)(cell % L.n[0]);
    const long long rr = cell / L.n[0];
    const int cy = (int)(rr % L.n[1]), cz = (int)(rr / L.n[1]);
    T G[NQ][6], Cm[NQ][9], Wd[NQ];
    const T mu = L.mu_cell ? L.mu_cell[cell] : L.mu;
    col_geometry<K, T, false, true>(L, ix, iy, cx, cy, cz, mu, L.gamma_rho, G, Cm, Wd);
    T *base = geo + cell * (long long)(16 * ST) + iy * NV + ix;
#pragma unroll
    for (int qz = 0; qz < NQ; ++qz) {
      T *q = base + qz * NV * NV;
#pragma unroll
      for (int i = 0; i < 6; ++i) q[i * ST] = G[qz][i];
#pragma unroll
      for (int i = 0; i < 9; ++i) q[(6 + i) * ST] = Cm[qz][i];
      q[15 * ST] = Wd[qz];
    }
  }
}

}  // namespace smf
