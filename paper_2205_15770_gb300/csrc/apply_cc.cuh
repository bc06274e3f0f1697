// 3D cell kernel, "cell-component" layout (launch shape 5): one thread per (cell, velocity
// component).  Same operator as stokes_cell_apply_col and stokes_cell_apply (paper Sec. 3.1:
// K x = sum_tau P_tau K_tau P_tau^T x with the element action by sum factorisation; Sec. 2
// bilinear forms a(u,v) = mu grad u : grad v + gamma rho u.v and b(v,q) = -q div v), mapped so
// that a thread holds the whole (k+1)^3 tensor of its velocity component in registers: every 1D
// contraction is a register loop against uniform tables and no value crosses lanes (the column
// kernel moves x / y contractions through warp shuffles, which bound its issue rate).
//   * 10 cells per warp, lane = c * 10 + s (velocity component c, cell s of the warp's group);
//     lanes 30 and 31 idle.
//   * Trilinear cells (FP32, k = 2): the three threads of a cell evaluate the cell-map geometry
//     of one plane of Gauss points each (qz = c) and share it through shared memory
//     (G = mu w adj(J) adj(J)^T / det J, gamma rho w det J, and the columns of w adj(J)), so each
//     point's geometry is computed once per cell; the point operation reads it back as float4.
//   * Cartesian cells (FP32 and FP64, k = 2, 3): the element matrices are Kronecker products of
//     the 1D stiffness, mass and mixed matrices (exact for the (k+1)-point Gauss rule used
//     everywhere else), so the A block is 7 sweeps of 1D matrices over the nodal values and
//     B, B^T are 3 sweeps each; no quadrature-point arrays, no shared memory.
//   * Scatter by atomicAdd at the gather's indices; constrained DoFs read as 0 and not written.
#pragma once
#include <algorithm>

#include "apply.cuh"
#include "host_tables.h"
#include "vec.cuh"

namespace smf {

constexpr int kCcCells = 10;  // cells per warp of the cell-component kernel

// 1D tables of this translation unit's degree for the cell-component kernel.
template <typename T>
struct CCTab {
  // pairs for the packed (two FMAs per instruction) FP32 sweeps of the Cartesian A block, first in
  // the struct so that they are 8-byte aligned: MK[2(i*NV+j) + 0 / 1] = (Mh, Kh)[i*NV+j],
  // MM[2(i*NV+j) + 0 / 1] = Mh[i*NV+j] twice
  T MK[2 * kMaxN1 * kMaxN1];
  T MM[2 * kMaxN1 * kMaxN1];
  T S[kMaxN1 * kMaxN1];    // S[q*NV+m]  = l_m(x_q)   velocity basis at the Gauss points
  T D[kMaxN1 * kMaxN1];    // D[q*NQ+m]  = g_m'(x_q)  collocation derivative at the Gauss points
  T P[kMaxN1 * kMaxDeg];   // P[q*NPR+a] = psi_a(x_q) pressure basis at the Gauss points
  T W[kMaxN1];             // Gauss weights on [0,1]
  T X[kMaxN1];             // Gauss points on [0,1]
  T Kh[kMaxN1 * kMaxN1];   // Kh[i*NV+j] = int_0^1 l_i' l_j'
  T Mh[kMaxN1 * kMaxN1];   // Mh[i*NV+j] = int_0^1 l_i l_j
  T Gh[kMaxDeg * kMaxN1];  // Gh[a*NV+j] = int_0^1 psi_a l_j'
  T Nh[kMaxDeg * kMaxN1];  // Nh[a*NV+j] = int_0^1 psi_a l_j
};
static __constant__ __align__(16) CCTab<float> c_ccf;
static __constant__ __align__(16) CCTab<double> c_ccd;
template <typename T>
__device__ __forceinline__ const CCTab<T> &cct();
template <>
__device__ __forceinline__ const CCTab<float> &cct<float>() {
  return c_ccf;
}
template <>
__device__ __forceinline__ const CCTab<double> &cct<double>() {
  return c_ccd;
}

template <int K>
cudaError_t cc_prefer_shared();

// Fills this translation unit's tables from the FP64 1D tables (the integrals by the same
// (k+1)-point Gauss rule, exact for these polynomial degrees).
template <int K>
int upload_cc_tables(const Tab1D<double> &t, cudaStream_t s) {
  constexpr int NQ = K + 1, NV = K + 1, NPR = K;
  CCTab<double> h{};
  for (int q = 0; q < NQ; ++q) {
    for (int m = 0; m < NV; ++m) h.S[q * NV + m] = t.S[q * NV + m];
    for (int m = 0; m < NQ; ++m) h.D[q * NQ + m] = t.D[q * NQ + m];
    for (int a = 0; a < NPR; ++a) h.P[q * NPR + a] = t.Pv[q * NPR + a];
    h.W[q] = t.w[q];
    h.X[q] = t.x[q];
  }
  for (int i = 0; i < NV; ++i)
    for (int j = 0; j < NV; ++j) {
      double kk = 0, mm = 0;
      for (int q = 0; q < NQ; ++q) {
        kk += t.w[q] * t.Sd[q * NV + i] * t.Sd[q * NV + j];
        mm += t.w[q] * t.S[q * NV + i] * t.S[q * NV + j];
      }
      h.Kh[i * NV + j] = kk;
      h.Mh[i * NV + j] = mm;
      h.MK[2 * (i * NV + j)] = mm;
      h.MK[2 * (i * NV + j) + 1] = kk;
      h.MM[2 * (i * NV + j)] = mm;
      h.MM[2 * (i * NV + j) + 1] = mm;
    }
  for (int a = 0; a < NPR; ++a)
    for (int j = 0; j < NV; ++j) {
      double gg = 0, nn = 0;
      for (int q = 0; q < NQ; ++q) {
        gg += t.w[q] * t.Pv[q * NPR + a] * t.Sd[q * NV + j];
        nn += t.w[q] * t.Pv[q * NPR + a] * t.S[q * NV + j];
      }
      h.Gh[a * NV + j] = gg;
      h.Nh[a * NV + j] = nn;
    }
  CCTab<float> f{};
  {
    const double *src = reinterpret_cast<const double *>(&h);
    float *dst = reinterpret_cast<float *>(&f);
    for (size_t i = 0; i < sizeof(h) / sizeof(double); ++i) dst[i] = (float)src[i];
  }
  cudaError_t e = cc_prefer_shared<K>();
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_ccd, &h, sizeof(h), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_ccf, &f, sizeof(f), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? 0 : (int)e;
}

// 1D contractions of a register tensor a[z][y][x] along x (0), y (1) or z (2):
//   out[.. i ..] = sum_j M(i, j) in[.. j ..]
template <int NI, int NO, int E1, int E2, typename T, typename F>
__device__ __forceinline__ void cc_sweep0(const T (&in)[E2][E1][NI], T (&out)[E2][E1][NO], F M) {
#pragma unroll
  for (int z = 0; z < E2; ++z)
#pragma unroll
    for (int y = 0; y < E1; ++y)
#pragma unroll
      for (int i = 0; i < NO; ++i) {
        T s = M(i, 0) * in[z][y][0];
#pragma unroll
        for (int j = 1; j < NI; ++j) s += M(i, j) * in[z][y][j];
        out[z][y][i] = s;
      }
}
template <int NI, int NO, int E0, int E2, typename T, typename F>
__device__ __forceinline__ void cc_sweep1(const T (&in)[E2][NI][E0], T (&out)[E2][NO][E0], F M) {
#pragma unroll
  for (int z = 0; z < E2; ++z)
#pragma unroll
    for (int x = 0; x < E0; ++x)
#pragma unroll
      for (int i = 0; i < NO; ++i) {
        T s = M(i, 0) * in[z][0][x];
#pragma unroll
        for (int j = 1; j < NI; ++j) s += M(i, j) * in[z][j][x];
        out[z][i][x] = s;
      }
}
template <int NI, int NO, int E0, int E1, typename T, typename F>
__device__ __forceinline__ void cc_sweep2(const T (&in)[NI][E1][E0], T (&out)[NO][E1][E0], F M) {
#pragma unroll
  for (int y = 0; y < E1; ++y)
#pragma unroll
    for (int x = 0; x < E0; ++x)
#pragma unroll
      for (int i = 0; i < NO; ++i) {
        T s = M(i, 0) * in[0][y][x];
#pragma unroll
        for (int j = 1; j < NI; ++j) s += M(i, j) * in[j][y][x];
        out[i][y][x] = s;
      }
}

// Shared-memory geometry record of one Gauss point of one cell (trilinear, FP32): NF = NA + NB
// float4, with the A block [0] = (G00, G01, G02, G11), [1] = (G12, G22, gamma rho w det, 0),
// G = mu w adj adj^T / det (NA = 2), and with a B block [NA + j] = column j of w adj(J) (NB = 3).
template <int MODE>
struct CcGeo {
  static constexpr int NA = (MODE & kApplyA) ? 2 : 0;
  static constexpr int NB = (MODE & (kApplyB | kApplyBT)) ? 3 : 0;
  static constexpr int NF = NA + NB;
};

#ifndef SMF_CC_SLICE_UNROLL
#define SMF_CC_SLICE_UNROLL 1
#endif
#ifndef SMF_CC_TARGET_WARPS
#define SMF_CC_TARGET_WARPS 16
#endif
template <int K, typename T, int MODE, bool CART>
struct CcLaunch {
  static constexpr int NQ = K + 1;
  // trilinear cells: FP32 shares the geometry through shared memory, FP64 reads the per-point
  // geometry stored at setup (the column kernel's layout)
  static constexpr bool SMEM_GEO = !CART && sizeof(T) == 4;
  static constexpr int WARPS = (SMEM_GEO && CcGeo<MODE>::NF > 3) ? 2 : 4;
  static constexpr size_t GEO_BYTES =
      SMEM_GEO ? (size_t)WARPS * NQ * NQ * NQ * CcGeo<MODE>::NF * kCcCells * sizeof(float4) : 0;
  // deterministic launches: the three component threads' pressure sums of a cell meet here
  static constexpr size_t RED_BYTES = (MODE & kApplyB) ? (size_t)WARPS * kCcCells * 3 * K * K * K * sizeof(T) : 0;
  static constexpr size_t SMEM = GEO_BYTES;
  static constexpr size_t SMEM_DET = GEO_BYTES + RED_BYTES;
  // resident warps per SM the register allocation is held to (FP32; FP64 keeps its registers)
  static constexpr int MINB = (sizeof(T) == 4 && K == 2) ? (SMF_CC_TARGET_WARPS + WARPS - 1) / WARPS : 1;
};

// Cells of colour class `colour` (bit a = parity of the cell index along axis a): no two of them
// share a velocity or pressure node.
__host__ __device__ inline long long colour_extent(const int n[3], int colour, int a) {
  const int par = (colour >> a) & 1;
  return (n[a] - par + 1) / 2;
}

// One warp's group of cells.  colour < 0: cells group * 10 .. + 9 in lexicographic order, scatter
// by atomicAdd.  colour >= 0 (DET): the group-th 10 cells of that colour class, scatter by plain
// read-modify-write through L2 (no other thread touches the node in this class), the three
// component threads' pressure sums added in a fixed order: bitwise reproducible results.
// FUSED: the inputs are the pointwise combinations of the Fuse descriptor F (the smoother's vector
// updates, Sec. 3.3.1), evaluated while gathering; the owner of each gathered node (thread of its
// component in the owning cell; component 0 for pressure nodes) performs F's side effects.
// COH: inputs read through L2 only (see ld_in).  LOCAL (owner-computes deterministic form): yu / yp
// receive this thread's local results instead of the scatter, yu[(i * 3 + c) * n_cells + cell] for
// the velocity node i of the cell (z, y, x lexicographic) and yp[(a * 3 + c) * n_cells + cell] for
// the pressure node a (component c's part of B u); k_cc_owner_gather sums them per DoF.
template <int K, typename T, int MODE, bool CART, bool DET, bool FUSED = false, bool COH = false,
          bool LOCAL = false>
__device__ __forceinline__ void cc_group(const LevelDesc<T> &L, const T *__restrict__ u, const T *__restrict__ p,
                                         T *__restrict__ yu, T *__restrict__ yp, const T *__restrict__ geo,
                                         long long group, int colour, const Fuse<T> &F = Fuse<T>{}) {
  constexpr int NV = K + 1, NQ = K + 1, NPR = K, CPW = kCcCells;
  constexpr bool DO_A = MODE & kApplyA, DO_BT = MODE & kApplyBT, DO_B = MODE & kApplyB;
  constexpr bool NEED_U = DO_A || DO_B;
  using CL = CcLaunch<K, T, MODE, CART>;
  static_assert(CART || K == 2, "trilinear cell-component kernel: k = 2");
  static_assert(!(COH && (FUSED || DET)), "coherent loads: plain form only");
  static_assert(!(LOCAL && (FUSED || DET || COH)), "owner-computes form: plain gathers");
  const CCTab<T> &tb = cct<T>();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool pad = lane >= 3 * CPW;
  const int c = pad ? 0 : lane / CPW;
  const int s = pad ? 0 : lane - c * CPW;
  bool valid;
  int cx = 0, cy = 0, cz = 0;
  if (!DET) {
    const long long cell_raw = group * CPW + s;
    valid = !pad && cell_raw < L.n_cells;
    const long long cl = valid ? cell_raw : 0;
    cx = (int)(cl % L.n[0]);
    const long long rr = cl / L.n[0];
    cy = (int)(rr % L.n[1]);
    cz = (int)(rr / L.n[1]);
  } else {
    const long long ex = colour_extent(L.n, colour, 0), ey = colour_extent(L.n, colour, 1);
    const long long ez = colour_extent(L.n, colour, 2);
    const long long k = group * CPW + s;
    valid = !pad && k < ex * ey * ez;
    if (valid) {
      cx = 2 * (int)(k % ex) + (colour & 1);
      cy = 2 * (int)((k / ex) % ey) + ((colour >> 1) & 1);
      cz = 2 * (int)(k / (ex * ey)) + ((colour >> 2) & 1);
    }
  }
  const long long cell = ((long long)cz * L.n[1] + cy) * L.n[0] + cx;
  const int gx0 = K * cx, gy0 = K * cy, gz0 = K * cz;

  // free (unconstrained) velocity nodes per direction; invalid lanes have none
  bool fx[NV], fy[NV], fz[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    fx[i] = valid && !((L.faces & 1u) && gx0 + i == 0) && !((L.faces & 2u) && gx0 + i == L.N[0] - 1);
    fy[i] = !((L.faces & 4u) && gy0 + i == 0) && !((L.faces & 8u) && gy0 + i == L.N[1] - 1);
    fz[i] = !((L.faces & 16u) && gz0 + i == 0) && !((L.faces & 32u) && gz0 + i == L.N[2] - 1);
  }
  const long long N0 = L.N[0], N01 = (long long)L.N[0] * L.N[1];
  const long long vbase = c * L.nv + ((long long)gz0 * L.N[1] + gy0) * N0 + gx0;
  // A warp whose cells all lie inside (every node free; idle lanes do not count) gathers and
  // scatters without per-node predicates.
  bool interior = true;
#pragma unroll
  for (int i = 0; i < NV; ++i) interior = interior && fx[i] && fy[i] && fz[i];
  const bool fast = __all_sync(0xffffffffu, interior || pad);

  // ---- gathers --------------------------------------------------------------------------------
  T uv[NV][NV][NV];
  const T *ub = u + vbase;
  if constexpr (FUSED) {
    bool ox[NV], oy[NV], oz[NV];  // this cell owns the node (local index below the last, or last cell)
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      ox[i] = valid && (i < K || cx == L.n[0] - 1);
      oy[i] = i < K || cy == L.n[1] - 1;
      oz[i] = i < K || cz == L.n[2] - 1;
    }
#pragma unroll
    for (int iz = 0; iz < NV; ++iz)
#pragma unroll
      for (int iy = 0; iy < NV; ++iy)
#pragma unroll
        for (int ix = 0; ix < NV; ++ix) {
          const long long gi = vbase + iz * N01 + iy * N0 + ix;
          const bool fr = fx[ix] && fy[iy] && fz[iz];
          const bool own = ox[ix] && oy[iy] && oz[iz];
          T val = T(0);
          if ((fr && NEED_U) || (own && F.vstore)) {
            if (F.nv > 0) {
              T sum = F.vc[0] * F.vv[0][gi];
#pragma unroll
              for (int j = 1; j < kFuseVel; ++j)
                if (j < F.nv) sum += F.vc[j] * F.vv[j][gi];
              val = (F.vb ? F.vb[gi] : T(0)) + (F.vd ? F.vd[gi] : T(1)) * sum;
            } else {
              val = u[gi];
            }
          }
          uv[iz][iy][ix] = fr ? val : T(0);
          if (own) {
            if (F.vstore) F.vstore[gi] = val;
            if (F.vzero[0]) F.vzero[0][gi] = T(0);
            if (F.vzero[1]) F.vzero[1][gi] = T(0);
          }
        }
  } else if (NEED_U && !CART) {
    if (fast) {
#pragma unroll
      for (int iz = 0; iz < NV; ++iz)
#pragma unroll
        for (int iy = 0; iy < NV; ++iy)
#pragma unroll
          for (int ix = 0; ix < NV; ++ix) uv[iz][iy][ix] = ld_in<COH>(ub + iz * N01 + iy * N0 + ix);
    } else {
#pragma unroll
      for (int iz = 0; iz < NV; ++iz)
#pragma unroll
        for (int iy = 0; iy < NV; ++iy)
#pragma unroll
          for (int ix = 0; ix < NV; ++ix)
            uv[iz][iy][ix] = (fx[ix] && fy[iy] && fz[iz]) ? ld_in<COH>(ub + iz * N01 + iy * N0 + ix) : T(0);
    }
  }
  T pv[NPR][NPR][NPR];
  const long long P0 = L.Pn[0], P01 = (long long)L.Pn[0] * L.Pn[1];
  const long long pbase = ((long long)((K - 1) * cz) * L.Pn[1] + (K - 1) * cy) * P0 + (K - 1) * cx;
  if (DO_BT && FUSED) {
#pragma unroll
    for (int a3 = 0; a3 < NPR; ++a3)
#pragma unroll
      for (int a2 = 0; a2 < NPR; ++a2)
#pragma unroll
        for (int a1 = 0; a1 < NPR; ++a1) {
          const long long gi = pbase + a3 * P01 + a2 * P0 + a1;
          T val = T(0);
          if (valid) {
            if (F.np > 0) {
              T sum = T(0);
#pragma unroll
              for (int j = 0; j < kFusePre; ++j)
                if (j < F.np) sum += F.pc[j] * F.pv[j][gi];
              val = F.pd[gi] * sum;
            } else {
              val = p[gi];
            }
          }
          pv[a3][a2][a1] = val;
          const bool pown = valid && c == 0 && (a1 < K - 1 || cx == L.n[0] - 1) && (a2 < K - 1 || cy == L.n[1] - 1) &&
                            (a3 < K - 1 || cz == L.n[2] - 1);
          if (pown) {
            if (F.pacc) F.pacc[gi] += val;
#pragma unroll
            for (int j = 0; j < kFusePre; ++j)
              if (F.pzero[j]) F.pzero[j][gi] = T(0);
          }
        }
  } else if (DO_BT && !CART) {
#pragma unroll
    for (int a3 = 0; a3 < NPR; ++a3)
#pragma unroll
      for (int a2 = 0; a2 < NPR; ++a2)
#pragma unroll
        for (int a1 = 0; a1 < NPR; ++a1)
          pv[a3][a2][a1] = valid ? ld_in<COH>(p + pbase + a3 * P01 + a2 * P0 + a1) : T(0);
  }
  const T mu = L.mu_cell ? L.mu_cell[cell] : L.mu;

  T yv[NV][NV][NV];   // velocity test-function sums (nodal) of this component
  T qn[NPR][NPR][NPR];  // pressure test-function sums of this component's B u_c
  if constexpr (CART) {
    // Kronecker form, one x-slice (all (z, y) nodes at x-node i) at a time so that only the
    // output tensor, a slice and its transforms are live:
    //   A u_c = ax Kh x Mh x Mh + ay Mh x Kh x Mh + az Mh x Mh x Kh + be Mh x Mh x Mh  (x, y, z)
    //   B u_c = (Bx x By x Bz) u_c,  B^T p = (Bx x By x Bz)^T p
    // with ax = mu h_y h_z / h_x (and cyclic), be = gamma rho h_x h_y h_z; the 1D factors of B are
    // Gh along the component's own direction and Nh along the others, scaled by -prod_{d != c} h_d.
    const T h0 = L.h[0], h1 = L.h[1], h2 = L.h[2];
    const T bsc = -(c == 0 ? h1 * h2 : (c == 1 ? h0 * h2 : h0 * h1));
    T Bx[NPR][NV], By[NPR][NV], Bz[NPR][NV];  // lane-dependent (component c); Bz carries bsc
    if (DO_B || DO_BT) {
#pragma unroll
      for (int a = 0; a < NPR; ++a)
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          const T g = tb.Gh[a * NV + j], n = tb.Nh[a * NV + j];
          Bx[a][j] = c == 0 ? g : n;
          By[a][j] = c == 1 ? g : n;
          Bz[a][j] = bsc * (c == 2 ? g : n);
        }
    }
    const T ax = mu * h1 * h2 / h0, ay = mu * h0 * h2 / h1, az = mu * h0 * h1 / h2;
    const T be = L.gamma_rho * h0 * h1 * h2;
    if (DO_A || DO_BT) {
#pragma unroll
      for (int z = 0; z < NV; ++z)
#pragma unroll
        for (int y = 0; y < NV; ++y)
#pragma unroll
          for (int x = 0; x < NV; ++x) yv[z][y][x] = T(0);
    }
    if (DO_B) {
#pragma unroll
      for (int a3 = 0; a3 < NPR; ++a3)
#pragma unroll
        for (int a2 = 0; a2 < NPR; ++a2)
#pragma unroll
          for (int a1 = 0; a1 < NPR; ++a1) qn[a3][a2][a1] = T(0);
    }
    if (NEED_U) {
      // FP64 and k = 3: the slice loop stays rolled (registers for the output tensor first)
      constexpr int SLICE_UNROLL = (K == 2 && (sizeof(T) == 4 || FUSED)) ? NV : SMF_CC_SLICE_UNROLL;
      unsigned fxm = 0;
#pragma unroll
      for (int i = 0; i < NV; ++i) fxm |= fx[i] ? (1u << i) : 0u;
#pragma unroll SLICE_UNROLL
      for (int i = 0; i < NV; ++i) {
        T sl[NV][NV];  // [z][y] at x-node i
        const bool fxi = (fxm >> i) & 1u;
#pragma unroll
        for (int z = 0; z < NV; ++z)
#pragma unroll
          for (int y = 0; y < NV; ++y)
            sl[z][y] = FUSED ? uv[z][y][i]
                             : ((fast || (fxi && fy[y] && fz[z])) ? ld_in<COH>(ub + z * N01 + y * N0 + i) : T(0));
        if (DO_B) {
          T t1[NV][NPR];
#pragma unroll
          for (int z = 0; z < NV; ++z)
#pragma unroll
            for (int b = 0; b < NPR; ++b) {
              T acc = By[b][0] * sl[z][0];
#pragma unroll
              for (int y = 1; y < NV; ++y) acc += By[b][y] * sl[z][y];
              t1[z][b] = acc;
            }
#pragma unroll
          for (int a3 = 0; a3 < NPR; ++a3)
#pragma unroll
            for (int b = 0; b < NPR; ++b) {
              T q = Bz[a3][0] * t1[0][b];
#pragma unroll
              for (int z = 1; z < NV; ++z) q += Bz[a3][z] * t1[z][b];
#pragma unroll
              for (int a = 0; a < NPR; ++a) qn[a3][b][a] += Bx[a][i] * q;
            }
        }
        if constexpr (DO_A && sizeof(T) == 4) {
          // the same sweeps with the Mh and Kh results of a node in one register pair: packed
          // FP32 multiply-adds (two per instruction, the same roundings)
          const float2 *MK = reinterpret_cast<const float2 *>(tb.MK);
          const float2 *MM = reinterpret_cast<const float2 *>(tb.MM);
          float2 a12[NV][NV];  // [z][y']: (Mh, Kh) along y
#pragma unroll
          for (int z = 0; z < NV; ++z)
#pragma unroll
            for (int yo = 0; yo < NV; ++yo) {
              float2 acc = __fmul2_rn(MK[yo * NV], make_float2(sl[z][0], sl[z][0]));
#pragma unroll
              for (int y = 1; y < NV; ++y) acc = __ffma2_rn(MK[yo * NV + y], make_float2(sl[z][y], sl[z][y]), acc);
              a12[z][yo] = acc;
            }
#pragma unroll
          for (int zo = 0; zo < NV; ++zo)
#pragma unroll
            for (int y = 0; y < NV; ++y) {
              float2 vt = __fmul2_rn(MM[zo * NV], a12[0][y]);  // (v, t2): Mh along z of (a1, a2)
              T t3 = tb.Kh[zo * NV] * a12[0][y].x;
#pragma unroll
              for (int z = 1; z < NV; ++z) {
                vt = __ffma2_rn(MM[zo * NV + z], a12[z][y], vt);
                t3 += tb.Kh[zo * NV + z] * a12[z][y].x;
              }
              const T w = ay * vt.y + az * t3 + be * vt.x;
              const T av = ax * vt.x;
#pragma unroll
              for (int j = 0; j < NV; ++j) yv[zo][y][j] += tb.Kh[j * NV + i] * av + tb.Mh[j * NV + i] * w;
            }
        } else if (DO_A) {
          T a1[NV][NV], a2[NV][NV];  // [z][y']: Mh and Kh along y
#pragma unroll
          for (int z = 0; z < NV; ++z)
#pragma unroll
            for (int yo = 0; yo < NV; ++yo) {
              T m = tb.Mh[yo * NV] * sl[z][0], k = tb.Kh[yo * NV] * sl[z][0];
#pragma unroll
              for (int y = 1; y < NV; ++y) {
                m += tb.Mh[yo * NV + y] * sl[z][y];
                k += tb.Kh[yo * NV + y] * sl[z][y];
              }
              a1[z][yo] = m;
              a2[z][yo] = k;
            }
#pragma unroll
          for (int zo = 0; zo < NV; ++zo)
#pragma unroll
            for (int y = 0; y < NV; ++y) {
              T v = tb.Mh[zo * NV] * a1[0][y], t2 = tb.Mh[zo * NV] * a2[0][y], t3 = tb.Kh[zo * NV] * a1[0][y];
#pragma unroll
              for (int z = 1; z < NV; ++z) {
                v += tb.Mh[zo * NV + z] * a1[z][y];
                t2 += tb.Mh[zo * NV + z] * a2[z][y];
                t3 += tb.Kh[zo * NV + z] * a1[z][y];
              }
              const T w = ay * t2 + az * t3 + be * v;
              const T av = ax * v;
#pragma unroll
              for (int j = 0; j < NV; ++j) yv[zo][y][j] += tb.Kh[j * NV + i] * av + tb.Mh[j * NV + i] * w;
            }
        }
      }
    }
    if (DO_BT) {  // yv += (Bx x By x Bz)^T p, one pressure x-slice at a time
#pragma unroll
      for (int a = 0; a < NPR; ++a) {
        T ps[NPR][NPR];  // [c3][b] at pressure x-node a
#pragma unroll
        for (int c3 = 0; c3 < NPR; ++c3)
#pragma unroll
          for (int b = 0; b < NPR; ++b)
            ps[c3][b] = FUSED ? pv[c3][b][a] : (valid ? ld_in<COH>(p + pbase + c3 * P01 + b * P0 + a) : T(0));
        T t[NPR][NV];  // [c3][y]
#pragma unroll
        for (int c3 = 0; c3 < NPR; ++c3)
#pragma unroll
          for (int y = 0; y < NV; ++y) {
            T acc = By[0][y] * ps[c3][0];
#pragma unroll
            for (int b = 1; b < NPR; ++b) acc += By[b][y] * ps[c3][b];
            t[c3][y] = acc;
          }
#pragma unroll
        for (int z = 0; z < NV; ++z)
#pragma unroll
          for (int y = 0; y < NV; ++y) {
            T r = Bz[0][z] * t[0][y];
#pragma unroll
            for (int c3 = 1; c3 < NPR; ++c3) r += Bz[c3][z] * t[c3][y];
#pragma unroll
            for (int j = 0; j < NV; ++j) yv[z][y][j] += Bx[a][j] * r;
          }
      }
    }
  } else {
    // ---- trilinear geometry: plane qz = c of this cell, shared through shared memory ----------
    constexpr int NF = CcGeo<MODE>::NF;
    extern __shared__ float4 cc_geo_smem[];
    float4 *gs = cc_geo_smem + (size_t)warp * (NQ * NQ * NQ * NF * CPW);
    if constexpr (CL::SMEM_GEO) {
      T X[8][3];
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const long long gv =
            ((long long)(cz + ((v >> 2) & 1)) * (L.n[1] + 1) + (cy + ((v >> 1) & 1))) * (L.n[0] + 1) + (cx + (v & 1));
#pragma unroll
        for (int a = 0; a < 3; ++a) X[v][a] = L.vert[gv * 3 + a];
      }
      // edge vectors: ex[y][z] along x, ey[x][z] along y, ez[x][y] along z (vertex v = x + 2y + 4z)
      const T zeta = tb.X[c], wz = tb.W[c];
      T ce[2][3], cf[2][3], ez[2][2][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          const T e0 = X[1 + 2 * y][a] - X[2 * y][a], e1 = X[5 + 2 * y][a] - X[4 + 2 * y][a];
          ce[y][a] = e0 + zeta * (e1 - e0);
        }
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          const T f0 = X[x + 2][a] - X[x][a], f1 = X[x + 6][a] - X[x + 4][a];
          cf[x][a] = f0 + zeta * (f1 - f0);
        }
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
          for (int y = 0; y < 2; ++y) ez[x][y][a] = X[x + 2 * y + 4][a] - X[x + 2 * y][a];
      }
      const T grho = L.gamma_rho;
#pragma unroll
      for (int qy = 0; qy < NQ; ++qy) {
        const T eta = tb.X[qy];
        T c0[3], gl[2][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          c0[a] = ce[0][a] + eta * (ce[1][a] - ce[0][a]);
#pragma unroll
          for (int x = 0; x < 2; ++x) gl[x][a] = ez[x][0][a] + eta * (ez[x][1][a] - ez[x][0][a]);
        }
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) {
          const T xi = tb.X[qx];
          T c1[3], c2[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            c1[a] = cf[0][a] + xi * (cf[1][a] - cf[0][a]);
            c2[a] = gl[0][a] + xi * (gl[1][a] - gl[0][a]);
          }
          // rows of adj(J) for J = [c0 c1 c2]: c1 x c2, c2 x c0, c0 x c1
          T r[3][3];
          r[0][0] = c1[1] * c2[2] - c1[2] * c2[1];
          r[0][1] = c1[2] * c2[0] - c1[0] * c2[2];
          r[0][2] = c1[0] * c2[1] - c1[1] * c2[0];
          r[1][0] = c2[1] * c0[2] - c2[2] * c0[1];
          r[1][1] = c2[2] * c0[0] - c2[0] * c0[2];
          r[1][2] = c2[0] * c0[1] - c2[1] * c0[0];
          r[2][0] = c0[1] * c1[2] - c0[2] * c1[1];
          r[2][1] = c0[2] * c1[0] - c0[0] * c1[2];
          r[2][2] = c0[0] * c1[1] - c0[1] * c1[0];
          const T w = tb.W[qx] * tb.W[qy] * wz;
          const int pt = (c * NQ + qy) * NQ + qx;
          constexpr int NA = CcGeo<MODE>::NA;
          if (!pad) {
            float4 *g = gs + (size_t)pt * NF * CPW + s;
            if constexpr (NA > 0) {  // the A block's metric (the B blocks need only w adj(J))
              const T det = c0[0] * r[0][0] + c0[1] * r[0][1] + c0[2] * r[0][2];
              const T wd = __fdividef(mu * w, det);
              auto dot = [&](int i, int j) { return r[i][0] * r[j][0] + r[i][1] * r[j][1] + r[i][2] * r[j][2]; };
              g[0] = make_float4(wd * dot(0, 0), wd * dot(0, 1), wd * dot(0, 2), wd * dot(1, 1));
              g[CPW] = make_float4(wd * dot(1, 2), wd * dot(2, 2), grho * w * det, 0.f);
            }
            if constexpr (CcGeo<MODE>::NB > 0) {
#pragma unroll
              for (int j = 0; j < 3; ++j) g[(NA + j) * CPW] = make_float4(w * r[0][j], w * r[1][j], w * r[2][j], 0.f);
            }
          }
        }
      }
      __syncwarp();
    }
    // FP64: the per-point factors stored at setup, [cell][field][qz][qy][qx]: G (6, mu
    // included), w adj (9, row-major), gamma rho w det (1)
    constexpr int GST = NQ * NQ * NQ;
    const T *gc = CL::SMEM_GEO ? nullptr : geo + cell * (long long)(16 * GST);

    // ---- this component at the Gauss points --------------------------------------------------
    auto Sf = [&](int i, int j) { return tb.S[i * NV + j]; };
    auto St = [&](int i, int j) { return tb.S[j * NV + i]; };
    auto Pf = [&](int i, int j) { return tb.P[i * NPR + j]; };
    auto Pt = [&](int i, int j) { return tb.P[j * NPR + i]; };
    T uq[NQ][NQ][NQ];
    if (NEED_U) {
      T t1[NV][NV][NQ], t2[NV][NQ][NQ];
      cc_sweep0<NV, NQ, NV, NV>(uv, t1, Sf);
      cc_sweep1<NV, NQ, NQ, NV>(t1, t2, Sf);
      cc_sweep2<NV, NQ, NQ, NQ>(t2, uq, Sf);
    }
    T pq[NQ][NQ][NQ];
    if (DO_BT) {
      T t1[NPR][NPR][NQ], t2[NPR][NQ][NQ];
      cc_sweep0<NPR, NQ, NPR, NPR>(pv, t1, Pf);
      cc_sweep1<NPR, NQ, NQ, NPR>(t1, t2, Pf);
      cc_sweep2<NPR, NQ, NQ, NQ>(t2, pq, Pf);
    }
    T tq[NQ][NQ][NQ], qacc[NQ][NQ][NQ];
#pragma unroll
    for (int qz = 0; qz < NQ; ++qz)
#pragma unroll
      for (int qy = 0; qy < NQ; ++qy)
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) tq[qz][qy][qx] = T(0);
#pragma unroll
    for (int qz = 0; qz < NQ; ++qz)
#pragma unroll
      for (int qy = 0; qy < NQ; ++qy)
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) {
          const int pt = (qz * NQ + qy) * NQ + qx;
          const float4 *g = gs + (size_t)pt * NF * CPW + s;
          // G00 G01 G02 G11 G12 G22 (mu included), gamma rho w det, column c of w adj
          auto geo_G = [&](T(&gg)[7]) {
            if constexpr (CL::SMEM_GEO) {
              const float4 g0 = g[0], g1 = g[CPW];
              gg[0] = g0.x; gg[1] = g0.y; gg[2] = g0.z; gg[3] = g0.w; gg[4] = g1.x; gg[5] = g1.y; gg[6] = g1.z;
            } else {
#pragma unroll
              for (int i = 0; i < 6; ++i) gg[i] = gc[i * GST + pt];
              gg[6] = gc[15 * GST + pt];
            }
          };
          auto geo_C = [&](T(&cc)[3]) {
            if constexpr (CL::SMEM_GEO) {
              const float4 v = g[(CcGeo<MODE>::NA + c) * CPW];
              cc[0] = v.x; cc[1] = v.y; cc[2] = v.z;
            } else {
#pragma unroll
              for (int a = 0; a < 3; ++a) cc[a] = gc[(6 + 3 * a + c) * GST + pt];
            }
          };
          T gx = T(0), gy = T(0), gz = T(0);
          if (NEED_U) {
#pragma unroll
            for (int m = 0; m < NQ; ++m) {
              gx += tb.D[qx * NQ + m] * uq[qz][qy][m];
              gy += tb.D[qy * NQ + m] * uq[qz][m][qx];
              gz += tb.D[qz * NQ + m] * uq[m][qy][qx];
            }
          }
          T f0 = T(0), f1 = T(0), f2 = T(0);
          if (DO_A) {
            T G[7];
            geo_G(G);
            f0 = G[0] * gx + G[1] * gy + G[2] * gz;
            f1 = G[1] * gx + G[3] * gy + G[4] * gz;
            f2 = G[2] * gx + G[4] * gy + G[5] * gz;
            tq[qz][qy][qx] += G[6] * uq[qz][qy][qx];
          }
          if (DO_B || DO_BT) {
            T cc[3];
            geo_C(cc);
            if (DO_BT) {
              f0 -= pq[qz][qy][qx] * cc[0];
              f1 -= pq[qz][qy][qx] * cc[1];
              f2 -= pq[qz][qy][qx] * cc[2];
            }
            if (DO_B) qacc[qz][qy][qx] = -(cc[0] * gx + cc[1] * gy + cc[2] * gz);
          }
          if (DO_A || DO_BT) {
#pragma unroll
            for (int m = 0; m < NQ; ++m) {
              tq[qz][qy][m] += tb.D[qx * NQ + m] * f0;
              tq[qz][m][qx] += tb.D[qy * NQ + m] * f1;
              tq[m][qy][qx] += tb.D[qz * NQ + m] * f2;
            }
          }
        }
    if (DO_A || DO_BT) {
      T t1[NV][NQ][NQ], t2[NV][NV][NQ];
      cc_sweep2<NQ, NV, NQ, NQ>(tq, t1, St);
      cc_sweep1<NQ, NV, NQ, NV>(t1, t2, St);
      cc_sweep0<NQ, NV, NV, NV>(t2, yv, St);
    }
    if (DO_B) {
      T t1[NPR][NQ][NQ], t2[NPR][NPR][NQ];
      cc_sweep2<NQ, NPR, NQ, NQ>(qacc, t1, Pt);
      cc_sweep1<NQ, NPR, NQ, NPR>(t1, t2, Pt);
      cc_sweep0<NQ, NPR, NPR, NPR>(t2, qn, Pt);
    }
  }

  // ---- scatter ---------------------------------------------------------------------------------
  if constexpr (LOCAL) {
    if (valid) {
      const long long nc = L.n_cells;
      if (DO_A || DO_BT) {
#pragma unroll
        for (int iz = 0; iz < NV; ++iz)
#pragma unroll
          for (int iy = 0; iy < NV; ++iy)
#pragma unroll
            for (int ix = 0; ix < NV; ++ix)
              yu[((long long)((iz * NV + iy) * NV + ix) * 3 + c) * nc + cell] = yv[iz][iy][ix];
      }
      if (DO_B) {
#pragma unroll
        for (int a3 = 0; a3 < NPR; ++a3)
#pragma unroll
          for (int a2 = 0; a2 < NPR; ++a2)
#pragma unroll
            for (int a1 = 0; a1 < NPR; ++a1)
              yp[((long long)((a3 * NPR + a2) * NPR + a1) * 3 + c) * nc + cell] = qn[a3][a2][a1];
      }
    }
    __syncwarp();
    return;
  }
  if (DO_A || DO_BT) {
    T *yb = yu + vbase;
    if (DET) {
#pragma unroll
      for (int iz = 0; iz < NV; ++iz)
#pragma unroll
        for (int iy = 0; iy < NV; ++iy)
#pragma unroll
          for (int ix = 0; ix < NV; ++ix)
            if (fx[ix] && fy[iy] && fz[iz]) {
              T *a = &yb[iz * N01 + iy * N0 + ix];
              __stcg(a, __ldcg(a) + yv[iz][iy][ix]);
            }
    } else if (fast) {
      if (!pad) {
#pragma unroll
        for (int iz = 0; iz < NV; ++iz)
#pragma unroll
          for (int iy = 0; iy < NV; ++iy)
#pragma unroll
            for (int ix = 0; ix < NV; ++ix) atomicAdd(&yb[iz * N01 + iy * N0 + ix], yv[iz][iy][ix]);
      }
    } else {
#pragma unroll
      for (int iz = 0; iz < NV; ++iz)
#pragma unroll
        for (int iy = 0; iy < NV; ++iy)
#pragma unroll
          for (int ix = 0; ix < NV; ++ix)
            if (fx[ix] && fy[iy] && fz[iz]) atomicAdd(&yb[iz * N01 + iy * N0 + ix], yv[iz][iy][ix]);
    }
  }
  if (DO_B) {
    constexpr int NP3 = NPR * NPR * NPR;
    if (DET) {
      // the cell's three component sums meet in shared memory; component 0 adds them in order
      extern __shared__ float4 cc_geo_smem[];
      T *red = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(cc_geo_smem) + CL::GEO_BYTES) +
               (size_t)warp * CPW * 3 * NP3;
      if (!pad) {
#pragma unroll
        for (int a3 = 0; a3 < NPR; ++a3)
#pragma unroll
          for (int a2 = 0; a2 < NPR; ++a2)
#pragma unroll
            for (int a1 = 0; a1 < NPR; ++a1) red[(s * 3 + c) * NP3 + (a3 * NPR + a2) * NPR + a1] = qn[a3][a2][a1];
      }
      __syncwarp();
      if (valid && c == 0) {
#pragma unroll
        for (int a3 = 0; a3 < NPR; ++a3)
#pragma unroll
          for (int a2 = 0; a2 < NPR; ++a2)
#pragma unroll
            for (int a1 = 0; a1 < NPR; ++a1) {
              const int e = (a3 * NPR + a2) * NPR + a1;
              const T v = (red[(s * 3 + 0) * NP3 + e] + red[(s * 3 + 1) * NP3 + e]) + red[(s * 3 + 2) * NP3 + e];
              T *a = &yp[pbase + a3 * P01 + a2 * P0 + a1];
              __stcg(a, __ldcg(a) + v);
            }
      }
    } else if (valid) {
#pragma unroll
      for (int a3 = 0; a3 < NPR; ++a3)
#pragma unroll
        for (int a2 = 0; a2 < NPR; ++a2)
#pragma unroll
          for (int a1 = 0; a1 < NPR; ++a1) atomicAdd(&yp[pbase + a3 * P01 + a2 * P0 + a1], qn[a3][a2][a1]);
    }
  }
  __syncwarp();  // the warp's shared memory is reused by its next group
}

template <int K, typename T, int MODE, bool CART>
__global__ void __launch_bounds__(32 * CcLaunch<K, T, MODE, CART>::WARPS, CcLaunch<K, T, MODE, CART>::MINB)
    stokes_cell_apply_cc(const LevelDesc<T> L, const T *__restrict__ u, const T *__restrict__ p,
                         T *__restrict__ yu, T *__restrict__ yp, const T *__restrict__ geo) {
  pdl_enter();
  cc_group<K, T, MODE, CART, false>(L, u, p, yu, yp, geo,
                                    (long long)blockIdx.x * CcLaunch<K, T, MODE, CART>::WARPS + (threadIdx.x >> 5), -1);
}

// Fused smoothing form (k = 2): inputs and owner side effects from the Fuse descriptor.
template <int K, typename T, int MODE, bool CART>
__global__ void __launch_bounds__(32 * CcLaunch<K, T, MODE, CART>::WARPS, CcLaunch<K, T, MODE, CART>::MINB)
    stokes_cell_apply_cc_fused(const LevelDesc<T> L, const T *__restrict__ u, const T *__restrict__ p,
                               T *__restrict__ yu, T *__restrict__ yp, const T *__restrict__ geo, const Fuse<T> F) {
  pdl_enter();
  cc_group<K, T, MODE, CART, false, true>(
      L, u, p, yu, yp, geo, (long long)blockIdx.x * CcLaunch<K, T, MODE, CART>::WARPS + (threadIdx.x >> 5), -1, F);
}

// Owner-computes deterministic form, pass 1: every (cell, component) thread stores its local results.
template <int K, typename T, int MODE, bool CART>
__global__ void __launch_bounds__(32 * CcLaunch<K, T, MODE, CART>::WARPS, CcLaunch<K, T, MODE, CART>::MINB)
    stokes_cell_apply_cc_local(const LevelDesc<T> L, const T *__restrict__ u, const T *__restrict__ p,
                               T *__restrict__ lu, T *__restrict__ lp, const T *__restrict__ geo) {
  pdl_enter();
  cc_group<K, T, MODE, CART, false, false, false, true>(
      L, u, p, lu, lp, geo, (long long)blockIdx.x * CcLaunch<K, T, MODE, CART>::WARPS + (threadIdx.x >> 5), -1);
}

// The cells holding global node g along one axis (node spacing s = k for velocity, k - 1 for
// pressure, n cells): g = s c + a.  Interior-of-cell nodes have one (cell, local index), nodes on a
// cell boundary two (the lower cell's last index first), the domain ends one.
__device__ __forceinline__ int owner_cells(int g, int s, int n, int (&cell)[2], int (&loc)[2]) {
  const int c = g / s, a = g - c * s;
  if (a != 0) {
    cell[0] = c;
    loc[0] = a;
    return 1;
  }
  int m = 0;
  if (c > 0) {
    cell[m] = c - 1;
    loc[m] = s;
    ++m;
  }
  if (c < n) {
    cell[m] = c;
    loc[m] = 0;
    ++m;
  }
  return m;
}

// Pass 2: y += the sum of the local results of every cell holding the DoF, cells in a fixed
// (z, y, x) order and, for pressure, the three component parts of a cell summed first: the same
// operator as the atomic scatter (the paper's K x = sum_tau P_tau K_tau P_tau^T x), bitwise
// reproducible.  Constrained velocity DoFs are left alone.
template <int K, typename T>
__global__ void k_cc_owner_gather(const LevelDesc<T> L, const T *__restrict__ lu, const T *__restrict__ lp,
                                  T *__restrict__ yu, T *__restrict__ yp, int do_u, int do_p) {
  pdl_enter();
  constexpr int NV = K + 1, NPR = K;
  const long long nc = L.n_cells, nu = do_u ? L.n_u : 0, np = do_p ? L.n_p : 0;
  SMF_GRID_LOOP(i, nu + np) {
    int cx[2], ax[2], cy[2], ay[2], cz[2], az[2];
    if (i < nu) {
      const int c = (int)(i / L.nv);
      const long long j = i - c * L.nv;
      const int gx = (int)(j % L.N[0]), gy = (int)((j / L.N[0]) % L.N[1]), gz = (int)(j / ((long long)L.N[0] * L.N[1]));
      if (vel_constrained(L.N, L.faces, 3, gx, gy, gz)) continue;
      const int mx = owner_cells(gx, K, L.n[0], cx, ax), my = owner_cells(gy, K, L.n[1], cy, ay),
                mz = owner_cells(gz, K, L.n[2], cz, az);
      T s = T(0);
      for (int z = 0; z < mz; ++z)
        for (int y = 0; y < my; ++y)
          for (int x = 0; x < mx; ++x) {
            const long long cell = ((long long)cz[z] * L.n[1] + cy[y]) * L.n[0] + cx[x];
            const int loc = (az[z] * NV + ay[y]) * NV + ax[x];
            s += lu[((long long)loc * 3 + c) * nc + cell];
          }
      yu[i] += s;
    } else {
      const long long j = i - nu;
      const int px = (int)(j % L.Pn[0]), py = (int)((j / L.Pn[0]) % L.Pn[1]),
                pz = (int)(j / ((long long)L.Pn[0] * L.Pn[1]));
      const int mx = owner_cells(px, K - 1, L.n[0], cx, ax), my = owner_cells(py, K - 1, L.n[1], cy, ay),
                mz = owner_cells(pz, K - 1, L.n[2], cz, az);
      T s = T(0);
      for (int z = 0; z < mz; ++z)
        for (int y = 0; y < my; ++y)
          for (int x = 0; x < mx; ++x) {
            const long long cell = ((long long)cz[z] * L.n[1] + cy[y]) * L.n[0] + cx[x];
            const long long base = (long long)((az[z] * NPR + ay[y]) * NPR + ax[x]) * 3 * nc + cell;
            s += (lp[base] + lp[base + nc]) + lp[base + 2 * nc];
          }
      yp[j] += s;
    }
  }
}

// Deterministic form: one cooperative launch walks the 8 colour classes of cells in order, each
// class by all CTAs (a warp per group of 10 cells), with a grid barrier between classes.  The
// barrier waits are bounded (GridBarrier::budget); a wait that runs out sets the error flag and
// every CTA returns.
template <int K, typename T, int MODE, bool CART>
__global__ void __launch_bounds__(32 * CcLaunch<K, T, MODE, CART>::WARPS, CcLaunch<K, T, MODE, CART>::MINB)
    stokes_cell_apply_cc_det(const LevelDesc<T> L, const T *__restrict__ u, const T *__restrict__ p,
                             T *__restrict__ yu, T *__restrict__ yp, const T *__restrict__ geo, const GridBarrier gb) {
  pdl_enter();
  constexpr int WARPS = CcLaunch<K, T, MODE, CART>::WARPS;
  const long long wstride = (long long)gridDim.x * WARPS;
  for (int colour = 0; colour < 8; ++colour) {
    const long long cells = colour_extent(L.n, colour, 0) * colour_extent(L.n, colour, 1) *
                            colour_extent(L.n, colour, 2);
    const long long groups = (cells + kCcCells - 1) / kCcCells;
    for (long long g = (long long)blockIdx.x * WARPS + (threadIdx.x >> 5); g < groups; g += wstride)
      cc_group<K, T, MODE, CART, true>(L, u, p, yu, yp, geo, g, colour);
    if (colour < 7 && !grid_barrier(gb)) return;
  }
}

// The trilinear kernels keep their geometry in shared memory: ask for the largest shared-memory
// carveout so that occupancy is set by registers, not by the default L1 / shared split, and allow
// the launch's dynamic shared memory where it exceeds the default 48 KB.
template <typename F>
static cudaError_t cc_smem_attrs(F *kern, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}
template <int K, typename T, int MODE>
static cudaError_t cc_carveout_mode() {
  using CL = CcLaunch<K, T, MODE, false>;
  cudaError_t e = cc_smem_attrs(stokes_cell_apply_cc<K, T, MODE, false>, CL::SMEM);
  if (e == cudaSuccess) e = cc_smem_attrs(stokes_cell_apply_cc_det<K, T, MODE, false>, CL::SMEM_DET);
  if (e == cudaSuccess) e = cc_smem_attrs(stokes_cell_apply_cc_fused<K, T, MODE, false>, CL::SMEM);
  if (e == cudaSuccess) e = cc_smem_attrs(stokes_cell_apply_cc_local<K, T, MODE, false>, CL::SMEM);
  return e;
}
template <int K>
cudaError_t cc_prefer_shared() {
  if constexpr (K == 2) {
    cudaError_t e = cc_carveout_mode<2, float, kApplyA>();
    if (e == cudaSuccess) e = cc_carveout_mode<2, float, kApplyBT>();
    if (e == cudaSuccess) e = cc_carveout_mode<2, float, kApplyB>();
    if (e == cudaSuccess) e = cc_carveout_mode<2, float, kApplyA | kApplyBT>();
    if (e == cudaSuccess) e = cc_carveout_mode<2, float, kApplyA | kApplyBT | kApplyB>();
    return e;
  }
  return cudaSuccess;
}

template <int K, typename T, int MODE, bool CART>
static void launch_cc_mode(const LevelDesc<T> &L, const T *u, const T *p, T *yu, T *yp, const T *geo,
                           cudaStream_t s) {
  using CL = CcLaunch<K, T, MODE, CART>;
  const long long cpb = (long long)kCcCells * CL::WARPS;
  const long long blocks = (L.n_cells + cpb - 1) / cpb;
  launch_kernel(stokes_cell_apply_cc<K, T, MODE, CART>, dim3((unsigned)blocks), dim3(32 * CL::WARPS), CL::SMEM, s, L,
                u, p, yu, yp, geo);
}

// Cooperative launch of the deterministic form: at most as many CTAs as can be resident at once
// (the occupancy of this instantiation times the SM count), so that every CTA reaches every
// barrier; never more than the largest colour class needs.
template <int K, typename T, int MODE, bool CART>
static int launch_cc_det_mode(const LevelDesc<T> &L, const T *u, const T *p, T *yu, T *yp, const T *geo,
                              const GridBarrier &gb, cudaStream_t s) {
  using CL = CcLaunch<K, T, MODE, CART>;
  if (gb.owner) {  // owner-computes: local results, then the per-DoF sums
    T *lu = static_cast<T *>(sizeof(T) == 4 ? gb.loc32 : gb.loc64);
    T *lp = lu + (long long)3 * (K + 1) * (K + 1) * (K + 1) * L.n_cells;
    const long long cpb = (long long)kCcCells * CL::WARPS;
    launch_kernel(stokes_cell_apply_cc_local<K, T, MODE, CART>, dim3((unsigned)((L.n_cells + cpb - 1) / cpb)),
                  dim3(32 * CL::WARPS), CL::SMEM, s, L, u, p, lu, lp, geo);
    constexpr bool DU = MODE & (kApplyA | kApplyBT), DP = MODE & kApplyB;
    launch_kernel(k_cc_owner_gather<K, T>, dim3(vec_blocks((DU ? L.n_u : 0) + (DP ? L.n_p : 0))), dim3(kVecThreads), 0,
                  s, L, (const T *)lu, (const T *)lp, yu, yp, DU ? 1 : 0, DP ? 1 : 0);
    return (int)cudaGetLastError();
  }
  static int resident = -1;
  if (resident < 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stokes_cell_apply_cc_det<K, T, MODE, CART>,
                                                      32 * CL::WARPS, CL::SMEM_DET) != cudaSuccess)
      return (int)cudaGetLastError();
    resident = per_sm * sms;
  }
  if (resident <= 0) return (int)cudaErrorCooperativeLaunchTooLarge;
  long long biggest = 0;
  for (int colour = 0; colour < 8; ++colour)
    biggest = std::max(biggest, colour_extent(L.n, colour, 0) * colour_extent(L.n, colour, 1) *
                                    colour_extent(L.n, colour, 2));
  const long long cpb = (long long)kCcCells * CL::WARPS;
  const long long need = std::max(1ll, (biggest + cpb - 1) / cpb);
  const unsigned grid = (unsigned)std::min<long long>(need, resident);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32 * CL::WARPS);
  cfg.dynamicSmemBytes = CL::SMEM_DET;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, stokes_cell_apply_cc_det<K, T, MODE, CART>, L, u, p, yu, yp, geo, gb);
}

// Whether this kernel serves the level: 3D; Cartesian k = 2, 3; trilinear k = 2 in FP32, and in
// FP64 where the per-point geometry is stored (geo).
template <typename T>
inline bool cc_serves(const LevelDesc<T> &L, const T *geo) {
  if (!cc_level_supported(L.dim, L.k, L.cartesian, sizeof(T))) return false;
  return L.cartesian || sizeof(T) == 4 || geo != nullptr;
}

// Launches shape 5 for the modes the kernel has (A, B^T, B, A + B^T, full); -1 otherwise.
// det: the deterministic cooperative form with the grid barrier *det (returns a cudaError_t code
// > 0 when that launch fails).
template <int K, typename T>
int launch_cell_apply_cc_k(const LevelDesc<T> &L, int mode, const T *u, const T *p, T *yu, T *yp, const T *geo,
                           const GridBarrier *det, cudaStream_t s) {
  if (L.k != K || !cc_serves(L, geo)) return -1;
#define SMF_CC_CASE(M)                                                                   \
  case M:                                                                                \
    if (L.cartesian)                                                                     \
      return det ? launch_cc_det_mode<K, T, M, true>(L, u, p, yu, yp, geo, *det, s)      \
                 : (launch_cc_mode<K, T, M, true>(L, u, p, yu, yp, geo, s), 0);          \
    if constexpr (K == 2)                                                                \
      return det ? launch_cc_det_mode<K, T, M, false>(L, u, p, yu, yp, geo, *det, s)     \
                 : (launch_cc_mode<K, T, M, false>(L, u, p, yu, yp, geo, s), 0);         \
    return -1;
  switch (mode) {
    SMF_CC_CASE(kApplyA)
    SMF_CC_CASE(kApplyBT)
    SMF_CC_CASE(kApplyB)
    SMF_CC_CASE(kApplyA | kApplyBT)
    SMF_CC_CASE(kApplyA | kApplyBT | kApplyB)
    default: return -1;
  }
#undef SMF_CC_CASE
}

// Fused smoothing applications on a level served by this kernel (k = 2); -1 otherwise.
template <int K, typename T>
int launch_cell_apply_cc_fused_k(const LevelDesc<T> &L, int mode, const T *u, const T *p, T *yu, T *yp,
                                 const T *geo, const Fuse<T> &F, cudaStream_t s) {
  if constexpr (K != 2) {
    return -1;
  } else {
    if (L.k != 2 || !cc_serves(L, geo)) return -1;
#define SMF_CCF_CASE(M)                                                                                         \
  case M: {                                                                                                     \
    using CL = CcLaunch<2, T, M, false>;                                                                        \
    using CC = CcLaunch<2, T, M, true>;                                                                         \
    const long long cpb = (long long)kCcCells * (L.cartesian ? CC::WARPS : CL::WARPS);                          \
    const unsigned blocks = (unsigned)((L.n_cells + cpb - 1) / cpb);                                            \
    if (L.cartesian)                                                                                            \
      launch_kernel(stokes_cell_apply_cc_fused<2, T, M, true>, dim3(blocks), dim3(32 * CC::WARPS), CC::SMEM, s, L, \
                    u, p, yu, yp, geo, F);                                                                      \
    else                                                                                                        \
      launch_kernel(stokes_cell_apply_cc_fused<2, T, M, false>, dim3(blocks), dim3(32 * CL::WARPS), CL::SMEM, s, \
                    L, u, p, yu, yp, geo, F);                                                                   \
    return 0;                                                                                                   \
  }
    switch (mode) {
      SMF_CCF_CASE(kApplyA)
      SMF_CCF_CASE(kApplyBT)
      SMF_CCF_CASE(kApplyB)
      SMF_CCF_CASE(kApplyA | kApplyBT)
      SMF_CCF_CASE(kApplyA | kApplyBT | kApplyB)
      default: return -1;
    }
#undef SMF_CCF_CASE
  }
}

}  // namespace smf
