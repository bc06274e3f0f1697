// Grid transfers (paper Sec. 3.2): prolongation = canonical injection of the coarse
// Q_k x Q_{k-1} space into the fine one, restriction = its transpose.  On the structured
// hierarchy the injection is a tensor product of 1D matrices: fine node g along an axis lies in
// fine cell f (local node a), child h = f mod 2 of coarse cell c = f / 2, and takes the coarse
// basis values at reference coordinate (h + t_a)/2.  Constrained velocity DoFs are dropped on
// both sides (P_eff = Z_fine P Z_coarse); a node is free iff it is free along every axis, so the
// masks are tensor products too and are folded into the 1D weights.
//
// The 1D matrices of a level pair are stored per axis and space as padded rows of
// (node, weight) pairs without zeros: prolongation rows (per fine node, <= deg+1 entries) and
// restriction rows (per coarse node, <= 4 deg + 1 entries), built on the host at setup.  Both
// kernels are DoF-parallel, write every output once (no atomics) and sum the tensor-product
// terms in nested loops.
#pragma once
#include "common.cuh"
#include "vec.cuh"

namespace smf {

// One axis, one space: rows of up to W (node, weight) pairs.
template <typename T>
struct Xfer1D {
  const int *cnt = nullptr;  // [rows]
  const int *idx = nullptr;  // [rows * W]
  const T *w = nullptr;      // [rows * W]
};
// All 1D matrices of a level pair: [space: 0 velocity, 1 pressure][axis]; row width W = 4k + 1.
template <typename T>
struct XferTabs {
  Xfer1D<T> r[2][3];  // restriction: per coarse node, the fine nodes of its basis function's support
  Xfer1D<T> p[2][3];  // prolongation: per fine node, the coarse nodes of its coarse cell
  int W = 0;
};

// Restriction row of coarse DoF i (P^T in, or P^T (in - minus) with SUB), summed over its (z, y)
// term pairs t = t0, t0 + dt, ... (all of them for t0 = 0, dt = 1).
template <typename T, int W, bool SUB, bool COH = false>
__device__ __forceinline__ T restrict_terms(const LevelDesc<T> &F, const LevelDesc<T> &C, const XferTabs<T> &X,
                                            const T *in, const T *minus, long long i, int t0, int dt) {
  const bool vel = i < C.n_u;
  const int sp = vel ? 0 : 1;
  const int *Nc = vel ? C.N : C.Pn, *Nf = vel ? F.N : F.Pn;
  const long long j = vel ? i % C.nv : i - C.n_u;
  const int G0 = (int)(j % Nc[0]), G1 = (int)((j / Nc[0]) % Nc[1]), G2 = (int)(j / ((long long)Nc[0] * Nc[1]));
  const long long off = vel ? (i / C.nv) * F.nv : F.n_u;
  const T *src = in + off;
  const T *ssrc = SUB ? minus + off : nullptr;
  const Xfer1D<T> &ax = X.r[sp][0], &ay = X.r[sp][1], &az = X.r[sp][2];
  const int n0 = ax.cnt[G0], n1 = ay.cnt[G1], n2 = az.cnt[G2];
  int f0[W];
  T w0[W];
#pragma unroll
  for (int a = 0; a < W; ++a) {
    f0[a] = a < n0 ? ax.idx[G0 * W + a] : 0;
    w0[a] = a < n0 ? ax.w[G0 * W + a] : T(0);
  }
  T s = T(0);
  for (int t = t0; t < n1 * n2; t += dt) {
    const int a1 = t % n1, a2 = t / n1;
    const int f1 = ay.idx[G1 * W + a1], f2 = az.idx[G2 * W + a2];
    const T w21 = ay.w[G1 * W + a1] * az.w[G2 * W + a2];
    const long long ro = ((long long)f2 * Nf[1] + f1) * Nf[0];
    const T *row = src + ro;
    T r = T(0);
    if (SUB) {
      const T *srow = ssrc + ro;
#pragma unroll
      for (int a = 0; a < W; ++a)
        if (a < n0) r += w0[a] * (ld_in<COH>(row + f0[a]) - ld_in<COH>(srow + f0[a]));
    } else {
#pragma unroll
      for (int a = 0; a < W; ++a)
        if (a < n0) r += w0[a] * ld_in<COH>(row + f0[a]);
    }
    s += w21 * r;
  }
  return s;
}

// out (coarse) = P^T in (fine); zero_c (coarse-sized, may be null) is zeroed on the way.
// SUB: out = P^T (in - minus), the residual b - K x of Algorithm 1 formed while restricting it.
// LANES consecutive lanes share one coarse DoF and split its (z, y) term pairs; the partial sums
// are combined with shuffles (LANES > 1 on small coarse levels, where there are too few DoFs to
// fill the GPU).
template <typename T, int W, int LANES, bool SUB = false>
__global__ void k_restrict(const LevelDesc<T> F, const LevelDesc<T> C, const XferTabs<T> X, const T *__restrict__ in,
                           T *__restrict__ out, T *__restrict__ zero_c, const T *__restrict__ minus = nullptr) {
  pdl_enter();
  const long long total = (C.n_u + C.n_p) * LANES;
  const int sub = threadIdx.x & (LANES - 1);
  // the loop condition depends only on the warp's first index, so all 32 lanes iterate together
  // and the full-mask shuffles below are converged
  for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid - (threadIdx.x & 31) < total;
       gid += (long long)gridDim.x * blockDim.x) {
    const long long i = gid / LANES;
    const bool active = i < C.n_u + C.n_p;
    T s = active ? restrict_terms<T, W, SUB>(F, C, X, in, minus, i, sub, LANES) : T(0);
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, LANES);
    if (active && sub == 0) {
      out[i] = s;
      if (zero_c) zero_c[i] = T(0);
    }
  }
}

// Prolongation row of fine DoF i: (P in)_i.
template <typename T, int W, bool COH = false>
__device__ __forceinline__ T prolong_entry(const LevelDesc<T> &F, const LevelDesc<T> &C, const XferTabs<T> &X,
                                           const T *in, long long i) {
  const bool vel = i < F.n_u;
  const int sp = vel ? 0 : 1;
  const int *Nc = vel ? C.N : C.Pn, *Nf = vel ? F.N : F.Pn;
  const long long j = vel ? i % F.nv : i - F.n_u;
  const int g0 = (int)(j % Nf[0]), g1 = (int)((j / Nf[0]) % Nf[1]), g2 = (int)(j / ((long long)Nf[0] * Nf[1]));
  const T *src = in + (vel ? (i / F.nv) * C.nv : C.n_u);
  const Xfer1D<T> &ax = X.p[sp][0], &ay = X.p[sp][1], &az = X.p[sp][2];
  const int n0 = ax.cnt[g0], n1 = ay.cnt[g1], n2 = az.cnt[g2];
  T s = T(0);
  for (int a2 = 0; a2 < n2; ++a2) {
    const int G2 = az.idx[g2 * W + a2];
    const T w2 = az.w[g2 * W + a2];
    for (int a1 = 0; a1 < n1; ++a1) {
      const T *row = src + ((long long)G2 * Nc[1] + ay.idx[g1 * W + a1]) * Nc[0];
      T r = T(0);
      for (int a0 = 0; a0 < n0; ++a0) r += ax.w[g0 * W + a0] * ld_in<COH>(row + ax.idx[g0 * W + a0]);
      s += w2 * ay.w[g1 * W + a1] * r;
    }
  }
  return s;
}

// out (fine) = P in (coarse); add != 0: out += P in.  Covers velocity and pressure.  z0 / z1
// (fine velocity-sized, may be null) and zf (fine full-sized, may be null: the residual's K x
// accumulator) are zeroed on the way.
template <typename T, int W>
__global__ void k_prolongate(const LevelDesc<T> F, const LevelDesc<T> C, const XferTabs<T> X, const T *__restrict__ in,
                             T *__restrict__ out, int add, T *__restrict__ z0, T *__restrict__ z1,
                             T *__restrict__ zf = nullptr) {
  pdl_enter();
  SMF_GRID_LOOP(i, F.n_u + F.n_p) {
    const bool vel = i < F.n_u;
    if (zf) zf[i] = T(0);
    if (vel) {
      if (z0) z0[i] = T(0);
      if (z1) z1[i] = T(0);
    }
    const T s = prolong_entry<T, W>(F, C, X, in, i);
    out[i] = add ? out[i] + s : s;
  }
}

}  // namespace smf
