// Grid transfers (paper Sec. 3.2): prolongation = canonical injection of the coarse
// Q_k x Q_{k-1} space into the fine one, restriction = its transpose.  On the structured
// hierarchy the injection is a tensor product of 1D matrices: fine node g along an axis
// lies in fine cell f (local node a), child h = f mod 2 of coarse cell c = f / 2, and takes
// the coarse basis values at reference coordinate (h + t_a)/2.  Constrained velocity DoFs
// are dropped on both sides (P_eff = Z_fine P Z_coarse).
//
// Both kernels are DoF-parallel and write every output once (no atomics):
//   prolongation: each fine DoF gathers the (deg+1)^d coarse values of its coarse cell;
//   restriction:  each coarse DoF gathers the fine DoFs in the support of its basis function.
#pragma once
#include "common.cuh"
#include "vec.cuh"

namespace smf {

constexpr int kMaxAxis = 4 * kMaxDeg + 1;

// Row of the 1D injection for fine node g (degree deg, nc coarse cells): coarse nodes G[m] with weights w[m].
template <typename T>
__device__ __forceinline__ int inj_row(int g, int deg, int nc, const T *tab, int *G, T *w) {
  int f = g / deg;
  if (f > 2 * nc - 1) f = 2 * nc - 1;
  const int a = g - deg * f, c = f >> 1, h = f & 1;
  for (int m = 0; m <= deg; ++m) {
    G[m] = deg * c + m;
    w[m] = tab[(h * (deg + 1) + a) * (deg + 1) + m];
  }
  return deg + 1;
}

// Column of the 1D injection for coarse node G: fine nodes g[j] with weights w[j] != 0.
template <typename T>
__device__ __forceinline__ int inj_col(int G, int deg, int nc, const T *tab, int *g, T *w) {
  int c_lo = G / deg, c_hi = G / deg;
  if (G % deg == 0) c_lo -= 1;
  if (c_lo < 0) c_lo = 0;
  if (c_hi > nc - 1) c_hi = nc - 1;
  int cnt = 0;
  for (int gi = 2 * deg * c_lo; gi <= 2 * deg * c_hi + 2 * deg; ++gi) {
    int f = gi / deg;
    if (f > 2 * nc - 1) f = 2 * nc - 1;
    const int a = gi - deg * f, c = f >> 1, h = f & 1, m = G - deg * c;
    if (m < 0 || m > deg) continue;
    const T v = tab[(h * (deg + 1) + a) * (deg + 1) + m];
    if (v != T(0)) {
      g[cnt] = gi;
      w[cnt] = v;
      ++cnt;
    }
  }
  return cnt;
}

// out (fine) = P in (coarse); add != 0: out += P in.  Covers velocity and pressure.
template <typename T>
__global__ void k_prolongate(const LevelDesc<T> F, const LevelDesc<T> C, const TransferTab<T> *__restrict__ tt,
                             const T *__restrict__ in, T *__restrict__ out, int add) {
  pdl_enter();
  const int dim = F.dim, k = F.k;
  SMF_GRID_LOOP(i, F.n_u + F.n_p) {
    const bool vel = i < F.n_u;
    const int deg = vel ? k : k - 1;
    const T *tab = vel ? tt->vel : tt->pre;
    const int *Nf = vel ? F.N : F.Pn;
    const long long nodes = vel ? F.nv : F.n_p;
    const long long j = vel ? i % F.nv : i - F.n_u;
    const int comp = vel ? (int)(i / F.nv) : 0;
    int g[3] = {(int)(j % Nf[0]), (int)((j / Nf[0]) % Nf[1]), dim == 3 ? (int)(j / ((long long)Nf[0] * Nf[1])) : 0};
    (void)nodes;
    if (vel && vel_constrained(F.N, F.faces, dim, g[0], g[1], g[2])) {
      if (!add) out[i] = T(0);
      continue;
    }
    int G[3][kMaxN1];
    T w[3][kMaxN1];
    int cnt[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) cnt[a] = inj_row(g[a], deg, C.n[a], tab, G[a], w[a]);
    if (dim == 2) {
      G[2][0] = 0;
      w[2][0] = T(1);
    }
    T s = T(0);
    for (int c2 = 0; c2 < cnt[2]; ++c2)
      for (int c1 = 0; c1 < cnt[1]; ++c1) {
        const T w12 = w[2][c2] * w[1][c1];
        if (w12 == T(0)) continue;
        for (int c0 = 0; c0 < cnt[0]; ++c0) {
          const T ww = w12 * w[0][c0];
          if (ww == T(0)) continue;
          if (vel) {
            if (vel_constrained(C.N, C.faces, dim, G[0][c0], G[1][c1], G[2][c2])) continue;
            const long long ci = dim == 3 ? ((long long)G[2][c2] * C.N[1] + G[1][c1]) * C.N[0] + G[0][c0]
                                          : (long long)G[1][c1] * C.N[0] + G[0][c0];
            s += ww * in[comp * C.nv + ci];
          } else {
            const long long ci = dim == 3 ? ((long long)G[2][c2] * C.Pn[1] + G[1][c1]) * C.Pn[0] + G[0][c0]
                                          : (long long)G[1][c1] * C.Pn[0] + G[0][c0];
            s += ww * in[C.n_u + ci];
          }
        }
      }
    out[i] = add ? out[i] + s : s;
  }
}

// out (coarse) = P^T in (fine); zero_c (coarse-sized, may be null) is zeroed on the way.
// LANES consecutive lanes share one coarse DoF: the (up to (4k+1)^d) fine terms of its support
// are split across them and combined with warp shuffles (LANES = 8 on small coarse levels,
// where there are too few DoFs to fill the GPU; 1 on large ones).
template <typename T, int LANES>
__global__ void k_restrict(const LevelDesc<T> F, const LevelDesc<T> C, const TransferTab<T> *__restrict__ tt,
                           const T *__restrict__ in, T *__restrict__ out, T *__restrict__ zero_c) {
  pdl_enter();
  const int dim = F.dim, k = F.k;
  const long long total = (C.n_u + C.n_p) * LANES;
  const int sub = threadIdx.x & (LANES - 1);
  // grid-stride over (DoF, lane) pairs; the loop condition depends only on the warp's first
  // index, so all 32 lanes iterate together and the full-mask shuffles below are converged
  for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid - (threadIdx.x & 31) < total;
       gid += (long long)gridDim.x * blockDim.x) {
    const long long i = gid / LANES;
    const bool active = i < C.n_u + C.n_p;
    T s = T(0);
    bool constrained = false;
    if (active) {
      const bool vel = i < C.n_u;
      const int deg = vel ? k : k - 1;
      const T *tab = vel ? tt->vel : tt->pre;
      const int *Nc = vel ? C.N : C.Pn;
      const long long j = vel ? i % C.nv : i - C.n_u;
      const int comp = vel ? (int)(i / C.nv) : 0;
      int G[3] = {(int)(j % Nc[0]), (int)((j / Nc[0]) % Nc[1]), dim == 3 ? (int)(j / ((long long)Nc[0] * Nc[1])) : 0};
      constrained = vel && vel_constrained(C.N, C.faces, dim, G[0], G[1], G[2]);
      if (!constrained) {
        int g[3][kMaxAxis];
        T w[3][kMaxAxis];
        int cnt[3] = {1, 1, 1};
        for (int a = 0; a < dim; ++a) cnt[a] = inj_col(G[a], deg, C.n[a], tab, g[a], w[a]);
        if (dim == 2) {
          g[2][0] = 0;
          w[2][0] = T(1);
        }
        const int nterms = cnt[0] * cnt[1] * cnt[2];
        for (int t = sub; t < nterms; t += LANES) {
          const int c0 = t % cnt[0], c1 = (t / cnt[0]) % cnt[1], c2 = t / (cnt[0] * cnt[1]);
          const T ww = w[2][c2] * w[1][c1] * w[0][c0];
          if (vel) {
            if (vel_constrained(F.N, F.faces, dim, g[0][c0], g[1][c1], g[2][c2])) continue;
            const long long fi = dim == 3 ? ((long long)g[2][c2] * F.N[1] + g[1][c1]) * F.N[0] + g[0][c0]
                                          : (long long)g[1][c1] * F.N[0] + g[0][c0];
            s += ww * in[comp * F.nv + fi];
          } else {
            const long long fi = dim == 3 ? ((long long)g[2][c2] * F.Pn[1] + g[1][c1]) * F.Pn[0] + g[0][c0]
                                          : (long long)g[1][c1] * F.Pn[0] + g[0][c0];
            s += ww * in[F.n_u + fi];
          }
        }
      }
    }
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, LANES);
    if (active && sub == 0) {
      out[i] = s;
      if (zero_c) zero_c[i] = T(0);
    }
  }
}

}  // namespace smf
