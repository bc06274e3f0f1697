// Vector kernels: Chebyshev-Jacobi recurrence (Sec. 3.3.1), residuals, precision
// conversion, FP64 reductions for the Krylov loop and Lanczos, SplitMix64 start vectors.
#pragma once
#include <initializer_list>

#include "common.cuh"

namespace smf {

constexpr int kVecThreads = 256;
constexpr int kRedBlocks = 304;  // 2 x 152 SMs; fixed so that reductions are deterministic

inline int vec_blocks(long long n) {
  long long b = (n + kVecThreads - 1) / kVecThreads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

// Host: true if every non-null pointer is aligned to `bytes`.
inline bool all_aligned(size_t bytes, std::initializer_list<const void *> ptrs) {
  for (const void *p : ptrs)
    if (p && (reinterpret_cast<uintptr_t>(p) % bytes) != 0) return false;
  return true;
}

#define SMF_GRID_LOOP(i, n) \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// out = a - b
template <typename T>
__global__ void k_sub(const T *__restrict__ a, const T *__restrict__ b, T *__restrict__ out, long long n) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) out[i] = a[i] - b[i];
}

// x += s * b
template <typename T>
__global__ void k_axpy(T *__restrict__ x, T s, const T *__restrict__ b, long long n) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) x[i] += s * b[i];
}

template <typename T>
__global__ void k_scale(const T *a, T s, T *out, long long n) {  // a and out may be the same vector
  pdl_enter();
  SMF_GRID_LOOP(i, n) out[i] = s * a[i];
}

template <typename T>
__global__ void k_mul(const T *a, const T *b, T *out, long long n) {  // out may be a or b (in place)
  pdl_enter();
  SMF_GRID_LOOP(i, n) out[i] = a[i] * b[i];
}

template <typename T>
__global__ void k_add_scalar(T *__restrict__ x, const double *__restrict__ sum, double scale, long long n) {
  pdl_enter();
  const T s = (T)(sum[0] * scale);
  SMF_GRID_LOOP(i, n) x[i] += s;
}

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin *__restrict__ a, Tout *__restrict__ out, long long n) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) out[i] = (Tout)a[i];
}

// ---- packed (16-byte) element access for the cycle's vector kernels -------------------------
template <typename T, int V>
struct alignas(sizeof(T) * V) Pack {
  T v[V];
};
template <int V, typename T>
__device__ __forceinline__ Pack<T, V> ldp(const T *p, long long j) {
  return *reinterpret_cast<const Pack<T, V> *>(p + j * V);
}
template <int V, typename T>
__device__ __forceinline__ void stp(T *p, long long j, const Pack<T, V> &v) {
  *reinterpret_cast<Pack<T, V> *>(p + j * V) = v;
}
template <int V, typename T>
__device__ __forceinline__ Pack<T, V> ldp_or0(const T *p, long long j) {
  Pack<T, V> r;
  if (p) {
    r = ldp<V>(p, j);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) r.v[k] = T(0);
  }
  return r;
}
// 16-byte packs read through L2 only (COH, see ld_in) or plainly.
template <int V, bool COH, typename T>
__device__ __forceinline__ Pack<T, V> ldpc(const T *p, long long j) {
  if constexpr (COH) {
    static_assert(sizeof(T) * V == 16, "16-byte packs");
    Pack<T, V> r;
    *reinterpret_cast<float4 *>(&r) = __ldcg(reinterpret_cast<const float4 *>(p + j * V));
    return r;
  } else {
    return ldp<V>(p, j);
  }
}
template <int V, bool COH, typename T>
__device__ __forceinline__ Pack<T, V> ldpc_or0(const T *p, long long j) {
  Pack<T, V> r;
  if (p) {
    r = ldpc<V, COH>(p, j);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) r.v[k] = T(0);
  }
  return r;
}
// Elements [0, n) as n/V packs plus a scalar tail handled by the first threads of the grid.
#define SMF_PACK_LOOP(j, n, V) SMF_GRID_LOOP(j, (n) / (V))
#define SMF_TAIL_LOOP(i, n, V)                                                                       \
  for (long long i = ((n) / (V)) * (V) + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (long long)gridDim.x * blockDim.x)

// Chebyshev start from x = 0 (Sec. 3.3.1): r = sr * (a - b) (a or b may be null),
// d = x = c0 * Dinv * r; r is stored if r_out != null.  za / zb (may alias a / b) are zeroed
// after they are read: apply targets are kept zero between uses, so the cycle needs no memset.
// With final_out / acc_out the degree-0 result f = base + fscale * x is written / accumulated.
// One element of k_cheb_init / k_cheb_step (the scalar tail of the packed kernels, and the work
// items of the persistent queue kernel with COH loads).
template <typename T, bool COH = false>
__device__ __forceinline__ void cheb_init_elem(long long i, const T *a, const T *b, T sr, const T *Dinv, T c0, T *r_out,
                                               T *d, T *x, const T *base, T fscale, T *final_out, T *acc_out, T *za,
                                               T *zb) {
  const T av = a ? ld_in<COH>(a + i) : T(0), bv = b ? ld_in<COH>(b + i) : T(0);
  if (za) za[i] = T(0);
  if (zb) zb[i] = T(0);
  const T r = sr * (av - bv);
  if (r_out) r_out[i] = r;
  const T v = c0 * ld_in<COH>(Dinv + i) * r;
  d[i] = v;
  x[i] = v;
  const T f = (base ? ld_in<COH>(base + i) : T(0)) + fscale * v;
  if (final_out) final_out[i] = f;
  if (acc_out) acc_out[i] = ld_in<COH>(acc_out + i) + f;
}
template <typename T, bool COH = false>
__device__ __forceinline__ void cheb_step_elem(long long i, const T *r, T *t, const T *Dinv, T c1, T c2, T *d, T *x,
                                               const T *base, T fscale, T *final_out, T *acc_out) {
  const T tv = ld_in<COH>(t + i);
  t[i] = T(0);
  const T dn = c1 * ld_in<COH>(d + i) + c2 * ld_in<COH>(Dinv + i) * (ld_in<COH>(r + i) - tv);
  const T xn = ld_in<COH>(x + i) + dn;
  d[i] = dn;
  x[i] = xn;
  const T f = (base ? ld_in<COH>(base + i) : T(0)) + fscale * xn;
  if (final_out) final_out[i] = f;
  if (acc_out) acc_out[i] = ld_in<COH>(acc_out + i) + f;
}
template <typename T, int V>
__device__ __forceinline__ void cheb_init_pack(const Pack<T, V> &A, const Pack<T, V> &B, T sr, const Pack<T, V> &Di,
                                               T c0, Pack<T, V> &R, Pack<T, V> &X) {
#pragma unroll
  for (int k = 0; k < V; ++k) {
    R.v[k] = sr * (A.v[k] - B.v[k]);
    X.v[k] = c0 * Di.v[k] * R.v[k];
  }
}
// Pack j of k_cheb_init (also a work item of the persistent queue kernel, COH).
template <typename T, int V, bool COH = false>
__device__ __forceinline__ void cheb_init_packj(long long j, const T *a, const T *b, T sr, const T *Dinv, T c0,
                                                T *r_out, T *d, T *x, const T *base, T fscale, T *final_out,
                                                T *acc_out, T *za, T *zb) {
  {
    const Pack<T, V> A = ldpc_or0<V, COH>(a, j), B = ldpc_or0<V, COH>(b, j), Di = ldpc<V, COH>(Dinv, j);
    const Pack<T, V> Bs = ldpc_or0<V, COH>(base, j), Ac = ldpc_or0<V, COH>(acc_out, j);
    Pack<T, V> R, X, Z;
    cheb_init_pack(A, B, sr, Di, c0, R, X);
#pragma unroll
    for (int k = 0; k < V; ++k) Z.v[k] = T(0);
    if (za) stp<V>(za, j, Z);
    if (zb) stp<V>(zb, j, Z);
    if (r_out) stp<V>(r_out, j, R);
    stp<V>(d, j, X);
    stp<V>(x, j, X);
    if (final_out || acc_out) {
      Pack<T, V> F, Anew;
#pragma unroll
      for (int k = 0; k < V; ++k) {
        F.v[k] = Bs.v[k] + fscale * X.v[k];
        Anew.v[k] = Ac.v[k] + F.v[k];
      }
      if (final_out) stp<V>(final_out, j, F);
      if (acc_out) stp<V>(acc_out, j, Anew);
    }
  }
}
// a / b may be the vectors za / zb that the same thread zeroes after reading them (the smoother's
// accumulators are consumed and cleared in one pass), so neither is declared __restrict__.
template <typename T, int V>
__global__ void k_cheb_init(const T *a, const T *b, T sr, const T *__restrict__ Dinv,
                            T c0, T *__restrict__ r_out, T *__restrict__ d, T *__restrict__ x, const T *__restrict__ base,
                            T fscale, T *__restrict__ final_out, T *__restrict__ acc_out, T *za, T *zb, long long n) {
  pdl_enter();
  SMF_PACK_LOOP(j, n, V)
  cheb_init_packj<T, V>(j, a, b, sr, Dinv, c0, r_out, d, x, base, fscale, final_out, acc_out, za, zb);
  SMF_TAIL_LOOP(i, n, V) cheb_init_elem(i, a, b, sr, Dinv, c0, r_out, d, x, base, fscale, final_out, acc_out, za, zb);
}

// One Chebyshev step: d = c1 d + c2 Dinv (r - t); x += d; t is zeroed after it is read.  With
// final_out / acc_out, f = base + fscale * x_new is written / accumulated.
template <typename T, int V, bool COH = false>
__device__ __forceinline__ void cheb_step_packj(long long j, const T *r, T *t, const T *Dinv, T c1, T c2, T *d, T *x,
                                                const T *base, T fscale, T *final_out, T *acc_out) {
  {
    const Pack<T, V> R = ldpc<V, COH>(r, j), Tt = ldpc<V, COH>(t, j), Di = ldpc<V, COH>(Dinv, j),
                     Dd = ldpc<V, COH>(d, j), X = ldpc<V, COH>(x, j);
    const Pack<T, V> Bs = ldpc_or0<V, COH>(base, j), Ac = ldpc_or0<V, COH>(acc_out, j);
    Pack<T, V> Dn, Xn, Z;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      Dn.v[k] = c1 * Dd.v[k] + c2 * Di.v[k] * (R.v[k] - Tt.v[k]);
      Xn.v[k] = X.v[k] + Dn.v[k];
      Z.v[k] = T(0);
    }
    stp<V>(t, j, Z);
    stp<V>(d, j, Dn);
    stp<V>(x, j, Xn);
    if (final_out || acc_out) {
      Pack<T, V> F, Anew;
#pragma unroll
      for (int k = 0; k < V; ++k) {
        F.v[k] = Bs.v[k] + fscale * Xn.v[k];
        Anew.v[k] = Ac.v[k] + F.v[k];
      }
      if (final_out) stp<V>(final_out, j, F);
      if (acc_out) stp<V>(acc_out, j, Anew);
    }
  }
}
template <typename T, int V>
__global__ void k_cheb_step(const T *__restrict__ r, T *__restrict__ t, const T *__restrict__ Dinv, T c1, T c2,
                            T *__restrict__ d, T *__restrict__ x, const T *__restrict__ base, T fscale,
                            T *__restrict__ final_out, T *__restrict__ acc_out, long long n) {
  pdl_enter();
  SMF_PACK_LOOP(j, n, V) cheb_step_packj<T, V>(j, r, t, Dinv, c1, c2, d, x, base, fscale, final_out, acc_out);
  SMF_TAIL_LOOP(i, n, V) cheb_step_elem(i, r, t, Dinv, c1, c2, d, x, base, fscale, final_out, acc_out);
}

// End of a fused smoothing sequence: the last line of the compact Uzawa step,
//   u[i] = uhat[i] + Dinv[i] (ca a[i] + cb b[i])   (i < n_u; a, b zeroed afterwards),
// and the pressure work vectors pz[0..npz) zeroed (i < n_p).
template <typename T>
struct ZeroList {
  T *p[kFusePre];
  int n;
};
template <typename T>
__global__ void k_fused_finish(const T *__restrict__ uhat, const T *__restrict__ Dinv, T *__restrict__ a,
                               T *__restrict__ b, T ca, T cb, T *__restrict__ u, long long n_u, ZeroList<T> pz,
                               long long n_p) {
  pdl_enter();
  const long long n = n_u > n_p ? n_u : n_p;
  SMF_GRID_LOOP(i, n) {
    if (i < n_u) {
      u[i] = uhat[i] + Dinv[i] * (ca * a[i] + cb * b[i]);
      a[i] = T(0);
      b[i] = T(0);
    }
    if (i < n_p)
      for (int j = 0; j < pz.n; ++j) pz.p[j][i] = T(0);
  }
}

// out = (Tout) a; zero (may be null) is zeroed.
template <typename Tin, typename Tout, int V>
__global__ void k_convert_zero(const Tin *__restrict__ a, Tout *__restrict__ out, Tout *__restrict__ zero, long long n) {
  pdl_enter();
  SMF_PACK_LOOP(j, n, V) {
    const Pack<Tin, V> A = ldp<V>(a, j);
    Pack<Tout, V> O, Z;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      O.v[k] = (Tout)A.v[k];
      Z.v[k] = Tout(0);
    }
    stp<V>(out, j, O);
    if (zero) stp<V>(zero, j, Z);
  }
  SMF_TAIL_LOOP(i, n, V) {
    out[i] = (Tout)a[i];
    if (zero) zero[i] = Tout(0);
  }
}

// y = x on constrained velocity DoFs (identity rows of K), 0 on every other entry of [u | p]:
// the start of y = K x before the cell kernel accumulates into the free rows.
template <typename T>
__global__ void k_init_identity(const LevelDesc<T> L, const T *__restrict__ x, T *__restrict__ y) {
  pdl_enter();
  SMF_GRID_LOOP(i, L.n_u + L.n_p) {
    T v = T(0);
    if (i < L.n_u) {
      const long long node = i % L.nv;
      const int gx = (int)(node % L.N[0]);
      const long long r = node / L.N[0];
      const int gy = (int)(r % L.N[1]), gz = (int)(r / L.N[1]);
      if (vel_constrained(L.N, L.faces, L.dim, gx, gy, gz)) v = x[i];
    }
    y[i] = v;
  }
}

// zero constrained velocity entries
template <typename T>
__global__ void k_zero_constrained(const LevelDesc<T> L, T *__restrict__ y) {
  pdl_enter();
  SMF_GRID_LOOP(i, L.n_u) {
    long long node = i % L.nv;
    int gx = (int)(node % L.N[0]);
    long long r = node / L.N[0];
    int gy = (int)(r % L.N[1]);
    int gz = (int)(r / L.N[1]);
    if (vel_constrained(L.N, L.faces, L.dim, gx, gy, gz)) y[i] = T(0);
  }
}

// D_A over the full velocity vector from the scalar per-node diagonal (per_comp: already one
// value per velocity DoF, the symmetric form); 1 on constrained DoFs.
template <typename T>
__global__ void k_expand_diag(const LevelDesc<T> L, const T *__restrict__ dAs, T *__restrict__ DA, int per_comp) {
  pdl_enter();
  SMF_GRID_LOOP(i, L.n_u) {
    long long node = i % L.nv;
    int gx = (int)(node % L.N[0]);
    long long r = node / L.N[0];
    int gy = (int)(r % L.N[1]);
    int gz = (int)(r / L.N[1]);
    DA[i] = vel_constrained(L.N, L.faces, L.dim, gx, gy, gz) ? T(1) : dAs[per_comp ? i : node];
  }
}

template <typename T>
__global__ void k_reciprocal(const T *__restrict__ a, T *__restrict__ out, long long n) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) out[i] = T(1) / a[i];
}

template <typename T>
__global__ void k_rsqrt(const T *__restrict__ a, T *__restrict__ out, long long n) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) out[i] = T(1) / sqrt(a[i]);
}

// SplitMix64 (Steele, Lea, Flood 2014): z = seed + (i+1)*0x9E3779B97F4A7C15, output mix,
// mapped to 2*(z>>11)*2^-53 - 1 in [-1, 1).  mask_level (optional) zeroes constrained velocity DoFs.
__device__ __forceinline__ double splitmix64_uniform(unsigned long long seed, long long i) {
  unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

__global__ void k_splitmix(unsigned long long seed, double *__restrict__ out, long long n);

// ---- deterministic FP64 reductions ---------------------------------------------------
template <typename T>
__device__ __forceinline__ double block_reduce_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

// partial[j * gridDim.x + blockIdx.x] = sum_i V[j*ldv + i] * w[i]   (j < nvec); V null -> sum w[i]^2 not used
__global__ void k_mdot_partial(const double *__restrict__ V, long long ldv, int nvec, const double *__restrict__ w,
                               long long n, double *__restrict__ partial);
__global__ void k_sum_partial(const double *__restrict__ a, long long n, double *__restrict__ partial);
__global__ void k_final_reduce(const double *__restrict__ partial, int nparts, int nvec, double *__restrict__ out);
// w -= sum_j h[j] V[j]
__global__ void k_maxpy(const double *__restrict__ V, long long ldv, int nvec, const double *__restrict__ h,
                        double *__restrict__ w, long long n, double sign);
// dense coarse solve (setup): unit vectors, augmented bordered matrix, Gauss-Jordan steps
__global__ void k_unit(double *__restrict__ e, long long n, long long j);
__global__ void k_build_augmented(const double *__restrict__ K0, int n0, long long n_u, int bordered,
                                  double *__restrict__ M);
__global__ void k_gj_pivot(double *__restrict__ M, int nb, int k, double *__restrict__ fac, int *__restrict__ err);
__global__ void k_gj_elim(double *__restrict__ M, int nb, int k, const double *__restrict__ fac);
__global__ void k_extract_inverse(const double *__restrict__ M, int nb, int n0, double *__restrict__ Kinv);
// out = w / norm where norm = sqrt(*nrm2)
__global__ void k_scale_by_inv_sqrt(const double *__restrict__ w, const double *__restrict__ nrm2,
                                    double *__restrict__ out, long long n);

}  // namespace smf

namespace smf {

// ---- FGMRES with the Arnoldi state on the device ----------------------------------------------
// The inner iterations of one restart cycle run as a CUDA graph with a conditional while node:
// every kernel reads the iteration index j from device memory (ctl[0]), and k_fgmres_givens
// decides on the device whether the loop continues.  ctl = {j, it, stop, maxit}; stop: 0 running,
// 1 converged (|g_{j+1}| <= thresh), 2 maxit, 3 non-finite, 4 restart length reached.
struct KrylovDev {
  double *H = nullptr;     // (m+1) x m Hessenberg, row-major H[i * m + j] (rotated in place)
  double *cs = nullptr, *sn = nullptr;  // Givens rotations (m)
  double *g = nullptr;     // rotated right-hand side (m + 1)
  double *y = nullptr;     // triangular-solve result (m)
  double *hcol = nullptr;  // CGS2 coefficients of the two passes ([0, m+2), [m+2, 2m+4)) and ||w||^2
  double *thresh = nullptr;  // rtol * ||b||
  int *ctl = nullptr;
  unsigned *ticket = nullptr;  // finished blocks of k_mdot_final_cnt (returns to 0 after every launch)
  int m = 0;
};
// k_mdot_partial_cnt and k_final_reduce_cnt in one launch: every block writes its partial sums, the
// last block to finish (a ticket counter, after a fence) sums them per vector in the same fixed
// order as k_final_reduce_cnt and writes out[jj] for jj < ctl[0] + add (V == w, add == 1 - ctl[0]
// gives ||w||^2 through ctl = null: then one vector, V = w).
__global__ void k_mdot_final_cnt(const double *__restrict__ V, long long ldv, const int *__restrict__ ctl, int add,
                                 const double *__restrict__ w, long long n, double *__restrict__ partial,
                                 unsigned *__restrict__ ticket, double *__restrict__ out);
// partial[jj * gridDim.x + b] = block b's part of V_jj . w for jj < ctl[0] + add
__global__ void k_mdot_partial_cnt(const double *__restrict__ V, long long ldv, const int *__restrict__ ctl, int add,
                                   const double *__restrict__ w, long long n, double *__restrict__ partial);
// out[jj] = sum_b partial[jj * nparts + b], one block per jj; blocks jj >= ctl[0] + add return
__global__ void k_final_reduce_cnt(const double *__restrict__ partial, int nparts, const int *__restrict__ ctl, int add,
                                   double *__restrict__ out);
// w += sign * sum_{jj < ctl[0] + add} h[jj] V_jj
__global__ void k_maxpy_cnt(const double *__restrict__ V, long long ldv, const int *__restrict__ ctl, int add,
                            const double *__restrict__ h, double *__restrict__ w, long long n, double sign);
// V_{ctl[0] + 1} = w / sqrt(*nrm2)
__global__ void k_scale_to_slot(const double *__restrict__ w, const double *__restrict__ nrm2, double *__restrict__ V,
                                long long ldv, const int *__restrict__ ctl, long long n);
// one Arnoldi column: Hessenberg entries, earlier rotations, new rotation, residual estimate,
// stop decision; sets the while-node condition
__global__ void k_fgmres_givens(KrylovDev K, cudaGraphConditionalHandle cond, int set_cond);
// Batched Arnoldi loop: member i runs its iteration while its ctl[i][2] == 0 (conditional if
// nodes, one per member, inside one while node that runs while any member does).
constexpr int kBatchMax = 64;
struct BatchCond {
  int n = 0;
  int has_post = 0;                                    // post[] in use (work-queue form)
  cudaGraphConditionalHandle loop{};                   // work-queue form: the iteration loop
  cudaGraphConditionalHandle member[kBatchMax] = {};  // a member's iterations (or its part before the queue)
  cudaGraphConditionalHandle post[kBatchMax] = {};    // work-queue form: its part after the queue
  const int *ctl[kBatchMax] = {};
};
__global__ void k_batch_select(const BatchCond B);  // member conditions from their stop flags
__global__ void k_batch_any(const BatchCond B);     // loop condition: any member still running
// y = R^{-1} g on the first ctl[0] columns (R the rotated Hessenberg, upper triangular)
__global__ void k_fgmres_trisolve(KrylovDev K);

// out = (Tout) V_{ctl[0]}, zero (may be null) zeroed: the preconditioner's right-hand side
template <typename Tout>
__global__ void k_slot_convert(const double *__restrict__ V, long long ldv, const int *__restrict__ ctl,
                               Tout *__restrict__ out, Tout *__restrict__ zero, long long n) {
  pdl_enter();
  const double *a = V + (long long)ctl[0] * ldv;
  SMF_GRID_LOOP(i, n) {
    out[i] = (Tout)a[i];
    if (zero) zero[i] = Tout(0);
  }
}
// z = (double) a and Z_{ctl[0]} = z (the preconditioned vector for the operator and the update),
// and y = the identity rows of z (z on constrained velocity DoFs, 0 elsewhere): the start of
// y = K z (k_init_identity) in the same pass.
template <typename Tin>
__global__ void k_convert_to_slot_id(const LevelDesc<double> L, const Tin *__restrict__ a, double *__restrict__ z,
                                     double *__restrict__ Z, long long ldz, const int *__restrict__ ctl,
                                     double *__restrict__ y) {
  pdl_enter();
  double *zj = Z + (long long)ctl[0] * ldz;
  SMF_GRID_LOOP(i, L.n_u + L.n_p) {
    const double v = (double)a[i];
    z[i] = v;
    zj[i] = v;
    double yi = 0.0;
    if (i < L.n_u) {
      const long long node = i % L.nv;
      const int gx = (int)(node % L.N[0]);
      const long long r = node / L.N[0];
      const int gy = (int)(r % L.N[1]), gz = (int)(r / L.N[1]);
      if (vel_constrained(L.N, L.faces, L.dim, gx, gy, gz)) yi = v;
    }
    y[i] = yi;
  }
}

}  // namespace smf
