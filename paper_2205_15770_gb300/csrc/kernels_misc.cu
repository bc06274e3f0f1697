// Non-template kernels: SplitMix64 vectors, deterministic FP64 reductions, Gauss-Jordan
// inverse of the (bordered) coarse matrix, and the dense coarse solve.
#include "vec.cuh"

namespace smf {

__global__ void k_splitmix(unsigned long long seed, double *__restrict__ out, long long n) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) out[i] = splitmix64_uniform(seed, i);
}

__global__ void k_mdot_partial(const double *__restrict__ V, long long ldv, int nvec, const double *__restrict__ w,
                               long long n, double *__restrict__ partial) {
  pdl_enter();
  __shared__ double sh[32];
  for (int j = 0; j < nvec; ++j) {
    const double *v = V + (long long)j * ldv;
    double s = 0.0;
    SMF_GRID_LOOP(i, n) s += v[i] * w[i];
    s = block_reduce_sum<double>(s, sh);
    if (threadIdx.x == 0) partial[(long long)j * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_sum_partial(const double *__restrict__ a, long long n, double *__restrict__ partial) {
  pdl_enter();
  __shared__ double sh[32];
  double s = 0.0;
  SMF_GRID_LOOP(i, n) s += a[i];
  s = block_reduce_sum<double>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[j] = sum_b partial[j*nparts + b]; one block per j
__global__ void k_final_reduce(const double *__restrict__ partial, int nparts, int nvec, double *__restrict__ out) {
  pdl_enter();
  __shared__ double sh[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += partial[(long long)j * nparts + b];
  s = block_reduce_sum<double>(s, sh);
  if (threadIdx.x == 0) out[j] = s;
}

__global__ void k_maxpy(const double *__restrict__ V, long long ldv, int nvec, const double *__restrict__ h,
                        double *__restrict__ w, long long n, double sign) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) {
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s += h[j] * V[(long long)j * ldv + i];
    w[i] += sign * s;
  }
}

__global__ void k_scale_by_inv_sqrt(const double *__restrict__ w, const double *__restrict__ nrm2,
                                    double *__restrict__ out, long long n) {
  pdl_enter();
  const double s = 1.0 / sqrt(nrm2[0]);
  SMF_GRID_LOOP(i, n) out[i] = s * w[i];
}

__global__ void k_unit(double *__restrict__ e, long long n, long long j) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) e[i] = (i == j) ? 1.0 : 0.0;
}

// Augmented [Kb | I] (row-major nb x 2nb) from the column-major n0 x n0 coarse matrix K0;
// bordered (nb = n0 + 1) with e = (0, 1_p) when `bordered`.
__global__ void k_build_augmented(const double *__restrict__ K0, int n0, long long n_u, int bordered,
                                  double *__restrict__ M) {
  const int nb = n0 + bordered;
  SMF_GRID_LOOP(idx, (long long)nb * 2 * nb) {
    const int i = (int)(idx / (2 * nb)), j = (int)(idx % (2 * nb));
    double v;
    if (j >= nb)
      v = (j - nb == i) ? 1.0 : 0.0;
    else if (i < n0 && j < n0)
      v = K0[(long long)j * n0 + i];
    else if (i == n0 && j == n0)
      v = 0.0;
    else {
      const int other = (i == n0) ? j : i;
      v = other >= n_u ? 1.0 : 0.0;
    }
    M[idx] = v;
  }
}

// Pivot step k of Gauss-Jordan (single block): partial pivoting on column k, row swap,
// row scaling, and the elimination factors fac[i] = M[i][k] (fac[k] = 0).
__global__ void k_gj_pivot(double *__restrict__ M, int nb, int k, double *__restrict__ fac, int *__restrict__ err) {
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  const int ld = 2 * nb;
  double best = -1.0;
  int besti = k;
  for (int i = k + threadIdx.x; i < nb; i += blockDim.x) {
    const double a = fabs(M[(long long)i * ld + k]);
    if (a > best) {
      best = a;
      besti = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      if (bv[threadIdx.x + s] > bv[threadIdx.x] ||
          (bv[threadIdx.x + s] == bv[threadIdx.x] && bi[threadIdx.x + s] < bi[threadIdx.x])) {
        bv[threadIdx.x] = bv[threadIdx.x + s];
        bi[threadIdx.x] = bi[threadIdx.x + s];
      }
    }
    __syncthreads();
  }
  const int p = bi[0];
  if (!(bv[0] > 0.0)) {
    if (threadIdx.x == 0) err[0] = 1;
    return;
  }
  if (p != k)
    for (int j = threadIdx.x; j < ld; j += blockDim.x) {
      const double a = M[(long long)k * ld + j];
      M[(long long)k * ld + j] = M[(long long)p * ld + j];
      M[(long long)p * ld + j] = a;
    }
  __syncthreads();
  const double inv = 1.0 / M[(long long)k * ld + k];
  __syncthreads();
  for (int j = threadIdx.x; j < ld; j += blockDim.x) M[(long long)k * ld + j] *= inv;
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) fac[i] = (i == k) ? 0.0 : M[(long long)i * ld + k];
}

__global__ void k_gj_elim(double *__restrict__ M, int nb, int k, const double *__restrict__ fac) {
  const int ld = 2 * nb;
  const int i = blockIdx.y;
  const double f = fac[i];
  if (f == 0.0) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ld; j += gridDim.x * blockDim.x)
    M[(long long)i * ld + j] -= f * M[(long long)k * ld + j];
}

// Kinv (row-major n0 x n0) = top-left block of the right half of M.
__global__ void k_extract_inverse(const double *__restrict__ M, int nb, int n0, double *__restrict__ Kinv) {
  SMF_GRID_LOOP(idx, (long long)n0 * n0) {
    const int i = (int)(idx / n0), j = (int)(idx % n0);
    Kinv[idx] = M[(long long)i * 2 * nb + nb + j];
  }
}

}  // namespace smf

namespace smf {

__global__ void k_mdot_partial_cnt(const double *__restrict__ V, long long ldv, const int *__restrict__ ctl, int add,
                                   const double *__restrict__ w, long long n, double *__restrict__ partial) {
  pdl_enter();
  __shared__ double sh[32];
  const int nvec = ctl[0] + add;
  for (int j = 0; j < nvec; ++j) {
    const double *v = V + (long long)j * ldv;
    double s = 0.0;
    SMF_GRID_LOOP(i, n) s += v[i] * w[i];
    s = block_reduce_sum<double>(s, sh);
    if (threadIdx.x == 0) partial[(long long)j * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_mdot_final_cnt(const double *__restrict__ V, long long ldv, const int *__restrict__ ctl, int add,
                                 const double *__restrict__ w, long long n, double *__restrict__ partial,
                                 unsigned *__restrict__ ticket, double *__restrict__ out) {
  pdl_enter();
  __shared__ double sh[32];
  __shared__ int last;
  const int nvec = ctl ? ctl[0] + add : 1;
  for (int j = 0; j < nvec; ++j) {
    const double *v = ctl ? V + (long long)j * ldv : w;
    double s = 0.0;
    SMF_GRID_LOOP(i, n) s += v[i] * w[i];
    s = block_reduce_sum<double>(s, sh);
    if (threadIdx.x == 0) partial[(long long)j * gridDim.x + blockIdx.x] = s;
  }
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partial sums before its ticket
    last = atomicInc(ticket, gridDim.x - 1) == gridDim.x - 1;  // the counter wraps back to 0
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int nparts = gridDim.x;
  for (int j = 0; j < nvec; ++j) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += __ldcg(partial + (long long)j * nparts + b);
    s = block_reduce_sum<double>(s, sh);
    if (threadIdx.x == 0) out[j] = s;
  }
}

__global__ void k_final_reduce_cnt(const double *__restrict__ partial, int nparts, const int *__restrict__ ctl, int add,
                                   double *__restrict__ out) {
  pdl_enter();
  __shared__ double sh[32];
  const int j = blockIdx.x;
  if (j >= ctl[0] + add) return;  // uniform per block
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += partial[(long long)j * nparts + b];
  s = block_reduce_sum<double>(s, sh);
  if (threadIdx.x == 0) out[j] = s;
}

__global__ void k_maxpy_cnt(const double *__restrict__ V, long long ldv, const int *__restrict__ ctl, int add,
                            const double *__restrict__ h, double *__restrict__ w, long long n, double sign) {
  pdl_enter();
  const int nvec = ctl[0] + add;
  SMF_GRID_LOOP(i, n) {
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s += h[j] * V[(long long)j * ldv + i];
    w[i] += sign * s;
  }
}

__global__ void k_scale_to_slot(const double *__restrict__ w, const double *__restrict__ nrm2, double *__restrict__ V,
                                long long ldv, const int *__restrict__ ctl, long long n) {
  pdl_enter();
  const double s = 1.0 / sqrt(nrm2[0]);
  double *out = V + (long long)(ctl[0] + 1) * ldv;
  SMF_GRID_LOOP(i, n) out[i] = s * w[i];
}

__global__ void k_fgmres_givens(KrylovDev K, cudaGraphConditionalHandle cond, int set_cond) {
  pdl_enter();
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int m = K.m, j = K.ctl[0];
  double *H = K.H;
  for (int i = 0; i <= j; ++i) H[i * m + j] = K.hcol[i] + K.hcol[(m + 2) + i];
  H[(j + 1) * m + j] = sqrt(K.hcol[2 * (m + 2)]);
  for (int i = 0; i < j; ++i) {
    const double a = H[i * m + j], b = H[(i + 1) * m + j];
    H[i * m + j] = K.cs[i] * a + K.sn[i] * b;
    H[(i + 1) * m + j] = -K.sn[i] * a + K.cs[i] * b;
  }
  const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
  K.cs[j] = H[j * m + j] / den;
  K.sn[j] = H[(j + 1) * m + j] / den;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  const double gj = K.g[j];
  K.g[j + 1] = -K.sn[j] * gj;
  K.g[j] = K.cs[j] * gj;
  const int it = K.ctl[1] + 1;
  K.ctl[1] = it;
  K.ctl[0] = j + 1;
  int stop = 0;
  if (!isfinite(K.g[j + 1]))
    stop = 3;
  else if (fabs(K.g[j + 1]) <= K.thresh[0])
    stop = 1;
  else if (it >= K.ctl[3])
    stop = 2;
  else if (j + 1 >= m)
    stop = 4;
  K.ctl[2] = stop;
  if (set_cond) cudaGraphSetConditional(cond, stop == 0 ? 1u : 0u);
}

__global__ void k_fgmres_trisolve(KrylovDev K) {
  pdl_enter();
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int m = K.m, jd = K.ctl[0];
  for (int i = jd - 1; i >= 0; --i) {
    double s = K.g[i];
    for (int c = i + 1; c < jd; ++c) s -= K.H[i * m + c] * K.y[c];
    K.y[i] = s / K.H[i * m + i];
  }
}

}  // namespace smf

namespace smf {

__global__ void k_batch_select(const BatchCond B) {
  pdl_enter();
  const int i = threadIdx.x;
  if (blockIdx.x == 0 && i < B.n) {
    const unsigned on = B.ctl[i][2] == 0 ? 1u : 0u;
    cudaGraphSetConditional(B.member[i], on);
    if (B.has_post) cudaGraphSetConditional(B.post[i], on);
  }
}

__global__ void k_batch_any(const BatchCond B) {
  pdl_enter();
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int any = 0;
  for (int i = 0; i < B.n; ++i) any |= B.ctl[i][2] == 0;
  cudaGraphSetConditional(B.loop, any ? 1u : 0u);
}


}  // namespace smf
