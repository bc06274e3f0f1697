// Shared definitions of the CUDA library: level descriptors, 1D tables, helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

namespace smf {

constexpr int kMaxDeg = 4;            // highest velocity degree k supported
constexpr int kMaxN1 = kMaxDeg + 1;   // nodes / Gauss points per direction
constexpr int kMaxCMatrixNodes = 27;  // stored element matrices of C up to this many pressure nodes per cell

// Operator block selection for the cell kernel (bit set).
enum ApplyMode : int {
  kApplyA = 1,     // yu += A u  (mu grad:grad + gamma*rho mass)
  kApplyBT = 2,    // yu += B^T p
  kApplyB = 4,     // yp += B u
  kApplyMass = 8,      // yu += Z M_v u (right-hand sides b = Z M_v f; every node of u is read)
  kApplyMassAll = 16,  // yu += M_v Z u (its transpose: free nodes of u read, every row written)
  kApplyUnmasked = 32, // with A / BT / B: read u at constrained nodes too (K_full u_D for lifting)
  kApplyC = 64,        // yp -= C p (stabilisation block of K = [A B^T; B -C])
  kApplySym = 128,     // with A: the symmetric-gradient form mu eps(u):eps(v) (generic kernel)
};

// 1D tables of one velocity degree k on the reference interval, (k+1) Gauss points.
// Row index = Gauss point q, column = node / function m.
template <typename T>
struct Tab1D {
  T S[kMaxN1 * kMaxN1];    // S[q*(k+1)+m]  = l_m(x_q)       velocity Lagrange basis at Gauss points
  T Sd[kMaxN1 * kMaxN1];   // Sd[q*(k+1)+m] = l_m'(x_q)      its derivative
  T D[kMaxN1 * kMaxN1];    // D[q*nq+m]     = g_m'(x_q)      collocation derivative (Lagrange through Gauss points)
  T Pv[kMaxN1 * kMaxDeg];  // Pv[q*k+m]     = pressure basis (degree k-1) at Gauss points
  T Pd[kMaxN1 * kMaxDeg];  // Pd[q*k+m]     = its derivative
  T w[kMaxN1];             // Gauss weights on [0,1]
  T x[kMaxN1];             // Gauss points on [0,1]
  T nodes[kMaxN1];         // velocity Gauss-Lobatto nodes on [0,1]
};

// Transfer tables: for child h in {0,1}, fine local node a, coarse local node m:
// weight of coarse basis m at the fine node (reference coordinate (h + t_a)/2).
template <typename T>
struct TransferTab {
  T vel[2 * kMaxN1 * kMaxN1];   // [(h*(k+1)+a)*(k+1)+m]
  T pre[2 * kMaxDeg * kMaxDeg]; // [(h*k+a)*k+m]   (degree k-1, k nodes)
};

// Device-side description of one level of the structured hierarchy.
template <typename T>
struct LevelDesc {
  int dim, k;
  int n[3];          // cells per direction (n[2] = 1 in 2D)
  int N[3];          // velocity nodes per direction (k n + 1; 1 in unused dim)
  int Pn[3];         // pressure nodes per direction
  long long nv;      // nodes per velocity component
  long long n_u, n_p;
  long long n_cells;
  unsigned faces;    // Dirichlet face bits
  int cartesian;     // 1: axis-aligned uniform cells of size h (no vertex array)
  T h[3];            // Cartesian cell sizes
  const T *vert;     // (n+1)^d x d vertex coordinates (null if cartesian)
  const T *mu_cell;  // per-cell viscosity (null: constant mu)
  T mu, gamma_rho;
};

// Vector updates of the smoother folded into a 3D cell-kernel application (Sec. 3.3.1:
// Chebyshev-Jacobi recurrence and the inexact Uzawa step).  The kernel's input is not a stored
// vector but a pointwise combination evaluated while gathering,
//   velocity  u_in[i] = vb[i] + vd[i] * sum_{j < nv} vc[j] * vv[j][i]   (vb / vd may be null:
//             0 / 1; nv == 0: u_in = u),
//   pressure  p_in[i] = pd[i] * sum_{j < np} pc[j] * pv[j][i]           (np == 0: p_in = p),
// and the one cell that owns a node (the cell whose local index along each axis is below the
// last one, or the last cell along that axis) performs the side effects on that node:
//   vstore[i] = u_in[i]; vzero[*][i] = 0; pacc[i] += p_in[i]; pzero[*][i] = 0.
// Buffers written through these side effects are never read by the same launch.
constexpr int kFuseVel = 3, kFusePre = 6;
template <typename T>
struct Fuse {
  const T *vb = nullptr, *vd = nullptr;
  const T *vv[kFuseVel] = {};
  T vc[kFuseVel] = {};
  int nv = 0;
  T *vstore = nullptr;
  T *vzero[2] = {};
  const T *pd = nullptr;
  const T *pv[kFusePre] = {};
  T pc[kFusePre] = {};
  int np = 0;
  T *pacc = nullptr;
  T *pzero[kFusePre] = {};
};

__host__ __device__ inline bool vel_constrained(const int N[3], unsigned faces, int dim, int gx, int gy,
                                                int gz) {
  if ((faces & 1u) && gx == 0) return true;
  if ((faces & 2u) && gx == N[0] - 1) return true;
  if ((faces & 4u) && gy == 0) return true;
  if ((faces & 8u) && gy == N[1] - 1) return true;
  if (dim == 3) {
    if ((faces & 16u) && gz == 0) return true;
    if ((faces & 32u) && gz == N[2] - 1) return true;
  }
  return false;
}

// Programmatic dependent launch: let the next kernel in the stream start launching, then wait
// until every kernel this one depends on has completed and its writes are visible.  Both are
// no-ops when the kernel was launched without the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Grid-wide barrier of a cooperative launch with a bounded wait.  state (device, zeroed by the
// host before a launch sequence): [0] arrivals of the current round, [1] round counter, [2] error
// flag, [3] wait budget in clock64() cycles (as an unsigned; 0 means 2^31).  A CTA that waits longer
// than the budget sets the error flag and returns false; every CTA that sees the flag returns false,
// so no CTA waits for one that has left.
struct GridBarrier {
  unsigned *state = nullptr;
  // owner-computes form (owner != 0): no barrier; per-cell local results in loc32 / loc64 (by
  // precision), summed per DoF in a fixed order by a second pass
  int owner = 0;
  void *loc32 = nullptr, *loc64 = nullptr;
};
#if defined(__CUDACC__)
// Input loads of the kernels: plain (the compiler may use the read-only path) or, in the
// persistent work-queue kernel whose inputs are written by earlier work items of the same launch,
// L2 loads that bypass the per-SM caches (COH).  (L1-cached loads after the acquire fence measured
// the same: 14.2 ms for one cycle of the 16-member batch.)
template <bool COH, typename T>
__device__ __forceinline__ T ld_in(const T *p) {
  if constexpr (COH)
    return __ldcg(p);
  else
    return *p;
}

__device__ __forceinline__ bool grid_barrier(const GridBarrier &B) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *st = B.state;
    const unsigned round = st[1];
    __threadfence();
    int good = 1;
    if (atomicAdd(&B.state[0], 1u) == gridDim.x - 1) {
      atomicExch(&B.state[0], 0u);
      __threadfence();
      atomicAdd(&B.state[1], 1u);
    } else {
      const unsigned bud = st[3];
      const long long budget = bud ? (long long)bud : (1ll << 31);
      const long long t0 = clock64();
      while (st[1] == round) {
        if (st[2]) {
          good = 0;
          break;
        }
        if (clock64() - t0 > budget) {
          atomicExch(&B.state[2], 1u);
          good = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok = good && st[2] == 0;
  }
  __syncthreads();
  return ok != 0;
}
#endif

// Host side: launch with the programmatic-stream-serialization attribute (PDL) where pdl_on(s)
// says so (by default outside stream capture only).  Every kernel of the library begins with
// pdl_enter().
bool pdl_on(cudaStream_t s);
template <typename... KArgs, typename... Args>
inline void launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  if (pdl_on(s)) {
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

#define SMF_CUDA_OK(expr)                                        \
  do {                                                           \
    cudaError_t _e = (expr);                                     \
    if (_e != cudaSuccess) return ::smf::cuda_fail(_e, #expr, __FILE__, __LINE__); \
  } while (0)

int cuda_fail(cudaError_t e, const char *what, const char *file, int line);
void set_error(const std::string &msg);

}  // namespace smf
