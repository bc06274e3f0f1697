// C ABI of the matrix-free monolithic multigrid library: context, setup (Algorithm 2),
// smoother (Sec. 3.3.1), multigrid cycle (Algorithm 1), coarse solve (Sec. 4.1) and the
// FP64 flexible-GMRES outer loop.  Host code orchestrates; every vector operation runs
// in the kernels of apply.cuh, vec.cuh, transfer.cuh and kernels_misc.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/stokes_mf.h"
#include "common.cuh"
#include "host_tables.h"
#include "queue.h"
#include "transfer.cuh"
#include "vec.cuh"

namespace smf {

static thread_local std::string g_last_error;
// Programmatic dependent launch: 1 (default) for launches outside stream capture (direct calls
// such as stokes_vmult, where the next kernel's launch overlaps the current one), 0 inside
// captured graphs (measured faster for the solver's long chains of small kernels), 2 everywhere
// (STOKES_PDL=all), 0 everywhere (STOKES_NO_PDL=1).
static int pdl_mode() {
  static int v = -1;
  if (v < 0) {
    const char *e = getenv("STOKES_NO_PDL");
    const char *a = getenv("STOKES_PDL");
    v = (e && e[0] == '1') ? 0 : ((a && std::strcmp(a, "all") == 0) ? 2 : 1);
  }
  return v;
}
bool pdl_on(cudaStream_t s) {
  const int m = pdl_mode();
  if (m != 1) return m == 2;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs == cudaStreamCaptureStatusNone;
}
void set_error(const std::string &m) { g_last_error = m; }
int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  set_error(std::string("CUDA error '") + cudaGetErrorString(e) + "' in " + what + " (" + file + ":" +
            std::to_string(line) + ")");
  return STOKES_ECUDA;
}

template <typename T>
int launch_cell_apply(const LevelDesc<T> &L, const Tab1D<T> *tab, int mode, const T *u, const T *p, T *yu, T *yp,
                      cudaStream_t s, int shape, const T *geo, const T *rho, const GridBarrier *det) {
  if (shape == 5 || det) {
    // cell-component kernel (Laplacian form, constant rho); the column kernel serves the rest.
    // det: its deterministic cooperative form (setup admits deterministic mode only where it serves
    // every application of the solve)
    const bool generic_a = (mode & kApplyA) && ((mode & kApplySym) || rho);
    if (!generic_a) {
      const int r = L.k == 2 ? launch_cell_apply_cc_k<2, T>(L, mode, u, p, yu, yp, geo, det, s)
                             : (L.k == 3 ? launch_cell_apply_cc_k<3, T>(L, mode, u, p, yu, yp, geo, det, s) : -1);
      if (r == 0) return 0;
      if (r > 0) return cuda_fail((cudaError_t)r, "deterministic cell-kernel launch", __FILE__, __LINE__);
    }
    shape = 4;
  }
  switch (L.k) {
    case 2: return launch_cell_apply_k<2, T>(L, tab, mode, u, p, yu, yp, s, shape, geo, rho);
    case 3: return launch_cell_apply_k<3, T>(L, tab, mode, u, p, yu, yp, s, shape, geo, rho);
    default: return launch_cell_apply_k<4, T>(L, tab, mode, u, p, yu, yp, s, shape, geo, rho);
  }
}
template <typename T>
int launch_cell_C(const LevelDesc<T> &L, const Tab1D<T> *tab, T cm, T cg, const T *p, T *yp, T sign, T *diag,
                  const T *Ce, cudaStream_t s) {
  switch (L.k) {
    case 2: return launch_cell_C_k<2, T>(L, tab, cm, cg, p, yp, sign, diag, Ce, s);
    case 3: return launch_cell_C_k<3, T>(L, tab, cm, cg, p, yp, sign, diag, Ce, s);
    default: return launch_cell_C_k<4, T>(L, tab, cm, cg, p, yp, sign, diag, Ce, s);
  }
}
int launch_cell_C_matrix(const LevelDesc<double> &L, const Tab1D<double> *tab, double cm, double cg, double *Ce,
                         cudaStream_t s) {
  switch (L.k) {
    case 2: return launch_cell_C_matrix_k<2, double>(L, tab, cm, cg, Ce, s);
    case 3: return launch_cell_C_matrix_k<3, double>(L, tab, cm, cg, Ce, s);
    default: return launch_cell_C_matrix_k<4, double>(L, tab, cm, cg, Ce, s);
  }
}
template <typename T>
int launch_col_geometry(const LevelDesc<T> &L, T *geo, cudaStream_t s) {
  switch (L.k) {
    case 2: return launch_col_geometry_k<2, T>(L, geo, s);
    case 3: return launch_col_geometry_k<3, T>(L, geo, s);
    default: return launch_col_geometry_k<4, T>(L, geo, s);
  }
}
template <typename T>
int launch_cell_apply_fused(const LevelDesc<T> &L, int mode, const T *u, const T *p, T *yu, T *yp, cudaStream_t s,
                            int shape, const Fuse<T> &F, const T *geo) {
  switch (L.k) {
    case 2: return launch_cell_apply_fused_k<2, T>(L, mode, u, p, yu, yp, s, shape, F, geo);
    case 3: return launch_cell_apply_fused_k<3, T>(L, mode, u, p, yu, yp, s, shape, F, geo);
    default: return launch_cell_apply_fused_k<4, T>(L, mode, u, p, yu, yp, s, shape, F, geo);
  }
}
template <>
int launch_cell_diag<double>(const LevelDesc<double> &L, const Tab1D<double> *tab, double *a, double *b, double *c,
                             cudaStream_t s, const double *rho, int sym) {
  switch (L.k) {
    case 2: return launch_cell_diag_k<2, double>(L, tab, a, b, c, s, rho, sym);
    case 3: return launch_cell_diag_k<3, double>(L, tab, a, b, c, s, rho, sym);
    default: return launch_cell_diag_k<4, double>(L, tab, a, b, c, s, rho, sym);
  }
}

// x = Kinv b on the coarse level: one warp per row, FP64 accumulation.
template <typename T>
__global__ void k_coarse_apply(const double *__restrict__ Kinv, int n0, const T *__restrict__ b, T *__restrict__ x) {
  pdl_enter();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n0) return;
  const double *row = Kinv + (long long)warp * n0;
  double s = 0.0;
  for (int j = lane; j < n0; j += 32) s += row[j] * (double)b[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[warp] = (T)s;
}

// x[i * stride] += s
__global__ void k_add_strided(double *x, long long stride, double s, long long n) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) x[i * stride] += s;
}

// Physical coordinates of the velocity nodes of a level: node (g_x, g_y[, g_z]) lies in cell
// min(g / k, n - 1) at reference coordinate = Gauss-Lobatto node (g - k c); the cell map is the
// bi/trilinear map through its vertices (or the Cartesian box).  out: nv x dim, interleaved.
__global__ void k_velocity_nodes(const LevelDesc<double> L, const Tab1D<double> *__restrict__ tab, double *out) {
  pdl_enter();
  const int dim = L.dim, k = L.k;
  SMF_GRID_LOOP(i, L.nv) {
    const int g[3] = {(int)(i % L.N[0]), (int)((i / L.N[0]) % L.N[1]), dim == 3 ? (int)(i / ((long long)L.N[0] * L.N[1])) : 0};
    int c[3] = {0, 0, 0};
    double xi[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      c[a] = min(g[a] / k, L.n[a] - 1);
      xi[a] = tab->nodes[g[a] - k * c[a]];
    }
    for (int a = 0; a < dim; ++a) {
      double v = 0.0;
      if (L.cartesian) {
        v = (c[a] + xi[a]) * L.h[a];
      } else {
        for (int vtx = 0; vtx < (1 << dim); ++vtx) {
          const int vb[3] = {vtx & 1, (vtx >> 1) & 1, (vtx >> 2) & 1};
          double wgt = 1.0;
          for (int d = 0; d < dim; ++d) wgt *= vb[d] ? xi[d] : 1.0 - xi[d];
          const long long gv = dim == 3
                                   ? ((long long)(c[2] + vb[2]) * (L.n[1] + 1) + (c[1] + vb[1])) * (L.n[0] + 1) + (c[0] + vb[0])
                                   : (long long)(c[1] + vb[1]) * (L.n[0] + 1) + (c[0] + vb[0]);
          v += wgt * L.vert[gv * dim + a];
        }
      }
      out[i * dim + a] = v;
    }
  }
}

// ------------------------------------------------------------------------------------------
template <typename T>
struct LevelRT {
  LevelDesc<T> d{};
  int shape = 0;  // 3D cell-kernel launch shape chosen by the autotuner (see launch_cell_apply_k)
  int fshape = 4;  // column-kernel shape of the fused smoother's launches (1, 3 or 4)
  XferTabs<T> xf{};  // 1D transfer matrices between this level and the next coarser one
  bool fuse = true;  // fused smoothing on this level (set by the setup's timing, when eligible)
  const T *geo = nullptr;  // 3D trilinear: precomputed per-point geometry the column kernel reads
  const T *geo_stored = nullptr;  // FP32: the stored geometry, used (geo) where the setup's timing keeps it
  const T *rho = nullptr;  // per-cell density of the gamma rho mass term (null: rho = 1)
  const T *Ce = nullptr;   // packed element matrices of the stabilisation block C (null: on the fly)
  T *DAinv = nullptr, *DSinv = nullptr;
  T *x = nullptr, *b = nullptr, *r = nullptr, *kx = nullptr;                   // full vectors
  T *tu = nullptr, *ru = nullptr, *uhat = nullptr, *cx = nullptr, *cd = nullptr, *ct = nullptr;  // velocity
  T *r2 = nullptr, *cx2 = nullptr, *cd2 = nullptr, *ct2 = nullptr, *au = nullptr;              // nested in S~
  T *pt = nullptr, *rp = nullptr, *px = nullptr, *pd = nullptr, *ps = nullptr, *dp = nullptr;  // pressure
};

struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
};

// FMA throughput probe: 8 independent multiply-add chains per thread (x <- x m + c, contracting
// towards c / (1 - m)), `iters` x 16 rounds; the result is stored only if it equals -1, which the
// compiler cannot rule out, so no chain is removed.
template <typename T>
__global__ void k_fma_peak(T *out, int iters, T seed) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + T(threadIdx.x + j) * T(1e-7);
  const T m = T(0.999999), c = T(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
  }
  T sum = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) sum += a[j];
  if (sum == T(-1)) out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}
// The same chains in packed pairs: 4 float2 chains per thread, each step one paired FP32
// multiply-add (two FMAs per instruction).
__global__ void k_fma_peak_x2(float *out, int iters, float seed) {
  float2 a[4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
    a[j] = make_float2(seed + float(threadIdx.x + 2 * j) * 1e-7f, seed + float(threadIdx.x + 2 * j + 1) * 1e-7f);
  const float2 m = make_float2(0.999999f, 0.999999f), c = make_float2(1e-7f, 1e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) a[j] = __ffma2_rn(a[j], m, c);
  }
  float sum = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) sum += a[j].x + a[j].y;
  if (sum == -1.f) out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

}  // namespace smf

using namespace smf;

struct stokes_ctx {
  int dim = 0, k = 0, nl = 0;
  int device = -1;  // the CUDA device that was current at setup (every buffer lives there)
  stokes_opts o{};
  double mu = 1, gamma_rho = 0;
  double c_mass = 0, c_grad = 0;  // stabilisation block C (0: none)
  bool sym = false;               // symmetric-gradient form of a(u,v)
  std::vector<double> rho_host;   // caller's per-cell rho (finest level), kept for stokes_set_viscosity
  bool pker = false;
  std::vector<LevelRT<double>> L64;
  std::vector<LevelRT<float>> L32;
  std::vector<double *> DA, DS;    // FP64 diagonals per level (device)
  Tab1D<double> *tab64 = nullptr;
  Tab1D<float> *tab32 = nullptr;
  std::vector<double> betaA, betaS;
  double sigma = 1, tau = 1;
  int n0 = 0;
  double *Kinv = nullptr;
  // Krylov / Lanczos work space (FP64, finest level size)
  double *V = nullptr, *Z = nullptr, *w = nullptr, *hdev = nullptr, *partial = nullptr, *scal = nullptr;
  double *lz0 = nullptr, *lz1 = nullptr, *lz2 = nullptr, *lz3 = nullptr, *sq = nullptr;
  int restart = 30;
  std::vector<void *> allocs;
  std::string err;
  long long launches = 0;
  bool capturing = false;
  long long cap_count = 0;
  // recording of the FP32 cycle for the batched work-queue kernel (queue.h): while set, the FP32
  // Runner appends its operations here instead of launching them
  std::vector<PqOp> *pq = nullptr;
  int pq_member = 0;
  bool use_graphs = true;
  bool fuse = true;  // fused smoothing where eligible (STOKES_NO_FUSE=1: the unfused path)
  GraphSlot g32[2], g64[2];  // [x_zero]
  // FGMRES with the Arnoldi state on the device: one graph (conditional while node over the inner
  // iterations of a restart cycle) replayed per cycle; kry_mode -1 not built yet, 0 host-driven
  // loop (STOKES_HOST_KRYLOV=1, or conditional graph nodes unavailable), 1 device loop
  KrylovDev kd{};
  double *zcur = nullptr;
  // deterministic mode (opts.deterministic): every 3D cell-kernel application runs in the
  // cooperative colour-class form; gb: its grid-barrier state (arrivals, round, error, budget)
  bool det = false;
  GridBarrier gb{};
  cudaGraphExec_t kry = nullptr;
  long long kry_body = 0;
  int kry_mode = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // setup inputs, kept for stokes_set_viscosity
  stokes_mesh mesh{};
  std::vector<double> mesh_vertices;
  double mu_const = 1.0;
};

namespace smf {

template <typename T>
static int dalloc(stokes_ctx *C, T **p, long long n) {
  if (n <= 0) n = 1;
  cudaError_t e = cudaMalloc((void **)p, (size_t)n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of " + std::to_string((long long)n * sizeof(T)) + " bytes failed");
    return STOKES_ENOMEM;
  }
  C->allocs.push_back((void *)*p);
  SMF_CUDA_OK(cudaMemsetAsync(*p, 0, (size_t)n * sizeof(T), C->s));
  return STOKES_OK;
}

template <typename T>
std::vector<LevelRT<T>> &levels(stokes_ctx *C);
template <>
std::vector<LevelRT<double>> &levels<double>(stokes_ctx *C) { return C->L64; }
template <>
std::vector<LevelRT<float>> &levels<float>(stokes_ctx *C) { return C->L32; }
template <typename T>
const Tab1D<T> *tables(stokes_ctx *C);
template <>
const Tab1D<double> *tables<double>(stokes_ctx *C) { return C->tab64; }
template <>
const Tab1D<float> *tables<float>(stokes_ctx *C) { return C->tab32; }
template <typename T>
GraphSlot &graph_slot(stokes_ctx *C, bool x_zero);
template <>
GraphSlot &graph_slot<double>(stokes_ctx *C, bool x_zero) { return C->g64[x_zero ? 1 : 0]; }
template <>
GraphSlot &graph_slot<float>(stokes_ctx *C, bool x_zero) { return C->g32[x_zero ? 1 : 0]; }

// Chebyshev three-term recurrence coefficients (Sec. 3.3.1) for [alpha, beta] = [beta/2, beta].
struct ChebCoef {
  double c0;
  int k;
  double c1[17], c2[17];
};
static ChebCoef cheb_coef(int k, double beta) {
  ChebCoef c{};
  const double alpha = 0.5 * beta, theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha);
  const double s1 = theta / delta;
  double rho = 1.0 / s1;
  c.c0 = 1.0 / theta;
  c.k = k;
  for (int j = 1; j <= k; ++j) {
    const double rn = 1.0 / (2.0 * s1 - rho);
    c.c1[j] = rn * rho;
    c.c2[j] = 2.0 * rn / delta;
    rho = rn;
  }
  return c;
}

static double lemma1_scaling(int k) {
  // sigma = C_{k+1}(3) / (1 + C_{k+1}(3)), Chebyshev polynomial by its recurrence (Lemma 1)
  double c0 = 1.0, c1 = 3.0;
  for (int j = 1; j < k + 1; ++j) {
    double c2 = 6.0 * c1 - c0;
    c0 = c1;
    c1 = c2;
  }
  return c1 / (1.0 + c1);
}

template <typename T>
struct Runner {
  stokes_ctx *C;
  cudaStream_t s;
  std::vector<LevelRT<T>> &L;
  const Tab1D<T> *tab;
  explicit Runner(stokes_ctx *c) : C(c), s(c->s), L(levels<T>(c)), tab(tables<T>(c)) {}
  // launches on the caller's stream (which may be the default stream 0)
  struct OnStream {};
  Runner(stokes_ctx *c, cudaStream_t stream, OnStream) : C(c), s(stream), L(levels<T>(c)), tab(tables<T>(c)) {}

  void note() {
    if (C->capturing)
      ++C->cap_count;
    else
      ++C->launches;
  }
  void zero(T *p, long long n) { cudaMemsetAsync(p, 0, (size_t)n * sizeof(T), s); }
  long long nu(int l) const { return L[l].d.n_u; }
  long long np(int l) const { return L[l].d.n_p; }
  template <typename... KA, typename... A>
  void vec(void (*k)(KA...), long long n, A... args) {
    launch_kernel(k, dim3(vec_blocks(n)), dim3(kVecThreads), 0, s, args...);
    note();
  }
  // Packed launch: kv processes 16-byte packs (VW elements), k1 single elements; kv is chosen
  // when every pointer in `ptrs` is 16-byte aligned.
  static constexpr int VW = 16 / sizeof(T);
  template <typename K1, typename KV, typename... A>
  void vecp(K1 k1, KV kv, std::initializer_list<const void *> ptrs, long long n, A... args) {
    if (all_aligned(16, ptrs))
      launch_kernel(kv, dim3(vec_blocks((n + VW - 1) / VW)), dim3(kVecThreads), 0, s, args...);
    else
      launch_kernel(k1, dim3(vec_blocks(n)), dim3(kVecThreads), 0, s, args...);
    note();
  }

  // Public form: outputs are zeroed, then accumulated by the cell kernel.
  void apply(int l, int mode, const T *u, const T *p, T *yu, T *yp) {
    if (yu) zero(yu, nu(l));
    if (yp) zero(yp, np(l));
    apply_nz(l, mode, u, p, yu, yp);
  }
  // Recording for the work-queue kernel (FP32 only): the operation is appended instead of launched.
  bool rec() const { return std::is_same<T, float>::value && C->pq != nullptr; }
  PqOp &rec_op(int type, int l) {
    C->pq->emplace_back();
    PqOp &o = C->pq->back();
    o.type = type;
    o.member = C->pq_member;
    if constexpr (std::is_same<T, float>::value) o.F = L[l].d;
    return o;
  }
  void rec_xfer(PqOp &o, int lf) {
    if constexpr (std::is_same<T, float>::value) {
      o.Cd = L[lf - 1].d;
      o.X = L[lf].xf;
    }
  }
  static float *fp(T *p) { return reinterpret_cast<float *>(p); }
  static const float *fp(const T *p) { return reinterpret_cast<const float *>(p); }
  // Cycle form: the outputs are already zero (work buffers are zeroed by the kernel that
  // consumes them, so the captured cycle contains kernels only).
  void apply_nz(int l, int mode, const T *u, const T *p, T *yu, T *yp) {
    if (rec()) {
      PqOp &o = rec_op(kPqCell, l);
      o.mode = mode;
      o.in[0] = fp(u);
      o.in[1] = fp(p);
      o.out[0] = fp(yu);
      o.out[1] = fp(yp);
      o.items = pq_items(o);
      return;
    }
    launch_cell_apply<T>(L[l].d, tab, form(mode), u, p, yu, yp, s, L[l].shape, L[l].geo, L[l].rho,
                         C->det ? &C->gb : nullptr);
    note();
  }
  void vmult(int l, const T *x, T *y, bool identity) {
    if (identity) {  // y = identity rows of x (0 elsewhere), then the cell kernel accumulates
      vec(k_init_identity<T>, nu(l) + np(l), L[l].d, x, y);
      apply_nz(l, kApplyA | kApplyBT | kApplyB, x, x + nu(l), y, y + nu(l));
    } else {
      apply(l, kApplyA | kApplyBT | kApplyB, x, x + nu(l), y, y + nu(l));
    }
    applyC(l, x + nu(l), y + nu(l), T(-1));
  }
  // Stabilisation block (no launch when C = 0): yp += sign C p.
  bool hasC() const { return C->c_mass != 0.0 || C->c_grad != 0.0; }
  // the velocity block's form: the symmetric-gradient bit joins every application of A
  int form(int mode) const { return (C->sym && (mode & kApplyA)) ? (mode | kApplySym) : mode; }
  void applyC(int l, const T *p, T *yp, T sign) {
    if (!hasC()) return;
    launch_cell_C<T>(L[l].d, tab, (T)C->c_mass, (T)C->c_grad, p, yp, sign, (T *)nullptr, L[l].Ce, s);
    note();
  }
  void sub(const T *a, const T *b, T *out, long long n) { vec(k_sub<T>, n, a, b, out, n); }

  // Chebyshev-Jacobi application (Sec. 3.3.1) from a zero start on r = sr (a - b):
  //   f = base + fscale * scale * Cheb(M, D, k) r, written to out and/or accumulated into acc.
  // velocity: M = A, D = D_A, (k, beta, scale) = (k_A, beta_A, sigma)
  // pressure: M = S~ = B A^-1_hat B^T, D = D_S, (k_S, beta_S, tau)
  // za / zb: buffers zeroed after a / b are read (apply targets).
  void cheb(int l, bool velocity, bool nested, const T *a, const T *b, T *za, T *zb, T sr, const T *base, T fscale,
            T *out, T *acc) {
    LevelRT<T> &R = L[l];
    const int kd = velocity ? C->o.kA : C->o.kS;
    const ChebCoef cc = cheb_coef(kd, velocity ? C->betaA[l] : C->betaS[l]);
    const T scale = (T)(fscale * (velocity ? C->sigma : C->tau));
    const T *Dinv = velocity ? R.DAinv : R.DSinv;
    const long long n = velocity ? nu(l) : np(l);
    T *rb, *xb, *db, *tb;
    if (velocity) {
      rb = nested ? R.r2 : R.ru;
      xb = nested ? R.cx2 : R.cx;
      db = nested ? R.cd2 : R.cd;
      tb = nested ? R.ct2 : R.ct;
    } else {
      rb = R.rp;
      xb = R.px;
      db = R.pd;
      tb = R.ps;
    }
    if (kd == 0) {
      cheb_init_op(l, n, a, b, sr, Dinv, (T)cc.c0, (T *)nullptr, db, xb, base, scale, out, acc, za, zb);
      return;
    }
    cheb_init_op(l, n, a, b, sr, Dinv, (T)cc.c0, rb, db, xb, (const T *)nullptr, T(0), (T *)nullptr, (T *)nullptr, za,
                 zb);
    for (int j = 1; j <= kd; ++j) {
      if (velocity)
        apply_nz(l, kApplyA, xb, nullptr, tb, nullptr);
      else
        S_tilde(l, xb, tb);
      const bool last = j == kd;
      const T *bs = last ? base : nullptr;
      T *fo = last ? out : nullptr, *ac = last ? acc : nullptr;
      cheb_step_op(l, n, rb, tb, Dinv, (T)cc.c1[j], (T)cc.c2[j], db, xb, bs, scale, fo, ac);
    }
  }
  // The two Chebyshev vector kernels (k_cheb_init / k_cheb_step), launched or recorded.
  void cheb_init_op(int l, long long n, const T *a, const T *b, T sr, const T *Dinv, T c0, T *r_out, T *d, T *x,
                    const T *base, T fscale, T *final_out, T *acc_out, T *za, T *zb) {
    if (rec()) {
      PqOp &o = rec_op(kPqChebInit, l);
      o.n = n;
      const float *in[4] = {fp(a), fp(b), fp(Dinv), fp(base)};
      float *out[7] = {fp(r_out), fp(d), fp(x), fp(final_out), fp(acc_out), fp(za), fp(zb)};
      std::copy(in, in + 4, o.in);
      std::copy(out, out + 7, o.out);
      o.sc[0] = (float)sr;
      o.sc[1] = (float)c0;
      o.sc[2] = (float)fscale;
      o.vec4 = all_aligned(16, {a, b, Dinv, r_out, d, x, base, final_out, acc_out, za, zb}) ? 1 : 0;
      o.items = pq_items(o);
      return;
    }
    vecp(k_cheb_init<T, 1>, k_cheb_init<T, VW>, {a, b, Dinv, r_out, d, x, base, final_out, acc_out, za, zb}, n, a, b,
         sr, Dinv, c0, r_out, d, x, base, fscale, final_out, acc_out, za, zb, n);
  }
  void cheb_step_op(int l, long long n, const T *r, T *t, const T *Dinv, T c1, T c2, T *d, T *x, const T *base,
                    T fscale, T *final_out, T *acc_out) {
    if (rec()) {
      PqOp &o = rec_op(kPqChebStep, l);
      o.n = n;
      o.in[0] = fp(r);
      o.in[1] = fp(Dinv);
      o.in[2] = fp(base);
      float *out[5] = {fp(t), fp(d), fp(x), fp(final_out), fp(acc_out)};
      std::copy(out, out + 5, o.out);
      o.sc[0] = (float)c1;
      o.sc[1] = (float)c2;
      o.sc[2] = (float)fscale;
      o.vec4 = all_aligned(16, {r, t, Dinv, d, x, base, final_out, acc_out}) ? 1 : 0;
      o.items = pq_items(o);
      return;
    }
    vecp(k_cheb_step<T, 1>, k_cheb_step<T, VW>, {r, t, Dinv, d, x, base, final_out, acc_out}, n, r, t, Dinv, c1, c2,
         d, x, base, fscale, final_out, acc_out, n);
  }
  // y = B A^-1_hat B^T q   (y zero on entry)
  void S_tilde(int l, const T *q, T *y) {
    LevelRT<T> &R = L[l];
    apply_nz(l, kApplyBT, nullptr, q, R.tu, nullptr);
    cheb(l, true, true, R.tu, nullptr, R.tu, nullptr, T(1), nullptr, T(1), R.au, nullptr);
    apply_nz(l, kApplyB, R.au, nullptr, nullptr, y);
    applyC(l, q, y, T(1));  // S~ = B A^-1_hat B^T + C
  }
  // One inexact symmetric Uzawa step in compact form (Sec. 3.3.1, K_hat):
  //   u_hat = u + A^-1_hat (f - A u - B^T p); dp = S^-1_hat (B u_hat - g);
  //   u = u_hat - A^-1_hat B^T dp; p = p + dp
  // x_zero: x is known to be zero on entry (first step on a coarse level), so A u + B^T p = 0.
  void smooth_step(int l, T *x, const T *bv, bool x_zero) {
    LevelRT<T> &R = L[l];
    const long long n_u = nu(l);
    T *u = x, *p = x + n_u;
    const T *f = bv, *g = bv + n_u;
    if (!x_zero) apply_nz(l, kApplyA | kApplyBT, u, p, R.tu, nullptr);
    cheb(l, true, false, f, x_zero ? nullptr : R.tu, nullptr, x_zero ? nullptr : R.tu, T(1), u, T(1), R.uhat,
         nullptr);
    apply_nz(l, kApplyB, R.uhat, nullptr, nullptr, R.pt);
    applyC(l, p, R.pt, T(-1));  // B u_hat - C p
    cheb(l, false, false, R.pt, g, R.pt, nullptr, T(1), nullptr, T(1), R.dp, p);
    apply_nz(l, kApplyBT, nullptr, R.dp, R.tu, nullptr);
    cheb(l, true, false, R.tu, nullptr, R.tu, nullptr, T(1), R.uhat, T(-1), u, nullptr);
  }
  void coarse(const T *b, T *x) {
    const int n0 = C->n0;
    if (rec()) {
      PqOp &o = rec_op(kPqCoarse, 0);
      o.in[0] = fp(b);
      o.out[0] = fp(x);
      o.Kinv = (const double *)C->Kinv;
      o.n0 = n0;
      o.items = pq_items(o);
      return;
    }
    launch_kernel(k_coarse_apply<T>, dim3((n0 * 32 + 255) / 256), dim3(256), 0, s, (const double *)C->Kinv, n0, b, x);
    note();
  }
  // restriction out = P^T in, or P^T (in - sub) (the residual formed while restricting)
  template <int W>
  void restrict_w(int lf, const T *in, T *out, T *zero_c, const T *sub) {
    const long long n = nu(lf - 1) + np(lf - 1);
    if (rec()) {
      PqOp &o = rec_op(kPqRestrict, lf);
      rec_xfer(o, lf);
      o.W = W;
      o.in[0] = fp(in);
      o.in[1] = fp(sub);
      o.out[0] = fp(out);
      o.out[1] = fp(zero_c);
      o.items = pq_items(o);
      return;
    }
    if (sub) {
      if (n < 32768)
        vec(k_restrict<T, W, 8, true>, n * 8, L[lf].d, L[lf - 1].d, L[lf].xf, in, out, zero_c, sub);
      else
        vec(k_restrict<T, W, 1, true>, n, L[lf].d, L[lf - 1].d, L[lf].xf, in, out, zero_c, sub);
    } else {
      if (n < 32768)
        vec(k_restrict<T, W, 8, false>, n * 8, L[lf].d, L[lf - 1].d, L[lf].xf, in, out, zero_c, sub);
      else
        vec(k_restrict<T, W, 1, false>, n, L[lf].d, L[lf - 1].d, L[lf].xf, in, out, zero_c, sub);
    }
  }
  void restrict_to(int lf, const T *in, T *out, T *zero_c, const T *sub = nullptr) {
    switch (L[lf].d.k) {
      case 2: restrict_w<9>(lf, in, out, zero_c, sub); break;
      case 3: restrict_w<13>(lf, in, out, zero_c, sub); break;
      default: restrict_w<17>(lf, in, out, zero_c, sub); break;
    }
  }
  void prolongate(int lf, const T *in, T *out, int add, T *z0 = nullptr, T *z1 = nullptr, T *zf = nullptr) {
    const long long n = nu(lf) + np(lf);
    if (rec()) {
      PqOp &o = rec_op(kPqProlong, lf);
      rec_xfer(o, lf);
      o.W = L[lf].xf.W;
      o.in[0] = fp(in);
      o.out[0] = fp(out);
      o.out[1] = fp(z0);
      o.out[2] = fp(z1);
      o.out[3] = fp(zf);
      o.add = add;
      o.items = pq_items(o);
      return;
    }
    switch (L[lf].d.k) {
      case 2: vec(k_prolongate<T, 9>, n, L[lf].d, L[lf - 1].d, L[lf].xf, in, out, add, z0, z1, zf); break;
      case 3: vec(k_prolongate<T, 13>, n, L[lf].d, L[lf - 1].d, L[lf].xf, in, out, add, z0, z1, zf); break;
      default: vec(k_prolongate<T, 17>, n, L[lf].d, L[lf - 1].d, L[lf].xf, in, out, add, z0, z1, zf); break;
    }
  }
  // ---- fused smoothing: k_A = 1, 3D column kernel ------------------------------------------
  // The Chebyshev-Jacobi and Uzawa vector updates of smooth_step are folded into the gathers of
  // the cell-kernel applications (Fuse descriptors), so a step is 5 + 3 k_S launches instead of
  // 10 + 6 k_S.  Work buffers: two velocity pairs (TU: B^T / A|B^T target, T: A target) used
  // alternately, the stored u_hat, and the pressure targets pt, ps_1..ps_kS.  Every buffer
  // accumulated into is zero when the launch that accumulates starts; the launch that last
  // reads it is followed by one whose owners zero it.  A step ends with the update
  // u = u_hat - A^-1_hat B^T dp still pending; it is folded into the next gather of u (next
  // step, residual) or written by k_fused_finish.
  bool fused_ok(int l) const { return fused_eligible(l) && L[l].fuse; }
  bool fused_eligible(int l) const {
    return C->fuse && !C->det && !hasC() && !C->sym && !L[l].rho && C->o.kA == 1 && C->o.kS >= 1 && C->o.kS <= 4 &&
           L[l].d.dim == 3 && L[l].shape >= 0;
  }
  T *pairU(int l, int pr) { return pr == 0 ? L[l].tu : L[l].cx; }
  T *pairT(int l, int pr) { return pr == 0 ? L[l].ct : L[l].ct2; }
  T *psb(int l, int j) {
    LevelRT<T> &R = L[l];
    T *b[4] = {R.ps, R.rp, R.px, R.pd};
    return b[j];
  }
  void fapply(int l, int mode, const T *u, const T *p, T *yu, T *yp, const Fuse<T> &F) {
    if (L[l].shape == 5) {  // the cell-component kernel's fused form where it has one (k = 2)
      const int r = launch_cell_apply_cc_fused_k<2, T>(L[l].d, mode, u, p, yu, yp, L[l].geo, F, s);
      if (r == 0) {
        note();
        return;
      }
    }
    const int sh = L[l].shape == 5 ? L[l].fshape : L[l].shape;
    launch_cell_apply_fused<T>(L[l].d, mode, u, p, yu, yp, s, sh, F, L[l].geo);
    note();
  }
  // Velocity Chebyshev with k_A = 1 from zero on r: x_1 = c0 D^-1 r, t = A x_1,
  // x_2 = D^-1 (ra r + ta t)  (Sec. 3.3.1 recurrence with one step).
  struct VelCoef {
    double c0, ra, ta;
  };
  VelCoef vcoef(int l) const {
    const ChebCoef cc = cheb_coef(1, C->betaA[l]);
    return {cc.c0, (1 + cc.c1[1]) * cc.c0 + cc.c2[1], -cc.c2[1]};
  }
  // Pressure Chebyshev with k_S steps from zero on r, in the basis {r, t_1, ..., t_kS} scaled by
  // D_S^-1: x_j = D_S^-1 (X[j][0] r + sum_i X[j][i] t_i), t_j = S~ x_j, j = 1..k_S+1.
  void pcoef(int l, double X[6][6]) const {
    const int k = C->o.kS;
    const ChebCoef cc = cheb_coef(k, C->betaS[l]);
    double x[6] = {cc.c0, 0, 0, 0, 0, 0}, d[6] = {cc.c0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 6; ++i) X[1][i] = x[i];
    for (int j = 1; j <= k; ++j) {
      for (int i = 0; i < 6; ++i) d[i] *= cc.c1[j];
      d[0] += cc.c2[j];
      d[j] -= cc.c2[j];
      for (int i = 0; i < 6; ++i) x[i] += d[i];
      for (int i = 0; i < 6; ++i) X[j + 1][i] = x[i];
    }
  }
  // The pending last line of the previous step as the velocity input, stored into u.
  void set_pending(Fuse<T> &F, int l, int pend, T *u) {
    const VelCoef vc = vcoef(l);
    const double sg = C->sigma;
    F.vb = L[l].uhat;
    F.vd = L[l].DAinv;
    F.vv[0] = pairU(l, pend);
    F.vc[0] = (T)(-sg * vc.ra);
    F.vv[1] = pairT(l, pend);
    F.vc[1] = (T)(-sg * vc.ta);
    F.nv = 2;
    F.vstore = u;
  }
  void set_pzero(Fuse<T> &F, int l) {
    F.pzero[0] = L[l].pt;
    for (int j = 0; j < C->o.kS; ++j) F.pzero[1 + j] = psb(l, j);
  }
  // One inexact Uzawa step (same arithmetic as smooth_step, fused).  pend: in, the pair holding
  // the previous step's pending update (-1: none); out, this step's.
  void fused_step(int l, T *x, const T *bv, bool x_zero, int &pend) {
    LevelRT<T> &R = L[l];
    const long long n_u = nu(l);
    T *u = x, *p = x + n_u;
    const T *f = bv, *g = bv + n_u;
    const VelCoef vc = vcoef(l);
    const double sg = C->sigma, tau = C->tau;
    const int kS = C->o.kS;
    double X[6][6] = {};
    pcoef(l, X);
    int pr = pend >= 0 ? 1 - pend : 0;
    if (!x_zero) {  // TU = A u + B^T p
      Fuse<T> F;
      const T *uin = u;
      if (pend >= 0) {
        set_pending(F, l, pend, u);
        uin = nullptr;
      }
      set_pzero(F, l);
      fapply(l, kApplyA | kApplyBT, uin, p, pairU(l, pr), nullptr, F);
    }
    {  // T = A x_1, x_1 = c0 D_A^-1 (f - TU)
      Fuse<T> F;
      F.vd = R.DAinv;
      F.vv[0] = f;
      F.vc[0] = (T)vc.c0;
      F.nv = 1;
      if (!x_zero) {
        F.vv[1] = pairU(l, pr);
        F.vc[1] = (T)(-vc.c0);
        F.nv = 2;
      }
      if (pend >= 0) {
        F.vzero[0] = pairU(l, pend);
        F.vzero[1] = pairT(l, pend);
      }
      fapply(l, kApplyA, nullptr, nullptr, pairT(l, pr), nullptr, F);
    }
    pend = -1;
    {  // u_hat = u + sigma x_2 (stored); pt = B u_hat
      Fuse<T> F;
      F.vd = R.DAinv;
      int j = 0;
      F.vv[j] = f;
      F.vc[j++] = (T)(sg * vc.ra);
      if (!x_zero) {
        F.vv[j] = pairU(l, pr);
        F.vc[j++] = (T)(-sg * vc.ra);
        F.vb = u;
      }
      F.vv[j] = pairT(l, pr);
      F.vc[j++] = (T)(sg * vc.ta);
      F.nv = j;
      F.vstore = R.uhat;
      fapply(l, kApplyB, nullptr, nullptr, nullptr, R.pt, F);
    }
    // dp = tau Cheb(S~, D_S, k_S)(pt - g); each S~ x_j = B A^-1_hat B^T x_j
    for (int j = 1; j <= kS + 1; ++j) {
      const bool last = j == kS + 1;
      const int prev = pr;
      pr = 1 - pr;
      const double sc = last ? tau : 1.0;
      {  // TU = B^T x_j  (last: B^T dp, and p += dp)
        Fuse<T> F;
        F.pd = R.DSinv;
        F.pv[0] = R.pt;
        F.pc[0] = (T)(sc * X[j][0]);
        F.pv[1] = g;
        F.pc[1] = (T)(-sc * X[j][0]);
        for (int i = 1; i < j; ++i) {
          F.pv[1 + i] = psb(l, i - 1);
          F.pc[1 + i] = (T)(sc * X[j][i]);
        }
        F.np = j + 1;
        F.vzero[0] = pairU(l, prev);
        F.vzero[1] = pairT(l, prev);
        if (last) F.pacc = p;
        fapply(l, kApplyBT, nullptr, nullptr, pairU(l, pr), nullptr, F);
      }
      {  // T = A (c0 D_A^-1 TU)
        Fuse<T> F;
        F.vd = R.DAinv;
        F.vv[0] = pairU(l, pr);
        F.vc[0] = (T)vc.c0;
        F.nv = 1;
        fapply(l, kApplyA, nullptr, nullptr, pairT(l, pr), nullptr, F);
      }
      if (!last) {  // t_j = B (sigma D_A^-1 (ra TU + ta T))
        Fuse<T> F;
        F.vd = R.DAinv;
        F.vv[0] = pairU(l, pr);
        F.vc[0] = (T)(sg * vc.ra);
        F.vv[1] = pairT(l, pr);
        F.vc[1] = (T)(sg * vc.ta);
        F.nv = 2;
        fapply(l, kApplyB, nullptr, nullptr, nullptr, psb(l, j - 1), F);
      }
    }
    pend = pr;
  }
  // kx = K x with the pending update folded in (x stored), pressure work vectors zeroed.
  void fused_residual_apply(int l, T *x, int pend) {
    LevelRT<T> &R = L[l];
    Fuse<T> F;
    const T *uin = x;
    if (pend >= 0) {
      set_pending(F, l, pend, x);
      uin = nullptr;
    }
    set_pzero(F, l);
    fapply(l, kApplyA | kApplyBT | kApplyB, uin, x + nu(l), R.kx, R.kx + nu(l), F);
  }
  void fused_finish(int l, T *x, int pend) {
    LevelRT<T> &R = L[l];
    const VelCoef vc = vcoef(l);
    const double sg = C->sigma;
    ZeroList<T> z{};
    z.p[0] = R.pt;
    for (int j = 0; j < C->o.kS; ++j) z.p[1 + j] = psb(l, j);
    z.n = 1 + C->o.kS;
    vec(k_fused_finish<T>, std::max(nu(l), np(l)), (const T *)R.uhat, (const T *)R.DAinv, pairU(l, pend),
        pairT(l, pend), (T)(-sg * vc.ra), (T)(-sg * vc.ta), x, nu(l), z, np(l));
  }
  // `steps` smoothing steps on level l (x_zero: x is zero on entry).
  void smooth(int l, T *x, const T *b, int steps, bool x_zero) {
    if (!fused_ok(l)) {
      for (int i = 0; i < steps; ++i) smooth_step(l, x, b, x_zero && i == 0);
      return;
    }
    int pend = -1;
    for (int i = 0; i < steps; ++i) fused_step(l, x, b, x_zero && i == 0, pend);
    if (pend >= 0) fused_finish(l, x, pend);
  }

  // Algorithm 1: MG(x_l, b_l) with gamma = 1 (V) or 2 (W); returns after the coarse solve on l = 0.
  void cycle(int l, T *x, const T *b, bool x_zero) {
    if (l == 0) {
      coarse(b, x);
      return;
    }
    LevelRT<T> &R = L[l];
    const bool fz = fused_ok(l);
    int pend = -1;
    for (int i = 0; i < C->o.m; ++i) {
      if (fz)
        fused_step(l, x, b, x_zero && i == 0, pend);
      else
        smooth_step(l, x, b, x_zero && i == 0);
    }
    // residual b - K x (Algorithm 1) formed inside the restriction; the K x accumulator is zeroed
    // again by the prolongation below
    const bool kx_used = !(C->o.m == 0 && x_zero);
    if (!kx_used) {
      restrict_to(l, b, L[l - 1].b, L[l - 1].x);  // r = b - K 0
    } else {
      if (fz)
        fused_residual_apply(l, x, pend);
      else
        apply_nz(l, kApplyA | kApplyBT | kApplyB, x, x + nu(l), R.kx, R.kx + nu(l));
      applyC(l, x + nu(l), R.kx + nu(l), T(-1));
      restrict_to(l, b, L[l - 1].b, L[l - 1].x, R.kx);
    }
    const int gam = C->o.cycle == 1 ? 2 : 1;
    for (int j = 0; j < gam; ++j) cycle(l - 1, L[l - 1].x, L[l - 1].b, j == 0);
    prolongate(l, L[l - 1].x, x, 1, pend >= 0 ? pairU(l, pend) : nullptr, pend >= 0 ? pairT(l, pend) : nullptr,
               kx_used ? R.kx : nullptr);
    pend = -1;
    for (int i = 0; i < C->o.m; ++i) {
      if (fz)
        fused_step(l, x, b, false, pend);
      else
        smooth_step(l, x, b, false);
    }
    if (pend >= 0) fused_finish(l, x, pend);
  }
  // One cycle on the finest level on the internal top-level buffers, replayed from a captured
  // graph (one graph per precision and per "x is zero on entry").
  int top_cycle(bool x_zero) {
    const int top = C->nl - 1;
    if (!C->use_graphs) {
      cycle(top, L[top].x, L[top].b, x_zero);
      return STOKES_OK;
    }
    GraphSlot &g = graph_slot<T>(C, x_zero);
    if (!g.exec) {
      SMF_CUDA_OK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      C->capturing = true;
      C->cap_count = 0;
      cycle(top, L[top].x, L[top].b, x_zero);
      C->capturing = false;
      cudaGraph_t graph;
      SMF_CUDA_OK(cudaStreamEndCapture(s, &graph));
      cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      SMF_CUDA_OK(e);
      g.kernels = C->cap_count;
    }
    SMF_CUDA_OK(cudaGraphLaunch(g.exec, s));
    C->launches += g.kernels;
    return STOKES_OK;
  }
};

// ---- FP64 reductions returning host scalars ------------------------------------------------
static int dot64(stokes_ctx *C, const double *a, const double *b, long long n, double *out) {
  k_mdot_partial<<<kRedBlocks, kVecThreads, 0, C->s>>>(a, n, 1, b, n, C->partial);
  k_final_reduce<<<1, kVecThreads, 0, C->s>>>(C->partial, kRedBlocks, 1, C->scal);
  C->launches += 2;
  SMF_CUDA_OK(cudaMemcpyAsync(out, C->scal, sizeof(double), cudaMemcpyDeviceToHost, C->s));
  SMF_CUDA_OK(cudaStreamSynchronize(C->s));
  return STOKES_OK;
}

static int sum64(stokes_ctx *C, const double *a, long long n, double *dev_out) {
  k_sum_partial<<<kRedBlocks, kVecThreads, 0, C->s>>>(a, n, C->partial);
  k_final_reduce<<<1, kVecThreads, 0, C->s>>>(C->partial, kRedBlocks, 1, dev_out);
  C->launches += 2;
  return STOKES_OK;
}

// Largest Ritz value of plain Lanczos on D^{-1/2} M D^{-1/2} (Algorithm 2's lambda_max).
// velocity: M = A on level l; pressure: M = S~.  Start vector: SplitMix64(seed) (velocity,
// constrained entries zeroed) or SplitMix64(seed + 1) with the kernel direction D^{1/2} 1
// projected out under full Dirichlet data.
// ---- Schur-complement diagonals "d" and "exact" (Algorithm 2, choice of D_S~) by probing -----
// On the structured grid, velocity nodes whose indices differ by a multiple of 2k+1 along every
// axis never share a pressure row of B, and pressure nodes (k-1)(k_A+3)+1 apart along every axis
// are never coupled by S~ = B A^-1_hat B^T (its reach is B^T, k_A applications of A and B, about
// k_A + 2 cells).  Probing with one vector per colour therefore yields one entry per row.
__device__ __forceinline__ bool probe_colour(const int *g, int dim, int P, int cx, int cy, int cz) {
  return g[0] % P == cx && g[1] % P == cy && (dim < 3 || g[2] % P == cz);
}
// v = D_A^-1/2 on the free DoFs of velocity component comp in the colour, 0 elsewhere.
__global__ void k_probe_vel(const LevelDesc<double> L, int comp, int P, int cx, int cy, int cz,
                            const double *__restrict__ DAinv, double *__restrict__ v) {
  pdl_enter();
  SMF_GRID_LOOP(i, L.n_u) {
    const long long node = i % L.nv;
    const int c = (int)(i / L.nv);
    const int g[3] = {(int)(node % L.N[0]), (int)((node / L.N[0]) % L.N[1]), (int)(node / ((long long)L.N[0] * L.N[1]))};
    const bool on = c == comp && probe_colour(g, L.dim, P, cx, cy, cz) &&
                    !vel_constrained(L.N, L.faces, L.dim, g[0], g[1], g[2]);
    v[i] = on ? sqrt(DAinv[i]) : 0.0;
  }
}
__global__ void k_add_sq(const double *__restrict__ y, double *__restrict__ acc, long long n) {
  pdl_enter();
  SMF_GRID_LOOP(i, n) acc[i] += y[i] * y[i];
}
// q = 1 on the pressure nodes of the colour; with add_from: acc += w on those nodes.
__global__ void k_probe_pre(const LevelDesc<double> L, int P, int cx, int cy, int cz, double *__restrict__ q,
                            const double *__restrict__ add_from, double *__restrict__ acc) {
  pdl_enter();
  SMF_GRID_LOOP(i, L.n_p) {
    const int g[3] = {(int)(i % L.Pn[0]), (int)((i / L.Pn[0]) % L.Pn[1]), (int)(i / ((long long)L.Pn[0] * L.Pn[1]))};
    const bool on = probe_colour(g, L.dim, P, cx, cy, cz);
    if (add_from) {
      if (on) acc[i] += add_from[i];
    } else {
      q[i] = on ? 1.0 : 0.0;
    }
  }
}

// D_d[i] = sum_j B_ij^2 / D_A,jj: one B application per colour and velocity component on the
// probe D_A^-1/2 restricted to the colour; its squared entries add up to D_d.
static int schur_diag_d(stokes_ctx *C, int l, double *dS) {
  Runner<double> R(C);
  LevelRT<double> &LV = C->L64[l];
  const LevelDesc<double> &d = LV.d;
  const int P = 2 * d.k + 1, nz = d.dim == 3 ? P : 1;
  double *v = C->lz0, *y = C->lz1;
  SMF_CUDA_OK(cudaMemsetAsync(dS, 0, d.n_p * sizeof(double), C->s));
  for (int comp = 0; comp < d.dim; ++comp)
    for (int cz = 0; cz < nz; ++cz)
      for (int cy = 0; cy < P; ++cy)
        for (int cx = 0; cx < P; ++cx) {
          R.vec(k_probe_vel, d.n_u, d, comp, P, cx, cy, cz, (const double *)LV.DAinv, v);
          R.apply(l, kApplyB, v, nullptr, nullptr, y);
          R.vec(k_add_sq, d.n_p, (const double *)y, dS, d.n_p);
        }
  SMF_CUDA_OK(cudaGetLastError());
  return STOKES_OK;
}

// D_exact[i] = (B A^-1_hat B^T)_ii with A^-1_hat = sigma Cheb(A, D_A, k_A): one S~ application per
// pressure colour.  Meant for small meshes: more than 4096 colours are rejected.
static int schur_diag_exact(stokes_ctx *C, int l, double *dS) {
  Runner<double> R(C);
  const LevelDesc<double> &d = C->L64[l].d;
  const int P = (d.k - 1) * (C->o.kA + 3) + 1;
  const int px = std::min(P, d.Pn[0]), py = std::min(P, d.Pn[1]), pz = d.dim == 3 ? std::min(P, d.Pn[2]) : 1;
  if ((long long)px * py * pz > 4096) {
    set_error("schur_diag exact: " + std::to_string((long long)px * py * pz) +
              " probes needed (more than 4096); the exact diagonal is for small meshes");
    return STOKES_EINVAL;
  }
  double *q = C->lz0, *w = C->lz1;
  SMF_CUDA_OK(cudaMemsetAsync(dS, 0, d.n_p * sizeof(double), C->s));
  for (int cz = 0; cz < pz; ++cz)
    for (int cy = 0; cy < py; ++cy)
      for (int cx = 0; cx < px; ++cx) {
        R.vec(k_probe_pre, d.n_p, d, P, cx, cy, cz, q, (const double *)nullptr, (double *)nullptr);
        SMF_CUDA_OK(cudaMemsetAsync(w, 0, d.n_p * sizeof(double), C->s));
        R.S_tilde(l, q, w);
        R.vec(k_probe_pre, d.n_p, d, P, cx, cy, cz, (double *)nullptr, (const double *)w, dS);
      }
  SMF_CUDA_OK(cudaGetLastError());
  return STOKES_OK;
}

static int lanczos(stokes_ctx *C, int l, bool velocity, double *est) {
  Runner<double> R(C);
  LevelRT<double> &LV = C->L64[l];
  const long long n = velocity ? LV.d.n_u : LV.d.n_p;
  const int nb = vec_blocks(n);
  double *v = C->lz0, *vprev = C->lz1, *w = C->lz2, *tmp = C->lz3, *sq = C->sq;
  const double *Dg = velocity ? C->DA[l] : C->DS[l];
  k_rsqrt<double><<<nb, kVecThreads, 0, C->s>>>(Dg, sq, n);
  k_splitmix<<<nb, kVecThreads, 0, C->s>>>(C->o.seed + (velocity ? 0ull : 1ull), v, n);
  C->launches += 2;
  if (velocity) {
    k_zero_constrained<double><<<nb, kVecThreads, 0, C->s>>>(LV.d, v);
    ++C->launches;
  } else if (C->pker) {
    // z = sqrt(D_S) = 1 / sq
    k_reciprocal<double><<<nb, kVecThreads, 0, C->s>>>(sq, tmp, n);
    ++C->launches;
    double vz, zz;
    int st = dot64(C, v, tmp, n, &vz);
    if (st) return st;
    st = dot64(C, tmp, tmp, n, &zz);
    if (st) return st;
    k_axpy<double><<<nb, kVecThreads, 0, C->s>>>(v, -vz / zz, tmp, n);
    ++C->launches;
  }
  double nrm2;
  int st = dot64(C, v, v, n, &nrm2);
  if (st) return st;
  k_scale<double><<<nb, kVecThreads, 0, C->s>>>(v, 1.0 / std::sqrt(nrm2), v, n);
  SMF_CUDA_OK(cudaMemsetAsync(vprev, 0, n * sizeof(double), C->s));
  ++C->launches;
  std::vector<double> al, be;
  double bprev = 0.0;
  const int steps = std::max(1, C->o.eig_iters);
  for (int j = 0; j < steps; ++j) {
    k_mul<double><<<nb, kVecThreads, 0, C->s>>>(sq, v, tmp, n);
    ++C->launches;
    if (velocity) {
      R.apply(l, kApplyA, tmp, nullptr, w, nullptr);
    } else {
      SMF_CUDA_OK(cudaMemsetAsync(w, 0, n * sizeof(double), C->s));
      R.S_tilde(l, tmp, w);
    }
    k_mul<double><<<nb, kVecThreads, 0, C->s>>>(sq, w, w, n);
    k_axpy<double><<<nb, kVecThreads, 0, C->s>>>(w, -bprev, vprev, n);
    C->launches += 2;
    double a;
    st = dot64(C, w, v, n, &a);
    if (st) return st;
    k_axpy<double><<<nb, kVecThreads, 0, C->s>>>(w, -a, v, n);
    ++C->launches;
    al.push_back(a);
    double b2;
    st = dot64(C, w, w, n, &b2);
    if (st) return st;
    const double b = std::sqrt(b2);
    if (!std::isfinite(a) || !std::isfinite(b)) {
      set_error("Lanczos produced a non-finite value");
      return STOKES_EBREAKDOWN;
    }
    if (j == steps - 1 || b <= 1e-14 * std::max(std::fabs(a), 1.0)) break;
    be.push_back(b);
    std::swap(vprev, v);  // vprev <- v
    k_scale<double><<<nb, kVecThreads, 0, C->s>>>(w, 1.0 / b, v, n);
    ++C->launches;
    bprev = b;
  }
  be.resize(al.size() > 0 ? al.size() - 1 : 0);
  *est = tridiag_max_eig(al, be);
  return STOKES_OK;
}

// Dense coarse matrix K_0 by applying the FP64 operator to unit vectors, then the inverse of
// the (bordered) matrix by Gauss-Jordan with partial pivoting, all on the device.
static int setup_coarse(stokes_ctx *C) {
  Runner<double> R(C);
  LevelRT<double> &L0 = C->L64[0];
  const long long n0 = L0.d.n_u + L0.d.n_p;
  if (n0 > 20000) {
    set_error("coarse level has " + std::to_string(n0) + " DoFs; the dense direct solve allows at most 20000");
    return STOKES_EINVAL;
  }
  C->n0 = (int)n0;
  double *K0 = nullptr, *e = nullptr, *M = nullptr, *fac = nullptr;
  int *err = nullptr;
  int st;
  if ((st = dalloc(C, &K0, n0 * n0))) return st;
  if ((st = dalloc(C, &e, n0))) return st;
  const int bord = C->pker ? 1 : 0;
  const int nb = (int)n0 + bord;
  if ((st = dalloc(C, &M, (long long)nb * 2 * nb))) return st;
  if ((st = dalloc(C, &fac, nb))) return st;
  if ((st = dalloc(C, &err, 1))) return st;
  if ((st = dalloc(C, &C->Kinv, n0 * n0))) return st;
  for (long long j = 0; j < n0; ++j) {
    k_unit<<<vec_blocks(n0), kVecThreads, 0, C->s>>>(e, n0, j);
    ++C->launches;
    R.vmult(0, e, K0 + j * n0, true);
  }
  k_build_augmented<<<vec_blocks((long long)nb * 2 * nb), kVecThreads, 0, C->s>>>(K0, (int)n0, L0.d.n_u, bord, M);
  ++C->launches;
  for (int k = 0; k < nb; ++k) {
    k_gj_pivot<<<1, 1024, 0, C->s>>>(M, nb, k, fac, err);
    dim3 g((2 * nb + 255) / 256, nb);
    k_gj_elim<<<g, 256, 0, C->s>>>(M, nb, k, fac);
    C->launches += 2;
  }
  k_extract_inverse<<<vec_blocks(n0 * n0), kVecThreads, 0, C->s>>>(M, nb, (int)n0, C->Kinv);
  ++C->launches;
  int herr = 0;
  SMF_CUDA_OK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, C->s));
  SMF_CUDA_OK(cudaStreamSynchronize(C->s));
  if (herr) {
    set_error("coarse matrix is singular");
    return STOKES_EBREAKDOWN;
  }
  return STOKES_OK;
}

template <typename T>
static int alloc_level_buffers(stokes_ctx *C, LevelRT<T> &R) {
  const long long nu = R.d.n_u, np = R.d.n_p, n = nu + np;
  int st;
  T **full[] = {&R.x, &R.b, &R.r, &R.kx};
  for (auto p : full)
    if ((st = dalloc(C, p, n))) return st;
  T **vel[] = {&R.DAinv, &R.tu, &R.ru, &R.uhat, &R.cx, &R.cd, &R.ct, &R.r2, &R.cx2, &R.cd2, &R.ct2, &R.au};
  for (auto p : vel)
    if ((st = dalloc(C, p, nu))) return st;
  T **pre[] = {&R.DSinv, &R.pt, &R.rp, &R.px, &R.pd, &R.ps, &R.dp};
  for (auto p : pre)
    if ((st = dalloc(C, p, np))) return st;
  return STOKES_OK;
}

// 1D injection matrices of the level pair (fine F, coarse Cd) per space and axis with the
// Dirichlet masks folded in (a node constrained along an axis gets an empty row / column), as
// padded (node, weight) rows of width 4k + 1 (the support of a coarse vertex function: two coarse
// cells, four fine ones) for the transfer kernels.
template <typename T>
static int build_xfer(stokes_ctx *C, const LevelDesc<T> &F, const LevelDesc<T> &Cd, const TransferTab<double> &tt,
                      XferTabs<T> &X) {
  const int k = F.k, W = 4 * k + 1, dim = F.dim;
  X.W = W;
  for (int sp = 0; sp < 2; ++sp) {
    const int deg = sp == 0 ? k : k - 1;
    const double *tab = sp == 0 ? tt.vel : tt.pre;
    for (int a = 0; a < 3; ++a) {
      const int Nf = sp == 0 ? F.N[a] : F.Pn[a], Nc = sp == 0 ? Cd.N[a] : Cd.Pn[a];
      std::vector<std::vector<std::pair<int, double>>> rows(Nf), cols(Nc);
      if (a >= dim) {
        rows[0].push_back({0, 1.0});
        cols[0].push_back({0, 1.0});
      } else {
        const int nc = Cd.n[a];
        auto free_node = [&](int g, int N) {
          if (sp != 0) return true;
          if (((F.faces >> (2 * a)) & 1u) && g == 0) return false;
          if (((F.faces >> (2 * a + 1)) & 1u) && g == N - 1) return false;
          return true;
        };
        for (int g = 0; g < Nf; ++g) {
          if (!free_node(g, Nf)) continue;
          int f = g / deg;
          if (f > 2 * nc - 1) f = 2 * nc - 1;
          const int aa = g - deg * f, c = f >> 1, h = f & 1;
          for (int m = 0; m <= deg; ++m) {
            const int G = deg * c + m;
            const double w = tab[(h * (deg + 1) + aa) * (deg + 1) + m];
            if (w == 0.0 || !free_node(G, Nc)) continue;
            rows[g].push_back({G, w});
            cols[G].push_back({g, w});
          }
        }
      }
      for (int dir = 0; dir < 2; ++dir) {
        const auto &R = dir == 0 ? cols : rows;  // dir 0: restriction rows (per coarse node)
        const int n = (int)R.size();
        std::vector<int> cnt(n), idx((size_t)n * W, 0);
        std::vector<T> w((size_t)n * W, T(0));
        for (int r = 0; r < n; ++r) {
          if ((int)R[r].size() > W) {
            set_error("transfer table row wider than 4k+1");
            return STOKES_EINVAL;
          }
          cnt[r] = (int)R[r].size();
          for (size_t e = 0; e < R[r].size(); ++e) {
            idx[(size_t)r * W + e] = R[r][e].first;
            w[(size_t)r * W + e] = (T)R[r][e].second;
          }
        }
        int *dc, *di;
        T *dw;
        int st;
        if ((st = dalloc(C, &dc, n))) return st;
        if ((st = dalloc(C, &di, (long long)n * W))) return st;
        if ((st = dalloc(C, &dw, (long long)n * W))) return st;
        SMF_CUDA_OK(cudaMemcpyAsync(dc, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice, C->s));
        SMF_CUDA_OK(cudaMemcpyAsync(di, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, C->s));
        SMF_CUDA_OK(cudaMemcpyAsync(dw, w.data(), w.size() * sizeof(T), cudaMemcpyHostToDevice, C->s));
        SMF_CUDA_OK(cudaStreamSynchronize(C->s));  // host vectors go out of scope
        Xfer1D<T> &x = dir == 0 ? X.r[sp][a] : X.p[sp][a];
        x.cnt = dc;
        x.idx = di;
        x.w = dw;
      }
    }
  }
  return STOKES_OK;
}

// Zero every smoother work vector of a level (accumulation targets must start at zero; the
// unfused and fused smoothers leave different state vectors behind).
template <typename T>
static int zero_level_work(stokes_ctx *C, LevelRT<T> &R) {
  const long long nu = R.d.n_u, np = R.d.n_p;
  T *vel[] = {R.tu, R.ru, R.uhat, R.cx, R.cd, R.ct, R.r2, R.cx2, R.cd2, R.ct2, R.au};
  for (T *p : vel) SMF_CUDA_OK(cudaMemsetAsync(p, 0, (size_t)nu * sizeof(T), C->s));
  T *pre[] = {R.pt, R.rp, R.px, R.pd, R.ps, R.dp};
  for (T *p : pre) SMF_CUDA_OK(cudaMemsetAsync(p, 0, (size_t)np * sizeof(T), C->s));
  SMF_CUDA_OK(cudaMemsetAsync(R.kx, 0, (size_t)(nu + np) * sizeof(T), C->s));
  return STOKES_OK;
}

struct StreamGuard {
  stokes_ctx *C;
  cudaStream_t user;
  StreamGuard(stokes_ctx *c, void *u) : C(c), user((cudaStream_t)u) {
    cudaEventRecord(C->ev_in, user);
    cudaStreamWaitEvent(C->s, C->ev_in, 0);
  }
  ~StreamGuard() {
    cudaEventRecord(C->ev_out, C->s);
    cudaStreamWaitEvent(user, C->ev_out, 0);
  }
};

static int det_check(stokes_ctx *C, cudaStream_t s);
static int finish(stokes_ctx *C, int st) {
  if (st != STOKES_OK) {
    C->err = g_last_error;
    return st;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_fail(e, "kernel launch", __FILE__, __LINE__);
    C->err = g_last_error;
    return STOKES_ECUDA;
  }
  if ((st = det_check(C, C->s)) != STOKES_OK) C->err = g_last_error;
  return st;
}

// The setup's timings replay CUDA graphs of the candidate work, so that they compare the GPU's
// time for the work and not the host's launch rate (which a profiler attached to the process
// changes).
template <typename F>
static int capture_graph(stokes_ctx *C, F &&work, cudaGraphExec_t *exec) {
  SMF_CUDA_OK(cudaStreamBeginCapture(C->s, cudaStreamCaptureModeThreadLocal));
  C->capturing = true;
  C->cap_count = 0;
  work();
  C->capturing = false;
  cudaGraph_t g;
  SMF_CUDA_OK(cudaStreamEndCapture(C->s, &g));
  const cudaError_t e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  SMF_CUDA_OK(e);
  return STOKES_OK;
}
static int time_graph(stokes_ctx *C, cudaGraphExec_t ex, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  SMF_CUDA_OK(cudaEventRecord(e0, C->s));
  SMF_CUDA_OK(cudaGraphLaunch(ex, C->s));
  SMF_CUDA_OK(cudaEventRecord(e1, C->s));
  SMF_CUDA_OK(cudaEventSynchronize(e1));
  SMF_CUDA_OK(cudaEventElapsedTime(ms, e0, e1));
  return STOKES_OK;
}

// Autotuner of the 3D cell-kernel launch shape, per level and precision: the velocity-block
// apply is timed (graph replays, CUDA events on the context stream) for the column kernel with
// 1 and 4 warps per CTA, the column kernel with the velocity components split over 3 warps, the
// point-per-thread kernel and, where it serves the level, the cell-component kernel (shape 5).
// Candidates are interleaved over several rounds and each keeps its best round, so clock ramps
// and one-off effects do not bias the choice; the default shape (4 warps) is kept unless another
// is faster by more than 3 %.  The fastest column shape is also kept apart (fshape): the fused
// smoother's launches run in the column kernel.  Where an FP32 level has its per-point geometry
// stored (geo_stored), the column shapes are timed with the stored geometry as well, and the level
// reads it (geo) if the column shape kept for it is fastest that way.
template <typename T>
static int autotune_level(stokes_ctx *C, LevelRT<T> &R, const Tab1D<T> *tab) {
  if (R.d.dim != 3) return STOKES_OK;
  const bool cc = cc_level_supported(R.d.dim, R.d.k, R.d.cartesian, sizeof(T)) && !C->sym && !R.rho &&
                  (R.d.cartesian || sizeof(T) == 4 || R.geo);
  const bool sg = R.geo_stored && !R.geo;
  // candidates: column shapes 4, 1, 3 (on-the-fly geometry), point kernel, cell-component kernel,
  // then the column shapes reading the stored geometry
  constexpr int NMAX = 8;
  const int cands[NMAX] = {4, 1, 3, -1, 5, 4, 1, 3};
  const bool cgeo[NMAX] = {false, false, false, false, false, true, true, true};
  bool use[NMAX] = {true, true, true, true, cc, sg, sg, sg};
  const int reps = sizeof(T) == 8 ? 3 : 20, rounds = 3;
  cudaEvent_t e0, e1;
  SMF_CUDA_OK(cudaEventCreate(&e0));
  SMF_CUDA_OK(cudaEventCreate(&e1));
  cudaGraphExec_t ex[NMAX] = {};
  float best[NMAX];
  for (float &b : best) b = 1e30f;
  int st = STOKES_OK;
  const T *geo0 = R.geo;
  for (int ci = 0; ci < NMAX && st == STOKES_OK; ++ci) {
    if (!use[ci]) continue;
    R.shape = cands[ci];
    R.geo = cgeo[ci] ? R.geo_stored : geo0;
    st = capture_graph(
        C,
        [&] {
          for (int r = 0; r < reps; ++r)
            launch_cell_apply<T>(R.d, tab, C->sym ? kApplyA | kApplySym : kApplyA, R.x, nullptr, R.r, nullptr, C->s,
                                 R.shape, R.geo, R.rho);
        },
        &ex[ci]);
  }
  R.geo = geo0;
  for (int round = -1; round < rounds && st == STOKES_OK; ++round)  // round -1: warm-up
    for (int ci = 0; ci < NMAX && st == STOKES_OK; ++ci) {
      if (!use[ci]) continue;
      float ms = 0.f;
      st = time_graph(C, ex[ci], e0, e1, &ms);
      if (round >= 0) best[ci] = std::min(best[ci], ms);
      C->launches += reps;
    }
  for (auto e : ex)
    if (e) cudaGraphExecDestroy(e);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != STOKES_OK) return st;
  int choice = 0;
  for (int ci = 1; ci < NMAX; ++ci)
    if (use[ci] && best[ci] < 0.97f * best[choice]) choice = ci;
  R.shape = cands[choice];
  int fc = 0;  // column shapes only: 4, 1, 3, each with the stored geometry where timed
  for (int ci = 1; ci < NMAX; ++ci)
    if (use[ci] && (cands[ci] == 1 || cands[ci] == 3 || cands[ci] == 4) && best[ci] < 0.97f * best[fc]) fc = ci;
  if (cands[choice] == 1 || cands[choice] == 3 || cands[choice] == 4) fc = choice;
  R.fshape = cands[fc];
  R.geo = cgeo[fc] ? R.geo_stored : geo0;
  SMF_CUDA_OK(cudaMemsetAsync(R.r, 0, (R.d.n_u + R.d.n_p) * sizeof(T), C->s));
  return STOKES_OK;
}

// Fused or unfused smoothing per level: where the fused smoother is eligible, smoothing steps of
// each kind are timed (graph replays, CUDA events on the context stream, interleaved rounds, best
// round kept) on the level's own buffers; the fused form is kept unless the unfused one is faster by more
// than 3 %.  The fused form saves launches and vector passes but makes every cell-kernel gather
// read several vectors, which costs more than it saves on the largest levels.
template <typename T>
static int autotune_fusion(stokes_ctx *C, int l) {
  Runner<T> R(C);
  LevelRT<T> &L = R.L[l];
  if (!R.fused_eligible(l)) return STOKES_OK;
  const int reps = sizeof(T) == 8 ? 1 : 4, rounds = sizeof(T) == 8 ? 2 : 3;
  cudaEvent_t e0, e1;
  SMF_CUDA_OK(cudaEventCreate(&e0));
  SMF_CUDA_OK(cudaEventCreate(&e1));
  cudaGraphExec_t ex[2] = {};
  float best[2] = {1e30f, 1e30f};
  int st = STOKES_OK;
  for (int f = 0; f < 2 && st == STOKES_OK; ++f) {
    L.fuse = f == 1;
    st = capture_graph(
        C,
        [&] {
          for (int r = 0; r < reps; ++r) R.smooth(l, L.x, L.b, 1, false);
        },
        &ex[f]);
  }
  for (int round = -1; round < rounds && st == STOKES_OK; ++round)  // round -1: warm-up
    for (int f = 0; f < 2 && st == STOKES_OK; ++f) {
      float ms = 0.f;
      st = time_graph(C, ex[f], e0, e1, &ms);
      if (round >= 0) best[f] = std::min(best[f], ms);
    }
  for (auto e : ex)
    if (e) cudaGraphExecDestroy(e);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != STOKES_OK) return st;
  L.fuse = !(best[0] < 0.97f * best[1]);
  SMF_CUDA_OK(cudaMemsetAsync(L.x, 0, (L.d.n_u + L.d.n_p) * sizeof(T), C->s));
  return zero_level_work(C, L);
}

// STOKES_TUNING="s32=a,b,..;s64=..;f32=..;f64=..[;g32=..]" replaces the setup's timings: launch
// shapes (1, 3, 4, -1 or 5) and smoother forms (1 fused, 0 unfused) per level, coarsest first, for
// FP32 and FP64, and optionally whether the FP32 column kernels read the stored per-point geometry
// (1) or evaluate it (0, the default).  Timings taken under a profiler differ from plain runs; a
// profile of the configuration that a plain run chose passes that run's choices here
// (stokes_get_launch_shape, stokes_get_smoother_fusion and stokes_get_geometry_stored read them).
static int parse_tuning(const char *spec, int nl, std::vector<int> tune[5]) {
  const char *keys[5] = {"s32=", "s64=", "f32=", "f64=", "g32="};
  for (int t = 0; t < 5; ++t) {
    const char *p = std::strstr(spec, keys[t]);
    if (!p && t == 4) {
      tune[t].assign(nl, 0);
      continue;
    }
    if (!p) {
      set_error(std::string("STOKES_TUNING lacks ") + keys[t]);
      return STOKES_EINVAL;
    }
    p += 4;
    tune[t].clear();
    while (true) {
      char *end = nullptr;
      const long v = std::strtol(p, &end, 10);
      if (end == p) break;
      const bool ok = t < 2 ? (v == 1 || v == 3 || v == 4 || v == -1 || v == 5) : (v == 0 || v == 1);
      if (!ok) {
        set_error(std::string("STOKES_TUNING: invalid value in ") + keys[t]);
        return STOKES_EINVAL;
      }
      tune[t].push_back((int)v);
      p = end;
      if (*p != ',') break;
      ++p;
    }
    if ((int)tune[t].size() != nl) {
      set_error(std::string("STOKES_TUNING: ") + keys[t] + " needs one value per level");
      return STOKES_EINVAL;
    }
  }
  return STOKES_OK;
}

// Cell values of the next coarser level (n cells per direction): the mean of the 2^d children.
static std::vector<double> coarsen_mean(const std::vector<double> &fm, const int n[3], int dim) {
  std::vector<double> cm((size_t)n[0] * n[1] * n[2], 0.0);
  const int fx = 2 * n[0], fy = 2 * n[1];
  for (int cz = 0; cz < n[2]; ++cz)
    for (int cy = 0; cy < n[1]; ++cy)
      for (int cx = 0; cx < n[0]; ++cx) {
        double sum = 0.0;
        for (int dz = 0; dz < (dim == 3 ? 2 : 1); ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) sum += fm[((size_t)(2 * cz + dz) * fy + (2 * cy + dy)) * fx + (2 * cx + dx)];
        cm[((size_t)cz * n[1] + cy) * n[0] + cx] = sum / (dim == 3 ? 8.0 : 4.0);
      }
  return cm;
}

static int do_setup(const stokes_mesh *mesh, int k, double mu, double gamma_rho, const double *mu_cell,
                    const stokes_opts *opts, stokes_ctx *C) {
  const int dim = mesh->dim, nl = mesh->n_levels;
  C->mesh = *mesh;
  if (mesh->vertices) {
    const long long nvert = (long long)(mesh->n[0] + 1) * (mesh->n[1] + 1) * (dim == 3 ? mesh->n[2] + 1 : 1);
    C->mesh_vertices.assign(mesh->vertices, mesh->vertices + nvert * dim);
    C->mesh.vertices = C->mesh_vertices.data();
  }
  C->mu_const = mu;
  C->dim = dim;
  C->k = k;
  C->nl = nl;
  C->mu = mu;
  C->gamma_rho = gamma_rho;
  if (opts)
    C->o = *opts;
  else
    stokes_default_opts(&C->o);
  if (C->o.kA < 0 || C->o.kA > 16 || C->o.kS < 0 || C->o.kS > 16 || C->o.m < 0 || C->o.gmres_restart < 1 ||
      C->o.schur_diag < 0 || C->o.schur_diag > 3 || C->o.cycle < 0 || C->o.cycle > 1) {
    set_error("invalid stokes_opts (kA, kS in [0,16], m >= 0, restart >= 1, schur_diag in {0,1,2,3}, cycle in {0,1})");
    return STOKES_EINVAL;
  }
  if (!(C->o.c_mass >= 0) || !(C->o.c_grad >= 0) || !std::isfinite(C->o.c_mass) || !std::isfinite(C->o.c_grad)) {
    set_error("invalid stokes_opts: c_mass and c_grad must be finite and >= 0");
    return STOKES_EINVAL;
  }
  C->c_mass = C->o.c_mass;
  C->c_grad = C->o.c_grad;
  C->sym = C->o.sym_grad != 0;
  C->det = C->o.deterministic != 0;
  if (C->o.deterministic < 0 || C->o.deterministic > 2) {
    set_error("opts.deterministic must be 0, 1 (owner-computes) or 2 (colour classes)");
    return STOKES_EINVAL;
  }
  if (C->det && (dim != 3 || (k != 2 && k != 3) || (k == 3 && mesh->vertices) || C->sym || C->o.rho_cell ||
                 C->c_mass != 0.0 || C->c_grad != 0.0)) {
    set_error("deterministic mode needs 3D, k = 2 (any mesh) or k = 3 (Cartesian), the Laplacian form with a "
              "constant rho and C = 0");
    return STOKES_EINVAL;
  }
  if (C->o.rho_cell) {
    const long long nc = (long long)mesh->n[0] * mesh->n[1] * (dim == 3 ? mesh->n[2] : 1);
    C->rho_host.assign(C->o.rho_cell, C->o.rho_cell + nc);
    for (double v : C->rho_host)
      if (!(v > 0) || !std::isfinite(v)) {
        set_error("rho_cell entries must be positive");
        return STOKES_EINVAL;
      }
    C->o.rho_cell = C->rho_host.data();
  }
  const unsigned full = dim == 3 ? 0x3Fu : 0xFu;
  const unsigned faces = mesh->dirichlet_faces & full;
  // constant pressures span the kernel of K under full Dirichlet data, unless C has a mass part
  C->pker = faces == full && C->c_mass == 0.0;
  const char *env = getenv("STOKES_NO_GRAPHS");
  C->use_graphs = !(env && env[0] == '1');
  const char *nofuse = getenv("STOKES_NO_FUSE");
  C->fuse = !(nofuse && nofuse[0] == '1');
  C->restart = C->o.gmres_restart;
  int st;
  SMF_CUDA_OK(cudaStreamCreateWithFlags(&C->s, cudaStreamNonBlocking));
  SMF_CUDA_OK(cudaEventCreateWithFlags(&C->ev_in, cudaEventDisableTiming));
  SMF_CUDA_OK(cudaEventCreateWithFlags(&C->ev_out, cudaEventDisableTiming));

  // tables
  Tab1D<double> t64;
  build_tables(k, t64);
  Tab1D<float> t32;
  {
    const double *src = reinterpret_cast<const double *>(&t64);
    float *dst = reinterpret_cast<float *>(&t32);
    for (size_t i = 0; i < sizeof(t64) / sizeof(double); ++i) dst[i] = (float)src[i];
  }
  TransferTab<double> tt64;
  build_transfer(k, tt64);
  if ((st = dalloc(C, &C->tab64, 1))) return st;
  if ((st = dalloc(C, &C->tab32, 1))) return st;
  SMF_CUDA_OK(cudaMemcpyAsync(C->tab64, &t64, sizeof(t64), cudaMemcpyHostToDevice, C->s));
  SMF_CUDA_OK(cudaMemcpyAsync(C->tab32, &t32, sizeof(t32), cudaMemcpyHostToDevice, C->s));
  {
    const int e = k == 2 ? upload_col_tables<2>(t64, C->s) : (k == 3 ? upload_col_tables<3>(t64, C->s)
                                                                     : upload_col_tables<4>(t64, C->s));
    if (e) SMF_CUDA_OK((cudaError_t)e);
    const int e2 = k == 2 ? upload_cc_tables<2>(t64, C->s) : (k == 3 ? upload_cc_tables<3>(t64, C->s) : 0);
    if (e2) SMF_CUDA_OK((cudaError_t)e2);
  }

  // level hierarchy (host copies of geometry and viscosity, coarse from fine)
  C->L64.resize(nl);
  C->L32.resize(nl);
  C->DA.resize(nl, nullptr);
  C->DS.resize(nl, nullptr);
  C->betaA.assign(nl, 0.0);
  C->betaS.assign(nl, 0.0);
  const int nf[3] = {mesh->n[0], mesh->n[1], dim == 3 ? mesh->n[2] : 1};
  std::vector<double> mu_fine;
  if (mu_cell) mu_fine.assign(mu_cell, mu_cell + (long long)nf[0] * nf[1] * nf[2]);
  std::vector<std::vector<double>> mu_levels(nl), rho_levels(nl);
  for (int l = nl - 1; l >= 0; --l) {
    const int s = 1 << (nl - 1 - l);
    int n[3] = {nf[0] / s, nf[1] / s, dim == 3 ? nf[2] / s : 1};
    if (!C->rho_host.empty())  // per-cell rho: coarse values are the mean of the 2^d children
      rho_levels[l] = l == nl - 1 ? C->rho_host : coarsen_mean(rho_levels[l + 1], n, dim);
    if (mu_cell) {
      if (l < nl - 1) {  // mean of the 2^d children (fine level l+1 has 2n cells per direction)
        std::vector<double> &fm = mu_levels[l + 1];
        std::vector<double> cm((size_t)n[0] * n[1] * n[2], 0.0);
        const int fx = 2 * n[0], fy = 2 * n[1];
        for (int cz = 0; cz < n[2]; ++cz)
          for (int cy = 0; cy < n[1]; ++cy)
            for (int cx = 0; cx < n[0]; ++cx) {
              double sum = 0.0;
              for (int dz = 0; dz < (dim == 3 ? 2 : 1); ++dz)
                for (int dy = 0; dy < 2; ++dy)
                  for (int dx = 0; dx < 2; ++dx)
                    sum += fm[((size_t)(2 * cz + dz) * fy + (2 * cy + dy)) * fx + (2 * cx + dx)];
              cm[((size_t)cz * n[1] + cy) * n[0] + cx] = sum / (dim == 3 ? 8.0 : 4.0);
            }
        mu_levels[l] = cm;
      } else {
        mu_levels[l] = mu_fine;
      }
    }
    LevelDesc<double> d{};
    double *geo_l = nullptr;
    d.dim = dim;
    d.k = k;
    for (int a = 0; a < 3; ++a) {
      d.n[a] = n[a];
      d.N[a] = a < dim ? k * n[a] + 1 : 1;
      d.Pn[a] = a < dim ? (k - 1) * n[a] + 1 : 1;
    }
    d.nv = (long long)d.N[0] * d.N[1] * d.N[2];
    d.n_u = dim * d.nv;
    d.n_p = (long long)d.Pn[0] * d.Pn[1] * d.Pn[2];
    d.n_cells = (long long)n[0] * n[1] * n[2];
    d.faces = faces;
    d.cartesian = mesh->vertices ? 0 : 1;
    for (int a = 0; a < 3; ++a) d.h[a] = a < dim ? (mesh->hi[a] - mesh->lo[a]) / n[a] : 1.0;
    d.mu = mu;
    d.gamma_rho = gamma_rho;
    LevelDesc<float> f{};
    f.dim = d.dim;
    f.k = d.k;
    for (int a = 0; a < 3; ++a) {
      f.n[a] = d.n[a];
      f.N[a] = d.N[a];
      f.Pn[a] = d.Pn[a];
      f.h[a] = (float)d.h[a];
    }
    f.nv = d.nv;
    f.n_u = d.n_u;
    f.n_p = d.n_p;
    f.n_cells = d.n_cells;
    f.faces = d.faces;
    f.cartesian = d.cartesian;
    f.mu = (float)mu;
    f.gamma_rho = (float)gamma_rho;
    if (mesh->vertices) {
      const long long nvert = (long long)(n[0] + 1) * (n[1] + 1) * (dim == 3 ? n[2] + 1 : 1);
      std::vector<double> hv((size_t)nvert * dim);
      std::vector<float> hf((size_t)nvert * dim);
      for (int vz = 0; vz < (dim == 3 ? n[2] + 1 : 1); ++vz)
        for (int vy = 0; vy <= n[1]; ++vy)
          for (int vx = 0; vx <= n[0]; ++vx) {
            const long long fi = ((long long)(vz * s) * (nf[1] + 1) + vy * s) * (nf[0] + 1) + vx * s;
            const long long ci = ((long long)vz * (n[1] + 1) + vy) * (n[0] + 1) + vx;
            for (int a = 0; a < dim; ++a) {
              hv[ci * dim + a] = mesh->vertices[fi * dim + a];
              hf[ci * dim + a] = (float)hv[ci * dim + a];
            }
          }
      double *dv;
      float *fv;
      if ((st = dalloc(C, &dv, nvert * dim))) return st;
      if ((st = dalloc(C, &fv, nvert * dim))) return st;
      SMF_CUDA_OK(cudaMemcpyAsync(dv, hv.data(), hv.size() * sizeof(double), cudaMemcpyHostToDevice, C->s));
      SMF_CUDA_OK(cudaMemcpyAsync(fv, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice, C->s));
      SMF_CUDA_OK(cudaStreamSynchronize(C->s));
      d.vert = dv;
      f.vert = fv;
    }
    if (mu_cell) {
      std::vector<double> &m = mu_levels[l];
      std::vector<float> mf(m.begin(), m.end());
      double *dm;
      float *fm;
      if ((st = dalloc(C, &dm, (long long)m.size()))) return st;
      if ((st = dalloc(C, &fm, (long long)m.size()))) return st;
      SMF_CUDA_OK(cudaMemcpyAsync(dm, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice, C->s));
      SMF_CUDA_OK(cudaMemcpyAsync(fm, mf.data(), mf.size() * sizeof(float), cudaMemcpyHostToDevice, C->s));
      SMF_CUDA_OK(cudaStreamSynchronize(C->s));
      d.mu_cell = dm;
      f.mu_cell = fm;
    }
    if (!rho_levels[l].empty()) {
      std::vector<double> &m = rho_levels[l];
      std::vector<float> mf(m.begin(), m.end());
      double *dr;
      float *fr;
      if ((st = dalloc(C, &dr, (long long)m.size()))) return st;
      if ((st = dalloc(C, &fr, (long long)m.size()))) return st;
      SMF_CUDA_OK(cudaMemcpyAsync(dr, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice, C->s));
      SMF_CUDA_OK(cudaMemcpyAsync(fr, mf.data(), mf.size() * sizeof(float), cudaMemcpyHostToDevice, C->s));
      SMF_CUDA_OK(cudaStreamSynchronize(C->s));
      C->L64[l].rho = dr;
      C->L32[l].rho = fr;
    }
    // per-point geometry of the FP64 column kernel (mu and gamma rho folded in), precomputed once
    // (the geometry is a quarter of the FP64 flops of an application; STOKES_GEO=none keeps it on
    // the fly); after the level's viscosity is in place
    if (mesh->vertices && dim == 3) {
      const char *gs = getenv("STOKES_GEO");
      const bool g64 = !(gs && std::strcmp(gs, "none") == 0);
      const long long per = 16LL * (k + 1) * (k + 1) * (k + 1), cells = d.n_cells;
      // stored when it takes at most 1/16 of the device's memory (17.8 GB on a GB300; 7.2 GB for
      // a trilinear 128^3 level), a fixed budget so that the choice does not depend on what other
      // processes hold; skipped only when it would take more than half of the memory still free
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = total_b = 0;
      const long long gbytes = cells * per * (long long)sizeof(double);
      if (g64 && gbytes <= (long long)(total_b / 16) && gbytes <= (long long)(free_b / 2)) {
        if ((st = dalloc(C, &geo_l, cells * per))) return st;
        launch_col_geometry<double>(d, geo_l, C->s);
        SMF_CUDA_OK(cudaGetLastError());
      }
      // FP32 levels of at most 32^3 cells (56.6 MB for k = 2): stored as a candidate that the
      // setup's timing keeps or drops per level.  On the small levels a launch is a dependency
      // chain (vertex loads, Jacobian, adjugate and its division, then the contractions); stored
      // factors are loaded together with the DoF values instead.
      if (g64 && cells <= 32768) {
        float *gf = nullptr;
        if ((st = dalloc(C, &gf, cells * per))) return st;
        launch_col_geometry<float>(f, gf, C->s);
        SMF_CUDA_OK(cudaGetLastError());
        C->L32[l].geo_stored = gf;
      }
    }
    C->L64[l].d = d;
    C->L32[l].d = f;
    C->L64[l].geo = geo_l;
    if ((st = alloc_level_buffers(C, C->L64[l]))) return st;
    if ((st = alloc_level_buffers(C, C->L32[l]))) return st;
  }

  // element matrices of C where the pressure space is small (at most 27 nodes per cell: packed
  // 378 entries per cell), built in FP64 and rounded for the FP32 levels; larger pressure spaces
  // and STOKES_C_MATRIX=none keep C on the fly
  {
    const int npp = dim == 3 ? k * k * k : k * k;  // Q_{k-1}: k pressure nodes per direction
    const char *cs = getenv("STOKES_C_MATRIX");
    if ((C->c_mass != 0.0 || C->c_grad != 0.0) && npp <= kMaxCMatrixNodes && !(cs && std::strcmp(cs, "none") == 0)) {
      for (int l = 0; l < nl; ++l) {
        const LevelDesc<double> &d = C->L64[l].d;
        const long long ne = d.n_cells * (long long)(npp * (npp + 1) / 2);
        double *c64;
        float *c32;
        if ((st = dalloc(C, &c64, ne))) return st;
        if ((st = dalloc(C, &c32, ne))) return st;
        launch_cell_C_matrix(d, C->tab64, C->c_mass, C->c_grad, c64, C->s);
        k_convert<double, float><<<vec_blocks(ne), kVecThreads, 0, C->s>>>(c64, c32, ne);
        SMF_CUDA_OK(cudaGetLastError());
        C->L64[l].Ce = c64;
        C->L32[l].Ce = c32;
      }
    }
  }

  // transfer matrices between consecutive levels
  for (int l = 1; l < nl; ++l) {
    if ((st = build_xfer(C, C->L64[l].d, C->L64[l - 1].d, tt64, C->L64[l].xf))) return st;
    if ((st = build_xfer(C, C->L32[l].d, C->L32[l - 1].d, tt64, C->L32[l].xf))) return st;
  }

  // deterministic mode: grid-barrier state, the cell-component kernel on every level
  if (C->det) {
    for (int l = 0; l < nl; ++l)
      if (!C->L64[l].d.cartesian && !C->L64[l].geo) {
        set_error("deterministic mode: level " + std::to_string(l) +
                  " is too large to keep its FP64 per-point geometry stored (1/16 of the device memory)");
        return STOKES_EINVAL;
      }
    if ((st = dalloc(C, &C->gb.state, 4))) return st;
    if (C->o.deterministic == 1) {
      // owner-computes form: per-cell local results of the largest level, both precisions
      long long cells = 0;
      for (int l = 0; l < nl; ++l) cells = std::max(cells, C->L64[l].d.n_cells);
      const long long per = 3LL * ((k + 1) * (k + 1) * (k + 1) + k * k * k);
      float *l32 = nullptr;
      double *l64 = nullptr;
      if ((st = dalloc(C, &l32, per * cells))) return st;
      if ((st = dalloc(C, &l64, per * cells))) return st;
      C->gb.owner = 1;
      C->gb.loc32 = l32;
      C->gb.loc64 = l64;
    }
    // setup runs with the default budget; opts.wait_cycles applies from the end of setup on
    const unsigned hs[4] = {0u, 0u, 0u, 0u};
    SMF_CUDA_OK(cudaMemcpyAsync(C->gb.state, hs, sizeof(hs), cudaMemcpyHostToDevice, C->s));
    for (int l = 0; l < nl; ++l) {
      C->L32[l].shape = C->L64[l].shape = 5;
      C->L32[l].fuse = C->L64[l].fuse = false;
    }
  }

  // launch-shape autotuning (STOKES_NO_AUTOTUNE=1 keeps the default shape; STOKES_TUNING fixes
  // shapes and smoother forms instead, see parse_tuning)
  std::vector<int> tune[5];
  const bool pinned = getenv("STOKES_TUNING") != nullptr && !C->det;
  if (pinned && (st = parse_tuning(getenv("STOKES_TUNING"), nl, tune))) return st;
  if (pinned) {
    for (int l = 0; l < nl; ++l) {
      if (dim == 3) {
        C->L32[l].shape = tune[0][l];
        C->L64[l].shape = tune[1][l];
        if (tune[4][l] && !C->L32[l].geo_stored) {
          set_error("STOKES_TUNING: g32 asks for stored FP32 geometry on level " + std::to_string(l) +
                    ", which has none (3D trilinear levels of at most 32^3 cells)");
          return STOKES_EINVAL;
        }
        C->L32[l].geo = tune[4][l] ? C->L32[l].geo_stored : nullptr;
      }
    }
  }
  {
    const char *na = getenv("STOKES_NO_AUTOTUNE");
    if (!(na && na[0] == '1') && !pinned && !C->det) {
      for (int l = 0; l < nl; ++l) {
        if ((st = autotune_level<double>(C, C->L64[l], C->tab64))) return st;
        if ((st = autotune_level<float>(C, C->L32[l], C->tab32))) return st;
      }
    }
  }
  // stored FP32 geometry that the timing (or the pinned tuning) did not keep is released
  for (int l = 0; l < nl; ++l) {
    LevelRT<float> &R = C->L32[l];
    if (R.geo_stored && !R.geo) {
      void *g = const_cast<float *>(R.geo_stored);
      C->allocs.erase(std::remove(C->allocs.begin(), C->allocs.end(), g), C->allocs.end());
      SMF_CUDA_OK(cudaFree(g));
      R.geo_stored = nullptr;
    }
  }

  // Krylov / Lanczos work space
  const LevelDesc<double> &top = C->L64[nl - 1].d;
  const long long N = top.n_u + top.n_p;
  if ((st = dalloc(C, &C->V, (long long)(C->restart + 1) * N))) return st;
  if ((st = dalloc(C, &C->Z, (long long)C->restart * N))) return st;
  if ((st = dalloc(C, &C->w, N))) return st;
  if ((st = dalloc(C, &C->hdev, 3 * (C->restart + 2)))) return st;
  if ((st = dalloc(C, &C->partial, (long long)kRedBlocks * (C->restart + 2)))) return st;
  if ((st = dalloc(C, &C->scal, 4))) return st;
  double **lz[] = {&C->lz0, &C->lz1, &C->lz2, &C->lz3, &C->sq};
  for (auto p : lz)
    if ((st = dalloc(C, p, N))) return st;
  {
    const int m = C->restart;
    KrylovDev &K = C->kd;
    K.m = m;
    if ((st = dalloc(C, &K.H, (long long)(m + 1) * m))) return st;
    if ((st = dalloc(C, &K.cs, m))) return st;
    if ((st = dalloc(C, &K.sn, m))) return st;
    if ((st = dalloc(C, &K.g, m + 1))) return st;
    if ((st = dalloc(C, &K.y, m))) return st;
    if ((st = dalloc(C, &K.thresh, 1))) return st;
    if ((st = dalloc(C, &K.ctl, 4))) return st;
    if ((st = dalloc(C, &K.ticket, 1))) return st;
    K.hcol = C->hdev;
    if ((st = dalloc(C, &C->zcur, N))) return st;
  }

  // smoother setup per level (Algorithm 2), FP64
  C->sigma = lemma1_scaling(C->o.kA);
  C->tau = lemma1_scaling(C->o.kS);
  for (int l = 1; l < nl; ++l) {
    LevelRT<double> &R = C->L64[l];
    const LevelDesc<double> &d = R.d;
    double *dAs, *dSloc, *dMp;
    if ((st = dalloc(C, &dAs, C->sym ? d.n_u : d.nv))) return st;
    if ((st = dalloc(C, &dSloc, d.n_p))) return st;
    if ((st = dalloc(C, &dMp, d.n_p))) return st;
    if ((st = dalloc(C, &C->DA[l], d.n_u))) return st;
    launch_cell_diag<double>(d, C->tab64, dAs, dSloc, dMp, C->s, R.rho, C->sym ? 1 : 0);
    ++C->launches;
    k_expand_diag<double><<<vec_blocks(d.n_u), kVecThreads, 0, C->s>>>(d, dAs, C->DA[l], C->sym ? 1 : 0);
    k_reciprocal<double><<<vec_blocks(d.n_u), kVecThreads, 0, C->s>>>(C->DA[l], R.DAinv, d.n_u);
    C->launches += 2;
    double est;
    if ((st = lanczos(C, l, true, &est))) return st;
    C->betaA[l] = C->o.eig_safety * est;
    switch (C->o.schur_diag) {
      case 0: C->DS[l] = dSloc; break;
      case 1: C->DS[l] = dMp; break;
      default: {  // 2: d = diag(B D_A^-1 B^T), 3: exact = diag(B A^-1_hat B^T), both by probing
        double *dS;
        if ((st = dalloc(C, &dS, d.n_p))) return st;
        if ((st = C->o.schur_diag == 2 ? schur_diag_d(C, l, dS) : schur_diag_exact(C, l, dS))) return st;
        C->DS[l] = dS;
      }
    }
    if (C->o.schur_diag != 3 && (C->c_mass != 0.0 || C->c_grad != 0.0)) {  // D_S~ += diag(C)
      launch_cell_C<double>(d, C->tab64, C->c_mass, C->c_grad, nullptr, nullptr, 1.0, C->DS[l], nullptr, C->s);
      ++C->launches;
    }
    k_reciprocal<double><<<vec_blocks(d.n_p), kVecThreads, 0, C->s>>>(C->DS[l], R.DSinv, d.n_p);
    ++C->launches;
    if ((st = lanczos(C, l, false, &est))) return st;
    C->betaS[l] = C->o.eig_safety * est;
    LevelRT<float> &F = C->L32[l];
    k_convert<double, float><<<vec_blocks(d.n_u), kVecThreads, 0, C->s>>>(R.DAinv, F.DAinv, d.n_u);
    k_convert<double, float><<<vec_blocks(d.n_p), kVecThreads, 0, C->s>>>(R.DSinv, F.DSinv, d.n_p);
    C->launches += 2;
  }
  if ((st = setup_coarse(C))) return st;
  for (int l = 0; l < nl; ++l) {
    if ((st = zero_level_work(C, C->L64[l]))) return st;
    if ((st = zero_level_work(C, C->L32[l]))) return st;
  }
  // fused or unfused smoothing per level (STOKES_NO_AUTOTUNE=1 keeps the fused form)
  {
    const char *na = getenv("STOKES_NO_AUTOTUNE");
    if (pinned) {
      for (int l = 0; l < nl; ++l) {
        C->L32[l].fuse = tune[2][l] != 0;
        C->L64[l].fuse = tune[3][l] != 0;
      }
    } else if (!(na && na[0] == '1') && !C->det) {
      for (int l = 1; l < nl; ++l) {
        if ((st = autotune_fusion<float>(C, l))) return st;
        if ((st = autotune_fusion<double>(C, l))) return st;
      }
    }
  }
  SMF_CUDA_OK(cudaStreamSynchronize(C->s));
  SMF_CUDA_OK(cudaGetLastError());
  if (C->det) {
    if ((st = det_check(C, C->s))) return st;
    SMF_CUDA_OK(cudaMemcpyAsync(C->gb.state + 3, &C->o.wait_cycles, sizeof(unsigned), cudaMemcpyHostToDevice, C->s));
    SMF_CUDA_OK(cudaStreamSynchronize(C->s));
  }
  return STOKES_OK;
}

static bool check_level(stokes_ctx *C, int level) {
  if (!C || level < 0 || level >= C->nl) {
    set_error("level out of range");
    if (C) C->err = g_last_error;
    return false;
  }
  return true;
}

// FP64 flexible GMRES (restarted), right-preconditioned by one multigrid cycle per iteration.
// Deterministic mode: clear the grid-barrier state (arrivals, round, error flag) on stream s before
// a call's launches; after them, synchronise and report a wait that ran out as STOKES_ETIMEOUT.
static int det_begin(stokes_ctx *C, cudaStream_t s) {
  if (C->det) SMF_CUDA_OK(cudaMemsetAsync(C->gb.state, 0, 3 * sizeof(unsigned), s));
  return STOKES_OK;
}
static int det_check(stokes_ctx *C, cudaStream_t s) {
  if (!C->det) return STOKES_OK;
  unsigned err = 0;
  SMF_CUDA_OK(cudaMemcpyAsync(&err, C->gb.state + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  SMF_CUDA_OK(cudaStreamSynchronize(s));
  if (err) {
    // reported once: the state is cleared for the calls that follow
    SMF_CUDA_OK(cudaMemsetAsync(C->gb.state, 0, 3 * sizeof(unsigned), s));
    SMF_CUDA_OK(cudaStreamSynchronize(s));
    set_error("a grid-barrier wait of the deterministic cell kernel ran out of its budget (opts.wait_cycles); "
              "results of this call are invalid");
    return STOKES_ETIMEOUT;
  }
  return STOKES_OK;
}

// Destroys every captured graph of the context (cycles and the device Krylov loop).
static void drop_graphs(stokes_ctx *C) {
  for (int i = 0; i < 2; ++i) {
    if (C->g32[i].exec) cudaGraphExecDestroy(C->g32[i].exec);
    if (C->g64[i].exec) cudaGraphExecDestroy(C->g64[i].exec);
    C->g32[i].exec = nullptr;
    C->g64[i].exec = nullptr;
  }
  if (C->kry) cudaGraphExecDestroy(C->kry);
  C->kry = nullptr;
  if (C->kry_mode == 1) C->kry_mode = -1;
}

// The inner FGMRES iteration on the device (one Arnoldi step, Sec. 4 outer loop around the
// multigrid preconditioner of Algorithm 1): z_j = MG(0, v_j) into zcur and Z_j, w = K z_j (FP64),
// CGS2 against v_0..v_j, v_{j+1} = w / ||w||, then the Givens update that sets `cond`.
// Split at the FP32 cycle for the batched work-queue form: krylov_pre converts v_j into the
// cycle's right-hand side (and zeroes x), krylov_post takes the cycle's result from there on.
static void krylov_pre(stokes_ctx *C) {
  Runner<float> R32(C);
  const int top = C->nl - 1;
  const long long N = C->L64[top].d.n_u + C->L64[top].d.n_p;
  LevelRT<float> &T32 = C->L32[top];
  R32.vec(k_slot_convert<float>, N, (const double *)C->V, N, (const int *)C->kd.ctl, T32.b, T32.x, N);
}
static void krylov_post(stokes_ctx *C, cudaGraphConditionalHandle cond, bool set_cond, bool from_fp32);
static void krylov_body(stokes_ctx *C, cudaGraphConditionalHandle cond, bool set_cond) {
  Runner<double> R64(C);
  Runner<float> R32(C);
  const int top = C->nl - 1;
  const long long N = C->L64[top].d.n_u + C->L64[top].d.n_p;
  const int *ctl = C->kd.ctl;
  if (C->o.vcycle_fp32) {
    LevelRT<float> &T32 = C->L32[top];
    krylov_pre(C);
    R32.cycle(top, T32.x, T32.b, true);
  } else {
    LevelRT<double> &T64 = C->L64[top];
    R64.vec(k_slot_convert<double>, N, (const double *)C->V, N, ctl, T64.b, T64.x, N);
    R64.cycle(top, T64.x, T64.b, true);
  }
  krylov_post(C, cond, set_cond, C->o.vcycle_fp32 != 0);
}
static void krylov_post(stokes_ctx *C, cudaGraphConditionalHandle cond, bool set_cond, bool from_fp32) {
  Runner<double> R64(C);
  Runner<float> R32(C);
  const int top = C->nl - 1;
  const long long N = C->L64[top].d.n_u + C->L64[top].d.n_p;
  const int nb = vec_blocks(N), m = C->restart;
  const int *ctl = C->kd.ctl;
  // w = K z_j: the conversion writes the operator's identity rows too (no separate k_init_identity)
  const LevelDesc<double> &Lt = C->L64[top].d;
  if (from_fp32)
    launch_kernel(k_convert_to_slot_id<float>, dim3(nb), dim3(kVecThreads), 0, C->s, Lt,
                  (const float *)C->L32[top].x, C->zcur, C->Z, N, ctl, C->w);
  else
    launch_kernel(k_convert_to_slot_id<double>, dim3(nb), dim3(kVecThreads), 0, C->s, Lt,
                  (const double *)C->L64[top].x, C->zcur, C->Z, N, ctl, C->w);
  R64.apply_nz(top, kApplyA | kApplyBT | kApplyB, C->zcur, C->zcur + Lt.n_u, C->w, C->w + Lt.n_u);
  R64.applyC(top, C->zcur + Lt.n_u, C->w + Lt.n_u, -1.0);
  // CGS2 (two passes) and ||w||^2, each dot set with its final sums in the same launch
  for (int pass = 0; pass < 2; ++pass) {
    k_mdot_final_cnt<<<kRedBlocks, kVecThreads, 0, C->s>>>(C->V, N, ctl, 1, C->w, N, C->partial, C->kd.ticket,
                                                           C->hdev + pass * (m + 2));
    k_maxpy_cnt<<<nb, kVecThreads, 0, C->s>>>(C->V, N, ctl, 1, C->hdev + pass * (m + 2), C->w, N, -1.0);
  }
  k_mdot_final_cnt<<<kRedBlocks, kVecThreads, 0, C->s>>>(nullptr, N, nullptr, 0, C->w, N, C->partial, C->kd.ticket,
                                                         C->hdev + 2 * (m + 2));
  k_scale_to_slot<<<nb, kVecThreads, 0, C->s>>>(C->w, C->hdev + 2 * (m + 2), C->V, N, ctl, N);
  k_fgmres_givens<<<1, 32, 0, C->s>>>(C->kd, cond, set_cond ? 1 : 0);
  C->cap_count += 8;
}

// Builds the device Krylov graph: a conditional while node whose body is krylov_body.  Returns
// false (and leaves kry_mode at 0, the host-driven loop) when the runtime refuses conditional
// nodes; errors of that attempt are cleared.
static bool krylov_build(stokes_ctx *C) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  cudaGraphConditionalHandle cond{};
  if (ok) ok = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t wnode = nullptr;
  if (ok) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ok = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
  }
  if (ok) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(C->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      C->capturing = true;
      C->cap_count = 0;
      krylov_body(C, cond, true);
      C->capturing = false;
      cudaGraph_t out = body;
      ok = cudaStreamEndCapture(C->s, &out) == cudaSuccess;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    if (ex) cudaGraphExecDestroy(ex);
    cudaGetLastError();
    C->kry_mode = 0;
    return false;
  }
  C->kry = ex;
  C->kry_body = C->cap_count;
  C->kry_mode = 1;
  return true;
}

static int fgmres(stokes_ctx *C, const double *b, double *x, double rtol, int maxit, int *iters, double *final_rel) {
  Runner<double> R64(C);
  Runner<float> R32(C);
  const int top = C->nl - 1;
  const long long n_u = C->L64[top].d.n_u, n_p = C->L64[top].d.n_p, N = n_u + n_p;
  const int nb = vec_blocks(N);
  const int m = C->restart;
  int st;
  double bn2;
  if ((st = dot64(C, b, b, N, &bn2))) return st;
  const double bnorm = std::sqrt(bn2);
  if (iters) *iters = 0;
  if (bnorm == 0.0) {
    SMF_CUDA_OK(cudaMemsetAsync(x, 0, N * sizeof(double), C->s));
    if (final_rel) *final_rel = 0.0;
    return STOKES_OK;
  }
  int it = 0;
  double rel = 1.0, beta0 = -1.0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hcol(2 * (m + 2));
  int status = STOKES_OK;
  double xn2;
  if ((st = dot64(C, x, x, N, &xn2))) return st;
  bool x_is_zero = xn2 == 0.0;
  if (C->kry_mode < 0) {
    const char *hk = getenv("STOKES_HOST_KRYLOV");
    if ((hk && hk[0] == '1') || !C->use_graphs)
      C->kry_mode = 0;
    else
      krylov_build(C);
  }
  while (true) {
    if (x_is_zero) {  // r = b - K 0
      SMF_CUDA_OK(cudaMemcpyAsync(C->V, b, N * sizeof(double), cudaMemcpyDeviceToDevice, C->s));
      x_is_zero = false;
    } else {
      R64.vmult(top, x, C->w, true);
      R64.sub(b, C->w, C->V, N);
    }
    double beta2;
    if ((st = dot64(C, C->V, C->V, N, &beta2))) return st;
    if ((st = det_check(C, C->s))) return st;
    const double beta = std::sqrt(beta2);
    if (beta0 < 0) beta0 = beta;
    rel = beta / bnorm;
    if (!std::isfinite(beta) || beta > 1e6 * beta0) {
      set_error("FGMRES breakdown: residual is not finite or grew by 1e6");
      status = STOKES_EBREAKDOWN;
      break;
    }
    if (rel <= rtol) break;
    if (it >= maxit) {
      set_error("FGMRES reached maxit before rtol");
      status = STOKES_ENOTCONV;
      break;
    }
    k_scale<double><<<nb, kVecThreads, 0, C->s>>>(C->V, 1.0 / beta, C->V, N);
    ++C->launches;
    if (C->kry_mode == 1) {
      // inner iterations on the device: one graph launch per restart cycle, then y = R^-1 g and
      // x += Z y; the host reads the iteration count once per cycle
      int hctl[4] = {0, it, 0, maxit};
      const double g0 = beta, th = rtol * bnorm;
      SMF_CUDA_OK(cudaMemcpyAsync(C->kd.ctl, hctl, sizeof(hctl), cudaMemcpyHostToDevice, C->s));
      SMF_CUDA_OK(cudaMemcpyAsync(C->kd.g, &g0, sizeof(double), cudaMemcpyHostToDevice, C->s));
      SMF_CUDA_OK(cudaMemcpyAsync(C->kd.thresh, &th, sizeof(double), cudaMemcpyHostToDevice, C->s));
      SMF_CUDA_OK(cudaGraphLaunch(C->kry, C->s));
      k_fgmres_trisolve<<<1, 32, 0, C->s>>>(C->kd);
      k_maxpy_cnt<<<nb, kVecThreads, 0, C->s>>>(C->Z, N, C->kd.ctl, 0, C->kd.y, x, N, 1.0);
      SMF_CUDA_OK(cudaMemcpyAsync(hctl, C->kd.ctl, sizeof(hctl), cudaMemcpyDeviceToHost, C->s));
      SMF_CUDA_OK(cudaStreamSynchronize(C->s));
      C->launches += C->kry_body * (long long)(hctl[1] - it) + 2;
      it = hctl[1];
      continue;
    }
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jd = 0;
    for (int j = 0; j < m; ++j) {
      double *vj = C->V + (long long)j * N, *zj = C->Z + (long long)j * N;
      // z_j = MG(0, v_j) in FP32 or FP64
      if (C->o.vcycle_fp32) {
        LevelRT<float> &T32 = C->L32[top];
        R32.vec(k_convert_zero<double, float, 1>, N, (const double *)vj, T32.b, T32.x, N);
        if ((st = R32.top_cycle(true))) return st;
        R32.vec(k_convert_zero<float, double, 1>, N, (const float *)T32.x, zj, (double *)nullptr, N);
      } else {
        LevelRT<double> &T64 = C->L64[top];
        R64.vecp(k_convert_zero<double, double, 1>, k_convert_zero<double, double, 2>, {vj, T64.b, T64.x}, N,
                 (const double *)vj, T64.b, T64.x, N);
        if ((st = R64.top_cycle(true))) return st;
        R64.vecp(k_convert_zero<double, double, 1>, k_convert_zero<double, double, 2>, {T64.x, zj}, N,
                 (const double *)T64.x, zj, (double *)nullptr, N);
      }
      R64.vmult(top, zj, C->w, true);
      // classical Gram-Schmidt with one re-orthogonalisation (CGS2)
      for (int pass = 0; pass < 2; ++pass) {
        k_mdot_partial<<<kRedBlocks, kVecThreads, 0, C->s>>>(C->V, N, j + 1, C->w, N, C->partial);
        k_final_reduce<<<j + 1, kVecThreads, 0, C->s>>>(C->partial, kRedBlocks, j + 1, C->hdev + pass * (m + 2));
        k_maxpy<<<nb, kVecThreads, 0, C->s>>>(C->V, N, j + 1, C->hdev + pass * (m + 2), C->w, N, -1.0);
        C->launches += 3;
      }
      k_mdot_partial<<<kRedBlocks, kVecThreads, 0, C->s>>>(C->w, N, 1, C->w, N, C->partial);
      k_final_reduce<<<1, kVecThreads, 0, C->s>>>(C->partial, kRedBlocks, 1, C->hdev + 2 * (m + 2));
      k_scale_by_inv_sqrt<<<nb, kVecThreads, 0, C->s>>>(C->w, C->hdev + 2 * (m + 2), C->V + (long long)(j + 1) * N, N);
      C->launches += 3;
      SMF_CUDA_OK(cudaMemcpyAsync(hcol.data(), C->hdev, (2 * (m + 2) + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                                  C->s));
      SMF_CUDA_OK(cudaStreamSynchronize(C->s));
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i] + hcol[(m + 2) + i];
      const double hn = std::sqrt(hcol[2 * (m + 2)]);
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = t;
      }
      const double den = std::hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
      cs[j] = H[(size_t)j * m + j] / den;
      sn[j] = H[(size_t)(j + 1) * m + j] / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jd = j + 1;
      if (!std::isfinite(g[j + 1])) break;
      if (std::fabs(g[j + 1]) <= rtol * bnorm || it >= maxit) break;
    }
    // y = H^{-1} g (upper triangular), x += Z y
    std::vector<double> y(jd);
    for (int i = jd - 1; i >= 0; --i) {
      double s = g[i];
      for (int c = i + 1; c < jd; ++c) s -= H[(size_t)i * m + c] * y[c];
      y[i] = s / H[(size_t)i * m + i];
    }
    SMF_CUDA_OK(cudaMemcpyAsync(C->hdev, y.data(), jd * sizeof(double), cudaMemcpyHostToDevice, C->s));
    k_maxpy<<<nb, kVecThreads, 0, C->s>>>(C->Z, N, jd, C->hdev, x, N, 1.0);
    ++C->launches;
    SMF_CUDA_OK(cudaStreamSynchronize(C->s));
  }
  // zero-mean pressure under full Dirichlet data (the constant pressure spans the kernel)
  if (C->pker && status != STOKES_EBREAKDOWN) {
    sum64(C, x + n_u, n_p, C->scal + 1);
    k_add_scalar<double><<<vec_blocks(n_p), kVecThreads, 0, C->s>>>(x + n_u, C->scal + 1, -1.0 / (double)n_p, n_p);
    ++C->launches;
  }
  SMF_CUDA_OK(cudaStreamSynchronize(C->s));
  if (iters) *iters = it;
  if (final_rel) *final_rel = rel;
  return status;
}


// ---- batched multi-mesh solves (layer on top of the paper's method) -------------------------
// A batch owns one context per mesh.  One FP32 V-cycle of every mesh is captured into a single
// CUDA graph with one parallel branch per mesh (each branch on that mesh's stream); the FP64
// FGMRES iterations of all meshes advance in lockstep, each mesh's FP64 work on its own stream,
// with one host synchronisation per iteration for the whole batch.
struct BatchState {
  stokes_ctx *C = nullptr;
  const double *b = nullptr;
  double *x = nullptr;
  double bnorm = 0, beta0 = -1, rel = 1;
  int it = 0, j = 0, status = STOKES_OK;
  bool done = false, need_start = true, x_zero = false;
  std::vector<double> H, cs, sn, g;
  double *hhost = nullptr;  // pinned: h columns + norms
};

}  // namespace smf

struct stokes_batch {
  std::vector<stokes_ctx *> ctx;
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0;
  std::vector<double *> pinned;
  std::string err;
  // Arnoldi loops of all members on the device: one graph per batch (while node over the
  // iterations, an if node per member); kmode -1 not built, 0 host-driven lockstep, 1 device
  cudaGraphExec_t kgraph = nullptr;
  std::vector<long long> kbody;
  int kmode = -1;
  // work-queue form (kmode 2, queue.h): the members' FP32 cycles as one persistent kernel launch
  // per iteration; qmem holds the operations, segments, member control pointers and queue state
  void *qmem = nullptr;
  PqRun qrun{};
  size_t qsmem = 0;
  unsigned qbudget = 0;
};

namespace smf {

static int batch_capture(stokes_batch *Bt) {
  SMF_CUDA_OK(cudaStreamBeginCapture(Bt->s, cudaStreamCaptureModeThreadLocal));
  SMF_CUDA_OK(cudaEventRecord(Bt->fork, Bt->s));
  long long kernels = 0;
  for (size_t i = 0; i < Bt->ctx.size(); ++i) {
    stokes_ctx *C = Bt->ctx[i];
    SMF_CUDA_OK(cudaStreamWaitEvent(C->s, Bt->fork, 0));
    Runner<float> R(C);
    const int top = C->nl - 1;
    C->capturing = true;
    C->cap_count = 0;
    R.cycle(top, C->L32[top].x, C->L32[top].b, true);
    C->capturing = false;
    kernels += C->cap_count;
    SMF_CUDA_OK(cudaEventRecord(Bt->join[i], C->s));
    SMF_CUDA_OK(cudaStreamWaitEvent(Bt->s, Bt->join[i], 0));
  }
  cudaGraph_t graph;
  SMF_CUDA_OK(cudaStreamEndCapture(Bt->s, &graph));
  cudaError_t e = cudaGraphInstantiate(&Bt->graph, graph, 0);
  cudaGraphDestroy(graph);
  SMF_CUDA_OK(e);
  Bt->graph_kernels = kernels;
  return STOKES_OK;
}

// launch a device-side dot product into dev_out (no host sync)
static void dot64_async(stokes_ctx *C, const double *a, const double *b, long long n, double *dev_out) {
  k_mdot_partial<<<kRedBlocks, kVecThreads, 0, C->s>>>(a, n, 1, b, n, C->partial);
  k_final_reduce<<<1, kVecThreads, 0, C->s>>>(C->partial, kRedBlocks, 1, dev_out);
  C->launches += 2;
}

// The device Arnoldi graph of a batch: k_batch_select (each member's condition from its stop
// flag), then one conditional while node per member, each holding that member's krylov_body, as
// independent branches with no edge between members: every member runs its inner iterations to
// its own stopping test at its own pace, so a member that needs fewer iterations, or a small mesh,
// never waits for the others inside the launch.
static bool batch_kbuild(stokes_batch *Bt) {
  const int nm = (int)Bt->ctx.size();
  Bt->kmode = 0;
  if (nm > kBatchMax) return false;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  BatchCond bc;
  bc.n = nm;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  for (int i = 0; i < nm && ok; ++i) {
    ok = cudaGraphConditionalHandleCreate(&bc.member[i], g, 0, 0) == cudaSuccess;
    bc.ctl[i] = Bt->ctx[i]->kd.ctl;
  }
  cudaGraphNode_t seln = nullptr;
  void *args[1] = {&bc};
  if (ok) {
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_batch_select;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(kBatchMax);
    kp.kernelParams = args;
    ok = cudaGraphAddKernelNode(&seln, g, nullptr, 0, &kp) == cudaSuccess;
  }
  Bt->kbody.assign(nm, 0);
  for (int i = 0; i < nm && ok; ++i) {
    stokes_ctx *C = Bt->ctx[i];
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = bc.member[i];
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn = nullptr;
    ok = cudaGraphAddNode(&wn, g, &seln, nullptr, 1, &wp) == cudaSuccess;
    if (!ok) break;
    cudaGraph_t wb = wp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(C->s, wb, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (!ok) break;
    C->capturing = true;
    C->cap_count = 0;
    krylov_body(C, bc.member[i], true);
    C->capturing = false;
    cudaGraph_t out = wb;
    ok = cudaStreamEndCapture(C->s, &out) == cudaSuccess;
    Bt->kbody[i] = C->cap_count;
  }
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    if (ex) cudaGraphExecDestroy(ex);
    cudaGetLastError();
    return false;
  }
  Bt->kgraph = ex;
  Bt->kmode = 1;
  return true;
}

// The work-queue form of the batch (kmode 2).  Every member's FP32 cycle is recorded once as its
// operation list (unfused smoothing, the same arithmetic as the launched cycle) and queued by a
// list schedule (batch_qrecord).  The device Arnoldi graph is then a while node whose body runs
// k_batch_select, per member an if node with the conversion of v_j, the queue state reset and
// ONE launch of the persistent queue kernel (every active member's cycle), per member an if node
// with the rest of its iteration (FP64 operator, CGS2, Givens) and k_batch_any.  Served: every
// member 3D, k = 2, FP32 cycle, no stabilisation, symmetric-gradient or rho term.
static bool batch_qrecord(stokes_batch *Bt) {
  if (Bt->qmem) return true;  // recorded before (stokes_batch_vcycle or an earlier build)
  const int nm = (int)Bt->ctx.size();
  bool tri = false;
  for (auto *C : Bt->ctx) {
    if (C->dim != 3 || C->k != 2 || !C->o.vcycle_fp32 || C->sym || C->c_mass != 0.0 || C->c_grad != 0.0 || C->det)
      return false;
    for (int l = 0; l < C->nl; ++l) {
      if (C->L32[l].rho) return false;
      tri = tri || !C->L32[l].d.cartesian;
    }
  }
  std::vector<std::vector<PqOp>> rec(nm);
  for (int m = 0; m < nm; ++m) {
    stokes_ctx *C = Bt->ctx[m];
    std::vector<bool> fz(C->nl);
    for (int l = 0; l < C->nl; ++l) {
      fz[l] = C->L32[l].fuse;
      C->L32[l].fuse = false;
    }
    C->pq = &rec[m];
    C->pq_member = m;
    const int top = C->nl - 1;
    Runner<float>(C).cycle(top, C->L32[top].x, C->L32[top].b, true);
    C->pq = nullptr;
    for (int l = 0; l < C->nl; ++l) C->L32[l].fuse = fz[l];
  }
  // flatten: global operation index = member offset + operation.  Queue order: a list schedule,
  // each operation at the time it could start if its member ran alone (a latency plus its items
  // spread over the resident CTAs), so a small member's later operations come before a large
  // member's; an operation always follows its member's previous one.
  std::vector<int> off(nm + 1, 0);
  for (int m = 0; m < nm; ++m) off[m + 1] = off[m] + (int)rec[m].size();
  const int nops = off[nm];
  std::vector<PqOp> ops((size_t)nops);
  for (int m = 0; m < nm; ++m) std::copy(rec[m].begin(), rec[m].end(), ops.begin() + off[m]);
  const double ctas = std::max(1, queue_resident_ctas(queue_smem_bytes(tri, kPqSmemSegments)));
  struct Slot {
    double t;
    int m, o;
  };
  std::vector<Slot> order;
  order.reserve((size_t)nops);
  for (int m = 0; m < nm; ++m) {
    double t = 0.0;
    for (int o = 0; o < (int)rec[m].size(); ++o) {
      order.push_back({t, m, o});
      t += 1.0 + std::ceil((double)rec[m][(size_t)o].items / ctas);  // in units of one item's duration
    }
  }
  std::stable_sort(order.begin(), order.end(), [](const Slot &a, const Slot &b) {
    return a.t < b.t || (a.t == b.t && (a.o < b.o || (a.o == b.o && a.m < b.m)));
  });
  std::vector<long long> start, need;
  std::vector<int> sop, sdep;
  long long total = 0;
  for (const Slot &sl : order) {
    const int g = off[sl.m] + sl.o;
    start.push_back(total);
    sop.push_back(g);
    sdep.push_back(sl.o > 0 ? g - 1 : -1);
    need.push_back(sl.o > 0 ? ops[(size_t)g - 1].items : 0);
    total += ops[(size_t)g].items;
  }
  const int nseg = (int)sop.size();
  start.push_back(total);
  // one device block: ops | seg_start | seg_need | seg_op | seg_dep | active | state
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_ops = al(sizeof(PqOp) * nops), b_start = al(sizeof(long long) * (nseg + 1)),
               b_need = al(sizeof(long long) * nseg), b_op = al(sizeof(int) * nseg), b_dep = al(sizeof(int) * nseg),
               b_act = al(sizeof(int *) * nm), b_state = al(sizeof(unsigned) * (5 + nops));
  char *mem = nullptr;
  if (cudaMalloc(&mem, b_ops + b_start + b_need + b_op + b_dep + b_act + b_state) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  Bt->qmem = mem;
  std::vector<const int *> act(nm);
  for (int m = 0; m < nm; ++m) act[m] = Bt->ctx[m]->kd.ctl;
  std::vector<unsigned> st(5 + nops, 0u);
  st[4 + nops] = Bt->qbudget;
  char *p = mem;
  PqRun R;
  bool ok = true;
  auto put = [&](const void *src, size_t n, size_t span) {
    void *dst = p;
    if (n) ok = ok && cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice) == cudaSuccess;
    p += span;
    return dst;
  };
  R.ops = (const PqOp *)put(ops.data(), sizeof(PqOp) * nops, b_ops);
  R.seg_start = (const long long *)put(start.data(), sizeof(long long) * (nseg + 1), b_start);
  R.seg_need = (const long long *)put(need.data(), sizeof(long long) * nseg, b_need);
  R.seg_op = (const int *)put(sop.data(), sizeof(int) * nseg, b_op);
  R.seg_dep = (const int *)put(sdep.data(), sizeof(int) * nseg, b_dep);
  R.active = (const int *const *)put(act.data(), sizeof(int *) * nm, b_act);
  R.state = (unsigned *)put(st.data(), sizeof(unsigned) * (5 + nops), b_state);
  R.nseg = nseg;
  R.nops = nops;
  R.total = total;
  R.geo_smem = (unsigned)queue_geo_smem_bytes(tri);
  Bt->qrun = R;
  Bt->qsmem = queue_smem_bytes(tri, nseg);
  if (!ok || queue_resident_ctas(Bt->qsmem) <= 0) {
    cudaGetLastError();
    cudaFree(Bt->qmem);
    Bt->qmem = nullptr;
    return false;
  }
  return true;
}

static bool batch_qbuild(stokes_batch *Bt) {
  const int nm = (int)Bt->ctx.size();
  Bt->kmode = 0;
  if (nm > kBatchMax || !batch_qrecord(Bt)) return false;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  BatchCond bc;
  bc.n = nm;
  bc.has_post = 1;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  if (ok) ok = cudaGraphConditionalHandleCreate(&bc.loop, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams wp = {};
  cudaGraphNode_t wn = nullptr;
  if (ok) {
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = bc.loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    ok = cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp) == cudaSuccess;
  }
  cudaGraph_t body = ok ? wp.conditional.phGraph_out[0] : nullptr;
  for (int i = 0; i < nm && ok; ++i) {
    ok = cudaGraphConditionalHandleCreate(&bc.member[i], body, 0, 0) == cudaSuccess &&
         cudaGraphConditionalHandleCreate(&bc.post[i], body, 0, 0) == cudaSuccess;
    bc.ctl[i] = Bt->ctx[i]->kd.ctl;
  }
  void *args[1] = {&bc};
  cudaGraphNode_t seln = nullptr, anyn = nullptr;
  if (ok) {
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_batch_select;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(kBatchMax);
    kp.kernelParams = args;
    ok = cudaGraphAddKernelNode(&seln, body, nullptr, 0, &kp) == cudaSuccess;
  }
  // an if node per member on its own stream, `capture` filling its body
  auto add_if = [&](cudaGraphConditionalHandle h, const cudaGraphNode_t *deps, size_t nd, stokes_ctx *C,
                    const std::function<void()> &capture, cudaGraphNode_t *node) {
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    bool r = cudaGraphAddNode(node, body, deps, nullptr, nd, &ip) == cudaSuccess;
    if (r) {
      cudaGraph_t ib = ip.conditional.phGraph_out[0];
      r = cudaStreamBeginCaptureToGraph(C->s, ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
          cudaSuccess;
      if (r) {
        C->capturing = true;
        C->cap_count = 0;
        capture();
        C->capturing = false;
        cudaGraph_t out = ib;
        r = cudaStreamEndCapture(C->s, &out) == cudaSuccess;
      }
    }
    return r;
  };
  std::vector<cudaGraphNode_t> pre(nm, nullptr), post(nm, nullptr);
  Bt->kbody.assign(nm, 0);
  for (int i = 0; i < nm && ok; ++i) {
    stokes_ctx *C = Bt->ctx[i];
    ok = add_if(bc.member[i], &seln, 1, C, [&] { krylov_pre(C); }, &pre[i]);
    Bt->kbody[i] = C->cap_count;
  }
  // queue state reset and the persistent kernel, after every member's conversion
  cudaGraphNode_t qnode = nullptr;
  if (ok) {
    ok = cudaStreamBeginCaptureToGraph(Bt->s, body, pre.data(), nullptr, nm, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      cudaMemsetAsync(Bt->qrun.state, 0, sizeof(unsigned) * (4 + Bt->qrun.nops), Bt->s);
      const int e = launch_queue(Bt->qrun, Bt->qsmem, Bt->s);
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t *deps = nullptr;
      size_t nd = 0;
      ok = e == 0 && cudaStreamGetCaptureInfo(Bt->s, &cs, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess &&
           nd == 1;
      if (ok) qnode = deps[0];
      cudaGraph_t out = body;
      ok = cudaStreamEndCapture(Bt->s, &out) == cudaSuccess && ok;
    }
  }
  for (int i = 0; i < nm && ok; ++i) {
    stokes_ctx *C = Bt->ctx[i];
    ok = add_if(bc.post[i], &qnode, 1, C, [&] { krylov_post(C, cudaGraphConditionalHandle{}, false, true); },
                &post[i]);
    Bt->kbody[i] += C->cap_count;
  }
  if (ok) {
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_batch_any;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    ok = cudaGraphAddKernelNode(&anyn, body, post.data(), nm, &kp) == cudaSuccess;
  }
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    if (ex) cudaGraphExecDestroy(ex);
    cudaGetLastError();
    if (Bt->qmem) cudaFree(Bt->qmem);
    Bt->qmem = nullptr;
    return false;
  }
  Bt->kgraph = ex;
  Bt->kmode = 2;
  return true;
}

static int batch_solve(stokes_batch *Bt, const double *const *b, double *const *x, double rtol, int maxit, int *iters,
                       double *final_rel) {
  const int nm = (int)Bt->ctx.size();
  if (Bt->kmode < 0) {
    const char *hk = getenv("STOKES_HOST_KRYLOV");
    const char *qe = getenv("STOKES_BATCH_QUEUE");
    if ((hk && hk[0] == '1') || !Bt->ctx[0]->use_graphs)
      Bt->kmode = 0;
    else if (!(qe && qe[0] == '1' && batch_qbuild(Bt)))
      batch_kbuild(Bt);
  }
  std::vector<BatchState> S(nm);
  for (int i = 0; i < nm; ++i) {
    BatchState &st = S[i];
    st.C = Bt->ctx[i];
    st.b = b[i];
    st.x = x[i];
    const int m = st.C->restart;
    st.H.assign((size_t)(m + 1) * m, 0.0);
    st.cs.assign(m, 0.0);
    st.sn.assign(m, 0.0);
    st.g.assign(m + 1, 0.0);
    st.hhost = Bt->pinned[i];
    const int top = st.C->nl - 1;
    const long long N = st.C->L64[top].d.n_u + st.C->L64[top].d.n_p;
    dot64_async(st.C, st.b, st.b, N, st.C->scal);
    dot64_async(st.C, st.x, st.x, N, st.C->scal + 1);
    SMF_CUDA_OK(cudaMemcpyAsync(st.hhost, st.C->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st.C->s));
  }
  for (int i = 0; i < nm; ++i) {
    SMF_CUDA_OK(cudaStreamSynchronize(S[i].C->s));
    S[i].bnorm = std::sqrt(S[i].hhost[0]);
    S[i].x_zero = S[i].hhost[1] == 0.0;
    if (S[i].bnorm == 0.0) {
      const int top = S[i].C->nl - 1;
      const long long N = S[i].C->L64[top].d.n_u + S[i].C->L64[top].d.n_p;
      SMF_CUDA_OK(cudaMemsetAsync(S[i].x, 0, N * sizeof(double), S[i].C->s));
      S[i].done = true;
      S[i].rel = 0.0;
    }
  }
  while (true) {
    // (a) restart-cycle start: r = b - K x, beta = ||r||
    bool any_start = false;
    for (auto &st : S) {
      if (st.done || !st.need_start) continue;
      any_start = true;
      stokes_ctx *C = st.C;
      Runner<double> R64(C);
      const int top = C->nl - 1;
      const long long N = R64.nu(top) + R64.np(top);
      if (st.x_zero) {
        SMF_CUDA_OK(cudaMemcpyAsync(C->V, st.b, N * sizeof(double), cudaMemcpyDeviceToDevice, C->s));
        st.x_zero = false;
      } else {
        R64.vmult(top, st.x, C->w, true);
        R64.sub(st.b, C->w, C->V, N);
      }
      dot64_async(C, C->V, C->V, N, C->scal);
      SMF_CUDA_OK(cudaMemcpyAsync(st.hhost, C->scal, sizeof(double), cudaMemcpyDeviceToHost, C->s));
    }
    if (any_start) {
      for (auto &st : S) {
        if (st.done || !st.need_start) continue;
        SMF_CUDA_OK(cudaStreamSynchronize(st.C->s));
        const double beta = std::sqrt(st.hhost[0]);
        if (st.beta0 < 0) st.beta0 = beta;
        st.rel = beta / st.bnorm;
        st.need_start = false;
        if (!std::isfinite(beta) || beta > 1e6 * st.beta0) {
          st.status = STOKES_EBREAKDOWN;
          st.done = true;
        } else if (st.rel <= rtol) {
          st.done = true;
        } else if (st.it >= maxit) {
          st.status = STOKES_ENOTCONV;
          st.done = true;
        } else {
          stokes_ctx *C = st.C;
          const int top = C->nl - 1;
          const long long N = C->L64[top].d.n_u + C->L64[top].d.n_p;
          k_scale<double><<<vec_blocks(N), kVecThreads, 0, C->s>>>(C->V, 1.0 / beta, C->V, N);
          ++C->launches;
          std::fill(st.H.begin(), st.H.end(), 0.0);
          std::fill(st.g.begin(), st.g.end(), 0.0);
          st.g[0] = beta;
          st.j = 0;
        }
      }
    }
    int nactive = 0;
    for (auto &st : S) nactive += st.done ? 0 : 1;
    if (nactive == 0) break;
    if (Bt->kmode >= 1) {
      // (b') every active member's inner iterations in one graph launch: members independent
      // (kmode 1), or in lockstep around the work-queue kernel of their cycles (kmode 2)
      for (auto &st : S) {
        stokes_ctx *C = st.C;
        int hctl[4] = {0, st.it, st.done ? 5 : 0, maxit};
        SMF_CUDA_OK(cudaMemcpyAsync(C->kd.ctl, hctl, sizeof(hctl), cudaMemcpyHostToDevice, C->s));
        if (!st.done) {
          const double g0 = st.g[0], th = rtol * st.bnorm;
          SMF_CUDA_OK(cudaMemcpyAsync(C->kd.g, &g0, sizeof(double), cudaMemcpyHostToDevice, C->s));
          SMF_CUDA_OK(cudaMemcpyAsync(C->kd.thresh, &th, sizeof(double), cudaMemcpyHostToDevice, C->s));
        }
      }
      for (int i = 0; i < nm; ++i) {
        SMF_CUDA_OK(cudaEventRecord(Bt->join[i], Bt->ctx[i]->s));
        SMF_CUDA_OK(cudaStreamWaitEvent(Bt->s, Bt->join[i], 0));
      }
      SMF_CUDA_OK(cudaGraphLaunch(Bt->kgraph, Bt->s));
      SMF_CUDA_OK(cudaEventRecord(Bt->fork, Bt->s));
      for (auto &st : S) {
        stokes_ctx *C = st.C;
        SMF_CUDA_OK(cudaStreamWaitEvent(C->s, Bt->fork, 0));
        if (st.done) continue;
        const int top = C->nl - 1;
        const long long N = C->L64[top].d.n_u + C->L64[top].d.n_p;
        k_fgmres_trisolve<<<1, 32, 0, C->s>>>(C->kd);
        k_maxpy_cnt<<<vec_blocks(N), kVecThreads, 0, C->s>>>(C->Z, N, C->kd.ctl, 0, C->kd.y, st.x, N, 1.0);
        SMF_CUDA_OK(cudaMemcpyAsync(st.hhost, C->kd.ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, C->s));
      }
      for (int i = 0; i < nm; ++i) {
        BatchState &st = S[i];
        if (st.done) continue;
        SMF_CUDA_OK(cudaStreamSynchronize(st.C->s));
        int hctl[4];
        std::memcpy(hctl, st.hhost, sizeof(hctl));
        st.C->launches += Bt->kbody[i] * (long long)(hctl[1] - st.it) + 2;
        st.it = hctl[1];
        st.need_start = true;
      }
      if (Bt->kmode == 2) {
        unsigned qerr = 0;
        SMF_CUDA_OK(cudaMemcpyAsync(&qerr, Bt->qrun.state + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, Bt->s));
        SMF_CUDA_OK(cudaStreamSynchronize(Bt->s));
        if (qerr) {
          set_error("batched work-queue kernel: a dependency wait exceeded its budget");
          return STOKES_ETIMEOUT;
        }
      }
      continue;
    }
    // (b) one Arnoldi step for every active mesh; the FP32 cycles of all meshes in one graph
    for (auto &st : S) {
      if (st.done) continue;
      stokes_ctx *C = st.C;
      const int top = C->nl - 1;
      const long long N = C->L64[top].d.n_u + C->L64[top].d.n_p;
      Runner<float> R32(C);
      R32.vec(k_convert_zero<double, float, 1>, N, (const double *)(C->V + (long long)st.j * N), C->L32[top].b,
              C->L32[top].x, N);
    }
    if (nactive == nm) {
      if (!Bt->graph) {
        int st = batch_capture(Bt);
        if (st) return st;
      }
      // the batch stream waits for every member's input conversion before the graph starts
      for (int i = 0; i < nm; ++i) {
        SMF_CUDA_OK(cudaEventRecord(Bt->join[i], Bt->ctx[i]->s));
        SMF_CUDA_OK(cudaStreamWaitEvent(Bt->s, Bt->join[i], 0));
      }
      SMF_CUDA_OK(cudaGraphLaunch(Bt->graph, Bt->s));
      for (auto *C : Bt->ctx) C->launches += Bt->graph_kernels / nm;
      SMF_CUDA_OK(cudaEventRecord(Bt->fork, Bt->s));
      for (auto *C : Bt->ctx) SMF_CUDA_OK(cudaStreamWaitEvent(C->s, Bt->fork, 0));
    } else {
      for (auto &st : S) {
        if (st.done) continue;
        int e = Runner<float>(st.C).top_cycle(true);
        if (e) return e;
      }
    }
    for (auto &st : S) {
      if (st.done) continue;
      stokes_ctx *C = st.C;
      Runner<double> R64(C);
      Runner<float> R32(C);
      const int top = C->nl - 1;
      const long long N = R64.nu(top) + R64.np(top);
      const int m = C->restart, j = st.j;
      double *zj = C->Z + (long long)j * N;
      R32.vec(k_convert_zero<float, double, 1>, N, (const float *)C->L32[top].x, zj, (double *)nullptr, N);
      R64.vmult(top, zj, C->w, true);
      const int nb = vec_blocks(N);
      for (int pass = 0; pass < 2; ++pass) {
        k_mdot_partial<<<kRedBlocks, kVecThreads, 0, C->s>>>(C->V, N, j + 1, C->w, N, C->partial);
        k_final_reduce<<<j + 1, kVecThreads, 0, C->s>>>(C->partial, kRedBlocks, j + 1, C->hdev + pass * (m + 2));
        k_maxpy<<<nb, kVecThreads, 0, C->s>>>(C->V, N, j + 1, C->hdev + pass * (m + 2), C->w, N, -1.0);
        C->launches += 3;
      }
      k_mdot_partial<<<kRedBlocks, kVecThreads, 0, C->s>>>(C->w, N, 1, C->w, N, C->partial);
      k_final_reduce<<<1, kVecThreads, 0, C->s>>>(C->partial, kRedBlocks, 1, C->hdev + 2 * (m + 2));
      k_scale_by_inv_sqrt<<<nb, kVecThreads, 0, C->s>>>(C->w, C->hdev + 2 * (m + 2), C->V + (long long)(j + 1) * N, N);
      C->launches += 3;
      SMF_CUDA_OK(cudaMemcpyAsync(st.hhost, C->hdev, (2 * (m + 2) + 1) * sizeof(double), cudaMemcpyDeviceToHost, C->s));
    }
    for (auto &st : S) {
      if (st.done) continue;
      stokes_ctx *C = st.C;
      SMF_CUDA_OK(cudaStreamSynchronize(C->s));
      const int m = C->restart, j = st.j;
      std::vector<double> &H = st.H;
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = st.hhost[i] + st.hhost[(m + 2) + i];
      H[(size_t)(j + 1) * m + j] = std::sqrt(st.hhost[2 * (m + 2)]);
      for (int i = 0; i < j; ++i) {
        const double t = st.cs[i] * H[(size_t)i * m + j] + st.sn[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)(i + 1) * m + j] = -st.sn[i] * H[(size_t)i * m + j] + st.cs[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = t;
      }
      const double den = std::hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
      st.cs[j] = H[(size_t)j * m + j] / den;
      st.sn[j] = H[(size_t)(j + 1) * m + j] / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      st.g[j + 1] = -st.sn[j] * st.g[j];
      st.g[j] = st.cs[j] * st.g[j];
      ++st.it;
      ++st.j;
      const bool end_cycle = !std::isfinite(st.g[st.j]) || std::fabs(st.g[st.j]) <= rtol * st.bnorm ||
                             st.it >= maxit || st.j == m;
      if (end_cycle) {
        const int jd = st.j;
        std::vector<double> y(jd);
        for (int i = jd - 1; i >= 0; --i) {
          double sum = st.g[i];
          for (int c = i + 1; c < jd; ++c) sum -= H[(size_t)i * m + c] * y[c];
          y[i] = sum / H[(size_t)i * m + i];
        }
        const int top = C->nl - 1;
        const long long N = C->L64[top].d.n_u + C->L64[top].d.n_p;
        for (int i = 0; i < jd; ++i) st.hhost[i] = y[i];
        SMF_CUDA_OK(cudaMemcpyAsync(C->hdev, st.hhost, jd * sizeof(double), cudaMemcpyHostToDevice, C->s));
        k_maxpy<<<vec_blocks(N), kVecThreads, 0, C->s>>>(C->Z, N, jd, C->hdev, st.x, N, 1.0);
        ++C->launches;
        st.need_start = true;
      }
    }
  }
  for (int i = 0; i < nm; ++i) {
    BatchState &st = S[i];
    stokes_ctx *C = st.C;
    const int top = C->nl - 1;
    const long long n_u = C->L64[top].d.n_u, n_p = C->L64[top].d.n_p;
    if (C->pker && st.status != STOKES_EBREAKDOWN && st.bnorm > 0) {
      sum64(C, st.x + n_u, n_p, C->scal + 1);
      k_add_scalar<double><<<vec_blocks(n_p), kVecThreads, 0, C->s>>>(st.x + n_u, C->scal + 1, -1.0 / (double)n_p,
                                                                       n_p);
      ++C->launches;
    }
  }
  int status = STOKES_OK;
  for (int i = 0; i < nm; ++i) {
    SMF_CUDA_OK(cudaStreamSynchronize(S[i].C->s));
    if (iters) iters[i] = S[i].it;
    if (final_rel) final_rel[i] = S[i].rel;
    if (S[i].status != STOKES_OK && status == STOKES_OK) status = S[i].status;
  }
  if (status == STOKES_ENOTCONV) set_error("a batch member reached maxit before rtol");
  if (status == STOKES_EBREAKDOWN) set_error("FGMRES breakdown in a batch member");
  return status;
}

// ---- allocation-free smoothing --------------------------------------------------------------
// Scratch of stokes_smooth_noalloc: one file-scope device array, present on every GPU that loads
// the library until the process exits.  Host code cannot hand the array's name to a kernel (on
// the host it only stands for the symbol), so its device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, and cached here.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
constexpr int kNoAllocMaxDevices = 64;
static void *g_noalloc_addr[kNoAllocMaxDevices];

static int noalloc_scratch_address(void **out) {
  int dev = 0;
  SMF_CUDA_OK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("device index out of range for the allocation-free scratch table");
    return STOKES_EINVAL;
  }
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    SMF_CUDA_OK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return STOKES_OK;
}

static long long noalloc_pad(long long n) { return (n + 63) / 64 * 64; }

// Bytes of smoother scratch a level needs: 11 velocity and 6 pressure work vectors.
static size_t noalloc_bytes(long long n_u, long long n_p, size_t elt) {
  return (size_t)(11 * noalloc_pad(n_u) + 6 * noalloc_pad(n_p)) * elt;
}

// Run `steps` smoothing steps on `level` with every work vector of the smoother carved out of
// the static scratch (the context's own work vectors of that level are swapped out meanwhile).
template <typename T>
static void smooth_noalloc_run(stokes_ctx *C, int level, int steps, void *base, const T *b, T *x) {
  std::vector<LevelRT<T>> &Ls = levels<T>(C);
  const LevelRT<T> saved = Ls[level];
  LevelRT<T> &R = Ls[level];
  const long long nu = R.d.n_u, np = R.d.n_p;
  T *cur = static_cast<T *>(base);
  auto take = [&](long long n) {
    T *q = cur;
    cur += noalloc_pad(n);
    return q;
  };
  T **vel[] = {&R.tu, &R.ru, &R.uhat, &R.cx, &R.cd, &R.ct, &R.r2, &R.cx2, &R.cd2, &R.ct2, &R.au};
  for (auto q : vel) *q = take(nu);
  T **pre[] = {&R.pt, &R.rp, &R.px, &R.pd, &R.ps, &R.dp};
  for (auto q : pre) *q = take(np);
  Runner<T>(C).smooth(level, x, b, steps, false);
  Ls[level] = saved;
}

}  // namespace smf

// ================================ C ABI ========================================================
extern "C" {

void stokes_default_opts(stokes_opts *o) {
  if (!o) return;
  o->kA = 3;
  o->kS = 3;
  o->m = 2;
  o->cycle = 0;
  o->schur_diag = 0;
  o->vcycle_fp32 = 1;
  o->gmres_restart = 30;
  o->eig_iters = 40;
  o->eig_safety = 1.1;
  o->seed = 0x5EEDull;
  o->c_mass = 0.0;
  o->c_grad = 0.0;
  o->sym_grad = 0;
  o->rho_cell = nullptr;
  o->deterministic = 0;
  o->wait_cycles = 0;
}

// Every cell of a vertex-given mesh must be a proper image of the reference cell (Sec. 2: T_tau
// bijective): finite coordinates and det J > 0 at each of its 2^d corners, J formed from the cell's
// edges that leave the corner along the +x, +y (+z) reference directions.  Host-side, before any
// device work.
static int check_cell_orientation(const stokes_mesh *mesh) {
  const int dim = mesh->dim, nx = mesh->n[0], ny = mesh->n[1], nz = dim == 3 ? mesh->n[2] : 1;
  const double *V = mesh->vertices;
  auto vx = [&](int i, int j, int k2, int a) { return V[(((long long)k2 * (ny + 1) + j) * (nx + 1) + i) * dim + a]; };
  const long long nv = (long long)(nx + 1) * (ny + 1) * (dim == 3 ? nz + 1 : 1) * dim;
  for (long long i = 0; i < nv; ++i)
    if (!std::isfinite(V[i])) {
      set_error("vertices: coordinate " + std::to_string(i) + " is not finite");
      return STOKES_EINVAL;
    }
  for (int k2 = 0; k2 < nz; ++k2)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        for (int c = 0; c < (1 << dim); ++c) {
          const int ci = i + (c & 1), cj = j + ((c >> 1) & 1), ck = k2 + (dim == 3 ? (c >> 2) & 1 : 0);
          // edge along axis a from this corner to its neighbour in the cell, oriented along +a
          double e[3][3] = {};
          for (int a = 0; a < dim; ++a) {
            const int s = ((c >> a) & 1) ? -1 : 1;
            const int ni = ci + (a == 0 ? s : 0), nj = cj + (a == 1 ? s : 0), nk = ck + (a == 2 ? s : 0);
            for (int b = 0; b < dim; ++b) e[a][b] = s * (vx(ni, nj, nk, b) - vx(ci, cj, ck, b));
          }
          const double det = dim == 3 ? e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                                            e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                                            e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0])
                                      : e[0][0] * e[1][1] - e[0][1] * e[1][0];
          if (!(det > 0)) {
            set_error("vertices: cell (" + std::to_string(i) + ", " + std::to_string(j) +
                      (dim == 3 ? ", " + std::to_string(k2) : std::string()) +
                      ") is inverted or degenerate at one of its corners (det J <= 0)");
            return STOKES_EINVAL;
          }
        }
  return STOKES_OK;
}

int stokes_setup(const stokes_mesh *mesh, int k, double mu, double gamma_rho, const double *mu_cell,
                 const stokes_opts *opts, void *stream, stokes_ctx **out) {
  if (!out) {
    set_error("out is NULL");
    return STOKES_EINVAL;
  }
  *out = nullptr;
  if (!mesh || (mesh->dim != 2 && mesh->dim != 3) || k < 2 || k > kMaxDeg || mesh->n_levels < 1 ||
      mesh->n_levels > STOKES_MAX_LEVELS || !(mu > 0) || !(gamma_rho >= 0)) {
    set_error("invalid mesh / k / mu / gamma_rho (dim in {2,3}, k in {2,3,4}, 1 <= n_levels <= 12, mu > 0, gamma >= 0)");
    return STOKES_EINVAL;
  }
  for (int a = 0; a < mesh->dim; ++a) {
    const int s = 1 << (mesh->n_levels - 1);
    if (mesh->n[a] < 1 || mesh->n[a] % s != 0 || !(mesh->hi[a] > mesh->lo[a])) {
      set_error("n[a] must be a positive multiple of 2^(n_levels-1) and hi > lo");
      return STOKES_EINVAL;
    }
  }
  if (mu_cell) {
    const long long nc = (long long)mesh->n[0] * mesh->n[1] * (mesh->dim == 3 ? mesh->n[2] : 1);
    for (long long i = 0; i < nc; ++i)
      if (!(mu_cell[i] > 0)) {
        set_error("mu_cell entries must be positive");
        return STOKES_EINVAL;
      }
  }
  if (mesh->vertices && check_cell_orientation(mesh) != STOKES_OK) return STOKES_EINVAL;
  {
    void *scratch = nullptr;  // device address of the allocation-free scratch, once per device
    const int sa = noalloc_scratch_address(&scratch);
    if (sa != STOKES_OK) return sa;
  }
  stokes_ctx *C = new (std::nothrow) stokes_ctx();
  if (!C) {
    set_error("host allocation failed");
    return STOKES_ENOMEM;
  }
  cudaStream_t user = (cudaStream_t)stream;
  cudaStreamSynchronize(user);
  if (cudaGetDevice(&C->device) != cudaSuccess) {
    cudaGetLastError();
    C->device = -1;
  }
  int st = do_setup(mesh, k, mu, gamma_rho, mu_cell, opts, C);
  if (st == STOKES_OK) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "setup kernels", __FILE__, __LINE__);
  }
  if (st != STOKES_OK) {
    stokes_destroy(C);
    return st;
  }
  *out = C;
  return STOKES_OK;
}

int stokes_sizes(const stokes_ctx *C, int level, long long *n_u, long long *n_p) {
  if (!C || level < 0 || level >= C->nl) {
    set_error("level out of range");
    return STOKES_EINVAL;
  }
  if (n_u) *n_u = C->L64[level].d.n_u;
  if (n_p) *n_p = C->L64[level].d.n_p;
  return STOKES_OK;
}

int stokes_vmult(stokes_ctx *C, int level, int precision, const void *x, void *y, void *stream) {
  if (!check_level(C, level) || !x || !y || (precision != 32 && precision != 64)) {
    set_error("invalid stokes_vmult arguments");
    if (C) C->err = "invalid stokes_vmult arguments";
    return STOKES_EINVAL;
  }
  // The operator reads only x and the context's read-only level data, so it is launched directly
  // on the caller's stream (no join with the context stream).
  if (det_begin(C, (cudaStream_t)stream) != STOKES_OK) {
    C->err = g_last_error;
    return STOKES_ECUDA;
  }
  if (precision == 64)
    Runner<double>(C, (cudaStream_t)stream, Runner<double>::OnStream{}).vmult(level, (const double *)x, (double *)y,
                                                                           true);
  else
    Runner<float>(C, (cudaStream_t)stream, Runner<float>::OnStream{}).vmult(level, (const float *)x, (float *)y, true);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_fail(e, "stokes_vmult launch", __FILE__, __LINE__);
    C->err = g_last_error;
    return STOKES_ECUDA;
  }
  const int dst = det_check(C, (cudaStream_t)stream);
  if (dst != STOKES_OK) C->err = g_last_error;
  return dst;
}

int stokes_apply_blocks(stokes_ctx *C, int level, int precision, int blocks, const void *u, const void *p, void *yu,
                        void *yp, void *stream) {
  const bool withC = blocks & kApplyC;
  const int base = blocks & ~kApplyC;
  const bool mass = base == kApplyMass || base == kApplyMassAll;
  if (!check_level(C, level) || (precision != 32 && precision != 64) || blocks <= 0 || (base > 7 && !mass) ||
      (mass && withC) || ((base & (1 | 8 | 16)) && (!u || !yu)) || ((base & 2) && (!p || !yu)) ||
      ((base & 4) && (!u || !yp)) || (withC && (!p || !yp))) {
    set_error("invalid stokes_apply_blocks arguments");
    if (C) C->err = "invalid stokes_apply_blocks arguments";
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  det_begin(C, C->s);
  const bool wu = base & (1 | 2 | 8 | 16), wp = base & 4;
  if (precision == 64) {
    Runner<double> R(C);
    if (base) R.apply(level, base, (const double *)u, (const double *)p, wu ? (double *)yu : nullptr,
                      wp ? (double *)yp : nullptr);
    if (withC) {
      if (!wp) cudaMemsetAsync(yp, 0, R.np(level) * sizeof(double), C->s);
      R.applyC(level, (const double *)p, (double *)yp, -1.0);
    }
  } else {
    Runner<float> R(C);
    if (base) R.apply(level, base, (const float *)u, (const float *)p, wu ? (float *)yu : nullptr,
                      wp ? (float *)yp : nullptr);
    if (withC) {
      if (!wp) cudaMemsetAsync(yp, 0, R.np(level) * sizeof(float), C->s);
      R.applyC(level, (const float *)p, (float *)yp, -1.0f);
    }
  }
  return finish(C, STOKES_OK);
}

int stokes_mass_rhs(stokes_ctx *C, int level, int precision, const void *f, void *b, void *stream) {
  if (!check_level(C, level) || !f || !b || (precision != 32 && precision != 64)) {
    set_error("invalid stokes_mass_rhs arguments");
    if (C) C->err = "invalid stokes_mass_rhs arguments";
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  if (precision == 64) {
    Runner<double> R(C);
    R.apply(level, kApplyMass, (const double *)f, nullptr, (double *)b, nullptr);
    cudaMemsetAsync((double *)b + R.nu(level), 0, R.np(level) * sizeof(double), C->s);
  } else {
    Runner<float> R(C);
    R.apply(level, kApplyMass, (const float *)f, nullptr, (float *)b, nullptr);
    cudaMemsetAsync((float *)b + R.nu(level), 0, R.np(level) * sizeof(float), C->s);
  }
  return finish(C, STOKES_OK);
}

int stokes_smooth(stokes_ctx *C, int level, int precision, int steps, const void *b, void *x, void *stream) {
  if (!check_level(C, level) || level < 1 || steps < 0 || !b || !x || (precision != 32 && precision != 64)) {
    set_error("invalid stokes_smooth arguments (level must be >= 1)");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  det_begin(C, C->s);
  if (precision == 64)
    Runner<double>(C).smooth(level, (double *)x, (const double *)b, steps, false);
  else
    Runner<float>(C).smooth(level, (float *)x, (const float *)b, steps, false);
  return finish(C, STOKES_OK);
}

int stokes_smooth_noalloc(stokes_ctx *C, int level, int precision, int steps, const void *b, void *x, void *stream) {
  if (!check_level(C, level) || level < 1 || steps < 0 || !b || !x || (precision != 32 && precision != 64)) {
    set_error("invalid stokes_smooth_noalloc arguments (level must be >= 1)");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  const long long nu = C->L64[level].d.n_u, np = C->L64[level].d.n_p;
  const size_t need = noalloc_bytes(nu, np, precision == 64 ? sizeof(double) : sizeof(float));
  if (need > kNoAllocScratchBytes) {
    set_error("stokes_smooth_noalloc: level " + std::to_string(level) + " needs " + std::to_string(need) +
              " bytes of smoother scratch, more than the " + std::to_string(kNoAllocScratchBytes) +
              " bytes of the static scratch array; use stokes_smooth");
    C->err = g_last_error;
    return STOKES_EINVAL;
  }
  // the static array has one instance per device: use the context's, which needs its device current
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != C->device) {
    cudaGetLastError();
    set_error("stokes_smooth_noalloc: make the context's device (" + std::to_string(C->device) +
              ") current before the call");
    C->err = g_last_error;
    return STOKES_EINVAL;
  }
  void *base = nullptr;
  int st = noalloc_scratch_address(&base);
  if (st != STOKES_OK) {
    C->err = g_last_error;
    return st;
  }
  StreamGuard sg(C, stream);
  det_begin(C, C->s);  // deterministic mode: a fresh grid-barrier state, as in stokes_smooth
  // the scratch keeps the previous call's contents: the smoother's accumulation targets must start
  // at zero, so the used part is cleared first
  cudaMemsetAsync(base, 0, need, C->s);
  if (precision == 64)
    smooth_noalloc_run<double>(C, level, steps, base, (const double *)b, (double *)x);
  else
    smooth_noalloc_run<float>(C, level, steps, base, (const float *)b, (float *)x);
  return finish(C, STOKES_OK);
}

int stokes_transfer(stokes_ctx *C, int fine_level, int precision, int direction, const void *in, void *out,
                    void *stream) {
  if (!check_level(C, fine_level) || fine_level < 1 || !in || !out || (direction != 0 && direction != 1) ||
      (precision != 32 && precision != 64)) {
    set_error("invalid stokes_transfer arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  if (precision == 64) {
    Runner<double> R(C);
    if (direction == 0)
      R.restrict_to(fine_level, (const double *)in, (double *)out, nullptr);
    else
      R.prolongate(fine_level, (const double *)in, (double *)out, 0);
  } else {
    Runner<float> R(C);
    if (direction == 0)
      R.restrict_to(fine_level, (const float *)in, (float *)out, nullptr);
    else
      R.prolongate(fine_level, (const float *)in, (float *)out, 0);
  }
  return finish(C, STOKES_OK);
}

int stokes_coarse_solve(stokes_ctx *C, int precision, const void *b, void *x, void *stream) {
  if (!C || !b || !x || (precision != 32 && precision != 64)) {
    set_error("invalid stokes_coarse_solve arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  if (precision == 64)
    Runner<double>(C).coarse((const double *)b, (double *)x);
  else
    Runner<float>(C).coarse((const float *)b, (float *)x);
  return finish(C, STOKES_OK);
}

int mg_vcycle(stokes_ctx *C, int precision, const void *b, void *x, void *stream) {
  if (!C || !b || !x || (precision != 32 && precision != 64)) {
    set_error("invalid mg_vcycle arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  det_begin(C, C->s);
  const int top = C->nl - 1;
  int st;
  if (precision == 64) {
    Runner<double> R(C);
    const long long N = R.nu(top) + R.np(top);
    cudaMemcpyAsync(C->L64[top].b, b, N * sizeof(double), cudaMemcpyDeviceToDevice, C->s);
    cudaMemcpyAsync(C->L64[top].x, x, N * sizeof(double), cudaMemcpyDeviceToDevice, C->s);
    st = R.top_cycle(false);
    cudaMemcpyAsync(x, C->L64[top].x, N * sizeof(double), cudaMemcpyDeviceToDevice, C->s);
  } else {
    Runner<float> R(C);
    const long long N = R.nu(top) + R.np(top);
    cudaMemcpyAsync(C->L32[top].b, b, N * sizeof(float), cudaMemcpyDeviceToDevice, C->s);
    cudaMemcpyAsync(C->L32[top].x, x, N * sizeof(float), cudaMemcpyDeviceToDevice, C->s);
    st = R.top_cycle(false);
    cudaMemcpyAsync(x, C->L32[top].x, N * sizeof(float), cudaMemcpyDeviceToDevice, C->s);
  }
  return finish(C, st);
}

int stokes_solve(stokes_ctx *C, const double *b, double *x, double rtol, int maxit, int *iters, double *final_rel_res,
                 void *stream) {
  if (!C || !b || !x || !(rtol > 0) || maxit < 0) {
    set_error("invalid stokes_solve arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  det_begin(C, C->s);
  int st = fgmres(C, b, x, rtol, maxit, iters, final_rel_res);
  return finish(C, st);
}

int stokes_solve_host(stokes_ctx *C, const double *b_host, double *x_host, double rtol, int maxit, int *iters,
                      double *final_rel_res, void *stream) {
  if (!C || !b_host || !x_host || !(rtol > 0) || maxit < 0) {
    set_error("invalid stokes_solve_host arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  const int top = C->nl - 1;
  const long long N = C->L64[top].d.n_u + C->L64[top].d.n_p;
  StreamGuard sg(C, stream);
  det_begin(C, C->s);
  double *db = C->lz0, *dx = C->lz1;
  cudaMemcpyAsync(db, b_host, N * sizeof(double), cudaMemcpyHostToDevice, C->s);
  cudaMemsetAsync(dx, 0, N * sizeof(double), C->s);
  int st = fgmres(C, db, dx, rtol, maxit, iters, final_rel_res);
  cudaMemcpyAsync(x_host, dx, N * sizeof(double), cudaMemcpyDeviceToHost, C->s);
  cudaStreamSynchronize(C->s);
  return finish(C, st);
}

int stokes_get_level_params(const stokes_ctx *C, int level, double *beta_A, double *beta_S, double *sigma,
                            double *tau) {
  if (!C || level < 1 || level >= C->nl) {
    set_error("level out of range (parameters exist on levels >= 1)");
    return STOKES_EINVAL;
  }
  if (beta_A) *beta_A = C->betaA[level];
  if (beta_S) *beta_S = C->betaS[level];
  if (sigma) *sigma = C->sigma;
  if (tau) *tau = C->tau;
  return STOKES_OK;
}

int stokes_get_diagonals(stokes_ctx *C, int level, double *DA, double *DS, void *stream) {
  if (!C || level < 1 || level >= C->nl) {
    set_error("level out of range (diagonals exist on levels >= 1)");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  if (DA) cudaMemcpyAsync(DA, C->DA[level], C->L64[level].d.n_u * sizeof(double), cudaMemcpyDeviceToDevice, C->s);
  if (DS) cudaMemcpyAsync(DS, C->DS[level], C->L64[level].d.n_p * sizeof(double), cudaMemcpyDeviceToDevice, C->s);
  return finish(C, STOKES_OK);
}

int stokes_cell_grad(stokes_ctx *C, const double *u, const double *lam, double *dJ_dmu, void *stream) {
  if (!C || !u || !lam || !dJ_dmu || C->sym) {
    set_error(C && C->sym ? "stokes_cell_grad is the gradient of the Laplacian form; the context uses the "
                            "symmetric-gradient form"
                          : "invalid stokes_cell_grad arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  const LevelDesc<double> &d = C->L64[C->nl - 1].d;
  switch (d.k) {
    case 2: launch_cell_grad_k<2, double>(d, C->tab64, u, lam, dJ_dmu, C->s); break;
    case 3: launch_cell_grad_k<3, double>(d, C->tab64, u, lam, dJ_dmu, C->s); break;
    default: launch_cell_grad_k<4, double>(d, C->tab64, u, lam, dJ_dmu, C->s); break;
  }
  ++C->launches;
  return finish(C, STOKES_OK);
}

int stokes_set_viscosity(stokes_ctx *C, const double *mu_cell, void *stream) {
  if (!C || !mu_cell) {
    set_error("invalid stokes_set_viscosity arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  const long long nc = (long long)C->mesh.n[0] * C->mesh.n[1] * (C->dim == 3 ? C->mesh.n[2] : 1);
  for (long long i = 0; i < nc; ++i)
    if (!(mu_cell[i] > 0)) {
      set_error("mu_cell entries must be positive");
      C->err = g_last_error;
      return STOKES_EINVAL;
    }
  cudaStreamSynchronize((cudaStream_t)stream);
  if (C->s) cudaStreamSynchronize(C->s);
  // rebuild every mu-dependent part (level viscosities, diagonals, eigenvalue estimates,
  // coarse inverse, captured graphs) in a fresh context, then take over its contents
  stokes_ctx *T = nullptr;
  stokes_mesh mesh = C->mesh;
  const int st = stokes_setup(&mesh, C->k, C->mu_const, C->gamma_rho, mu_cell, &C->o, stream, &T);
  if (st != STOKES_OK) {
    C->err = g_last_error;
    return st;
  }
  const long long launches = C->launches;
  std::swap(*C, *T);
  C->launches += launches;
  stokes_destroy(T);
  return STOKES_OK;
}

int stokes_velocity_nodes(stokes_ctx *C, int level, double *xyz, void *stream) {
  if (!check_level(C, level) || !xyz) {
    set_error("invalid stokes_velocity_nodes arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  LevelDesc<double> d = C->L64[level].d;
  // the Cartesian box offset is applied on the host side of the descriptor
  Runner<double> R(C);
  R.vec(k_velocity_nodes, d.nv, d, (const Tab1D<double> *)C->tab64, xyz);
  if (d.cartesian) {
    for (int a = 0; a < C->dim; ++a)
      if (C->mesh.lo[a] != 0.0)
        launch_kernel(k_add_strided, dim3(vec_blocks(d.nv)), dim3(kVecThreads), 0, C->s, xyz + a, (long long)C->dim,
                      C->mesh.lo[a], d.nv);
  }
  return finish(C, STOKES_OK);
}

int stokes_lift_rhs(stokes_ctx *C, const double *uD, double *b, void *stream) {
  if (!C || !uD || !b) {
    set_error("invalid stokes_lift_rhs arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  Runner<double> R(C);
  const int top = C->nl - 1;
  LevelRT<double> &L = C->L64[top];
  const long long nu = L.d.n_u, n = nu + L.d.n_p;
  // kx = [A B^T; B 0] u_D with the Dirichlet values read (rows of constrained DoFs stay zero)
  R.zero(L.kx, n);
  launch_cell_apply<double>(L.d, C->tab64, Runner<double>(C).form(kApplyA | kApplyBT | kApplyB | kApplyUnmasked), uD,
                            uD + nu, L.kx, L.kx + nu, C->s, -1, nullptr, L.rho);
  ++C->launches;
  R.vec(k_axpy<double>, n, b, -1.0, (const double *)L.kx, n);
  R.zero(L.kx, n);
  return finish(C, STOKES_OK);
}

int stokes_mg_iterate(stokes_ctx *C, const double *b, double *x, int max_iter, double reduction, int *iters,
                      double *res_history, double *rate, void *stream) {
  if (!C || !b || !x || max_iter < 0 || !(reduction > 0)) {
    set_error("invalid stokes_mg_iterate arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  det_begin(C, C->s);
  Runner<double> R(C);
  const int top = C->nl - 1;
  LevelRT<double> &L = C->L64[top];
  const long long N = L.d.n_u + L.d.n_p;
  std::vector<double> res;
  auto resnorm = [&](double *out) -> int {
    R.vmult(top, x, C->w, true);
    R.sub(b, C->w, C->w, N);
    double r2;
    int st = dot64(C, C->w, C->w, N, &r2);
    *out = std::sqrt(r2);
    return st;
  };
  double r;
  int st = resnorm(&r);
  if (st) return finish(C, st);
  res.push_back(r);
  int it = 0;
  while (it < max_iter && res.back() > reduction * res[0]) {
    // x <- MG(x, b), FP64 cycle (Algorithm 1 iterated as a stationary method, Sec. 4.1)
    SMF_CUDA_OK(cudaMemcpyAsync(L.b, b, N * sizeof(double), cudaMemcpyDeviceToDevice, C->s));
    SMF_CUDA_OK(cudaMemcpyAsync(L.x, x, N * sizeof(double), cudaMemcpyDeviceToDevice, C->s));
    if ((st = R.top_cycle(false))) return finish(C, st);
    SMF_CUDA_OK(cudaMemcpyAsync(x, L.x, N * sizeof(double), cudaMemcpyDeviceToDevice, C->s));
    if ((st = resnorm(&r))) return finish(C, st);
    res.push_back(r);
    ++it;
    if (!std::isfinite(r) || r > 1e6 * res[0]) {
      set_error("stationary multigrid diverged");
      C->err = g_last_error;
      if (iters) *iters = it;
      return STOKES_EBREAKDOWN;
    }
  }
  if (iters) *iters = it;
  if (res_history)
    for (size_t i = 0; i < res.size(); ++i) res_history[i] = res[i];
  if (rate) *rate = it >= 3 ? std::pow(res[it] / res[it - 3], 1.0 / 3.0) : std::nan("");
  return finish(C, res.back() <= reduction * res[0] ? STOKES_OK : STOKES_ENOTCONV);
}

int stokes_fma_peak(int precision, double *tflops, void *stream) {
  if ((precision != 32 && precision != 64 && precision != 2) || !tflops) {
    set_error("invalid stokes_fma_peak arguments");
    return STOKES_EINVAL;
  }
  int dev = 0, sms = 0;
  SMF_CUDA_OK(cudaGetDevice(&dev));
  SMF_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = (cudaStream_t)stream;
  const int threads = 256, blocks = sms * 8;
  const int iters = precision == 64 ? 100 : 4000;  // about 5-10 ms per launch on GB300
  void *out = nullptr;
  SMF_CUDA_OK(cudaMalloc(&out, (size_t)blocks * threads * 8));
  cudaEvent_t e0, e1;
  SMF_CUDA_OK(cudaEventCreate(&e0));
  SMF_CUDA_OK(cudaEventCreate(&e1));
  auto launch = [&]() {
    if (precision == 32)
      k_fma_peak<float><<<blocks, threads, 0, s>>>((float *)out, iters, 1.0f);
    else if (precision == 2)
      k_fma_peak_x2<<<blocks, threads, 0, s>>>((float *)out, iters, 1.0f);
    else
      k_fma_peak<double><<<blocks, threads, 0, s>>>((double *)out, iters, 1.0);
  };
  launch();  // warm-up
  const int reps = 5;
  SMF_CUDA_OK(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) launch();
  SMF_CUDA_OK(cudaEventRecord(e1, s));
  SMF_CUDA_OK(cudaEventSynchronize(e1));
  float ms = 0.f;
  SMF_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const double fmas = (double)blocks * threads * iters * 16.0 * 8.0 * reps;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return STOKES_OK;
}

int stokes_time_apply(stokes_ctx *C, int level, int precision, int blocks, int reps, double *avg_ms, void *stream) {
  if (!check_level(C, level) || (precision != 32 && precision != 64) || blocks <= 0 || blocks > 15 || reps < 1 ||
      !avg_ms) {
    set_error("invalid stokes_time_apply arguments");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  StreamGuard sg(C, stream);
  det_begin(C, C->s);
  cudaEvent_t e0, e1;
  SMF_CUDA_OK(cudaEventCreate(&e0));
  SMF_CUDA_OK(cudaEventCreate(&e1));
  SMF_CUDA_OK(cudaEventRecord(e0, C->s));
  for (int r = 0; r < reps; ++r) {
    if (precision == 64) {
      LevelRT<double> &R = C->L64[level];
      launch_cell_apply<double>(R.d, C->tab64, Runner<double>(C).form(blocks), R.x, R.x + R.d.n_u, R.r, R.r + R.d.n_u,
                                C->s, R.shape, R.geo, R.rho, C->det ? &C->gb : nullptr);
    } else {
      LevelRT<float> &R = C->L32[level];
      launch_cell_apply<float>(R.d, C->tab32, Runner<float>(C).form(blocks), R.x, R.x + R.d.n_u, R.r, R.r + R.d.n_u,
                               C->s, R.shape, R.geo, R.rho, C->det ? &C->gb : nullptr);
    }
    ++C->launches;
  }
  SMF_CUDA_OK(cudaEventRecord(e1, C->s));
  SMF_CUDA_OK(cudaEventSynchronize(e1));
  float ms = 0.f;
  SMF_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *avg_ms = (double)ms / reps;
  return finish(C, STOKES_OK);
}

int stokes_setup_batch(int n_meshes, const stokes_mesh *meshes, const int *k, const double *mu,
                       const double *gamma_rho, const stokes_opts *opts, void *stream, stokes_batch **out) {
  if (!out || n_meshes < 1 || !meshes || !k || !mu || !gamma_rho) {
    set_error("invalid stokes_setup_batch arguments");
    return STOKES_EINVAL;
  }
  *out = nullptr;
  if (opts && opts->deterministic) {
    set_error("stokes_setup_batch: deterministic mode is for single contexts (its cooperative launches "
              "assume the whole GPU)");
    return STOKES_EINVAL;
  }
  stokes_batch *Bt = new (std::nothrow) stokes_batch();
  if (!Bt) {
    set_error("host allocation failed");
    return STOKES_ENOMEM;
  }
  for (int i = 0; i < n_meshes; ++i) {
    stokes_ctx *C = nullptr;
    const int st = stokes_setup(&meshes[i], k[i], mu[i], gamma_rho[i], nullptr, opts, stream, &C);
    if (st != STOKES_OK) {
      const std::string e = g_last_error;
      stokes_destroy_batch(Bt);
      set_error("batch member " + std::to_string(i) + ": " + e);
      return st;
    }
    Bt->ctx.push_back(C);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&Bt->s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&Bt->fork, cudaEventDisableTiming);
  Bt->join.resize(n_meshes, nullptr);
  for (int i = 0; i < n_meshes && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&Bt->join[i], cudaEventDisableTiming);
  for (int i = 0; i < n_meshes && e == cudaSuccess; ++i) {
    double *h = nullptr;
    e = cudaMallocHost((void **)&h, (size_t)(3 * (Bt->ctx[i]->restart + 2) + 4) * sizeof(double));
    Bt->pinned.push_back(h);
  }
  if (e != cudaSuccess) {
    const int st = cuda_fail(e, "batch streams/events", __FILE__, __LINE__);
    stokes_destroy_batch(Bt);
    return st;
  }
  *out = Bt;
  return STOKES_OK;
}

int stokes_batch_context(stokes_batch *Bt, int mesh, stokes_ctx **ctx) {
  if (!Bt || !ctx || mesh < 0 || mesh >= (int)Bt->ctx.size()) {
    set_error("invalid stokes_batch_context arguments");
    return STOKES_EINVAL;
  }
  *ctx = Bt->ctx[mesh];
  return STOKES_OK;
}

int stokes_solve_batch(stokes_batch *Bt, const double *const *b, double *const *x, double rtol, int maxit, int *iters,
                       double *final_rel_res, void *stream) {
  if (!Bt || !b || !x || !(rtol > 0) || maxit < 0) {
    set_error("invalid stokes_solve_batch arguments");
    if (Bt) Bt->err = g_last_error;
    return STOKES_EINVAL;
  }
  for (size_t i = 0; i < Bt->ctx.size(); ++i)
    if (!b[i] || !x[i]) {
      set_error("null vector in stokes_solve_batch");
      Bt->err = g_last_error;
      return STOKES_EINVAL;
    }
  cudaStream_t user = (cudaStream_t)stream;
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, user);
  for (auto *C : Bt->ctx) cudaStreamWaitEvent(C->s, ev, 0);
  int st = batch_solve(Bt, b, x, rtol, maxit, iters, final_rel_res);
  for (auto *C : Bt->ctx) {
    cudaEventRecord(C->ev_out, C->s);
    cudaStreamWaitEvent(user, C->ev_out, 0);
  }
  cudaEventDestroy(ev);
  if (st == STOKES_OK) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "batch kernels", __FILE__, __LINE__);
  }
  if (st != STOKES_OK) Bt->err = g_last_error;
  return st;
}

const char *stokes_batch_last_error(const stokes_batch *Bt) { return Bt ? Bt->err.c_str() : g_last_error.c_str(); }

void stokes_destroy_batch(stokes_batch *Bt) {
  if (!Bt) return;
  if (Bt->s) cudaStreamSynchronize(Bt->s);
  if (Bt->graph) cudaGraphExecDestroy(Bt->graph);
  if (Bt->kgraph) cudaGraphExecDestroy(Bt->kgraph);
  if (Bt->qmem) cudaFree(Bt->qmem);
  for (auto *C : Bt->ctx) stokes_destroy(C);
  for (auto *h : Bt->pinned)
    if (h) cudaFreeHost(h);
  for (auto e : Bt->join)
    if (e) cudaEventDestroy(e);
  if (Bt->fork) cudaEventDestroy(Bt->fork);
  if (Bt->s) cudaStreamDestroy(Bt->s);
  delete Bt;
}

int stokes_get_geometry_stored(const stokes_ctx *C, int level, int precision, int *stored) {
  if (!C || level < 0 || level >= C->nl || !stored || (precision != 32 && precision != 64)) {
    set_error("invalid stokes_get_geometry_stored arguments");
    return STOKES_EINVAL;
  }
  *stored = (precision == 64 ? C->L64[level].geo != nullptr : C->L32[level].geo != nullptr) ? 1 : 0;
  return STOKES_OK;
}

int stokes_get_launch_shape(const stokes_ctx *C, int level, int precision, int *shape) {
  if (!C || level < 0 || level >= C->nl || !shape || (precision != 32 && precision != 64)) {
    set_error("invalid stokes_get_launch_shape arguments");
    return STOKES_EINVAL;
  }
  *shape = precision == 64 ? C->L64[level].shape : C->L32[level].shape;
  return STOKES_OK;
}

int stokes_get_smoother_fusion(stokes_ctx *C, int level, int precision, int *fused) {
  if (!C || level < 0 || level >= C->nl || !fused || (precision != 32 && precision != 64)) {
    set_error("invalid stokes_get_smoother_fusion arguments");
    return STOKES_EINVAL;
  }
  if (level == 0)
    *fused = 0;
  else if (precision == 64)
    *fused = Runner<double>(C).fused_ok(level) ? 1 : 0;
  else
    *fused = Runner<float>(C).fused_ok(level) ? 1 : 0;
  return STOKES_OK;
}

int stokes_set_launch_shape(stokes_ctx *C, int level, int precision, int shape) {
  if (!C || level < 0 || level >= C->nl || (precision != 32 && precision != 64) ||
      !(shape == 1 || shape == 3 || shape == 4 || shape == -1 || shape == 5)) {
    set_error("invalid stokes_set_launch_shape arguments (shape in {1,3,4,-1,5})");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  if (precision == 64)
    C->L64[level].shape = shape;
  else
    C->L32[level].shape = shape;
  // the shape decides between the fused and the unfused smoother on this level: start from
  // zeroed work vectors
  int st = precision == 64 ? zero_level_work(C, C->L64[level]) : zero_level_work(C, C->L32[level]);
  if (st == STOKES_OK && cudaStreamSynchronize(C->s) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "set_launch_shape", __FILE__, __LINE__);
  if (st != STOKES_OK) {
    C->err = g_last_error;
    return st;
  }
  // captured cycles baked the previous shape in: drop them so the next call recaptures
  drop_graphs(C);
  return STOKES_OK;
}

long long stokes_launch_count(const stokes_ctx *C) { return C ? C->launches : 0; }
int stokes_krylov_mode(const stokes_ctx *C) { return C ? C->kry_mode : -1; }
int stokes_set_wait_cycles(stokes_ctx *C, unsigned int cycles) {
  if (!C || !C->det) {
    set_error("stokes_set_wait_cycles: the context is not in deterministic mode");
    if (C) C->err = g_last_error;
    return STOKES_EINVAL;
  }
  C->o.wait_cycles = cycles;
  SMF_CUDA_OK(cudaMemcpyAsync(C->gb.state + 3, &cycles, sizeof(unsigned), cudaMemcpyHostToDevice, C->s));
  SMF_CUDA_OK(cudaStreamSynchronize(C->s));
  return STOKES_OK;
}
int stokes_batch_krylov_mode(const stokes_batch *Bt) { return Bt ? Bt->kmode : -1; }
int stokes_batch_vcycle(stokes_batch *Bt, const float *const *b, float *const *x, void *stream) {
  if (!Bt || !b || !x) {
    set_error("invalid stokes_batch_vcycle arguments");
    return STOKES_EINVAL;
  }
  const int nm = (int)Bt->ctx.size();
  for (int i = 0; i < nm; ++i)
    if (!b[i] || !x[i]) {
      set_error("null vector in stokes_batch_vcycle");
      return STOKES_EINVAL;
    }
  if (!Bt->qmem && !batch_qrecord(Bt)) {
    set_error("stokes_batch_vcycle: the work-queue form does not serve this batch (every member 3D, k = 2, FP32 "
              "cycle, no stabilisation, symmetric gradient or rho term)");
    return STOKES_EINVAL;
  }
  cudaStream_t user = (cudaStream_t)stream;
  SMF_CUDA_OK(cudaEventRecord(Bt->fork, user));
  SMF_CUDA_OK(cudaStreamWaitEvent(Bt->s, Bt->fork, 0));
  for (int i = 0; i < nm; ++i) {
    stokes_ctx *C = Bt->ctx[i];
    const int top = C->nl - 1;
    const long long n = C->L32[top].d.n_u + C->L32[top].d.n_p;
    SMF_CUDA_OK(cudaMemcpyAsync(C->L32[top].b, b[i], n * sizeof(float), cudaMemcpyDeviceToDevice, Bt->s));
    SMF_CUDA_OK(cudaMemsetAsync(C->L32[top].x, 0, n * sizeof(float), Bt->s));
  }
  PqRun R = Bt->qrun;
  R.active = nullptr;  // every member
  SMF_CUDA_OK(cudaMemsetAsync(R.state, 0, sizeof(unsigned) * (4 + R.nops), Bt->s));
  const int e = launch_queue(R, Bt->qsmem, Bt->s);
  if (e) return cuda_fail((cudaError_t)e, "launch_queue", __FILE__, __LINE__);
  for (int i = 0; i < nm; ++i) {
    stokes_ctx *C = Bt->ctx[i];
    const int top = C->nl - 1;
    const long long n = C->L32[top].d.n_u + C->L32[top].d.n_p;
    SMF_CUDA_OK(cudaMemcpyAsync(x[i], C->L32[top].x, n * sizeof(float), cudaMemcpyDeviceToDevice, Bt->s));
  }
  unsigned qerr = 0;
  SMF_CUDA_OK(cudaMemcpyAsync(&qerr, R.state + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, Bt->s));
  SMF_CUDA_OK(cudaStreamSynchronize(Bt->s));
  if (qerr) {
    set_error("batched work-queue kernel: a dependency wait exceeded its budget");
    return STOKES_ETIMEOUT;
  }
  return STOKES_OK;
}
int stokes_batch_set_wait_cycles(stokes_batch *Bt, unsigned int cycles) {
  if (!Bt) {
    set_error("invalid stokes_batch_set_wait_cycles arguments");
    return STOKES_EINVAL;
  }
  Bt->qbudget = cycles;
  if (Bt->qmem) {
    SMF_CUDA_OK(cudaMemcpyAsync(Bt->qrun.state + 4 + Bt->qrun.nops, &cycles, sizeof(unsigned), cudaMemcpyHostToDevice,
                                Bt->s));
    SMF_CUDA_OK(cudaStreamSynchronize(Bt->s));
  }
  return STOKES_OK;
}

const char *stokes_last_error(const stokes_ctx *C) { return C ? C->err.c_str() : g_last_error.c_str(); }
const char *stokes_global_last_error(void) { return g_last_error.c_str(); }

void stokes_destroy(stokes_ctx *C) {
  if (!C) return;
  if (C->s) cudaStreamSynchronize(C->s);
  drop_graphs(C);
  for (void *p : C->allocs) cudaFree(p);
  if (C->ev_in) cudaEventDestroy(C->ev_in);
  if (C->ev_out) cudaEventDestroy(C->ev_out);
  if (C->s) cudaStreamDestroy(C->s);
  delete C;
}

}  // extern "C"
