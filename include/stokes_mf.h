/*
 * stokes_mf.h -- C ABI of the GB300 matrix-free monolithic multigrid library for
 * Q_k-Q_{k-1} Taylor-Hood discretisations of the (generalized) Stokes system
 *
 *     [ A  B^T ] [u]   [f]        a(u,v) = int mu grad u : grad v + gamma*rho u.v
 *     [ B  -C  ] [p] = [g],       b(v,q) = -int q div v,   C = 0
 *
 * (paper Sec. 1, Eq. LinearSystem; Sec. 2, Eqs. a(u,v), b(v,q), Kx=f).
 *
 * Conventions shared by every entry point:
 *  - Meshes are structured boxes of n[0] x n[1] (x n[2]) quadrilateral / hexahedral
 *    cells; level l of the hierarchy has n / 2^(L-l) cells per direction (Sec. 3.1).
 *    Cells are bi/trilinear images of (0,1)^d (Sec. 2).
 *  - Vector layout (every vector argument): [u_1 | ... | u_d | p]; each velocity
 *    component is lexicographic over the (k n_x + 1) x (k n_y + 1) (x (k n_z + 1))
 *    node lattice with x fastest, the pressure over the ((k-1) n + 1)^d lattice.
 *    Nodes are the tensor-product Gauss-Lobatto points of each cell.
 *  - Dirichlet velocity DoFs stay in the vector; their rows and columns of K are
 *    the identity.  Right-hand sides must be zero there (lift inhomogeneous data).
 *  - Vector pointers are DEVICE pointers owned by the caller unless the entry point
 *    says HOST.  precision = 64 means double*, 32 means float*.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *    are stream-ordered and asynchronous unless they return host scalars.
 *  - Every call returns a status; on error, stokes_last_error(ctx) (or
 *    stokes_global_last_error() when no context exists) holds a message.  No C++
 *    exception crosses this boundary.  A context is not thread-safe.
 *
 * Environment variables (read at setup or at the first use; they choose among forms of the same
 * arithmetic, so none changes a result beyond rounding order):
 *  - STOKES_NO_AUTOTUNE=1: no setup timing; default launch shapes, fused smoothing where eligible,
 *    per-point geometry evaluated by the FP32 kernels.
 *  - STOKES_TUNING="s32=..;s64=..;f32=..;f64=..[;g32=..]": the setup's choices pinned (see
 *    stokes_get_launch_shape).
 *  - STOKES_NO_FUSE=1: unfused smoothing everywhere.  STOKES_NO_GRAPHS=1: no CUDA-graph capture.
 *  - STOKES_HOST_KRYLOV=1: the FGMRES iterations driven from the host (stokes_krylov_mode).
 *  - STOKES_BATCH_QUEUE=1: the batch's FP32 cycles in the persistent work-queue kernel.
 *  - STOKES_GEO=none: no stored per-point geometry (stokes_get_geometry_stored).
 *    STOKES_C_MATRIX=none: the stabilisation block C on the fly instead of stored element matrices.
 *  - STOKES_NO_PDL=1: no programmatic dependent launch; STOKES_PDL=all: PDL inside captured graphs
 *    too (off there by default).  STOKES_GENERIC_KERNEL=1: every 3D application in the
 *    point-per-thread kernel (for comparisons).
 */
#ifndef STOKES_MF_H
#define STOKES_MF_H

#ifdef __cplusplus
extern "C" {
#endif

#define STOKES_MAX_LEVELS 12

typedef enum {
  STOKES_OK = 0,
  STOKES_EINVAL = 1,      /* bad argument (sizes, k, null pointers, unknown option) */
  STOKES_ENOMEM = 2,      /* device allocation failed */
  STOKES_ECUDA = 3,       /* a CUDA call failed */
  STOKES_ENOTCONV = 4,    /* iteration limit reached before the tolerance */
  STOKES_EBREAKDOWN = 5,  /* NaN/Inf or residual growth > 1e6 r0 detected */
  STOKES_ETIMEOUT = 6     /* a bounded device-side wait expired */
} stokes_status;

typedef struct stokes_ctx stokes_ctx;
typedef struct stokes_batch stokes_batch;

/* Mesh of the finest level.  vertices (HOST, nullable): (n+1)^d vertex coordinates,
 * x fastest, coordinates interleaved ((n_z+1)(n_y+1)(n_x+1) x d doubles); coarse
 * levels use every 2^(L-l)-th vertex.  NULL = the Cartesian box [lo, hi].
 * dirichlet_faces: bit 2a = face x_a = lo, bit 2a+1 = face x_a = hi; other faces
 * carry the natural (do-nothing) condition.  0x3F (3D) / 0xF (2D) = all faces. */
typedef struct {
  int dim;
  int n[3];
  int n_levels;
  double lo[3];
  double hi[3];
  const double *vertices;
  unsigned int dirichlet_faces;
} stokes_mesh;

/* Smoother and solver options (Algorithm 2 inputs k_A, k_S; Sec. 4.1 knobs). */
typedef struct {
  int kA;               /* Chebyshev degree of A^-1_hat (number of A applications) */
  int kS;               /* Chebyshev degree of S^-1_hat */
  int m;                /* pre- and post-smoothing steps */
  int cycle;            /* 0 = V-cycle, 1 = W-cycle (Algorithm 1, gamma = 1 / 2) */
  int schur_diag;       /* D_S~ of the pressure Chebyshev (Algorithm 2): 0 = local diagonal (Eq. diag loc),
                           1 = pressure mass (Eq. diag p), 2 = diag(B D_A^-1 B^T) (Eq. diag d),
                           3 = exact diag(B A^-1_hat B^T) (small meshes only: setup fails with
                           STOKES_EINVAL when it needs more than 4096 probes) */
  int vcycle_fp32;      /* 1: stokes_solve preconditions with the FP32 cycle, 0: FP64 */
  int gmres_restart;    /* FGMRES restart length */
  int eig_iters;        /* Lanczos steps for lambda_max estimates */
  double eig_safety;    /* beta = eig_safety * Lanczos estimate */
  unsigned long long seed; /* SplitMix64 seed of the Lanczos start vectors */
  double c_mass;        /* stabilisation block C of K = [A B^T; B -C] (Sec. 1 leaves C open; zero by
                           default): c(p,q) = c_mass int p q + c_grad sum_tau h_tau^2 int_tau
                           grad p . grad q, h_tau = |tau|^(1/d); both >= 0.  With c_mass > 0 the
                           constant pressure is no longer in the kernel of K (no zero-mean fixing).
                           Where the pressure space has at most 27 nodes per cell (k <= 3 in 3D, any k
                           in 2D) setup stores C's packed symmetric element matrices on the device
                           (k^d (k^d + 1) / 2 entries per cell: 36 for k = 2, 378 for k = 3 in
                           3D; FP64 and FP32 copies); otherwise, and with the environment variable
                           STOKES_C_MATRIX=none, C is evaluated on the fly */
  double c_grad;
  int sym_grad;         /* 1: a(u,v) = int mu eps(u):eps(v) + gamma rho u.v, the symmetric-gradient form of
                           Sec. 2 (eps(u) = (grad u + grad u^T)/2); 0: int mu grad u:grad v + gamma rho u.v */
  const double *rho_cell; /* HOST, nullable: per-cell rho of the gamma rho u.v term on the finest level
                           (n cells, x fastest; copied at setup; coarse levels take the mean of the
                           2^d children); null: rho = 1.  Entries must be > 0 */
  int deterministic;    /* bitwise-reproducible operator applications (no atomic scatter; the smoother is
                           the unfused one).  1 (owner-computes): every cell-kernel application is two
                           launches, the cell-component kernel storing each cell's local results
                           (K_tau P_tau^T x of the paper's K x = sum_tau P_tau K_tau P_tau^T x) and a
                           per-DoF pass summing the results of the cells that hold the DoF in a fixed
                           order.  2 (colour classes): one cooperative launch walks the 8 classes of
                           cells with equal index parities (no two cells of a class share a node) with
                           a grid barrier between classes and scatters by plain read-modify-write.
                           3D, k = 2 (any mesh) or k = 3 (Cartesian), Laplacian form, constant rho,
                           C = 0 (else STOKES_EINVAL); 0: atomic scatter */
  unsigned int wait_cycles; /* deterministic mode 2: clock64() cycles a CTA waits at a grid barrier
                           before it gives up, flags the error and returns (0: 2^31, about 1 s); calls
                           then return STOKES_ETIMEOUT */
} stokes_opts;

/* Fill *o with kA = kS = 3, m = 2, V-cycle, local Schur diagonal, FP32 cycle,
 * restart 30, 40 Lanczos steps, safety 1.1, seed 0x5EED, no stabilisation, the Laplacian form,
 * atomic (not deterministic) scatter: the smoother of Sec. 3.3.1 at one of the settings the paper
 * sweeps (Sec. 4.3-4.5; its runs use the W-cycle of Sec. 4.1, opts.cycle = 1).  A null o is
 * ignored. */
void stokes_default_opts(stokes_opts *o);

/* Build the level hierarchy, geometry, 1D tables, Jacobi/Schur diagonals, the
 * lambda_max estimates (Lanczos, FP64), sigma/tau (Lemma 1) and the factorised
 * coarse matrix (Sec. 3.1-3.3, Algorithm 2).  k in {2,3,4}; dim in {2,3}; every
 * n[a] divisible by 2^(n_levels-1); mu > 0, gamma_rho >= 0.  mu_cell (HOST,
 * nullable): per-cell viscosity of the finest level (n_cells doubles, x fastest);
 * coarse cells take the mean of their 2^d children.  Synchronises the stream.
 * On success *out owns all device memory until stokes_destroy.  STOKES_EINVAL (before any device
 * work) for sizes or coefficients out of range, non-positive mu_cell entries, non-finite vertex
 * coordinates, or a cell whose map is not a proper image of the reference cell (det J <= 0 at a
 * corner, from the cell's edges there). */
int stokes_setup(const stokes_mesh *mesh, int k, double mu, double gamma_rho,
                 const double *mu_cell, const stokes_opts *opts, void *stream,
                 stokes_ctx **out);

/* Sizes of level `level` (0 = coarsest, n_levels-1 = finest): n_u = dim x the velocity nodes of
 * the Q_k lattice, n_p = the Q_{k-1} pressure nodes (Sec. 2; Dirichlet DoFs included, as in the
 * paper's DoF counts).  HOST outputs (nullable); STOKES_EINVAL for a null context or a level out
 * of range. */
int stokes_sizes(const stokes_ctx *ctx, int level, long long *n_u, long long *n_p);

/* y = K x on `level` (Sec. 3.1: Kx = sum_tau P_tau K_tau P_tau^T x by sum
 * factorisation; K = [A B^T; B -C], C = 0 unless opts.c_mass / c_grad are set).  x, y: device
 * vectors of n_u + n_p entries; must not alias.  Launched on `stream` itself. */
int stokes_vmult(stokes_ctx *ctx, int level, int precision, const void *x, void *y, void *stream);

/* Block applications on `level`: blocks is a bit set of 1 = A u, 2 = B^T p (both into
 * yu), 4 = B u (into yp); or exactly 8 = Z M_v u (velocity mass, constrained rows zero, every
 * entry of u read) or 16 = M_v Z u (its transpose: constrained entries of u read as 0, every
 * row written), Z = identity on free velocity DoFs, 0 on constrained ones.  Bit 64 adds -C p
 * to yp (the stabilisation block; with bit 4, yp = B u - C p; not with 8 / 16).  Outputs are
 * overwritten; unused pointers may be NULL.  For blocks 1-7, rows of constrained velocity DoFs
 * of yu are zero (no identity term) and constrained entries of u are ignored.  The blocks are the
 * forms a(u, v), b(v, q) and c(p, q) of Sec. 2 applied as in Sec. 3.1.  Device vectors in the
 * precision given; STOKES_EINVAL for an unknown bit set. */
int stokes_apply_blocks(stokes_ctx *ctx, int level, int precision, int blocks, const void *u,
                        const void *p, void *yu, void *yp, void *stream);

/* b = [Z M_v f ; 0]: right-hand side of a forcing given by its velocity nodal values
 * f (n_u entries).  Constrained rows are zero.  The load (f, v) of Sec. 2 for an f interpolated
 * at the velocity nodes; f and b are device vectors in the precision given (b: n_u + n_p). */
int stokes_mass_rhs(stokes_ctx *ctx, int level, int precision, const void *f, void *b, void *stream);

/* `steps` steps of the inexact symmetric Uzawa smoother in compact form
 * x <- x + K_hat^{-1}(b - K x) (Sec. 3.3.1) on a level >= 1; x in/out. */
int stokes_smooth(stokes_ctx *ctx, int level, int precision, int steps, const void *b, void *x,
                  void *stream);

/* stokes_smooth without any device allocation.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory at the point of the call -- code that
 * runs under stream capture, real-time or latency-critical loops, or applications whose own
 * allocator owns all device memory.  Every work vector of the smoother lives in one static device
 * array of 16 MiB compiled into the library (present on every GPU that loads it, until exit); a
 * level needing more (11 velocity + 6 pressure work vectors, each padded to 64 entries, in the
 * given precision) is rejected with STOKES_EINVAL and a message.  The context, b and x are as for
 * stokes_smooth and must exist already; the call performs no cudaMalloc/cudaFree and calls no
 * allocating library routine.  The array is shared by all calls and keeps the last call's
 * contents (the used part is cleared at the start of each call): calls that overlap on the GPU --
 * different streams, contexts or host threads -- race on it.  The array's device address is looked
 * up once per device (in stokes_setup, or by the first call on a device that had no setup); make
 * that first call before any stream capture.  Call it with the context's device current (the one
 * current at stokes_setup): the array has one instance per device, and another device's instance
 * is rejected with STOKES_EINVAL. */
int stokes_smooth_noalloc(stokes_ctx *ctx, int level, int precision, int steps, const void *b,
                          void *x, void *stream);

/* Grid transfer between fine_level and fine_level-1 (Sec. 3.2): direction 0 =
 * restriction out = P^T in (fine -> coarse), 1 = prolongation out = P in (coarse ->
 * fine).  Constrained velocity DoFs are removed on both sides. */
int stokes_transfer(stokes_ctx *ctx, int fine_level, int precision, int direction, const void *in,
                    void *out, void *stream);

/* Coarse direct solve on level 0 (Sec. 4.1): x = K_0^{-1} b; under full Dirichlet
 * data the bordered system fixes sum(p) = 0. */
int stokes_coarse_solve(stokes_ctx *ctx, int precision, const void *b, void *x, void *stream);

/* One multigrid cycle on the finest level, x <- MG(x, b) (Algorithm 1). */
int mg_vcycle(stokes_ctx *ctx, int precision, const void *b, void *x, void *stream);

/* FP64 flexible GMRES on the finest level, right-preconditioned by one cycle per
 * iteration (FP32 or FP64 per opts.vcycle_fp32), from the initial guess in x, to
 * ||b - K x||_2 <= rtol ||b||_2.  b, x: device double vectors.  Synchronises the
 * stream.  Under full Dirichlet data the returned pressure has zero mean.
 * iters, final_rel_res: HOST outputs (nullable).  STOKES_ENOTCONV after maxit, STOKES_EBREAKDOWN
 * on a non-finite residual, STOKES_EINVAL for rtol <= 0 or maxit < 0.  The outer loop is a layer
 * on the paper's method (it iterates the cycle as a stationary method, Sec. 4.1; Algorithm 1 is
 * the preconditioner here). */
int stokes_solve(stokes_ctx *ctx, const double *b, double *x, double rtol, int maxit, int *iters,
                 double *final_rel_res, void *stream);

/* Where stokes_solve and stokes_solve_batch run the inner FGMRES iterations: 1 = on the device
 * (the Hessenberg update, Givens rotations and the stopping test run in a kernel; the iterations
 * of one restart cycle are one CUDA-graph launch with a conditional while node, and the host
 * synchronises once per restart cycle), 0 = host-driven (one synchronisation per iteration;
 * STOKES_HOST_KRYLOV=1, STOKES_NO_GRAPHS=1, or conditional graph nodes refused by the runtime),
 * -1 = not decided yet (no solve so far, or a null context).  No counterpart in the paper (the
 * outer Krylov loop is a layer on top of its Algorithm 1). */
int stokes_krylov_mode(const stokes_ctx *ctx);

/* Deterministic mode (opts.deterministic): replace the grid-barrier wait budget of opts.wait_cycles
 * (clock64() cycles; 0 = 2^31).  Synchronises the context stream; STOKES_EINVAL for a context not in
 * deterministic mode.  No counterpart in the paper. */
int stokes_set_wait_cycles(stokes_ctx *ctx, unsigned int cycles);

/* Where stokes_solve_batch runs: 1 = device iterations, one while node per member as independent
 * graph branches; 2 = device iterations in lockstep with the members' FP32 cycles run by ONE
 * persistent work-queue kernel per iteration (STOKES_BATCH_QUEUE=1 at the first solve; every
 * member 3D, k = 2, FP32 cycle, no stabilisation / symmetric gradient / rho term; otherwise 1):
 * each cycle is recorded once as its operation list (cell-kernel applications, Chebyshev-Jacobi
 * vector steps, restriction with the residual, prolongation, coarse solve), split into work items
 * (bricks of 160 cells, ranges of DoFs), and the kernel's CTAs take items from one queue (a list
 * schedule: each operation at the time it could start were its member alone), each waiting until
 * the member's previous operation has finished; 0 =
 * host-driven lockstep; -1 = no solve yet (or a null batch).  No counterpart in the paper (a layer
 * on Algorithm 1). */
int stokes_batch_krylov_mode(const stokes_batch *batch);

/* Work-queue mode (2): the budget of every dependency wait in clock64() cycles (0 = 2^31, about a
 * second); a wait that runs out ends the launch, and stokes_solve_batch returns STOKES_ETIMEOUT
 * (the batch stays usable).  Stored for a later build of the queue if called before the first
 * solve; synchronises.  No counterpart in the paper. */
int stokes_batch_set_wait_cycles(stokes_batch *batch, unsigned int cycles);

/* One FP32 cycle (Algorithm 1, from x = 0) of every member in ONE launch of the persistent
 * work-queue kernel: b[i] / x[i] are device float vectors of member i (right-hand side in,
 * cycle result out).  Builds the queue on first use; STOKES_EINVAL where the work-queue form does
 * not serve the batch (see stokes_batch_krylov_mode), STOKES_ETIMEOUT when a dependency wait ran
 * out.  Synchronises the stream.  No counterpart in the paper (the batch layer). */
int stokes_batch_vcycle(stokes_batch *batch, const float *const *b, float *const *x, void *stream);

/* stokes_solve with HOST vectors: copies b in, solves from x = 0, copies x out (pinned or
 * pageable host memory of n_u + n_p doubles each; the copies are ordered after the work already
 * on `stream` and the call returns with x_host written).  Same arguments checks and status codes
 * as stokes_solve.  No counterpart in the paper (an end-to-end entry point). */
int stokes_solve_host(stokes_ctx *ctx, const double *b_host, double *x_host, double rtol, int maxit,
                      int *iters, double *final_rel_res, void *stream);

/* Replace the per-cell viscosity of the finest level (HOST, n_cells positive doubles, x
 * fastest) and rebuild everything that depends on it (coarse viscosities = mean of the 2^d
 * children, diagonals, lambda_max estimates, coarse inverse).  Synchronises the stream; the
 * context pointer stays valid.  No counterpart in the paper (the paper's mu is constant). */
int stokes_set_viscosity(stokes_ctx *ctx, const double *mu_cell, void *stream);

/* Adjoint viscosity gradient on the finest level: dJ_dmu[c] = - sum over velocity components of
 * int_c grad lam_i . grad u_i dx, i.e. -lam^T (dK/dmu_c) u, for the solution u of K(mu) u = b
 * and the adjoint lam of K lam = dJ/du (K is symmetric).  u, lam: device double vectors of
 * n_u + n_p entries (velocity part used; constrained entries read as 0); dJ_dmu: device, n_cells
 * doubles (x fastest).  No counterpart in the paper (constant mu there).  Laplacian form only:
 * STOKES_EINVAL for a context of the symmetric-gradient form. */
int stokes_cell_grad(stokes_ctx *ctx, const double *u, const double *lam, double *dJ_dmu, void *stream);

/* Physical coordinates of the velocity nodes of `level` (the Gauss-Lobatto nodes of every cell
 * mapped by its bi/trilinear map), for building nodal data (forcing, Dirichlet values): xyz is a
 * device array of nv x dim doubles, interleaved, in the lattice order of one velocity component
 * (nv = n_u / dim).  The node placement of reading R8 (Sec. 2 leaves it to Fig. 1): Gauss-Lobatto
 * nodes per cell. */
int stokes_velocity_nodes(stokes_ctx *ctx, int level, double *xyz, void *stream);

/* Lifting of inhomogeneous Dirichlet data on the finest level: b -= Z K_full u_D, where uD
 * (device, n_u + n_p doubles) holds the Dirichlet values on constrained velocity DoFs (zero
 * elsewhere) and K_full reads them (Z zeroes the rows of constrained DoFs).  Solving K x0 = b
 * and adding uD gives the solution with u = u_D on the Dirichlet faces (Sec. 1: nonzero u_D in
 * the paper's experiments). */
int stokes_lift_rhs(stokes_ctx *ctx, const double *uD, double *b, void *stream);

/* The paper's solver driver (Sec. 4.1): x <- MG(x, b) iterated as a stationary method with the
 * FP64 cycle of opts (V or W), from the x given, until ||b - K x||_2 <= reduction ||b - K x0||_2
 * or max_iter cycles.  HOST outputs (nullable): iters, res_history (max_iter + 1 entries: the
 * residual norms r^0..r^iters), rate = q = (r^j / r^{j-3})^{1/3} at the last cycle j (NaN if
 * j < 3).  STOKES_ENOTCONV if the reduction was not reached, STOKES_EBREAKDOWN on divergence. */
int stokes_mg_iterate(stokes_ctx *ctx, const double *b, double *x, int max_iter, double reduction,
                      int *iters, double *res_history, double *rate, void *stream);

/* Smoother parameters of a level >= 1 (Algorithm 2): beta of D_A^-1 A and of
 * D_S^-1 S_tilde (safety factor included), sigma and tau (Lemma 1).  HOST outputs. */
int stokes_get_level_params(const stokes_ctx *ctx, int level, double *beta_A, double *beta_S,
                            double *sigma, double *tau);

/* Copy the FP64 Jacobi diagonal D_A (n_u) and the Schur diagonal approximation
 * D_S (n_p) of a level into device buffers (either may be NULL): the diagonals of Sec. 3.3.1 that
 * Algorithm 2 computes (D_S by opts.schur_diag: loc, p, d or exact).  STOKES_EINVAL for level 0
 * (no smoother there) or a level out of range. */
int stokes_get_diagonals(stokes_ctx *ctx, int level, double *DA, double *DS, void *stream);

/* Measurement helper: launch the cell kernel of `blocks` (as in stokes_apply_blocks) on
 * `level` reps times back to back on the library's internal stream, between two CUDA
 * events recorded on that stream, using internal buffers as input and output (no
 * allocation, no memset between launches).  *avg_ms (HOST) = elapsed / reps.
 * Synchronises the stream.  No counterpart in the paper (measurement); STOKES_EINVAL for reps < 1
 * or an unknown bit set. */
int stokes_time_apply(stokes_ctx *ctx, int level, int precision, int blocks, int reps, double *avg_ms,
                      void *stream);

/* Measurement helper (no counterpart in the paper): FMA throughput of the current device in
 * `precision` (32 or 64; 2: FP32 in packed pairs, one paired multiply-add instruction per two
 * FMAs), from 5 launches of a kernel running 8 independent multiply-add chains per thread on
 * 8 x 256-thread CTAs per SM, timed by CUDA events on `stream` (NULL: the legacy default stream);
 * *tflops (HOST) = 2 x FMAs / elapsed / 1e12.  No context; allocates and frees a small output
 * buffer; synchronises the stream.  STOKES_EINVAL on a bad precision or a NULL output. */
int stokes_fma_peak(int precision, double *tflops, void *stream);

/* Batched solves of independent meshes (no counterpart in the paper; a layer on its method).
 * stokes_setup_batch builds one context per mesh (meshes[i], k[i], mu[i], gamma_rho[i], shared
 * opts; every mesh with its own hierarchy and coarse level).  Synchronises the stream. */
int stokes_setup_batch(int n_meshes, const stokes_mesh *meshes, const int *k, const double *mu,
                       const double *gamma_rho, const stokes_opts *opts, void *stream,
                       stokes_batch **out);

/* The context of batch member `mesh` (owned by the batch; for sizes, right-hand sides, vmult):
 * *ctx is valid until stokes_destroy_batch and must not be destroyed by the caller.  STOKES_EINVAL
 * for an index out of range.  No counterpart in the paper (the batch layer). */
int stokes_batch_context(stokes_batch *batch, int mesh, stokes_ctx **ctx);

/* Solve every member: b[i], x[i] are device double vectors of member i (x[i] = initial guess
 * in, solution out).  FP64 FGMRES of every member; with the iterations on the device
 * (stokes_batch_krylov_mode 1) one restart cycle of all members is one CUDA-graph launch holding
 * one conditional while node per member as independent branches, so each member iterates to its
 * own stopping test without waiting for the others; in mode 2 the members' FP32 cycles of an
 * iteration are one persistent work-queue kernel; host-driven (mode 0), the members advance in
 * lockstep, the FP32 cycles of one iteration of all members as one graph launch.  iters,
 * final_rel_res: HOST arrays of n_meshes entries (nullable).  Synchronises the stream.  Returns
 * the first non-OK member status (STOKES_ENOTCONV / STOKES_EBREAKDOWN), or STOKES_ETIMEOUT when a
 * work-queue wait ran out.  No counterpart in the paper (the batch layer). */
int stokes_solve_batch(stokes_batch *batch, const double *const *b, double *const *x, double rtol,
                       int maxit, int *iters, double *final_rel_res, void *stream);

/* Text of the batch's last error (see stokes_last_error), and the release of the batch with every
 * member context and its device memory (a null batch is ignored).  No counterpart in the paper. */
const char *stokes_batch_last_error(const stokes_batch *batch);
void stokes_destroy_batch(stokes_batch *batch);

/* Launch shape of the 3D cell kernel that setup's autotuner chose for `level` and `precision`:
 * 1 or 4 = column kernel with that many warps per CTA, 3 = column kernel with the three velocity
 * components on the three warps of a CTA (shorter per-warp chain for small levels), -1 =
 * point-per-thread kernel, 5 = cell-component kernel (one thread per cell and velocity component,
 * the component's whole tensor in registers; 3D Cartesian levels with k = 2, 3 and FP32 trilinear
 * levels with k = 2, the Laplacian form with a constant rho; other applications on such a level run
 * in the 4-warp column kernel), 0 = not tuned (2D, or STOKES_NO_AUTOTUNE=1).  The environment variable
 * STOKES_TUNING="s32=..;s64=..;f32=..;f64=..[;g32=..]" (comma lists, one value per level, coarsest first)
 * replaces the setup's timings of shapes and smoother forms, e.g. to profile the configuration a
 * plain run chose (a profiler changes the timings); malformed values make setup fail with
 * STOKES_EINVAL.  HOST output.  No counterpart in the paper (a launch choice of this library). */
int stokes_get_launch_shape(const stokes_ctx *ctx, int level, int precision, int *shape);

/* 1 if the column kernels of `level` in `precision` (32 or 64) read the per-point geometry (G,
 * w adj(J), w det J per Gauss point with mu and gamma rho folded in; 3D trilinear levels) stored at
 * setup, 0 if they evaluate it on the fly.  FP64: stored unless the level is Cartesian,
 * STOKES_GEO=none, or the level is larger than the budget (1/16 of the device memory, and at most
 * half of the memory free at setup).  FP32: stored for levels of at most 32^3 cells and read where
 * the setup's timing of the column kernel keeps it (STOKES_TUNING's g32 list otherwise; 0 without
 * autotuning), released at setup where it is not kept; STOKES_GEO=none stores neither precision.
 * The cell-component kernel (shape 5) evaluates the FP32 geometry itself either way.  The geometry
 * is that of the cells' bi/trilinear maps T_tau (Sec. 2) at the Gauss points.  HOST output;
 * STOKES_EINVAL for a level out of range or a precision other than 32 / 64. */
int stokes_get_geometry_stored(const stokes_ctx *ctx, int level, int precision, int *stored);

/* 1 if smoothing on `level` / `precision` runs in the fused form (k_A = 1, 3D, column kernel: the
 * Chebyshev-Jacobi and Uzawa vector updates of Sec. 3.3.1 evaluated inside the cell-kernel
 * gathers, 5 + 3 k_S launches per step), 0 if in the unfused form (separate vector kernels).
 * Setup times both forms per level and keeps the faster (STOKES_NO_AUTOTUNE=1: fused wherever
 * eligible; STOKES_NO_FUSE=1: never).  Level 0 (direct solve) reports 0.  HOST output. */
int stokes_get_smoother_fusion(stokes_ctx *ctx, int level, int precision, int *fused);

/* Override the launch shape of `level` / `precision` (values as above; 0 is not accepted).
 * Captured cycle graphs of the context are dropped and recaptured on next use.  No counterpart in
 * the paper (a launch choice); STOKES_EINVAL for a shape outside {1, 3, 4, -1, 5} (a shape the
 * level's kernels do not serve falls back to the 4-warp column kernel where it applies). */
int stokes_set_launch_shape(stokes_ctx *ctx, int level, int precision, int shape);

/* Number of kernel launches this context issued since setup (a counter kept by the
 * library for reporting; not thread-safe; graph-replayed kernels included; 0 for a null context).
 * No counterpart in the paper. */
long long stokes_launch_count(const stokes_ctx *ctx);

/* Text of the last error of a context (of the calling thread's last call with no usable context,
 * such as a failed setup or a null handle, when ctx is null; stokes_batch_last_error likewise for a
 * batch).  The pointer stays valid until the next call on the same context or thread.  HOST.
 * stokes_destroy releases a context and all its device memory (a null context is ignored).  No
 * counterpart in the paper. */
const char *stokes_last_error(const stokes_ctx *ctx);
const char *stokes_global_last_error(void);
void stokes_destroy(stokes_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* STOKES_MF_H */
