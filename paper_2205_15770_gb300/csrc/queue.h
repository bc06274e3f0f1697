// Persistent work-queue form of the batched FP32 V-cycle (a layer on Algorithm 1 for many
// independent meshes): the cycle of every batch member is recorded once as its list of
// operations (cell-kernel applications, Chebyshev-Jacobi vector steps, restriction with the
// residual, prolongation, coarse solve), each split into work items (bricks of cells or ranges of
// DoFs).  One kernel launch then runs the V-cycles of all members: its CTAs take work items from
// one global queue in order, and an item starts once every item of the member's previous
// operation has finished (a per-operation completion counter; bounded wait).
#pragma once
#include "common.cuh"
#include "transfer.cuh"

namespace smf {

enum PqType : int { kPqCell = 1, kPqChebInit = 2, kPqChebStep = 3, kPqRestrict = 4, kPqProlong = 5, kPqCoarse = 6 };

constexpr int kPqThreads = 128;       // 4 warps per CTA
constexpr int kPqGroupsPerWarp = 4;   // cell operations: 4 cell-component groups of 10 cells per warp
constexpr int kPqCellsPerItem = 160;  //   (160 cells per item)
constexpr int kPqVecPerItem = 4096;   // Chebyshev vector steps: 32 entries per thread
constexpr int kPqRestrictPerItem = 512;  // restriction: 4 coarse DoFs per thread
constexpr int kPqProlongPerItem = 2048;  // prolongation: 16 fine DoFs per thread
constexpr int kPqCoarsePerItem = 16;     // coarse solve: 4 rows per warp
constexpr int kPqSmemSegments = 4096;    // segment starts kept in shared memory up to this count

// One recorded operation of a member's cycle.  Pointer and scalar slots by type:
//   cell:       in = {u, p}, out = {yu, yp}, mode = block bit set
//   cheb init:  in = {a, b, Dinv, base}, out = {r_out, d, x, final_out, acc_out, za, zb},
//               sc = {sr, c0, fscale}
//   cheb step:  in = {r, Dinv, base}, out = {t, d, x, final_out, acc_out}, sc = {c1, c2, fscale}
//   restrict:   in = {fine in, minus (may be null)}, out = {coarse out, zero_c}; F fine, Cd coarse
//   prolong:    in = {coarse in}, out = {fine out, z0, z1, zf}, add
//   coarse:     in = {b}, out = {x}, Kinv, n0
struct PqOp {
  int type = 0, mode = 0, member = 0, W = 0;
  long long items = 0, n = 0;
  LevelDesc<float> F{}, Cd{};
  XferTabs<float> X{};
  const float *in[4] = {};
  float *out[7] = {};
  float sc[3] = {};
  int add = 0, n0 = 0;
  int vec4 = 0;  // Chebyshev steps: every vector 16-byte aligned (packs of 4)
  const double *Kinv = nullptr;
};

// The queue of one launch: segments (one per member operation, in a list-schedule order in which
// every operation follows its member's previous one) hold consecutive items; segment s waits for
// operation seg_dep[s] to count seg_need[s]
// finished items.  state: [0..1] next item (64-bit), [2] error flag, [3] unused, [4, 4 + nops)
// finished items per operation (these zeroed before every launch), [4 + nops] wait budget in
// clock64() cycles (0: 2^31).
struct PqRun {
  const PqOp *ops = nullptr;
  const long long *seg_start = nullptr;  // nseg + 1 entries
  const int *seg_op = nullptr, *seg_dep = nullptr;
  const long long *seg_need = nullptr;
  const int *const *active = nullptr;  // per member: FGMRES control block (stop flag at [2]), or null
  unsigned *state = nullptr;
  int nseg = 0, nops = 0;
  long long total = 0;
  unsigned geo_smem = 0;  // bytes of dynamic shared memory before the segment starts
};

inline long long pq_items(const PqOp &o) {
  switch (o.type) {
    case kPqCell: return (o.F.n_cells + kPqCellsPerItem - 1) / kPqCellsPerItem;
    case kPqChebInit:
    case kPqChebStep: return (o.n + kPqVecPerItem - 1) / kPqVecPerItem;
    case kPqRestrict: return (o.Cd.n_u + o.Cd.n_p + kPqRestrictPerItem - 1) / kPqRestrictPerItem;
    case kPqProlong: return (o.F.n_u + o.F.n_p + kPqProlongPerItem - 1) / kPqProlongPerItem;
    default: return (o.n0 + kPqCoarsePerItem - 1) / kPqCoarsePerItem;
  }
}

// Dynamic shared memory the queue kernel needs: the Gauss point geometry of the trilinear cell
// operations, then the segment starts (nseg + 1, when at most kPqSmemSegments); and its launch:
// grid = resident CTAs (occupancy x SMs); returns a cudaError_t code.  The queue kernel serves 3D
// k = 2 levels in FP32 (cell-component kernel).
size_t queue_geo_smem_bytes(bool trilinear);
size_t queue_smem_bytes(bool trilinear, int nseg);
int launch_queue(const PqRun &R, size_t smem, cudaStream_t s);
int queue_resident_ctas(size_t smem);

}  // namespace smf
