// Device side of the persistent work-queue V-cycle (queue.h): the kernel and its work items.
// Included by the k = 2 cell-component translation unit, whose 1D tables the cell items use.
// Every input an item reads may have been written by an earlier item of the same launch on
// another SM, so items read through L2 (ld_in<true>), write with plain stores or L2 atomics,
// fence, and count themselves finished after a CTA barrier; a waiting CTA acquires the counter,
// fences and passes a CTA barrier before its loads.
#pragma once
#include "apply_cc.cuh"
#include "queue.h"
#include "transfer.cuh"
#include "vec.cuh"

namespace smf {

static_assert(kPqCellsPerItem == (kPqThreads / 32) * kPqGroupsPerWarp * kCcCells, "cell-component groups per item");

__device__ __forceinline__ int pq_ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return (int)v;
}

template <int MODE>
__device__ __forceinline__ void pq_cell_mode(const PqOp &o, long long group) {
  if (o.F.cartesian)
    cc_group<2, float, MODE, true, false, false, true>(o.F, o.in[0], o.in[1], o.out[0], o.out[1], nullptr, group, -1);
  else
    cc_group<2, float, MODE, false, false, false, true>(o.F, o.in[0], o.in[1], o.out[0], o.out[1], nullptr, group,
                                                        -1);
}

__device__ __forceinline__ void pq_item(const PqOp &o, long long b) {
  const int t = threadIdx.x;
  switch (o.type) {
    case kPqCell: {
      constexpr int W = kPqThreads / 32;
      const long long first = b * (W * kPqGroupsPerWarp), ngroups = (o.F.n_cells + kCcCells - 1) / kCcCells;
      for (int j = 0; j < kPqGroupsPerWarp; ++j) {
        const long long group = first + j * W + (t >> 5);
        if (first + j * W >= ngroups) break;  // uniform over the CTA
        switch (o.mode) {
          case kApplyA: pq_cell_mode<kApplyA>(o, group); break;
          case kApplyBT: pq_cell_mode<kApplyBT>(o, group); break;
          case kApplyB: pq_cell_mode<kApplyB>(o, group); break;
          case kApplyA | kApplyBT: pq_cell_mode<kApplyA | kApplyBT>(o, group); break;
          default: pq_cell_mode<kApplyA | kApplyBT | kApplyB>(o, group); break;
        }
      }
      break;
    }
    case kPqChebInit:
    case kPqChebStep: {
      // packs of 4 where every vector is 16-byte aligned (the scalar tail in the last item), else entries
      const bool init = o.type == kPqChebInit;
      long long s0 = b * kPqVecPerItem, s1 = min(o.n, (b + 1) * kPqVecPerItem);
      if (o.vec4) {
        const long long np4 = o.n / 4, p1 = min(np4, (b + 1) * (kPqVecPerItem / 4));
        for (long long j = b * (kPqVecPerItem / 4) + t; j < p1; j += kPqThreads) {
          if (init)
            cheb_init_packj<float, 4, true>(j, o.in[0], o.in[1], o.sc[0], o.in[2], o.sc[1], o.out[0], o.out[1],
                                            o.out[2], o.in[3], o.sc[2], o.out[3], o.out[4], o.out[5], o.out[6]);
          else
            cheb_step_packj<float, 4, true>(j, o.in[0], o.out[0], o.in[1], o.sc[0], o.sc[1], o.out[1], o.out[2],
                                            o.in[2], o.sc[2], o.out[3], o.out[4]);
        }
        s0 = np4 * 4;
        if (b != o.items - 1) s1 = s0;  // the tail belongs to the last item
      }
      for (long long i = s0 + t; i < s1; i += kPqThreads) {
        if (init)
          cheb_init_elem<float, true>(i, o.in[0], o.in[1], o.sc[0], o.in[2], o.sc[1], o.out[0], o.out[1], o.out[2],
                                      o.in[3], o.sc[2], o.out[3], o.out[4], o.out[5], o.out[6]);
        else
          cheb_step_elem<float, true>(i, o.in[0], o.out[0], o.in[1], o.sc[0], o.sc[1], o.out[1], o.out[2], o.in[2],
                                      o.sc[2], o.out[3], o.out[4]);
      }
      break;
    }
    case kPqRestrict: {
      const long long end = min(o.Cd.n_u + o.Cd.n_p, (b + 1) * kPqRestrictPerItem);
      for (long long i = b * kPqRestrictPerItem + t; i < end; i += kPqThreads) {
        const float s = o.in[1] ? restrict_terms<float, 9, true, true>(o.F, o.Cd, o.X, o.in[0], o.in[1], i, 0, 1)
                                : restrict_terms<float, 9, false, true>(o.F, o.Cd, o.X, o.in[0], nullptr, i, 0, 1);
        o.out[0][i] = s;
        if (o.out[1]) o.out[1][i] = 0.f;
      }
      break;
    }
    case kPqProlong: {
      const long long end = min(o.F.n_u + o.F.n_p, (b + 1) * kPqProlongPerItem);
      for (long long i = b * kPqProlongPerItem + t; i < end; i += kPqThreads) {
        if (o.out[3]) o.out[3][i] = 0.f;
        if (i < o.F.n_u) {
          if (o.out[1]) o.out[1][i] = 0.f;
          if (o.out[2]) o.out[2][i] = 0.f;
        }
        const float s = prolong_entry<float, 9, true>(o.F, o.Cd, o.X, o.in[0], i);
        o.out[0][i] = o.add ? ld_in<true>(o.out[0] + i) + s : s;
      }
      break;
    }
    default: {  // coarse solve: x = Kinv b, one row per warp at a time (the arithmetic of k_coarse_apply)
      const int lane = t & 31;
      for (int row = (int)(b * kPqCoarsePerItem) + (t >> 5); row < min((long long)o.n0, (b + 1) * kPqCoarsePerItem);
           row += kPqThreads / 32) {
        const double *kr = o.Kinv + (long long)row * o.n0;
        double s = 0.0;
        for (int j = lane; j < o.n0; j += 32) s += kr[j] * (double)ld_in<true>(o.in[0] + j);
        for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
        if (lane == 0) o.out[0][row] = (float)s;
      }
      break;
    }
  }
}

// The persistent kernel: each CTA takes the next item, waits (bounded) until the member's
// previous operation is complete, runs the item and counts it finished.  Items are taken in
// queue order and only wait for earlier items, all of which are held by running CTAs, so the
// queue drains; a wait that exceeds the budget sets the error flag and every CTA returns.
__global__ void __launch_bounds__(kPqThreads, 4) k_queue_run(const PqRun R) {
  pdl_enter();
  __shared__ long long s_item;
  __shared__ int s_seg, s_ok;
  extern __shared__ float4 cc_geo_smem[];
  // the segment starts in shared memory (after the geometry region) where they fit
  long long *sstart = reinterpret_cast<long long *>(reinterpret_cast<unsigned char *>(cc_geo_smem) + R.geo_smem);
  const bool seg_smem = R.nseg <= kPqSmemSegments;
  if (seg_smem)
    for (int i = threadIdx.x; i <= R.nseg; i += kPqThreads) sstart[i] = R.seg_start[i];
  const long long *starts = seg_smem ? sstart : R.seg_start;
  __syncthreads();
  unsigned long long *head = reinterpret_cast<unsigned long long *>(R.state);
  unsigned *err = R.state + 2, *done = R.state + 4;
  // thread 0 takes the next item while the CTA runs the current one (taking it early keeps the
  // queue order: items are still held only by running CTAs and taken in increasing order)
  long long next = threadIdx.x == 0 ? (long long)atomicAdd(head, 1ull) : 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = next;
      int seg = 0, ok = it < R.total && *((volatile unsigned *)err) == 0;
      if (ok) {
        int lo = 0, hi = R.nseg - 1;  // the last segment starting at or before it
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (starts[mid] <= it)
            lo = mid;
          else
            hi = mid - 1;
        }
        seg = lo;
        const int dep = R.seg_dep[seg];
        if (dep >= 0) {
          const unsigned bud = *((volatile unsigned *)(R.state + 4 + R.nops));
          const long long budget = bud ? (long long)bud : (1ll << 31), t0 = clock64();
          while (pq_ld_acquire(done + dep) < R.seg_need[seg]) {
            if (*((volatile unsigned *)err)) {
              ok = 0;
              break;
            }
            if (clock64() - t0 > budget) {
              atomicExch(err, 1u);
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
          __threadfence();  // acquire side: the item's loads follow the producers' writes
        }
      }
      s_item = it;
      s_seg = seg;
      s_ok = ok;
      if (ok) next = (long long)atomicAdd(head, 1ull);
    }
    __syncthreads();
    if (!s_ok) return;
    const int seg = s_seg;
    const int op = R.seg_op[seg];
    const PqOp &o = R.ops[op];
    const bool act = !R.active || !R.active[o.member] || R.active[o.member][2] == 0;
    if (act) pq_item(o, s_item - starts[seg]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(done + op, 1u);
  }
}

size_t queue_geo_smem_bytes(bool trilinear) {
  return trilinear ? (size_t)(kPqThreads / 32) * 27 * CcGeo<kApplyA | kApplyBT | kApplyB>::NF * kCcCells *
                         sizeof(float4)
                   : 0;
}
size_t queue_smem_bytes(bool trilinear, int nseg) {
  return queue_geo_smem_bytes(trilinear) + (nseg <= kPqSmemSegments ? sizeof(long long) * (nseg + 1) : 0);
}

int queue_resident_ctas(size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(k_queue_run, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_queue_run, kPqThreads, smem);
  if (e != cudaSuccess) return -(int)e;
  return per_sm * sms;
}

int launch_queue(const PqRun &R, size_t smem, cudaStream_t s) {
  const int grid = queue_resident_ctas(smem);
  if (grid <= 0) return grid < 0 ? -grid : (int)cudaErrorInvalidConfiguration;
  launch_kernel(k_queue_run, dim3((unsigned)grid), dim3(kPqThreads), smem, s, R);
  return (int)cudaGetLastError();
}

}  // namespace smf
