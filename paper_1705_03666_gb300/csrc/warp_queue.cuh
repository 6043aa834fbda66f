// warp_queue.cuh -- warp-level work claiming for short work units (walks of
// a dozen jumps, small trees).  Taking one index per idle lane from a single
// global cursor costs one same-address atomic per warp per loop trip, which
// limits kernels whose units finish every few trips; here a warp takes C
// consecutive indices with one atomic and hands them to its idle lanes in
// index order.  Results do not depend on the claiming order (every unit
// writes its own slot).
#pragma once

#include "common.cuh"

namespace pdd {

struct WarpQueue {
  unsigned long long next = 0, end = 0;  // warp-uniform local range [next, end)
  bool exhausted = false;                // the global range ran out (warp-uniform)
};

// Lanes whose unit finished wait until at least this many lanes of the warp
// are idle (or all are) before the warp claims new units together: the claim
// and set-up code then runs once for several lanes instead of once per
// finishing lane.  Units of a few loop trips (small trees) finish on nearly
// every trip anyway and claim with B = 1.
constexpr int kClaimBatch = 8;

template <int B = kClaimBatch>
__device__ __forceinline__ bool claim_time(bool active) {
  const unsigned idle = __ballot_sync(kFull, !active);
  return __popc(idle) >= B || idle == kFull;
}

// Called by all 32 lanes together.  A lane with `need` set receives the next
// index in [0, total) in `idx` (returns true, need cleared); once the global
// range is exhausted the remaining lanes get none (need cleared, false).
template <unsigned C>
__device__ __forceinline__ bool warp_claim(WarpQueue &q, unsigned long long *cursor,
                                           unsigned long long total, bool &need,
                                           unsigned long long &idx) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  bool got = false;
  if (q.exhausted) {
    need = false;
    return false;
  }
  unsigned needmask = __ballot_sync(kFull, need);
  while (needmask) {
    if (q.next >= q.end) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(cursor, static_cast<unsigned long long>(C));
      base = __shfl_sync(kFull, base, 0);
      if (base >= total) {
        q.next = q.end = total;
        q.exhausted = true;
        need = false;
        break;
      }
      q.next = base;
      q.end = base + C < total ? base + C : total;
    }
    const unsigned avail = static_cast<unsigned>(q.end - q.next);
    const unsigned cnt = __popc(needmask);
    const unsigned take = avail < cnt ? avail : cnt;
    if (need) {
      const unsigned r = __popc(needmask & lt_mask);
      if (r < take) {
        idx = q.next + r;
        need = false;
        got = true;
      }
    }
    q.next += take;
    needmask = __ballot_sync(kFull, need);
  }
  return got;
}

// Per-lane cache of the node a claimed index belongs to.  Units are
// node-major (index g = node * per_node + k) and claimed in consecutive
// runs, so the node usually repeats: its index range and start point are
// kept, and the division g / per_node (64-bit: emulated in FP64 arithmetic,
// a 1/64-rate pipe on this part) and the FP64 -> R conversions of the node
// coordinates run only when a lane moves to another node.
template <typename R, int D>
struct NodeCache {
  unsigned long long node = 0, lo = 1, hi = 0;  // empty range
  R x[D > 0 ? D : 1];
  __device__ __forceinline__ void locate(unsigned long long g, unsigned long long per_node,
                                         unsigned long long end, const double *nodes,
                                         int stride = D) {
    if (g >= lo && g < hi) return;
    if (end <= 0xffffffffull)
      node = static_cast<uint32_t>(g) / static_cast<uint32_t>(per_node);
    else
      node = g / per_node;
    lo = node * per_node;
    hi = lo + per_node;
#pragma unroll
    for (int d = 0; d < D; ++d) x[d] = static_cast<R>(nodes[node * stride + d]);
  }
};

}  // namespace pdd
