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
};

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
  unsigned needmask = __ballot_sync(kFull, need);
  while (needmask) {
    if (q.next >= q.end) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(cursor, static_cast<unsigned long long>(C));
      base = __shfl_sync(kFull, base, 0);
      if (base >= total) {
        q.next = q.end = total;
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

}  // namespace pdd
