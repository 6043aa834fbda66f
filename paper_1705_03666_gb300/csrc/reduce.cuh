// reduce.cuh -- per-node sample mean / standard error of per-path scores
// (the Monte Carlo estimator of Sec. 2: the mean over independent
// realisations, with its statistical error).
//
// Each wave of the path index space is reduced by one block per node: the
// block sums the shifted scores (s - K, with K the node's first score in the
// wave) and their squares with compensated FP64 accumulators, combines the
// threads in a fixed tree (warp shuffles, then shared memory), and merges the
// wave's (count, mean, M2) into the node's running triple with Chan's formula.
// Waves are processed in order, so the result is deterministic.
#pragma once

#include "common.cuh"
#include "nodefix.cuh"

namespace pdd {

constexpr int kReduceBlock = 256;

struct NodeAcc {  // running (count, mean, M2) per node, FP64
  double n, mean, m2;
};

// Per-thread accumulation.  Binary32 scores are summed on the FP32 pipe as
// two-float values (Knuth's TwoSum: a ~48-bit significand, far below the
// scores' own rounding), the shift s - K split exactly into two floats and
// the square's rounding error recovered with an FMA; binary64 scores are
// summed plainly in FP64 (a few thousand terms per thread).  FP64 is a
// 1/64-rate pipe on this part, so a compensated FP64 sum per score would
// make the reduction, not the paths, the cost of short-path workloads.
// Threads are then combined with compensated FP64 sums in a fixed tree.
struct F2Sum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
  }
};

template <typename R, bool kSkipNaN>
struct ThreadSums;
template <bool kSkipNaN>
struct ThreadSums<float, kSkipNaN> {
  F2Sum s1, s2;
  unsigned kept = 0;  // below 2^32: a wave holds at most 2^31 scores
  __device__ __forceinline__ void add(float v, float K) {
    if constexpr (kSkipNaN) {
      // K = 0 here: a NaN score is replaced by 0, which adds exactly zero,
      // and the shift needs no split
      const bool ok = !isnan(v);
      kept += ok ? 1u : 0u;
      v = ok ? v : 0.0f;
      s1.add(v);
      const float q = v * v;
      const float e = fmaf(v, v, -q);
      s2.add(q);
      s2.lo += e;
      return;
    }
    ++kept;
    const float d = v - K;  // d + dl = v - K exactly
    const float bb = d - v;
    const float dl = (v - (d - bb)) + (-K - bb);
    s1.add(d);
    s1.lo += dl;
    const float q = d * d;
    const float e = fmaf(d, d, -q);
    s2.add(q);
    s2.lo += e + 2.0f * d * dl;
  }
  __device__ __forceinline__ void out(CSum &c1, CSum &c2) const {
    c1.add(static_cast<double>(s1.hi));
    c1.add(static_cast<double>(s1.lo));
    c2.add(static_cast<double>(s2.hi));
    c2.add(static_cast<double>(s2.lo));
  }
};
template <bool kSkipNaN>
struct ThreadSums<double, kSkipNaN> {
  double s1 = 0.0, s2 = 0.0;
  unsigned long long kept = 0;
  __device__ __forceinline__ void add(double v, double K) {
    if (kSkipNaN && isnan(v)) return;
    ++kept;
    const double d = v - K;
    s1 += d;
    s2 = fma(d, d, s2);
  }
  __device__ __forceinline__ void out(CSum &c1, CSum &c2) const {
    c1.add(s1);
    c2.add(s2);
  }
};

// kSkipNaN: NaN scores mark discarded samples (pruned trees) and are left
// out of the count; the shift K is then 0 (scores are bounded weights).
template <typename R, bool kSkipNaN = false>
__global__ void __launch_bounds__(kReduceBlock)
reduce_wave_kernel(const R *__restrict__ score, uint64_t begin, uint64_t end,
                   uint64_t n_paths, uint64_t node_lo, NodeAcc *acc,
                   uint64_t score_plane = 0, uint64_t acc_plane = 0) {
  // blockIdx.y selects a plane (score + y score_plane, acc + y acc_plane):
  // several score planes of one wave reduced by one launch
  score += blockIdx.y * score_plane;
  acc += blockIdx.y * acc_plane;
  const uint64_t node = node_lo + blockIdx.x;
  const uint64_t lo = max(begin, node * n_paths);
  const uint64_t hi = min(end, (node + 1) * n_paths);
  if (lo >= hi) return;
  const R *s = score + (lo - begin);
  const uint64_t cnt = hi - lo;
  const R Kr = kSkipNaN ? R(0) : s[0];
  const double K = static_cast<double>(Kr);
  ThreadSums<R, kSkipNaN> ts;
  if constexpr (sizeof(R) == 4) {
    // binary32 scores: scalar up to a 16-byte boundary, then four per load
    // with several loads in flight per thread (the reduction is bound by
    // memory latency otherwise), then the scalar tail
    uint64_t head = ((16u - (reinterpret_cast<uintptr_t>(s) & 15u)) & 15u) / 4u;
    if (head > cnt) head = cnt;
    if (threadIdx.x < head) ts.add(s[threadIdx.x], Kr);
    const float4 *v = reinterpret_cast<const float4 *>(s + head);
    const uint64_t n4 = (cnt - head) / 4;
#pragma unroll 4
    for (uint64_t j = threadIdx.x; j < n4; j += kReduceBlock) {
      const float4 q = __ldcs(v + j);
      ts.add(q.x, Kr);
      ts.add(q.y, Kr);
      ts.add(q.z, Kr);
      ts.add(q.w, Kr);
    }
    for (uint64_t i = head + 4 * n4 + threadIdx.x; i < cnt; i += kReduceBlock) ts.add(s[i], Kr);
  } else {
    for (uint64_t i = threadIdx.x; i < cnt; i += kReduceBlock) ts.add(s[i], Kr);
  }
  CSum s1, s2;
  ts.out(s1, s2);
  unsigned long long kept = ts.kept;
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    s1.merge(shfl_xor(s1, m));
    s2.merge(shfl_xor(s2, m));
    kept += __shfl_xor_sync(kFull, kept, m);
  }
  __shared__ CSum sh1[kReduceBlock / 32], sh2[kReduceBlock / 32];
  __shared__ unsigned long long shk[kReduceBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh1[warp] = s1;
    sh2[warp] = s2;
    shk[warp] = kept;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum t1 = sh1[0], t2 = sh2[0];
    unsigned long long tk = shk[0];
    for (int w = 1; w < kReduceBlock / 32; ++w) {
      t1.merge(sh1[w]);
      t2.merge(sh2[w]);
      tk += shk[w];
    }
    if (tk == 0) return;
    const double nb = static_cast<double>(tk);
    const double S1 = t1.value(), S2 = t2.value();
    const double mean_b = K + S1 / nb;
    const double m2_b = fmax(0.0, S2 - S1 * S1 / nb);
    NodeAcc A = acc[node];
    const double nt = A.n + nb;
    const double d = mean_b - A.mean;
    A.mean = A.mean + d * (nb / nt);
    A.m2 = A.m2 + m2_b + d * d * (A.n * nb / nt);
    A.n = nt;
    acc[node] = A;
  }
}

// Mean, standard error and count per node; with `flags`, PDD_NODE_EMPTY is
// OR-ed into the node's flags when no sample was kept (the kernels OR in the
// rarer events themselves).
static __global__ void finalize_kernel(const NodeAcc *acc, int64_t n_nodes, double *mean,
                                       double *se, int64_t *npaths, int32_t *flags = nullptr) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n_nodes) return;
  const NodeAcc A = acc[i];
  mean[i] = A.n > 0.0 ? A.mean : static_cast<double>(NAN);  // no sample kept
  se[i] = A.n > 1.0 ? sqrt(A.m2 / (A.n - 1.0) / A.n) : (A.n > 0.0 ? 0.0 : static_cast<double>(NAN));
  if (npaths) npaths[i] = static_cast<int64_t>(A.n);
  if (flags && !(A.n > 0.0)) flags[i] |= kNodeEmpty;
}

template <typename R>
__global__ void widen_scores_kernel(const R *__restrict__ src, double *dst, uint64_t count) {
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    dst[i] = static_cast<double>(src[i]);
}

}  // namespace pdd
