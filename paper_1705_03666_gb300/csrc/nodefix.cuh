// nodefix.cuh -- exact, order-independent per-node sums of path scores (the
// Monte Carlo estimator of Sec. 2: the mean over independent realisations and
// its statistical error), formed inside the path kernel.
//
// Each score s is truncated once to the fixed-point grid 2^-60 and written
// as five base-2^24 digits (weights 2^-60, 2^-36, 2^-12, 2^12, 2^36), and so
// is s^2, formed exactly from the significand in integers.  A warp sums the
// digits of its lanes' paths of one node with one 32-bit reduction
// instruction per digit (32 digits below 2^24 in magnitude cannot overflow),
// and the node's first lane adds the totals to the node's 64-bit words with
// atomics, without carries between digits (at most 2^32 paths per node keep
// every word within 2^56).  Integer addition is associative: the totals are
// the same whichever lane, warp or launch added which path, so the estimate is
// bitwise reproducible while no per-path score is ever stored.
//
// Range: |s| < 2^30 (so that s^2 < 2^60).  A score outside it, or NaN (a node
// outside the closed domain), is counted in `bad` and makes the node's
// estimate NaN.  Truncation at 2^-60 changes a score by less than 2^-60 in
// absolute value, far below the rounding of the score itself.
#pragma once

#include "common.cuh"

namespace pdd {

constexpr int kFixDigits = 5;
struct NodeFix {
  long long n;                 // paths scored (boundary starts included)
  long long s1[kFixDigits];    // digit sums of s
  long long s2[kFixDigits];    // digit sums of s^2
  long long capped;            // paths stopped by the step cap
  long long bad;               // NaN or out-of-range scores
  long long boundary;          // paths that started on the boundary (tau = 0)
};
constexpr int kFixWords = 2 + 2 * kFixDigits + 2;
static_assert(sizeof(NodeFix) == kFixWords * sizeof(long long), "NodeFix layout");
constexpr int kFixCapped = 1 + 2 * kFixDigits, kFixBad = kFixCapped + 1,
              kFixBoundary = kFixCapped + 2;

// Per-node flags (include/pdd.h, pdd_diag.d_node_flags).
constexpr int32_t kNodeOnBoundary = 1;
constexpr int32_t kNodeOutside = 2;
constexpr int32_t kNodeCapped = 4;
constexpr int32_t kNodeDiscarded = 8;
constexpr int32_t kNodeEmpty = 16;
constexpr int32_t kNodeSeUnmet = 32;

constexpr uint32_t kDigitMask = (1u << 24) - 1;

// Digit k of floor(M 2^sh) for M < 2^24: floor(M 2^(sh - 24k)) mod 2^24
// (the 32-bit shift keeps the low 24 bits of M 2^t for 0 <= t < 24).
__device__ __forceinline__ int32_t fix_digit24(uint32_t M, int t) {
  if (t >= 24 || t <= -24) return 0;
  return static_cast<int32_t>(t >= 0 ? (M << t) & kDigitMask : M >> (-t));
}
// The same for M < 2^48 (a product of two 24-bit significands).
__device__ __forceinline__ int32_t fix_digit48(unsigned long long M, int t) {
  if (t >= 24 || t <= -48) return 0;
  return static_cast<int32_t>((t >= 0 ? M << t : M >> (-t)) & kDigitMask);
}
// The same for M < 2^106 (a product of two 53-bit significands).
__device__ __forceinline__ int32_t fix_digit106(unsigned __int128 M, int t) {
  if (t >= 24 || t <= -106) return 0;
  return static_cast<int32_t>(static_cast<unsigned long long>(t >= 0 ? M << t : M >> (-t)) &
                              kDigitMask);
}

// Digits of s 2^60 (d1, with the sign of s) and of s^2 2^60 (d2), each
// truncated toward zero, from the bits of s: s = +-m 2^e, so s 2^60 =
// m 2^(e + 60) and s^2 2^60 = m^2 2^(2e + 60) with m^2 formed exactly in
// integers.  Integer arithmetic only (the FP64 pipe is a 1/64-rate unit on
// this part).  Requires |s| < 2^30.
__device__ __forceinline__ void fix_limbs(float s, int32_t *d1, int32_t *d2) {
  const uint32_t b = __float_as_uint(s);
  const int E = static_cast<int>((b >> 23) & 0xffu);
  const uint32_t m = (b & 0x7fffffu) | (E ? 0x800000u : 0u);
  const int e = (E ? E : 1) - 150;  // s = m 2^e
  const unsigned long long m2 = static_cast<unsigned long long>(m) * m;
  const bool neg = (b >> 31) != 0;
#pragma unroll
  for (int k = 0; k < kFixDigits; ++k) {
    const int32_t v = fix_digit24(m, e + 60 - 24 * k);
    d1[k] = neg ? -v : v;
    d2[k] = fix_digit48(m2, 2 * e + 60 - 24 * k);
  }
}
__device__ __forceinline__ void fix_limbs(double s, int32_t *d1, int32_t *d2) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(s));
  const int E = static_cast<int>((b >> 52) & 0x7ffu);
  const unsigned long long m = (b & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull);
  const int e = (E ? E : 1) - 1075;  // s = m 2^e
  const unsigned __int128 m2 = static_cast<unsigned __int128>(m) * m;
  const bool neg = (b >> 63) != 0;
#pragma unroll
  for (int k = 0; k < kFixDigits; ++k) {
    const int32_t v = fix_digit106(m, e + 60 - 24 * k);
    d1[k] = neg ? -v : v;
    d2[k] = fix_digit106(m2, 2 * e + 60 - 24 * k);
  }
}

// Called by all 32 lanes of a warp.  A lane with `has` set adds one path of
// node `node` with score s (capped: stopped by the step cap; boundary: started
// on the boundary; NaN s: invalid start).  Every lane forms its digits first
// (no divergence); then, one node at a time, each digit is summed over the
// node's lanes with one warp reduction and the node's first lane issues the
// atomics.  The rare events (capped, boundary, invalid) are counted with
// per-lane atomics.
template <typename R>
__device__ __forceinline__ void fix_commit(NodeFix *fix, bool has, uint64_t node, R s,
                                           bool capped, bool boundary) {
  const bool valid = has && fabs(s) < R(0x1p30);  // false for NaN
  if (has) {
    unsigned long long *w = reinterpret_cast<unsigned long long *>(fix + node);
    if (!valid) atomicAdd(w + kFixBad, 1ull);
    if (valid && capped) atomicAdd(w + kFixCapped, 1ull);
    if (valid && boundary) atomicAdd(w + kFixBoundary, 1ull);
  }
  int32_t d[2 * kFixDigits];
#pragma unroll
  for (int k = 0; k < 2 * kFixDigits; ++k) d[k] = 0;
  if (valid) fix_limbs(s, d, d + kFixDigits);
  const unsigned lane = threadIdx.x & 31u;
  unsigned pending = __ballot_sync(kFull, valid);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const uint64_t ln = __shfl_sync(kFull, node, leader);
    const bool mem = valid && node == ln;
    const unsigned members = __ballot_sync(kFull, mem);
    unsigned long long *w = reinterpret_cast<unsigned long long *>(fix + ln);
    int32_t r[2 * kFixDigits];
#pragma unroll
    for (int k = 0; k < 2 * kFixDigits; ++k) r[k] = __reduce_add_sync(kFull, mem ? d[k] : 0);
    if (lane == static_cast<unsigned>(leader)) {
      atomicAdd(w, static_cast<unsigned long long>(__popc(members)));
#pragma unroll
      for (int k = 0; k < 2 * kFixDigits; ++k)
        if (r[k] != 0)
          atomicAdd(w + 1 + k, static_cast<unsigned long long>(static_cast<long long>(r[k])));
    }
    pending &= ~members;
  }
}

// One lane adds `count` paths of node `node` that all score s (a node on the
// boundary: tau = 0 for every path, so u = g there), or, for NaN s (a node
// outside the closed domain), counts them as invalid.  Per-lane atomics:
// such nodes are rare, and count * digit stays far below 2^63.
template <typename R>
__device__ __forceinline__ void fix_add_repeated(NodeFix *fix, uint64_t node, R s,
                                                 long long count) {
  unsigned long long *w = reinterpret_cast<unsigned long long *>(fix + node);
  if (!(fabs(s) < R(0x1p30))) {
    atomicAdd(w + kFixBad, static_cast<unsigned long long>(count));
    return;
  }
  int32_t d[2 * kFixDigits];
  fix_limbs(s, d, d + kFixDigits);
  atomicAdd(w, static_cast<unsigned long long>(count));
#pragma unroll
  for (int k = 0; k < 2 * kFixDigits; ++k)
    if (d[k] != 0)
      atomicAdd(w + 1 + k, static_cast<unsigned long long>(count * static_cast<long long>(d[k])));
  atomicAdd(w + kFixBoundary, static_cast<unsigned long long>(count));
}

// Double-double helpers for the finalisation (Dekker/Knuth error-free
// transformations with FMA).
struct DD {
  double hi, lo;
};
__device__ __forceinline__ DD dd_two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DD dd_norm(double hi, double lo) {
  const double s = hi + lo;
  return {s, lo - (s - hi)};
}
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  const DD s = dd_two_sum(a.hi, b.hi);
  return dd_norm(s.hi, s.lo + a.lo + b.lo);
}
__device__ __forceinline__ DD dd_mul(DD a, DD b) {
  const double p = a.hi * b.hi;
  const double e = fma(a.hi, b.hi, -p);
  return dd_norm(p, e + a.hi * b.lo + a.lo * b.hi);
}
__device__ __forceinline__ DD dd_div(DD a, double d) {
  const double q1 = a.hi / d;
  const double p = q1 * d;
  const double e = fma(q1, d, -p);
  const double r = ((a.hi - p) - e) + a.lo;
  return dd_norm(q1, r / d);
}
// The exact digit total sum_k l[k] 2^(24k - 60) as a double-double.
__device__ __forceinline__ DD fix_total(const long long *l) {
  DD t{0.0, 0.0};
#pragma unroll
  for (int k = 0; k < kFixDigits; ++k) {
    const double sc = ldexp(1.0, 24 * k - 60);
    const double hi = static_cast<double>(l[k]);
    const double lo = static_cast<double>(l[k] - static_cast<long long>(hi));
    t = dd_add(t, DD{hi * sc, lo * sc});
  }
  return t;
}

// Mean and the sum of squared deviations M2 of a node's scores from its
// exact sums: mean = S1/n, M2 = S2 - S1^2/n in double-double (M2 = 0 when
// every path started on the boundary, or with one path).  Both NaN when a
// path was invalid or nothing was scored.
__device__ __forceinline__ void fix_moments(const NodeFix &F, double *mean, double *m2) {
  const double nn = static_cast<double>(F.n);
  *mean = static_cast<double>(NAN);
  *m2 = static_cast<double>(NAN);
  if (F.bad != 0 || F.n <= 0) return;
  const DD S1 = fix_total(F.s1), S2 = fix_total(F.s2);
  const DD mu = dd_div(S1, nn);
  *mean = mu.hi + mu.lo;
  *m2 = 0.0;
  if (F.boundary != F.n && F.n > 1) {
    const DD q = dd_mul(S1, mu);
    const DD d = dd_add(S2, DD{-q.hi, -q.lo});
    *m2 = fmax(0.0, d.hi + d.lo);
  }
}

// Mean, standard error of the mean, path count and flags per node from the
// exact sums: se = sqrt(M2 / (n - 1) / n), 0 when every path started on the
// boundary (tau = 0, the estimate is exact) or with one path; NaN when a
// path was invalid or nothing was scored.
static __global__ void fix_finalize_kernel(const NodeFix *fix, int64_t n_nodes, double *mean,
                                           double *se, int64_t *npaths, int32_t *flags) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n_nodes) return;
  const NodeFix F = fix[i];
  const double nn = static_cast<double>(F.n);
  double m, M2;
  fix_moments(F, &m, &M2);
  const double e = F.n > 1 ? sqrt(M2 / (nn - 1.0) / nn) : M2;  // M2 is 0 or NaN for n <= 1
  mean[i] = m;
  se[i] = e;
  if (npaths) npaths[i] = F.n;
  if (flags) {
    int32_t f = 0;
    if (F.boundary > 0) f |= kNodeOnBoundary;
    if (F.bad > 0) f |= kNodeOutside;
    if (F.capped > 0) f |= kNodeCapped;
    if (F.n == 0) f |= kNodeEmpty;
    flags[i] = f;
  }
}

}  // namespace pdd
