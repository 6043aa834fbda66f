// batch_kernel.cuh -- one persistent work-queue launch over a heterogeneous,
// ragged batch of interface nodes (several domains and PDE families, per-node
// time steps, per-node path counts).
//
// The unit of queued work is a lane-chunk: up to K consecutive paths of one
// node, run one after the other by a single lane, which accumulates their
// shifted scores (s - K_i) and squares in registers and writes one partial
// per chunk.  A lane that finishes its chunk takes the next chunk from a
// warp-aggregated cursor, so lanes never wait for one another; partials are
// indexed by chunk, so the per-node merge (fixed order) does not depend on
// scheduling.  Chunk counts may live in device memory, so a launch sized on
// the host can consume a work list produced on the device (the adaptive
// pass), and the whole pipeline can be captured in a CUDA graph.
//
// The nodes are grouped by domain/family (a stable partition built on the
// device, `perm`), the chunk list follows that order, and each family runs
// its own instantiation of the kernel over its own chunk range: a kernel
// compiled for one family has the registers and the code of that family's
// path unit only.  (One kernel dispatching on the family per lane ran at
// about half the speed of the plain path kernel on the same paths.)
#pragma once

#include "path_kernel.cuh"
#include "reduce.cuh"

namespace pdd {

constexpr int kMaxBatchProblems = 4;

// Domain/family combinations the batch kernel dispatches on.
enum : int32_t {
  kComboSquareLaplace = 0,   // LaplaceExpCos on Box<2>
  kComboLShapeLaplace = 1,   // LaplaceExpCos on LShape
  kComboCubeElliptic = 2,    // EllipticManufactured on Box<3>
  kComboSquarePoisson = 3    // PoissonFourier on Box<2>
};

struct BatchProblem {
  ModelConst mc;
  int32_t combo;
  int32_t bridge;
  double sigma;
  double c_kill;  // constant killing rate (paper's c)
};

struct ChunkPartial {  // n, sum (s - K_i), sum (s - K_i)^2
  double n, s1, s2;
};

struct BatchArgs {
  const double *nodes;      // [n][3] (z ignored by 2-D families)
  const int32_t *prob;      // [n] index into probs
  const double *dt;         // [n]
  int64_t n;
  // node order grouped by family: perm[j] is the node at position j; family c
  // holds positions [cstart[c], cstart[c+1])
  const int32_t *perm;
  const int64_t *cstart;
  // work list, in that order: the node at position j owns chunks
  // [chunk_off[j], chunk_off[j+1]) covering paths [first[i], end[i]) of node
  // i = perm[j] in pieces of K; chunk_off[n] = total chunks
  const int64_t *chunk_off;
  const int64_t *first;
  const int64_t *end;
  const double *shift;      // [n] per-node shift K_i of the sums
  int32_t K;
  unsigned long long *cursor;  // [4]: one per family
  unsigned long long *counters;  // [0] path steps, [1] capped, [2] bad nodes
  ChunkPartial *partial;    // [chunk_off[n]]
  RoundKeys rk;
  int32_t max_steps;
  int32_t n_probs;
  BatchProblem probs[kMaxBatchProblems];
};

struct BatchEnv {
  const ModelConst &mc;
  int32_t bridge;
};

// Lane state that survives across loop iterations.
struct BatchLane {
  float X[3];
  float Y, Z;
  int32_t n;
  PhiloxPath pp;
};

// One loop unit (path_unit) of a path of family Model on domain Geom.
// Returns true when the path exited (score in s); the caller handles the cap.
template <class Model, class Geom>
__device__ __forceinline__ bool batch_unit(const BatchEnv &env, const StepConst<float> &k,
                                           const RoundKeys &rk, int32_t max_steps, BatchLane &L,
                                           float &s) {
  float xe[Model::D], lr[1];
  return path_unit<Model, Geom, float, false>(env, k, L.pp, rk, max_steps, L.X, L.Y, L.Z, L.n, s,
                                              xe, lr);
}

// Score of a capped path: g at the projection on the nearest face.
template <class Model, class Geom>
__device__ __forceinline__ float batch_capped(const ModelConst &mc, const BatchLane &L) {
  constexpr int D = Model::D;
  float xe[D];
#pragma unroll
  for (int d = 0; d < D; ++d) xe[d] = L.X[d];
  Geom::project(Geom::nearest_face(xe), xe);
  return Model::g(mc, xe) * L.Y + L.Z;
}

template <class Model, class Geom>
__device__ __forceinline__ bool batch_inside(const float *x) {
  return Geom::inside_open(x);
}
template <class Model, class Geom>
__device__ __forceinline__ bool batch_closed(const float *x) {
  return Geom::inside_closed(x);
}

template <int C> struct ComboTraits;
template <> struct ComboTraits<kComboSquareLaplace> { using M = LaplaceExpCos; using G = Box<2>; };
template <> struct ComboTraits<kComboLShapeLaplace> { using M = LaplaceExpCos; using G = LShape; };
template <> struct ComboTraits<kComboCubeElliptic> { using M = EllipticManufactured; using G = Box<3>; };
template <> struct ComboTraits<kComboSquarePoisson> { using M = PoissonFourier; using G = Box<2>; };

constexpr int kBatchBlock = 256;

template <int C>
__global__ void __launch_bounds__(kBatchBlock)
batch_kernel(const __grid_constant__ BatchArgs a) {
  using M = typename ComboTraits<C>::M;
  using G = typename ComboTraits<C>::G;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  // this family's positions and chunks
  const int64_t jlo = a.cstart[C], jhi = a.cstart[C + 1];
  if (jlo >= jhi) return;
  const uint64_t c_lo = static_cast<uint64_t>(a.chunk_off[jlo]);
  const uint64_t c_hi = static_cast<uint64_t>(a.chunk_off[jhi]);
  unsigned long long *cursor = a.cursor + C;
  BatchLane L;
  float x0[3] = {0.f, 0.f, 0.f};  // the chunk's node, converted once per chunk
  StepConst<float> k;
  int32_t pi = 0;
  uint32_t node = 0;
  int64_t path = 0, path_end = 0;
  uint64_t chunk = 0;
  // per-chunk sums of (s - K_i) and its square as two-float values on the
  // FP32 pipe (FP64 adds per path, at 1/64 rate in divergent code, were a
  // visible cost); the chunk partial is written in FP64
  float shift_f = 0.f;
  double shift = 0.0;
  F2Sum s1, s2;
  int32_t cnt = 0;
  bool active = false, need = true;
  unsigned long long my_steps = 0, my_capped = 0, my_bad = 0;

  for (;;) {
    for (;;) {
      const unsigned needmask = __ballot_sync(kFull, need);
      if (!needmask) break;
      const int leader = __ffs(needmask) - 1;
      unsigned long long base = 0;
      if (static_cast<int>(lane) == leader)
        base = atomicAdd(cursor, static_cast<unsigned long long>(__popc(needmask)));
      base = __shfl_sync(kFull, base, leader);
      if (need) {
        need = false;
        const unsigned long long c = c_lo + base + __popc(needmask & lt_mask);
        if (c < c_hi) {
          chunk = c;
          // position owning chunk c: last j in [jlo, jhi) with chunk_off[j] <= c
          int64_t lo = jlo, hi = jhi;
          while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (static_cast<uint64_t>(a.chunk_off[mid]) <= c) lo = mid; else hi = mid;
          }
          const int64_t i = a.perm[lo];
          node = static_cast<uint32_t>(i);
          const int64_t jj = static_cast<int64_t>(c) - a.chunk_off[lo];
          path = a.first[i] + jj * a.K;
          path_end = min(a.end[i], path + a.K);
          pi = a.prob[i];
          const BatchProblem &P = a.probs[pi];
          k = make_step_const(a.dt[i], P.sigma, P.c_kill, P.bridge != 0);
          shift = a.shift ? a.shift[i] : 0.0;
          shift_f = static_cast<float>(shift);
          s1 = F2Sum();
          s2 = F2Sum();
          cnt = 0;
          x0[0] = static_cast<float>(a.nodes[i * 3 + 0]);
          x0[1] = static_cast<float>(a.nodes[i * 3 + 1]);
          x0[2] = static_cast<float>(a.nodes[i * 3 + 2]);
          L.X[0] = x0[0];
          L.X[1] = x0[1];
          L.X[2] = x0[2];
          if (!batch_inside<M, G>(L.X)) {
            // node on (or, invalid, outside) the boundary: every path scores g
            const bool closed = batch_closed<M, G>(L.X);
            const double v = closed ? static_cast<double>(M::g(P.mc, L.X)) - shift
                                    : static_cast<double>(NAN);
            if (!closed) ++my_bad;
            const double cn = static_cast<double>(path_end - path);
            a.partial[chunk] = ChunkPartial{cn, cn * v, cn * v * v};
            need = true;
          } else {
            L.Y = 1.f;
            L.Z = 0.f;
            L.n = 0;
            L.pp = philox_path(static_cast<uint32_t>(path), node, 0u, a.rk);
            active = true;
          }
        }
      }
    }
    if (!__any_sync(kFull, active)) break;
    if (!active) continue;

    const BatchProblem &P = a.probs[pi];
    const BatchEnv env{P.mc, P.bridge};
    float s = 0.f;
    bool done = batch_unit<M, G>(env, k, a.rk, a.max_steps, L, s);
    if (!done && L.n >= a.max_steps) {
      s = batch_capped<M, G>(P.mc, L);
      ++my_capped;
      done = true;
    }
    if (done) {
      // s - shift_f split exactly into two floats (the shift is rounded to
      // FP32 once per chunk; the FP64 partial corrects for shift - shift_f)
      const float d = s - shift_f;
      const float bb = d - s;
      const float dl = (s - (d - bb)) + (-shift_f - bb);
      s1.add(d);
      s1.lo += dl;
      const float q = d * d;
      s2.add(q);
      s2.lo += fmaf(d, d, -q) + 2.0f * d * dl;
      ++cnt;
      my_steps += static_cast<unsigned long long>(L.n);
      ++path;
      if (path < path_end) {
        L.X[0] = x0[0];
        L.X[1] = x0[1];
        L.X[2] = x0[2];
        L.Y = 1.f;
        L.Z = 0.f;
        L.n = 0;
        L.pp = philox_path(static_cast<uint32_t>(path), node, 0u, a.rk);
      } else {
        // sums of v = s - shift_f; with e = shift - shift_f the partial holds
        // sum (v - e) = S1 - n e and sum (v - e)^2 = S2 - 2 e S1 + n e^2
        const double n_d = static_cast<double>(cnt);
        const double S1 = static_cast<double>(s1.hi) + static_cast<double>(s1.lo);
        const double S2 = static_cast<double>(s2.hi) + static_cast<double>(s2.lo);
        const double e = shift - static_cast<double>(shift_f);
        a.partial[chunk] = ChunkPartial{n_d, S1 - n_d * e, S2 - 2.0 * e * S1 + n_d * e * e};
        active = false;
        need = true;
      }
    }
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    my_steps += __shfl_xor_sync(kFull, my_steps, m);
    my_capped += __shfl_xor_sync(kFull, my_capped, m);
    my_bad += __shfl_xor_sync(kFull, my_bad, m);
  }
  if (lane == 0) {
    if (my_steps) atomicAdd(&a.counters[0], my_steps);
    if (my_capped) atomicAdd(&a.counters[1], my_capped);
    if (my_bad) atomicAdd(&a.counters[2], my_bad);
  }
}



}  // namespace pdd
