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
  int32_t K;
  unsigned long long *cursor;  // [4]: one per family
  unsigned long long *counters;  // [0] path steps, [1] capped, [2] bad nodes
  NodeFix *fix;             // [n] exact per-node sums (both passes add to them)
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

// Ended paths of a warp, parked until 32 can be scored together: the start
// and end of the last step (or the position of a capped path), Y, Z, the
// exit code and the node and problem the path belongs to.
struct BatchExitQueue {
  float x[3][32], xn[3][32];
  float y[32], z[32];
  int32_t code[32];
  uint32_t node[32];
  int32_t prob[32];
};

// Called by all 32 lanes: score the first cnt parked paths, one per lane,
// and add the scores to their nodes' exact sums.
template <class Model, class Geom>
__device__ __forceinline__ void batch_flush(const BatchArgs &a, BatchExitQueue &q, int cnt) {
  constexpr int D = Model::D;
  const int lane = static_cast<int>(threadIdx.x & 31u);
  __syncwarp();
  float s = 0.f;
  uint32_t node = 0;
  bool capped = false;
  if (lane < cnt) {
    float X[D], Xn[D], xe[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      X[d] = q.x[d][lane];
      Xn[d] = q.xn[d][lane];
    }
    const int code = q.code[lane];
    const ModelConst &mc = a.probs[q.prob[lane]].mc;
    node = q.node[lane];
    capped = code == kStepCapped;
    if (capped) {
#pragma unroll
      for (int d = 0; d < D; ++d) xe[d] = X[d];
      Geom::project(Geom::nearest_face(X), xe);
      s = Model::g(mc, xe) * q.y[lane] + q.z[lane];
    } else {
      s = exit_score<Model, Geom, float>(mc, code, X, Xn, q.y[lane], q.z[lane], xe);
    }
  }
  fix_commit<float>(a.fix, lane < cnt, node, s, capped, false);
  __syncwarp();
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
  constexpr int D = M::D;
  __shared__ BatchExitQueue queue_all[kBatchBlock / 32];
  BatchExitQueue &queue = queue_all[threadIdx.x >> 5];
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  // this family's positions and chunks
  const int64_t jlo = a.cstart[C], jhi = a.cstart[C + 1];
  if (jlo >= jhi) return;
  const uint64_t c_lo = static_cast<uint64_t>(a.chunk_off[jlo]);
  const uint64_t c_hi = static_cast<uint64_t>(a.chunk_off[jhi]);
  unsigned long long *cursor = a.cursor + C;
  float X[3] = {0.f, 0.f, 0.f}, Xn[3];
  float Y = 1.f, Z = 0.f;
  int32_t n = 0;
  PhiloxPath pp{0, 0, 0};
  float x0[3] = {0.f, 0.f, 0.f};  // the chunk's node, converted once per chunk
  StepConst<float> k;
  int32_t pi = 0;
  uint32_t node = 0;
  int64_t path = 0, path_end = 0;
  bool active = false, need = true;
  int n_exit = 0;  // parked paths (warp-uniform)
  unsigned long long my_steps = 0, my_capped = 0, my_bad = 0;

  for (;;) {
    // ---- lanes without a path take the next chunk (warp-aggregated claims)
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
#pragma unroll
          for (int d = 0; d < 3; ++d) x0[d] = static_cast<float>(a.nodes[i * 3 + d]);
          if (!batch_inside<M, G>(x0)) {
            // node on (or, invalid, outside) the boundary: every path scores g
            const bool closed = batch_closed<M, G>(x0);
            if (!closed) ++my_bad;
            fix_add_repeated<float>(a.fix, node, closed ? M::g(P.mc, x0) : NAN,
                                    path_end - path);
            need = true;
          } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) X[d] = x0[d];
            Y = 1.f;
            Z = 0.f;
            n = 0;
            pp = philox_path(static_cast<uint32_t>(path), node, 0u, a.rk);
            active = true;
          }
        }
      }
    }
    if (!__any_sync(kFull, active)) break;

    // ---- advance the lane's path by one unit
    int code = kStepContinue;
    bool done = false;
    if (active) {
      const BatchEnv env{a.probs[pi].mc, a.probs[pi].bridge};
      code = path_unit_code<M, G, float, false, true>(env, k, pp, a.rk, a.max_steps, X, Y, Z, n,
                                                     Xn, nullptr);
      done = code != kStepContinue || n >= a.max_steps;
      if (done) {
        my_steps += static_cast<unsigned long long>(n);
        if (code == kStepContinue) {
          code = kStepCapped;
          ++my_capped;
        }
      }
    }

    // ---- ended paths: parked, scored 32 at a time; the lane goes on with
    // the next path of its chunk at once
    const unsigned dm = __ballot_sync(kFull, done);
    if (dm) {
      const int nd = __popc(dm);
      if (n_exit + nd > 32) {
        batch_flush<M, G>(a, queue, n_exit);
        n_exit = 0;
      }
      if (done) {
        const int e = n_exit + __popc(dm & lt_mask);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          queue.x[d][e] = X[d];
          queue.xn[d][e] = Xn[d];
        }
        queue.y[e] = Y;
        queue.z[e] = Z;
        queue.code[e] = code;
        queue.node[e] = node;
        queue.prob[e] = pi;
        ++path;
        if (path < path_end) {
#pragma unroll
          for (int d = 0; d < 3; ++d) X[d] = x0[d];
          Y = 1.f;
          Z = 0.f;
          n = 0;
          pp = philox_path(static_cast<uint32_t>(path), node, 0u, a.rk);
        } else {
          active = false;
          need = true;
        }
      }
      n_exit += nd;
    }
  }
  if (n_exit > 0) batch_flush<M, G>(a, queue, n_exit);
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
