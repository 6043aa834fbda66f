// path_kernel.cuh -- the interface-node path kernel (stage one of PDD).
//
// One persistent launch advances every (node, path) of a wave of the global,
// node-major path index space g = node * n_paths + p.  Each lane owns one
// path at a time; when its path exits the lane takes the next index from a
// warp-aggregated atomic cursor, so no lane waits for a long path of another
// node (lane refill) and the only idle time is at the very end of the wave.
// A path's score and exit step go to a per-path slot; a separate reduction
// (reduce.cu) forms the per-node mean and standard error in a fixed order, so
// the result does not depend on which lane ran which path.
//
// Per step (Eq. 2.8, Dirichlet/elliptic reduction of Sec. 2.2, left-point rule):
//   X' = X + b(X) dt + sigma sqrt(dt) xi,  Y' = Y e^{c(X) dt},  Z' = Z + f(X) Y dt,
// then the exit test: hard exit when X' leaves the closed domain (exit point =
// first crossing of the segment), else, with the bridge test, exit when
// U < P = 1 - prod_j (1 - exp(-2 d_j d'_j / (sigma^2 dt))) over faces with
// 2 d_j d'_j < 18 sigma^2 dt (exit point = X' projected on the face with the
// largest term).  P is accumulated without cancellation (bridge_exit) and
// near-ties of the FP32 path are decided in FP64.
// Score = g(X_tau) Y' + Z' (Eq. 2.7).
#pragma once

#include "common.cuh"
#include "models.cuh"

namespace pdd {

constexpr int kPathBlock = 256;

struct PathArgs {
  const double *nodes;          // [n_nodes][D]
  uint64_t n_paths;             // paths per node
  uint64_t path_offset;         // first path index
  uint64_t begin, end;          // global index range of this wave
  unsigned long long *cursor;   // queue cursor for this wave (starts at 0)
  unsigned long long *counters; // [0] path steps, [1] capped, [2] bad nodes
  void *score;                  // R[end - begin]
  int32_t *steps;               // [end - begin] or null
  RoundKeys rk;
  double inv_s2dt;              // 1 / (sigma^2 dt)
  double dt_d, sdt_d, thr_d;    // FP64 path: dt, sigma sqrt(dt), 9 sigma^2 dt
  double ecdt_d;                // e^{c dt} for constant killing (FP64)
  float dt_f, sdt_f, thr_f;     // FP32 path
  float l2cdt_f;                // c dt log2(e) for constant killing (FP32)
  int32_t max_steps;
  int32_t bridge;
  ModelConst mc;
};

// Constant killing: Y_n = e^{c n dt}.  Every path runs through the same
// sequence Y_0, Y_1, ..., so a rounded recurrence Y <- Y e^{c dt} would carry
// the same rounding error into every path (in binary32 it drifts by ~1e-5
// over 500 steps); the FP32 path therefore evaluates Y_n from n directly
// (exp2 of n c dt log2 e, a few ulp, no accumulation).  In FP64 the
// recurrence is accurate to n ulp and is kept.
template <typename R> struct StepConst;
template <> struct StepConst<float> {
  float dt, sdt, thr, l2cdt, inv_s2dt;
  __device__ __forceinline__ StepConst(const PathArgs &a)
      : dt(a.dt_f), sdt(a.sdt_f), thr(a.thr_f), l2cdt(a.l2cdt_f),
        inv_s2dt(static_cast<float>(a.inv_s2dt)) {}
  __device__ __forceinline__ float kill(float, int32_t n_next) const {
    return exp2f(static_cast<float>(n_next) * l2cdt);
  }
};
template <> struct StepConst<double> {
  double dt, sdt, thr, e, inv_s2dt;
  __device__ __forceinline__ StepConst(const PathArgs &a)
      : dt(a.dt_d), sdt(a.sdt_d), thr(a.thr_d), e(a.ecdt_d), inv_s2dt(a.inv_s2dt) {}
  __device__ __forceinline__ double kill(double y, int32_t) const { return y * e; }
};

// Brownian-bridge exit probability over the faces within reach,
// P = 1 - prod_j (1 - p_j), p_j = exp(-2 d_j d'_j / (sigma^2 dt)), accumulated
// as P <- P + p_j (1 - P) (no cancellation, so accurate for tiny P).  FP32
// path: compensated binary32, and a decision with |U - P| within 2^-18 P is
// re-taken from the same distances in FP64.  Returns the face with the
// largest p_j, or -1 when no face is within reach or U >= P.
template <class Geom, typename R>
__device__ __forceinline__ int bridge_exit(const StepConst<R> &k, const R *X, const R *Xn,
                                           R U) {
  R P = R(0), pbest = R(-1);
  int jbest = -1;
#pragma unroll
  for (int j = 0; j < Geom::kFaces; ++j) {
    const R aa = R(2) * Geom::face_dist(j, X) * Geom::face_dist(j, Xn) * k.inv_s2dt;
    if (aa < R(18)) {
      const R p = m_exp(-aa);
      P = P + p * (R(1) - P);
      if (p > pbest) { pbest = p; jbest = j; }
    }
  }
  if (jbest < 0) return -1;
  bool take = U < P;
  if constexpr (sizeof(R) == 4) {
    if (fabsf(U - P) <= 3.814697265625e-06f * P) {  // near tie: FP64 from the same distances
      double Pd = 0.0;
      const double s = 2.0 * static_cast<double>(k.inv_s2dt);
#pragma unroll
      for (int j = 0; j < Geom::kFaces; ++j) {
        const double aa = s * static_cast<double>(Geom::face_dist(j, X)) *
                          static_cast<double>(Geom::face_dist(j, Xn));
        if (aa < 18.0) {
          const double p = exp(-aa);
          Pd = Pd + p * (1.0 - Pd);
        }
      }
      take = static_cast<double>(U) < Pd;
    }
  }
  return take ? jbest : -1;
}

// One Euler-Maruyama step with the exit test.  Returns true on exit, with
// the score in `s`.  X, Y, Z advance only when the path stays inside.
template <class Model, class Geom, typename R>
__device__ __forceinline__ bool em_step(const PathArgs &a, const StepConst<R> &k,
                                        R *X, R &Y, R &Z, const R *xi, uint32_t uw,
                                        int32_t n, R &s) {
  constexpr int D = Model::D;
  R b[D];
  R f = R(0);
#pragma unroll
  for (int d = 0; d < D; ++d) b[d] = R(0);
  if constexpr (Model::kDrift || Model::kSource) Model::coeffs(a.mc, X, b, f);
  R Xn[D];
#pragma unroll
  for (int d = 0; d < D; ++d) Xn[d] = X[d] + b[d] * k.dt + k.sdt * xi[d];
  R Zn = Z;
  if constexpr (Model::kSource) Zn = Z + f * Y * k.dt;
  R Yn = Y;
  if constexpr (Model::kKill == 1) Yn = k.kill(Y, n + 1);
  if (!Geom::inside_closed(Xn)) {
    R xe[D];
    Geom::segment_exit(X, Xn, xe);
    s = Model::g(a.mc, xe) * Yn + Zn;
    return true;
  }
  if (a.bridge && Geom::near_any(X, Xn, k.thr)) {
    const int jbest = bridge_exit<Geom, R>(k, X, Xn, unif<R>(uw));
    if (jbest >= 0) {
      R xe[D];
#pragma unroll
      for (int d = 0; d < D; ++d) xe[d] = Xn[d];
      Geom::project(jbest, xe);
      s = Model::g(a.mc, xe) * Yn + Zn;
      return true;
    }
  }
#pragma unroll
  for (int d = 0; d < D; ++d) X[d] = Xn[d];
  Y = Yn;
  Z = Zn;
  return false;
}

template <class Model, class Geom, typename R>
__global__ void __launch_bounds__(kPathBlock)
path_kernel(const __grid_constant__ PathArgs a) {
  constexpr int D = Model::D;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  const StepConst<R> k(a);
  R X[D];
  R Y = R(1), Z = R(0);
  PhiloxPath pp{0, 0, 0};
  uint64_t slot = 0;
  int32_t n = 0;
  bool active = false, need = true;
  unsigned long long my_steps = 0, my_capped = 0, my_bad = 0;
  R *score = static_cast<R *>(a.score);

  for (;;) {
    // ---- refill: lanes without a path take the next indices of the wave
    for (;;) {
      const unsigned needmask = __ballot_sync(kFull, need);
      if (!needmask) break;
      const int leader = __ffs(needmask) - 1;
      unsigned long long base = 0;
      if (static_cast<int>(lane) == leader)
        base = atomicAdd(a.cursor, static_cast<unsigned long long>(__popc(needmask)));
      base = __shfl_sync(kFull, base, leader);
      if (need) {
        need = false;
        const unsigned long long q = base + __popc(needmask & lt_mask);
        const unsigned long long g = a.begin + q;
        if (g < a.end) {
          slot = q;
          const uint64_t node = g / a.n_paths;
          const uint64_t path = g - node * a.n_paths + a.path_offset;
          pp = philox_path(static_cast<uint32_t>(path), static_cast<uint32_t>(node), 0u, a.rk);
#pragma unroll
          for (int d = 0; d < D; ++d) X[d] = static_cast<R>(a.nodes[node * D + d]);
          Y = R(1);
          Z = R(0);
          n = 0;
          if (!Geom::inside_open(X)) {
            // Node on the boundary: tau = 0, u = g (Eq. 2.1).  Outside the
            // closed domain: invalid input, NaN score, counted.
            R s = Model::g(a.mc, X);
            if (!Geom::inside_closed(X)) {
              s = R(NAN);
              ++my_bad;
            }
            score[slot] = s;
            if (a.steps) a.steps[slot] = 0;
            need = true;
          } else {
            active = true;
          }
        }
      }
    }
    if (!__any_sync(kFull, active)) break;
    if (!active) continue;

    // ---- advance the lane's path
    R s = R(0);
    bool done;
    if constexpr (D == 3) {
      // pair of steps 2m, 2m+1 from Philox blocks 2m and 2m+1
      const uint32_t j = static_cast<uint32_t>(n);  // n is even here
      const uint4 A = philox10_path(j, pp, a.rk);
      const uint4 B = philox10_path(j + 1u, pp, a.rk);
      R xi[3], e;
      box_muller<R>(A.x, A.y, xi[0], xi[1]);
      box_muller<R>(A.z, A.w, xi[2], e);
      done = em_step<Model, Geom, R>(a, k, X, Y, Z, xi, B.z, n, s);
      ++n;
      if (!done && n < a.max_steps) {
        R p, q;
        box_muller<R>(B.x, B.y, p, q);
        xi[0] = e;
        xi[1] = p;
        xi[2] = q;
        done = em_step<Model, Geom, R>(a, k, X, Y, Z, xi, B.w, n, s);
        ++n;
      }
    } else {
      const uint4 A = philox10_path(static_cast<uint32_t>(n), pp, a.rk);
      R xi[2], z1;
      box_muller<R>(A.x, A.y, xi[0], z1);
      if constexpr (D == 2) xi[1] = z1;
      done = em_step<Model, Geom, R>(a, k, X, Y, Z, xi, A.z, n, s);
      ++n;
    }
    int32_t st = n;
    if (!done && n >= a.max_steps) {
      // step cap: score at the projection on the nearest face, counted
      R xe[D];
#pragma unroll
      for (int d = 0; d < D; ++d) xe[d] = X[d];
      Geom::project(Geom::nearest_face(X), xe);
      s = Model::g(a.mc, xe) * Y + Z;
      st = -a.max_steps;
      ++my_capped;
      done = true;
    }
    if (done) {
      score[slot] = s;
      if (a.steps) a.steps[slot] = st;
      my_steps += static_cast<unsigned long long>(n);
      active = false;
      need = true;
    }
  }

  // ---- per-warp totals
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
