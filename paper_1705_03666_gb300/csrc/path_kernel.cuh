// path_kernel.cuh -- the interface-node path kernel (stage one of PDD).
//
// One persistent launch advances every (node, path) of a wave of the global,
// node-major path index space g = node * n_paths + p.  Each lane owns one
// path at a time; when its path exits the lane takes the next path from its
// warp's stash of set-up paths (refilled 32 indices at a time from an atomic
// cursor), so no lane waits for a long path of another node (lane refill) and
// the only idle time is at the very end of the wave.
// Ended paths are parked per warp and scored 32 at a time, and the scores are
// added at once to exact per-node integer sums (nodefix.cuh), so the per-node
// mean and standard error do not depend on which lane ran which path and no
// per-path score is stored (the gradient mode keeps a per-path record for its
// Jacobian reduction).
//
// Per step (Eq. 2.8, Dirichlet/elliptic reduction of Sec. 2.2, left-point rule):
//   X' = X + b(X) dt + sigma sqrt(dt) xi,  Y' = Y e^{c(X) dt},  Z' = Z + f(X) Y dt,
// then the exit test: hard exit when X' leaves the closed domain (exit point =
// first crossing of the segment), else, with the bridge test, exit when
// U < P = 1 - prod_j (1 - exp(-2 d_j d'_j / (sigma^2 dt))) over faces with
// 2 d_j d'_j < 18 sigma^2 dt (exit point = X' projected on the face with the
// largest term).  P is accumulated without cancellation (bridge_exit) and
// near-ties of the FP32 path are decided in FP64.  Both tests sit behind one
// screen: the smallest d d' (> 0 proves X' inside) and a union bound on P
// above which no crossing is possible, so most steps form neither.
// Score = g(X_tau) Y' + Z' (Eq. 2.7).
#pragma once

#include "common.cuh"
#include "models.cuh"
#include "nodefix.cuh"

namespace pdd {

// Threads per block of the persistent path kernels, by path precision.  With
// 128-thread blocks ptxas gives the binary32 kernels ~70 registers and the
// SM holds 7 blocks (28 warps); with 256-thread blocks it held them to 64
// registers for 4 blocks (32 warps), and the 3-D solve ran 840 against
// 836 ms.  The FP64 kernels keep 256-thread blocks (their 2-D two-stage run
// was 11.4 against 13.0 ms).
template <typename R>
constexpr int kPathBlockOf = sizeof(R) == 4 ? 128 : 256;

struct PathArgs {
  const double *nodes;          // [n_nodes][D]
  uint64_t n_paths;             // paths per node
  uint64_t path_offset;         // first path index
  uint32_t node_offset;         // stream index of node 0 (node j draws node_offset + j)
  uint64_t begin, end;          // global index range of this launch (a wave)
  unsigned long long *cursor;   // queue cursor for this wave (starts at 0)
  unsigned long long *counters; // [0] path steps, [1] capped, [2] bad nodes
  NodeFix *fix;                 // forward mode: per-node exact sums [n_nodes]
  void *score;                  // gradient mode: GradRec[end - begin]
  double *dump_score;           // forward mode, optional: score per path [end - begin]
  double *dump_exit;            // forward mode, optional: exit point per path [end - begin][D]
  int32_t *steps;               // [end - begin] or null
  RoundKeys rk;
  double inv_s2dt;              // 1 / (sigma^2 dt)
  double dt_d, sdt_d, thr_d;    // FP64 path: dt, sigma sqrt(dt), 9 sigma^2 dt
  double ecdt_d;                // e^{c dt} for constant killing (FP64)
  float dt_f, sdt_f, thr_f;     // FP32 path
  float l2cdt_f;                // c dt log2(e) for constant killing (FP32)
  int32_t max_steps;
  int32_t bridge;
  float lr_scale;               // sqrt(dt) / sigma (gradient mode)
  ModelConst mc;
};

// Constant killing: Y_n = e^{c n dt}.  Every path runs through the same
// sequence Y_0, Y_1, ..., so a rounded recurrence Y <- Y e^{c dt} would carry
// the same rounding error into every path (in binary32 it drifts by ~1e-5
// over 500 steps); the FP32 path therefore evaluates Y_n from n directly
// (exp2 of n c dt log2 e, a few ulp, no accumulation).  In FP64 the
// recurrence is accurate to n ulp and is kept.
// log2 of a face count (the union bound's factor), counts 1 .. 6.
constexpr float kLog2Count[7] = {0.0f, 0.0f, 1.0f, 1.5849625007211562f, 2.0f,
                                 2.321928094887362f, 2.584962500721156f};

template <typename R> struct StepConst;
template <> struct StepConst<float> {
  float dt, sdt, thr, l2cdt, inv_s2dt;
  float b2;    // -2 log2(e) / (sigma^2 dt): exp(-2 m / (sigma^2 dt)) = 2^(b2 m)
  float boff;  // 0 with the bridge test, -inf without (every bound below is 0)
  StepConst() = default;
  __device__ __forceinline__ StepConst(const PathArgs &a)
      : dt(a.dt_f), sdt(a.sdt_f), thr(a.thr_f), l2cdt(a.l2cdt_f),
        inv_s2dt(static_cast<float>(a.inv_s2dt)),
        b2(static_cast<float>(-2.0 * 1.4426950408889634 * a.inv_s2dt)),
        boff(a.bridge ? 0.0f : -INFINITY) {}
  // half-space crossing probability for a step with d d' = m
  __device__ __forceinline__ float cross_p(float m) const { return ex2_approx(b2 * m); }
  // Bound on every crossing probability of a step whose smallest d d' over
  // D candidate faces is m: 1 - prod_j (1 - p_j) <= D p(m), raised by the
  // factor 2^(2^-12) = 1 + 1.7e-4, which covers the near-tie window (2^-18
  // relative) and the rounding of the exponents (< 1e-5 relative for the
  // probabilities above 2^-26 that a uniform can fall below).  0 without the
  // bridge test.
  template <int D> __device__ __forceinline__ float cross_bound(float m) const {
    constexpr float kOff = kLog2Count[D] + 2.44140625e-4f;
    return ex2_approx(fmaf(b2, m, kOff + boff));
  }
  __device__ __forceinline__ float kill(float, int32_t n_next) const {
    return ex2_approx(static_cast<float>(n_next) * l2cdt);
  }
  // e^{-a} for a >= 0 (hardware exp2, ~2 ulp; a near-tie decision is redone
  // in FP64 by the caller).
  __device__ __forceinline__ float exp_neg(float a) const {
    return ex2_approx(-1.4426950408889634f * a);
  }
};
template <> struct StepConst<double> {
  double dt, sdt, thr, e, inv_s2dt;
  double boff;  // 0 with the bridge test, -inf without
  __device__ __forceinline__ StepConst(const PathArgs &a)
      : dt(a.dt_d), sdt(a.sdt_d), thr(a.thr_d), e(a.ecdt_d), inv_s2dt(a.inv_s2dt),
        boff(a.bridge ? 0.0 : -INFINITY) {}
  __device__ __forceinline__ double kill(double y, int32_t) const { return y * e; }
  __device__ __forceinline__ double exp_neg(double a) const { return exp(-a); }
  __device__ __forceinline__ double cross_p(double m) const { return exp(-2.0 * m * inv_s2dt); }
  template <int D> __device__ __forceinline__ double cross_bound(double m) const {
    return static_cast<double>(D) * 1.0000001 * exp(boff - 2.0 * m * inv_s2dt);
  }
};

// FP32 step constants for time step dt, generator (1/2) sigma^2 Lap, a
// constant killing rate c and the bridge test on or off, rounded from the
// same FP64 expressions the host uses for PathArgs.
__device__ __forceinline__ StepConst<float> make_step_const(double dt, double sigma, double c,
                                                            bool bridge) {
  StepConst<float> k;
  k.dt = static_cast<float>(dt);
  k.sdt = static_cast<float>(sigma * sqrt(dt));
  k.thr = static_cast<float>(9.0 * sigma * sigma * dt);
  k.l2cdt = static_cast<float>(c * dt * 1.4426950408889634);
  k.inv_s2dt = static_cast<float>(1.0 / (sigma * sigma * dt));
  k.b2 = static_cast<float>(-2.0 * 1.4426950408889634 / (sigma * sigma * dt));
  k.boff = bridge ? 0.0f : -INFINITY;
  return k;
}

// FP64 re-decision of a near tie of the 2-D box bridge test from the same
// binary32 products d_j d'_j, kept out of line: it almost never runs, and
// inlined its FP64 code enlarged the 2-D kernels enough to stall them on
// instruction fetch (the gradient pass 156 -> 121 ms once it moved out; the
// 3-D kernel measured faster with its three-face form inline, 850 against
// 857 ms).
static __device__ __noinline__ bool bridge_box2_tie(float U, float inv_s2dt, float p0, float p1) {
  const float pr[2] = {p0, p1};
  double Pd = 0.0;
  const double s = 2.0 * static_cast<double>(inv_s2dt);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const double aa = s * static_cast<double>(pr[c]);
    if (aa < 18.0) {
      const double p = exp(-aa);
      Pd = Pd + p * (1.0 - Pd);
    }
  }
  return static_cast<double>(U) < Pd;
}

// Brownian-bridge exit probability over the faces within reach,
// P = 1 - prod_j (1 - p_j), p_j = exp(-2 d_j d'_j / (sigma^2 dt)), accumulated
// as P <- P + p_j (1 - P) (no cancellation, so accurate for tiny P).  FP32
// path: compensated binary32, and a decision with |U - P| within 2^-18 P is
// re-taken from the same distances in FP64.  Returns the face with the
// largest p_j, or -1 when no face is within reach or U >= P.
template <int NC, typename R>
__device__ __forceinline__ int bridge_exit(const StepConst<R> &k, const R *prod, const int *face,
                                           R U) {
  R P = R(0), pbest = R(-1);
  int jbest = -1;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const R aa = R(2) * prod[c] * k.inv_s2dt;
    if (aa < R(18)) {
      const R p = k.exp_neg(aa);
      P = P + p * (R(1) - P);
      if (p > pbest) { pbest = p; jbest = face[c]; }
    }
  }
  if (jbest < 0) return -1;
  bool take = U < P;
  if constexpr (sizeof(R) == 4) {
    if (fabsf(U - P) <= 3.814697265625e-06f * P) {  // near tie: FP64 from the same products
      if constexpr (NC == 2) {
        take = bridge_box2_tie(U, k.inv_s2dt, prod[0], prod[1]);
      } else {
        double Pd = 0.0;
        const double s = 2.0 * static_cast<double>(k.inv_s2dt);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const double aa = s * static_cast<double>(prod[c]);
          if (aa < 18.0) {
            const double p = exp(-aa);
            Pd = Pd + p * (1.0 - Pd);
          }
        }
        take = static_cast<double>(U) < Pd;
      }
    }
  }
  return take ? jbest : -1;
}

// FP64 re-decision of a near tie of the general-domain bridge test, from the
// same binary32 face distances (kept out of line: it almost never runs, and
// inlined it put FP64 instructions into the step code of every warp that
// reaches the bridge test).  2-D geometries.
template <class Geom>
static __device__ __noinline__ bool bridge_generic_tie(float U, float inv_s2dt, float x0, float x1,
                                                       float xn0, float xn1) {
  const float X[2] = {x0, x1}, Xn[2] = {xn0, xn1};
  double Pd = 0.0;
  const double s = 2.0 * static_cast<double>(inv_s2dt);
#pragma unroll
  for (int j = 0; j < Geom::kFaces; ++j) {
    const double aa = s * static_cast<double>(Geom::face_dist(j, X) * Geom::face_dist(j, Xn));
    if (aa < 18.0) {
      const double p = exp(-aa);
      Pd = Pd + p * (1.0 - Pd);
    }
  }
  return static_cast<double>(U) < Pd;
}

// Bridge over all faces of a general domain (distances from Geom::face_dist):
// P = 1 - prod_j (1 - p_j) accumulated as P + p (1 - P) over the faces with
// 2 d d' / (sigma^2 dt) < 18; FP32 near-ties decided in FP64.  Returns the
// face with the largest p_j if U < P, else -1.
template <class Geom, typename R>
__device__ __forceinline__ int bridge_generic(const StepConst<R> &k, const R *X, const R *Xn, R U) {
  R P = R(0), pbest = R(-1);
  int jbest = -1;
#pragma unroll
  for (int j = 0; j < Geom::kFaces; ++j) {
    const R aa = R(2) * (Geom::face_dist(j, X) * Geom::face_dist(j, Xn)) * k.inv_s2dt;
    if (aa < R(18)) {
      const R p = k.exp_neg(aa);
      P = P + p * (R(1) - P);
      if (p > pbest) { pbest = p; jbest = j; }
    }
  }
  if (jbest < 0) return -1;
  bool take = U < P;
  if constexpr (sizeof(R) == 4) {
    static_assert(Geom::D == 2, "the out-of-line tie test takes 2-D points");
    if (fabsf(U - P) <= 3.814697265625e-06f * P)
      take = bridge_generic_tie<Geom>(U, k.inv_s2dt, X[0], X[1], Xn[0], Xn[1]);
  }
  return take ? jbest : -1;
}

// Number of likelihood-ratio accumulators carried per path (gradient mode).
constexpr int kMaxLR = 16;

// FP64 re-decision of a near tie U ~ exp(-2 m / (sigma^2 dt)) (kept out of
// line: it almost never runs and would otherwise be inlined at every step).
static __device__ __noinline__ bool bridge_tie_fp64(float U, float mn, float inv_s2dt) {
  return static_cast<double>(U) <
         exp(-2.0 * static_cast<double>(mn) * static_cast<double>(inv_s2dt));
}

// Exit codes of em_step.
constexpr int kStepContinue = -2;
constexpr int kStepHardExit = -1;   // >= 0: bridge exit through that face

// One Euler-Maruyama step with the exit test.  On kStepContinue, X, Y, Z
// advance; on an exit, X keeps the start of the step, Xn receives its end,
// Y and Z receive their exit values, and the caller resolves the exit point
// (exit_score): the path kernel 32 paths at a time from its exit queue, the
// other kernels through path_unit.  With kLR the drift-weight likelihood-ratio
// sums L are advanced by this step's noise (the exiting step included).
template <class Model, class Geom, typename R, bool kLR, class Env>
__device__ __forceinline__ int em_step(const Env &a, const StepConst<R> &k, R *X, R &Y, R &Z,
                                       const R *xi, uint32_t uw, int32_t n, R *Xn, R *L) {
  constexpr int D = Model::D;
  R b[D];
  R f = R(0);
#pragma unroll
  for (int d = 0; d < D; ++d) b[d] = R(0);
  if constexpr (kLR) {
    Model::coeffs_lr(a.mc, X, b, f, xi, L);
  } else if constexpr (Model::kDrift || Model::kSource) {
    Model::coeffs(a.mc, X, b, f);
  }
  // (an axis without drift skips b dt: X + 0 dt is X exactly, so the result
  // is the same)
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if ((Model::kDriftAxes >> d) & 1u)
      Xn[d] = X[d] + b[d] * k.dt + k.sdt * xi[d];
    else
      Xn[d] = X[d] + k.sdt * xi[d];
  }
  R Zn = Z;
  if constexpr (Model::kSource) Zn = Z + f * Y * k.dt;
  R Yn = Y;
  if constexpr (Model::kKill == 1) Yn = k.kill(Y, n + 1);
  Y = Yn;
  Z = Zn;
  if constexpr (!Geom::kFastScreen) {
    // general domains: a lower bound on the smallest d d' (> 0: X' inside)
    // and the union bound over all faces screen the step; below the bound,
    // the exact tests (every face within reach, P = 1 - prod (1 - p_j))
    const R mnb = Geom::screen_lb(X, Xn);
    const R U = unif<R>(uw);
    if (!(mnb > R(0)) || U < k.template cross_bound<Geom::kFaces>(mnb)) {
      if (!Geom::inside_closed(Xn)) return kStepHardExit;
      if (a.bridge) {
        const int jbest = bridge_generic<Geom, R>(k, X, Xn, U);
        if (jbest >= 0) return jbest;
      }
    }
  } else {
    const R mn = Geom::screen_mn(X, Xn);
    // mn > 0 puts X' strictly inside.  U lies above every crossing
    // probability the step can have (and above its near-tie window) at most
    // steps: one bound decides that, and the probability itself is formed
    // only below it.  Both tests share one branch.
    const R U = unif<R>(uw);
    const R bnd = k.template cross_bound<D>(mn);
    if (!(mn > R(0)) || U < bnd) {
      if (!(mn > R(0)) && !Geom::inside_closed(Xn)) return kStepHardExit;
      if (U < bnd) {
        // A step within reach of one face crosses with
        // exp(-2 min d d' / (sigma^2 dt)); a step within reach of two or more
        // faces (an edge or a corner) takes the general combination.
        R prod[D];
        int face[D];
        Geom::screen(X, Xn, prod, face);
        bool cross;
        if (Geom::second_min(prod) < k.thr) {
          cross = bridge_exit<D, R>(k, prod, face, U) >= 0;
        } else {
          const R p = k.cross_p(mn);
          cross = U < p;
          if constexpr (sizeof(R) == 4) {
            if (fabsf(U - p) <= 3.814697265625e-06f * p) cross = bridge_tie_fp64(U, mn, k.inv_s2dt);
          }
        }
        if (cross) {
          int jbest = face[0];
          R pmin = prod[0];
#pragma unroll
          for (int d = 1; d < D; ++d)
            if (prod[d] < pmin) { pmin = prod[d]; jbest = face[d]; }
          return jbest;
        }
      }
    }
  }
#pragma unroll
  for (int d = 0; d < D; ++d) X[d] = Xn[d];
  return kStepContinue;
}

// Exit point of a step that left the domain (first crossing of X -> Xn) or
// crossed a face by the bridge (Xn projected on it), and the path's score
// g(X_tau) Y + Z (Eq. 2.7).
template <class Model, class Geom, typename R>
__device__ __forceinline__ R exit_score(const ModelConst &mc, int code, const R *X, const R *Xn,
                                        R Y, R Z, R *xe) {
  constexpr int D = Model::D;
  if (code == kStepHardExit) {
    Geom::segment_exit(X, Xn, xe);
  } else {
#pragma unroll
    for (int d = 0; d < D; ++d) xe[d] = Xn[d];
    Geom::project(code, xe);
  }
  return Model::g(mc, xe) * Y + Z;
}

// Word whose bytes 3, 2, 1 are the low bytes of c, b, a: the bridge uniform
// of a 3-D step comes from bits the Box-Muller maps (bits 9..31) do not use.
__device__ __forceinline__ uint32_t low_bytes_word(uint32_t a, uint32_t b, uint32_t c) {
  return __byte_perm(__byte_perm(a, b, 0x0400u), c, 0x4210u);
}

// Random numbers of the four-step unit that starts at step n = 4q: normals
// z[D j .. D j + D - 1] and the bridge-uniform word u[j] of step n + j, from
// the twelve words w0..w11 of Philox blocks 3q, 3q+1, 3q+2.  d <= 2: step
// 4q + j takes BM(w[2j], w[2j+1]) (d = 1: the first) and the uniform word
// w[8+j].  d = 3: normals z0..z11 = BM of the word pairs (w0,w1) ..
// (w10,w11), step 4q + j takes z[3j..3j+2] and low_bytes_word(w[3j],
// w[3j+1], w[3j+2]).  Either way 0.75 blocks per step, the least that holds
// the step's normals and a 23-bit uniform.
template <int D, typename R>
__device__ __forceinline__ void unit_randoms(int32_t n, const PhiloxPath &pp, const RoundKeys &rk,
                                             R *z, uint32_t *u) {
  if constexpr (D == 3) {
    const uint32_t q3 = 3u * (static_cast<uint32_t>(n) >> 2);
    const uint4 A = philox10_path(q3, pp, rk);
    const uint4 B = philox10_path(q3 + 1u, pp, rk);
    const uint4 C = philox10_path(q3 + 2u, pp, rk);
    box_muller<R>(A.x, A.y, z[0], z[1]);
    box_muller<R>(A.z, A.w, z[2], z[3]);
    box_muller<R>(B.x, B.y, z[4], z[5]);
    box_muller<R>(B.z, B.w, z[6], z[7]);
    box_muller<R>(C.x, C.y, z[8], z[9]);
    box_muller<R>(C.z, C.w, z[10], z[11]);
    u[0] = low_bytes_word(A.x, A.y, A.z);
    u[1] = low_bytes_word(A.w, B.x, B.y);
    u[2] = low_bytes_word(B.z, B.w, C.x);
    u[3] = low_bytes_word(C.y, C.z, C.w);
  } else {
    const uint32_t q3 = 3u * (static_cast<uint32_t>(n) >> 2);
    const uint4 A = philox10_path(q3, pp, rk);
    const uint4 B = philox10_path(q3 + 1u, pp, rk);
    const uint4 C = philox10_path(q3 + 2u, pp, rk);
    const uint32_t w[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      R z1;
      box_muller<R>(w[2 * j], w[2 * j + 1], z[D * j], z1);
      if constexpr (D == 2) z[D * j + 1] = z1;
    }
    u[0] = C.x;
    u[1] = C.y;
    u[2] = C.z;
    u[3] = C.w;
  }
}

// One loop unit of a path: up to four steps, with the random numbers of
// unit_randoms.  They are formed before the unit's first step: they do not
// depend on the path, so their integer work can interleave with the steps'
// floating-point work.  n counts the steps taken; the unit stops at an exit
// (returns its code, X the start and Xn the end of the exiting step) or at
// max_steps (returns kStepContinue).
template <class Model, class Geom, typename R, bool kLR, bool kSplitCap, class Env>
__device__ __forceinline__ int path_unit_code(const Env &a, const StepConst<R> &k,
                                              const PhiloxPath &pp, const RoundKeys &rk,
                                              int32_t max_steps, R *X, R &Y, R &Z, int32_t &n,
                                              R *Xn, R *L) {
  constexpr int D = Model::D;
  int code;
  R z[4 * D];
  uint32_t u[4];
  unit_randoms<D, R>(n, pp, rk, z, u);
  // kSplitCap: a unit that cannot reach the step cap tests only for exits;
  // one that can (rare: a path near max_steps) takes the steps one at a time
  // with the cap test, its random numbers shifted down by static indices.
  // Without it (kernels whose own body is large, where the second copy of
  // the unit cost more than the tests it saves), every step tests both.
  if (!kSplitCap) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      code = em_step<Model, Geom, R, kLR>(a, k, X, Y, Z, z + D * j, u[j], n, Xn, L);
      ++n;
      if (code != kStepContinue || n >= max_steps) break;
    }
  } else if (n <= max_steps - 4) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      code = em_step<Model, Geom, R, kLR>(a, k, X, Y, Z, z + D * j, u[j], n, Xn, L);
      ++n;
      if (code != kStepContinue) break;
    }
  } else {
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      code = em_step<Model, Geom, R, kLR>(a, k, X, Y, Z, z, u[0], n, Xn, L);
      ++n;
      if (code != kStepContinue || n >= max_steps) break;
#pragma unroll
      for (int i = 0; i < 3 * D; ++i) z[i] = z[i + D];
#pragma unroll
      for (int i = 0; i < 3; ++i) u[i] = u[i + 1];
    }
  }
  return code;
}

// path_unit_code followed, at an exit, by the path's score (returns true,
// score in s, exit point in xe).
template <class Model, class Geom, typename R, bool kLR, class Env>
__device__ __forceinline__ bool path_unit(const Env &a, const StepConst<R> &k, const PhiloxPath &pp,
                                          const RoundKeys &rk, int32_t max_steps, R *X, R &Y,
                                          R &Z, int32_t &n, R &s, R *xe, R *L) {
  R Xn[Model::D];
  const int code =
      path_unit_code<Model, Geom, R, kLR, false>(a, k, pp, rk, max_steps, X, Y, Z, n, Xn, L);
  if (code == kStepContinue) return false;
  s = exit_score<Model, Geom, R>(a.mc, code, X, Xn, Y, Z, xe);
  return true;
}

// Per-path record of the gradient mode: score, exit point, and the
// likelihood-ratio sums L_j (already scaled by sqrt(dt)/sigma).
struct GradRec {
  float s, x, y, z;
  float L[kMaxLR];
};

// Gradient mode: the record's first four words (score and exit point) with
// the step count, and the likelihood-ratio sums.
template <int D, typename R>
__device__ __forceinline__ void write_score(const PathArgs &a, uint64_t slot, R s, int32_t st,
                                            const R *xe) {
  float4 *o = reinterpret_cast<float4 *>(static_cast<GradRec *>(a.score) + slot);
  o[0] = make_float4(static_cast<float>(s), static_cast<float>(xe[0]),
                     D > 1 ? static_cast<float>(xe[D > 1 ? 1 : 0]) : 0.f,
                     D > 2 ? static_cast<float>(xe[D > 2 ? 2 : 0]) : 0.f);
  if (a.steps) a.steps[slot] = st;
}
template <typename R>
__device__ __forceinline__ void write_lr_sums(const PathArgs &a, uint64_t slot, const R *L) {
  float4 *o = reinterpret_cast<float4 *>(static_cast<GradRec *>(a.score) + slot);
  const float c = a.lr_scale;
#pragma unroll
  for (int q = 0; q < kMaxLR / 4; ++q)
    o[1 + q] = make_float4(c * static_cast<float>(L[4 * q]), c * static_cast<float>(L[4 * q + 1]),
                           c * static_cast<float>(L[4 * q + 2]), c * static_cast<float>(L[4 * q + 3]));
}

// Node of global path index g (32-bit division when the indices fit).
__device__ __forceinline__ uint64_t path_node(const PathArgs &a, uint64_t g) {
  if (a.end <= 0xffffffffull)
    return static_cast<uint32_t>(g) / static_cast<uint32_t>(a.n_paths);
  return g / a.n_paths;
}

// Forward mode: optional per-path record (score, exit step, exit point) for
// parity checks, in the caller's buffers.
template <int D, typename R>
__device__ __forceinline__ void dump_path(const PathArgs &a, uint64_t slot, R s, int32_t st,
                                          const R *xe) {
  if (a.dump_score) a.dump_score[slot] = static_cast<double>(s);
  if (a.steps) a.steps[slot] = st;
  if (a.dump_exit) {
#pragma unroll
    for (int d = 0; d < D; ++d) a.dump_exit[slot * D + d] = static_cast<double>(xe[d]);
  }
}

// Per-warp staging in shared memory (one column per lane).  Claiming and
// setting up a path (atomic, node division, Philox key, FP64 node load) and
// scoring an ended path (exit point, accurate g) happen once per path, at
// times that differ from lane to lane: done where they occur, each would run
// with one lane of the warp active.  Instead a warp claims 32 consecutive
// paths at once and sets them all up with every lane busy (StartStash), and
// ended paths are parked (ExitQueue) and scored 32 at a time.  Every path
// writes its own slot, so the results do not depend on this order.
template <int D, typename R>
struct StartStash {
  unsigned long long slot[32];  // index in the wave
  uint32_t w0[32], w1[32];      // PhiloxPath words (tag 0)
  R x[D][32];                   // start point
};
template <int D, typename R>
struct ExitQueue {
  unsigned long long slot[32];
  int32_t st[32], code[32];     // step count (or -max_steps) and exit code
  R x[D][32], xn[D][32], y[32], z[32];
};
template <int D, typename R>
struct PathStage {
  StartStash<D, R> start;
  ExitQueue<D, R> exit;
};

// Exit code of a path stopped by the step cap: scored at the projection of
// its last point on the nearest face.
constexpr int kStepCapped = -3;

// Called by all 32 lanes: claim the next 32 indices of the wave, set each up,
// score at once the ones that start on the boundary (tau = 0, u = g, Eq. 2.1)
// or outside the closed domain (invalid input: NaN, counted), and stage the
// interior ones.  Returns how many were staged (warp-uniform).
template <class Model, class Geom, typename R, bool kLR>
__device__ __forceinline__ int stage_starts(const PathArgs &a, StartStash<Model::D, R> &st,
                                            unsigned long long span, bool &exhausted,
                                            unsigned long long &my_bad) {
  constexpr int D = Model::D;
  const unsigned lane = threadIdx.x & 31u;
  __syncwarp();  // earlier reads of the stash are done
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(a.cursor, 32ull);
  base = __shfl_sync(kFull, base, 0);
  if (base + 32 >= span) exhausted = true;
  const unsigned long long q = base + lane;
  bool interior = false;
  R x[D];
  PhiloxPath pp{0, 0, 0};
  uint64_t node = 0;
  R s0 = R(0);
  if (q < span) {
    const unsigned long long g = a.begin + q;
    node = path_node(a, g);
    const uint64_t path = g - node * a.n_paths + a.path_offset;
    pp = philox_path(static_cast<uint32_t>(path), static_cast<uint32_t>(node) + a.node_offset, 0u,
                     a.rk);
#pragma unroll
    for (int d = 0; d < D; ++d) x[d] = static_cast<R>(a.nodes[node * D + d]);
    interior = Geom::inside_open(x);
    if (!interior) {
      s0 = Model::g(a.mc, x);
      if (!Geom::inside_closed(x)) {
        s0 = R(NAN);
        ++my_bad;
      }
      if constexpr (kLR) {
        R L0[kMaxLR];
#pragma unroll
        for (int j = 0; j < kMaxLR; ++j) L0[j] = R(0);
        write_score<D, R>(a, q, s0, 0, x);
        write_lr_sums<R>(a, q, L0);
      } else {
        dump_path<D, R>(a, q, s0, 0, x);
      }
    }
  }
  if constexpr (!kLR) {
    // starts on the boundary (u = g, tau = 0) or outside the closed domain
    // (NaN) go straight into the node's sums
    const bool at_bnd = q < span && !interior;
    if (__any_sync(kFull, at_bnd))
      fix_commit<R>(a.fix, at_bnd, node, s0, false, true);
  }
  const unsigned im = __ballot_sync(kFull, interior);
  if (interior) {
    const int e = __popc(im & ((1u << lane) - 1u));
    st.slot[e] = q;
    st.w0[e] = pp.r0_w0;
    st.w1[e] = pp.r0_w1;
#pragma unroll
    for (int d = 0; d < D; ++d) st.x[d][e] = x[d];
  }
  __syncwarp();
  return __popc(im);
}

// Called by all 32 lanes: score the first cnt parked paths, one per lane, and
// add the scores to their nodes' sums (gradient mode: write the record's score
// and exit point; the likelihood-ratio sums were written when the path ended).
template <class Model, class Geom, typename R, bool kLR>
__device__ __forceinline__ void flush_exits(const PathArgs &a, ExitQueue<Model::D, R> &q, int cnt) {
  constexpr int D = Model::D;
  const int lane = static_cast<int>(threadIdx.x & 31u);
  __syncwarp();
  R s = R(0);
  uint64_t node = 0;
  bool capped = false;
  if (lane < cnt) {
    R X[D], Xn[D], xe[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      X[d] = q.x[d][lane];
      Xn[d] = q.xn[d][lane];
    }
    const int code = q.code[lane];
    capped = code == kStepCapped;
    if (capped) {
#pragma unroll
      for (int d = 0; d < D; ++d) xe[d] = X[d];
      Geom::project(Geom::nearest_face(X), xe);
      s = Model::g(a.mc, xe) * q.y[lane] + q.z[lane];
    } else {
      s = exit_score<Model, Geom, R>(a.mc, code, X, Xn, q.y[lane], q.z[lane], xe);
    }
    if constexpr (kLR) {
      write_score<D, R>(a, q.slot[lane], s, q.st[lane], xe);
    } else {
      node = path_node(a, a.begin + q.slot[lane]);
      dump_path<D, R>(a, q.slot[lane], s, q.st[lane], xe);
    }
  }
  if constexpr (!kLR) fix_commit<R>(a.fix, lane < cnt, node, s, capped, false);
  __syncwarp();
}

template <class Model, class Geom, typename R, bool kLR = false>
__global__ void __launch_bounds__(kPathBlockOf<R>)
path_kernel(const __grid_constant__ PathArgs a) {
  constexpr int D = Model::D;
  constexpr int NL = kLR ? kMaxLR : 1;
  __shared__ PathStage<D, R> stage_all[kPathBlockOf<R> / 32];
  PathStage<D, R> &stage = stage_all[threadIdx.x >> 5];
  R L[NL];
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  const StepConst<R> k(a);
  const unsigned long long span = a.end - a.begin;
  R X[D], Xn[D];
  R Y = R(1), Z = R(0);
  PhiloxPath pp{0, 0, 0};
  unsigned long long slot = 0;
  int32_t n = 0;
  bool active = false;
  int n_start = 0, n_exit = 0;  // stash / queue fill (warp-uniform)
  bool exhausted = false;       // the wave's indices are all claimed (warp-uniform)
  unsigned long long my_steps = 0, my_capped = 0, my_bad = 0;

  for (;;) {
    // ---- idle lanes take staged paths; the stash is refilled when empty
    unsigned needmask = __ballot_sync(kFull, !active);
    if (needmask) {
    while (needmask) {
      if (n_start == 0) {
        if (exhausted) break;
        n_start = stage_starts<Model, Geom, R, kLR>(a, stage.start, span, exhausted, my_bad);
        continue;
      }
      const int cnt = __popc(needmask);
      const int take = cnt < n_start ? cnt : n_start;
      if (!active) {
        const int r = __popc(needmask & lt_mask);
        if (r < take) {
          const int e = n_start - 1 - r;
          slot = stage.start.slot[e];
          pp.r0_w0 = stage.start.w0[e];
          pp.r0_w1 = stage.start.w1[e];
          pp.tag = 0u;
#pragma unroll
          for (int d = 0; d < D; ++d) X[d] = stage.start.x[d][e];
          Y = R(1);
          Z = R(0);
          n = 0;
#pragma unroll
          for (int j = 0; j < NL; ++j) L[j] = R(0);
          active = true;
        }
      }
      n_start -= take;
      needmask = __ballot_sync(kFull, !active);
    }
    if (!__any_sync(kFull, active)) break;
    }

    // ---- advance the lane's path by one unit
    int code = kStepContinue;
    bool done = false;
    if (active) {
      code = path_unit_code<Model, Geom, R, kLR, true>(a, k, pp, a.rk, a.max_steps, X, Y, Z, n, Xn, L);
      done = code != kStepContinue || n >= a.max_steps;
      if (done) {
        my_steps += static_cast<unsigned long long>(n);
        if (code == kStepContinue) {
          code = kStepCapped;
          ++my_capped;
        }
      }
    }

    // ---- ended paths: parked, and scored 32 at a time (gradient mode writes
    // the likelihood-ratio sums at once)
    const unsigned dm = __ballot_sync(kFull, done);
    if (dm) {
      const int nd = __popc(dm);
      if (n_exit + nd > 32) {
        flush_exits<Model, Geom, R, kLR>(a, stage.exit, n_exit);
        n_exit = 0;
      }
      if (done) {
        if constexpr (kLR) write_lr_sums<R>(a, slot, L);
        const int e = n_exit + __popc(dm & lt_mask);
        ExitQueue<D, R> &q = stage.exit;
        q.slot[e] = slot;
        q.st[e] = code == kStepCapped ? -a.max_steps : n;
        q.code[e] = code;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          q.x[d][e] = X[d];
          q.xn[d][e] = Xn[d];
        }
        q.y[e] = Y;
        q.z[e] = Z;
        active = false;
      }
      n_exit += nd;
    }
  }
  if (n_exit > 0) flush_exits<Model, Geom, R, kLR>(a, stage.exit, n_exit);

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
