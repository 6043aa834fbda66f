// reflect.cu -- interface paths with reflecting faces: the mixed BVP of
// Eq. 2.4 (Robin data du/dN = phi u + psi on the reflecting part of the
// boundary) through the local-time system of Eq. 2.9: X is pushed back into
// the domain by the local time xi (dX = ... - N dxi), Y gains phi Y dxi and
// Z gains psi Y dxi.
//
// A step is the Euler-Maruyama step of the path kernel (same streams, tag 0)
// followed, for every reflecting face within bridge reach, by Lepingle's
// half-space reflection: with distances y (start) and y' (free end), the
// Brownian bridge's minimum is m = (y + y' - sqrt((y' - y)^2 - 2 sigma^2 dt
// ln U')) / 2, the local time L = max(0, -m), and the end point moves in by
// L.  U' for axis k comes from the tag-4 stream Philox((b, p, i, 4)): in 3-D
// word k of block b = n; in 2-D word 2 (n mod 2) + k of block b = n / 2, so
// one block serves two steps.  It matters only when a reflecting face is
// within reach (2 y y' / (sigma^2 dt) < 18; beyond, L = 0 for every
// U' >= 2^-24).  Along the local time the weights are integrated
// exactly with psi frozen at the end point's projection: Z += psi Y (e^{phi
// L} - 1) / phi, Y *= e^{phi L}; then the time part as in the path kernel
// (left point).  Absorbing faces keep the hard-exit and bridge tests.
// Y is formed as exp(n c dt + sum phi L) so binary32 rounding does not
// accumulate along the path.  Per step, one test over the reflecting faces
// (the reflection's own reach test) and one bound over the absorbing faces
// (smallest d d' > 0 and U above 2D exp(-2 min d d' / (sigma^2 dt))) skip
// the per-face work at most steps; the decisions are those of the per-face
// loops.
#include <cmath>
#include <cstring>

#include "ctx.hpp"
#include "models.cuh"
#include "path_kernel.cuh"
#include "reduce.cuh"
#include "warp_queue.cuh"

namespace pdd {

struct ReflectArgs {
  const double *nodes;
  uint64_t n_paths, path_offset, begin, end;
  uint32_t node_offset;          // stream index of node 0
  unsigned long long *cursor;
  unsigned long long *counters;  // [0] steps, [1] capped, [2] bad nodes
  void *score;
  int32_t *steps;
  int32_t *flags;                // per-node flags or null (rare events, atomicOr)
  double *exit;                  // exit point per path [end - begin][D] or null
  RoundKeys rk;
  double dt, sdt, s2dt, cdt, phi;  // dt, sigma sqrt(dt), sigma^2 dt, c dt, Robin phi
  // the binary32 step constants, rounded on the host (dt, sdt, s2dt, cdt, phi,
  // 1 / s2dt, b2, boff of ReflectConst): formed in the kernel from the FP64
  // fields, they were re-formed inside the step loop on the FP64 pipe
  float kf[8];
  int32_t mask;                    // bit j: face j reflects
  int32_t max_steps, bridge;
  ModelConst mc;
};

// Optional per-path exit point (parity checks).
template <int D, typename R>
__device__ __forceinline__ void dump_exit_point(double *exit, uint64_t slot, const R *x) {
  if (exit) {
#pragma unroll
    for (int d = 0; d < D; ++d) exit[slot * D + d] = static_cast<double>(x[d]);
  }
}

// Special functions of the reflection branch.  A reflecting problem's paths
// linger near their reflecting faces, so this branch runs, diverged, at most
// warp-steps: binary32 takes the hardware approximations (relative errors of
// order 1e-7 against the 1e-4 per-path and 1e-5 per-node parity bars),
// binary64 the accurate library functions.  expm1 stays accurate: its
// argument phi L is small, where exp(v) - 1 would cancel.
__device__ __forceinline__ float rb_exp(float x) { return exp_fast(x); }
__device__ __forceinline__ double rb_exp(double x) { return exp(x); }
__device__ __forceinline__ float rb_cos(float x) { return cos_approx(x); }   // |x| <= 1 here
__device__ __forceinline__ double rb_cos(double x) { return cos(x); }
__device__ __forceinline__ float rb_sin(float x) { return sin_approx(x); }
__device__ __forceinline__ double rb_sin(double x) { return sin(x); }
__device__ __forceinline__ float rb_sinpi(float x) { return sin_approx(3.14159265358979324f * x); }
__device__ __forceinline__ double rb_sinpi(double x) { return sinpi(x); }
__device__ __forceinline__ float rb_cospi(float x) { return cos_approx(3.14159265358979324f * x); }
__device__ __forceinline__ double rb_cospi(double x) { return cospi(x); }

// Outward-normal derivative of the family's exact solution on face j.
template <class Model> struct RobinData;
template <> struct RobinData<LaplaceExpCos> {
  template <typename R>
  __device__ static R dudn(int j, const R *x) {
    const R e = rb_exp(x[0]);
    const R g = (j >> 1) == 0 ? e * rb_cos(x[1]) : -e * rb_sin(x[1]);
    return (j & 1) ? g : -g;
  }
  template <typename R>
  __device__ static R u(const R *x) { return rb_exp(x[0]) * rb_cos(x[1]); }
};
template <> struct RobinData<EllipticManufactured> {
  template <typename R>
  __device__ static R dudn(int j, const R *x) {
    constexpr double kPi = 3.14159265358979323846;
    const int k = j >> 1;
    const R ez = rb_exp(x[2]);
    R g;
    if (k == 0) g = R(kPi) * rb_cospi(x[0]) * rb_sinpi(x[1]) * ez;
    else if (k == 1) g = R(kPi) * rb_sinpi(x[0]) * rb_cospi(x[1]) * ez;
    else g = rb_sinpi(x[0]) * rb_sinpi(x[1]) * ez;
    return (j & 1) ? g : -g;
  }
  template <typename R>
  __device__ static R u(const R *x) { return rb_sinpi(x[0]) * rb_sinpi(x[1]) * rb_exp(x[2]); }
};

template <typename R> __device__ __forceinline__ R r_exp(R v);
template <> __device__ __forceinline__ float r_exp<float>(float v) { return exp_fast(v); }
template <> __device__ __forceinline__ double r_exp<double>(double v) { return exp(v); }
template <typename R> __device__ __forceinline__ R r_expm1(R v);
template <> __device__ __forceinline__ float r_expm1<float>(float v) { return expm1f(v); }
template <> __device__ __forceinline__ double r_expm1<double>(double v) { return expm1(v); }
template <typename R> __device__ __forceinline__ R r_log(R v);
template <> __device__ __forceinline__ float r_log<float>(float v) {
  return 0.6931471805599453f * lg2_approx(v);
}
template <> __device__ __forceinline__ double r_log<double>(double v) { return log(v); }
__device__ __forceinline__ float r_sqrt(float v) { return sqrt_approx(fmaxf(v, 0.0f)); }
__device__ __forceinline__ double r_sqrt(double v) { return sqrt(v); }

// Step constants of the reflecting kernel in the path precision.
template <typename R>
struct ReflectConst {
  R dt, sdt, s2dt, cdt, phi, inv_s2dt;
  R b2;    // -2 log2(e) / (sigma^2 dt): exp(-2 m / (sigma^2 dt)) = 2^(b2 m)
  R boff;  // log2(2D) + 2^-12 with the bridge test, -inf without
};

// Bound on the absorbing faces' crossing probability of a step whose smallest
// d d' over them is m: P = 1 - prod (1 - p_j) <= sum p_j <= 2D exp(-2 m /
// (sigma^2 dt)), raised by 2^(2^-12) for the rounding of the exponents.
__device__ __forceinline__ float reflect_bound(const ReflectConst<float> &k, float m) {
  return ex2_approx(fmaf(k.b2, m, k.boff));
}
__device__ __forceinline__ double reflect_bound(const ReflectConst<double> &k, double m) {
  return exp2(k.b2 * m + k.boff);
}

// One step of a reflecting path from X (Z, sphil and n its running sums):
// the Euler-Maruyama move with normals xi, Lepingle's reflection on the
// reflecting faces within reach (axis k's uniform word: word wo + k of the
// tag-4 block rw), and the absorbing exit tests with the bridge uniform word
// wu.  Returns true when the path left through an absorbing
// face (xe its exit point, Zn its source sum); otherwise X, Z advance.
template <class Model, typename R>
__device__ __forceinline__ bool reflect_step(const ReflectArgs &a, const ReflectConst<R> &k,
                                             const uint4 &rw, int wo, R *X, R &Z, R &sphil,
                                             int32_t n, const R *xi, uint32_t wu, R *xe, R &Zn) {
  constexpr int D = Model::D;
  using G = Box<D>;
  R b[3] = {R(0), R(0), R(0)}, f = R(0);
  Model::template coeffs<R>(a.mc, X, b, f);
  // Y at the step's start; needed every step only with a source term
  constexpr bool kYStep = Model::kSource;
  const R Y = kYStep ? r_exp<R>(static_cast<R>(n) * k.cdt + sphil) : R(0);
  R Xn[3];
#pragma unroll
  for (int q = 0; q < D; ++q) Xn[q] = X[q] + b[q] * k.dt + k.sdt * xi[q];

  // ---- reflection on the reflecting faces within reach.  The bridge
  // minimum is formed for every reflecting face and step (full lanes: paths
  // linger near these faces, so a branch on reach would run, diverged, at
  // most warp-steps); only an actual reflection (L > 0) branches.
  R zr = R(0), yr = Y;
  bool have_y = kYStep;
#pragma unroll
  for (int j = 0; j < 2 * D; ++j) {
    if (!((a.mask >> j) & 1)) continue;
    const R y0 = G::template face_dist<R>(j, X), y1 = G::template face_dist<R>(j, Xn);
    const bool reach = R(2) * y0 * y1 * k.inv_s2dt < R(18);
    const int q = j >> 1;
    const int w = wo + q;
    const uint32_t wk = w == 0 ? rw.x : w == 1 ? rw.y : w == 2 ? rw.z : rw.w;
    const R dy = y1 - y0;
    const R mn = R(0.5) * (y0 + y1 - r_sqrt(dy * dy - R(2) * k.s2dt * r_log<R>(unif<R>(wk))));
    const R L = (reach && mn < R(0)) ? -mn : R(0);
    if (L > R(0)) {
      if (j & 1) Xn[q] = fmin(Xn[q] - L, R(1));
      else Xn[q] = fmax(Xn[q] + L, R(0));
      R xp[3] = {Xn[0], Xn[1], Xn[2]};
      xp[q] = R(j & 1);
      const R psi = RobinData<Model>::template dudn<R>(j, xp) - k.phi * RobinData<Model>::template u<R>(xp);
      if (!have_y) {
        yr = r_exp<R>(static_cast<R>(n) * k.cdt + sphil);
        have_y = true;
      }
      const R g1 = k.phi != R(0) ? r_expm1<R>(k.phi * L) / k.phi : L;
      zr += psi * yr * g1;
      yr *= r_exp<R>(k.phi * L);
      sphil += k.phi * L;
    }
  }
  Zn = kYStep ? Z + f * Y * k.dt + zr : Z + zr;

  // ---- exit through absorbing faces.  am > 0 puts X' strictly inside the
  // absorbing faces (the reflecting ones keep it in [0, 1]); above the bound
  // no absorbing crossing is possible.  Below, the exact tests.
  R am = R(1);
#pragma unroll
  for (int j = 0; j < 2 * D; ++j)
    if (!((a.mask >> j) & 1))
      am = fmin(am, G::template face_dist<R>(j, X) * G::template face_dist<R>(j, Xn));
  const R U = unif<R>(wu);
  bool out = false;
  if (!(am > R(0)) || U < reflect_bound(k, am)) {
#pragma unroll
    for (int q = 0; q < D; ++q) xe[q] = Xn[q];
    if (!G::template inside_closed<R>(Xn)) {
      G::template segment_exit<R>(X, Xn, xe);
      out = true;
    } else if (a.bridge) {
      R P = R(0), pb = R(-1);
      int jb = -1;
#pragma unroll
      for (int j = 0; j < 2 * D; ++j) {
        if ((a.mask >> j) & 1) continue;
        const R e = R(2) * G::template face_dist<R>(j, X) * G::template face_dist<R>(j, Xn) * k.inv_s2dt;
        if (e < R(18)) {
          const R p = r_exp<R>(-e);
          P = P + p * (R(1) - P);
          if (p > pb) {
            pb = p;
            jb = j;
          }
        }
      }
      if (jb >= 0 && U < P) {
#pragma unroll
        for (int j = 0; j < 2 * D; ++j)
          if (j == jb) G::template project<R>(j, xe);
        out = true;
      }
    }
  }
  if (out) return true;
#pragma unroll
  for (int q = 0; q < D; ++q) X[q] = Xn[q];
  Z = Zn;
  return false;
}

template <class Model, typename R>
__global__ void __launch_bounds__(kPathBlockOf<R>) reflect_kernel(const __grid_constant__ ReflectArgs a) {
  constexpr int D = Model::D;
  using G = Box<D>;
  const unsigned lane = threadIdx.x & 31u;
  ReflectConst<R> k;
  if constexpr (sizeof(R) == 4) {
    k.dt = a.kf[0];
    k.sdt = a.kf[1];
    k.s2dt = a.kf[2];
    k.cdt = a.kf[3];
    k.phi = a.kf[4];
    k.inv_s2dt = a.kf[5];
    k.b2 = a.kf[6];
    k.boff = a.kf[7];
  } else {
    k.dt = a.dt;
    k.sdt = a.sdt;
    k.s2dt = a.s2dt;
    k.cdt = a.cdt;
    k.phi = a.phi;
    k.inv_s2dt = 1.0 / k.s2dt;
    k.b2 = -2.0 * 1.4426950408889634 / a.s2dt;
    k.boff = a.bridge ? (D == 2 ? 2.0 : 2.584962500721156) + 2.44140625e-4 : -INFINITY;
  }
  R X[3] = {R(0), R(0), R(0)};
  R Z = R(0), sphil = R(0);  // source sum; phi * (local time so far)
  PhiloxPath pp{0, 0, 0}, pp4{0, 0, 4u};
  int32_t n = 0;
  uint64_t slot = 0;
  bool active = false, need = true;
  unsigned long long my_steps = 0, my_capped = 0, my_bad = 0;
  R *score = static_cast<R *>(a.score);
  WarpQueue wq;
  NodeCache<R, D> nc;
  const unsigned long long total = a.end - a.begin;

  for (;;) {
    while (__any_sync(kFull, need)) {
      unsigned long long q = 0;
      if (warp_claim<32>(wq, a.cursor, total, need, q)) {
        slot = q;
        const unsigned long long g = a.begin + q;
        nc.locate(g, a.n_paths, a.end, a.nodes);
        const uint32_t node = static_cast<uint32_t>(nc.node) + a.node_offset;
        const uint32_t path = static_cast<uint32_t>(g - nc.lo + a.path_offset);
        pp = philox_path(path, node, 0u, a.rk);
        pp4 = philox_path(path, node, 4u, a.rk);
#pragma unroll
        for (int q2 = 0; q2 < D; ++q2) X[q2] = nc.x[q2];
        n = 0;
        Z = R(0);
        sphil = R(0);
        bool on_abs = !G::template inside_closed<R>(X);
        const bool bad = on_abs;
#pragma unroll
        for (int q2 = 0; q2 < D; ++q2)
          on_abs = on_abs || (X[q2] <= R(0) && !((a.mask >> (2 * q2)) & 1)) ||
                   (X[q2] >= R(1) && !((a.mask >> (2 * q2 + 1)) & 1));
        if (bad) {
          score[slot] = R(NAN);
          if (a.steps) a.steps[slot] = 0;
          dump_exit_point<D>(a.exit, slot, X);
          if (a.flags) atomicOr(a.flags + nc.node, kNodeOutside);
          ++my_bad;
          need = true;
        } else if (on_abs) {
          score[slot] = Model::template g<R>(a.mc, X);
          if (a.steps) a.steps[slot] = 0;
          dump_exit_point<D>(a.exit, slot, X);
          if (a.flags) atomicOr(a.flags + nc.node, kNodeOnBoundary);
          need = true;
        } else {
          active = true;
        }
      }
    }
    if (!__any_sync(kFull, active)) break;
    if (!active) continue;

    // ---- one unit: up to four steps, random numbers formed up front (the
    // stream layout of the path kernel).  The step loop is not unrolled: each
    // step carries sizeable rare branches (a reflection with its Robin
    // weights, the exact absorbing tests), and four inlined copies ran 1.5x
    // slower.
    R z[4 * D];
    uint32_t u[4];
    unit_randoms<D, R>(n, pp, a.rk, z, u);
    bool out = false, capped = false;
    R xe[3] = {R(0), R(0), R(0)}, Zn = R(0);
    uint4 rw = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      // the tag-4 block: one per two steps in 2-D (n is 4q + j here), one per
      // step in 3-D
      if (D == 3 || (j & 1) == 0)
        rw = philox10_path(static_cast<uint32_t>(D == 3 ? n : n >> 1), pp4, a.rk);
      out = reflect_step<Model, R>(a, k, rw, D == 2 ? 2 * (j & 1) : 0, X, Z, sphil, n, z, u[0],
                                   xe, Zn);
      ++n;
      if (out) break;
      if (n >= a.max_steps) {
        capped = true;
        break;
      }
#pragma unroll
      for (int i = 0; i < 3 * D; ++i) z[i] = z[i + D];
#pragma unroll
      for (int i = 0; i < 3; ++i) u[i] = u[i + 1];
    }
    if (out) {
      const R Yn = r_exp<R>(static_cast<R>(n) * k.cdt + sphil);  // n already advanced
      score[slot] = Model::template g<R>(a.mc, xe) * Yn + Zn;
      if (a.steps) a.steps[slot] = n;
      dump_exit_point<D>(a.exit, slot, xe);
      my_steps += static_cast<unsigned long long>(n);
      active = false;
      need = true;
    } else if (capped) {
      // cap: score at the projection on the nearest absorbing face
      int jn = -1;
      R dn = R(1e30);
#pragma unroll
      for (int j = 0; j < 2 * D; ++j) {
        if ((a.mask >> j) & 1) continue;
        const R d = G::template face_dist<R>(j, X);
        if (d < dn) {
          dn = d;
          jn = j;
        }
      }
      R xc[3] = {X[0], X[1], X[2]};
#pragma unroll
      for (int j = 0; j < 2 * D; ++j)
        if (j == jn) G::template project<R>(j, xc);
      const R Yn = r_exp<R>(static_cast<R>(n) * k.cdt + sphil);
      score[slot] = Model::template g<R>(a.mc, xc) * Yn + Z;
      if (a.steps) a.steps[slot] = -n;
      dump_exit_point<D>(a.exit, slot, xc);
      if (a.flags) atomicOr(a.flags + nc.node, kNodeCapped);
      my_steps += static_cast<unsigned long long>(n);
      ++my_capped;
      active = false;
      need = true;
    }
  }
#pragma unroll
  for (int s2 = 16; s2 > 0; s2 >>= 1) {
    my_steps += __shfl_xor_sync(kFull, my_steps, s2);
    my_capped += __shfl_xor_sync(kFull, my_capped, s2);
    my_bad += __shfl_xor_sync(kFull, my_bad, s2);
  }
  if (lane == 0) {
    if (my_steps) atomicAdd(&a.counters[0], my_steps);
    if (my_capped) atomicAdd(&a.counters[1], my_capped);
    if (my_bad) atomicAdd(&a.counters[2], my_bad);
  }
}

template <class Model, typename R>
static pdd_status run_reflect(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                              const pdd_mc_params *mc, double *d_mean, double *d_se,
                              int64_t *d_npaths, pdd_diag *diag) {
  const uint64_t N = static_cast<uint64_t>(mc->n_paths);
  const uint64_t total = static_cast<uint64_t>(n) * N;
  const uint64_t wave = std::min<uint64_t>(total, ctx->wave_max_paths);
  const size_t acc_off = 256;
  const size_t score_off = align_up(acc_off + static_cast<size_t>(n) * sizeof(NodeAcc), 256);
  pdd_status st = ensure_scratch(ctx, align_up(score_off + wave * sizeof(R), 256));
  if (st != PDD_OK) return st;
  char *base = static_cast<char *>(ctx->scratch);
  auto *counters = reinterpret_cast<unsigned long long *>(base);
  auto *acc = reinterpret_cast<NodeAcc *>(base + acc_off);
  R *score = reinterpret_cast<R *>(base + score_off);
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, score_off, ctx->stream));
  int32_t *flags = diag ? diag->d_node_flags : nullptr;
  if (flags) PDD_CUDA_TRY(ctx, cudaMemsetAsync(flags, 0, static_cast<size_t>(n) * 4, ctx->stream));
  ReflectArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes = d_nodes;
  a.n_paths = N;
  a.path_offset = static_cast<uint64_t>(mc->path_offset);
  a.node_offset = static_cast<uint32_t>(mc->node_offset);
  a.cursor = counters + 4;
  a.counters = counters;
  a.score = score;
  a.rk = make_round_keys(mc->seed);
  const double sig = ctx->prob.sigma;
  a.dt = mc->dt;
  a.sdt = sig * std::sqrt(mc->dt);
  a.s2dt = sig * sig * mc->dt;
  a.cdt = constant_kill(ctx->prob.kind) * mc->dt;
  a.mask = static_cast<int32_t>(ctx->params[0]);
  a.phi = ctx->params[1];
  a.max_steps = static_cast<int32_t>(mc->max_steps);
  a.bridge = mc->bridge ? 1 : 0;
  {
    const float s2dt_f = static_cast<float>(a.s2dt);
    const float kf[8] = {static_cast<float>(a.dt), static_cast<float>(a.sdt), s2dt_f,
                         static_cast<float>(a.cdt), static_cast<float>(a.phi), 1.0f / s2dt_f,
                         static_cast<float>(-2.0 * 1.4426950408889634 / a.s2dt),
                         a.bridge ? static_cast<float>((Model::D == 2 ? 2.0 : 2.584962500721156) +
                                                       2.44140625e-4)
                                  : -INFINITY};
    for (int i = 0; i < 8; ++i) a.kf[i] = kf[i];
  }
  a.mc = ctx->mc;
  a.flags = flags;
  auto kern = reflect_kernel<Model, R>;
  int bps = 0;
  PDD_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kPathBlockOf<R>, 0));
  if (bps < 1) bps = 1;
  if (ctx->path_blocks_per_sm > 0) bps = std::min(bps, ctx->path_blocks_per_sm);
  uint64_t grid = static_cast<uint64_t>(bps) * ctx->num_sms;
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (wave + kPathBlockOf<R> - 1) / kPathBlockOf<R>));
  for (uint64_t b0 = 0; b0 < total; b0 += wave) {
    const uint64_t b1 = std::min(total, b0 + wave);
    if (b0 > 0) PDD_CUDA_TRY(ctx, cudaMemsetAsync(a.cursor, 0, sizeof(unsigned long long), ctx->stream));
    a.begin = b0;
    a.end = b1;
    a.steps = (diag && diag->d_path_steps) ? diag->d_path_steps + b0 : nullptr;
    a.exit = (diag && diag->d_path_exit) ? diag->d_path_exit + b0 * Model::D : nullptr;
    const auto ev = prof_slot(ctx);
    if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
    kern<<<static_cast<unsigned>(grid), kPathBlockOf<R>, 0, ctx->stream>>>(a);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
    const uint64_t node_lo = b0 / N, node_hi = (b1 - 1) / N;
    reduce_wave_kernel<R><<<static_cast<unsigned>(node_hi - node_lo + 1), kReduceBlock, 0,
                            ctx->stream>>>(score, b0, b1, N, node_lo, acc);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (diag && diag->d_path_score) {
      const uint64_t cnt = b1 - b0;
      const unsigned g = static_cast<unsigned>(std::min<uint64_t>((cnt + 255) / 256, 8192));
      widen_scores_kernel<R><<<g, 256, 0, ctx->stream>>>(score, diag->d_path_score + b0, cnt);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  finalize_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, ctx->stream>>>(
      acc, n, d_mean, d_se, d_npaths, flags);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (diag) {
    unsigned long long h[4] = {0, 0, 0, 0};
    PDD_CUDA_TRY(ctx, cudaMemcpyAsync(h, counters, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    diag->path_steps = static_cast<int64_t>(h[0]);
    diag->capped = static_cast<int64_t>(h[1]);
    if (h[2]) return fail(ctx, PDD_EINVAL, "%llu paths started outside the closed domain", h[2]);
    if (h[1]) return fail(ctx, PDD_ECAP, "%llu paths hit max_steps", h[1]);
  }
  return PDD_OK;
}

pdd_status reflect_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                              const pdd_mc_params *mc, double *d_mean, double *d_se,
                              int64_t *d_npaths, pdd_diag *diag) {
  const bool fp64 = mc->precision == PDD_FP64;
  switch (ctx->prob.kind) {
    case PDD_PROB_LAPLACE_EXPCOS:
      return fp64 ? run_reflect<LaplaceExpCos, double>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag)
                  : run_reflect<LaplaceExpCos, float>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag);
    case PDD_PROB_ELLIPTIC_MANUFACTURED:
      return fp64 ? run_reflect<EllipticManufactured, double>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag)
                  : run_reflect<EllipticManufactured, float>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag);
    default:
      return fail(ctx, PDD_EINVAL, "reflecting faces need the Laplace or the 3-D manufactured family");
  }
}

}  // namespace pdd
