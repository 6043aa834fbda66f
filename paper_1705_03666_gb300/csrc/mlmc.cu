// mlmc.cu -- one level of the multilevel Monte Carlo estimator (Sec. 2.1
// names Giles' multilevel method as the next acceleration of the Euler
// scheme):  E[P_L] = E[P_0] + sum_{l=1..L} E[P_l - P_{l-1}],  P_l the score of
// the Euler-Maruyama path with step dt_l = dt_0 / R^l.
//
// A lane owns one coupled pair: the fine path (step dt_l) and the coarse path
// (step dt_{l-1} = R dt_l) driven by the same Brownian motion -- the coarse
// increment is the sum of the R fine increments -- each stopping at its own
// exit (hard exit at the segment crossing, or the half-space bridge test over
// the faces within reach, exit at the end of the step).  Fine step k of pair
// p at node i reads Philox(seed, (k, p, i, 16 + l)): normals BM(w0, w1) and
// the bridge uniform U(w2); the coarse step closing a group of R fine steps
// takes the uniform of the group's last fine step (independent of every
// normal, so each path has exactly the law of the plain scheme at its step,
// and the shared uniform couples the exit decisions).  Level 0 is the plain
// scheme (fine path only).  Left point for Y and Z.  Dimensions 1 and 2.
//
// Outputs per node: the mean and variance of P_l - P_{l-1} and the fine and
// coarse means (three score planes, each reduced by reduce_wave_kernel).
#include <cmath>
#include <cstring>

#include "ctx.hpp"
#include "models.cuh"
#include "path_kernel.cuh"
#include "reduce.cuh"
#include "warp_queue.cuh"

namespace pdd {

struct MlmcArgs {
  const double *nodes;
  uint64_t n_paths, begin, end, wave;
  unsigned long long *cursor;
  unsigned long long *counters;  // [0] fine steps, [1] capped walks, [2] bad nodes
  void *score;                   // R[3][wave]: difference, fine, coarse
  int32_t *steps;
  double *aux;                   // [end - begin][8] per-walk records, or null
  RoundKeys rk;
  double dtf, sdtf, s2;          // fine step, sqrt(fine step), sigma^2
  int32_t level, refine, max_steps, bridge;
  ModelConst mc;
};

// Constants of one walk's step: length dt, sigma, 1 / (sigma^2 dt) and the
// screening bound's exponent scale -2 log2(e) / (sigma^2 dt) and offset
// (log2 of the face count + 2^-12 with the bridge test, -inf without).
template <typename R>
struct MlmcStep {
  R dt, sig, inv, b2, boff;
};
template <typename R>
__device__ __forceinline__ MlmcStep<R> mlmc_step_const(double dt, double s2, int faces, bool bridge) {
  MlmcStep<R> c;
  c.dt = static_cast<R>(dt);
  c.sig = static_cast<R>(sqrt(s2));
  c.inv = R(1) / (static_cast<R>(s2) * c.dt);
  c.b2 = static_cast<R>(-2.0 * 1.4426950408889634 / (s2 * dt));
  c.boff = bridge ? static_cast<R>(log2(static_cast<double>(faces)) + 2.44140625e-4)
                  : static_cast<R>(-INFINITY);
  return c;
}
// Bound on the step's crossing probability over all faces (the union bound
// at the smallest d d' m, raised by 2^(2^-12) for the exponents' rounding).
__device__ __forceinline__ float mlmc_bound(const MlmcStep<float> &c, float m) {
  return ex2_approx(fmaf(c.b2, m, c.boff));
}
__device__ __forceinline__ double mlmc_bound(const MlmcStep<double> &c, double m) {
  return exp2(c.b2 * m + c.boff);
}

template <class Model, class Geom, typename R>
struct MlmcWalk {
  R X[2], Y, Z, s;
  R xe[2];  // exit point (set when the walk ends)
  bool done;

  // One Euler step with the (unscaled-by-sigma) increment dW.  A lower bound
  // on the smallest d d' (> 0: X' inside) and the union bound screen the
  // step; below the bound, the exact tests.
  __device__ __forceinline__ void step(const MlmcArgs &a, const MlmcStep<R> &c, const R *dW, R U) {
    constexpr int D = Model::D;
    R b[2] = {R(0), R(0)}, f = R(0);
    if constexpr (Model::kDrift || Model::kSource) Model::coeffs(a.mc, X, b, f);
    R Xn[2] = {X[0], X[1]};
#pragma unroll
    for (int k = 0; k < D; ++k) Xn[k] = X[k] + b[k] * c.dt + c.sig * dW[k];
    const R Zn = Model::kSource ? Z + f * Y * c.dt : Z;
    const R mn = Geom::screen_lb(X, Xn);
    if (!(mn > R(0)) || U < mlmc_bound(c, mn)) {
      if (!Geom::inside_closed(Xn)) {
        Geom::segment_exit(X, Xn, xe);
        s = Model::g(a.mc, xe) * Y + Zn;
        done = true;
        return;
      }
      if (a.bridge) {
        R P = R(0), pb = R(-1);
        int jb = -1;
#pragma unroll
        for (int j = 0; j < Geom::kFaces; ++j) {
          const R e = R(2) * Geom::face_dist(j, X) * Geom::face_dist(j, Xn) * c.inv;
          if (e < R(18)) {
            const R p = exp_fast(-e);
            P = P + p * (R(1) - P);
            if (p > pb) {
              pb = p;
              jb = j;
            }
          }
        }
        if (jb >= 0 && U < P) {
          xe[0] = Xn[0];
          xe[1] = Xn[1];
#pragma unroll
          for (int j = 0; j < Geom::kFaces; ++j)
            if (j == jb) Geom::project(j, xe);
          s = Model::g(a.mc, xe) * Y + Zn;
          done = true;
          return;
        }
      }
    }
    X[0] = Xn[0];
    X[1] = Xn[1];
    Z = Zn;
  }
  __device__ __forceinline__ void cap(const MlmcArgs &a) {
    xe[0] = X[0];
    xe[1] = X[1];
    const int jn = Geom::nearest_face(X);
#pragma unroll
    for (int j = 0; j < Geom::kFaces; ++j)
      if (j == jn) Geom::project(j, xe);
    s = Model::g(a.mc, xe) * Y + Z;
    done = true;
  }
};

template <class Model, class Geom, typename R>
__global__ void __launch_bounds__(kPathBlockOf<R>) mlmc_kernel(const __grid_constant__ MlmcArgs a) {
  constexpr int D = Model::D;
  const unsigned lane = threadIdx.x & 31u;
  R *out = static_cast<R *>(a.score);
  const R sdtf = static_cast<R>(a.sdtf);
  const MlmcStep<R> cf = mlmc_step_const<R>(a.dtf, a.s2, Geom::kFaces, a.bridge != 0);
  const MlmcStep<R> cc = mlmc_step_const<R>(static_cast<double>(static_cast<R>(a.dtf) *
                                                                static_cast<R>(a.refine)),
                                            a.s2, Geom::kFaces, a.bridge != 0);
  MlmcWalk<Model, Geom, R> fw, cw;
  R dWc[2] = {R(0), R(0)};
  PhiloxPath pp{0, 0, 0};
  uint64_t slot = 0;
  int32_t k = 0, kc = 0;  // fine steps; fine steps since the last coarse step
  int32_t kf = 0, kcs = 0;  // exit steps of the fine and coarse walks
  bool active = false, need = true;
  unsigned long long my_steps = 0, my_capped = 0, my_bad = 0;
  WarpQueue wq;
  NodeCache<R, D> nc;
  const unsigned long long total = a.end - a.begin;
  // per-walk record of a finished pair (parity checks): scores, exit steps
  // (fine steps, coarse steps) and exit points of the fine and coarse walks
  auto write_aux = [&]() {
    if (!a.aux) return;
    double *o = a.aux + 8 * slot;
    o[0] = static_cast<double>(fw.s);
    o[1] = a.level == 0 ? 0.0 : static_cast<double>(cw.s);
    o[2] = static_cast<double>(kf);
    o[3] = a.level == 0 ? 0.0 : static_cast<double>(kcs);
    o[4] = static_cast<double>(fw.xe[0]);
    o[5] = static_cast<double>(fw.xe[1]);
    o[6] = a.level == 0 ? 0.0 : static_cast<double>(cw.xe[0]);
    o[7] = a.level == 0 ? 0.0 : static_cast<double>(cw.xe[1]);
  };
  for (;;) {
    if (claim_time(active)) {
      need = !active;
      while (__any_sync(kFull, need)) {
        unsigned long long q = 0;
        if (warp_claim<64>(wq, a.cursor, total, need, q)) {
          slot = q;
          const unsigned long long g = a.begin + q;
          nc.locate(g, a.n_paths, a.end, a.nodes);
          pp = philox_path(static_cast<uint32_t>(g - nc.lo), static_cast<uint32_t>(nc.node),
                           16u + static_cast<uint32_t>(a.level), a.rk);
          fw.X[0] = nc.x[0];
          fw.X[1] = D > 1 ? nc.x[D > 1 ? 1 : 0] : R(0);
          fw.Y = R(1);
          fw.Z = R(0);
          fw.done = false;
          cw = fw;
          cw.done = a.level == 0;
          dWc[0] = dWc[1] = R(0);
          k = 0;
          kc = 0;
          kf = 0;
          kcs = 0;
          fw.xe[0] = cw.xe[0] = fw.X[0];
          fw.xe[1] = cw.xe[1] = fw.X[1];
          if (!Geom::inside_closed(fw.X)) {
            out[slot] = out[a.wave + slot] = out[2 * a.wave + slot] = R(NAN);
            if (a.steps) a.steps[slot] = 0;
            fw.s = cw.s = R(NAN);
            write_aux();
            ++my_bad;
            need = true;
          } else if (!Geom::inside_open(fw.X)) {
            const R g0 = Model::g(a.mc, fw.X);
            out[slot] = a.level == 0 ? g0 : R(0);
            out[a.wave + slot] = g0;
            out[2 * a.wave + slot] = a.level == 0 ? R(0) : g0;
            if (a.steps) a.steps[slot] = 0;
            fw.s = cw.s = g0;
            write_aux();
            need = true;
          } else {
            active = true;
          }
        }
      }
      if (!__any_sync(kFull, active)) break;
    }
    if (!active) continue;

    // ---- one fine step (and a coarse step every R fine steps)
    const uint4 w = philox10_path(static_cast<uint32_t>(k), pp, a.rk);
    R z0, z1;
    box_muller<R>(w.x, w.y, z0, z1);
    const R dW[2] = {sdtf * z0, D > 1 ? sdtf * z1 : R(0)};
    const R U = unif<R>(w.z);
    if (!fw.done) {
      fw.step(a, cf, dW, U);
      if (fw.done) kf = k + 1;
    }
    dWc[0] += dW[0];
    dWc[1] += dW[1];
    ++k;
    if (a.level > 0 && ++kc == a.refine) {
      if (!cw.done) {
        cw.step(a, cc, dWc, U);
        if (cw.done) kcs = k / a.refine;
      }
      dWc[0] = dWc[1] = R(0);
      kc = 0;
    }
    bool finish = fw.done && cw.done;
    if (!finish && k >= a.max_steps) {
      if (!fw.done) {
        fw.cap(a);
        kf = -k;
        ++my_capped;
      }
      if (!cw.done) {
        cw.cap(a);
        kcs = -(k / a.refine);
        ++my_capped;
      }
      finish = true;
    }
    if (finish) {
      out[slot] = a.level == 0 ? fw.s : fw.s - cw.s;
      out[a.wave + slot] = fw.s;
      out[2 * a.wave + slot] = a.level == 0 ? R(0) : cw.s;
      if (a.steps) a.steps[slot] = k;
      write_aux();
      my_steps += static_cast<unsigned long long>(k);
      active = false;
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

// acc planes: [3][n]; var = M2 / (count - 1)
static __global__ void mlmc_finalize_kernel(const NodeAcc *acc, int64_t n, double *mean,
                                            double *var, double *fine_mean, double *coarse_mean) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const NodeAcc A = acc[i];
  mean[i] = A.n > 0.0 ? A.mean : static_cast<double>(NAN);
  var[i] = A.n > 1.0 ? A.m2 / (A.n - 1.0) : 0.0;
  if (fine_mean) fine_mean[i] = acc[n + i].mean;
  if (coarse_mean) coarse_mean[i] = acc[2 * n + i].mean;
}

template <class Model, class Geom, typename R>
static pdd_status run_mlmc(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_mlmc_params *mp,
                           double *d_mean, double *d_var, double *d_fine, double *d_coarse,
                           pdd_diag *diag) {
  const uint64_t N = static_cast<uint64_t>(mp->n_paths);
  const uint64_t total = static_cast<uint64_t>(n) * N;
  const uint64_t wave = std::min<uint64_t>(total, ctx->wave_max_paths / 3 + 1);
  const size_t acc_off = 256;
  const size_t score_off = align_up(acc_off + 3 * static_cast<size_t>(n) * sizeof(NodeAcc), 256);
  pdd_status st = ensure_scratch(ctx, align_up(score_off + 3 * wave * sizeof(R), 256));
  if (st != PDD_OK) return st;
  char *base = static_cast<char *>(ctx->scratch);
  auto *counters = reinterpret_cast<unsigned long long *>(base);
  auto *acc = reinterpret_cast<NodeAcc *>(base + acc_off);
  R *score = reinterpret_cast<R *>(base + score_off);
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, score_off, ctx->stream));
  MlmcArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes = d_nodes;
  a.n_paths = N;
  a.wave = wave;
  a.cursor = counters + 4;
  a.counters = counters;
  a.score = score;
  a.rk = make_round_keys(mp->seed);
  a.dtf = mp->dt0 / std::pow(static_cast<double>(mp->refine), static_cast<double>(mp->level));
  a.sdtf = std::sqrt(a.dtf);
  a.s2 = ctx->prob.sigma * ctx->prob.sigma;
  a.level = mp->level;
  a.refine = mp->refine;
  a.max_steps = static_cast<int32_t>(mp->max_steps);
  a.bridge = mp->bridge ? 1 : 0;
  a.mc = ctx->mc;
  auto kern = mlmc_kernel<Model, Geom, R>;
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
    a.aux = (diag && diag->d_path_aux) ? diag->d_path_aux + 8 * b0 : nullptr;
    const auto ev = prof_slot(ctx);
    if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
    kern<<<static_cast<unsigned>(grid), kPathBlockOf<R>, 0, ctx->stream>>>(a);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
    const uint64_t node_lo = b0 / N, node_hi = (b1 - 1) / N;
    for (int plane = 0; plane < 3; ++plane) {
      reduce_wave_kernel<R, true><<<static_cast<unsigned>(node_hi - node_lo + 1), kReduceBlock, 0,
                                    ctx->stream>>>(score + plane * wave, b0, b1, N, node_lo,
                                                   acc + static_cast<size_t>(plane) * n);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
    }
    if (diag && diag->d_path_score) {
      const uint64_t cnt = b1 - b0;
      const unsigned g = static_cast<unsigned>(std::min<uint64_t>((cnt + 255) / 256, 8192));
      widen_scores_kernel<R><<<g, 256, 0, ctx->stream>>>(score, diag->d_path_score + b0, cnt);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  mlmc_finalize_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, ctx->stream>>>(
      acc, n, d_mean, d_var, d_fine, d_coarse);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (diag) {
    unsigned long long h[4] = {0, 0, 0, 0};
    PDD_CUDA_TRY(ctx, cudaMemcpyAsync(h, counters, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    diag->path_steps = static_cast<int64_t>(h[0]);
    diag->capped = static_cast<int64_t>(h[1]);
    if (h[2]) return fail(ctx, PDD_EINVAL, "%llu pairs started outside the closed domain", h[2]);
    if (h[1]) return fail(ctx, PDD_ECAP, "%llu walks hit max_steps", h[1]);
  }
  return PDD_OK;
}

pdd_status mlmc_level_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_mlmc_params *mp,
                           double *d_mean, double *d_var, double *d_fine, double *d_coarse,
                           pdd_diag *diag) {
  if (!mp) return fail(ctx, PDD_EINVAL, "params is NULL");
  if (n < 0 || n > (int64_t(1) << 32)) return fail(ctx, PDD_EINVAL, "n out of range");
  if (mp->n_paths < 1 || mp->n_paths > (int64_t(1) << 32))
    return fail(ctx, PDD_EINVAL, "n_paths out of range");
  if (!(mp->dt0 > 0.0) || !std::isfinite(mp->dt0)) return fail(ctx, PDD_EINVAL, "dt0 must be > 0");
  if (mp->level < 0 || mp->level > 12 || mp->refine < 2 || mp->refine > 16)
    return fail(ctx, PDD_EINVAL, "level in [0, 12], refine in [2, 16]");
  if (mp->max_steps < 1 || mp->max_steps > 2147483647LL)
    return fail(ctx, PDD_EINVAL, "max_steps out of range");
  if (mp->precision != PDD_FP32 && mp->precision != PDD_FP64)
    return fail(ctx, PDD_EINVAL, "unknown precision");
  if (ctx->prob.sigma * ctx->prob.sigma * mp->dt0 > 1.0 / 36.0)
    return fail(ctx, PDD_EINVAL, "sigma^2 dt0 must be <= 1/36");
  if (reflect_mask(ctx) != 0) return fail(ctx, PDD_EINVAL, "the multilevel solve covers Dirichlet data");
  if (diag) {
    diag->path_steps = 0;
    diag->capped = 0;
  }
  if (n == 0) return PDD_OK;
  if (!d_nodes || !d_mean || !d_var) return fail(ctx, PDD_EINVAL, "null buffer");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const bool fp64 = mp->precision == PDD_FP64;
#define PDD_MLMC(M, G)                                                                      \
  (fp64 ? run_mlmc<M, G, double>(ctx, d_nodes, n, mp, d_mean, d_var, d_fine, d_coarse, diag) \
        : run_mlmc<M, G, float>(ctx, d_nodes, n, mp, d_mean, d_var, d_fine, d_coarse, diag))
  switch (ctx->prob.kind) {
    case PDD_PROB_LAPLACE_EXPCOS:
      if (ctx->prob.geometry == PDD_GEOM_L_SHAPE) return PDD_MLMC(LaplaceExpCos, LShape);
      return PDD_MLMC(LaplaceExpCos, Box<2>);
    case PDD_PROB_POISSON_FOURIER:
      return PDD_MLMC(PoissonFourier, Box<2>);
    default:
      return fail(ctx, PDD_EINVAL, "the multilevel solve covers the 2-D families");
  }
#undef PDD_MLMC
}

// The multilevel estimate from its levels, per node, in level order:
// mean = sum_l mean_l, se = sqrt(sum_l var_l / N_l) (independent levels).
struct LevelCounts {
  double n[13];
};
static __global__ void mlmc_combine_kernel(const double *lmean, const double *lvar, int64_t n,
                                           int32_t L, LevelCounts N, double *mean, double *se) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  double m = 0.0, v = 0.0;
  for (int l = 0; l < L; ++l) {
    m += lmean[static_cast<int64_t>(l) * n + i];
    v += lvar[static_cast<int64_t>(l) * n + i] / N.n[l];
  }
  mean[i] = m;
  se[i] = sqrt(v);
}

pdd_status mlmc_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                           const pdd_mlmc_params *mp, int32_t n_levels,
                           const int64_t *h_n_per_level, double *d_mean, double *d_se,
                           double *d_level_mean, double *d_level_var, pdd_diag *diag) {
  if (!mp || !h_n_per_level) return fail(ctx, PDD_EINVAL, "params or path counts NULL");
  if (n_levels < 1 || n_levels > 13) return fail(ctx, PDD_EINVAL, "n_levels must be in [1, 13]");
  for (int l = 0; l < n_levels; ++l)
    if (h_n_per_level[l] < 1) return fail(ctx, PDD_EINVAL, "level %d has no pairs", l);
  if (n < 0 || n > (int64_t(1) << 32)) return fail(ctx, PDD_EINVAL, "n out of range");
  if (diag) {
    diag->path_steps = 0;
    diag->capped = 0;
  }
  if (n == 0) return PDD_OK;
  if (!d_mean || !d_se) return fail(ctx, PDD_EINVAL, "null buffer");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // level means and variances: the caller's buffers, or the auxiliary buffer
  // (the level calls use the context scratch themselves)
  double *lm = d_level_mean, *lv = d_level_var;
  const size_t plane = static_cast<size_t>(n) * n_levels * sizeof(double);
  if (!lm || !lv) {
    const pdd_status st = ensure_aux(ctx, 2 * plane);
    if (st != PDD_OK) return st;
    if (!lm) lm = static_cast<double *>(ctx->aux);
    if (!lv) lv = reinterpret_cast<double *>(static_cast<char *>(ctx->aux) + plane);
  }
  LevelCounts N{};
  pdd_status worst = PDD_OK;
  int64_t steps = 0, capped = 0;
  for (int l = 0; l < n_levels; ++l) {
    pdd_mlmc_params lp = *mp;
    lp.level = l;
    lp.n_paths = h_n_per_level[l];
    N.n[l] = static_cast<double>(h_n_per_level[l]);
    pdd_diag ld{};
    const pdd_status st = mlmc_level_impl(ctx, d_nodes, n, &lp, lm + static_cast<size_t>(l) * n,
                                          lv + static_cast<size_t>(l) * n, nullptr, nullptr,
                                          diag ? &ld : nullptr);
    if (st != PDD_OK && st != PDD_ECAP) return st;
    if (st == PDD_ECAP) worst = PDD_ECAP;
    steps += ld.path_steps;
    capped += ld.capped;
  }
  mlmc_combine_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, ctx->stream>>>(
      lm, lv, n, n_levels, N, d_mean, d_se);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (diag) {
    diag->path_steps = steps;
    diag->capped = capped;
    if (worst == PDD_ECAP) return fail(ctx, PDD_ECAP, "%lld walks hit max_steps",
                                       static_cast<long long>(capped));
  }
  return PDD_OK;
}

}  // namespace pdd
