// branch_grid.cu -- branching Brownian motion on a time grid: one tree per
// sample scores every grid time T_1 < ... < T_m (Algorithm 3.1 evaluates the
// particles alive at each T_i), in free space (Eq. 3.1) or with absorbing
// boundaries (Eq. 3.2: a particle that hits the boundary at tau contributes
// g(X_tau, T_i - tau) to every T_i >= tau, a particle alive at T_i
// contributes psi(X_{T_i}); marked weights alpha_k / q_k of Sec. 3.2 enter
// the estimates of the times after the branching).
//
// Times are integer ticks of 2^-k (k = 31 - e for T_m = f 2^e, f in [1/2,1)),
// so the cut points of every walk -- grid times, lifetime ends and, in a
// bounded domain, steps of at most dt -- are exact integers shared with the
// oracle.  Positions, lifetimes and the per-time products are binary32
// (FP64 is a 1/64-rate pipe on this part and these operations sit in
// divergent code); a lifetime can thus end a few ticks away from the
// oracle's, which moves a cut point only in rare cases (counted as a flip by
// the parity tests).  In a bounded domain each step takes the
// exit test of the linear paths: hard exit at the first crossing of the
// segment, else the half-space bridge probability p = exp(-2 d d' / h) over
// the faces with 2 d d' / h < 18, combined as P <- P + p (1 - P); the exit
// point is the projection of the step's end on the face of largest p.
//
// Streams: particle id of tree s at node i draws block j of
// Philox(seed, ((id << 20) | j, s, i, 3)); block 0 gives the lifetime
// -ln U(w0) / beta and the offspring count from U(w3); block j >= 1 gives
// step j: normals BM(w0, w1) and the bridge uniform U(w2).  Tree order,
// ids and pruning as for the free-space trees (branch_kernel.cuh).
//
// Lane layout: one lane owns one tree and walks it depth-first (pending
// particles on a per-lane stack in local memory), one step per loop trip;
// warps claim trees in chunks (warp_queue.cuh).  The estimate of tree g for
// time k goes to score[k * wave + slot] (FP32); one NaN-skipping FP64
// reduction per time plane gives (count, mean, M2) per (time, node).
#include <cmath>
#include <cstring>

#include "branch_kernel.cuh"
#include "ctx.hpp"
#include "models.cuh"
#include "reduce.cuh"
#include "warp_queue.cuh"

namespace pdd {

constexpr int kGridMaxTimes = 32;
constexpr unsigned kGridChunk = 64;  // trees claimed per warp-level atomic

struct FreeSpace {};

template <class Geom>
struct GeomTraits {
  static constexpr bool kBounded = true;
};
template <>
struct GeomTraits<FreeSpace> {
  static constexpr bool kBounded = false;
};

struct GridArgs {
  const double *nodes;  // [n][D]
  uint64_t n_trees, tree_offset, begin, end, wave;
  unsigned long long *cursor;
  unsigned long long *counters;  // [0] steps, [1] discarded trees, [2] bad nodes
  float *score;                  // [m][wave]
  int32_t *steps;                // [end - begin] or null
  RoundKeys rk;
  float tps, inv_tps;             // ticks per unit time (2^k) and its inverse
  float beta_f, inv_beta;
  int32_t psi_kind;
  float psi_prm;
  float psi_l2;                   // psi_prm log2(e)
  int32_t K, m;
  uint32_t dt_ticks;
  int32_t bridge;
  float cum[kMaxOffspring + 1];    // cumulative q (rounded from FP64 sums)
  float ratio[kMaxOffspring + 1];  // alpha_k / q_k
  uint32_t T[kGridMaxTimes];
  int64_t max_particles;
  int32_t max_depth;
};

// psi at a particle's position (the hardware exp2 and reciprocal, a few ulp,
// as in the free-space trees).
template <int D>
__device__ __forceinline__ float grid_psi(const GridArgs &a, const float *x) {
  switch (a.psi_kind) {
    case 0: return a.psi_prm;
    case 1: return rcp_approx(1.0f + ex2_approx(-a.psi_l2 * x[0]));
    case 2: {
      const float e = 1.0f + ex2_approx(a.psi_l2 * x[0]);
      return 1.0f - rcp_approx(e * e);
    }
    default: return sinpif(x[0]) * (D > 1 ? sinpif(x[1]) : 1.0f);
  }
}

// Boundary data g(x, s) by the psi kind: const c -> c / (c + (1 - c) e^{beta s})
// (the KPP ODE), sigmoid -> psi(x), travelling -> the wave at time s, sine -> 0.
template <int D>
__device__ __forceinline__ float grid_g(const GridArgs &a, const float *x, float s) {
  switch (a.psi_kind) {
    case 0: return a.psi_prm / (a.psi_prm + (1.0f - a.psi_prm) * expf(a.beta_f * s));
    case 1: return grid_psi<D>(a, x);
    case 2: {
      const float e = 1.0f + expf(a.psi_prm * x[0] - (5.0f / 6.0f) * a.beta_f * s);
      return 1.0f - __fdividef(1.0f, e * e);
    }
    default: return 0.0f;
  }
}

// Exit test of one step x0 -> x1 of duration h (Geom bounded).  Returns true
// with the exit point in xe.
template <class Geom, int D>
__device__ __forceinline__ bool grid_exit(const GridArgs &a, const float *x0, const float *x1,
                                          float h, uint32_t wu, float *xe) {
  if (!Geom::template inside_closed<float>(x1)) {
    Geom::template segment_exit<float>(x0, x1, xe);
    return true;
  }
  if (!a.bridge) return false;
  const float inv = 2.0f / h;
  float P = 0.0f, pb = -1.0f;
  int jb = -1;
#pragma unroll
  for (int j = 0; j < Geom::kFaces; ++j) {
    const float e = Geom::template face_dist<float>(j, x0) * Geom::template face_dist<float>(j, x1) * inv;
    if (e < 18.0f) {
      const float p = exp_fast(-e);
      P = P + p * (1.0f - P);
      if (p > pb) {
        pb = p;
        jb = j;
      }
    }
  }
  if (jb < 0 || !(unif_f(wu) < P)) return false;
#pragma unroll
  for (int k = 0; k < D; ++k) xe[k] = x1[k];
#pragma unroll
  for (int j = 0; j < Geom::kFaces; ++j)
    if (j == jb) Geom::template project<float>(j, xe);
  return true;
}

// kBinary: two children with probability one and the classical weight (the
// KPP law), so the offspring count and the mark are constants.
template <class Geom, int D, bool kBinary>
__global__ void __launch_bounds__(kBranchBlock) branch_grid_kernel(const __grid_constant__ GridArgs a) {
  constexpr bool kBounded = GeomTraits<Geom>::kBounded;
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t Tm = a.T[a.m - 1];
  float4 stk[kBranchMaxDepth];  // pending particles: (x1, x2, birth tick, id | ti << 16)
  // per-time products in shared memory (bank = lane): a local array indexed
  // by the running time index lives in local memory, whose footprint over the
  // grid exceeds L2 and went to DRAM
  __shared__ float sprod[kGridMaxTimes][kBranchBlock];
  float *prod_col = &sprod[0][threadIdx.x];
#define PROD(k) prod_col[(k) * kBranchBlock]
  int sp = 0;
  float X[2] = {0.f, 0.f};
  uint32_t id = 0, t = 0, tend = 0, j = 0, u_off = 0;
  int ti = 0;
  bool start = false;
  PhiloxPath pp{0, 0, 3u};  // the (tree, node, tag 3) half of Philox round one
  uint32_t next_id = 0;
  int64_t particles = 0;
  int32_t nsteps = 0;
  uint64_t slot = 0;
  bool active = false, need = true;
  unsigned long long my_steps = 0, my_disc = 0, my_bad = 0;
  WarpQueue wq;
  NodeCache<float, D> nc;
  const unsigned long long total = a.end - a.begin;

  for (;;) {
    if (claim_time(active)) {
      need = !active;
      while (__any_sync(kFull, need)) {
        unsigned long long q = 0;
        if (warp_claim<kGridChunk>(wq, a.cursor, total, need, q)) {
          slot = q;
          const unsigned long long g = a.begin + q;
          nc.locate(g, a.n_trees, a.end, a.nodes);
          pp = philox_path(static_cast<uint32_t>(g - nc.lo + a.tree_offset),
                           static_cast<uint32_t>(nc.node), 3u, a.rk);
          X[0] = nc.x[0];
          X[1] = D > 1 ? nc.x[D > 1 ? 1 : 0] : 0.f;
          for (int k = 0; k < a.m; ++k) PROD(k) = 1.0f;
          t = 0;
          ti = 0;  // T_1 > 0
          id = 0;
          next_id = 1;
          sp = 0;
          particles = 1;
          nsteps = 0;
          start = true;
          bool done = false;
          if constexpr (kBounded) {
            if (!Geom::template inside_closed<float>(X)) {
              for (int k = 0; k < a.m; ++k) a.score[k * a.wave + slot] = NAN;
              if (a.steps) a.steps[slot] = 0;
              ++my_bad;
              done = true;
            } else if (!Geom::template inside_open<float>(X)) {
              // on the boundary: absorbed at time 0
              for (int k = 0; k < a.m; ++k)
                a.score[k * a.wave + slot] = grid_g<D>(a, X, static_cast<float>(a.T[k]) * a.inv_tps);
              if (a.steps) a.steps[slot] = 0;
              done = true;
            }
          }
          if (done) need = true;
          else active = true;
        }
      }
      if (!__any_sync(kFull, active)) break;
    }
    if (!active) continue;

    // one Philox block per trip: on the trip that starts a particle, block 0
    // of its stream (lifetime and offspring count), else the block of its
    // next step (Philox((id << 20 | j, tree, node, 3)))
    const bool starting = start;
    const uint4 v = philox10_path(starting ? id << 20 : (id << 20) | j, pp, a.rk);
    if (starting) {
      const float ltk = 0.5f * neg2log(unif_f(v.x)) * a.inv_beta * a.tps;
      const uint64_t e = ltk >= 4294967040.0f ? 4294967295ull : static_cast<uint64_t>(__float2uint_rz(ltk));
      const uint64_t te = static_cast<uint64_t>(t) + e;
      tend = te < Tm ? static_cast<uint32_t>(te) : Tm;
      u_off = v.w;
      // ti (first grid time after t) is carried: a child starts where its
      // parent's walk ended, after the parent scored any grid time equal to t
      j = 1;
      start = false;
    }

    // one step of the current particle (none on its starting trip, and none
    // at all when its lifetime is under a tick)
    bool pdone = false;
    if (!starting && t < tend) {
      uint32_t nxt = tend;
      if (ti < a.m && a.T[ti] < nxt) nxt = a.T[ti];
      if (kBounded && nxt - t > a.dt_ticks) nxt = t + a.dt_ticks;
      const float h = static_cast<float>(nxt - t) * a.inv_tps;
      ++j;
      ++nsteps;
      float z0, z1;
      box_muller<float>(v.x, v.y, z0, z1);
      const float sh = sqrt_approx(h);
      float Xn[2] = {X[0] + sh * z0, D > 1 ? X[1] + sh * z1 : 0.f};
      if constexpr (kBounded) {
        float xe[2] = {0.f, 0.f};
        if (grid_exit<Geom, D>(a, X, Xn, h, v.z, xe)) {
          for (int k = ti; k < a.m; ++k)
            PROD(k) *= grid_g<D>(a, xe, static_cast<float>(a.T[k] - nxt) * a.inv_tps);
          pdone = true;
        }
      }
      if (!pdone) {
        X[0] = Xn[0];
        X[1] = Xn[1];
        t = nxt;
        if (ti < a.m && t == a.T[ti]) {
          PROD(ti) *= grid_psi<D>(a, X);
          ++ti;
        }
      }
    }
    bool tree_done = false, bad = false;
    if (!pdone && t == tend) {
      if (tend == Tm) {
        pdone = true;
      } else {
        // lifetime over before T_m: branch
        int k = 2;
        if constexpr (!kBinary) {
          const float u3 = unif_f(u_off);
          k = a.K;
          for (int kk = 0; kk <= a.K; ++kk) {
            if (u3 < a.cum[kk]) {
              k = kk;
              break;
            }
          }
          const float r = a.ratio[k];
          if (r != 1.0f)  // classical weights: nothing to do
            for (int kk = ti; kk < a.m; ++kk) PROD(kk) *= r;
        }
        particles += k;
        if (particles > a.max_particles || sp + k > a.max_depth) {
          bad = true;
          tree_done = true;
        } else if (k == 0) {
          pdone = true;
        } else if constexpr (kBinary) {
          stk[sp++] = make_float4(X[0], X[1], __uint_as_float(tend),
                                  __uint_as_float((next_id + 1) | (static_cast<uint32_t>(ti) << 16)));
          id = next_id;
          next_id += 2;
          start = true;  // continue with the first child from (X, tend)
        } else {
          for (int c = k - 1; c >= 1; --c)
            stk[sp++] = make_float4(X[0], X[1], __uint_as_float(tend),
                                    __uint_as_float((next_id + c) | (static_cast<uint32_t>(ti) << 16)));
          id = next_id;
          next_id += k;
          start = true;  // continue with the first child from (X, tend)
        }
      }
    }
    if (pdone) {
      if (sp == 0) {
        tree_done = true;
      } else {
        const float4 p = stk[--sp];
        X[0] = p.x;
        X[1] = p.y;
        t = __float_as_uint(p.z);
        id = __float_as_uint(p.w) & 0xffffu;
        ti = static_cast<int>(__float_as_uint(p.w) >> 16);
        start = true;
      }
    }
    if (tree_done) {
      for (int k = 0; k < a.m; ++k)
        a.score[k * a.wave + slot] = bad ? NAN : PROD(k);
      if (a.steps) a.steps[slot] = bad ? -nsteps : nsteps;
      my_steps += static_cast<unsigned long long>(nsteps);
      if (bad) ++my_disc;
      active = false;
      need = true;
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    my_steps += __shfl_xor_sync(kFull, my_steps, s);
    my_disc += __shfl_xor_sync(kFull, my_disc, s);
    my_bad += __shfl_xor_sync(kFull, my_bad, s);
  }
  if (lane == 0) {
    if (my_steps) atomicAdd(&a.counters[0], my_steps);
    if (my_disc) atomicAdd(&a.counters[1], my_disc);
    if (my_bad) atomicAdd(&a.counters[2], my_bad);
  }
#undef PROD
}

// acc is [m][n]; outputs are [n][m].
static __global__ void grid_finalize_kernel(const NodeAcc *acc, int64_t n, int32_t m,
                                            double *mean, double *se) {
  const int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (q >= n * m) return;
  const int64_t i = q / m, k = q - i * m;
  const NodeAcc A = acc[k * n + i];
  mean[q] = A.n > 0.0 ? A.mean : static_cast<double>(NAN);
  se[q] = A.n > 1.0 ? sqrt(A.m2 / (A.n - 1.0) / A.n) : (A.n > 0.0 ? 0.0 : static_cast<double>(NAN));
}

static __global__ void grid_kept_kernel(const NodeAcc *acc, int64_t n, int64_t *kept) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) kept[i] = static_cast<int64_t>(acc[i].n);
}

// score [m][wave] -> dst [(b0 + q) * m + k]
static __global__ void grid_dump_kernel(const float *score, uint64_t wave, uint64_t cnt, int32_t m,
                                        double *dst) {
  for (uint64_t q = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; q < cnt * m;
       q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint64_t g = q / m, k = q - g * m;
    dst[q] = static_cast<double>(score[k * wave + g]);
  }
}

template <class Geom, int D>
static pdd_status run_grid(pdd_ctx *ctx, const double *d_nodes, int64_t n, const uint32_t *T,
                           int32_t m, double tps, uint32_t dt_ticks,
                           const pdd_grid_branch_params *bp, double *d_mean, double *d_se,
                           int64_t *d_nkept, pdd_diag *diag) {
  const uint64_t N = static_cast<uint64_t>(bp->n_trees);
  const uint64_t total = static_cast<uint64_t>(n) * N;
  const uint64_t wave = std::min<uint64_t>(total, std::max<uint64_t>(1, ctx->wave_max_paths / m));
  const size_t acc_off = 256;
  const size_t score_off =
      align_up(acc_off + static_cast<size_t>(n) * m * sizeof(NodeAcc), 256);
  pdd_status st = ensure_scratch(ctx, align_up(score_off + wave * m * sizeof(float), 256));
  if (st != PDD_OK) return st;
  char *base = static_cast<char *>(ctx->scratch);
  auto *counters = reinterpret_cast<unsigned long long *>(base);
  auto *acc = reinterpret_cast<NodeAcc *>(base + acc_off);
  float *score = reinterpret_cast<float *>(base + score_off);
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, score_off, ctx->stream));

  const double *prm = ctx->params.data();
  GridArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes = d_nodes;
  a.n_trees = N;
  a.tree_offset = static_cast<uint64_t>(bp->tree_offset);
  a.wave = wave;
  a.cursor = counters + 4;
  a.counters = counters;
  a.score = score;
  a.rk = make_round_keys(bp->seed);
  a.beta_f = static_cast<float>(prm[0]);
  a.inv_beta = static_cast<float>(1.0 / prm[0]);
  a.tps = static_cast<float>(tps);
  a.inv_tps = static_cast<float>(1.0 / tps);
  a.psi_kind = static_cast<int32_t>(prm[1]);
  a.psi_prm = static_cast<float>(prm[2]);
  a.psi_l2 = static_cast<float>(prm[2] * 1.4426950408889634);
  a.K = static_cast<int32_t>(prm[3]);
  a.m = m;
  a.dt_ticks = dt_ticks;
  a.bridge = bp->bridge ? 1 : 0;
  double cum = 0.0;
  for (int k = 0; k <= a.K; ++k) {
    const double q = prm[4 + k], al = prm[5 + a.K + k];
    cum += q;
    a.cum[k] = static_cast<float>(cum);
    a.ratio[k] = static_cast<float>(q > 0.0 ? al / q : 0.0);
  }
  for (int k = 0; k < m; ++k) a.T[k] = T[k];
  a.max_particles = bp->max_particles;
  a.max_depth = bp->max_depth;

  // two children with probability one and the classical weight (KPP)
  const bool binary = a.K == 2 && prm[4] == 0.0 && prm[5] == 0.0 && prm[6] == 1.0 &&
                      prm[5 + a.K + 2] == 1.0;
  auto kern = binary ? branch_grid_kernel<Geom, D, true> : branch_grid_kernel<Geom, D, false>;
  int bps = 0;
  PDD_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kBranchBlock, 0));
  if (bps < 1) bps = 1;
  if (ctx->path_blocks_per_sm > 0) bps = std::min(bps, ctx->path_blocks_per_sm);
  uint64_t grid = static_cast<uint64_t>(bps) * ctx->num_sms;
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (wave + kBranchBlock - 1) / kBranchBlock));

  for (uint64_t b0 = 0; b0 < total; b0 += wave) {
    const uint64_t b1 = std::min(total, b0 + wave);
    if (b0 > 0) PDD_CUDA_TRY(ctx, cudaMemsetAsync(a.cursor, 0, sizeof(unsigned long long), ctx->stream));
    a.begin = b0;
    a.end = b1;
    a.steps = (diag && diag->d_path_steps) ? diag->d_path_steps + b0 : nullptr;
    const auto ev = prof_slot(ctx);
    if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
    kern<<<static_cast<unsigned>(grid), kBranchBlock, 0, ctx->stream>>>(a);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
    const uint64_t node_lo = b0 / N, node_hi = (b1 - 1) / N;
    // the m time planes in one launch (blockIdx.y = plane)
    reduce_wave_kernel<float, true>
        <<<dim3(static_cast<unsigned>(node_hi - node_lo + 1), static_cast<unsigned>(m)),
           kReduceBlock, 0, ctx->stream>>>(score, b0, b1, N, node_lo, acc, wave,
                                           static_cast<uint64_t>(n));
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (diag && diag->d_path_score) {
      const uint64_t cnt = b1 - b0;
      const unsigned g = static_cast<unsigned>(std::min<uint64_t>((cnt * m + 255) / 256, 8192));
      grid_dump_kernel<<<g, 256, 0, ctx->stream>>>(score, wave, cnt, m, diag->d_path_score + b0 * m);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  const int64_t nm = n * m;
  grid_finalize_kernel<<<static_cast<unsigned>((nm + 255) / 256), 256, 0, ctx->stream>>>(acc, n, m, d_mean, d_se);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (d_nkept) {
    grid_kept_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, ctx->stream>>>(acc, n, d_nkept);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
  }
  if (diag) {
    unsigned long long h[4] = {0, 0, 0, 0};
    PDD_CUDA_TRY(ctx, cudaMemcpyAsync(h, counters, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    diag->path_steps = static_cast<int64_t>(h[0]);
    diag->capped = static_cast<int64_t>(h[1]);
    if (h[2]) return fail(ctx, PDD_EINVAL, "%llu trees started outside the closed domain", h[2]);
    if (h[1]) return fail(ctx, PDD_ECAP, "%llu trees discarded by the caps", h[1]);
  }
  return PDD_OK;
}

pdd_status branching_grid_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                     const double *h_times, int32_t m,
                                     const pdd_grid_branch_params *bp, double *d_mean,
                                     double *d_se, int64_t *d_nkept, pdd_diag *diag) {
  if (!bp) return fail(ctx, PDD_EINVAL, "params is NULL");
  if (ctx->prob.kind != PDD_PROB_KPP)
    return fail(ctx, PDD_EINVAL, "pdd_branching_grid_solve needs a KPP problem");
  const int geom = ctx->prob.geometry, dim = ctx->prob.dim;
  const bool bounded = geom != PDD_GEOM_FREE_SPACE;
  if (dim < 1 || dim > 2) return fail(ctx, PDD_EINVAL, "dimension must be 1 or 2");
  if (bounded && !((dim == 1 && geom == PDD_GEOM_INTERVAL) ||
                   (dim == 2 && (geom == PDD_GEOM_UNIT_SQUARE || geom == PDD_GEOM_L_SHAPE))))
    return fail(ctx, PDD_EINVAL, "bounded trees need the interval (1-D), unit square or L-shape (2-D)");
  if (n < 0 || n > (int64_t(1) << 32)) return fail(ctx, PDD_EINVAL, "n out of range");
  if (bp->n_trees < 1 || bp->tree_offset < 0 || bp->tree_offset + bp->n_trees > (int64_t(1) << 32))
    return fail(ctx, PDD_EINVAL, "tree indices must fit in 32 bits");
  if (bp->max_particles < 1 || bp->max_particles > 4096)
    return fail(ctx, PDD_EINVAL, "max_particles must be in [1, 4096] (12-bit particle ids)");
  if (bp->max_depth < 1 || bp->max_depth > kBranchMaxDepth)
    return fail(ctx, PDD_EINVAL, "max_depth must be in [1, %d]", kBranchMaxDepth);
  if (m < 1 || m > kGridMaxTimes || !h_times)
    return fail(ctx, PDD_EINVAL, "need 1..%d grid times", kGridMaxTimes);
  for (int k = 0; k < m; ++k)
    if (!(h_times[k] > 0.0) || !std::isfinite(h_times[k]) || (k > 0 && !(h_times[k] > h_times[k - 1])))
      return fail(ctx, PDD_EINVAL, "grid times must be finite, positive and increasing");
  const int psik = static_cast<int>(ctx->params[1]);
  if (psik < 0 || psik > 3) return fail(ctx, PDD_EINVAL, "unknown initial-data kind");
  int e = 0;
  std::frexp(h_times[m - 1], &e);
  const double tps = std::ldexp(1.0, 31 - e);
  uint32_t T[kGridMaxTimes];
  for (int k = 0; k < m; ++k) T[k] = static_cast<uint32_t>(std::floor(h_times[k] * tps + 0.5));
  for (int k = 1; k < m; ++k)
    if (T[k] <= T[k - 1]) return fail(ctx, PDD_EINVAL, "grid times closer than one tick");
  uint32_t dt_ticks = 4294967295u;
  if (bounded) {
    if (!(bp->dt > 0.0)) return fail(ctx, PDD_EINVAL, "dt must be positive");
    const double d = std::floor(bp->dt * tps + 0.5);
    dt_ticks = d < 1.0 ? 1u : d > 4294967295.0 ? 4294967295u : static_cast<uint32_t>(d);
    if (static_cast<double>(T[m - 1]) / dt_ticks + m + 2 > 1048575.0)
      return fail(ctx, PDD_EINVAL, "more than 2^20 - 1 steps per particle (dt too small)");
  }
  if (diag) {
    diag->path_steps = 0;
    diag->capped = 0;
  }
  if (n == 0) return PDD_OK;
  if (!d_nodes || !d_mean || !d_se) return fail(ctx, PDD_EINVAL, "null buffer");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
#define PDD_GRID_RUN(G, D) run_grid<G, D>(ctx, d_nodes, n, T, m, tps, dt_ticks, bp, d_mean, d_se, d_nkept, diag)
  if (!bounded) return dim == 1 ? PDD_GRID_RUN(FreeSpace, 1) : PDD_GRID_RUN(FreeSpace, 2);
  if (dim == 1) return PDD_GRID_RUN(Box<1>, 1);
  if (geom == PDD_GEOM_L_SHAPE) return PDD_GRID_RUN(LShape, 2);
  return PDD_GRID_RUN(Box<2>, 2);
#undef PDD_GRID_RUN
}

}  // namespace pdd
