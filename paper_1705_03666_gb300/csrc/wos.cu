// wos.cu -- Walk on Spheres for the Laplace problem (Eq. 1.1), the scheme
// Sec. 2.1 recommends for stopped Brownian motion when it applies: from x the
// walk jumps to a uniform point on the largest circle inside the domain
// (radius d(x) = distance to the nearest face) and stops when d(x) <= eps,
// scoring g at the projection on that face.  No time step; the bias is
// O(eps) and a path takes O(log 1/eps) jumps.  Same persistent lane-refill
// layout and per-path score slots as the path kernel, one Philox block per
// four jumps (block n/4 of stream tag 2), the per-node reduction of reduce.cuh.
#include <cmath>
#include <cstring>

#include "ctx.hpp"
#include "path_kernel.cuh"
#include "reduce.cuh"
#include "warp_queue.cuh"

namespace pdd {

constexpr unsigned kWosChunk = 256;  // walks claimed per warp-level atomic

struct WosArgs {
  const double *nodes;
  uint64_t n_paths, path_offset, begin, end;
  unsigned long long *cursor;
  unsigned long long *counters;  // [0] jumps, [1] capped, [2] bad nodes
  void *score;
  int32_t *steps;
  double *exit;                  // [end - begin][2] stopping points (projected), or null
  RoundKeys rk;
  double eps;
  int32_t max_steps;
  ModelConst mc;
};

// A jump of length d in direction 2 pi U.
__device__ __forceinline__ void wos_dir(float U, float &cx, float &sy) {
  const float th = 6.28318530717958648f * (U - 0.5f);  // centred: cos(2pi U) = -cos(th)
  cx = -cos_approx(th);
  sy = -sin_approx(th);
}
__device__ __forceinline__ void wos_dir(double U, double &cx, double &sy) {
  sincospi(2.0 * U, &sy, &cx);
}

// Distance to the nearest face and its index, with every face index a
// compile-time constant so the position stays in registers.
template <class Geom, typename R>
__device__ __forceinline__ R wos_nearest(const R *x, int &jb) {
  R db = Geom::template face_dist<R>(0, x);
  jb = 0;
#pragma unroll
  for (int j = 1; j < Geom::kFaces; ++j) {
    const R d = Geom::template face_dist<R>(j, x);
    if (d < db) {
      db = d;
      jb = j;
    }
  }
  return db;
}
template <class Geom, typename R>
__device__ __forceinline__ void wos_project(int jb, R *x) {
#pragma unroll
  for (int j = 0; j < Geom::kFaces; ++j)
    if (j == jb) Geom::template project<R>(j, x);
}

template <class Geom, typename R>
__global__ void __launch_bounds__(kPathBlockOf<R>) wos_kernel(const __grid_constant__ WosArgs a) {
  const unsigned lane = threadIdx.x & 31u;
  const R eps = static_cast<R>(a.eps);
  R X[2] = {R(0), R(0)};
  PhiloxPath pp{0, 0, 0};
  uint4 blk = make_uint4(0, 0, 0, 0);
  uint64_t slot = 0;
  int32_t n = 0;
  bool active = false, need = true;
  unsigned long long my_steps = 0, my_capped = 0, my_bad = 0;
  R *score = static_cast<R *>(a.score);
  WarpQueue wq;
  NodeCache<R, 2> nc;
  const unsigned long long total = a.end - a.begin;
  bool pending = false;  // stopped walk whose score is written at the next claim
  for (;;) {
    if (claim_time(active)) {
      if (pending) {
        score[slot] = LaplaceExpCos::g<R>(a.mc, X);
        if (a.steps) a.steps[slot] = n;
        if (a.exit) {
          a.exit[2 * slot] = static_cast<double>(X[0]);
          a.exit[2 * slot + 1] = static_cast<double>(X[1]);
        }
        my_steps += static_cast<unsigned long long>(n);
        pending = false;
      }
      need = !active;
      while (__any_sync(kFull, need)) {
        unsigned long long q = 0;
        if (warp_claim<kWosChunk>(wq, a.cursor, total, need, q)) {
          slot = q;
          const unsigned long long g = a.begin + q;
          nc.locate(g, a.n_paths, a.end, a.nodes);
          const uint64_t path = g - nc.lo + a.path_offset;
          pp = philox_path(static_cast<uint32_t>(path), static_cast<uint32_t>(nc.node), 2u, a.rk);
          X[0] = nc.x[0];
          X[1] = nc.x[1];
          n = 0;
          if (!Geom::inside_closed(X)) {
            score[slot] = R(NAN);
            if (a.steps) a.steps[slot] = 0;
            if (a.exit) {
              a.exit[2 * slot] = static_cast<double>(X[0]);
              a.exit[2 * slot + 1] = static_cast<double>(X[1]);
            }
            ++my_bad;
            need = true;
          } else {
            active = true;
          }
        }
      }
      if (!__any_sync(kFull, active)) break;
    }
    if (!active) continue;
    int jb;
    const R d = wos_nearest<Geom, R>(X, jb);
    if (d <= eps || n >= a.max_steps) {
      if (n >= a.max_steps && d > eps) ++my_capped;
      wos_project<Geom, R>(jb, X);
      active = false;
      pending = true;
      continue;
    }
    if ((n & 3) == 0) blk = philox10_path(static_cast<uint32_t>(n >> 2), pp, a.rk);
    // word n mod 4 of the block: take the front word and rotate
    const uint32_t w = blk.x;
    blk.x = blk.y;
    blk.y = blk.z;
    blk.z = blk.w;
    R cx, sy;
    wos_dir(unif<R>(w), cx, sy);
    X[0] += d * cx;
    X[1] += d * sy;
    ++n;
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

template <class Geom, typename R>
static pdd_status run_wos(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_wos_params *wp,
                          double *d_mean, double *d_se, int64_t *d_npaths, pdd_diag *diag) {
  const uint64_t N = static_cast<uint64_t>(wp->n_paths);
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
  WosArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes = d_nodes;
  a.n_paths = N;
  a.path_offset = static_cast<uint64_t>(wp->path_offset);
  a.cursor = counters + 4;
  a.counters = counters;
  a.score = score;
  a.rk = make_round_keys(wp->seed);
  a.eps = wp->eps;
  a.max_steps = static_cast<int32_t>(wp->max_steps);
  a.mc = ctx->mc;
  auto kern = wos_kernel<Geom, R>;
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
    a.exit = (diag && diag->d_path_exit) ? diag->d_path_exit + 2 * b0 : nullptr;
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
  finalize_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, ctx->stream>>>(acc, n, d_mean,
                                                                                d_se, d_npaths);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (diag) {
    unsigned long long h[4] = {0, 0, 0, 0};
    PDD_CUDA_TRY(ctx, cudaMemcpyAsync(h, counters, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    diag->path_steps = static_cast<int64_t>(h[0]);
    diag->capped = static_cast<int64_t>(h[1]);
    if (h[2]) return fail(ctx, PDD_EINVAL, "%llu paths started outside the closed domain", h[2]);
    if (h[1]) return fail(ctx, PDD_ECAP, "%llu walks hit max_steps", h[1]);
  }
  return PDD_OK;
}

pdd_status wos_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_wos_params *wp,
                          double *d_mean, double *d_se, int64_t *d_npaths, pdd_diag *diag) {
  if (!wp) return fail(ctx, PDD_EINVAL, "params is NULL");
  if (ctx->prob.kind != PDD_PROB_LAPLACE_EXPCOS)
    return fail(ctx, PDD_EINVAL, "Walk on Spheres needs the Laplace problem (Eq. 1.1)");
  if (reflect_mask(ctx) != 0)
    return fail(ctx, PDD_EINVAL, "Walk on Spheres needs Dirichlet data on every face");
  if (n < 0 || n > (int64_t(1) << 32) || wp->n_paths < 1 || wp->path_offset < 0 ||
      wp->path_offset + wp->n_paths > (int64_t(1) << 32))
    return fail(ctx, PDD_EINVAL, "sizes out of range");
  if (!(wp->eps > 0.0) || !(wp->eps < 0.5)) return fail(ctx, PDD_EINVAL, "eps must be in (0, 1/2)");
  if (wp->max_steps < 1 || wp->max_steps > 2147483647LL)
    return fail(ctx, PDD_EINVAL, "max_steps out of range");
  if (wp->precision != PDD_FP32 && wp->precision != PDD_FP64)
    return fail(ctx, PDD_EINVAL, "unknown precision");
  if (wp->precision == PDD_FP32 && wp->eps < 1e-6)
    return fail(ctx, PDD_EINVAL, "FP32 walks need eps >= 1e-6");
  if (diag) {
    diag->path_steps = 0;
    diag->capped = 0;
  }
  if (n == 0) return PDD_OK;
  if (!d_nodes || !d_mean || !d_se) return fail(ctx, PDD_EINVAL, "null buffer");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const bool l = ctx->prob.geometry == PDD_GEOM_L_SHAPE;
  if (wp->precision == PDD_FP64)
    return l ? run_wos<LShape, double>(ctx, d_nodes, n, wp, d_mean, d_se, d_npaths, diag)
             : run_wos<Box<2>, double>(ctx, d_nodes, n, wp, d_mean, d_se, d_npaths, diag);
  return l ? run_wos<LShape, float>(ctx, d_nodes, n, wp, d_mean, d_se, d_npaths, diag)
           : run_wos<Box<2>, float>(ctx, d_nodes, n, wp, d_mean, d_se, d_npaths, diag);
}

}  // namespace pdd
