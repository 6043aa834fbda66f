// naive.cu -- the plain GPU form of stage one, kept as the comparison
// baseline for the persistent path kernel: one launch per node, one thread
// per path (FP32, the same step arithmetic and random streams), block sums
// of s and s^2 added to the node's FP64 accumulators with atomics.  Each
// block waits for its slowest path and each launch for its slowest block.
#include <cmath>
#include <cstring>

#include "ctx.hpp"
#include "path_kernel.cuh"

namespace pdd {

constexpr int kNaiveBlock = 256;

template <class Model, class Geom>
__global__ void __launch_bounds__(kNaiveBlock)
naive_node_kernel(const __grid_constant__ PathArgs a, uint32_t node, double *acc) {
  constexpr int D = Model::D;
  const uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const StepConst<float> k(a);
  double s_d = 0.0, s2_d = 0.0, cnt = 0.0;
  if (p < a.n_paths) {
    float X[D], xe[D], lr[1];
#pragma unroll
    for (int d = 0; d < D; ++d) X[d] = static_cast<float>(a.nodes[static_cast<uint64_t>(node) * D + d]);
    float Y = 1.f, Z = 0.f, s = 0.f;
    int32_t n = 0;
    const PhiloxPath pp =
        philox_path(static_cast<uint32_t>(p + a.path_offset), node + a.node_offset, 0u, a.rk);
    bool done = !Geom::inside_open(X);
    if (done) s = Model::g(a.mc, X);
    while (!done && n < a.max_steps)
      done = path_unit<Model, Geom, float, false>(a, k, pp, a.rk, a.max_steps, X, Y, Z, n, s, xe, lr);
    if (!done) {
#pragma unroll
      for (int d = 0; d < D; ++d) xe[d] = X[d];
      Geom::project(Geom::nearest_face(xe), xe);
      s = Model::g(a.mc, xe) * Y + Z;
    }
    s_d = s;
    s2_d = static_cast<double>(s) * s;
    cnt = 1.0;
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    s_d += __shfl_xor_sync(kFull, s_d, m);
    s2_d += __shfl_xor_sync(kFull, s2_d, m);
    cnt += __shfl_xor_sync(kFull, cnt, m);
  }
  __shared__ double sh[3][kNaiveBlock / 32];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = s_d;
    sh[1][w] = s2_d;
    sh[2][w] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0, t1 = 0, t2 = 0;
    for (int i = 0; i < kNaiveBlock / 32; ++i) {
      t0 += sh[0][i];
      t1 += sh[1][i];
      t2 += sh[2][i];
    }
    atomicAdd(acc + 0, t0);
    atomicAdd(acc + 1, t1);
    atomicAdd(acc + 2, t2);
  }
}

__global__ void naive_finalize(const double *acc, int64_t n, double *mean, double *se,
                               int64_t *npaths) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const double s = acc[3 * i], s2 = acc[3 * i + 1], c = acc[3 * i + 2];
  const double m = s / c;
  mean[i] = m;
  se[i] = c > 1.0 ? sqrt(fmax(0.0, s2 - c * m * m) / (c - 1.0) / c) : 0.0;
  if (npaths) npaths[i] = static_cast<int64_t>(c);
}

template <class Model, class Geom>
static pdd_status run_naive(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_mc_params *mc,
                            double *d_mean, double *d_se, int64_t *d_npaths) {
  pdd_status st = ensure_scratch(ctx, static_cast<size_t>(n) * 3 * sizeof(double) + 256);
  if (st != PDD_OK) return st;
  double *acc = static_cast<double *>(ctx->scratch);
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(acc, 0, static_cast<size_t>(n) * 3 * sizeof(double), ctx->stream));
  PathArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes = d_nodes;
  a.n_paths = static_cast<uint64_t>(mc->n_paths);
  a.path_offset = static_cast<uint64_t>(mc->path_offset);
  a.node_offset = static_cast<uint32_t>(mc->node_offset);
  a.rk = make_round_keys(mc->seed);
  const double sig = ctx->prob.sigma, dt = mc->dt;
  const double c_kill = constant_kill(ctx->prob.kind);
  a.inv_s2dt = 1.0 / (sig * sig * dt);
  a.dt_f = static_cast<float>(dt);
  a.sdt_f = static_cast<float>(sig * std::sqrt(dt));
  a.thr_f = static_cast<float>(9.0 * sig * sig * dt);
  a.l2cdt_f = static_cast<float>(c_kill * dt * 1.4426950408889634);
  a.max_steps = static_cast<int32_t>(mc->max_steps);
  a.bridge = mc->bridge ? 1 : 0;
  a.mc = ctx->mc;
  const unsigned blocks = static_cast<unsigned>((mc->n_paths + kNaiveBlock - 1) / kNaiveBlock);
  const auto ev = prof_slot(ctx);
  if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
  for (int64_t i = 0; i < n; ++i)
    naive_node_kernel<Model, Geom><<<blocks, kNaiveBlock, 0, ctx->stream>>>(
        a, static_cast<uint32_t>(i), acc + 3 * i);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
  naive_finalize<<<static_cast<unsigned>((n + 255) / 256), 256, 0, ctx->stream>>>(acc, n, d_mean, d_se,
                                                                               d_npaths);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  return PDD_OK;
}

pdd_status interface_solve_naive_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                      const pdd_mc_params *mc, double *d_mean, double *d_se,
                                      int64_t *d_npaths) {
  if (!mc || n < 0 || n > (int64_t(1) << 32) || mc->n_paths < 1 || !(mc->dt > 0.0) ||
      mc->max_steps < 1 || mc->max_steps > 2147483647LL || mc->precision != PDD_FP32 ||
      mc->path_offset < 0 || mc->path_offset + mc->n_paths > (int64_t(1) << 32) ||
      mc->node_offset < 0 || mc->node_offset + n > (int64_t(1) << 32) ||
      ctx->prob.sigma * ctx->prob.sigma * mc->dt > 1.0 / 36.0)
    return fail(ctx, PDD_EINVAL, "invalid parameters for the naive solve (FP32 only)");
  if (reflect_mask(ctx) != 0)
    return fail(ctx, PDD_EINVAL, "the naive solve has no reflecting faces");
  if (n == 0) return PDD_OK;
  if (!d_nodes || !d_mean || !d_se) return fail(ctx, PDD_EINVAL, "null buffer");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  switch (ctx->prob.kind) {
    case PDD_PROB_LAPLACE_EXPCOS:
      if (ctx->prob.geometry == PDD_GEOM_L_SHAPE)
        return run_naive<LaplaceExpCos, LShape>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths);
      return run_naive<LaplaceExpCos, Box<2>>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths);
    case PDD_PROB_ELLIPTIC_MANUFACTURED:
      return run_naive<EllipticManufactured, Box<3>>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths);
    case PDD_PROB_POISSON_FOURIER:
      return run_naive<PoissonFourier, Box<2>>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths);
    default:
      return fail(ctx, PDD_EINVAL, "problem kind has no path kernel");
  }
}

}  // namespace pdd
