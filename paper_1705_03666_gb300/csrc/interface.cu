// interface.cu -- host side of pdd_interface_solve: scratch layout, waves,
// launches of the path kernel and the per-node reduction, diagnostics.
#include <cmath>
#include <cstring>

#include "ctx.hpp"
#include "path_kernel.cuh"

namespace pdd {

__global__ void philox_stream_kernel(RoundKeys rk, uint32_t j0, uint32_t c1, uint32_t c2,
                                     uint32_t c3, int64_t n, uint4 *out) {
  for (int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; b < n;
       b += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[b] = philox10(j0 + static_cast<uint32_t>(b), c1, c2, c3, rk);
}

// FP32 normals and uniforms exactly as the path kernels form them:
// pair j: BM(w0, w1) of Philox((j, c1, c2, c3)), uniform of w2.
__global__ void normals_kernel(RoundKeys rk, uint32_t c1, uint32_t c2, uint32_t c3, int64_t n,
                               float *z, float *u) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint4 w = philox10(static_cast<uint32_t>(j), c1, c2, c3, rk);
    float z0, z1;
    box_muller<float>(w.x, w.y, z0, z1);
    z[2 * j] = z0;
    z[2 * j + 1] = z1;
    if (u) u[j] = unif_f(w.z);
  }
}

pdd_status normals_impl(pdd_ctx *ctx, uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3,
                        int64_t n_pairs, float *d_z, float *d_u) {
  if (n_pairs < 0 || (n_pairs > 0 && !d_z)) return fail(ctx, PDD_EINVAL, "bad arguments");
  if (n_pairs == 0) return PDD_OK;
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int grid = static_cast<int>(std::min<int64_t>((n_pairs + 255) / 256, 8192));
  normals_kernel<<<grid, 256, 0, ctx->stream>>>(make_round_keys(seed), c1, c2, c3, n_pairs, d_z,
                                                d_u);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  return PDD_OK;
}

pdd_status philox_stream_impl(pdd_ctx *ctx, uint64_t seed, uint32_t j0, uint32_t c1,
                              uint32_t c2, uint32_t c3, int64_t n_blocks, uint32_t *d_out) {
  if (n_blocks < 0) return fail(ctx, PDD_EINVAL, "n_blocks < 0");
  if (n_blocks == 0) return PDD_OK;
  if (!d_out) return fail(ctx, PDD_EINVAL, "d_out is NULL");
  if (reinterpret_cast<uintptr_t>(d_out) % 16)
    return fail(ctx, PDD_EINVAL, "d_out must be 16-byte aligned");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int grid = static_cast<int>(std::min<int64_t>((n_blocks + 255) / 256, 4096));
  philox_stream_kernel<<<grid, 256, 0, ctx->stream>>>(make_round_keys(seed), j0, c1, c2, c3,
                                                       n_blocks, reinterpret_cast<uint4 *>(d_out));
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  return PDD_OK;
}

// Scratch layout for one interface solve (offsets in bytes):
//   [0, 256)          counters (4 x u64) and the queue cursor
//   [256, +n*112)     per-node exact sums (NodeFix)
// No per-path score is stored: the path kernel adds every score to its node's
// integer sums when the path ends, in one launch over all paths.
constexpr size_t kFixOff = 256;

template <class Model, class Geom, typename R>
static pdd_status run_paths(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                            const pdd_mc_params *mc, double *d_mean, double *d_se,
                            int64_t *d_npaths, pdd_diag *diag) {
  const uint64_t N = static_cast<uint64_t>(mc->n_paths);
  const uint64_t total = static_cast<uint64_t>(n) * N;
  const size_t bytes = align_up(kFixOff + static_cast<size_t>(n) * sizeof(NodeFix), 256);
  pdd_status st = ensure_scratch(ctx, bytes);
  if (st != PDD_OK) return st;
  char *base = static_cast<char *>(ctx->scratch);
  auto *counters = reinterpret_cast<unsigned long long *>(base);
  auto *cursor = counters + 4;
  auto *fix = reinterpret_cast<NodeFix *>(base + kFixOff);
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, bytes, ctx->stream));

  PathArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes = d_nodes;
  a.n_paths = N;
  a.path_offset = static_cast<uint64_t>(mc->path_offset);
  a.node_offset = static_cast<uint32_t>(mc->node_offset);
  a.cursor = cursor;
  a.counters = counters;
  a.fix = fix;
  a.begin = 0;
  a.end = total;
  a.rk = make_round_keys(mc->seed);
  const double sig = ctx->prob.sigma, dt = mc->dt;
  const double c_kill = constant_kill(ctx->prob.kind);
  a.inv_s2dt = 1.0 / (sig * sig * dt);
  a.dt_d = dt;
  a.sdt_d = sig * std::sqrt(dt);
  a.thr_d = 9.0 * sig * sig * dt;
  a.ecdt_d = std::exp(c_kill * dt);
  a.dt_f = static_cast<float>(a.dt_d);
  a.sdt_f = static_cast<float>(a.sdt_d);
  a.thr_f = static_cast<float>(a.thr_d);
  a.l2cdt_f = static_cast<float>(c_kill * dt * 1.4426950408889634);
  a.max_steps = static_cast<int32_t>(mc->max_steps);
  a.bridge = mc->bridge ? 1 : 0;
  a.mc = ctx->mc;
  if (diag) {
    a.dump_score = diag->d_path_score;
    a.steps = diag->d_path_steps;
    a.dump_exit = diag->d_path_exit;
  }

  auto kern = path_kernel<Model, Geom, R>;
  int bps = 0;
  PDD_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kPathBlockOf<R>, 0));
  if (bps < 1) bps = 1;
  if (ctx->path_blocks_per_sm > 0) bps = std::min(bps, ctx->path_blocks_per_sm);
  uint64_t grid = static_cast<uint64_t>(bps) * ctx->num_sms;
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (total + kPathBlockOf<R> - 1) / kPathBlockOf<R>));

  const auto ev = prof_slot(ctx);
  if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
  kern<<<static_cast<unsigned>(grid), kPathBlockOf<R>, 0, ctx->stream>>>(a);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
  fix_finalize_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, ctx->stream>>>(
      fix, n, d_mean, d_se, d_npaths, diag ? diag->d_node_flags : nullptr);
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

template <class Model, class Geom>
static pdd_status run_prec(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                           const pdd_mc_params *mc, double *d_mean, double *d_se,
                           int64_t *d_npaths, pdd_diag *diag) {
  if (mc->precision == PDD_FP64)
    return run_paths<Model, Geom, double>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag);
  return run_paths<Model, Geom, float>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag);
}

pdd_status interface_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                const pdd_mc_params *mc, double *d_mean, double *d_se,
                                int64_t *d_npaths, pdd_diag *diag) {
  if (!mc) return fail(ctx, PDD_EINVAL, "mc is NULL");
  if (n < 0 || n > (int64_t(1) << 32)) return fail(ctx, PDD_EINVAL, "n out of range");
  if (mc->n_paths < 1) return fail(ctx, PDD_EINVAL, "n_paths < 1");
  if (mc->path_offset < 0 || mc->path_offset + mc->n_paths > (int64_t(1) << 32))
    return fail(ctx, PDD_EINVAL, "path indices must fit in 32 bits");
  if (mc->node_offset < 0 || mc->node_offset + n > (int64_t(1) << 32))
    return fail(ctx, PDD_EINVAL, "node stream indices must fit in 32 bits");
  if (!(mc->dt > 0.0) || !std::isfinite(mc->dt)) return fail(ctx, PDD_EINVAL, "dt must be > 0");
  if (mc->max_steps < 1 || mc->max_steps > 2147483647LL)
    return fail(ctx, PDD_EINVAL, "max_steps out of range");
  if (mc->precision != PDD_FP32 && mc->precision != PDD_FP64)
    return fail(ctx, PDD_EINVAL, "unknown precision");
  if (ctx->prob.sigma * ctx->prob.sigma * mc->dt > 1.0 / 36.0)
    return fail(ctx, PDD_EINVAL, "sigma^2 dt must be <= 1/36");
  if (ctx->prob.kind == PDD_PROB_KPP)
    return fail(ctx, PDD_EINVAL, "KPP problems use pdd_branching_solve");
  if (n > 0 && (!d_nodes || !d_mean || !d_se)) return fail(ctx, PDD_EINVAL, "null buffer");
  if (static_cast<double>(n) * static_cast<double>(mc->n_paths) > 9.0e18)
    return fail(ctx, PDD_EINVAL, "too many paths");
  if (diag) {
    diag->path_steps = 0;
    diag->capped = 0;
  }
  if (n == 0) return PDD_OK;
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (reflect_mask(ctx) != 0)
    return reflect_solve_impl(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag);
  switch (ctx->prob.kind) {
    case PDD_PROB_LAPLACE_EXPCOS:
      if (ctx->prob.geometry == PDD_GEOM_L_SHAPE)
        return run_prec<LaplaceExpCos, LShape>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag);
      return run_prec<LaplaceExpCos, Box<2>>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag);
    case PDD_PROB_ELLIPTIC_MANUFACTURED:
      return run_prec<EllipticManufactured, Box<3>>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths,
                                                     diag);
    case PDD_PROB_POISSON_FOURIER:
      return run_prec<PoissonFourier, Box<2>>(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag);
    default:
      return fail(ctx, PDD_EINVAL, "problem kind %d has no path kernel", ctx->prob.kind);
  }
}

}  // namespace pdd
