// branching.cu -- host side of pdd_branching_solve: waves of trees, launches
// of the branching kernel and the NaN-skipping per-node reduction.
#include <cmath>
#include <cstring>

#include "branch_kernel.cuh"
#include "ctx.hpp"
#include "reduce.cuh"

namespace pdd {

// Space-time nodes in binary32 (x1, x2 or 0, t, 0): the branching kernel
// starts a tree every few segments, and converting the FP64 coordinates there
// would put three conversions per tree on the 1/64-rate FP64 pipe.
__global__ void node_xt_f32_kernel(const double *xt, int64_t n, int d, float4 *out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double *p = xt + i * (d + 1);
    out[i] = make_float4(static_cast<float>(p[0]), d == 2 ? static_cast<float>(p[1]) : 0.0f,
                         static_cast<float>(p[d]), 0.0f);
  }
}

template <int D>
static pdd_status run_branching(pdd_ctx *ctx, const double *d_nodes_xt, int64_t n,
                                const pdd_branch_params *bp, double *d_mean, double *d_se,
                                int64_t *d_nkept, pdd_diag *diag) {
  const uint64_t N = static_cast<uint64_t>(bp->n_trees);
  const uint64_t total = static_cast<uint64_t>(n) * N;
  // at most 2^31 trees per wave (the kernel indexes a wave's trees in 32 bits)
  const uint64_t wave = std::min<uint64_t>(std::min<uint64_t>(total, ctx->wave_max_paths),
                                           uint64_t(1) << 31);
  const size_t acc_off = 256;
  const size_t xt_off = align_up(acc_off + static_cast<size_t>(n) * sizeof(NodeAcc), 256);
  const size_t score_off = align_up(xt_off + static_cast<size_t>(n) * sizeof(float4), 256);
  const size_t bytes = align_up(score_off + wave * sizeof(float), 256);
  pdd_status st = ensure_scratch(ctx, bytes);
  if (st != PDD_OK) return st;
  char *base = static_cast<char *>(ctx->scratch);
  auto *counters = reinterpret_cast<unsigned long long *>(base);
  auto *cursor = counters + 4;
  auto *acc = reinterpret_cast<NodeAcc *>(base + acc_off);
  auto *xt_f = reinterpret_cast<float4 *>(base + xt_off);
  float *score = reinterpret_cast<float *>(base + score_off);
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, xt_off, ctx->stream));
  node_xt_f32_kernel<<<static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 4096)), 256, 0,
                       ctx->stream>>>(d_nodes_xt, n, D, xt_f);
  PDD_CUDA_TRY(ctx, cudaGetLastError());

  const double *prm = ctx->params.data();
  BranchArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes_f = xt_f;
  a.n_trees = N;
  a.tree_offset = static_cast<uint64_t>(bp->tree_offset);
  a.cursor = cursor;
  a.counters = counters;
  a.score = score;
  a.rk = make_round_keys(bp->seed);
  a.inv_beta = static_cast<float>(1.0 / prm[0]);
  a.psi_kind = static_cast<int32_t>(prm[1]);
  a.psi_prm = static_cast<float>(prm[2]);
  a.psi_l2 = static_cast<float>(prm[2] * 1.4426950408889634);
  a.K = static_cast<int32_t>(prm[3]);
  double cum = 0.0;
  for (int k = 0; k <= a.K; ++k) {
    const double q = prm[4 + k], al = prm[5 + a.K + k];
    cum += q;
    a.cum[k] = static_cast<float>(cum);
    a.ratio[k] = static_cast<float>(q > 0.0 ? al / q : 0.0);
  }
  // (with 2^32 trees per node every index below 2^32 - 1 is in node 0)
  branch_divisor(N < (uint64_t(1) << 32) ? static_cast<uint32_t>(N) : 0xffffffffu, &a.nt_m,
                 &a.nt_s1, &a.nt_s2);
  a.max_particles = bp->max_particles;
  a.max_depth = bp->max_depth;
  int32_t *flags = diag ? diag->d_node_flags : nullptr;
  if (flags) PDD_CUDA_TRY(ctx, cudaMemsetAsync(flags, 0, static_cast<size_t>(n) * 4, ctx->stream));
  a.flags = flags;
  // two children with probability one and the classical weight (KPP)
  const bool binary = a.K == 2 && prm[4] == 0.0 && prm[5] == 0.0 && prm[6] == 1.0 &&
                      prm[5 + a.K + 2] == 1.0;

  // the KPP law gets one instantiation per initial-data kind; other laws read
  // the kind at run time
  void (*kern)(BranchArgs) = branch_kernel<D, false, -1>;
  if (binary) {
    switch (a.psi_kind) {
      case 0: kern = branch_kernel<D, true, 0>; break;
      case 1: kern = branch_kernel<D, true, 1>; break;
      case 2: kern = branch_kernel<D, true, 2>; break;
      default: kern = branch_kernel<D, true, 3>; break;
    }
  }
  int bps = 0;
  PDD_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kBranchBlock, 0));
  if (bps < 1) bps = 1;
  if (ctx->path_blocks_per_sm > 0) bps = std::min(bps, ctx->path_blocks_per_sm);
  uint64_t grid = static_cast<uint64_t>(bps) * ctx->num_sms;
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (wave + kBranchBlock - 1) / kBranchBlock));

  for (uint64_t b0 = 0; b0 < total; b0 += wave) {
    const uint64_t b1 = std::min(total, b0 + wave);
    if (b0 > 0) PDD_CUDA_TRY(ctx, cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), ctx->stream));
    a.begin = b0;
    a.end = b1;
    a.segs = (diag && diag->d_path_steps) ? diag->d_path_steps + b0 : nullptr;
    const auto ev = prof_slot(ctx);
    if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
    kern<<<static_cast<unsigned>(grid), kBranchBlock, 0, ctx->stream>>>(a);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
    const uint64_t node_lo = b0 / N, node_hi = (b1 - 1) / N;
    reduce_wave_kernel<float, true><<<static_cast<unsigned>(node_hi - node_lo + 1), kReduceBlock,
                                       0, ctx->stream>>>(score, b0, b1, N, node_lo, acc);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (diag && diag->d_path_score) {
      const uint64_t cnt = b1 - b0;
      const unsigned g = static_cast<unsigned>(std::min<uint64_t>((cnt + 255) / 256, 8192));
      widen_scores_kernel<float><<<g, 256, 0, ctx->stream>>>(score, diag->d_path_score + b0, cnt);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  finalize_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, ctx->stream>>>(
      acc, n, d_mean, d_se, d_nkept, flags);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (diag) {
    unsigned long long h[4] = {0, 0, 0, 0};
    PDD_CUDA_TRY(ctx, cudaMemcpyAsync(h, counters, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    diag->path_steps = static_cast<int64_t>(h[0]);
    diag->capped = static_cast<int64_t>(h[1]);
    if (h[1]) return fail(ctx, PDD_ECAP, "%llu trees discarded by the caps", h[1]);
  }
  return PDD_OK;
}

pdd_status branching_solve_impl(pdd_ctx *ctx, const double *d_nodes_xt, int64_t n,
                                const pdd_branch_params *bp, double *d_mean, double *d_se,
                                int64_t *d_nkept, pdd_diag *diag) {
  if (!bp) return fail(ctx, PDD_EINVAL, "params is NULL");
  if (ctx->prob.kind != PDD_PROB_KPP)
    return fail(ctx, PDD_EINVAL, "pdd_branching_solve needs a KPP problem");
  if (ctx->prob.geometry != PDD_GEOM_FREE_SPACE)
    return fail(ctx, PDD_EINVAL, "pdd_branching_solve is the free-space estimator; bounded "
                                 "domains use pdd_branching_grid_solve");
  if (n < 0 || n > (int64_t(1) << 32)) return fail(ctx, PDD_EINVAL, "n out of range");
  if (bp->n_trees < 1) return fail(ctx, PDD_EINVAL, "n_trees < 1");
  if (bp->tree_offset < 0 || bp->tree_offset + bp->n_trees > (int64_t(1) << 32))
    return fail(ctx, PDD_EINVAL, "tree indices must fit in 32 bits");
  if (bp->max_particles < 1) return fail(ctx, PDD_EINVAL, "max_particles < 1");
  if (bp->max_particles > (int64_t(1) << 31))
    return fail(ctx, PDD_EINVAL, "max_particles above 2^31 (particle ids are 32-bit)");
  if (bp->max_depth < 1 || bp->max_depth > kBranchMaxDepth)
    return fail(ctx, PDD_EINVAL, "max_depth must be in [1, %d]", kBranchMaxDepth);
  if (n > 0 && (!d_nodes_xt || !d_mean || !d_se)) return fail(ctx, PDD_EINVAL, "null buffer");
  if (diag) {
    diag->path_steps = 0;
    diag->capped = 0;
  }
  if (n == 0) return PDD_OK;
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (ctx->prob.dim == 1)
    return run_branching<1>(ctx, d_nodes_xt, n, bp, d_mean, d_se, d_nkept, diag);
  return run_branching<2>(ctx, d_nodes_xt, n, bp, d_mean, d_se, d_nkept, diag);
}

}  // namespace pdd
