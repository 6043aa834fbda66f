// autotune.cu -- launch-shape tuner.  Runs short trial solves on the caller's
// own inputs for each candidate (resident blocks per SM of the persistent
// kernels; lane-chunk size of the batch kernel), times each with CUDA events
// on the context's stream (best of `repeats`), and stores the fastest in the
// context.  Results never depend on the launch shape, only the time does.
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.hpp"

namespace pdd {

namespace {

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

pdd_status autotune_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_mc_params *mc,
                         double *d_scratch_out, int32_t repeats, int32_t *best_bps,
                         double *best_ms) {
  if (!mc || !d_nodes || n < 1 || !d_scratch_out || repeats < 1 || repeats > 16)
    return fail(ctx, PDD_EINVAL, "autotune needs nodes, a 2n-double output buffer, repeats 1..16");
  if (reflect_mask(ctx) != 0)
    return fail(ctx, PDD_EINVAL, "autotune covers the absorbing-boundary path kernels");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  int max_bps = 0;
  // occupancy bound of the path kernels (7 blocks of 128 threads at most for
  // binary32 paths, fewer of 256 for FP64)
  PDD_CUDA_TRY(ctx, cudaDeviceGetAttribute(&max_bps, cudaDevAttrMaxBlocksPerMultiprocessor, ctx->device));
  max_bps = std::min(max_bps, 8);
  EventPair ev;
  PDD_CUDA_TRY(ctx, cudaEventCreate(&ev.a));
  PDD_CUDA_TRY(ctx, cudaEventCreate(&ev.b));
  const int saved = ctx->path_blocks_per_sm;
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  double best = DBL_MAX;
  int best_b = 0;
  for (int b = 1; b <= max_bps; ++b) {
    ctx->path_blocks_per_sm = b;
    double t_best = DBL_MAX;
    for (int r = 0; r < repeats + 1; ++r) {  // first run warms up
      PDD_CUDA_TRY(ctx, cudaEventRecord(ev.a, ctx->stream));
      pdd_status st = interface_solve_impl(ctx, d_nodes, n, mc, d_scratch_out, d_scratch_out + n,
                                           nullptr, nullptr);
      if (st != PDD_OK) {
        ctx->path_blocks_per_sm = saved;
        ctx->profiling = prof;
        return st;
      }
      PDD_CUDA_TRY(ctx, cudaEventRecord(ev.b, ctx->stream));
      PDD_CUDA_TRY(ctx, cudaEventSynchronize(ev.b));
      float ms = 0.f;
      PDD_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ev.a, ev.b));
      if (r > 0) t_best = std::min(t_best, static_cast<double>(ms));
    }
    if (t_best < best * 0.99) {  // prefer fewer resident blocks on near-ties
      best = t_best;
      best_b = b;
    }
  }
  ctx->profiling = prof;
  ctx->path_blocks_per_sm = best_b;
  if (best_bps) *best_bps = best_b;
  if (best_ms) *best_ms = best;
  return PDD_OK;
}

pdd_status autotune_batch_impl(pdd_ctx *ctx, const pdd_problem *problems, int32_t n_problems,
                               const pdd_batch_nodes *nodes, const pdd_batch_params *bp,
                               double *d_scratch_out, int32_t repeats, int32_t *best_chunk,
                               double *best_ms) {
  if (!bp || !nodes || nodes->n < 1 || !d_scratch_out || repeats < 1 || repeats > 16)
    return fail(ctx, PDD_EINVAL, "autotune needs nodes, a 2n-double output buffer, repeats 1..16");
  if (reflect_mask(ctx) != 0)
    return fail(ctx, PDD_EINVAL, "autotune covers the absorbing-boundary path kernels");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  EventPair ev;
  PDD_CUDA_TRY(ctx, cudaEventCreate(&ev.a));
  PDD_CUDA_TRY(ctx, cudaEventCreate(&ev.b));
  const int candidates[] = {32, 64, 128, 256, 512, 1024};
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  double best = DBL_MAX;
  int best_k = 0;
  for (int K : candidates) {
    pdd_batch_params p = *bp;
    p.chunk = K;
    double t_best = DBL_MAX;
    for (int r = 0; r < repeats + 1; ++r) {
      PDD_CUDA_TRY(ctx, cudaEventRecord(ev.a, ctx->stream));
      pdd_status st = batch_solve_impl(ctx, problems, n_problems, nodes, &p, d_scratch_out,
                                       d_scratch_out + nodes->n, nullptr, 0, nullptr);
      if (st != PDD_OK) {
        ctx->profiling = prof;
        return st;
      }
      PDD_CUDA_TRY(ctx, cudaEventRecord(ev.b, ctx->stream));
      PDD_CUDA_TRY(ctx, cudaEventSynchronize(ev.b));
      float ms = 0.f;
      PDD_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ev.a, ev.b));
      if (r > 0) t_best = std::min(t_best, static_cast<double>(ms));
    }
    if (t_best < best * 0.99) {
      best = t_best;
      best_k = K;
    }
  }
  ctx->profiling = prof;
  ctx->batch_chunk = best_k;
  if (best_chunk) *best_chunk = best_k;
  if (best_ms) *best_ms = best;
  return PDD_OK;
}

}  // namespace pdd
