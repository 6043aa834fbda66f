// batch.cu -- pdd_batch_solve: variance-adaptive interface solve over a
// heterogeneous batch of nodes, as one device-driven pipeline that can be
// captured once in a CUDA graph and replayed.
//
//   0. the nodes are grouped by domain/family (stable partition on the
//      device); chunk lists follow that order, one kernel per family;
//   1. pilot: n_pilot paths per node (lane-chunk queue, batch_kernel), their
//      scores added to the node's exact sums (nodefix.cuh);
//   2. per node: pilot mean and variance s^2 from those sums, path count
//      N_i = clamp(ceil(s^2 / SE*^2), max(n_min, n_pilot), n_max);
//   3. exclusive scan of the per-node chunk counts of paths [n_pilot, N_i);
//   4. main pass over that device-built work list (same persistent kernel),
//      adding to the same sums;
//   5. per node: mean, standard error and count from the sums.
// Paths [0, N_i) of node i are the streams pdd_interface_solve would use, so
// the pilot paths are part of the final estimate, and a batch with a fixed
// count N reproduces pdd_interface_solve's estimate bit for bit (integer sums
// do not depend on the order in which paths are added).
#include <cmath>
#include <cstring>

#include "batch_kernel.cuh"
#include "ctx.hpp"
#include "reduce.cuh"

namespace pdd {

constexpr int kScanBlock = 1024;

// Stable partition of the nodes by family: perm[j] is the node at position j,
// family c holds positions [cstart[c], cstart[c+1]) (c = 0..3); nodes whose
// problem index is out of range go to the end, [cstart[4], n), which no
// kernel processes (their results are NaN, counted as bad nodes).
// One block; each thread takes a contiguous segment of nodes, so the order
// within a family is the node order.
__global__ void __launch_bounds__(kScanBlock)
batch_partition(int64_t n, const int32_t *prob, int32_t n_probs, int4 combo_of_prob,
                int32_t *perm, int64_t *cstart, unsigned long long *bad) {
  __shared__ int64_t part[kScanBlock];
  __shared__ int64_t base;
  const int cp[4] = {combo_of_prob.x, combo_of_prob.y, combo_of_prob.z, combo_of_prob.w};
  const int64_t per = (n + kScanBlock - 1) / kScanBlock;
  const int64_t b = threadIdx.x * per, e = min(n, b + per);
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c = 0; c <= 4; ++c) {
    int64_t cnt = 0;
    for (int64_t i = b; i < e; ++i) {
      const int32_t pi = prob[i];
      const int ci = (pi >= 0 && pi < n_probs) ? cp[pi] : 4;
      cnt += ci == c;
    }
    part[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      cstart[c] = base;
      int64_t acc = base;
      for (int t = 0; t < kScanBlock; ++t) {
        const int64_t v = part[t];
        part[t] = acc;
        acc += v;
      }
      base = acc;
      if (c == 4) {
        cstart[5] = acc;
        if (acc > cstart[4]) atomicAdd(bad, static_cast<unsigned long long>(acc - cstart[4]));
      }
    }
    __syncthreads();
    int64_t pos = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) {
      const int32_t pi = prob[i];
      const int ci = (pi >= 0 && pi < n_probs) ? cp[pi] : 4;
      if (ci == c) perm[pos++] = static_cast<int32_t>(i);
    }
    __syncthreads();
  }
}

// Pilot work list: every node gets paths [0, n_pilot).
__global__ void batch_pilot_setup(int64_t n, int64_t n_pilot, int32_t K, int64_t *chunk_off,
                                  int64_t *first, int64_t *end) {
  const int64_t cpn = (n_pilot + K - 1) / K;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i <= n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    chunk_off[i] = i * cpn;
    if (i < n) {
      first[i] = 0;
      end[i] = n_pilot;
    }
  }
}

// Per node, from the exact sums of its pilot paths: the sample variance,
// N_i and the main work list's per-node entries.  K: paths per main-pass
// chunk.  Runs over positions j (node i = perm[j]); count2 is written by
// position (the main scan's order) and the other outputs by node.  Positions
// of invalid nodes (problem index out of range) get no chunks and are marked
// invalid in the sums, so that they finish with NaN and a count of 0.
__global__ void batch_pilot_stats(int64_t n, int64_t n_pilot, int32_t K, const int32_t *perm,
                                  const int64_t *cstart, NodeFix *fix, double inv_se2,
                                  int64_t n_min, int64_t n_max, int64_t *first2, int64_t *end2,
                                  int64_t *count2) {
  const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (j >= n) return;
  const int64_t i = perm[j];
  if (j >= cstart[4]) {
    fix[i].bad = 1;
    first2[i] = end2[i] = n_pilot;
    count2[j] = 0;
    return;
  }
  const NodeFix F = fix[i];
  double mean, m2;
  fix_moments(F, &mean, &m2);
  const double nt = static_cast<double>(F.n);
  const double var = nt > 1.0 ? m2 / (nt - 1.0) : 0.0;
  double want = ceil(var * inv_se2);
  const int64_t lo = max(n_min, n_pilot);
  int64_t Ni = want >= static_cast<double>(n_max) ? n_max : static_cast<int64_t>(want);
  Ni = max(lo, min(n_max, Ni));
  if (isnan(var)) Ni = lo;
  first2[i] = n_pilot;
  end2[i] = Ni;
  count2[j] = (Ni - n_pilot + K - 1) / K;
}

// Exclusive scan of count[0..n) into off[0..n] (single block, fixed order).
__global__ void __launch_bounds__(kScanBlock)
batch_scan(int64_t n, const int64_t *count, int64_t *off) {
  __shared__ int64_t part[kScanBlock];
  const int64_t per = (n + kScanBlock - 1) / kScanBlock;
  const int64_t b = threadIdx.x * per, e = min(n, b + per);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += count[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int t = 0; t < kScanBlock; ++t) {
      const int64_t v = part[t];
      part[t] = acc;
      acc += v;
    }
    off[n] = acc;
  }
  __syncthreads();
  int64_t acc = part[threadIdx.x];
  for (int64_t i = b; i < e; ++i) {
    off[i] = acc;
    acc += count[i];
  }
}

// Per-node flags of the adaptive batch: the target standard error not
// reached (N_i stopped at n_max, or the final variance exceeded the pilot's),
// or no estimate (a node outside the closed domain or of an unknown problem).
__global__ void batch_flags(int64_t n, const double *mean, const double *se, double target_se,
                            int32_t *flags) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  int32_t f = 0;
  if (isnan(mean[i])) f |= kNodeOutside;
  else if (se[i] > target_se) f |= kNodeSeUnmet;
  flags[i] = f;
}

namespace {

int combo_of(const pdd_problem &p) {
  if (p.kind == PDD_PROB_LAPLACE_EXPCOS && p.dim == 2 && p.geometry == PDD_GEOM_UNIT_SQUARE)
    return kComboSquareLaplace;
  if (p.kind == PDD_PROB_LAPLACE_EXPCOS && p.dim == 2 && p.geometry == PDD_GEOM_L_SHAPE)
    return kComboLShapeLaplace;
  if (p.kind == PDD_PROB_ELLIPTIC_MANUFACTURED && p.dim == 3 && p.geometry == PDD_GEOM_UNIT_CUBE)
    return kComboCubeElliptic;
  if (p.kind == PDD_PROB_POISSON_FOURIER && p.dim == 2 && p.geometry == PDD_GEOM_UNIT_SQUARE &&
      p.n_params >= 80)
    return kComboSquarePoisson;
  return -1;
}

struct BatchLayout {
  size_t off_first, off_end, off_chunk, off_first2, off_end2, off_cnt2, off_chunk2, off_fix,
      off_perm, off_cstart, total;
};

BatchLayout batch_layout(int64_t n) {
  BatchLayout L;
  size_t o = 256;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  const size_t nn = static_cast<size_t>(n);
  L.off_first = take(nn * 8);
  L.off_end = take(nn * 8);
  L.off_chunk = take((nn + 1) * 8);
  L.off_first2 = take(nn * 8);
  L.off_end2 = take(nn * 8);
  L.off_cnt2 = take(nn * 8);
  L.off_chunk2 = take((nn + 1) * 8);
  L.off_fix = take(nn * sizeof(NodeFix));
  L.off_perm = take(nn * sizeof(int32_t));
  L.off_cstart = take(8 * sizeof(int64_t));
  L.total = o;
  return L;
}

}  // namespace

// One launch of each present family's kernel over its chunk range.  The
// first family runs on the context's stream, the others on side streams
// forked from it and joined back (event record / wait, which stream capture
// records as graph dependencies), so the families' kernels overlap and the
// tail of one (lanes idle while its last chunks finish) is filled by another.
static pdd_status launch_families(pdd_ctx *ctx, const BatchArgs &a, const unsigned *grid) {
  int launched = 0;
  for (int c = 0; c < 4; ++c) {
    if (!grid[c]) continue;
    cudaStream_t s = ctx->stream;
    if (launched > 0) {  // side stream launched - 1
      if (launched == 1) PDD_CUDA_TRY(ctx, cudaEventRecord(ctx->batch_fork, ctx->stream));
      s = ctx->batch_side[launched - 1];
      PDD_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->batch_fork, 0));
    }
    switch (c) {
      case kComboSquareLaplace:
        batch_kernel<kComboSquareLaplace><<<grid[c], kBatchBlock, 0, s>>>(a);
        break;
      case kComboLShapeLaplace:
        batch_kernel<kComboLShapeLaplace><<<grid[c], kBatchBlock, 0, s>>>(a);
        break;
      case kComboCubeElliptic:
        batch_kernel<kComboCubeElliptic><<<grid[c], kBatchBlock, 0, s>>>(a);
        break;
      default:
        batch_kernel<kComboSquarePoisson><<<grid[c], kBatchBlock, 0, s>>>(a);
        break;
    }
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (launched > 0) {
      PDD_CUDA_TRY(ctx, cudaEventRecord(ctx->batch_join[launched - 1], s));
      PDD_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->batch_join[launched - 1], 0));
    }
    ++launched;
  }
  return PDD_OK;
}

// Side streams and events for launch_families (created once per context).
static pdd_status ensure_side_streams(pdd_ctx *ctx) {
  if (ctx->batch_fork) return PDD_OK;
  for (int k = 0; k < 3; ++k) {
    PDD_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->batch_side[k], cudaStreamNonBlocking));
    PDD_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->batch_join[k], cudaEventDisableTiming));
  }
  PDD_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->batch_fork, cudaEventDisableTiming));
  return PDD_OK;
}

static pdd_status enqueue_batch(pdd_ctx *ctx, const BatchArgs &proto, const BatchLayout &Lay,
                                const pdd_batch_nodes *nodes, const pdd_batch_params *bp,
                                int32_t K, int32_t Kp, const unsigned *grid, int4 combo_of_prob,
                                int32_t n_probs, double *d_mean, double *d_se,
                                int64_t *d_npaths) {
  char *base = static_cast<char *>(ctx->scratch);
  auto *counters = reinterpret_cast<unsigned long long *>(base);
  auto *first = reinterpret_cast<int64_t *>(base + Lay.off_first);
  auto *end = reinterpret_cast<int64_t *>(base + Lay.off_end);
  auto *chunk = reinterpret_cast<int64_t *>(base + Lay.off_chunk);
  auto *first2 = reinterpret_cast<int64_t *>(base + Lay.off_first2);
  auto *end2 = reinterpret_cast<int64_t *>(base + Lay.off_end2);
  auto *cnt2 = reinterpret_cast<int64_t *>(base + Lay.off_cnt2);
  auto *chunk2 = reinterpret_cast<int64_t *>(base + Lay.off_chunk2);
  auto *fix = reinterpret_cast<NodeFix *>(base + Lay.off_fix);
  auto *perm = reinterpret_cast<int32_t *>(base + Lay.off_perm);
  auto *cstart = reinterpret_cast<int64_t *>(base + Lay.off_cstart);
  auto *cursors = counters + 8;  // one per family
  const int64_t n = nodes->n;
  const unsigned nb = static_cast<unsigned>((n + 255) / 256);

  PDD_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, 256, ctx->stream));
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(fix, 0, static_cast<size_t>(n) * sizeof(NodeFix), ctx->stream));
  batch_partition<<<1, kScanBlock, 0, ctx->stream>>>(n, nodes->d_problem, n_probs, combo_of_prob,
                                                     perm, cstart, counters + 2);
  batch_pilot_setup<<<nb + 1, 256, 0, ctx->stream>>>(n, bp->n_pilot, Kp, chunk, first, end);
  BatchArgs a = proto;
  a.perm = perm;
  a.cstart = cstart;
  a.K = Kp;
  a.chunk_off = chunk;
  a.first = first;
  a.end = end;
  a.cursor = cursors;
  a.counters = counters;
  a.fix = fix;
  pdd_status st = launch_families(ctx, a, grid);
  if (st != PDD_OK) return st;
  batch_pilot_stats<<<nb, 256, 0, ctx->stream>>>(n, bp->n_pilot, K, perm, cstart, fix,
                                                 1.0 / (bp->target_se * bp->target_se),
                                                 bp->n_min, bp->n_max, first2, end2, cnt2);
  batch_scan<<<1, kScanBlock, 0, ctx->stream>>>(n, cnt2, chunk2);
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(cursors, 0, 4 * sizeof(unsigned long long), ctx->stream));
  a.K = K;
  a.chunk_off = chunk2;
  a.first = first2;
  a.end = end2;
  const auto ev = prof_slot(ctx);
  if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
  st = launch_families(ctx, a, grid);
  if (st != PDD_OK) return st;
  if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
  fix_finalize_kernel<<<nb, 256, 0, ctx->stream>>>(fix, n, d_mean, d_se, d_npaths, nullptr);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  return PDD_OK;
}

pdd_status batch_solve_impl(pdd_ctx *ctx, const pdd_problem *problems, int32_t n_problems,
                            const pdd_batch_nodes *nodes, const pdd_batch_params *bp,
                            double *d_mean, double *d_se, int64_t *d_npaths, int32_t use_graph,
                            pdd_diag *diag) {
  if (!problems || !nodes || !bp) return fail(ctx, PDD_EINVAL, "null argument");
  if (n_problems < 1 || n_problems > kMaxBatchProblems)
    return fail(ctx, PDD_EINVAL, "n_problems must be in [1, %d]", kMaxBatchProblems);
  if (nodes->n < 0 || nodes->n > (int64_t(1) << 31)) return fail(ctx, PDD_EINVAL, "n out of range");
  if (bp->n_pilot < 2 || bp->n_min < 1 || bp->n_max < bp->n_pilot || bp->n_max < bp->n_min)
    return fail(ctx, PDD_EINVAL, "need 2 <= n_pilot <= n_max and n_min <= n_max");
  if (bp->n_max > (int64_t(1) << 32)) return fail(ctx, PDD_EINVAL, "n_max above 2^32");
  if (!(bp->target_se > 0.0) || !std::isfinite(bp->target_se))
    return fail(ctx, PDD_EINVAL, "target_se must be > 0");
  if (bp->max_steps < 1 || bp->max_steps > 2147483647LL)
    return fail(ctx, PDD_EINVAL, "max_steps out of range");
  if (bp->chunk < 0 || bp->chunk > (1 << 20)) return fail(ctx, PDD_EINVAL, "chunk out of range");
  if (nodes->n > 0 && (!nodes->d_nodes || !nodes->d_problem || !nodes->d_dt || !d_mean || !d_se))
    return fail(ctx, PDD_EINVAL, "null buffer");
  BatchArgs proto;
  std::memset(&proto, 0, sizeof proto);
  for (int p = 0; p < n_problems; ++p) {
    const pdd_problem &P = problems[p];
    const int combo = combo_of(P);
    if (combo < 0) return fail(ctx, PDD_EINVAL, "problem %d has no batch kernel", p);
    if ((P.kind == PDD_PROB_LAPLACE_EXPCOS || P.kind == PDD_PROB_ELLIPTIC_MANUFACTURED) &&
        P.n_params > 0 && P.params && P.params[0] != 0.0)
      return fail(ctx, PDD_EINVAL, "problem %d has reflecting faces (no batch kernel)", p);
    if (!(P.sigma > 0.0) || !std::isfinite(P.sigma)) return fail(ctx, PDD_EINVAL, "sigma");
    if (P.n_params < 0 || P.n_params > kMaxParams || (P.n_params > 0 && !P.params))
      return fail(ctx, PDD_EINVAL, "params");
    BatchProblem &B = proto.probs[p];
    B.combo = combo;
    B.bridge = bp->bridge ? 1 : 0;
    B.sigma = P.sigma;
    B.c_kill = constant_kill(P.kind);
    B.mc.n_params = P.n_params;
    for (int i = 0; i < P.n_params; ++i) {
      if (!std::isfinite(P.params[i])) return fail(ctx, PDD_EINVAL, "non-finite parameter");
      B.mc.prm[i] = P.params[i];
      B.mc.prmf[i] = static_cast<float>(P.params[i]);
    }
  }
  proto.n_probs = n_problems;
  proto.nodes = nodes->d_nodes;
  proto.prob = nodes->d_problem;
  proto.dt = nodes->d_dt;
  proto.n = nodes->n;
  proto.rk = make_round_keys(bp->seed);
  proto.max_steps = static_cast<int32_t>(bp->max_steps);
  const int32_t K = bp->chunk > 0 ? bp->chunk : (ctx->batch_chunk > 0 ? ctx->batch_chunk : 256);
  proto.K = K;
  if (diag) {
    diag->path_steps = 0;
    diag->capped = 0;
  }
  if (nodes->n == 0) return PDD_OK;
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // one kernel per family present in the problem list, each sized by its own
  // occupancy (0 = family absent)
  unsigned grid[4] = {0, 0, 0, 0};
  int cp[4] = {4, 4, 4, 4};
  for (int p = 0; p < n_problems; ++p) {
    const int c = proto.probs[p].combo;
    cp[p] = c;
    if (grid[c]) continue;
    int bps = 0;
    const void *fn = c == kComboSquareLaplace ? reinterpret_cast<const void *>(batch_kernel<kComboSquareLaplace>)
                   : c == kComboLShapeLaplace ? reinterpret_cast<const void *>(batch_kernel<kComboLShapeLaplace>)
                   : c == kComboCubeElliptic  ? reinterpret_cast<const void *>(batch_kernel<kComboCubeElliptic>)
                                              : reinterpret_cast<const void *>(batch_kernel<kComboSquarePoisson>);
    PDD_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBatchBlock, 0));
    if (bps < 1) bps = 1;
    if (ctx->path_blocks_per_sm > 0) bps = std::min(bps, ctx->path_blocks_per_sm);
    grid[c] = static_cast<unsigned>(bps * ctx->num_sms);
  }
  const int4 combo_of_prob = make_int4(cp[0], cp[1], cp[2], cp[3]);
  unsigned max_grid = 0;
  for (int c = 0; c < 4; ++c) max_grid = std::max(max_grid, grid[c]);
  // pilot chunks: the pilot is small (n_pilot paths per node), and chunks of
  // K paths could leave lanes without work; aim at >= 8 chunks per lane
  const double pilot_paths = static_cast<double>(nodes->n) * static_cast<double>(bp->n_pilot);
  const double per_lane = pilot_paths / (8.0 * max_grid * kBatchBlock);
  const int32_t Kp = static_cast<int32_t>(std::max(1.0, std::min<double>(K, std::floor(per_lane))));
  const BatchLayout Lay = batch_layout(nodes->n);
  pdd_status st = ensure_scratch(ctx, Lay.total);
  if (st != PDD_OK) return st;
  st = ensure_side_streams(ctx);
  if (st != PDD_OK) return st;

  if (!use_graph) {
    st = enqueue_batch(ctx, proto, Lay, nodes, bp, K, Kp, grid, combo_of_prob, n_problems,
                       d_mean, d_se, d_npaths);
    if (st != PDD_OK) return st;
  } else {
    if (!ctx->stream) return fail(ctx, PDD_EINVAL, "graph capture needs a non-default stream");
    // the graph bakes in every pointer and scalar: rebuild when any changes
    BatchGraphKey key{};
    key.nodes = *nodes;
    key.bp = *bp;
    key.out[0] = d_mean;
    key.out[1] = d_se;
    key.out[2] = d_npaths;
    key.scratch = ctx->scratch;
    for (int c = 0; c < 4; ++c) key.grid[c] = grid[c];
    key.K = K;
    key.probs_hash = 0;
    const unsigned char *pb = reinterpret_cast<const unsigned char *>(proto.probs);
    for (size_t i = 0; i < sizeof(proto.probs); ++i)
      key.probs_hash = (key.probs_hash ^ pb[i]) * 1099511628211ull;
    if (!ctx->batch_graph || std::memcmp(&key, &ctx->batch_key, sizeof key) != 0) {
      if (ctx->batch_graph) {
        cudaGraphExecDestroy(ctx->batch_graph);
        ctx->batch_graph = nullptr;
      }
      const bool prof = ctx->profiling;
      ctx->profiling = false;  // no event records inside the capture
      PDD_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      st = enqueue_batch(ctx, proto, Lay, nodes, bp, K, Kp, grid, combo_of_prob, n_problems,
                       d_mean, d_se, d_npaths);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
      ctx->profiling = prof;
      if (st != PDD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
      const cudaError_t ei = cudaGraphInstantiate(&ctx->batch_graph, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) return cuda_fail(ctx, ei, "cudaGraphInstantiate");
      ctx->batch_key = key;
    }
    const auto ev = prof_slot(ctx);
    if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
    PDD_CUDA_TRY(ctx, cudaGraphLaunch(ctx->batch_graph, ctx->stream));
    if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
  }
  if (diag && diag->d_node_flags) {
    batch_flags<<<static_cast<unsigned>((nodes->n + 255) / 256), 256, 0, ctx->stream>>>(
        nodes->n, d_mean, d_se, bp->target_se, diag->d_node_flags);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
  }
  if (diag) {
    unsigned long long h[4] = {0, 0, 0, 0};
    PDD_CUDA_TRY(ctx, cudaMemcpyAsync(h, ctx->scratch, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    diag->path_steps = static_cast<int64_t>(h[0]);
    diag->capped = static_cast<int64_t>(h[1]);
    if (h[2]) return fail(ctx, PDD_EINVAL, "%llu nodes outside the closed domain", h[2]);
    if (h[1]) return fail(ctx, PDD_ECAP, "%llu paths hit max_steps", h[1]);
  }
  return PDD_OK;
}

}  // namespace pdd
