// grad.cu -- pdd_interface_grad: derivatives of the node estimates with
// respect to the problem's parameters, paths recomputed from their Philox keys
// (nothing is stored by the forward solve).
//
// For the Poisson-Fourier family (params theta[64], phi[16]):
//   d u / d theta_mn = E[cos(m pi X_tau,x) cos(n pi X_tau,y)]   (exact pathwise:
//                      the paths do not depend on theta and g is linear in it),
//   d u / d phi_j    = E[s L_j],  L_j = sum over steps of xi_n . db/dphi_j(X_n)
//                      sqrt(dt)/sigma  (likelihood ratio of the Gaussian
//                      transition of the discrete scheme; the bridge uniform
//                      and the exit rule do not depend on phi).
// The path kernel runs in its gradient mode and writes one 80-byte record per
// path (score, exit point, L); jac_reduce_kernel and jac_merge_kernel form the
// per-node means of the 80 components with compensated sums in a fixed order;
// vjp_kernel contracts them with a cotangent over the nodes.
#include <cmath>
#include <cstring>

#include "ctx.hpp"
#include "path_kernel.cuh"
#include "reduce.cuh"

namespace pdd {

constexpr int kJacW = 80;       // 64 theta + 16 phi components
constexpr int kJacLanes = 8;    // threads per path: thread m owns cos(m pi x)
constexpr int kJacBlock = 256;  // 32 path groups x 8
constexpr int kJacGroups = kJacBlock / kJacLanes;

// Merge a batch of nb records with sums S1, S2 of one component into the
// node's running (count, mean, M2) (Chan).
__device__ __forceinline__ void jac_chan_merge(NodeAcc *jacc, uint64_t node, int comp, double S1,
                                               double S2, double nb) {
  const double mean_b = S1 / nb;
  const double m2_b = fmax(0.0, S2 - S1 * mean_b);
  NodeAcc A = jacc[node * kJacW + comp];
  const double nt = A.n + nb;
  const double d = mean_b - A.mean;
  A.mean = A.mean + d * (nb / nt);
  A.m2 = A.m2 + m2_b + d * d * (A.n * nb / nt);
  A.n = nt;
  jacc[node * kJacW + comp] = A;
}

// Per part of a node's records (one block): for each path record, thread m
// of a path group forms cos(m pi x) and, by the Chebyshev recurrence from
// cos(pi y), cos(n pi y) for n = 0..7, and accumulates its eight theta components (8m + n) and the two
// phi components m and 8 + m (s * L_j) with their squares.  A group takes
// its records four at a time (records grp + 32 r of the block, r = 0..3):
// thread m forms cos(pi y) of record m mod 4 once and the group shares the
// four values by shuffles; the four contributions of each component are
// summed in binary32 (error <= 3 u of their absolute sum) and the block sum
// goes into a two-float sum on the FP32 pipe (~48-bit; FP64 is a 1/64-rate
// pipe here), so a row carries at most 3 u of its mean absolute contribution
// beyond the contributions' own evaluation.  The squares, which feed only the
// standard error, take the same four-record blocks by FMA.  A node's records
// of the wave are split into `parts` contiguous ranges, one block each (so
// that a wave of a few hundred nodes still fills the GPU); a block combines
// its 32 groups in FP64 in a fixed order and writes the part's two sums per
// component, and jac_merge_kernel adds the parts in order and merges them
// into the node's running (count, mean, M2) per component (Chan); with one
// part the block merges its sums itself.  Launch
// bounds of three blocks per SM (80 registers): at 105 registers and two
// blocks the kernel was 24 % slower.
__global__ void __launch_bounds__(kJacBlock, 3)
jac_reduce_kernel(const GradRec *__restrict__ rec, uint64_t begin, uint64_t end,
                  uint64_t n_paths, uint64_t node_lo, int parts, double2 *part_sums,
                  NodeAcc *jacc) {
  constexpr int kRecs = 4;  // records per group and block
  const uint64_t node = node_lo + blockIdx.x / parts;
  const uint64_t part = blockIdx.x % parts;
  const uint64_t nlo = max(begin, node * n_paths);
  const uint64_t nhi = min(end, (node + 1) * n_paths);
  const uint64_t ncnt = nhi > nlo ? nhi - nlo : 0;
  const uint64_t lo = nlo + ncnt * part / parts;
  const uint64_t hi = nlo + ncnt * (part + 1) / parts;
  double2 *out = part_sums + static_cast<uint64_t>(blockIdx.x) * kJacW;
  if (lo >= hi) {  // an empty part adds zeros
    if (parts > 1 && threadIdx.x < kJacW) out[threadIdx.x] = make_double2(0.0, 0.0);
    return;
  }
  const GradRec *r = rec + (lo - begin);
  const uint64_t cnt = hi - lo;
  const int m = threadIdx.x % kJacLanes, grp = threadIdx.x / kJacLanes;
  const float fm = static_cast<float>(m);
  F2Sum s1[10], s2[10];  // two-float sums on the FP32 pipe (see reduce.cuh)
  // block-uniform trip count (the shuffles need every lane of the warp);
  // records past the end contribute exact zeros
  const uint64_t trips = (cnt + kJacGroups * kRecs - 1) / (kJacGroups * kRecs);
  for (uint64_t it = 0; it < trips; ++it) {
    const uint64_t base = it * (kJacGroups * kRecs) + grp;
    const uint64_t py = min(base + kJacGroups * (m % kRecs), cnt - 1);
    const float cy_own = cospif(r[py].y);
    float t1[10], t2[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) t1[c] = t2[c] = 0.0f;
#pragma unroll
    for (int q = 0; q < kRecs; ++q) {
      const uint64_t p = base + kJacGroups * q;
      const bool ok = p < cnt;
      const uint64_t pc = ok ? p : cnt - 1;
      const float cy1 = __shfl_sync(kFull, cy_own, q, kJacLanes);
      const float cxm = ok ? cospif(fm * r[pc].x) : 0.0f;
      const float two_c = 2.0f * cy1;
      float cprev = 1.0f, ccur = cy1;
      float v[10];
      v[0] = cxm;
      v[1] = cxm * cy1;
#pragma unroll
      for (int n = 2; n < 8; ++n) {
        const float cn = two_c * ccur - cprev;
        cprev = ccur;
        ccur = cn;
        v[n] = cxm * cn;
      }
      const float sc = r[pc].s;
      v[8] = ok ? sc * r[pc].L[m] : 0.0f;
      v[9] = ok ? sc * r[pc].L[8 + m] : 0.0f;
#pragma unroll
      for (int c = 0; c < 10; ++c) {
        t1[c] += v[c];
        t2[c] = fmaf(v[c], v[c], t2[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 10; ++c) {
      s1[c].add(t1[c]);
      s2[c].add(t2[c]);
    }
  }
  __shared__ double sh1[kJacGroups][kJacLanes * 10], sh2[kJacGroups][kJacLanes * 10];
#pragma unroll
  for (int c = 0; c < 10; ++c) {
    sh1[grp][m * 10 + c] = static_cast<double>(s1[c].hi) + static_cast<double>(s1[c].lo);
    sh2[grp][m * 10 + c] = static_cast<double>(s2[c].hi) + static_cast<double>(s2[c].lo);
  }
  __syncthreads();
  // 80 threads finish one component each: slot t = m*10 + c
  if (threadIdx.x < kJacLanes * 10) {
    const int t = threadIdx.x;
    double S1 = 0.0, S2 = 0.0;
    for (int gq = 0; gq < kJacGroups; ++gq) {
      S1 += sh1[gq][t];
      S2 += sh2[gq][t];
    }
    const int mm = t / 10, c = t % 10;
    const int comp = c < 8 ? 8 * mm + c : (c == 8 ? 64 + mm : 72 + mm);
    if (parts > 1)
      out[comp] = make_double2(S1, S2);
    else  // one part: merged here (part_sums unused)
      jac_chan_merge(jacc, node, comp, S1, S2, static_cast<double>(cnt));
  }
}

// One block per node of the wave, one thread per component: the parts' sums
// added in part order, then merged into the node's running (count, mean, M2)
// (Chan).
__global__ void jac_merge_kernel(const double2 *part_sums, uint64_t begin, uint64_t end,
                                 uint64_t n_paths, uint64_t node_lo, int parts, NodeAcc *jacc) {
  const int comp = threadIdx.x;
  if (comp >= kJacW) return;
  const uint64_t node = node_lo + blockIdx.x;
  const uint64_t lo = max(begin, node * n_paths);
  const uint64_t hi = min(end, (node + 1) * n_paths);
  if (lo >= hi) return;
  double S1 = 0.0, S2 = 0.0;
  for (int q = 0; q < parts; ++q) {
    const double2 v = part_sums[(static_cast<uint64_t>(blockIdx.x) * parts + q) * kJacW + comp];
    S1 += v.x;
    S2 += v.y;
  }
  jac_chan_merge(jacc, node, comp, S1, S2, static_cast<double>(hi - lo));
}

__global__ void jac_finalize_kernel(const NodeAcc *jacc, int64_t count, double *jac,
                                    double *jac_se) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= count) return;
  const NodeAcc A = jacc[i];
  jac[i] = A.mean;
  if (jac_se) jac_se[i] = A.n > 1.0 ? sqrt(A.m2 / (A.n - 1.0) / A.n) : 0.0;
}

// out[c] = sum_i w[i] jac[i][c], fixed order (one block per component).
__global__ void vjp_kernel(const double *jac, const double *w, int64_t n, double *dtheta,
                           double *dphi) {
  const int c = blockIdx.x;
  CSum s;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s.add(w[i] * jac[i * kJacW + c]);
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) s.merge(shfl_xor(s, m));
  __shared__ CSum sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum t = sh[0];
    for (int k = 1; k < static_cast<int>(blockDim.x >> 5); ++k) t.merge(sh[k]);
    if (c < 64) {
      if (dtheta) dtheta[c] = t.value();
    } else if (dphi) {
      dphi[c - 64] = t.value();
    }
  }
}

// Per-path dump: score to score_out, (x, y, L_1..L_16) to aux_out [count][18].
__global__ void grad_dump_kernel(const GradRec *rec, uint64_t count, double *score_out,
                                 double *aux_out) {
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    if (score_out) score_out[i] = rec[i].s;
    if (aux_out) {
      double *o = aux_out + i * 18;
      o[0] = rec[i].x;
      o[1] = rec[i].y;
      for (int j = 0; j < kMaxLR; ++j) o[2 + j] = rec[i].L[j];
    }
  }
}

pdd_status interface_grad_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                               const pdd_mc_params *mc, const double *d_grad_out, double *d_jac,
                               double *d_jac_se, double *d_dtheta, double *d_dphi,
                               pdd_diag *diag) {
  if (!mc) return fail(ctx, PDD_EINVAL, "mc is NULL");
  if (ctx->prob.kind != PDD_PROB_POISSON_FOURIER)
    return fail(ctx, PDD_EINVAL, "derivatives are provided for the POISSON_FOURIER family");
  if (mc->precision != PDD_FP32) return fail(ctx, PDD_EINVAL, "gradient paths are FP32");
  if (n < 0 || n > (int64_t(1) << 32)) return fail(ctx, PDD_EINVAL, "n out of range");
  if (mc->n_paths < 1) return fail(ctx, PDD_EINVAL, "n_paths < 1");
  if (mc->path_offset < 0 || mc->path_offset + mc->n_paths > (int64_t(1) << 32))
    return fail(ctx, PDD_EINVAL, "path indices must fit in 32 bits");
  if (mc->node_offset < 0 || mc->node_offset + n > (int64_t(1) << 32))
    return fail(ctx, PDD_EINVAL, "node stream indices must fit in 32 bits");
  if (!(mc->dt > 0.0) || !std::isfinite(mc->dt)) return fail(ctx, PDD_EINVAL, "dt must be > 0");
  if (ctx->prob.sigma * ctx->prob.sigma * mc->dt > 1.0 / 36.0)
    return fail(ctx, PDD_EINVAL, "sigma^2 dt must be <= 1/36");
  if (mc->max_steps < 1 || mc->max_steps > 2147483647LL)
    return fail(ctx, PDD_EINVAL, "max_steps out of range");
  if (n > 0 && !d_nodes) return fail(ctx, PDD_EINVAL, "null nodes");
  if ((d_dtheta || d_dphi) && !d_grad_out)
    return fail(ctx, PDD_EINVAL, "d_dtheta/d_dphi need d_grad_out");
  if (diag) {
    diag->path_steps = 0;
    diag->capped = 0;
  }
  if (n == 0) {
    if (d_dtheta) PDD_CUDA_TRY(ctx, cudaMemsetAsync(d_dtheta, 0, 64 * sizeof(double), ctx->stream));
    if (d_dphi) PDD_CUDA_TRY(ctx, cudaMemsetAsync(d_dphi, 0, 16 * sizeof(double), ctx->stream));
    return PDD_OK;
  }
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));

  const uint64_t N = static_cast<uint64_t>(mc->n_paths);
  const uint64_t total = static_cast<uint64_t>(n) * N;
  const uint64_t wave = std::min<uint64_t>(total, std::max<uint64_t>(1, ctx->wave_max_paths / 8));
  const size_t jacc_off = 256;
  const size_t jac_off = align_up(jacc_off + static_cast<size_t>(n) * kJacW * sizeof(NodeAcc), 256);
  const size_t rec_off = align_up(jac_off + static_cast<size_t>(n) * kJacW * sizeof(double), 256);
  // parts per node in the Jacobian reduction: four while a node has at least
  // 4 x 8192 paths (a wave then holds few nodes), fewer below (fixed by
  // n_paths, so the reduction order does not depend on the device)
  const int parts = static_cast<int>(std::min<uint64_t>(4, std::max<uint64_t>(1, N / 8192)));
  const uint64_t part_blocks = parts > 1 ? (wave / N + 2) * parts : 0;  // N >= 16384 here
  const size_t part_off = align_up(rec_off + wave * sizeof(GradRec), 256);
  const size_t bytes = align_up(part_off + part_blocks * kJacW * sizeof(double2), 256);
  pdd_status st = ensure_scratch(ctx, bytes);
  if (st != PDD_OK) return st;
  char *base = static_cast<char *>(ctx->scratch);
  auto *counters = reinterpret_cast<unsigned long long *>(base);
  auto *cursor = counters + 4;
  auto *jacc = reinterpret_cast<NodeAcc *>(base + jacc_off);
  double *jac = reinterpret_cast<double *>(base + jac_off);
  auto *rec = reinterpret_cast<GradRec *>(base + rec_off);
  auto *part_sums = reinterpret_cast<double2 *>(base + part_off);
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, jac_off, ctx->stream));

  PathArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes = d_nodes;
  a.n_paths = N;
  a.path_offset = static_cast<uint64_t>(mc->path_offset);
  a.node_offset = static_cast<uint32_t>(mc->node_offset);
  a.cursor = cursor;
  a.counters = counters;
  a.score = rec;
  a.rk = make_round_keys(mc->seed);
  const double sig = ctx->prob.sigma, dt = mc->dt;
  a.inv_s2dt = 1.0 / (sig * sig * dt);
  a.dt_d = dt;
  a.sdt_d = sig * std::sqrt(dt);
  a.thr_d = 9.0 * sig * sig * dt;
  a.ecdt_d = 1.0;
  a.dt_f = static_cast<float>(dt);
  a.sdt_f = static_cast<float>(a.sdt_d);
  a.thr_f = static_cast<float>(a.thr_d);
  a.l2cdt_f = 0.0f;
  a.lr_scale = static_cast<float>(std::sqrt(dt) / sig);
  a.max_steps = static_cast<int32_t>(mc->max_steps);
  a.bridge = mc->bridge ? 1 : 0;
  a.mc = ctx->mc;

  auto kern = path_kernel<PoissonFourier, Box<2>, float, true>;
  int bps = 0;
  PDD_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kPathBlockOf<float>, 0));
  if (bps < 1) bps = 1;
  if (ctx->path_blocks_per_sm > 0) bps = std::min(bps, ctx->path_blocks_per_sm);
  uint64_t grid = static_cast<uint64_t>(bps) * ctx->num_sms;
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (wave + kPathBlockOf<float> - 1) / kPathBlockOf<float>));

  for (uint64_t b0 = 0; b0 < total; b0 += wave) {
    const uint64_t b1 = std::min(total, b0 + wave);
    if (b0 > 0) PDD_CUDA_TRY(ctx, cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), ctx->stream));
    a.begin = b0;
    a.end = b1;
    a.steps = (diag && diag->d_path_steps) ? diag->d_path_steps + b0 : nullptr;
    const auto ev = prof_slot(ctx);
    if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
    kern<<<static_cast<unsigned>(grid), kPathBlockOf<float>, 0, ctx->stream>>>(a);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
    const uint64_t node_lo = b0 / N, node_hi = (b1 - 1) / N;
    const unsigned nw = static_cast<unsigned>(node_hi - node_lo + 1);
    jac_reduce_kernel<<<nw * parts, kJacBlock, 0, ctx->stream>>>(rec, b0, b1, N, node_lo, parts,
                                                                  part_sums, jacc);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    if (parts > 1) {
      jac_merge_kernel<<<nw, 128, 0, ctx->stream>>>(part_sums, b0, b1, N, node_lo, parts, jacc);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
    }
    if (diag && (diag->d_path_score || diag->d_path_aux)) {
      const uint64_t cnt = b1 - b0;
      const unsigned g = static_cast<unsigned>(std::min<uint64_t>((cnt + 255) / 256, 8192));
      grad_dump_kernel<<<g, 256, 0, ctx->stream>>>(
          rec, cnt, diag->d_path_score ? diag->d_path_score + b0 : nullptr,
          diag->d_path_aux ? diag->d_path_aux + b0 * 18 : nullptr);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  const int64_t cnt = n * kJacW;
  jac_finalize_kernel<<<static_cast<unsigned>((cnt + 255) / 256), 256, 0, ctx->stream>>>(
      jacc, cnt, d_jac ? d_jac : jac, d_jac_se);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (d_grad_out && (d_dtheta || d_dphi)) {
    vjp_kernel<<<kJacW, 256, 0, ctx->stream>>>(d_jac ? d_jac : jac, d_grad_out, n, d_dtheta, d_dphi);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
  }
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

}  // namespace pdd
