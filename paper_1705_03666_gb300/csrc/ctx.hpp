// ctx.hpp -- the library context behind the C ABI (include/pdd.h): device,
// stream, problem constants and the library-owned device scratch.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "pdd.h"
#include "models.cuh"

// Everything a captured batch graph depends on.
struct BatchGraphKey {
  pdd_batch_nodes nodes;
  pdd_batch_params bp;
  void *out[3];
  void *scratch;
  unsigned grid[4];
  int32_t K;
  unsigned long long probs_hash;
};

struct pdd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  pdd_problem prob{};
  std::vector<double> params;
  pdd::ModelConst mc{};
  int num_sms = 0;
  // library-owned scratch, grown on demand
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  // a second library-owned buffer for results an entry point keeps across
  // its own calls of other entry points (which use `scratch`)
  void *aux = nullptr;
  size_t aux_bytes = 0;
  std::string last_error;
  // launch shape of the path kernels (warps per block fixed at compile time;
  // resident blocks per SM chosen by the occupancy query or the tuner)
  int path_blocks_per_sm = 0;
  uint64_t wave_max_paths = 1ull << 29;
  // batch solve: lane-chunk size and the cached graph of the last call
  int batch_chunk = 0;
  cudaGraphExec_t batch_graph = nullptr;
  BatchGraphKey batch_key{};
  // batch solve: side streams and events that run the per-family kernels
  // concurrently (forked from and joined back into `stream`); created on
  // first use
  cudaStream_t batch_side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t batch_fork = nullptr;
  cudaEvent_t batch_join[3] = {nullptr, nullptr, nullptr};
  // kernel timing (pdd_profile): event pairs recorded around path launches
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  size_t prof_used = 0;
};

namespace pdd {

// Reflecting faces of the problem (bit j: face j of the box), from the
// optional [mask, phi] parameters of the Laplace and 3-D manufactured
// families; 0 for every other problem.
inline int reflect_mask(const pdd_ctx *ctx) {
  if (ctx->prob.kind != PDD_PROB_LAPLACE_EXPCOS && ctx->prob.kind != PDD_PROB_ELLIPTIC_MANUFACTURED)
    return 0;
  if (ctx->params.size() < 2) return 0;
  return static_cast<int>(ctx->params[0]);
}

// The paper's constant killing rate c of a family (Eq. 2.3 in the elliptic
// form; 0 where the family has no killing): the 3-D manufactured problem
// (1/2) Lap u + b . grad u - u = F has c = -1.
inline double constant_kill(int kind) {
  return kind == PDD_PROB_ELLIPTIC_MANUFACTURED ? -1.0 : 0.0;
}

inline pdd_status fail(pdd_ctx *ctx, pdd_status st, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return st;
}

inline pdd_status cuda_fail(pdd_ctx *ctx, cudaError_t e, const char *where) {
  return fail(ctx, PDD_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define PDD_CUDA_TRY(ctx, expr)                                   \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return ::pdd::cuda_fail(ctx, _e, #expr); \
  } while (0)

// Make sure the scratch holds at least `bytes`; grows by reallocation.
inline pdd_status ensure_scratch(pdd_ctx *ctx, size_t bytes) {
  if (ctx->scratch_bytes >= bytes) return PDD_OK;
  if (ctx->scratch) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
  }
  size_t want = bytes + (bytes >> 3);
  cudaError_t e = cudaMalloc(&ctx->scratch, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, PDD_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", want,
                cudaGetErrorString(e));
  }
  ctx->scratch_bytes = want;
  return PDD_OK;
}

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Make sure the auxiliary buffer holds at least `bytes`.
inline pdd_status ensure_aux(pdd_ctx *ctx, size_t bytes) {
  if (ctx->aux_bytes >= bytes) return PDD_OK;
  if (ctx->aux) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    cudaFree(ctx->aux);
    ctx->aux = nullptr;
    ctx->aux_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->aux, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, PDD_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  ctx->aux_bytes = bytes;
  return PDD_OK;
}

// Event pair for the next profiled launch (nullptr events when profiling is
// off or event creation failed).
inline std::pair<cudaEvent_t, cudaEvent_t> prof_slot(pdd_ctx *ctx) {
  if (!ctx->profiling) return {nullptr, nullptr};
  if (ctx->prof_used == ctx->prof_events.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return {nullptr, nullptr};
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return {nullptr, nullptr};
    }
    ctx->prof_events.push_back({a, b});
  }
  return ctx->prof_events[ctx->prof_used++];
}

// Entry points implemented in the kernel translation units.
pdd_status interface_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                const pdd_mc_params *mc, double *d_mean, double *d_se,
                                int64_t *d_npaths, pdd_diag *diag);
pdd_status branching_solve_impl(pdd_ctx *ctx, const double *d_nodes_xt, int64_t n,
                                const pdd_branch_params *bp, double *d_mean, double *d_se,
                                int64_t *d_nkept, pdd_diag *diag);
pdd_status subdomain_solve_impl(pdd_ctx *ctx, const pdd_subdomain *sd, const double *d_iface_s,
                                const double *d_iface_vals, int64_t m, double *d_u,
                                int64_t *iters, double *resid);
pdd_status interface_grad_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                               const pdd_mc_params *mc, const double *d_grad_out, double *d_jac,
                               double *d_jac_se, double *d_dtheta, double *d_dphi,
                               pdd_diag *diag);
pdd_status batch_solve_impl(pdd_ctx *ctx, const pdd_problem *problems, int32_t n_problems,
                            const pdd_batch_nodes *nodes, const pdd_batch_params *bp,
                            double *d_mean, double *d_se, int64_t *d_npaths, int32_t use_graph,
                            pdd_diag *diag);
pdd_status interface_solve_naive_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                      const pdd_mc_params *mc, double *d_mean, double *d_se,
                                      int64_t *d_npaths);
pdd_status autotune_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_mc_params *mc,
                         double *d_scratch_out, int32_t repeats, int32_t *best_bps,
                         double *best_ms);
pdd_status autotune_batch_impl(pdd_ctx *ctx, const pdd_problem *problems, int32_t n_problems,
                               const pdd_batch_nodes *nodes, const pdd_batch_params *bp,
                               double *d_scratch_out, int32_t repeats, int32_t *best_chunk,
                               double *best_ms);
pdd_status normals_impl(pdd_ctx *ctx, uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3,
                        int64_t n_pairs, float *d_z, float *d_u);
pdd_status wos_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_wos_params *wp,
                          double *d_mean, double *d_se, int64_t *d_npaths, pdd_diag *diag);
pdd_status branching_grid_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                     const double *h_times, int32_t m,
                                     const pdd_grid_branch_params *bp, double *d_mean,
                                     double *d_se, int64_t *d_nkept, pdd_diag *diag);
pdd_status reflect_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                              const pdd_mc_params *mc, double *d_mean, double *d_se,
                              int64_t *d_npaths, pdd_diag *diag);
pdd_status mlmc_level_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_mlmc_params *mp,
                           double *d_mean, double *d_var, double *d_fine, double *d_coarse,
                           pdd_diag *diag);
pdd_status mlmc_solve_impl(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                           const pdd_mlmc_params *mp, int32_t n_levels,
                           const int64_t *h_n_per_level, double *d_mean, double *d_se,
                           double *d_level_mean, double *d_level_var, pdd_diag *diag);
pdd_status interface_interp_impl(pdd_ctx *ctx, int32_t n_planes, const int32_t *h_axis,
                                 const double *h_pos, const int64_t *h_node_count,
                                 const double *d_nodes, const double *d_vals, int32_t n_bnd,
                                 const int64_t *h_query_count, const double *d_query,
                                 double *d_out);
pdd_status subdomain_solve3d_impl(pdd_ctx *ctx, const pdd_subdomain *sd, const double *d_face,
                                  int64_t m, double *d_u, int64_t *iters, double *resid);
pdd_status subdomain_solve3d_batch_impl(pdd_ctx *ctx, const pdd_subdomain *sds, int32_t nb,
                                        const double *d_face, int64_t m, double *d_u,
                                        int64_t *iters, double *resid, int64_t *iters_each,
                                        double *resid_each);
pdd_status philox_stream_impl(pdd_ctx *ctx, uint64_t seed, uint32_t j0, uint32_t c1,
                              uint32_t c2, uint32_t c3, int64_t n_blocks, uint32_t *d_out);

}  // namespace pdd
