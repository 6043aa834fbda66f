// api.cu -- the extern "C" entry points of include/pdd.h: argument checks,
// context lifetime and dispatch to the kernel translation units.
#include <cmath>
#include <new>
#include <string>

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define PDD_HAVE_NVTX 1
#endif

#include "ctx.hpp"

using pdd::fail;

namespace {

// Reason the calling thread's last pdd_create failed ("" after a success):
// there is no context yet to hold it.
thread_local std::string g_create_error;

pdd_status create_fail(pdd_status st, const char *why) {
  g_create_error = why;
  return st;
}

// Named NVTX range around an entry point's host work and launches (a span
// on a profiler's timeline; a no-op when no tool is attached, and compiled
// out where the toolkit has no NVTX headers).
struct TraceRange {
#ifdef PDD_HAVE_NVTX
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
#else
  explicit TraceRange(const char *) {}
#endif
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

bool finite_params(const pdd_problem *p) {
  for (int i = 0; i < p->n_params; ++i)
    if (!std::isfinite(p->params[i])) return false;
  return true;
}

// Optional reflecting faces: params = [] or [mask, phi], mask an integer with
// one bit per face of the box, phi <= 0 (Eq. 2.4 requires phi <= 0).
const char *check_robin(const pdd_problem *p) {
  if (p->n_params == 0) return nullptr;
  if (p->n_params != 2) return "reflecting-face params are [mask, phi]";
  const double m = p->params[0];
  if (m != std::floor(m) || m < 0.0 || m >= static_cast<double>(1 << (2 * p->dim)))
    return "reflect mask must be an integer with one bit per face";
  if (p->params[1] > 0.0) return "Robin phi must be <= 0";
  return nullptr;
}

// Family / dimension / geometry combinations that have kernels, and the KPP
// offspring law check (q a probability distribution, Assumption 3.1; alpha_k
// real weights with q_k > 0 wherever alpha_k != 0, Sec. 3.2).
const char *check_problem(const pdd_problem *p) {
  if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return "sigma must be > 0";
  if (p->n_params < 0 || p->n_params > pdd::kMaxParams) return "n_params out of range";
  if (p->n_params > 0 && !p->params) return "params is NULL";
  if (!finite_params(p)) return "non-finite parameter";
  switch (p->kind) {
    case PDD_PROB_LAPLACE_EXPCOS:
      if (p->dim != 2 || (p->geometry != PDD_GEOM_UNIT_SQUARE && p->geometry != PDD_GEOM_L_SHAPE))
        return "LAPLACE_EXPCOS needs dim 2 on the unit square or the L-shape";
      if (p->geometry == PDD_GEOM_L_SHAPE && p->n_params > 0 && p->params[0] != 0.0)
        return "reflecting faces need the unit square";
      return check_robin(p);
    case PDD_PROB_ELLIPTIC_MANUFACTURED:
      if (p->dim != 3 || p->geometry != PDD_GEOM_UNIT_CUBE)
        return "ELLIPTIC_MANUFACTURED needs dim 3 on the unit cube";
      return check_robin(p);
    case PDD_PROB_POISSON_FOURIER:
      if (p->dim != 2 || p->geometry != PDD_GEOM_UNIT_SQUARE)
        return "POISSON_FOURIER needs dim 2 on the unit square";
      if (p->n_params < 80) return "POISSON_FOURIER needs 80 params (theta[64], phi[16])";
      return nullptr;
    case PDD_PROB_KPP: {
      if (p->dim < 1 || p->dim > 2) return "KPP needs dim 1 or 2";
      if (p->geometry != PDD_GEOM_FREE_SPACE &&
          !(p->dim == 1 && p->geometry == PDD_GEOM_INTERVAL) &&
          !(p->dim == 2 && (p->geometry == PDD_GEOM_UNIT_SQUARE || p->geometry == PDD_GEOM_L_SHAPE)))
        return "KPP geometry: free space, the interval (1-D), the unit square or the L-shape (2-D)";
      if (p->n_params < 4) return "KPP needs params";
      if (!(p->params[0] > 0.0)) return "KPP beta must be > 0";
      const double kind = p->params[1];
      if (kind != 0.0 && kind != 1.0 && kind != 2.0 && kind != 3.0) return "unknown psi kind";
      const double Kd = p->params[3];
      if (Kd != std::floor(Kd) || Kd < 0.0 || Kd > 7.0) return "K must be an integer in [0,7]";
      const int K = static_cast<int>(Kd);
      if (p->n_params < 6 + 2 * K) return "KPP needs q[0..K] and alpha[0..K]";
      double sum = 0.0;
      for (int k = 0; k <= K; ++k) {
        const double q = p->params[4 + k], al = p->params[5 + K + k];
        if (q < 0.0) return "q_k must be >= 0";
        if (al != 0.0 && !(q > 0.0)) return "q_k must be > 0 where alpha_k != 0";
        sum += q;
      }
      if (std::fabs(sum - 1.0) > 1e-12) return "q must sum to 1";
      return nullptr;
    }
    default:
      return "unknown problem kind";
  }
}

}  // namespace

extern "C" {

pdd_status pdd_create(pdd_ctx **out, const pdd_problem *problem, int device, void *cuda_stream) {
  g_create_error.clear();
  if (!out || !problem) return create_fail(PDD_EINVAL, "out or problem is NULL");
  *out = nullptr;
  if (const char *why = check_problem(problem)) return create_fail(PDD_EINVAL, why);
  if (device < 0) return create_fail(PDD_EINVAL, "device must be >= 0");
  int ndev = 0;
  const cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device >= ndev) {
    cudaGetLastError();
    return create_fail(PDD_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "no such device");
  }
  pdd_ctx *ctx = new (std::nothrow) pdd_ctx();
  if (!ctx) return create_fail(PDD_ENOMEM, "host allocation of the context failed");
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->prob = *problem;
  ctx->params.assign(problem->params, problem->params + problem->n_params);
  ctx->prob.params = ctx->params.data();
  ctx->mc.n_params = problem->n_params;
  for (int i = 0; i < problem->n_params; ++i) {
    ctx->mc.prm[i] = problem->params[i];
    ctx->mc.prmf[i] = static_cast<float>(problem->params[i]);
  }
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    const cudaError_t e2 = cudaGetLastError();
    delete ctx;
    return create_fail(PDD_ECUDA, cudaGetErrorString(e2));
  }
  *out = ctx;
  return PDD_OK;
}

pdd_status pdd_set_stream(pdd_ctx *ctx, void *cuda_stream) {
  if (!ctx) return PDD_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return PDD_OK;
}

pdd_status pdd_set_tuning(pdd_ctx *ctx, int blocks_per_sm, int64_t wave_max_paths) {
  if (!ctx || blocks_per_sm < 0 || blocks_per_sm > 64 || wave_max_paths < 0) return PDD_EINVAL;
  ctx->path_blocks_per_sm = blocks_per_sm;
  ctx->wave_max_paths = wave_max_paths > 0 ? static_cast<uint64_t>(wave_max_paths) : (1ull << 29);
  return PDD_OK;
}

pdd_status pdd_interface_solve(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                               const pdd_mc_params *mc, double *d_mean, double *d_se,
                               int64_t *d_npaths, pdd_diag *diag) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::interface_solve_impl(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths, diag);
}

pdd_status pdd_branching_solve(pdd_ctx *ctx, const double *d_nodes_xt, int64_t n,
                               const pdd_branch_params *bp, double *d_mean, double *d_se,
                               int64_t *d_nkept, pdd_diag *diag) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  if (bp && bp->reserved != 0) return fail(ctx, PDD_EINVAL, "reserved must be 0");
  return pdd::branching_solve_impl(ctx, d_nodes_xt, n, bp, d_mean, d_se, d_nkept, diag);
}

pdd_status pdd_subdomain_solve(pdd_ctx *ctx, const pdd_subdomain *sd, const double *d_iface_s,
                               const double *d_iface_vals, int64_t m, double *d_u,
                               int64_t *iters, double *resid) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::subdomain_solve_impl(ctx, sd, d_iface_s, d_iface_vals, m, d_u, iters, resid);
}

pdd_status pdd_subdomain_solve_batch(pdd_ctx *ctx, const pdd_subdomain *sds, int32_t n_boxes,
                                     const double *d_face, int64_t m, double *d_u,
                                     int64_t *iters, double *resid, int64_t *iters_each,
                                     double *resid_each) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::subdomain_solve3d_batch_impl(ctx, sds, n_boxes, d_face, m, d_u, iters, resid,
                                           iters_each, resid_each);
}

pdd_status pdd_interface_grad(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                              const pdd_mc_params *mc, const double *d_grad_out, double *d_jac,
                              double *d_jac_se, double *d_dtheta, double *d_dphi,
                              pdd_diag *diag) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::interface_grad_impl(ctx, d_nodes, n, mc, d_grad_out, d_jac, d_jac_se, d_dtheta,
                                  d_dphi, diag);
}

pdd_status pdd_set_params(pdd_ctx *ctx, const double *params, int32_t n_params) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  if (n_params != ctx->prob.n_params) return fail(ctx, PDD_EINVAL, "n_params differs");
  if (n_params > 0 && !params) return fail(ctx, PDD_EINVAL, "params is NULL");
  pdd_problem p = ctx->prob;
  p.params = params;
  if (const char *why = check_problem(&p)) return fail(ctx, PDD_EINVAL, "%s", why);
  ctx->params.assign(params, params + n_params);
  ctx->prob.params = ctx->params.data();
  for (int i = 0; i < n_params; ++i) {
    ctx->mc.prm[i] = params[i];
    ctx->mc.prmf[i] = static_cast<float>(params[i]);
  }
  return PDD_OK;
}

pdd_status pdd_batch_solve(pdd_ctx *ctx, const pdd_problem *problems, int32_t n_problems,
                           const pdd_batch_nodes *nodes, const pdd_batch_params *bp,
                           double *d_mean, double *d_se, int64_t *d_npaths, int32_t use_graph,
                           pdd_diag *diag) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::batch_solve_impl(ctx, problems, n_problems, nodes, bp, d_mean, d_se, d_npaths,
                               use_graph, diag);
}

pdd_status pdd_interface_solve_naive(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                     const pdd_mc_params *mc, double *d_mean, double *d_se,
                                     int64_t *d_npaths) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::interface_solve_naive_impl(ctx, d_nodes, n, mc, d_mean, d_se, d_npaths);
}

pdd_status pdd_autotune(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_mc_params *mc,
                        double *d_scratch_out, int32_t repeats, int32_t *best_blocks_per_sm,
                        double *best_ms) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::autotune_impl(ctx, d_nodes, n, mc, d_scratch_out, repeats, best_blocks_per_sm,
                            best_ms);
}

pdd_status pdd_autotune_batch(pdd_ctx *ctx, const pdd_problem *problems, int32_t n_problems,
                              const pdd_batch_nodes *nodes, const pdd_batch_params *bp,
                              double *d_scratch_out, int32_t repeats, int32_t *best_chunk,
                              double *best_ms) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::autotune_batch_impl(ctx, problems, n_problems, nodes, bp, d_scratch_out, repeats,
                                  best_chunk, best_ms);
}

pdd_status pdd_wos_solve(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_wos_params *wp,
                         double *d_mean, double *d_se, int64_t *d_npaths, pdd_diag *diag) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  if (wp && wp->reserved != 0) return fail(ctx, PDD_EINVAL, "reserved must be 0");
  return pdd::wos_solve_impl(ctx, d_nodes, n, wp, d_mean, d_se, d_npaths, diag);
}

pdd_status pdd_branching_grid_solve(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                    const double *h_times, int32_t m,
                                    const pdd_grid_branch_params *bp, double *d_mean,
                                    double *d_se, int64_t *d_nkept, pdd_diag *diag) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::branching_grid_solve_impl(ctx, d_nodes, n, h_times, m, bp, d_mean, d_se, d_nkept,
                                        diag);
}

pdd_status pdd_mlmc_level(pdd_ctx *ctx, const double *d_nodes, int64_t n, const pdd_mlmc_params *mp,
                          double *d_mean, double *d_var, double *d_fine_mean, double *d_coarse_mean,
                          pdd_diag *diag) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::mlmc_level_impl(ctx, d_nodes, n, mp, d_mean, d_var, d_fine_mean, d_coarse_mean, diag);
}

pdd_status pdd_interface_interp(pdd_ctx *ctx, int32_t n_planes, const int32_t *axis,
                                const double *pos, const int64_t *node_count,
                                const double *d_nodes, const double *d_vals, int32_t n_bnd,
                                const int64_t *query_count, const double *d_query,
                                double *d_out) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::interface_interp_impl(ctx, n_planes, axis, pos, node_count, d_nodes, d_vals, n_bnd,
                                    query_count, d_query, d_out);
}

pdd_status pdd_mlmc_solve(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                          const pdd_mlmc_params *mp, int32_t n_levels,
                          const int64_t *n_per_level, double *d_mean, double *d_se,
                          double *d_level_mean, double *d_level_var, pdd_diag *diag) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::mlmc_solve_impl(ctx, d_nodes, n, mp, n_levels, n_per_level, d_mean, d_se,
                              d_level_mean, d_level_var, diag);
}

pdd_status pdd_profile(pdd_ctx *ctx, int enable) {
  if (!ctx) return PDD_EINVAL;
  ctx->profiling = enable != 0;
  ctx->prof_used = 0;
  return PDD_OK;
}

pdd_status pdd_profile_read(pdd_ctx *ctx, double *kernel_ms, int64_t *launches) {
  if (!ctx || !kernel_ms || !launches) return PDD_EINVAL;
  *kernel_ms = 0.0;
  *launches = 0;
  cudaSetDevice(ctx->device);
  PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  for (size_t k = 0; k < ctx->prof_used; ++k) {
    float ms = 0.0f;
    PDD_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->prof_events[k].first,
                                           ctx->prof_events[k].second));
    *kernel_ms += ms;
  }
  *launches = static_cast<int64_t>(ctx->prof_used);
  ctx->prof_used = 0;
  return PDD_OK;
}

pdd_status pdd_normals(pdd_ctx *ctx, uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3,
                       int64_t n_pairs, float *d_z, float *d_u) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::normals_impl(ctx, seed, c1, c2, c3, n_pairs, d_z, d_u);
}

pdd_status pdd_philox_stream(pdd_ctx *ctx, uint64_t seed, uint32_t j0, uint32_t c1,
                             uint32_t c2, uint32_t c3, int64_t n_blocks, uint32_t *d_out) {
  if (!ctx) return PDD_EINVAL;
  ctx->last_error.clear();
  const TraceRange trace(__func__);
  return pdd::philox_stream_impl(ctx, seed, j0, c1, c2, c3, n_blocks, d_out);
}

void pdd_destroy(pdd_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
  for (int k = 0; k < 3; ++k) {
    if (ctx->batch_side[k]) cudaStreamDestroy(ctx->batch_side[k]);
    if (ctx->batch_join[k]) cudaEventDestroy(ctx->batch_join[k]);
  }
  if (ctx->batch_fork) cudaEventDestroy(ctx->batch_fork);
  for (auto &e : ctx->prof_events) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  cudaGetLastError();
  delete ctx;
}

const char *pdd_status_string(pdd_status s) {
  switch (s) {
    case PDD_OK: return "ok";
    case PDD_EINVAL: return "invalid argument";
    case PDD_ENOMEM: return "device allocation failed";
    case PDD_ECUDA: return "CUDA runtime error";
    case PDD_ETIMEOUT: return "bounded device loop ran out of iterations";
    case PDD_ECAP: return "some paths or trees were capped (results valid, counted)";
    default: return "unknown status";
  }
}

const char *pdd_last_error(const pdd_ctx *ctx) {
  return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

}  // extern "C"
