// static_solve.cu -- pdd_interface_solve_static: the interface solve for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA
// graph capture that forbids allocation, allocators that own the whole device
// pool, real-time or embedded loops where allocation latency and failure are
// unacceptable, or plug-in hosts that only hand out pre-allocated buffers.
// This entry point runs the same path kernel and per-node reduction as
// pdd_interface_solve, but its scratch (counters, per-node running sums, one
// wave of per-path scores) lives in a file-scope __device__ array of fixed
// size instead of context-owned memory, and it needs no context.  It calls no
// cudaMalloc, cudaFree or allocating library routine.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ctx.hpp"
#include "path_kernel.cuh"
#include "reduce.cuh"

namespace pdd {
namespace {

// 32 MiB on every GPU that loads the library, held until process exit.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int64_t kStaticMaxNodes = 65536;
constexpr size_t kStaticAccOff = 256;
constexpr size_t kStaticScoreOff = kStaticAccOff + kStaticMaxNodes * sizeof(NodeAcc);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch on `device` (current).  The host-side
// name g_static_scratch is only a stand-in; the address must come from the
// runtime, once per device.
cudaError_t scratch_address(int device, void **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

bool supported(const pdd_problem *p) {
  if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return false;
  if (p->n_params < 0 || p->n_params > kMaxParams || (p->n_params > 0 && !p->params)) return false;
  for (int i = 0; i < p->n_params; ++i)
    if (!std::isfinite(p->params[i])) return false;
  switch (p->kind) {
    // reflecting faces ([mask, phi] with mask != 0) have their own kernel
    case PDD_PROB_LAPLACE_EXPCOS:
      return p->dim == 2 && p->geometry == PDD_GEOM_UNIT_SQUARE &&
             (p->n_params == 0 || p->params[0] == 0.0);
    case PDD_PROB_ELLIPTIC_MANUFACTURED:
      return p->dim == 3 && p->geometry == PDD_GEOM_UNIT_CUBE &&
             (p->n_params == 0 || p->params[0] == 0.0);
    case PDD_PROB_POISSON_FOURIER:
      return p->dim == 2 && p->geometry == PDD_GEOM_UNIT_SQUARE && p->n_params >= 80;
    default: return false;
  }
}

template <class Model, class Geom, typename R>
pdd_status run_static(char *base, int device, cudaStream_t stream, const pdd_problem *prob,
                      const double *d_nodes, int64_t n, const pdd_mc_params *mc, double *d_mean,
                      double *d_se, int64_t *d_npaths) {
  const uint64_t N = static_cast<uint64_t>(mc->n_paths);
  const uint64_t total = static_cast<uint64_t>(n) * N;
  const uint64_t wave = std::min<uint64_t>(total, (kStaticScratchBytes - kStaticScoreOff) / sizeof(R));
  auto *counters = reinterpret_cast<unsigned long long *>(base);
  auto *cursor = counters + 4;
  auto *acc = reinterpret_cast<NodeAcc *>(base + kStaticAccOff);
  R *score = reinterpret_cast<R *>(base + kStaticScoreOff);
  // the array keeps the previous call's contents: clear what must start at 0
  if (cudaMemsetAsync(base, 0, kStaticAccOff + static_cast<size_t>(n) * sizeof(NodeAcc), stream) !=
      cudaSuccess)
    return PDD_ECUDA;

  PathArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes = d_nodes;
  a.n_paths = N;
  a.path_offset = static_cast<uint64_t>(mc->path_offset);
  a.cursor = cursor;
  a.counters = counters;
  a.score = score;
  a.rk = make_round_keys(mc->seed);
  const double sig = prob->sigma, dt = mc->dt;
  const double c_kill = prob->kind == PDD_PROB_ELLIPTIC_MANUFACTURED ? -1.0 : 0.0;
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
  a.mc.n_params = prob->n_params;
  for (int i = 0; i < prob->n_params; ++i) {
    a.mc.prm[i] = prob->params[i];
    a.mc.prmf[i] = static_cast<float>(prob->params[i]);
  }

  auto kern = path_kernel<Model, Geom, R>;
  int bps = 0, num_sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kPathBlock, 0) != cudaSuccess ||
      cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return PDD_ECUDA;
  uint64_t grid = static_cast<uint64_t>(std::max(bps, 1)) * static_cast<uint64_t>(num_sms);
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (wave + kPathBlock - 1) / kPathBlock));
  for (uint64_t b0 = 0; b0 < total; b0 += wave) {
    const uint64_t b1 = std::min(total, b0 + wave);
    if (b0 > 0 && cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), stream) != cudaSuccess)
      return PDD_ECUDA;
    a.begin = b0;
    a.end = b1;
    kern<<<static_cast<unsigned>(grid), kPathBlock, 0, stream>>>(a);
    const uint64_t node_lo = b0 / N, node_hi = (b1 - 1) / N;
    reduce_wave_kernel<R><<<static_cast<unsigned>(node_hi - node_lo + 1), kReduceBlock, 0, stream>>>(
        score, b0, b1, N, node_lo, acc);
  }
  finalize_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(acc, n, d_mean, d_se,
                                                                           d_npaths);
  return cudaGetLastError() == cudaSuccess ? PDD_OK : PDD_ECUDA;
}

template <class Model, class Geom>
pdd_status run_static_prec(char *base, int device, cudaStream_t stream, const pdd_problem *prob,
                           const double *d_nodes, int64_t n, const pdd_mc_params *mc,
                           double *d_mean, double *d_se, int64_t *d_npaths) {
  if (mc->precision == PDD_FP64)
    return run_static<Model, Geom, double>(base, device, stream, prob, d_nodes, n, mc, d_mean,
                                           d_se, d_npaths);
  return run_static<Model, Geom, float>(base, device, stream, prob, d_nodes, n, mc, d_mean, d_se,
                                        d_npaths);
}

}  // namespace
}  // namespace pdd

extern "C" pdd_status pdd_interface_solve_static(const pdd_problem *problem, int device,
                                                 void *cuda_stream, const double *d_nodes,
                                                 int64_t n, const pdd_mc_params *mc,
                                                 double *d_mean, double *d_se,
                                                 int64_t *d_npaths) {
  using namespace pdd;
  if (!problem || !mc || !supported(problem)) return PDD_EINVAL;
  if (n < 0 || n > kStaticMaxNodes) return PDD_EINVAL;
  if (mc->n_paths < 1 || mc->path_offset < 0 ||
      mc->path_offset + mc->n_paths > (int64_t(1) << 32))
    return PDD_EINVAL;
  if (!(mc->dt > 0.0) || !std::isfinite(mc->dt) ||
      problem->sigma * problem->sigma * mc->dt > 1.0 / 36.0)
    return PDD_EINVAL;
  if (mc->max_steps < 1 || mc->max_steps > 2147483647LL) return PDD_EINVAL;
  if (mc->precision != PDD_FP32 && mc->precision != PDD_FP64) return PDD_EINVAL;
  if (device < 0 || device >= kMaxDevices) return PDD_EINVAL;
  if (n == 0) return PDD_OK;
  if (!d_nodes || !d_mean || !d_se) return PDD_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return PDD_ECUDA;
  void *addr = nullptr;
  if (scratch_address(device, &addr) != cudaSuccess) {
    cudaGetLastError();
    return PDD_ECUDA;
  }
  char *base = static_cast<char *>(addr);
  auto stream = static_cast<cudaStream_t>(cuda_stream);
  switch (problem->kind) {
    case PDD_PROB_LAPLACE_EXPCOS:
      return run_static_prec<LaplaceExpCos, Box<2>>(base, device, stream, problem, d_nodes, n, mc,
                                                     d_mean, d_se, d_npaths);
    case PDD_PROB_ELLIPTIC_MANUFACTURED:
      return run_static_prec<EllipticManufactured, Box<3>>(base, device, stream, problem, d_nodes,
                                                            n, mc, d_mean, d_se, d_npaths);
    default:
      return run_static_prec<PoissonFourier, Box<2>>(base, device, stream, problem, d_nodes, n,
                                                      mc, d_mean, d_se, d_npaths);
  }
}
