// static_solve.cu -- pdd_interface_solve_static: the interface solve for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: allocators that own the whole
// device pool, real-time or embedded loops where allocation latency and
// failure are unacceptable, or plug-in hosts that only hand out pre-allocated
// buffers.  This entry point runs the same path kernel and per-node
// finalisation as pdd_interface_solve, but its scratch (counters and the
// per-node exact sums) lives in a file-scope __device__ array of fixed size
// instead of context-owned memory, and it needs no context.  It calls no
// cudaMalloc, cudaFree or allocating library routine.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ctx.hpp"
#include "path_kernel.cuh"

namespace pdd {
namespace {

// 8 MiB on every GPU that loads the library, held until process exit:
// 256 bytes of counters and 112 bytes of exact sums per node.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;
constexpr int64_t kStaticMaxNodes = 65536;
constexpr size_t kStaticFixOff = 256;
static_assert(kStaticFixOff + kStaticMaxNodes * sizeof(NodeFix) <= kStaticScratchBytes,
              "static scratch too small for its node limit");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
bool g_loaded[kMaxDevices] = {};

// Load every kernel this entry point can launch (module loading may be lazy),
// once per device, so that no later call has to load one.
cudaError_t load_kernels() {
  cudaFuncAttributes fa;
  const void *kernels[] = {
      reinterpret_cast<const void *>(path_kernel<LaplaceExpCos, Box<2>, float>),
      reinterpret_cast<const void *>(path_kernel<LaplaceExpCos, Box<2>, double>),
      reinterpret_cast<const void *>(path_kernel<EllipticManufactured, Box<3>, float>),
      reinterpret_cast<const void *>(path_kernel<EllipticManufactured, Box<3>, double>),
      reinterpret_cast<const void *>(path_kernel<PoissonFourier, Box<2>, float>),
      reinterpret_cast<const void *>(path_kernel<PoissonFourier, Box<2>, double>),
      reinterpret_cast<const void *>(fix_finalize_kernel)};
  for (const void *k : kernels) {
    const cudaError_t e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Device address of the static scratch on the current device.  The host-side
// name g_static_scratch is only a stand-in; the address comes from the
// runtime, looked up on every call (no allocation), so a module reloaded
// after a device reset is never reached through a stale pointer.  The first
// call on a device also loads the kernels.
cudaError_t scratch_address(int device, void **out) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_loaded[device]) {
      const cudaError_t e = load_kernels();
      if (e != cudaSuccess) return e;
      g_loaded[device] = true;
    }
  }
  return cudaGetSymbolAddress(out, g_static_scratch);
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
  auto *counters = reinterpret_cast<unsigned long long *>(base);
  auto *fix = reinterpret_cast<NodeFix *>(base + kStaticFixOff);
  // the array keeps the previous call's contents: clear what must start at 0
  if (cudaMemsetAsync(base, 0, kStaticFixOff + static_cast<size_t>(n) * sizeof(NodeFix), stream) !=
      cudaSuccess)
    return PDD_ECUDA;

  PathArgs a;
  std::memset(&a, 0, sizeof a);
  a.nodes = d_nodes;
  a.n_paths = N;
  a.path_offset = static_cast<uint64_t>(mc->path_offset);
  a.node_offset = static_cast<uint32_t>(mc->node_offset);
  a.cursor = counters + 4;
  a.counters = counters;
  a.fix = fix;
  a.begin = 0;
  a.end = total;
  a.rk = make_round_keys(mc->seed);
  const double sig = prob->sigma, dt = mc->dt;
  const double c_kill = constant_kill(prob->kind);
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
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kPathBlockOf<R>, 0) != cudaSuccess ||
      cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return PDD_ECUDA;
  uint64_t grid = static_cast<uint64_t>(std::max(bps, 1)) * static_cast<uint64_t>(num_sms);
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (total + kPathBlockOf<R> - 1) / kPathBlockOf<R>));
  kern<<<static_cast<unsigned>(grid), kPathBlockOf<R>, 0, stream>>>(a);
  fix_finalize_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(
      fix, n, d_mean, d_se, d_npaths, nullptr);
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
  if (mc->node_offset < 0 || mc->node_offset + n > (int64_t(1) << 32)) return PDD_EINVAL;
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
