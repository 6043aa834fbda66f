// stencil.cu -- stage two of PDD (Sec. 2.1, Fig. 2.2): the interface
// interpolator and the subdomain solver for the Laplace problem (Eq. 1.1).
//
// 1. spline_kernel: a cubic spline with not-a-knot end conditions through the
//    interface end points (values of g, which they lie on) and the Monte Carlo
//    node values (one thread; tridiagonal after eliminating the not-a-knot
//    rows).
// 2. fill_kernel: Dirichlet data on the grid boundary -- g on the physical
//    sides, the spline on the interface side -- and a zero interior.
// 3. cg_kernel / cg_mixed_kernel / jacobi_kernel: the 5-point system
//      (u[i+1,j] - 2u + u[i-1,j]) / hx^2 + (u[i,j+1] - 2u + u[i,j-1]) / hy^2 = 0
//    by conjugate gradients in FP64 or as FP32 CG inside FP64 iterative
//    refinement (one CTA, vectors L2-resident, fixed-order block reductions),
//    or Jacobi sweeps, all bounded by max_iter; or directly by discrete sine
//    transforms (dst.cu).
#include <cooperative_groups.h>

#include <cmath>
#include <cstring>

#include "ctx.hpp"

namespace pdd {

// Direct solve by discrete sine transforms (dst.cu).
size_t dst_scratch_bytes(int nx, int ny);
pdd_status dst_solve(pdd_ctx *ctx, double *d_u, int nx, int ny, double hx, double hy, char *work,
                     int64_t *it_d, double *res_d);

constexpr int kStencilBlock = 1024;

// ---- spline ---------------------------------------------------------------
// Knots s[0..K] (increasing), values y[0..K], second derivatives M[0..K].
// Interior rows: h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1}
//                = 6 ((y_{i+1} - y_i)/h_i - (y_i - y_{i-1})/h_{i-1}),
// not-a-knot:    h_1 M_0 - (h_0 + h_1) M_1 + h_0 M_2 = 0 and the mirror row,
// which are used to eliminate M_0 and M_K; Thomas algorithm on M_1..M_{K-1}.
__global__ void spline_kernel(const double *s, const double *y, int K, double *M, double *work) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double *a = work, *b = work + (K + 1), *c = work + 2 * (K + 1), *d = work + 3 * (K + 1);
  for (int i = 1; i < K; ++i) {
    const double h0 = s[i] - s[i - 1], h1 = s[i + 1] - s[i];
    a[i] = h0;
    b[i] = 2.0 * (h0 + h1);
    c[i] = h1;
    d[i] = 6.0 * ((y[i + 1] - y[i]) / h1 - (y[i] - y[i - 1]) / h0);
  }
  const double h0 = s[1] - s[0], h1 = s[2] - s[1];
  const double hl = s[K] - s[K - 1], hm = s[K - 1] - s[K - 2];
  if (K == 3) {
    // rows 1 and 2 only; M0 = ((h0+h1) M1 - h0 M2)/h1, M3 = ((hm+hl) M2 - hl M1)/hm
    const double b1 = b[1] + a[1] * (h0 + h1) / h1, c1 = c[1] - a[1] * h0 / h1;
    const double a2 = a[2] - c[2] * hl / hm, b2 = b[2] + c[2] * (hm + hl) / hm;
    const double det = b1 * b2 - c1 * a2;
    M[1] = (d[1] * b2 - c1 * d[2]) / det;
    M[2] = (b1 * d[2] - a2 * d[1]) / det;
  } else {
    b[1] += a[1] * (h0 + h1) / h1;
    c[1] -= a[1] * h0 / h1;
    a[1] = 0.0;
    b[K - 1] += c[K - 1] * (hm + hl) / hm;
    a[K - 1] -= c[K - 1] * hl / hm;
    c[K - 1] = 0.0;
    for (int i = 2; i < K; ++i) {
      const double w = a[i] / b[i - 1];
      b[i] -= w * c[i - 1];
      d[i] -= w * d[i - 1];
    }
    M[K - 1] = d[K - 1] / b[K - 1];
    for (int i = K - 2; i >= 1; --i) M[i] = (d[i] - c[i] * M[i + 1]) / b[i];
  }
  M[0] = ((h0 + h1) * M[1] - h0 * M[2]) / h1;
  M[K] = ((hm + hl) * M[K - 1] - hl * M[K - 2]) / hm;
}

__device__ double spline_eval(const double *s, const double *y, const double *M, int K, double t) {
  int lo = 0, hi = K;
  while (hi - lo > 1) {  // s[lo] <= t < s[hi]
    const int mid = (lo + hi) >> 1;
    if (s[mid] <= t) lo = mid; else hi = mid;
  }
  const double h = s[lo + 1] - s[lo];
  const double A = s[lo + 1] - t, B = t - s[lo];
  return M[lo] * A * A * A / (6.0 * h) + M[lo + 1] * B * B * B / (6.0 * h) +
         (y[lo] / h - M[lo] * h / 6.0) * A + (y[lo + 1] / h - M[lo + 1] * h / 6.0) * B;
}

// Interface knots: s[0] and s[K] are the interface end points, where the data
// are g; s[1..K-1] are the node coordinates along the interface.
__global__ void knots_kernel(const double *node_s, const double *vals, int64_t m, double s_lo,
                             double s_hi, double fixed, int along_axis, double *s, double *y) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i > m + 1) return;
  if (i == 0 || i == m + 1) {
    const double t = i == 0 ? s_lo : s_hi;
    const double x = along_axis == 1 ? fixed : t, yy = along_axis == 1 ? t : fixed;
    s[i] = t;
    y[i] = exp(x) * cos(yy);  // g of the Laplace family, Eq. 1.1 data
  } else {
    s[i] = node_s[i - 1];
    y[i] = vals[i - 1];
  }
}

// Boundary data and zero interior on an [ny][nx] grid.
__global__ void fill_kernel(double *u, int nx, int ny, double x0, double y0, double hx,
                            double hy, int iface_axis, int iface_side, const double *s,
                            const double *y, const double *M, int K) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<int64_t>(nx) * ny) return;
  const int i = static_cast<int>(idx % nx), j = static_cast<int>(idx / nx);
  const bool bnd = i == 0 || j == 0 || i == nx - 1 || j == ny - 1;
  if (!bnd) {
    u[idx] = 0.0;
    return;
  }
  const double x = x0 + i * hx, yy = y0 + j * hy;
  bool on_iface;
  double t;
  if (iface_axis == 0) {
    on_iface = i == (iface_side ? nx - 1 : 0);
    t = yy;
  } else {
    on_iface = j == (iface_side ? ny - 1 : 0);
    t = x;
  }
  u[idx] = on_iface ? spline_eval(s, y, M, K, t) : exp(x) * cos(yy);
}

// ---- block reductions (fixed order) ---------------------------------------
__device__ double block_sum(double v, double *sh) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kStencilBlock / 32; ++w) t += sh[w];
    sh[32] = t;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

__device__ double block_max(double v, double *sh) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, m));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kStencilBlock / 32; ++w) t = fmax(t, sh[w]);
    sh[32] = t;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

// Grid position of a block-strided flat index k = threadIdx.x + t * blockDim,
// advanced without divisions (the 64-bit k / nx, k % nx of a plain loop cost
// more than the stencil arithmetic).
struct GridWalk {
  int k, i, j, di, dj, nx;
  __device__ __forceinline__ GridWalk(int nx_) : nx(nx_) {
    k = threadIdx.x;
    i = k % nx;
    j = k / nx;
    di = kStencilBlock % nx;
    dj = kStencilBlock / nx;
  }
  __device__ __forceinline__ void next() {
    k += kStencilBlock;
    i += di;
    j += dj;
    if (i >= nx) {
      i -= nx;
      ++j;
    }
  }
};

// FP32 block sum in a fixed tree (warp shuffles, then warp 0 over the 32
// warp partials), broadcast to every thread.
__device__ float block_sum_f(float v, float *sh) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    float t = sh[lane];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(kFull, t, m);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  const float r = sh[32];
  __syncthreads();
  return r;
}

// Conjugate gradients on the interior unknowns of A = -Lap_h (SPD).  With the
// interior initialised to 0, r0 = Lap_h(u) over the full grid = b.
__global__ void __launch_bounds__(kStencilBlock)
cg_kernel(double *u, int nx, int ny, double ihx2, double ihy2, double *r, double *p, double *q,
          int64_t max_iter, double tol, int64_t *iters_out, double *resid_out) {
  __shared__ double sh[33];
  const int N = nx * ny;
  const double diag = 2.0 * ihx2 + 2.0 * ihy2;
  double rr_loc = 0.0;
  for (GridWalk w(nx); w.k < N; w.next()) {
    const int k = w.k, i = w.i, j = w.j;
    double v = 0.0;
    if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1)
      v = ihx2 * (u[k - 1] + u[k + 1]) + ihy2 * (u[k - nx] + u[k + nx]) - diag * u[k];
    r[k] = v;
    p[k] = v;
    rr_loc += v * v;
  }
  double rr = block_sum(rr_loc, sh);
  const double bnorm = sqrt(rr);
  int64_t it = 0;
  double res = bnorm > 0.0 ? 1.0 : 0.0;
  while (it < max_iter && bnorm > 0.0 && sqrt(rr) > tol * bnorm) {
    double pq_loc = 0.0;
    for (GridWalk w(nx); w.k < N; w.next()) {
      const int k = w.k, i = w.i, j = w.j;
      double v = 0.0;
      if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) {
        const double pw = i > 1 ? p[k - 1] : 0.0, pe = i < nx - 2 ? p[k + 1] : 0.0;
        const double ps = j > 1 ? p[k - nx] : 0.0, pn = j < ny - 2 ? p[k + nx] : 0.0;
        v = diag * p[k] - ihx2 * (pw + pe) - ihy2 * (ps + pn);
      }
      q[k] = v;
      pq_loc += p[k] * v;
    }
    const double pq = block_sum(pq_loc, sh);
    const double alpha = rr / pq;
    double rn_loc = 0.0;
    for (GridWalk w(nx); w.k < N; w.next()) {
      const int k = w.k, i = w.i, j = w.j;
      if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) {
        u[k] += alpha * p[k];
        const double rk = r[k] - alpha * q[k];
        r[k] = rk;
        rn_loc += rk * rk;
      }
    }
    const double rn = block_sum(rn_loc, sh);
    const double beta = rn / rr;
    rr = rn;
    for (int k = threadIdx.x; k < N; k += kStencilBlock) p[k] = r[k] + beta * p[k];
    __syncthreads();
    ++it;
    res = sqrt(rr) / bnorm;
  }
  if (threadIdx.x == 0) {
    *iters_out = it;
    *resid_out = res;
  }
}

// The same conjugate gradients on a thread-block cluster of kCgCluster
// blocks (FP64 arithmetic runs at a per-SM rate, and one block held the
// solve to one SM): block b owns the grid rows [b ny / C, (b + 1) ny / C).
// Each iteration: the block's part of q = A p (reading its neighbours' rows
// of p through L2), the cluster-wide p.q (every block sums the C block
// partials in rank order, read from each other's shared memory, so all
// blocks take the same alpha), the update of u and r, the cluster-wide r.r,
// and p = r + beta p.  Three cluster barriers per iteration: before q = A p
// (p complete), after each partial sum.
constexpr int kCgCluster = 8;

__global__ void __cluster_dims__(kCgCluster, 1, 1) __launch_bounds__(kStencilBlock)
cg_cluster_kernel(double *u, int nx, int ny, double ihx2, double ihy2, double *r, double *p,
                  double *q, int64_t max_iter, double tol, int64_t *iters_out, double *resid_out) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ double sh[33];
  __shared__ double slot_pq, slot_rr;
  const int rank = static_cast<int>(cluster.block_rank());
  const int j0 = static_cast<int>(static_cast<int64_t>(rank) * ny / kCgCluster);
  const int j1 = static_cast<int>(static_cast<int64_t>(rank + 1) * ny / kCgCluster);
  const int k0 = j0 * nx, k1 = j1 * nx;
  const double diag = 2.0 * ihx2 + 2.0 * ihy2;
  auto cluster_sum = [&](double *slot, double v_block) -> double {
    if (threadIdx.x == 0) *slot = v_block;
    cluster.sync();
    double t = 0.0;
    for (int b = 0; b < kCgCluster; ++b) t += *cluster.map_shared_rank(slot, b);
    return t;
  };
  double rr_loc = 0.0;
  for (int k = k0 + threadIdx.x; k < k1; k += kStencilBlock) {
    const int i = k % nx, j = k / nx;
    double v = 0.0;
    if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1)
      v = ihx2 * (u[k - 1] + u[k + 1]) + ihy2 * (u[k - nx] + u[k + nx]) - diag * u[k];
    r[k] = v;
    p[k] = v;
    rr_loc += v * v;
  }
  double rr = cluster_sum(&slot_rr, block_sum(rr_loc, sh));
  const double bnorm = sqrt(rr);
  int64_t it = 0;
  double res = bnorm > 0.0 ? 1.0 : 0.0;
  while (it < max_iter && bnorm > 0.0 && sqrt(rr) > tol * bnorm) {
    cluster.sync();  // p complete (and every block done reading slot_rr)
    double pq_loc = 0.0;
    for (int k = k0 + threadIdx.x; k < k1; k += kStencilBlock) {
      const int i = k % nx, j = k / nx;
      double v = 0.0;
      const double pk = __ldcg(p + k);
      if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) {
        const double pw = i > 1 ? __ldcg(p + k - 1) : 0.0, pe = i < nx - 2 ? __ldcg(p + k + 1) : 0.0;
        const double ps = j > 1 ? __ldcg(p + k - nx) : 0.0, pn = j < ny - 2 ? __ldcg(p + k + nx) : 0.0;
        v = diag * pk - ihx2 * (pw + pe) - ihy2 * (ps + pn);
      }
      q[k] = v;
      pq_loc += pk * v;
    }
    const double pq = cluster_sum(&slot_pq, block_sum(pq_loc, sh));
    const double alpha = rr / pq;
    double rn_loc = 0.0;
    for (int k = k0 + threadIdx.x; k < k1; k += kStencilBlock) {
      const int i = k % nx, j = k / nx;
      if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) {
        u[k] += alpha * __ldcg(p + k);
        const double rk = r[k] - alpha * q[k];
        r[k] = rk;
        rn_loc += rk * rk;
      }
    }
    const double rn = cluster_sum(&slot_rr, block_sum(rn_loc, sh));
    const double beta = rn / rr;
    rr = rn;
    for (int k = k0 + threadIdx.x; k < k1; k += kStencilBlock) p[k] = r[k] + beta * __ldcg(p + k);
    ++it;
    res = sqrt(rr) / bnorm;
  }
  cluster.sync();  // no block leaves while another may read its slots
  if (rank == 0 && threadIdx.x == 0) {
    *iters_out = it;
    *resid_out = res;
  }
}

// Mixed-precision conjugate gradients (iterative refinement): the FP64
// residual r = b - A u is formed, scaled to unit norm and rounded to FP32;
// CG in FP32 (vectors, arithmetic and fixed-tree block sums) solves A e = r
// to a relative residual of 1e-4, or just below what the stopping rule still
// needs; u += ||r|| e in FP64; repeat until the FP64 residual meets the
// stopping rule.  FP64 runs at 1/64 of the FP32 rate on this part and one
// CTA owns the solve, so the inner iterations are what the FP32 pipe makes
// cheap; the answer is the FP64 solution to the same tolerance.  rf/ef
// share v0 and pf/qf share v1 (two FP32 vectors per FP64-sized buffer), the
// FP64 residual is r64.
template <bool kSmem>
__global__ void __launch_bounds__(kStencilBlock)
cg_mixed_kernel(double *u, int nx, int ny, double ihx2, double ihy2, double *v0, double *v1,
                double *r64, int64_t max_iter, double tol, int64_t *iters_out, double *resid_out) {
  __shared__ double sh[33];
  __shared__ float shf[33];
  extern __shared__ float dsm[];
  const int N = nx * ny;
  float *rf, *ef, *pf, *qf;
  if constexpr (kSmem) {  // the three FP32 vectors in shared memory; A p recomputed
    rf = dsm;
    pf = dsm + N;
    ef = dsm + 2 * N;
    qf = nullptr;
  } else {
    rf = reinterpret_cast<float *>(v0);
    ef = rf + N;
    pf = reinterpret_cast<float *>(v1);
    qf = pf + N;
  }
  const double diag = 2.0 * ihx2 + 2.0 * ihy2;
  const float diag_f = static_cast<float>(diag), ihx2_f = static_cast<float>(ihx2),
              ihy2_f = static_cast<float>(ihy2);
  // A p at an interior point (zero Dirichlet data for the correction)
  auto apply = [&](int k, int i, int j) -> float {
    const float pw = i > 1 ? pf[k - 1] : 0.f, pe = i < nx - 2 ? pf[k + 1] : 0.f;
    const float ps = j > 1 ? pf[k - nx] : 0.f, pn = j < ny - 2 ? pf[k + nx] : 0.f;
    return diag_f * pf[k] - ihx2_f * (pw + pe) - ihy2_f * (ps + pn);
  };
  constexpr float kInnerTol = 1e-4f;
  constexpr int kMaxOuter = 64;
  int64_t it = 0;
  double bnorm = 0.0, res = 0.0;
  for (int outer = 0; outer < kMaxOuter; ++outer) {
    // FP64 residual of the current iterate (interior unknowns)
    double rr_loc = 0.0;
    for (GridWalk w(nx); w.k < N; w.next()) {
      const int k = w.k, i = w.i, j = w.j;
      double v = 0.0;
      if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1)
        v = ihx2 * (u[k - 1] + u[k + 1]) + ihy2 * (u[k - nx] + u[k + nx]) - diag * u[k];
      r64[k] = v;
      rr_loc += v * v;
    }
    const double rnorm = sqrt(block_sum(rr_loc, sh));
    if (outer == 0) bnorm = rnorm;
    res = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    if (!(bnorm > 0.0) || res <= tol || it >= max_iter) break;
    // reduce the residual by 1e-4, or by just what the stopping rule needs
    const float need = static_cast<float>(0.5 * tol / res);
    const float tol_in = need > kInnerTol ? need : kInnerTol;
    const double sc = 1.0 / rnorm;
    float rr_f = 0.f;
    for (int k = threadIdx.x; k < N; k += kStencilBlock) {
      const float v = static_cast<float>(r64[k] * sc);
      rf[k] = v;
      pf[k] = v;
      ef[k] = 0.f;
      rr_f += v * v;
    }
    float rr = block_sum_f(rr_f, shf);
    const float stop = tol_in * tol_in * rr;
    while (it < max_iter && rr > stop) {
      float pq_f = 0.f;
      for (GridWalk w(nx); w.k < N; w.next()) {
        const int k = w.k, i = w.i, j = w.j;
        const float v = (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) ? apply(k, i, j) : 0.f;
        if constexpr (!kSmem) qf[k] = v;
        pq_f += pf[k] * v;
      }
      const float pq = block_sum_f(pq_f, shf);
      const float alpha = rr / pq;
      float rn_f = 0.f;
      for (GridWalk w(nx); w.k < N; w.next()) {
        const int k = w.k, i = w.i, j = w.j;
        float q;
        if constexpr (kSmem) q = (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) ? apply(k, i, j) : 0.f;
        else q = qf[k];
        ef[k] += alpha * pf[k];
        const float rk = rf[k] - alpha * q;
        rf[k] = rk;
        rn_f += rk * rk;
      }
      const float rn = block_sum_f(rn_f, shf);
      const float beta = rn / rr;
      rr = rn;
      for (int k = threadIdx.x; k < N; k += kStencilBlock) pf[k] = rf[k] + beta * pf[k];
      __syncthreads();
      ++it;
    }
    for (int k = threadIdx.x; k < N; k += kStencilBlock) u[k] += static_cast<double>(ef[k]) * rnorm;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *iters_out = it;
    *resid_out = res;
  }
}

// Jacobi sweeps u <- (ihx2 (W + E) + ihy2 (S + N)) / diag, ping-pong between
// u and tmp; stops when the largest update is below tol or after max_iter.
__global__ void __launch_bounds__(kStencilBlock)
jacobi_kernel(double *u, double *tmp, int nx, int ny, double ihx2, double ihy2, int64_t max_iter,
              double tol, int64_t *iters_out, double *resid_out) {
  __shared__ double sh[33];
  const int N = nx * ny;
  const double inv_diag = 1.0 / (2.0 * ihx2 + 2.0 * ihy2);
  for (int k = threadIdx.x; k < N; k += kStencilBlock) tmp[k] = u[k];
  __syncthreads();
  double *src = u, *dst = tmp;
  int64_t it = 0;
  double change = 0.0;
  while (it < max_iter) {
    double mx = 0.0;
    for (GridWalk w(nx); w.k < N; w.next()) {
      const int k = w.k, i = w.i, j = w.j;
      if (i > 0 && j > 0 && i < nx - 1 && j < ny - 1) {
        const double v = (ihx2 * (src[k - 1] + src[k + 1]) + ihy2 * (src[k - nx] + src[k + nx])) * inv_diag;
        mx = fmax(mx, fabs(v - src[k]));
        dst[k] = v;
      }
    }
    change = block_max(mx, sh);
    double *t = src;
    src = dst;
    dst = t;
    ++it;
    if (change < tol) break;
  }
  if (src != u)
    for (int k = threadIdx.x; k < N; k += kStencilBlock) u[k] = src[k];
  if (threadIdx.x == 0) {
    *iters_out = it;
    *resid_out = change;
  }
}

pdd_status subdomain_solve_impl(pdd_ctx *ctx, const pdd_subdomain *sd, const double *d_iface_s,
                                const double *d_iface_vals, int64_t m, double *d_u,
                                int64_t *iters, double *resid) {
  if (!sd || !d_u || !iters || !resid) return fail(ctx, PDD_EINVAL, "null argument");
  if (sd->n[2] > 1) return subdomain_solve3d_impl(ctx, sd, d_iface_vals, m, d_u, iters, resid);
  if (ctx->prob.kind != PDD_PROB_LAPLACE_EXPCOS)
    return fail(ctx, PDD_EINVAL, "the subdomain solver covers the Laplace family (Eq. 1.1)");
  const int nx = sd->n[0], ny = sd->n[1];
  if (nx < 3 || ny < 3 || sd->n[2] != 1) return fail(ctx, PDD_EINVAL, "grid must be 2-D, >= 3x3");
  if (static_cast<int64_t>(nx) * ny > (int64_t(1) << 26)) return fail(ctx, PDD_EINVAL, "grid too large");
  if (!(sd->hi[0] > sd->lo[0]) || !(sd->hi[1] > sd->lo[1])) return fail(ctx, PDD_EINVAL, "empty box");
  if (sd->lo[0] < 0.0 || sd->lo[1] < 0.0 || sd->hi[0] > 1.0 || sd->hi[1] > 1.0)
    return fail(ctx, PDD_EINVAL, "box must lie in the unit square");
  if (sd->iface_axis < 0 || sd->iface_axis > 1 || sd->iface_side < 0 || sd->iface_side > 1)
    return fail(ctx, PDD_EINVAL, "bad interface side");
  if (m < 2 || !d_iface_s || !d_iface_vals) return fail(ctx, PDD_EINVAL, "need >= 2 interface nodes");
  if (sd->max_iter < 0 || !(sd->tol >= 0.0)) return fail(ctx, PDD_EINVAL, "bad stopping rule");
  if (sd->method != PDD_STENCIL_CG && sd->method != PDD_STENCIL_JACOBI &&
      sd->method != PDD_STENCIL_CG_MIXED && sd->method != PDD_STENCIL_DST)
    return fail(ctx, PDD_EINVAL, "unknown method");
  if (sd->method == PDD_STENCIL_DST && (nx - 2 > 8192 || ny - 2 > 8192))
    return fail(ctx, PDD_EINVAL, "the sine-transform solve takes at most 8192 interior points per axis");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int K = static_cast<int>(m) + 1;
  const size_t npts = static_cast<size_t>(nx) * ny;
  const size_t knot_bytes = align_up(static_cast<size_t>(K + 1) * sizeof(double), 256);
  // scratch: s, y, M, work(4 x), then 3 grid vectors, then 2 result words
  const size_t off_s = 0, off_y = knot_bytes, off_M = 2 * knot_bytes, off_w = 3 * knot_bytes;
  const size_t off_v = off_w + 4 * knot_bytes;
  const size_t vec = align_up(npts * sizeof(double), 256);
  const size_t off_out = off_v + 3 * vec;
  const size_t off_dst = off_out + 256;
  const size_t dst_bytes = sd->method == PDD_STENCIL_DST ? dst_scratch_bytes(nx, ny) : 0;
  pdd_status st = ensure_scratch(ctx, off_dst + dst_bytes);
  if (st != PDD_OK) return st;
  char *base = static_cast<char *>(ctx->scratch);
  double *s = reinterpret_cast<double *>(base + off_s), *y = reinterpret_cast<double *>(base + off_y);
  double *M = reinterpret_cast<double *>(base + off_M), *w = reinterpret_cast<double *>(base + off_w);
  double *v0 = reinterpret_cast<double *>(base + off_v);
  double *v1 = reinterpret_cast<double *>(base + off_v + vec);
  double *v2 = reinterpret_cast<double *>(base + off_v + 2 * vec);
  auto *it_d = reinterpret_cast<int64_t *>(base + off_out);
  auto *res_d = reinterpret_cast<double *>(base + off_out + 8);

  const int ax = sd->iface_axis, along = 1 - ax;
  const double fixed = sd->iface_side ? sd->hi[ax] : sd->lo[ax];
  knots_kernel<<<static_cast<unsigned>((m + 2 + 255) / 256), 256, 0, ctx->stream>>>(
      d_iface_s, d_iface_vals, m, sd->lo[along], sd->hi[along], fixed, along, s, y);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  spline_kernel<<<1, 32, 0, ctx->stream>>>(s, y, K, M, w);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  const double hx = (sd->hi[0] - sd->lo[0]) / (nx - 1), hy = (sd->hi[1] - sd->lo[1]) / (ny - 1);
  fill_kernel<<<static_cast<unsigned>((npts + 255) / 256), 256, 0, ctx->stream>>>(
      d_u, nx, ny, sd->lo[0], sd->lo[1], hx, hy, ax, sd->iface_side, s, y, M, K);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  const double ihx2 = 1.0 / (hx * hx), ihy2 = 1.0 / (hy * hy);
  const auto ev = prof_slot(ctx);
  if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
  if (sd->method == PDD_STENCIL_DST) {
    st = dst_solve(ctx, d_u, nx, ny, hx, hy, base + off_dst, it_d, res_d);
    if (st != PDD_OK) return st;
  } else if (sd->method == PDD_STENCIL_CG) {
    // a cluster of kCgCluster blocks when every block gets at least one row
    if (ny >= kCgCluster)
      cg_cluster_kernel<<<kCgCluster, kStencilBlock, 0, ctx->stream>>>(
          d_u, nx, ny, ihx2, ihy2, v0, v1, v2, sd->max_iter, sd->tol, it_d, res_d);
    else
      cg_kernel<<<1, kStencilBlock, 0, ctx->stream>>>(d_u, nx, ny, ihx2, ihy2, v0, v1, v2,
                                                      sd->max_iter, sd->tol, it_d, res_d);
  }
  else if (sd->method == PDD_STENCIL_CG_MIXED) {
    // the three FP32 vectors in shared memory when they fit (129 x 129: 200 KB)
    const size_t smem = 3 * npts * sizeof(float);
    int max_smem = 0;
    PDD_CUDA_TRY(ctx, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                             ctx->device));
    if (smem + 1024 <= static_cast<size_t>(max_smem)) {
      PDD_CUDA_TRY(ctx, cudaFuncSetAttribute(cg_mixed_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem)));
      cg_mixed_kernel<true><<<1, kStencilBlock, smem, ctx->stream>>>(
          d_u, nx, ny, ihx2, ihy2, v0, v1, v2, sd->max_iter, sd->tol, it_d, res_d);
    } else {
      cg_mixed_kernel<false><<<1, kStencilBlock, 0, ctx->stream>>>(
          d_u, nx, ny, ihx2, ihy2, v0, v1, v2, sd->max_iter, sd->tol, it_d, res_d);
    }
  } else
    jacobi_kernel<<<1, kStencilBlock, 0, ctx->stream>>>(d_u, v0, nx, ny, ihx2, ihy2,
                                                        sd->max_iter, sd->tol, it_d, res_d);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
  int64_t h_it = 0;
  double h_res = 0.0;
  PDD_CUDA_TRY(ctx, cudaMemcpyAsync(&h_it, it_d, sizeof h_it, cudaMemcpyDeviceToHost, ctx->stream));
  PDD_CUDA_TRY(ctx, cudaMemcpyAsync(&h_res, res_d, sizeof h_res, cudaMemcpyDeviceToHost, ctx->stream));
  PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  *iters = h_it;
  *resid = h_res;
  if (sd->method == PDD_STENCIL_DST) return PDD_OK;  // direct: no stopping rule
  if (h_it >= sd->max_iter && !(h_res <= sd->tol))
    return fail(ctx, PDD_ETIMEOUT, "stopping rule not met after %lld iterations (%.3e)",
                static_cast<long long>(h_it), h_res);
  return PDD_OK;
}

}  // namespace pdd
