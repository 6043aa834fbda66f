// stage2_3d.cu -- stage two of PDD in three dimensions (Sec. 2.1, Fig. 2.2):
// the interface interpolation that turns Monte Carlo node values on the
// internal planes of the cube into Dirichlet data, and the independent
// subdomain solves of the elliptic problem
//   (1/2) sigma^2 Lap u + b . grad u + c u + f = 0   (Eq. 2.3 without time)
// by 7-point second differences and central first differences.
//
// Interpolation (pdd_interface_interp): per plane, a radial basis function
// interpolant with the cubic kernel |r|^3 and a linear polynomial term through
// the plane's nodes and n_bnd points per edge of the plane's perimeter, where
// the boundary data g are known.  The saddle-point system
//   [Phi P; P^T 0] [w; c] = [v; 0],  Phi_ij = |x_i - x_j|^3,  P_i = (1, s_i, t_i)
// is solved in FP64 by Gaussian elimination with partial pivoting, one block
// per plane (the planes of one call in one launch), then evaluated at the
// query points, one thread per point.
//
// Subdomain solve (pdd_subdomain_solve with a 3-D grid): defect correction
//   u <- u + P^{-1} (rhs - A u)
// with A the full operator (FP64 residual) and P its constant-coefficient part
// (1/2) sigma^2 Lap_h + c, which the three-dimensional discrete sine
// transform diagonalises on a box with Dirichlet data.  P^{-1} is applied in
// binary32 (three dense passes of the sine matrices, a division by the
// eigenvalues, three passes back); the drift is a small perturbation of P on
// a subdomain (|b| / |grad| against the Laplacian's scale), so the error
// contracts by roughly ten per iteration, down to the FP64 residual
// tolerance.  A plain Jacobi sweep is kept as the reference method.
#include <cooperative_groups.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.hpp"
#include "models.cuh"

namespace pdd {

// ---------------------------------------------------------------------------
// Interface interpolation on planes
// ---------------------------------------------------------------------------
constexpr int kRbfBlock = 1024;
constexpr int64_t kRbfMaxSystem = 6144;  // unknowns per plane (weights + 3)

struct RbfPlane {
  int64_t node0, m;      // this plane's nodes: [node0, node0 + m) of the call's list
  int64_t sys0;          // offset of its system (M x M matrix, then M right-hand side)
  int64_t pts0;          // offset of its 2-D points (M - 3 of them) and values
  int64_t q0, q;         // its query points
  int32_t axis, M;       // plane normal axis; system size
  double pos;
};

// The plane's two in-plane coordinates of a 3-D point.
__device__ __forceinline__ void plane_coords(int axis, const double *x, double &s, double &t) {
  s = x[axis == 0 ? 1 : 0];
  t = x[axis == 2 ? 1 : 2];
}

// Interpolation points of every plane: its nodes, then n_bnd points per edge
// of its perimeter (corners once) with the boundary data g.
template <class Model>
__global__ void rbf_points_kernel(const RbfPlane *planes, int32_t n_planes, const double *nodes,
                                  const double *vals, int32_t n_bnd, ModelConst mc, double *pts,
                                  double *pv) {
  const int p = blockIdx.y;
  if (p >= n_planes) return;
  const RbfPlane P = planes[p];
  const int64_t npt = P.M - 3;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < npt;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double s, t, v;
    if (i < P.m) {
      plane_coords(P.axis, nodes + 3 * (P.node0 + i), s, t);
      v = vals[P.node0 + i];
    } else {
      // perimeter of the unit square in (s, t): edge e, point k of n_bnd
      const int64_t b = i - P.m;
      const int e = static_cast<int>(b / n_bnd);
      const double u = static_cast<double>(b % n_bnd) / n_bnd;
      s = e == 0 ? u : (e == 1 ? 1.0 : (e == 2 ? 1.0 - u : 0.0));
      t = e == 0 ? 0.0 : (e == 1 ? u : (e == 2 ? 1.0 : 1.0 - u));
      double x[3];
      x[P.axis] = P.pos;
      x[P.axis == 0 ? 1 : 0] = s;
      x[P.axis == 2 ? 1 : 2] = t;
      v = Model::template g<double>(mc, x);
    }
    pts[2 * (P.pts0 + i)] = s;
    pts[2 * (P.pts0 + i) + 1] = t;
    pv[P.pts0 + i] = v;
  }
}

__global__ void rbf_assemble_kernel(const RbfPlane *planes, int32_t n_planes, const double *pts,
                                    const double *pv, double *sys) {
  const int p = blockIdx.y;
  if (p >= n_planes) return;
  const RbfPlane P = planes[p];
  const int64_t M = P.M, npt = M - 3;
  double *A = sys + P.sys0, *rhs = sys + P.sys0 + M * M;
  const double *xy = pts + 2 * P.pts0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < M * M;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / M, j = e % M;
    double a;
    if (i < npt && j < npt) {
      const double ds = xy[2 * i] - xy[2 * j], dt = xy[2 * i + 1] - xy[2 * j + 1];
      const double r2 = ds * ds + dt * dt;
      a = r2 * sqrt(r2);
    } else if (i < npt) {
      a = j == npt ? 1.0 : xy[2 * i + (j - npt - 1)];
    } else if (j < npt) {
      a = i == npt ? 1.0 : xy[2 * j + (i - npt - 1)];
    } else {
      a = 0.0;
    }
    A[e] = a;
    if (j == 0) rhs[i] = i < npt ? pv[P.pts0 + i] : 0.0;
  }
}

// Gaussian elimination with partial pivoting and back substitution, one
// thread-block cluster of kRbfCluster blocks per plane (the systems are
// dense FP64 and GB300's FP64 rate is per SM, so a plane's elimination is
// spread over several SMs).  Rows are not moved: block r of the cluster owns
// rows i = r (mod kRbfCluster) and keeps its rows' "already a pivot" flags;
// step k takes as pivot the unused row with the largest |A[i][k]| (lowest
// index on ties), every block reads that row, and each block eliminates
// column k from its own unused rows.  One cluster barrier per step: the
// blocks' pivot candidates sit in double-buffered shared slots read across
// the cluster, and a block only writes its own rows, which no other block
// reads before the next barrier (the pivot row is read after it).  Then the
// first block back-substitutes in pivot order.  On return rhs holds [w; c].
// A zero pivot sets *singular.
constexpr int kRbfCluster = 8;

__global__ void __cluster_dims__(kRbfCluster, 1, 1) __launch_bounds__(kRbfBlock)
rbf_solve_kernel(const RbfPlane *planes, int32_t n_planes, double *sys, int *singular) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int p = blockIdx.x / kRbfCluster;
  const int r = static_cast<int>(cluster.block_rank());
  if (p >= n_planes) return;  // whole clusters: every block of it returns
  const int64_t M = planes[p].M;
  double *A = sys + planes[p].sys0, *b = A + M * M;
  // dynamic shared memory: the pivot row (M doubles, with its right-hand
  // side last), then (first block) the solution and the pivot order, then
  // the used flags of this block's rows
  extern __shared__ double dsm[];
  double *rowk = dsm;                                   // M + 1
  double *x = rowk + M + 1;                             // M (block 0)
  int32_t *perm = reinterpret_cast<int32_t *>(x + M);  // M (block 0)
  unsigned char *used = reinterpret_cast<unsigned char *>(perm + M);  // M / kRbfCluster + 1
  __shared__ double cand_v[2];
  __shared__ int64_t cand_i[2];
  __shared__ double red_v[kRbfBlock / 32];
  __shared__ int64_t red_i[kRbfBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int64_t nrow = (M - r + kRbfCluster - 1) / kRbfCluster;  // rows r, r + C, ...
  __shared__ int64_t steps;  // elimination steps completed (M unless a pivot was missing)
  for (int64_t t = tid; t < nrow; t += blockDim.x) used[t] = 0;
  if (tid == 0) steps = M;
  __syncthreads();
  for (int64_t k = 0; k < M; ++k) {
    const int slot = static_cast<int>(k & 1);
    // this block's candidate: the largest |A[i][k]| over its unused rows
    double best = -1.0;
    int64_t bi = M;
    for (int64_t t = tid; t < nrow; t += blockDim.x) {
      if (used[t]) continue;
      const int64_t i = r + t * kRbfCluster;
      const double v = fabs(A[i * M + k]);
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(kFull, best, o);
      const int64_t oi = __shfl_xor_sync(kFull, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = red_v[0];
      int64_t bj = red_i[0];
      for (int w = 1; w < nw; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bj)) { bv = red_v[w]; bj = red_i[w]; }
      cand_v[slot] = bv;
      cand_i[slot] = bj;
    }
    // the candidates of step k, and every block's rows as updated in step
    // k - 1, are visible across the cluster after this barrier
    cluster.sync();
    __shared__ int64_t piv;
    if (tid == 0) {
      double bv = -1.0;
      int64_t bj = M;
      for (int q = 0; q < kRbfCluster; ++q) {
        const double v = *cluster.map_shared_rank(&cand_v[slot], q);
        const int64_t ii = *cluster.map_shared_rank(&cand_i[slot], q);
        if (v > bv || (v == bv && ii < bj)) { bv = v; bj = ii; }
      }
      piv = bj;
      if (r == 0) {
        perm[k] = static_cast<int32_t>(bj);
        if (!(bv > 0.0)) *singular = 1;
      }
      if (bj < M && bj % kRbfCluster == r) used[bj / kRbfCluster] = 1;
    }
    __syncthreads();
    const int64_t pr = piv;
    if (pr >= M) {  // no unused row left (singular; flagged above)
      if (tid == 0) steps = k;
      break;
    }
    // the pivot row (columns k .. M - 1) and its right-hand side, read
    // through L2: its owner wrote it in an earlier step
    for (int64_t j = k + tid; j < M; j += blockDim.x) rowk[j] = __ldcg(A + pr * M + j);
    if (tid == 0) rowk[M] = __ldcg(b + pr);
    __syncthreads();
    const double akk = rowk[k], bk = rowk[M];
    // this block's unused rows: multiplier, then the row update (a warp per row)
    for (int64_t t = warp; t < nrow; t += nw) {
      if (used[t]) continue;
      const int64_t i = r + t * kRbfCluster;
      const double l = A[i * M + k] / akk;
      __syncwarp();  // every lane has read A[i][k] before lane 0 clears it
      for (int64_t j = k + 1 + lane; j < M; j += 32) A[i * M + j] = fma(-l, rowk[j], A[i * M + j]);
      if (lane == 0) {
        A[i * M + k] = 0.0;
        b[i] = fma(-l, bk, b[i]);
      }
    }
  }
  // every row's final state is written before the first block reads it
  cluster.sync();
  if (r != 0) return;
  if (steps < M) {  // incomplete elimination: no solution
    for (int64_t k = tid; k < M; k += blockDim.x) b[k] = static_cast<double>(NAN);
    return;
  }
  // back substitution in pivot order: x_k = (b_pk - sum_{j>k} A_pk,j x_j) / A_pk,k
  for (int64_t k = M - 1; k >= 0; --k) {
    const int64_t pk = perm[k];
    double acc = 0.0;
    for (int64_t j = k + 1 + tid; j < M; j += blockDim.x) acc = fma(__ldcg(A + pk * M + j), x[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0) red_v[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red_v[w];
      x[k] = (__ldcg(b + pk) - s) / __ldcg(A + pk * M + k);
    }
    __syncthreads();
  }
  for (int64_t k = tid; k < M; k += blockDim.x) b[k] = x[k];
}

__global__ void rbf_eval_kernel(const RbfPlane *planes, int32_t n_planes, const double *pts,
                                const double *sys, const double *query, double *out) {
  const int p = blockIdx.y;
  if (p >= n_planes) return;
  const RbfPlane P = planes[p];
  const int64_t M = P.M, npt = M - 3;
  const double *w = sys + P.sys0 + M * M;
  const double *xy = pts + 2 * P.pts0;
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < P.q;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double s, t;
    plane_coords(P.axis, query + 3 * (P.q0 + j), s, t);
    double acc = w[npt] + w[npt + 1] * s + w[npt + 2] * t;
    for (int64_t i = 0; i < npt; ++i) {
      const double ds = s - xy[2 * i], dt = t - xy[2 * i + 1];
      const double r2 = ds * ds + dt * dt;
      acc = fma(w[i], r2 * sqrt(r2), acc);
    }
    out[P.q0 + j] = acc;
  }
}

pdd_status interface_interp_impl(pdd_ctx *ctx, int32_t n_planes, const int32_t *h_axis,
                                 const double *h_pos, const int64_t *h_node_count,
                                 const double *d_nodes, const double *d_vals, int32_t n_bnd,
                                 const int64_t *h_query_count, const double *d_query,
                                 double *d_out) {
  if (ctx->prob.dim != 3 || ctx->prob.kind != PDD_PROB_ELLIPTIC_MANUFACTURED)
    return fail(ctx, PDD_EINVAL, "interface interpolation on planes covers the 3-D family");
  if (n_planes < 1 || n_planes > 64) return fail(ctx, PDD_EINVAL, "n_planes must be in [1, 64]");
  if (!h_axis || !h_pos || !h_node_count || !h_query_count)
    return fail(ctx, PDD_EINVAL, "null host array");
  if (n_bnd < 1 || n_bnd > 1024) return fail(ctx, PDD_EINVAL, "n_bnd must be in [1, 1024]");
  std::vector<RbfPlane> pl(static_cast<size_t>(n_planes));
  int64_t node0 = 0, sys0 = 0, pts0 = 0, q0 = 0;
  int32_t Mmax = 0;
  for (int p = 0; p < n_planes; ++p) {
    if (h_axis[p] < 0 || h_axis[p] > 2) return fail(ctx, PDD_EINVAL, "axis must be 0, 1 or 2");
    if (!(h_pos[p] > 0.0 && h_pos[p] < 1.0)) return fail(ctx, PDD_EINVAL, "plane outside (0, 1)");
    if (h_node_count[p] < 0 || h_query_count[p] < 0) return fail(ctx, PDD_EINVAL, "negative count");
    const int64_t M = h_node_count[p] + 4LL * n_bnd + 3;
    if (M > kRbfMaxSystem) return fail(ctx, PDD_EINVAL, "plane %d: system of %lld unknowns above %lld",
                                       p, static_cast<long long>(M), static_cast<long long>(kRbfMaxSystem));
    RbfPlane &P = pl[p];
    P.node0 = node0;
    P.m = h_node_count[p];
    P.sys0 = sys0;
    P.pts0 = pts0;
    P.q0 = q0;
    P.q = h_query_count[p];
    P.axis = h_axis[p];
    P.M = static_cast<int32_t>(M);
    P.pos = h_pos[p];
    node0 += P.m;
    sys0 += M * M + M;
    pts0 += M - 3;
    q0 += P.q;
    Mmax = std::max(Mmax, P.M);
  }
  if ((node0 > 0 && (!d_nodes || !d_vals)) || (q0 > 0 && (!d_query || !d_out)))
    return fail(ctx, PDD_EINVAL, "null buffer");
  if (q0 == 0) return PDD_OK;
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const size_t off_pl = 256;
  const size_t off_pts = align_up(off_pl + pl.size() * sizeof(RbfPlane), 256);
  const size_t off_pv = align_up(off_pts + static_cast<size_t>(pts0) * 2 * sizeof(double), 256);
  const size_t off_sys = align_up(off_pv + static_cast<size_t>(pts0) * sizeof(double), 256);
  const size_t bytes = align_up(off_sys + static_cast<size_t>(sys0) * sizeof(double), 256);
  pdd_status st = ensure_scratch(ctx, bytes);
  if (st != PDD_OK) return st;
  char *base = static_cast<char *>(ctx->scratch);
  int *singular = reinterpret_cast<int *>(base);
  auto *d_pl = reinterpret_cast<RbfPlane *>(base + off_pl);
  double *pts = reinterpret_cast<double *>(base + off_pts);
  double *pv = reinterpret_cast<double *>(base + off_pv);
  double *sys = reinterpret_cast<double *>(base + off_sys);
  PDD_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, 256, ctx->stream));
  PDD_CUDA_TRY(ctx, cudaMemcpyAsync(d_pl, pl.data(), pl.size() * sizeof(RbfPlane),
                                    cudaMemcpyHostToDevice, ctx->stream));
  const dim3 g1(static_cast<unsigned>(std::min<int64_t>((Mmax + 255) / 256, 64)),
                static_cast<unsigned>(n_planes));
  rbf_points_kernel<EllipticManufactured><<<g1, 256, 0, ctx->stream>>>(
      d_pl, n_planes, d_nodes, d_vals, n_bnd, ctx->mc, pts, pv);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  const dim3 g2(static_cast<unsigned>(std::min<int64_t>((int64_t(Mmax) * Mmax + 255) / 256, 4096)),
                static_cast<unsigned>(n_planes));
  rbf_assemble_kernel<<<g2, 256, 0, ctx->stream>>>(d_pl, n_planes, pts, pv, sys);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  // pivot row + solution (doubles), pivot order (int32), used flags (bytes)
  const size_t smem = static_cast<size_t>(2 * Mmax + 1) * sizeof(double) +
                      static_cast<size_t>(Mmax) * sizeof(int32_t) +
                      static_cast<size_t>(Mmax / kRbfCluster + 8);
  PDD_CUDA_TRY(ctx, cudaFuncSetAttribute(rbf_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
  rbf_solve_kernel<<<static_cast<unsigned>(n_planes) * kRbfCluster, kRbfBlock, smem, ctx->stream>>>(
      d_pl, n_planes, sys, singular);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  int64_t qmax = 0;
  for (const auto &P : pl) qmax = std::max(qmax, P.q);
  const dim3 g3(static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((qmax + 127) / 128, 4096))),
                static_cast<unsigned>(n_planes));
  rbf_eval_kernel<<<g3, 128, 0, ctx->stream>>>(d_pl, n_planes, pts, sys, d_query, d_out);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  int hs = 0;
  PDD_CUDA_TRY(ctx, cudaMemcpyAsync(&hs, singular, sizeof hs, cudaMemcpyDeviceToHost, ctx->stream));
  PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (hs) return fail(ctx, PDD_EINVAL, "singular interpolation system (coincident nodes?)");
  return PDD_OK;
}

// ---------------------------------------------------------------------------
// Subdomain solves on 3-D boxes.  The subdomains of stage two are independent
// problems (Sec. 2), so one call solves a batch of boxes of the same grid
// size together: every kernel below takes the box from blockIdx.y, and a box
// whose correction loop has stopped is skipped (live[b] == 0).  A batch of
// one box is the single solve; each box's arithmetic does not depend on the
// others, so a box gets the same bits alone or in a batch.
// ---------------------------------------------------------------------------
constexpr int kBox3MaxInterior = 126;  // interior points per axis (sine matrix in shared memory)
constexpr int kBox3Block = 256;

struct Box3 {
  double lo[3], h[3];
  int n[3];           // grid points per axis, boundary included
  int P[3];           // interior points per axis
  int mask;           // bit 2a + side: that face carries interface data
  int64_t face_off[6];  // offset of each face's data in the caller's array
};

__device__ __forceinline__ int64_t box3_index(const Box3 &B, int i, int j, int k) {
  return (static_cast<int64_t>(k) * B.n[1] + j) * B.n[0] + i;
}
__device__ __forceinline__ int64_t box3_total(const Box3 &B) {
  return static_cast<int64_t>(B.n[0]) * B.n[1] * B.n[2];
}
__device__ __forceinline__ int64_t box3_np(const Box3 &B) {
  return static_cast<int64_t>(B.P[0]) * B.P[1] * B.P[2];
}

// Dirichlet data and coefficients: boundary layer of u from the faces (a
// point on a face without interface data -- the physical boundary -- takes g;
// otherwise the interface face of lowest index), interior u = 0, and per
// interior point b, c and f of the family.
template <class Model>
__global__ void box3_setup_kernel(const Box3 *boxes, ModelConst mc, const double *face, double *u,
                                  double *coef) {
  const Box3 B = boxes[blockIdx.y];
  const int64_t total = box3_total(B);
  const int64_t np = box3_np(B);
  u += blockIdx.y * total;
  coef += blockIdx.y * 4 * np;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e % B.n[0]);
    const int j = static_cast<int>((e / B.n[0]) % B.n[1]);
    const int k = static_cast<int>(e / (static_cast<int64_t>(B.n[0]) * B.n[1]));
    const int idx[3] = {i, j, k};
    double x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = B.lo[a] + B.h[a] * idx[a];
    const bool interior = i > 0 && j > 0 && k > 0 && i < B.n[0] - 1 && j < B.n[1] - 1 &&
                          k < B.n[2] - 1;
    if (interior) {
      u[e] = 0.0;
      double b[3], f = 0.0;
      Model::template coeffs<double>(mc, x, b, f);
      const int64_t q = (static_cast<int64_t>(k - 1) * B.P[1] + (j - 1)) * B.P[0] + (i - 1);
      coef[q] = b[0];
      coef[np + q] = b[1];
      coef[2 * np + q] = b[2];
      coef[3 * np + q] = f;
      continue;
    }
    bool physical = false;
    int fbest = -1;
    for (int fc = 0; fc < 6; ++fc) {
      const int a = fc >> 1, side = fc & 1;
      const bool on = side ? idx[a] == B.n[a] - 1 : idx[a] == 0;
      if (!on) continue;
      if ((B.mask >> fc) & 1) {
        if (fbest < 0) fbest = fc;
      } else {
        physical = true;
      }
    }
    double v;
    if (physical || fbest < 0) {
      v = Model::template g<double>(mc, x);
    } else {
      // face grid of face fbest: the two other axes, the higher one slow
      const int a = fbest >> 1;
      const int a1 = a == 0 ? 1 : 0, a2 = a == 2 ? 1 : 2;
      v = face[B.face_off[fbest] + static_cast<int64_t>(idx[a2]) * B.n[a1] + idx[a1]];
    }
    u[e] = v;
  }
}

// r = -f - A u at the interior points (FP64), and the block's sum of r^2
// (part[box][block]).
__global__ void __launch_bounds__(kBox3Block)
box3_residual_kernel(const Box3 *boxes, const int32_t *live, double s2, double c, const double *u,
                     const double *coef, double *r, double *part) {
  if (!live[blockIdx.y]) return;
  const Box3 B = boxes[blockIdx.y];
  const int64_t np = box3_np(B);
  u += blockIdx.y * box3_total(B);
  coef += blockIdx.y * 4 * np;
  r += blockIdx.y * np;
  const double w0 = 0.5 * s2 / (B.h[0] * B.h[0]), w1 = 0.5 * s2 / (B.h[1] * B.h[1]),
               w2 = 0.5 * s2 / (B.h[2] * B.h[2]);
  const double d0 = 0.5 / B.h[0], d1 = 0.5 / B.h[1], d2 = 0.5 / B.h[2];
  const double diag = c - 2.0 * (w0 + w1 + w2);
  double acc = 0.0;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < np;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(q % B.P[0]) + 1;
    const int j = static_cast<int>((q / B.P[0]) % B.P[1]) + 1;
    const int k = static_cast<int>(q / (static_cast<int64_t>(B.P[0]) * B.P[1])) + 1;
    const int64_t e = box3_index(B, i, j, k);
    const int64_t sy = B.n[0], sz = static_cast<int64_t>(B.n[0]) * B.n[1];
    const double uc = u[e];
    const double ux0 = u[e - 1], ux1 = u[e + 1], uy0 = u[e - sy], uy1 = u[e + sy],
                 uz0 = u[e - sz], uz1 = u[e + sz];
    double Au = diag * uc + w0 * (ux0 + ux1) + w1 * (uy0 + uy1) + w2 * (uz0 + uz1);
    Au += coef[q] * d0 * (ux1 - ux0) + coef[np + q] * d1 * (uy1 - uy0) +
          coef[2 * np + q] * d2 * (uz1 - uz0);
    const double rv = -coef[3 * np + q] - Au;
    r[q] = rv;
    acc = fma(rv, rv, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  __shared__ double sh[kBox3Block / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBox3Block / 32; ++w) t += sh[w];
    part[static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x] = t;
  }
}

// Per box: the sum of its block partials in block order (deterministic), as
// a 2-norm (residual) or the largest (Jacobi change); one thread per box.
template <bool kMax>
__global__ void box3_combine_kernel(const double *part, int nblk, int nb, const int32_t *live,
                                    double *out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !live[b]) return;
  double t = 0.0;
  for (int k = 0; k < nblk; ++k) {
    const double v = part[static_cast<int64_t>(b) * nblk + k];
    t = kMax ? fmax(t, v) : t + v;
  }
  out[b] = kMax ? t : sqrt(t);
}

// The sine matrices S_a[k][j] = sin(pi (k+1)(j+1) / (P_a + 1)), binary32,
// the argument reduced exactly in integers.
__global__ void box3_sine_kernel(int P, float *S) {
  const int64_t n = static_cast<int64_t>(P) * P;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t k = e / P + 1, j = e % P + 1;
    const int64_t m = (k * j) % (2 * (P + 1));
    S[e] = static_cast<float>(sinpi(static_cast<double>(m) / (P + 1)));
  }
}

// out = S applied along axis AX of the P0 x P1 x P2 array of box blockIdx.y
// (x fastest): out[.., k, ..] = sum_j S[k][j] in[.., j, ..].  The matrix is
// staged in shared memory; threads of a warp take consecutive outputs, so
// along axes 1 and 2 their reads are coalesced and along axis 0 they read the
// same line.
template <int AX>
__global__ void __launch_bounds__(kBox3Block)
box3_dst_kernel(int P0, int P1, int P2, const int32_t *live, const float *__restrict__ S,
                const float *__restrict__ in, float *__restrict__ out,
                const double *__restrict__ rnorm, const double *__restrict__ in64) {
  if (!live[blockIdx.y]) return;
  extern __shared__ float Ss[];
  const int P = AX == 0 ? P0 : (AX == 1 ? P1 : P2);
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) Ss[e] = S[e];
  __syncthreads();
  const int64_t np = static_cast<int64_t>(P0) * P1 * P2;
  const int64_t off = blockIdx.y * np;
  const int64_t stride = AX == 0 ? 1 : (AX == 1 ? P0 : static_cast<int64_t>(P0) * P1);
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < np;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int kk = static_cast<int>((q / stride) % P);
    const int64_t base = off + q - kk * stride;
    const float *row = Ss + kk * P;
    float acc = 0.f;
    if (in64) {  // first pass: the FP64 residual scaled by 1 / |r|_2, then rounded
      const double inv = 1.0 / rnorm[blockIdx.y];
      for (int j = 0; j < P; ++j)
        acc = fmaf(row[j], static_cast<float>(in64[base + j * stride] * inv), acc);
    } else {
      for (int j = 0; j < P; ++j) acc = fmaf(row[j], in[base + j * stride], acc);
    }
    out[off + q] = acc;
  }
}

// cos(pi k / (P_a + 1)) - 1 for k = 1 .. P_a on each axis (cm1[a][k - 1]),
// formed once per solve: the eigenvalue factors of the 1-D second difference.
__global__ void box3_cos_kernel(int P0, int P1, int P2, double *cm1) {
  const int a = blockIdx.y;
  const int P = a == 0 ? P0 : (a == 1 ? P1 : P2);
  for (int k = threadIdx.x; k < P; k += blockDim.x)
    cm1[a * kBox3MaxInterior + k] = cospi(static_cast<double>(k + 1) / (P + 1)) - 1.0;
}

// Division by the eigenvalues of (1/2) sigma^2 Lap_h + c in the sine basis,
// lambda = sum_a (sigma^2 / h_a^2) (cos(pi k_a / (P_a + 1)) - 1) + c, and the
// normalisation of the two transforms, 8 / prod_a (P_a + 1).
__global__ void box3_eig_kernel(const Box3 *boxes, const int32_t *live, double s2, double c,
                                const double *__restrict__ cm1, float *v) {
  if (!live[blockIdx.y]) return;
  const Box3 B = boxes[blockIdx.y];
  const int64_t np = box3_np(B);
  v += blockIdx.y * np;
  const double norm = 8.0 / ((B.P[0] + 1.0) * (B.P[1] + 1.0) * (B.P[2] + 1.0));
  const double e0 = s2 / (B.h[0] * B.h[0]), e1 = s2 / (B.h[1] * B.h[1]),
               e2 = s2 / (B.h[2] * B.h[2]);
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < np;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int k0 = static_cast<int>(q % B.P[0]);
    const int k1 = static_cast<int>((q / B.P[0]) % B.P[1]);
    const int k2 = static_cast<int>(q / (static_cast<int64_t>(B.P[0]) * B.P[1]));
    const double lam = e0 * cm1[k0] + e1 * cm1[kBox3MaxInterior + k1] +
                       e2 * cm1[2 * kBox3MaxInterior + k2] + c;
    v[q] = static_cast<float>(static_cast<double>(v[q]) * (norm / lam));
  }
}

// u += (correction * |r|) at the interior points (undoing the scaling).
__global__ void box3_update_kernel(const Box3 *boxes, const int32_t *live, const float *v,
                                   const double *rnorm, double *u) {
  if (!live[blockIdx.y]) return;
  const Box3 B = boxes[blockIdx.y];
  const int64_t np = box3_np(B);
  v += blockIdx.y * np;
  u += blockIdx.y * box3_total(B);
  const double sc = rnorm[blockIdx.y];
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < np;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(q % B.P[0]) + 1;
    const int j = static_cast<int>((q / B.P[0]) % B.P[1]) + 1;
    const int k = static_cast<int>(q / (static_cast<int64_t>(B.P[0]) * B.P[1])) + 1;
    u[box3_index(B, i, j, k)] += static_cast<double>(v[q]) * sc;
  }
}

// One Jacobi sweep (the plain reference method): u' = (-f - offdiag(A) u) / diag,
// the block's largest change in part[box][block].
__global__ void __launch_bounds__(kBox3Block)
box3_jacobi_kernel(const Box3 *boxes, const int32_t *live, double s2, double c, const double *u,
                   double *un, const double *coef, double *part) {
  if (!live[blockIdx.y]) return;
  const Box3 B = boxes[blockIdx.y];
  const int64_t np = box3_np(B);
  u += blockIdx.y * box3_total(B);
  un += blockIdx.y * box3_total(B);
  coef += blockIdx.y * 4 * np;
  const double w0 = 0.5 * s2 / (B.h[0] * B.h[0]), w1 = 0.5 * s2 / (B.h[1] * B.h[1]),
               w2 = 0.5 * s2 / (B.h[2] * B.h[2]);
  const double d0 = 0.5 / B.h[0], d1 = 0.5 / B.h[1], d2 = 0.5 / B.h[2];
  const double diag = c - 2.0 * (w0 + w1 + w2);
  double mx = 0.0;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < np;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(q % B.P[0]) + 1;
    const int j = static_cast<int>((q / B.P[0]) % B.P[1]) + 1;
    const int k = static_cast<int>(q / (static_cast<int64_t>(B.P[0]) * B.P[1])) + 1;
    const int64_t e = box3_index(B, i, j, k);
    const int64_t sy = B.n[0], sz = static_cast<int64_t>(B.n[0]) * B.n[1];
    const double ux0 = u[e - 1], ux1 = u[e + 1], uy0 = u[e - sy], uy1 = u[e + sy],
                 uz0 = u[e - sz], uz1 = u[e + sz];
    const double off = (w0 - coef[q] * d0) * ux0 + (w0 + coef[q] * d0) * ux1 +
                       (w1 - coef[np + q] * d1) * uy0 + (w1 + coef[np + q] * d1) * uy1 +
                       (w2 - coef[2 * np + q] * d2) * uz0 + (w2 + coef[2 * np + q] * d2) * uz1;
    const double v = (-coef[3 * np + q] - off) / diag;
    mx = fmax(mx, fabs(v - u[e]));
    un[e] = v;
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
  __shared__ double sh[kBox3Block / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBox3Block / 32; ++w) t = fmax(t, sh[w]);
    part[static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x] = t;
  }
}

// A batch of nb boxes with the same grid size and method: the faces of box b
// follow those of box b - 1 in d_face, and d_u is [nb][n2][n1][n0].  *iters
// and *resid (if non-null) get the largest count and relative residual over
// the boxes; iters_each / resid_each (host, nb entries, may be null) get each
// box's own.
pdd_status subdomain_solve3d_batch_impl(pdd_ctx *ctx, const pdd_subdomain *sds, int32_t nb,
                                        const double *d_face, int64_t m, double *d_u,
                                        int64_t *iters, double *resid, int64_t *iters_each,
                                        double *resid_each) {
  if (!sds || nb < 1 || nb > 65535) return fail(ctx, PDD_EINVAL, "batch of 1 .. 65535 boxes");
  if (ctx->prob.kind != PDD_PROB_ELLIPTIC_MANUFACTURED || ctx->prob.dim != 3)
    return fail(ctx, PDD_EINVAL, "the 3-D subdomain solver covers the 3-D family");
  if (reflect_mask(ctx) != 0)
    return fail(ctx, PDD_EINVAL, "the 3-D subdomain solver takes Dirichlet data only");
  const pdd_subdomain &S0 = sds[0];
  std::vector<Box3> boxes(static_cast<size_t>(nb));
  int64_t off = 0;
  for (int32_t b = 0; b < nb; ++b) {
    const pdd_subdomain *sd = sds + b;
    Box3 &B = boxes[static_cast<size_t>(b)];
    for (int a = 0; a < 3; ++a) {
      if (sd->n[a] < 3 || sd->n[a] - 2 > kBox3MaxInterior)
        return fail(ctx, PDD_EINVAL, "3-D grids take 3 .. %d points per axis", kBox3MaxInterior + 2);
      if (sd->n[a] != S0.n[a])
        return fail(ctx, PDD_EINVAL, "the boxes of a batch share one grid size");
      if (!(sd->hi[a] > sd->lo[a]) || sd->lo[a] < 0.0 || sd->hi[a] > 1.0)
        return fail(ctx, PDD_EINVAL, "box must be non-empty and inside the unit cube");
      B.lo[a] = sd->lo[a];
      B.n[a] = sd->n[a];
      B.P[a] = sd->n[a] - 2;
      B.h[a] = (sd->hi[a] - sd->lo[a]) / (sd->n[a] - 1);
    }
    if (sd->iface_axis < 0 || sd->iface_axis > 63 || sd->iface_side != 0)
      return fail(ctx, PDD_EINVAL, "3-D: iface_axis is a mask of interface faces (0..63), "
                                   "iface_side must be 0");
    if (sd->method != PDD_STENCIL_DST && sd->method != PDD_STENCIL_JACOBI)
      return fail(ctx, PDD_EINVAL, "3-D methods: PDD_STENCIL_DST or PDD_STENCIL_JACOBI");
    if (sd->method != S0.method || sd->max_iter != S0.max_iter || !(sd->tol == S0.tol))
      return fail(ctx, PDD_EINVAL, "the boxes of a batch share one method and stopping rule");
    if (sd->max_iter < 1 || !(sd->tol >= 0.0)) return fail(ctx, PDD_EINVAL, "bad stopping rule");
    B.mask = sd->iface_axis;
    for (int fc = 0; fc < 6; ++fc) {
      B.face_off[fc] = off;
      if ((B.mask >> fc) & 1) {
        const int a = fc >> 1;
        off += static_cast<int64_t>(B.n[a == 0 ? 1 : 0]) * B.n[a == 2 ? 1 : 2];
      }
    }
  }
  if (m != off) return fail(ctx, PDD_EINVAL, "expected %lld face values, got %lld",
                            static_cast<long long>(off), static_cast<long long>(m));
  if (off > 0 && !d_face) return fail(ctx, PDD_EINVAL, "null face data");
  if (!d_u) return fail(ctx, PDD_EINVAL, "null output");
  PDD_CUDA_TRY(ctx, cudaSetDevice(ctx->device));

  const Box3 &B0 = boxes[0];
  const bool jacobi = S0.method == PDD_STENCIL_JACOBI;
  const int64_t total = static_cast<int64_t>(B0.n[0]) * B0.n[1] * B0.n[2];
  const int64_t np = static_cast<int64_t>(B0.P[0]) * B0.P[1] * B0.P[2];
  const size_t NB = static_cast<size_t>(nb);
  const int nblk = static_cast<int>(std::min<int64_t>((np + kBox3Block - 1) / kBox3Block, 1024));
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  const size_t off_rn = take(NB * sizeof(double));
  const size_t off_live = take(NB * sizeof(int32_t));
  const size_t off_box = take(NB * sizeof(Box3));
  const size_t off_coef = take(NB * 4 * np * sizeof(double));
  const size_t off_r = take(NB * np * sizeof(double));
  const size_t off_part = take(NB * nblk * sizeof(double));
  const size_t off_un = take(jacobi ? NB * total * sizeof(double) : 0);
  const size_t off_v0 = take(NB * np * sizeof(float));
  const size_t off_v1 = take(NB * np * sizeof(float));
  const size_t off_S = take(3 * kBox3MaxInterior * kBox3MaxInterior * sizeof(float));
  const size_t off_cm1 = take(3 * kBox3MaxInterior * sizeof(double));
  pdd_status st = ensure_scratch(ctx, o);
  if (st != PDD_OK) return st;
  char *base = static_cast<char *>(ctx->scratch);
  double *rn = reinterpret_cast<double *>(base + off_rn);  // per box: |r|_2 (Jacobi: largest change)
  int32_t *live = reinterpret_cast<int32_t *>(base + off_live);
  Box3 *d_boxes = reinterpret_cast<Box3 *>(base + off_box);
  double *coef = reinterpret_cast<double *>(base + off_coef);
  double *r = reinterpret_cast<double *>(base + off_r);
  double *part = reinterpret_cast<double *>(base + off_part);
  double *un = reinterpret_cast<double *>(base + off_un);
  float *v0 = reinterpret_cast<float *>(base + off_v0), *v1 = reinterpret_cast<float *>(base + off_v1);
  float *S[3];
  for (int a = 0; a < 3; ++a)
    S[a] = reinterpret_cast<float *>(base + off_S) + a * kBox3MaxInterior * kBox3MaxInterior;
  double *cm1 = reinterpret_cast<double *>(base + off_cm1);

  // host state of the correction loop (copied to and from the device
  // synchronously, so these buffers outlive every copy)
  std::vector<int32_t> h_live(NB, 1);
  std::vector<double> h_rn(NB, 0.0), h_r0(NB, -1.0), h_res(NB, 0.0);
  std::vector<int64_t> h_it(NB, 0);
  PDD_CUDA_TRY(ctx, cudaMemcpyAsync(d_boxes, boxes.data(), NB * sizeof(Box3),
                                    cudaMemcpyHostToDevice, ctx->stream));
  PDD_CUDA_TRY(ctx, cudaMemcpyAsync(live, h_live.data(), NB * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, ctx->stream));
  const unsigned gset = static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 4096));
  box3_setup_kernel<EllipticManufactured><<<dim3(gset, nb), 256, 0, ctx->stream>>>(
      d_boxes, ctx->mc, d_face, d_u, coef);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  const double s2 = ctx->prob.sigma * ctx->prob.sigma;
  const double c = constant_kill(ctx->prob.kind);
  const unsigned gcomb = static_cast<unsigned>((nb + 127) / 128);
  const auto ev = prof_slot(ctx);
  if (ev.first) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.first, ctx->stream));
  // read the per-box measures, then decide per box whether it goes on
  auto read_measures = [&]() -> pdd_status {
    PDD_CUDA_TRY(ctx, cudaMemcpyAsync(h_rn.data(), rn, NB * sizeof(double), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return PDD_OK;
  };
  auto push_live = [&]() -> pdd_status {
    PDD_CUDA_TRY(ctx, cudaMemcpyAsync(live, h_live.data(), NB * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, ctx->stream));
    return PDD_OK;
  };
  if (jacobi) {
    // each box sweeps between its own two buffers; a box that stops keeps its
    // latest iterate where its own step count left it
    PDD_CUDA_TRY(ctx, cudaMemcpyAsync(un, d_u, NB * total * sizeof(double),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    const unsigned gj = static_cast<unsigned>(nblk);
    int n_live = nb;
    for (int64_t it = 1; it <= S0.max_iter && n_live > 0; ++it) {
      const bool odd = (it & 1) != 0;
      box3_jacobi_kernel<<<dim3(gj, nb), kBox3Block, 0, ctx->stream>>>(
          d_boxes, live, s2, c, odd ? d_u : un, odd ? un : d_u, coef, part);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
      for (size_t b = 0; b < NB; ++b)
        if (h_live[b]) h_it[b] = it;
      if (it % 16 == 0 || it == S0.max_iter) {
        box3_combine_kernel<true><<<gcomb, 128, 0, ctx->stream>>>(part, nblk, nb, live, rn);
        PDD_CUDA_TRY(ctx, cudaGetLastError());
        st = read_measures();
        if (st != PDD_OK) return st;
        for (size_t b = 0; b < NB; ++b) {
          if (!h_live[b]) continue;
          h_res[b] = h_rn[b];
          if (h_rn[b] < S0.tol || it == S0.max_iter) {
            h_live[b] = 0;
            --n_live;
          }
        }
        st = push_live();
        if (st != PDD_OK) return st;
      }
    }
    // a box whose last sweep was odd holds its iterate in un
    for (size_t b = 0; b < NB; ++b)
      if (h_it[b] & 1)
        PDD_CUDA_TRY(ctx, cudaMemcpyAsync(d_u + b * total, un + b * total, total * sizeof(double),
                                          cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    for (int a = 0; a < 3; ++a) {
      box3_sine_kernel<<<static_cast<unsigned>((B0.P[a] * B0.P[a] + 255) / 256), 256, 0, ctx->stream>>>(
          B0.P[a], S[a]);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
    }
    box3_cos_kernel<<<dim3(1, 3), 128, 0, ctx->stream>>>(B0.P[0], B0.P[1], B0.P[2], cm1);
    PDD_CUDA_TRY(ctx, cudaGetLastError());
    int smax = 0;
    for (int a = 0; a < 3; ++a) smax = std::max(smax, B0.P[a] * B0.P[a]);
    const size_t smem = static_cast<size_t>(smax) * sizeof(float);
    PDD_CUDA_TRY(ctx, cudaFuncSetAttribute(box3_dst_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
    PDD_CUDA_TRY(ctx, cudaFuncSetAttribute(box3_dst_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
    PDD_CUDA_TRY(ctx, cudaFuncSetAttribute(box3_dst_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
    const unsigned gt = static_cast<unsigned>(std::min<int64_t>((np + kBox3Block - 1) / kBox3Block, 2048));
    const dim3 gr(static_cast<unsigned>(nblk), nb), gd(gt, nb);
    for (int64_t it = 0;; ++it) {
      box3_residual_kernel<<<gr, kBox3Block, 0, ctx->stream>>>(d_boxes, live, s2, c, d_u, coef, r,
                                                              part);
      box3_combine_kernel<false><<<gcomb, 128, 0, ctx->stream>>>(part, nblk, nb, live, rn);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
      st = read_measures();
      if (st != PDD_OK) return st;
      int n_live = 0;
      for (size_t b = 0; b < NB; ++b) {
        if (!h_live[b]) continue;
        if (h_r0[b] < 0.0) h_r0[b] = h_rn[b];
        h_it[b] = it;
        h_res[b] = h_r0[b] > 0.0 ? h_rn[b] / h_r0[b] : 0.0;
        if (h_rn[b] <= S0.tol * h_r0[b] || h_rn[b] == 0.0 || it >= S0.max_iter)
          h_live[b] = 0;
        else
          ++n_live;
      }
      if (n_live == 0) break;
      st = push_live();
      if (st != PDD_OK) return st;
      // forward transform (x from the scaled FP64 residual, then y, z), the
      // eigenvalues, the inverse transform (x, y, z), the update
      box3_dst_kernel<0><<<gd, kBox3Block, smem, ctx->stream>>>(B0.P[0], B0.P[1], B0.P[2], live, S[0], nullptr, v0, rn, r);
      box3_dst_kernel<1><<<gd, kBox3Block, smem, ctx->stream>>>(B0.P[0], B0.P[1], B0.P[2], live, S[1], v0, v1, nullptr, nullptr);
      box3_dst_kernel<2><<<gd, kBox3Block, smem, ctx->stream>>>(B0.P[0], B0.P[1], B0.P[2], live, S[2], v1, v0, nullptr, nullptr);
      box3_eig_kernel<<<gd, kBox3Block, 0, ctx->stream>>>(d_boxes, live, s2, c, cm1, v0);
      box3_dst_kernel<0><<<gd, kBox3Block, smem, ctx->stream>>>(B0.P[0], B0.P[1], B0.P[2], live, S[0], v0, v1, nullptr, nullptr);
      box3_dst_kernel<1><<<gd, kBox3Block, smem, ctx->stream>>>(B0.P[0], B0.P[1], B0.P[2], live, S[1], v1, v0, nullptr, nullptr);
      box3_dst_kernel<2><<<gd, kBox3Block, smem, ctx->stream>>>(B0.P[0], B0.P[1], B0.P[2], live, S[2], v0, v1, nullptr, nullptr);
      box3_update_kernel<<<gd, kBox3Block, 0, ctx->stream>>>(d_boxes, live, v1, rn, d_u);
      PDD_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  if (ev.second) PDD_CUDA_TRY(ctx, cudaEventRecord(ev.second, ctx->stream));
  PDD_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  int64_t it_max = 0;
  double res_max = 0.0;
  bool unmet = false;
  for (size_t b = 0; b < NB; ++b) {
    it_max = std::max(it_max, h_it[b]);
    res_max = std::max(res_max, h_res[b]);
    unmet |= jacobi ? h_res[b] >= S0.tol : h_res[b] > S0.tol;
    if (iters_each) iters_each[b] = h_it[b];
    if (resid_each) resid_each[b] = h_res[b];
  }
  if (iters) *iters = it_max;
  if (resid) *resid = res_max;
  if (unmet) return fail(ctx, PDD_ETIMEOUT, "max_iter reached before the tolerance");
  return PDD_OK;
}

pdd_status subdomain_solve3d_impl(pdd_ctx *ctx, const pdd_subdomain *sd, const double *d_face,
                                  int64_t m, double *d_u, int64_t *iters, double *resid) {
  return subdomain_solve3d_batch_impl(ctx, sd, 1, d_face, m, d_u, iters, resid, nullptr, nullptr);
}

}  // namespace pdd
