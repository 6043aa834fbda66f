// dst.cu -- direct subdomain solve of stage two (Sec. 2.1) by discrete sine
// transforms.  On a rectangle with Dirichlet data the 5-point operator
//   A U = (2/hx^2 + 2/hy^2) U - (U_W + U_E)/hx^2 - (U_S + U_N)/hy^2
// over the P x Q interior points (P = nx - 2, Q = ny - 2) is diagonal in the
// DST-I basis: with S_P[i][k] = sin(pi (i+1)(k+1) / (P+1)) (symmetric,
// S_P^2 = (P+1)/2 I) and the eigenvalues
//   lambda_k = 4/hx^2 sin^2(pi (k+1) / (2 (P+1))),
//   nu_l     = 4/hy^2 sin^2(pi (l+1) / (2 (Q+1))),
// the solution of A U = F (F: the boundary values moved to the right) is
//   U = 4 / ((P+1)(Q+1)) S_Q [(S_Q F S_P) ./ (nu_l + lambda_k)] S_P,
// the same discrete solution the iterative methods converge to, here to
// rounding.  Four dense FP64 products of the sine matrices (O(PQ(P+Q))
// flops) replace the iterations.
#include <algorithm>
#include <cmath>

#include "ctx.hpp"

namespace pdd {

constexpr int kDstTile = 16;  // 16 x 16 outputs per block: the FP64 rate is per SM, so more blocks

// S[i][k] = sin(pi (i+1)(k+1) / (n+1)), i, k < n: the product is reduced
// modulo 2(n+1) in integers, so sinpi sees an exact argument in [0, 2).
__global__ void dst_matrix_kernel(double *S, int n) {
  const int64_t total = static_cast<int64_t>(n) * n;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = t / n, k = t - i * n;
    const int64_t r = ((i + 1) * (k + 1)) % (2 * static_cast<int64_t>(n + 1));
    S[t] = sinpi(static_cast<double>(r) / static_cast<double>(n + 1));
  }
}

// F[j][i] (j < Q rows along y, i < P columns along x): the Dirichlet values
// next to interior point (i+1, j+1), weighted by 1/h^2.
__global__ void dst_rhs_kernel(const double *u, int nx, int ny, double ihx2, double ihy2,
                               double *F) {
  const int P = nx - 2, Q = ny - 2;
  const int64_t total = static_cast<int64_t>(P) * Q;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(t / P), i = static_cast<int>(t - static_cast<int64_t>(j) * P);
    const int64_t row = static_cast<int64_t>(j + 1) * nx;
    double f = 0.0;
    if (i == 0) f += u[row] * ihx2;
    if (i == P - 1) f += u[row + nx - 1] * ihx2;
    if (j == 0) f += u[i + 1] * ihy2;
    if (j == Q - 1) f += u[static_cast<int64_t>(ny - 1) * nx + i + 1] * ihy2;
    F[t] = f;
  }
}

// C[M][N] = A[M][K] B[K][N], FP64, row-major; 16 x 16 output tiles staged
// through shared memory, one output per thread.
__global__ void __launch_bounds__(kDstTile * kDstTile)
dst_gemm_kernel(const double *A, const double *B, double *C, int M, int N, int K) {
  __shared__ double As[kDstTile][kDstTile + 1];
  __shared__ double Bs[kDstTile][kDstTile + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * kDstTile + ty, col = blockIdx.x * kDstTile + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += kDstTile) {
    As[ty][tx] = (row < M && k0 + tx < K) ? A[static_cast<int64_t>(row) * K + k0 + tx] : 0.0;
    Bs[ty][tx] = (k0 + ty < K && col < N) ? B[static_cast<int64_t>(k0 + ty) * N + col] : 0.0;
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kDstTile; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (row < M && col < N) C[static_cast<int64_t>(row) * N + col] = acc;
}

// Fh[l][k] <- Fh[l][k] * 4 / ((P+1)(Q+1)) / (nu_l + lambda_k)
__global__ void dst_divide_kernel(double *Fh, int P, int Q, double ihx2, double ihy2) {
  const int64_t total = static_cast<int64_t>(P) * Q;
  const double scale = 4.0 / (static_cast<double>(P + 1) * static_cast<double>(Q + 1));
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int l = static_cast<int>(t / P), k = static_cast<int>(t - static_cast<int64_t>(l) * P);
    const double sx = sinpi(static_cast<double>(k + 1) / (2.0 * (P + 1)));
    const double sy = sinpi(static_cast<double>(l + 1) / (2.0 * (Q + 1)));
    Fh[t] *= scale / (4.0 * ihx2 * sx * sx + 4.0 * ihy2 * sy * sy);
  }
}

__global__ void dst_scatter_kernel(const double *U, int nx, int ny, double *u) {
  const int P = nx - 2, Q = ny - 2;
  const int64_t total = static_cast<int64_t>(P) * Q;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(t / P), i = static_cast<int>(t - static_cast<int64_t>(j) * P);
    u[static_cast<int64_t>(j + 1) * nx + i + 1] = U[t];
  }
}

// ||F - A U||_2 / ||F||_2 over the interior (0 when F = 0), in a fixed
// order: each block sums a fixed slice of points (part[2 b], part[2 b + 1]),
// then one block adds the partials in block order; *it = 0 (a direct solve).
constexpr int kDstResBlocks = 64;
__global__ void dst_residual_part_kernel(const double *u, const double *F, int nx, int ny,
                                         double ihx2, double ihy2, double *part) {
  __shared__ double sr[256], sb[256];
  const int P = nx - 2, Q = ny - 2;
  const int64_t total = static_cast<int64_t>(P) * Q;
  const double diag = 2.0 * ihx2 + 2.0 * ihy2;
  double r2 = 0.0, b2 = 0.0;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(t / P), i = static_cast<int>(t - static_cast<int64_t>(j) * P);
    const int64_t c = static_cast<int64_t>(j + 1) * nx + i + 1;
    // interior neighbours only: the boundary ones are in F
    const double w = i > 0 ? u[c - 1] : 0.0, e = i < P - 1 ? u[c + 1] : 0.0;
    const double s = j > 0 ? u[c - nx] : 0.0, n = j < Q - 1 ? u[c + nx] : 0.0;
    const double Au = diag * u[c] - ihx2 * (w + e) - ihy2 * (s + n);
    const double r = F[t] - Au;
    r2 += r * r;
    b2 += F[t] * F[t];
  }
  sr[threadIdx.x] = r2;
  sb[threadIdx.x] = b2;
  __syncthreads();
  for (int m = blockDim.x / 2; m > 0; m >>= 1) {
    if (static_cast<int>(threadIdx.x) < m) {
      sr[threadIdx.x] += sr[threadIdx.x + m];
      sb[threadIdx.x] += sb[threadIdx.x + m];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sr[0];
    part[2 * blockIdx.x + 1] = sb[0];
  }
}
__global__ void dst_residual_final_kernel(const double *part, int nparts, int64_t *it,
                                          double *res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double r2 = 0.0, b2 = 0.0;
  for (int b = 0; b < nparts; ++b) {
    r2 += part[2 * b];
    b2 += part[2 * b + 1];
  }
  *it = 0;
  *res = b2 > 0.0 ? sqrt(r2 / b2) : sqrt(r2);
}

static unsigned dst_grid(int64_t work) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096)));
}

static void dst_gemm(cudaStream_t st, const double *A, const double *B, double *C, int M, int N,
                     int K) {
  const dim3 grid((N + kDstTile - 1) / kDstTile, (M + kDstTile - 1) / kDstTile);
  dst_gemm_kernel<<<grid, dim3(kDstTile, kDstTile), 0, st>>>(A, B, C, M, N, K);
}

size_t dst_scratch_bytes(int nx, int ny) {
  const size_t P = static_cast<size_t>(nx - 2), Q = static_cast<size_t>(ny - 2);
  return align_up(P * P * sizeof(double), 256) + align_up(Q * Q * sizeof(double), 256) +
         2 * align_up(P * Q * sizeof(double), 256) + 2 * kDstResBlocks * sizeof(double);
}

// d_u holds the Dirichlet data on the boundary (interior ignored); on return
// the interior holds the solution.  work: dst_scratch_bytes(nx, ny) bytes.
pdd_status dst_solve(pdd_ctx *ctx, double *d_u, int nx, int ny, double hx, double hy, char *work,
                     int64_t *it_d, double *res_d) {
  const int P = nx - 2, Q = ny - 2;
  const double ihx2 = 1.0 / (hx * hx), ihy2 = 1.0 / (hy * hy);
  double *SP = reinterpret_cast<double *>(work);
  double *SQ = reinterpret_cast<double *>(work + align_up(static_cast<size_t>(P) * P * sizeof(double), 256));
  double *F = reinterpret_cast<double *>(reinterpret_cast<char *>(SQ) +
                                         align_up(static_cast<size_t>(Q) * Q * sizeof(double), 256));
  double *T = reinterpret_cast<double *>(reinterpret_cast<char *>(F) +
                                         align_up(static_cast<size_t>(P) * Q * sizeof(double), 256));
  const int64_t pq = static_cast<int64_t>(P) * Q;
  cudaStream_t st = ctx->stream;
  dst_matrix_kernel<<<dst_grid(static_cast<int64_t>(P) * P), 256, 0, st>>>(SP, P);
  dst_matrix_kernel<<<dst_grid(static_cast<int64_t>(Q) * Q), 256, 0, st>>>(SQ, Q);
  dst_rhs_kernel<<<dst_grid(pq), 256, 0, st>>>(d_u, nx, ny, ihx2, ihy2, F);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  dst_gemm(st, F, SP, T, Q, P, P);   // T  = F S_P
  dst_gemm(st, SQ, T, F, Q, P, Q);   // Fh = S_Q T   (F no longer needed as data)
  dst_divide_kernel<<<dst_grid(pq), 256, 0, st>>>(F, P, Q, ihx2, ihy2);
  dst_gemm(st, F, SP, T, Q, P, P);   // T  = Uh S_P
  dst_gemm(st, SQ, T, F, Q, P, Q);   // U  = S_Q T
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  dst_scatter_kernel<<<dst_grid(pq), 256, 0, st>>>(F, nx, ny, d_u);
  // the residual against the right-hand side, rebuilt from the boundary
  dst_rhs_kernel<<<dst_grid(pq), 256, 0, st>>>(d_u, nx, ny, ihx2, ihy2, T);
  double *part = reinterpret_cast<double *>(reinterpret_cast<char *>(T) +
                                            align_up(static_cast<size_t>(P) * Q * sizeof(double), 256));
  dst_residual_part_kernel<<<kDstResBlocks, 256, 0, st>>>(d_u, T, nx, ny, ihx2, ihy2, part);
  dst_residual_final_kernel<<<1, 32, 0, st>>>(part, kDstResBlocks, it_d, res_d);
  PDD_CUDA_TRY(ctx, cudaGetLastError());
  return PDD_OK;
}

}  // namespace pdd
