/*
 * oracle.c -- plain, slow FP64 CPU oracle for the interface-node Monte Carlo
 * of Probabilistic Domain Decomposition (Bernal, dos Reis, Smith,
 * arXiv:1705.03666).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code with the CUDA path:
 * it has its own Philox, its own normal/uniform maps, its own coefficient
 * formulas, geometry and stepping.  The only thing both sides agree on is the
 * documented layout of the random streams (which counter feeds which draw),
 * so that both consume identical 32-bit words.
 *
 * Everything is double precision and follows the paper's equations in the
 * order they are written:
 *   - Feynman-Kac / Dynkin representation, Eq. 2.1-2.2 (Laplace) and
 *     Eq. 2.5-2.9 with the elliptic, purely Dirichlet reduction of Sec. 2.2
 *     (u = E[g(X_tau) Y_tau + Z_tau], dX = b dt + sigma dW,
 *      dY = c Y dt, dZ = f Y dt);
 *   - Euler-Maruyama with a boundary test and the boundary-corrected
 *     (Brownian-bridge, half-space) exit test the paper cites in Sec. 2.1;
 *   - the Monte Carlo sample mean over independent realisations (Sec. 2);
 *   - branching Brownian motion for the KPP-type equation Eq. 3.1 with
 *     exponential lifetimes and offspring law alpha (Sec. 3.1, Assumption
 *     3.1, the KPP representation of Sec. 3.1.1 and Algorithm 3.1 with
 *     per-particle lifetimes), including the marked weights alpha_k/q_k of
 *     Sec. 3.2;
 *   - the likelihood-ratio derivative of the discrete scheme with respect to
 *     drift parameters, and the exact pathwise derivative with respect to
 *     linear boundary-data parameters;
 *   - reflecting (Neumann/Robin) faces of the mixed problem Eq. 2.4 through
 *     the local-time terms of Eq. 2.9 (Lepingle's half-space reflection);
 *   - Walk on Spheres for the Laplace problem (the scheme Sec. 2.1 names for
 *     stopped Brownian motion);
 *   - branching trees on a time grid (Algorithm 3.1's time-point sharing),
 *     in free space or with absorbing boundaries (Eq. 3.2);
 *   - one level of the multilevel estimator (Giles' method, Sec. 2.1) with
 *     coupled fine/coarse Euler paths.
 *
 * Readings where the paper is silent (exit point, bridge formula, left-point
 * quadrature, stream layout, tree ordering) are listed in the design notes and
 * restated at each function below.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Enumerations (integer values are part of the documented interface).       */
/* ------------------------------------------------------------------------ */
enum { ORC_GEOM_INTERVAL = 0, ORC_GEOM_UNIT_SQUARE = 1, ORC_GEOM_L_SHAPE = 2,
       ORC_GEOM_UNIT_CUBE = 3, ORC_GEOM_FREE_SPACE = 4 };
enum { ORC_PROB_LAPLACE_EXPCOS = 1, ORC_PROB_ELLIPTIC_MANUFACTURED = 2,
       ORC_PROB_POISSON_FOURIER = 3, ORC_PROB_BERNAL_ACEBRON = 4,
       ORC_PROB_POLY1D = 5, ORC_PROB_TORSION = 6, ORC_PROB_KPP = 7 };
enum { ORC_PSI_CONST = 0, ORC_PSI_SIGMOID = 1, ORC_PSI_TRAVELLING = 2, ORC_PSI_SINE = 3 };

typedef struct {
  int32_t kind, geometry, dim, n_params;
  const double *params;
  double sigma;
} orc_problem;

typedef struct {
  uint64_t seed;
  double dt;
  int64_t n_paths;
  int64_t max_steps;
  int32_t bridge;
  int32_t n_threads;
} orc_mc;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the description in Salmon, Moraes, Dror and   */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds,  */
/* each multiplying counter words 0 and 2 by two fixed odd constants, taking */
/* the 64-bit products apart into high and low halves, mixing the high      */
/* halves with the other two words and the round key by XOR and permuting;  */
/* the two key words are bumped by the Weyl constants between rounds.       */
/* ------------------------------------------------------------------------ */
static const uint32_t PHX_M0 = 0xD2511F53u, PHX_M1 = 0xCD9E8D57u;
static const uint32_t PHX_W0 = 0x9E3779B9u, PHX_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHX_W0;
    k1 += PHX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Dump n_blocks consecutive Philox outputs for counters
 * (j0 + b, c1, c2, c3), b = 0..n_blocks-1, key = (seed lo, seed hi).       */
void orc_philox_stream(uint64_t seed, uint32_t j0, uint32_t c1, uint32_t c2,
                       uint32_t c3, int64_t n_blocks, uint32_t *out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t b = 0; b < n_blocks; ++b) {
    uint32_t ctr[4] = {j0 + (uint32_t)b, c1, c2, c3};
    orc_philox4x32_10(ctr, key, out + 4 * b);
  }
}

/* Uniform on (0,1): U = (floor(w / 2^9) + 1/2) * 2^-23.  Every value is an
 * odd multiple of 2^-24, never 0 or 1, and exactly representable in binary32
 * as well as binary64.                                                     */
static double unif(uint32_t w) {
  return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Box-Muller: two uniforms -> two independent standard normals.            */
static void box_muller(uint32_t a, uint32_t b, double *z0, double *z1) {
  double r = sqrt(-2.0 * log(unif(a)));
  double th = 2.0 * M_PI * unif(b);
  *z0 = r * cos(th);
  *z1 = r * sin(th);
}

/* n normals BM(w0, w1) of blocks Philox((j, c1, c2, c3)), j = 0..n/2-1,
 * and the matching uniforms unif(w2): for statistical checks of the maps.  */
void orc_normals(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3,
                 int64_t n_pairs, double *z, double *u) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t j = 0; j < n_pairs; ++j) {
    uint32_t ctr[4] = {(uint32_t)j, c1, c2, c3}, w[4];
    orc_philox4x32_10(ctr, key, w);
    box_muller(w[0], w[1], z + 2 * j, z + 2 * j + 1);
    if (u) u[j] = unif(w[2]);
  }
}

/* The four Philox constants (multipliers, then Weyl key increments).       */
void orc_philox_constants(uint32_t out[4]) {
  out[0] = PHX_M0; out[1] = PHX_M1; out[2] = PHX_W0; out[3] = PHX_W1;
}

/* ------------------------------------------------------------------------ */
/* Coefficients of the PDE in the paper's form (Eq. 2.3-2.4, elliptic limit): */
/*   (1/2) sigma^2 Lap u + b.grad u + c u + f = 0 in Omega,  u = g on dOmega */
/* c is the paper's c (<= 0), f the paper's f.                               */
/* ------------------------------------------------------------------------ */

/* Eq. 2.10 exact solution and the source that makes it exact (sigma^2 = 2,
 * so the generator is the full Laplacian as written in Eq. 2.10).          */
static double ba_u(double x, double y) {
  return 2.0 * cos(2.0 * (y - 2.0) * x) + sin(3.0 * (x - 2.0) * y) + 3.1;
}
static double ba_h(double x, double y) { return cos(x + y) / (1.1 + sin(x + y)); }
static double ba_c(double x, double y) {
  return -(x * x + y * y) / (1.1 + sin(x + y));
}
static double ba_f(double x, double y) {
  double A = 2.0 * (y - 2.0) * x, B = 3.0 * (x - 2.0) * y;
  double ux = -4.0 * (y - 2.0) * sin(A) + 3.0 * y * cos(B);
  double uy = -4.0 * x * sin(A) + 3.0 * (x - 2.0) * cos(B);
  double lap = -8.0 * ((y - 2.0) * (y - 2.0) + x * x) * cos(A)
               - 9.0 * (y * y + (x - 2.0) * (x - 2.0)) * sin(B);
  /* Lap u + h (u_x + u_y) + c u + f = 0 */
  return -(lap + ba_h(x, y) * (ux + uy) + ba_c(x, y) * ba_u(x, y));
}

/* Manufactured 3-D problem: (1/2) Lap u + b.grad u - u = F with
 * u = sin(pi x) sin(pi y) e^z, b = (0.5 sin 2 pi y, 0.5 cos 2 pi x, 0).
 * In the paper's form c = -1 and f = -F.                                  */
static double em_u(const double *x) {
  return sin(M_PI * x[0]) * sin(M_PI * x[1]) * exp(x[2]);
}
static double em_F(const double *x) {
  double sx = sin(M_PI * x[0]), cx = cos(M_PI * x[0]);
  double sy = sin(M_PI * x[1]), cy = cos(M_PI * x[1]);
  double ez = exp(x[2]);
  double u = sx * sy * ez;
  double half_lap = 0.5 * (1.0 - 2.0 * M_PI * M_PI) * u;
  double bgrad = 0.5 * sin(2.0 * M_PI * x[1]) * M_PI * cx * sy * ez
               + 0.5 * cos(2.0 * M_PI * x[0]) * M_PI * sx * cy * ez;
  return half_lap + bgrad - u;
}

static void coef_drift(const orc_problem *P, const double *x, double *b) {
  b[0] = b[1] = b[2] = 0.0;
  switch (P->kind) {
  case ORC_PROB_ELLIPTIC_MANUFACTURED:
    b[0] = 0.5 * sin(2.0 * M_PI * x[1]);
    b[1] = 0.5 * cos(2.0 * M_PI * x[0]);
    break;
  case ORC_PROB_POISSON_FOURIER: {
    /* params: theta[64] (theta_mn at m*8+n), then phi[16] */
    const double *phi = P->params + 64;
    for (int j = 1; j <= 8; ++j) {
      b[0] += phi[j - 1] * sin(j * M_PI * x[1]);
      b[1] += phi[8 + j - 1] * sin(j * M_PI * x[0]);
    }
    break;
  }
  case ORC_PROB_BERNAL_ACEBRON:
    b[0] = b[1] = ba_h(x[0], x[1]);
    break;
  case ORC_PROB_POLY1D:
    /* params: b0, b1, c0, f0, f1, g0, g1 */
    b[0] = P->params[0] + P->params[1] * x[0];
    break;
  default:
    break;
  }
}

static double coef_c(const orc_problem *P, const double *x) {
  switch (P->kind) {
  case ORC_PROB_ELLIPTIC_MANUFACTURED: return -1.0;
  case ORC_PROB_BERNAL_ACEBRON: return ba_c(x[0], x[1]);
  case ORC_PROB_POLY1D: return P->params[2];
  default: return 0.0;
  }
}

static double coef_f(const orc_problem *P, const double *x) {
  switch (P->kind) {
  case ORC_PROB_ELLIPTIC_MANUFACTURED: return -em_F(x);
  case ORC_PROB_POISSON_FOURIER: return 1.0;
  case ORC_PROB_BERNAL_ACEBRON: return ba_f(x[0], x[1]);
  case ORC_PROB_POLY1D: return P->params[3] + P->params[4] * x[0];
  case ORC_PROB_TORSION: return 1.0;
  default: return 0.0;
  }
}

static double coef_g(const orc_problem *P, const double *x) {
  switch (P->kind) {
  case ORC_PROB_LAPLACE_EXPCOS: return exp(x[0]) * cos(x[1]);
  case ORC_PROB_ELLIPTIC_MANUFACTURED: return em_u(x);
  case ORC_PROB_POISSON_FOURIER: {
    double s = 0.0;
    for (int m = 0; m < 8; ++m)
      for (int n = 0; n < 8; ++n)
        s += P->params[m * 8 + n] * cos(m * M_PI * x[0]) * cos(n * M_PI * x[1]);
    return s;
  }
  case ORC_PROB_BERNAL_ACEBRON: return ba_u(x[0], x[1]);
  case ORC_PROB_POLY1D: return (x[0] < 0.5) ? P->params[5] : P->params[6];
  default: return 0.0;
  }
}

/* Reflecting faces (Eq. 2.4 with dOmega_R non-empty): on a reflecting face
 * the condition is du/dN = phi u + psi, N the outward normal, phi <= 0.
 * The Laplace, 3-D manufactured and torsion families accept two optional
 * parameters [reflect mask (bit j: face j of the box is reflecting), phi];
 * psi is what keeps the family's exact solution exact, du/dN - phi u
 * (Laplace: u = e^x cos y; 3-D: the manufactured u), and 0 for torsion
 * (homogeneous Robin data).  Boxes only.                                   */
static int reflect_mask(const orc_problem *P) {
  if (P->kind != ORC_PROB_LAPLACE_EXPCOS && P->kind != ORC_PROB_ELLIPTIC_MANUFACTURED &&
      P->kind != ORC_PROB_TORSION)
    return 0;
  if (P->geometry == ORC_GEOM_L_SHAPE || P->geometry == ORC_GEOM_FREE_SPACE) return 0;
  if (P->n_params < 2) return 0;
  return (int)P->params[0] & ((1 << (2 * P->dim)) - 1);
}

static double robin_psi(const orc_problem *P, int j, const double *x) {
  const int k = j >> 1;
  const double s = (j & 1) ? 1.0 : -1.0; /* outward normal = s e_k */
  const double phi = P->params[1];
  double grad[3] = {0, 0, 0}, u = 0.0;
  if (P->kind == ORC_PROB_LAPLACE_EXPCOS) {
    u = exp(x[0]) * cos(x[1]);
    grad[0] = u;
    grad[1] = -exp(x[0]) * sin(x[1]);
  } else if (P->kind == ORC_PROB_ELLIPTIC_MANUFACTURED) {
    u = em_u(x);
    grad[0] = M_PI * cos(M_PI * x[0]) * sin(M_PI * x[1]) * exp(x[2]);
    grad[1] = M_PI * sin(M_PI * x[0]) * cos(M_PI * x[1]) * exp(x[2]);
    grad[2] = u;
  } else {
    return 0.0;
  }
  return s * grad[k] - phi * u;
}

/* Coefficients at a point, for tests: out = (b0, b1, b2, c, f, g).        */
void orc_eval_coeffs(const orc_problem *P, const double *x, double *out) {
  double b[3];
  coef_drift(P, x, b);
  out[0] = b[0]; out[1] = b[1]; out[2] = b[2];
  out[3] = coef_c(P, x);
  out[4] = coef_f(P, x);
  out[5] = coef_g(P, x);
}

/* The same at n points x[n][3]: out[n][6].                                  */
void orc_eval_coeffs_many(const orc_problem *P, const double *x, int64_t n, double *out) {
  for (int64_t i = 0; i < n; ++i) orc_eval_coeffs(P, x + 3 * i, out + 6 * i);
}

/* ------------------------------------------------------------------------ */
/* Geometry.  Boxes [0,1]^d and the L-shape [0,1]^2 minus (1/2,1]x(1/2,1].  */
/* ------------------------------------------------------------------------ */
static int in_notch(const double *x) { return x[0] > 0.5 && x[1] > 0.5; }

static int inside_closed(int geom, int dim, const double *x) {
  for (int k = 0; k < dim; ++k)
    if (x[k] < 0.0 || x[k] > 1.0) return 0;
  if (geom == ORC_GEOM_L_SHAPE && in_notch(x)) return 0;
  return 1;
}

static int inside_open(int geom, int dim, const double *x) {
  for (int k = 0; k < dim; ++k)
    if (!(x[k] > 0.0 && x[k] < 1.0)) return 0;
  if (geom == ORC_GEOM_L_SHAPE && x[0] >= 0.5 && x[1] >= 0.5) return 0;
  return 1;
}

/* Faces.  Box: face 2k+s lies on x_k = s, inside is x_k > 0 (s=0) or
 * x_k < 1 (s=1).  L-shape: the four outer faces of the square plus the two
 * edges of the notch: face 4 on y = 1/2 (segment x in [1/2,1], inside y<1/2)
 * and face 5 on x = 1/2 (segment y in [1/2,1], inside x < 1/2).           */
static int n_faces(int geom, int dim) {
  return geom == ORC_GEOM_L_SHAPE ? 6 : 2 * dim;
}

/* Distance from x to the line/plane of face j, measured positive on the
 * domain side.  For the notch edges this is the distance to the edge segment
 * (Euclidean), so that points far from the segment see no crossing.       */
static double face_dist(int geom, int j, const double *x) {
  if (geom == ORC_GEOM_L_SHAPE && j >= 4) {
    double a, b; /* along-edge coordinate, normal distance */
    if (j == 4) { a = x[0]; b = 0.5 - x[1]; }
    else { a = x[1]; b = 0.5 - x[0]; }
    if (a >= 0.5) return b;
    double da = 0.5 - a;
    return sqrt(da * da + b * b);
  }
  int k = j >> 1, s = j & 1;
  return s ? 1.0 - x[k] : x[k];
}

/* Project x onto face j (set the face's coordinate to its value).          */
static void face_project(int geom, int j, double *x) {
  if (geom == ORC_GEOM_L_SHAPE && j >= 4) {
    if (j == 4) { x[1] = 0.5; if (x[0] < 0.5) x[0] = 0.5; }
    else { x[0] = 0.5; if (x[1] < 0.5) x[1] = 0.5; }
    return;
  }
  x[j >> 1] = (double)(j & 1);
}

/* First point where the straight segment x0 -> x1 leaves the closed domain,
 * given x0 inside and x1 outside.  The crossed coordinate is set exactly to
 * the face value.                                                          */
static void segment_exit(int geom, int dim, const double *x0, const double *x1,
                         double *xe) {
  double tbest = 2.0;
  int kbest = -1;
  double vbest = 0.0;
  for (int k = 0; k < dim; ++k) {
    if (x1[k] < 0.0) {
      double t = x0[k] / (x0[k] - x1[k]);
      if (t < tbest) { tbest = t; kbest = k; vbest = 0.0; }
    } else if (x1[k] > 1.0) {
      double t = (1.0 - x0[k]) / (x1[k] - x0[k]);
      if (t < tbest) { tbest = t; kbest = k; vbest = 1.0; }
    }
  }
  if (geom == ORC_GEOM_L_SHAPE) {
    /* Entry into the open notch {x > 1/2, y > 1/2}: for each axis the
     * parameter interval where that coordinate exceeds 1/2; the notch is
     * entered at the later of the two interval starts.                     */
    double lo = -1e300, hi = 1e300;
    int kent = -1;
    for (int k = 0; k < 2; ++k) {
      double a = x0[k], d = x1[k] - x0[k];
      double tl, th;
      if (d == 0.0) {
        if (a > 0.5) { tl = 0.0; th = 1.0; } else { tl = 2.0; th = -1.0; }
      } else if (d > 0.0) {
        tl = (0.5 - a) / d; th = 2.0;
      } else {
        tl = -1.0; th = (0.5 - a) / d;
      }
      if (tl > lo) { lo = tl; kent = k; }
      if (th < hi) hi = th;
    }
    if (kent >= 0 && lo < hi && lo <= 1.0 && hi > 0.0) {
      double tent = lo > 0.0 ? lo : 0.0;
      if (tent < tbest) { tbest = tent; kbest = kent; vbest = 0.5; }
    }
  }
  if (kbest < 0) { /* numerically degenerate: fall back to x1 clamped */
    for (int k = 0; k < dim; ++k) xe[k] = fmin(1.0, fmax(0.0, x1[k]));
    return;
  }
  for (int k = 0; k < dim; ++k) xe[k] = x0[k] + tbest * (x1[k] - x0[k]);
  xe[kbest] = vbest;
  for (int k = 0; k < dim; ++k) xe[k] = fmin(1.0, fmax(0.0, xe[k]));
}

/* Nearest face of x (used only for paths stopped by the step cap).        */
static int nearest_face(int geom, int dim, const double *x) {
  int jb = 0;
  double db = 1e300;
  for (int j = 0; j < n_faces(geom, dim); ++j) {
    double d = face_dist(geom, j, x);
    if (d < db) { db = d; jb = j; }
  }
  return jb;
}

/* ------------------------------------------------------------------------ */
/* One diffusion path (Eq. 2.8, Dirichlet/elliptic reduction).              */
/*                                                                          */
/* Stream layout: word k of path p of node i is word (k mod 4) of            */
/*   Philox4x32-10(key = (seed lo, seed hi), ctr = (k div 4, p, i, 0)).      */
/* Step n = 4q + j draws d normals xi_n and one uniform U_n from the twelve  */
/* words v0..v11 of blocks 3q, 3q+1, 3q+2:                                  */
/*   d = 1: xi = BM(v[2j], v[2j+1]).first,          U = v[8+j]               */
/*   d = 2: xi = BM(v[2j], v[2j+1]),                U = v[8+j]               */
/*   d = 3: normals z0..z11 = BM(v0,v1), ..., BM(v10,v11); xi = z[3j..3j+2], */
/*          U from the low bytes of v[3j], v[3j+1], v[3j+2]                  */
/*                                                                          */
/* Step n -> n+1 (left-point rule for Y and Z, Eq. 2.8):                     */
/*   X' = X + b(X) dt + sigma sqrt(dt) xi,  Y' = Y exp(c(X) dt),             */
/*   Z' = Z + f(X) Y dt.                                                    */
/* Exit at step n+1 if X' is outside the closed domain (exit point = first   */
/* crossing of the segment X -> X'), else, with the bridge test on, if       */
/* U < P = 1 - prod_j (1 - p_j), p_j = exp(-2 d_j d'_j / (sigma^2 dt)) over  */
/* faces with 2 d_j d'_j / (sigma^2 dt) < 18 (exit point = X' projected on   */
/* the face with the largest p_j).  Score = g(X_tau) Y' + Z'.                */
/* A node on the boundary exits at step 0 with score g(x).                  */
/* ------------------------------------------------------------------------ */
/* Number of linear boundary-data parameters (theta) and drift parameters
 * (phi) a family exposes to the derivative estimators.                     */
static int n_theta(const orc_problem *P) {
  return P->kind == ORC_PROB_POISSON_FOURIER ? 64 : P->kind == ORC_PROB_POLY1D ? 2 : 0;
}
static int n_phi(const orc_problem *P) {
  return P->kind == ORC_PROB_POISSON_FOURIER ? 16 : P->kind == ORC_PROB_POLY1D ? 2 : 0;
}

/* d b / d phi_j at x (a d-vector).  Poisson-Fourier: b_x = sum_j phi_j
 * sin(j pi y), b_y = sum_j phi_{8+j} sin(j pi x).  poly1d: b = b0 + b1 x.  */
static void drift_dphi(const orc_problem *P, int j, const double *x, double *db) {
  db[0] = db[1] = db[2] = 0.0;
  if (P->kind == ORC_PROB_POISSON_FOURIER) {
    if (j < 8) db[0] = sin((j + 1) * M_PI * x[1]);
    else db[1] = sin((j - 7) * M_PI * x[0]);
  } else if (P->kind == ORC_PROB_POLY1D) {
    db[0] = j == 0 ? 1.0 : x[0];
  }
}

/* d g / d theta_k at an exit point.  Poisson-Fourier: cos(m pi x) cos(n pi y)
 * with k = 8m + n.  poly1d: g = g0 at x = 0, g1 at x = 1.                  */
static double g_dtheta(const orc_problem *P, int k, const double *x) {
  if (P->kind == ORC_PROB_POISSON_FOURIER)
    return cos((k / 8) * M_PI * x[0]) * cos((k % 8) * M_PI * x[1]);
  if (P->kind == ORC_PROB_POLY1D) return (k == 0) == (x[0] < 0.5) ? 1.0 : 0.0;
  return 0.0;
}

static void simulate_path(const orc_problem *P, const orc_mc *M, uint32_t node,
                          uint32_t path, const double *x0, double *score,
                          int32_t *steps, double *xexit, double *Lphi,
                          double *yexit) {
  const int dim = P->dim, geom = P->geometry;
  const double dt = M->dt, sig = P->sigma;
  const double sdt = sig * sqrt(dt);
  const uint32_t key[2] = {(uint32_t)M->seed, (uint32_t)(M->seed >> 32)};
  double X[3] = {0, 0, 0}, Xn[3] = {0, 0, 0}, Y = 1.0, Z = 0.0;
  for (int k = 0; k < dim; ++k) X[k] = x0[k];
  const int nphi = n_phi(P);
  if (Lphi) for (int j = 0; j < nphi; ++j) Lphi[j] = 0.0;
  if (yexit) *yexit = 1.0;
  const int rmask = reflect_mask(P);
  const double phiR = rmask ? P->params[1] : 0.0;
  /* a start on an absorbing face exits at once; on a reflecting face the
   * walk starts normally */
  int on_abs = !inside_closed(geom, dim, X);
  for (int k = 0; k < dim && !on_abs; ++k)
    on_abs = (X[k] <= 0.0 && !((rmask >> (2 * k)) & 1)) ||
             (X[k] >= 1.0 && !((rmask >> (2 * k + 1)) & 1));
  if (geom == ORC_GEOM_L_SHAPE && !inside_open(geom, dim, X)) on_abs = 1;
  if (on_abs) {
    *score = coef_g(P, X);
    *steps = 0;
    if (xexit) for (int k = 0; k < 3; ++k) xexit[k] = X[k];
    return;
  }
  uint32_t W12[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  double N12[12];
  for (int64_t n = 0; n < M->max_steps; ++n) {
    double xi[3] = {0, 0, 0}, U;
    if (dim <= 2) {
      /* d = 1, 2: steps 4q .. 4q+3 use the 12 words w[0..11] of blocks 3q,
       * 3q+1, 3q+2; step 4q+j takes the normals BM(w[2j], w[2j+1]) (d = 1:
       * the first) and the uniform of w[8+j].                             */
      uint32_t q = (uint32_t)(n >> 2);
      int j = (int)(n & 3);
      if (j == 0) {
        for (int b = 0; b < 3; ++b) {
          uint32_t cb[4] = {3u * q + (uint32_t)b, path, node, 0u};
          orc_philox4x32_10(cb, key, W12 + 4 * b);
        }
      }
      double z0, z1;
      box_muller(W12[2 * j], W12[2 * j + 1], &z0, &z1);
      xi[0] = z0;
      if (dim == 2) xi[1] = z1;
      U = unif(W12[8 + j]);
    } else {
      /* d = 3: steps 4q .. 4q+3 use the 12 words w[0..11] of blocks 3q,
       * 3q+1, 3q+2; normals nrm[0..11] = Box-Muller of the word pairs
       * (w0,w1), ..., (w10,w11); step 4q+j takes nrm[3j..3j+2] and the
       * uniform of the word whose bytes 3, 2, 1 are the low bytes of
       * w[3j+2], w[3j+1], w[3j] (bits the Box-Muller maps do not use).   */
      uint32_t q = (uint32_t)(n >> 2);
      int j = (int)(n & 3);
      if (j == 0) {
        for (int b = 0; b < 3; ++b) {
          uint32_t cb[4] = {3u * q + (uint32_t)b, path, node, 0u};
          orc_philox4x32_10(cb, key, W12 + 4 * b);
        }
        for (int pr = 0; pr < 6; ++pr)
          box_muller(W12[2 * pr], W12[2 * pr + 1], &N12[2 * pr], &N12[2 * pr + 1]);
      }
      xi[0] = N12[3 * j]; xi[1] = N12[3 * j + 1]; xi[2] = N12[3 * j + 2];
      uint32_t wu = ((W12[3 * j + 2] & 255u) << 24) | ((W12[3 * j + 1] & 255u) << 16) |
                    ((W12[3 * j] & 255u) << 8);
      U = unif(wu);
    }
    double b[3];
    coef_drift(P, X, b);
    double c = coef_c(P, X), f = coef_f(P, X);
    if (Lphi) {
      /* Likelihood-ratio increment of the Gaussian transition density of
       * X' given X:  d/dphi_j log density = xi . db/dphi_j(X) sqrt(dt)/sigma */
      for (int j = 0; j < nphi; ++j) {
        double db[3];
        drift_dphi(P, j, X, db);
        double dot = 0.0;
        for (int k = 0; k < dim; ++k) dot += xi[k] * db[k];
        Lphi[j] += dot * sqrt(dt) / sig;
      }
    }
    for (int k = 0; k < dim; ++k) Xn[k] = X[k] + b[k] * dt + sdt * xi[k];
    /* Reflection (Lepingle's scheme for a half-space): on a reflecting face
     * j with distances y (start) and y' (free end), the Brownian bridge's
     * minimum over the step is m = (y + y' - sqrt((y' - y)^2 - 2 sigma^2 dt
     * ln U')) / 2 with U' uniform; the local time increment is L = max(0,
     * -m) and the end point is pushed in by L.  U' for axis k comes from the
     * tag-4 stream: word k of Philox((n, p, i, 4)) in 3-D, word
     * 2 (n mod 2) + k of Philox((n / 2, p, i, 4)) in 2-D (one block for two
     * steps); it matters only when 2 y y' / (sigma^2 dt) < 18
     * (else L = 0 for every U' >= 2^-24).  Along the local time the
     * weights solve dY = phi Y dxi, dZ = psi Y dxi exactly for psi frozen
     * at the end point projected on face j: Z gains psi Y (e^{phi L} - 1) /
     * phi (psi Y L when phi = 0) and Y gains the factor e^{phi L}; then
     * the time part, Y' = Y e^{c dt}, Z' = Z + f Y dt (left point).        */
    double yr = Y, zr = 0.0;
    if (rmask) {
      uint32_t R[4];
      int have_r = 0;
      for (int j = 0; j < 2 * dim; ++j) {
        if (!((rmask >> j) & 1)) continue;
        double y0 = face_dist(geom, j, X), y1 = face_dist(geom, j, Xn);
        if (2.0 * y0 * y1 / (sig * sig * dt) >= 18.0) continue;
        if (!have_r) {
          uint32_t blk = dim == 2 ? (uint32_t)(n / 2) : (uint32_t)n;
          uint32_t cr[4] = {blk, path, node, 4u};
          orc_philox4x32_10(cr, key, R);
          have_r = 1;
        }
        int k = j >> 1;
        int word = dim == 2 ? 2 * (int)(n % 2) + k : k;
        double dy = y1 - y0;
        double mn = 0.5 * (y0 + y1 - sqrt(dy * dy - 2.0 * sig * sig * dt * log(unif(R[word]))));
        double L = mn < 0.0 ? -mn : 0.0;
        if (L > 0.0) {
          if (j & 1) { Xn[k] -= L; if (Xn[k] > 1.0) Xn[k] = 1.0; }
          else { Xn[k] += L; if (Xn[k] < 0.0) Xn[k] = 0.0; }
          double xp[3] = {Xn[0], Xn[1], Xn[2]};
          xp[k] = (double)(j & 1);
          double g1 = phiR != 0.0 ? expm1(phiR * L) / phiR : L;
          zr += robin_psi(P, j, xp) * yr * g1;
          yr *= exp(phiR * L);
        }
      }
    }
    double Yn = yr * exp(c * dt);
    double Zn = Z + f * Y * dt + zr;
    if (!inside_closed(geom, dim, Xn)) {
      double xe[3] = {0, 0, 0};
      segment_exit(geom, dim, X, Xn, xe);
      *score = coef_g(P, xe) * Yn + Zn;
      *steps = (int32_t)(n + 1);
      if (xexit) for (int k = 0; k < 3; ++k) xexit[k] = xe[k];
      if (yexit) *yexit = Yn;
      return;
    }
    if (M->bridge) {
      double keep = 1.0, pbest = -1.0;
      int jbest = -1;
      for (int j = 0; j < n_faces(geom, dim); ++j) {
        if ((rmask >> j) & 1) continue; /* reflecting: no exit */
        double d0 = face_dist(geom, j, X), d1 = face_dist(geom, j, Xn);
        double a = 2.0 * d0 * d1 / (sig * sig * dt);
        if (a < 18.0) {
          double p = exp(-a);
          keep *= (1.0 - p);
          if (p > pbest) { pbest = p; jbest = j; }
        }
      }
      double Pexit = 1.0 - keep;
      if (jbest >= 0 && U < Pexit) {
        double xe[3] = {Xn[0], Xn[1], Xn[2]};
        face_project(geom, jbest, xe);
        *score = coef_g(P, xe) * Yn + Zn;
        *steps = (int32_t)(n + 1);
        if (xexit) for (int k = 0; k < 3; ++k) xexit[k] = xe[k];
        if (yexit) *yexit = Yn;
        return;
      }
    }
    for (int k = 0; k < dim; ++k) X[k] = Xn[k];
    Y = Yn;
    Z = Zn;
  }
  /* Step cap reached: score at the projection onto the nearest face.     */
  double xe[3] = {X[0], X[1], X[2]};
  int jn = -1;
  double dn = 1e300;
  for (int j = 0; j < n_faces(geom, dim); ++j) {
    if ((rmask >> j) & 1) continue;
    double d = face_dist(geom, j, X);
    if (d < dn) { dn = d; jn = j; }
  }
  if (jn >= 0) face_project(geom, jn, xe);
  *score = coef_g(P, xe) * Y + Z;
  *steps = (int32_t)(-M->max_steps);
  if (xexit) for (int k = 0; k < 3; ++k) xexit[k] = xe[k];
  if (yexit) *yexit = Y;
}

/* ------------------------------------------------------------------------ */
/* Thread pool over nodes (results do not depend on the thread count).     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int tid, nthreads;
  void (*fn)(void *ctx, int64_t i);
  void *ctx;
  int64_t n;
} worker_arg;

static void *worker_main(void *p) {
  worker_arg *w = (worker_arg *)p;
  for (int64_t i = w->tid; i < w->n; i += w->nthreads) w->fn(w->ctx, i);
  return NULL;
}

static void parallel_for(int64_t n, int nthreads, void (*fn)(void *, int64_t),
                         void *ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 512) nthreads = 512;
  if (nthreads == 1 || n <= 1) {
    for (int64_t i = 0; i < n; ++i) fn(ctx, i);
    return;
  }
  pthread_t th[512];
  worker_arg args[512];
  for (int t = 0; t < nthreads; ++t) {
    args[t].tid = t; args[t].nthreads = nthreads; args[t].fn = fn;
    args[t].ctx = ctx; args[t].n = n;
    pthread_create(&th[t], NULL, worker_main, &args[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Interface solve: per node, the sample mean and standard error of the     */
/* path scores (Welford's running mean / sum of squared deviations).        */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_problem *P;
  const orc_mc *M;
  const double *nodes;
  double *mean, *se;
  int64_t *npaths;
  double *path_score;
  int32_t *path_steps;
  double *path_exit;       /* [n][N][dim] exit points, or NULL */
  int64_t *steps_per_node, *capped_per_node;
  int64_t path_offset;
  const int64_t *node_ids; /* stream node index per node, or NULL (= i) */
} solve_ctx;

static void solve_node(void *vp, int64_t i) {
  solve_ctx *S = (solve_ctx *)vp;
  const int dim = S->P->dim;
  const int64_t N = S->M->n_paths;
  double mean = 0.0, m2 = 0.0;
  int64_t steps_total = 0, capped = 0;
  for (int64_t p = 0; p < N; ++p) {
    double s;
    int32_t st;
    uint32_t sid = (uint32_t)(S->node_ids ? S->node_ids[i] : i);
    double xe[3];
    simulate_path(S->P, S->M, sid, (uint32_t)(p + S->path_offset),
                  S->nodes + i * dim, &s, &st, xe, NULL, NULL);
    if (S->path_exit)
      for (int k = 0; k < dim; ++k) S->path_exit[(i * N + p) * dim + k] = xe[k];
    double delta = s - mean;
    mean += delta / (double)(p + 1);
    m2 += delta * (s - mean);
    if (st < 0) { capped++; steps_total += -st; } else steps_total += st;
    if (S->path_score) S->path_score[i * N + p] = s;
    if (S->path_steps) S->path_steps[i * N + p] = st;
  }
  S->mean[i] = mean;
  S->se[i] = N > 1 ? sqrt(m2 / (double)(N - 1) / (double)N) : 0.0;
  if (S->npaths) S->npaths[i] = N;
  S->steps_per_node[i] = steps_total;
  S->capped_per_node[i] = capped;
}

/* Returns 0 on success, 1 on invalid arguments.                            */
int orc_interface_solve(const orc_problem *P, const double *nodes, int64_t n,
                        const int64_t *node_ids, const orc_mc *M,
                        int64_t path_offset, double *mean,
                        double *se, int64_t *npaths, double *path_score,
                        int32_t *path_steps, double *path_exit,
                        int64_t *total_steps, int64_t *total_capped) {
  if (!P || !M || n < 0 || M->n_paths < 1 || M->dt <= 0.0 || P->dim < 1 ||
      P->dim > 3 || M->max_steps < 1)
    return 1;
  int64_t *spn = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int64_t *cpn = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  solve_ctx S = {P, M, nodes, mean, se, npaths, path_score, path_steps,
                 path_exit, spn, cpn, path_offset, node_ids};
  parallel_for(n, M->n_threads, solve_node, &S);
  int64_t ts = 0, tc = 0;
  for (int64_t i = 0; i < n; ++i) { ts += spn[i]; tc += cpn[i]; }
  if (total_steps) *total_steps = ts;
  if (total_capped) *total_capped = tc;
  free(spn);
  free(cpn);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Derivatives of the node estimate (families with parameters):             */
/*   J[i][k]         = E[dg/dtheta_k(X_tau) Y_tau]   k < n_theta            */
/*                     (exact pathwise: the paths do not depend on theta);  */
/*   J[i][n_theta+j] = E[s * L_j],  L_j = sum over the steps taken of       */
/*                     xi_n . db/dphi_j(X_n) sqrt(dt)/sigma                 */
/*                     (likelihood ratio of the discrete Gaussian transition */
/*                     kernel; the bridge uniform and the exit rule do not  */
/*                     depend on phi, so this is unbiased for the scheme).  */
/* Poisson-Fourier: theta = 64 Fourier weights of g, phi = 16 drift weights. */
/* poly1d: theta = (g0, g1), phi = (b0, b1).                                 */
/* The paths are the same streams as the interface solve.                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_problem *P;
  const orc_mc *M;
  const double *nodes;
  double *jac;    /* [n][W] */
  double *jac_se; /* [n][W] or NULL */
  double *rec;    /* [n][N][4 + n_phi]: s, exit point (3), L_j; or NULL */
  int32_t *steps; /* [n][N] or NULL */
} grad_ctx;

static void grad_node(void *vp, int64_t i) {
  grad_ctx *G = (grad_ctx *)vp;
  const orc_problem *P = G->P;
  const int nt = n_theta(P), np_ = n_phi(P), W = nt + np_;
  const int64_t N = G->M->n_paths;
  double mean[80], m2[80];
  for (int k = 0; k < W; ++k) mean[k] = m2[k] = 0.0;
  for (int64_t p = 0; p < N; ++p) {
    double s, xe[3], L[16], v[80], ye;
    int32_t st;
    simulate_path(P, G->M, (uint32_t)i, (uint32_t)p, G->nodes + i * P->dim, &s,
                  &st, xe, L, &ye);
    if (G->rec) {
      double *r = G->rec + ((size_t)i * (size_t)N + (size_t)p) * (size_t)(4 + np_);
      r[0] = s; r[1] = xe[0]; r[2] = xe[1]; r[3] = xe[2];
      for (int j = 0; j < np_; ++j) r[4 + j] = L[j];
    }
    if (G->steps) G->steps[i * N + p] = st;
    for (int k = 0; k < nt; ++k) v[k] = g_dtheta(P, k, xe) * ye;
    for (int j = 0; j < np_; ++j) v[nt + j] = s * L[j];
    for (int k = 0; k < W; ++k) {
      double d = v[k] - mean[k];
      mean[k] += d / (double)(p + 1);
      m2[k] += d * (v[k] - mean[k]);
    }
  }
  for (int k = 0; k < W; ++k) {
    G->jac[i * W + k] = mean[k];
    if (G->jac_se)
      G->jac_se[i * W + k] = N > 1 ? sqrt(m2[k] / (double)(N - 1) / (double)N) : 0.0;
  }
}

/* Width of a Jacobian row for this family (0: no parameters).             */
int orc_jacobian_width(const orc_problem *P) { return n_theta(P) + n_phi(P); }

int orc_interface_jacobian(const orc_problem *P, const double *nodes, int64_t n,
                           const orc_mc *M, double *jac, double *jac_se,
                           double *path_rec, int32_t *path_steps) {
  if (!P || !M || M->n_paths < 1 || n_theta(P) + n_phi(P) == 0 ||
      P->n_params < (P->kind == ORC_PROB_POISSON_FOURIER ? 80 : 7))
    return 1;
  grad_ctx G = {P, M, nodes, jac, jac_se, path_rec, path_steps};
  parallel_for(n, M->n_threads, grad_node, &G);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Branching Brownian motion for u_t = (1/2) Lap u + beta (sum_k alpha_k     */
/* u^k - u), u(.,0) = psi (Eq. 3.1 with L = (1/2) Lap, free space), and its  */
/* marked form (Sec. 3.2): particles live Exp(beta), move as independent     */
/* Brownian motions, and at death are replaced by k offspring drawn with     */
/* probability q_k, the tree weight being multiplied by alpha_k / q_k.  The  */
/* score of a tree is weight * prod over particles alive at time t of        */
/* psi(position).  u(x,t) = E[score] (Sec. 3.1.1; Algorithm 3.1 with         */
/* per-particle lifetimes, which is equal in law to its global clock by the  */
/* memoryless property).                                                    */
/*                                                                          */
/* params: [0] beta, [1] psi kind, [2] psi parameter, [3] K (max offspring  */
/*         count, <= 7), [4..4+K] q_0..q_K, [5+K..5+2K] alpha_0..alpha_K.   */
/* Tree order: depth-first; the root has id 0; when a particle branches     */
/* into k children they get ids next_id .. next_id+k-1 and the lowest id is */
/* processed first.  Particle id j of tree s at node i draws                */
/* w = Philox(key, (j, s, i, 1)): lifetime from w0, the Brownian increment   */
/* from BM(w1, w2), the offspring count from w3.                            */
/* A tree whose particle count exceeds max_particles or whose pending stack */
/* exceeds max_depth is discarded and counted (pruning, Algorithm 3.1).     */
/* ------------------------------------------------------------------------ */
static double psi_eval(int kind, double prm, const double *x, int dim) {
  switch (kind) {
  case ORC_PSI_CONST: return prm;
  case ORC_PSI_SIGMOID: return 1.0 / (1.0 + exp(-prm * x[0]));
  case ORC_PSI_TRAVELLING: {
    double e = 1.0 + exp(prm * x[0]);
    return 1.0 - 1.0 / (e * e);
  }
  case ORC_PSI_SINE: return sin(M_PI * x[0]) * (dim > 1 ? sin(M_PI * x[1]) : 1.0);
  default: return 0.0;
  }
}

typedef struct {
  const orc_problem *P;
  const orc_mc *M;
  const double *nodes_xt; /* [n][dim+1] */
  int64_t max_particles;
  int32_t max_depth;
  double *mean, *se;
  int64_t *n_kept, *n_discarded;
  double *tree_score;   /* [n*N] or NULL; NaN for discarded */
  int32_t *tree_segments; /* [n*N] or NULL; negative for discarded */
} branch_ctx;

typedef struct { double x[3]; double tb; uint32_t id; } particle;

static void branch_node(void *vp, int64_t i) {
  branch_ctx *C = (branch_ctx *)vp;
  const orc_problem *P = C->P;
  const int dim = P->dim;
  const double beta = P->params[0];
  const int psik = (int)P->params[1];
  const double psip = P->params[2];
  const int K = (int)P->params[3];
  const double *q = P->params + 4, *alpha = P->params + 5 + K;
  const double *xt = C->nodes_xt + i * (dim + 1);
  const double t = xt[dim];
  const uint32_t key[2] = {(uint32_t)C->M->seed, (uint32_t)(C->M->seed >> 32)};
  const int64_t N = C->M->n_paths;
  particle *stack = (particle *)malloc(sizeof(particle) * (size_t)(C->max_depth + 8));
  double mean = 0.0, m2 = 0.0;
  int64_t kept = 0, disc = 0;
  for (int64_t s = 0; s < N; ++s) {
    int sp = 0;
    particle root;
    for (int k = 0; k < 3; ++k) root.x[k] = k < dim ? xt[k] : 0.0;
    root.tb = 0.0;
    root.id = 0;
    stack[sp++] = root;
    uint32_t next_id = 1;
    int64_t particles = 1;
    int32_t segments = 0;
    double prod = 1.0, weight = 1.0;
    int bad = 0;
    while (sp > 0) {
      particle cur = stack[--sp];
      uint32_t ctr[4] = {cur.id, (uint32_t)s, (uint32_t)i, 1u};
      uint32_t w[4];
      orc_philox4x32_10(ctr, key, w);
      segments++;
      double life = -log(unif(w[0])) / beta;
      double tend = cur.tb + life;
      int reaches = tend >= t;
      if (reaches) tend = t;
      double z0, z1;
      box_muller(w[1], w[2], &z0, &z1);
      double h = sqrt(tend - cur.tb);
      cur.x[0] += h * z0;
      if (dim >= 2) cur.x[1] += h * z1;
      if (reaches) {
        prod *= psi_eval(psik, psip, cur.x, dim);
        continue;
      }
      double u3 = unif(w[3]), cum = 0.0;
      int k = K;
      for (int kk = 0; kk <= K; ++kk) {
        cum += q[kk];
        if (u3 < cum) { k = kk; break; }
      }
      weight *= alpha[k] / q[k];
      particles += k;
      if (particles > C->max_particles || sp + k > C->max_depth) { bad = 1; break; }
      for (int c = k - 1; c >= 0; --c) {
        particle ch = cur;
        ch.tb = tend;
        ch.id = next_id + (uint32_t)c;
        stack[sp++] = ch;
      }
      next_id += (uint32_t)k;
    }
    if (bad) {
      disc++;
      if (C->tree_score) C->tree_score[i * N + s] = NAN;
      if (C->tree_segments) C->tree_segments[i * N + s] = -segments;
      continue;
    }
    double sc = weight * prod;
    kept++;
    double d = sc - mean;
    mean += d / (double)kept;
    m2 += d * (sc - mean);
    if (C->tree_score) C->tree_score[i * N + s] = sc;
    if (C->tree_segments) C->tree_segments[i * N + s] = segments;
  }
  free(stack);
  C->mean[i] = mean;
  C->se[i] = kept > 1 ? sqrt(m2 / (double)(kept - 1) / (double)kept) : 0.0;
  C->n_kept[i] = kept;
  C->n_discarded[i] = disc;
}

int orc_branching_solve(const orc_problem *P, const double *nodes_xt, int64_t n,
                        const orc_mc *M, int64_t max_particles,
                        int32_t max_depth, double *mean, double *se,
                        int64_t *n_kept, int64_t *n_discarded,
                        double *tree_score, int32_t *tree_segments) {
  if (!P || P->kind != ORC_PROB_KPP || P->dim < 1 || P->dim > 2 || !M ||
      M->n_paths < 1 || P->n_params < 4)
    return 1;
  int K = (int)P->params[3];
  if (K < 0 || K > 7 || P->n_params < 6 + 2 * K || P->params[0] <= 0.0) return 1;
  branch_ctx C = {P, M, nodes_xt, max_particles, max_depth, mean, se,
                  n_kept, n_discarded, tree_score, tree_segments};
  parallel_for(n, M->n_threads, branch_node, &C);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Multilevel Monte Carlo for the interface estimate (Sec. 2.1 names Giles'  */
/* multilevel method as the next acceleration of the Euler scheme):          */
/*   E[P_L] = E[P_0] + sum_{l=1..L} E[P_l - P_{l-1}],                       */
/* P_l the score of the Euler-Maruyama path with step dt_l = dt_0 / R^l     */
/* (R = refine).  Level l >= 1 samples a coupled pair: the fine path with   */
/* dt_l and the coarse path with dt_{l-1} driven by the same Brownian       */
/* motion, the coarse increment being the sum of the R fine ones; each path */
/* stops at its own exit (hard exit or the half-space bridge test of the    */
/* linear paths) and the pair is done when both are.  Fine step k of sample */
/* p at node i reads Philox(key, (k, p, i, 16 + l)): normals BM(w0, w1),    */
/* bridge uniform U(w2); the coarse step that closes a group of R fine       */
/* steps takes the uniform of the group's last fine step (independent of   */
/* every normal, so each path has the law of the plain scheme at its step;   */
/* the pair shares it to couple the exit decisions).  Level 0 is the plain  */
/* scheme with step dt_0 on tag 16.  Dimensions 1 and 2, Dirichlet data.    */
/* ------------------------------------------------------------------------ */
typedef struct {
  double X[3], Y, Z;
  int done;
  double score;
  double xe[3];  /* exit point, set when the walk ends */
} mlmc_walk;

/* One Euler-Maruyama step of a walk with time step dt and Brownian increment
 * dW (already scaled), exit tests with the bridge uniform U (left point for
 * Y and Z, exit at the end of the step).                                  */
static void mlmc_step(const orc_problem *P, const orc_mc *M, double dt, const double *dW,
                      double U, mlmc_walk *w) {
  const int dim = P->dim, geom = P->geometry;
  const double sig = P->sigma;
  double b[3];
  coef_drift(P, w->X, b);
  const double c = coef_c(P, w->X), f = coef_f(P, w->X);
  double Xn[3] = {0, 0, 0};
  for (int k = 0; k < dim; ++k) Xn[k] = w->X[k] + b[k] * dt + sig * dW[k];
  const double Yn = w->Y * exp(c * dt);
  const double Zn = w->Z + f * w->Y * dt;
  if (!inside_closed(geom, dim, Xn)) {
    double xe[3] = {0, 0, 0};
    segment_exit(geom, dim, w->X, Xn, xe);
    w->score = coef_g(P, xe) * Yn + Zn;
    for (int k = 0; k < 3; ++k) w->xe[k] = xe[k];
    w->done = 1;
    return;
  }
  if (M->bridge) {
    double keep = 1.0, pbest = -1.0;
    int jbest = -1;
    for (int j = 0; j < n_faces(geom, dim); ++j) {
      double a = 2.0 * face_dist(geom, j, w->X) * face_dist(geom, j, Xn) / (sig * sig * dt);
      if (a < 18.0) {
        double p = exp(-a);
        keep *= 1.0 - p;
        if (p > pbest) { pbest = p; jbest = j; }
      }
    }
    if (jbest >= 0 && U < 1.0 - keep) {
      double xe[3] = {Xn[0], Xn[1], Xn[2]};
      face_project(geom, jbest, xe);
      w->score = coef_g(P, xe) * Yn + Zn;
      for (int k = 0; k < 3; ++k) w->xe[k] = xe[k];
      w->done = 1;
      return;
    }
  }
  for (int k = 0; k < dim; ++k) w->X[k] = Xn[k];
  w->Y = Yn;
  w->Z = Zn;
}

static void mlmc_cap(const orc_problem *P, mlmc_walk *w) {
  double xe[3] = {w->X[0], w->X[1], w->X[2]};
  face_project(P->geometry, nearest_face(P->geometry, P->dim, w->X), xe);
  w->score = coef_g(P, xe) * w->Y + w->Z;
  for (int k = 0; k < 3; ++k) w->xe[k] = xe[k];
  w->done = 1;
}

typedef struct {
  const orc_problem *P;
  const orc_mc *M;
  const double *nodes;
  int level, refine;
  double *mean, *var, *fine_mean, *coarse_mean, *path_diff;
  int32_t *path_steps;
  int64_t *capped;
  double *path_aux;  /* [n][N][8] per-walk records (scores, exit steps, exit points), or NULL */
} mlmc_ctx;

static void mlmc_node(void *vp, int64_t i) {
  mlmc_ctx *C = (mlmc_ctx *)vp;
  const orc_problem *P = C->P;
  const orc_mc *M = C->M;
  const int dim = P->dim, l = C->level, R = C->refine;
  const double dtf = M->dt / pow((double)R, (double)l);
  const double sdf = sqrt(dtf);
  const uint32_t key[2] = {(uint32_t)M->seed, (uint32_t)(M->seed >> 32)};
  const int64_t N = M->n_paths;
  double m = 0.0, m2 = 0.0, mf = 0.0, mc = 0.0;
  int64_t caps = 0;
  for (int64_t p = 0; p < N; ++p) {
    mlmc_walk fw, cw;
    memset(&fw, 0, sizeof fw);
    for (int k = 0; k < dim; ++k) fw.X[k] = fw.xe[k] = C->nodes[i * dim + k];
    fw.Y = 1.0;
    cw = fw;
    if (!inside_open(P->geometry, dim, fw.X)) {
      fw.score = cw.score = coef_g(P, fw.X);
      fw.done = cw.done = 1;
    }
    if (l == 0) cw.done = 1;
    double dWc[3] = {0, 0, 0};
    int64_t k = 0, kf = 0, kc = 0;  /* fine steps; exit steps of the two walks */
    while (!(fw.done && cw.done) && k < M->max_steps) {
      uint32_t ctr[4] = {(uint32_t)k, (uint32_t)p, (uint32_t)i, 16u + (uint32_t)l}, w[4];
      orc_philox4x32_10(ctr, key, w);
      double z0, z1;
      box_muller(w[0], w[1], &z0, &z1);
      const double dW[3] = {sdf * z0, dim > 1 ? sdf * z1 : 0.0, 0.0};
      const double U = unif(w[2]);
      if (!fw.done) {
        mlmc_step(P, M, dtf, dW, U, &fw);
        if (fw.done) kf = k + 1;
      }
      for (int d = 0; d < dim; ++d) dWc[d] += dW[d];
      ++k;
      if (l > 0 && k % R == 0) {
        if (!cw.done) {
          mlmc_step(P, M, dtf * R, dWc, U, &cw);
          if (cw.done) kc = k / R;
        }
        dWc[0] = dWc[1] = dWc[2] = 0.0;
      }
    }
    if (!fw.done) { mlmc_cap(P, &fw); kf = -k; ++caps; }
    if (l > 0 && !cw.done) { mlmc_cap(P, &cw); kc = -(k / R); ++caps; }
    if (C->path_aux) {
      double *o = C->path_aux + (i * N + p) * 8;
      o[0] = fw.score;
      o[1] = l > 0 ? cw.score : 0.0;
      o[2] = (double)kf;
      o[3] = l > 0 ? (double)kc : 0.0;
      o[4] = fw.xe[0];
      o[5] = dim > 1 ? fw.xe[1] : 0.0;
      o[6] = l > 0 ? cw.xe[0] : 0.0;
      o[7] = l > 0 && dim > 1 ? cw.xe[1] : 0.0;
    }
    const double y = l > 0 ? fw.score - cw.score : fw.score;
    const double d = y - m;
    m += d / (double)(p + 1);
    m2 += d * (y - m);
    mf += (fw.score - mf) / (double)(p + 1);
    if (l > 0) mc += (cw.score - mc) / (double)(p + 1);
    if (C->path_diff) C->path_diff[i * N + p] = y;
    if (C->path_steps) C->path_steps[i * N + p] = (int32_t)k;
  }
  C->mean[i] = m;
  C->var[i] = N > 1 ? m2 / (double)(N - 1) : 0.0;
  if (C->fine_mean) C->fine_mean[i] = mf;
  if (C->coarse_mean) C->coarse_mean[i] = mc;
  C->capped[i] = caps;
}

int orc_mlmc_level(const orc_problem *P, const double *nodes, int64_t n, const orc_mc *M,
                   int32_t level, int32_t refine, double *mean, double *var,
                   double *fine_mean, double *coarse_mean, double *path_diff,
                   int32_t *path_steps, int64_t *total_capped, double *path_aux) {
  if (!P || !M || n < 0 || M->n_paths < 1 || !(M->dt > 0.0) || P->dim < 1 || P->dim > 2 ||
      M->max_steps < 1 || level < 0 || level > 12 || refine < 2 || refine > 16)
    return 1;
  int64_t *cap = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  mlmc_ctx C = {P, M, nodes, level, refine, mean, var, fine_mean, coarse_mean,
                path_diff, path_steps, cap, path_aux};
  parallel_for(n, M->n_threads, mlmc_node, &C);
  int64_t tc = 0;
  for (int64_t i = 0; i < n; ++i) tc += cap[i];
  if (total_capped) *total_capped = tc;
  free(cap);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Branching Brownian motion on a time grid, with absorbing boundaries       */
/* (Eq. 3.2) and one tree per node for every time point (Algorithm 3.1).     */
/*                                                                          */
/* u(x, t) = E[ prod over the particles of the tree run for a time t of     */
/*   psi(X_t) if the particle is alive at t, or g(X_tau, t - tau) if it     */
/*   hit the boundary at tau <= t ]  (Eq. 3.2; alpha_k / q_k weights of      */
/*   Sec. 3.2 for branchings before t).                                     */
/* The tree restricted to [0, T_i] is a tree run for a time T_i, so one tree */
/* scores every T_i of the grid (Algorithm 3.1 evaluates the particles      */
/* alive at each T_i).  Free space: no boundary, and Brownian increments    */
/* are exact, so a particle moves in one piece between grid times.  Boxes   */
/* and the L-shape: the particle moves in steps of at most dt, each with    */
/* the exit test of the linear paths (hard exit at the segment crossing,    */
/* else the half-space bridge probability over faces with a < 18; exit at  */
/* the end of the step).                                                    */
/*                                                                          */
/* Boundary data g(x, s) by the psi kind (the exact solution of the         */
/* unbounded problem where there is one): const c -> the solution of         */
/* v' = beta (v^2 - v), v(0) = c, i.e. c / (c + (1 - c) e^{beta s});        */
/* sigmoid -> psi(x); travelling (parameter a) -> 1 - (1 + e^{a x1 - 5 beta */
/* s / 6})^-2, the travelling wave of u_t = (1/2) u'' + beta (u^2 - u) when  */
/* a = sqrt(beta / 3); sine -> 0.                                           */
/*                                                                          */
/* Times are integers ("ticks") of 2^-k with k = 31 - e, T_m = f 2^e,        */
/* f in [1/2, 1): T_i -> floor(T_i 2^k + 1/2), dt -> max(1, floor(dt 2^k +  */
/* 1/2)), a lifetime E -> floor(E 2^k) (capped at 2^32 - 1).  A particle     */
/* born at tick b with lifetime ticks e lives to min(b + e, T_m); its walk   */
/* is cut at every grid time and at most dt apart.  Streams: particle id of */
/* tree s at node i draws block j from Philox(key, ((id << 20) | j, s, i,   */
/* 3)); j = 0: lifetime -ln U(w0) / beta, offspring count from U(w3) by the */
/* inverse CDF of q; j >= 1: step j, normals BM(w0, w1), bridge U(w2).       */
/* Order and pruning as for the free-space trees.                           */
/* ------------------------------------------------------------------------ */
static double g_bound(int kind, double prm, double beta, const double *x, double s,
                      int dim) {
  switch (kind) {
  case ORC_PSI_CONST: return prm / (prm + (1.0 - prm) * exp(beta * s));
  case ORC_PSI_SIGMOID: return psi_eval(kind, prm, x, dim);
  case ORC_PSI_TRAVELLING: {
    double e = 1.0 + exp(prm * x[0] - 5.0 * beta * s / 6.0);
    return 1.0 - 1.0 / (e * e);
  }
  default: return 0.0;
  }
}

typedef struct {
  const orc_problem *P;
  const orc_mc *M;
  const double *nodes; /* [n][dim] */
  const uint32_t *T;   /* [m] ticks */
  int m;
  uint32_t dt_ticks;
  double tps;          /* ticks per unit time, 2^k */
  int64_t max_particles;
  int32_t max_depth;
  double *mean, *se;   /* [n][m] */
  int64_t *n_kept, *n_discarded;
  double *tree_score;  /* [n][N][m] or NULL */
  int32_t *tree_steps; /* [n][N] or NULL */
} gbranch_ctx;

typedef struct { double x[2]; uint32_t tb; uint32_t id; } gparticle;

static void gbranch_node(void *vp, int64_t i) {
  gbranch_ctx *C = (gbranch_ctx *)vp;
  const orc_problem *P = C->P;
  const int dim = P->dim, geom = P->geometry, m = C->m;
  const int bounded = geom != ORC_GEOM_FREE_SPACE;
  const double beta = P->params[0];
  const int psik = (int)P->params[1];
  const double psip = P->params[2];
  const int K = (int)P->params[3];
  const double *q = P->params + 4, *alpha = P->params + 5 + K;
  const uint32_t key[2] = {(uint32_t)C->M->seed, (uint32_t)(C->M->seed >> 32)};
  const int64_t N = C->M->n_paths;
  const uint32_t Tm = C->T[m - 1];
  gparticle *stack = (gparticle *)malloc(sizeof(gparticle) * (size_t)(C->max_depth + 8));
  double *prod = (double *)malloc(sizeof(double) * (size_t)m);
  double *mean = C->mean + i * m, *m2 = (double *)calloc((size_t)m, sizeof(double));
  for (int k = 0; k < m; ++k) mean[k] = 0.0;
  int64_t kept = 0, disc = 0;
  for (int64_t s = 0; s < N; ++s) {
    for (int k = 0; k < m; ++k) prod[k] = 1.0;
    int sp = 0, bad = 0;
    gparticle root;
    root.x[0] = C->nodes[i * dim];
    root.x[1] = dim > 1 ? C->nodes[i * dim + 1] : 0.0;
    root.tb = 0;
    root.id = 0;
    stack[sp++] = root;
    uint32_t next_id = 1;
    int64_t particles = 1;
    int32_t steps = 0;
    if (bounded && !inside_open(geom, dim, root.x)) {
      /* on the boundary: absorbed at time 0 */
      for (int k = 0; k < m; ++k)
        prod[k] = g_bound(psik, psip, beta, root.x, C->T[k] / C->tps, dim);
      sp = 0;
    }
    while (sp > 0) {
      gparticle cur = stack[--sp];
      uint32_t w[4];
      uint32_t ctr[4] = {(cur.id << 20), (uint32_t)s, (uint32_t)i, 3u};
      orc_philox4x32_10(ctr, key, w);
      double life = -log(unif(w[0])) / beta;
      double lt = life * C->tps;
      uint64_t e = lt >= 4294967295.0 ? 4294967295ull : (uint64_t)lt;
      uint64_t tend64 = (uint64_t)cur.tb + e;
      uint32_t tend = tend64 < Tm ? (uint32_t)tend64 : Tm;
      int ti = 0;
      while (ti < m && C->T[ti] <= cur.tb) ++ti;
      uint32_t t = cur.tb, j = 1;
      double X[2] = {cur.x[0], cur.x[1]};
      int exited = 0;
      while (t < tend) {
        uint32_t nxt = tend;
        if (ti < m && C->T[ti] < nxt) nxt = C->T[ti];
        if (bounded && nxt - t > C->dt_ticks) nxt = t + C->dt_ticks;
        double h = (double)(nxt - t) / C->tps;
        uint32_t cj[4] = {(cur.id << 20) | j, (uint32_t)s, (uint32_t)i, 3u};
        uint32_t v[4];
        orc_philox4x32_10(cj, key, v);
        ++j;
        ++steps;
        double z0, z1;
        box_muller(v[0], v[1], &z0, &z1);
        double Xn[3] = {X[0] + sqrt(h) * z0, dim > 1 ? X[1] + sqrt(h) * z1 : 0.0, 0.0};
        if (bounded) {
          double xe[3] = {0, 0, 0};
          int out = 0;
          double X3[3] = {X[0], X[1], 0.0};
          if (!inside_closed(geom, dim, Xn)) {
            segment_exit(geom, dim, X3, Xn, xe);
            out = 1;
          } else if (C->M->bridge) {
            double keep = 1.0, pbest = -1.0;
            int jbest = -1;
            for (int f = 0; f < n_faces(geom, dim); ++f) {
              double a = 2.0 * face_dist(geom, f, X3) * face_dist(geom, f, Xn) / h;
              if (a < 18.0) {
                double p = exp(-a);
                keep *= 1.0 - p;
                if (p > pbest) { pbest = p; jbest = f; }
              }
            }
            if (jbest >= 0 && unif(v[2]) < 1.0 - keep) {
              for (int k = 0; k < 3; ++k) xe[k] = Xn[k];
              face_project(geom, jbest, xe);
              out = 1;
            }
          }
          if (out) {
            /* absorbed at the end of the step: every later grid time sees g */
            for (int k = ti; k < m; ++k)
              prod[k] *= g_bound(psik, psip, beta, xe, (double)(C->T[k] - nxt) / C->tps, dim);
            exited = 1;
            break;
          }
        }
        X[0] = Xn[0];
        X[1] = Xn[1];
        t = nxt;
        if (ti < m && t == C->T[ti]) {
          prod[ti] *= psi_eval(psik, psip, X, dim);
          ++ti;
        }
      }
      if (exited || tend == Tm) continue;
      /* lifetime over before T_m: branch */
      double u3 = unif(w[3]), cum = 0.0;
      int k = K;
      for (int kk = 0; kk <= K; ++kk) {
        cum += q[kk];
        if (u3 < cum) { k = kk; break; }
      }
      double r = alpha[k] / q[k];
      for (int kk = ti; kk < m; ++kk) prod[kk] *= r;
      particles += k;
      if (particles > C->max_particles || sp + k > C->max_depth) { bad = 1; break; }
      for (int c = k - 1; c >= 0; --c) {
        gparticle ch;
        ch.x[0] = X[0];
        ch.x[1] = X[1];
        ch.tb = tend;
        ch.id = next_id + (uint32_t)c;
        stack[sp++] = ch;
      }
      next_id += (uint32_t)k;
    }
    if (C->tree_steps) C->tree_steps[i * N + s] = bad ? -steps : steps;
    if (bad) {
      disc++;
      if (C->tree_score)
        for (int k = 0; k < m; ++k) C->tree_score[(i * N + s) * m + k] = NAN;
      continue;
    }
    kept++;
    for (int k = 0; k < m; ++k) {
      double d = prod[k] - mean[k];
      mean[k] += d / (double)kept;
      m2[k] += d * (prod[k] - mean[k]);
      if (C->tree_score) C->tree_score[(i * N + s) * m + k] = prod[k];
    }
  }
  for (int k = 0; k < m; ++k)
    C->se[i * m + k] = kept > 1 ? sqrt(m2[k] / (double)(kept - 1) / (double)kept) : 0.0;
  C->n_kept[i] = kept;
  C->n_discarded[i] = disc;
  free(stack);
  free(prod);
  free(m2);
}

/* Tick scale for a grid ending at T_m: 2^k with k = 31 - e, T_m = f 2^e.    */
double orc_grid_ticks_per_unit(double Tm) {
  int e = 0;
  frexp(Tm, &e);
  return ldexp(1.0, 31 - e);
}

int orc_branching_grid_solve(const orc_problem *P, const double *nodes, int64_t n,
                             const double *times, int32_t m, const orc_mc *M,
                             int64_t max_particles, int32_t max_depth, double *mean,
                             double *se, int64_t *n_kept, int64_t *n_discarded,
                             double *tree_score, int32_t *tree_steps) {
  if (!P || P->kind != ORC_PROB_KPP || P->dim < 1 || P->dim > 2 || !M ||
      M->n_paths < 1 || P->n_params < 4 || m < 1 || m > 32)
    return 1;
  int K = (int)P->params[3];
  if (K < 0 || K > 7 || P->n_params < 6 + 2 * K || P->params[0] <= 0.0) return 1;
  if (max_particles < 1 || max_particles > 4096) return 1;
  for (int k = 0; k < m; ++k)
    if (!(times[k] > 0.0) || (k > 0 && !(times[k] > times[k - 1]))) return 1;
  const int bounded = P->geometry != ORC_GEOM_FREE_SPACE;
  double tps = orc_grid_ticks_per_unit(times[m - 1]);
  uint32_t *T = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m);
  for (int k = 0; k < m; ++k) T[k] = (uint32_t)floor(times[k] * tps + 0.5);
  double dtt = bounded ? floor(M->dt * tps + 0.5) : 4294967295.0;
  uint32_t dt_ticks = dtt < 1.0 ? 1u : dtt > 4294967295.0 ? 4294967295u : (uint32_t)dtt;
  int ok = 1;
  for (int k = 1; k < m; ++k) ok = ok && T[k] > T[k - 1];
  /* at most 2^20 - 1 step blocks per particle */
  if (bounded && (double)T[m - 1] / dt_ticks + m + 2 > 1048575.0) ok = 0;
  for (int64_t i = 0; ok && bounded && i < n; ++i) {
    double x[3] = {nodes[i * P->dim], P->dim > 1 ? nodes[i * P->dim + 1] : 0.0, 0.0};
    if (!inside_closed(P->geometry, P->dim, x)) ok = 0;
  }
  if (!ok) { free(T); return 1; }
  gbranch_ctx C = {P, M, nodes, T, m, dt_ticks, tps, max_particles, max_depth,
                   mean, se, n_kept, n_discarded, tree_score, tree_steps};
  parallel_for(n, M->n_threads, gbranch_node, &C);
  free(T);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Walk on Spheres for the Laplace problem Eq. 1.1 (Sec. 2.1 names it as the */
/* scheme to use for stopped Brownian motion): from x, jump to a uniform     */
/* point on the circle of radius d(x) = distance to the boundary (the       */
/* largest circle inside the domain); stop when d(x) <= eps and score g at   */
/* the projection of x on the nearest face.  E[g(X_stop)] -> u(x) as        */
/* eps -> 0 (bias O(eps)), with no time-step bias.  d(x) = min over faces of */
/* face_dist, which never exceeds the true distance to the boundary (outer  */
/* faces are treated as full lines).  Step n of path p at node i takes the  */
/* angle 2 pi U, U = unif(word n mod 4 of Philox(key, (n div 4, p, i, 2))). */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_problem *P;
  const orc_mc *M;
  const double *nodes;
  const int64_t *node_ids;
  double eps;
  double *mean, *se;
  int64_t *npaths;
  double *path_score;
  int32_t *path_steps;
  int64_t *steps_per_node;
  double *path_exit;  /* [n][N][2] stopping points (projected), or NULL */
} wos_ctx;

static void wos_node(void *vp, int64_t i) {
  wos_ctx *W = (wos_ctx *)vp;
  const orc_problem *P = W->P;
  const int geom = P->geometry, dim = P->dim;
  const int64_t N = W->M->n_paths;
  const uint32_t key[2] = {(uint32_t)W->M->seed, (uint32_t)(W->M->seed >> 32)};
  const uint32_t sid = (uint32_t)(W->node_ids ? W->node_ids[i] : i);
  double mean = 0.0, m2 = 0.0;
  int64_t steps_total = 0;
  for (int64_t p = 0; p < N; ++p) {
    double X[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) X[k] = W->nodes[i * dim + k];
    uint32_t blk[4] = {0, 0, 0, 0};
    int64_t n = 0;
    for (;;) {
      int jb = nearest_face(geom, dim, X);
      double d = face_dist(geom, jb, X);
      if (d <= W->eps || n >= W->M->max_steps) {
        face_project(geom, jb, X);
        break;
      }
      if ((n & 3) == 0) {
        uint32_t ctr[4] = {(uint32_t)(n >> 2), (uint32_t)p, sid, 2u};
        orc_philox4x32_10(ctr, key, blk);
      }
      double th = 2.0 * M_PI * unif(blk[n & 3]);
      X[0] += d * cos(th);
      X[1] += d * sin(th);
      ++n;
    }
    double sc = coef_g(P, X);
    double delta = sc - mean;
    mean += delta / (double)(p + 1);
    m2 += delta * (sc - mean);
    steps_total += n;
    if (W->path_score) W->path_score[i * N + p] = sc;
    if (W->path_steps) W->path_steps[i * N + p] = (int32_t)n;
    if (W->path_exit) {
      W->path_exit[(i * N + p) * 2] = X[0];
      W->path_exit[(i * N + p) * 2 + 1] = X[1];
    }
  }
  W->mean[i] = mean;
  W->se[i] = N > 1 ? sqrt(m2 / (double)(N - 1) / (double)N) : 0.0;
  if (W->npaths) W->npaths[i] = N;
  W->steps_per_node[i] = steps_total;
}

int orc_wos_solve(const orc_problem *P, const double *nodes, int64_t n,
                  const int64_t *node_ids, const orc_mc *M, double eps,
                  double *mean, double *se, int64_t *npaths, double *path_score,
                  int32_t *path_steps, int64_t *total_steps, double *path_exit) {
  if (!P || P->kind != ORC_PROB_LAPLACE_EXPCOS || P->dim != 2 || !M ||
      M->n_paths < 1 || !(eps > 0.0))
    return 1;
  int64_t *spn = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  wos_ctx W = {P,          M,          nodes, node_ids, eps, mean, se, npaths,
               path_score, path_steps, spn,   path_exit};
  parallel_for(n, M->n_threads, wos_node, &W);
  int64_t ts = 0;
  for (int64_t i = 0; i < n; ++i) ts += spn[i];
  if (total_steps) *total_steps = ts;
  free(spn);
  return 0;
}
