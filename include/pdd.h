/*
 * pdd.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot path
 * of Probabilistic Domain Decomposition (PDD; Bernal, dos Reis, Smith,
 * arXiv:1705.03666): Monte Carlo Feynman-Kac estimates of a PDE solution at
 * interface nodes (stage one of PDD, Sec. 2 and Fig. 2.2), the branching
 * representation of semilinear problems (Sec. 3), and the deterministic
 * stage two (interface interpolation and independent subdomain solves,
 * Sec. 2.1).
 *
 * Conventions shared by every entry point:
 *  - Pointers named d_* are DEVICE pointers on the context's device, owned by
 *    the caller, contiguous, little-endian, row-major.  Host pointers are
 *    named without the prefix.  Nothing is retained after a call returns.
 *  - All device work is enqueued on the context's CUDA stream; calls return
 *    after enqueueing, except where a host-side output (pdd_diag counters,
 *    iteration counts) is requested, in which case the call synchronises the
 *    stream before returning.
 *  - Errors are returned as pdd_status, never thrown, trapped or printed;
 *    pdd_last_error() gives a one-line description of the last failure on a
 *    context.  PDD_ECAP is non-fatal: results are valid, but some paths or
 *    trees hit a cap and were counted (see pdd_diag).
 *  - Same inputs (seed, nodes, parameters) give bitwise-identical outputs:
 *    random numbers are counter-based (Philox4x32-10) and every reduction has
 *    a fixed order.
 *  - A context is bound to one device and one stream and is not thread-safe.
 *    The library owns the context and its device scratch (grown on demand,
 *    freed by pdd_destroy).
 */
#ifndef PDD_H
#define PDD_H

#include <stdint.h>

#if defined(__GNUC__)
#define PDD_API __attribute__((visibility("default")))
#else
#define PDD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PDD_OK = 0,
  PDD_EINVAL = 1,   /* invalid argument (sizes, NaN parameters, null pointers) */
  PDD_ENOMEM = 2,   /* device allocation failed */
  PDD_ECUDA = 3,    /* a CUDA runtime call failed (message in pdd_last_error) */
  PDD_ETIMEOUT = 4, /* a bounded device loop ran out of iterations */
  PDD_ECAP = 5      /* non-fatal: some paths/trees were capped and counted */
} pdd_status;

/* Domains.  Boxes are [0,1]^d; the L-shape is [0,1]^2 minus (1/2,1]x(1/2,1]. */
enum {
  PDD_GEOM_INTERVAL = 0,
  PDD_GEOM_UNIT_SQUARE = 1,
  PDD_GEOM_L_SHAPE = 2,
  PDD_GEOM_UNIT_CUBE = 3,
  PDD_GEOM_FREE_SPACE = 4
};

/* PDE families, written in the paper's elliptic form (Eq. 2.3-2.4 with the
 * time dependence dropped, Sec. 2.2):
 *   (1/2) sigma^2 Lap u + b . grad u + c u + f = 0 in Omega, u = g on dOmega.
 * LAPLACE_EXPCOS          Eq. 1.1 with g = e^x cos y (harmonic), d = 2, on the
 *                         unit square or the L-shape.
 * ELLIPTIC_MANUFACTURED   d = 3, b = (0.5 sin 2 pi y, 0.5 cos 2 pi x, 0),
 *                         c = -1, f chosen so that u = sin(pi x) sin(pi y) e^z,
 *                         g = u on the boundary.
 * POISSON_FOURIER         d = 2, f = 1, c = 0, params = theta[64] then phi[16]:
 *                         g = sum_{m,n<8} theta[8m+n] cos(m pi x) cos(n pi y),
 *                         b = (sum_j phi[j-1] sin(j pi y),
 *                              sum_j phi[7+j] sin(j pi x)), j = 1..8.
 * KPP                     u_t = (1/2) Lap u + beta (sum_k alpha_k u^k - u),
 *                         u(.,0) = psi, d = 1 or 2, free space (Eq. 3.1 and
 *                         Sec. 3.2) or, for pdd_branching_grid_solve, the
 *                         interval / unit square / L-shape with absorbing
 *                         boundaries (Eq. 3.2).  params: [0] beta, [1] psi
 *                         kind (0 const, 1 sigmoid 1/(1+e^{-a x1}), 2
 *                         travelling 1-(1+e^{a x1})^-2, 3 sine
 *                         prod_k sin(pi x_k)), [2] psi parameter (c or a),
 *                         [3] K = max offspring count (<= 7), [4..4+K] q_k
 *                         (sampling law), [5+K..5+2K] alpha_k.            */
enum {
  PDD_PROB_LAPLACE_EXPCOS = 1,
  PDD_PROB_ELLIPTIC_MANUFACTURED = 2,
  PDD_PROB_POISSON_FOURIER = 3,
  PDD_PROB_KPP = 7
};

/* Arithmetic of the per-step path state. */
enum { PDD_FP32 = 0, PDD_FP64 = 1 };

typedef struct {
  int32_t kind;          /* PDD_PROB_* */
  int32_t geometry;      /* PDD_GEOM_* */
  int32_t dim;           /* spatial dimension d */
  int32_t n_params;      /* length of params */
  const double *params;  /* host; copied by pdd_create */
  double sigma;          /* generator (1/2) sigma^2 Lap + b . grad (sigma > 0) */
} pdd_problem;

typedef struct {
  uint64_t seed;         /* Philox key */
  double dt;             /* Euler-Maruyama time step (> 0, sigma^2 dt <= 1/36) */
  int64_t n_paths;       /* paths per node (>= 1) */
  int64_t max_steps;     /* per-path step cap (>= 1, <= 2^31-1); capped paths
                            are scored at the nearest face and counted */
  int64_t path_offset;   /* index of the first path (resume/extend a run) */
  int32_t precision;     /* PDD_FP32 or PDD_FP64 path arithmetic */
  int32_t bridge;        /* 1: Brownian-bridge exit test, 0: plain test */
  int64_t node_offset;   /* stream index of the first node: node j of the call
                            draws the streams of node node_offset + j, so a
                            block of a larger node list solved on its own (one
                            rank of a node-sharded run) reproduces the
                            single-call paths; node_offset + n <= 2^32 */
} pdd_mc_params;

/* Per-node flags (pdd_diag.d_node_flags), OR-ed. */
enum {
  PDD_NODE_ON_BOUNDARY = 1, /* node on the boundary: u = g exactly, no steps */
  PDD_NODE_OUTSIDE = 2,     /* node outside the closed domain (or a score
                               beyond 2^30 in magnitude): mean and se are NaN */
  PDD_NODE_CAPPED = 4,      /* some path / walk hit the step cap (counted) */
  PDD_NODE_DISCARDED = 8,   /* branching: some trees were pruned (discarded) */
  PDD_NODE_EMPTY = 16,      /* no sample kept: mean and se are NaN */
  PDD_NODE_SE_UNMET = 32    /* adaptive batch: N_i stopped at n_max with the
                               standard error still above target_se */
};

/* Optional diagnostics.  Inputs: the optional device buffers receive, for
 * every (node, path) in node-major order, the path's score (FP64), its exit
 * step (0 for a node on the boundary, -max_steps for a capped path) and
 * (pdd_interface_solve, pdd_wos_solve) its exit point (FP64 [dim], the
 * projection on the nearest face for a capped path or a stopped walk), and
 * per node its flags (PDD_NODE_*; pdd_interface_solve, pdd_branching_solve,
 * pdd_batch_solve).
 * Outputs (host, valid when the call returns): total Euler steps taken and the
 * number of capped paths/trees. */
typedef struct {
  double *d_path_score;    /* [n * n_paths] or NULL */
  int32_t *d_path_steps;   /* [n * n_paths] or NULL */
  double *d_path_aux;      /* pdd_interface_grad: [n * n_paths][18] per-path
                              exit point (x, y) and likelihood-ratio sums
                              L_1..L_16; pdd_mlmc_level: [n * n_paths][8] per
                              pair the fine and coarse scores, their exit
                              steps (fine steps; coarse steps; negative when
                              capped) and exit points (x, y each; 0 for the
                              coarse walk at level 0); or NULL */
  int64_t path_steps;      /* out */
  int64_t capped;          /* out */
  double *d_path_exit;     /* [n * n_paths][dim] or NULL */
  int32_t *d_node_flags;   /* [n] or NULL */
} pdd_diag;

typedef struct pdd_ctx pdd_ctx;

/* Create a context for one problem on `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The problem's params
 * are copied.  Returns PDD_EINVAL for an unknown family, a dimension or
 * geometry the family does not support, sigma <= 0, a non-finite parameter or
 * a KPP offspring law that is not a probability distribution (Assumption 3.1
 * for q; alpha may be any real weights, Sec. 3.2).                          */
PDD_API pdd_status pdd_create(pdd_ctx **out, const pdd_problem *problem, int device,
                      void *cuda_stream);

/* Rebind the context to another stream on the same device. */
PDD_API pdd_status pdd_set_stream(pdd_ctx *ctx, void *cuda_stream);

/* Stage one of PDD for linear problems (Sec. 2, Fig. 2.2): for each node
 * x_i (d_nodes is [n][dim] FP64, inside the closed domain) estimate
 * u(x_i) = E[g(X_tau) Y_tau + Z_tau] (Eq. 2.1, 2.5-2.9 in the elliptic
 * Dirichlet reduction) from n_paths Euler-Maruyama paths with the plain or
 * Brownian-bridge exit test (the boundary-corrected integrators cited in
 * Sec. 2.1).  Writes d_mean[n], d_se[n] (standard error of the mean, FP64)
 * and, if non-NULL, d_npaths[n] (int64).  A node on the boundary gets
 * u = g(x_i) with zero error.  Path i of node j uses the Philox stream
 * (key = seed, counter = (block, path_offset + i, node_offset + j, 0)); the
 * per-step use of
 * that stream is fixed: three blocks per four steps (2-D: step 4q+j takes
 * its normals from words 2j, 2j+1 of blocks 3q..3q+2 by Box-Muller and its
 * bridge uniform from word 8+j; 3-D: normals from the word pairs, bridge
 * uniforms from the words' low bytes).
 * The per-node mean and standard error come from exact integer sums of the
 * scores and their squares (each truncated once to 2^-60), so they are
 * bitwise independent of scheduling and launch shape, and no per-path score
 * is stored: the call needs 112 bytes of context scratch per node.
 * With diag non-NULL the call synchronises and returns PDD_ECAP if some path
 * hit max_steps, PDD_EINVAL if a node lies outside the closed domain (its
 * mean is NaN either way).                                                 */
PDD_API pdd_status pdd_interface_solve(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                               const pdd_mc_params *mc, double *d_mean,
                               double *d_se, int64_t *d_npaths,
                               pdd_diag *diag);

/* Derivatives of stage one (POISSON_FOURIER family, FP32 paths): for each
 * node the Jacobian row of the estimate with respect to theta (64 Fourier
 * weights of g) and phi (16 drift weights), computed on the same paths as
 * pdd_interface_solve with the same mc (the paths are re-simulated from their
 * Philox keys; nothing is kept from the forward call):
 *   J[i][k]      = E[cos(m pi X_tau,x) cos(n pi X_tau,y)], k = 8m + n (exact
 *                  pathwise derivative: the paths do not depend on theta);
 *   J[i][64 + j] = E[s L_j], L_j = sum over the steps of xi . db/dphi_j(X)
 *                  sqrt(dt)/sigma (likelihood ratio of the Euler-Maruyama
 *                  transition density; the exit rule does not depend on phi).
 * d_jac / d_jac_se ([n][80] FP64, optional) receive J and its standard errors.
 * With d_grad_out ([n] FP64 cotangent) the vector-Jacobian products
 * d_dtheta[64] = sum_i w_i J[i][0:64] and d_dphi[16] = sum_i w_i J[i][64:80]
 * are written (either may be NULL).  Optional diag as for
 * pdd_interface_solve, plus d_path_aux.                                    */
PDD_API pdd_status pdd_interface_grad(pdd_ctx *ctx, const double *d_nodes,
                                      int64_t n, const pdd_mc_params *mc,
                                      const double *d_grad_out, double *d_jac,
                                      double *d_jac_se, double *d_dtheta,
                                      double *d_dphi, pdd_diag *diag);

/* Replace the problem's parameters (same family and length), e.g. new
 * theta/phi between forward evaluations.  Host array, copied.             */
PDD_API pdd_status pdd_set_params(pdd_ctx *ctx, const double *params,
                                  int32_t n_params);

/* Batched, variance-adaptive stage one over a heterogeneous node set.
 * Nodes may belong to different problems (up to 4 pdd_problem entries:
 * LAPLACE_EXPCOS on the unit square or the L-shape, ELLIPTIC_MANUFACTURED on
 * the unit cube, POISSON_FOURIER on the unit square) and carry their own
 * time step.  Per node i (paths are FP32; every score goes into the node's
 * exact integer sums, as in pdd_interface_solve):
 *   1. a pilot of n_pilot paths gives the sample variance s_i^2;
 *   2. N_i = clamp(ceil(s_i^2 / target_se^2), max(n_min, n_pilot), n_max);
 *   3. paths n_pilot .. N_i - 1 are added and the estimate uses all N_i.
 * Node i's path p uses the same Philox stream as pdd_interface_solve
 * (counter = (block, p, i, 0)), and the sums are the same, so with
 * n_min = n_max = N the results equal pdd_interface_solve's bit for bit.
 * The work list of the second pass is built
 * on the device, and one persistent launch consumes it (lanes take chunks of
 * `chunk` consecutive paths of one node), so the call has no host round trip.
 * With use_graph != 0 the whole sequence is captured once into a CUDA graph
 * (rebuilt when any argument or the scratch changes) and replayed; this
 * needs a non-default stream.  Writes d_mean[n], d_se[n] and, if non-NULL,
 * d_npaths[n] (= N_i; 0 for a node outside the closed domain or of an
 * unknown problem, whose mean and se are NaN).  diag (optional) reports total steps / capped paths
 * and synchronises; its d_node_flags receives PDD_NODE_SE_UNMET for the nodes
 * whose final standard error is above target_se and PDD_NODE_OUTSIDE for
 * the nodes without an estimate.                                           */
typedef struct {
  const double *d_nodes;     /* [n][3] FP64 (z ignored by 2-D problems) */
  const int32_t *d_problem;  /* [n] index into the problems array */
  const double *d_dt;        /* [n] Euler-Maruyama step, sigma^2 dt <= 1/36 */
  int64_t n;
} pdd_batch_nodes;

typedef struct {
  uint64_t seed;
  int64_t n_pilot;           /* pilot paths per node (>= 2) */
  int64_t n_min, n_max;      /* clamp of the adaptive path count */
  double target_se;          /* standard error aimed for (> 0) */
  int64_t max_steps;         /* per-path step cap */
  int32_t chunk;             /* paths per lane-chunk (0 = tuned default) */
  int32_t bridge;            /* Brownian-bridge exit test on/off */
} pdd_batch_params;

PDD_API pdd_status pdd_batch_solve(pdd_ctx *ctx, const pdd_problem *problems,
                                   int32_t n_problems,
                                   const pdd_batch_nodes *nodes,
                                   const pdd_batch_params *bp, double *d_mean,
                                   double *d_se, int64_t *d_npaths,
                                   int32_t use_graph, pdd_diag *diag);

/* Walk on Spheres for the Laplace problem (Eq. 1.1; Sec. 2.1 recommends it
 * for stopped Brownian motion): from x the walk jumps to a uniform point on
 * the largest circle inside the domain (radius = distance to the nearest
 * face; the L-shape's notch edges by segment distance) and stops when that
 * distance is <= eps, scoring g at the projection on the nearest face.
 * No time step; bias O(eps); O(log 1/eps) jumps per walk.  Walk p of node i
 * takes jump n's angle 2 pi U from word n mod 4 of Philox(key = seed,
 * counter = (n div 4, path_offset + p, i, 2)).  LAPLACE_EXPCOS problems
 * (unit square or L-shape).  Outputs and diag as for pdd_interface_solve
 * (path_steps counts jumps).                                               */
typedef struct {
  uint64_t seed;
  int64_t n_paths;
  int64_t path_offset;
  int64_t max_steps;     /* jump cap (walks that hit it are counted) */
  double eps;            /* stopping shell, (0, 1/2); FP32 needs >= 1e-6 */
  int32_t precision;     /* PDD_FP32 or PDD_FP64 */
  int32_t reserved;      /* must be 0 */
} pdd_wos_params;

PDD_API pdd_status pdd_wos_solve(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                 const pdd_wos_params *wp, double *d_mean,
                                 double *d_se, int64_t *d_npaths,
                                 pdd_diag *diag);

/* Monte Carlo parameters of the branching estimator. */
typedef struct {
  uint64_t seed;          /* Philox key */
  int64_t n_trees;        /* trees per node (>= 1) */
  int64_t tree_offset;    /* index of the first tree (resume/extend a run) */
  int64_t max_particles;  /* pruning: a tree with more particles is discarded
                             and counted (Algorithm 3.1), >= 1, <= 2^31 */
  int32_t max_depth;      /* pending-particle stack cap per tree, 1..64; a
                             tree exceeding it is discarded and counted */
  int32_t reserved;       /* must be 0 */
} pdd_branch_params;

/* Stage one of PDD for the semilinear KPP-type problem (Sec. 3.1-3.2,
 * Algorithm 3.1): for each space-time node (d_nodes_xt is [n][dim+1] FP64:
 * position then time t >= 0) estimate u(x, t) = E[W prod_{alive at t}
 * psi(X^(k)_t)] from n_trees branching Brownian motions with Exp(beta)
 * lifetimes and offspring law q, W the product of alpha_k / q_k over the
 * branchings (W = 1 when alpha = q).  Writes d_mean[n], d_se[n] and, if
 * non-NULL, d_nkept[n] (trees kept after pruning).  Tree s of node i uses
 * the Philox stream (key = seed, counter = (particle id, tree_offset + s, i,
 * 1)) with depth-first particle ids.  psi kinds: const, sigmoid,
 * travelling wave, sine (problem parameters, see pdd_problem).  Positions
 * and times are FP32; a tree's product of psi values and marks alpha_k / q_k
 * is accumulated as a float-float value (error-free binary32 products,
 * ~2^-44 relative per factor) and rounded once to binary32; the per-node sums
 * are FP64.  Per-node flags: PDD_NODE_DISCARDED, PDD_NODE_EMPTY.
 * With diag non-NULL the call synchronises; diag->d_path_score receives
 * per-tree scores (NaN if discarded),
 * d_path_steps per-tree segment counts (negative if discarded), path_steps
 * the total segments and capped the discarded trees (status PDD_ECAP when
 * non-zero).  A node whose trees are all discarded gets NaN.             */
PDD_API pdd_status pdd_branching_solve(pdd_ctx *ctx, const double *d_nodes_xt,
                                       int64_t n, const pdd_branch_params *bp,
                                       double *d_mean, double *d_se,
                                       int64_t *d_nkept, pdd_diag *diag);

/* One level of the multilevel Monte Carlo estimator (Sec. 2.1 names Giles'
 * multilevel method as the next acceleration of the Euler scheme):
 *   E[P_L] = E[P_0] + sum_{l=1..L} E[P_l - P_{l-1}],
 * P_l the score of the Euler-Maruyama path (Eq. 2.8, with the exit test of
 * pdd_interface_solve) with step dt_l = dt0 / refine^l.  Level l >= 1 draws
 * coupled pairs: the fine path with dt_l and the coarse path with dt_{l-1}
 * driven by the same Brownian motion (coarse increment = sum of the refine
 * fine increments), each stopping at its own exit.  Fine step k of pair p at
 * node i reads Philox(key = seed, counter = (k, p, i, 16 + level)): normals
 * BM(w0, w1), bridge uniform U(w2); a coarse step takes the uniform of the
 * last fine step of its group.  Level 0 is the plain scheme with dt0.
 * Dirichlet data, 2-D families (LAPLACE_EXPCOS on the square or L-shape,
 * POISSON_FOURIER).  Writes, per node, d_mean (mean of P_l - P_{l-1}, or of
 * P_0), d_var (its sample variance) and, if non-NULL, the fine and coarse
 * means.  pdd_mlmc_solve runs the levels and combines them.  diag as for
 * pdd_interface_solve (path_steps counts fine steps; d_path_score receives
 * P_l - P_{l-1} per pair).                                                */
typedef struct {
  uint64_t seed;
  int64_t n_paths;     /* pairs per node at this level */
  int64_t max_steps;   /* fine-step cap per pair (capped walks are counted) */
  double dt0;          /* level-0 step; sigma^2 dt0 <= 1/36 */
  int32_t level;       /* 0..12 */
  int32_t refine;      /* step ratio between levels, 2..16 */
  int32_t precision;   /* PDD_FP32 or PDD_FP64 */
  int32_t bridge;      /* 1 = bridge exit test */
} pdd_mlmc_params;

PDD_API pdd_status pdd_mlmc_level(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                  const pdd_mlmc_params *mp, double *d_mean,
                                  double *d_var, double *d_fine_mean,
                                  double *d_coarse_mean, pdd_diag *diag);

/* The multilevel estimate (Sec. 2.1, Giles' method): levels 0 .. n_levels-1
 * of pdd_mlmc_level (mp gives seed, dt0, refine, precision, bridge and the
 * step cap; mp->level and mp->n_paths are ignored), level l with
 * n_per_level[l] pairs per node (host array), and per node
 *   d_mean = sum_l mean_l,   d_se = sqrt(sum_l var_l / n_per_level[l])
 * (independent levels), summed in level order on the device.  d_level_mean
 * and d_level_var ([n_levels][n] FP64, optional) receive the levels' means
 * and variances; without them the library keeps the levels in a buffer of
 * its own (2 n_levels n doubles, grown on demand, freed by pdd_destroy).
 * 1 <= n_levels <= 13.  diag: summed path_steps and capped counts
 * (PDD_ECAP if any walk hit the cap).                                      */
PDD_API pdd_status pdd_mlmc_solve(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                  const pdd_mlmc_params *mp, int32_t n_levels,
                                  const int64_t *n_per_level, double *d_mean,
                                  double *d_se, double *d_level_mean,
                                  double *d_level_var, pdd_diag *diag);

/* Parameters of the time-grid branching estimator. */
typedef struct {
  uint64_t seed;          /* Philox key */
  int64_t n_trees;        /* trees per node (>= 1) */
  int64_t tree_offset;    /* index of the first tree */
  int64_t max_particles;  /* pruning cap, 1..4096 (12-bit particle ids) */
  int32_t max_depth;      /* pending-particle stack cap, 1..64 */
  int32_t bridge;         /* bounded domains: 1 = Brownian-bridge exit test */
  double dt;              /* bounded domains: largest step of a walk (> 0) */
} pdd_grid_branch_params;

/* The KPP-type problem of pdd_branching_solve on a time grid, with one tree
 * per sample scoring every grid time (Algorithm 3.1 evaluates the particles
 * alive at each T_i), in free space (Eq. 3.1) or, when the problem's
 * geometry is the interval (1-D), the unit square or the L-shape (2-D), with
 * absorbing boundaries (Eq. 3.2): a particle that hits the boundary at tau
 * contributes g(X_tau, T_i - tau) to every T_i >= tau, a particle alive at
 * T_i contributes psi(X_{T_i}), and the weights alpha_k / q_k of Sec. 3.2
 * enter the times after each branching.  Boundary data by the psi kind:
 * const c -> c / (c + (1 - c) e^{beta s}); sigmoid -> psi(x); travelling
 * wave (parameter a) -> 1 - (1 + e^{a x1 - 5 beta s / 6})^-2; sine
 * (psi = prod_k sin(pi x_k)) -> 0.
 * d_nodes is [n][dim] FP64 (device); h_times [m] (host, 1 <= m <= 32) are
 * the grid times, positive and increasing.  Times are integer ticks of
 * 2^-k, k = 31 - e for T_m = f 2^e (f in [1/2, 1)): T_i and dt are rounded
 * to ticks, lifetimes truncated; a particle's walk is cut at every grid time,
 * at its lifetime's end and, in a bounded domain, at most dt ticks apart,
 * each piece with the exit test of pdd_interface_solve (hard exit at the
 * segment crossing; with bridge, the half-space crossing probability over
 * the faces within reach, exit at the face of largest probability).
 * Particle id of tree s at node i draws block j of Philox(key = seed,
 * counter = ((id << 20) | j, tree_offset + s, i, 3)): block 0 gives the
 * lifetime -ln U(w0) / beta and the offspring count from U(w3); block j >= 1
 * the normals BM(w0, w1) and the bridge uniform U(w2) of step j.  Positions,
 * lifetimes and tree products are FP32, the per-node sums FP64.  Writes
 * d_mean[n][m], d_se[n][m]
 * and, if non-NULL, d_nkept[n].  With diag non-NULL the call synchronises:
 * d_path_score receives [n][n_trees][m] tree scores (NaN if discarded),
 * d_path_steps [n][n_trees] step counts (negative if discarded), path_steps
 * the total steps, capped the discarded trees (PDD_ECAP when non-zero); a
 * node outside the closed domain gives PDD_EINVAL (NaN without diag).
 * PDD_EINVAL also for more than 2^20 - 1 steps per particle.             */
PDD_API pdd_status pdd_branching_grid_solve(pdd_ctx *ctx, const double *d_nodes,
                                            int64_t n, const double *h_times,
                                            int32_t m,
                                            const pdd_grid_branch_params *bp,
                                            double *d_mean, double *d_se,
                                            int64_t *d_nkept, pdd_diag *diag);

/* Interface interpolation on the internal planes of the unit cube (stage two
 * of PDD, Sec. 2.1: the Monte Carlo node values become Dirichlet data on the
 * artificial interfaces; the paper names Chebyshev or RBF interpolation).
 * For each of n_planes planes x_axis[p] = pos[p] (axis 0, 1 or 2, pos in
 * (0, 1)), a radial basis function interpolant with the cubic kernel |r|^3
 * and a linear polynomial term in the two in-plane coordinates, through the
 * plane's node_count[p] nodes (d_nodes [..][3] FP64 and d_vals [..] FP64,
 * the planes' nodes one after the other) and n_bnd points per edge of the
 * plane's perimeter on the cube's boundary (edge points at k / n_bnd of each
 * edge, corners once), which carry the problem's boundary data g; evaluated
 * at the plane's query_count[p] points (d_query [..][3], planes one after
 * the other) into d_out.  The interpolation systems ([Phi P; P^T 0], at most
 * 6144 unknowns per plane) are solved in FP64 by Gaussian elimination with
 * partial pivoting.  3-D family (ELLIPTIC_MANUFACTURED); 1 <= n_planes <=
 * 64; axis, pos, node_count and query_count are host arrays.  Synchronises;
 * PDD_EINVAL for a singular system (coincident nodes).                     */
PDD_API pdd_status pdd_interface_interp(pdd_ctx *ctx, int32_t n_planes, const int32_t *axis,
                                        const double *pos, const int64_t *node_count,
                                        const double *d_nodes, const double *d_vals,
                                        int32_t n_bnd, const int64_t *query_count,
                                        const double *d_query, double *d_out);

/* Stage two of PDD (Sec. 2.1, Fig. 2.2) for the Laplace family (Eq. 1.1):
 * the interpolator and the subdomain solver.  The subdomain is the box
 * [lo[0], hi[0]] x [lo[1], hi[1]] inside the unit square, discretised by an
 * n[0] x n[1] grid including its boundary (n[2] must be 1).  One side is an
 * artificial interface (axis iface_axis, at lo when iface_side = 0, at hi
 * when 1); its Dirichlet data are the cubic spline with not-a-knot end
 * conditions through the interface end points (value g, as they lie on the
 * physical boundary) and the m >= 2 Monte Carlo nodes (d_iface_s: node
 * coordinates along the interface, strictly increasing inside the side;
 * d_iface_vals: node values, both FP64 device arrays).  The other sides get
 * g.  The interior solves the 5-point system
 *   (u_{i+1,j} - 2u_{ij} + u_{i-1,j})/hx^2 + (u_{i,j+1} - 2u_{ij} + u_{i,j-1})/hy^2 = 0
 * by conjugate gradients in FP64 (stop at ||r||_2 <= tol ||b||_2), by FP32
 * conjugate gradients inside FP64 iterative refinement (CG_MIXED: the FP64
 * residual is scaled and solved to 1e-4 in FP32, the correction added in
 * FP64; same FP64 stopping rule; iterations count the FP32 ones), or Jacobi
 * sweeps (stop when max |u^{k+1} - u^k| < tol), at most max_iter
 * iterations; or directly (DST): the operator with Dirichlet data on a
 * rectangle is diagonal in the discrete sine basis, so four dense FP64
 * products of the sine matrices and a division by the eigenvalues give the
 * discrete solution to rounding (at most 8192 interior points per axis;
 * max_iter and tol are not used, *iters is 0).
 * d_u is [n[1]][n[0]] FP64 (row = y), written in full.  *iters and *resid
 * (host) receive the iteration count and the final residual measure; the call
 * synchronises.  Returns PDD_ETIMEOUT when max_iter ran out first (d_u holds
 * the last iterate).
 *
 * Three-dimensional subdomains (n[2] > 1; the 3-D family
 * ELLIPTIC_MANUFACTURED, the elliptic problem of Eq. 2.3 without time,
 * (1/2) sigma^2 Lap u + b . grad u + c u + f = 0): the box [lo, hi] inside
 * the unit cube with an n[0] x n[1] x n[2] grid including its boundary
 * (3 .. 128 points per axis), the 7-point system
 *   sum_a (1/2) sigma^2 (u_{+a} - 2u + u_{-a}) / h_a^2
 *     + sum_a b_a (u_{+a} - u_{-a}) / (2 h_a) + c u + f = 0
 * at the interior points.  iface_axis is then a mask of the faces that are
 * artificial interfaces (bit 2a + side: face x_a = lo[a] for side 0, hi[a]
 * for side 1); their Dirichlet data come in d_iface_vals, the masked faces
 * one after the other in bit order, each face's full grid with the higher
 * of its two axes slow ([n2][n1] for an x-face, [n2][n0] for a y-face,
 * [n1][n0] for a z-face); m is the total count of those values;
 * d_iface_s is not used and iface_side must be 0.  The other faces take g.
 * A grid point on several faces takes g if one of them has no interface
 * data, else the data of the first interface face.  Methods: DST (defect
 * correction u <- u + P^{-1} r with the FP64 residual r and P the
 * constant-coefficient part of the operator inverted by three-dimensional
 * sine transforms in binary32; stop at ||r||_2 <= tol ||r_0||_2, *iters
 * = corrections applied, *resid = ||r||_2 / ||r_0||_2) or JACOBI (stop when
 * max |u^{k+1} - u^k| < tol, *resid that change).  d_u is [n[2]][n[1]][n[0]],
 * written in full.                                                        */
enum { PDD_STENCIL_CG = 0, PDD_STENCIL_JACOBI = 1, PDD_STENCIL_CG_MIXED = 2, PDD_STENCIL_DST = 3 };

typedef struct {
  double lo[3], hi[3];
  int32_t n[3];
  int32_t iface_axis;
  int32_t iface_side;
  int32_t method;       /* PDD_STENCIL_CG, _JACOBI, _CG_MIXED or _DST */
  int64_t max_iter;
  double tol;
} pdd_subdomain;

PDD_API pdd_status pdd_subdomain_solve(pdd_ctx *ctx, const pdd_subdomain *sd,
                                       const double *d_iface_s,
                                       const double *d_iface_vals, int64_t m,
                                       double *d_u, int64_t *iters,
                                       double *resid);

/* Several three-dimensional subdomains solved together (the subdomains of
 * stage two are independent problems, Sec. 2): n_boxes entries of sds, each
 * a 3-D box as for pdd_subdomain_solve (its own lo, hi and interface mask),
 * all with the same grid size n, method (DST or JACOBI), max_iter and tol.
 * d_face holds each box's interface data as pdd_subdomain_solve takes them,
 * box after box (m values in all); d_u is [n_boxes][n[2]][n[1]][n[0]] FP64,
 * written in full.  Each box runs its own stopping rule; *iters and *resid
 * (host) get the largest count and residual measure over the boxes, and
 * iters_each / resid_each (host arrays of n_boxes, may be NULL) each box's
 * own.  A box's result is bit-identical to its pdd_subdomain_solve.  At most
 * 65535 boxes; PDD_EINVAL for mixed sizes or rules, PDD_ETIMEOUT when a box
 * ran out of max_iter (d_u then holds its last iterate).  Synchronises. */
PDD_API pdd_status pdd_subdomain_solve_batch(pdd_ctx *ctx, const pdd_subdomain *sds,
                                             int32_t n_boxes, const double *d_face,
                                             int64_t m, double *d_u, int64_t *iters,
                                             double *resid, int64_t *iters_each,
                                             double *resid_each);

/* The plain GPU form of pdd_interface_solve, kept as a comparison baseline:
 * one kernel launch per node, one thread per path, block sums added to FP64
 * node accumulators with atomics (so the last bits depend on scheduling), no
 * work queue, no graph.  Same estimator and random streams as
 * pdd_interface_solve (FP32 paths only).  Writes d_mean, d_se, d_npaths.  */
PDD_API pdd_status pdd_interface_solve_naive(pdd_ctx *ctx, const double *d_nodes,
                                             int64_t n, const pdd_mc_params *mc,
                                             double *d_mean, double *d_se,
                                             int64_t *d_npaths);

/* Autotuner (launch shape only; results never depend on it).  Runs the
 * given interface solve (use a reduced n_paths: each candidate runs
 * repeats + 1 times) for every resident-blocks-per-SM count the device
 * allows (up to 8), times each on the context's stream, keeps the fastest
 * (fewer blocks on ties within 1%) in the context and reports it.
 * d_scratch_out is a caller buffer of 2n doubles for the trial outputs.
 * Synchronises.                                                            */
PDD_API pdd_status pdd_autotune(pdd_ctx *ctx, const double *d_nodes, int64_t n,
                                const pdd_mc_params *mc, double *d_scratch_out,
                                int32_t repeats, int32_t *best_blocks_per_sm,
                                double *best_ms);

/* Same for pdd_batch_solve's lane-chunk size (32 .. 1024 paths). */
PDD_API pdd_status pdd_autotune_batch(pdd_ctx *ctx, const pdd_problem *problems,
                                      int32_t n_problems,
                                      const pdd_batch_nodes *nodes,
                                      const pdd_batch_params *bp,
                                      double *d_scratch_out, int32_t repeats,
                                      int32_t *best_chunk, double *best_ms);

/* Launch-shape and memory knobs of the path kernels (no effect on results,
 * which do not depend on scheduling):
 *   blocks_per_sm    resident blocks per SM for the persistent path kernels
 *                    (128 threads for binary32 paths, 256 for FP64; 0 = the
 *                    occupancy maximum);
 *   wave_max_paths   paths per wave of the kernels that store one score per
 *                    path in the context's scratch (Walk on Spheres,
 *                    reflecting faces, branching, multilevel, gradient; 4 or
 *                    8 bytes per path), each wave reduced before the next
 *                    starts (0 = default 2^29).  pdd_interface_solve with
 *                    absorbing faces stores no per-path score and runs all
 *                    paths in one launch.                                   */
PDD_API pdd_status pdd_set_tuning(pdd_ctx *ctx, int blocks_per_sm,
                                  int64_t wave_max_paths);

/* Kernel timing.  With profiling on, the library records a CUDA event pair on
 * the context's stream around every launch of its dominant kernel (the path
 * kernel of pdd_interface_solve).  pdd_profile_read synchronises the stream and
 * returns the summed elapsed milliseconds and the launch count since the last
 * read (or since profiling was switched on), then resets both.            */
PDD_API pdd_status pdd_profile(pdd_ctx *ctx, int enable);
PDD_API pdd_status pdd_profile_read(pdd_ctx *ctx, double *kernel_ms,
                                    int64_t *launches);

/* pdd_interface_solve without any device allocation.  The paper has no
 * counterpart: this is a deployment variant for callers that cannot call
 * cudaMalloc -- hosts whose memory pool owns the whole device, plug-ins that
 * only receive pre-allocated buffers, and latency-critical loops where an
 * allocation (or its failure) is not acceptable.
 * It computes the same estimate as pdd_interface_solve (same kernels, same
 * streams, same exact per-node sums, no diagnostics) on `device` and
 * `cuda_stream`, without a context, in one path-kernel launch and one
 * finalisation launch.  The caller still provides the inputs and outputs
 * (device pointers, as for pdd_interface_solve).  Scratch comes from one
 * static 8 MiB device array that every GPU loading this library holds until
 * process exit (256 bytes of counters and 112 bytes per node); n is limited
 * to 65536 nodes and node_offset + n to 2^32 (PDD_EINVAL beyond), the path
 * count is not limited.  The first call on a device loads the kernels; every
 * call looks up the array's device address (no allocation).  All calls share
 * the array and each clears it at the start, so calls that overlap on the GPU
 * (different streams, or different threads) race: serialise them.
 * It calls no cudaMalloc, cudaFree or allocating library routine.          */
PDD_API pdd_status pdd_interface_solve_static(const pdd_problem *problem,
                                              int device, void *cuda_stream,
                                              const double *d_nodes, int64_t n,
                                              const pdd_mc_params *mc,
                                              double *d_mean, double *d_se,
                                              int64_t *d_npaths);

/* Philox4x32-10 (Salmon et al., SC'11) blocks for counters
 * (j0 + b, c1, c2, c3), b < n_blocks, key = (seed low, seed high), written to
 * d_out[n_blocks][4].  Exposes the generator the estimators consume, so that
 * its stream can be checked bit for bit.                                    */
PDD_API pdd_status pdd_philox_stream(pdd_ctx *ctx, uint64_t seed, uint32_t j0,
                             uint32_t c1, uint32_t c2, uint32_t c3,
                             int64_t n_blocks, uint32_t *d_out);

/* The FP32 standard normals and uniforms the path kernels draw: for pair j
 * (j < n_pairs) the Box-Muller pair of words 0 and 1 of
 * Philox((j, c1, c2, c3), key = seed) into d_z[2j], d_z[2j+1] and the
 * uniform of word 2 into d_u[j] (d_u may be NULL).  Exposes the binary32
 * normal generator so that it can be checked against an FP64 one.        */
PDD_API pdd_status pdd_normals(pdd_ctx *ctx, uint64_t seed, uint32_t c1,
                               uint32_t c2, uint32_t c3, int64_t n_pairs,
                               float *d_z, float *d_u);

/* Release the context and its device scratch (synchronises its stream). */
PDD_API void pdd_destroy(pdd_ctx *ctx);

/* Static description of a status code. */
PDD_API const char *pdd_status_string(pdd_status status);

/* One-line description of the last failure on ctx ("" if none).  With
 * ctx = NULL: why the calling thread's last pdd_create failed ("" if it
 * succeeded).                                                             */
PDD_API const char *pdd_last_error(const pdd_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PDD_H */
