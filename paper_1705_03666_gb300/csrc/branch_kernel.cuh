// branch_kernel.cuh -- branching Brownian motion for the semilinear problem
//   u_t = (1/2) Lap u + beta (sum_k alpha_k u^k - u),  u(., 0) = psi
// in free space (Eq. 3.1 with the classical weights of Assumption 3.1, and
// the marked weights alpha_k / q_k of Sec. 3.2).  u(x, t) = E[weight * prod of
// psi over the particles alive at time t] (Sec. 3.1.1; Algorithm 3.1 with
// per-particle Exp(beta) lifetimes, equal in law to its global clock).
//
// One lane owns one tree at a time and walks it depth-first; the pending
// siblings of the current lineage live in a per-lane stack (local memory,
// only its top few entries are touched).  Warps claim trees in chunks
// (warp_queue.cuh), and each tree's score goes to its own slot, so the
// per-node reduction does not depend on scheduling.  The tree's product,
// weight and offspring choice are binary32: FP64 is a 1/64-rate pipe on
// this part and these operations sit in divergent per-segment code.
//
// Tree order (shared with the oracle): the root has id 0; a particle that
// branches into k children gives them ids next_id .. next_id + k - 1 and the
// lowest id is followed first.  Particle id j of tree s at node i draws
// w = Philox(seed, (j, s, i, 1)): lifetime -ln U(w0) / beta, Brownian
// increment sqrt(duration) * BM(w1, w2), offspring count from U(w3) by the
// inverse CDF of q.  A tree whose particle count exceeds max_particles or
// whose pending stack would exceed max_depth is discarded (NaN score) and
// counted (pruning, Algorithm 3.1).
#pragma once

#include "common.cuh"
#include "warp_queue.cuh"

namespace pdd {

constexpr int kBranchBlock = 256;
constexpr int kBranchMaxDepth = 64;
constexpr int kMaxOffspring = 7;
constexpr unsigned kBranchChunk = 64;  // trees claimed per warp-level atomic

struct BranchArgs {
  const float4 *nodes_f;        // [n]: (x1, x2 or 0, t, 0) in binary32
  uint64_t n_trees, tree_offset;
  uint64_t begin, end;          // tree index range of this wave
  unsigned long long *cursor;
  unsigned long long *counters; // [0] segments, [1] discarded trees
  float *score;                 // [end - begin]; NaN for discarded trees
  int32_t *segs;                // [end - begin] or null
  RoundKeys rk;
  float inv_beta;
  int32_t psi_kind;             // 0 const, 1 sigmoid, 2 travelling wave, 3 sine
  float psi_prm;
  int32_t K;                    // largest offspring count
  float cum[kMaxOffspring + 1];    // cumulative q (FP64 sums, rounded)
  float ratio[kMaxOffspring + 1];  // alpha_k / q_k (1 for classical weights)
  int64_t max_particles;
  int32_t max_depth;
};

template <int D>
__device__ __forceinline__ float psi_eval(const BranchArgs &a, float x1, float x2) {
  switch (a.psi_kind) {
    case 0: return a.psi_prm;
    case 1: return __fdividef(1.0f, 1.0f + expf(-a.psi_prm * x1));
    case 2: {
      const float e = 1.0f + expf(a.psi_prm * x1);
      return 1.0f - __fdividef(1.0f, e * e);
    }
    default: return sinpif(x1) * (D > 1 ? sinpif(x2) : 1.0f);
  }
}

template <int D>
__global__ void __launch_bounds__(kBranchBlock)
branch_kernel(const __grid_constant__ BranchArgs a) {
  const unsigned lane = threadIdx.x & 31u;
  float4 stk[kBranchMaxDepth];  // pending particles: (x1, x2, t_birth, id bits)
  int sp = 0;
  // current particle
  float x0 = 0.f, x1 = 0.f, tb = 0.f;
  uint32_t id = 0;
  // current tree: the (tree, node, tag 1) half of Philox round one
  PhiloxPath pp{0, 0, 1u};
  uint32_t next_id = 0;
  float t = 0.f;
  float prod = 1.0f, weight = 1.0f;
  int64_t particles = 0;
  int32_t segments = 0;
  uint64_t slot = 0;
  bool active = false, need = true;
  unsigned long long my_segs = 0, my_disc = 0;
  WarpQueue wq;
  const unsigned long long total = a.end - a.begin;

  for (;;) {
    if (claim_time<1>(active)) {
      need = !active;
      while (__any_sync(kFull, need)) {
        unsigned long long q = 0;
        if (warp_claim<kBranchChunk>(wq, a.cursor, total, need, q)) {
          slot = q;
          const unsigned long long g = a.begin + q;
          // trees take ~2.5 segments: a per-lane node cache costs more in
          // registers (occupancy) than the division it saves
          const uint64_t nd = a.end <= 0xffffffffull
                                  ? static_cast<uint32_t>(g) / static_cast<uint32_t>(a.n_trees)
                                  : g / a.n_trees;
          const uint32_t tree = static_cast<uint32_t>(g - nd * a.n_trees + a.tree_offset);
          pp = philox_path(tree, static_cast<uint32_t>(nd), 1u, a.rk);
          const float4 xt = a.nodes_f[nd];  // converted once per call, not per tree
          x0 = xt.x;
          x1 = xt.y;
          t = xt.z;
          tb = 0.f;
          id = 0;
          next_id = 1;
          sp = 0;
          prod = 1.0f;
          weight = 1.0f;
          particles = 1;
          segments = 0;
          active = true;
        }
      }
      if (!__any_sync(kFull, active)) break;
    }
    if (!active) continue;

    // ---- one particle segment
    const uint4 w = philox10_path(id, pp, a.rk);  // = Philox((id, tree, node, 1))
    const float life = 0.5f * neg2log(unif_f(w.x)) * a.inv_beta;  // -ln U / beta
    float tend = tb + life;
    const bool reaches = tend >= t;
    if (reaches) tend = t;
    float z0, z1;
    box_muller<float>(w.y, w.z, z0, z1);
    const float h = sqrt_approx(tend - tb);
    x0 += h * z0;
    if (D == 2) x1 += h * z1;
    ++segments;
    bool tree_done = false, bad = false, pop = false;
    if (reaches) {
      prod *= psi_eval<D>(a, x0, x1);
      pop = true;
    } else {
      const float u3 = unif_f(w.w);
      int k = a.K;
      for (int kk = 0; kk <= a.K; ++kk) {
        if (u3 < a.cum[kk]) {
          k = kk;
          break;
        }
      }
      weight *= a.ratio[k];
      particles += k;
      if (particles > a.max_particles || sp + k > a.max_depth) {
        bad = true;
        tree_done = true;
      } else if (k == 0) {
        pop = true;
      } else {
        for (int c = k - 1; c >= 1; --c)
          stk[sp++] = make_float4(x0, x1, tend, __uint_as_float(next_id + c));
        id = next_id;
        tb = tend;
        next_id += k;
      }
    }
    if (pop) {
      if (sp == 0) {
        tree_done = true;
      } else {
        const float4 p = stk[--sp];
        x0 = p.x;
        x1 = p.y;
        tb = p.z;
        id = __float_as_uint(p.w);
      }
    }
    if (tree_done) {
      a.score[slot] = bad ? NAN : weight * prod;
      if (a.segs) a.segs[slot] = bad ? -segments : segments;
      my_segs += static_cast<unsigned long long>(segments);
      if (bad) ++my_disc;
      active = false;
      need = true;
    }
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    my_segs += __shfl_xor_sync(kFull, my_segs, m);
    my_disc += __shfl_xor_sync(kFull, my_disc, m);
  }
  if (lane == 0) {
    if (my_segs) atomicAdd(&a.counters[0], my_segs);
    if (my_disc) atomicAdd(&a.counters[1], my_disc);
  }
}

}  // namespace pdd
