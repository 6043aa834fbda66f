// branch_kernel.cuh -- branching Brownian motion for the semilinear problem
//   u_t = (1/2) Lap u + beta (sum_k alpha_k u^k - u),  u(., 0) = psi
// in free space (Eq. 3.1 with the classical weights of Assumption 3.1, and
// the marked weights alpha_k / q_k of Sec. 3.2).  u(x, t) = E[weight * prod of
// psi over the particles alive at time t] (Sec. 3.1.1; Algorithm 3.1 with
// per-particle Exp(beta) lifetimes, equal in law to its global clock).
//
// One lane owns one tree at a time and walks it depth-first, one particle
// segment per loop trip; the pending siblings of the current lineage live in
// a per-lane stack (local memory, only its top few entries are touched).
// Trees are short (about 2.5 segments at beta = t = 1), so starting one must
// be cheap: a lane works through a run of consecutive trees (16, fewer near
// the end of the wave) and holds the next run in reserve; the warp refills
// the reserves of half its lanes at once with one atomic, so no lane waits
// for a claim.  A lane keeps its node's coordinates and the node's half of
// Philox round one while its trees stay on that node, so a tree start is a
// handful of register moves.  The segment itself is the
// same straight-line code for a particle that reaches t and one that
// branches: the factor it contributes (psi at its end point, or the mark
// alpha_k / q_k) multiplies the tree's float-float product, an error-free
// binary32 product (~2^-44 relative per factor, the binary64-class
// accumulation the semilinear problem asks for, on the FP32 pipe).  Each
// tree's score goes to its own slot, so the per-node reduction does not
// depend on scheduling.
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
#include "nodefix.cuh"

namespace pdd {

constexpr int kBranchBlock = 256;
constexpr int kBranchMaxDepth = 64;
constexpr int kMaxOffspring = 7;

struct BranchArgs {
  const float4 *nodes_f;        // [n]: (x1, x2 or 0, t, 0) in binary32
  uint64_t n_trees, tree_offset;
  uint64_t begin, end;          // tree index range of this wave
  unsigned long long *cursor;
  unsigned long long *counters; // [0] segments, [1] discarded trees
  float *score;                 // [end - begin]; NaN for discarded trees
  int32_t *segs;                // [end - begin] or null
  int32_t *flags;               // per-node flags or null (discarded trees)
  RoundKeys rk;
  float inv_beta;
  int32_t psi_kind;             // 0 const, 1 sigmoid, 2 travelling wave, 3 sine
  float psi_prm;
  float psi_l2;                 // psi_prm log2(e) (sigmoid, travelling wave)
  int32_t K;                    // largest offspring count
  float cum[kMaxOffspring + 1];    // cumulative q (FP64 sums, rounded)
  float ratio[kMaxOffspring + 1];  // alpha_k / q_k (1 for classical weights)
  int64_t max_particles;
  int32_t max_depth;
};

// psi at a particle's end point.  The sigmoid and the travelling wave use the
// hardware exp2 and reciprocal (a few ulp); the sine data the accurate sinpi.
template <int D>
__device__ __forceinline__ float psi_eval(const BranchArgs &a, float x1, float x2) {
  switch (a.psi_kind) {
    case 0: return a.psi_prm;
    case 1: return __frcp_rn(1.0f + ex2_approx(-a.psi_l2 * x1));
    case 2: {
      const float e = 1.0f + ex2_approx(a.psi_l2 * x1);
      return 1.0f - __frcp_rn(e * e);
    }
    default: return sinpif(x1) * (D > 1 ? sinpif(x2) : 1.0f);
  }
}

// (hi, lo) <- (hi, lo) * f without rounding error in the product hi * f
// (Dekker's product by FMA), renormalised: a float-float accumulator.
__device__ __forceinline__ void ff_mul(float &hi, float &lo, float f) {
  const float p = hi * f;
  const float e = fmaf(hi, f, -p);
  const float l = fmaf(lo, f, e);
  hi = p + l;
  lo = l - (hi - p);
}

// kBinary: the offspring law is two children with probability one and the
// classical weight (the KPP problem), so the count and the mark are constants.
template <int D, bool kBinary>
__global__ void __launch_bounds__(kBranchBlock)
branch_kernel(const __grid_constant__ BranchArgs a) {
  const unsigned lane = threadIdx.x & 31u;
  float4 stk[kBranchMaxDepth];  // pending particles: (x1, x2, t_birth, id bits)
  int sp = 0;
  // current particle
  float x0 = 0.f, x1 = 0.f, tb = 0.f;
  uint32_t id = 0;
  // current tree
  PhiloxPath pp{0, 0, 1u};
  uint32_t next_id = 0;
  float ph = 1.0f, pl = 0.0f;  // float-float product of the tree's factors
  uint32_t particles = 0;
  int32_t segments = 0;
  // the lane's run of trees [g, gend) within the wave (at most 2^31 trees),
  // the next run [ng, ngend) held in reserve, and the lane's node cache
  uint32_t g = 0, gend = 0, ng = 0, ngend = 0;
  uint32_t wlast = 0;        // warp-uniform: base of the warp's last claim
  bool exhausted = false;    // warp-uniform: the wave's trees are all claimed
  unsigned long long nlo = 1, nhi = 0;
  uint64_t node = 0;
  float nx0 = 0.f, nx1 = 0.f, t = 0.f;
  uint32_t nw0 = 0, nw1 = 0;  // node half of Philox round one
  bool active = false;
  unsigned long long my_segs = 0, my_disc = 0;
  const uint32_t total = static_cast<uint32_t>(a.end - a.begin);
  const uint32_t lanes = gridDim.x * blockDim.x;
  const unsigned lt_mask = (1u << lane) - 1u;
  const uint32_t max_particles =
      a.max_particles < 0x80000000ll ? static_cast<uint32_t>(a.max_particles) : 0x80000000u;

  // start tree g of the lane's run (node cache refreshed at node changes)
  auto start_tree = [&]() {
    const unsigned long long gg = a.begin + g;
    if (gg >= nhi || gg < nlo) {
      node = a.end <= 0xffffffffull ? static_cast<uint32_t>(gg) / static_cast<uint32_t>(a.n_trees)
                                    : gg / a.n_trees;
      nlo = node * a.n_trees;
      nhi = nlo + a.n_trees;
      const float4 xt = a.nodes_f[node];  // converted once per call, not per tree
      nx0 = xt.x;
      nx1 = xt.y;
      t = xt.z;
      const PhiloxPath np = philox_path(0u, static_cast<uint32_t>(node), 1u, a.rk);
      nw0 = np.r0_w0;  // hi(M1 node) ^ rk0 (the tree index is XORed in per tree)
      nw1 = np.r0_w1;
    }
    pp.r0_w0 = nw0 ^ static_cast<uint32_t>(gg - nlo + a.tree_offset);
    pp.r0_w1 = nw1;
    x0 = nx0;
    x1 = nx1;
    tb = 0.f;
    id = 0;
    next_id = 1;
    sp = 0;
    ph = 1.0f;
    pl = 0.0f;
    particles = 1;
    segments = 0;
  };
  // the next tree of the current run, else of the reserve run; false if none
  auto next_tree = [&]() -> bool {
    if (g >= gend && ng < ngend) {
      g = ng;
      gend = ngend;
      ng = ngend;
    }
    if (g >= gend) return false;
    start_tree();
    return true;
  };

  for (;;) {
    // ---- the warp refills its lanes' reserve runs together, with one
    // atomic, once half of them are used up (or a lane has nothing left)
    const bool need = ng >= ngend && !exhausted;
    const unsigned empty = __ballot_sync(kFull, need);
    if (empty && (__popc(empty) >= 16 || __any_sync(kFull, !active && need))) {
      // runs of 16 trees while plenty remain, shorter near the end
      const uint32_t rem = total > wlast ? total - wlast : 0u;
      const uint32_t R = rem > 64u * lanes ? 16u : (rem > 4u * lanes ? rem / (4u * lanes) : 1u);
      uint32_t base = 0;
      if (lane == 0) {
        const unsigned long long b =
            atomicAdd(a.cursor, static_cast<unsigned long long>(R) * __popc(empty));
        base = b < total ? static_cast<uint32_t>(b) : total;
      }
      base = __shfl_sync(kFull, base, 0);
      wlast = base;
      if (base >= total) {
        exhausted = true;
      } else if (need) {
        const uint32_t lo = base + R * __popc(empty & lt_mask);
        ng = lo < total ? lo : total;
        ngend = lo < total && total - lo > R ? lo + R : total;
      }
    }
    if (!active) active = next_tree();
    if (!__any_sync(kFull, active)) {
      if (exhausted) break;
      continue;
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
    int k = 2;
    float mark = 1.0f;
    if constexpr (!kBinary) {
      // inverse CDF of q: the number of cumulative sums at or below U(w3)
      const float u3 = unif_f(w.w);
      k = 0;
#pragma unroll
      for (int kk = 0; kk < kMaxOffspring; ++kk)
        k += (kk < a.K && u3 >= a.cum[kk]) ? 1 : 0;
      mark = a.ratio[k];
    }
    ff_mul(ph, pl, reaches ? psi_eval<D>(a, x0, x1) : mark);
    bool pop = reaches, bad = false;
    if (!reaches) {
      particles += static_cast<uint32_t>(k);
      if (particles > max_particles || sp + k > a.max_depth) {
        bad = true;
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
    bool tree_done = bad;
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
      a.score[g] = bad ? NAN : ph + pl;
      if (a.segs) a.segs[g] = bad ? -segments : segments;
      my_segs += static_cast<unsigned long long>(segments);
      if (bad) {
        ++my_disc;
        if (a.flags) atomicOr(a.flags + node, kNodeDiscarded);
      }
      ++g;
      active = next_tree();  // the lane goes straight on with its next tree
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
