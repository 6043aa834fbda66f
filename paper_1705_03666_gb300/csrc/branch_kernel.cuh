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
constexpr int kBranchTrips = 8;  // segments per lane between reserve checks

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
  // x / n_trees for 32-bit x by one multiply-high and shifts (Granlund and
  // Montgomery, division by invariant integers): q = (t + ((x - t) >> s1))
  // >> s2 with t = mulhi(nt_m, x); used while the wave's tree indices fit in
  // 32 bits
  uint32_t nt_m;
  int32_t nt_s1, nt_s2;
};

// The multiplier and shifts of BranchArgs::nt_m for a divisor d >= 1:
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, s1 = min(l, 1),
// s2 = max(l - 1, 0).
inline void branch_divisor(uint32_t d, uint32_t *m, int32_t *s1, int32_t *s2) {
  int l = 0;
  while (l < 32 && (uint64_t(1) << l) < d) ++l;
  *m = static_cast<uint32_t>(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
  *s1 = l < 1 ? l : 1;
  *s2 = l > 1 ? l - 1 : 0;
}

// psi at a particle's end point.  The sigmoid and the travelling wave use the
// hardware exp2 and reciprocal (a few ulp in all, for arguments that stay
// normal: 1 + 2^y >= 1); the sine data the accurate sinpi.
template <int D, int kPsi>
__device__ __forceinline__ float psi_value(const BranchArgs &a, float x1, float x2) {
  if constexpr (kPsi == 0) {
    return a.psi_prm;
  } else if constexpr (kPsi == 1) {
    return rcp_approx(1.0f + ex2_approx(-a.psi_l2 * x1));
  } else if constexpr (kPsi == 2) {
    const float e = 1.0f + ex2_approx(a.psi_l2 * x1);
    return 1.0f - rcp_approx(e * e);
  } else {
    return sinpif(x1) * (D > 1 ? sinpif(x2) : 1.0f);
  }
}
// The same with the kind read at run time (psi_kind in 0..3).
template <int D>
__device__ __forceinline__ float psi_eval(const BranchArgs &a, float x1, float x2) {
  switch (a.psi_kind) {
    case 0: return psi_value<D, 0>(a, x1, x2);
    case 1: return psi_value<D, 1>(a, x1, x2);
    case 2: return psi_value<D, 2>(a, x1, x2);
    default: return psi_value<D, 3>(a, x1, x2);
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
// classical weight (the KPP problem), so the count and the mark are
// constants.  kPsi: the initial-data kind fixed at compile time (0..3), or
// -1 to read it at run time.
//
// Control flow.  Every loop trip, each active lane runs one segment; what
// follows is short and mostly predicated, so that a warp pays little for its
// lanes taking different turns: a branching particle pushes its second child
// (one 16-byte local store), a particle that reaches t pops the next pending
// one (one 16-byte local load), and a lane whose tree is done stores the
// score and starts the next tree of its run in place.  Tree indices within
// the wave are 32-bit; the tree's Philox key is the node's key XORed with
// (run position + a per-node base), so a tree start is a few register moves.
template <int D, bool kBinary, int kPsi>
__global__ void __launch_bounds__(kBranchBlock)
branch_kernel(const __grid_constant__ BranchArgs a) {
  const unsigned lane = threadIdx.x & 31u;
  float4 stk[kBranchMaxDepth];  // pending particles: (x1, x2, t_birth, id bits)
  int sp = 0;
  // current particle
  float x0 = 0.f, x1 = 0.f, tb = 0.f;
  uint32_t id = 0;
  // current tree: Philox round-one word (node key ^ tree index), the next
  // particle id (= particles created so far), the float-float product
  uint32_t pw0 = 0;
  uint32_t next_id = 1;
  float ph = 1.0f, pl = 0.0f;
  uint32_t seg0 = 0;   // my_cnt at the tree's start
  // the lane's run of trees [g, gend) within the wave (at most 2^31 trees),
  // the next run [ng, ngend) held in reserve
  uint32_t g = 0, gend = 0, ng = 0, ngend = 0;
  uint32_t wlast = 0;        // warp-uniform: base of the warp's last claim
  bool exhausted = false;    // warp-uniform: the wave's trees are all claimed
  // node cache: the node of tree g, the wave index where its trees end, the
  // key base (tree index within the node = g + kbase mod 2^32), coordinates,
  // time, and the node's half of Philox round one
  uint32_t node = 0, node_end = 0, kbase = 0;
  float nx0 = 0.f, nx1 = 0.f, t = 0.f;
  uint32_t nw0 = 0, nw1 = 0;
  bool active = false;
  unsigned long long my_segs = 0;
  uint32_t my_cnt = 0, my_folded = 0;  // segments run by the lane (mod 2^32)
  uint32_t my_disc = 0;
  const uint32_t total = static_cast<uint32_t>(a.end - a.begin);
  const uint32_t lanes = gridDim.x * blockDim.x;
  const unsigned lt_mask = (1u << lane) - 1u;
  const uint32_t max_particles =
      a.max_particles < 0x80000000ll ? static_cast<uint32_t>(a.max_particles) : 0x80000000u;
  const int max_depth = a.max_depth;

  // the node cache for tree g
  auto refresh_node = [&]() {
    const unsigned long long gg = a.begin + g;
    uint64_t nd;
    if (a.end <= 0xffffffffull) {
      const uint32_t x = static_cast<uint32_t>(gg);
      const uint32_t tq = __umulhi(a.nt_m, x);
      nd = (tq + ((x - tq) >> a.nt_s1)) >> a.nt_s2;
    } else {
      nd = gg / a.n_trees;
    }
    const unsigned long long nlo = nd * a.n_trees;
    const unsigned long long ne = nlo + a.n_trees - a.begin;
    node = static_cast<uint32_t>(nd);
    node_end = ne < total ? static_cast<uint32_t>(ne) : total;
    kbase = static_cast<uint32_t>(a.tree_offset + a.begin - nlo);
    const float4 xt = a.nodes_f[nd];  // converted once per call, not per tree
    nx0 = xt.x;
    nx1 = xt.y;
    t = xt.z;
    const PhiloxPath np = philox_path(0u, node, 1u, a.rk);
    nw0 = np.r0_w0;  // hi(M1 node) ^ rk0 (the tree index is XORed in per tree)
    nw1 = np.r0_w1;
  };
  // start tree g (g < gend)
  auto begin_tree = [&]() {
    if (g >= node_end) refresh_node();
    pw0 = nw0 ^ (g + kbase);
    x0 = nx0;
    x1 = nx1;
    tb = 0.f;
    id = 0;
    next_id = 1;
    sp = 0;
    ph = 1.0f;
    pl = 0.0f;
    seg0 = my_cnt;
  };
  // move to the reserve run when the current one is used up; false if none
  auto have_tree = [&]() -> bool {
    if (g >= gend) {
      g = ng;
      gend = ngend;
      ng = ngend;
    }
    return g < gend;
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
    if (!active && have_tree()) {
      begin_tree();
      active = true;
    }
    my_segs += my_cnt - my_folded;
    my_folded = my_cnt;
    if (!__any_sync(kFull, active)) {
      if (exhausted) break;
      continue;
    }
    // ---- kTrips segments per lane before the warp looks at its reserves
    // again (a lane whose runs run dry idles for the rest of them)
#pragma unroll 1
    for (int trip = 0; trip < kBranchTrips; ++trip) {
      if (!active) continue;
      const uint4 w = philox10_path(id, PhiloxPath{pw0, nw1, 1u}, a.rk);  // Philox((id, tree, node, 1))
      const float life = 0.5f * neg2log(unif_f(w.x)) * a.inv_beta;  // -ln U / beta
      float tend = tb + life;
      const bool reaches = tend >= t;
      tend = reaches ? t : tend;
      float z0, z1;
      box_muller<float>(w.y, w.z, z0, z1);
      const float h = sqrt_approx(tend - tb);
      x0 += h * z0;
      if (D == 2) x1 += h * z1;
      ++my_cnt;
      uint32_t k = 2;
      float mark = 1.0f;
      if constexpr (!kBinary) {
        // inverse CDF of q: the number of cumulative sums at or below U(w3)
        const float u3 = unif_f(w.w);
        k = 0;
#pragma unroll
        for (int kk = 0; kk < kMaxOffspring; ++kk)
          k += (kk < a.K && u3 >= a.cum[kk]) ? 1u : 0u;
        mark = a.ratio[k];
      }
      // psi for every lane (cheaper than a divergent branch), used at t
      const float psi = kPsi >= 0 ? psi_value<D, (kPsi >= 0 ? kPsi : 0)>(a, x0, x1)
                                  : psi_eval<D>(a, x0, x1);
      ff_mul(ph, pl, reaches ? psi : mark);
      // a branching particle: its first child continues in place, the others
      // wait on the stack; a tree over either cap is discarded
      const bool bad =
          !reaches && (next_id + k > max_particles || sp + static_cast<int>(k) > max_depth);
      const bool branch = !reaches && !bad && k > 0;
      const bool ends = !bad && (reaches || k == 0);  // the particle has no child to follow
      const bool pop = ends && sp > 0;
      const bool done = bad || (ends && sp == 0);
      if constexpr (kBinary) {
        // the second child goes to slot sp whatever happens (sp < max_depth
        // always holds, and the slot is above the top unless the particle
        // branches); the top is read whatever happens and used on a pop
        stk[sp] = make_float4(x0, x1, tend, __uint_as_float(next_id + 1u));
        const float4 p = stk[sp > 0 ? sp - 1 : 0];
        sp += branch ? 1 : (pop ? -1 : 0);
        x0 = pop ? p.x : x0;
        x1 = pop ? p.y : x1;
        tb = pop ? p.z : (branch ? tend : tb);
        id = pop ? __float_as_uint(p.w) : (branch ? next_id : id);
        next_id += branch ? 2u : 0u;
      } else {
        if (branch) {
          for (uint32_t c = k - 1; c >= 1; --c)
            stk[sp++] = make_float4(x0, x1, tend, __uint_as_float(next_id + c));
          id = next_id;
          tb = tend;
          next_id += k;
        }
        if (pop) {
          const float4 p = stk[--sp];
          x0 = p.x;
          x1 = p.y;
          tb = p.z;
          id = __float_as_uint(p.w);
        }
      }
      if (done) {
        // the tree is done: its score, then the next tree of the lane's runs
        a.score[g] = bad ? NAN : ph + pl;
        if (a.segs) {
          const int32_t segments = static_cast<int32_t>(my_cnt - seg0);
          a.segs[g] = bad ? -segments : segments;
        }
        if (bad) {
          ++my_disc;
          if (a.flags) atomicOr(a.flags + node, kNodeDiscarded);
        }
      }
      g += done ? 1u : 0u;
      if (done && g >= gend) {
        g = ng;
        gend = ngend;
        ng = ngend;
      }
      active = !done || g < gend;
      if (done && active) {
        if (g >= node_end) refresh_node();
        pw0 = nw0 ^ (g + kbase);
        x0 = nx0;
        x1 = nx1;
        tb = 0.f;
        id = 0;
        next_id = 1;
        sp = 0;
        ph = 1.0f;
        pl = 0.0f;
        seg0 = my_cnt;
      }
    }
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    my_segs += __shfl_xor_sync(kFull, my_segs, m);
    my_disc += __shfl_xor_sync(kFull, my_disc, m);
  }
  if (lane == 0) {
    if (my_segs) atomicAdd(&a.counters[0], my_segs);
    if (my_disc) atomicAdd(&a.counters[1], static_cast<unsigned long long>(my_disc));
  }
}

}  // namespace pdd
