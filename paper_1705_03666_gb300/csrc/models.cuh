// models.cuh -- PDE families and domains for the path kernels.
//
// A model supplies, in the paper's elliptic form (Eq. 2.3-2.4, Sec. 2.2)
//   (1/2) sigma^2 Lap u + b . grad u + c u + f = 0 in Omega,  u = g on dOmega,
// the drift b, the killing rate c (the paper's c <= 0), the source f and the
// boundary data g, evaluated in the path precision R.  A geometry supplies the
// closed/open membership tests, the faces used by the bridge exit test, the
// first crossing of a step segment and projections onto faces.
#pragma once

#include "common.cuh"

namespace pdd {

constexpr int kMaxParams = 96;

// Problem constants passed by value with every launch.
struct ModelConst {
  double prm[kMaxParams];
  float prmf[kMaxParams];
  int32_t n_params;
};

template <typename R> __device__ __forceinline__ R prm(const ModelConst &mc, int i);
template <> __device__ __forceinline__ float prm<float>(const ModelConst &mc, int i) { return mc.prmf[i]; }
template <> __device__ __forceinline__ double prm<double>(const ModelConst &mc, int i) { return mc.prm[i]; }

// ---------------------------------------------------------------------------
// Eq. 1.1 with harmonic data g = e^x cos y (no drift, killing or source).
// ---------------------------------------------------------------------------
struct LaplaceExpCos {
  static constexpr int D = 2;
  static constexpr bool kDrift = false, kSource = false;
  static constexpr unsigned kDriftAxes = 0u;  // axes whose drift can be nonzero
  static constexpr int kKill = 0;  // 0: none, 1: constant, 2: variable
  template <typename R>
  __device__ __forceinline__ static void coeffs(const ModelConst &, const R *, R *, R &) {}
  template <typename R>
  __device__ __forceinline__ static R g(const ModelConst &, const R *x) {
    return m_exp(x[0]) * m_cos(x[1]);
  }
};

// ---------------------------------------------------------------------------
// (1/2) Lap u + b . grad u - u = F on [0,1]^3, b = (0.5 sin 2 pi y,
// 0.5 cos 2 pi x, 0), manufactured from u = sin(pi x) sin(pi y) e^z.
// Paper form: c = -1 (constant), f = -F.  With sx = sin(pi x) etc.:
//   b0 = sy cy, b1 = 1/2 - sx^2,
//   F  = ((1 - 2 pi^2)/2 - 1) u + pi (sy cy) cx sy e^z + pi (1/2 - sx^2) sx cy e^z.
// ---------------------------------------------------------------------------
struct EllipticManufactured {
  static constexpr int D = 3;
  static constexpr bool kDrift = true, kSource = true;
  static constexpr unsigned kDriftAxes = 3u;  // b2 = 0
  static constexpr int kKill = 1;  // c = -1
  template <typename R>
  __device__ __forceinline__ static void coeffs(const ModelConst &, const R *x, R *b, R &f) {
    R sx, cx, sy, cy;
    sincospi01(x[0], &sx, &cx);
    sincospi01(x[1], &sy, &cy);
    const R ez = exp_fast(x[2]);
    const R syz = sy * ez;
    const R b0 = sy * cy;
    const R b1 = R(0.5) - sx * sx;
    b[0] = b0;
    b[1] = b1;
    b[2] = R(0);
    constexpr double kPi = 3.14159265358979323846;
    const R a_u = R(0.5 * (1.0 - 2.0 * kPi * kPi) - 1.0);
    const R F = a_u * sx * syz + R(kPi) * (b0 * cx * syz + b1 * sx * cy * ez);
    f = -F;
  }
  template <typename R>
  __device__ __forceinline__ static R g(const ModelConst &, const R *x) {
    return m_sinpi(x[0]) * m_sinpi(x[1]) * m_exp(x[2]);
  }
};

// ---------------------------------------------------------------------------
// Poisson problem (1/2) Lap u + b_phi . grad u = -1 (paper's f = 1) with
// Fourier boundary data g_theta.  params = theta[64] (theta[8m+n]) then phi[16].
//   g  = sum_{m,n<8} theta_mn cos(m pi x) cos(n pi y),
//   b  = (sum_{j=1..8} phi_j sin(j pi y), sum_{j=1..8} phi_{8+j} sin(j pi x)).
// sin(j pi t) and cos(m pi t) come from the Chebyshev recurrences
//   s_{j+1} = 2 cos(pi t) s_j - s_{j-1},  c_{m+1} = 2 cos(pi t) c_m - c_{m-1}.
// ---------------------------------------------------------------------------
struct PoissonFourier {
  static constexpr int D = 2;
  static constexpr bool kDrift = true, kSource = true;
  static constexpr unsigned kDriftAxes = 3u;
  static constexpr int kKill = 0;
  template <typename R>
  __device__ __forceinline__ static void sines(R t, R *s) {  // s[j-1] = sin(j pi t), t in [0,1]
    R s1, c1;
    sincospi01(t, &s1, &c1);
    const R two_c = R(2) * c1;
    s[0] = s1;
    s[1] = two_c * s1;
#pragma unroll
    for (int j = 2; j < 8; ++j) s[j] = two_c * s[j - 1] - s[j - 2];
  }
  template <typename R>
  __device__ __forceinline__ static void cosines(R t, R *c) {  // c[m] = cos(m pi t)
    R s1, c1;
    m_sincospi(t, &s1, &c1);
    const R two_c = R(2) * c1;
    c[0] = R(1);
    c[1] = c1;
#pragma unroll
    for (int m = 2; m < 8; ++m) c[m] = two_c * c[m - 1] - c[m - 2];
  }
  template <typename R>
  __device__ __forceinline__ static void coeffs(const ModelConst &mc, const R *x, R *b, R &f) {
    R sy[8], sx[8];
    sines(x[1], sy);
    sines(x[0], sx);
    R b0 = R(0), b1 = R(0);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      b0 += prm<R>(mc, 64 + j) * sy[j];
      b1 += prm<R>(mc, 72 + j) * sx[j];
    }
    b[0] = b0;
    b[1] = b1;
    f = R(1);
  }
  // coeffs plus the likelihood-ratio increments of the 16 drift weights:
  // L_j += xi . db/dphi_j (X), db/dphi_j = (sin(j pi y), 0) for j <= 8 and
  // (0, sin((j-8) pi x)) for j > 8 (scaled by sqrt(dt)/sigma at the exit).
  template <typename R>
  __device__ __forceinline__ static void coeffs_lr(const ModelConst &mc, const R *x, R *b, R &f,
                                                   const R *xi, R *L) {
    R sy[8], sx[8];
    sines(x[1], sy);
    sines(x[0], sx);
    R b0 = R(0), b1 = R(0);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      b0 += prm<R>(mc, 64 + j) * sy[j];
      b1 += prm<R>(mc, 72 + j) * sx[j];
      L[j] += xi[0] * sy[j];
      L[8 + j] += xi[1] * sx[j];
    }
    b[0] = b0;
    b[1] = b1;
    f = R(1);
  }
  template <typename R>
  __device__ __forceinline__ static R g(const ModelConst &mc, const R *x) {
    R cx[8], cy[8];
    cosines(x[0], cx);
    cosines(x[1], cy);
    R s = R(0);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      R row = R(0);
#pragma unroll
      for (int n = 0; n < 8; ++n) row += prm<R>(mc, 8 * m + n) * cy[n];
      s += cx[m] * row;
    }
    return s;
  }
};

// ---------------------------------------------------------------------------
// Geometry: the box [0,1]^D.  Face j = 2k + s lies on x_k = s.
// ---------------------------------------------------------------------------
template <int Dim>
struct Box {
  static constexpr int D = Dim;
  static constexpr int kFaces = 2 * D;
  static constexpr bool kFastScreen = true;  // one candidate face per axis

  template <typename R>
  __device__ __forceinline__ static bool inside_closed(const R *x) {
    bool in = true;
#pragma unroll
    for (int k = 0; k < D; ++k) in = in && (x[k] >= R(0)) && (x[k] <= R(1));
    return in;
  }
  template <typename R>
  __device__ __forceinline__ static bool inside_open(const R *x) {
    bool in = true;
#pragma unroll
    for (int k = 0; k < D; ++k) in = in && (x[k] > R(0)) && (x[k] < R(1));
    return in;
  }
  // Distance to the plane of face j, positive on the domain side.
  template <typename R>
  __device__ __forceinline__ static R face_dist(int j, const R *x) {
    const R v = x[j >> 1];
    return (j & 1) ? R(1) - v : v;
  }
  // Screening of a step X -> X' (X in the closed box): the smallest
  //   d d' = min over k of min(x_k x'_k, (1 - x_k)(1 - x'_k))
  // over the face of each axis that can be within bridge reach (the other
  // one cannot while sigma^2 dt <= 1/36).  A result > 0 puts X' strictly
  // inside the box: with x_k in [0, 1], both products of an axis are positive
  // only for x'_k in (0, 1) (a rounded product keeps its sign; an underflow
  // to zero gives 0).
  template <typename R>
  __device__ __forceinline__ static R screen_mn(const R *x0, const R *x1) {
    R p[2 * D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      p[2 * k] = x0[k] * x1[k];
      p[2 * k + 1] = (R(1) - x0[k]) * (R(1) - x1[k]);
    }
    if constexpr (D == 1) return fmin(p[0], p[1]);
    else if constexpr (D == 2) return fmin(min3(p[0], p[1], p[2]), p[3]);
    else return fmin(min3(p[0], p[1], p[2]), min3(p[3], p[4], p[5]));
  }
  // The exact smallest d d' is also the lower bound general callers screen
  // with (LShape::screen_lb).
  template <typename R>
  __device__ __forceinline__ static R screen_lb(const R *x0, const R *x1) {
    return screen_mn<R>(x0, x1);
  }
  // Second smallest of m[0..D-1] (D <= 3): below the reach threshold means
  // the step is within reach of two faces (an edge or a corner).
  template <typename R>
  __device__ __forceinline__ static R second_min(const R *m) {
    if constexpr (D == 1) return R(1);
    else if constexpr (D == 2) return fmax(m[0], m[1]);
    else return fmax(fmin(m[0], m[1]), fmin(fmax(m[0], m[1]), m[2]));
  }
  // Candidate faces with their d d' (rarely needed: corners and exits).
  template <typename R>
  __device__ __forceinline__ static R screen(const R *x0, const R *x1, R *prod, int *face) {
    R mn = R(1);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const R lo = x0[k] * x1[k], hi = (R(1) - x0[k]) * (R(1) - x1[k]);
      const bool up = hi < lo;
      prod[k] = up ? hi : lo;
      face[k] = 2 * k + (up ? 1 : 0);
      mn = fmin(mn, prod[k]);
    }
    return mn;
  }
  template <typename R>
  __device__ __forceinline__ static void project(int j, R *x) {
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k == (j >> 1)) x[k] = R(j & 1);
  }
  // First crossing of the segment x0 -> x1 (x0 inside, x1 outside): the
  // smallest crossing parameter over the violated coordinates; the crossed
  // coordinate is set exactly to its face and the rest clamped to [0,1].
  template <typename R>
  __device__ __forceinline__ static void segment_exit(const R *x0, const R *x1, R *xe) {
    R tb = R(2);
    int kb = 0;
    R vb = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (x1[k] < R(0)) {
        const R t = x0[k] / (x0[k] - x1[k]);
        if (t < tb) { tb = t; kb = k; vb = R(0); }
      } else if (x1[k] > R(1)) {
        const R t = (R(1) - x0[k]) / (x1[k] - x0[k]);
        if (t < tb) { tb = t; kb = k; vb = R(1); }
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      R v = x0[k] + tb * (x1[k] - x0[k]);
      v = (k == kb) ? vb : v;
      xe[k] = fmin(R(1), fmax(R(0), v));
    }
  }
  template <typename R>
  __device__ __forceinline__ static int nearest_face(const R *x) {
    int jb = 0;
    R db = face_dist<R>(0, x);
#pragma unroll
    for (int j = 1; j < kFaces; ++j) {
      const R d = face_dist<R>(j, x);
      if (d < db) { db = d; jb = j; }
    }
    return jb;
  }
};

// ---------------------------------------------------------------------------
// Geometry: the L-shape [0,1]^2 minus the open notch (1/2,1] x (1/2,1].
// Faces 0-3 are the four sides of the square (as half-planes, face 2k+s on
// x_k = s); face 4 is the notch edge y = 1/2, x in [1/2, 1] (domain side
// y < 1/2) and face 5 the notch edge x = 1/2, y in [1/2, 1] (domain side
// x < 1/2).  Distances to the notch edges are distances to the segments, so
// points away from an edge see no crossing (the re-entrant corner is handled
// by the half-plane formula only approximately, like every corner).
// ---------------------------------------------------------------------------
struct LShape {
  static constexpr int D = 2;
  static constexpr int kFaces = 6;
  static constexpr bool kFastScreen = false;

  template <typename R>
  __device__ __forceinline__ static bool inside_closed(const R *x) {
    return x[0] >= R(0) && x[0] <= R(1) && x[1] >= R(0) && x[1] <= R(1) &&
           !(x[0] > R(0.5) && x[1] > R(0.5));
  }
  template <typename R>
  __device__ __forceinline__ static bool inside_open(const R *x) {
    return x[0] > R(0) && x[0] < R(1) && x[1] > R(0) && x[1] < R(1) &&
           !(x[0] >= R(0.5) && x[1] >= R(0.5));
  }
  template <typename R>
  __device__ __forceinline__ static R face_dist(int j, const R *x) {
    if (j < 4) {
      const R v = x[j >> 1];
      return (j & 1) ? R(1) - v : v;
    }
    const R a = j == 4 ? x[0] : x[1];          // along the edge
    const R b = R(0.5) - (j == 4 ? x[1] : x[0]);  // towards the domain
    if (a >= R(0.5)) return b;
    const R da = R(0.5) - a;
    return m_sqrt(da * da + b * b);
  }
  // Lower bound on the smallest face_dist(j, x0) * face_dist(j, x1) over the
  // six faces (x0 in the closed domain), without square roots: the sides'
  // products are exact; a notch edge's distance to a point beside it
  // (a < 1/2), sqrt(da^2 + b^2), is bounded below by max(da, |b|), and is b
  // itself beyond it.  A result > 0 puts x1 inside the closed domain: a
  // point in the notch has b < 0 on the edge y = 1/2 (face 4), whose product
  // with x0's nonnegative bound is then <= 0.
  template <typename R>
  __device__ __forceinline__ static R notch_dist_lb(int j, const R *x) {
    const R a = j == 4 ? x[0] : x[1];
    const R b = R(0.5) - (j == 4 ? x[1] : x[0]);
    return a >= R(0.5) ? b : fmax(R(0.5) - a, fabs(b));
  }
  template <typename R>
  __device__ __forceinline__ static R screen_lb(const R *x0, const R *x1) {
    const R s0 = x0[0] * x1[0], s1 = (R(1) - x0[0]) * (R(1) - x1[0]);
    const R s2 = x0[1] * x1[1], s3 = (R(1) - x0[1]) * (R(1) - x1[1]);
    const R n4 = notch_dist_lb<R>(4, x0) * notch_dist_lb<R>(4, x1);
    const R n5 = notch_dist_lb<R>(5, x0) * notch_dist_lb<R>(5, x1);
    return fmin(min3(s0, s1, s2), min3(s3, n4, n5));
  }
  template <typename R>
  __device__ __forceinline__ static void project(int j, R *x) {
    if (j < 4) {
      x[j >> 1] = R(j & 1);
    } else if (j == 4) {
      x[1] = R(0.5);
      x[0] = fmax(x[0], R(0.5));
    } else {
      x[0] = R(0.5);
      x[1] = fmax(x[1], R(0.5));
    }
  }
  // First crossing of x0 -> x1 (x0 inside, x1 outside): the square's sides
  // as for the box, and entry into the notch at the later of the parameters
  // where each coordinate passes 1/2.
  template <typename R>
  __device__ __forceinline__ static void segment_exit(const R *x0, const R *x1, R *xe) {
    R tb = R(2), vb = R(0);
    int kb = -1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (x1[k] < R(0)) {
        const R t = x0[k] / (x0[k] - x1[k]);
        if (t < tb) { tb = t; kb = k; vb = R(0); }
      } else if (x1[k] > R(1)) {
        const R t = (R(1) - x0[k]) / (x1[k] - x0[k]);
        if (t < tb) { tb = t; kb = k; vb = R(1); }
      }
    }
    R lo = R(-1e30), hi = R(1e30);
    int kent = -1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const R a = x0[k], d = x1[k] - x0[k];
      R tl, th;
      if (d == R(0)) {
        if (a > R(0.5)) { tl = R(0); th = R(1); } else { tl = R(2); th = R(-1); }
      } else if (d > R(0)) {
        tl = (R(0.5) - a) / d; th = R(2);
      } else {
        tl = R(-1); th = (R(0.5) - a) / d;
      }
      if (tl > lo) { lo = tl; kent = k; }
      if (th < hi) hi = th;
    }
    if (kent >= 0 && lo < hi && lo <= R(1) && hi > R(0)) {
      const R tent = lo > R(0) ? lo : R(0);
      if (tent < tb) { tb = tent; kb = kent; vb = R(0.5); }
    }
    if (kb < 0) {
#pragma unroll
      for (int k = 0; k < 2; ++k) xe[k] = fmin(R(1), fmax(R(0), x1[k]));
      return;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      R v = x0[k] + tb * (x1[k] - x0[k]);
      v = (k == kb) ? vb : v;
      xe[k] = fmin(R(1), fmax(R(0), v));
    }
  }
  template <typename R>
  __device__ __forceinline__ static int nearest_face(const R *x) {
    int jb = 0;
    R db = face_dist<R>(0, x);
#pragma unroll
    for (int j = 1; j < kFaces; ++j) {
      const R d = face_dist<R>(j, x);
      if (d < db) { db = d; jb = j; }
    }
    return jb;
  }
};

}  // namespace pdd
