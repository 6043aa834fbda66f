// common.cuh -- device building blocks shared by the PDD kernels:
// counter-based random numbers, the uniform / normal / exponential maps, math
// overloads for the two path precisions, and compensated FP64 sums.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pdd {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Ten rounds; each
// multiplies counter words 0 and 2 by the two round multipliers, keeps the
// low halves, and XORs the high halves into words 1 and 3 together with the
// round key; the key is advanced by the Weyl increments between rounds.  The
// ten round keys depend only on the seed, so the host precomputes them
// (RoundKeys) and they reach the kernel as constant-bank parameters.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct RoundKeys {
  uint32_t k[20];  // (k0 + r W0, k1 + r W1) for r = 0..9
};

inline RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0;
    rk.k[2 * r + 1] = k1;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return rk;
}

__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2,
                                          uint32_t c3, const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c0;
    const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c2;
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ rk.k[2 * r];
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ rk.k[2 * r + 1];
    c1 = static_cast<uint32_t>(p1);
    c3 = static_cast<uint32_t>(p0);
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Per-path precomputation: counter words 1 (path) and 2 (node) are fixed for
// a path and word 3 (stream tag) is a constant, so half of round one depends
// only on (path, node, tag).
struct PhiloxPath {
  uint32_t r0_w0;  // hi(M1 * node) ^ path ^ rk0   (round-one output word 0)
  uint32_t r0_w1;  // lo(M1 * node)                (round-one output word 1)
  uint32_t tag;    // counter word 3
};

__device__ __forceinline__ PhiloxPath philox_path(uint32_t path, uint32_t node,
                                                  uint32_t tag, const RoundKeys &rk) {
  const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * node;
  PhiloxPath pp;
  pp.r0_w0 = static_cast<uint32_t>(p1 >> 32) ^ path ^ rk.k[0];
  pp.r0_w1 = static_cast<uint32_t>(p1);
  pp.tag = tag;
  return pp;
}

// Same value as philox10(j, path, node, tag, rk).
__device__ __forceinline__ uint4 philox10_path(uint32_t j, const PhiloxPath &pp,
                                               const RoundKeys &rk) {
  const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * j;
  uint32_t c0 = pp.r0_w0;
  uint32_t c1 = pp.r0_w1;
  uint32_t c2 = static_cast<uint32_t>(p0 >> 32) ^ pp.tag ^ rk.k[1];
  uint32_t c3 = static_cast<uint32_t>(p0);
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    const uint64_t q0 = static_cast<uint64_t>(kPhiloxM0) * c0;
    const uint64_t q1 = static_cast<uint64_t>(kPhiloxM1) * c2;
    const uint32_t n0 = static_cast<uint32_t>(q1 >> 32) ^ c1 ^ rk.k[2 * r];
    const uint32_t n2 = static_cast<uint32_t>(q0 >> 32) ^ c3 ^ rk.k[2 * r + 1];
    c1 = static_cast<uint32_t>(q1);
    c3 = static_cast<uint32_t>(q0);
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// ---------------------------------------------------------------------------
// Uniform on (0,1): U = (floor(w / 2^9) + 1/2) 2^-23, an odd multiple of 2^-24
// that binary32 and binary64 both hold exactly (so both path precisions and
// the FP64 oracle draw the same U from the same word).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float unif_f(uint32_t w) {
  // 1 + k 2^-23 minus (1 - 2^-24): exact (Sterbenz), = (2k+1) 2^-24.  The
  // exponent bits are added (they do not overlap k), one shift-and-add.
  return __int_as_float((w >> 9) + 0x3f800000u) - 0.999999940395355224609375f;
}
__device__ __forceinline__ double unif_d(uint32_t w) {
  return static_cast<double>((w >> 9) * 2u + 1u) * 5.9604644775390625e-08;  // 2^-24
}

template <typename R> __device__ __forceinline__ R unif(uint32_t w);
template <> __device__ __forceinline__ float unif<float>(uint32_t w) { return unif_f(w); }
template <> __device__ __forceinline__ double unif<double>(uint32_t w) { return unif_d(w); }

// ---------------------------------------------------------------------------
// Math overloads (CUDA's own accurate library functions in both precisions).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_cos(float x) { return cosf(x); }
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ void m_sincospi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void m_sincospi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ float m_sinpi(float x) { return sinpif(x); }
__device__ __forceinline__ double m_sinpi(double x) { return sinpi(x); }

// Box-Muller: r = sqrt(-2 ln U_a), angle 2 pi U_b; (r cos, r sin).
template <typename R>
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, R &z0, R &z1) {
  const R r = m_sqrt(R(-2) * m_log(unif<R>(a)));
  R s, c;
  m_sincospi(R(2) * unif<R>(b), &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// binary32 Box-Muller with the hardware sine/cosine.  The angle is centred,
// theta = 2 pi (U_b - 1/2) in (-pi, pi), where the hardware sin/cos have an
// absolute error below 2^-21.4; cos(2 pi U_b) = -cos theta and
// sin(2 pi U_b) = -sin theta.  -2 ln U_a comes from the hardware log2,
// whose absolute error (~2^-22 near U_a = 1) gives r = sqrt(-2 ln U_a) an
// error ~1e-7 / r: relatively large only for the rare tiny radii, where the
// displacement r sqrt(dt) itself is tiny.  The radius is the hardware square
// root of the magnitude of the scaled log2 (near U_a = 1 the log2 may come
// out 0 or tiny and positive).
//
// -2 ln u accurate to 2e-7 relative for all u in (0, 1) (used where a single
// log sets a decision, e.g. branching lifetimes), from the atanh series:
// write u = 2^e m with m in [sqrt(1/2), sqrt(2)) (exponent split on the bit
// pattern), then ln u = e ln 2 + 2 atanh(t), t = (m - 1)/(m + 1), |t| <= 0.1716,
// atanh t = t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9 + ...), truncation below
// 3.5e-10 relative.  m - 1 is exact (Sterbenz), so the relative accuracy holds
// as u -> 1, where a hardware log2 loses it.  e is converted with the
// 1.5 * 2^23 magic constant (exact for |e| < 2^22).
__device__ __forceinline__ float neg2log(float u) {
  const uint32_t bits = __float_as_uint(u);
  const int32_t e = static_cast<int32_t>(bits - 0x3f3504f3u) >> 23;
  const float m = __uint_as_float(bits - (static_cast<uint32_t>(e) << 23));
  const float t = __fdividef(m - 1.0f, m + 1.0f);
  const float s = t * t;
  float p = fmaf(s, 1.0f / 9.0f, 1.0f / 7.0f);
  p = fmaf(s, p, 1.0f / 5.0f);
  p = fmaf(s, p, 1.0f / 3.0f);
  p = fmaf(s, p, 1.0f);
  const float ef = __int_as_float(0x4b400000 + e) - 12582912.0f;
  // -2 ln u = -2 ln2 e - 4 t p
  return fmaf(-1.3862943611198906f, ef, -4.0f * t * p);
}

// Hardware approximations (PTX .approx.ftz: one special-function-unit
// operation each).  Subnormal arguments and results are flushed to zero; the
// kernels pass normal numbers or zero (uniforms >= 2^-24, squared radii 0 or
// above 1e-8, centred angles at least 2^-24 away from 0), where the flush
// changes nothing and the subnormal scaling the non-ftz forms add around the
// operation is left out.
__device__ __forceinline__ float ex2_approx(float x) {  // 2^x, about 2 ulp relative
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {  // log2 x, abs. error ~2^-22 near 1
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {  // 1/x, about 1 ulp
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sin_approx(float x) {  // abs. error < 2^-21.4 on [-pi, pi]
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Smallest of three (one three-input min in binary32).
__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ double min3(double a, double b, double c) { return fmin(fmin(a, b), c); }

template <>
__device__ __forceinline__ void box_muller<float>(uint32_t a, uint32_t b, float &z0, float &z1) {
  // hardware log2 (absolute error ~2^-22 near u = 1, where it may return 0
  // or a tiny positive value: its magnitude is taken, an operand modifier
  // rather than a clamp) and hardware square root
  const float mr = -sqrt_approx(fabsf(1.3862943611198906f * lg2_approx(unif_f(a))));
  // theta = 2 pi (U_b - 1/2) from x = 1 + k 2^-23 (k = b >> 9, exponent bits
  // added): U_b - 1/2 = (x - 3/2) + 2^-24 with x - 3/2 exact, so theta is one
  // subtraction and one FMA, rounded once (the same value as 2 pi (U_b - 1/2)
  // formed from the uniform)
  const float xb = __int_as_float((b >> 9) + 0x3f800000u);
  const float th = fmaf(xb - 1.5f, 6.28318530717958648f, 6.28318530717958648f * 0x1p-24f);
  z0 = mr * cos_approx(th);
  z1 = mr * sin_approx(th);
}

// sin(pi x), cos(pi x) for x in [0, 1] (points of the closed unit box).  FP32:
// hardware sin/cos of pi x in [0, pi], absolute error below 2^-21.4 -- used
// for drift and source values inside the domain, never for boundary data.
__device__ __forceinline__ void sincospi01(float x, float *s, float *c) {
  const float t = 3.14159265358979324f * x;
  *s = sin_approx(t);
  *c = cos_approx(t);
}
__device__ __forceinline__ void sincospi01(double x, double *s, double *c) { sincospi(x, s, c); }

// e^x for moderate x: FP32 hardware exp2 of x log2 e (about 2 ulp).
__device__ __forceinline__ float exp_fast(float x) { return ex2_approx(1.4426950408889634f * x); }
__device__ __forceinline__ double exp_fast(double x) { return exp(x); }

// ---------------------------------------------------------------------------
// Compensated (Neumaier) FP64 accumulator and its exact merge.
// ---------------------------------------------------------------------------
struct CSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double v) {
    const double t = s + v;
    c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
  }
  __device__ __forceinline__ void merge(const CSum &o) {
    add(o.s);
    c += o.c;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

__device__ __forceinline__ CSum shfl_xor(const CSum &v, int m) {
  CSum o;
  o.s = __shfl_xor_sync(kFull, v.s, m);
  o.c = __shfl_xor_sync(kFull, v.c, m);
  return o;
}

}  // namespace pdd
