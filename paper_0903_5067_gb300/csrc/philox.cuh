// Counter-based random numbers for the fluctuating terms.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3" (SC'11): ten rounds, each multiplying counter words 0 and 2 by the two
// round multipliers, exchanging the high/low product halves into the other lanes and
// xoring in the key, the key advanced by the two Weyl increments between rounds.
//
// Stream layout (library convention): key = (seed_lo32, tag | replica << 8); counter =
// (step, index, call, 0); tag 0 = fluid modes (3 calls per node, each cut into six uniforms
// of 21 bits), tag 1 = beads (1 call), tag 3 = Brownian dynamics (1 call).
#pragma once
#include <stdint.h>

namespace gblb {

struct U4 {
  uint32_t x, y, z, w;
};

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = mulhi32(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = mulhi32(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

// The ten round keys of a Philox key, computed once on the host and passed in a kernel's
// parameter block, so that each round costs two 32x32->64-bit multiplies and two
// three-input xors.
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

inline RoundKeys make_round_keys(uint32_t k0, uint32_t k1) {
  RoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return rk;
}

__device__ __forceinline__ U4 philox4x32_10_rk(U4 c, const RoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c.z;
    c = U4{(uint32_t)(p1 >> 32) ^ c.y ^ rk.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk.k1[r],
           (uint32_t)p0};
  }
  return c;
}

// u = ((x >> 9) + 1/2) * 2^-23 in (0, 1): 23 random bits, exact in float and double.
__device__ __forceinline__ float uniform_f32(uint32_t x) {
  // 1 + (x>>9) 2^-23 in [1, 2), minus (1 - 2^-24): exact (Sterbenz), result representable
  return __fsub_rn(__uint_as_float(0x3f800000u | (x >> 9)), 0x1.fffffep-1f);
}
__host__ __device__ __forceinline__ double uniform_f64(uint32_t x) {
  return ((double)(x >> 9) + 0.5) * 0x1p-23;
}

// Box & Muller (1958) with the angle taken in (-pi, pi): (u0, u1) -> two independent standard
// normals  g0 = sqrt(-2 ln u0) cos(theta),  g1 = sqrt(-2 ln u0) sin(theta),  theta = 2 pi (u1 - 1/2)
// (the hardware sine and cosine are accurate on that range).
__device__ __forceinline__ void box_muller(float u0, float u1, float& g0, float& g1) {
  const float r = sqrtf(-2.0f * logf(u0));
  float s, c;
  __sincosf(6.28318530717958647692f * (u1 - 0.5f), &s, &c);
  g0 = r * c;
  g1 = r * s;
}
__device__ __forceinline__ void box_muller(double u0, double u1, double& g0, double& g1) {
  const double r = sqrt(-2.0 * log(u0));
  double s, c;
  sincospi(2.0 * u1 - 1.0, &s, &c);
  g0 = r * c;
  g1 = r * s;
}

// ---------------------------------------------------------------------------------------
// The fluid's noise stream.  Call c = 0, 1, 2 with counter (step, node, c, 0) gives a 128-bit
// string w_0 .. w_3 (word j holds bits 32 j .. 32 j + 31, least significant first), cut into
// six uniforms: uniform i = 0..5 takes the 21 bits 21 i .. 21 i + 20 as an integer k,
// u = (k + 1/2) 2^-21.  Box-Muller pair p = 3 c + q turns uniforms (2q, 2q + 1) of call c into
// (g_2p, g_2p+1); mode k = 4..18 takes g_(k-4).  The stress modes 4..9 thus draw on call 0
// alone; the kinetic modes 10..18 on calls 1 and 2 (pairs 3..7; g_15 and pair 8 are not
// formed).
// ---------------------------------------------------------------------------------------
template <int J>
__device__ __forceinline__ uint32_t word_of(const U4& w) {
  static_assert(J >= 0 && J < 4, "a Philox call has four words");
  return J == 0 ? w.x : J == 1 ? w.y : J == 2 ? w.z : w.w;
}

// uniform I of one call's words, as the 21-bit integer k (double) or as the float
// 1 + k 2^-21 (the integer placed in the top 21 mantissa bits)
template <int I>
__device__ __forceinline__ uint32_t fluid_k21(const U4& w) {
  constexpr int b = 21 * I, q = b / 32, s = b % 32;
  static_assert(b + 21 <= 128, "six uniforms per call");
  if constexpr (s + 21 <= 32)
    return (word_of<q>(w) >> s) & 0x1fffffu;
  else
    return __funnelshift_r(word_of<q>(w), word_of<q + 1>(w), s) & 0x1fffffu;
}
template <int I>
__device__ __forceinline__ float fluid_mant21(const U4& w) {
  constexpr int b = 21 * I;
  static_assert(b + 21 <= 128, "six uniforms per call");
  uint32_t v;  // bits b .. b + 20 of the call's string at bit positions 2 .. 22
  if constexpr (b == 0) {
    v = w.x << 2;
  } else {
    constexpr int q = (b - 2) / 32, s = (b - 2) % 32;
    if constexpr (s + 23 <= 32 || q == 3)  // (q == 3: bits up to b + 20 < 128 lie in word 3)
      v = word_of<q>(w) >> s;
    else
      v = __funnelshift_r(word_of<q>(w), word_of<q + 1>(w), s);
  }
  return __uint_as_float(0x3f800000u | (v & 0x7ffffcu));
}

// Hardware approximations of the special-function unit in their flush-to-zero forms.  The
// plain forms (as __log2f, rsqrtf, __sinf, __cosf compile without -ftz) wrap each unit
// operation in a rescaling for subnormal arguments, several instructions each; every argument
// below is a normal number by construction, where both forms give the same result.
__device__ __forceinline__ float approx_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float approx_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float approx_sin(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float approx_cos(float x) {
  float r;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float approx_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Per-node scale of the fluid Gaussians: they come out multiplied by sqrt(rho) (rho > 0;
// non-positive densities draw no noise).  Single precision folds rho into the Box-Muller
// radius, r = sqrt(rho x) with x = -2 ln u0, through one constant cl = -2 ln(2) rho:
// rho x = cl log2(u0); a non-positive rho enters as 1e-30, whose noise lies below the
// rounding of any population.
template <class R>
struct NoiseScale {
  R sr;  // sqrt(rho), 0 for rho <= 0
  __device__ __forceinline__ explicit NoiseScale(R rho) : sr(rho > R(0) ? sqrt(rho) : R(0)) {}
};
template <>
struct NoiseScale<float> {
  float cl;
  __device__ __forceinline__ explicit NoiseScale(float rho) : cl(-1.38629436112f * (rho > 0.0f ? rho : 1.0e-30f)) {}
};

// Box-Muller pair Q (0..2) of one call's words, times sqrt(rho) (Box & Muller 1958, angle in
// (-pi, pi)).  Single precision: u0 and the angle come from the uniforms as floats 1 + k 2^-21,
// both exact steps; log2, 1/sqrt, sin and cos on the special-function unit.  Near u0 = 1 the hardware log2's absolute error (2^-22) would dominate
// -ln u0; there (t = 1 - u0 < 1e-3) log2(u0) is the series -(t + t^2/2 + t^3/3) / ln 2
// (truncation below 3e-10 relative).  SECOND = false forms g0 only.
template <int Q, bool SECOND>
__device__ __forceinline__ void fluid_pair(const U4& w, const NoiseScale<float>& ns, float& g0, float& g1) {
  const float u0 = fluid_mant21<2 * Q>(w) - 0x1.fffff8p-1f;  // (k0 + 1/2) 2^-21
  const float t = 1.0f - u0;
  const float l2 = t < 1.0e-3f ? t * (-1.44269504f + t * (-0.721347520f + t * -0.480898347f)) : approx_lg2(u0);
  const float x = ns.cl * l2;  // rho (-2 ln u0): >= 1e-30 * 2^-22, a normal number
  const float r = x * approx_rsqrt(x);
  const float d = fluid_mant21<2 * Q + 1>(w) - 1.5f;  // u1 - 1/2 - 2^-22, exact
  const float th = fmaf(6.28318530717958647692f, d, 1.49802816e-6f);  // 2 pi (u1 - 1/2), |th| >= 1.5e-6
  g0 = r * approx_cos(th);
  if (SECOND) g1 = r * approx_sin(th);
}
template <int Q, bool SECOND>
__device__ __forceinline__ void fluid_pair(const U4& w, const NoiseScale<double>& ns, double& g0, double& g1) {
  const double u0 = ((double)fluid_k21<2 * Q>(w) + 0.5) * 0x1p-21;
  const double u1 = ((double)fluid_k21<2 * Q + 1>(w) + 0.5) * 0x1p-21;
  const double r = ns.sr * sqrt(-2.0 * log(u0));
  double s, c;
  sincospi(2.0 * u1 - 1.0, &s, &c);
  g0 = r * c;
  if (SECOND) g1 = r * s;
}

template <int P, bool SECOND = true, class R, class Emit>
__device__ __forceinline__ void fluid_pair_emit(const U4& w, const NoiseScale<R>& ns, Emit& emit) {
  R g0, g1;
  fluid_pair<P % 3, SECOND>(w, ns, g0, g1);
  emit(2 * P, g0);
  if (SECOND) emit(2 * P + 1, g1);
}

// The Gaussians of one node, times sqrt(rho), handed out as emit(j, g_j) for mode 4 + j:
// j = 0..5 (stress modes) always, j = 6..14 (kinetic modes) when `kinetic`.
template <class R, class Emit>
__device__ __forceinline__ void fluid_noise(uint32_t step, uint32_t node, const RoundKeys& rk, bool kinetic,
                                            const NoiseScale<R>& ns, Emit emit) {
  U4 w = philox4x32_10_rk(U4{step, node, 0u, 0u}, rk);
  fluid_pair_emit<0>(w, ns, emit);
  fluid_pair_emit<1>(w, ns, emit);
  fluid_pair_emit<2>(w, ns, emit);
  if (!kinetic) return;
  w = philox4x32_10_rk(U4{step, node, 1u, 0u}, rk);
  fluid_pair_emit<3>(w, ns, emit);
  fluid_pair_emit<4>(w, ns, emit);
  fluid_pair_emit<5>(w, ns, emit);
  w = philox4x32_10_rk(U4{step, node, 2u, 0u}, rk);
  fluid_pair_emit<6>(w, ns, emit);
  fluid_pair_emit<7, false>(w, ns, emit);
}

template <class R>
__device__ __forceinline__ R uniform01(uint32_t x);
template <>
__device__ __forceinline__ float uniform01<float>(uint32_t x) { return uniform_f32(x); }
template <>
__device__ __forceinline__ double uniform01<double>(uint32_t x) { return uniform_f64(x); }

// Four standard normals from one Philox call with counter (step, index, call, 0).
template <class R>
__device__ __forceinline__ void gauss4(uint32_t step, uint32_t index, uint32_t call, uint32_t k0,
                                       uint32_t k1, R g[4]) {
  const U4 r = philox4x32_10(U4{step, index, call, 0u}, k0, k1);
  box_muller(uniform01<R>(r.x), uniform01<R>(r.y), g[0], g[1]);
  box_muller(uniform01<R>(r.z), uniform01<R>(r.w), g[2], g[3]);
}

}  // namespace gblb
