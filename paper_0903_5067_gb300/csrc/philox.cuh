// Counter-based random numbers for the fluctuating terms.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3" (SC'11): ten rounds, each multiplying counter words 0 and 2 by the two
// round multipliers, exchanging the high/low product halves into the other lanes and
// xoring in the key, the key advanced by the two Weyl increments between rounds.
//
// Stream layout (library convention): key = (seed_lo32, tag | replica << 8); counter =
// (step, index, call, 0); tag 0 = fluid modes (4 calls per node), tag 1 = beads (1 call).
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

// Box & Muller (1958): (u0, u1) -> two independent standard normals
//   g0 = sqrt(-2 ln u0) cos(2 pi u1),  g1 = sqrt(-2 ln u0) sin(2 pi u1).
// Single precision: the angle is reduced to (-pi, pi) through cos(2 pi u) = -cos(2 pi (u - 1/2))
// so that the hardware sine/cosine stay in their accurate range.
__device__ __forceinline__ void box_muller(float u0, float u1, float& g0, float& g1) {
  const float r = sqrtf(-2.0f * logf(u0));
  const float th = 6.28318530717958647692f * (u1 - 0.5f);
  float s, c;
  __sincosf(th, &s, &c);
  g0 = -r * c;
  g1 = -r * s;
}
__device__ __forceinline__ void box_muller(double u0, double u1, double& g0, double& g1) {
  const double r = sqrt(-2.0 * log(u0));
  double s, c;
  sincospi(2.0 * u1, &s, &c);
  g0 = r * c;
  g1 = r * s;
}

// -ln(u), u in (0, 1), single precision.  The hardware log2 has an absolute error bound
// of 2^-22 on [0.5, 2], which would dominate the result near u = 1 (where the Box-Muller
// radius is small); there, with t = 1 - u (exact), -ln(1 - t) is summed as its Taylor series
// t + t^2/2 + t^3/3 (truncation below 3e-10 relative for t < 1e-3).
__device__ __forceinline__ float neg_log_unit(float u) {
  const float t = 1.0f - u;
  const float series = t * (1.0f + t * (0.5f + t * 0.333333343f));
  const float fast = -0.693147182f * __log2f(u);
  return t < 1.0e-3f ? series : fast;
}

// Box-Muller in single precision on the hardware transcendental units, both normals
// multiplied by `scale`: r = sqrt(-2 ln u0) as x * rsqrt(x), angle reduced to (-pi, pi)
// through cos(2 pi u) = -cos(2 pi (u - 1/2)).
__device__ __forceinline__ void box_muller_fast(float u0, float u1, float scale, float& g0, float& g1) {
  const float x = 2.0f * neg_log_unit(u0);
  const float r = -scale * (x * rsqrtf(x));
  float s, c;
  __sincosf(6.28318530717958647692f * (u1 - 0.5f), &s, &c);
  g0 = r * c;
  g1 = r * s;
}

template <class R>
__device__ __forceinline__ void box_muller_lb(R u0, R u1, R scale, R& g0, R& g1) {
  box_muller(u0, u1, g0, g1);
  g0 *= scale;
  g1 *= scale;
}
template <>
__device__ __forceinline__ void box_muller_lb<float>(float u0, float u1, float scale, float& g0, float& g1) {
  box_muller_fast(u0, u1, scale, g0, g1);
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

// Four standard normals times `scale` from one Philox call (precomputed round keys), the
// fluid's transform: fast single-precision Box-Muller for float, full precision for double.
template <class R>
__device__ __forceinline__ void gauss4_rk(uint32_t step, uint32_t index, uint32_t call, const RoundKeys& rk,
                                          R scale, R g[4]) {
  const U4 r = philox4x32_10_rk(U4{step, index, call, 0u}, rk);
  box_muller_lb<R>(uniform01<R>(r.x), uniform01<R>(r.y), scale, g[0], g[1]);
  box_muller_lb<R>(uniform01<R>(r.z), uniform01<R>(r.w), scale, g[2], g[3]);
}

}  // namespace gblb
