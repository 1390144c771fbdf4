// Counter-based random numbers for the fluctuating terms.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3" (SC'11): ten rounds, each multiplying counter words 0 and 2 by the two
// round multipliers, exchanging the high/low product halves into the other lanes and
// xoring in the key, the key advanced by the two Weyl increments between rounds.
//
// Stream layout (library convention): key = (seed_lo32, tag | replica << 8); counter =
// (step, index, call, 0); tag 0 = fluid modes (2 calls per node, each 32-bit word one
// Box-Muller pair), tag 1 = beads (1 call), tag 3 = Brownian dynamics (1 call).
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
// The fluid's noise stream.  Call c = 0, 1 with counter (step, node, c, 0) gives four 32-bit
// words; word j is Box-Muller pair p = 4 c + j: its 21 high bits k_r = w >> 11 give the radius
// uniform u0 = (k_r + 1/2) 2^-21, its 11 low bits k_a = w & 0x7ff the angle uniform
// u1 = (k_a + 1/2) 2^-11 (2048 equally spaced angles offset by half a step: every average of
// cos^m sin^n of order below 2048 equals its continuous value, so each Gaussian's moments and
// the independence of a pair's two Gaussians are those of the continuous angle).  Pair p gives
// (g_2p, g_2p+1); mode k = 4..18 takes g_(k-4).  The stress modes 4..9 draw on words 0..2 of
// call 0 alone; the kinetic modes 10..18 on word 3 of call 0 and the four words of call 1
// (g_15 is not formed).
// ---------------------------------------------------------------------------------------
// the radius uniform of a word as the float 1 + k_r 2^-21 (k_r in the top 21 mantissa bits)
__device__ __forceinline__ float fluid_radius_1p(uint32_t w) {
  return __uint_as_float(0x3f800000u | ((w >> 9) & 0x7ffffcu));
}
// the angle uniform of a word as the float 1 + k_a 2^-11 (k_a in the top 11 mantissa bits)
__device__ __forceinline__ float fluid_angle_1p(uint32_t w) {
  return __uint_as_float(0x3f800000u | ((w << 12) & 0x7ff000u));
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

// Box-Muller pair of one word, times sqrt(rho) (Box & Muller 1958, angle in (-pi, pi)).
// Single precision: u0 and the angle come from the uniforms as floats 1 + k 2^-21 and
// 1 + k 2^-11, both exact steps; log2, 1/sqrt, sin and cos on the special-function unit.  Near
// u0 = 1 the hardware log2's absolute error (2^-22) would dominate -ln u0; there
// (t = 1 - u0 < 1e-3) log2(u0) is the series -(t + t^2/2 + t^3/3) / ln 2 (truncation below
// 3e-10 relative).  SECOND = false forms g0 only.
template <bool SECOND>
__device__ __forceinline__ void fluid_pair(uint32_t w, const NoiseScale<float>& ns, float& g0, float& g1) {
  const float u0 = fluid_radius_1p(w) - 0x1.fffff8p-1f;  // (k_r + 1/2) 2^-21
  const float t = 1.0f - u0;
  const float l2 = t < 1.0e-3f ? t * (-1.44269504f + t * (-0.721347520f + t * -0.480898347f)) : approx_lg2(u0);
  const float x = ns.cl * l2;  // rho (-2 ln u0): >= 1e-30 * 2^-22, a normal number
  const float r = x * approx_rsqrt(x);
  const float d = fluid_angle_1p(w) - 1.5f;                             // k_a 2^-11 - 1/2, exact
  const float th = fmaf(6.28318530717958647692f, d, 1.53398078788564123e-3f);  // 2 pi (u1 - 1/2), |th| >= pi/2048
  g0 = r * approx_cos(th);
  if (SECOND) g1 = r * approx_sin(th);
}
// Double precision.  The angle theta = pi j / 2048, j = 2 k_a + 1 - 2048 (odd, |j| < 2048),
// takes 2048 values; with `tab` (two tables of (cos, sin) filled by fill_angle_tables) its
// cosine and sine come from j = 64 a + b (a = j >> 6 in [-32, 31], b = j & 63) by the angle
// addition formulas, four operations instead of sincospi; without, from sincospi.
struct AngleTab {
  double2 a[64];  // (cos, sin)(pi a / 32), a = -32 .. 31 at index a + 32
  double2 b[64];  // (cos, sin)(pi b / 2048), b = 0 .. 63
};
// fill the tables with the block's threads 0..127 (the caller synchronises the block)
__device__ __forceinline__ void fill_angle_tables(AngleTab* t, unsigned tid) {
  double s, c;
  if (tid < 64) {
    sincospi((double)((int)tid - 32) / 32.0, &s, &c);
    t->a[tid] = make_double2(c, s);
  } else if (tid < 128) {
    sincospi((double)(tid - 64) / 2048.0, &s, &c);
    t->b[tid - 64] = make_double2(c, s);
  }
}
template <bool SECOND>
__device__ __forceinline__ void fluid_pair(uint32_t w, const NoiseScale<double>& ns, double& g0, double& g1,
                                           const AngleTab* tab = nullptr) {
  const double u0 = ((double)(w >> 11) + 0.5) * 0x1p-21;
  const double r = ns.sr * sqrt(-2.0 * log(u0));
  double s, c;
  if (tab) {
    const int j = 2 * (int)(w & 0x7ffu) + 1 - 2048;
    const double2 A = tab->a[(j >> 6) + 32], B = tab->b[j & 63];
    c = fma(A.x, B.x, -(A.y * B.y));
    s = fma(A.y, B.x, A.x * B.y);
  } else {
    const double u1 = ((double)(w & 0x7ffu) + 0.5) * 0x1p-11;
    sincospi(2.0 * u1 - 1.0, &s, &c);
  }
  g0 = r * c;
  if (SECOND) g1 = r * s;
}

template <int P, bool SECOND = true, class R, class Emit>
__device__ __forceinline__ void fluid_pair_emit(uint32_t w, const NoiseScale<R>& ns, Emit& emit, const AngleTab* tab) {
  R g0, g1;
  if constexpr (sizeof(R) == 8)
    fluid_pair<SECOND>(w, ns, g0, g1, tab);
  else
    fluid_pair<SECOND>(w, ns, g0, g1);
  emit(2 * P, g0);
  if (SECOND) emit(2 * P + 1, g1);
}

// The Gaussians of one node, times sqrt(rho), handed out as emit(j, g_j) for mode 4 + j:
// j = 0..5 (stress modes) always, j = 6..14 (kinetic modes) when `kinetic`.  tab: the angle
// tables of the double-precision pairs (null: sincospi; ignored in single precision).
template <class R, class Emit>
__device__ __forceinline__ void fluid_noise(uint32_t step, uint32_t node, const RoundKeys& rk, bool kinetic,
                                            const NoiseScale<R>& ns, Emit emit, const AngleTab* tab = nullptr) {
  U4 w = philox4x32_10_rk(U4{step, node, 0u, 0u}, rk);
  fluid_pair_emit<0>(w.x, ns, emit, tab);
  fluid_pair_emit<1>(w.y, ns, emit, tab);
  fluid_pair_emit<2>(w.z, ns, emit, tab);
  if (!kinetic) return;
  fluid_pair_emit<3>(w.w, ns, emit, tab);
  w = philox4x32_10_rk(U4{step, node, 1u, 0u}, rk);
  fluid_pair_emit<4>(w.x, ns, emit, tab);
  fluid_pair_emit<5>(w.y, ns, emit, tab);
  fluid_pair_emit<6>(w.z, ns, emit, tab);
  fluid_pair_emit<7, false>(w.w, ns, emit, tab);
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
